/*
 * bh_oracle.c -- plain, slow, FP64 CPU oracle of the sparse-octree
 * gravitational tree-code of Bedorf, Gaburov & Portegies Zwart
 * ("A sparse octree gravitational N-body code that runs entirely on the
 * GPU processor", arXiv:1106.1900).
 *
 * TEST INFRASTRUCTURE.  Only the tests, the smoke check and the benchmark's
 * CPU-baseline leg use this file.  It shares no code, header or table with
 * the CUDA library and never calls it.
 *
 * Every step follows the paper's own order and notation:
 *   frame + integer quantisation ........ App. B
 *   Morton key (bit interleave) ......... App. B, Listing 1
 *   radix sort (stable) ................. §2.1, App. A (split-based LSD sort)
 *   level-by-level cell construction .... §2.1, Fig. 1
 *   tree link ........................... §2.1, Fig. 2
 *   groups (cells with <= N_crit) ....... §2.2
 *   multipole moments (mono + quad) ..... §3.2, Fig. 4
 *   opening criterion d > l/theta + delta  §3.3, Eq. 1, Fig. 5
 *   breadth-first group walk ............ §2.2, Fig. 3
 *   direct summation .................... §4.2.1 (the reference the paper
 *                                          measures Eq. 2 against)
 * Where the paper is silent the readings are:
 *   - frame: origin = per-axis minimum; L = smallest power of two not
 *     below E*(1+2^-20), E the largest per-axis extent; L = 1 if E = 0.
 *   - quantisation: q = floor((x - origin) * 2^D/L), clamped to [0, 2^D-1],
 *     D the key depth in levels: 20 (the paper's 60-bit keys) or up to 30
 *     (the 90-bit keys App. B names as the way past 20 levels).
 *   - key: bit b of qx, qy, qz at bits 3b, 3b+1, 3b+2 (3D bits, D levels),
 *     stored as two words: hi = levels 1..20 (the top 60 bits), lo = levels
 *     21..D (the low 3(D-20) bits, 0 when D = 20); a forest orders by
 *     (system, key).
 *   - sort ties keep input order.
 *   - level 0 is the root; a cell with n <= N_leaf, or any cell at level
 *     D, is a leaf.
 *   - a group is a cell with n <= N_crit whose parent has n > N_crit (or a
 *     root with n <= N_crit); a leaf with n > N_crit is cut into
 *     consecutive chunks of N_crit bodies.
 *   - quadrupole Q_ab = sum m (3 r_a r_b - r^2 delta_ab) about the centre
 *     of mass; the softened particle-cell force and potential replace |r|
 *     by s = sqrt(r^2 + eps^2):
 *       a = -M r/s^3 + Q r/s^5 - (5/2)(r.Q.r) r/s^7,
 *       phi = -M/s - (1/2)(r.Q.r)/s^5.
 *   - particle-particle: Plummer softening, the body itself is skipped.
 *   - opening test: d = distance from the centre of mass to the group's
 *     tight bounding box (0 inside); the cell is accepted iff
 *     d^2 > (l/theta + delta)^2.
 * Built with -ffp-contract=off so that the FP64 frame and key arithmetic
 * rounds the same way on every host.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_LEVELS_MAX 30 /* deepest key: 90 bits */

typedef unsigned __int128 or_key_t; /* a whole 3D-bit key */

static int bad_levels(int D) { return D < 20 || D > OR_LEVELS_MAX; }

/* The whole key of body i from its two stored words. */
static or_key_t full_key(const uint64_t *hi, const uint64_t *lo, int D, int64_t i)
{
    return ((or_key_t)hi[i] << (3 * (D - 20))) | (or_key_t)lo[i];
}

/* ------------------------------------------------------------------ App. B */

/* Spread the low 10 bits of v so that bit b lands on bit 3b (App. B,
 * Listing 1 computes the same with shift-add-mask steps). */
uint32_t or_dilate10(uint32_t v)
{
    uint32_t out = 0;
    for (int b = 0; b < 10; ++b)
        out |= ((v >> b) & 1u) << (3 * b);
    return out;
}

/* Smallest power of two that is >= v (v > 0). */
static double pow2_at_least(double v)
{
    double L = 1.0;
    while (L < v) L *= 2.0;
    while (L * 0.5 >= v) L *= 0.5;
    return L;
}

/* Per-system frame: frame[4s+0..2] = origin (per-axis minimum), frame[4s+3] = L. */
int or_frames(int64_t n, const double *pos, int32_t nsys, const int64_t *offs, double *frame)
{
    (void)n;
    for (int32_t s = 0; s < nsys; ++s) {
        double lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
        int64_t b = offs[s], e = offs[s + 1];
        if (e > b) {
            for (int a = 0; a < 3; ++a) lo[a] = hi[a] = pos[3 * b + a];
            for (int64_t i = b; i < e; ++i)
                for (int a = 0; a < 3; ++a) {
                    double x = pos[3 * i + a];
                    if (x < lo[a]) lo[a] = x;
                    if (x > hi[a]) hi[a] = x;
                }
        }
        double E = 0.0;
        for (int a = 0; a < 3; ++a)
            if (hi[a] - lo[a] > E) E = hi[a] - lo[a];
        double L = (E > 0.0) ? pow2_at_least(E * (1.0 + 0x1p-20)) : 1.0;
        for (int a = 0; a < 3; ++a) frame[4 * s + a] = lo[a];
        frame[4 * s + 3] = L;
    }
    return 0;
}

/* Quantise every body in its system's frame (2^D cells per axis) and form
 * its 3D-bit Morton key by interleaving bit b of (qx, qy, qz) into bits
 * (3b, 3b+1, 3b+2); stored as key_hi (levels 1..20) and key_lo (21..D). */
int or_keys(int64_t n, const double *pos, int32_t nsys, const int64_t *offs, const double *frame, int32_t D,
            int32_t *q, uint64_t *key_hi, uint64_t *key_lo, int32_t *sys)
{
    (void)n;
    if (bad_levels(D)) return -1;
    const double qmax = ldexp(1.0, D);
    const int lo_bits = 3 * (D - 20);
    for (int32_t s = 0; s < nsys; ++s) {
        double scale = qmax / frame[4 * s + 3];
        for (int64_t i = offs[s]; i < offs[s + 1]; ++i) {
            int64_t qi[3];
            for (int a = 0; a < 3; ++a) {
                double t = floor((pos[3 * i + a] - frame[4 * s + a]) * scale);
                if (t < 0.0) t = 0.0;
                if (t > qmax - 1.0) t = qmax - 1.0;
                qi[a] = (int64_t)t;
                q[3 * i + a] = (int32_t)qi[a];
            }
            or_key_t k = 0;
            for (int b = 0; b < D; ++b)
                for (int a = 0; a < 3; ++a)
                    k |= (or_key_t)((qi[a] >> b) & 1) << (3 * b + a);
            key_hi[i] = (uint64_t)(k >> lo_bits);
            key_lo[i] = (uint64_t)(k & (((or_key_t)1 << lo_bits) - 1));
            sys[i] = s;
        }
    }
    return 0;
}

/* ------------------------------------------------------------ §2.1 sort */

static const uint64_t *g_key_hi, *g_key_lo;
static const int32_t *g_sys;
static int g_levels;

static int cmp_sys_key_index(const void *pa, const void *pb)
{
    int64_t a = *(const int64_t *)pa, b = *(const int64_t *)pb;
    if (g_sys[a] != g_sys[b]) return g_sys[a] < g_sys[b] ? -1 : 1;
    or_key_t ka = full_key(g_key_hi, g_key_lo, g_levels, a), kb = full_key(g_key_hi, g_key_lo, g_levels, b);
    if (ka != kb) return ka < kb ? -1 : 1;
    return (a < b) ? -1 : (a > b); /* stable: equal keys keep input order */
}

/* perm[i] = input index of the i-th body in (system, key) order. */
int or_sort(int64_t n, const uint64_t *key_hi, const uint64_t *key_lo, int32_t D, const int32_t *sys, int64_t *perm)
{
    if (bad_levels(D)) return -1;
    for (int64_t i = 0; i < n; ++i) perm[i] = i;
    g_key_hi = key_hi;
    g_key_lo = key_lo;
    g_levels = D;
    g_sys = sys;
    qsort(perm, (size_t)n, sizeof(int64_t), cmp_sys_key_index);
    return 0;
}

/* ------------------------------------------- §2.1, Fig. 1: level by level */

/* Mask keeping the top 3k bits of a 3D-bit key (footnote to §2.1). */
static or_key_t level_mask(int k, int D)
{
    if (k == 0) return 0;
    or_key_t all = ((or_key_t)1 << (3 * D)) - 1;
    return all & ~(((or_key_t)1 << (3 * (D - k))) - 1);
}

/* skey/ssys: keys (two words each) and systems in sorted order.  For every
 * level, the keys of the bodies not yet in a leaf are masked; consecutive
 * bodies with equal masked keys (and the same system) form one cell; cells
 * with at most N_leaf bodies (or at level D) become leaves and flag their
 * bodies.  The loop stops when every body is in a leaf.  Returns the cell
 * count, or -1 if more than cap cells would be made. */
int64_t or_build_levels(int64_t n, const uint64_t *skey_hi, const uint64_t *skey_lo, int32_t D,
                        const int32_t *ssys, int32_t n_leaf, int64_t cap, int32_t *level, int64_t *pbeg,
                        int64_t *pend, int32_t *is_leaf, int32_t *csys)
{
    if (bad_levels(D)) return -1;
    unsigned char *flag = (unsigned char *)calloc((size_t)(n > 0 ? n : 1), 1);
    int64_t C = 0;
    for (int k = 0; k <= D; ++k) {
        or_key_t mask = level_mask(k, D);
        int64_t made = 0;
        int64_t i = 0;
        while (i < n) {
            if (flag[i]) { ++i; continue; }
            or_key_t mk = full_key(skey_hi, skey_lo, D, i) & mask;
            int64_t j = i + 1;
            while (j < n && !flag[j] && ssys[j] == ssys[i] && (full_key(skey_hi, skey_lo, D, j) & mask) == mk) ++j;
            if (C >= cap) { free(flag); return -1; }
            int leaf = (j - i <= n_leaf) || (k == D);
            level[C] = k;
            pbeg[C] = i;
            pend[C] = j;
            is_leaf[C] = leaf;
            csys[C] = ssys[i];
            ++C;
            ++made;
            if (leaf)
                for (int64_t t = i; t < j; ++t) flag[t] = 1;
            i = j;
        }
        if (made == 0) break;
    }
    free(flag);
    return C;
}

/* §2.1, Fig. 2: every cell finds its parent by a binary search of its masked
 * key among the cells one level up (sorted by system and key), increments
 * the parent's child counter and offers itself as the first child. */
int or_link(int64_t C, const int32_t *level, const int64_t *pbeg, const int32_t *csys, const uint64_t *skey_hi,
            const uint64_t *skey_lo, int32_t D, int64_t *parent, int64_t *first_child, int32_t *n_children)
{
    if (bad_levels(D)) return -1;
    /* start of each level in the cell array */
    int64_t lstart[OR_LEVELS_MAX + 2];
    for (int k = 0; k <= D + 1; ++k) lstart[k] = C;
    for (int64_t c = C - 1; c >= 0; --c) lstart[level[c]] = c;
    for (int k = D; k >= 0; --k)
        if (lstart[k] > lstart[k + 1]) lstart[k] = lstart[k + 1];
    for (int64_t c = 0; c < C; ++c) {
        parent[c] = -1;
        first_child[c] = -1;
        n_children[c] = 0;
    }
    for (int64_t c = 0; c < C; ++c) {
        int k = level[c];
        if (k == 0) continue;
        or_key_t want = full_key(skey_hi, skey_lo, D, pbeg[c]) & level_mask(k - 1, D);
        int32_t s = csys[c];
        int64_t lo = lstart[k - 1], hi = lstart[k] - 1, found = -1;
        while (lo <= hi) {
            int64_t mid = lo + (hi - lo) / 2;
            or_key_t mk = full_key(skey_hi, skey_lo, D, pbeg[mid]) & level_mask(k - 1, D);
            int32_t ms = csys[mid];
            if (ms == s && mk == want) { found = mid; break; }
            if (ms < s || (ms == s && mk < want)) lo = mid + 1;
            else hi = mid - 1;
        }
        if (found < 0) return -1;
        parent[c] = found;
        n_children[found] += 1;
        if (first_child[found] < 0 || c < first_child[found]) first_child[found] = c;
    }
    return 0;
}

/* ------------------------------------------------------------ §2.2 groups */

/* Groups in body order: descend from every root; a cell with n <= N_crit is
 * one group; a leaf with more bodies is cut into chunks of N_crit.
 * Returns the group count, or -1 if more than cap groups would be made. */
int64_t or_groups(int64_t C, const int32_t *level, const int64_t *pbeg, const int64_t *pend,
                  const int32_t *is_leaf, const int64_t *first_child, const int32_t *n_children, int32_t n_crit,
                  int64_t cap, int64_t *gbeg, int64_t *gend)
{
    int64_t G = 0;
    int64_t *stack = (int64_t *)malloc(sizeof(int64_t) * (size_t)(C > 0 ? C : 1));
    for (int64_t r = 0; r < C && level[r] == 0; ++r) {
        int64_t sp = 0;
        stack[sp++] = r;
        while (sp > 0) {
            int64_t c = stack[--sp];
            int64_t n = pend[c] - pbeg[c];
            if (n <= n_crit || is_leaf[c]) {
                for (int64_t b = pbeg[c]; b < pend[c]; b += n_crit) {
                    if (G >= cap) { free(stack); return -1; }
                    gbeg[G] = b;
                    gend[G] = (b + n_crit < pend[c]) ? b + n_crit : pend[c];
                    ++G;
                }
            } else {
                /* push children in reverse so that the first child is visited first */
                for (int32_t j = n_children[c] - 1; j >= 0; --j) stack[sp++] = first_child[c] + j;
            }
        }
    }
    free(stack);
    return G;
}

/* ----------------------------------------------------- §3.2 moments, geometry */

/* For every cell, directly from its own bodies (sorted order spos/smass):
 * mass M, centre of mass com, traceless quadrupole Q (xx,yy,zz,xy,xz,yz)
 * about com; side l = L/2^k; geometric centre ctr = origin + (i + 1/2) l with
 * i the cell's integer corner (top k bits of the body's quantised
 * coordinate); delta = |com - ctr|. */
int or_moments(int64_t C, const int32_t *level, const int64_t *pbeg, const int64_t *pend, const int32_t *csys,
               const double *spos, const double *smass, const int32_t *sq, const double *frame, int32_t D,
               double *M, double *com, double *Q, double *ctr, double *size, double *delta)
{
    if (bad_levels(D)) return -1;
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t c = 0; c < C; ++c) {
        int k = level[c];
        int32_t s = csys[c];
        double l = frame[4 * s + 3] / (double)(1u << k);
        double g[3];
        for (int a = 0; a < 3; ++a) {
            int64_t corner = (int64_t)sq[3 * pbeg[c] + a] >> (D - k);
            g[a] = frame[4 * s + a] + ((double)corner + 0.5) * l;
        }
        double m = 0.0, cm[3] = {0, 0, 0};
        for (int64_t i = pbeg[c]; i < pend[c]; ++i) {
            m += smass[i];
            for (int a = 0; a < 3; ++a) cm[a] += smass[i] * spos[3 * i + a];
        }
        if (m > 0.0)
            for (int a = 0; a < 3; ++a) cm[a] /= m;
        else
            for (int a = 0; a < 3; ++a) cm[a] = g[a];
        double q[6] = {0, 0, 0, 0, 0, 0};
        for (int64_t i = pbeg[c]; i < pend[c]; ++i) {
            double r[3];
            for (int a = 0; a < 3; ++a) r[a] = spos[3 * i + a] - cm[a];
            double r2 = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
            double w = smass[i];
            q[0] += w * (3.0 * r[0] * r[0] - r2);
            q[1] += w * (3.0 * r[1] * r[1] - r2);
            q[2] += w * (3.0 * r[2] * r[2] - r2);
            q[3] += w * 3.0 * r[0] * r[1];
            q[4] += w * 3.0 * r[0] * r[2];
            q[5] += w * 3.0 * r[1] * r[2];
        }
        M[c] = m;
        double d2 = 0.0;
        for (int a = 0; a < 3; ++a) {
            com[3 * c + a] = cm[a];
            ctr[3 * c + a] = g[a];
            d2 += (cm[a] - g[a]) * (cm[a] - g[a]);
        }
        for (int j = 0; j < 6; ++j) Q[6 * c + j] = q[j];
        size[c] = l;
        delta[c] = sqrt(d2);
    }
    return 0;
}

/* ---------------------------------------------------------- forces (§3) */

static double norm3(const double *v) { return sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]); }

/* Softened particle-cell interaction (monopole + quadrupole), target at x. */
static void pc_force(const double *x, double M, const double *cm, const double *Q, double eps2, double *acc,
                     double *pot)
{
    double r[3] = {x[0] - cm[0], x[1] - cm[1], x[2] - cm[2]};
    double s2 = r[0] * r[0] + r[1] * r[1] + r[2] * r[2] + eps2;
    double s = sqrt(s2);
    double s3 = s2 * s, s5 = s3 * s2, s7 = s5 * s2;
    double Qr[3] = {Q[0] * r[0] + Q[3] * r[1] + Q[4] * r[2],
                    Q[3] * r[0] + Q[1] * r[1] + Q[5] * r[2],
                    Q[4] * r[0] + Q[5] * r[1] + Q[2] * r[2]};
    double rQr = r[0] * Qr[0] + r[1] * Qr[1] + r[2] * Qr[2];
    for (int a = 0; a < 3; ++a) acc[a] += -M * r[a] / s3 + Qr[a] / s5 - 2.5 * rQr * r[a] / s7;
    *pot += -M / s - 0.5 * rQr / s5;
}

/* Softened particle-particle interaction of source (xs, m) on target x. */
static void pp_force(const double *x, const double *xs, double m, double eps2, double *acc, double *pot)
{
    double r[3] = {xs[0] - x[0], xs[1] - x[1], xs[2] - x[2]};
    double s2 = r[0] * r[0] + r[1] * r[1] + r[2] * r[2] + eps2;
    double s = sqrt(s2);
    for (int a = 0; a < 3; ++a) acc[a] += m * r[a] / (s2 * s);
    *pot += -m / s;
}

/* §2.2 + §3.3: breadth-first walk of every listed group.  The group's tight
 * bounding box is tested against each cell in the current level with Eq. 1
 * (mac = 0: d > l/theta + delta, d from the cell's centre of mass to the box)
 * or with the minimal-distance criterion the paper also implemented (§2.3,
 * Salmon & Warren 1994; mac = 1: d > l/theta, d between the box and the
 * cell's geometric cube, centre ctr, side l); accepted cells go to the cell list, opened nodes put their children on the
 * next level, opened leaves put their bodies on the particle list.  Every
 * body of the group then sums the cell list and the particle list (skipping
 * itself).  Bodies and outputs are in sorted order.
 *   groups[]:    indices of the groups to walk (ng of them)
 *   sys_root[s]: root cell of system s
 *   stats[5*j]:  cell-list length, particle-list length, sum of listed cell
 *                indices, sum of listed body indices, and (as a double bit
 *                pattern) the smallest relative margin |d - r_open|/r_open
 *                of any opening decision of group groups[j].
 *   amag[i]:     sum over the body's interactions of |a_ij| (how much the
 *                terms of the sum cancel: |a_i| / amag[i] near 0 means the
 *                result is small against its terms). */
int or_walk(int64_t ng, const int64_t *groups, const int64_t *gbeg, const int64_t *gend, const int32_t *gsys,
            const int64_t *sys_root, int64_t C, const int32_t *is_leaf, const int64_t *pbeg, const int64_t *pend,
            const int64_t *first_child, const int32_t *n_children, const double *M, const double *com,
            const double *Q, const double *ctr, const double *size, const double *delta, int64_t n,
            const double *spos, const double *smass, double theta, double eps, int mac, double *acc, double *pot,
            int64_t *stats, double *amag)
{
    double eps2 = eps * eps;
#pragma omp parallel
    {
        int64_t *cur = (int64_t *)malloc(sizeof(int64_t) * (size_t)(C + 1));
        int64_t *nxt = (int64_t *)malloc(sizeof(int64_t) * (size_t)(C + 1));
        int64_t *clist = (int64_t *)malloc(sizeof(int64_t) * (size_t)(C + 1));
        int64_t *plist = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n + 1));
#pragma omp for schedule(dynamic, 1)
        for (int64_t j = 0; j < ng; ++j) {
            int64_t g = groups[j];
            double bmin[3], bmax[3];
            for (int a = 0; a < 3; ++a) bmin[a] = bmax[a] = spos[3 * gbeg[g] + a];
            for (int64_t i = gbeg[g]; i < gend[g]; ++i)
                for (int a = 0; a < 3; ++a) {
                    double x = spos[3 * i + a];
                    if (x < bmin[a]) bmin[a] = x;
                    if (x > bmax[a]) bmax[a] = x;
                }
            int64_t ncur = 0, nc = 0, np = 0;
            uint64_t csum = 0, psum = 0;
            double min_margin = INFINITY;
            cur[ncur++] = sys_root[gsys[g]];
            while (ncur > 0) {
                int64_t nnext = 0;
                for (int64_t t = 0; t < ncur; ++t) {
                    int64_t c = cur[t];
                    double d2 = 0.0;
                    for (int a = 0; a < 3; ++a) {
                        double e = 0.0;
                        if (mac == 0) {  /* centre of mass to the group's box */
                            double x = com[3 * c + a];
                            if (x < bmin[a]) e = bmin[a] - x;
                            else if (x > bmax[a]) e = x - bmax[a];
                        } else {         /* the cell's cube to the group's box */
                            double lo = ctr[3 * c + a] - 0.5 * size[c], hi = ctr[3 * c + a] + 0.5 * size[c];
                            if (hi < bmin[a]) e = bmin[a] - hi;
                            else if (lo > bmax[a]) e = lo - bmax[a];
                        }
                        d2 += e * e;
                    }
                    double r_open = (mac == 0) ? size[c] / theta + delta[c] : size[c] / theta;
                    double margin = fabs(sqrt(d2) - r_open) / r_open;
                    if (margin < min_margin) min_margin = margin;
                    if (d2 > r_open * r_open) {
                        clist[nc++] = c;
                        csum += (uint64_t)c;
                    } else if (is_leaf[c]) {
                        for (int64_t i = pbeg[c]; i < pend[c]; ++i) {
                            plist[np++] = i;
                            psum += (uint64_t)i;
                        }
                    } else {
                        for (int32_t h = 0; h < n_children[c]; ++h) nxt[nnext++] = first_child[c] + h;
                    }
                }
                int64_t *tmp = cur;
                cur = nxt;
                nxt = tmp;
                ncur = nnext;
            }
            for (int64_t i = gbeg[g]; i < gend[g]; ++i) {
                double a[3] = {0, 0, 0}, p = 0.0, mag = 0.0;
                const double *x = spos + 3 * i;
                for (int64_t t = 0; t < nc; ++t) {
                    int64_t c = clist[t];
                    double ai[3] = {0, 0, 0}, pi = 0.0;
                    pc_force(x, M[c], com + 3 * c, Q + 6 * c, eps2, ai, &pi);
                    for (int b = 0; b < 3; ++b) a[b] += ai[b];
                    p += pi;
                    mag += norm3(ai);
                }
                for (int64_t t = 0; t < np; ++t) {
                    int64_t s = plist[t];
                    if (s == i) continue;
                    double ai[3] = {0, 0, 0}, pi = 0.0;
                    pp_force(x, spos + 3 * s, smass[s], eps2, ai, &pi);
                    for (int b = 0; b < 3; ++b) a[b] += ai[b];
                    p += pi;
                    mag += norm3(ai);
                }
                for (int b = 0; b < 3; ++b) acc[3 * i + b] = a[b];
                pot[i] = p;
                amag[i] = mag;
            }
            stats[5 * j + 0] = nc;
            stats[5 * j + 1] = np;
            stats[5 * j + 2] = (int64_t)csum;
            stats[5 * j + 3] = (int64_t)psum;
            memcpy(&stats[5 * j + 4], &min_margin, sizeof(double));
        }
        free(cur);
        free(nxt);
        free(clist);
        free(plist);
    }
    return 0;
}

/* Direct summation: acceleration and potential on the listed targets from
 * every other body of the same system (pairs j != i), FP64. */
int or_direct(int64_t n, const double *pos, const double *mass, int32_t nsys, const int64_t *offs, int64_t nt,
              const int64_t *targets, double eps, double *acc, double *pot)
{
    (void)n;
    double eps2 = eps * eps;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t t = 0; t < nt; ++t) {
        int64_t i = targets[t];
        int32_t s = 0;
        while (s + 1 < nsys && offs[s + 1] <= i) ++s;
        double a[3] = {0, 0, 0}, p = 0.0;
        for (int64_t j = offs[s]; j < offs[s + 1]; ++j) {
            if (j == i) continue;
            pp_force(pos + 3 * i, pos + 3 * j, mass[j], eps2, a, &p);
        }
        for (int b = 0; b < 3; ++b) acc[3 * t + b] = a[b];
        pot[t] = p;
    }
    return 0;
}

/* Exact gravity of one cell's own bodies on a target (for moment pins). */
int or_cell_exact(int64_t c_beg, int64_t c_end, const double *spos, const double *smass, const double *x,
                  double eps, double *acc, double *pot)
{
    double a[3] = {0, 0, 0}, p = 0.0;
    for (int64_t j = c_beg; j < c_end; ++j) pp_force(x, spos + 3 * j, smass[j], eps * eps, a, &p);
    for (int b = 0; b < 3; ++b) acc[b] = a[b];
    *pot = p;
    return 0;
}

/* The multipole approximation of one cell on a target (for moment pins). */
int or_cell_multipole(double Mc, const double *cm, const double *Qc, const double *x, double eps, double *acc,
                      double *pot)
{
    double a[3] = {0, 0, 0}, p = 0.0;
    pc_force(x, Mc, cm, Qc, eps * eps, a, &p);
    for (int b = 0; b < 3; ++b) acc[b] = a[b];
    *pot = p;
    return 0;
}

/* ------------------------------------------- block time-steps: tree refresh */

/* Cell sizes after a moment refresh on an unchanged tree (§4: between
 * rebuilds only the moments of cells whose bodies moved are recomputed; the
 * tree-cell size grows as bodies drift, which opens more cells).  Reading: a
 * cell keeps its geometric centre ctr; its size becomes the side of the
 * smallest cube about ctr that holds its bodies (a leaf) or its children's
 * cubes (a node), never below the size it was built with.  size[] holds the
 * built sizes on entry.  Children have larger indices than their parents
 * ((level, key) order), so one pass from the last cell down suffices. */
int or_refresh_sizes(int64_t C, const int32_t *is_leaf, const int64_t *pbeg, const int64_t *pend,
                     const int64_t *first_child, const int32_t *n_children, const double *spos,
                     const double *ctr, double *size)
{
    for (int64_t c = C - 1; c >= 0; --c) {
        double l = size[c];
        if (is_leaf[c]) {
            for (int64_t i = pbeg[c]; i < pend[c]; ++i)
                for (int a = 0; a < 3; ++a) {
                    double e = 2.0 * fabs(spos[3 * i + a] - ctr[3 * c + a]);
                    if (e > l) l = e;
                }
        } else {
            for (int32_t h = 0; h < n_children[c]; ++h) {
                double e = 0.5 * size[c] + size[first_child[c] + h];
                if (e > l) l = e;
            }
        }
        size[c] = l;
    }
    return 0;
}
