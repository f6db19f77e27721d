"""GB300 (sm_103a) sparse-octree gravitational tree-code: Python binding.

A thin ctypes binding of the C ABI declared in ``include/bh.h``.  Every step
of the computation runs in the library's CUDA kernels (``csrc/``); this module
only builds the library in-tree, marshals pointers and sizes, and owns the
device workspace as a torch tensor.  There is no CPU path: without the built
library or a CUDA device every call raises.

Functions keep the C names (``bh_build``, ``bh_compute_forces``, ...);
:class:`TreeCode` wraps one context plus its workspace.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from concurrent.futures import ThreadPoolExecutor

_HERE = os.path.dirname(os.path.abspath(__file__))
_ROOT = os.path.dirname(_HERE)
_CSRC = os.path.join(_HERE, "csrc")
_INCLUDE = os.path.join(_ROOT, "include")
_BUILD = os.path.join(_HERE, "_build")
LIB_PATH = os.path.join(_HERE, "libbh.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "--ftz=true", "-Xcompiler", "-fPIC", "-I" + _INCLUDE]

BH_OK = 0
STATUS_CAPACITY = 2
BH_NPHASES = 9
PHASES = ("frame+keys", "sort", "move", "cells+link+groups", "moments", "walk", "leapfrog", "call",
          "walk eval")
STATUS = {
    0: "ok", 1: "invalid argument", 2: "capacity exceeded", 3: "non-finite input",
    4: "bounded device wait gave up", 5: "CUDA runtime error", 6: "call order violated",
    7: "no or too small workspace bound",
}

_lock = threading.Lock()
_lib = None


class BHError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"{what}: {STATUS.get(code, 'unknown')} ({code})")
        self.code = code


def _sources():
    return sorted(f for f in os.listdir(_CSRC) if f.endswith(".cu"))


def _stale() -> bool:
    if not os.path.exists(LIB_PATH):
        return True
    t = os.path.getmtime(LIB_PATH)
    deps = [os.path.join(_CSRC, f) for f in os.listdir(_CSRC)] + [os.path.join(_INCLUDE, "bh.h")]
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile every ``csrc/*.cu`` for sm_103a (in parallel) and link ``libbh.so``."""
    if not force and not _stale():
        return LIB_PATH
    os.makedirs(_BUILD, exist_ok=True)
    srcs = _sources()

    def compile_one(f):
        obj = os.path.join(_BUILD, f[:-3] + ".o")
        cmd = ["nvcc", *ARCH, *NVCC_FLAGS, "-c", os.path.join(_CSRC, f), "-o", obj]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {f}:\n{r.stderr}")
        return obj, r.stderr

    with ThreadPoolExecutor(max_workers=min(8, len(srcs))) as ex:
        results = list(ex.map(compile_one, srcs))
    if verbose:
        for _, err in results:
            print(err)
    tmp = LIB_PATH + ".tmp"
    cmd = ["nvcc", *ARCH, "-shared", "-cudart", "static", "-o", tmp] + [o for o, _ in results]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, LIB_PATH)
    return LIB_PATH


class bh_params(ctypes.Structure):
    _fields_ = [
        ("n_leaf", ctypes.c_int32),
        ("n_crit", ctypes.c_int32),
        ("stack_capacity", ctypes.c_int32),
        ("walk_variant", ctypes.c_int32),
        ("walk_warps", ctypes.c_int32),
        ("walk_blocks_per_sm", ctypes.c_int32),
        ("list_capacity", ctypes.c_int32),
        ("pool_per_body", ctypes.c_int32),
        ("walk_split", ctypes.c_int32),
        ("mac", ctypes.c_int32),
        ("key_levels", ctypes.c_int32),
        ("list_buffer", ctypes.c_int32),
    ]


_SIG = {
    "bh_default_params": [ctypes.POINTER(bh_params)],
    "bh_workspace_bytes": [ctypes.POINTER(bh_params), ctypes.c_int64, ctypes.c_int32, ctypes.c_int,
                           ctypes.POINTER(ctypes.c_size_t)],
    "bh_create": [ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(bh_params), ctypes.c_int64, ctypes.c_int32,
                  ctypes.c_int],
    "bh_bind_workspace": [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t],
    "bh_build": [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p],
    "bh_build_forest": [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                        ctypes.c_int32, ctypes.c_void_p],
    "bh_compute_forces": [ctypes.c_void_p, ctypes.c_float, ctypes.c_float, ctypes.c_void_p, ctypes.c_void_p,
                          ctypes.c_void_p],
    "bh_forces_host": [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_float,
                       ctypes.c_float, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p],
    "bh_set_state": [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                     ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p],
    "bh_get_state": [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                     ctypes.c_void_p],
    "bh_step": [ctypes.c_void_p, ctypes.c_double, ctypes.c_float, ctypes.c_float, ctypes.c_void_p],
    "bh_step_graph": [ctypes.c_void_p, ctypes.c_double, ctypes.c_float, ctypes.c_float, ctypes.c_void_p],
    "bh_step_begin": [ctypes.c_void_p, ctypes.c_double, ctypes.c_int32, ctypes.c_void_p],
    "bh_walk_groups": [ctypes.c_void_p, ctypes.c_float, ctypes.c_float, ctypes.c_int32, ctypes.c_int32,
                       ctypes.c_void_p],
    "bh_sorted_forces": [ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)],
    "bh_step_end": [ctypes.c_void_p, ctypes.c_double, ctypes.c_int32, ctypes.c_void_p],
    "bh_diagnostics": [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p],
    "bh_block_start": [ctypes.c_void_p, ctypes.c_double, ctypes.c_int32, ctypes.c_double, ctypes.c_float,
                       ctypes.c_float, ctypes.c_void_p],
    "bh_block_step": [ctypes.c_void_p, ctypes.c_float, ctypes.c_float, ctypes.c_int32, ctypes.c_void_p],
    "bh_block_info": [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p],
    "bh_block_levels": [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p],
    "bh_status": [ctypes.c_void_p, ctypes.c_void_p],
    "bh_get_counts": [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p],
    "bh_reset_counters": [ctypes.c_void_p, ctypes.c_void_p],
    "bh_get_tree": [ctypes.c_void_p] + [ctypes.c_void_p] * 11 + [ctypes.c_void_p],
    "bh_get_keys_lo": [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p],
    "bh_wait_probe": [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p],
    "bh_get_moments": [ctypes.c_void_p] + [ctypes.c_void_p] * 5 + [ctypes.c_void_p],
    "bh_get_group_stats": [ctypes.c_void_p] + [ctypes.c_void_p] * 4 + [ctypes.c_void_p],
    "bh_set_profiling": [ctypes.c_void_p, ctypes.c_int],
    "bh_phase_times": [ctypes.c_void_p, ctypes.c_void_p],
    "bh_walk_time": [ctypes.c_void_p, ctypes.c_void_p],
    "bh_prim_exclusive_scan": [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                               ctypes.c_void_p, ctypes.c_void_p],
    "bh_fp32_peak_probe": [ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p],
    "bh_exclusive_scan_noalloc": [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                                  ctypes.c_void_p],
    "bh_prim_split2": [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p,
                       ctypes.c_void_p, ctypes.c_void_p],
    "bh_direct_forces": [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64,
                         ctypes.c_float, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p],
}

NOALLOC_SCAN_MAX_N = 1 << 26


def exported_symbols() -> list[str]:
    """Every entry point the binding expects the library to export (include/bh.h)."""
    return sorted(list(_SIG) + ["bh_destroy", "bh_status_string"])


def load(build_if_missing: bool = True):
    """Load ``libbh.so`` (building it first if needed); raises if it cannot be loaded."""
    global _lib
    with _lock:
        if _lib is None:
            if build_if_missing:
                build()
            if not os.path.exists(LIB_PATH):
                raise RuntimeError("libbh.so is not built; run paper_1106_1900_gb300.build()")
            lib = ctypes.CDLL(LIB_PATH)
            for name, args in _SIG.items():
                f = getattr(lib, name)
                f.argtypes = args
                f.restype = ctypes.c_int
            lib.bh_destroy.argtypes = [ctypes.c_void_p]
            lib.bh_destroy.restype = None
            lib.bh_status_string.argtypes = [ctypes.c_int]
            lib.bh_status_string.restype = ctypes.c_char_p
            _lib = lib
    return _lib


def _check(rc: int, what: str):
    if rc != BH_OK:
        raise BHError(rc, what)


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _arg(t, dtype, what: str, cols: int = 0, cuda: bool = True, optional: bool = False):
    """Pointer of a contiguous tensor of the given dtype (and row length) on
    the GPU (or the host); raises before the library sees a wrong buffer."""
    import torch

    if t is None:
        if optional:
            return None
        raise ValueError(f"{what}: a tensor is required")
    if not isinstance(t, torch.Tensor) or t.dtype != dtype or not t.is_contiguous():
        raise ValueError(f"{what}: a contiguous {dtype} tensor is required")
    if t.is_cuda != cuda:
        raise ValueError(f"{what}: the tensor must be on the {'GPU' if cuda else 'host'}")
    if cols and (t.dim() != 2 or t.shape[1] != cols):
        raise ValueError(f"{what}: shape [n, {cols}] is required")
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    import torch

    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def default_params(**over) -> bh_params:
    p = bh_params()
    _check(load().bh_default_params(ctypes.byref(p)), "bh_default_params")
    names = {f[0] for f in bh_params._fields_}
    for k, v in over.items():
        if k not in names:
            raise ValueError(f"unknown parameter {k!r} (bh_params has {sorted(names)})")
        setattr(p, k, int(v))
    return p


def workspace_bytes(params: bh_params, n_max: int, n_sys_max: int = 1, device: int = 0) -> int:
    """Device workspace bytes of a context (``bh_workspace_bytes``)."""
    nbytes = ctypes.c_size_t(0)
    _check(load().bh_workspace_bytes(ctypes.byref(params), n_max, n_sys_max, device, ctypes.byref(nbytes)),
           "bh_workspace_bytes")
    return nbytes.value


def fp32_peak(device: int = 0, iters: int = 4096, stream=None) -> float:
    """Measured FP32 FMA throughput (FLOP/s) of the device."""
    out = ctypes.c_double(0)
    _check(load().bh_fp32_peak_probe(device, iters, ctypes.byref(out), _stream(stream)), "bh_fp32_peak_probe")
    return out.value


def direct_forces(pos, mass, targets, eps: float, stream=None):
    """Direct-summation accelerations and potentials on ``targets`` (int32
    CUDA tensor of body indices) from every other body: ``bh_direct_forces``."""
    import torch

    nt = targets.numel()
    acc = torch.empty((nt, 3), dtype=torch.float32, device=pos.device)
    pot = torch.empty(nt, dtype=torch.float32, device=pos.device)
    _check(load().bh_direct_forces(_ptr(pos), _ptr(mass), pos.shape[0], _ptr(targets), nt, float(eps), _ptr(acc),
                                   _ptr(pot), _stream(stream)), "bh_direct_forces")
    return acc, pot


def split2(x, f, stream=None):
    """The step kernels' conversions element by element through
    ``bh_prim_split2``: (hi, lo) floats of the FP64 tensor ``x`` (hi = x
    rounded, lo = the rest rounded) and the FP64 widening of the float32
    tensor ``f`` (same length, both contiguous CUDA tensors)."""
    import torch

    px = _arg(x, torch.float64, "x")
    pf = _arg(f, torch.float32, "f")
    if x.numel() != f.numel():
        raise ValueError("x and f must have the same length")
    hi = torch.empty(x.numel(), dtype=torch.float32, device=x.device)
    lo = torch.empty_like(hi)
    wide = torch.empty(x.numel(), dtype=torch.float64, device=x.device)
    _check(load().bh_prim_split2(px, pf, x.numel(), _ptr(hi), _ptr(lo), _ptr(wide), _stream(stream)),
           "bh_prim_split2")
    return hi, lo, wide


def exclusive_scan_noalloc(x, out=None, total=None, stream=None):
    """Exclusive prefix sum of a contiguous int32 CUDA tensor through
    ``bh_exclusive_scan_noalloc`` (no context, no workspace; the library
    allocates nothing).  The values are read as uint32 and the prefix sums
    wrap modulo 2^32.  ``total``, if given, is a contiguous 1-element int64
    CUDA tensor on the same device that receives the exact sum (as uint64
    bits).  The call runs with ``x``'s device current, on ``stream`` (that
    device's current stream by default)."""
    import torch

    _arg(x, torch.int32, "x")
    if out is None:
        out = torch.empty_like(x)
    _arg(out, torch.int32, "out")
    _arg(total, torch.int64, "total", optional=True)
    if out.numel() != x.numel():
        raise ValueError("out: as many elements as x are required")
    if total is not None and total.numel() != 1:
        raise ValueError("total: one element is required")
    for t in (out, total):
        if t is not None and t.device != x.device:
            raise ValueError("out and total must be on x's device")
    with torch.cuda.device(x.device):
        _check(load().bh_exclusive_scan_noalloc(_ptr(x), _ptr(out), x.numel(), _ptr(total), _stream(stream)),
               "bh_exclusive_scan_noalloc")
    return out


class TreeCode:
    """One library context plus its device workspace (a torch uint8 tensor)."""

    def __init__(self, n_max: int, n_sys_max: int = 1, device: int = 0, **params):
        import torch

        self.lib = load()
        self.device = device
        self.params = default_params(**params)
        nbytes = ctypes.c_size_t(0)
        _check(self.lib.bh_workspace_bytes(ctypes.byref(self.params), n_max, n_sys_max, device,
                                           ctypes.byref(nbytes)), "bh_workspace_bytes")
        self.ctx = ctypes.c_void_p()
        _check(self.lib.bh_create(ctypes.byref(self.ctx), ctypes.byref(self.params), n_max, n_sys_max, device),
               "bh_create")
        self.workspace = torch.empty(nbytes.value, dtype=torch.uint8, device=f"cuda:{device}")
        _check(self.lib.bh_bind_workspace(self.ctx, _ptr(self.workspace), nbytes.value), "bh_bind_workspace")
        self.n_max, self.n_sys_max = n_max, n_sys_max

    def close(self):
        if getattr(self, "ctx", None):
            self.lib.bh_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- force evaluation on device tensors (float64 pos [n,3], mass [n])
    def build(self, pos, mass, offsets=None, stream=None):
        import torch

        n = pos.shape[0]
        pp = _arg(pos, torch.float64, "pos", cols=3)
        mp = _arg(mass, torch.float64, "mass")
        if offsets is None or len(offsets) <= 2:
            _check(self.lib.bh_build(self.ctx, pp, mp, n, _stream(stream)), "bh_build")
        else:
            import numpy as np

            off = np.ascontiguousarray(offsets, dtype=np.int64)
            _check(self.lib.bh_build_forest(self.ctx, pp, mp, n, off.ctypes.data_as(ctypes.c_void_p), len(off) - 1,
                                            _stream(stream)), "bh_build_forest")

    def compute_forces(self, theta: float, eps: float, acc=None, pot=None, stream=None):
        import torch

        n = self.counts()["n"] if acc is None else acc.shape[0]
        if acc is None:
            acc = torch.empty((n, 3), dtype=torch.float32, device=f"cuda:{self.device}")
            pot = torch.empty(n, dtype=torch.float32, device=f"cuda:{self.device}")
        _check(self.lib.bh_compute_forces(self.ctx, float(theta), float(eps), _arg(acc, torch.float32, "acc", cols=3),
                                          _arg(pot, torch.float32, "pot"), _stream(stream)),
               "bh_compute_forces")
        return acc, pot

    def forces_host(self, pos, mass, theta: float, eps: float, acc, pot, stream=None):
        """pos/mass/acc/pot are (pinned) CPU tensors."""
        import torch

        args = (_arg(pos, torch.float64, "pos", cols=3, cuda=False), _arg(mass, torch.float64, "mass", cuda=False))
        outs = (_arg(acc, torch.float32, "acc", cols=3, cuda=False), _arg(pot, torch.float32, "pot", cuda=False))
        _check(self.lib.bh_forces_host(self.ctx, *args, pos.shape[0], float(theta), float(eps), *outs,
                                       _stream(stream)), "bh_forces_host")

    # ---- integration
    def set_state(self, pos, vel, mass, offsets=None, stream=None):
        import numpy as np
        import torch

        n = pos.shape[0]
        _arg(pos, torch.float64, "pos", cols=3)
        _arg(vel, torch.float64, "vel", cols=3)
        _arg(mass, torch.float64, "mass")
        if offsets is not None and len(offsets) > 2:
            off = np.ascontiguousarray(offsets, dtype=np.int64)
            optr, ns = off.ctypes.data_as(ctypes.c_void_p), len(off) - 1
        else:
            optr, ns = None, 1
        _check(self.lib.bh_set_state(self.ctx, _ptr(pos), _ptr(vel), _ptr(mass), n, optr, ns, _stream(stream)),
               "bh_set_state")
        self.n_state = n

    def get_state(self, pos=None, vel=None, acc=None, pot=None, stream=None):
        _check(self.lib.bh_get_state(self.ctx, _ptr(pos), _ptr(vel), _ptr(acc), _ptr(pot), _stream(stream)),
               "bh_get_state")

    def step(self, dt: float, theta: float, eps: float, graph: bool = False, stream=None):
        f = self.lib.bh_step_graph if graph else self.lib.bh_step
        _check(f(self.ctx, float(dt), float(theta), float(eps), _stream(stream)), "bh_step")

    # ---- the step in parts (groups shared out among ranks: see shard.py)
    def step_begin(self, dt: float, init: bool = False, stream=None):
        _check(self.lib.bh_step_begin(self.ctx, float(dt), int(init), _stream(stream)), "bh_step_begin")

    def walk_groups(self, theta: float, eps: float, g_begin: int, g_end: int, stream=None):
        _check(self.lib.bh_walk_groups(self.ctx, float(theta), float(eps), int(g_begin), int(g_end),
                                       _stream(stream)), "bh_walk_groups")

    def step_end(self, dt: float, init: bool = False, stream=None):
        _check(self.lib.bh_step_end(self.ctx, float(dt), int(init), _stream(stream)), "bh_step_end")

    def sorted_forces(self):
        """The context's sorted force array as a float32 [n, 4] CUDA tensor
        (a view of the workspace: a.x, a.y, a.z, phi per sorted body)."""
        import torch

        ptr = ctypes.c_void_p()
        _check(self.lib.bh_sorted_forces(self.ctx, ctypes.byref(ptr)), "bh_sorted_forces")
        n = self.counts()["n"]
        off = ptr.value - self.workspace.data_ptr()
        if off < 0 or off % 16 or off + 16 * n > self.workspace.numel():
            raise RuntimeError("bh_sorted_forces: address outside the bound workspace")
        return self.workspace[off:off + 16 * n].view(torch.float32).view(n, 4)

    def group_begins(self, stream=None):
        """Sorted first body of each group of the last build, then the end: int64 [G + 1]."""
        import numpy as np

        G = self.counts(stream)["groups"]
        if G == 0:
            return np.zeros(1, np.int64)
        gb = np.zeros(G, np.int32)
        ge = np.zeros(G, np.int32)
        nul = [None] * 9
        _check(self.lib.bh_get_tree(self.ctx, *nul, gb.ctypes.data_as(ctypes.c_void_p),
                                    ge.ctypes.data_as(ctypes.c_void_p), _stream(stream)), "bh_get_tree")
        return np.concatenate([gb.astype(np.int64), ge[-1:].astype(np.int64)])

    def diagnostics(self, stream=None):
        out = (ctypes.c_double * 5)()
        _check(self.lib.bh_diagnostics(self.ctx, out, _stream(stream)), "bh_diagnostics")
        return {"ekin": out[0], "epot": out[1], "mom": (out[2], out[3], out[4])}

    # ---- block time-steps
    def block_start(self, dt_max: float, k_max: int, eta: float, theta: float, eps: float, stream=None):
        """Forces at t = 0 and first levels on the loaded state (bh_block_start)."""
        _check(self.lib.bh_block_start(self.ctx, float(dt_max), int(k_max), float(eta), float(theta), float(eps),
                                       _stream(stream)), "bh_block_start")
        self.blk = (float(dt_max), int(k_max))

    def block_step(self, theta: float, eps: float, rebuild: bool = True, stream=None):
        """One block step: rebuild the tree or refresh its moments (bh_block_step)."""
        _check(self.lib.bh_block_step(self.ctx, float(theta), float(eps), int(bool(rebuild)), _stream(stream)),
               "bh_block_step")

    def block_info(self, stream=None) -> dict:
        out = (ctypes.c_int64 * 4)()
        _check(self.lib.bh_block_info(self.ctx, out, _stream(stream)), "bh_block_info")
        dt_max, k_max = self.blk
        return {"tick": out[0], "time": out[0] * dt_max / 2.0 ** k_max, "active": out[1], "groups": out[2],
                "deepest": out[3]}

    def block_levels(self, stream=None):
        """(levels int32 [n], ticks int64 [n]) in the caller's order, on the device."""
        import torch

        lv = torch.empty(self.n_state, dtype=torch.int32, device=f"cuda:{self.device}")
        tk = torch.empty(self.n_state, dtype=torch.int64, device=f"cuda:{self.device}")
        _check(self.lib.bh_block_levels(self.ctx, ctypes.c_void_p(lv.data_ptr()), ctypes.c_void_p(tk.data_ptr()),
                                        _stream(stream)), "bh_block_levels")
        return lv, tk

    # ---- status and exports
    def status(self, stream=None) -> int:
        return self.lib.bh_status(self.ctx, _stream(stream))

    def check(self, stream=None):
        _check(self.status(stream), "device status")

    def wait_probe(self, spin_limit: int = 1000, stream=None):
        """Run a bounded device wait that nothing ends (failure-detection test
        hook); the status word then reads BH_ERR_TIMEOUT."""
        _check(self.lib.bh_wait_probe(self.ctx, spin_limit, _stream(stream)), "bh_wait_probe")

    def counts(self, stream=None) -> dict:
        out = (ctypes.c_int64 * 9)()
        _check(self.lib.bh_get_counts(self.ctx, out, _stream(stream)), "bh_get_counts")
        keys = ("n", "cells", "groups", "systems", "deepest", "walks", "pp", "pc", "launches")
        return dict(zip(keys, list(out)))

    def reset_counters(self, stream=None):
        _check(self.lib.bh_reset_counters(self.ctx, _stream(stream)), "bh_reset_counters")

    def tree(self, stream=None) -> dict:
        import numpy as np

        c = self.counts(stream)
        n, C, G = c["n"], c["cells"], c["groups"]
        out = {
            "skey": np.zeros(n, np.uint64), "perm": np.zeros(n, np.int32),
            "level": np.zeros(C, np.int32), "pbeg": np.zeros(C, np.int32), "pend": np.zeros(C, np.int32),
            "parent": np.zeros(C, np.int32), "first_child": np.zeros(C, np.int32),
            "n_children": np.zeros(C, np.int32), "is_leaf": np.zeros(C, np.int32),
            "gbeg": np.zeros(G, np.int32), "gend": np.zeros(G, np.int32),
        }
        order = ("skey", "perm", "level", "pbeg", "pend", "parent", "first_child", "n_children", "is_leaf",
                 "gbeg", "gend")
        args = [out[k].ctypes.data_as(ctypes.c_void_p) for k in order]
        _check(self.lib.bh_get_tree(self.ctx, *args, _stream(stream)), "bh_get_tree")
        out["skey_lo"] = np.zeros(n, np.uint64)
        _check(self.lib.bh_get_keys_lo(self.ctx, out["skey_lo"].ctypes.data_as(ctypes.c_void_p), _stream(stream)),
               "bh_get_keys_lo")
        return out

    def moments(self, stream=None) -> dict:
        import numpy as np

        C = self.counts(stream)["cells"]
        out = {"mass": np.zeros(C, np.float32), "com": np.zeros((C, 3)), "quad": np.zeros((C, 6), np.float32),
               "delta": np.zeros(C, np.float32), "size": np.zeros(C, np.float32)}
        args = [out[k].ctypes.data_as(ctypes.c_void_p) for k in ("mass", "com", "quad", "delta", "size")]
        _check(self.lib.bh_get_moments(self.ctx, *args, _stream(stream)), "bh_get_moments")
        return out

    def group_stats(self, stream=None) -> dict:
        import numpy as np

        G = self.counts(stream)["groups"]
        out = {"nc": np.zeros(G, np.int32), "np": np.zeros(G, np.int32), "csum": np.zeros(G, np.uint64),
               "psum": np.zeros(G, np.uint64)}
        args = [out[k].ctypes.data_as(ctypes.c_void_p) for k in ("nc", "np", "csum", "psum")]
        _check(self.lib.bh_get_group_stats(self.ctx, *args, _stream(stream)), "bh_get_group_stats")
        return out

    def set_profiling(self, on: bool = True):
        _check(self.lib.bh_set_profiling(self.ctx, int(on)), "bh_set_profiling")

    def phase_times(self) -> dict:
        ms = (ctypes.c_float * BH_NPHASES)()
        _check(self.lib.bh_phase_times(self.ctx, ms), "bh_phase_times")
        return dict(zip(PHASES, list(ms)))

    def exclusive_scan(self, x, stream=None):
        import torch

        out = torch.empty_like(x)
        total = ctypes.c_uint64(0)
        _check(self.lib.bh_prim_exclusive_scan(self.ctx, _ptr(x), _ptr(out), x.numel(), ctypes.byref(total),
                                               _stream(stream)), "bh_prim_exclusive_scan")
        return out, total.value
