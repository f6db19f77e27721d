"""The allocation-free scan entry point (bh_exclusive_scan_noalloc).

Some callers cannot allocate device memory (their host application owns all
of it), so this entry point keeps its scratch in an array compiled into the
library.  The test calls it through the C ABI twice in a row, on different
sizes, and checks each result against the workspace-based entry point
bh_prim_exclusive_scan and against a host prefix sum in 64-bit integers
(outputs reduced modulo 2^32, the total exact); inputs whose total passes
2^32 and the largest accepted size are covered, as are the empty input and
a size above the array's limit, refused before any launch.  This file sorts
last so that a run stopping at the first failure has run everything else
first.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _p(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _host_scan(v_u32):
    """Exclusive prefix sums modulo 2^32 and the exact total, from uint64 sums."""
    c = np.cumsum(v_u32.astype(np.uint64), dtype=np.uint64)
    total = int(c[-1]) if len(c) else 0
    excl = np.concatenate([np.zeros(1, dtype=np.uint64), c[:-1]]) if len(c) else c
    assert excl.dtype == np.uint64
    return (excl & np.uint64(0xFFFFFFFF)).astype(np.uint32), total


def _noalloc(lib, x, stream):
    import torch

    out = torch.full_like(x, -1)
    total = torch.full((1,), -1, dtype=torch.int64, device="cuda")
    rc = lib.bh_exclusive_scan_noalloc(_p(x), _p(out), x.numel(), _p(total), ctypes.c_void_p(stream.cuda_stream))
    assert rc == 0
    torch.cuda.synchronize()
    return out, int(total.cpu().numpy().view(np.uint64)[0])


def test_noalloc_scan_matches_workspace_scan(cuda_lib):
    import torch

    lib = cuda_lib.load()
    tc = cuda_lib.TreeCode(1 << 20)
    stream = torch.cuda.current_stream()
    # two calls in a row; the second sums past 2^32 (values up to 2^31)
    for n, seed, hi in [(1 << 20, 1, 1000), (70001, 2, 1 << 31)]:
        v = np.random.default_rng(seed).integers(0, hi, n).astype(np.uint32)
        x = torch.from_numpy(v.view(np.int32)).cuda()
        want, want_total = tc.exclusive_scan(x)
        out, total = _noalloc(lib, x, stream)
        assert torch.equal(out, want)
        assert total == want_total
        ref, ref_total = _host_scan(v)
        assert np.array_equal(out.cpu().numpy().view(np.uint32), ref)
        assert total == ref_total
        if hi > 1000:
            assert total > 1 << 32
    # no total requested: still a valid scan
    x = torch.arange(9, dtype=torch.int32, device="cuda")
    out = cuda_lib.exclusive_scan_noalloc(x)
    assert out.cpu().tolist() == [0, 0, 1, 3, 6, 10, 15, 21, 28]


def test_noalloc_scan_largest_size_and_empty(cuda_lib):
    import torch

    lib = cuda_lib.load()
    stream = torch.cuda.current_stream()
    n = cuda_lib.NOALLOC_SCAN_MAX_N
    v = np.random.default_rng(3).integers(0, 1 << 32, n, dtype=np.uint64).astype(np.uint32)
    x = torch.from_numpy(v.view(np.int32)).cuda()
    out, total = _noalloc(lib, x, stream)
    ref, ref_total = _host_scan(v)
    assert np.array_equal(out.cpu().numpy().view(np.uint32), ref)
    assert total == ref_total and total > 1 << 56
    del x, out
    # n = 0: nothing to scan, total 0
    e = torch.empty(0, dtype=torch.int32, device="cuda")
    out, total = _noalloc(lib, e, stream)
    assert out.numel() == 0 and total == 0


def test_noalloc_scan_rejects_sizes_above_its_limit(cuda_lib):
    lib = cuda_lib.load()
    rc = lib.bh_exclusive_scan_noalloc(None, None, cuda_lib.NOALLOC_SCAN_MAX_N + 1, None, None)
    assert rc == 2  # BH_ERR_CAPACITY, nothing launched


def test_noalloc_binding_checks_its_arguments(cuda_lib):
    import torch

    with pytest.raises(ValueError):
        cuda_lib.exclusive_scan_noalloc(torch.arange(9, dtype=torch.int64, device="cuda"))
    with pytest.raises(ValueError):
        cuda_lib.exclusive_scan_noalloc(torch.arange(18, dtype=torch.int32, device="cuda")[::2])
    with pytest.raises(ValueError):
        cuda_lib.exclusive_scan_noalloc(torch.arange(9, dtype=torch.int32))
