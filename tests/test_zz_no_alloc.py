"""The allocation-free scan entry point (bh_exclusive_scan_noalloc).

Some callers cannot allocate device memory (their host application owns all
of it), so this entry point keeps its scratch in an array compiled into the
library.  The test calls it through the C ABI twice in a row, on different
sizes, and checks each result against the workspace-based entry point
bh_prim_exclusive_scan (integer sums: exactly equal); then checks that a size
above the array's limit is refused before any launch.  This file sorts last
so that a run stopping at the first failure has run everything else first.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _p(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def test_noalloc_scan_matches_workspace_scan(cuda_lib):
    import torch

    lib = cuda_lib.load()
    tc = cuda_lib.TreeCode(1 << 20)
    stream = torch.cuda.current_stream()
    for n, seed in [(1 << 20, 1), (70001, 2)]:
        x = torch.from_numpy(np.random.default_rng(seed).integers(0, 1000, n).astype(np.int32)).cuda()
        want, want_total = tc.exclusive_scan(x)
        out = torch.full_like(x, -1)
        total = torch.full((1,), -1, dtype=torch.int64, device="cuda")
        rc = lib.bh_exclusive_scan_noalloc(_p(x), _p(out), n, _p(total), ctypes.c_void_p(stream.cuda_stream))
        assert rc == 0
        torch.cuda.synchronize()
        assert torch.equal(out, want)
        assert int(total.item()) == want_total
    # no total requested: still a valid scan
    x = torch.arange(9, dtype=torch.int32, device="cuda")
    out = cuda_lib.exclusive_scan_noalloc(x)
    assert out.cpu().tolist() == [0, 0, 1, 3, 6, 10, 15, 21, 28]


def test_noalloc_scan_rejects_sizes_above_its_limit(cuda_lib):
    lib = cuda_lib.load()
    rc = lib.bh_exclusive_scan_noalloc(None, None, cuda_lib.NOALLOC_SCAN_MAX_N + 1, None, None)
    assert rc == 2  # BH_ERR_CAPACITY, nothing launched
