"""The C ABI library builds for sm_103a and exports every entry point of
include/bh.h (no GPU needed: the library is only loaded, nothing is called
that touches a device)."""
import ctypes
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "bh.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(bh_[a-z0-9_]+)\s*\(", txt)))


@pytest.mark.skipif(shutil.which("nvcc") is None, reason="nvcc not available")
def test_library_exports_every_declared_symbol():
    import paper_1106_1900_gb300 as bh

    bh.build()
    lib = ctypes.CDLL(bh.LIB_PATH)
    declared = _declared()
    assert len(declared) >= 20
    missing = [s for s in declared if not hasattr(lib, s)]
    assert not missing, f"not exported: {missing}"
    # the binding marshals exactly the declared entry points
    assert sorted(bh.exported_symbols()) == declared


@pytest.mark.skipif(shutil.which("nvcc") is None, reason="nvcc not available")
def test_status_strings_without_device():
    import paper_1106_1900_gb300 as bh

    lib = bh.load()
    for code, text in bh.STATUS.items():
        assert lib.bh_status_string(code).decode() == text
    p = bh.default_params()
    assert (p.n_leaf, p.n_crit, p.walk_variant) == (16, 64, 0)


def test_oracle_and_library_share_nothing():
    # the oracle never imports the CUDA package and vice versa
    osrc = open(os.path.join(ROOT, "oracle", "__init__.py")).read() + open(
        os.path.join(ROOT, "oracle", "bh_oracle.c")).read()
    assert not re.search(r"(import|from)\s+paper_1106_1900_gb300", osrc) and "#include" not in osrc.replace(
        "#include <", "")
    pkg = os.path.join(ROOT, "paper_1106_1900_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                src = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in src and "from oracle" not in src and "bh_oracle" not in src, f


def test_binding_rejects_wrong_buffers_and_parameters():
    """The binding checks argument buffers and parameter names before the
    library sees them (argument marshalling only; no device needed)."""
    import torch

    import paper_1106_1900_gb300 as bh

    ok = torch.zeros((4, 3), dtype=torch.float64)
    assert bh._arg(ok, torch.float64, "pos", cols=3, cuda=False) is not None
    for bad in (torch.zeros((4, 3), dtype=torch.float32), torch.zeros((3, 4), dtype=torch.float64).t(),
                torch.zeros((4, 2), dtype=torch.float64)):
        with pytest.raises(ValueError):
            bh._arg(bad, torch.float64, "pos", cols=3, cuda=False)
    with pytest.raises(ValueError):
        bh._arg(ok, torch.float64, "pos", cols=3, cuda=True)  # a host tensor where a device one is needed
    with pytest.raises(ValueError):
        bh._arg(None, torch.float64, "pos")
    assert bh.default_params(n_crit=96, key_levels=30).n_crit == 96
    with pytest.raises(ValueError):
        bh.default_params(n_crti=96)
