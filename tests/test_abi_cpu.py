"""The C-ABI library builds for sm_103a, loads, and exports every entry point
that include/bfm.h declares (no GPU needed: nothing is called)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for f in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not f.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", f)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"\b(bfm_[a-z0-9_]+)\s*\(", text)
    return sorted(set(names))


@pytest.fixture(scope="module")
def libbfm():
    from paper_1905_12154_gb300 import build as cuda_build
    path = cuda_build.build()
    return ctypes.CDLL(path)


def test_header_declares_entry_points():
    names = declared_functions()
    for must in ("bfm_solve", "bfm_ctransform", "bfm_poisson", "bfm_pushforward", "bfm_map",
                 "bfm_interpolate", "bfm_workspace_bytes", "bfm_solve_host"):
        assert must in names


def test_library_exports_every_declared_symbol(libbfm):
    missing = [n for n in declared_functions() if not hasattr(libbfm, n)]
    assert not missing, missing


def test_host_only_calls(libbfm):
    """Calls that touch no device: status strings, options, workspace sizes."""
    from paper_1905_12154_gb300 import binding as B
    assert B.status_string(0) == "BFM_OK"
    assert B.status_string(-5) == "BFM_ERR_UNSUPPORTED"
    o = B._options()
    assert (o.beta1, o.beta2, o.alpha1, o.alpha2, o.sigma_min) == (0.25, 0.75, 1.25, 0.8, 0.01)
    nb = B.bfm_workspace_bytes((64, 64), B.BFM_FP32, 10)
    assert nb >= 4 * 64 * 64 * 4
    assert B.bfm_workspace_bytes((64, 64), B.BFM_FP64, 10) > nb
    assert B.bfm_workspace_bytes_host((64, 64), B.BFM_FP32, 10) > nb
    g = B.grid_of((8, 1))                       # n0 = 1 is not a grid
    assert B.lib().bfm_workspace_bytes(ctypes.byref(g), 0, 1) == 0


def test_library_is_sm103a():
    """The build targets sm_103a only (the flag list, not the binary, is read)."""
    from paper_1905_12154_gb300 import build as cuda_build
    assert cuda_build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]
