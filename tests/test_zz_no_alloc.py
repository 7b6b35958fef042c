"""bfm_poisson_noalloc: the Poisson solve for callers that cannot allocate.

Callers whose device memory belongs to another allocator, or that may not
allocate after start-up (cudaMalloc/cudaFree synchronise the device), cannot
pass a workspace.  bfm_poisson_noalloc keeps its scratch in an array built
into the library instead.  These checks call it through the C ABI (ctypes) and
compare it with bfm_poisson, which takes a caller workspace, within the
tolerances of the Poisson parity tests: two calls in a row with different
grids and precisions, so the second call runs on scratch the first one left
behind.  The file is named to be collected last.
"""
import ctypes

import numpy as np
import pytest

import synthetic_inputs as si

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

TOL = {torch.float64: 1e-10, torch.float32: 2e-5}     # as in the Poisson parity tests


def _noalloc(B, f):
    """Call the C entry point directly; returns (status, g, G)."""
    out = torch.empty_like(f)
    grid = B.grid_of(f.shape)
    G = ctypes.c_double(float("nan"))
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    prec = B.BFM_FP64 if f.dtype == torch.float64 else B.BFM_FP32
    s = B.lib().bfm_poisson_noalloc(ctypes.c_void_p(f.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                    ctypes.byref(grid), prec, ctypes.byref(G), stream)
    return s, out, G.value


def test_noalloc_poisson_matches_workspace_poisson():
    from paper_1905_12154_gb300 import binding as B
    cases = [((12, 18, 24), torch.float64, 21),     # first call: 3D FP64
             ((96, 128), torch.float32, 22)]        # second call: 2D FP32 on reused scratch
    for shape, dtype, seed in cases:
        f = torch.as_tensor(si.random_field(shape, seed), dtype=dtype, device="cuda")
        s, g, G = _noalloc(B, f)
        assert s == B.BFM_OK, B.last_error()
        g_ref, G_ref = B.bfm_poisson(f)
        torch.cuda.synchronize()
        scale = torch.max(torch.abs(g_ref)).item()
        assert torch.max(torch.abs(g - g_ref)).item() <= TOL[dtype] * scale
        assert abs(G - G_ref) <= TOL[dtype] * abs(G_ref)


def test_noalloc_poisson_rejects_grids_beyond_its_scratch():
    from paper_1905_12154_gb300 import binding as B
    f = torch.zeros(8, dtype=torch.float64, device="cuda")   # never read: rejected first
    grid = B.bfm_grid()
    grid.ndim = 2
    grid.n[0], grid.n[1], grid.n[2] = 8192, 8192, 1
    G = ctypes.c_double(0.0)
    s = B.lib().bfm_poisson_noalloc(ctypes.c_void_p(f.data_ptr()), ctypes.c_void_p(f.data_ptr()),
                                    ctypes.byref(grid), B.BFM_FP64, ctypes.byref(G), None)
    assert s == B.BFM_ERR_UNSUPPORTED
    assert "scratch" in B.last_error()
