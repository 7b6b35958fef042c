"""Parity of the 3-D c-transform on lines of 384 cells inside a solve (marked gpu).

A ball -> two anisotropic Gaussians problem on 384 x 384 x 128 cells, FP32,
runs five iterations of the step-wise solver; its lines along axes 0 and 1
have the 384 cells of the 384^3 workload (the row kernel on rows, and on
interleaved tiles of 16 columns with double-buffered tile loads), those
along axis 2 take the tile kernel.  psi = phi^c (Definition 2.1, dimension
splitting of Section 4.1) of the GPU's own iterate phi_5 is then checked on
every cell against the oracle's Legendre-line transform of the same phi_5
widened to FP64: 4 ulp of the field scale, the tolerance of the smaller
FP32 c-transform tests.  The solve's own c-transforms ran the same kernels
on the way to phi_5; the dual values they produced must be finite and the
mass of T#mu must be conserved.
"""
import numpy as np
import pytest

import oracle
import synthetic_inputs as si

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

SHAPE_XYZ = (384, 384, 128)


@pytest.fixture(scope="module")
def B():
    from paper_1905_12154_gb300 import binding
    binding.lib()
    return binding


def _problem():
    mu = si.normalise(si.ball(SHAPE_XYZ, (0.3, 0.3, 0.35), 0.25))
    means = [(0.6, 0.7, 0.5), (0.75, 0.45, 0.6)]
    sig = [(0.07, 0.045, 0.1), (0.04, 0.07, 0.07)]
    nu = si.gaussian_mixture(SHAPE_XYZ, means, sig, weights=[2.0 / 3.0, 1.0 / 3.0])
    nu = np.where(nu < 1e-3 * nu.max(), 0.0, nu)
    return mu, si.normalise(nu)


def test_3d_384_lines_psi_whole_field(B):
    mu, nu = _problem()
    m = torch.as_tensor(mu, dtype=torch.float32, device="cuda")
    n = torch.as_tensor(nu, dtype=torch.float32, device="cuda")
    assert (B.CT_KIND_ROW_COLS, 384) in B.bfm_tune_passes(m.shape, B.BFM_FP32)
    s = B.BfmSolver(m, n, tol=0.0, max_iter=10)
    s.iterate(5)
    torch.cuda.synchronize()
    phi = s.phi.clone()
    psi = B.bfm_ctransform(phi).double().cpu().numpy()
    phi64 = phi.double().cpu().numpy()
    want = oracle.ctransform(phi64, "linear")
    scale = 1.0 + np.max(np.abs(phi64))
    err = np.max(np.abs(psi - want))
    assert err <= 4 * np.finfo(np.float32).eps * scale, err
    r = s.finish(with_map=False)
    assert r["iters"] == 5 and np.all(np.isfinite(r["dual"]))
    rho = B.bfm_pushforward(r["psi"], m)
    assert abs(float(rho.double().sum()) / mu.size - 1.0) < 1e-5
