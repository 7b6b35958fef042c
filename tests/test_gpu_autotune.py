"""The c-transform shape tuner on the GPU (marked gpu).

Every candidate launch shape (K cells per thread, W lines per CTA) of every
kernel kind gives the oracle's c-transform (Definition 2.1, Section 4.1) on
lines of that length: FP64 to 1e-12 of the field scale, FP32 to 4 ulp of it,
the tolerances of the default shapes' tests.  The tuner's pick is a
candidate, is stored for later plans, and solves with tuned shapes still
match the oracle (FP64 iterates to rounding).
"""
import numpy as np
import pytest

import oracle
import synthetic_inputs as si

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def B():
    from paper_1905_12154_gb300 import binding
    binding.lib()
    return binding


@pytest.fixture(autouse=True)
def clean_table(B):
    B.bfm_tune_clear()
    yield
    B.bfm_tune_clear()


def _shape(kind, n, lines=37):
    # the grid whose passes take (kind, n): rows of n cells, or columns of n
    return (n, lines) if kind in (1, 3) else (lines, n)


CASES = [(0, 64), (0, 100), (0, 128), (0, 256), (1, 64), (1, 128), (1, 200), (1, 256),
         (1, 1024), (2, 384), (2, 512), (2, 1000), (2, 1024), (2, 4096), (3, 300), (3, 384),
         (3, 512)]


@pytest.mark.parametrize("kind,n", CASES, ids=lambda v: str(v))
@pytest.mark.parametrize("dt", [torch.float64, torch.float32], ids=["fp64", "fp32"])
def test_every_candidate_shape_matches_oracle(B, kind, n, dt):
    prec = B.BFM_FP64 if dt == torch.float64 else B.BFM_FP32
    shape = _shape(kind, n)
    assert (kind, n) in B.bfm_tune_passes(shape, prec, batched=True)
    phi = si.smooth_potential(tuple(reversed(shape)), 17 + n, 0.2)
    phi = phi + 1e-3 * si.random_field(shape, 3 + n)
    if dt == torch.float32:
        phi = phi.astype(np.float32).astype(np.float64)
    want = oracle.ctransform(phi, "brute")
    scale = 1.0 + np.max(np.abs(phi))
    tol = 1e-12 * scale if dt == torch.float64 else 4 * np.finfo(np.float32).eps * scale
    x = torch.as_tensor(phi, dtype=dt, device="cuda")
    for K, W in B.bfm_tune_candidates(kind, n, prec):
        B.bfm_tune_set(kind, n, K, W, prec)
        got = B.bfm_ctransform(x).double().cpu().numpy()
        err = np.max(np.abs(got - want))
        assert err <= tol, (kind, n, K, W, err)


@pytest.mark.parametrize("kind,n", [(1, 128), (2, 512), (2, 4096), (3, 384)], ids=str)
def test_autotune_picks_a_candidate_and_stores_it(B, kind, n):
    r = B.bfm_autotune(kind, n, B.BFM_FP32)
    cand = B.bfm_tune_candidates(kind, n, B.BFM_FP32)
    assert (r["K"], r["W"]) in cand
    assert all(c["ms"] > 0 for c in r["candidates"])
    assert B.bfm_tune_get(kind, n, B.BFM_FP32) == (r["K"], r["W"], True)
    best = min(c["ms"] for c in r["candidates"])
    chosen = [c["ms"] for c in r["candidates"] if (c["K"], c["W"]) == (r["K"], r["W"])][0]
    assert chosen <= 1.02 * best + 1e-9 or (r["K"], r["W"]) == r["default"]


def test_solves_with_tuned_shapes_match_oracle(B):
    mu, nu = si.workload_gauss_disc_64(64)
    tuned = B.autotune_grid(mu.shape, torch.float64)
    assert {(t["kind"], t["n"]) for t in tuned} == {("tile_rows", 64), ("tile_cols", 64)}
    # force shapes other than the defaults, so the solve runs on them
    for kind in (0, 1):
        K0, W0 = B.bfm_tune_default(kind, 64, B.BFM_FP64)
        other = [c for c in B.bfm_tune_candidates(kind, 64, B.BFM_FP64) if c[0] != K0][0]
        B.bfm_tune_set(kind, 64, *other, B.BFM_FP64)
    r = B.bfm_solve(torch.as_tensor(mu, device="cuda"), torch.as_tensor(nu, device="cuda"),
                    tol=0.0, max_iter=12)
    ref = oracle.solve(mu, nu, tol=0.0, max_iter=12)
    assert np.max(np.abs(r["dual"] - ref["dual"])) <= 1e-12
    assert np.max(np.abs(r["phi"].cpu().numpy() - ref["phi"])) <= 1e-10
