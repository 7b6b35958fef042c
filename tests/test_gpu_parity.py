"""Parity of the CUDA path with the FP64 oracle, step by step (marked gpu).

Each test runs a C-ABI entry point of libbfm.so through the thin binding and
compares it element by element with the oracle on the same seeded inputs, at
sizes that span several line tiles and leave ragged tails (line counts that
are not multiples of the tile width, line lengths that are not multiples of
the per-thread chunk).

Tolerances:
  FP64  c-transform / map / pushforward: 1e-12 relative to the field scale (a
        minimum over identical candidates can differ only by rounding);
        Poisson 1e-10 (FFT vs definition order of summation).
  FP32  the oracle is run on the FP32 input widened to FP64, so the only
        differences are FP32 rounding in the kernels: c-transform 4 ulp of
        the field scale, Poisson 2e-5 relative, pushforward 2e-5 of max rho.
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


def dev(x, dt=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(x), dtype=dt, device="cuda")


def host(t):
    return t.detach().double().cpu().numpy()


# rows of more than 256 cells take the row kernel (one thread group per row,
# 16 cells per thread below 1024, else 32): aligned, ragged (257, 300, 1500)
# and unaligned (511, 1027) lengths, in 2-D and 3-D; lines of more than 256
# cells along axes 1 and 2 take the same kernel on interleaved tiles of 16
# lines (257-, 300- and 384-cell columns), with the last tile of a plane
# partly filled where the axis-0 length is not a multiple of 16 (3, 8, 40,
# 20); shorter lines and 1024-cell columns take tiles of the tile kernel
CT_SHAPES = [(2, 2), (7, 5), (64, 64), (33, 100), (257, 96), (48, 31, 20), (9, 40, 13),
             (300, 5, 3), (511, 7), (1024, 3), (1500, 4), (1027, 3), (4096, 2),
             (6, 384, 32), (384, 4, 8), (3, 384), (3, 300, 40), (260, 3, 20)]


@pytest.mark.parametrize("shape", CT_SHAPES, ids=str)
def test_ctransform_fp64(B, shape):
    for seed, phi in ((1, si.random_field(shape, 1, 0.1)),
                      (2, si.smooth_potential(tuple(reversed(shape)), 2, 0.2))):
        want = oracle.ctransform(phi, "brute" if phi.size <= 70000 else "linear")
        got = host(B.bfm_ctransform(dev(phi)))
        scale = 1.0 + np.max(np.abs(phi))
        assert np.max(np.abs(got - want)) <= 1e-12 * scale, (shape, seed)


@pytest.mark.parametrize("shape", CT_SHAPES, ids=str)
def test_ctransform_fp32(B, shape):
    phi = si.smooth_potential(tuple(reversed(shape)), 3, 0.2) + 0.01 * si.random_field(shape, 3)
    phi32 = phi.astype(np.float32)
    want = oracle.ctransform(phi32.astype(np.float64), "linear")
    got = host(B.bfm_ctransform(dev(phi32, torch.float32)))
    scale = 1.0 + np.max(np.abs(phi))
    assert np.max(np.abs(got - want)) <= 4 * np.finfo(np.float32).eps * scale


# |x|^2/2 - phi affine along every line: the rounded FP32 values leave many
# parabolas on the envelope that meet at nearly one point, where the FP32
# owner ranking can see start cells decrease and hands the line to the sweep;
# rows of 4096 and 1500 (row kernel), 300- and 384-cell columns (row kernel
# on interleaved tiles) and short rows (tiles)
DEGENERATE_SHAPES = [(4096, 3), (6, 1500), (300, 64), (40, 200), (5, 384, 9)]


@pytest.mark.parametrize("shape", DEGENERATE_SHAPES, ids=str)
def test_ctransform_degenerate_envelope(B, shape):
    phi = si.quadratic_potential(tuple(reversed(shape)), 7)
    scale = 1.0 + np.max(np.abs(phi))
    want = oracle.ctransform(phi, "linear")
    got = host(B.bfm_ctransform(dev(phi)))
    assert np.max(np.abs(got - want)) <= 1e-12 * scale
    phi32 = phi.astype(np.float32)
    want32 = oracle.ctransform(phi32.astype(np.float64), "linear")
    got32 = host(B.bfm_ctransform(dev(phi32, torch.float32)))
    assert np.max(np.abs(got32 - want32)) <= 4 * np.finfo(np.float32).eps * scale


def test_ctransform_in_place_and_invariants(B):
    phi = dev(si.random_field((40, 56), 4, 0.1))
    c1 = B.bfm_ctransform(phi)
    c2 = B.bfm_ctransform(c1)
    c3 = B.bfm_ctransform(c2)
    assert torch.all(phi <= c2 + 1e-15)            # Lemma 2.2(i)
    assert torch.max(torch.abs(c3 - c1)).item() < 1e-14
    x = c1.clone()
    B.bfm_ctransform(x, out=x)                      # in place
    assert torch.equal(x, c2)


def test_ctransform_long_rows_in_place(B):
    """The row kernel reads a whole row before writing it: in place equals out of place."""
    phi = dev(si.smooth_potential((5, 2048), 11, 0.2) + 0.01 * si.random_field((2048, 5), 11))
    c1 = B.bfm_ctransform(phi)
    x = phi.clone()
    B.bfm_ctransform(x, out=x)
    assert torch.equal(x, c1)


POISSON_SHAPES = [(2, 3), (16, 12), (64, 48), (96, 128), (27, 32), (384, 8), (12, 18, 16),
                  (24, 6, 9)]


@pytest.mark.parametrize("shape", POISSON_SHAPES, ids=str)
def test_poisson_fp64(B, shape):
    f = si.random_field(shape, 5)
    g_want, G_want = oracle.poisson(f, "definition" if f.size <= 5000 else "fft")
    g_got, G_got = B.bfm_poisson(dev(f))
    g_got = host(g_got)
    scale = np.max(np.abs(g_want))
    assert np.max(np.abs(g_got - g_want)) <= 1e-10 * scale
    assert abs(G_got - G_want) <= 1e-10 * abs(G_want)


@pytest.mark.parametrize("shape", [(64, 48), (256, 96), (12, 18, 16)], ids=str)
def test_poisson_fp32(B, shape):
    f = si.random_field(shape, 6).astype(np.float32)
    g_want, G_want = oracle.poisson(f.astype(np.float64))
    g_got, G_got = B.bfm_poisson(dev(f, torch.float32))
    g_got = host(g_got)
    assert np.max(np.abs(g_got - g_want)) <= 2e-5 * np.max(np.abs(g_want))
    assert abs(G_got - G_want) <= 2e-5 * abs(G_want)


# Rows of 512 to 4096 FP32 cells take the compile-time row kernel
# (float4 rows, one line pair per CTA); odd row counts leave a last pair with
# one line.
@pytest.mark.parametrize("shape", [(3, 4096), (16, 4096), (27, 2048), (48, 1024), (9, 1024), (9, 512)],
                         ids=str)
def test_poisson_fp32_long_rows(B, shape):
    f = si.random_field(shape, 7).astype(np.float32)
    g_want, G_want = oracle.poisson(f.astype(np.float64))
    g_got, G_got = B.bfm_poisson(dev(f, torch.float32))
    g_got = host(g_got)
    assert np.max(np.abs(g_got - g_want)) <= 2e-5 * np.max(np.abs(g_want))
    assert abs(G_got - G_want) <= 2e-5 * abs(G_want)


# Lines of 384 FP32 cells take the register FFT of radices 4 x 4 x 4 x 6 with
# tiles of 32 whole lines: rows (axis 0), interleaved lines of axis 1 and the
# middle pass along the last axis (2-D and 3-D, with the eigenvalues of both
# other axes).
@pytest.mark.parametrize("shape", [(64, 384), (384, 32), (384, 8, 32), (32, 384, 64), (24, 32, 384)],
                         ids=str)
def test_poisson_fp32_384(B, shape):
    f = si.random_field(shape, 8).astype(np.float32)
    g_want, G_want = oracle.poisson(f.astype(np.float64))
    g_got, G_got = B.bfm_poisson(dev(f, torch.float32))
    g_got = host(g_got)
    assert np.max(np.abs(g_got - g_want)) <= 2e-5 * np.max(np.abs(g_want))
    assert abs(G_got - G_want) <= 2e-5 * abs(G_want)


def test_poisson_unsupported_size(B):
    with pytest.raises(B.BfmError) as e:
        B.bfm_poisson(dev(np.zeros((7, 8))))
    assert e.value.status == B.BFM_ERR_UNSUPPORTED


@pytest.mark.parametrize("shape", [(64, 64), (37, 50), (20, 18, 22)], ids=str)
def test_map_and_pushforward_fp64(B, shape):
    mu = si.normalise(np.abs(si.random_field(shape, 7)) * (si.random_field(shape, 8) > -0.5))
    psi = si.smooth_potential(tuple(reversed(shape)), 9, 0.1)
    tmap = host(B.bfm_map(dev(psi)))
    assert np.max(np.abs(tmap - oracle.transport_map(psi))) <= 1e-13
    rho = host(B.bfm_pushforward(dev(psi), dev(mu)))
    want = oracle.pushforward(psi, mu)
    assert np.max(np.abs(rho - want)) <= 1e-12 * np.max(want)
    assert abs(rho.sum() - mu.sum()) <= 1e-12 * mu.sum()


def test_pushforward_fp32(B):
    shape = (128, 96)
    mu = si.normalise(np.abs(si.random_field(shape, 10))).astype(np.float32)
    psi = si.smooth_potential((96, 128), 11, 0.1).astype(np.float32)
    rho = host(B.bfm_pushforward(dev(psi, torch.float32), dev(mu, torch.float32)))
    want = oracle.pushforward(psi.astype(np.float64), mu.astype(np.float64))
    assert np.max(np.abs(rho - want)) <= 2e-5 * np.max(want)


@pytest.mark.parametrize("shape", [(1028, 6), (64, 40), (12, 10, 8), (6, 9), (8, 6, 5)], ids=str)
@pytest.mark.parametrize("amp", [0.1, 2.0])
def test_pushforward_fp32_shapes(B, shape, amp):
    """Lines of 4k cells take the vector row kernel (one 16-byte vector per
    thread, ragged last segment at 1028), others the per-cell kernel; amp 2
    sends much of the mass past the box and onto its faces."""
    mu = si.normalise(np.abs(si.random_field(shape, 12)) * (si.random_field(shape, 13) > -0.3))
    mu = mu.astype(np.float32)
    psi = (amp * si.smooth_potential(tuple(reversed(shape)), 14, 0.1)).astype(np.float32)
    rho = host(B.bfm_pushforward(dev(psi, torch.float32), dev(mu, torch.float32)))
    want = oracle.pushforward(psi.astype(np.float64), mu.astype(np.float64))
    assert np.max(np.abs(rho - want)) <= 2e-5 * np.max(want)
    assert abs(rho.sum() - mu.astype(np.float64).sum()) <= 1e-5 * mu.sum()


def test_interpolate(B):
    n = 64
    mu, nu = si.translated_discs(n)
    x, y = si.centres((n, n))
    T = np.stack([np.minimum(x + 0.5, 1 - 0.5 / n), np.minimum(y + 0.5, 1 - 0.5 / n)])
    for t in (0.0, 0.3, 0.5, 1.0):
        got = host(B.bfm_interpolate(dev(T), dev(mu), t))
        assert np.max(np.abs(got - oracle.interpolate(T, mu, t))) <= 1e-12 * np.max(mu)


# --- the whole method ---------------------------------------------------------

def test_solve_translated_discs_fp64(B):
    """Table 1 case: GPU and oracle follow the same iterates to rounding."""
    mu, nu = si.translated_discs(64)
    ref = oracle.solve(mu, nu, tol=0.0, max_iter=8)
    r = B.bfm_solve(dev(mu), dev(nu), tol=0.0, max_iter=8)
    assert r["iters"] == ref["iters"] == 8
    assert np.max(np.abs(r["dual"] - ref["dual"])) < 1e-12
    assert np.max(np.abs(r["resid"] - ref["resid"])) < 1e-9
    assert np.max(np.abs(r["sigma"] - ref["sigma"])) < 1e-12
    assert abs(r["w2sq"] - 0.5) < 1e-12
    assert np.max(np.abs(host(r["phi"]) - ref["phi"])) < 1e-10
    assert np.max(np.abs(host(r["psi"]) - ref["psi"])) < 1e-10
    assert np.max(np.abs(host(r["map"]) - ref["map"])) * 64 < 1e-8     # in cells


def test_solve_gauss_disc_64_fp64(B):
    """3 Gaussians -> disc, 64x64, FP64 plain method, tol 1e-6 or 300 iterations."""
    mu, nu = si.workload_gauss_disc_64()
    ref = oracle.solve(mu, nu, tol=1e-6, max_iter=300)
    r = B.bfm_solve(dev(mu), dev(nu), tol=1e-6, max_iter=300)
    assert r["iters"] == ref["iters"]
    assert r["converged"] == ref["converged"]
    k = min(len(r["dual"]), len(ref["dual"]))
    assert np.max(np.abs(r["dual"][:k] - ref["dual"][:k])) < 1e-9
    assert np.max(np.abs(r["resid"][:k] - ref["resid"][:k])) < 1e-6
    assert abs(r["w2sq"] - ref["w2sq"]) / ref["w2sq"] < 1e-9
    assert np.max(np.abs(host(r["map"]) - ref["map"])) * 64 < 1e-4      # in cells


def test_solve_3d_fp64(B):
    mu, nu = si.translated_balls(24)
    ref = oracle.solve(mu, nu, tol=0.0, max_iter=6)
    r = B.bfm_solve(dev(mu), dev(nu), tol=0.0, max_iter=6)
    assert np.max(np.abs(r["dual"] - ref["dual"])) < 1e-11
    assert abs(r["w2sq"] - ref["w2sq"]) < 1e-11


def test_solve_3d_fp32_384_lines(B):
    """FP32 3-D solve whose axis-0 and axis-2 lines have 384 cells (the
    384-point register FFT on rows and on the middle pass)."""
    shape = (384, 4, 384)
    rng = np.random.default_rng(46)
    mu = si.normalise(si.gaussian_mixture(shape, rng.uniform(0.3, 0.7, (2, 3)), [0.12, 0.08]))
    nu = si.normalise(si.gaussian_mixture(shape, rng.uniform(0.3, 0.7, (3, 3)), [0.1, 0.1, 0.07]))
    ref = oracle.solve(mu, nu, tol=0.0, max_iter=3)
    r = B.bfm_solve(dev(mu, torch.float32), dev(nu, torch.float32), tol=0.0, max_iter=3)
    assert r["iters"] == 3
    assert abs(r["w2sq"] - ref["w2sq"]) / ref["w2sq"] < 1e-5
    assert np.max(np.abs(r["resid"] - ref["resid"])) < 1e-3


def test_solve_fp32_matches_fp64_oracle(B):
    """FP32 bulk with FP64 reductions: W2^2 within 1e-5 relative of the oracle."""
    mu, nu = si.workload_annulus_5g_4096(256)
    ref = oracle.solve(mu, nu, tol=0.0, max_iter=30)
    r = B.bfm_solve(dev(mu, torch.float32), dev(nu, torch.float32), tol=0.0, max_iter=30)
    assert r["iters"] == 30
    assert abs(r["w2sq"] - ref["w2sq"]) / ref["w2sq"] < 1e-5
    assert np.max(np.abs(r["resid"] - ref["resid"])) < 1e-3
    assert np.max(np.abs(host(r["map"]) - ref["map"])) * 256 < 0.05     # in cells


def test_solve_host_buffers(B):
    mu, nu = si.translated_discs(32)
    r = B.bfm_solve_host(mu, nu, tol=0.0, max_iter=5)
    ref = oracle.solve(mu, nu, tol=0.0, max_iter=5)
    assert abs(r["w2sq"] - ref["w2sq"]) < 1e-12
    assert np.max(np.abs(r["phi"] - ref["phi"])) < 1e-10
    # results into caller-owned page-locked arrays: the same values, in place
    outs = {k: torch.empty(shape, dtype=torch.float64).pin_memory().numpy()
            for k, shape in (("phi", mu.shape), ("psi", mu.shape), ("map", (2,) + mu.shape))}
    r2 = B.bfm_solve_host(mu, nu, tol=0.0, max_iter=5, out=outs)
    assert r2["phi"] is outs["phi"] and r2["map"] is outs["map"]
    for k in ("phi", "psi", "map"):
        assert np.array_equal(r2[k], r[k])
    with pytest.raises(ValueError):
        B.bfm_solve_host(mu, nu, tol=0.0, max_iter=5, out={"phi": np.empty((3, 3))})


def test_solve_converges_and_stops(B):
    mu, nu = si.translated_discs(64)
    r = B.bfm_solve(dev(mu), dev(nu), tol=1e-2, max_iter=50)
    ref = oracle.solve(mu, nu, tol=1e-2, max_iter=50)
    assert r["converged"] and r["status"] == B.BFM_OK
    assert r["iters"] == ref["iters"] < 50
    assert r["resid"][-1] < 1e-2


def test_solve_rejects_bad_input(B):
    mu, nu = si.translated_discs(16)
    for bad in (-mu, np.zeros_like(mu), np.where(mu > 0, np.nan, 0.0)):
        with pytest.raises(B.BfmError) as e:
            B.bfm_solve(dev(bad), dev(nu), max_iter=2)
        assert e.value.status == B.BFM_ERR_INVALID_ARG
    with pytest.raises(B.BfmError) as e:
        B.bfm_solve(dev(np.ones((5, 7))), dev(np.ones((5, 7))), max_iter=2)
    assert e.value.status == B.BFM_ERR_UNSUPPORTED
    ws = torch.empty(1024, dtype=torch.uint8, device="cuda")
    with pytest.raises(B.BfmError) as e:
        B.bfm_solve(dev(mu), dev(nu), max_iter=2, workspace=ws)
    assert e.value.status == B.BFM_ERR_WORKSPACE


def test_solve_nonfinite_returns_status(B):
    """A non-finite dual value or gradient norm ends the solve with
    BFM_ERR_NONFINITE (made on the host: nothing faults).  FP32: a first step
    of 1e300 turns phi into infinities; FP64: a warm start whose phi is
    infinite on the target's support.  The context stays usable."""
    mu, nu = si.translated_discs(32)
    with pytest.raises(B.BfmError) as e:
        B.bfm_solve(dev(mu, torch.float32), dev(nu, torch.float32), tol=0.0, max_iter=4,
                    sigma0=1e300)
    assert e.value.status == B.BFM_ERR_NONFINITE
    phi0 = np.where(nu > 0, np.inf, 0.0)
    with pytest.raises(B.BfmError) as e:
        B.bfm_solve(dev(mu), dev(nu), tol=0.0, max_iter=4, phi_init=dev(phi0))
    assert e.value.status == B.BFM_ERR_NONFINITE
    r = B.bfm_solve(dev(mu), dev(nu), tol=0.0, max_iter=2)
    ref = oracle.solve(mu, nu, tol=0.0, max_iter=2)
    assert abs(r["w2sq"] - ref["w2sq"]) < 1e-12


def test_solve_max_iter_zero(B):
    mu, nu = si.translated_discs(16)
    r = B.bfm_solve(dev(mu), dev(nu), tol=0.0, max_iter=0)
    ref = oracle.solve(mu, nu, tol=0.0, max_iter=0)
    assert r["iters"] == 0 and r["status"] == B.BFM_NOT_CONVERGED
    assert abs(r["resid"][0] - ref["resid"][0]) < 1e-12


def test_stepwise_solver_matches_solve(B):
    """bfm_solver_init / iterate / finish give exactly what bfm_solve gives."""
    mu, nu = si.workload_gauss_disc_64(32)
    r = B.bfm_solve(dev(mu), dev(nu), tol=0.0, max_iter=7)
    s = B.BfmSolver(dev(mu), dev(nu), tol=0.0, max_iter=7)
    s.iterate(3)
    s.iterate(2)
    q = s.finish()                 # stops at iteration 5 and measures phi_5
    ref5 = oracle.solve(mu, nu, tol=0.0, max_iter=5)
    assert q["iters"] == 5
    assert abs(q["w2sq"] - ref5["w2sq"]) < 1e-12
    assert np.max(np.abs(q["resid"] - ref5["resid"])) < 1e-9
    s2 = B.BfmSolver(dev(mu), dev(nu), tol=0.0, max_iter=7)
    s2.iterate(20)                 # iterations past max_iter do no work
    q2 = s2.finish()
    assert q2["iters"] == r["iters"] == 7
    # the pushforward's atomic adds land in any order, so equal up to rounding
    assert abs(q2["w2sq"] - r["w2sq"]) < 1e-14
    assert torch.max(torch.abs(q2["phi"] - r["phi"])).item() < 1e-12
    assert torch.max(torch.abs(q2["psi"] - r["psi"])).item() < 1e-12


def test_warm_start(B):
    """Resuming from phi_n (checkpoint/resume) continues the iteration."""
    mu, nu = si.translated_discs(32)
    r = B.bfm_solve(dev(mu), dev(nu), tol=0.0, max_iter=3)
    r2 = B.bfm_solve(dev(mu), dev(nu), tol=0.0, max_iter=3, phi_init=r["phi"])
    assert r2["dual"][0] == pytest.approx(r["dual"][-1], abs=1e-14)
    assert r2["w2sq"] >= r["w2sq"] - 1e-12


def test_profiler_counts_launches(B):
    mu, nu = si.translated_discs(32)
    s = B.BfmSolver(dev(mu), dev(nu), tol=0.0, max_iter=10)
    B.bfm_profile_begin(200)
    s.iterate(2)
    prof = B.bfm_profile_end()
    # per iteration in 2D: 8 c-transform passes, 2 pushforwards, 2 x (fwd, mid, inv)
    # DCT passes, 6 reduction/step kernels
    assert prof["ct_pass_axis0"][1] == 8 and prof["ct_pass_axis1"][1] == 8
    assert prof["pushforward"][1] == 4
    assert prof["dct_fwd"][1] == prof["dct_mid"][1] == prof["dct_inv"][1] == 4
    assert prof["reduce_step"][1] == 12
    assert prof["transpose"][1] == 0          # short columns: interleaved column tiles
    assert prof["_dropped"][1] == 0
    assert all(v[0] > 0 for k, v in prof.items() if not k.startswith("_") and v[1])


# --- long columns: axis-1 sweeps along the rows of a transposed copy ----------
# A tile of neighbouring columns holds only a few lines when the columns are
# long (from 1024 FP64 or 2048 FP32 cells), so 2-D grids with such columns
# transpose the field, sweep rows and transpose back.  The grids below are
# narrow (few columns) so that the oracle stays fast, and n0 is not a power
# of two so the row sweeps of the original layout take the general DCT path.

def long_column_pair(shape, seed):
    rng = np.random.default_rng(seed)
    mu = si.normalise(si.gaussian_mixture(shape, rng.uniform(0.3, 0.7, (2, 2)), [0.12, 0.08]))
    nu = si.normalise(si.gaussian_mixture(shape, rng.uniform(0.3, 0.7, (3, 2)), [0.1, 0.1, 0.07]))
    return mu, nu


def test_solve_long_columns_fp64(B):
    mu, nu = long_column_pair((48, 1024), 41)
    ref = oracle.solve(mu, nu, tol=0.0, max_iter=6)
    r = B.bfm_solve(dev(mu), dev(nu), tol=0.0, max_iter=6)
    assert r["iters"] == ref["iters"] == 6
    assert np.max(np.abs(r["dual"] - ref["dual"])) < 1e-12
    assert np.max(np.abs(r["resid"] - ref["resid"])) < 1e-9
    assert np.max(np.abs(r["sigma"] - ref["sigma"])) < 1e-12
    assert abs(r["w2sq"] - ref["w2sq"]) < 1e-12
    assert np.max(np.abs(host(r["phi"]) - ref["phi"])) < 1e-10
    assert np.max(np.abs(host(r["psi"]) - ref["psi"])) < 1e-10
    assert np.max(np.abs(host(r["map"]) - ref["map"])) * 1024 < 1e-8    # in cells


def test_solve_long_columns_fp32(B):
    mu, nu = long_column_pair((24, 2048), 42)
    ref = oracle.solve(mu, nu, tol=0.0, max_iter=10)
    r = B.bfm_solve(dev(mu, torch.float32), dev(nu, torch.float32), tol=0.0, max_iter=10)
    assert r["iters"] == 10
    assert abs(r["w2sq"] - ref["w2sq"]) / ref["w2sq"] < 1e-5
    assert np.max(np.abs(r["resid"] - ref["resid"])) < 1e-3


@pytest.mark.parametrize("shape,dt", [((48, 1024), torch.float64), ((24, 2048), torch.float32)],
                         ids=["fp64", "fp32"])
def test_long_columns_take_transposed_sweeps(B, shape, dt):
    """Per iteration on a grid whose columns are long and rows short: the
    phi-half runs in the grid's layout (its first c-transform leaves psi~
    transposed for the pushforward, its Poisson solve transposes before and
    after its axis-1 sweep), the psi-half on the transposed grid (whose
    columns are short: no transposes), and the c-transforms phi -> psi and
    psi -> phi leave their outputs transposed (one transpose each):
    1 + 2 + 1 + 1."""
    mu, nu = long_column_pair(shape, 43)
    s = B.BfmSolver(dev(mu, dt), dev(nu, dt), tol=0.0, max_iter=10)
    B.bfm_profile_begin(200)
    s.iterate(1)
    prof = B.bfm_profile_end()
    assert prof["transpose"][1] == 5
    assert prof["ct_pass_axis0"][1] == prof["ct_pass_axis1"][1] == 4
    assert prof["dct_fwd"][1] == prof["dct_mid"][1] == prof["dct_inv"][1] == 2
    assert prof["_dropped"][1] == 0


# FP32 grids with long columns and long rows: both sweeps of every c-transform
# take the row kernel (the axis-1 sweep on the transposed copy); 324 columns
# leave a partial last round of 8-line CTAs in the sweep of the copy, and
# rows of 288 or 324 cells take 16 cells per thread and 16 lines per CTA.
# psi = phi^c of the returned phi is checked cell by cell.

@pytest.mark.parametrize("shape", [(288, 2048), (324, 2048), (16, 4096), (4096, 12)], ids=str)
def test_solve_long_rows_and_columns_fp32(B, shape):
    mu, nu = long_column_pair(shape, 44)
    ref = oracle.solve(mu, nu, tol=0.0, max_iter=6)
    r = B.bfm_solve(dev(mu, torch.float32), dev(nu, torch.float32), tol=0.0, max_iter=6)
    assert r["iters"] == 6
    assert abs(r["w2sq"] - ref["w2sq"]) / ref["w2sq"] < 1e-5
    assert np.max(np.abs(r["resid"] - ref["resid"])) < 1e-3
    phi = host(r["phi"])
    want = oracle.ctransform(phi, "linear")
    scale = 1.0 + np.max(np.abs(phi))
    assert np.max(np.abs(host(r["psi"]) - want)) <= 4 * np.finfo(np.float32).eps * scale


# Long columns whose length is not a multiple of 4 cells: the pushforward's
# row form cannot read psi~ in the transposed layout, so psi~ goes back to
# the potential's layout by a transpose (with the dual dot) and the plain
# pushforward runs there (1458 = 2 x 3^6 cells, FP32 and FP64).
@pytest.mark.parametrize("shape,dt", [((12, 1458), torch.float32), ((6, 1458), torch.float64)],
                         ids=["fp32", "fp64"])
def test_solve_long_columns_not_multiple_of_4(B, shape, dt):
    mu, nu = long_column_pair(shape, 46)
    ref = oracle.solve(mu, nu, tol=0.0, max_iter=6)
    r = B.bfm_solve(dev(mu, dt), dev(nu, dt), tol=0.0, max_iter=6)
    assert r["iters"] == 6
    if dt == torch.float64:
        assert np.max(np.abs(r["dual"] - ref["dual"])) < 1e-12
        assert np.max(np.abs(host(r["phi"]) - ref["phi"])) < 1e-10
    else:
        assert abs(r["w2sq"] - ref["w2sq"]) / ref["w2sq"] < 1e-5
        assert np.max(np.abs(r["resid"] - ref["resid"])) < 1e-3
    s = B.BfmSolver(dev(mu, dt), dev(nu, dt), tol=0.0, max_iter=10)
    B.bfm_profile_begin(200)
    s.iterate(1)
    prof = B.bfm_profile_end()
    assert prof["transpose"][1] == 6                   # 2 + 2 + 1 + 1: psi~ transposed back


@pytest.mark.parametrize("shape,transposes", [((288, 2048), 5), ((2048, 2048), 8), ((486, 2048), 5),
                                              ((2048, 288), 0)], ids=str)
def test_transposes_follow_column_length(B, shape, transposes):
    """FP32 columns of 2048 cells are swept as rows of a transposed copy
    whatever the row length; short columns (2048 x 288) use column tiles.
    With long columns psi is kept transposed and the pushforward reads psi~
    in the transposed layout: 4 transposes per half step that sweeps long
    columns (psi~, the two around the Poisson middle pass, the flip), 1 per
    half step that does not (the flip): 5 per iteration when the rows are
    short, 8 when both axes are long."""
    mu, nu = long_column_pair(shape, 45)
    s = B.BfmSolver(dev(mu, torch.float32), dev(nu, torch.float32), tol=0.0, max_iter=10)
    B.bfm_profile_begin(200)
    s.iterate(1)
    prof = B.bfm_profile_end()
    assert prof["transpose"][1] == transposes
    assert prof["ct_pass_axis0"][1] == prof["ct_pass_axis1"][1] == 4
    assert prof["_dropped"][1] == 0


# --- the gradient-ascent baseline of Section 5 (Tables 5-6) -------------------

def test_gradient_ascent_fp64_matches_oracle(B):
    """phi += sigma grad J(phi), phi = phi^cc: the GPU keeps phi^c from the
    previous step (2 c-transforms per iteration), the oracle recomputes it;
    both follow the same iterates to rounding."""
    mu, nu = si.translated_discs(64)
    ref = oracle.solve(mu, nu, tol=0.0, max_iter=30, method="ga")
    r = B.bfm_solve(dev(mu), dev(nu), tol=0.0, max_iter=30, method="ga")
    assert r["iters"] == ref["iters"] == 30
    assert np.max(np.abs(r["dual"] - ref["dual"])) < 1e-11
    assert np.max(np.abs(r["resid"] - ref["resid"])) < 1e-8
    assert np.max(np.abs(r["sigma"] - ref["sigma"])) < 1e-12
    assert np.max(np.abs(host(r["phi"]) - ref["phi"])) < 1e-9
    assert np.max(np.abs(host(r["psi"]) - ref["psi"])) < 1e-9


def test_gradient_ascent_fp32_and_stepwise(B):
    mu, nu = si.workload_gauss_disc_64(64)
    ref = oracle.solve(mu, nu, tol=0.0, max_iter=25, method="ga")
    r = B.bfm_solve(dev(mu, torch.float32), dev(nu, torch.float32), tol=0.0, max_iter=25,
                    method="ga")
    assert abs(r["w2sq"] - ref["w2sq"]) / ref["w2sq"] < 1e-5
    s = B.BfmSolver(dev(mu, torch.float32), dev(nu, torch.float32), tol=0.0, max_iter=25,
                    method="ga")
    B.bfm_profile_begin(400)
    s.iterate(3)
    prof = B.bfm_profile_end()
    # per iteration: 2 c-transforms (2 sweeps each), 1 pushforward, 1 Poisson solve
    assert prof["ct_pass_axis0"][1] == prof["ct_pass_axis1"][1] == 6
    assert prof["pushforward"][1] == 3
    assert prof["dct_fwd"][1] == prof["dct_mid"][1] == prof["dct_inv"][1] == 3
    s.iterate(22)
    rs = s.finish(with_map=False)
    assert rs["iters"] == r["iters"]
    # FP32 atomics in the pushforward add in a run-dependent order
    assert np.max(np.abs(rs["dual"] - r["dual"])) < 1e-7


def test_gradient_ascent_rejected_by_batched_solver(B):
    mu, nu = si.translated_discs(16)
    with pytest.raises(B.BfmError):
        B.bfm_solve_batched([dev(mu)], [dev(nu)], tol=0.0, max_iter=3, method="ga")
