"""Separable power costs of Section 5 (eq. p_costs) on the GPU (marked gpu).

c(x,y) = sum_a |y_a - x_a|^{p_a}/p_a.  The c-transform passes (divide and
conquer over the monotone minimiser) are compared with the oracle's brute-force
lines, the map x - (grad h)^{-1}(grad psi) with the oracle's map, whole solves
with the oracle's solve, and the GPU solve with the closed forms the oracle is
pinned to: a translation costs h(a), and Section 5's two-disc example moves all
mass vertically at p = (1.1, 3).

Tolerances: FP64 1e-12 of the field scale (the minimum over the same
candidates, the cost table by CUDA's pow vs the C library's); FP32 8 ulp of
the field scale plus the cost's (the table by powf).
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


SHAPES = [((2, 2), (1.5, 2.5)), ((7, 5), (1.3, 3.0)), ((64, 64), (1.5, 2.5)),
          ((33, 100), (1.1, 3.0)), ((257, 96), (2.0, 1.25)), ((1024, 3), (1.75, 2.25)),
          ((48, 31, 20), (1.5, 2.0, 2.5)), ((9, 40, 13), (3.0, 1.2, 1.6))]


@pytest.mark.parametrize("shape,p", SHAPES, ids=[str(s) for s, _ in SHAPES])
def test_ctransform_power_fp64(B, shape, p):
    for seed, phi in ((1, si.random_field(shape, 1, 0.1)),
                      (2, si.smooth_potential(tuple(reversed(shape)), 2, 0.2))):
        want = oracle.ctransform_p(phi, p)
        got = host(B.bfm_ctransform(dev(phi), p=p))
        scale = 1.0 + np.max(np.abs(phi))
        assert np.max(np.abs(got - want)) <= 1e-12 * scale, (shape, seed)


@pytest.mark.parametrize("shape,p", SHAPES[2:6], ids=[str(s) for s, _ in SHAPES[2:6]])
def test_ctransform_power_fp32(B, shape, p):
    phi = (si.smooth_potential(tuple(reversed(shape)), 3, 0.2) + 0.01 * si.random_field(shape, 3)).astype(np.float32)
    want = oracle.ctransform_p(phi.astype(np.float64), p)
    got = host(B.bfm_ctransform(dev(phi, torch.float32), p=p))
    scale = 1.0 + np.max(np.abs(phi)) + 1.0
    assert np.max(np.abs(got - want)) <= 8 * np.finfo(np.float32).eps * scale


def test_map_power_fp64(B):
    shape, p = (40, 56), (1.4, 2.6)
    psi = si.smooth_potential(tuple(reversed(shape)), 4, 0.1)
    want = oracle.transport_map(psi, p)
    got = host(B.bfm_map(dev(psi), p=p))
    assert np.max(np.abs(got - want)) < 1e-12


def test_solve_power_fp64_matches_oracle(B):
    mu, nu = si.diagonal_to_antidiagonal_discs(64)
    p = (1.5, 2.5)
    ref = oracle.solve(mu, nu, tol=0.0, max_iter=8, p=p)
    r = B.bfm_solve(dev(mu), dev(nu), tol=0.0, max_iter=8, p=p)
    assert r["iters"] == ref["iters"] == 8
    assert np.max(np.abs(r["dual"] - ref["dual"])) < 1e-10
    assert np.max(np.abs(r["sigma"] - ref["sigma"])) < 1e-12
    assert np.max(np.abs(host(r["phi"]) - ref["phi"])) < 1e-8
    assert np.max(np.abs(host(r["map"]) - ref["map"])) * 64 < 1e-6      # in cells


def test_power_translation_closed_form(B):
    """A translation is optimal for any strictly convex h(y - x): cost h((1/2, 1/2))."""
    mu, nu = si.translated_discs(256)
    p = (1.5, 2.5)
    exact = 0.5 ** p[0] / p[0] + 0.5 ** p[1] / p[1]
    r = B.bfm_solve(dev(mu), dev(nu), tol=0.0, max_iter=15, p=p, with_map=False)
    assert np.all(r["dual"] <= exact + 1e-10)
    assert abs(r["dual"][-1] - exact) < 1e-8


def test_power_vertical_transport(B):
    """Section 5: with p = (1.1, 3) all mass of the diagonal discs moves
    vertically to the anti-diagonal discs, at cost (1/2)^3/3 = 1/24."""
    mu, nu = si.diagonal_to_antidiagonal_discs(256)
    r = B.bfm_solve(dev(mu), dev(nu), tol=0.0, max_iter=30, p=(1.1, 3.0))
    x, y = si.centres((256, 256))
    T = host(r["map"])
    m = mu > 0
    vertical = np.sum(mu[m] * (np.abs(T[1] - y)[m] > np.abs(T[0] - x)[m])) / np.sum(mu[m])
    assert vertical > 0.99
    assert abs(r["dual"][-1] - 1.0 / 24.0) < 1e-6


def test_power_cost_fp32_solve(B):
    mu, nu = si.diagonal_to_antidiagonal_discs(128)
    p = (1.5, 2.5)
    ref = oracle.solve(mu, nu, tol=0.0, max_iter=10, p=p)
    r = B.bfm_solve(dev(mu, torch.float32), dev(nu, torch.float32), tol=0.0, max_iter=10, p=p)
    assert abs(r["w2sq"] - ref["w2sq"]) / ref["w2sq"] < 1e-5


def test_power_cost_rejections(B):
    mu, nu = si.translated_discs(16)
    with pytest.raises(B.BfmError):
        B.bfm_solve(dev(mu), dev(nu), tol=0.0, max_iter=2, p=(1.0, 2.0))      # p must exceed 1
    with pytest.raises(B.BfmError):
        B.bfm_ctransform(dev(mu), p=(2.0, 20.0))                             # nor exceed 16
    with pytest.raises(B.BfmError):
        B.bfm_solve_batched([dev(mu)], [dev(nu)], tol=0.0, max_iter=2, p=(1.5, 2.5))
