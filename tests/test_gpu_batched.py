"""Batched uneven solves and the W2^2 backward (marked gpu).

The batched solver runs every problem with its own step size and convergence
flag in shared launches (one per grid shape and kernel step, replayed from a
CUDA graph); each problem must give what its own bfm_solve gives and what the
FP64 oracle gives.  The backward returns the mean-zero potentials (envelope
theorem on the dual problem), checked against the oracle's potentials and by
finite differences of the loss along mass-preserving perturbations.
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


def uneven_problems(count, sides, seed):
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        n = int(rng.choice(sides))
        pair = []
        for _ in range(2):
            k = int(rng.integers(1, 4))
            rho = si.gaussian_mixture((n, n), rng.uniform(0.25, 0.75, (k, 2)), rng.uniform(0.05, 0.15, k))
            pair.append(si.normalise(rho))
        out.append(tuple(pair))
    return out


def test_batched_equals_single_solves_fp64(B):
    probs = uneven_problems(7, (16, 24, 32, 48), 31)
    res = B.bfm_solve_batched([dev(m) for m, _ in probs], [dev(v) for _, v in probs],
                              tol=5e-2, max_iter=60, with_map=True)
    iters = set()
    for (m, v), r in zip(probs, res):
        single = B.bfm_solve(dev(m), dev(v), tol=5e-2, max_iter=60)
        assert r["iters"] == single["iters"]
        assert r["converged"] == single["converged"]
        assert abs(r["w2sq"] - single["w2sq"]) < 1e-12
        assert np.max(np.abs(r["dual"] - single["dual"])) < 1e-12
        assert torch.max(torch.abs(r["phi"] - single["phi"])).item() < 1e-10
        assert torch.max(torch.abs(r["map"] - single["map"])).item() < 1e-10
        iters.add(r["iters"])
    assert len(iters) > 1            # problems stopped at different iterations


def test_batched_matches_oracle(B):
    probs = uneven_problems(5, (16, 32), 32)
    res = B.bfm_solve_batched([dev(m) for m, _ in probs], [dev(v) for _, v in probs],
                              tol=0.0, max_iter=12)
    for (m, v), r in zip(probs, res):
        ref = oracle.solve(m, v, tol=0.0, max_iter=12)
        assert r["iters"] == 12
        assert abs(r["w2sq"] - ref["w2sq"]) < 1e-11
        assert np.max(np.abs(r["resid"] - ref["resid"])) < 1e-8


def test_batched_fp32_uneven_sizes(B):
    """FP32 fields with FP64 reductions: W2^2 within 1e-5 of the FP64 oracle."""
    probs = uneven_problems(6, (32, 64, 128), 33)
    res = B.bfm_solve_batched([dev(m, torch.float32) for m, _ in probs],
                              [dev(v, torch.float32) for _, v in probs], tol=0.0, max_iter=20)
    for (m, v), r in zip(probs, res):
        ref = oracle.solve(m, v, tol=0.0, max_iter=20)
        assert abs(r["w2sq"] - ref["w2sq"]) / ref["w2sq"] < 1e-5


def test_batched_fp32_long_rows(B):
    """Sides of 512 and 1024: the batched forms of the c-transform's row kernel
    and of the compile-time DCT row kernel; each problem as its own FP32 solve
    and within 1e-5 of the FP64 oracle."""
    probs = uneven_problems(3, (512, 1024), 35)
    res = B.bfm_solve_batched([dev(m, torch.float32) for m, _ in probs],
                              [dev(v, torch.float32) for _, v in probs], tol=0.0, max_iter=8)
    for (m, v), r in zip(probs, res):
        ref = oracle.solve(m, v, tol=0.0, max_iter=8)
        assert abs(r["w2sq"] - ref["w2sq"]) / ref["w2sq"] < 1e-5
        single = B.bfm_solve(dev(m, torch.float32), dev(v, torch.float32), tol=0.0, max_iter=8)
        assert abs(r["w2sq"] - single["w2sq"]) / single["w2sq"] < 1e-6


def test_batched_masks_stop_converged_problems(B):
    """A problem that converges early stops (its iteration count is its own)
    while a harder one keeps iterating in the same launches."""
    easy = si.translated_discs(32)
    hard = si.workload_gauss_disc_64(32)
    res = B.bfm_solve_batched([dev(easy[0]), dev(hard[0])], [dev(easy[1]), dev(hard[1])],
                              tol=2e-2, max_iter=40)
    ref_e = oracle.solve(*easy, tol=2e-2, max_iter=40)
    ref_h = oracle.solve(*hard, tol=2e-2, max_iter=40)
    assert res[0]["iters"] == ref_e["iters"]
    assert res[1]["iters"] == ref_h["iters"]
    assert res[0]["iters"] < res[1]["iters"]


def test_backward_equals_oracle_potentials(B):
    mu, nu = si.workload_loss_pairs_256(2, 32)[1]
    r = B.bfm_solve(dev(mu), dev(nu), tol=0.0, max_iter=40)
    ref = oracle.solve(mu, nu, tol=0.0, max_iter=40)
    gmu_ref, gnu_ref = oracle.w2_gradient(ref["phi"], ref["psi"], grad_out=1.5)
    gmu, gnu = B.bfm_w2_backward([r["phi"]], [r["psi"]], [r["mass_mu"]], [r["mass_nu"]],
                                 dev(np.array([1.5])))
    scale = np.max(np.abs(gmu_ref))
    assert np.max(np.abs(gmu[0].cpu().numpy() - gmu_ref)) < 1e-9 * scale
    assert np.max(np.abs(gnu[0].cpu().numpy() - gnu_ref)) < 1e-9 * np.max(np.abs(gnu_ref))
    assert abs(gmu[0].sum().item()) < 1e-12 and abs(gnu[0].sum().item()) < 1e-12


def test_w2_loss_autograd_and_finite_differences(B):
    """torch.autograd through the loss gives the backward kernel's gradients,
    and they agree with central differences of the loss along mass-preserving
    perturbations (the loss is the iteration's output, so a loose bound)."""
    pairs = si.workload_loss_pairs_256(2, 32)
    mu = torch.stack([dev(p[0]) for p in pairs]).requires_grad_(True)
    nu = torch.stack([dev(p[1]) for p in pairs]).requires_grad_(True)
    kw = dict(tol=0.0, max_iter=300)
    loss = B.w2_loss(mu, nu, **kw)
    w = torch.tensor([1.0, -0.5], dtype=torch.float64, device="cuda")
    gmu, gnu = torch.autograd.grad((loss * w).sum(), [mu, nu])
    assert gmu.shape == mu.shape and gnu.shape == nu.shape
    rng = np.random.default_rng(34)
    fd, an = [], []
    eps = 1e-4
    for _ in range(8):
        d = torch.as_tensor(rng.standard_normal(mu.shape), device="cuda") * mu.detach()
        d = d - mu.detach() * (d.sum(dim=(1, 2), keepdim=True) / mu.detach().sum(dim=(1, 2), keepdim=True))
        lp = (B.w2_loss(mu.detach() + eps * d, nu.detach(), **kw) * w).sum().item()
        lm = (B.w2_loss(mu.detach() - eps * d, nu.detach(), **kw) * w).sum().item()
        fd.append((lp - lm) / (2 * eps))
        an.append(float((gmu * d).sum().item()))
    fd, an = np.array(fd), np.array(an)
    cos = fd @ an / (np.linalg.norm(fd) * np.linalg.norm(an))
    assert cos > 0.9, (fd, an)
