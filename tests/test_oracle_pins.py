"""Pins for the FP64 oracle: what the paper and the mathematics fix.

None of these compares the oracle with itself.  Each checks it against a
closed form printed in the paper (tests/golden/paper_closed_forms.json), a
textbook/library routine (scipy's DCT, an LP solver), brute force on tiny
inputs, or an exact invariant of the method (Lemma 2.2(i), the c-transform
steps of Section 3.2, weak duality).  The mutation test in
test_oracle_mutants.py plants plausible mistakes in a copy of the oracle and
checks that the fast subset ``FAST_PINS`` catches every one.
"""
import json
import os

import numpy as np
import pytest
import scipy.fft

import oracle
import synthetic_inputs as si

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden",
                                     "paper_closed_forms.json")))


# --- c-transform: Definition 2.1, Section 4.1 -------------------------------

def pin_ct_splitting_equals_definition():
    """Dimension splitting (Section 4.1) equals the unsplit definition."""
    for shape, seed in (((5, 6), 1), ((4, 3, 5), 2), ((7, 1 + 6), 3)):
        phi = si.random_field(shape, seed, 0.05)
        full = oracle.ctransform(phi, "full")
        assert np.max(np.abs(oracle.ctransform(phi, "brute") - full)) < 1e-14
        assert np.max(np.abs(oracle.ctransform(phi, "linear") - full)) < 1e-13


def pin_ct_linear_matches_brute():
    """Legendre-transform lines (Section 4.1) equal brute force."""
    for shape, seed in (((33, 17), 4), ((9, 8, 7), 5), ((64, 3), 6)):
        for phi in (si.random_field(shape, seed, 0.1),
                    si.smooth_potential(tuple(reversed(shape)), seed)):
            d = oracle.ctransform(phi, "linear") - oracle.ctransform(phi, "brute")
            assert np.max(np.abs(d)) < 1e-13


def pin_ct_lemma22_properties():
    """Lemma 2.2(i): phi <= phi^cc and phi^ccc = phi^c (here for the grid transform)."""
    phi = si.random_field((12, 10), 7, 0.1)
    c1 = oracle.ctransform(phi, "brute")
    c2 = oracle.ctransform(c1, "brute")
    c3 = oracle.ctransform(c2, "brute")
    assert np.all(phi <= c2 + 1e-15)
    assert np.max(np.abs(c3 - c1)) < 1e-14
    assert np.max(c2 - phi) > 1e-3          # a random field is not c-concave


def pin_ct_closed_forms():
    """0^c = 0 on the grid; for phi(y) = a.y with a a whole number of cells,
    phi^c(x) = -a.x - |a|^2/2 wherever x + a is a grid point."""
    n0, n1 = 16, 12
    z = np.zeros((n1, n0))
    assert np.array_equal(oracle.ctransform(z, "brute"), z)
    a = np.array([3.0 / n0, -2.0 / n1])
    x, y = si.centres((n0, n1))
    phi = a[0] * x + a[1] * y
    got = oracle.ctransform(phi, "brute")
    want = -(a[0] * x + a[1] * y) - 0.5 * (a @ a)
    i = np.arange(n0)[None, :]
    j = np.arange(n1)[:, None]
    inside = (i + 3 < n0) & (j - 2 >= 0)
    assert np.max(np.abs((got - want)[inside])) < 1e-14
    assert np.all(got[~inside] >= want[~inside] - 1e-14)   # a minimum over fewer points


# --- DCT and Poisson: Lemma 2.3, Section 4.3 --------------------------------

def pin_dct_matches_scipy():
    """DCT-II and its inverse equal scipy's (DCT-II of scipy is twice ours)."""
    for n in (2, 3, 5, 6, 8, 12, 17, 64, 96):
        x = si.random_field((3, n), n)
        for mode in ("definition", "fft"):
            X = oracle.dct_axis(x, 0, mode=mode)
            assert np.max(np.abs(X - 0.5 * scipy.fft.dct(x, type=2, axis=1))) < 1e-12
            back = oracle.dct_axis(X, 0, inverse=True, mode=mode)
            assert np.max(np.abs(back - x)) < 1e-12
    x = si.random_field((6, 5, 4), 9)
    X = oracle.dct_axis(x, 2, mode="fft")
    assert np.max(np.abs(X - 0.5 * scipy.fft.dct(x, type=2, axis=0))) < 1e-12


def pin_poisson_inverts_neumann_laplacian():
    """-Delta_h g = f - mean f with reflected ghost cells; g has mean zero;
    G = hd sum g f equals the discrete Dirichlet energy hd sum |grad_h g|^2."""
    for shape in ((24, 20), (8, 6, 10), (96, 64)):
        f = si.random_field(shape, 11)
        g, G = oracle.poisson(f)
        lap = oracle.neg_laplacian(g)
        assert np.max(np.abs(lap - (f - f.mean()))) < 1e-9 * np.max(np.abs(f))
        assert abs(g.mean()) < 1e-12
        energy = 0.0
        for ax in range(g.ndim):
            n = g.shape[ax]
            energy += np.sum((np.diff(g, axis=ax) * n) ** 2)
        energy /= g.size
        assert abs(G - energy) < 1e-10 * energy


def pin_poisson_eigenfunction():
    """A DCT cosine is an eigenvector with eigenvalue 4 n^2 sin^2(pi k / 2n)."""
    n0, n1 = 32, 24
    x, y = si.centres((n0, n1))
    k0, k1 = 3, 5
    f = np.cos(np.pi * k0 * x) * np.cos(np.pi * k1 * y)
    lam = 4 * n0**2 * np.sin(np.pi * k0 / (2 * n0))**2 + 4 * n1**2 * np.sin(np.pi * k1 / (2 * n1))**2
    for mode in ("definition", "fft"):
        g, G = oracle.poisson(f, mode)
        assert np.max(np.abs(g - f / lam)) < 1e-14
        assert abs(G - np.mean(f * f) / lam) < 1e-14


# --- map and pushforward: Lemma 2.2(ii), Section 2.1 ------------------------

def pin_pushforward_identity_and_mass():
    mu = si.normalise(si.random_field((20, 18), 12) ** 2)
    # T = identity: each cell keeps its own mass (up to the rounding of x / h)
    assert np.max(np.abs(oracle.pushforward(np.zeros_like(mu), mu) - mu)) < 1e-13
    psi = si.smooth_potential((18, 20), 13, 0.2)
    rho = oracle.pushforward(psi, mu)
    assert abs(rho.sum() - mu.sum()) < 1e-12 * mu.sum()
    assert np.all(rho >= 0)


def pin_pushforward_translation():
    """psi(x) = -a.x with a a whole number of cells: T(x) = x + a, so T#mu is mu
    shifted by a (central differences of a linear function are exact)."""
    n0, n1 = 24, 16
    mu = np.zeros((n1, n0))
    mu[3:9, 2:10] = si.random_field((6, 8), 14) ** 2 + 0.1
    a = np.array([5.0 / n0, 4.0 / n1])
    x, y = si.centres((n0, n1))
    psi = -(a[0] * x + a[1] * y)
    rho = oracle.pushforward(psi, mu)
    want = np.zeros_like(mu)
    want[7:13, 7:15] = mu[3:9, 2:10]
    assert np.max(np.abs(rho - want)) < 1e-12
    T = oracle.transport_map(psi)
    assert np.max(np.abs(T[0][3:9, 2:10] - (x + a[0])[3:9, 2:10])) < 1e-14
    # one-sided differences at the first and last cell are exact for a linear
    # potential too: the whole map is x + a, clamped to the cell-centre box
    b = np.array([0.5 / n0, -1.5 / n1])
    T = oracle.transport_map(-(b[0] * x + b[1] * y))
    assert np.max(np.abs(T[0] - np.clip(x + b[0], 0.5 / n0, 1 - 0.5 / n0))) < 1e-14
    assert np.max(np.abs(T[1] - np.clip(y + b[1], 0.5 / n1, 1 - 0.5 / n1))) < 1e-14


def pin_map_quadratic_and_bilinear_weights():
    """psi = alpha |x|^2 / 2 gives T = (1 - alpha) x at interior cells; one cell
    of mass sent to a point between centres splits by the bilinear weights."""
    n = 16
    x, y = si.centres((n, n))
    alpha = 0.3
    T = oracle.transport_map(0.5 * alpha * (x * x + y * y))
    assert np.max(np.abs(T[0][1:-1, 1:-1] - (1 - alpha) * x[1:-1, 1:-1])) < 1e-13
    assert np.max(np.abs(T[1][1:-1, 1:-1] - (1 - alpha) * y[1:-1, 1:-1])) < 1e-13
    mu = np.zeros((n, n))
    mu[5, 4] = 1.0                                  # cell (i=4, j=5)
    # choose psi linear so that T(x_{4,5}) = centre(6,7) + (0.25 h, 0.6 h)
    h = 1.0 / n
    target = np.array([(6 + 0.5 + 0.25) * h, (7 + 0.5 + 0.6) * h])
    src = np.array([(4 + 0.5) * h, (5 + 0.5) * h])
    a = target - src
    rho = oracle.pushforward(-(a[0] * x + a[1] * y), mu)
    want = np.zeros_like(mu)
    want[7, 6] = 0.75 * 0.4
    want[7, 7] = 0.25 * 0.4
    want[8, 6] = 0.75 * 0.6
    want[8, 7] = 0.25 * 0.6
    assert np.max(np.abs(rho - want)) < 1e-12


# --- the whole method: Algorithm 1, Section 4.2, Section 4.3 ----------------

def pin_solve_translated_discs():
    """Table 1: cost 1/4; error 1e-8 after ~5 iterations at any grid size."""
    gold = GOLDEN["translated_discs_2d"]
    mu, nu = si.translated_discs(64)
    r = oracle.solve(mu, nu, tol=0.0, max_iter=9)
    err = np.abs(r["dual"] - gold["exact_cost"])
    first = lambda e: int(np.argmax(err < e)) if np.any(err < e) else 99
    assert first(1e-4) <= gold["iterations_to_error"]["1e-4"] + 2
    assert first(1e-8) <= gold["iterations_to_error"]["1e-8"] + 2
    # weak duality against the exact cost, and the primal/dual gap closes up to
    # the central differences taken at the edge cells of the disc, which read
    # psi outside the support
    assert np.all(r["dual"] <= gold["exact_cost"] + 1e-12)
    assert abs(r["w2sq"] - 2 * gold["exact_cost"]) < 1e-12      # W2^2 = 2 C
    T = r["map"]
    x, y = si.centres((64, 64))
    primal = 0.5 * np.mean(((T[0] - x) ** 2 + (T[1] - y) ** 2) * mu)
    assert abs(primal - gold["exact_cost"]) < 2e-5


def pin_solve_square_to_four():
    """Table 3: cost 1/16 (grid-aligned at 64^2, so reachable exactly)."""
    gold = GOLDEN["square_to_four_squares_2d"]
    mu, nu = si.square_to_four(64)
    r = oracle.solve(mu, nu, tol=0.0, max_iter=20)
    err = np.abs(r["dual"] - gold["exact_cost"])
    assert err.min() < 1e-6
    assert int(np.argmax(err < 1e-5)) <= gold["iterations_to_error"]["1e-5"] + 3
    assert np.all(r["dual"] <= gold["exact_cost"] + 1e-12)


def pin_gradient_ascent_baseline():
    """Section 5, Tables 5-6: the H1-dot gradient ascent on J alone (phi +=
    sigma grad J, then phi^cc) reaches the closed-form cost of the two discs
    (Table 1's 1/4) but needs many more iterations than the back-and-forth
    method (Table 5: 50 vs 3 to 1e-4).  Its first gradient step is Algorithm
    1's first phi-half step (same phi_0, same gradient), so J(phi_{1/2})
    agrees exactly."""
    gold = GOLDEN["translated_discs_2d"]
    mu, nu = si.translated_discs(64)
    ga = oracle.solve(mu, nu, tol=0.0, max_iter=120, method="ga")
    bf = oracle.solve(mu, nu, tol=0.0, max_iter=10)
    first = lambda r, e: int(np.argmax(np.abs(r["dual"] - gold["exact_cost"]) < e)) \
        if np.any(np.abs(r["dual"] - gold["exact_cost"]) < e) else 10 ** 6
    assert first(ga, 1e-6) < 120                       # converges to the exact cost
    assert first(ga, 1e-4) >= 4 * first(bf, 1e-4)
    assert ga["half"][0, 0] == bf["half"][0, 0]
    assert np.all(ga["dual"] <= gold["exact_cost"] + 1e-12)   # weak duality


# --- separable power costs (Section 5, eq. p_costs) ------------------------------

def pin_power_cost_definition_and_p2():
    """The power-cost c-transform by dimension splitting equals the minimum of
    sum_a |x_a - y_a|^{p_a}/p_a - phi(y) over every grid point y (brute force
    on a tiny grid, no splitting); p = (2, 2) reproduces the quadratic
    c-transform and solve."""
    shape = (5, 6)                       # (n1, n0)
    phi = si.random_field(shape, 21, 0.2)
    p = (1.3, 2.7)
    x, y = si.centres((6, 5))
    X, Y = x.ravel(), y.ravel()
    cost = (np.abs(X[:, None] - X[None, :]) ** p[0] / p[0] +
            np.abs(Y[:, None] - Y[None, :]) ** p[1] / p[1])
    want = np.min(cost - phi.ravel()[None, :], axis=1).reshape(shape)
    assert np.max(np.abs(oracle.ctransform_p(phi, p) - want)) < 1e-14
    phi2 = si.random_field((20, 24), 22, 0.1)
    assert np.max(np.abs(oracle.ctransform_p(phi2, (2.0, 2.0)) - oracle.ctransform(phi2))) < 1e-14
    mu, nu = si.translated_discs(32)
    a = oracle.solve(mu, nu, tol=0.0, max_iter=5)
    b = oracle.solve(mu, nu, tol=0.0, max_iter=5, p=(2.0, 2.0))
    assert np.max(np.abs(a["dual"] - b["dual"])) < 1e-14


def pin_power_cost_translation():
    """A translation by a is optimal for any strictly convex cost h(y - x):
    the two discs of Table 1 cost h((1/2, 1/2)) = sum_a (1/2)^{p_a} / p_a, and
    the map moves mu's cells by a."""
    mu, nu = si.translated_discs(48)
    p = (1.5, 2.5)
    exact = 0.5 ** p[0] / p[0] + 0.5 ** p[1] / p[1]
    r = oracle.solve(mu, nu, tol=0.0, max_iter=15, p=p)
    assert abs(r["dual"][-1] - exact) < 1e-10
    assert np.all(r["dual"] <= exact + 1e-12)
    x, y = si.centres((48, 48))
    m = mu > 0
    inner = m & (np.hypot(x - 0.25, y - 0.25) < 0.125 - 2.0 / 48)   # away from the edge cells
    assert np.max(np.abs(r["map"][0][inner] - x[inner] - 0.5)) < 1.0 / 48
    assert np.max(np.abs(r["map"][1][inner] - y[inner] - 0.5)) < 1.0 / 48


def pin_power_cost_direction_of_transport():
    """Section 5's two-disc example: with p = (2, 2) each disc of mu splits
    evenly between the two discs of nu; with p = (1.1, 3) horizontal moves
    are so expensive that all mass moves vertically by 1/2, at cost
    (1/2)^3 / 3 = 1/24."""
    mu, nu = si.diagonal_to_antidiagonal_discs(48)
    x, y = si.centres((48, 48))
    m = mu > 0
    def vertical(p):
        r = oracle.solve(mu, nu, tol=0.0, max_iter=30, p=p)
        dx, dy = r["map"][0] - x, r["map"][1] - y
        return np.sum(mu[m] * (np.abs(dy[m]) > np.abs(dx[m]))) / np.sum(mu[m]), r
    v2, _ = vertical((2.0, 2.0))
    assert abs(v2 - 0.5) < 0.05
    v, r = vertical((1.1, 3.0))
    assert v > 0.99
    assert abs(r["dual"][-1] - 1.0 / 24.0) < 1e-8


def pin_solve_chain_invariants():
    """Section 3.2: a c-transform never lowers the dual value, so
    J(phi_{n+1/2}) <= I(psi_{n+1/2}) and I(psi_{n+1}) <= J(phi_{n+1})."""
    mu, nu = si.workload_gauss_disc_64(32)
    r = oracle.solve(mu, nu, tol=0.0, max_iter=25)
    h, d = r["half"], r["dual"]
    assert np.all(h[:, 0] <= h[:, 1] + 1e-14)
    assert np.all(h[:, 2] <= d[1:] + 1e-14)
    assert d[-1] > d[1] > 0


def pin_solve_weak_duality_lp():
    """J(phi_n) never exceeds the discrete transport cost between the grid
    measures (an LP solved by scipy's HiGHS)."""
    from scipy.optimize import linprog
    n = 6
    rng = np.random.default_rng(15)
    mu = si.normalise(rng.uniform(0.2, 1.0, (n, n)))
    nu = si.normalise(rng.uniform(0.0, 1.0, (n, n)) ** 2)
    x, y = si.centres((n, n))
    P = np.stack([x.ravel(), y.ravel()], 1)
    C = 0.5 * ((P[:, None, :] - P[None, :, :]) ** 2).sum(-1)
    a = mu.ravel() / mu.size
    b = nu.ravel() / nu.size
    N = n * n
    A = np.zeros((2 * N, N * N))
    for i in range(N):
        A[i, i * N:(i + 1) * N] = 1.0
        A[N + i, i::N] = 1.0
    lp = linprog(C.ravel(), A_eq=A, b_eq=np.concatenate([a, b]), bounds=(0, None),
                 method="highs")
    assert lp.status == 0
    r = oracle.solve(mu, nu, tol=0.0, max_iter=30, ct_mode="brute", dct_mode="definition")
    assert np.all(r["dual"] <= lp.fun + 1e-12)
    assert r["dual"].max() > 0.9 * lp.fun


def pin_solve_monotone_rearrangement():
    """Densities constant along y: the map is the 1-D monotone rearrangement.
    mu uniform on [1/4,1/2], nu uniform on [1/4,3/4]: T(x) = 1/4 + 2(x-1/4),
    W2^2 = int_{1/4}^{1/2} 4 (x-1/4)^2 dx = 1/48."""
    errs = []
    for n in (32, 64):
        x, _ = si.centres((n, 8))
        mu = si.normalise(((x > 0.25) & (x < 0.5)).astype(float))
        nu = si.normalise(((x > 0.25) & (x < 0.75)).astype(float))
        r = oracle.solve(mu, nu, tol=0.0, max_iter=40)
        errs.append(abs(r["w2sq"] - 1.0 / 48))
        assert np.max(np.abs(r["map"][1] - si.centres((n, 8))[1])) < 1e-9
    assert errs[1] < 2e-3 / 48 and errs[1] < errs[0]


def pin_solve_gaussians_bures():
    """Gaussian -> Gaussian: W2^2 = |m1-m2|^2 + sum_a (s1_a - s2_a)^2 (diagonal
    covariances).  Within 1% at 32^2 and 48^2 (the rest is discretisation and
    the slow tail of the iteration once the step size reaches sigma_min)."""
    m1, m2 = np.array([0.4, 0.45]), np.array([0.58, 0.55])
    s1, s2 = np.array([0.06, 0.05]), np.array([0.05, 0.08])
    exact = np.sum((m1 - m2) ** 2) + np.sum((s1 - s2) ** 2)
    for n in (32, 48):
        mu = si.normalise(si.gaussian_mixture((n, n), [m1], [s1]))
        nu = si.normalise(si.gaussian_mixture((n, n), [m2], [s2]))
        r = oracle.solve(mu, nu, tol=0.0, max_iter=150)
        assert abs(r["w2sq"] - exact) < 0.01 * exact
        # the map moves the mean: the mean of T under mu is m2
        T = r["map"]
        mean_T = np.array([np.mean(T[0] * mu), np.mean(T[1] * mu)])
        assert np.max(np.abs(mean_T - m2)) < 2.0 / n


def pin_interpolate_translation():
    """Displacement interpolation (Section 4.3) along the exact translation
    T(x) = x + (1/2, 1/2) of the translated discs: t=0 gives mu, t=1 gives nu,
    t=1/2 the disc halfway (all grid-aligned at 64^2)."""
    n = 64
    mu, nu = si.translated_discs(n)
    x, y = si.centres((n, n))
    T = np.stack([np.minimum(x + 0.5, 1 - 0.5 / n), np.minimum(y + 0.5, 1 - 0.5 / n)])
    assert np.max(np.abs(oracle.interpolate(T, mu, 0.0) - mu)) < 1e-12
    assert np.max(np.abs(oracle.interpolate(T, mu, 1.0) - nu)) < 1e-12
    mid = si.normalise(si.ball((n, n), (0.5, 0.5), 0.125))
    assert np.max(np.abs(oracle.interpolate(T, mu, 0.5) - mid)) < 1e-12


def pin_step_rule_constants():
    """Section 4.2: the first step is 8 min(1/|mu|inf, 1/|nu|inf)."""
    mu, nu = si.translated_discs(32)
    r = oracle.solve(mu, nu, tol=0.0, max_iter=1)
    assert abs(r["sigma"][0] - 8.0 / max(mu.max(), nu.max())) < 1e-15


def _first_steps(**opts):
    mu, nu = si.translated_discs(32)
    s0 = 8.0 / max(mu.max(), nu.max())
    return s0, oracle.solve(mu, nu, tol=0.0, max_iter=6, **{k: (v * s0 if k == "sigma0" else v)
                                                             for k, v in opts.items()})


def pin_step_rule_shrinks_on_overshoot():
    """Section 4.2: a step far too long loses dual value (the gain is below
    beta1 sigma G), so every half step multiplies sigma by alpha2 = 4/5: 0.64
    per iteration until the step fits."""
    _, r = _first_steps(sigma0=1000.0)
    ratio = r["sigma"][1:] / r["sigma"][:-1]
    assert np.all(np.abs(ratio - 0.64) < 1e-14), ratio


def pin_step_rule_grows_on_short_step():
    """Section 4.2: for a short step the dual value rises by about sigma G
    (first order in sigma, Lemma 2.3's gradient), above beta2 sigma G = 3/4
    sigma G, so every half step multiplies sigma by alpha1 = 5/4: 25/16 per
    iteration."""
    _, r = _first_steps(sigma0=1e-3)
    ratio = r["sigma"][1:] / r["sigma"][:-1]
    assert np.all(np.abs(ratio - 1.5625) < 1e-14), ratio


def pin_step_rule_floor():
    """Section 4.2: decreases never take sigma below sigma_min.  With
    sigma_min set far above the stable step, sigma falls by 0.64 per
    iteration from 50 and then stays at sigma_min exactly."""
    mu, nu = si.translated_discs(32)
    r = oracle.solve(mu, nu, tol=0.0, max_iter=14, sigma0=50.0, sigma_min=1.0)
    s = r["sigma"]
    assert s.min() == 1.0 and np.all(s[-4:] == 1.0), s
    k = int(np.argmax(s == 1.0))
    assert np.all(np.abs(s[1:k] / s[:k - 1] - 0.64) < 1e-14), s


def pin_step_rule_window():
    """Section 4.2: a gain between beta1 sigma G and beta2 sigma G keeps sigma.
    On the paper's two discs from the paper's sigma_0 some iteration changes
    sigma by exactly one factor alpha2 (one half step shrinks, the other is
    kept), and once sigma has settled it is kept for whole iterations."""
    mu, nu = si.translated_discs(32)
    r = oracle.solve(mu, nu, tol=0.0, max_iter=30)
    ratio = r["sigma"][1:] / r["sigma"][:-1]
    assert np.any(np.abs(ratio - 0.8) < 1e-14), ratio
    assert np.all(ratio[-10:] == 1.0), ratio


def pin_residual_uniform_target():
    """A uniform target has ||nu - 1||_{H^-1} = 0, so the residual is the
    absolute H^-1 norm of nu - T#mu there (reading of the stopping norm).  At
    phi_0 = 0 the map is the identity and T#mu = mu, so r_0 = ||1 -
    mu||_{H^-1} = sqrt(hd sum_k c_k^2 / lambda_k) with c the orthonormal
    DCT-II of 1 - mu (scipy) and lambda_k the Neumann eigenvalues."""
    rng = np.random.default_rng(3)
    mu = si.normalise(si.gaussian_mixture((24, 20), rng.uniform(0.3, 0.7, (2, 2)), [0.12, 0.1]))
    nu = np.ones_like(mu)
    r = oracle.solve(mu, nu, tol=0.0, max_iter=4)
    f = 1.0 - mu
    c = scipy.fft.dctn(f, type=2, norm="ortho")
    n1, n0 = f.shape
    k1 = np.arange(n1)[:, None]
    k0 = np.arange(n0)[None, :]
    lam = 4 * n0**2 * np.sin(np.pi * k0 / (2 * n0))**2 + 4 * n1**2 * np.sin(np.pi * k1 / (2 * n1))**2
    lam[0, 0] = np.inf
    want = np.sqrt(np.sum(c**2 / lam) / f.size)
    assert abs(r["resid"][0] - want) < 1e-13 * want
    assert np.all(np.isfinite(r["resid"])) and r["resid"][-1] < 0.5 * r["resid"][0]


FAST_PINS = [
    pin_ct_splitting_equals_definition, pin_ct_linear_matches_brute,
    pin_ct_lemma22_properties, pin_ct_closed_forms, pin_dct_matches_scipy,
    pin_poisson_inverts_neumann_laplacian, pin_poisson_eigenfunction,
    pin_pushforward_identity_and_mass, pin_pushforward_translation,
    pin_map_quadratic_and_bilinear_weights, pin_solve_translated_discs,
    pin_solve_chain_invariants, pin_step_rule_constants, pin_interpolate_translation,
    pin_step_rule_shrinks_on_overshoot, pin_step_rule_grows_on_short_step,
    pin_step_rule_floor, pin_step_rule_window, pin_residual_uniform_target,
]
ALL_PINS = FAST_PINS + [pin_solve_square_to_four, pin_gradient_ascent_baseline,
                        pin_power_cost_definition_and_p2, pin_power_cost_translation,
                        pin_power_cost_direction_of_transport,
                        pin_solve_weak_duality_lp,
                        pin_solve_monotone_rearrangement, pin_solve_gaussians_bures]


@pytest.mark.parametrize("pin", ALL_PINS, ids=lambda f: f.__name__)
def test_pin(pin):
    pin()


def _lp_cost(mu, nu):
    """Discrete transport cost between the grid measures (scipy HiGHS LP) and
    the dual marginals of the source / target constraints."""
    from scipy.optimize import linprog
    n1, n0 = mu.shape
    x, y = si.centres((n0, n1))
    P = np.stack([x.ravel(), y.ravel()], 1)
    C = 0.5 * ((P[:, None, :] - P[None, :, :]) ** 2).sum(-1)
    N = mu.size
    A = np.zeros((2 * N, N * N))
    for i in range(N):
        A[i, i * N:(i + 1) * N] = 1.0
        A[N + i, i::N] = 1.0
    lp = linprog(C.ravel(), A_eq=A, b_eq=np.concatenate([mu.ravel(), nu.ravel()]) / N,
                 bounds=(0, None), method="highs")
    assert lp.status == 0
    m = lp.eqlin.marginals
    return lp.fun, m[N:].reshape(mu.shape), m[:N].reshape(mu.shape)


def test_w2_gradient_formula_against_lp():
    """dW2^2/dmu = 2 hd (psi - mean psi) on mass-preserving perturbations:
    psi here is the LP's exact dual potential and the derivative is taken by
    central differences of the exact LP value, so the check pins the
    formula's factors (W2^2 = 2C, the cell-volume weight hd, the mean-zero
    projection) independently of the iteration."""
    rng = np.random.default_rng(17)
    n = 5
    mu = si.normalise(rng.uniform(0.3, 1.0, (n, n)))
    nu = si.normalise(rng.uniform(0.3, 1.0, (n, n)))
    c0, phi_lp, psi_lp = _lp_cost(mu, nu)
    gmu, gnu = oracle.w2_gradient(phi_lp, psi_lp)
    eps = 1e-6
    for _ in range(3):
        d = rng.standard_normal(mu.shape)
        d -= d.mean()
        fd_mu = (2 * _lp_cost(mu + eps * d, nu)[0] - 2 * _lp_cost(mu - eps * d, nu)[0]) / (2 * eps)
        fd_nu = (2 * _lp_cost(mu, nu + eps * d)[0] - 2 * _lp_cost(mu, nu - eps * d)[0]) / (2 * eps)
        assert abs(fd_mu - np.sum(gmu * d)) < 1e-6 * (1 + abs(fd_mu))
        assert abs(fd_nu - np.sum(gnu * d)) < 1e-6 * (1 + abs(fd_nu))
