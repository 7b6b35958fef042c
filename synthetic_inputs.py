"""Seeded synthetic densities on cell-centred grids over [0,1]^d.

The one module shared by the CUDA path's tests/benchmark and the FP64 oracle.
It builds input densities only and holds none of the method's arithmetic.

Layout: a d-dim field is a C-order numpy array of shape (n1, n0) in 2D or
(n2, n1, n0) in 3D, axis 0 (x) fastest; cell i on an axis of n cells has its
centre at (i + 1/2)/n.  Every generator returns float64 density values
normalised to unit integral: sum(rho) / N = 1.

Workloads (each seeded with numpy.random.default_rng(12154 + k), draws in the
order written):
  workload_gauss_disc_64     3 isotropic Gaussians -> disc, 64x64
  workload_annulus_5g_4096   annulus -> 5 truncated Gaussians, 4096x4096
  workload_ball_4g_384       ball -> 4 anisotropic Gaussians, 384^3
  workload_batched_uneven    128 problems, sides in {64,128,256,512}
  workload_loss_pairs_256    32 pairs of Gaussian mixtures, 256x256
and the closed-form shapes of the paper's Section 4.3 (translated discs and
balls, one square to four squares, one cube to eight cubes) and the two-disc
pair of its power-cost experiment (Section 5).
"""
from __future__ import annotations

import numpy as np


def centres(shape_xyz):
    """Cell-centre coordinate arrays (x, y[, z]) broadcast to the C-order field."""
    nd = len(shape_xyz)
    axes = [(np.arange(n) + 0.5) / n for n in shape_xyz]
    # C-order field shape is reversed (slowest axis first)
    mesh = np.meshgrid(*reversed(axes), indexing="ij")
    return list(reversed(mesh))[:nd]


def normalise(rho):
    rho = np.asarray(rho, dtype=np.float64)
    m = rho.mean()
    if not m > 0:
        raise ValueError("density has no mass on the grid")
    return rho / m


def gaussian_mixture(shape_xyz, means, sigmas, weights=None):
    """Sum of normalised Gaussian pdfs; sigmas is (k,) isotropic or (k, d)."""
    xs = centres(shape_xyz)
    nd = len(shape_xyz)
    means = np.atleast_2d(np.asarray(means, dtype=np.float64))
    sig = np.asarray(sigmas, dtype=np.float64)
    if sig.ndim == 1:
        sig = np.repeat(sig[:, None], nd, axis=1)
    k = means.shape[0]
    w = np.ones(k) / k if weights is None else np.asarray(weights, dtype=np.float64)
    out = np.zeros(xs[0].shape)
    for c in range(k):
        e = np.zeros_like(out)
        norm = 1.0
        for a in range(nd):
            e += ((xs[a] - means[c, a]) / sig[c, a]) ** 2
            norm *= np.sqrt(2 * np.pi) * sig[c, a]
        out += w[c] * np.exp(-0.5 * e) / norm
    return out


def ball(shape_xyz, centre, radius):
    """Indicator of cells whose centre lies within ``radius`` of ``centre``."""
    xs = centres(shape_xyz)
    r2 = sum((xs[a] - centre[a]) ** 2 for a in range(len(shape_xyz)))
    return (r2 <= radius * radius).astype(np.float64)


def annulus(shape_xyz, centre, r_in, r_out):
    xs = centres(shape_xyz)
    r2 = sum((xs[a] - centre[a]) ** 2 for a in range(len(shape_xyz)))
    return ((r2 >= r_in * r_in) & (r2 <= r_out * r_out)).astype(np.float64)


def box(shape_xyz, centre, side):
    """Indicator of cells whose centre lies in the axis-aligned cube."""
    xs = centres(shape_xyz)
    m = np.ones(xs[0].shape, dtype=bool)
    for a in range(len(shape_xyz)):
        m &= np.abs(xs[a] - centre[a]) <= side / 2
    return m.astype(np.float64)


# --- the paper's closed-form shapes (Section 4.3) ---------------------------

def translated_discs(n):
    """Disc r=1/8 at (1/4,1/4) -> the same disc at (3/4,3/4); cost 1/4."""
    mu = ball((n, n), (0.25, 0.25), 0.125)
    nu = ball((n, n), (0.75, 0.75), 0.125)
    return normalise(mu), normalise(nu)


def translated_balls(n):
    """Ball r=1/8 at (1/4,1/4,1/4) -> (3/4,3/4,3/4); cost 3/8."""
    mu = ball((n, n, n), (0.25,) * 3, 0.125)
    nu = ball((n, n, n), (0.75,) * 3, 0.125)
    return normalise(mu), normalise(nu)


def square_to_four(n):
    """Square side 1/4 at the centre -> four squares side 1/8 at
    (3/16 + 5i/8, 3/16 + 5j/8); cost 1/16."""
    mu = box((n, n), (0.5, 0.5), 0.25)
    nu = np.zeros_like(mu)
    for i in (0, 1):
        for j in (0, 1):
            nu += box((n, n), (3 / 16 + 5 * i / 8, 3 / 16 + 5 * j / 8), 0.125)
    return normalise(mu), normalise(nu)


def cube_to_eight(n):
    """Cube side 1/4 at the centre -> eight cubes side 1/8; cost 3/32."""
    mu = box((n, n, n), (0.5,) * 3, 0.25)
    nu = np.zeros_like(mu)
    for i in (0, 1):
        for j in (0, 1):
            for k in (0, 1):
                c = (3 / 16 + 5 * i / 8, 3 / 16 + 5 * j / 8, 3 / 16 + 5 * k / 8)
                nu += box((n, n, n), c, 0.125)
    return normalise(mu), normalise(nu)


def diagonal_to_antidiagonal_discs(n):
    """Section 5, separable power costs: discs r=1/8 at (1/4,1/4) and (3/4,3/4)
    -> discs r=1/8 at (1/4,3/4) and (3/4,1/4)."""
    mu = ball((n, n), (0.25, 0.25), 0.125) + ball((n, n), (0.75, 0.75), 0.125)
    nu = ball((n, n), (0.25, 0.75), 0.125) + ball((n, n), (0.75, 0.25), 0.125)
    return normalise(mu), normalise(nu)


# --- the benchmark workloads -------------------------------------------------

def workload_gauss_disc_64(n=64):
    """mu: 3 isotropic Gaussians (centres U[0.2,0.8]^2, sigma U[0.05,0.15],
    equal weights); nu: disc r=0.3 at (0.5,0.5).  Seed 12154+1."""
    rng = np.random.default_rng(12154 + 1)
    means = rng.uniform(0.2, 0.8, size=(3, 2))
    sig = rng.uniform(0.05, 0.15, size=3)
    mu = gaussian_mixture((n, n), means, sig)
    nu = ball((n, n), (0.5, 0.5), 0.3)
    return normalise(mu), normalise(nu)


def workload_annulus_5g_4096(n=4096):
    """mu: uniform annulus r in [0.15,0.35] at (0.3,0.5); nu: 5 Gaussians
    (centres U[0.5,0.9] x U[0.1,0.9], sigma U[0.02,0.08], equal weights)
    truncated to zero below 1e-3 * max.  Seed 12154+2."""
    rng = np.random.default_rng(12154 + 2)
    cx = rng.uniform(0.5, 0.9, size=5)
    cy = rng.uniform(0.1, 0.9, size=5)
    sig = rng.uniform(0.02, 0.08, size=5)
    mu = annulus((n, n), (0.3, 0.5), 0.15, 0.35)
    nu = gaussian_mixture((n, n), np.stack([cx, cy], 1), sig)
    nu[nu < 1e-3 * nu.max()] = 0.0
    return normalise(mu), normalise(nu)


def workload_ball_4g_384(n=384):
    """mu: ball r=0.25 at (0.3,0.3,0.3); nu: 4 anisotropic Gaussians (means
    U[0.4,0.8]^3, diagonal sigma U[0.03,0.1]).  Seed 12154+3."""
    rng = np.random.default_rng(12154 + 3)
    means = rng.uniform(0.4, 0.8, size=(4, 3))
    sig = rng.uniform(0.03, 0.1, size=(4, 3))
    mu = ball((n, n, n), (0.3, 0.3, 0.3), 0.25)
    nu = gaussian_mixture((n, n, n), means, sig)
    return normalise(mu), normalise(nu)


def _masked_mixture(rng, n):
    k = int(rng.integers(1, 7))
    means = rng.uniform(0.15, 0.85, size=(k, 2))
    sig = rng.uniform(0.02, 0.15, size=k)
    rho = gaussian_mixture((n, n), means, sig)
    frac = rng.uniform(0.0, 0.4)
    if frac > 0:
        thr = np.quantile(rho, frac)
        rho = np.where(rho <= thr, 0.0, rho)
    return normalise(rho)


def workload_batched_uneven(count=128, sides=(64, 128, 256, 512)):
    """``count`` independent 2D problems; side drawn from ``sides``; mu and nu
    each a mixture of 1-6 Gaussians (sigma U[0.02,0.15]) with the lowest
    0-40% of cells zeroed by a threshold.  Seed 12154+4."""
    rng = np.random.default_rng(12154 + 4)
    out = []
    for _ in range(count):
        n = int(rng.choice(sides))
        mu = _masked_mixture(rng, n)
        nu = _masked_mixture(rng, n)
        out.append((mu, nu))
    return out


def workload_loss_pairs_256(count=32, n=256):
    """``count`` pairs of 2-4 component Gaussian mixtures (sigma U[0.04,0.12])
    on n x n.  Seed 12154+5."""
    rng = np.random.default_rng(12154 + 5)
    out = []
    for _ in range(count):
        pair = []
        for _ in range(2):
            k = int(rng.integers(2, 5))
            means = rng.uniform(0.25, 0.75, size=(k, 2))
            sig = rng.uniform(0.04, 0.12, size=k)
            pair.append(normalise(gaussian_mixture((n, n), means, sig)))
        out.append(tuple(pair))
    return out


def random_field(shape, seed, scale=1.0):
    """Seeded standard-normal field (c-transform / DCT parity inputs)."""
    return scale * np.random.default_rng(seed).standard_normal(shape)


def quadratic_potential(shape_xyz, seed):
    """phi(x) = |x|^2/2 - a.x with a seeded a in [0.2, 0.8]^d: along every grid
    line |x|^2/2 - phi is affine, so all the line's lifted points lie on one
    line (up to the rounding of phi) -- the degenerate case of the lower
    envelope, where many parabolas meet at nearly one point."""
    rng = np.random.default_rng(seed)
    xs = centres(shape_xyz)
    a = rng.uniform(0.2, 0.8, size=len(shape_xyz))
    return sum(0.5 * xs[k] ** 2 - a[k] * xs[k] for k in range(len(shape_xyz)))


def smooth_potential(shape_xyz, seed, amp=0.05):
    """A smooth random potential (sum of a few cosines) of small amplitude,
    the kind of field the method's iterates are."""
    rng = np.random.default_rng(seed)
    xs = centres(shape_xyz)
    out = np.zeros(xs[0].shape)
    for _ in range(6):
        k = rng.integers(0, 4, size=len(shape_xyz))
        ph = rng.uniform(0, 2 * np.pi)
        arg = sum(np.pi * k[a] * xs[a] for a in range(len(shape_xyz)))
        out += rng.uniform(-amp, amp) * np.cos(arg + ph)
    return out
