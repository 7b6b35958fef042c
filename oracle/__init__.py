"""FP64 CPU oracle for the back-and-forth method -- TEST INFRASTRUCTURE.

This package is the plain, slow, obviously-correct restatement of the method
of Jacobs & Leger (arXiv 1905.12154) that the CUDA library is checked against.
Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline /
reference arm may import it.  It shares no code with the CUDA path; the two
meet only in the seeded input generators of ``synthetic_inputs``.

Every array is numpy float64 in the grid layout of the C source: a d-dim field
is stored with axis 0 fastest, so a numpy array of shape ``(n2, n1, n0)`` (3D)
or ``(n1, n0)`` (2D) in C order, and ``grid`` is given as ``(n0, n1[, n2])``.

Functions and the passage each follows:
  ctransform          Definition 2.1, Section 4.1 (splitting; brute / Legendre lines)
  ctransform_full     Definition 2.1 with no splitting (tiny grids)
  dct_axis            Section 4.3 "using the FFT" (DCT-II and its inverse)
  poisson             Lemma 2.3, eq. (gradients_J_I), eq. (defHm1dot)
  neg_laplacian       the discrete Neumann Laplacian the Poisson solve inverts
  transport_map       Lemma 2.2(ii)
  pushforward         Section 2.1 pushforward, Lemma 3.1
  ctransform_p        the c-transform of a separable power cost (Section 5)
  solve               Algorithm 1 with the step rule of Section 4.2 (quadratic
                      or separable power cost; or the gradient-ascent baseline)
  interpolate         displacement interpolation, Section 4.3
  w2_gradient         envelope theorem on eq. (symmetric_dual)
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bfm_oracle.c")
_LIB_PATH = os.path.join(_HERE, "libbfm_oracle.so")
_lock = threading.Lock()
_lib = None

_DP = ctypes.POINTER(ctypes.c_double)
_IP = ctypes.POINTER(ctypes.c_int)


def build(force: bool = False) -> str:
    """Compile the C oracle into ``oracle/libbfm_oracle.so`` (gcc, OpenMP)."""
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
           "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _configure(lib):
    """Declare the C signatures on a loaded oracle library."""
    lib.bfm_oracle_ctransform.argtypes = [_DP, _DP, ctypes.c_int, _IP, ctypes.c_int]
    lib.bfm_oracle_ctransform_full.argtypes = [_DP, _DP, ctypes.c_int, _IP]
    lib.bfm_oracle_dct_axis.argtypes = [_DP, ctypes.c_int, _IP, ctypes.c_int,
                                        ctypes.c_int, ctypes.c_int]
    lib.bfm_oracle_poisson.argtypes = [_DP, _DP, ctypes.c_int, _IP, ctypes.c_int, _DP]
    lib.bfm_oracle_neg_laplacian.argtypes = [_DP, _DP, ctypes.c_int, _IP]
    lib.bfm_oracle_map.argtypes = [_DP, _DP, ctypes.c_int, _IP]
    lib.bfm_oracle_pushforward.argtypes = [_DP, _DP, _DP, ctypes.c_int, _IP]
    lib.bfm_oracle_ctransform_p.argtypes = [_DP, _DP, ctypes.c_int, _IP, _DP]
    lib.bfm_oracle_map_p.argtypes = [_DP, _DP, ctypes.c_int, _IP, _DP]
    lib.bfm_oracle_pushforward_p.argtypes = [_DP, _DP, _DP, ctypes.c_int, _IP, _DP]
    lib.bfm_oracle_solve.argtypes = [_DP, _DP, ctypes.c_int, _IP, ctypes.c_double,
                                     ctypes.c_int, _DP, _DP, _DP, _DP, _DP, _DP,
                                     _DP, _DP, _DP]
    lib.bfm_oracle_interpolate.argtypes = [_DP, _DP, ctypes.c_double, _DP,
                                           ctypes.c_int, _IP]
    lib.bfm_oracle_omp_threads.restype = ctypes.c_int
    return lib


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            _lib = _configure(ctypes.CDLL(_LIB_PATH))
    return _lib


def use_library(path: str | None):
    """Point this module at another build of the oracle source (the mutation
    tests load deliberately broken copies); None restores the default."""
    global _lib
    with _lock:
        _lib = None if path is None else _configure(ctypes.CDLL(path))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(_DP)


def _grid(shape) -> tuple[int, ctypes.Array]:
    """numpy C-order shape (.., n1, n0) -> (ndim, int[3] of n0, n1, n2)."""
    n = list(reversed(shape))
    arr = (ctypes.c_int * 3)(*(n + [1] * (3 - len(n))))
    return len(n), arr


def threads() -> int:
    """OpenMP threads the oracle's parallel loops use."""
    return _load().bfm_oracle_omp_threads()


def ctransform(phi, mode: str = "brute") -> np.ndarray:
    """phi^c on the grid (Definition 2.1) by dimension splitting (Section 4.1).

    mode: "brute" (O(n^2) per line), "linear" (Legendre transform through the
    lower convex hull, O(n) per line) or "full" (no splitting, O(N^2))."""
    phi = _f64(phi)
    out = np.empty_like(phi)
    nd, n = _grid(phi.shape)
    lib = _load()
    if mode == "full":
        rc = lib.bfm_oracle_ctransform_full(_ptr(phi), _ptr(out), nd, n)
    else:
        rc = lib.bfm_oracle_ctransform(_ptr(phi), _ptr(out), nd, n,
                                       {"brute": 0, "linear": 1}[mode])
    assert rc == 0
    return out


def dct_axis(x, axis: int, inverse: bool = False, mode: str = "definition") -> np.ndarray:
    """DCT-II (or its exact inverse) along grid axis ``axis`` (0 = fastest)."""
    w = _f64(x).copy()
    nd, n = _grid(w.shape)
    rc = _load().bfm_oracle_dct_axis(_ptr(w), nd, n, axis, 1 if inverse else 0,
                                     {"definition": 0, "fft": 1}[mode])
    assert rc == 0
    return w


def poisson(f, mode: str = "fft") -> tuple[np.ndarray, float]:
    """g = (-Delta)^{-1}(f - mean f) with zero Neumann conditions, and
    G = hd * sum g (f - mean f) = ||f - mean f||^2_{H^-1}."""
    f = _f64(f)
    g = np.empty_like(f)
    G = ctypes.c_double(0.0)
    nd, n = _grid(f.shape)
    rc = _load().bfm_oracle_poisson(_ptr(f), _ptr(g), nd, n,
                                    {"definition": 0, "fft": 1}[mode], ctypes.byref(G))
    assert rc == 0
    return g, G.value


def neg_laplacian(u) -> np.ndarray:
    u = _f64(u)
    out = np.empty_like(u)
    nd, n = _grid(u.shape)
    assert _load().bfm_oracle_neg_laplacian(_ptr(u), _ptr(out), nd, n) == 0
    return out


def _exponents(p, nd):
    """Per-axis exponents of the separable power cost as a double[3] (axis 0 first)."""
    q = [float(x) for x in p] + [2.0] * (3 - len(p))
    assert len(p) == nd and all(x > 1.0 for x in p)
    return np.array(q, dtype=np.float64)


def ctransform_p(phi, p) -> np.ndarray:
    """phi^c for the separable power cost sum_a |y_a - x_a|^{p_a}/p_a (Section 5,
    eq. p_costs), by dimension splitting with brute-force lines; p lists the
    exponents from axis 0 (x) on."""
    phi = _f64(phi)
    out = np.empty_like(phi)
    nd, n = _grid(phi.shape)
    pe = _exponents(p, nd)
    assert _load().bfm_oracle_ctransform_p(_ptr(phi), _ptr(out), nd, n, _ptr(pe)) == 0
    return out


def transport_map(psi, p=None) -> np.ndarray:
    """T(x) = x - (grad h)^{-1}(grad psi(x)) (the identity for the quadratic
    cost, sign(w)|w|^{1/(p_a-1)} per axis for a power cost), clamped to the box
    of cell centres; shape (d, *grid)."""
    psi = _f64(psi)
    nd, n = _grid(psi.shape)
    out = np.empty((nd,) + psi.shape)
    if p is None:
        assert _load().bfm_oracle_map(_ptr(psi), _ptr(out), nd, n) == 0
    else:
        pe = _exponents(p, nd)
        assert _load().bfm_oracle_map_p(_ptr(psi), _ptr(out), nd, n, _ptr(pe)) == 0
    return out


def pushforward(psi, mu, p=None) -> np.ndarray:
    """rho = T#mu with the map above and a multilinear deposit (density values)."""
    psi, mu = _f64(psi), _f64(mu)
    rho = np.empty_like(mu)
    nd, n = _grid(mu.shape)
    if p is None:
        assert _load().bfm_oracle_pushforward(_ptr(psi), _ptr(mu), _ptr(rho), nd, n) == 0
    else:
        pe = _exponents(p, nd)
        assert _load().bfm_oracle_pushforward_p(_ptr(psi), _ptr(mu), _ptr(rho), nd, n,
                                                _ptr(pe)) == 0
    return rho


def interpolate(tmap, mu, t: float) -> np.ndarray:
    """Displacement interpolation rho_t = ((1-t) x + t T)#mu."""
    tmap, mu = _f64(tmap), _f64(mu)
    rho = np.empty_like(mu)
    nd, n = _grid(mu.shape)
    assert _load().bfm_oracle_interpolate(_ptr(tmap), _ptr(mu), float(t), _ptr(rho), nd, n) == 0
    return rho


DEFAULTS = dict(beta1=0.25, beta2=0.75, alpha1=1.25, alpha2=0.8, sigma0=0.0,
                sigma_min=0.01)


def solve(mu, nu, tol: float = 1e-6, max_iter: int = 300, ct_mode: str = "linear",
          dct_mode: str = "fft", method: str = "bfm", p=None, **opts) -> dict:
    """Algorithm 1 with the step rule of Section 4.2, in FP64 (method "bfm"),
    or the H1-dot gradient ascent on J it is compared with in Section 5
    (method "ga": phi += sigma grad J(phi), then phi = phi^cc).  p: exponents
    of a separable power cost (axis 0 first; None: the quadratic cost).

    Returns phi, psi (= phi^c), map (d, *grid), w2sq (= 2 J(phi)), iters,
    converged, dual / resid / sigma logs (length iters+1) and the half-step
    values half[n] = (J(phi_{n+1/2}), I(psi_{n+1/2}), I(psi_{n+1}))."""
    mu, nu = _f64(mu), _f64(nu)
    assert mu.shape == nu.shape
    o = dict(DEFAULTS)
    o.update(opts)
    optv = np.array([o["beta1"], o["beta2"], o["alpha1"], o["alpha2"], o["sigma0"],
                     o["sigma_min"], {"brute": 0, "linear": 1}[ct_mode],
                     {"definition": 0, "fft": 1}[dct_mode],
                     {"bfm": 0, "ga": 1}[method], 0.0, 0.0, 0.0], dtype=np.float64)
    nd, n = _grid(mu.shape)
    if p is not None:
        optv[9:12] = _exponents(p, nd)
    phi = np.empty_like(mu)
    psi = np.empty_like(mu)
    tmap = np.empty((nd,) + mu.shape)
    dual = np.zeros(max_iter + 1)
    resid = np.zeros(max_iter + 1)
    sig = np.zeros(max_iter + 1)
    half = np.zeros(3 * max(max_iter, 1))
    info = np.zeros(6)
    rc = _load().bfm_oracle_solve(_ptr(mu), _ptr(nu), nd, n, float(tol), int(max_iter),
                                  _ptr(optv), _ptr(phi), _ptr(psi), _ptr(tmap),
                                  _ptr(dual), _ptr(resid), _ptr(sig), _ptr(half), _ptr(info))
    if rc < 0:
        raise ValueError(f"oracle solve rejected its input (code {rc})")
    it = int(info[0])
    return dict(phi=phi, psi=psi, map=tmap, w2sq=float(info[2]), iters=it,
                converged=bool(info[1]), mass_mu=float(info[3]), mass_nu=float(info[4]),
                sigma_final=float(info[5]), dual=dual[:it + 1], resid=resid[:it + 1],
                sigma=sig[:it + 1], half=half[:3 * it].reshape(it, 3))


def w2_gradient(phi, psi, grad_out: float = 1.0) -> tuple[np.ndarray, np.ndarray]:
    """dW2^2/dmu and dW2^2/dnu with respect to the density values, restricted
    to mass-preserving perturbations (envelope theorem on eq. (symmetric_dual)
    at the optimum: dC/dmu = psi, dC/dnu = phi, W2^2 = 2C, integration weight hd)."""
    psi = _f64(psi)
    phi = _f64(phi)
    hd = 1.0 / psi.size
    gmu = 2.0 * hd * (psi - psi.mean()) * grad_out
    gnu = 2.0 * hd * (phi - phi.mean()) * grad_out
    return gmu, gnu
