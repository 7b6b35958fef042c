"""Thin Python binding of the C ABI in include/bfm.h.

Argument marshalling only: every step of the method runs in the CUDA library
libbfm.so.  Functions carry the C names.  Fields are torch CUDA tensors in the
library's layout (C-order shape (n1, n0) in 2D or (n2, n1, n0) in 3D, axis 0
fastest), float32 (BFM_FP32) or float64 (BFM_FP64), contiguous.  Work is
enqueued on torch's current CUDA stream.  There is no CPU fallback: if the
library is missing or fails to load, every call raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libbfm.so")

BFM_OK = 0
BFM_NOT_CONVERGED = 1
BFM_ERR_INVALID_ARG = -1
BFM_ERR_NONFINITE = -2
BFM_ERR_CUDA = -3
BFM_ERR_TIMEOUT = -4
BFM_ERR_UNSUPPORTED = -5
BFM_ERR_WORKSPACE = -6
BFM_FP32 = 0
BFM_FP64 = 1
BFM_BACK_AND_FORTH = 0
BFM_GRADIENT_ASCENT = 1
BFM_COST_QUADRATIC = 0
BFM_COST_POWER = 1


class bfm_grid(ctypes.Structure):
    _fields_ = [("ndim", ctypes.c_int), ("n", ctypes.c_int * 3)]


class bfm_options(ctypes.Structure):
    _fields_ = [("beta1", ctypes.c_double), ("beta2", ctypes.c_double),
                ("alpha1", ctypes.c_double), ("alpha2", ctypes.c_double),
                ("sigma0", ctypes.c_double), ("sigma_min", ctypes.c_double),
                ("poll_every", ctypes.c_int), ("warm_start", ctypes.c_int),
                ("method", ctypes.c_int), ("cost_p", ctypes.c_double * 3)]


class bfm_result(ctypes.Structure):
    _fields_ = [("phi", ctypes.c_void_p), ("psi", ctypes.c_void_p), ("map", ctypes.c_void_p),
                ("dual", ctypes.POINTER(ctypes.c_double)),
                ("resid", ctypes.POINTER(ctypes.c_double)),
                ("sigma", ctypes.POINTER(ctypes.c_double)),
                ("w2sq", ctypes.c_double), ("mass_mu", ctypes.c_double),
                ("mass_nu", ctypes.c_double), ("max_mu", ctypes.c_double),
                ("max_nu", ctypes.c_double), ("sigma_final", ctypes.c_double),
                ("iters", ctypes.c_int), ("converged", ctypes.c_int)]


class BfmError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str = ""):
        self.status = status
        super().__init__(f"{where}: {status_string(status)}" + (f" ({detail})" if detail else ""))


_lock = threading.Lock()
_lib = None

_P = ctypes.c_void_p
_GP = ctypes.POINTER(bfm_grid)
_DP3 = ctypes.POINTER(ctypes.c_double * 3)
_SIGS = {
    "bfm_default_options": (None, [ctypes.POINTER(bfm_options)]),
    "bfm_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "bfm_last_error": (ctypes.c_char_p, []),
    "bfm_workspace_bytes": (ctypes.c_size_t, [_GP, ctypes.c_int, ctypes.c_int]),
    "bfm_workspace_bytes_host": (ctypes.c_size_t, [_GP, ctypes.c_int, ctypes.c_int]),
    "bfm_poisson_workspace_bytes": (ctypes.c_size_t, [_GP, ctypes.c_int]),
    "bfm_solve": (ctypes.c_int, [_P, _P, _GP, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                 ctypes.c_int, ctypes.POINTER(bfm_options), _P, ctypes.c_size_t,
                                 _P, ctypes.POINTER(bfm_result)]),
    "bfm_solve_host": (ctypes.c_int, [_P, _P, _GP, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                      ctypes.c_int, ctypes.POINTER(bfm_options), _P,
                                      ctypes.c_size_t, _P, ctypes.POINTER(bfm_result)]),
    "bfm_ctransform": (ctypes.c_int, [_P, _P, _GP, ctypes.c_int, _P]),
    "bfm_ctransform_power": (ctypes.c_int, [_P, _P, _GP, ctypes.c_int, _DP3, _P]),
    "bfm_map_power": (ctypes.c_int, [_P, _P, _GP, ctypes.c_int, _DP3, _P]),
    "bfm_poisson": (ctypes.c_int, [_P, _P, _GP, ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                   _P, ctypes.c_size_t, _P]),
    "bfm_poisson_noalloc": (ctypes.c_int, [_P, _P, _GP, ctypes.c_int,
                                           ctypes.POINTER(ctypes.c_double), _P]),
    "bfm_map": (ctypes.c_int, [_P, _P, _GP, ctypes.c_int, _P]),
    "bfm_pushforward": (ctypes.c_int, [_P, _P, _P, _GP, ctypes.c_int, _P]),
    "bfm_interpolate": (ctypes.c_int, [_P, _P, ctypes.c_double, _P, _GP, ctypes.c_int, _P]),
    "bfm_solver_init": (ctypes.c_int, [_P, _P, _GP, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                       ctypes.c_int, ctypes.POINTER(bfm_options), _P,
                                       ctypes.c_size_t, _P, _P, _P]),
    "bfm_solver_iterate": (ctypes.c_int, [_GP, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                          ctypes.POINTER(bfm_options), _P, ctypes.c_size_t, _P,
                                          _P, _P]),
    "bfm_solver_finish": (ctypes.c_int, [_GP, ctypes.c_int, ctypes.c_int, _P, ctypes.c_size_t,
                                         _P, ctypes.POINTER(bfm_result)]),
    "bfm_workspace_bytes_batched": (ctypes.c_size_t, [ctypes.c_int, _GP, ctypes.c_int,
                                                      ctypes.c_int]),
    "bfm_solve_batched": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(ctypes.c_void_p),
                                         ctypes.POINTER(ctypes.c_void_p), _GP, ctypes.c_int,
                                         ctypes.c_int, ctypes.c_double, ctypes.c_int,
                                         ctypes.POINTER(bfm_options), _P, ctypes.c_size_t, _P,
                                         ctypes.POINTER(bfm_result)]),
    "bfm_w2_backward_workspace_bytes": (ctypes.c_size_t, [ctypes.c_int]),
    "bfm_w2_backward": (ctypes.c_int, [ctypes.c_int, _GP, ctypes.c_int,
                                       ctypes.POINTER(ctypes.c_void_p),
                                       ctypes.POINTER(ctypes.c_void_p),
                                       ctypes.POINTER(ctypes.c_double),
                                       ctypes.POINTER(ctypes.c_double), _P,
                                       ctypes.POINTER(ctypes.c_void_p),
                                       ctypes.POINTER(ctypes.c_void_p), _P, ctypes.c_size_t, _P]),
    "bfm_tune_candidates": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                           ctypes.POINTER(ctypes.c_int),
                                           ctypes.POINTER(ctypes.c_int), ctypes.c_int]),
    "bfm_tune_default": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                        ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]),
    "bfm_tune_set": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                    ctypes.c_int]),
    "bfm_tune_get": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                    ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]),
    "bfm_tune_clear": (None, []),
    "bfm_tune_pick": (ctypes.c_int, [ctypes.POINTER(ctypes.c_double), ctypes.c_int, ctypes.c_int,
                                     ctypes.c_double]),
    "bfm_tune_passes": (ctypes.c_int, [_GP, ctypes.c_int, ctypes.c_int,
                                       ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                       ctypes.c_int]),
    "bfm_autotune_scratch_bytes": (ctypes.c_size_t, [ctypes.c_int, ctypes.c_int, ctypes.c_int]),
    "bfm_autotune": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, _P, ctypes.c_size_t,
                                    _P, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                    ctypes.POINTER(ctypes.c_double), ctypes.c_int]),
    "bfm_profile_kinds": (ctypes.c_int, []),
    "bfm_profile_kind_name": (ctypes.c_char_p, [ctypes.c_int]),
    "bfm_profile_begin": (ctypes.c_int, [ctypes.c_int]),
    "bfm_profile_end": (ctypes.c_int, [ctypes.POINTER(ctypes.c_double),
                                       ctypes.POINTER(ctypes.c_int), ctypes.c_int,
                                       ctypes.POINTER(ctypes.c_int)]),
}


def lib():
    """The loaded libbfm.so (raises if it was not built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"{LIB_PATH} is missing: run __graft_entry__.build() "
                                   "(there is no CPU fallback)")
            L = ctypes.CDLL(LIB_PATH)
            for name, (res, args) in _SIGS.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def status_string(s: int) -> str:
    return lib().bfm_status_string(int(s)).decode()


def last_error() -> str:
    return lib().bfm_last_error().decode()


def _check(s: int, where: str, ok=(BFM_OK,)):
    if s not in ok:
        raise BfmError(s, where, last_error() if s == BFM_ERR_CUDA or s < 0 else "")
    return s


# --- marshalling helpers -------------------------------------------------------

def grid_of(shape) -> bfm_grid:
    n = list(reversed(tuple(shape)))
    if len(n) not in (2, 3):
        raise ValueError("fields are 2D (n1, n0) or 3D (n2, n1, n0)")
    g = bfm_grid()
    g.ndim = len(n)
    for a in range(3):
        g.n[a] = n[a] if a < len(n) else 1
    return g


def _prec(t) -> int:
    import torch
    if t.dtype == torch.float32:
        return BFM_FP32
    if t.dtype == torch.float64:
        return BFM_FP64
    raise TypeError("fields must be float32 or float64")


def _dev(t, name):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return t


def _stream():
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _workspace(nbytes: int, device):
    """A 256-byte aligned device buffer (torch storage, so torch owns it)."""
    import torch
    buf = torch.empty(int(nbytes) + 256, dtype=torch.uint8, device=device)
    off = (-buf.data_ptr()) % 256
    return buf, buf.data_ptr() + off


def _user_workspace(buf):
    """A caller's uint8 CUDA tensor: its 256-aligned start and usable size."""
    _dev(buf, "workspace")
    off = (-buf.data_ptr()) % 256
    return buf, buf.data_ptr() + off, max(0, buf.numel() * buf.element_size() - off)


METHODS = {"bfm": BFM_BACK_AND_FORTH, "back_and_forth": BFM_BACK_AND_FORTH,
           "ga": BFM_GRADIENT_ASCENT, "gradient_ascent": BFM_GRADIENT_ASCENT}


def _options(**kw) -> bfm_options:
    """bfm_options with the paper's defaults, overridden by keyword (method may
    be given as "bfm" / "ga"; p = exponents of a separable power cost)."""
    o = bfm_options()
    lib().bfm_default_options(ctypes.byref(o))
    for k, v in kw.items():
        if v is None:
            continue
        if k == "p":
            vals = [float(x) for x in v]
            o.cost_p = (ctypes.c_double * 3)(*(vals + [0.0] * (3 - len(vals))))
            continue
        if k == "method" and isinstance(v, str):
            v = METHODS[v]
        setattr(o, k, v)
    return o


def _cost(opts) -> int:
    """The bfm_cost of a call: the separable power cost when p is given."""
    return BFM_COST_POWER if opts.get("p") is not None else BFM_COST_QUADRATIC


def _exponents(p, nd):
    if p is None or len(p) != nd:
        raise ValueError(f"p needs one exponent per axis ({nd})")
    return (ctypes.c_double * 3)(*([float(x) for x in p] + [0.0] * (3 - nd)))


# --- entry points ----------------------------------------------------------------

def bfm_workspace_bytes(shape, prec: int, max_iter: int) -> int:
    return int(lib().bfm_workspace_bytes(ctypes.byref(grid_of(shape)), prec, max_iter))


def bfm_workspace_bytes_host(shape, prec: int, max_iter: int) -> int:
    return int(lib().bfm_workspace_bytes_host(ctypes.byref(grid_of(shape)), prec, max_iter))


def bfm_poisson_workspace_bytes(shape, prec: int) -> int:
    return int(lib().bfm_poisson_workspace_bytes(ctypes.byref(grid_of(shape)), prec))


def bfm_ctransform(phi, out=None, p=None):
    """out = phi^c on the grid (Definition 2.1, Section 4.1); p: exponents of a
    separable power cost (Section 5, axis 0 first), None for the quadratic cost."""
    import torch
    _dev(phi, "phi")
    out = torch.empty_like(phi) if out is None else _dev(out, "out")
    g = grid_of(phi.shape)
    if p is None:
        _check(lib().bfm_ctransform(phi.data_ptr(), out.data_ptr(), ctypes.byref(g), _prec(phi),
                                    _stream()), "bfm_ctransform")
    else:
        _check(lib().bfm_ctransform_power(phi.data_ptr(), out.data_ptr(), ctypes.byref(g),
                                          _prec(phi), _exponents(p, phi.dim()), _stream()),
               "bfm_ctransform_power")
    return out


def bfm_poisson(f, out=None, want_G: bool = True):
    """g = (-Delta)^{-1}(f - mean f) with Neumann conditions (Lemma 2.3); returns (g, G)."""
    import torch
    _dev(f, "f")
    out = torch.empty_like(f) if out is None else _dev(out, "out")
    g = grid_of(f.shape)
    prec = _prec(f)
    nb = lib().bfm_poisson_workspace_bytes(ctypes.byref(g), prec)
    keep, ws = _workspace(nb, f.device)
    G = ctypes.c_double(0.0)
    _check(lib().bfm_poisson(f.data_ptr(), out.data_ptr(), ctypes.byref(g), prec,
                             ctypes.byref(G) if want_G else None, ws, nb, _stream()),
           "bfm_poisson")
    del keep
    return out, (G.value if want_G else None)


def bfm_poisson_noalloc(f, out=None):
    """bfm_poisson without a workspace (the library's built-in scratch); returns (g, G)."""
    import torch
    _dev(f, "f")
    out = torch.empty_like(f) if out is None else _dev(out, "out")
    g = grid_of(f.shape)
    G = ctypes.c_double(0.0)
    _check(lib().bfm_poisson_noalloc(f.data_ptr(), out.data_ptr(), ctypes.byref(g), _prec(f),
                                     ctypes.byref(G), _stream()), "bfm_poisson_noalloc")
    return out, G.value


def bfm_map(psi, out=None, p=None):
    """T(x) = x - (grad h)^{-1}(grad psi(x)) (Lemma 2.2(ii)); shape (ndim, *grid);
    p: exponents of a separable power cost, None for the quadratic cost."""
    import torch
    _dev(psi, "psi")
    nd = psi.dim()
    out = torch.empty((nd,) + tuple(psi.shape), dtype=psi.dtype, device=psi.device) if out is None else _dev(out, "out")
    g = grid_of(psi.shape)
    if p is None:
        _check(lib().bfm_map(psi.data_ptr(), out.data_ptr(), ctypes.byref(g), _prec(psi),
                             _stream()), "bfm_map")
    else:
        _check(lib().bfm_map_power(psi.data_ptr(), out.data_ptr(), ctypes.byref(g), _prec(psi),
                                   _exponents(p, nd), _stream()), "bfm_map_power")
    return out


def bfm_pushforward(psi, mu, out=None):
    """rho = (x - grad psi) # mu with multilinear deposit (Section 2.1, Lemma 3.1)."""
    import torch
    _dev(psi, "psi"); _dev(mu, "mu")
    out = torch.empty_like(mu) if out is None else _dev(out, "out")
    g = grid_of(mu.shape)
    _check(lib().bfm_pushforward(psi.data_ptr(), mu.data_ptr(), out.data_ptr(), ctypes.byref(g),
                                 _prec(mu), _stream()), "bfm_pushforward")
    return out


def bfm_interpolate(tmap, mu, t: float, out=None):
    """rho_t = ((1-t) x + t T) # mu (displacement interpolation, Section 4.3)."""
    import torch
    _dev(tmap, "map"); _dev(mu, "mu")
    out = torch.empty_like(mu) if out is None else _dev(out, "out")
    g = grid_of(mu.shape)
    _check(lib().bfm_interpolate(tmap.data_ptr(), mu.data_ptr(), float(t), out.data_ptr(),
                                 ctypes.byref(g), _prec(mu), _stream()), "bfm_interpolate")
    return out


def bfm_solve(mu, nu, tol: float = 1e-6, max_iter: int = 300, with_map: bool = True,
              phi_init=None, workspace=None, **opts) -> dict:
    """Algorithm 1 with the Section 4.2 step rule; returns phi, psi, map, w2sq,
    iters, converged, status and the per-iteration dual / resid / sigma logs."""
    import torch
    _dev(mu, "mu"); _dev(nu, "nu")
    if mu.shape != nu.shape or mu.dtype != nu.dtype:
        raise ValueError("mu and nu must have the same shape and dtype")
    g = grid_of(mu.shape)
    prec = _prec(mu)
    nd = mu.dim()
    phi = torch.empty_like(mu)
    if phi_init is not None:
        phi.copy_(phi_init)
        opts["warm_start"] = 1
    psi = torch.empty_like(mu)
    tmap = torch.empty((nd,) + tuple(mu.shape), dtype=mu.dtype, device=mu.device) if with_map else None
    L = max_iter + 1
    dual = np.zeros(L); resid = np.zeros(L); sig = np.zeros(L)
    res = bfm_result()
    res.phi = phi.data_ptr(); res.psi = psi.data_ptr()
    res.map = tmap.data_ptr() if with_map else None
    res.dual = dual.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    res.resid = resid.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    res.sigma = sig.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    nb = lib().bfm_workspace_bytes(ctypes.byref(g), prec, max_iter)
    if workspace is None:
        keep, ws = _workspace(nb, mu.device)
    else:
        keep, ws, nb = _user_workspace(workspace)
    o = _options(**opts)
    s = lib().bfm_solve(mu.data_ptr(), nu.data_ptr(), ctypes.byref(g), _cost(opts), prec,
                        float(tol), int(max_iter), ctypes.byref(o), ws, nb, _stream(),
                        ctypes.byref(res))
    _check(s, "bfm_solve", ok=(BFM_OK, BFM_NOT_CONVERGED))
    it = res.iters
    del keep
    return dict(phi=phi, psi=psi, map=tmap, w2sq=res.w2sq, iters=it, converged=bool(res.converged),
                status=s, mass_mu=res.mass_mu, mass_nu=res.mass_nu, max_mu=res.max_mu,
                max_nu=res.max_nu, sigma_final=res.sigma_final, dual=dual[:it + 1].copy(),
                resid=resid[:it + 1].copy(), sigma=sig[:it + 1].copy())


def bfm_solve_host(mu: np.ndarray, nu: np.ndarray, tol: float = 1e-6, max_iter: int = 300,
                   with_map: bool = True, workspace=None, device=None, out=None, **opts) -> dict:
    """bfm_solve on host (numpy) arrays: the library copies the inputs to the
    device workspace and the results back.  out: optional dict of C-contiguous
    arrays "phi", "psi" (and "map" with with_map) of the inputs' dtype that
    receive the results, e.g. views of page-locked memory, which copies
    faster than freshly allocated pageable arrays."""
    import torch
    dt = np.float32 if mu.dtype == np.float32 else np.float64
    prec = BFM_FP32 if dt == np.float32 else BFM_FP64
    mu = np.ascontiguousarray(mu, dtype=dt); nu = np.ascontiguousarray(nu, dtype=dt)
    g = grid_of(mu.shape)
    nd = mu.ndim

    def given(name, shape):
        a = (out or {}).get(name)
        if a is None:
            return np.empty(shape, dtype=dt)
        if a.shape != shape or a.dtype != dt or not a.flags["C_CONTIGUOUS"] or not a.flags["WRITEABLE"]:
            raise ValueError(f"out[{name!r}] must be a writeable C-contiguous {np.dtype(dt).name} "
                             f"array of shape {shape}")
        return a
    phi = given("phi", mu.shape); psi = given("psi", mu.shape)
    tmap = given("map", (nd,) + mu.shape) if with_map else None
    L = max_iter + 1
    dual = np.zeros(L); resid = np.zeros(L); sig = np.zeros(L)
    res = bfm_result()
    res.phi = phi.ctypes.data; res.psi = psi.ctypes.data
    res.map = tmap.ctypes.data if with_map else None
    res.dual = dual.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    res.resid = resid.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    res.sigma = sig.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    nb = lib().bfm_workspace_bytes_host(ctypes.byref(g), prec, max_iter)
    dev = device if device is not None else torch.device("cuda", torch.cuda.current_device())
    if workspace is None:
        keep, ws = _workspace(nb, dev)
    else:
        keep, ws, nb = _user_workspace(workspace)
    o = _options(**opts)
    s = lib().bfm_solve_host(mu.ctypes.data, nu.ctypes.data, ctypes.byref(g), _cost(opts),
                             prec, float(tol), int(max_iter), ctypes.byref(o), ws, nb, _stream(),
                             ctypes.byref(res))
    _check(s, "bfm_solve_host", ok=(BFM_OK, BFM_NOT_CONVERGED))
    it = res.iters
    del keep
    return dict(phi=phi, psi=psi, map=tmap, w2sq=res.w2sq, iters=it, converged=bool(res.converged),
                status=s, dual=dual[:it + 1].copy(), resid=resid[:it + 1].copy(),
                sigma=sig[:it + 1].copy(), max_mu=res.max_mu, max_nu=res.max_nu)


class BfmSolver:
    """Step-wise solve (bfm_solver_init / bfm_solver_iterate / bfm_solver_finish):
    the caller decides when to iterate and when to read results.  phi and psi
    are the device iterates; `workspace` holds all solver state."""

    def __init__(self, mu, nu, tol: float = 0.0, max_iter: int = 1000, phi_init=None, **opts):
        import torch
        _dev(mu, "mu"); _dev(nu, "nu")
        self.grid = grid_of(mu.shape)
        self.prec = _prec(mu)
        self.max_iter = int(max_iter)
        self.shape = tuple(mu.shape)
        self.phi = torch.empty_like(mu)
        self.psi = torch.empty_like(mu)
        if phi_init is not None:
            self.phi.copy_(phi_init)
            opts["warm_start"] = 1
        self.nbytes = lib().bfm_workspace_bytes(ctypes.byref(self.grid), self.prec, self.max_iter)
        self._ws_keep, self._ws = _workspace(self.nbytes, mu.device)
        self._opts = _options(**opts)
        _check(lib().bfm_solver_init(mu.data_ptr(), nu.data_ptr(), ctypes.byref(self.grid),
                                     _cost(opts), self.prec, float(tol), self.max_iter,
                                     ctypes.byref(self._opts), self._ws, self.nbytes, _stream(),
                                     self.phi.data_ptr(), self.psi.data_ptr()),
               "bfm_solver_init")

    def iterate(self, k: int = 1):
        _check(lib().bfm_solver_iterate(ctypes.byref(self.grid), self.prec, self.max_iter, int(k),
                                        ctypes.byref(self._opts), self._ws, self.nbytes, _stream(),
                                        self.phi.data_ptr(), self.psi.data_ptr()),
               "bfm_solver_iterate")

    def finish(self, with_map: bool = True) -> dict:
        import torch
        nd = len(self.shape)
        tmap = torch.empty((nd,) + self.shape, dtype=self.phi.dtype, device=self.phi.device) if with_map else None
        L = self.max_iter + 1
        dual = np.zeros(L); resid = np.zeros(L); sig = np.zeros(L)
        res = bfm_result()
        res.phi = self.phi.data_ptr(); res.psi = self.psi.data_ptr()
        res.map = tmap.data_ptr() if with_map else None
        res.dual = dual.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        res.resid = resid.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        res.sigma = sig.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        s = lib().bfm_solver_finish(ctypes.byref(self.grid), self.prec, self.max_iter, self._ws,
                                    self.nbytes, _stream(), ctypes.byref(res))
        _check(s, "bfm_solver_finish", ok=(BFM_OK, BFM_NOT_CONVERGED))
        it = res.iters
        return dict(phi=self.phi, psi=self.psi, map=tmap, w2sq=res.w2sq, iters=it,
                    converged=bool(res.converged), status=s, dual=dual[:it + 1].copy(),
                    resid=resid[:it + 1].copy(), sigma=sig[:it + 1].copy(),
                    max_mu=res.max_mu, max_nu=res.max_nu)


# --- launch shapes of the line c-transform (autotuner) -------------------------

CT_KIND_TILE_ROWS, CT_KIND_TILE_COLS, CT_KIND_ROW, CT_KIND_ROW_COLS = 0, 1, 2, 3
CT_KIND_NAMES = {0: "tile_rows", 1: "tile_cols", 2: "row", 3: "row_cols"}


def _prec_of_dtype(dtype) -> int:
    import torch
    return BFM_FP64 if dtype in (torch.float64, np.float64) else BFM_FP32


def bfm_tune_candidates(kind: int, n: int, prec: int = BFM_FP32) -> list:
    """The (K cells per thread, W lines per CTA; 0 = as many as fit) shapes
    the tuner tries for lines of n cells taking kernel `kind`."""
    m = lib().bfm_tune_candidates(kind, n, prec, None, None, 0)
    if m < 0:
        raise ValueError("unknown kernel kind or line length")
    K = (ctypes.c_int * max(m, 1))()
    W = (ctypes.c_int * max(m, 1))()
    lib().bfm_tune_candidates(kind, n, prec, K, W, m)
    return [(K[i], W[i]) for i in range(m)]


def bfm_tune_default(kind: int, n: int, prec: int = BFM_FP32) -> tuple:
    K, W = ctypes.c_int(), ctypes.c_int()
    if lib().bfm_tune_default(kind, n, prec, ctypes.byref(K), ctypes.byref(W)) < 0:
        raise ValueError("unknown kernel kind or line length")
    return K.value, W.value


def bfm_tune_set(kind: int, n: int, K: int, W: int, prec: int = BFM_FP32) -> None:
    _check(lib().bfm_tune_set(kind, n, prec, K, W), "bfm_tune_set")


def bfm_tune_get(kind: int, n: int, prec: int = BFM_FP32) -> tuple:
    """(K, W, tuned): the shape plans take now, and whether it was stored."""
    K, W = ctypes.c_int(), ctypes.c_int()
    t = lib().bfm_tune_get(kind, n, prec, ctypes.byref(K), ctypes.byref(W))
    return K.value, W.value, bool(t)


def bfm_tune_clear() -> None:
    lib().bfm_tune_clear()


def bfm_tune_pick(ms, default_index: int, margin: float = 0.02) -> int:
    a = (ctypes.c_double * len(ms))(*[float(v) for v in ms])
    return lib().bfm_tune_pick(a, len(ms), default_index, margin)


def bfm_tune_passes(shape, prec: int = BFM_FP32, batched: bool = False) -> list:
    """The (kind, n) pairs whose shapes the c-transforms of a solve on this
    grid read (batched: the batched solver's passes)."""
    g = grid_of(shape)
    K = (ctypes.c_int * 6)()
    N = (ctypes.c_int * 6)()
    m = lib().bfm_tune_passes(ctypes.byref(g), prec, int(batched), K, N, 6)
    if m < 0:
        raise ValueError("unsupported grid")
    return [(K[i], N[i]) for i in range(m)]


def bfm_autotune(kind: int, n: int, prec: int = BFM_FP32, device=None) -> dict:
    """Time every candidate shape of kernel `kind` on lines of n cells and
    store the fastest for this process (bfm_autotune in include/bfm.h).
    Scratch comes from torch here; the library allocates nothing."""
    import torch
    dev = torch.device("cuda", torch.cuda.current_device()) if device is None else device
    nb = lib().bfm_autotune_scratch_bytes(kind, n, prec)
    if nb == 0:
        raise ValueError("unknown kernel kind or line length")
    buf = torch.empty(nb + 256, dtype=torch.uint8, device=dev)
    p = (buf.data_ptr() + 255) & ~255
    cand = bfm_tune_candidates(kind, n, prec)
    ms = (ctypes.c_double * len(cand))()
    K, W = ctypes.c_int(), ctypes.c_int()
    _check(lib().bfm_autotune(kind, n, prec, p, nb, _stream(), ctypes.byref(K), ctypes.byref(W),
                              ms, len(cand)), "bfm_autotune")
    del buf
    return {"kind": CT_KIND_NAMES[kind], "n": n, "K": K.value, "W": W.value,
            "default": bfm_tune_default(kind, n, prec),
            "candidates": [{"K": c[0], "W": c[1], "ms": ms[i]} for i, c in enumerate(cand)]}


def autotune_grid(shape, dtype=None, batched: bool = False) -> list:
    """Tune every (kind, n) the c-transforms of a solve on this grid take."""
    import torch
    prec = _prec_of_dtype(dtype if dtype is not None else torch.float32)
    return [bfm_autotune(k, n, prec) for (k, n) in bfm_tune_passes(shape, prec, batched)]


def bfm_profile_begin(max_records: int = 4096):
    _check(lib().bfm_profile_begin(int(max_records)), "bfm_profile_begin")


def bfm_profile_end() -> dict:
    """{kind name: (milliseconds, kernel launches)} since bfm_profile_begin."""
    k = lib().bfm_profile_kinds()
    ms = (ctypes.c_double * k)()
    cnt = (ctypes.c_int * k)()
    dropped = ctypes.c_int(0)
    _check(lib().bfm_profile_end(ms, cnt, k, ctypes.byref(dropped)), "bfm_profile_end")
    out = {lib().bfm_profile_kind_name(i).decode(): (ms[i], cnt[i]) for i in range(k)}
    out["_dropped"] = (0.0, dropped.value)
    return out


def _ptr_array(tensors):
    arr = (ctypes.c_void_p * len(tensors))()
    for i, t in enumerate(tensors):
        arr[i] = t.data_ptr() if t is not None else None
    return arr


def bfm_solve_batched(mus, nus, tol: float = 1e-4, max_iter: int = 500, with_map: bool = False,
                      autotune: bool = False, **opts) -> list:
    """Independent problems of uneven grid sizes solved together (one batched
    launch per kernel step and grid shape, per-problem convergence).  `mus`,
    `nus`: lists of CUDA tensors (same dtype).  autotune: first time the
    c-transform's launch shapes for every line length of the batch that has
    no stored shape yet (bfm_autotune).  Returns one dict per problem."""
    import torch
    n = len(mus)
    if n == 0 or len(nus) != n:
        raise ValueError("mus and nus must be non-empty lists of equal length")
    if autotune:
        prec0 = _prec(mus[0])
        todo = set()
        for m in mus:
            for kind, ln in bfm_tune_passes(tuple(m.shape), prec0, batched=True):
                if not bfm_tune_get(kind, ln, prec0)[2]:
                    todo.add((kind, ln))
        for kind, ln in sorted(todo):
            bfm_autotune(kind, ln, prec0, device=mus[0].device)
    prec = _prec(mus[0])
    grids = (bfm_grid * n)()
    results = (bfm_result * n)()
    keep, logs = [], []
    for i, (m, v) in enumerate(zip(mus, nus)):
        _dev(m, "mu"); _dev(v, "nu")
        if m.shape != v.shape or _prec(m) != prec or _prec(v) != prec:
            raise ValueError("each mu/nu pair must share shape and dtype")
        g = grid_of(m.shape)
        grids[i] = g
        phi = torch.empty_like(m); psi = torch.empty_like(m)
        tmap = torch.empty((m.dim(),) + tuple(m.shape), dtype=m.dtype, device=m.device) if with_map else None
        L = max_iter + 1
        lg = (np.zeros(L), np.zeros(L), np.zeros(L))
        r = results[i]
        r.phi = phi.data_ptr(); r.psi = psi.data_ptr(); r.map = tmap.data_ptr() if with_map else None
        r.dual = lg[0].ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        r.resid = lg[1].ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        r.sigma = lg[2].ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        keep.append((phi, psi, tmap))
        logs.append(lg)
    nb = lib().bfm_workspace_bytes_batched(n, grids, prec, max_iter)
    if nb == 0:
        raise BfmError(BFM_ERR_INVALID_ARG, "bfm_workspace_bytes_batched")
    ws_keep, ws = _workspace(nb, mus[0].device)
    o = _options(**opts)
    s = lib().bfm_solve_batched(n, _ptr_array(mus), _ptr_array(nus), grids, BFM_COST_QUADRATIC,
                                prec, float(tol), int(max_iter), ctypes.byref(o), ws, nb,
                                _stream(), results)
    _check(s, "bfm_solve_batched", ok=(BFM_OK, BFM_NOT_CONVERGED))
    out = []
    for i in range(n):
        r = results[i]
        it = r.iters
        phi, psi, tmap = keep[i]
        out.append(dict(phi=phi, psi=psi, map=tmap, w2sq=r.w2sq, iters=it,
                        converged=bool(r.converged), mass_mu=r.mass_mu, mass_nu=r.mass_nu,
                        max_mu=r.max_mu, max_nu=r.max_nu, dual=logs[i][0][:it + 1].copy(),
                        resid=logs[i][1][:it + 1].copy(), sigma=logs[i][2][:it + 1].copy()))
    del ws_keep
    return out


def bfm_w2_backward(phis, psis, mass_mu, mass_nu, grad_out, want_mu: bool = True,
                    want_nu: bool = True):
    """Gradients of W2^2 with respect to the density values (envelope theorem):
    returns (grad_mu list, grad_nu list); grad_out is a CUDA tensor of len(phis)."""
    import torch
    n = len(phis)
    prec = _prec(phis[0])
    grids = (bfm_grid * n)()
    for i, p in enumerate(phis):
        grids[i] = grid_of(p.shape)
    gmu = [torch.empty_like(p) for p in psis] if want_mu else None
    gnu = [torch.empty_like(p) for p in phis] if want_nu else None
    mm = (ctypes.c_double * n)(*[float(x) for x in mass_mu])
    mn = (ctypes.c_double * n)(*[float(x) for x in mass_nu])
    go = _dev(grad_out.to(phis[0].dtype).contiguous(), "grad_out")
    nb = lib().bfm_w2_backward_workspace_bytes(n)
    ws_keep, ws = _workspace(nb, phis[0].device)
    s = lib().bfm_w2_backward(n, grids, prec, _ptr_array(phis), _ptr_array(psis), mm, mn,
                              go.data_ptr(), _ptr_array(gmu) if want_mu else None,
                              _ptr_array(gnu) if want_nu else None, ws, nb, _stream())
    _check(s, "bfm_w2_backward")
    del ws_keep
    return gmu, gnu


def _autograd_function():
    import torch

    class W2Loss(torch.autograd.Function):
        """W2^2(mu_b, nu_b) for a batch of density pairs on one grid, shape
        (B, *grid); the backward kernel returns the mean-zero potentials as the
        gradients (envelope theorem)."""

        @staticmethod
        def forward(ctx, mu, nu, tol, max_iter):
            mus = [m.contiguous() for m in mu.detach()]
            nus = [v.contiguous() for v in nu.detach()]
            res = bfm_solve_batched(mus, nus, tol=tol, max_iter=max_iter)
            ctx.phis = [r["phi"] for r in res]
            ctx.psis = [r["psi"] for r in res]
            ctx.mass_mu = [r["mass_mu"] for r in res]
            ctx.mass_nu = [r["mass_nu"] for r in res]
            ctx.results = res
            return torch.tensor([r["w2sq"] for r in res], dtype=mu.dtype, device=mu.device)

        @staticmethod
        def backward(ctx, grad_out):
            gmu, gnu = bfm_w2_backward(ctx.phis, ctx.psis, ctx.mass_mu, ctx.mass_nu, grad_out,
                                       want_mu=ctx.needs_input_grad[0],
                                       want_nu=ctx.needs_input_grad[1])
            return (torch.stack(gmu) if gmu is not None else None,
                    torch.stack(gnu) if gnu is not None else None, None, None)

    return W2Loss


_W2 = None


def w2_loss(mu, nu, tol: float = 1e-5, max_iter: int = 500):
    """Differentiable W2^2 between batches of densities mu, nu of shape (B, *grid)."""
    global _W2
    if _W2 is None:
        _W2 = _autograd_function()
    return _W2.apply(mu, nu, tol, max_iter)
