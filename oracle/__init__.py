"""FP64 CPU oracle for the IB-GM time step (Wiens & Stockie, arxiv 1305.3976).

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the CPU-baseline leg of
the benchmark may import this package; the product path never does.  The C
source (ib_oracle.c) follows the paper step by step in FP64 and shares no code
with the CUDA implementation.  This module only marshals numpy arrays.

Field layout: a scalar field is a C-contiguous array of shape (nz, ny, nx)
(2D: (ny, nx)); a velocity is (dim, nz, ny, nx) with component c living on
the c-faces of the MAC grid (Sec. 3.2).  Markers are (n_markers, dim).
"""
import ctypes as C
import os

import numpy as np

from . import build as _build

_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        dp = C.POINTER(C.c_double)
        ip = C.POINTER(C.c_int32)
        P = C.POINTER(Params)
        L.ibo_phi.restype = C.c_double
        L.ibo_phi.argtypes = [C.c_int, C.c_double]
        L.ibo_interp.argtypes = [P, dp, dp, C.c_int64, dp]
        L.ibo_spread.argtypes = [P, dp, dp, C.c_int64, dp]
        L.ibo_force_edges.argtypes = [C.c_int, C.c_double, dp, C.c_int64, ip, dp, dp, C.c_int64, dp]
        L.ibo_fiber_force_2d.argtypes = [dp, C.c_int64, C.c_double, C.c_double, dp]
        L.ibo_second_diff.argtypes = [P, C.c_int, dp, dp]
        L.ibo_gradient.argtypes = [P, dp, dp]
        L.ibo_divergence.argtypes = [P, dp, dp]
        L.ibo_advection.argtypes = [P, dp, dp]
        L.ibo_cyclic_solve.restype = C.c_int
        L.ibo_cyclic_solve.argtypes = [C.c_int, C.c_int, dp, dp, dp, dp, dp]
        L.ibo_solve_lines.restype = C.c_int
        L.ibo_solve_lines.argtypes = [P, C.c_int, C.c_double, dp]
        L.ibo_step.restype = C.c_int
        L.ibo_step.argtypes = [P, C.POINTER(State)]
        L.ibo_area_2d.restype = C.c_double
        L.ibo_area_2d.argtypes = [dp, ip, C.c_int64]
        L.ibo_volume_3d.restype = C.c_double
        L.ibo_volume_3d.argtypes = [dp, ip, C.c_int64]
        L.ibo_elastic_energy.restype = C.c_double
        L.ibo_elastic_energy.argtypes = [C.c_int, dp, ip, dp, dp, C.c_int64]
        _lib = L
    return _lib


class Params(C.Structure):
    _fields_ = [("dim", C.c_int), ("n", C.c_int * 3), ("H", C.c_double), ("rho", C.c_double),
                ("mu", C.c_double), ("dt", C.c_double), ("chi", C.c_double), ("kernel", C.c_int),
                ("rotate", C.c_int), ("schur_P", C.c_int), ("scheme", C.c_int)]


class State(C.Structure):
    _fields_ = [("u", C.POINTER(C.c_double)), ("p", C.POINTER(C.c_double)),
                ("psi", C.POINTER(C.c_double)), ("Nprev", C.POINTER(C.c_double)),
                ("X", C.POINTER(C.c_double)), ("Uprev", C.POINTER(C.c_double)),
                ("nm", C.c_int64), ("edges", C.POINTER(C.c_int32)),
                ("kappa", C.POINTER(C.c_double)), ("rest", C.POINTER(C.c_double)),
                ("ne", C.c_int64), ("step", C.c_int64)]


KERNELS = {"peskin4": 0, "cos4": 1}


SCHEMES = {"gm2": 0, "gm1": 1}


def params(dim, n, H=1.0, rho=1.0, mu=0.1, dt=1e-3, chi=0.6, kernel="peskin4", rotate=False,
           schur_P=1, scheme="gm2"):
    """Problem parameters; n is an int (same N on every axis) or a sequence.
    scheme: "gm2" (the paper's second-order GM variant) or "gm1" (its
    first-order variant, Sec. 3.1)."""
    if np.isscalar(n):
        n = [int(n)] * dim
    n = list(n) + [1] * (3 - len(n))
    if dim == 2:
        n[2] = 1
    P = Params()
    P.dim = dim
    P.n[0], P.n[1], P.n[2] = n
    P.H, P.rho, P.mu, P.dt, P.chi = H, rho, mu, dt, chi
    P.kernel = KERNELS[kernel] if isinstance(kernel, str) else int(kernel)
    P.rotate = int(bool(rotate))
    P.schur_P = int(schur_P)
    P.scheme = SCHEMES[scheme] if isinstance(scheme, str) else int(scheme)
    return P


def field_shape(P):
    return (P.n[1], P.n[0]) if P.dim == 2 else (P.n[2], P.n[1], P.n[0])


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _ip(a):
    return a.ctypes.data_as(C.POINTER(C.c_int32))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def phi(r, kernel="peskin4"):
    """The 1D kernel phi(r) of eq. (discretedelta) (or the cosine kernel)."""
    k = KERNELS[kernel] if isinstance(kernel, str) else int(kernel)
    r = np.asarray(r, dtype=np.float64)
    out = np.array([lib().ibo_phi(k, float(x)) for x in r.ravel()])
    return out.reshape(r.shape)


def interp(P, u, X):
    """Step 1a: U_k = sum u delta_h(x - X_k) h^d."""
    u = _f64(u)
    X = _f64(X)
    U = np.zeros_like(X)
    lib().ibo_interp(C.byref(P), _dp(u), _dp(X), X.shape[0], _dp(U))
    return U


def spread(P, X, G):
    """Step 2b with nodal forces G_k = F_k h_s: returns f on the MAC faces."""
    X = _f64(X)
    G = _f64(G)
    f = np.zeros((P.dim,) + field_shape(P))
    lib().ibo_spread(C.byref(P), _dp(X), _dp(G), X.shape[0], _dp(f))
    return f


def force_edges(X, edges, kappa, rest=None, H=1.0):
    """Step 2a over force connections (Sec. 4.1): nodal force G."""
    X = _f64(X)
    e = np.ascontiguousarray(edges, dtype=np.int32)
    k = _f64(kappa)
    r = _f64(rest) if rest is not None else np.zeros_like(k)
    G = np.zeros_like(X)
    lib().ibo_force_edges(X.shape[1], H, _dp(X), X.shape[0], _ip(e), _dp(k), _dp(r), e.shape[0], _dp(G))
    return G


def fiber_force_2d(X, sigma, L=0.0):
    """Step 2a written literally for one closed 2D fiber: F_k (a density)."""
    X = _f64(X)
    F = np.zeros_like(X)
    lib().ibo_fiber_force_2d(_dp(X), X.shape[0], sigma, L, _dp(F))
    return F


def second_diff(P, axis, q):
    q = _f64(q)
    out = np.zeros_like(q)
    lib().ibo_second_diff(C.byref(P), axis, _dp(q), _dp(out))
    return out


def gradient(P, p):
    p = _f64(p)
    g = np.zeros((P.dim,) + p.shape)
    lib().ibo_gradient(C.byref(P), _dp(p), _dp(g))
    return g


def divergence(P, u):
    u = _f64(u)
    d = np.zeros(u.shape[1:])
    lib().ibo_divergence(C.byref(P), _dp(u), _dp(d))
    return d


def advection(P, u):
    u = _f64(u)
    N = np.zeros_like(u)
    lib().ibo_advection(C.byref(P), _dp(u), _dp(N))
    return N


def cyclic_solve(a, b, c, f, P=1):
    """Cyclic tridiagonal solve, row i: c_i x_{i-1} + a_i x_i + b_i x_{i+1} = f_i."""
    a, b, c, f = (_f64(v) for v in (a, b, c, f))
    x = np.zeros_like(f)
    rc = lib().ibo_cyclic_solve(len(f), int(P), _dp(a), _dp(b), _dp(c), _dp(f), _dp(x))
    if rc != 0:
        raise ValueError("cyclic_solve: need n >= 2P")
    return x


def solve_lines(P, axis, r, q):
    """(I - r D2)^{-1} along `axis` (D2 the unit periodic second difference)."""
    q = _f64(q).copy()
    rc = lib().ibo_solve_lines(C.byref(P), axis, r, _dp(q))
    if rc != 0:
        raise ValueError("solve_lines failed")
    return q


def area_2d(X, edges):
    X = _f64(X)
    e = np.ascontiguousarray(edges, dtype=np.int32)
    return lib().ibo_area_2d(_dp(X), _ip(e), e.shape[0])


def volume_3d(X, tris):
    X = _f64(X)
    t = np.ascontiguousarray(tris, dtype=np.int32)
    return lib().ibo_volume_3d(_dp(X), _ip(t), t.shape[0])


def elastic_energy(X, edges, kappa, rest=None):
    X = _f64(X)
    e = np.ascontiguousarray(edges, dtype=np.int32)
    k = _f64(kappa)
    r = _f64(rest) if rest is not None else np.zeros_like(k)
    return lib().ibo_elastic_energy(X.shape[1], _dp(X), _ip(e), _dp(k), _dp(r), e.shape[0])


class Simulation:
    """Oracle state (u^n, p^{n-1/2}, psi^{n-1/2}, N(u^{n-1}), X^n, U^{n-1}, n)
    advanced by ibo_step (Sec. 3.4).  Initial state per Sec. 3.4's n = 0
    replacements: p = psi = 0; U^{-1} and N^{-1} are never read."""

    def __init__(self, P, X0=None, edges=None, kappa=None, rest=None, u0=None):
        self.P = P
        d = P.dim
        shp = field_shape(P)
        self.u = np.zeros((d,) + shp) if u0 is None else _f64(u0).copy()
        if self.u.shape != (d,) + shp:
            raise ValueError(f"u0 has shape {self.u.shape}, the grid needs {(d,) + shp}")
        self.p = np.zeros(shp)
        self.psi = np.zeros(shp)
        self.Nprev = np.zeros((d,) + shp)
        X0 = np.zeros((0, d)) if X0 is None else X0
        self.X = _f64(X0).copy().reshape(-1, d)
        self.Uprev = np.zeros_like(self.X)
        self.edges = np.ascontiguousarray(np.zeros((0, 2)) if edges is None else edges, dtype=np.int32)
        ne = self.edges.shape[0]
        self.kappa = _f64(np.zeros(ne) if kappa is None else kappa).copy()
        self.rest = _f64(np.zeros(ne) if rest is None else rest).copy()
        if ne and (self.edges.shape[1] != 2 or self.kappa.shape != (ne,) or self.rest.shape != (ne,)):
            raise ValueError("edges must be (n_e, 2) with n_e stiffnesses and rest lengths")
        if ne and (self.edges.min() < 0 or self.edges.max() >= self.X.shape[0]):
            raise ValueError("edge index out of range")
        self.n = 0

    def _state(self):
        S = State()
        S.u, S.p, S.psi, S.Nprev = _dp(self.u), _dp(self.p), _dp(self.psi), _dp(self.Nprev)
        # ctypes needs a non-null pointer even for empty marker sets
        if self.X.size == 0:
            self._xpad = np.zeros(1)
            S.X = S.Uprev = _dp(self._xpad)
        else:
            S.X, S.Uprev = _dp(self.X), _dp(self.Uprev)
        S.nm = self.X.shape[0]
        if self.edges.size == 0:
            self._epad = np.zeros(2, dtype=np.int32)
            self._kpad = np.zeros(1)
            S.edges, S.kappa, S.rest = _ip(self._epad), _dp(self._kpad), _dp(self._kpad)
        else:
            S.edges, S.kappa, S.rest = _ip(self.edges), _dp(self.kappa), _dp(self.rest)
        S.ne = self.edges.shape[0]
        S.step = self.n
        return S

    def step(self, k=1):
        for _ in range(k):
            S = self._state()
            rc = lib().ibo_step(C.byref(self.P), C.byref(S))
            if rc != 0:
                raise RuntimeError("ibo_step failed")
            self.n = S.step
        return self
