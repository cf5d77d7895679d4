"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the oracle.

This module builds geometry and random fields only: marker positions, force
connections (edges with their spring constants and rest lengths), triangle
lists for volume diagnostics, and seeded random velocity fields.  It contains
none of the time-stepping arithmetic of the method.

Shapes follow the paper's workloads: the closed elliptical fiber of Sec. 5.1
(X(s) = (1/2 + r1 cos 2 pi s, 1/2 + r2 sin 2 pi s)), discretised at s_k = k h_s
(Sec. 3.2), and ellipsoidal membranes made of force connections between the
vertices of a geodesic (subdivided icosahedron) mesh, the 3D analogue of the
paper's fiber networks (Sec. 4.1, Fig. 3).

Every generator is deterministic given its seed (numpy PCG64).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

DEFAULT_SEED = 1305


def rng(seed: int = DEFAULT_SEED) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


# --------------------------------------------------------------------------
# fibers and membranes


def ellipse_points(ns: int, r1: float, r2: float, center=(0.5, 0.5)) -> np.ndarray:
    """ns equally spaced parameter values s_k = k/ns on the ellipse of Sec. 5.1."""
    s = np.arange(ns) / ns
    return np.stack([center[0] + r1 * np.cos(2 * np.pi * s),
                     center[1] + r2 * np.sin(2 * np.pi * s)], axis=1)


def closed_fiber_connections(ns: int, sigma: float, rest_length: float = 0.0, offset: int = 0):
    """Force connections of one closed fiber of ns points (Sec. 4.1, Fig. 3).

    Connection k joins points k and k+1 (mod ns).  With h_s = 1/ns the fiber
    force F_k h_s of Step 2a is reproduced by spring constant sigma/h_s and
    rest length L h_s per connection.
    """
    k = np.arange(ns)
    edges = np.stack([k, (k + 1) % ns], axis=1).astype(np.int32) + offset
    kappa = np.full(ns, sigma * ns, dtype=np.float64)
    rest = np.full(ns, rest_length / ns, dtype=np.float64)
    return edges, kappa, rest


_ICO_T = (1.0 + 5.0 ** 0.5) / 2.0
_ICO_V = np.array([[-1, _ICO_T, 0], [1, _ICO_T, 0], [-1, -_ICO_T, 0], [1, -_ICO_T, 0],
                   [0, -1, _ICO_T], [0, 1, _ICO_T], [0, -1, -_ICO_T], [0, 1, -_ICO_T],
                   [_ICO_T, 0, -1], [_ICO_T, 0, 1], [-_ICO_T, 0, -1], [-_ICO_T, 0, 1]], dtype=np.float64)
_ICO_F = np.array([[0, 11, 5], [0, 5, 1], [0, 1, 7], [0, 7, 10], [0, 10, 11], [1, 5, 9], [5, 11, 4],
                   [11, 10, 2], [10, 7, 6], [7, 1, 8], [3, 9, 4], [3, 4, 2], [3, 2, 6], [3, 6, 8],
                   [3, 8, 9], [4, 9, 5], [2, 4, 11], [6, 2, 10], [8, 6, 7], [9, 8, 1]], dtype=np.int64)


def icosphere(nu: int):
    """Frequency-nu geodesic sphere: 10 nu^2 + 2 unit vertices, 20 nu^2
    outward-oriented triangles, 30 nu^2 unique edges."""
    if nu < 1:
        raise ValueError("nu >= 1")
    key_to_id: dict = {}
    verts = []
    tris = []

    def vid(face, i, j):
        a, b, c = face
        w = {a: nu - i - j, b: i, c: j}
        key = tuple(sorted((v, wt) for v, wt in w.items() if wt > 0))
        if key not in key_to_id:
            key_to_id[key] = len(verts)
            p = sum(_ICO_V[v] * wt for v, wt in key) / nu
            verts.append(p / np.linalg.norm(p))
        return key_to_id[key]

    for face in _ICO_F:
        face = tuple(int(x) for x in face)
        for i in range(nu):
            for j in range(nu - i):
                tris.append((vid(face, i, j), vid(face, i + 1, j), vid(face, i, j + 1)))
                if i + j < nu - 1:
                    tris.append((vid(face, i + 1, j), vid(face, i + 1, j + 1), vid(face, i, j + 1)))
    V = np.array(verts)
    T = np.array(tris, dtype=np.int64)
    # orient every triangle outward
    A, B, Cc = V[T[:, 0]], V[T[:, 1]], V[T[:, 2]]
    outward = np.einsum("ij,ij->i", np.cross(B - A, Cc - A), A + B + Cc) > 0
    T[~outward] = T[~outward][:, [0, 2, 1]]
    E = np.concatenate([T[:, [0, 1]], T[:, [1, 2]], T[:, [2, 0]]])
    E = np.unique(np.sort(E, axis=1), axis=0)
    return V, T.astype(np.int32), E.astype(np.int32)


def random_rotation(g: np.random.Generator) -> np.ndarray:
    """Uniform random rotation from a normalised Gaussian quaternion."""
    q = g.standard_normal(4)
    q /= np.linalg.norm(q)
    w, x, y, z = q
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
                     [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
                     [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)]])


@dataclass
class Scene:
    """A problem instance: grid, physics, markers and force connections."""
    dim: int
    n: tuple
    rho: float
    mu: float
    dt: float
    steps: int
    X: np.ndarray                       # (n_markers, dim) FP64
    edges: np.ndarray                   # (n_edges, 2) int32
    kappa: np.ndarray                   # (n_edges,) FP64
    rest: np.ndarray                    # (n_edges,) FP64
    tris: np.ndarray | None = None      # (n_tris, 3) int32, oriented outward
    H: float = 1.0
    chi: float = 0.6
    kernel: str = "peskin4"
    name: str = ""
    extra: dict = field(default_factory=dict)

    @property
    def cells(self) -> int:
        return int(np.prod(self.n))


def ellipsoid_membrane(nu, axes, center, R=None, sigma=1.0):
    """Icosphere mesh mapped onto an ellipsoid x = c + R diag(axes) v; each
    mesh edge is one force connection with spring constant sigma and zero
    rest length."""
    V, T, E = icosphere(nu)
    X = V * np.asarray(axes)[None, :]
    if R is not None:
        X = X @ np.asarray(R).T
    X = X + np.asarray(center)[None, :]
    kappa = np.full(E.shape[0], float(sigma))
    rest = np.zeros(E.shape[0])
    return X, E, kappa, rest, T


def thin_ellipse_2d(n=64, ns=256, r1=0.2, r2=0.25, sigma=1.0, rho=1.0, mu=0.1, dt=1e-3,
                    steps=100, kernel="cos4", rest_length=0.0) -> Scene:
    """2D closed elliptical fiber in the periodic unit square (Sec. 5.1 shape).
    Defaults: 64x64, 256 markers, semi-axes 0.2/0.25, sigma=1, mu=0.1,
    dt=1e-3, 100 steps, cosine 4-point kernel."""
    X = ellipse_points(ns, r1, r2)
    edges, kappa, rest = closed_fiber_connections(ns, sigma, rest_length)
    return Scene(dim=2, n=(n, n), rho=rho, mu=mu, dt=dt, steps=steps, X=X, edges=edges,
                 kappa=kappa, rest=rest, kernel=kernel, name=f"2D ellipse {n}^2, {ns} markers")


def ellipsoid_3d(n=128, nu=64, axes=(0.2, 0.25, 0.3), sigma=1.0, rho=1.0, mu=0.05, dt=5e-4,
                 steps=200, kernel="peskin4") -> Scene:
    """3D ellipsoidal membrane centred in the periodic unit cube.  Defaults:
    128^3, icosahedral nu=64 mesh (40962 markers, 122880 connections),
    semi-axes 0.2/0.25/0.3, sigma=1, mu=0.05, dt=5e-4, 200 steps."""
    X, E, kappa, rest, T = ellipsoid_membrane(nu, axes, (0.5, 0.5, 0.5), None, sigma)
    return Scene(dim=3, n=(n, n, n), rho=rho, mu=mu, dt=dt, steps=steps, X=X, edges=E,
                 kappa=kappa, rest=rest, tris=T, kernel=kernel,
                 name=f"3D ellipsoid {n}^3, nu={nu} ({X.shape[0]} markers)")


def random_velocity(dim, n, seed=DEFAULT_SEED, amplitude=1.0) -> np.ndarray:
    """Seeded smooth-plus-noise MAC velocity (dim, [nz,] ny, nx), FP64."""
    g = rng(seed)
    shape = (dim,) + tuple(reversed(n[:dim]))
    return amplitude * g.standard_normal(shape)


def random_markers(dim, count, seed=DEFAULT_SEED, lo=0.0, hi=1.0) -> np.ndarray:
    g = rng(seed)
    return g.uniform(lo, hi, size=(count, dim))


def thick_shell_2d(n=64, r1=0.2, r2=0.25, gamma=0.0625, mu=0.01, rho=1.0, dt=0.08 / 512,
                   steps=None, t_end=0.4, kernel="peskin4") -> Scene:
    """Thick elliptical shell of Sec. 5.2: N_r nested closed fibers (N_r = 3N/8),
    each of N_s = 75N/16 points, at radial parameters r_l = (l + 1/2)/N_r,
    X(s, r) = (1/2 + (r1 + gamma (r - 1/2)) cos 2 pi s, 1/2 + (r2 + gamma (r - 1/2)) sin 2 pi s),
    stiffness sigma(r) = 1 - cos 2 pi r.  Spreading weighs every point by
    h_s h_r, so fiber l gets spring constant sigma(r_l) h_r / h_s."""
    ns, nr = 75 * n // 16, 3 * n // 8
    hs, hr = 1.0 / ns, 1.0 / nr
    Xs, Es, Ks, Rs = [], [], [], []
    for l in range(nr):
        r = (l + 0.5) * hr
        X = ellipse_points(ns, r1 + gamma * (r - 0.5), r2 + gamma * (r - 0.5))
        sig = 1.0 - np.cos(2 * np.pi * r)
        e, _, rest = closed_fiber_connections(ns, 1.0, 0.0, offset=l * ns)
        Xs.append(X)
        Es.append(e)
        Ks.append(np.full(ns, sig * hr / hs))
        Rs.append(rest)
    if steps is None:
        steps = int(round(t_end / dt))
    return Scene(dim=2, n=(n, n), rho=rho, mu=mu, dt=dt, steps=steps, X=np.concatenate(Xs),
                 edges=np.concatenate(Es), kappa=np.concatenate(Ks), rest=np.concatenate(Rs),
                 kernel=kernel, name=f"2D thick shell {n}^2, {ns}x{nr} markers")


def cylinder_3d(n=32, r1=5 / 28, r2=7 / 20, sigma_s=1.0, sigma_r=1.0, L=1.0, mu=0.01, rho=1.0, dt=None,
                steps=100, kernel="peskin4") -> Scene:
    """Cylindrical elastic shell of Sec. 6: X(s, r) = (r, 1/2 + r1 cos 2 pi s,
    1/2 + r2 sin 2 pi s), N_s = 19N/4 circumferential points times N_r = 3N
    axial points, each end joined to its periodic copy.  Circumferential
    connections: spring sigma_s h_r / h_s, rest length 0; axial connections:
    spring sigma_r h_s / h_r, rest length L h_r (quadrature weight h_s h_r per
    point).  Default dt = 0.04/N."""
    ns, nr = 19 * n // 4, 3 * n
    hs, hr = 1.0 / ns, 1.0 / nr
    s = np.arange(ns) * hs
    r = np.arange(nr) * hr
    S, Rr = np.meshgrid(s, r, indexing="ij")                 # point (k, l) -> k * nr + l
    X = np.stack([Rr.ravel(), 0.5 + r1 * np.cos(2 * np.pi * S.ravel()),
                  0.5 + r2 * np.sin(2 * np.pi * S.ravel())], axis=1)
    idx = np.arange(ns * nr).reshape(ns, nr)
    e_s = np.stack([idx.ravel(), np.roll(idx, -1, axis=0).ravel()], axis=1)
    e_r = np.stack([idx.ravel(), np.roll(idx, -1, axis=1).ravel()], axis=1)
    edges = np.concatenate([e_s, e_r]).astype(np.int32)
    kappa = np.concatenate([np.full(len(e_s), sigma_s * hr / hs), np.full(len(e_r), sigma_r * hs / hr)])
    rest = np.concatenate([np.zeros(len(e_s)), np.full(len(e_r), L * hr)])
    if dt is None:
        dt = 0.04 / n
    return Scene(dim=3, n=(n, n, n), rho=rho, mu=mu, dt=dt, steps=steps, X=X, edges=edges, kappa=kappa,
                 rest=rest, kernel=kernel, name=f"3D cylinder {n}^3, {ns}x{nr} markers")


def tiled_ellipses_2d(tiles=2, n_per_tile=32, r1=5 / 28, r2=7 / 20, sigma=1.0, mu=0.01, rho=1.0, dt=None,
                      steps=100, kernel="peskin4") -> Scene:
    """tiles x tiles copies of the thin ellipse of Sec. 5.1, one per unit
    tile of the periodic box [0, tiles]^2 (Sec. 6.3), with spacing h_s = 4h/19
    along each ellipse; the fluid starts with the uniform background velocity
    (1/2, sqrt(3)/2) set through Scene.extra['u0'].  Default dt = 0.01 h."""
    n = tiles * n_per_tile
    h = tiles / n
    perim = np.pi * (3 * (r1 + r2) - np.sqrt((3 * r1 + r2) * (r1 + 3 * r2)))  # Ramanujan
    ns = int(round(perim / (4 * h / 19)))
    Xs, Es, Ks, Rs = [], [], [], []
    for ty in range(tiles):
        for tx in range(tiles):
            X = ellipse_points(ns, r1, r2, center=(tx + 0.5, ty + 0.5))
            e, k, rr = closed_fiber_connections(ns, sigma, 0.0, offset=len(Xs) * ns)
            Xs.append(X)
            Es.append(e)
            Ks.append(k)
            Rs.append(rr)
    if dt is None:
        dt = 0.01 * h
    u0 = np.zeros((2, n, n))
    u0[0] = 0.5
    u0[1] = np.sqrt(3.0) / 2
    return Scene(dim=2, n=(n, n), rho=rho, mu=mu, dt=dt, steps=steps, X=np.concatenate(Xs),
                 edges=np.concatenate(Es), kappa=np.concatenate(Ks), rest=np.concatenate(Rs), H=float(tiles),
                 kernel=kernel, name=f"2D {tiles}x{tiles} tiled ellipses {n}^2", extra={"u0": u0})


def ensemble_members(count=48, seed=DEFAULT_SEED, sizes=(48, 64, 96, 128), dt128=5e-4):
    """Independent 3D runs: grid N uniform over `sizes`, one ellipsoidal
    membrane (semi-axes 0.2/0.25/0.3, icosahedral nu = N/2, about 2 markers per
    h), stiffness sigma log-uniform in [0.1, 10], viscosity mu uniform in
    [0.01, 0.1], dt = dt128 (128/N) min(1, sigma^-1/2)."""
    g = rng(seed)
    meshes = {}
    out = []
    for _ in range(count):
        n = int(g.choice(sizes))
        sigma = float(np.exp(g.uniform(np.log(0.1), np.log(10.0))))
        mu = float(g.uniform(0.01, 0.1))
        nu = n // 2
        if nu not in meshes:
            meshes[nu] = icosphere(nu)
        V, T, E = meshes[nu]
        X = V * np.array([0.2, 0.25, 0.3])[None, :] + 0.5
        dt = dt128 * (128.0 / n) * min(1.0, sigma ** -0.5)
        out.append(Scene(dim=3, n=(n, n, n), rho=1.0, mu=mu, dt=dt, steps=100, X=X, edges=E,
                         kappa=np.full(E.shape[0], sigma), rest=np.zeros(E.shape[0]), tris=T,
                         name=f"ensemble member {n}^3 sigma={sigma:.3g} mu={mu:.3g}"))
    return out


def random_ellipsoids_3d(n=512, count=8, nu=80, seed=DEFAULT_SEED, mu=0.01, dt=3.125e-5, steps=50,
                         axes_range=(0.05, 0.1), sigma=1.0) -> Scene:
    """`count` ellipsoidal membranes with semi-axes uniform in axes_range,
    uniformly random orientations (normalised Gaussian quaternions) and
    centres drawn by rejection until every pair is farther apart (periodic
    distance) than the sum of their largest semi-axes plus 4h of the 512^3 grid
    (the same bodies at every n); icosahedral meshes of frequency nu
    (10 nu^2 + 2 markers each).  dt = 3.125e-5 is the largest of 1.25e-4,
    6.25e-5 and 3.125e-5 that stays stable for 50 steps at 512^3 (1.25e-4
    overflows within 30 steps; 6.25e-5 shows a growing divergence)."""
    g = rng(seed)
    V, T, E = icosphere(nu)
    h = 1.0 / 512
    bodies = []
    while len(bodies) < count:
        axes = g.uniform(*axes_range, size=3)
        c = g.uniform(0, 1, size=3)
        ok = True
        for c2, a2 in bodies:
            dvec = c - c2
            dvec -= np.round(dvec)
            if np.linalg.norm(dvec) <= axes.max() + a2.max() + 4 * h:
                ok = False
                break
        if ok:
            bodies.append((c, axes))
    Xs, Es, Ts = [], [], []
    for i, (c, axes) in enumerate(bodies):
        R = random_rotation(g)
        Xs.append((V * axes[None, :]) @ R.T + c[None, :])
        Es.append(E + i * V.shape[0])
        Ts.append(T + i * V.shape[0])
    Eall = np.concatenate(Es).astype(np.int32)
    return Scene(dim=3, n=(n, n, n), rho=1.0, mu=mu, dt=dt, steps=steps, X=np.concatenate(Xs), edges=Eall,
                 kappa=np.full(Eall.shape[0], sigma), rest=np.zeros(Eall.shape[0]),
                 tris=np.concatenate(Ts).astype(np.int32),
                 name=f"3D {count} random ellipsoids {n}^3, nu={nu}")


def stiffness_fit_3d(n=96, nu=28, seed=DEFAULT_SEED, axes=(0.2, 0.25, 0.3), sigma_range=(0.5, 2.0), rho=1.0,
                     mu=0.05, dt=5e-4, steps=200, kernel="peskin4") -> Scene:
    """Stiffness-gradient problem: the ellipsoidal membrane of ellipsoid_3d
    (icosahedral nu mesh, 10 nu^2 + 2 markers; nu = 28 gives 7842 markers
    and 23520 connections) with one stiffness per connection drawn uniform in
    sigma_range, zero rest lengths.  extra["target"] holds the same mesh on
    the sphere of equal volume (radius (a b c)^(1/3), same centre) plus
    Gaussian jitter of standard deviation h / 10; the loss is
    sum_k |X_k - target_k|^2 after `steps` steps."""
    g = rng(seed)
    X, E, _, rest, T = ellipsoid_membrane(nu, axes, (0.5, 0.5, 0.5))
    kappa = g.uniform(*sigma_range, size=E.shape[0])
    V, _, _ = icosphere(nu)
    r = float(np.prod(axes)) ** (1.0 / 3.0)
    target = V * r + 0.5 + g.normal(0.0, 0.1 / n, size=V.shape)
    return Scene(dim=3, n=(n, n, n), rho=rho, mu=mu, dt=dt, steps=steps, X=X, edges=E, kappa=kappa, rest=rest,
                 tris=T, kernel=kernel, name=f"stiffness fit {n}^3, nu={nu} ({X.shape[0]} markers)",
                 extra={"target": target})


def stiffness_fit_2d(n=32, ns=64, seed=DEFAULT_SEED, r1=0.2, r2=0.25, sigma_range=(0.5, 2.0), rho=1.0, mu=0.1,
                     dt=1e-3, steps=20, kernel="cos4") -> Scene:
    """2D counterpart of stiffness_fit_3d: a closed elliptical fiber of ns
    points with kappa_e = sigma_e ns, sigma_e uniform in sigma_range, zero
    rest lengths; target: the circle of equal area plus h / 10 jitter."""
    g = rng(seed)
    X = ellipse_points(ns, r1, r2)
    edges, _, rest = closed_fiber_connections(ns, 1.0, 0.0)
    kappa = g.uniform(*sigma_range, size=ns) * ns
    r = float(np.sqrt(r1 * r2))
    target = ellipse_points(ns, r, r) + g.normal(0.0, 0.1 / n, size=X.shape)
    return Scene(dim=2, n=(n, n), rho=rho, mu=mu, dt=dt, steps=steps, X=X, edges=edges, kappa=kappa, rest=rest,
                 kernel=kernel, name=f"2D stiffness fit {n}^2, {ns} markers", extra={"target": target})
