"""Pins of the FP64 CPU oracle against what the paper and the mathematics fix.

None of these tests re-types an oracle formula: each checks a closed form,
an invariant, a textbook property, a library routine or a brute-force sum.
"""
import numpy as np
import pytest

import oracle as O
from paper_1305_3976_gb300 import inputs as I


def l2(x):
    return float(np.sqrt(np.sum(np.asarray(x) ** 2)))


# ---------------------------------------------------------------------------
# eq. (discretedelta): Peskin's conditions on the 4-point kernel


@pytest.mark.parametrize("r0", list(np.random.default_rng(1).uniform(0, 1, 12)) + [0.0, 0.5])
def test_phi_peskin_conditions(r0):
    j = np.arange(-4, 5)
    r = r0 - j
    ph = O.phi(r)
    assert abs(ph.sum() - 1.0) < 1e-15                    # partition of unity
    assert abs(ph[j % 2 == 0].sum() - 0.5) < 1e-15        # even / odd sums
    assert abs(ph[j % 2 == 1].sum() - 0.5) < 1e-15
    assert abs((r * ph).sum()) < 1e-15                   # first moment
    assert abs((ph ** 2).sum() - 3.0 / 8.0) < 1e-15       # sum of squares = 3/8
    assert np.all(ph >= 0) and np.all(ph[np.abs(r) >= 2] == 0)


def test_phi_values_and_continuity():
    # phi(0) = 1/2, phi(1) = 1/4 (both branches agree there) and phi(2) = 0
    assert O.phi(np.array([0.0]))[0] == pytest.approx(0.5, abs=1e-16)
    assert O.phi(np.array([1.0]))[0] == pytest.approx(0.25, abs=1e-16)
    assert O.phi(np.array([2.0]))[0] == 0.0
    e = 1e-7
    for x in (1.0, 2.0, -1.0, -2.0):
        lo, hi = O.phi(np.array([x - e, x + e]))
        assert abs(lo - hi) < 1e-6                        # continuous
    # C^1: one-sided slopes agree at |r| = 1
    s_lo = (O.phi(np.array([1 - e]))[0] - O.phi(np.array([1 - 2 * e]))[0]) / e
    s_hi = (O.phi(np.array([1 + 2 * e]))[0] - O.phi(np.array([1 + e]))[0]) / e
    assert abs(s_lo - s_hi) < 1e-5
    assert O.phi(np.array([0.3]))[0] == O.phi(np.array([-0.3]))[0]   # even


def test_phi_cosine_partition_of_unity():
    for r0 in np.linspace(0, 1, 7):
        j = np.arange(-4, 5)
        ph = O.phi(r0 - j, kernel="cos4")
        assert abs(ph.sum() - 1.0) < 1e-15
        assert abs(ph[j % 2 == 0].sum() - 0.5) < 1e-15


# ---------------------------------------------------------------------------
# Sec. 4.2: the cyclic tridiagonal solve by Schur complement


def _dense_cyclic(a, b, c):
    n = len(a)
    M = np.zeros((n, n))
    for i in range(n):
        M[i, i] += a[i]
        M[i, (i + 1) % n] += b[i]
        M[i, (i - 1) % n] += c[i]
    return M


@pytest.mark.parametrize("n", [2, 3, 4, 5, 8, 12, 17, 48, 96])
@pytest.mark.parametrize("P", [1, 2, 3, 4])
def test_cyclic_solve_vs_dense(n, P):
    if n < 2 * P:
        pytest.skip("every Schur block needs an interior row")
    g = np.random.default_rng(n * 10 + P)
    b = g.uniform(-1, 1, n)
    c = g.uniform(-1, 1, n)
    a = np.abs(b) + np.abs(c) + g.uniform(0.5, 2, n)
    f = g.standard_normal(n)
    x = O.cyclic_solve(a, b, c, f, P=P)
    ref = np.linalg.solve(_dense_cyclic(a, b, c), f)
    assert np.max(np.abs(x - ref)) < 1e-13 * max(1.0, np.max(np.abs(ref)))


@pytest.mark.parametrize("n", [8, 48, 96, 128])
@pytest.mark.parametrize("r", [0.2048, 1.0, 16384.0])
@pytest.mark.parametrize("k", [0, 1, 3])
def test_cyclic_solve_fourier_mode(n, r, k):
    # (1 + 2r) x_i - r x_{i-1} - r x_{i+1} is a symmetric circulant whose
    # eigenvalue on the mode cos(2 pi k i / n + t) is 1 + 4 r sin^2(pi k / n)
    i = np.arange(n)
    f = np.cos(2 * np.pi * k * i / n + 0.3)
    lam = 1 + 4 * r * np.sin(np.pi * k / n) ** 2
    for P in (1, 4):
        x = O.cyclic_solve(np.full(n, 1 + 2 * r), np.full(n, -r), np.full(n, -r), f, P=P)
        assert np.max(np.abs(x - f / lam)) < 1e-11 * np.max(np.abs(f / lam)) * max(1.0, r / n)


@pytest.mark.parametrize("dim", [2, 3])
def test_solve_lines_each_axis_vs_dense(dim):
    n = (6, 5, 4)[:dim]
    P = O.params(dim, n)
    g = np.random.default_rng(7)
    q = g.standard_normal(O.field_shape(P))
    for axis in range(dim):
        r = 0.7 + axis
        m = n[axis]
        M = _dense_cyclic(np.full(m, 1 + 2 * r), np.full(m, -r), np.full(m, -r))
        npax = dim - 1 - axis
        qa = np.moveaxis(q, npax, 0)
        ref = np.moveaxis(np.linalg.solve(M, qa.reshape(m, -1)).reshape(qa.shape), 0, npax)
        got = O.solve_lines(P, axis, r, q)
        assert np.max(np.abs(got - ref)) < 1e-13


# ---------------------------------------------------------------------------
# Steps 1a / 2b: interpolation and spreading


def _brute_interp(P, u, X, kernel):
    """Sum over every node of the grid and its periodic images."""
    d = P.dim
    n = [P.n[a] for a in range(d)]
    h = [P.H / n[a] for a in range(d)]
    U = np.zeros_like(X)
    for k in range(X.shape[0]):
        for c in range(d):
            tot = 0.0
            for idx in np.ndindex(*reversed(n)):
                q = list(reversed(idx))
                w = 1.0
                for a in range(d):
                    off = 0.0 if a == c else 0.5
                    node = (q[a] + off) * h[a]
                    w *= sum(O.phi(np.array([(node + m * P.H - X[k, a]) / h[a]]), kernel)[0]
                             for m in (-1, 0, 1))
                tot += u[(c,) + idx] * w
            U[k, c] = tot
    return U


@pytest.mark.parametrize("dim,kernel", [(2, "peskin4"), (3, "peskin4"), (2, "cos4")])
def test_interp_brute_force(dim, kernel):
    n = (7, 6, 5)[:dim]
    P = O.params(dim, n, kernel=kernel)
    g = np.random.default_rng(3)
    u = g.standard_normal((dim,) + O.field_shape(P))
    X = g.uniform(-0.2, 1.2, size=(5, dim))      # includes points outside [0,1): wrap
    X[0] = 0.0                                    # exactly on a node
    got = O.interp(P, u, X)
    ref = _brute_interp(P, u, X, kernel)
    assert np.max(np.abs(got - ref)) < 1e-13


@pytest.mark.parametrize("dim", [2, 3])
def test_interp_linear_field_exact(dim):
    # the first-moment condition makes the 4-point kernel reproduce linear
    # functions exactly; a wrong MAC offset would shift the result by h/2
    n = 16
    P = O.params(dim, n)
    h = 1.0 / n
    shp = O.field_shape(P)
    coords = np.meshgrid(*[np.arange(s) for s in reversed(shp)], indexing="ij")  # x, y, z
    u = np.zeros((dim,) + shp)
    slope = np.array([0.3, -1.1, 0.7])[:dim]
    for c in range(dim):
        val = 2.0
        for a in range(dim):
            pos = (coords[a] + (0.0 if a == c else 0.5)) * h
            val = val + slope[a] * pos
        u[c] = np.transpose(val)        # (x, y, z) -> (z, y, x)
    g = np.random.default_rng(5)
    X = g.uniform(0.35, 0.65, size=(20, dim))     # support never wraps
    U = O.interp(P, u, X)
    for c in range(dim):
        assert np.max(np.abs(U[:, c] - (2.0 + X @ slope))) < 1e-13


@pytest.mark.parametrize("dim,kernel", [(2, "peskin4"), (3, "peskin4"), (2, "cos4")])
def test_spread_interp_adjoint_and_momentum(dim, kernel):
    n = (12, 10, 9)[:dim]
    P = O.params(dim, n, kernel=kernel)
    g = np.random.default_rng(11)
    u = g.standard_normal((dim,) + O.field_shape(P))
    X = g.uniform(-0.3, 1.3, size=(40, dim))
    G = g.standard_normal((40, dim))
    f = O.spread(P, X, G)
    vol = np.prod([1.0 / n[a] for a in range(dim)])
    lhs = np.sum(f * u) * vol
    rhs = np.sum(G * O.interp(P, u, X))
    assert abs(lhs - rhs) < 1e-12 * (abs(lhs) + 1)
    # partition of unity: total spread force equals total nodal force
    for c in range(dim):
        assert abs(f[c].sum() * vol - G[:, c].sum()) < 1e-12


# ---------------------------------------------------------------------------
# Step 2a: force connections vs the fiber form, and conservation


@pytest.mark.parametrize("L", [0.0, 0.3])
def test_edge_force_equals_fiber_force(L):
    ns = 80
    X = I.ellipse_points(ns, 0.2, 0.27)
    X += np.random.default_rng(2).normal(scale=1e-3, size=X.shape)
    F = O.fiber_force_2d(X, sigma=1.7, L=L)
    e, k, r = I.closed_fiber_connections(ns, 1.7, L)
    G = O.force_edges(X, e, k, r)
    assert np.max(np.abs(G - F / ns)) < 1e-10 * np.max(np.abs(F / ns))


@pytest.mark.parametrize("L", [0.0, 0.01])
def test_force_conserves_momentum_and_angular_momentum(L):
    X, E, K, R, T = I.ellipsoid_membrane(4, (0.2, 0.25, 0.3), (0.5, 0.5, 0.5))
    X = X + np.random.default_rng(4).normal(scale=1e-3, size=X.shape)
    G = O.force_edges(X, E, K * 1.3, R + L)
    scale = np.abs(G).max()
    assert np.max(np.abs(G.sum(axis=0))) < 1e-13 * scale * len(X)
    torque = np.cross(X, G).sum(axis=0)
    assert np.max(np.abs(torque)) < 1e-13 * scale * len(X)


def test_force_through_periodic_image():
    # a fiber that closes on itself through the box (Sec. 6 cylinder)
    ns = 16
    X = np.stack([np.arange(ns) / ns, 0.5 + 0.01 * np.sin(2 * np.pi * np.arange(ns) / ns)], axis=1)
    e, k, r = I.closed_fiber_connections(ns, 1.0, 0.0)
    G = O.force_edges(X, e, k, r)
    Xs = X.copy()
    Xs[:, 0] += 0.25                      # the same structure shifted along the axis
    Gs = O.force_edges(Xs, e, k, r)
    assert np.max(np.abs(G - Gs)) < 1e-12
    assert np.max(np.abs(G[:, 0])) < 1e-12   # equal spacing in x: no axial force


# ---------------------------------------------------------------------------
# Sec. 3.3 operators and the skew-symmetric advection term


@pytest.mark.parametrize("dim", [2, 3])
def test_div_grad_is_laplacian(dim):
    n = (8, 6, 5)[:dim]
    P = O.params(dim, n)
    g = np.random.default_rng(9)
    p = g.standard_normal(O.field_shape(P))
    lap = sum(O.second_diff(P, a, p) for a in range(dim))
    dg = O.divergence(P, O.gradient(P, p))
    assert np.max(np.abs(dg - lap)) < 1e-11 * np.max(np.abs(lap))
    u = g.standard_normal((dim,) + O.field_shape(P))
    # summation by parts: <G p, u> = -<p, D.u>, and sum of D.u is zero
    assert abs(np.sum(O.gradient(P, p) * u) + np.sum(p * O.divergence(P, u))) < 1e-10
    assert abs(np.sum(O.divergence(P, u))) < 1e-10


@pytest.mark.parametrize("dim", [2, 3])
def test_advection_is_skew_symmetric(dim):
    n = (10, 8, 6)[:dim]
    P = O.params(dim, n)
    g = np.random.default_rng(12)
    for _ in range(3):
        u = g.standard_normal((dim,) + O.field_shape(P))
        N = O.advection(P, u)
        assert abs(np.sum(u * N)) < 1e-12 * np.sum(np.abs(u * N))
    u = np.ones((dim,) + O.field_shape(P)) * np.array([0.3, -0.2, 0.1])[:dim].reshape((dim,) + (1,) * dim)
    assert np.max(np.abs(O.advection(P, u))) < 1e-14


def _exact_skew_2d(N):
    sp = pytest.importorskip("sympy")
    x, y = sp.symbols("x y")
    pi = sp.pi
    uu = sp.sin(2 * pi * x) * sp.cos(4 * pi * y) + sp.Rational(3, 10)
    vv = sp.cos(2 * pi * x + 1) * sp.sin(2 * pi * y) - sp.Rational(1, 5)
    div = sp.diff(uu, x) + sp.diff(vv, y)
    # skew form = (u.grad) u + 1/2 u (div u)
    Nu = uu * sp.diff(uu, x) + vv * sp.diff(uu, y) + uu * div / 2
    Nv = uu * sp.diff(vv, x) + vv * sp.diff(vv, y) + vv * div / 2
    f = [sp.lambdify((x, y), e, "numpy") for e in (uu, vv, Nu, Nv)]
    h = 1.0 / N
    i = np.arange(N)
    XU, YU = np.meshgrid(i * h, (i + 0.5) * h)        # u faces, shape (y, x)
    XV, YV = np.meshgrid((i + 0.5) * h, i * h)        # v faces
    u = np.stack([f[0](XU, YU) * np.ones_like(XU), f[1](XV, YV) * np.ones_like(XV)])
    ex = np.stack([f[2](XU, YU), f[3](XV, YV)])
    return u, ex


def test_advection_second_order_consistent_2d():
    errs = []
    for N in (16, 32, 64):
        u, ex = _exact_skew_2d(N)
        P = O.params(2, N)
        errs.append(np.max(np.abs(O.advection(P, u) - ex)))
    assert errs[0] / errs[1] > 3.5 and errs[1] / errs[2] > 3.7


def test_advection_second_order_consistent_3d():
    sp = pytest.importorskip("sympy")
    x, y, z = sp.symbols("x y z")
    pi = sp.pi
    U = [sp.sin(2 * pi * x) * sp.cos(2 * pi * z) + sp.Rational(1, 4),
         sp.cos(2 * pi * y + 1) * sp.sin(2 * pi * x),
         sp.sin(2 * pi * z) * sp.cos(2 * pi * y) - sp.Rational(1, 3)]
    div = sum(sp.diff(U[a], v) for a, v in enumerate((x, y, z)))
    Nex = [sum(U[a] * sp.diff(U[c], v) for a, v in enumerate((x, y, z))) + U[c] * div / 2 for c in range(3)]
    fu = [sp.lambdify((x, y, z), e, "numpy") for e in U]
    fn = [sp.lambdify((x, y, z), e, "numpy") for e in Nex]
    errs = []
    for N in (8, 16, 32):
        h = 1.0 / N
        i = np.arange(N)
        u = np.zeros((3, N, N, N))
        ex = np.zeros((3, N, N, N))
        for c in range(3):
            pos = [(i + (0.0 if a == c else 0.5)) * h for a in range(3)]
            Zg, Yg, Xg = np.meshgrid(pos[2], pos[1], pos[0], indexing="ij")
            u[c] = fu[c](Xg, Yg, Zg) * np.ones_like(Xg)
            ex[c] = fn[c](Xg, Yg, Zg) * np.ones_like(Xg)
        P = O.params(3, N)
        errs.append(np.max(np.abs(O.advection(P, u) - ex)))
    assert errs[0] / errs[1] > 3.3 and errs[1] / errs[2] > 3.6


# ---------------------------------------------------------------------------
# Full steps with closed-form answers


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("rotate", [False, True])
def test_shear_wave_amplification_and_marker_ab2(dim, rotate):
    # u = A sin(2 pi k y) on x-faces, v = w = 0: N(u) = 0, D.u = 0, psi = p = 0
    # and each Douglas step multiplies u by g = (1 - a kap)/(1 + a kap),
    # a = mu dt / (2 rho), kap = 4 sin^2(pi k h)/h^2.  A passive marker moves
    # along x with U^n = g^n U^0 under forward Euler then AB2 (Steps 1b, 1c).
    N, k, A = 16, 2, 0.8
    mu, rho, dt = 0.05, 1.3, 0.01
    P = O.params(dim, N, mu=mu, rho=rho, dt=dt, rotate=rotate)
    h = 1.0 / N
    u0 = np.zeros((dim,) + O.field_shape(P))
    yprof = A * np.sin(2 * np.pi * k * (np.arange(N) + 0.5) * h)
    if dim == 2:
        u0[0] = yprof[:, None]
    else:
        u0[0] = yprof[None, :, None]
    X0 = np.array([[0.31, 0.47, 0.52][:dim]])
    sim = O.Simulation(P, X0=X0, u0=u0)
    U0 = O.interp(P, u0, X0)[0, 0]
    a = mu * dt / (2 * rho)
    kap = 4 * np.sin(np.pi * k * h) ** 2 / h ** 2
    g = (1 - a * kap) / (1 + a * kap)
    steps = 7
    sim.step(steps)
    assert np.max(np.abs(sim.u - g ** steps * u0)) < 1e-13
    assert np.max(np.abs(sim.p)) < 1e-12 and np.max(np.abs(sim.psi)) < 1e-12
    x = X0[0, 0] + dt * U0
    for n in range(1, steps):
        x += dt * (1.5 * g ** n - 0.5 * g ** (n - 1)) * U0
    assert abs(sim.X[0, 0] - x) < 1e-14
    assert np.all(sim.X[0, 1:] == X0[0, 1:])


@pytest.mark.parametrize("dim", [2, 3])
def test_gradient_mode_closed_form(dim):
    # u = A G(phi), phi = cos(2 pi k (i+1/2) h) along x.  Linear analysis of
    # Steps 3a-3f on this single mode (nonlinear term O(A^2) made negligible):
    # D.G = -kap, D_xx = -kap on the mode, (1 - D_xx) -> 1 + kap.
    N, k, A = 16, 3, 1e-9
    mu, rho, dt, chi = 0.07, 1.2, 2e-3, 0.6
    P = O.params(dim, N, mu=mu, rho=rho, dt=dt, chi=chi, rotate=True)
    h = 1.0 / N
    i = np.arange(N)
    phi = np.cos(2 * np.pi * k * (i + 0.5) * h)
    gphi = (phi - np.roll(phi, 1)) / h
    kap = 4 * np.sin(np.pi * k * h) ** 2 / h ** 2
    shp = O.field_shape(P)
    u0 = np.zeros((dim,) + shp)
    u0[0] = A * np.broadcast_to(gphi, shp)
    sim = O.Simulation(P, u0=u0)
    a = mu * dt / (2 * rho)
    Au, Pp, Ps, scale = A, 0.0, 0.0, 0.0
    for n in range(6):
        sim.step(1)
        pstar = 0.0 if n == 0 else Pp + Ps
        ustar = Au + dt * (mu * (-kap) * Au - pstar) / rho
        A1 = (ustar + a * kap * Au) / (1 + a * kap)
        Ps = rho * kap * A1 / (dt * (1 + kap))
        Pp = Pp + Ps + chi * mu * kap * (A1 + Au) / 2
        Au = A1
        phif = np.broadcast_to(phi, shp)
        scale = max(scale, abs(Ps), abs(Pp))     # p crosses zero: compare to its size
        assert np.max(np.abs(sim.u[0] - Au * np.broadcast_to(gphi, shp))) < 1e-9 * A * np.max(gphi)
        assert np.max(np.abs(sim.psi - Ps * phif)) < 1e-9 * scale
        assert np.max(np.abs(sim.p - Pp * phif)) < 1e-9 * scale


def test_psi_factor_solve_single_mode_3d():
    # (1 - D_xx)(1 - D_yy)(1 - D_zz) psi = rhs on one Fourier mode
    N = 12
    P = O.params(3, (N, 10, 8))
    n = (N, 10, 8)
    kk = (2, 1, 3)
    idx = [np.arange(n[a]) for a in range(3)]
    Z, Y, Xg = np.meshgrid(idx[2], idx[1], idx[0], indexing="ij")
    rhs = np.cos(2 * np.pi * (kk[0] * Xg / n[0] + kk[1] * Y / n[1] + kk[2] * Z / n[2]) + 0.2)
    psi = rhs.copy()
    for a in range(3):
        psi = O.solve_lines(P, a, float(n[a]) ** 2, psi)
    lam = np.prod([1 + 4 * n[a] ** 2 * np.sin(np.pi * kk[a] / n[a]) ** 2 for a in range(3)])
    assert np.max(np.abs(psi - rhs / lam)) < 1e-14


def test_taylor_green_second_order():
    # 2D Taylor-Green vortex: u = sin 2pi x cos 2pi y F, v = -cos 2pi x sin 2pi y F,
    # F = exp(-8 pi^2 nu t) solves the Navier-Stokes equations exactly
    mu, rho, T = 0.01, 1.0, 0.25
    errs = []
    for N in (16, 32, 64):
        h = 1.0 / N
        dt = h / 8
        P = O.params(2, N, mu=mu, rho=rho, dt=dt, rotate=True)
        i = np.arange(N)
        XU, YU = np.meshgrid(i * h, (i + 0.5) * h)
        XV, YV = np.meshgrid((i + 0.5) * h, i * h)
        u0 = np.stack([np.sin(2 * np.pi * XU) * np.cos(2 * np.pi * YU),
                       -np.cos(2 * np.pi * XV) * np.sin(2 * np.pi * YV)])
        sim = O.Simulation(P, u0=u0)
        steps = int(round(T / dt))
        sim.step(steps)
        F = np.exp(-8 * np.pi ** 2 * mu / rho * steps * dt)
        errs.append(np.sqrt(h * h * np.sum((sim.u - F * u0) ** 2)))
    assert errs[0] / errs[1] > 3.5 and errs[1] / errs[2] > 3.5, errs


# ---------------------------------------------------------------------------
# Symmetries of the full step


def _ellipse_sim(N=32, rotate=False, schur_P=1, shift=(0, 0)):
    sc = I.thin_ellipse_2d(n=N, ns=96, r1=0.2, r2=0.27, mu=0.02, dt=2e-3, kernel="peskin4")
    P = O.params(2, N, mu=sc.mu, dt=sc.dt, rotate=rotate, schur_P=schur_P)
    X = sc.X + np.array(shift) / N
    return O.Simulation(P, X, sc.edges, sc.kappa, sc.rest)


def test_rotation_and_schur_blocks_change_only_rounding():
    base = _ellipse_sim().step(6)
    rot = _ellipse_sim(rotate=True).step(6)
    blk = _ellipse_sim(schur_P=4).step(6)
    for other in (rot, blk):
        assert np.max(np.abs(other.u - base.u)) < 1e-10 * np.max(np.abs(base.u))
        assert np.max(np.abs(other.p - base.p)) < 1e-10 * np.max(np.abs(base.p))
        assert np.max(np.abs(other.X - base.X)) < 1e-13


def test_translation_invariance():
    base = _ellipse_sim().step(4)
    sh = _ellipse_sim(shift=(3, 5)).step(4)
    assert np.max(np.abs(np.roll(base.u, (5, 3), axis=(1, 2)) - sh.u)) < 1e-11 * np.max(np.abs(base.u))
    assert np.max(np.abs(np.roll(base.p, (5, 3), axis=(0, 1)) - sh.p)) < 1e-11 * np.max(np.abs(base.p))
    assert np.max(np.abs(base.X + np.array([3, 5]) / 32 - sh.X)) < 1e-13


def test_symmetric_ellipse_keeps_mirror_symmetry():
    # centred ellipse with points symmetric under x -> 1 - x: the solution
    # stays mirror-symmetric (up to rounding) when the split order is symmetric
    # in x (any order: the factors commute)
    sim = _ellipse_sim(N=32).step(5)
    X = sim.X
    ns = X.shape[0]
    # point k at s_k mirrors to point ns/2 - k under x -> 1 - x
    mirror = (ns // 2 - np.arange(ns)) % ns
    assert np.max(np.abs(X[:, 0] + X[mirror, 0] - 1.0)) < 1e-12
    assert np.max(np.abs(X[:, 1] - X[mirror, 1])) < 1e-12


def test_energy_decays_and_its_window_increases_vanish_with_dt():
    # Kinetic energy 1/2 rho h^2 sum |u|^2 plus the connections' potential
    # 1/2 sum kappa |X_b - X_a|^2 (whose negative gradient is the connection
    # force) is dissipated by viscosity.  The discrete step (AB2 markers and
    # advection, pseudo-compressibility) does not make it monotone, but its
    # increases over 10-step windows vanish faster than dt (measured 1.5e-3,
    # 5.5e-4, 1.6e-4 relative for dt = 5e-4, 2.5e-4, 1.25e-4) while the decay
    # over t in [0, 0.2] converges (8.6 %, 8.0 %, 7.8 %).  Thin ellipse of
    # Sec. 5.1, 32^2.
    def run(dt, T=0.2, N=32, ns=128):
        sc = I.thin_ellipse_2d(n=N, ns=ns, r1=5 / 28, r2=7 / 20, mu=0.01, dt=dt, kernel="peskin4")
        P = O.params(2, N, rho=1.0, mu=0.01, dt=dt, chi=0.6, kernel="peskin4", rotate=True)
        sim = O.Simulation(P, sc.X, sc.edges, sc.kappa, sc.rest)
        h = 1.0 / N

        def energy():
            # kinetic energy plus the oracle's connection energy (pinned in
            # test_oracle_diagnostics.py: its gradient is minus the force)
            return 0.5 * h * h * np.sum(sim.u ** 2) + O.elastic_energy(sim.X, sc.edges, sc.kappa, sc.rest)

        E = [energy()]
        for _ in range(int(round(T / dt)) // 10):
            sim.step(10)
            E.append(energy())
        E = np.array(E)
        return 1.0 - E[-1] / E[0], np.max(np.diff(E) / E[:-1])

    res = [run(dt) for dt in (5e-4, 2.5e-4, 1.25e-4)]
    decay = [r[0] for r in res]
    inc = [r[1] for r in res]
    assert all(0.06 < d < 0.10 for d in decay), decay
    assert abs(decay[2] - decay[1]) < abs(decay[1] - decay[0]), decay
    assert inc[0] / inc[1] > 2.0 and inc[1] / inc[2] > 2.0, inc


def test_simulation_rejects_misshapen_inputs():
    # the binding hands raw pointers to C: a wrong shape must raise, not corrupt memory
    P = O.params(2, (16, 16), rho=1.0, mu=0.1, dt=1e-3)
    X = I.ellipse_points(8, 0.2, 0.25)
    E, K, R = I.closed_fiber_connections(8, 1.0)
    with pytest.raises(ValueError):
        O.Simulation(P, X, E, K, R, u0=np.zeros((8, 3)))
    with pytest.raises(ValueError):
        O.Simulation(P, X, E, K[:-1], R)
    with pytest.raises(ValueError):
        O.Simulation(P, X[:4], E, K, R)
