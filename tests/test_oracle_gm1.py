"""Pins of the oracle's pressure handling for both GM variants.

- The paper's second-order variant (Sec. 3.4, Steps 3a, 3e, 3f) and its
  first-order variant (Sec. 3.1: (eps/rho) A p + D.u = 0 with eps = dt, the
  momentum step seeing p^{n-1/2}) against a closed-form recurrence for one
  Fourier mode of a gradient velocity field.  Every linear operator of the
  step is diagonal on such a mode, with the symbols
      sigma_a = 4 sin^2(pi k_a h_a) / h_a^2   (of -D_aa),
      Lambda  = sum_a sigma_a                  (of -D.G, -L),
  so u^n = alpha_n G phi, p = beta phi and psi = gamma phi with scalar
  recurrences written out below from the step's definition.  The advection
  term is quadratic in the amplitude eps and is below the tolerance.
- The first-order variant's defining identity (dt/rho) A p^{n+1/2} +
  D.u^{n+1} = 0 on an immersed-boundary problem, with A applied as the
  stencil product prod_a (1 - D_aa) (no solve).
- With chi = 0 both variants give the same first step.
"""
import numpy as np
import pytest

import oracle as O
from paper_1305_3976_gb300 import inputs as I


def grad_mode(n, k, H=1.0):
    """phi = cos(2 pi (k . x)) at cell centres and G phi on the faces."""
    d = len(n)
    h = [H / m for m in n]
    axes = [(np.arange(m) + 0.5) * hh for m, hh in zip(n, h)]
    grids = np.meshgrid(*axes[::-1], indexing="ij")          # field index order (z,) y, x
    x = grids[::-1]
    phi = np.cos(2 * np.pi * sum(kk * xx for kk, xx in zip(k, x)))
    G = np.stack([(phi - np.roll(phi, 1, axis=d - 1 - c)) / h[c] for c in range(d)])
    sigma = [4 * np.sin(np.pi * kk * hh) ** 2 / hh ** 2 for kk, hh in zip(k, h)]
    return phi, G, sigma


def mode_recurrence(scheme, steps, sigma, rho, mu, dt, chi):
    """(alpha, beta, gamma) after each step, alpha_0 = 1."""
    Lam = sum(sigma)
    a = mu * dt / (2 * rho)
    M = np.prod([1 + a * s for s in sigma])        # symbol of prod (I - a D_aa)
    A = np.prod([1 + s for s in sigma])            # symbol of prod (1 - D_aa)
    alpha, beta, gamma = 1.0, 0.0, 0.0
    out = []
    for n in range(steps):
        if n == 0:
            pstar = 0.0
        else:
            pstar = beta if scheme == "gm1" else beta + gamma
        # R = dt (mu L u - G p*) / rho; u^{n+1} = u^n + M^{-1} R
        alpha_new = alpha + dt / rho * (-mu * Lam * alpha - pstar) / M
        # A psi = -rho/dt D.u^{n+1} = rho/dt Lambda alpha_new phi
        gamma = rho / dt * Lam * alpha_new / A
        if scheme == "gm1":
            beta = gamma
        else:
            # p += psi - chi mu D.(u^{n+1} + u^n)/2 with D.G phi = -Lambda phi
            beta = beta + gamma + chi * mu * Lam * (alpha_new + alpha) / 2
        alpha = alpha_new
        out.append((alpha, beta, gamma))
    return out


@pytest.mark.parametrize("scheme", ["gm2", "gm1"])
@pytest.mark.parametrize("dim,n,k", [(2, (16, 24), (1, 2)), (3, (8, 12, 16), (1, 1, 2))])
def test_single_fourier_mode_recurrence(scheme, dim, n, k):
    rho, mu, dt, chi, eps = 1.3, 0.07, 2e-3, 0.6, 1e-7
    phi, G, sigma = grad_mode(n, k)
    P = O.params(dim, list(n), rho=rho, mu=mu, dt=dt, chi=chi, scheme=scheme, rotate=True)
    sim = O.Simulation(P, u0=eps * G)
    ref = mode_recurrence(scheme, 6, sigma, rho, mu, dt, chi)
    for alpha, beta, gamma in ref:
        sim.step(1)
        assert np.max(np.abs(sim.u - eps * alpha * G)) <= 1e-6 * eps * np.max(np.abs(G)) * abs(alpha)
        assert np.max(np.abs(sim.p - eps * beta * phi)) <= 1e-6 * eps * abs(beta)
        assert np.max(np.abs(sim.psi - eps * gamma * phi)) <= 1e-6 * eps * abs(gamma)
    # the two variants really differ on this mode
    other = mode_recurrence("gm1" if scheme == "gm2" else "gm2", 6, sigma, rho, mu, dt, chi)
    assert abs(other[-1][1] - ref[-1][1]) > 1e-3 * abs(ref[-1][1])


def apply_A(p, n, H=1.0):
    """prod_a (1 - D_aa) p by periodic stencils."""
    d = len(n)
    out = p.copy()
    for a in range(d):
        h = H / n[a]
        ax = d - 1 - a
        out = out - (np.roll(out, -1, axis=ax) - 2 * out + np.roll(out, 1, axis=ax)) / h ** 2
    return out


def divergence(u, n, H=1.0):
    d = len(n)
    return sum((np.roll(u[c], -1, axis=d - 1 - c) - u[c]) / (H / n[c]) for c in range(d))


def test_first_order_variant_satisfies_its_perturbed_constraint():
    sc = I.thin_ellipse_2d(n=32, ns=128, dt=2e-3)
    P = O.params(2, sc.n, rho=sc.rho, mu=sc.mu, dt=sc.dt, chi=sc.chi, kernel=sc.kernel, scheme="gm1")
    sim = O.Simulation(P, sc.X, sc.edges, sc.kappa, sc.rest)
    for _ in range(5):
        sim.step(1)
        du = divergence(sim.u, sc.n)
        res = sc.dt / sc.rho * apply_A(sim.p, sc.n) + du
        assert np.linalg.norm(du) > 1e-3
        assert np.linalg.norm(res) <= 1e-9 * np.linalg.norm(du)


def test_variants_share_the_first_step_when_chi_is_zero():
    sc = I.thin_ellipse_2d(n=32, ns=128, dt=2e-3)
    sims = []
    for scheme in ("gm1", "gm2"):
        P = O.params(2, sc.n, rho=sc.rho, mu=sc.mu, dt=sc.dt, chi=0.0, kernel=sc.kernel, scheme=scheme)
        sims.append(O.Simulation(P, sc.X, sc.edges, sc.kappa, sc.rest).step(1))
    a, b = sims
    assert np.array_equal(a.u, b.u) and np.array_equal(a.p, b.p) and np.array_equal(a.X, b.X)
    a.step(1)
    b.step(1)
    assert not np.allclose(a.p, b.p, rtol=1e-3)
