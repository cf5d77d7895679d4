"""The first-order Guermond-Minev variant (Sec. 3.1, eps = dt) on the GPU.

- Parity with the oracle's first-order variant (tolerances as in
  tests/test_gpu_step.py);
- its defining identity (dt/rho) A p^{n+1/2} + D.u^{n+1} = 0 on the GPU
  state, with A applied as the stencil product prod_a (1 - D_aa);
- the adjoint of the variant against central differences of the oracle;
- the divergence error on the thick shell problem of Table 6 (mu = 0.01,
  t = 0.4): the first-order variant against the oracle after the whole run,
  and the second-order variant's dependence on chi.
"""
import json
import os

import numpy as np
import pytest

import oracle as O
import paper_runs as R
from paper_1305_3976_gb300 import inputs as I

from test_gpu_adjoint import loss_of
from test_gpu_step import assert_fp32, assert_fp64, compare, psi_bound, small_ellipsoid
from test_oracle_gm1 import apply_A, divergence
import paper_1305_3976_gb300 as ib

pytestmark = pytest.mark.gpu

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_tables.json")))


def pair(sc, precision="fp64", scheme="gm1"):
    P = O.params(sc.dim, sc.n, H=sc.H, rho=sc.rho, mu=sc.mu, dt=sc.dt, chi=sc.chi, kernel=sc.kernel, rotate=True,
                 scheme=scheme)
    ora = O.Simulation(P, sc.X, sc.edges, sc.kappa, sc.rest)
    g = ib.Grid(sc.dim, sc.n, H=sc.H, rho=sc.rho, mu=sc.mu, dt=sc.dt, chi=sc.chi, precision=precision,
                kernel=sc.kernel, rotate_split=True, scheme=scheme)
    g.add_fiber(sc.X, sc.edges, sc.kappa, sc.rest, sc.tris)
    return ora, g


def test_first_order_variant_2d_fp64():
    sc = I.thin_ellipse_2d(n=64, ns=256)
    ora, g = pair(sc)
    for steps in (1, 4, 15):
        ora.step(steps)
        g.step(steps)
        e = compare(ora, g)
        assert_fp64(e, ora.n)
        assert e["psi"] < psi_bound(sc, ora.n), e
        f = g.fields()
        assert np.array_equal(f["p"], f["psi"])               # the solve is the pressure
    g.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_first_order_variant_3d(precision):
    sc = small_ellipsoid()
    ora, g = pair(sc, precision)
    ora.step(3)
    g.step(3)
    e = compare(ora, g)
    if precision == "fp64":
        assert_fp64(e, 3)
        assert e["psi"] < psi_bound(sc, 3), e
    else:
        assert_fp32(e, 1.0 / 32, 3)
    g.close()


def test_first_order_variant_satisfies_its_constraint_on_the_gpu():
    sc = I.thin_ellipse_2d(n=64, ns=256, dt=2e-3)
    _, g = pair(sc)
    for _ in range(3):
        g.step(4)
        f = g.fields()
        du = divergence(np.stack([f["u"], f["v"]]), sc.n)
        res = sc.dt / sc.rho * apply_A(f["p"], sc.n) + du
        assert np.linalg.norm(res) <= 1e-9 * np.linalg.norm(du)
    g.close()


def test_first_order_variant_adjoint_against_oracle_differences():
    sc = I.stiffness_fit_2d(n=32, ns=64, steps=10)
    P = O.params(2, sc.n, rho=sc.rho, mu=sc.mu, dt=sc.dt, chi=sc.chi, kernel=sc.kernel, rotate=True, scheme="gm1")

    def oracle_loss(kappa):
        ora = O.Simulation(P, sc.X, sc.edges, kappa, sc.rest)
        ora.step(10)
        return loss_of(ora.X, sc.extra["target"])

    g = ib.Grid(2, sc.n, rho=sc.rho, mu=sc.mu, dt=sc.dt, chi=sc.chi, precision="fp64", kernel=sc.kernel,
                rotate_split=True, scheme="gm1")
    g.add_fiber(sc.X, sc.edges, sc.kappa, sc.rest)
    L, dk = g.adjoint(10, sc.extra["target"], 4)
    g.close()
    assert abs(L - oracle_loss(sc.kappa)) <= 1e-12 * L
    fd = []
    edges = [5, 22, 51]
    for e in edges:
        h = 1e-4 * sc.kappa[e]
        kp, km = sc.kappa.copy(), sc.kappa.copy()
        kp[e] += h
        km[e] -= h
        fd.append((oracle_loss(kp) - oracle_loss(km)) / (2 * h))
    fd = np.array(fd)
    assert np.max(np.abs(dk[edges] - fd)) <= 1e-4 * np.max(np.abs(fd)), (dk[edges], fd)


def oracle_thick_shell_div(N, dt, scheme, chi=0.6, t=0.4):
    sc = I.thick_shell_2d(n=N, dt=dt, t_end=t)
    P = O.params(2, N, rho=sc.rho, mu=sc.mu, dt=dt, chi=chi, kernel=sc.kernel, rotate=True, scheme=scheme)
    ora = O.Simulation(P, sc.X, sc.edges, sc.kappa, sc.rest)
    ora.step(sc.steps)
    return R.l2_cells(divergence(ora.u, sc.n), N)


def test_first_order_variant_divergence_error_on_the_thick_shell():
    # Table 6's problem (mu = 0.01, t = 0.4, N = 64, dt = 0.08/512, 2560
    # steps) with the first-order variant: the GPU and the oracle agree on
    # E[div u] after the whole run, and it is far above the paper's
    # second-order value at the same dt (measured 1.81 against 6.34e-3)
    ref2 = GOLD["table6_thick_shell_divergence"]["runs"][0]
    assert ref2["dt"] == pytest.approx(0.08 / 512)
    e_gpu = R.l2_cells(R.thick_shell(64, 0.01, 0.08 / 512, scheme="gm1")["div"], 64)
    e_ora = oracle_thick_shell_div(64, 0.08 / 512, "gm1")
    assert e_gpu == pytest.approx(e_ora, rel=1e-2)
    assert e_gpu > 100 * ref2["E_div"]["64"]


@pytest.mark.parametrize("N", [64, 128])
def test_divergence_error_decreases_with_chi(N):
    # the Delta t / chi study of the second-order variant: at dt = 0.08/512
    # and 0.04/512, E[div u] at t = 0.4 falls as chi grows through 0, 0.3,
    # 0.6, 1 (chi = 0.6 is Table 6)
    for dt in (0.08 / 512, 0.04 / 512):
        e = [R.l2_cells(R.thick_shell(N, 0.01, dt, chi=chi)["div"], N) for chi in (0.0, 0.3, 0.6, 1.0)]
        assert all(a > b for a, b in zip(e, e[1:])), (N, dt, e)
