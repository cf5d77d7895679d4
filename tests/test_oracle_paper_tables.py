"""The oracle against numbers printed in the paper (tests/golden/, each cited).

E[div u; 64] of the thin ellipse (Table 2) and of the thick shell (Table 6)
depend on every part of the step: the force, spreading, the skew advection,
the Douglas momentum sweeps, the psi solve and the pressure update.  These
runs take 10-40 s each on one core.
"""
import json
import os

import numpy as np
import pytest

import oracle as O
from paper_1305_3976_gb300 import inputs as I

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_divergence_errors.json")))


def _div_l2(P, u):
    h = 1.0 / P.n[0]
    return float(np.sqrt(h * h * np.sum(O.divergence(P, u) ** 2)))


@pytest.mark.slow
@pytest.mark.parametrize("case", [c for c in GOLD["thin_ellipse"]["cases"] if c["sigma"] in (1.0, 10.0)],
                         ids=lambda c: f"sigma{c['sigma']}")
def test_thin_ellipse_divergence_error_table2(case):
    N, dt = case["N"], case["dt"]
    sc = I.thin_ellipse_2d(n=N, ns=19 * N // 4, r1=5 / 28, r2=7 / 20, mu=0.01, dt=dt,
                           kernel="peskin4", sigma=case["sigma"])
    P = O.params(2, N, rho=1.0, mu=0.01, dt=dt, kernel="peskin4", rotate=True)
    sim = O.Simulation(P, sc.X, sc.edges, sc.kappa, sc.rest)
    sim.step(int(round(case["t"] / dt)))
    got = _div_l2(P, sim.u)
    # the paper prints three digits; the skew stencil and split-order
    # rotation are readings, so allow 2%
    assert got == pytest.approx(case["E_div"], rel=0.02)


@pytest.mark.slow
def test_thick_shell_divergence_error_table6():
    case = GOLD["thick_shell"]["cases"][0]
    N, dt = case["N"], case["dt"]
    sc = I.thick_shell_2d(n=N, dt=dt, t_end=0.4)
    P = O.params(2, N, rho=1.0, mu=0.01, dt=dt, kernel="peskin4", rotate=True)
    sim = O.Simulation(P, sc.X, sc.edges, sc.kappa, sc.rest)
    sim.step(sc.steps)
    assert _div_l2(P, sim.u) == pytest.approx(case["E_div"], rel=0.02)
