"""Marker re-sorting (ib_resort_markers / ib_set_resort_interval).

The tiled thin ellipses of Sec. 6.3 on 8 x 8 tiles of 64^2 cells (the box
[0, 8]^2, 512^2 grid, 64 ellipses) carried through the top of the periodic
box by the background flow, re-numbered every 20 steps, against the FP64
oracle over 120 steps at the stated FP64 target; and re-sorting leaves the
state, the caller's marker order and the results unchanged up to the
summation order of the spreading atomics.
"""
import numpy as np
import pytest

import oracle as O
import paper_1305_3976_gb300 as ib
from paper_1305_3976_gb300 import inputs as I

from test_gpu_step import assert_fp64, compare, psi_bound, rel, small_ellipsoid

pytestmark = pytest.mark.gpu


def test_tiled_ellipses_8x8_resorted_every_20_steps_vs_oracle():
    # the ellipses are raised by 0.3 so that the top row straddles the
    # periodic boundary y = 8 and hundreds more markers cross it during the
    # 120 steps (carrying the unshifted ellipses across would take minutes of
    # oracle time at a dt that stays stable: 2e-3 blows up near t = 0.45)
    sc = I.tiled_ellipses_2d(tiles=8, n_per_tile=64, dt=1e-3)
    X = sc.X + np.array([0.0, 0.3])
    P = O.params(2, sc.n, H=sc.H, rho=sc.rho, mu=sc.mu, dt=sc.dt, chi=sc.chi, kernel=sc.kernel, rotate=True)
    ora = O.Simulation(P, X, sc.edges, sc.kappa, sc.rest, u0=sc.extra["u0"])
    g = ib.Grid(2, sc.n, H=sc.H, rho=sc.rho, mu=sc.mu, dt=sc.dt, chi=sc.chi, precision="fp64", kernel=sc.kernel,
                rotate_split=True)
    g.add_fiber(X, sc.edges, sc.kappa, sc.rest)
    g.set_velocity(sc.extra["u0"])
    g.set_resort_interval(20)
    for k in (60, 60):
        ora.step(k)
        g.step(k)
        e = compare(ora, g)
        # markers integrate the velocity, held to 1e-12 relative per step:
        # sum_n dt n 1e-12 max|u| = n^2 dt max|u| 1e-12 / 2
        speed = float(np.max(np.abs(ora.u)))
        assert_fp64(e, ora.n, x_tol=1e-13 + 0.5 * ora.n ** 2 * sc.dt * speed * 1e-12)
        assert e["psi"] < psi_bound(sc, ora.n), e
    crossed = np.sum(g.markers()[:, 1] >= sc.H) - np.sum(X[:, 1] >= sc.H)
    assert crossed > 200, crossed                    # markers have left the box through the top
    g.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_resort_keeps_the_state_and_the_caller_order(prec):
    sc = small_ellipsoid(n=32, nu=8)
    grids = []
    for _ in range(2):
        g = ib.Grid(3, 32, rho=sc.rho, mu=sc.mu, dt=sc.dt, precision=prec, rotate_split=True)
        g.add_fiber(sc.X + np.array([0.3, 0.0, 0.45]), sc.edges, sc.kappa, sc.rest, sc.tris)
        g.step(4)
        grids.append(g)
    a, b = grids
    X0 = a.markers()
    vol0 = a.diagnostics()["volume"]
    a.resort_markers()
    assert np.array_equal(a.markers(), X0)                 # caller order, same positions
    assert a.diagnostics()["volume"] == pytest.approx(vol0, rel=1e-14)
    a.step(5)
    b.step(5)
    tol = 1e-12 if prec == "fp64" else 1e-5
    assert rel(a.velocity(), b.velocity()) < tol
    assert np.max(np.abs(a.markers() - b.markers())) < (1e-13 if prec == "fp64" else 1e-8)
    for g in grids:
        g.close()
