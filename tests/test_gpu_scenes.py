"""GPU vs oracle on the paper's other structures (FP64 fields):

- the thick elliptical shell of Sec. 5.2 (nested fibers, stiffness 1 - cos 2 pi r);
- the cylindrical shell of Sec. 6 (axial connections with rest length L = 1,
  closed through the periodic box);
- tiled thin ellipses in a background flow (Sec. 6.3) on the box [0, 2]^2,
  run until markers cross the periodic boundary;
and the FP32 path at the full 128^3 benchmark size.
Tolerances: see tests/test_gpu_step.py.
"""
import numpy as np
import pytest

from paper_1305_3976_gb300 import inputs as I

from test_gpu_step import compare, make_pair, psi_bound

pytestmark = pytest.mark.gpu


def test_thick_shell_2d_fp64():
    sc = I.thick_shell_2d(n=32, dt=4e-4)
    ora, g = make_pair(sc, "fp64")
    for k in (1, 9):
        ora.step(k)
        g.step(k)
        e = compare(ora, g)
        assert e["u"] < psi_bound(sc, ora.n) and e["p"] < psi_bound(sc, ora.n), e
        assert e["X"] < 1e-13, e
    g.close()


def test_cylinder_3d_rest_length_and_periodic_closure_fp64():
    sc = I.cylinder_3d(n=24, dt=2e-3)
    ora, g = make_pair(sc, "fp64")
    for k in (1, 2):
        ora.step(k)
        g.step(k)
        e = compare(ora, g)
        assert e["u"] < psi_bound(sc, ora.n) and e["p"] < psi_bound(sc, ora.n), e
        assert e["X"] < 1e-13, e
    g.close()


def test_tiled_ellipses_cross_the_periodic_boundary_fp64():
    sc = I.tiled_ellipses_2d(tiles=2, n_per_tile=32, dt=4e-3)
    ora, g = make_pair(sc, "fp64", u0=sc.extra["u0"])
    ora.step(110)
    g.step(110)
    X = g.markers()
    assert X[:, 1].max() > sc.H          # markers have left the box through the top
    e = compare(ora, g)
    assert e["u"] < psi_bound(sc, 110) and e["p"] < psi_bound(sc, 110), e
    assert e["X"] < 1e-12, e
    g.close()


def test_fp32_full_size_ellipsoid_128():
    # FP32 fields with FP64 markers in the benchmark's configuration, against
    # the FP64 oracle (measured: 5e-6 relative velocity, 3e-10 marker error)
    sc = I.ellipsoid_3d(n=128, nu=64)
    ora, g = make_pair(sc, "fp32")
    ora.step(2)
    g.step(2)
    e = compare(ora, g)
    assert e["u"] < 1e-4, e
    assert e["X"] < 1e-6 / 128, e
    g.close()
