"""GPU vs oracle on the paper's other structures (FP64 fields):

- the thick elliptical shell of Sec. 5.2 (nested fibers, stiffness 1 - cos 2 pi r);
- the cylindrical shell of Sec. 6 (axial connections with rest length L = 1,
  closed through the periodic box);
- tiled thin ellipses in a background flow (Sec. 6.3) on the box [0, 2]^2,
  run until markers cross the periodic boundary;
and the FP32 path at the full 128^3 benchmark size: against the oracle after
2 steps, and over the 200 steps of the benchmark configuration against the
FP64 GPU run (itself tied to the oracle at this size over 10 steps in
tests/test_gpu_step.py).
Tolerances: the stated targets (assert_fp64 / assert_fp32 in
tests/test_gpu_step.py).
"""
import numpy as np
import pytest

import paper_1305_3976_gb300 as ib
from paper_1305_3976_gb300 import inputs as I

from test_gpu_step import assert_fp32, assert_fp64, compare, make_pair, psi_bound, rel, rel_max

pytestmark = pytest.mark.gpu


def test_thick_shell_2d_fp64():
    sc = I.thick_shell_2d(n=32, dt=4e-4)
    ora, g = make_pair(sc, "fp64")
    for k in (1, 9):
        ora.step(k)
        g.step(k)
        e = compare(ora, g)
        assert_fp64(e, ora.n)
        assert e["psi"] < psi_bound(sc, ora.n), e
    g.close()


def test_cylinder_3d_rest_length_and_periodic_closure_fp64():
    sc = I.cylinder_3d(n=24, dt=2e-3)
    ora, g = make_pair(sc, "fp64")
    for k in (1, 2):
        ora.step(k)
        g.step(k)
        e = compare(ora, g)
        assert_fp64(e, ora.n)
        assert e["psi"] < psi_bound(sc, ora.n), e
    g.close()


def test_tiled_ellipses_cross_the_periodic_boundary_fp64():
    sc = I.tiled_ellipses_2d(tiles=2, n_per_tile=32, dt=4e-3)
    ora, g = make_pair(sc, "fp64", u0=sc.extra["u0"])
    ora.step(110)
    g.step(110)
    X = g.markers()
    assert X[:, 1].max() > sc.H          # markers have left the box through the top
    e = compare(ora, g)
    assert_fp64(e, 110, x_tol=1e-12)
    assert e["psi"] < psi_bound(sc, 110), e
    g.close()


def test_fp32_full_size_ellipsoid_128():
    # FP32 fields with FP64 markers in the benchmark's configuration, against
    # the FP64 oracle after 2 steps
    sc = I.ellipsoid_3d(n=128, nu=64)
    ora, g = make_pair(sc, "fp32")
    ora.step(2)
    g.step(2)
    assert_fp32(compare(ora, g), 1.0 / 128, 2)
    g.close()


def test_fp32_benchmark_configuration_200_steps_vs_fp64():
    # the benchmark configuration over its 200 steps: FP32 fields against the
    # FP64 GPU run (same kernels, same summation structure), after 100 and
    # 200 steps
    sc = I.ellipsoid_3d(n=128, nu=64)
    h = 1.0 / 128
    grids = {}
    for prec in ("fp64", "fp32"):
        g = ib.Grid(3, sc.n, rho=sc.rho, mu=sc.mu, dt=sc.dt, chi=sc.chi, precision=prec, rotate_split=True)
        g.add_fiber(sc.X, sc.edges, sc.kappa, sc.rest, sc.tris)
        grids[prec] = g
    for k in (100, 100):
        out = {}
        for prec, g in grids.items():
            g.step(k)
            f = g.fields(("u", "v", "w", "p"))
            out[prec] = (np.stack([f["u"], f["v"], f["w"]]).astype(np.float64), f["p"].astype(np.float64),
                         g.markers())
        (u32, p32, X32), (u64, p64, X64) = out["fp32"], out["fp64"]
        e = {"u": rel(u32, u64), "u_max": rel_max(u32, u64), "p": rel(p32, p64), "p_max": rel_max(p32, p64),
             "X": float(np.max(np.abs(X32 - X64))), "_N": 128, "_M": u64.size}
        steps = grids["fp64"].diagnostics()["step"]
        assert_fp32(e, h, steps)
        # the pressure, which the target leaves open, stays at the velocity's
        # level in this relaxation (measured 1.2e-6 after 200 steps)
        assert e["p"] < 1e-5, e
    for g in grids.values():
        g.close()
