"""FP32 fields on unusual 3D grids against the FP64 oracle (and every FP64
line-solve shape):

  - sizes that are not multiples of the kernels' tiles in y and z, with a
    random velocity field so every periodic neighbour carries data;
  - long x rows (n_x = 256 with a membrane, n_x = 512);
  - the first-order variant (p* = p, psi unused).
FP32 tolerances: the stated targets, 1e-5 relative velocity (norm-wise and
element-wise) and 1e-6 h markers, pressure within the bound that the FP32
psi solve gives (fp32_bounds in tests/test_gpu_step.py).
"""
import numpy as np
import pytest

import oracle as O
import paper_1305_3976_gb300 as ib
from paper_1305_3976_gb300 import inputs as I

from test_gpu_step import assert_fp32, compare, make_pair, small_ellipsoid

pytestmark = pytest.mark.gpu


def fluid_scene(n, seed=7):
    return I.Scene(dim=3, n=n, rho=1.3, mu=0.02, dt=1e-3, steps=0, X=np.zeros((0, 3)),
                   edges=np.zeros((0, 2), np.int32), kappa=np.zeros(0), rest=np.zeros(0))


@pytest.mark.parametrize("n", [(24, 30, 42), (8, 9, 11), (36, 40, 17)])
def test_ragged_sizes_fluid_only(n):
    sc = fluid_scene(n)
    u0 = I.random_velocity(3, n, seed=7, amplitude=0.3)
    ora, g = make_pair(sc, "fp32", u0=u0)
    for k in (1, 3):
        ora.step(k)
        g.step(k)
        assert_fp32(compare(ora, g), 1.0 / max(n), ora.n)
    assert g.diagnostics()["step"] == 4
    g.close()


def test_wide_rows_with_membrane():
    X, E, K, R, T = I.ellipsoid_membrane(16, (0.2, 0.25, 0.3), (0.5, 0.5, 0.5))
    sc = I.Scene(dim=3, n=(256, 24, 20), rho=1.0, mu=0.05, dt=2e-4, steps=0, X=X, edges=E, kappa=K, rest=R,
                 tris=T)
    u0 = I.random_velocity(3, sc.n, seed=3, amplitude=0.1)
    ora, g = make_pair(sc, "fp32", u0=u0)
    ora.step(2)
    g.step(2)
    assert_fp32(compare(ora, g), 1.0 / 24, 2)
    g.close()


def test_first_order_variant_fp32():
    sc = small_ellipsoid(n=32, nu=8)
    P = O.params(3, sc.n, rho=sc.rho, mu=sc.mu, dt=sc.dt, chi=sc.chi, kernel=sc.kernel, rotate=True, scheme="gm1")
    ora = O.Simulation(P, sc.X, sc.edges, sc.kappa, sc.rest)
    g = ib.Grid(3, sc.n, rho=sc.rho, mu=sc.mu, dt=sc.dt, chi=sc.chi, precision="fp32", kernel=sc.kernel,
                rotate_split=True, scheme="gm1")
    g.add_fiber(sc.X, sc.edges, sc.kappa, sc.rest, sc.tris)
    ora.step(4)
    g.step(4)
    assert_fp32(compare(ora, g), 1.0 / 32, 4)
    g.close()


def test_rows_of_512():
    # the psi operator along x has condition number up to 1 + 4 * 512^2, so
    # FP32 pressure carries more rounding here (measured 2.3e-4 to 3.7e-4)
    sc = fluid_scene((512, 8, 8))
    u0 = I.random_velocity(3, sc.n, seed=5, amplitude=0.3)
    ora, g = make_pair(sc, "fp32", u0=u0)
    ora.step(2)
    g.step(2)
    assert_fp32(compare(ora, g), 1.0 / 512, 2)
    g.close()


# every strided line-solve shape (vector width, chunk, warps per line) and
# the TMA kernel (id 11), fixed on the y axis: over three steps the rotated
# split order puts the y sweep in every role (plain momentum, u^n + e,
# plain psi, the divergence sweep, p + psi)
STRIDED = {0: (1, 8, 8), 1: (2, 8, 8), 2: (4, 8, 8), 3: (1, 16, 8), 4: (2, 8, 16), 5: (4, 8, 16),
           6: (1, 16, 16), 7: (2, 16, 16), 8: (1, 16, 32), 9: (2, 16, 32), 10: (1, 32, 16),
           12: (1, 32, 4), 13: (2, 16, 8), 14: (1, 32, 8), 11: (1, 32, 4)}


@pytest.mark.parametrize("ragged", [False, True])
@pytest.mark.parametrize("cfg", sorted(STRIDED))
def test_every_strided_shape_on_y_lines_vs_oracle(cfg, ragged):
    vw, ch, w = STRIDED[cfg]
    ny = ch * w - (3 if ragged else 0)       # full-length lines, or lines that leave a ragged last chunk
    n = (32, ny, 8)
    sc = fluid_scene(n, seed=cfg)
    u0 = I.random_velocity(3, n, seed=100 + cfg, amplitude=0.3)
    ora, g = make_pair(sc, "fp32", u0=u0)
    g.fix_sweep_configs([0, cfg, 0])
    for k in (1, 2):
        ora.step(k)
        g.step(k)
        assert_fp32(compare(ora, g), 1.0 / max(n), ora.n)
    g.close()


@pytest.mark.parametrize("cfg", [0, 3, 6, 8, 10])
def test_every_fp64_strided_shape_on_y_lines_vs_oracle(cfg):
    from test_gpu_step import assert_fp64
    vw, ch, w = STRIDED[cfg]
    n = (32, ch * w - 3, 8)
    sc = fluid_scene(n, seed=cfg)
    u0 = I.random_velocity(3, n, seed=200 + cfg, amplitude=0.3)
    ora, g = make_pair(sc, "fp64", u0=u0)
    g.fix_sweep_configs([0, cfg, 0])
    for k in (1, 2):
        ora.step(k)
        g.step(k)
        assert_fp64(compare(ora, g), ora.n)
    g.close()
