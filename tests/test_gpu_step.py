"""Full IB-GM steps on the GPU (through the C ABI) against the FP64 oracle.

FP64 fields: the GPU and the oracle evaluate the same algorithm with different
summation orders (atomics in spreading, CSR vs edge-order force sums, the
two-factor recurrence vs the Schur solve) and a different but equivalent
Douglas form (increment form, Sec. 3.4 Steps 3c-3d).  The psi operator has
condition number up to 1 + 4 N^2, so two correct FP64 evaluations may differ
by up to ~ (1 + 4 N^2) n eps norm-wise in p and psi per step (psi_bound); u
and X inherit a smaller share through the gradient.  The stated target is
tighter: u and p within 1e-12 relative (norm-wise) per step, markers 1e-13
absolute; measured at most 4.6e-14 (u), 3.5e-13 (p, 128^3) and 3.3e-16 (X).
psi, an increment near zero, is held to psi_bound (measured 3.9e-12 after two
128^3 steps).

FP32 fields (FP64 markers): within 1e-5 relative velocity and 1e-6 h marker
error after the 100 steps of the 2D workload (measured 1.3e-7 and 5.5e-8 h).
"""
import numpy as np
import pytest

import oracle as O
import paper_1305_3976_gb300 as ib
from paper_1305_3976_gb300 import inputs as I

pytestmark = pytest.mark.gpu

EPS64 = 2.0 ** -53


def rel(a, b):
    nb = np.linalg.norm(np.ravel(b))
    return np.linalg.norm(np.ravel(a) - np.ravel(b)) / (nb if nb > 0 else 1.0)


def make_pair(sc, precision="fp64", rotate=True, kernel=None, u0=None):
    kernel = kernel or sc.kernel
    P = O.params(sc.dim, sc.n, H=sc.H, rho=sc.rho, mu=sc.mu, dt=sc.dt, chi=sc.chi, kernel=kernel, rotate=rotate)
    ora = O.Simulation(P, sc.X, sc.edges, sc.kappa, sc.rest, u0=u0)
    g = ib.Grid(sc.dim, sc.n, H=sc.H, rho=sc.rho, mu=sc.mu, dt=sc.dt, chi=sc.chi, precision=precision,
                kernel=kernel, rotate_split=rotate)
    if sc.X.shape[0]:
        g.add_fiber(sc.X, sc.edges, sc.kappa, sc.rest, sc.tris)
    if u0 is not None:
        g.set_velocity(u0)
    return ora, g


def compare(ora, g):
    f = g.fields()
    d = ora.P.dim
    out = {"u": rel(np.stack([f[k] for k in ("u", "v", "w")[:d]]), ora.u),
           "p": rel(f["p"], ora.p), "psi": rel(f["psi"], ora.psi)}
    if ora.X.shape[0]:
        out["X"] = np.max(np.abs(g.markers() - ora.X))
    return out


def small_ellipsoid(n=32, nu=8, mu=0.05, dt=5e-4):
    X, E, K, R, T = I.ellipsoid_membrane(nu, (0.2, 0.25, 0.3), (0.5, 0.5, 0.5))
    return I.Scene(dim=3, n=(n, n, n), rho=1.0, mu=mu, dt=dt, steps=0, X=X, edges=E, kappa=K, rest=R, tris=T)


def psi_bound(sc, steps):
    N = max(sc.n)
    return 64.0 * steps * N * EPS64 * (1 + 4.0 * N * N)


def assert_fp64(e, steps):
    """The FP64 targets: u and p 1e-12 relative per step, markers 1e-13
    (absent for fluid-only runs); psi is checked against psi_bound."""
    assert e["u"] <= 1e-12 * steps and e["p"] <= 1e-12 * steps, e
    if "X" in e:
        assert e["X"] < 1e-13, e


@pytest.mark.parametrize("kernel", ["peskin4", "cos4"])
@pytest.mark.parametrize("rotate", [True, False])
def test_fp64_thin_ellipse_2d(kernel, rotate):
    sc = I.thin_ellipse_2d(n=64, ns=256, kernel=kernel)      # the 2D 64^2 ellipse workload
    ora, g = make_pair(sc, "fp64", rotate=rotate)
    for steps in (1, 4, 15):
        ora.step(steps)
        g.step(steps)
        e = compare(ora, g)
        assert_fp64(e, ora.n)
        assert e["psi"] < psi_bound(sc, ora.n), e
    g.close()


def test_fp64_ellipsoid_3d_small():
    sc = small_ellipsoid()
    ora, g = make_pair(sc, "fp64")
    for steps in (1, 3):
        ora.step(steps)
        g.step(steps)
        e = compare(ora, g)
        assert_fp64(e, ora.n)
        assert e["psi"] < psi_bound(sc, ora.n), e
    g.close()


def test_fp64_ragged_anisotropic_fluid_only():
    # no markers, n not a multiple of 4 along x, all axes different
    n = (50, 37, 29)
    u0 = I.random_velocity(3, n, seed=7, amplitude=0.3)
    sc = I.Scene(dim=3, n=n, rho=1.3, mu=0.02, dt=1e-3, steps=0, X=np.zeros((0, 3)),
                 edges=np.zeros((0, 2), np.int32), kappa=np.zeros(0), rest=np.zeros(0))
    ora, g = make_pair(sc, "fp64", u0=u0)
    ora.step(3)
    g.step(3)
    e = compare(ora, g)
    assert_fp64(e, 3)
    assert e["psi"] < psi_bound(sc, 3), e
    g.close()


def test_fp64_full_size_ellipsoid_128_one_step():
    # the 128^3, nu=64 (40962-marker) membrane in the launch configuration the
    # benchmark times; the oracle needs about 10 s for one step
    sc = I.ellipsoid_3d(n=128, nu=64)
    ora, g = make_pair(sc, "fp64")
    ora.step(2)
    g.step(2)
    e = compare(ora, g)
    assert_fp64(e, 2)
    assert e["psi"] < psi_bound(sc, 2), e
    g.close()


def test_fp32_thin_ellipse_100_steps_error_vs_fp64_oracle():
    # FP32 fields with FP64 markers after the 100 steps of the 2D workload
    sc = I.thin_ellipse_2d(n=64, ns=256)
    ora, g = make_pair(sc, "fp32")
    ora.step(100)
    g.step(100)
    e = compare(ora, g)
    h = 1.0 / 64
    assert e["u"] < 1e-5, e
    assert e["X"] < 1e-6 * h, e
    g.close()


def test_diagnostics_match_oracle():
    sc = small_ellipsoid()
    ora, g = make_pair(sc, "fp64")
    ora.step(2)
    g.step(2)
    d = g.diagnostics()
    assert d["step"] == 2
    assert d["volume"] == pytest.approx(O.volume_3d(ora.X, sc.tris), rel=1e-12)
    assert d["elastic"] == pytest.approx(O.elastic_energy(ora.X, sc.edges, sc.kappa), rel=1e-11)
    P = ora.P
    div = O.divergence(P, ora.u)
    assert d["div_l2"] == pytest.approx(np.sqrt(np.sum(div ** 2) / 32 ** 3), rel=1e-6)
    assert d["kinetic"] == pytest.approx(0.5 * np.sum(ora.u ** 2) / 32 ** 3, rel=1e-10)
    g.close()


def test_state_errors():
    sc = small_ellipsoid(n=16, nu=4)
    g = ib.Grid(3, 16, precision="fp64")
    g.add_fiber(sc.X, sc.edges, sc.kappa, sc.rest, sc.tris)
    g.step(1)
    with pytest.raises(ib.IBError) as ex:
        g.add_fiber(sc.X, sc.edges, sc.kappa)
    assert ex.value.code == ib.IB_ERR_STATE
    bad = sc.X.copy()
    bad[3, 1] = np.nan
    g2 = ib.Grid(3, 16, precision="fp64")
    with pytest.raises(ib.IBError) as ex:
        g2.add_fiber(bad, sc.edges, sc.kappa)
    assert ex.value.code == ib.IB_ERR_NONFINITE
    g.close()
    g2.close()


def test_fixed_sweep_configuration_replaces_the_autotuner():
    sc = small_ellipsoid(n=32, nu=8)
    _, g0 = make_pair(sc, "fp32")
    g0.step(2)
    ids = [c[0] for c in g0.sweep_configs()]
    _, g1 = make_pair(sc, "fp32")
    with pytest.raises(ib.IBError) as ex:
        ib.ib_fix_sweep_config(g1.h, 1, 99)
    assert ex.value.code == ib.IB_ERR_ARG
    g1.fix_sweep_configs(ids)
    g1.step(2)
    assert [c[0] for c in g1.sweep_configs()] == ids
    assert rel(g1.velocity(), g0.velocity()) < 1e-5
    with pytest.raises(ib.IBError) as ex:
        g1.fix_sweep_configs(ids)
    assert ex.value.code == ib.IB_ERR_STATE
    g0.close()
    g1.close()
