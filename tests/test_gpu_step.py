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

Every field comparison is made twice: norm-wise (||a - b|| / ||b||) and
element-wise (max |a - b| / max |b|), against the same bound.  With the
environment variable IB_PARITY_LOG set to a file name, every checked error is
appended to that file as one JSON line (test, errors, bound), which is where
the measured values quoted in the docstrings come from.
"""
import json
import os

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


def rel_max(a, b):
    """max |a - b| over all elements, relative to max |b|"""
    mb = np.max(np.abs(b)) if np.size(b) else 0.0
    return float(np.max(np.abs(np.asarray(a, np.float64) - b)) / (mb if mb > 0 else 1.0)) if np.size(b) else 0.0


def record(e, bound=None):
    """Append the measured errors of the running test to $IB_PARITY_LOG."""
    path = os.environ.get("IB_PARITY_LOG")
    if not path:
        return
    test = os.environ.get("PYTEST_CURRENT_TEST", "?").split(" ")[0]
    with open(path, "a") as fh:
        fh.write(json.dumps({"test": test, "errors": {k: float(v) for k, v in e.items()}, "bound": bound}) + "\n")


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
    """Errors of grid g against oracle run ora: u, p, psi norm-wise, u_max,
    p_max element-wise (rel_max), X the largest marker difference."""
    f = g.fields()
    d = ora.P.dim
    u = np.stack([f[k] for k in ("u", "v", "w")[:d]]).astype(np.float64)
    out = {"u": rel(u, ora.u), "p": rel(f["p"], ora.p), "psi": rel(f["psi"], ora.psi),
           "u_max": rel_max(u, ora.u), "p_max": rel_max(f["p"], ora.p),
           "_N": max(ora.P.n[:d]) if hasattr(ora.P, "n") else max(u.shape[1:]), "_M": u.size}
    if ora.X.shape[0]:
        out["X"] = float(np.max(np.abs(g.markers() - ora.X)))
    return out


def small_ellipsoid(n=32, nu=8, mu=0.05, dt=5e-4):
    X, E, K, R, T = I.ellipsoid_membrane(nu, (0.2, 0.25, 0.3), (0.5, 0.5, 0.5))
    return I.Scene(dim=3, n=(n, n, n), rho=1.0, mu=mu, dt=dt, steps=0, X=X, edges=E, kappa=K, rest=R, tris=T)


def psi_bound(sc, steps):
    N = max(sc.n)
    return 64.0 * steps * N * EPS64 * (1 + 4.0 * N * N)


def assert_fp64(e, steps, x_tol=1e-13):
    """The FP64 targets: u and p within 1e-12 relative per step, norm-wise
    and element-wise, markers within x_tol (1e-13; absent for fluid-only
    runs); psi is checked by the caller against psi_bound."""
    b = 1e-12 * steps
    record(e, {"u": b, "p": b, "X": x_tol})
    assert e["u"] <= b and e["p"] <= b, e
    assert e["u_max"] <= b and e["p_max"] <= b, e
    if "X" in e:
        assert e["X"] < x_tol, e


EPS32 = 2.0 ** -24


def fp32_bounds(e, h, steps, x_tol=None):
    """The FP32 bounds (FP32 fields with FP64 markers against an FP64 run) for
    errors e of a grid with e["_N"] cells along its longest axis and e["_M"]
    velocity values:
      u      1e-5 relative, norm-wise: the stated target;
      u_max  sqrt(2 ln M) 1e-5 element-wise: the largest of M noise-like
             errors exceeds their RMS by about sqrt(2 ln M), and
             RMS(u) <= max |u|;
      p      1e-4 norm-wise and element-wise for N <= 128, growing with the
             condition number 1 + 4N^2 of the psi operator beyond (the
             targets state no bound for the pressure; measured at most
             3.8e-5 up to N = 128 and 3.7e-4 for rows of 512);
      X      1e-6 h (the stated target), or x_tol where the caller states why."""
    N = e["_N"]
    return {"u": 1e-5, "u_max": np.sqrt(2.0 * np.log(e["_M"])) * 1e-5,
            "p": 1e-4 * max(1.0, (1.0 + 4.0 * N * N) / (1.0 + 4.0 * 128 * 128)),
            "X": 1e-6 * h if x_tol is None else x_tol}


def assert_fp32(e, h, steps, x_tol=None):
    """Check errors e (from compare, or with the same keys) against fp32_bounds."""
    b = fp32_bounds(e, h, steps, x_tol)
    record(e, b)
    assert e["u"] < b["u"] and e["u_max"] < b["u_max"], (e, b)
    assert e["p"] < b["p"] and e["p_max"] < b["p"], (e, b)
    if "X" in e:
        assert e["X"] < b["X"], (e, b)


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


def test_fp64_full_size_ellipsoid_128_ten_steps():
    # the 128^3, nu=64 (40962-marker) membrane in the launch configuration the
    # benchmark times, through the first-step replacements and one full
    # rotation of the split order and beyond; the oracle needs about 2 s a step
    sc = I.ellipsoid_3d(n=128, nu=64)
    ora, g = make_pair(sc, "fp64")
    for k in (2, 8):
        ora.step(k)
        g.step(k)
        e = compare(ora, g)
        assert_fp64(e, ora.n)
        assert e["psi"] < psi_bound(sc, ora.n), e
    g.close()


def test_fp32_thin_ellipse_100_steps_error_vs_fp64_oracle():
    # FP32 fields with FP64 markers after the 100 steps of the 2D workload
    sc = I.thin_ellipse_2d(n=64, ns=256)
    ora, g = make_pair(sc, "fp32")
    ora.step(100)
    g.step(100)
    assert_fp32(compare(ora, g), 1.0 / 64, 100)
    g.close()


def test_nonfinite_velocity_is_reported_after_a_step():
    # one NaN cell planted in the initial velocity (host side) spreads through
    # the step's stencils and line solves; the device-side scan of
    # ib_diagnostics must report it
    sc = small_ellipsoid(n=16, nu=4)
    for prec in ("fp64", "fp32"):
        g = ib.Grid(3, 16, precision=prec, rotate_split=True)
        g.add_fiber(sc.X, sc.edges, sc.kappa, sc.rest, sc.tris)
        u0 = np.zeros((3, 16, 16, 16))
        u0[1, 5, 7, 3] = np.nan
        g.set_velocity(u0)
        g.step(1)
        d, rc = ib.ib_diagnostics(g.h, check=False)
        assert rc == ib.IB_ERR_NONFINITE, (prec, rc, d)
        with pytest.raises(ib.IBError) as ex:
            g.diagnostics()
        assert ex.value.code == ib.IB_ERR_NONFINITE
        g.close()
    # a finite state reports IB_OK
    g = ib.Grid(3, 16, precision="fp32", rotate_split=True)
    g.add_fiber(sc.X, sc.edges, sc.kappa, sc.rest, sc.tris)
    g.step(2)
    assert ib.ib_diagnostics(g.h, check=False)[1] == ib.IB_OK
    g.close()


def test_area_diagnostic_2d_matches_oracle_and_closed_form():
    # 2D volume diagnostic = area enclosed by the directed fiber loops
    # (Sec. 5.1): at n = 0 the ellipse polygon's closed form
    # r1 r2 (ns/2) sin(2 pi/ns), after steps the oracle's area of its markers
    sc = I.thin_ellipse_2d(n=64, ns=256)
    ora, g = make_pair(sc, "fp64")
    d0 = g.diagnostics()
    assert d0["volume"] == pytest.approx(0.2 * 0.25 * 128 * np.sin(2 * np.pi / 256), rel=1e-13)
    ora.step(20)
    g.step(20)
    assert g.diagnostics()["volume"] == pytest.approx(O.area_2d(ora.X, sc.edges), rel=1e-12)
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


def test_add_fiber_from_device_arrays():
    # the structure passed as device arrays (torch CUDA tensors) gives the same
    # steps as the same structure passed from host memory (to the rounding
    # of the spreading atomics' order, which differs from run to run)
    import torch

    sc = small_ellipsoid(n=32, nu=8)
    out = []
    for on_device in (False, True):
        g = ib.Grid(3, 32, rho=sc.rho, mu=sc.mu, dt=sc.dt, precision="fp64", rotate_split=True)
        arrs = (sc.X, sc.edges.astype(np.int32), sc.kappa, sc.rest, sc.tris.astype(np.int32))
        if on_device:
            arrs = tuple(torch.tensor(np.ascontiguousarray(a), device="cuda") for a in arrs)
        g.add_fiber(*arrs)
        g.step(3)
        out.append((g.velocity(), g.markers(), g.diagnostics()["volume"]))
        g.close()
    assert np.max(np.abs(out[0][1] - out[1][1])) < 1e-14
    assert out[0][2] == pytest.approx(out[1][2], rel=1e-13)
    assert rel(out[0][0], out[1][0]) < 1e-12


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_runs_of_steps_equal_single_steps(prec):
    # runs of several steps in one ib_step call (graph replays, the first step
    # enqueued directly) and single steps give the same states, to the
    # summation order of the spreading atomics
    sc = small_ellipsoid(n=32, nu=8)
    grids = []
    for _ in range(3):
        g = ib.Grid(3, 32, rho=sc.rho, mu=sc.mu, dt=sc.dt, precision=prec, rotate_split=True)
        g.add_fiber(sc.X, sc.edges, sc.kappa, sc.rest, sc.tris)
        grids.append(g)
    grids[0].step(9)
    for k in (3, 1, 5):
        grids[1].step(k)
    for _ in range(9):
        grids[2].step(1)
    ref = grids[2]
    # FP32 pressure: the psi operator's conditioning amplifies the atomics'
    # reordering (two identical FP32 runs differ in p by up to 1e-3)
    tol = {"u": 1e-12, "p": 1e-12} if prec == "fp64" else {"u": 1e-5, "p": 1e-3}
    for g in grids[:2]:
        assert g.diagnostics()["step"] == 9
        for k in ("u", "v", "w", "p"):
            assert rel(g.fields((k,))[k], ref.fields((k,))[k]) < tol["p" if k == "p" else "u"], k
        assert np.max(np.abs(g.markers() - ref.markers())) < (1e-13 if prec == "fp64" else 1e-8)
    for g in grids:
        g.close()
