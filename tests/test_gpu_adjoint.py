"""Discrete adjoint of the step (ib_adjoint_run) against finite differences.

The adjoint differentiates loss = sum_k |X_k^n - T_k|^2 after n steps with
respect to every connection stiffness kappa_e.  Its pins are independent of
the adjoint code:
  - central differences of the FP64 oracle's loss on small 2D and 3D problems
    (the oracle shares no code with the CUDA path);
  - central differences of the FP64 GPU forward (ib_step) at the 96^3,
    7842-marker problem, 200 steps, checkpoints every 20 steps, on 16 seeded
    connections, step eps = 1e-4 in kappa.
FD error: the truncation term is O(eps^2) relative; the rounding term is
~ 1e-16 L / eps.  Bounds: |adjoint - FD| <= 1e-4 max|FD| over the sample
(plus the rounding term), and a loss equal to the forward's to 1e-12.
FP32 fields: the adjoint of the FP32 path is compared with the FP64 gradient
(norm-wise relative error, bound stated below with the measured value).
"""
import numpy as np
import pytest

import oracle as O
import paper_1305_3976_gb300 as ib
from paper_1305_3976_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def grid_of(sc, kappa=None, precision="fp64", rotate=True):
    g = ib.Grid(sc.dim, sc.n, H=sc.H, rho=sc.rho, mu=sc.mu, dt=sc.dt, chi=sc.chi, precision=precision,
                kernel=sc.kernel, rotate_split=rotate)
    g.add_fiber(sc.X, sc.edges, sc.kappa if kappa is None else kappa, sc.rest, sc.tris)
    return g


def loss_of(X, T):
    return float(np.sum((X - T) ** 2))


def oracle_loss(sc, kappa, steps, rotate=True):
    P = O.params(sc.dim, sc.n, H=sc.H, rho=sc.rho, mu=sc.mu, dt=sc.dt, chi=sc.chi, kernel=sc.kernel,
                 rotate=rotate)
    ora = O.Simulation(P, sc.X, sc.edges, kappa, sc.rest)
    ora.step(steps)
    return loss_of(ora.X, sc.extra["target"])


def gpu_loss(sc, kappa, steps, precision="fp64"):
    g = grid_of(sc, kappa, precision)
    g.step(steps)
    L = loss_of(g.markers(), sc.extra["target"])
    g.close()
    return L


def fd_check(sc, steps, ck, edges, loss_fn, rel_eps=1e-4):
    g = grid_of(sc)
    L, dk = g.adjoint(steps, sc.extra["target"], ck)
    g.close()
    fd = []
    for e in edges:
        h = rel_eps * sc.kappa[e]
        kp, km = sc.kappa.copy(), sc.kappa.copy()
        kp[e] += h
        km[e] -= h
        fd.append((loss_fn(sc, kp, steps) - loss_fn(sc, km, steps)) / (2 * h))
    return L, dk, np.array(fd)


def test_adjoint_2d_against_oracle_differences():
    sc = I.stiffness_fit_2d(n=32, ns=64, steps=12)
    edges = np.random.default_rng(7).choice(sc.edges.shape[0], 8, replace=False)
    L, dk, fd = fd_check(sc, 12, 5, edges, oracle_loss)           # segments of 5, 5, 2 steps
    assert abs(L - oracle_loss(sc, sc.kappa, 12)) <= 1e-12 * L
    err = np.max(np.abs(dk[edges] - fd))
    assert err <= 1e-4 * np.max(np.abs(fd)), (dk[edges], fd)


@pytest.mark.parametrize("kernel", ["peskin4", "cos4"])
def test_adjoint_3d_against_oracle_differences(kernel):
    sc = I.stiffness_fit_3d(n=16, nu=4, steps=6, kernel=kernel)   # 162 markers, 480 connections
    edges = np.random.default_rng(8).choice(sc.edges.shape[0], 6, replace=False)
    L, dk, fd = fd_check(sc, 6, 4, edges, oracle_loss)
    assert abs(L - oracle_loss(sc, sc.kappa, 6)) <= 1e-12 * L
    err = np.max(np.abs(dk[edges] - fd))
    assert err <= 1e-4 * np.max(np.abs(fd)), (dk[edges], fd)


def test_adjoint_leaves_the_forward_state_and_ignores_checkpoint_spacing():
    sc = I.stiffness_fit_3d(n=24, nu=6, steps=9)
    ref = grid_of(sc)
    ref.step(9)
    Xr, fr = ref.markers(), ref.fields()
    ref.close()
    grads = []
    for ck in (1, 4, 9, 50):
        g = grid_of(sc)
        L, dk = g.adjoint(9, sc.extra["target"], ck)
        X, f = g.markers(), g.fields()
        assert g.diagnostics()["step"] == 9
        g.close()
        assert np.max(np.abs(X - Xr)) < 1e-14
        assert abs(L - loss_of(Xr, sc.extra["target"])) <= 1e-13 * L
        for k in ("u", "v", "w", "p"):
            assert np.max(np.abs(f[k] - fr[k])) <= 1e-12 * max(1.0, np.max(np.abs(fr[k])))
        grads.append(dk)
    for dk in grads[1:]:
        assert np.max(np.abs(dk - grads[0])) <= 1e-10 * np.max(np.abs(grads[0]))


def test_adjoint_window_starting_after_the_first_step():
    # a grid already at step 4: the adjoint differentiates steps 4..9 only
    # (kappa perturbed in those steps, state at step 4 held), which the
    # oracle reproduces by changing its stiffnesses after 4 steps
    sc = I.stiffness_fit_2d(n=32, ns=64, steps=10)
    edges = [3, 17, 40]
    P = O.params(sc.dim, sc.n, H=sc.H, rho=sc.rho, mu=sc.mu, dt=sc.dt, chi=sc.chi, kernel=sc.kernel, rotate=True)

    def windowed(kappa):
        ora = O.Simulation(P, sc.X, sc.edges, sc.kappa, sc.rest)
        ora.step(4)
        ora.kappa[:] = kappa
        ora.step(6)
        return loss_of(ora.X, sc.extra["target"])

    g = grid_of(sc)
    g.step(4)
    L, dk = g.adjoint(6, sc.extra["target"], 4)                   # segments of 4 and 2 steps
    g.close()
    assert abs(L - windowed(sc.kappa)) <= 1e-12 * L
    fd = []
    for e in edges:
        h = 1e-4 * sc.kappa[e]
        kp, km = sc.kappa.copy(), sc.kappa.copy()
        kp[e] += h
        km[e] -= h
        fd.append((windowed(kp) - windowed(km)) / (2 * h))
    fd = np.array(fd)
    assert np.max(np.abs(dk[edges] - fd)) <= 1e-4 * np.max(np.abs(fd)), (dk[edges], fd)


def test_adjoint_full_size_fp64_against_gpu_differences():
    sc = I.stiffness_fit_3d()                                     # 96^3, 7842 markers, 23520 connections
    assert sc.X.shape[0] == 7842 and sc.edges.shape[0] == 23520
    edges = np.random.default_rng(5).choice(sc.edges.shape[0], 16, replace=False)
    g = grid_of(sc)
    L, dk = g.adjoint(sc.steps, sc.extra["target"], 20)
    g.close()
    fd = []
    for e in edges:
        kp, km = sc.kappa.copy(), sc.kappa.copy()
        kp[e] += 1e-4
        km[e] -= 1e-4
        fd.append((gpu_loss(sc, kp, sc.steps) - gpu_loss(sc, km, sc.steps)) / 2e-4)
    fd = np.array(fd)
    err = np.abs(dk[edges] - fd)
    assert np.max(err) <= 1e-4 * np.max(np.abs(fd)) + 1e-16 * L / 1e-4 * 4, (dk[edges], fd)


def test_adjoint_fp32_against_fp64_gradient():
    # FP32 fields (FP64 markers, FP64 gradient accumulation) at the full size
    sc = I.stiffness_fit_3d()
    g = grid_of(sc, precision="fp64")
    L64, dk64 = g.adjoint(sc.steps, sc.extra["target"], 20)
    g.close()
    g = grid_of(sc, precision="fp32")
    L32, dk32 = g.adjoint(sc.steps, sc.extra["target"], 20)
    g.close()
    assert abs(L32 - L64) <= 1e-5 * L64
    e = np.linalg.norm(dk32 - dk64) / np.linalg.norm(dk64)
    assert e < 1e-5, e                                          # measured 3.6e-7


def test_kappa_loss_autograd():
    torch = pytest.importorskip("torch")
    sc = I.stiffness_fit_2d(n=32, ns=64, steps=8)

    def build(kap):
        return grid_of(sc, kap)

    kap = torch.tensor(sc.kappa, dtype=torch.float64, requires_grad=True)
    loss = ib.kappa_loss(kap, build, 8, sc.extra["target"], 3)
    (3.0 * loss).backward()
    g = grid_of(sc)
    L, dk = g.adjoint(8, sc.extra["target"], 8)
    g.close()
    assert abs(loss.item() - L) <= 1e-13 * L
    assert np.max(np.abs(kap.grad.numpy() - 3.0 * dk)) <= 1e-10 * np.max(np.abs(dk))


def test_adjoint_rejects_rest_lengths_and_bad_spacing():
    sc = I.thin_ellipse_2d(n=32, ns=64, rest_length=1.0)
    sc.extra["target"] = sc.X.copy()
    g = grid_of(sc)
    with pytest.raises(ib.IBError) as ex:
        g.adjoint(2, sc.extra["target"], 1)
    assert ex.value.code == ib.IB_ERR_ARG
    g.close()
    sc = I.stiffness_fit_2d(n=32, ns=64)
    g = grid_of(sc)
    with pytest.raises(ib.IBError):
        g.adjoint(2, sc.extra["target"], 0)
    L, dk = g.adjoint(0, sc.extra["target"], 1)
    assert L == pytest.approx(loss_of(sc.X, sc.extra["target"]), rel=1e-15) and not np.any(dk)
    g.close()
