"""Helpers shared by the tests that reproduce the paper's tables on the GPU:
runs of the thin ellipse (Sec. 5.1) and thick shell (Sec. 5.2) problems, the
discrete l2 norms of eqs. ScalarDiscreteL2 / VectorDiscreteL2, and the
fine-to-coarse transfer used by the convergence rate of eq. EstConvergence.

Transfer (the paper does not give it): a coarse cell-centred value is the
mean of its 2^d child cells; a coarse face value is the mean of the 2^(d-1)
fine faces on it; markers (N_s proportional to N) keep every other point
along each fiber.  The thick shell's fibers sit at the midpoints
r_l = (l + 1/2)/N_r, which do not nest under refinement: a coarse fiber is the
mean of the two fine fibers around it, and the Lagrangian norm carries the
weight h_s h_r.
"""
import numpy as np

import paper_1305_3976_gb300 as ib
from paper_1305_3976_gb300 import inputs as I


def thin_ellipse(N, sigma=1.0, dt=0.04 / 512, t=0.31, precision="fp64"):
    sc = I.thin_ellipse_2d(n=N, ns=19 * N // 4, r1=5 / 28, r2=7 / 20, mu=0.01, dt=dt, kernel="peskin4",
                           sigma=sigma)
    return run(sc, int(round(t / dt)), precision)


def thick_shell(N, mu=0.01, dt=0.08 / 512, t=0.4, precision="fp64", scheme="gm2", chi=0.6):
    sc = I.thick_shell_2d(n=N, mu=mu, dt=dt, t_end=t)
    sc.chi = chi
    return run(sc, sc.steps, precision, scheme)


def run(sc, steps, precision, scheme="gm2"):
    g = ib.Grid(2, sc.n, rho=sc.rho, mu=sc.mu, dt=sc.dt, chi=sc.chi, precision=precision, kernel=sc.kernel,
                rotate_split=True, scheme=scheme)
    g.add_fiber(sc.X, sc.edges, sc.kappa, sc.rest)
    g.step(steps)
    f = g.fields()
    out = {"u": np.stack([f["u"], f["v"]]), "p": f["p"], "div": f["div"], "X": g.markers(), "N": sc.n[0]}
    g.close()
    return out


def l2_cells(q, N):
    return float(np.sqrt(np.sum(np.asarray(q, dtype=np.float64) ** 2) / N ** 2))


def l2_markers(X, ns_per_fiber):
    # h_s sum |X_k|^2 with h_s = 1 / N_s (Euclidean norm over components)
    return float(np.sqrt(np.sum(np.asarray(X) ** 2) / ns_per_fiber))


def coarsen(r):
    """Fine (2N) solution -> coarse (N) grid."""
    u, p, X = r["u"], r["p"], r["X"]
    pc = 0.25 * (p[0::2, 0::2] + p[1::2, 0::2] + p[0::2, 1::2] + p[1::2, 1::2])
    uc = 0.5 * (u[0][0::2, 0::2] + u[0][1::2, 0::2])   # x-faces: x = 2i, y cells 2j, 2j+1
    vc = 0.5 * (u[1][0::2, 0::2] + u[1][0::2, 1::2])   # y-faces: y = 2j, x cells 2i, 2i+1
    return {"u": np.stack([uc, vc]), "p": pc, "X": X}


def coarse_markers(X, fibers, pair_fibers):
    """Fine markers (fibers x 2n points) -> coarse (every other point; with
    pair_fibers the mean of fine fibers 2l and 2l+1)."""
    n = X.shape[0] // fibers
    Y = X.reshape(fibers, n, -1)[:, 0::2, :]
    if pair_fibers:
        Y = 0.5 * (Y[0::2] + Y[1::2])
    return Y.reshape(-1, X.shape[1])


def rate(r1, r2, r4, fibers=1, thick=False):
    """R[q; N] for q in u, p, X (eq. EstConvergence).  fibers: number of
    fibers at resolution N (doubles with N when thick)."""
    N = r1["N"]
    c2, c4 = coarsen(r2), coarsen(r4)
    out = {}
    for q in ("u", "p"):
        num = l2_cells(r1[q] - c2[q], N)
        den = l2_cells(r2[q] - c4[q], 2 * N)
        out[q] = float(np.log2(num / den))
    f2 = 2 * fibers if thick else fibers
    ns1 = r1["X"].shape[0] // fibers
    w1 = 1.0 / (ns1 * fibers) if thick else 1.0 / ns1          # h_s (h_r)
    w2 = w1 / 4 if thick else w1 / 2
    num = np.sqrt(w1 * np.sum((r1["X"] - coarse_markers(r2["X"], f2, thick)) ** 2))
    den = np.sqrt(w2 * np.sum((r2["X"] - coarse_markers(r4["X"], 2 * f2 if thick else fibers, thick)) ** 2))
    out["X"] = float(np.log2(num / den))
    return out


def thin_ellipse_area_history(N, dt, t_end=4.0, t_fit=2.0, sample=0.05, precision="fp64"):
    """Relative area loss (A0 - A(t)) / A0 of the thin ellipse (sigma = 1,
    Sec. 5.1) sampled every `sample` time units from t_fit to t_end, and the
    final marker positions.  A is the area enclosed by the fiber (signed
    shoelace sum over its connections, ib_diagnostics), A0 = pi r1 r2."""
    r1, r2 = 5 / 28, 7 / 20
    sc = I.thin_ellipse_2d(n=N, ns=19 * N // 4, r1=r1, r2=r2, mu=0.01, dt=dt, kernel="peskin4", sigma=1.0)
    g = ib.Grid(2, sc.n, rho=sc.rho, mu=sc.mu, dt=dt, precision=precision, kernel="peskin4", rotate_split=True)
    g.add_fiber(sc.X, sc.edges, sc.kappa, sc.rest)
    A0 = np.pi * r1 * r2
    total, chunk = int(round(t_end / dt)), int(round(sample / dt))
    ts, loss = [], []
    done = 0
    while done < total:
        g.step(chunk)
        done += chunk
        if done * dt >= t_fit - 1e-9:
            ts.append(done * dt)
            loss.append((A0 - g.diagnostics()["volume"]) / A0)
    X = g.markers()
    g.close()
    return np.array(ts), np.array(loss), X
