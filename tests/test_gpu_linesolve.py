"""GPU line solves (ib_cyclic_solve_lines / ib_split_solve, through the C ABI)
against the FP64 oracle's Schur-complement solve (Sec. 4.2) on seeded inputs.

Tolerance (derived from the arithmetic): both sides are backward-stable
solvers of A x = b with A = (1+2r) I - r (S + S^-1), whose condition number
is at most 1 + 4r.  A relative backward error of c n eps turns into a forward
error of at most (1 + 4r) c n eps.  We use c = 4 on ||x_gpu - x_ref||_inf /
||x_ref||_inf, with eps the unit roundoff of the GPU precision (the FP64
oracle's own error is 2^-53 times the same factor, below the FP32 bound).
"""
import numpy as np
import pytest
import torch

import oracle as O
import paper_1305_3976_gb300 as ib

pytestmark = pytest.mark.gpu

EPS = {ib.IB_FP32: 2.0 ** -24, ib.IB_FP64: 2.0 ** -53}
TORCH = {ib.IB_FP32: torch.float32, ib.IB_FP64: torch.float64}

SHAPES = [
    (2, (8, 8)), (2, (64, 48)), (2, (512, 16)), (2, (16, 512)), (2, (130, 72)),
    (3, (8, 8, 8)), (3, (48, 40, 36)), (3, (50, 37, 29)), (3, (96, 64, 48)),
    (3, (128, 128, 128)), (3, (256, 24, 16)), (3, (24, 256, 16)), (3, (16, 24, 264)),
]


def _tol(prec, n, r):
    return 4.0 * n * EPS[prec] * (1.0 + 4.0 * r)


@pytest.mark.parametrize("prec", [ib.IB_FP64, ib.IB_FP32], ids=["fp64", "fp32"])
@pytest.mark.parametrize("dim,n", SHAPES, ids=[f"{d}d_{'x'.join(map(str, n))}" for d, n in SHAPES])
def test_cyclic_solve_lines_vs_oracle(dim, n, prec):
    P = O.params(dim, n)
    g = np.random.default_rng(sum(n) + dim)
    b = g.standard_normal(O.field_shape(P))
    bd = torch.tensor(b, dtype=TORCH[prec], device="cuda")
    for axis in range(dim):
        for r in (0.2048, float(n[axis]) ** 2):
            ref = O.solve_lines(P, axis, r, b.astype(np.float32).astype(np.float64) if prec == ib.IB_FP32 else b)
            out = torch.empty_like(bd)
            ib.ib_cyclic_solve_lines(prec, dim, n, axis, r, bd, out)
            # in place must give the same answer
            inpl = bd.clone()
            ib.ib_cyclic_solve_lines(prec, dim, n, axis, r, inpl, inpl)
            torch.cuda.synchronize()
            got = out.double().cpu().numpy()
            err = np.max(np.abs(got - ref)) / np.max(np.abs(ref))
            assert err < _tol(prec, n[axis], r), (axis, r, err)
            assert torch.equal(out, inpl)


@pytest.mark.parametrize("prec", [ib.IB_FP64, ib.IB_FP32], ids=["fp64", "fp32"])
def test_split_solve_poisson_comparison_mode(prec):
    # Sec. 6.1: (1 - D_xx)(1 - D_yy)(1 - D_zz) psi = sin 2 pi x cos 2 pi y cos 2 pi z;
    # on the grid the right-hand side is one Fourier mode, so
    # psi = f / prod_a (1 + 4 n^2 sin^2(pi / n))
    N = 128
    x = (np.arange(N) + 0.5) / N
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    f = np.sin(2 * np.pi * X) * np.cos(2 * np.pi * Y) * np.cos(2 * np.pi * Z)
    lam = (1 + 4 * N * N * np.sin(np.pi / N) ** 2) ** 3
    fd = torch.tensor(f, dtype=TORCH[prec], device="cuda")
    psi = torch.empty_like(fd)
    ib.ib_split_solve(prec, 3, (N, N, N), (N * N, N * N, N * N), fd, psi)
    torch.cuda.synchronize()
    err = np.max(np.abs(psi.double().cpu().numpy() - f / lam)) / np.max(np.abs(f / lam))
    assert err < 3 * _tol(prec, N, N * N), err
