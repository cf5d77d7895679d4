"""ib_split_solve_noalloc, the allocation-free variant of ib_split_solve for
callers that cannot allocate device memory (their device memory belongs to
another allocator, or their loop must not call cudaMalloc because it
synchronises the device), against ib_split_solve, through the C ABI.

Two calls in a row with different sizes, coefficients and precisions: the
fixed scratch array inside the library is shared by all calls, so the second
call must not see anything the first one left behind.  The results are also
checked against the FP64 oracle's Schur-complement line solves (Sec. 4.2) and
against the closed form of the paper's Poisson-comparison problem (Sec. 6.1,
one Fourier mode), and a call with line coefficients never seen before must
leave the device's free memory unchanged.  The tolerance is the one of the
line-solve parity tests.  This file is collected last so that a run stopping
at the first failure has already run every other test; it also passes on its
own in a fresh process.
"""
import numpy as np
import pytest
import torch

import oracle as O
import paper_1305_3976_gb300 as ib

pytestmark = pytest.mark.gpu

EPS = {ib.IB_FP32: 2.0 ** -24, ib.IB_FP64: 2.0 ** -53}
TORCH = {ib.IB_FP32: torch.float32, ib.IB_FP64: torch.float64}


def _tol(prec, n, r):
    return 4.0 * n * EPS[prec] * (1.0 + 4.0 * r)


CALLS = [
    (ib.IB_FP32, 3, (128, 96, 64), (128.0 ** 2, 96.0 ** 2, 64.0 ** 2)),
    (ib.IB_FP64, 3, (50, 37, 29), (0.2048, 0.31, 0.05)),
    (ib.IB_FP64, 2, (512, 24), (512.0 ** 2, 0.7)),
]


def test_noalloc_matches_split_solve_on_consecutive_calls():
    g = np.random.default_rng(2024)
    for prec, dim, n, r in CALLS:
        shape = tuple(reversed(n[:dim]))
        f = torch.tensor(g.standard_normal(shape), dtype=TORCH[prec], device="cuda")
        ref = torch.empty_like(f)
        got = torch.full_like(f, float("nan"))
        ib.ib_split_solve(prec, dim, n, r, f, ref)
        ib.ib_split_solve_noalloc(prec, dim, n, r, f, got)
        torch.cuda.synchronize()
        a, b = got.double().cpu().numpy(), ref.double().cpu().numpy()
        assert np.all(np.isfinite(a))
        err = np.max(np.abs(a - b)) / np.max(np.abs(b))
        tol = max(_tol(prec, n[q], r[q]) for q in range(dim))
        assert err < tol, (prec, n, err, tol)


def test_noalloc_rejects_lines_beyond_its_fixed_scratch():
    f = torch.zeros(16, 16, 520, device="cuda")
    with pytest.raises(ib.IBError) as ex:
        ib.ib_split_solve_noalloc(ib.IB_FP32, 3, (520, 16, 16), (1.0, 1.0, 1.0), f, f)
    assert ex.value.code == ib.IB_ERR_ARG
    assert "512" in str(ex.value)


@pytest.mark.parametrize("prec", [ib.IB_FP64, ib.IB_FP32], ids=["fp64", "fp32"])
def test_noalloc_matches_the_oracle_line_solves(prec):
    # (I - r0 D2_x)(I - r1 D2_y)(I - r2 D2_z) psi = f as three oracle line solves
    n, r = (48, 40, 36), (48.0 ** 2, 0.37, 40.0 ** 2)
    P = O.params(3, n)
    f = np.random.default_rng(77).standard_normal(O.field_shape(P))
    if prec == ib.IB_FP32:
        f = f.astype(np.float32).astype(np.float64)
    ref = f
    for a in range(3):
        ref = O.solve_lines(P, a, r[a], ref)
    fd = torch.tensor(f, dtype=TORCH[prec], device="cuda")
    for _ in range(2):
        got = torch.full_like(fd, float("nan"))
        ib.ib_split_solve_noalloc(prec, 3, n, r, fd, got)
        torch.cuda.synchronize()
        err = np.max(np.abs(got.double().cpu().numpy() - ref)) / np.max(np.abs(ref))
        assert err < max(_tol(prec, n[q], r[q]) for q in range(3)), err


@pytest.mark.parametrize("prec", [ib.IB_FP64, ib.IB_FP32], ids=["fp64", "fp32"])
def test_noalloc_poisson_comparison_closed_form(prec):
    # Sec. 6.1: f = sin 2 pi x cos 2 pi y cos 2 pi z is one Fourier mode of the
    # grid, so psi = f / prod_a (1 + 4 N^2 sin^2(pi / N)) exactly
    N = 128
    x = (np.arange(N) + 0.5) / N
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    f = np.sin(2 * np.pi * X) * np.cos(2 * np.pi * Y) * np.cos(2 * np.pi * Z)
    exact = f / (1 + 4 * N * N * np.sin(np.pi / N) ** 2) ** 3
    fd = torch.tensor(f, dtype=TORCH[prec], device="cuda")
    psi = torch.empty_like(fd)
    ib.ib_split_solve_noalloc(prec, 3, (N, N, N), (N * N,) * 3, fd, psi)
    torch.cuda.synchronize()
    err = np.max(np.abs(psi.double().cpu().numpy() - exact)) / np.max(np.abs(exact))
    assert err < 3 * _tol(prec, N, N * N), err


def test_noalloc_leaves_device_memory_unchanged():
    # every buffer is made first; one call loads the kernels; then a call with
    # (n, r) that no other call of this process used must not change the
    # device's free memory (ib_split_solve would build a new table of powers)
    n = (96, 40, 56)
    f = torch.randn(56, 40, 96, device="cuda")
    out = torch.empty_like(f)
    ib.ib_split_solve_noalloc(ib.IB_FP32, 3, n, (1.5, 2.5, 3.5), f, out)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    ib.ib_split_solve_noalloc(ib.IB_FP32, 3, n, (123.25, 0.0625, 77.75), f, out)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert torch.isfinite(out).all()
