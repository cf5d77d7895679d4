"""ib_split_solve_noalloc, the allocation-free variant of ib_split_solve for
callers that cannot allocate device memory (their device memory belongs to
another allocator, or their loop must not call cudaMalloc because it
synchronises the device), against ib_split_solve, through the C ABI.

Two calls in a row with different sizes, coefficients and precisions: the
fixed scratch array inside the library is shared by all calls, so the second
call must not see anything the first one left behind.  The tolerance is the
one of the line-solve parity tests (both entry points run the same sweeps;
only the tables of powers are computed differently).  This file is collected
last so that a run stopping at the first failure has already run every other
test; it also passes on its own in a fresh process.
"""
import numpy as np
import pytest
import torch

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
