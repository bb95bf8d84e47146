"""The refinement residual R = B - A X on the tensor cores (exact bf16
slicing of A per 128 x 128 tile and of X per 128-row block and column).

* integer inputs: every slice product and every partial sum is exact, so R
  must equal the exact residual bit for bit (ragged n, two column chunks);
* binary64 inputs, uniform and graded scales: on sampled entries the result
  is compared with the exact rational residual; the error must stay below
  2^-45 sum_J 2^(e_r + e_c) plus (3 Mt + 4) u (|b| + |A||x|).  Per product
  the omitted slice products (s + t >= 10, at most 7 of 2^-56 each) and the
  two slicing remainders (below 2^-56 each) add up to less than 1.25 2^-53
  times 2^(e_r + e_c) (e_r, e_c the exponents of the row of tile (I, J) and
  of the column of block J), so less than 1.25 2^-46 2^(e_r + e_c) per tile
  of 128 products; each tile's contribution is added with two binary64
  roundings, and at most Mt partial sums plus B are combined at the end;
* B omitted gives -A X; only the lower triangle of A is read (the upper is
  filled with NaN).
"""
from fractions import Fraction

import numpy as np
import pytest

import seeded_inputs as si

pytestmark = pytest.mark.gpu

U = 2.0 ** -53


def _run(A, X, B):
    import torch

    import paper_2606_11937_gb300 as chol
    n, nrhs = X.shape
    Al = np.tril(A).copy()
    Al[np.triu_indices(n, 1)] = np.nan  # the kernel must not read the upper triangle
    dA = chol.colmajor(Al)
    dX = chol.colmajor(X)
    dB = chol.colmajor(B) if B is not None else None
    dR = torch.empty_strided((n, nrhs), (1, n), dtype=torch.float64, device="cuda")
    rc = chol.lib().chol_test_oz_residual(n, dA.data_ptr(), n, dX.data_ptr(), n,
                                          dB.data_ptr() if dB is not None else None, n, dR.data_ptr(), n, nrhs)
    assert rc == 0, chol.chol_last_error()
    return dR.cpu().numpy()


@pytest.mark.parametrize("n,nrhs", [(700, 17), (1024, 1), (300, 5)])
def test_residual_exact_on_integers(n, nrhs):
    r = si.rng(10 + n)
    L = r.integers(-1000, 1001, size=(n, n))
    A = np.tril(L) + np.tril(L, -1).T  # symmetric integer matrix
    X = r.integers(-1000, 1001, size=(n, nrhs))
    B = r.integers(-10 ** 9, 10 ** 9, size=(n, nrhs))
    want = B - A @ X  # int64, exact (|.| < 2^53)
    got = _run(A.astype(np.float64), X.astype(np.float64), B.astype(np.float64))
    assert np.array_equal(got, want.astype(np.float64))
    got0 = _run(A.astype(np.float64), X.astype(np.float64), None)
    assert np.array_equal(got0, (-(A @ X)).astype(np.float64))


def _exact(A, X, B, i, c):
    s = Fraction(B[i, c]) if B is not None else Fraction(0)
    for k in range(A.shape[0]):
        s -= Fraction(A[i, k]) * Fraction(X[k, c])
    return s


def _tile_bound(A, X):
    """sum_J 2^(e_r + e_c) per (row, column): e_r from the row of tile (I, J),
    e_c from column c of block J."""
    n, nrhs = X.shape
    Mt = -(-n // 128)
    out = np.zeros((n, nrhs))
    for J in range(Mt):
        a = np.abs(A[:, J * 128:(J + 1) * 128]).max(axis=1)
        x = np.abs(X[J * 128:(J + 1) * 128, :]).max(axis=0)
        er = np.where(a > 0, np.frexp(a)[1], -1100).astype(np.float64)
        ec = np.where(x > 0, np.frexp(x)[1], -1100).astype(np.float64)
        out += np.exp2(er[:, None] + ec[None, :])
    return out


@pytest.mark.parametrize("scale", ["uniform", "graded"])
@pytest.mark.parametrize("n,nrhs", [(1500, 3), (1200, 20)])
def test_residual_binary64_accuracy(scale, n, nrhs):
    r = si.rng(20 + nrhs)
    A = si.se_covariance(n, seed=3, nugget=1e-2)
    X = r.standard_normal((n, nrhs))
    if scale == "graded":  # rows / columns and right-hand sides over many binades
        d = np.exp2(r.integers(-20, 21, size=n).astype(np.float64))
        A = d[:, None] * A * d[None, :]
        X = X * np.exp2(r.integers(-20, 21, size=(n, 1)).astype(np.float64))
    B = A @ X + 1e-3 * r.standard_normal((n, nrhs)) * np.abs(A @ X).max()
    got = _run(A, X, B)
    Mt = -(-n // 128)
    absax = np.abs(A) @ np.abs(X)
    tb = _tile_bound(A, X)
    # coarse check everywhere against the binary64 product (its own error is
    # below n u |A||x|)
    ref = B - A @ X
    tol_all = 2.0 ** -45 * tb + (n + 3 * Mt + 4) * U * (np.abs(B) + absax)
    assert np.all(np.abs(got - ref) <= tol_all), float(np.max(np.abs(got - ref) / tol_all))
    # exact rational reference on sampled entries
    idx = [(int(i), int(c)) for i, c in zip(r.integers(0, n, 24), r.integers(0, nrhs, 24))]
    idx += [(n - 1, nrhs - 1), (0, 0), (127, 0), (128, nrhs - 1)]
    for i, c in idx:
        ex = _exact(A, X, B, i, c)
        err = abs(Fraction(got[i, c]) - ex)
        tol = 2.0 ** -45 * tb[i, c] + (3 * Mt + 4) * U * (abs(B[i, c]) + absax[i, c])
        assert err <= Fraction(tol), (i, c, float(err), tol)
