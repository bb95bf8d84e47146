"""Seeded synthetic inputs shared by the tests, smoke() and bench.py.

This module builds input matrices and right-hand sides only; it contains none
of the factorization's arithmetic.  The paper times "randomly generated
symmetric positive-definite matrices" without fixing a construction (Section
4); the constructions below are the ones the workloads name:

* ``gram_plus_identity``: A = G G^T / n + I, G i.i.d. N(0, 1)
  (eigenvalues in about [1, 5], well conditioned);
* ``se_covariance``: squared-exponential covariance of n points uniform in the
  unit square, exp(-|x_i - x_j|^2 / (2 l^2)) + nugget * delta_ij, the kernel
  matrix of Gaussian-process regression named in Section 1;
* ``pascal``: the symmetric Pascal matrix C(i+j, i), whose factor is the lower
  Pascal matrix C(i, j) exactly for n <= 29;
* ``exact_integer_factor``: A = L0 L0^T with small-integer L0 (diagonal in
  {1, 2, 4}), so every intermediate of any factorization order is an integer
  and the factor is L0 exactly;
* ``tridiag``: the [-1, 2, -1] matrix, whose factor has a closed form.

All matrices are returned as Fortran-ordered float64 numpy arrays (full
symmetric storage; the library reads only the lower triangle).  The ``*_torch``
variants build the same kind of matrix directly in device memory for sizes
whose host construction would be too slow; they take the seed through
``torch.Generator`` and so draw different numbers than the numpy variants.
"""
from __future__ import annotations

import math

import numpy as np


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def _sym_from_lower(A: np.ndarray) -> np.ndarray:
    L = np.tril(A)
    return np.asfortranarray(L + np.tril(L, -1).T)


def gram_plus_identity(n: int, seed: int = 0) -> np.ndarray:
    G = rng(seed).standard_normal((n, n))
    A = G @ G.T / n + np.eye(n)
    return _sym_from_lower(A)


def se_points(n: int, seed: int = 1) -> np.ndarray:
    return rng(seed).uniform(0.0, 1.0, size=(n, 2))


def se_covariance(n: int, seed: int = 1, lengthscale: float = 0.1, nugget: float = 1e-2) -> np.ndarray:
    x = se_points(n, seed)
    d2 = ((x[:, None, :] - x[None, :, :]) ** 2).sum(-1)
    A = np.exp(-d2 / (2.0 * lengthscale * lengthscale)) + nugget * np.eye(n)
    return _sym_from_lower(A)


def pascal(n: int) -> np.ndarray:
    P = np.empty((n, n), dtype=np.float64, order="F")
    for i in range(n):
        for j in range(n):
            P[i, j] = float(math.comb(i + j, i))
    return P


def pascal_lower(n: int) -> np.ndarray:
    L = np.zeros((n, n), dtype=np.float64, order="F")
    for i in range(n):
        for j in range(i + 1):
            L[i, j] = float(math.comb(i, j))
    return L


def exact_integer_L0(n: int, seed: int = 5, band: int | None = None) -> np.ndarray:
    """Lower-triangular L0: diagonal drawn from {1, 2, 4}, entries below it from
    {-2, ..., 2}; with ``band`` only the first ``band`` subdiagonals are set."""
    r = rng(seed)
    L = np.tril(r.integers(-2, 3, size=(n, n)).astype(np.float64), -1)
    if band is not None:
        L = np.triu(L, -band)
    np.fill_diagonal(L, r.choice(np.array([1.0, 2.0, 4.0]), size=n))
    return np.asfortranarray(L)


def exact_integer_factor(n: int, seed: int = 5, band: int | None = None):
    """Return (A, L0) with A = L0 L0^T formed exactly (integer products and
    sums well below 2^53 are exact in float64 in any order)."""
    L0 = exact_integer_L0(n, seed, band)
    A = L0 @ L0.T
    return _sym_from_lower(A), L0


def tridiag(n: int) -> np.ndarray:
    A = 2.0 * np.eye(n) - np.eye(n, k=1) - np.eye(n, k=-1)
    return np.asfortranarray(A)


def rhs(n: int, nrhs: int, seed: int = 2) -> np.ndarray:
    return np.asfortranarray(rng(seed).standard_normal((n, nrhs)))


def batched_sizes(count: int = 4096, seed: int = 3, lo: int = 32, hi: int = 2048) -> np.ndarray:
    """n_i = floor(exp(U(ln lo, ln hi))), i.e. log-uniform in [lo, hi]."""
    u = rng(seed).uniform(math.log(lo), math.log(hi), size=count)
    return np.clip(np.floor(np.exp(u)).astype(np.int64), lo, hi)


# --------------------------------------------------------------------------
# device-side builders (torch only; used for sizes where host construction is
# too slow).  They return column-major storage as a torch tensor of shape
# (n, n) whose memory is the Fortran layout (i.e. the transpose view of a
# C-contiguous buffer); for a symmetric matrix both views hold the same bytes.
# --------------------------------------------------------------------------

def se_covariance_torch(n: int, seed: int = 1, lengthscale: float = 0.1, nugget: float = 1e-2,
                        device="cuda", chunk: int = 4096):
    import torch

    x = torch.from_numpy(se_points(n, seed)).to(device)
    A = torch.empty((n, n), dtype=torch.float64, device=device)
    inv = -1.0 / (2.0 * lengthscale * lengthscale)
    for s in range(0, n, chunk):
        e = min(n, s + chunk)
        d2 = ((x[s:e, None, :] - x[None, :, :]) ** 2).sum(-1)
        A[s:e] = torch.exp(d2 * inv)
    A.diagonal().add_(nugget)
    return A


def gram_plus_identity_torch(n: int, seed: int = 0, device="cuda"):
    import torch

    g = torch.Generator(device=device)
    g.manual_seed(seed)
    G = torch.randn((n, n), dtype=torch.float64, device=device, generator=g)
    A = G @ G.T / n
    A = torch.tril(A) + torch.tril(A, -1).T
    A.diagonal().add_(1.0)
    return A


def exact_integer_band_torch(n: int, band: int, seed: int = 5, device="cuda"):
    """Banded exact-integer pair (A, L0) built in O(n * band^2) host work and
    expanded on the device.  Returns (A, L0) as device tensors in the
    column-major convention above (A symmetric; L0 returned as its own
    column-major buffer, i.e. tensor.T of the row-major array)."""
    import torch

    r = rng(seed)
    # Lb[i, d] = L0[i, i - d] for d = 0..band
    Lb = r.integers(-2, 3, size=(n, band + 1)).astype(np.float64)
    Lb[:, 0] = r.choice(np.array([1.0, 2.0, 4.0]), size=n)
    for d in range(1, band + 1):
        Lb[:d, d] = 0.0
    # Ab[i, e] = A[i, i - e] = sum_{d >= e} L0[i, i-d] L0[i-e, i-d]
    Ab = np.zeros((n, band + 1))
    for e in range(band + 1):
        for d in range(e, band + 1):
            # L0[i-e, i-d] = Lb[i-e, d-e]
            Ab[e:, e] += Lb[e:, d] * Lb[: n - e, d - e]
    i = torch.arange(n, device=device)
    A = torch.zeros((n, n), dtype=torch.float64, device=device)
    L = torch.zeros((n, n), dtype=torch.float64, device=device)
    Abt = torch.from_numpy(Ab).to(device)
    Lbt = torch.from_numpy(Lb).to(device)
    for e in range(band + 1):
        rows = i[e:]
        cols = rows - e
        # column-major element (r, c) of A is row-major element (c, r)
        A[cols, rows] = Abt[e:, e]
        A[rows, cols] = Abt[e:, e]
        L[cols, rows] = Lbt[e:, e]
    return A, L
