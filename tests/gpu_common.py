"""Helpers shared by the GPU tests: device copies, oracle results cached per
input, and the error measures the tolerances are stated in."""
import functools
import math

import numpy as np

import oracle
import seeded_inputs as si

# Tolerances (stated once, used by every FP64 parity test):
#  * scaled entrywise error  max_{i>=j} |L_ij - L*_ij| / sqrt(A_ii) <= 1e-11
#    (row i of L has 2-norm sqrt(A_ii), so this is the entrywise error
#    relative to the row's scale; plain |dL|/|L*| is undefined for zeros);
#  * residual ||A - L L^T||_F / ||A||_F <= 1e-14 sqrt(n), or its randomized
#    estimate with Gaussian probe vectors where the exact product is too slow.
TOL_SCALED = 1e-11
TOL_RESID = 1e-14


def scaled_error(L, Lref, A) -> float:
    scale = np.sqrt(np.diag(A))[:, None]
    return float(np.max(np.abs(np.tril(L) - np.tril(Lref)) / scale))


@functools.lru_cache(maxsize=32)
def matrix(gen: str, n: int, seed: int, param: float = 0.0):
    if gen == "gram":
        return si.gram_plus_identity(n, seed)
    if gen == "se":
        return si.se_covariance(n, seed, nugget=param or 1e-2)
    if gen == "pascal":
        return si.pascal(n)
    if gen == "int":
        return si.exact_integer_factor(n, seed)[0]
    raise ValueError(gen)


@functools.lru_cache(maxsize=32)
def oracle_factor(gen: str, n: int, seed: int, param: float = 0.0):
    A = matrix(gen, n, seed, param)
    L, info = oracle.potrf_unblocked(A)
    return np.tril(L), info


def gpu_factor(A, **kw):
    """Factor a host matrix on the GPU; return (L lower as numpy, info, stats, status)."""
    import torch

    import paper_2606_11937_gb300 as chol

    dA = chol.colmajor(A)
    rc, info, st = chol.chol_factor_ex(dA, chol.opts(**kw), raise_on_error=False)
    torch.cuda.synchronize()
    return np.tril(dA.cpu().numpy()), info, st, rc


def probe_residual(A, L, k: int = 4, seed: int = 99) -> float:
    X = si.rhs(A.shape[0], k, seed=seed)
    return oracle.residual_probe(A, L, X)


def resid_bound(n: int) -> float:
    return TOL_RESID * math.sqrt(n)
