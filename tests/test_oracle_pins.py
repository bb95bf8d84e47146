"""Pins for the CPU oracle, checked against values fixed by the paper and by
the mathematics -- never against the oracle itself or the CUDA library.

Each pin targets a plausible mistake: closed forms and the Pascal/integer
factors catch dropped terms, wrong signs and transposed operands exactly;
the task-count formula (Section 4.2) and Fig. 2 pin the loop structure of
Fig. 1; numpy's LAPACK Cholesky is an independent library routine.
"""
import math

import numpy as np
import pytest

import oracle
import seeded_inputs as si
from paper_facts import GEMM, POTRF, SYRK, TRSM, load_op_map, task_counts

pytestmark = pytest.mark.filterwarnings("ignore")


def both(A, nb):
    """Factor with the unblocked and the Fig. 1 tiled oracle."""
    Lu, iu = oracle.potrf_unblocked(A)
    Lt, it, _ = oracle.potrf_tiled(A, nb)
    return (Lu, iu), (Lt, it)


# --------------------------------------------------------------- closed forms

def test_2x2_closed_form():
    A = np.array([[4.0, 2.0], [2.0, 3.0]])
    for nb in (1, 2, 3):
        for L, info in both(A, nb):
            assert info == 0
            assert L[0, 0] == 2.0 and L[1, 0] == 1.0
            assert L[1, 1] == math.sqrt(2.0)  # correctly rounded sqrt(3 - 1)


def test_3x3_textbook():
    A = np.array([[4.0, 12.0, -16.0], [12.0, 37.0, -43.0], [-16.0, -43.0, 98.0]])
    want = np.array([[2.0, 0, 0], [6.0, 1.0, 0], [-8.0, 5.0, 3.0]])
    for nb in (1, 2, 3, 4):
        for L, info in both(A, nb):
            assert info == 0
            assert np.array_equal(np.tril(L), want)


def test_identity_and_diagonal():
    d = np.array([1.0, 4.0, 9.0, 2.0, 0.25, 1e-6, 1e6])
    for nb in (1, 3, 7, 8):
        for L, info in both(np.eye(7), nb):
            assert info == 0 and np.array_equal(np.tril(L), np.eye(7))
        for L, info in both(np.diag(d), nb):
            assert info == 0 and np.array_equal(np.tril(L), np.diag(np.sqrt(d)))


@pytest.mark.parametrize("n", [1, 2, 5, 12, 17, 29])
def test_pascal_exact(n):
    """Symmetric Pascal C(i+j, i) factors into lower Pascal C(i, j) exactly:
    every partial sum is an integer below 2^53 for n <= 29."""
    P, want = si.pascal(n), si.pascal_lower(n)
    for nb in (1, 3, 4, 7, 8, 29, 32):
        for L, info in both(P, nb):
            assert info == 0
            assert np.array_equal(np.tril(L), want)


@pytest.mark.parametrize("n,nb,band", [(37, 8, None), (64, 16, None), (100, 32, None),
                                       (200, 64, None), (150, 50, 7), (129, 128, None)])
def test_exact_integer_factor(n, nb, band):
    """A = L0 L0^T with small-integer L0 (diagonal 1, 2 or 4): every
    intermediate is an integer and every division is by a power of two, so the
    factor is L0 exactly in any order of operations."""
    A, L0 = si.exact_integer_factor(n, seed=11 + n, band=band)
    for L, info in both(A, nb):
        assert info == 0
        assert np.array_equal(np.tril(L), L0)


def test_tridiagonal_closed_form():
    """[-1, 2, -1]: L_ii = sqrt((i+1)/i), L_{i+1,i} = -sqrt(i/(i+1)) (1-based)."""
    n = 500
    A = si.tridiag(n)
    i = np.arange(1, n + 1, dtype=np.float64)
    diag = np.sqrt((i + 1) / i)
    sub = -np.sqrt(i[:-1] / (i[:-1] + 1))
    for L, info in both(A, 64):
        assert info == 0
        assert np.allclose(np.diag(L), diag, rtol=8e-16 * 8, atol=0)
        assert np.allclose(np.diag(L, -1), sub, rtol=8e-16 * 8, atol=0)
        assert np.count_nonzero(np.tril(L, -2)) == 0


def test_against_numpy_lapack():
    """Special case that reduces to a library routine: LAPACK dpotrf via numpy."""
    A = si.gram_plus_identity(150, seed=7)
    want = np.linalg.cholesky(A)
    scale = np.sqrt(np.diag(A))[:, None]
    for L, info in both(A, 32):
        assert info == 0
        assert np.max(np.abs(np.tril(L) - want) / scale) < 1e-14


# --------------------------------------------------------------- invariants

@pytest.mark.parametrize("n,nb", [(300, 16), (300, 37), (300, 64), (300, 300), (300, 512), (257, 128)])
def test_unblocked_vs_tiled(n, nb):
    A = si.se_covariance(n, seed=3, nugget=1e-1)
    (Lu, iu), (Lt, it) = both(A, nb)
    assert iu == 0 and it == 0
    scale = np.sqrt(np.diag(A))[:, None]
    assert np.max(np.abs(np.tril(Lu) - np.tril(Lt)) / scale) <= 1e-13


@pytest.mark.parametrize("gen", ["gram", "se"])
def test_factor_invariants(gen):
    n = 240
    A = si.gram_plus_identity(n, 1) if gen == "gram" else si.se_covariance(n, 1, nugget=1e-2)
    marker = np.triu(np.full((n, n), 123.5), 1)
    Aup = np.tril(A) + marker            # strict upper holds junk the oracle must not touch
    for L, info in both(Aup, 48):
        assert info == 0
        assert np.array_equal(np.triu(L, 1), marker)      # upper triangle untouched
        Lo = np.tril(L)
        assert np.all(np.diag(Lo) > 0)
        assert oracle.residual_fro(A, Lo) <= 1e-14 * math.sqrt(n)


def test_non_spd_info():
    """info = 1-based index of the first leading minor that is not positive
    definite; checked against numpy eigenvalues of the leading minors."""
    n = 60
    A = si.gram_plus_identity(n, 4)
    for k in (0, 1, 17, 31, 32, 59):
        B = A.copy()
        B[k, k] -= 50.0                   # makes the leading (k+1) minor indefinite
        want = next(m for m in range(1, n + 1) if np.linalg.eigvalsh(B[:m, :m])[0] <= 0)
        assert want == k + 1
        for nb in (1, 8, 16, 32, 64):
            for _, info in both(B, nb):
                assert info == want
    C = np.diag([1.0, 1.0, -1.0, 1.0])
    for _, info in both(C, 2):
        assert info == 3
    D = np.eye(9)
    D[4, 4] = np.nan
    for _, info in both(D, 4):
        assert info == 5
    Z = np.eye(5)
    Z[2, 2] = 0.0
    for _, info in both(Z, 2):
        assert info == 3


# --------------------------------------------------------------- Fig. 1 structure

@pytest.mark.parametrize("m", list(range(1, 13)))
def test_task_counts_formula(m):
    """Section 4.2 task counts, for the oracle's execution of Fig. 1."""
    nb = 3
    A = si.gram_plus_identity(m * nb, 2)
    _, info, counts = oracle.potrf_tiled(A, nb)
    assert info == 0
    assert tuple(int(c) for c in counts) == task_counts(m)


def test_fig2_first_iteration():
    """Fig. 2: the operation each tile of a 4 x 4 tiling receives when J = 0."""
    want = load_op_map("fig2_first_iteration.txt")
    A = si.gram_plus_identity(16, 3)
    _, info, counts, log = oracle.potrf_tiled(A, 4, with_log=True)
    got = {}
    for ty, I, K, J in log:
        if J == 0:
            assert (I, K) not in got
            got[(int(I), int(K))] = int(ty)
    assert got == want


def test_task_log_respects_dependencies():
    """Every task runs after the tasks whose output it reads, and every tile
    receives its updates in ascending J (Section 3.2, task dependencies)."""
    m, nb = 7, 2
    A = si.gram_plus_identity(m * nb, 5)
    _, _, _, log = oracle.potrf_tiled(A, nb, with_log=True)
    done = {}
    for pos, (ty, I, K, J) in enumerate(log):
        ty, I, K, J = int(ty), int(I), int(K), int(J)
        if ty == POTRF:
            needs = [(SYRK, I, I, J - 1)] if J > 0 else []
        elif ty == TRSM:
            needs = [(POTRF, J, J, J)] + ([(GEMM, I, J, J - 1)] if J > 0 else [])
        elif ty == SYRK:
            needs = [(TRSM, I, J, J)] + ([(SYRK, I, I, J - 1)] if J > 0 else [])
        else:
            needs = [(TRSM, I, J, J), (TRSM, K, J, J)] + ([(GEMM, I, K, J - 1)] if J > 0 else [])
        for nd in needs:
            assert nd in done and done[nd] < pos
        done[(ty, I, K, J)] = pos


def test_tiled_tasks_bitwise_equals_tiled():
    """The OpenMP-dependency version applies each tile's updates in the same
    order, so it must agree bit for bit with the sequential Fig. 1 version."""
    A = si.se_covariance(333, seed=9, nugget=1e-2)
    Lt, it, _ = oracle.potrf_tiled(A, 32)
    for th in (1, 3, 8):
        Lp, ip = oracle.potrf_tiled_tasks(A, 32, nthreads=th)
        assert ip == it == 0
        assert np.array_equal(np.tril(Lp), np.tril(Lt))
    B = A.copy()
    B[100, 100] = -1.0
    _, ib, _ = oracle.potrf_tiled(B, 32)
    _, ipb = oracle.potrf_tiled_tasks(B, 32, nthreads=4)
    assert ib == ipb == 101


# --------------------------------------------------------------- tile operations

def _int_tile(nb, seed, lo=-3, hi=4):
    return si.rng(seed).integers(lo, hi, size=(nb, nb)).astype(np.float64)


@pytest.mark.parametrize("nb", [1, 5, 16, 33])
def test_tile_ops_exact_integers(nb):
    """Tile formulas on integer tiles, where every result is exact: GEMM is
    C - A B^T (not A B, not A^T B), SYRK touches only the lower triangle, TRSM
    inverts X -> X L^T, POTRF returns L0."""
    A, B, C = _int_tile(nb, 1), _int_tile(nb, 2), _int_tile(nb, 3)
    got = oracle.tile_op("gemm", A, B, C)
    assert np.array_equal(got, C - A @ B.T)
    got = oracle.tile_op("syrk", A, C)
    want = C.copy()
    want[np.tril_indices(nb)] = (C - A @ A.T)[np.tril_indices(nb)]
    assert np.array_equal(got, want)
    L0 = si.exact_integer_L0(nb, seed=nb)
    X0 = _int_tile(nb, 4)
    got = oracle.tile_op("trsm", L0, X0 @ L0.T)
    assert np.array_equal(got, X0)
    got, info = oracle.tile_op("potrf", L0 @ L0.T)
    assert info == 0 and np.array_equal(np.tril(got), L0)


# --------------------------------------------------------------- solve and error measures

def test_potrs_exact_integer():
    """With an integer factor and an integer solution, forward and backward
    substitution are exact: y = L0^T x is integer, divisions by 1, 2, 4."""
    n = 90
    A, L0 = si.exact_integer_factor(n, seed=21)
    X0 = si.rng(22).integers(-5, 6, size=(n, 3)).astype(np.float64)
    B = A @ X0
    X = oracle.potrs(L0, B)
    assert np.array_equal(X, X0)


def test_potrs_against_numpy():
    n = 120
    A = si.gram_plus_identity(n, 8)
    B = si.rhs(n, 4, seed=9)
    L, info = oracle.potrf_unblocked(A)
    X = oracle.potrs(np.tril(L), B)
    want = np.linalg.solve(A, B)
    assert np.max(np.abs(X - want)) < 1e-12
    assert oracle.backward_error(A, X, B) < 1e-15


def test_backward_error_closed_form():
    """A = I, x = b + delta e_3: ||b - x||_inf / (||x||_inf + ||b||_inf)."""
    n = 8
    b = np.arange(1.0, n + 1.0).reshape(-1, 1)
    x = b.copy()
    x[3, 0] += 0.5
    got = oracle.backward_error(np.eye(n), x, b)
    assert got == 0.5 / (8.0 + 8.0)
    A2 = 2.0 * np.eye(n)
    got = oracle.backward_error(A2, b / 2.0, b)      # exact solution
    assert got == 0.0


def test_residual_closed_form():
    """A = I, L = I + d e_3 e_1^T: A - L L^T has entries -d (twice) and -d^2."""
    n, d = 10, 0.25
    L = np.eye(n)
    L[3, 1] = d
    want = math.sqrt(2 * d * d + d ** 4) / math.sqrt(n)
    assert abs(oracle.residual_fro(np.eye(n), L) - want) < 1e-15
    assert abs(oracle.residual_probe(np.eye(n), L, np.eye(n)) - want) < 1e-15


@pytest.mark.parametrize("n,band", [(300, 5), (257, 64)])
def test_banded_integer_generator_and_oracle(n, band):
    """The device builder of the full-size exact-integer input (run here on
    the CPU device) gives A = L0 L0^T exactly (integer arithmetic), L0 banded
    with diagonal in {1, 2, 4}; the oracle factors A back to L0 exactly."""
    torch = pytest.importorskip("torch")
    A, L = si.exact_integer_band_torch(n, band, seed=7, device="cpu")
    A = A.T.numpy()  # column-major convention: element (i, j) of A
    L0 = L.T.numpy()  # element (i, j) of L0
    assert np.array_equal(L0, np.tril(L0))
    assert np.all(np.isin(np.diag(L0), [1.0, 2.0, 4.0]))
    assert np.all(np.tril(L0, -band - 1) == 0)
    Li = L0.astype(np.int64)
    assert np.array_equal(A.astype(np.int64), Li @ Li.T)
    Lo, info = oracle.potrf_unblocked(A)
    assert info == 0 and np.array_equal(np.tril(Lo), L0)
