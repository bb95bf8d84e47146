"""The oracle's pins must catch plausible mistakes.

Each case plants one mistake in a temporary copy of oracle.c (a flipped sign,
a wrong index, a transposed operand, a dropped term or loop iteration),
compiles it on the CPU, and runs the pin battery below against it: at least
one pin must fail.  The unmodified oracle must pass the same battery.
"""
import os
import shutil
import tempfile

import numpy as np
import pytest

import oracle
import seeded_inputs as si
from paper_facts import task_counts

SRC = os.path.join(os.path.dirname(oracle.__file__), "oracle.c")

# (name, text to find, replacement).  Each text must occur in oracle.c.
MUTANTS = [
    ("crout_diag_sign", "d -= Lj[k] * Lj[k];", "d += Lj[k] * Lj[k];"),
    ("crout_wrong_index", "s -= Li[k] * Lj[k];", "s -= Li[k] * Li[k];"),
    ("crout_no_sqrt", "const double ljj = sqrt(d);\n        W[j * n + j] = ljj;",
     "const double ljj = d;\n        W[j * n + j] = ljj;"),
    ("potrf_tile_sum_bound", "for (int64_t k = 0; k < j; ++k) s -= RM(T, nb, i, k) * RM(T, nb, j, k);",
     "for (int64_t k = 0; k + 1 < j; ++k) s -= RM(T, nb, i, k) * RM(T, nb, j, k);"),
    ("trsm_no_divide", "RM(B, nb, r, j) = x / RM(L, nb, j, j);", "RM(B, nb, r, j) = x;"),
    ("trsm_transposed_L", "x -= RM(B, nb, r, k) * RM(L, nb, j, k);", "x -= RM(B, nb, r, k) * RM(L, nb, k, j);"),
    ("syrk_skips_diagonal", "for (int64_t j = 0; j <= i; ++j) {\n            double s = RM(C, nb, i, j);",
     "for (int64_t j = 0; j < i; ++j) {\n            double s = RM(C, nb, i, j);"),
    ("gemm_transposed_B", "s -= RM(A, nb, i, k) * RM(B, nb, j, k);", "s -= RM(A, nb, i, k) * RM(B, nb, k, j);"),
    ("gemm_sign", "s -= RM(A, nb, i, k) * RM(B, nb, j, k);", "s += RM(A, nb, i, k) * RM(B, nb, j, k);"),
    ("fig1_drops_last_gemm", "for (int64_t K = J + 1; K < I; ++K) {\n                LOG(3",
     "for (int64_t K = J + 1; K + 1 < I; ++K) {\n                LOG(3"),
    ("fig1_trsm_skips_first", "for (int64_t I = J + 1; I < M; ++I) {\n            LOG(1",
     "for (int64_t I = J + 2; I < M; ++I) {\n            LOG(1"),
    ("pad_with_zero", "} else if (i == j) {\n                        v = 1.0;",
     "} else if (i == j) {\n                        v = 0.0;"),
    ("potrs_backward_transposed", "s -= CM(L, ldl, k, i) * b[k];", "s -= CM(L, ldl, i, k) * b[k];"),
    ("potrs_forward_bound", "for (int64_t k = 0; k < i; ++k) s -= CM(L, ldl, i, k) * b[k];",
     "for (int64_t k = 1; k < i; ++k) s -= CM(L, ldl, i, k) * b[k];"),
    ("info_off_by_one", "info = J * nb + ti;", "info = J * nb + ti - 1;"),
    ("residual_drops_diag_term", "for (int64_t k = 0; k <= m; ++k) s += CM(L, ldl, i, k) * CM(L, ldl, j, k);",
     "for (int64_t k = 0; k < m; ++k) s += CM(L, ldl, i, k) * CM(L, ldl, j, k);"),
]


def battery(lib) -> list[str]:
    """Run the pins against `lib`; return the names of the pins that fail."""
    failed = []

    def check(name, cond):
        if not cond:
            failed.append(name)

    def guard(name, fn):
        try:
            check(name, bool(fn()))
        except Exception:  # a crash or a bad value is a failed pin too
            failed.append(name)

    def fac(A, nb):
        Lu, iu = oracle.potrf_unblocked(A, lib=lib)
        Lt, it, cnt = oracle.potrf_tiled(A, nb, lib=lib)
        return Lu, iu, Lt, it, cnt

    A3 = np.array([[4.0, 12.0, -16.0], [12.0, 37.0, -43.0], [-16.0, -43.0, 98.0]])
    W3 = np.array([[2.0, 0, 0], [6.0, 1.0, 0], [-8.0, 5.0, 3.0]])

    def p3():
        ok = True
        for nb in (1, 2, 3):
            Lu, iu, Lt, it, _ = fac(A3, nb)
            ok &= iu == 0 and it == 0 and np.array_equal(np.tril(Lu), W3) and np.array_equal(np.tril(Lt), W3)
        return ok
    guard("3x3", p3)

    def ppascal():
        ok = True
        for nb in (3, 7, 29):
            Lu, iu, Lt, it, _ = fac(si.pascal(29), nb)
            want = si.pascal_lower(29)
            ok &= iu == 0 and it == 0 and np.array_equal(np.tril(Lu), want) and np.array_equal(np.tril(Lt), want)
        return ok
    guard("pascal", ppascal)

    def pint():
        A, L0 = si.exact_integer_factor(45, seed=3)
        ok = True
        for nb in (8, 16, 45, 64):
            Lu, iu, Lt, it, _ = fac(A, nb)
            ok &= iu == 0 and it == 0 and np.array_equal(np.tril(Lu), L0) and np.array_equal(np.tril(Lt), L0)
        return ok
    guard("integer", pint)

    def pcounts():
        ok = True
        for m in (1, 2, 4, 6):
            _, info, cnt = oracle.potrf_tiled(si.gram_plus_identity(3 * m, 2), 3, lib=lib)
            ok &= info == 0 and tuple(int(c) for c in cnt) == task_counts(m)
        return ok
    guard("counts", pcounts)

    def ptiles():
        nb = 9
        r = si.rng(1)
        A, B, C = (r.integers(-3, 4, size=(nb, nb)).astype(float) for _ in range(3))
        ok = np.array_equal(oracle.tile_op("gemm", A, B, C, lib=lib), C - A @ B.T)
        want = C.copy()
        want[np.tril_indices(nb)] = (C - A @ A.T)[np.tril_indices(nb)]
        ok &= np.array_equal(oracle.tile_op("syrk", A, C, lib=lib), want)
        L0 = si.exact_integer_L0(nb, seed=4)
        ok &= np.array_equal(oracle.tile_op("trsm", L0, A @ L0.T, lib=lib), A)
        return ok
    guard("tiles", ptiles)

    def psolve():
        A, L0 = si.exact_integer_factor(40, seed=5)
        X0 = si.rng(6).integers(-5, 6, size=(40, 2)).astype(float)
        return np.array_equal(oracle.potrs(L0, A @ X0, lib=lib), X0)
    guard("solve", psolve)

    def pinfo():
        B = si.gram_plus_identity(20, 4)
        B[13, 13] -= 50.0
        _, iu, _, it, _ = fac(B, 8)
        return iu == 14 and it == 14
    guard("info", pinfo)

    def presid():
        L = np.eye(6)
        L[3, 1] = 0.25
        want = np.sqrt(2 * 0.25 ** 2 + 0.25 ** 4) / np.sqrt(6)
        return abs(oracle.residual_fro(np.eye(6), L, lib=lib) - want) < 1e-15
    guard("residual", presid)
    return failed


def test_unmodified_oracle_passes_battery():
    assert battery(oracle.load()) == []


@pytest.mark.parametrize("name,find,repl", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_mutant_is_caught(name, find, repl, tmp_path):
    src = open(SRC).read()
    assert src.count(find) >= 1, f"mutation site for {name} not found"
    mutated = src.replace(find, repl, 1)
    d = tempfile.mkdtemp(dir=tmp_path)
    path = os.path.join(d, "oracle_mut.c")
    with open(path, "w") as f:
        f.write(mutated)
    shutil.copy(os.path.join(os.path.dirname(SRC), "oracle.h"), d)
    so = oracle.build(src=path, out=os.path.join(d, f"lib_{name}.so"))
    lib = oracle.load(so)
    assert battery(lib), f"mutant {name} passed every pin"
