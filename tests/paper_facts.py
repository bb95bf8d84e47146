"""Facts the paper states, restated for the tests.

Each function cites the passage it restates.  Nothing here computes a
factorization; these are the independent values the oracle and the CUDA
library are checked against.
"""
import os

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")

POTRF, TRSM, SYRK, GEMM = 0, 1, 2, 3
OP_NAMES = {"P": POTRF, "T": TRSM, "S": SYRK, "G": GEMM}


def task_counts(m: int):
    """Section 4.2: with m tiles per dimension the right-looking factorization
    issues m POTRF, m(m-1)/2 TRSM and SYRK tasks each, and m(m-1)(m-2)/6 GEMM
    tasks."""
    return (m, m * (m - 1) // 2, m * (m - 1) // 2, m * (m - 1) * (m - 2) // 6)


def total_tasks(m: int) -> int:
    return sum(task_counts(m))


def load_op_map(name: str):
    """Read a golden tile -> operation map: lines 'I K OP' (OP in P/T/S/G)."""
    out = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            i, k, op = line.split()
            out[(int(i), int(k))] = OP_NAMES[op]
    return out
