"""Mixed-precision factorization (tcgen05 SYRK/GEMM, FP64 POTRF, FP32 TRSM)
and FP64 iterative refinement, against the FP64 oracle.

* exact pin: A = L0 L0^T with small-integer L0 is reproduced bit for bit by
  every precision (all operands, products and partial sums are exact);
* the factor's error against the FP64 oracle is reported and held under a
  loose per-precision bound (a gross indexing or scaling error fails it);
* refinement reaches the FP64 backward error 1e-14 on well-conditioned
  inputs, checked with the oracle's backward error;
* the two schedules produce identical bits.
"""
import numpy as np
import pytest

import oracle
import seeded_inputs as si
from gpu_common import matrix, oracle_factor, scaled_error
from paper_facts import task_counts

pytestmark = pytest.mark.gpu

PRECS = ["fp32", "tf32", "bf16", "fp16"]
# bound on the scaled entrywise error of the low-precision factor (reported
# quantity; about 50x the unit roundoff of the operand format at n = 2048)
FACTOR_BOUND = {"fp32": 1e-4, "tf32": 5e-2, "fp16": 5e-2, "bf16": 2e-1}


def mixed(A, prec, sched="dataflow", nb=128, **kw):
    import torch

    import paper_2606_11937_gb300 as chol
    dA = chol.colmajor(A)
    kw.setdefault("timeout_s", 20.0)
    rc, h = chol.chol_mixed_factor(dA, chol.opts(precision=prec, schedule=sched, nb=nb, **kw), raise_on_error=False)
    torch.cuda.synchronize()
    return rc, h, dA


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("n,nb", [(1024, 128), (1500, 256), (1000, 384), (700, 512)])
def test_mixed_exact_integer_factor(prec, n, nb):
    A, L0 = si.exact_integer_factor(n, seed=n + 1)
    for sched in ("dataflow", "fork_join"):
        rc, h, dA = mixed(A, prec, sched, nb)
        assert rc == 0 and h.info == 0
        L = np.tril(h.factor().cpu().numpy())
        assert np.array_equal(L, L0), (prec, sched, float(np.max(np.abs(L - L0))))
        h.close()


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("nb", [128, 256, 384, 512])
def test_mixed_factor_error_and_schedules(prec, nb):
    """Tile orders above 128 factor each diagonal tile by 128 x 128 blocks
    (binary64 POTRF of each, binary32 TRSM and update between them) and solve
    each panel tile by column blocks of 128: same error bound, and the same
    bits under every schedule."""
    import paper_2606_11937_gb300 as chol
    n = 2048
    A = matrix("gram", n, 0)
    Lref, _ = oracle_factor("gram", n, 0)
    outs = []
    for sched in ("dataflow", "fork_join", "fork_join_naive", "left_looking", "top_looking"):
        rc, h, dA = mixed(A, prec, sched, nb)
        assert rc == 0 and h.info == 0
        st = chol.chol_mixed_last_stats()
        assert tuple(st.tasks) == task_counts(-(-n // nb))
        L = np.tril(h.factor().cpu().numpy())
        err = scaled_error(L, Lref, A)
        print(f"{prec} {sched}: scaled error vs FP64 oracle {err:.3e}")
        assert err <= FACTOR_BOUND[prec]
        outs.append(L)
        h.close()
    for L in outs[1:]:
        assert np.array_equal(outs[0], L)


@pytest.mark.parametrize("nb,col", [(128, 300), (256, 400), (256, 100), (512, 1100)])
def test_mixed_info_inside_blocked_potrf(nb, col):
    """A non-positive pivot anywhere inside a diagonal tile (first or later
    128-block) reports the oracle's info."""
    A = matrix("gram", 1500, 7).copy()
    A[col, col] = -1e6
    _, want = oracle.potrf_unblocked(A)
    assert want == col + 1
    for prec in ("fp32", "bf16"):
        rc, h, dA = mixed(A, prec, "dataflow", nb)
        assert rc == 0 and h.info == want, (prec, nb, h.info, want)
        h.close()


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("n,nrhs", [(2048, 4), (1000, 17)])
def test_refinement_reaches_fp64_backward_error(prec, n, nrhs):
    import torch

    import paper_2606_11937_gb300 as chol
    A = matrix("gram", n, 3)
    B = si.rhs(n, nrhs, seed=4)
    rc, h, dA = mixed(A, prec, "dataflow", 128)
    assert rc == 0
    dB = chol.colmajor(B)
    rc, dX, iters, berr = h.solve(dB)
    torch.cuda.synchronize()
    X = dX.cpu().numpy()
    be = oracle.backward_error(A, X, B)
    print(f"{prec}: iterations {iters}, reported berr {berr:.2e}, oracle berr {be:.2e}")
    assert rc == 0 and berr <= 1e-14
    assert be <= 1e-14
    Lref, _ = oracle_factor("gram", n, 3)
    Xref = oracle.potrs(Lref, B)
    assert np.max(np.abs(X - Xref)) <= 1e-12 * np.max(np.abs(Xref))
    h.close()


def test_refinement_status_on_harder_input():
    """SE covariance (nugget 1e-1): each precision either converges to 1e-14
    (checked by the oracle) or says it did not."""
    import torch

    import paper_2606_11937_gb300 as chol
    n = 1536
    A = matrix("se", n, 1, 1e-1)
    B = si.rhs(n, 2, seed=5)
    for prec in PRECS:
        rc, h, dA = mixed(A, prec, "dataflow", 128, max_iter=40)
        if rc != 0 or h.info != 0:
            continue  # a low-precision factor may legitimately break down
        rc, dX, iters, berr = h.solve(chol.colmajor(B), raise_on_error=False)
        torch.cuda.synchronize()
        be = oracle.backward_error(A, dX.cpu().numpy(), B)
        print(f"{prec}: rc {rc} iterations {iters} berr {berr:.2e} oracle {be:.2e}")
        if rc == 0:
            assert be <= 1e-14
        else:
            assert rc == chol.CHOL_ERR_NOT_CONVERGED
        h.close()


@pytest.mark.parametrize("prec", ["tf32", "fp16"])
@pytest.mark.parametrize("nugget", [1e-1, 1e-2])
def test_gmres_refinement(prec, nugget):
    """CHOL_FLAG_GMRES_IR: each correction by GMRES preconditioned with the
    low-precision factor.  Where the factor exists, the solve reaches the
    FP64 backward error 1e-14 (checked by the oracle) and matches the oracle's
    solution, also where classic refinement stalls."""
    import torch

    import paper_2606_11937_gb300 as chol
    n = 1536
    A = matrix("se", n, 1, nugget)
    B = si.rhs(n, 3, seed=6)
    rc, h, dA = mixed(A, prec, "dataflow", 128, max_iter=40, flags=chol.CHOL_FLAG_GMRES_IR)
    if rc != 0 or h.info != 0:
        pytest.skip(f"{prec} factor breaks down at nugget {nugget} (info {h.info})")
    rc, dX, napply, berr = h.solve(chol.colmajor(B), raise_on_error=False)
    torch.cuda.synchronize()
    X = dX.cpu().numpy()
    be = oracle.backward_error(A, X, B)
    h.close()
    rc2, h2, _ = mixed(A, prec, "dataflow", 128, max_iter=40)
    rc2, _, iters, berr2 = h2.solve(chol.colmajor(B), raise_on_error=False)
    h2.close()
    print(f"{prec} nugget {nugget}: GMRES rc {rc} applications {napply} berr {berr:.2e} oracle {be:.2e}; "
          f"classic rc {rc2} iterations {iters} berr {berr2:.2e}")
    assert rc == 0 and berr <= 1e-14 and be <= 1e-14
    Lref, _ = oracle_factor("se", n, 1, nugget)
    Xref = oracle.potrs(Lref, B)
    kappa_u = 1e-16 * np.linalg.cond(A, 1)
    assert np.max(np.abs(X - Xref)) <= max(1e-12, 10 * kappa_u) * np.max(np.abs(Xref))


@pytest.mark.parametrize("flags", [0, 32])
def test_refinement_many_columns_and_a_zero_column(flags):
    """20 right-hand sides (two 16-column chunks of the tensor-core residual),
    one of them zero: classic and GMRES-based refinement reach 1e-14 on every
    column (oracle), and the zero column's solution is exactly zero."""
    import torch

    import paper_2606_11937_gb300 as chol
    n = 1300
    A = matrix("se", n, 2, 1e-2)
    B = si.rhs(n, 20, seed=9)
    B[:, 7] = 0.0
    rc, h, dA = mixed(A, "tf32", "dataflow", 128, max_iter=40, flags=flags)
    assert rc == 0 and h.info == 0
    rc, dX, iters, berr = h.solve(chol.colmajor(B), raise_on_error=False)
    torch.cuda.synchronize()
    X = dX.cpu().numpy()
    h.close()
    print(f"flags {flags}: rc {rc} iterations {iters} berr {berr:.2e}")
    assert rc == 0 and berr <= 1e-14
    assert oracle.backward_error(A, X, B) <= 1e-14
    assert np.all(X[:, 7] == 0.0)


def test_mixed_non_spd_info():
    n = 1024
    A = matrix("gram", n, 4).copy()
    A[300, 300] -= 1e4
    _, want = oracle.potrf_unblocked(A)
    for prec in PRECS:
        for sched in ("dataflow", "fork_join"):
            rc, h, dA = mixed(A, prec, sched, 128)
            assert rc == 0 and h.info == want
            h.close()


def test_breakdown_is_reported_not_solved():
    """A factor that broke down (info > 0) refuses to solve; NaN never
    passes as converged."""
    import paper_2606_11937_gb300 as chol
    n = 1024
    A = matrix("gram", n, 4).copy()
    A[500, 500] = -1.0
    rc, h, dA = mixed(A, "bf16", "dataflow", 128)
    assert rc == 0 and h.info > 0
    rc, X, iters, berr = h.solve(chol.colmajor(si.rhs(n, 2, seed=1)), raise_on_error=False)
    assert rc == chol.CHOL_ERR_NOT_SPD
    h.close()
