"""FP64 factorization with SYRK/GEMM on the tensor cores (CHOL_FLAG_FP64_TC):
binary64 accuracy from exact bf16 slicing.

* the tile update alone: on integer data every slice product is exact, so
  the update must be exact; on random binary64 data the error must stay at
  binary64 level.  The reference is the oracle's sequential C - sum_k a_k b_k,
  whose own error is at most gamma_(k+1) (|C| + sum_k |a_k||b_k|); the
  device's error is below 2^-40 * 2^(e_r + e_c) (2^e_r, 2^e_c bound the row
  and column magnitudes; 56 retained bits, 28 omitted low-order products, 8
  rounded binary64 additions) plus one rounding of the result;
* the factorization meets the same FP64 parity bar as the DFMA path
  (scaled error <= 1e-11 vs the oracle, residual <= 1e-14 sqrt(n)), is exact
  on Pascal and integer inputs, and the schedules agree bit for bit;
* TRSMs multiply by the inverted diagonal tile on the tensor cores when it is
  well conditioned (the SE and Gram inputs: kappa_inf of every diagonal tile
  below 500), and keep the substitution kernel otherwise (the integer factors,
  kappa_inf ~ 1e12, which therefore stay exact).
"""
import math

import numpy as np
import pytest

import oracle
import seeded_inputs as si
from gpu_common import TOL_SCALED, gpu_factor, matrix, oracle_factor, probe_residual, resid_bound, scaled_error
from paper_facts import task_counts

pytestmark = pytest.mark.gpu


def _update(A, B, C):
    import torch

    import paper_2606_11937_gb300 as chol
    dA = torch.from_numpy(np.ascontiguousarray(A)).cuda()
    dB = torch.from_numpy(np.ascontiguousarray(B)).cuda()
    dC = torch.from_numpy(np.ascontiguousarray(C)).cuda()
    rc = chol.lib().chol_test_ozaki_update(dA.data_ptr(), dB.data_ptr(), dC.data_ptr())
    assert rc == 0, chol.chol_last_error()
    return dC.cpu().numpy()


def test_ozaki_update_exact_on_integers():
    r = si.rng(3)
    A = r.integers(-1000, 1001, size=(128, 128)).astype(np.float64)
    B = r.integers(-1000, 1001, size=(128, 128)).astype(np.float64)
    C = r.integers(-10 ** 6, 10 ** 6, size=(2, 128, 128)).astype(np.float64)
    got = _update(A, B, C)
    for k in range(2):
        assert np.array_equal(got[k], oracle.tile_op("gemm", A, B, C[k]))


@pytest.mark.parametrize("scale", ["uniform", "graded"])
@pytest.mark.parametrize("cmag", [0.0, 10.0])
def test_ozaki_update_binary64_accuracy(scale, cmag):
    r = si.rng(4)
    A = r.standard_normal((128, 128))
    B = r.standard_normal((128, 128))
    if scale == "graded":  # rows / columns spanning many binades
        A *= np.exp2(r.integers(-30, 30, size=(128, 1)))
        B *= np.exp2(r.integers(-30, 30, size=(128, 1)))
    C = r.standard_normal((2, 128, 128)) * cmag
    got = _update(A, B, C)
    ea = np.frexp(np.max(np.abs(A), axis=1))[1].astype(np.float64)
    eb = np.frexp(np.max(np.abs(B), axis=1))[1].astype(np.float64)
    bound = 2.0 ** -40 * np.exp2(ea[:, None] + eb[None, :])
    u = 2.0 ** -53
    absprod = np.abs(A) @ np.abs(B).T
    for k in range(2):
        want = oracle.tile_op("gemm", A, B, C[k])
        err = np.abs(got[k] - want)
        ref_err = (128 + 1) * u / (1 - (128 + 1) * u) * (np.abs(C[k]) + absprod)
        tol = bound + 2 * u * np.abs(want) + ref_err
        assert np.all(err <= tol), float(np.max(err / tol))


@pytest.mark.parametrize("sched", ["dataflow", "fork_join"])
def test_fp64tc_config1_parity(sched):
    import paper_2606_11937_gb300 as chol
    A = matrix("gram", 2048, 0)
    Lref, _ = oracle_factor("gram", 2048, 0)
    L, info, st, rc = gpu_factor(A, schedule=sched, flags=chol.CHOL_FLAG_FP64_TC)
    assert rc == 0 and info == 0 and st.nb == 128
    assert scaled_error(L, Lref, A) <= TOL_SCALED
    assert probe_residual(A, L) <= resid_bound(2048)
    assert tuple(st.tasks) == task_counts(16)


def test_fp64tc_ragged_exact_and_schedules():
    import paper_2606_11937_gb300 as chol
    f = chol.CHOL_FLAG_FP64_TC
    P = si.pascal(29)
    L, info, _, rc = gpu_factor(P, schedule="dataflow", flags=f)
    assert rc == 0 and np.array_equal(L, si.pascal_lower(29))
    A, L0 = si.exact_integer_factor(1000, seed=77)
    outs = []
    for sched in ("dataflow", "fork_join", "fork_join_naive", "left_looking", "top_looking"):
        L, info, _, rc = gpu_factor(A, schedule=sched, flags=f)
        assert rc == 0 and info == 0 and np.array_equal(L, L0)
    S = matrix("se", 1111, 3, 1e-2)
    Lref, _ = oracle_factor("se", 1111, 3, 1e-2)
    for sched in ("dataflow", "fork_join", "left_looking", "top_looking"):
        L, info, _, rc = gpu_factor(S, schedule=sched, flags=f)
        assert rc == 0 and info == 0
        assert scaled_error(L, Lref, S) <= TOL_SCALED
        outs.append(L)
    for L in outs[1:]:
        assert np.array_equal(outs[0], L)


def test_fp64tc_non_spd_info():
    import paper_2606_11937_gb300 as chol
    A = matrix("gram", 700, 4).copy()
    A[301, 301] -= 1000.0
    _, want = oracle.potrf_unblocked(A)
    for sched in ("dataflow", "fork_join", "left_looking", "top_looking"):
        _, info, _, rc = gpu_factor(A, schedule=sched, flags=chol.CHOL_FLAG_FP64_TC)
        assert rc == 0 and info == want


@pytest.mark.parametrize("nugget", [1e-2, 1e-3])
def test_fp64tc_inverse_trsm_parity(nugget):
    """SE covariance, ragged n: the TRSMs take the inverse path; FP64 parity
    bar against the oracle, residual bound, and bitwise agreement of the two
    schedules."""
    import paper_2606_11937_gb300 as chol
    n = 1500
    S = matrix("se", n, 5, nugget)
    Lref, _ = oracle_factor("se", n, 5, nugget)
    outs = []
    for sched in ("dataflow", "fork_join"):
        L, info, _, rc = gpu_factor(S, schedule=sched, flags=chol.CHOL_FLAG_FP64_TC | chol.CHOL_FLAG_PRIORITY)
        assert rc == 0 and info == 0
        assert scaled_error(L, Lref, S) <= TOL_SCALED
        assert probe_residual(S, L) <= resid_bound(n)
        outs.append(L)
    assert np.array_equal(outs[0], outs[1])


def test_fp64tc_withheld_dependency_times_out():
    """Fault made on the host, tensor-core engine: the last POTRF is never
    released, so CTAs holding a deferred quarter complete it and then wait on
    the queues until the bounded waits expire: CHOL_ERR_TIMEOUT, and the next
    factorization on the same context is correct."""
    import paper_2606_11937_gb300 as chol
    A = matrix("gram", 1024, 1)
    f = chol.CHOL_FLAG_FP64_TC | chol.CHOL_FLAG_PRIORITY
    _, info, st, rc = gpu_factor(A, schedule="dataflow", flags=f | chol.CHOL_FLAG_TEST_WITHHOLD, timeout_s=0.25)
    assert rc == chol.CHOL_ERR_TIMEOUT
    Lref, _ = oracle_factor("gram", 1024, 1)
    L, info, st, rc = gpu_factor(A, schedule="dataflow", flags=f)
    assert rc == 0 and scaled_error(L, Lref, A) <= TOL_SCALED


def test_fp64tc_trace_respects_dependencies():
    """With deferred completions a SYRK/GEMM's record ends when its last
    quarter is stored; every task still starts after its predecessors ended,
    and every task appears once."""
    import ctypes

    import torch

    import paper_2606_11937_gb300 as chol
    from paper_facts import GEMM, POTRF, SYRK, TRSM
    n = 2048
    A = matrix("gram", n, 2)
    m = n // 128
    cap = sum(task_counts(m)) + 10
    rsz = ctypes.sizeof(chol.chol_trace_rec)
    buf = torch.zeros(cap * rsz, dtype=torch.uint8, device="cuda")
    f = chol.CHOL_FLAG_FP64_TC | chol.CHOL_FLAG_PRIORITY
    _, info, st, rc = gpu_factor(A, schedule="dataflow", flags=f, trace=buf.data_ptr(), trace_capacity=cap)
    assert rc == 0 and st.trace_records == sum(task_counts(m))
    raw = buf.cpu().numpy()[: st.trace_records * rsz]
    rec = raw.view(np.dtype([("type", "<i4"), ("I", "<i4"), ("K", "<i4"), ("J", "<i4"), ("sm", "<i4"),
                             ("matrix", "<i4"), ("t0", "<u8"), ("t1", "<u8")]))
    ev = {(int(r["type"]), int(r["I"]), int(r["K"]), int(r["J"])): (int(r["t0"]), int(r["t1"])) for r in rec}
    assert len(ev) == sum(task_counts(m))
    for (ty, I, K, J), (t0, t1) in ev.items():
        assert t1 >= t0
        if ty == POTRF:
            needs = [(SYRK, I, I, J - 1)] if J > 0 else []
        elif ty == TRSM:
            needs = [(POTRF, J, J, J)] + ([(GEMM, I, J, J - 1)] if J > 0 else [])
        elif ty == SYRK:
            needs = [(TRSM, I, J, J)] + ([(SYRK, I, I, J - 1)] if J > 0 else [])
        else:
            needs = [(TRSM, I, J, J), (TRSM, K, J, J)] + ([(GEMM, I, K, J - 1)] if J > 0 else [])
        for nd in needs:
            assert ev[nd][1] <= t0, ((ty, I, K, J), nd)
