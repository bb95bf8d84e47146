"""The FP64 engine the default call selects above order 1024: SYRK/GEMM/TRSM
as exact bf16 slice products on the tensor cores, at tile orders nb = 128 r
(the paper's tile-size sweep, Section 4.1, runs over these).

A task on a tile of order 128 r runs its r x r blocks of order 128 in the
order the tiled algorithm (Section 3.1, Fig. 1) gives them at tile order 128,
so every tile order and every schedule must give the SAME bits; the battery
of the FP64 parity tests runs on this engine:

* against the oracle: scaled entrywise error <= 1e-11 and residual
  <= 1e-14 sqrt(n) (config 1: n = 2048, A = G G^T / n + I, seed 0, at
  nb = 128, 256, 512, 1024; ragged orders);
* exact inputs: the integer factor A = L0 L0^T and the Pascal matrix are
  reproduced bit for bit;
* Section 4.2 task counts at the task tile order; LAPACK info of a matrix
  that is not positive definite; the strict upper triangle and rows past n
  untouched; host buffers; the paper-shaped chol_factor(n, nb, A, lda);
* the trace: every task starts after its predecessors ended.
"""
import ctypes

import numpy as np
import pytest

import seeded_inputs as si
from gpu_common import TOL_SCALED, gpu_factor, matrix, oracle_factor, probe_residual, resid_bound, scaled_error
from paper_facts import GEMM, POTRF, SYRK, TRSM, task_counts

pytestmark = pytest.mark.gpu

SCHEDS = ["dataflow", "fork_join", "fork_join_naive", "left_looking", "top_looking"]


def test_default_engine_is_the_tensor_core_engine_above_1024():
    """The default call gives the bits of CHOL_FLAG_FP64_TC above order 1024,
    and of CHOL_FLAG_FP64_SIMT at or below it (the choice depends on n and nb
    only)."""
    import paper_2606_11937_gb300 as chol
    A = matrix("gram", 1100, 21)
    d, *_ = gpu_factor(A, schedule="dataflow", nb=256)
    t, *_ = gpu_factor(A, schedule="dataflow", nb=256, flags=chol.CHOL_FLAG_FP64_TC)
    assert np.array_equal(d, t)
    B = matrix("gram", 1000, 22)
    d, *_ = gpu_factor(B, schedule="dataflow", nb=256)
    s, *_ = gpu_factor(B, schedule="dataflow", nb=256, flags=chol.CHOL_FLAG_FP64_SIMT)
    assert np.array_equal(d, s)
    # a tile order that is not a multiple of 128 stays on the DFMA engine
    d, *_ = gpu_factor(A, schedule="dataflow", nb=100)
    s, *_ = gpu_factor(A, schedule="dataflow", nb=100, flags=chol.CHOL_FLAG_FP64_SIMT)
    assert np.array_equal(d, s)
    # ... and the tensor-core engine refuses it
    _, info, st, rc = gpu_factor(A, schedule="dataflow", nb=100, flags=chol.CHOL_FLAG_FP64_TC)
    assert rc == chol.CHOL_ERR_ARG


def test_config1_every_tile_order_and_schedule_same_bits():
    A = matrix("gram", 2048, 0)
    Lref, _ = oracle_factor("gram", 2048, 0)
    ref = None
    for nb in (128, 256, 512, 1024):
        for sched in SCHEDS:
            L, info, st, rc = gpu_factor(A, schedule=sched, nb=nb)
            assert rc == 0 and info == 0
            assert st.nb == nb
            assert tuple(st.tasks) == task_counts(2048 // nb)
            if ref is None:
                ref = L
                assert scaled_error(L, Lref, A) <= TOL_SCALED
                assert probe_residual(A, L) <= resid_bound(2048)
            assert np.array_equal(L, ref), (nb, sched)


@pytest.mark.parametrize("n", [1111, 1500, 2100])
def test_ragged_tile_orders_same_bits(n):
    """n not a multiple of 128 r: the blocks past the matrix are skipped (the
    last tile is padded with the identity); every tile order, priorities on
    or off, gives the bits of tile order 128."""
    import paper_2606_11937_gb300 as chol
    A = matrix("se", n, 3, 1e-2)
    Lref, _ = oracle_factor("se", n, 3, 1e-2)
    ref = None
    for nb in (128, 256, 384, 640):
        for sched, flags in (("dataflow", 0), ("dataflow", chol.CHOL_FLAG_PRIORITY), ("fork_join", 0),
                             ("top_looking", 0)):
            L, info, st, rc = gpu_factor(A, schedule=sched, nb=nb, flags=flags)
            assert rc == 0 and info == 0
            assert tuple(st.tasks) == task_counts(-(-n // nb))
            if ref is None:
                ref = L
                assert scaled_error(L, Lref, A) <= TOL_SCALED
            assert np.array_equal(L, ref), (nb, sched, flags)


@pytest.mark.parametrize("nb", [128, 256, 512])
def test_exact_integer_factor(nb):
    A, L0 = si.exact_integer_factor(1500, seed=1500)
    for sched in SCHEDS:
        L, info, _, rc = gpu_factor(A, schedule=sched, nb=nb)
        assert rc == 0 and info == 0
        assert np.array_equal(L, L0), (nb, sched)


@pytest.mark.parametrize("nb", [128, 256])
def test_pascal_exact_on_the_tensor_core_engine(nb):
    """n = 29 < 128: one padded block (forced onto this engine)."""
    import paper_2606_11937_gb300 as chol
    P = si.pascal(29)
    for sched in SCHEDS:
        L, info, _, rc = gpu_factor(P, schedule=sched, nb=nb, flags=chol.CHOL_FLAG_FP64_TC)
        assert rc == 0 and info == 0
        assert np.array_equal(L, si.pascal_lower(29))


def test_non_spd_info():
    """info = the first failing leading minor, as the oracle reports it, at
    block boundaries and inside blocks, for every tile order."""
    import oracle
    n = 1300
    A = matrix("gram", n, 4).copy()
    for k in (0, 127, 128, 300, 700, 1299):
        B = A.copy()
        B[k, k] -= 1000.0
        _, want = oracle.potrf_unblocked(B)
        assert want == k + 1
        for nb in (128, 256, 512):
            for sched in ("dataflow", "fork_join", "top_looking"):
                _, info, _, rc = gpu_factor(B, schedule=sched, nb=nb)
                assert rc == 0 and info == want, (sched, nb, k, info)


def test_upper_triangle_untouched_and_lda():
    import torch

    import paper_2606_11937_gb300 as chol
    n, lda = 1200, 1333
    A = matrix("gram", n, 6)
    Lref, _ = oracle_factor("gram", n, 6)
    host = np.full((lda, n), 7.25)
    host[:n, :n] = np.tril(A) + np.triu(np.full((n, n), -3.5), 1)
    buf = torch.from_numpy(np.asfortranarray(host)).cuda()
    dA = torch.empty_strided((lda, n), (1, lda), dtype=torch.float64, device="cuda")
    sub = dA[:n, :]
    for nb in (128, 256):
        for sched in ("dataflow", "fork_join"):
            dA.copy_(buf)
            rc, info, st = chol.chol_factor_ex(sub, chol.opts(schedule=sched, nb=nb), n=n, lda=lda)
            torch.cuda.synchronize()
            out = dA.cpu().numpy()
            assert info == 0 and st.nb == nb
            assert np.array_equal(np.triu(out[:n, :n], 1), np.triu(host[:n, :n], 1))
            assert np.array_equal(out[n:, :], host[n:, :])
            assert scaled_error(out[:n, :n], Lref, A) <= TOL_SCALED


def test_host_buffer_entry():
    import torch

    import paper_2606_11937_gb300 as chol
    n, lda = 1300, 1310
    A = matrix("gram", n, 9)
    Lref, _ = oracle_factor("gram", n, 9)
    h = torch.full((n, lda), -7.25, dtype=torch.float64).pin_memory()
    hv = h.T
    hv[:n, :] = torch.from_numpy(A)
    before = hv.clone()
    info, st = chol.chol_factor_host(hv, chol.opts(nb=256, schedule="dataflow"), n=n, lda=lda)
    assert info == 0 and st.nb == 256
    out = hv.numpy()
    assert scaled_error(out[:n, :n], Lref, A) <= TOL_SCALED
    assert np.array_equal(np.triu(out[:n, :n], 1), np.triu(before.numpy()[:n, :n], 1))
    assert np.array_equal(out[n:, :], before.numpy()[n:, :])


def test_chol_factor_plain_entry():
    """chol_factor(n, nb, A, lda), the paper-shaped call, on this engine."""
    import torch

    import paper_2606_11937_gb300 as chol
    n = 2048
    A = matrix("gram", n, 0)
    Lref, _ = oracle_factor("gram", n, 0)
    dA = chol.colmajor(A)
    assert chol.chol_factor(n, 256, dA) == chol.CHOL_OK
    torch.cuda.synchronize()
    assert scaled_error(dA.cpu().numpy(), Lref, A) <= TOL_SCALED
    B = A.copy()
    B[1500, 1500] = -5.0
    dB = chol.colmajor(B)
    assert chol.chol_factor(n, 256, dB) == chol.CHOL_ERR_NOT_SPD
    assert chol.chol_last_info() == 1501


@pytest.mark.parametrize("nb", [256, 512])
def test_trace_respects_dependencies(nb):
    import torch

    import paper_2606_11937_gb300 as chol
    n = 2048
    A = matrix("gram", n, 2)
    m = n // nb
    cap = sum(task_counts(m)) + 10
    rsz = ctypes.sizeof(chol.chol_trace_rec)
    buf = torch.zeros(cap * rsz, dtype=torch.uint8, device="cuda")
    for flags in (0, chol.CHOL_FLAG_PRIORITY):
        buf.zero_()
        _, info, st, rc = gpu_factor(A, schedule="dataflow", nb=nb, flags=flags, trace=buf.data_ptr(),
                                     trace_capacity=cap)
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


def test_withheld_dependency_times_out_at_tile_order_256():
    import paper_2606_11937_gb300 as chol
    A = matrix("gram", 2048, 1)
    _, info, st, rc = gpu_factor(A, schedule="dataflow", nb=256, flags=chol.CHOL_FLAG_TEST_WITHHOLD, timeout_s=0.25)
    assert rc == chol.CHOL_ERR_TIMEOUT
    Lref, _ = oracle_factor("gram", 2048, 1)
    L, info, st, rc = gpu_factor(A, schedule="dataflow", nb=256)
    assert rc == 0 and scaled_error(L, Lref, A) <= TOL_SCALED


@pytest.mark.parametrize("sched", ["dataflow", "fork_join"])
def test_host_buffer_not_spd_and_schedules(sched):
    """The host-buffer call on this engine: with the dataflow schedule each
    block column is copied back as soon as it is final (a copy stream waits on
    per-column flags); a matrix that is not positive definite still returns
    (every flag is released after the schedule) with the oracle's info, and
    the fork-join schedule copies back after the factorization."""
    import torch

    import oracle
    import paper_2606_11937_gb300 as chol
    n = 1300
    A = matrix("gram", n, 9)
    Lref, _ = oracle_factor("gram", n, 9)
    for nb in (128, 256):
        h = torch.from_numpy(np.asfortranarray(A)).T.contiguous().T.pin_memory()
        info, st = chol.chol_factor_host(h, chol.opts(nb=nb, schedule=sched))
        assert info == 0
        assert scaled_error(h.numpy(), Lref, A) <= TOL_SCALED
    B = A.copy()
    B[900, 900] -= 1000.0
    _, want = oracle.potrf_unblocked(B)
    h = torch.from_numpy(np.asfortranarray(B)).T.contiguous().T.pin_memory()
    info, st = chol.chol_factor_host(h, chol.opts(nb=128, schedule=sched))
    assert info == want == 901
