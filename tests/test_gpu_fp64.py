"""FP64 factorization on the GPU against the oracle, through the C ABI.

Parity: scaled entrywise error <= 1e-11 against the oracle's unblocked
factor, residual <= 1e-14 sqrt(n), bit-exact on inputs whose factor is exact
(Pascal, integer L0).  Schedules: fork-join (collapsed and naive) and the
dataflow kernel must give identical bits (same per-tile update order), and
execute exactly the task counts of Section 4.2.
"""
import ctypes

import numpy as np
import pytest

from gpu_common import TOL_SCALED, gpu_factor, matrix, oracle_factor, probe_residual, resid_bound, scaled_error
from paper_facts import task_counts

pytestmark = pytest.mark.gpu

SCHEDS = ["dataflow", "fork_join", "fork_join_naive", "left_looking", "top_looking"]


@pytest.mark.parametrize("sched", SCHEDS)
def test_config1_n2048_nb256(sched):
    """A = G G^T / n + I, n = 2048, nb = 256 (8 x 8 tiles), seed 0: entrywise."""
    A = matrix("gram", 2048, 0)
    Lref, _ = oracle_factor("gram", 2048, 0)
    L, info, st, rc = gpu_factor(A, schedule=sched, nb=256)
    assert rc == 0 and info == 0
    assert scaled_error(L, Lref, A) <= TOL_SCALED
    assert probe_residual(A, L) <= resid_bound(2048)
    assert tuple(st.tasks) == task_counts(8)


@pytest.mark.parametrize("n,nb", [(1000, 128), (777, 64), (37, 64), (1, 16), (2, 1), (129, 128), (700, 96),
                                  (513, 32), (300, 300), (257, 17)])
def test_ragged_and_small(n, nb):
    """n not a multiple of nb, n < nb, odd tile orders: identity padding."""
    A = matrix("se", n, 3, 1e-1)
    Lref, _ = oracle_factor("se", n, 3, 1e-1)
    outs = []
    for sched in SCHEDS:
        L, info, st, rc = gpu_factor(A, schedule=sched, nb=nb)
        assert rc == 0 and info == 0
        assert scaled_error(L, Lref, A) <= TOL_SCALED
        m = -(-n // nb)
        assert tuple(st.tasks) == task_counts(m)
        outs.append(L)
    for L in outs[1:]:
        assert np.array_equal(L, outs[0])


@pytest.mark.parametrize("nb", [1, 3, 8, 16, 29, 32, 64])
def test_pascal_exact(nb):
    import seeded_inputs as si
    P = si.pascal(29)
    for sched in SCHEDS:
        L, info, _, rc = gpu_factor(P, schedule=sched, nb=nb)
        assert rc == 0 and info == 0
        assert np.array_equal(L, si.pascal_lower(29))


@pytest.mark.parametrize("n,nb", [(1500, 128), (1024, 256), (600, 64), (333, 50)])
def test_exact_integer_factor(n, nb):
    import seeded_inputs as si
    A, L0 = si.exact_integer_factor(n, seed=n)
    for sched in SCHEDS:
        L, info, _, rc = gpu_factor(A, schedule=sched, nb=nb)
        assert rc == 0 and info == 0
        assert np.array_equal(L, L0)


@pytest.mark.parametrize("nb", [16, 64, 100])
def test_schedules_bitwise_equal_with_priority(nb):
    import paper_2606_11937_gb300 as chol
    A = matrix("se", 900, 5, 1e-2)
    ref, *_ = gpu_factor(A, schedule="fork_join", nb=nb)
    for flags in (0, chol.CHOL_FLAG_PRIORITY):
        for ctas in (0, 7, 1000):
            L, info, st, rc = gpu_factor(A, schedule="dataflow", nb=nb, flags=flags, num_ctas=ctas)
            assert rc == 0 and info == 0
            assert np.array_equal(L, ref)


@pytest.mark.parametrize("sched", ["fork_join", "fork_join_naive", "left_looking", "top_looking"])
def test_graph_replay_same_bits(sched):
    """CHOL_FLAG_GRAPH: the launch-ordered schedules captured into a CUDA graph
    give the bits of the direct launches, with the same launch count."""
    import paper_2606_11937_gb300 as chol
    A = matrix("se", 1000, 6, 1e-2)
    L0, info0, st0, rc0 = gpu_factor(A, schedule=sched, nb=64)
    L1, info1, st1, rc1 = gpu_factor(A, schedule=sched, nb=64, flags=chol.CHOL_FLAG_GRAPH)
    assert rc0 == rc1 == 0 and info0 == info1 == 0
    assert np.array_equal(L0, L1)
    assert st0.launches == st1.launches
    assert tuple(st1.tasks) == task_counts(16)


def test_left_looking_launch_count():
    """Left-looking: per block column K an update launch (K > 0), the POTRF and
    the TRSM grid (K < M - 1): 3M - 2 schedule launches, as many as the
    right-looking fork-join (POTRF, TRSM grid, update grid per step J < M - 1,
    and the last POTRF); the same bits."""
    A = matrix("gram", 1024, 2)
    L, info, st, rc = gpu_factor(A, schedule="left_looking", nb=128)
    Lr, info_r, st_r, rc_r = gpu_factor(A, schedule="fork_join", nb=128)
    assert rc == rc_r == 0 and info == info_r == 0
    assert st.launches == st_r.launches
    assert np.array_equal(L, Lr)


def test_non_spd_info():
    """info = first failing leading minor, as the oracle reports it."""
    import oracle
    n = 700
    A = matrix("gram", n, 4).copy()
    for k in (0, 5, 63, 64, 301, 699):
        B = A.copy()
        B[k, k] -= 1000.0
        _, want = oracle.potrf_unblocked(B)
        assert want == k + 1
        for sched in SCHEDS:
            for nb in (32, 64, 128):
                _, info, _, rc = gpu_factor(B, schedule=sched, nb=nb)
                assert rc == 0 and info == want, (sched, nb, k, info)
    C = np.eye(100)
    C[40, 40] = np.nan
    for sched in SCHEDS:
        _, info, _, rc = gpu_factor(C, schedule=sched, nb=32)
        assert info == 41


def test_upper_triangle_untouched_and_lda():
    import torch

    import paper_2606_11937_gb300 as chol
    n, lda = 500, 640
    A = matrix("gram", n, 6)
    Lref, _ = oracle_factor("gram", n, 6)
    host = np.full((lda, n), 7.25)
    host[:n, :n] = np.tril(A) + np.triu(np.full((n, n), -3.5), 1)
    buf = torch.from_numpy(np.asfortranarray(host)).cuda()
    dA = torch.empty_strided((lda, n), (1, lda), dtype=torch.float64, device="cuda")
    dA.copy_(buf)
    sub = dA[:n, :]
    for sched in SCHEDS:
        dA.copy_(buf)
        rc, info, _ = chol.chol_factor_ex(sub, chol.opts(schedule=sched, nb=64), n=n, lda=lda)
        torch.cuda.synchronize()
        out = dA.cpu().numpy()
        assert info == 0
        assert np.array_equal(np.triu(out[:n, :n], 1), np.triu(host[:n, :n], 1))
        assert np.array_equal(out[n:, :], host[n:, :])
        assert scaled_error(out[:n, :n], Lref, A) <= TOL_SCALED


def test_argument_errors():
    import paper_2606_11937_gb300 as chol
    L = chol.lib()
    assert L.chol_factor(0, 64, None, 1) == chol.CHOL_OK
    assert L.chol_factor(-1, 64, None, 1) == chol.CHOL_ERR_ARG
    assert L.chol_factor(10, 0, None, 10) == chol.CHOL_ERR_ARG
    assert L.chol_factor(10, 4, None, 10) == chol.CHOL_ERR_ARG
    assert L.chol_factor(10, 4, 12345, 5) == chol.CHOL_ERR_ARG
    assert "lda" in chol.chol_last_error()


def test_chol_factor_plain_entry():
    """chol_factor(n, nb, A, lda) -- the paper-shaped entry point."""
    import torch

    import paper_2606_11937_gb300 as chol
    n = 640
    A = matrix("gram", n, 8)
    Lref, _ = oracle_factor("gram", n, 8)
    dA = chol.colmajor(A)
    assert chol.chol_factor(n, 64, dA) == chol.CHOL_OK
    torch.cuda.synchronize()
    assert scaled_error(dA.cpu().numpy(), Lref, A) <= TOL_SCALED
    B = A.copy()
    B[10, 10] = -5.0
    dB = chol.colmajor(B)
    assert chol.chol_factor(n, 64, dB) == chol.CHOL_ERR_NOT_SPD
    assert chol.chol_last_info() == 11


@pytest.mark.parametrize("n,lda", [(513, 513), (1300, 1310)])
def test_host_buffer_entry(n, lda):
    """Host buffer in and out (only the lower triangle travels, in blocks of
    512 columns): the factor in the lower triangle, the strict upper triangle
    and the padding rows beyond n exactly as they were."""
    import torch

    import paper_2606_11937_gb300 as chol
    A = matrix("gram", n, 9)
    Lref, _ = oracle_factor("gram", n, 9)
    h = torch.full((n, lda), -7.25, dtype=torch.float64).pin_memory()  # column j at h[j, :]
    hv = h.T  # lda x n column-major view
    hv[:n, :] = torch.from_numpy(A)
    before = hv.clone()
    info, st = chol.chol_factor_host(hv, chol.opts(nb=64, schedule="dataflow"), n=n, lda=lda)
    assert info == 0
    out = hv.numpy()
    assert scaled_error(out[:n, :n], Lref, A) <= TOL_SCALED
    assert np.array_equal(np.triu(out[:n, :n], 1), np.triu(before.numpy()[:n, :n], 1))
    assert np.array_equal(out[n:, :], before.numpy()[n:, :])


def test_noop_mode_runs_the_task_graph():
    """Section 4.2 no-op runs: every task body replaced by nothing; the task
    graph still runs to completion with the exact task counts."""
    import paper_2606_11937_gb300 as chol
    A = matrix("gram", 2048, 0)
    for sched in SCHEDS:
        for nb in (16, 64):
            _, info, st, rc = gpu_factor(A, schedule=sched, nb=nb, flags=chol.CHOL_FLAG_NOOP)
            assert rc == 0 and info == 0
            assert tuple(st.tasks) == task_counts(2048 // nb)


def test_withheld_dependency_times_out():
    """Fault test made on the host: the dataflow kernel is told never to
    release the last POTRF; every wait is bounded, so the call returns
    CHOL_ERR_TIMEOUT and the context stays usable."""
    import paper_2606_11937_gb300 as chol
    A = matrix("gram", 512, 1)
    _, info, st, rc = gpu_factor(A, schedule="dataflow", nb=64, flags=chol.CHOL_FLAG_TEST_WITHHOLD, timeout_s=0.25)
    assert rc == chol.CHOL_ERR_TIMEOUT
    Lref, _ = oracle_factor("gram", 512, 1)
    L, info, st, rc = gpu_factor(A, schedule="dataflow", nb=64)
    assert rc == 0 and scaled_error(L, Lref, A) <= TOL_SCALED


@pytest.mark.parametrize("flags", [0, 16])
def test_top_looking_withheld_tile_times_out(flags):
    """Fault made on the host, top-looking wavefront: tile (M-1, 0) is never
    published, so the row's other tiles wait until the bounded waits expire:
    CHOL_ERR_TIMEOUT, and the next factorization on the context is correct
    (DFMA and tensor-core engines)."""
    import paper_2606_11937_gb300 as chol
    A = matrix("gram", 640, 3)
    nb = 128 if flags else 64
    _, info, st, rc = gpu_factor(A, schedule="top_looking", nb=nb, flags=flags | chol.CHOL_FLAG_TEST_WITHHOLD,
                                 timeout_s=0.25)
    assert rc == chol.CHOL_ERR_TIMEOUT
    Lref, _ = oracle_factor("gram", 640, 3)
    L, info, st, rc = gpu_factor(A, schedule="top_looking", nb=nb, flags=flags)
    assert rc == 0 and scaled_error(L, Lref, A) <= TOL_SCALED


def test_trace_respects_dependencies():
    """Per-task %globaltimer records: every task starts after its predecessors
    ended, and each tile's updates run in ascending J."""
    import torch

    import paper_2606_11937_gb300 as chol
    from paper_facts import GEMM, POTRF, SYRK, TRSM
    A = matrix("gram", 1024, 2)
    m = 1024 // 64
    cap = sum(task_counts(m)) + 10
    rsz = ctypes.sizeof(chol.chol_trace_rec)
    assert rsz == 40
    buf = torch.zeros(cap * rsz, dtype=torch.uint8, device="cuda")
    for sched in ("dataflow", "fork_join"):
        buf.zero_()
        _, info, st, rc = gpu_factor(A, schedule=sched, nb=64, trace=buf.data_ptr(), trace_capacity=cap)
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


@pytest.mark.parametrize("nrhs", [3, 5])
def test_solve_exact_integer_factor(nrhs):
    """L0 with diagonal in {1, 2, 4} and small integer entries, x integer, b = A x:
    every intermediate of both sweeps is an integer, so the solve must return x
    exactly.  The diagonal blocks of L0 are ill-conditioned (kappa_inf about
    1e12), so this also runs the substitution the solve keeps for them."""
    import torch

    import paper_2606_11937_gb300 as chol
    import seeded_inputs as si
    n = 1000
    A, L0 = si.exact_integer_factor(n, seed=31)
    r = si.rng(32)
    X0 = r.integers(-3, 4, size=(n, nrhs)).astype(np.float64)
    B = A @ X0
    assert np.max(np.abs(B)) < 2.0 ** 50
    dL = chol.colmajor(L0)
    dB = chol.colmajor(B)
    chol.chol_solve_ex(dL, dB)
    torch.cuda.synchronize()
    assert np.array_equal(dB.cpu().numpy(), X0)


@pytest.mark.parametrize("n,nrhs", [(2048, 1), (1000, 16), (777, 37), (64, 3), (1, 1)])
def test_solve_fp64(n, nrhs):
    import torch

    import oracle
    import paper_2606_11937_gb300 as chol
    import seeded_inputs as si
    A = matrix("gram", n, 11)
    Lref, _ = oracle_factor("gram", n, 11)
    B = si.rhs(n, nrhs, seed=12)
    Xref = oracle.potrs(Lref, B)
    dL = chol.colmajor(Lref)
    dB = chol.colmajor(B)
    chol.chol_solve_ex(dL, dB)
    torch.cuda.synchronize()
    X = dB.cpu().numpy()
    assert np.max(np.abs(X - Xref)) / np.max(np.abs(Xref)) <= 1e-12
    assert oracle.backward_error(A, X, B) <= 1e-14
    dB2 = chol.colmajor(B)
    assert chol.chol_solve(n, nrhs, dL, dB2) == 0
    torch.cuda.synchronize()
    assert np.array_equal(dB2.cpu().numpy(), X)
