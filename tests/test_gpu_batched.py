"""Batched factor + solve in one persistent launch (CUDA graph).

* every batched factor equals the solo chol_factor_ex factor of the same
  matrix with the same tile order, bit for bit (same task bodies, same per-
  tile update order), and matches the oracle entrywise on a subset;
* every solution reaches the FP64 backward error 1e-14 (oracle-checked);
* a non-SPD matrix reports its info and leaves the others untouched;
* the graph replays with new data; FP32 batches match the oracle within a
  binary32 tolerance.
"""
import numpy as np
import pytest

import oracle
import seeded_inputs as si
from gpu_common import TOL_SCALED, scaled_error

pytestmark = pytest.mark.gpu


def make_batch(ns, seed0):
    As = [si.gram_plus_identity(int(n), seed0 + i) for i, n in enumerate(ns)]
    Bs = [si.rhs(int(n), 1, seed=seed0 + 1000 + i)[:, 0] for i, n in enumerate(ns)]
    return As, Bs


def run_batch(plan, As, Bs):
    import torch

    import paper_2606_11937_gb300 as chol
    dA = [chol.colmajor(A) for A in As]
    dB = [torch.from_numpy(b.copy()).cuda() for b in Bs]
    info = plan.run(dA, dB)
    torch.cuda.synchronize()
    return [np.tril(a.cpu().numpy()) for a in dA], [b.cpu().numpy() for b in dB], info


@pytest.mark.parametrize("cap", [0, 64, 2048])
def test_batched_fp64_matches_solo_and_oracle(cap):
    import paper_2606_11937_gb300 as chol
    ns = list(si.batched_sizes(48, seed=3, lo=32, hi=1024)) + [1, 2, 31, 33, 2048]
    As, Bs = make_batch(ns, 50)
    plan = chol.chol_batch_plan(ns, chol.opts(nb=cap))
    Ls, Xs, info = run_batch(plan, As, Bs)
    assert all(i == 0 for i in info)
    st = plan.stats()
    for k, (A, L, x, b) in enumerate(zip(As, Ls, Xs, Bs)):
        n = A.shape[0]
        assert oracle.backward_error(A, x.reshape(-1, 1), b.reshape(-1, 1)) <= 1e-14
        if k % 6 == 0 or n <= 33 or n > 1024:
            nb = cap if cap > 0 else chol.chol_default_nb(n, "fp64")
            nb = min(nb, n)
            Ls_solo, info_s, _, rc = _solo(A, nb)
            assert rc == 0, chol.chol_last_error()
            assert np.array_equal(L, Ls_solo), (k, n, nb)
            if n <= 1100:
                Lref, _ = oracle.potrf_unblocked(A)
                assert scaled_error(L, Lref, A) <= TOL_SCALED
    assert st.tasks[0] > 0
    plan.close()


def _solo(A, nb):
    import paper_2606_11937_gb300 as chol
    from gpu_common import gpu_factor
    # a batch factors matrices of order above 1024 on the tensor-core engine
    # (tile order 128, the default single factorization), the others with the
    # DFMA bodies at the batch's tile order
    if A.shape[0] > 1024:
        return gpu_factor(A, schedule="dataflow", nb=128)
    return gpu_factor(A, schedule="dataflow", nb=nb, flags=chol.CHOL_FLAG_FP64_SIMT)


def test_batched_failure_is_isolated_and_graph_replays():
    import paper_2606_11937_gb300 as chol
    ns = [300, 517, 64, 1000, 128]
    As, Bs = make_batch(ns, 70)
    plan = chol.chol_batch_plan(ns)
    L1, X1, info1 = run_batch(plan, As, Bs)
    assert info1 == [0] * 5
    bad = [A.copy() for A in As]
    bad[1][200, 200] = -1e6
    _, want = oracle.potrf_unblocked(bad[1])
    L2, X2, info2 = run_batch(plan, bad, Bs)
    assert info2[1] == want and all(info2[i] == 0 for i in (0, 2, 3, 4))
    for i in (0, 2, 3, 4):
        assert np.array_equal(L2[i], L1[i]) and np.array_equal(X2[i], X1[i])
    # replay with new data
    As3, Bs3 = make_batch(ns, 90)
    L3, X3, info3 = run_batch(plan, As3, Bs3)
    assert info3 == [0] * 5
    for A, x, b in zip(As3, X3, Bs3):
        assert oracle.backward_error(A, x.reshape(-1, 1), b.reshape(-1, 1)) <= 1e-14
    plan.close()


def test_batched_fp32():
    import paper_2606_11937_gb300 as chol
    ns = list(si.batched_sizes(24, seed=5, lo=32, hi=1500))
    As, Bs = make_batch(ns, 110)
    plan = chol.chol_batch_plan(ns, chol.opts(precision="fp32"))
    Ls, Xs, info = run_batch(plan, As, Bs)
    assert all(i == 0 for i in info)
    for A, L, x, b in zip(As, Ls, Xs, Bs):
        n = A.shape[0]
        if n <= 1100:
            Lref, _ = oracle.potrf_unblocked(A)
            assert scaled_error(L, Lref, A) <= 1e-5  # binary32 factor
        assert oracle.backward_error(A, x.reshape(-1, 1), b.reshape(-1, 1)) <= 1e-6
    plan.close()


def test_batched_arguments():
    import paper_2606_11937_gb300 as chol
    with pytest.raises(chol.CholError):
        chol.chol_batch_plan([10, 4096])
    with pytest.raises(chol.CholError):
        chol.chol_batch_plan([10], chol.opts(precision="bf16"))


def test_batched_tensor_core_part():
    """FP64 matrices of order above 1024 run in the batch's tensor-core part
    (one persistent kernel of the tensor-core engine for all of them, with
    the fused SOLVE task): each factor equals the single default FP64
    factorization (tile order 128) bit for bit, every solution reaches the
    1e-14 backward error, a failing large matrix reports the oracle's info and
    leaves the others untouched, a batch of large matrices only works, and
    CHOL_FLAG_FP64_SIMT keeps every matrix on the CUDA-core bodies."""
    import paper_2606_11937_gb300 as chol
    ns = [1100, 300, 2048, 1025, 64, 1536, 700, 1300]
    As, Bs = make_batch(ns, 130)
    plan = chol.chol_batch_plan(ns)
    Ls, Xs, info = run_batch(plan, As, Bs)
    assert info == [0] * len(ns)
    for A, L, x, b in zip(As, Ls, Xs, Bs):
        n = A.shape[0]
        assert oracle.backward_error(A, x.reshape(-1, 1), b.reshape(-1, 1)) <= 1e-14
        if n > 1024:
            Lsolo, info_s, _, rc = _solo(A, 128)
            assert rc == 0 and info_s == 0 and np.array_equal(L, Lsolo), n
    # failures inside the tensor-core part: one at the first diagonal tile
    # (every later task of that matrix a no-op while the others still run),
    # one deep inside
    _check_failures(plan, As, Bs, Ls, Xs, (3, 5))
    plan.close()
    # only large matrices
    big = [1200, 1800, 1030]
    Ab, Bb = make_batch(big, 150)
    plan = chol.chol_batch_plan(big)
    Lb, Xb, infob = run_batch(plan, Ab, Bb)
    assert infob == [0] * 3
    for A, x, b in zip(Ab, Xb, Bb):
        assert oracle.backward_error(A, x.reshape(-1, 1), b.reshape(-1, 1)) <= 1e-14
    plan.close()
    # forced onto the CUDA-core bodies
    plan = chol.chol_batch_plan(big, chol.opts(nb=64, flags=chol.CHOL_FLAG_FP64_SIMT))
    Ls2, Xs2, infos2 = run_batch(plan, Ab, Bb)
    assert infos2 == [0] * 3
    from gpu_common import gpu_factor
    for A, L in zip(Ab, Ls2):
        Lsolo, _, _, rc = gpu_factor(A, schedule="dataflow", nb=64, flags=chol.CHOL_FLAG_FP64_SIMT)
        assert rc == 0 and np.array_equal(L, Lsolo)
    plan.close()


def _check_failures(plan, As, Bs, Ls, Xs, which):
    bad = [A.copy() for A in As]
    bad[which[0]][5, 5] = -1e6
    bad[which[1]][900, 900] = -1e6
    want = {i: oracle.potrf_unblocked(bad[i])[1] for i in which}
    L2, X2, info2 = run_batch(plan, bad, Bs)
    for i in range(len(As)):
        if i in which:
            assert info2[i] == want[i], (i, info2[i], want[i])
        else:
            assert info2[i] == 0 and np.array_equal(L2[i], Ls[i]) and np.array_equal(X2[i], Xs[i]), i


def _fp32_alone_equals_mix(ns, As, Bs, Ls, o, which):
    """Each matrix in `which` factored in a batch of its own gives the bits it
    got in the mixed batch (the bits of a matrix do not depend on the rest)."""
    import paper_2606_11937_gb300 as chol
    for k in which:
        plan = chol.chol_batch_plan([ns[k]], o)
        L1, _, info1 = run_batch(plan, [As[k]], [Bs[k]])
        plan.close()
        assert info1 == [0] and np.array_equal(L1[0], Ls[k]), ns[k]


def test_batched_fp32_tensor_core_part():
    """FP32 matrices of order above 1024 run in the batch's tensor-core part
    (tile order 128: diagonal tiles factored in binary32 in shared memory,
    binary32 TRSM, SYRK/GEMM as three TF32 products, one persistent kernel with
    the fused binary32 SOLVE): exact-integer inputs A = L0 L0^T give L0 bit for
    bit; factors are within the binary32 tolerance of the oracle and each
    matrix gets the same bits alone and in the batch; every solution reaches
    the binary32 backward error; failing matrices report the oracle's info and
    leave the others untouched; tc_min_order = 2048 keeps every matrix on the
    CUDA cores."""
    import paper_2606_11937_gb300 as chol
    ns = [1100, 300, 2048, 1025, 64, 1536, 700, 1300]
    o = chol.opts(precision="fp32")
    # exact pin: every operation on these integers is exact in binary32
    ints = [si.exact_integer_factor(n, seed=230 + i) for i, n in enumerate([1100, 1536, 2048])]
    plan = chol.chol_batch_plan([A.shape[0] for A, _ in ints], o)
    Li, _, infoi = run_batch(plan, [A for A, _ in ints], [si.rhs(A.shape[0], 1, seed=7)[:, 0] for A, _ in ints])
    plan.close()
    assert infoi == [0, 0, 0]
    for (A, L0), L in zip(ints, Li):
        assert np.array_equal(L, L0), A.shape[0]
    As, Bs = make_batch(ns, 190)
    plan = chol.chol_batch_plan(ns, o)
    Ls, Xs, info = run_batch(plan, As, Bs)
    assert info == [0] * len(ns)
    assert plan.stats().tasks[3] > 0
    for A, L, x, b in zip(As, Ls, Xs, Bs):
        assert oracle.backward_error(A, x.reshape(-1, 1), b.reshape(-1, 1)) <= 1e-6
        Lref, _ = oracle.potrf_unblocked(A)
        assert scaled_error(L, Lref, A) <= 1e-5, A.shape[0]
    _check_failures(plan, As, Bs, Ls, Xs, (0, 5))
    plan.close()
    _fp32_alone_equals_mix(ns, As, Bs, Ls, o, (0, 2, 3))
    # every matrix on the CUDA cores
    plan = chol.chol_batch_plan(ns, chol.opts(precision="fp32", tc_min_order=2048))
    Lc, Xc, infoc = run_batch(plan, As, Bs)
    assert infoc == [0] * len(ns)
    for A, L, x, b in zip(As, Lc, Xc, Bs):
        assert oracle.backward_error(A, x.reshape(-1, 1), b.reshape(-1, 1)) <= 1e-6
        if A.shape[0] <= 1100:
            Lref, _ = oracle.potrf_unblocked(A)
            assert scaled_error(L, Lref, A) <= 1e-5
    plan.close()


def test_batched_fp32_tensor_core_small_orders():
    """tc_min_order = 100 in an FP32 plan: matrices of one padded tile of order
    128 (n = 101, 128), of two tiles with a one-row ragged tile (129) and a few
    tiles run in the tensor-core part: exact-integer inputs give L0 bit for
    bit, the others are within the binary32 tolerance of the oracle, get the
    same bits alone and in the batch and reach the binary32 backward error;
    the matrix below the split stays on the CUDA cores."""
    import paper_2606_11937_gb300 as chol
    ns = [101, 128, 129, 250, 90, 384]
    o = chol.opts(precision="fp32", tc_min_order=100)
    ints = [si.exact_integer_factor(n, seed=250 + i) for i, n in enumerate(ns)]
    plan = chol.chol_batch_plan(ns, o)
    Li, _, infoi = run_batch(plan, [A for A, _ in ints], [si.rhs(n, 1, seed=8)[:, 0] for n in ns])
    plan.close()
    assert infoi == [0] * len(ns)
    for (A, L0), L in zip(ints, Li):
        assert np.array_equal(L, L0), A.shape[0]
    As, Bs = make_batch(ns, 210)
    plan = chol.chol_batch_plan(ns, o)
    Ls, Xs, info = run_batch(plan, As, Bs)
    assert info == [0] * len(ns)
    for A, L, x, b in zip(As, Ls, Xs, Bs):
        assert oracle.backward_error(A, x.reshape(-1, 1), b.reshape(-1, 1)) <= 1e-6
        Lref, _ = oracle.potrf_unblocked(A)
        assert scaled_error(L, Lref, A) <= 1e-5
    plan.close()
    _fp32_alone_equals_mix(ns, As, Bs, Ls, o, (0, 2, 5))


def test_batched_tensor_core_split_order():
    """tc_min_order = 256: the matrices of order above 256 run in the
    tensor-core part and each equals the single factorization with
    CHOL_FLAG_FP64_TC at tile order 128 bit for bit."""
    import paper_2606_11937_gb300 as chol
    from gpu_common import gpu_factor
    ns = [200, 257, 640, 1100, 100]
    As, Bs = make_batch(ns, 170)
    plan = chol.chol_batch_plan(ns, chol.opts(tc_min_order=256))
    Ls, Xs, info = run_batch(plan, As, Bs)
    assert info == [0] * len(ns)
    for A, L, x, b in zip(As, Ls, Xs, Bs):
        assert oracle.backward_error(A, x.reshape(-1, 1), b.reshape(-1, 1)) <= 1e-14
        if A.shape[0] > 256:
            Lsolo, _, _, rc = gpu_factor(A, schedule="dataflow", nb=128, flags=chol.CHOL_FLAG_FP64_TC)
            assert rc == 0 and np.array_equal(L, Lsolo), A.shape[0]
    plan.close()
