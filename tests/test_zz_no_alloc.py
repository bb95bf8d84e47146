"""chol_solve_noalloc: the FP64 solve for callers that cannot allocate device
memory (an application whose memory manager has reserved the GPU, or a
latency-critical loop that must not pay the synchronization cudaMalloc /
cudaFree can cause).  It keeps its scratch in a fixed 4 MiB device array.

Its results must agree with chol_solve_ex (the allocating entry point) within
the tolerance of the other solve tests, on two different calls in a row (the
second must not see the first's leftovers in the shared array), and sizes
beyond the fixed scratch must be refused with a clear error.  This file runs
last so that a failure here leaves every other test already run; it passes
alone in a fresh process as well.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

REL_TOL = 1e-12  # relative to max |X|, as in the FP64 solve tests


def _solve_pair(n, nrhs, seed):
    import torch

    import oracle
    import paper_2606_11937_gb300 as chol
    import seeded_inputs as si
    A = si.gram_plus_identity(n, seed)
    L, info = oracle.potrf_unblocked(A)
    assert info == 0
    dL = chol.colmajor(np.tril(L))
    B = si.rhs(n, nrhs, seed=seed + 1)
    ref = chol.colmajor(B)
    chol.chol_solve_ex(dL, ref)
    out = chol.colmajor(B)
    stream = torch.cuda.current_stream().cuda_stream
    rc = chol.lib().chol_solve_noalloc(n, nrhs, dL.data_ptr(), dL.stride(1), out.data_ptr(), out.stride(1),
                                       ctypes.c_void_p(stream))
    torch.cuda.synchronize()
    return rc, out.cpu().numpy(), ref.cpu().numpy()


def test_noalloc_solve_matches_allocating_solve_twice():
    import paper_2606_11937_gb300 as chol
    for n, nrhs, seed in ((1500, 7, 31), (777, 33, 32)):
        rc, X, Xref = _solve_pair(n, nrhs, seed)
        assert rc == chol.CHOL_OK, chol.chol_last_error()
        assert np.max(np.abs(X - Xref)) <= REL_TOL * np.max(np.abs(Xref))


def test_noalloc_solve_refuses_oversized_scratch():
    import paper_2606_11937_gb300 as chol
    # 2 * ceil(n/64) * ceil(nrhs/16) * 4 bytes > 4 MiB: refused before any device work
    rc = chol.lib().chol_solve_noalloc(1 << 20, 1024, ctypes.c_void_p(16), 1 << 20, ctypes.c_void_p(16), 1 << 20,
                                       None)
    assert rc == chol.CHOL_ERR_ARG
    assert "scratch" in chol.chol_last_error()
