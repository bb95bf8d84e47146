"""chol_solve_noalloc: the FP64 solve for callers that cannot allocate device
memory (an application whose memory manager has reserved the GPU, or a
latency-critical loop that must not pay the synchronization cudaMalloc /
cudaFree can cause).  It keeps its scratch in a fixed 4 MiB device array.

Its results are checked against the oracle's forward/backward substitution
(entry by entry) and by the backward error recomputed from A, X and B, and
against chol_solve_ex (the allocating entry point), on two different calls in
a row (the second must not see the first's leftovers in the shared array);
both slice widths of the sweep are covered (at most four right-hand sides use
4-column slices, more use 16-column slices).  Around one call the device's
free memory and the stream-ordered pool's used and reserved bytes must stay
unchanged, and sizes beyond the fixed scratch must be refused with a clear
error.  This file runs last so that a failure here leaves every other test
already run; it passes alone in a fresh process as well.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

REL_TOL = 1e-12  # relative to max |X|, as in the FP64 solve tests
BERR_TOL = 1e-14  # normwise backward error of a solve with an exact-to-rounding factor


def _device_memory():
    import paper_2606_11937_gb300 as chol
    f, u, r = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_uint64()
    rc = chol.lib().chol_test_device_memory(ctypes.byref(f), ctypes.byref(u), ctypes.byref(r))
    assert rc == chol.CHOL_OK, chol.chol_last_error()
    return f.value, u.value, r.value


def _solve_pair(n, nrhs, seed):
    import torch

    import oracle
    import paper_2606_11937_gb300 as chol
    import seeded_inputs as si
    A = si.gram_plus_identity(n, seed)
    L, info = oracle.potrf_unblocked(A)
    assert info == 0
    L = np.tril(L)
    dL = chol.colmajor(L)
    B = si.rhs(n, nrhs, seed=seed + 1)
    ref = chol.colmajor(B)
    chol.chol_solve_ex(dL, ref)
    out = chol.colmajor(B)
    stream = torch.cuda.current_stream().cuda_stream
    torch.cuda.synchronize()
    before = _device_memory()
    rc = chol.lib().chol_solve_noalloc(n, nrhs, dL.data_ptr(), dL.stride(1), out.data_ptr(), out.stride(1),
                                       ctypes.c_void_p(stream))
    after = _device_memory()
    torch.cuda.synchronize()
    return rc, A, L, B, out.cpu().numpy(), ref.cpu().numpy(), before, after


@pytest.mark.parametrize("cases", [((1500, 7, 31), (777, 33, 32)), ((1024, 3, 41), (1500, 1, 42))],
                         ids=["16-column slices", "4-column slices"])
def test_noalloc_solve_matches_oracle_twice(cases):
    import oracle
    import paper_2606_11937_gb300 as chol
    for n, nrhs, seed in cases:
        rc, A, L, B, X, Xref, before, after = _solve_pair(n, nrhs, seed)
        assert rc == chol.CHOL_OK, chol.chol_last_error()
        # the oracle's forward then backward substitution with the same factor
        Xo = oracle.potrs(L, B)
        assert np.max(np.abs(X - Xo)) <= REL_TOL * np.max(np.abs(Xo))
        assert oracle.backward_error(A, X, B) <= BERR_TOL
        # and the allocating entry point
        assert np.max(np.abs(X - Xref)) <= REL_TOL * np.max(np.abs(Xref))
        # nothing was allocated: free device memory and the pool are unchanged
        assert after == before, (before, after)


def test_noalloc_solve_refuses_oversized_scratch():
    import paper_2606_11937_gb300 as chol
    # 2 * ceil(n/64) * ceil(nrhs/16) * 4 bytes > 4 MiB: refused before any device work
    rc = chol.lib().chol_solve_noalloc(1 << 20, 1024, ctypes.c_void_p(16), 1 << 20, ctypes.c_void_p(16), 1 << 20,
                                       None)
    assert rc == chol.CHOL_ERR_ARG
    assert "scratch" in chol.chol_last_error()
