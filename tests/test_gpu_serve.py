"""Serving loop: continuous batching under a memory budget, resident factors,
and results that are the same alone and in the mix."""
import numpy as np
import pytest

import oracle
import seeded_inputs as si

pytestmark = pytest.mark.gpu


def _req(server, A, B, fid=0, prec="fp64", reuse=False):
    import torch

    import paper_2606_11937_gb300 as chol
    dB = chol.colmajor(B)
    dX = torch.empty_like(dB)
    dA = None if reuse else chol.colmajor(A)
    t = server.submit(dB, dX, A=dA, factor_id=fid, precision=prec)
    return t, (dA, dB, dX)


def test_served_results_same_alone_and_in_mix():
    """Alone (one slot: each factorization's persistent grid is the whole
    device) and in the mix (four slots: a quarter of the SMs each, requests
    overlapping): the same bits, and the oracle's backward error."""
    import torch

    import paper_2606_11937_gb300 as chol
    # 1500, 2048, 5000: FP64 requests on the tensor-core engine (order above 1024)
    sizes = [300, 1500, 64, 777, 2048, 129, 1024, 500, 5000]
    precs = ["fp64", "fp32", "fp64", "bf16", "fp64", "tf32", "fp64", "fp16", "fp64"]
    mats = [si.gram_plus_identity(n, 200 + i) if i % 2 == 0 else si.se_covariance(n, 300 + i, nugget=1e-1)
            for i, n in enumerate(sizes)]
    rhs = [si.rhs(n, 1 + (i * 7) % 32, seed=400 + i) for i, n in enumerate(sizes)]
    # alone: one slot, one request at a time
    alone = []
    srv = chol.Server(8 << 30, slots=1)
    for A, B, p in zip(mats, rhs, precs):
        t, keep = _req(srv, A, B, prec=p)
        r = srv.wait(t)
        assert r["status"] == 0, r
        alone.append(keep[2].cpu().numpy())
    srv.close()
    # in the mix: all at once on 4 slots
    srv = chol.Server(8 << 30, slots=4)
    ts = [_req(srv, A, B, prec=p) for A, B, p in zip(mats, rhs, precs)]
    outs = []
    for t, keep in ts:
        r = srv.wait(t)
        assert r["status"] == 0, r
        outs.append(keep[2].cpu().numpy())
    st = srv.stats()
    srv.close()
    assert st["completed"] == len(sizes) and st["p99_ms"] >= st["p50_ms"] > 0
    for A, B, X1, X2 in zip(mats, rhs, alone, outs):
        assert np.array_equal(X1, X2)
        assert oracle.backward_error(A, X2, B) <= 1e-14


def test_resident_factor_reuse_and_release():
    import paper_2606_11937_gb300 as chol
    n = 900
    A = si.gram_plus_identity(n, 5)
    B1, B2 = si.rhs(n, 3, seed=6), si.rhs(n, 5, seed=7)
    srv = chol.Server(4 << 30, slots=2)
    t1, k1 = _req(srv, A, B1, fid=42)
    t2, k2 = _req(srv, None, B2, fid=42, reuse=True)   # waits for factor 42
    r1, r2 = srv.wait(t1), srv.wait(t2)
    assert r1["status"] == 0 and r2["status"] == 0 and r2["reused_factor"] == 1
    assert oracle.backward_error(A, k2[2].cpu().numpy(), B2) <= 1e-14
    assert srv.stats()["resident_factors"] == 1
    assert srv.release(42) == 0
    t3, _ = _req(srv, None, B2, fid=42, reuse=True)
    assert srv.wait(t3)["status"] == chol.CHOL_ERR_HANDLE
    srv.close()


def test_budget_rejects_oversized_and_admits_the_rest():
    import paper_2606_11937_gb300 as chol
    srv = chol.Server(16 << 20, slots=2)   # 16 MiB
    big = si.gram_plus_identity(3000, 1)   # its FP64 tile store alone (about 37 MB) exceeds the budget
    small = si.gram_plus_identity(200, 2)
    tb, _ = _req(srv, big, si.rhs(3000, 1, seed=1))
    ts, ks = _req(srv, small, si.rhs(200, 1, seed=2))
    assert srv.wait(tb)["status"] == chol.CHOL_ERR_NOMEM
    rs = srv.wait(ts)
    assert rs["status"] == 0
    st = srv.stats()
    assert st["rejected"] == 1 and st["completed"] == 1
    srv.close()


def test_mixed_resident_factor_refines():
    import paper_2606_11937_gb300 as chol
    n = 1200
    A = si.gram_plus_identity(n, 9)
    srv = chol.Server(4 << 30, slots=2)
    dA = chol.colmajor(A)   # a resident mixed factor references A: keep it alive
    import torch
    B1 = chol.colmajor(si.rhs(n, 2, seed=1))
    X1 = torch.empty_like(B1)
    t1 = srv.submit(B1, X1, A=dA, factor_id=7, precision="fp32")
    B2 = chol.colmajor(si.rhs(n, 4, seed=2))
    X2 = torch.empty_like(B2)
    t2 = srv.submit(B2, X2, A=None, factor_id=7, precision="fp32", n=n)
    r1, r2 = srv.wait(t1), srv.wait(t2)
    assert r1["status"] == 0 and r2["status"] == 0 and r2["reused_factor"] == 1
    assert r2["berr"] <= 1e-14
    assert oracle.backward_error(A, X2.cpu().numpy(), si.rhs(n, 4, seed=2)) <= 1e-14
    srv.close()
