"""Parity at the benchmark's full sizes (n = 32768 and n = 65536, the order
bench.py times by default), in the launch configuration bench.py times (FP64
on the tensor cores, dataflow schedule with priorities, tiles of order 128),
through properties that hold at any size:

* exact-integer pin: A = L0 L0^T with a banded integer L0 (diagonal in
  {1, 2, 4}, entries in {-2 .. 2}): every intermediate is a small integer, so
  the computed factor must equal L0 bit for bit over all n^2 / 2 entries;
* the bench's own input (SE covariance, nugget 1e-2, seed 1): randomized
  residual ||A X - L (L^T X)||_F / ||A X||_F <= 1e-14 sqrt(n) with Gaussian
  probes (the products in binary64 on the device);
* the host-buffer entry point at n = 65536 (the first order whose n^2
  elements exceed 2^31, so every 64-bit element offset of the copies, the
  repack and the unpack is exercised): the exact-integer factor comes back
  into pinned host memory bit for bit;
* the mixed-precision configuration (FP32 factor, 16 right-hand sides,
  refinement to 1e-14): the normwise backward error recomputed from A, X and
  B independently of the library's own estimate.
"""
import math

import pytest

import seeded_inputs as si

pytestmark = pytest.mark.gpu

N = 32768
SIZES = (32768, 65536)
BLK = 4096  # column block of the comparisons (bounded temporaries)


def _bench_opts():
    import paper_2606_11937_gb300 as chol
    return chol.opts(schedule="dataflow", nb=128, flags=chol.CHOL_FLAG_FP64_TC | chol.CHOL_FLAG_PRIORITY)


def _factor_tc(dA):
    import torch

    import paper_2606_11937_gb300 as chol
    rc, info, st = chol.chol_factor_ex(dA, _bench_opts(), raise_on_error=False)
    torch.cuda.synchronize()
    return rc, info, st


def _assert_lower_equal(got, want, n):
    """Lower triangles of two column-major (n, n) tensors equal bit for bit;
    `got` may live in host memory (its blocks are copied to the device)."""
    import torch
    for c0 in range(0, n, BLK):
        c1 = min(n, c0 + BLK)
        g = got[:, c0:c1].to("cuda")
        assert torch.equal(torch.tril(g, diagonal=-c0), torch.tril(want[:, c0:c1], diagonal=-c0)), c0


@pytest.mark.parametrize("n", SIZES)
def test_fullsize_exact_integer_factor(n):
    A, L = si.exact_integer_band_torch(n, band=64, seed=41)
    dA = A.T  # column-major view of the symmetric A
    rc, info, st = _factor_tc(dA)
    assert rc == 0 and info == 0
    _assert_lower_equal(dA, L.T, n)  # L.T: element (i, j) of the column-major L0


@pytest.mark.parametrize("n", SIZES)
def test_fullsize_bench_input_residual(n):
    import torch
    A = si.se_covariance_torch(n, seed=1, lengthscale=0.1, nugget=1e-2).T  # symmetric: both triangles
    L = A.clone()
    rc, info, st = _factor_tc(L)
    assert rc == 0 and info == 0
    g = torch.Generator(device="cuda")
    g.manual_seed(99)
    X = torch.randn((n, 4), dtype=torch.float64, device="cuda", generator=g)
    AX = A @ X
    del A
    # Y = L^T X and L Y by column blocks of the lower triangle of L
    Y = torch.empty_like(X)
    for c0 in range(0, n, BLK):
        c1 = min(n, c0 + BLK)
        Y[c0:c1] = torch.tril(L[:, c0:c1], diagonal=-c0).T @ X
    LY = torch.zeros_like(X)
    for c0 in range(0, n, BLK):
        c1 = min(n, c0 + BLK)
        LY += torch.tril(L[:, c0:c1], diagonal=-c0) @ Y[c0:c1]
    rel = float(torch.linalg.norm(AX - LY) / torch.linalg.norm(AX))
    print(f"n={n}: probe residual {rel:.3e} (bound {1e-14 * math.sqrt(n):.3e})")
    assert rel <= 1e-14 * math.sqrt(n)


def test_fullsize_host_buffer_roundtrip_65536():
    import torch

    import paper_2606_11937_gb300 as chol
    n = 65536
    A, L = si.exact_integer_band_torch(n, band=32, seed=43)
    h = torch.empty_strided((n, n), (1, n), dtype=torch.float64, pin_memory=True)
    h.copy_(A.T)
    del A
    torch.cuda.synchronize()
    info, st = chol.chol_factor_host(h, _bench_opts())
    assert info == 0
    _assert_lower_equal(h, L.T, n)


def test_fullsize_mixed_refinement_backward_error():
    import torch

    import paper_2606_11937_gb300 as chol
    A = si.se_covariance_torch(N, seed=1, lengthscale=0.1, nugget=1e-2).T
    g = torch.Generator(device="cuda")
    g.manual_seed(2)
    B = torch.randn((16, N), dtype=torch.float64, device="cuda", generator=g).T
    o = chol.opts(precision="fp32", schedule="dataflow", nb=128, flags=chol.CHOL_FLAG_PRIORITY, max_iter=50)
    rc, h = chol.chol_mixed_factor(A, o)
    assert rc == 0 and h.info == 0
    rc, X, iters, berr = h.solve(B)
    torch.cuda.synchronize()
    h.close()
    assert rc == 0 and berr <= 1e-14
    R = B - A @ X
    anorm = float(torch.max(torch.sum(torch.abs(A), dim=1)))
    be = torch.max(torch.abs(R), dim=0).values / (
        anorm * torch.max(torch.abs(X), dim=0).values + torch.max(torch.abs(B), dim=0).values)
    print(f"n={N}: {iters} refinement iterations, reported berr {berr:.2e}, recomputed {float(be.max()):.2e}")
    assert float(be.max()) <= 1e-14
