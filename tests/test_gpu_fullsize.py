"""Parity at the benchmark's full size (n = 32768), in the launch configuration
bench.py times (FP64 on the tensor cores, dataflow schedule with priorities,
tiles of order 128), through properties that hold at any size:

* exact-integer pin: A = L0 L0^T with a banded integer L0 (diagonal in
  {1, 2, 4}, entries in {-2 .. 2}): every intermediate is a small integer, so
  the computed factor must equal L0 bit for bit over all n^2 / 2 entries;
* the bench's own input (SE covariance, nugget 1e-2, seed 1): randomized
  residual ||A X - L (L^T X)||_F / ||A X||_F <= 1e-14 sqrt(n) with Gaussian
  probes (the products in binary64 on the device);
* the mixed-precision configuration (FP32 factor, 16 right-hand sides,
  refinement to 1e-14): the normwise backward error recomputed from A, X and
  B independently of the library's own estimate.
"""
import math

import pytest

import seeded_inputs as si

pytestmark = pytest.mark.gpu

N = 32768


def _factor_tc(dA):
    import torch

    import paper_2606_11937_gb300 as chol
    rc, info, st = chol.chol_factor_ex(
        dA, chol.opts(schedule="dataflow", nb=128, flags=chol.CHOL_FLAG_FP64_TC | chol.CHOL_FLAG_PRIORITY),
        raise_on_error=False)
    torch.cuda.synchronize()
    return rc, info, st


def test_fullsize_exact_integer_factor():
    import torch
    A, L = si.exact_integer_band_torch(N, band=64, seed=41)
    dA = A.T  # column-major view of the symmetric A
    rc, info, st = _factor_tc(dA)
    assert rc == 0 and info == 0
    want = L.T  # element (i, j) of the column-major L0
    del A
    # compare the lower triangles in column blocks (bounded temporaries)
    for c0 in range(0, N, 4096):
        c1 = c0 + 4096
        got = torch.tril(dA[:, c0:c1], diagonal=-c0)
        ref = torch.tril(want[:, c0:c1], diagonal=-c0)
        assert torch.equal(got, ref), c0


def test_fullsize_bench_input_residual():
    import torch
    A = si.se_covariance_torch(N, seed=1, lengthscale=0.1, nugget=1e-2).T
    L = A.clone()
    rc, info, st = _factor_tc(L)
    assert rc == 0 and info == 0
    L = torch.tril(L)
    g = torch.Generator(device="cuda")
    g.manual_seed(99)
    X = torch.randn((N, 4), dtype=torch.float64, device="cuda", generator=g)
    AX = torch.tril(A) @ X + torch.tril(A, -1).T @ X  # A from its lower triangle
    R = AX - L @ (L.T @ X)
    rel = float(torch.linalg.norm(R) / torch.linalg.norm(AX))
    print(f"n={N}: probe residual {rel:.3e} (bound {1e-14 * math.sqrt(N):.3e})")
    assert rel <= 1e-14 * math.sqrt(N)


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
