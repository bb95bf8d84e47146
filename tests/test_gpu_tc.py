"""The tcgen05 tile update alone (TMA-staged operands, TMEM accumulator)
against the same update computed in binary64 from the exact operand values.

Tolerance, from the arithmetic: the products of two bf16 / fp16 / tf32
operands are exact in binary32; each of the <= nb accumulation steps in
binary32 adds at most one unit of 2^-23 relative to the running sum (which
is bounded by sum_k |a_k b_k|), and the final subtraction from C one more
rounding: |err| <= (2 nb + 8) 2^-24 s sum_k |a_k||b_k| + 2^-23 |C|.
"""
import numpy as np
import pytest

import oracle
import seeded_inputs as si
from lowprec import bf16_bits, bf16_value, tf32_round

pytestmark = pytest.mark.gpu


def operands(prec, nb, seed, eA, eB):
    r = si.rng(seed)
    A = r.standard_normal((nb, nb)).astype(np.float32)
    B = r.standard_normal((nb, nb)).astype(np.float32)
    if prec == "bf16":
        a, b = bf16_bits(A * np.float32(2.0 ** eA)), bf16_bits(B * np.float32(2.0 ** eB))
        ops = np.concatenate([a, b]).view(np.uint8)
        pairs = [(bf16_value(a).astype(np.float64), bf16_value(b).astype(np.float64))]
    elif prec == "fp16":
        a, b = (A * np.float32(2.0 ** eA)).astype(np.float16), (B * np.float32(2.0 ** eB)).astype(np.float16)
        ops = np.concatenate([a, b]).view(np.uint8)
        pairs = [(a.astype(np.float64), b.astype(np.float64))]
    elif prec == "tf32":
        a, b = tf32_round(A), tf32_round(B)
        ops = np.concatenate([a, b]).view(np.uint8)
        pairs = [(a.astype(np.float64), b.astype(np.float64))]
    else:  # fp32 = hi*hi + hi*lo + lo*hi
        ah, bh = tf32_round(A), tf32_round(B)
        al, bl = tf32_round(A - ah), tf32_round(B - bh)
        ops = np.concatenate([ah, bh, al, bl]).view(np.uint8)
        f = lambda x: x.astype(np.float64)
        pairs = [(f(ah), f(bh)), (f(ah), f(bl)), (f(al), f(bh))]
    return np.ascontiguousarray(ops), pairs


@pytest.mark.parametrize("prec", ["bf16", "fp16", "tf32", "fp32"])
@pytest.mark.parametrize("nb", [128, 256, 384, 512])
@pytest.mark.parametrize("lower", [False, True])
def test_tc_tile_update(prec, nb, lower):
    import torch

    import paper_2606_11937_gb300 as chol
    eA, eB = (3, -2) if prec in ("bf16", "fp16") else (0, 0)
    ops, pairs = operands(prec, nb, 100 + nb, eA, eB)
    C = si.rng(7).standard_normal((2, nb, nb)).astype(np.float32)
    dops = torch.from_numpy(ops).cuda()
    dC = torch.from_numpy(C.copy()).cuda()
    rc = chol.chol_test_tc_update(prec, nb, dops, eA, eB, dC, lower)
    assert rc == 0, chol.chol_last_error()
    got = dC.cpu().numpy().astype(np.float64)
    s = 2.0 ** (-eA - eB)
    want = C.astype(np.float64)
    absum = np.zeros((nb, nb))
    for a, b in pairs:
        want = np.stack([oracle.tile_op("gemm", a * s, b, want[r]) for r in range(2)])
        absum += np.abs(a) @ np.abs(b).T * s
    tol = [(2 * nb + 8) * 2.0 ** -24 * absum + 2.0 ** -23 * np.abs(C[r].astype(np.float64)) for r in range(2)]
    mask = np.ones((nb, nb), dtype=bool)
    if lower:
        # sub-tiles (128 rows by 256 columns where 256 divides nb, else 128)
        # strictly above the diagonal are skipped
        SR, NN = 128, (256 if nb % 256 == 0 else 128)
        for ri in range(nb // SR):
            for ci in range(nb // NN):
                if ci * NN >= (ri + 1) * SR:
                    mask[ri * SR:(ri + 1) * SR, ci * NN:(ci + 1) * NN] = False
    for r in range(2):
        err = np.abs(got[r] - want[r])
        assert np.all(err[mask] <= tol[r][mask]), (prec, nb, float(np.max(err[mask] / tol[r][mask])))
        assert np.array_equal(got[r][~mask], C[r].astype(np.float64)[~mask])
