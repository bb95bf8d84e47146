"""Rounding of binary32 values to the tensor-core operand formats, written
from the IEEE / PTX definitions (used to build exact test operands on the
host; the library receives the rounded bits, so no rounding decision is
taken twice).

* bfloat16: the top 16 bits of binary32, round to nearest, ties to even;
* tf32 (cvt.rna): 10 explicit mantissa bits, round to nearest, ties away
  from zero, stored in a binary32 container with the low 13 bits zero;
* binary16: numpy's float16 conversion (round to nearest, ties to even).
"""
import numpy as np


def bf16_bits(x: np.ndarray) -> np.ndarray:
    b = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    r = (b + 0x7FFF + ((b >> 16) & 1)) >> 16
    return r.astype(np.uint16)


def bf16_value(bits: np.ndarray) -> np.ndarray:
    return (bits.astype(np.uint32) << 16).view(np.float32)


def tf32_round(x: np.ndarray) -> np.ndarray:
    b = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    r = ((b + 0x1000) & 0xFFFFE000).astype(np.uint32)
    return r.view(np.float32)
