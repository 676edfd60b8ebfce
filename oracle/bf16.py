"""BF16 rounding and the hi/lo split of FP32 values -- TEST INFRASTRUCTURE ONLY.

bfloat16 keeps the top 16 bits of an IEEE-754 binary32 value.  Rounding to
nearest, ties to even, is done on the bit pattern: add 0x7FFF plus the lowest
kept bit, then truncate (NaN stays NaN).  The split used by the 3-pass tensor
core path writes x = hi + lo + r with hi = bf16(x), lo = bf16(x - hi), the
subtraction being exact in binary32.
"""
from __future__ import annotations

import numpy as np


def to_bf16_bits(x: np.ndarray) -> np.ndarray:
    x = np.ascontiguousarray(x, np.float32)
    u = x.view(np.uint32).astype(np.uint64)
    nan = np.isnan(x)
    bias = 0x7FFF + ((u >> 16) & 1)
    r = ((u + bias) >> 16).astype(np.uint16)
    r[nan] = 0x7FC0
    return r


def bf16_bits_to_f32(b: np.ndarray) -> np.ndarray:
    return (np.asarray(b, np.uint16).astype(np.uint32) << 16).view(np.float32)


def round_bf16(x: np.ndarray) -> np.ndarray:
    """float32 array of the bf16-rounded values."""
    return bf16_bits_to_f32(to_bf16_bits(x))


def split_bf16(x: np.ndarray):
    """(hi, lo) as float32 arrays holding bf16 values."""
    x = np.asarray(x, np.float32)
    hi = round_bf16(x)
    lo = round_bf16((x - hi).astype(np.float32))
    return hi, lo
