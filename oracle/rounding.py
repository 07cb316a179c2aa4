"""Rounding to BF16, as the tensor-core deflation projections take their factors.

BF16 keeps 8 significant bits (1 implicit + 7 stored) and the exponent range of
FP32.  Reading (the paper fixes no reduced precision; this is how the factors of
the BF16 projections are defined here): an FP64 value is rounded to FP32 and the
FP32 value to BF16, both to nearest with ties to even.  Applied to the real and
imaginary parts separately.

Plain definition on the FP32 bit pattern: add 0x7FFF plus the lowest kept bit,
then clear the 16 low bits (round half to even).  Pinned in
tests/test_oracle_rounding.py against hand-computed ties (including a case where
the two-step rounding differs from a direct FP64 -> BF16 rounding) and against
PyTorch's FP32 -> BF16 conversion.
"""
from __future__ import annotations

import numpy as np


def bf16(x) -> np.ndarray:
    """x (real or complex, any shape) rounded to BF16, returned as float64/complex128."""
    x = np.asarray(x)
    if np.iscomplexobj(x):
        return bf16(x.real) + 1j * bf16(x.imag)
    f = np.ascontiguousarray(x, dtype=np.float64).astype(np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> np.uint64(16)) & np.uint64(1)
    u = (u + np.uint64(0x7FFF) + lsb) & np.uint64(0xFFFF0000)
    return u.astype(np.uint32).view(np.float32).astype(np.float64)
