"""Z2 noise of the Hutchinson estimator (Sect. 1-2), counter-based.

Reading (the paper only says "Z2 noise"): real entries x_i in {+1, -1}, each
with probability 1/2, i.i.d., so E[x_i] = 0 and E[x_i x_j] = delta_ij.  Entry i
of sample j of the term whose fine level is ``term`` is

    h = sm(sm(sm(seed XOR term) XOR j) XOR i),   x_i = +1 if h is even else -1,

with sm(z) = mix(z + 0x9E3779B97F4A7C15) the splitmix64 step of Steele, Lea
& Flood (OOPSLA 2014): mix(z) = z ^ (z >> 31) after
z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9, z = (z ^ (z >> 27)) * 0x94D049BB133111EB,
all modulo 2^64.  This is an independent implementation of the generator; the
CUDA path has its own.

Pinned in tests/test_oracle_noise.py by the properties the estimator needs
(zero mean, unit second moment, uncorrelated entries and samples).
"""
from __future__ import annotations

import numpy as np

_MASK = (1 << 64) - 1
_G = np.uint64(0x9E3779B97F4A7C15)
_C1 = np.uint64(0xBF58476D1CE4E5B9)
_C2 = np.uint64(0x94D049BB133111EB)


def _sm(z: np.ndarray) -> np.ndarray:
    with np.errstate(over="ignore"):
        z = z + _G
        z = (z ^ (z >> np.uint64(30))) * _C1
        z = (z ^ (z >> np.uint64(27))) * _C2
        return z ^ (z >> np.uint64(31))


def z2_noise(seed: int, term: int, first_sample: int, nsamples: int, n: int) -> np.ndarray:
    """Real +-1 array of shape (nsamples, n)."""
    kt = _sm(np.uint64((seed ^ term) & _MASK))
    j = np.arange(first_sample, first_sample + nsamples, dtype=np.uint64)
    ks = _sm(kt ^ j)                                   # (nsamples,)
    i = np.arange(n, dtype=np.uint64)
    h = _sm(ks[:, None] ^ i[None, :])
    return 1.0 - 2.0 * (h & np.uint64(1)).astype(np.float64)
