"""Pins of oracle.rounding.bf16 (the BF16 factors of the tensor-core deflation)."""
import numpy as np
import pytest

from oracle import rounding


def test_ties_round_to_even():
    u = 2.0 ** -7                        # spacing of BF16 values in [1, 2)
    x = np.array([1.0, 1 + u / 2, 1 + u, 1 + 1.5 * u, 1 + 0.49 * u, 1 + 0.51 * u, -1 - u / 2, 3 + 3 * u])
    want = np.array([1.0, 1.0, 1 + u, 1 + 2 * u, 1.0, 1 + u, -1.0, 3 + 4 * u])
    assert np.array_equal(rounding.bf16(x), want)


def test_two_step_rounding():
    # just above a BF16 tie: the FP64 -> FP32 step lands exactly on the tie, which
    # then goes to even; a direct FP64 -> BF16 rounding would go up
    u = 2.0 ** -7
    x = np.array([1 + u / 2 + 2.0 ** -40])
    assert rounding.bf16(x)[0] == 1.0


def test_complex_parts_and_magnitudes():
    rng = np.random.default_rng(3)
    z = (rng.standard_normal(1000) + 1j * rng.standard_normal(1000)) * 10.0 ** rng.integers(-20, 20, 1000)
    r = rounding.bf16(z)
    assert np.array_equal(r.real, rounding.bf16(z.real)) and np.array_equal(r.imag, rounding.bf16(z.imag))
    # relative error of each part at most 2^-8 (plus the FP32 step)
    for a, b in ((z.real, r.real), (z.imag, r.imag)):
        assert np.all(np.abs(a - b) <= (2.0 ** -8 + 2.0 ** -24) * np.abs(a))
        # idempotent: BF16 values are representable
        assert np.array_equal(rounding.bf16(b), b)


def test_against_torch_conversion():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(7)
    x = rng.standard_normal(100000) * 10.0 ** rng.integers(-10, 10, 100000)
    # FP32 inputs, including exact ties
    f = np.concatenate([x.astype(np.float32), (1 + np.arange(1, 200) * 2.0 ** -8).astype(np.float32)])
    ref = torch.from_numpy(f).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(rounding.bf16(f.astype(np.float64)), ref)
