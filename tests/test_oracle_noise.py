"""Pins of the oracle's Z2 noise: the properties the Hutchinson estimator needs (Sect. 1)."""
import numpy as np

from oracle import noise


def test_values_and_moments():
    X = noise.z2_noise(12345, 1, 0, 200, 5000)
    assert set(np.unique(X)) == {-1.0, 1.0}
    m = X.size
    assert abs(X.mean()) < 5 / np.sqrt(m)                 # E[x_i] = 0
    c1 = (X[:, 1:] * X[:, :-1]).mean()                    # E[x_i x_{i+1}] = 0
    c2 = (X[1:, :] * X[:-1, :]).mean()                    # samples uncorrelated
    assert abs(c1) < 5 / np.sqrt(m) and abs(c2) < 5 / np.sqrt(m)


def test_counter_based():
    a = noise.z2_noise(7, 2, 0, 8, 100)
    b = noise.z2_noise(7, 2, 5, 3, 100)
    assert np.array_equal(a[5:8], b)
    assert not np.array_equal(noise.z2_noise(7, 3, 0, 8, 100), a)
    assert not np.array_equal(noise.z2_noise(8, 2, 0, 8, 100), a)


def test_known_bits():
    # A few values of the definition h = sm(sm(sm(seed^term)^j)^i), low bit of h,
    # evaluated with Python integers as a second, scalar implementation.
    M = (1 << 64) - 1

    def sm(z):
        z = (z + 0x9E3779B97F4A7C15) & M
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M
        return z ^ (z >> 31)

    seed, term = 0xDEADBEEF, 3
    X = noise.z2_noise(seed, term, 10, 2, 40)
    for j in (10, 11):
        for i in (0, 1, 17, 39):
            h = sm(sm(sm(seed ^ term) ^ j) ^ i)
            assert X[j - 10, i] == (1.0 if h % 2 == 0 else -1.0)
