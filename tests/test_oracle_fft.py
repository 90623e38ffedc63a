"""Pins for the oracle's radix-2 FFT: brute-force DFT, Parseval, round trip."""
import numpy as np
import pytest

import oracle


def naive_dft(x, sign):
    n = x.size
    j = np.arange(n)
    W = np.exp(sign * 2j * np.pi * np.outer(j, j) / n)
    return W @ x


@pytest.mark.parametrize("n", [1, 2, 4, 8, 16, 32, 64])
@pytest.mark.parametrize("sign", [-1, 1])
def test_fft_matches_naive_dft(n, sign):
    rng = np.random.default_rng(n + 7 * (sign + 1))
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    got = oracle.fft(x, sign)
    ref = naive_dft(x, sign)
    assert np.max(np.abs(got - ref)) <= 1e-13 * max(1.0, np.max(np.abs(ref)))


@pytest.mark.parametrize("M", [2, 4, 8, 16])
def test_fft2_matches_naive_2d_dft(M):
    rng = np.random.default_rng(M)
    x = rng.standard_normal((M, M)) + 1j * rng.standard_normal((M, M))
    j = np.arange(M)
    W = np.exp(-2j * np.pi * np.outer(j, j) / M)
    ref = W @ x @ W.T
    got = oracle.fft2(x, -1)
    assert np.max(np.abs(got - ref)) <= 1e-13 * np.max(np.abs(ref))


def test_parseval_and_round_trip():
    rng = np.random.default_rng(3)
    n = 1024
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    X = oracle.fft(x, -1)
    assert abs(np.sum(np.abs(X) ** 2) / n - np.sum(np.abs(x) ** 2)) <= 1e-12 * np.sum(np.abs(x) ** 2)
    back = oracle.fft(X, +1) / n
    assert np.max(np.abs(back - x)) <= 1e-13


def test_delta_and_constant():
    n = 32
    d = np.zeros(n, complex)
    d[0] = 1
    assert np.allclose(oracle.fft(d), np.ones(n), atol=1e-15)
    # a shifted delta gives a pure phase ramp exp(-2 pi i k m / n)
    d = np.zeros(n, complex)
    d[5] = 1
    k = np.arange(n)
    assert np.allclose(oracle.fft(d), np.exp(-2j * np.pi * 5 * k / n), atol=1e-14)


def test_fft_rejects_non_power_of_two():
    with pytest.raises(RuntimeError):
        oracle.fft(np.ones(6))
