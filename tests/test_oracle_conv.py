"""Pins for the coupling operator C (Eq. 1b with the G of Eq. 1c)."""
import numpy as np
import pytest

import fc_inputs
import oracle


@pytest.mark.parametrize("L", [1, 2, 3, 5, 8, 16, 33, 48])
def test_fft_route_matches_direct_sum(L):
    """Two independent algorithms: the padded-FFT route of Listing 4 vs the sum of Eq. 1b."""
    rng = np.random.default_rng(L)
    x = rng.standard_normal(L * L)
    yd = oracle.conv_direct(L, x)
    yf = oracle.conv_fft(L, x)
    assert np.max(np.abs(yf - yd)) <= 1e-13 * max(1.0, np.max(np.abs(yd)))


@pytest.mark.parametrize("pos", [(0, 0), (3, 5), (6, 6)])
def test_delta_response(pos):
    L = 7
    y0, x0 = pos
    x = np.zeros(L * L)
    x[y0 * L + x0] = 1.0
    y = oracle.conv_direct(L, x).reshape(L, L)
    for iy in range(L):
        for ix in range(L):
            assert y[iy, ix] == oracle.G(ix - x0, iy - y0)


def test_translation_invariance_inside_grid():
    L = 12
    rng = np.random.default_rng(1)
    x = np.zeros((L, L))
    x[2:5, 3:6] = rng.standard_normal((3, 3))
    xs = np.roll(np.roll(x, 2, axis=0), 3, axis=1)  # stays inside the grid
    y = oracle.conv_fft(L, x.ravel()).reshape(L, L)
    ys = oracle.conv_fft(L, xs.ravel()).reshape(L, L)
    assert np.allclose(ys[2:, 3:], y[:-2, :-3], atol=1e-13)


def test_symmetry_of_C():
    L = 16
    rng = np.random.default_rng(2)
    x, z = rng.standard_normal(L * L), rng.standard_normal(L * L)
    a = z @ oracle.conv_fft(L, x)
    b = x @ oracle.conv_fft(L, z)
    assert abs(a - b) <= 1e-12 * abs(a)


@pytest.mark.parametrize("L,lo,hi", [(8, 0.60, 0.63), (16, 0.60, 0.62)])
def test_positive_definite(L, lo, hi):
    """Section 3: translation invariance makes the operator symmetric positive definite."""
    A = oracle.dense_operator(L)
    assert np.array_equal(A, A.T)
    lam = np.linalg.eigvalsh(A)
    assert lo < lam[0] < hi
    assert 0.9 < lam[-1] / L < 1.0


def test_dense_operator_matches_direct():
    L = 6
    p = fc_inputs.problem(L, seed=0)
    rng = np.random.default_rng(5)
    x = rng.standard_normal(L * L)
    A = oracle.dense_operator(L, p["s"])
    assert np.allclose(A @ x, oracle.conv_direct(L, x) + p["s"] * x, rtol=1e-14, atol=1e-13)


@pytest.mark.parametrize("L", [1, 3, 8, 32])
def test_spectrum_real_positive(L):
    """An even real kernel has a real spectrum; DC term = sum of the table / M^2."""
    S = oracle.spectrum(L)
    M = oracle.padded_side(L)
    assert np.max(np.abs(S.imag)) <= 1e-14 * np.max(np.abs(S.real))
    k = oracle.kernel_table(L)
    assert S[0, 0].real == pytest.approx(k.sum() / M**2, rel=1e-13)
    assert np.min(S.real) > 0.0
    # even in each frequency coordinate separately
    R = S.real
    idx = (-np.arange(M)) % M
    assert np.allclose(R, R[idx, :], atol=1e-15) and np.allclose(R, R[:, idx], atol=1e-15)
    assert np.allclose(R, R.T, atol=1e-15)
