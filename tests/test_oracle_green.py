"""Pins for the Green's function G of Eq. 1c (a = 1, (1-nu^2)/E = 1)."""
import math

import numpy as np
import pytest
from scipy import integrate

import oracle


def cell_integral_over_pi(dx, dy):
    """(1/pi) * integral over the unit cell centred at (dx, dy) of dA/|r| (Eq. 1c)."""
    f = lambda y, x: 1.0 / math.hypot(x, y)
    val, err = integrate.dblquad(f, dx - 0.5, dx + 0.5, dy - 0.5, dy + 0.5,
                                 epsabs=1e-13, epsrel=1e-12)
    return val / math.pi


def test_self_term_closed_form(golden):
    g = golden("green_self_term.txt")
    assert oracle.G(0, 0) == pytest.approx(g["G0"], rel=1e-15)


def test_self_term_by_quadrature():
    # polar form of the singular cell integral: int_0^{2pi} R(th) dth
    R = lambda th: 0.5 / max(abs(math.cos(th)), abs(math.sin(th)))
    pts = [k * math.pi / 4 for k in range(1, 8)]
    val, _ = integrate.quad(R, 0.0, 2 * math.pi, points=pts, epsabs=1e-14, epsrel=1e-13)
    assert oracle.G(0, 0) == pytest.approx(val / math.pi, rel=1e-12)


@pytest.mark.parametrize("d", [(5, 0), (3, 4), (10, 7), (0, 12), (20, 21)])
def test_far_field_against_cell_integral(d, golden):
    """The point form differs from the cell integral of Eq. 1c by 1/(24 r^2) + O(r^-4)."""
    coef = golden("green_self_term.txt")["FAR_FIELD_COEF"]
    dx, dy = d
    r = math.hypot(dx, dy)
    ratio = cell_integral_over_pi(dx, dy) / oracle.G(dx, dy)
    assert abs(ratio - 1.0 - coef / r**2) <= 0.05 / r**4


def test_symmetries():
    for dx in range(-6, 7):
        for dy in range(-6, 7):
            g = oracle.G(dx, dy)
            assert g == oracle.G(-dx, dy) == oracle.G(dx, -dy) == oracle.G(dy, dx)
            assert g > 0


def test_kernel_table_wrap():
    L = 5
    M = oracle.padded_side(L)
    assert M == 16
    k = oracle.kernel_table(L)
    for jy in range(M):
        for jx in range(M):
            dx = jx if jx < L else (jx - M if jx > M - L else None)
            dy = jy if jy < L else (jy - M if jy > M - L else None)
            want = 0.0 if dx is None or dy is None else oracle.G(dx, dy)
            assert k[jy, jx] == want


def test_padded_side():
    assert [oracle.padded_side(L) for L in (1, 2, 3, 4, 5, 8, 1024)] == [2, 4, 8, 8, 16, 16, 2048]


# ------------------------------------------- Eq. 1c's cell integral (all r) --

def test_cell_self_term(golden):
    assert oracle.G_cell(0, 0) == pytest.approx(golden("green_self_term.txt")["G0"], rel=1e-15)


@pytest.mark.parametrize("d", [(1, 0), (1, 1), (2, 1), (0, 3), (4, 4), (7, 2), (12, 5)])
def test_cell_against_adaptive_quadrature(d):
    dx, dy = d
    assert oracle.G_cell(dx, dy) == pytest.approx(cell_integral_over_pi(dx, dy), rel=1e-11)


@pytest.mark.parametrize("k", [1, 2, 3, 5])
def test_cell_additivity_over_blocks(k, golden):
    """The cells of a centred (2k+1) x (2k+1) block tile a square of side
    2k+1, and the integral of 1/r over a centred square grows linearly with
    its side, so the block sum is (2k+1) G(0) exactly."""
    tot = sum(oracle.G_cell(a, b) for a in range(-k, k + 1) for b in range(-k, k + 1))
    assert tot == pytest.approx((2 * k + 1) * golden("green_self_term.txt")["G0"], rel=1e-14)


@pytest.mark.parametrize("d", [(10, 10), (30, 0), (100, 37), (700, 700), (2000, 5), (4095, 4095)])
def test_cell_far_field(d, golden):
    """Cell average of 1/r = point value x (1 + 1/(24 r^2) + c4(theta)/r^4 +
    O(r^-6)).  The fourth-order Taylor term over the cell, (1/24) <(u.grad)^4>
    1/r with <u_x^4> = 1/80 and <u_x^2 u_y^2> = 1/144, is c4 = (7/384)
    sin^2(2 theta) - 7/1920 relative to 1/r.  At large r this also checks that
    the corner sum kept full precision despite its terms of size r ln r."""
    coef = golden("green_self_term.txt")["FAR_FIELD_COEF"]
    dx, dy = d
    r = math.hypot(dx, dy)
    th = math.atan2(dy, dx)
    c4 = 7.0 / 384.0 * math.sin(2 * th) ** 2 - 7.0 / 1920.0
    ratio = oracle.G_cell(dx, dy) / oracle.G(dx, dy)
    assert abs(ratio - 1.0 - coef / r**2 - c4 / r**4) <= 0.01 / r**6 + 4e-16


def test_cell_symmetries():
    for dx in range(-5, 6):
        for dy in range(-5, 6):
            g = oracle.G_cell(dx, dy)
            assert g == oracle.G_cell(-dx, dy) == oracle.G_cell(dx, -dy) == oracle.G_cell(dy, dx)


def test_cell_kernel_selection_reaches_every_oracle_path():
    """Inside use_green(GREEN_CELL) the table, the direct sum, the dense
    operator and the FFT route all use the cell integral, and the FFT route
    still equals the direct sum."""
    L = 6
    rng = np.random.default_rng(3)
    x = rng.standard_normal(L * L)
    with oracle.use_green(oracle.GREEN_CELL, L):
        k = oracle.kernel_table(L)
        yd = oracle.conv_direct(L, x)
        yf = oracle.conv_fft(L, x)
        A = oracle.dense_operator(L)
    assert k[0, 1] == oracle.G_cell(1, 0) and k[2, 3] == oracle.G_cell(3, 2)
    assert np.allclose(yf, yd, rtol=0, atol=1e-13 * np.abs(yd).max())
    assert np.allclose(A @ x, yd, rtol=0, atol=1e-13 * np.abs(yd).max())
    # outside, the point form again
    assert oracle.kernel_table(L)[0, 1] == oracle.G(1, 0)
