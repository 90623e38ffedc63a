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
