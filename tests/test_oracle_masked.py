"""Pin for the quasi-static removal loop: brute force with dense re-solves."""
import numpy as np
import pytest

import fc_inputs
import oracle


@pytest.mark.parametrize("L,steps", [(3, 8), (5, 12), (6, 20)])
def test_masked_loop_brute_force(L, steps):
    p = fc_inputs.problem(L, seed=11, b_kind="ones", with_t=True)
    out = oracle.masked_loop(L, p["s"], p["b"], p["t"], steps, rtol=1e-13)
    A_full = oracle.dense_operator(L, p["s"])
    mask = np.ones(L * L, bool)
    for st in range(steps):
        act = np.flatnonzero(mask)
        x = np.zeros(L * L)
        x[act] = np.linalg.solve(A_full[np.ix_(act, act)], p["b"][act])
        ratio = np.where(mask, np.abs(x) / p["t"], -np.inf)
        k = int(np.argmax(ratio))  # numpy argmax returns the first maximum
        # the pick must be unique enough that rounding cannot flip it
        top2 = np.sort(ratio[mask])[-2:] if act.size > 1 else None
        if top2 is not None and top2[1] - top2[0] < 1e-9 * top2[1]:
            pytest.skip("near tie")
        assert out["picks"][st] == k
        assert out["ratios"][st] == pytest.approx(ratio[k], rel=1e-10)
        mask[k] = False
    assert np.array_equal(out["mask"].astype(bool), mask)


def test_argmax_ties_to_lowest_index():
    x = np.array([1.0, -2.0, 2.0, 0.5])
    t = np.ones(4)
    k, r = oracle.argmax_ratio(x, t)
    assert k == 1 and r == 2.0
    k, _ = oracle.argmax_ratio(x, t, mask=np.array([1, 0, 1, 1], np.uint8))
    assert k == 2


@pytest.mark.parametrize("L", [1, 2, 5, 9])
def test_front_brute_force(L):
    """Front readout against a direct scan of each column."""
    rng = np.random.default_rng(L)
    for dens in (0.0, 0.3, 0.7, 1.0):
        m = (rng.random(L * L) >= dens).astype(np.uint8)
        fi, de = oracle.front(L, m)
        g = m.reshape(L, L)
        for ix in range(L):
            col = g[:, ix]
            intact = np.flatnonzero(col == 1)
            broken = np.flatnonzero(col == 0)
            assert fi[ix] == (intact[0] if intact.size else L)
            assert de[ix] == (broken[-1] + 1 if broken.size else 0)


def test_threshold_gradient_inputs():
    """t = xi + g (iy + 1/2)/L with the same xi as the gradient-free draw."""
    L, g = 8, 3.0
    a = fc_inputs.problem(L, seed=4, with_t=True)
    b = fc_inputs.problem(L, seed=4, with_t=True, t_gradient=g)
    iy = np.arange(L * L) // L
    assert np.allclose(b["t"] - a["t"], g * (iy + 0.5) / L, rtol=0, atol=1e-15)
    assert np.array_equal(a["s"], b["s"])
