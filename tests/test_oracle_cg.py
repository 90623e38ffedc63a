"""Pins for the oracle's CG (Listing 2) and dense Cholesky solve."""
import math

import numpy as np
import pytest

import fc_inputs
import oracle


def test_L1_closed_form(golden):
    g0 = golden("green_self_term.txt")["G0"]
    s, b = np.array([0.7]), np.array([2.5])
    x, rc, it, rel = oracle.cg(1, s, b, rtol=1e-14)
    assert rc == 0
    assert x[0] == pytest.approx(2.5 / (g0 + 0.7), rel=1e-14)


def test_cholesky_matches_lapack():
    rng = np.random.default_rng(0)
    for n in (1, 5, 40):
        B = rng.standard_normal((n, n))
        A = B @ B.T + n * np.eye(n)
        b = rng.standard_normal(n)
        assert np.allclose(oracle.cholesky_solve(A, b), np.linalg.solve(A, b), rtol=1e-12, atol=1e-13)


def test_cholesky_rejects_indefinite():
    with pytest.raises(RuntimeError):
        oracle.cholesky_solve(np.array([[1.0, 2.0], [2.0, 1.0]]), np.ones(2))


@pytest.mark.parametrize("L,b_kind", [(2, "ones"), (3, "normal"), (8, "ones"), (16, "normal")])
def test_cg_matches_dense_solves(L, b_kind):
    p = fc_inputs.problem(L, seed=L, b_kind=b_kind)
    A = oracle.dense_operator(L, p["s"])
    xc = oracle.cholesky_solve(A, p["b"])
    xl = np.linalg.solve(A, p["b"])
    x, rc, it, rel = oracle.cg(L, p["s"], p["b"], rtol=1e-13)
    assert rc == 0 and rel <= 1e-13
    assert np.max(np.abs(xc - xl)) <= 1e-12 * np.max(np.abs(xl))
    assert np.max(np.abs(x - xl)) <= 1e-11 * np.max(np.abs(xl))


def test_cg_masked_matches_dense_restricted():
    L = 8
    p = fc_inputs.problem(L, seed=3, b_kind="normal")
    rng = np.random.default_rng(4)
    mask = (rng.random(L * L) > 0.3).astype(np.uint8)
    act = np.flatnonzero(mask)
    A = oracle.dense_operator(L, p["s"])[np.ix_(act, act)]
    want = np.zeros(L * L)
    want[act] = np.linalg.solve(A, p["b"][act])
    x0 = rng.standard_normal(L * L)  # warm start, including junk off the active set
    x, rc, it, rel = oracle.cg(L, p["s"], p["b"], x0=x0, mask=mask, rtol=1e-13)
    assert rc == 0
    assert np.all(x[mask == 0] == 0.0)
    assert np.max(np.abs(x - want)) <= 1e-11 * np.max(np.abs(want))


def test_cg_warm_start_at_solution_takes_no_iterations():
    L = 4
    p = fc_inputs.problem(L, seed=1)
    x, _, _, _ = oracle.cg(L, p["s"], p["b"], rtol=1e-13)
    x2, rc, it, rel = oracle.cg(L, p["s"], p["b"], x0=x, rtol=1e-12)
    assert rc == 0 and it == 0


def test_cg_iteration_count_scales_with_condition_number():
    """Textbook bound: iterations <= ceil(sqrt(kappa)/2 * ln(2/rtol))."""
    L = 16
    p = fc_inputs.problem(L, seed=0)
    lam = np.linalg.eigvalsh(oracle.dense_operator(L, p["s"]))
    kappa = lam[-1] / lam[0]
    x, rc, it, rel = oracle.cg(L, p["s"], p["b"], rtol=1e-10)
    # the bound is on the A-norm error; allow the usual sqrt(kappa) slack for the residual
    bound = math.ceil(0.5 * math.sqrt(kappa) * math.log(2 * math.sqrt(kappa) / 1e-10))
    assert rc == 0 and it <= bound


def test_cg_maxit_status():
    L = 16
    p = fc_inputs.problem(L, seed=0)
    x, rc, it, rel = oracle.cg(L, p["s"], p["b"], rtol=1e-14, maxit=3)
    assert rc == 1 and it == 3 and rel > 1e-14


def test_apply_A_masks():
    L = 5
    p = fc_inputs.problem(L, seed=2)
    mask = np.ones(L * L, np.uint8)
    mask[[0, 7, 24]] = 0
    x = np.arange(L * L, dtype=float)
    q = oracle.apply_A(L, p["s"], x, mask)
    xm = x * mask
    want = (oracle.conv_direct(L, xm) + p["s"] * xm) * mask
    assert np.allclose(q, want, rtol=1e-13, atol=1e-12)
