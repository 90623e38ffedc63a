"""Parity of cg_solve (FP64 and mixed) and fc_masked_step with the oracle."""
import math

import numpy as np
import pytest
import torch

import fc_inputs
import oracle
import paper_1305_3625_b300 as fc
from gpu_util import dev, host, rel2

pytestmark = pytest.mark.gpu

_plans = {}


def plan(L):
    if L not in _plans:
        _plans[L] = fc.fftconv_plan_create(L, fc.FC_F32 | fc.FC_F64)
    return _plans[L]


def solve(L, s, b, mode, rtol, x0=None, mask=None, **kw):
    x = dev(np.zeros(L * L) if x0 is None else x0)
    m = None if mask is None else dev(mask, torch.uint8)
    res = fc.cg_solve(plan(L), dev(s), dev(b), x, mask=m, rtol=rtol, mode=mode, **kw)
    return host(x), res


def dense_solution(L, s, b, mask=None):
    A = oracle.dense_operator(L, s)
    if mask is None:
        return np.linalg.solve(A, b)
    act = np.flatnonzero(mask)
    x = np.zeros(L * L)
    x[act] = np.linalg.solve(A[np.ix_(act, act)], b[act])
    return x


# Targets (relative solution error): 1e-10 for the FP64 path, 1e-6 for the
# mixed path.  error <= kappa * residual and kappa ~ 0.8 L, so the residual
# tolerances below leave a factor >= 10 of margin at L <= 32.
F64_RTOL, F64_ERR = 1e-12, 1e-10
MIX_RTOL, MIX_ERR = 1e-9, 1e-6


def test_L1_closed_form(golden):
    g0 = golden("green_self_term.txt")["G0"]
    for mode in (fc.FC_MODE_F64, fc.FC_MODE_MIXED):
        x, res = solve(1, np.array([0.7]), np.array([2.5]), mode, 1e-14)
        assert res["status"] == fc.FC_OK
        assert x[0] == pytest.approx(2.5 / (g0 + 0.7), rel=1e-13)


@pytest.mark.parametrize("L", [2, 3, 5, 8, 16, 32])
@pytest.mark.parametrize("b_kind", ["ones", "normal"])
def test_solve_matches_dense(L, b_kind):
    p = fc_inputs.problem(L, seed=L, b_kind=b_kind)
    want = dense_solution(L, p["s"], p["b"])
    x64, r64 = solve(L, p["s"], p["b"], fc.FC_MODE_F64, F64_RTOL)
    assert r64["status"] == fc.FC_OK and r64["true_rel_resid"] <= F64_RTOL
    assert rel2(x64, want) <= F64_ERR
    xm, rm = solve(L, p["s"], p["b"], fc.FC_MODE_MIXED, MIX_RTOL)
    assert rm["status"] == fc.FC_OK and rm["true_rel_resid"] <= MIX_RTOL
    assert rel2(xm, want) <= MIX_ERR


def test_config1_plain_fp64_L32():
    """L = 32, s ~ U[0.5, 1.5] seed 0, b = 1, CG from x = 0 to rtol 1e-10."""
    L = 32
    p = fc_inputs.problem(L, seed=0)
    want = dense_solution(L, p["s"], p["b"])
    xo, rc, it_o, rel_o = oracle.cg(L, p["s"], p["b"], rtol=1e-10)
    x, res = solve(L, p["s"], p["b"], fc.FC_MODE_F64, 1e-10)
    assert res["status"] == fc.FC_OK and res["true_rel_resid"] <= 1e-10
    # recompute the residual with the oracle's own operator
    r = p["b"] - oracle.apply_A(L, p["s"], x)
    assert np.linalg.norm(r) / np.linalg.norm(p["b"]) <= 1e-10 * (1 + 1e-3)
    kappa = 25.7  # kappa(C + S) at L = 32 (eigenvalues of the oracle's dense operator)
    assert rel2(x, want) <= kappa * 1e-10
    assert rel2(x, xo) <= 2 * kappa * 1e-10
    # same Krylov method, same stopping rule: iteration counts agree closely
    assert abs(res["iters"] - it_o) <= 2


def test_masked_warm_start_matches_dense():
    L = 16
    p = fc_inputs.problem(L, seed=5, b_kind="normal")
    rng = np.random.default_rng(9)
    mask = (rng.random(L * L) > 0.25).astype(np.uint8)
    want = dense_solution(L, p["s"], p["b"], mask)
    x0 = rng.standard_normal(L * L)  # junk everywhere, including inactive sites
    for mode, rtol, err in ((fc.FC_MODE_F64, F64_RTOL, F64_ERR), (fc.FC_MODE_MIXED, MIX_RTOL, MIX_ERR)):
        x, res = solve(L, p["s"], p["b"], mode, rtol, x0=x0, mask=mask)
        assert res["status"] == fc.FC_OK
        assert np.all(x[mask == 0] == 0.0)
        assert rel2(x, want) <= err


def test_warm_start_at_solution_needs_no_iterations():
    L = 8
    p = fc_inputs.problem(L, seed=1)
    x, _ = solve(L, p["s"], p["b"], fc.FC_MODE_F64, 1e-13)
    x2, res = solve(L, p["s"], p["b"], fc.FC_MODE_F64, 1e-11, x0=x)
    assert res["status"] == fc.FC_OK and res["iters"] == 0 and res["refinements"] == 1


def test_zero_rhs_gives_zero():
    L = 8
    p = fc_inputs.problem(L, seed=1)
    x, res = solve(L, p["s"], np.zeros(L * L), fc.FC_MODE_MIXED, 1e-10, x0=np.ones(L * L), x0_zero=True)
    assert res["status"] == fc.FC_OK and np.all(x == 0.0)


def test_max_iter_status():
    L = 32
    p = fc_inputs.problem(L, seed=0)
    x, res = solve(L, p["s"], p["b"], fc.FC_MODE_F64, 1e-14, max_iter=3)
    assert res["rc"] == fc.FC_ENOCONV and res["status"] == fc.FC_ENOCONV and res["iters"] == 3


def test_nan_in_rhs_is_reported():
    L = 8
    p = fc_inputs.problem(L, seed=0)
    b = p["b"].copy()
    b[5] = np.nan
    for mode in (fc.FC_MODE_F64, fc.FC_MODE_MIXED):
        x, res = solve(L, p["s"], b, mode, 1e-10)
        assert res["status"] == fc.FC_ENANINF


def test_solve_is_deterministic():
    L = 64
    p = fc_inputs.problem(L, seed=3, b_kind="normal")
    for mode in (fc.FC_MODE_F64, fc.FC_MODE_MIXED):
        a, ra = solve(L, p["s"], p["b"], mode, 1e-10)
        b, rb = solve(L, p["s"], p["b"], mode, 1e-10)
        keys = ("status", "iters", "refinements", "true_rel_resid", "bnorm")
        assert np.array_equal(a, b) and all(ra[k] == rb[k] for k in keys)


@pytest.mark.parametrize("L", [128, 1024])
def test_full_size_residual_and_agreement(L):
    """Config 2 scale: FP64 and mixed solves from x = 0 to rtol 1e-10; the
    residual is recomputed by the oracle's FP64 operator, and the two
    solutions agree within the mixed target."""
    p = fc_inputs.problem(L, seed=0)
    x64, r64 = solve(L, p["s"], p["b"], fc.FC_MODE_F64, 1e-10)
    xm, rm = solve(L, p["s"], p["b"], fc.FC_MODE_MIXED, 1e-10)
    nb = np.linalg.norm(p["b"])
    for x, res in ((x64, r64), (xm, rm)):
        assert res["status"] == fc.FC_OK
        r = p["b"] - oracle.apply_A(L, p["s"], x)
        assert np.linalg.norm(r) / nb <= 1e-10 * 1.01
    kappa = 0.8 * L
    assert rel2(xm, x64) <= 2 * kappa * 1e-10


# ------------------------------------------------------- masked removal --

def test_masked_step_matches_oracle_argmax():
    L = 64
    p = fc_inputs.problem(L, seed=2, with_t=True)
    rng = np.random.default_rng(1)
    x = rng.standard_normal(L * L)
    mask = (rng.random(L * L) > 0.1).astype(np.uint8)
    want, _ = oracle.argmax_ratio(x, p["t"], mask)
    xd, md = dev(x), dev(mask, torch.uint8)
    rem = torch.empty(1, device="cuda", dtype=torch.int64)
    fc.fc_masked_step(plan(L), dev(p["t"]), md, xd, rem)
    assert int(host(rem)[0]) == want
    mh, xh = host(md), host(xd)
    assert mh[want] == 0 and xh[want] == 0.0
    mask[want] = 0
    assert np.array_equal(mh, mask)


def test_masked_step_ties_and_empty():
    L = 4
    t = np.ones(16)
    x = np.zeros(16)
    x[[3, 9, 12]] = 2.0  # three-way tie: lowest index wins
    xd, md = dev(x), dev(np.ones(16), torch.uint8)
    rem = torch.empty(1, device="cuda", dtype=torch.int64)
    fc.fc_masked_step(plan(L), dev(t), md, xd, rem)
    assert int(host(rem)[0]) == 3
    md = dev(np.zeros(16), torch.uint8)
    fc.fc_masked_step(plan(L), dev(t), md, xd, rem)
    assert int(host(rem)[0]) == -1


@pytest.mark.parametrize("case", ["near_ties", "exact_ties", "extreme", "zeros"])
def test_masked_step_edge_ratios(case):
    """The removal kernel screens sites by an FP32 estimate of |x|/t before
    the exact FP64 quotient decides; its pick must still be the oracle's,
    bit for bit: ratios within 1e-12 of the maximum (where the estimate
    cannot tell them apart), exact ties at scattered sites (lowest index),
    ratios and operands beyond FP32's range (1e-40 .. 1e40), and x = 0."""
    L = 300
    N = L * L
    rng = np.random.default_rng(7)
    x = rng.standard_normal(N)
    t = rng.uniform(0.05, 1.0, N)
    mask = (rng.random(N) > 0.05).astype(np.uint8)
    if case == "near_ties":
        top = np.max(np.abs(x) / t) * 2.0
        idx = rng.choice(N, 40, replace=False)
        x[idx] = top * t[idx] * (1.0 + rng.integers(-5, 5, 40) * 1e-13)
    elif case == "exact_ties":
        idx = np.sort(rng.choice(N, 12, replace=False))
        t[idx] = 0.25
        x[idx] = 1e3  # ratio 4000 exactly at every one of them
        mask[idx[0]] = 0  # the lowest is masked out: the next one wins
    elif case == "extreme":
        idx = rng.choice(N, 30, replace=False)
        x[idx[:10]] = 1e-40
        t[idx[10:20]] = 1e-38
        x[idx[20:]] = 1e40
        t[idx[25:]] = 1e35
    else:
        x[:] = 0.0
        x[rng.choice(N, 3, replace=False)] = -0.0
    want, wr = oracle.argmax_ratio(x, t, mask)
    xd, md = dev(x), dev(mask, torch.uint8)
    rem = torch.empty(1, device="cuda", dtype=torch.int64)
    fc.fc_masked_step(plan(L), dev(t), md, xd, rem)
    got = int(host(rem)[0])
    print(f"{case}: oracle {want} ({wr:.17g}), kernel {got}")
    assert got == want


@pytest.mark.parametrize("mode,rtol,rel_tie", [(0, 1e-12, 1e-9), (1, 1e-10, 1e-5)])
def test_masked_loop_against_oracle(mode, rtol, rel_tie):
    """Quasi-static loop: solve, remove argmax |x|/t, warm start.  At each step
    the GPU's pick must carry a ratio within rel_tie of the oracle's maximum;
    on a legitimate near-tie divergence the oracle's pick is replayed."""
    L, steps = 16, 12
    p = fc_inputs.problem(L, seed=0, with_t=True)
    mask = np.ones(L * L, np.uint8)
    x = np.zeros(L * L)
    rem = torch.empty(1, device="cuda", dtype=torch.int64)
    diverged = 0
    for st in range(steps):
        xg, res = solve(L, p["s"], p["b"], mode, rtol, x0=x, mask=mask)
        assert res["status"] == fc.FC_OK
        xo, rc, _, _ = oracle.cg(L, p["s"], p["b"], x0=x, mask=mask, rtol=1e-13)
        ko, ro = oracle.argmax_ratio(xo, p["t"], mask)
        xd, md = dev(xg), dev(mask, torch.uint8)
        fc.fc_masked_step(plan(L), dev(p["t"]), md, xd, rem)
        kg = int(host(rem)[0])
        assert abs(abs(xo[kg]) / p["t"][kg] - ro) <= rel_tie * ro
        if kg != ko:
            diverged += 1
        mask[ko] = 0
        x = xo.copy()
        x[ko] = 0.0
    assert diverged <= 1


@pytest.mark.parametrize("L", [32, 100, 256])
def test_every_inner_loop_variant_solves(L):
    """The per-pass graph loop and every compiled persistent inner-CG kernel
    reach the same solution (dense solve at L = 32, FP64 solve otherwise)."""
    p = fc_inputs.problem(L, seed=7, b_kind="normal")
    if L <= 32:
        want = dense_solution(L, p["s"], p["b"])
    else:
        want, r = solve(L, p["s"], p["b"], fc.FC_MODE_F64, 1e-13)
        assert r["status"] == fc.FC_OK
    n = fc.fftconv_plan_solver(plan(L), fc.FC_F32)["n"]
    assert n >= 1
    for k in [-1] + list(range(n)):
        pl = fc.fftconv_plan_create(L, persistent=k)
        info = fc.fftconv_plan_solver(pl, fc.FC_F32)
        assert info["chosen"] == k or (k >= 0 and info["chosen"] == -1)
        for mode, rtol, err in ((fc.FC_MODE_F64, F64_RTOL, F64_ERR), (fc.FC_MODE_MIXED, MIX_RTOL, MIX_ERR)):
            x = dev(np.zeros(L * L))
            res = fc.cg_solve(pl, dev(p["s"]), dev(p["b"]), x, rtol=rtol, mode=mode)
            assert res["status"] == fc.FC_OK, (k, mode, res)
            assert rel2(host(x), want) <= (err if L <= 32 else 10 * err), (k, mode)


# ------------------------------------------------ preconditioned CG --------

@pytest.mark.parametrize("L", [1, 3, 8, 32])
def test_pcg_matches_dense(L):
    p = fc_inputs.problem(L, seed=40 + L, b_kind="normal")
    want = dense_solution(L, p["s"], p["b"])
    for mode, rtol, err in ((fc.FC_MODE_F64, F64_RTOL, F64_ERR), (fc.FC_MODE_MIXED, MIX_RTOL, MIX_ERR)):
        x, res = solve(L, p["s"], p["b"], mode, rtol, precond=True)
        assert res["status"] == fc.FC_OK, (mode, res)
        assert rel2(x, want) <= err


def test_pcg_masked_warm_start():
    L = 16
    p = fc_inputs.problem(L, seed=8, b_kind="normal")
    rng = np.random.default_rng(2)
    mask = (rng.random(L * L) > 0.2).astype(np.uint8)
    want = dense_solution(L, p["s"], p["b"], mask)
    x0 = rng.standard_normal(L * L)
    for mode, rtol, err in ((fc.FC_MODE_F64, F64_RTOL, F64_ERR), (fc.FC_MODE_MIXED, MIX_RTOL, MIX_ERR)):
        x, res = solve(L, p["s"], p["b"], mode, rtol, x0=x0, mask=mask, precond=True)
        assert res["status"] == fc.FC_OK
        assert np.all(x[mask == 0] == 0.0)
        assert rel2(x, want) <= err


@pytest.mark.parametrize("L", [256, 1024])
def test_pcg_residual_and_fewer_iterations(L):
    """Same solution (residual recomputed by the oracle's operator) in far
    fewer iterations: the preconditioned spectrum does not grow with L."""
    p = fc_inputs.problem(L, seed=0)
    x_cg, r_cg = solve(L, p["s"], p["b"], fc.FC_MODE_F64, 1e-10)
    for mode in (fc.FC_MODE_F64, fc.FC_MODE_MIXED):
        x, res = solve(L, p["s"], p["b"], mode, 1e-10, precond=True)
        assert res["status"] == fc.FC_OK
        r = p["b"] - oracle.apply_A(L, p["s"], x)
        assert np.linalg.norm(r) / np.linalg.norm(p["b"]) <= 1e-10 * 1.01
        assert rel2(x, x_cg) <= 2 * 0.8 * L * 1e-10
        assert res["iters"] * 2 < r_cg["iters"], (res["iters"], r_cg["iters"])


@pytest.mark.parametrize("L", [64, 128, 512])
def test_every_pass_shape_solves(L):
    """Each compiled shape of the row passes (whose epilogues carry the CG
    reductions) solves the preconditioned mixed system to tolerance."""
    p = fc_inputs.problem(L, seed=31, b_kind="normal")
    n = fc.fftconv_plan_shapes(plan(L), fc.FC_F32)["n_shapes"]
    for k in range(max(n[0], n[2])):
        shapes = (min(k, n[0] - 1), 0, min(k, n[2] - 1))
        pl = fc.fftconv_plan_create(L, fc.FC_F32 | fc.FC_F64, shapes=shapes)
        x = dev(np.zeros(L * L))
        r = fc.cg_solve(pl, dev(p["s"]), dev(p["b"]), x, rtol=1e-8, mode=fc.FC_MODE_MIXED, precond=True)
        assert r["status"] == fc.FC_OK and r["true_rel_resid"] <= 1e-8, (L, shapes, r)


@pytest.mark.parametrize("L", [100, 1024])
def test_product_dot_products_fp64_grade(L):
    """The FP32 passes' dot products p.q, r.q, q.q against exact sums of the
    same FP32 vectors' products (math.fsum of the FP64 products, which are
    exact for FP32 factors).  Each thread's Dot2 pair and the two-float block
    and grid combination keep the error at the order of (16 u)^2 and
    2^-44 per combining level of sum |a_i b_i|: 1e-11 of it is allowed,
    against about 1e-6 for plain FP32 partial sums of 16 products."""
    import math
    plan = fc.fftconv_plan_create(L, fc.FC_F32 | fc.FC_F64)
    rng = np.random.default_rng(L)
    pv = dev(rng.standard_normal(L * L), torch.float32)
    rv = dev(rng.standard_normal(L * L), torch.float32)
    sv = dev(rng.uniform(0.5, 1.5, L * L), torch.float32)
    q = torch.empty_like(pv)
    got = fc.fftconv_cg_product(plan, fc.FC_F32, pv, rv, sv, q)
    ph, rh, qh = (host(t).astype(np.float64) for t in (pv, rv, q))
    for name, a, b, g in (("p.q", ph, qh, got[0]), ("r.q", rh, qh, got[1]), ("q.q", qh, qh, got[2])):
        terms = a * b
        exact = math.fsum(terms)
        scale = math.fsum(np.abs(terms))
        print(f"L={L} {name}: {g:.17g} exact {exact:.17g}, error {abs(g - exact) / scale:.2e} of sum |terms|")
        assert abs(g - exact) <= 1e-11 * scale, (name, g, exact)
    # FP64 passes: FP64 sums of the FP64 vectors' products
    p64, r64, s64 = (dev(host(t).astype(np.float64)) for t in (pv, rv, sv))
    q64 = torch.empty_like(p64)
    got64 = fc.fftconv_cg_product(plan, fc.FC_F64, p64, r64, s64, q64)
    qh64 = host(q64)
    for a, b, g in ((ph, qh64, got64[0]), (rh, qh64, got64[1]), (qh64, qh64, got64[2])):
        assert abs(g - math.fsum(a * b)) <= 1e-12 * math.fsum(np.abs(a * b))
