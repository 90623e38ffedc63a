"""Parity of plans built with the cell-integrated Green's function of Eq. 1c
(FC_GREEN_CELL) with the oracle's cell integral."""
import numpy as np
import pytest
import torch

import fc_inputs
import oracle
import paper_1305_3625_b300 as fc
from gpu_util import U32, U64, conv_err, conv_rel_bound, dev, host, rel2

pytestmark = pytest.mark.gpu

_plans = {}


def plan(L):
    if L not in _plans:
        _plans[L] = fc.fftconv_plan_create(L, fc.FC_F32 | fc.FC_F64, green=fc.FC_GREEN_CELL)
    return _plans[L]


def apply(L, x, prec):
    dt = torch.float32 if prec == fc.FC_F32 else torch.float64
    y = torch.empty(L * L, device="cuda", dtype=dt)
    fc.fftconv_apply_prec(plan(L), prec, dev(x, dt), y)
    return host(y).astype(np.float64)


@pytest.mark.parametrize("L", [2, 3, 7, 16])
def test_delta_response_is_the_cell_integral(L):
    """C applied to a unit load at site (0, 0) returns G(r_i) at every site:
    the whole offset table, compared entry by entry."""
    x = np.zeros(L * L)
    x[0] = 1.0
    y = apply(L, x, fc.FC_F64)
    want = np.array([oracle.G_cell(i % L, i // L) for i in range(L * L)])
    M = fc_inputs.padded_side(L)
    # each output is one kernel value carried through the FFT round trip
    assert np.max(np.abs(y - want)) <= conv_rel_bound(U64, M) * np.linalg.norm(want)
    assert rel2(y, want) <= conv_rel_bound(U64, M)


def test_cell_and_point_plans_differ_by_the_far_field_term():
    """Outside the self term the two operators differ by about 1/(24 r^2)
    relative: the cell plan's delta response is not the point plan's."""
    L = 8
    x = np.zeros(L * L)
    x[0] = 1.0
    y_cell = apply(L, x, fc.FC_F64)
    pp = fc.fftconv_plan_create(L, fc.FC_F64)
    yp = torch.empty(L * L, device="cuda", dtype=torch.float64)
    fc.fftconv_apply_prec(pp, fc.FC_F64, dev(x), yp)
    y_point = host(yp)
    assert y_cell[0] == pytest.approx(y_point[0], rel=1e-13)  # same self term
    r = np.hypot(np.arange(L * L) % L, np.arange(L * L) // L)[1:]
    ratio = y_cell[1:] / y_point[1:]
    assert np.all(np.abs(ratio - 1 - 1 / (24 * r**2)) <= 0.02 / r**4 + 1e-12)


@pytest.mark.parametrize("L", [1, 5, 17, 33, 64])
def test_apply_matches_direct_sum(L):
    rng = np.random.default_rng(700 + L)
    x = rng.standard_normal(L * L)
    M = fc_inputs.padded_side(L)
    x32 = x.astype(np.float32).astype(np.float64)
    with oracle.use_green(oracle.GREEN_CELL, L):
        ref64 = oracle.conv_direct(L, x)
        ref32 = oracle.conv_direct(L, x32)
    assert conv_err(apply(L, x, fc.FC_F64), ref64) <= conv_rel_bound(U64, M)
    assert conv_err(apply(L, x32, fc.FC_F32), ref32) <= conv_rel_bound(U32, M)


def test_apply_sampled_at_L512():
    """At L = 512 (offsets up to 722, all three quadrature orders) sampled
    outputs against the oracle's direct sums."""
    L = 512
    rng = np.random.default_rng(5)
    x = rng.uniform(0.5, 1.5, L * L)
    y = apply(L, x, fc.FC_F64)
    pts = [(0, 0), (L - 1, L - 1), (0, L - 1), (L // 2, 17), (301, 488), (9, 9)]
    with oracle.use_green(oracle.GREEN_CELL, L):
        for iy, ix in pts:
            want = oracle.conv_direct_at(L, x, iy, ix)
            assert y[iy * L + ix] == pytest.approx(want, rel=1e-12)


@pytest.mark.parametrize("mode,precond", [(fc.FC_MODE_F64, False), (fc.FC_MODE_MIXED, True)])
def test_solve_matches_dense(mode, precond):
    L = 12
    p = fc_inputs.problem(L, seed=21, b_kind="normal")
    with oracle.use_green(oracle.GREEN_CELL, L):
        want = np.linalg.solve(oracle.dense_operator(L, p["s"]), p["b"])
    x = dev(np.zeros(L * L))
    rtol = 1e-12 if mode == fc.FC_MODE_F64 else 1e-10
    r = fc.cg_solve(plan(L), dev(p["s"]), dev(p["b"]), x, rtol=rtol, mode=mode, precond=precond)
    assert r["status"] == fc.FC_OK and r["true_rel_resid"] <= rtol
    assert rel2(host(x), want) <= 100 * rtol


def test_warm_residual_update_uses_the_cell_table():
    """The warm-start residual update reads the plan's offset table, so with
    the cell kernel it must reproduce the oracle's cell-kernel residual."""
    L = 40
    p = fc_inputs.problem(L, seed=8, with_t=True)
    s, b, t = dev(p["s"]), dev(p["b"]), dev(p["t"])
    mask = dev(np.ones(L * L), torch.uint8)
    x = dev(np.zeros(L * L))
    rem = torch.empty(1, device="cuda", dtype=torch.int64)
    pl = plan(L)
    r = fc.cg_solve(pl, s, b, x, mask=mask, rtol=1e-11, mode=fc.FC_MODE_F64)
    assert r["status"] == fc.FC_OK
    fc.fc_masked_step(pl, t, mask, x, rem)
    xh, mh = host(x).copy(), host(mask).copy()
    r = fc.cg_solve(pl, s, b, x, mask=mask, rtol=1.0, mode=fc.FC_MODE_F64)
    assert r["resid_updated"] == 1
    with oracle.use_green(oracle.GREEN_CELL, L):
        res = np.where(mh > 0, p["b"] - oracle.apply_A(L, p["s"], np.where(mh > 0, xh, 0.0), mh), 0.0)
    want = np.linalg.norm(res) / np.linalg.norm(np.where(mh > 0, p["b"], 0.0))
    assert r["true_rel_resid"] == pytest.approx(want, rel=1e-10)


def test_invalid_green_kind():
    with pytest.raises(fc.FcError):
        fc.fftconv_plan_create(8, fc.FC_F64, green=7)
