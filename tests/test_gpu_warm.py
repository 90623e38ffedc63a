"""Warm-start residual update of cg_solve.

After a breaking step (one fibre removed, its x zeroed) the first true
residual of the next solve is the previous solve's final FP64 residual plus
the exact rank-K correction P'(r - A D), D the change of the masked iterate.
These tests pin the updated residual to the oracle's FP64 residual of the
same iterate, compare whole breaking loops with and without the update, and
check every case in which the update must not be used."""
import numpy as np
import pytest
import torch

import fc_inputs
import oracle
import paper_1305_3625_b300 as fc
from gpu_util import dev, host, rel2

pytestmark = pytest.mark.gpu

MODES = [(fc.FC_MODE_F64, False), (fc.FC_MODE_F64, True), (fc.FC_MODE_MIXED, False), (fc.FC_MODE_MIXED, True)]


def fresh(L):
    return fc.fftconv_plan_create(L, fc.FC_F32 | fc.FC_F64)


def oracle_rel_resid(L, s, b, x, mask):
    """||P(b - A x)|| / ||P b|| in FP64 on the host (x taken as masked)."""
    m = mask.astype(bool)
    xm = np.where(m, x, 0.0)
    r = np.where(m, b - oracle.apply_A(L, s, xm, mask), 0.0)
    return float(np.linalg.norm(r) / np.linalg.norm(np.where(m, b, 0.0)))


class Solver:
    """One plan with its device copies of s, b, t, mask and x."""

    def __init__(self, L, p, **kw):
        self.L, self.p, self.kw = L, p, kw
        self.plan = fresh(L)
        self.s, self.b, self.t = dev(p["s"]), dev(p["b"]), dev(p["t"])
        self.mask = dev(np.ones(L * L), torch.uint8)
        self.x = dev(np.zeros(L * L))
        self.rem = torch.empty(1, device="cuda", dtype=torch.int64)

    def solve(self, rtol, **kw):
        args = dict(self.kw)
        args.update(kw)
        return fc.cg_solve(self.plan, self.s, self.b, self.x, mask=self.mask, rtol=rtol, **args)

    def brk(self):
        fc.fc_masked_step(self.plan, self.t, self.mask, self.x, self.rem)
        return int(host(self.rem)[0])


@pytest.mark.parametrize("mode,precond", MODES)
def test_updated_residual_matches_oracle_and_recomputed(mode, precond):
    """rtol = 1 stops a solve at its first true residual, so the reported
    residual is the updated one; it must equal the oracle's FP64 residual of
    the same iterate and the recomputed FP64 product's."""
    L = 100  # M = 256: ragged against every row and column tile
    p = fc_inputs.problem(L, seed=3, with_t=True)
    a = Solver(L, p, mode=mode, precond=precond)
    r = a.solve(1e-10)
    assert r["status"] == fc.FC_OK and r["resid_updated"] == 0
    k = a.brk()
    assert k >= 0
    x_before = host(a.x).copy()
    first = a.solve(1.0)
    assert first["status"] == fc.FC_OK and first["resid_updated"] == 1 and first["iters"] == 0
    assert np.array_equal(host(a.x), x_before)  # stopped at the first residual: x untouched
    mask = host(a.mask)
    want = oracle_rel_resid(L, p["s"], p["b"], x_before, mask)
    assert want > 1e-6  # the removal left a residual far above the tolerance
    assert abs(first["true_rel_resid"] - want) <= 1e-10 * want
    # the same first residual by the FP64 product (update switched off)
    b_ = Solver(L, p, mode=mode, precond=precond)
    b_.x.copy_(a.x)
    b_.mask.copy_(a.mask)
    rec = b_.solve(1.0, warm_resid=False)
    assert rec["resid_updated"] == 0 and rec["iters"] == 0
    assert abs(rec["true_rel_resid"] - first["true_rel_resid"]) <= 1e-10 * want
    # the update with no change at all (K = 0) and then the solve to tolerance
    rtol = 1e-12 if mode == fc.FC_MODE_F64 else 1e-10
    done = a.solve(rtol)
    assert done["status"] == fc.FC_OK and done["resid_updated"] == 1 and done["true_rel_resid"] <= rtol
    xo, rc, _, _ = oracle.cg(L, p["s"], p["b"], x0=x_before, mask=mask, rtol=1e-13)
    assert rc == 0
    assert rel2(host(a.x), xo) <= 100 * rtol  # error <= kappa rtol, kappa ~ 0.8 L


@pytest.mark.parametrize("mode,precond", [(fc.FC_MODE_F64, False), (fc.FC_MODE_MIXED, True)])
def test_breaking_loop_with_and_without_update(mode, precond):
    """Eight breaking steps on two plans, one updating the first residual and
    one recomputing it: the same fibres break, every solve is certified by its
    own FP64 residual, and the final fields agree to the solve tolerance."""
    L, steps = 64, 8
    rtol = 1e-12 if mode == fc.FC_MODE_F64 else 1e-10
    p = fc_inputs.problem(L, seed=5, with_t=True)
    a = Solver(L, p, mode=mode, precond=precond)
    b_ = Solver(L, p, mode=mode, precond=precond, warm_resid=False)
    for st in range(steps):
        ra, rb = a.solve(rtol), b_.solve(rtol)
        for r in (ra, rb):
            assert r["status"] == fc.FC_OK and r["true_rel_resid"] <= rtol
        assert ra["resid_updated"] == (1 if st > 0 else 0)
        assert rb["resid_updated"] == 0
        # the update saves one FP64 product per solve, nothing else changes
        assert rel2(host(a.x), host(b_.x)) <= 1e3 * rtol
        ka, kb = a.brk(), b_.brk()
        assert ka == kb
    assert np.array_equal(host(a.mask), host(b_.mask))


def test_update_only_where_it_applies():
    """The update is used only when s and b are bitwise unchanged, the active
    set did not grow and at most 32 entries of the masked x changed; the
    first residual is checked against the oracle in the applied cases."""
    L = 48
    p = fc_inputs.problem(L, seed=11, with_t=True)
    a = Solver(L, p, mode=fc.FC_MODE_MIXED, precond=True)
    rng = np.random.default_rng(4)

    def check(expect, rtol=1e-10, **kw):
        x_in, m_in = host(a.x).copy(), host(a.mask).copy()
        r = a.solve(rtol, **kw)
        assert r["status"] == fc.FC_OK
        assert r["resid_updated"] == expect
        if rtol >= 1.0 and expect:
            want = oracle_rel_resid(L, host(a.s), host(a.b), x_in, m_in)
            assert abs(r["true_rel_resid"] - want) <= 1e-10 * want + 1e-15
        return r

    check(0)  # fresh plan
    check(1)  # nothing changed (K = 0)
    # s changed in one entry
    s2 = host(a.s).copy()
    s2[7] *= 1.0 + 2.0 ** -40
    a.s.copy_(dev(s2))
    check(0)
    # b changed in one entry
    b2 = host(a.b).copy()
    b2[100] = 1.5
    a.b.copy_(dev(b2))
    check(0)
    # a site removed without a breaking step, and then re-activated
    a.brk()
    check(1, rtol=1.0)
    check(1)
    m = host(a.mask).copy()
    gone = int(np.flatnonzero(m == 0)[0])
    m[gone] = 1
    a.mask.copy_(dev(m, torch.uint8))
    check(0)
    # exactly 32 changed entries of x: applied; 33: recomputed
    for count, expect in ((32, 1), (33, 0)):
        x = host(a.x).copy()
        idx = rng.choice(np.flatnonzero(host(a.mask)), size=count, replace=False)
        x[idx] *= 0.5
        a.x.copy_(dev(x))
        check(expect, rtol=1.0)
        check(1)  # nothing changed since the last (finished) solve
    # entries of x that the mask removes do not count as changes: 40 sites
    # leave the active set (40 changes, recomputed), then their x is set
    m = host(a.mask).copy()
    off = rng.choice(np.flatnonzero(m), size=40, replace=False)
    m[off] = 0
    a.mask.copy_(dev(m, torch.uint8))
    check(0)
    x = host(a.x).copy()
    x[off] = 123.0
    a.x.copy_(dev(x))
    check(1, rtol=1.0)
    # x0_zero and warm_resid=False recompute
    check(0, x0_zero=True)
    check(0, warm_resid=False)
    check(1)


def test_update_after_capped_solve():
    """A solve stopped by max_iter (FC_ENOCONV) still ends on a true residual
    of its final iterate, so the next solve may update it."""
    L = 40
    p = fc_inputs.problem(L, seed=9, with_t=True)
    a = Solver(L, p, mode=fc.FC_MODE_F64, precond=False)
    r = a.solve(1e-12, max_iter=3)
    assert r["status"] == fc.FC_ENOCONV
    a.brk()
    x_in, m_in = host(a.x).copy(), host(a.mask).copy()
    r = a.solve(1.0)
    assert r["status"] == fc.FC_OK and r["resid_updated"] == 1
    want = oracle_rel_resid(L, p["s"], p["b"], x_in, m_in)
    assert abs(r["true_rel_resid"] - want) <= 1e-10 * want


def test_blocking_wait_mode_gives_the_same_solve():
    """fftconv_plan_sync_mode only changes how the host waits: a solve on a
    plan that blocks returns bitwise the same iterate and status."""
    L = 48
    p = fc_inputs.problem(L, seed=12, with_t=True)
    out = []
    for blocking in (False, True):
        pl = fresh(L)
        fc.fftconv_plan_sync_mode(pl, blocking)
        x = dev(np.zeros(L * L))
        r = fc.cg_solve(pl, dev(p["s"]), dev(p["b"]), x, rtol=1e-10, mode=fc.FC_MODE_MIXED, precond=True)
        assert r["status"] == fc.FC_OK
        out.append((host(x), r["iters"], r["refinements"]))
    assert np.array_equal(out[0][0], out[1][0]) and out[0][1:] == out[1][1:]
    with pytest.raises(fc.FcError):
        fc.fftconv_plan_sync_mode(fresh(8), 2)


@pytest.mark.parametrize("precond", [False, True])
def test_fp32_diagonal_copy_follows_s(precond):
    """A mixed solve keeps the FP32 copy of s from the previous solve only
    when that solve was a mixed one and the warm check finds s bitwise
    unchanged.  After an FP64-mode solve on the same plan, and after s
    changes between warm-started mixed solves, the copy is made anew: each
    solve meets its tolerance by the oracle's FP64 residual."""
    L, rtol = 48, 1e-10
    p = fc_inputs.problem(L, seed=5, with_t=True)
    sv = Solver(L, p, precond=precond)
    m = np.ones(L * L)
    # FP64 solve first (the FP32 copy is not made), then a warm mixed solve
    assert sv.solve(rtol, mode=fc.FC_MODE_F64)["status"] == fc.FC_OK
    r = sv.solve(rtol, mode=fc.FC_MODE_MIXED)
    assert r["status"] == fc.FC_OK
    assert oracle_rel_resid(L, p["s"], p["b"], host(sv.x), m) <= 1.01 * rtol
    # warm mixed solve with the same s (the copy is kept), then with a new s
    r = sv.solve(rtol, mode=fc.FC_MODE_MIXED)
    assert r["status"] == fc.FC_OK
    s2 = p["s"] * 1.25
    sv.s = dev(s2)
    r = sv.solve(rtol, mode=fc.FC_MODE_MIXED)
    assert r["status"] == fc.FC_OK
    assert oracle_rel_resid(L, s2, p["b"], host(sv.x), m) <= 1.01 * rtol
