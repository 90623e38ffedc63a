"""Failure detection without a GPU fault: allocation failures injected on the
host (every allocation point of a plan's set-up, a batch workspace, a server
request), bounded device waits made to run out by a flag nothing else sets
(the persistent kernel's grid barrier, the TMA pass C's mbarriers), and guard
bands around every workspace checked after the odd-size cases.  Each failure
returns its status and leaves the context usable: the next call succeeds."""
import time

import numpy as np
import pytest
import torch

import fc_inputs
import oracle
import paper_1305_3625_b300 as fc
from gpu_util import dev, host, rel2

pytestmark = pytest.mark.gpu


def live():
    torch.cuda.synchronize()
    m = fc.fc_mem_stats()
    return m["live_allocs"], m["live_bytes"]


def test_plan_create_fails_cleanly_at_every_allocation():
    """The n-th allocation of a plan's set-up fails, for every n: the call
    returns FC_ENOMEM and the library holds exactly what it held before."""
    base = live()
    made = None
    for n in range(1, 400):
        fc.fc_debug_inject(None, fc.FC_INJECT_ALLOC, n)
        try:
            made = fc.fftconv_plan_create(5, fc.FC_F32 | fc.FC_F64, no_autotune=True)
        except fc.FcError as e:
            assert e.code == fc.FC_ENOMEM, (n, e)
            assert live() == base, n
            continue
        break
    fc.fc_debug_inject(None, fc.FC_INJECT_ALLOC, 0)
    assert made is not None and n > 20  # every set-up allocation was failed once
    x = dev(np.ones(25))
    y = torch.empty_like(x)
    fc.fftconv_apply_prec(made, fc.FC_F64, x, y)
    assert np.allclose(host(y), oracle.conv_direct(5, np.ones(25)), rtol=1e-13)
    made.close()
    assert live() == base


def test_batch_workspace_and_server_request_fail_cleanly():
    L = 24
    plan = fc.fftconv_plan_create(L, no_autotune=True)
    p = fc_inputs.problem(L, seed=3, b_kind="normal")
    s, b = dev(np.stack([p["s"]] * 3)), dev(np.stack([p["b"]] * 3))
    for n in (1, 2, 5):
        x = dev(np.zeros((3, L * L)))
        fc.fc_debug_inject(None, fc.FC_INJECT_ALLOC, n)
        with pytest.raises(fc.FcError) as ei:
            fc.cg_solve_batch(plan, s, b, x, rtol=1e-8, mode=fc.FC_MODE_MIXED, x0_zero=True, check=True)
        assert ei.value.code == fc.FC_ENOMEM
    fc.fc_debug_inject(None, fc.FC_INJECT_ALLOC, 0)
    x = dev(np.zeros((3, L * L)))
    rc, rs = fc.cg_solve_batch(plan, s, b, x, rtol=1e-8, mode=fc.FC_MODE_MIXED, x0_zero=True)
    assert rc == fc.FC_OK and all(r["true_rel_resid"] <= 1e-8 for r in rs)
    assert fc.fftconv_plan_check_guards(plan) == 0
    plan.close()
    # a server request whose plan cannot be made ends with FC_ENOMEM; the next one runs
    base = live()
    sv = fc.cg_server_create(1 << 30, max_slots=1)
    fc.fc_debug_inject(None, fc.FC_INJECT_ALLOC, 1)
    t1 = fc.cg_batch_submit(sv, L, p["s"], p["b"], rtol=1e-8)
    r1 = None
    t0 = time.time()
    while r1 is None and time.time() - t0 < 60:
        r1 = fc.cg_poll(sv, t1)
        time.sleep(0.001)
    assert r1 is not None and r1["status"] == fc.FC_ENOMEM
    fc.fc_debug_inject(None, fc.FC_INJECT_ALLOC, 0)
    o = np.zeros(L * L)
    t2 = fc.cg_batch_submit(sv, L, p["s"], p["b"], x_out=o, rtol=1e-8)
    r2 = None
    while r2 is None and time.time() - t0 < 120:
        r2 = fc.cg_poll(sv, t2)
        time.sleep(0.001)
    assert r2 is not None and r2["status"] == fc.FC_OK and r2["true_rel_resid"] <= 1e-8
    sv.close()
    assert live() == base


def test_persistent_grid_barrier_times_out():
    """The persistent inner-CG kernel's last block leaves before its first
    grid-barrier arrival: the other blocks' bounded waits run out, the solve
    returns FC_ETIMEOUT, and the next solve on the same plan is correct."""
    L = 256
    plan = fc.fftconv_plan_create(L, persistent=0)
    info = fc.fftconv_plan_solver(plan, fc.FC_F32)
    assert info["chosen"] == 0 and info["grid"] > 1, info
    p = fc_inputs.problem(L, seed=1)
    s, b = dev(p["s"]), dev(p["b"])
    fc.fc_debug_inject(plan, fc.FC_INJECT_BARRIER, 1 << 14)
    x = torch.zeros_like(s)
    r = fc.cg_solve(plan, s, b, x, rtol=1e-8, mode=fc.FC_MODE_MIXED, x0_zero=True)
    assert r["status"] == fc.FC_ETIMEOUT, r
    fc.fc_debug_inject(plan, fc.FC_INJECT_BARRIER, 0)
    x = torch.zeros_like(s)
    r = fc.cg_solve(plan, s, b, x, rtol=1e-8, mode=fc.FC_MODE_MIXED, x0_zero=True)
    assert r["status"] == fc.FC_OK and r["true_rel_resid"] <= 1e-8
    q = oracle.apply_A(L, p["s"], host(x))
    assert np.linalg.norm(p["b"] - q) <= 1.01e-8 * np.linalg.norm(p["b"])


def test_tma_staged_copy_wait_times_out():
    """The TMA-staged pass C issues no copy for each block's first row pair:
    its bounded mbarrier waits run out, the solve returns FC_ETIMEOUT, and
    the next solve on the same plan is correct."""
    L = 256
    probe = fc.fftconv_plan_create(L, fc.FC_F32, no_autotune=True)
    n = fc.fftconv_plan_shapes(probe, fc.FC_F32)["n_shapes"]
    probe.close()
    # the TMA-staged pass C is the last compiled pass-C shape from M = 256 up
    plan = fc.fftconv_plan_create(L, shapes=(0, 0, n[2] - 1), persistent=-1)
    p = fc_inputs.problem(L, seed=2)
    s, b = dev(p["s"]), dev(p["b"])
    fc.fc_debug_inject(plan, fc.FC_INJECT_TMA, 1 << 12)
    x = torch.zeros_like(s)
    r = fc.cg_solve(plan, s, b, x, rtol=1e-8, mode=fc.FC_MODE_MIXED, x0_zero=True)
    assert r["status"] == fc.FC_ETIMEOUT, r
    fc.fc_debug_inject(plan, fc.FC_INJECT_TMA, 0)
    x = torch.zeros_like(s)
    r = fc.cg_solve(plan, s, b, x, rtol=1e-8, mode=fc.FC_MODE_MIXED, x0_zero=True)
    assert r["status"] == fc.FC_OK and r["true_rel_resid"] <= 1e-8
    q = oracle.apply_A(L, p["s"], host(x))
    assert np.linalg.norm(p["b"] - q) <= 1.01e-8 * np.linalg.norm(p["b"])


@pytest.mark.parametrize("L", [1, 2, 3, 5, 7, 33])
def test_guard_bands_intact_after_odd_sizes(L):
    """Every path on an odd or tiny grid (FP32 and FP64 applies, FP64 and
    mixed solves with and without the preconditioner, a removal step, a
    batched solve): no kernel wrote outside its buffers."""
    plan = fc.fftconv_plan_create(L)
    p = fc_inputs.problem(L, seed=L, with_t=True)
    s, b, t = dev(p["s"]), dev(p["b"]), dev(p["t"])
    for prec, dt in ((fc.FC_F32, torch.float32), (fc.FC_F64, torch.float64)):
        x = dev(p["s"] - 1.0, dt)
        y = torch.empty_like(x)
        fc.fftconv_apply_prec(plan, prec, x, y)
    mask = torch.ones(L * L, device="cuda", dtype=torch.uint8)
    for mode in (fc.FC_MODE_F64, fc.FC_MODE_MIXED):
        for precond in (False, True):
            x = torch.zeros_like(s)
            r = fc.cg_solve(plan, s, b, x, mask=mask, rtol=1e-10, mode=mode, precond=precond)
            assert r["status"] == fc.FC_OK
    rem = torch.empty(1, device="cuda", dtype=torch.int64)
    fc.fc_masked_step(plan, t, mask, x, rem)
    xb = torch.zeros(3 * L * L, device="cuda", dtype=torch.float64)
    rc, _ = fc.cg_solve_batch(plan, s.repeat(3), b.repeat(3), xb, rtol=1e-10, mode=fc.FC_MODE_MIXED,
                              precond=True, x0_zero=True)
    assert rc == fc.FC_OK
    torch.cuda.synchronize()
    assert fc.fftconv_plan_check_guards(plan) == 0
