"""Breaking runs under a threshold gradient (fc_fracture_run) and the front
readout (fc_front), against the oracle's masked loop and front."""
import numpy as np
import pytest
import torch

import fc_inputs
import oracle
import paper_1305_3625_b300 as fc
from gpu_util import dev, host

pytestmark = pytest.mark.gpu


def gpu_front(plan, L, mask_np):
    fi = torch.empty(L, device="cuda", dtype=torch.int32)
    de = torch.empty(L, device="cuda", dtype=torch.int32)
    fc.fc_front(plan, dev(mask_np, torch.uint8), fi, de)
    return host(fi), host(de)


@pytest.mark.parametrize("L", [1, 5, 32, 33, 100])
def test_front_matches_oracle(L):
    pl = fc.fftconv_plan_create(L, fc.FC_F64)
    rng = np.random.default_rng(L)
    masks = [np.ones(L * L, np.uint8), np.zeros(L * L, np.uint8)]
    masks += [(rng.random(L * L) >= d).astype(np.uint8) for d in (0.1, 0.5, 0.9)]
    # a rough front: rows below h(ix) broken
    h = rng.integers(0, L + 1, L)
    masks.append((np.arange(L * L) // L >= h[np.arange(L * L) % L]).astype(np.uint8))
    for m in masks:
        fi, de = gpu_front(pl, L, m)
        wfi, wde = oracle.front(L, m)
        assert np.array_equal(fi, wfi) and np.array_equal(de, wde)


def run_gpu(L, p, steps, mode, rtol, precond=False):
    pl = fc.fftconv_plan_create(L, fc.FC_F32 | fc.FC_F64)
    mask = dev(np.ones(L * L), torch.uint8)
    x = dev(np.zeros(L * L))
    removed = torch.full((steps,), -2, device="cuda", dtype=torch.int64)
    ratio = torch.zeros(steps, device="cuda", dtype=torch.float64)
    r = fc.fc_fracture_run(pl, dev(p["s"]), dev(p["b"]), dev(p["t"]), mask, x, steps, removed, ratio,
                           rtol=rtol, mode=mode, precond=precond)
    return pl, r, host(removed), host(ratio), host(mask), host(x)


def test_fracture_run_matches_oracle_loop():
    """FP64 run under a threshold gradient: the same fibres break in the same
    order with the same load ratios, and the fronts agree."""
    L, steps = 16, 30
    p = fc_inputs.problem(L, seed=2, with_t=True, t_gradient=2.0)
    pl, r, rem, rat, mask, _ = run_gpu(L, p, steps, fc.FC_MODE_F64, 1e-12)
    assert r["status"] == fc.FC_OK and r["steps_done"] == steps
    assert r["resid_updated"] == steps - 1  # every solve after the first
    want = oracle.masked_loop(L, p["s"], p["b"], p["t"], steps, rtol=1e-13)
    assert np.array_equal(rem, want["picks"])
    assert np.allclose(rat, want["ratios"], rtol=1e-9, atol=0)
    assert np.array_equal(mask, want["mask"])
    fi, de = gpu_front(pl, L, mask)
    wfi, wde = oracle.front(L, want["mask"])
    assert np.array_equal(fi, wfi) and np.array_equal(de, wde)
    # the gradient makes the weak rows (small iy) break first
    assert np.mean(rem // L) < L / 2


def test_mixed_run_follows_fp64_run():
    """Mixed-precision preconditioned run at L = 64: the same picks as the FP64
    run (ratios within the mixed tolerance), and the damage advances from the
    weak edge."""
    L, steps = 64, 24
    p = fc_inputs.problem(L, seed=6, with_t=True, t_gradient=3.0)
    _, r64, rem64, rat64, mask64, _ = run_gpu(L, p, steps, fc.FC_MODE_F64, 1e-12)
    pl, rmx, remx, ratx, maskx, _ = run_gpu(L, p, steps, fc.FC_MODE_MIXED, 1e-10, precond=True)
    assert r64["status"] == rmx["status"] == fc.FC_OK
    assert np.allclose(ratx, rat64, rtol=1e-5, atol=0)
    assert np.array_equal(remx, rem64)
    fi, de = gpu_front(pl, L, maskx)
    assert np.all(de >= fi)  # the broken region never extends past the damage edge
    assert rmx["resid_updated"] == r64["resid_updated"] == steps - 1


def test_run_stops_when_nothing_is_left():
    L, steps = 2, 6
    p = fc_inputs.problem(L, seed=1, with_t=True, t_gradient=1.0)
    _, r, rem, rat, mask, _ = run_gpu(L, p, steps, fc.FC_MODE_F64, 1e-12)
    assert r["status"] == fc.FC_OK and r["steps_done"] == 4
    assert sorted(rem[:4].tolist()) == [0, 1, 2, 3] and rem[4] == -1
    assert rat[4] == -1.0 and np.all(rat[:4] > 0)
    assert not mask.any()


def test_batched_runs_match_oracle_loops():
    """Three independent FP64 runs in one fc_fracture_run_batch: each breaks
    the oracle's fibres in the oracle's order with its load ratios, the
    problem sizes' smallest (L = 5) running out of fibres mid-run."""
    L, nb, steps = 5, 3, 30
    ps = [fc_inputs.problem(L, seed=20 + k, with_t=True, t_gradient=1.0 + k) for k in range(nb)]
    pl = fc.fftconv_plan_create(L, fc.FC_F32 | fc.FC_F64)
    st = lambda key: dev(np.stack([q[key] for q in ps]))
    mask = dev(np.ones((nb, L * L)), torch.uint8)
    x = dev(np.zeros((nb, L * L)))
    removed = torch.full((nb * steps,), -2, device="cuda", dtype=torch.int64)
    ratio = torch.zeros(nb * steps, device="cuda", dtype=torch.float64)
    rc, rs = fc.fc_fracture_run_batch(pl, st("s"), st("b"), st("t"), mask, x, steps, removed, ratio,
                                      rtol=1e-12, mode=fc.FC_MODE_F64)
    assert rc == fc.FC_OK
    rem, rat, mk = host(removed).reshape(nb, steps), host(ratio).reshape(nb, steps), host(mask).reshape(nb, -1)
    for k, q in enumerate(ps):
        assert rs[k]["status"] == fc.FC_OK and rs[k]["steps_done"] == L * L
        assert rs[k]["resid_updated"] >= L * L - 1  # every solve after the first
        want = oracle.masked_loop(L, q["s"], q["b"], q["t"], L * L, rtol=1e-13)
        assert np.array_equal(rem[k, :L * L], want["picks"])
        assert np.allclose(rat[k, :L * L], want["ratios"], rtol=1e-9, atol=0)
        assert np.all(rem[k, L * L:] == -1) and np.all(rat[k, L * L:] == -1.0)
        assert not mk[k].any()


@pytest.mark.parametrize("warm", [True, False])
@pytest.mark.parametrize("mode,precond", [(fc.FC_MODE_F64, False), (fc.FC_MODE_MIXED, True)])
def test_batched_runs_match_single_runs(mode, precond, warm):
    """Four runs at L = 24 (different gradients), with and without the
    residual update after each removal: the same picks as each run alone
    through fc_fracture_run, ratios within the solve tolerance, one FP64
    product fewer per step with the update."""
    L, nb, steps = 24, 4, 12
    rtol = 1e-12 if mode == fc.FC_MODE_F64 else 1e-10
    ps = [fc_inputs.problem(L, seed=40 + k, with_t=True, t_gradient=0.5 * k) for k in range(nb)]
    pl = fc.fftconv_plan_create(L, fc.FC_F32 | fc.FC_F64)
    st = lambda key: dev(np.stack([q[key] for q in ps]))
    mask = dev(np.ones((nb, L * L)), torch.uint8)
    x = dev(np.zeros((nb, L * L)))
    removed = torch.empty(nb * steps, device="cuda", dtype=torch.int64)
    ratio = torch.empty(nb * steps, device="cuda", dtype=torch.float64)
    rc, rs = fc.fc_fracture_run_batch(pl, st("s"), st("b"), st("t"), mask, x, steps, removed, ratio, rtol=rtol,
                                      mode=mode, precond=precond, warm_resid=warm)
    assert rc == fc.FC_OK and all(r["steps_done"] == steps for r in rs)
    for r in rs:
        assert r["resid_updated"] == (steps - 1 if warm else 0)
    rem, rat = host(removed).reshape(nb, steps), host(ratio).reshape(nb, steps)
    for k, q in enumerate(ps):
        _, r1, rem1, rat1, mask1, x1 = run_gpu(L, q, steps, mode, rtol, precond=precond)
        assert np.array_equal(rem[k], rem1)
        assert np.allclose(rat[k], rat1, rtol=1e-6 if mode == fc.FC_MODE_MIXED else 1e-9, atol=0)
        assert np.array_equal(host(mask).reshape(nb, -1)[k], mask1)
