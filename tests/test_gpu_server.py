"""The continuous-batching solve server (cg_server_*): results in a mix equal
the same requests solved alone, requests of one size run as batches, budget
admission, polling."""
import time

import numpy as np
import pytest
import torch

import fc_inputs
import oracle
import paper_1305_3625_b300 as fc
from gpu_util import dev, host

pytestmark = pytest.mark.gpu


def alone(L, s, b, rtol, mode, precond=False):
    """The request solved by itself: the server's batched solve with one
    problem, on a fresh plan of its size."""
    plan = fc.fftconv_plan_create(L)
    x = dev(np.zeros(L * L))
    rc, rs = fc.cg_solve_batch(plan, dev(s), dev(b), x, rtol=rtol, mode=mode, x0_zero=True, precond=precond)
    return host(x), rs[0]


def wait_all(sv, tickets, timeout=120.0):
    out = {}
    t0 = time.time()
    while len(out) < len(tickets):
        for t in tickets:
            if t not in out:
                r = fc.cg_poll(sv, t)
                if r is not None:
                    out[t] = r
        assert time.time() - t0 < timeout, "server did not finish"
        time.sleep(0.001)
    return out


def test_mix_equals_alone():
    reqs = []
    for k, (L, mode, tol) in enumerate([(8, 1, 1e-8), (16, 0, 1e-10), (32, 1, 1e-6), (64, 1, 1e-8),
                                        (16, 1, 1e-8), (33, 0, 1e-9), (64, 0, 1e-10), (8, 1, 1e-6)]):
        p = fc_inputs.problem(L, seed=100 + k, b_kind="normal")
        reqs.append((L, mode, tol, p["s"], p["b"]))
    want = [alone(L, s, b, tol, mode) for (L, mode, tol, s, b) in reqs]
    sv = fc.cg_server_create(8 << 30, max_slots=4)
    outs = [np.zeros(L * L) for (L, *_rest) in reqs]
    tickets = [fc.cg_batch_submit(sv, L, s, b, x_out=o, rtol=tol, mode=mode)
               for (L, mode, tol, s, b), o in zip(reqs, outs)]
    res = wait_all(sv, tickets)
    for (xa, ra), o, t in zip(want, outs, tickets):
        r = res[t]
        assert r["status"] == fc.FC_OK and r["latency_s"] >= r["run_s"] > 0
        assert r["iters"] == ra["iters"] and r["refinements"] == ra["refinements"]
        assert np.array_equal(o, xa)  # bitwise: a solve depends only on its own inputs
    st = fc.cg_server_stats(sv)
    assert st["queued"] == 0 and st["plans"] >= 4 and st["peak"] <= 8 << 30
    sv.close()


def test_same_size_requests_run_as_batches():
    """A burst of requests of one size with mixed tolerances: one slot takes
    them into batched solves, each result bitwise the request alone."""
    L = 48
    reqs = []
    for k in range(20):
        p = fc_inputs.problem(L, seed=900 + k, b_kind="normal")
        reqs.append((p["s"], p["b"], (1e-6, 1e-8, 1e-10)[k % 3]))
    sv = fc.cg_server_create(4 << 30, max_slots=1)
    # occupy the slot so that the burst queues up behind it
    big = fc_inputs.problem(256, seed=1, b_kind="normal")
    first = fc.cg_batch_submit(sv, 256, big["s"], big["b"], rtol=1e-10, mode=1, precond=True)
    outs = [np.zeros(L * L) for _ in reqs]
    tickets = [fc.cg_batch_submit(sv, L, s, b, x_out=o, rtol=tol, mode=1, precond=True)
               for (s, b, tol), o in zip(reqs, outs)]
    res = wait_all(sv, [first] + tickets)
    st = fc.cg_server_batches(sv)
    assert st["solves"] == 21 and st["max_batch"] > 1 and st["batches"] < 21
    for (s, b, tol), o, t in zip(reqs, outs, tickets):
        xa, ra = alone(L, s, b, tol, 1, precond=True)
        r = res[t]
        assert r["status"] == fc.FC_OK and r["true_rel_resid"] <= tol
        assert r["iters"] == ra["iters"] and np.array_equal(o, xa)
    sv.close()


def test_borrowed_inputs():
    """FC_REQ_BORROW: s and b are read when the request runs, not copied at
    submit; the results are bitwise those of copied requests."""
    L = 40
    probs = [fc_inputs.problem(L, seed=70 + k, b_kind="normal") for k in range(6)]
    sv = fc.cg_server_create(4 << 30, max_slots=2)
    outs = {False: [np.zeros(L * L) for _ in probs], True: [np.zeros(L * L) for _ in probs]}
    for borrow in (False, True):
        ts = [fc.cg_batch_submit(sv, L, p["s"], p["b"], x_out=o, rtol=1e-9, mode=1, precond=True, borrow=borrow)
              for p, o in zip(probs, outs[borrow])]
        res = wait_all(sv, ts)
        assert all(r["status"] == fc.FC_OK for r in res.values())
    for a, b in zip(outs[False], outs[True]):
        assert np.array_equal(a, b)
    sv.close()


def test_budget_admission_and_eviction():
    L1, L2 = 64, 128
    p1, p2 = fc_inputs.problem(L1, seed=1), fc_inputs.problem(L2, seed=2)
    one_plan = 40 << 20  # holds one L=128 plan (about 25 MB) but not two
    sv = fc.cg_server_create(one_plan, max_slots=2)
    outs, tickets = [], []
    for k in range(6):
        L, p = (L1, p1) if k % 2 == 0 else (L2, p2)
        o = np.zeros(L * L)
        outs.append(o)
        tickets.append(fc.cg_batch_submit(sv, L, p["s"], p["b"], x_out=o, rtol=1e-8, mode=1))
    res = wait_all(sv, tickets)
    assert all(r["status"] == fc.FC_OK for r in res.values())
    assert fc.cg_server_stats(sv)["peak"] <= one_plan
    x1, _ = alone(L1, p1["s"], p1["b"], 1e-8, 1)
    assert np.array_equal(outs[0], x1) and np.array_equal(outs[2], x1)
    # a request that can never fit is refused at submit
    big = fc_inputs.problem(1024, seed=3)  # about 110 MB of plan
    with pytest.raises(fc.FcError) as ei:
        fc.cg_batch_submit(sv, 1024, big["s"], big["b"], rtol=1e-8)
    assert ei.value.code == fc.FC_EBUDGET
    with pytest.raises(fc.FcError) as ei:
        fc.cg_poll(sv, 987654321)
    assert ei.value.code == fc.FC_ENOTFOUND
    sv.close()


def test_many_small_requests_batch():
    """24 small requests through one slot run as batched solves and finish
    sooner than the same solves one at a time on one plan (medians of three
    repeats of each, so that one slow sample on a shared GPU decides
    nothing)."""
    L = 64
    probs = [fc_inputs.problem(L, seed=500 + k, b_kind="normal") for k in range(24)]
    sv = fc.cg_server_create(4 << 30, max_slots=1)
    wait_all(sv, [fc.cg_batch_submit(sv, L, p["s"], p["b"], rtol=1e-8) for p in probs])  # plan, workspace
    t_server = []
    for _ in range(3):
        t0 = time.perf_counter()
        wait_all(sv, [fc.cg_batch_submit(sv, L, p["s"], p["b"], rtol=1e-8) for p in probs])
        t_server.append(time.perf_counter() - t0)
    assert fc.cg_server_batches(sv)["max_batch"] > 1
    sv.close()
    plan = fc.fftconv_plan_create(L)
    inputs = [(dev(p["s"]), dev(p["b"])) for p in probs]
    x = dev(np.zeros(L * L))
    fc.cg_solve(plan, *inputs[0], x, rtol=1e-8, mode=1, x0_zero=True)  # graph built
    torch.cuda.synchronize()
    t_alone = []
    for _ in range(3):
        t0 = time.perf_counter()
        for s, b in inputs:
            fc.cg_solve(plan, s, b, x, rtol=1e-8, mode=1, x0_zero=True)
        t_alone.append(time.perf_counter() - t0)
    assert sorted(t_server)[1] < sorted(t_alone)[1]


def test_config4_sizes_against_oracle():
    """Requests of the serving mix's sizes, L = 32, 1024 and 2048 (their
    batched plans at M = 64, 2048, 4096), with tolerances 1e-6 and 1e-8,
    through a server with several slots: each result's residual
    b - (C + S) x recomputed by the oracle's FP64 operator is within the
    request's tolerance, and the large ones are bitwise the request solved
    alone."""
    spec = [(32, 1e-6), (1024, 1e-8), (2048, 1e-6), (32, 1e-8), (1024, 1e-6), (2048, 1e-8), (32, 1e-8),
            (1024, 1e-8)]
    reqs = []
    for k, (L, tol) in enumerate(spec):
        p = fc_inputs.problem(L, seed=4400 + k, b_kind="normal")
        reqs.append((L, tol, p["s"], p["b"]))
    sv = fc.cg_server_create(24 << 30, max_slots=4)
    outs = [np.zeros(L * L) for (L, *_rest) in reqs]
    tickets = [fc.cg_batch_submit(sv, L, s, b, x_out=o, rtol=tol, mode=fc.FC_MODE_MIXED, precond=True)
               for (L, tol, s, b), o in zip(reqs, outs)]
    res = wait_all(sv, tickets, timeout=300.0)
    sv.close()
    for (L, tol, s, b), o, t in zip(reqs, outs, tickets):
        r = res[t]
        assert r["status"] == fc.FC_OK and r["true_rel_resid"] <= tol
        rr = b - oracle.apply_A(L, s, o)
        rel = float(np.linalg.norm(rr) / np.linalg.norm(b))
        print(f"L={L} tol={tol:g}: oracle residual {rel:.3e}, {r['iters']} iterations")
        assert rel <= 1.01 * tol
    for k in (1, 2):
        L, tol, s, b = reqs[k]
        xa, ra = alone(L, s, b, tol, fc.FC_MODE_MIXED, precond=True)
        assert np.array_equal(outs[k], xa) and res[tickets[k]]["iters"] == ra["iters"]


def test_reserve_makes_plans_ahead():
    """cg_server_reserve makes a size's plans before any request (at most the
    plans per size, within the budget); requests then run on them, and a
    reservation that cannot fit the budget is refused."""
    sv = fc.cg_server_create(2 << 30, max_slots=2)
    fc.cg_server_reserve(sv, 64, 2)
    fc.cg_server_reserve(sv, 64, 5)  # capped at the plans per size
    st = fc.cg_server_stats(sv)
    assert st["plans"] == 2 and st["used"] > 0
    p = fc_inputs.problem(64, seed=3, b_kind="normal")
    o = np.zeros(64 * 64)
    r = wait_all(sv, [fc.cg_batch_submit(sv, 64, p["s"], p["b"], x_out=o, rtol=1e-8)])
    assert all(v["status"] == fc.FC_OK for v in r.values())
    assert fc.cg_server_stats(sv)["plans"] == 2
    xa, _ = alone(64, p["s"], p["b"], 1e-8, fc.FC_MODE_MIXED)
    assert np.array_equal(o, xa)
    sv.close()
    small = fc.cg_server_create(32 << 20, max_slots=1)
    with pytest.raises(fc.FcError) as ei:
        fc.cg_server_reserve(small, 1024, 1)  # about 110 MB of plan
    assert ei.value.code == fc.FC_EBUDGET
    small.close()
