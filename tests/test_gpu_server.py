"""The continuous-batching solve server (cg_server_*): results in a mix equal
the same requests solved alone, budget admission, polling."""
import time

import numpy as np
import pytest
import torch

import fc_inputs
import paper_1305_3625_b300 as fc
from gpu_util import dev, host

pytestmark = pytest.mark.gpu


def alone(L, s, b, rtol, mode):
    plan = fc.fftconv_plan_create(L)
    x = dev(np.zeros(L * L))
    r = fc.cg_solve(plan, dev(s), dev(b), x, rtol=rtol, mode=mode, x0_zero=True)
    return host(x), r


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


def test_many_small_requests_overlap():
    """Throughput with several slots exceeds one slot on many small solves."""
    L = 64
    probs = [fc_inputs.problem(L, seed=500 + k, b_kind="normal") for k in range(24)]

    def run(slots):
        sv = fc.cg_server_create(4 << 30, max_slots=slots)
        warm = fc.cg_batch_submit(sv, L, probs[0]["s"], probs[0]["b"], rtol=1e-8)
        wait_all(sv, [warm])
        t0 = time.perf_counter()
        ts = [fc.cg_batch_submit(sv, L, p["s"], p["b"], rtol=1e-8) for p in probs]
        wait_all(sv, ts)
        dt = time.perf_counter() - t0
        sv.close()
        return dt

    t1, t8 = run(1), run(8)
    assert t8 < t1
