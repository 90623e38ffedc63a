"""Benchmark of the fibre-bundle FFT-convolution CG solve on B300.

Workload (one "step"): one step of the quasi-static breaking loop on an
L = 1024 grid (padded 2048 x 2048 FFT): a CG solve of P (C + S) P x = P b,
warm-started from the previous solution, to a relative residual of 1e-10
(certified on the FP64 recomputed residual), followed by the removal of the
fibre with the largest |x_i| / t_i.  s ~ U[0.5, 1.5] (seed 0), b = 1,
t ~ U(0, 1).  The timed solves use the mixed path (FP32 FFTs and vectors,
FP64 reductions and FP64 true residuals driving refinement) with the Fourier
preconditioner; each solve's first true residual is the previous solve's
final FP64 residual with the exact rank-1 correction for the removed fibre,
and every later one (including the one that certifies convergence) is an
FP64 product.  The same steps are then re-run from the same state with the
plain FP64 path (Listing 2, first residual computed) and other variants for
the comparison, and the FFT-convolution matvec is timed on its own for the
roofline.

`python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]`
prints one JSON line.  Under torchrun each rank runs its own replica (seed =
rank): independent problems, no collective on the data path.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

os.environ.setdefault("OMP_NUM_THREADS", str(os.cpu_count() or 1))

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

L_BENCH = 1024
RTOL = 1e-10
# DRAM bytes (read + write) of the three FP32 passes of one L = 1024 apply, summed over the
# passes of one ncu capture (cold cache per launch; the writes stay in L2)
MATVEC_TRAFFIC_L1024 = 25.2e6
FRAC_GRADIENT = 2.0  # thresholds xi + 2 (iy + 1/2)/L in the fracture-run section
METRIC = "CG matvec GB/s vs HBM peak; solves/sec + p50/p99 latency, mixed vs FP64 plain"
WORKLOAD = ("quasi-static breaking loop, L=1024 (padded 2048^2 FFT): warm-started (preconditioned) CG to "
            "rtol 1e-10 + argmax |x|/t removal per step; s~U[0.5,1.5] seed 0, b=1, t~U(0,1)")


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6400.0, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(prefix="clk", suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [v.strip() for v in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for k, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(k)
        os.unlink(self.path)
        busy = [v for v in sm if v > 0.5 * (max(smax) if smax else 1)] or sm
        return {"sm_mhz": statistics.median(busy) if busy else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    pg = None
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if args.impl == "ours" else "gloo"
        dist.init_process_group(backend=backend)
        pg = dist
    return world, rank, local, pg


def aggregate_rate(units: float, local_ms: float, pg=None, device="cpu"):
    """Whole-job rate over the ranks of a replica run: units summed over
    ranks, time = the slowest rank's timed region.  Returns (rate per s,
    max ms, total units)."""
    if pg is None:
        return units / (local_ms * 1e-3), local_ms, units
    import torch
    import torch.distributed as dist
    t = torch.tensor([local_ms], dtype=torch.float64, device=device)
    u = torch.tensor([units], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(u.item()) / (float(t.item()) * 1e-3), float(t.item()), float(u.item())


# ---------------------------------------------------------------- oracle --

def cpu_model():
    try:
        with open("/proc/cpuinfo") as fh:
            for line in fh:
                if line.lower().startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


class OracleLoop:
    """The breaking loop of the bench workload run by the FP64 CPU oracle as
    it stands: each step a warm-started masked CG solve (Listing 2, plain
    FP64, first residual computed) to the bench's tolerance, then the
    removal of argmax |x|/t.  The first step starts from x = 0."""

    def __init__(self, L, seed):
        import fc_inputs
        self.L = L
        p = fc_inputs.problem(L, seed=seed, with_t=True)
        self.s, self.b, self.t = p["s"], p["b"], p["t"]
        self.x = np.zeros(L * L)
        self.mask = np.ones(L * L, dtype=np.uint8)
        self.steps = 0

    def step(self):
        import oracle
        t0 = time.perf_counter()
        x, rc, it, rel = oracle.cg(self.L, self.s, self.b, x0=self.x, mask=self.mask, rtol=RTOL)
        if rc != 0 or rel > RTOL:
            raise RuntimeError(f"oracle solve failed: rc={rc} rel={rel}")
        k, _ = oracle.argmax_ratio(x, self.t, self.mask)
        if k >= 0:
            self.mask[k] = 0
            x[k] = 0.0
        self.x = x
        self.steps += 1
        return time.perf_counter() - t0, it


# --------------------------------------------------------------- serving --

def pct(v, q):
    """q-quantile of the sorted list v (nearest rank)."""
    return v[min(len(v) - 1, max(0, int(math.ceil(q * len(v))) - 1))]


def serve_run(args, fc, fc_inputs, sv, drain, dev):
    """The serving workload: requests of L = 2^round(U[5,11]) with tolerances
    from {1e-6, 1e-8} (mixed, preconditioned), Poisson arrivals at 0.5, 0.7
    and 0.9 of the closed-loop capacity measured on the same mix.  Each
    request's s and b come from a pool of seeded problems of its size (16 per
    size: bounded host memory); its size, tolerance and arrival are its own.
    Also: the library's measured device high-water mark, plain FP64 CG and FP64
    PCG one request at a time on the capacity run's requests, and the oracle's
    residual of spot-checked results."""
    import torch
    import oracle
    n = args.serve_requests
    base = fc_inputs.request_stream(n, seed=777, rate_per_s=1.0)
    pool = {}
    for L in sorted({rq["L"] for rq in base}):
        pool[L] = [fc_inputs.problem(L, seed=777_000 + 97 * L + j, b_kind="normal") for j in range(16)]

    def prob(rq):
        return pool[rq["L"]][rq["k"] % 16]

    def submit(rq, x_out=None):
        pk = prob(rq)
        return fc.cg_batch_submit(sv, rq["L"], pk["s"], pk["b"], x_out=x_out, rtol=rq["tol"],
                                  mode=fc.FC_MODE_MIXED, precond=True, borrow=True)

    # the server's plans made ahead (two per size), then closed-loop capacity
    # (all submitted at once; the first round, untimed, grows the batch
    # workspaces and staging)
    for L in sorted(pool):
        fc.cg_server_reserve(sv, L, 2)
    ncap = min(len(base), args.serve_f64)
    mem0 = fc.fc_mem_stats(reset_peak=True)
    for timed in (False, True):
        c0 = time.perf_counter()
        drain([submit(rq) for rq in base[:ncap]])
        cap = ncap / (time.perf_counter() - c0)
    rates = []
    for rel in (0.5, 0.7, 0.9):
        stream_ = fc_inputs.request_stream(n, seed=777, rate_per_s=rel * cap)
        b0 = fc.cg_server_batches(sv)
        t0 = time.perf_counter()
        tickets = []
        for rq in stream_:
            while time.perf_counter() - t0 < rq["arrival_s"]:
                time.sleep(0.0001)
            tickets.append(submit(rq))
        res = drain(tickets)
        dt = time.perf_counter() - t0
        assert all(r["status"] == fc.FC_OK for r in res.values())
        lat = sorted(r["latency_s"] * 1e3 for r in res.values())
        by_l = {}
        for rq, tk in zip(stream_, tickets):
            by_l.setdefault(rq["L"], []).append(res[tk]["latency_s"] * 1e3)
        b1 = fc.cg_server_batches(sv)
        nb = max(b1["batches"] - b0["batches"], 1)
        rates.append({"rate_rel_capacity": rel, "rate_per_s": round(rel * cap, 1),
                      "solves_per_s": round(len(stream_) / dt, 2),
                      "p50_ms": round(pct(lat, 0.5), 3), "p99_ms": round(pct(lat, 0.99), 3),
                      "mean_batch": round((b1["solves"] - b0["solves"]) / nb, 2),
                      "p99_ms_by_L": {str(L): round(pct(sorted(v), 0.99), 2) for L, v in sorted(by_l.items())}})
    mem1 = fc.fc_mem_stats()
    st = fc.cg_server_stats(sv)
    # one request at a time on exactly the requests of the capacity run: plain
    # FP64 CG (Listing 2) and FP64 PCG, each from x = 0 to the request's tolerance
    f64 = {}
    for name, pre in (("f64_one_at_a_time", False), ("f64_pcg_one_at_a_time", True)):
        t64, lat64, plans64 = 0.0, [], {}
        for rq in base[:ncap]:
            Lq = rq["L"]
            if Lq not in plans64:
                plans64[Lq] = fc.fftconv_plan_create(Lq, fc.FC_F64)
            pk = prob(rq)
            sd, bd = torch.tensor(pk["s"], device=dev), torch.tensor(pk["b"], device=dev)
            xd = torch.zeros_like(sd)
            torch.cuda.synchronize()
            a0 = time.perf_counter()
            fc.cg_solve(plans64[Lq], sd, bd, xd, rtol=rq["tol"], mode=fc.FC_MODE_F64, x0_zero=True, precond=pre)
            xd.cpu()
            a1 = time.perf_counter()
            t64 += a1 - a0
            lat64.append((a1 - a0) * 1e3)
        f64[name] = {"requests": ncap, "solves_per_s": round(ncap / t64, 2),
                     "p50_ms": round(pct(sorted(lat64), 0.5), 3),
                     "mode": "plain FP64 CG (Listing 2)" if not pre else "FP64 PCG (same preconditioner)"}
        del plans64
    # spot checks: results of the first requests of the stream (closed loop,
    # outside the timed runs) against the oracle's FP64 residual b - (C + S) x
    nspot = min(args.serve_spot, len(base))
    outs = [np.zeros(rq["L"] ** 2) for rq in base[:nspot]]
    res = drain([submit(rq, o) for rq, o in zip(base[:nspot], outs)])
    worst = 0.0
    for rq, o in zip(base[:nspot], outs):
        pk = prob(rq)
        r = pk["b"] - oracle.apply_A(rq["L"], pk["s"], o)
        worst = max(worst, float(np.linalg.norm(r) / np.linalg.norm(pk["b"])) / rq["tol"])
    serving = {"requests_per_rate": n, "of_configuration": 20000,
               "inputs": "16 seeded problems per size, reused by the stream's requests",
               "capacity_per_s": round(cap, 1), "L": "2^round(U[5,11])", "tol": "{1e-6,1e-8}",
               "slots": args.slots, "rates": rates,
               "mem_peak_GB_measured": round((mem1["peak_bytes"] - mem0["live_bytes"]) / 1e9, 3),
               "mem_peak_GB_reserved": round(st["peak"] / 1e9, 2), "budget_GB": 150,
               "oracle_spot_checks": {"requests": nspot, "max_residual_over_tol": round(worst, 4)}}
    serving.update(f64)
    serving["capacity_vs_f64_one_at_a_time"] = round(cap / f64["f64_one_at_a_time"]["solves_per_s"], 2)
    serving["capacity_vs_f64_pcg_one_at_a_time"] = round(cap / f64["f64_pcg_one_at_a_time"]["solves_per_s"], 2)
    return serving


# ------------------------------------------------------------------ ours --

def run_ours(args, world, rank, local, pg):
    import torch

    import fc_inputs
    import paper_1305_3625_b300 as fc

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    L = L_BENCH
    N = L * L
    p = fc_inputs.problem(L, seed=rank, with_t=True)
    plan = fc.fftconv_plan_create(L, fc.FC_F32 | fc.FC_F64)
    s = torch.tensor(p["s"], device=dev)
    b = torch.tensor(p["b"], device=dev)
    t = torch.tensor(p["t"], device=dev)
    mask = torch.ones(N, device=dev, dtype=torch.uint8)
    x = torch.zeros(N, device=dev, dtype=torch.float64)
    removed = torch.empty(1, device=dev, dtype=torch.int64)
    flush = torch.empty(256 * 1024 * 1024 // 4, device=dev, dtype=torch.float32)  # > 126 MB L2

    def step(mode, x_, mask_, precond=True, warm_resid=True):
        r = fc.cg_solve(plan, s, b, x_, mask=mask_, rtol=RTOL, mode=mode, precond=precond, warm_resid=warm_resid)
        if r["status"] != fc.FC_OK:
            raise RuntimeError(f"solve failed: {r}")
        fc.fc_masked_step(plan, t, mask_, x_, removed)
        return r

    def launches(r, mode, precond=True):
        # warm-start check and residual update (every timed step follows a
        # finished solve), prologue (FP32 copy of s; preconditioner shift and
        # spectrum), per true residual 3 passes + final update, 3 passes per
        # product (6 per preconditioned iteration), 1 removal kernel
        pro = 2 + (1 if mode == fc.FC_MODE_MIXED else 0) + (2 if precond else 0)
        return pro + 4 * r["refinements"] + (6 if precond else 3) * r["iters"] + 1

    # warm-up: the cold first solve plus W-1 warm steps
    for _ in range(max(args.warmup, 3)):
        step(fc.FC_MODE_MIXED, x, mask)
    torch.cuda.synchronize()
    x_start, mask_start = x.clone(), mask.clone()

    def timed_loop(mode, K, precond=True, warm_resid=True):
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
        res = []
        for k in range(K):
            flush.zero_()
            ev[k][0].record(stream)
            res.append(step(mode, x, mask, precond, warm_resid))
            ev[k][1].record(stream)
        torch.cuda.synchronize()
        ms = [a.elapsed_time(bb) for a, bb in ev]
        return ms, res

    clocks = ClockSampler(local)
    if pg:
        pg.barrier()
    torch.cuda.synchronize()
    clocks.start()
    t0 = time.perf_counter()
    torch.cuda.nvtx.range_push("timed_solves")  # profilers select the timed region by this range
    ms_mixed, res_mixed = timed_loop(fc.FC_MODE_MIXED, args.steps)
    torch.cuda.nvtx.range_pop()
    wall_mixed = time.perf_counter() - t0
    torch.cuda.synchronize()
    if pg:
        pg.barrier()

    # the same steps from the same state: plain FP64 CG (Listing 2, the
    # baseline: every solve starts from a computed residual), FP64 with the
    # preconditioner, mixed without it, and the headline configuration with
    # the first residual recomputed instead of updated
    x.copy_(x_start)
    mask.copy_(mask_start)
    k64 = max(1, min(args.steps, args.f64_steps))
    ms_f64, res_f64 = timed_loop(fc.FC_MODE_F64, k64, precond=False, warm_resid=False)
    x.copy_(x_start)
    mask.copy_(mask_start)
    ms_f64p, res_f64p = timed_loop(fc.FC_MODE_F64, k64, precond=True)
    x.copy_(x_start)
    mask.copy_(mask_start)
    kmc = max(1, min(args.steps, 10))
    ms_mcg, res_mcg = timed_loop(fc.FC_MODE_MIXED, kmc, precond=False)
    x.copy_(x_start)
    mask.copy_(mask_start)
    ms_nou, res_nou = timed_loop(fc.FC_MODE_MIXED, kmc, warm_resid=False)

    # matvec roofline: FP32 fftconv_apply (3 passes).  Two measurements:
    # streamed, back-to-back applies over rotating (x, y) pairs whose total
    # exceeds the 126 MB L2 (each apply reads a cold x and writes a new y; the
    # spectrum and the intermediate are reused as in a solve), the roofline
    # figure; and one apply after a 256 MB L2-flushing write, for context.
    xin = torch.rand(N, device=dev, dtype=torch.float32)
    yout = torch.empty_like(xin)

    def time_apply(pl, xi, yo, reps):
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
        for _ in range(3):
            fc.fftconv_apply_prec(pl, fc.FC_F32, xi, yo)
        for a, bb in evs:
            flush.zero_()
            a.record(stream)
            fc.fftconv_apply_prec(pl, fc.FC_F32, xi, yo)
            bb.record(stream)
        torch.cuda.synchronize()
        return statistics.median(a.elapsed_time(bb) for a, bb in evs)

    def time_apply_streamed(pl, n, rounds=5):
        """Mean per apply over back-to-back applies cycling through pairs of
        (x, y) buffers totalling more than 3x the L2 (median of `rounds`
        runs, each over every pair twice); the pairs, and the number of
        applies per run."""
        npair = max(2, -(-3 * 126 * 2**20 // (8 * n)))
        xs = [torch.rand(n, device=dev, dtype=torch.float32) for _ in range(npair)]
        ys = [torch.empty_like(xs[0]) for _ in range(npair)]
        per = 2 * npair
        for k in range(npair):
            fc.fftconv_apply_prec(pl, fc.FC_F32, xs[k], ys[k])
        out = []
        for _ in range(rounds):
            a, bb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            for k in range(per):
                fc.fftconv_apply_prec(pl, fc.FC_F32, xs[k % npair], ys[k % npair])
            bb.record(stream)
            torch.cuda.synchronize()
            out.append(a.elapsed_time(bb) / per)
        del xs, ys
        return statistics.median(out), npair, per

    torch.cuda.nvtx.range_push("matvec")
    mv_flushed_ms = time_apply(plan, xin, yout, 50)
    mv_ms, mv_pairs, mv_per = time_apply_streamed(plan, N)
    torch.cuda.nvtx.range_pop()
    clk = clocks.stop()
    M = plan.M
    Q = M // 2 + 1
    # x, y (4N each), 4 passes over the L x M/2 half-spectrum intermediate (8N each), spectrum quarter
    mv_bytes = 40 * N + 4 * Q * Q
    peak, peak_kind = load_peaks()
    mv_gbs = mv_bytes / (mv_ms * 1e-3) / 1e9

    big = None
    large_loop = None
    if args.big:
        L4 = 4096
        plan4 = fc.fftconv_plan_create(L4, fc.FC_F32 | fc.FC_F64)
        x4 = torch.rand(L4 * L4, device=dev, dtype=torch.float32)
        y4 = torch.empty_like(x4)
        ms4f = time_apply(plan4, x4, y4, 20)
        del x4, y4
        ms4, np4, _ = time_apply_streamed(plan4, L4 * L4, rounds=3)
        Q4 = plan4.M // 2 + 1
        b4 = 40 * L4 * L4 + 4 * Q4 * Q4
        big = {"L": L4, "ms": round(ms4, 4), "bytes": b4, "GB_s": round(b4 / (ms4 * 1e-3) / 1e9, 1),
               "frac_of_hbm": round(b4 / (ms4 * 1e-3) / 1e9 / peak, 3),
               "timing": f"streamed: back-to-back applies over {np4} rotating x/y pairs (> L2)",
               "ms_after_l2_flush": round(ms4f, 4),
               "model_frac_c2c_88N": round(88 * L4 * L4 / (ms4 * 1e-3) / 1e9 / peak, 3),
               "model_note": "88 N bytes is the traffic of an unpacked C2C route; this packed route never moves them"}
        if args.big_steps > 0:
            # the large single instance: a cold mixed solve refined to 1e-8, then a
            # masked removal loop with t ~ U(0, 1) (fc_fracture_run)
            p4 = fc_inputs.problem(L4, seed=rank, with_t=True)
            s4, b4v, t4 = (torch.tensor(p4[k], device=dev) for k in ("s", "b", "t"))
            m4 = torch.ones(L4 * L4, device=dev, dtype=torch.uint8)
            xx4 = torch.zeros(L4 * L4, device=dev, dtype=torch.float64)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            rc4 = fc.cg_solve(plan4, s4, b4v, xx4, mask=m4, rtol=1e-8, mode=fc.FC_MODE_MIXED, precond=True)
            cold_s = time.perf_counter() - t0
            rem4 = torch.empty(args.big_steps, device=dev, dtype=torch.int64)
            fr4 = fc.fc_fracture_run(plan4, s4, b4v, t4, m4, xx4, args.big_steps, rem4, rtol=1e-8,
                                     mode=fc.FC_MODE_MIXED, precond=True)
            steps = max(fr4["steps_done"], 1)
            large_loop = {"L": L4, "rtol": 1e-8, "mode": "mixed, Fourier-preconditioned",
                          "cold_solve": {"s": round(cold_s, 4), "iters": rc4["iters"],
                                         "true_rel_resid": rc4["true_rel_resid"]},
                          "steps": fr4["steps_done"], "status": fr4["status"],
                          "steps_per_s": round(fr4["steps_done"] / fr4["seconds"], 2),
                          "iters_per_step": round(fr4["iters"] / steps, 2),
                          "fp64_products_per_step": round(fr4["fp64_products"] / steps, 2)}
            del s4, b4v, t4, m4, xx4, rem4
        del plan4

    # end-to-end through the C ABI with host buffers: inputs up, result down.
    # Every step uploads its inputs s, b and t from pinned host memory (one
    # step ahead, on a copy stream, into one of two device buffers) and
    # downloads its result: the field x, the mask and the removed index, from
    # a device snapshot taken right after the removal, on a second copy
    # stream, so that the download overlaps the next step.  x and the mask
    # are the loop's state and stay on the device between steps (uploaded
    # once, inside the timed region).
    e2e = None
    if args.e2e_steps > 0:
        hs = torch.tensor(p["s"]).pin_memory()
        hb = torch.tensor(p["b"]).pin_memory()
        ht = torch.tensor(p["t"]).pin_memory()
        hx0 = x_start.cpu().pin_memory()
        hm0 = mask_start.cpu().pin_memory()
        hx = [torch.empty_like(hx0).pin_memory() for _ in range(2)]
        hm = [torch.empty_like(hm0).pin_memory() for _ in range(2)]
        hrem = [torch.empty(1, dtype=torch.int64).pin_memory() for _ in range(2)]
        bufs = [(torch.empty_like(s), torch.empty_like(b), torch.empty_like(t)) for _ in range(2)]
        snap = [(torch.empty_like(x), torch.empty_like(mask), torch.empty_like(removed)) for _ in range(2)]
        up_stream = torch.cuda.Stream(device=dev)
        down_stream = torch.cuda.Stream(device=dev)
        ev_in = [torch.cuda.Event() for _ in range(2)]
        ev_used = [torch.cuda.Event() for _ in range(2)]
        ev_snap = [torch.cuda.Event() for _ in range(2)]
        ev_down = [torch.cuda.Event() for _ in range(2)]
        for ev in ev_used + ev_down:
            ev.record(stream)

        def stage(k):
            with torch.cuda.stream(up_stream):
                up_stream.wait_event(ev_used[k])
                for dbuf, hbuf in zip(bufs[k], (hs, hb, ht)):
                    dbuf.copy_(hbuf, non_blocking=True)
                ev_in[k].record(up_stream)

        torch.cuda.synchronize()
        e0 = time.perf_counter()
        ke = args.e2e_steps
        x.copy_(hx0, non_blocking=True)
        mask.copy_(hm0, non_blocking=True)
        stage(0)
        for i in range(ke):
            k = i & 1
            if i + 1 < ke:
                stage(k ^ 1)
            stream.wait_event(ev_in[k])
            ds, db, dt_ = bufs[k]
            r = fc.cg_solve(plan, ds, db, x, mask=mask, rtol=RTOL, mode=fc.FC_MODE_MIXED, precond=True)
            fc.fc_masked_step(plan, dt_, mask, x, removed)
            ev_used[k].record(stream)
            sx, sm, sr = snap[k]
            stream.wait_event(ev_down[k])  # the snapshot buffer's last download is done
            sx.copy_(x)
            sm.copy_(mask)
            sr.copy_(removed)
            ev_snap[k].record(stream)
            with torch.cuda.stream(down_stream):
                down_stream.wait_event(ev_snap[k])
                hx[k].copy_(sx, non_blocking=True)
                hm[k].copy_(sm, non_blocking=True)
                hrem[k].copy_(sr, non_blocking=True)
                ev_down[k].record(down_stream)
        torch.cuda.synchronize()
        e2e_s = time.perf_counter() - e0
        assert int(hrem[(ke - 1) & 1][0]) >= 0
        h2d = 3 * 8 * N
        d2h = 8 * N + N + 8
        e2e = {"value": round(ke / e2e_s, 3), "unit": "solves/s", "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h, "steps": ke,
               "state_upload_bytes_once": 8 * N + N,
               "pipeline": "inputs s, b, t up one step ahead; x, mask, removed index down from a device "
                           "snapshot during the next step; x and mask stay on the device"}

    # batched workload: 256 independent mixed solves, L ~ U{64,128,256,512},
    # b ~ N(0,1), rtol 1e-8, from x = 0: one cg_solve_groups call (one graph,
    # each size's batched solve a parallel branch of it); the same requests
    # through the solve server as a second figure
    batched = None
    batched_server = None
    serving = None
    sizes = [64, 128, 256, 512]
    rng_l = fc_inputs.uniform(12345, 0, max(args.batch_solves, 1))
    breqs = []
    for k in range(args.batch_solves):
        Lk = sizes[min(int(rng_l[k] * 4), 3)]
        pk = fc_inputs.problem(Lk, seed=10_000 + k, b_kind="normal")
        breqs.append((Lk, pk))
    if breqs:
        by_l = {}
        for Lk, pk in breqs:
            by_l.setdefault(Lk, []).append(pk)
        groups = []
        for Lk in sorted(by_l):
            ps = by_l[Lk]
            gp = fc.fftconv_plan_create(Lk, fc.FC_F32 | fc.FC_F64)
            gs = torch.tensor(np.stack([q["s"] for q in ps]), dtype=torch.float64, device="cuda")
            gb = torch.tensor(np.stack([q["b"] for q in ps]), dtype=torch.float64, device="cuda")
            gx = torch.zeros_like(gs)
            groups.append((gp, gs, gb, gx, None))
        kw = dict(rtol=1e-8, mode=fc.FC_MODE_MIXED, precond=True, x0_zero=True)
        fc.cg_solve_groups(groups, **kw)  # graphs built, buffers allocated
        times, res = [], None
        for _ in range(3):
            flush.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            rc, res = fc.cg_solve_groups(groups, **kw)
            times.append(time.perf_counter() - t0)
            assert rc == fc.FC_OK
        allr = [r for g in res for r in g]
        assert all(r["status"] == fc.FC_OK and r["true_rel_resid"] <= 1e-8 for r in allr)
        dt = statistics.median(times)
        # each size's batch alone (one cg_solve_batch call), for the split of the time
        per_size = {}
        for gp, gs, gb, gx, _ in groups:
            gx.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            fc.cg_solve_batch(gp, gs, gb, gx, **kw)
            per_size[str(gp.L)] = round(1e3 * (time.perf_counter() - t0), 2)
        # FP64 one solve at a time on a sample of the same requests (every
        # 8th), each from x = 0 to the same tolerance: plain CG (Listing 2) and
        # CG with the same preconditioner
        f64_plans, f64_t, f64p_t, f64_n = {}, 0.0, 0.0, 0
        for k in range(0, len(breqs), 8):
            Lk, pk = breqs[k]
            if Lk not in f64_plans:
                f64_plans[Lk] = fc.fftconv_plan_create(Lk, fc.FC_F64)
            s_, b_ = (torch.tensor(pk[n_], dtype=torch.float64, device="cuda") for n_ in ("s", "b"))
            for pre in (False, True):
                x_ = torch.zeros_like(s_)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                r = fc.cg_solve(f64_plans[Lk], s_, b_, x_, rtol=1e-8, mode=fc.FC_MODE_F64, x0_zero=True,
                                precond=pre)
                if pre:
                    f64p_t += time.perf_counter() - t0
                else:
                    f64_t += time.perf_counter() - t0
                assert r["status"] == fc.FC_OK
            f64_n += 1
        f64_rate = f64_n / f64_t
        f64p_rate = f64_n / f64p_t
        batched = {"solves": len(allr), "L": "U{64,128,256,512}", "groups": {str(g[0].L): int(g[3].shape[0])
                                                                          for g in groups},
                   "rtol": 1e-8, "mode": "mixed, Fourier-preconditioned, x0 = 0",
                   "launch": "cg_solve_groups: one graph launch, a batched solve per size as parallel branches",
                   "seconds": round(dt, 4), "seconds_runs": [round(t, 4) for t in times],
                   "ms_each_size_alone": per_size,
                   "solves_per_s": round(len(allr) / dt, 1),
                   "iters_mean": round(statistics.mean(r["iters"] for r in allr), 1),
                   "fp64_products_mean": round(statistics.mean(r["fp64_products"] for r in allr), 2),
                   "max_true_rel_resid": max(r["true_rel_resid"] for r in allr),
                   "f64_one_at_a_time": {"solves": f64_n, "solves_per_s": round(f64_rate, 1),
                                         "mode": "plain FP64 CG (Listing 2), x0 = 0"},
                   "vs_f64_one_at_a_time": round(len(allr) / dt / f64_rate, 1),
                   "f64_pcg_one_at_a_time": {"solves": f64_n, "solves_per_s": round(f64p_rate, 1),
                                             "mode": "FP64 CG with the same preconditioner, x0 = 0"},
                   "vs_f64_pcg_one_at_a_time": round(len(allr) / dt / f64p_rate, 1)}
        del groups, f64_plans
    if args.batch_solves > 0 or args.serve_requests > 0:
        sv = fc.cg_server_create(150 << 30, max_slots=args.slots)

        def drain(tickets, t_arrival=None):
            done, lat = {}, []
            while len(done) < len(tickets):
                progressed = False
                for t in tickets:
                    if t in done:
                        continue
                    r = fc.cg_poll(sv, t)
                    if r is not None:
                        done[t] = r
                        progressed = True
                if not progressed:
                    time.sleep(0.0002)
            return done

        if breqs:
            # the same 256 requests once untimed (plans, batch workspaces and
            # staging made), then timed
            drain([fc.cg_batch_submit(sv, Lk, pk["s"], pk["b"], rtol=1e-8, mode=fc.FC_MODE_MIXED, precond=True,
                                      borrow=True) for Lk, pk in breqs])
            bs0 = fc.cg_server_batches(sv)
            t0 = time.perf_counter()
            tk = [fc.cg_batch_submit(sv, Lk, pk["s"], pk["b"], rtol=1e-8, mode=fc.FC_MODE_MIXED, precond=True,
                                     borrow=True) for Lk, pk in breqs]
            res = drain(tk)
            dt = time.perf_counter() - t0
            assert all(r["status"] == fc.FC_OK for r in res.values())
            batched_server = {"solves": len(breqs), "L": "U{64,128,256,512}", "rtol": 1e-8, "mode": "mixed",
                       "slots": args.slots, "seconds": round(dt, 4), "solves_per_s": round(len(breqs) / dt, 2),
                       "iters_mean": round(statistics.mean(r["iters"] for r in res.values()), 1)}
            bs1 = fc.cg_server_batches(sv)
            batched_server["batches"] = bs1["batches"] - bs0["batches"]
        if args.serve_requests > 0:
            serving = serve_run(args, fc, fc_inputs, sv, drain, dev)
        sv.close()

    # a fracture run under a threshold gradient (fc_fracture_run): the
    # breaking loop driven inside the library, front read out at the end
    frac = None
    if args.frac_steps > 0:
        pg_ = fc_inputs.problem(L, seed=rank, with_t=True, t_gradient=FRAC_GRADIENT)
        fs, fb, ft = (torch.tensor(pg_[k], device=dev) for k in ("s", "b", "t"))
        fmask = torch.ones(N, device=dev, dtype=torch.uint8)
        fx = torch.zeros(N, device=dev, dtype=torch.float64)
        frem = torch.empty(args.frac_steps, device=dev, dtype=torch.int64)
        frat = torch.empty(args.frac_steps, device=dev, dtype=torch.float64)
        fr = fc.fc_fracture_run(plan, fs, fb, ft, fmask, fx, args.frac_steps, frem, frat, rtol=RTOL,
                                mode=fc.FC_MODE_MIXED, precond=True)
        fi = torch.empty(L, device=dev, dtype=torch.int32)
        de = torch.empty(L, device=dev, dtype=torch.int32)
        fc.fc_front(plan, fmask, fi, de)
        torch.cuda.synchronize()
        rows = (frem[:fr["steps_done"]] // L).float()
        frac = {"L": L, "t_gradient": FRAC_GRADIENT, "steps": fr["steps_done"], "status": fr["status"],
                "steps_per_s": round(fr["steps_done"] / fr["seconds"], 2),
                "iters_per_step": round(fr["iters"] / max(fr["steps_done"], 1), 2),
                "fp64_products_per_step": round(fr["fp64_products"] / max(fr["steps_done"], 1), 2),
                "mean_broken_row": round(float(rows.mean()), 2) if fr["steps_done"] else None,
                "front_first_intact_mean": round(float(fi.float().mean()), 3),
                "front_damage_end_mean": round(float(de.float().mean()), 3),
                "load_1_over_ratio_first_last": [round(1.0 / float(frat[0]), 6),
                                                 round(1.0 / float(frat[fr["steps_done"] - 1]), 6)]
                if fr["steps_done"] else None}
        del fs, fb, ft, fmask, fx

    # an ensemble of breaking runs (fc_fracture_run_batch): independent
    # samples of the model in lockstep, against one run at a time
    ensemble = None
    if args.ensemble_runs > 0 and args.frac_steps > 0:
        Le, ne, se = 128, args.ensemble_runs, 50
        pe = [fc_inputs.problem(Le, seed=3000 + k, with_t=True, t_gradient=FRAC_GRADIENT) for k in range(ne)]
        st_ = lambda key: torch.tensor(np.stack([q[key] for q in pe]), device=dev)
        es, eb, et = st_("s"), st_("b"), st_("t")
        eplan = fc.fftconv_plan_create(Le, fc.FC_F32 | fc.FC_F64)
        kw = dict(rtol=RTOL, mode=fc.FC_MODE_MIXED, precond=True)

        def ens_run():
            em = torch.ones(ne * Le * Le, device=dev, dtype=torch.uint8)
            ex_ = torch.zeros(ne * Le * Le, device=dev, dtype=torch.float64)
            er = torch.empty(ne * se, device=dev, dtype=torch.int64)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            rc_, rr = fc.fc_fracture_run_batch(eplan, es, eb, et, em, ex_, se, er, **kw)
            return time.perf_counter() - t0, rc_, rr

        ens_run()  # graphs and workspaces made
        torch.cuda.nvtx.range_push("ensemble")
        et_s, erc, err_ = ens_run()
        torch.cuda.nvtx.range_pop()
        assert erc == fc.FC_OK
        # one run at a time, on the first runs of the same ensemble
        n1, t1 = min(4, ne), 0.0
        for k in range(n1):
            m1 = torch.ones(Le * Le, device=dev, dtype=torch.uint8)
            x1 = torch.zeros(Le * Le, device=dev, dtype=torch.float64)
            r1 = torch.empty(se, device=dev, dtype=torch.int64)
            fr1 = fc.fc_fracture_run(eplan, es[k], eb[k], et[k], m1, x1, se, r1, **kw)
            t1 += fr1["seconds"]
        ensemble = {"runs": ne, "L": Le, "steps_per_run": se, "t_gradient": FRAC_GRADIENT,
                    "mode": "mixed, Fourier-preconditioned", "seconds": round(et_s, 4),
                    "removal_steps_per_s": round(sum(r["steps_done"] for r in err_) / et_s, 1),
                    "iters_per_step": round(sum(r["iters"] for r in err_) / max(sum(r["steps_done"] for r in err_), 1), 2),
                    "one_run_at_a_time_steps_per_s": round(n1 * se / t1, 1),
                    "vs_one_at_a_time": round(sum(r["steps_done"] for r in err_) / et_s / (n1 * se / t1), 1)}
        del eplan

    # aggregate over ranks: units summed, slowest rank's time
    value, tot_ms, _ = aggregate_rate(args.steps, sum(ms_mixed), pg, dev)

    out = None
    if rank == 0:
        srt = sorted(ms_mixed)

        iters = [r["iters"] for r in res_mixed]
        iters64 = [r["iters"] for r in res_f64]
        f64_rate = k64 / (sum(ms_f64) * 1e-3)
        # the oracle on the host cores: whole steps of the same loop (the cold
        # first step, then timed warm-started steps while the budget lasts)
        cpu = OracleLoop(L, seed=rank)
        cold_s, cold_it = cpu.step()
        cpu_times, cpu_its = [], []
        while not cpu_times or (sum(cpu_times) < args.cpu_budget and len(cpu_times) < 5):
            dt_, it_ = cpu.step()
            cpu_times.append(dt_)
            cpu_its.append(it_)
        out = {
            "metric": METRIC,
            "value": round(value, 3),
            "unit": "solves/s",
            "n_gpus": world,
            "steps": args.steps,
            "warmup": max(args.warmup, 3),
            "ms_per_step": round(tot_ms / args.steps, 4),
            "higher_is_better": True,
            "scaling": "weak",
            "vs_baseline": None,
            "dtype": "f32+f64 (mixed: FP32 FFT/vectors, FP64 reductions and true residuals)",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "L": L, "M": M, "rtol": RTOL,
                       "mode": "mixed FP32/FP64, Fourier-preconditioned CG",
                       "l2": "flushed between steps (256 MB write)", "parallelism": f"replicas x{world}"},
            "p50_ms": round(pct(srt, 0.5), 4),
            "p99_ms": round(pct(srt, 0.99), 4),
            "iters_per_solve": round(statistics.mean(iters), 2),
            "true_residuals_per_solve": round(statistics.mean(r["refinements"] for r in res_mixed), 2),
            "fp64_products_per_solve": round(
                statistics.mean(r["fp64_products"] for r in res_mixed), 2),
            "first_residual_updated": round(statistics.mean(r["resid_updated"] for r in res_mixed), 2),
            "f64_plain": {"value": round(f64_rate, 3), "unit": "solves/s", "steps": k64,
                          "p50_ms": round(statistics.median(ms_f64), 3),
                          "p99_ms": round(max(ms_f64), 3),
                          "iters_per_solve": round(statistics.mean(iters64), 2)},
            "mixed_over_f64": round(value / world / f64_rate, 2),
            "mixed_over_f64_pcg": round(value / world / (k64 / (sum(ms_f64p) * 1e-3)), 2),
            "f64_pcg": {"value": round(k64 / (sum(ms_f64p) * 1e-3), 3), "unit": "solves/s",
                        "iters_per_solve": round(statistics.mean(r["iters"] for r in res_f64p), 2)},
            "mixed_cg_no_precond": {"value": round(kmc / (sum(ms_mcg) * 1e-3), 3), "unit": "solves/s",
                                    "iters_per_solve": round(statistics.mean(r["iters"] for r in res_mcg), 2),
                                    "true_residuals_per_solve": round(
                                        statistics.mean(r["refinements"] for r in res_mcg), 2)},
            "mixed_pcg_first_residual_recomputed": {
                "value": round(kmc / (sum(ms_nou) * 1e-3), 3), "unit": "solves/s",
                "p50_ms": round(statistics.median(ms_nou), 4),
                "iters_per_solve": round(statistics.mean(r["iters"] for r in res_nou), 2)},
            "matvec": {"L": L, "ms": round(mv_ms, 4), "bytes": mv_bytes, "GB_s": round(mv_gbs, 1),
                       "frac_of_hbm": round(mv_gbs / peak, 3),
                       "timing": f"streamed: {mv_per} back-to-back applies over {mv_pairs} rotating x/y pairs "
                                 f"({mv_pairs * 8 * N / 2**20:.0f} MB > L2), median of 5",
                       "ms_after_l2_flush": round(mv_flushed_ms, 4),
                       "frac_after_l2_flush": round(mv_bytes / (mv_flushed_ms * 1e-3) / 1e9 / peak, 3),
                       "model_frac_c2c_88N": round(88 * N / (mv_ms * 1e-3) / 1e9 / peak, 3),
                       "model_note": "88 N bytes is the traffic of an unpacked C2C route; this packed route "
                                     "never moves them"},
            "matvec_L4096": big,
            "large_loop_L4096": large_loop,
            "batched": batched,
            "fracture_ensemble": ensemble,
            "batched_server": batched_server,
            "serving": serving,
            "roofline": {"bound": "hbm", "kernel": "fftconv_apply FP32 (3 passes), L=1024",
                         "achieved": round(mv_gbs, 1), "peak": peak, "unit": "GB/s",
                         "frac": round(mv_gbs / peak, 3), "traffic": args.traffic,
                         "timing": "streamed applies, inputs larger than L2 (matvec.timing)",
                         "peak_kind": peak_kind},
            "cpu_baseline": {"value": round(len(cpu_times) / sum(cpu_times), 5), "unit": "solves/s",
                             "cores": int(os.environ.get("OMP_NUM_THREADS", "1")), "cpu_model": cpu_model(),
                             "kind": "oracle",
                             "sample": (f"whole steps of the same breaking loop at L={L} by the FP64 oracle "
                                        f"(plain CG to rtol {RTOL:g}, warm-started, + removal): steps 2-"
                                        f"{1 + len(cpu_times)} timed ({sum(cpu_times):.1f} s, "
                                        f"{statistics.mean(cpu_its):.0f} iterations each) after the cold "
                                        f"first step ({cold_s:.1f} s, {cold_it} iterations)")},
            "e2e": e2e,
            "fracture_run": frac,
            "pass_shapes_L1024": {
                "apply_f32": fc.fftconv_plan_shape_set(plan, fc.FC_F32, fc.FC_SHAPES_APPLY),
                "solve_f32": fc.fftconv_plan_shape_set(plan, fc.FC_F32, fc.FC_SHAPES_SOLVE),
                "f64": fc.fftconv_plan_shape_set(plan, fc.FC_F64, fc.FC_SHAPES_SOLVE)},
            "gpu_launches": sum(launches(r, fc.FC_MODE_MIXED) for r in res_mixed),
            "clocks": clk,
            "wall_s_timed_region": round(wall_mixed, 3),
        }
    return out


def run_reference(args, world, rank):
    """The oracle, as it stands, on the host cores: W untimed and K timed
    whole steps of the bench's breaking loop (each a warm-started FP64 CG
    solve to rtol 1e-10 plus the removal; the first warm-up step is the cold
    solve from x = 0).  Rank 0 alone runs it."""
    if rank != 0:
        return None
    L = L_BENCH
    loop = OracleLoop(L, seed=0)
    for _ in range(args.warmup):
        loop.step()
    ms, its = [], []
    t0 = time.perf_counter()
    for _ in range(args.steps):
        dt, it = loop.step()
        ms.append(dt * 1e3)
        its.append(it)
    wall = time.perf_counter() - t0
    value = len(ms) / (sum(ms) * 1e-3)
    cores = int(os.environ.get("OMP_NUM_THREADS", "1"))
    sample = (f"{args.steps} whole steps of the breaking loop at L={L} after {args.warmup} warm-up steps: "
              f"warm-started oracle FP64 CG (Listing 2) to rtol {RTOL:g} + removal, "
              f"{statistics.mean(its):.1f} iterations per solve")
    return {"impl": "reference", "metric": METRIC, "value": round(value, 6), "unit": "solves/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(statistics.mean(ms), 3), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "L": L, "rtol": RTOL, "mode": "oracle FP64 CG (CPU), plain"},
            "p50_ms": round(statistics.median(ms), 3),
            "cpu_baseline": {"value": round(value, 6), "unit": "solves/s", "cores": cores,
                             "cpu_model": cpu_model(), "kind": "oracle", "sample": sample},
            "e2e": {"value": round(value, 6), "unit": "solves/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0},
            "wall_s_timed_region": round(wall, 3)}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--f64-steps", type=int, default=6, dest="f64_steps")
    ap.add_argument("--e2e-steps", type=int, default=100, dest="e2e_steps")
    ap.add_argument("--cpu-budget", type=float, default=12.0, dest="cpu_budget",
                    help="seconds of timed warm oracle steps in the cpu_baseline leg (at least one step)")
    ap.add_argument("--big", type=int, default=1)
    ap.add_argument("--big-steps", type=int, default=200, dest="big_steps")
    ap.add_argument("--frac-steps", type=int, default=100, dest="frac_steps")
    ap.add_argument("--ensemble-runs", type=int, default=64, dest="ensemble_runs")
    ap.add_argument("--batch-solves", type=int, default=256, dest="batch_solves")
    ap.add_argument("--serve-requests", type=int, default=2000, dest="serve_requests",
                    help="requests per arrival rate of the serving run (configuration: 20000)")
    ap.add_argument("--serve-spot", type=int, default=200, dest="serve_spot",
                    help="served results checked against the oracle's residual")
    ap.add_argument("--serve-f64", type=int, default=160, dest="serve_f64",
                    help="requests of the serving mix solved closed-loop and by one-at-a-time FP64")
    ap.add_argument("--slots", type=int, default=8)
    ap.add_argument("--traffic", type=float, default=MATVEC_TRAFFIC_L1024,
                    help="ncu dram bytes per matvec from a capture of the current kernels")
    args = ap.parse_args()
    if args.impl == "reference":
        # the oracle on rank 0's host cores; other ranks have no work
        out = run_reference(args, int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")))
        if out is not None:
            print(json.dumps(out), flush=True)
        return
    world, rank, local, pg = dist_setup(args)
    out = run_ours(args, world, rank, local, pg)
    if out is not None:
        print(json.dumps(out), flush=True)
    if pg:
        pg.barrier()
        pg.destroy_process_group()


if __name__ == "__main__":
    main()
