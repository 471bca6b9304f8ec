#!/usr/bin/env python3
"""Benchmark: box evaluations per second of the GPU interval branch and bound.

The default line measures the largest single-GPU workload (mixed10k below)
and nests the figures of the n = 100 chain workload (chain100) and of the
serving stream (serving) under its config, so one run reports every part of
the metric: box-evals/s, served solves/s against one-at-a-time FP64 solves
at width 1e-6, and p50/p99 latency.

Workloads (one "step" = one complete solve, every row of the hot path):

mixed10k (default)
  n = 10,000: separable cosine terms on even i, chain terms on odd i, box
  [-5.12, 5.12]^n, width 1e-6, FP32 prefilter + FP64, blocks of 100, 2^10
  children of one box per generation, block-record box pool.
chain100
  coupled quartic chain, n = 100, seed 0 (synthetic.chain): alpha~U[50,150],
  beta~U[0.5,2], s~U[-1,2], box [-5,10]^100, min f = 0 at the planted s,
  enclosure width target 1e-6, FP64, variable cycling over blocks of 10
  coordinates with the paper's partition: the 10 coordinates of the block cut
  into 4 pieces each (4^10 = 1,048,576 children), one selected box per
  generation (best-first).
ackley1000
  shifted Ackley-type family, n = 1000, box [-32.768, 32.768]^1000, width
  1e-6, FP32 prefilter + FP64, blocks of 10, 2^10 children of one box per
  generation, 16 generations per host synchronisation (CUDA graphs).
levy50_paper
  the paper's own procedure on its Levy function (Eq. S11-S13), n = 50: 4^10
  children of one region per iteration, 10 diagonal GUB samples, first-order
  test on every coordinate, region width 1e-4; metric = solve time, compared
  with the time the paper prints for it (Table 2).
paper (--family F --n N [--pool-mode 2])
  the same procedure on any of the paper's functions (SI Appendix A, F) at
  any n; compared with the cloud-server time the paper prints for (F, N)
  when it prints one (Table 2, Tables S2-S10, S14).
serving
  512 requests, Poisson arrivals (20/s), n log-uniform on [2, 2000], family
  uniform over sep_cos / chain / ackley, width 1e-6, 150 GB pool budget:
  served solves/s and p50/p99 latency against one-at-a-time FP64 solves.

value      box evaluations (F + interval gradient + first-order test, FP64 and
           FP32 children) per second over the timed solves, problem and
           coefficients resident on the device, device time from CUDA events
           on the library's stream.
e2e        the same metric through the public C ABI from host buffers:
           gb_create_problem (DAG, tables and bounds copied host -> device),
           gb_solve (boxes and trace copied device -> host), gb_destroy_problem.
roofline   the child evaluation (per-parent term tables and child kernels,
           FP64 or FP32, whichever takes longer): directed-rounding
           operations they execute (counted in the kernels: the static
           per-instruction costs of every instruction run) per second of
           their CUDA-event time, against the pipe rate of the chip at the
           sampled SM clock (FP64: 2 operations per SM per clock; FP32: 128)
           times the SM count read from the device.  Workloads that replay
           generations from CUDA graphs time the kernels on one extra solve
           with a host synchronisation per generation (per-kernel events).
cpu_baseline / --impl reference
           the CPU oracle (plain C, fesetround) on the host cores, one thread
           and one thread per core, on a bounded sample of the same workload.

Under torchrun (N > 1) every rank solves its own replica (seed = rank): the
solves are independent, there is no collective on the data path.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import tempfile
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synthetic as S  # noqa: E402

FP64_OPS_PER_SM_CLK = 2.0    # GB300: 1.25 TFLOP/s FP64 (FMA = 2) at 2.07 GHz over 152 SMs
FP32_OPS_PER_SM_CLK = 128.0  # 128 FP32 lanes per SM (directed add / mul at full rate)
WORKLOADS = {
    "chain100": dict(family="chain", n=100, block=10, split_m=4, split_d=10, max_children=1 << 20, fp32=0,
                     gens_per_sync=0, pool_gb=16.0, cpu_parents=4, cpu_split_m=2, cpu_split_d=10, cpu_gens=20,
                     # DRAM bytes (read + write) of one k_eval64_tab launch, ncu capture in
                     # profiles/k_eval64_tab_chain100.md
                     traffic=0.645e6,
                     name="chain n=100 (coupled quartic, planted min 0), FP64, B=10, 4-way split of the 10 "
                          "block coordinates (4^10 children) of 1 best box per generation, tol_f=1e-6"),
    "ackley1000": dict(family="ackley", n=1000, block=10, split_m=2, split_d=10, max_children=1 << 10, fp32=1,
                       gens_per_sync=16, pool_gb=32.0, cpu_parents=1, cpu_split_m=2, cpu_split_d=10, cpu_gens=12,
                       name="ackley n=1000 (exp/sqrt/cos mean form + quadratic, planted min 0), FP32 "
                            "prefilter + FP64, B=10, 2-way split of 10 coordinates of 1 best box per generation, "
                            "tol_f=1e-6"),
    "mixed10k": dict(family="mixed", n=10000, block=100, split_m=2, split_d=10, max_children=1 << 10, fp32=1,
                     gens_per_sync=16, pool_gb=64.0, cpu_parents=1, cpu_split_m=2, cpu_split_d=10, cpu_gens=2,
                     name="mixed n=10000 (separable cosine terms on even i, chain terms on odd i, planted min 0), "
                          "FP32 prefilter + FP64, B=100, 2-way split of 10 coordinates of 1 best box per "
                          "generation, block-record pool, tol_f=1e-6"),
    "levy50_paper": dict(family="paper_levy", n=50, block=10, split_m=4, split_d=10, max_children=1 << 20, fp32=0,
                         gens_per_sync=0, pool_gb=16.0, cpu_parents=1, cpu_split_m=4, cpu_split_d=5, cpu_gens=2,
                         paper=True, baseline_s=15.0, paper_iters=45,
                         name="the paper's procedure on Levy n=50 (Eq. S11-S13): 4-way split of the 10 block "
                              "coordinates (4^10 children) of 1 best region per iteration, 10 diagonal samples, "
                              "first-order test on every coordinate, region width tolerance 1e-4"),
}


# The paper's procedure: iterations per block of 10 coordinates and the
# cloud-server (GH200) solve times it prints, by function and n (Table 2,
# Tables S2-S10, S14).
PAPER_PRINTED = {
    "paper_levy": (9, {50: 15, 100: 42, 500: 909, 1000: 3582, 2000: 14543, 5000: 93447, 10000: 376589}),
    "paper_ackley": (10, {50: 11, 100: 29, 500: 565, 1000: 2288}),
    "paper_belegundu": (9, {50: 6, 100: 15, 500: 426, 1000: 1896}),
    "paper_breiman": (8, {50: 5, 100: 13, 500: 301, 1000: 1218}),
    "paper_fu": (9, {50: 13, 100: 41, 500: 892, 1000: 3538}),
    "paper_griewank": (11, {50: 9, 100: 28, 500: 605, 1000: 2523}),
    "paper_rastrigin": (9, {50: 6, 100: 18, 500: 400, 1000: 1727}),
    "paper_salomon": (11, {50: 5, 100: 12, 500: 328, 1000: 1435}),
    "paper_styblinski": (9, {50: 7, 100: 21, 500: 419, 1000: 1791}),
    "paper_zabinsky": (8, {50: 9, 100: 26, 500: 619, 1000: 2635}),
    "paper_discontinuous": (9, {50: 35, 100: 114, 500: 2527, 1000: 9928}),
}


def _paper_workload(family, n, pool_mode, pool_gb):
    per_block, times = PAPER_PRINTED[family]
    return dict(family=family, n=n, block=10, split_m=4, split_d=10, max_children=1 << 20, fp32=0,
                gens_per_sync=0, pool_gb=pool_gb or 32.0, pool_mode=pool_mode, cpu_parents=1, cpu_split_m=4,
                cpu_split_d=5, cpu_gens=2, paper=True, baseline_s=times.get(n), paper_iters=per_block * n // 10,
                name=f"the paper's procedure on {family[6:]} n={n}: 4-way split of the 10 block coordinates "
                     "(4^10 children) of 1 best region per iteration, 10 diagonal samples, first-order test "
                     "on every coordinate, region width tolerance 1e-4"
                     + (", block-record pool" if pool_mode == 2 else ""))


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb", choices=["gb", "reference"])
    ap.add_argument("--workload", default="mixed10k", choices=sorted(WORKLOADS) + ["serving", "paper"])
    ap.add_argument("--family", default="paper_levy", choices=sorted(PAPER_PRINTED),
                    help="paper workload: the function")
    ap.add_argument("--n", type=int, default=50, help="paper workload: the dimension")
    ap.add_argument("--pool-mode", type=int, default=0, help="paper workload: 2 for block records")
    ap.add_argument("--max-children", type=int, default=0, help="children per generation (0: the workload's)")
    ap.add_argument("--eval-mode", type=int, default=-1, help="child evaluation kernels (gb_options.eval_mode; "
                    "-1: the workload's)")
    ap.add_argument("--split-m", type=int, default=0, help="pieces per split coordinate (0: the workload's)")
    ap.add_argument("--split-d", type=int, default=0, help="coordinates split per generation (0: the workload's)")
    ap.add_argument("--no-nested", action="store_true",
                    help="default workload: leave out the nested chain100 and serving figures")
    ap.add_argument("--no-serving", action="store_true", help="default workload: leave out the serving figures")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-gens", type=int, default=0, help="generations in the oracle sample (0: the workload's)")
    ap.add_argument("--pool-gb", type=float, default=0.0, help="device memory for the box pool (0: the workload's)")
    ap.add_argument("--max-gens", type=int, default=0, help="stop each solve after this many generations")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--requests", type=int, default=512)
    ap.add_argument("--n-max", type=int, default=2000)
    ap.add_argument("--autotune", action="store_true",
                    help="serving: tune fan-out / parents / kernel shape per family and n range first")
    return ap.parse_args()


def _workload(a):
    if a.workload == "paper":
        return _paper_workload(a.family, a.n, a.pool_mode, a.pool_gb)
    return WORKLOADS[a.workload if a.workload in WORKLOADS else "mixed10k"]


def _problem(w, seed=0):
    if w["family"].startswith("paper_"):   # the paper's functions are fixed (no seed)
        return S.make(w["family"], n=w["n"])
    return S.make(w["family"], n=w["n"], seed=seed)


class ClockSampler:
    """nvidia-smi sampling of SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        # raw samples: BENCH_CLOCKS_DIR if set, else a temporary directory
        d = os.environ.get("BENCH_CLOCKS_DIR") or tempfile.mkdtemp(prefix="gb_clocks_")
        self.path = os.path.join(d, f"clocks_rank{index}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for name, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        if not sm:
            return None
        load = [v for v in sm if v > 0.5 * max(sm)] or sm
        return {"sm_mhz": statistics.median(load), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def flush_l2(torch, dev, buf):
    buf.add_(1.0)          # 512 MB written: larger than the 129 MB L2
    torch.cuda.synchronize(dev)


def host_cpu():
    """The host's processor (model or part, architecture, logical cores)."""
    import platform
    model = ""
    try:
        with open("/proc/cpuinfo") as fh:
            for line in fh:
                key = line.split(":")[0].strip().lower()
                if key in ("model name", "cpu part") and ":" in line:
                    model = line.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    return f"{model or platform.processor() or 'unknown'} ({platform.machine()}, {os.cpu_count()} logical cores)"


def cpu_baseline(w, gens, threads=1):
    """Oracle on the workload's problem: the first `gens` generations with
    2^d children per parent (d = the workload's split width) and the
    workload's FP32 setting, its per-child passes on `threads` threads.
    Every child costs what a child of the timed workload costs (same block,
    same terms re-evaluated, same first-order test); only the batching
    differs, which keeps the sample to seconds."""
    import oracle
    p = _problem(w, 0)
    o = oracle.Oracle(p, block=w["block"])
    t = time.perf_counter()
    paper = dict(samples=10, mono_all=True, tol_x=1e-4) if w.get("paper") else {}
    r = o.solve(split_m=w["cpu_split_m"], split_d=w["cpu_split_d"], max_parents=w["cpu_parents"], max_gen=gens,
                fp32=bool(w["fp32"]), threads=threads, **paper)
    dt = time.perf_counter() - t
    evals = r.evals64 + r.evals32
    return {"value": evals / dt, "unit": "box-evals/s", "cores": threads, "kind": "oracle", "host": host_cpu(),
            "sample": f"first {r.generations} generations of the {w['family']} n={w['n']} solve, "
                      f"{w['cpu_parents']} parents x {w['cpu_split_m'] ** w['cpu_split_d']} children per "
                      f"generation ({evals} box evaluations, {dt:.1f} s, {threads} thread"
                      f"{'s' if threads > 1 else ''})"}


def cpu_baseline_both(w, gens):
    """The oracle with one thread per host core (the reported value) and on
    one thread (beside it), each on a bounded sample of the workload."""
    cores = os.cpu_count() or 1
    multi = cpu_baseline(w, gens, threads=cores)
    single = cpu_baseline(w, max(1, gens // 2), threads=1)
    multi["single_thread"] = {k: single[k] for k in ("value", "cores", "sample")}
    return multi


def run_reference(a):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    oracle.build()
    w = _workload(a)
    gens = a.cpu_gens or w["cpu_gens"]
    cores = os.cpu_count() or 1
    vals = []
    for i in range(a.warmup):
        cpu_baseline(w, 1, threads=cores)
    for i in range(a.steps):
        vals.append(cpu_baseline(w, max(1, gens // 2), threads=cores))
    v = statistics.median([x["value"] for x in vals])
    metric, unit, hib, note = "box-evals/s", "box-evals/s", True, None
    if w.get("paper"):
        # the procedure fixes the work of a solve: iterations x 4^10 children
        metric, unit, hib = "solve time", "s", False
        v = w["paper_iters"] * w["split_m"] ** w["split_d"] / v
        note = (f"extrapolated: {w['paper_iters']} iterations x {w['split_m'] ** w['split_d']} children "
                "at the sampled oracle rate")
    line = {"impl": "reference", "metric": metric, "value": v, "unit": unit,
            "n_gpus": a.gpus, "steps": a.steps, "warmup": a.warmup, "ms_per_step": None,
            "higher_is_better": hib, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+f64" if w["fp32"] else "f64",
            "data": "synthetic", "config": {"workload": w["name"], "note": note},
            "cpu_baseline": {"kind": "oracle", "cores": cores, "sample": vals[0]["sample"], "value": v,
                             "host": vals[0]["host"]},
            "e2e": {"value": v, "unit": unit, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def _serving_opts(gb, p, fp32):
    """One best box per generation (2^B children, B = min(n, 10)): the dive
    keeps each request's pool small and its generations short; the GPU is
    filled by the concurrent requests."""
    B = min(p.n, 10)
    return gb.gb_default_options(block=B, split_m=2, split_d=B, max_children=1 << 10,
                                 fp32_prefilter=int(fp32), pool_bytes=4 << 30, gens_per_sync=4)


N_BUCKETS = (8, 32, 128, 512, 1 << 30)


def _bucket(p):
    return p.family, next(i for i, b in enumerate(N_BUCKETS) if p.n < b)


def _bucket_name(key):
    fam, i = key
    lo = N_BUCKETS[i - 1] if i else 2
    return f"{fam} n>={lo}" if i == len(N_BUCKETS) - 1 else f"{fam} {lo}<=n<{N_BUCKETS[i]}"


def _tune_serving(gb, stream, budget_ms=1500.0):
    """gb_autotune on the first request of every (family, n range) bucket."""
    tuned, t0 = {}, time.perf_counter()
    for _, p in stream:
        key = _bucket(p)
        if key in tuned:
            continue
        best, ms = gb.gb_autotune(p, budget_ms=budget_ms, base=_serving_opts(gb, p, True))
        fan = best.split_m ** best.split_d
        # relative to the block, so that it applies to every n of the bucket
        tuned[key] = (dict(split_m=best.split_m, half_block=best.split_d < best.block,
                           parents=best.max_children // fan, eval_mode=best.eval_mode), ms)
    return tuned, time.perf_counter() - t0


def serving_block(a):
    """Stream of minimisation requests served with continuous batching
    (FP32 prefilter + FP64) against the same problems solved one at a time in
    FP64 on the same GPU.

    Phase 1: Poisson arrivals, served: per-request latency (submit -> result,
             host clock), observed.
    Phase 2: the same problems one at a time (FP64): service times; their
             latencies under the same arrival times follow from a FIFO queue
             model (computed, not observed).
    Phase 3: saturation -- every request submitted at once -- for the served
             capacity (solves/s), per-request CUDA graphs and fused steps,
             against the sum of the one-at-a-time times.
    Also: the enclosure widths of the FP32-prefilter results beside those of
    the FP64-only solves of the same problems, per family."""
    import paper_2507_01770_gb300 as gb
    gb.load()
    stream = S.serving_stream(count=a.requests, seed=0, rate=20.0, n_min=2, n_max=a.n_max, tol_f=1e-6)
    arrivals = np.array([t for t, _ in stream]) - stream[0][0]
    tuned, tune_s = _tune_serving(gb, stream) if a.autotune else ({}, 0.0)

    def served_opts(p):
        o = _serving_opts(gb, p, True)
        t = tuned.get(_bucket(p))
        if t:
            t = t[0]
            o.split_m = t["split_m"]
            o.split_d = (o.block + 1) // 2 if t["half_block"] else o.block
            if o.split_m == 4 and o.split_d > 10:
                o.split_d = 10
            o.max_children = t["parents"] * t["split_m"] ** o.split_d
            o.eval_mode = t["eval_mode"]
        return o

    def serve(times, fused=False):
        srv = gb.Server(pool_budget_bytes=150 << 30, device=0, max_active=32, fused=fused)
        for _, p in stream[:3]:                       # warm-up
            rid = srv.submit(p, _serving_opts(gb, p, True))
            while srv.poll(rid) is None:
                time.sleep(0.0005)
        t0 = time.perf_counter()
        pending, done, k = {}, {}, 0
        while len(done) < len(stream):
            now = time.perf_counter() - t0
            while k < len(stream) and times[k] <= now:
                p = stream[k][1]
                pending[srv.submit(p, served_opts(p))] = k
                k += 1
            for rid in list(pending):
                r = srv.poll(rid)
                if r is not None:
                    done[pending.pop(rid)] = (r, time.perf_counter() - t0)
            time.sleep(0.0002)
        srv.close()
        return done

    def valid(r):
        return r.status == 0 and r.fmin_lo <= 0.0 <= r.fmin_hi and r.fmin_hi - r.fmin_lo <= 1e-6

    live = serve(arrivals)
    lat = np.array([live[i][0].latency_ms for i in range(len(stream))])
    makespan = max(t for _, t in live.values())
    ok = all(valid(live[i][0]) for i in range(len(stream)))
    # one at a time, FP64 only
    service, seq = [], []
    for _, p in stream:
        o = _serving_opts(gb, p, False)
        s = gb.Solver(p, **{f: getattr(o, f) for f in ("block", "split_m", "split_d", "max_children",
                                                        "pool_bytes", "gens_per_sync")})
        t0 = time.perf_counter()
        r = s.solve()
        service.append(time.perf_counter() - t0)
        seq.append(r)
        s.close()
    seq_ok = all(valid(r) for r in seq)
    finish, fifo_lat = 0.0, []
    for t, sv in zip(arrivals, service):
        finish = max(finish, t) + sv
        fifo_lat.append(1e3 * (finish - t))
    fifo_lat = np.array(fifo_lat)
    # saturation, every request advancing on its own, and with the fused
    # child evaluation over the requests of a step
    sat = serve(np.zeros(len(stream)))
    sat_t = max(t for _, t in sat.values())
    sat_u = serve(np.zeros(len(stream)), fused=True)
    sat_ut = max(t for _, t in sat_u.values())
    same = all(sat[i][0].fmin_lo == sat_u[i][0].fmin_lo and sat[i][0].fmin_hi == sat_u[i][0].fmin_hi
               and sat[i][0].fmin_lo == live[i][0].fmin_lo and sat[i][0].fmin_hi == live[i][0].fmin_hi
               for i in range(len(stream)))
    ok = ok and all(valid(sat[i][0]) and valid(sat_u[i][0]) for i in range(len(stream)))
    fams, widths = {}, {}
    for i, (_, p) in enumerate(stream):
        fams[p.family] = fams.get(p.family, 0) + 1
        wd = widths.setdefault(p.family, ([], []))
        wd[0].append(live[i][0].fmin_hi - live[i][0].fmin_lo)
        wd[1].append(seq[i].fmin_hi - seq[i].fmin_lo)

    def stats(v):
        v = np.array(v)
        return {"median": float(np.median(v)), "max": float(v.max())}

    best = max(len(stream) / sat_t, len(stream) / sat_ut)
    return {
        "workload": f"serving stream: {len(stream)} requests, Poisson arrivals 20/s, n log-uniform [2, {a.n_max}], "
                    f"families {fams}, tol_f=1e-6, FP32 prefilter + FP64, 150 GB budget, 32 slots, 4 GB per "
                    "request, one best box per generation",
        "served_solves_per_s": best,
        "served_solves_per_s_is": "capacity: all requests submitted at once, the better of the two serving modes",
        "per_request_graphs_solves_per_s": len(stream) / sat_t,
        "fused_steps_solves_per_s": len(stream) / sat_ut,
        "fused_is": "the children of the requests of a step evaluated in one persistent launch per generation "
                    "(gb_server_set_fused)",
        "sequential_fp64_solves_per_s": len(stream) / sum(service),
        "speedup_vs_sequential_fp64": best / (len(stream) / sum(service)),
        "poisson_20_per_s": {
            "served_p50_ms": float(np.percentile(lat, 50)),
            "served_p99_ms": float(np.percentile(lat, 99)),
            "served_latency_is": "observed: submit -> result on the host clock",
            "served_solves_per_s": len(stream) / makespan,
            "one_at_a_time_fp64_p50_ms_fifo_model": float(np.percentile(fifo_lat, 50)),
            "one_at_a_time_fp64_p99_ms_fifo_model": float(np.percentile(fifo_lat, 99)),
            "one_at_a_time_latency_is": "computed: a FIFO queue replay of the measured one-at-a-time service "
                                        "times under the same arrival times",
        },
        "enclosure_width_by_family": {f: {"fp32_prefilter_served": stats(w[0]), "fp64_only": stats(w[1])}
                                      for f, w in sorted(widths.items())},
        "all_enclosures_valid": bool(ok and seq_ok),
        "served_results_identical_across_modes": bool(same),
        "autotune": ({_bucket_name(k): dict(v[0], solve_ms=v[1]) for k, v in tuned.items()} if tuned else None),
        "autotune_s": tune_s,
    }


def run_serving(a):
    blk = serving_block(a)
    line = {"metric": "served solves/s", "value": blk["served_solves_per_s"], "unit": "solves/s",
            "n_gpus": 1, "steps": 1, "warmup": 3, "ms_per_step": 1e3 * a.requests / blk["served_solves_per_s"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64",
            "data": "synthetic", "config": blk}
    print(json.dumps(line), flush=True)


def reduce_ranks(torch, dist, device, dev_ms, e2e_t, evals, e2e_evals):
    """Replicas: the job time is the slowest rank's (max), the work is every
    rank's (sum); the whole-job value is sum / max."""
    t = torch.tensor([dev_ms, e2e_t], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    c = torch.tensor([evals, e2e_evals], dtype=torch.float64, device=device)
    dist.all_reduce(c, op=dist.ReduceOp.SUM)
    return float(t[0]), float(t[1]), float(c[0]), float(c[1])


def _options(a, w, local, override=True):
    opts = dict(block=w["block"], split_m=(a.split_m if override and a.split_m else w["split_m"]),
                split_d=(a.split_d if override and a.split_d else w["split_d"]),
                max_children=(a.max_children if override and a.max_children else w["max_children"]),
                fp32_prefilter=w["fp32"], gens_per_sync=w["gens_per_sync"], device=local,
                pool_bytes=int(((a.pool_gb if override and a.pool_gb else 0) or w["pool_gb"]) * (1 << 30)))
    if w.get("paper"):
        opts.update(samples=10, mono_all=1, tol_x=1e-4)
        if w.get("pool_mode"):
            opts["pool_mode"] = w["pool_mode"]
    if override and a.max_gens > 0:
        opts["max_generations"] = a.max_gens
    if override and a.eval_mode >= 0:
        opts["eval_mode"] = a.eval_mode
    elif w.get("eval_mode") is not None:
        opts["eval_mode"] = w["eval_mode"]
    return opts


def measure(a, w, gb, torch, dev, local, rank, dist, steps, warmup, e2e_steps, opts, clocks=None):
    """Times `steps` complete solves of workload w (after `warmup`), then the
    evaluation kernels on one solve with per-generation events when the
    workload replays CUDA graphs, then `e2e_steps` solves through the C ABI
    from host buffers."""
    p = _problem(w, seed=rank)
    solver = gb.Solver(p, **opts)
    info = solver.info()
    flush = torch.zeros(64 * 1024 * 1024, dtype=torch.float64, device=dev)
    for _ in range(warmup):
        solver.solve(device_only=True)
    if clocks:
        clocks.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize(dev)
    results, host_t = [], 0.0
    for _ in range(steps):
        flush_l2(torch, dev, flush)
        t0 = time.perf_counter()
        r = solver.solve(device_only=True)
        host_t += time.perf_counter() - t0
        results.append(r)
    torch.cuda.synchronize(dev)
    if dist:
        dist.barrier()
    ck = clocks.stop() if clocks else None
    solver.close()

    # per-kernel event times of the evaluation (graph replays carry no
    # per-kernel events: one extra solve with a host synchronisation per
    # generation times the kernels)
    prof = results
    if w["gens_per_sync"] > 1:
        psolver = gb.Solver(p, **dict(opts, gens_per_sync=1))
        prof = [psolver.solve(device_only=True)]
        psolver.close()

    e2e_t, e2e_evals, d2h = 0.0, 0, 0
    h2d = p.nodes.nbytes + sum(t.nbytes for t in p.tables) + p.l.nbytes + p.u.nbytes
    for _ in range(e2e_steps):
        flush_l2(torch, dev, flush)
        t0 = time.perf_counter()
        h = gb.gb_create_problem(p.nodes, p.root, p.tables, p.n, p.l, p.u, p.tol_f, gb.gb_default_options(**opts))
        r = gb.gb_solve(h)
        h.close()
        e2e_t += time.perf_counter() - t0
        e2e_evals += r.box_evals_fp64 + r.box_evals_fp32
        d2h = r.n_boxes * (2 * p.n + 1) * 8 + r.generations * (48 + 256) + 256
    del flush
    return dict(p=p, info=info, results=results, prof=prof, host_t=host_t, clocks=ck, e2e_t=e2e_t,
                e2e_evals=e2e_evals, h2d=h2d, d2h=d2h)


def roofline(m, w, opts, sm_mhz, sms, gb, local):
    """The evaluation's directed operations per second of its event time
    against the ALU roofline: FP64 and FP32 operations each at their pipe
    rate (2 and 128 per SM per clock), combined as FP64-equivalent
    operations (an FP32 operation counts 2/128 of an FP64 one)."""
    prof = m["prof"]
    ms = sum(r.eval64_ms for r in prof)
    n = sum(r.eval64_launches for r in prof)
    o64 = sum(r.ops64 for r in prof)
    o32 = sum(r.ops32 for r in prof)
    evals = sum(r.box_evals_fp64 + r.box_evals_fp32 for r in prof)
    peak64 = FP64_OPS_PER_SM_CLK * sms * sm_mhz * 1e6
    eq = o64 + o32 * FP64_OPS_PER_SM_CLK / FP32_OPS_PER_SM_CLK
    achieved = eq / (ms * 1e-3) if ms > 0 else None
    warp = opts["max_children"] < (1 << 16)
    if w.get("paper"):
        kname = "k_eval32 + k_eval64 (bytecode interpreter)" if w["fp32"] else "k_eval64 (bytecode interpreter)"
    elif w["fp32"] and warp:
        kname = "k_ptab + k_ptab_d + k_eval3264_tabw (tables, then FP32 and FP64 in one warp-per-child kernel)"
    else:
        kname = ("k_ptab + k_ptab_d + " + ("k_eval32_tab + compaction + " if w["fp32"] else "") + "k_eval64_tab"
                 + ("w" if warp else ""))
    try:
        probe64, _ = gb.gb_measure_peak(local, 0)
    except Exception:
        probe64 = None
    return {"bound": "alu", "achieved": achieved / 1e12 if achieved else None, "peak": peak64 / 1e12,
            "unit": "TFLOP/s", "frac": (achieved / peak64) if achieved else None, "traffic": w.get("traffic"),
            "kernel": kname,
            "ops": "directed-rounding FP64 operations plus FP32 operations x 2/128, executed by the per-parent "
                   "table kernels and the child kernels (counted in the kernels)",
            "ops64_per_eval": o64 / max(1, evals), "ops32_per_eval": o32 / max(1, evals),
            "static_ops_per_eval": m["info"]["ops_eval"] + m["info"]["ops_mid"],
            "peak_source": f"{FP64_OPS_PER_SM_CLK:.0f} FP64 ops/SM/clk x {sms} SMs (device attribute) x "
                           f"{sm_mhz:.0f} MHz (sampled median); nominal issue rate, MEASURED_PEAKS has no FP64 figure",
            "timed_on": "the timed solves" if prof is m["results"] else "one extra solve, per-generation sync",
            "avg_launch_ms": ms / max(1, n), "launches": n,
            "probe_measured_fp64_tops": probe64 / 1e12 if probe64 else None}


def _summary(m, w, opts, sm_mhz, sms, gb, local):
    res = m["results"]
    dev_ms = sum(r.device_ms for r in res)
    evals = sum(r.box_evals_fp64 + r.box_evals_fp32 for r in res)
    fstar = m["p"].meta.get("fstar", 0.0)
    ok = all(r.status == 0 and r.fmin_lo <= fstar <= r.fmin_hi and
             (w.get("paper") or r.fmin_hi - r.fmin_lo <= m["p"].tol_f) for r in res)
    last = res[-1]
    return {"workload": w["name"], "box_evals_per_s": evals / (dev_ms * 1e-3), "ms_per_solve": dev_ms / len(res),
            "solves_per_s": len(res) / (dev_ms * 1e-3), "solves_timed": len(res),
            "generations_per_solve": last.generations, "ms_per_generation": dev_ms / len(res) / max(1, last.generations),
            "kernel_launches_per_generation": last.kernel_launches / max(1, last.generations),
            "mid_evals_per_s": sum(r.mid_evals for r in res) / (dev_ms * 1e-3),
            "fp32_evals_per_solve": last.box_evals_fp32, "fp64_evals_per_solve": last.box_evals_fp64,
            "pool": "block records" if last.pool_mode == 2 else "dense rows",
            "peak_pool_boxes": int(last.trace["pool"].max()) if len(last.trace["pool"]) else 1,
            "all_enclosures_valid": ok, "enclosure": [last.fmin_lo, last.fmin_hi],
            "options": {k: opts[k] for k in ("block", "split_m", "split_d", "max_children", "fp32_prefilter",
                                              "gens_per_sync")},
            "roofline": roofline(m, w, opts, sm_mhz, sms, gb, local)}


def main():
    a = _args()
    if a.impl == "reference":
        run_reference(a)
        return
    if a.workload == "serving":
        run_serving(a)
        return
    import torch
    import paper_2507_01770_gb300 as gb

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    gb.load()
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    w = _workload(a)
    opts = _options(a, w, local)
    clocks = ClockSampler(local)
    e2e_steps = 0 if a.no_e2e else max(1, min(3, a.steps))
    m = measure(a, w, gb, torch, dev, local, rank, dist, a.steps, a.warmup, e2e_steps, opts, clocks)
    res = m["results"]
    dev_ms = sum(r.device_ms for r in res)
    evals = sum(r.box_evals_fp64 + r.box_evals_fp32 for r in res)
    launches = sum(r.kernel_launches for r in res)
    e2e_t, e2e_evals = m["e2e_t"], m["e2e_evals"]
    if dist:
        dev_ms, e2e_t, evals, e2e_evals = reduce_ranks(torch, dist, dev, dev_ms, e2e_t, evals, e2e_evals)
    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    ck = m["clocks"]
    sm_mhz = ck["sm_mhz"] if ck else 2070.0
    summ = _summary(m, w, opts, sm_mhz, sms, gb, local)
    value = evals / (dev_ms * 1e-3)
    metric, unit, hib, vsb = "box-evals/s", "box-evals/s", True, None
    if w.get("paper"):   # the paper prints solve times for its procedure
        metric, unit, hib = "solve time", "s", False
        value = dev_ms * 1e-3 / a.steps
        vsb = value / w["baseline_s"] if w.get("baseline_s") else None
    rl = summ.pop("roofline")
    config = dict(summ, l2="flushed between steps (512 MB write)", paper_time_s=w.get("baseline_s"),
                  host_ms_per_step=1e3 * m["host_t"] / a.steps, parallelism="replicas" if world > 1 else "1 GPU",
                  sms=sms)
    nested = a.workload == "mixed10k" and not a.no_nested and world == 1
    if nested:
        # the n = 100 chain workload (FP64, 4^10 children per generation)
        w1 = WORKLOADS["chain100"]
        o1 = _options(a, w1, local, override=False)
        m1 = measure(a, w1, gb, torch, dev, local, rank, None, min(a.steps, 10), 3, 0, o1)
        config["chain100"] = _summary(m1, w1, o1, sm_mhz, sms, gb, local)
        # the serving stream (served solves/s against one-at-a-time FP64, p50 / p99)
        if not a.no_serving:
            config["serving"] = serving_block(a)
    line = {
        "metric": metric, "value": value, "unit": unit, "n_gpus": world,
        "steps": a.steps, "warmup": a.warmup, "ms_per_step": dev_ms / a.steps,
        "higher_is_better": hib, "scaling": "weak", "vs_baseline": vsb,
        "dtype": "f32+f64" if w["fp32"] else "f64", "data": "synthetic",
        "config": config,
        "e2e": ({"value": (e2e_t / e2e_steps) if w.get("paper") else e2e_evals / e2e_t,
                 "unit": unit, "h2d_bytes_per_step": int(m["h2d"]),
                 "d2h_bytes_per_step": int(m["d2h"])} if e2e_t > 0 else None),
        "gpu_launches": int(launches),
        "roofline": rl,
        "clocks": ck,
    }
    if not a.no_cpu_baseline:
        import oracle
        oracle.build()
        line["cpu_baseline"] = cpu_baseline_both(w, a.cpu_gens or w["cpu_gens"])
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
