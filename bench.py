#!/usr/bin/env python
"""Benchmark of the selective-update hot path on GB300.

Default workload: the large predation model (2048x2048 periodic grid, 1,000,000
sheep / 250,000 wolves, capacity 8Mi / 4Mi, Philox seed 1, 1000 steps). A
"step" is one predation step -- select, compact, add, remove, distinct update
and conflict resolution for both species. ``--warmup W`` steps run untimed,
then ``--steps K`` steps are timed with CUDA events (default W + K = 1000, the
whole run). Metric: agent-steps/s = sum over timed steps of the live agents at
the start of the step, divided by the device time.

The same JSON line carries the selective-update microbenchmark (2^24 slots x 8
int32 fields, p in {0.001, 0.05, 0.5}, plus the Zipf conflict pass) in HBM
GB/s, the roofline of the dominant kernel, the oracle's CPU timing and the
end-to-end (host API) rate.

``--impl reference`` times the sequential CPU oracle on the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import workloads  # noqa: E402

METRIC = "agent-steps/s (predation)"
UNIT = "agent-steps/s"
PHASES = ("sheep_move", "sheep_scan", "sheep_births", "wolf_move", "wolf_scan", "wolf_births")
KERNELS = ("k_move<0>", "k_scan<0>", "k_births<0>", "k_move<1>", "k_scan<1>", "k_births<1>")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=995)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-extras", action="store_true", help="skip the microbenchmark legs")
    return ap.parse_args()


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return float(d.get("hbm_gbs", 6800.0)), "measured"
    return 6800.0, "fallback"


def config_block():
    c = workloads.PRED_LARGE
    return {"workload": c["name"], "side": c["side"], "n0": list(c["n0"]), "cap": list(c["cap"]),
            "seed": c["seed"], "run_steps": c["steps"],
            "rules": "sheep gain 4, wolf gain 20, reproduce 0.04 / 0.05 (u32 thresholds), "
                     "grass regrowth 30, metabolism 1, 50% initial grass",
            "l2": "inputs larger than L2: 8Mi+4Mi slots x 20 B + 4Mi cells x 28 B = 352 MiB resident",
            "parallelism": "replicas (one independent model per GPU)"}


# ----------------------------------------------------------------------------
# clocks during the timed region

class ClockSampler:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.p = None
        return self

    def __exit__(self, *exc):
        self.out = ""
        if self.p is not None:
            time.sleep(0.25)
            self.p.terminate()
            try:
                self.out, _ = self.p.communicate(timeout=5)
            except Exception:
                self.p.kill()
        return False

    def summary(self):
        rows = [r.split(",") for r in (self.out or "").strip().splitlines() if r.count(",") >= 8]
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        sm = [float(r[1]) for r in rows if r[1].strip().replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].strip().replace(".", "").isdigit()]
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        reasons = sorted({n for r in rows for n, v in zip(names, r[5:9]) if "Active" in v and "Not" not in v})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": reasons, "samples": len(rows)}


# ----------------------------------------------------------------------------
# algorithmic bytes per kernel launch (units and per-unit bytes listed in the design doc)

def kernel_bytes(k: int, st: dict) -> int:
    s = 0 if k < 3 else 1
    n, E = st["n_start"][s], st["extent"][s]
    if k % 3 == 0:  # move: live flags over the extent; agent record read+write; cell lookups
        per = 16 + 16 + (8 + 4 if s == 0 else 8)  # sheep: victim reset + regrow read; wolf: victim read
        return 4 * E + n * per
    if k % 3 == 1:  # scan: flags; agent read + claim read; winners; lists; deaths; victim entry
        win = st["grass_eaten"] if s == 0 else st["eaten"]
        win_b = 4 + 8 + 4 if s == 0 else 4 + 8 + 8 + 8 + 4
        free = max(E - n, 0)
        b = 4 * E + n * (16 + 8) + win * win_b + 4 * min(free, n) + 4 * st["parents"][s] + 4 * st["starved"][s]
        if s == 0:
            b += 8 * (n - st["starved"][s])
        return b
    births = st["births"][s]  # births: indices, parent read/write, child write, live flag (+ victim key)
    return births * (4 + 4 + 16 + 4 + 16 + 4 + (8 if s == 0 else 0))


# ----------------------------------------------------------------------------

def dist_init(args):
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if args.impl == "ours" else "gloo"
        dist.init_process_group(backend=backend)
    return rank, world, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x: float, world: int, device=None) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x: float, world: int, device=None) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def oracle_predation_rate(steps: int, warmup: int, budget_s: float | None = None):
    """Sequential oracle on the large predation run: (agent-steps/s, steps timed, seconds)."""
    import oracle
    c = workloads.PRED_LARGE
    w = oracle.World(c["side"], c["seed"], c["model"], c["params"], c["cap"], c["n0"])
    w.step(warmup)
    agents, n, t0 = 0, 0, time.perf_counter()
    while n < steps:
        st = w.step()[0]
        agents += st["n_start"][0] + st["n_start"][1]
        n += 1
        if budget_s is not None and time.perf_counter() - t0 > budget_s:
            break
    dt = time.perf_counter() - t0
    return agents / dt, n, dt


def run_reference(args, rank, world):
    if rank != 0:
        return
    rate, n, dt = oracle_predation_rate(args.steps, args.warmup)
    line = {"impl": "reference", "metric": METRIC, "value": rate, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * dt / max(n, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
            "data": "synthetic (Philox-seeded)", "config": config_block(),
            "cpu_baseline": {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"steps {args.warmup}..{args.warmup + n - 1} of the large "
                                       f"predation run, sequential C oracle, 1 thread"},
            "e2e": {"value": rate, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def selective_update_leg(torch, engine, abm, hbm_peak, steps=8, warmup=3):
    """Selective-update microbenchmark: 2^24 slots x 8 fields, fused remove/update/add call."""
    c = workloads.SELECTIVE
    n, F = c["n"], c["F"]
    # L2 eviction between timed calls by READING 256 MiB (a written buffer would leave
    # dirty lines whose write-back lands inside the next timed call)
    flush = torch.ones(64 << 20, dtype=torch.int32, device="cuda")
    out = {}
    for p in c["p"]:
        T, k = workloads.threshold(p), workloads.k_for(p, n)
        s = engine.Slab(n, F, seed=c["seed"], init=abm.INIT_HALF_LIVE)
        rec = torch.empty((k, F), dtype=torch.int32, device="cuda")
        dl = torch.empty((k, F), dtype=torch.int32, device="cuda")
        cnt = torch.zeros(3, dtype=torch.int32, device="cuda")
        times, nbytes = [], []
        for it in range(warmup + steps):
            s.philox_records(it, abm.P_NEWREC0, abm.P_NEWREC1, k, out=rec)
            s.philox_records(it, abm.P_DELTA0, abm.P_DELTA1, k, out=dl)
            flush.max()
            torch.cuda._sleep(100000)  # device busy while the host enqueues the timed call
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            s.selective_update(it, T, rec, dl, out_counts=cnt)
            e1.record()
            e1.synchronize()
            if it >= warmup:
                removed, added, updated = cnt.tolist()
                times.append(e0.elapsed_time(e1))
                nbytes.append(4 * n + 4 * (removed + added) + added * (32 + 32) + updated * (32 + 32 + 32))
        s.check()
        ms = statistics.median(times)
        b = statistics.median(nbytes)
        gbs = b / (ms * 1e-3) / 1e9
        out[str(p)] = {"k": k, "ms": ms, "algorithmic_bytes": int(b), "gbs": gbs, "frac": gbs / hbm_peak}
        del s, rec, dl
    # conflict pass: M = N/4 claims over R = N/64 resources, Zipf(1.1)
    M, R = n // 4, n // 64
    res = torch.from_numpy(workloads.zipf_claims(M, R, s=c["zipf_s"], seed=c["zipf_seed"])).cuda()
    ps = engine.Slab(1, 1, seed=c["seed"])
    prio = ps.philox_records(0, abm.P_RESOURCE, abm.P_RESOURCE, M).reshape(-1)
    rv = engine.Resolver(R)
    isw = torch.empty(M, dtype=torch.uint8, device="cuda")
    times = []
    for it in range(warmup + steps):
        flush.max()
        torch.cuda._sleep(100000)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        rv(res, prio, isw)
        e1.record()
        e1.synchronize()
        if it >= warmup:
            times.append(e0.elapsed_time(e1))
    ms = statistics.median(times)
    b = 17 * M + 20 * R
    out["resolve"] = {"M": M, "R": R, "ms": ms, "algorithmic_bytes": b, "gbs": b / (ms * 1e-3) / 1e9,
                      "frac": b / (ms * 1e-3) / 1e9 / hbm_peak, "bound": "L2 atomics (2 MiB table)"}
    del flush
    return out


def run_ours(args, rank, world, local):
    import torch
    torch.cuda.set_device(local)
    from paper_2508_16508_gb300 import abm, engine
    abm.lib()
    hbm_peak, peak_kind = peaks()
    c = workloads.PRED_LARGE
    # each rank runs an independent replica (its own Philox model id)
    gw = engine.World(c["side"], c["seed"], c["model"] + rank, c["params"], c["cap"], c["n0"])
    K, W = args.steps, args.warmup
    stats = gw.new_stats(max(K, 1))
    gw.step(W)
    torch.cuda.synchronize()
    barrier(world)
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        phase = gw.step_profiled(K, stats)  # events on the launching stream, synchronises
    torch.cuda.synchronize()
    barrier(world)
    gw.check()
    ms_total = phase[7]
    st_rows = engine.decode_stats(stats[:K])
    cnt_after = gw.counters()
    # extents at the start of each timed step: replay the recorded populations
    # (extent only grows, by births beyond the free slots inside it)
    agents = sum(r["n_start"][0] + r["n_start"][1] for r in st_rows)
    local_rate = agents / (ms_total * 1e-3)
    t_max = max_over_ranks(ms_total, world, device="cuda")
    total_agents = sum_over_ranks(agents, world, device="cuda")
    value = total_agents / (t_max * 1e-3)

    # roofline of the dominant kernel
    shares = [phase[i] / max(sum(phase[:6]), 1e-9) for i in range(6)]
    dom = max(range(6), key=lambda i: phase[i])
    dom_bytes = sum(kernel_bytes(dom, r) for r in st_rows)
    achieved = dom_bytes / (phase[dom] * 1e-3) / 1e9
    roofline = {"kernel": KERNELS[dom], "bound": "hbm", "achieved": achieved, "peak": hbm_peak,
                "peak_kind": peak_kind, "unit": "GB/s", "frac": achieved / hbm_peak,
                "traffic": None, "launch_ms": phase[dom] / max(K, 1),
                "algorithmic_bytes_per_launch": dom_bytes / max(K, 1)}

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": W,
            "ms_per_step": t_max / max(K, 1), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "int32", "data": "synthetic (Philox-seeded initial state)",
            "config": config_block(), "roofline": roofline, "gpu_launches": 6 * K,
            "clocks": clk.summary(),
            "phases_ms_per_step": {n: phase[i] / max(K, 1) for i, n in enumerate(PHASES)},
            "phase_share": {n: shares[i] for i, n in enumerate(PHASES)},
            "end_counters": cnt_after}

    if rank == 0 and not args.no_extras:
        # end to end through the public API: one abm_step per step, then the
        # step's statistics read back to pinned host memory
        ew = engine.World(c["side"], c["seed"], c["model"], c["params"], c["cap"], c["n0"])
        ne = min(K, 300)
        sdev = ew.new_stats(1)
        shost = torch.empty_like(sdev, device="cpu").pin_memory()
        ew.step(W)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ea = 0
        for _ in range(ne):
            ew.step(1, sdev)
            shost.copy_(sdev, non_blocking=True)
            torch.cuda.current_stream().synchronize()
            r = engine.decode_stats(shost)[0]
            ea += r["n_start"][0] + r["n_start"][1]
        e2e_dt = time.perf_counter() - t0
        line["e2e"] = {"value": ea / e2e_dt, "unit": UNIT, "h2d_bytes_per_step": 0,
                       "d2h_bytes_per_step": abm.STATS_BYTES,
                       "note": "abm_step + synchronous read-back of the step's statistics; the model "
                               "state lives on the device, so a step has no host input"}
        del ew
        line["selective_update"] = selective_update_leg(torch, engine, abm, hbm_peak)
        # the oracle on the machine's host cores, bounded sample
        rate, n, dt = oracle_predation_rate(10**9, 0, budget_s=15.0)
        line["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle",
                                "sample": f"first {n} steps of the large predation run "
                                          f"({dt:.1f} s, sequential C oracle, 1 thread)"}
    if rank == 0:
        print(json.dumps(line), flush=True)


def main():
    args = parse()
    rank, world, local = dist_init(args)
    if args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_ours(args, rank, world, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
