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
GB/s; the batched legs (4096 models, 500 steps: plain fixed capacity vs
learned capacity); the order-book leg (one matching round of 65536 books x 1024
slots, and the 500-book, 100-step market run eager and from a CUDA graph); the
roofline of the timed kernel; the oracle's CPU timing; and the end-to-end
(host API) rate. ``--leg selective|batched|lob|predation`` runs one leg alone.

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

import numpy as np  # noqa: E402

import workloads  # noqa: E402

METRIC = "agent-steps/s (predation)"
NOMINAL_HBM_GBS = 8000.0  # GB300 HBM3e, nominal
UNIT = "agent-steps/s"
PHASES = ("sheep_move", "sheep_scan", "sheep_births", "wolf_move", "wolf_scan", "wolf_births")
KERNELS = ("k_move<0>", "k_scan<0>", "k_births<0>", "k_move<1>", "k_scan<1>", "k_births<1>")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=995)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the microbenchmark, batched and CPU legs")
    ap.add_argument("--leg", default="all", choices=["all", "predation", "selective", "batched", "lob"],
                    help="run one leg alone (profiling); 'all' prints the benchmark line")
    ap.add_argument("--no-tune", action="store_true",
                    help="default launch shapes instead of the autotuner (fixed launch sequence for ncu)")
    ap.add_argument("--p", type=float, action="append", help="selective leg: only these p")
    ap.add_argument("--batch-models", type=int, default=None)
    ap.add_argument("--batch-steps", type=int, default=None)
    ap.add_argument("--lob-books", type=int, default=None, help="lob leg: books in the matching round")
    ap.add_argument("--lob-warps", type=int, default=None, choices=[1, 2, 4],
                    help="lob leg: warps per book instead of the sweep (fixed launch sequence for ncu)")
    a = ap.parse_args()
    if a.leg == "predation":
        a.no_extras = True
    return a


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
# algorithmic bytes per kernel launch: each access of a phase counted once at its
# natural size, from the step's statistics (agents moved, winners, parents, ...)

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
        b = 4 * E + n * (16 + 8) + win * win_b + 4 * min(free, st["parents"][s]) + 4 * st["parents"][s] \
            + 4 * st["starved"][s]
        if s == 0:
            b += 8 * (n - st["starved"][s])
        return b
    births = st["births"][s]  # births: indices, parent read/write, child write, live flag (+ victim key)
    return births * (4 + 4 + 16 + 4 + 16 + 4 + (8 if s == 0 else 0))


TRAFFIC_FILE = os.path.join(ROOT, "profiles", "k_persistent_large_predation_traffic.txt")
TRAFFIC_SOURCES = ("pred_persistent.cu", "pred_world.cuh", "pred_rules.cuh", "common.cuh")
LOB_TRAFFIC_FILE = os.path.join(ROOT, "profiles", "k_lob_match_levels_65536x1024.md")
LOB_TRAFFIC_SOURCES = ("lob.cu", "common.cuh")


def sources_sha256(names) -> str:
    import hashlib
    h = hashlib.sha256()
    for name in names:
        with open(os.path.join(ROOT, "paper_2508_16508_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def persistent_sources_sha256() -> str:
    return sources_sha256(TRAFFIC_SOURCES)


def stored_traffic(path: str, sources, **must):
    """DRAM bytes (read + write) of one launch from a stored single-pass ncu
    capture (key = value lines), or None when the capture was of another
    launch (any `must` key differs) or the kernel's sources changed since."""
    try:
        with open(path) as f:
            kv = dict(ln.split("=", 1) for ln in (x.strip() for x in f) if "=" in ln and not ln.startswith("#"))
        kv = {k.strip(): v.strip() for k, v in kv.items()}
        if kv.get("sources_sha256") != sources_sha256(sources):
            return None
        if any(int(kv[k]) != int(v) for k, v in must.items()):
            return None
        return int(kv["dram_bytes_read"]) + int(kv["dram_bytes_write"])
    except (OSError, KeyError, ValueError):
        return None


def persistent_traffic(K: int, W: int, ctas_per_sm: int):
    """DRAM bytes of the timed k_persistent launch (see stored_traffic)."""
    return stored_traffic(TRAFFIC_FILE, TRAFFIC_SOURCES, steps=K, warmup=W, ctas_per_sm=ctas_per_sm)


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


def selective_update_leg(torch, engine, abm, autotune, hbm_peak, steps=8, warmup=3, tune=True, ps=None):
    """Selective-update microbenchmark: 2^24 slots x 8 fields, fused remove/update/add call."""
    c = workloads.SELECTIVE
    n, F = c["n"], c["F"]
    # L2 eviction between timed calls by READING 256 MiB (a written buffer would leave
    # dirty lines whose write-back lands inside the next timed call)
    flush = torch.ones(64 << 20, dtype=torch.int32, device="cuda")
    out = {}
    for p in (ps or c["p"]):
        T, k = workloads.threshold(p), workloads.k_for(p, n)
        tuned = autotune.tune_slab(n, F, p, k, seed=c["seed"]) if tune else None
        s = engine.Slab(n, F, seed=c["seed"], init=abm.INIT_HALF_LIVE)
        if tuned:
            s.tune(tuned["threads"], tuned["ctas_per_sm"])
        else:
            tuned = {"threads": "default", "ctas_per_sm": "default"}
        rec = torch.empty((k, F), dtype=torch.int32, device="cuda")
        dl = torch.empty((k, F), dtype=torch.int32, device="cuda")
        cnt = torch.zeros(3, dtype=torch.int32, device="cuda")
        times, nbytes, sbytes = [], [], []
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
                # sector-granular: every flag change touches its own 32-byte sector (an upper bound)
                sbytes.append(4 * n + 32 * (removed + added) + added * (32 + 32) + updated * (32 + 32 + 32))
        s.check()
        ms = statistics.median(times)
        b = statistics.median(nbytes)
        gbs = b / (ms * 1e-3) / 1e9
        sb = statistics.median(sbytes)
        out[str(p)] = {"k": k, "ms": ms, "algorithmic_bytes": int(b), "gbs": gbs, "frac": gbs / hbm_peak,
                       "frac_of_nominal_8tbs": gbs / NOMINAL_HBM_GBS, "sector_bytes_upper": int(sb),
                       "sector_gbs_upper": sb / (ms * 1e-3) / 1e9,
                       "launch": f"{tuned['threads']} threads x {tuned['ctas_per_sm']} CTAs/SM"
                                 + (" (autotuned)" if tune else "")}
        del s, rec, dl
    # sort_agents on the same slab shape: live agents first, ascending by one field
    s = engine.Slab(n, F, seed=c["seed"], init=abm.INIT_HALF_LIVE)
    times = []
    for it in range(warmup + steps):
        flush.max()
        torch.cuda._sleep(100000)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        s.sort(it % F)
        e1.record()
        e1.synchronize()
        if it >= warmup:
            times.append(e0.elapsed_time(e1))
    s.check()
    del s
    ms = statistics.median(times)
    # per slot: key + value built (read flag + key field, write 8 B), five passes of
    # (histogram read 4 B, scatter read 8 B + write 8 B), the row gather (value read 4 B,
    # row read + write 4 F B each, live flag and permutation written 4 B each)
    b = n * (8 + 8 + 5 * 20 + 4 + 2 * 4 * F + 8)
    out["sort_agents"] = {"ms": ms, "algorithmic_bytes": b, "gbs": b / (ms * 1e-3) / 1e9,
                          "frac": b / (ms * 1e-3) / 1e9 / hbm_peak,
                          "method": "LSD radix sort, 4 key-byte passes + 1 live-flag pass, then the row gather"}
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


def batched_leg(torch, engine, capacity, autotune, abm, hbm_peak, n_models=None, steps=None, tune=True):
    """Batched models: plain fixed capacity (static shapes, the whole capacity
    swept every step) vs learned capacity (MLP-sized slabs, device overflow
    detection, fixed-capacity rerun of the overflowed models)."""
    B = workloads.BATCH
    steps = steps or B["steps"]
    n_models = n_models or B["n_models"]
    tab = workloads.sample_models(B["n_models"], B["sampler_seed"])
    fixed = workloads.fixed_caps(tab["side"])[:n_models]
    models = [dict(side=int(tab["side"][i]), seed=B["philox_seed"], model=i, params=tab["params"][i],
                   cap=fixed[i], n0=tab["n0"][i]) for i in range(n_models)]
    default = {"threads": 512, "ctas_per_sm": 2, "models_per_cta": 1, "agents_per_thread": 16}
    tf = autotune.tune_batch(models, steps, abm.SWEEP_CAPACITY) if tune else default
    th, cps, g, apt = tf["threads"], tf["ctas_per_sm"], tf.get("models_per_cta", 1), tf.get("agents_per_thread", 16)
    trials = lambda tt: [[x["threads"], x["ctas_per_sm"], x.get("models_per_cta", 1),  # noqa: E731
                          x.get("agents_per_thread", 16), round(x["ms"], 2)]
                         for x in tt.get("trials", [])]
    shape = lambda tt: (f"{tt['threads']} threads x {tt['ctas_per_sm']} CTAs/SM x {tt.get('models_per_cta', 1)} "  # noqa: E731
                        f"models/CTA x {tt.get('agents_per_thread', 16)} slots/thread"
                        + (" (autotuned)" if tune else ""))
    out = {"workload": B["name"] if n_models == B["n_models"] and steps == B["steps"]
           else f"{n_models} models of {B['name']}, {steps} steps",
           "models": n_models, "steps": steps,
           "launch_fixed": shape(tf),
           "tune_trials_fixed_ms": trials(tf), "tune_trial_columns": ["threads", "ctas_per_sm", "models_per_cta", "agents_per_thread", "ms"]}
    # plain fixed capacity (one persistent launch for all 500 steps)
    b = engine.Batch(models)
    b.tune(th, cps, models_per_cta=g, agents_per_thread=apt)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    b.run(steps, sweep=abm.SWEEP_CAPACITY)
    e1.record()
    e1.synchronize()
    t_fixed = e0.elapsed_time(e1)
    want = b.digest().cpu().numpy()
    out["_digest_fixed"] = want
    cnt = b.counters()
    b.check()
    info = b.info()
    del b
    torch.cuda.empty_cache()
    agents = sum(c["agent_steps"] for c in cnt)
    hw = np.array([c["hw"] for c in cnt], dtype=np.int64)
    # bytes of the capacity sweep: each live flag read from memory once per species
    # per step (the move's sweep; the scan reads its shared-memory bitmask)
    sweep_bytes = 4 * (info["slots"][0] + info["slots"][1]) * steps
    out["fixed"] = {"ms": t_fixed, "agent_steps_per_s": agents / (t_fixed * 1e-3),
                    "slots": info["slots"], "live_flag_sweep_gbs": sweep_bytes / (t_fixed * 1e-3) / 1e9}
    # the same models with extent sweeps (a stronger plain baseline: placeholders past
    # the highest slot ever used are never visited), with the launch shape tuned for it
    tfe = autotune.tune_batch(models, steps, abm.SWEEP_EXTENT) if tune else default
    out["launch_fixed_extent"] = shape(tfe)
    out["tune_trials_fixed_extent_ms"] = trials(tfe)
    b = engine.Batch(models)
    b.tune(tfe["threads"], tfe["ctas_per_sm"], models_per_cta=tfe.get("models_per_cta", 1),
           agents_per_thread=tfe.get("agents_per_thread", 16))
    e0.record()
    b.run(steps, sweep=abm.SWEEP_EXTENT)
    e1.record()
    e1.synchronize()
    t_ext = e0.elapsed_time(e1)
    ext_ok = bool(np.array_equal(b.digest().cpu().numpy(), want))
    del b
    torch.cuda.empty_cache()
    out["fixed_extent_sweep"] = {"ms": t_ext, "agent_steps_per_s": agents / (t_ext * 1e-3), "bit_exact": ext_ok}
    # learned capacity
    wpath = os.path.join(ROOT, "paper_2508_16508_gb300", "data", "capacity_mlp.npz")
    m = capacity.CapacityModel.load(wpath)
    e0.record()
    learned = m.capacities(m.features(capacity.table_of(models, steps)), fixed, tab["n0"][:n_models], margin=0.0)
    e1.record()
    e1.synchronize()
    t_mlp = e0.elapsed_time(e1)
    lmodels = [dict(m, cap=(int(cc[0]), int(cc[1]))) for m, cc in zip(models, learned)]
    tl = autotune.tune_batch(lmodels, steps, abm.SWEEP_CAPACITY) if tune else default
    # one small learned-capacity run with a rerun first, so that the timed runs
    # do not pay the first call's one-time costs (module loading, first allocations)
    capacity.run_learned(models[:8], np.maximum(np.asarray(tab["n0"][:8]), 1), fixed[:8], 20)
    out["launch_learned"] = shape(tl)
    out["tune_trials_learned_ms"] = trials(tl)
    res = capacity.run_learned(models, learned, fixed, steps, threads=tl["threads"], ctas_per_sm=tl["ctas_per_sm"],
                               models_per_cta=tl.get("models_per_cta", 1),
                               agents_per_thread=tl.get("agents_per_thread", 16))
    t_learned = res["ms_learned"] + res["ms_rerun"] + t_mlp
    out["_digest_learned"] = res["digest"]
    n_over = np.array([max(c["overflow"]) for c in res["counters"]])
    out["learned"] = {"ms": t_learned, "ms_run": res["ms_learned"], "ms_rerun": res["ms_rerun"], "ms_mlp": t_mlp,
                      "agent_steps_per_s": agents / (t_learned * 1e-3),
                      "speedup_vs_fixed": t_fixed / t_learned,
                      "overflowed_models": len(res["overflowed"]), "rerun_models": res["rerun"],
                      # models whose reported result is still truncated after the rerun
                      "unrecovered_overflows": int(res["unrecovered"]),
                      "truncated_after_rerun": int(n_over.sum()),
                      "bit_exact_vs_fixed": bool(np.array_equal(res["digest"], want)),
                      "capacity_sum_fixed": int(fixed.sum()), "capacity_sum_learned": int(learned.sum()),
                      "peak_sum": int(hw.sum()),
                      "wasted_capacity": (int(learned.sum()) - int(hw.sum())) / int(hw.sum())}
    # learned capacities (memory) with extent sweeps (work): compared with the
    # extent-sweep fixed run, the fair plain baseline for it; its own tuned shape
    tle = autotune.tune_batch(lmodels, steps, abm.SWEEP_EXTENT) if tune else default
    out["launch_learned_extent"] = shape(tle)
    out["tune_trials_learned_extent_ms"] = trials(tle)
    res = capacity.run_learned(models, learned, fixed, steps, sweep=abm.SWEEP_EXTENT, threads=tle["threads"],
                               ctas_per_sm=tle["ctas_per_sm"], models_per_cta=tle.get("models_per_cta", 1),
                               agents_per_thread=tle.get("agents_per_thread", 16))
    t_le = res["ms_learned"] + res["ms_rerun"] + t_mlp
    out["learned_extent_sweep"] = {"ms": t_le, "ms_run": res["ms_learned"], "ms_rerun": res["ms_rerun"],
                                   "agent_steps_per_s": agents / (t_le * 1e-3),
                                   "speedup_vs_fixed_extent_sweep": t_ext / t_le,
                                   "speedup_vs_fixed": t_fixed / t_le,
                                   "overflowed_models": len(res["overflowed"]),
                                   "unrecovered_overflows": int(res["unrecovered"]),
                                   "bit_exact_vs_fixed": bool(np.array_equal(res["digest"], want))}
    out["note"] = ("speedup_vs_fixed compares with the paper's static shapes (every slot swept every step); "
                   "learned_extent_sweep.speedup_vs_fixed_extent_sweep compares two runs that both stop at the "
                   "extent, where capacity only saves memory")
    return out


def small_world_leg(torch, engine, abm, reps=10):
    """The 40x40 world (100 sheep / 25 wolves, 200 steps): launch- and
    latency-bound, so no roofline. Three ways to run it: the persistent
    kernel (one launch for all steps), the per-phase kernels replayed from a
    CUDA graph, and the batched runner with a batch of one (one CTA)."""
    c = workloads.PRED_SMALL
    n = c["steps"]

    def timed(fn):
        ts = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            fn()
            e1.record()
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
        return statistics.median(ts)

    mk = lambda: engine.World(c["side"], c["seed"], c["model"], c["params"], c["cap"], c["n0"])
    # agent-steps of the run, from one reference run
    ref = mk()
    st = ref.new_stats(n)
    ref.step(n, st)
    rows = engine.decode_stats(st)
    agents = sum(r["n_start"][0] + r["n_start"][1] for r in rows)
    want = ref.counters()
    out = {"workload": c["name"], "steps": n, "agent_steps": agents, "timing": f"median of {reps} runs, CUDA events"}
    # persistent kernel: a fresh world per run (results are checked below)
    worlds = [mk() for _ in range(reps)]
    it = iter(worlds)
    ms = timed(lambda: next(it).step(n))
    same = all(w_.counters() == want for w_ in worlds)
    out["persistent_one_launch"] = {"ms": ms, "us_per_step": 1e3 * ms / n, "agent_steps_per_s": agents / (ms * 1e-3),
                                    "same_result": same}
    del worlds
    # per-phase kernels in a CUDA graph (captured once, replayed per run)
    s = torch.cuda.Stream()
    worlds = [mk() for _ in range(reps + 1)]
    for w_ in worlds:
        w_.tune(abm.ENGINE_KERNELS)
    with torch.cuda.stream(s):
        worlds[0].step_graph(n, 1, stream=s)  # capture + first replay
        s.synchronize()
        it = iter(worlds[1:])
        # each world captures its own graph on first use; replay = one graph launch of n steps
        for w_ in worlds[1:]:
            w_.step_graph(n, 0, stream=s)  # capture only
        s.synchronize()
        ms = timed(lambda: next(it).step_graph(n, 1, stream=s))
    same = all(w_.counters() == want for w_ in worlds)
    out["kernels_cuda_graph"] = {"ms": ms, "us_per_step": 1e3 * ms / n, "agent_steps_per_s": agents / (ms * 1e-3),
                                 "same_result": same}
    del worlds
    # one model through the batched runner (one CTA, __syncthreads between phases)
    model = dict(side=c["side"], seed=c["seed"], model=c["model"], params=c["params"], cap=c["cap"], n0=c["n0"])
    batches = [engine.Batch([model]) for _ in range(reps)]
    for b in batches:
        b.tune(512, 1)
    it = iter(batches)
    ms = timed(lambda: next(it).run(n, sweep=abm.SWEEP_EXTENT))
    same = all(b.counters()[0]["agent_steps"] == agents for b in batches)
    out["batched_one_cta"] = {"ms": ms, "us_per_step": 1e3 * ms / n, "agent_steps_per_s": agents / (ms * 1e-3),
                              "same_agent_steps": same}
    del batches
    return out


def many_wolves_leg(torch, engine, abm, K, W, ctas_per_sm):
    """The large world under the several-wolves-per-cell variant (rank-matched
    meals per cell): same timing as the headline (one persistent launch)."""
    c = workloads.PRED_LARGE
    gw = engine.World(c["side"], c["seed"], c["model"], c["params"], c["cap"], c["n0"],
                      variant=abm.VARIANT_MANY_WOLVES)
    gw.tune(abm.ENGINE_PERSISTENT, ctas_per_sm)
    stats = gw.new_stats(max(K, 1))
    gw.step(W)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    gw.step(K, stats)
    e1.record()
    e1.synchronize()
    gw.check()
    ms = e0.elapsed_time(e1)
    rows = engine.decode_stats(stats[:K])
    agents = sum(r["n_start"][0] + r["n_start"][1] for r in rows)
    return {"workload": c["name"] + " (several wolves per cell)", "steps": K, "warmup": W, "ms": ms,
            "us_per_step": 1e3 * ms / max(K, 1), "agent_steps_per_s": agents / (ms * 1e-3),
            "eaten": sum(r["eaten"] for r in rows), "end_counters": gw.counters()}


def lob_leg(torch, engine, hbm_peak, reps=10, n_books=None, warps=None):
    """Order-book matching (Section 5.3): one matching round of 65536 books x
    1024 slots (half live), timed kernel-only on a freshly restored book each
    rep (inputs 1.3 GB, larger than L2; L2 also flushed); plus the finance
    model's scale (500 books x 1000 slots, 100 steps of order placement +
    matching)."""
    W = workloads.LOB
    nb_ = n_books or W["n_books"]
    book = workloads.random_books(nb_, W["cap"], W["fill"], W["seed"])
    pristine = engine.OrderBooks(book)
    work = engine.OrderBooks(book)
    vol = torch.empty(nb_, dtype=torch.int64, device="cuda")
    px = torch.empty(nb_, dtype=torch.int32, device="cuda")
    flush = torch.ones(64 << 20, dtype=torch.int32, device="cuda")

    def restore():
        for f in engine.OrderBooks.FIELDS:
            work.t[f].copy_(pristine.t[f])

    # the words the matching round must move (see the roofline note)
    restore()
    work.match(vol, px)
    torch.cuda.synchronize()
    live = int(pristine.t["active"].sum())
    qty_w = int((work.t["qty"] != pristine.t["qty"]).sum())
    act_w = int((work.t["active"] != pristine.t["active"]).sum())
    slots = nb_ * W["cap"]
    alg = 4 * slots + 12 * live + 4 * qty_w + 4 * act_w + 12 * nb_
    want = (int(vol.sum()), int(px.sum()))

    def timed(n):
        ts = []
        for _ in range(n):
            restore()
            flush.max()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            work.match(vol, px)
            e1.record()
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
        return ts

    # launch shape: warps per book on the price-level path (results identical);
    # a fixed shape skips the sweep (a fixed launch sequence for ncu)
    trials = {}
    for g in ((warps,) if warps else (1, 2, 4)):
        engine.OrderBooks.tune(g)
        trials[g] = statistics.median(timed(4)) if not warps else None
    best_g = warps or min(trials, key=trials.get)
    engine.OrderBooks.tune(best_g)
    ts = timed(reps)
    same = (int(vol.sum()), int(px.sum())) == want
    ms = statistics.median(ts)
    gbs = alg / (ms * 1e-3) / 1e9
    out = {"workload": W["name"] if nb_ == W["n_books"] else f"lob_{nb_}x{W['cap']}",
           "kernel": "k_lob_match_levels", "warps_per_book": best_g,
           "tune_trials_ms": {str(g): v for g, v in trials.items()}, "ms": ms, "ms_all": ts, "books_per_s": nb_ / (ms * 1e-3),
           "live_orders_per_s": live / (ms * 1e-3), "live_orders": live, "traded_shares": want[0],
           "books_crossed": int((vol > 0).sum()), "same_result_every_rep": same,
           "roofline": {"bound": "hbm", "achieved": gbs, "peak": hbm_peak, "unit": "GB/s", "frac": gbs / hbm_peak,
                        "traffic": stored_traffic(LOB_TRAFFIC_FILE, LOB_TRAFFIC_SOURCES, n_books=nb_, cap=W["cap"],
                                                  warps_per_book=best_g),
                        "algorithmic_bytes_per_launch": alg,
                        "bytes_per_slot": {"algorithmic": alg / slots, "sector_min": None},
                        "note": "algorithmic words: active of every slot, side/price/qty of live slots, the "
                                "qty/active words written, 12 B of output per book (time words of the few "
                                "orders on the two marginal price levels not counted)"},
           "timing": f"median of {reps} launches, CUDA events, book restored and L2 flushed before each"}
    # 32-byte sectors that hold those words (what DRAM must move at the least)
    act = pristine.t["active"].view(-1, 8)
    sec_live = int((act != 0).any(dim=1).sum())
    out["roofline"]["bytes_per_slot"]["sector_min"] = (32 * act.shape[0] + 3 * 32 * sec_live + 8 * (
        qty_w + act_w)) / slots if W["cap"] % 8 == 0 else None
    del pristine, work, flush
    torch.cuda.empty_cache()

    # the finance model's scale: each step up to 10 new orders per book, then
    # a matching round (inputs for all steps resident on the device)
    M = workloads.LOB_MARKET
    orders, ks = workloads.market_orders(M["n_books"], M["traders"], M["steps"], M["seed"])
    mbook = workloads.random_books(M["n_books"], M["cap"], M["fill"], M["seed"])
    d_orders = torch.from_numpy(orders).cuda()
    d_k = torch.from_numpy(ks).cuda()
    mv = torch.empty(M["steps"], M["n_books"], dtype=torch.int64, device="cuda")
    mp = torch.empty(M["steps"], M["n_books"], dtype=torch.int32, device="cuda")
    ma = torch.empty(M["steps"], M["n_books"], dtype=torch.int32, device="cuda")
    mts = []
    for _ in range(5):
        mb = engine.OrderBooks(mbook)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for st in range(M["steps"]):
            mb.add(d_orders[st], d_k[st], out=ma[st])
            mb.match(mv[st], mp[st])
        e1.record()
        e1.synchronize()
        mts.append(e0.elapsed_time(e1))
    eager = (int(mv.sum()), int(ma.sum()), int(mp.sum()))
    # the same 100 steps captured once in a CUDA graph (no host launch cost),
    # replayed from a restored book each time
    mb = engine.OrderBooks(mbook)
    start = {f: mb.t[f].clone() for f in engine.OrderBooks.FIELDS}
    gs = torch.cuda.Stream()
    gs.wait_stream(torch.cuda.current_stream())
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.stream(gs):
        with torch.cuda.graph(graph, stream=gs):
            for st in range(M["steps"]):
                mb.add(d_orders[st], d_k[st], out=ma[st])
                mb.match(mv[st], mp[st])
    torch.cuda.current_stream().wait_stream(gs)
    gts, same_graph = [], True
    for _ in range(5):
        for f in engine.OrderBooks.FIELDS:
            mb.t[f].copy_(start[f])
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        graph.replay()
        e1.record()
        e1.synchronize()
        gts.append(e0.elapsed_time(e1))
        same_graph &= (int(mv.sum()), int(ma.sum()), int(mp.sum())) == eager
    del graph
    out["market"] = {"workload": M["name"], "ms_100_steps": statistics.median(mts), "ms_all": mts,
                     "us_per_step": 1e3 * statistics.median(mts) / M["steps"],
                     "graph_ms_100_steps": statistics.median(gts), "graph_ms_all": gts,
                     "graph_us_per_step": 1e3 * statistics.median(gts) / M["steps"],
                     "graph_same_result": same_graph,
                     "traded_shares": eager[0], "orders_placed": eager[1],
                     "launches": 3 * M["steps"],
                     "paper_ms_100_steps_500_books": 2212.47,
                     "note": "paper figure: Table 4 (JAX, its own hardware): context, not a target"}
    return out


def lob_cpu_baseline(n_sample=4096, budget_s=15.0):
    """The oracle (sequential C, 1 thread) on a bounded sample of the same
    workloads: the first n_sample books of the 65536 x 1024 matching round,
    and the whole 500-book market run."""
    import oracle
    W = workloads.LOB
    book = workloads.random_books(n_sample, W["cap"], W["fill"], W["seed"])
    t0 = time.perf_counter()
    reps = 0
    while True:
        b = {f: v.copy() for f, v in book.items()}
        oracle.lob_match(b)
        reps += 1
        if time.perf_counter() - t0 > budget_s / 2 or reps >= 50:
            break
    dt = (time.perf_counter() - t0) / reps
    M = workloads.LOB_MARKET
    orders, ks = workloads.market_orders(M["n_books"], M["traders"], M["steps"], M["seed"])
    mb = workloads.random_books(M["n_books"], M["cap"], M["fill"], M["seed"])
    t1 = time.perf_counter()
    for st in range(M["steps"]):
        oracle.lob_add(mb, orders[st], ks[st])
        oracle.lob_match(mb)
    mdt = time.perf_counter() - t1
    return {"value": n_sample / dt, "unit": "books/s", "cores": 1, "kind": "oracle",
            "sample": f"first {n_sample} books of {W['name']}, {reps} matching rounds",
            "market_ms_100_steps": 1e3 * mdt}


def _oracle_model_run(args):
    """One batched-workload model on the sequential oracle (process-pool
    worker): agent-steps, seconds, and the digest of its final state."""
    side, seed, model, params, cap, n0, steps = args
    import oracle
    from oracle import digest
    w = oracle.World(side, seed, model, params, cap, n0)
    t0 = time.perf_counter()
    st = w.step(steps)
    dt = time.perf_counter() - t0
    return sum(r["n_start"][0] + r["n_start"][1] for r in st), dt, digest.state_digest(w)


def batched_cpu_baseline(n_sample=48, sample_seed=7):
    """The oracle on the batched workload, one model per host core: a random
    sample of the 4096 models for all 500 steps, scaled to the whole batch."""
    import multiprocessing as mp
    B = workloads.BATCH
    tab = workloads.sample_models(B["n_models"], B["sampler_seed"])
    fixed = workloads.fixed_caps(tab["side"])
    pick = np.random.default_rng(sample_seed).choice(B["n_models"], size=n_sample, replace=False)
    jobs = [(int(tab["side"][i]), B["philox_seed"], int(i), [int(x) for x in tab["params"][i]],
             [int(x) for x in fixed[i]], [int(x) for x in tab["n0"][i]], B["steps"]) for i in pick]
    cores = os.cpu_count() or 1
    t0 = time.perf_counter()
    with mp.get_context("spawn").Pool(cores) as pool:
        res = pool.map(_oracle_model_run, jobs, chunksize=1)
    wall = time.perf_counter() - t0
    agents = sum(a for a, _, _ in res)
    return {"value": agents / wall, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{n_sample} random models (numpy seed {sample_seed}) of the 4096, all {B['steps']} steps, "
                      f"one model per core, {wall:.1f} s wall",
            "cpu_seconds": sum(d for _, d, _ in res),
            "_models": [int(i) for i in pick], "_digests": [int(d) for _, _, d in res]}


def run_ours(args, rank, world, local):
    import numpy as _np  # noqa: F401
    import torch
    torch.cuda.set_device(local)
    from paper_2508_16508_gb300 import abm, autotune, capacity, engine
    abm.lib()
    hbm_peak, peak_kind = peaks()
    if args.leg in ("selective", "batched", "lob"):
        if rank == 0:
            with ClockSampler(local) as clk:
                if args.leg == "selective":
                    out = selective_update_leg(torch, engine, abm, autotune, hbm_peak, tune=not args.no_tune,
                                               ps=args.p)
                elif args.leg == "lob":
                    out = lob_leg(torch, engine, hbm_peak, n_books=args.lob_books, warps=args.lob_warps)
                else:
                    out = batched_leg(torch, engine, capacity, autotune, abm, hbm_peak, n_models=args.batch_models,
                                      steps=args.batch_steps, tune=not args.no_tune)
            out = {k: v for k, v in out.items() if not k.startswith("_")}  # arrays kept for the full run
            print(json.dumps({"leg": args.leg, "result": out, "clocks": clk.summary()}), flush=True)
        return
    c = workloads.PRED_LARGE
    # each rank runs an independent replica (its own Philox model id)
    tw = autotune.tune_world(c) if not args.no_tune else {"engine": abm.ENGINE_PERSISTENT, "ctas_per_sm": 2}
    gw = engine.World(c["side"], c["seed"], c["model"] + rank, c["params"], c["cap"], c["n0"])
    gw.tune(tw["engine"], tw["ctas_per_sm"])
    K, W = args.steps, args.warmup
    stats = gw.new_stats(max(K, 1))
    gw.step(W)
    torch.cuda.synchronize()
    barrier(world)
    torch.cuda.synchronize()
    clk = ClockSampler(local)
    clk.__enter__()
    # the product call: one abm_step for all K steps (one cooperative launch on
    # the persistent engine), CUDA events around it on the launching stream
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    gw.step(K, stats)
    e1.record()
    e1.synchronize()
    barrier(world)
    gw.check()
    ms_total = e0.elapsed_time(e1)
    st_rows = engine.decode_stats(stats[:K])
    agents = sum(r["n_start"][0] + r["n_start"][1] for r in st_rows)
    t_max = max_over_ranks(ms_total, world, device="cuda")
    total_agents = sum_over_ranks(agents, world, device="cuda")
    value = total_agents / (t_max * 1e-3)
    persistent = tw["engine"] == abm.ENGINE_PERSISTENT

    # roofline of the (only) kernel of the timed region: algorithmic bytes of
    # every phase of every step over the launch's duration
    step_bytes = sum(kernel_bytes(k, r) for r in st_rows for k in range(6))
    achieved = step_bytes / (ms_total * 1e-3) / 1e9
    roofline = {"kernel": "k_persistent (all phases of all timed steps, one cooperative launch)" if persistent
                else "six per-phase kernels per step",
                "bound": "hbm", "achieved": achieved, "peak": hbm_peak, "peak_kind": peak_kind,
                "unit": "GB/s", "frac": achieved / hbm_peak,
                "traffic": persistent_traffic(K, W, tw["ctas_per_sm"]) if persistent else None,
                "launch_ms": ms_total, "algorithmic_bytes_per_launch": step_bytes,
                "frac_of_nominal_8tbs": achieved / NOMINAL_HBM_GBS,
                "bytes_per_agent_step": {"algorithmic": step_bytes / max(agents, 1)},
                "note": "latency-bound: dependent random cell accesses and the grid barriers of each step"}
    if roofline["traffic"]:
        roofline["bytes_per_agent_step"]["dram"] = roofline["traffic"] / max(agents, 1)

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": W,
            "ms_per_step": t_max / max(K, 1), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "int32", "data": "synthetic (Philox-seeded initial state)",
            "config": dict(config_block(), engine=("persistent" if persistent else "kernels"),
                           ctas_per_sm=tw["ctas_per_sm"], launch="default" if args.no_tune else "autotuned",
                           timed_call="abm_step(K steps)",
                           tune_trials_ms=[[("persistent" if x["engine"] == abm.ENGINE_PERSISTENT else "kernels"),
                                            x["ctas_per_sm"], round(x["ms"], 3)] for x in tw.get("trials", [])]),
            "gpu_launches": 1 if persistent else 6 * K,
            "end_counters": gw.counters(), "roofline": roofline}

    extras = rank == 0 and not args.no_extras
    if extras:
        # where the time of a step goes: the same K steps again on a second world,
        # through abm_step_profiled (block 0's global-timer laps between the grid
        # barriers); not the timed call
        pw = engine.World(c["side"], c["seed"], c["model"] + rank, c["params"], c["cap"], c["n0"])
        pw.tune(tw["engine"], tw["ctas_per_sm"])
        pw.step(W)
        phase = pw.step_profiled(K)
        line["phases_us_per_step"] = {n: 1e3 * phase[i] / max(K, 1) for i, n in enumerate(
            ("P1_prev_wolf_ranks_sheep_move", "P2_prev_wolf_births_sheep_eat_select", "P3_sheep_ranks_wolf_move",
             "P4_sheep_births", "P5_wolf_eat_select", "closing_wolf_ranks"))}
        line["phases_us_per_step"]["same_trajectory"] = pw.counters() == gw.counters()
        del pw
        # end to end through the public API: the state loaded from host memory,
        # one abm_step per step with its statistics row written into pinned host
        # memory, the final state saved to host memory
        ew = engine.World(c["side"], c["seed"], c["model"] + rank, c["params"], c["cap"], c["n0"])
        ew.tune(tw["engine"], tw["ctas_per_sm"])
        ne = K
        # the statistics rows live in pinned host memory: the kernel writes them
        # there (unified addressing), so they reach the host with no copy
        shost = [torch.zeros((1, abm.STATS_WORDS), dtype=torch.int32).pin_memory() for _ in range(2)]
        sview = [h.numpy() for h in shost]
        ev = [torch.cuda.Event() for _ in range(2)]
        n_start = abm.STATS_FIELD_OFFSETS["n_start"] // 4  # int32 words of n_start[0], n_start[1]
        ew.step(W)
        nb = ew.image_bytes()  # the checkpoint image of the state: slots up to the extents
        img_in = torch.empty(nb, dtype=torch.uint8).pin_memory()
        img_out = torch.empty(ew.image_capacity(), dtype=torch.uint8).pin_memory()  # fits any final state
        ew.save_into(img_in)  # the state after the warm-up steps, as a host checkpoint

        def e2e_run(n):
            ew.load_from(img_in)  # the run's input: the whole state, host -> device
            ea = 0
            # one abm_step call per step; its statistics row, written by the kernel
            # into pinned host memory, is read there one step later, while the next
            # step runs
            for i in range(n + 1):
                if i < n:
                    b = i & 1
                    ew.step(1, shost[b])
                    ev[b].record()
                if i > 0:
                    b = (i - 1) & 1
                    ev[b].synchronize()
                    ea += int(sview[b][0, n_start]) + int(sview[b][0, n_start + 1])
            return ea, ew.save_into(img_out)  # the run's output: the whole state, device -> host

        e2e_run(max(W, 1))  # untimed warm-up of the same sequence (the buffers' first use)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ea, nb_out = e2e_run(ne)
        e2e_dt = time.perf_counter() - t0
        line["e2e"] = {"value": ea / e2e_dt, "unit": UNIT, "h2d_bytes_per_step": nb / max(ne, 1),
                       "d2h_bytes_per_step": abm.STATS_BYTES + nb_out / max(ne, 1),
                       "steps": ne, "state_bytes": nb, "state_bytes_out": nb_out,
                       "same_trajectory_as_timed_run": ew.counters() == gw.counters(),
                       "note": "after one untimed pass of the same sequence: "
                               "abm_load of the state from pinned host memory, then per step one abm_step "
                               "call whose kernel writes the step's statistics row into pinned host memory, "
                               "read by the host one step later (double-buffered), then abm_save of the final state "
                               "to pinned host memory (checkpoint images hold the slots up to each "
                               "species' extent); wall clock"}
        del ew, img_in, img_out
        line["selective_update"] = selective_update_leg(torch, engine, abm, autotune, hbm_peak)
        line["batched"] = batched_leg(torch, engine, capacity, autotune, abm, hbm_peak)
        line["small_world"] = small_world_leg(torch, engine, abm)
        line["many_wolves"] = many_wolves_leg(torch, engine, abm, K, W, tw["ctas_per_sm"])
        line["lob"] = lob_leg(torch, engine, hbm_peak)
    clk.__exit__(None, None, None)
    line["clocks"] = clk.summary()
    if extras:
        # the oracle on the machine's host cores, on the timed window's steps (bounded)
        rate, n, dt = oracle_predation_rate(K, W, budget_s=20.0)
        line["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle",
                                "sample": f"steps {W}..{W + n - 1} of the large predation run (the timed window"
                                          f"{'' if n == K else ', cut at 20 s'}; {dt:.1f} s, sequential C oracle, "
                                          f"1 thread)",
                                "host_cores": os.cpu_count()}
        bt = line["batched"]
        cb = batched_cpu_baseline()
        picks, odig = cb.pop("_models"), cb.pop("_digests")
        dfix, dlearn = bt.pop("_digest_fixed"), bt.pop("_digest_learned")
        ok_fixed = [int(dfix[m]) & (2**64 - 1) == d for m, d in zip(picks, odig)]
        ok_learned = [int(dlearn[m]) & (2**64 - 1) == d for m, d in zip(picks, odig)]
        bt["oracle_subset"] = {"models": len(picks), "steps": workloads.BATCH["steps"],
                               "fixed_bit_exact": sum(ok_fixed), "learned_bit_exact": sum(ok_learned),
                               "how": "digest of each sampled model's final state: oracle vs GPU batch"}
        bt["cpu_baseline"] = cb
        cb["full_batch_s_estimate"] = bt["fixed"]["agent_steps_per_s"] * bt["fixed"]["ms"] * 1e-3 / cb["value"]
        line["lob"]["cpu_baseline"] = lob_cpu_baseline()
        line["summary"] = summary(line)
    if rank == 0:
        print(json.dumps(line), flush=True)


def summary(line: dict) -> dict:
    """The three headline measurements in a few hundred bytes (printed last)."""
    su, bt, lob = line["selective_update"], line["batched"], line["lob"]
    r3 = lambda x: round(float(x), 3)  # noqa: E731
    return {
        "predation": {"agent_steps_per_s": r3(line["value"]), "us_per_step": r3(1e3 * line["ms_per_step"]),
                      "hbm_frac": r3(line["roofline"]["frac"]), "cpu_oracle": r3(line["cpu_baseline"]["value"]),
                      "e2e": r3(line["e2e"]["value"])},
        "selective_update_hbm_frac": {p: r3(su[p]["frac"]) for p in ("0.001", "0.05", "0.5") if p in su},
        "selective_update_gbs": {p: round(su[p]["gbs"]) for p in ("0.001", "0.05", "0.5") if p in su},
        "batched_ms": {"fixed": r3(bt["fixed"]["ms"]), "fixed_extent": r3(bt["fixed_extent_sweep"]["ms"]),
                       "learned": r3(bt["learned"]["ms"]), "learned_extent": r3(bt["learned_extent_sweep"]["ms"])},
        "learned_speedup": {"vs_fixed": r3(bt["learned"]["speedup_vs_fixed"]),
                            "extent_vs_fixed_extent": r3(bt["learned_extent_sweep"]["speedup_vs_fixed_extent_sweep"])},
        "learned_unrecovered": bt["learned"]["unrecovered_overflows"],
        "learned_bit_exact": bt["learned"]["bit_exact_vs_fixed"] and bt["learned_extent_sweep"]["bit_exact_vs_fixed"],
        "batched_oracle_subset": [bt["oracle_subset"]["fixed_bit_exact"], bt["oracle_subset"]["learned_bit_exact"],
                                  bt["oracle_subset"]["models"]],
        "lob_hbm_frac": r3(lob["roofline"]["frac"]),
    }


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
