"""Launch-shape autotuner (times candidates on the GPU, caches the winner).

Results never depend on the launch shape -- only the time does -- so the tuner
runs each candidate on a short, representative slice of the real work, keeps
the fastest, and records it in a JSON cache keyed by the device name and a
signature of the workload. Tuned knobs:

  batched runs    CTA size (threads), CTAs per SM, models per CTA, steps per launch
  large worlds    engine (persistent / per-phase kernels), CTAs per SM
  slab passes     CTA size, CTAs per SM of the fused selective-update call
"""
from __future__ import annotations

import hashlib
import json
import os
import time

import numpy as np
import torch

from . import abm, engine

CACHE = os.environ.get("ABM_TUNE_CACHE", os.path.join(os.path.expanduser("~"), ".cache", "abm_gb300_tune.json"))


def _key(kind: str, sig: dict) -> str:
    dev = torch.cuda.get_device_name()
    blob = json.dumps(sig, sort_keys=True, default=str)
    return f"{kind}|{dev}|{hashlib.sha1(blob.encode()).hexdigest()[:16]}"


def _load() -> dict:
    try:
        with open(CACHE) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store(key: str, value: dict):
    d = _load()
    d[key] = value
    try:
        os.makedirs(os.path.dirname(CACHE), exist_ok=True)
        tmp = CACHE + f".{os.getpid()}"
        with open(tmp, "w") as f:
            json.dump(d, f, indent=1, sort_keys=True)
        os.replace(tmp, CACHE)
    except OSError:
        pass


def _time(fn) -> float:
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    fn()
    e1.record()
    e1.synchronize()
    return e0.elapsed_time(e1)


def tune_batch(models: list, steps: int, sweep: int, trial_steps: int | None = None, rounds: int = 1,
               use_cache: bool = True, **_ignored) -> dict:
    """Pick (threads, ctas_per_sm, models_per_cta, agents_per_thread) for a batch of models. By default every
    candidate runs the whole batch for all `steps` from the initial state, so
    each times exactly the work it will be chosen for (populations change a
    lot over a run, so a short slice of it misjudges the shapes); a smaller
    trial_steps trades accuracy for tuning time, with candidates interleaved
    over `rounds` passes."""
    sig = {"n": len(models), "steps": steps, "sweep": sweep,
           "sides": np.histogram([m["side"] for m in models], bins=8)[0].tolist(),
           "cap": int(sum(int(m["cap"][0]) + int(m["cap"][1]) for m in models))}
    key = _key("batch3", sig)
    if use_cache:
        hit = _load().get(key)
        if hit:
            return hit
    # shapes whose CTAs can all be resident at 64 registers per thread: CTA
    # size, CTAs per SM, models per CTA (groups of at least 128 threads), agent
    # slots per thread in a sweep chunk (16 everywhere; 8 and 32 on the shapes
    # that came closest with 16; 32 needs at most 512 threads)
    cands = [(256, 1, 1, 16), (256, 2, 1, 16), (256, 4, 1, 16), (512, 1, 1, 16), (512, 2, 1, 16),
             (1024, 1, 1, 16), (256, 4, 2, 16), (512, 2, 2, 16), (512, 2, 4, 16), (1024, 1, 2, 16),
             (1024, 1, 4, 16), (512, 2, 1, 8), (1024, 1, 1, 8), (256, 4, 1, 8), (1024, 1, 2, 8),
             (512, 2, 1, 32), (256, 4, 1, 32), (512, 2, 2, 32), (256, 4, 2, 32)]
    acc = {cnd: 0.0 for cnd in cands}
    if trial_steps is None or trial_steps >= steps:
        for _ in range(rounds):
            for th, cps, g, a in cands:
                b = engine.Batch(models)
                b.tune(th, cps, models_per_cta=g, agents_per_thread=a)
                acc[(th, cps, g, a)] += _time(lambda: b.run(steps, sweep=sweep))
                b.check()
                del b
    else:
        b = engine.Batch(models)
        b.run(2, sweep=sweep)
        for _ in range(rounds):
            for th, cps, g, a in cands:
                b.tune(th, cps, models_per_cta=g, agents_per_thread=a)
                acc[(th, cps, g, a)] += _time(lambda: b.run(trial_steps, sweep=sweep))
        b.check()
        del b
    torch.cuda.empty_cache()
    results = sorted((ms, th, cps, g, a) for (th, cps, g, a), ms in acc.items())
    ms, th, cps, g, a = results[0]
    best = {"threads": th, "ctas_per_sm": cps, "models_per_cta": g, "agents_per_thread": a,
            "steps_per_launch": max(steps, 1), "trial_ms": ms,
            "trials": [{"threads": t, "ctas_per_sm": c, "models_per_cta": gg, "agents_per_thread": aa, "ms": m}
                       for m, t, c, gg, aa in results],
            "tuned_at": time.strftime("%Y-%m-%dT%H:%M:%S")}
    _store(key, best)
    return best


def tune_world(cfg: dict, warm_steps: int = 5, trial_steps: int = 30, use_cache: bool = True) -> dict:
    """Pick the engine and CTAs per SM for one large predation world."""
    sig = {k: (list(v) if isinstance(v, (tuple, list, np.ndarray)) else v) for k, v in cfg.items()
           if k in ("side", "n0", "cap")}
    key = _key("world", sig)
    if use_cache:
        hit = _load().get(key)
        if hit:
            return hit
    results = []
    for eng, cps in ((abm.ENGINE_PERSISTENT, 1), (abm.ENGINE_PERSISTENT, 2), (abm.ENGINE_KERNELS, 1)):
        w = engine.World(cfg["side"], cfg["seed"], cfg["model"], cfg["params"], cfg["cap"], cfg["n0"])
        try:
            w.tune(eng, cps)
        except abm.AbmError:
            continue
        w.step(warm_steps)
        ms = _time(lambda: w.step(trial_steps))
        w.check()
        del w
        results.append((ms, eng, cps))
    results.sort()
    ms, eng, cps = results[0]
    best = {"engine": eng, "ctas_per_sm": cps, "trial_ms": ms,
            "trials": [{"engine": e, "ctas_per_sm": c, "ms": m} for m, e, c in results]}
    _store(key, best)
    return best


def tune_slab(n: int, F: int, p: float, k: int, seed: int = 0, reps: int = 4, use_cache: bool = True) -> dict:
    """Pick (threads, ctas_per_sm) of the fused selective-update call. The slab
    is first brought to the state repeated calls settle in (each call refills
    half of the free slots, so the slab fills up over the first calls), then
    the candidates take turns, `reps` rounds, so that all see the same state."""
    key = _key("slab2", {"n": n, "F": F, "p": p, "k": k})
    if use_cache:
        hit = _load().get(key)
        if hit:
            return hit
    T = int(p * 2**32)
    s = engine.Slab(n, F, seed=seed, init=abm.INIT_HALF_LIVE)
    rec = s.philox_records(0, abm.P_NEWREC0, abm.P_NEWREC1, k).clone()
    dl = s.philox_records(0, abm.P_DELTA0, abm.P_DELTA1, k).clone()
    step = 0
    for _ in range(8):
        s.selective_update(step, T, rec, dl)
        step += 1
    cands = [(th, cps) for th in (128, 256, 512) for cps in (2, 4, 8, 16) if th * cps <= 2048]
    acc = {c: [] for c in cands}
    for _ in range(reps):
        for th, cps in cands:
            s.tune(th, cps)
            acc[(th, cps)].append(_time(lambda: s.selective_update(step, T, rec, dl)))
            step += 1
    results = [(float(np.median(v)), th, cps) for (th, cps), v in acc.items()]
    s.check()
    results.sort()
    ms, th, cps = results[0]
    best = {"threads": th, "ctas_per_sm": cps, "trial_ms": ms}
    _store(key, best)
    return best
