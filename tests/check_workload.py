"""Workloads run by tests/test_gpu_check.py in both the normal and the check
build of the library (the check build is chosen by ABM_LIBRARY=check, which
must be set before the binding is imported). Prints one JSON object: the
digests of every result and the status of every *_check call."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402
import torch  # noqa: E402

import workloads  # noqa: E402


def tensor_digest(*ts) -> str:
    import hashlib
    h = hashlib.sha256()
    for t in ts:
        h.update(t.detach().cpu().numpy().tobytes())
    return h.hexdigest()[:32]


def status(fn, *args) -> int:
    from paper_2508_16508_gb300 import abm
    return int(fn(*args))


def run() -> dict:
    from paper_2508_16508_gb300 import abm, engine
    L = abm.lib()
    st = abm.stream_handle()
    out = {"version": int(L.abm_version()), "digests": {}, "checks": {}}
    d, ck = out["digests"], out["checks"]
    c = workloads.PRED_SMALL
    for eng_kind in (abm.ENGINE_PERSISTENT, abm.ENGINE_KERNELS):
        w = engine.World(c["side"], c["seed"], c["model"], c["params"], c["cap"], c["n0"])
        w.tune(eng_kind, 2)
        w.step(c["steps"])
        d[f"small_{eng_kind}"] = w.digest() & ((1 << 64) - 1)
        ck[f"small_{eng_kind}"] = status(L.abm_world_check, w.h, st)
    big = workloads.PRED_LARGE
    w = engine.World(big["side"], big["seed"], big["model"], big["params"], big["cap"], big["n0"])
    w.step(30)
    d["large_30"] = w.digest() & ((1 << 64) - 1)
    ck["large_30"] = status(L.abm_world_check, w.h, st)
    # a world's sheep edited as a Set, then stepped on
    w = engine.World(c["side"], c["seed"], c["model"], c["params"], c["cap"], c["n0"])
    w.step(10)
    v = w.slab(0)
    v.remove(abm.pred(abm.PRED_BERNOULLI, threshold=workloads.threshold(0.3), step=77, purpose=abm.P_MASK))
    rec = torch.tensor([[5, 3, 0, 1]] * 9, dtype=torch.int32, device="cuda")
    v.add(rec, id_field=2)
    w.slab_commit(0)
    w.step(20)
    d["world_slab"] = w.digest() & ((1 << 64) - 1)
    ck["world_slab"] = status(L.abm_world_check, w.h, st)
    ck["world_slab_view"] = status(L.abm_slab_check, v.h, st)
    # batches in both sweeps, and a learned-capacity rerun
    rng = np.random.default_rng(3)
    models = []
    for i in range(24):
        side = int(rng.integers(4, 40))
        cap = (int(rng.integers(40, 500)), int(rng.integers(20, 300)))
        n0 = (int(rng.integers(0, cap[0] // 2)), int(rng.integers(0, cap[1] // 2)))
        params = workloads.predation_params(sheep_repro=0.2, wolf_repro=0.1, sheep_gain=5)
        models.append(dict(side=side, seed=9, model=i, params=params, cap=cap, n0=n0))
    for sweep in (abm.SWEEP_CAPACITY, abm.SWEEP_EXTENT):
        b = engine.Batch(models)
        b.run(45, sweep=sweep)
        d[f"batch_{sweep}"] = tensor_digest(b.digest())
        ck[f"batch_{sweep}"] = status(L.abm_batch_check, b.h, st)
    small = [dict(m, cap=(max(m["n0"][0], 8), max(m["n0"][1], 8))) for m in models]
    b = engine.Batch(small)
    b.run(45, sweep=abm.SWEEP_CAPACITY)
    nr, nu = b.rerun_overflowed(np.array([m["cap"] for m in models], np.int32))
    d["rerun"] = [nr, nu, tensor_digest(b.digest())]
    ck["rerun"] = status(L.abm_batch_check, b.h, st)
    # slab calls: both selective-update paths, select, sort, add / remove / update
    n = 100_003
    s = engine.Slab(n, 8, seed=2, init=abm.INIT_HALF_LIVE)
    for step, p in enumerate((0.05, 0.5, 0.001)):
        k = workloads.k_for(p, n)
        r1 = s.philox_records(step, abm.P_NEWREC0, abm.P_NEWREC1, k)
        r2 = s.philox_records(step, abm.P_DELTA0, abm.P_DELTA1, k)
        s.selective_update(step, workloads.threshold(p), r1, r2)
    idx, cnt = s.select(abm.pred(abm.PRED_FIELD, field=3, cmp=abm.CMP_LT, value=0))
    s.add(torch.arange(800, dtype=torch.int32, device="cuda").reshape(100, 8), id_field=1)
    s.update_distinct(abm.pred(abm.PRED_LIVE), torch.ones((500, 8), dtype=torch.int32, device="cuda"))
    perm = s.sort(5)
    d["slab"] = tensor_digest(s.read(-1), s.fields(), idx[: int(cnt.item())], perm)
    ck["slab"] = status(L.abm_slab_check, s.h, st)
    return out


if __name__ == "__main__":
    torch.cuda.set_device(0)
    print(json.dumps(run()))
