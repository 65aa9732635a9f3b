"""The autotuner picks a launch shape by timing; results never depend on it."""
import numpy as np
import pytest

import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_tune_batch_and_world_and_slab(tmp_path, monkeypatch):
    assert torch.cuda.is_available()
    from paper_2508_16508_gb300 import abm, autotune, engine
    monkeypatch.setattr(autotune, "CACHE", str(tmp_path / "tune.json"))
    tab = workloads.sample_models(200, 7, side_lo=16, side_hi=64)
    caps = workloads.fixed_caps(tab["side"])
    models = [dict(side=int(tab["side"][i]), seed=1, model=i, params=tab["params"][i], cap=caps[i], n0=tab["n0"][i])
              for i in range(200)]
    best = autotune.tune_batch(models, 30, abm.SWEEP_CAPACITY, trial_steps=3, rounds=1)
    assert best["threads"] in (256, 512, 1024) and best["ctas_per_sm"] in (1, 2, 4)
    assert best["models_per_cta"] in (1, 2, 4) and best["threads"] // best["models_per_cta"] >= 128
    assert best["agents_per_thread"] in (8, 16, 32)
    assert autotune.tune_batch(models, 30, abm.SWEEP_CAPACITY) == best  # cached
    digests = []
    for th, cps, g, a in ((best["threads"], best["ctas_per_sm"], best["models_per_cta"], best["agents_per_thread"]),
                          (256, 1, 1, 16), (1024, 2, 1, 8), (1024, 1, 4, 16), (512, 2, 2, 8), (512, 2, 1, 32)):
        b = engine.Batch(models)
        b.tune(th, cps, 7, models_per_cta=g, agents_per_thread=a)
        b.run(30)
        digests.append(b.digest().cpu().numpy())
    assert all(np.array_equal(d, digests[0]) for d in digests)
    c = dict(workloads.PRED_SMALL)
    w = autotune.tune_world(c, trial_steps=5)
    assert w["engine"] in (abm.ENGINE_PERSISTENT, abm.ENGINE_KERNELS)
    sl = autotune.tune_slab(20000, 8, 0.05, 1000, reps=1)
    assert sl["threads"] in (128, 256, 512)


def test_models_per_cta_limits():
    """Groups keep at least 128 threads; a smaller CTA size resets the packing;
    a sweep chunk holds 8, 16 or 32 slots per thread (32 up to 512 threads)."""
    assert torch.cuda.is_available()
    from paper_2508_16508_gb300 import abm, engine
    c = workloads.PRED_SMALL
    b = engine.Batch([dict(side=c["side"], seed=c["seed"], model=c["model"], params=c["params"], cap=c["cap"],
                           n0=c["n0"])])
    L = abm.lib()
    assert L.abm_batch_tune(b.h, 512, 2, 100) == abm.OK
    assert L.abm_batch_models_per_cta(b.h, 4) == abm.OK
    assert L.abm_batch_models_per_cta(b.h, 3) == abm.ERR_ARG
    assert L.abm_batch_tune(b.h, 256, 2, 100) == abm.OK  # 256 / 4 < 128: back to one model per CTA
    assert L.abm_batch_models_per_cta(b.h, 4) == abm.ERR_ARG
    assert L.abm_batch_models_per_cta(b.h, 2) == abm.OK
    assert L.abm_batch_agents_per_thread(b.h, 8) == abm.OK
    assert L.abm_batch_agents_per_thread(b.h, 4) == abm.ERR_ARG
    assert L.abm_batch_agents_per_thread(b.h, 32) == abm.OK  # 256 threads
    assert L.abm_batch_tune(b.h, 1024, 1, 100) == abm.OK  # a larger CTA: back to 16 slots per thread
    assert L.abm_batch_agents_per_thread(b.h, 32) == abm.ERR_ARG
    assert L.abm_batch_agents_per_thread(b.h, 16) == abm.OK
