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
    assert autotune.tune_batch(models, 30, abm.SWEEP_CAPACITY) == best  # cached
    digests = []
    for th, cps in ((best["threads"], best["ctas_per_sm"]), (256, 1), (1024, 2)):
        b = engine.Batch(models)
        b.tune(th, cps, 7)
        b.run(30)
        digests.append(b.digest().cpu().numpy())
    assert all(np.array_equal(d, digests[0]) for d in digests)
    c = dict(workloads.PRED_SMALL)
    w = autotune.tune_world(c, trial_steps=5)
    assert w["engine"] in (abm.ENGINE_PERSISTENT, abm.ENGINE_KERNELS)
    sl = autotune.tune_slab(20000, 8, 0.05, 1000, reps=1)
    assert sl["threads"] in (128, 256, 512)
