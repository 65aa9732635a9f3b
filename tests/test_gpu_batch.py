"""GPU parity: the batched many-model runner vs the oracle, model by model.

Both sweeps (whole capacity, extent) must give the oracle's state bit for bit,
for any split of the run into launches and any launch shape.
"""
import numpy as np
import pytest

import oracle
import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FIELDS = ("active", "cell", "energy", "id", "age")


@pytest.fixture(scope="module")
def eng():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2508_16508_gb300 import abm, engine
    abm.lib()
    return engine


def random_models(n, seed, max_side=40):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        side = int(rng.integers(1, max_side))
        cap = (int(rng.integers(1, 500)), int(rng.integers(1, 300)))
        n0 = (int(rng.integers(0, cap[0] + 1)), int(rng.integers(0, cap[1] + 1)))
        params = workloads.predation_params(
            sheep_gain=int(rng.integers(0, 8)), wolf_gain=int(rng.integers(0, 30)),
            sheep_repro=float(rng.choice([0.0, 0.04, 0.3, 0.9])),
            wolf_repro=float(rng.choice([0.0, 0.05, 0.5])), regrowth=int(rng.integers(1, 40)),
            sheep_metab=int(rng.integers(0, 3)), wolf_metab=int(rng.integers(0, 3)),
            grass_init=float(rng.choice([0.1, 0.5, 0.95])))
        out.append(dict(side=side, seed=int(rng.integers(0, 2**32)), model=i, params=params,
                        cap=cap, n0=n0))
    return out


def compare_model(b, m, ow, where):
    for s in range(2):
        for f in FIELDS:
            g = b.agents(m, s, f).cpu().numpy()
            o = ow.agents(s, f)
            assert np.array_equal(g, o), (where, m, s, f, np.flatnonzero(g != o)[:5])
    grown = ow.grass("grown")
    wait = np.where(grown != 0, 0, np.maximum(ow.grass("countdown"), 1))
    assert np.array_equal(b.grass(m, "grown").cpu().numpy(), grown), (where, m)
    assert np.array_equal(b.grass(m, "wait").cpu().numpy(), wait), (where, m)


@pytest.mark.parametrize("sweep", [0, 1])
@pytest.mark.parametrize("threads,spl,mpc,apt", [(256, 1 << 30, 1, 16), (128, 7, 1, 16), (512, 13, 1, 16),
                                                 (256, 11, 2, 16), (512, 1 << 30, 4, 16), (1024, 9, 2, 16),
                                                 (1024, 1 << 30, 4, 16), (512, 17, 2, 16), (256, 1 << 30, 1, 8),
                                                 (128, 7, 1, 8), (1024, 9, 2, 8), (512, 17, 4, 8),
                                                 (512, 1 << 30, 1, 32), (256, 13, 2, 32), (128, 5, 1, 32)])
def test_random_batch_vs_oracle(eng, sweep, threads, spl, mpc, apt):
    """Every launch shape (CTA size, steps per launch, models per CTA, slots
    per thread in a sweep chunk) gives the oracle's models."""
    models = random_models(20, 100 + threads + sweep + 7 * mpc + apt)
    b = eng.Batch(models)
    b.tune(threads, 2 if threads < 1024 else 1, spl, models_per_cta=mpc, agents_per_thread=apt)
    b.run(45, sweep=sweep)
    cnt = b.counters()
    for m, md in enumerate(models):
        ow = oracle.World(md["side"], md["seed"], md["model"], md["params"], md["cap"], md["n0"])
        agents = 0
        for st in ow.step(45):
            agents += st["n_start"][0] + st["n_start"][1]
        compare_model(b, m, ow, f"sweep {sweep}")
        oc = ow.counters()
        for k in ("n_active", "next_id", "hw", "overflow", "step"):
            assert cnt[m][k] == oc[k], (m, k, cnt[m][k], oc[k])
        assert cnt[m]["agent_steps"] == agents
    b.check()


def test_small_config_as_one_model_batch(eng):
    c = workloads.PRED_SMALL
    b = eng.Batch([dict(side=c["side"], seed=c["seed"], model=c["model"], params=c["params"],
                        cap=c["cap"], n0=c["n0"])])
    ow = oracle.World(c["side"], c["seed"], c["model"], c["params"], c["cap"], c["n0"])
    for t in range(0, c["steps"], 20):
        b.run(20)
        ow.step(20)
        compare_model(b, 0, ow, f"step {t + 20}")


def test_batched_sampler_subset(eng):
    """Models drawn by the batched workload's sampler, fixed capacity 4 side^2."""
    tab = workloads.sample_models(4096, workloads.BATCH["sampler_seed"])
    caps = workloads.fixed_caps(tab["side"])
    rng = np.random.default_rng(0)
    pick = sorted(rng.choice(4096, size=12, replace=False).tolist())
    models = [dict(side=int(tab["side"][i]), seed=workloads.BATCH["philox_seed"], model=i,
                   params=tab["params"][i], cap=caps[i], n0=tab["n0"][i]) for i in pick]
    b = eng.Batch(models)
    b.run(60, sweep=0)
    for m, md in enumerate(models):
        ow = oracle.World(md["side"], md["seed"], md["model"], md["params"], md["cap"], md["n0"])
        ow.step(60)
        compare_model(b, m, ow, "sampler")


def test_overflow_list(eng):
    params = workloads.predation_params(sheep_repro=0.5, wolf_repro=0.5, sheep_gain=6)
    models = [dict(side=10, seed=3, model=i, params=params, cap=(40 if i % 2 else 4000, 2000), n0=(30, 10))
              for i in range(6)]
    b = eng.Batch(models)
    b.run(40, sweep=1)
    ov = b.overflowed()
    want = []
    for m, md in enumerate(models):
        ow = oracle.World(md["side"], md["seed"], md["model"], md["params"], md["cap"], md["n0"])
        ow.step(40)
        if max(ow.counters()["overflow"]):
            want.append(m)
        compare_model(b, m, ow, "overflow")
    assert ov == want and len(want) > 0


@pytest.mark.parametrize("sweep", [0, 1])
def test_sampler_models_full_horizon(eng, sweep):
    """The batched workload at its own horizon: 10 models of its sampler with
    sides spread over [16, 256] (fixed capacity 4 side^2) run all 500 steps in
    one launch, against the oracle model by model (whole state and counters).
    In this workload the wolves boom and eat the sheep; on the oracle these
    models lose their sheep by step 8-23 and their wolves by step 53-137, so
    the horizon covers growth, collapse and the empty slabs after it."""
    B = workloads.BATCH
    tab = workloads.sample_models(B["n_models"], B["sampler_seed"])
    caps = workloads.fixed_caps(tab["side"])
    order = np.argsort(tab["side"], kind="stable")
    pick = [int(order[int(q)]) for q in np.linspace(0, len(order) - 1, 10)]
    models = [dict(side=int(tab["side"][i]), seed=B["philox_seed"], model=i, params=tab["params"][i],
                   cap=caps[i], n0=tab["n0"][i]) for i in pick]
    b = eng.Batch(models)
    b.run(B["steps"], sweep=sweep)
    cnt = b.counters()
    b.check()
    for m, md in enumerate(models):
        ow = oracle.World(md["side"], md["seed"], md["model"], md["params"], md["cap"], md["n0"])
        agents = sum(st["n_start"][0] + st["n_start"][1] for st in ow.step(B["steps"]))
        compare_model(b, m, ow, f"model {pick[m]} (side {md['side']})")
        oc = ow.counters()
        for k in ("n_active", "next_id", "hw", "overflow", "step"):
            assert cnt[m][k] == oc[k], (pick[m], k, cnt[m][k], oc[k])
        assert cnt[m]["agent_steps"] == agents


def test_batch_run_replays_from_a_cuda_graph(eng):
    """A batch run's launches can be captured in a CUDA graph and replayed: the
    model queue resets itself at the end of every launch, so three replays of a
    captured 10-step launch give the same models as 30 eager steps."""
    models = random_models(12, 4242)
    a = eng.Batch(models)
    a.tune(256, 2, 10)
    a.run(30)
    warm = eng.Batch(models)  # the launch shape's first use (attributes) outside the capture
    warm.tune(256, 2, 10)
    warm.run(10)
    torch.cuda.synchronize()
    b = eng.Batch(models)
    b.tune(256, 2, 10)
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        b.run(10, stream=s)
    for _ in range(3):
        g.replay()
    torch.cuda.synchronize()
    assert torch.equal(a.digest(), b.digest())
    assert [c["step"] for c in b.counters()] == [30] * len(models)
