"""GPU parity of the rule variants against the oracle's (which are pinned by
the list-of-agents simulator): several wolves per cell (the i-th wolf of a
cell, by (PRIO draw, slot), eats the i-th sheep, by (VICTIM draw, slot)),
grass off (sheep neither eat nor spend energy), and both. Whole state, bit
for bit."""
import numpy as np
import pytest

import oracle
import workloads
from test_gpu_predation import FIELDS, compare_state, compare_stats

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def eng():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2508_16508_gb300 import abm, engine
    abm.lib()
    return engine


MANY, OFF = oracle.VARIANT_MANY_WOLVES, oracle.VARIANT_GRASS_OFF
VARIANTS = [MANY, OFF, MANY | OFF]


def make(eng, c, cps=2, variant=MANY):
    from paper_2508_16508_gb300 import abm
    gw = eng.World(c["side"], c["seed"], c["model"], c["params"], c["cap"], c["n0"], variant=variant)
    gw.tune(abm.ENGINE_PERSISTENT, cps)
    ow = oracle.World(c["side"], c["seed"], c["model"], c["params"], c["cap"], c["n0"], variant=variant)
    return gw, ow


@pytest.mark.parametrize("variant", VARIANTS)
def test_small_config_every_step(eng, variant):
    c = workloads.PRED_SMALL
    gw, ow = make(eng, c, variant=variant)
    stats = gw.new_stats(1)
    eaten = 0
    for t in range(c["steps"]):
        gw.step(1, stats)
        ost = ow.step()[0]
        compare_stats(eng.decode_stats(stats)[0], ost, energy=False)
        compare_state(gw, ow, f"step {t}")
        eaten += ost["eaten"]
        if variant & OFF:
            assert ost["grass_eaten"] == 0
    assert eaten > 0
    gw.check()


@pytest.mark.parametrize("seed", range(20))
def test_crowded_random_worlds(eng, seed):
    """Small worlds with many wolves per cell, several launches."""
    rng = np.random.default_rng(900 + seed)
    side = int(rng.integers(1, 12))
    cap = (int(rng.integers(1, 500)), int(rng.integers(1, 400)))
    n0 = (int(rng.integers(0, cap[0] + 1)), int(rng.integers(0, cap[1] + 1)))
    params = workloads.predation_params(
        sheep_gain=int(rng.integers(0, 8)), wolf_gain=int(rng.integers(0, 30)),
        sheep_repro=float(rng.choice([0.0, 0.04, 0.3, 0.9])), wolf_repro=float(rng.choice([0.0, 0.05, 0.5])),
        regrowth=int(rng.integers(1, 40)), grass_init=float(rng.choice([0.1, 0.5, 0.95])))
    c = dict(side=side, n0=n0, cap=cap, seed=seed, model=int(rng.integers(0, 1000)), params=params)
    gw, ow = make(eng, c, variant=VARIANTS[seed % 3])
    stats = gw.new_stats(60)
    for k in range(3):
        gw.step(20, stats[20 * k:20 * (k + 1)])
    ost = ow.step(60)
    for g, o in zip(eng.decode_stats(stats), ost):
        compare_stats(g, o, energy=False)
    compare_state(gw, ow, f"seed {seed}")
    gw.check()


def test_large_config_first_steps(eng):
    c = workloads.PRED_LARGE
    gw, ow = make(eng, c)
    stats = gw.new_stats(10)
    gw.step(10, stats)
    ost = ow.step(10)
    for g, o in zip(eng.decode_stats(stats), ost):
        compare_stats(g, o, energy=False)
    compare_state(gw, ow, "step 10")
    gw.check()


def test_large_config_launch_shapes_agree(eng):
    """One CTA per SM (units over several rounds) and two CTAs per SM, 150 steps."""
    c = workloads.PRED_LARGE
    a, _ = make(eng, c, cps=2)
    b, _ = make(eng, c, cps=1)
    sa, sb = a.new_stats(150), b.new_stats(150)
    a.step(150, sa)
    for k in range(3):
        b.step(50, sb[50 * k:50 * (k + 1)])
    torch.cuda.synchronize()
    assert torch.equal(sa, sb)
    for s in range(2):
        for f in FIELDS:
            assert torch.equal(a.agents(s, f), b.agents(s, f)), (s, f)
    a.check()
    b.check()


def test_variant_refuses_per_phase_kernels(eng):
    from paper_2508_16508_gb300 import abm
    gw, _ = make(eng, workloads.PRED_SMALL)
    with pytest.raises(abm.AbmError):
        gw.tune(abm.ENGINE_KERNELS)
    with pytest.raises(abm.AbmError):
        gw.step(1, gw.new_stats(1), want_energy=True)
    with pytest.raises(abm.AbmError):
        gw.step_graph(2, 1, stream=torch.cuda.current_stream())
