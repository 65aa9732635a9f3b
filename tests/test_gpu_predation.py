"""GPU parity: the predation step (Section 5.1) vs the sequential oracle.

The whole state -- every slot of both species (live flag, cell, energy, id,
age, including the stale fields of placeholders), the grass (grown flag and
steps until edible), the counters and the per-step statistics -- is compared
bit for bit.
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


def oracle_wait(ow):
    grown = ow.grass("grown")
    cd = ow.grass("countdown")
    return grown, np.where(grown != 0, 0, np.maximum(cd, 1))


def compare_state(gw, ow, where=""):
    torch.cuda.synchronize()
    for s, name in ((0, "sheep"), (1, "wolf")):
        for f in FIELDS:
            g = gw.agents(s, f).cpu().numpy()
            o = ow.agents(s, f)
            if not np.array_equal(g, o):
                bad = np.flatnonzero(g != o)
                raise AssertionError(f"{where} {name}.{f}: {bad.size} slots differ, first {bad[:5]} "
                                     f"gpu {g[bad[:5]]} oracle {o[bad[:5]]}")
    grown, wait = oracle_wait(ow)
    np.testing.assert_array_equal(gw.grass("grown").cpu().numpy(), grown, err_msg=f"{where} grown")
    np.testing.assert_array_equal(gw.grass("wait").cpu().numpy(), wait, err_msg=f"{where} wait")
    gc, oc = gw.counters(), ow.counters()
    for k in ("n_active", "next_id", "hw", "overflow", "step"):
        assert gc[k] == oc[k], (where, k, gc[k], oc[k])


def compare_stats(gst, ost, energy=True):
    keys = ["n_start", "parents", "births", "starved", "eaten", "grass_eaten", "n_end", "hw", "overflow"]
    if energy:
        keys.append("energy")
    for k in keys:
        assert gst[k] == ost[k], (k, gst[k], ost[k])


def make(eng, c, seed=None, engine=0):
    seed = c["seed"] if seed is None else seed
    gw = eng.World(c["side"], seed, c["model"], c["params"], c["cap"], c["n0"])
    gw.tune(engine)
    ow = oracle.World(c["side"], seed, c["model"], c["params"], c["cap"], c["n0"])
    return gw, ow


ENGINES = [0, 1]  # persistent cooperative kernel, six kernels per step


def energies(gw):
    e = []
    for s in range(2):
        a = gw.agents(s, "active").cpu().numpy().astype(bool)
        e.append(int(gw.agents(s, "energy").cpu().numpy()[a].astype(np.int64).sum()))
    return e


@pytest.mark.parametrize("engine", ENGINES)
def test_small_config_every_step(eng, engine):
    """40x40, 100 sheep / 25 wolves, capacity 2048/1024, 200 steps, seed 0."""
    c = workloads.PRED_SMALL
    gw, ow = make(eng, c, engine=engine)
    compare_state(gw, ow, "init")
    stats = gw.new_stats(1)
    for t in range(c["steps"]):
        gw.step(1, stats, want_energy=engine == 1)
        ost = ow.step()[0]
        gst = eng.decode_stats(stats)[0]
        compare_stats(gst, ost, energy=engine == 1)
        if engine == 0:
            assert energies(gw) == ost["energy"]
        assert gst["step"] == t
        compare_state(gw, ow, f"step {t}")
    gw.check()
    # and the stored trajectory
    import os
    traj = np.loadtxt(os.path.join(os.path.dirname(__file__), "golden", "pred_small_trajectory.txt"),
                      dtype=np.int64, comments="#")
    assert traj[-1].tolist() == [c["steps"] - 1] + gw.counters()["n_active"]


@pytest.mark.parametrize("engine", ENGINES)
@pytest.mark.parametrize("seed", range(24))
def test_random_small_worlds(eng, seed, engine):
    rng = np.random.default_rng(500 + seed)
    side = int(rng.integers(1, 40))
    cap = (int(rng.integers(1, 700)), int(rng.integers(1, 300)))
    n0 = (int(rng.integers(0, cap[0] + 1)), int(rng.integers(0, cap[1] + 1)))
    params = workloads.predation_params(
        sheep_gain=int(rng.integers(0, 8)), wolf_gain=int(rng.integers(0, 30)),
        sheep_repro=float(rng.choice([0.0, 0.04, 0.3, 0.9])), wolf_repro=float(rng.choice([0.0, 0.05, 0.5])),
        regrowth=int(rng.integers(1, 40)), sheep_metab=int(rng.integers(0, 3)),
        wolf_metab=int(rng.integers(0, 3)), grass_init=float(rng.choice([0.1, 0.5, 0.95])))
    c = dict(side=side, n0=n0, cap=cap, seed=seed, model=int(rng.integers(0, 1000)), params=params)
    gw, ow = make(eng, c, engine=engine)
    stats = gw.new_stats(60)
    gw.step(60, stats, want_energy=engine == 1)
    ost = ow.step(60)
    for g, o in zip(eng.decode_stats(stats), ost):
        compare_stats(g, o, energy=engine == 1)
    compare_state(gw, ow, f"seed {seed}")
    gw.check()


def test_graph_replay_equals_eager(eng):
    c = dict(workloads.PRED_SMALL)
    a, _ = make(eng, c, engine=0)
    b, _ = make(eng, c, engine=1)
    sa = a.new_stats(25)
    sb = b.new_stats(25)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        for _ in range(4):
            a.step(25, sa)
        b.step_graph(25, 4, sb, stream=s)
    s.synchronize()
    assert torch.equal(sa, sb)
    for sp in range(2):
        for f in FIELDS:
            assert torch.equal(a.agents(sp, f), b.agents(sp, f))
    assert a.counters() == b.counters()


def test_checkpoint_resume_bit_exact(eng):
    c = dict(workloads.PRED_SMALL)
    a, ow = make(eng, c)
    a.step(50)
    img = a.save()
    a.step(70)
    b, _ = make(eng, c)
    b.load(img)
    b.step(70)
    for sp in range(2):
        for f in FIELDS:
            assert torch.equal(a.agents(sp, f), b.agents(sp, f))
    assert torch.equal(a.grass("wait"), b.grass("wait"))
    assert a.counters() == b.counters()
    ow.step(120)
    compare_state(b, ow, "resumed")


def test_checkpoint_image_follows_the_extent(eng):
    """The image holds each species' slots up to its extent: its size follows
    the extents, a larger buffer serves for both calls, a smaller one is
    refused, and a world that had run further than the image comes back with
    the slots past the image's extents empty -- the same state, slot for slot,
    as the oracle's."""
    from paper_2508_16508_gb300 import abm
    c = dict(workloads.PRED_SMALL)
    a, ow = make(eng, c)
    a.step(40)
    ow.step(40)
    cnt = a.counters()
    nb = a.image_bytes()
    cells = c["side"] * c["side"]
    hdr = nb - sum(e * 20 for e in cnt["extent"]) - 4 * cells
    assert 0 < hdr <= 256  # the counters
    assert a.image_capacity() == hdr + 20 * sum(c["cap"]) + 4 * cells
    big = torch.zeros(a.image_capacity() + 100, dtype=torch.uint8)
    assert a.save_into(big) == nb
    with pytest.raises(abm.AbmError):
        a.save_into(torch.zeros(nb - 1, dtype=torch.uint8))
    b, _ = make(eng, c)
    b.step(90)  # further than the image: larger extents, other records
    assert any(x > y for x, y in zip(b.counters()["extent"], cnt["extent"]))
    with pytest.raises(abm.AbmError):
        b.load_from(big[: nb - 1])
    b.load_from(big)
    compare_state(b, ow, "loaded")
    b.step(30)
    ow.step(30)
    compare_state(b, ow, "resumed")


@pytest.mark.parametrize("engine", ENGINES)
def test_stats_into_pinned_host_memory(eng, engine):
    """abm_step writes its statistics rows straight into pinned host memory
    (unified addressing): the rows equal those written to device memory."""
    from paper_2508_16508_gb300 import abm
    c = dict(workloads.PRED_SMALL)
    a, _ = make(eng, c, engine=engine)
    b, _ = make(eng, c, engine=engine)
    dev = a.new_stats(12)
    host = torch.zeros((12, abm.STATS_WORDS), dtype=torch.int32).pin_memory()
    for i in range(12):  # one call per step, as an end-to-end loop makes them
        a.step(1, dev[i:i + 1])
        b.step(1, host[i:i + 1])
    torch.cuda.synchronize()
    assert torch.equal(dev.cpu(), host)
    assert eng.decode_stats(host)[11]["step"] == 11


def test_overflow_truncates_like_oracle(eng):
    params = workloads.predation_params(sheep_repro=0.5, wolf_repro=0.5, sheep_gain=6)
    c = dict(side=10, n0=(30, 10), cap=(40, 20), seed=3, model=0, params=params)
    gw, ow = make(eng, c)
    gw.step(60)
    ow.step(60)
    compare_state(gw, ow, "overflow")
    assert max(gw.counters()["overflow"]) == 1


@pytest.mark.parametrize("engine", ENGINES)
def test_large_config_first_steps(eng, engine):
    """2048x2048, 1M sheep / 250k wolves, capacity 8Mi / 4Mi: 12 steps, full state."""
    c = workloads.PRED_LARGE
    gw, ow = make(eng, c, engine=engine)
    compare_state(gw, ow, "init")
    stats = gw.new_stats(12)
    gw.step(12, stats, want_energy=engine == 1)
    ost = ow.step(12)
    for g, o in zip(eng.decode_stats(stats), ost):
        compare_stats(g, o, energy=engine == 1)
    compare_state(gw, ow, "step 12")
    gw.check()


def test_large_config_engines_agree_over_300_steps(eng):
    """Both engines over 300 steps of the large run (through the population
    crash and recovery), whole state compared."""
    c = workloads.PRED_LARGE
    a, _ = make(eng, c, engine=0)
    b, _ = make(eng, c, engine=1)
    sa, sb = a.new_stats(300), b.new_stats(300)
    a.step(300, sa)
    b.step(300, sb)
    torch.cuda.synchronize()
    ra, rb = eng.decode_stats(sa), eng.decode_stats(sb)
    for x, y in zip(ra, rb):
        for k in ("n_start", "parents", "births", "starved", "eaten", "grass_eaten", "n_end", "hw", "overflow"):
            assert x[k] == y[k], (k, x["step"])
    for s in range(2):
        for f in FIELDS:
            assert torch.equal(a.agents(s, f), b.agents(s, f)), (s, f)
    assert torch.equal(a.grass("wait"), b.grass("wait"))
    assert a.counters() == b.counters()
    a.check()


def test_large_config_one_cta_per_sm_multi_round(eng):
    """The persistent engine at one CTA per SM (the 128-register variant):
    the sheep extent then spans more than one round of units per CTA, so the
    move and count phases take the multi-round path. 150 steps, whole state,
    against the per-phase kernel engine."""
    c = workloads.PRED_LARGE
    a, _ = make(eng, c, engine=0)
    a.tune(0, 1)
    b, _ = make(eng, c, engine=1)
    sa, sb = a.new_stats(150), b.new_stats(150)
    for i in range(3):  # several launches: the barrier counter carries over
        a.step(50, sa[i * 50:(i + 1) * 50])
    b.step(150, sb)
    torch.cuda.synchronize()
    for x, y in zip(eng.decode_stats(sa), eng.decode_stats(sb)):
        for k in ("n_start", "parents", "births", "starved", "eaten", "grass_eaten", "n_end", "hw", "overflow"):
            assert x[k] == y[k], (k, x["step"])
    for s in range(2):
        for f in FIELDS:
            assert torch.equal(a.agents(s, f), b.agents(s, f)), (s, f)
    assert torch.equal(a.grass("wait"), b.grass("wait"))
    assert a.counters() == b.counters()
    a.check()


def test_engine_switches_mid_run(eng):
    """Steps alternate between the engines and launch shapes on one world;
    the result equals the oracle's."""
    c = workloads.PRED_SMALL
    gw, ow = make(eng, c)
    plan = [(0, 2, 7), (1, 1, 5), (0, 1, 9), (0, 2, 1), (1, 1, 3), (0, 2, 25)]
    for engine, cps, n in plan:
        gw.tune(engine, cps)
        gw.step(n)
    ow.step(sum(n for _, _, n in plan))
    compare_state(gw, ow, "switches")
    gw.check()


@pytest.mark.slow
def test_large_config_full_run(eng):
    """The full 1000-step large run: populations every step, full state at the end."""
    c = workloads.PRED_LARGE
    gw, ow = make(eng, c, engine=0)
    stats = gw.new_stats(c["steps"])
    gw.step(c["steps"], stats)
    ost = ow.step(c["steps"])
    for g, o in zip(eng.decode_stats(stats), ost):
        compare_stats(g, o, energy=False)
    compare_state(gw, ow, "end")
    gw.check()


def test_create_argument_errors(eng):
    from paper_2508_16508_gb300 import abm
    import ctypes as C
    cfg = abm.abm_config()
    cfg.side = 0
    h = C.c_void_p()
    assert abm.lib().abm_create(C.byref(cfg), None, C.byref(h)) == abm.ERR_ARG
    cfg.side, cfg.cap[0], cfg.cap[1], cfg.n0[0] = 10, 5, 5, 6
    cfg.params[4] = 3
    assert abm.lib().abm_create(C.byref(cfg), None, C.byref(h)) == abm.ERR_ARG


def test_large_config_full_run_vs_stored_oracle(eng):
    """All 1000 steps of the large run on the persistent engine: every step's
    counts against the oracle's stored trajectory, and the SHA-256 of the final
    state against the oracle's (tests/golden/make_golden.py large)."""
    import os
    import sys
    path = os.path.join(os.path.dirname(__file__), "golden", "pred_large_trajectory.txt")
    if not os.path.exists(path):
        pytest.skip("stored large trajectory not written")
    sys.path.insert(0, os.path.join(os.path.dirname(__file__), "golden"))
    from make_golden import state_sha256
    with open(path) as f:
        want_sha = [ln.split()[2] for ln in f if ln.startswith("# final_state_sha256")][0]
    want = np.loadtxt(path, dtype=np.int64, comments="#")
    c = workloads.PRED_LARGE
    gw = eng.World(c["side"], c["seed"], c["model"], c["params"], c["cap"], c["n0"])
    stats = gw.new_stats(c["steps"])
    gw.step(c["steps"], stats)
    got = np.array([[r["step"], *r["n_start"], *r["parents"], *r["births"], *r["starved"], r["eaten"],
                     r["grass_eaten"], *r["n_end"], *r["hw"]] for r in eng.decode_stats(stats)])
    np.testing.assert_array_equal(got, want)
    st = {}
    for s, name in ((0, "sheep"), (1, "wolf")):
        for f in FIELDS:
            st[f"{name}.{f}"] = gw.agents(s, f).cpu().numpy()
    st["grass.grown"] = gw.grass("grown").cpu().numpy()
    st["grass.wait"] = gw.grass("wait").cpu().numpy()
    assert state_sha256(st) == want_sha
    gw.check()
