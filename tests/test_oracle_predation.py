"""Pins for the oracle's predation step (Section 5.1), CPU only.

The paper prints no trajectory, so the dynamics are pinned by (1) an
independent list-of-agents simulator on tiny worlds, (2) invariants checked
every step, (3) special cases with a known outcome.
"""
import numpy as np
import pytest

import oracle
import workloads
from brute_predation import BruteWorld


def compare(ow: oracle.World, bw: BruteWorld):
    L = bw.L
    for s, name in ((0, "sheep"), (1, "wolf")):
        act = ow.agents(s, "active")
        assert set(np.flatnonzero(act).tolist()) == set(bw.agents[s]), (name, bw.t)
        cell, e = ow.agents(s, "cell"), ow.agents(s, "energy")
        ids, age = ow.agents(s, "id"), ow.agents(s, "age")
        for slot, a in bw.agents[s].items():
            assert cell[slot] == a["y"] * L + a["x"]
            assert e[slot] == a["e"] and ids[slot] == a["id"] and age[slot] == a["age"]
    grown, cd = ow.grass("grown"), ow.grass("countdown")
    for (x, y), g in bw.grass.items():
        assert grown[y * L + x] == int(g["grown"])
        assert cd[y * L + x] == g["countdown"]
    c = ow.counters()
    assert c["next_id"] == bw.next_id and c["hw"] == bw.hw and c["overflow"] == bw.overflow


@pytest.mark.parametrize("seed", range(100))
def test_brute_force_tiny_worlds(seed):
    rng = np.random.default_rng(1000 + seed)
    side = int(rng.integers(1, 9))
    cap = (int(rng.integers(1, 24)), int(rng.integers(1, 16)))
    n0 = (int(rng.integers(0, cap[0] + 1)), int(rng.integers(0, cap[1] + 1)))
    params = workloads.predation_params(
        sheep_gain=int(rng.integers(1, 6)), wolf_gain=int(rng.integers(2, 25)),
        sheep_repro=float(rng.choice([0.04, 0.2, 0.5])), wolf_repro=float(rng.choice([0.05, 0.2, 0.5])),
        regrowth=int(rng.integers(1, 12)), grass_init=float(rng.choice([0.25, 0.5, 0.9])))
    ow = oracle.World(side, seed, 7, params, cap, n0)
    bw = BruteWorld(side, seed, 7, params, cap, n0)
    compare(ow, bw)
    for _ in range(50):
        st = ow.step()[0]
        bst = bw.step()
        assert st["grass_eaten"] == bst["grass_eaten"] and st["eaten"] == bst["eaten"]
        assert st["births"] == [bst["births0"], bst["births1"]]
        assert st["starved"] == [bst["starved0"], bst["starved1"]]
        assert st["parents"] == [bst["parents0"], bst["parents1"]]
        compare(ow, bw)


@pytest.mark.parametrize("seed", range(60))
def test_brute_force_tiny_worlds_many_wolves(seed):
    """The rule variants (several wolves per cell, grass off, both) against
    the list-of-agents simulator: tiny, crowded worlds so that cells often
    hold several wolves."""
    rng = np.random.default_rng(3000 + seed)
    variant = [oracle.VARIANT_MANY_WOLVES, oracle.VARIANT_GRASS_OFF,
               oracle.VARIANT_MANY_WOLVES | oracle.VARIANT_GRASS_OFF][seed % 3]
    side = int(rng.integers(1, 5))
    cap = (int(rng.integers(1, 30)), int(rng.integers(1, 20)))
    n0 = (int(rng.integers(0, cap[0] + 1)), int(rng.integers(0, cap[1] + 1)))
    params = workloads.predation_params(
        sheep_gain=int(rng.integers(1, 6)), wolf_gain=int(rng.integers(2, 25)),
        sheep_repro=float(rng.choice([0.04, 0.2, 0.5])), wolf_repro=float(rng.choice([0.05, 0.2, 0.5])),
        regrowth=int(rng.integers(1, 12)), grass_init=float(rng.choice([0.25, 0.5, 0.9])))
    ow = oracle.World(side, seed, 7, params, cap, n0, variant=variant)
    bw = BruteWorld(side, seed, 7, params, cap, n0, many_wolves=bool(variant & oracle.VARIANT_MANY_WOLVES),
                    grass_off=bool(variant & oracle.VARIANT_GRASS_OFF))
    compare(ow, bw)
    for _ in range(40):
        st = ow.step()[0]
        bst = bw.step()
        assert st["grass_eaten"] == bst["grass_eaten"] and st["eaten"] == bst["eaten"]
        assert st["births"] == [bst["births0"], bst["births1"]]
        assert st["starved"] == [bst["starved0"], bst["starved1"]]
        compare(ow, bw)


def test_many_wolves_single_cell_eat_min():
    """One cell: every wolf faces every sheep, so min(#sheep, #wolves) sheep
    are eaten (no reproduction, so the counts are those after the sheep die)."""
    params = workloads.predation_params(sheep_repro=0.0, wolf_repro=0.0, sheep_gain=3, wolf_gain=5)
    for n0 in [(10, 4), (3, 7), (5, 5), (0, 3), (4, 0)]:
        ow = oracle.World(1, 11, 0, params, (16, 16), n0, variant=oracle.VARIANT_MANY_WOLVES)
        for _ in range(5):
            st = ow.step()[0]
            sheep_left = st["n_start"][0] - st["starved"][0]
            assert st["eaten"] == min(sheep_left, st["n_start"][1]), (n0, st)
        one = oracle.World(1, 11, 0, params, (16, 16), n0)  # default: one wolf eats per cell
        st = one.step()[0]
        assert st["eaten"] == min(1, st["n_start"][0] - st["starved"][0], st["n_start"][1])


def test_grass_off_sheep_alone_keep_their_energy():
    """Without grass, wolves and reproduction, sheep never gain, spend or lose
    energy: every sheep keeps its initial energy and none dies."""
    params = workloads.predation_params(sheep_repro=0.0, wolf_repro=0.0)
    ow = oracle.World(12, 5, 0, params, (300, 10), (200, 0), variant=oracle.VARIANT_GRASS_OFF)
    e0 = ow.agents(0, "energy").copy()
    for st in ow.step(30):
        assert st["grass_eaten"] == 0 and st["starved"] == [0, 0] and st["n_end"][0] == 200
    np.testing.assert_array_equal(ow.agents(0, "energy"), e0)
    np.testing.assert_array_equal(ow.agents(0, "age")[:200], np.full(200, 30))


def check_invariants(before, after, st, counters_before, counters_after, params, ncells):
    p = [int(x) & 0xFFFFFFFF for x in params]
    gain, metab = (p[0], p[1]), (p[5], p[6])
    for s, name in ((0, "sheep"), (1, "wolf")):
        act0 = before[f"{name}.active"].astype(bool)
        act1 = after[f"{name}.active"].astype(bool)
        eaten = st["eaten"] if s == 0 else 0
        # population change = births - deaths - eaten
        assert act1.sum() == act0.sum() + st["births"][s] - st["starved"][s] - eaten
        assert act1.sum() == counters_after["n_active"][s]
        # live ids unique and below next_id
        ids = after[f"{name}.id"][act1]
        assert np.unique(ids).size == ids.size
        assert ids.size == 0 or ids.max() < counters_after["next_id"][s]
        # children fill the lowest free slots: the highest live slot is below the
        # high-water mark of the post-birth count
        if act1.any():
            assert np.flatnonzero(act1).max() < counters_after["hw"][s]
        # energy ledger (int64): births conserve energy; removed agents keep
        # their energy at removal in their now-inactive slot
        born = after[f"{name}.id"] >= counters_before["next_id"][s]
        removed = ~act1 & (act0 | born)
        e0 = before[f"{name}.energy"][act0].astype(np.int64).sum()
        e1 = after[f"{name}.energy"][act1].astype(np.int64).sum()
        gained = gain[s] * (st["grass_eaten"] if s == 0 else st["eaten"])
        lost = after[f"{name}.energy"][removed].astype(np.int64).sum()
        assert e1 == e0 - metab[s] * st["n_start"][s] + gained - lost
        assert e1 == st["energy"][s]
        assert removed.sum() == st["starved"][s] + eaten
    # at most one grass winner and one wolf winner per cell
    assert st["grass_eaten"] <= before["grass.grown"].sum()
    assert st["eaten"] <= ncells


@pytest.mark.parametrize("seed", range(4))
def test_invariants_small_config(seed):
    c = workloads.PRED_SMALL
    w = oracle.World(c["side"], seed, 0, c["params"], c["cap"], c["n0"])
    before, cb = w.state(), w.counters()
    for _ in range(c["steps"]):
        st = w.step()[0]
        after, ca = w.state(), w.counters()
        check_invariants(before, after, st, cb, ca, c["params"], c["side"] ** 2)
        before, cb = after, ca


def test_invariants_with_overflow():
    # tiny capacity: births are truncated at r = min(parents, free)
    params = workloads.predation_params(sheep_repro=0.5, wolf_repro=0.5, sheep_gain=6)
    w = oracle.World(10, 3, 0, params, (40, 20), (30, 10))
    before, cb = w.state(), w.counters()
    saw_overflow = False
    for _ in range(60):
        st = w.step()[0]
        after, ca = w.state(), w.counters()
        check_invariants(before, after, st, cb, ca, params, 100)
        saw_overflow |= bool(ca["overflow"][0] or ca["overflow"][1])
        before, cb = after, ca
    assert saw_overflow


def test_no_reproduction_no_wolves_monotone():
    params = workloads.predation_params(sheep_repro=0.0, wolf_repro=0.0)
    w = oracle.World(20, 1, 0, params, (500, 10), (300, 0))
    last = 300
    for _ in range(40):
        st = w.step()[0]
        assert st["births"] == [0, 0] and st["n_end"][0] <= last
        last = st["n_end"][0]


def test_regrowth_one_keeps_grass_available():
    params = workloads.predation_params(regrowth=1, grass_init=0.99999)
    w = oracle.World(12, 2, 0, params, (400, 100), (50, 5))
    for _ in range(30):
        w.step()
        assert w.grass("grown").all()


def test_single_agent_walk_by_hand():
    # one sheep, no grass (threshold 0), no reproduction: its cell follows the
    # MOVE draws' top three bits through the 8-neighbour table, on a torus
    L = 7
    params = workloads.predation_params(sheep_repro=0.0, grass_init=0.0, sheep_gain=50)
    w = oracle.World(L, 9, 4, params, (1, 1), (1, 0))
    cell = int(w.agents(0, "cell")[0])
    e = int(w.agents(0, "energy")[0])
    table = [(-1, -1), (0, -1), (1, -1), (-1, 0), (1, 0), (-1, 1), (0, 1), (1, 1)]
    ate = 0
    for t in range(min(e, 20)):
        u = int(oracle.philox([t, 0, oracle.P_MOVE, 0], [9, 4])[0])
        dx, dy = table[u >> 29]
        x, y = cell % L, cell // L
        cell = ((y + dy) % L) * L + (x + dx) % L
        ate += w.step()[0]["grass_eaten"]
        assert int(w.agents(0, "cell")[0]) == cell
        assert int(w.agents(0, "energy")[0]) == e - (t + 1) + 50 * ate
        assert int(w.agents(0, "age")[0]) == t + 1


def test_grass_regrows_after_delay():
    # a cell eaten at step t is edible again from step t + regrowth
    params = workloads.predation_params(sheep_repro=0.0, grass_init=0.99999, regrowth=5, sheep_gain=10)
    w = oracle.World(1, 0, 0, params, (1, 1), (1, 0))   # 1x1 torus: the sheep never leaves
    assert w.grass("grown")[0] == 1
    eaten_at = [t for t in range(16) if w.step()[0]["grass_eaten"]]
    assert eaten_at == [0, 5, 10, 15]


def test_golden_small_trajectory():
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "pred_small_trajectory.txt")
    if not os.path.exists(path):
        pytest.skip("golden trajectory not written yet")
    want = np.loadtxt(path, dtype=np.int64, comments="#")
    c = workloads.PRED_SMALL
    w = oracle.World(c["side"], c["seed"], c["model"], c["params"], c["cap"], c["n0"])
    got = np.array([[t, s["n_end"][0], s["n_end"][1]] for t, s in enumerate(w.step(c["steps"]))])
    np.testing.assert_array_equal(got, want)
