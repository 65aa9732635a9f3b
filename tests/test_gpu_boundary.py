"""GPU tests of the boundary calls that tie the Set operations, the digest and
the learned-capacity recovery to worlds and batches (Section 2 API list):

- abm_digest of a world equals the batch digest of the same model and a
  digest computed here from the oracle's state;
- a world's species edited through abm_world_slab (remove, distinct update,
  add) and committed continues exactly like the oracle given the same edits;
- abm_batch_rerun_overflowed makes a learned-capacity batch report the fixed
  capacity run's digests, counters and agents, through the C ABI alone.
"""
import ctypes as C

import numpy as np
import pytest

import oracle
import workloads
from oracle import digest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FIELDS = ("active", "cell", "energy", "id", "age")
M64 = (1 << 64) - 1


@pytest.fixture(scope="module")
def lib():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2508_16508_gb300 import abm, engine
    abm.lib()
    return abm, engine


def oracle_digest(ow):
    """The digest's definition applied to the oracle's state (pinned on the CPU
    against a plain loop in test_oracle_digest.py)."""
    return digest.state_digest(ow)


def as_u64(x):
    return int(x) & M64


def compare_world(gw, ow, where):
    torch.cuda.synchronize()
    for s in range(2):
        for f in FIELDS:
            g, o = gw.agents(s, f).cpu().numpy(), ow.agents(s, f)
            assert np.array_equal(g, o), (where, s, f, np.flatnonzero(g != o)[:5])
    gc, oc = gw.counters(), ow.counters()
    for k in ("n_active", "next_id", "hw", "overflow", "step"):
        assert gc[k] == oc[k], (where, k, gc[k], oc[k])
    assert as_u64(gw.digest()) == oracle_digest(ow), where


@pytest.mark.parametrize("engine_kind", [0, 1])
def test_world_digest(lib, engine_kind):
    abm, eng = lib
    c = workloads.PRED_SMALL
    gw = eng.World(c["side"], c["seed"], c["model"], c["params"], c["cap"], c["n0"])
    gw.tune(engine_kind, 2)
    ow = oracle.World(c["side"], c["seed"], c["model"], c["params"], c["cap"], c["n0"])
    b = eng.Batch([dict(side=c["side"], seed=c["seed"], model=c["model"], params=c["params"],
                        cap=(c["cap"][0] * 2, c["cap"][1] + 7), n0=c["n0"])])  # capacity does not enter
    assert as_u64(gw.digest()) == oracle_digest(ow)
    for _ in range(4):
        gw.step(25)
        ow.step(25)
        b.run(25, sweep=abm.SWEEP_EXTENT)
        d = as_u64(gw.digest())
        assert d == oracle_digest(ow)
        assert d == as_u64(b.digest()[0].item())
    # a one-agent change moves the digest
    ew = ow.agents_view(0, "energy")
    i = int(np.flatnonzero(ow.agents(0, "active"))[0])
    ew[i] += 1
    assert oracle_digest(ow) != as_u64(gw.digest())


def oracle_slab_of(ow, sp):
    s = oracle.Slab(ow.cap[sp], 4)
    s.active[:] = ow.agents(sp, "active")
    for f, name in enumerate(FIELDS[1:]):
        s.fields[f] = ow.agents(sp, name)
    return s


def oracle_commit(ow, sp, s, next_id, overflow):
    ow.agents_view(sp, "active")[:] = s.active
    for f, name in enumerate(FIELDS[1:]):
        ow.agents_view(sp, name)[:] = s.fields[f]
    k = ow.counters()
    n = int((s.active != 0).sum())
    ow.set_counters(sp, n, next_id, max(k["hw"][sp], n), int(k["overflow"][sp] or overflow))


@pytest.mark.parametrize("engine_kind", [0, 1])
def test_world_slab_edits_vs_oracle(lib, engine_kind):
    """Between steps: remove sheep by a Bernoulli draw, give the first k sheep
    with energy below 5 a distinct energy bonus each, add new lambs with fresh
    ids, retire old wolves; commit; then both sides keep stepping."""
    abm, eng = lib
    c = workloads.PRED_SMALL
    L2 = c["side"] ** 2
    gw = eng.World(c["side"], c["seed"], c["model"], c["params"], c["cap"], c["n0"])
    gw.tune(engine_kind, 2)
    ow = oracle.World(c["side"], c["seed"], c["model"], c["params"], c["cap"], c["n0"])
    rng = np.random.default_rng(3 + engine_kind)
    gw.step(20)
    ow.step(20)
    compare_world(gw, ow, "before the edits")
    for rnd in range(3):
        # ---- sheep
        T, step, purpose = workloads.threshold(0.2), 5000 + rnd, abm.P_MASK
        v = gw.slab(0)
        v.remove(abm.pred(abm.PRED_BERNOULLI, threshold=T, step=step, purpose=purpose, species=0))
        k_upd = int(rng.integers(0, 30))
        upd = np.zeros((k_upd, 4), np.int32)
        upd[:, 1] = rng.integers(1, 20, size=k_upd)
        v.update_distinct(abm.pred(abm.PRED_FIELD, field=1, cmp=abm.CMP_LT, value=5),
                          torch.from_numpy(upd).cuda(), op=abm.OP_ADD)
        k_add = int(rng.integers(0, 40))
        rec = np.stack([rng.integers(0, L2, size=k_add), rng.integers(0, 9, size=k_add),
                        np.zeros(k_add, np.int64), rng.integers(0, 3, size=k_add)], axis=1).astype(np.int32)
        v.add(torch.from_numpy(rec).cuda(), id_field=2)
        gw.slab_commit(0)
        # the same edits on the oracle's arrays
        s = oracle_slab_of(ow, 0)
        live = s.active != 0
        draw = oracle.philox_words(c["seed"], c["model"], step, purpose, 0, 0, s.n, word=0)
        s.remove(live & (draw < T))
        s.update_distinct((s.active != 0) & (s.fields[1] < 5), upd, op=0)
        nid = ow.counters()["next_id"][0]
        r, _ = s.add(rec, id_field=2, id_base=nid)
        oracle_commit(ow, 0, s, nid + r, k_add > r)
        # ---- wolves older than 25 steps leave
        w = gw.slab(1)
        w.remove(abm.pred(abm.PRED_FIELD, field=3, cmp=abm.CMP_GE, value=25))
        gw.slab_commit(1)
        s = oracle_slab_of(ow, 1)
        s.remove((s.active != 0) & (s.fields[3] >= 25))
        oracle_commit(ow, 1, s, ow.counters()["next_id"][1], 0)
        compare_world(gw, ow, f"round {rnd} after the edits")
        for _ in range(3):
            gw.step(5)
            ow.step(5)
            compare_world(gw, ow, f"round {rnd} stepping")
    gw.check()


def test_world_slab_is_owned_by_the_world(lib):
    abm, eng = lib
    c = workloads.PRED_SMALL
    gw = eng.World(c["side"], c["seed"], c["model"], c["params"], c["cap"], c["n0"])
    v = gw.slab(0)
    assert abm.lib().abm_slab_destroy(v.h) == abm.ERR_STATE
    assert abm.lib().abm_sort(v.h, 1, None, abm.stream_handle()) == abm.ERR_STATE
    assert abm.lib().abm_world_slab(gw.h, 2, C.byref(C.c_void_p()), abm.stream_handle()) == abm.ERR_ARG
    w2 = eng.World(c["side"], c["seed"], c["model"], c["params"], c["cap"], c["n0"])
    assert abm.lib().abm_world_slab_commit(w2.h, 0, abm.stream_handle()) == abm.ERR_STATE
    # reading through the view gives the world's arrays
    torch.cuda.synchronize()
    assert torch.equal(v.read(-1), gw.agents(0, "active"))
    assert torch.equal(v.read(1), gw.agents(0, "energy"))


def overflow_models(n, seed):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        side = int(rng.integers(8, 40))
        params = workloads.predation_params(sheep_repro=float(rng.choice([0.04, 0.2])),
                                            wolf_repro=float(rng.choice([0.05, 0.2])), sheep_gain=6)
        n0 = (int(rng.integers(10, 60)), int(rng.integers(2, 20)))
        out.append(dict(side=side, seed=int(seed), model=i, params=params, cap=(4 * side * side, 4 * side * side),
                        n0=n0))
    return out


def test_batch_rerun_overflowed(lib):
    """Learned capacities too small for some models: the rerun through the C
    ABI makes the batch report the fixed-capacity run, and both keep stepping."""
    abm, eng = lib
    models = overflow_models(40, 11)
    fixed = np.array([m["cap"] for m in models], np.int32)
    ref = eng.Batch(models)
    ref.run(60, sweep=abm.SWEEP_CAPACITY)
    want_d, want_c = ref.digest().cpu().numpy(), ref.counters()
    hw = np.array([c["hw"] for c in want_c])
    rng = np.random.default_rng(1)
    small = np.where(rng.random((40, 1)) < 0.4, np.maximum(hw // 2, 1), hw + 5)  # 40% too small
    small = np.maximum(small, np.array([m["n0"] for m in models]))
    lm = [dict(m, cap=(int(s[0]), int(s[1]))) for m, s in zip(models, small)]
    b = eng.Batch(lm)
    b.tune(256, 2)
    b.run(60, sweep=abm.SWEEP_CAPACITY)
    ov = b.overflowed()
    assert 0 < len(ov) < 40
    n_rerun, n_unrec = b.rerun_overflowed(fixed, sweep=abm.SWEEP_CAPACITY)
    assert (n_rerun, n_unrec) == (len(ov), 0)
    assert np.array_equal(b.digest().cpu().numpy(), want_d)
    got_c = b.counters()
    for m in range(40):
        assert got_c[m] == want_c[m], m
        assert b.capacity(m) == (list(fixed[m]) if m in ov else list(small[m]))
    m = ov[0]
    for s in range(2):
        for f in FIELDS:
            assert torch.equal(b.agents(m, s, f), ref.agents(m, s, f)), (m, s, f)
    assert torch.equal(b.grass(m, "wait"), ref.grass(m, "wait"))
    # both batches go on stepping: the rerun models at their fixed capacity stay
    # equal to the reference; a model that was not rerun keeps its learned
    # capacity, sized for 60 steps, and stays equal unless it now overflows
    b.run(15, sweep=abm.SWEEP_EXTENT)
    ref.run(15, sweep=abm.SWEEP_EXTENT)
    d_b, d_ref, c_b = b.digest().cpu().numpy(), ref.digest().cpu().numpy(), b.counters()
    for m in range(40):
        if m in ov or not max(c_b[m]["overflow"]):
            assert d_b[m] == d_ref[m], m
    b.check()
    # one rerun per batch
    cf = np.ascontiguousarray(fixed)
    st = abm.lib().abm_batch_rerun_overflowed(b.h, cf.ctypes.data_as(C.c_void_p), 0, None, None, abm.stream_handle())
    assert st == abm.ERR_STATE


def test_batch_rerun_unrecovered(lib):
    """A rerun capacity that is still too small is reported as unrecovered."""
    abm, eng = lib
    models = overflow_models(6, 5)
    tiny = np.array([[max(m["n0"][0], 1) + 1, max(m["n0"][1], 1) + 1] for m in models], np.int32)
    b = eng.Batch([dict(m, cap=tuple(int(x) for x in t)) for m, t in zip(models, tiny)])
    b.run(40, sweep=abm.SWEEP_CAPACITY)
    ov = b.overflowed()
    n_rerun, n_unrec = b.rerun_overflowed(tiny + 1, sweep=abm.SWEEP_CAPACITY)
    assert n_rerun == len(ov) > 0 and 0 < n_unrec <= n_rerun
    cnt = b.counters()
    assert sum(1 for m in ov if max(cnt[m]["overflow"])) == n_unrec
    # the same models straight at those capacities agree with the rerun
    direct = eng.Batch([dict(models[m], cap=tuple(int(x) for x in tiny[m] + 1)) for m in ov])
    direct.run(40, sweep=abm.SWEEP_CAPACITY)
    assert np.array_equal(b.digest().cpu().numpy()[ov], direct.digest().cpu().numpy())
