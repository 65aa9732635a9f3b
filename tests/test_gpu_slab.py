"""GPU parity: generic slab primitives and conflict resolution vs the oracle.

Every comparison is element by element and bit-exact (all arithmetic is
integer). Sizes span several 2048-slot tiles plus ragged tails, and the
selective-update microbenchmark is also checked at its full size (2^24 slots
x 8 fields) against the oracle on the same seeded inputs.
"""
import numpy as np
import pytest

import oracle
import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def eng():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2508_16508_gb300 import abm, engine
    abm.lib()
    return engine


def np_of(t):
    return t.cpu().numpy()


def slab_state(s):
    torch.cuda.synchronize()
    return np_of(s.read(-1)), np.stack([np_of(s.read(f)) for f in range(s.F)])


SIZES = [1, 3, 33, 2047, 2048, 2049, 4096 * 3 + 17, 100_003]


@pytest.mark.parametrize("n", SIZES)
def test_half_live_init(eng, n):
    s = eng.Slab(n, 8, seed=2, init=1)
    o = oracle.Slab(n, 8)
    o.c1_init(seed=2)
    act, fld = slab_state(s)
    np.testing.assert_array_equal(act, o.active)
    np.testing.assert_array_equal(fld, o.fields)
    assert s.counters()["n_active"] == int(o.active.sum())


@pytest.mark.parametrize("n", SIZES)
@pytest.mark.parametrize("p", [0.001, 0.05, 0.5])
def test_selective_update_parity(eng, n, p):
    from paper_2508_16508_gb300 import abm
    F = 8
    T, k = workloads.threshold(p), max(workloads.k_for(p, n), 1)
    s = eng.Slab(n, F, seed=2, init=1)
    o = oracle.Slab(n, F)
    o.c1_init(seed=2)
    for step in range(4):
        rec = s.philox_records(step, abm.P_NEWREC0, abm.P_NEWREC1, k)
        dl = s.philox_records(step, abm.P_DELTA0, abm.P_DELTA1, k)
        np.testing.assert_array_equal(np_of(rec), oracle.c1_records(2, 0, step, oracle.P_NEWREC0,
                                                                    oracle.P_NEWREC1, k, F))
        cnt = np_of(s.selective_update(step, T, rec, dl))
        want = o.c1_call(step, T, k, seed=2)
        act, fld = slab_state(s)
        s.check()
        assert cnt.tolist() == [want["removed"], want["added"], want["updated"]]
        np.testing.assert_array_equal(act, o.active)
        np.testing.assert_array_equal(fld, o.fields)
        assert s.counters()["n_active"] == int(o.active.sum())


@pytest.mark.parametrize("offset", [0, 4, 1])
@pytest.mark.parametrize("p", [0.05, 0.5])
def test_selective_update_record_alignment(eng, offset, p):
    """Records and deltas starting 0, 16 or 4 bytes past a 32-byte boundary
    (the three ways the apply pass moves 8-field rows) give the same slab."""
    from paper_2508_16508_gb300 import abm
    n, F = 20_011, 8
    T, k = workloads.threshold(p), workloads.k_for(p, n)
    s = eng.Slab(n, F, seed=4, init=1)
    o = oracle.Slab(n, F)
    o.c1_init(seed=4)
    rb = torch.empty(k * F + 8, dtype=torch.int32, device="cuda")
    db = torch.empty(k * F + 8, dtype=torch.int32, device="cuda")
    rec, dl = rb[offset:offset + k * F].view(k, F), db[offset:offset + k * F].view(k, F)
    for step in range(3):
        s.philox_records(step, abm.P_NEWREC0, abm.P_NEWREC1, k, out=rec)
        s.philox_records(step, abm.P_DELTA0, abm.P_DELTA1, k, out=dl)
        cnt = np_of(s.selective_update(step, T, rec, dl))
        want = o.c1_call(step, T, k, seed=4)
        assert cnt.tolist() == [want["removed"], want["added"], want["updated"]]
        act, fld = slab_state(s)
        np.testing.assert_array_equal(act, o.active)
        np.testing.assert_array_equal(fld, o.fields)
    s.check()


def test_live_flag_values(eng):
    """Nonzero flags other than 1 count as live everywhere; a call that fills a
    16-slot group (add) or empties an 8-slot group (the fused call) writes that
    group's flags as 0/1, and every other flag keeps its value."""
    from paper_2508_16508_gb300 import abm
    n, F = 4000, 3
    rng = np.random.default_rng(8)
    flags = np.where(rng.random(n) < 0.7, rng.choice([1, 7, -2], size=n), 0).astype(np.int32)
    s = eng.Slab(n, F)
    s.write(-1, torch.from_numpy(flags).cuda())
    o = oracle.Slab(n, F)
    o.active[:] = flags != 0
    k = 40
    rec = rng.integers(-9, 9, size=(k, F)).astype(np.int32)
    slots, cnt = s.add(torch.from_numpy(rec).cuda())
    r, want_slots = o.add(rec)
    assert int(cnt.item()) == r == k
    np.testing.assert_array_equal(np_of(slots[:r]), want_slots)
    got = np_of(s.read(-1))
    np.testing.assert_array_equal(got != 0, o.active != 0)
    filled = np.zeros(n, bool)
    for g in np.unique(want_slots // 16):
        filled[16 * g:16 * g + 16] = True
    assert set(np.unique(got[filled]).tolist()) <= {0, 1}
    np.testing.assert_array_equal(got[~filled], flags[~filled])
    # a mask array that starts 4 bytes past an aligned address (scalar loads)
    buf = torch.zeros(n + 1, dtype=torch.int32, device="cuda")
    tm = (rng.random(n) < 0.5).astype(np.int32)
    buf[1:] = torch.from_numpy(tm).cuda()
    d = rng.integers(-5, 5, size=(300, F)).astype(np.int32)
    rmask = torch.zeros(301, dtype=torch.int32, device="cuda")
    rm = (rng.random(300) < 0.5).astype(np.int32)
    rmask[1:] = torch.from_numpy(rm).cuda()
    _, ucnt = s.update_distinct(abm.pred(abm.PRED_MASK, mask=buf[1:]), torch.from_numpy(d).cuda(),
                                rmask[1:], op=abm.OP_ADD)
    ru, _ = o.update_distinct(tm.astype(bool) & (o.active != 0), d, rec_mask=rm, op=0)
    assert int(ucnt.item()) == ru
    _, fld = slab_state(s)
    np.testing.assert_array_equal(fld, o.fields)
    s.check()


def test_selective_update_equals_separate_calls(eng):
    from paper_2508_16508_gb300 import abm
    n, F, p = 50_000, 8, 0.05
    T, k = workloads.threshold(p), workloads.k_for(p, n)
    a = eng.Slab(n, F, seed=5, init=1)
    b = eng.Slab(n, F, seed=5, init=1)
    for step in range(3):
        rec = a.philox_records(step, abm.P_NEWREC0, abm.P_NEWREC1, k)
        dl = a.philox_records(step, abm.P_DELTA0, abm.P_DELTA1, k)
        a.selective_update(step, T, rec, dl)
        # the same call as remove -> distinct update -> add through the generic API,
        # with the two draws made into explicit masks
        # slots 2j and 2j+1 share draw j: words (0, 1) and (2, 3) = (remove, choose)
        w = np.stack([oracle.philox_words(5, 0, step, oracle.P_MASK, 0, 0, (n + 1) // 2, q)
                      for q in range(4)]).astype(np.int64)
        slot = np.arange(n)
        rm = torch.from_numpy((w[2 * (slot & 1), slot >> 1] < T).astype(np.int32)).cuda()
        ch = torch.from_numpy((w[2 * (slot & 1) + 1, slot >> 1] < T).astype(np.int32)).cuda()
        b.remove(abm.pred(abm.PRED_MASK, mask=rm))
        b.update_distinct(abm.pred(abm.PRED_MASK, mask=ch), dl, op=abm.OP_ADD)
        b.add(rec)
        for f in range(-1, F):
            assert torch.equal(a.read(f), b.read(f))


def test_selective_update_full_size(eng):
    """2^24 slots x 8 fields, all three p, three calls each: full-state parity."""
    from paper_2508_16508_gb300 import abm
    c = workloads.SELECTIVE
    n, F = c["n"], c["F"]
    for p in c["p"]:
        T, k = workloads.threshold(p), workloads.k_for(p, n)
        s = eng.Slab(n, F, seed=c["seed"], init=1)
        o = oracle.Slab(n, F)
        o.c1_init(seed=c["seed"])
        for step in range(3):
            rec = s.philox_records(step, abm.P_NEWREC0, abm.P_NEWREC1, k)
            dl = s.philox_records(step, abm.P_DELTA0, abm.P_DELTA1, k)
            cnt = np_of(s.selective_update(step, T, rec, dl))
            want = o.c1_call(step, T, k, seed=c["seed"])
            assert cnt.tolist() == [want["removed"], want["added"], want["updated"]]
        act, fld = slab_state(s)
        s.check()
        np.testing.assert_array_equal(act, o.active)
        np.testing.assert_array_equal(fld, o.fields)
        del s


@pytest.mark.parametrize("n", [1, 31, 2048, 2049, 9000])
def test_select_predicates(eng, n):
    from paper_2508_16508_gb300 import abm
    s = eng.Slab(n, 3, seed=9, init=1)
    act, fld = slab_state(s)
    rng = np.random.default_rng(n)
    mask = (rng.random(n) < 0.3).astype(np.int32)
    cases = [
        (abm.pred(abm.PRED_LIVE), act != 0),
        (abm.pred(abm.PRED_FREE), act == 0),
        (abm.pred(abm.PRED_BERNOULLI, threshold=workloads.threshold(0.25), step=4, purpose=abm.P_REPRO),
         (act != 0) & (oracle.philox_words(9, 0, 4, oracle.P_REPRO, 0, 0, n) < workloads.threshold(0.25))),
        (abm.pred(abm.PRED_MASK, mask=torch.from_numpy(mask).cuda()), (act != 0) & (mask != 0)),
        (abm.pred(abm.PRED_FIELD, field=1, cmp=abm.CMP_EQ, and_mask=1, value=0),
         (act != 0) & ((fld[1] & 1) == 0)),
        (abm.pred(abm.PRED_FIELD, field=2, cmp=abm.CMP_LT, value=0), (act != 0) & (fld[2] < 0)),
        (abm.pred(abm.PRED_FIELD, field=0, cmp=abm.CMP_GE, value=12345), (act != 0) & (fld[0] >= 12345)),
        (abm.pred(abm.PRED_FIELD, field=0, cmp=abm.CMP_NE, and_mask=3, value=2),
         (act != 0) & ((fld[0] & 3) != 2)),
    ]
    for p, want_mask in cases:
        idx, cnt = s.select(p)
        c = int(cnt.item())
        want = oracle.flatnonzero(want_mask.astype(np.int32))
        assert c == want.size
        np.testing.assert_array_equal(np_of(idx[:c]), want)


@pytest.mark.parametrize("n", [1, 33, 2049, 4096 * 3 + 17])
def test_select_permutation(eng, n):
    """SCI's index exposure (Algorithm 2): the selected slots ascending, then
    the rest ascending -- the stable argsort of the mask with true first."""
    from paper_2508_16508_gb300 import abm
    s = eng.Slab(n, 3, seed=6, init=1)
    act, fld = slab_state(s)
    T = workloads.threshold(0.5)
    cases = [(abm.pred(abm.PRED_LIVE), act != 0),
             (abm.pred(abm.PRED_FREE), act == 0),
             (abm.pred(abm.PRED_BERNOULLI, threshold=T, step=3, purpose=abm.P_REPRO, species=1),
              (act != 0) & (oracle.philox_words(6, 0, 3, oracle.P_REPRO, 1, 0, n) < T)),
             (abm.pred(abm.PRED_FIELD, field=2, cmp=abm.CMP_LT, and_mask=0xFF, value=100),
              (act != 0) & ((fld[2] & 0xFF) < 100))]
    for p, m in cases:
        perm, cnt = s.select_permutation(p)
        sel = oracle.flatnonzero(m.astype(np.int32))
        rest = oracle.flatnonzero((~m).astype(np.int32))
        assert int(cnt.item()) == sel.size
        np.testing.assert_array_equal(np_of(perm), np.concatenate([sel, rest]))
        np.testing.assert_array_equal(np_of(perm), np.argsort(~m, kind="stable"))
    s.check()


@pytest.mark.parametrize("n", [1, 33, 2049, 4096 * 3 + 17, 100_003])
def test_sort_agents(eng, n):
    """sort_agents vs the oracle: whole state and permutation, keys with many
    ties (stability) and full-range keys, twice in a row (the second call
    sorts by another field and reuses the buffers)."""
    F = 5
    rng = np.random.default_rng(n)
    s = eng.Slab(n, F, seed=4, init=1)
    o = oracle.Slab(n, F)
    o.c1_init(seed=4)
    ties = rng.integers(-3, 4, size=n).astype(np.int32)
    s.write(1, torch.from_numpy(ties).cuda())
    o.fields[1] = ties
    for field in (1, 3, 0):
        perm = np_of(s.sort(field))
        want = o.sort(field)
        np.testing.assert_array_equal(perm, want)
        act, fld = slab_state(s)
        np.testing.assert_array_equal(act, o.active)
        np.testing.assert_array_equal(fld, o.fields)
    assert s.counters()["n_active"] == int(o.active.sum())
    # live flags other than 0 / 1 (written by the caller) move unchanged
    odd = np.where(o.active != 0, 7, 0).astype(np.int32)
    s.write(-1, torch.from_numpy(odd).cuda())
    o.active[:] = odd
    np.testing.assert_array_equal(np_of(s.sort(2)), o.sort(2))
    act, fld = slab_state(s)
    np.testing.assert_array_equal(act, o.active)
    np.testing.assert_array_equal(fld, o.fields)
    s.check()


def test_maximum_capacity(eng):
    """The largest slab abm_slab_create accepts (2^28 - 1 slots, one field):
    half-live init, one selective-update call and a select, against the
    oracle; then a sort by the field."""
    from paper_2508_16508_gb300 import abm
    n, F, p = (1 << 28) - 1, 1, 0.001
    T, k = workloads.threshold(p), workloads.k_for(p, n)
    s = eng.Slab(n, F, seed=8, init=1)
    o = oracle.Slab(n, F)
    o.c1_init(seed=8)
    rec = s.philox_records(0, abm.P_NEWREC0, abm.P_NEWREC1, k)
    dl = s.philox_records(0, abm.P_DELTA0, abm.P_DELTA1, k)
    cnt = np_of(s.selective_update(0, T, rec, dl))
    want = o.c1_call(0, T, k, seed=8)
    assert cnt.tolist() == [want["removed"], want["added"], want["updated"]]
    act, fld = slab_state(s)
    np.testing.assert_array_equal(act, o.active)
    np.testing.assert_array_equal(fld, o.fields)
    del act, fld
    idx, c = s.select(abm.pred(abm.PRED_LIVE))
    live = int(c.item())
    assert live == int(o.active.sum()) == s.counters()["n_active"]
    assert bool((idx[1:live] > idx[:live - 1]).all())
    del idx
    # the sort, by the properties that define it (the oracle's sort is O(n log n)
    # on one core; the small and 2^24 cases compare with it directly)
    act0, key0 = o.active, o.fields[0]
    perm = np_of(s.sort(0)).astype(np.int64)
    assert (np.bincount(perm, minlength=n) == 1).all()  # a permutation
    act, fld = slab_state(s)
    np.testing.assert_array_equal(act, act0[perm])
    np.testing.assert_array_equal(fld[0], key0[perm])
    assert (act[:live] != 0).all() and (act[live:] == 0).all()
    k = fld[0][:live].astype(np.int64)
    pl = perm[:live]
    assert ((k[1:] > k[:-1]) | ((k[1:] == k[:-1]) & (pl[1:] > pl[:-1]))).all()  # ascending, stable
    assert (np.diff(perm[live:]) > 0).all()  # placeholders in slot order
    s.check()


def test_sort_agents_full_size(eng):
    """2^24 slots x 8 fields (the selective-update slab), after three
    selective-update calls; sorted by two fields."""
    from paper_2508_16508_gb300 import abm
    c = workloads.SELECTIVE
    n, F, p = c["n"], c["F"], 0.05
    T, k = workloads.threshold(p), workloads.k_for(p, n)
    s = eng.Slab(n, F, seed=c["seed"], init=1)
    o = oracle.Slab(n, F)
    o.c1_init(seed=c["seed"])
    for step in range(3):
        rec = s.philox_records(step, abm.P_NEWREC0, abm.P_NEWREC1, k)
        dl = s.philox_records(step, abm.P_DELTA0, abm.P_DELTA1, k)
        s.selective_update(step, T, rec, dl)
        o.c1_call(step, T, k, seed=c["seed"])
    for field in (2, 7):
        np.testing.assert_array_equal(np_of(s.sort(field)), o.sort(field))
    act, fld = slab_state(s)
    np.testing.assert_array_equal(act, o.active)
    np.testing.assert_array_equal(fld, o.fields)
    s.check()


@pytest.mark.parametrize("n", [5, 2049, 7000])
def test_add_remove_update_vs_oracle(eng, n):
    from paper_2508_16508_gb300 import abm
    F = 5
    rng = np.random.default_rng(n)
    s = eng.Slab(n, F)
    o = oracle.Slab(n, F)
    next_id = 0
    for it in range(6):
        k = int(rng.integers(0, n // 2 + 2))
        rec = rng.integers(-2**31, 2**31, size=(k, F), dtype=np.int64).astype(np.int32)
        slots, cnt = s.add(torch.from_numpy(rec).cuda(), id_field=4)
        r, want_slots = o.add(rec, id_field=4, id_base=next_id)
        next_id += r
        assert int(cnt.item()) == r
        np.testing.assert_array_equal(np_of(slots[:r]), want_slots)
        m = (rng.random(n) < 0.2).astype(np.int32)
        rem = s.remove(abm.pred(abm.PRED_MASK, mask=torch.from_numpy(m).cuda()))
        assert int(rem.item()) == o.remove(m)
        tm = (rng.random(n) < 0.4).astype(np.int32)
        kd = int(rng.integers(0, n // 3 + 2))
        d = rng.integers(-2**31, 2**31, size=(kd, F), dtype=np.int64).astype(np.int32)
        rm = (rng.random(kd) < 0.6).astype(np.int32) if it % 2 else None
        op = abm.OP_ADD if it % 3 else abm.OP_SET
        us, ucnt = s.update_distinct(abm.pred(abm.PRED_MASK, mask=torch.from_numpy(tm).cuda()),
                                     torch.from_numpy(d).cuda(),
                                     None if rm is None else torch.from_numpy(rm).cuda(), op=op)
        ru, want_us = o.update_distinct(tm.astype(bool) & o.active.astype(bool), d, rec_mask=rm, op=op)
        assert int(ucnt.item()) == ru
        np.testing.assert_array_equal(np_of(us[:ru]), want_us)
        act, fld = slab_state(s)
        np.testing.assert_array_equal(act, o.active)
        np.testing.assert_array_equal(fld, o.fields)
        assert s.counters()["n_active"] == int(o.active.sum())
        assert s.counters()["next_id"] == next_id
    s.check()


def test_add_overflow_flag(eng):
    s = eng.Slab(10, 2)
    slots, cnt = s.add(torch.arange(24, dtype=torch.int32, device="cuda").reshape(12, 2))
    assert int(cnt.item()) == 10
    c = s.counters()
    assert c["overflow"] == 1 and c["n_active"] == 10


def test_toy_task_on_gpu(eng):
    """Section 4's toy task through update_distinct (SET) with both masks."""
    from paper_2508_16508_gb300 import abm
    import os
    d = {}
    with open(os.path.join(os.path.dirname(__file__), "golden", "toy_task.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                k, v = line.split(":")
                d[k.strip()] = [int(x) for x in v.split()]
    a, b = d["a"], d["b"]
    s = eng.Slab(len(a), 1)
    s.add(torch.tensor(a, dtype=torch.int32, device="cuda").reshape(-1, 1))
    bt = torch.tensor(b, dtype=torch.int32, device="cuda").reshape(-1, 1)
    _, cnt = s.update_distinct(abm.pred(abm.PRED_FIELD, field=0, cmp=abm.CMP_EQ, and_mask=1, value=0),
                               bt, record_mask=(bt[:, 0] & 1), op=abm.OP_SET)
    assert int(cnt.item()) == d["r"][0]
    assert np_of(s.read(0)).tolist() == d["expected"]


@pytest.mark.parametrize("M,R", [(0, 5), (1, 1), (1000, 7), (4097, 300), (100_000, 65_536), (300_001, 1024)])
def test_resolve_vs_oracle(eng, M, R):
    rng = np.random.default_rng(M + R)
    res = rng.integers(-2, R + 2, size=M).astype(np.int32)
    if M > 10:
        res[: M // 3] = workloads.zipf_claims(M // 3, R, seed=M)
    prio = rng.integers(0, 8, size=M).astype(np.uint32) * np.uint32(0x20000000)
    r = eng.Resolver(R)
    isw = torch.empty(max(M, 1), dtype=torch.uint8, device="cuda")
    dres = torch.from_numpy(res).cuda()
    dprio = torch.from_numpy(prio.view(np.int32)).cuda()
    for rep in range(2):  # the scratch table must come back clean
        w = r(dres, dprio, isw[:M] if M else None)
        ow, oisw = oracle.resolve(res, prio, R)
        np.testing.assert_array_equal(np_of(w), ow)
        if M:
            np.testing.assert_array_equal(np_of(isw[:M]), oisw)
    assert torch.all(r.table == -1)


def test_resolve_full_size(eng):
    c = workloads.SELECTIVE
    N = c["n"]
    M, R = N // 4, N // 64
    res = workloads.zipf_claims(M, R, s=c["zipf_s"], seed=c["zipf_seed"])
    prio = oracle.philox_words(c["seed"], 0, 0, oracle.P_RESOURCE, 0, 0, M)
    r = eng.Resolver(R)
    isw = torch.empty(M, dtype=torch.uint8, device="cuda")
    w = r(torch.from_numpy(res).cuda(), torch.from_numpy(prio.view(np.int32)).cuda(), isw)
    ow, oisw = oracle.resolve(res, prio, R)
    np.testing.assert_array_equal(np_of(w), ow)
    np.testing.assert_array_equal(np_of(isw), oisw)


def test_argument_errors(eng):
    from paper_2508_16508_gb300 import abm
    import ctypes as C
    h = C.c_void_p()
    L = abm.lib()
    assert L.abm_slab_create(0, 8, 0, 0, 0, None, C.byref(h)) == abm.ERR_ARG
    assert L.abm_slab_create(10, 17, 0, 0, 0, None, C.byref(h)) == abm.ERR_ARG
    assert L.abm_slab_create(1 << 28, 1, 0, 0, 0, None, C.byref(h)) == abm.ERR_ARG
    assert L.abm_resolve(None, None, 5, 3, None, None, None, None) == abm.ERR_ARG
    s = eng.Slab(10, 2)
    assert L.abm_select(s.h, None, None, None, None) == abm.ERR_ARG
    p = abm.pred(abm.PRED_FIELD, field=2)
    assert L.abm_select(s.h, C.byref(p), None, None, None) == abm.ERR_ARG
