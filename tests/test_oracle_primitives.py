"""Pins for the oracle's primitives (CPU only).

Select/compact is pinned to numpy.flatnonzero; the distinct update to literal
transcriptions of Rank-Match (Algorithm 1) and Sort-Count-Iterate (Algorithm 2)
and to the hand-worked toy task of Section 4; resolve to a brute-force
lexicographic minimum per resource; add/remove to a set-based slot allocator.
"""
import os

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def rank_match_literal(a, b, ma, mb):
    """Algorithm 1 written out: ranks = cumsum(mask) * mask; for each a, the
    candidate list over all b; argmax of the applied-mask picks the update.
    Reading: ranks match only when they are nonzero (unselected agents carry
    rank 0 and are never updated)."""
    ra = np.cumsum(ma) * ma
    rb = np.cumsum(mb) * mb
    out = []
    for a_i, r_a in zip(a, ra):
        cands, applied = [], []
        for b_j, r_b in zip(b, rb):
            if r_a == r_b and r_a > 0:
                cands.append(b_j)
                applied.append(1)
            else:
                cands.append(a_i)
                applied.append(0)
        if not cands:
            out.append(a_i)
            continue
        i = int(np.argmax(applied))
        out.append(cands[i])
    return np.array(out, dtype=np.int64)


def sci_literal(a, b, ma, mb):
    """Algorithm 2 written out: r = min of the sums; argsort with the true
    entries first (stable); a sequential loop over the first r indices."""
    a = np.array(a, dtype=np.int64).copy()
    r = min(int(np.sum(ma)), int(np.sum(mb)))
    ia = np.argsort(~np.asarray(ma, bool), kind="stable")
    ib = np.argsort(~np.asarray(mb, bool), kind="stable")
    for i in range(r):
        a[ia[i]] = b[ib[i]]
    return a, r


def read_toy():
    d = {}
    with open(os.path.join(GOLDEN, "toy_task.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            k, v = line.split(":")
            d[k.strip()] = np.array([int(x) for x in v.split()], dtype=np.int64)
    return d


def test_toy_task_hand_example():
    d = read_toy()
    a, b = d["a"], d["b"]
    ma, mb = (a % 2 == 0).astype(np.int32), (b % 2 == 1).astype(np.int32)
    got, r = oracle.assign_ranked(a, ma, b, mb)
    assert r == int(d["r"][0])
    np.testing.assert_array_equal(got, d["expected"])
    np.testing.assert_array_equal(rank_match_literal(a, b, ma, mb), d["expected"])
    np.testing.assert_array_equal(sci_literal(a, b, ma, mb)[0], d["expected"])


def test_rank_zero_reading_matters():
    # Without the "nonzero rank" reading, Algorithm 1's comparison r_a == r_b
    # would also pair unselected entries (rank 0 on both sides).
    a = np.array([1, 2]); b = np.array([4, 3])
    ma = (a % 2 == 0).astype(np.int32); mb = (b % 2 == 1).astype(np.int32)
    got, r = oracle.assign_ranked(a, ma, b, mb)
    assert r == 1
    np.testing.assert_array_equal(got, [1, 3])


@pytest.mark.parametrize("seed", range(60))
def test_rm_sci_oracle_agree(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(0, 14))
    m = int(rng.integers(0, 14))
    a = rng.integers(-50, 50, size=n)
    b = rng.integers(-50, 50, size=m)
    ma, mb = (a % 2 == 0).astype(np.int32), (b % 2 != 0).astype(np.int32)
    want_rm = rank_match_literal(a, b, ma, mb)
    want_sci, r_sci = sci_literal(a, b, ma, mb)
    got, r = oracle.assign_ranked(a, ma, b, mb)
    np.testing.assert_array_equal(want_rm, want_sci)
    np.testing.assert_array_equal(got, want_sci)
    assert r == r_sci == min(int(ma.sum()), int(mb.sum()))


def test_flatnonzero_matches_numpy():
    rng = np.random.default_rng(0)
    for n in [0, 1, 31, 32, 33, 1000, 4097]:
        for p in [0.0, 0.01, 0.5, 1.0]:
            m = (rng.random(n) < p).astype(np.int32)
            np.testing.assert_array_equal(oracle.flatnonzero(m), np.flatnonzero(m))


def test_exhaustive_small_subsets():
    # brute force over every (mask_a, mask_b) pair for n = m = 4
    a = np.array([10, 11, 12, 13]); b = np.array([20, 21, 22, 23])
    for xa in range(16):
        for xb in range(16):
            ma = np.array([(xa >> i) & 1 for i in range(4)], dtype=np.int32)
            mb = np.array([(xb >> i) & 1 for i in range(4)], dtype=np.int32)
            got, r = oracle.assign_ranked(a, ma, b, mb)
            np.testing.assert_array_equal(got, rank_match_literal(a, b, ma, mb))


def resolve_brute(res, prio, R):
    groups = {}
    for m, (r, p) in enumerate(zip(res, prio)):
        if 0 <= r < R:
            groups.setdefault(int(r), []).append((int(p), m))
    winner = np.full(R, -1, dtype=np.int64)
    for r, g in groups.items():
        winner[r] = sorted(g)[0][1]
    isw = np.array([1 if 0 <= r < R and winner[r] == m else 0 for m, r in enumerate(res)])
    return winner, isw


@pytest.mark.parametrize("seed", range(20))
def test_resolve_brute_force(seed):
    rng = np.random.default_rng(seed)
    M = int(rng.integers(0, 300)); R = int(rng.integers(1, 40))
    res = rng.integers(-3, R + 3, size=M).astype(np.int32)
    # few distinct priorities so that ties on the priority are common
    prio = rng.integers(0, 4, size=M).astype(np.uint32) * np.uint32(0x40000000)
    w, isw = oracle.resolve(res, prio, R)
    bw, bisw = resolve_brute(res, prio, R)
    np.testing.assert_array_equal(w, bw)
    np.testing.assert_array_equal(isw, bisw)
    # at most one winner per resource
    assert np.bincount(res[isw == 1], minlength=R).max(initial=0) <= 1


def test_add_remove_update_set_semantics():
    rng = np.random.default_rng(5)
    n, F = 64, 3
    s = oracle.Slab(n, F)
    live = set()
    fields = {}
    for it in range(30):
        rm = (rng.random(n) < 0.2).astype(np.int32)
        removed = s.remove(rm)
        gone = {i for i in live if rm[i]}
        live -= gone
        assert removed == len(gone)
        k = int(rng.integers(0, 20))
        rec = rng.integers(-1000, 1000, size=(k, F)).astype(np.int32)
        r, slots = s.add(rec)
        # brute force: repeatedly take the smallest unused slot
        want = []
        for j in range(k):
            free = sorted(set(range(n)) - live)
            if not free:
                break
            live.add(free[0]); want.append(free[0]); fields[free[0]] = rec[j].copy()
        assert r == len(want) and slots.tolist() == want
        tm = ((rng.random(n) < 0.3) & s.active.astype(bool)).astype(np.int32)
        kd = int(rng.integers(0, 10))
        d = rng.integers(-5, 5, size=(kd, F)).astype(np.int32)
        ru, us = s.update_distinct(tm, d, op=0)
        tgt = sorted(i for i in range(n) if tm[i])
        assert ru == min(len(tgt), kd)
        for j in range(ru):
            fields[tgt[j]] = fields[tgt[j]] + d[j]
        assert set(np.flatnonzero(s.active).tolist()) == live
        for i in live:
            np.testing.assert_array_equal(s.fields[:, i], fields[i])


def test_update_distinct_record_mask_and_overwrite():
    s = oracle.Slab(6, 1)
    s.active[:] = 1
    s.fields[0] = [2, 3, 4, 6, 7, 8]
    rec = np.array([[1], [2], [5], [9]], dtype=np.int32)
    r, slots = s.update_distinct((s.fields[0] % 2 == 0).astype(np.int32), rec,
                                 rec_mask=(rec[:, 0] % 2 == 1).astype(np.int32), op=1)
    assert r == 3 and slots.tolist() == [0, 2, 3]
    np.testing.assert_array_equal(s.fields[0], [1, 3, 5, 9, 7, 8])


def test_update_wraps_int32():
    s = oracle.Slab(2, 1)
    s.active[:] = 1
    s.fields[0] = [2**31 - 1, -2**31]
    s.update_distinct(np.array([1, 1]), np.array([[1], [-1]], dtype=np.int32), op=0)
    np.testing.assert_array_equal(s.fields[0], [-2**31, 2**31 - 1])


def philox_rows(seed, model, step, purpose, species, n):
    """Words [n][4] of the Philox block at counters (step, j, purpose, species),
    j < n, one generator call per counter (the generator itself is pinned to
    Triton's philox in test_oracle_philox.py)."""
    out = np.zeros((n, 4), dtype=np.uint32)
    for j in range(n):
        out[j] = oracle.philox([step & 0xFFFFFFFF, j, purpose, species], [seed, model])
    return out


def records_by_philox(seed, model, step, p0, p1, k, F):
    """Record j, field f = word f % 4 of the block of counter (step, j, p0 or p1, 0)."""
    lo, hi = philox_rows(seed, model, step, p0, 0, k), philox_rows(seed, model, step, p1, 0, k)
    rec = np.zeros((k, F), dtype=np.uint32)
    for f in range(F):
        rec[:, f] = (lo if f < 4 else hi)[:, f % 4]
    return rec.view(np.int32)


@pytest.mark.parametrize("seed,model,step,k,F", [(2, 0, 0, 5, 8), (7, 3, 11, 1, 4), (0, 1, 0xFFFFFFFF, 9, 6),
                                                 (5, 0, 2, 3, 1)])
def test_c1_records_word_by_word(seed, model, step, k, F):
    """The microbenchmark's records against the generator, word by word: field
    f of record j is word f % 4 of counter (step, j, NEWREC0 / NEWREC1 for the
    upper four fields, 0) under key (seed, model)."""
    got = oracle.c1_records(seed, model, step, oracle.P_NEWREC0, oracle.P_NEWREC1, k, F)
    assert got.shape == (k, F)
    for j in range(k):
        w0 = oracle.philox([step, j, oracle.P_NEWREC0, 0], [seed, model])
        w1 = oracle.philox([step, j, oracle.P_NEWREC1, 0], [seed, model])
        for f in range(F):
            assert np.uint32(got[j, f]) == (w0 if f < 4 else w1)[f % 4], (j, f)
    # the delta records take the other two purposes
    d = oracle.c1_records(seed, model, step, oracle.P_DELTA0, oracle.P_DELTA1, k, F)
    np.testing.assert_array_equal(d, records_by_philox(seed, model, step, oracle.P_DELTA0, oracle.P_DELTA1, k, F))
    assert oracle.c1_records(seed, model, step, oracle.P_NEWREC0, oracle.P_NEWREC1, 0, F).shape == (0, F)


@pytest.mark.parametrize("n,F,seed,model", [(37, 8, 2, 0), (10, 5, 9, 4), (1, 1, 0, 0)])
def test_c1_init_word_by_word(n, F, seed, model):
    """Initial microbenchmark slab: slot i is live iff word 0 of counter
    (INIT_STEP, i, INIT_ACTIVE, 0) is below 2^31 (compared as unsigned), and
    its field f is word f % 4 of counter (INIT_STEP, i, NEWREC0 or NEWREC1, 0)."""
    s = oracle.Slab(n, F)
    s.c1_init(seed=seed, model=model)
    for i in range(n):
        a = oracle.philox([oracle.INIT_STEP, i, oracle.P_INIT_ACTIVE, 0], [seed, model])
        assert s.active[i] == (1 if int(a[0]) < 2**31 else 0), i
        w0 = oracle.philox([oracle.INIT_STEP, i, oracle.P_NEWREC0, 0], [seed, model])
        w1 = oracle.philox([oracle.INIT_STEP, i, oracle.P_NEWREC1, 0], [seed, model])
        for f in range(F):
            assert np.uint32(s.fields[f, i]) == (w0 if f < 4 else w1)[f % 4], (i, f)
    if n >= 10:
        assert 0 < s.active.sum() < n  # both outcomes occur: the comparison is not constant


def c1_call_brute(active, fields, seed, step, T, k):
    """Microbenchmark call restated with numpy on Philox draws."""
    n, F = fields.shape[1], fields.shape[0]
    active = active.copy(); fields = fields.copy().astype(np.int64)
    # slots 2j and 2j+1 share draw j: words (0, 1) and (2, 3) = (remove, choose)
    half = (n + 1) // 2
    w = philox_rows(seed, 0, step, oracle.P_MASK, 0, half).T
    slot = np.arange(n)
    mask = w[2 * (slot & 1), slot >> 1] < T
    removed = int(np.sum(active.astype(bool) & mask))
    active[mask] = 0
    choose = w[2 * (slot & 1) + 1, slot >> 1] < T
    chosen = np.flatnonzero(active.astype(bool) & choose)
    free = np.flatnonzero(active == 0)
    d = records_by_philox(seed, 0, step, oracle.P_DELTA0, oracle.P_DELTA1, k, F)
    rec = records_by_philox(seed, 0, step, oracle.P_NEWREC0, oracle.P_NEWREC1, k, F)
    ru = min(k, chosen.size); ra = min(k, free.size)
    fields[:, chosen[:ru]] += d[:ru].T
    fields = ((fields + 2**31) % 2**32 - 2**31)
    fields[:, free[:ra]] = rec[:ra].T
    active[free[:ra]] = 1
    return active, fields.astype(np.int32), (removed, ra, ru)


@pytest.mark.parametrize("n,p", [(1, 0.5), (33, 0.05), (1000, 0.001), (1000, 0.5), (4099, 0.05)])
def test_c1_call_matches_numpy_restatement(n, p):
    from workloads import k_for, threshold
    s = oracle.Slab(n, 8)
    s.c1_init(seed=2)
    T, k = threshold(p), max(k_for(p, n), 1)
    act, fld = s.active.copy(), s.fields.copy()
    if n >= 1000:
        assert abs(act.mean() - 0.5) < 0.05
    for step in range(3):
        cnt = s.c1_call(step, T, k, seed=2)
        act, fld, (rm, ra, ru) = c1_call_brute(act, fld, 2, step, T, k)
        assert (cnt["removed"], cnt["added"], cnt["updated"]) == (rm, ra, ru)
        np.testing.assert_array_equal(s.active, act)
        np.testing.assert_array_equal(s.fields, fld)


@pytest.mark.parametrize("seed", range(20))
def test_sort_agents_vs_numpy_and_brute_force(seed):
    """sort_agents against numpy's stable lexsort and a Python sorted() on
    tuples (placeholder flag, key, slot); rows move whole."""
    rng = np.random.default_rng(70 + seed)
    n, F = int(rng.integers(0, 300)), int(rng.integers(1, 5))
    o = oracle.Slab(n, F)
    o.active[:] = rng.random(n) < rng.random()
    o.fields[:] = rng.integers(-5, 6, size=(F, n)) if seed % 2 else rng.integers(-2**31, 2**31, size=(F, n))
    field = int(rng.integers(0, F))
    act0, fld0 = o.active.copy(), o.fields.copy()
    perm = o.sort(field)
    key = np.where(act0 != 0, fld0[field], 0)
    want = np.lexsort((np.arange(n), key, act0 == 0))  # last key sorts first
    np.testing.assert_array_equal(perm, want)
    brute = [s for _, _, s in sorted((0 if act0[i] else 1, int(key[i]), i) for i in range(n))]
    assert perm.tolist() == brute
    np.testing.assert_array_equal(o.active, act0[perm])
    np.testing.assert_array_equal(o.fields, fld0[:, perm])
    live = int((act0 != 0).sum())
    assert (o.active[:live] != 0).all() and (o.active[live:] == 0).all()
    assert (np.diff(o.fields[field][:live].astype(np.int64)) >= 0).all()
