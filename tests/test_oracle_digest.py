"""Pin of the oracle's state digest (numpy) against its definition written as
a plain Python loop, on small worlds at several steps."""
import numpy as np
import pytest

import oracle
import workloads
from oracle import digest

M64, M32 = (1 << 64) - 1, (1 << 32) - 1
FIELDS = ("active", "cell", "energy", "id", "age")


def mix64(z):
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M64
    return z ^ (z >> 31)


def loop_digest(ow):
    h = 0
    for sp in range(2):
        a = {f: ow.agents(sp, f) for f in FIELDS}
        for i in range(a["active"].size):
            if not a["active"][i]:
                continue
            z = mix64((sp << 40) ^ i)
            z = mix64(z ^ (((int(a["cell"][i]) & M32) << 32) | (int(a["energy"][i]) & M32)))
            z = mix64(z ^ (((int(a["id"][i]) & M32) << 32) | (int(a["age"][i]) & M32)))
            h += z
    grown, cd = ow.grass("grown"), ow.grass("countdown")
    for c in range(grown.size):
        wait = 0 if grown[c] else max(int(cd[c]), 1)
        h += mix64((2 << 40) ^ (c << 8) ^ (wait << 40))
    k = ow.counters()
    for sp in range(2):
        h += mix64(0xC0FFEE + sp * 7 + ((k["n_active"][sp] & M32) << 20))
        h += mix64(0xBAD + sp * 11 + ((k["next_id"][sp] & M32) << 20))
        h += mix64(0xF00D + sp * 13 + ((k["hw"][sp] & M32) << 20))
    return h & M64


def test_mix64_known_values():
    # numpy's wrapping uint64 arithmetic against Python integers masked to 64 bits; mix64(0) = 0
    assert int(digest.mix64(np.array([0], np.uint64))[0]) == 0
    for z in (1, 0xDEADBEEF, (1 << 64) - 1, 12345678901234567):
        assert int(digest.mix64(np.array([z], np.uint64))[0]) == mix64(z)


@pytest.mark.parametrize("steps", [0, 7, 60])
def test_state_digest_matches_loop(steps):
    c = workloads.PRED_SMALL
    ow = oracle.World(c["side"], c["seed"], c["model"], c["params"], c["cap"], c["n0"])
    ow.step(steps)
    assert digest.state_digest(ow) == loop_digest(ow)


def test_state_digest_sees_every_part():
    c = workloads.PRED_SMALL
    ow = oracle.World(c["side"], c["seed"], c["model"], c["params"], c["cap"], c["n0"])
    ow.step(10)
    d0 = digest.state_digest(ow)
    i = int(np.flatnonzero(ow.agents(1, "active"))[0])
    for f in ("cell", "energy", "id", "age"):
        v = ow.agents_view(1, f)
        v[i] += 1
        assert digest.state_digest(ow) != d0, f
        v[i] -= 1
    assert digest.state_digest(ow) == d0
    k = ow.counters()
    ow.set_counters(0, k["n_active"][0], k["next_id"][0] + 1, k["hw"][0], k["overflow"][0])
    assert digest.state_digest(ow) != d0
