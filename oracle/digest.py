"""Digest of an oracle world's state (test infrastructure only).

The same definition as the library's world and batch digests, written here
with numpy: the wrapping 64-bit sum of one hash per live agent (species,
slot, cell, energy, id, age), one per cell (steps until its grass is edible)
and one per species counter (live agents, next id, high-water mark); the hash
is the splitmix64 finaliser (Steele, Lea, Flood, OOPSLA 2014). A sum of
per-item terms does not depend on the order of the items, so the oracle's
digest can be compared with a digest reduced in parallel on the GPU. Pinned
by a plain Python loop over the same definition (tests/test_oracle_digest.py).
"""
from __future__ import annotations

import numpy as np

_C1 = np.uint64(0xBF58476D1CE4E5B9)
_C2 = np.uint64(0x94D049BB133111EB)
_M32 = np.uint64(0xFFFFFFFF)


def mix64(z: np.ndarray) -> np.ndarray:
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _C1
        z = (z ^ (z >> np.uint64(27))) * _C2
    return z ^ (z >> np.uint64(31))


def _u32(a) -> np.ndarray:
    return np.asarray(a, dtype=np.int64).astype(np.uint64) & _M32


def _sum(z: np.ndarray) -> int:
    return int(np.sum(z, dtype=np.uint64)) if z.size else 0


def state_digest(world) -> int:
    """Digest of an oracle.World (its arrays, grass and counters)."""
    h = 0
    for sp in range(2):
        act = world.agents(sp, "active")
        idx = np.flatnonzero(act)
        cell, energy = world.agents(sp, "cell")[idx], world.agents(sp, "energy")[idx]
        aid, age = world.agents(sp, "id")[idx], world.agents(sp, "age")[idx]
        z = mix64((np.uint64(sp) << np.uint64(40)) ^ idx.astype(np.uint64))
        z = mix64(z ^ ((_u32(cell) << np.uint64(32)) | _u32(energy)))
        z = mix64(z ^ ((_u32(aid) << np.uint64(32)) | _u32(age)))
        h += _sum(z)
    grown, cd = world.grass("grown"), world.grass("countdown")
    wait = np.where(grown != 0, 0, np.maximum(cd, 1)).astype(np.uint64)
    c = np.arange(grown.size, dtype=np.uint64)
    h += _sum(mix64((np.uint64(2) << np.uint64(40)) ^ (c << np.uint64(8)) ^ (wait << np.uint64(40))))
    k = world.counters()
    for sp in range(2):
        for base, mul, key in ((0xC0FFEE, 7, "n_active"), (0xBAD, 11, "next_id"), (0xF00D, 13, "hw")):
            v = (base + sp * mul + ((k[key][sp] & 0xFFFFFFFF) << 20)) & ((1 << 64) - 1)
            h += int(mix64(np.array([v], dtype=np.uint64))[0])
    return h & ((1 << 64) - 1)
