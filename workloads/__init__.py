"""Seeded synthetic inputs shared by the oracle side and the GPU side.

This module holds configuration tables and host samplers only: it performs none
of the method's arithmetic (no selection, ranking, update, conflict resolution
or predation rule). Random numbers the method itself draws come from Philox on
each side separately; the samplers here (numpy PCG64, float64) only build the
integer inputs both sides consume: Zipf claim targets for the conflict pass and
the integer model table of the batched runs.
"""
from __future__ import annotations

from fractions import Fraction

import numpy as np


def threshold(p) -> int:
    """Probability -> u32 threshold floor(p * 2^32); an event happens iff draw < T."""
    q = Fraction(str(p)) if not isinstance(p, Fraction) else p
    t = (q.numerator << 32) // q.denominator
    if not 0 <= t <= 0xFFFFFFFF:
        raise ValueError(f"probability {p} out of range")
    return t


def as_i32(u: int) -> int:
    """u32 bit pattern -> the int32 with the same bits (params travel as int32)."""
    u &= 0xFFFFFFFF
    return u - (1 << 32) if u >= 1 << 31 else u


# rule parameter order (int32 each; the three thresholds are u32 bit patterns)
PARAM_NAMES = ("sheep_gain", "wolf_gain", "sheep_repro_T", "wolf_repro_T",
               "grass_regrowth", "sheep_metabolism", "wolf_metabolism", "grass_init_T")


def predation_params(sheep_gain=4, wolf_gain=20, sheep_repro=0.04, wolf_repro=0.05,
                     regrowth=30, sheep_metab=1, wolf_metab=1, grass_init=0.5) -> np.ndarray:
    vals = [sheep_gain, wolf_gain, threshold(sheep_repro), threshold(wolf_repro), regrowth,
            sheep_metab, wolf_metab, threshold(grass_init)]
    return np.array([as_i32(v) for v in vals], dtype=np.int32)


# Predation, small: 40x40, 100 sheep / 25 wolves, capacity 2048 / 1024, 200 steps, seed 0.
PRED_SMALL = dict(name="predation_40x40", side=40, n0=(100, 25), cap=(2048, 1024),
                  steps=200, seed=0, model=0, params=predation_params())
# Predation, large: 2048x2048, 1,000,000 sheep / 250,000 wolves, capacity 8Mi / 4Mi,
# 1000 steps, seed 1.
PRED_LARGE = dict(name="predation_2048x2048", side=2048, n0=(1_000_000, 250_000),
                  cap=(8 << 20, 4 << 20), steps=1000, seed=1, model=0,
                  params=predation_params())

# Selective-update microbenchmark: N = 2^24 slots x 8 int32 fields, 50% live.
SELECTIVE = dict(name="selective_update_2^24x8", n=1 << 24, F=8, p=(0.001, 0.05, 0.5),
                 seed=2, model=0, zipf_s=1.1, zipf_seed=11)


def k_for(p, n) -> int:
    """k = round(p * n), round half to even on the exact rational."""
    return int(round(Fraction(str(p)) * n))


def zipf_claims(M: int, R: int, s: float = 1.1, seed: int = 11, shuffle: bool = False) -> np.ndarray:
    """M claim targets over R resources: Zipf(s) rank k in 1..R by inverse CDF
    (float64), rank k -> resource k-1 (or through a seeded permutation)."""
    rng = np.random.default_rng(seed)
    ranks = np.arange(1, R + 1, dtype=np.float64)
    pmf = ranks ** (-s)
    cdf = np.cumsum(pmf)
    cdf /= cdf[-1]
    u = rng.random(M)
    k = np.searchsorted(cdf, u, side="right")
    k = np.minimum(k, R - 1).astype(np.int64)
    if shuffle:
        perm = rng.permutation(R)
        k = perm[k]
    return k.astype(np.int32)


# Batched predation: 4096 models, side ~ U[16, 256], densities lognormal(0, 0.5) * 0.5
# clipped to [0.1, 2] agents per cell, 8 params jittered +-25%, cap = 4 side^2 per
# species, 500 steps.
BATCH = dict(name="batched_4096", n_models=4096, side_lo=16, side_hi=256, steps=500,
             sampler_seed=3, philox_seed=3, cap_factor=4)


def sample_models(n_models: int, sampler_seed: int, side_lo: int = 16, side_hi: int = 256,
                  base_params: np.ndarray | None = None) -> dict:
    """Integer model table for a batch of independent predation models."""
    rng = np.random.default_rng(sampler_seed)
    base = predation_params() if base_params is None else np.asarray(base_params, np.int32)
    side = rng.integers(side_lo, side_hi + 1, size=n_models).astype(np.int64)
    dens = np.clip(rng.lognormal(0.0, 0.5, size=(n_models, 2)) * 0.5, 0.1, 2.0)
    n0 = np.rint(dens * (side * side)[:, None]).astype(np.int64)
    params = np.zeros((n_models, 8), dtype=np.int64)
    u = rng.integers(0, 1 << 32, size=(n_models, 8), dtype=np.uint64)
    for j in range(8):
        v = int(np.uint32(base[j].view(np.uint32)))
        d = v >> 2
        # v' = v - d + floor(u * (2d+1) / 2^32): uniform in [v-d, v+d]
        params[:, j] = v - d + ((u[:, j].astype(object) * (2 * d + 1)) >> 32).astype(np.int64)
    params_i32 = np.array([[as_i32(int(x)) for x in row] for row in params], dtype=np.int32)
    return dict(side=side.astype(np.int32), n0=n0.astype(np.int32), params=params_i32,
                dens=dens)


def fixed_caps(side: np.ndarray, factor: int = 4) -> np.ndarray:
    c = factor * side.astype(np.int64) ** 2
    return np.stack([c, c], axis=1).astype(np.int32)


# Limit order books (Section 5.3: noisy traders, books of at most 1000 orders):
# 65,536 books of 1024 slots, about half holding an order; prices around 100
# ticks, quantities 1..100, arrival times unique within a book.
LOB = dict(name="lob_65536x1024", n_books=65536, cap=1024, fill=0.5, seed=21)
# the finance model's scale (Section 5.3, Table 4: 500 books of at most 1000
# orders, 100 steps); each step up to `traders` new orders per book, then a
# matching round of every book
LOB_MARKET = dict(name="lob_market_500x1000_100steps", n_books=500, cap=1000, fill=0.2, traders=10, steps=100,
                  seed=23)


def market_orders(n_books: int, traders: int, steps: int, seed: int):
    """Every step's new orders ([steps][n_books][traders][4]) and counts
    ([steps][n_books]), times increasing from step to step."""
    out = [random_new_orders(n_books, traders, seed + 1 + s, time0=(1 << 20) + s * traders) for s in range(steps)]
    return np.stack([o for o, _ in out]), np.stack([k for _, k in out])


def random_books(n_books: int, cap: int, fill: float, seed: int, price_mid: int = 100, price_spread: int = 10,
                 qty_max: int = 100) -> dict:
    """Seeded random order books: arrays [n_books][cap] active, side, price,
    qty, time (int32). Buy prices sit a little below the mid, sell prices a
    little above, with overlap, so that books cross."""
    rng = np.random.default_rng(seed)
    shape = (n_books, cap)
    active = (rng.random(shape) < fill).astype(np.int32)
    side = rng.integers(0, 2, size=shape, dtype=np.int32)
    offset = rng.integers(-price_spread, price_spread + 1, size=shape, dtype=np.int32)
    price = np.where(side == 0, price_mid - 2 + offset, price_mid + 2 + offset).astype(np.int32)
    qty = rng.integers(1, qty_max + 1, size=shape, dtype=np.int32)
    # time: a permutation of 0 .. cap - 1 per book
    time = np.ascontiguousarray(rng.permuted(np.broadcast_to(np.arange(cap, dtype=np.int32), shape), axis=1))
    return dict(active=active, side=side, price=price, qty=qty, time=time)


def random_new_orders(n_books: int, kmax: int, seed: int, price_mid: int = 100, price_spread: int = 10,
                      qty_max: int = 100, time0: int = 1 << 20):
    """Seeded new orders per book ([n_books][kmax][4] = side, price, qty, time)
    and how many each book gets (k[b] <= kmax)."""
    rng = np.random.default_rng(seed)
    side = rng.integers(0, 2, size=(n_books, kmax), dtype=np.int32)
    offset = rng.integers(-price_spread, price_spread + 1, size=(n_books, kmax), dtype=np.int32)
    price = np.where(side == 0, price_mid - 2 + offset, price_mid + 2 + offset).astype(np.int32)
    qty = rng.integers(1, qty_max + 1, size=(n_books, kmax), dtype=np.int32)
    time = (time0 + np.arange(kmax, dtype=np.int32))[None, :].repeat(n_books, axis=0)
    k = rng.integers(0, kmax + 1, size=n_books, dtype=np.int32)
    return np.stack([side, price, qty, time], axis=2).astype(np.int32), k
