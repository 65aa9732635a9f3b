"""Train the capacity predictor on trajectories of the batched-model sampler.

    python -m paper_2508_16508_gb300.train_capacity --out capacity_mlp.npz

Draws models from the batched workload's sampler (grid side U[16,256],
lognormal densities, +-25% parameter jitter) with sampler seeds disjoint from
the benchmark's, simulates half of them for 200 steps and half for 500 on the
GPU, and fits the MLP to the log of each model's peak sheep and wolf counts
with the pinball loss at tau = 0.99 using the library's training kernels.
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

import numpy as np
import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import workloads  # noqa: E402
from paper_2508_16508_gb300 import abm, capacity  # noqa: E402


def sample(n: int, sampler_seed: int, philox_seed: int) -> list:
    tab = workloads.sample_models(n, sampler_seed)
    caps = workloads.fixed_caps(tab["side"])
    return [dict(side=int(tab["side"][i]), seed=philox_seed, model=i, params=tab["params"][i],
                 cap=caps[i], n0=tab["n0"][i]) for i in range(n)]


def dataset(n_total: int, horizons=(200, 500), chunk: int = 4096, seed0: int = 1000):
    tabs, ys = [], []
    per_h = n_total // len(horizons)
    k = 0
    for h in horizons:
        done = 0
        while done < per_h:
            n = min(chunk, per_h - done)
            models = sample(n, seed0 + k, seed0 + k)
            k += 1
            hw = capacity.peak_counts(models, h, chunk=chunk)
            tabs.append(capacity.table_of(models, h))
            ys.append(np.log(np.maximum(hw, 1)).astype(np.float32))
            done += n
    return np.concatenate(tabs), np.concatenate(ys)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", required=True)
    ap.add_argument("--samples", type=int, default=50_000)
    ap.add_argument("--epochs", type=int, default=300)
    ap.add_argument("--batch", type=int, default=1024)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--holdout", type=float, default=0.1)
    args = ap.parse_args()
    abm.lib()
    t0 = time.time()
    table, y = dataset(args.samples)
    t_data = time.time() - t0
    n = table.shape[0]
    n_val = int(n * args.holdout)
    rng = np.random.default_rng(0)
    perm = rng.permutation(n)
    val, tr = perm[:n_val], perm[n_val:]
    model = capacity.CapacityModel(workloads.predation_params(), seed=0)
    x_tr = model.features(table[tr])
    y_tr = torch.from_numpy(y[tr]).cuda()
    t1 = time.time()
    hist = model.fit(x_tr, y_tr, epochs=args.epochs, batch=args.batch, lr=args.lr, log_every=25)
    torch.cuda.synchronize()
    t_fit = time.time() - t1
    yv = model.predict(model.features(table[val])).cpu().numpy()
    cover = float(np.mean(np.all(y[val] <= yv, axis=1)))
    cover_s = float(np.mean(y[val][:, 0] <= yv[:, 0]))
    cover_w = float(np.mean(y[val][:, 1] <= yv[:, 1]))
    meta = dict(samples=n, train=len(tr), holdout=len(val), epochs=args.epochs, batch=args.batch, lr=args.lr,
                tau=0.99, data_s=round(t_data, 1), fit_s=round(t_fit, 1), holdout_coverage=cover,
                holdout_coverage_sheep=cover_s, holdout_coverage_wolf=cover_w, loss=hist)
    model.save(args.out, meta)
    print(json.dumps(meta))


if __name__ == "__main__":
    main()
