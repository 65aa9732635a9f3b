"""Learned capacity for batched models (marshalling over the library's kernels).

An FP32 MLP (12 -> 3 x 128 ReLU -> 2) predicts, from a model's grid side,
initial populations, rule parameters and horizon, a high quantile (pinball
loss, tau = 0.99) of the log of its peak sheep and wolf counts; the slabs of a
batch are then sized from the prediction instead of the worst case. The MLP
only sizes buffers and never touches agent state: a model whose births ever
outgrow its learned slab is detected on the device (overflow flag) and rerun
with the fixed worst-case capacity, so the results equal the fixed-capacity
run exactly.

Training, inference, feature extraction and capacity sizing all run in the
library's CUDA kernels (abm_mlp_*, abm_capacity_*); this module only moves
arguments.
"""
from __future__ import annotations

import ctypes as C
import time

import numpy as np
import torch

from . import abm, engine
from .abm import call, ptr

N_IN, N_OUT = 12, 2


def table_of(models: list, horizon: int) -> np.ndarray:
    """int32[B][12]: side, n0 sheep, n0 wolves, 8 params, horizon."""
    t = np.zeros((len(models), 12), dtype=np.int64)
    for i, m in enumerate(models):
        t[i, 0] = m["side"]
        t[i, 1], t[i, 2] = m["n0"][0], m["n0"][1]
        t[i, 3:11] = np.asarray(m["params"], dtype=np.int64)
        t[i, 11] = horizon
    return t.astype(np.int32)


class CapacityModel:
    def __init__(self, nominal, hidden: int = 128, layers: int = 3, seed: int = 0,
                 max_batch: int = 1 << 16, stream=None):
        self.nominal = np.asarray(nominal, dtype=np.int32).copy()
        self.hidden, self.layers, self.seed, self.max_batch = hidden, layers, seed, max_batch
        h = C.c_void_p()
        call("abm_mlp_create", N_IN, hidden, layers, N_OUT, seed & 0xFFFFFFFF, max_batch,
             abm.stream_handle(stream), C.byref(h))
        self.h = h
        cnt = C.c_int64()
        call("abm_mlp_params", self.h, None, None, C.byref(cnt))
        self.nparams = cnt.value
        self.dev = f"cuda:{torch.cuda.current_device()}"
        self._nominal_dev = torch.from_numpy(self.nominal).to(self.dev)

    def close(self):
        if getattr(self, "h", None) and self.h.value:
            abm.lib().abm_mlp_destroy(self.h)
            self.h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- parameters
    def params(self) -> torch.Tensor:
        out = torch.empty(self.nparams, dtype=torch.float32, device=self.dev)
        call("abm_mlp_get_params", self.h, ptr(out), self.nparams, abm.stream_handle())
        return out

    def grads(self) -> torch.Tensor:
        out = torch.empty(self.nparams, dtype=torch.float32, device=self.dev)
        call("abm_mlp_get_grads", self.h, ptr(out), self.nparams, abm.stream_handle())
        return out

    def set_params(self, flat: torch.Tensor):
        flat = flat.to(self.dev, torch.float32).contiguous()
        call("abm_mlp_set_params", self.h, ptr(flat), self.nparams, abm.stream_handle())
        torch.cuda.current_stream().synchronize()

    def save(self, path: str, meta: dict | None = None):
        np.savez(path, params=self.params().cpu().numpy(), nominal=self.nominal,
                 hidden=self.hidden, layers=self.layers, meta=np.array(str(meta or {})))

    @classmethod
    def load(cls, path: str, max_batch: int = 1 << 16):
        z = np.load(path)
        m = cls(z["nominal"], hidden=int(z["hidden"]), layers=int(z["layers"]), max_batch=max_batch)
        m.set_params(torch.from_numpy(z["params"]))
        return m

    # ---- kernels
    def features(self, table: np.ndarray) -> torch.Tensor:
        t = torch.from_numpy(np.ascontiguousarray(table, dtype=np.int32)).to(self.dev)
        x = torch.empty((t.shape[0], N_IN), dtype=torch.float32, device=self.dev)
        call("abm_capacity_features", ptr(t), t.shape[0], ptr(self._nominal_dev), ptr(x), abm.stream_handle())
        return x

    def predict(self, x: torch.Tensor) -> torch.Tensor:
        B = x.shape[0]
        y = torch.empty((B, N_OUT), dtype=torch.float32, device=self.dev)
        for i in range(0, B, self.max_batch):
            j = min(B, i + self.max_batch)
            call("abm_mlp_forward", self.h, ptr(x[i:j]), j - i, ptr(y[i:j]), abm.stream_handle())
        return y

    def gradients(self, x, y, tau=0.99, B=None, perm=(0, 0, 0, 0)):
        """Loss and parameter gradients (see grads()) on B rows; perm = (rows, a, c, m0)
        gathers row (a * (m0 + r) + c) mod rows of x and y."""
        loss = torch.zeros(1, dtype=torch.float32, device=self.dev)
        B = x.shape[0] if B is None else B
        call("abm_mlp_gradients", self.h, ptr(x), ptr(y), B, tau, perm[0], perm[1], perm[2], perm[3],
             ptr(loss), abm.stream_handle())
        return loss

    def train_step(self, x, y, lr=1e-3, tau=0.99, B=None, perm=(0, 0, 0, 0)):
        loss = torch.zeros(1, dtype=torch.float32, device=self.dev)
        B = x.shape[0] if B is None else B
        call("abm_mlp_train_step", self.h, ptr(x), ptr(y), B, tau, lr, perm[0], perm[1], perm[2], perm[3],
             ptr(loss), abm.stream_handle())
        return loss

    def fit(self, x: torch.Tensor, y: torch.Tensor, epochs: int = 200, batch: int = 1024,
            lr: float = 1e-3, tau: float = 0.99, log_every: int = 0) -> list:
        """Adam on the pinball loss; each epoch visits the rows in an affine
        permuted order (row = (a * i + c) mod N with a coprime to N)."""
        N = x.shape[0]
        loss = torch.zeros(1, dtype=torch.float32, device=self.dev)
        hist = []
        rng = np.random.default_rng(self.seed)
        for ep in range(epochs):
            while True:
                a = int(rng.integers(1, N)) | 1
                if np.gcd(a, N) == 1:
                    break
            c = int(rng.integers(0, N))
            for i0 in range(0, N - batch + 1, batch):
                call("abm_mlp_train_step", self.h, ptr(x), ptr(y), batch, tau, lr, N, a, c, i0, ptr(loss),
                     abm.stream_handle())
            if log_every and (ep % log_every == 0 or ep == epochs - 1):
                hist.append((ep, float(loss.item())))
        return hist

    def capacities(self, x: torch.Tensor, cap_max: np.ndarray, n0: np.ndarray, margin: float = 0.1,
                   round_to: int = 128) -> np.ndarray:
        yhat = self.predict(x)
        cm = torch.from_numpy(np.ascontiguousarray(cap_max, dtype=np.int32)).to(self.dev)
        nn = torch.from_numpy(np.ascontiguousarray(n0, dtype=np.int32)).to(self.dev)
        cap = torch.empty_like(cm)
        call("abm_capacity_from_prediction", ptr(yhat), yhat.shape[0], float(margin), round_to, ptr(cm),
             ptr(nn), ptr(cap), abm.stream_handle())
        return cap.cpu().numpy()


def peak_counts(models: list, horizon: int, sweep: int = abm.SWEEP_EXTENT, chunk: int = 4096) -> np.ndarray:
    """Run the models for `horizon` steps on the GPU; return their peak
    post-birth counts hw[B][2] (the training labels)."""
    out = np.zeros((len(models), 2), dtype=np.int64)
    for i in range(0, len(models), chunk):
        part = models[i:i + chunk]
        b = engine.Batch(part)
        b.run(horizon, sweep=sweep)
        cnt = b.counters()
        b.check()
        out[i:i + len(part)] = [c["hw"] for c in cnt]
        del b
        torch.cuda.empty_cache()
    return out


def run_learned(models: list, learned_caps: np.ndarray, fixed_caps: np.ndarray, steps: int,
                sweep: int = abm.SWEEP_CAPACITY, threads: int = 512, ctas_per_sm: int = 2,
                models_per_cta: int = 1, agents_per_thread: int = 16) -> dict:
    """Learned-capacity batch run: one launch at the learned capacities, then
    abm_batch_rerun_overflowed reruns every model whose slab overflowed at its
    fixed capacity and reports through the same batch. Returns the per-model
    digests and counters of the final result, the rerun counts and the GPU
    times (the rerun's includes setting up its batch)."""
    lm = [dict(m, cap=(int(c[0]), int(c[1]))) for m, c in zip(models, learned_caps)]
    b = engine.Batch(lm)
    b.tune(threads, ctas_per_sm, models_per_cta=models_per_cta, agents_per_thread=agents_per_thread)
    e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
    e0.record()
    b.run(steps, sweep=sweep)
    e1.record()
    ov = b.overflowed()
    n_rerun, n_unrec = b.rerun_overflowed(np.asarray(fixed_caps, dtype=np.int32), sweep=sweep)
    e2.record()
    e2.synchronize()
    dig = b.digest().cpu().numpy()
    cnt = b.counters()
    b.check()
    out = {"digest": dig, "counters": cnt, "overflowed": ov, "rerun": n_rerun, "unrecovered": n_unrec,
           "ms_learned": e0.elapsed_time(e1), "ms_rerun": e1.elapsed_time(e2) if n_rerun else 0.0}
    del b
    torch.cuda.empty_cache()
    return out
