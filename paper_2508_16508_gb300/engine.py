"""Thin object layer over the C ABI for torch users (marshalling only).

Device buffers are torch tensors on the current CUDA device; every method
enqueues library calls on the current torch stream (or the one given).
"""
from __future__ import annotations

import ctypes as C

import torch

from . import abm
from .abm import call, ptr


def _stream(stream):
    return abm.stream_handle(stream)


class Slab:
    """Fixed-capacity agent set with F int32 fields per slot (ABMax `Set`)."""

    def __init__(self, capacity: int, n_fields: int, seed: int = 0, model: int = 0,
                 init: int = abm.INIT_EMPTY, stream=None):
        self.capacity, self.F = int(capacity), int(n_fields)
        self.seed, self.model = seed, model
        h = C.c_void_p()
        call("abm_slab_create", self.capacity, self.F, seed & 0xFFFFFFFF, model & 0xFFFFFFFF,
             init, _stream(stream), C.byref(h))
        self.h = h
        dev = torch.cuda.current_device()
        self._i32 = dict(dtype=torch.int32, device=f"cuda:{dev}")

    def close(self):
        if getattr(self, "h", None) and self.h.value:
            abm.lib().abm_slab_destroy(self.h)
            self.h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def check(self, stream=None):
        call("abm_slab_check", self.h, _stream(stream))

    def read(self, field: int, n: int | None = None, stream=None) -> torch.Tensor:
        n = self.capacity if n is None else n
        out = torch.empty(n, **self._i32)
        call("abm_slab_read", self.h, field, ptr(out), n, _stream(stream))
        return out

    def write(self, field: int, src: torch.Tensor, stream=None):
        src = src.to(torch.int32).contiguous()
        call("abm_slab_write", self.h, field, ptr(src), src.numel(), _stream(stream))

    def fields(self, stream=None) -> torch.Tensor:
        return torch.stack([self.read(f, stream=stream) for f in range(self.F)])

    def counters(self, stream=None) -> dict:
        c = abm.abm_slab_counters()
        call("abm_slab_counters_get", self.h, C.byref(c), _stream(stream))
        return {"n_active": c.n_active, "next_id": c.next_id, "overflow": c.overflow}

    def select(self, p: abm.abm_pred, stream=None):
        idx = torch.empty(self.capacity, **self._i32)
        cnt = torch.zeros(1, **self._i32)
        call("abm_select", self.h, C.byref(p), ptr(idx), ptr(cnt), _stream(stream))
        return idx, cnt

    def select_permutation(self, p: abm.abm_pred, stream=None):
        """All slots, those satisfying p first (ascending), then the rest (ascending)."""
        perm = torch.empty(self.capacity, **self._i32)
        cnt = torch.zeros(1, **self._i32)
        call("abm_select_permutation", self.h, C.byref(p), ptr(perm), ptr(cnt), _stream(stream))
        return perm, cnt

    def sort(self, field: int, stream=None) -> torch.Tensor:
        """sort_agents: live agents first, ascending by `field` (stable), then the
        placeholders; returns the permutation (old slot of each new slot)."""
        perm = torch.empty(self.capacity, **self._i32)
        call("abm_sort", self.h, int(field), ptr(perm), _stream(stream))
        return perm

    def remove(self, p: abm.abm_pred, stream=None) -> torch.Tensor:
        cnt = torch.zeros(1, **self._i32)
        call("abm_remove", self.h, C.byref(p), ptr(cnt), _stream(stream))
        return cnt

    def add(self, records: torch.Tensor, id_field: int = -1, stream=None):
        rec = records.to(torch.int32).contiguous()
        k = rec.shape[0] if rec.numel() else 0
        slots = torch.empty(max(k, 1), **self._i32)
        cnt = torch.zeros(1, **self._i32)
        call("abm_add", self.h, ptr(rec) if k else None, k, id_field, ptr(slots), ptr(cnt),
             _stream(stream))
        return slots, cnt

    def update_distinct(self, p: abm.abm_pred, records: torch.Tensor, record_mask=None,
                        op: int = abm.OP_ADD, stream=None):
        rec = records.to(torch.int32).contiguous()
        k = rec.shape[0] if rec.numel() else 0
        rm = None if record_mask is None else record_mask.to(torch.int32).contiguous()
        slots = torch.empty(max(min(k, self.capacity), 1), **self._i32)
        cnt = torch.zeros(1, **self._i32)
        call("abm_update_distinct", self.h, C.byref(p), ptr(rec) if k else None, ptr(rm), k, op,
             ptr(slots), ptr(cnt), _stream(stream))
        return slots, cnt

    def selective_update(self, step: int, threshold: int, records: torch.Tensor,
                         deltas: torch.Tensor, out_counts: torch.Tensor | None = None, stream=None):
        k = records.shape[0]
        out = torch.zeros(3, **self._i32) if out_counts is None else out_counts
        call("abm_selective_update", self.h, step & 0xFFFFFFFF, threshold & 0xFFFFFFFF,
             ptr(records), ptr(deltas), k, ptr(out), _stream(stream))
        return out

    def tune(self, threads: int, ctas_per_sm: int, stream=None):
        call("abm_slab_tune", self.h, threads, ctas_per_sm, _stream(stream))

    def philox_records(self, step: int, purpose0: int, purpose1: int, k: int, out=None,
                       stream=None) -> torch.Tensor:
        out = torch.empty((max(k, 1), self.F), **self._i32) if out is None else out
        call("abm_philox_records", self.h, step & 0xFFFFFFFF, purpose0, purpose1, k, ptr(out),
             _stream(stream))
        return out[:k]


class WorldSlab(Slab):
    """A species of a World as a Set (abm_world_slab): F = 4 fields (cell,
    energy, id, age) over the world's own arrays. Owned by the world; call
    World.slab_commit after editing, before the next step."""

    def __init__(self, world, species: int, stream=None):
        h = C.c_void_p()
        call("abm_world_slab", world.h, int(species), C.byref(h), _stream(stream))
        self.h = h
        self.world = world  # the view lives as long as the world
        self.capacity, self.F = world.cap[species], 4
        self._i32 = dict(dtype=torch.int32, device=world.dev)

    def close(self):
        self.h = C.c_void_p()  # freed with the world


class Resolver:
    """Per-resource conflict resolution with a reusable scratch table."""

    def __init__(self, R: int, stream=None):
        self.R = int(R)
        dev = torch.cuda.current_device()
        self.table = torch.empty(self.R, dtype=torch.int64, device=f"cuda:{dev}")
        self.winner = torch.empty(self.R, dtype=torch.int32, device=f"cuda:{dev}")
        call("abm_resolve_table_init", ptr(self.table), self.R, _stream(stream))

    def __call__(self, res: torch.Tensor, prio: torch.Tensor, is_winner: torch.Tensor | None = None,
                 stream=None):
        M = res.numel()
        call("abm_resolve", ptr(res), ptr(prio), M, self.R, ptr(self.table), ptr(self.winner),
             ptr(is_winner), _stream(stream))
        return self.winner


AGENT_FIELDS = ("active", "cell", "energy", "id", "age")


class World:
    """One predation model (wolf-sheep-grass) on the GPU."""

    def __init__(self, side, seed, model, params, cap, n0, stream=None, variant=abm.VARIANT_ONE_WOLF):
        cfg = abm.abm_config()
        cfg.side, cfg.seed, cfg.model = int(side), seed & 0xFFFFFFFF, model & 0xFFFFFFFF
        cfg.variant = int(variant)
        for i in range(8):
            cfg.params[i] = int(params[i])
        for s in range(2):
            cfg.cap[s], cfg.n0[s] = int(cap[s]), int(n0[s])
        h = C.c_void_p()
        call("abm_create", C.byref(cfg), _stream(stream), C.byref(h))
        self.h = h
        self.side, self.cap = int(side), [int(cap[0]), int(cap[1])]
        self.dev = f"cuda:{torch.cuda.current_device()}"

    def close(self):
        if getattr(self, "h", None) and self.h.value:
            abm.lib().abm_destroy(self.h)
            self.h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, nsteps: int = 1, stats: torch.Tensor | None = None, want_energy=False,
             stream=None):
        call("abm_step", self.h, nsteps, ptr(stats), 1 if want_energy else 0, _stream(stream))

    def tune(self, engine: int = abm.ENGINE_PERSISTENT, ctas_per_sm: int = 2):
        call("abm_world_tune", self.h, engine, ctas_per_sm)

    def step_graph(self, nsteps: int, reps: int = 1, stats: torch.Tensor | None = None,
                   stream=None):
        call("abm_step_graph", self.h, nsteps, reps, ptr(stats), _stream(stream))

    def step_profiled(self, nsteps: int, stats: torch.Tensor | None = None, stream=None) -> list:
        """Steps with per-kernel CUDA-event timing; returns the 8 phase sums (ms)."""
        ms = (C.c_float * 8)()
        call("abm_step_profiled", self.h, nsteps, ptr(stats), ms, _stream(stream))
        return list(ms)

    def new_stats(self, nsteps: int) -> torch.Tensor:
        return torch.zeros((nsteps, abm.STATS_WORDS), dtype=torch.int32, device=self.dev)

    def check(self, stream=None):
        call("abm_world_check", self.h, _stream(stream))

    def digest(self, stream=None) -> int:
        out = torch.zeros(1, dtype=torch.int64, device=self.dev)
        call("abm_digest", self.h, ptr(out), _stream(stream))
        return int(out.item())

    def slab(self, species: int, stream=None) -> "WorldSlab":
        """The species as a Set for edits between steps (commit with slab_commit)."""
        return WorldSlab(self, species, stream)

    def slab_commit(self, species: int, stream=None):
        call("abm_world_slab_commit", self.h, int(species), _stream(stream))

    def agents(self, species: int, which: str, stream=None) -> torch.Tensor:
        out = torch.empty(self.cap[species], dtype=torch.int32, device=self.dev)
        call("abm_read_agents", self.h, species, AGENT_FIELDS.index(which), ptr(out), _stream(stream))
        return out

    def grass(self, which: str, stream=None) -> torch.Tensor:
        out = torch.empty(self.side * self.side, dtype=torch.int32, device=self.dev)
        call("abm_read_grass", self.h, 0 if which == "grown" else 1, ptr(out), _stream(stream))
        return out

    def counters(self, stream=None) -> dict:
        c = abm.abm_world_counters()
        call("abm_world_counters_get", self.h, C.byref(c), _stream(stream))
        return {"n_active": list(c.n_active), "next_id": list(c.next_id), "hw": list(c.hw),
                "overflow": list(c.overflow), "extent": list(c.extent), "step": c.step}

    def save(self, stream=None) -> bytes:
        n = C.c_size_t(0)
        call("abm_save", self.h, None, C.byref(n), _stream(stream))
        buf = C.create_string_buffer(n.value)
        call("abm_save", self.h, buf, C.byref(n), _stream(stream))
        return buf.raw

    def load(self, image: bytes, stream=None):
        buf = C.create_string_buffer(image, len(image))
        call("abm_load", self.h, buf, len(image), _stream(stream))

    def image_bytes(self) -> int:
        """Size of the checkpoint image of the current state (slots up to the extents)."""
        n = C.c_size_t(0)
        call("abm_save", self.h, None, C.byref(n), None)
        return n.value

    def image_capacity(self) -> int:
        """Largest checkpoint image this world can produce (fits any later state)."""
        n = C.c_size_t(0)
        call("abm_image_capacity", self.h, C.byref(n))
        return n.value

    def save_into(self, host: torch.Tensor, stream=None) -> int:
        """Checkpoint into a host uint8 tensor (pinned for full copy speed) of at
        least image_bytes(); returns the image's size."""
        n = C.c_size_t(host.numel())
        call("abm_save", self.h, ptr(host), C.byref(n), _stream(stream))
        return n.value

    def load_from(self, host: torch.Tensor, stream=None):
        """Restore from a host uint8 tensor written by save / save_into."""
        call("abm_load", self.h, ptr(host), host.numel(), _stream(stream))


class OrderBooks:
    """n_books limit order books of `cap` slots (Section 5.3): int32 device
    arrays [n_books][cap] active, side, price, qty, time."""

    FIELDS = ("active", "side", "price", "qty", "time")

    def __init__(self, arrays: dict, device=None):
        dev = device if device is not None else f"cuda:{torch.cuda.current_device()}"
        self.t = {f: torch.as_tensor(arrays[f], dtype=torch.int32).to(dev).contiguous() for f in self.FIELDS}
        self.n_books, self.cap = self.t["active"].shape

    def _ptrs(self):
        return [ptr(self.t[f]) for f in self.FIELDS]

    def match(self, out_volume=None, out_price=None, stream=None):
        """One matching round of every book; returns (volume int64, price int32)."""
        dev = self.t["active"].device
        vol = out_volume if out_volume is not None else torch.empty(self.n_books, dtype=torch.int64, device=dev)
        px = out_price if out_price is not None else torch.empty(self.n_books, dtype=torch.int32, device=dev)
        call("abm_lob_match", self.n_books, self.cap, *self._ptrs(), ptr(vol), ptr(px), _stream(stream))
        return vol, px

    def add(self, new_orders: torch.Tensor, k: torch.Tensor, out=None, stream=None) -> torch.Tensor:
        """new_orders [n_books][kmax][4] (side, price, qty, time), k[b] of them
        for book b, into each book's lowest free slots; returns orders placed."""
        dev = self.t["active"].device
        no = new_orders.to(device=dev, dtype=torch.int32).contiguous()
        kk = k.to(device=dev, dtype=torch.int32).contiguous()
        kmax = int(no.shape[1]) if no.dim() == 3 else 0
        out = out if out is not None else torch.empty(self.n_books, dtype=torch.int32, device=dev)
        call("abm_lob_add", self.n_books, self.cap, *self._ptrs(), ptr(no) if no.numel() else None, ptr(kk),
             kmax, ptr(out), _stream(stream))
        return out

    def numpy(self) -> dict:
        return {f: self.t[f].cpu().numpy() for f in self.FIELDS}

    @staticmethod
    def tune(warps_per_book: int = 0):
        """Warps matching one book on the price-level path (process-wide)."""
        call("abm_lob_tune", int(warps_per_book))


def decode_stats(t: torch.Tensor) -> list[dict]:
    """Device stats rows (int32 words) -> list of dicts."""
    rows = t.cpu().contiguous()
    out = []
    for r in rows:
        s = abm.abm_step_stats.from_buffer_copy(r.numpy().tobytes())
        d = {}
        for name, _ in s._fields_:
            v = getattr(s, name)
            d[name] = list(v) if hasattr(v, "__len__") else int(v)
        out.append(d)
    return out


class Batch:
    """Many independent predation models in one persistent launch."""

    def __init__(self, models: list, stream=None):
        arr = (abm.abm_batch_model * len(models))()
        self.sides, self.caps = [], []
        for i, m in enumerate(models):
            arr[i].side, arr[i].seed, arr[i].model = int(m["side"]), m["seed"] & 0xFFFFFFFF, m["model"] & 0xFFFFFFFF
            for j in range(8):
                arr[i].params[j] = int(m["params"][j])
            for s in range(2):
                arr[i].cap[s], arr[i].n0[s] = int(m["cap"][s]), int(m["n0"][s])
            self.sides.append(int(m["side"]))
            self.caps.append([int(m["cap"][0]), int(m["cap"][1])])
        h = C.c_void_p()
        call("abm_batch_create", arr, len(models), _stream(stream), C.byref(h))
        self.h = h
        self.n = len(models)
        self.dev = f"cuda:{torch.cuda.current_device()}"

    def close(self):
        if getattr(self, "h", None) and self.h.value:
            abm.lib().abm_batch_destroy(self.h)
            self.h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def tune(self, threads: int, ctas_per_sm: int, steps_per_launch: int = 1 << 30, models_per_cta: int = 1,
             agents_per_thread: int = 16):
        call("abm_batch_tune", self.h, threads, ctas_per_sm, steps_per_launch)
        call("abm_batch_models_per_cta", self.h, models_per_cta)
        call("abm_batch_agents_per_thread", self.h, agents_per_thread)

    def run(self, nsteps: int, sweep: int = abm.SWEEP_CAPACITY, stream=None):
        call("abm_batch_run", self.h, nsteps, sweep, _stream(stream))

    def check(self, stream=None):
        call("abm_batch_check", self.h, _stream(stream))

    def counters(self, stream=None) -> list:
        arr = (abm.abm_batch_counters * self.n)()
        call("abm_batch_counters_get", self.h, arr, _stream(stream))
        out = []
        for c in arr:
            out.append({"n_active": list(c.n_active), "next_id": list(c.next_id), "hw": list(c.hw),
                        "overflow": list(c.overflow), "extent": list(c.extent), "step": c.step,
                        "agent_steps": c.agent_steps})
        return out

    def capacity(self, m: int) -> list:
        """Current capacities of model m (its rerun's after rerun_overflowed)."""
        cap = (C.c_int32 * 2)()
        call("abm_batch_capacity", self.h, int(m), cap)
        return [cap[0], cap[1]]

    def rerun_overflowed(self, cap_fixed, sweep: int = abm.SWEEP_CAPACITY, stream=None) -> tuple:
        """Rerun the overflowed models at cap_fixed[m] (int32 [n][2]); returns
        (models rerun, rerun models that overflowed again)."""
        import numpy as np
        cf = np.ascontiguousarray(np.asarray(cap_fixed, dtype=np.int32).reshape(self.n, 2))
        nr, nu = C.c_int32(), C.c_int32()
        call("abm_batch_rerun_overflowed", self.h, cf.ctypes.data_as(C.c_void_p), sweep, C.byref(nr), C.byref(nu),
             _stream(stream))
        return nr.value, nu.value

    def agents(self, m: int, species: int, which: str, stream=None) -> torch.Tensor:
        out = torch.empty(self.capacity(m)[species], dtype=torch.int32, device=self.dev)
        call("abm_batch_read_agents", self.h, m, species, AGENT_FIELDS.index(which), ptr(out),
             _stream(stream))
        return out

    def grass(self, m: int, which: str, stream=None) -> torch.Tensor:
        out = torch.empty(self.sides[m] ** 2, dtype=torch.int32, device=self.dev)
        call("abm_batch_read_grass", self.h, m, 0 if which == "grown" else 1, ptr(out), _stream(stream))
        return out

    def overflowed(self, stream=None) -> list:
        lst = torch.empty(self.n, dtype=torch.int32, device=self.dev)
        cnt = torch.zeros(1, dtype=torch.int32, device=self.dev)
        call("abm_batch_overflowed", self.h, ptr(lst), ptr(cnt), _stream(stream))
        c = int(cnt.item())
        return lst[:c].cpu().tolist()

    def digest(self, stream=None) -> torch.Tensor:
        out = torch.empty(self.n, dtype=torch.int64, device=self.dev)
        call("abm_batch_digest", self.h, ptr(out), _stream(stream))
        return out

    def info(self) -> dict:
        a, b, c = C.c_int64(), C.c_int64(), C.c_int64()
        call("abm_batch_info", self.h, C.byref(a), C.byref(b), C.byref(c))
        return {"slots": [a.value, b.value], "cells": c.value}
