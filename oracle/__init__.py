"""CPU oracle for the ABMax selective-update hot path (arXiv 2508.16508).

TEST INFRASTRUCTURE ONLY: tests/, ``__graft_entry__.smoke()`` and bench.py's
``cpu_baseline`` / ``--impl reference`` legs are the only callers. The product
path (``paper_2508_16508_gb300``) never imports this package, and this package
never imports the product.

The arithmetic lives in ``oracle.c`` (plain sequential C, compiled with gcc into
``liboracle.so`` beside it); this module only marshals numpy arrays. Each
function cites the passage of the paper it restates.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

# Philox purposes (counter word c2); species word c3: 0 sheep/slab, 1 wolf, 2 grass.
P_MOVE, P_PRIO, P_REPRO, P_VICTIM = 1, 2, 3, 4
P_INIT_AGENT, P_GRASS_INIT, P_MASK = 5, 6, 7
P_NEWREC0, P_NEWREC1, P_DELTA0, P_DELTA1 = 9, 10, 11, 12
P_RESOURCE, P_INIT_ACTIVE = 13, 14
INIT_STEP = 0xFFFFFFFF


def build(force: bool = False) -> str:
    """Compile oracle.c with gcc (portable flags only: x86 and Arm hosts)."""
    src = [os.path.join(_HERE, "oracle.c")]
    dep = src + [os.path.join(_HERE, "oracle.h")]
    if not force and os.path.exists(_SO) and all(
            os.path.getmtime(_SO) >= os.path.getmtime(d) for d in dep):
        return _SO
    tmp = _SO + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-Wall",
                           "-o", tmp] + src)
    os.replace(tmp, _SO)
    return _SO


class Stats(C.Structure):
    _fields_ = [("n_start", C.c_int32 * 2), ("parents", C.c_int32 * 2),
                ("births", C.c_int32 * 2), ("starved", C.c_int32 * 2),
                ("eaten", C.c_int32), ("grass_eaten", C.c_int32),
                ("n_end", C.c_int32 * 2), ("hw", C.c_int32 * 2),
                ("overflow", C.c_int32 * 2), ("pad", C.c_int32),
                ("energy", C.c_int64 * 2)]

    def as_dict(self) -> dict:
        d = {}
        for name, _ in self._fields_:
            if name == "pad":
                continue
            v = getattr(self, name)
            d[name] = list(v) if hasattr(v, "__len__") else int(v)
        return d


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(_SO)
            i32p, u32p, i64p = C.POINTER(C.c_int32), C.POINTER(C.c_uint32), C.POINTER(C.c_int64)
            u8p = C.POINTER(C.c_uint8)
            L.orc_philox4x32_10.argtypes = [u32p, u32p, u32p]
            L.orc_philox_words.argtypes = [C.c_uint32] * 6 + [C.c_int64, C.c_int, u32p]
            L.orc_flatnonzero.argtypes = [i32p, C.c_int64, i32p]
            L.orc_flatnonzero.restype = C.c_int64
            L.orc_assign_ranked.argtypes = [i32p, i32p, C.c_int64, i32p, i32p, C.c_int64]
            L.orc_assign_ranked.restype = C.c_int64
            L.orc_remove.argtypes = [i32p, i32p, C.c_int64]
            L.orc_remove.restype = C.c_int64
            L.orc_add.argtypes = [i32p, i32p, C.c_int64, C.c_int, i32p, C.c_int64, C.c_int,
                                  C.c_int32, i32p]
            L.orc_add.restype = C.c_int64
            L.orc_update_distinct.argtypes = [i32p, C.c_int64, C.c_int, i32p, i32p, i32p,
                                              C.c_int64, C.c_int, i32p]
            L.orc_update_distinct.restype = C.c_int64
            L.orc_resolve.argtypes = [i32p, u32p, C.c_int64, C.c_int64, i32p, u8p]
            L.orc_c1_init.argtypes = [i32p, i32p, C.c_int64, C.c_int, C.c_uint32, C.c_uint32]
            L.orc_c1_records.argtypes = [C.c_uint32] * 5 + [C.c_int64, C.c_int, i32p]
            L.orc_c1_call.argtypes = [i32p, i32p, C.c_int64, C.c_int, C.c_uint32, C.c_uint32,
                                      C.c_uint32, C.c_uint32, C.c_int64, i64p]
            L.orc_sort.argtypes = [i32p, i32p, C.c_int64, C.c_int, C.c_int, i32p]
            L.orc_lob_match.argtypes = [C.c_int32, C.c_int32, i32p, i32p, i32p, i32p, i32p, i64p, i32p]
            L.orc_lob_add.argtypes = [C.c_int32, C.c_int32, i32p, i32p, i32p, i32p, i32p, i32p, i32p,
                                      C.c_int32, i32p]
            L.orc_pred_create.argtypes = [C.c_int32, C.c_uint32, C.c_uint32, i32p, i32p, i32p]
            L.orc_pred_create.restype = C.c_void_p
            L.orc_pred_free.argtypes = [C.c_void_p]
            L.orc_pred_step.argtypes = [C.c_void_p, C.POINTER(Stats)]
            L.orc_pred_set_variant.argtypes = [C.c_void_p, C.c_int32]
            L.orc_pred_agents.argtypes = [C.c_void_p, C.c_int, C.c_int]
            L.orc_pred_agents.restype = i32p
            L.orc_pred_grass.argtypes = [C.c_void_p, C.c_int]
            L.orc_pred_grass.restype = i32p
            L.orc_pred_counters.argtypes = [C.c_void_p, i32p]
            L.orc_pred_set_counters.argtypes = [C.c_void_p, C.c_int] + [C.c_int32] * 4
            _lib = L
    return _lib


def _p(a: np.ndarray, ctype):
    return a.ctypes.data_as(C.POINTER(ctype))


def _i32(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.int32))


# --------------------------------------------------------------------------
# Philox4x32-10 (Salmon et al., SC'11)

def philox(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(np.asarray(ctr, dtype=np.uint32))
    k = np.ascontiguousarray(np.asarray(key, dtype=np.uint32))
    out = np.zeros(4, dtype=np.uint32)
    lib().orc_philox4x32_10(_p(c, C.c_uint32), _p(k, C.c_uint32), _p(out, C.c_uint32))
    return out


def philox_words(seed, model, step, purpose, species, slot0, n, word=0) -> np.ndarray:
    out = np.zeros(max(int(n), 0), dtype=np.uint32)
    if n > 0:
        lib().orc_philox_words(seed & 0xFFFFFFFF, model & 0xFFFFFFFF, step & 0xFFFFFFFF,
                               purpose, species, slot0 & 0xFFFFFFFF, int(n), word,
                               _p(out, C.c_uint32))
    return out


# --------------------------------------------------------------------------
# primitives (Section 2 API list; Section 4, Algorithms 1 and 2)

def flatnonzero(mask) -> np.ndarray:
    m = _i32(mask)
    out = np.zeros(max(m.size, 1), dtype=np.int32)
    n = lib().orc_flatnonzero(_p(m, C.c_int32), m.size, _p(out, C.c_int32))
    return out[:n].copy()


def assign_ranked(a, mask_a, b, mask_b):
    """Distinct updates (Alg. 1 / Alg. 2): returns (a', r)."""
    a2 = _i32(a).copy()
    ma, bb, mb = _i32(mask_a), _i32(b), _i32(mask_b)
    r = lib().orc_assign_ranked(_p(a2, C.c_int32), _p(ma, C.c_int32), a2.size,
                                _p(bb, C.c_int32), _p(mb, C.c_int32), bb.size)
    return a2, int(r)


class Slab:
    """Generic fixed-capacity set: active[n] and fields[F][n] (Section 2 `Set`)."""

    def __init__(self, n: int, F: int):
        self.n, self.F = int(n), int(F)
        self.active = np.zeros(self.n, dtype=np.int32)
        self.fields = np.zeros((self.F, self.n), dtype=np.int32)

    def sort(self, field: int) -> np.ndarray:
        """sort_agents: live agents first ascending by fields[field], then the
        placeholders; returns the permutation (old slot of each new slot)."""
        perm = np.zeros(max(self.n, 1), dtype=np.int32)
        lib().orc_sort(_p(self.active, C.c_int32), _p(self.fields, C.c_int32), self.n, self.F, int(field),
                       _p(perm, C.c_int32))
        return perm[:self.n].copy()

    def remove(self, mask) -> int:
        m = _i32(mask)
        return int(lib().orc_remove(_p(self.active, C.c_int32), _p(m, C.c_int32), self.n))

    def add(self, records, id_field=-1, id_base=0):
        rec = _i32(records).reshape(-1, self.F)
        k = rec.shape[0]
        slots = np.zeros(max(k, 1), dtype=np.int32)
        r = lib().orc_add(_p(self.active, C.c_int32), _p(self.fields, C.c_int32), self.n,
                          self.F, _p(rec, C.c_int32), k, id_field, id_base,
                          _p(slots, C.c_int32))
        return int(r), slots[:r].copy()

    def update_distinct(self, target_mask, records, rec_mask=None, op=0):
        tm = _i32(target_mask)
        rec = _i32(records).reshape(-1, self.F)
        k = rec.shape[0]
        rm = None if rec_mask is None else _i32(rec_mask)
        slots = np.zeros(max(min(k, self.n), 1), dtype=np.int32)
        r = lib().orc_update_distinct(_p(self.fields, C.c_int32), self.n, self.F,
                                      _p(tm, C.c_int32), _p(rec, C.c_int32),
                                      None if rm is None else _p(rm, C.c_int32), k, op,
                                      _p(slots, C.c_int32))
        return int(r), slots[:r].copy()

    # Selective-update microbenchmark (one slab, F fields, Philox inputs)
    def c1_init(self, seed=0, model=0):
        lib().orc_c1_init(_p(self.active, C.c_int32), _p(self.fields, C.c_int32), self.n,
                          self.F, seed, model)

    def c1_call(self, step, T, k, seed=0, model=0):
        out = np.zeros(3, dtype=np.int64)
        lib().orc_c1_call(_p(self.active, C.c_int32), _p(self.fields, C.c_int32), self.n,
                          self.F, seed, model, step, T & 0xFFFFFFFF, int(k),
                          _p(out, C.c_int64))
        return {"removed": int(out[0]), "added": int(out[1]), "updated": int(out[2])}


def c1_records(seed, model, step, p0, p1, k, F) -> np.ndarray:
    out = np.zeros((max(int(k), 1), F), dtype=np.int32)
    if k > 0:
        lib().orc_c1_records(seed, model, step, p0, p1, int(k), F, _p(out, C.c_int32))
    return out[:k].copy()


def resolve(res, prio, R):
    """Per-resource winner = lexicographic min of (priority, claim index)."""
    r = _i32(res)
    pr = np.ascontiguousarray(np.asarray(prio, dtype=np.uint32))
    winner = np.zeros(max(int(R), 1), dtype=np.int32)
    isw = np.zeros(max(r.size, 1), dtype=np.uint8)
    lib().orc_resolve(_p(r, C.c_int32), _p(pr, C.c_uint32), r.size, int(R),
                      _p(winner, C.c_int32), _p(isw, C.c_uint8))
    return winner[:R].copy(), isw[:r.size].copy()


# --------------------------------------------------------------------------
# predation (Section 5.1)

AGENT_FIELDS = ("active", "cell", "energy", "id", "age")


def lob_match(book: dict):
    """One matching round of every order book (Section 5.3; rules in
    orc_lob_match). book: arrays [nbooks][cap] active, side, price, qty, time;
    active and qty are updated in place. Returns (volume int64[nbooks],
    clearing price int32[nbooks])."""
    a = book["active"]
    nb, cap = a.shape
    for f in ("active", "side", "price", "qty", "time"):
        assert book[f].dtype == np.int32 and book[f].flags.c_contiguous and book[f].shape == (nb, cap)
    vol = np.zeros(max(nb, 1), dtype=np.int64)
    px = np.zeros(max(nb, 1), dtype=np.int32)
    lib().orc_lob_match(nb, cap, _p(book["active"], C.c_int32), _p(book["side"], C.c_int32),
                        _p(book["price"], C.c_int32), _p(book["qty"], C.c_int32), _p(book["time"], C.c_int32),
                        _p(vol, C.c_int64), _p(px, C.c_int32))
    return vol[:nb], px[:nb]


def lob_add(book: dict, new_orders: np.ndarray, k: np.ndarray) -> np.ndarray:
    """New orders (new_orders[nbooks][kmax][4] = side, price, qty, time; k[b]
    of them for book b) into each book's lowest free slots. Returns the
    orders placed per book."""
    a = book["active"]
    nb, cap = a.shape
    no = np.ascontiguousarray(new_orders, dtype=np.int32)
    kk = np.ascontiguousarray(k, dtype=np.int32)
    out = np.zeros(max(nb, 1), dtype=np.int32)
    lib().orc_lob_add(nb, cap, _p(book["active"], C.c_int32), _p(book["side"], C.c_int32),
                      _p(book["price"], C.c_int32), _p(book["qty"], C.c_int32), _p(book["time"], C.c_int32),
                      _p(no, C.c_int32), _p(kk, C.c_int32), no.shape[1], _p(out, C.c_int32))
    return out[:nb]


VARIANT_ONE_WOLF, VARIANT_MANY_WOLVES, VARIANT_GRASS_OFF = 0, 1, 2  # bits


class World:
    """One predation model (wolf-sheep-grass) stepped by the sequential oracle."""

    def __init__(self, side, seed, model, params, cap, n0, variant=0):
        """variant: bits -- VARIANT_MANY_WOLVES (the i-th wolf of a cell eats its
        i-th sheep; default: at most one wolf eats per cell per step) and
        VARIANT_GRASS_OFF (sheep neither eat grass nor spend energy)."""
        self.side = int(side)
        p, c, n = _i32(params), _i32(cap), _i32(n0)
        assert p.size == 8 and c.size == 2 and n.size == 2
        self._w = lib().orc_pred_create(self.side, seed & 0xFFFFFFFF, model & 0xFFFFFFFF,
                                        _p(p, C.c_int32), _p(c, C.c_int32), _p(n, C.c_int32))
        if not self._w:
            raise ValueError("invalid predation configuration")
        if variant & ~(VARIANT_MANY_WOLVES | VARIANT_GRASS_OFF):
            raise ValueError("unknown rule variant")
        lib().orc_pred_set_variant(self._w, variant)
        self.cap = [int(c[0]), int(c[1])]

    def __del__(self):
        w = getattr(self, "_w", None)
        if w:
            lib().orc_pred_free(w)
            self._w = None

    def step(self, n=1):
        out = []
        for _ in range(n):
            st = Stats()
            lib().orc_pred_step(self._w, C.byref(st))
            out.append(st.as_dict())
        return out

    def agents(self, species: int, which: str) -> np.ndarray:
        ptr = lib().orc_pred_agents(self._w, species, AGENT_FIELDS.index(which))
        return np.ctypeslib.as_array(ptr, shape=(self.cap[species],)).copy()

    def agents_view(self, species: int, which: str) -> np.ndarray:
        """Writable view of one of the species' arrays (for edits between steps)."""
        ptr = lib().orc_pred_agents(self._w, species, AGENT_FIELDS.index(which))
        return np.ctypeslib.as_array(ptr, shape=(self.cap[species],))

    def set_counters(self, species: int, n_active: int, next_id: int, hw: int, overflow: int):
        lib().orc_pred_set_counters(self._w, species, int(n_active), int(next_id), int(hw), int(overflow))

    def grass(self, which: str) -> np.ndarray:
        ptr = lib().orc_pred_grass(self._w, 0 if which == "grown" else 1)
        return np.ctypeslib.as_array(ptr, shape=(self.side * self.side,)).copy()

    def counters(self) -> dict:
        out = np.zeros(9, dtype=np.int32)
        lib().orc_pred_counters(self._w, _p(out, C.c_int32))
        return {"n_active": out[0:2].tolist(), "next_id": out[2:4].tolist(),
                "hw": out[4:6].tolist(), "overflow": out[6:8].tolist(), "step": int(out[8])}

    def state(self) -> dict:
        d = {}
        for s, name in ((0, "sheep"), (1, "wolf")):
            for f in AGENT_FIELDS:
                d[f"{name}.{f}"] = self.agents(s, f)
        d["grass.grown"] = self.grass("grown")
        d["grass.countdown"] = self.grass("countdown")
        return d
