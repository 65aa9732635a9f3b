"""Python binding of the C ABI in include/abm.h (argument marshalling only).

Every function here forwards to ``libabm.so``; all computation happens in the
library's CUDA kernels. Device buffers are passed as raw pointers (for torch
tensors, ``t.data_ptr()``), streams as ``cudaStream_t`` handles (for torch,
``torch.cuda.current_stream().cuda_stream``). There is no CPU fallback: if
the library is missing or fails to load, :func:`lib` raises.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
# ABM_LIBRARY=check selects the check build (libabm_check.so: index tests and
# canaries, slower), for the whole process
CHECK_BUILD = os.environ.get("ABM_LIBRARY", "") == "check"
LIB_PATH = os.path.join(_HERE, "libabm_check.so" if CHECK_BUILD else "libabm.so")
_lock = threading.Lock()
_lib = None

OK, ERR_ARG, ERR_OOM, ERR_CUDA, ERR_DEVICE_TIMEOUT, ERR_OVERFLOW, ERR_STATE, ERR_TOO_LARGE, ERR_CHECK = range(9)
RESOLVE_STATIC_MAX_R = 1 << 18

P_MOVE, P_PRIO, P_REPRO, P_VICTIM = 1, 2, 3, 4
P_INIT_AGENT, P_GRASS_INIT, P_MASK = 5, 6, 7
P_NEWREC0, P_NEWREC1, P_DELTA0, P_DELTA1 = 9, 10, 11, 12
P_RESOURCE, P_INIT_ACTIVE = 13, 14
INIT_STEP = 0xFFFFFFFF

INIT_EMPTY, INIT_HALF_LIVE = 0, 1
PRED_LIVE, PRED_FREE, PRED_BERNOULLI, PRED_MASK, PRED_FIELD = range(5)
CMP_EQ, CMP_NE, CMP_LT, CMP_GE = range(4)
OP_ADD, OP_SET = 0, 1


class AbmError(RuntimeError):
    def __init__(self, status: int, where: str):
        super().__init__(f"{where}: {strerror(status)} (status {status})")
        self.status = status


class abm_pred(C.Structure):
    _fields_ = [("kind", C.c_int32), ("threshold", C.c_uint32), ("step", C.c_uint32),
                ("purpose", C.c_uint32), ("species", C.c_uint32), ("mask", C.c_void_p),
                ("field", C.c_int32), ("cmp", C.c_int32), ("and_mask", C.c_int32),
                ("value", C.c_int32)]


VARIANT_ONE_WOLF, VARIANT_MANY_WOLVES, VARIANT_GRASS_OFF = 0, 1, 2  # bits
LOB_MAX_CAP = 2048  # order slots per book, at most


class abm_config(C.Structure):
    _fields_ = [("side", C.c_int32), ("seed", C.c_uint32), ("model", C.c_uint32),
                ("params", C.c_int32 * 8), ("cap", C.c_int32 * 2), ("n0", C.c_int32 * 2),
                ("variant", C.c_int32)]


class abm_step_stats(C.Structure):
    _fields_ = [("n_start", C.c_int32 * 2), ("parents", C.c_int32 * 2),
                ("births", C.c_int32 * 2), ("starved", C.c_int32 * 2), ("eaten", C.c_int32),
                ("grass_eaten", C.c_int32), ("n_end", C.c_int32 * 2), ("hw", C.c_int32 * 2),
                ("overflow", C.c_int32 * 2), ("step", C.c_int32), ("extent", C.c_int32 * 2),
                ("reserved", C.c_int32), ("energy", C.c_int64 * 2)]


STATS_BYTES = C.sizeof(abm_step_stats)
STATS_WORDS = STATS_BYTES // 4
STATS_FIELD_OFFSETS = {name: getattr(abm_step_stats, name).offset for name, _ in abm_step_stats._fields_}


class abm_world_counters(C.Structure):
    _fields_ = [("n_active", C.c_int32 * 2), ("next_id", C.c_int32 * 2), ("hw", C.c_int32 * 2),
                ("overflow", C.c_int32 * 2), ("extent", C.c_int32 * 2), ("step", C.c_int32),
                ("reserved", C.c_int32)]


class abm_batch_model(C.Structure):
    _fields_ = [("side", C.c_int32), ("seed", C.c_uint32), ("model", C.c_uint32),
                ("params", C.c_int32 * 8), ("cap", C.c_int32 * 2), ("n0", C.c_int32 * 2)]


class abm_batch_counters(C.Structure):
    _fields_ = [("n_active", C.c_int32 * 2), ("next_id", C.c_int32 * 2), ("hw", C.c_int32 * 2),
                ("overflow", C.c_int32 * 2), ("extent", C.c_int32 * 2), ("step", C.c_int32),
                ("reserved", C.c_int32), ("agent_steps", C.c_int64)]


SWEEP_CAPACITY, SWEEP_EXTENT = 0, 1
ENGINE_PERSISTENT, ENGINE_KERNELS = 0, 1


class abm_slab_counters(C.Structure):
    _fields_ = [("n_active", C.c_int32), ("next_id", C.c_int32), ("overflow", C.c_int32),
                ("reserved", C.c_int32)]


def _sig(L):
    vp, i32, u32, i64 = C.c_void_p, C.c_int32, C.c_uint32, C.c_int64
    pp = C.POINTER(C.c_void_p)
    st = C.c_int32
    sigs = {
        "abm_strerror": ([i32], C.c_char_p),
        "abm_version": ([], i32),
        "abm_slab_create": ([i32, i32, u32, u32, i32, vp, pp], st),
        "abm_slab_destroy": ([vp], st),
        "abm_slab_check": ([vp, vp], st),
        "abm_slab_arrays": ([vp, pp, pp, C.POINTER(i32)], st),
        "abm_slab_read": ([vp, i32, vp, i32, vp], st),
        "abm_slab_write": ([vp, i32, vp, i32, vp], st),
        "abm_select": ([vp, C.POINTER(abm_pred), vp, vp, vp], st),
        "abm_select_permutation": ([vp, C.POINTER(abm_pred), vp, vp, vp], st),
        "abm_sort": ([vp, i32, vp, vp], st),
        "abm_remove": ([vp, C.POINTER(abm_pred), vp, vp], st),
        "abm_add": ([vp, vp, i32, i32, vp, vp, vp], st),
        "abm_update_distinct": ([vp, C.POINTER(abm_pred), vp, vp, i32, i32, vp, vp, vp], st),
        "abm_selective_update": ([vp, u32, u32, vp, vp, i32, vp, vp], st),
        "abm_slab_tune": ([vp, i32, i32, vp], st),
        "abm_philox_records": ([vp, u32, u32, u32, i32, vp, vp], st),
        "abm_slab_counters_get": ([vp, C.POINTER(abm_slab_counters), vp], st),
        "abm_resolve_table_init": ([vp, i32, vp], st),
        "abm_resolve": ([vp, vp, i32, i32, vp, vp, vp, vp], st),
        "abm_resolve_static": ([vp, vp, i32, i32, vp, vp, vp], st),
        "abm_create": ([C.POINTER(abm_config), vp, pp], st),
        "abm_destroy": ([vp], st),
        "abm_step": ([vp, i32, vp, i32, vp], st),
        "abm_step_graph": ([vp, i32, i32, vp, vp], st),
        "abm_step_profiled": ([vp, i32, vp, C.POINTER(C.c_float), vp], st),
        "abm_world_check": ([vp, vp], st),
        "abm_world_tune": ([vp, i32, i32], st),
        "abm_diag_barrier_timeout": ([i32, vp], st),
        "abm_read_agents": ([vp, i32, i32, vp, vp], st),
        "abm_read_grass": ([vp, i32, vp, vp], st),
        "abm_world_counters_get": ([vp, C.POINTER(abm_world_counters), vp], st),
        "abm_save": ([vp, vp, C.POINTER(C.c_size_t), vp], st),
        "abm_load": ([vp, vp, C.c_size_t, vp], st),
        "abm_image_capacity": ([vp, C.POINTER(C.c_size_t)], st),
        "abm_batch_create": ([C.POINTER(abm_batch_model), i32, vp, pp], st),
        "abm_batch_destroy": ([vp], st),
        "abm_batch_tune": ([vp, i32, i32, i32], st),
        "abm_batch_run": ([vp, i32, i32, vp], st),
        "abm_batch_counters_get": ([vp, C.POINTER(abm_batch_counters), vp], st),
        "abm_batch_read_agents": ([vp, i32, i32, i32, vp, vp], st),
        "abm_batch_read_grass": ([vp, i32, i32, vp, vp], st),
        "abm_batch_overflowed": ([vp, vp, vp, vp], st),
        "abm_batch_check": ([vp, vp], st),
        "abm_batch_info": ([vp, C.POINTER(i64), C.POINTER(i64), C.POINTER(i64)], st),
        "abm_mlp_create": ([i32, i32, i32, i32, u32, i32, vp, pp], st),
        "abm_mlp_destroy": ([vp], st),
        "abm_mlp_forward": ([vp, vp, i32, vp, vp], st),
        "abm_mlp_gradients": ([vp, vp, vp, i32, C.c_float, i64, i64, i64, i64, vp, vp], st),
        "abm_mlp_train_step": ([vp, vp, vp, i32, C.c_float, C.c_float, i64, i64, i64, i64, vp, vp], st),
        "abm_mlp_params": ([vp, pp, pp, C.POINTER(i64)], st),
        "abm_mlp_reset_adam": ([vp, vp], st),
        "abm_mlp_set_params": ([vp, vp, i64, vp], st),
        "abm_mlp_get_params": ([vp, vp, i64, vp], st),
        "abm_mlp_get_grads": ([vp, vp, i64, vp], st),
        "abm_batch_digest": ([vp, vp, vp], st),
        "abm_batch_capacity": ([vp, i32, vp], st),
        "abm_batch_models_per_cta": ([vp, i32], st),
        "abm_batch_agents_per_thread": ([vp, i32], st),
        "abm_batch_rerun_overflowed": ([vp, vp, i32, vp, vp, vp], st),
        "abm_digest": ([vp, vp, vp], st),
        "abm_world_slab": ([vp, i32, pp, vp], st),
        "abm_world_slab_commit": ([vp, i32, vp], st),
        "abm_diag_check_index": ([i64, i64, vp], st),
        "abm_capacity_features": ([vp, i32, vp, vp, vp], st),
        "abm_capacity_from_prediction": ([vp, i32, C.c_float, i32, vp, vp, vp, vp], st),
        "abm_lob_match": ([i32, i32, vp, vp, vp, vp, vp, vp, vp, vp], st),
        "abm_lob_add": ([i32, i32, vp, vp, vp, vp, vp, vp, vp, i32, vp, vp], st),
        "abm_lob_tune": ([i32], st),
    }
    global EXPORTED
    for name, (args, res) in sigs.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = res
    EXPORTED = tuple(sigs)
    return L


EXPORTED = None  # filled by lib(): the names declared above


def lib():
    """Load libabm.so (building it first if it is missing or stale)."""
    global _lib, EXPORTED
    with _lock:
        if _lib is None:
            from . import build as _build
            if not _build.up_to_date(CHECK_BUILD):
                _build.build(check=CHECK_BUILD)
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"{os.path.basename(LIB_PATH)} not found at {LIB_PATH}")
            _lib = _sig(C.CDLL(LIB_PATH))
    return _lib


def strerror(status: int) -> str:
    try:
        return lib().abm_strerror(status).decode()
    except Exception:  # pragma: no cover - library not loadable
        return f"status {status}"


def check(status: int, where: str = "abm") -> None:
    if status != OK:
        raise AbmError(status, where)


def call(name: str, *args) -> None:
    check(getattr(lib(), name)(*args), name)


def ptr(t) -> C.c_void_p:
    """Raw device pointer of a torch tensor (or an int / None)."""
    if t is None:
        return C.c_void_p(None)
    if isinstance(t, int):
        return C.c_void_p(t)
    return C.c_void_p(t.data_ptr())


def stream_handle(stream=None) -> C.c_void_p:
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def pred(kind=PRED_LIVE, threshold=0, step=0, purpose=0, species=0, mask=None, field=0,
         cmp=CMP_EQ, and_mask=-1, value=0) -> abm_pred:
    p = abm_pred()
    p.kind, p.threshold, p.step, p.purpose, p.species = kind, threshold & 0xFFFFFFFF, step & 0xFFFFFFFF, purpose, species
    p.mask = None if mask is None else (mask if isinstance(mask, int) else mask.data_ptr())
    p._keep = mask  # the struct holds a raw pointer: keep the buffer alive with it
    p.field, p.cmp, p.and_mask, p.value = field, cmp, and_mask, value
    return p
