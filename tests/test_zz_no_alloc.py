"""The allocation-free conflict-resolution entry point (abm_resolve_static).

It exists for callers that may not allocate device memory while running; its
scratch table is a fixed file-scope device array. Checked through the C ABI
against abm_resolve (the entry point with a caller-provided table) on two
calls in a row, so a second call sees whatever the first left in the array.
Collected last on purpose: it must pass both alone and after every other test.
"""
import ctypes as C

import numpy as np
import pytest

import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2508_16508_gb300 import abm
    return abm


def call_pair(abm, res, prio, R):
    M = res.numel()
    stream = abm.stream_handle()
    table = torch.empty(R, dtype=torch.int64, device="cuda")
    abm.check(abm.lib().abm_resolve_table_init(abm.ptr(table), R, stream))
    w_ref = torch.empty(R, dtype=torch.int32, device="cuda")
    f_ref = torch.empty(max(M, 1), dtype=torch.uint8, device="cuda")
    abm.check(abm.lib().abm_resolve(abm.ptr(res), abm.ptr(prio), M, R, abm.ptr(table), abm.ptr(w_ref),
                                    abm.ptr(f_ref), stream))
    w = torch.full((R,), 12345, dtype=torch.int32, device="cuda")
    f = torch.full((max(M, 1),), 7, dtype=torch.uint8, device="cuda")
    abm.check(abm.lib().abm_resolve_static(abm.ptr(res), abm.ptr(prio), M, R, abm.ptr(w), abm.ptr(f), stream))
    torch.cuda.synchronize()
    return w_ref, f_ref[:M], w, f[:M]


@pytest.mark.parametrize("M,R,seed", [(100_000, 4096, 1), (4_194_304, 262_144, 2)])
def test_static_resolve_matches_resolve_twice(lib, M, R, seed):
    abm = lib
    rng = np.random.default_rng(seed)
    for call in range(2):  # the second call runs on the array the first one used
        res = workloads.zipf_claims(M, R, seed=seed * 10 + call, shuffle=call == 1)
        res[: M // 50] = rng.integers(-3, R + 3, size=M // 50)  # some claims outside [0, R)
        prio = rng.integers(0, 1 << 32, size=M, dtype=np.uint64).astype(np.uint32)
        prio[::7] = prio[0]  # ties on the priority, broken by the claim index
        dres = torch.from_numpy(res).cuda()
        dprio = torch.from_numpy(prio.view(np.int32)).cuda()
        w_ref, f_ref, w, f = call_pair(abm, dres, dprio, R if call == 0 else R // 2)
        assert torch.equal(w, w_ref)
        assert torch.equal(f, f_ref)


def test_static_resolve_edge_cases(lib):
    """No claims; no per-claim flags wanted; claim arrays that start one element
    past a 16-byte boundary (the flags then take the unaligned path)."""
    abm = lib
    rng = np.random.default_rng(5)
    R = 1000
    st = abm.stream_handle()
    # M = 0: every resource reports no winner, whatever the array held before
    w = torch.full((R,), 77, dtype=torch.int32, device="cuda")
    abm.check(abm.lib().abm_resolve_static(None, None, 0, R, abm.ptr(w), None, st))
    torch.cuda.synchronize()
    assert bool((w == -1).all())
    M = 50_001
    res = torch.from_numpy(rng.integers(-2, R + 2, size=M + 1).astype(np.int32)).cuda()
    prio = torch.from_numpy(rng.integers(0, 1 << 32, size=M + 1, dtype=np.uint64).astype(np.uint32).view(np.int32)).cuda()
    for off in (0, 1):
        r_, p_ = res[off:off + M], prio[off:off + M]
        w_ref, f_ref, w, f = call_pair(abm, r_, p_, R)
        assert torch.equal(w, w_ref) and torch.equal(f, f_ref)
        # the same call without the per-claim flags
        w2 = torch.full((R,), 5, dtype=torch.int32, device="cuda")
        abm.check(abm.lib().abm_resolve_static(abm.ptr(r_), abm.ptr(p_), M, R, abm.ptr(w2), None, st))
        torch.cuda.synchronize()
        assert torch.equal(w2, w_ref)
    # flags written from an odd address as well
    fb = torch.zeros(M + 1, dtype=torch.uint8, device="cuda")
    abm.check(abm.lib().abm_resolve_static(abm.ptr(res[1:]), abm.ptr(prio[1:]), M, R, abm.ptr(w2),
                                           abm.ptr(fb[1:]), st))
    torch.cuda.synchronize()
    assert torch.equal(fb[1:], f_ref)


def test_static_resolve_allocates_nothing(lib):
    """Once a device has run the call, further calls leave the device's free
    memory unchanged: the scratch table is the library's own fixed array."""
    abm = lib
    M, R = 1 << 20, 1 << 16
    res = torch.from_numpy(workloads.zipf_claims(M, R, seed=9)).cuda()
    prio = torch.from_numpy(np.random.default_rng(9).integers(0, 1 << 31, size=M).astype(np.int32)).cuda()
    w = torch.empty(R, dtype=torch.int32, device="cuda")
    f = torch.empty(M, dtype=torch.uint8, device="cuda")
    st = abm.stream_handle()
    abm.check(abm.lib().abm_resolve_static(abm.ptr(res), abm.ptr(prio), M, R, abm.ptr(w), abm.ptr(f), st))
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        abm.check(abm.lib().abm_resolve_static(abm.ptr(res), abm.ptr(prio), M, R, abm.ptr(w), abm.ptr(f), st))
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0


def test_static_resolve_rejects_oversize(lib):
    abm = lib
    R = abm.RESOLVE_STATIC_MAX_R + 1
    res = torch.zeros(4, dtype=torch.int32, device="cuda")
    prio = torch.zeros(4, dtype=torch.int32, device="cuda")
    w = torch.empty(R, dtype=torch.int32, device="cuda")
    st = abm.lib().abm_resolve_static(abm.ptr(res), abm.ptr(prio), 4, R, abm.ptr(w), None, abm.stream_handle())
    assert st == abm.ERR_TOO_LARGE
    assert "maximum" in abm.strerror(st)
