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


def test_static_resolve_rejects_oversize(lib):
    abm = lib
    R = abm.RESOLVE_STATIC_MAX_R + 1
    res = torch.zeros(4, dtype=torch.int32, device="cuda")
    prio = torch.zeros(4, dtype=torch.int32, device="cuda")
    w = torch.empty(R, dtype=torch.int32, device="cuda")
    st = abm.lib().abm_resolve_static(abm.ptr(res), abm.ptr(prio), 4, R, abm.ptr(w), None, abm.stream_handle())
    assert st == abm.ERR_TOO_LARGE
    assert "maximum" in abm.strerror(st)
