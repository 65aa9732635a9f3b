"""Failure detection without faulting the GPU.

A bounded device-side wait that can never complete (a grid barrier expecting
one CTA more than the grid has) must end with ABM_ERR_DEVICE_TIMEOUT, and the
context must stay usable: a predation world run right after still matches the
oracle. Host-side failures (bad arguments, impossible sizes) are rejected
before anything is enqueued.
"""
import ctypes as C

import numpy as np
import pytest

import oracle
import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def eng():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2508_16508_gb300 import abm, engine
    abm.lib()
    return abm, engine


def test_barrier_wait_times_out_and_context_survives(eng):
    abm, engine = eng
    st = abm.lib().abm_diag_barrier_timeout(1 << 14, abm.stream_handle())
    assert st == abm.ERR_DEVICE_TIMEOUT
    assert abm.lib().abm_diag_barrier_timeout(0, abm.stream_handle()) == abm.ERR_ARG
    c = workloads.PRED_SMALL
    gw = engine.World(c["side"], c["seed"], c["model"], c["params"], c["cap"], c["n0"])
    ow = oracle.World(c["side"], c["seed"], c["model"], c["params"], c["cap"], c["n0"])
    gw.step(40)
    ow.step(40)
    for s in range(2):
        for f in ("active", "cell", "energy", "id", "age"):
            assert np.array_equal(gw.agents(s, f).cpu().numpy(), ow.agents(s, f))
    gw.check()


def test_host_side_rejections(eng):
    abm, engine = eng
    L = abm.lib()
    h = C.c_void_p()
    cfg = abm.abm_config()
    cfg.side = 10
    cfg.cap[0] = cfg.cap[1] = 10
    cfg.n0[0] = 11  # more initial agents than slots
    cfg.params[4] = 5
    assert L.abm_create(C.byref(cfg), None, C.byref(h)) == abm.ERR_ARG
    cfg.n0[0] = 5
    cfg.params[4] = 0  # regrowth delay must be >= 1
    assert L.abm_create(C.byref(cfg), None, C.byref(h)) == abm.ERR_ARG
    arr = (abm.abm_batch_model * 1)()
    arr[0].side = 0
    assert L.abm_batch_create(arr, 1, None, C.byref(h)) == abm.ERR_ARG
    assert L.abm_mlp_create(12, 128, 3, 2, 0, 0, None, C.byref(h)) == abm.ERR_ARG
    s = engine.Slab(8, 2)
    assert L.abm_slab_tune(s.h, 96, 2, None) == abm.ERR_ARG
    assert L.abm_slab_read(s.h, 5, None, 8, None) == abm.ERR_ARG
