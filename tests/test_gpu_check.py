"""The check build (libabm_check.so: the library compiled with -DABM_CHECK,
which tests every data-dependent index before use and keeps canaries past
each slab's capacity) on the GPU -- the stand-in for a memory checker, which
is not available here. The same workloads run in both builds in separate
processes: every check reports clean and every result is identical. The
canary and index tests themselves are shown to fire without any access out
of bounds: a canary is overwritten through the slab's own allocation, and
the index test runs on a value with no access behind it."""
import ctypes as C
import json
import os
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


def run_workload(check: bool) -> dict:
    env = dict(os.environ)
    env["ABM_LIBRARY"] = "check" if check else ""
    p = subprocess.run([sys.executable, os.path.join(HERE, "check_workload.py")], env=env, capture_output=True,
                       text=True, timeout=1800)
    assert p.returncode == 0, p.stderr[-3000:]
    return json.loads(p.stdout.strip().splitlines()[-1])


@pytest.fixture(scope="module")
def results():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return run_workload(False), run_workload(True)


def test_check_build_is_clean_and_identical(results):
    plain, checked = results
    assert plain["version"] > 0 and checked["version"] < 0
    assert all(v == 0 for v in checked["checks"].values()), checked["checks"]
    assert all(v == 0 for v in plain["checks"].values()), plain["checks"]
    assert checked["digests"] == plain["digests"]


def test_canary_and_index_test_fire():
    """In the check build only: a slab whose padding is overwritten (through
    its own allocation) reports ABM_ERR_CHECK, and the index test reports an
    index out of range. Run in a child process so this one keeps the normal build."""
    code = r'''
import ctypes as C, json, sys, torch
sys.path.insert(0, %r)
from paper_2508_16508_gb300 import abm, engine
L = abm.lib()
st = abm.stream_handle()
out = {"version": int(L.abm_version())}
s = engine.Slab(1000, 8)
out["clean"] = int(L.abm_slab_check(s.h, st))
act, fld, stride = C.c_void_p(), C.c_void_p(), C.c_int32()
abm.check(L.abm_slab_arrays(s.h, C.byref(act), C.byref(fld), C.byref(stride)))
pad = torch.empty(1, dtype=torch.int32, device="cuda")  # keeps torch's context alive
torch.cuda.synchronize()
# slot 1000 is past the capacity but inside the allocation (padded to 16384 slots)
import os
rt = None
for name in ("/usr/local/cuda/lib64/libcudart.so", "libcudart.so"):
    try:
        rt = C.CDLL(name)
        break
    except OSError:
        pass
rt.cudaMemset.argtypes = [C.c_void_p, C.c_int, C.c_size_t]
assert rt.cudaMemset(C.c_void_p(fld.value + 1000 * 8 * 4), 0, 32) == 0
assert rt.cudaDeviceSynchronize() == 0
out["damaged"] = int(L.abm_slab_check(s.h, st))
out["index_in"] = int(L.abm_diag_check_index(2, 3, st))
out["index_out"] = int(L.abm_diag_check_index(5, 3, st))
out["index_neg"] = int(L.abm_diag_check_index(-1, 3, st))
print(json.dumps(out))
''' % os.path.dirname(HERE)
    env = dict(os.environ)
    env["ABM_LIBRARY"] = "check"
    p = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=900)
    assert p.returncode == 0, p.stderr[-3000:]
    r = json.loads(p.stdout.strip().splitlines()[-1])
    from paper_2508_16508_gb300 import abm
    assert r["version"] < 0
    assert r["clean"] == abm.OK
    assert r["damaged"] == abm.ERR_CHECK
    assert (r["index_in"], r["index_out"], r["index_neg"]) == (abm.OK, abm.ERR_CHECK, abm.ERR_CHECK)
