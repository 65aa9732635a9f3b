"""Philox4x32-10 against NVIDIA's cuRAND implementation of the same generator.

cuRAND's device header ships `curand_Philox4x32_10(counter, key)`, the
Philox4x32-10 block function of Salmon et al. (SC'11). A small program built
here runs it on the GPU for random counters and keys; its words must equal
the oracle's Philox (written from the paper's description) and the engine's
device draws (read back through abm_philox_records), word for word.
"""
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

PROGRAM = r"""
#include <cstdio>
#include <cstdlib>
#include <curand_kernel.h>
__global__ void k(const uint4* c, const uint2* key, uint4* out, int n) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = curand_Philox4x32_10(c[i], key[i]);
}
int main(int argc, char** argv) {
  FILE* f = fopen(argv[1], "rb");
  int n = 0;
  if (!f || fread(&n, 4, 1, f) != 1 || n <= 0 || n > (1 << 20)) return 2;
  uint4* hc = (uint4*)malloc(16 * (size_t)n);
  uint2* hk = (uint2*)malloc(8 * (size_t)n);
  if (fread(hc, 16, n, f) != (size_t)n || fread(hk, 8, n, f) != (size_t)n) return 3;
  fclose(f);
  uint4 *dc, *dout;
  uint2* dk;
  if (cudaMalloc(&dc, 16 * (size_t)n) || cudaMalloc(&dk, 8 * (size_t)n) || cudaMalloc(&dout, 16 * (size_t)n)) return 4;
  cudaMemcpy(dc, hc, 16 * (size_t)n, cudaMemcpyHostToDevice);
  cudaMemcpy(dk, hk, 8 * (size_t)n, cudaMemcpyHostToDevice);
  k<<<(n + 255) / 256, 256>>>(dc, dk, dout, n);
  if (cudaDeviceSynchronize() != cudaSuccess) return 5;
  cudaMemcpy(hc, dout, 16 * (size_t)n, cudaMemcpyDeviceToHost);
  FILE* g = fopen(argv[2], "wb");
  if (!g || fwrite(hc, 16, n, g) != (size_t)n) return 6;
  fclose(g);
  return 0;
}
"""


@pytest.fixture(scope="module")
def curand_philox(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    d = tmp_path_factory.mktemp("curand")
    src, exe = d / "p.cu", d / "p"
    src.write_text(PROGRAM)
    subprocess.run([nvcc, "-O2", "-gencode", "arch=compute_103a,code=sm_103a", "-o", str(exe), str(src)],
                   check=True, timeout=300)

    def run(counters: np.ndarray, keys: np.ndarray) -> np.ndarray:
        n = counters.shape[0]
        fin, fout = d / "in.bin", d / "out.bin"
        with open(fin, "wb") as f:
            f.write(np.int32(n).tobytes())
            f.write(np.ascontiguousarray(counters, dtype=np.uint32).tobytes())
            f.write(np.ascontiguousarray(keys, dtype=np.uint32).tobytes())
        subprocess.run([str(exe), str(fin), str(fout)], check=True, timeout=120)
        return np.fromfile(fout, dtype=np.uint32).reshape(n, 4)

    return run


def test_oracle_philox_equals_curand(curand_philox):
    rng = np.random.default_rng(2024)
    n = 4096
    counters = rng.integers(0, 2**32, size=(n, 4), dtype=np.uint64).astype(np.uint32)
    keys = rng.integers(0, 2**32, size=(n, 2), dtype=np.uint64).astype(np.uint32)
    counters[:4] = [[0, 0, 0, 0], [0xFFFFFFFF] * 4, [1, 2, 3, 4], [0xFFFFFFFF, 7, 5, 1]]
    keys[:4] = [[0, 0], [0xFFFFFFFF] * 2, [5, 6], [1, 0]]
    got = curand_philox(counters, keys)
    want = np.array([oracle.philox(c.tolist(), k.tolist()) for c, k in zip(counters, keys)], dtype=np.uint32)
    np.testing.assert_array_equal(want, got)


def test_engine_draws_equal_curand(curand_philox):
    """abm_philox_records: words 0-3 of record j = Philox((step, j, p0, 0), (seed, model)),
    words 4-7 the same with p1."""
    from paper_2508_16508_gb300 import abm, engine
    abm.lib()
    seed, model, step, k = 12345, 77, 9, 3000
    s = engine.Slab(16, 8, seed=seed, model=model)
    rec = s.philox_records(step, abm.P_NEWREC0, abm.P_NEWREC1, k).cpu().numpy().view(np.uint32)
    j = np.arange(k, dtype=np.uint32)
    keys = np.tile(np.array([[seed, model]], dtype=np.uint32), (k, 1))
    for half, purpose in ((0, abm.P_NEWREC0), (1, abm.P_NEWREC1)):
        counters = np.stack([np.full(k, step, np.uint32), j, np.full(k, purpose, np.uint32),
                             np.zeros(k, np.uint32)], axis=1)
        np.testing.assert_array_equal(rec[:, 4 * half:4 * half + 4], curand_philox(counters, keys))
