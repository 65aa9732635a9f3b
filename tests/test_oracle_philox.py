"""Pin the oracle's Philox4x32-10 to a library implementation (CPU only).

Triton's ``tl.philox`` (run by Triton's CPU interpreter) implements the same
published generator (Salmon et al., SC'11) with key = (seed low word, seed high
word); the oracle's key is (seed, model). The GPU test suite pins the CUDA
side to cuRAND's ``curand_Philox4x32_10`` the same way.
"""
import os
import subprocess
import sys
import textwrap

import numpy as np
import pytest

import oracle

TRITON_SCRIPT = textwrap.dedent("""
    import os, sys, json
    os.environ["TRITON_INTERPRET"] = "1"
    import torch, triton, triton.language as tl

    @triton.jit
    def k(c_ptr, out_ptr, seed, n, BLOCK: tl.constexpr):
        i = tl.arange(0, BLOCK)
        m = i < n
        c0 = tl.load(c_ptr + 4 * i + 0, mask=m).to(tl.uint32)
        c1 = tl.load(c_ptr + 4 * i + 1, mask=m).to(tl.uint32)
        c2 = tl.load(c_ptr + 4 * i + 2, mask=m).to(tl.uint32)
        c3 = tl.load(c_ptr + 4 * i + 3, mask=m).to(tl.uint32)
        a, b, c, d = tl.philox(seed, c0, c1, c2, c3)
        tl.store(out_ptr + 4 * i + 0, a.to(tl.int64), mask=m)
        tl.store(out_ptr + 4 * i + 1, b.to(tl.int64), mask=m)
        tl.store(out_ptr + 4 * i + 2, c.to(tl.int64), mask=m)
        tl.store(out_ptr + 4 * i + 3, d.to(tl.int64), mask=m)

    req = json.loads(sys.stdin.read())
    res = []
    for seed, ctrs in req:
        c = torch.tensor(ctrs, dtype=torch.int64)
        out = torch.zeros_like(c)
        n = c.shape[0]
        k[(1,)](c, out, seed, n, BLOCK=triton.next_power_of_2(n))
        res.append([[x & 0xFFFFFFFF for x in row] for row in out.tolist()])
    print(json.dumps(res))
""")


def test_philox_matches_triton_interpreter():
    pytest.importorskip("triton")
    import json
    rng = np.random.default_rng(1)
    cases = []
    for _ in range(6):
        key = [int(x) for x in rng.integers(0, 2**32, size=2)]
        ctrs = rng.integers(0, 2**32, size=(16, 4)).tolist()
        ctrs[0] = [0, 0, 0, 0]
        ctrs[1] = [0xFFFFFFFF] * 4
        cases.append((key, ctrs))
    cases.append(([0, 0], [[0, 0, 0, 0], [1, 2, 3, 4]]))
    req = [[(k[1] << 32) | k[0], c] for k, c in cases]
    env = dict(os.environ, TRITON_INTERPRET="1")
    p = subprocess.run([sys.executable, "-c", TRITON_SCRIPT], input=json.dumps(req),
                       capture_output=True, text=True, env=env, timeout=600)
    if p.returncode != 0:
        pytest.skip("triton interpreter unavailable: " + p.stderr.strip().splitlines()[-1])
    got = json.loads(p.stdout.strip().splitlines()[-1])
    for (key, ctrs), want in zip(cases, got):
        for c, w in zip(ctrs, want):
            np.testing.assert_array_equal(oracle.philox(c, key), np.array(w, dtype=np.uint32))


def test_philox_words_layout():
    # bulk draws are the per-counter generator with the slot in counter word 1
    seed, model, step, purpose, species = 7, 3, 11, oracle.P_MOVE, 1
    for word in range(4):
        bulk = oracle.philox_words(seed, model, step, purpose, species, 100, 5, word)
        for i in range(5):
            one = oracle.philox([step, 100 + i, purpose, species], [seed, model])
            assert bulk[i] == one[word]


def test_philox_bits_uniform():
    # coarse chi-square on the top byte and per-bit balance of word 0
    u = oracle.philox_words(1, 0, 0, oracle.P_MASK, 0, 0, 1 << 16)
    hist = np.bincount((u >> 24).astype(np.int64), minlength=256)
    e = u.size / 256
    chi2 = float(((hist - e) ** 2 / e).sum())
    assert chi2 < 400  # 255 dof: mean 255, sd ~22.6
    bits = ((u[:, None] >> np.arange(32, dtype=np.uint32)) & 1).mean(axis=0)
    assert np.all(np.abs(bits - 0.5) < 0.01)
