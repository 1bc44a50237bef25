"""Pins for the oracle's Philox4x32-10 and its integer decision rules.

Philox4x32-10 is checked against an independent implementation run as a
library: Triton's ``tl.philox`` executed by the Triton interpreter on the CPU
(key = the 64-bit seed split into low/high words, counter = c0..c3).
"""
import json
import os
import subprocess
import sys
from fractions import Fraction

import numpy as np
import pytest

import oracle

_TRITON_SCRIPT = r"""
import json, os, sys
os.environ["TRITON_INTERPRET"] = "1"
import numpy as np, torch, triton, triton.language as tl

@triton.jit
def k(out_ptr, c_ptr, seed, n, BLOCK: tl.constexpr):
    offs = tl.arange(0, BLOCK)
    m = offs < n
    c0 = tl.load(c_ptr + offs * 4 + 0, mask=m)
    c1 = tl.load(c_ptr + offs * 4 + 1, mask=m)
    c2 = tl.load(c_ptr + offs * 4 + 2, mask=m)
    c3 = tl.load(c_ptr + offs * 4 + 3, mask=m)
    a, b, c, d = tl.philox(seed, c0, c1, c2, c3, 10)
    tl.store(out_ptr + offs * 4 + 0, a, mask=m)
    tl.store(out_ptr + offs * 4 + 1, b, mask=m)
    tl.store(out_ptr + offs * 4 + 2, c, mask=m)
    tl.store(out_ptr + offs * 4 + 3, d, mask=m)

cases = json.loads(sys.stdin.read())
res = []
for seed, ctrs in cases:
    c = torch.tensor(np.array(ctrs, dtype=np.uint32).reshape(-1).view(np.int32)).view(torch.uint32)
    n = len(ctrs)
    out = torch.zeros(4 * n, dtype=torch.uint32)
    k[(1,)](out, c, seed, n, BLOCK=triton.next_power_of_2(n))
    res.append(out.view(torch.int32).numpy().view(np.uint32).reshape(n, 4).tolist())
print(json.dumps(res))
"""


def _triton_philox(cases):
    pytest.importorskip("triton")
    r = subprocess.run([sys.executable, "-c", _TRITON_SCRIPT], input=json.dumps(cases),
                       capture_output=True, text=True, timeout=600, env=dict(os.environ, TRITON_INTERPRET="1"))
    if r.returncode != 0:
        pytest.skip("Triton interpreter unavailable: " + r.stderr[-300:])
    return json.loads(r.stdout.strip().splitlines()[-1])


def test_philox_matches_triton_interpreter():
    rng = np.random.default_rng(11)
    cases = []
    seeds = [0, 1, 0xFFFFFFFF, 0x123456789ABCDEF0, int(rng.integers(0, 2**63))]
    for s in seeds:
        ctrs = [[0, 0, 0, 0], [1, 2, 3, 4], [0xFFFFFFFF] * 4] + \
               rng.integers(0, 2**32, size=(13, 4), dtype=np.uint64).tolist()
        cases.append([s, [[int(x) for x in c] for c in ctrs]])
    ref = _triton_philox(cases)
    for (seed, ctrs), outs in zip(cases, ref):
        key = [seed & 0xFFFFFFFF, seed >> 32]
        for c, o in zip(ctrs, outs):
            assert oracle.philox(c, key).tolist() == o, (seed, c)


def test_philox_words_look_uniform():
    # 4 * 20000 words; each of 16 equal bins of the top 4 bits must be within 5 sigma
    words = np.array([oracle.philox([i, 7, 0, 0], [3, 0]) for i in range(20000)]).reshape(-1)
    counts = np.bincount(words >> 28, minlength=16)
    exp = words.size / 16
    assert np.all(np.abs(counts - exp) < 5 * np.sqrt(exp))


@pytest.mark.parametrize("p", [0.0, 1e-12, 0.3, 0.5, 0.8, 0.95, 1 - 2**-40, 1.0, 1.5, -0.1])
def test_threshold_is_floor_p_times_2_32(p):
    if p <= 0:
        want = 0
    elif p >= 1:
        want = 2**32
    else:
        want = int(Fraction(p) * 2**32)  # exact rational floor
    assert oracle.threshold(p) == want


def test_poisson_thresholds_match_library_cdf():
    scipy_stats = pytest.importorskip("scipy.stats")
    for mean in (0.5, 2.0, 3.7):
        thr = oracle.poisson_thresholds(mean).astype(np.int64)
        ref = np.floor(scipy_stats.poisson.cdf(np.arange(15), mean) * 2**32).astype(np.int64)
        assert np.all(np.abs(thr - ref) <= 1), (mean, thr - ref)
        assert np.all(np.diff(thr) >= 0)


def test_random_contacts_distribution():
    """Daily random network: count ~ Poisson(mean) capped at 15, contacts uniform over
    the other n-1 agents, never the agent itself."""
    scipy_stats = pytest.importorskip("scipy.stats")
    n, mean = 50, 2.0
    counts = []
    hits = np.zeros(n, np.int64)
    for step in range(40):
        for j in range(n):
            c = oracle.random_contacts(99, n, j, step, mean)
            assert np.all(c != j) and np.all(c < n)
            counts.append(c.size)
            hits[c] += 1
    counts = np.array(counts)
    obs = np.bincount(counts, minlength=16)[:8].astype(float)
    expct = scipy_stats.poisson.pmf(np.arange(8), mean) * counts.size
    chi2 = float(((obs - expct) ** 2 / np.maximum(expct, 1e-9))[expct > 5].sum())
    assert chi2 < 30, chi2
    assert abs(counts.mean() - mean) < 5 * np.sqrt(mean / counts.size)
    assert hits.min() > 0.6 * hits.mean() and hits.max() < 1.4 * hits.mean()


@pytest.mark.gpu
def test_philox_matches_curand(tmp_path):
    """The oracle's Philox4x32-10 against cuRAND's device implementation (a
    library, compiled and run on the GPU by this test) on 10^5 random
    (key, counter) pairs, including the day words the method uses (0xFFFFFFFF
    and 0xFFFFFFFE are out of cuRAND's offset range here, so c1 < 2^30)."""
    import shutil
    import subprocess
    try:
        import torch
        if not torch.cuda.is_available():
            pytest.skip("needs a CUDA GPU")
    except ImportError:
        pytest.skip("needs torch")
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    exe = tmp_path / "curand_philox_ref"
    src = os.path.join(os.path.dirname(__file__), "curand_philox_ref.cu")
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O2", "-o", str(exe), src], check=True)
    rng = np.random.default_rng(2024)
    n = 100_000
    rec = rng.integers(0, 2**32, size=(n, 6), dtype=np.uint64).astype(np.uint32)
    rec[:, 3] &= (1 << 30) - 1
    inp = tmp_path / "in.bin"
    with open(inp, "wb") as f:
        f.write(np.uint32(n).tobytes())
        f.write(rec.tobytes())
    out = tmp_path / "out.bin"
    subprocess.run([str(exe), str(inp), str(out)], check=True, timeout=120)
    ref = np.fromfile(out, dtype=np.uint32).reshape(n, 4)
    for i in range(n):
        got = oracle.philox(rec[i, 2:6], rec[i, 0:2])
        assert np.array_equal(got, ref[i]), (i, rec[i], got, ref[i])
