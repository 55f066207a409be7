"""Pins for the oracle's Philox4x32-10 streams (CPU only)."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

from oracle import philox

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

_TRITON_SCRIPT = r"""
import json, os, sys
os.environ["TRITON_INTERPRET"] = "1"
import numpy as np, torch, triton, triton.language as tl

@triton.jit
def _k(c_ptr, out_ptr, seed, n: tl.constexpr):
    i = tl.arange(0, n)
    c0 = tl.load(c_ptr + 4 * i + 0)
    c1 = tl.load(c_ptr + 4 * i + 1)
    c2 = tl.load(c_ptr + 4 * i + 2)
    c3 = tl.load(c_ptr + 4 * i + 3)
    a, b, c, d = tl.philox(seed, c0, c1, c2, c3)
    tl.store(out_ptr + 4 * i + 0, a)
    tl.store(out_ptr + 4 * i + 1, b)
    tl.store(out_ptr + 4 * i + 2, c)
    tl.store(out_ptr + 4 * i + 3, d)

cfg = json.loads(sys.argv[1])
ctr = np.array(cfg["ctr"], dtype=np.uint32).view(np.int32)
out = torch.zeros(ctr.size, dtype=torch.int32)
_k[(1,)](torch.from_numpy(ctr.copy()), out, cfg["seed"], ctr.size // 4)
print(json.dumps(out.numpy().view(np.uint32).tolist()))
"""


def test_philox_matches_library_implementation():
    """Triton's tl.philox (run by its CPU interpreter) is an independent
    Philox4x32-10: key (seed lo, seed hi), counter (c0..c3)."""
    pytest.importorskip("triton")
    pytest.importorskip("torch")
    g = np.random.default_rng(7)
    n = 64
    ctr = g.integers(0, 2 ** 32, size=(n, 4), dtype=np.uint64)
    ctr[0] = 0
    ctr[1] = 0xFFFFFFFF
    for seed in (0, 2008054010, 0x123456789ABCDEF, 2 ** 63 - 25):
        env = dict(os.environ, TRITON_INTERPRET="1")
        res = subprocess.run([sys.executable, "-c", _TRITON_SCRIPT,
                              json.dumps({"ctr": ctr.ravel().tolist(), "seed": int(seed)})],
                             capture_output=True, text=True, env=env, timeout=600)
        assert res.returncode == 0, res.stderr[-2000:]
        lib = np.array(json.loads(res.stdout.strip().splitlines()[-1]), dtype=np.uint32).reshape(n, 4)
        ours = np.stack(philox.philox4x32_10(ctr[:, 0], ctr[:, 1], ctr[:, 2], ctr[:, 3],
                                             seed & 0xFFFFFFFF, seed >> 32), axis=1)
        np.testing.assert_array_equal(ours, lib)


def test_stream_layout_and_range():
    seed, chains = 99, np.array([0, 1, 2 ** 32 - 1], dtype=np.uint64)
    w = philox.words(seed, chains, 5, 3, 10)
    for c, cid in enumerate(chains):
        for n in range(10):
            blk = philox.philox4x32_10(n // 4, 3, 5, int(cid), seed, 0)
            assert w[c, n] == blk[n % 4]
    u = philox.uniforms(seed, chains, 5, 3, 10)
    assert np.all(u > 0) and np.all(u < 1)
    # extreme words map strictly inside (0, 1)
    assert (0 + 0.5) * 2.0 ** -32 > 0 and (2 ** 32 - 1 + 0.5) * 2.0 ** -32 < 1


def test_uniformity_and_stream_independence():
    seed = 2008054010
    chains = np.arange(64, dtype=np.uint64)
    u = philox.uniforms(seed, chains, 0, 0, 4096).ravel()
    counts, _ = np.histogram(u, bins=64, range=(0, 1))
    expected = u.size / 64
    chi2 = ((counts - expected) ** 2 / expected).sum()
    assert chi2 < 63 + 6 * np.sqrt(2 * 63)          # ~6 sigma of chi^2_63
    assert abs(u.mean() - 0.5) < 6 * np.sqrt(1 / 12 / u.size)
    # neighbouring tags / steps / chains / seeds give unrelated words
    a = philox.words(seed, chains, 0, 0, 256)
    for other in (philox.words(seed, chains, 1, 0, 256), philox.words(seed, chains, 0, 1, 256),
                  philox.words(seed, chains + 1, 0, 0, 256), philox.words(seed + 1, chains, 0, 0, 256)):
        assert (a == other).mean() < 1e-3
        corr = np.corrcoef(a.ravel().astype(float), other.ravel().astype(float))[0, 1]
        assert abs(corr) < 6 / np.sqrt(a.size)
