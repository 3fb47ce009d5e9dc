"""Pins of the oracle's random force (Sec. III.C).

Philox4x32-10 is compared with ATen's independent header-only engine (a
library routine, compiled here from torch's headers). Box-Muller is pinned by
its defining invariants (radius and angle of each pair) and by the moments
and distribution of many draws.
"""
import ctypes
import math
import os
import subprocess

import numpy as np
import pytest
from scipy import stats

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def aten():
    torch = pytest.importorskip("torch")
    inc = os.path.join(os.path.dirname(torch.__file__), "include")
    if not os.path.exists(os.path.join(inc, "ATen", "core", "PhiloxRNGEngine.h")):
        pytest.skip("ATen Philox header not available")
    out = os.path.join(HERE, "_lib")
    os.makedirs(out, exist_ok=True)
    so = os.path.join(out, "libatenphilox.so")
    src = os.path.join(HERE, "aten_philox.cpp")
    if not os.path.exists(so) or os.path.getmtime(so) < os.path.getmtime(src):
        subprocess.check_call(["g++", "-O1", "-std=c++17", "-fPIC", "-shared", "-I", inc, "-o", so, src])
    L = ctypes.CDLL(so)
    L.aten_philox_block.argtypes = [ctypes.c_uint64] * 3 + [ctypes.c_void_p]
    return L


def test_philox_matches_aten(orc, aten):
    rng = np.random.default_rng(0)
    cases = [(0, 0, 0), (2**64 - 1, 2**64 - 1, 2**64 - 1), (1, 0, 0), (0, 1, 0), (0, 0, 1)]
    cases += [tuple(int(v) for v in rng.integers(0, 2**63, size=3, dtype=np.int64)) for _ in range(200)]
    out = np.zeros(4, np.uint32)
    for seed, sub, off in cases:
        aten.aten_philox_block(seed, sub, off, out.ctypes.data)
        # ATen: key = seed, counter = (offset lo, offset hi, subsequence lo, subsequence hi)
        mine = orc.philox([off & 0xFFFFFFFF, off >> 32, sub & 0xFFFFFFFF, sub >> 32],
                          [seed & 0xFFFFFFFF, seed >> 32])
        assert np.array_equal(out, mine), (seed, sub, off)


def test_noise_uses_seed_step_bead_counter(orc, aten):
    # orc_noise(seed, step, bead) draws the block with key = seed, counter = (step, bead, 0)
    out = np.zeros(4, np.uint32)
    for seed, step, bead in ((7, 0, 0), (3, 12345, 77), (2**40 + 5, 2**33 + 9, 1_000_000)):
        aten.aten_philox_block(seed, bead, step, out.ctypes.data)
        assert np.array_equal(orc.box_muller(out), orc.noise(seed, step, bead))


def test_box_muller_invariants(orc):
    rng = np.random.default_rng(1)
    for x in rng.integers(0, 2**32, size=(500, 4), dtype=np.uint64).astype(np.uint32):
        g = orc.box_muller(x)
        u1 = (float(x[0]) + 1.0) / 2**32
        u2 = float(x[1]) / 2**32
        u3 = (float(x[2]) + 1.0) / 2**32
        u4 = float(x[3]) / 2**32
        # radius of the first pair, angle of the first pair, and g2 on the second pair's circle
        assert g[0] ** 2 + g[1] ** 2 == pytest.approx(-2.0 * math.log(u1), rel=1e-12, abs=1e-300)
        ang = math.atan2(g[1], g[0]) % (2 * math.pi)
        if g[0] ** 2 + g[1] ** 2 > 1e-20:
            assert min(abs(ang - 2 * math.pi * u2), 2 * math.pi - abs(ang - 2 * math.pi * u2)) < 1e-9
        assert abs(g[2]) <= math.sqrt(-2.0 * math.log(u3)) * (1 + 1e-14)
        assert math.copysign(1.0, g[2]) == math.copysign(1.0, math.cos(2 * math.pi * u4)) or g[2] == 0.0


def test_box_muller_edges(orc):
    # x0 = 2^32 - 1 gives u1 = 1 and a zero radius; x0 = 0 gives the largest radius sqrt(64 ln 2).
    g = orc.box_muller(np.array([0xFFFFFFFF, 123, 0xFFFFFFFF, 5], np.uint32))
    assert np.all(g == 0.0)
    g = orc.box_muller(np.array([0, 0, 0, 0], np.uint32))
    assert g[0] == pytest.approx(math.sqrt(64.0 * math.log(2.0)), rel=1e-14)
    assert g[1] == 0.0
    assert np.all(np.isfinite(g))


def test_noise_moments_and_distribution(orc):
    n = 40000
    g = np.array([orc.noise(12345, s, b) for s in range(4) for b in range(n // 4)])
    se = 1.0 / math.sqrt(len(g))
    assert np.all(np.abs(g.mean(0)) < 5 * se)
    assert np.all(np.abs(g.var(0) - 1.0) < 5 * math.sqrt(2.0) * se)
    k = stats.kurtosis(g, axis=0, fisher=False)
    assert np.all(np.abs(k - 3.0) < 5 * math.sqrt(24.0) * se)
    for c in range(3):
        assert stats.kstest(g[:, c], "norm").pvalue > 1e-4
    cor = np.corrcoef(g.T)
    assert np.abs(cor - np.eye(3)).max() < 5 * se
