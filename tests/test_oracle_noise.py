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


# ---------------------------------------------------------------------------------------
# Hybrid Taus (Algorithm 6): each component is pinned against its defining bit-level
# recurrence, the LCG against its closed form, both with the paper's printed constants
# (tests/golden/paper_values.json, Sec. III.C). A Tausworthe component with state 0 stays
# 0, so one component's sequence is isolated by XOR-ing two runs that differ only in it.
# ---------------------------------------------------------------------------------------
def _golden_taus():
    import json
    with open(os.path.join(HERE, "golden", "paper_values.json")) as f:
        return json.load(f)["sec_III_C_algorithm_6_hybrid_taus"]


def _outputs(orc, state, n):
    st = np.array(state, np.uint32)
    return np.array([orc.taus_next(st) for _ in range(n)], np.uint64)


def _isolated(orc, comp, seed_word, lcg_seed, n):
    state = [0, 0, 0, lcg_seed]
    state[comp] = seed_word
    return _outputs(orc, state, n) ^ _outputs(orc, [0, 0, 0, lcg_seed], n)


def _bit_recurrence_words(seed_word, q, kms, s, mask, n):
    """Words n = 1..n of the Tausworthe generator defined bit by bit: b_j = b_{j-k+q} xor
    b_{j-k} (characteristic trinomial z^k + z^q + 1), word n = bits b_{ns} .. b_{ns+31}, most
    significant first; b_0 .. b_{k-1} are the top k bits of the seed word."""
    k = bin(mask).count("1")
    assert mask == (0xFFFFFFFF << (32 - k)) & 0xFFFFFFFF and kms + s == k
    bits = [(seed_word >> (31 - t)) & 1 for t in range(k)]
    need = n * s + 32
    while len(bits) < need:
        j = len(bits)
        bits.append(bits[j - k + q] ^ bits[j - k])
    words = []
    for m in range(1, n + 1):
        w = 0
        for t in range(32):
            w = (w << 1) | bits[m * s + t]
        words.append(w)
    return np.array(words, np.uint64)


@pytest.mark.parametrize("comp", [0, 1, 2])
def test_taus_components_follow_their_recurrences(orc, comp):
    g = _golden_taus()
    q, kms, s, mask = g["tausworthe_q_kms_s_mask"][comp]
    rng = np.random.default_rng(11 + comp)
    for seed_word in [int(x) for x in rng.integers(1 << 28, 1 << 32, size=4)] + [0xFFFFFFFF]:
        got = _isolated(orc, comp, seed_word, 12345, 200)
        ref = _bit_recurrence_words(seed_word, q, kms, s, mask, 200)
        assert np.array_equal(got, ref), (comp, seed_word)


def test_taus_lcg_closed_form(orc):
    g = _golden_taus()
    a, c = g["lcg_a"], g["lcg_c"]
    for y0 in (0, 1, 2 ** 31 + 7, 4294967295):
        got = _outputs(orc, [0, 0, 0, y0], 300)
        for n in (1, 2, 3, 17, 100, 299):
            geom = (pow(a, n) - 1) // (a - 1)          # sum_{i<n} a^i, exact
            ref = (pow(a, n, 1 << 32) * y0 + c * geom) % (1 << 32)
            assert int(got[n - 1]) == ref, (y0, n)


def test_taus_output_is_xor_of_components(orc):
    st = [0x9E3779B9, 0x7F4A7C15, 0xF39CC060, 0x5CEDC834]
    full = _outputs(orc, st, 100)
    parts = [_outputs(orc, [st[0], 0, 0, 0], 100), _outputs(orc, [0, st[1], 0, 0], 100),
             _outputs(orc, [0, 0, st[2], 0], 100), _outputs(orc, [0, 0, 0, 0], 100)]
    lcg0 = parts[3]
    comb = (parts[0] ^ lcg0) ^ (parts[1] ^ lcg0) ^ (parts[2] ^ lcg0) ^ _outputs(orc, [0, 0, 0, st[3]], 100)
    assert np.array_equal(full, comb)


def test_taus_uniforms_and_normals(orc):
    g = _golden_taus()
    st = np.array([0x12345678, 0x9ABCDEF0, 0x0FEDCBA9, 0x87654321], np.uint32)
    u = _outputs(orc, st, 200000).astype(np.float64) * g["mult"]
    assert stats.kstest(u, "uniform").pvalue > 1e-3
    assert abs(u.mean() - 0.5) < 5 * math.sqrt(1 / 12 / len(u))
    # the noise of one bead-step: Box-Muller of four successive outputs
    s0 = np.array([0x12345678, 0x9ABCDEF0, 0x0FEDCBA9, 0x87654321], np.uint32)
    x = _outputs(orc, s0, 4).astype(np.uint32)
    m = orc.Model(np.array([[0.0, 0.0, 0.0]]), np.zeros(1, np.int32), np.zeros(1, np.int32))
    m.set_taus_state(s0.reshape(1, 4))
    F = np.zeros((1, 3))
    x1 = m.ermak_update(np.zeros((1, 3)), F, seed=0, step=0)
    amp = math.sqrt(2 * orc.kB() * 300.0 * 0.1 / 50.0)
    assert np.allclose(x1[0], orc.box_muller(x) * amp, rtol=0, atol=1e-15)
    st2 = s0.copy()
    for _ in range(4):
        orc.taus_next(st2)
    assert np.array_equal(m.taus_state()[0], st2)
