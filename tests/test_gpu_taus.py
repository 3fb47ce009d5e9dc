"""Hybrid Taus noise (Algorithm 6) through the C ABI against the FP64 oracle (needs a GPU).

The generator state is integer work: after a run the GPU's per-bead state must equal the
oracle's bit for bit (a bead's generator advances by four outputs in each step in which
the bead moves). Positions after 100 steps from the same states agree within 1e-3 A RMS.
"""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

RMS_TOL = 1e-3


@pytest.fixture(scope="module")
def sop():
    from paper_1003_1148_gb300 import build, sop as s
    build.build()
    s.load()
    return s


def random_state(rng, R, n):
    st = rng.integers(0, 2 ** 32, size=(R, n, 4), dtype=np.uint64).astype(np.uint32)
    st[..., 0] = np.maximum(st[..., 0], 2)
    st[..., 1] = np.maximum(st[..., 1], 8)
    st[..., 2] = np.maximum(st[..., 2], 16)
    return st


def oracle_model(orc, w, x_start):
    m = orc.model_from_workload(w)
    if w.pulls:
        sys_of = w.system_of_bead()
        m.start_pulls([(int(sys_of[p.anchor]), p.anchor, p.pulled, p.k_s, p.v) for p in w.pulls], x_start)
    return m


@pytest.mark.parametrize("schedule", ["batched", "streamed", "pairs", "plain", "batched_pairs"])
def test_taus_trajectory_and_state_match_oracle(sop, orc, synth, schedule):
    w = synth.uneven(n_chains=5, lo=50, hi=240, steps=100)
    R = 2
    sim = sop.from_workload(w, n_replicas=R, schedule=schedule, rng="taus")
    st0 = random_state(np.random.default_rng(5), R, w.n_beads)
    sim.set_rng_state(st0)
    x0 = sim.get_positions(0)
    sim.step(100)
    st1 = sim.get_rng_state()
    for r in range(R):
        m = oracle_model(orc, w, x0)
        m.set_taus_state(st0[r])
        xo, _, _, _ = m.run(x0, 100, seed=0)
        assert np.array_equal(st1[r], m.taus_state()), (schedule, r)
        rms = float(np.sqrt(((sim.get_positions(r) - xo) ** 2).sum(1).mean()))
        assert rms <= RMS_TOL, (schedule, r, rms)
    # fixed beads (the pull anchors) never draw
    fixed = np.zeros(w.n_beads, bool) if w.fixed is None else np.asarray(w.fixed, bool).copy()
    for p in w.pulls:
        fixed[p.anchor] = True
    assert np.array_equal(st1[:, fixed], st0[:, fixed])
    assert not np.any(np.all(st1[:, ~fixed] == st0[:, ~fixed], axis=-1))
    sim.close()


def splitmix64(x):
    """SplitMix64 (Steele, Lea, Flood, OOPSLA'14): returns (output, new state)."""
    M = (1 << 64) - 1
    x = (x + 0x9E3779B97F4A7C15) & M
    z = x
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M
    return z ^ (z >> 31), x


def test_taus_default_seeding(sop, synth):
    w = synth.chain64()
    sim = sop.from_workload(w, n_replicas=3, schedule="streamed", rng="taus")
    st = sim.get_rng_state()
    seed = w.seed
    for r in range(3):
        for i in (0, 1, 31, 63):
            x = (((seed + r) << 32) + i) & ((1 << 64) - 1)
            a, x = splitmix64(x)
            b, x = splitmix64(x)
            ref = [a & 0xFFFFFFFF, a >> 32, b & 0xFFFFFFFF, b >> 32]
            ref[0] += 2 if ref[0] < 2 else 0
            ref[1] += 8 if ref[1] < 8 else 0
            ref[2] += 16 if ref[2] < 16 else 0
            assert st[r, i].tolist() == ref
    bad = st.copy()
    bad[0, 0, 1] = 3
    with pytest.raises(sop.SopError) as e:
        sim.set_rng_state(bad)
    assert e.value.status == sop.ERR_INVALID_ARG
    sim.close()
    phil = sop.from_workload(w, n_replicas=1, schedule="streamed")
    with pytest.raises(sop.SopError) as e:
        phil.get_rng_state()
    assert e.value.status == sop.ERR_UNSUPPORTED
    phil.close()


@pytest.mark.parametrize("schedule", ["batched", "streamed"])
def test_taus_checkpoint_resume_bit_exact(sop, synth, schedule):
    w = synth.replicas(n_replicas=3, n=100, steps=100)
    sim = sop.from_workload(w, schedule=schedule, rng="taus")
    sim.step(23)
    state = sim.get_state()
    sim.step(41)
    a, sa = sim.get_positions(-1).copy(), sim.get_rng_state().copy()
    sim.set_state(state)
    sim.step(41)
    assert np.array_equal(a, sim.get_positions(-1))
    assert np.array_equal(sa, sim.get_rng_state())
    sim.close()


@pytest.mark.parametrize("schedule", ["batched", "streamed"])
def test_taus_free_diffusion(sop, orc, schedule):
    """Single beads, no forces: <|dr|^2> = 6 (kT/zeta) t within 3 standard errors."""
    n = 4096
    rng = np.random.default_rng(9)
    xyz = rng.uniform(-1e4, 1e4, size=(n, 3))
    offs = np.arange(n + 1, dtype=np.int32)
    sim = sop.Simulation(xyz, offs, params={"pair_cut": 1.0}, n_replicas=1, seed=3, schedule=schedule,
                         rng="taus")
    x0 = sim.get_positions(0)
    steps = 200
    sim.step(steps)
    d2 = ((sim.get_positions(0) - x0) ** 2).sum(1)
    expect = 6 * orc.kB() * 300.0 / 50.0 * 0.1 * steps
    se = d2.std() / math.sqrt(n)
    assert abs(d2.mean() - expect) < 3 * se, (d2.mean(), expect, se)
    sim.close()
