"""Full-size workloads against the FP64 oracle on sampled outputs (needs a GPU).

The benchmark's own configuration (8,192 replicas of a 128-bead chain on the
batched kernel, tuned as bench.py runs it) and the other workloads at their
stated sizes: the 4,096-bead pulled fiber, the 2,048-chain uneven batch and the
150,000-bead shell with its indenter. Sampled replicas or chains are rerun by
the oracle from the same start with the same Philox stream; forces are checked
at identical positions. Bars as in test_gpu_parity.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

FORCE_TOL = 1e-5
RMS_TOL = 1e-3


@pytest.fixture(scope="module")
def sop():
    from paper_1003_1148_gb300 import build, sop as s
    build.build()
    s.load()
    return s


def rms(a, b):
    return float(np.sqrt(((a - b) ** 2).sum(1).mean()))


def test_bench_configuration_replicas8192x128(sop, orc, synth):
    w = synth.replicas(n_replicas=8192, n=128, seed=3)
    sim = sop.from_workload(w, schedule="batched", obs_capacity=4 * 8192)
    x0 = sim.get_positions(0)
    m = orc.model_from_workload(w)
    sim.step(100)
    rng = np.random.default_rng(7)
    sample = sorted(set([0, 1, 8191] + rng.integers(0, 8192, size=5).tolist()))
    allx = sim.get_positions(-1)
    for r in sample:
        xo, _, _, _ = m.run(x0, 100, seed=w.seed + r)
        assert rms(allx[r], xo) <= RMS_TOL, r
    for r in sample[:3]:
        F, E = sim.forces(r)
        Fo, Ao, Eo = m.forces(allx[r], step=100)
        assert (np.abs(F - Fo) / Ao).max() <= FORCE_TOL
        assert E == pytest.approx(Eo[:3].sum(), rel=1e-9)
    # every replica moved and none failed
    assert np.all(sim.replica_status() == 0)
    assert np.all(np.isfinite(allx))
    # the Verlet list of a sampled replica is the definition's set
    sim.pairlist_rebuild()
    rp, col = sim.get_pairlist(8191)
    x = sim.get_positions(8191)
    pi, pj = m.pairlist(x)
    got = {(i, int(j)) for i in range(128) for j in col[rp[i]:rp[i + 1]] if j > i}
    assert got == set(zip(pi.tolist(), pj.tolist()))


def test_fiber4096_pulled(sop, orc, synth):
    w = synth.fiber4096()
    sim = sop.from_workload(w, schedule="auto")
    assert sim.stats()["schedule"] in (sop.SCHED_STREAMED, sop.SCHED_PAIRS)
    x0 = sim.get_positions(0)
    m = orc.model_from_workload(w)
    m.start_pulls([(0, p.anchor, p.pulled, p.k_s, p.v) for p in w.pulls], x0)
    m.set_cells(True)
    sim.step(100)
    xo, obs, _, _ = m.run(x0, 100, seed=w.seed, obs_every=100)
    xg = sim.get_positions(0)
    assert rms(xg, xo) <= RMS_TOL
    rec, _ = sim.get_observables()
    assert rec.shape[0] == 1 and rec[0, 0] == 100
    # the pulling force readout follows the oracle's within the trajectory tolerance
    assert abs(rec[0, 4] - obs[0, 3]) <= 1e-3   # k_s times the position tolerance
    F, E = sim.forces(0)
    Fo, Ao, Eo = m.forces(xg, pl=m.pairlist(xg), step=100)
    assert (np.abs(F - Fo) / Ao).max() <= FORCE_TOL


def test_uneven2048_sampled_chains(sop, orc, synth):
    w = synth.uneven()
    sim = sop.from_workload(w, schedule="auto")
    xall0 = sim.get_positions(0)
    sim.step(100)
    xall = sim.get_positions(0)
    sizes = np.diff(w.chain_offsets)
    rng = np.random.default_rng(11)
    picks = [int(np.argmin(sizes)), int(np.argmax(sizes))] + rng.integers(0, w.n_chains, size=4).tolist()
    for c in picks:
        lo, hi = int(w.chain_offsets[c]), int(w.chain_offsets[c + 1])
        n = hi - lo
        m = orc.Model(w.xyz[lo:hi], np.zeros(n, np.int32), np.zeros(n, np.int32), w.fixed[lo:hi], w.params)
        m.set_noise_offset(lo)
        x0 = xall0[lo:hi]
        m.start_pulls([(0, 0, n - 1, w.pulls[c].k_s, w.pulls[c].v)], x0)
        xo, _, _, _ = m.run(x0, 100, seed=w.seed)
        assert rms(xall[lo:hi], xo) <= RMS_TOL, (c, n)


def test_shell150k_indenter(sop, orc, synth):
    w = synth.shell()
    sim = sop.from_workload(w, schedule="auto")
    x0 = sim.get_positions(0)
    m = orc.model_from_workload(w)
    ind = w.indenter
    m.set_indenter(ind.center, ind.direction, ind.radius, ind.v)
    m.set_cells(True)
    rp, col, r0 = sim.get_native_map()
    assert len(col) == 2 * len(m.nat_i)
    F, E = sim.forces(0)
    Fo, Ao, Eo = m.forces(x0, pl=m.pairlist(x0), step=0)
    assert (np.abs(F - Fo) / Ao).max() <= FORCE_TOL
    assert E == pytest.approx(Eo[:3].sum(), rel=1e-9)
    sim.step(20)
    xo, _, _, _ = m.run(x0, 20, seed=w.seed)
    assert rms(sim.get_positions(0), xo) <= RMS_TOL
    # substrate beads never move
    fixed = w.fixed.astype(bool)
    assert np.array_equal(sim.get_positions(0)[fixed], x0[fixed])
