"""The cluster form of the batched schedule (one system over a thread-block cluster,
partners read from the owner CTA's shared memory) through the C ABI (needs a GPU).

The tuning override SOP_FORCE_CLUSTER=sh makes every bucket with systems larger than
2^sh beads run in the cluster form with 2^sh beads per CTA, so small systems exercise
clusters of several CTAs (including CTAs that own no bead of a shorter system).
* with one lane per bead, the same arithmetic in the same order as the one-CTA form:
  positions bit-identical (SOP_CLUSTER_LANES=1); with 2 or 4 lanes per bead, oracle parity;
* parity with the FP64 oracle: Verlet lists bit-exact, forces within 1e-5 of the term
  scale, 100-step trajectories within 1e-3 A RMS, FP64 observables;
* checkpoint/resume bit-exact; a failing replica freezes alone (the failure decision is
  taken by every CTA of the cluster from the same values).
"""
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sop():
    from paper_1003_1148_gb300 import build, sop as s
    build.build()
    s.load()
    return s


def clustered(sop, w, sh, lanes=None, **kw):
    os.environ["SOP_FORCE_CLUSTER"] = str(sh)
    if lanes:
        os.environ["SOP_CLUSTER_LANES"] = str(lanes)
    try:
        sim = sop.from_workload(w, schedule="batched", **kw)
    finally:
        del os.environ["SOP_FORCE_CLUSTER"]
        os.environ.pop("SOP_CLUSTER_LANES", None)
    assert sim.stats()["cluster_buckets"] > 0
    return sim


def small_uneven(synth):
    return synth.uneven(n_chains=6, lo=90, hi=300, steps=100)


def test_cluster_equals_one_cta_form(sop, synth):
    w = small_uneven(synth)
    os.environ["SOP_TUNE"] = "0"          # the untuned default: one CTA per system, rows in shared memory
    try:
        a = sop.from_workload(w, n_replicas=2, schedule="batched")
    finally:
        del os.environ["SOP_TUNE"]
    b = clustered(sop, w, 5, lanes=1, n_replicas=2)   # one lane per bead: the one-CTA order
    assert a.stats()["cluster_buckets"] == 0
    a.step(57)
    b.step(57)
    assert np.array_equal(a.get_positions(-1), b.get_positions(-1))
    ra, ca = a.get_pairlist(1)
    rb, cb = b.get_pairlist(1)
    assert np.array_equal(ra, rb) and np.array_equal(ca, cb)


@pytest.mark.parametrize("sh,lanes", [(5, 1), (6, 1), (5, 4), (6, 2), (6, 4)])
def test_cluster_parity_with_oracle(sop, orc, synth, sh, lanes):
    w = small_uneven(synth)
    R = 2
    sim = clustered(sop, w, sh, lanes, n_replicas=R)
    x0 = sim.get_positions(0)
    m = orc.model_from_workload(w)
    sys_of = w.system_of_bead()
    m.start_pulls([(int(sys_of[p.anchor]), p.anchor, p.pulled, p.k_s, p.v) for p in w.pulls], x0)
    sim.step(30)
    sim.pairlist_rebuild()     # the dumped list is the one of the positions of the last rebuild
    for r in range(R):
        x = sim.get_positions(r)
        rp, col = sim.get_pairlist(r)
        pi, pj = m.pairlist(x)
        got = {(i, int(j)) for i in range(len(rp) - 1) for j in col[rp[i]:rp[i + 1]] if j > i}
        assert got == set(zip(pi.tolist(), pj.tolist()))
        F, E = sim.forces(r)
        Fo, Ao, Eo = m.forces(x, step=30)
        assert (np.abs(F - Fo) / Ao).max() <= 1e-5
        assert E == pytest.approx(Eo[0] + Eo[1] + Eo[2], rel=1e-9, abs=1e-9)
    sim.close()
    sim = clustered(sop, w, sh, lanes, n_replicas=R, obs_every=20)
    sim.step(100)
    for r in range(R):
        xo, _, _, _ = m.run(x0, 100, seed=w.seed + r)
        rms = float(np.sqrt(((sim.get_positions(r) - xo) ** 2).sum(1).mean()))
        assert rms <= 1e-3, (sh, r, rms)
    rec, lost = sim.get_observables()
    assert lost == 0 and len(rec) == 5 * R * w.n_systems
    last = rec[rec[:, 0] == 100]
    for r in range(R):
        x = sim.get_positions(r)
        ref = m.observables(x, pl=m.pairlist(x), step=100)
        got = last[last[:, 1] == r]
        got = got[np.argsort(got[:, 2])]
        assert np.allclose(got[:, 3], ref[:, 2], rtol=1e-9, atol=1e-9)
        assert np.array_equal(got[:, 6], ref[:, 5])
    sim.close()


@pytest.mark.parametrize("lanes", [1, 4])
def test_cluster_checkpoint_and_failure(sop, synth, lanes):
    w = small_uneven(synth)
    sim = clustered(sop, w, 5, lanes, n_replicas=3)
    sim.step(23)
    state = sim.get_state()
    sim.step(41)
    a = sim.get_positions(-1).copy()
    sim.set_state(state)
    sim.step(41)
    assert np.array_equal(a, sim.get_positions(-1))
    # stretch one bond of replica 1 beyond R0: that replica fails and freezes alone
    x = sim.get_positions(1)
    i = int(w.chain_offsets[2]) + 40
    x[i + 1:int(w.chain_offsets[3])] += np.array([5.0, 0.0, 0.0])
    sim.set_positions(x, replica=1)
    frozen = sim.get_positions(1).copy()
    rc = sim.step(30, raise_on_error=False)
    st = sim.replica_status()
    assert st[1] == sop.ERR_FENE_BREAK and st[0] == 0 and st[2] == 0
    after = sim.get_positions(1)
    moved = np.abs(after - frozen).max(axis=1) > 0
    assert moved.sum() < w.n_beads          # the failed replica stopped within its first step
    sim.step(10, raise_on_error=False)
    assert np.array_equal(sim.get_positions(1), after)
    sim.close()


def test_cluster_with_taus_and_underdamped(sop, orc, synth):
    """The cluster form draws Hybrid Taus noise and takes BAOAB steps like the other forms."""
    w = small_uneven(synth)
    R = 2
    rng = np.random.default_rng(8)
    st0 = rng.integers(0, 2 ** 32, size=(R, w.n_beads, 4), dtype=np.uint64).astype(np.uint32)
    st0[..., 0] |= 2
    st0[..., 1] |= 8
    st0[..., 2] |= 16
    sim = clustered(sop, w, 5, n_replicas=R, rng="taus")
    sim.set_rng_state(st0)
    x0 = sim.get_positions(0)
    sim.step(60)
    st1 = sim.get_rng_state()
    sys_of = w.system_of_bead()
    for r in range(R):
        m = orc.model_from_workload(w)
        m.start_pulls([(int(sys_of[p.anchor]), p.anchor, p.pulled, p.k_s, p.v) for p in w.pulls], x0)
        m.set_taus_state(st0[r])
        xo, _, _, _ = m.run(x0, 60, seed=0)
        assert np.array_equal(st1[r], m.taus_state())
        assert float(np.sqrt(((sim.get_positions(r) - xo) ** 2).sum(1).mean())) <= 1e-3
    sim.close()
    w.params = dict(w.params, dt=0.02, zeta=0.5)
    sim = clustered(sop, w, 5, n_replicas=R, integrator="baoab", mass=1.0)
    sim.step(60)
    for r in range(R):
        m = orc.model_from_workload(w)
        m.start_pulls([(int(sys_of[p.anchor]), p.anchor, p.pulled, p.k_s, p.v) for p in w.pulls], x0)
        m.set_underdamped(1.0)
        xo, _, _, _ = m.run(x0, 60, seed=w.seed + r)
        assert float(np.sqrt(((sim.get_positions(r) - xo) ** 2).sum(1).mean())) <= 1e-3
        vth = np.sqrt(orc.kB() * w.params["T"] / 1.0)
        assert float(np.sqrt(((sim.get_velocities(r) - m.velocities()) ** 2).sum(1).mean())) <= 1e-3 * vth
    sim.close()
