"""Degenerate and extreme inputs through the C ABI (needs a GPU): zero temperature,
every bead fixed, a chain with no native contact, the largest system the batched
schedule takes (8,192 beads), and a ragged last block of 32 beads."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sop():
    from paper_1003_1148_gb300 import build, sop as s
    build.build()
    s.load()
    return s


@pytest.mark.parametrize("schedule", ["batched", "streamed", "batched_pairs"])
def test_zero_temperature_follows_the_oracle_and_descends(sop, orc, synth, schedule):
    w = synth.chain64()
    w.params = dict(w.params, T=0.0)
    sim = sop.from_workload(w, n_replicas=2, schedule=schedule)
    x0 = sim.get_positions(0)
    _, e0 = sim.forces(0)
    sim.step(200)
    m = orc.model_from_workload(w)
    xo, _, _, _ = m.run(x0, 200, seed=w.seed)
    for r in range(2):
        assert float(np.sqrt(((sim.get_positions(r) - xo) ** 2).sum(1).mean())) <= 1e-4
    # no noise: both replicas take the same path, and the energy goes down
    assert np.array_equal(sim.get_positions(0), sim.get_positions(1))
    _, e1 = sim.forces(0)
    assert e1 < e0
    sim.close()


@pytest.mark.parametrize("schedule", ["batched", "streamed", "plain", "batched_pairs"])
def test_all_beads_fixed(sop, synth, schedule):
    w = synth.chain64()
    sim = sop.Simulation(w.xyz, w.chain_offsets, None, np.ones(w.n_beads, np.uint8), w.params, n_replicas=2,
                         seed=5, obs_every=10, schedule=schedule)
    x0 = sim.get_positions(-1).copy()
    sim.step(50)
    assert np.array_equal(sim.get_positions(-1), x0)
    rec, lost = sim.get_observables()
    assert lost == 0 and len(rec) == 5 * 2 and np.all(rec[:, 6] == 1.0)   # Q stays 1
    sim.close()


@pytest.mark.parametrize("schedule", ["batched", "streamed", "batched_pairs"])
def test_chain_without_native_contacts(sop, orc, schedule):
    n = 40
    xyz = np.zeros((n, 3))
    xyz[:, 0] = 3.8 * np.arange(n)             # straight: |i - j| >= 3 is at least 11.4 A apart
    sim = sop.Simulation(xyz, [0, n], params={}, n_replicas=1, seed=2, obs_every=10, schedule=schedule)
    rp, col, r0 = sim.get_native_map()
    assert len(col) == 0
    sim.step(30)
    x = sim.get_positions(0)
    m = orc.Model(xyz, np.zeros(n, np.int32), np.zeros(n, np.int32))
    F, E = sim.forces(0)
    Fo, Ao, Eo = m.forces(x)
    assert (np.abs(F - Fo) / Ao).max() <= 1e-5
    rec, _ = sim.get_observables()
    assert np.all(rec[:, 6] == 0.0)             # Q of a system without native contacts is 0
    sim.close()


def test_largest_batched_system(sop, orc, synth):
    """The largest systems of the batched schedule against the oracle: 4,096 beads (the
    cluster form's limit) and 3,001 beads (one CTA, rows in global memory, a ragged last
    block of 32 beads); 4,097 beads are refused."""
    with pytest.raises(sop.SopError) as e:
        sop.from_workload(synth.fiber4096(n=4097, steps=20), schedule="batched")
    assert e.value.status == sop.ERR_UNSUPPORTED
    for n in (4096, 3001):
        w = synth.fiber4096(n=n, steps=20)
        sim = sop.from_workload(w, schedule="batched")
        x0 = sim.get_positions(0)
        m = orc.model_from_workload(w)
        sys_of = w.system_of_bead()
        m.start_pulls([(int(sys_of[p.anchor]), p.anchor, p.pulled, p.k_s, p.v) for p in w.pulls], x0)
        F, E = sim.forces(0)
        Fo, Ao, Eo = m.forces(x0)
        assert (np.abs(F - Fo) / Ao).max() <= 1e-5, n
        sim.step(20)
        xo, _, _, _ = m.run(x0, 20, seed=w.seed)
        assert float(np.sqrt(((sim.get_positions(0) - xo) ** 2).sum(1).mean())) <= 1e-3, n
        sim.close()
