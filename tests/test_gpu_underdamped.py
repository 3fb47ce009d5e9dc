"""Underdamped Langevin dynamics (BAOAB) through the C ABI against the FP64 oracle
(needs a GPU).

* positions and velocities after 100 steps from the same Philox stream: RMS <= 1e-3 A
  (positions) and <= 1e-3 of the thermal speed sqrt(kT/m) (velocities), every schedule;
* checkpoint/resume bit-exact with velocities;
* a bead on the cantilever spring (tip speed 0) samples the exact harmonic variance
  kT / k_s at h w = 1 over 4,096 replicas (within 3 standard errors).
"""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

PARAMS = dict(dt=0.02, zeta=0.5)
MASS = 1.0


@pytest.fixture(scope="module")
def sop():
    from paper_1003_1148_gb300 import build, sop as s
    build.build()
    s.load()
    return s


@pytest.mark.parametrize("schedule", ["batched", "streamed", "pairs", "plain", "batched_pairs"])
def test_baoab_trajectory_matches_oracle(sop, orc, synth, schedule):
    w = synth.uneven(n_chains=5, lo=50, hi=240, steps=100)
    w.params = dict(w.params, **PARAMS)
    R = 2
    sim = sop.from_workload(w, n_replicas=R, schedule=schedule, integrator="baoab", mass=MASS)
    x0 = sim.get_positions(0)
    sim.step(100)
    vth = math.sqrt(orc.kB() * w.params["T"] / MASS)
    for r in range(R):
        m = orc.model_from_workload(w)
        sys_of = w.system_of_bead()
        m.start_pulls([(int(sys_of[p.anchor]), p.anchor, p.pulled, p.k_s, p.v) for p in w.pulls], x0)
        m.set_underdamped(MASS)
        xo, _, _, _ = m.run(x0, 100, seed=w.seed + r)
        rms = float(np.sqrt(((sim.get_positions(r) - xo) ** 2).sum(1).mean()))
        assert rms <= 1e-3, (schedule, r, rms)
        vrms = float(np.sqrt(((sim.get_velocities(r) - m.velocities()) ** 2).sum(1).mean()))
        assert vrms <= 1e-3 * vth, (schedule, r, vrms)
    sim.close()


@pytest.mark.parametrize("schedule", ["batched", "streamed"])
def test_baoab_checkpoint_resume_bit_exact(sop, synth, schedule):
    w = synth.replicas(n_replicas=3, n=100, steps=100)
    w.params = dict(w.params, **PARAMS)
    sim = sop.from_workload(w, schedule=schedule, integrator="baoab", mass=MASS)
    sim.step(23)
    state = sim.get_state()
    sim.step(41)
    a, va = sim.get_positions(-1).copy(), sim.get_velocities(-1).copy()
    sim.set_state(state)
    sim.step(41)
    assert np.array_equal(a, sim.get_positions(-1))
    assert np.array_equal(va, sim.get_velocities(-1))
    with pytest.raises(sop.SopError):
        sop.from_workload(w, schedule=schedule).get_velocities(0)
    sim.close()


@pytest.mark.parametrize("schedule", ["batched", "streamed"])
def test_baoab_harmonic_variance_on_gpu(sop, orc, schedule):
    k_s, mass, zeta, dt, T = 100.0, 1.0, 5.0, 0.1, 300.0    # h w = 1
    xyz = np.array([[0.0, 0.0, 0.0], [100.0, 0.0, 0.0]])
    R = 4096
    sim = sop.Simulation(xyz, [0, 1, 2], [0, 2], params=dict(zeta=zeta, dt=dt, T=T), n_replicas=R, seed=17,
                         schedule=schedule, integrator="baoab", mass=mass)
    sim.pull([(0, 0, 1, k_s, 0.0)])
    sim.step(200)
    samples = []
    for _ in range(10):
        sim.step(20)
        samples.append(sim.get_positions(-1)[:, 1] - xyz[1])
    s = np.array(samples).ravel()
    kT = orc.kB() * T
    se = kT / k_s * math.sqrt(2.0 / len(s))
    assert abs(s.var() - kT / k_s) < 3 * se, (s.var(), kT / k_s, se)
    assert np.array_equal(sim.get_positions(-1)[:, 0], np.zeros((R, 3)))
    sim.close()
