"""Observable records of the CUDA path against closed forms (needs a GPU).

Every bead is fixed, so positions stay at their FP32 starting values and each
record has a value fixed by geometry (Sec. IV.B pulling protocol, Fig. 3
quantities): the spring force k_s v (n - n0) of a tip that started on the pulled
bead at step n0, the anchor-to-pulled distance, the end-to-end distance of each
system's first chain, the indenter's push 6 eps (sigma/g)^6 / g projected on its
motion and the distance it has travelled. The expected values are computed here
in FP64 from the positions read back through the ABI.
"""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

# record layout: step, replica, system, energy, f_ext, extension, q, r_ee
STEP, REP, SYS, E, F, EXT, Q, REE = range(8)
SCHEDULES = ["batched", "streamed", "pairs", "plain", "batched_pairs"]


@pytest.fixture(scope="module")
def sop():
    from paper_1003_1148_gb300 import build, sop as s
    build.build()
    s.load()
    return s


def straight(n, step=3.8, origin=(0.0, 0.0, 0.0), axis=0):
    x = np.zeros((n, 3))
    x[:, axis] = step * np.arange(n)
    return x + np.asarray(origin, np.float64)


def dist(a, b):
    d = np.asarray(a, np.float64) - np.asarray(b, np.float64)
    return math.sqrt((d[0] * d[0] + d[1] * d[1]) + d[2] * d[2])


@pytest.mark.parametrize("schedule", SCHEDULES)
def test_pull_records_follow_the_moving_tip(sop, schedule):
    # two systems: A = chains 0, 1 (7 and 5 beads), B = chain 2 (6 beads); A pulled from
    # bead 1 (anchor) by bead 5, B from bead 12 by bead 17, started at step 40
    x = np.concatenate([straight(7), straight(5, 3.8, (0, 60, 0), 1), straight(6, 3.8, (0, 0, 120))])
    n = len(x)
    fixed = np.ones(n, np.uint8)
    sim = sop.Simulation(x, [0, 7, 12, 18], [0, 2, 3], fixed, dict(T=300.0), n_replicas=2, seed=5,
                         obs_every=20, schedule=schedule)
    xs = sim.get_positions(0)
    sim.step(40)
    sim.get_observables()
    k_a, v_a, k_b, v_b = 0.05, 0.01, 0.2, 0.005
    sim.pull([(0, 1, 5, k_a, v_a), (1, 12, 17, k_b, v_b)])
    sim.step(160)
    rec, lost = sim.get_observables()
    assert lost == 0 and len(rec) == 8 * 2 * 2
    assert np.array_equal(sim.get_positions(1), xs)
    for r in rec:
        s, n_ = int(r[SYS]), r[STEP]
        k, v, a, b = (k_a, v_a, 1, 5) if s == 0 else (k_b, v_b, 12, 17)
        assert r[F] == pytest.approx(k * v * (n_ - 40), rel=1e-12)
        assert r[EXT] == dist(xs[b], xs[a])
        first, last = (0, 6) if s == 0 else (12, 17)   # each system's first chain
        assert r[REE] == dist(xs[last], xs[first])
        assert r[Q] == 0.0                               # straight chains hold no native contact
    sim.close()


@pytest.mark.parametrize("schedule", SCHEDULES)
def test_indenter_records_are_the_projected_wall_force(sop, schedule):
    # one-bead chains far apart (no bonds, no contacts): bead 0 straight ahead of the
    # indenter at gap sigma when the record is taken, bead 1 at 60 degrees, bead 2 behind
    R, sig, v, n1 = 50.0, 3.8, 0.005, 200
    c_rec = np.array([0.0, 0.0, -v * n1])            # centre at the record step
    th = math.pi / 3
    x = np.array([c_rec + [0.0, 0.0, -(R + sig)],
                  c_rec + (R + 2 * sig) * np.array([math.sin(th), 0.0, -math.cos(th)]),
                  c_rec + [0.0, 0.0, R + 3 * sig]])
    fixed = np.ones(3, np.uint8)
    sim = sop.Simulation(x, [0, 1, 2, 3], [0, 3], fixed, dict(T=300.0), n_replicas=1, seed=1,
                         obs_every=n1, schedule=schedule)
    xs = sim.get_positions(0)
    sim.indenter((0.0, 0.0, 0.0), (0.0, 0.0, -1.0), R, v)
    sim.step(n1)
    rec, _ = sim.get_observables()
    assert len(rec) == 1 and rec[0, STEP] == n1
    c = np.array([0.0, 0.0, -v * n1])
    want = 0.0
    for b in range(3):
        e = xs[b] - c
        r = math.sqrt((e[0] * e[0] + e[1] * e[1]) + e[2] * e[2])
        g = r - R
        want += 6.0 * (sig / g) ** 6 / g * (-e[2] / r)
    assert rec[0, F] == pytest.approx(want, rel=1e-9)
    assert rec[0, F] == pytest.approx(6.0 / sig * (1 + 0.5 / 2 ** 7) - 6.0 / sig / 3 ** 7, rel=3e-5)
    assert rec[0, EXT] == pytest.approx(v * n1, rel=1e-15)
    sim.close()


@pytest.mark.parametrize("schedule", SCHEDULES)
def test_q_has_its_own_cadence(sop, synth, schedule, monkeypatch):
    """obs_every (the force-extension cadence) 100 and obs_every_q 300: the records are those
    of the run with Q at every record, bit for bit, except that q is NaN where the step is not
    a multiple of 300 (Sec. IV.B samples f(R) and Q at different cadences). Both contexts take
    the untuned configuration, so that their FP64 sums group alike."""
    monkeypatch.setenv("SOP_TUNE", "0")
    w = synth.replicas(n_replicas=3, n=64, seed=7, steps=900)
    runs = []
    for q_every in (0, 300):
        sim = sop.from_workload(w, schedule=schedule, obs_every=100, obs_every_q=q_every)
        sim.step(900)
        rec, lost = sim.get_observables()
        sim.close()
        assert lost == 0 and len(rec) == 9 * 3
        runs.append(rec)
    a, b = runs
    on_q = b[:, 0] % 300 == 0
    assert np.array_equal(np.isnan(b[:, 6]), ~on_q)
    assert np.array_equal(a[on_q], b[on_q])
    cols = [0, 1, 2, 3, 4, 5, 7]
    assert np.array_equal(a[~on_q][:, cols], b[~on_q][:, cols])
    with pytest.raises(sop.SopError):
        sop.from_workload(w, schedule=schedule, obs_every=100, obs_every_q=250)
