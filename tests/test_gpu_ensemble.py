"""Ensemble averages of the CUDA path against independent oracle trajectories
(needs a GPU). As in the paper's CPU/GPU comparison (Sec. IV.B), single
trajectories are not comparable over long times, their statistics are: the
time-averaged fraction of native contacts, end-to-end distance, energy and
pulling force must agree within 2 combined standard errors. GPU and oracle
replicas use disjoint Philox keys, so the two samples are independent.
"""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sop():
    from paper_1003_1148_gb300 import build, sop as s
    build.build()
    s.load()
    return s


def per_replica_means(rec, n_rep, cols):
    out = np.zeros((n_rep, len(cols)))
    for r in range(n_rep):
        sel = rec[rec[:, 0] == r]
        out[r] = [sel[:, c].mean() for c in cols]
    return out


def z_scores(a, b):
    ma, mb = a.mean(0), b.mean(0)
    se = np.sqrt(a.var(0, ddof=1) / len(a) + b.var(0, ddof=1) / len(b))
    return (ma - mb) / se


@pytest.mark.parametrize("schedule", ["batched", "streamed"])
def test_equilibrium_ensemble_chain64(sop, orc, synth, schedule):
    w = synth.chain64()
    steps, every = 2000, 100
    n_gpu, n_orc = 256, 48
    sim = sop.from_workload(w, n_replicas=n_gpu, schedule=schedule, obs_every=every, obs_capacity=n_gpu * 64)
    sim.step(steps)
    rec, lost = sim.get_observables()
    assert lost == 0
    # records: step, replica, system, energy, f_ext, extension, q, r_ee
    g = per_replica_means(rec[:, 1:], n_gpu, [2, 5, 6])
    m = orc.model_from_workload(w)
    o = []
    for r in range(n_orc):
        _, obs, _, _ = m.run(w.xyz, steps, seed=100_000 + r, obs_every=every)
        o.append([obs[:, 2].mean(), obs[:, 5].mean(), obs[:, 6].mean()])
    o = np.array(o)
    z = z_scores(g, o)
    assert np.all(np.abs(z) < 2.0), dict(zip(["energy", "q", "r_ee"], z.round(2)))


def test_pulling_ensemble(sop, orc, synth):
    """Force-extension of a pulled 48-bead chain: mean force and extension over the run."""
    from paper_1003_1148_gb300.synth import Pull, Workload, compact_chain, default_params
    n = 48
    xyz = compact_chain(n, 31)
    fixed = np.zeros(n, np.uint8)
    fixed[0] = 1
    w = Workload("pull48", xyz, np.array([0, n], np.int32), np.array([0, 1], np.int32), fixed, 1, 1500, 0,
                 default_params(), pulls=[Pull(0, n - 1, 0.05, 0.02)], obs_every=100)
    n_gpu, n_orc = 256, 48
    sim = sop.from_workload(w, n_replicas=n_gpu, schedule="batched", obs_capacity=n_gpu * 64)
    sim.step(w.steps)
    rec, _ = sim.get_observables()
    g = per_replica_means(rec[:, 1:], n_gpu, [3, 4])
    m = orc.model_from_workload(w)
    m.start_pulls([(0, 0, n - 1, 0.05, 0.02)], xyz.astype(np.float32).astype(np.float64))
    o = []
    for r in range(n_orc):
        _, obs, _, _ = m.run(xyz.astype(np.float32).astype(np.float64), w.steps, seed=200_000 + r, obs_every=100)
        o.append([obs[:, 3].mean(), obs[:, 4].mean()])
    z = z_scores(g, np.array(o))
    assert np.all(np.abs(z) < 2.0), dict(zip(["f_ext", "extension"], z.round(2)))
