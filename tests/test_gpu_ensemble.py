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


@pytest.fixture(scope="module")
def pull48(sop, orc):
    """A pulled 48-bead chain (N-terminus fixed, C-terminus on a spring moving at 0.02 A per
    step, Sec. IV.B): 256 GPU replicas and 48 independent oracle trajectories, records
    every 100 steps for 1,500 steps. Returns the GPU records and the oracle's, per replica."""
    from paper_1003_1148_gb300.synth import Pull, Workload, compact_chain, default_params
    n = 48
    xyz = compact_chain(n, 31)
    fixed = np.zeros(n, np.uint8)
    fixed[0] = 1
    w = Workload("pull48", xyz, np.array([0, n], np.int32), np.array([0, 1], np.int32), fixed, 1, 1500, 0,
                 default_params(), pulls=[Pull(0, n - 1, 0.05, 0.02)], obs_every=100)
    n_gpu, n_orc = 256, 128
    sim = sop.from_workload(w, n_replicas=n_gpu, schedule="batched", obs_capacity=n_gpu * 64)
    sim.step(w.steps)
    rec, lost = sim.get_observables()
    sim.close()
    assert lost == 0
    x0 = xyz.astype(np.float32).astype(np.float64)
    m = orc.model_from_workload(w)
    m.start_pulls([(0, 0, n - 1, 0.05, 0.02)], x0)
    o = [m.run(x0, w.steps, seed=200_000 + r, obs_every=100)[1] for r in range(n_orc)]
    return rec, o


def test_pulling_ensemble(pull48):
    """Force-extension of the pulled chain: mean force and extension over the run."""
    rec, o = pull48
    g = per_replica_means(rec[:, 1:], 256, [3, 4])
    z = z_scores(g, np.array([[obs[:, 3].mean(), obs[:, 4].mean()] for obs in o]))
    assert np.all(np.abs(z) < 2.0), dict(zip(["f_ext", "extension"], z.round(2)))


def test_force_extension_curve_per_checkpoint(pull48):
    """The force-extension curve itself: at every record (every 100 steps) the ensemble mean
    force and mean extension of the GPU replicas against those of the oracle trajectories,
    one independent sample per replica and checkpoint. Each difference is measured in
    combined standard errors; with k = 30 comparisons (15 records, two quantities) the bound
    is the Bonferroni one for a family-wise 5 % level, |z| < z(1 - 0.025 / k) = 3.14, and at
    least 90 % of the comparisons must also lie within 2 combined standard errors."""
    from statistics import NormalDist
    rec, o = pull48
    steps = np.unique(rec[:, 0])
    assert len(steps) == 15
    zs = {}
    for s in steps:
        g = rec[rec[:, 0] == s]
        g = g[np.argsort(g[:, 1])]
        assert len(g) == 256
        ob = np.array([obs[obs[:, 0] == s][0] for obs in o])
        zs[int(s)] = z_scores(g[:, [4, 5]], ob[:, [3, 4]])
    z = np.array(list(zs.values()))
    bound = NormalDist().inv_cdf(1.0 - 0.025 / z.size)
    assert np.abs(z).max() < bound, {k: v.round(2) for k, v in zs.items()}
    assert (np.abs(z) < 2.0).mean() >= 0.9, {k: v.round(2) for k, v in zs.items()}
    # the curve rises: the spring pulls harder as the chain is stretched
    f_mean = [rec[rec[:, 0] == s][:, 4].mean() for s in steps]
    r_mean = [rec[rec[:, 0] == s][:, 5].mean() for s in steps]
    assert r_mean[-1] > r_mean[0] and f_mean[-1] > f_mean[0]
