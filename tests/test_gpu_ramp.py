"""The Sec. IV.C experiment (Brownian particle under a ramp force) on the GPU against the
FP64 oracle, through the C ABI (needs a GPU).

* Every run's X after a ragged number of steps (not a multiple of the 4-step noise block,
  several launches) equals the oracle's run with the same Philox stream within
  1e-5 of the spread of X (FP32 arithmetic with a compensated position).
* The checkpoint means and variances equal the FP64 reductions of the oracle's runs.
* Noise-free, one run follows the FP64 mean recursion (Eq. 4, Eq. 5 as printed, the
  complete second-order step) within 1e-5 relative over 10^6 steps.
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


@pytest.mark.parametrize("order", [1, 2, 3])
def test_ramp_runs_match_oracle(sop, orc, order):
    K, xi, kT, h, r_f, X0 = 1.0, 10.0, 0.6, 0.1, 0.3, 0.5
    runs, steps, seed = 300, 1003, 77
    mean, var, xf = sop.brownian_ramp(K, xi, kT, h, r_f, runs, steps, X0=X0, order=order, n_out=3, seed=seed,
                                      x_final=True)
    r = orc.Ramp(K, xi, kT, h, r_f, X0, order)
    ref = np.array([r.run(seed, k, steps) for k in range(runs)])
    spread = ref.std()
    assert np.abs(xf - ref).max() <= 1e-5 * spread
    for k in range(3):
        n = steps * (k + 1) // 3
        xs = np.array([r.run(seed, j, n) for j in range(runs)])
        assert mean[k] == pytest.approx(xs.mean(), abs=1e-5 * spread)
        assert var[k] == pytest.approx(xs.var(), rel=1e-4)


@pytest.mark.parametrize("order", [1, 2, 3])
def test_ramp_noise_free_follows_recursion(sop, orc, order):
    # the paper's particle in pN, nm, ps: K = 40 pN/nm, D = kT/xi = 1.5e-9 nm^2/ps,
    # r_f = 1e-8 pN/ps, h = 50 ps; 10^6 steps (t = 0.72 tau)
    kT = 4.14
    K, xi, h, r_f = 40.0, kT / 1.5e-9, 50.0, 1e-8
    steps = 1_000_000
    mean, var = sop.brownian_ramp(K, xi, 0.0, h, r_f, 1, steps, order=order, n_out=4)
    r = orc.Ramp(K, xi, 0.0, h, r_f, 0.0, order)
    for k in range(4):
        ref = r.mean(steps * (k + 1) // 4)
        assert mean[k] == pytest.approx(ref, rel=1e-5), (order, k)
        assert var[k] == 0.0


def test_ramp_rejects_bad_parameters(sop):
    with pytest.raises(sop.SopError) as e:
        sop.brownian_ramp(-1.0, 1.0, 0.0, 0.1, 0.0, 10, 10)
    assert e.value.status == sop.ERR_INVALID_ARG
    with pytest.raises(sop.SopError):
        sop.brownian_ramp(1.0, 1.0, 0.0, 0.1, 0.0, 10, 10, order=4)
    with pytest.raises(sop.SopError):
        sop.brownian_ramp(1.0, 1.0, 0.0, 0.1, 0.0, 10, 10, n_out=11)
