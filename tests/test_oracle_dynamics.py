"""Pins of the oracle's integrator and step sequence (Algorithm 7, Sec. IV.C).

The first-order update is checked against the exactly solvable Brownian
particle in a harmonic well under a force ramp (Eqs. 3 and 4), the free
diffusion law <dr^2> = 6 (kT/zeta) t, the centre-of-mass diffusion of a chain
(internal forces cancel: 6 kT t / (N zeta)), and the stationary variance of
the discrete Ornstein-Uhlenbeck recursion.
"""
import json
import math
import os

import numpy as np
import pytest

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


def free_beads(orc, n, T=300.0, zeta=50.0, dt=0.1):
    """n beads far apart, each its own chain and system: no bonds, no contacts."""
    x = np.zeros((n, 3))
    x[:, 0] = 1000.0 * np.arange(n)
    p = dict(T=T, zeta=zeta, dt=dt)
    m = orc.Model(x, np.arange(n, dtype=np.int32), np.arange(n, dtype=np.int32), params=p)
    assert len(m.bond_i) == 0 and len(m.nat_i) == 0
    return m, x


def ramp_model_units():
    """Sec. IV.C parameters in A, kcal/mol, ps: K_sp, r_f, xi (from D = kT/xi)."""
    g = GOLD["sec_IV_C_brownian_particle"]
    N_per_kcalmolA = 4184.0 / 6.02214076e23 / 1e-10            # 1 kcal/mol/A in N
    K = g["K_sp_pN_per_nm"] * 1e-12 / 1e-9 / (N_per_kcalmolA / 1e-10)   # kcal/mol/A^2
    rf = g["r_f_pN_per_ns"] * 1e-12 / 1e3 / N_per_kcalmolA             # kcal/mol/A per ps
    D = g["D_cm2_per_s"] * 1e16 / 1e12                                  # A^2/ps
    return K, rf, D


def test_paper_ramp_rate_is_kappa_times_speed():
    g = GOLD["sec_IV_C_brownian_particle"]
    # r_f = kappa * nu0: 10 pN/nm * 1 um/s = 1e4 pN/s = 1e-5 pN/ns
    assert g["kappa_pN_per_nm"] * g["nu0_um_per_s"] * 1e3 * 1e-9 == pytest.approx(g["r_f_pN_per_ns"])


@pytest.mark.parametrize("h_factor", [1.0, 0.5])
def test_harmonic_ramp_deterministic_matches_eq4_and_eq3(orc, h_factor):
    """T = 0: the update is exactly the recursion of Eq. 4 and converges to Eq. 3 at first order."""
    K, rf, D = ramp_model_units()
    kT = orc.kB() * 300.0
    xi = kT / D
    tau = xi / K
    # the paper's h (50 ps) leaves h/tau ~ 1e-6; to see first-order convergence in a
    # short test, the same recursion is driven with h = tau/50 (and tau/100).
    h = tau / 50.0 * h_factor
    m, x = free_beads(orc, 1, T=0.0, zeta=xi, dt=h)
    x[:] = 0.0
    n_steps = int(round(5 * tau / h))
    X_rec = 0.0
    worst_rec = 0.0
    for n in range(n_steps):
        t = n * h
        F = np.array([[rf * t - K * x[0, 0], 0.0, 0.0]])
        x = m.ermak_update(x, F, seed=1, step=n)
        X_rec = X_rec + (rf * t / xi - X_rec / tau) * h          # Eq. 4
        worst_rec = max(worst_rec, abs(x[0, 0] - X_rec) / abs(X_rec) if X_rec else 0.0)
    assert worst_rec < 1e-12
    t = n_steps * h
    X_th = 0.0 * math.exp(-t / tau) + rf * tau / xi * (t - tau * (1 - math.exp(-t / tau)))   # Eq. 3
    rel = abs(x[0, 0] - X_th) / X_th
    # first-order scheme: the error is O(h/tau); record it for the convergence check
    test_harmonic_ramp_deterministic_matches_eq4_and_eq3.errs[h_factor] = rel
    assert rel < 2.0 * h / tau
    if len(test_harmonic_ramp_deterministic_matches_eq4_and_eq3.errs) == 2:
        e = test_harmonic_ramp_deterministic_matches_eq4_and_eq3.errs
        assert e[1.0] / e[0.5] == pytest.approx(2.0, rel=0.1)   # halving h halves the error


test_harmonic_ramp_deterministic_matches_eq4_and_eq3.errs = {}


def test_harmonic_noise_stationary_variance(orc):
    """T > 0, no ramp: X_{n+1} = (1 - h/tau) X_n + b g, stationary Var = (kT/K) / (1 - h/(2 tau))."""
    R = 4000
    K = 0.5
    zeta = 50.0
    dt = 1.0
    m, x = free_beads(orc, R, T=300.0, zeta=zeta, dt=dt)
    x0 = x.copy()
    tau = zeta / K
    for n in range(int(8 * tau)):
        F = -K * (x - x0)
        x = m.ermak_update(x, F, seed=99, step=n)
    d = (x - x0).ravel()
    kT = orc.kB() * 300.0
    var_th = kT / K / (1.0 - dt / (2 * tau))
    se = var_th * math.sqrt(2.0 / d.size)
    assert abs(d.var() - var_th) < 5 * se
    assert abs(d.mean()) < 5 * math.sqrt(var_th / d.size)


def test_free_diffusion_msd(orc):
    R, steps = 3000, 50
    m, x0 = free_beads(orc, R)
    x, obs, rc, _ = m.run(x0, steps, seed=5)
    msd = ((x - x0) ** 2).sum(1)
    kT = orc.kB() * 300.0
    th = 6.0 * kT / 50.0 * steps * 0.1
    se = msd.std() / math.sqrt(R)
    assert abs(msd.mean() - th) < 5 * se


def test_chain_centre_of_mass_diffusion(orc, synth):
    """Internal forces sum to zero, so the centre of mass of a free chain
    diffuses with D = kT / (N zeta) whatever the conformation."""
    n, steps, reps = 16, 100, 400
    xn = synth.compact_chain(n, 21)
    m = orc.Model(xn, np.zeros(n, np.int32), np.zeros(n, np.int32))
    d2 = []
    for r in range(reps):
        x, _, _, _ = m.run(xn, steps, seed=1000 + r)
        d2.append(((x.mean(0) - xn.mean(0)) ** 2).sum())
    d2 = np.array(d2)
    kT = orc.kB() * 300.0
    th = 6.0 * kT / (n * 50.0) * steps * 0.1
    assert abs(d2.mean() - th) < 5 * d2.std() / math.sqrt(reps)


def test_run_equals_explicit_loop(orc, synth):
    """orc_run is the step sequence: rebuild at n % K == 0, forces, update."""
    n = 48
    xn = synth.compact_chain(n, 4)
    m = orc.Model(xn, np.zeros(n, np.int32), np.zeros(n, np.int32))
    xr, obs, rc, _ = m.run(xn, 35, seed=7, obs_every=10)
    x = xn.copy()
    for step in range(35):
        if step % 10 == 0:
            pl = m.pairlist(x)
        F, _, _ = m.forces(x, pl=pl, step=step)
        x = m.ermak_update(x, F, seed=7, step=step)
        if (step + 1) % 10 == 0:
            rec = obs[(step + 1) // 10 - 1]
            pl_obs = m.pairlist(x) if (step + 1) % 10 == 0 else pl
            assert np.array_equal(rec, m.observables(x, pl=pl_obs, step=step + 1)[0])
    assert np.array_equal(x, xr)
    assert obs.shape == (3, 8) and list(obs[:, 0]) == [10, 20, 30]


def test_pulling_holds_anchor_and_stretches(orc, synth):
    n = 40
    xn = synth.compact_chain(n, 8)
    fixed = np.zeros(n, np.uint8)
    fixed[0] = 1
    m = orc.Model(xn, np.zeros(n, np.int32), np.zeros(n, np.int32), fixed=fixed)
    m.start_pulls([(0, 0, n - 1, 0.05, 0.05)], xn)
    x, obs, rc, _ = m.run(xn, 2000, seed=3, obs_every=100)
    assert np.array_equal(x[0], xn[0])
    ext, f = obs[:, 4], obs[:, 3]
    # overdamped: the pulled bead moves 0.002 A per step per kcal/mol/A, so it
    # lags the tip (0.05 A/step) and the spring force builds up with time
    assert ext[-1] > ext[0] + 2.0
    assert f[-1] > f[0] > 0.0


def test_fene_break_is_reported(orc):
    x = np.array([[0.0, 0, 0], [3.8, 0, 0]])
    m = orc.Model(x, [0, 0], [0, 0])
    far = np.array([[0.0, 0, 0], [3.8 + 2.5, 0, 0]])
    xr, obs, rc, fail = m.run(far, 5, seed=1, raise_on_error=False)
    assert rc == 3 and fail == 0


# ---------------------------------------------------------------------------------------
# Sec. IV.C experiment functions (orc_ramp_*): the mean recursion against the closed
# form of a linear recursion (exact rationals), the order of Eqs. 4 and 5 against Eq. 3,
# and the stochastic run's noise stream and moments.
# ---------------------------------------------------------------------------------------
def _recursion_closed_form(K, xi, h, r_f, X0, order, n):
    """X_n of X_{k+1} = a X_k + b k + c (t_k = k h) in exact rationals:
    X_n = a^n X0 + b (a^n - n a + n - 1) / (1 - a)^2 + c (1 - a^n) / (1 - a)."""
    from fractions import Fraction as Fr
    K, xi, h, r_f, X0 = (Fr(v) for v in (K, xi, h, r_f, X0))
    tau = xi / K
    a = 1 - h / tau
    b = r_f * h * h / xi
    c = Fr(0)
    if order >= 2:
        a += h * h / (2 * tau * tau)
        b *= 1 - h / (2 * tau)
    if order == 3:
        c = r_f * h * h / (2 * xi)
    an = a ** n
    return float(an * X0 + b * (an - n * a + n - 1) / (1 - a) ** 2 + c * (1 - an) / (1 - a))


@pytest.mark.parametrize("order", [1, 2, 3])
def test_ramp_mean_recursion_closed_form(orc, order):
    K, xi, h, r_f, X0 = 0.5, 8.0, 0.25, 0.125, 1.5       # binary fractions: exact inputs
    r = orc.Ramp(K, xi, 0.0, h, r_f, X0, order)
    for n in (1, 2, 3, 50, 400):
        ref = _recursion_closed_form(K, xi, h, r_f, X0, order, n)
        assert r.mean(n) == pytest.approx(ref, rel=1e-12, abs=1e-14), (order, n)


@pytest.mark.parametrize("order,ratio", [(1, 2.0), (2, 2.0), (3, 4.0)])
def test_ramp_scheme_order_against_eq3(orc, order, ratio):
    """Halving h divides the error against Eq. 3 by 2 for Eq. 4 and for Eq. 5 as printed
    (its h^2 term lacks the ramp's r_f h^2 / (2 xi), so it stays first order), and by 4 for
    the complete second-order Taylor step."""
    K, xi, r_f, X0, t = 1.0, 10.0, 0.3, 2.0, 25.0
    errs = []
    for h in (0.05, 0.025, 0.0125):
        r = orc.Ramp(K, xi, 0.0, h, r_f, X0, order)
        errs.append(abs(r.mean(int(round(t / h))) - r.theory(t)))
    for e0, e1 in zip(errs, errs[1:]):
        assert e0 / e1 == pytest.approx(ratio, rel=0.05), (order, errs)


def test_ramp_run_noise_stream_and_moments(orc):
    # noise-free run = the mean recursion
    r0 = orc.Ramp(1.0, 10.0, 0.0, 0.1, 0.3, 0.5, 1)
    assert r0.run(7, 3, 333) == r0.mean(333)
    # one step from X0 = 0 at t = 0 is the first normal of block 0 of this run's stream
    r = orc.Ramp(1.0, 10.0, 0.6, 0.1, 0.3, 0.0, 1)
    amp = math.sqrt(2 * 0.6 * 0.1 / 10.0)
    for run in (0, 5):
        x = orc.philox([0, 0, run, 1], [11, 0])
        g = orc.box_muller4(x)
        assert r.run(11, run, 1) == pytest.approx(amp * g[0], rel=1e-15)
        g3 = orc.box_muller(x)
        assert np.allclose(g[:3], g3, rtol=0, atol=0)
        u3 = (float(x[2]) + 1.0) / 2 ** 32
        assert g[2] ** 2 + g[3] ** 2 == pytest.approx(-2 * math.log(u3), rel=1e-12)
    # ensemble: mean = recursion, variance = sigma^2 (1 - a^(2n)) / (1 - a^2)
    n, runs = 120, 3000
    xs = np.array([r.run(11, k, n) for k in range(runs)])
    a = 1 - 0.1 / 10.0
    var = amp ** 2 * (1 - a ** (2 * n)) / (1 - a * a)
    assert abs(xs.mean() - r.mean(n)) < 4 * math.sqrt(var / runs)
    assert xs.var(ddof=1) == pytest.approx(var, rel=4 * math.sqrt(2 / (runs - 1)))


# ---------------------------------------------------------------------------------------
# Underdamped BAOAB (orc_baoab_update): a bead on the cantilever spring (tip speed 0) is a
# 3-D harmonic oscillator. Without friction and noise the scheme is velocity Verlet, whose
# orbit has the closed form x_n = A cos(n theta) + B sin(n theta), cos theta = 1 - (h w)^2/2;
# with friction and noise BAOAB samples the exact configurational variance kT / k_s of a
# harmonic oscillator at any stable h (tested at h w = 1, where a scheme with the A and O
# sub-steps swapped would be a third off).
# ---------------------------------------------------------------------------------------
def _oscillator(orc, k_s, mass, zeta, T, dt, disp):
    xyz = np.array([[0.0, 0.0, 0.0], [100.0, 0.0, 0.0]])
    m = orc.Model(xyz, np.array([0, 1], np.int32), np.array([0, 0], np.int32),
                  params=dict(zeta=zeta, T=T, dt=dt))
    m.start_pulls([(0, 0, 1, k_s, 0.0)], xyz)
    m.set_underdamped(mass)
    x0 = xyz.copy()
    x0[1] += disp
    return m, x0


def test_baoab_without_friction_is_velocity_verlet(orc):
    k_s, mass, dt = 9.0, 1.0, 0.1                 # h w = 0.3
    disp = np.array([0.5, -0.2, 0.1])
    m, x = _oscillator(orc, k_s, mass, 0.0, 0.0, dt, disp)
    hw2 = dt * dt * k_s / mass
    theta = math.acos(1 - hw2 / 2)
    A = disp
    B = (disp * (1 - hw2) - disp * math.cos(theta)) / math.sin(theta)
    for block in range(30):
        x, _, _, _ = m.run(x, 10, seed=1, step0=10 * block)
        n = 10 * (block + 1)
        ref = A * math.cos(n * theta) + B * math.sin(n * theta)
        assert np.allclose(x[1] - np.array([100.0, 0, 0]), ref, rtol=0, atol=1e-11), n
    assert np.array_equal(x[0], [0.0, 0.0, 0.0])      # the anchor never moves


def test_baoab_harmonic_configurational_variance_is_exact(orc):
    k_s, mass, zeta, dt, T = 100.0, 1.0, 5.0, 0.1, 300.0   # h w = 1
    kT = orc.kB() * T
    samples = []
    for seed in range(48):
        m, x = _oscillator(orc, k_s, mass, zeta, T, dt, np.zeros(3))
        for block in range(400):
            x, _, _, _ = m.run(x, 10, seed=seed, step0=10 * block)
            if block >= 40:
                samples.append(x[1] - np.array([100.0, 0.0, 0.0]))
    s = np.array(samples).ravel()
    var = s.var()
    # about 1e5 nearly independent samples (relaxation within a few steps)
    assert var == pytest.approx(kT / k_s, rel=0.03)
    assert abs(s.mean()) < 5 * math.sqrt(kT / k_s / len(s) * 10)
