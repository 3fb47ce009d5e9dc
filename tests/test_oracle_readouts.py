"""Pins of the oracle's readouts (Sec. IV.B pulling protocol, Fig. 3 quantities).

Every record of ``orc_observables`` is checked here against a value fixed by
geometry alone, on configurations built so that a plausible mistake changes the
number: a force not projected on the pulling direction, an extension measured
from the wrong bead or along the wrong axis, an end-to-end distance taken over the
whole system instead of its first chain, a tip position that ignores the step at
which pulling started, a wall readout with the wrong sign or projection, a native
contact counted on the wrong side of its r0 + 2 A threshold. None of the checks
re-types the oracle's expressions.
"""
import math

import numpy as np
import pytest

P = dict(k_fene=14.0, R0=2.0, eps_h=1.0, native_cut=8.0, eps_l=1.0, sigma=3.8, T=300.0, zeta=50.0, dt=0.1,
         pair_cut=10.0, rebuild_every=10)
NO_LIST = (np.zeros(0, np.int32), np.zeros(0, np.int32))
# record layout: step, system, energy, f_ext, extension, Q, R_ee, 0
STEP, SYS, E, F, EXT, Q, REE = range(7)


def straight(n, step=3.8, origin=(0.0, 0.0, 0.0), axis=0):
    x = np.zeros((n, 3))
    x[:, axis] = step * np.arange(n)
    return x + np.asarray(origin, np.float64)


def test_end_to_end_of_a_straight_chain(orc):
    for n in (2, 7, 64):
        x = straight(n)
        m = orc.Model(x, np.zeros(n, np.int32), np.zeros(n, np.int32), params=P)
        rec = m.observables(x, pl=NO_LIST)[0]
        assert rec[REE] == 3.8 * (n - 1)


def test_end_to_end_uses_the_first_chain_of_each_system(orc):
    # system 0: chains 0 (5 beads along x) and 1 (4 beads along y, far away);
    # system 1: chains 2 (3 beads along z) and 3 (6 beads along x).
    parts = [straight(5), straight(4, 2.0, (0, 100, 0), 1), straight(3, 3.0, (0, 0, 200), 2),
             straight(6, 3.8, (300, 0, 0))]
    x = np.concatenate(parts)
    chain = np.concatenate([np.full(len(p), c, np.int32) for c, p in enumerate(parts)])
    sys = np.concatenate([np.zeros(9, np.int32), np.ones(9, np.int32)])
    m = orc.Model(x, chain, sys, params=P)
    rec = m.observables(x, pl=NO_LIST)
    assert rec[0, REE] == 4 * 3.8          # not |r_8 - r_0| (the system's last bead)
    assert rec[1, REE] == 2 * 3.0          # system 1's first chain is chain 2
    assert rec[0, SYS] == 0 and rec[1, SYS] == 1


def pulled_chain(orc, n=5, anchor=1, pulled=3, fixed=None):
    # one chain per bead (no bonds, so any displacement is a valid configuration), one system
    x = straight(n)
    m = orc.Model(x, np.arange(n, dtype=np.int32), np.zeros(n, np.int32), fixed=fixed, params=P)
    return m, x


def test_pull_force_is_the_spring_along_the_pulling_direction(orc):
    k_s = 0.05
    m, x = pulled_chain(orc)
    m.start_pulls([(0, 1, 3, k_s, 0.0)], x)    # direction +x (anchor 1 -> pulled 3), tip at r_3
    for par, perp in ((0.0, 0.0), (-0.75, 0.0), (-0.75, 2.5), (1.25, -4.0), (0.0, 3.0)):
        y = x.copy()
        y[3] += np.array([par, perp, 0.5 * perp])   # the bead is displaced from the tip
        rec = m.observables(y, pl=NO_LIST)[0]
        # spring force k_s (tip - r) projected on d = +x: only the parallel part counts
        assert rec[F] == pytest.approx(-k_s * par, abs=1e-15)


def test_pull_direction_is_fixed_at_the_start(orc):
    # pulling along a diagonal: d = (3, 4, 0) / 5 from the anchor at the start
    k_s = 0.2
    x = np.array([[0.0, 0.0, 0.0], [3.0, 4.0, 0.0], [3.0, 4.0, 3.8]])
    m = orc.Model(x, np.array([0, 1, 2], np.int32), np.zeros(3, np.int32), params=P)
    m.start_pulls([(0, 0, 1, k_s, 0.0)], x)
    y = x.copy()
    y[1] = [3.0 - 3.0, 4.0 + 1.0, 2.0]          # displacement (-3, +1, +2): along d it is (-9 + 4) / 5 = -1
    rec = m.observables(y, pl=NO_LIST)[0]
    assert rec[F] == pytest.approx(k_s * 1.0, rel=1e-14)
    assert rec[EXT] == pytest.approx(math.sqrt(0.0 + 25.0 + 4.0), rel=1e-15)   # |r_1 - r_0|


def test_extension_is_pulled_to_anchor_distance(orc):
    m, x = pulled_chain(orc, n=6, anchor=1, pulled=4)
    m.start_pulls([(0, 1, 4, 0.05, 0.01)], x)
    y = x.copy()
    y[1] = [10.0, 20.0, 30.0]
    y[4] = [13.0, 24.0, 30.0]                    # 3-4-5 triangle from the anchor
    y[0] = [-500.0, 0.0, 0.0]                    # bead 0 and the last bead do not enter
    y[5] = [900.0, 0.0, 0.0]
    rec = m.observables(y, pl=NO_LIST, step=123)[0]
    assert rec[EXT] == 5.0


def test_tip_moves_from_the_start_step(orc):
    # the pulled bead sits where the tip started: the spring then stretches by the
    # tip's travel v (n - n0), so f = k_s v (n - n0), negative before n0
    k_s, v, n0 = 0.05, 0.01, 40
    m, x = pulled_chain(orc)
    m.start_pulls([(0, 1, 3, k_s, v)], x, step=n0)
    for n in (0, 39, 40, 41, 1000, 123456):
        rec = m.observables(x, pl=NO_LIST, step=n)[0]
        assert rec[F] == pytest.approx(k_s * v * (n - n0), rel=1e-12, abs=1e-15)
        assert rec[STEP] == n


def test_pull_force_record_during_a_run(orc):
    # anchor and pulled bead both fixed, no noise: the records of a run carry the tip
    # position of their own step, k_s v (n - n0) along d
    n = 5
    fixed = np.zeros(n, np.uint8)
    fixed[[1, 3]] = 1
    q = dict(P, T=0.0)
    x = straight(n)
    m = orc.Model(x, np.zeros(n, np.int32), np.zeros(n, np.int32), fixed=fixed, params=q)
    k_s, v, n0 = 0.05, 0.01, 30
    m.start_pulls([(0, 1, 3, k_s, v)], x, step=n0)
    xr, obs, rc, _ = m.run(x, 200, seed=1, obs_every=20)
    assert list(obs[:, STEP]) == list(range(20, 201, 20))
    for rec in obs:
        assert rec[F] == pytest.approx(k_s * v * (rec[STEP] - n0), rel=1e-12, abs=1e-15)
        assert rec[EXT] == pytest.approx(2 * 3.8, rel=1e-15)
    assert np.array_equal(xr[[1, 3]], x[[1, 3]])


def indenter_model(orc, beads, sys=None):
    x = np.asarray(beads, np.float64)
    n = len(x)
    chain = np.arange(n, dtype=np.int32)       # one chain per bead: no bonds, no natives
    m = orc.Model(x, chain, np.zeros(n, np.int32) if sys is None else np.asarray(sys, np.int32), params=P)
    return m, x


def test_indenter_readout_at_gap_sigma(orc):
    # a bead at gap sigma ahead of the indenter is pushed with 6 eps / sigma along the motion
    R, sig = 50.0, 3.8
    m, x = indenter_model(orc, [[0.0, 0.0, -(R + sig)]])
    m.set_indenter((0.0, 0.0, 0.0), (0.0, 0.0, -1.0), R, 0.0)
    rec = m.observables(x, pl=NO_LIST)[0]
    assert rec[F] == pytest.approx(6.0 / sig, rel=1e-14)
    # behind the indenter the push is against its motion
    m.set_indenter((0.0, 0.0, 0.0), (0.0, 0.0, 1.0), R, 0.0)
    assert m.observables(x, pl=NO_LIST)[0][F] == pytest.approx(-6.0 / sig, rel=1e-14)


def test_indenter_readout_is_projected_on_its_motion(orc):
    # at angle theta to the motion the readout is (6 eps / sigma) cos(theta); at gap 2 sigma
    # the wall force falls by 2^7
    R, sig = 50.0, 3.8
    th = math.pi / 3
    u = np.array([math.sin(th), 0.0, math.cos(th)])
    m, x = indenter_model(orc, [(R + sig) * u, (R + 2 * sig) * np.array([0.0, 1.0, 0.0])])
    m.set_indenter((0.0, 0.0, 0.0), (0.0, 0.0, 1.0), R, 0.0)
    rec = m.observables(x, pl=NO_LIST)[0]
    assert rec[F] == pytest.approx(6.0 / sig * math.cos(th), rel=1e-13)   # the second bead is perpendicular
    m.set_indenter((0.0, 0.0, 0.0), (0.0, 1.0, 0.0), R, 0.0)
    rec = m.observables(x, pl=NO_LIST)[0]
    assert rec[F] == pytest.approx(6.0 / sig / 2 ** 7, rel=1e-13)


def test_indenter_centre_and_travel_follow_the_step(orc):
    # the centre starts at c0 and moves v (n - n0) along its direction; the bead sits at
    # gap sigma from where the centre is at step n1, so the readout is 6 eps / sigma there
    R, sig, v, n0, n1 = 50.0, 3.8, 0.005, 100, 2100
    m, x = indenter_model(orc, [[0.0, 0.0, -(R + sig) - v * (n1 - n0)]])
    m.set_indenter((0.0, 0.0, 0.0), (0.0, 0.0, -1.0), R, v, step=n0)
    rec = m.observables(x, pl=NO_LIST, step=n1)[0]
    assert rec[F] == pytest.approx(6.0 / sig, rel=1e-12)
    assert rec[EXT] == pytest.approx(v * (n1 - n0), rel=1e-15)
    far = m.observables(x, pl=NO_LIST, step=n0)[0]
    gap = R + sig + v * (n1 - n0) - R
    assert far[F] == pytest.approx(6.0 * (sig / gap) ** 6 / gap, rel=1e-12)
    assert far[EXT] == 0.0


def test_indenter_readout_sums_each_system_and_a_pulled_system_reports_its_spring(orc):
    R, sig = 50.0, 3.8
    beads = [[0.0, 0.0, -(R + sig)], [0.0, 0.0, -(R + sig) - 200.0],   # system 0
             [0.0, 0.0, -(R + sig)], [0.0, 3.8, -(R + sig) - 100.0],    # system 1 (pulled)
             [0.0, 0.0, -(R + 2 * sig)]]                                # system 2
    m, x = indenter_model(orc, beads, sys=[0, 0, 1, 1, 2])
    m.set_indenter((0.0, 0.0, 0.0), (0.0, 0.0, -1.0), R, 0.001, step=0)
    m.start_pulls([(1, 2, 3, 0.05, 0.0)], x)
    rec = m.observables(x, pl=NO_LIST, step=0)
    far = 6.0 * (sig / 203.8) ** 6 / 203.8
    assert rec[0, F] == pytest.approx(6.0 / sig + far, rel=1e-13)
    assert rec[0, EXT] == 0.0
    assert rec[1, F] == 0.0                                # the spring, at rest
    assert rec[1, EXT] == pytest.approx(math.hypot(3.8, 100.0), rel=1e-15)
    assert rec[2, F] == pytest.approx(6.0 / sig / 2 ** 7, rel=1e-13)


def test_fraction_of_native_contacts_threshold(orc):
    # two systems of two one-bead chains: every pair across chains of a system within
    # R_C is native, so each system holds one contact at its native length r0
    r0a, r0b = 5.0, 6.0
    xn = np.array([[0.0, 0.0, 0.0], [r0a, 0.0, 0.0], [0.0, 100.0, 0.0], [r0b, 100.0, 0.0]])
    m = orc.Model(xn, np.arange(4, dtype=np.int32), np.array([0, 0, 1, 1], np.int32), params=P)
    assert len(m.nat_i) == 2
    for da, db, qa, qb in ((0.0, 0.0, 1.0, 1.0), (1.999, 2.0, 1.0, 0.0), (2.0, 1.5, 0.0, 1.0),
                           (-1.0, 7.0, 1.0, 0.0)):
        y = xn.copy()
        y[1, 0] += da
        y[3, 0] += db
        rec = m.observables(y, pl=NO_LIST)
        assert rec[0, Q] == qa and rec[1, Q] == qb        # formed iff r < r0 + 2 A


def test_fraction_of_native_contacts_counts_over_the_system(orc):
    # one system, four contacts (chains of one bead); breaking one gives Q = 3/4
    xn = np.array([[0.0, 0.0, 0.0], [5.0, 0.0, 0.0], [0.0, 50.0, 0.0], [6.0, 50.0, 0.0]])
    xn = np.concatenate([xn, xn + [0.0, 0.0, 200.0]])
    m = orc.Model(xn, np.arange(8, dtype=np.int32), np.zeros(8, np.int32), params=P)
    assert len(m.nat_i) == 4
    y = xn.copy()
    y[7, 0] += 2.5
    assert m.observables(y, pl=NO_LIST)[0, Q] == 0.75


def test_energy_record_of_a_stretched_bond_and_a_listed_pair(orc):
    # Eq. 1 at a configuration with a closed form: one bond stretched so that the FENE
    # log argument is 1/2 ((k/2) R0^2 ln 2) and one listed non-native pair at sigma (eps)
    d = 2.0 / math.sqrt(2.0)
    xn = np.array([[0.0, 0.0, 0.0], [3.8, 0.0, 0.0], [0.0, 50.0, 0.0], [0.0, 50.0 + 12.0, 0.0]])
    m = orc.Model(xn, np.array([0, 0, 1, 2], np.int32), np.zeros(4, np.int32), params=P)
    assert len(m.nat_i) == 0 and len(m.bond_i) == 1
    y = xn.copy()
    y[1, 0] = 3.8 + d
    y[3, 1] = 50.0 + 3.8
    rec = m.observables(y, pl=(np.array([2], np.int32), np.array([3], np.int32)))[0]
    assert rec[E] == pytest.approx(0.5 * 14.0 * 4.0 * math.log(2.0) + 1.0, rel=1e-13)


def test_cantilever_force_is_a_3d_spring_to_the_moving_tip(orc):
    # the force on the pulled bead is k_s (X_tip(n) - r) in full (not projected), with the
    # tip at tip0 + v (n - n0) d; here d = +x and tip0 = r_3 of the start configuration
    k_s, v, n0, n = 0.05, 0.01, 40, 240
    x = straight(5, 12.0)                     # beads beyond R_C: no native contacts
    m = orc.Model(x, np.arange(5, dtype=np.int32), np.zeros(5, np.int32), params=P)
    assert len(m.nat_i) == 0
    m.start_pulls([(0, 1, 3, k_s, v)], x, step=n0)
    y = x.copy()
    dx, dy, dz = 0.5, -1.5, 2.0
    y[3] += [dx, dy, dz]
    F, A, _ = m.forces(y, pl=NO_LIST, step=n)
    assert F[3] == pytest.approx(k_s * np.array([v * (n - n0) - dx, -dy, -dz]), rel=1e-12)
    assert np.all(F[[0, 1, 2, 4]] == 0.0)     # the anchor is held by being fixed, not by a force


def test_indenter_force_follows_the_moving_centre(orc):
    # at step n1 the centre has moved v (n1 - n0) along its direction; a bead at gap sigma
    # from it there feels 6 eps / sigma along (r - c) / |r - c|
    R, sig, v, n0, n1 = 50.0, 3.8, 0.005, 100, 2100
    u = np.array([0.6, 0.0, -0.8])
    c1 = np.array([0.0, 0.0, -v * (n1 - n0)])
    m, x = indenter_model(orc, [c1 + (R + sig) * u])
    m.set_indenter((0.0, 0.0, 0.0), (0.0, 0.0, -1.0), R, v, step=n0)
    F, A, E = m.forces(x, pl=NO_LIST, step=n1)
    assert F[0] == pytest.approx(6.0 / sig * u, rel=1e-12)
    assert E[3] == pytest.approx(1.0, rel=1e-12)
