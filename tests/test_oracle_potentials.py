"""Pins of the oracle's potentials, forces and lists (Eq. 1, Algorithms 1 and 3).

Nothing here re-types the oracle's force expressions: each check is a value
fixed by the mathematics of Eq. 1 at a special distance, a derivative taken
numerically, an invariant of central pair forces, or an independent library
(scipy's KD-tree) evaluating the definition of a list.
"""
import json
import math
import os

import numpy as np
import pytest
from scipy.spatial import cKDTree

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))
P = dict(k_fene=14.0, R0=2.0, eps_h=1.0, native_cut=8.0, eps_l=1.0, sigma=3.8, T=300.0, zeta=50.0, dt=0.1,
         pair_cut=10.0, rebuild_every=10)


def two_beads(orc, r_native, r_now, same_chain_gap):
    """Two beads on the x axis. same_chain_gap = 1: bonded pair; 3: native-eligible
    pair of one chain; 2: (i, i+2)-like pair (two chains so no bond is made)."""
    nat = np.array([[0.0, 0, 0], [r_native, 0, 0]])
    now = np.array([[0.0, 0, 0], [r_now, 0, 0]])
    if same_chain_gap == 1:
        m = orc.Model(nat, [0, 0], [0, 0], params=P)
    elif same_chain_gap == 3:
        # a 4-bead chain where beads 0 and 3 carry the contact; 1, 2 far away
        nat = np.array([[0.0, 0, 0], [100.0, 0, 0], [200.0, 0, 0], [r_native, 0, 0]])
        now = np.array([[0.0, 0, 0], [100.0, 0, 0], [200.0, 0, 0], [r_now, 0, 0]])
        m = orc.Model(nat, [0, 1, 2, 3], [0, 0, 0, 0], params=P)  # separate chains: no bonds
        m.bond_i = m.bond_j = np.zeros(0, np.int32)
        m.bond_r0 = np.zeros(0)
        m._sync()
    else:
        m = orc.Model(nat, [0, 1], [0, 0], params=P)
    return m, now


def test_paper_parameters_match_golden():
    g = GOLD["sec_IV_A_sop_model"]
    assert P["R0"] == g["R0_A"] and P["sigma"] == g["sigma_A"] == g["sigma_i_i2_A"]
    assert P["eps_l"] == g["eps_r_kcal_mol"] and P["native_cut"] == g["native_cutoff_RC_A"]


def test_kB_matches_paper_room_temperature(orc):
    # Sec. IV.B: k_B T = 4.14 pN nm at room temperature. 1 kcal/mol = 4184 J / N_A.
    NA = 6.02214076e23
    kT_pNnm = orc.kB() * 300.0 * 4184.0 / NA * 1e21
    assert round(kT_pNnm, 2) == GOLD["sec_IV_B_benchmark"]["kBT_room_pN_nm"]


def test_fene_minimum_and_special_point(orc):
    m, now = two_beads(orc, 3.8, 3.8, 1)
    F, A, E = m.forces(now, pl=(np.zeros(0, np.int32), np.zeros(0, np.int32)))
    assert E[0] == 0.0 and np.all(F == 0.0)
    # at (r - r0)^2 = R0^2 / 2 the log argument is 1/2: V = (k/2) R0^2 ln 2
    r = 3.8 + 2.0 / math.sqrt(2.0)
    m, now = two_beads(orc, 3.8, r, 1)
    F, A, E = m.forces(now, pl=(np.zeros(0, np.int32), np.zeros(0, np.int32)))
    assert E[0] == pytest.approx(0.5 * 14.0 * 4.0 * math.log(2.0), rel=1e-14)
    # stretched bond pulls the beads together: force on bead 0 points to +x
    assert F[0, 0] > 0 and F[1, 0] == -F[0, 0]


def test_fene_symmetric_in_stretch_and_diverges(orc):
    ep = two_beads(orc, 3.8, 3.8 + 1.3, 1)
    em = two_beads(orc, 3.8, 3.8 - 1.3, 1)
    none = (np.zeros(0, np.int32), np.zeros(0, np.int32))
    Ep = ep[0].forces(ep[1], pl=none)[2][0]
    Em = em[0].forces(em[1], pl=none)[2][0]
    assert Ep == pytest.approx(Em, rel=1e-12)
    m, now = two_beads(orc, 3.8, 3.8 + 2.0, 1)   # |r - r0| = R0: log argument 0
    with pytest.raises(orc.OracleError):
        m.forces(now, pl=none)


def test_native_lj_minimum_and_zero(orc):
    r0 = 6.0
    none = (np.zeros(0, np.int32), np.zeros(0, np.int32))
    m, now = two_beads(orc, r0, r0, 3)
    assert len(m.nat_i) == 1
    F, A, E = m.forces(now, pl=none)
    assert E[1] == pytest.approx(-1.0, rel=1e-15)          # V(r0) = -eps_h
    assert np.abs(F).max() < 1e-14                          # minimum
    r = r0 * 2.0 ** (-1.0 / 6.0)                            # V = 0 where (r0/r)^6 = 2
    m, now = two_beads(orc, r0, r, 3)
    F, A, E = m.forces(now, pl=none)
    assert abs(E[1]) < 1e-14
    # there s^6 = 4, s^3 = 2: |F| = 24 eps_h / r, repulsive (bead 3 pushed to +x)
    assert F[3, 0] == pytest.approx(24.0 / r, rel=1e-13)


def test_repulsion_at_sigma(orc):
    m, now = two_beads(orc, 20.0, 3.8, 2)
    pl = (np.array([0], np.int32), np.array([1], np.int32))
    F, A, E = m.forces(now, pl=pl)
    assert E[2] == pytest.approx(1.0, rel=1e-15)            # eps (sigma/sigma)^6
    assert F[1, 0] == pytest.approx(6.0 / 3.8, rel=1e-14)   # 6 eps / sigma, pushing apart
    m, now = two_beads(orc, 20.0, 7.6, 2)
    F, A, E = m.forces(now, pl=pl)
    assert E[2] == pytest.approx(1.0 / 64.0, rel=1e-14)


def perturbed_chain(synth, n=64, seed=1, amp=0.3):
    x = synth.compact_chain(n, seed)
    rng = np.random.default_rng(seed + 100)
    return x, x + amp * rng.standard_normal(x.shape)


def test_forces_are_minus_energy_gradient(orc, synth):
    xn, x = perturbed_chain(synth)
    m = orc.Model(xn, np.zeros(64, np.int32), np.zeros(64, np.int32), params=P)
    pl = m.pairlist(x)
    F, A, _ = m.forces(x, pl=pl)
    h = 1e-5
    worst = 0.0
    for i in range(0, 64, 3):
        for k in range(3):
            xp, xm = x.copy(), x.copy()
            xp[i, k] += h
            xm[i, k] -= h
            Ep = m.forces(xp, pl=pl)[2].sum()
            Em = m.forces(xm, pl=pl)[2].sum()
            fd = -(Ep - Em) / (2 * h)
            worst = max(worst, abs(fd - F[i, k]) / A[i, k])
    assert worst < 1e-6


def test_net_force_and_torque_vanish(orc, synth):
    xn, x = perturbed_chain(synth, 128, 3)
    m = orc.Model(xn, np.zeros(128, np.int32), np.zeros(128, np.int32), params=P)
    F, A, _ = m.forces(x)
    scale = np.abs(F).sum()
    assert np.abs(F.sum(0)).max() < 1e-13 * scale
    torque = np.cross(x, F).sum(0)
    assert np.abs(torque).max() < 1e-12 * scale * np.abs(x).max()


def test_energy_invariant_under_rigid_motion(orc, synth):
    xn, x = perturbed_chain(synth)
    m = orc.Model(xn, np.zeros(64, np.int32), np.zeros(64, np.int32), params=P)
    pl = m.pairlist(x)
    E0 = m.forces(x, pl=pl)[2].sum()
    th = 0.7
    R = np.array([[math.cos(th), -math.sin(th), 0], [math.sin(th), math.cos(th), 0], [0, 0, 1]])
    x2 = x @ R.T + np.array([12.0, -3.0, 40.0])
    E1 = m.forces(x2, pl=pl)[2].sum()
    assert E1 == pytest.approx(E0, rel=1e-11)


def test_native_state_energy_and_q(orc, synth):
    x = synth.compact_chain(64, 1)
    m = orc.Model(x, np.zeros(64, np.int32), np.zeros(64, np.int32), params=P)
    pl = m.pairlist(x)
    F, A, E = m.forces(x, pl=pl)
    assert E[0] == 0.0                                     # every bond at r0
    assert E[1] == pytest.approx(-1.0 * len(m.nat_i), rel=1e-13)  # every contact at its minimum
    obs = m.observables(x, pl=pl, step=0)
    assert obs[0, 5] == 1.0                                # Q = 1 in the native state
    assert obs[0, 2] == pytest.approx(E.sum() - E[3], rel=1e-13)


def _kdtree_pairs(x, cut):
    return {(int(a), int(b)) for a, b in cKDTree(x).query_pairs(cut)}


def test_native_map_matches_kdtree_definition(orc, synth):
    for n, seed in ((64, 1), (300, 7)):
        x = synth.compact_chain(n, seed)
        ni, nj, r0 = orc.native_pairs(x, np.zeros(n, np.int32), np.zeros(n, np.int32), 8.0)
        ref = {(a, b) for a, b in _kdtree_pairs(x, 8.0) if b - a > 2}
        assert set(zip(ni.tolist(), nj.tolist())) == ref
        assert np.allclose(r0, np.linalg.norm(x[ni] - x[nj], axis=1), rtol=1e-15)
        assert np.all(r0 < 8.0)


def test_native_map_multichain_and_systems(orc, synth):
    # two chains in one system: inter-chain contacts have no sequence-gap rule;
    # a third chain in another system never contacts the others.
    x = synth.compact_chain(90, 11)
    chain = np.repeat(np.arange(3), 30).astype(np.int32)
    sys = np.array([0] * 60 + [1] * 30, np.int32)
    ni, nj, _ = orc.native_pairs(x, chain, sys, 8.0)
    ref = set()
    for a, b in _kdtree_pairs(x, 8.0):
        if sys[a] != sys[b]:
            continue
        if chain[a] == chain[b] and b - a <= 2:
            continue
        ref.add((a, b))
    assert set(zip(ni.tolist(), nj.tolist())) == ref
    ci, cj, _ = orc.native_pairs(x, chain, sys, 8.0, cells=True)
    assert np.array_equal(ci, ni) and np.array_equal(cj, nj)


def test_pairlist_matches_kdtree_and_cells(orc, synth):
    for n, seed, amp in ((64, 1, 0.5), (256, 5, 1.0), (1000, 9, 1.0)):
        xn, x = perturbed_chain(synth, n, seed, amp)
        m = orc.Model(xn, np.zeros(n, np.int32), np.zeros(n, np.int32), params=P)
        bi, bj = m.pairlist(x)
        nat = set(zip(m.nat_i.tolist(), m.nat_j.tolist()))
        ref = {(a, b) for a, b in _kdtree_pairs(x, 10.0) if b - a >= 2 and (a, b) not in nat}
        assert set(zip(bi.tolist(), bj.tolist())) == ref
        ci, cj = m.pairlist(x, cells=True)
        assert np.array_equal(ci, bi) and np.array_equal(cj, bj)
        # sorted by (i, j)
        key = bi.astype(np.int64) * n + bj
        assert np.all(np.diff(key) > 0)


def test_table_I_bond_counts_shape(orc):
    # Table I: a single chain of N residues has N-1 covalent bonds (WW 34/33, Ig27 89/88, C2A 126/125).
    t = GOLD["table_I"]
    for N, nb in zip(t["residues"][:3], t["covalent_bonds"][:3]):
        x = np.cumsum(np.tile([[3.8, 0, 0]], (N, 1)), axis=0)
        bi, bj, r0 = orc.bonds(x, np.zeros(N, np.int32))
        assert len(bi) == nb
        assert np.allclose(r0, 3.8)


def test_indenter_wall_value_and_gradient(orc, synth):
    """Wall V = eps (sigma / (|r - c| - R))^6: equals eps where the gap is sigma, and
    the forces it adds are minus the gradient of its energy."""
    x = np.array([[0.0, 0.0, 50.0 + 3.8]])
    m = orc.Model(x, [0], [0])
    m.set_indenter((0.0, 0.0, 0.0), (0.0, 0.0, -1.0), 50.0, 0.0)
    none = (np.zeros(0, np.int32), np.zeros(0, np.int32))
    F, A, E = m.forces(x, pl=none)
    assert E[3] == pytest.approx(1.0, rel=1e-14)
    assert F[0, 2] == pytest.approx(6.0 / 3.8, rel=1e-13)
    xn, xp = perturbed_chain(synth, 40, 2, 0.3)
    xp = xp + np.array([0.0, 0.0, 80.0])
    m = orc.Model(xn, np.zeros(40, np.int32), np.zeros(40, np.int32), params=P)
    m.set_indenter((0.0, 0.0, 20.0), (0.0, 0.0, 1.0), 40.0, 0.01, step=0)
    pl = m.pairlist(xp)
    F, A, _ = m.forces(xp, pl=pl, step=500)
    h = 1e-5
    for i in range(0, 40, 7):
        for k in range(3):
            a, b = xp.copy(), xp.copy()
            a[i, k] += h
            b[i, k] -= h
            fd = -(m.forces(a, pl=pl, step=500)[2].sum() - m.forces(b, pl=pl, step=500)[2].sum()) / (2 * h)
            assert abs(fd - F[i, k]) < 1e-6 * A[i, k]
    with pytest.raises(orc.OracleError):     # a bead inside the indenter is an error
        m.forces(xp, pl=pl, step=10_000)


def test_crosslink_is_the_chain_bond_term(orc):
    """A cross-link (a covalent bond between beads that are not i, i+1 of one chain) is the
    FENE term of Eq. 1: two single-bead chains of one system, linked, give the closed-form
    FENE energy (k/2) R0^2 ln 2 at (r - r0)^2 = R0^2 / 2, and the same forces as the two
    beads bonded as one chain."""
    r = 3.8 + 2.0 / math.sqrt(2.0)
    nat = np.array([[0.0, 0, 0], [3.8, 0, 0]])
    now = np.array([[0.0, 0, 0], [r, 0, 0]])
    none = (np.zeros(0, np.int32), np.zeros(0, np.int32))
    linked = orc.Model(nat, [0, 1], [0, 0], params=P, extra_bonds=[(0, 1)])
    chain = orc.Model(nat, [0, 0], [0, 0], params=P)
    Fl, _, El = linked.forces(now, pl=none)
    Fc, _, Ec = chain.forces(now, pl=none)
    assert El[0] == pytest.approx(0.5 * 14.0 * 4.0 * math.log(2.0), rel=1e-14)
    assert np.array_equal(Fl, Fc) and El[0] == Ec[0]
    assert len(linked.nat_i) == 0 and len(linked.pairlist(now)[0]) == 0


def test_crosslink_leaves_the_native_map_and_the_list(orc, synth):
    """A linked pair is neither a native contact nor a Verlet-list pair, and its force is
    that of a lone bond of the same geometry: the KD-tree definition of the list minus the
    link, and the force difference with and without the link equal to a two-bead chain's."""
    xn, x = perturbed_chain(synth)
    n = len(xn)
    base = orc.Model(xn, np.zeros(n, np.int32), np.zeros(n, np.int32), params=P)
    nat = set(zip(base.nat_i.tolist(), base.nat_j.tolist()))
    # a native pair, and a pair far from both cutoffs in the native structure
    i1, j1 = next((i, j) for i, j in sorted(nat) if j - i > 5)
    d = np.linalg.norm(xn[:, None, :] - xn[None, :, :], axis=2)
    i2, j2 = next((i, j) for i in range(n) for j in range(i + 6, n) if d[i, j] > 12.0)
    m = orc.Model(xn, np.zeros(n, np.int32), np.zeros(n, np.int32), params=P, extra_bonds=[(j1, i1), (i2, j2)])
    assert set(zip(m.nat_i.tolist(), m.nat_j.tolist())) == nat - {(i1, j1)}
    tree = cKDTree(x)
    want = {(a, b) for a, b in tree.query_pairs(P["pair_cut"] - 1e-9)
            if b != a + 1 and (a, b) not in nat and (a, b) not in {(i1, j1), (i2, j2)}}
    for cells in (False, True):
        pi, pj = m.pairlist(x, cells=cells)
        assert set(zip(pi.tolist(), pj.tolist())) == want
    # with the list of the linked model, the far link adds exactly a lone bond's force
    pl = m.pairlist(x)
    no_far = orc.Model(xn, np.zeros(n, np.int32), np.zeros(n, np.int32), params=P, extra_bonds=[(j1, i1)])
    dF = m.forces(x, pl=pl)[0] - no_far.forces(x, pl=pl)[0]
    lone = orc.Model(xn[[i2, j2]], [0, 0], [0, 0], params=P)
    Fl = lone.forces(x[[i2, j2]], pl=(np.zeros(0, np.int32), np.zeros(0, np.int32)))[0]
    assert np.allclose(dF[[i2, j2]], Fl, rtol=1e-12, atol=1e-12)
    others = np.ones(n, bool)
    others[[i2, j2]] = False
    assert np.allclose(dF[others], 0.0, atol=1e-12)
