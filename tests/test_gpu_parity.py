"""CUDA path against the FP64 oracle, through the C ABI (needs a GPU).

Bars (from the method's arithmetic):
  * native map and Verlet list: bit-exact as sets (FP64 decisions on both sides);
  * forces at identical positions: |F_gpu - F_64| <= 1e-5 * A per component, A the
    oracle's term-magnitude scale (sum over terms of each term evaluated with
    magnitudes, which bounds rounding error);
  * energy (FP64 accumulation on both sides): relative 1e-9;
  * positions after 100 steps with the same Philox stream: RMS <= 1e-3 A.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

FORCE_TOL = 1e-5
RMS_TOL = 1e-3


@pytest.fixture(scope="module")
def sop():
    from paper_1003_1148_gb300 import build, sop as s
    build.build()
    s.load()
    return s


def csr_pairs(rp, col):
    out = set()
    for i in range(len(rp) - 1):
        for j in col[rp[i]:rp[i + 1]]:
            if j > i:
                out.add((i, int(j)))
    return out


def csr_is_symmetric_sorted(rp, col):
    for i in range(len(rp) - 1):
        row = col[rp[i]:rp[i + 1]]
        if np.any(np.diff(row) <= 0):
            return False
    pairs = {(i, int(j)) for i in range(len(rp) - 1) for j in col[rp[i]:rp[i + 1]]}
    return all((j, i) in pairs for i, j in pairs)


def small_workloads(synth):
    ws = [synth.chain64(), synth.replicas(n_replicas=6, n=128, steps=100)]
    ws.append(synth.uneven(n_chains=12, lo=50, hi=400, steps=100))
    ws.append(synth.fiber4096(n=700, steps=100))
    ws.append(synth.shell(n_copies=6, n_per=150, r_in=60.0, r_out=80.0, ind_radius=20.0, steps=100))
    return ws


@pytest.fixture(scope="module")
def workloads(synth):
    return small_workloads(synth)


def test_native_map_bit_exact(sop, orc, workloads):
    for w in workloads:
        sim = sop.from_workload(w, n_replicas=1, schedule="streamed")
        rp, col, r0 = sim.get_native_map()
        m = orc.model_from_workload(w)
        got = csr_pairs(rp, col)
        ref = set(zip(m.nat_i.tolist(), m.nat_j.tolist()))
        assert got == ref, w.name
        assert csr_is_symmetric_sorted(rp, col)
        # FP64 r0 identical
        lookup = {(a, b): v for a, b, v in zip(m.nat_i.tolist(), m.nat_j.tolist(), m.nat_r0.tolist())}
        for i in range(len(rp) - 1):
            for k in range(rp[i], rp[i + 1]):
                j = int(col[k])
                assert r0[k] == lookup[(min(i, j), max(i, j))]
        sim.close()


@pytest.mark.parametrize("schedule", ["streamed", "batched", "batched_pairs"])
def test_pairlist_bit_exact_after_steps(sop, orc, workloads, schedule):
    for w in workloads:
        if schedule.startswith("batched") and max(np.diff(w.chain_offsets)) > 2048:
            continue
        if schedule.startswith("batched") and w.n_systems == 1 and w.n_beads > 2048:
            continue
        R = 2
        sim = sop.from_workload(w, n_replicas=R, schedule=schedule)
        m = orc.model_from_workload(w)
        for steps in (0, 23):
            if steps:
                sim.step(steps)
                sim.pairlist_rebuild()
            for r in range(R):
                x = sim.get_positions(r)
                rp, col = sim.get_pairlist(r)
                pi, pj = m.pairlist(x, cells=w.n_beads > 1500)
                assert csr_pairs(rp, col) == set(zip(pi.tolist(), pj.tolist())), (w.name, schedule, steps, r)
                assert csr_is_symmetric_sorted(rp, col)
        sim.close()


@pytest.mark.parametrize("n", [1000, 4096, 8192, 8193])
def test_pairlist_every_build_path_bit_exact(sop, orc, synth, n):
    """One system of n beads: up to 8,192 beads the rows come from the block-culled all-pairs
    build (one, 64 and 128 blocks of 64 beads here), above that from the staged cell list;
    each against the oracle's list at the same positions, after 0 and 23 steps."""
    if n <= 4096:
        w = synth.fiber4096(n=n, steps=100)
    else:   # shell assemblies are quick to generate at these sizes
        copies = 8 if n == 8192 else 3
        w = synth.shell(n_copies=copies, n_per=n // copies, r_in=80.0, r_out=110.0, ind_radius=20.0, steps=100)
        assert w.n_beads == n
    sim = sop.from_workload(w, n_replicas=1, schedule="streamed")
    m = orc.model_from_workload(w)
    for steps in (0, 23):
        if steps:
            sim.step(steps)
            sim.pairlist_rebuild()
        x = sim.get_positions(0)
        rp, col = sim.get_pairlist(0)
        pi, pj = m.pairlist(x, cells=True)
        assert csr_pairs(rp, col) == set(zip(pi.tolist(), pj.tolist())), (n, steps)
        assert csr_is_symmetric_sorted(rp, col)
    sim.close()


def oracle_with_externals(orc, w, x_start):
    m = orc.model_from_workload(w)
    if w.pulls:
        sys_of = w.system_of_bead()
        m.start_pulls([(int(sys_of[p.anchor]), p.anchor, p.pulled, p.k_s, p.v) for p in w.pulls], x_start)
    if w.indenter is not None:
        ind = w.indenter
        m.set_indenter(ind.center, ind.direction, ind.radius, ind.v)
    return m


@pytest.mark.parametrize("schedule", ["streamed", "batched", "pairs", "batched_pairs"])
def test_forces_within_tolerance(sop, orc, workloads, schedule):
    for w in workloads:
        if schedule.startswith("batched") and w.n_systems == 1 and w.n_beads > 2048:
            continue
        sim = sop.from_workload(w, n_replicas=2, schedule=schedule)
        x0 = sim.get_positions(0)
        m = oracle_with_externals(orc, w, x0)
        sim.step(30)
        for r in range(2):
            x = sim.get_positions(r)
            F, E = sim.forces(r)
            Fo, Ao, Eo = m.forces(x, step=30)
            err = np.abs(F - Fo) / Ao
            assert err.max() <= FORCE_TOL, (w.name, schedule, r, err.max())
            e_ref = Eo[0] + Eo[1] + Eo[2]
            assert E == pytest.approx(e_ref, rel=1e-9, abs=1e-9), (w.name, schedule)
        sim.close()


@pytest.mark.parametrize("schedule", ["streamed", "batched", "plain", "pairs", "batched_pairs"])
def test_trajectory_100_steps(sop, orc, workloads, schedule):
    for w in workloads:
        if schedule.startswith("batched") and w.n_systems == 1 and w.n_beads > 2048:
            continue
        R = 2
        sim = sop.from_workload(w, n_replicas=R, schedule=schedule)
        x0 = sim.get_positions(0)
        m = oracle_with_externals(orc, w, x0)
        sim.step(100)
        for r in range(R):
            xg = sim.get_positions(r)
            xo, _, _, _ = m.run(x0, 100, seed=w.seed + r)
            rms = float(np.sqrt(((xg - xo) ** 2).sum(1).mean()))
            assert rms <= RMS_TOL, (w.name, schedule, r, rms)
        sim.close()


@pytest.mark.parametrize("schedule", ["streamed", "batched", "plain", "pairs", "batched_pairs"])
def test_indenter_in_contact(sop, orc, synth, schedule):
    """The indenter's wall term where it matters: a shell assembly with the indenter's
    surface 3 A (below sigma = 3.8 A) above its topmost bead, so that on the beads under it
    the wall force (Sec. IV.B's indentation; its repulsion follows Eq. 1's (sigma/r)^6 term)
    outweighs the sum of the Eq. 1 forces. Forces against the oracle at identical positions
    within 1e-5 of the term scale, and the same 100 steps within an RMS of 1e-3 A."""
    import dataclasses
    from paper_1003_1148_gb300.synth import Indenter
    base = synth.shell(n_copies=6, n_per=150, r_in=60.0, r_out=80.0, ind_radius=20.0, steps=100)
    x32 = base.xyz.astype(np.float32).astype(np.float64)
    top = int(np.argmax(x32[:, 2]))
    gap, radius = 3.0, 20.0
    centre = (float(x32[top, 0]), float(x32[top, 1]), float(x32[top, 2]) + radius + gap)
    w = dataclasses.replace(base, indenter=Indenter(center=centre, direction=(0.0, 0.0, -1.0), radius=radius, v=0.005))
    # the wall term dominates some beads: the oracle with and without the indenter
    m_in = oracle_with_externals(orc, w, x32)
    m_out = orc.model_from_workload(base)
    f_in, _, _ = m_in.forces(x32, step=0)
    f_out, _, _ = m_out.forces(x32, step=0)
    wall = np.linalg.norm(f_in - f_out, axis=1)
    assert (wall > np.linalg.norm(f_out, axis=1)).sum() >= 1, wall.max()
    sim = sop.from_workload(w, n_replicas=2, schedule=schedule)
    x0 = sim.get_positions(0)
    m = oracle_with_externals(orc, w, x0)
    if schedule != "plain":
        F, E = sim.forces(0)
        Fo, Ao, Eo = m.forces(x0, step=0)
        err = np.abs(F - Fo) / Ao
        assert err.max() <= FORCE_TOL, (schedule, err.max())
    sim.step(100)
    for r in range(2):
        xo, _, _, _ = m.run(x0, 100, seed=w.seed + r)
        rms = float(np.sqrt(((sim.get_positions(r) - xo) ** 2).sum(1).mean()))
        assert rms <= RMS_TOL, (schedule, r, rms)
    sim.close()


def test_plain_equals_streamed_bitwise(sop, synth):
    w = synth.uneven(n_chains=5, lo=60, hi=300, steps=50)
    a = sop.from_workload(w, n_replicas=2, schedule="streamed")
    b = sop.from_workload(w, n_replicas=2, schedule="plain")
    a.step(37)
    b.step(37)
    assert np.array_equal(a.get_positions(-1), b.get_positions(-1))


def test_cooperative_chunk_equals_plain_bitwise(sop, synth, monkeypatch):
    """The opt-in cooperative K-step chunk (SOP_COOP=1) does the arithmetic of the per-step
    launches, with a grid barrier between steps: the trajectory is bit-identical."""
    w = synth.uneven(n_chains=5, lo=60, hi=300, steps=50)
    b = sop.from_workload(w, n_replicas=2, schedule="plain")
    monkeypatch.setenv("SOP_COOP", "1")
    a = sop.from_workload(w, n_replicas=2, schedule="streamed")
    monkeypatch.setenv("SOP_COOP", "0")
    c = sop.from_workload(w, n_replicas=2, schedule="streamed")
    for sim in (a, b, c):
        sim.step(37)
    assert np.array_equal(a.get_positions(-1), b.get_positions(-1))
    # one cooperative launch replaces the K step launches of each chunk
    assert a.stats()["kernel_launches"] < c.stats()["kernel_launches"]


def test_spread_step_equals_per_bead_step_bitwise(sop, synth):
    """Launches of at least 152 x 256 beads take k_step_spread, whose update is advance_bead's;
    smaller ones take k_step, which loads the bead's data and draws its Philox noise before
    the gather and then updates with its own copy of that arithmetic. The streamed form over
    one batch of about 42,000 beads (one spread launch per step) and the plain form (one
    k_step launch per chain) must therefore agree bit for bit."""
    w = synth.uneven(n_chains=200, lo=150, hi=300, steps=50)
    assert w.n_beads >= 152 * 256
    a = sop.from_workload(w, n_replicas=1, schedule="streamed")
    b = sop.from_workload(w, n_replicas=1, schedule="plain")
    a.step(23)
    b.step(23)
    assert np.array_equal(a.get_positions(-1), b.get_positions(-1))
    a.close()
    b.close()


def test_observables_match_oracle_at_gpu_positions(sop, orc, synth):
    for schedule in ("streamed", "batched", "pairs", "plain", "batched_pairs"):
        w = synth.uneven(n_chains=4, lo=60, hi=200, steps=100)
        sim = sop.from_workload(w, n_replicas=2, schedule=schedule, obs_every=20)
        x0 = sim.get_positions(0)
        m = oracle_with_externals(orc, w, x0)
        sim.step(40)
        rec, lost = sim.get_observables()
        assert lost == 0 and len(rec) == 2 * 2 * w.n_systems
        last = rec[rec[:, 0] == 40]
        for r in range(2):
            x = sim.get_positions(r)
            ref = m.observables(x, pl=m.pairlist(x), step=40)
            got = last[last[:, 1] == r]
            got = got[np.argsort(got[:, 2])]
            assert np.allclose(got[:, 3], ref[:, 2], rtol=1e-9, atol=1e-9), schedule       # energy
            assert np.allclose(got[:, 4], ref[:, 3], rtol=1e-9, atol=1e-12), schedule      # pull force
            assert np.allclose(got[:, 5], ref[:, 4], rtol=1e-12), schedule                 # extension
            assert np.array_equal(got[:, 6], ref[:, 5]), schedule                          # Q
            assert np.allclose(got[:, 7], ref[:, 6], rtol=1e-12), schedule                 # R_ee
        sim.close()


@pytest.mark.parametrize("schedule", ["streamed", "batched", "pairs", "batched_pairs"])
def test_checkpoint_resume_bit_exact(sop, synth, schedule):
    w = synth.replicas(n_replicas=3, n=100, steps=100)
    sim = sop.from_workload(w, schedule=schedule)
    sim.step(37)
    state = sim.get_state()
    sim.step(55)
    a = sim.get_positions(-1).copy()
    sim.set_state(state)
    sim.step(55)
    b = sim.get_positions(-1)
    assert np.array_equal(a, b)


@pytest.mark.parametrize("schedule", ["batched", "batched_pairs"])
def test_replica_sharding_is_exact(sop, synth, schedule):
    """Replicas split over two contexts (seed offset) reproduce one context bit for bit."""
    w = synth.replicas(n_replicas=5, n=96, steps=60)
    whole = sop.from_workload(w, schedule=schedule)
    whole.step(60)
    x = whole.get_positions(-1)
    a = sop.Simulation(w.xyz, w.chain_offsets, w.system_offsets, w.fixed, w.params, n_replicas=2, seed=w.seed,
                       schedule=schedule)
    b = sop.Simulation(w.xyz, w.chain_offsets, w.system_offsets, w.fixed, w.params, n_replicas=3, seed=w.seed + 2,
                       schedule=schedule)
    a.step(60)
    b.step(60)
    assert np.array_equal(np.concatenate([a.get_positions(-1), b.get_positions(-1)]), x)


@pytest.mark.parametrize("schedule", ["streamed", "batched", "batched_pairs"])
def test_fene_break_freezes_only_that_replica(sop, synth, schedule):
    w = synth.replicas(n_replicas=3, n=64, steps=10)
    sim = sop.from_workload(w, schedule=schedule)
    bad = w.xyz.copy()
    bad[40:] += np.array([30.0, 0.0, 0.0])       # bond 39-40 stretched far beyond R0
    sim.set_positions(bad, replica=1)
    rc = sim.step(10, raise_on_error=False)
    assert rc == sop.ERR_FENE_BREAK
    st = sim.replica_status()
    assert st[1] == sop.ERR_FENE_BREAK and st[0] == 0 and st[2] == 0
    frozen = sim.get_positions(1).copy()
    # the beads of the broken bond never moved; the replica stays frozen
    bad32 = bad.astype(np.float32).astype(np.float64)
    assert np.array_equal(frozen[39:41], bad32[39:41])
    rc = sim.step(10, raise_on_error=False)
    assert rc == sop.ERR_FENE_BREAK
    assert np.array_equal(sim.get_positions(1), frozen)
    assert not np.array_equal(sim.get_positions(0), w.xyz.astype(np.float32).astype(np.float64))


def test_pairlist_overflow_reported(sop, synth):
    w = synth.replicas(n_replicas=1, n=128, steps=10)
    with pytest.raises(sop.SopError) as e:
        sim = sop.from_workload(w, schedule="streamed", pairs_per_bead=2)
        sim.step(10)
    assert e.value.status == sop.ERR_PAIRLIST_OVERFLOW


def test_abort_stops_a_long_run(sop, synth):
    import threading
    w = synth.replicas(n_replicas=64, n=128, steps=10)
    sim = sop.from_workload(w, schedule="batched")
    t = threading.Timer(0.5, sim.abort)
    t.start()
    rc = sim.step(10_000_000, raise_on_error=False)
    t.join()
    assert rc == sop.ERR_ABORTED
    assert sim.stats()["steps"] < 10_000_000


def test_pair_based_is_deterministic_and_close_to_particle_based(sop, synth):
    """The pair-based form writes every force slot from one thread and sums slots in row
    order: two runs agree bit for bit. Its sums differ from the particle-based gather only
    by rounding order."""
    w = synth.shell(n_copies=6, n_per=150, r_in=60.0, r_out=80.0, ind_radius=20.0, steps=100)
    a = sop.from_workload(w, n_replicas=2, schedule="pairs")
    b = sop.from_workload(w, n_replicas=2, schedule="pairs")
    c = sop.from_workload(w, n_replicas=2, schedule="streamed")
    assert a.stats()["schedule"] == sop.SCHED_PAIRS
    for s in (a, b, c):
        s.step(45)
    xa, xb, xc = a.get_positions(-1), b.get_positions(-1), c.get_positions(-1)
    assert np.array_equal(xa, xb)
    assert float(np.sqrt(((xa - xc) ** 2).sum(-1).mean())) <= RMS_TOL
    # forces of both forms at the same positions
    c.set_positions(xa, replica=-1)
    Fa, Ea = a.forces(1)
    Fc, Ec = c.forces(1)
    assert Ea == pytest.approx(Ec, rel=1e-12)
    assert np.abs(Fa - Fc).max() <= 1e-4 * max(1.0, np.abs(Fc).max())
    for s in (a, b, c):
        s.close()


def test_auto_streamed_form_is_timed(sop, synth):
    """For a large single system the automatic schedule is the streamed one, in whichever
    force form (particle- or pair-based) its trial timed faster."""
    w = synth.fiber4096(n=3000, steps=10)
    sim = sop.from_workload(w, schedule="auto")
    st = sim.stats()
    assert st["schedule"] in (sop.SCHED_STREAMED, sop.SCHED_PAIRS)
    assert st["tune_ms"] > 0
    sim.step(20)
    assert np.all(np.isfinite(sim.get_positions(0)))
    sim.close()


def test_spread_step_equals_group_step(sop, synth):
    """Above 38,912 beads per launch the streamed step gathers with the same lanes but
    finishes each bead in its own lane; forces and positions stay bit-identical to the
    per-system launches of the plain form."""
    w = synth.replicas(n_replicas=320, n=128, steps=50)     # 40,960 beads in one launch
    a = sop.from_workload(w, schedule="streamed")
    b = sop.from_workload(w, schedule="plain")
    a.step(33)
    b.step(33)
    assert np.array_equal(a.get_positions(-1), b.get_positions(-1))
    a.close()
    b.close()


def test_pair_form_is_used_and_reproducible(sop, synth):
    """The pair form (each pair evaluated once) runs every bucket of systems up to 256 beads
    when asked for, and two contexts take the same trajectory bit for bit (its sums have a
    fixed order whatever slot a bead lands in)."""
    w = synth.uneven(n_chains=6, lo=50, hi=250, steps=100)
    a = sop.from_workload(w, n_replicas=3, schedule="batched_pairs")
    b = sop.from_workload(w, n_replicas=3, schedule="batched_pairs")
    st = a.stats()
    assert st["pair_buckets"] == st["buckets"] >= 1
    a.step(57)
    b.step(57)
    assert np.array_equal(a.get_positions(-1), b.get_positions(-1))
    g = sop.from_workload(w, n_replicas=3, schedule="batched")
    assert g.stats()["pair_buckets"] == 0


def crosslinked(synth):
    """Two 120-bead chains of one system with five cross-links: three between the chains at
    native contact distances (so they leave the native map), two inside the first chain
    between beads 8.5 to 9.5 A apart (inside the list cutoff, so they leave the list)."""
    from paper_1003_1148_gb300.synth import Workload, default_params
    xyz = synth.compact_chain(240, 11)
    d = np.linalg.norm(xyz[:, None, :] - xyz[None, :, :], axis=2)
    links, used = [], set()
    for lo, hi, ok, want in ((0, 240, lambda i, j: i < 120 <= j and 4.5 < d[i, j] < 7.5, 3),
                             (0, 120, lambda i, j: j > i + 6 and 8.5 < d[i, j] < 9.5, 2)):
        got = 0
        for i in range(lo, hi):
            for j in range(i + 1, hi):
                if got < want and i not in used and j not in used and ok(i, j):
                    links.append((i, j))
                    used |= {i, j}
                    got += 1
    assert len(links) == 5
    return Workload("xlink240", xyz, np.array([0, 120, 240], np.int32), np.array([0, 2], np.int32),
                    np.zeros(240, np.uint8), 1, 100, 0, default_params(), obs_every=10,
                    extra_bonds=[(j, i) if k % 2 else (i, j) for k, (i, j) in enumerate(links)])


@pytest.mark.parametrize("schedule", ["streamed", "plain", "pairs"])
def test_crosslinks_against_the_oracle(sop, orc, synth, schedule):
    """Cross-links on every streamed form: the native map and the Verlet list bit-exact,
    forces within 1e-5 of the term scale, the energy within 1e-9 and 100 steps within an RMS
    of 1e-3 A of the oracle's, which takes the links as FENE terms of Eq. 1."""
    w = crosslinked(synth)
    sim = sop.from_workload(w, n_replicas=2, schedule=schedule)
    m = orc.model_from_workload(w)
    rp, col, _ = sim.get_native_map()
    assert csr_pairs(rp, col) == set(zip(m.nat_i.tolist(), m.nat_j.tolist()))
    x0 = sim.get_positions(0)
    for steps in (0, 30):
        if steps:
            sim.step(steps)
            sim.pairlist_rebuild()
        x = sim.get_positions(1)
        rpl, cl = sim.get_pairlist(1)
        pi, pj = m.pairlist(x)
        assert csr_pairs(rpl, cl) == set(zip(pi.tolist(), pj.tolist())), steps
        F, E = sim.forces(1)
        Fo, Ao, Eo = m.forces(x, step=sim.stats()["steps"])
        assert (np.abs(F - Fo) / Ao).max() <= FORCE_TOL
        assert E == pytest.approx(Eo[0] + Eo[1] + Eo[2], rel=1e-9)
    sim.close()
    sim = sop.from_workload(w, n_replicas=1, schedule=schedule)
    sim.step(100)
    xo, _, _, _ = m.run(x0, 100, seed=w.seed)
    assert float(np.sqrt(((sim.get_positions(0) - xo) ** 2).sum(1).mean())) <= RMS_TOL
    sim.close()


def test_crosslinks_take_a_streamed_schedule(sop, synth):
    w = crosslinked(synth)
    for schedule in ("batched", "batched_pairs"):
        with pytest.raises(sop.SopError) as e:
            sop.from_workload(w, n_replicas=2, schedule=schedule)
        assert e.value.status == sop.ERR_UNSUPPORTED
    sim = sop.from_workload(w, n_replicas=2, schedule="auto")
    assert sim.stats()["schedule"] in (sop.SCHED_STREAMED, sop.SCHED_PAIRS)
    sim.close()
    bad = [(0, 1)], [(5, 5)], [(3, 300)], [(4, 90), (90, 4)]
    for links in bad:
        with pytest.raises(sop.SopError):
            sop.Simulation(w.xyz, w.chain_offsets, w.system_offsets, params=w.params, extra_bonds=links)
