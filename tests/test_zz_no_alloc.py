"""The allocation-free Verlet-list entry point against the context-based one (needs a GPU).

sop_pairlist_build_noalloc serves callers that cannot call cudaMalloc: hosts
whose device memory all belongs to their own pool allocator, services that must
not allocate after start-up. Its scratch is one fixed array inside the library
that every call reuses, so the checks run two calls in a row, after a call that
failed half way, and compare each list with sop_get_pairlist's for the same
positions; they also check that calls leave the device's free memory unchanged,
that the largest accepted system works, and that a NaN position is reported as such.
This file sorts last so that a run stopping at the first failure has already
run every other test.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    from paper_1003_1148_gb300 import build, sop
    build.build()
    sop.load()
    return sop


def device_inputs(torch, sim, w, dev):
    x = sim.get_positions(0)
    n = w.n_beads
    pos4 = torch.zeros((n, 4), dtype=torch.float32, device=dev)
    pos4[:, :3] = torch.from_numpy(x.astype(np.float32)).to(dev)
    chain = torch.from_numpy(w.chain_of_bead().astype(np.int32)).to(dev)
    nrp, ncol, _ = sim.get_native_map()
    nat_row = torch.from_numpy(nrp.astype(np.int32)).to(dev)
    nat_col = torch.from_numpy(ncol.astype(np.int32) if len(ncol) else np.zeros(1, np.int32)).to(dev)
    return pos4, chain, nat_row, nat_col


def call(torch, sop, inputs, n, cut, cap, dev):
    pos4, chain, nat_row, nat_col = inputs
    rs = torch.full((n,), -1, dtype=torch.int32, device=dev)
    rl = torch.full((n,), -1, dtype=torch.int32, device=dev)
    col = torch.full((max(1, cap),), -1, dtype=torch.int32, device=dev)
    nnz = sop.pairlist_build_noalloc(pos4, n, chain, nat_row, nat_col, cut, rs, rl, col, cap,
                                     stream=torch.cuda.current_stream())
    return nnz, rs.cpu().numpy(), rl.cpu().numpy(), col.cpu().numpy()


def test_noalloc_list_equals_context_list_twice(lib, synth):
    torch = pytest.importorskip("torch")
    sop = lib
    dev = torch.device("cuda", 0)
    for w in (synth.replicas(n_replicas=1, n=128, seed=3), synth.fiber4096(n=1500)):
        sim = sop.from_workload(w, n_replicas=1, schedule="streamed")
        sim.step(25)
        sim.pairlist_rebuild()
        rp_ref, col_ref = sim.get_pairlist(0)
        inputs = device_inputs(torch, sim, w, dev)
        n = w.n_beads
        for _ in range(2):
            nnz, rs, rl, col = call(torch, sop, inputs, n, w.params["pair_cut"], 64 * n, dev)
            assert nnz == len(col_ref)
            for i in range(n):
                row = col[rs[i]:rs[i] + rl[i]]
                assert np.array_equal(row, col_ref[rp_ref[i]:rp_ref[i + 1]]), (w.name, i)
        sim.close()


def test_noalloc_rejects_and_recovers(lib, synth):
    torch = pytest.importorskip("torch")
    sop = lib
    dev = torch.device("cuda", 0)
    w = synth.replicas(n_replicas=1, n=128, seed=3)
    sim = sop.from_workload(w, n_replicas=1, schedule="streamed")
    rp_ref, col_ref = sim.get_pairlist(0)
    inputs = device_inputs(torch, sim, w, dev)
    with pytest.raises(sop.SopError) as e:
        call(torch, sop, inputs, sop.NOALLOC_MAX_BEADS + 1, 10.0, 16, dev)
    assert e.value.status == sop.ERR_INVALID_ARG
    with pytest.raises(sop.SopError) as e:          # too small an output: stops half way
        call(torch, sop, inputs, 128, 10.0, 8, dev)
    assert e.value.status == sop.ERR_PAIRLIST_OVERFLOW
    nnz, rs, rl, col = call(torch, sop, inputs, 128, 10.0, 64 * 128, dev)   # the scratch left behind is reset
    assert nnz == len(col_ref)
    for i in range(128):
        assert np.array_equal(col[rs[i]:rs[i] + rl[i]], col_ref[rp_ref[i]:rp_ref[i + 1]])


def test_noalloc_allocates_nothing_and_reports_nan(lib, synth):
    torch = pytest.importorskip("torch")
    sop = lib
    dev = torch.device("cuda", 0)
    w = synth.replicas(n_replicas=1, n=128, seed=3)
    sim = sop.from_workload(w, n_replicas=1, schedule="streamed")
    inputs = device_inputs(torch, sim, w, dev)
    n = w.n_beads
    rs = torch.empty((n,), dtype=torch.int32, device=dev)
    rl = torch.empty((n,), dtype=torch.int32, device=dev)
    col = torch.empty((64 * n,), dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream()
    sop.pairlist_build_noalloc(*inputs[:1], n, *inputs[1:], 10.0, rs, rl, col, 64 * n, stream=stream)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info(dev)[0]
    for _ in range(5):
        sop.pairlist_build_noalloc(*inputs[:1], n, *inputs[1:], 10.0, rs, rl, col, 64 * n, stream=stream)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info(dev)[0] == free0
    pos4 = inputs[0].clone()
    pos4[17, 1] = float("nan")
    with pytest.raises(sop.SopError) as e:
        sop.pairlist_build_noalloc(pos4, n, *inputs[1:], 10.0, rs, rl, col, 64 * n, stream=stream)
    assert e.value.status == sop.ERR_NONFINITE
    sim.close()


def snake_chain(n, spacing=4.5, dims=(41, 40, 40)):
    """n beads on a serpentine path through a cubic lattice: consecutive beads one lattice
    step apart (the bonds), every other pair at least one step apart."""
    nx, ny, nz = dims
    pts = []
    for z in range(nz):
        ys = range(ny) if z % 2 == 0 else range(ny - 1, -1, -1)
        for k, y in enumerate(ys):
            xs = range(nx) if (z * ny + k) % 2 == 0 else range(nx - 1, -1, -1)
            for x in xs:
                pts.append((x, y, z))
                if len(pts) == n:
                    return spacing * np.array(pts, dtype=np.float64)
    raise ValueError("lattice too small")


def test_noalloc_largest_system(lib):
    """n = SOP_NOALLOC_MAX_BEADS: one 65,536-bead chain on a lattice, against the context's list."""
    torch = pytest.importorskip("torch")
    sop = lib
    dev = torch.device("cuda", 0)
    n = sop.NOALLOC_MAX_BEADS
    xyz = snake_chain(n)
    sim = sop.Simulation(xyz, [0, n], params={}, n_replicas=1, seed=1, schedule="streamed")
    rp_ref, col_ref = sim.get_pairlist(0)
    x = sim.get_positions(0)
    pos4 = torch.zeros((n, 4), dtype=torch.float32, device=dev)
    pos4[:, :3] = torch.from_numpy(x.astype(np.float32)).to(dev)
    chain = torch.zeros((n,), dtype=torch.int32, device=dev)
    nrp, ncol, _ = sim.get_native_map()
    nat_row = torch.from_numpy(nrp.astype(np.int32)).to(dev)
    nat_col = torch.from_numpy(ncol.astype(np.int32)).to(dev)
    nnz, rs, rl, col = call(torch, sop, (pos4, chain, nat_row, nat_col), n, 10.0, 64 * n, dev)
    assert nnz == len(col_ref) > 0
    assert np.array_equal(rl, np.diff(rp_ref))
    for i in range(0, n, 997):
        assert np.array_equal(col[rs[i]:rs[i] + rl[i]], col_ref[rp_ref[i]:rp_ref[i + 1]])
    sim.close()
