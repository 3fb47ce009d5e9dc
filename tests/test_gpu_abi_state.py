"""Host-side state of the C ABI (needs a GPU): pulling records replaced or removed
keep the beads that the topology fixed, a failing call leaves the context as it was,
and a corrupted checkpoint is refused before anything changes."""
import struct

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sop():
    from paper_1003_1148_gb300 import build, sop as s
    build.build()
    s.load()
    return s


@pytest.mark.parametrize("schedule", ["batched", "streamed"])
def test_unpulling_keeps_the_fixed_mask(sop, synth, schedule):
    """fiber4096 fixes its N-terminus through the topology and also anchors the
    cantilever there: removing or replacing the spring must not release it."""
    w = synth.fiber4096(steps=20)
    sim = sop.from_workload(w, schedule=schedule)
    x0 = sim.get_positions(0)
    sim.step(20)
    sim.pull([])                                     # remove pulling
    sim.step(20)
    x1 = sim.get_positions(0)
    assert np.array_equal(x1[0], x0[0])
    sim.pull([(0, 0, 2000, 0.05, 0.01)])             # replace it: same anchor, another pulled bead
    sim.step(20)
    sim.pull([(0, 100, 4095, 0.05, 0.01)])           # replace it: another anchor
    sim.step(20)
    x2 = sim.get_positions(0)
    assert np.array_equal(x2[0], x0[0])
    assert not np.array_equal(x2[4095], x1[4095])
    sim.close()


def test_unpulling_releases_an_anchor_the_mask_did_not_fix(sop, synth):
    w = synth.chain64()
    sim = sop.from_workload(w, n_replicas=1, schedule="batched")
    sim.pull([(0, 5, 63, 0.05, 0.01)])
    x0 = sim.get_positions(0)
    sim.step(20)
    assert np.array_equal(sim.get_positions(0)[5], x0[5])    # anchored
    sim.pull([])
    sim.step(20)
    assert not np.array_equal(sim.get_positions(0)[5], x0[5])
    sim.close()


def test_failing_pull_leaves_the_context_unchanged(sop, synth):
    w = synth.fiber4096(n=512, steps=20)
    sim = sop.from_workload(w, schedule="streamed")
    sim.step(10)
    x = sim.get_positions(0)
    x[300] = x[200]                                  # two coincident beads
    sim.set_positions(x)
    before = sim.get_state()
    with pytest.raises(sop.SopError) as e:
        sim.pull([(0, 200, 300, 0.05, 0.01)])
    assert e.value.status == sop.ERR_INVALID_ARG
    assert sim.get_state() == before
    sim.close()


def _layout(sim, blob):
    """Byte offsets of the parts of a state blob (the layout sop_get_state writes)."""
    hdr = struct.unpack_from("<16q", blob, 0)
    n, R, npull = hdr[2], hdr[3], hdr[6]
    off_pos = 16 * 8
    off_status = off_pos + 3 * R * n * 16
    off_pull = off_status + 4 * R
    return dict(hdr=hdr, npull=npull, status=off_status, sys=off_pull, anchor=off_pull + 4 * npull,
                bead=off_pull + 8 * npull, ks=off_pull + 12 * npull)


@pytest.mark.parametrize("schedule", ["batched", "streamed"])
def test_corrupted_checkpoint_is_refused(sop, synth, schedule):
    w = synth.fiber4096(n=512, steps=20)
    sim = sop.from_workload(w, n_replicas=2, schedule=schedule, obs_every=10)
    sim.step(20)
    good = sim.get_state()
    lay = _layout(sim, good)
    assert lay["npull"] == 1

    def patched(offset, fmt, value):
        b = bytearray(good)
        struct.pack_into(fmt, b, offset, value)
        return bytes(b)

    bad = [
        patched(6 * 8, "<q", 1 << 40),                 # record count far beyond the systems
        patched(6 * 8, "<q", -1),
        patched(4 * 8, "<q", -5),                      # negative step
        patched(lay["bead"], "<i", 1 << 30),           # pulled bead outside the system
        patched(lay["anchor"], "<i", -7),
        patched(lay["sys"], "<i", 3),                  # system out of range
        patched(lay["bead"], "<i", 0),                 # pulled bead == anchor (bead 0)
        patched(lay["ks"], "<d", float("nan")),
        patched(lay["status"], "<i", 1234),            # not a status
        good[:-8],                                      # truncated
    ]
    for blob in bad:
        with pytest.raises(sop.SopError) as e:
            sim.set_state(blob)
        assert e.value.status == sop.ERR_INVALID_ARG
        assert sim.get_state() == good
    # the context still runs and still accepts its own checkpoint
    sim.set_state(good)
    sim.step(10)
    assert np.all(sim.replica_status() == 0)
    sim.close()
