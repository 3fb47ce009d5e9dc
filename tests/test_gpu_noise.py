"""The noise of the step (Sec. III.C) through the C ABI against the FP64 oracle (needs a GPU).

The device computes in FP32 from the same 32-bit words; the bound per normal is
radius x 8e-7: the angle's FP32 input is rounded to 24 bits (at most 1.9e-7 rad), and
the logarithm, square root and sine/cosine add a few ulp (each well under 1e-7).
A dropped "+1" in u, a swapped sine and cosine, a wrong sign or a counter word in the
wrong place each moves a normal by far more.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sop():
    from paper_1003_1148_gb300 import build, sop as s
    build.build()
    s.load()
    return s


EDGE = [0, 1, 2, 3, 0x00FFFFFF, 0x01000000, 0x3FFFFFFF, 0x40000000, 0x7FFFFFFE, 0x7FFFFFFF, 0x80000000,
        0x80000001, 0xBFFFFFFF, 0xC0000000, 0xFFFFFF00, 0xFFFFFFFD, 0xFFFFFFFE, 0xFFFFFFFF]


def radii(orc, x):
    """FP64 Box-Muller radii of the blocks (first, second pair)."""
    u1 = (x[:, 0].astype(np.float64) + 1.0) * 2.0 ** -32
    u3 = (x[:, 2].astype(np.float64) + 1.0) * 2.0 ** -32
    return np.sqrt(-2.0 * np.log(u1)), np.sqrt(-2.0 * np.log(u3))


def check(orc, x, got):
    ref = np.array([orc.box_muller(b) for b in x])
    ra, rb = radii(orc, x)
    tol = 8e-7 * np.stack([ra, ra, rb], 1) + 1e-12
    err = np.abs(got - ref)
    assert (err <= tol).all(), (err / tol).max()
    return ref


def test_box_muller_edge_words(sop, orc):
    # every edge value in every word position, the other words random
    rng = np.random.default_rng(5)
    blocks = []
    for pos in range(4):
        for v in EDGE:
            b = rng.integers(0, 2 ** 32, size=4, dtype=np.uint64).astype(np.uint32)
            b[pos] = v
            blocks.append(b)
    x = np.array(blocks, np.uint32)
    got = sop.box_muller(x)
    ref = check(orc, x, got)
    # u = 1 exactly gives radius 0: both sides return exact zeros
    one = x[:, 0] == 0xFFFFFFFF
    assert np.all(got[one, :2] == 0.0) and np.all(ref[one, :2] == 0.0)
    # the smallest u gives the largest radius, sqrt(64 ln 2)
    small = x[:, 0] == 0
    assert np.allclose(np.hypot(got[small, 0], got[small, 1]), np.sqrt(64 * np.log(2)), rtol=1e-6)


def test_box_muller_random_words(sop, orc):
    rng = np.random.default_rng(6)
    x = rng.integers(0, 2 ** 32, size=(20000, 4), dtype=np.uint64).astype(np.uint32)
    check(orc, x, sop.box_muller(x))


def test_bead_noise_matches_oracle_key_and_counter(sop, orc):
    cases = [(0, 0, 0), (7, 123, 5), (2 ** 40 + 3, 2 ** 33 + 17, 1000), (2 ** 64 - 1, 2 ** 63 - 5, 2 ** 32 - 64)]
    for key, step, lo in cases:
        n = 64
        got = sop.bead_noise(key, step, lo, n)
        ref = np.array([orc.noise(key, step, lo + k) for k in range(n)])
        blocks = np.array([orc.philox([step & 0xFFFFFFFF, step >> 32, lo + k, 0], [key & 0xFFFFFFFF, key >> 32])
                           for k in range(n)], np.uint32)
        ra, rb = radii(orc, blocks)
        tol = 8e-7 * np.stack([ra, ra, rb], 1) + 1e-12
        assert (np.abs(got - ref) <= tol).all(), (key, step, lo)


def test_bead_noise_is_standard_normal(sop):
    g = sop.bead_noise(11, 5, 0, 1 << 20)
    m, v = g.mean(0), g.var(0)
    se = 1.0 / np.sqrt(len(g))
    assert np.all(np.abs(m) < 5 * se) and np.all(np.abs(v - 1.0) < 5 * np.sqrt(2.0) * se)


def test_noise_rejects_bad_arguments(sop):
    with pytest.raises(sop.SopError):
        sop.bead_noise(0, 0, 2 ** 32 - 4, 8)
