"""ctypes marshalling for the FP64 oracle in ``sop_oracle.c``.

TEST INFRASTRUCTURE ONLY (see the package docstring): tests, the smoke check
and the benchmark's CPU-baseline leg are its only users.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sop_oracle.c")
_HDR = os.path.join(_HERE, "sop_oracle.h")
_OUT = os.path.join(_HERE, "_lib")
_SO = os.path.join(_OUT, "liborc.so")
_lock = threading.Lock()
_lib = None

ERRORS = {0: "ok", 1: "bad argument", 2: "capacity", 3: "FENE bond broken", 4: "bead inside indenter",
          5: "non-finite position"}


class OracleError(RuntimeError):
    def __init__(self, code: int, where: str = ""):
        super().__init__(f"oracle error {code} ({ERRORS.get(code, '?')}) {where}")
        self.code = code


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/_lib/liborc.so``."""
    os.makedirs(_OUT, exist_ok=True)
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < newest:
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-std=c11", "-ffp-contract=off",
                               "-fno-fast-math", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


class _Pull(C.Structure):
    _fields_ = [("system", C.c_int32), ("anchor", C.c_int32), ("pulled", C.c_int32), ("k_s", C.c_double),
                ("v", C.c_double), ("dir", C.c_double * 3), ("tip0", C.c_double * 3), ("n0", C.c_int64)]


class _Indenter(C.Structure):
    _fields_ = [("c0", C.c_double * 3), ("dir", C.c_double * 3), ("radius", C.c_double), ("v", C.c_double),
                ("n0", C.c_int64)]


class _Model(C.Structure):
    _fields_ = [("n", C.c_int32), ("chain", C.c_void_p), ("sys", C.c_void_p), ("fixed", C.c_void_p),
                ("n_bonds", C.c_int32), ("bond_i", C.c_void_p), ("bond_j", C.c_void_p), ("bond_r0", C.c_void_p),
                ("n_nat", C.c_int64), ("nat_i", C.c_void_p), ("nat_j", C.c_void_p), ("nat_r0", C.c_void_p),
                ("k_fene", C.c_double), ("R0", C.c_double), ("eps_h", C.c_double), ("eps_l", C.c_double),
                ("sigma", C.c_double), ("T", C.c_double), ("zeta", C.c_double), ("dt", C.c_double),
                ("pair_cut", C.c_double), ("rebuild_every", C.c_int32), ("use_cells", C.c_int32),
                ("noise_offset", C.c_int32),
                ("n_pull", C.c_int32), ("pulls", C.c_void_p), ("indenter", C.c_void_p), ("taus", C.c_void_p),
                ("integrator", C.c_int32), ("mass", C.c_double), ("vel", C.c_void_p)]


def _L():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(_SO)
            vp, i32, i64, f64, u64 = C.c_void_p, C.c_int32, C.c_int64, C.c_double, C.c_uint64
            L.orc_kB.restype = f64
            L.orc_bonds.argtypes = [i32, vp, vp, vp, vp, vp]
            L.orc_bonds.restype = i32
            for f in (L.orc_native_pairs, L.orc_native_pairs_cells):
                f.argtypes = [i32, vp, vp, vp, f64, vp, vp, vp, i64]
                f.restype = i64
            for f in (L.orc_pairlist_brute, L.orc_pairlist_cells):
                f.argtypes = [vp, vp, vp, vp, i64]
                f.restype = i64
            L.orc_forces.argtypes = [vp, vp, i64, vp, vp, i64, vp, vp, vp]
            L.orc_forces.restype = C.c_int
            L.orc_philox4x32_10.argtypes = [vp, vp, vp]
            L.orc_box_muller.argtypes = [vp, vp]
            L.orc_noise.argtypes = [u64, i64, i32, vp]
            L.orc_ramp_theory.argtypes = [vp, f64]
            L.orc_ramp_theory.restype = f64
            L.orc_ramp_mean.argtypes = [vp, i64]
            L.orc_ramp_mean.restype = f64
            L.orc_box_muller4.argtypes = [vp, vp]
            L.orc_ramp_run.argtypes = [vp, u64, i64, i64]
            L.orc_ramp_run.restype = f64
            L.orc_taus_next.argtypes = [vp]
            L.orc_taus_next.restype = C.c_uint32
            L.orc_taus_noise.argtypes = [vp, vp]
            L.orc_ermak_update.argtypes = [vp, vp, vp, u64, i64]
            L.orc_baoab_update.argtypes = [vp, vp, vp, u64, i64]
            L.orc_observables.argtypes = [vp, vp, i64, vp, vp, i64, i32, vp]
            L.orc_observables.restype = C.c_int
            L.orc_run.argtypes = [vp, vp, i64, i64, u64, i32, i32, vp, i64, vp, vp]
            L.orc_run.restype = C.c_int
            _lib = L
    return _lib


def _p(a: np.ndarray | None):
    return None if a is None else a.ctypes.data


def kB() -> float:
    """Boltzmann constant, kcal/(mol K)."""
    return float(_L().orc_kB())


def bonds(xyz: np.ndarray, chain: np.ndarray):
    """FENE bonds (i, i+1) of every chain with their native lengths."""
    xyz = np.ascontiguousarray(xyz, np.float64)
    chain = np.ascontiguousarray(chain, np.int32)
    n = len(chain)
    bi, bj, r0 = np.zeros(n, np.int32), np.zeros(n, np.int32), np.zeros(n, np.float64)
    nb = _L().orc_bonds(n, _p(xyz), _p(chain), _p(bi), _p(bj), _p(r0))
    return bi[:nb], bj[:nb], r0[:nb]


def native_pairs(xyz, chain, sys, cut: float = 8.0, cells: bool = False):
    """Native contacts (i < j, |i-j| > 2 in a chain, same system, r < cut) of Eq. 1."""
    xyz = np.ascontiguousarray(xyz, np.float64)
    chain = np.ascontiguousarray(chain, np.int32)
    sys = np.ascontiguousarray(sys, np.int32)
    n = len(chain)
    cap = max(1024, 64 * n)
    while True:
        ni, nj, r0 = np.zeros(cap, np.int32), np.zeros(cap, np.int32), np.zeros(cap, np.float64)
        f = _L().orc_native_pairs_cells if cells else _L().orc_native_pairs
        cnt = f(n, _p(xyz), _p(chain), _p(sys), cut, _p(ni), _p(nj), _p(r0), cap)
        if cnt >= 0:
            return ni[:cnt].copy(), nj[:cnt].copy(), r0[:cnt].copy()
        cap *= 4


def philox(ctr, key) -> np.ndarray:
    """One Philox4x32-10 block: 4 uint32 from counter (4 uint32) and key (2 uint32)."""
    c = np.ascontiguousarray(ctr, np.uint32)
    k = np.ascontiguousarray(key, np.uint32)
    out = np.zeros(4, np.uint32)
    _L().orc_philox4x32_10(_p(c), _p(k), _p(out))
    return out


def box_muller(x) -> np.ndarray:
    """Three normals from one block of 4 uint32 (Box-Muller)."""
    xx = np.ascontiguousarray(x, np.uint32)
    g = np.zeros(3, np.float64)
    _L().orc_box_muller(_p(xx), _p(g))
    return g


def noise(seed: int, step: int, bead: int) -> np.ndarray:
    """Gaussian 3-vector of `bead` at `step` for the replica keyed by `seed`."""
    g = np.zeros(3, np.float64)
    _L().orc_noise(seed, step, bead, _p(g))
    return g


class Model:
    """One replica's topology, parameters and external forces, as the oracle sees them.

    chain/sys are per-bead chain and system ids, fixed a per-bead 0/1 mask.
    Natives and bonds come from the native coordinates (FP64). Pulls are
    (system, anchor, pulled, k_s, v) with the direction and tip taken from
    the positions given to ``start_pulls``.
    """

    def __init__(self, native_xyz, chain, sys, fixed=None, params=None, native_cells: bool = False,
                 extra_bonds=None):
        p = dict(k_fene=14.0, R0=2.0, eps_h=1.0, native_cut=8.0, eps_l=1.0, sigma=3.8, T=300.0, zeta=50.0,
                 dt=0.1, pair_cut=10.0, rebuild_every=10)
        p.update(params or {})
        self.params = p
        self.native_xyz = np.ascontiguousarray(native_xyz, np.float64)
        self.chain = np.ascontiguousarray(chain, np.int32)
        self.sys = np.ascontiguousarray(sys, np.int32)
        self.n = len(self.chain)
        self.n_systems = int(self.sys.max()) + 1 if self.n else 0
        self.fixed = np.ascontiguousarray(fixed if fixed is not None else np.zeros(self.n), np.uint8)
        self.bond_i, self.bond_j, self.bond_r0 = bonds(self.native_xyz, self.chain)
        self.nat_i, self.nat_j, self.nat_r0 = native_pairs(self.native_xyz, self.chain, self.sys,
                                                           p["native_cut"], cells=native_cells)
        xb = np.asarray(extra_bonds if extra_bonds is not None else [], np.int32).reshape(-1, 2)
        if len(xb):
            # cross-links: more FENE terms of Eq. 1 with their native lengths; a covalently
            # linked pair is not a (non-covalent) native contact
            a, b = xb.min(1), xb.max(1)
            d = self.native_xyz[a] - self.native_xyz[b]
            r0 = np.sqrt((d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1]) + d[:, 2] * d[:, 2])
            self.bond_i = np.concatenate([self.bond_i, a]).astype(np.int32)
            self.bond_j = np.concatenate([self.bond_j, b]).astype(np.int32)
            self.bond_r0 = np.concatenate([self.bond_r0, r0])
            linked = set(zip(a.tolist(), b.tolist()))
            keep = np.array([(i, j) not in linked for i, j in zip(self.nat_i.tolist(), self.nat_j.tolist())],
                            dtype=bool)
            self.nat_i, self.nat_j, self.nat_r0 = self.nat_i[keep], self.nat_j[keep], self.nat_r0[keep]
        self.pulls = (_Pull * 1)()
        self.n_pull = 0
        self.indenter = None
        self.use_cells = 0
        self.noise_offset = 0
        self.taus = None
        self.integrator, self.mass, self.vel = 0, 0.0, None
        self._sync()

    def _sync(self):
        p = self.params
        self._m = _Model(self.n, _p(self.chain), _p(self.sys), _p(self.fixed), len(self.bond_i),
                         _p(self.bond_i), _p(self.bond_j), _p(self.bond_r0), len(self.nat_i), _p(self.nat_i),
                         _p(self.nat_j), _p(self.nat_r0), p["k_fene"], p["R0"], p["eps_h"], p["eps_l"],
                         p["sigma"], p["T"], p["zeta"], p["dt"], p["pair_cut"], int(p["rebuild_every"]),
                         int(self.use_cells), int(self.noise_offset), self.n_pull, C.addressof(self.pulls) if self.n_pull else None,
                         C.addressof(self.indenter) if self.indenter is not None else None,
                         _p(self.taus) if self.taus is not None else None, int(self.integrator),
                         float(self.mass), _p(self.vel) if self.vel is not None else None)

    def set_cells(self, on: bool):
        self.use_cells = 1 if on else 0
        self._sync()

    def set_noise_offset(self, offset: int):
        """Bead index offset of the noise counter (for a chain taken out of a larger topology)."""
        self.noise_offset = int(offset)
        self._sync()

    def set_taus_state(self, state):
        """Use Hybrid Taus noise (Algorithm 6) with per-bead state [n, 4] (uint32), advanced in
        place by every update; None returns to Philox."""
        self.taus = None if state is None else np.ascontiguousarray(state, np.uint32).reshape(self.n, 4).copy()
        self._sync()

    def set_underdamped(self, mass: float, vel=None):
        """Underdamped BAOAB dynamics (mass in (kcal/mol) ps^2/A^2, friction = zeta) with the
        stored velocities vel [n, 3] (default 0), advanced in place; mass None returns to the
        overdamped update."""
        if mass is None:
            self.integrator, self.mass, self.vel = 0, 0.0, None
        else:
            self.integrator, self.mass = 1, float(mass)
            self.vel = np.zeros((self.n, 3)) if vel is None else np.ascontiguousarray(vel, np.float64).reshape(
                self.n, 3).copy()
        self._sync()

    def velocities(self):
        return None if self.vel is None else self.vel.copy()

    def baoab_update(self, xyz, F, seed: int, step: int):
        xyz = np.ascontiguousarray(xyz, np.float64).copy()
        F = np.ascontiguousarray(F, np.float64)
        _L().orc_baoab_update(C.byref(self._m), _p(xyz), _p(F), seed, step)
        return xyz

    def taus_state(self):
        return None if self.taus is None else self.taus.copy()

    def start_pulls(self, pulls, xyz, step: int = 0):
        """pulls: iterable of (system, anchor, pulled, k_s, v); direction anchor->pulled at xyz."""
        pulls = list(pulls)
        arr = (_Pull * max(1, len(pulls)))()
        for k, (s, a, b, ks, v) in enumerate(pulls):
            d = np.asarray(xyz[b], np.float64) - np.asarray(xyz[a], np.float64)
            d = d / np.sqrt((d[0] * d[0] + d[1] * d[1]) + d[2] * d[2])
            arr[k] = _Pull(int(s), int(a), int(b), float(ks), float(v), (C.c_double * 3)(*d),
                           (C.c_double * 3)(*np.asarray(xyz[b], np.float64)), int(step))
        self.pulls, self.n_pull = arr, len(pulls)
        self._sync()

    def set_indenter(self, center, direction, radius: float, v: float, step: int = 0):
        self.indenter = _Indenter((C.c_double * 3)(*center), (C.c_double * 3)(*direction), float(radius),
                                  float(v), int(step))
        self._sync()

    def pairlist(self, xyz, cells: bool | None = None):
        """Verlet list (i < j) at positions xyz; brute force unless cells."""
        xyz = np.ascontiguousarray(xyz, np.float64)
        use = self.use_cells if cells is None else cells
        cap = max(4096, 128 * self.n)
        while True:
            pi, pj = np.zeros(cap, np.int32), np.zeros(cap, np.int32)
            f = _L().orc_pairlist_cells if use else _L().orc_pairlist_brute
            cnt = f(C.byref(self._m), _p(xyz), _p(pi), _p(pj), cap)
            if cnt >= 0:
                return pi[:cnt].copy(), pj[:cnt].copy()
            cap *= 4

    def forces(self, xyz, pl=None, step: int = 0):
        """(F [n,3], A [n,3], E_parts[4]) at xyz with list pl (default: built at xyz)."""
        xyz = np.ascontiguousarray(xyz, np.float64)
        pi, pj = pl if pl is not None else self.pairlist(xyz)
        pi, pj = np.ascontiguousarray(pi, np.int32), np.ascontiguousarray(pj, np.int32)
        F, A, E = np.zeros((self.n, 3)), np.zeros((self.n, 3)), np.zeros(4)
        rc = _L().orc_forces(C.byref(self._m), _p(xyz), len(pi), _p(pi), _p(pj), step, _p(F), _p(A), _p(E))
        if rc:
            raise OracleError(rc, "in forces")
        return F, A, E

    def ermak_update(self, xyz, F, seed: int, step: int):
        xyz = np.ascontiguousarray(xyz, np.float64).copy()
        F = np.ascontiguousarray(F, np.float64)
        _L().orc_ermak_update(C.byref(self._m), _p(xyz), _p(F), seed, step)
        return xyz

    def observables(self, xyz, pl=None, step: int = 0):
        xyz = np.ascontiguousarray(xyz, np.float64)
        pi, pj = pl if pl is not None else self.pairlist(xyz)
        pi, pj = np.ascontiguousarray(pi, np.int32), np.ascontiguousarray(pj, np.int32)
        out = np.zeros((self.n_systems, 8))
        rc = _L().orc_observables(C.byref(self._m), _p(xyz), len(pi), _p(pi), _p(pj), step, self.n_systems,
                                  _p(out))
        if rc:
            raise OracleError(rc, "in observables")
        return out

    def run(self, xyz, n_steps: int, seed: int, step0: int = 0, obs_every: int = 0, raise_on_error=True):
        """Run one replica; returns (xyz, obs [k, 8], rc, fail_step)."""
        xyz = np.ascontiguousarray(xyz, np.float64).copy()
        n_rec = (n_steps // obs_every + 1) * self.n_systems if obs_every > 0 else 0
        obs = np.zeros((max(1, n_rec), 8))
        n_obs, fail = C.c_int64(0), C.c_int64(-1)
        rc = _L().orc_run(C.byref(self._m), _p(xyz), step0, n_steps, seed, self.n_systems, obs_every, _p(obs),
                          n_rec, C.byref(n_obs), C.byref(fail))
        if rc and raise_on_error:
            raise OracleError(rc, f"at step {fail.value}")
        return xyz, obs[:n_obs.value].copy(), rc, fail.value


class _Ramp(C.Structure):
    _fields_ = [("K", C.c_double), ("xi", C.c_double), ("kT", C.c_double), ("h", C.c_double),
                ("r_f", C.c_double), ("X0", C.c_double), ("order", C.c_int32)]


class Ramp:
    """The harmonic Brownian particle under a ramp force of Sec. IV.C (any consistent units)."""

    def __init__(self, K, xi, kT, h, r_f, X0=0.0, order=1):
        self._p = _Ramp(float(K), float(xi), float(kT), float(h), float(r_f), float(X0), int(order))
        self.K, self.xi, self.kT, self.h, self.r_f, self.X0, self.order = K, xi, kT, h, r_f, X0, order

    def theory(self, t: float) -> float:
        """Eq. 3."""
        return _L().orc_ramp_theory(C.byref(self._p), float(t))

    def mean(self, n: int) -> float:
        """Eq. 4 (order 1) or Eq. 5 (order 2) iterated n steps."""
        return _L().orc_ramp_mean(C.byref(self._p), int(n))

    def run(self, seed: int, run: int, n_steps: int) -> float:
        """X after n_steps of stochastic run `run`."""
        return _L().orc_ramp_run(C.byref(self._p), int(seed), int(run), int(n_steps))


def box_muller4(x):
    x = np.ascontiguousarray(x, np.uint32)
    g = np.zeros(4)
    _L().orc_box_muller4(_p(x), _p(g))
    return g


def taus_next(state):
    """One Hybrid Taus output; state (4 uint32) is advanced in place."""
    st = np.ascontiguousarray(state, np.uint32)
    out = _L().orc_taus_next(_p(st))
    state[:] = st
    return int(out)


def model_from_workload(w, native_cells: bool | None = None) -> Model:
    """Oracle model of one replica of a synthetic workload (duck-typed: xyz,
    chain_of_bead(), system_of_bead(), fixed, params, pulls, indenter)."""
    if native_cells is None:
        native_cells = w.n_beads > 4096
    m = Model(w.xyz, w.chain_of_bead(), w.system_of_bead(), w.fixed, w.params, native_cells=native_cells,
              extra_bonds=getattr(w, "extra_bonds", None))
    return m
