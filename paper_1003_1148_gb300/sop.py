"""ctypes binding of the C ABI in ``include/sop.h`` (argument marshalling only).

Every step of the simulation runs in the CUDA library ``_lib/libsop.so``; this
module converts numpy arrays to the C structs and pointers the ABI expects and
raises ``SopError`` for any non-OK status. There is no CPU fallback: if the
library is missing or cannot be loaded, ``load()`` raises.

PyTorch is optional here and only supplies a CUDA stream (``stream=`` takes a
``torch.cuda.Stream`` or a raw ``cudaStream_t`` integer).
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libsop.so")
_lock = threading.Lock()
_lib = None

OK, ERR_INVALID_ARG, ERR_CUDA, ERR_OOM, ERR_FENE_BREAK, ERR_NONFINITE, ERR_PAIRLIST_OVERFLOW, ERR_ABORTED, \
    ERR_TIMEOUT, ERR_INDENTER_OVERLAP, ERR_UNSUPPORTED, ERR_CAPACITY = range(12)
STATUS_NAMES = ["OK", "INVALID_ARG", "CUDA", "OOM", "FENE_BREAK", "NONFINITE", "PAIRLIST_OVERFLOW", "ABORTED",
                "TIMEOUT", "INDENTER_OVERLAP", "UNSUPPORTED", "CAPACITY"]
SCHED_AUTO, SCHED_BATCHED, SCHED_STREAMED, SCHED_PLAIN, SCHED_PAIRS, SCHED_BATCHED_PAIRS = range(6)
SCHEDULES = {"auto": SCHED_AUTO, "batched": SCHED_BATCHED, "streamed": SCHED_STREAMED, "plain": SCHED_PLAIN,
             "pairs": SCHED_PAIRS, "batched_pairs": SCHED_BATCHED_PAIRS}

EXPORTED = ["sop_create", "sop_step", "sop_forces", "sop_pairlist_rebuild", "sop_pull", "sop_indenter",
            "sop_get_positions", "sop_set_positions", "sop_get_pairlist", "sop_get_native_map",
            "sop_get_observables", "sop_get_state", "sop_set_state", "sop_replica_status", "sop_abort",
            "sop_get_stats", "sop_last_error", "sop_destroy", "sop_pairlist_build_noalloc", "sop_get_rng_state",
            "sop_set_rng_state", "sop_brownian_ramp", "sop_get_velocities", "sop_set_velocities",
            "sop_box_muller", "sop_bead_noise", "sop_fp32_peak"]
INTEGRATOR_OVERDAMPED, INTEGRATOR_BAOAB = 0, 1
INTEGRATORS = {"overdamped": INTEGRATOR_OVERDAMPED, "baoab": INTEGRATOR_BAOAB}
RNG_PHILOX, RNG_HYBRID_TAUS = 0, 1
RNGS = {"philox": RNG_PHILOX, "taus": RNG_HYBRID_TAUS}


class SopError(RuntimeError):
    def __init__(self, status: int, msg: str):
        name = STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else str(status)
        super().__init__(f"SOP_ERR_{name}: {msg}")
        self.status = status


class Topology(C.Structure):
    _fields_ = [("n_beads", C.c_int32), ("n_chains", C.c_int32), ("chain_offsets", C.c_void_p),
                ("n_systems", C.c_int32), ("system_offsets", C.c_void_p), ("fixed_mask", C.c_void_p),
                ("n_extra_bonds", C.c_int32), ("extra_bonds", C.c_void_p)]


class Params(C.Structure):
    _fields_ = [("k_fene", C.c_double), ("R0", C.c_double), ("eps_h", C.c_double), ("native_cut", C.c_double),
                ("eps_l", C.c_double), ("sigma", C.c_double), ("T", C.c_double), ("zeta", C.c_double),
                ("dt", C.c_double), ("pair_cut", C.c_double), ("rebuild_every", C.c_int32),
                ("n_replicas", C.c_int32), ("seed", C.c_uint64), ("obs_every", C.c_int32),
                ("obs_capacity", C.c_int32), ("pairs_per_bead", C.c_int32), ("schedule", C.c_int32),
                ("cuda_stream", C.c_void_p), ("rng", C.c_int32), ("integrator", C.c_int32), ("mass", C.c_double),
                ("obs_every_q", C.c_int32)]


class PullParams(C.Structure):
    _fields_ = [("system", C.c_int32), ("anchor", C.c_int32), ("pulled", C.c_int32), ("k_s", C.c_double),
                ("v", C.c_double)]


class RampParams(C.Structure):
    _fields_ = [("K", C.c_double), ("xi", C.c_double), ("kT", C.c_double), ("h", C.c_double),
                ("r_f", C.c_double), ("X0", C.c_double), ("n_runs", C.c_int64), ("n_steps", C.c_int64),
                ("order", C.c_int32), ("n_out", C.c_int32), ("seed", C.c_uint64)]


class Record(C.Structure):
    _fields_ = [(k, C.c_double) for k in ("step", "replica", "system", "energy", "f_ext", "extension", "q", "r_ee")]


RECORD_FIELDS = [f for f, _ in Record._fields_]


class Stats(C.Structure):
    _fields_ = [("steps", C.c_int64), ("kernel_launches", C.c_int64), ("graph_launches", C.c_int64),
                ("rebuilds", C.c_int64), ("schedule", C.c_int32), ("block_threads", C.c_int32),
                ("pairs_per_bead", C.c_int32), ("beads_per_thread", C.c_int32), ("min_blocks", C.c_int32),
                ("buckets", C.c_int32),
                ("pairlist_entries", C.c_int64), ("native_entries", C.c_int64), ("tune_ms", C.c_double),
                ("cluster_buckets", C.c_int32), ("cluster_size", C.c_int32), ("pair_buckets", C.c_int32)]


def load(path: str | None = None):
    """Load libsop.so (raises when it is missing: there is no fallback)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise RuntimeError(f"{p} is missing: build it with paper_1003_1148_gb300.build.build()")
        L = C.CDLL(p)
        vp, i32, i64, f64 = C.c_void_p, C.c_int32, C.c_int64, C.c_double
        sig = {
            "sop_create": ([vp, vp, vp, vp], C.c_int),
            "sop_step": ([vp, i64], C.c_int),
            "sop_forces": ([vp, i32, vp, vp], C.c_int),
            "sop_pairlist_rebuild": ([vp], C.c_int),
            "sop_pull": ([vp, i32, vp], C.c_int),
            "sop_indenter": ([vp, vp, vp, f64, f64], C.c_int),
            "sop_get_positions": ([vp, i32, vp], C.c_int),
            "sop_set_positions": ([vp, i32, vp], C.c_int),
            "sop_get_pairlist": ([vp, i32, vp, vp, i64, vp], C.c_int),
            "sop_get_native_map": ([vp, vp, vp, vp, i64, vp], C.c_int),
            "sop_get_observables": ([vp, vp, i64, vp, vp], C.c_int),
            "sop_get_state": ([vp, vp, i64, vp], C.c_int),
            "sop_set_state": ([vp, vp, i64], C.c_int),
            "sop_replica_status": ([vp, vp], C.c_int),
            "sop_abort": ([vp], None),
            "sop_get_stats": ([vp, vp], C.c_int),
            "sop_last_error": ([vp], C.c_char_p),
            "sop_destroy": ([vp], None),
            "sop_pairlist_build_noalloc": ([vp, i32, vp, vp, vp, f64, vp, vp, vp, i64, vp, vp], C.c_int),
            "sop_get_rng_state": ([vp, vp, i64], C.c_int),
            "sop_set_rng_state": ([vp, vp, i64], C.c_int),
            "sop_brownian_ramp": ([vp, vp, vp, vp, vp], C.c_int),
            "sop_get_velocities": ([vp, i32, vp], C.c_int),
            "sop_set_velocities": ([vp, i32, vp], C.c_int),
            "sop_box_muller": ([vp, i64, vp, vp], C.c_int),
            "sop_bead_noise": ([C.c_uint64, i64, C.c_uint32, i64, vp, vp], C.c_int),
            "sop_fp32_peak": ([f64, vp, vp, vp], C.c_int),
        }
        for name, (args, res) in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        _lib = L
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data


def _stream_handle(stream) -> int | None:
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return int(getattr(stream, "cuda_stream"))


class Simulation:
    """One context of the library: a topology, its parameters and R replicas.

    Arguments follow ``sop_create``: ``native_xyz`` [n, 3] FP64 native (and
    starting) coordinates; ``chain_offsets`` [n_chains+1]; ``system_offsets``
    [n_systems+1] in chains (None: every chain is its own system); ``fixed``
    [n] 0/1; ``params`` a dict with the keys of ``sop_params``.
    """

    def __init__(self, native_xyz, chain_offsets, system_offsets=None, fixed=None, params=None, n_replicas=1,
                 seed=0, obs_every=0, obs_capacity=0, pairs_per_bead=0, schedule="auto", stream=None,
                 rng="philox", integrator="overdamped", mass=0.0, obs_every_q=0, extra_bonds=None):
        L = load()
        self._L = L
        xyz = np.ascontiguousarray(native_xyz, np.float64).reshape(-1, 3)
        self.n = xyz.shape[0]
        self.R = int(n_replicas)
        co = np.ascontiguousarray(chain_offsets, np.int32)
        so = None if system_offsets is None else np.ascontiguousarray(system_offsets, np.int32)
        fx = None if fixed is None else np.ascontiguousarray(fixed, np.uint8)
        self.n_systems = (len(co) - 1) if so is None else len(so) - 1
        xb = np.ascontiguousarray(extra_bonds if extra_bonds is not None else np.zeros((0, 2)), np.int32).reshape(-1, 2)
        topo = Topology(self.n, len(co) - 1, _ptr(co), 0 if so is None else len(so) - 1, _ptr(so), _ptr(fx),
                        len(xb), _ptr(xb) if len(xb) else None)
        p = dict(k_fene=14.0, R0=2.0, eps_h=1.0, native_cut=8.0, eps_l=1.0, sigma=3.8, T=300.0, zeta=50.0, dt=0.1,
                 pair_cut=10.0, rebuild_every=10)
        p.update(params or {})
        sched = SCHEDULES[schedule] if isinstance(schedule, str) else int(schedule)
        prm = Params(p["k_fene"], p["R0"], p["eps_h"], p["native_cut"], p["eps_l"], p["sigma"], p["T"], p["zeta"],
                     p["dt"], p["pair_cut"], int(p["rebuild_every"]), self.R, int(seed), int(obs_every),
                     int(obs_capacity), int(pairs_per_bead), sched, _stream_handle(stream),
                     RNGS[rng] if isinstance(rng, str) else int(rng),
                     INTEGRATORS[integrator] if isinstance(integrator, str) else int(integrator), float(mass),
                     int(obs_every_q))
        self.params = p
        self.obs_every = int(obs_every)
        ctx = C.c_void_p()
        rc = L.sop_create(C.byref(topo), _ptr(xyz), C.byref(prm), C.byref(ctx))
        if rc != OK:
            raise SopError(rc, L.sop_last_error(None).decode())
        self._ctx = ctx

    # -- helpers
    def _check(self, rc):
        if rc != OK:
            raise SopError(rc, self._L.sop_last_error(self._ctx).decode())

    def close(self):
        if getattr(self, "_ctx", None):
            self._L.sop_destroy(self._ctx)
            self._ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- the ABI, one method per entry point
    def step(self, n_steps: int, raise_on_error: bool = True) -> int:
        rc = self._L.sop_step(self._ctx, int(n_steps))
        if raise_on_error:
            self._check(rc)
        return rc

    def get_velocities(self, replica: int = 0):
        """Stored velocities of the underdamped integrator, [n, 3] (or [R, n, 3] for replica -1)."""
        shape = (self.R, self.n, 3) if replica == -1 else (self.n, 3)
        out = np.zeros(shape)
        self._check(self._L.sop_get_velocities(self._ctx, replica, _ptr(out)))
        return out

    def set_velocities(self, v, replica: int = 0):
        a = np.ascontiguousarray(v, np.float64)
        need = (self.R if replica == -1 else 1) * self.n * 3
        if a.size != need:
            raise ValueError(f"expected {need} components, got {a.size}")
        self._check(self._L.sop_set_velocities(self._ctx, replica, _ptr(a)))

    def get_rng_state(self):
        """Hybrid Taus state [R, n, 4] uint32 (contexts created with rng="taus")."""
        out = np.zeros((self.R, self.n, 4), np.uint32)
        self._check(self._L.sop_get_rng_state(self._ctx, _ptr(out), out.size))
        return out

    def set_rng_state(self, state):
        a = np.ascontiguousarray(state, np.uint32)
        if a.size != self.R * self.n * 4:
            raise ValueError(f"expected {self.R * self.n * 4} words, got {a.size}")
        self._check(self._L.sop_set_rng_state(self._ctx, _ptr(a), a.size))

    def forces(self, replica: int = 0):
        """(F [n,3] FP64 from FP32 arithmetic, energy FP64) at the current positions."""
        f = np.zeros((self.n, 3))
        e = C.c_double(0.0)
        self._check(self._L.sop_forces(self._ctx, replica, _ptr(f), C.byref(e)))
        return f, e.value

    def pairlist_rebuild(self):
        self._check(self._L.sop_pairlist_rebuild(self._ctx))

    def pull(self, pulls):
        """pulls: iterable of (system, anchor, pulled, k_s, v)."""
        pulls = list(pulls)
        arr = (PullParams * max(1, len(pulls)))(*[PullParams(int(s), int(a), int(b), float(k), float(v))
                                                   for s, a, b, k, v in pulls])
        self._check(self._L.sop_pull(self._ctx, len(pulls), arr))

    def indenter(self, center, direction, radius: float, v: float):
        c = np.ascontiguousarray(center, np.float64)
        d = np.ascontiguousarray(direction, np.float64)
        self._check(self._L.sop_indenter(self._ctx, _ptr(c), _ptr(d), float(radius), float(v)))

    def get_positions(self, replica: int = 0, out: np.ndarray | None = None) -> np.ndarray:
        shape = (self.R, self.n, 3) if replica == -1 else (self.n, 3)
        if out is None:
            out = np.zeros(shape)
        assert out.dtype == np.float64 and out.flags.c_contiguous and out.size == int(np.prod(shape))
        self._check(self._L.sop_get_positions(self._ctx, replica, _ptr(out)))
        return out

    def set_positions(self, xyz, replica: int = 0):
        a = np.ascontiguousarray(xyz, np.float64)
        need = (self.R if replica == -1 else 1) * self.n * 3
        if a.size != need:
            raise ValueError(f"expected {need} coordinates, got {a.size}")
        self._check(self._L.sop_set_positions(self._ctx, replica, _ptr(a)))

    def get_pairlist(self, replica: int = 0):
        """(row_ptr [n+1], col [nnz]) canonical CSR, both directions."""
        rp = np.zeros(self.n + 1, np.int32)
        nnz = C.c_int64(0)
        rc = self._L.sop_get_pairlist(self._ctx, replica, _ptr(rp), None, 0, C.byref(nnz))
        if rc not in (OK, ERR_CAPACITY):
            self._check(rc)
        col = np.zeros(max(1, nnz.value), np.int32)
        self._check(self._L.sop_get_pairlist(self._ctx, replica, _ptr(rp), _ptr(col), len(col), C.byref(nnz)))
        return rp, col[:nnz.value]

    def get_native_map(self):
        """(row_ptr [n+1], col [nnz], r0 [nnz] FP64), both directions."""
        rp = np.zeros(self.n + 1, np.int32)
        nnz = C.c_int64(0)
        rc = self._L.sop_get_native_map(self._ctx, _ptr(rp), None, None, 0, C.byref(nnz))
        if rc not in (OK, ERR_CAPACITY):
            self._check(rc)
        col = np.zeros(max(1, nnz.value), np.int32)
        r0 = np.zeros(max(1, nnz.value), np.float64)
        self._check(self._L.sop_get_native_map(self._ctx, _ptr(rp), _ptr(col), _ptr(r0), len(col), C.byref(nnz)))
        return rp, col[:nnz.value], r0[:nnz.value]

    def get_observables(self):
        """Structured array of the records taken since the last call, and the count lost."""
        n = C.c_int64(0)
        lost = C.c_int64(0)
        rc = self._L.sop_get_observables(self._ctx, None, 0, C.byref(n), C.byref(lost))
        if rc not in (OK, ERR_CAPACITY):
            self._check(rc)
        buf = (Record * max(1, n.value))()
        self._check(self._L.sop_get_observables(self._ctx, buf, n.value, C.byref(n), C.byref(lost)))
        arr = np.frombuffer(buf, dtype=np.float64).reshape(-1, 8)[:n.value].copy()
        return arr, lost.value

    def get_state(self) -> bytes:
        size = C.c_int64(0)
        self._check(self._L.sop_get_state(self._ctx, None, 0, C.byref(size)))
        buf = (C.c_char * size.value)()
        self._check(self._L.sop_get_state(self._ctx, buf, size.value, C.byref(size)))
        return bytes(buf)

    def set_state(self, state: bytes):
        buf = C.create_string_buffer(state, len(state))
        self._check(self._L.sop_set_state(self._ctx, buf, len(state)))

    def replica_status(self) -> np.ndarray:
        out = np.zeros(self.R, np.int32)
        self._check(self._L.sop_replica_status(self._ctx, _ptr(out)))
        return out

    def abort(self):
        self._L.sop_abort(self._ctx)

    def stats(self) -> dict:
        s = Stats()
        self._check(self._L.sop_get_stats(self._ctx, C.byref(s)))
        return {k: getattr(s, k) for k, _ in Stats._fields_}


def from_workload(w, n_replicas: int | None = None, schedule="auto", stream=None, obs_every=None, **kw) -> Simulation:
    """A Simulation of a synthetic workload (duck-typed: xyz, chain_offsets,
    system_offsets, fixed, params, n_replicas, seed, pulls, indenter, obs_every).
    Pulling and the indenter start at step 0."""
    kw.setdefault("extra_bonds", getattr(w, "extra_bonds", None) or None)
    sim = Simulation(w.xyz, w.chain_offsets, w.system_offsets, w.fixed, w.params,
                     n_replicas=w.n_replicas if n_replicas is None else n_replicas, seed=w.seed,
                     obs_every=w.obs_every if obs_every is None else obs_every, schedule=schedule, stream=stream, **kw)
    if w.pulls:
        sys_of = w.system_of_bead()
        sim.pull([(int(sys_of[p.anchor]), p.anchor, p.pulled, p.k_s, p.v) for p in w.pulls])
    if w.indenter is not None:
        ind = w.indenter
        sim.indenter(ind.center, ind.direction, ind.radius, ind.v)
    return sim


def fp32_peak(seconds: float = 0.5) -> dict:
    """``sop_fp32_peak``: the measured FP32 FMA rate of the current device (TFLOP/s), the
    duration of its last launch (ms) and the SM count."""
    L = load()
    t, ms, sms = C.c_double(0.0), C.c_double(0.0), C.c_int32(0)
    rc = L.sop_fp32_peak(float(seconds), C.byref(t), C.byref(ms), C.byref(sms))
    if rc != OK:
        raise SopError(rc, L.sop_last_error(None).decode())
    return {"tflops": t.value, "ms": ms.value, "sm_count": sms.value}


def box_muller(x, stream=None):
    """``sop_box_muller``: three normals per block of four uint32 words, x [n, 4] -> [n, 3]."""
    L = load()
    a = np.ascontiguousarray(x, np.uint32).reshape(-1, 4)
    out = np.zeros((a.shape[0], 3))
    rc = L.sop_box_muller(_ptr(a), a.shape[0], _ptr(out), _stream_handle(stream))
    if rc != OK:
        raise SopError(rc, L.sop_last_error(None).decode())
    return out


def bead_noise(key: int, step: int, bead_lo: int, n: int, stream=None):
    """``sop_bead_noise``: the normals of beads bead_lo .. bead_lo + n - 1 at `step` for
    the replica keyed by `key`, [n, 3]."""
    L = load()
    out = np.zeros((int(n), 3))
    rc = L.sop_bead_noise(int(key), int(step), int(bead_lo), int(n), _ptr(out), _stream_handle(stream))
    if rc != OK:
        raise SopError(rc, L.sop_last_error(None).decode())
    return out


def brownian_ramp(K, xi, kT, h, r_f, n_runs, n_steps, X0=0.0, order=1, n_out=1, seed=0, x_final=False,
                  stream=None):
    """``sop_brownian_ramp``: the Sec. IV.C experiment on the GPU. Returns (mean [n_out],
    var [n_out]) or, with x_final, (mean, var, X of every run after the last step)."""
    L = load()
    prm = RampParams(float(K), float(xi), float(kT), float(h), float(r_f), float(X0), int(n_runs), int(n_steps),
                     int(order), int(n_out), int(seed))
    mean, var = np.zeros(n_out), np.zeros(n_out)
    xf = np.zeros(int(n_runs)) if x_final else None
    rc = L.sop_brownian_ramp(C.byref(prm), _ptr(mean), _ptr(var), _ptr(xf), _stream_handle(stream))
    if rc != OK:
        raise SopError(rc, L.sop_last_error(None).decode())
    return (mean, var, xf) if x_final else (mean, var)


NOALLOC_MAX_BEADS = 65536


def pairlist_build_noalloc(pos4, n: int, chain, nat_row, nat_col, pair_cut: float, row_start, row_len, col,
                           cap: int, stream=None) -> int:
    """``sop_pairlist_build_noalloc``: the Verlet list of one system from device
    buffers, for callers that cannot allocate device memory (the library's own
    fixed scratch array is used). Every buffer argument is a device pointer
    (int) or an object with ``data_ptr()`` (e.g. a torch CUDA tensor): pos4
    float32 [n, 4]; chain int32 [n]; nat_row int32 [n+1]; nat_col int32;
    outputs row_start, row_len int32 [n] and col int32 [cap]. Returns nnz."""
    L = load()

    def dp(x):
        return int(x) if isinstance(x, int) else int(x.data_ptr())

    nnz = C.c_int64(0)
    rc = L.sop_pairlist_build_noalloc(dp(pos4), int(n), dp(chain), dp(nat_row), dp(nat_col), float(pair_cut),
                                      dp(row_start), dp(row_len), dp(col), int(cap), C.byref(nnz),
                                      _stream_handle(stream))
    if rc != OK:
        raise SopError(rc, L.sop_last_error(None).decode())
    return nnz.value
