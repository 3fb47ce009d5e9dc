"""Seeded synthetic workloads for the SOP-model Langevin path.

The paper benchmarks Calpha models of PDB structures (Table I: WW domain up to
the HK97 capsid). Those structures are not available, so every workload here
is built from seeded compact self-avoiding walks (``saw.c``) whose shapes and
sizes follow the paper's systems: small single proteins, a long fiber-like
chain, many replicas of one small protein, an uneven batch of proteins between
50 and 2,000 residues, and a spherical shell assembly of 150,000 beads.

This module only makes inputs (coordinates, chain and system layout, fixed
beads, pulling and indenter set-up, run lengths). It computes no part of the
simulation method, and both the CUDA path and the oracle take its output.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "saw.c")
_OUT_DIR = os.path.join(os.path.dirname(_HERE), "_lib")
_SO = os.path.join(_OUT_DIR, "libsynth.so")
_lock = threading.Lock()
_handle = None

BOND = 3.8          # A, Calpha-Calpha virtual bond length
MIN_DIST = 4.0      # A, closest approach of non-bonded beads in the walk
VOL_PER_BEAD = 110.0  # A^3 per residue, sets the confinement size


def build(force: bool = False) -> str:
    """Compile ``saw.c`` into ``_lib/libsynth.so`` (gcc, no fast-math, no FMA contraction)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math",
                               "-std=c11", "-D_DEFAULT_SOURCE", "-o", tmp, _SRC, "-lm", "-lpthread"])
        os.replace(tmp, _SO)
    return _SO


def _lib():
    global _handle
    with _lock:
        if _handle is None:
            build()
            h = ctypes.CDLL(_SO)
            h.synth_walk.argtypes = [ctypes.c_int32, ctypes.c_uint64, ctypes.c_int32, ctypes.c_double,
                                     ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_void_p]
            h.synth_walk.restype = ctypes.c_int
            h.synth_shell.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_uint64, ctypes.c_double,
                                      ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_void_p]
            h.synth_shell.restype = ctypes.c_int
            h.synth_walk_many.argtypes = [ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                          ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_int32,
                                          ctypes.c_void_p]
            h.synth_walk_many.restype = ctypes.c_int
            _handle = h
    return _handle


def sphere_radius(n: int, v: float = VOL_PER_BEAD) -> float:
    """Radius of the sphere that holds n beads at v A^3 each."""
    return (3.0 * n * v / (4.0 * math.pi)) ** (1.0 / 3.0)


def compact_chain(n: int, seed: int, shape: str = "sphere", radius: float | None = None,
                  v: float = VOL_PER_BEAD) -> np.ndarray:
    """Coordinates [n, 3] (float64, A) of one compact self-avoiding walk.

    shape="sphere": confined to the sphere of volume n*v (radius given or derived).
    shape="cylinder": confined to a cylinder of the given radius (default 25 A)
    whose length holds n*v.
    """
    xyz = np.zeros((n, 3), dtype=np.float64)
    if shape == "sphere":
        kind, a, b = 0, radius if radius is not None else sphere_radius(n, v), 0.0
    elif shape == "cylinder":
        a = radius if radius is not None else 25.0
        kind, b = 1, 0.5 * n * v / (math.pi * a * a)
    else:
        raise ValueError(f"unknown shape {shape!r}")
    rc = _lib().synth_walk(n, seed, kind, a, b, BOND, MIN_DIST, xyz.ctypes.data)
    if rc < 0:
        raise RuntimeError(f"self-avoiding walk failed (n={n}, seed={seed}, shape={shape})")
    return xyz


def shell_assembly(n_copies: int, n_per: int, seed: int, r_in: float, r_out: float) -> np.ndarray:
    """Coordinates [n_copies*n_per, 3] of chains grown in the angular cells of a shell."""
    xyz = np.zeros((n_copies * n_per, 3), dtype=np.float64)
    rc = _lib().synth_shell(n_copies, n_per, seed, r_in, r_out, BOND, MIN_DIST, xyz.ctypes.data)
    if rc < 0:
        raise RuntimeError("shell assembly walk failed")
    return xyz


def uneven_sizes(n_chains: int, lo: int, hi: int, seed: int) -> np.ndarray:
    """Chain sizes round(exp(U[ln lo, ln hi])) (log-uniform), seeded."""
    rng = np.random.default_rng(seed)
    s = np.rint(np.exp(rng.uniform(math.log(lo), math.log(hi), size=n_chains))).astype(np.int64)
    return np.clip(s, lo, hi)


# --------------------------------------------------------------------------
# Workloads
# --------------------------------------------------------------------------
@dataclass
class Pull:
    """Constant-velocity cantilever on one system: `anchor` is held fixed and a
    spring of stiffness k_s (kcal/mol/A^2) drags `pulled` at v (A/step) along the
    anchor->pulled direction at the start of pulling. Bead indices are global."""
    anchor: int
    pulled: int
    k_s: float
    v: float


@dataclass
class Indenter:
    """Repulsive sphere of radius `radius` (A) whose centre starts at `center`
    and moves along the unit vector `direction` at v (A/step)."""
    center: tuple
    direction: tuple
    radius: float
    v: float


@dataclass
class Workload:
    name: str
    xyz: np.ndarray                 # [n, 3] float64 native (and starting) coordinates, one replica
    chain_offsets: np.ndarray       # [n_chains + 1] int32, chains are contiguous bead ranges
    system_offsets: np.ndarray      # [n_systems + 1] int32, in chains; beads interact only within a system
    fixed: np.ndarray               # [n] uint8, 1 = held fixed
    n_replicas: int
    steps: int
    seed: int                       # Philox key of replica r is seed + r
    params: dict = field(default_factory=dict)
    pulls: list = field(default_factory=list)   # list[Pull], at most one per system
    indenter: Indenter | None = None
    obs_every: int = 0
    extra_bonds: list = field(default_factory=list)   # cross-links (i, j): more FENE bonds of Eq. 1

    @property
    def n_beads(self) -> int:
        return int(self.xyz.shape[0])

    @property
    def n_chains(self) -> int:
        return len(self.chain_offsets) - 1

    @property
    def n_systems(self) -> int:
        return len(self.system_offsets) - 1

    def chain_of_bead(self) -> np.ndarray:
        out = np.zeros(self.n_beads, dtype=np.int32)
        for c in range(self.n_chains):
            out[self.chain_offsets[c]:self.chain_offsets[c + 1]] = c
        return out

    def system_of_bead(self) -> np.ndarray:
        chain_sys = np.zeros(self.n_chains, dtype=np.int32)
        for s in range(self.n_systems):
            chain_sys[self.system_offsets[s]:self.system_offsets[s + 1]] = s
        return chain_sys[self.chain_of_bead()]


def default_params(**over) -> dict:
    """The physical parameters shared by all workloads (A, kcal/mol, ps, K)."""
    p = dict(k_fene=14.0, R0=2.0, eps_h=1.0, native_cut=8.0, eps_l=1.0, sigma=3.8, T=300.0,
             zeta=50.0, dt=0.1, pair_cut=10.0, rebuild_every=10)
    p.update(over)
    return p


def _single_chain_layout(n: int):
    return np.array([0, n], dtype=np.int32), np.array([0, 1], dtype=np.int32)


def chain64(seed: int = 1) -> Workload:
    """One compact chain of 64 beads (a small protein like WW or Ig27)."""
    xyz = compact_chain(64, seed)
    co, so = _single_chain_layout(64)
    return Workload("chain64", xyz, co, so, np.zeros(64, np.uint8), 1, 1000, 0, default_params(), obs_every=100)


def fiber4096(seed: int = 2, n: int = 4096, steps: int = 100_000) -> Workload:
    """One long fiber-like chain, N-terminus fixed, C-terminus pulled at 0.01 A/step."""
    xyz = compact_chain(n, seed, shape="cylinder", radius=25.0)
    co, so = _single_chain_layout(n)
    fixed = np.zeros(n, np.uint8)
    fixed[0] = 1
    return Workload("fiber4096", xyz, co, so, fixed, 1, steps, 0, default_params(),
                    pulls=[Pull(0, n - 1, 0.05, 0.01)], obs_every=100)


def replicas(n_replicas: int = 8192, n: int = 128, seed: int = 3, steps: int = 100_000) -> Workload:
    """Many independent trajectories of one small chain; replica r uses Philox key r."""
    xyz = compact_chain(n, seed)
    co, so = _single_chain_layout(n)
    return Workload(f"replicas{n_replicas}x{n}", xyz, co, so, np.zeros(n, np.uint8), n_replicas, steps, 0,
                    default_params(), obs_every=1000)


def uneven(n_chains: int = 2048, lo: int = 50, hi: int = 2000, seed: int = 4, steps: int = 100_000,
           pull_v: float = 0.005) -> Workload:
    """Independent chains of log-uniform size, each its own system, each pulled by its C-terminus."""
    sizes = uneven_sizes(n_chains, lo, hi, seed)
    offs = np.zeros(n_chains + 1, dtype=np.int64)
    offs[1:] = np.cumsum(sizes)
    xyz = np.zeros((int(offs[-1]), 3))
    sizes32 = np.ascontiguousarray(sizes, dtype=np.int32)
    seeds = np.array([seed * 1_000_003 + c for c in range(n_chains)], dtype=np.uint64)
    offs64 = np.ascontiguousarray(offs[:-1], dtype=np.int64)
    rc = _lib().synth_walk_many(n_chains, sizes32.ctypes.data, seeds.ctypes.data, offs64.ctypes.data,
                                VOL_PER_BEAD, BOND, MIN_DIST, os.cpu_count() or 1, xyz.ctypes.data)
    if rc != 0:
        raise RuntimeError("uneven batch walk failed")
    fixed = np.zeros(int(offs[-1]), np.uint8)
    fixed[offs[:-1]] = 1
    pulls = [Pull(int(offs[c]), int(offs[c + 1] - 1), 0.05, pull_v) for c in range(n_chains)]
    return Workload(f"uneven{n_chains}", xyz, offs.astype(np.int32), np.arange(n_chains + 1, dtype=np.int32),
                    fixed, 1, steps, 0, default_params(), pulls=pulls, obs_every=100)


def shell(n_copies: int = 60, n_per: int = 2500, seed: int = 5, steps: int = 20_000,
          r_in: float = 237.0, r_out: float = 263.0, ind_radius: float = 50.0, ind_v: float = 0.005) -> Workload:
    """A spherical shell assembly indented from +z by a repulsive sphere; the
    beads within 10 A of the bottom of the shell are held fixed (substrate)."""
    xyz = shell_assembly(n_copies, n_per, seed, r_in, r_out)
    co = (np.arange(n_copies + 1) * n_per).astype(np.int32)
    so = np.array([0, n_copies], dtype=np.int32)
    fixed = (xyz[:, 2] < -r_out + 10.0).astype(np.uint8)
    ind = Indenter(center=(0.0, 0.0, r_out + ind_radius + 10.0), direction=(0.0, 0.0, -1.0),
                   radius=ind_radius, v=ind_v)
    return Workload(f"shell{n_copies}x{n_per}", xyz, co, so, fixed, 1, steps, 0,
                    default_params(rebuild_every=20), indenter=ind, obs_every=100)
