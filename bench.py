"""Benchmark: bead-steps/s of the SOP-model Langevin hot path on GB300.

Workload (default): 8,192 independent replicas of one 128-bead compact chain
(seeded synthetic stand-in for the paper's many-runs-per-GPU experiment), run
by the batched persistent kernel. One benchmark step = 1,000 Langevin steps of
every replica: 100 Verlet-list rebuilds, 1,000 force + Philox noise +
compensated-update steps and one FP64 observable record per replica.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line. `value` is device-timed (CUDA events on the library's
stream, inputs resident, L2 flushed between timed steps); by default 100 timed
steps, i.e. the configuration's 1e5 Langevin steps. `e2e` times the same work
through the public API with host buffers (every step uploads the positions it
starts from out of pinned memory and reads back the new positions and the
observable records). `--impl reference` times the
FP64 CPU oracle on the host cores on bounded samples of the same workload.
The same line carries, under "workloads", the other configurations (chain64,
fiber4096, uneven2048, shell60x2500), each timed in this run with its rate, time per
MD step and its HBM and FP32 roofline fractions, and the FP32 peak measured in
this run (sop_fp32_peak).
Under torchrun every rank runs its own 8,192 replicas (weak scaling).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import multiprocessing as mp
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_1003_1148_gb300 import dist  # noqa: E402  (host-only helpers; loads no library)

METRIC = "bead-steps/s on 1 GB300, batched FP32 vs plain per-chain; force err vs FP64"
UNIT = "bead-steps/s"
MD_STEPS_PER_STEP = 1000
FP32_LANES_PER_SM = 128   # FP32 FMA lanes per SM of the Blackwell SM (the derived peak beside the measured one)

# Algorithmic FP32 operations, an FMA counted as 2, each unique interaction once (Newton's
# third law): a FENE bond 20, a native 12-6 pair 25, a listed (sigma/r)^6 pair 20; per bead
# the Box-Muller transform 40 and the update with its compensation 30.
FLOP_FENE, FLOP_NATIVE, FLOP_REP, FLOP_BEAD = 20, 25, 20, 70
FLOP_MODEL = ("20 per bond, 25 per native pair, 20 per listed pair (each unique pair once), 70 per bead "
              "(Box-Muller 40, update and compensation 30); an FMA counts 2")

# The other workloads, timed in the same run after the headline (one line carries them all):
# name -> (MD steps per timed chunk, timed chunks)
SUB_WORKLOADS = {"chain64": (1000, 3), "fiber4096": (1000, 3), "uneven2048": (1000, 2), "shell60x2500": (1000, 2)}


def workload(name: str):
    from paper_1003_1148_gb300 import synth
    if name == "replicas8192x128":
        return synth.replicas(n_replicas=8192, n=128, seed=3, steps=100_000)
    if name == "uneven2048":
        return synth.uneven()
    if name == "fiber4096":
        return synth.fiber4096()
    if name == "shell60x2500":
        return synth.shell()
    if name == "chain64":
        return synth.chain64()
    if name.startswith("replicas"):
        r, n = name[len("replicas"):].split("x")
        return synth.replicas(n_replicas=int(r), n=int(n), seed=3, steps=100_000)
    raise SystemExit(f"unknown workload {name}")


def kernel_revision() -> str:
    """Hash of the batched kernel's sources; a profile summary records the one it measured."""
    h = hashlib.sha256()
    for f in ("k_batched.cu", "sop_device.cuh", "sop_internal.h", "sop_step.cuh"):
        with open(os.path.join(ROOT, "paper_1003_1148_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def measured_hbm_gbs():
    """The measured HBM copy rate of the GB300 (GB/s, MEASURED_PEAKS.json), else 6,800."""
    try:
        return float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"])
    except (OSError, ValueError, KeyError):
        return 6800.0


def recorded_counter(name: str, key: str):
    """A per-launch count recorded in profiles/<name>.md as "<key>: <integer>", or None when
    that capture measured other kernel sources than the ones built now."""
    path = os.path.join(ROOT, "profiles", f"{name}.md")
    if not os.path.exists(path):
        return None
    rev = value = None
    for line in open(path):
        if line.startswith("Kernel source revision:"):
            rev = line.split("`")[1] if "`" in line else None
        elif line.startswith(key + ":"):
            value = int(line.split(":")[1])
    return value if rev == kernel_revision() else None


def recorded_traffic(name: str):
    """DRAM bytes per launch (ncu dram__bytes_read.sum + dram__bytes_write.sum)."""
    return recorded_counter(name, "traffic_bytes_per_launch")


# ----------------------------------------------------------------------------------------
# clocks sampled during the timed region
# ----------------------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for k, nm in enumerate(names):
                if f[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ----------------------------------------------------------------------------------------
# oracle legs (host cores only)
# ----------------------------------------------------------------------------------------
def _oracle_replica(args):
    """Run one replica of the oracle (in a spawned worker); returns bead-steps and seconds."""
    xyz, chain_offsets, seed, n_steps, params = args
    sys.path.insert(0, ROOT)
    import oracle
    n = xyz.shape[0]
    chain = np.zeros(n, np.int32)
    for c in range(len(chain_offsets) - 1):
        chain[chain_offsets[c]:chain_offsets[c + 1]] = c
    m = oracle.Model(xyz, chain, np.zeros(n, np.int32), params=params)
    t0 = time.perf_counter()
    m.run(xyz, n_steps, seed=seed)
    return n * n_steps, time.perf_counter() - t0


def cpu_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def cpu_baseline_leg(w, n_replicas: int, n_steps: int, pool=None):
    """The FP64 oracle as it stands, replicas spread over the host cores.
    Returns (bead-steps/s, cores, sample text)."""
    cores = cpu_cores()
    jobs = [(w.xyz, w.chain_offsets, w.seed + r, n_steps, w.params) for r in range(n_replicas)]
    t0 = time.perf_counter()
    if pool is not None:
        res = pool.map(_oracle_replica, jobs)
    else:
        res = [_oracle_replica(j) for j in jobs]
    wall = time.perf_counter() - t0
    work = sum(r[0] for r in res)
    sample = (f"{n_replicas} replicas x {n_steps} steps x {w.xyz.shape[0]} beads of the same chain "
              f"({work:.3g} bead-steps) on {min(cores, n_replicas)} processes")
    return work / wall, min(cores, n_replicas), sample


def force_error_leg(w, samples):
    """FP32 GPU forces against the FP64 oracle at identical positions (part of the
    CPU-baseline leg: the only place the benchmark calls the oracle besides timing).
    samples: [(replica, positions, gpu forces)]. Reports the gate's measure (per component,
    relative to the term-magnitude scale), the plain relative error per component
    (|dF| / |F64| where |F64| is above 1e-3 of its median) and per bead (|dF_i| / |F64_i|)."""
    import oracle
    n = w.xyz.shape[0]
    m = oracle.Model(w.xyz, np.zeros(n, np.int32), np.zeros(n, np.int32), params=w.params)
    gate = plain_c = plain_b = amax = 0.0
    med = []
    for _, x, F in samples:
        Fo, Ao, _ = m.forces(x, step=0)
        d = np.abs(F - Fo)
        gate = max(gate, float((d / Ao).max()))
        amax = max(amax, float(d.max()))
        a = np.abs(Fo)
        big = a > 1e-3 * np.median(a)
        plain_c = max(plain_c, float((d[big] / a[big]).max()))
        nb = np.linalg.norm(F - Fo, axis=1) / np.maximum(np.linalg.norm(Fo, axis=1), 1e-30)
        plain_b = max(plain_b, float(nb.max()))
        med.append(float(np.median(d / np.maximum(a, 1e-12))))
    return {"max_rel_to_term_scale": gate, "max_abs_kcal_mol_A": amax,
            "max_plain_rel_component": plain_c, "max_plain_rel_per_bead": plain_b,
            "median_rel": float(np.median(med)), "gate": 1e-5,
            "sample": f"replicas {[r for r, _, _ in samples]} after the timed run, all beads, FP64 oracle; "
                      "plain per component over components above 1e-3 of the median |F64|"}


def fp32_peak_leg(sop, local):
    """Measured FP32 FMA rate (sop_fp32_peak, about 0.5 s) with the SM clocks sampled
    during it; the derived peak uses the device's SM count and its maximum SM clock."""
    with ClockSampler(local) as clk:
        pk = sop.fp32_peak(0.5)
    c = clk.summary()
    derived = None
    if c["sm_max_mhz"]:
        derived = pk["sm_count"] * FP32_LANES_PER_SM * 2 * c["sm_max_mhz"] * 1e6 / 1e12
    return {"tflops": pk["tflops"], "sm_count": pk["sm_count"], "sm_mhz_median": c["sm_mhz"],
            "sm_max_mhz": c["sm_max_mhz"], "derived_tflops": derived, "launch_ms": pk["ms"],
            "reasons": c["reasons"]}


def sub_workload_leg(name, sop, torch, stream, flush, fp32_peak):
    """One more workload of the same run: created with the automatic schedule, one chunk of
    warm-up, then `chunks` timed chunks of MD steps (CUDA events on the library's stream,
    L2 flushed between chunks; records read back outside the timed region). Rate, time per
    MD step, and both rooflines from the algorithmic FLOPs and bytes per bead-step."""
    md, chunks = SUB_WORKLOADS[name]
    w = workload(name)
    R = w.n_replicas
    per_chunk = (md // w.obs_every + 1) if w.obs_every else 0
    t0 = time.perf_counter()
    sim = sop.from_workload(w, schedule="auto", stream=stream, obs_capacity=max(4096, 4 * R * w.n_systems * per_chunk))
    create_s = time.perf_counter() - t0
    ms = 0.0
    with torch.cuda.stream(stream):
        sim.step(md)
        sim.get_observables()
        for _ in range(chunks):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            sim.step(md)
            e1.record(stream)
            torch.cuda.synchronize()
            ms += e0.elapsed_time(e1)
            sim.get_observables()
    work = R * w.n_beads * md * chunks
    rate = work / (ms / 1e3)
    flop_bs, counts = algorithmic_flops_per_bead_step(sim, w)
    bps = algorithmic_bytes_per_bead_step(counts, w.n_beads, int(w.params["rebuild_every"]))
    hbm_peak = measured_hbm_gbs()
    st = sim.stats()
    out = {"value": rate, "unit": UNIT, "ms_per_md_step": ms / (md * chunks), "md_steps_timed": md * chunks,
           "beads": R * w.n_beads, "systems": R * w.n_systems, "schedule": schedule_name(sop, st),
           "create_s": create_s, "failed_replicas": int(np.count_nonzero(sim.replica_status())),
           "roofline": {"hbm": {"achieved_gbs": bps * rate / 1e9, "peak_gbs": hbm_peak,
                                "frac": bps * rate / 1e9 / hbm_peak, "bytes_per_bead_step": bps},
                        "alu": {"achieved_tflops": flop_bs * rate / 1e12, "peak_tflops": fp32_peak,
                                "frac": flop_bs * rate / 1e12 / fp32_peak if fp32_peak else None,
                                "flop_per_bead_step": flop_bs},
                        "list_sizes_replica0": counts}}
    sim.close()
    return out


def schedule_name(sop, st):
    names = {sop.SCHED_BATCHED: "batched", sop.SCHED_STREAMED: "streamed", sop.SCHED_PAIRS: "pairs",
             sop.SCHED_PLAIN: "plain"}
    nm = names.get(st["schedule"], str(st["schedule"]))
    if st["schedule"] == sop.SCHED_BATCHED and st.get("pair_buckets"):
        nm += f" ({st['pair_buckets']} of {st['buckets']} buckets in the pair form)"
    if st["schedule"] == sop.SCHED_BATCHED and st.get("cluster_buckets"):
        nm += f" ({st['cluster_buckets']} of {st['buckets']} buckets in the cluster form)"
    return nm


# ----------------------------------------------------------------------------------------
# arms
# ----------------------------------------------------------------------------------------
def run_reference(args):
    world, rank, _ = dist.rank_env()
    if rank != 0:
        return 0
    w = workload(args.workload)
    ctx = mp.get_context("spawn")
    per_step_reps = max(1, min(cpu_cores(), 32))
    with ctx.Pool(cpu_cores()) as pool:
        for _ in range(args.warmup):
            cpu_baseline_leg(w, per_step_reps, 100, pool)
        t0 = time.perf_counter()
        work = 0.0
        for _ in range(args.steps):
            rate, cores, sample = cpu_baseline_leg(w, per_step_reps, 100, pool)
            work += per_step_reps * 100 * w.xyz.shape[0]
        wall = time.perf_counter() - t0
    value = work / wall
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * wall / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded compact self-avoiding walk; PDB inputs unavailable)",
            "config": config_dict(args, w),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"each step: {sample}"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def config_dict(args, w):
    return {"workload": args.workload, "replicas_per_gpu": w.n_replicas, "beads_per_replica": w.n_beads,
            "md_steps_per_step": MD_STEPS_PER_STEP, "rebuild_every": w.params["rebuild_every"],
            "obs_every": w.obs_every, "dt_ps": w.params["dt"], "T_K": w.params["T"],
            "pair_cut_A": w.params["pair_cut"], "schedule": args.schedule,
            "l2": "flushed between timed steps (256 MiB write)", "parallelism": f"replicas x{args.gpus}"}


def algorithmic_flops_per_bead_step(sim, w) -> tuple[float, dict]:
    rp, col = sim.get_pairlist(0)
    n_pl = len(col) / 2.0
    n_nat = sim.stats()["native_entries"]
    n_bonds = w.n_beads - w.n_chains
    f = (FLOP_FENE * n_bonds + FLOP_NATIVE * n_nat + FLOP_REP * n_pl) / w.n_beads + FLOP_BEAD
    return f, {"bonds": n_bonds, "native_pairs": int(n_nat), "verlet_pairs": int(n_pl)}


def algorithmic_bytes_per_bead_step(counts: dict, n_beads: int, K: int) -> float:
    """Bytes a bead-step of the streamed form moves at least once: position read and
    write, compensation read and write, Verlet columns, native columns with r0^2, bond
    lengths, row pointers, and the rebuild (positions, cell id, sorted id, column writes)
    amortised over the K steps between rebuilds."""
    v = 2.0 * counts["verlet_pairs"] / n_beads
    m = 2.0 * counts["native_pairs"] / n_beads
    return 16 + 16 + 32 + 4 * v + 8 * m + 8 + 12 + (16 + 4 + 8 + 4 * v) / K


def run_ours(args):
    import torch
    from paper_1003_1148_gb300 import sop

    world, rank, local = dist.rank_env()
    group = dist.init(world)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    w = workload(args.workload)
    R = w.n_replicas

    # the CPU baseline runs first, from spawned workers, before any GPU work
    cpu = None
    if rank == 0 and not args.no_cpu:
        ctx = mp.get_context("spawn")
        n_rep = max(2, min(cpu_cores(), 64))
        with ctx.Pool(cpu_cores()) as pool:
            probe_rate, _, _ = cpu_baseline_leg(w, min(n_rep, cpu_cores()), 200, pool)
            # size the sample to about 15 s of CPU work
            steps = int(max(200, min(5000, 15.0 * probe_rate / (n_rep * w.n_beads))))
            rate, cores, sample = cpu_baseline_leg(w, n_rep, steps, pool)
        # one core, one replica at a time (the form of the paper's CPU comparison), about 3 s
        one_steps = int(max(50, min(50000, 3.0 * probe_rate / max(1, min(n_rep, cpu_cores())) / w.n_beads)))
        work1, t1 = _oracle_replica((w.xyz, w.chain_offsets, w.seed, one_steps, w.params))
        cpu = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample,
               "single_core": {"value": work1 / t1, "unit": UNIT, "cores": 1,
                               "sample": f"1 replica x {one_steps} steps x {w.xyz.shape[0]} beads in one process"}}

    stream = torch.cuda.Stream(device=dev)
    first, _ = dist.replica_range(rank, world, per_rank=R)
    w.seed = w.seed + first                 # replica r of the job draws Philox key seed + r
    sim = sop.from_workload(w, schedule=args.schedule, stream=stream, obs_capacity=max(4096, 4 * R * w.n_systems))
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    work_per_step = R * w.n_beads * MD_STEPS_PER_STEP
    n_chains = w.n_chains

    def one_step():
        sim.step(MD_STEPS_PER_STEP)

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            one_step()
            sim.get_observables()
        torch.cuda.synchronize()
        launches0 = sim.stats()["kernel_launches"]
        starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        dist.barrier(group)
        torch.cuda.synchronize()
        with ClockSampler(local) as clk:
            # one more untimed step while the sampler starts up (its start can stall the
            # launches for tens of milliseconds), so that the timed steps do not carry it
            one_step()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for k in range(args.steps):
                flush.zero_()                      # L2 flush, outside the timed events
                starts[k].record(stream)
                one_step()
                ends[k].record(stream)
            torch.cuda.synchronize()
            wall = time.perf_counter() - t0
        dist.barrier(group)
        launches = sim.stats()["kernel_launches"] - launches0
        dev_ms = sum(s.elapsed_time(e) for s, e in zip(starts, ends))
        sim.get_observables()

        # end to end through the public API with host buffers: every step uploads the
        # state it starts from (positions, pinned host memory), steps, and reads back its
        # result (the new positions and the observable records)
        pinned = torch.empty((R, w.n_beads, 3), dtype=torch.float64, pin_memory=True)
        pinned.numpy()[:] = sim.get_positions(-1)
        torch.cuda.synchronize()
        e2e_steps = max(1, min(args.steps, 5))
        t1 = time.perf_counter()
        d2h = 0
        for _ in range(e2e_steps):
            sim.set_positions(pinned.numpy(), replica=-1)
            one_step()
            sim.get_positions(-1, out=pinned.numpy())
            rec, lost = sim.get_observables()
            d2h = pinned.numpy().nbytes + rec.nbytes
        e2e_wall = time.perf_counter() - t1
    h2d = R * w.n_beads * 3 * 8

    t_dev = dist.max_over_ranks(group, dev_ms / 1e3)
    t_e2e = dist.max_over_ranks(group, e2e_wall)
    value = world * work_per_step * args.steps / t_dev
    e2e_value = world * work_per_step * e2e_steps / t_e2e

    if rank != 0:
        sim.close()
        return 0

    # roofline of the dominant kernel (the batched persistent kernel; one launch per step)
    flop_bs, counts = algorithmic_flops_per_bead_step(sim, w)
    clocks = clk.summary()
    fpk = fp32_peak_leg(sop, local)
    peak = fpk["tflops"]
    per_launch_s = dev_ms / 1e3 / args.steps
    achieved = flop_bs * work_per_step / per_launch_s / 1e12
    st = sim.stats()
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "peak_measured": peak, "peak_derived": fpk["derived_tflops"], "sm_count": fpk["sm_count"],
                "sm_mhz_median": fpk["sm_mhz_median"], "fp32_peak_clock_reasons": fpk["reasons"],
                "frac_of_derived": achieved / fpk["derived_tflops"] if fpk["derived_tflops"] else None,
                "flop_model": FLOP_MODEL,
                "traffic": None, "kernel": {
                    sop.SCHED_BATCHED: "k_batched (one launch of 1,000 steps per benchmark step)",
                    sop.SCHED_STREAMED: "k_step (one launch per step, CUDA-graph replay) and the cell rebuild",
                    sop.SCHED_PAIRS: "k_pairs + k_pairs_step (two launches per step) and the cell rebuild"}.get(
                        st["schedule"], "per-step kernels"),
                "kernel_config": {"schedule": schedule_name(sop, st),
                                  "threads": st["block_threads"], "beads_per_thread": st["beads_per_thread"],
                                  "register_cap": 65536 // (256 * st["min_blocks"]) if st["min_blocks"] else 64,
                                  "size_buckets": st["buckets"],
                                  "verlet_capacity": st["pairs_per_bead"]},
                "flop_per_bead_step": flop_bs, "list_sizes_replica0": counts,
                "peak_note": "peak: sop_fp32_peak measured in this run (independent FMA chains, about 0.5 s, "
                             "sm_mhz_median the SM clock sampled during it); peak_derived: SMs x 128 FP32 "
                             "lanes x 2 x the maximum SM clock"}
    if st["schedule"] in (sop.SCHED_STREAMED, sop.SCHED_PAIRS):
        # the streamed step against the HBM roofline: its algorithmic bytes at the whole-step rate
        hbm_peak = measured_hbm_gbs()
        bps = algorithmic_bytes_per_bead_step(counts, w.n_beads, int(w.params["rebuild_every"]))
        gbs = bps * work_per_step / per_launch_s / 1e9
        roofline["hbm"] = {"achieved_gbs": gbs, "peak_gbs": hbm_peak, "frac": gbs / hbm_peak,
                           "bytes_per_bead_step": bps,
                           "source": "algorithmic bytes per bead-step x the whole-step rate (all kernels of the step)"}
    roofline["traffic"] = (recorded_traffic("k_batched_replicas8192x128")
                           if args.workload == "replicas8192x128" and st["schedule"] == sop.SCHED_BATCHED else None)
    if roofline["traffic"] is not None:
        # the same launch against the HBM roofline: its measured DRAM bytes over its duration
        hbm_peak = measured_hbm_gbs()
        gbs = roofline["traffic"] / per_launch_s / 1e9
        roofline["hbm"] = {"achieved_gbs": gbs, "peak_gbs": hbm_peak, "frac": gbs / hbm_peak if hbm_peak else None,
                           "source": "ncu DRAM bytes per launch / CUDA-event launch time; peak of measured copy"}
        # ...and against the instruction-issue rate, its actual bound: the warp instructions of
        # the same capture over the launch time, against one warp instruction per cycle per
        # scheduler (4 per SM) at the SM clock sampled during the timed region
        inst = recorded_counter("k_batched_replicas8192x128", "warp_instructions_per_launch")
        if inst is not None and clocks["sm_mhz"] and fpk["sm_count"]:
            rate = inst / per_launch_s / 1e12
            peak_issue = fpk["sm_count"] * 4 * clocks["sm_mhz"] * 1e6 / 1e12
            roofline["issue"] = {"achieved_twips": rate, "peak_twips": peak_issue, "frac": rate / peak_issue,
                                 "warp_instructions_per_launch": inst,
                                 "source": "ncu smsp__inst_executed.sum per launch / CUDA-event launch time; "
                                           "peak = SMs x 4 schedulers x sampled SM clock (tera warp instructions/s)"}

    # plain per-chain GPU form on a subset of replicas (same kernels' math, one chain per launch)
    plain = None
    if not args.no_plain:
        n_plain, s_plain = 4, 200
        ps = sop.Simulation(w.xyz, w.chain_offsets, w.system_offsets, w.fixed, w.params, n_replicas=n_plain,
                            seed=w.seed, schedule="plain", stream=stream)
        with torch.cuda.stream(stream):
            ps.step(20)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ps.step(s_plain)
            e1.record(stream)
            torch.cuda.synchronize()
        pv = n_plain * w.n_beads * s_plain / (e0.elapsed_time(e1) / 1e3)
        pflop, pcounts = algorithmic_flops_per_bead_step(ps, w)
        pbytes = algorithmic_bytes_per_bead_step(pcounts, w.n_beads, int(w.params["rebuild_every"]))
        hbm_peak = measured_hbm_gbs()
        plain = {"value": pv, "unit": UNIT, "sample": f"{n_plain} replicas x {s_plain} steps, one chain per "
                 "launch sequence (per-step fused kernel, cell-list rebuild every 10 steps), chains in sequence",
                 "ms_per_md_step": e0.elapsed_time(e1) / s_plain,
                 "batched_over_plain": value / world / pv,
                 "roofline": {"hbm": {"achieved_gbs": pbytes * pv / 1e9, "peak_gbs": hbm_peak,
                                      "frac": pbytes * pv / 1e9 / hbm_peak, "bytes_per_bead_step": pbytes},
                              "alu": {"achieved_tflops": pflop * pv / 1e12, "peak_tflops": peak,
                                      "frac": pflop * pv / 1e12 / peak, "flop_per_bead_step": pflop},
                              "bound": "launch latency (one chain per launch sequence)"}}
        ps.close()

    ferr = None
    if not args.no_cpu:
        samples = []
        for r in sorted({0, R // 3, (2 * R) // 3, R - 1}):
            F, _ = sim.forces(r)
            samples.append((r, sim.get_positions(r), F))
        ferr = force_error_leg(w, samples)

    # the other workloads of the configuration list, each timed in this run
    subs = None
    if world == 1 and not args.no_workloads:
        subs = {}
        for name in SUB_WORKLOADS:
            if name == args.workload:
                continue
            subs[name] = sub_workload_leg(name, sop, torch, stream, flush, peak)

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": dev_ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded compact self-avoiding walk; "
            "PDB inputs unavailable)", "config": config_dict(args, w),
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                    "steps": e2e_steps},
            "gpu_launches": launches, "wall_s_timed_region": wall,
            "clocks": {"sm_mhz": clocks["sm_mhz"], "sm_max_mhz": clocks["sm_max_mhz"], "reasons": clocks["reasons"]},
            "roofline": roofline, "cpu_baseline": cpu, "plain_per_chain": plain, "force_err_vs_fp64": ferr,
            "workloads": subs,
            "replicas_failed": int(np.count_nonzero(sim.replica_status()))}
    print(json.dumps(line))
    sim.close()
    return 0


def main():
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="replicas8192x128")
    ap.add_argument("--schedule", default="auto", choices=["batched", "streamed", "pairs", "auto", "batched_pairs"])
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle legs (profiling runs)")
    ap.add_argument("--no-plain", action="store_true", help="skip the plain per-chain comparison")
    ap.add_argument("--no-workloads", action="store_true", help="skip the other workloads (profiling runs)")
    args = ap.parse_args()
    if args.warmup < 3:
        raise SystemExit("--warmup must be >= 3")
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
