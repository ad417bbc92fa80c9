"""Benchmark of one timestep of the bonded-particle magneto-elastic rod model
on GB300, through the C ABI of include/bpm.h.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME]
                    [--impl reference]

A step is one pass of the whole hot path: bond forces/torques + Zeeman +
dipole orientation + all-pairs dipole-dipole + velocity Verlet / Richardson
update.  Default workload: the 16384-particle writhing helix in FP64 (268M
ordered dipole pairs per step).  The L2 cache (129 MB) is flushed by a
256 MiB write before every timed step (the workload itself fits in L2).

Under torchrun (N > 1) every rank runs an independent replica of the workload
(the single-rod workload has no partition without a collective); the time is
the maximum over ranks and `value` counts the particle-steps of all ranks.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2603_27279_gb300 import workloads as W  # noqa: E402

METRIC = "particle-steps/s and dipole pair-interactions/s vs FP64 plain on 1 GB300; % roofline"
UNIT = "particle-steps/s"

# The unit of dipole work, fixed once from the pair expression of the first
# kernels (bpm_dipole.cu) and kept as the algorithmic count whatever the
# current kernel's instruction count (the FP64 kernel now needs fewer): FP64
# operations of one ordered pair, FMA counted as 2: r (3), r^2 (5), 1/r as
# two Newton steps (12; FP32 path: 1 MUFU, counted 0), powers (3), a, b, d
# (15), s (4), A, S (2), force sums (12), b/r^5 and its sum (2), 3 b/r^5 (1),
# field sums (12).
FLOPS_PER_PAIR_FP64 = 71
FLOPS_PER_PAIR_FP32 = 65  # no Newton steps (one MUFU rsqrt); the hi/lo difference adds 6 adds
# The symmetric kernel (pair_sym) evaluates each unordered pair once: the
# 71 flops above plus the j-side terms, 6 FMA for F~_j, 1 mul + 6 FMA for
# H~_j and 1 add for Bs_j (26 flops) = 97 per unordered pair, i.e. 48.5 per
# ordered pair (the ordered pairs inside diagonal tiles, under 1 % of the
# pairs for N >= 16384, are counted at the same rate).
FLOPS_PER_PAIR_SYM_FP64 = 97 / 2
# the same j-side terms on the FP32 pair (pair_mix): 65 + 26 = 91 per
# unordered pair
FLOPS_PER_PAIR_SYM_FP32 = 91 / 2
# The float-float kernel (bpm_dipole_ff.cu, pair_ff with both sides) per
# unordered pair, counted from the source: FP32-pipe operations (add, mul and
# fma each one): r 21, r^2 28, 1/r 15 (+1 MUFU), powers 12, the three dot
# products 84, 5ab/r^2 and d - it 25, A, S, b/r^5 12, i-side sums 152
# (9 product accumulations of 12 operations, the shared product S r 3 x 4,
# two sums of 8 per component and Bs), j-side sums 140, renormalisation of
# the 20 accumulators every fourth pair 15 = 504; the same with FMA counted
# as 2 flops (128 FMA) = 632.
FF_PIPE_OPS_PER_PAIR = 504
FF_FLOPS_PER_PAIR = 632
# The packed FP32-pair kernels, FP32-pipe lane operations per pair counted
# from the source (one f32x2 add, mul or fma is one operation on each of its
# two pairs; one MUFU rsqrt besides): r from hi and lo differences 9, r^2 3,
# powers 3, a, b, d 9, s 3, A, S 2, force sums 6, b/r^5, its sum and 3 b/r^5
# 3, field sums 6 = 44 per ordered pair (pair_fp32x2); the symmetric kernel
# adds the j side, force 6, 3 A 1, field 6, Bs 1 = 58 per unordered pair
# (pair_mix2).
MIX_PIPE_OPS_PER_PAIR = 44
MIX_SYM_PIPE_OPS_PER_PAIR = 58
# DFMA lanes per SM per clock on GB300 (measured: 1.9 per SM per clock at the
# maximum clock with an 8-way independent DFMA chain), FP32 FMA lanes per SM.
FP64_FMA_PER_SM_CLK = 2
FP32_FMA_PER_SM_CLK = 128
L2_FLUSH_BYTES = 256 << 20

# DRAM bytes (read + write) per launch of the dominant kernel, from one ncu
# capture of the same kernel build on the same workload
# (profiles/k_dipole_sym_fp64_helix_16384.md): dram__bytes_read.sum
# 1.807616 MB + dram__bytes_write.sum 62.122752 MB.  An entry must be removed
# when its kernel changes.
NCU_TRAFFIC = {("helix_16384", "k_dipole_sym_fp64"): 63.930368e6}

def _helix_contact():
    s = W.helix()
    s.contact = W.ContactParams(E=1e4, nu=0.3, mu=0.5, gamma_n=0.1, gamma_t=0.05, exclude=3)
    return s


def _helix_damped():
    s = W.helix()
    # per-mode bond damping at about a tenth of each mode's critical value
    s.bond_damping = np.array([[5.0, 2.0, 0.05, 0.05]])
    return s


WORKLOADS = {
    "helix_16384": lambda: W.helix(),
    "helix_16384_contact": _helix_contact,
    "helix_16384_damped": _helix_damped,
    "granular_128": lambda: W.granular(128, 128, 128),
    "fluid_cilia": lambda: W.fluid_cilia(),
    "fluid_cilia_mixed": lambda: W.fluid_cilia(precision=W.PRECISION_MIXED),
    "fluid_cilia_ff": lambda: W.fluid_cilia(precision=W.PRECISION_FF),
    "fluid_cilia_128": lambda: W.fluid_cilia(8, 8, 64, lattice=(128, 128, 128)),
    "fluid_cilia_128_mixed": lambda: W.fluid_cilia(8, 8, 64, lattice=(128, 128, 128), precision=W.PRECISION_MIXED),
    "fluid_cilia_128_ff": lambda: W.fluid_cilia(8, 8, 64, lattice=(128, 128, 128), precision=W.PRECISION_FF),
    "granular_64": lambda: W.granular(64, 64, 64),
    "helix_16384_mixed": lambda: W.helix(precision=W.PRECISION_MIXED),
    "helix_16384_ff": lambda: W.helix(precision=W.PRECISION_FF),
    "cilia_512x256_ff": lambda: W.cilia(precision=W.PRECISION_FF),
    "cilia_512x256_fp64": lambda: W.cilia(precision=W.PRECISION_FP64),
    "batched_rods_2048_ff": lambda: W.batched_rods(precision=W.PRECISION_FF),
    "batched_rods_2048_fp64": lambda: W.batched_rods(precision=W.PRECISION_FP64),
    "straight_rod_64": lambda: W.straight_rod(),
    "batched_rods_2048": lambda: W.batched_rods(),
    "cilia_512x256": lambda: W.cilia(),
    "adjoint_rod_2048": lambda: W.adjoint_rod(),
}


# Algorithmic bytes of the contact pass per particle (cell list + pair
# kernel), c = contacts per particle: own x, v, w, radius, rod index read
# (84); f, t read and written (96); history counts read and written (8);
# per contact the partner index and xi read from one level and written to the
# other (2 x 28); cell list: bucket key and order written, bucket counts and
# starts at H/N = 2 buckets per particle read and written (40).  Neighbour
# reads are counted once, in the own-particle term.
CONTACT_BYTES_FIXED = 84 + 96 + 8 + 40
CONTACT_BYTES_PER_CONTACT = 56


def contacts_per_particle(sysm) -> float:
    """Mean number of overlapping, non-excluded partners (host-side count for
    the byte model; a k-d tree query)."""
    from scipy.spatial import cKDTree
    x, R = sysm.x, sysm.radius
    pairs = cKDTree(x).query_pairs(r=2.0 * float(R.max()), output_type="ndarray")
    if len(pairs) == 0:
        return 0.0
    i, j = pairs[:, 0], pairs[:, 1]
    d = np.linalg.norm(x[i] - x[j], axis=1)
    hit = d < R[i] + R[j]
    rod = np.repeat(np.arange(sysm.n_rods), np.diff(sysm.rod_offset))
    excl = (rod[i] == rod[j]) & (np.abs(i - j) <= sysm.contact.exclude)
    return 2.0 * float(np.count_nonzero(hit & ~excl)) / sysm.n


# FP64 flops of one contact evaluation in k_contact phase B, from the
# source, FMA = 2: d (3), |d|^2 (5), R_i + R_j and its square (2), refined
# 1/|d| (12), delta (2), n (3), R* delta with a refined reciprocal (11),
# contact radius with a refined rsqrt (13), Hertz force (3), R_i w_i + R_j w_j
# (9), its cross product with n (9), v_rel (6), v_n (5), v_t (6), history
# carried into the tangent plane (50), xi update (6), k_t (2), F_t (9),
# Coulomb test (7), force sum (11), torque sum (15) = 189.  Every contact is
# evaluated from both particles; steady contacts have a stored history.
CONTACT_FLOPS_PER_EVAL = 189


# One LBM node update in k_lbm_step, from the source (FMA = 2): moments 48,
# forces 3, refined reciprocal of rho 8, half-step velocity 9, u.u and u.F
# 10, the direction-independent term K 7, omega rho 1, the per-class factors
# A, B, C, G, H (3 x 5 = 15), the rest direction 2, e.u and e.F of the 12
# edge directions 24, and five fused multiply-adds per moving direction
# (18 x 10 = 180) = 307 flops.  Bytes per node update: 19 distributions read
# and written and the 3-component reaction field read and zeroed, 8 bytes
# each with FP64 storage and 4 with FP32 storage.
LBM_FLOPS_PER_NODE = 307
LBM_BYTES_PER_NODE = {True: 19 * 8 * 2 + 48, False: 19 * 4 * 2 + 24}


def _lbm_roofline(timing, sysm, fp64_peak, fp32_peak, peak_notes, hbm_gbs, hbm_note):
    d = timing.get("lbm")
    if not d or d["launches"] == 0:
        return None
    fp64 = sysm.precision != W.PRECISION_MIXED  # only mixed handles store the fluid in FP32
    avg_ms = d["ms"] / d["launches"]
    nodes = d["units"] / d["launches"]
    flops = nodes * LBM_FLOPS_PER_NODE / (avg_ms * 1e-3) / 1e12
    gbs = nodes * LBM_BYTES_PER_NODE[fp64] / (avg_ms * 1e-3) / 1e9
    alu = {"bound": "alu", "achieved": flops, "peak": fp64_peak if fp64 else fp32_peak, "unit": "TFLOP/s",
           "frac": flops / (fp64_peak if fp64 else fp32_peak), "peak_source": peak_notes[0 if fp64 else 1]}
    hbm = {"bound": "hbm", "achieved": gbs, "peak": hbm_gbs, "unit": "GB/s", "frac": gbs / hbm_gbs,
           "peak_source": hbm_note, "algorithmic_bytes_per_launch": nodes * LBM_BYTES_PER_NODE[fp64]}
    ff = sysm.precision == W.PRECISION_FF  # FP64 storage, float-float collision
    if ff:
        alu = {"bound": "alu", "note": "float-float collision on the FP32 pipe; FP64 operations per node "
               "about 60 (deviations, output adds)"}
    main, other = (alu, hbm) if fp64 and not ff else (hbm, alu)
    main = dict(main)
    main.update({"kernel": "k_lbm_step_ff" if ff else ("k_lbm_step<double>" if fp64 else "k_lbm_step<float>"),
                 "traffic": None,
                 "avg_launch_ms": avg_ms, "node_updates_per_s": nodes / (avg_ms * 1e-3),
                 "secondary": other})
    return main


def _contact_roofline(timing, sysm, fp64_peak, fp64_note, hbm_gbs, hbm_note):
    d = timing.get("contact")
    if not d or d["launches"] == 0:
        return None
    c = contacts_per_particle(sysm)
    avg_ms = d["ms"] / d["launches"]
    flops = sysm.n * c * CONTACT_FLOPS_PER_EVAL
    achieved = flops / (avg_ms * 1e-3) / 1e12
    bytes_launch = sysm.n * (CONTACT_BYTES_FIXED + CONTACT_BYTES_PER_CONTACT * c)
    gbs = bytes_launch / (avg_ms * 1e-3) / 1e9
    return {"bound": "alu", "kernel": "contact pass (k_ct_* + k_contact)", "achieved": achieved,
            "peak": fp64_peak, "unit": "TFLOP/s", "frac": achieved / fp64_peak, "traffic": None,
            "avg_launch_ms": avg_ms, "flops_per_launch": flops, "contacts_per_particle": c,
            "peak_source": fp64_note,
            "hbm": {"algorithmic_bytes_per_launch": bytes_launch, "achieved": gbs, "peak": hbm_gbs,
                    "unit": "GB/s", "frac": gbs / hbm_gbs, "peak_source": hbm_note}}


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        return json.load(open(path))
    except Exception:
        return {}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.thread.join(timeout=5)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    if ws <= 1:
        return 0, 1, 0
    import torch.distributed as dist
    backend = "nccl" if _cuda_available() else "gloo"
    dist.init_process_group(backend=backend)
    return dist.get_rank(), dist.get_world_size(), int(os.environ.get("LOCAL_RANK", "0"))


def _cuda_available():
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


def reduce_max(value: float, world: int, device=None) -> float:
    """Maximum of a float over all ranks (identity for one rank)."""
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world: int, device=None):
    if world > 1:
        import torch
        import torch.distributed as dist
        t = torch.zeros(1, device=device)
        dist.all_reduce(t)


def aggregate(units_per_rank: float, seconds_max: float, world: int) -> float:
    """Whole-job throughput: every rank processed units_per_rank in at most
    seconds_max."""
    return units_per_rank * world / seconds_max


# ----------------------------------------------------------------------------
# CPU oracle timing (the reference arm and the cpu_baseline key)
# ----------------------------------------------------------------------------

def _oracle_full_pass_is_cheap(sysm) -> bool:
    """The oracle's contact search is brute force over all pairs: above about
    2e8 pair checks a full force pass is skipped in favour of a sample."""
    return sysm.contact is None or sysm.n * (sysm.n - 1) / 2 <= 2e8


def time_oracle(sysm: W.RodSystem, budget_s: float = 12.0, max_steps: int = 1000):
    """Times oracle steps of the workload on the host cores within a bounded
    budget; for systems whose single step exceeds the budget, times the bond/
    Zeeman pass on all particles plus the all-pairs sums of a particle sample."""
    from oracle import Oracle
    o = Oracle(sysm)
    cores = os.cpu_count() or 1
    if not _oracle_full_pass_is_cheap(sysm):
        return _time_oracle_sampled(sysm, o, budget_s, None, cores)
    if sysm.lbm is not None:
        # one whole LBM cycle (n_sub steps and the LBM step)
        t0 = time.perf_counter()
        o.run(sysm.lbm.n_sub)
        dt = time.perf_counter() - t0
        return {"value": sysm.n * sysm.lbm.n_sub / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
                "sample": f"one LBM cycle of {sysm.name}: {sysm.lbm.n_sub} oracle steps and one LBM step of "
                          f"{sysm.lbm.nodes} nodes"}, dt / sysm.lbm.n_sub
    t0 = time.perf_counter()
    o.forces()  # forces at t, as the first step needs them
    o.forces_valid = True
    t_force = time.perf_counter() - t0
    if t_force * 2 < budget_s:
        steps = max(1, min(max_steps, int(budget_s / max(t_force, 1e-6)) // 2))
        t0 = time.perf_counter()
        o.run(steps)
        dt = time.perf_counter() - t0
        return {"value": sysm.n * steps / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
                "sample": f"{steps} full oracle steps of {sysm.name} ({sysm.n} particles)"}, dt / steps
    return _time_oracle_sampled(sysm, o, budget_s, t_force, cores)


def _time_oracle_sampled(sysm, o, budget_s, t_force, cores):
    """O(N) part on all particles; the all-pairs parts (dipole sums and the
    brute-force contact search) on a particle sample scaled to N, the sample
    sized by a short calibration run to about half the budget."""
    from oracle import Oracle
    lin = sysm.copy()
    lin.dipole_mode = W.DIPOLE_OFF
    lin.contact = None
    ob = Oracle(lin)
    t0 = time.perf_counter()
    _, _, m = ob.forces(want_m=True)
    t_lin = time.perf_counter() - t0
    parts = []
    if sysm.dipole_mode != W.DIPOLE_OFF:
        parts.append("dipole sums")
    if sysm.contact is not None:
        parts.append("contact search")

    def sample(idx):
        t0 = time.perf_counter()
        if sysm.dipole_mode != W.DIPOLE_OFF:
            o.dipole_sample(idx, m=m)
        if sysm.contact is not None:
            o.contact_sample(idx)
        return time.perf_counter() - t0

    k0 = min(sysm.n, 64)
    t0s = sample(np.linspace(0, sysm.n - 1, k0).astype(np.int64))
    k = int(min(sysm.n, max(k0, k0 * 0.5 * budget_s / max(t0s, 1e-6))))
    idx = np.linspace(0, sysm.n - 1, k).astype(np.int64)
    t_s = sample(idx)
    per_step = t_lin + t_s * sysm.n / k
    return {"value": sysm.n / per_step, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"one force pass of {sysm.name}: bond/Zeeman on all {sysm.n} particles, "
                      f"{' and '.join(parts)} on {k} sampled particles scaled to {sysm.n}"}, per_step


def run_reference(args, rank, world):
    if rank != 0:
        return
    sysm = WORKLOADS[args.workload]()
    from oracle import Oracle
    o = Oracle(sysm)
    cores = os.cpu_count() or 1
    t_force = None
    if _oracle_full_pass_is_cheap(sysm):
        t0 = time.perf_counter()
        o.forces()
        o.forces_valid = True
        t_force = time.perf_counter() - t0
    # each reference step is a bounded sample: a full oracle step when it is
    # cheap, otherwise the sampled force pass of time_oracle
    sampled = t_force is None or t_force > 2.0 or sysm.lbm is not None
    if sampled:
        base, per = time_oracle(sysm, budget_s=4.0)
        ms = per * 1e3
        sample = base["sample"]
    else:
        for _ in range(args.warmup):
            o.run(1)
        t0 = time.perf_counter()
        o.run(args.steps)
        ms = (time.perf_counter() - t0) * 1e3 / args.steps
        sample = f"{args.steps} full oracle steps of {sysm.name}"
    value = sysm.n / (ms / 1e3)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": _config(sysm, args),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def _config(sysm, args):
    return {"workload": args.workload, "n_particles": sysm.n, "n_rods": sysm.n_rods,
            "n_bonds": sysm.n_bonds, "ordered_pairs_per_step": sysm.ordered_pairs(),
            "dipole_mode": {0: "off", 1: "all pairs", 2: "per rod"}[sysm.dipole_mode],
            "precision": {W.PRECISION_FP64: "fp64", W.PRECISION_MIXED: "fp32-pair/fp64-accum",
                          W.PRECISION_FF: "float-float pairs/fp64-accum"}[sysm.precision],
            "dt": sysm.dt, "l2": "flushed before every timed step (256 MiB write)",
            "contact": None if sysm.contact is None else
            {"model": "hertz-mindlin", "E": sysm.contact.E, "nu": sysm.contact.nu, "mu": sysm.contact.mu,
             "exclude": sysm.contact.exclude},
            "bond_damping": sysm.bond_damping is not None,
            "lbm": None if sysm.lbm is None else
            {"lattice": [sysm.lbm.nx, sysm.lbm.ny, sysm.lbm.nz], "n_sub": sysm.lbm.n_sub, "tau": sysm.lbm.tau,
             "storage": "fp32 deviations" if sysm.precision == W.PRECISION_MIXED else "fp64"},
            "parallelism": "replicas"}


# ----------------------------------------------------------------------------
# GPU arm
# ----------------------------------------------------------------------------

def _timed_steps(sim, torch, stream, flush, k: int):
    """k single steps, each bracketed by CUDA events on the handle's stream,
    with an L2 flush before each (outside the events).  Returns ms/step."""
    evs = []
    for _ in range(k):
        with torch.cuda.stream(stream):
            flush.zero_()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        sim.step(1)
        b.record(stream)
        evs.append((a, b))
    torch.cuda.synchronize()
    return sum(a.elapsed_time(b) for a, b in evs) / k


def _roofline(timing, kind_units_flops, peak_tflops, unit_note, kernel="k_dipole"):
    d = timing["dipole"]
    if d["launches"] == 0:
        return None
    avg_ms = d["ms"] / d["launches"]
    flops = kind_units_flops * d["units"] / d["launches"]
    achieved = flops / (avg_ms * 1e-3) / 1e12
    return {"bound": "alu", "kernel": kernel, "achieved": achieved, "peak": peak_tflops, "unit": "TFLOP/s",
            "frac": achieved / peak_tflops, "traffic": None, "avg_launch_ms": avg_ms,
            "peak_source": unit_note}


def _roofline_pipe(timing, n_sm, sm_max, kernel, ops_per_pair, flops_per_pair, symmetric):
    """An FP32-pipe dipole kernel against the FP32 pipe: FP32-pipe lane
    operations per second over the pipe's 128 lanes per SM per clock (each
    add, mul or fma holds a lane for one clock); the flop rate (FMA = 2)
    alongside.  The counts are per unordered pair (symmetric kernels) or per
    ordered pair."""
    d = timing["dipole"]
    if d["launches"] == 0:
        return None
    avg_ms = d["ms"] / d["launches"]
    pairs = d["units"] / d["launches"] / (2.0 if symmetric else 1.0)
    ops = pairs * ops_per_pair / (avg_ms * 1e-3) / 1e12
    peak = n_sm * FP32_FMA_PER_SM_CLK * sm_max * 1e6 / 1e12
    flops = pairs * flops_per_pair / (avg_ms * 1e-3) / 1e12
    fpeak = 2.0 * peak
    what = "unordered" if symmetric else "ordered"
    return {"bound": "alu", "kernel": kernel, "achieved": ops, "peak": peak,
            "unit": "Tops/s (FP32-pipe lane operations)", "frac": ops / peak, "traffic": None,
            "avg_launch_ms": avg_ms,
            "peak_source": f"derived FP32 pipe: {n_sm} SMs x {FP32_FMA_PER_SM_CLK} lanes/clk x {sm_max:.0f} MHz",
            "ops_per_pair": f"{ops_per_pair} FP32-pipe operations per {what} pair",
            "flops": {"achieved": flops, "peak": fpeak, "unit": "TFLOP/s", "frac": flops / fpeak,
                      "note": f"{flops_per_pair:g} flops per {what} pair (FMA = 2)"}}


def _roofline_ff(timing, n_sm, sm_max, kernel="k_dipole_sym_ff"):
    """k_dipole_sym_ff against the FP32 pipe (see _roofline_pipe)."""
    return _roofline_pipe(timing, n_sm, sm_max, kernel, FF_PIPE_OPS_PER_PAIR, FF_FLOPS_PER_PAIR, True)


def _roofline_mixed(timing, n_sm, sm_max, symmetric):
    """The packed FP32-pair kernels against the FP32 pipe (see _roofline_pipe)."""
    if symmetric:
        return _roofline_pipe(timing, n_sm, sm_max, "k_dipole_sym_mixed", MIX_SYM_PIPE_OPS_PER_PAIR,
                              2 * FLOPS_PER_PAIR_SYM_FP32, True)
    return _roofline_pipe(timing, n_sm, sm_max, "k_dipole_mixed", MIX_PIPE_OPS_PER_PAIR, FLOPS_PER_PAIR_FP32,
                          False)


def run_gpu(args, rank, world, local_rank):
    import torch
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU (no CPU fallback)")
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    from paper_2603_27279_gb300 import build as B
    if rank == 0:
        B.build()
    barrier(world, dev)
    from paper_2603_27279_gb300 import bpm
    sysm = WORKLOADS[args.workload]()
    props = torch.cuda.get_device_properties(dev)
    n_sm = props.multi_processor_count
    peaks = _peaks()
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    fp64_peak = n_sm * FP64_FMA_PER_SM_CLK * 2 * sm_max * 1e6 / 1e12
    fp32_peak = n_sm * FP32_FMA_PER_SM_CLK * 2 * sm_max * 1e6 / 1e12
    stream = torch.cuda.Stream(device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    sim = bpm.Simulation(sysm, stream=stream.cuda_stream)
    if args.dipole_plan:
        kind, param = (int(v) for v in args.dipole_plan.split(":"))
        sim.set_dipole_plan(kind, param)
    if args.overlap != -1:
        sim.set_overlap(args.overlap)
    for _ in range(args.warmup):
        with torch.cuda.stream(stream):
            flush.zero_()
        sim.step(1)
    sim.set_timing(True)
    sampler = ClockSampler(local_rank)
    sampler.start()
    barrier(world, dev)
    torch.cuda.synchronize()
    ms = _timed_steps(sim, torch, stream, flush, args.steps)
    torch.cuda.synchronize()
    barrier(world, dev)
    clocks = sampler.stop()
    timing = sim.timing()
    plan = sim.dipole_plan()
    overlap = sim.overlap()
    sim.set_timing(False)
    ms_max = reduce_max(ms, world, dev)
    value = aggregate(sysm.n, ms_max / 1e3, world)
    pairs_per_s = aggregate(float(sysm.ordered_pairs()), ms_max / 1e3, world)
    fp64 = sysm.precision == W.PRECISION_FP64
    ff = sysm.precision == W.PRECISION_FF
    flops_pair = ((FLOPS_PER_PAIR_SYM_FP64 if plan[0] == 2 else FLOPS_PER_PAIR_FP64) if fp64 else
                  (FLOPS_PER_PAIR_SYM_FP32 if plan[0] == 2 else FLOPS_PER_PAIR_FP32))
    roof = _roofline(timing, flops_pair,
                     fp64_peak if fp64 else fp32_peak,
                     (f"derived FP64 peak: {n_sm} SMs x {FP64_FMA_PER_SM_CLK} DFMA/clk x 2 flop x {sm_max:.0f} MHz"
                      if fp64 else
                      f"derived FP32 peak: {n_sm} SMs x {FP32_FMA_PER_SM_CLK} FFMA/clk x 2 flop x {sm_max:.0f} MHz"),
                     kernel=(("k_dipole_symw_fp64" if plan[1] == 0 else "k_dipole_sym_fp64") if plan[0] == 2
                             else "k_dipole_fp64") if fp64 else
                     ("k_dipole_sym_mixed" if plan[0] == 2 else "k_dipole_mixed"))
    if ff:
        roof = _roofline_ff(timing, n_sm, sm_max, "k_dipole_symw_ff" if plan[1] == 0 else "k_dipole_sym_ff")
    elif not fp64 and sysm.dipole_mode != W.DIPOLE_OFF:
        roof = _roofline_mixed(timing, n_sm, sm_max, plan[0] == 2)
    # the kernel kind with the most time; "integrate" is several small kernels
    dominant = max((k for k in timing if k != "integrate"), key=lambda k: timing[k]["ms"])
    hbm_note = ("measured HBM copy bandwidth (MEASURED_PEAKS.json hbm_gbs)" if "hbm_gbs" in peaks
                else "fallback HBM 6800 GB/s")
    if dominant == "lbm":
        roof = _lbm_roofline(timing, sysm, fp64_peak, fp32_peak,
                             (f"derived FP64 peak: {n_sm} SMs x {FP64_FMA_PER_SM_CLK} DFMA/clk x 2 flop x "
                              f"{sm_max:.0f} MHz",
                              f"derived FP32 peak: {n_sm} SMs x {FP32_FMA_PER_SM_CLK} FFMA/clk x 2 flop x "
                              f"{sm_max:.0f} MHz"), float(peaks.get("hbm_gbs", 6800.0)), hbm_note)
    if (roof is None or dominant == "contact") and sysm.contact is not None:
        hbm = float(peaks.get("hbm_gbs", 6800.0))
        roof = _contact_roofline(timing, sysm, fp64_peak,
                                 f"derived FP64 peak: {n_sm} SMs x {FP64_FMA_PER_SM_CLK} DFMA/clk x 2 flop x "
                                 f"{sm_max:.0f} MHz", hbm,
                                 "measured HBM copy bandwidth (MEASURED_PEAKS.json hbm_gbs)"
                                 if "hbm_gbs" in peaks else "fallback HBM 6800 GB/s")
    if roof is not None:
        roof["traffic"] = NCU_TRAFFIC.get((args.workload, roof["kernel"]))
    launches_per_step = sum(timing[k]["launches"] for k in timing) / args.steps

    # end to end through the public API with pinned host buffers: upload the
    # state, one step, read the state back, every step
    n = sysm.n
    pin = {k: torch.empty((n, c), dtype=torch.float64, pin_memory=True).numpy()
           for k, c in (("x", 3), ("q", 4), ("v", 3), ("w", 3))}
    x, q, v, w, t = sim.get_state()
    pin["x"][:] = x
    pin["q"][:] = q
    pin["v"][:] = v
    pin["w"][:] = w
    k_e2e = max(3, min(args.steps, 20))
    barrier(world, dev)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(k_e2e):
        sim.set_state(pin["x"], pin["q"], pin["v"], pin["w"], t)
        sim.step(1)
        t = bpm.bpm_get_state(sim.h, pin["x"], pin["q"], pin["v"], pin["w"])
    torch.cuda.synchronize()
    e2e_s = reduce_max((time.perf_counter() - t0) / k_e2e, world, dev)
    state_bytes = n * 13 * 8
    sim.close()

    variants = {}
    if args.workload == "helix_16384" and not args.no_variants:
        vs = W.helix(precision=W.PRECISION_MIXED)
        vsim = bpm.Simulation(vs, stream=stream.cuda_stream)
        for _ in range(args.warmup):
            vsim.step(1)
        vsim.set_timing(True)
        vms = _timed_steps(vsim, torch, stream, flush, args.steps)
        vt = vsim.timing()
        vplan = vsim.dipole_plan()
        vsim.close()
        vms = reduce_max(vms, world, dev)
        variants["fp32_pair_fp64_accum"] = {
            "value": aggregate(vs.n, vms / 1e3, world), "ms_per_step": vms,
            "pairs_per_s": aggregate(float(vs.ordered_pairs()), vms / 1e3, world),
            "speedup_vs_fp64": ms_max / vms,
            "dipole_plan": {"kind": {0: "auto", 1: "ordered", 2: "symmetric"}[vplan[0]], "param": vplan[1]},
            "roofline": _roofline_mixed(vt, n_sm, sm_max, vplan[0] == 2)}

        # float-float dipole pairs: FP64-class accuracy on the FP32 pipe; its
        # step-1 forces against those of the FP64 path on the same state
        vs = W.helix(precision=W.PRECISION_FF)
        vsim = bpm.Simulation(vs, stream=stream.cuda_stream)
        fsim = bpm.Simulation(W.helix(), stream=stream.cuda_stream)
        f_ff, t_ff = vsim.forces()
        f_64, t_64 = fsim.forces()
        fsim.close()
        for _ in range(args.warmup):
            vsim.step(1)
        vsim.set_timing(True)
        vms = reduce_max(_timed_steps(vsim, torch, stream, flush, args.steps), world, dev)
        vt = vsim.timing()
        vplan = vsim.dipole_plan()
        vsim.close()
        variants["float_float_dipole"] = {
            "value": aggregate(vs.n, vms / 1e3, world), "ms_per_step": vms,
            "pairs_per_s": aggregate(float(vs.ordered_pairs()), vms / 1e3, world),
            "speedup_vs_fp64": ms_max / vms,
            "rel_force_diff_vs_fp64": float(np.linalg.norm(f_ff - f_64) / np.linalg.norm(f_64)),
            "rel_torque_diff_vs_fp64": float(np.linalg.norm(t_ff - t_64) / np.linalg.norm(t_64)),
            "dipole_plan": {"kind": "symmetric", "param": vplan[1]},
            "kernel_ms_per_step": {k: vt[k]["ms"] / args.steps for k in vt},
            "roofline": _roofline_ff(vt, n_sm, sm_max, "k_dipole_symw_ff" if vplan[1] == 0 else "k_dipole_sym_ff")}

        for vname, mk in (("with_contact", _helix_contact), ("with_bond_damping", _helix_damped)):
            vs = mk()
            vsim = bpm.Simulation(vs, stream=stream.cuda_stream)
            for _ in range(args.warmup):
                vsim.step(1)
            vsim.set_timing(True)
            vms = reduce_max(_timed_steps(vsim, torch, stream, flush, args.steps), world, dev)
            vt = vsim.timing()
            vsim.close()
            variants[vname] = {"value": aggregate(vs.n, vms / 1e3, world), "ms_per_step": vms,
                               "overhead_vs_plain": vms / ms_max - 1.0,
                               "kernel_ms_per_step": {k: vt[k]["ms"] / args.steps for k in vt}}

    # the adjoint of the time stepping (config of the magnetisation-profile
    # design pattern): forward with checkpoints, then the reverse sweep
    adjoint = None
    if args.workload == "adjoint_rod_2048":
        steps_a, every_a = 500, 50
        tip = sysm.n - 1

        def run_adjoint(precision):
            asim = bpm.Simulation(sysm, stream=stream.cuda_stream, precision=precision)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            asim.adjoint_begin(steps_a, every_a)
            t1 = time.perf_counter()
            xa = asim.get_state()[0]
            dL = np.zeros_like(xa)
            dL[tip] = 2.0 * (xa[tip] - xa[tip] * 0.99)
            t2 = time.perf_counter()
            gm, gB = asim.adjoint_end(dL)
            t3 = time.perf_counter()
            asim.close()
            return (t1 - t0) * 1e3, (t3 - t2) * 1e3, gm, gB

        f_ms, r_ms, gm, gB = run_adjoint(W.PRECISION_FP64)
        adjoint = {"steps": steps_a, "checkpoint_every": every_a, "forward_ms": f_ms,
                   "reverse_ms": r_ms, "reverse_over_forward": r_ms / max(f_ms, 1e-12),
                   "gradient_finite": bool(np.isfinite(gm).all() and np.isfinite(gB).all()),
                   "note": "host wall time of bpm_adjoint_begin (500 steps with checkpoints) and bpm_adjoint_end "
                           "(segment recompute + reverse sweep) for dL/dm~ and dL/dB of a tip loss"}
        # the same on a BPM_FF handle: float-float dipole pairs forward and
        # in the dipole VJP; its gradient against the FP64 one
        f2, r2, gm2, gB2 = run_adjoint(W.PRECISION_FF)
        scale = max(np.abs(gm).max(), np.abs(gB).max())
        adjoint["float_float"] = {
            "forward_ms": f2, "reverse_ms": r2, "speedup_vs_fp64": (f_ms + r_ms) / max(f2 + r2, 1e-12),
            "max_gradient_diff_vs_fp64": float(max(np.abs(gm2 - gm).max(), np.abs(gB2 - gB).max()) / scale)}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu, _ = time_oracle(sysm)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None,
                "dtype": "f64" if fp64 else ("f32x2 float-float pairs/f64-accum" if ff else "f32-pair/f64-accum"),
                "data": "synthetic",
                "config": _config(sysm, args), "pairs_per_s": pairs_per_s,
                "roofline": roof, "cpu_baseline": cpu,
                "e2e": {"value": aggregate(n, e2e_s, world), "unit": UNIT,
                        "h2d_bytes_per_step": state_bytes, "d2h_bytes_per_step": state_bytes,
                        "note": "bpm_set_state from pinned host buffers + bpm_step(1) + bpm_get_state to "
                                "pinned host buffers per step; the uploaded state needs its forces "
                                "recomputed, so each e2e step evaluates forces twice"},
                "gpu_launches": int(round(launches_per_step * args.steps)),
                "kernel_ms_per_step": {k: timing[k]["ms"] / args.steps for k in timing},
                "dipole_plan": {"kind": {0: "auto", 1: "ordered", 2: "symmetric"}[plan[0]], "param": plan[1],
                                "bond_beside_dipole": bool(overlap[0]),
                                "dipole_blocks_beside_bond": overlap[1] or None,
                                "bond_blocks_beside_dipole": overlap[2] or None},
                "clocks": clocks, "variants": variants}
        if overlap[0]:
            line["kernel_ms_note"] = ("the bond kernel runs on a second stream beside the dipole kernel: their "
                                      "per-launch times overlap and include the sharing of the SMs")
        if adjoint is not None:
            line["adjoint"] = adjoint
        print(json.dumps(line), flush=True)


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--workload", default="helix_16384", choices=sorted(WORKLOADS))
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-variants", action="store_true", help="skip the mixed-precision variant")
    ap.add_argument("--dipole-plan", default="", metavar="KIND:PARAM",
                    help="fix the dipole plan instead of autotuning it (1:chunks ordered, 2:g symmetric)")
    ap.add_argument("--overlap", type=int, default=-1, choices=[-1, 0, 1],
                    help="bond kernel beside the dipole kernel: -1 tuned (default), 0 never, 1 whenever possible")
    args = ap.parse_args(argv)
    if args.warmup < 3:
        raise SystemExit("--warmup must be >= 3")
    rank, world, local_rank = _dist()
    try:
        if args.impl == "reference":
            run_reference(args, rank, world)
        else:
            run_gpu(args, rank, world, local_rank)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
