"""Benchmark of one timestep of the bonded-particle magneto-elastic rod model
on GB300, through the C ABI of include/bpm.h.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME]
                    [--impl reference] [--peaks]

A step is one pass of the whole hot path: bond forces/torques + Zeeman +
dipole orientation + all-pairs dipole-dipole + velocity Verlet / Richardson
update.  Default workload: the cilia array of 512 rods x 256 particles
(131072 particles, 1.7e10 ordered dipole pairs per step) in FP64, the largest
single-GPU configuration.  Each timed step is one bpm_step(1), replayed from
the library's CUDA graphs, between CUDA events on the handle's stream; the
L2 cache (129 MB) is flushed by a 256 MiB write before every timed step,
outside the events.  Per-kernel times come from a second pass of the same
steps with the library's kernel events (eager launches; a kernel's own
duration does not depend on how it was launched).  The other precisions and
workloads (cilia in float-float and FP32 pairs, the 2048 batched rods and
the 16384-particle helix in three precisions) are reported under
`variants`, each with its error against the CPU FP64 oracle.

--peaks runs the library's pipe throughput probe (bpm_measure_pipes) and
writes MEASURED_PEAKS_EXT.json, whose rates are the roofline denominators of
the ALU-bound kernels.  --record-traffic parses an ncu raw CSV export of one
kernel and stores its DRAM bytes per launch in profiles/dram_traffic.json,
keyed by a hash of the kernel's sources: a changed kernel reports no traffic
until it is profiled again.

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
# 3, field sums 6 = 44 per ordered pair (pair_fp32x2).  The symmetric kernel
# (pair_mix2) keeps its sums scaled (the field over 3, the j-side force and
# Bs negated) and shares -1/(3 r^3) between the sides: r 9, r^2 3, powers 3,
# a, b, d 9, s 3, A, S, b/r^5 3, -1/(3 r^3) 1, i side force 6, Bs 1, field 6,
# j side force 6, field 6, Bs 1 = 57 per unordered pair.
MIX_PIPE_OPS_PER_PAIR = 44
MIX_SYM_PIPE_OPS_PER_PAIR = 57
# FP64 operations of one bond's force and torque as the oracle's bond_impl
# evaluates them (the plain definition: each +, -, x, / one operation,
# quaternion products and rotations written out in full): 579, besides 9
# square roots and 4 atan2, which are not counted.  The count is the one that
# tests/test_bench_counts.py obtains by compiling the oracle with an
# operation-counting number type.  The kernel reaches the same results with
# about 323 FP64 instructions, the particle's own work included (rotation
# matrices, the C' alignment in closed form, sparse products, series for
# small angles).
BOND_FLOPS_ORACLE = 579
# Nominal lanes per SM per clock of GB300's FMA pipes (kept beside the
# measured rates of MEASURED_PEAKS_EXT.json, which take precedence).
FP64_FMA_PER_SM_CLK = 2
FP32_FMA_PER_SM_CLK = 128
L2_FLUSH_BYTES = 256 << 20
L2_BYTES = 129e6
DEFAULT_WORKLOAD = "cilia_512x256_fp64"
PEAKS_EXT = "MEASURED_PEAKS_EXT.json"
TRAFFIC_FILE = os.path.join("profiles", "dram_traffic.json")

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
    # the cilia lattice with rods of 32 particles (16384 particles): the
    # headline kernels on a size that an ncu capture of many passes takes
    "cilia_16x32x32_fp64": lambda: W.cilia(16, 32, 32, precision=W.PRECISION_FP64),
    "batched_rods_2048_ff": lambda: W.batched_rods(precision=W.PRECISION_FF),
    "batched_rods_2048_fp64": lambda: W.batched_rods(precision=W.PRECISION_FP64),
    "straight_rod_64": lambda: W.straight_rod(),
    "batched_rods_2048": lambda: W.batched_rods(),
    "batched_rods_2048_mixed": lambda: W.batched_rods(precision=W.PRECISION_MIXED),
    "cilia_512x256": lambda: W.cilia(),
    "cilia_512x256_mixed": lambda: W.cilia(precision=W.PRECISION_MIXED),
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
    2e8 pair checks a full force pass is skipped in favour of a sample; so is
    a dipole pass of more than 2e9 ordered pairs (seconds on the host)."""
    if sysm.dipole_mode != W.DIPOLE_OFF and sysm.ordered_pairs() > 2e9:
        return False
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
    if sampled and sysm.lbm is None:
        # W untimed and K timed steps, each the O(N) terms on all particles
        # and the all-pairs sums of a particle sample scaled to N, the
        # sample sized so that the whole run takes about two minutes
        budget = min(4.0, max(0.5, 120.0 / (args.steps + args.warmup)))
        for _ in range(args.warmup):
            _time_oracle_sampled(sysm, o, budget, None, cores)
        per = []
        for _ in range(args.steps):
            base, p = _time_oracle_sampled(sysm, o, budget, None, cores)
            per.append(p)
        ms = 1e3 * sum(per) / len(per)
        sample = f"{args.steps} timed steps after {args.warmup} untimed ones, each {base['sample']}"
    elif sampled:
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
# peaks, traffic records
# ----------------------------------------------------------------------------

def _peaks_ext():
    try:
        return json.load(open(os.path.join(ROOT, PEAKS_EXT)))
    except Exception:
        return {}


def pipe_peaks(n_sm: int, sm_max: float) -> dict:
    """Denominators of the ALU-bound rooflines: FP64 TFLOP/s (FMA = 2) and
    FP32-pipe lane operations per second (Tops), measured by the pipe probe
    (MEASURED_PEAKS_EXT.json) where present, else the nominal unit counts at
    the maximum clock; both are returned."""
    nom64 = n_sm * FP64_FMA_PER_SM_CLK * 2 * sm_max * 1e6 / 1e12
    nom32 = n_sm * FP32_FMA_PER_SM_CLK * sm_max * 1e6 / 1e12
    out = {"fp64_tflops": nom64, "fp32_tops": nom32, "fp64_nominal": nom64, "fp32_nominal": nom32,
           "fp64_source": f"nominal: {n_sm} SMs x {FP64_FMA_PER_SM_CLK} DFMA/clk x 2 flop x {sm_max:.0f} MHz",
           "fp32_source": f"nominal: {n_sm} SMs x {FP32_FMA_PER_SM_CLK} lanes/clk x {sm_max:.0f} MHz",
           "measured": False}
    ext = _peaks_ext().get("pipes")
    if ext:
        # the FP64 pipe's instruction rate: the faster of the fma and add
        # probes, two flops per instruction slot
        d = max((ext[k] for k in ("fp64_fma", "fp64_add") if k in ext), key=lambda r: r["per_s"])
        out["fp64_tflops"] = 2.0 * d["per_s"] / 1e12
        out["fp64_source"] = (f"measured ({PEAKS_EXT}: FP64 pipe probe, {d['per_sm_per_clk']:.3f} instructions "
                              f"per SM per clock at {d['sm_mhz']:.0f} MHz, 2 flops each)")
        f1, f2 = ext["fp32_fma"], ext["fp32x2_fma"]
        best = f1 if f1["per_s"] >= f2["per_s"] else f2
        out["fp32_tops"] = best["per_s"] / 1e12
        out["fp32_source"] = (f"measured ({PEAKS_EXT}: FP32 fma probes, {best['per_sm_per_clk']:.1f} lanes per SM "
                              f"per clock at {best['sm_mhz']:.0f} MHz)")
        out["measured"] = True
    return out


# the translation unit that defines each kernel; its hash, with the shared
# headers, keys the traffic records
KERNEL_SOURCES = [("k_dipole_sym_ff", "bpm_dipole_ff.cu"), ("k_dipole_symw_ff", "bpm_dipole_ff.cu"),
                  ("k_ff_encode", "bpm_dipole_ff.cu"), ("k_dipole", "bpm_dipole.cu"),
                  ("k_reduce_slots", "bpm_integrate.cu"), ("k_bond", "bpm_bond.cu"), ("k_orient", "bpm_bond.cu"),
                  ("k_first_half", "bpm_integrate.cu"), ("k_finish", "bpm_integrate.cu"),
                  ("k_contact", "bpm_contact.cu"), ("contact", "bpm_contact.cu"), ("k_lbm", "bpm_lbm.cu"),
                  ("k_ibm", "bpm_lbm.cu")]


def kernel_source_hash(kernel: str):
    import hashlib
    csrc = os.path.join(ROOT, "paper_2603_27279_gb300", "csrc")
    tu = next((f for k, f in KERNEL_SOURCES if kernel.startswith(k)), None)
    if tu is None:
        return None
    files = [os.path.join(csrc, tu)] + sorted(os.path.join(csrc, f) for f in os.listdir(csrc)
                                              if f.endswith((".h", ".cuh")))
    files.append(os.path.join(ROOT, "include", "bpm.h"))
    h = hashlib.sha256()
    for f in files:
        h.update(open(f, "rb").read())
    return h.hexdigest()[:16]


def recorded_traffic(workload: str, kernel: str):
    """DRAM bytes per launch of the kernel on the workload from the ncu record,
    or None when there is none or the kernel's sources changed since."""
    try:
        recs = json.load(open(os.path.join(ROOT, TRAFFIC_FILE)))
    except Exception:
        return None
    for r in recs:
        if r["workload"] == workload and r["kernel"] == kernel:
            if r.get("source_hash") == kernel_source_hash(kernel):
                return r["dram_bytes_per_launch"]
    return None


def record_traffic(csv_path: str, kernel: str, workload: str, scale: float, note: str):
    """Stores DRAM read + write bytes per launch of `kernel` from an ncu raw
    CSV export (ncu -i REP --page raw --csv), averaged over its launches and
    multiplied by `scale` (units of a full launch over units captured)."""
    import csv
    rows = list(csv.reader(open(csv_path)))
    hdr = rows[0]
    ki = hdr.index("Kernel Name")
    ri = hdr.index("dram__bytes_read.sum")
    wi = hdr.index("dram__bytes_write.sum")
    units = rows[1]
    mult = {"byte": 1.0, "Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9, "KB": 1e3, "MB": 1e6, "GB": 1e9}
    import re

    def base_name(full):
        # "void ns::k_name<...>(args)" -> "k_name"
        return re.sub(r"^void\s+", "", full).split("(")[0].split("<")[0].split("::")[-1]

    vals = []
    for r in rows[2:]:
        if len(r) > max(ki, ri, wi) and base_name(r[ki]).startswith(kernel):
            rd = float(r[ri].replace(",", "")) * mult.get(units[ri], 1.0)
            wr = float(r[wi].replace(",", "")) * mult.get(units[wi], 1.0)
            vals.append(rd + wr)
    if not vals:
        raise SystemExit(f"no launch of {kernel} in {csv_path}")
    path = os.path.join(ROOT, TRAFFIC_FILE)
    try:
        recs = json.load(open(path))
    except Exception:
        recs = []
    recs = [r for r in recs if not (r["workload"] == workload and r["kernel"] == kernel)]
    recs.append({"workload": workload, "kernel": kernel, "dram_bytes_per_launch": scale * sum(vals) / len(vals),
                 "launches_captured": len(vals), "scale": scale, "note": note,
                 "source_hash": kernel_source_hash(kernel)})
    json.dump(recs, open(path, "w"), indent=1)
    print(json.dumps(recs[-1]))


def run_peaks(args):
    import torch
    if not torch.cuda.is_available():
        raise SystemExit("--peaks needs a CUDA GPU")
    from paper_2603_27279_gb300 import build as B
    B.build()
    from paper_2603_27279_gb300 import bpm
    sampler = ClockSampler(0)
    sampler.start()
    res = bpm.bpm_measure_pipes()
    clocks = sampler.stop()
    out = {"gpu_name": torch.cuda.get_device_name(0),
           "when": time.strftime("%Y-%m-%dT%H:%M:%SZ", time.gmtime()),
           "how": "python bench.py --peaks: bpm_measure_pipes, eight independent chains per thread of one "
                  "operation on fully occupied SMs for about 50 ms each; rate = lane operations / (event time x "
                  "SMs x SM clock of the run from the cycle counter and the global timer)",
           "pipes": res, "clocks": clocks}
    json.dump(out, open(os.path.join(ROOT, PEAKS_EXT), "w"), indent=1)
    print(json.dumps(out))


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


def _roofline_fp64(timing, flops_per_unit, peaks, kernel):
    d = timing["dipole"]
    if d["launches"] == 0:
        return None
    avg_ms = d["ms"] / d["launches"]
    flops = flops_per_unit * d["units"] / d["launches"]
    achieved = flops / (avg_ms * 1e-3) / 1e12
    return {"bound": "alu", "kernel": kernel, "achieved": achieved, "peak": peaks["fp64_tflops"],
            "unit": "TFLOP/s", "frac": achieved / peaks["fp64_tflops"], "traffic": None, "avg_launch_ms": avg_ms,
            "peak_source": peaks["fp64_source"],
            "nominal": {"peak": peaks["fp64_nominal"], "frac": achieved / peaks["fp64_nominal"],
                        "source": f"nominal {FP64_FMA_PER_SM_CLK} DFMA per SM per clock at the maximum clock"},
            "flops_per_launch": flops}


def _roofline_pipe(timing, peaks, kernel, ops_per_pair, flops_per_pair, symmetric):
    """An FP32-pipe dipole kernel against the FP32 pipe: FP32-pipe lane
    operations per second (each add, mul or fma holds a lane for one clock,
    packed halves counted apart); the flop rate (FMA = 2) alongside.  The
    counts are per unordered pair (symmetric kernels) or per ordered pair."""
    d = timing["dipole"]
    if d["launches"] == 0:
        return None
    avg_ms = d["ms"] / d["launches"]
    pairs = d["units"] / d["launches"] / (2.0 if symmetric else 1.0)
    ops = pairs * ops_per_pair / (avg_ms * 1e-3) / 1e12
    peak = peaks["fp32_tops"]
    flops = pairs * flops_per_pair / (avg_ms * 1e-3) / 1e12
    what = "unordered" if symmetric else "ordered"
    return {"bound": "alu", "kernel": kernel, "achieved": ops, "peak": peak,
            "unit": "Tops/s (FP32-pipe lane operations)", "frac": ops / peak, "traffic": None,
            "avg_launch_ms": avg_ms, "peak_source": peaks["fp32_source"],
            "nominal": {"peak": peaks["fp32_nominal"], "frac": ops / peaks["fp32_nominal"],
                        "source": f"nominal {FP32_FMA_PER_SM_CLK} lanes per SM per clock at the maximum clock"},
            "ops_per_pair": f"{ops_per_pair} FP32-pipe operations per {what} pair",
            "flops": {"achieved": flops, "peak": 2.0 * peak, "unit": "TFLOP/s", "frac": flops / (2.0 * peak),
                      "note": f"{flops_per_pair:g} flops per {what} pair (FMA = 2)"}}


def _dipole_roofline(sysm, timing, plan, peaks):
    if sysm.dipole_mode == W.DIPOLE_OFF:
        return None
    sym = plan[0] == 2
    if sysm.precision == W.PRECISION_FF:
        return _roofline_pipe(timing, peaks, "k_dipole_symw_ff" if plan[1] == 0 else "k_dipole_sym_ff",
                              FF_PIPE_OPS_PER_PAIR, FF_FLOPS_PER_PAIR, True)
    if sysm.precision == W.PRECISION_MIXED:
        if sym:
            return _roofline_pipe(timing, peaks, "k_dipole_symw_mixed" if plan[1] == 0 else "k_dipole_sym_mixed",
                                  MIX_SYM_PIPE_OPS_PER_PAIR, 2 * FLOPS_PER_PAIR_SYM_FP32, True)
        return _roofline_pipe(timing, peaks, "k_dipole_mixed", MIX_PIPE_OPS_PER_PAIR, FLOPS_PER_PAIR_FP32, False)
    kern = ("k_dipole_symw_fp64" if plan[1] == 0 else "k_dipole_sym_fp64") if sym else "k_dipole_fp64"
    return _roofline_fp64(timing, FLOPS_PER_PAIR_SYM_FP64 if sym else FLOPS_PER_PAIR_FP64, peaks, kern)


def _rel(a, b):
    nb = float(np.linalg.norm(b))
    return float(np.linalg.norm(a - b)) / (nb if nb > 0 else 1.0)


class OracleReference:
    """Step-1 forces of a workload's initial state from the CPU FP64 oracle,
    computed once and shared by every precision of the workload: the whole
    field, or for systems whose all-pairs pass is long on the host the O(N)
    terms of all particles plus the dipole sums of a particle sample."""

    def __init__(self, sysm, full_pairs_max=2e9, sample=96, seed=0):
        from oracle import Oracle
        t0 = time.perf_counter()
        self.o = Oracle(sysm)
        if sysm.ordered_pairs() <= full_pairs_max:
            self.idx = np.arange(sysm.n)
            self.f, self.t = self.o.forces()
            self.what = f"all {sysm.n} particles"
        else:
            rng = np.random.default_rng(seed)
            self.idx = np.sort(np.concatenate([rng.choice(sysm.n, sample - 6, replace=False),
                                               [0, 1, 255, 256, sysm.n - 2, sysm.n - 1]]))
            nod = sysm.copy()
            nod.dipole_mode = W.DIPOLE_OFF
            from oracle import Oracle as O2
            fb, tb, m = O2(nod).forces(want_m=True)
            Fd, Td, _ = self.o.dipole_sample(self.idx, m=m)
            self.f = fb[self.idx] + Fd
            self.t = tb[self.idx] + Td
            self.what = f"{len(self.idx)} sampled particles (dipole sums over all partners) of {sysm.n}"
        # per-particle condition scales on at most 4096 of the compared rows
        rows = np.arange(len(self.idx))
        if len(rows) > 4096:
            rows = np.sort(np.random.default_rng(seed + 1).choice(len(rows), 4096, replace=False))
        self.rows = rows
        self.Sf, self.St = self.o.term_scales(self.idx[rows])
        self.seconds = time.perf_counter() - t0

    def error(self, f, t) -> dict:
        fi, ti = f[self.idx], t[self.idx]
        dfi = np.linalg.norm(fi[self.rows] - self.f[self.rows], axis=1)
        dti = np.linalg.norm(ti[self.rows] - self.t[self.rows], axis=1)
        return {"rel_force": _rel(fi, self.f), "rel_torque": _rel(ti, self.t),
                "max_particle_force": float((dfi / np.maximum(self.Sf, 1e-300)).max()),
                "max_particle_torque": float((dti / np.maximum(self.St, 1e-300)).max()),
                "compared": self.what,
                "metric": "norm-wise relative error of step-1 forces and torques against the CPU FP64 oracle; "
                          "per particle |dF_i| / sum_j |F_ij| (max over "
                          f"{len(self.rows)} particles)"}


def measure(bpm, torch, sysm, stream, flush, steps, warmup, timing_steps, plan=None, overlap=-1):
    """Step-1 forces, then graph-path timed steps, then a kernel-timing pass.
    Returns (sim, forces, ms_per_step, timing, kernel_steps)."""
    sim = bpm.Simulation(sysm, stream=stream.cuda_stream)
    if plan:
        sim.set_dipole_plan(*plan)
    if overlap != -1:
        sim.set_overlap(overlap)
    f, t = sim.forces()  # the autotuner fixes the plan here
    for _ in range(warmup):
        with torch.cuda.stream(stream):
            flush.zero_()
        sim.step(1)
    torch.cuda.synchronize()
    ms = _timed_steps(sim, torch, stream, flush, steps)
    sim.set_timing(True)
    _timed_steps(sim, torch, stream, flush, timing_steps)
    timing = sim.timing()
    sim.set_timing(False)
    return sim, (f, t), ms, timing, timing_steps


# bytes of device state per particle that a step reads (state, forces,
# dipoles, bond constants, partial sums): a working set above L2 for the
# batched rods
STATE_BYTES_PER_PARTICLE = 400


def chained_ms(sim, torch, stream, steps):
    """ms per step of one bpm_step(steps) call (the 16-step CUDA graphs
    replayed back to back, one host synchronisation), timed by CUDA events;
    only for systems whose working set exceeds L2, so that no flush is
    needed between steps."""
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(stream)
    sim.step(steps)
    b.record(stream)
    torch.cuda.synchronize()
    return a.elapsed_time(b) / steps


def describe(sysm, sim, timing, ksteps, peaks, workload):
    plan = sim.dipole_plan()
    overlap = sim.overlap()
    roof = _dipole_roofline(sysm, timing, plan, peaks)
    dominant = max((k for k in timing if k != "integrate"), key=lambda k: timing[k]["ms"])
    if roof is not None:
        roof["traffic"] = recorded_traffic(workload, roof["kernel"])
        hbm_gbs = _peaks().get("hbm_gbs")
        if roof["traffic"] is not None and hbm_gbs:
            t_ms = roof["traffic"] / (float(hbm_gbs) * 1e9) * 1e3
            roof["traffic_note"] = (
                f"DRAM bytes of one launch from the ncu record ({TRAFFIC_FILE}); the dipole inputs are "
                f"48 B per particle ({48 * sysm.n / 1e6:.1f} MB); the rest are the FP64 partial sums written "
                f"per (particle, partner supertile) for the deterministic slot reduction: "
                f"{t_ms:.3f} ms at the measured HBM bandwidth, {100 * t_ms / roof['avg_launch_ms']:.2f} % "
                "of the launch")
    bond = None
    b = timing.get("bond")
    if b and b["launches"] > 0 and b["units"] > 0:
        avg_ms = b["ms"] / b["launches"]
        bonds = b["units"] / b["launches"]
        ach = BOND_FLOPS_ORACLE * bonds / (avg_ms * 1e-3) / 1e12
        bond = {"bound": "alu", "kernel": "k_bond", "achieved": ach, "peak": peaks["fp64_tflops"],
                "unit": "TFLOP/s", "frac": ach / peaks["fp64_tflops"], "avg_launch_ms": avg_ms,
                "bonds_per_launch": bonds, "peak_source": peaks["fp64_source"],
                "flops_per_bond": f"{BOND_FLOPS_ORACLE} FP64 operations per bond, counted from the oracle's "
                                  "bond_impl (9 square roots and 4 atan2 not counted)",
                "beside_dipole": bool(sim.overlap()[0])}
    return {"kernel_ms_per_step": {k: timing[k]["ms"] / ksteps for k in timing},
            "bond_roofline": bond,
            "dipole_plan": {"kind": {0: "auto", 1: "ordered", 2: "symmetric"}[plan[0]], "param": plan[1],
                            "bond_beside_dipole": bool(overlap[0]),
                            "dipole_blocks_beside_bond": overlap[1] or None,
                            "bond_blocks_beside_dipole": overlap[2] or None},
            "dominant": dominant, "roofline": roof,
            "launches_per_step": sum(timing[k]["launches"] for k in timing) / ksteps}


# variants reported beside the default workload: name -> (workload, the FP64
# plain workload its speedup is quoted against)
VARIANTS = {
    "cilia_float_float": ("cilia_512x256_ff", "cilia_512x256_fp64"),
    "cilia_fp32_pair_fp64_accum": ("cilia_512x256_mixed", "cilia_512x256_fp64"),
    "batched_rods_fp64": ("batched_rods_2048_fp64", "batched_rods_2048_fp64"),
    "batched_rods_fp32_pair_fp64_accum": ("batched_rods_2048_mixed", "batched_rods_2048_fp64"),
    "batched_rods_float_float": ("batched_rods_2048_ff", "batched_rods_2048_fp64"),
    "helix_fp64": ("helix_16384", "helix_16384"),
    "helix_fp32_pair_fp64_accum": ("helix_16384_mixed", "helix_16384"),
    "helix_float_float": ("helix_16384_ff", "helix_16384"),
}


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
    pk = pipe_peaks(n_sm, sm_max)
    stream = torch.cuda.Stream(device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    timing_steps = max(1, min(args.steps, 5))
    plan = tuple(int(v) for v in args.dipole_plan.split(":")) if args.dipole_plan else None

    # ---- the headline workload; clocks sampled over its timed steps
    sampler = ClockSampler(local_rank)
    sim = bpm.Simulation(sysm, stream=stream.cuda_stream)
    if plan:
        sim.set_dipole_plan(*plan)
    if args.overlap != -1:
        sim.set_overlap(args.overlap)
    f0, t0 = sim.forces()
    for _ in range(args.warmup):
        with torch.cuda.stream(stream):
            flush.zero_()
        sim.step(1)
    sampler.start()
    barrier(world, dev)
    torch.cuda.synchronize()
    ms = _timed_steps(sim, torch, stream, flush, args.steps)
    torch.cuda.synchronize()
    barrier(world, dev)
    clocks = sampler.stop()
    sim.set_timing(True)
    _timed_steps(sim, torch, stream, flush, timing_steps)
    timing = sim.timing()
    sim.set_timing(False)
    info = describe(sysm, sim, timing, timing_steps, pk, args.workload)
    ms_max = reduce_max(ms, world, dev)
    value = aggregate(sysm.n, ms_max / 1e3, world)
    pairs_per_s = aggregate(float(sysm.ordered_pairs()), ms_max / 1e3, world)
    roof = info["roofline"]
    if roof is None or info["dominant"] in ("lbm", "contact"):
        hbm = float(peaks.get("hbm_gbs", 6800.0))
        hbm_note = ("measured HBM copy bandwidth (MEASURED_PEAKS.json hbm_gbs)" if "hbm_gbs" in peaks
                    else "fallback HBM 6800 GB/s")
        if info["dominant"] == "lbm":
            roof = _lbm_roofline(timing, sysm, pk["fp64_tflops"], 2 * pk["fp32_tops"],
                                 (pk["fp64_source"], pk["fp32_source"]), hbm, hbm_note)
        elif sysm.contact is not None:
            roof = _contact_roofline(timing, sysm, pk["fp64_tflops"], pk["fp64_source"], hbm, hbm_note)

    # ---- end to end through the public API with pinned host buffers: the
    # step's input state and forces uploaded (bpm_set_state, bpm_set_forces),
    # one step, the new state and forces read back, every step
    n = sysm.n
    pin = {k: torch.empty((n, c), dtype=torch.float64, pin_memory=True).numpy()
           for k, c in (("x", 3), ("q", 4), ("v", 3), ("w", 3), ("f", 3), ("tau", 3))}
    tcur = bpm.bpm_get_state(sim.h, pin["x"], pin["q"], pin["v"], pin["w"])
    bpm.bpm_get_forces(sim.h, pin["f"], pin["tau"])
    k_e2e = max(3, min(args.steps, 10))
    barrier(world, dev)
    torch.cuda.synchronize()
    t_e = time.perf_counter()
    for _ in range(k_e2e):
        bpm.bpm_set_state(sim.h, pin["x"], pin["q"], pin["v"], pin["w"], tcur)
        bpm.bpm_set_forces(sim.h, pin["f"], pin["tau"])
        sim.step(1)
        tcur = bpm.bpm_get_state(sim.h, pin["x"], pin["q"], pin["v"], pin["w"])
        bpm.bpm_get_forces(sim.h, pin["f"], pin["tau"])
    torch.cuda.synchronize()
    e2e_s = reduce_max((time.perf_counter() - t_e) / k_e2e, world, dev)
    state_bytes = n * 19 * 8
    sim.close()

    # ---- error of the headline's step-1 forces against the CPU FP64 oracle
    def system_key(wl):
        # one oracle reference per system, shared by its precisions
        return wl.replace("_ff", "").replace("_mixed", "").replace("_fp64", "")

    refs = {}
    error = None
    if rank == 0 and not args.no_oracle_error:
        refs[system_key(args.workload)] = OracleReference(sysm)
        error = refs[system_key(args.workload)].error(f0, t0)

    # ---- variants: other precisions and workloads
    variants = {}
    fp64_ms = {args.workload: ms_max}
    if args.workload == DEFAULT_WORKLOAD and not args.no_variants:
        for vname, (wl, base) in VARIANTS.items():
            vs = WORKLOADS[wl]()
            try:
                vsim, (vf, vt), vms, vtiming, vk = measure(bpm, torch, vs, stream, flush, args.steps,
                                                           args.warmup, timing_steps)
            except bpm.BpmError as e:
                # reported, not hidden: the variant's line carries the error
                variants[vname] = {"workload": wl, "error": str(e)}
                print(f"variant {vname} ({wl}) failed: {e}", file=sys.stderr, flush=True)
                continue
            vinfo = describe(vs, vsim, vtiming, vk, pk, wl)
            chained = None
            if vs.n * STATE_BYTES_PER_PARTICLE > 2 * L2_BYTES:
                chained = reduce_max(chained_ms(vsim, torch, stream, vs.n_steps), world, dev)
            vsim.close()
            vms = reduce_max(vms, world, dev)
            if wl == base:
                fp64_ms[wl] = vms
            rec = {"workload": wl, "value": aggregate(vs.n, vms / 1e3, world), "unit": UNIT, "ms_per_step": vms,
                   "pairs_per_s": aggregate(float(vs.ordered_pairs()), vms / 1e3, world),
                   "precision": _config(vs, argparse.Namespace(workload=wl))["precision"],
                   "speedup_vs_fp64": (fp64_ms[base] / vms) if base in fp64_ms else None,
                   **{k: vinfo[k] for k in ("kernel_ms_per_step", "dipole_plan", "roofline", "bond_roofline")}}
            if chained is not None:
                rec["chained"] = {"ms_per_step": chained, "value": aggregate(vs.n, chained / 1e3, world),
                                  "note": f"one bpm_step({vs.n_steps}) call, the configuration's horizon: the "
                                          "16-step CUDA graphs back to back, no host synchronisation between "
                                          f"steps; the working set (about {vs.n * STATE_BYTES_PER_PARTICLE / 1e6:.0f}"
                                          " MB) exceeds L2"}
            if rank == 0 and not args.no_oracle_error:
                key = system_key(wl)
                if key not in refs:
                    refs[key] = OracleReference(vs)
                rec["error_vs_oracle"] = refs[key].error(vf, vt)
            variants[vname] = rec

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu, _ = time_oracle(sysm)

    if rank == 0:
        fp64 = sysm.precision == W.PRECISION_FP64
        ff = sysm.precision == W.PRECISION_FF
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None,
                "dtype": "f64" if fp64 else ("f32x2 float-float pairs/f64-accum" if ff else "f32-pair/f64-accum"),
                "data": "synthetic",
                "config": _config(sysm, args), "pairs_per_s": pairs_per_s,
                "timing": "value: bpm_step(1) replayed from CUDA graphs between CUDA events, L2 flushed before "
                          "each step; kernel_ms_per_step and roofline: a second pass of "
                          f"{timing_steps} steps with the library's kernel events",
                "roofline": roof, "cpu_baseline": cpu, "error_vs_oracle": error,
                "e2e": {"value": aggregate(n, e2e_s, world), "unit": UNIT,
                        "h2d_bytes_per_step": state_bytes, "d2h_bytes_per_step": state_bytes,
                        "note": "per step: bpm_set_state and bpm_set_forces from pinned host buffers, "
                                "bpm_step(1), bpm_get_state and bpm_get_forces to pinned host buffers "
                                "(x, q, v, omega, f, tau: 19 doubles per particle each way)"},
                "gpu_launches": int(round(info["launches_per_step"] * args.steps)),
                "kernel_ms_per_step": info["kernel_ms_per_step"], "dipole_plan": info["dipole_plan"],
                "bond_roofline": info["bond_roofline"],
                "peaks": {"fp64_tflops": pk["fp64_tflops"], "fp32_tops": pk["fp32_tops"],
                          "measured": pk["measured"]},
                "clocks": clocks, "variants": variants}
        if info["dipole_plan"]["bond_beside_dipole"]:
            line["kernel_ms_note"] = ("the bond kernel runs on a second stream beside the dipole kernel: their "
                                      "per-launch times overlap and include the sharing of the SMs")
        if args.workload == "adjoint_rod_2048":
            line["adjoint"] = run_adjoint_bench(bpm, torch, sysm, stream)
        print(json.dumps(line), flush=True)


def run_adjoint_bench(bpm, torch, sysm, stream):
    """The adjoint of the time stepping (magnetisation-profile design):
    forward with checkpoints, then the reverse sweep, in FP64 and on a
    BPM_FF handle."""
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
    f2, r2, gm2, gB2 = run_adjoint(W.PRECISION_FF)
    scale = max(np.abs(gm).max(), np.abs(gB).max())
    adjoint["float_float"] = {
        "forward_ms": f2, "reverse_ms": r2, "speedup_vs_fp64": (f_ms + r_ms) / max(f2 + r2, 1e-12),
        "max_gradient_diff_vs_fp64": float(max(np.abs(gm2 - gm).max(), np.abs(gB2 - gB).max()) / scale)}
    return adjoint


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50,
                    help="timed steps (default 50, the cilia configuration's horizon: about 40 s of timed work)")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=sorted(WORKLOADS))
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-variants", action="store_true", help="skip the other precisions and workloads")
    ap.add_argument("--no-oracle-error", action="store_true", help="skip the errors against the CPU FP64 oracle")
    ap.add_argument("--peaks", action="store_true", help="measure the pipe throughputs, write " + PEAKS_EXT)
    ap.add_argument("--record-traffic", default="", metavar="NCU_RAW_CSV",
                    help="store the DRAM bytes per launch of --kernel on --workload from an ncu raw CSV export")
    ap.add_argument("--kernel", default="", help="kernel name prefix for --record-traffic")
    ap.add_argument("--traffic-scale", type=float, default=1.0,
                    help="units of a full launch over units of the captured launch (--record-traffic)")
    ap.add_argument("--traffic-note", default="", help="how the capture was made (--record-traffic)")
    ap.add_argument("--dipole-plan", default="", metavar="KIND:PARAM",
                    help="fix the dipole plan instead of autotuning it (1:chunks ordered, 2:g symmetric)")
    ap.add_argument("--overlap", type=int, default=-1, choices=[-1, 0, 1],
                    help="bond kernel beside the dipole kernel: -1 tuned (default), 0 never, 1 whenever possible")
    args = ap.parse_args(argv)
    if args.record_traffic:
        record_traffic(args.record_traffic, args.kernel, args.workload, args.traffic_scale, args.traffic_note)
        return
    if args.peaks:
        run_peaks(args)
        return
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
