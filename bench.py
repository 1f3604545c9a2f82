#!/usr/bin/env python3
"""NEP molecular-dynamics throughput on GB300: atom-steps/s of plain FP32 NEP-MD.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--workload NAME]
                    [--form plain|mix_bf16|mix_fp16|student|student_bf16_fallback|student_fallback] [--no-configs]

One step = one velocity-Verlet MD step of the whole hot path on the 1,048,576-atom fcc Cu workload
(64x64x64 cells, 300 K, 1 fs): half kick + drift, neighbour-rebuild check (a rebuild runs every 10
steps -- the refresh interval of the paper's MD protocol -- and whenever an atom moved more than
skin/2), cell sort + neighbour list when rebuilding, descriptors + network, forces + virial, half
kick, energy/virial/kinetic sums.  Inputs are resident in HBM when the timed region starts.  The
timed region replays the captured CUDA graph of one MD step, the launch path md_verlet_step uses; the
per-kernel breakdown ("kernels") and the roofline come from an eager pass of the same length with
per-kernel-class CUDA events.  The roofline's peak is the FP32 throughput measured in the same run by
the library's microbenchmark (nep_fp32_peak), with the SM clock sampled during it.

--form selects the form whose throughput is the headline value (default: plain FP32).  The other
forms are then timed on the same workload and start state ("forms": atom-steps/s, speedup, and force
RMSE/max against the plain FP32 forces on 8,192 sampled atoms; their error against the FP64 oracle is
a GPU test).  "configs" (default run, --no-configs skips it) times the forms on the 16,384,000-atom
workload at 300 K and from the 1200 K start, and the plain teacher against the student with teacher
fallback on the 131,027,885-atom void workload, each with its own clocks.

N > 1 (torchrun): every rank runs an independent replica on its own GPU (no collective on the data
path); value = atom-steps of all ranks / max-over-ranks time ("scaling": "weak").

--impl reference times the FP64 CPU oracle (the method as written, plain C) on the host cores for
the same metric on the same workload: one velocity-Verlet call over a bounded number of steps.
"""
from __future__ import annotations

import argparse
import hashlib
import json
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

import nep_inputs as ni  # noqa: E402

METRIC = "NEP MD atom-steps/s on 1 GB300: plain FP32 vs mixed/student at stated force RMSE"
UNIT = "atom-steps/s"

# Algorithmic FP32 FLOPs of the method per unit: a static count of the arithmetic each unit needs in the
# kernels (FMA = 2, add/mul = 1, each transcendental = 1, a packed float2 operation counts both halves),
# for the compiled teacher shape (5 radial + 5 angular channels, 8 basis functions, l = 1..4, 4-body,
# 30 neurons).  Fixed-point conversions of the force scatter and of the sums, the stand-in pairs of
# lanes that only take part in warp-collective loads and the zero padding of the network row are not
# counted.  Pieces (teacher shape):
#   list entry 11: displacement (6 adds) and r^2 (1 mul + 2 FMA);
#   active pair, descriptor 2: rsqrt and r;
#   radial pair, descriptor 38: the Chebyshev factors 22 (r/rc, pi r/rc and the hardware cosine 3, the
#     cutoff half h = (1 + cos) / 4 as one FMA 2, x = 2 (r/rc - 1)^2 - 1 5, 6 recurrence FMAs 12) and the
#     sums h T_k in 4 paired FMAs 16 (sum f_k = sum h T_k + sum h: 8 adds per atom); the angular basis
#     f_k = h (T_k + 1) of an angular pair is formed (40);
#   LJ pair, descriptor 15: 1/r^2 with one Newton step 5, r^-6 2, the shifted energy factored as
#     r^-6 (c12 r^-6 - c6) + (rc E'(rc) - E(rc)) - r E'(rc) in three FMAs 6, half of it summed 2;
#   angular pair, descriptor 410: unit vector 3 + basis 40 + 5 channel dot products 75 + the 24
#     harmonic polynomials without their constant factors 52 (the fused kernels keep the sums and the
#     adjoint row over Ph_lm = Yh_lm / hnorm(lm); with the constants, as the separate kernels, 81) +
#     120 paired FMAs into s_nlm 240;
#   atom, descriptor 5114: the radial sums' 8 adds, q_n 80, q_nl 335 (240 + the 95 hnorm scalings of the sums), 4-body tensors and
#     q4 130, network 3870 (scaling 60 and 30 neurons x (30 FMAs forward, tanh, energy, gradient
#     factor, 30 FMAs back)), 4-body adjoint 350 (330 + 20 scalings), adjoint row 260 (G' = 2 hnorm^2 Fp
#     s' + hnorm f4 g4: 16 distinct hnorm^2 Fp factors per channel 80, 120 products, 10 hnorm f4
#     factors, 25 FMAs), radial adjoint in basis space 80, site energy 1;
#   active pair, force from the pair records 28: r^2, rsqrt, r (7), d = coef r + v (6), F_i (3),
#     virial upper triangle (12); the list-walking force kernel: 23 plus 11 per list entry;
#   radial pair, force 80 (fused kernels): the Chebyshev factors and their derivatives 50 (h, h', x'(r) h,
#     T_k and T_k' recurrences) and the radial-adjoint contraction h' sum t_k T_k + x' h sum t_k T_k'
#     without forming the f_k' 30 (paired, two records per iteration; 84 one at a time: the angular
#     pairs' radial part, +4 in their angular count, and the student); the list-walking force kernels
#     form the f_k': 117 (basis and derivative 101 + dot with the radial adjoint 15 + 1/r);
#   LJ pair, force 15: 1/r^2, r^-6 (7), dE/dr = r^-6 (-12 c12 r^-6 + 6 c6) / r - E'(rc) (5), half of it / r
#     added to the pair coefficient (3);
#   angular pair, force 1109 (fused kernels, over Ph_lm): 4 for its radial part one at a time + unit vector 3 + basis and derivative 101 +
#     2 x 5 channel dots 150 + the polynomials 52 + per (l, m) the sums A_lm, B_lm over the channels 480
#     + (A - l B / r) Ph 96 + the l / r factors 12 + the polynomials' gradients 86 and their 58 non-zero
#     FMAs 116 + 9; the list-walking force kernels over Yh_lm: 1177 (harmonics 81, gradients 129);
#   the half-list force (float16 rows): H = G^i + (-1)^l G^j adds 240 per angular pair and 8 per radial
#     pair; its LJ term is the whole pair force (14).
# The FP32 op counters of one fused launch (ffma, fadd, fmul, paired ops, MUFU) agree with this count to
# within the conversions and padding named above (profiles/k_nep_fused_cu64x64x64.md).
# The mixed-precision forms run the same fused kernel with the network as two tensor-core GEMMs
# (32 x 32 tiles, bf16/f16 operands): per atom 1514 FP32 FLOPs remain (5114 - 3870 for the float32
# network + scaling 30, per neuron z - b0, tanh, energy FMA and gradient factor 7, Fp 30); the GEMMs'
# 4096 tensor FLOPs per atom are not part of the FP32 count.
FLOPS = {
    "descriptor": dict(list_entry=11, active_pair=2, radial_pair=38, lj_pair=15, angular_pair=410, atom=5114),
    "descriptor_mixed": dict(list_entry=11, active_pair=2, radial_pair=38, lj_pair=15, angular_pair=410, atom=1514),
    "force_rec": dict(list_entry=0, active_pair=28, radial_pair=80, lj_pair=15, angular_pair=1109, atom=0),
    "force_full": dict(list_entry=11, active_pair=23, radial_pair=117, lj_pair=15, angular_pair=1177, atom=0),
    "force": dict(list_entry=11, active_pair=23, radial_pair=125, lj_pair=14, angular_pair=1417, atom=0),
}
# The same count for the student shape (4 + 4 channels, 8 basis functions, l = 1, 2, no 4-body term,
# 16 neurons): register-resident sums, scalar channel dots (16 per channel), 8 harmonics (14),
# network 888.  Its float32 form runs the fused kernel, which keeps the sums and the adjoint row over
# the polynomials without their constant factors as the teacher's fused kernels do: the 8 polynomials
# cost 10 (descriptor_rec: 182 per angular pair; per atom 1169, the 16 hnorm scalings of the sums and 8
# more adjoint factors), and its force pass over the pair records per angular pair: unit vector 3 +
# basis and derivative 101 + 2 x 4 channel dots 120 + polynomials 10 + the sums A_lm, B_lm 128 +
# (A - l B / r) Ph 32 + the l / r factors 8 + the polynomials' gradients 3 and their 14 non-zero FMAs
# 28 + 9; its mixed form runs the separate kernels (harmonics with their constants) with the force over
# the half list.
FLOPS_STUDENT = {
    "descriptor": dict(list_entry=11, active_pair=2, radial_pair=38, lj_pair=15, angular_pair=185, atom=1153),
    "descriptor_rec": dict(list_entry=11, active_pair=2, radial_pair=38, lj_pair=15, angular_pair=181, atom=1177),
    "force": dict(list_entry=11, active_pair=23, radial_pair=125, lj_pair=14, angular_pair=510, atom=0),
    "force_rec": dict(list_entry=0, active_pair=28, radial_pair=84, lj_pair=15, angular_pair=442, atom=0),
}
# Algorithmic HBM bytes per atom-step: the integrator reads and writes x, v (96) in the kick + drift and
# v (48) in the second kick, and reads the forces in both kicks (48); the force kernel reads the atom's
# position (16) and its walked neighbour-list entries (4 each), writes the site energy (4) and the
# forces (24).  The neighbour build is amortised over the rebuild interval and not counted.
BYTES = dict(per_atom=96 + 48 + 48 + 16 + 4 + 24, per_list_entry=4)


def force_kind(form: str) -> str:
    """FLOP table of the force pass a form runs: the fused kernels' pass over their pair records for the
    teacher (float32 or mixed-precision network) and the float32 student, the half list for the
    student's mixed-precision form."""
    f = FORMS[form]
    return "force_rec" if f["model"] == "teacher" or f["precision"] == "fp32" else "force"


def descriptor_kind(form: str) -> str:
    """FLOP table of the descriptor part: the mixed-precision teacher forms' network is on the tensor
    cores; the float32 student runs its fused kernel (descriptor_rec of FLOPS_STUDENT)."""
    f = FORMS[form]
    if f["model"] == "student":
        return "descriptor_rec" if f["precision"] == "fp32" else "descriptor"
    return "descriptor_mixed" if form in ("mix_bf16", "mix_fp16") else "descriptor"


def kernel_flops(kind: str, c: dict, n_atoms_evals: int, table: dict = FLOPS) -> float:
    f = table[kind]
    if kind.startswith("descriptor"):
        lst, act, rad, ang = c["list_entries"], c["active_pairs"], c["radial_pairs"], c["angular_pairs"]
    else:
        lst, act, rad, ang = (c["force_list_entries"], c["force_active_pairs"], c["force_radial_pairs"],
                              c["force_angular_pairs"])
    return (f["list_entry"] * lst + f["active_pair"] * act + f["radial_pair"] * rad + f["lj_pair"] * rad +
            f["angular_pair"] * ang + f["atom"] * n_atoms_evals)


# The sources each profiled kernel is built from: a committed traffic figure is used only while they
# are unchanged (kernel names as in profiles/traffic_per_launch.txt; ":form" for the non-plain forms).
_CORE = ("nep_common.cuh", "nep_descriptor.cuh", "nep_tc.cuh")
KERNEL_SOURCES = {
    "neighbors": ("nep_neighbor.cu", "nep_common.cuh"),
    "descriptor": ("nep_force.cu",) + _CORE,
    "force": ("nep_force.cu",) + _CORE,
    "fused": ("nep_force.cu",) + _CORE,
    "fused:mix_bf16": ("nep_force.cu",) + _CORE,
    "fused:mix_fp16": ("nep_force.cu",) + _CORE,
    "fused:student": ("nep_force.cu",) + _CORE,
    "descriptor:student_bf16_fallback": ("nep_mixed.cu", "nep_fallback.cu") + _CORE,
    "force:student_bf16_fallback": ("nep_force.cu", "nep_fallback.cu") + _CORE,
}
SOURCE_FILES = tuple(sorted({f for v in KERNEL_SOURCES.values() for f in v}))


def source_hash(kernel: str | None = None) -> str:
    """Hash of the sources of `kernel` (all kernel sources when None)."""
    files = SOURCE_FILES if kernel is None else KERNEL_SOURCES.get(kernel, SOURCE_FILES)
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, "paper_2604_24816_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def profiled_traffic(kernel: str):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, if it was captured on the
    current kernel source; else None."""
    path = os.path.join(ROOT, "profiles", "traffic_per_launch.txt")
    if not os.path.exists(path):
        return None
    cur = source_hash(kernel)
    for line in open(path):
        parts = line.split()
        if len(parts) >= 4 and parts[0] == kernel and parts[1] == cur:
            return dict(bytes=float(parts[2]), atoms=int(parts[3]))
    return None


# ---------------------------------------------------------------------------------------------------
class ClockSampler:
    """nvidia-smi clocks/throttle reasons sampled every 50 ms in a background thread."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.samples = []
        self.proc = None
        self.window = None
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "50", "-i", str(gpu_index)], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
        except OSError:
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.samples.append((time.perf_counter(), line.strip()))

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self, t0: float, t1: float) -> dict:
        rows = [s for t, s in self.samples if t0 <= t <= t1]
        if len(rows) < 3:        # very short timed region: widen to the nearest samples around it
            rows = [s for t, s in self.samples if t0 - 0.5 <= t <= t1 + 0.5]
        sm, smax, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for r in rows:
            p = [x.strip() for x in r.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1])); smax.append(float(p[2]))
            except ValueError:
                continue
            for k, nm in enumerate(names):
                if p[5 + k].lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------------------------------
def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    if ws <= 1:
        return 0, 1, 0
    import torch.distributed as dist
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", str(rank)))
    import torch
    backend = "nccl" if torch.cuda.is_available() else "gloo"
    dist.init_process_group(backend=backend)
    return rank, ws, local


def dist_barrier(ws: int):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def dist_max(x: float, ws: int, device=None) -> float:
    """Max of a scalar over ranks (identity at world size 1)."""
    if ws <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def dist_sum(x: float, ws: int, device=None) -> float:
    if ws <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def load_peaks() -> dict:
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        d["source"] = "measured"
        return d
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0, "source": "fallback"}


def cpu_baseline(seconds_hint: float = 15.0) -> dict:
    """The FP64 oracle, as it stands, timed on the host cores on a bounded sample of the workload: a
    2-step probe on 16x16x16 cells sets the number of steps that fills about `seconds_hint` seconds,
    and that run is the one reported."""
    import oracle
    oracle.build()
    cores = os.cpu_count() or 1
    oracle.set_threads(cores)
    model = oracle.load_model(os.path.join(ROOT, "paper_2604_24816_gb300", "params", "cu_nep4_synth.json"))
    wl = ni.workload("cu_16x16x16")
    t0 = time.perf_counter()
    oracle.md_nve(model, wl.pos, wl.vel, wl.box, ni.M_CU, 1.0, 2)
    per_step = (time.perf_counter() - t0) / 3.0          # 2 steps = 3 force evaluations
    steps = int(min(200, max(2, seconds_hint / max(per_step, 1e-3))))
    t0 = time.perf_counter()
    oracle.md_nve(model, wl.pos, wl.vel, wl.box, ni.M_CU, 1.0, steps)
    dt = time.perf_counter() - t0
    used = oracle.get_threads()
    # the same oracle on one thread, 2 steps (a few seconds)
    oracle.set_threads(1)
    t1 = time.perf_counter()
    oracle.md_nve(model, wl.pos, wl.vel, wl.box, ni.M_CU, 1.0, 2)
    dt1 = time.perf_counter() - t1
    oracle.set_threads(cores)
    return {"value": wl.n * steps / dt, "unit": UNIT, "cores": used, "kind": "oracle",
            "sample": f"fcc Cu 16x16x16 cells ({wl.n} atoms), {steps} velocity-Verlet steps "
                      f"({steps + 1} force evaluations, fresh neighbour search each), FP64, {dt:.1f} s",
            "value_1_thread": wl.n * 2 / dt1, "sample_1_thread": f"same cell, 2 steps on 1 thread, {dt1:.1f} s"}


# ---------------------------------------------------------------------------------------------------
REFERENCE_BUDGET_S = 150.0


def run_reference(args, rank: int, ws: int):
    """Reference arm: the FP64 CPU oracle timed on the host cores (rank 0 only), on the GPU arm's
    workload.  One oracle velocity-Verlet call over k steps does k + 1 force evaluations (the call
    starts with the forces of the initial state); a warm-up call of 0 steps times that initial
    evaluation alone, and it is subtracted, so the value counts k steps of one evaluation each.  k is
    --steps, bounded so that the whole arm takes about REFERENCE_BUDGET_S seconds."""
    if rank != 0:
        return
    import oracle
    oracle.build()
    cores = os.cpu_count() or 1
    oracle.set_threads(cores)
    model = oracle.load_model(os.path.join(ROOT, "paper_2604_24816_gb300", "params", "cu_nep4_synth.json"))
    wl = ni.workload(args.workload)
    t0 = time.perf_counter()
    oracle.md_nve(model, wl.pos, wl.vel, wl.box, ni.M_CU, wl.dt_fs, 0)
    t_eval = time.perf_counter() - t0
    k = int(max(1, min(args.steps, (REFERENCE_BUDGET_S - 2 * t_eval) // max(t_eval, 1e-6))))
    t0 = time.perf_counter()
    oracle.md_nve(model, wl.pos, wl.vel, wl.box, ni.M_CU, wl.dt_fs, k)
    dt = max(time.perf_counter() - t0 - t_eval, 1e-9)
    value = wl.n * k / dt
    sample = (f"{args.workload} ({wl.n} atoms), {k} velocity-Verlet steps of the FP64 oracle in one call, one force "
              f"evaluation per step (the call's initial evaluation, {t_eval:.1f} s, timed alone and subtracted)"
              + ("" if k == args.steps else f"; {k} of the requested {args.steps} steps (time bound)"))
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": k,
        "warmup": 1, "ms_per_step": 1e3 * dt / k, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "atoms_per_gpu": wl.n, "sample": sample,
                   "parallelism": "host cores (OpenMP)",
                   "warmup": (f"one initial force evaluation (timed alone, then subtracted) instead of the requested "
                              f"{args.warmup} steps: the CPU program has no caches or graphs to warm, and each "
                              f"oracle step at this size takes {t_eval:.0f} s")},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.get_threads(), "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def measure_fp32_peak(stream, local: int) -> dict:
    """FP32 throughput of this GPU (nep_fp32_peak: FMA chains on every SM, packed float2 and scalar):
    median over 60 launches of ~5 ms each, the FMAs per SM clock cycle counted in the kernel, and the
    SM clock sampled while it runs.  The peak is the faster form's median."""
    from paper_2604_24816_gb300 import fp32_peak
    clocks = ClockSampler(local)
    time.sleep(0.2)
    t0 = time.perf_counter()
    packed = fp32_peak(True, 5.0, 60, stream.cuda_stream)
    scalar = fp32_peak(False, 5.0, 60, stream.cuda_stream)
    half2 = fp32_peak("half2", 5.0, 20, stream.cuda_stream)
    t1 = time.perf_counter()
    clocks.stop()
    top = packed if packed["median_tflops"] >= scalar["median_tflops"] else scalar
    sms = top["sm_count"]
    return {"tflops": top["median_tflops"], "form": "packed float2" if top is packed else "scalar",
            "packed_tflops": packed["median_tflops"], "scalar_tflops": scalar["median_tflops"],
            "packed_best_tflops": packed["best_tflops"],
            "fma_per_clock_sm": {"packed": round(packed["fma_per_clock_sm"], 2),
                                 "scalar": round(scalar["fma_per_clock_sm"], 2),
                                 "half2": round(half2["fma_per_clock_sm"], 2)},
            "half2_tflops": half2["median_tflops"],
            "implied_sm_mhz": (round(top["median_tflops"] * 1e6 / (2 * sms * top["fma_per_clock_sm"]), 1)
                               if top["fma_per_clock_sm"] > 0 else None),
            "sm_count": sms, "clocks": clocks.summary(t0, t1)}


# form name -> library precision, model (teacher or distilled student), per-atom fallback to the
# teacher, arithmetic types, description
_MIX = ("network GEMMs on tcgen05 tensor cores with {} operands and f32 accumulation inside the fused "
        "kernel, FP32 descriptors and forces, float64 integration and sums")
_MIX_STUDENT = ("network GEMMs on tcgen05 tensor cores with {} operands and f32 accumulation, float16 adjoint "
                "rows between its descriptor and half-list force kernels, FP32 descriptors and forces, float64 "
                "integration and sums")
FORMS = {
    "plain": dict(precision="fp32", model="teacher", fallback=False, dtype="f32",
                  desc="plain FP32 NEP, seeded teacher weights (float64 integration and sums)"),
    "mix_bf16": dict(precision="mix_bf16", model="teacher", fallback=False, dtype="bf16/f32",
                     desc="mixed precision: " + _MIX.format("bf16")),
    "mix_fp16": dict(precision="mix_fp16", model="teacher", fallback=False, dtype="f16/f32",
                     desc="mixed precision: " + _MIX.format("f16")),
    "student": dict(precision="fp32", model="student", fallback=False, dtype="f32",
                    desc="distilled student NEP (n_max 3/3, l_max 2, no 4-body, 16 neurons), FP32"),
    "student_bf16_fallback": dict(precision="mix_bf16", model="student", fallback=True, dtype="bf16/f32",
                                  desc="distilled student NEP, " + _MIX_STUDENT.format("bf16") + "; per-atom fallback to the "
                                       "FP32 teacher for atoms outside the student's training range (5 % margin)"),
    "student_fallback": dict(precision="fp32", model="student", fallback=True, dtype="f32",
                             desc="distilled student NEP, FP32 (one fused kernel); per-atom fallback to the FP32 teacher "
                                  "for atoms outside the student's training range (5 % margin)"),
}
FALLBACK_MARGIN = 0.05
STUDENT_PATH = os.path.join(ROOT, "paper_2604_24816_gb300", "params", "cu_student_trained.json")


def load_student() -> dict:
    with open(STUDENT_PATH) as f:
        return json.load(f)


def make_nep(form, teacher, student, stream, args):
    from paper_2604_24816_gb300 import NEP
    f = FORMS[form]
    h = NEP(student if f["model"] == "student" else teacher, stream=stream.cuda_stream,
            rebuild_every=args.rebuild_every, precision=f["precision"], max_neighbors=args.max_neighbors)
    if f["fallback"]:
        h.set_fallback(teacher, student["q_lo"], student["q_hi"], margin=FALLBACK_MARGIN)
    return h


def time_form(form, teacher, student, wl, args, stream, dev, ws, atoms_total):
    """Throughput of another form on the same workload and start state (warm-up, then --form-steps
    CUDA-graph MD steps timed with events), plus its forces on the start state."""
    import torch
    with make_nep(form, teacher, student, stream, args) as h:
        h.set_state(wl.pos, wl.vel, wl.box)
        _, F, _ = h.compute()
        h.step(wl.dt_fs, args.warmup)
        c0 = h.counters()
        s = torch.cuda.Event(enable_timing=True)
        e = torch.cuda.Event(enable_timing=True)
        dist_barrier(ws)
        torch.cuda.synchronize(dev)
        s.record(stream)
        h.step(wl.dt_fs, args.form_steps)
        e.record(stream)
        torch.cuda.synchronize(dev)
        ms = dist_max(s.elapsed_time(e), ws, dev)
        th = h.thermo()
        c1 = h.counters()
    rec = {"value": atoms_total * args.form_steps / (ms * 1e-3), "ms_per_step": ms / args.form_steps,
           "steps": args.form_steps, "dtype": FORMS[form]["dtype"], "pe_per_atom_end": th["pe"] / wl.n, "_F": F}
    if FORMS[form]["fallback"]:
        ev = max(1, c1["evaluations"] - c0["evaluations"])
        rec["fallback_fraction"] = (c1["fallback_atoms"] - c0["fallback_atoms"]) / (ev * wl.n)
    return rec


# Workloads of the "configs" block: (name, workload, forms, timed steps, neighbour-list capacity, probe
# sigma).  The forces compared between forms are those of the start state, unless the start positions
# are perfect lattice sites (the void workload: bulk forces cancel by symmetry there); then they are
# those of a probe state, the start positions with seeded N(0, sigma^2) displacements.
CONFIGS = (
    ("cu_160x160x160", "cu_160x160x160", ("plain", "mix_bf16", "mix_fp16"), 20, 0, None),
    ("cu_160x160x160_1200K", "cu_160x160x160_1200K", ("plain", "mix_bf16", "mix_fp16"), 20, 0, None),
    ("cu_320_void", "cu_320_void", ("plain", "student_bf16_fallback", "student_fallback"), 10, 96, 0.05),
)


def time_config_form(form, teacher, student, wl, steps, warmup, max_neighbors, idx, stream, dev, local, ws,
                     ablate=False, probe=None):
    """One form on one workload: forces on the sampled atoms (of `probe` positions if given, else of
    the start state), then `warmup` and `steps` CUDA-graph MD steps from the start state, the latter
    timed with events on the library's stream while the SM clock is sampled."""
    import torch
    from paper_2604_24816_gb300 import NEP
    f = FORMS[form]
    with NEP(student if f["model"] == "student" else teacher, stream=stream.cuda_stream, rebuild_every=10,
             precision=f["precision"], max_neighbors=max_neighbors) as h:
        if f["fallback"]:
            h.set_fallback(teacher, student["q_lo"], student["q_hi"], margin=FALLBACK_MARGIN)
        h.set_state(wl.pos if probe is None else probe, wl.vel, wl.box)
        Fd = torch.empty((wl.n, 3), dtype=torch.float64, device=dev)
        h.compute(out=Fd)
        F = Fd[torch.from_numpy(idx).to(dev)].cpu().numpy()
        del Fd
        if probe is not None:
            # back to the start state with a list built there (an upload keeps the probe state's list)
            h.set_state(wl.pos, wl.vel, wl.box)
            h.build_neighbors()
        h.step(wl.dt_fs, warmup)
        c0 = h.counters()
        clocks = ClockSampler(local)
        time.sleep(0.2)
        s = torch.cuda.Event(enable_timing=True)
        e = torch.cuda.Event(enable_timing=True)
        dist_barrier(ws)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        s.record(stream)
        h.step(wl.dt_fs, steps)
        e.record(stream)
        torch.cuda.synchronize(dev)
        t1 = time.perf_counter()
        clocks.stop()
        ms = dist_max(s.elapsed_time(e), ws, dev)
        th = h.thermo()
        c1 = h.counters()
        abl = None
        if form == "plain" and ablate:
            # the list-walking force kernels on the state after the timed steps (rows of unequal lengths)
            abl = {v + "_ms": round(min(h.run_variant(v)[0] for _ in range(2)), 3)
                   for v in ("separate_force", "cpb1", "cpb2", "cpb3")}
            p90, cpb = h.angular_p90()
            abl["cpb_rule"] = {"p90_angular_pairs": p90, "centres_per_warp": cpb}
    rec = {"value": dist_sum(wl.n, ws, dev) * steps / (ms * 1e-3), "ms_per_step": ms / steps, "steps": steps,
           "dtype": f["dtype"], "clocks": clocks.summary(t0, t1), "pe_per_atom_end": th["pe"] / wl.n,
           "rebuilds": c1["rebuilds"] - c0["rebuilds"] if "rebuilds" in c1 else None, "_F": F}
    if f["fallback"]:
        ev = max(1, c1["evaluations"] - c0["evaluations"])
        rec["fallback_fraction"] = (c1["fallback_atoms"] - c0["fallback_atoms"]) / (ev * wl.n)
    if abl is not None:
        rec["ablations"] = abl
    return rec


def run_configs(teacher, student, args, stream, dev, local, ws) -> dict:
    """The larger workloads: every form of CONFIGS on its workload, throughput and force RMSE / max
    against the plain float32 forces on 8,192 sampled atoms (of the start state or the probe state)."""
    import gc
    out = {}
    for name, wname, forms, steps, cap, probe_sigma in CONFIGS:
        t_gen = time.perf_counter()
        wl = ni.workload(wname)
        probe = (None if probe_sigma is None else
                 ni.gaussian_displace(wl.pos, wl.box, probe_sigma, np.random.default_rng(13)))
        t_gen = time.perf_counter() - t_gen
        idx = ni.sample_indices(wl.n, 8192, seed=11)
        recs = {}
        for form in forms:
            recs[form] = time_config_form(form, teacher, student, wl, steps, 3, cap, idx, stream, dev, local, ws,
                                          ablate=name == "cu_160x160x160_1200K", probe=probe)
        Fp = recs["plain"]["_F"]
        for form, rec in recs.items():
            d = rec.pop("_F") - Fp
            if form != "plain":
                rec["force_rmse_vs_plain"] = float(np.sqrt(np.mean(d ** 2)))
                rec["force_max_vs_plain"] = float(np.abs(d).max())
                rec["speedup_vs_plain"] = round(rec["value"] / recs["plain"]["value"], 4)
        out[name] = {"atoms": wl.n, "temperature_K": wl.temperature, "input_generation_s": round(t_gen, 1),
                     "forces_compared_on": ("start state" if probe is None else
                                            f"probe state: start positions + N(0, {probe_sigma}^2) A displacements"),
                     "forms": recs}
        del wl, probe
        gc.collect()
    return out


def run_ours(args, rank: int, ws: int, local: int):
    import torch
    from paper_2604_24816_gb300 import load_model, build

    build.build()
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    model = load_model()
    student = load_student()
    wl = ni.workload(args.workload)       # every rank runs an independent replica of the same workload
    stream = torch.cuda.Stream(device=dev)
    peak = measure_fp32_peak(stream, local)
    nep = make_nep(args.form, model, student, stream, args)
    nep.set_state(wl.pos, wl.vel, wl.box)
    nep.compute(forces=False)

    # warm-up (untimed) on both launch paths.  The timed region replays the captured CUDA graph of one
    # MD step (what md_verlet_step runs); a second pass of the same length launches eagerly with
    # per-kernel-class CUDA events and gives the kernel breakdown and the roofline.
    nep.set_timing(True)
    nep.step(wl.dt_fs, args.warmup)
    nep.set_timing(False)
    nep.step(wl.dt_fs, args.warmup)
    torch.cuda.synchronize(dev)
    c0 = nep.counters()
    th0 = nep.thermo()
    clocks = ClockSampler(local)
    time.sleep(0.3)

    start = torch.cuda.Event(enable_timing=True)
    end = torch.cuda.Event(enable_timing=True)
    dist_barrier(ws)
    torch.cuda.synchronize(dev)
    t_host0 = time.perf_counter()
    start.record(stream)
    nep.step(wl.dt_fs, args.steps)
    end.record(stream)
    torch.cuda.synchronize(dev)
    t_host1 = time.perf_counter()
    dist_barrier(ws)
    ms = start.elapsed_time(end)
    ms_max = dist_max(ms, ws, dev)
    atoms_total = dist_sum(wl.n, ws, dev)
    value = atoms_total * args.steps / (ms_max * 1e-3)

    c1 = nep.counters()
    th = nep.thermo()
    dg = {k: c1[k] - c0[k] for k in c1}          # the timed (graph) region
    nep.set_timing(True)
    t_host2 = time.perf_counter()
    nep.step(wl.dt_fs, args.steps)
    torch.cuda.synchronize(dev)
    t_host3 = time.perf_counter()
    clocks.stop()
    tim = nep.timing()
    c2 = nep.counters()
    dc = {k: c2[k] - c1[k] for k in c2}          # the eager pass with per-kernel events
    evals = dc["evaluations"]
    table = FLOPS_STUDENT if FORMS[args.form]["model"] == "student" else FLOPS
    f_desc = kernel_flops(descriptor_kind(args.form), dc, evals * wl.n, table)
    f_force = kernel_flops(force_kind(args.form), dc, evals * wl.n, table)
    clk = clocks.summary(t_host0, t_host1)
    clk_kernels = clocks.summary(t_host2, t_host3)
    kern = {k: {"ms": round(v[0], 4), "launches": v[1]} for k, v in tim.items()}
    fused = tim["descriptor"][1] == 0 and tim["force"][1] > 0      # one kernel does descriptors and forces
    dominant = "force" if fused else max(("descriptor", "force"), key=lambda k: tim[k][0])
    dom_flops = f_desc + f_force if fused else (f_force if dominant == "force" else f_desc)
    dom_ms = tim[dominant][0]
    dom_launches = max(1, tim[dominant][1])
    achieved = dom_flops / (dom_ms * 1e-3) / 1e12
    kind = "fused" if fused else dominant
    traffic = profiled_traffic(kind if args.form == "plain" else f"{kind}:{args.form}")
    dom_name = (("k_nep_fused_reg" if FORMS[args.form]["model"] == "student" else
                 "k_nep_fused" if args.form == "plain" else "k_nep_fused_mixed") if fused else
                "k_descriptor_mixed" if dominant == "descriptor" and args.form != "plain" else f"k_{dominant}")
    pk_mhz, kn_mhz = peak["clocks"].get("sm_mhz"), clk_kernels.get("sm_mhz")
    roofline = {
        "bound": "alu",
        "kernel": dom_name, "achieved": round(achieved, 3), "peak": round(peak["tflops"], 2),
        "unit": "TFLOP/s", "frac": round(achieved / peak["tflops"], 4),
        "traffic": (round(traffic["bytes"] * wl.n / traffic["atoms"]) if traffic else None),
        "peak_source": (f"measured in this run: nep_fp32_peak FP32 FMA microbenchmark on the {peak['sm_count']} SMs "
                        f"read from the device, median of 60 launches of ~5 ms ({peak['form']}: packed float2 "
                        f"{peak['packed_tflops']:.2f}, scalar {peak['scalar_tflops']:.2f} TFLOP/s; "
                        f"{peak['fma_per_clock_sm']['packed']} / {peak['fma_per_clock_sm']['scalar']} FMA per SM "
                        f"cycle counted in the kernel, i.e. an SM clock of {peak['implied_sm_mhz']} MHz; "
                        f"nvidia-smi median {pk_mhz} MHz while it ran)"),
        "peak_sm_mhz": pk_mhz, "kernel_sm_mhz": kn_mhz,
        "frac_same_clock": (round(achieved / (peak["tflops"] * kn_mhz / pk_mhz), 4) if pk_mhz and kn_mhz else None),
        "flops_per_launch": round(dom_flops / dom_launches),
        "ms_per_launch": round(dom_ms / dom_launches, 5),
    }
    both_ms = tim["descriptor"][0] + tim["force"][0]
    both = (f_desc + f_force) / (both_ms * 1e-3) / 1e12 if both_ms > 0 else 0.0

    # end to end through the public API with pinned host buffers: every step uploads the state read
    # back by the previous step, runs one MD step and reads the state and the thermodynamics back.  An
    # upload that leaves every atom's float32 position unchanged keeps the forces, so each step does
    # one force evaluation, as a step on resident data does.
    e2e = None
    if not args.no_e2e:
        xo = torch.from_numpy(wl.pos.copy()).pin_memory()
        vo = torch.from_numpy(wl.vel.copy()).pin_memory()
        nep.set_timing(False)
        nep.set_state(xo, vo, wl.box)
        for _ in range(2):
            nep.step(wl.dt_fs, 1); nep.get_state(xo, vo); nep.thermo(); nep.set_state(xo, vo, wl.box)
        dist_barrier(ws)
        torch.cuda.synchronize(dev)
        c_e0 = nep.counters()
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            nep.set_state(xo, vo, wl.box)
            nep.step(wl.dt_fs, 1)
            nep.get_state(xo, vo)
            nep.thermo()
        torch.cuda.synchronize(dev)
        te = dist_max(time.perf_counter() - t0, ws, dev)
        c_e1 = nep.counters()
        dist_barrier(ws)
        e2e = {"value": atoms_total * args.e2e_steps / te, "unit": UNIT, "h2d_bytes_per_step": 48 * wl.n,
               "d2h_bytes_per_step": 48 * wl.n + 8 * 16, "steps": args.e2e_steps,
               "force_evaluations_per_step": (c_e1["evaluations"] - c_e0["evaluations"]) / args.e2e_steps,
               "note": "per step: nep_set_state(x, v read back by the previous step, pinned host) + md_verlet_step(1) "
                       "+ nep_get_state(x, v to pinned host) + thermo; the upload leaves the float32 positions "
                       "unchanged, so the library keeps the forces and the step evaluates them once"}
    ablations = None
    if args.form == "plain" and not args.no_ablations:
        # kernel variants of the paper's design on the same state, against the production kernels
        nep.set_state(wl.pos, wl.vel, wl.box)
        nep.set_timing(True)
        nep.compute(forces=False)
        t_ref = nep.timing()
        nep.set_timing(False)
        ablations = {"fused_ms": round(t_ref["force"][0] + t_ref["descriptor"][0], 4)}
        for v in ("separate_descriptor", "separate_force", "float_scatter", "half_list", "tile1", "tile3",
                  "cpb1", "cpb2", "cpb3"):
            ablations[v + "_ms"] = round(min(nep.run_variant(v)[0] for _ in range(3)), 4)
        p90, cpb = nep.angular_p90()
        ablations["cpb_rule"] = {"p90_angular_pairs": p90, "centres_per_warp": cpb}
        ablations["note"] = ("fused: the production kernel (descriptors, network and forces in one launch, adjoint "
                             "rows in tensor memory, the force pass over the descriptor walk's pair records); "
                             "separate_descriptor + separate_force: descriptors and full-row forces as two launches "
                             "with the adjoint rows through device memory and the force kernel walking the "
                             "neighbour list; float_scatter: the separate force kernel with float atomicAdd "
                             "(order-dependent sums) instead of fixed-point integer atomics; half_list: force "
                             "kernel over each unordered pair once, gathering the neighbour's adjoint row; "
                             "tile1/tile3: descriptor kernel with 1 or 3 angular channels per neighbour pass and "
                             "s_nlm through global memory instead of all 5 channels in tensor memory; cpb1/2/3: "
                             "force kernel in the paper's thread-per-neighbour form, 1, 2 or 3 centre atoms per "
                             "32-lane warp (adaptive centres-per-block; cpb_rule: the 90th percentile of the "
                             "angular pair count and the CPB it selects); single launches, CUDA events")
    F_plain = F_this = None
    others = [] if args.no_forms else [f for f in FORMS if f != args.form]
    if others:
        nep.set_state(wl.pos, wl.vel, wl.box)
        _, F_this, _ = nep.compute()
    nep.close()
    forms = {}
    for f in others:
        forms[f] = time_form(f, model, student, wl, args, stream, dev, ws, atoms_total)
        if f == "plain":
            F_plain = forms[f].pop("_F")
    if args.form == "plain":
        F_plain = F_this
    if F_plain is not None and F_this is not None:
        idx = ni.sample_indices(wl.n, 8192, seed=11)
        for f, rec in forms.items():
            if "_F" in rec:
                d = rec.pop("_F")[idx] - F_plain[idx]
                rec["force_rmse_vs_plain"] = float(np.sqrt(np.mean(d ** 2)))
                rec["force_max_vs_plain"] = float(np.abs(d).max())
            rec["speedup_vs_this"] = round(rec["value"] / value, 4)
        if args.form != "plain":
            d = F_this[idx] - F_plain[idx]
            forms["this_form_vs_plain"] = {"force_rmse": float(np.sqrt(np.mean(d ** 2))), "force_max": float(np.abs(d).max())}
    wl_dt, wl_temp = wl.dt_fs, wl.temperature
    del wl
    configs = None if args.no_configs else run_configs(model, student, args, stream, dev, local, ws)

    if rank != 0:
        return
    n_rep = int(atoms_total // ws)
    walked = dc["list_entries"] / max(1, evals * n_rep)         # walked list entries per atom-evaluation
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_max / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": FORMS[args.form]["dtype"], "data": "synthetic",
        "config": {"workload": args.workload, "atoms_per_gpu": n_rep, "form": FORMS[args.form]["desc"],
                   "dt_fs": wl_dt, "temperature_K": wl_temp,
                   "neighbor_rebuild": f"every {args.rebuild_every} steps + displacement check (skin/2)",
                   "rebuilds_in_timed_region": dg["rebuilds"],
                   "timing": "timed region: CUDA-graph replay of the MD step (CUDA events on the library's "
                             "stream); kernels and roofline: an eager pass of the same length with per-kernel-class "
                             "CUDA events",
                   **({"fallback_fraction": dg["fallback_atoms"] / max(1, dg["evaluations"] * n_rep),
                       "fallback_margin": FALLBACK_MARGIN} if FORMS[args.form]["fallback"] else {}),
                   "l2": "inputs larger than L2: per-step algorithmic HBM traffic ~"
                         f"{n_rep * (BYTES['per_atom'] + BYTES['per_list_entry'] * walked) / 1e9:.2f} GB"
                         " (state, forces, positions, walked neighbour-list entries) vs 129 MB L2",
                   "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU"},
        "roofline": roofline,
        "clocks": clk,
        "clocks_kernel_pass": clk_kernels,
        "gpu_launches": dg["launches"],
        "kernels": kern,
        "descriptor_plus_force_tflops": round(both, 3),
        "pairs_per_atom": {"list": walked, "radial": dc["radial_pairs"] / max(1, evals * n_rep),
                           "angular": dc["angular_pairs"] / max(1, evals * n_rep),
                           "force_kernel_angular": dc["force_angular_pairs"] / max(1, evals * n_rep)},
        "thermo_end": {"pe_per_atom": th["pe"] / n_rep, "temperature": th["temperature"],
                       "energy_change_per_atom": ((th["pe"] + th["ke"]) - (th0["pe"] + th0["ke"])) / n_rep,
                       "over_fs": args.steps * wl_dt},
        "fp32_peak": {k: v for k, v in peak.items()},
        "e2e": e2e,
        "forms": forms or None,
        "configs": configs,
        "ablations": ablations,
        "source_hash": source_hash(),
    }
    if ws == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline()
    print(json.dumps(line), flush=True)


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=("ours", "reference"))
    ap.add_argument("--workload", default="cu_64x64x64")
    ap.add_argument("--rebuild-every", type=int, default=10)
    ap.add_argument("--e2e-steps", type=int, default=10)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--form", default="plain", choices=tuple(FORMS))
    ap.add_argument("--form-steps", type=int, default=50)
    ap.add_argument("--max-neighbors", type=int, default=0, help="neighbour-list capacity per atom (0 = 128)")
    ap.add_argument("--no-forms", action="store_true")
    ap.add_argument("--no-ablations", action="store_true")
    ap.add_argument("--no-configs", action="store_true", help="skip the 16.4M- and 131M-atom workloads")
    args = ap.parse_args(argv)
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    rank, ws, local = dist_setup()
    if args.impl == "reference":
        run_reference(args, rank, ws)
    else:
        run_ours(args, rank, ws, local)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
