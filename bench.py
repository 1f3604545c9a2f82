#!/usr/bin/env python3
"""NEP molecular-dynamics throughput on GB300: atom-steps/s of plain FP32 NEP-MD.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--workload NAME]
                    [--form plain|mix_bf16|mix_fp16]

One step = one velocity-Verlet MD step of the whole hot path on the 1,048,576-atom fcc Cu workload
(64x64x64 cells, 300 K, 1 fs): half kick + drift, neighbour-rebuild check (a rebuild runs every 10
steps -- the refresh interval of the paper's MD protocol -- and whenever an atom moved more than
skin/2), cell sort + neighbour list when rebuilding, descriptors + network, forces + virial, half
kick, energy/virial/kinetic sums.  Inputs are resident in HBM when the timed region starts.  The
timed region replays the captured CUDA graph of one MD step, the launch path md_verlet_step uses; the
per-kernel breakdown ("kernels") and the roofline come from an eager pass of the same length with
per-kernel-class CUDA events (about 3 % slower per step than the graph).

--form selects the form whose throughput is the headline value (default: plain FP32).  The other
forms are then timed on the same workload and start state ("forms": atom-steps/s, speedup, and force
RMSE/max against the plain FP32 forces on 8,192 sampled atoms; their error against the FP64 oracle is
a GPU test).  --workload cu_160x160x160 (16,384,000 atoms, 300 K) or cu_160x160x160_1200K runs the
mixed-precision workload.

N > 1 (torchrun): every rank runs an independent replica on its own GPU (no collective on the data
path); value = atom-steps of all ranks / max-over-ranks time ("scaling": "weak").

--impl reference times the FP64 CPU oracle (the method as written, plain C) on the host cores for
the same metric, each step on a bounded sample of the workload.
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
N_SMS = 152
FP32_LANES_PER_SM = 128

# Algorithmic FP32 FLOPs of the method per unit (static count of the arithmetic each unit needs,
# FMA = 2, add/mul = 1, each transcendental = 1), for the compiled shape (5 radial + 5 angular
# channels, 8 basis functions, l = 1..4, 4-body, 30 neurons).  The descriptor kernel visits every
# list entry of every atom.  The force kernel of the float32 teacher ("force_full") visits every
# ordered pair with the own adjoint row only; the half-list form ("force": float16 rows, and the
# half-list ablation) visits each unordered pair once and forms H = G^i + (-1)^l G^j (120 more FMAs
# per angular pair, and fp_i + fp_j per radial pair).
FLOPS = {
    "descriptor": dict(list_entry=11, active_pair=2, radial_pair=56, lj_pair=12, angular_pair=464, atom=4815),
    "force": dict(list_entry=11, active_pair=2 + 27 + 3, radial_pair=149, lj_pair=13, angular_pair=1465, atom=3),
    "force_full": dict(list_entry=11, active_pair=2 + 27 + 3, radial_pair=141, lj_pair=14, angular_pair=1225,
                       atom=3),
}
# The same static count for the student shape (4 radial + 4 angular channels, 8 basis functions,
# l = 1, 2, no 4-body, 16 neurons), used for the student forms.
FLOPS_STUDENT = {
    "descriptor": dict(list_entry=11, active_pair=2, radial_pair=56, lj_pair=12, angular_pair=193, atom=1144),
    "force": dict(list_entry=11, active_pair=2 + 27 + 3, radial_pair=149, lj_pair=13, angular_pair=570, atom=3),
}
# Algorithmic bytes per atom per force evaluation (HBM, float32 path): positions 16 (x2 kernels), list
# entries 4 each (descriptor: full row, force: owned half), adjoint row 512 written + read, fixed-point
# force 24 zeroed + accumulated, site energy 4.
BYTES = dict(per_atom=16 * 2 + 512 * 2 + 24 * 2 + 4, per_list_entry=4 * 1.5)


def force_kind(form: str) -> str:
    """FLOP table of the force kernel a form runs: the full-row form for the float32 teacher."""
    return "force_full" if form == "plain" else "force"


def kernel_flops(kind: str, c: dict, n_atoms_evals: int, table: dict = FLOPS) -> float:
    f = table[kind]
    if kind == "descriptor":
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
    "descriptor:mix_bf16": ("nep_mixed.cu",) + _CORE,
    "force:mix_bf16": ("nep_force.cu",) + _CORE,
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
def run_reference(args, rank: int, ws: int):
    """Reference arm: the FP64 CPU oracle timed on the host cores (rank 0 only)."""
    if rank != 0:
        return
    import oracle
    oracle.build()
    cores = os.cpu_count() or 1
    oracle.set_threads(cores)
    model = oracle.load_model(os.path.join(ROOT, "paper_2604_24816_gb300", "params", "cu_nep4_synth.json"))
    # size the per-step sample so that warmup + steps take about two minutes
    probe = ni.fcc_cu_workload(6, 300.0, 0.05, seed=2)
    t0 = time.perf_counter()
    oracle.md_nve(model, probe.pos, probe.vel, probe.box, ni.M_CU, 1.0, 1)
    t_atom_step = (time.perf_counter() - t0) / (2 * probe.n)
    budget = 120.0 / max(1, args.steps + args.warmup)
    cells = int(max(4, min(16, round((budget / t_atom_step / 4) ** (1 / 3)))))
    wl = ni.fcc_cu_workload(cells, 300.0, 0.05, seed=2)
    x, v = wl.pos.copy(), wl.vel.copy()
    for _ in range(args.warmup):
        x, v, _ = oracle.md_nve(model, x, v, wl.box, ni.M_CU, 1.0, 1)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        x, v, _ = oracle.md_nve(model, x, v, wl.box, ni.M_CU, 1.0, 1)
    dt = time.perf_counter() - t0
    value = wl.n * args.steps / dt
    sample = (f"fcc Cu {cells}x{cells}x{cells} cells ({wl.n} atoms) per step, FP64 oracle velocity-Verlet "
              f"(each step: 2 force evaluations with a fresh neighbour search, as the oracle stands)")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "sample": sample, "parallelism": "host cores (OpenMP)"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.get_threads(), "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


# form name -> library precision, model (teacher or distilled student), per-atom fallback to the
# teacher, arithmetic types, description
_MIX = ("network GEMMs on tcgen05 tensor cores with {} operands and f32 accumulation, float16 adjoint rows, "
        "FP32 descriptors, float64 integration and sums")
FORMS = {
    "plain": dict(precision="fp32", model="teacher", fallback=False, dtype="f32",
                  desc="plain FP32 NEP (float64 integration and sums)"),
    "mix_bf16": dict(precision="mix_bf16", model="teacher", fallback=False, dtype="bf16/f32",
                     desc="mixed precision: " + _MIX.format("bf16")),
    "mix_fp16": dict(precision="mix_fp16", model="teacher", fallback=False, dtype="f16/f32",
                     desc="mixed precision: " + _MIX.format("f16")),
    "student": dict(precision="fp32", model="student", fallback=False, dtype="f32",
                    desc="distilled student NEP (n_max 3/3, l_max 2, no 4-body, 16 neurons), FP32"),
    "student_bf16_fallback": dict(precision="mix_bf16", model="student", fallback=True, dtype="bf16/f32",
                                  desc="distilled student NEP, " + _MIX.format("bf16") + "; per-atom fallback to the "
                                       "FP32 teacher for atoms outside the student's training range (5 % margin)"),
}
FALLBACK_MARGIN = 0.05
STUDENT_PATH = os.path.join(ROOT, "paper_2604_24816_gb300", "params", "cu_student_trained.json")


def row_bytes(form: str) -> int:
    """Bytes of one adjoint row G of the form's model (teacher 128 / student 40 values; float32 in the
    plain forms, float16 in the mixed ones)."""
    f = FORMS[form]
    return (40 if f["model"] == "student" else 128) * (4 if f["precision"] == "fp32" else 2)


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
    clocks.stop()
    ms = start.elapsed_time(end)
    ms_max = dist_max(ms, ws, dev)
    atoms_total = dist_sum(wl.n, ws, dev)
    value = atoms_total * args.steps / (ms_max * 1e-3)

    c1 = nep.counters()
    th = nep.thermo()
    dg = {k: c1[k] - c0[k] for k in c1}          # the timed (graph) region
    nep.set_timing(True)
    nep.step(wl.dt_fs, args.steps)
    torch.cuda.synchronize(dev)
    tim = nep.timing()
    c2 = nep.counters()
    dc = {k: c2[k] - c1[k] for k in c2}          # the eager pass with per-kernel events
    evals = dc["evaluations"]
    table = FLOPS_STUDENT if FORMS[args.form]["model"] == "student" else FLOPS
    f_desc = kernel_flops("descriptor", dc, evals * wl.n, table)
    f_force = kernel_flops(force_kind(args.form), dc, evals * wl.n, table)
    peaks = load_peaks()
    clk = clocks.summary(t_host0, t_host1)
    peak_tflops = N_SMS * FP32_LANES_PER_SM * 2 * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
    kern = {k: {"ms": round(v[0], 4), "launches": v[1]} for k, v in tim.items()}
    fused = tim["descriptor"][1] == 0 and tim["force"][1] > 0      # one kernel does descriptors and forces
    dominant = "force" if fused else max(("descriptor", "force"), key=lambda k: tim[k][0])
    dom_flops = f_desc + f_force if fused else (f_force if dominant == "force" else f_desc)
    dom_ms = tim[dominant][0]
    dom_launches = max(1, tim[dominant][1])
    achieved = dom_flops / (dom_ms * 1e-3) / 1e12
    traffic = profiled_traffic("fused" if fused else (dominant if args.form == "plain" else f"{dominant}:{args.form}"))
    dom_name = ("k_nep_fused" if fused else
                "k_descriptor_mixed" if dominant == "descriptor" and args.form != "plain" else f"k_{dominant}")
    roofline = {
        "bound": "alu",
        "kernel": dom_name, "achieved": round(achieved, 3), "peak": round(peak_tflops, 2),
        "unit": "TFLOP/s", "frac": round(achieved / peak_tflops, 4),
        "traffic": (round(traffic["bytes"] * wl.n / traffic["atoms"]) if traffic else None),
        "peak_source": f"FP32 FFMA: {N_SMS} SMs x {FP32_LANES_PER_SM} lanes x 2 FLOP x "
                       f"{peaks.get('sm_max_mhz', 2070.0):.0f} MHz ({peaks['source']} max SM clock)",
        "flops_per_launch": round(dom_flops / dom_launches),
        "ms_per_launch": round(dom_ms / dom_launches, 5),
        "frac_at_measured_clock": (round(achieved / (N_SMS * FP32_LANES_PER_SM * 2 * clk["sm_mhz"] * 1e-6), 4)
                                   if clk.get("sm_mhz") else None),
    }
    both_ms = tim["descriptor"][0] + tim["force"][0]
    both = (f_desc + f_force) / (both_ms * 1e-3) / 1e12 if both_ms > 0 else 0.0

    # end-to-end through the public API with pinned host buffers: every step uploads (x, v), runs one
    # MD step (which must rebuild and recompute forces for the uploaded state) and downloads (x, v, E)
    e2e = None
    if not args.no_e2e:
        xh = torch.from_numpy(wl.pos).pin_memory()
        vh = torch.from_numpy(wl.vel).pin_memory()
        xo = torch.empty_like(xh).pin_memory()
        vo = torch.empty_like(vh).pin_memory()
        nep.set_timing(False)
        for _ in range(2):
            nep.set_state(xh, vh, wl.box); nep.step(wl.dt_fs, 1); nep.get_state(xo, vo); nep.thermo()
        dist_barrier(ws)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            nep.set_state(xh, vh, wl.box)
            nep.step(wl.dt_fs, 1)
            nep.get_state(xo, vo)
            nep.thermo()
        torch.cuda.synchronize(dev)
        te = dist_max(time.perf_counter() - t0, ws, dev)
        dist_barrier(ws)
        e2e = {"value": atoms_total * args.e2e_steps / te, "unit": UNIT, "h2d_bytes_per_step": 48 * wl.n,
               "d2h_bytes_per_step": 48 * wl.n + 8 * 16, "steps": args.e2e_steps,
               "note": "per step: nep_set_state(x, v from pinned host) + md_verlet_step(1) (rebuild + 2 force "
                       "evaluations for the uploaded state) + nep_get_state(x, v to pinned host) + thermo"}
    ablations = None
    if args.form == "plain" and not args.no_ablations:
        # kernel variants of the paper's design on the same state, against the production kernels
        nep.set_state(wl.pos, wl.vel, wl.box)
        nep.set_timing(True)
        nep.compute(forces=False)
        t_ref = nep.timing()
        nep.set_timing(False)
        ablations = {"fused_ms": round(t_ref["force"][0] + t_ref["descriptor"][0], 4)}
        for v in ("separate_descriptor", "separate_force", "float_scatter", "half_list", "tile1", "tile3"):
            ablations[v + "_ms"] = round(min(nep.run_variant(v)[0] for _ in range(3)), 4)
        ablations["note"] = ("fused: the production kernel (descriptors, network and full-row forces in one launch, "
                             "adjoint rows in tensor memory); separate_descriptor + separate_force: the same work "
                             "as two launches with the adjoint rows through device memory; float_scatter: the "
                             "separate full-row force kernel with float atomicAdd (order-dependent sums) instead "
                             "of fixed-point integer atomics; half_list: force kernel over each unordered pair "
                             "once, gathering the neighbour's adjoint row, instead of every ordered pair with the "
                             "own row; tile1/tile3: descriptor kernel with 1 or 3 angular channels per neighbour "
                             "pass and s_nlm through global memory instead of all 5 channels in tensor memory; "
                             "single launches, CUDA events")
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

    if rank != 0:
        return
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_max / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": FORMS[args.form]["dtype"], "data": "synthetic",
        "config": {"workload": args.workload, "atoms_per_gpu": wl.n, "form": FORMS[args.form]["desc"],
                   "dt_fs": wl.dt_fs, "temperature_K": wl.temperature,
                   "neighbor_rebuild": f"every {args.rebuild_every} steps + displacement check (skin/2)",
                   "rebuilds_in_timed_region": dg["rebuilds"],
                   "timing": "timed region: CUDA-graph replay of the MD step (CUDA events on the library's "
                             "stream); kernels and roofline: an eager pass of the same length with per-kernel-class "
                             "CUDA events",
                   **({"fallback_fraction": dg["fallback_atoms"] / max(1, dg["evaluations"] * wl.n),
                       "fallback_margin": FALLBACK_MARGIN} if FORMS[args.form]["fallback"] else {}),
                   "l2": "inputs larger than L2: per-step algorithmic traffic ~"
                         f"{(wl.n * (row_bytes(args.form) * 2 + BYTES['per_atom'] - 512 * 2 + 48 * 2) + dc['list_entries'] / max(1, evals) * BYTES['per_list_entry']) / 1e9:.2f} GB"
                         " (neighbour list, adjoint rows, state) vs 129 MB L2",
                   "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU", "model": "cu_nep4_synth (seeded)"},
        "roofline": roofline,
        "clocks": clk,
        "gpu_launches": dg["launches"],
        "kernels": kern,
        "descriptor_plus_force_tflops": round(both, 3),
        "pairs_per_atom": {"list": dc["list_entries"] / max(1, evals * wl.n),
                           "radial": dc["radial_pairs"] / max(1, evals * wl.n),
                           "angular": dc["angular_pairs"] / max(1, evals * wl.n),
                           "force_kernel_angular": dc["force_angular_pairs"] / max(1, evals * wl.n)},
        "thermo_end": {"pe_per_atom": th["pe"] / wl.n, "temperature": th["temperature"],
                       "energy_change_per_atom": ((th["pe"] + th["ke"]) - (th0["pe"] + th0["ke"])) / wl.n,
                       "over_fs": args.steps * wl.dt_fs},
        "e2e": e2e,
        "forms": forms or None,
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
