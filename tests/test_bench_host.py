"""Host-side logic of bench.py on CPU: replica bookkeeping over two gloo ranks (max-over-ranks time,
summed atom counts), the FLOP model, the ncu-traffic lookup and the clock-sample parser."""
import os
import socket

import pytest

import bench


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    t = bench.dist_max(1.0 + rank, world)          # per-rank timings 1.0 and 2.0
    n = bench.dist_sum(1000 * (rank + 1), world)   # replicas of 1000 and 2000 atoms
    bench.dist_barrier(world)
    dist.destroy_process_group()
    q.put((rank, t, n))


def test_two_rank_replica_bookkeeping():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res == [(0, 2.0, 3000.0), (1, 2.0, 3000.0)]


def test_single_rank_helpers_are_identity():
    assert bench.dist_max(3.5, 1) == 3.5 and bench.dist_sum(7, 1) == 7


def test_flop_model_counts_units():
    """The FLOP model is the table's per-unit counts times the pair counters of the right kernel
    (descriptor: full rows; force: the rows the force kernel walked), for both model shapes."""
    half = dict(list_entries=78, active_pairs=42, radial_pairs=42, angular_pairs=18, force_list_entries=39,
                force_active_pairs=21, force_radial_pairs=21, force_angular_pairs=9)
    for table in (bench.FLOPS, bench.FLOPS_STUDENT):
        d, f = table["descriptor"], table["force"]
        f_desc = bench.kernel_flops("descriptor", half, 1, table)
        f_force = bench.kernel_flops("force", half, 1, table)
        assert f_desc == (d["list_entry"] * 78 + d["active_pair"] * 42 + (d["radial_pair"] + d["lj_pair"]) * 42 +
                          d["angular_pair"] * 18 + d["atom"])
        assert f_force == (f["list_entry"] * 39 + f["active_pair"] * 21 + (f["radial_pair"] + f["lj_pair"]) * 21 +
                           f["angular_pair"] * 9 + f["atom"])
    teacher = bench.kernel_flops("force", half, 1) + bench.kernel_flops("descriptor", half, 1)
    student = (bench.kernel_flops("force", half, 1, bench.FLOPS_STUDENT) +
               bench.kernel_flops("descriptor", half, 1, bench.FLOPS_STUDENT))
    assert 25e3 < teacher < 45e3 and 8e3 < student < 0.6 * teacher
    # the full-row form: every ordered pair, without the H_nlm and fp_i + fp_j terms of the half list
    full = dict(half, force_list_entries=78, force_active_pairs=42, force_radial_pairs=42, force_angular_pairs=18)
    h, g = bench.FLOPS["force"], bench.FLOPS["force_full"]
    assert g["angular_pair"] == h["angular_pair"] - 2 * 120 and g["radial_pair"] == h["radial_pair"] - 8
    assert g["lj_pair"] == h["lj_pair"] + 1
    ratio = bench.kernel_flops("force_full", full, 1) / bench.kernel_flops("force", half, 1)
    assert 1.4 < ratio < 2.0
    # the fused kernel's force pass reads each active pair's record instead of walking the list: no
    # per-entry term, and r^2 (5 FLOP) recomputed from the recorded displacement per active pair
    r = bench.FLOPS["force_rec"]
    assert r["list_entry"] == 0 and r["active_pair"] == g["active_pair"] + 5
    assert all(r[k] == g[k] for k in ("lj_pair", "atom"))
    # ... contracts the radial adjoint with the Chebyshev factors instead of forming the 8 basis
    # derivatives (117 -> 80 per radial pair, two at a time; 84 one at a time, for the angular pairs'
    # radial part) and keeps its row over the harmonic polynomials without their constants: 81 -> 52
    # FLOPs for the 24 values, 129 -> 86 for their gradients
    assert r["radial_pair"] == g["radial_pair"] - 37
    assert r["angular_pair"] == g["angular_pair"] - (81 - 52) - (129 - 86) + 4
    assert all(bench.force_kind(f) == ("force_rec" if bench.FORMS[f]["model"] == "teacher" or
                                       bench.FORMS[f]["precision"] == "fp32" else "force") for f in bench.FORMS)
    # the student's fused kernel: its record pass has the teacher's per-pair terms except the angular
    # one, whose channel sums scale with the 4 x 8 instead of 5 x 24 (l, m) components
    rs, hs = bench.FLOPS_STUDENT["force_rec"], bench.FLOPS_STUDENT["force"]
    assert all(rs[k] == r[k] for k in ("list_entry", "active_pair", "lj_pair", "atom"))
    assert rs["radial_pair"] == r["radial_pair"] + 4      # one record at a time
    assert 0.3 * r["angular_pair"] < rs["angular_pair"] < hs["angular_pair"]
    # ... and its descriptor part keeps the sums over the polynomials without their constants (8 of them:
    # 14 -> 10 FLOPs per angular pair; 16 + 8 more scalings per atom), used by the float32 student only
    ds, dr = bench.FLOPS_STUDENT["descriptor"], bench.FLOPS_STUDENT["descriptor_rec"]
    assert dr["angular_pair"] == ds["angular_pair"] - 4 and dr["atom"] == ds["atom"] + 24
    assert all(dr[k] == ds[k] for k in ("list_entry", "active_pair", "radial_pair", "lj_pair"))
    assert rs["angular_pair"] == 452 - 4 - 6      # polynomials 14 -> 10, gradients 9 -> 3
    for f, m in bench.FORMS.items():
        want = (("descriptor_rec" if m["precision"] == "fp32" else "descriptor") if m["model"] == "student" else
                ("descriptor_mixed" if f in ("mix_bf16", "mix_fp16") else "descriptor"))
        assert bench.descriptor_kind(f) == want
    # the mixed forms' descriptor part differs only in the network (on the tensor cores)
    dm, dd = bench.FLOPS["descriptor_mixed"], bench.FLOPS["descriptor"]
    assert all(dm[k] == dd[k] for k in dd if k != "atom") and dm["atom"] < dd["atom"]
    # per active pair the force kernels spend 2 (rsqrt, r) + 6 (d) + 3 (F_i) + 12 (6 virial components)
    assert g["active_pair"] == 2 + 6 + 3 + 12 and h["active_pair"] == g["active_pair"]


def test_traffic_lookup_requires_matching_source(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    (tmp_path / "profiles").mkdir()
    (tmp_path / "paper_2604_24816_gb300" / "csrc").mkdir(parents=True)
    for f in bench.SOURCE_FILES:
        (tmp_path / "paper_2604_24816_gb300" / "csrc" / f).write_text("x")
    h = bench.source_hash("force")
    hn = bench.source_hash("neighbors")
    (tmp_path / "profiles" / "traffic_per_launch.txt").write_text(
        f"# header\nforce {h} 1000 10\nforce deadbeef 5 1\nneighbors {hn} 300 10\n")
    assert bench.profiled_traffic("force") == dict(bytes=1000.0, atoms=10)
    # a change to another kernel's source leaves the force figure valid, a change to its own does not
    (tmp_path / "paper_2604_24816_gb300" / "csrc" / "nep_neighbor.cu").write_text("changed")
    assert bench.profiled_traffic("force") == dict(bytes=1000.0, atoms=10)
    assert bench.profiled_traffic("neighbors") is None
    (tmp_path / "paper_2604_24816_gb300" / "csrc" / "nep_force.cu").write_text("changed")
    assert bench.profiled_traffic("force") is None


def test_clock_summary_parses_throttle_reasons():
    cs = bench.ClockSampler.__new__(bench.ClockSampler)
    cs.samples = [(1.0, "0, 2070, 2070, 900.0, 0x0, Not Active, Not Active, Not Active, Not Active"),
                  (1.1, "0, 1965, 2070, 1380.0, 0x4, Not Active, Not Active, Not Active, Active"),
                  (1.2, "0, 2070, 2070, 950.0, 0x0, Not Active, Not Active, Not Active, Not Active")]
    s = cs.summary(0.9, 1.3)
    assert s["sm_mhz"] == 2070.0 and s["sm_max_mhz"] == 2070.0 and s["reasons"] == ["sw_power_cap"]
    assert s["samples"] == 3
