"""GPU parity: the CUDA path through the C ABI against the FP64 oracle, element by element.

Tolerances (float32 path vs float64 oracle):
  neighbour sets        bit-exact (as sets of atom ids), for the radial list and its angular prefix
  forces                max |dF| <= 1e-4 eV/Angstrom (LJ + NEP); NEP-only forces also relative 1e-3 of max |F|
  total energy          |dE| / |E| <= 1e-6
  site energies         max |dU| <= 1e-5 eV: U_i ~ -2.2 eV is a float32 sum of ~42 LJ pair terms (|e| up to
                        0.35 eV) plus the network output; n * eps32 * sum|e| ~ 42 * 6e-8 * 4 eV = 1e-5
  virial                max |dW| <= 1e-5 * max |W|
  descriptors           |dq| <= 2e-5 * max(1, |q|) per component, relative to each column's scale
  10-step trajectory    positions 1e-6 Angstrom, velocities 1e-7 Angstrom/fs
"""
import numpy as np
import pytest

import nep_inputs as ni
import oracle

pytestmark = pytest.mark.gpu

FAR_EDGE = 0.4    # the far band of a list row starts at rc_R + FAR_EDGE * skin


@pytest.fixture(scope="module")
def api():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2604_24816_gb300 import build
    build.build()
    import paper_2604_24816_gb300 as pkg
    pkg.lib()
    return pkg


@pytest.fixture(scope="module")
def c1():
    return ni.workload("cu_4x4x4")


def _sets_from_gpu(counts, lst):
    return [set(lst[i, :counts[i]].tolist()) for i in range(len(counts))]


def _sets_from_oracle(off, lst):
    return [set(lst[off[i]:off[i + 1]].tolist()) for i in range(len(off) - 1)]


def _min_gap_to_cutoffs(pos, box, cuts):
    d = pos[None, :, :] - pos[:, None, :]
    d -= box * np.round(d / box)
    r = np.sqrt((d ** 2).sum(-1))
    return min(np.abs(r - c).min() for c in cuts)


def _bands(pos, box, i, js, edges):
    d = pos[js] - pos[i]
    d -= box * np.round(d / box)
    return np.searchsorted(edges, np.sqrt((d ** 2).sum(1)), side="right")


@pytest.mark.parametrize("cells", [(4, 4, 4), (4, 4, 5), (6, 5, 4)])
def test_neighbor_sets_bit_exact(api, model_params, cells):
    wl = ni.fcc_cu_workload(0, sigma=0.05, seed=21 + sum(cells), cells_xyz=cells)
    rl = model_params["rc_R"] + model_params["skin"]
    ra = model_params["rc_A"] + model_params["skin"]
    fs = model_params["rc_R"] + FAR_EDGE * model_params["skin"]
    assert _min_gap_to_cutoffs(wl.pos, wl.box, (rl, ra, fs)) > 1e-5, "ambiguous pair within 1e-5 A of a cutoff"
    with api.NEP(model_params) as nep:
        nep.set_state(wl.pos, wl.vel, wl.box)
        nep.build_neighbors()
        counts, nang, nown, lst = nep.neighbors(cap=160)
    o_off, o_lst = oracle.neighbor_lists(wl.pos, wl.box, rl, use_cells=False)
    a_off, a_lst = oracle.neighbor_lists(wl.pos, wl.box, ra, use_cells=False)
    full = _sets_from_gpu(counts, lst)
    assert full == _sets_from_oracle(o_off, o_lst)
    assert np.array_equal(nang, np.diff(a_off))
    # every unordered pair has exactly one owner
    owned = [set(lst[i, :nown[i]].tolist()) for i in range(wl.n)]
    for i in range(wl.n):
        for j in full[i]:
            assert (j in owned[i]) != (i in owned[j])
    # row layout: [owned | other], each grouped by band r < rc_A, rc_A + skin, rc_R, rc_R + 0.4 skin,
    # rc_R + skin
    edges = np.array([model_params["rc_A"], ra, model_params["rc_R"], fs, rl])
    for i in range(0, wl.n, 7):
        b_own = _bands(wl.pos, wl.box, i, lst[i, :nown[i]], edges)
        b_oth = _bands(wl.pos, wl.box, i, lst[i, nown[i]:counts[i]], edges)
        assert np.all(np.diff(b_own) >= 0) and np.all(np.diff(b_oth) >= 0)
        assert np.sum(b_own <= 1) + np.sum(b_oth <= 1) == nang[i]


def test_perfect_lattice_owns_half_of_each_shell(api, model_params):
    pos, box = ni.fcc_lattice(5, 5, 5)
    with api.NEP(model_params) as nep:
        nep.set_state(pos, None, box)
        nep.build_neighbors()
        counts, nang, nown, lst = nep.neighbors(cap=160)
    assert set(counts.tolist()) == {78} and set(nang.tolist()) == {42} and set(nown.tolist()) == {39}


def test_descriptors(api, model_params, model, c1):
    with api.NEP(model_params) as nep:
        nep.set_state(c1.pos, c1.vel, c1.box)
        q = nep.descriptors().astype(np.float64)
    qo = oracle.descriptors(model, c1.pos, c1.box)
    scale = np.maximum(1.0, np.abs(qo).max(axis=0))
    assert (np.abs(q - qo) / scale).max() < 2e-5


@pytest.mark.parametrize("cells", [(4, 4, 4), (4, 4, 5), (6, 6, 6)])
def test_energy_forces_virial(api, model_params, model, cells):
    wl = ni.fcc_cu_workload(0, sigma=0.05, seed=5 + sum(cells), cells_xyz=cells)
    with api.NEP(model_params) as nep:
        nep.set_state(wl.pos, wl.vel, wl.box)
        E, F, W = nep.compute()
        U = nep.site_energies()
    Eo, Uo, Fo, Wo = oracle.energy_forces(model, wl.pos, wl.box)
    assert np.abs(F - Fo).max() <= 1e-4
    assert abs(E - Eo) / abs(Eo) <= 1e-6
    assert np.abs(U - Uo).max() <= 1e-5
    assert np.abs(W - Wo).max() <= 1e-5 * np.abs(Wo).max()


def test_nep_only_forces(api, model_params, model, c1):
    """Without the LJ term the forces are the NEP chain rule alone (max |F| ~ 0.2 eV/A)."""
    m0 = model.with_changes(lj_eps=0.0)
    with api.NEP(model_params, lj=False) as nep:
        nep.set_state(c1.pos, c1.vel, c1.box)
        E, F, W = nep.compute()
    Eo, Uo, Fo, Wo = oracle.energy_forces(m0, c1.pos, c1.box)
    assert np.abs(F - Fo).max() <= 1e-3 * np.abs(Fo).max()
    assert np.abs(F - Fo).max() <= 1e-4
    assert abs(E - Eo) <= 1e-6 * c1.n
    assert np.abs(W - Wo).max() <= 1e-4 * np.abs(Wo).max()


def test_md_trajectory_10_steps(api, model_params, model, c1):
    with api.NEP(model_params) as nep:
        nep.set_state(c1.pos, c1.vel, c1.box)
        nep.step(1.0, 10)
        x, v = nep.get_state()
        th = nep.thermo()
    xo, vo, tho = oracle.md_nve(model, c1.pos, c1.vel, c1.box, ni.M_CU, 1.0, 10)
    dx = x - xo
    dx -= c1.box * np.round(dx / c1.box)
    assert np.abs(dx).max() <= 1e-6
    assert np.abs(v - vo).max() <= 1e-7
    assert abs(th["pe"] - tho[-1, 0]) / abs(tho[-1, 0]) <= 1e-6
    assert abs(th["ke"] - tho[-1, 1]) / abs(tho[-1, 1]) <= 1e-6


def test_deterministic_runs(api, model_params, c1):
    out = []
    for _ in range(2):
        with api.NEP(model_params, rebuild_every=3) as nep:
            nep.set_state(c1.pos, c1.vel, c1.box)
            nep.step(1.0, 7)
            E, F, W = nep.compute()
            x, v = nep.get_state()
            out.append((E, F, W, x, v))
    for a, b in zip(out[0], out[1]):
        assert np.array_equal(np.asarray(a), np.asarray(b))


def test_graph_and_eager_paths_identical(api, model_params, c1):
    res = []
    for timing in (False, True):
        with api.NEP(model_params, rebuild_every=4) as nep:
            nep.set_state(c1.pos, c1.vel, c1.box)
            nep.set_timing(timing)
            nep.step(1.0, 9)
            res.append(nep.get_state())
            if timing:
                t = nep.timing()
                assert t["force"][1] >= 9 and t["force"][0] > 0
    assert np.array_equal(res[0][0], res[1][0]) and np.array_equal(res[0][1], res[1][1])


def test_device_and_host_pointers_agree(api, model_params, c1):
    import torch
    with api.NEP(model_params) as nep:
        nep.set_state(torch.from_numpy(c1.pos).cuda(), torch.from_numpy(c1.vel).cuda(), c1.box)
        Fd = torch.zeros((c1.n, 3), dtype=torch.float64, device="cuda")
        Ed, _, Wd = nep.compute(out=Fd)
        nep.set_state(c1.pos, c1.vel, c1.box)
        Eh, Fh, Wh = nep.compute()
    assert Ed == Eh and np.array_equal(Fd.cpu().numpy(), Fh) and np.array_equal(Wd, Wh)


def test_rebuild_policy_does_not_change_physics(api, model_params, c1):
    res = []
    for every in (0, 1):
        with api.NEP(model_params, rebuild_every=every) as nep:
            nep.set_state(c1.pos, c1.vel, c1.box)
            nep.step(1.0, 20)
            res.append(nep.get_state()[0])
            c = nep.counters()
            assert c["steps"] == 20
            if every == 1:
                assert c["rebuilds"] >= 21
    d = res[0] - res[1]
    d -= c1.box * np.round(d / c1.box)
    assert np.abs(d).max() < 1e-6


def test_atoms_crossing_the_boundary_and_rebuilds(api, model_params, model):
    """Hot small cell: atoms leave their cells and cross the periodic boundary between rebuilds; the
    60-step GPU trajectory follows the oracle's trajectory from the same seeded start."""
    wl = ni.fcc_cu_workload(4, temperature=1500.0, sigma=0.1, seed=33)
    with api.NEP(model_params) as nep:
        nep.set_state(wl.pos, wl.vel, wl.box)
        nep.step(1.0, 60)
        x, v = nep.get_state()
        th = nep.thermo()
        assert nep.counters()["rebuilds"] >= 2
    assert np.all((x >= 0) & (x < wl.box))
    xo, vo, tho = oracle.md_nve(model, wl.pos, wl.vel, wl.box, ni.M_CU, 1.0, 60)
    dx = x - xo
    dx -= wl.box * np.round(dx / wl.box)
    assert np.abs(dx).max() <= 1e-5
    assert abs(th["pe"] - tho[-1, 0]) / abs(tho[-1, 0]) <= 1e-6


def test_nve_energy_drift_gpu(api, model_params, c1):
    """Plain FP32 forces with FP64 integration: the slope of a linear fit of the total energy over 10 ps
    (10^4 steps, sampled every 50) is below 1e-5 eV/atom/ps."""
    with api.NEP(model_params) as nep:
        nep.set_state(c1.pos, c1.vel, c1.box)
        et = []
        for _ in range(200):
            nep.step(1.0, 50)
            th = nep.thermo()
            et.append((th["pe"] + th["ke"]) / c1.n)
    t_ps = np.arange(1, 201) * 0.05
    assert abs(np.polyfit(t_ps, np.array(et), 1)[0]) < 1e-5


# ----------------------------------------------------------------------------------------------------
# Edge cases and error statuses (host-detected or reported through the device status word).

def test_empty_system(api, model_params):
    with api.NEP(model_params) as nep:
        nep.set_state(np.zeros((0, 3)), None, [20.0, 20.0, 20.0])
        E, F, W = nep.compute()
        nep.step(1.0, 3)
        assert E == 0.0 and F.shape == (0, 3) and np.all(W == 0)


def test_box_too_small(api, model_params):
    with api.NEP(model_params) as nep:
        with pytest.raises(api.NepError) as e:
            nep.set_state(np.zeros((4, 3)), None, [11.0, 20.0, 20.0])
        assert e.value.name == "NEP_ERR_BOX_TOO_SMALL"


def test_nan_positions_reported(api, model_params, c1):
    x = c1.pos.copy()
    x[17, 1] = np.nan
    with api.NEP(model_params) as nep:
        with pytest.raises(api.NepError) as e:
            nep.set_state(x, None, c1.box)
        assert e.value.name == "NEP_ERR_NAN"


def test_neighbor_overflow_reported(api, model_params, c1):
    with api.NEP(model_params, max_neighbors=40) as nep:
        nep.set_state(c1.pos, c1.vel, c1.box)
        with pytest.raises(api.NepError) as e:
            nep.compute()
        assert e.value.name == "NEP_ERR_NEIGH_OVERFLOW"


def test_compute_before_state(api, model_params):
    with api.NEP(model_params) as nep:
        with pytest.raises(api.NepError) as e:
            nep.compute()
        assert e.value.name == "NEP_ERR_STATE"


def test_unwrapped_input_positions(api, model_params, model, c1):
    shifted = c1.pos + c1.box * np.array([1.0, -2.0, 3.0])
    with api.NEP(model_params) as nep:
        nep.set_state(shifted, c1.vel, c1.box)
        E, F, W = nep.compute()
    Eo, Uo, Fo, Wo = oracle.energy_forces(model, c1.pos, c1.box)
    assert np.abs(F - Fo).max() <= 1e-4 and abs(E - Eo) / abs(Eo) <= 1e-6


def test_checkpoint_resume_is_bit_identical(api, model_params):
    """Checkpoint/resume through nep_get_state/nep_set_state: 20 steps in one run equal 10 steps, a
    checkpoint to host memory, a fresh handle and 10 more steps, bit for bit (the checkpoint falls on a
    scheduled rebuild, and every kernel is deterministic)."""
    wl = ni.fcc_cu_workload(6, 300.0, 0.05, seed=97)
    with api.NEP(model_params, rebuild_every=10) as nep:
        nep.set_state(wl.pos, wl.vel, wl.box)
        nep.step(1.0, 20)
        xa, va = nep.get_state()
        assert nep.counters()["rebuilds"] == 3
    with api.NEP(model_params, rebuild_every=10) as nep:
        nep.set_state(wl.pos, wl.vel, wl.box)
        nep.step(1.0, 10)
        x10, v10 = nep.get_state()
    with api.NEP(model_params, rebuild_every=10) as nep:
        nep.set_state(x10, v10, wl.box)
        nep.step(1.0, 10)
        xb, vb = nep.get_state()
    assert np.array_equal(xa, xb) and np.array_equal(va, vb)


def test_step_grouping_is_bit_identical(api, model_params):
    """md_verlet_step(20) and twenty md_verlet_step(1) give the same bits: each step's closing half kick
    is applied by the next step's opening kick kernel or, after the last step of a call, by the kick
    that ends the call, with the same two FMAs either way; the rebuild chain runs inside the captured
    step only when the control kernel asks for it."""
    wl = ni.fcc_cu_workload(6, 300.0, 0.05, seed=99)
    with api.NEP(model_params, rebuild_every=10) as nep:
        nep.set_state(wl.pos, wl.vel, wl.box)
        nep.step(1.0, 20)
        xa, va = nep.get_state()
        ta = nep.thermo()
        ca = nep.counters()
    with api.NEP(model_params, rebuild_every=10) as nep:
        nep.set_state(wl.pos, wl.vel, wl.box)
        for _ in range(20):
            nep.step(1.0, 1)
        xb, vb = nep.get_state()
        tb = nep.thermo()
        cb = nep.counters()
    assert np.array_equal(xa, xb) and np.array_equal(va, vb)
    assert ta["pe"] == tb["pe"] and ta["ke"] == tb["ke"]
    assert ca["rebuilds"] == cb["rebuilds"] == 3 and ca["evaluations"] == cb["evaluations"] == 21


def test_bounded_wait_runs_out_and_reports(api):
    """The tensor-core kernels wait on mbarriers with a poll limit; a wait on a barrier that nothing
    arrives on ends the kernel with the timeout bit set, and the context stays usable."""
    import ctypes as C
    L = api.lib()
    flag = C.c_int(-1)
    assert L.nep_selftest_bounded_wait(1 << 12, C.byref(flag)) == 0
    assert flag.value == 1
    # the context still works afterwards
    wl = ni.workload("cu_4x4x4")
    with api.NEP(precision="mix_bf16") as nep:
        nep.set_state(wl.pos, wl.vel, wl.box)
        E, F, W = nep.compute()
    assert np.isfinite(E) and np.all(np.isfinite(F))


def test_reupload_keeps_the_list_within_the_skin(api, model_params, model):
    """nep_set_state on the same system keeps the neighbour list while every atom stays within
    skin/2 of where the list was built (positions may come back as another periodic image), and the
    forces are the oracle's for the uploaded positions."""
    wl = ni.fcc_cu_workload(4, 300.0, 0.05, seed=71)
    rng = np.random.default_rng(72)
    with api.NEP(model_params, rebuild_every=0) as nep:
        nep.set_state(wl.pos, wl.vel, wl.box)
        nep.step(1.0, 5)
        x, v = nep.get_state()
        r0 = nep.counters()["rebuilds"]
        x2 = x + 0.03 * rng.standard_normal(x.shape)
        x2[0] += wl.box                                   # another periodic image of atom 0
        x2[1, 2] -= wl.box[2]
        nep.set_state(x2, v, wl.box)
        E, F, W = nep.compute()
        assert nep.counters()["rebuilds"] == r0
        nep.step(1.0, 2)                                  # and MD continues from the uploaded state
    Eo, Uo, Fo, Wo = oracle.energy_forces(model, x2, wl.box)
    assert np.abs(F - Fo).max() <= 1e-4
    assert abs(E - Eo) / abs(Eo) <= 1e-6


def test_reupload_rebuilds_when_atoms_moved_beyond_the_skin(api, model_params):
    """A rigid translation by 0.7 A (> skin/2) forces a rebuild; the forces are translation invariant."""
    wl = ni.fcc_cu_workload(4, 300.0, 0.05, seed=73)
    with api.NEP(model_params, rebuild_every=0) as nep:
        nep.set_state(wl.pos, wl.vel, wl.box)
        E0, F0, _ = nep.compute()
        r0 = nep.counters()["rebuilds"]
        nep.set_state(wl.pos + np.array([0.7, -0.4, 0.3]), wl.vel, wl.box)
        E1, F1, _ = nep.compute()
        assert nep.counters()["rebuilds"] == r0 + 1
    # float32 rounding of the shifted cell-relative coordinates: the float32 path's bound
    assert np.abs(F1 - F0).max() <= 1e-4
    assert abs(E1 - E0) <= 1e-6 * abs(E0)


def test_round_trip_upload_keeps_forces(api, model_params):
    """Uploading the state just read back (velocities possibly changed) leaves every float32 position
    as it was: the handle keeps the last evaluation's forces, energy and virial (no new evaluation),
    the kinetic energy follows the uploaded velocities, and MD continues as without the round trip.
    A changed position makes the next step evaluate the forces again."""
    wl = ni.fcc_cu_workload(5, 300.0, 0.05, seed=81)
    with api.NEP(model_params, rebuild_every=10) as ref:
        ref.set_state(wl.pos, wl.vel, wl.box)
        ref.step(1.0, 4)
        th4 = ref.thermo()
        ref.step(1.0, 3)
        xr, vr = ref.get_state()
    with api.NEP(model_params, rebuild_every=10) as nep:
        nep.set_state(wl.pos, wl.vel, wl.box)
        nep.step(1.0, 4)
        x, v = nep.get_state()
        ev0 = nep.counters()["evaluations"]
        nep.set_state(x, 2.0 * v, wl.box)
        assert nep.counters()["evaluations"] == ev0
        th = nep.thermo()
        assert th["pe"] == th4["pe"]
        assert abs(th["ke"] - 4.0 * th4["ke"]) <= 1e-9 * th4["ke"]
        nep.set_state(x, v, wl.box)
        nep.step(1.0, 3)
        assert nep.counters()["evaluations"] == ev0 + 3
        xb, vb = nep.get_state()
        # the round trip through wrapped host positions may move a coordinate by an ulp of float64
        assert np.abs(xb - xr).max() <= 1e-10 and np.abs(vb - vr).max() <= 1e-12
        x[0, 0] += 1e-3
        nep.set_state(x, v, wl.box)
        nep.step(1.0, 1)
        assert nep.counters()["evaluations"] == ev0 + 5


def test_state_transfer_paths_agree(api, model_params):
    """nep_set_state / nep_get_state read and write page-locked host arrays and device arrays directly
    and other host arrays through a staging copy: after MD steps (cell order != caller order) the three
    paths return the same bits, and the same steps after an upload through each path end in the same
    state."""
    import torch
    wl = ni.fcc_cu_workload(6, 300.0, 0.05, seed=83)
    n = wl.n

    def arrays(kind):
        if kind == "pageable":
            return np.zeros((n, 3)), np.zeros((n, 3))
        if kind == "pinned":
            return (torch.zeros((n, 3), dtype=torch.float64).pin_memory(),
                    torch.zeros((n, 3), dtype=torch.float64).pin_memory())
        return (torch.zeros((n, 3), dtype=torch.float64, device="cuda"),
                torch.zeros((n, 3), dtype=torch.float64, device="cuda"))

    def host(a):
        return a if isinstance(a, np.ndarray) else a.cpu().numpy()

    got, ends = {}, {}
    for kind in ("pageable", "pinned", "device"):
        with api.NEP(model_params, rebuild_every=10) as nep:
            nep.set_state(wl.pos, wl.vel, wl.box)
            nep.step(1.0, 12)                      # one rebuild: the cell order has changed
            x, v = arrays(kind)
            nep.get_state(x, v)
            got[kind] = (host(x).copy(), host(v).copy())
            nep.set_state(x, v, wl.box)            # the same state back through the same path
            nep.step(1.0, 3)
            ends[kind] = nep.get_state()
    for kind in ("pinned", "device"):
        assert np.array_equal(got[kind][0], got["pageable"][0]) and np.array_equal(got[kind][1], got["pageable"][1])
        assert np.array_equal(ends[kind][0], ends["pageable"][0])
        assert np.array_equal(ends[kind][1], ends["pageable"][1])


def test_state_transfer_alignment_and_odd_counts(api, model_params):
    """nep_get_state writes 16-byte aligned arrays a block of rows at a time (16-byte stores of the
    block's span, an odd last double when the block holds an odd number of atoms) and other arrays one
    row per thread: with 255 atoms (one block, 765 doubles) and after a rebuild (cell order != caller
    order), the page-locked and device arrays at a 16-byte boundary and one double past it, and the
    pageable arrays through the staging copy, all hold the same bits; an upload from arrays one double
    past a 16-byte boundary continues the same trajectory as one from pageable arrays."""
    import torch
    wl = ni.fcc_cu_workload(4, 300.0, 0.05, seed=91)
    keep = np.ones(wl.n, dtype=bool)
    keep[17] = False                                   # a vacancy: 255 atoms
    pos, vel = np.ascontiguousarray(wl.pos[keep]), np.ascontiguousarray(wl.vel[keep])
    n = pos.shape[0]
    assert n == 255

    def buffers(kind):
        """(x, v) of shape (n, 3); 'off' kinds start one double past a 16-byte boundary."""
        if kind == "pageable":
            return np.zeros((n, 3)), np.zeros((n, 3))
        dev = "cuda" if kind.startswith("device") else "cpu"
        off = 1 if kind.endswith("off") else 0
        out = []
        for _ in range(2):
            base = torch.zeros(3 * n + 2, dtype=torch.float64, device=dev)
            if dev == "cpu":
                base = base.pin_memory()
            t = base[off:off + 3 * n].view(n, 3)
            assert (t.data_ptr() % 16 == 0) == (off == 0)
            out.append(t)
        return tuple(out)

    def host(a):
        return a if isinstance(a, np.ndarray) else a.cpu().numpy()

    got, ends = {}, {}
    kinds = ("pageable", "pinned", "pinned_off", "device", "device_off")
    for kind in kinds:
        with api.NEP(model_params, rebuild_every=10) as nep:
            nep.set_state(pos, vel, wl.box)
            nep.step(1.0, 12)                          # one rebuild: the cell order has changed
            x, v = buffers(kind)
            nep.get_state(x, v)
            got[kind] = (host(x).copy(), host(v).copy())
            nep.set_state(x, v, wl.box)                # back through the same (possibly offset) buffers
            nep.step(1.0, 3)
            ends[kind] = nep.get_state()
    assert np.isfinite(got["pageable"][0]).all() and np.abs(got["pageable"][1]).max() > 0.0
    for kind in kinds[1:]:
        assert np.array_equal(got[kind][0], got["pageable"][0]), kind
        assert np.array_equal(got[kind][1], got["pageable"][1]), kind
        assert np.array_equal(ends[kind][0], ends["pageable"][0]), kind
        assert np.array_equal(ends[kind][1], ends["pageable"][1]), kind


def _pair_r(pos, box, i, js):
    d = pos[js] - pos[i]
    d -= box * np.round(d / box)
    return np.sqrt((d ** 2).sum(-1))


@pytest.mark.parametrize("precision", ["fp32", "mix_fp16"])
def test_far_bands_left_out_only_while_no_pair_can_enter(api, model_params, model, precision):
    """The row walks leave out the far bands (entries built at r >= rc_R + 0.4 skin) while no atom
    has moved more than (0.4 skin - 0.02)/2 since the build, and walk them again after a larger move: a pair
    built in the far band and brought inside rc_R by two 0.45 A moves (each below skin/2, so the list
    is kept) must contribute.  Both forms run the fused kernel, whose force pass visits the descriptor
    walk's active pairs (so the force counters equal the descriptor walk's).  Forces are the oracle's in
    both cases: the float32 form within 1e-4 eV/A, the mixed-precision form (float16 network operands)
    within its own bounds (3 meV/A, 3e-5 relative energy)."""
    wl = ni.fcc_cu_workload(4, 300.0, 0.05, seed=75)
    rc, skin = model_params["rc_R"], model_params["skin"]
    fs = rc + FAR_EDGE * skin
    rng = np.random.default_rng(76)
    with api.NEP(model_params, rebuild_every=0, precision=precision) as nep:
        nep.set_state(wl.pos, wl.vel, wl.box)
        counts, nang, nown, lst = nep.neighbors(cap=160)
        total = int(counts.sum())
        r_build = [_pair_r(wl.pos, wl.box, i, lst[i, :counts[i]]) for i in range(wl.n)]
        n_far = sum(int((r >= fs).sum()) for r in r_build)
        n_edge = sum(int((np.abs(r - fs) < 1e-4).sum()) for r in r_build)
        assert n_far > 0.1 * total

        # (a) every atom within 0.08 A of its build position: far bands skipped
        u = rng.standard_normal(wl.pos.shape)
        u *= (0.08 * rng.random(wl.n) ** (1 / 3) / np.linalg.norm(u, axis=1))[:, None]
        x1 = wl.pos + u
        c0 = nep.counters()
        nep.set_state(x1, wl.vel, wl.box)
        E1, F1, _ = nep.compute()
        c1 = nep.counters()
        assert c1["rebuilds"] == c0["rebuilds"]
        walked = c1["list_entries"] - c0["list_entries"]
        assert abs(walked - (total - n_far)) <= n_edge
        assert c1["force_list_entries"] - c0["force_list_entries"] == walked

        # (b) one far-band pair pulled 0.9 A closer: the whole rows are walked
        best = None
        for i in range(wl.n):
            r = r_build[i]
            for k in np.nonzero((r > fs + 0.02) & (r < fs + 0.15))[0]:
                j = int(lst[i, k])
                d = wl.pos[j] - wl.pos[i]
                d -= wl.box * np.round(d / wl.box)
                e = d / np.linalg.norm(d)
                x2 = wl.pos.copy()
                x2[i] += 0.45 * e
                x2[j] -= 0.45 * e
                closest = min(np.delete(_pair_r(x2, wl.box, a, np.arange(wl.n)), a).min() for a in (i, j))
                if best is None or closest > best[0]:
                    best = (closest, i, j, x2)
            if best is not None and best[0] > 2.3:
                break
        closest, i, j, x2 = best
        assert _pair_r(x2, wl.box, i, np.array([j]))[0] < rc - 0.3
        nep.set_state(x2, wl.vel, wl.box)
        E2, F2, _ = nep.compute()
        c2 = nep.counters()
        assert c2["rebuilds"] == c0["rebuilds"]
        assert c2["list_entries"] - c1["list_entries"] == total
        assert c2["force_list_entries"] - c1["force_list_entries"] == total
    for x, E, F in ((x1, E1, F1), (x2, E2, F2)):
        Eo, Uo, Fo, Wo = oracle.energy_forces(model, x, wl.box)
        if precision == "fp32":
            assert np.abs(F - Fo).max() <= 1e-4
            assert abs(E - Eo) / abs(Eo) <= 1e-6
        else:
            assert np.abs(F - Fo).max() <= 3e-3            # the mixed form's bounds (test_gpu_mixed)
            assert abs(E - Eo) / abs(Eo) <= 3e-5
