"""Per-atom fallback from the student to the teacher (nep_set_fallback) on the GPU against the oracle.

The oracle's energy_forces_select evaluates E = sum_i U_i^(model of i) and F = -grad E at a fixed
assignment.  Flags are compared with the oracle's own range test on its float64 descriptors (atoms
within 1e-4 of the range width from a bound may differ between float32 and float64 and are skipped);
energies and forces are compared at the GPU's assignment with the plain path's bounds.
"""
import numpy as np
import pytest

import nep_inputs as ni
import oracle

pytestmark = pytest.mark.gpu


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
def cell():
    pos, box = ni.student_cell(77, (5, 5, 5), 0.07, (0.02, 0.0, -0.01), 3)
    vel = ni.maxwell_boltzmann(pos.shape[0], 600.0, ni.M_CU, np.random.default_rng(78))
    return pos, vel, box


def _scaled(student_params, pos, box):
    q = oracle.descriptors(oracle.Model(student_params), pos, box)
    return q * np.asarray(student_params["q_scale"], np.float32).astype(np.float64)


def _narrow_range(qt, lo_pct=15, hi_pct=85):
    return np.percentile(qt, lo_pct, axis=0), np.percentile(qt, hi_pct, axis=0)


def test_fallback_flags_energy_forces(api, cell, trained_student_params, model_params):
    pos, vel, box = cell
    sp = trained_student_params
    qt = _scaled(sp, pos, box)
    lo, hi = _narrow_range(qt)
    lo32, hi32 = lo.astype(np.float32), hi.astype(np.float32)
    with api.NEP(sp) as nep:
        nep.set_fallback(model_params, lo32, hi32, margin=0.0, max_fraction=1.0)
        nep.set_state(pos, vel, box)
        E, F, W = nep.compute()
        U = nep.site_energies()
        flags, cnt = nep.fallback()
        c = nep.counters()
    assert cnt == int(flags.sum()) and c["fallback_atoms"] == cnt
    w = hi - lo
    ref = np.any((qt < lo32) | (qt > hi32), axis=1)
    near = np.any(np.minimum(np.abs(qt - lo32), np.abs(qt - hi32)) < 1e-4 * w, axis=1)
    assert 0.2 * pos.shape[0] < cnt < 0.95 * pos.shape[0]
    assert np.array_equal(flags[~near].astype(bool), ref[~near])
    Eo, Uo, Fo, Wo = oracle.energy_forces_select(oracle.Model(sp), oracle.Model(model_params), flags, pos, box)
    assert np.abs(F - Fo).max() <= 1e-4
    assert abs(E - Eo) / abs(Eo) <= 1e-6
    assert np.abs(U - Uo).max() <= 1e-5
    assert np.abs(W - Wo).max() <= 1e-5 * np.abs(Wo).max()


def test_fallback_limits(api, cell, trained_student_params, model_params):
    """No atom out of range -> the student alone; every atom out of range -> the teacher alone."""
    pos, vel, box = cell
    sp = trained_student_params
    big = np.full(12, 1e30, np.float32)
    with api.NEP(sp) as nep:
        nep.set_fallback(model_params, -big, big, margin=0.0)
        nep.set_state(pos, vel, box)
        E0, F0, W0 = nep.compute()
        assert nep.fallback()[1] == 0
    Es, Us, Fs, Ws = oracle.energy_forces(oracle.Model(sp), pos, box)
    assert np.abs(F0 - Fs).max() <= 1e-4 and abs(E0 - Es) / abs(Es) <= 1e-6
    with api.NEP(sp) as nep:
        nep.set_fallback(model_params, big, -big, margin=0.0, max_fraction=1.0)
        nep.set_state(pos, vel, box)
        E1, F1, W1 = nep.compute()
        assert nep.fallback()[1] == pos.shape[0]
    Et, Ut, Ft, Wt = oracle.energy_forces(oracle.Model(model_params), pos, box)
    assert np.abs(F1 - Ft).max() <= 1e-4 and abs(E1 - Et) / abs(Et) <= 1e-6


def test_fallback_overflow_is_reported(api, cell, trained_student_params, model_params):
    pos, vel, box = cell
    big = np.full(12, 1e30, np.float32)
    with api.NEP(trained_student_params) as nep:
        nep.set_fallback(model_params, big, -big, margin=0.0, max_fraction=0.01)
        nep.set_state(pos, vel, box)
        with pytest.raises(api.NepError) as ei:
            nep.compute()
        assert "FALLBACK_OVERFLOW" in str(ei.value)


def test_fallback_mixed_precision_student(api, cell, trained_student_params, model_params):
    pos, vel, box = cell
    sp = trained_student_params
    lo, hi = _narrow_range(_scaled(sp, pos, box))
    with api.NEP(sp, precision="mix_bf16") as nep:
        nep.set_fallback(model_params, lo.astype(np.float32), hi.astype(np.float32), margin=0.0, max_fraction=1.0)
        nep.set_state(pos, vel, box)
        E, F, W = nep.compute()
        flags, cnt = nep.fallback()
    Eo, Uo, Fo, Wo = oracle.energy_forces_select(oracle.Model(sp), oracle.Model(model_params), flags, pos, box)
    assert float(np.sqrt(np.mean((F - Fo) ** 2))) <= 5e-3
    assert abs(E - Eo) / abs(Eo) <= 2e-4


def test_fallback_md_deterministic(api, cell, trained_student_params, model_params):
    pos, vel, box = cell
    sp = trained_student_params
    lo, hi = _narrow_range(_scaled(sp, pos, box), 5, 95)
    out = []
    for _ in range(2):
        with api.NEP(sp, rebuild_every=5) as nep:
            nep.set_fallback(model_params, lo.astype(np.float32), hi.astype(np.float32), margin=0.0,
                             max_fraction=1.0)
            nep.set_state(pos, vel, box)
            nep.step(1.0, 30)
            x, v = nep.get_state()
            c = nep.counters()
            out.append((x, v, c["fallback_atoms"]))
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])
    assert out[0][2] == out[1][2] > 0


def test_void_surface_atoms_fall_back(api, trained_student_params, model_params):
    """A strained cell with a spherical void: with the student's own training range (5 % margin) the
    flagged atoms sit at the void surface."""
    sp = trained_student_params
    wl = ni.void_strain_workload(16, void_radius=12.0, strain_z=0.02, temperature=300.0, seed=5)
    with api.NEP(sp, precision="mix_bf16") as nep:
        nep.set_fallback(model_params, sp["q_lo"], sp["q_hi"], margin=0.05)
        nep.set_state(wl.pos, wl.vel, wl.box)
        nep.compute()
        flags, cnt = nep.fallback()
    centre = 0.5 * wl.box
    d = wl.pos - centre
    d -= wl.box * np.round(d / wl.box)
    r = np.sqrt((d ** 2).sum(axis=1))
    print(f"void cell: {wl.n} atoms, {cnt} flagged ({cnt / wl.n:.2%}), radius of flagged atoms "
          f"{r[flags == 1].min() if cnt else 0:.1f}-{r[flags == 1].max() if cnt else 0:.1f} A")
    assert cnt > 0
    assert np.mean(r[flags == 1] < 12.0 + 6.0) >= 0.9
