"""Student-shaped kernels (radial n_max 3, angular n_max 3, l_max 2, no 4-body, 16 neurons) on the GPU
against the FP64 oracle, with a seeded untrained student: the same kernels, templated on the model
shape, that run the trained student in MD.  Bounds as for the teacher's plain path (forces 1e-4
eV/Angstrom max, energy 1e-6 relative, site energies 1e-5 eV); the mixed forms against the workload's
5 meV/Angstrom RMSE bound.
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


@pytest.mark.parametrize("cells", [(4, 4, 4), (5, 6, 4)])
def test_student_energy_forces_descriptors(api, student_params, student_model, cells):
    wl = ni.fcc_cu_workload(0, sigma=0.08, seed=31 + sum(cells), cells_xyz=cells)
    with api.NEP(student_params) as nep:
        nep.set_state(wl.pos, wl.vel, wl.box)
        E, F, W = nep.compute()
        U = nep.site_energies()
        q = nep.descriptors().astype(np.float64)
    assert q.shape == (wl.n, 12)
    Eo, Uo, Fo, Wo = oracle.energy_forces(student_model, wl.pos, wl.box)
    qo = oracle.descriptors(student_model, wl.pos, wl.box)
    assert np.abs(F - Fo).max() <= 1e-4
    assert abs(E - Eo) / abs(Eo) <= 1e-6
    assert np.abs(U - Uo).max() <= 1e-5
    assert np.abs(W - Wo).max() <= 1e-5 * np.abs(Wo).max()
    assert (np.abs(q - qo) / np.maximum(1.0, np.abs(qo).max(axis=0))).max() < 2e-5


def test_student_nep_only_forces(api, student_params, student_model):
    wl = ni.fcc_cu_workload(4, 300.0, 0.08, seed=41)
    with api.NEP(student_params, lj=False) as nep:
        nep.set_state(wl.pos, wl.vel, wl.box)
        E, F, W = nep.compute()
    Eo, Uo, Fo, Wo = oracle.energy_forces(student_model.with_changes(lj_eps=0.0), wl.pos, wl.box)
    assert np.abs(F - Fo).max() <= 1e-3 * np.abs(Fo).max() + 1e-6
    assert abs(E - Eo) <= 1e-6 * wl.n


def test_student_trajectory(api, student_params, student_model):
    c1 = ni.workload("cu_4x4x4")
    with api.NEP(student_params, rebuild_every=5) as nep:
        nep.set_state(c1.pos, c1.vel, c1.box)
        nep.step(1.0, 10)
        x, v = nep.get_state()
        th = nep.thermo()
    xo, vo, tho = oracle.md_nve(student_model, c1.pos, c1.vel, c1.box, ni.M_CU, 1.0, 10)
    dx = x - xo
    dx -= c1.box * np.round(dx / c1.box)
    assert np.abs(dx).max() <= 1e-6
    assert np.abs(v - vo).max() <= 1e-7
    assert abs(th["pe"] - tho[-1, 0]) / abs(tho[-1, 0]) <= 1e-6


@pytest.mark.parametrize("mode", ["mix_bf16", "mix_fp16"])
def test_student_mixed(api, student_params, student_model, mode):
    wl = ni.fcc_cu_workload(5, 300.0, 0.08, seed=43)
    with api.NEP(student_params, precision=mode) as nep:
        nep.set_state(wl.pos, wl.vel, wl.box)
        E, F, W = nep.compute()
    Eo, Uo, Fo, Wo = oracle.energy_forces(student_model, wl.pos, wl.box)
    rmse = float(np.sqrt(np.mean((F - Fo) ** 2)))
    print(f"student {mode}: force RMSE {rmse:.2e}, max {np.abs(F - Fo).max():.2e} eV/A")
    assert rmse <= 5e-3
    assert abs(E - Eo) / abs(Eo) <= 2e-4


def test_trained_student_against_oracle(api, trained_student_params):
    """The distilled student model file through the MD kernels, against the oracle."""
    m = oracle.Model(trained_student_params)
    wl = ni.fcc_cu_workload(5, 600.0, 0.05, seed=47)
    with api.NEP(trained_student_params) as nep:
        nep.set_state(wl.pos, wl.vel, wl.box)
        E, F, W = nep.compute()
    Eo, Uo, Fo, Wo = oracle.energy_forces(m, wl.pos, wl.box)
    assert np.abs(F - Fo).max() <= 1e-4
    assert abs(E - Eo) / abs(Eo) <= 1e-6


def test_trained_student_vs_teacher_on_fresh_md(api, model_params, trained_student_params):
    """Teacher-MD snapshots from trajectories not used in training (another seed): student vs teacher
    NEP-only forces, both on the GPU, against the workload's 30 meV/Angstrom bound."""
    from paper_2604_24816_gb300 import distill
    snaps = distill.generate(model_params, 4, 5, 25, 200, seed=9191, log=None)
    d, ref = [], []
    with api.NEP(trained_student_params, lj=False) as st:
        for x, box, E, F, sp in snaps:
            st.set_state(x, None, box)
            Es, Fs, Ws = st.compute()
            d.append(Fs - F)
            ref.append(F)
    d, ref = np.concatenate(d), np.concatenate(ref)
    rmse = float(np.sqrt(np.mean(d ** 2)))
    print(f"trained student vs teacher on fresh MD: force RMSE {rmse * 1e3:.1f} meV/A "
          f"(teacher NEP-only force rms {np.sqrt(np.mean(ref ** 2)) * 1e3:.1f})")
    assert rmse <= 0.030
