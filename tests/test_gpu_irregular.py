"""Irregular inputs for the kernels whose neighbour walk runs warp-uniformly (the teacher's descriptor
and force kernels keep their per-atom arrays in tensor memory, whose accesses are warp-collective):
a strained, displaced cell with vacancies, a small cell with a spherical void and a sparse gas (a single
partial block; some atoms without any angular neighbour), so that the rows of the atoms in one warp
differ in length and in their angular entries, and the atom counts leave the last block partly empty.  Float32 path, float16-row path and the half-list force variant, each
against the oracle."""
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


def _gas(n=37, box=(13.0, 13.5, 14.0), rmin=2.3, seed=404):
    """A sparse gas: n atoms placed at random with no pair closer than rmin -- one partial block,
    rows of 0 to 6 angular and 9 to 15 list entries."""
    rng = np.random.default_rng(seed)
    box = np.asarray(box)
    pts = []
    while len(pts) < n:
        p = rng.uniform(0.0, 1.0, 3) * box
        d = np.asarray(pts).reshape(-1, 3) - p
        d -= box * np.round(d / box)
        if not len(pts) or np.sqrt((d ** 2).sum(1)).min() >= rmin:
            pts.append(p)
    return np.asarray(pts), box


def _cells():
    # 0.07 A displacements: closest pair 2.24 A, |F| up to 10 eV/A (stronger disorder brings atoms
    # within 1.5 A, where float32 rounding of the LJ core alone exceeds the 1e-4 eV/A bound)
    pos, box = ni.student_cell(306, (5, 5, 5), 0.07, (0.01, -0.02, 0.0), 10)
    void = ni.void_strain_workload(6, void_radius=5.0, strain_z=0.02, seed=9)
    return {"disordered": (pos, box), "void": (void.pos, void.box), "gas": _gas()}


CELLS = _cells()


@pytest.fixture(scope="module", params=sorted(CELLS))
def cell(request, model):
    pos, box = CELLS[request.param]
    ang = np.diff(oracle.neighbor_lists(pos, box, 4.0)[0])
    row = np.diff(oracle.neighbor_lists(pos, box, 6.0)[0])
    assert pos.shape[0] % 128 != 0                  # ragged last block
    assert ang.max() - ang.min() >= 3 and row.max() - row.min() >= 5   # rows of unequal length
    if request.param == "gas":
        assert ang.min() == 0                       # atoms without an angular neighbour
    return request.param, pos, box, oracle.energy_forces(model, pos, box)


def test_float32_against_oracle(api, model_params, cell):
    name, pos, box, (Eo, Uo, Fo, Wo) = cell
    with api.NEP(model_params) as nep:
        nep.set_state(pos, np.zeros_like(pos), box)
        E, F, W = nep.compute()
        U = nep.site_energies()
    print(f"{name}: {pos.shape[0]} atoms, max |dF| {np.abs(F - Fo).max():.2e} eV/A")
    assert np.abs(F - Fo).max() <= 1e-4
    assert abs(E - Eo) / abs(Eo) <= 1e-6
    assert np.abs(U - Uo).max() <= 1e-5
    assert np.abs(W - Wo).max() <= 1e-5 * np.abs(Wo).max()


def test_half_list_variant_against_oracle(api, model_params, cell):
    name, pos, box, (Eo, Uo, Fo, Wo) = cell
    with api.NEP(model_params) as nep:
        nep.set_state(pos, np.zeros_like(pos), box)
        _, F = nep.run_variant("half_list")
    assert np.abs(F - Fo).max() <= 1e-4


def test_float16_rows_against_oracle(api, model_params, cell):
    name, pos, box, (Eo, Uo, Fo, Wo) = cell
    with api.NEP(model_params, precision="mix_fp16") as nep:
        nep.set_state(pos, np.zeros_like(pos), box)
        E, F, W = nep.compute()
    dF = F - Fo
    rmse = float(np.sqrt(np.mean(dF ** 2)))
    print(f"{name} mix_fp16: force RMSE {rmse:.2e}, max {np.abs(dF).max():.2e} eV/A")
    assert rmse <= 5e-3 and np.abs(dF).max() <= 3e-3
    assert abs(E - Eo) / abs(Eo) <= 3e-5
