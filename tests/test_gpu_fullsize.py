"""Full-size checks at the 1,048,576-atom fcc Cu workload (64x64x64 cells), in the launch configuration
the benchmark times (same kernels, same N, CUDA-graph MD steps).

The oracle computes forces and site energies atom by atom on a seeded sample of 4,096 atoms of the
initial configuration (element-by-element parity there), and the neighbour sets of sampled atoms bit for
bit (its cell search over the whole system); properties that hold at any size (sum of forces, energy
conservation, determinism) are checked on the trajectory.
"""
import numpy as np
import pytest

import nep_inputs as ni
import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def big():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2604_24816_gb300 import build
    build.build()
    return ni.workload("cu_64x64x64")


def test_sampled_forces_full_size(big, model_params, model):
    import paper_2604_24816_gb300 as pkg
    with pkg.NEP(model_params, rebuild_every=10) as nep:
        nep.set_state(big.pos, big.vel, big.box)
        E, F, W = nep.compute()
        U = nep.site_energies()
    idx = ni.sample_indices(big.n, 4096, seed=7)
    Fo, Uo = oracle.forces_sampled(model, big.pos, big.box, idx)
    assert np.abs(F[idx] - Fo).max() <= 1e-4
    assert np.abs(U[idx] - Uo).max() <= 1e-5
    # extensive energy: the mean site energy matches the sample mean to sampling accuracy
    assert abs(E / big.n - Uo.mean()) < 5 * Uo.std() / np.sqrt(idx.size) + 1e-6
    assert np.abs(F.sum(axis=0)).max() < 1e-6 * big.n


def test_full_size_md_conserves_energy_and_is_deterministic(big, model_params):
    import paper_2604_24816_gb300 as pkg
    runs = []
    for _ in range(2):
        with pkg.NEP(model_params, rebuild_every=10) as nep:
            nep.set_state(big.pos, big.vel, big.box)
            nep.compute()
            th0 = nep.thermo()
            nep.step(1.0, 50)
            th1 = nep.thermo()
            x, v = nep.get_state()
            c = nep.counters()
            runs.append((th0, th1, x, v, c))
    th0, th1, x, v, c = runs[0]
    assert c["rebuilds"] >= 5 and c["steps"] == 50
    e0 = (th0["pe"] + th0["ke"]) / big.n
    e1 = (th1["pe"] + th1["ke"]) / big.n
    # Velocity Verlet from the displaced start: the oracle's own 256-atom cells of the same distribution
    # (seeds 1-4) move by 5.5e-5 to 8.3e-5 eV/atom over these 50 steps; allow 2.5x the largest.
    assert abs(e1 - e0) < 2e-4
    assert np.array_equal(runs[0][2], runs[1][2]) and np.array_equal(runs[0][3], runs[1][3])
    assert np.all(np.isfinite(x)) and np.all((x >= 0) & (x < big.box))


@pytest.mark.parametrize("rebuild_every, steps", [(10, 25), (0, 40)])
def test_sampled_forces_after_md_full_size(big, model_params, model, rebuild_every, steps):
    """Forces of the MD state after `steps` graph steps, evaluated on the list the MD path kept (5 steps
    old with rebuilds every 10 steps; with displacement-triggered rebuilds only, old enough that the
    largest displacement passes the far-band threshold and the far bands are walked again), against the
    oracle on 4,096 sampled atoms of the same positions."""
    import paper_2604_24816_gb300 as pkg
    with pkg.NEP(model_params, rebuild_every=rebuild_every) as nep:
        nep.set_state(big.pos, big.vel, big.box)
        nep.step(1.0, steps)
        x, _ = nep.get_state()
        E, F, W = nep.compute()
        c = nep.counters()
    idx = ni.sample_indices(big.n, 4096, seed=11)
    Fo, Uo = oracle.forces_sampled(model, x, big.box, idx)
    print(f"rebuild_every={rebuild_every}: {c['rebuilds']} rebuilds, "
          f"{c['list_entries'] / (c['evaluations'] * big.n):.1f} list entries walked per atom-evaluation, "
          f"max |dF| {np.abs(F[idx] - Fo).max():.2e} eV/A")
    assert np.abs(F[idx] - Fo).max() <= 1e-4


def _check_sampled_neighbor_sets(nep, x, box, params, idx):
    """The GPU rows of the sampled atoms against the oracle's cell search over the whole system, as sets
    of atom ids (radial list r < rc_R + skin and its angular count r < rc_A + skin), and every unordered
    pair of a sampled row owned by exactly one of its atoms.  A pair within 1e-5 A of a cutoff may fall
    either way in float32 and is excluded (counted)."""
    rl = params["rc_R"] + params["skin"]
    ra = params["rc_A"] + params["skin"]
    counts, nang, nown, lst = nep.neighbors(cap=160)
    off, ol = oracle.neighbor_lists(x, box, rl + 1e-4)
    ambiguous = 0
    for i in idx:
        js = ol[off[i]:off[i + 1]]
        d = x[js] - x[i]
        d -= box * np.round(d / box)
        r = np.sqrt((d ** 2).sum(1))
        amb = (np.abs(r - rl) < 1e-5) | (np.abs(r - ra) < 1e-5)
        ambiguous += int(amb.sum())
        gpu = set(lst[i, :counts[i]].tolist())
        ref = set(js[r < rl].tolist())
        skip = set(js[amb].tolist())
        assert gpu - skip == ref - skip, f"atom {i}"
        if not amb.any():
            assert nang[i] == int((r < ra).sum()), f"atom {i}"
        own_i = set(lst[i, :nown[i]].tolist())
        for j in gpu:
            assert (j in own_i) != (i in set(lst[j, :nown[j]].tolist())), f"pair {i}, {j}"
    return ambiguous


def test_neighbor_sets_full_size(big, model_params):
    """Bit-exact neighbour sets on 4,096 sampled atoms of the 1,048,576-atom workload (38^3 cells, the
    capped-grid neighbour scan the benchmark runs), after 25 MD steps (two rebuilds)."""
    import paper_2604_24816_gb300 as pkg
    with pkg.NEP(model_params, rebuild_every=10) as nep:
        nep.set_state(big.pos, big.vel, big.box)
        nep.step(1.0, 20)
        x, _ = nep.get_state()
        nep.set_state(x, None, big.box)
        nep.build_neighbors()
        amb = _check_sampled_neighbor_sets(nep, x, big.box, model_params, ni.sample_indices(big.n, 4096, seed=5))
    print(f"{amb} pairs within 1e-5 A of a cutoff excluded")
    assert amb <= 2


def test_neighbor_sets_void_under_strain(model_params):
    """Bit-exact neighbour sets of a 40^3-cell fcc Cu block with a 30 A void and 2 % strain along z:
    2,048 atoms sampled at random and 2,048 from the void surface (fewer neighbours, irregular rows)."""
    import paper_2604_24816_gb300 as pkg
    wl = ni.void_strain_workload(40, void_radius=30.0, strain_z=0.02, seed=8)
    centre = 0.5 * wl.box
    rc = np.sqrt(((wl.pos - centre) ** 2).sum(1))
    surface = np.nonzero(rc < 33.0)[0]
    rng = np.random.default_rng(9)
    idx = np.unique(np.concatenate([rng.choice(wl.n, 2048, replace=False), rng.choice(surface, 2048, replace=False)]))
    with pkg.NEP(model_params) as nep:
        nep.set_state(wl.pos, wl.vel, wl.box)
        nep.build_neighbors()
        amb = _check_sampled_neighbor_sets(nep, wl.pos, wl.box, model_params, idx)
    print(f"{amb} pairs within 1e-5 A of a cutoff excluded")
    assert amb <= 2
