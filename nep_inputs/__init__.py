"""Seeded synthetic inputs for NEP molecular dynamics of fcc Cu.

This module is shared by the FP64 oracle's tests and by the GPU path's tests and benchmark.  It only
draws random numbers and lays out lattices: it contains none of the method's arithmetic (no cutoff,
basis, descriptor, network, force or integrator code).  Every array it returns is plain numpy, so
both sides consume exactly the same input values.

Workloads follow the paper's Cu runs (fcc Cu, 1 fs steps, Maxwell-Boltzmann velocities at 300 K,
Section VI.A) with seeded random NEP weights in place of trained ones.

Units: Angstrom, fs, eV, amu.
"""
from __future__ import annotations

import dataclasses
import numpy as np

A_CU = 3.615            # fcc Cu lattice constant, Angstrom
M_CU = 63.546           # Cu mass, amu
KB_EV = 8.617333262e-5  # Boltzmann constant, eV/K
EV_PER_AMU_A2_FS2 = 103.642696562  # 1 amu*A^2/fs^2 in eV  (kinetic-energy unit conversion)

# NEP hyperparameters of the Cu model (Section VI.A: n_max 4, basis size 8, 3-body l_max 4,
# 4-body l_max 2, 30 neurons; cutoffs 5.0 / 4.0 Angstrom as the workload specifies).
NEP_DIMS = dict(n_max_R=4, n_max_A=4, basis_R=8, basis_A=8, l_max_3b=4, l_max_4b=2, n_neu=30)
# the distilled student: fewer channels, l <= 2, no 4-body term, narrower hidden layer
STUDENT_DIMS = dict(n_max_R=3, n_max_A=3, basis_R=8, basis_A=8, l_max_3b=2, l_max_4b=0, n_neu=16)
N_DES = (NEP_DIMS["n_max_R"] + 1) + (NEP_DIMS["n_max_A"] + 1) * NEP_DIMS["l_max_3b"] + (NEP_DIMS["n_max_A"] + 1)
RC_R = 5.0
RC_A = 4.0
LJ = dict(eps=0.4093, sigma=2.338, rc=5.0)   # Cu Lennard-Jones pair term, shifted-force form
SKIN = 1.0


def fcc_lattice(nx: int, ny: int, nz: int, a: float = A_CU):
    """Perfect fcc lattice of nx*ny*nz conventional cells; atoms ordered (ix, iy, iz, basis)."""
    basis = np.array([[0.0, 0.0, 0.0], [0.5, 0.5, 0.0], [0.5, 0.0, 0.5], [0.0, 0.5, 0.5]])
    ix, iy, iz = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    cells = np.stack([ix.ravel(), iy.ravel(), iz.ravel()], axis=1).astype(np.float64)
    pos = (cells[:, None, :] + basis[None, :, :]).reshape(-1, 3) * a
    box = np.array([nx * a, ny * a, nz * a], dtype=np.float64)
    return pos, box


def gaussian_displace(pos: np.ndarray, box: np.ndarray, sigma: float, rng: np.random.Generator):
    """Add N(0, sigma^2) displacements per component and wrap into [0, box)."""
    out = pos + rng.normal(0.0, sigma, size=pos.shape)
    return np.mod(out, box)


def maxwell_boltzmann(n: int, temperature: float, mass: float, rng: np.random.Generator):
    """Velocities (Angstrom/fs) drawn from N(0, kT/m) per component, centre-of-mass momentum removed,
    then rescaled so that the kinetic temperature with 3N-3 degrees of freedom is exactly T."""
    if n < 2 or temperature <= 0.0:
        return np.zeros((n, 3))
    var = KB_EV * temperature / mass / EV_PER_AMU_A2_FS2          # (Angstrom/fs)^2
    v = rng.normal(0.0, np.sqrt(var), size=(n, 3))
    v -= v.mean(axis=0, keepdims=True)
    ke = 0.5 * mass * np.sum(v * v) * EV_PER_AMU_A2_FS2
    t_now = 2.0 * ke / ((3 * n - 3) * KB_EV)
    return v * np.sqrt(temperature / t_now)


def random_nep_weights(seed: int, dims: dict = NEP_DIMS):
    """Seeded random NEP parameters: Chebyshev expansion coefficients c ~ U(-1, 1); hidden weights and
    biases ~ N(0, 1/fan_in); output weights ~ N(0, 1/fan_in) scaled by 0.05 eV; output bias 0."""
    rng = np.random.default_rng(seed)
    nR, nA = dims["n_max_R"] + 1, dims["n_max_A"] + 1
    kR, kA = dims["basis_R"], dims["basis_A"]
    n_des = nR + nA * dims["l_max_3b"] + (nA if dims["l_max_4b"] > 0 else 0)
    nneu = dims["n_neu"]
    c_R = rng.uniform(-1.0, 1.0, size=(nR, kR))
    c_A = rng.uniform(-1.0, 1.0, size=(nA, kA))
    W0 = rng.normal(0.0, np.sqrt(1.0 / n_des), size=(nneu, n_des))
    b0 = rng.normal(0.0, np.sqrt(1.0 / n_des), size=(nneu,))
    w1 = rng.normal(0.0, np.sqrt(1.0 / nneu), size=(nneu,)) * 0.05
    return dict(c_R=c_R, c_A=c_A, W0=W0, b0=b0, w1=w1, b1=0.0)


@dataclasses.dataclass
class Workload:
    name: str
    pos: np.ndarray     # (N, 3) float64, wrapped into [0, box)
    vel: np.ndarray     # (N, 3) float64, Angstrom/fs
    box: np.ndarray     # (3,) float64
    temperature: float
    dt_fs: float
    steps: int

    @property
    def n(self) -> int:
        return self.pos.shape[0]


def fcc_cu_workload(cells: int, temperature: float = 300.0, sigma: float = 0.05, seed: int = 1,
                    steps: int = 10, dt_fs: float = 1.0, cells_xyz=None, name=None) -> Workload:
    """fcc Cu supercell with seeded Gaussian displacements and Maxwell-Boltzmann velocities."""
    nx, ny, nz = cells_xyz if cells_xyz is not None else (cells, cells, cells)
    pos, box = fcc_lattice(nx, ny, nz)
    rng = np.random.default_rng(seed)
    if sigma > 0:
        pos = gaussian_displace(pos, box, sigma, rng)
    vel = maxwell_boltzmann(pos.shape[0], temperature, M_CU, rng)
    return Workload(name or f"fcc_cu_{nx}x{ny}x{nz}", pos, vel, box, temperature, dt_fs, steps)


def void_strain_workload(cells: int, void_radius: float = 50.0, strain_z: float = 0.02,
                         temperature: float = 300.0, seed: int = 5, steps: int = 100) -> Workload:
    """fcc Cu supercell with a spherical void at the centre and a uniaxial strain along z."""
    pos, box = fcc_lattice(cells, cells, cells)
    centre = 0.5 * box
    keep = np.sum((pos - centre) ** 2, axis=1) >= void_radius ** 2
    pos = pos[keep]
    scale = np.array([1.0, 1.0, 1.0 + strain_z])
    pos = pos * scale
    box = box * scale
    rng = np.random.default_rng(seed)
    vel = maxwell_boltzmann(pos.shape[0], temperature, M_CU, rng)
    return Workload(f"fcc_cu_{cells}^3_void{void_radius:g}_strain{strain_z:g}", np.mod(pos, box), vel,
                    box, temperature, 1.0, steps)


def student_cell(seed: int, cells=(4, 4, 4), temperature_sigma: float = 0.05, strain=(0.0, 0.0, 0.0),
                 vacancies: int = 0):
    """One small periodic fcc Cu cell for student training and tests: nx*ny*nz conventional cells,
    `vacancies` atoms removed at random, a diagonal strain (1 + e_x, 1 + e_y, 1 + e_z) applied to box and
    positions, then Gaussian displacements of `temperature_sigma` Angstrom.  Returns (pos, box)."""
    rng = np.random.default_rng(seed)
    pos, box = fcc_lattice(*cells)
    if vacancies > 0:
        keep = np.ones(pos.shape[0], dtype=bool)
        keep[rng.choice(pos.shape[0], size=vacancies, replace=False)] = False
        pos = pos[keep]
    scale = 1.0 + np.asarray(strain, dtype=np.float64)
    pos = pos * scale
    box = box * scale
    pos = gaussian_displace(pos, box, temperature_sigma, rng)
    return pos, box


# Named workloads (sizes of the paper-shaped Cu runs).
def workload(name: str) -> Workload:
    if name == "cu_4x4x4":        # 256 atoms, sigma 0.05 A, 300 K, 10 steps
        return fcc_cu_workload(4, 300.0, 0.05, seed=1, steps=10, name=name)
    if name == "cu_64x64x64":     # 1,048,576 atoms, 300 K, 200 steps
        return fcc_cu_workload(64, 300.0, 0.05, seed=2, steps=200, name=name)
    if name == "cu_16x16x16":     # 16,384 atoms (CPU baseline sample)
        return fcc_cu_workload(16, 300.0, 0.05, seed=3, steps=10, name=name)
    if name == "cu_160x160x160":  # 16,384,000 atoms, 300 K
        return fcc_cu_workload(160, 300.0, 0.05, seed=4, steps=100, name=name)
    if name == "cu_160x160x160_1200K":
        return fcc_cu_workload(160, 1200.0, 0.1, seed=4, steps=100, name=name)
    if name == "cu_320_void":
        return void_strain_workload(320)
    raise KeyError(name)


def sample_indices(n: int, count: int, seed: int = 7) -> np.ndarray:
    """Seeded sample of distinct atom indices (sorted) for per-atom spot checks."""
    rng = np.random.default_rng(seed)
    count = min(count, n)
    return np.sort(rng.choice(n, size=count, replace=False)).astype(np.int64)
