"""Pins for the FP64 oracle against what the physics and the mathematics fix (no GPU).

Each test targets a plausible mistake in the oracle: a wrong derivative (finite differences), a wrong
sign or index in the force scatter (sum of forces, invariances, finite-strain virial), wrong
Chebyshev/cutoff/Legendre arithmetic (closed forms from numpy/scipy library routines), wrong
harmonic constants (addition theorem against an independent Y_lm route), a wrong 4-body contraction
(Wigner-3j route with scipy harmonics and sympy 3j symbols), a transposed network weight or a flipped
bias sign (sparse network with a hand-evaluated output), and broken neighbour search (brute force).
"""
import math

import numpy as np
import pytest
from numpy.polynomial import chebyshev as npcheb
from scipy.special import eval_legendre

import nep_inputs as ni
import oracle


def _g_ref(c, r, rc):
    """Radial functions from numpy's Chebyshev evaluation and the cosine cutoff (independent route)."""
    x = 2.0 * (r / rc - 1.0) ** 2 - 1.0
    fc = 0.5 * (1.0 + math.cos(math.pi * r / rc)) if r < rc else 0.0
    K = c.shape[1]
    f = np.array([0.5 * (npcheb.chebval(x, np.eye(K)[k]) + 1.0) * fc for k in range(K)])
    return c @ f


@pytest.fixture(scope="module")
def c1():
    return ni.workload("cu_4x4x4")


def _fd_force(model, x, box, i, a, h=2e-5):
    xp = x.copy(); xp[i, a] += h
    xm = x.copy(); xm[i, a] -= h
    Ep = oracle.energy_forces(model, xp, box)[0]
    Em = oracle.energy_forces(model, xm, box)[0]
    return -(Ep - Em) / (2 * h)


@pytest.mark.parametrize("lj_on", [True, False])
def test_forces_are_minus_energy_gradient(model, c1, lj_on):
    m = model if lj_on else model.with_changes(lj_eps=0.0)
    E, U, F, W = oracle.energy_forces(m, c1.pos, c1.box)
    rng = np.random.default_rng(11)
    picks = [(int(rng.integers(c1.n)), int(rng.integers(3))) for _ in range(10)]
    for i, a in picks:
        fd = _fd_force(m, c1.pos, c1.box, i, a)
        assert abs(fd - F[i, a]) <= 1e-7 * max(1.0, abs(F[i, a])), (i, a, fd, F[i, a])


def test_sum_of_forces_is_zero(model, c1):
    F = oracle.energy_forces(model, c1.pos, c1.box)[2]
    assert np.abs(F.sum(axis=0)).max() < 1e-10


def test_site_energies_sum_to_total(model, c1):
    E, U, F, W = oracle.energy_forces(model, c1.pos, c1.box)
    assert abs(U.sum() - E) < 1e-9


def test_translation_invariance(model, c1):
    E, U, F, W = oracle.energy_forces(model, c1.pos, c1.box)
    shift = np.array([1.234, -7.77, 3.3])
    E2, U2, F2, W2 = oracle.energy_forces(model, np.mod(c1.pos + shift, c1.box), c1.box)
    assert abs(E2 - E) < 1e-9 * abs(E)
    np.testing.assert_allclose(F2, F, atol=1e-10)
    np.testing.assert_allclose(U2, U, atol=1e-11)


def test_cube_rotation_invariance(model, c1):
    """A 90-degree rotation about z maps the cubic periodic box onto itself exactly."""
    E, U, F, W = oracle.energy_forces(model, c1.pos, c1.box)
    L = c1.box[0]
    R = np.array([[0.0, -1.0, 0.0], [1.0, 0.0, 0.0], [0.0, 0.0, 1.0]])
    xr = np.mod(c1.pos @ R.T, L)
    E2, U2, F2, W2 = oracle.energy_forces(model, xr, c1.box)
    assert abs(E2 - E) < 1e-9 * abs(E)
    np.testing.assert_allclose(F2, F @ R.T, atol=1e-10)
    np.testing.assert_allclose(W2, R @ W @ R.T, atol=1e-8)


def _cluster(seed=3, radius=6.5):
    pos, _ = ni.fcc_lattice(5, 5, 5)
    c = pos.mean(axis=0)
    keep = np.sum((pos - c) ** 2, axis=1) < radius ** 2
    rng = np.random.default_rng(seed)
    cl = pos[keep] - c + rng.normal(0, 0.08, size=(keep.sum(), 3))
    box = np.array([80.0, 80.0, 80.0])
    return cl, box


def test_open_cluster_rotation_invariance(model):
    cl, box = _cluster()
    E, U, F, W = oracle.energy_forces(model, cl + 40.0, box)
    rng = np.random.default_rng(5)
    A = rng.normal(size=(3, 3))
    Q, _ = np.linalg.qr(A)
    if np.linalg.det(Q) < 0:
        Q[:, 0] *= -1
    E2, U2, F2, W2 = oracle.energy_forces(model, cl @ Q.T + 40.0, box)
    assert abs(E2 - E) < 1e-10 * abs(E)
    np.testing.assert_allclose(F2, F @ Q.T, atol=1e-9)


def test_virial_by_finite_strain_cluster(model):
    """Open cluster: a general (non-symmetric) strain of positions; W = (-dE/d eps)^T."""
    cl, box = _cluster()
    E, U, F, W = oracle.energy_forces(model, cl + 40.0, box)
    h = 1e-5
    dE = np.zeros((3, 3))
    for a in range(3):
        for b in range(3):
            ep = np.eye(3); ep[a, b] += h
            em = np.eye(3); em[a, b] -= h
            Ep = oracle.energy_forces(model, cl @ ep.T + 40.0, box)[0]
            Em = oracle.energy_forces(model, cl @ em.T + 40.0, box)[0]
            dE[a, b] = (Ep - Em) / (2 * h)
    np.testing.assert_allclose(W, -dE.T, atol=2e-6 * max(1.0, np.abs(W).max()))


def test_virial_by_finite_strain_periodic(model, c1):
    """Periodic box: diagonal strains scale box and positions together."""
    E, U, F, W = oracle.energy_forces(model, c1.pos, c1.box)
    h = 1e-6
    for a in range(3):
        s = np.ones(3); s[a] += h
        Ep = oracle.energy_forces(model, c1.pos * s, c1.box * s)[0]
        s = np.ones(3); s[a] -= h
        Em = oracle.energy_forces(model, c1.pos * s, c1.box * s)[0]
        assert abs(W[a, a] + (Ep - Em) / (2 * h)) < 1e-5 * abs(W[a, a])


def test_addition_theorem_routes_agree(model, c1):
    q = oracle.descriptors(model, c1.pos, c1.box)
    q3 = oracle.q3b_ylm(model, c1.pos, c1.box)
    np.testing.assert_allclose(q[:, model.nR:model.nR + model.nA * model.lmax], q3, rtol=1e-12, atol=1e-13)


def test_four_body_matches_wigner3j_route(model):
    """tr(T_n^3) equals a fixed multiple of sum 3j(2 2 2; m1 m2 m3) A_m1 A_m2 A_m3 with complex
    Y_2m from scipy and 3j symbols from sympy; the multiple is fixed by one neighbour on the z axis."""
    from scipy.special import sph_harm_y
    from sympy.physics.wigner import wigner_3j
    w3 = {}
    for m1 in range(-2, 3):
        for m2 in range(-2, 3):
            m3 = -m1 - m2
            if abs(m3) <= 2:
                w3[(m1, m2, m3)] = float(wigner_3j(2, 2, 2, m1, m2, m3))
    C = (2.0 / 9.0) / (w3[(0, 0, 0)] * (5.0 / (4 * math.pi)) ** 1.5)
    rng = np.random.default_rng(8)
    cA = model.p["c_A"]
    for trial in range(5):
        nn = 3 + trial
        d = rng.normal(size=(nn, 3))
        d *= (rng.uniform(2.2, 3.9, size=nn) / np.linalg.norm(d, axis=1))[:, None]
        U, dU, q = oracle.atom_site(model.with_changes(lj_eps=0.0), d)
        r = np.linalg.norm(d, axis=1)
        theta = np.arccos(d[:, 2] / r)
        phi = np.arctan2(d[:, 1], d[:, 0])
        for n in range(model.nA):
            g = np.array([_g_ref(cA, ri, model.params["rc_A"])[n] for ri in r])
            A = {m: np.sum(g * sph_harm_y(2, m, theta, phi)) for m in range(-2, 3)}
            val = sum(w * A[m1] * A[m2] * A[m3] for (m1, m2, m3), w in w3.items())
            assert abs(val.imag) < 1e-12
            q4 = q[model.nR + model.nA * model.lmax + n]
            assert abs(q4 - C * val.real) < 1e-10 * max(1.0, abs(q4))


def test_single_neighbor_closed_forms(model):
    r = 3.1
    d = np.array([[0.3, -1.2, math.sqrt(r * r - 0.09 - 1.44)]])
    U, dU, q = oracle.atom_site(model.with_changes(lj_eps=0.0), d)
    gR = _g_ref(model.p["c_R"], r, model.params["rc_R"])
    gA = _g_ref(model.p["c_A"], r, model.params["rc_A"])
    nR, nA, L = model.nR, model.nA, model.lmax
    np.testing.assert_allclose(q[:nR], gR, rtol=1e-12, atol=1e-14)
    for n in range(nA):
        for l in range(1, L + 1):
            assert abs(q[nR + n * L + l - 1] - gA[n] ** 2) < 1e-12 * max(1, gA[n] ** 2)
        assert abs(q[nR + nA * L + n] - 2.0 / 9.0 * gA[n] ** 3) < 1e-12 * max(1, abs(gA[n]) ** 3)


def test_two_neighbor_closed_forms(model):
    r1, r2, theta = 2.6, 3.5, 1.1
    d = np.array([[r1, 0.0, 0.0], [r2 * math.cos(theta), r2 * math.sin(theta), 0.0]])
    U, dU, q = oracle.atom_site(model.with_changes(lj_eps=0.0), d)
    g1 = _g_ref(model.p["c_A"], r1, model.params["rc_A"])
    g2 = _g_ref(model.p["c_A"], r2, model.params["rc_A"])
    nR, L = model.nR, model.lmax
    for n in range(model.nA):
        for l in range(1, L + 1):
            ref = g1[n] ** 2 + g2[n] ** 2 + 2 * g1[n] * g2[n] * eval_legendre(l, math.cos(theta))
            assert abs(q[nR + n * L + l - 1] - ref) < 1e-12 * max(1.0, abs(ref))


def test_radial_function_and_cutoff(model):
    for which, rc, c in ((0, model.params["rc_R"], model.p["c_R"]), (1, model.params["rc_A"], model.p["c_A"])):
        for r in (1.0, 2.5, 0.99 * rc):
            g, dg = oracle.radial(model, which, r)
            np.testing.assert_allclose(g, _g_ref(c, r, rc), rtol=1e-12, atol=1e-14)
            h = 1e-6
            gp, _ = oracle.radial(model, which, r + h)
            gm, _ = oracle.radial(model, which, r - h)
            np.testing.assert_allclose(dg, (gp - gm) / (2 * h), atol=1e-7)
        g, dg = oracle.radial(model, which, rc)
        assert np.abs(g).max() == 0.0 and np.abs(dg).max() == 0.0
        g, dg = oracle.radial(model, which, rc - 1e-4)
        assert np.abs(g).max() < 1e-6 and np.abs(dg).max() < 1e-3


def test_lj_shifted_force_properties(model):
    """The shifted-force pair energy is fixed uniquely by E'' = phi'' (phi the 12-6 LJ potential, whose
    second derivative is 4 eps (156 s^12 / r^14 - 42 s^6 / r^8)) together with E(rc) = E'(rc) = 0."""
    eps, sig, rc = model.params["lj_eps"], model.params["lj_sigma"], model.params["lj_rc"]
    e, de = oracle.lj(model, rc)
    assert e == 0.0 and de == 0.0
    e, de = oracle.lj(model, rc - 1e-6)
    assert abs(e) < 1e-12 and abs(de) < 1e-6
    for r in (2.2, 2.6, 3.4, 4.5):
        e, de = oracle.lj(model, r)
        h = 1e-4
        ep, dep = oracle.lj(model, r + h)
        em, dem = oracle.lj(model, r - h)
        assert abs(de - (ep - em) / (2 * h)) < 1e-7 * max(1.0, abs(de))
        phi2 = 4 * eps * (156 * sig ** 12 / r ** 14 - 42 * sig ** 6 / r ** 8)
        assert abs((dep - dem) / (2 * h) - phi2) < 1e-6 * max(1.0, abs(phi2))


def test_network_index_order_and_bias_signs(model):
    """Sparse network: only W0[2][7], b0[2], w1[2] and b1 are nonzero.  Descriptor 7 is q_{n=0,l=3},
    which for one neighbour equals g^A_0(r)^2.  U = w1_2 tanh(W0_27 * s_7 * q_7 - b0_2) - b1."""
    nneu, ndes = len(model.params["b0"]), model.ndes
    W0 = np.zeros((nneu, ndes)); W0[2, 7] = 0.9
    b0 = np.zeros(nneu); b0[2] = 0.1
    w1 = np.zeros(nneu); w1[2] = 0.3
    qs = np.ones(ndes); qs[7] = 2.0
    m = model.with_changes(W0=W0.tolist(), b0=b0.tolist(), w1=w1.tolist(), b1=0.05, q_scale=qs.tolist(),
                           lj_eps=0.0)
    r = 2.9
    d = np.array([[0.0, r, 0.0]])
    U, dU, q = oracle.atom_site(m, d)
    g = _g_ref(model.p["c_A"], r, model.params["rc_A"])[0]
    assert abs(U - (0.3 * math.tanh(0.9 * 2.0 * g * g - 0.1) - 0.05)) < 1e-13


def test_neighbor_search_cells_match_brute_force():
    wl = ni.fcc_cu_workload(8, sigma=0.1, seed=9)        # 2048 atoms, 4 cells per dimension at 6 A
    for rc in (4.0 + ni.SKIN, 5.0 + ni.SKIN):
        o1, l1 = oracle.neighbor_lists(wl.pos, wl.box, rc, use_cells=False)
        o2, l2 = oracle.neighbor_lists(wl.pos, wl.box, rc, use_cells=True)
        np.testing.assert_array_equal(o1, o2)
        np.testing.assert_array_equal(l1, l2)


def test_neighbor_lists_are_symmetric(c1):
    off, lst = oracle.neighbor_lists(c1.pos, c1.box, 6.0, use_cells=False)
    pairs = set()
    for i in range(c1.n):
        for j in lst[off[i]:off[i + 1]]:
            pairs.add((i, int(j)))
    assert all((j, i) in pairs for (i, j) in pairs)


def test_perfect_fcc(model):
    pos, box = ni.fcc_lattice(4, 4, 4)
    off, _ = oracle.neighbor_lists(pos, box, model.params["rc_A"])
    assert set(np.diff(off)) == {18}          # 12 + 6 neighbours within 4 A
    off, _ = oracle.neighbor_lists(pos, box, model.params["rc_R"])
    assert set(np.diff(off)) == {42}          # 12 + 6 + 24 within 5 A
    E, U, F, W = oracle.energy_forces(model, pos, box)
    assert np.ptp(U) < 1e-12
    assert np.abs(F).max() < 1e-10
    assert abs(W[0, 0] - W[1, 1]) < 1e-9 and abs(W[1, 1] - W[2, 2]) < 1e-9
    assert np.abs(W - np.diag(np.diag(W))).max() < 1e-9


def test_sampled_forces_match_full(model):
    wl = ni.fcc_cu_workload(6, sigma=0.07, seed=4)        # 864 atoms, 3 cells per dimension
    E, U, F, W = oracle.energy_forces(model, wl.pos, wl.box)
    idx = ni.sample_indices(wl.n, 40, seed=1)
    Fs, Us = oracle.forces_sampled(model, wl.pos, wl.box, idx)
    np.testing.assert_allclose(Fs, F[idx], atol=1e-11)
    np.testing.assert_allclose(Us, U[idx], atol=1e-12)
    Fs, Us = oracle.forces_sampled(model, ni.workload("cu_4x4x4").pos, ni.workload("cu_4x4x4").box, idx[:10])
    F4 = oracle.energy_forces(model, ni.workload("cu_4x4x4").pos, ni.workload("cu_4x4x4").box)[2]
    np.testing.assert_allclose(Fs, F4[idx[:10]], atol=1e-11)


def test_nve_energy_drift(model):
    """Velocity Verlet at 1 fs: the slope of a linear fit of the total energy over 10 ps (10^4 steps,
    256 atoms) is below 1e-5 eV/atom/ps."""
    wl = ni.workload("cu_4x4x4")
    x, v, th = oracle.md_nve(model, wl.pos, wl.vel, wl.box, ni.M_CU, 1.0, 10000)
    et = th[:, 2] / wl.n
    t_ps = np.arange(et.size) * 1e-3
    drift = np.polyfit(t_ps, et, 1)[0]
    assert abs(drift) < 1e-5
    assert np.all(np.isfinite(x)) and np.all((x >= 0) & (x < wl.box))


def test_maxwell_boltzmann_generator():
    rng = np.random.default_rng(0)
    v = ni.maxwell_boltzmann(1000, 300.0, ni.M_CU, rng)
    ke = 0.5 * ni.M_CU * np.sum(v * v) * ni.EV_PER_AMU_A2_FS2
    assert abs(2 * ke / ((3 * 1000 - 3) * ni.KB_EV) - 300.0) < 1e-9
    assert np.abs(v.sum(axis=0)).max() < 1e-12
