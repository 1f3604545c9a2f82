"""Pins for the FP64 oracle on the student model shape (radial n_max 3, angular n_max 3, l_max 2, no
4-body term, 16 neurons; no GPU).

Besides the physics pins (forces = -grad E, sum F = 0, rotation invariance, closed forms for one and
two neighbours), the student is tied to the pinned teacher route: a teacher-shaped model whose fifth
channels, l = 3, 4 and 4-body weights are zero and whose remaining weights are the student's
computes the same site energies, which fails on any index or shape mistake of the student path.
"""
import math

import numpy as np
import pytest
from numpy.polynomial import chebyshev as npcheb
from scipy.special import eval_legendre

import nep_inputs as ni
import oracle


def _g_ref(c, r, rc):
    x = 2.0 * (r / rc - 1.0) ** 2 - 1.0
    fc = 0.5 * (1.0 + math.cos(math.pi * r / rc)) if r < rc else 0.0
    K = c.shape[1]
    f = np.array([0.5 * (npcheb.chebval(x, np.eye(K)[k]) + 1.0) * fc for k in range(K)])
    return c @ f


@pytest.fixture(scope="module")
def cell():
    return ni.fcc_cu_workload(4, 300.0, 0.08, seed=21)


def test_student_descriptor_count(student_model):
    assert student_model.ndes == 4 + 4 * 2 == 12
    assert student_model.nR == 4 and student_model.nA == 4 and student_model.lmax == 2


@pytest.mark.parametrize("lj_on", [True, False])
def test_student_forces_are_minus_energy_gradient(student_model, cell, lj_on):
    m = student_model if lj_on else student_model.with_changes(lj_eps=0.0)
    E, U, F, W = oracle.energy_forces(m, cell.pos, cell.box)
    rng = np.random.default_rng(12)
    h = 2e-5
    for _ in range(8):
        i, a = int(rng.integers(cell.n)), int(rng.integers(3))
        xp = cell.pos.copy(); xp[i, a] += h
        xm = cell.pos.copy(); xm[i, a] -= h
        fd = -(oracle.energy_forces(m, xp, cell.box)[0] - oracle.energy_forces(m, xm, cell.box)[0]) / (2 * h)
        assert abs(fd - F[i, a]) <= 1e-7 * max(1.0, abs(F[i, a]))
    assert np.abs(F.sum(axis=0)).max() < 1e-10


def test_student_cube_rotation_invariance(student_model, cell):
    E0 = oracle.energy_forces(student_model, cell.pos, cell.box)[0]
    # 90-degree rotation about z in a cubic box, mapped back into the box
    R = np.array([[0.0, -1.0, 0.0], [1.0, 0.0, 0.0], [0.0, 0.0, 1.0]])
    x = np.mod(cell.pos @ R.T, cell.box)
    E1 = oracle.energy_forces(student_model, x, cell.box)[0]
    assert abs(E1 - E0) < 1e-10 * abs(E0)


def test_student_single_and_two_neighbor_closed_forms(student_model):
    m = student_model.with_changes(lj_eps=0.0)
    r = 3.1
    d = np.array([[0.3, -1.2, math.sqrt(r * r - 0.09 - 1.44)]])
    q = oracle.atom_site(m, d)[2]
    assert q.shape == (12,)
    np.testing.assert_allclose(q[:4], _g_ref(m.p["c_R"], r, 5.0), rtol=1e-12, atol=1e-14)
    gA = _g_ref(m.p["c_A"], r, 4.0)
    for n in range(4):
        for l in (1, 2):
            assert abs(q[4 + 2 * n + l - 1] - gA[n] ** 2) < 1e-12 * max(1, gA[n] ** 2)
    r1, r2, th = 2.6, 3.5, 1.1
    d = np.array([[r1, 0.0, 0.0], [r2 * math.cos(th), r2 * math.sin(th), 0.0]])
    q = oracle.atom_site(m, d)[2]
    g1, g2 = _g_ref(m.p["c_A"], r1, 4.0), _g_ref(m.p["c_A"], r2, 4.0)
    for n in range(4):
        for l in (1, 2):
            ref = g1[n] ** 2 + g2[n] ** 2 + 2 * g1[n] * g2[n] * eval_legendre(l, math.cos(th))
            assert abs(q[4 + 2 * n + l - 1] - ref) < 1e-12 * max(1.0, abs(ref))


def test_student_equals_embedded_teacher(student_params, cell):
    """Embed the student in the teacher shape (zero fifth channels, l = 3, 4 and 4-body weights)."""
    sp = student_params
    nneu_t = 30
    cR = np.zeros((5, 8)); cR[:4] = np.asarray(sp["c_R"])
    cA = np.zeros((5, 8)); cA[:4] = np.asarray(sp["c_A"])
    W0s = np.asarray(sp["W0"]); qs_s = np.asarray(sp["q_scale"])
    W0 = np.zeros((nneu_t, 30)); qs = np.ones(30)
    b0 = np.zeros(nneu_t); w1 = np.zeros(nneu_t)
    b0[:16] = sp["b0"]; w1[:16] = sp["w1"]
    # student index -> teacher index: radial n -> n; q_{n,l} (l = 1, 2) -> 5 + 4 n + l - 1
    cols = list(range(4)) + [5 + 4 * n + l - 1 for n in range(4) for l in (1, 2)]
    for k, c in enumerate(cols):
        W0[:16, c] = W0s[:, k]
        qs[c] = qs_s[k]
    # neurons 16..29 get b0 = 0, w1 = 0 (no contribution); their tanh(0) is 0 anyway
    teacher = dict(ni.NEP_DIMS, rc_R=5.0, rc_A=4.0, c_R=cR.tolist(), c_A=cA.tolist(), W0=W0.tolist(),
                   b0=b0.tolist(), w1=w1.tolist(), b1=sp["b1"], q_scale=qs.tolist(), lj_eps=sp["lj_eps"],
                   lj_sigma=sp["lj_sigma"], lj_rc=sp["lj_rc"])
    Es, Us, Fs, Ws = oracle.energy_forces(oracle.Model(sp), cell.pos, cell.box)
    Et, Ut, Ft, Wt = oracle.energy_forces(oracle.Model(teacher), cell.pos, cell.box)
    np.testing.assert_allclose(Us, Ut, rtol=0, atol=1e-12)
    np.testing.assert_allclose(Fs, Ft, rtol=0, atol=1e-11)


def test_select_reduces_to_single_models(student_model, model, cell):
    n = cell.n
    for flags, ref in ((np.zeros(n), student_model), (np.ones(n), model)):
        E, U, F, W = oracle.energy_forces_select(student_model, model, flags, cell.pos, cell.box)
        Er, Ur, Fr, Wr = oracle.energy_forces(ref, cell.pos, cell.box)
        assert abs(E - Er) < 1e-12 * abs(Er)
        np.testing.assert_allclose(F, Fr, rtol=0, atol=1e-12)
        np.testing.assert_allclose(W, Wr, rtol=0, atol=1e-10)


def test_select_forces_are_minus_gradient_with_fixed_flags(student_model, model, cell):
    """A mixed assignment (every third atom on the teacher): forces = -grad E at fixed flags."""
    flags = (np.arange(cell.n) % 3 == 0).astype(np.int32)
    E, U, F, W = oracle.energy_forces_select(student_model, model, flags, cell.pos, cell.box)
    assert np.abs(F.sum(axis=0)).max() < 1e-10
    Us = oracle.energy_forces(student_model, cell.pos, cell.box)[1]
    Ut = oracle.energy_forces(model, cell.pos, cell.box)[1]
    np.testing.assert_allclose(U, np.where(flags == 1, Ut, Us), rtol=0, atol=1e-12)
    rng = np.random.default_rng(13)
    h = 2e-5
    for _ in range(6):
        i, a = int(rng.integers(cell.n)), int(rng.integers(3))
        xp = cell.pos.copy(); xp[i, a] += h
        xm = cell.pos.copy(); xm[i, a] -= h
        fd = -(oracle.energy_forces_select(student_model, model, flags, xp, cell.box)[0] -
               oracle.energy_forces_select(student_model, model, flags, xm, cell.box)[0]) / (2 * h)
        assert abs(fd - F[i, a]) <= 1e-7 * max(1.0, abs(F[i, a]))
