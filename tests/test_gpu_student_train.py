"""Student training kernels (include/nep_student.h) on the GPU against the FP64 oracle.

  forward       energies, forces and descriptors of the student on three periodic cells vs the oracle
                (NEP-only, float32 kernels): forces 2e-5 eV/Angstrom, energies 1e-6 relative
  JVP           directional derivatives of the descriptors along a random field v, assembled from the
                kernel's basis-sum derivatives, vs central differences of the oracle's descriptors
  gradient      dL/dtheta from the autograd Function (st_jvp + st_grad) vs central differences of the
                same loss evaluated by the FP64 oracle, for parameters of every group
  Adam          the st_adam kernel vs the textbook update written in numpy
  determinism   two gradient evaluations are bitwise equal
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
    from paper_2604_24816_gb300 import student
    student.lib()
    return student


@pytest.fixture(scope="module")
def cells():
    """Three small periodic cells: a displaced fcc cell, a strained one with vacancies, a mixed size."""
    out = []
    wl = ni.fcc_cu_workload(4, 300.0, 0.08, seed=51)
    out.append((wl.pos, wl.box))
    pos, box = ni.student_cell(seed=52, cells=(5, 4, 4), temperature_sigma=0.1, strain=(0.02, -0.03, 0.01),
                               vacancies=3)
    out.append((pos, box))
    wl = ni.fcc_cu_workload(0, sigma=0.06, seed=53, cells_xyz=(4, 4, 5))
    out.append((wl.pos, wl.box))
    return out


@pytest.fixture(scope="module")
def labels(cells, model):
    """Teacher NEP-only energies and forces from the oracle (the training target)."""
    m0 = model.with_changes(lj_eps=0.0)
    E, F = [], []
    for p, b in cells:
        e, u, f, w = oracle.energy_forces(m0, p, b)
        E.append(e); F.append(f)
    return np.array(E), np.concatenate(F)


def _theta32(api, params):
    return api.pack(params).astype(np.float32)


def _oracle_student(api, theta32, base):
    """The student with the float32 parameter values the GPU uses, NEP only."""
    return oracle.Model(api.unpack(theta32.astype(np.float64), dict(base, lj_eps=0.0)))


def test_forward_matches_oracle(api, cells, student_params):
    import torch
    cs = api.CellSet(cells)
    th = _theta32(api, student_params)
    theta = torch.tensor(th, device="cuda")
    qs = torch.tensor(np.asarray(student_params["q_scale"], np.float32), device="cuda")
    E, F = api.student_ef(theta, qs, cs)
    q = cs.descriptors(theta, qs).cpu().numpy().astype(np.float64)
    E, F = E.cpu().numpy(), F.cpu().numpy().astype(np.float64)
    m = _oracle_student(api, th, student_params)
    for s, (p, b) in enumerate(cells):
        a0, a1 = cs.atoms(s, s + 1)
        eo, uo, fo, wo = oracle.energy_forces(m, p, b)
        qo = oracle.descriptors(m, p, b)
        assert abs(E[s] - eo) <= 1e-6 * abs(eo) + 1e-6
        assert np.abs(F[a0:a1] - fo).max() <= 2e-5
        assert (np.abs(q[a0:a1] - qo) / np.maximum(1.0, np.abs(qo).max(axis=0))).max() < 2e-5


def test_jvp_matches_oracle_directional_derivative(api, cells, student_params):
    import torch
    cs = api.CellSet(cells)
    L = api.lib()
    rng = np.random.default_rng(61)
    v = rng.normal(size=(cs.n, 3)).astype(np.float32)
    vt = torch.tensor(v, device="cuda")
    rc = L.st_jvp(0, cs.n, cs.n, cs.cap, api._p(cs.nbr), api._p(cs.dvec), api._p(cs.nnum), cs.rc, api._p(vt),
                  api._p(cs.dQ), api._p(cs.dS), api._stream())
    assert rc == 0
    dQ = cs.dQ.cpu().numpy().astype(np.float64)
    dS = cs.dS.cpu().numpy().astype(np.float64).reshape(-1, 8, 8)      # [atom][k][lm]
    S = cs.S.cpu().numpy().astype(np.float64).reshape(-1, 8, 8)
    th = api.unpack(_theta32(api, student_params).astype(np.float64), student_params)
    cR, cA = np.asarray(th["c_R"]), np.asarray(th["c_A"])
    s = np.einsum("nk,akc->anc", cA, S)
    ds = np.einsum("nk,akc->anc", cA, dS)
    dq = np.zeros((cs.n, 12))
    dq[:, :4] = dQ @ cR.T
    dq[:, 4::2] = 2 * np.einsum("anc,anc->an", s[:, :, :3], ds[:, :, :3])
    dq[:, 5::2] = 2 * np.einsum("anc,anc->an", s[:, :, 3:], ds[:, :, 3:])
    m = _oracle_student(api, _theta32(api, student_params), student_params)
    eps = 1e-4
    for c, (p, b) in enumerate(cells):
        a0, a1 = cs.atoms(c, c + 1)
        vv = v[a0:a1].astype(np.float64)
        fd = (oracle.descriptors(m, p + eps * vv, b) - oracle.descriptors(m, p - eps * vv, b)) / (2 * eps)
        scale = np.abs(fd).max(axis=0)
        assert (np.abs(dq[a0:a1] - fd) / np.maximum(scale, 1e-3)).max() < 5e-4


def _oracle_loss(api, th32, base, cells, E_ref, F_ref, w_E=1.0, w_F=10.0):
    m = _oracle_student(api, th32, base)
    de, df = [], []
    o = 0
    for s, (p, b) in enumerate(cells):
        e, u, f, w = oracle.energy_forces(m, p, b)
        de.append((e - E_ref[s]) / p.shape[0])
        df.append(f - F_ref[o:o + p.shape[0]])
        o += p.shape[0]
    de, df = np.array(de), np.concatenate(df)
    return w_E * np.mean(de ** 2) + w_F * np.mean(df ** 2)


def _gpu_grad(api, cs, th32, qs32):
    import torch
    theta = torch.tensor(th32, device="cuda", requires_grad=True)
    qs = torch.tensor(qs32, device="cuda")
    E, F = api.student_ef(theta, qs, cs)
    loss = api.loss_fn(E, F, cs, 0, cs.n_cells)
    loss.backward()
    return float(loss.item()), theta.grad.detach().cpu().numpy().astype(np.float64)


def test_parameter_gradient_matches_oracle_finite_differences(api, cells, labels, student_params):
    E_ref, F_ref = labels
    cs = api.CellSet(cells, E=E_ref, F=F_ref)
    th32 = _theta32(api, student_params)
    qs32 = np.asarray(student_params["q_scale"], np.float32)
    loss_gpu, g = _gpu_grad(api, cs, th32, qs32)
    loss_o = _oracle_loss(api, th32, student_params, cells, E_ref, F_ref)
    assert abs(loss_gpu - loss_o) <= 1e-5 * loss_o
    # three parameters of each group: c_R, c_A, W0, b0, w1 and b1
    offs = np.cumsum([0] + [int(np.prod(s)) for _, s in api.LAYOUT])
    rng = np.random.default_rng(71)
    picks = [int(offs[-2])]
    for gi in range(5):
        picks += [int(x) for x in rng.choice(np.arange(offs[gi], offs[gi + 1]), size=3, replace=False)]
    gmax = np.abs(g).max()
    for p in picks:
        h = 1e-3 * max(1.0, abs(float(th32[p])))
        tp = th32.astype(np.float64).copy(); tp[p] += h
        tm = th32.astype(np.float64).copy(); tm[p] -= h
        fd = (_oracle_loss(api, tp, student_params, cells, E_ref, F_ref) -
              _oracle_loss(api, tm, student_params, cells, E_ref, F_ref)) / (2 * h)
        assert abs(g[p] - fd) <= 2e-3 * abs(fd) + 1e-4 * gmax, (p, g[p], fd)


def test_gradient_is_deterministic(api, cells, labels, student_params):
    E_ref, F_ref = labels
    cs = api.CellSet(cells, E=E_ref, F=F_ref)
    th32 = _theta32(api, student_params)
    qs32 = np.asarray(student_params["q_scale"], np.float32)
    g1 = _gpu_grad(api, cs, th32, qs32)[1]
    g2 = _gpu_grad(api, cs, th32, qs32)[1]
    assert np.array_equal(g1, g2)


def test_adam_kernel_matches_textbook_update(api):
    import torch
    rng = np.random.default_rng(81)
    n = api.NPAR
    th = rng.normal(size=n).astype(np.float32)
    m = np.zeros(n, np.float32); v = np.zeros(n, np.float32)
    tt, mt, vt = (torch.tensor(a, device="cuda") for a in (th, m, v))
    lr, b1, b2, eps = 1e-2, 0.9, 0.999, 1e-8
    thr, mr, vr = th.astype(np.float64), m.astype(np.float64), v.astype(np.float64)
    for t in range(1, 6):
        g = rng.normal(size=n).astype(np.float32)
        api.adam_step(tt, torch.tensor(g, device="cuda"), mt, vt, lr, t, b1, b2, eps)
        mr = b1 * mr + (1 - b1) * g
        vr = b2 * vr + (1 - b2) * g.astype(np.float64) ** 2
        thr = thr - lr * (mr / (1 - b1 ** t)) / (np.sqrt(vr / (1 - b2 ** t)) + eps)
    np.testing.assert_allclose(tt.cpu().numpy(), thr, rtol=0, atol=2e-6)


def test_short_training_lowers_the_loss(api, cells, labels, student_params):
    import torch
    E_ref, F_ref = labels
    cs = api.CellSet(cells, E=E_ref, F=F_ref)
    theta = torch.tensor(_theta32(api, student_params), device="cuda", requires_grad=True)
    qs = torch.tensor(np.asarray(student_params["q_scale"], np.float32), device="cuda")
    m = torch.zeros_like(theta); v = torch.zeros_like(theta)
    losses = []
    for t in range(1, 61):
        theta.grad = None
        E, F = api.student_ef(theta, qs, cs)
        loss = api.loss_fn(E, F, cs, 0, cs.n_cells)
        loss.backward()
        losses.append(float(loss.item()))
        with torch.no_grad():
            api.adam_step(theta.data, theta.grad, m, v, 3e-3, t)
    assert losses[-1] < 0.5 * losses[0]
