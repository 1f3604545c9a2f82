"""nep_compute_noalloc: the force evaluation for callers that cannot allocate GPU memory where they
need forces -- a plugin held to its host program's memory pool or allocation budget, or an embedded
runtime that forbids cudaMalloc after start-up -- and so cannot create a handle.  It keeps every
intermediate buffer in a fixed array inside the library, so it is checked here against the
handle-based entry point (nep_compute) and the FP64 oracle on consecutive calls (a call must not see the
previous call's leftovers), with host, device and NULL output pointers, and against its size limits.

This file is named to be collected last, so a run that stops at the first failure has already run
every other test; it also passes on its own in a fresh process.
"""
import ctypes as C

import numpy as np
import pytest

import nep_inputs as ni

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2604_24816_gb300 import build
    build.build()
    from paper_2604_24816_gb300 import nep
    return nep


def _params(nep, model):
    keep = {k: np.ascontiguousarray(np.asarray(model[k], dtype=np.float32).ravel())
            for k in ("c_R", "c_A", "W0", "b0", "w1", "q_scale")}
    fp = lambda k: keep[k].ctypes.data_as(C.POINTER(C.c_float))
    p = nep.nep_params(model["n_max_R"], model["n_max_A"], model["basis_R"], model["basis_A"], model["l_max_3b"],
                       model["l_max_4b"], model["n_neu"], model["rc_R"], model["rc_A"], fp("c_R"), fp("c_A"),
                       fp("W0"), fp("b0"), fp("w1"), float(model.get("b1", 0.0)), fp("q_scale"), model["lj_eps"],
                       model["lj_sigma"], model["lj_rc"], model["mass_amu"], model["skin"], 0, 0, 0)
    return p, keep


def _noalloc(nep, p, x, box, on_device):
    import torch
    n = x.shape[0]
    box_c = np.ascontiguousarray(box, dtype=np.float64)
    if on_device:
        xd = torch.from_numpy(np.ascontiguousarray(x)).cuda()
        E = torch.zeros(1, dtype=torch.float64, device="cuda")
        F = torch.zeros((n, 3), dtype=torch.float64, device="cuda")
        W = torch.zeros(9, dtype=torch.float64, device="cuda")
        st = nep.lib().nep_compute_noalloc(C.byref(p), n, xd.data_ptr(), box_c.ctypes.data_as(C.POINTER(C.c_double)),
                                           E.data_ptr(), F.data_ptr(), W.data_ptr(), None)
        return st, float(E.item()), F.cpu().numpy(), W.cpu().numpy().reshape(3, 3)
    xh = np.ascontiguousarray(x, dtype=np.float64)
    E = np.zeros(1); F = np.zeros((n, 3)); W = np.zeros(9)
    st = nep.lib().nep_compute_noalloc(C.byref(p), n, xh.ctypes.data, box_c.ctypes.data_as(C.POINTER(C.c_double)),
                                       E.ctypes.data, F.ctypes.data, W.ctypes.data, None)
    return st, float(E[0]), F, W.reshape(3, 3)


def _reference(nep, model, wl):
    with nep.NEP(model) as h:
        h.set_state(wl.pos, wl.vel, wl.box)
        return h.compute()


def test_noalloc_matches_handle_api_on_consecutive_calls(lib, model_params, model):
    import oracle
    p, keep = _params(lib, model_params)
    a = ni.workload("cu_4x4x4")                                   # 256 atoms
    b = ni.fcc_cu_workload(0, sigma=0.07, seed=12, cells_xyz=(6, 6, 5))   # 720 atoms, other box
    for wl, on_device in ((a, True), (b, False), (a, False), (b, True)):
        st, E, F, W = _noalloc(lib, p, wl.pos, wl.box, on_device)
        assert st == 0, lib.lib().nep_status_string(st)
        Er, Fr, Wr = _reference(lib, model_params, wl)
        assert np.abs(F - Fr).max() <= 1e-4
        assert abs(E - Er) <= 1e-6 * abs(Er)
        assert np.abs(W - Wr).max() <= 1e-5 * np.abs(Wr).max()
        # and the FP64 oracle, at the float32 path's bounds
        Eo, Uo, Fo, Wo = oracle.energy_forces(model, wl.pos, wl.box)
        assert np.abs(F - Fo).max() <= 1e-4
        assert abs(E - Eo) <= 1e-6 * abs(Eo)
        assert np.abs(W - Wo).max() <= 1e-5 * np.abs(Wo).max()


def test_noalloc_output_pointers(lib, model_params):
    """No atoms (E and virial zeroed, host or device); forces on the device with E and virial on the
    host; no forces requested."""
    import torch
    p, keep = _params(lib, model_params)
    L = lib.lib()
    dp = lambda a: a.ctypes.data_as(C.POINTER(C.c_double))
    box = np.array([20.0, 20.0, 20.0])
    Eh, Wh = np.full(1, 7.0), np.full(9, 7.0)
    assert L.nep_compute_noalloc(C.byref(p), 0, None, dp(box), Eh.ctypes.data, None, Wh.ctypes.data, None) == 0
    assert Eh[0] == 0.0 and not Wh.any()
    Ed = torch.full((1,), 7.0, dtype=torch.float64, device="cuda")
    Wd = torch.full((9,), 7.0, dtype=torch.float64, device="cuda")
    assert L.nep_compute_noalloc(C.byref(p), 0, None, dp(box), Ed.data_ptr(), None, Wd.data_ptr(), None) == 0
    assert float(Ed.item()) == 0.0 and not Wd.any().item()
    wl = ni.workload("cu_4x4x4")
    Er, Fr, Wr = _reference(lib, model_params, wl)
    x = np.ascontiguousarray(wl.pos)
    Fd = torch.zeros((wl.n, 3), dtype=torch.float64, device="cuda")
    E, W = np.zeros(1), np.zeros(9)
    assert L.nep_compute_noalloc(C.byref(p), wl.n, x.ctypes.data, dp(wl.box), E.ctypes.data, Fd.data_ptr(),
                                 W.ctypes.data, None) == 0
    assert np.abs(Fd.cpu().numpy() - Fr).max() <= 1e-4 and abs(E[0] - Er) <= 1e-6 * abs(Er)
    assert np.abs(W.reshape(3, 3) - Wr).max() <= 1e-5 * np.abs(Wr).max()
    E2 = np.zeros(1)
    assert L.nep_compute_noalloc(C.byref(p), wl.n, x.ctypes.data, dp(wl.box), E2.ctypes.data, None, None, None) == 0
    assert E2[0] == E[0]


def test_noalloc_rejects_sizes_beyond_its_scratch(lib, model_params):
    """Too many atoms, or a box of more neighbour cells than the scratch array holds (few atoms): both
    NEP_ERR_ARG before any GPU work."""
    p, keep = _params(lib, model_params)
    L = lib.lib()
    E = np.zeros(1)
    n = 8193
    x = np.zeros((n, 3))
    box = np.array([80.0, 80.0, 80.0])
    st = L.nep_compute_noalloc(C.byref(p), n, x.ctypes.data, box.ctypes.data_as(C.POINTER(C.c_double)),
                               E.ctypes.data, None, None, None)
    assert L.nep_status_string(st) == b"NEP_ERR_ARG"
    rl = model_params["rc_R"] + model_params["skin"]
    # 33 x 32 x 32 = 33,792 cells of edge >= rc_R + skin, one more row than NEP_NOALLOC_MAX_CELLS allows
    big = np.array([33 * rl + 0.1, 32 * rl + 0.1, 32 * rl + 0.1])
    x = np.random.default_rng(3).random((10, 3)) * big
    st = L.nep_compute_noalloc(C.byref(p), 10, x.ctypes.data, big.ctypes.data_as(C.POINTER(C.c_double)),
                               E.ctypes.data, None, None, None)
    assert L.nep_status_string(st) == b"NEP_ERR_ARG"
    ok = np.array([32 * rl + 0.1, 32 * rl + 0.1, 32 * rl + 0.1])  # exactly 32,768 cells: accepted
    x = np.array([[5.0 + 15.0 * k, 7.0, 7.0] for k in range(10)])  # isolated atoms, 15 A apart
    st = L.nep_compute_noalloc(C.byref(p), 10, x.ctypes.data, ok.ctypes.data_as(C.POINTER(C.c_double)),
                               E.ctypes.data, None, None, None)
    assert st == 0, L.nep_status_string(st)
