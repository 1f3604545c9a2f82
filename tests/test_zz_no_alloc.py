"""nep_compute_noalloc: the force evaluation for callers that cannot allocate GPU memory (for example
a plugin held to its host program's memory pool, or code running while that program captures a
stream).  It keeps every intermediate buffer in a fixed array inside the library, so it is checked
here against the handle-based entry point (nep_compute) on consecutive calls: a call must not see
the previous call's leftovers.

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


def test_noalloc_matches_handle_api_on_consecutive_calls(lib, model_params):
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


def test_noalloc_rejects_sizes_beyond_its_scratch(lib, model_params):
    p, keep = _params(lib, model_params)
    n = 8193
    x = np.zeros((n, 3))
    box = np.array([80.0, 80.0, 80.0])
    E = np.zeros(1)
    st = lib.lib().nep_compute_noalloc(C.byref(p), n, x.ctypes.data, box.ctypes.data_as(C.POINTER(C.c_double)),
                                       E.ctypes.data, None, None, None)
    assert lib.lib().nep_status_string(st) == b"NEP_ERR_ARG"
