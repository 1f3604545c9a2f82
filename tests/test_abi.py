"""C-ABI checks that need no GPU: the library loads, exports every symbol the header declares, and
rejects invalid models before touching the device."""
import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "nep_gb300.h")
HEADERS = sorted(os.path.join(ROOT, "include", f) for f in os.listdir(os.path.join(ROOT, "include")) if f.endswith(".h"))


@pytest.fixture(scope="module")
def L():
    from paper_2604_24816_gb300 import build
    build.build()
    from paper_2604_24816_gb300 import nep
    return nep.lib()


def _declared_functions(header=HEADER):
    text = open(header).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(\w+)\s*\(", text, flags=re.M)))


def test_header_declares_the_boundary():
    names = _declared_functions()
    for f in ("nep_create", "nep_build_neighbors", "nep_compute", "md_verlet_step", "nep_set_state", "nep_destroy"):
        assert f in names


def test_library_exports_every_declared_symbol(L):
    assert len(HEADERS) >= 2
    for h in HEADERS:
        for name in _declared_functions(h):
            assert hasattr(L, name), (h, name)


def test_binding_covers_every_declared_symbol():
    from paper_2604_24816_gb300 import nep, student
    declared = set()
    for h in HEADERS:
        declared |= set(_declared_functions(h))
    assert declared <= set(nep.EXPORTED) | set(student.EXPORTED)


def test_status_strings(L):
    assert L.nep_status_string(0) == b"NEP_OK"
    assert L.nep_status_string(3) == b"NEP_ERR_NEIGH_OVERFLOW"
    assert L.nep_status_string(99) == b"NEP_ERR_UNKNOWN"


def _params(model, **kw):
    from paper_2604_24816_gb300 import nep
    keep = {k: np.ascontiguousarray(np.asarray(model[k], dtype=np.float32).ravel())
            for k in ("c_R", "c_A", "W0", "b0", "w1", "q_scale")}
    fp = lambda k: keep[k].ctypes.data_as(C.POINTER(C.c_float))
    vals = dict(n_max_R=model["n_max_R"], n_max_A=model["n_max_A"], basis_R=model["basis_R"],
                basis_A=model["basis_A"], l_max_3b=model["l_max_3b"], l_max_4b=model["l_max_4b"],
                n_neu=model["n_neu"], rc_R=model["rc_R"], rc_A=model["rc_A"], lj_eps=model["lj_eps"],
                lj_sigma=model["lj_sigma"], lj_rc=model["lj_rc"], mass_amu=model["mass_amu"], skin=1.0,
                max_neighbors=0, rebuild_every=0, precision=0)
    vals.update(kw)
    p = nep.nep_params(vals["n_max_R"], vals["n_max_A"], vals["basis_R"], vals["basis_A"], vals["l_max_3b"],
                       vals["l_max_4b"], vals["n_neu"], vals["rc_R"], vals["rc_A"], fp("c_R"), fp("c_A"), fp("W0"),
                       fp("b0"), fp("w1"), 0.0, fp("q_scale"), vals["lj_eps"], vals["lj_sigma"], vals["lj_rc"],
                       vals["mass_amu"], vals["skin"], vals["precision"], vals["max_neighbors"], vals["rebuild_every"])
    return p, keep


@pytest.mark.parametrize("change,expected", [
    (dict(n_neu=16), 8), (dict(l_max_3b=2), 8), (dict(basis_R=9), 8), (dict(precision=7), 8),
    (dict(rc_A=6.0), 1), (dict(lj_rc=7.0), 1), (dict(skin=-1.0), 1), (dict(max_neighbors=1000), 1),
    (dict(mass_amu=0.0), 1),
])
def test_create_rejects_invalid_models_before_device_work(L, model_params, change, expected):
    p, keep = _params(model_params, **change)
    h = C.c_void_p()
    assert L.nep_create(C.byref(p), None, C.byref(h)) == expected
    assert not h.value


def test_null_arguments(L):
    h = C.c_void_p()
    assert L.nep_create(None, None, C.byref(h)) == 1
    assert L.nep_destroy(None) == 0
    assert L.nep_compute(None, None, None, None) == 1
    assert L.md_verlet_step(None, 1.0, 1) == 1
    assert L.nep_last_error(None) == b"null handle"
