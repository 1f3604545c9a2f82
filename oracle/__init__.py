"""FP64 CPU oracle for NEP molecular dynamics -- TEST INFRASTRUCTURE ONLY.

Only the test suite, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg may import this
package.  The product path (the CUDA library and its binding) never imports it and shares no code
with it.  The arithmetic lives in ``nep_oracle.c`` (plain C, double precision, OpenMP over atoms with
fixed-order reductions); this module compiles it with gcc and marshals numpy arrays.
"""
from __future__ import annotations

import ctypes as C
import json
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "nep_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle shared library with gcc (-O2, OpenMP).  Returns its path."""
    os.makedirs(_BUILD, exist_ok=True)
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Params(C.Structure):
    _fields_ = [
        ("nR", C.c_int), ("nA", C.c_int), ("kR", C.c_int), ("kA", C.c_int), ("lmax", C.c_int),
        ("nneu", C.c_int), ("ndes", C.c_int), ("fourbody", C.c_int),
        ("rcR", C.c_double), ("rcA", C.c_double),
        ("cR", C.POINTER(C.c_double)), ("cA", C.POINTER(C.c_double)), ("W0", C.POINTER(C.c_double)),
        ("b0", C.POINTER(C.c_double)), ("w1", C.POINTER(C.c_double)), ("b1", C.c_double),
        ("qscale", C.POINTER(C.c_double)),
        ("lj_eps", C.c_double), ("lj_sigma", C.c_double), ("lj_rc", C.c_double),
    ]


_D = C.POINTER(C.c_double)
_I32 = C.POINTER(C.c_int32)
_I64 = C.POINTER(C.c_int64)


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            P = C.POINTER(_Params)
            L.oracle_set_threads.argtypes = [C.c_int]
            L.oracle_get_threads.restype = C.c_int
            L.oracle_neighbor_counts.argtypes = [C.c_int, _D, _D, C.c_double, C.c_int, _I32]
            L.oracle_neighbor_lists.argtypes = [C.c_int, _D, _D, C.c_double, C.c_int, _I64, _I32]
            L.oracle_descriptors.argtypes = [P, C.c_int, _D, _D, _D]
            L.oracle_energy_forces.argtypes = [P, C.c_int, _D, _D, _D, _D, _D, _D]
            L.oracle_energy_forces_select.argtypes = [P, P, _I32, C.c_int, _D, _D, _D, _D, _D, _D]
            L.oracle_forces_sampled.argtypes = [P, C.c_int, _D, _D, C.c_int, _I64, _D, _D]
            L.oracle_q3b_ylm.argtypes = [P, C.c_int, _D, _D, _D]
            L.oracle_radial.argtypes = [P, C.c_int, C.c_double, _D, _D]
            L.oracle_lj.argtypes = [P, C.c_double, _D, _D]
            L.oracle_atom_site.argtypes = [P, C.c_int, _D, _D, _D]
            L.oracle_atom_site.restype = C.c_double
            L.oracle_md_nve.argtypes = [P, C.c_int, _D, _D, _D, C.c_double, C.c_double, C.c_int, _D]
            for f in ("oracle_neighbor_counts", "oracle_neighbor_lists", "oracle_descriptors",
                      "oracle_energy_forces", "oracle_energy_forces_select", "oracle_forces_sampled",
                      "oracle_q3b_ylm", "oracle_md_nve"):
                getattr(L, f).restype = C.c_int
            _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(_D)


def _f64(a, shape=None):
    out = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    if shape is not None:
        out = out.reshape(shape)
    return out


class Model:
    """NEP parameters held as contiguous float64 arrays plus the ctypes struct that points at them."""

    def __init__(self, params: dict):
        self.p = {}
        nR = int(params["n_max_R"]) + 1
        nA = int(params["n_max_A"]) + 1
        kR, kA = int(params["basis_R"]), int(params["basis_A"])
        lmax, nneu = int(params["l_max_3b"]), int(params["n_neu"])
        fourbody = 1 if int(params.get("l_max_4b", 2)) > 0 else 0
        ndes = nR + nA * lmax + (nA if fourbody else 0)
        self.ndes, self.nR, self.nA, self.lmax = ndes, nR, nA, lmax
        for k, shape in (("c_R", (nR, kR)), ("c_A", (nA, kA)), ("W0", (nneu, ndes)), ("b0", (nneu,)),
                         ("w1", (nneu,)), ("q_scale", (ndes,))):
            self.p[k] = _f64(params[k], shape)
        self.s = _Params(nR, nA, kR, kA, lmax, nneu, ndes, fourbody, float(params["rc_R"]), float(params["rc_A"]),
                         _dp(self.p["c_R"]), _dp(self.p["c_A"]), _dp(self.p["W0"]), _dp(self.p["b0"]),
                         _dp(self.p["w1"]), float(params.get("b1", 0.0)), _dp(self.p["q_scale"]),
                         float(params.get("lj_eps", 0.0)), float(params.get("lj_sigma", 1.0)),
                         float(params.get("lj_rc", 0.0)))
        self.params = dict(params)

    def ref(self):
        return C.byref(self.s)

    def with_changes(self, **kw) -> "Model":
        p = dict(self.params)
        p.update(kw)
        return Model(p)


def load_model(path: str) -> Model:
    with open(path) as f:
        return Model(json.load(f))


def set_threads(t: int) -> None:
    lib().oracle_set_threads(int(t))


def get_threads() -> int:
    return int(lib().oracle_get_threads())


def neighbor_lists(x, box, rc: float, use_cells: bool = True):
    """CSR neighbour lists (strict r < rc, minimum image, ascending j per row)."""
    x = _f64(x, (-1, 3)); box = _f64(box, (3,))
    n = x.shape[0]
    counts = np.zeros(n, dtype=np.int32)
    if lib().oracle_neighbor_counts(n, _dp(x), _dp(box), rc, int(use_cells), counts.ctypes.data_as(_I32)) != 0:
        raise RuntimeError("oracle neighbour search overflow")
    off = np.zeros(n + 1, dtype=np.int64)
    lst = np.zeros(max(int(counts.sum()), 1), dtype=np.int32)
    if lib().oracle_neighbor_lists(n, _dp(x), _dp(box), rc, int(use_cells), off.ctypes.data_as(_I64),
                                   lst.ctypes.data_as(_I32)) != 0:
        raise RuntimeError("oracle neighbour search overflow")
    return off, lst[: off[-1]]


def descriptors(model: Model, x, box):
    x = _f64(x, (-1, 3)); box = _f64(box, (3,))
    q = np.zeros((x.shape[0], model.ndes))
    if lib().oracle_descriptors(model.ref(), x.shape[0], _dp(x), _dp(box), _dp(q)) != 0:
        raise RuntimeError("oracle_descriptors failed")
    return q


def energy_forces(model: Model, x, box):
    """Returns (E, U[n], F[n,3], W[3,3])."""
    x = _f64(x, (-1, 3)); box = _f64(box, (3,))
    n = x.shape[0]
    E = np.zeros(1); U = np.zeros(n); F = np.zeros((n, 3)); W = np.zeros(9)
    if lib().oracle_energy_forces(model.ref(), n, _dp(x), _dp(box), _dp(E), _dp(U), _dp(F), _dp(W)) != 0:
        raise RuntimeError("oracle_energy_forces failed")
    return float(E[0]), U, F, W.reshape(3, 3)


def energy_forces_select(model_a: Model, model_b: Model, flags, x, box):
    """Energy, site energies, forces and virial when atom i's site energy comes from model_b where
    flags[i] != 0 and from model_a elsewhere (each atom's own model differentiated).
    Returns (E, U[n], F[n,3], W[3,3])."""
    x = _f64(x, (-1, 3)); box = _f64(box, (3,))
    n = x.shape[0]
    fl = np.ascontiguousarray(np.asarray(flags, dtype=np.int32).reshape(n))
    E = np.zeros(1); U = np.zeros(n); F = np.zeros((n, 3)); W = np.zeros(9)
    if lib().oracle_energy_forces_select(model_a.ref(), model_b.ref(), fl.ctypes.data_as(_I32), n, _dp(x), _dp(box),
                                         _dp(E), _dp(U), _dp(F), _dp(W)) != 0:
        raise RuntimeError("oracle_energy_forces_select failed")
    return float(E[0]), U, F, W.reshape(3, 3)


def forces_sampled(model: Model, x, box, idx):
    """Forces and site energies on the atoms idx only.  Returns (F[len,3], U[len])."""
    x = _f64(x, (-1, 3)); box = _f64(box, (3,))
    idx = np.ascontiguousarray(np.asarray(idx, dtype=np.int64))
    F = np.zeros((idx.size, 3)); U = np.zeros(idx.size)
    if lib().oracle_forces_sampled(model.ref(), x.shape[0], _dp(x), _dp(box), idx.size,
                                   idx.ctypes.data_as(_I64), _dp(F), _dp(U)) != 0:
        raise RuntimeError("oracle_forces_sampled failed")
    return F, U


def q3b_ylm(model: Model, x, box):
    x = _f64(x, (-1, 3)); box = _f64(box, (3,))
    q = np.zeros((x.shape[0], model.nA * model.lmax))
    if lib().oracle_q3b_ylm(model.ref(), x.shape[0], _dp(x), _dp(box), _dp(q)) != 0:
        raise RuntimeError("oracle_q3b_ylm failed")
    return q


def radial(model: Model, which: int, r: float):
    n = model.nR if which == 0 else model.nA
    g = np.zeros(n); dg = np.zeros(n)
    lib().oracle_radial(model.ref(), int(which), float(r), _dp(g), _dp(dg))
    return g, dg


def lj(model: Model, r: float):
    e = np.zeros(1); de = np.zeros(1)
    lib().oracle_lj(model.ref(), float(r), _dp(e), _dp(de))
    return float(e[0]), float(de[0])


def atom_site(model: Model, dvecs):
    """Site energy, dU/dr_ij and unscaled descriptors of one atom with neighbour vectors dvecs[nn,3]."""
    d = _f64(dvecs, (-1, 3))
    dU = np.zeros_like(d); q = np.zeros(model.ndes)
    U = lib().oracle_atom_site(model.ref(), d.shape[0], _dp(d), _dp(dU), _dp(q))
    return float(U), dU, q


def md_nve(model: Model, x, v, box, mass: float, dt: float, nsteps: int):
    """Velocity-Verlet NVE.  Returns (x, v, thermo[nsteps+1, 4] = (PE, KE, Etot, T))."""
    x = _f64(x, (-1, 3)).copy(); v = _f64(v, (-1, 3)).copy(); box = _f64(box, (3,))
    th = np.zeros((nsteps + 1, 4))
    if lib().oracle_md_nve(model.ref(), x.shape[0], _dp(x), _dp(v), _dp(box), float(mass), float(dt),
                           int(nsteps), _dp(th)) != 0:
        raise RuntimeError("oracle_md_nve failed")
    return x, v, th
