"""Python binding of the C ABI in include/nep_gb300.h (ctypes; argument marshalling only).

Every step of the NEP force evaluation and of the MD integration runs in the CUDA kernels of
libnep_gb300.so.  This module only converts numpy arrays / torch tensors to pointers, forwards the
calls and turns status codes into exceptions.  There is no CPU fallback: if the compiled library is
missing, loading fails with an error.

Arrays may live on the host (numpy, or CPU torch tensors) or on the GPU (CUDA torch tensors); the
library detects which.  Positions, velocities and forces are float64 [n, 3] in the caller's order.
"""
from __future__ import annotations

import ctypes as C
import json
import os
import threading

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_build", "libnep_gb300.so")
DEFAULT_MODEL = os.path.join(_PKG, "params", "cu_nep4_synth.json")
N_KERNEL_CLASSES = 9
PRECISION = {"fp32": 0, "mix_bf16": 1, "mix_fp16": 2}
KERNEL_CLASSES = ("drift", "cell_sort", "neighbors", "descriptor", "force", "kick", "reduce", "other", "fallback")

_lock = threading.Lock()
_lib = None


class NepError(RuntimeError):
    def __init__(self, status: int, name: str, message: str):
        super().__init__(f"{name}: {message}")
        self.status = status
        self.name = name


class nep_params(C.Structure):
    _fields_ = [
        ("n_max_R", C.c_int), ("n_max_A", C.c_int), ("basis_R", C.c_int), ("basis_A", C.c_int),
        ("l_max_3b", C.c_int), ("l_max_4b", C.c_int), ("n_neu", C.c_int),
        ("rc_R", C.c_float), ("rc_A", C.c_float),
        ("c_R", C.POINTER(C.c_float)), ("c_A", C.POINTER(C.c_float)), ("W0", C.POINTER(C.c_float)),
        ("b0", C.POINTER(C.c_float)), ("w1", C.POINTER(C.c_float)), ("b1", C.c_float),
        ("q_scale", C.POINTER(C.c_float)),
        ("lj_eps", C.c_float), ("lj_sigma", C.c_float), ("lj_rc", C.c_float),
        ("mass_amu", C.c_double), ("skin", C.c_float), ("precision", C.c_int),
        ("max_neighbors", C.c_int), ("rebuild_every", C.c_int),
    ]


EXPORTED = ("nep_create", "nep_destroy", "nep_set_state", "nep_build_neighbors", "nep_compute", "md_verlet_step",
            "nep_get_state", "nep_get_thermo", "nep_get_neighbors", "nep_get_descriptors", "nep_get_site_energies",
            "nep_set_timing", "nep_get_timing", "nep_get_counters", "nep_last_error", "nep_status_string",
            "nep_compute_noalloc", "nep_set_fallback", "nep_get_fallback", "nep_run_variant",
            "nep_selftest_bounded_wait", "nep_fp32_peak", "nep_angular_p90")


def lib():
    """Load libnep_gb300.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with `python -m paper_2604_24816_gb300.build`")
        L = C.CDLL(LIB_PATH)
        vp, i64, d = C.c_void_p, C.c_int64, C.POINTER(C.c_double)
        L.nep_create.argtypes = [C.POINTER(nep_params), vp, C.POINTER(vp)]
        L.nep_destroy.argtypes = [vp]
        L.nep_set_state.argtypes = [vp, i64, vp, vp, d]
        L.nep_build_neighbors.argtypes = [vp]
        L.nep_compute.argtypes = [vp, d, vp, d]
        L.md_verlet_step.argtypes = [vp, C.c_double, C.c_int]
        L.nep_get_state.argtypes = [vp, vp, vp]
        L.nep_get_thermo.argtypes = [vp, d]
        L.nep_get_neighbors.argtypes = [vp, vp, vp, vp, vp, C.c_int]
        L.nep_get_descriptors.argtypes = [vp, vp]
        L.nep_get_site_energies.argtypes = [vp, vp]
        L.nep_set_timing.argtypes = [vp, C.c_int]
        L.nep_get_timing.argtypes = [vp, d, C.POINTER(C.c_int64)]
        L.nep_get_counters.argtypes = [vp, C.POINTER(C.c_int64)]
        L.nep_last_error.argtypes = [vp]
        L.nep_last_error.restype = C.c_char_p
        L.nep_status_string.argtypes = [C.c_int]
        L.nep_status_string.restype = C.c_char_p
        L.nep_compute_noalloc.argtypes = [C.POINTER(nep_params), i64, vp, d, vp, vp, vp, vp]
        L.nep_set_fallback.argtypes = [vp, C.POINTER(nep_params), C.POINTER(C.c_float), C.POINTER(C.c_float),
                                       C.c_float, C.c_double]
        L.nep_get_fallback.argtypes = [vp, vp, C.POINTER(C.c_int64)]
        L.nep_run_variant.argtypes = [vp, C.c_int, d, vp]
        L.nep_angular_p90.argtypes = [vp, C.POINTER(C.c_int), C.POINTER(C.c_int)]
        L.nep_selftest_bounded_wait.argtypes = [i64, C.POINTER(C.c_int)]
        L.nep_fp32_peak.argtypes = [C.c_int, C.c_double, C.c_int, vp, d, d, d, C.POINTER(C.c_int)]
        for f in EXPORTED:
            if f not in ("nep_last_error", "nep_status_string"):
                getattr(L, f).restype = C.c_int
        _lib = L
        return L


def load_model(path: str = DEFAULT_MODEL) -> dict:
    with open(path) as f:
        return json.load(f)


def _ptr(a):
    """Data pointer of a numpy array or torch tensor (None -> NULL)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        return a.ctypes.data
    return a.data_ptr()          # torch.Tensor (host or device)


def _as_f64_rows(a, n):
    if isinstance(a, np.ndarray):
        out = np.ascontiguousarray(a, dtype=np.float64)
        if out.shape != (n, 3):
            raise ValueError(f"expected shape ({n}, 3), got {out.shape}")
        return out
    import torch
    if a.dtype != torch.float64 or not a.is_contiguous() or tuple(a.shape) != (n, 3):
        raise ValueError("torch arrays must be contiguous float64 of shape (n, 3)")
    return a


class NEP:
    """One handle of the CUDA library: a model plus one atomic configuration on the GPU."""

    def __init__(self, model: dict | None = None, stream=None, max_neighbors: int = 0, rebuild_every: int = 0,
                 skin: float | None = None, lj: bool = True, precision: str = "fp32"):
        self._L = lib()
        m = load_model() if model is None else model
        f32 = lambda k: np.ascontiguousarray(np.asarray(m[k], dtype=np.float32).ravel())
        self._keep = {k: f32(k) for k in ("c_R", "c_A", "W0", "b0", "w1", "q_scale")}
        fp = lambda k: self._keep[k].ctypes.data_as(C.POINTER(C.c_float))
        p = nep_params(int(m["n_max_R"]), int(m["n_max_A"]), int(m["basis_R"]), int(m["basis_A"]), int(m["l_max_3b"]),
                       int(m["l_max_4b"]), int(m["n_neu"]), float(m["rc_R"]), float(m["rc_A"]),
                       fp("c_R"), fp("c_A"), fp("W0"), fp("b0"), fp("w1"), float(m.get("b1", 0.0)), fp("q_scale"),
                       float(m.get("lj_eps", 0.0)) if lj else 0.0, float(m.get("lj_sigma", 1.0)),
                       float(m.get("lj_rc", m["rc_R"])), float(m.get("mass_amu", 63.546)),
                       float(m.get("skin", 1.0) if skin is None else skin), PRECISION[precision], int(max_neighbors),
                       int(rebuild_every))
        self.model = m
        nA = int(m["n_max_A"]) + 1
        self.n_des = (int(m["n_max_R"]) + 1) + nA * int(m["l_max_3b"]) + (nA if int(m["l_max_4b"]) == 2 else 0)
        h = C.c_void_p()
        st = self._L.nep_create(C.byref(p), C.c_void_p(stream) if stream else None, C.byref(h))
        if st != 0:
            raise NepError(st, self._L.nep_status_string(st).decode(), "nep_create failed")
        self._h = h
        self.n = 0

    # -- plumbing ---------------------------------------------------------------------------------
    def _check(self, st: int):
        if st != 0:
            raise NepError(st, self._L.nep_status_string(st).decode(), self._L.nep_last_error(self._h).decode())

    def close(self):
        if getattr(self, "_h", None):
            self._L.nep_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- C ABI ----------------------------------------------------------------------------------------
    def set_state(self, x, v=None, box=None):
        n = int(x.shape[0])
        x = _as_f64_rows(x, n)
        v = None if v is None else _as_f64_rows(v, n)
        b = np.ascontiguousarray(np.asarray(box, dtype=np.float64).reshape(3))
        self._keep_state = (x, v)
        self._check(self._L.nep_set_state(self._h, n, _ptr(x), _ptr(v), b.ctypes.data_as(C.POINTER(C.c_double))))
        self.n = n

    def build_neighbors(self):
        self._check(self._L.nep_build_neighbors(self._h))

    def compute(self, forces=True, out=None):
        """Returns (E, F [n,3] float64 or None, W [3,3]).  out: optional preallocated host/device buffer."""
        E = C.c_double()
        W = np.zeros(9)
        F = None
        if forces:
            F = out if out is not None else np.zeros((self.n, 3))
        self._check(self._L.nep_compute(self._h, C.byref(E), _ptr(F), W.ctypes.data_as(C.POINTER(C.c_double))))
        return E.value, F, W.reshape(3, 3)

    def step(self, dt_fs: float, n_steps: int = 1):
        self._check(self._L.md_verlet_step(self._h, float(dt_fs), int(n_steps)))

    def get_state(self, x=None, v=None):
        x = np.zeros((self.n, 3)) if x is None else x
        v = np.zeros((self.n, 3)) if v is None else v
        self._check(self._L.nep_get_state(self._h, _ptr(x), _ptr(v)))
        return x, v

    def thermo(self) -> dict:
        out = np.zeros(8)
        self._check(self._L.nep_get_thermo(self._h, out.ctypes.data_as(C.POINTER(C.c_double))))
        return dict(pe=out[0], ke=out[1], temperature=out[2], pressure=out[3], w_diag=out[4:7], rebuilds=int(out[7]))

    def neighbors(self, cap: int = 160):
        """Returns (counts, n_ang, n_own, list[n, cap]) in original atom ids."""
        counts = np.zeros(self.n, dtype=np.int32)
        nang = np.zeros(self.n, dtype=np.int32)
        nown = np.zeros(self.n, dtype=np.int32)
        lst = np.zeros((self.n, cap), dtype=np.int32)
        self._check(self._L.nep_get_neighbors(self._h, counts.ctypes.data, nang.ctypes.data, nown.ctypes.data,
                                              lst.ctypes.data, cap))
        return counts, nang, nown, lst

    def descriptors(self):
        q = np.zeros((self.n, self.n_des), dtype=np.float32)
        self._check(self._L.nep_get_descriptors(self._h, q.ctypes.data))
        return q

    def site_energies(self):
        U = np.zeros(self.n)
        self._check(self._L.nep_get_site_energies(self._h, U.ctypes.data))
        return U

    def set_timing(self, enable: bool = True):
        self._check(self._L.nep_set_timing(self._h, int(enable)))

    def timing(self):
        ms = np.zeros(N_KERNEL_CLASSES)
        cnt = np.zeros(N_KERNEL_CLASSES, dtype=np.int64)
        self._check(self._L.nep_get_timing(self._h, ms.ctypes.data_as(C.POINTER(C.c_double)),
                                           cnt.ctypes.data_as(C.POINTER(C.c_int64))))
        return {k: (float(ms[i]), int(cnt[i])) for i, k in enumerate(KERNEL_CLASSES)}

    def counters(self) -> dict:
        out = np.zeros(13, dtype=np.int64)
        self._check(self._L.nep_get_counters(self._h, out.ctypes.data_as(C.POINTER(C.c_int64))))
        return dict(radial_pairs=int(out[0]), angular_pairs=int(out[1]), evaluations=int(out[2]),
                    rebuilds=int(out[3]), steps=int(out[4]), launches=int(out[5]), list_entries=int(out[6]),
                    active_pairs=int(out[7]), force_list_entries=int(out[8]), force_active_pairs=int(out[9]),
                    force_radial_pairs=int(out[10]), force_angular_pairs=int(out[11]),
                    fallback_atoms=int(out[12]))

    def set_fallback(self, teacher: dict | None, q_lo=None, q_hi=None, margin: float = 0.05,
                     max_fraction: float = 0.0):
        """Per-atom fallback of this (student-shaped) model to `teacher` for atoms whose scaled
        descriptors leave [q_lo - margin w, q_hi + margin w], w = q_hi - q_lo (nep_set_fallback)."""
        if teacher is None:
            self._check(self._L.nep_set_fallback(self._h, None, None, None, 0.0, 0.0))
            return
        f32 = lambda k: np.ascontiguousarray(np.asarray(teacher[k], dtype=np.float32).ravel())
        self._fb_keep = {k: f32(k) for k in ("c_R", "c_A", "W0", "b0", "w1", "q_scale")}
        fp = lambda k: self._fb_keep[k].ctypes.data_as(C.POINTER(C.c_float))
        m = teacher
        p = nep_params(int(m["n_max_R"]), int(m["n_max_A"]), int(m["basis_R"]), int(m["basis_A"]), int(m["l_max_3b"]),
                       int(m["l_max_4b"]), int(m["n_neu"]), float(m["rc_R"]), float(m["rc_A"]),
                       fp("c_R"), fp("c_A"), fp("W0"), fp("b0"), fp("w1"), float(m.get("b1", 0.0)), fp("q_scale"),
                       0.0, float(m.get("lj_sigma", 1.0)), float(m.get("lj_rc", m["rc_R"])),
                       float(m.get("mass_amu", 63.546)), float(m.get("skin", 1.0)), 0, 0, 0)
        lo = np.ascontiguousarray(np.asarray(q_lo, dtype=np.float32))
        hi = np.ascontiguousarray(np.asarray(q_hi, dtype=np.float32))
        self._fb_keep["lo"], self._fb_keep["hi"] = lo, hi
        self._check(self._L.nep_set_fallback(self._h, C.byref(p), lo.ctypes.data_as(C.POINTER(C.c_float)),
                                             hi.ctypes.data_as(C.POINTER(C.c_float)), float(margin),
                                             float(max_fraction)))

    VARIANTS = {"float_scatter": 1, "tile1": 2, "tile3": 3, "half_list": 4, "separate_descriptor": 5,
                "separate_force": 6, "cpb1": 7, "cpb2": 8, "cpb3": 9, "cpb_auto": 10}

    def angular_p90(self):
        """(p90 of the per-atom angular pair count, centres per warp of the CPB rule) (nep_angular_p90)."""
        p90, cpb = C.c_int(0), C.c_int(0)
        self._check(self._L.nep_angular_p90(self._h, C.byref(p90), C.byref(cpb)))
        return p90.value, cpb.value

    def run_variant(self, name: str):
        """One force evaluation with a kernel variant kept for ablation (nep_run_variant): returns
        (variant kernel milliseconds, forces [n][3])."""
        ms = np.zeros(1)
        F = np.zeros((max(self.n, 1), 3))
        self._check(self._L.nep_run_variant(self._h, self.VARIANTS[name], ms.ctypes.data_as(C.POINTER(C.c_double)),
                                            F.ctypes.data))
        return float(ms[0]), F[:self.n]

    def fallback(self):
        """(flags[n] int32, 1 = teacher; number of flagged atoms) of the last force evaluation."""
        flags = np.zeros(max(self.n, 1), dtype=np.int32)
        cnt = C.c_int64(0)
        self._check(self._L.nep_get_fallback(self._h, flags.ctypes.data, C.byref(cnt)))
        return flags[:self.n], int(cnt.value)


def fp32_peak(packed=True, launch_ms: float = 5.0, reps: int = 20, stream=None) -> dict:
    """FP32 throughput of the current device (nep_fp32_peak): FMA chains on every SM, scalar
    (packed=False), packed float2 (True) or packed half2 ("half2", the 16-bit comparison).  Returns best
    and median TFLOP/s over `reps` launches, FMAs per SM clock cycle and the SM count read from the
    device."""
    L = lib()
    form = 2 if packed == "half2" else int(bool(packed))
    best, med, fpc, sms = C.c_double(0), C.c_double(0), C.c_double(0), C.c_int(0)
    st = L.nep_fp32_peak(form, float(launch_ms), int(reps), C.c_void_p(stream) if stream else None,
                         C.byref(best), C.byref(med), C.byref(fpc), C.byref(sms))
    if st != 0:
        raise NepError(st, L.nep_status_string(st).decode(), "nep_fp32_peak failed")
    return {"best_tflops": best.value, "median_tflops": med.value, "fma_per_clock_sm": fpc.value,
            "sm_count": sms.value}
