"""Student-NEP training through the hand-written kernels declared in include/nep_student.h.

    cells = CellSet([(pos, box), ...], E=..., F=...)          # neighbour lists + basis sums on the GPU
    theta = torch.tensor(pack(model), device="cuda", requires_grad=True)
    E, F = StudentEF.apply(theta, q_scale, cells, s0, s1)     # energies of cells [s0, s1), their forces
    loss(E, F).backward()                                     # theta.grad from st_jvp + st_grad

The model is the NEP form of Section III.B with the student shape (radial n_max 3, angular n_max 3,
l_max 2, no 4-body term, 16 neurons).  Every step of the forward and backward pass runs in the CUDA
kernels; this module only allocates device buffers (PyTorch) and marshals pointers.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import nep as _nep

EXPORTED = ("st_pairs", "st_basis", "st_forward", "st_energy", "st_force", "st_jvp", "st_grad_scratch", "st_grad",
            "st_adam")
DIMS = dict(n_max_R=3, n_max_A=3, basis_R=8, basis_A=8, l_max_3b=2, l_max_4b=0, n_neu=16)
NR, NA, KB, NLM, NDES, NNEU, GS = 4, 4, 8, 8, 12, 16, 40
NSB = KB * NLM
# parameter vector: c_R [4][8] | c_A [4][8] | W0 [16][12] | b0 [16] | w1 [16] | b1
LAYOUT = (("c_R", (NR, KB)), ("c_A", (NA, KB)), ("W0", (NNEU, NDES)), ("b0", (NNEU,)), ("w1", (NNEU,)), ("b1", ()))
NPAR = sum(int(np.prod(s)) for _, s in LAYOUT)


class st_cutoffs(C.Structure):
    _fields_ = [("rc_R", C.c_float), ("rc_A", C.c_float)]


_ready = False


def lib():
    global _ready
    L = _nep.lib()
    if not _ready:
        vp, i = C.c_void_p, C.c_int
        L.st_pairs.argtypes = [i, vp, vp, vp, st_cutoffs, i, vp, vp, vp, vp, vp]
        L.st_basis.argtypes = [i, i, i, i, vp, vp, vp, st_cutoffs, vp, vp, vp]
        L.st_forward.argtypes = [i, i, vp, vp, vp, vp, vp, vp, vp, vp]
        L.st_energy.argtypes = [i, i, vp, vp, vp, vp]
        L.st_force.argtypes = [i, i, i, i, vp, vp, vp, st_cutoffs, vp, vp, vp, vp]
        L.st_jvp.argtypes = [i, i, i, i, vp, vp, vp, st_cutoffs, vp, vp, vp, vp]
        L.st_grad_scratch.argtypes = [i, i]
        L.st_grad_scratch.restype = C.c_int64
        L.st_grad.argtypes = [i, i, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp]
        L.st_adam.argtypes = [i, vp, vp, vp, vp, C.c_float, C.c_float, C.c_float, C.c_float, i, vp]
        for f in EXPORTED:
            if f != "st_grad_scratch":
                getattr(L, f).restype = C.c_int
        _ready = True
    return L


def _chk(rc: int, what: str):
    if rc != 0:
        raise RuntimeError(f"{what}: CUDA error {rc}")


def _p(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream():
    import torch
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def pack(model: dict) -> np.ndarray:
    """Model dict -> float32 parameter vector in the kernels' order."""
    return np.concatenate([np.asarray(model[k], dtype=np.float64).reshape(-1) for k, _ in LAYOUT]).astype(np.float32)


def unpack(theta, base: dict) -> dict:
    """Parameter vector -> model dict (other fields taken from `base`)."""
    t = np.asarray(theta, dtype=np.float64).reshape(-1)
    out, o = dict(base), 0
    for k, shape in LAYOUT:
        m = int(np.prod(shape))
        v = t[o:o + m]
        out[k] = float(v[0]) if shape == () else v.reshape(shape).tolist()
        o += m
    return out


class CellSet:
    """Periodic cells resident on the GPU, stored one after another, with their neighbour lists and the
    per-atom basis sums Q, S (both built once, by st_pairs and st_basis).  Optional labels: E [cells]
    (float64) and F [atoms][3]."""

    def __init__(self, cells, rc_R: float = 5.0, rc_A: float = 4.0, cap: int = 96, E=None, F=None,
                 device: str = "cuda"):
        import torch
        L = lib()
        self.n_cells = len(cells)
        sizes = [int(np.asarray(p).shape[0]) for p, _ in cells]
        self.start_h = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
        self.n = int(self.start_h[-1])
        pos = np.zeros((self.n, 4), dtype=np.float32)
        boxes = np.zeros((self.n_cells, 3), dtype=np.float32)
        for s, (p, b) in enumerate(cells):
            b = np.asarray(b, dtype=np.float64)
            if np.any(b < 2 * rc_R):
                raise ValueError(f"cell {s}: box {b} smaller than 2 * rc_R")
            a0, a1 = self.start_h[s], self.start_h[s + 1]
            pos[a0:a1, :3] = np.mod(np.asarray(p, dtype=np.float64), b)
            pos[a0:a1, 3] = np.array([s], dtype=np.int32).view(np.float32)[0]
            boxes[s] = b
        self.rc = st_cutoffs(rc_R, rc_A)
        self.cap = cap
        dev = torch.device(device)
        self.pos = torch.from_numpy(pos).to(dev)
        self.start = torch.from_numpy(self.start_h.astype(np.int32)).to(dev)
        self.boxes = torch.from_numpy(boxes).to(dev)
        self.nbr = torch.empty((cap, max(self.n, 1)), dtype=torch.int32, device=dev)
        self.dvec = torch.empty((cap, max(self.n, 1), 4), dtype=torch.float32, device=dev)
        self.nnum = torch.empty(max(self.n, 1), dtype=torch.int32, device=dev)
        status = torch.zeros(1, dtype=torch.int32, device=dev)
        _chk(L.st_pairs(self.n, _p(self.pos), _p(self.start), _p(self.boxes), self.rc, cap, _p(self.nbr),
                        _p(self.dvec), _p(self.nnum), _p(status), _stream()), "st_pairs")
        if int(status.item()) != 0:
            raise RuntimeError(f"a neighbour row is longer than cap = {cap}")
        self.Q = torch.empty((max(self.n, 1), KB), dtype=torch.float32, device=dev)
        self.S = torch.empty((max(self.n, 1), NSB), dtype=torch.float32, device=dev)
        _chk(L.st_basis(0, self.n, self.n, cap, _p(self.nbr), _p(self.dvec), _p(self.nnum), self.rc, _p(self.Q),
                        _p(self.S), _stream()), "st_basis")
        # work buffers
        self.U = torch.empty(max(self.n, 1), dtype=torch.float32, device=dev)
        self.G = torch.empty((max(self.n, 1), GS), dtype=torch.float32, device=dev)
        self.dQ = torch.empty_like(self.Q)
        self.dS = torch.empty_like(self.S)
        self.scratch = torch.empty(max(int(L.st_grad_scratch(0, self.n)), 1), dtype=torch.float32, device=dev)
        self.E_ref = None if E is None else torch.as_tensor(np.asarray(E, dtype=np.float64), device=dev)
        self.F_ref = None if F is None else torch.as_tensor(np.asarray(F, dtype=np.float32).reshape(-1, 3), device=dev)
        self.natoms = torch.from_numpy(np.diff(self.start_h).astype(np.float64)).to(dev)

    def atoms(self, s0: int, s1: int):
        return int(self.start_h[s0]), int(self.start_h[s1])

    def descriptors(self, theta, q_scale):
        """Unscaled descriptors [n][12] of every atom (st_forward's optional output)."""
        import torch
        q = torch.empty((max(self.n, 1), NDES), dtype=torch.float32, device=self.pos.device)
        _chk(lib().st_forward(0, self.n, _p(theta), _p(q_scale), _p(self.Q), _p(self.S), _p(self.U), _p(self.G),
                              _p(q), _stream()), "st_forward")
        return q[:self.n]


def _student_ef():
    import torch

    class StudentEF(torch.autograd.Function):
        """(theta, q_scale, cells, s0, s1) -> (E [s1 - s0] float64, F [atoms of those cells][3])."""

        @staticmethod
        def forward(ctx, theta, q_scale, cells, s0, s1):
            L = lib()
            a0, a1 = cells.atoms(s0, s1)
            dev = cells.pos.device
            E = torch.empty(max(cells.n_cells, 1), dtype=torch.float64, device=dev)
            F = torch.empty((max(cells.n, 1), 3), dtype=torch.float32, device=dev)
            st = _stream()
            _chk(L.st_forward(a0, a1, _p(theta), _p(q_scale), _p(cells.Q), _p(cells.S), _p(cells.U), _p(cells.G),
                              None, st), "st_forward")
            _chk(L.st_energy(s0, s1, _p(cells.start), _p(cells.U), _p(E), st), "st_energy")
            _chk(L.st_force(a0, a1, cells.n, cells.cap, _p(cells.nbr), _p(cells.dvec), _p(cells.nnum), cells.rc,
                            _p(theta), _p(cells.G), _p(F), st), "st_force")
            ctx.save_for_backward(theta, q_scale)
            ctx.cells, ctx.rng = cells, (s0, s1, a0, a1)
            return E[s0:s1].clone(), F[a0:a1].clone()

        @staticmethod
        def backward(ctx, gE, gF):
            theta, q_scale = ctx.saved_tensors
            cells = ctx.cells
            s0, s1, a0, a1 = ctx.rng
            L = lib()
            dev = cells.pos.device
            gE_full = torch.zeros(max(cells.n_cells, 1), dtype=torch.float64, device=dev)
            v = torch.zeros((max(cells.n, 1), 3), dtype=torch.float32, device=dev)
            if gE is not None:
                gE_full[s0:s1] = gE.to(torch.float64)
            if gF is not None:
                v[a0:a1] = gF.to(torch.float32)
            st = _stream()
            _chk(L.st_jvp(a0, a1, cells.n, cells.cap, _p(cells.nbr), _p(cells.dvec), _p(cells.nnum), cells.rc, _p(v),
                          _p(cells.dQ), _p(cells.dS), st), "st_jvp")
            grad = torch.empty(NPAR, dtype=torch.float32, device=dev)
            _chk(L.st_grad(a0, a1, _p(theta), _p(q_scale), _p(cells.pos), _p(cells.Q), _p(cells.S), _p(cells.dQ),
                           _p(cells.dS), _p(gE_full), _p(cells.scratch), _p(grad), st), "st_grad")
            return grad, None, None, None, None

    return StudentEF


_EF = None


def student_ef(theta, q_scale, cells: CellSet, s0: int = 0, s1: int | None = None):
    """Energies of cells [s0, s1) and the forces on their atoms, differentiable in theta."""
    global _EF
    if _EF is None:
        _EF = _student_ef()
    return _EF.apply(theta, q_scale, cells, s0, cells.n_cells if s1 is None else s1)


def loss_fn(E, F, cells: CellSet, s0: int, s1: int, w_E: float = 1.0, w_F: float = 10.0):
    """w_E * mean_s ((E_s - E*_s) / n_s)^2 + w_F * mean over force components (F - F*)^2."""
    a0, a1 = cells.atoms(s0, s1)
    de = (E - cells.E_ref[s0:s1]) / cells.natoms[s0:s1]
    df = F - cells.F_ref[a0:a1]
    return w_E * (de * de).mean() + w_F * (df.double() * df.double()).mean()


def adam_step(theta, grad, m, v, lr: float, t: int, beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8):
    """In-place Adam update of theta (float32 device tensors) by the st_adam kernel."""
    _chk(lib().st_adam(theta.numel(), _p(theta), _p(grad), _p(m), _p(v), lr, beta1, beta2, eps, t, _stream()),
         "st_adam")
