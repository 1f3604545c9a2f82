"""Distil the student NEP from the teacher: generate data with teacher NEP-MD on the GPU, train the
student with the hand-written training kernels, evaluate it on held-out trajectories.

    python -m paper_2604_24816_gb300.distill [--snapshots 2000] [--steps 20000] [--out FILE] [--report FILE]

Data: periodic fcc Cu cells of 256-864 atoms (4-6 conventional cells per edge), each trajectory with a
random temperature in [300, 1500] K, a random diagonal strain within +-3 % and 1-4 vacancies, run
with the teacher (plain float32 NEP + LJ, velocity Verlet, 1 fs); snapshots are taken every `stride`
steps after an equilibration run.  Labels are the teacher's NEP-only energies and forces (the LJ term
is shared by teacher and student and is not learned).  The last 10 % of the trajectories are held out.

Training: Adam on the 289 student parameters, loss = mean per-atom energy error squared + 10 x mean
force-component error squared, mini-batches of whole cells.  The descriptor scale q_scale is the
range scaler 1 / (max - min) of the initial student's descriptors over the training atoms (then
fixed).  The output model file also stores the range of every scaled descriptor over the training
atoms (q_lo, q_hi), which the fallback to the teacher uses.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import sys
import time

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
_ROOT = os.path.dirname(_PKG)
if _ROOT not in sys.path:
    sys.path.insert(0, _ROOT)

import nep_inputs as ni  # noqa: E402

from . import nep as _nep  # noqa: E402
from . import student as st  # noqa: E402

DEFAULT_OUT = os.path.join(_PKG, "params", "cu_student_trained.json")
SIZES = [(4, 4, 4), (4, 4, 5), (4, 5, 5), (5, 5, 5), (4, 5, 6), (5, 5, 6), (5, 6, 6), (6, 6, 6)]


def trajectory_spec(t: int, seed: int):
    rng = np.random.default_rng(seed * 1000 + t)
    cells = SIZES[int(rng.integers(len(SIZES)))]
    T = float(rng.uniform(300.0, 1500.0))
    strain = tuple(float(x) for x in rng.uniform(-0.03, 0.03, size=3))
    vac = int(rng.integers(1, 5))
    return dict(cells=cells, T=T, strain=strain, vacancies=vac, seed=seed * 1000 + t)


def generate(teacher: dict, n_traj: int, per_traj: int, stride: int, equil: int, seed: int, log=print):
    """Teacher NEP-MD snapshots and their NEP-only labels: list of (pos, box, E, F, spec)."""
    out = []
    md = None
    lab = _nep.NEP(teacher, lj=False)
    for t in range(n_traj):
        sp = trajectory_spec(t, seed)
        sigma = 0.05 * math.sqrt(sp["T"] / 300.0)
        pos, box = ni.student_cell(sp["seed"], sp["cells"], sigma, sp["strain"], sp["vacancies"])
        rng = np.random.default_rng(sp["seed"] + 7)
        vel = ni.maxwell_boltzmann(pos.shape[0], sp["T"], ni.M_CU, rng)
        if md is not None:
            md.close()
        md = _nep.NEP(teacher, rebuild_every=10)
        md.set_state(pos, vel, box)
        # equilibration with velocity rescaling to the target temperature every 20 steps (the
        # displaced start holds potential energy that would otherwise heat the cell), then NVE
        for _ in range(max(1, equil // 20)):
            md.step(1.0, 20)
            x, v = md.get_state()
            T_now = md.thermo()["temperature"]
            md.set_state(x, v * math.sqrt(sp["T"] / max(T_now, 1.0)), box)
        for k in range(per_traj):
            md.step(1.0, stride)
            x, v = md.get_state()
            lab.set_state(x, None, box)
            E, F, W = lab.compute()
            out.append((np.mod(x, box), np.asarray(box, dtype=np.float64), float(E), F.copy(), sp))
        if log and (t + 1) % max(1, n_traj // 10) == 0:
            th = md.thermo()
            log(f"  trajectory {t + 1}/{n_traj}: {pos.shape[0]} atoms, T0 {sp['T']:.0f} K, "
                f"T now {th['temperature']:.0f} K")
    if md is not None:
        md.close()
    lab.close()
    return out


def cellset(snaps):
    return st.CellSet([(p, b) for p, b, *_ in snaps], E=[e for _, _, e, _, _ in snaps],
                      F=np.concatenate([f for *_, f, _ in snaps]))


def evaluate(theta, qs, cs):
    """Force RMSE (eV/A), energy MAE (eV/atom) and energy RMSE (eV/atom) of the student vs the labels."""
    import torch
    with torch.no_grad():
        E, F = st.student_ef(theta, qs, cs)
        de = ((E - cs.E_ref) / cs.natoms).cpu().numpy()
        df = (F - cs.F_ref).double().cpu().numpy()
        fr = cs.F_ref.double().cpu().numpy()
    return dict(force_rmse=float(np.sqrt(np.mean(df ** 2))), force_max=float(np.abs(df).max()),
                label_force_rms=float(np.sqrt(np.mean(fr ** 2))), energy_mae_per_atom=float(np.mean(np.abs(de))),
                energy_rmse_per_atom=float(np.sqrt(np.mean(de ** 2))))


def train(cs_train, cs_val, init: dict, steps: int, batch: int, lr0: float, lr1: float, seed: int, log=print):
    import torch
    theta = torch.tensor(st.pack(init), device="cuda", requires_grad=True)
    # range scaler from the initial student's descriptors over the training atoms
    ones = torch.ones(st.NDES, device="cuda")
    q0 = cs_train.descriptors(theta.detach(), ones)
    qs = (1.0 / (q0.max(dim=0).values - q0.min(dim=0).values).clamp_min(1e-12)).float().contiguous()
    m = torch.zeros_like(theta)
    v = torch.zeros_like(theta)
    rng = np.random.default_rng(seed)
    n_batches = max(1, cs_train.n_cells // batch)
    order = rng.permutation(n_batches)
    hist = []
    t0 = time.perf_counter()
    for step in range(1, steps + 1):
        lr = lr0 * (lr1 / lr0) ** ((step - 1) / max(1, steps - 1))
        b = int(order[(step - 1) % n_batches])
        if (step - 1) % n_batches == n_batches - 1:
            order = rng.permutation(n_batches)
        s0, s1 = b * batch, min(cs_train.n_cells, (b + 1) * batch)
        theta.grad = None
        E, F = st.student_ef(theta, qs, cs_train, s0, s1)
        loss = st.loss_fn(E, F, cs_train, s0, s1)
        loss.backward()
        with torch.no_grad():
            st.adam_step(theta.data, theta.grad, m, v, lr, step)
        if step % max(1, steps // 20) == 0 or step == steps:
            ev = evaluate(theta.detach(), qs, cs_val)
            hist.append(dict(step=step, lr=lr, loss=float(loss.item()), **ev))
            if log:
                log(f"  step {step}: loss {loss.item():.3e}, held-out force RMSE {ev['force_rmse'] * 1e3:.2f} meV/A, "
                    f"energy MAE {ev['energy_mae_per_atom'] * 1e3:.3f} meV/atom")
    torch.cuda.synchronize()
    return theta.detach(), qs, hist, time.perf_counter() - t0


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--snapshots", type=int, default=2000)
    ap.add_argument("--per-traj", type=int, default=20)
    ap.add_argument("--stride", type=int, default=25)
    ap.add_argument("--equil", type=int, default=200)
    ap.add_argument("--steps", type=int, default=20000)
    ap.add_argument("--batch", type=int, default=40)
    ap.add_argument("--lr0", type=float, default=5e-3)
    ap.add_argument("--lr1", type=float, default=5e-5)
    ap.add_argument("--seed", type=int, default=4242)
    ap.add_argument("--init-seed", type=int, default=7331)
    ap.add_argument("--out", default=DEFAULT_OUT)
    ap.add_argument("--report", default=None)
    ap.add_argument("--teacher-low-l", action="store_true",
                    help="diagnostic: zero the teacher's weights on its l = 3, 4 and 4-body descriptors, i.e. a "
                         "teacher built only from descriptor families the student shape has")
    args = ap.parse_args(argv)
    import torch
    assert torch.cuda.is_available(), "distillation runs on the GPU"
    from . import build
    build.build()
    teacher = _nep.load_model()
    if args.teacher_low_l:
        teacher = restrict_teacher(teacher)
    n_traj = max(2, args.snapshots // args.per_traj)
    t0 = time.perf_counter()
    print(f"generating {n_traj} teacher trajectories x {args.per_traj} snapshots", flush=True)
    snaps = generate(teacher, n_traj, args.per_traj, args.stride, args.equil, args.seed)
    t_gen = time.perf_counter() - t0
    n_val_traj = max(1, n_traj // 10)
    split = (n_traj - n_val_traj) * args.per_traj
    train_snaps, val_snaps = snaps[:split], snaps[split:]
    # shuffle training cells so that mini-batches mix trajectories (seeded)
    perm = np.random.default_rng(args.seed + 1).permutation(len(train_snaps))
    train_snaps = [train_snaps[i] for i in perm]
    cs_train, cs_val = cellset(train_snaps), cellset(val_snaps)
    print(f"  {len(train_snaps)} training cells ({cs_train.n} atoms), {len(val_snaps)} held-out cells "
          f"({cs_val.n} atoms), {t_gen:.1f} s", flush=True)
    init = _init_student(teacher, args.init_seed)
    theta, qs, hist, t_train = train(cs_train, cs_val, init, args.steps, args.batch, args.lr0, args.lr1, args.seed)
    ev_val = evaluate(theta, qs, cs_val)
    ev_train = evaluate(theta, qs, cs_train)
    # scaled-descriptor range over the training atoms (for the teacher fallback)
    qt = cs_train.descriptors(theta, qs) * qs
    q_lo = qt.min(dim=0).values.cpu().numpy().astype(np.float64)
    q_hi = qt.max(dim=0).values.cpu().numpy().astype(np.float64)
    model = st.unpack(theta.cpu().numpy(), init)
    model["q_scale"] = qs.cpu().numpy().astype(np.float64).tolist()
    model["q_lo"], model["q_hi"] = q_lo.tolist(), q_hi.tolist()
    model["training"] = dict(teacher="restricted to l <= 2, no 4-body (diagnostic)" if args.teacher_low_l
                             else "cu_nep4_synth", snapshots=len(snaps), trajectories=n_traj, train_cells=len(train_snaps),
                             heldout_cells=len(val_snaps), steps=args.steps, batch_cells=args.batch, lr0=args.lr0,
                             lr1=args.lr1, seed=args.seed, init_seed=args.init_seed, loss="E-MSE/atom + 10 F-MSE",
                             heldout=ev_val, train=ev_train, seconds_generate=t_gen, seconds_train=t_train)
    model.pop("weight_seed", None)
    os.makedirs(os.path.dirname(os.path.abspath(args.out)), exist_ok=True)
    with open(args.out, "w") as f:
        json.dump(model, f, indent=1)
    rep = dict(heldout=ev_val, train=ev_train, history=hist, seconds_generate=t_gen, seconds_train=t_train,
               out=args.out)
    if args.report:
        with open(args.report, "w") as f:
            json.dump(rep, f, indent=1)
    print(json.dumps(dict(heldout=ev_val, train=ev_train, seconds_train=t_train)), flush=True)


def restrict_teacher(teacher: dict) -> dict:
    """The teacher with zero weights on its l = 3, 4 (3-body) and 4-body descriptors."""
    t = dict(teacher)
    W0 = np.array(teacher["W0"], dtype=np.float64)
    nR, nA, L = teacher["n_max_R"] + 1, teacher["n_max_A"] + 1, teacher["l_max_3b"]
    for n in range(nA):
        for l in range(3, L + 1):
            W0[:, nR + n * L + l - 1] = 0.0
        W0[:, nR + nA * L + n] = 0.0
    t["W0"] = W0.tolist()
    return t


def _init_student(teacher: dict, seed: int) -> dict:
    """Seeded initial student: the teacher's cutoffs, LJ term, mass and skin with the student shape."""
    w = ni.random_nep_weights(seed, ni.STUDENT_DIMS)
    m = dict(ni.STUDENT_DIMS)
    for k in ("rc_R", "rc_A", "lj_eps", "lj_sigma", "lj_rc", "mass_amu", "skin"):
        m[k] = teacher[k]
    for k in ("c_R", "c_A", "W0", "b0", "w1"):
        m[k] = np.asarray(w[k]).tolist()
    m["b1"] = float(w["b1"])
    m["q_scale"] = [1.0] * 12
    return m


if __name__ == "__main__":
    main()
