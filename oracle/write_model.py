"""Write the synthetic Cu NEP model file used by every test and benchmark.

The weights come from the seeded generator (nep_inputs.random_nep_weights).  The descriptor scale
q_scale[nu] = 1 / (max_i q_nu^i - min_i q_nu^i) is a range scaler over a small reference set -- three
seeded 4x4x4 fcc Cu cells (768 atoms) with 0.05 Angstrom Gaussian displacements, the distribution of
the 256-atom parity workload -- computed by the FP64 oracle.  It is the only value in the file
that needs descriptor arithmetic; the paper gives no scaler, and NEP implementations use a
training-set range scaler of this kind.

Usage:  python -m oracle.write_model [output.json]
"""
from __future__ import annotations

import json
import os
import sys

import numpy as np

_ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if _ROOT not in sys.path:
    sys.path.insert(0, _ROOT)

import nep_inputs as ni  # noqa: E402
import oracle  # noqa: E402

DEFAULT_OUT = os.path.join(_ROOT, "paper_2604_24816_gb300", "params", "cu_nep4_synth.json")
WEIGHT_SEED = 2604
SCALER_SIGMAS = (0.05, 0.05, 0.05)


def make_model(dims: dict = ni.NEP_DIMS, seed: int = WEIGHT_SEED) -> dict:
    """Seeded model of shape `dims` (the teacher by default; ni.STUDENT_DIMS gives a seeded, untrained
    student used by the parity tests of the student-shaped kernels)."""
    w = ni.random_nep_weights(seed, dims)
    params = dict(dims)
    params.update(rc_R=ni.RC_R, rc_A=ni.RC_A, lj_eps=ni.LJ["eps"], lj_sigma=ni.LJ["sigma"], lj_rc=ni.LJ["rc"],
                  mass_amu=ni.M_CU, skin=ni.SKIN, weight_seed=seed)
    for k in ("c_R", "c_A", "W0", "b0", "w1"):
        params[k] = np.asarray(w[k]).tolist()
    params["b1"] = float(w["b1"])
    params["q_scale"] = [1.0] * np.asarray(w["W0"]).shape[1]
    qs = []
    for k, sigma in enumerate(SCALER_SIGMAS):
        wl = ni.fcc_cu_workload(4, 300.0, sigma, seed=100 + k)
        qs.append(oracle.descriptors(oracle.Model(params), wl.pos, wl.box))
    q = np.concatenate(qs, axis=0)
    params["q_scale"] = (1.0 / (q.max(axis=0) - q.min(axis=0))).tolist()
    params["q_scale_source"] = ("1/(max-min) of FP64 oracle descriptors over seeded 4x4x4 fcc Cu cells with "
                                "Gaussian displacements " + ", ".join(f"{s:g}" for s in SCALER_SIGMAS) + " A")
    return params


def main(argv):
    out = argv[1] if len(argv) > 1 else DEFAULT_OUT
    os.makedirs(os.path.dirname(out), exist_ok=True)
    with open(out, "w") as f:
        json.dump(make_model(), f, indent=1)
    print(out)


if __name__ == "__main__":
    main(sys.argv)
