"""Write the synthetic Cu NEP model file used by every test and benchmark.

The weights come from the seeded generator (nep_inputs.random_nep_weights).  The descriptor scale
q_scale[nu] = 1 / RMS_i(q_nu^i) is computed by the FP64 oracle on the seeded 4x4x4 fcc Cu cell
(256 atoms, 0.05 Angstrom Gaussian displacements), the only value in the file that needs descriptor
arithmetic; NEP implementations use a training-set scaler of this kind and the paper does not give one.

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


def make_model() -> dict:
    w = ni.random_nep_weights(WEIGHT_SEED)
    params = dict(ni.NEP_DIMS)
    params.update(rc_R=ni.RC_R, rc_A=ni.RC_A, lj_eps=ni.LJ["eps"], lj_sigma=ni.LJ["sigma"], lj_rc=ni.LJ["rc"],
                  mass_amu=ni.M_CU, skin=ni.SKIN, weight_seed=WEIGHT_SEED)
    for k in ("c_R", "c_A", "W0", "b0", "w1"):
        params[k] = np.asarray(w[k]).tolist()
    params["b1"] = float(w["b1"])
    params["q_scale"] = [1.0] * ni.N_DES
    wl = ni.workload("cu_4x4x4")
    q = oracle.descriptors(oracle.Model(params), wl.pos, wl.box)
    rms = np.sqrt(np.mean(q * q, axis=0))
    params["q_scale"] = (1.0 / rms).tolist()
    params["q_scale_source"] = "1/RMS of FP64 oracle descriptors on the seeded 4x4x4 fcc Cu cell (256 atoms)"
    return params


def main(argv):
    out = argv[1] if len(argv) > 1 else DEFAULT_OUT
    os.makedirs(os.path.dirname(out), exist_ok=True)
    with open(out, "w") as f:
        json.dump(make_model(), f, indent=1)
    print(out)


if __name__ == "__main__":
    main(sys.argv)
