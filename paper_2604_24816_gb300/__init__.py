"""GB300-native (sm_103a) NEP molecular dynamics: CUDA kernels behind a C ABI (include/nep_gb300.h).

    from paper_2604_24816_gb300 import NEP, load_model
    nep = NEP(load_model())
    nep.set_state(x, v, box)
    E, F, W = nep.compute()
    nep.step(1.0, 100)
"""
from .nep import NEP, NepError, load_model, lib, fp32_peak, DEFAULT_MODEL  # noqa: F401
