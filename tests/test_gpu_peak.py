"""nep_fp32_peak, the FP32 throughput microbenchmark that gives the roofline's denominator: it runs,
reads the SM count from the device, and counts FMAs per SM cycle within what an SM can issue (128 FP32
lanes per cycle on this GPU family; a count far above would mean the timed kernel is not doing the
work); bad arguments are refused before any launch."""
import ctypes as C

import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2604_24816_gb300 import build
    build.build()
    import paper_2604_24816_gb300 as p
    p.lib()
    return p


@pytest.mark.parametrize("form", [False, True, "half2"])
def test_fp32_peak_forms(pkg, form):
    import torch
    r = pkg.fp32_peak(form, 1.0, 3)
    assert r["sm_count"] == torch.cuda.get_device_properties(0).multi_processor_count
    assert 0.0 < r["median_tflops"] <= r["best_tflops"]
    # FMAs per SM cycle: positive and at most the SM's 128 lanes (+1 % for the clock64 span's edges)
    assert 16.0 < r["fma_per_clock_sm"] <= 129.3
    # TFLOP/s = 2 FMA FLOP x lanes per cycle x SMs x clock: the implied clock must be a plausible SM clock
    mhz = r["median_tflops"] * 1e6 / (2 * r["sm_count"] * r["fma_per_clock_sm"])
    assert 300.0 < mhz < 3000.0


def test_fp32_peak_rejects_bad_arguments(pkg):
    L = pkg.lib()
    d = C.c_double(0)
    i = C.c_int(0)
    for packed, ms, reps in ((3, 1.0, 1), (-1, 1.0, 1), (1, 0.0, 1), (1, 1001.0, 1), (1, 1.0, 0), (1, 1.0, 10001)):
        st = L.nep_fp32_peak(packed, ms, reps, None, C.byref(d), C.byref(d), C.byref(d), C.byref(i))
        assert L.nep_status_string(st) == b"NEP_ERR_ARG"
