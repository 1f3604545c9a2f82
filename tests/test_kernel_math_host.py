"""The kernels' harmonic helpers (csrc/nep_common.cuh), compiled by nvcc for the host and run on the CPU.

The fused kernels keep the angular sums and the adjoint row over the polynomials Ph_lm without their
constant factors and apply hnorm(lm) once per atom (s' = s / hnorm, G' = hnorm G), so that each angular
pair forms G' Ph and G' grad Ph where the method has G Yh and G grad Yh.  That is exact only if
hnorm(lm) Ph_lm = Yh_lm and hnorm(lm) grad Ph_lm = grad Yh_lm for every component: checked here against
the normalised helpers the separate kernels use (harmonics, harmonic_grad) on seeded points, on and off
the unit sphere (the gradients treat x, y, z as free variables), together with the per-component form
harmonic_p and the zero pattern harmonic_grad_mask.  The normalised helpers themselves are pinned
through the GPU parity tests against the FP64 oracle (descriptors, forces).
"""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2604_24816_gb300", "csrc")

PROGRAM = r"""
#include "nep_common.cuh"
#include <cmath>
#include <cstdio>
#include <cstdint>
using namespace nep;

static uint64_t state = 0x9E3779B97F4A7C15ull;
static double uniform() {                      // splitmix64 -> [0, 1)
  uint64_t z = (state += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return (double)((z ^ (z >> 31)) >> 11) * 0x1.0p-53;
}

int main() {
  double ey = 0, eg = 0, ep = 0, e8 = 0;
  int mask_bad = 0;
  for (int t = 0; t < 20000; ++t) {
    double v[3], n2 = 0;
    for (int d = 0; d < 3; ++d) { v[d] = 3.0 * uniform() - 1.5; n2 += v[d] * v[d]; }
    const double s = (t & 1) ? 1.0 / sqrt(n2) : 1.0;   // odd points on the unit sphere
    const float x = (float)(v[0] * s), y = (float)(v[1] * s), z = (float)(v[2] * s);
    const double scale = fmax(1.0, pow(sqrt((double)x * x + (double)y * y + (double)z * z), 4));
    float Y[24], P[24], Y8[8], P8[8];
    harmonics<24>(x, y, z, Y);
    harmonics_p<24>(x, y, z, P);
    harmonics<8>(x, y, z, Y8);
    harmonics_p<8>(x, y, z, P8);
    for (int lm = 0; lm < 24; ++lm) {
      ey = fmax(ey, fabs(Y[lm] - (double)hnorm(lm) * P[lm]) / scale);
      ep = fmax(ep, fabs(P[lm] - harmonic_p(lm, x, y, z)) / scale);
      if (lm < 8) e8 = fmax(e8, fabs(Y8[lm] - (double)hnorm(lm) * P8[lm]) / scale);
      float a[3], b[3];
      harmonic_grad(lm, x, y, z, a);
      harmonic_grad_p(lm, x, y, z, b);
      const int m = harmonic_grad_mask(lm);
      for (int d = 0; d < 3; ++d) {
        eg = fmax(eg, fabs(a[d] - (double)hnorm(lm) * b[d]) / scale);
        if (!((m >> d) & 1) && (a[d] != 0.f || b[d] != 0.f)) ++mask_bad;
      }
    }
  }
  printf("%.6e %.6e %.6e %.6e %d\n", ey, eg, ep, e8, mask_bad);
  return 0;
}
"""


def test_unnormalised_harmonics_reproduce_the_normalised_ones(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    src = tmp_path / "harmonics_check.cu"
    src.write_text(PROGRAM)
    exe = tmp_path / "harmonics_check"
    r = subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-std=c++17", "--expt-relaxed-constexpr",
                        "-I", os.path.join(ROOT, "include"), "-I", CSRC, "-o", str(exe), str(src)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-3000:]
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()
    ey, eg, ep, e8, mask_bad = float(out[0]), float(out[1]), float(out[2]), float(out[3]), int(out[4])
    # float32 evaluation of degree <= 4 polynomials with |coefficients| <= 35 (times |r|^4 off the
    # sphere): a few units of 2^-24 relative to the largest term
    assert ey < 2e-5 and e8 < 2e-5, (ey, e8)
    assert eg < 5e-5, eg
    assert ep == 0.0, ep              # harmonic_p is the same arithmetic as harmonics_p, component by component
    assert mask_bad == 0
