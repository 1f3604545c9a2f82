// nep_fallback.cu -- per-atom fallback from the student to the teacher model.
//
// The student's descriptor kernel flags every atom whose scaled descriptors leave the training range
// (Fallback in nep_descriptor.cuh), gives it a zero adjoint row and leaves only its LJ energy in the
// site energy.  For the flagged atoms these kernels then evaluate the teacher (plain float32):
//   k_fb_descriptor  descriptors, network, site energy U_i^teacher (added to usite and to the energy
//                    partial sums) and the teacher adjoint row of each flagged atom;
//   k_fb_force       dU_i^teacher/dr_ij for every neighbour j of each flagged atom i (its full row),
//                    scattered as F_i += D, F_j -= D with the same fixed-point integer atomics as the
//                    force kernel, and the virial -d_ij (x) D.
// So E = sum_i U_i^(model of i) and F = -grad E with each atom's own model (the LJ term, shared by both
// models, stays in the student's kernels).  Both kernels run on a fixed grid and loop over the flagged
// list, whose length they read on the device, so an MD step stays one CUDA graph.
#include <algorithm>

#include "nep_descriptor.cuh"

namespace nep {
namespace {

constexpr int FB_BLOCK = 128;
constexpr int FB_DE = 8, FB_DP = 4;

// Block sum of NV int64 values added atomically into dst[0..NV-1] (integer addition: the result does
// not depend on the order of the blocks).
template <int NV>
__device__ __forceinline__ void block_sum_atomic(long long (&v)[NV], long long *dst) {
  __shared__ long long red[32][NV];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < NV; ++k)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
  if (lane == 0)
#pragma unroll
    for (int k = 0; k < NV; ++k) red[warp][k] = v[k];
  __syncthreads();
  if (threadIdx.x == 0) {
    const int nw = blockDim.x >> 5;
    for (int k = 0; k < NV; ++k) {
      long long t = 0;
      for (int w = 0; w < nw; ++w) t += red[w][k];
      if (t != 0) atomicAdd(reinterpret_cast<unsigned long long *>(dst + k), (unsigned long long)t);
    }
  }
}

template <class S>
__global__ void __launch_bounds__(FB_BLOCK, 2)
k_fb_descriptor(const __grid_constant__ Model<S> P, const Geom geom, const int n, const float4 *__restrict__ pos,
                const int32_t *__restrict__ nbr, const int32_t *__restrict__ nnum, const int *__restrict__ list,
                const int *__restrict__ count, const int cap, float *__restrict__ Gt, float *__restrict__ usite,
                long long *__restrict__ part_d, long long *__restrict__ counters, int *__restrict__ status) {
  __shared__ float4 shift[27];
  __shared__ uint32_t ring_e[FB_DE * FB_BLOCK];
  __shared__ float4 ring_p[FB_DP * FB_BLOCK];
  fill_shift_table(shift, geom);
  __syncthreads();
  const int m = min(*count, cap);
  if (blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(reinterpret_cast<unsigned long long *>(counters + 9),
                                                     (unsigned long long)m);
  long long acc[1] = {0};
  for (int slot = blockIdx.x * FB_BLOCK + threadIdx.x; slot < m; slot += gridDim.x * FB_BLOCK) {
    const int i = list[slot];
    AtomSums<S> A;
    accumulate_atom<S, FB_DE, FB_DP, FB_BLOCK>(P, shift, i, n, pos, nbr, nnum[i], ring_e, ring_p, A);
    float q[S::NDES];
    FourBody<S> T;
    descriptors_of<S>(P, A, q, T);
    float qt[S::NDES], dq[S::NDES];
#pragma unroll
    for (int v = 0; v < S::NDES; ++v) { qt[v] = q[v] * P.qs[v]; dq[v] = 0.f; }
    float U = -P.b1;
#pragma unroll
    for (int mu = 0; mu < S::NNEU; ++mu) {
      float z = -P.b0[mu];
#pragma unroll
      for (int v = 0; v < S::NDES; ++v) z = fmaf(P.W0[mu][v], qt[v], z);
      const float h = tanhf(z);
      U = fmaf(P.w1[mu], h, U);
      const float t = P.w1[mu] * (1.f - h * h);
#pragma unroll
      for (int v = 0; v < S::NDES; ++v) dq[v] = fmaf(t, P.W0[mu][v], dq[v]);
    }
    float Fp[S::NDES];
#pragma unroll
    for (int v = 0; v < S::NDES; ++v) Fp[v] = dq[v] * P.qs[v];
    float *Gi = Gt + (size_t)slot * S::GS;
#pragma unroll
    for (int a = 0; a < S::NA; ++a) {
      float gl[S::NLM];
      adjoint_channel<S>(a, A, T, Fp, gl);
#pragma unroll
      for (int c = 0; c < S::NLM; c += 4)
        *reinterpret_cast<float4 *>(Gi + a * S::NLM + c) = make_float4(gl[c], gl[c + 1], gl[c + 2], gl[c + 3]);
    }
    float tail[8];
    radial_tail<S>(P, Fp, tail);
#pragma unroll
    for (int t = 0; t < 8; ++t) Gi[S::NA * S::NLM + t] = tail[t];
    usite[i] += U;                       // the student kernel left the LJ energy there
    if (!isfinite(U)) atomicOr(status, ST_NAN);
    acc[0] += to_fix32(U);
  }
  block_sum_atomic<1>(acc, part_d);      // energy slot of the descriptor partial sums
}

template <class S>
__global__ void __launch_bounds__(FB_BLOCK, 2)
k_fb_force(const __grid_constant__ Model<S> P, const Geom geom, const int n, const float4 *__restrict__ pos,
           const int32_t *__restrict__ nbr, const int32_t *__restrict__ nnum, const int *__restrict__ list,
           const int *__restrict__ count, const int cap, const float *__restrict__ Gt,
           unsigned long long *__restrict__ Ffix, long long *__restrict__ part_f, int *__restrict__ status) {
  __shared__ float4 shift[27];
  __shared__ uint32_t ring_e[FB_DE * FB_BLOCK];
  __shared__ float4 ring_p[FB_DP * FB_BLOCK];
  fill_shift_table(shift, geom);
  __syncthreads();
  const int m = min(*count, cap);
  long long acc[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  for (int slot = blockIdx.x * FB_BLOCK + threadIdx.x; slot < m; slot += gridDim.x * FB_BLOCK) {
    const int i = list[slot];
    const float4 pi = pos[i];
    const float *Gi = Gt + (size_t)slot * S::GS;
    float gi[S::NA][S::NLM];
#pragma unroll
    for (int a = 0; a < S::NA; ++a)
#pragma unroll
      for (int c = 0; c < S::NLM; c += 4) {
        const float4 t = *reinterpret_cast<const float4 *>(Gi + a * S::NLM + c);
        gi[a][c] = t.x; gi[a][c + 1] = t.y; gi[a][c + 2] = t.z; gi[a][c + 3] = t.w;
      }
    float fpi[S::KR];
#pragma unroll
    for (int k = 0; k < S::KR; ++k) fpi[k] = Gi[S::NA * S::NLM + k];
    float fx = 0.f, fy = 0.f, fz = 0.f;
    float wxx = 0.f, wxy = 0.f, wxz = 0.f, wyx = 0.f, wyy = 0.f, wyz = 0.f, wzx = 0.f, wzy = 0.f, wzz = 0.f;
    const int cnt = nnum[i];
    NbrPipe<FB_DE, FB_DP, FB_BLOCK> pipe;
    pipe.start(ring_e, ring_p, nbr + i, (size_t)n, pos, cnt);
    for (int k = 0; k < cnt; ++k) {
      uint32_t e;
      float4 pj;
      pipe.get(k, e, pj);
      const int j = (int)(e & J_MASK);
      const float4 o = shift[e >> J_BITS];
      const float dx = pj.x - pi.x + o.x, dy = pj.y - pi.y + o.y, dz = pj.z - pi.z + o.z;
      const float r2 = dx * dx + dy * dy + dz * dz;
      if (r2 >= P.rcR2) continue;
      const float ir = rsqrtf(r2);
      const float r = r2 * ir;
      float coef = 0.f, vx = 0.f, vy = 0.f, vz = 0.f;
      {
        float f[S::KR], df[S::KR];
        cheb_basis_d<S::KR>(r, P.inv_rcR, f, df);
        float c = 0.f;
#pragma unroll
        for (int k = 0; k < S::KR; ++k) c = fmaf(fpi[k], df[k], c);
        coef = c * ir;
      }
      if (r2 < P.rcA2) {
        float f[S::KA], df[S::KA];
        cheb_basis_d<S::KA>(r, P.inv_rcA, f, df);
        float g[S::NA], dg[S::NA];
#pragma unroll
        for (int a = 0; a < S::NA; ++a) {
          float t = 0.f, dt = 0.f;
#pragma unroll
          for (int b = 0; b < S::KA; ++b) { t = fmaf(P.cA[a][b], f[b], t); dt = fmaf(P.cA[a][b], df[b], dt); }
          g[a] = t; dg[a] = dt;
        }
        const float ux = dx * ir, uy = dy * ir, uz = dz * ir;
        float Y[S::NLM];
        harmonics<S::NLM>(ux, uy, uz, Y);
        float along = 0.f, bx = 0.f, by = 0.f, bz = 0.f;
#pragma unroll
        for (int c = 0; c < S::NLM; ++c) {
          float av = 0.f, bv = 0.f;
#pragma unroll
          for (int a = 0; a < S::NA; ++a) { av = fmaf(gi[a][c], dg[a], av); bv = fmaf(gi[a][c], g[a], bv); }
          along = fmaf(av - (float)lm_l(c) * ir * bv, Y[c], along);
          harmonic_grad_acc(c, ux, uy, uz, bv, bx, by, bz);
        }
        coef = fmaf(along, ir, coef);
        vx = bx * ir; vy = by * ir; vz = bz * ir;
      }
      // D = dU_i/dd_ij: F_i += D, F_j -= D
      const float Dx = fmaf(coef, dx, vx), Dy = fmaf(coef, dy, vy), Dz = fmaf(coef, dz, vz);
      fx += Dx; fy += Dy; fz += Dz;
      red_add(Ffix + j, -to_fix32(Dx));
      red_add(Ffix + (size_t)n + j, -to_fix32(Dy));
      red_add(Ffix + 2 * (size_t)n + j, -to_fix32(Dz));
      wxx = fmaf(dx, Dx, wxx); wxy = fmaf(dx, Dy, wxy); wxz = fmaf(dx, Dz, wxz);
      wyx = fmaf(dy, Dx, wyx); wyy = fmaf(dy, Dy, wyy); wyz = fmaf(dy, Dz, wyz);
      wzx = fmaf(dz, Dx, wzx); wzy = fmaf(dz, Dy, wzy); wzz = fmaf(dz, Dz, wzz);
    }
    pipe.finish();
    red_add(Ffix + i, to_fix32(fx));
    red_add(Ffix + (size_t)n + i, to_fix32(fy));
    red_add(Ffix + 2 * (size_t)n + i, to_fix32(fz));
    if (!(isfinite(fx) && isfinite(fy) && isfinite(fz))) atomicOr(status, ST_NAN);
    acc[0] -= to_fix32(wxx); acc[1] -= to_fix32(wxy); acc[2] -= to_fix32(wxz);
    acc[3] -= to_fix32(wyx); acc[4] -= to_fix32(wyy); acc[5] -= to_fix32(wyz);
    acc[6] -= to_fix32(wzx); acc[7] -= to_fix32(wzy); acc[8] -= to_fix32(wzz);
  }
  block_sum_atomic<9>(acc, part_f);      // virial slots of the force partial sums
}

// flags[id[i]] = 1 for every flagged atom i (flags zeroed by the caller).
__global__ void k_fb_flags(const int *__restrict__ list, const int *__restrict__ count, int cap,
                           const int *__restrict__ id, int *__restrict__ flags) {
  const int m = min(*count, cap);
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < m; s += gridDim.x * blockDim.x) flags[id[list[s]]] = 1;
}

int fb_grid(int cap) { return std::max(1, std::min((cap + FB_BLOCK - 1) / FB_BLOCK, 152 * 8)); }

}  // namespace

template <class S>
cudaError_t launch_fallback_descriptor(const Model<S> &P, const Geom &g, int n, const float4 *pos, const int32_t *nbr,
                                       const int32_t *nnum, const int *list, const int *count, int cap, float *Gt,
                                       float *usite, long long *part_d, long long *counters, int *status,
                                       cudaStream_t st) {
  if (n <= 0 || cap <= 0) return cudaSuccess;
  k_fb_descriptor<S><<<fb_grid(cap), FB_BLOCK, 0, st>>>(P, g, n, pos, nbr, nnum, list, count, cap, Gt, usite, part_d,
                                                        counters, status);
  return cudaGetLastError();
}

template <class S>
cudaError_t launch_fallback_force(const Model<S> &P, const Geom &g, int n, const float4 *pos, const int32_t *nbr,
                                  const int32_t *nnum, const int *list, const int *count, int cap, const float *Gt,
                                  long long *Ffix, long long *part_f, int *status, cudaStream_t st) {
  if (n <= 0 || cap <= 0) return cudaSuccess;
  k_fb_force<S><<<fb_grid(cap), FB_BLOCK, 0, st>>>(P, g, n, pos, nbr, nnum, list, count, cap, Gt,
                                                   reinterpret_cast<unsigned long long *>(Ffix), part_f, status);
  return cudaGetLastError();
}

cudaError_t launch_fallback_flags(const int *list, const int *count, int cap, const int *id, int *flags,
                                  cudaStream_t st) {
  if (cap <= 0) return cudaSuccess;
  k_fb_flags<<<fb_grid(cap), FB_BLOCK, 0, st>>>(list, count, cap, id, flags);
  return cudaGetLastError();
}

template cudaError_t launch_fallback_descriptor<CuShape>(const Model<CuShape> &, const Geom &, int, const float4 *,
                                                         const int32_t *, const int32_t *, const int *, const int *,
                                                         int, float *, float *, long long *, long long *, int *,
                                                         cudaStream_t);
template cudaError_t launch_fallback_force<CuShape>(const Model<CuShape> &, const Geom &, int, const float4 *,
                                                    const int32_t *, const int32_t *, const int *, const int *, int,
                                                    const float *, long long *, long long *, int *, cudaStream_t);

}  // namespace nep
