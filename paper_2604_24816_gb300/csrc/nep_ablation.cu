// nep_ablation.cu -- paper-faithful kernel variants kept for ablation (nep_run_variant).
//
//   k_descriptor_tiled<S, NT>  the descriptor + network kernel with the channel tiling of the paper's
//                              Algorithm 1: the angular neighbours are walked once per tile of NT
//                              channels, so a thread holds NT x NLM accumulators s_nlm instead of
//                              NA x NLM, and the geometry (cutoff, basis, harmonics) is recomputed for
//                              every tile.  As in the paper, s_nlm (sum_fxyz) goes through a global
//                              array between the descriptor and the adjoint stage.
//   k_store_float3             float forces [3][n] (cell order) -> float64 [n][3] (caller's order), for
//                              the float-atomic scatter variant of the force kernel (nep_force.cu).
#include "nep_descriptor.cuh"

namespace nep {
namespace {

constexpr int TB = 128;
constexpr int T_DE = 8, T_DP = 4;

template <class S, int NT>
__global__ void __launch_bounds__(TB, 2)
k_descriptor_tiled(const __grid_constant__ Model<S> P, const Geom geom, const int n, const float4 *__restrict__ pos,
                   const int32_t *__restrict__ nbr, const RowExt X, float *__restrict__ G,
                   float *__restrict__ usite, long long *__restrict__ Ffix, long long *__restrict__ part,
                   int *__restrict__ status, float *__restrict__ sbuf) {
  __shared__ float4 shift[27];
  __shared__ uint32_t ring_e[T_DE * TB];
  __shared__ float4 ring_p[T_DP * TB];
  fill_shift_table(shift, geom);
  __syncthreads();
  const int i = blockIdx.x * TB + threadIdx.x;
  long long acc[5] = {0, 0, 0, 0, 0};
  if (i < n) {
    Ffix[i] = 0; Ffix[(size_t)n + i] = 0; Ffix[2 * (size_t)n + i] = 0;
    const float4 pi = pos[i];
    const RowSpan sp = full_row(X, i, skip_far(X));
    const int cnt = sp.c;
    // radial basis sums and LJ energy over the full row
    float QR[S::KR];
#pragma unroll
    for (int k = 0; k < S::KR; ++k) QR[k] = 0.f;
    float elj = 0.f;
    int nrad = 0, nang = 0, nact = 0;
    {
      NbrPipe<T_DE, T_DP, TB> pipe;
      pipe.start(ring_e, ring_p, nbr + i, (size_t)n, pos, sp);
      for (int k = 0; k < cnt; ++k) {
        uint32_t e;
        float4 pj;
        pipe.get(k, e, pj);
        const float4 o = shift[e >> J_BITS];
        const float dx = pj.x - pi.x + o.x, dy = pj.y - pi.y + o.y, dz = pj.z - pi.z + o.z;
        const float r2 = dx * dx + dy * dy + dz * dz;
        if (r2 >= P.rmax2) continue;
        ++nact;
        const float ir = rsqrtf(r2);
        const float r = r2 * ir;
        if (r2 < P.rcR2) {
          float f[S::KR];
          cheb_basis<S::KR>(r, P.inv_rcR, f);
#pragma unroll
          for (int k2 = 0; k2 < S::KR; ++k2) QR[k2] += f[k2];
          ++nrad;
        }
        if (P.lj_on != 0.f && r2 < P.lj_rc2) {
          float el, dl;
          lj_pair<S>(P, r2, r, ir, el, dl);
          elj = fmaf(0.5f, el, elj);
        }
        if (r2 < P.rcA2) ++nang;
      }
      pipe.finish();
    }
    float q[S::NDES];
#pragma unroll
    for (int a = 0; a < S::NR; ++a) {
      float t = 0.f;
#pragma unroll
      for (int k = 0; k < S::KR; ++k) t = fmaf(P.cR[a][k], QR[k], t);
      q[a] = t;
    }
    // angular channels, NT at a time; s_nlm to the global array [NA * NLM][n]
#pragma unroll 1
    for (int t0 = 0; t0 < S::NA; t0 += NT) {
      float s[NT][S::NLM];
#pragma unroll
      for (int a = 0; a < NT; ++a)
#pragma unroll
        for (int c = 0; c < S::NLM; ++c) s[a][c] = 0.f;
      NbrPipe<T_DE, T_DP, TB> pipe;
      pipe.start(ring_e, ring_p, nbr + i, (size_t)n, pos, sp);
      for (int k = 0; k < cnt; ++k) {
        uint32_t e;
        float4 pj;
        pipe.get(k, e, pj);
        const float4 o = shift[e >> J_BITS];
        const float dx = pj.x - pi.x + o.x, dy = pj.y - pi.y + o.y, dz = pj.z - pi.z + o.z;
        const float r2 = dx * dx + dy * dy + dz * dz;
        if (r2 >= P.rcA2) continue;
        const float ir = rsqrtf(r2);
        const float r = r2 * ir;
        float f[S::KA];
        cheb_basis<S::KA>(r, P.inv_rcA, f);
        float Y[S::NLM];
        harmonics<S::NLM>(dx * ir, dy * ir, dz * ir, Y);
#pragma unroll
        for (int a = 0; a < NT; ++a) {
          if (t0 + a >= S::NA) break;
          float g = 0.f;
#pragma unroll
          for (int b = 0; b < S::KA; ++b) g = fmaf(P.cA[t0 + a][b], f[b], g);
#pragma unroll
          for (int c = 0; c < S::NLM; ++c) s[a][c] = fmaf(g, Y[c], s[a][c]);
        }
      }
      pipe.finish();
#pragma unroll
      for (int a = 0; a < NT; ++a) {
        const int ch = t0 + a;
        if (ch >= S::NA) break;
#pragma unroll
        for (int l = 1; l <= S::LMAX; ++l) {
          float t = 0.f;
#pragma unroll
          for (int c = l * l - 1; c < (l + 1) * (l + 1) - 1; ++c) t = fmaf(s[a][c], s[a][c], t);
          q[S::NR + ch * S::LMAX + (l - 1)] = t;
        }
        if constexpr (S::FOURBODY) {
          const float i3 = 0.57735026918962576f, third = 1.f / 3.f;
          const float xy = s[a][3] * i3, yz = s[a][4] * i3, xz = s[a][6] * i3;
          const float xx = s[a][7] * i3 - s[a][5] * third, yy = -s[a][7] * i3 - s[a][5] * third;
          const float zz = 2.f * s[a][5] * third;
          q[S::NR + S::NA * S::LMAX + ch] =
              3.f * (xx * (yy * zz - yz * yz) - xy * (xy * zz - yz * xz) + xz * (xy * yz - yy * xz));
        }
#pragma unroll
        for (int c = 0; c < S::NLM; ++c) sbuf[(size_t)(ch * S::NLM + c) * n + i] = s[a][c];
      }
    }
    // network
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
    // adjoint rows from s_nlm read back per channel
    float *Gi = G + (size_t)i * S::GS;
#pragma unroll 1
    for (int a = 0; a < S::NA; ++a) {
      float sa[S::NLM], gl[S::NLM];
#pragma unroll
      for (int c = 0; c < S::NLM; ++c) sa[c] = sbuf[(size_t)(a * S::NLM + c) * n + i];
#pragma unroll
      for (int c = 0; c < S::NLM; ++c) gl[c] = 2.f * Fp[S::NR + a * S::LMAX + lm_l(c) - 1] * sa[c];
      if constexpr (S::FOURBODY) {
        const float f4 = Fp[S::NR + S::NA * S::LMAX + a];
        const float i3 = 0.57735026918962576f, third = 1.f / 3.f, s3 = 1.7320508075688772f;
        const float xy = sa[3] * i3, yz = sa[4] * i3, xz = sa[6] * i3;
        const float xx = sa[7] * i3 - sa[5] * third, yy = -sa[7] * i3 - sa[5] * third, zz = 2.f * sa[5] * third;
        const float Mxx = xx * xx + xy * xy + xz * xz, Myy = xy * xy + yy * yy + yz * yz;
        const float Mzz = xz * xz + yz * yz + zz * zz, Mxy = xx * xy + xy * yy + xz * yz;
        const float Myz = xy * xz + yy * yz + yz * zz, Mxz = xx * xz + xy * yz + xz * zz;
        gl[3] = fmaf(f4, 2.f * s3 * Mxy, gl[3]);
        gl[4] = fmaf(f4, 2.f * s3 * Myz, gl[4]);
        gl[5] = fmaf(f4, 2.f * Mzz - Mxx - Myy, gl[5]);
        gl[6] = fmaf(f4, 2.f * s3 * Mxz, gl[6]);
        gl[7] = fmaf(f4, s3 * (Mxx - Myy), gl[7]);
      }
#pragma unroll
      for (int c = 0; c < S::NLM; c += 4)
        *reinterpret_cast<float4 *>(Gi + a * S::NLM + c) = make_float4(gl[c], gl[c + 1], gl[c + 2], gl[c + 3]);
    }
    float tail[8];
    radial_tail<S>(P, Fp, tail);
    *reinterpret_cast<float4 *>(Gi + S::NA * S::NLM) = make_float4(tail[0], tail[1], tail[2], tail[3]);
    *reinterpret_cast<float4 *>(Gi + S::NA * S::NLM + 4) = make_float4(tail[4], tail[5], tail[6], tail[7]);
    const float ui = U + elj;
    usite[i] = ui;
    if (!isfinite(ui)) atomicOr(status, ST_NAN);
    acc[0] = to_fix32(ui);
    acc[1] = nrad;
    acc[2] = nang;
    acc[3] = cnt;
    acc[4] = nact;
  }
  block_sum_store<5>(acc, part);
}

__global__ void k_store_float3(int n, const int *__restrict__ id, const float *__restrict__ Ff,
                               double *__restrict__ out) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  const size_t o = 3 * (size_t)id[s];
  out[o] = Ff[s];
  out[o + 1] = Ff[(size_t)n + s];
  out[o + 2] = Ff[2 * (size_t)n + s];
}

}  // namespace

template <class S, int NT>
cudaError_t launch_descriptor_tiled(const Model<S> &P, const Geom &g, int n, const float4 *pos, const int32_t *nbr,
                                    const RowExt &X, float *G, float *usite, long long *Ffix, long long *part,
                                    int *status, float *sbuf, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  k_descriptor_tiled<S, NT><<<(n + TB - 1) / TB, TB, 0, st>>>(P, g, n, pos, nbr, X, G, usite, Ffix, part, status,
                                                               sbuf);
  return cudaGetLastError();
}

cudaError_t launch_store_float3(int n, const int *id, const float *Ff, double *out, cudaStream_t st) {
  if (n > 0) k_store_float3<<<(n + 255) / 256, 256, 0, st>>>(n, id, Ff, out);
  return cudaGetLastError();
}

int tiled_descriptor_blocks(int n) { return (n + TB - 1) / TB; }

template cudaError_t launch_descriptor_tiled<CuShape, 1>(const Model<CuShape> &, const Geom &, int, const float4 *,
                                                         const int32_t *, const RowExt &, float *, float *,
                                                         long long *, long long *, int *, float *, cudaStream_t);
template cudaError_t launch_descriptor_tiled<CuShape, 3>(const Model<CuShape> &, const Geom &, int, const float4 *,
                                                         const int32_t *, const RowExt &, float *, float *,
                                                         long long *, long long *, int *, float *, cudaStream_t);

}  // namespace nep
