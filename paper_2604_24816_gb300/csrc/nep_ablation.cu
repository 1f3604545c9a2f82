// nep_ablation.cu -- paper-faithful kernel variants kept for ablation (nep_run_variant).
//
//   k_descriptor_tiled<S, NT>  the descriptor + network kernel with the channel tiling of the paper's
//                              Algorithm 1: the angular neighbours are walked once per tile of NT
//                              channels, so a thread holds NT x NLM accumulators s_nlm instead of
//                              NA x NLM, and the geometry (cutoff, basis, harmonics) is recomputed for
//                              every tile.  As in the paper, s_nlm (sum_fxyz) goes through a global
//                              array between the descriptor and the adjoint stage.
//   k_force_cpb<S, CPB>        the full-row force kernel in the paper's thread-per-neighbour form with
//                              its adaptive centres-per-block scheduling (Section V.B, Optimization 3):
//                              a warp takes CPB centre atoms at a time, its 32 lanes split into CPB
//                              groups (32 / 16+16 / 11+11+10); a group's lanes stride over the centre's
//                              row for the radial and LJ pair forces, collecting its angular pairs in
//                              shared memory, then over those angular pairs (the three-body backward)
//                              with the centre's adjoint row in shared memory.
//   k_angular_counts           angular pairs per atom (r < rc_A), for the 90th-percentile rule that
//                              chooses CPB.
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

// The angular part of one pair's force with the centre's adjoint row in shared memory (Gs: [NA][NLM]
// then the radial tail): the arithmetic of the production kernels' angular_pair on a row read with
// 16-byte broadcast loads instead of tensor memory.
template <class S>
__device__ __forceinline__ void angular_pair_smem(const Model<S> &P, const float *Gs, float r, float ir, float dx,
                                                  float dy, float dz, float2 &al, float2 (&gv)[3]) {
  const float ux = dx * ir, uy = dy * ir, uz = dz * ir;
  float f[S::KA], df[S::KA];
  cheb_basis_d<S::KA>(r, P.inv_rcA, f, df);
  float g[S::NA], dg[S::NA];
#pragma unroll
  for (int a = 0; a < S::NA; ++a) dot_pairs2<S::KA>(P.cA[a], f, df, g[a], dg[a]);
  float Y[S::NLM];
  harmonics<S::NLM>(ux, uy, uz, Y);
  const float2 air2 = bc2(ir);
  al = bc2(0.f);
  gv[0] = gv[1] = gv[2] = bc2(0.f);
#pragma unroll
  for (int k = 0; k < S::NLM / 4; ++k) {
    const int lm0 = 4 * k;
    float2 av01 = bc2(0.f), av23 = bc2(0.f), bv01 = bc2(0.f), bv23 = bc2(0.f);
#pragma unroll
    for (int a = 0; a < S::NA; ++a) {
      const float4 h = *reinterpret_cast<const float4 *>(Gs + a * S::NLM + lm0);
      const float2 h01 = pr(h.x, h.y), h23 = pr(h.z, h.w);
      const float2 dg2 = bc2(dg[a]), g2 = bc2(g[a]);
      av01 = fma2(h01, dg2, av01);
      av23 = fma2(h23, dg2, av23);
      bv01 = fma2(h01, g2, bv01);
      bv23 = fma2(h23, g2, bv23);
    }
    const float2 nl01 = mul2(pr(-(float)lm_l(lm0), -(float)lm_l(lm0 + 1)), air2);
    const float2 nl23 = mul2(pr(-(float)lm_l(lm0 + 2), -(float)lm_l(lm0 + 3)), air2);
    al = fma2(fma2(nl01, bv01, av01), pr(Y[lm0], Y[lm0 + 1]), al);
    al = fma2(fma2(nl23, bv23, av23), pr(Y[lm0 + 2], Y[lm0 + 3]), al);
    harmonic_grad_acc2(lm0, ux, uy, uz, bv01, gv);
    harmonic_grad_acc2(lm0 + 2, ux, uy, uz, bv23, gv);
  }
}

constexpr int CPB_ANG_CAP = 64;   // angular pairs per centre held in shared memory

template <int CPB>
__device__ __forceinline__ void cpb_group(int lane, int &c, int &s, int &gsz) {
  // CPB groups of consecutive lanes: 32; 16 + 16; 11 + 11 + 10
  constexpr int base = 32 / CPB, extra = 32 % CPB;
  c = 0;
  int start = 0, size = base + (extra > 0 ? 1 : 0);
#pragma unroll
  for (int g = 1; g < CPB; ++g) {
    if (lane >= start + size) { start += size; size = base + (g < extra ? 1 : 0); c = g; }
  }
  s = lane - start;
  gsz = size;
}

template <class S, int CPB>
__global__ void __launch_bounds__(TB, 2)
k_force_cpb(const __grid_constant__ Model<S> P, const Geom geom, const int n, const float4 *__restrict__ pos,
            const int32_t *__restrict__ nbr, const RowExt X, const float *__restrict__ G,
            unsigned long long *__restrict__ Ffix, long long *__restrict__ part, int *__restrict__ status) {
  static_assert(CPB >= 1 && CPB <= 3 && S::GS % 4 == 0, "1 to 3 centres per warp");
  constexpr int NW = TB / 32;
  __shared__ float4 shift[27];
  __shared__ __align__(16) float gs[NW][CPB][S::GS];
  __shared__ float4 arec[NW][CPB][CPB_ANG_CAP];
  __shared__ int acount[NW][CPB];
  fill_shift_table(shift, geom);
  __syncthreads();
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int c, s, gsz;
  cpb_group<CPB>(lane, c, s, gsz);
  const int wbase = blockIdx.x * TB + w * 32;      // this warp's 32 centre atoms, CPB at a time
  const bool skip = skip_far(X);
  float wxx = 0.f, wxy = 0.f, wxz = 0.f, wyy = 0.f, wyz = 0.f, wzz = 0.f;
  long long cnt_list = 0, cnt_act = 0, cnt_rad = 0, cnt_ang = 0;
  auto apply = [&](int a, int j, float dx, float dy, float dz, float D0, float D1, float D2, float &fx, float &fy,
                   float &fz) {
    fx += D0; fy += D1; fz += D2;
    long long ox, oy, oz;
    to_fix32x3(-D0, -D1, -D2, ox, oy, oz);
    red_add(Ffix + j, ox);
    red_add(Ffix + (size_t)n + j, oy);
    red_add(Ffix + 2 * (size_t)n + j, oz);
    wxx = fmaf(dx, D0, wxx); wxy = fmaf(dx, D1, wxy); wxz = fmaf(dx, D2, wxz);
    wyy = fmaf(dy, D1, wyy); wyz = fmaf(dy, D2, wyz); wzz = fmaf(dz, D2, wzz);
  };
  for (int r0 = 0; r0 < 32; r0 += CPB) {
    const int a = wbase + r0 + c;
    const bool have = r0 + c < 32 && a < n;
    if (have) {
      const float4 *src = reinterpret_cast<const float4 *>(G + (size_t)a * S::GS);
      for (int t = s; t < S::GS / 4; t += gsz) reinterpret_cast<float4 *>(gs[w][c])[t] = __ldg(src + t);
    }
    if (s == 0) acount[w][c] = 0;
    __syncwarp();
    float fx = 0.f, fy = 0.f, fz = 0.f;
    if (have) {
      const float *Gs = gs[w][c];
      const float4 pi = pos[a];
      const RowSpan sp = full_row(X, a, skip);
      if (s == 0) cnt_list += sp.c;
      // radial and LJ pair forces over the row; the angular pairs are collected
      for (int k = s; k < sp.c; k += gsz) {
        const size_t slot = (size_t)(k < sp.c1 ? k : k + sp.gap);
        const uint32_t e = (uint32_t)nbr[slot * n + a];
        const int j = (int)(e & J_MASK);
        const float4 pj = pos[j];
        const float4 o = shift[e >> J_BITS];
        const float dx = pj.x - pi.x + o.x, dy = pj.y - pi.y + o.y, dz = pj.z - pi.z + o.z;
        const float r2 = dx * dx + dy * dy + dz * dz;
        if (r2 >= P.rmax2) continue;
        ++cnt_act;
        const float ir = rsqrtf(r2);
        const float r = r2 * ir;
        float coef = 0.f;
        if (r2 < P.rcR2) {
          ++cnt_rad;
          float f[S::KR], df[S::KR], tail[8];
#pragma unroll
          for (int b = 0; b < 8; ++b) tail[b] = Gs[S::NA * S::NLM + b];
          cheb_basis_d<S::KR>(r, P.inv_rcR, f, df);
          coef = dot_pairs<S::KR>(*reinterpret_cast<const float(*)[S::KR]>(&tail[0]), df) * ir;
        }
        if (P.lj_on != 0.f && r2 < P.lj_rc2) {
          float el, dl;
          lj_pair<S>(P, r2, r, ir, el, dl);
          coef = fmaf(0.5f * dl, ir, coef);
        }
        if (r2 < P.rcA2) {
          const int m = atomicAdd(&acount[w][c], 1);
          if (m < CPB_ANG_CAP) arec[w][c][m] = make_float4(dx, dy, dz, __int_as_float(j));
          else atomicOr(status, ST_OVERFLOW);
        }
        apply(a, j, dx, dy, dz, coef * dx, coef * dy, coef * dz, fx, fy, fz);
      }
    }
    __syncwarp();
    if (have) {
      // the three-body backward over the centre's angular pairs, lanes strided
      const float *Gs = gs[w][c];
      const int na = min(acount[w][c], CPB_ANG_CAP);
      if (s == 0) cnt_ang += na;
      for (int m = s; m < na; m += gsz) {
        const float4 q = arec[w][c][m];
        const float r2 = q.x * q.x + q.y * q.y + q.z * q.z;
        const float ir = rsqrtf(r2);
        const float r = r2 * ir;
        float2 al, gv[3];
        angular_pair_smem<S>(P, Gs, r, ir, q.x, q.y, q.z, al, gv);
        const float ca = hsum(al) * ir;
        apply(a, __float_as_int(q.w), q.x, q.y, q.z, fmaf(ca, q.x, hsum(gv[0]) * ir), fmaf(ca, q.y, hsum(gv[1]) * ir),
              fmaf(ca, q.z, hsum(gv[2]) * ir), fx, fy, fz);
      }
      // F_i: each lane's share in fixed point (integer sums: the order of the additions does not matter)
      if (fx != 0.f || fy != 0.f || fz != 0.f) {
        long long ox, oy, oz;
        to_fix32x3(fx, fy, fz, ox, oy, oz);
        red_add(Ffix + a, ox);
        red_add(Ffix + (size_t)n + a, oy);
        red_add(Ffix + 2 * (size_t)n + a, oz);
      }
      if (!(isfinite(fx) && isfinite(fy) && isfinite(fz))) atomicOr(status, ST_NAN);
    }
    __syncwarp();
  }
  long long acc[13];
  acc[0] = -to_fix32(wxx); acc[1] = -to_fix32(wxy); acc[2] = -to_fix32(wxz);
  acc[3] = acc[1]; acc[4] = -to_fix32(wyy); acc[5] = -to_fix32(wyz);
  acc[6] = acc[2]; acc[7] = acc[5]; acc[8] = -to_fix32(wzz);
  acc[9] = cnt_list; acc[10] = cnt_act; acc[11] = cnt_rad; acc[12] = cnt_ang;
  block_sum_store<13, NW>(acc, part);
}

// Angular pairs (r < rc_A) of every atom's walked row.
__global__ void k_angular_counts(const int n, const float4 *__restrict__ pos, const int32_t *__restrict__ nbr,
                                 const RowExt X, const Geom geom, float rcA2, int *__restrict__ out) {
  __shared__ float4 shift[27];
  fill_shift_table(shift, geom);
  __syncthreads();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const RowSpan sp = full_row(X, i, skip_far(X));
  const float4 pi = pos[i];
  int na = 0;
  for (int k = 0; k < sp.c; ++k) {
    const uint32_t e = (uint32_t)nbr[(size_t)(k < sp.c1 ? k : k + sp.gap) * n + i];
    const float4 pj = pos[e & J_MASK];
    const float4 o = shift[e >> J_BITS];
    const float dx = pj.x - pi.x + o.x, dy = pj.y - pi.y + o.y, dz = pj.z - pi.z + o.z;
    na += (dx * dx + dy * dy + dz * dz < rcA2) ? 1 : 0;
  }
  out[i] = na;
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

template <class S>
cudaError_t launch_force_cpb(int cpb, const Model<S> &P, const Geom &g, int n, const float4 *pos, const int32_t *nbr,
                             const RowExt &X, const float *G, long long *Ffix, long long *part, int *status,
                             cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  const int grid = (n + TB - 1) / TB;
  unsigned long long *F = reinterpret_cast<unsigned long long *>(Ffix);
  if (cpb == 1) k_force_cpb<S, 1><<<grid, TB, 0, st>>>(P, g, n, pos, nbr, X, G, F, part, status);
  else if (cpb == 2) k_force_cpb<S, 2><<<grid, TB, 0, st>>>(P, g, n, pos, nbr, X, G, F, part, status);
  else if (cpb == 3) k_force_cpb<S, 3><<<grid, TB, 0, st>>>(P, g, n, pos, nbr, X, G, F, part, status);
  else return cudaErrorInvalidValue;
  return cudaGetLastError();
}
template cudaError_t launch_force_cpb<CuShape>(int, const Model<CuShape> &, const Geom &, int, const float4 *,
                                               const int32_t *, const RowExt &, const float *, long long *, long long *,
                                               int *, cudaStream_t);

cudaError_t launch_angular_counts(int n, const float4 *pos, const int32_t *nbr, const RowExt &X, const Geom &g,
                                  float rcA2, int *out, cudaStream_t st) {
  if (n > 0) k_angular_counts<<<(n + 255) / 256, 256, 0, st>>>(n, pos, nbr, X, g, rcA2, out);
  return cudaGetLastError();
}

template cudaError_t launch_descriptor_tiled<CuShape, 1>(const Model<CuShape> &, const Geom &, int, const float4 *,
                                                         const int32_t *, const RowExt &, float *, float *,
                                                         long long *, long long *, int *, float *, cudaStream_t);
template cudaError_t launch_descriptor_tiled<CuShape, 3>(const Model<CuShape> &, const Geom &, int, const float4 *,
                                                         const int32_t *, const RowExt &, float *, float *,
                                                         long long *, long long *, int *, float *, cudaStream_t);

}  // namespace nep
