// nep_force.cu -- NEP descriptors, network and chain-rule forces on sm_103a.
//
// Two kernels per force evaluation, one thread per atom (cell-sorted order), both reading the
// distance-sorted neighbour list of nep_neighbor.cu:
//
//  k_descriptor  radial descriptors q_n (Section III.B), shifted-force LJ energy, angular sums
//                s_nlm = sum_j g_n(r_ij) Yh_lm(u_ij) for l = 1..4 (24 (l,m) components per channel,
//                all NA channels updated in one neighbour pass: the geometry -- cutoff, Chebyshev
//                basis, harmonics -- is computed once per neighbour and reused, the channel tiling of
//                Algorithm 1 with the whole channel range as one tile), q_nl = sum_m s_nlm^2 (equal to
//                the two-neighbour Legendre sum by the addition theorem), 4-body q4_n = tr(T_n^3) with
//                T_n rebuilt from the l = 2 sums, then the one-hidden-layer tanh network (Section III.B
//                equation) with its gradient.  It stores the per-atom adjoint G_nlm = dU_i/ds_nlm and
//                dU_i/dq_n (radial), and the site energy.
//  k_force       F_i = sum_j D_ij with D_ij = dU_i/dr_ij - dU_j/dr_ji.  The radial part uses both atoms'
//                dU/dq_n; the angular part uses H_nlm = G^i_nlm + (-1)^l G^j_nlm because the pair
//                geometry g_n(r) Yh_lm(u) is shared by both directions (Yh_lm(-u) = (-1)^l Yh_lm(u)).
//                Since D_ji = -D_ij exactly, each unordered pair is evaluated once, by its owner (the
//                owned part of the list), which adds D_ij to F_i and -D_ij to F_j.  The scatter uses
//                64-bit fixed-point integer atomics (2^-32 eV/Angstrom units): integer addition is
//                associative, so the forces are bitwise reproducible whatever the order of the
//                atomics -- the atomic scatter of the paper's consolidated backward kernel (Section V.B,
//                Optimization 1) made deterministic.  Virial W = -sum_pairs r_ij (x) D_ij.
//
// Everything is float32 except the per-block energy/virial partial sums (float64).
#include "nep_common.cuh"

namespace nep {

constexpr int DESC_BLOCK = 128;
#ifndef NEP_FORCE_BLOCK
#define NEP_FORCE_BLOCK 128
#endif
constexpr int FORCE_BLOCK = NEP_FORCE_BLOCK;
// Minimum resident blocks per SM requested from the compiler (register budget per thread =
// 65536 / (block * min_blocks)); the defaults are the measured best on GB300.
#ifndef NEP_DESC_MINB
#define NEP_DESC_MINB 2
#endif
#ifndef NEP_FORCE_MINB
#define NEP_FORCE_MINB 2
#endif

__device__ __forceinline__ void prefetch_l1(const void *p) { asm volatile("prefetch.global.L1 [%0];" ::"l"(p)); }

constexpr int PIPE_DE = 8;    // list entries in flight per thread
constexpr int PIPE_DP = 4;    // neighbour positions in flight per thread

template <class S>
__global__ void __launch_bounds__(DESC_BLOCK, NEP_DESC_MINB)
k_descriptor(const __grid_constant__ Model<S> P, const Geom geom, const int n, const float4 *__restrict__ pos,
             const int32_t *__restrict__ nbr, const int32_t *__restrict__ nnum, float *__restrict__ G,
             float *__restrict__ usite, float *__restrict__ qout, long long *__restrict__ Ffix,
             long long *__restrict__ part, int *__restrict__ status) {
  __shared__ float4 shift[27];
  __shared__ uint32_t ring_e[PIPE_DE * DESC_BLOCK];
  __shared__ float4 ring_p[PIPE_DP * DESC_BLOCK];
  fill_shift_table(shift, geom);
  __syncthreads();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  long long acc[5] = {0, 0, 0, 0, 0};
  if (i < n) {
    Ffix[i] = 0; Ffix[(size_t)n + i] = 0; Ffix[2 * (size_t)n + i] = 0;
    const float4 pi = pos[i];
    float qR[S::NR];
    float s[S::NA][N_LM];
#pragma unroll
    for (int a = 0; a < S::NR; ++a) qR[a] = 0.f;
#pragma unroll
    for (int a = 0; a < S::NA; ++a)
#pragma unroll
      for (int c = 0; c < N_LM; ++c) s[a][c] = 0.f;
    float elj = 0.f;
    int nrad = 0, nang = 0, nact = 0;
    const int cnt = nnum[i];
    NbrPipe<PIPE_DE, PIPE_DP, DESC_BLOCK> pipe;
    pipe.start(ring_e, ring_p, nbr + i, (size_t)n, pos, cnt);
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
        for (int a = 0; a < S::NR; ++a)
#pragma unroll
          for (int b = 0; b < S::KR; ++b) qR[a] = fmaf(P.cR[a][b], f[b], qR[a]);
        ++nrad;
      }
      if (P.lj_on != 0.f && r2 < P.lj_rc2) {
        float el, dl;
        lj_pair<S>(P, r2, r, el, dl);
        elj = fmaf(0.5f, el, elj);
      }
      if (r2 < P.rcA2) {
        float f[S::KA];
        cheb_basis<S::KA>(r, P.inv_rcA, f);
        float g[S::NA];
#pragma unroll
        for (int a = 0; a < S::NA; ++a) {
          float t = 0.f;
#pragma unroll
          for (int b = 0; b < S::KA; ++b) t = fmaf(P.cA[a][b], f[b], t);
          g[a] = t;
        }
        float Y[N_LM];
        harmonics(dx * ir, dy * ir, dz * ir, Y);
#pragma unroll
        for (int a = 0; a < S::NA; ++a)
#pragma unroll
          for (int c = 0; c < N_LM; ++c) s[a][c] = fmaf(g[a], Y[c], s[a][c]);
        ++nang;
      }
    }
    pipe.finish();

    // Descriptors: [q_n | q_nl (n-major, l = 1..4) | q4_n].
    float q[S::NDES];
#pragma unroll
    for (int a = 0; a < S::NR; ++a) q[a] = qR[a];
#pragma unroll
    for (int a = 0; a < S::NA; ++a) {
#pragma unroll
      for (int l = 1; l <= 4; ++l) {
        float t = 0.f;
#pragma unroll
        for (int c = l * l - 1; c < (l + 1) * (l + 1) - 1; ++c) t = fmaf(s[a][c], s[a][c], t);
        q[S::NR + a * 4 + (l - 1)] = t;
      }
    }
    // 4-body: T_n from the l = 2 sums (components 3..7 = m -2..2), tr(T^3) = 3 det T (T traceless).
    float Txx[S::NA], Tyy[S::NA], Tzz[S::NA], Txy[S::NA], Tyz[S::NA], Txz[S::NA];
    if (S::FOURBODY) {
      const float i3 = 0.57735026918962576f, third = 1.f / 3.f;
#pragma unroll
      for (int a = 0; a < S::NA; ++a) {
        Txy[a] = s[a][3] * i3;
        Tyz[a] = s[a][4] * i3;
        Txz[a] = s[a][6] * i3;
        Txx[a] = s[a][7] * i3 - s[a][5] * third;
        Tyy[a] = -s[a][7] * i3 - s[a][5] * third;
        Tzz[a] = 2.f * s[a][5] * third;
        const float det = Txx[a] * (Tyy[a] * Tzz[a] - Tyz[a] * Tyz[a]) - Txy[a] * (Txy[a] * Tzz[a] - Tyz[a] * Txz[a]) +
                          Txz[a] * (Txy[a] * Tyz[a] - Tyy[a] * Txz[a]);
        q[S::NR + S::NA * 4 + a] = 3.f * det;
      }
    }
    if (qout != nullptr) {
#pragma unroll
      for (int v = 0; v < S::NDES; ++v) qout[(size_t)i * S::NDES + v] = q[v];
    }
    // Park s_nlm in this atom's adjoint row while the network runs (frees ~120 registers); it is
    // read back below and overwritten in place by G_nlm.
    float *Gi = G + (size_t)i * GSTRIDE;
#pragma unroll
    for (int a = 0; a < S::NA; ++a)
#pragma unroll
      for (int c = 0; c < N_LM; c += 4)
        *reinterpret_cast<float4 *>(Gi + a * N_LM + c) = make_float4(s[a][c], s[a][c + 1], s[a][c + 2], s[a][c + 3]);
    asm volatile("" ::: "memory");

    // Network: U = sum_mu w1 tanh(sum_nu W0 q~_nu - b0) - b1; dU/dq~ accumulated in dq.
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

    // Adjoint G_nlm = dU/ds_nlm = 2 Fp_nl s_nlm (+ 4-body term for l = 2), s read back from the row.
    asm volatile("" ::: "memory");
#pragma unroll
    for (int a = 0; a < S::NA; ++a) {
      float gl[N_LM];
#pragma unroll
      for (int c = 0; c < N_LM; c += 4) {
        const float4 t = *reinterpret_cast<const float4 *>(Gi + a * N_LM + c);
        gl[c] = t.x; gl[c + 1] = t.y; gl[c + 2] = t.z; gl[c + 3] = t.w;
      }
#pragma unroll
      for (int c = 0; c < N_LM; ++c) gl[c] *= 2.f * Fp[S::NR + a * 4 + lm_l(c) - 1];
      if (S::FOURBODY) {
        // d tr(T^3)/d s_m = 3 (T^2) : dT/ds_m, M = T^2.
        const float f4 = Fp[S::NR + S::NA * 4 + a];
        const float Mxx = Txx[a] * Txx[a] + Txy[a] * Txy[a] + Txz[a] * Txz[a];
        const float Myy = Txy[a] * Txy[a] + Tyy[a] * Tyy[a] + Tyz[a] * Tyz[a];
        const float Mzz = Txz[a] * Txz[a] + Tyz[a] * Tyz[a] + Tzz[a] * Tzz[a];
        const float Mxy = Txx[a] * Txy[a] + Txy[a] * Tyy[a] + Txz[a] * Tyz[a];
        const float Myz = Txy[a] * Txz[a] + Tyy[a] * Tyz[a] + Tyz[a] * Tzz[a];
        const float Mxz = Txx[a] * Txz[a] + Txy[a] * Tyz[a] + Txz[a] * Tzz[a];
        const float s3 = 1.7320508075688772f;
        gl[3] = fmaf(f4, 2.f * s3 * Mxy, gl[3]);
        gl[4] = fmaf(f4, 2.f * s3 * Myz, gl[4]);
        gl[5] = fmaf(f4, 2.f * Mzz - Mxx - Myy, gl[5]);
        gl[6] = fmaf(f4, 2.f * s3 * Mxz, gl[6]);
        gl[7] = fmaf(f4, s3 * (Mxx - Myy), gl[7]);
      }
#pragma unroll
      for (int c = 0; c < N_LM; c += 4)
        *reinterpret_cast<float4 *>(Gi + a * N_LM + c) = make_float4(gl[c], gl[c + 1], gl[c + 2], gl[c + 3]);
    }
    {
      float tail[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
      for (int a = 0; a < S::NR; ++a) tail[a] = Fp[a];
      *reinterpret_cast<float4 *>(Gi + S::NA * N_LM) = make_float4(tail[0], tail[1], tail[2], tail[3]);
      *reinterpret_cast<float4 *>(Gi + S::NA * N_LM + 4) = make_float4(tail[4], tail[5], tail[6], tail[7]);
    }
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

template <class S>
__global__ void __launch_bounds__(FORCE_BLOCK, NEP_FORCE_MINB)
k_force(const __grid_constant__ Model<S> P, const Geom geom, const int n, const float4 *__restrict__ pos,
        const int32_t *__restrict__ nbr, const int32_t *__restrict__ nown, const int32_t *__restrict__ nband0,
        const float *__restrict__ G, unsigned long long *__restrict__ Ffix, long long *__restrict__ part,
        int *__restrict__ status) {
  __shared__ float4 shift[27];
  __shared__ uint32_t ring_e[PIPE_DE * FORCE_BLOCK];
  __shared__ float4 ring_p[PIPE_DP * FORCE_BLOCK];
  fill_shift_table(shift, geom);
  __syncthreads();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  long long acc[13] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
  if (i < n) {
    const float4 pi = pos[i];
    const float *Gi = G + (size_t)i * GSTRIDE;
    float gi[S::NA][N_LM];
#define GI(a, lm) gi[a][lm]
#pragma unroll
    for (int a = 0; a < S::NA; ++a)
#pragma unroll
      for (int c = 0; c < N_LM; c += 4) {
        const float4 t = __ldg(reinterpret_cast<const float4 *>(Gi + a * N_LM + c));
        GI(a, c) = t.x; GI(a, c + 1) = t.y; GI(a, c + 2) = t.z; GI(a, c + 3) = t.w;
      }
    float fpi[8];
    {
      const float4 t0 = __ldg(reinterpret_cast<const float4 *>(Gi + S::NA * N_LM));
      const float4 t1 = __ldg(reinterpret_cast<const float4 *>(Gi + S::NA * N_LM + 4));
      fpi[0] = t0.x; fpi[1] = t0.y; fpi[2] = t0.z; fpi[3] = t0.w;
      fpi[4] = t1.x; fpi[5] = t1.y; fpi[6] = t1.z; fpi[7] = t1.w;
    }
    float fx = 0.f, fy = 0.f, fz = 0.f;
    float wxx = 0.f, wxy = 0.f, wxz = 0.f, wyx = 0.f, wyy = 0.f, wyz = 0.f, wzx = 0.f, wzy = 0.f, wzz = 0.f;
    const int cnt = nown[i];
    const int nb0 = nband0[i];
    int nrad = 0, nang = 0, nact = 0;
    NbrPipe<PIPE_DE, PIPE_DP, FORCE_BLOCK> pipe;
    pipe.start(ring_e, ring_p, nbr + i, (size_t)n, pos, cnt);
    for (int k = 0; k < cnt; ++k) {
      uint32_t e;
      float4 pj;
      pipe.get(k, e, pj);
      // pull the next angular neighbour's adjoint row into L1 while this pair is computed
      if (k + 1 < nb0 && k + 1 < cnt) {
        const uint32_t en = pipe.re[((k + 1) % PIPE_DE) * FORCE_BLOCK];
        const char *gr = reinterpret_cast<const char *>(G + (size_t)(en & J_MASK) * GSTRIDE);
        prefetch_l1(gr); prefetch_l1(gr + 128); prefetch_l1(gr + 256); prefetch_l1(gr + 384);
      }
      const int j = (int)(e & J_MASK);
      const float4 o = shift[e >> J_BITS];
      const float dx = pj.x - pi.x + o.x, dy = pj.y - pi.y + o.y, dz = pj.z - pi.z + o.z;
      const float r2 = dx * dx + dy * dy + dz * dz;
      if (r2 >= P.rmax2) continue;
      ++nact;
      const float ir = rsqrtf(r2);
      const float r = r2 * ir;
      const float *Gj = G + (size_t)j * GSTRIDE;
      float coef = 0.f;                     // D = coef * d + (vx, vy, vz)
      float vx = 0.f, vy = 0.f, vz = 0.f;
      if (r2 < P.rcR2) {
        float f[S::KR], df[S::KR];
        cheb_basis_d<S::KR>(r, P.inv_rcR, f, df);
        const float4 t0 = __ldg(reinterpret_cast<const float4 *>(Gj + S::NA * N_LM));
        const float4 t1 = __ldg(reinterpret_cast<const float4 *>(Gj + S::NA * N_LM + 4));
        const float fpj[8] = {t0.x, t0.y, t0.z, t0.w, t1.x, t1.y, t1.z, t1.w};
        float c = 0.f;
#pragma unroll
        for (int a = 0; a < S::NR; ++a) {
          float dg = 0.f;
#pragma unroll
          for (int b = 0; b < S::KR; ++b) dg = fmaf(P.cR[a][b], df[b], dg);
          c = fmaf(fpi[a] + fpj[a], dg, c);
        }
        coef = c * ir;
        ++nrad;
      }
      if (P.lj_on != 0.f && r2 < P.lj_rc2) {
        float el, dl;
        lj_pair<S>(P, r2, r, el, dl);
        coef = fmaf(dl, ir, coef);
      }
      if (r2 < P.rcA2) {
        ++nang;
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
        float Y[N_LM];
        harmonics(ux, uy, uz, Y);
        float along = 0.f, bx = 0.f, by = 0.f, bz = 0.f;
        // d/dd [g_n(r) Yh_lm(u)] = (g_n' - l g_n / r) Yh_lm u + (g_n / r) grad P_lm(u)
#pragma unroll
        for (int c = 0; c < N_LM; c += 4) {
          float4 hj[S::NA];
#pragma unroll
          for (int a = 0; a < S::NA; ++a) hj[a] = __ldg(reinterpret_cast<const float4 *>(Gj + a * N_LM + c));
#pragma unroll
          for (int cc = 0; cc < 4; ++cc) {
            const int lm = c + cc;
            const float sgn = (lm_l(lm) & 1) ? -1.f : 1.f;
            float av = 0.f, bv = 0.f;
#pragma unroll
            for (int a = 0; a < S::NA; ++a) {
              const float gjv = cc == 0 ? hj[a].x : (cc == 1 ? hj[a].y : (cc == 2 ? hj[a].z : hj[a].w));
              const float H = fmaf(sgn, gjv, GI(a, lm));
              av = fmaf(H, dg[a], av);
              bv = fmaf(H, g[a], bv);
            }
            along = fmaf(av - (float)lm_l(lm) * ir * bv, Y[lm], along);
            harmonic_grad_acc(lm, ux, uy, uz, bv, bx, by, bz);
          }
        }
        coef = fmaf(along, ir, coef);
        vx = bx * ir; vy = by * ir; vz = bz * ir;
      }
      const float Dx = fmaf(coef, dx, vx), Dy = fmaf(coef, dy, vy), Dz = fmaf(coef, dz, vz);
      fx += Dx; fy += Dy; fz += Dz;
      // Newton's third law: F_j -= D_ij, accumulated in fixed point (order-independent sum)
      atomicAdd(Ffix + j, (unsigned long long)(-to_fix32(Dx)));
      atomicAdd(Ffix + (size_t)n + j, (unsigned long long)(-to_fix32(Dy)));
      atomicAdd(Ffix + 2 * (size_t)n + j, (unsigned long long)(-to_fix32(Dz)));
      wxx = fmaf(dx, Dx, wxx); wxy = fmaf(dx, Dy, wxy); wxz = fmaf(dx, Dz, wxz);
      wyx = fmaf(dy, Dx, wyx); wyy = fmaf(dy, Dy, wyy); wyz = fmaf(dy, Dz, wyz);
      wzx = fmaf(dz, Dx, wzx); wzy = fmaf(dz, Dy, wzy); wzz = fmaf(dz, Dz, wzz);
    }
    pipe.finish();
    atomicAdd(Ffix + i, (unsigned long long)to_fix32(fx));
    atomicAdd(Ffix + (size_t)n + i, (unsigned long long)to_fix32(fy));
    atomicAdd(Ffix + 2 * (size_t)n + i, (unsigned long long)to_fix32(fz));
    if (!(isfinite(fx) && isfinite(fy) && isfinite(fz))) atomicOr(status, ST_NAN);
    // each unordered pair once: W = -sum_pairs r_ij (x) D_ij
    acc[0] = -to_fix32(wxx); acc[1] = -to_fix32(wxy); acc[2] = -to_fix32(wxz);
    acc[3] = -to_fix32(wyx); acc[4] = -to_fix32(wyy); acc[5] = -to_fix32(wyz);
    acc[6] = -to_fix32(wzx); acc[7] = -to_fix32(wzy); acc[8] = -to_fix32(wzz);
    acc[9] = cnt; acc[10] = nact; acc[11] = nrad; acc[12] = nang;
  }
  block_sum_store<13>(acc, part);
#undef GI
}

// ---------------------------------------------------------------------------------------------------
// Host launchers (called from nep_api.cu).

template <class S>
cudaError_t launch_descriptor(const Model<S> &P, const Geom &g, int n, const float4 *pos, const int32_t *nbr,
                              const int32_t *nnum, float *G, float *usite, float *qout, long long *Ffix,
                              long long *part, int *status, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  const int grid = (n + DESC_BLOCK - 1) / DESC_BLOCK;
  k_descriptor<S><<<grid, DESC_BLOCK, 0, st>>>(P, g, n, pos, nbr, nnum, G, usite, qout, Ffix, part, status);
  return cudaGetLastError();
}

template <class S>
cudaError_t launch_force(const Model<S> &P, const Geom &g, int n, const float4 *pos, const int32_t *nbr,
                         const int32_t *nown, const int32_t *nband0, const float *G, long long *Ffix, long long *part,
                         int *status, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  const int grid = (n + FORCE_BLOCK - 1) / FORCE_BLOCK;
  k_force<S><<<grid, FORCE_BLOCK, 0, st>>>(P, g, n, pos, nbr, nown, nband0, G,
                                              reinterpret_cast<unsigned long long *>(Ffix), part, status);
  return cudaGetLastError();
}

int descriptor_blocks(int n) { return (n + DESC_BLOCK - 1) / DESC_BLOCK; }
int force_blocks(int n) { return (n + FORCE_BLOCK - 1) / FORCE_BLOCK; }

template cudaError_t launch_descriptor<CuShape>(const Model<CuShape> &, const Geom &, int, const float4 *,
                                                const int32_t *, const int32_t *, float *, float *, float *,
                                                long long *, long long *, int *, cudaStream_t);
template cudaError_t launch_force<CuShape>(const Model<CuShape> &, const Geom &, int, const float4 *,
                                           const int32_t *, const int32_t *, const int32_t *, const float *,
                                           long long *, long long *, int *, cudaStream_t);

}  // namespace nep
