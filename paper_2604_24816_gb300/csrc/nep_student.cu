// nep_student.cu -- training kernels of the student NEP (radial n_max 3, angular n_max 3, l_max 2, no
// 4-body term, 16 neurons), declared in nep_student.h.
//
// The student's descriptors are linear (radial) or quadratic (angular) in per-atom basis sums that
// depend on positions only:
//   q_n  = sum_k cR_nk Q_k,                 Q_k   = sum_j f^R_k(r_ij)
//   q_nl = sum_{m in l} s_nlm^2,  s_nlm = sum_k cA_nk S_klm,   S_klm = sum_j f^A_k(r_ij) Y_lm(u_ij)
// (the radial and angular descriptor definitions of Section III.B).  Q and S are computed once per
// training set; each training step then runs: st_forward (per atom) -> st_energy (per cell) ->
// st_force (pair gather) for the loss, and st_jvp (pair pass) -> st_grad (per atom + fixed-order
// reduction) for its gradient.
//
// Gradient of the force loss.  With v = dL/dF, sum_i v_i . F_i = -sum_i Fp_i . dq_i where
// dq_i = sum_k v_k . dq_i/dr_k is the directional derivative of the descriptors along v, so its
// parameter gradient is -d/dtheta sum_i Fp_i(theta) . dq_i(theta).  dq depends on theta through the
// expansion coefficients only: dq_n = sum_k cR_nk dQ_k, dq_nl = 2 sum_m s_nlm ds_nlm with
// ds_nlm = sum_k cA_nk dS_klm, where dQ, dS are the directional derivatives of the basis sums (st_jvp).
// For the one-hidden-layer network, J = Fp . dq = sum_mu w1_mu (1 - h_mu^2) zdot_mu with
// zdot_mu = sum_nu W0_mu,nu s_nu dq_nu, whose derivatives are written out in st_grad.
#include <cuda_runtime.h>

#include "nep_common.cuh"
#include "nep_student.h"

namespace nep {
namespace {

using SS = StudentShape;
constexpr int KB = SS::KR;                   // basis functions (radial and angular: 8)
constexpr int NLM = SS::NLM;                 // 8 harmonics (l = 1, 2)
constexpr int NSB = SS::KA * NLM;            // 64 angular basis sums
constexpr int NR = SS::NR, NA = SS::NA, ND = SS::NDES, NN = SS::NNEU;
constexpr int OFF_CR = 0, OFF_CA = OFF_CR + NR * KB, OFF_W0 = OFF_CA + NA * KB, OFF_B0 = OFF_W0 + NN * ND,
              OFF_W1 = OFF_B0 + NN, OFF_B1 = OFF_W1 + NN, NPAR = OFF_B1 + 1;
static_assert(NPAR == ST_NPAR && ND == ST_NDES && SS::GS == ST_GS, "header constants out of date");
static_assert(SS::KR == SS::KA, "one basis size for both cutoffs");

constexpr int BLOCK = 128;
constexpr int GRAD_BLOCK = 64;               // atoms per block of st_grad
constexpr int GREC = NPAR;                   // floats per atom record in st_grad's shared memory

struct Cut {
  float rcR2, rcA2, inv_rcR, inv_rcA;
};
Cut cut_of(st_cutoffs rc) { return Cut{rc.rc_R * rc.rc_R, rc.rc_A * rc.rc_A, 1.f / rc.rc_R, 1.f / rc.rc_A}; }

__device__ __forceinline__ int l_of(int lm) { return lm < 3 ? 1 : 2; }

// theta (and q_scale) staged in shared memory once per block.
__device__ __forceinline__ void stage_theta(float *sth, const float *theta, float *sqs, const float *qs) {
  for (int p = threadIdx.x; p < NPAR; p += blockDim.x) sth[p] = theta[p];
  if (sqs != nullptr)
    for (int p = threadIdx.x; p < ND; p += blockDim.x) sqs[p] = qs[p];
}

// ---------------------------------------------------------------------------------------------------
__global__ void k_st_pairs(int n, const float4 *__restrict__ pos, const int *__restrict__ start,
                           const float *__restrict__ boxes, float rc2, int cap, int *__restrict__ nbr,
                           float4 *__restrict__ dvec, int *__restrict__ nnum, int *__restrict__ status) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float4 pi = pos[i];
  const int s = __float_as_int(pi.w);
  const float bx = boxes[3 * s], by = boxes[3 * s + 1], bz = boxes[3 * s + 2];
  const float ibx = 1.f / bx, iby = 1.f / by, ibz = 1.f / bz;
  const int j0 = start[s], j1 = start[s + 1];
  int c = 0;
  for (int j = j0; j < j1; ++j) {
    if (j == i) continue;
    const float4 pj = pos[j];
    float dx = pj.x - pi.x, dy = pj.y - pi.y, dz = pj.z - pi.z;
    dx -= bx * rintf(dx * ibx);
    dy -= by * rintf(dy * iby);
    dz -= bz * rintf(dz * ibz);
    if (dx * dx + dy * dy + dz * dz < rc2) {
      if (c < cap) {
        nbr[(size_t)c * n + i] = j;
        dvec[(size_t)c * n + i] = make_float4(dx, dy, dz, 0.f);
      }
      ++c;
    }
  }
  nnum[i] = min(c, cap);
  if (c > cap) atomicOr(status, ST_OVERFLOW);
}

// ---------------------------------------------------------------------------------------------------
__global__ void k_st_basis(int a0, int a1, int n, const int *__restrict__ nnum, const float4 *__restrict__ dvec,
                           Cut C, float *__restrict__ Q, float *__restrict__ S) {
  const int a = a0 + blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= a1) return;
  float q[KB], s[KB][NLM];
#pragma unroll
  for (int k = 0; k < KB; ++k) {
    q[k] = 0.f;
#pragma unroll
    for (int c = 0; c < NLM; ++c) s[k][c] = 0.f;
  }
  const int cnt = nnum[a];
  for (int e = 0; e < cnt; ++e) {
    const float4 d = dvec[(size_t)e * n + a];
    const float r2 = d.x * d.x + d.y * d.y + d.z * d.z;
    const float ir = rsqrtf(r2), r = r2 * ir;
    if (r2 < C.rcR2) {
      float f[KB];
      cheb_basis<KB>(r, C.inv_rcR, f);
#pragma unroll
      for (int k = 0; k < KB; ++k) q[k] += f[k];
    }
    if (r2 < C.rcA2) {
      float f[KB], Y[NLM];
      cheb_basis<KB>(r, C.inv_rcA, f);
      harmonics<NLM>(d.x * ir, d.y * ir, d.z * ir, Y);
#pragma unroll
      for (int k = 0; k < KB; ++k)
#pragma unroll
        for (int c = 0; c < NLM; ++c) s[k][c] = fmaf(f[k], Y[c], s[k][c]);
    }
  }
#pragma unroll
  for (int k = 0; k < KB; ++k) Q[(size_t)a * KB + k] = q[k];
#pragma unroll
  for (int k = 0; k < KB; ++k)
#pragma unroll
    for (int c = 0; c < NLM; ++c) S[(size_t)a * NSB + k * NLM + c] = s[k][c];
}

// Per-atom forward pieces shared by st_forward and st_grad: descriptors, hidden layer, dU/dq.
struct AtomNet {
  float s[NA][NLM];     // s_nlm
  float q[ND];          // unscaled descriptors
  float h[NN];          // tanh activations
  float Fp[ND];         // dU/dq (unscaled q)
  float U;
};

__device__ __forceinline__ void atom_net(const float *th, const float *qs, const float *Qa, const float *Sa,
                                         AtomNet &A) {
#pragma unroll
  for (int nn = 0; nn < NR; ++nn) {
    float t = 0.f;
#pragma unroll
    for (int k = 0; k < KB; ++k) t = fmaf(th[OFF_CR + nn * KB + k], Qa[k], t);
    A.q[nn] = t;
  }
#pragma unroll
  for (int nn = 0; nn < NA; ++nn) {
#pragma unroll
    for (int c = 0; c < NLM; ++c) {
      float t = 0.f;
#pragma unroll
      for (int k = 0; k < KB; ++k) t = fmaf(th[OFF_CA + nn * KB + k], Sa[k * NLM + c], t);
      A.s[nn][c] = t;
    }
    float q1 = 0.f, q2 = 0.f;
#pragma unroll
    for (int c = 0; c < 3; ++c) q1 = fmaf(A.s[nn][c], A.s[nn][c], q1);
#pragma unroll
    for (int c = 3; c < NLM; ++c) q2 = fmaf(A.s[nn][c], A.s[nn][c], q2);
    A.q[NR + 2 * nn] = q1;
    A.q[NR + 2 * nn + 1] = q2;
  }
  float dq[ND];
#pragma unroll
  for (int v = 0; v < ND; ++v) dq[v] = 0.f;
  float U = -th[OFF_B1];
#pragma unroll
  for (int mu = 0; mu < NN; ++mu) {
    float z = -th[OFF_B0 + mu];
#pragma unroll
    for (int v = 0; v < ND; ++v) z = fmaf(th[OFF_W0 + mu * ND + v], qs[v] * A.q[v], z);
    const float h = tanhf(z);
    A.h[mu] = h;
    const float w1 = th[OFF_W1 + mu];
    U = fmaf(w1, h, U);
    const float t = w1 * (1.f - h * h);
#pragma unroll
    for (int v = 0; v < ND; ++v) dq[v] = fmaf(t, th[OFF_W0 + mu * ND + v], dq[v]);
  }
#pragma unroll
  for (int v = 0; v < ND; ++v) A.Fp[v] = dq[v] * qs[v];
  A.U = U;
}

__global__ void k_st_forward(int a0, int a1, const float *__restrict__ theta, const float *__restrict__ qscale,
                             const float *__restrict__ Q, const float *__restrict__ S, float *__restrict__ Uo,
                             float *__restrict__ G, float *__restrict__ qout) {
  __shared__ float th[NPAR], qs[ND];
  stage_theta(th, theta, qs, qscale);
  __syncthreads();
  const int a = a0 + blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= a1) return;
  float Qa[KB], Sa[NSB];
#pragma unroll
  for (int k = 0; k < KB; ++k) Qa[k] = Q[(size_t)a * KB + k];
#pragma unroll
  for (int c = 0; c < NSB; ++c) Sa[c] = S[(size_t)a * NSB + c];
  AtomNet A;
  atom_net(th, qs, Qa, Sa, A);
  Uo[a] = A.U;
  float *g = G + (size_t)a * SS::GS;
#pragma unroll
  for (int nn = 0; nn < NA; ++nn)
#pragma unroll
    for (int c = 0; c < NLM; ++c) g[nn * NLM + c] = 2.f * A.Fp[NR + 2 * nn + l_of(c) - 1] * A.s[nn][c];
#pragma unroll
  for (int t = 0; t < 8; ++t) g[NA * NLM + t] = t < NR ? A.Fp[t] : 0.f;
  if (qout != nullptr) {
#pragma unroll
    for (int v = 0; v < ND; ++v) qout[(size_t)a * ND + v] = A.q[v];
  }
}

// One warp per cell: lanes stride over its atoms, float64 sums combined by a fixed shuffle tree.
__global__ void k_st_energy(int s0, int s1, const int *__restrict__ start, const float *__restrict__ U,
                            double *__restrict__ E) {
  const int s = s0 + (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (s >= s1) return;
  double t = 0.0;
  for (int a = start[s] + lane; a < start[s + 1]; a += 32) t += (double)U[a];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
  if (lane == 0) E[s] = t;
}

// ---------------------------------------------------------------------------------------------------
// F_i = sum_j D_ij, D_ij = dU_i/dd_ij - dU_j/dd_ji: radial part (Fp_i + Fp_j) . g'(r) u, angular part
// with H_nlm = G^i_nlm + (-1)^l G^j_nlm contracted with grad_d [g^A_n(r) Y_lm(d/r)].
__global__ void k_st_force(int a0, int a1, int n, const int *__restrict__ nbr, const float4 *__restrict__ dvec,
                           const int *__restrict__ nnum, Cut C, const float *__restrict__ theta,
                           const float *__restrict__ G, float *__restrict__ F) {
  __shared__ float th[NPAR];
  stage_theta(th, theta, nullptr, nullptr);
  __syncthreads();
  const int a = a0 + blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= a1) return;
  float gi[SS::GS];
#pragma unroll
  for (int t = 0; t < SS::GS; ++t) gi[t] = G[(size_t)a * SS::GS + t];
  float fx = 0.f, fy = 0.f, fz = 0.f;
  const int cnt = nnum[a];
  for (int e = 0; e < cnt; ++e) {
    const int j = nbr[(size_t)e * n + a];
    const float4 d = dvec[(size_t)e * n + a];
    const float *gj = G + (size_t)j * SS::GS;
    const float r2 = d.x * d.x + d.y * d.y + d.z * d.z;
    const float ir = rsqrtf(r2), r = r2 * ir;
    float coef = 0.f, vx = 0.f, vy = 0.f, vz = 0.f;
    if (r2 < C.rcR2) {
      float f[KB], df[KB];
      cheb_basis_d<KB>(r, C.inv_rcR, f, df);
      float c = 0.f;
#pragma unroll
      for (int nn = 0; nn < NR; ++nn) {
        float dg = 0.f;
#pragma unroll
        for (int k = 0; k < KB; ++k) dg = fmaf(th[OFF_CR + nn * KB + k], df[k], dg);
        c = fmaf(gi[NA * NLM + nn] + gj[NA * NLM + nn], dg, c);
      }
      coef = c * ir;
    }
    if (r2 < C.rcA2) {
      float f[KB], df[KB];
      cheb_basis_d<KB>(r, C.inv_rcA, f, df);
      float g[NA], dg[NA];
#pragma unroll
      for (int nn = 0; nn < NA; ++nn) {
        float t = 0.f, dt = 0.f;
#pragma unroll
        for (int k = 0; k < KB; ++k) {
          t = fmaf(th[OFF_CA + nn * KB + k], f[k], t);
          dt = fmaf(th[OFF_CA + nn * KB + k], df[k], dt);
        }
        g[nn] = t; dg[nn] = dt;
      }
      const float ux = d.x * ir, uy = d.y * ir, uz = d.z * ir;
      float Y[NLM];
      harmonics<NLM>(ux, uy, uz, Y);
      float along = 0.f, bx = 0.f, by = 0.f, bz = 0.f;
#pragma unroll
      for (int c = 0; c < NLM; ++c) {
        const float sgn = (l_of(c) & 1) ? -1.f : 1.f;
        float av = 0.f, bv = 0.f;
#pragma unroll
        for (int nn = 0; nn < NA; ++nn) {
          const float H = fmaf(sgn, gj[nn * NLM + c], gi[nn * NLM + c]);
          av = fmaf(H, dg[nn], av);
          bv = fmaf(H, g[nn], bv);
        }
        along = fmaf(av - (float)l_of(c) * ir * bv, Y[c], along);
        harmonic_grad_acc(c, ux, uy, uz, bv, bx, by, bz);
      }
      coef = fmaf(along, ir, coef);
      vx = bx * ir; vy = by * ir; vz = bz * ir;
    }
    fx += fmaf(coef, d.x, vx);
    fy += fmaf(coef, d.y, vy);
    fz += fmaf(coef, d.z, vz);
  }
  F[3 * (size_t)a] = fx;
  F[3 * (size_t)a + 1] = fy;
  F[3 * (size_t)a + 2] = fz;
}

// ---------------------------------------------------------------------------------------------------
// dQ_k = sum_j f^R_k'(r) (u . w),  dS_klm = sum_j [f^A_k'(r) Y_lm (u . w) + f^A_k(r) (grad P_lm(u) . w
// - l Y_lm (u . w)) / r],  w = v_j - v_i: the change of the basis sums when every atom moves along v.
__global__ void k_st_jvp(int a0, int a1, int n, const int *__restrict__ nbr, const float4 *__restrict__ dvec,
                         const int *__restrict__ nnum, Cut C, const float *__restrict__ v, float *__restrict__ dQ,
                         float *__restrict__ dS) {
  const int a = a0 + blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= a1) return;
  const float vax = v[3 * (size_t)a], vay = v[3 * (size_t)a + 1], vaz = v[3 * (size_t)a + 2];
  float q[KB], s[KB][NLM];
#pragma unroll
  for (int k = 0; k < KB; ++k) {
    q[k] = 0.f;
#pragma unroll
    for (int c = 0; c < NLM; ++c) s[k][c] = 0.f;
  }
  const int cnt = nnum[a];
  for (int e = 0; e < cnt; ++e) {
    const int j = nbr[(size_t)e * n + a];
    const float4 d = dvec[(size_t)e * n + a];
    const float wx = v[3 * (size_t)j] - vax, wy = v[3 * (size_t)j + 1] - vay, wz = v[3 * (size_t)j + 2] - vaz;
    const float r2 = d.x * d.x + d.y * d.y + d.z * d.z;
    const float ir = rsqrtf(r2), r = r2 * ir;
    const float ux = d.x * ir, uy = d.y * ir, uz = d.z * ir;
    const float uw = ux * wx + uy * wy + uz * wz;
    if (r2 < C.rcR2) {
      float f[KB], df[KB];
      cheb_basis_d<KB>(r, C.inv_rcR, f, df);
#pragma unroll
      for (int k = 0; k < KB; ++k) q[k] = fmaf(df[k], uw, q[k]);
    }
    if (r2 < C.rcA2) {
      float f[KB], df[KB], Y[NLM];
      cheb_basis_d<KB>(r, C.inv_rcA, f, df);
      harmonics<NLM>(ux, uy, uz, Y);
#pragma unroll
      for (int c = 0; c < NLM; ++c) {
        float gx = 0.f, gy = 0.f, gz = 0.f;
        harmonic_grad_acc(c, ux, uy, uz, 1.f, gx, gy, gz);
        const float t1 = Y[c] * uw;
        const float t2 = (gx * wx + gy * wy + gz * wz - (float)l_of(c) * t1) * ir;
#pragma unroll
        for (int k = 0; k < KB; ++k) s[k][c] = fmaf(df[k], t1, fmaf(f[k], t2, s[k][c]));
      }
    }
  }
#pragma unroll
  for (int k = 0; k < KB; ++k) dQ[(size_t)a * KB + k] = q[k];
#pragma unroll
  for (int k = 0; k < KB; ++k)
#pragma unroll
    for (int c = 0; c < NLM; ++c) dS[(size_t)a * NSB + k * NLM + c] = s[k][c];
}

// ---------------------------------------------------------------------------------------------------
// Parameter gradient.  Per atom (U = network output, J = Fp . dq, both functions of theta):
//   dL/dtheta += gE dU/dtheta - dJ/dtheta.
// With qt = s (.) q, u = s (.) dq, zdot = W0 u, h = tanh(z), Fp = s (.) W0^T (w1 (.) (1 - h^2)),
// R = dJ/dq (at fixed dq) = s (.) W0^T (-2 w1 (.) zdot (.) h (.) (1 - h^2)):
//   W0_mu,nu : alpha_mu qt_nu + beta_mu u_nu,   alpha = w1 (1-h^2)(gE + 2 h zdot),  beta = -w1 (1-h^2)
//   b0_mu    : -alpha_mu
//   w1_mu    : gE h_mu - (1 - h_mu^2) zdot_mu
//   b1       : -gE
//   cR_nk    : rho_n Q_k + sigma_n dQ_k,        rho = gE Fp - R (radial), sigma = -Fp (radial)
//   cA_nk    : sum_lm kappa_nlm S_klm + lambda_nlm dS_klm,
//              kappa = 2 (gE Fp_nl - R_nl) s_nlm - 2 Fp_nl ds_nlm,  lambda = -2 Fp_nl s_nlm.
// Each thread builds its atom's record of these factors in shared memory; then thread t sums outputs
// t, t + 64, ... over the block's atoms.  Block partials are summed over blocks in float64 by
// k_st_grad_reduce in a fixed order.
namespace rec {
constexpr int QT = 0, U = QT + ND, AL = U + ND, BE = AL + NN, GW1 = BE + NN, GB1 = GW1 + NN, RHO = GB1 + 1,
              SIG = RHO + NR, KAP = SIG + NR, LAM = KAP + NA * NLM, Q = LAM + NA * NLM, DQ = Q + KB, S = DQ + KB,
              DS = S + NSB, END = DS + NSB;
}
static_assert(rec::END == GREC, "record layout");

__global__ void __launch_bounds__(GRAD_BLOCK)
k_st_grad(int a0, int a1, const float *__restrict__ theta, const float *__restrict__ qscale,
          const float4 *__restrict__ pos, const float *__restrict__ Q, const float *__restrict__ S,
          const float *__restrict__ dQ, const float *__restrict__ dS, const double *__restrict__ gE,
          float *__restrict__ part) {
  extern __shared__ float smem[];
  float *th = smem;                       // NPAR
  float *qs = th + NPAR;                  // ND (padded to 16)
  float *R = qs + 16;                     // GRAD_BLOCK records of GREC floats
  stage_theta(th, theta, qs, qscale);
  __syncthreads();
  const int t = threadIdx.x;
  const int a = a0 + blockIdx.x * GRAD_BLOCK + t;
  float *rc = R + t * GREC;
  if (a < a1) {
    float Qa[KB], Sa[NSB];
#pragma unroll
    for (int k = 0; k < KB; ++k) Qa[k] = Q[(size_t)a * KB + k];
#pragma unroll
    for (int c = 0; c < NSB; ++c) Sa[c] = S[(size_t)a * NSB + c];
    AtomNet A;
    atom_net(th, qs, Qa, Sa, A);
    const float ge = (float)gE[__float_as_int(pos[a].w)];
    // directional derivatives of the descriptors
    float dq[ND], ds[NA][NLM];
    float dQa[KB];
#pragma unroll
    for (int k = 0; k < KB; ++k) dQa[k] = dQ[(size_t)a * KB + k];
#pragma unroll
    for (int nn = 0; nn < NR; ++nn) {
      float tq = 0.f;
#pragma unroll
      for (int k = 0; k < KB; ++k) tq = fmaf(th[OFF_CR + nn * KB + k], dQa[k], tq);
      dq[nn] = tq;
    }
#pragma unroll
    for (int nn = 0; nn < NA; ++nn) {
      float d1 = 0.f, d2 = 0.f;
#pragma unroll
      for (int c = 0; c < NLM; ++c) {
        float tq = 0.f;
#pragma unroll
        for (int k = 0; k < KB; ++k) tq = fmaf(th[OFF_CA + nn * KB + k], dS[(size_t)a * NSB + k * NLM + c], tq);
        ds[nn][c] = tq;
        if (c < 3) d1 = fmaf(2.f * A.s[nn][c], tq, d1);
        else d2 = fmaf(2.f * A.s[nn][c], tq, d2);
      }
      dq[NR + 2 * nn] = d1;
      dq[NR + 2 * nn + 1] = d2;
    }
    float u[ND], zd[NN];
#pragma unroll
    for (int v = 0; v < ND; ++v) u[v] = qs[v] * dq[v];
#pragma unroll
    for (int mu = 0; mu < NN; ++mu) {
      float z = 0.f;
#pragma unroll
      for (int v = 0; v < ND; ++v) z = fmaf(th[OFF_W0 + mu * ND + v], u[v], z);
      zd[mu] = z;
    }
    float Rq[ND];
#pragma unroll
    for (int v = 0; v < ND; ++v) Rq[v] = 0.f;
#pragma unroll
    for (int mu = 0; mu < NN; ++mu) {
      const float h = A.h[mu], w1 = th[OFF_W1 + mu], d1h = 1.f - h * h;
      const float cr = -2.f * w1 * zd[mu] * h * d1h;
#pragma unroll
      for (int v = 0; v < ND; ++v) Rq[v] = fmaf(cr, th[OFF_W0 + mu * ND + v], Rq[v]);
      const float al = w1 * d1h * (ge + 2.f * h * zd[mu]);
      rc[rec::AL + mu] = al;
      rc[rec::BE + mu] = -w1 * d1h;
      rc[rec::GW1 + mu] = ge * h - d1h * zd[mu];
    }
#pragma unroll
    for (int v = 0; v < ND; ++v) {
      Rq[v] *= qs[v];
      rc[rec::QT + v] = qs[v] * A.q[v];
      rc[rec::U + v] = u[v];
    }
    rc[rec::GB1] = -ge;
#pragma unroll
    for (int nn = 0; nn < NR; ++nn) {
      rc[rec::RHO + nn] = ge * A.Fp[nn] - Rq[nn];
      rc[rec::SIG + nn] = -A.Fp[nn];
    }
#pragma unroll
    for (int nn = 0; nn < NA; ++nn)
#pragma unroll
      for (int c = 0; c < NLM; ++c) {
        const int v = NR + 2 * nn + l_of(c) - 1;
        rc[rec::KAP + nn * NLM + c] = 2.f * (ge * A.Fp[v] - Rq[v]) * A.s[nn][c] - 2.f * A.Fp[v] * ds[nn][c];
        rc[rec::LAM + nn * NLM + c] = -2.f * A.Fp[v] * A.s[nn][c];
      }
#pragma unroll
    for (int k = 0; k < KB; ++k) {
      rc[rec::Q + k] = Qa[k];
      rc[rec::DQ + k] = dQa[k];
    }
#pragma unroll
    for (int c = 0; c < NSB; ++c) {
      rc[rec::S + c] = Sa[c];
      rc[rec::DS + c] = dS[(size_t)a * NSB + c];
    }
  } else {
    for (int c = 0; c < GREC; ++c) rc[c] = 0.f;
  }
  __syncthreads();
  for (int p = t; p < NPAR; p += GRAD_BLOCK) {
    float acc = 0.f;
    if (p < OFF_CA) {
      const int nn = (p - OFF_CR) / KB, k = (p - OFF_CR) % KB;
      for (int b = 0; b < GRAD_BLOCK; ++b) {
        const float *r = R + b * GREC;
        acc = fmaf(r[rec::RHO + nn], r[rec::Q + k], fmaf(r[rec::SIG + nn], r[rec::DQ + k], acc));
      }
    } else if (p < OFF_W0) {
      const int nn = (p - OFF_CA) / KB, k = (p - OFF_CA) % KB;
      for (int b = 0; b < GRAD_BLOCK; ++b) {
        const float *r = R + b * GREC;
#pragma unroll
        for (int c = 0; c < NLM; ++c)
          acc = fmaf(r[rec::KAP + nn * NLM + c], r[rec::S + k * NLM + c],
                     fmaf(r[rec::LAM + nn * NLM + c], r[rec::DS + k * NLM + c], acc));
      }
    } else if (p < OFF_B0) {
      const int mu = (p - OFF_W0) / ND, v = (p - OFF_W0) % ND;
      for (int b = 0; b < GRAD_BLOCK; ++b) {
        const float *r = R + b * GREC;
        acc = fmaf(r[rec::AL + mu], r[rec::QT + v], fmaf(r[rec::BE + mu], r[rec::U + v], acc));
      }
    } else if (p < OFF_W1) {
      for (int b = 0; b < GRAD_BLOCK; ++b) acc -= R[b * GREC + rec::AL + (p - OFF_B0)];
    } else if (p < OFF_B1) {
      for (int b = 0; b < GRAD_BLOCK; ++b) acc += R[b * GREC + rec::GW1 + (p - OFF_W1)];
    } else {
      for (int b = 0; b < GRAD_BLOCK; ++b) acc += R[b * GREC + rec::GB1];
    }
    part[(size_t)blockIdx.x * NPAR + p] = acc;
  }
}

__global__ void k_st_grad_reduce(int nblk, const float *__restrict__ part, float *__restrict__ grad) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= NPAR) return;
  double t = 0.0;
  for (int b = 0; b < nblk; ++b) t += (double)part[(size_t)b * NPAR + p];
  grad[p] = (float)t;
}

__global__ void k_st_adam(int npar, float *__restrict__ theta, const float *__restrict__ grad, float *__restrict__ m,
                          float *__restrict__ v, float lr, float b1, float b2, float eps, float c1, float c2) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= npar) return;
  const float g = grad[p];
  const float mp = b1 * m[p] + (1.f - b1) * g;
  const float vp = b2 * v[p] + (1.f - b2) * g * g;
  m[p] = mp;
  v[p] = vp;
  theta[p] -= lr * (mp / c1) / (sqrtf(vp / c2) + eps);
}

constexpr size_t GRAD_SMEM = (NPAR + 16 + (size_t)GRAD_BLOCK * GREC) * sizeof(float);

int blocks_of(int n, int b) { return (n + b - 1) / b; }

}  // namespace
}  // namespace nep

using namespace nep;

extern "C" {

int st_pairs(int n, const float *pos, const int *start, const float *boxes, st_cutoffs rc, int cap, int *nbr,
             float *dvec, int *nnum, int *status, void *stream) {
  if (n <= 0) return 0;
  k_st_pairs<<<blocks_of(n, BLOCK), BLOCK, 0, (cudaStream_t)stream>>>(
      n, reinterpret_cast<const float4 *>(pos), start, boxes, rc.rc_R * rc.rc_R, cap, nbr,
      reinterpret_cast<float4 *>(dvec), nnum, status);
  return (int)cudaGetLastError();
}

int st_basis(int a0, int a1, int n, int cap, const int *nbr, const float *dvec, const int *nnum, st_cutoffs rc,
             float *Q, float *S, void *stream) {
  (void)cap; (void)nbr;
  if (a1 <= a0) return 0;
  k_st_basis<<<blocks_of(a1 - a0, BLOCK), BLOCK, 0, (cudaStream_t)stream>>>(
      a0, a1, n, nnum, reinterpret_cast<const float4 *>(dvec), cut_of(rc), Q, S);
  return (int)cudaGetLastError();
}

int st_forward(int a0, int a1, const float *theta, const float *q_scale, const float *Q, const float *S, float *U,
               float *G, float *q_out, void *stream) {
  if (a1 <= a0) return 0;
  k_st_forward<<<blocks_of(a1 - a0, BLOCK), BLOCK, 0, (cudaStream_t)stream>>>(a0, a1, theta, q_scale, Q, S, U, G,
                                                                              q_out);
  return (int)cudaGetLastError();
}

int st_energy(int s0, int s1, const int *start, const float *U, double *E, void *stream) {
  if (s1 <= s0) return 0;
  const int warps = s1 - s0;
  k_st_energy<<<blocks_of(warps * 32, BLOCK), BLOCK, 0, (cudaStream_t)stream>>>(s0, s1, start, U, E);
  return (int)cudaGetLastError();
}

int st_force(int a0, int a1, int n, int cap, const int *nbr, const float *dvec, const int *nnum, st_cutoffs rc,
             const float *theta, const float *G, float *F, void *stream) {
  (void)cap;
  if (a1 <= a0) return 0;
  k_st_force<<<blocks_of(a1 - a0, BLOCK), BLOCK, 0, (cudaStream_t)stream>>>(
      a0, a1, n, nbr, reinterpret_cast<const float4 *>(dvec), nnum, cut_of(rc), theta, G, F);
  return (int)cudaGetLastError();
}

int st_jvp(int a0, int a1, int n, int cap, const int *nbr, const float *dvec, const int *nnum, st_cutoffs rc,
           const float *v, float *dQ, float *dS, void *stream) {
  (void)cap;
  if (a1 <= a0) return 0;
  k_st_jvp<<<blocks_of(a1 - a0, BLOCK), BLOCK, 0, (cudaStream_t)stream>>>(
      a0, a1, n, nbr, reinterpret_cast<const float4 *>(dvec), nnum, cut_of(rc), v, dQ, dS);
  return (int)cudaGetLastError();
}

int64_t st_grad_scratch(int a0, int a1) {
  return a1 > a0 ? (int64_t)blocks_of(a1 - a0, GRAD_BLOCK) * NPAR : 0;
}

int st_grad(int a0, int a1, const float *theta, const float *q_scale, const float *pos, const float *Q,
            const float *S, const float *dQ, const float *dS, const double *gE, float *scratch, float *grad,
            void *stream) {
  cudaStream_t st = (cudaStream_t)stream;
  if (a1 <= a0) return (int)cudaMemsetAsync(grad, 0, NPAR * sizeof(float), st);
  static bool attr = false;
  if (!attr) {
    const cudaError_t e =
        cudaFuncSetAttribute(k_st_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)GRAD_SMEM);
    if (e != cudaSuccess) return (int)e;
    attr = true;
  }
  const int nblk = blocks_of(a1 - a0, GRAD_BLOCK);
  k_st_grad<<<nblk, GRAD_BLOCK, GRAD_SMEM, st>>>(a0, a1, theta, q_scale, reinterpret_cast<const float4 *>(pos), Q, S,
                                                 dQ, dS, gE, scratch);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return (int)e;
  k_st_grad_reduce<<<blocks_of(NPAR, BLOCK), BLOCK, 0, st>>>(nblk, scratch, grad);
  return (int)cudaGetLastError();
}

int st_adam(int npar, float *theta, const float *grad, float *m, float *v, float lr, float beta1, float beta2,
            float eps, int t, void *stream) {
  if (npar <= 0 || t < 1) return (int)cudaErrorInvalidValue;
  const float c1 = 1.f - powf(beta1, (float)t), c2 = 1.f - powf(beta2, (float)t);
  k_st_adam<<<blocks_of(npar, BLOCK), BLOCK, 0, (cudaStream_t)stream>>>(npar, theta, grad, m, v, lr, beta1, beta2,
                                                                       eps, c1, c2);
  return (int)cudaGetLastError();
}

}  // extern "C"
