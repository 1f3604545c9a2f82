// nep_descriptor.cuh -- per-atom descriptor pieces shared by the float32 and the mixed-precision
// descriptor kernels: the neighbour walk that accumulates the radial sums q_n, the LJ energy and the
// angular sums s_nlm (Section III.B; the geometry of each neighbour is computed once and reused for all
// channels, Algorithm 1 with one tile), the rotation invariants q_nl and q4_n, and the adjoint row
// G_nlm = dU/ds_nlm built from the network gradient.
#pragma once

#include <cuda_fp16.h>

#include "nep_common.cuh"
#include "nep_tc.cuh"

namespace nep {

// Adjoint rows are stored as float32 (plain form) or float16 (mixed-precision form); the force
// kernel reads them W values per 16-byte load.
template <class GT>
struct GTraits;
template <>
struct GTraits<float> {
  static constexpr int W = 4;
};
template <>
struct GTraits<__half> {
  static constexpr int W = 8;
};

__device__ __forceinline__ void load_vec(const float *p, float (&v)[4]) {
  const float4 t = __ldg(reinterpret_cast<const float4 *>(p));
  v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
}
__device__ __forceinline__ void load_vec(const __half *p, float (&v)[8]) {
  const uint4 t = __ldg(reinterpret_cast<const uint4 *>(p));
  const uint32_t w[4] = {t.x, t.y, t.z, t.w};
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const float2 f = __half22float2(*reinterpret_cast<const __half2 *>(&w[k]));
    v[2 * k] = f.x; v[2 * k + 1] = f.y;
  }
}
// The 8 values at the tail of a row (dU/dq_n of the radial descriptors and padding).
template <class GT>
__device__ __forceinline__ void load_tail8(const GT *row, int off, float (&v)[8]) {
  constexpr int W = GTraits<GT>::W;
#pragma unroll
  for (int b = 0; b < 8; b += W) {
    float t[W];
    load_vec(row + off + b, t);
#pragma unroll
    for (int k = 0; k < W; ++k) v[b + k] = t[k];
  }
}

// Per-atom fallback to another model (the teacher) for atoms whose scaled descriptors leave a box:
// an atom is flagged when some q~_nu = q_scale_nu q_nu lies outside [lo_nu, hi_nu].  Flagged atoms
// get a zero adjoint row and no site energy from this model; their indices are appended to `list`
// (order of arrival: the consumers only use integer atomics, so results do not depend on it).
struct Fallback {
  int on;
  int cap;                 // capacity of list
  int *list, *count;       // flagged atoms (cell-sorted indices), number flagged
  float lo[16], hi[16];
};

template <class S>
__device__ __forceinline__ bool out_of_range(const Fallback &fb, const Model<S> &P, const float (&q)[S::NDES]) {
  bool out = false;
  if constexpr (S::NDES <= 16) {       // the range box holds up to 16 descriptors (the student's 12)
#pragma unroll
    for (int v = 0; v < S::NDES; ++v) {
      const float t = q[v] * P.qs[v];
      out |= (t < fb.lo[v]) | (t > fb.hi[v]);
    }
  }
  return out;
}

// Append atom i to the fallback list (status bit ST_FB_OVERFLOW when the list is full).
__device__ __forceinline__ void flag_atom(const Fallback &fb, int i, int *status) {
  const int slot = atomicAdd(fb.count, 1);
  if (slot < fb.cap) fb.list[slot] = i;
  else atomicOr(status, ST_FB_OVERFLOW);
}

template <class S>
struct AtomSums {
  float QR[S::KR];        // radial basis sums sum_j f_k(r_ij); q_n = sum_k cR_nk QR_k
  static_assert(S::KR <= 8, "the radial adjoint in basis space lives in the 8-element row tail");
  float s[S::NA][S::NLM];
  float elj;
  int nrad, nang, nact, cnt;
};

// Walk atom i's full neighbour row and accumulate q_n, s_nlm and the LJ energy.  REC: every active pair
// is also recorded as (dx, dy, dz, j) at rec[off + slot * BLOCK], angular pairs from slot 0 up and the
// other active pairs from slot pmax - 1 down (the layout of accumulate_atom_tm's records).
// UN: the sums over the polynomials Ph_lm without their constant factors (s' = s / hnorm, harmonics_p).
template <class S, int DE, int DP, int BLOCK, bool REC = false, bool UN = false>
__device__ __forceinline__ void accumulate_atom(const Model<S> &P, const float4 *shift, int i, int n,
                                                const float4 *__restrict__ pos, const int32_t *__restrict__ nbr,
                                                RowSpan sp, uint32_t *ring_e, float4 *ring_p, AtomSums<S> &A,
                                                float4 *__restrict__ rec = nullptr, unsigned off = 0, int pmax = 0) {
  const int cnt = sp.c;
  const float4 pi = pos[i];
#pragma unroll
  for (int k = 0; k < S::KR; ++k) A.QR[k] = 0.f;
#pragma unroll
  for (int a = 0; a < S::NA; ++a)
#pragma unroll
    for (int c = 0; c < S::NLM; ++c) A.s[a][c] = 0.f;
  A.elj = 0.f;
  A.nrad = 0; A.nang = 0; A.nact = 0; A.cnt = cnt;
  NbrPipe<DE, DP, BLOCK> pipe;
  pipe.start(ring_e, ring_p, nbr + i, (size_t)n, pos, sp);
  for (int k = 0; k < cnt; ++k) {
    uint32_t e;
    float4 pj;
    pipe.get(k, e, pj);
    const float4 o = shift[e >> J_BITS];
    const float dx = pj.x - pi.x + o.x, dy = pj.y - pi.y + o.y, dz = pj.z - pi.z + o.z;
    const float r2 = dx * dx + dy * dy + dz * dz;
    if (r2 >= P.rmax2) continue;
    if constexpr (REC) {
      const int slot = r2 < P.rcA2 ? A.nang : pmax - 1 - (A.nact - A.nang);
      rec[off + (unsigned)slot * BLOCK] = make_float4(dx, dy, dz, __int_as_float((int)(e & J_MASK)));
    }
    ++A.nact;
    const float ir = rsqrtf(r2);
    const float r = r2 * ir;
    if (r2 < P.rcR2) {
      // sum h T_k here (T_0 = 1: QR[0] collects sum h); sum f_k = sum h T_k + sum h after the walk
      float h, T[S::KR];
      cheb_t<S::KR>(r, P.inv_rcR, h, T);
#pragma unroll
      for (int k = 0; k < S::KR; ++k) A.QR[k] = fmaf(h, T[k], A.QR[k]);
      ++A.nrad;
    }
    if (P.lj_on != 0.f && r2 < P.lj_rc2) {
      float el, dl;
      lj_pair<S>(P, r2, r, ir, el, dl);
      A.elj = fmaf(0.5f, el, A.elj);
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
      float Y[S::NLM];
      if constexpr (UN) harmonics_p<S::NLM>(dx * ir, dy * ir, dz * ir, Y);
      else harmonics<S::NLM>(dx * ir, dy * ir, dz * ir, Y);
#pragma unroll
      for (int a = 0; a < S::NA; ++a)
#pragma unroll
        for (int c = 0; c < S::NLM; ++c) A.s[a][c] = fmaf(g[a], Y[c], A.s[a][c]);
      ++A.nang;
    }
  }
  pipe.finish();
  const float hsum = A.QR[0];
#pragma unroll
  for (int k = 0; k < S::KR; ++k) A.QR[k] += hsum;
}
template <class S, int DE, int DP, int BLOCK>
__device__ __forceinline__ void accumulate_atom(const Model<S> &P, const float4 *shift, int i, int n,
                                                const float4 *__restrict__ pos, const int32_t *__restrict__ nbr,
                                                int cnt, uint32_t *ring_e, float4 *ring_p, AtomSums<S> &A) {
  accumulate_atom<S, DE, DP, BLOCK>(P, shift, i, n, pos, nbr, RowSpan{cnt, cnt, 0}, ring_e, ring_p, A);
}

// Traceless 4-body tensors T_n rebuilt from the l = 2 sums (components 3..7 = m -2..2).
template <class S>
struct FourBody {
  float xx[S::NA], yy[S::NA], zz[S::NA], xy[S::NA], yz[S::NA], xz[S::NA];
};

// Traceless T_n from the l = 2 sums s2[n][m] (components 3..7 of s_nl m, m = -2..2) and the 4-body
// descriptors q4_n = tr(T_n^3) = 3 det T_n, written to q[NR + NA LMAX + n].
template <class S>
__device__ __forceinline__ void fourbody_tensors(const float (&s2)[S::NA][5], FourBody<S> &T, float (&q)[S::NDES]) {
  const float i3 = 0.57735026918962576f, third = 1.f / 3.f;
#pragma unroll
  for (int a = 0; a < S::NA; ++a) {
    T.xy[a] = s2[a][0] * i3;
    T.yz[a] = s2[a][1] * i3;
    T.xz[a] = s2[a][3] * i3;
    T.xx[a] = s2[a][4] * i3 - s2[a][2] * third;
    T.yy[a] = -s2[a][4] * i3 - s2[a][2] * third;
    T.zz[a] = 2.f * s2[a][2] * third;
    const float det = T.xx[a] * (T.yy[a] * T.zz[a] - T.yz[a] * T.yz[a]) -
                      T.xy[a] * (T.xy[a] * T.zz[a] - T.yz[a] * T.xz[a]) +
                      T.xz[a] * (T.xy[a] * T.yz[a] - T.yy[a] * T.xz[a]);
    q[S::NR + S::NA * S::LMAX + a] = 3.f * det;
  }
}

// Descriptors [q_n | q_nl (n-major, l = 1..LMAX) | q4_n = tr(T_n^3) = 3 det T_n (teacher shape only)].
// UN: A holds s'_nlm (accumulate_atom<.., UN>), scaled by hnorm(lm) here.
template <class S, bool UN = false>
__device__ __forceinline__ void descriptors_of(const Model<S> &P, const AtomSums<S> &A, float (&q)[S::NDES],
                                               FourBody<S> &T) {
#pragma unroll
  for (int a = 0; a < S::NR; ++a) {
    float t = 0.f;
#pragma unroll
    for (int k = 0; k < S::KR; ++k) t = fmaf(P.cR[a][k], A.QR[k], t);
    q[a] = t;
  }
#pragma unroll
  for (int a = 0; a < S::NA; ++a) {
#pragma unroll
    for (int l = 1; l <= S::LMAX; ++l) {
      float t = 0.f;
#pragma unroll
      for (int c = l * l - 1; c < (l + 1) * (l + 1) - 1; ++c) {
        const float sc = UN ? hnorm(c) * A.s[a][c] : A.s[a][c];
        t = fmaf(sc, sc, t);
      }
      q[S::NR + a * S::LMAX + (l - 1)] = t;
    }
  }
  if constexpr (S::FOURBODY) {
    float s2[S::NA][5];
#pragma unroll
    for (int a = 0; a < S::NA; ++a)
#pragma unroll
      for (int m = 0; m < 5; ++m) s2[a][m] = UN ? hnorm(3 + m) * A.s[a][3 + m] : A.s[a][3 + m];
    fourbody_tensors<S>(s2, T, q);
  }
}

// The one-hidden-layer network (Section III.B equation): U = sum_mu w1_mu tanh(sum_nu W0_mu,nu q~_nu -
// b0_mu) - b1 with q~ = q_scale q; returns U and Fp_nu = dU/dq_nu (zero for an atom flagged for the
// fallback model, whose site energy comes from the other model).
template <class S>
__device__ __forceinline__ float network(const Model<S> &P, const float (&q)[S::NDES], bool flagged,
                                         float (&Fp)[S::NDES]) {
  float qt[S::NDES], dq[S::NDES];
#pragma unroll
  for (int v = 0; v < S::NDES; ++v) { qt[v] = q[v] * P.qs[v]; dq[v] = 0.f; }
  float U = -P.b1;
  // The teacher's 30 x 30 network, fully unrolled, is ~2k instructions of straight-line code that the
  // row-walk loops share the instruction cache with; one neuron per iteration (weights read from the
  // constant bank with a register offset) measured 2 % faster in the fused kernel.
  constexpr int UNROLL = S::NNEU * S::NDES > 400 ? 1 : S::NNEU;
#pragma unroll UNROLL
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
#pragma unroll
  for (int v = 0; v < S::NDES; ++v) Fp[v] = flagged ? 0.f : dq[v] * P.qs[v];
  return U;
}

// Radial adjoint in basis space, stored in the row tail: tail_k = dU/dQR_k = sum_n Fp_n cR_nk, so the
// force kernel contracts it directly with the basis derivatives f_k'(r) of each pair.
template <class S>
__device__ __forceinline__ void radial_tail(const Model<S> &P, const float (&Fp)[S::NDES], float (&tail)[8]) {
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    float t = 0.f;
    if (k < S::KR) {
#pragma unroll
      for (int a = 0; a < S::NR; ++a) t = fmaf(Fp[a], P.cR[a][k], t);
    }
    tail[k] = t;
  }
}

// The radial tail as the fused kernels' force pass contracts it with the Chebyshev factors (cheb_td):
// tail_0 + sum_k tail_k in place of tail_0 (the T_0 = 1 term then also carries sum_k tail_k dh).
__device__ __forceinline__ void radial_tail_td(float (&tail)[8]) {
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < 8; ++k) s += tail[k];
  tail[0] += s;
}

// 4-body part of the adjoint of channel a for the l = 2 components 3..7, per unit dU/dq4_a:
// d tr(T^3)/d s_m = 3 (T^2) : dT/ds_m.
template <class S>
__device__ __forceinline__ void fourbody_adjoint(int a, const FourBody<S> &T, float (&g4)[5]) {
  const float Mxx = T.xx[a] * T.xx[a] + T.xy[a] * T.xy[a] + T.xz[a] * T.xz[a];
  const float Myy = T.xy[a] * T.xy[a] + T.yy[a] * T.yy[a] + T.yz[a] * T.yz[a];
  const float Mzz = T.xz[a] * T.xz[a] + T.yz[a] * T.yz[a] + T.zz[a] * T.zz[a];
  const float Mxy = T.xx[a] * T.xy[a] + T.xy[a] * T.yy[a] + T.xz[a] * T.yz[a];
  const float Myz = T.xy[a] * T.xz[a] + T.yy[a] * T.yz[a] + T.yz[a] * T.zz[a];
  const float Mxz = T.xx[a] * T.xz[a] + T.xy[a] * T.yz[a] + T.xz[a] * T.zz[a];
  const float s3 = 1.7320508075688772f;
  g4[0] = 2.f * s3 * Mxy;
  g4[1] = 2.f * s3 * Myz;
  g4[2] = 2.f * Mzz - Mxx - Myy;
  g4[3] = 2.f * s3 * Mxz;
  g4[4] = s3 * (Mxx - Myy);
}

// Adjoint of channel a: gl[c] = dU/ds_{a,c} = 2 Fp_{a,l(c)} s_{a,c} (+ 4-body gradient for l = 2:
// d tr(T^3)/d s_m = 3 (T^2) : dT/ds_m).
// UN: A holds s'_nlm and the row is G'_nlm = hnorm(lm) G_nlm (adjoint_chunk).
template <class S, bool UN = false>
__device__ __forceinline__ void adjoint_channel(int a, const AtomSums<S> &A, const FourBody<S> &T,
                                                const float (&Fp)[S::NDES], float (&gl)[S::NLM]) {
#pragma unroll
  for (int c = 0; c < S::NLM; ++c) {
    const float h = UN ? hnorm(c) : 1.f;
    gl[c] = (2.f * h * h) * Fp[S::NR + a * S::LMAX + lm_l(c) - 1] * A.s[a][c];
  }
  if constexpr (S::FOURBODY) {
    const float f4 = Fp[S::NR + S::NA * S::LMAX + a];
    float g4[5];
    fourbody_adjoint<S>(a, T, g4);
#pragma unroll
    for (int m = 0; m < 5; ++m) gl[3 + m] = fmaf(UN ? hnorm(3 + m) * f4 : f4, g4[m], gl[3 + m]);
  }
}

// ---------------------------------------------------------------------------------------------------
// Teacher shape with the angular sums s_nlm of the first NT channels in tensor memory (TMEM) instead
// of registers (NT = 5: all 120; NT = 4: 96, the fifth channel's 24 in registers), in the chunked layout
// of tm_col (chunk k = components 4k..4k+3 of every channel: one x16 access for channels 0..3 and one x4
// access for channel 4), which the force pass's adjoint row shares.  All TMEM accesses are
// warp-collective, so the neighbour walk runs to the warp's longest row (threads past their own row, or
// past the last atom, idle with a predicate) and the angular update is made by whole warps, lanes
// without an angular pair adding g = 0.
constexpr int TMEM_W = 4;

// The sums of the channels kept in registers (NA - NT of them; one unused row when NT = NA).
template <class S, int NT>
struct RegSums {
  float s[S::NA > NT ? S::NA - NT : 1][S::NLM];
};

// Chunk k of the NT TMEM channels into v[0..NT-1] (one statement, waited for).
template <class S, int NT>
__device__ __forceinline__ void tm_load(uint32_t trow, int k, float (&v)[S::NA][TMEM_W]) {
  if constexpr (NT == 5) {
    tmem_ld_chunk<S::NLM>(trow, k, v);
  } else {
    float t[4][TMEM_W];
    tmem_ld_chunk<S::NLM>(trow, k, t);
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int c = 0; c < TMEM_W; ++c) v[a][c] = t[a][c];
  }
}
template <class S, int NT>
__device__ __forceinline__ void tm_store(uint32_t trow, int k, const float (&v)[S::NA][TMEM_W]) {
  if constexpr (NT == 5) {
    tmem_st_chunk<S::NLM, 5>(trow, k, v);
  } else {
    float t[4][TMEM_W];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int c = 0; c < TMEM_W; ++c) t[a][c] = v[a][c];
    tmem_st_chunk<S::NLM, 4>(trow, k, t);
  }
}

// Zero the sums, then walk atom ii's row (cnt entries; cnt = 0 for threads past the last atom):
// radial basis sums QR and the LJ energy in registers, s_nlm in TMEM (channels < NT) and R.
// The accumulations run in float2 pairs (two basis functions, or two (l, m) components, per instruction).
// REC: every active pair is also recorded as (dx, dy, dz, j) at rec[off + slot * BLOCK] (off: this
// thread's column of a [pmax][BLOCK] array): angular pairs (r < rc_A) from
// slot 0 up in walk order, the other active pairs from slot pmax - 1 down (pmax >= the row length, so
// the two never meet).
template <class S, int NT, int DE, int DP, int BLOCK, bool REC = false, bool UN = false>
__device__ __forceinline__ void accumulate_atom_tm(const Model<S> &P, const float4 *shift, uint32_t trow, int ii,
                                                   int n, const float4 *__restrict__ pos,
                                                   const int32_t *__restrict__ nbr, RowSpan sp, uint32_t *ring_e,
                                                   float4 *ring_p, float (&QR)[S::KR], RegSums<S, NT> &R,
                                                   float &elj, int &nrad, int &nang, int &nact,
                                                   float4 *__restrict__ rec = nullptr, unsigned off = 0, int pmax = 0) {
  static_assert(S::NA == 5 && S::NLM == 24 && (NT == 4 || NT == 5), "teacher shape");
  static_assert(S::KR % 2 == 0 && S::KA % 2 == 0, "basis sizes are paired");
  constexpr int W = TMEM_W;
  constexpr int NC = S::NLM / W;
  {
    float z[S::NA][W];
#pragma unroll
    for (int a = 0; a < S::NA; ++a)
#pragma unroll
      for (int c = 0; c < W; ++c) z[a][c] = 0.f;
#pragma unroll
    for (int k = 0; k < NC; ++k) tm_store<S, NT>(trow, k, z);
    tmem_wait_st();
  }
#pragma unroll
  for (int a = NT; a < S::NA; ++a)
#pragma unroll
    for (int c = 0; c < S::NLM; ++c) R.s[a - NT][c] = 0.f;
  float2 QR2[S::KR / 2];
#pragma unroll
  for (int k = 0; k < S::KR / 2; ++k) QR2[k] = bc2(0.f);
  elj = 0.f;
  nrad = 0; nang = 0; nact = 0;
  const float4 pi = pos[ii];
  const int cnt = sp.c;
  NbrPipe<DE, DP, BLOCK> pipe;
  pipe.start(ring_e, ring_p, nbr + ii, (size_t)n, pos, sp);
  const int trip = __reduce_max_sync(0xffffffffu, cnt);
  for (int k = 0; k < trip; ++k) {
    const bool valid = k < cnt;
    uint32_t e;
    float4 pj;
    // past the end of the row the ring slots are stale: act below is false for them, and e = 0 keeps
    // the shift-table index in range
    pipe.get(k, e, pj);
    e = valid ? e : 0u;
    const float4 o = shift[e >> J_BITS];
    const float dx = pj.x - pi.x + o.x, dy = pj.y - pi.y + o.y, dz = pj.z - pi.z + o.z;
    const float r2 = dx * dx + dy * dy + dz * dz;
    const bool act = valid && r2 < P.rmax2;
    const float ir = rsqrtf(r2);
    const float r = r2 * ir;
    if (act) {
      if constexpr (REC) {
        const int slot = r2 < P.rcA2 ? nang : pmax - 1 - (nact - nang);
        rec[off + (unsigned)slot * BLOCK] = make_float4(dx, dy, dz, __int_as_float((int)(e & J_MASK)));
      }
      ++nact;
      if (r2 < P.rcR2) {
        // sum h T_k here (T_0 = 1, so QR2[0].x collects sum h); sum f_k = sum h T_k + sum h below
        float h, T[S::KR];
        cheb_t<S::KR>(r, P.inv_rcR, h, T);
        const float2 h2 = bc2(h);
#pragma unroll
        for (int b = 0; b < S::KR / 2; ++b) QR2[b] = fma2(h2, pr(T[2 * b], T[2 * b + 1]), QR2[b]);
        ++nrad;
      }
      if (P.lj_on != 0.f && r2 < P.lj_rc2) {
        float el, dl;
        lj_pair<S>(P, r2, r, ir, el, dl);
        elj = fmaf(0.5f, el, elj);
      }
    }
    const bool ang = act && r2 < P.rcA2;
    if (__any_sync(0xffffffffu, ang)) {
      __syncwarp();
      const float ar = ang ? r : 1.f;
      const float ux = ang ? dx * ir : 1.f, uy = ang ? dy * ir : 0.f, uz = ang ? dz * ir : 0.f;
      float f[S::KA];
      cheb_basis<S::KA>(ar, P.inv_rcA, f);
      float g[S::NA];
#pragma unroll
      for (int a = 0; a < S::NA; ++a) {
        const float t = dot_pairs<S::KA>(P.cA[a], f);
        g[a] = ang ? t : 0.f;
      }
      // UN: the polynomials Ph_lm chunk by chunk (fewer live registers than 24 values); all channels in TMEM
      static_assert(!UN || NT == S::NA, "register-resident channels take the normalised harmonics");
      float Y[S::NLM];
      if constexpr (!UN) harmonics<S::NLM>(ux, uy, uz, Y);
#pragma unroll
      for (int k = 0; k < NC; ++k) {
        float sv[S::NA][W];
        tm_load<S, NT>(trow, k, sv);
        float2 y01, y23;
        if constexpr (UN) {
          y01 = pr(harmonic_p(W * k, ux, uy, uz), harmonic_p(W * k + 1, ux, uy, uz));
          y23 = pr(harmonic_p(W * k + 2, ux, uy, uz), harmonic_p(W * k + 3, ux, uy, uz));
        } else {
          y01 = pr(Y[W * k], Y[W * k + 1]);
          y23 = pr(Y[W * k + 2], Y[W * k + 3]);
        }
#pragma unroll
        for (int a = 0; a < NT; ++a) {
          const float2 g2 = bc2(g[a]);
          const float2 lo = fma2(g2, y01, pr(sv[a][0], sv[a][1]));
          const float2 hi = fma2(g2, y23, pr(sv[a][2], sv[a][3]));
          sv[a][0] = lo.x; sv[a][1] = lo.y; sv[a][2] = hi.x; sv[a][3] = hi.y;
        }
        tm_store<S, NT>(trow, k, sv);
      }
      // register-resident channels: scalar (paired updates would pin the sums to aligned register pairs)
#pragma unroll
      for (int a = NT; a < S::NA; ++a)
#pragma unroll
        for (int c = 0; c < S::NLM; ++c) R.s[a - NT][c] = fmaf(g[a], Y[c], R.s[a - NT][c]);
      tmem_wait_st();
      if (ang) ++nang;
    }
  }
  pipe.finish();
  const float hsum = QR2[0].x;
#pragma unroll
  for (int k = 0; k < S::KR / 2; ++k) { QR[2 * k] = QR2[k].x + hsum; QR[2 * k + 1] = QR2[k].y + hsum; }
}

// The sums of chunk k (components 4k..4k+3) of every channel: TMEM for a < NT, registers after.
template <class S, int NT>
__device__ __forceinline__ void sums_chunk(uint32_t trow, int k, const RegSums<S, NT> &R, float (&sv)[S::NA][TMEM_W]) {
  tm_load<S, NT>(trow, k, sv);
#pragma unroll
  for (int a = NT; a < S::NA; ++a)
#pragma unroll
    for (int cc = 0; cc < TMEM_W; ++cc) sv[a][cc] = R.s[a < NT ? 0 : a - NT][TMEM_W * k + cc];
}

// Descriptors from the radial basis sums and the sums s_nlm (q_nl = sum_m s_nlm^2, 4-body from the
// l = 2 sums), as descriptors_of.
// UN: sums over Ph_lm (accumulate_atom_tm), scaled by hnorm(lm) here.
template <class S, int NT, bool UN = false>
__device__ __forceinline__ void descriptors_tm(const Model<S> &P, uint32_t trow, const float (&QR)[S::KR],
                                               const RegSums<S, NT> &R, float (&q)[S::NDES], FourBody<S> &T) {
  constexpr int W = TMEM_W;
#pragma unroll
  for (int a = 0; a < S::NR; ++a) {
    float t = 0.f;
#pragma unroll
    for (int b = 0; b < S::KR; ++b) t = fmaf(P.cR[a][b], QR[b], t);
    q[a] = t;
  }
#pragma unroll
  for (int v = S::NR; v < S::NR + S::NA * S::LMAX; ++v) q[v] = 0.f;
  float s2[S::NA][5];
#pragma unroll
  for (int k = 0; k < S::NLM / W; ++k) {
    float sv[S::NA][W];
    sums_chunk<S, NT>(trow, k, R, sv);
#pragma unroll
    for (int a = 0; a < S::NA; ++a)
#pragma unroll
      for (int cc = 0; cc < W; ++cc) {
        const int lm = W * k + cc;
        if constexpr (UN) sv[a][cc] *= hnorm(lm);
        float &ql = q[S::NR + a * S::LMAX + lm_l(lm) - 1];
        ql = fmaf(sv[a][cc], sv[a][cc], ql);
        if (lm >= 3 && lm < 8) s2[a][lm - 3] = sv[a][cc];
      }
  }
  fourbody_tensors<S>(s2, T, q);
}

// 4-body adjoint factors g4[a] = 3 (T_a^2) : dT_a/ds_m of every channel, with the tensors T_a rebuilt
// from the l = 2 sums (components 3..7: chunk 0 holds component 3, chunk 1 components 4..7), so that
// T need not stay live across the network.
template <class S, int NT, bool UN = false>
__device__ __forceinline__ void fourbody_adjoint_tm(uint32_t trow, const RegSums<S, NT> &R, float (&g4)[S::NA][5]) {
  static_assert(S::FOURBODY && S::NLM == 24, "teacher shape");
  float c0[S::NA][TMEM_W], c1[S::NA][TMEM_W];
  sums_chunk<S, NT>(trow, 0, R, c0);
  sums_chunk<S, NT>(trow, 1, R, c1);
  float s2[S::NA][5];
#pragma unroll
  for (int a = 0; a < S::NA; ++a) {
    s2[a][0] = c0[a][3];
#pragma unroll
    for (int m = 1; m < 5; ++m) s2[a][m] = c1[a][m - 1];
    if constexpr (UN) {
#pragma unroll
      for (int m = 0; m < 5; ++m) s2[a][m] *= hnorm(3 + m);
    }
  }
  FourBody<S> T;
  float q[S::NDES];
  fourbody_tensors<S>(s2, T, q);
#pragma unroll
  for (int a = 0; a < S::NA; ++a) fourbody_adjoint<S>(a, T, g4[a]);
}

// The adjoint of components c..c+3 of channel a, gl = 2 Fp_{a,l} s + (4-body terms for l = 2), as
// adjoint_channel; g4 = fourbody_adjoint of channel a.
// UN: sv holds s'_nlm (sums over Ph_lm) and the row is G'_nlm = hnorm(lm) G_nlm, the weights of Ph_lm:
// G' = 2 hnorm^2 Fp s' + hnorm f4 g4.
template <class S, bool UN = false>
__device__ __forceinline__ void adjoint_chunk(int a, int c, const float (&sv)[TMEM_W], const float (&g4)[5],
                                              const float (&Fp)[S::NDES], float (&gl)[TMEM_W]) {
#pragma unroll
  for (int cc = 0; cc < TMEM_W; ++cc) {
    const int lm = c + cc;
    const float h = UN ? hnorm(lm) : 1.f;
    gl[cc] = (2.f * h * h) * Fp[S::NR + a * S::LMAX + lm_l(lm) - 1] * sv[cc];
    if (S::FOURBODY && lm >= 3 && lm < 8)
      gl[cc] = fmaf(UN ? h * Fp[S::NR + S::NA * S::LMAX + a] : Fp[S::NR + S::NA * S::LMAX + a], g4[lm - 3], gl[cc]);
  }
}

// ---------------------------------------------------------------------------------------------------
// The network with W0 staged in shared memory: rows of S::NDES weights padded to NDP (a multiple of 4)
// so that each is read with 16-byte broadcast loads (all lanes read the same address), and the forward
// and backward products of a neuron run in float2 pairs over the descriptors.  Same result as network()
// up to the order of the additions.
template <class S>
struct NetSmem {
  static constexpr int NDP = (S::NDES + 3) / 4 * 4;
  float W0[S::NNEU][NDP];
};
template <class S>
__device__ __forceinline__ void stage_network(const Model<S> &P, NetSmem<S> &N) {
  for (int t = threadIdx.x; t < S::NNEU * NetSmem<S>::NDP; t += blockDim.x) {
    const int mu = t / NetSmem<S>::NDP, v = t % NetSmem<S>::NDP;
    N.W0[mu][v] = v < S::NDES ? P.W0[mu][v] : 0.f;
  }
}
template <class S>
__device__ __forceinline__ float network_smem(const Model<S> &P, const NetSmem<S> &N, const float (&q)[S::NDES],
                                              bool flagged, float (&Fp)[S::NDES]) {
  constexpr int NDP = NetSmem<S>::NDP, NP = NDP / 2;
  float2 qt[NP], dq[NP];
#pragma unroll
  for (int p = 0; p < NP; ++p) {
    const int v0 = 2 * p, v1 = 2 * p + 1;
    qt[p] = pr(v0 < S::NDES ? q[v0 < S::NDES ? v0 : 0] * P.qs[v0 < S::NDES ? v0 : 0] : 0.f,
               v1 < S::NDES ? q[v1 < S::NDES ? v1 : 0] * P.qs[v1 < S::NDES ? v1 : 0] : 0.f);
    dq[p] = bc2(0.f);
  }
  float U = -P.b1;
#pragma unroll 1
  for (int mu = 0; mu < S::NNEU; ++mu) {
    // the row is read twice (forward, then backward) rather than held in registers
    const float4 *row = reinterpret_cast<const float4 *>(N.W0[mu]);
    float2 z2 = pr(-P.b0[mu], 0.f);
#pragma unroll
    for (int p = 0; p < NDP / 4; ++p) {
      const float4 t = row[p];
      z2 = fma2(pr(t.x, t.y), qt[2 * p], z2);
      z2 = fma2(pr(t.z, t.w), qt[2 * p + 1], z2);
    }
    const float h = tanhf(hsum(z2));
    U = fmaf(P.w1[mu], h, U);
    const float2 t2 = bc2(P.w1[mu] * (1.f - h * h));
#pragma unroll
    for (int p = 0; p < NDP / 4; ++p) {
      const float4 t = row[p];
      dq[2 * p] = fma2(t2, pr(t.x, t.y), dq[2 * p]);
      dq[2 * p + 1] = fma2(t2, pr(t.z, t.w), dq[2 * p + 1]);
    }
  }
#pragma unroll
  for (int v = 0; v < S::NDES; ++v) {
    const float d = (v & 1) ? dq[v / 2].y : dq[v / 2].x;
    Fp[v] = flagged ? 0.f : d * P.qs[v];
  }
  return U;
}

}  // namespace nep
