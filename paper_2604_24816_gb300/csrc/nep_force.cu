// nep_force.cu -- NEP descriptors, network and chain-rule forces on sm_103a.
//
// Two kernels per force evaluation, one thread per atom (cell-sorted order), both reading the
// distance-sorted neighbour list of nep_neighbor.cu.  For the teacher shape both keep their 120-value
// per-atom arrays (the sums s_nlm, the adjoint row G_i) in tensor memory (TMEM) rather than registers,
// which doubles (descriptor) or 1.5x (force) the resident warps:
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
//  k_force       forces and virial from the adjoint rows, in one of two forms (both deterministic):
//                full row (the float32 teacher): every ordered pair (i, j) of i's row gives
//                d_ij = dU_i/dr_ij from atom i's own row only -- radial sum_k dU/dQ_k f_k'(r) r^, angular
//                sum_nlm G_nlm d[g_n(r) Yh_lm(u)]/dr_ij, half of the LJ pair force -- which is added to F_i
//                and subtracted from F_j; no neighbour row is read.  Half list (float16 rows, the
//                student): D_ij = dU_i/dr_ij - dU_j/dr_ji for each unordered pair once, by its owner (the
//                owned part of the list), with H_nlm = G^i_nlm + (-1)^l G^j_nlm because the pair geometry
//                g_n(r) Yh_lm(u) is shared by both directions (Yh_lm(-u) = (-1)^l Yh_lm(u)) and D_ji = -D_ij
//                exactly; the owner adds D_ij to F_i and -D_ij to F_j.  The scatter uses 64-bit fixed-point
//                integer atomics (2^-32 eV/Angstrom units): integer addition is associative, so the forces
//                are bitwise reproducible whatever the order of the atomics -- the atomic scatter of the
//                paper's consolidated backward kernel (Section V.B, Optimization 1) made deterministic.
//                Virial W = -sum over the evaluated pairs of r_ij (x) (d_ij or D_ij).
//
// Everything is float32 except the per-block energy/virial partial sums (float64).
#include "nep_descriptor.cuh"
#include "nep_tc.cuh"

#include <type_traits>

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

constexpr int PIPE_DE = 8;    // list entries in flight per thread (descriptor kernel)
constexpr int PIPE_DP = 4;    // neighbour positions in flight per thread (descriptor kernel)
constexpr int FPIPE_DE = 6;   // the same for the force kernel, whose pairs take longer
constexpr int FPIPE_DP = 3;

template <class S>
__global__ void __launch_bounds__(DESC_BLOCK, NEP_DESC_MINB)
k_descriptor(const __grid_constant__ Model<S> P, const Geom geom, const int n, const float4 *__restrict__ pos,
             const int32_t *__restrict__ nbr, const RowExt X, float *__restrict__ G,
             float *__restrict__ usite, float *__restrict__ qout, long long *__restrict__ Ffix,
             long long *__restrict__ part, int *__restrict__ status, const __grid_constant__ Fallback fb) {
  __shared__ float4 shift[27];
  __shared__ uint32_t ring_e[PIPE_DE * DESC_BLOCK];
  __shared__ float4 ring_p[PIPE_DP * DESC_BLOCK];
  fill_shift_table(shift, geom);
  __syncthreads();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  long long acc[5] = {0, 0, 0, 0, 0};
  const bool skip = skip_far(X);
  if (i < n) {
    Ffix[i] = 0; Ffix[(size_t)n + i] = 0; Ffix[2 * (size_t)n + i] = 0;
    AtomSums<S> A;
    accumulate_atom<S, PIPE_DE, PIPE_DP, DESC_BLOCK>(P, shift, i, n, pos, nbr, full_row(X, i, skip), ring_e, ring_p,
                                                     A);
    float q[S::NDES];
    FourBody<S> T;
    descriptors_of<S>(P, A, q, T);
    if (qout != nullptr) {
#pragma unroll
      for (int v = 0; v < S::NDES; ++v) qout[(size_t)i * S::NDES + v] = q[v];
    }
    const bool flagged = fb.on && out_of_range<S>(fb, P, q);
    if (flagged) flag_atom(fb, i, status);

    float Fp[S::NDES];
    const float U = network<S>(P, q, flagged, Fp);   // flagged: no U_i from this model

    float *Gi = G + (size_t)i * S::GS;
#pragma unroll
    for (int a = 0; a < S::NA; ++a) {
      float gl[S::NLM];
      adjoint_channel<S>(a, A, T, Fp, gl);
#pragma unroll
      for (int c = 0; c < S::NLM; c += 4)
        *reinterpret_cast<float4 *>(Gi + a * S::NLM + c) = make_float4(gl[c], gl[c + 1], gl[c + 2], gl[c + 3]);
    }
    {
      float tail[8];
      radial_tail<S>(P, Fp, tail);
      *reinterpret_cast<float4 *>(Gi + S::NA * S::NLM) = make_float4(tail[0], tail[1], tail[2], tail[3]);
      *reinterpret_cast<float4 *>(Gi + S::NA * S::NLM + 4) = make_float4(tail[4], tail[5], tail[6], tail[7]);
    }
    const float ui = flagged ? A.elj : U + A.elj;
    usite[i] = ui;
    if (!isfinite(ui)) atomicOr(status, ST_NAN);
    acc[0] = to_fix32(ui);
    acc[1] = A.nrad;
    acc[2] = A.nang;
    acc[3] = A.cnt;
    acc[4] = A.nact;
  }
  block_sum_store<5, DESC_BLOCK / 32>(acc, part);
}

// Teacher-shape descriptor kernel with the 120 angular sums s_nlm accumulated in tensor memory (TMEM)
// instead of registers (accumulate_atom_tm), so that 4 blocks fit per SM instead of 2 (128 registers,
// 4 x 128 TMEM columns).
#ifndef NEP_DESC_MINB_TM
#define NEP_DESC_MINB_TM 4
#endif
template <class S>
__global__ void __launch_bounds__(DESC_BLOCK, NEP_DESC_MINB_TM)
k_descriptor_tm(const __grid_constant__ Model<S> P, const Geom geom, const int n, const float4 *__restrict__ pos,
                const int32_t *__restrict__ nbr, const RowExt X, float *__restrict__ G,
                float *__restrict__ usite, float *__restrict__ qout, long long *__restrict__ Ffix,
                long long *__restrict__ part, int *__restrict__ status, const __grid_constant__ Fallback fb) {
  static_assert(S::NA == 5 && S::NLM == 24 && S::FOURBODY && DESC_BLOCK == 128, "teacher shape, 4 warps");
  constexpr int W = TMEM_W;
  constexpr uint32_t TCOLS = 128;
  __shared__ float4 shift[27];
  __shared__ uint32_t ring_e[PIPE_DE * DESC_BLOCK];
  __shared__ float4 ring_p[PIPE_DP * DESC_BLOCK];
  __shared__ uint32_t tmem_base;
  if (threadIdx.x < 32) tmem_alloc(&tmem_base, TCOLS);
  tc_fence_before();
  fill_shift_table(shift, geom);
  __syncthreads();
  tc_fence_after();
  const uint32_t trow = tmem_base + ((uint32_t)(threadIdx.x & ~31u) << 16);
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const bool live = i < n;
  const int ii = live ? i : 0;
  long long acc[5] = {0, 0, 0, 0, 0};
  if (live) { Ffix[i] = 0; Ffix[(size_t)n + i] = 0; Ffix[2 * (size_t)n + i] = 0; }
  const RowSpan sp = live ? full_row(X, i, skip_far(X)) : RowSpan{0, 0, 0};
  const int cnt = sp.c;
  float QR[S::KR], elj;
  int nrad, nang, nact;
  RegSums<S, S::NA> R;                      // empty: every channel in TMEM
  accumulate_atom_tm<S, S::NA, PIPE_DE, PIPE_DP, DESC_BLOCK>(P, shift, trow, ii, n, pos, nbr, sp, ring_e, ring_p,
                                                             QR, R, elj, nrad, nang, nact);
  float q[S::NDES];
  FourBody<S> T;
  descriptors_tm<S, S::NA>(P, trow, QR, R, q, T);
  if (live && qout != nullptr) {
#pragma unroll
    for (int v = 0; v < S::NDES; ++v) qout[(size_t)i * S::NDES + v] = q[v];
  }
  const bool flagged = live && fb.on && out_of_range<S>(fb, P, q);
  if (flagged) flag_atom(fb, i, status);
  float Fp[S::NDES];
  const float U = network<S>(P, q, flagged, Fp);

  // adjoint row from the TMEM sums, then the radial tail
  float *Gi = G + (size_t)ii * S::GS;
  float g4[S::NA][5];
#pragma unroll
  for (int a = 0; a < S::NA; ++a) fourbody_adjoint<S>(a, T, g4[a]);
#pragma unroll
  for (int c = 0; c < S::NLM; c += W) {
    float sv[S::NA][W];
    sums_chunk<S, S::NA>(trow, c, R, sv);
#pragma unroll
    for (int a = 0; a < S::NA; ++a) {
      float gl[W];
      adjoint_chunk<S>(a, c, sv[a], g4[a], Fp, gl);
      if (live) *reinterpret_cast<float4 *>(Gi + a * S::NLM + c) = make_float4(gl[0], gl[1], gl[2], gl[3]);
    }
  }
  if (live) {
    float tail[8];
    radial_tail<S>(P, Fp, tail);
    *reinterpret_cast<float4 *>(Gi + S::NA * S::NLM) = make_float4(tail[0], tail[1], tail[2], tail[3]);
    *reinterpret_cast<float4 *>(Gi + S::NA * S::NLM + 4) = make_float4(tail[4], tail[5], tail[6], tail[7]);
    const float ui = flagged ? elj : U + elj;
    usite[i] = ui;
    if (!isfinite(ui)) atomicOr(status, ST_NAN);
    acc[0] = to_fix32(ui);
    acc[1] = nrad;
    acc[2] = nang;
    acc[3] = cnt;
    acc[4] = nact;
  }
  tc_fence_before();
  __syncthreads();
  if (threadIdx.x < 32) {
    tc_fence_after();
    tmem_dealloc(tmem_base, TCOLS);
  }
  block_sum_store<5, DESC_BLOCK / 32>(acc, part);
}

// Adjoint row G_i of the force kernel: in registers for small shapes; for the teacher shape (120
// angular values) it is parked in tensor memory (TMEM) and read back one chunk of lm components at a
// time.  TMEM is per-SM storage outside L1, so this cuts the register footprint (255 -> 128-168
// registers: 4 resident blocks for the full-row form, 3 for the half list) without taking L1 capacity
// from the gathered neighbour data.
#ifndef NEP_FORCE_MINB_TM
#define NEP_FORCE_MINB_TM 3
#endif
template <class S>
struct ForceCfg {
  static constexpr bool TM = S::NLM > 8 && S::NA == 5;
  static constexpr int MINB = TM ? NEP_FORCE_MINB_TM : NEP_FORCE_MINB;
  static constexpr uint32_t TCOLS = 128;   // TMEM columns per block: >= NA * NLM, a power of two
  // neighbour pipeline depth; with 3 resident blocks the shallower ring and no L1 prefetch of the
  // next neighbour row measured best
  static constexpr int DE = TM ? 4 : FPIPE_DE, DP = TM ? 2 : FPIPE_DP;
  static constexpr bool PREFETCH = !TM;
  static_assert(!TM || S::NA * S::NLM <= (int)TCOLS, "adjoint row does not fit the TMEM allocation");
  static_assert(!TM || FORCE_BLOCK == 128, "one TMEM lane per thread: 4 warps cover the 128 lanes");
};

// The pair loop of the force kernel (see k_force), for atom i whose adjoint row is already in place:
// in TMEM at trow (teacher shape) or in gi (registers), radial tail in fpi.  Adds d_ij (FULL) or D_ij
// to F_i and subtracts it from F_j, and leaves the virial and pair counters in acc.
template <class S, class GT, bool FS, bool FULL>
__device__ __forceinline__ void force_pairs(const Model<S> &P, const float4 *shift, uint32_t trow,
                                            const float (&gi)[ForceCfg<S>::TM ? 1 : S::NA][ForceCfg<S>::TM ? 1 : S::NLM],
                                            const float (&fpi)[8], int i, bool live, int ii, int n,
                                            const float4 *__restrict__ pos, const int32_t *__restrict__ nbr,
                                            RowSpan sp, int nb0, const GT *__restrict__ G, uint32_t *ring_e, float4 *ring_p,
                                            unsigned long long *__restrict__ Ffix, int *__restrict__ status,
                                            float *__restrict__ Ff, long long (&acc)[13]) {
  constexpr bool TM = ForceCfg<S>::TM;
  constexpr int W = GTraits<GT>::W;
  constexpr int DE = ForceCfg<S>::DE, DP = ForceCfg<S>::DP;
  const float4 pi = pos[ii];
  float fx = 0.f, fy = 0.f, fz = 0.f;
  float wxx = 0.f, wxy = 0.f, wxz = 0.f, wyx = 0.f, wyy = 0.f, wyz = 0.f, wzx = 0.f, wzy = 0.f, wzz = 0.f;
  const int cnt = sp.c;
  int nrad = 0, nang = 0, nact = 0;
  NbrPipe<DE, DP, FORCE_BLOCK> pipe;
  pipe.start(ring_e, ring_p, nbr + ii, (size_t)n, pos, sp);
  const int trip = TM ? __reduce_max_sync(0xffffffffu, cnt) : cnt;
  for (int k = 0; k < trip; ++k) {
    const bool valid = k < cnt;
    uint32_t e = 0u;
    float4 pj = pi;
    if (valid) {
      pipe.get(k, e, pj);
      // pull the next angular neighbour's adjoint row into L1 while this pair is computed
      if (ForceCfg<S>::PREFETCH && !FULL && k + 1 < nb0 && k + 1 < cnt) {
        const uint32_t en = pipe.re[((k + 1) % DE) * FORCE_BLOCK];
        const char *gr = reinterpret_cast<const char *>(G + (size_t)(en & J_MASK) * S::GS);
#pragma unroll
        for (int b = 0; b < (int)(S::GS * sizeof(GT)); b += 128) prefetch_l1(gr + b);
      }
    }
    const int j = (int)(e & J_MASK);
    const float4 o = shift[e >> J_BITS];
    const float dx = pj.x - pi.x + o.x, dy = pj.y - pi.y + o.y, dz = pj.z - pi.z + o.z;
    const float r2 = dx * dx + dy * dy + dz * dz;
    const bool act = valid && r2 < P.rmax2;
    if constexpr (!TM) {
      if (!act) continue;
    }
    const float ir = rsqrtf(r2);
    const float r = r2 * ir;
    float coef = 0.f;                     // D = coef * d + (vx, vy, vz)
    float vx = 0.f, vy = 0.f, vz = 0.f;
    if (act && r2 < P.rcR2) {
      float f[S::KR], df[S::KR];
      cheb_basis_d<S::KR>(r, P.inv_rcR, f, df);
      float c = 0.f;
      if constexpr (FULL) {
#pragma unroll
        for (int k = 0; k < S::KR; ++k) c = fmaf(fpi[k], df[k], c);
      } else {
        float fpj[8];
        load_tail8(G + (size_t)j * S::GS, S::NA * S::NLM, fpj);
#pragma unroll
        for (int k = 0; k < S::KR; ++k) c = fmaf(fpi[k] + fpj[k], df[k], c);
      }
      coef = c * ir;
      ++nrad;
    }
    if (act && P.lj_on != 0.f && r2 < P.lj_rc2) {
      float el, dl;
      lj_pair<S>(P, r2, r, ir, el, dl);
      coef = fmaf(FULL ? 0.5f * dl : dl, ir, coef);   // FULL: each atom of the pair takes half
    }
    const bool ang = act && r2 < P.rcA2;
    bool enter = ang;
    if constexpr (TM) enter = __any_sync(0xffffffffu, ang);
    if (enter) {
      if constexpr (TM) __syncwarp();
      // stand-in pair for lanes that only take part in the warp-collective loads: r = 1 along x,
      // the row of atom ii
      const bool si = TM && !ang;
      const float ar = si ? 1.f : r, air = si ? 1.f : ir;
      const float ux = si ? 1.f : dx * ir, uy = si ? 0.f : dy * ir, uz = si ? 0.f : dz * ir;
      const GT *Gj = G + (size_t)(si ? ii : j) * S::GS;
      float f[S::KA], df[S::KA];
      cheb_basis_d<S::KA>(ar, P.inv_rcA, f, df);
      float g[S::NA], dg[S::NA];
#pragma unroll
      for (int a = 0; a < S::NA; ++a) {
        float t = 0.f, dt = 0.f;
#pragma unroll
        for (int b = 0; b < S::KA; ++b) { t = fmaf(P.cA[a][b], f[b], t); dt = fmaf(P.cA[a][b], df[b], dt); }
        g[a] = t; dg[a] = dt;
      }
      float Y[S::NLM];
      harmonics<S::NLM>(ux, uy, uz, Y);
      float along = 0.f, bx = 0.f, by = 0.f, bz = 0.f;
      // d/dd [g_n(r) Yh_lm(u)] = (g_n' - l g_n / r) Yh_lm u + (g_n / r) grad P_lm(u)
#pragma unroll
      for (int c = 0; c < S::NLM; c += W) {
        float hj[S::NA][W], hi[S::NA][W];
        if constexpr (!FULL) {
#pragma unroll
          for (int a = 0; a < S::NA; ++a) load_vec(Gj + a * S::NLM + c, hj[a]);
        }
        if constexpr (TM) {
          uint32_t cols[S::NA];
#pragma unroll
          for (int a = 0; a < S::NA; ++a) cols[a] = trow + (uint32_t)(c * S::NA + a * W);
          tmem_ld5(cols, hi);
        } else {
#pragma unroll
          for (int a = 0; a < S::NA; ++a)
#pragma unroll
            for (int cc = 0; cc < W; ++cc) hi[a][cc] = gi[a][c + cc];
        }
#pragma unroll
        for (int cc = 0; cc < W; ++cc) {
          const int lm = c + cc;
          const float sgn = (lm_l(lm) & 1) ? -1.f : 1.f;
          float av = 0.f, bv = 0.f;
#pragma unroll
          for (int a = 0; a < S::NA; ++a) {
            const float H = FULL ? hi[a][cc] : fmaf(sgn, hj[a][cc], hi[a][cc]);
            av = fmaf(H, dg[a], av);
            bv = fmaf(H, g[a], bv);
          }
          along = fmaf(av - (float)lm_l(lm) * air * bv, Y[lm], along);
          harmonic_grad_acc(lm, ux, uy, uz, bv, bx, by, bz);
        }
      }
      if (ang) {
        ++nang;
        coef = fmaf(along, ir, coef);
        vx = bx * ir; vy = by * ir; vz = bz * ir;
      }
    }
    if (act) {
      ++nact;
      const float Dx = fmaf(coef, dx, vx), Dy = fmaf(coef, dy, vy), Dz = fmaf(coef, dz, vz);
      fx += Dx; fy += Dy; fz += Dz;
      // Newton's third law: F_j -= D_ij, accumulated in fixed point (order-independent sum)
      if constexpr (FS) {
        atomicAdd(Ff + j, -Dx); atomicAdd(Ff + (size_t)n + j, -Dy); atomicAdd(Ff + 2 * (size_t)n + j, -Dz);
      } else {
        atomicAdd(Ffix + j, (unsigned long long)(-to_fix32(Dx)));
        atomicAdd(Ffix + (size_t)n + j, (unsigned long long)(-to_fix32(Dy)));
        atomicAdd(Ffix + 2 * (size_t)n + j, (unsigned long long)(-to_fix32(Dz)));
      }
      wxx = fmaf(dx, Dx, wxx); wxy = fmaf(dx, Dy, wxy); wxz = fmaf(dx, Dz, wxz);
      wyx = fmaf(dy, Dx, wyx); wyy = fmaf(dy, Dy, wyy); wyz = fmaf(dy, Dz, wyz);
      wzx = fmaf(dz, Dx, wzx); wzy = fmaf(dz, Dy, wzy); wzz = fmaf(dz, Dz, wzz);
    }
  }
  pipe.finish();
  if (live) {
    if constexpr (FS) {
      atomicAdd(Ff + i, fx); atomicAdd(Ff + (size_t)n + i, fy); atomicAdd(Ff + 2 * (size_t)n + i, fz);
    } else {
      atomicAdd(Ffix + i, (unsigned long long)to_fix32(fx));
      atomicAdd(Ffix + (size_t)n + i, (unsigned long long)to_fix32(fy));
      atomicAdd(Ffix + 2 * (size_t)n + i, (unsigned long long)to_fix32(fz));
    }
    if (!(isfinite(fx) && isfinite(fy) && isfinite(fz))) atomicOr(status, ST_NAN);
    // each unordered pair once: W = -sum_pairs r_ij (x) D_ij
    acc[0] = -to_fix32(wxx); acc[1] = -to_fix32(wxy); acc[2] = -to_fix32(wxz);
    acc[3] = -to_fix32(wyx); acc[4] = -to_fix32(wyy); acc[5] = -to_fix32(wyz);
    acc[6] = -to_fix32(wzx); acc[7] = -to_fix32(wzy); acc[8] = -to_fix32(wzz);
    acc[9] = cnt; acc[10] = nact; acc[11] = nrad; acc[12] = nang;
  }
}

// FULL = true walks the whole row with atom i's own adjoint only; FULL = false walks the owned half
// and gathers the neighbour's row (see the file header).  Either leaves the far bands out when the
// control block allows it (RowExt, skip_far).  FS = true is the paper's scatter (Section V.B, Optimization 1) kept as an ablation: float
// atomicAdd into Ff, whose result depends on the order in which the additions arrive.
//
// With the row in TMEM the pair loop runs to the warp's largest owned count (threads past their own
// count, or past the last atom, idle with a predicate) so that the angular block, which holds the
// warp-collective TMEM loads, is entered by whole warps: lanes without an angular pair in that
// iteration compute on a harmless stand-in pair and discard the result.
#ifndef NEP_FORCE_MINB_FULL
#define NEP_FORCE_MINB_FULL 4
#endif
template <class S, class GT, bool FS = false, bool FULL = false>
__global__ void __launch_bounds__(FORCE_BLOCK, FULL && ForceCfg<S>::TM ? NEP_FORCE_MINB_FULL : ForceCfg<S>::MINB)
k_force(const __grid_constant__ Model<S> P, const Geom geom, const int n, const float4 *__restrict__ pos,
        const int32_t *__restrict__ nbr, const RowExt X, const GT *__restrict__ G,
        unsigned long long *__restrict__ Ffix, long long *__restrict__ part,
        int *__restrict__ status, float *__restrict__ Ff = nullptr) {
  constexpr bool TM = ForceCfg<S>::TM;
  constexpr int W = GTraits<GT>::W;
  __shared__ float4 shift[27];
  constexpr int DE = ForceCfg<S>::DE, DP = ForceCfg<S>::DP;
  __shared__ uint32_t ring_e[DE * FORCE_BLOCK];
  __shared__ float4 ring_p[DP * FORCE_BLOCK];
  __shared__ uint32_t tmem_base;
  if constexpr (TM) {
    if (threadIdx.x < 32) tmem_alloc(&tmem_base, ForceCfg<S>::TCOLS);
    tc_fence_before();
  }
  fill_shift_table(shift, geom);
  __syncthreads();
  uint32_t trow = 0;   // this thread's TMEM lane, column 0
  if constexpr (TM) {
    tc_fence_after();
    trow = tmem_base + ((uint32_t)(threadIdx.x & ~31u) << 16);
  }
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const bool live = i < n;
  const int ii = live ? i : 0;            // the row read (and ignored) by threads past the last atom
  long long acc[13] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
  const GT *Gi = G + (size_t)ii * S::GS;
  // G_i[a][lm] lives at TMEM column (lm - lm mod W) NA + a W + lm mod W: chunk c of W components
  // holds all channels in NA consecutive groups of W columns.
  float gi[TM ? 1 : S::NA][TM ? 1 : S::NLM];
#pragma unroll
  for (int a = 0; a < S::NA; ++a)
#pragma unroll
    for (int c = 0; c < S::NLM; c += W) {
      float t[W];
      load_vec(Gi + a * S::NLM + c, t);
      if constexpr (TM) {
        tmem_st(trow + (uint32_t)(c * S::NA + a * W), t);
      } else {
#pragma unroll
        for (int k = 0; k < W; ++k) gi[a][c + k] = t[k];
      }
    }
  if constexpr (TM) tmem_wait_st();
  float fpi[8];
  load_tail8(Gi, S::NA * S::NLM, fpi);
  const bool skip = skip_far(X);
  const RowSpan sp = !live ? RowSpan{0, 0, 0} : (FULL ? full_row(X, i, skip) : owned_row(X, i, skip));
  force_pairs<S, GT, FS, FULL>(P, shift, trow, gi, fpi, i, live, ii, n, pos, nbr, sp, live ? X.nband0[i] : 0, G,
                               ring_e, ring_p, Ffix, status, Ff, acc);
  if constexpr (TM) {
    tc_fence_before();
    __syncthreads();
    if (threadIdx.x < 32) {
      tc_fence_after();
      tmem_dealloc(tmem_base, ForceCfg<S>::TCOLS);
    }
  }
  block_sum_store<13, FORCE_BLOCK / 32>(acc, part);
}

// Descriptors, network and forces of the float32 teacher in one kernel.  The full-row force form reads
// no neighbour row, so no atom waits for another's adjoint row: the angular sums s_nlm are accumulated
// in TMEM, turned into the adjoint row in place, and the force pass walks the row again with it, so no
// adjoint row goes through HBM and one launch (and its tail wave) is saved.  The forces are scattered
// with atomics into Ffix, which the caller zeroes before the launch (a block may add to F_j before
// atom j's own block has started).
#ifndef NEP_FUSED_MINB
#define NEP_FUSED_MINB 4
#endif
template <class S>
__global__ void __launch_bounds__(DESC_BLOCK, NEP_FUSED_MINB)
k_nep_fused(const __grid_constant__ Model<S> P, const Geom geom, const int n, const float4 *__restrict__ pos,
            const int32_t *__restrict__ nbr, const RowExt X, float *__restrict__ usite,
            float *__restrict__ qout, unsigned long long *__restrict__ Ffix, long long *__restrict__ part_d,
            long long *__restrict__ part_f, int *__restrict__ status) {
  static_assert(ForceCfg<S>::TM && DESC_BLOCK == 128 && FORCE_BLOCK == 128, "teacher shape, 4 warps");
  static_assert(ForceCfg<S>::DE <= PIPE_DE && ForceCfg<S>::DP <= PIPE_DP, "one ring serves both passes");
  constexpr int W = TMEM_W;
  constexpr uint32_t TCOLS = 128;
  __shared__ float4 shift[27];
  __shared__ uint32_t ring_e[PIPE_DE * DESC_BLOCK];
  __shared__ float4 ring_p[PIPE_DP * DESC_BLOCK];
  __shared__ uint32_t tmem_base;
  if (threadIdx.x < 32) tmem_alloc(&tmem_base, TCOLS);
  tc_fence_before();
  fill_shift_table(shift, geom);
  __syncthreads();
  tc_fence_after();
  const uint32_t trow = tmem_base + ((uint32_t)(threadIdx.x & ~31u) << 16);
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const bool live = i < n;
  const int ii = live ? i : 0;
  const RowSpan sp = live ? full_row(X, i, skip_far(X)) : RowSpan{0, 0, 0};
  const int cnt = sp.c;

  // descriptors and network (as k_descriptor_tm)
  float QR[S::KR], elj;
  int nrad, nang, nact;
  RegSums<S, S::NA> R;
  accumulate_atom_tm<S, S::NA, PIPE_DE, PIPE_DP, DESC_BLOCK>(P, shift, trow, ii, n, pos, nbr, sp, ring_e, ring_p,
                                                             QR, R, elj, nrad, nang, nact);
  float q[S::NDES];
  FourBody<S> T;
  descriptors_tm<S, S::NA>(P, trow, QR, R, q, T);
  if (live && qout != nullptr) {
#pragma unroll
    for (int v = 0; v < S::NDES; ++v) qout[(size_t)i * S::NDES + v] = q[v];
  }
  float Fp[S::NDES];
  const float U = network<S>(P, q, false, Fp);

  // the adjoint row replaces the sums in TMEM (same columns, chunk by chunk); radial tail in registers
  float g4[S::NA][5];
#pragma unroll
  for (int a = 0; a < S::NA; ++a) fourbody_adjoint<S>(a, T, g4[a]);
#pragma unroll
  for (int c = 0; c < S::NLM; c += W) {
    float sv[S::NA][W];
    sums_chunk<S, S::NA>(trow, c, R, sv);
    uint32_t cols[S::NA];
    tmem_chunk_cols<S::NA>(trow, c, cols);
#pragma unroll
    for (int a = 0; a < S::NA; ++a) {
      float gl[W];
      adjoint_chunk<S>(a, c, sv[a], g4[a], Fp, gl);
      tmem_st(cols[a], gl);
    }
  }
  tmem_wait_st();
  float fpi[8];
  radial_tail<S>(P, Fp, fpi);
  long long acc_d[5] = {0, 0, 0, 0, 0};
  if (live) {
    const float ui = U + elj;
    usite[i] = ui;
    if (!isfinite(ui)) atomicOr(status, ST_NAN);
    acc_d[0] = to_fix32(ui);
    acc_d[1] = nrad;
    acc_d[2] = nang;
    acc_d[3] = cnt;
    acc_d[4] = nact;
  }
  block_sum_store<5, DESC_BLOCK / 32>(acc_d, part_d);   // before the force pass: fewer live registers

  // forces: every ordered pair of the row with the own adjoint row (as k_force, FULL)
  const float gi[1][1] = {{0.f}};
  long long acc_f[13] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
  force_pairs<S, float, false, true>(P, shift, trow, gi, fpi, i, live, ii, n, pos, nbr, sp, 0, nullptr, ring_e,
                                     ring_p, Ffix, status, nullptr, acc_f);
  tc_fence_before();
  __syncthreads();
  if (threadIdx.x < 32) {
    tc_fence_after();
    tmem_dealloc(tmem_base, TCOLS);
  }
  block_sum_store<13, DESC_BLOCK / 32>(acc_f, part_f);
}

// ---------------------------------------------------------------------------------------------------
// Host launchers (called from nep_api.cu).

#ifndef NEP_DESC_TM
#define NEP_DESC_TM 1
#endif
template <class S>
cudaError_t launch_descriptor(const Model<S> &P, const Geom &g, int n, const float4 *pos, const int32_t *nbr,
                              const RowExt &X, float *G, float *usite, float *qout, long long *Ffix,
                              long long *part, int *status, const Fallback &fb, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  const int grid = (n + DESC_BLOCK - 1) / DESC_BLOCK;
  if constexpr (ForceCfg<S>::TM && NEP_DESC_TM)
    k_descriptor_tm<S><<<grid, DESC_BLOCK, 0, st>>>(P, g, n, pos, nbr, X, G, usite, qout, Ffix, part, status, fb);
  else
    k_descriptor<S><<<grid, DESC_BLOCK, 0, st>>>(P, g, n, pos, nbr, X, G, usite, qout, Ffix, part, status, fb);
  return cudaGetLastError();
}

// Which form of the force kernel runs: the full-row gather-free form for the teacher shape with
// float32 rows (its half-list gathers of 512-byte rows are the slowest part), the half list with
// gathers otherwise (float16 rows and the student's 160-byte rows are cheap to gather, and the half
// list does 0.6x the arithmetic).
template <class S, class GT>
constexpr bool force_full_row() {
  return ForceCfg<S>::TM && std::is_same<GT, float>::value;
}

template <class S, class GT>
cudaError_t launch_force(const Model<S> &P, const Geom &g, int n, const float4 *pos, const int32_t *nbr,
                         const RowExt &X, const GT *G,
                         long long *Ffix, long long *part, int *status, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  const int grid = (n + FORCE_BLOCK - 1) / FORCE_BLOCK;
  constexpr bool full = force_full_row<S, GT>();
  k_force<S, GT, false, full><<<grid, FORCE_BLOCK, 0, st>>>(P, g, n, pos, nbr, X, G,
                                                           reinterpret_cast<unsigned long long *>(Ffix), part, status);
  return cudaGetLastError();
}

// Ablation: the teacher's half-list force kernel with float32 rows (each unordered pair once by its
// owner, gathering the neighbour's adjoint row), instead of the full-row form.
template <class S>
cudaError_t launch_force_half_list(const Model<S> &P, const Geom &g, int n, const float4 *pos, const int32_t *nbr,
                                   const RowExt &X, const float *G, long long *Ffix,
                                   long long *part, int *status, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  const int grid = (n + FORCE_BLOCK - 1) / FORCE_BLOCK;
  k_force<S, float, false, false><<<grid, FORCE_BLOCK, 0, st>>>(P, g, n, pos, nbr, X, G,
                                                               reinterpret_cast<unsigned long long *>(Ffix), part,
                                                               status);
  return cudaGetLastError();
}
template cudaError_t launch_force_half_list<CuShape>(const Model<CuShape> &, const Geom &, int, const float4 *,
                                                     const int32_t *, const RowExt &, const float *, long long *,
                                                     long long *, int *, cudaStream_t);

// Ablation: the production (full-row) force kernel with float atomicAdd scatter into Ff [3][n] (zeroed
// by the caller) instead of fixed-point integer atomics.
template <class S>
cudaError_t launch_force_float_scatter(const Model<S> &P, const Geom &g, int n, const float4 *pos, const int32_t *nbr,
                                       const RowExt &X, const float *G, float *Ff,
                                       long long *part, int *status, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  const int grid = (n + FORCE_BLOCK - 1) / FORCE_BLOCK;
  k_force<S, float, true, true><<<grid, FORCE_BLOCK, 0, st>>>(P, g, n, pos, nbr, X, G, nullptr, part,
                                                             status, Ff);
  return cudaGetLastError();
}
template cudaError_t launch_force_float_scatter<CuShape>(const Model<CuShape> &, const Geom &, int, const float4 *,
                                                         const int32_t *, const RowExt &, const float *, float *,
                                                         long long *, int *, cudaStream_t);

// Fused descriptor + force evaluation of the float32 teacher (k_nep_fused); Ffix must be zero.
template <class S>
cudaError_t launch_fused(const Model<S> &P, const Geom &g, int n, const float4 *pos, const int32_t *nbr,
                         const RowExt &X, float *usite, float *qout, long long *Ffix, long long *part_d,
                         long long *part_f, int *status, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  const int grid = (n + DESC_BLOCK - 1) / DESC_BLOCK;
  k_nep_fused<S><<<grid, DESC_BLOCK, 0, st>>>(P, g, n, pos, nbr, X, usite, qout,
                                              reinterpret_cast<unsigned long long *>(Ffix), part_d, part_f, status);
  return cudaGetLastError();
}
template cudaError_t launch_fused<CuShape>(const Model<CuShape> &, const Geom &, int, const float4 *, const int32_t *,
                                           const RowExt &, float *, float *, long long *, long long *, long long *,
                                           int *, cudaStream_t);

int descriptor_blocks(int n) { return (n + DESC_BLOCK - 1) / DESC_BLOCK; }
int force_blocks(int n) { return (n + FORCE_BLOCK - 1) / FORCE_BLOCK; }

#define NEP_INSTANTIATE(SH)                                                                                    \
  template cudaError_t launch_descriptor<SH>(const Model<SH> &, const Geom &, int, const float4 *, const int32_t *,   \
                                             const RowExt &, float *, float *, float *, long long *, long long *,    \
                                             int *, const Fallback &, cudaStream_t);                                  \
  template cudaError_t launch_force<SH, float>(const Model<SH> &, const Geom &, int, const float4 *, const int32_t *, \
                                               const RowExt &, const float *, long long *, long long *, int *,         \
                                               cudaStream_t);                                                         \
  template cudaError_t launch_force<SH, __half>(const Model<SH> &, const Geom &, int, const float4 *,                 \
                                                const int32_t *, const RowExt &, const __half *, long long *,         \
                                                long long *, int *, cudaStream_t);
NEP_INSTANTIATE(CuShape)
NEP_INSTANTIATE(StudentShape)
#undef NEP_INSTANTIATE

}  // namespace nep
