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
constexpr int PIPE_DP = 2;    // neighbour positions (and the fused force pass's records) in flight per thread
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
  __shared__ __align__(16) NetSmem<S> net;
  if (threadIdx.x < 32) tmem_alloc(&tmem_base, TCOLS);
  tc_fence_before();
  fill_shift_table(shift, geom);
  stage_network(P, net);
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
  const float U = network_smem<S>(P, net, q, flagged, Fp);

  // adjoint row from the TMEM sums, then the radial tail
  float *Gi = G + (size_t)ii * S::GS;
  float g4[S::NA][5];
  fourbody_adjoint_tm<S, S::NA>(trow, R, g4);
#pragma unroll
  for (int k = 0; k < S::NLM / W; ++k) {
    const int c = W * k;
    float sv[S::NA][W];
    sums_chunk<S, S::NA>(trow, k, R, sv);
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

// The angular part of one pair's force, d/dd of sum_nlm H_nlm g_n(r) Yh_lm(u) with H the adjoint row:
// H = G^i (FULL; in TMEM at trow for the teacher shape, else in gi) or G^i + (-1)^l G^j (half list, G^j
// gathered from Gj).  Returns sum_lm (A_lm - l B_lm / r) Yh_lm (al, even and odd lm apart) and
// sum_lm B_lm grad P_lm(u) (gv), A_lm = sum_n H_nlm g_n'(r), B_lm = sum_n H_nlm g_n(r).  si: a stand-in
// pair (r = 1 along x) for lanes that only take part in the warp-collective TMEM loads.  UN: the row
// holds G'_nlm = hnorm(lm) G_nlm, the weights of the polynomials Ph_lm (harmonics_p).
template <class S, class GT, bool FULL, bool UN = false>
__device__ __forceinline__ void angular_pair(const Model<S> &P, uint32_t trow,
                                             const float (&gi)[ForceCfg<S>::TM ? 1 : S::NA][ForceCfg<S>::TM ? 1 : S::NLM],
                                             const GT *__restrict__ Gj, bool si, float r, float ir, float dx, float dy,
                                             float dz, float2 &al, float2 (&gv)[3]) {
  constexpr bool TM = ForceCfg<S>::TM;
  constexpr int W = GTraits<GT>::W;
  const float ar = si ? 1.f : r, air = si ? 1.f : ir;
  const float ux = si ? 1.f : dx * ir, uy = si ? 0.f : dy * ir, uz = si ? 0.f : dz * ir;
  float f[S::KA], df[S::KA];
  cheb_basis_d<S::KA>(ar, P.inv_rcA, f, df);
  float g[S::NA], dg[S::NA];
#pragma unroll
  for (int a = 0; a < S::NA; ++a) dot_pairs2<S::KA>(P.cA[a], f, df, g[a], dg[a]);
  // UN: the polynomials Ph_lm are formed chunk by chunk below (fewer live registers than 24 values)
  float Y[S::NLM];
  if constexpr (!UN) harmonics<S::NLM>(ux, uy, uz, Y);
  const float2 air2 = bc2(air);
  // d/dd [g_n(r) Yh_lm(u)] = (g_n' - l g_n / r) Yh_lm u + (g_n / r) grad P_lm(u); per component
  // A_lm = sum_n H_nlm g_n', B_lm = sum_n H_nlm g_n, in pairs of consecutive components (lm, lm + 1)
  al = bc2(0.f);
  gv[0] = gv[1] = gv[2] = bc2(0.f);
  float hj8[S::NA][8];
#pragma unroll
  for (int k = 0; k < S::NLM / 4; ++k) {
    const int lm0 = 4 * k;
    float hi[S::NA][4];
    if constexpr (TM) {
      tm_load<S, S::NA>(trow, k, hi);
    } else {
#pragma unroll
      for (int a = 0; a < S::NA; ++a)
#pragma unroll
        for (int cc = 0; cc < 4; ++cc) hi[a][cc] = gi[a][lm0 + cc];
    }
    if constexpr (!FULL) {
      // H = G^i + (-1)^l G^j: the neighbour's row, W values per 16-byte load
      if (W == 4 || (k & 1) == 0) {
#pragma unroll
        for (int a = 0; a < S::NA; ++a) {
          float t[W];
          load_vec(Gj + a * S::NLM + (lm0 / W) * W, t);
#pragma unroll
          for (int cc = 0; cc < W; ++cc) hj8[a][cc] = t[cc];
        }
      }
      const int o = W == 4 ? 0 : (k & 1) * 4;
      const float2 s01 = pr((lm_l(lm0) & 1) ? -1.f : 1.f, (lm_l(lm0 + 1) & 1) ? -1.f : 1.f);
      const float2 s23 = pr((lm_l(lm0 + 2) & 1) ? -1.f : 1.f, (lm_l(lm0 + 3) & 1) ? -1.f : 1.f);
#pragma unroll
      for (int a = 0; a < S::NA; ++a) {
        const float2 h01 = fma2(s01, pr(hj8[a][o], hj8[a][o + 1]), pr(hi[a][0], hi[a][1]));
        const float2 h23 = fma2(s23, pr(hj8[a][o + 2], hj8[a][o + 3]), pr(hi[a][2], hi[a][3]));
        hi[a][0] = h01.x; hi[a][1] = h01.y; hi[a][2] = h23.x; hi[a][3] = h23.y;
      }
    }
    float2 av01 = bc2(0.f), av23 = bc2(0.f), bv01 = bc2(0.f), bv23 = bc2(0.f);
#pragma unroll
    for (int a = 0; a < S::NA; ++a) {
      const float2 h01 = pr(hi[a][0], hi[a][1]), h23 = pr(hi[a][2], hi[a][3]);
      const float2 dg2 = bc2(dg[a]), g2 = bc2(g[a]);
      av01 = fma2(h01, dg2, av01);
      av23 = fma2(h23, dg2, av23);
      bv01 = fma2(h01, g2, bv01);
      bv23 = fma2(h23, g2, bv23);
    }
    const float2 nl01 = mul2(pr(-(float)lm_l(lm0), -(float)lm_l(lm0 + 1)), air2);
    const float2 nl23 = mul2(pr(-(float)lm_l(lm0 + 2), -(float)lm_l(lm0 + 3)), air2);
    if constexpr (UN) {
      al = fma2(fma2(nl01, bv01, av01), pr(harmonic_p(lm0, ux, uy, uz), harmonic_p(lm0 + 1, ux, uy, uz)), al);
      al = fma2(fma2(nl23, bv23, av23), pr(harmonic_p(lm0 + 2, ux, uy, uz), harmonic_p(lm0 + 3, ux, uy, uz)), al);
    } else {
      al = fma2(fma2(nl01, bv01, av01), pr(Y[lm0], Y[lm0 + 1]), al);
      al = fma2(fma2(nl23, bv23, av23), pr(Y[lm0 + 2], Y[lm0 + 3]), al);
    }
    harmonic_grad_acc2<UN>(lm0, ux, uy, uz, bv01, gv);
    harmonic_grad_acc2<UN>(lm0 + 2, ux, uy, uz, bv23, gv);
  }
}

// The pair loop of the force kernel (see k_force), for atom i whose adjoint row is already in place:
// in TMEM at trow (teacher shape) or in gi (registers), radial tail (8 values) in shared memory at
// fps[0] and fps[FORCE_BLOCK].  Adds d_ij (FULL) or D_ij to F_i and subtracts it from F_j, and leaves
// the virial and (COUNT) the pair counters in acc.
//
// Virial: only the 6 components of the upper triangle are accumulated and mirrored.  The total
// W = -sum r_ij (x) d_ij is symmetric because every site energy U_i (and the LJ pair term) is invariant
// under a rigid rotation of its neighbours: for any antisymmetric Omega, sum_j (Omega r_ij) . d_ij = 0.
template <class S, class GT, bool FS, bool FULL, bool COUNT = true>
__device__ __forceinline__ void force_pairs(const Model<S> &P, const float4 *shift, uint32_t trow,
                                            const float (&gi)[ForceCfg<S>::TM ? 1 : S::NA][ForceCfg<S>::TM ? 1 : S::NLM],
                                            const float4 *fps, int i, bool live, int ii, int n,
                                            const float4 *__restrict__ pos, const int32_t *__restrict__ nbr,
                                            RowSpan sp, int nb0, const GT *__restrict__ G, uint32_t *ring_e, float4 *ring_p,
                                            unsigned long long *__restrict__ Ffix, int *__restrict__ status,
                                            float *__restrict__ Ff, long long (&acc)[13]) {
  constexpr bool TM = ForceCfg<S>::TM;
  constexpr int W = GTraits<GT>::W;
  constexpr int DE = ForceCfg<S>::DE, DP = ForceCfg<S>::DP;
  const float4 pi = pos[ii];
  float fx = 0.f, fy = 0.f, fz = 0.f;
  float wxx = 0.f, wxy = 0.f, wxz = 0.f, wyy = 0.f, wyz = 0.f, wzz = 0.f;
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
      float c;
      float fpi[8];
      {
        const float4 a = fps[0], b = fps[FORCE_BLOCK];
        fpi[0] = a.x; fpi[1] = a.y; fpi[2] = a.z; fpi[3] = a.w; fpi[4] = b.x; fpi[5] = b.y; fpi[6] = b.z; fpi[7] = b.w;
      }
      if constexpr (FULL) {
        c = dot_pairs<S::KR>(*reinterpret_cast<const float(*)[S::KR]>(&fpi[0]), df);
      } else {
        float fpj[8], fs[S::KR];
        load_tail8(G + (size_t)j * S::GS, S::NA * S::NLM, fpj);
#pragma unroll
        for (int k = 0; k < S::KR; k += 2) {
          const float2 t = add2(pr(fpi[k], fpi[k + 1]), pr(fpj[k], fpj[k + 1]));
          fs[k] = t.x; fs[k + 1] = t.y;
        }
        c = dot_pairs<S::KR>(fs, df);
      }
      coef = c * ir;
      if (COUNT) ++nrad;
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
      const bool si = TM && !ang;
      float2 al, gv[3];
      angular_pair<S, GT, FULL>(P, trow, gi, G + (size_t)(si ? ii : j) * S::GS, si, r, ir, dx, dy, dz, al, gv);
      if (ang) {
        if (COUNT) ++nang;
        coef = fmaf(hsum(al), ir, coef);
        vx = hsum(gv[0]) * ir; vy = hsum(gv[1]) * ir; vz = hsum(gv[2]) * ir;
      }
    }
    if (act) {
      if (COUNT) ++nact;
      const float Dx = fmaf(coef, dx, vx), Dy = fmaf(coef, dy, vy), Dz = fmaf(coef, dz, vz);
      fx += Dx; fy += Dy; fz += Dz;
      // Newton's third law: F_j -= D_ij, accumulated in fixed point (order-independent sum)
      if constexpr (FS) {
        atomicAdd(Ff + j, -Dx); atomicAdd(Ff + (size_t)n + j, -Dy); atomicAdd(Ff + 2 * (size_t)n + j, -Dz);
      } else {
        red_add(Ffix + j, -to_fix32(Dx));
        red_add(Ffix + (size_t)n + j, -to_fix32(Dy));
        red_add(Ffix + 2 * (size_t)n + j, -to_fix32(Dz));
      }
      wxx = fmaf(dx, Dx, wxx); wxy = fmaf(dx, Dy, wxy); wxz = fmaf(dx, Dz, wxz);
      wyy = fmaf(dy, Dy, wyy); wyz = fmaf(dy, Dz, wyz); wzz = fmaf(dz, Dz, wzz);
    }
  }
  pipe.finish();
  if (live) {
    if constexpr (FS) {
      atomicAdd(Ff + i, fx); atomicAdd(Ff + (size_t)n + i, fy); atomicAdd(Ff + 2 * (size_t)n + i, fz);
    } else {
      red_add(Ffix + i, to_fix32(fx));
      red_add(Ffix + (size_t)n + i, to_fix32(fy));
      red_add(Ffix + 2 * (size_t)n + i, to_fix32(fz));
    }
    if (!(isfinite(fx) && isfinite(fy) && isfinite(fz))) atomicOr(status, ST_NAN);
    // W = -sum over the evaluated pairs of r_ij (x) d_ij (or D_ij), upper triangle mirrored
    acc[0] = -to_fix32(wxx); acc[1] = -to_fix32(wxy); acc[2] = -to_fix32(wxz);
    acc[3] = acc[1]; acc[4] = -to_fix32(wyy); acc[5] = -to_fix32(wyz);
    acc[6] = acc[2]; acc[7] = acc[5]; acc[8] = -to_fix32(wzz);
    if (COUNT) { acc[9] = cnt; acc[10] = nact; acc[11] = nrad; acc[12] = nang; }
  }
}

// Radial and LJ part of one active pair's force coefficient (d = coef * r_ij + angular part): the
// radial adjoint in basis space (8 values in shared memory at fps[0], fps[FORCE_BLOCK], in
// radial_tail_td's form) against the basis derivatives, plus half of the shifted-force LJ pair force.  INSIDE_RC: the caller knows that
// r < rc_R (an angular pair: rc_A <= rc_R is checked by nep_create).
template <class S, bool INSIDE_RC = false>
__device__ __forceinline__ float radial_lj_coef(const Model<S> &P, const float4 *fps, float r2, float r, float ir) {
  float coef = 0.f;
  if (INSIDE_RC || r2 < P.rcR2) {
    // sum_k tail_k f_k' = dh (sum_k tail_k T_k + sum_k tail_k) + dxh sum_k tail_k D_k, the first sum
    // with the tail in radial_tail_td's form (tail_0 + sum_k tail_k at k = 0, T_0 = 1)
    float dh, dxh, T[S::KR], D[S::KR];
    cheb_td<S::KR>(r, P.inv_rcR, dh, dxh, T, D);
    float fpi[8];
    const float4 a = fps[0], b = fps[FORCE_BLOCK];
    fpi[0] = a.x; fpi[1] = a.y; fpi[2] = a.z; fpi[3] = a.w; fpi[4] = b.x; fpi[5] = b.y; fpi[6] = b.z; fpi[7] = b.w;
    const float(&tl)[S::KR] = *reinterpret_cast<const float(*)[S::KR]>(&fpi[0]);
    coef = fmaf(dh, dot_pairs<S::KR>(tl, T), dxh * dot_pairs<S::KR>(tl, D)) * ir;
  }
  if (P.lj_on != 0.f && r2 < P.lj_rc2) {
    float el, dl;
    lj_pair<S>(P, r2, r, ir, el, dl);
    coef = fmaf(0.5f * dl, ir, coef);
  }
  return coef;
}

// The force pass of the fused kernel over the pair records of its own descriptor walk (PairCache):
// first the na angular pairs (slots 0..na-1; warp-collective TMEM reads of the own adjoint row, so the
// loop runs to the warp's largest na and lanes past their own count compute a stand-in pair), then the
// nr other active pairs (slots pmax-1 down to pmax-nr; no TMEM).  Each pair gets the arithmetic of
// force_pairs<S, float, false, true> on the displacement the descriptor walk computed: d_ij added to F_i,
// subtracted from F_j (fixed point), W -= r_ij (x) d_ij (upper triangle, mirrored).  UN: the TMEM row is
// over Ph_lm (angular_pair).  The radial tail at fps is in radial_tail_td's form.
template <class S, int DQ, bool UN = false>
__device__ __forceinline__ void force_pairs_rec(const Model<S> &P, uint32_t trow,
                                                const float (&gi)[ForceCfg<S>::TM ? 1 : S::NA][ForceCfg<S>::TM ? 1 : S::NLM],
                                                const float4 *fps, int i, bool live,
                                                int n, const float4 *rec, unsigned off, int pmax, int na, int nr,
                                                float4 *ring,
                                                unsigned long long *__restrict__ Ffix, int *__restrict__ status,
                                                long long (&acc)[13]) {
  constexpr bool TM = ForceCfg<S>::TM;
  float fx = 0.f, fy = 0.f, fz = 0.f;
  float wxx = 0.f, wxy = 0.f, wxz = 0.f, wyy = 0.f, wyz = 0.f, wzz = 0.f;
  auto apply = [&](float dx, float dy, float dz, int j, float coef, float vx, float vy, float vz) {
    const float Dx = fmaf(coef, dx, vx), Dy = fmaf(coef, dy, vy), Dz = fmaf(coef, dz, vz);
    fx += Dx; fy += Dy; fz += Dz;
    long long ox, oy, oz;
    to_fix32x3(-Dx, -Dy, -Dz, ox, oy, oz);
    red_add(Ffix + j, ox);
    red_add(Ffix + (size_t)n + j, oy);
    red_add(Ffix + 2 * (size_t)n + j, oz);
    wxx = fmaf(dx, Dx, wxx); wxy = fmaf(dx, Dy, wxy); wxz = fmaf(dx, Dz, wxz);
    wyy = fmaf(dy, Dy, wyy); wyz = fmaf(dy, Dz, wyz); wzz = fmaf(dz, Dz, wzz);
  };
  {
    RecPipe<DQ, FORCE_BLOCK, FORCE_BLOCK> pa;
    pa.start(ring, rec, off, na);
    // with the row in TMEM the loop runs to the warp's largest count (warp-collective reads)
    const int trip = TM ? __reduce_max_sync(0xffffffffu, na) : na;
    for (int p = 0; p < trip; ++p) {
      const bool valid = p < na;
      float4 q = make_float4(1.f, 0.f, 0.f, 0.f);
      if (valid) q = pa.get(p);
      const float r2 = q.x * q.x + q.y * q.y + q.z * q.z;
      const float ir = rsqrtf(r2);
      const float r = r2 * ir;
      float coef = valid ? radial_lj_coef<S, true>(P, fps, r2, r, ir) : 0.f;
      if constexpr (TM) __syncwarp();
      float2 al, gv[3];
      angular_pair<S, float, true, UN>(P, trow, gi, static_cast<const float *>(nullptr), !valid, r, ir, q.x, q.y, q.z,
                                       al, gv);
      if (valid) {
        coef = fmaf(hsum(al), ir, coef);
        apply(q.x, q.y, q.z, __float_as_int(q.w), coef, hsum(gv[0]) * ir, hsum(gv[1]) * ir, hsum(gv[2]) * ir);
      }
    }
    pa.finish();
  }
  {
    RecPipe<DQ, FORCE_BLOCK, -FORCE_BLOCK> pb;
    pb.start(ring, rec, off + (unsigned)(pmax - 1) * FORCE_BLOCK, nr);
    int p0 = 0;
    // two records per iteration: geometry, basis derivatives, the radial-adjoint dot and the LJ
    // derivative in float2 pairs (the teacher's kernels 0.8 % faster than one at a time, the student's
    // 1.8 % slower); an odd last record alone below
    if constexpr (TM) {
      const float4 ta = fps[0], tb = fps[FORCE_BLOCK];
      const float tail[8] = {ta.x, ta.y, ta.z, ta.w, tb.x, tb.y, tb.z, tb.w};
      for (; p0 + 1 < nr; p0 += 2) {
        const float4 qa = pb.get(p0), qb = pb.get(p0 + 1);
        const float2 dxv = pr(qa.x, qb.x), dyv = pr(qa.y, qb.y), dzv = pr(qa.z, qb.z);
        const float2 r2 = fma2(dzv, dzv, fma2(dyv, dyv, mul2(dxv, dxv)));
        const float2 ir = pr(rsqrtf(r2.x), rsqrtf(r2.y));
        const float2 r = mul2(r2, ir);
        float2 coef = bc2(0.f);
        const bool ra = r2.x < P.rcR2, rb = r2.y < P.rcR2;
        if (ra || rb) {
          // the contraction of radial_lj_coef: dh (sum tail_k T_k) + dxh (sum tail_k D_k), T_0 = D_1 = 1
          float2 dh, dxh, T[S::KR], D[S::KR];
          cheb_td_x2<S::KR>(r, P.inv_rcR, dh, dxh, T, D);
          float2 s1 = bc2(tail[0]), s2 = bc2(tail[1]);
#pragma unroll
          for (int k = 1; k < S::KR; ++k) s1 = fma2(bc2(tail[k]), T[k], s1);
#pragma unroll
          for (int k = 2; k < S::KR; ++k) s2 = fma2(bc2(tail[k]), D[k], s2);
          const float2 dot = mul2(fma2(dh, s1, mul2(dxh, s2)), ir);
          coef = pr(ra ? dot.x : 0.f, rb ? dot.y : 0.f);
        }
        if (P.lj_on != 0.f) {
          const bool la = r2.x < P.lj_rc2, lb = r2.y < P.lj_rc2;
          if (la || lb) {
            const float2 dl = lj_deriv_x2<S>(P, r2, ir);
            const float2 t = mul2(mul2(bc2(0.5f), dl), ir);
            coef = add2(coef, pr(la ? t.x : 0.f, lb ? t.y : 0.f));
          }
        }
        apply(qa.x, qa.y, qa.z, __float_as_int(qa.w), coef.x, 0.f, 0.f, 0.f);
        apply(qb.x, qb.y, qb.z, __float_as_int(qb.w), coef.y, 0.f, 0.f, 0.f);
      }
    }
    for (int p = p0; p < nr; ++p) {
      const float4 q = pb.get(p);
      const float r2 = q.x * q.x + q.y * q.y + q.z * q.z;
      const float ir = rsqrtf(r2);
      const float r = r2 * ir;
      apply(q.x, q.y, q.z, __float_as_int(q.w), radial_lj_coef<S>(P, fps, r2, r, ir), 0.f, 0.f, 0.f);
    }
    pb.finish();
  }
  if (live) {
    red_add(Ffix + i, to_fix32(fx));
    red_add(Ffix + (size_t)n + i, to_fix32(fy));
    red_add(Ffix + 2 * (size_t)n + i, to_fix32(fz));
    if (!(isfinite(fx) && isfinite(fy) && isfinite(fz))) atomicOr(status, ST_NAN);
    acc[0] = -to_fix32(wxx); acc[1] = -to_fix32(wxy); acc[2] = -to_fix32(wxz);
    acc[3] = acc[1]; acc[4] = -to_fix32(wyy); acc[5] = -to_fix32(wyz);
    acc[6] = acc[2]; acc[7] = acc[5]; acc[8] = -to_fix32(wzz);
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
  __shared__ float4 fp_s[2 * FORCE_BLOCK];
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
  if constexpr (TM) {
    // chunked TMEM layout (tm_col): chunk k = components 4k..4k+3 of every channel
#pragma unroll
    for (int k = 0; k < S::NLM / 4; ++k) {
      float v[S::NA][4];
#pragma unroll
      for (int a = 0; a < S::NA; ++a) {
        if constexpr (W == 4) {
          load_vec(Gi + a * S::NLM + 4 * k, v[a]);
        } else {
          float t[W];
          load_vec(Gi + a * S::NLM + (4 * k / W) * W, t);
#pragma unroll
          for (int cc = 0; cc < 4; ++cc) v[a][cc] = t[(4 * k) % W + cc];
        }
      }
      tm_store<S, S::NA>(trow, k, v);
    }
    tmem_wait_st();
  } else {
#pragma unroll
    for (int a = 0; a < S::NA; ++a)
#pragma unroll
      for (int c = 0; c < S::NLM; c += W) {
        float t[W];
        load_vec(Gi + a * S::NLM + c, t);
#pragma unroll
        for (int k = 0; k < W; ++k) gi[a][c + k] = t[k];
      }
  }
  {
    float fpi[8];
    load_tail8(Gi, S::NA * S::NLM, fpi);
    fp_s[threadIdx.x] = make_float4(fpi[0], fpi[1], fpi[2], fpi[3]);
    fp_s[FORCE_BLOCK + threadIdx.x] = make_float4(fpi[4], fpi[5], fpi[6], fpi[7]);
  }
  const bool skip = skip_far(X);
  const RowSpan sp = !live ? RowSpan{0, 0, 0} : (FULL ? full_row(X, i, skip) : owned_row(X, i, skip));
  force_pairs<S, GT, FS, FULL>(P, shift, trow, gi, fp_s + threadIdx.x, i, live, ii, n, pos, nbr, sp,
                               live ? X.nband0[i] : 0, G, ring_e, ring_p, Ffix, status, Ff, acc);
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
// in TMEM, turned into the adjoint row in place, and the force pass evaluates every active pair again
// with it, so no adjoint row goes through HBM and one launch (and its tail wave) is saved.  The
// descriptor walk records each active pair's displacement and neighbour (PairCache; L2-resident
// regions reused block after block), so the force pass reads 16 bytes per active pair in order instead
// of walking the neighbour list a second time.  The forces are scattered with atomics into Ffix, which
// the caller zeroes before the launch (a block may add to F_j before atom j's own block has started).
#ifndef NEP_FUSED_MINB
#define NEP_FUSED_MINB 4
#endif
template <class S>
__global__ void __launch_bounds__(DESC_BLOCK, NEP_FUSED_MINB)
k_nep_fused(const __grid_constant__ Model<S> P, const Geom geom, const int n, const float4 *__restrict__ pos,
            const int32_t *__restrict__ nbr, const RowExt X, float *__restrict__ usite,
            float *__restrict__ qout, unsigned long long *__restrict__ Ffix, long long *__restrict__ part_d,
            long long *__restrict__ part_f, int *__restrict__ status, const PairCache pc) {
  static_assert(ForceCfg<S>::TM && DESC_BLOCK == 128 && FORCE_BLOCK == 128, "teacher shape, 4 warps");
  constexpr int W = TMEM_W;
  constexpr uint32_t TCOLS = 128;
  static_assert(PC_SLOTS * TCOLS == 512, "at most PC_SLOTS blocks per SM: one pair-record slot each");
  __shared__ float4 shift[27];
  __shared__ uint32_t ring_e[PIPE_DE * DESC_BLOCK];
  __shared__ float4 ring_p[PIPE_DP * DESC_BLOCK];
  __shared__ uint32_t tmem_base;
  __shared__ __align__(16) NetSmem<S> net;
  __shared__ float4 fp_s[2 * DESC_BLOCK];
  __shared__ int s_slot;
  if (threadIdx.x < 32) tmem_alloc(&tmem_base, TCOLS);
  if (threadIdx.x == 0) {
    // one free pair-record slot of this SM (at most PC_SLOTS blocks of this kernel are resident here)
    const int slot = acquire_record_slot(pc);
    if (slot < 0) atomicOr(status, ST_SLOT);   // results of this evaluation are then reported invalid
    __threadfence();
    s_slot = slot;
  }
  tc_fence_before();
  fill_shift_table(shift, geom);
  stage_network(P, net);
  __syncthreads();
  tc_fence_after();
  const int slot = s_slot;
  // element offset of this thread's record column; without a slot (reported above) the block still
  // writes only inside the array, to slot 0
  const unsigned rec_off = (unsigned)(slot < 0 ? 0 : slot) * (unsigned)pc.pmax * DESC_BLOCK + threadIdx.x;
  const uint32_t trow = tmem_base + ((uint32_t)(threadIdx.x & ~31u) << 16);
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const bool live = i < n;
  const int ii = live ? i : 0;
  const RowSpan sp = live ? full_row(X, i, skip_far(X)) : RowSpan{0, 0, 0};
  const int cnt = sp.c;

  // descriptors and network (as k_descriptor_tm), recording the active pairs
  float QR[S::KR], elj;
  int nrad, nang, nact;
  RegSums<S, S::NA> R;
  accumulate_atom_tm<S, S::NA, PIPE_DE, PIPE_DP, DESC_BLOCK, true, true>(P, shift, trow, ii, n, pos, nbr, sp, ring_e,
                                                                         ring_p, QR, R, elj, nrad, nang, nact, pc.rec,
                                                                         rec_off, pc.pmax);
  float q[S::NDES];
  FourBody<S> T;
  descriptors_tm<S, S::NA, true>(P, trow, QR, R, q, T);
  if (live && qout != nullptr) {
#pragma unroll
    for (int v = 0; v < S::NDES; ++v) qout[(size_t)i * S::NDES + v] = q[v];
  }
  float Fp[S::NDES];
  const float U = network_smem<S>(P, net, q, false, Fp);

  // the adjoint row replaces the sums in TMEM (same columns, chunk by chunk); radial tail in registers
  float g4[S::NA][5];
  fourbody_adjoint_tm<S, S::NA, true>(trow, R, g4);
#pragma unroll
  for (int k = 0; k < S::NLM / W; ++k) {
    float sv[S::NA][W], gl[S::NA][W];
    sums_chunk<S, S::NA>(trow, k, R, sv);
#pragma unroll
    for (int a = 0; a < S::NA; ++a) adjoint_chunk<S, true>(a, W * k, sv[a], g4[a], Fp, gl[a]);
    tm_store<S, S::NA>(trow, k, gl);
  }
  tmem_wait_st();
  {
    float fpi[8];
    radial_tail<S>(P, Fp, fpi);
    radial_tail_td(fpi);                 // the force pass's form (force_pairs_rec)
    fp_s[threadIdx.x] = make_float4(fpi[0], fpi[1], fpi[2], fpi[3]);
    fp_s[DESC_BLOCK + threadIdx.x] = make_float4(fpi[4], fpi[5], fpi[6], fpi[7]);
  }
  long long acc_d[5] = {0, 0, 0, 0, 0};
  long long acc_f[13] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
  if (live) {
    const float ui = U + elj;
    usite[i] = ui;
    if (!isfinite(ui)) atomicOr(status, ST_NAN);
    acc_d[0] = to_fix32(ui);
    acc_d[1] = nrad;
    acc_d[2] = nang;
    acc_d[3] = cnt;
    acc_d[4] = nact;
    // the force pass visits the descriptor walk's active pairs
    acc_f[9] = cnt; acc_f[10] = nact; acc_f[11] = nrad; acc_f[12] = nang;
  }
  // the energy and counters: summed over the warp now (fewer live registers in the force pass), over
  // the block after the closing barrier
  __shared__ long long wsum_d[DESC_BLOCK / 32][5];
  warp_sum_stage<5>(acc_d, wsum_d[threadIdx.x >> 5]);

  // forces: every active pair of the row with the own adjoint row, from the pair records
  const float gi[1][1] = {{0.f}};
  force_pairs_rec<S, PIPE_DP, true>(P, trow, gi, fp_s + threadIdx.x, i, live, n, pc.rec, rec_off, pc.pmax, nang,
                                    nact - nang, ring_p, Ffix, status, acc_f);
  tc_fence_before();
  __syncthreads();
  if (threadIdx.x < 32) {
    tc_fence_after();
    tmem_dealloc(tmem_base, TCOLS);
  }
  if (threadIdx.x == 0 && slot >= 0) {
    __threadfence();          // this block's record reads are complete (cp.async waited, barrier above)
    atomicAnd(pc.slot_mask + slot / pc.slots, ~(1u << (slot % pc.slots)));
  }
  block_store_staged<5, DESC_BLOCK / 32>(wsum_d, part_d);
  block_sum_store<13, DESC_BLOCK / 32>(acc_f, part_f);
}

// The fused kernel for shapes whose per-atom row fits in registers (the distilled student: 4 x 8
// angular sums, 32-value adjoint row): descriptors, network and full-row forces of 128 atoms per block
// with no tensor memory, so every thread walks its own row (no warp-collective steps).  The descriptor
// walk records the active pairs (PairCache, PC_SLOTS_REG regions per SM: the launch checks that no more
// blocks are resident), the adjoint row stays in registers and the force pass reads the records.  With
// the fallback on, an atom whose descriptors leave the training range is flagged as in k_descriptor
// (zero adjoint row, LJ energy only), and the teacher kernels then add its own model's part.  Ffix is
// zeroed by the caller before the launch.  Five resident blocks (at most 102 registers) measured 4 %
// faster than four.
#ifndef NEP_FUSED_REG_MINB
#define NEP_FUSED_REG_MINB 5
#endif
template <class S>
__global__ void __launch_bounds__(DESC_BLOCK, NEP_FUSED_REG_MINB)
k_nep_fused_reg(const __grid_constant__ Model<S> P, const Geom geom, const int n, const float4 *__restrict__ pos,
                const int32_t *__restrict__ nbr, const RowExt X, float *__restrict__ usite,
                float *__restrict__ qout, unsigned long long *__restrict__ Ffix, long long *__restrict__ part_d,
                long long *__restrict__ part_f, int *__restrict__ status, const __grid_constant__ Fallback fb,
                const PairCache pc) {
  static_assert(!ForceCfg<S>::TM && DESC_BLOCK == FORCE_BLOCK, "register-resident rows");
  __shared__ float4 shift[27];
  __shared__ uint32_t ring_e[PIPE_DE * DESC_BLOCK];
  __shared__ float4 ring_p[PIPE_DP * DESC_BLOCK];
  __shared__ float4 fp_s[2 * DESC_BLOCK];
  __shared__ int s_slot;
  if (threadIdx.x == 0) {
    const int slot = acquire_record_slot(pc);
    if (slot < 0) atomicOr(status, ST_SLOT);   // results of this evaluation are then reported invalid
    __threadfence();
    s_slot = slot;
  }
  fill_shift_table(shift, geom);
  __syncthreads();
  const int slot = s_slot;
  const unsigned rec_off = (unsigned)(slot < 0 ? 0 : slot) * (unsigned)pc.pmax * DESC_BLOCK + threadIdx.x;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  long long acc_d[5] = {0, 0, 0, 0, 0};
  long long acc_f[13] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
  if (i < n) {
    AtomSums<S> A;
    accumulate_atom<S, PIPE_DE, PIPE_DP, DESC_BLOCK, true, true>(P, shift, i, n, pos, nbr, full_row(X, i, skip_far(X)),
                                                           ring_e, ring_p, A, pc.rec, rec_off, pc.pmax);
    float q[S::NDES];
    FourBody<S> T;
    descriptors_of<S, true>(P, A, q, T);
    if (qout != nullptr) {
#pragma unroll
      for (int v = 0; v < S::NDES; ++v) qout[(size_t)i * S::NDES + v] = q[v];
    }
    const bool flagged = fb.on && out_of_range<S>(fb, P, q);
    if (flagged) flag_atom(fb, i, status);
    float Fp[S::NDES];
    const float U = network<S>(P, q, flagged, Fp);   // flagged: no U_i from this model, Fp = 0
    float gi[S::NA][S::NLM];
#pragma unroll
    for (int a = 0; a < S::NA; ++a) adjoint_channel<S, true>(a, A, T, Fp, gi[a]);
    {
      float tail[8];
      radial_tail<S>(P, Fp, tail);
      radial_tail_td(tail);              // the force pass's form (force_pairs_rec)
      fp_s[threadIdx.x] = make_float4(tail[0], tail[1], tail[2], tail[3]);
      fp_s[DESC_BLOCK + threadIdx.x] = make_float4(tail[4], tail[5], tail[6], tail[7]);
    }
    const float ui = flagged ? A.elj : U + A.elj;
    usite[i] = ui;
    if (!isfinite(ui)) atomicOr(status, ST_NAN);
    acc_d[0] = to_fix32(ui);
    acc_d[1] = A.nrad;
    acc_d[2] = A.nang;
    acc_d[3] = A.cnt;
    acc_d[4] = A.nact;
    acc_f[9] = A.cnt; acc_f[10] = A.nact; acc_f[11] = A.nrad; acc_f[12] = A.nang;
    force_pairs_rec<S, PIPE_DP, true>(P, 0u, gi, fp_s + threadIdx.x, i, true, n, pc.rec, rec_off, pc.pmax, A.nang,
                                A.nact - A.nang, ring_p, Ffix, status, acc_f);
  }
  __syncthreads();
  if (threadIdx.x == 0 && slot >= 0) {
    __threadfence();          // this block's record reads are complete (cp.async waited, barrier above)
    atomicAnd(pc.slot_mask + slot / pc.slots, ~(1u << (slot % pc.slots)));
  }
  block_sum_store<5, DESC_BLOCK / 32>(acc_d, part_d);
  block_sum_store<13, DESC_BLOCK / 32>(acc_f, part_f);
}

// Mixed-precision form of the fused kernel: the same descriptor walk (pair records), float32 adjoint
// row in TMEM and force pass over the records, with the one-hidden-layer network as two GEMMs on the
// 5th-generation tensor cores, one CTA = one 128-atom tile = the M of one tcgen05.mma:
//   forward   Z[128 x 32]  = Q~[128 x 32] . W0^T    (MT = bf16 or f16 operands, f32 accumulation)
//   backward  dQ[128 x 32] = T[128 x 32] . W0       T_mu = w1_mu (1 - tanh(z_mu - b0_mu)^2)
// (the batched network GEMM of Section V.B, Optimization 1, in the half-precision network input of
// Optimization 4).  The walk is the float32 kernel's (all 120 sums in TMEM); for the GEMMs the 24 sums
// of angular channel 4 move to registers, so that TMEM columns 96..127 take the GEMM accumulators, and
// afterwards channel 4's adjoint goes back to columns 96..119 (the layout of tm_col), over the consumed
// GEMM result (each warp only touches its own 32 lanes, after its own load of them completed).  The A
// tile (q~ rows, then T rows) has its own shared memory, so each thread writes its row as soon as its
// descriptors are known; one barrier precedes each GEMM.  Every wait on the tensor core is bounded
// (ST_TIMEOUT on expiry).
constexpr int FM_K = 32;             // descriptors padded to 32 (two K = 16 steps)
constexpr int FM_N = 32;             // neurons padded to 32
constexpr long FM_WAIT = 1L << 22;   // mbarrier polls before giving up

template <class S, class MT>
__global__ void __launch_bounds__(DESC_BLOCK, NEP_FUSED_MINB)
k_nep_fused_mixed(const __grid_constant__ Model<S> P, const Geom geom, const int n, const float4 *__restrict__ pos,
                  const int32_t *__restrict__ nbr, const RowExt X, float *__restrict__ usite,
                  float *__restrict__ qout, unsigned long long *__restrict__ Ffix, long long *__restrict__ part_d,
                  long long *__restrict__ part_f, int *__restrict__ status, const PairCache pc) {
  static_assert(ForceCfg<S>::TM && DESC_BLOCK == 128 && S::NDES <= FM_K && S::NNEU <= FM_N, "teacher shape");
  constexpr int NT = 4;
  constexpr int W = TMEM_W;
  constexpr uint32_t TCOLS = 128;
  constexpr uint32_t GCOL = NT * S::NLM;   // GEMM accumulator columns 96..127
  static_assert(GCOL + FM_N <= TCOLS && tm_col(4, 0, S::NLM) == GCOL, "channel 4's adjoint takes the GEMM columns");
  static_assert(PC_SLOTS * TCOLS == 512, "at most PC_SLOTS blocks per SM: one pair-record slot each");
  __shared__ float4 shift[27];
  __shared__ uint32_t ring_e[PIPE_DE * DESC_BLOCK];
  __shared__ float4 ring_p[PIPE_DP * DESC_BLOCK];
  __shared__ __align__(1024) MT sA[DESC_BLOCK * FM_K];
  __shared__ __align__(1024) MT sW[FM_N * FM_K];    // B of the forward GEMM: W0[neuron][descriptor]
  __shared__ __align__(1024) MT sWt[FM_K * FM_N];   // B of the backward GEMM: W0[descriptor][neuron]
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_base;
  __shared__ float4 fp_s[2 * DESC_BLOCK];
  __shared__ int s_slot;
  const int t = threadIdx.x;
  if (t < 32) {
    for (int k = 0; k < FM_K; ++k) {
      sW[tile_off(t, k, FM_K / 8)] = to_mma_type<MT>((t < S::NNEU && k < S::NDES) ? P.W0[t][k] : 0.f);
      sWt[tile_off(t, k, FM_K / 8)] = to_mma_type<MT>((t < S::NDES && k < S::NNEU) ? P.W0[k][t] : 0.f);
    }
    tmem_alloc(&tmem_base, TCOLS);
  }
  if (t == 0) {
    mbar_init(&mbar, 1);
    const int slot = acquire_record_slot(pc);
    if (slot < 0) atomicOr(status, ST_SLOT);
    __threadfence();
    s_slot = slot;
  }
  tc_fence_before();
  fill_shift_table(shift, geom);
  __syncthreads();
  tc_fence_after();
  const int slot = s_slot;
  const unsigned rec_off = (unsigned)(slot < 0 ? 0 : slot) * (unsigned)pc.pmax * DESC_BLOCK + t;
  const uint32_t trow = tmem_base + ((uint32_t)(t & ~31) << 16);
  const int i = blockIdx.x * DESC_BLOCK + t;
  const bool live = i < n;
  const int ii = live ? i : 0;
  const RowSpan sp = live ? full_row(X, i, skip_far(X)) : RowSpan{0, 0, 0};
  const int cnt = sp.c;

  float QR[S::KR], elj;
  int nrad, nang, nact;
  float q[S::NDES];
  {
    RegSums<S, S::NA> R5;
    accumulate_atom_tm<S, S::NA, PIPE_DE, PIPE_DP, DESC_BLOCK, true, true>(P, shift, trow, ii, n, pos, nbr, sp, ring_e, ring_p,
                                                                     QR, R5, elj, nrad, nang, nact, pc.rec, rec_off,
                                                                     pc.pmax);
    FourBody<S> T;
    descriptors_tm<S, S::NA, true>(P, trow, QR, R5, q, T);   // zero for threads past the last atom (empty row)
  }
  // channel 4's sums (columns 96..119) to registers: the GEMMs take columns 96..127
  RegSums<S, NT> R;
  {
    uint32_t r[24];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%24];\n\t"
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%16, %17, %18, %19, %20, %21, %22, %23}, [%25];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23])
        : "r"(trow + GCOL), "r"(trow + GCOL + 16));
#pragma unroll
    for (int c = 0; c < S::NLM; ++c) R.s[0][c] = __uint_as_float(r[c]);
  }
  if (live && qout != nullptr) {
#pragma unroll
    for (int v = 0; v < S::NDES; ++v) qout[(size_t)i * S::NDES + v] = q[v];
  }
#pragma unroll
  for (int k = 0; k < FM_K; ++k) sA[tile_off(t, k, FM_K / 8)] = to_mma_type<MT>(k < S::NDES ? q[k] * P.qs[k] : 0.f);
  fence_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t idesc = umma_idesc_f16(DESC_BLOCK, FM_N, MmaKind<MT>::bf16);
  const uint32_t lbo = 128, sbo = (FM_K / 8) * 128;
  if (t == 0) {
#pragma unroll
    for (int ks = 0; ks < FM_K / 16; ++ks)
      umma_f16(tmem_base + GCOL, umma_smem_desc(smem_addr(sA) + ks * 256, lbo, sbo),
               umma_smem_desc(smem_addr(sW) + ks * 256, lbo, sbo), idesc, ks);
    umma_commit(&mbar);
  }
  bool ok = mbar_wait(&mbar, 0, FM_WAIT);
  tc_fence_after();
  float U = -P.b1;
  {
    float z[32];
    tmem_ld32(trow + GCOL, z);
    float tr[FM_N];
#pragma unroll
    for (int mu = 0; mu < FM_N; ++mu) {
      if (mu < S::NNEU) {
        const float h = tanh_sfu(z[mu] - P.b0[mu]);   // error 2^-11: below that of z (16-bit inputs)
        U = fmaf(P.w1[mu], h, U);
        tr[mu] = P.w1[mu] * (1.f - h * h);
      } else {
        tr[mu] = 0.f;
      }
    }
    // the forward MMA has completed (mbarrier), so its A tile can be overwritten
#pragma unroll
    for (int k = 0; k < FM_N; ++k) sA[tile_off(t, k, FM_N / 8)] = to_mma_type<MT>(tr[k]);
  }
  fence_async_smem();
  tc_fence_before();   // every thread has read the forward result before the backward GEMM overwrites it
  __syncthreads();
  tc_fence_after();
  if (t == 0) {
#pragma unroll
    for (int ks = 0; ks < FM_N / 16; ++ks)
      umma_f16(tmem_base + GCOL, umma_smem_desc(smem_addr(sA) + ks * 256, lbo, sbo),
               umma_smem_desc(smem_addr(sWt) + ks * 256, lbo, sbo), idesc, ks);
    umma_commit(&mbar);
  }
  ok = mbar_wait(&mbar, 1, FM_WAIT) && ok;
  tc_fence_after();
  float Fp[S::NDES];
  {
    float dq[32];
    tmem_ld32(trow + GCOL, dq);
#pragma unroll
    for (int v = 0; v < S::NDES; ++v) Fp[v] = dq[v] * P.qs[v];
  }
  if (!ok && t == 0) atomicOr(status, ST_TIMEOUT);

  // adjoint row of all 5 channels in the chunked layout: channels 0..3 over their sums, channel 4 over
  // the GEMM columns this warp has just read
  float g4[S::NA][5];
  fourbody_adjoint_tm<S, NT, true>(trow, R, g4);
#pragma unroll
  for (int k = 0; k < S::NLM / W; ++k) {
    float sv[S::NA][W], gl[S::NA][W];
    sums_chunk<S, NT>(trow, k, R, sv);
#pragma unroll
    for (int a = 0; a < S::NA; ++a) adjoint_chunk<S, true>(a, W * k, sv[a], g4[a], Fp, gl[a]);
    tm_store<S, S::NA>(trow, k, gl);
  }
  tmem_wait_st();
  {
    float fpi[8];
    radial_tail<S>(P, Fp, fpi);
    radial_tail_td(fpi);                 // the force pass's form (force_pairs_rec)
    fp_s[t] = make_float4(fpi[0], fpi[1], fpi[2], fpi[3]);
    fp_s[DESC_BLOCK + t] = make_float4(fpi[4], fpi[5], fpi[6], fpi[7]);
  }
  long long acc_d[5] = {0, 0, 0, 0, 0};
  long long acc_f[13] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
  if (live) {
    const float ui = U + elj;
    usite[i] = ui;
    if (!isfinite(ui)) atomicOr(status, ST_NAN);
    acc_d[0] = to_fix32(ui);
    acc_d[1] = nrad;
    acc_d[2] = nang;
    acc_d[3] = cnt;
    acc_d[4] = nact;
    acc_f[9] = cnt; acc_f[10] = nact; acc_f[11] = nrad; acc_f[12] = nang;
  }
  __shared__ long long wsum_d[DESC_BLOCK / 32][5];
  warp_sum_stage<5>(acc_d, wsum_d[t >> 5]);
  const float gi[1][1] = {{0.f}};
  force_pairs_rec<S, PIPE_DP, true>(P, trow, gi, fp_s + t, i, live, n, pc.rec, rec_off, pc.pmax, nang, nact - nang, ring_p,
                              Ffix, status, acc_f);
  tc_fence_before();
  __syncthreads();
  if (t < 32) {
    tc_fence_after();
    tmem_dealloc(tmem_base, TCOLS);
  }
  if (t == 0 && slot >= 0) {
    __threadfence();
    atomicAnd(pc.slot_mask + slot / pc.slots, ~(1u << (slot % pc.slots)));
  }
  block_store_staged<5, DESC_BLOCK / 32>(wsum_d, part_d);
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
                         long long *part_f, int *status, const PairCache &pc, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  const int grid = (n + DESC_BLOCK - 1) / DESC_BLOCK;
  k_nep_fused<S><<<grid, DESC_BLOCK, 0, st>>>(P, g, n, pos, nbr, X, usite, qout,
                                              reinterpret_cast<unsigned long long *>(Ffix), part_d, part_f, status, pc);
  return cudaGetLastError();
}
template cudaError_t launch_fused<CuShape>(const Model<CuShape> &, const Geom &, int, const float4 *, const int32_t *,
                                           const RowExt &, float *, float *, long long *, long long *, long long *,
                                           int *, const PairCache &, cudaStream_t);

// Fused evaluation of a register-resident shape (k_nep_fused_reg); Ffix must be zero.  Fails with
// cudaErrorInvalidConfiguration if more blocks than PC_SLOTS_REG could be resident on an SM.
template <class S>
cudaError_t launch_fused_reg(const Model<S> &P, const Geom &g, int n, const float4 *pos, const int32_t *nbr,
                             const RowExt &X, float *usite, float *qout, long long *Ffix, long long *part_d,
                             long long *part_f, int *status, const Fallback &fb, const PairCache &pc,
                             cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_nep_fused_reg<S>, DESC_BLOCK, 0);
  if (e != cudaSuccess) return e;
  if (per_sm > pc.slots) return cudaErrorInvalidConfiguration;
  const int grid = (n + DESC_BLOCK - 1) / DESC_BLOCK;
  k_nep_fused_reg<S><<<grid, DESC_BLOCK, 0, st>>>(P, g, n, pos, nbr, X, usite, qout,
                                                  reinterpret_cast<unsigned long long *>(Ffix), part_d, part_f,
                                                  status, fb, pc);
  return cudaGetLastError();
}
template cudaError_t launch_fused_reg<StudentShape>(const Model<StudentShape> &, const Geom &, int, const float4 *,
                                                    const int32_t *, const RowExt &, float *, float *, long long *,
                                                    long long *, long long *, int *, const Fallback &,
                                                    const PairCache &, cudaStream_t);

// Mixed-precision fused evaluation of the teacher (k_nep_fused_mixed); Ffix must be zero.
template <class S, class MT>
cudaError_t launch_fused_mixed(const Model<S> &P, const Geom &g, int n, const float4 *pos, const int32_t *nbr,
                               const RowExt &X, float *usite, float *qout, long long *Ffix, long long *part_d,
                               long long *part_f, int *status, const PairCache &pc, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  const int grid = (n + DESC_BLOCK - 1) / DESC_BLOCK;
  k_nep_fused_mixed<S, MT><<<grid, DESC_BLOCK, 0, st>>>(P, g, n, pos, nbr, X, usite, qout,
                                                        reinterpret_cast<unsigned long long *>(Ffix), part_d, part_f,
                                                        status, pc);
  return cudaGetLastError();
}
template cudaError_t launch_fused_mixed<CuShape, __nv_bfloat16>(const Model<CuShape> &, const Geom &, int,
                                                                const float4 *, const int32_t *, const RowExt &,
                                                                float *, float *, long long *, long long *,
                                                                long long *, int *, const PairCache &, cudaStream_t);
template cudaError_t launch_fused_mixed<CuShape, __half>(const Model<CuShape> &, const Geom &, int, const float4 *,
                                                         const int32_t *, const RowExt &, float *, float *,
                                                         long long *, long long *, long long *, int *,
                                                         const PairCache &, cudaStream_t);

// Records per SM bound of the pair cache: %nsmid of the current device (synchronous).
__global__ void k_sm_bound(int *out) { *out = (int)sm_index_bound(); }
cudaError_t pair_cache_sm_bound(int *nsm) {
  int *d = nullptr;
  cudaError_t e = cudaMalloc(&d, sizeof(int));
  if (e != cudaSuccess) return e;
  k_sm_bound<<<1, 1>>>(d);
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpy(nsm, d, sizeof(int), cudaMemcpyDeviceToHost);
  cudaFree(d);
  return e;
}
// Pair records per region: one float4 per record, DESC_BLOCK threads.
size_t pair_cache_region_elems(int pmax) { return (size_t)pmax * DESC_BLOCK; }

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
