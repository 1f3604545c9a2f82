// nep_common.cuh -- device-side building blocks shared by the NEP kernels (sm_103a).
//
// Layout conventions (all per-atom arrays in cell-sorted order):
//   pos[i]   float4: position relative to the origin of the atom's cell at the last rebuild (x, y, z)
//            and the packed cell coordinates (w, as int bits: cx | cy << 10 | cz << 20).
//   nbr      int32 [cap][N] (neighbour-major, so a thread per atom reads coalesced rows); entry =
//            j | shift << 27, shift = (dx+1) + 3 (dy+1) + 9 (dz+1) the cell offset of j's image.
//            Row i = [pairs owned by i | the others], each part grouped by distance band; nown[i]
//            is the length of the owned part.
//   Ffix     int64 [3][N]: forces in fixed point (2^-32 eV/Angstrom units), accumulated with
//            integer atomics, so the sum does not depend on the order of the additions.
//   G        float or half [N][S::GS]: per-atom adjoint dU_i/ds_nlm (NA * NLM values, index n * NLM + lm)
//            followed by the radial adjoint in basis space dU_i/dQ_k = sum_n dU_i/dq_n cR_nk (KR <= 8
//            values, Q_k = sum_j f_k(r_ij) the radial basis sums) and padding
//            (teacher shape: 5 x 24 + 8 = 128 per row; student shape: 4 x 8 + 8 = 40).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace nep {

constexpr int J_BITS = 27;
constexpr uint32_t J_MASK = (1u << J_BITS) - 1u;
constexpr float FIX_SCALE = 4294967296.0f;        // 2^32 fixed-point units per eV/Angstrom
constexpr double FIX_INV = 1.0 / 4294967296.0;

// Status bits of the device status word.
enum : int {
  ST_OVERFLOW = 1,   // neighbour list capacity exceeded
  ST_NAN = 2,        // non-finite value seen
  ST_FB_OVERFLOW = 8, // more atoms flagged for the fallback model than its list holds
  ST_SLOT = 16        // a block found no free pair-record slot on its SM (not expected: see PairCache)
};

// The far band of a neighbour-list row starts at rc_R + FAR_EDGE * skin.  For fcc Cu at rc_R = 5 A and
// a 1 A skin this edge (5.4 A) lies between the 5.11 A and 5.72 A shells, so every atom's far band is
// the same shell and the walked rows stay aligned across the lanes of a warp; an edge inside a shell's
// thermal spread gives neighbouring atoms walked counts that differ by one or two, which misaligns the
// lanes' bands and costs more than the skipped entries save.
constexpr float FAR_EDGE = 0.4f;

// Device-side control block (one per handle).
struct Control {
  int status;           // OR of ST_* bits
  int moved;            // some atom moved more than skin/2 since the last rebuild
  int do_rebuild;       // decision of the current step
  int force_rebuild;    // host request
  int steps_since;      // MD steps since the last rebuild
  int rebuild_every;    // 0 = displacement-triggered only
  long long rebuilds;   // neighbour builds done
  long long steps;      // MD steps done
  int nb_next;          // next group of atoms for the neighbour scan (reset by each rebuild)
  float dmax2;          // largest squared displacement of an atom since the last rebuild (Angstrom^2)
  float far_dmax2;      // below this, no list entry of the far band can be inside the largest cutoff
  int skip_far;         // decision for the current evaluation: row walks may skip the far band
  int changed;          // an upload into the kept cell order changed some atom's float32 position
  int pending;          // the last MD step's closing half kick is still owed (applied by the next step's
                        // opening kick, or by the kick that ends md_verlet_step)
};

// Arguments of the rebuild chain (cell sort + neighbour list).
struct RebuildArgs {
  int n, ncell;
  double L[3], l[3];
  int nc[3];
  double *x, *y, *z, *vx, *vy, *vz, *xb, *yb, *zb, *vxb, *vyb, *vzb;
  int *id, *idb, *cell_of, *count, *cursor, *start, *tile_sums, *perm;
  float4 *pos, *pos_ref;
  int32_t *nbr, *nnum, *nang, *nown, *nband0, *nfar;
  int cap;
  float rl2, ra2, ba2, br2;   // (rc_R+skin)^2, (rc_A+skin)^2, rc_A^2, rc_R^2
  float fs2;                  // (rc_R + FAR_EDGE skin)^2: where the far band starts
  Control *ctrl;
};

// Compile-time model shape: NR radial functions, NA angular channels, KR/KA basis functions, 3-body
// harmonics l = 1..LMAX (NLM = LMAX (LMAX + 2) components), optional 4-body term (built from l = 2),
// NNEU hidden neurons.  GS = elements per adjoint row (NA * NLM, then an 8-element tail).
template <int NR_, int NA_, int KR_, int KA_, int LMAX_, bool FOURBODY_, int NNEU_>
struct Shape {
  static constexpr int NR = NR_, NA = NA_, KR = KR_, KA = KA_, LMAX = LMAX_, NNEU = NNEU_;
  static constexpr bool FOURBODY = FOURBODY_;
  static constexpr int NLM = LMAX * (LMAX + 2);
  static constexpr int NDES = NR + NA * LMAX + (FOURBODY ? NA : 0);
  static constexpr int GS = NA * NLM + 8;
  static_assert(NLM % 8 == 0, "rows are read in 16-byte vectors of up to 8 values: LMAX must be 2 or 4");
  static_assert(NR <= 8, "radial adjoint lives in the 8-element row tail");
  static_assert(!FOURBODY || LMAX >= 2, "the 4-body term is built from the l = 2 sums");
};

// The teacher NEP of the workload (n_max 4/4, basis 8/8, l_max 4, 4-body, 30 neurons) and the
// distilled student (n_max 3/3, basis 8/8, l_max 2, no 4-body, 16 neurons).
using CuShape = Shape<5, 5, 8, 8, 4, true, 30>;
using StudentShape = Shape<4, 4, 8, 8, 2, false, 16>;

// Model parameters, passed by value as a __grid_constant__ kernel argument so that every uniform
// access compiles to a constant-bank operand.
template <class S>
struct Model {
  float cR[S::NR][S::KR];
  float cA[S::NA][S::KA];
  float W0[S::NNEU][S::NDES];
  float b0[S::NNEU];
  float w1[S::NNEU];
  float qs[S::NDES];
  float b1;
  float rcR, rcA, rcR2, rcA2, inv_rcR, inv_rcA;
  float lj_on, lj_c12, lj_c6, lj_rc2, lj_e_rc, lj_de_rc, lj_rc;  // shifted-force LJ
  float lj_e0, lj_m12, lj_p6;   // rc E'(rc) - E(rc), -12 c12, 6 c6 (the factored forms of lj_pair)
  float rmax2;   // max(rcR, lj_rc)^2
};

// Pair records of the fused kernels: the descriptor walk stores every active pair's displacement and
// neighbour index, and the force pass reads them back instead of walking the neighbour list again.
// Each resident block owns one region [pmax][BLOCK] float4 of `rec`, chosen by the SM it runs on and a
// free slot among that SM's `slots` (one bit each in slot_mask[sm]).  The teacher's fused kernels use
// PC_SLOTS: at most that many of their blocks fit on an SM (each holds 512 / PC_SLOTS of the SM's
// tensor-memory columns); the student's register-resident fused kernel uses PC_SLOTS_REG, checked on
// the host against its occupancy.  So a slot is always free for a starting block.  Regions are reused
// block after block, so their lines stay in L2.
constexpr int PC_SLOTS = 4;
constexpr int PC_SLOTS_REG = 8;
struct PairCache {
  float4 *rec;           // [nsm * slots][pmax][BLOCK]
  unsigned *slot_mask;   // [nsm], zero-initialised; bit b: slot b of that SM is held
  int nsm;               // bound on the SM index (%nsmid)
  int pmax;              // records per atom: >= the neighbour-list capacity
  int slots;             // regions per SM index
};

__device__ __forceinline__ unsigned sm_index() {
  unsigned r;
  asm volatile("mov.u32 %0, %%smid;" : "=r"(r));
  return r;
}
__device__ __forceinline__ unsigned sm_index_bound() {
  unsigned r;
  asm volatile("mov.u32 %0, %%nsmid;" : "=r"(r));
  return r;
}

// A free pair-record region of this SM for the calling block (one thread calls it): sm * slots + b, or
// -1 after 64 rounds over the SM's slots (the caller reports that; it cannot happen while no more than
// `slots` blocks of the kernel are resident on an SM).
__device__ __forceinline__ int acquire_record_slot(const PairCache &pc) {
  const unsigned sm = sm_index();
  int slot = -1;
  if ((int)sm < pc.nsm) {
    for (int it = 0; it < 64 && slot < 0; ++it)
      for (int b = 0; b < pc.slots && slot < 0; ++b)
        if ((atomicOr(pc.slot_mask + sm, 1u << b) & (1u << b)) == 0u) slot = (int)sm * pc.slots + b;
  }
  return slot;
}

// Cell geometry of the current neighbour list.
struct Geom {
  float lx, ly, lz;      // cell edge lengths (float)
  int ncx, ncy, ncz;
};

__device__ __forceinline__ int cell_x(float w) { return __float_as_int(w) & 1023; }
__device__ __forceinline__ int cell_y(float w) { return (__float_as_int(w) >> 10) & 1023; }
__device__ __forceinline__ int cell_z(float w) { return (__float_as_int(w) >> 20) & 1023; }

// Offsets of the 27 neighbouring cell images: shift s = (dx+1) + 3(dy+1) + 9(dz+1).
__device__ __forceinline__ void fill_shift_table(float4 *tab, const Geom &g) {
  for (int s = threadIdx.x; s < 27; s += blockDim.x) {
    int dx = s % 3 - 1, dy = (s / 3) % 3 - 1, dz = s / 9 - 1;
    tab[s] = make_float4(dx * g.lx, dy * g.ly, dz * g.lz, 0.f);
  }
}

// Packed float2 arithmetic: two FP32 operations per instruction on the sm_100 family (FFMA2, FADD2,
// FMUL2), each rounded as its scalar counterpart.  The hot loops pair independent operations so that
// they issue half as many FP32 instructions.
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 bc2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 pr(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float hsum(float2 a) { return a.x + a.y; }

// sum_k c[k] f[k] (K even) as K/2 paired multiply-adds (even and odd k accumulated apart) and one add.
template <int K>
__device__ __forceinline__ float dot_pairs(const float (&c)[K], const float (&f)[K]) {
  static_assert(K % 2 == 0, "even length");
  float2 t = mul2(pr(c[0], c[1]), pr(f[0], f[1]));
#pragma unroll
  for (int k = 2; k < K; k += 2) t = fma2(pr(c[k], c[k + 1]), pr(f[k], f[k + 1]), t);
  return hsum(t);
}
// Two dot products with the same coefficients: sum_k c[k] f[k] and sum_k c[k] d[k].
template <int K>
__device__ __forceinline__ void dot_pairs2(const float (&c)[K], const float (&f)[K], const float (&d)[K], float &tf,
                                           float &td) {
  static_assert(K % 2 == 0, "even length");
  const float2 c0 = pr(c[0], c[1]);
  float2 a = mul2(c0, pr(f[0], f[1])), b = mul2(c0, pr(d[0], d[1]));
#pragma unroll
  for (int k = 2; k < K; k += 2) {
    const float2 ck = pr(c[k], c[k + 1]);
    a = fma2(ck, pr(f[k], f[k + 1]), a);
    b = fma2(ck, pr(d[k], d[k + 1]), b);
  }
  tf = hsum(a);
  td = hsum(b);
}

// Chebyshev basis f_k(r) = (T_k(x) + 1)/2 * fc(r), x = 2 (r/rc - 1)^2 - 1, fc = (1 + cos(pi r/rc))/2,
// evaluated as f_k = h T_k + h with h = fc / 2 (T_k by the three-term recurrence, the f_k in pairs).
// The cutoff uses the hardware sine/cosine (absolute error below 2^-21.4 for arguments in [-pi, pi];
// here pi r / rc lies in [0, pi]), a few instructions instead of the range-reduced library call.
template <int K>
__device__ __forceinline__ void cheb_basis(float r, float inv_rc, float (&f)[K]) {
  static_assert(K % 2 == 0 && K >= 2, "even basis size");
  float s, c;
  const float t = r * inv_rc;
  __sincosf(3.14159265358979f * t, &s, &c);
  const float h = fmaf(0.25f, c, 0.25f);         // fc / 2 (= (c + 1) / 4, one rounding)
  const float u = t - 1.f;
  const float x = fmaf(2.f * u, u, -1.f);
  const float x2 = x + x;
  float T[K];
  T[0] = 1.f; T[1] = x;
#pragma unroll
  for (int k = 2; k < K; ++k) T[k] = fmaf(x2, T[k - 1], -T[k - 2]);
  const float2 h2 = bc2(h);
#pragma unroll
  for (int k = 0; k < K; k += 2) {
    const float2 v = fma2(h2, pr(T[k], T[k + 1]), h2);
    f[k] = v.x; f[k + 1] = v.y;
  }
}

// Basis and radial derivative: f_k' = (T_k + 1) h' + T_k'(x) x'(r) h, with h = fc / 2, h' = fc' / 2,
// T_k' by the differentiated recurrence T_k' = 2 T_{k-1} + 2 x T_{k-1}' - T_{k-2}'.
template <int K>
__device__ __forceinline__ void cheb_basis_d(float r, float inv_rc, float (&f)[K], float (&df)[K]) {
  static_assert(K % 2 == 0 && K >= 2, "even basis size");
  float s, c;
  const float t = r * inv_rc;
  __sincosf(3.14159265358979f * t, &s, &c);
  const float h = fmaf(0.25f, c, 0.25f);                           // fc / 2
  const float dh = (-0.25f * 3.14159265358979f * inv_rc) * s;      // fc' / 2
  const float u = t - 1.f;
  const float x = fmaf(2.f * u, u, -1.f);
  const float x2 = x + x;
  const float dxh = (4.f * inv_rc) * u * h;                        // x'(r) h
  float T[K], D[K];
  T[0] = 1.f; T[1] = x;
  D[0] = 0.f; D[1] = 1.f;
#pragma unroll
  for (int k = 2; k < K; ++k) {
    T[k] = fmaf(x2, T[k - 1], -T[k - 2]);
    D[k] = fmaf(x2, D[k - 1], fmaf(2.f, T[k - 1], -D[k - 2]));
  }
  const float2 h2 = bc2(h), dh2 = bc2(dh), dxh2 = bc2(dxh);
#pragma unroll
  for (int k = 0; k < K; k += 2) {
    const float2 tk = pr(T[k], T[k + 1]);
    const float2 v = fma2(h2, tk, h2);
    const float2 d = fma2(pr(D[k], D[k + 1]), dxh2, fma2(tk, dh2, dh2));
    f[k] = v.x; f[k + 1] = v.y;
    df[k] = d.x; df[k + 1] = d.y;
  }
}

// The factors of cheb_basis / cheb_basis_d, for sums that never form f_k or f_k' themselves: h = fc / 2,
// dh = fc' / 2, dxh = x'(r) h, T_k(x) and D_k = T_k'(x) (T_0 = 1, D_0 = 0, D_1 = 1), so that
// f_k = h (T_k + 1) and f_k' = (T_k + 1) dh + D_k dxh.  Summed over pairs, sum f_k = sum h T_k + sum h,
// and a contraction sum_k t_k f_k' = dh (sum_k t_k T_k + sum_k t_k) + dxh sum_k t_k D_k.
template <int K>
__device__ __forceinline__ void cheb_t(float r, float inv_rc, float &h, float (&T)[K]) {
  static_assert(K >= 2, "basis size");
  const float t = r * inv_rc;
  h = fmaf(0.25f, __cosf(3.14159265358979f * t), 0.25f);
  const float u = t - 1.f;
  const float x = fmaf(2.f * u, u, -1.f);
  const float x2 = x + x;
  T[0] = 1.f; T[1] = x;
#pragma unroll
  for (int k = 2; k < K; ++k) T[k] = fmaf(x2, T[k - 1], -T[k - 2]);
}
template <int K>
__device__ __forceinline__ void cheb_td(float r, float inv_rc, float &dh, float &dxh, float (&T)[K], float (&D)[K]) {
  static_assert(K >= 2, "basis size");
  float s, c;
  const float t = r * inv_rc;
  __sincosf(3.14159265358979f * t, &s, &c);
  const float h = fmaf(0.25f, c, 0.25f);
  dh = (-0.25f * 3.14159265358979f * inv_rc) * s;
  const float u = t - 1.f;
  const float x = fmaf(2.f * u, u, -1.f);
  const float x2 = x + x;
  dxh = (4.f * inv_rc) * u * h;
  T[0] = 1.f; T[1] = x;
  D[0] = 0.f; D[1] = 1.f;
#pragma unroll
  for (int k = 2; k < K; ++k) {
    T[k] = fmaf(x2, T[k - 1], -T[k - 2]);
    D[k] = fmaf(x2, D[k - 1], fmaf(2.f, T[k - 1], -D[k - 2]));
  }
}
template <int K>
__device__ __forceinline__ void cheb_td_x2(float2 r, float inv_rc, float2 &dh, float2 &dxh, float2 (&T)[K],
                                           float2 (&D)[K]) {
  static_assert(K >= 2, "basis size");
  float2 s, cs;
  const float2 t = mul2(r, bc2(inv_rc));
  __sincosf(3.14159265358979f * t.x, &s.x, &cs.x);
  __sincosf(3.14159265358979f * t.y, &s.y, &cs.y);
  const float2 h = fma2(bc2(0.25f), cs, bc2(0.25f));
  dh = mul2(bc2(-0.25f * 3.14159265358979f * inv_rc), s);
  const float2 u = add2(t, bc2(-1.f));
  const float2 x = fma2(mul2(bc2(2.f), u), u, bc2(-1.f));
  const float2 x2 = add2(x, x);
  dxh = mul2(mul2(bc2(4.f * inv_rc), u), h);
  T[0] = bc2(1.f); T[1] = x;
  D[0] = bc2(0.f); D[1] = bc2(1.f);
#pragma unroll
  for (int k = 2; k < K; ++k) {
    T[k] = fma2(x2, T[k - 1], make_float2(-T[k - 2].x, -T[k - 2].y));
    D[k] = fma2(x2, D[k - 1], fma2(bc2(2.f), T[k - 1], make_float2(-D[k - 2].x, -D[k - 2].y)));
  }
}

// Normalised real harmonics Yh_lm(u) = sqrt(4 pi / (2l+1)) Y_lm(u), l = 1..4 (24 values, m = -l..l),
// so that sum_m Yh_lm(u) Yh_lm(v) = P_l(u . v).  Written as solid-harmonic polynomials of a unit vector.
// NLM = 8 computes l = 1, 2 only.
template <int NLM>
__host__ __device__ __forceinline__ void harmonics(float x, float y, float z, float (&Y)[NLM]) {
  static_assert(NLM == 8 || NLM == 24, "l_max 2 or 4");
  const float x2 = x * x, y2 = y * y, z2 = z * z;
  const float s3 = 1.7320508075688772f, s5 = 2.2360679774997896f, s6 = 2.449489742783178f;
  const float s10 = 3.1622776601683795f, s15 = 3.872983346207417f, s35 = 5.916079783099616f;
  const float s70 = 8.366600265340756f;
  // l = 1
  Y[0] = y; Y[1] = z; Y[2] = x;
  // l = 2
  Y[3] = s3 * x * y;
  Y[4] = s3 * y * z;
  Y[5] = z2 - 0.5f * (x2 + y2);
  Y[6] = s3 * x * z;
  Y[7] = 0.5f * s3 * (x2 - y2);
  if constexpr (NLM > 8) {
  // l = 3
  const float a3 = 4.f * z2 - x2 - y2;
  Y[8] = 0.25f * s10 * y * (3.f * x2 - y2);
  Y[9] = s15 * x * y * z;
  Y[10] = 0.25f * s6 * y * a3;
  Y[11] = z * (z2 - 1.5f * (x2 + y2));
  Y[12] = 0.25f * s6 * x * a3;
  Y[13] = 0.5f * s15 * z * (x2 - y2);
  Y[14] = 0.25f * s10 * x * (x2 - 3.f * y2);
  // l = 4
  const float rr = x2 + y2 + z2;
  const float b4 = 7.f * z2 - rr, c4 = 7.f * z2 - 3.f * rr;
  Y[15] = 0.5f * s35 * x * y * (x2 - y2);
  Y[16] = 0.25f * s70 * y * z * (3.f * x2 - y2);
  Y[17] = 0.5f * s5 * x * y * b4;
  Y[18] = 0.25f * s10 * y * z * c4;
  Y[19] = 0.125f * (35.f * z2 * z2 - 30.f * z2 * rr + 3.f * rr * rr);
  Y[20] = 0.25f * s10 * x * z * c4;
  Y[21] = 0.25f * s5 * (x2 - y2) * b4;
  Y[22] = 0.25f * s70 * x * z * (x2 - 3.f * y2);
  Y[23] = 0.125f * s35 * (x2 * x2 - 6.f * x2 * y2 + y2 * y2);
  }
}

// Gradient (ax, ay, az) of the solid-harmonic polynomial of component lm at (x, y, z).  lm is a
// compile-time constant after unrolling; harmonic_grad_mask(lm) has bit d set when component d can be
// non-zero, so callers skip the multiply-adds of the identically zero ones.
__host__ __device__ __forceinline__ void harmonic_grad(int lm, float x, float y, float z, float (&a)[3]) {
  const float x2 = x * x, y2 = y * y, z2 = z * z;
  const float s3 = 1.7320508075688772f, s5 = 2.2360679774997896f, s6 = 2.449489742783178f;
  const float s10 = 3.1622776601683795f, s15 = 3.872983346207417f, s35 = 5.916079783099616f;
  const float s70 = 8.366600265340756f;
  float ax = 0.f, ay = 0.f, az = 0.f;
  switch (lm) {
    case 0: ay = 1.f; break;
    case 1: az = 1.f; break;
    case 2: ax = 1.f; break;
    case 3: ax = s3 * y; ay = s3 * x; break;
    case 4: ay = s3 * z; az = s3 * y; break;
    case 5: ax = -x; ay = -y; az = 2.f * z; break;
    case 6: ax = s3 * z; az = s3 * x; break;
    case 7: ax = s3 * x; ay = -s3 * y; break;
    case 8: ax = 1.5f * s10 * x * y; ay = 0.75f * s10 * (x2 - y2); break;
    case 9: ax = s15 * y * z; ay = s15 * x * z; az = s15 * x * y; break;
    case 10: ax = -0.5f * s6 * x * y; ay = -0.25f * s6 * (x2 + 3.f * y2 - 4.f * z2); az = 2.f * s6 * y * z; break;
    case 11: ax = -3.f * x * z; ay = -3.f * y * z; az = -1.5f * (x2 + y2 - 2.f * z2); break;
    case 12: ax = -0.25f * s6 * (3.f * x2 + y2 - 4.f * z2); ay = -0.5f * s6 * x * y; az = 2.f * s6 * x * z; break;
    case 13: ax = s15 * x * z; ay = -s15 * y * z; az = 0.5f * s15 * (x2 - y2); break;
    case 14: ax = 0.75f * s10 * (x2 - y2); ay = -1.5f * s10 * x * y; break;
    case 15: ax = 0.5f * s35 * y * (3.f * x2 - y2); ay = 0.5f * s35 * x * (x2 - 3.f * y2); break;
    case 16: ax = 1.5f * s70 * x * y * z; ay = 0.75f * s70 * z * (x2 - y2); az = 0.25f * s70 * y * (3.f * x2 - y2); break;
    case 17: ax = -0.5f * s5 * y * (3.f * x2 + y2 - 6.f * z2); ay = -0.5f * s5 * x * (x2 + 3.f * y2 - 6.f * z2);
             az = 6.f * s5 * x * y * z; break;
    case 18: ax = -1.5f * s10 * x * y * z; ay = -0.25f * s10 * z * (3.f * x2 + 9.f * y2 - 4.f * z2);
             az = -0.75f * s10 * y * (x2 + y2 - 4.f * z2); break;
    case 19: ax = 1.5f * x * (x2 + y2 - 4.f * z2); ay = 1.5f * y * (x2 + y2 - 4.f * z2);
             az = -2.f * z * (3.f * x2 + 3.f * y2 - 2.f * z2); break;
    case 20: ax = -0.25f * s10 * z * (9.f * x2 + 3.f * y2 - 4.f * z2); ay = -1.5f * s10 * x * y * z;
             az = -0.75f * s10 * x * (x2 + y2 - 4.f * z2); break;
    case 21: ax = -s5 * x * (x2 - 3.f * z2); ay = s5 * y * (y2 - 3.f * z2); az = 3.f * s5 * z * (x2 - y2); break;
    case 22: ax = 0.75f * s70 * z * (x2 - y2); ay = -1.5f * s70 * x * y * z; az = 0.25f * s70 * x * (x2 - 3.f * y2); break;
    case 23: ax = 0.5f * s35 * x * (x2 - 3.f * y2); ay = -0.5f * s35 * y * (3.f * x2 - y2); break;
    default: break;
  }
  a[0] = ax; a[1] = ay; a[2] = az;
}
__host__ __device__ constexpr int harmonic_grad_mask(int lm) {
  return lm == 0 ? 2 : lm == 1 ? 4 : lm == 2 ? 1 : lm == 3 ? 3 : lm == 4 ? 6 : lm == 6 ? 5 :
         (lm == 7 || lm == 8 || lm == 14 || lm == 15 || lm == 23) ? 3 : 7;
}

// The same harmonics without their constant factors: Yh_lm = hnorm(lm) Ph_lm, with Ph_lm (harmonics_p)
// a polynomial with small integer coefficients.  A sum or an adjoint row kept over Ph instead of Yh
// (s'_nlm = s_nlm / hnorm(lm), G'_nlm = hnorm(lm) G_nlm) gives the same products G s and G dYh/du with
// the per-pair constant multiplies moved to one multiply per atom and component.
__host__ __device__ constexpr float hnorm(int lm) {
  constexpr float s3 = 1.7320508075688772f, s5 = 2.2360679774997896f, s6 = 2.449489742783178f;
  constexpr float s10 = 3.1622776601683795f, s15 = 3.872983346207417f, s35 = 5.916079783099616f;
  constexpr float s70 = 8.366600265340756f;
  return lm < 3 ? 1.f : lm == 3 || lm == 4 || lm == 6 ? s3 : lm == 5 ? 1.f : lm == 7 ? 0.5f * s3 :
         lm == 8 || lm == 14 ? 0.25f * s10 : lm == 9 ? s15 : lm == 10 || lm == 12 ? 0.25f * s6 :
         lm == 11 ? 1.f : lm == 13 ? 0.5f * s15 : lm == 15 ? 0.5f * s35 : lm == 16 || lm == 22 ? 0.25f * s70 :
         lm == 17 ? 0.5f * s5 : lm == 18 || lm == 20 ? 0.25f * s10 : lm == 19 ? 0.125f :
         lm == 21 ? 0.25f * s5 : 0.125f * s35;
}

template <int NLM>
__host__ __device__ __forceinline__ void harmonics_p(float x, float y, float z, float (&P)[NLM]) {
  static_assert(NLM == 8 || NLM == 24, "l_max 2 or 4");
  const float x2 = x * x, y2 = y * y, z2 = z * z;
  const float xy = x * y, yz = y * z, xz = x * z, d = x2 - y2, e = x2 + y2;
  P[0] = y; P[1] = z; P[2] = x;
  P[3] = xy;
  P[4] = yz;
  P[5] = fmaf(-0.5f, e, z2);
  P[6] = xz;
  P[7] = d;
  if constexpr (NLM > 8) {
  const float a3 = fmaf(4.f, z2, -e);          // 4 z^2 - x^2 - y^2
  const float p8 = y * fmaf(3.f, x2, -y2);     // y (3 x^2 - y^2)
  const float p14 = x * fmaf(-3.f, y2, x2);    // x (x^2 - 3 y^2)
  P[8] = p8;
  P[9] = xy * z;
  P[10] = y * a3;
  P[11] = z * fmaf(-1.5f, e, z2);
  P[12] = x * a3;
  P[13] = z * d;
  P[14] = p14;
  const float b4 = fmaf(6.f, z2, -e);          // 7 z^2 - r^2
  const float c4 = fmaf(-3.f, e, 4.f * z2);    // 7 z^2 - 3 r^2
  const float rr = e + z2;
  P[15] = xy * d;
  P[16] = z * p8;
  P[17] = xy * b4;
  P[18] = yz * c4;
  P[19] = fmaf(35.f * z2, z2, fmaf(-30.f * z2, rr, 3.f * rr * rr));
  P[20] = xz * c4;
  P[21] = d * b4;
  P[22] = z * p14;
  P[23] = fmaf(x2, x2, fmaf(-6.f * x2, y2, y2 * y2));
  }
}

// Ph_lm alone (lm a compile-time constant after unrolling), for loops that form the components chunk by
// chunk instead of holding all 24.
__host__ __device__ __forceinline__ float harmonic_p(int lm, float x, float y, float z) {
  const float x2 = x * x, y2 = y * y, z2 = z * z;
  const float xy = x * y, d = x2 - y2, e = x2 + y2;
  switch (lm) {
    case 0: return y;
    case 1: return z;
    case 2: return x;
    case 3: return xy;
    case 4: return y * z;
    case 5: return fmaf(-0.5f, e, z2);
    case 6: return x * z;
    case 7: return d;
    case 8: return y * fmaf(3.f, x2, -y2);
    case 9: return xy * z;
    case 10: return y * fmaf(4.f, z2, -e);
    case 11: return z * fmaf(-1.5f, e, z2);
    case 12: return x * fmaf(4.f, z2, -e);
    case 13: return z * d;
    case 14: return x * fmaf(-3.f, y2, x2);
    case 15: return xy * d;
    case 16: return z * (y * fmaf(3.f, x2, -y2));
    case 17: return xy * fmaf(6.f, z2, -e);
    case 18: return (y * z) * fmaf(-3.f, e, 4.f * z2);
    case 19: { const float rr = e + z2; return fmaf(35.f * z2, z2, fmaf(-30.f * z2, rr, 3.f * rr * rr)); }
    case 20: return (x * z) * fmaf(-3.f, e, 4.f * z2);
    case 21: return d * fmaf(6.f, z2, -e);
    case 22: return z * (x * fmaf(-3.f, y2, x2));
    case 23: return fmaf(x2, x2, fmaf(-6.f * x2, y2, y2 * y2));
    default: return 0.f;
  }
}

// Gradient of Ph_lm at (x, y, z) (harmonic_grad / hnorm(lm)); the same zero pattern (harmonic_grad_mask).
__host__ __device__ __forceinline__ void harmonic_grad_p(int lm, float x, float y, float z, float (&a)[3]) {
  const float x2 = x * x, y2 = y * y, z2 = z * z;
  const float xy = x * y, yz = y * z, xz = x * z, d = x2 - y2, e = x2 + y2;
  float ax = 0.f, ay = 0.f, az = 0.f;
  switch (lm) {
    case 0: ay = 1.f; break;
    case 1: az = 1.f; break;
    case 2: ax = 1.f; break;
    case 3: ax = y; ay = x; break;
    case 4: ay = z; az = y; break;
    case 5: ax = -x; ay = -y; az = 2.f * z; break;
    case 6: ax = z; az = x; break;
    case 7: ax = 2.f * x; ay = -2.f * y; break;
    case 8: ax = 6.f * xy; ay = 3.f * d; break;
    case 9: ax = yz; ay = xz; az = xy; break;
    case 10: ax = -2.f * xy; ay = fmaf(4.f, z2, -fmaf(3.f, y2, x2)); az = 8.f * yz; break;
    case 11: ax = -3.f * xz; ay = -3.f * yz; az = fmaf(-1.5f, e, 3.f * z2); break;
    case 12: ax = fmaf(4.f, z2, -fmaf(3.f, x2, y2)); ay = -2.f * xy; az = 8.f * xz; break;
    case 13: ax = 2.f * xz; ay = -2.f * yz; az = d; break;
    case 14: ax = 3.f * d; ay = -6.f * xy; break;
    case 15: ax = y * fmaf(3.f, x2, -y2); ay = x * fmaf(-3.f, y2, x2); break;
    case 16: ax = 6.f * xy * z; ay = 3.f * z * d; az = y * fmaf(3.f, x2, -y2); break;
    case 17: ax = y * fmaf(6.f, z2, -fmaf(3.f, x2, y2)); ay = x * fmaf(6.f, z2, -fmaf(3.f, y2, x2));
             az = 12.f * xy * z; break;
    case 18: ax = -6.f * xy * z; ay = z * fmaf(4.f, z2, -fmaf(9.f, y2, 3.f * x2));
             az = 3.f * y * fmaf(4.f, z2, -e); break;
    case 19: { const float w = fmaf(-4.f, z2, e);   // x^2 + y^2 - 4 z^2
               ax = 12.f * x * w; ay = 12.f * y * w; az = -16.f * z * fmaf(3.f, e, -2.f * z2); break; }
    case 20: ax = z * fmaf(4.f, z2, -fmaf(9.f, x2, 3.f * y2)); ay = -6.f * xy * z;
             az = 3.f * x * fmaf(4.f, z2, -e); break;
    case 21: ax = -4.f * x * fmaf(-3.f, z2, x2); ay = 4.f * y * fmaf(-3.f, z2, y2); az = 12.f * z * d; break;
    case 22: ax = 3.f * z * d; ay = -6.f * xy * z; az = x * fmaf(-3.f, y2, x2); break;
    case 23: ax = 4.f * x * fmaf(-3.f, y2, x2); ay = -4.f * y * fmaf(3.f, x2, -y2); break;
    default: break;
  }
  a[0] = ax; a[1] = ay; a[2] = az;
}

// Gradient of the solid-harmonic polynomial of component lm, evaluated at (x, y, z), accumulated
// with weight b into (gx, gy, gz).
__device__ __forceinline__ void harmonic_grad_acc(int lm, float x, float y, float z, float b, float &gx,
                                                  float &gy, float &gz) {
  float a[3];
  harmonic_grad(lm, x, y, z, a);
  const int m = harmonic_grad_mask(lm);
  if (m & 1) gx = fmaf(b, a[0], gx);
  if (m & 2) gy = fmaf(b, a[1], gy);
  if (m & 4) gz = fmaf(b, a[2], gz);
}

// The same for the two components lm0, lm0 + 1 with weights b = (b_lm0, b_lm0+1), accumulated into the
// component pairs g[d] (even and odd lm apart): paired multiply-adds where both are non-zero.
// UN: the gradients of the polynomials Ph (harmonic_grad_p), for weights taken over Ph.
template <bool UN = false>
__device__ __forceinline__ void harmonic_grad_acc2(int lm0, float x, float y, float z, float2 b, float2 (&g)[3]) {
  float a0[3], a1[3];
  if constexpr (UN) {
    harmonic_grad_p(lm0, x, y, z, a0);
    harmonic_grad_p(lm0 + 1, x, y, z, a1);
  } else {
    harmonic_grad(lm0, x, y, z, a0);
    harmonic_grad(lm0 + 1, x, y, z, a1);
  }
  const int m0 = harmonic_grad_mask(lm0), m1 = harmonic_grad_mask(lm0 + 1);
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const bool n0 = (m0 >> d) & 1, n1 = (m1 >> d) & 1;
    if (n0 && n1) g[d] = fma2(b, pr(a0[d], a1[d]), g[d]);
    else if (n0) g[d].x = fmaf(b.x, a0[d], g[d].x);
    else if (n1) g[d].y = fmaf(b.y, a1[d], g[d].y);
  }
}

__host__ __device__ constexpr int lm_l(int lm) { return lm < 3 ? 1 : (lm < 8 ? 2 : (lm < 15 ? 3 : 4)); }

// Shifted-force LJ pair energy E(r) and dE/dr, from r^2, r and ir = 1/r (reciprocal square root).
// No division: 1/r^2 = ir^2 refined by one Newton step (error about 1 ulp, which the twelfth power
// would otherwise amplify from the reciprocal square root's 2 ulp), 1/r = ir.
template <class S>
__device__ __forceinline__ void lj_pair(const Model<S> &P, float r2, float r, float ir, float &e, float &de) {
  float ir2 = ir * ir;
  ir2 = fmaf(ir2, fmaf(-r2, ir2, 1.f), ir2);
  const float ir6 = ir2 * ir2 * ir2;
  // E = c12 r^-12 - c6 r^-6 - E(rc) - (r - rc) E'(rc) = r^-6 (c12 r^-6 - c6) + (rc E'(rc) - E(rc)) - r E'(rc)
  e = fmaf(ir6, fmaf(P.lj_c12, ir6, -P.lj_c6), fmaf(-P.lj_de_rc, r, P.lj_e0));
  // dE/dr = r^-6 (-12 c12 r^-6 + 6 c6) / r - E'(rc)
  de = fmaf(ir6 * fmaf(P.lj_m12, ir6, P.lj_p6), ir, -P.lj_de_rc);
}

// lj_pair's derivative dE/dr for two pairs at once.
template <class S>
__device__ __forceinline__ float2 lj_deriv_x2(const Model<S> &P, float2 r2, float2 ir) {
  float2 ir2 = mul2(ir, ir);
  ir2 = fma2(ir2, fma2(make_float2(-r2.x, -r2.y), ir2, bc2(1.f)), ir2);
  const float2 ir6 = mul2(mul2(ir2, ir2), ir2);
  return fma2(mul2(ir6, fma2(bc2(P.lj_m12), ir6, bc2(P.lj_p6))), ir, bc2(-P.lj_de_rc));
}

// Exact conversion of a float to 64-bit fixed point with 32 fractional bits, without a 64-bit
// conversion instruction (those run on the narrow FP64 pipe).
// |v| < 2^12 (every force, energy and virial term of a physical configuration): v * 2^32 is split as
// h * 2^22 + l with h = rint(v * 2^10) and |l| <= 2^21.  Both parts are exact in float32 (l is the
// rounding remainder of v * 2^10, scaled by a power of two), and each is turned into an integer by
// adding 1.5 * 2^23, which places the rounded integer in the low mantissa bits: full-rate FP32 and
// integer instructions only, rounding to nearest (ties to even).
// Larger magnitudes, infinities and NaN take an integer bit-manipulation path (round half away from
// zero; valid for |v| < 2^30).  Either way the result is a fixed function of v, so fixed-point sums
// do not depend on the order of their terms.
__device__ __forceinline__ long long to_fix32(float v) {
  constexpr float SHIFT = 12582912.0f;          // 1.5 * 2^23
  if (fabsf(v) < 4096.f) {
    const float hm = fmaf(v, 1024.f, SHIFT);     // SHIFT + rint(v * 2^10)
    const float h = hm - SHIFT;
    const float l = fmaf(v, 4294967296.f, -h * 4194304.f);
    const int hi = __float_as_int(hm) - 0x4B400000;
    const int lo = __float_as_int(l + SHIFT) - 0x4B400000;
    return ((long long)hi << 22) + lo;
  }
  const uint32_t b = __float_as_uint(v);
  const int ex = (int)((b >> 23) & 0xffu);
  const long long man = (long long)((b & 0x7fffffu) | 0x800000u);
  const int sh = ex - 118;                      // v * 2^32 = man * 2^(ex - 127 - 23 + 32)
  long long r;
  if (sh >= 0) r = man << min(sh, 39);
  else r = (man + (1ll << (-sh - 1))) >> (-sh);
  return (b >> 31) ? -r : r;
}

// to_fix32 of three values with one range test and the float parts of x and y in float2 pairs (the
// same results as three to_fix32 calls).
__device__ __forceinline__ void to_fix32x3(float x, float y, float z, long long &a, long long &b, long long &cz) {
  constexpr float SHIFT = 12582912.0f;
  const float m = fmaxf(fmaxf(fabsf(x), fabsf(y)), fabsf(z));
  if (m < 4096.f) {
    const float2 xy = make_float2(x, y);
    const float2 hm = __ffma2_rn(xy, make_float2(1024.f, 1024.f), make_float2(SHIFT, SHIFT));
    const float hmz = fmaf(z, 1024.f, SHIFT);
    const float2 h = __fadd2_rn(hm, make_float2(-SHIFT, -SHIFT));
    const float hz = hmz - SHIFT;
    const float2 l = __ffma2_rn(xy, make_float2(4294967296.f, 4294967296.f), __fmul2_rn(h, make_float2(-4194304.f, -4194304.f)));
    const float lz = fmaf(z, 4294967296.f, hz * -4194304.f);
    const float2 lm = __fadd2_rn(l, make_float2(SHIFT, SHIFT));
    const float lmz = lz + SHIFT;
    a = ((long long)(__float_as_int(hm.x) - 0x4B400000) << 22) + (__float_as_int(lm.x) - 0x4B400000);
    b = ((long long)(__float_as_int(hm.y) - 0x4B400000) << 22) + (__float_as_int(lm.y) - 0x4B400000);
    cz = ((long long)(__float_as_int(hmz) - 0x4B400000) << 22) + (__float_as_int(lmz) - 0x4B400000);
  } else {
    a = to_fix32(x); b = to_fix32(y); cz = to_fix32(z);
  }
}

// Block-wide sum of NV int64 values into out[blockIdx.x * NV + v].  Integer addition is associative,
// so the result does not depend on the reduction order.  NW bounds the warps per block (the size of
// the shared scratch).
template <int NV, int NW = 32>
__device__ __forceinline__ void block_sum_store(long long (&v)[NV], long long *out) {
  static_assert(NW >= 1 && NW <= 32, "1..32 warps");
  __shared__ long long red[NW][NV];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < NV; ++k) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
  }
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) red[warp][k] = v[k];
  }
  __syncthreads();
  if (warp == 0) {
    const int nw = blockDim.x >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      long long t = lane < nw && lane < NW ? red[lane][k] : 0ll;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
      if (lane == 0) out[(size_t)blockIdx.x * NV + k] = t;
    }
  }
}

// block_sum_store in two halves, so that no block barrier is needed where the values become known:
// warp_sum_stage adds the warp's NV int64 values (lane 0 writes them to dst[0..NV-1]); after a later
// block barrier, block_store_staged adds the staged sums of the block's warps into
// out[blockIdx.x * NV + v].  Integer sums: the result does not depend on the order.
template <int NV>
__device__ __forceinline__ void warp_sum_stage(long long (&v)[NV], long long *dst) {
#pragma unroll
  for (int k = 0; k < NV; ++k) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
  }
  if ((threadIdx.x & 31) == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) dst[k] = v[k];
  }
}
template <int NV, int NW>
__device__ __forceinline__ void block_store_staged(const long long (*src)[NV], long long *out) {
  if (threadIdx.x < NV) {
    long long t = 0;
    const int nw = min(NW, (int)(blockDim.x >> 5));
    for (int w = 0; w < nw; ++w) t += src[w][threadIdx.x];
    out[(size_t)blockIdx.x * NV + threadIdx.x] = t;
  }
}


// ---------------------------------------------------------------------------------------------------
// Asynchronous per-thread neighbour pipeline (cp.async into shared memory).  The walk over an atom's
// list is a chain of dependent loads (list entry -> neighbour position); the pipeline keeps list
// entries DE ahead and neighbour positions DP ahead in shared-memory rings, so the loads of later
// entries are in flight while the current one is computed, without holding registers.
// Layout: ring_e[DE][BLOCK] uint32 and ring_p[DP][BLOCK] float4 (bank-conflict-free per thread).
__device__ __forceinline__ void cp_async4(void *smem, const void *gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gmem) : "memory");
}
// 16 bytes, cached in L2 only (records that are read once)
__device__ __forceinline__ void cp_async16_cg(void *smem, const void *gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// The entries of a row that a walk visits: c entries, the first c1 at list slots 0..c1-1, the rest
// after a gap of `gap` slots (the owned part's far band, skipped together with the other part's).
struct RowSpan {
  int c, c1, gap;
};
// Whole row [owned | not owned], each part ending with its far band (counts packed in nfar: owned in
// the low 16 bits).  skip: leave both far bands out.
__device__ __forceinline__ RowSpan full_row(int nnum, int nown, int nfar, bool skip) {
  if (!skip) return RowSpan{nnum, nnum, 0};
  const int of = nfar & 0xffff, nf = nfar >> 16;
  return RowSpan{nnum - of - nf, nown - of, of};
}
// The owned part only (each unordered pair once).
__device__ __forceinline__ RowSpan owned_row(int nown, int nfar, bool skip) {
  const int c = skip ? nown - (nfar & 0xffff) : nown;
  return RowSpan{c, c, 0};
}

// The per-atom extents of the neighbour list that the row walks read, and the control block whose
// skip_far says whether this evaluation leaves the far bands out (nullptr: never).
struct RowExt {
  const int32_t *nnum, *nown, *nband0, *nfar;
  const Control *ctrl;
};
__device__ __forceinline__ bool skip_far(const RowExt &X) { return X.ctrl != nullptr && X.ctrl->skip_far != 0; }
__device__ __forceinline__ RowSpan full_row(const RowExt &X, int i, bool skip) {
  return skip ? full_row(X.nnum[i], X.nown[i], X.nfar[i], true) : RowSpan{X.nnum[i], X.nnum[i], 0};
}
__device__ __forceinline__ RowSpan owned_row(const RowExt &X, int i, bool skip) {
  return skip ? owned_row(X.nown[i], X.nfar[i], true) : RowSpan{X.nown[i], X.nown[i], 0};
}

template <int DE, int DP, int BLOCK>
struct NbrPipe {
  static_assert(DE >= 2 * DP && DP >= 1, "entries must run at least twice as far ahead as positions");
  uint32_t *re;            // this thread's column of ring_e
  float4 *rp;              // this thread's column of ring_p
  const int32_t *row;      // &nbr[0 * n + i]
  size_t n;
  const float4 *pos;
  int cnt, c1, gap;        // the walked entries (RowSpan)

  // list slot of the k-th walked entry
  __device__ __forceinline__ size_t slot(int k) const { return (size_t)(k < c1 ? k : k + gap); }

  __device__ __forceinline__ void start(uint32_t *ring_e, float4 *ring_p, const int32_t *row_, size_t n_,
                                        const float4 *pos_, RowSpan sp) {
    re = ring_e + threadIdx.x; rp = ring_p + threadIdx.x; row = row_; n = n_; pos = pos_;
    cnt = sp.c; c1 = sp.c1; gap = sp.gap;
#pragma unroll
    for (int k = 0; k < DE; ++k)
      if (k < cnt) cp_async4(re + k * BLOCK, row + slot(k) * n);
    cp_async_commit();
    cp_async_wait<0>();
#pragma unroll
    for (int k = 0; k < DP; ++k) {
      if (k < cnt) cp_async16(rp + k * BLOCK, pos + (re[k * BLOCK] & J_MASK));
      cp_async_commit();
    }
  }
  __device__ __forceinline__ void start(uint32_t *ring_e, float4 *ring_p, const int32_t *row_, size_t n_,
                                        const float4 *pos_, int cnt_) {
    start(ring_e, ring_p, row_, n_, pos_, RowSpan{cnt_, cnt_, 0});
  }

  // Entry k (0 <= k < cnt, called for k = 0, 1, 2, ... in order): its packed list entry and the
  // neighbour's position; issues the copies for entries k + DE and k + DP.
  __device__ __forceinline__ void get(int k, uint32_t &e, float4 &p) {
    cp_async_wait<DP - 1>();
    e = re[(k % DE) * BLOCK];
    p = rp[(k % DP) * BLOCK];
    if (k + DE < cnt) cp_async4(re + ((k + DE) % DE) * BLOCK, row + slot(k + DE) * n);
    if (k + DP < cnt) cp_async16(rp + ((k + DP) % DP) * BLOCK, pos + (re[((k + DP) % DE) * BLOCK] & J_MASK));
    cp_async_commit();
  }

  // Entry k + DP (already in shared memory once get(k) returned), for look-ahead prefetches.
  __device__ __forceinline__ uint32_t ahead(int k) const { return re[((k + DP) % DE) * BLOCK]; }

  __device__ __forceinline__ void finish() { cp_async_wait<0>(); }
};

// 64-bit integer add to global memory whose result nobody reads (the fixed-point force scatter): a
// reduction, which returns nothing, so no register waits for the memory system (atomicAdd on a
// generic pointer becomes a value-returning atomic).  Integer addition is associative, so the sums do
// not depend on the order in which the additions arrive.
__device__ __forceinline__ void red_add(unsigned long long *p, long long v) {
  asm volatile("red.global.add.u64 [%0], %1;" ::"l"(__cvta_generic_to_global(p)), "l"(v));
}

// cp.async ring of pair records (16 bytes each, L2 only): record k of this thread is src[k * stride];
// DQ records in flight, as NbrPipe's positions.
template <int DQ, int BLOCK, int STRIDE>
struct RecPipe {
  float4 *rg;
  const float4 *base;   // the record array (a kernel parameter)
  unsigned off;         // element offset of record 0 of this thread
  int cnt;
  __device__ __forceinline__ void start(float4 *ring, const float4 *base_, unsigned off_, int cnt_) {
    rg = ring + threadIdx.x; base = base_; off = off_; cnt = cnt_;
#pragma unroll
    for (int k = 0; k < DQ; ++k) {
      if (k < cnt) cp_async16_cg(rg + k * BLOCK, base + (off + k * STRIDE));
      cp_async_commit();
    }
  }
  __device__ __forceinline__ float4 get(int k) {
    cp_async_wait<DQ - 1>();
    const float4 v = rg[(k % DQ) * BLOCK];
    if (k + DQ < cnt) cp_async16_cg(rg + ((k + DQ) % DQ) * BLOCK, base + (off + (k + DQ) * STRIDE));
    cp_async_commit();
    return v;
  }
  __device__ __forceinline__ void finish() { cp_async_wait<0>(); }
};

}  // namespace nep
