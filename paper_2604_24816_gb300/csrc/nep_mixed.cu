// nep_mixed.cu -- mixed-precision descriptor + network kernel (sm_103a, tcgen05 tensor cores).
//
// Same descriptors as k_descriptor (float32 neighbour walk, Section III.B), but the one-hidden-layer
// network runs as two GEMMs on the 5th-generation tensor cores, one CTA = one 128-atom tile:
//   forward   Z[128 x 32]  = Q~[128 x 32] . W0^T      (bf16 or f16 operands, f32 accumulation in TMEM)
//   backward  dQ[128 x 32] = T[128 x 32] . W0          T_mu = w1_mu (1 - tanh(z_mu - b0_mu)^2)
// (the batched network GEMM of Section V.B, Optimization 1 and Fig. 2c, with the half-precision network
// input of Optimization 4).  Thread t of the CTA owns atom row t: it writes its row of the A tile into
// shared memory and reads its row of the result from TMEM lane t.  The activation, the site energy and
// the descriptor adjoint are float32; the adjoint rows G are stored as float16 (the paper's half-precision
// storage of the per-atom gradient and angular accumulators), read by k_force<S, __half>.
#include "nep_descriptor.cuh"
#include "nep_gb300.h"
#include "nep_tc.cuh"

namespace nep {

constexpr int MIX_BLOCK = 128;       // = the M extent of one tcgen05.mma tile
constexpr int MIX_DE = 8, MIX_DP = 4;
constexpr int MIX_K = 32;            // descriptors padded to 32 (two K = 16 steps)
constexpr int MIX_N = 32;            // neurons padded to 32
constexpr long MIX_WAIT = 1L << 22;  // mbarrier polls before giving up

// Eight floats rounded to float16, packed for one 16-byte store.
__device__ __forceinline__ uint4 pack8_half(const float *v) {
  uint4 w;
  __half2 h;
  h = __floats2half2_rn(v[0], v[1]); w.x = *reinterpret_cast<uint32_t *>(&h);
  h = __floats2half2_rn(v[2], v[3]); w.y = *reinterpret_cast<uint32_t *>(&h);
  h = __floats2half2_rn(v[4], v[5]); w.z = *reinterpret_cast<uint32_t *>(&h);
  h = __floats2half2_rn(v[6], v[7]); w.w = *reinterpret_cast<uint32_t *>(&h);
  return w;
}

// Teacher shape: the angular sums of 4 of the 5 channels are accumulated in TMEM (96 columns,
// accumulate_atom_tm), the fifth channel's 24 in registers, and the two network GEMMs take turns in the
// remaining 32 columns (the forward result is read out before the backward GEMM overwrites it): 128
// columns per block and 4 resident blocks (124 registers) instead of 245 registers and 2.  The student shape keeps its
// sums in registers and asks for 6 resident blocks (measured best).
#ifndef NEP_MIX_MINB_TM
#define NEP_MIX_MINB_TM 4
#endif
template <class S, class MT>
__global__ void __launch_bounds__(MIX_BLOCK, S::NLM > 8 ? NEP_MIX_MINB_TM : 6)
k_descriptor_mixed(const __grid_constant__ Model<S> P, const Geom geom, const int n, const float4 *__restrict__ pos,
                   const int32_t *__restrict__ nbr, const RowExt X, __half *__restrict__ G,
                   float *__restrict__ usite, float *__restrict__ qout, long long *__restrict__ Ffix,
                   long long *__restrict__ part, int *__restrict__ status, const __grid_constant__ Fallback fb) {
  static_assert(S::NDES <= MIX_K && S::NNEU <= MIX_N, "network larger than one tensor-core tile");
  constexpr bool TM = S::NLM > 8;
  constexpr int NT = 4;                                   // TM: channels whose sums live in TMEM
  constexpr uint32_t TCOLS = TM ? 128 : 64;
  constexpr uint32_t ZCOL = TM ? NT * S::NLM : 0;         // forward GEMM result
  constexpr uint32_t DCOL = TM ? NT * S::NLM : 32;        // backward GEMM result (TM: the same columns)
  static_assert(!TM || (NT * S::NLM + MIX_N <= (int)TCOLS && MIX_BLOCK == 128), "TMEM budget");
  __shared__ float4 shift[27];
  // The neighbour-pipeline ring is dead once every thread has walked its row, so the GEMMs' A tile
  // (q~ rows, then T rows) overlays it: less shared memory per block leaves more of the unified
  // L1/shared storage to L1, which caches the gathered neighbour positions.
  constexpr int RING_BYTES = MIX_DP * MIX_BLOCK * 16 + MIX_DE * MIX_BLOCK * 4;
  constexpr int A_BYTES = MIX_BLOCK * MIX_K * (int)sizeof(MT);
  __shared__ __align__(1024) unsigned char smem_ring[RING_BYTES > A_BYTES ? RING_BYTES : A_BYTES];
  float4 *ring_p = reinterpret_cast<float4 *>(smem_ring);
  uint32_t *ring_e = reinterpret_cast<uint32_t *>(smem_ring + MIX_DP * MIX_BLOCK * 16);
  MT *sA = reinterpret_cast<MT *>(smem_ring);
  __shared__ __align__(1024) MT sW[MIX_N * MIX_K];         // B of the forward GEMM: W0[neuron][descriptor]
  __shared__ __align__(1024) MT sWt[MIX_K * MIX_N];        // B of the backward GEMM: W0[descriptor][neuron]
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_base;
  const int t = threadIdx.x;
  fill_shift_table(shift, geom);
  if (t < 32) {
    for (int k = 0; k < MIX_K; ++k) {
      sW[tile_off(t, k, MIX_K / 8)] = to_mma_type<MT>((t < S::NNEU && k < S::NDES) ? P.W0[t][k] : 0.f);
      sWt[tile_off(t, k, MIX_K / 8)] = to_mma_type<MT>((t < S::NDES && k < S::NNEU) ? P.W0[k][t] : 0.f);
    }
    tmem_alloc(&tmem_base, TCOLS);
    tc_fence_before();
  }
  if (t == 0) mbar_init(&mbar, 1);
  __syncthreads();

  const int i = blockIdx.x * MIX_BLOCK + t;
  const bool live = i < n;
  AtomSums<S> A;
  FourBody<S> T;
  float q[S::NDES];
  long long acc[5] = {0, 0, 0, 0, 0};
  bool flagged = false;
  RegSums<S, NT> R;
  uint32_t trow = 0;
  if constexpr (TM) {
    tc_fence_after();
    trow = tmem_base + ((uint32_t)(t & ~31) << 16);
    const RowSpan sp = live ? full_row(X, i, skip_far(X)) : RowSpan{0, 0, 0};
    A.cnt = sp.c;
    if (live) { Ffix[i] = 0; Ffix[(size_t)n + i] = 0; Ffix[2 * (size_t)n + i] = 0; }
    accumulate_atom_tm<S, NT, MIX_DE, MIX_DP, MIX_BLOCK>(P, shift, trow, live ? i : 0, n, pos, nbr, sp, ring_e,
                                                         ring_p, A.QR, R, A.elj, A.nrad, A.nang, A.nact);
    descriptors_tm<S, NT>(P, trow, A.QR, R, q, T);        // zero for threads past the last atom (empty row)
    if (live) {
      if (qout != nullptr) {
#pragma unroll
        for (int v = 0; v < S::NDES; ++v) qout[(size_t)i * S::NDES + v] = q[v];
      }
      flagged = fb.on && out_of_range<S>(fb, P, q);
      if (flagged) flag_atom(fb, i, status);
    }
  } else if (live) {
    Ffix[i] = 0; Ffix[(size_t)n + i] = 0; Ffix[2 * (size_t)n + i] = 0;
    accumulate_atom<S, MIX_DE, MIX_DP, MIX_BLOCK>(P, shift, i, n, pos, nbr, full_row(X, i, skip_far(X)), ring_e,
                                                  ring_p, A);
    descriptors_of<S>(P, A, q, T);
    if (qout != nullptr) {
#pragma unroll
      for (int v = 0; v < S::NDES; ++v) qout[(size_t)i * S::NDES + v] = q[v];
    }
    flagged = fb.on && out_of_range<S>(fb, P, q);
    if (flagged) flag_atom(fb, i, status);
  } else {
#pragma unroll
    for (int v = 0; v < S::NDES; ++v) q[v] = 0.f;
  }
  __syncthreads();     // every thread's row walk (and its ring copies) is done before the A tile overlays the ring
#pragma unroll
  for (int k = 0; k < MIX_K; ++k) sA[tile_off(t, k, MIX_K / 8)] = to_mma_type<MT>(k < S::NDES ? q[k] * P.qs[k] : 0.f);
  fence_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base;
  const uint32_t idesc = umma_idesc_f16(MIX_BLOCK, MIX_N, MmaKind<MT>::bf16);
  const uint32_t lbo = 128, sbo = (MIX_K / 8) * 128;
  if (t == 0) {
#pragma unroll
    for (int ks = 0; ks < MIX_K / 16; ++ks)
      umma_f16(tmem + ZCOL, umma_smem_desc(smem_addr(sA) + ks * 256, lbo, sbo),
               umma_smem_desc(smem_addr(sW) + ks * 256, lbo, sbo), idesc, ks);
    umma_commit(&mbar);
  }
  bool ok = mbar_wait(&mbar, 0, MIX_WAIT);
  tc_fence_after();
  const uint32_t lane_base = (uint32_t)(t & ~31) << 16;
  float z[32];
  tmem_ld32(tmem + lane_base + ZCOL, z);

  // activation, site energy and the backward GEMM operand, in float32
  float U = -P.b1;
  float tr[MIX_N];
#pragma unroll
  for (int mu = 0; mu < MIX_N; ++mu) {
    if (mu < S::NNEU) {
      const float h = tanhf(z[mu] - P.b0[mu]);
      U = fmaf(P.w1[mu], h, U);
      tr[mu] = P.w1[mu] * (1.f - h * h);
    } else {
      tr[mu] = 0.f;
    }
  }
  // the forward MMA has completed (mbarrier), so its A tile can be overwritten
#pragma unroll
  for (int k = 0; k < MIX_N; ++k) sA[tile_off(t, k, MIX_N / 8)] = to_mma_type<MT>(tr[k]);
  fence_async_smem();
  tc_fence_before();   // every thread has read the forward result before the backward GEMM may overwrite it
  __syncthreads();
  tc_fence_after();
  if (t == 0) {
#pragma unroll
    for (int ks = 0; ks < MIX_N / 16; ++ks)
      umma_f16(tmem + DCOL, umma_smem_desc(smem_addr(sA) + ks * 256, lbo, sbo),
               umma_smem_desc(smem_addr(sWt) + ks * 256, lbo, sbo), idesc, ks);
    umma_commit(&mbar);
  }
  ok = mbar_wait(&mbar, 1, MIX_WAIT) && ok;
  tc_fence_after();
  float dq[32];
  tmem_ld32(tmem + lane_base + DCOL, dq);
  if (!ok && t == 0) atomicOr(status, ST_TIMEOUT);

  float Fp[S::NDES];
#pragma unroll
  for (int v = 0; v < S::NDES; ++v) Fp[v] = flagged ? 0.f : dq[v] * P.qs[v];   // flagged: no U_i here
  __half *Gi = G + (size_t)(live ? i : 0) * S::GS;
  if constexpr (TM) {
    // adjoint from the sums (TMEM chunks read by whole warps; rows stored for live atoms only)
    float g4[S::NA][5];
#pragma unroll
    for (int a = 0; a < S::NA; ++a) fourbody_adjoint<S>(a, T, g4[a]);
#pragma unroll
    for (int k = 0; k < S::NLM / TMEM_W; ++k) {
      const int c = TMEM_W * k;
      float sv[S::NA][TMEM_W];
      sums_chunk<S, NT>(trow, k, R, sv);
#pragma unroll
      for (int a = 0; a < S::NA; ++a) {
        float gl[TMEM_W];
        adjoint_chunk<S>(a, c, sv[a], g4[a], Fp, gl);
        const __half2 h0 = __floats2half2_rn(gl[0], gl[1]), h1 = __floats2half2_rn(gl[2], gl[3]);
        if (live)
          *reinterpret_cast<uint2 *>(Gi + a * S::NLM + c) =
              make_uint2(*reinterpret_cast<const uint32_t *>(&h0), *reinterpret_cast<const uint32_t *>(&h1));
      }
    }
  }
  if (live) {
    if constexpr (!TM) {
#pragma unroll
      for (int a = 0; a < S::NA; ++a) {
        float gl[S::NLM];
        adjoint_channel<S>(a, A, T, Fp, gl);
#pragma unroll
        for (int c = 0; c < S::NLM; c += 8) *reinterpret_cast<uint4 *>(Gi + a * S::NLM + c) = pack8_half(gl + c);
      }
    }
    {
      float tail[8];
      radial_tail<S>(P, Fp, tail);
      *reinterpret_cast<uint4 *>(Gi + S::NA * S::NLM) = pack8_half(tail);
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
  tc_fence_before();
  __syncthreads();
  if (t < 32) tmem_dealloc(tmem, TCOLS);
  block_sum_store<5, MIX_BLOCK / 32>(acc, part);
}

template <class S, class MT>
cudaError_t launch_descriptor_mixed(const Model<S> &P, const Geom &g, int n, const float4 *pos, const int32_t *nbr,
                                    const RowExt &X, __half *G, float *usite, float *qout, long long *Ffix,
                                    long long *part, int *status, const Fallback &fb, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  const int grid = (n + MIX_BLOCK - 1) / MIX_BLOCK;
  k_descriptor_mixed<S, MT><<<grid, MIX_BLOCK, 0, st>>>(P, g, n, pos, nbr, X, G, usite, qout, Ffix, part, status,
                                                        fb);
  return cudaGetLastError();
}

int mixed_descriptor_blocks(int n) { return (n + MIX_BLOCK - 1) / MIX_BLOCK; }

#define NEP_INSTANTIATE(SH, MT)                                                                                \
  template cudaError_t launch_descriptor_mixed<SH, MT>(const Model<SH> &, const Geom &, int, const float4 *,          \
                                                       const int32_t *, const RowExt &, __half *, float *, float *,   \
                                                       long long *, long long *, int *, const Fallback &,             \
                                                       cudaStream_t);
NEP_INSTANTIATE(CuShape, __nv_bfloat16)
NEP_INSTANTIATE(CuShape, __half)
NEP_INSTANTIATE(StudentShape, __nv_bfloat16)
NEP_INSTANTIATE(StudentShape, __half)
#undef NEP_INSTANTIATE

}  // namespace nep

// ---------------------------------------------------------------------------------------------------
// Self-test of the bounded mbarrier wait used above: one block initialises an mbarrier that nothing
// ever arrives on, waits with the same helper and a small poll limit, and reports the outcome in the
// same status word the kernels use -- a wait that runs out ends the kernel normally.
namespace nep {
namespace {
__global__ void k_wait_selftest(long polls, int *status) {
  __shared__ __align__(8) uint64_t mbar;
  if (threadIdx.x == 0) mbar_init(&mbar, 1);
  __syncthreads();
  const bool ok = mbar_wait(&mbar, 0, polls);
  if (!ok && threadIdx.x == 0) atomicOr(status, ST_TIMEOUT);
}
}  // namespace
}  // namespace nep

extern "C" nep_status nep_selftest_bounded_wait(int64_t polls, int *timed_out) {
  if (!timed_out || polls < 1 || polls > (1LL << 24)) return NEP_ERR_ARG;
  int *d = nullptr;
  if (cudaMalloc(&d, sizeof(int)) != cudaSuccess) { cudaGetLastError(); return NEP_ERR_OOM; }
  cudaError_t e = cudaMemset(d, 0, sizeof(int));
  if (e == cudaSuccess) {
    nep::k_wait_selftest<<<1, 32>>>((long)polls, d);
    e = cudaGetLastError();
  }
  int h = 0;
  if (e == cudaSuccess) e = cudaMemcpy(&h, d, sizeof(int), cudaMemcpyDeviceToHost);
  cudaFree(d);
  if (e != cudaSuccess) return NEP_ERR_CUDA;
  *timed_out = (h & nep::ST_TIMEOUT) ? 1 : 0;
  return NEP_OK;
}
