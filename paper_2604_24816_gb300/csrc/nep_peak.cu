// nep_peak.cu -- FP32 throughput microbenchmark of the GPU the library runs on.
//
// It measures the denominator of the FP32 roofline that the force kernels are reported against: every
// thread runs CHAINS independent multiply-add chains acc = acc * a + b for `iters` rounds, either as
// scalar fused multiply-adds (one FMA per instruction) or as packed float2 ones (two FMAs per
// instruction, the sm_100 family's paired FP32 form); a third form runs packed half2 FMAs, for comparing
// the 16-bit rate of the CUDA cores with the FP32 one.  The grid fills every SM with as many resident
// blocks as fit, so the FMA pipes, not the issue slots or the occupancy, are the limit.  Arithmetic
// performed = threads * iters * CHAINS * 2 FLOP (FMA = 2).  a and b are kernel arguments (no constant
// folding), the chain converges to b / (1 - a) = 1 (no overflow, no denormals), and every thread stores
// its sum (no dead-code elimination).  Thread 0 of each block also records its SM index and the SM's
// cycle counter (clock64) at the block's start and end; per SM, the span from its first block's start
// to its last block's end gives the rate per SM clock (FMA per cycle per SM), which does not depend on
// the clock frequency.
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "nep_gb300.h"

namespace {

constexpr int PEAK_BLOCK = 256;
constexpr int PEAK_CHAINS = 16;   // independent accumulators per thread (float2 form: 8 pairs)
constexpr int PEAK_UNROLL = 8;    // rounds per loop iteration (iters is a multiple of it)

// FORM 0: scalar float, 1: packed float2, 2: packed half2
template <int FORM>
__global__ void __launch_bounds__(PEAK_BLOCK) k_fp32_peak(float a, float b, long long rounds, float *out,
                                                          long long *cycles) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  __syncthreads();
  const long long c0 = clock64();
  float s = 0.f;
  if constexpr (FORM == 2) {
    __half2 acc[PEAK_CHAINS / 2];
#pragma unroll
    for (int c = 0; c < PEAK_CHAINS / 2; ++c)
      acc[c] = __floats2half2_rn(1e-3f * (float)(t & 255), 1e-3f * (float)c);
    const __half2 a2 = __floats2half2_rn(a, a), b2 = __floats2half2_rn(b, b);
    for (long long it = 0; it < rounds; ++it) {
#pragma unroll
      for (int u = 0; u < PEAK_UNROLL; ++u)
#pragma unroll
        for (int c = 0; c < PEAK_CHAINS / 2; ++c) acc[c] = __hfma2(acc[c], a2, b2);
    }
#pragma unroll
    for (int c = 0; c < PEAK_CHAINS / 2; ++c) s += __low2float(acc[c]) + __high2float(acc[c]);
  } else if constexpr (FORM == 1) {
    float2 acc[PEAK_CHAINS / 2];
#pragma unroll
    for (int c = 0; c < PEAK_CHAINS / 2; ++c) acc[c] = make_float2(1e-3f * (float)(t & 255), 1e-3f * (float)c);
    const float2 a2 = make_float2(a, a), b2 = make_float2(b, b);
    for (long long it = 0; it < rounds; ++it) {
#pragma unroll
      for (int u = 0; u < PEAK_UNROLL; ++u)
#pragma unroll
        for (int c = 0; c < PEAK_CHAINS / 2; ++c) acc[c] = __ffma2_rn(acc[c], a2, b2);
    }
#pragma unroll
    for (int c = 0; c < PEAK_CHAINS / 2; ++c) s += acc[c].x + acc[c].y;
  } else {
    float acc[PEAK_CHAINS];
#pragma unroll
    for (int c = 0; c < PEAK_CHAINS; ++c) acc[c] = 1e-3f * (float)((t + c) & 255);
    for (long long it = 0; it < rounds; ++it) {
#pragma unroll
      for (int u = 0; u < PEAK_UNROLL; ++u)
#pragma unroll
        for (int c = 0; c < PEAK_CHAINS; ++c) acc[c] = fmaf(acc[c], a, b);
    }
#pragma unroll
    for (int c = 0; c < PEAK_CHAINS; ++c) s += acc[c];
  }
  out[t] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned sm;
    asm volatile("mov.u32 %0, %%smid;" : "=r"(sm));
    cycles[3 * blockIdx.x] = c0;
    cycles[3 * blockIdx.x + 1] = clock64();
    cycles[3 * blockIdx.x + 2] = sm;
  }
}

}  // namespace

extern "C" nep_status nep_fp32_peak(int packed, double launch_ms, int reps, void *cuda_stream, double *best_tflops,
                                    double *median_tflops, double *fma_per_clock_sm, int *sm_count) {
  if (reps < 1 || reps > 10000 || !(launch_ms > 0.0 && launch_ms <= 1000.0)) return NEP_ERR_ARG;
  if (packed < 0 || packed > 2) return NEP_ERR_ARG;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(cuda_stream);
  int dev = 0, sms = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return NEP_ERR_CUDA;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) return NEP_ERR_CUDA;
  cudaError_t e =
      packed == 2   ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fp32_peak<2>, PEAK_BLOCK, 0)
      : packed == 1 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fp32_peak<1>, PEAK_BLOCK, 0)
                    : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fp32_peak<0>, PEAK_BLOCK, 0);
  if (e != cudaSuccess || per_sm <= 0) return NEP_ERR_CUDA;
  const int grid = sms * per_sm;
  const long long threads = (long long)grid * PEAK_BLOCK;
  float *out = nullptr;
  long long *cyc = nullptr;
  if (cudaMalloc(&out, sizeof(float) * (size_t)threads) != cudaSuccess) return NEP_ERR_OOM;
  if (cudaMalloc(&cyc, 3 * sizeof(long long) * (size_t)grid) != cudaSuccess) {
    cudaFree(out);
    return NEP_ERR_OOM;
  }
  std::vector<long long> hcyc(3 * (size_t)grid);
  double fpc = 0.0;
  cudaEvent_t t0 = nullptr, t1 = nullptr;
  nep_status status = NEP_OK;
  std::vector<double> rate;
  auto launch = [&](long long rounds) {
    // half2: a = 0.75, b = 0.25 (exact in half precision; the chain converges to 1 as well)
    if (packed == 2)
      k_fp32_peak<2><<<grid, PEAK_BLOCK, 0, st>>>(0.75f, 0.25f, rounds, out, cyc);
    else if (packed == 1)
      k_fp32_peak<1><<<grid, PEAK_BLOCK, 0, st>>>(0.9999f, 1e-4f, rounds, out, cyc);
    else
      k_fp32_peak<0><<<grid, PEAK_BLOCK, 0, st>>>(0.9999f, 1e-4f, rounds, out, cyc);
  };
  auto timed = [&](long long rounds, float *ms) -> bool {
    if (cudaEventRecord(t0, st) != cudaSuccess) return false;
    launch(rounds);
    if (cudaGetLastError() != cudaSuccess || cudaEventRecord(t1, st) != cudaSuccess) return false;
    if (cudaEventSynchronize(t1) != cudaSuccess) return false;
    return cudaEventElapsedTime(ms, t0, t1) == cudaSuccess;
  };
  do {
    if (cudaEventCreate(&t0) != cudaSuccess || cudaEventCreate(&t1) != cudaSuccess) { status = NEP_ERR_CUDA; break; }
    // calibrate the rounds per launch to about launch_ms
    long long rounds = 256;
    float ms = 0.f;
    if (!timed(rounds, &ms)) { status = NEP_ERR_CUDA; break; }       // warm-up
    for (int k = 0; k < 20 && ms < 0.5 * launch_ms; ++k) {
      rounds *= 2;
      if (!timed(rounds, &ms)) { status = NEP_ERR_CUDA; break; }
    }
    if (status != NEP_OK) break;
    rounds = std::max(1LL, (long long)((double)rounds * launch_ms / std::max(1e-3, (double)ms)));
    const double flop = (double)threads * (double)rounds * PEAK_UNROLL * PEAK_CHAINS * 2.0;
    for (int r = 0; r < reps; ++r) {
      if (!timed(rounds, &ms)) { status = NEP_ERR_CUDA; break; }
      rate.push_back(flop / (ms * 1e-3) / 1e12);
    }
    if (status != NEP_OK) break;
    // FMA per SM cycle of the last launch: per SM, its blocks' FMAs over the span from the earliest
    // block start to the latest block end (one SM's counter); averaged over the SMs
    if (cudaMemcpy(hcyc.data(), cyc, 3 * sizeof(long long) * (size_t)grid, cudaMemcpyDeviceToHost) != cudaSuccess) {
      status = NEP_ERR_CUDA;
      break;
    }
    std::vector<long long> first, last, nblk;
    for (int b = 0; b < grid; ++b) {
      const size_t sm = (size_t)hcyc[3 * (size_t)b + 2];
      if (sm >= 4096) continue;
      if (sm >= first.size()) { first.resize(sm + 1, -1); last.resize(sm + 1, -1); nblk.resize(sm + 1, 0); }
      const long long c0 = hcyc[3 * (size_t)b], c1 = hcyc[3 * (size_t)b + 1];
      first[sm] = first[sm] < 0 ? c0 : std::min(first[sm], c0);
      last[sm] = std::max(last[sm], c1);
      nblk[sm] += 1;
    }
    double sum = 0.0;
    int used = 0;
    for (size_t sm = 0; sm < first.size(); ++sm) {
      if (nblk[sm] == 0 || last[sm] <= first[sm]) continue;
      sum += (double)nblk[sm] * PEAK_BLOCK * (double)rounds * PEAK_UNROLL * PEAK_CHAINS / (double)(last[sm] - first[sm]);
      ++used;
    }
    fpc = used > 0 ? sum / used : 0.0;
  } while (false);
  if (t0) cudaEventDestroy(t0);
  if (t1) cudaEventDestroy(t1);
  cudaFree(out);
  cudaFree(cyc);
  if (status != NEP_OK) return status;
  std::sort(rate.begin(), rate.end());
  if (best_tflops) *best_tflops = rate.back();
  if (median_tflops) *median_tflops = rate[rate.size() / 2];
  if (fma_per_clock_sm) *fma_per_clock_sm = fpc;
  if (sm_count) *sm_count = sms;
  return NEP_OK;
}
