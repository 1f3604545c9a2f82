// nep_md.cu -- velocity-Verlet integration, step control, reductions and layout kernels (sm_103a).
//
// Positions and velocities are float64 (structure of arrays, cell-sorted order); forces are float32.
// Between rebuilds positions are not wrapped, so each atom's cell-relative float32 coordinate
// p = x - (cell origin) stays continuous; wrapping happens in the rebuild.  The drift kernel flags any
// atom whose cell-relative coordinate moved more than skin/2 since the last rebuild; the control
// kernel then asks the next rebuild chain to run.
#include "nep_common.cuh"

#include <cfloat>

namespace nep {

constexpr double KE_CONV = 103.642696562;          // 1 amu Angstrom^2/fs^2 in eV

__device__ __forceinline__ double fix_to_double(long long f) { return (double)f * FIX_INV; }

// The warp's displacement news: any atom past skin/2 (-> rebuild), and the largest squared
// displacement since the rebuild (non-negative floats order like their bit patterns).
__device__ __forceinline__ void note_displacement(bool moved, float dd, Control *ctrl) {
  const unsigned m = __reduce_max_sync(0xffffffffu, __float_as_uint(dd));
  const bool any = __any_sync(0xffffffffu, moved);
  if ((threadIdx.x & 31) == 0) {
    if (any) atomicOr(&ctrl->moved, 1);
    if (m > 0u) atomicMax(reinterpret_cast<unsigned *>(&ctrl->dmax2), m);
  }
}

__global__ void k_kick_drift(int n, double *__restrict__ x, double *__restrict__ y, double *__restrict__ z,
                             double *__restrict__ vx, double *__restrict__ vy, double *__restrict__ vz,
                             const long long *__restrict__ F, float4 *__restrict__ pos,
                             const float4 *__restrict__ pos_ref, double kick, double dt, double lx, double ly,
                             double lz, float half_skin2, Control *ctrl) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  bool moved = false;
  float dd = 0.f;                      // squared displacement since the rebuild (capped; NaN -> cap)
  if (i < n) {
    // kick_fix = kick * 2^-32: one conversion and one FMA per component on the narrow FP64 pipe.  When
    // the previous step's closing half kick is owed (the same forces), it is applied first, as its own
    // FMA: the same arithmetic as two separate kicks, so trajectories do not depend on how the steps
    // are grouped into calls.
    const double kick_fix = kick * FIX_INV;
    const double fx = (double)F[i], fy = (double)F[(size_t)n + i], fz = (double)F[2 * (size_t)n + i];
    double ux = vx[i], uy = vy[i], uz = vz[i];
    if (ctrl->pending) {
      ux = fma(kick_fix, fx, ux);
      uy = fma(kick_fix, fy, uy);
      uz = fma(kick_fix, fz, uz);
    }
    ux = fma(kick_fix, fx, ux);
    uy = fma(kick_fix, fy, uy);
    uz = fma(kick_fix, fz, uz);
    vx[i] = ux; vy[i] = uy; vz[i] = uz;
    const double px = x[i] + dt * ux, py = y[i] + dt * uy, pz = z[i] + dt * uz;
    x[i] = px; y[i] = py; z[i] = pz;
    const float4 p = pos[i];
    const int cx = cell_x(p.w), cy = cell_y(p.w), cz = cell_z(p.w);
    const float4 q = make_float4((float)fma(-(double)cx, lx, px), (float)fma(-(double)cy, ly, py),
                                 (float)fma(-(double)cz, lz, pz), p.w);
    pos[i] = q;
    const float4 r = pos_ref[i];
    const float ddx = q.x - r.x, ddy = q.y - r.y, ddz = q.z - r.z;
    const float d2 = ddx * ddx + ddy * ddy + ddz * ddz;
    moved = !(d2 <= half_skin2);       // also true for NaN
    dd = d2 <= 1.0e30f ? d2 : 1.0e30f;
  }
  note_displacement(moved, dd, ctrl);
}

// Decide whether this step rebuilds the neighbour list.
// After the rebuild decision: may the row walks of this evaluation leave the far bands out (no atom
// moved far enough since the build to bring a far-band pair inside rc_R)?
__device__ __forceinline__ void decide_far(Control *ctrl) {
  if (ctrl->do_rebuild) ctrl->dmax2 = 0.f;
  ctrl->skip_far = ctrl->dmax2 < ctrl->far_dmax2 ? 1 : 0;
}

__device__ __forceinline__ int step_control(Control *ctrl) {
  ctrl->steps += 1;
  ctrl->steps_since += 1;
  int rb = ctrl->moved | ctrl->force_rebuild;
  if (ctrl->rebuild_every > 0 && ctrl->steps_since >= ctrl->rebuild_every) rb = 1;
  ctrl->do_rebuild = rb;
  if (rb) {
    ctrl->moved = 0;
    ctrl->force_rebuild = 0;
    ctrl->steps_since = 0;
    ctrl->rebuilds += 1;
  }
  decide_far(ctrl);
  ctrl->pending = 1;    // this step's closing half kick: done by the next step's opening kick or the final one
  return rb;
}
__global__ void k_control(Control *ctrl) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  step_control(ctrl);
}
// The same in a captured MD step, where the rebuild chain is the body of a conditional graph node:
// the decision also sets that node's condition, so that a step without a rebuild launches none of the
// chain's kernels.
__global__ void k_control_cond(Control *ctrl, cudaGraphConditionalHandle cond) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  cudaGraphSetConditional(cond, step_control(ctrl) ? 1u : 0u);
}

// Outside MD steps, after an upload that kept the list: rebuild only if an atom moved more than
// skin/2 (or a rebuild was requested); the step counters are not touched.
__global__ void k_control_check(Control *ctrl) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const int rb = ctrl->moved | ctrl->force_rebuild;
  ctrl->do_rebuild = rb;
  if (rb) {
    ctrl->moved = 0;
    ctrl->force_rebuild = 0;
    ctrl->steps_since = 0;
    ctrl->rebuilds += 1;
  }
  decide_far(ctrl);
}

// Rebuild unconditionally (outside MD steps).
__global__ void k_control_force(Control *ctrl) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  ctrl->do_rebuild = 1;
  ctrl->moved = 0;
  ctrl->force_rebuild = 0;
  ctrl->steps_since = 0;
  ctrl->rebuilds += 1;
  decide_far(ctrl);
}

// The closing half kick of md_verlet_step's last step, with the kinetic-energy partials.
__global__ void k_kick(int n, double *__restrict__ vx, double *__restrict__ vy, double *__restrict__ vz,
                       const long long *__restrict__ F, double kick, double mass, long long *__restrict__ part,
                       Control *ctrl) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i == 0) ctrl->pending = 0;
  long long acc[1] = {0};
  if (i < n) {
    const double kick_fix = kick * FIX_INV;
    const double ux = fma(kick_fix, (double)F[i], vx[i]);
    const double uy = fma(kick_fix, (double)F[(size_t)n + i], vy[i]);
    const double uz = fma(kick_fix, (double)F[2 * (size_t)n + i], vz[i]);
    vx[i] = ux; vy[i] = uy; vz[i] = uz;
    acc[0] = __double2ll_rn(0.5 * mass * KE_CONV * (ux * ux + uy * uy + uz * uz) * 4294967296.0);
  }
  block_sum_store<1>(acc, part);
}

// Kinetic energy only (no kick): for thermo outside MD steps.
__global__ void k_kinetic(int n, const double *__restrict__ vx, const double *__restrict__ vy,
                          const double *__restrict__ vz, double mass, long long *__restrict__ part) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  long long acc[1] = {0};
  if (i < n) acc[0] = __double2ll_rn(0.5 * mass * KE_CONV * (vx[i] * vx[i] + vy[i] * vy[i] + vz[i] * vz[i]) * 4294967296.0);
  block_sum_store<1>(acc, part);
}

// Reduction of the per-block int64 partials (fixed point for energies and virial), one block per
// reduced quantity v:
//   pd (stride 5):  {site energy, radial pairs, angular pairs, list entries, active pairs} (descriptor)
//   pf (stride 13): {virial W[9], owned list entries, owned active, owned radial, owned angular} (force)
//   pk (stride 1):  kinetic energy
// sums[v]: 0 E, 1..9 W, 10 KE, 11..14 descriptor counts, 15..18 force counts;
// counters[v - 11] += sums[v] for v >= 11, counters[8] += 1 per evaluation.
constexpr int N_SUMS = 19;

constexpr int FIN_THREADS = 1024;   // one block per sum; the partials are 8-byte integers, so the
                                    // order of the additions does not change the result
__global__ void __launch_bounds__(FIN_THREADS)
k_finalize(const long long *__restrict__ pd, int nbd, const long long *__restrict__ pf, int nbf,
           const long long *__restrict__ pk, int nbk, double *__restrict__ sums, long long *__restrict__ counters) {
  static_assert(FIN_THREADS == 1024, "32 warp sums, reduced by one warp");
  __shared__ long long red[FIN_THREADS / 32];
  const int v = blockIdx.x;
  const long long *src;
  int nb, stride, off;
  if (v == 0) { src = pd; nb = nbd; stride = 5; off = 0; }
  else if (v <= 9) { src = pf; nb = nbf; stride = 13; off = v - 1; }
  else if (v == 10) { src = pk; nb = nbk; stride = 1; off = 0; }
  else if (v <= 14) { src = pd; nb = nbd; stride = 5; off = v - 10; }
  else { src = pf; nb = nbf; stride = 13; off = 9 + (v - 15); }
  if (src == nullptr) return;
  long long t = 0;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) t += src[(size_t)b * stride + off];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = t;
  __syncthreads();
  if (threadIdx.x < 32) {
    t = red[threadIdx.x];                              // FIN_THREADS / 32 == 32 warp sums
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  }
  if (threadIdx.x == 0) {
    const long long tot = t;
    sums[v] = v <= 10 ? (double)tot * FIX_INV : (double)tot;       // energies/virial are fixed point
    if (counters != nullptr && v >= 11) counters[v - 11] += tot;
    if (counters != nullptr && v == 0) counters[8] += 1;
  }
}

// [n][3] float64 (original order) -> SoA float64, ids = 0..n-1.
__global__ void k_load_state(int n, const double *__restrict__ xin, const double *__restrict__ vin,
                             double *__restrict__ x, double *__restrict__ y, double *__restrict__ z,
                             double *__restrict__ vx, double *__restrict__ vy, double *__restrict__ vz,
                             int *__restrict__ id, int *__restrict__ status) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  const double a = xin[3 * (size_t)s], b = xin[3 * (size_t)s + 1], c = xin[3 * (size_t)s + 2];
  if (!(isfinite(a) && isfinite(b) && isfinite(c))) atomicOr(status, ST_NAN);
  x[s] = a; y[s] = b; z[s] = c;
  if (vin != nullptr) {
    vx[s] = vin[3 * (size_t)s]; vy[s] = vin[3 * (size_t)s + 1]; vz[s] = vin[3 * (size_t)s + 2];
  } else {
    vx[s] = 0.0; vy[s] = 0.0; vz[s] = 0.0;
  }
  id[s] = s;
}

// Upload into the current cell-sorted order, keeping the neighbour list: slot s takes the input atom
// id[s] (original order).  Each position is moved to its periodic image nearest the slot's current
// position (so the cell-relative coordinate stays continuous, as between rebuilds), the cell-relative
// float32 coordinate is refreshed in the slot's cell, and an atom that moved more than skin/2 from
// the positions the list was built for sets ctrl->moved (the next evaluation then rebuilds).
// inv[id[s]] = s: the cell-order slot of every atom (original order).
__global__ void k_inverse_order(int n, const int *__restrict__ id, int *__restrict__ inv) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s < n) inv[id[s]] = s;
}

// One thread per atom in the caller's order (i; its slot s = inv[i]), so that the reads of xin and vin
// are contiguous: they may live in host memory that the kernel reads directly.
__global__ void k_load_state_sorted(int n, const double *__restrict__ xin, const double *__restrict__ vin,
                                    const int *__restrict__ inv, double *__restrict__ x, double *__restrict__ y,
                                    double *__restrict__ z, double *__restrict__ vx, double *__restrict__ vy,
                                    double *__restrict__ vz, float4 *__restrict__ pos,
                                    const float4 *__restrict__ pos_ref, double lx, double ly, double lz, double Lx,
                                    double Ly, double Lz, float half_skin2, Control *ctrl) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  bool moved = false, changed = false;
  float dd = 0.f;
  if (i < n) {
    const int s = inv[i];
    const size_t o = 3 * (size_t)i;
    double a = xin[o], b = xin[o + 1], c = xin[o + 2];
    if (!(isfinite(a) && isfinite(b) && isfinite(c))) {
      atomicOr(&ctrl->status, ST_NAN);
      moved = true;
    } else {
      a -= Lx * rint((a - x[s]) / Lx);
      b -= Ly * rint((b - y[s]) / Ly);
      c -= Lz * rint((c - z[s]) / Lz);
      // a coordinate that differs from the current one only by the rounding of a periodic wrap (the
      // state read back by nep_get_state is wrapped into the box; adding the edge back can be an ulp
      // off) is the current one
      const double tx = 8.0 * DBL_EPSILON * Lx, ty = 8.0 * DBL_EPSILON * Ly, tz = 8.0 * DBL_EPSILON * Lz;
      if (fabs(a - x[s]) <= tx) a = x[s];
      if (fabs(b - y[s]) <= ty) b = y[s];
      if (fabs(c - z[s]) <= tz) c = z[s];
    }
    x[s] = a; y[s] = b; z[s] = c;
    if (vin != nullptr) {
      vx[s] = vin[o]; vy[s] = vin[o + 1]; vz[s] = vin[o + 2];
    } else {
      vx[s] = 0.0; vy[s] = 0.0; vz[s] = 0.0;
    }
    const float4 p = pos[s];
    const int cx = cell_x(p.w), cy = cell_y(p.w), cz = cell_z(p.w);
    const float4 q = make_float4((float)fma(-(double)cx, lx, a), (float)fma(-(double)cy, ly, b),
                                 (float)fma(-(double)cz, lz, c), p.w);
    pos[s] = q;
    // the forces depend on the positions only through these float32 coordinates
    changed = __float_as_uint(q.x) != __float_as_uint(p.x) || __float_as_uint(q.y) != __float_as_uint(p.y) ||
              __float_as_uint(q.z) != __float_as_uint(p.z);
    const float4 r = pos_ref[s];
    const float ddx = q.x - r.x, ddy = q.y - r.y, ddz = q.z - r.z;
    const float d2 = ddx * ddx + ddy * ddy + ddz * ddz;
    moved = moved || !(d2 <= half_skin2);
    dd = moved ? 1.0e30f : d2;
  }
  note_displacement(moved, dd, ctrl);
  if (__any_sync(0xffffffffu, changed) && (threadIdx.x & 31) == 0) atomicOr(&ctrl->changed, 1);
}

// Sorted SoA -> original-order [n][3] float64 (positions wrapped into the box when L != nullptr).
// One thread per atom in the caller's order (contiguous writes: out may be host memory).
constexpr int MD_STAGE = 256;   // threads per block of the row-staging form
// WIDE: out is 16-byte aligned; the block's rows go through shared memory and leave with 16-byte stores
// of consecutive addresses (blockDim.x == MD_STAGE), so page-locked host memory is written by the
// kernel itself in full lines.
template <bool WIDE>
__global__ void k_store_vec(int n, const int *__restrict__ inv, const double *__restrict__ a, const double *__restrict__ b,
                            const double *__restrict__ c, double Lx, double Ly, double Lz, int wrap,
                            double *__restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  __shared__ double so[WIDE ? 3 * MD_STAGE : 1];
  if (i < n) {
    const int s = inv[i];
    double u = a[s], v = b[s], w = c[s];
    if (wrap) {
      u -= Lx * floor(u / Lx); if (u >= Lx) u -= Lx;
      v -= Ly * floor(v / Ly); if (v >= Ly) v -= Ly;
      w -= Lz * floor(w / Lz); if (w >= Lz) w -= Lz;
    }
    if constexpr (WIDE) {
      const int t3 = 3 * (int)threadIdx.x;
      so[t3] = u; so[t3 + 1] = v; so[t3 + 2] = w;
    } else {
      const size_t o = 3 * (size_t)i;
      out[o] = u; out[o + 1] = v; out[o + 2] = w;
    }
  }
  if constexpr (WIDE) {
    __syncthreads();
    const int base = blockIdx.x * blockDim.x, cnt = min((int)blockDim.x, n - base), nd = 3 * cnt;
    double2 *g = reinterpret_cast<double2 *>(out + 3 * (size_t)base);
    for (int t = threadIdx.x; t < nd / 2; t += blockDim.x) g[t] = make_double2(so[2 * t], so[2 * t + 1]);
    if ((nd & 1) && threadIdx.x == 0) out[3 * (size_t)base + nd - 1] = so[nd - 1];
  }
}

__global__ void k_store_force(int n, const int *__restrict__ id, const long long *__restrict__ F,
                              double *__restrict__ out) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  const size_t o = 3 * (size_t)id[s];
  out[o] = fix_to_double(F[s]);
  out[o + 1] = fix_to_double(F[(size_t)n + s]);
  out[o + 2] = fix_to_double(F[2 * (size_t)n + s]);
}

__global__ void k_store_scalar(int n, const int *__restrict__ id, const float *__restrict__ u, double *__restrict__ out) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  out[id[s]] = u[s];
}

__global__ void k_store_rows(int n, int width, const int *__restrict__ id, const float *__restrict__ q,
                             float *__restrict__ out) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  for (int v = 0; v < width; ++v) out[(size_t)id[s] * width + v] = q[(size_t)s * width + v];
}

__global__ void k_store_neighbors(int n, int cap_in, int cap_out, const int *__restrict__ id, const int32_t *__restrict__ nbr,
                                  const int32_t *__restrict__ nnum, const int32_t *__restrict__ nang,
                                  const int32_t *__restrict__ nown, int32_t *__restrict__ counts,
                                  int32_t *__restrict__ n_ang, int32_t *__restrict__ n_own, int32_t *__restrict__ list) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  const int o = id[s];
  const int c = nnum[s];
  counts[o] = c;
  n_ang[o] = nang[s];
  n_own[o] = nown[s];
  for (int k = 0; k < c && k < cap_out; ++k) list[(size_t)o * cap_out + k] = id[nbr[(size_t)k * n + s] & J_MASK];
  for (int k = c; k < cap_out; ++k) list[(size_t)o * cap_out + k] = -1;
  (void)cap_in;
}

// ---------------------------------------------------------------------------------------------------
static int bl(long long m, int b) { return (int)((m + b - 1) / b); }

constexpr int MD_BLOCK = 256;
int md_blocks(int n) { return bl(n, MD_BLOCK); }

cudaError_t launch_kick_drift(int n, double *x, double *y, double *z, double *vx, double *vy, double *vz, const long long *F,
                              float4 *pos, const float4 *pos_ref, double kick, double dt, const double l[3],
                              float half_skin2, Control *ctrl, cudaStream_t st) {
  if (n > 0)
    k_kick_drift<<<bl(n, MD_BLOCK), MD_BLOCK, 0, st>>>(n, x, y, z, vx, vy, vz, F, pos, pos_ref, kick, dt, l[0], l[1],
                                                       l[2], half_skin2, ctrl);
  return cudaGetLastError();
}

cudaError_t launch_control_cond(Control *ctrl, cudaGraphConditionalHandle cond, cudaStream_t st) {
  k_control_cond<<<1, 32, 0, st>>>(ctrl, cond);
  return cudaGetLastError();
}

cudaError_t launch_control(Control *ctrl, bool force, cudaStream_t st) {
  if (force) k_control_force<<<1, 32, 0, st>>>(ctrl);
  else k_control<<<1, 32, 0, st>>>(ctrl);
  return cudaGetLastError();
}

cudaError_t launch_kick(int n, double *vx, double *vy, double *vz, const long long *F, double kick, double mass, long long *part,
                        Control *ctrl, cudaStream_t st) {
  if (n > 0) k_kick<<<bl(n, MD_BLOCK), MD_BLOCK, 0, st>>>(n, vx, vy, vz, F, kick, mass, part, ctrl);
  return cudaGetLastError();
}

cudaError_t launch_kinetic(int n, const double *vx, const double *vy, const double *vz, double mass, long long *part,
                           cudaStream_t st) {
  if (n > 0) k_kinetic<<<bl(n, MD_BLOCK), MD_BLOCK, 0, st>>>(n, vx, vy, vz, mass, part);
  return cudaGetLastError();
}

cudaError_t launch_finalize(const long long *pd, int nbd, const long long *pf, int nbf, const long long *pk, int nbk,
                            double *sums, long long *counters, cudaStream_t st) {
  k_finalize<<<N_SUMS, FIN_THREADS, 0, st>>>(pd, nbd, pf, nbf, pk, nbk, sums, counters);
  return cudaGetLastError();
}

cudaError_t launch_load_state(int n, const double *xin, const double *vin, double *x, double *y, double *z, double *vx,
                              double *vy, double *vz, int *id, int *status, cudaStream_t st) {
  if (n > 0) k_load_state<<<bl(n, 256), 256, 0, st>>>(n, xin, vin, x, y, z, vx, vy, vz, id, status);
  return cudaGetLastError();
}

cudaError_t launch_control_check(Control *ctrl, cudaStream_t st) {
  k_control_check<<<1, 32, 0, st>>>(ctrl);
  return cudaGetLastError();
}

cudaError_t launch_inverse_order(int n, const int *id, int *inv, cudaStream_t st) {
  if (n > 0) k_inverse_order<<<bl(n, 256), 256, 0, st>>>(n, id, inv);
  return cudaGetLastError();
}

cudaError_t launch_load_state_sorted(int n, const double *xin, const double *vin, const int *inv, double *x, double *y,
                                     double *z, double *vx, double *vy, double *vz, float4 *pos, const float4 *pos_ref,
                                     const double l[3], const double L[3], float half_skin2, Control *ctrl,
                                     cudaStream_t st) {
  if (n > 0)
    k_load_state_sorted<<<bl(n, 256), 256, 0, st>>>(n, xin, vin, inv, x, y, z, vx, vy, vz, pos, pos_ref, l[0], l[1],
                                                    l[2], L[0], L[1], L[2], half_skin2, ctrl);
  return cudaGetLastError();
}

cudaError_t launch_store_vec(int n, const int *inv, const double *a, const double *b, const double *c, const double L[3],
                             int wrap, double *out, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  if (((uintptr_t)out & 15) == 0)
    k_store_vec<true><<<bl(n, MD_STAGE), MD_STAGE, 0, st>>>(n, inv, a, b, c, L[0], L[1], L[2], wrap, out);
  else
    k_store_vec<false><<<bl(n, 256), 256, 0, st>>>(n, inv, a, b, c, L[0], L[1], L[2], wrap, out);
  return cudaGetLastError();
}

cudaError_t launch_store_force(int n, const int *id, const long long *F, double *out, cudaStream_t st) {
  if (n > 0) k_store_force<<<bl(n, 256), 256, 0, st>>>(n, id, F, out);
  return cudaGetLastError();
}

cudaError_t launch_store_scalar(int n, const int *id, const float *u, double *out, cudaStream_t st) {
  if (n > 0) k_store_scalar<<<bl(n, 256), 256, 0, st>>>(n, id, u, out);
  return cudaGetLastError();
}

cudaError_t launch_store_rows(int n, int width, const int *id, const float *q, float *out, cudaStream_t st) {
  if (n > 0) k_store_rows<<<bl(n, 256), 256, 0, st>>>(n, width, id, q, out);
  return cudaGetLastError();
}

cudaError_t launch_store_neighbors(int n, int cap_in, int cap_out, const int *id, const int32_t *nbr, const int32_t *nnum,
                                   const int32_t *nang, const int32_t *nown, int32_t *counts, int32_t *n_ang,
                                   int32_t *n_own, int32_t *list, cudaStream_t st) {
  if (n > 0)
    k_store_neighbors<<<bl(n, 256), 256, 0, st>>>(n, cap_in, cap_out, id, nbr, nnum, nang, nown, counts, n_ang, n_own,
                                                  list);
  return cudaGetLastError();
}

}  // namespace nep
