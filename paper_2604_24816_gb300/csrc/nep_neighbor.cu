// nep_neighbor.cu -- cell binning, cell sort and banded half/full neighbour lists on sm_103a.
//
// Rebuild pipeline (every kernel takes the control block and returns at once when the current step
// does not rebuild, so the whole MD step can be replayed as one CUDA graph):
//   k_cell_zero     clear per-cell counters
//   k_cell_assign   wrap x into the box (float64), cell = floor(x / l) per dimension, histogram
//   k_scan_*        exclusive scan of the histogram -> cell_start (3 kernels, integer, deterministic)
//   k_scatter       slot within the cell (arbitrary order), then
//   k_cell_sort     sort each cell's atoms by original id: the sorted order is a pure function of the
//                   positions, independent of launch timing and of the previous order
//   k_permute       gather x, v, id into the new order; cell-relative float32 coordinates
//   k_copy_back     copy the gathered arrays back (fixed device pointers for graph replay)
//   k_neighbors     for each atom, every j with |r_ij| < rc_R + skin among the 27 neighbouring cell
//                   images, split into the pairs this atom owns (one owner per unordered pair) and the
//                   rest, each part grouped by distance band so that the per-pair branches of the
//                   force kernels stay warp-uniform.
// Distances use cell-relative float32 coordinates plus the image offset of the neighbouring cell, so
// their error does not grow with the box size (float64 appears only in the wrap and cell assignment).
#include "nep_common.cuh"

#include <algorithm>

namespace nep {

constexpr int SCAN_THREADS = 1024;
constexpr int SCAN_ITEMS = 4;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

__global__ void k_cell_zero(int ncell, int *__restrict__ count, int *__restrict__ cursor, Control *ctrl) {
  if (!ctrl->do_rebuild) return;
  if (blockIdx.x == 0 && threadIdx.x == 0) ctrl->nb_next = 0;   // the neighbour scan's work counter
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < ncell; c += gridDim.x * blockDim.x) {
    count[c] = 0;
    cursor[c] = 0;
  }
}

__device__ __forceinline__ double wrap_coord(double x, double L) {
  double y = x - L * floor(x / L);
  if (y >= L) y -= L;
  if (y < 0.0) y = 0.0;
  return y;
}

__global__ void k_cell_assign(int n, double *__restrict__ x, double *__restrict__ y, double *__restrict__ z, double Lx,
                              double Ly, double Lz, double lx, double ly, double lz, int ncx, int ncy, int ncz,
                              int *__restrict__ cell_of, int *__restrict__ count, Control *ctrl) {
  if (!ctrl->do_rebuild) return;
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gridDim.x * blockDim.x) {
    double px = x[s], py = y[s], pz = z[s];
    if (!(isfinite(px) && isfinite(py) && isfinite(pz))) {
      atomicOr(&ctrl->status, ST_NAN);
      px = py = pz = 0.0;
    }
    px = wrap_coord(px, Lx); py = wrap_coord(py, Ly); pz = wrap_coord(pz, Lz);
    x[s] = px; y[s] = py; z[s] = pz;
    const int cx = min((int)(px / lx), ncx - 1), cy = min((int)(py / ly), ncy - 1), cz = min((int)(pz / lz), ncz - 1);
    const int c = (cz * ncy + cy) * ncx + cx;
    cell_of[s] = c;
    atomicAdd(count + c, 1);
  }
}

// Exclusive scan of count[0..m) into start[0..m], start[m] = total.  Tile scan + carry pass + add.
__global__ void __launch_bounds__(SCAN_THREADS)
k_scan_tiles(int m, const int *__restrict__ in, int *__restrict__ out, int *__restrict__ tile_sums, const Control *ctrl) {
  if (!ctrl->do_rebuild) return;
  __shared__ int warp_tot[SCAN_THREADS / 32];
  const int base = blockIdx.x * SCAN_TILE + threadIdx.x * SCAN_ITEMS;
  int v[SCAN_ITEMS], run = 0;
#pragma unroll
  for (int k = 0; k < SCAN_ITEMS; ++k) {
    v[k] = (base + k < m) ? in[base + k] : 0;
    run += v[k];
  }
  // inclusive warp scan of per-thread totals
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int t = run;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int u = __shfl_up_sync(0xffffffffu, t, o);
    if (lane >= o) t += u;
  }
  if (lane == 31) warp_tot[warp] = t;
  __syncthreads();
  if (warp == 0) {
    int w = warp_tot[lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int u = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += u;
    }
    warp_tot[lane] = w;
  }
  __syncthreads();
  int excl = t - run + (warp > 0 ? warp_tot[warp - 1] : 0);
#pragma unroll
  for (int k = 0; k < SCAN_ITEMS; ++k) {
    if (base + k < m) out[base + k] = excl;
    excl += v[k];
  }
  if (threadIdx.x == SCAN_THREADS - 1) tile_sums[blockIdx.x] = excl;
}

__global__ void k_scan_carry(int ntiles, int *__restrict__ tile_sums, int m, int *__restrict__ out, const Control *ctrl) {
  if (!ctrl->do_rebuild) return;
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  int run = 0;
  for (int b = 0; b < ntiles; ++b) {
    int s = tile_sums[b];
    tile_sums[b] = run;
    run += s;
  }
  out[m] = run;
}

__global__ void k_scan_add(int m, int *__restrict__ out, const int *__restrict__ tile_sums, const Control *ctrl) {
  if (!ctrl->do_rebuild) return;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < m; idx += gridDim.x * blockDim.x)
    out[idx] += tile_sums[idx / SCAN_TILE];
}

__global__ void k_scatter(int n, const int *__restrict__ cell_of, const int *__restrict__ start, int *__restrict__ cursor,
                          int *__restrict__ perm, const Control *ctrl) {
  if (!ctrl->do_rebuild) return;
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gridDim.x * blockDim.x) {
    const int c = cell_of[s];
    perm[start[c] + atomicAdd(cursor + c, 1)] = s;
  }
}

// One thread per cell: insertion sort of the cell's slots by original id (ids are unique).
__global__ void k_cell_sort(int ncell, const int *__restrict__ start, int *__restrict__ perm, const int *__restrict__ id,
                            const Control *ctrl) {
  if (!ctrl->do_rebuild) return;
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < ncell; c += gridDim.x * blockDim.x) {
    const int b = start[c], e = start[c + 1];
    for (int p = b + 1; p < e; ++p) {
      const int s = perm[p];
      const int key = id[s];
      int q = p;
      while (q > b && id[perm[q - 1]] > key) {
        perm[q] = perm[q - 1];
        --q;
      }
      perm[q] = s;
    }
  }
}

__global__ void k_permute(int n, const int *__restrict__ perm, const double *__restrict__ x, const double *__restrict__ y,
                          const double *__restrict__ z, const double *__restrict__ vx, const double *__restrict__ vy,
                          const double *__restrict__ vz, const int *__restrict__ id, const int *__restrict__ cell_of,
                          double *__restrict__ xb, double *__restrict__ yb, double *__restrict__ zb,
                          double *__restrict__ vxb, double *__restrict__ vyb, double *__restrict__ vzb,
                          int *__restrict__ idb, float4 *__restrict__ pos, float4 *__restrict__ pos_ref, double lx,
                          double ly, double lz, int ncx, int ncy, const Control *ctrl) {
  if (!ctrl->do_rebuild) return;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
    const int s = perm[t];
    const double px = x[s], py = y[s], pz = z[s];
    xb[t] = px; yb[t] = py; zb[t] = pz;
    vxb[t] = vx[s]; vyb[t] = vy[s]; vzb[t] = vz[s];
    idb[t] = id[s];
    const int c = cell_of[s];
    const int cx = c % ncx, cy = (c / ncx) % ncy, cz = c / (ncx * ncy);
    // the same expression as the drift and upload kernels (nep_md.cu), so that a position uploaded
    // unchanged gives bitwise the same cell-relative coordinates
    const float4 p = make_float4((float)fma(-(double)cx, lx, px), (float)fma(-(double)cy, ly, py),
                                 (float)fma(-(double)cz, lz, pz), __int_as_float(cx | (cy << 10) | (cz << 20)));
    pos[t] = p;
    pos_ref[t] = p;
  }
}

__global__ void k_copy_back(int n, double *__restrict__ x, double *__restrict__ y, double *__restrict__ z,
                            double *__restrict__ vx, double *__restrict__ vy, double *__restrict__ vz,
                            int *__restrict__ id, const double *__restrict__ xb, const double *__restrict__ yb,
                            const double *__restrict__ zb, const double *__restrict__ vxb,
                            const double *__restrict__ vyb, const double *__restrict__ vzb,
                            const int *__restrict__ idb, const Control *ctrl) {
  if (!ctrl->do_rebuild) return;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
    x[t] = xb[t]; y[t] = yb[t]; z[t] = zb[t];
    vx[t] = vxb[t]; vy[t] = vyb[t]; vz[t] = vzb[t];
    id[t] = idb[t];
  }
}

// One warp per atom over the candidates of the 27 neighbouring cell images (below).
//
// Segments: the pair (i, j) is "owned" by i when r_ij lies in the upper half-space (see owns_pair;
// exactly one of r_ij and r_ji = -r_ij is owned, so every unordered pair has one owner), and the row
// is laid out as [owned | not owned], each part grouped by build-time distance band:
// [0, rc_A), [rc_A, rc_A + skin), [rc_A + skin, rc_R), [rc_R, rc_R + e), [rc_R + e, rc_R + skin) with
// e = FAR_EDGE skin, in stencil order inside a band.  The half-list force kernels walk only the owned part (each pair once,
// Newton's third law); the other walks take the whole row.  The last ("far") band of each part can
// only hold a pair inside rc_R after some atom moved more than e/2 since the build, so while the
// largest displacement stays below that the walks leave both far bands out (their counts go to
// nfar).  Because every atom of a lattice owns exactly half of each shell and the bands follow the
// shells, the per-pair branches stay warp-uniform without a full sort.
// The placement's 4-byte stores into the neighbour-major list are scattered across rows; L2 merges
// them into full sectors before they reach DRAM.
constexpr int NB_WARPS = 8;            // atoms (one warp each) per block
constexpr int NB_STAGE = 128;          // staged entries per atom (lists longer than this are an overflow)
constexpr float OWN_EPS = 0.5f;        // Angstrom; lattice-vector components are either ~0 or >= a/2

struct Bands {
  float b0, b1, b2, b3, b4;  // squared band edges: rc_A^2, (rc_A+skin)^2, rc_R^2, (rc_R+e)^2, (rc_R+skin)^2
};
constexpr int NB_SEG = 10;             // segments of a row: [owned | not owned] x 5 distance bands

// Upper half-space test, exactly antisymmetric: owns_pair(d) != owns_pair(-d) for d != 0.  The
// tolerance makes near-zero components of lattice vectors (thermal noise) defer to the next axis, so
// each fcc shell splits into two equal halves for every atom.
__device__ __forceinline__ bool owns_pair(float dx, float dy, float dz) {
  if (dz > OWN_EPS) return true;
  if (dz < -OWN_EPS) return false;
  if (dy > OWN_EPS) return true;
  if (dy < -OWN_EPS) return false;
  if (dx != 0.f) return dx > 0.f;
  if (dy != 0.f) return dy > 0.f;
  return dz > 0.f;
}

// Squared distance with an explicit operation order, so that both passes classify a pair identically.
__device__ __forceinline__ float nb_r2(float a, float b, float c) { return fmaf(a, a, fmaf(b, b, c * c)); }

// Segment of an accepted pair: owned by i (0..4) or not (5..9), by build-time distance band.
__device__ __forceinline__ int segment_of(float dx, float dy, float dz, float r2, const Bands &B) {
  const int bd = (int)(r2 >= B.b0) + (int)(r2 >= B.b1) + (int)(r2 >= B.b2) + (int)(r2 >= B.b3);   // edges below r2
  return owns_pair(dx, dy, dz) ? bd : 5 + bd;
}

// This chunk's entries of segment `lane % 5` (lanes 0..4) or `5 + lane % 5` (lanes 5..9); key NB_SEG
// marks an empty slot.  fsh = 6 (lane % 5).
__device__ __forceinline__ int segment_counts(int key, int lane, unsigned fsh) {
  const unsigned lo = key < 5 ? 1u << (6 * key) : 0u;
  const unsigned hi = key >= 5 && key < NB_SEG ? 1u << (6 * (key - 5)) : 0u;
  const unsigned slo = __reduce_add_sync(0xffffffffu, lo), shi = __reduce_add_sync(0xffffffffu, hi);
  return (int)(((lane < 5 ? slo : shi) >> fsh) & 63u);
}

// The candidate scan and segment placement of atom i by one warp (see k_neighbors).
__device__ __forceinline__ void neighbors_of_atom(int i, int n, const float4 *__restrict__ pos,
                                                  const int *__restrict__ cell_start, const Geom &geom,
                                                  const Bands &B, int limit, float4 *stage,
                                                  uint8_t *skey, int lane, int32_t *__restrict__ nbr,
                                                  int32_t *__restrict__ nnum, int32_t *__restrict__ nang,
                                                  int32_t *__restrict__ nown, int32_t *__restrict__ nband0,
                                                  int32_t *__restrict__ nfar, Control *ctrl) {
  const unsigned lower = (1u << lane) - 1u;
  const float4 pi = pos[i];
  const int cx = cell_x(pi.w), cy = cell_y(pi.w), cz = cell_z(pi.w);
  const bool xwrap = cx == 0 || cx == geom.ncx - 1;
  int acc = 0;                                         // accepted so far (warp-uniform)
  // The candidate ranges in stencil order (dz, dy, then the x part), set up one per lane L = 9 (dz + 1)
  // + 3 (dy + 1) + part: a row of three cells that does not wrap around x is one range (part 0; its
  // left or right cell left out when atom i lies farther from its own cell's face than the reach left
  // after the row's (y, z) gap: every candidate there is at least that far away in x), a row that
  // wraps is three; rows whose (y, z) slab lies beyond the list radius are empty.  The 1e-4 margin
  // keeps every candidate a float32 distance test could accept, so the lists are unchanged.
  int rb = 0, rlen = 0;
  float roy = 0.f, roz = 0.f;
  int rcode = 0;                                       // shift-table base (dy, dz) | x part << 8
  if (lane < 27) {
    const int dz = lane / 9 - 1, dy = (lane / 3) % 3 - 1, part = lane % 3;
    roz = dz < 0 ? -geom.lz : (dz > 0 ? geom.lz : 0.f);   // the shift table's offsets
    roy = dy < 0 ? -geom.ly : (dy > 0 ? geom.ly : 0.f);
    rcode = (3 * (dy + 1) + 9 * (dz + 1)) | (part << 8);
    int zz = cz + dz;
    zz += zz < 0 ? geom.ncz : (zz >= geom.ncz ? -geom.ncz : 0);
    int yy = cy + dy;
    yy += yy < 0 ? geom.ncy : (yy >= geom.ncy ? -geom.ncy : 0);
    const int row = (zz * geom.ncy + yy) * geom.ncx;
    const float gy = dy < 0 ? pi.y : (dy > 0 ? geom.ly - pi.y : 0.f);
    const float gz = dz < 0 ? pi.z : (dz > 0 ? geom.lz - pi.z : 0.f);
    const float reach2 = B.b4 * 1.0001f - (gy * gy + gz * gz);
    if (reach2 >= 0.f) {
      const bool need_l = pi.x * pi.x <= reach2, need_r = (geom.lx - pi.x) * (geom.lx - pi.x) <= reach2;
      if (!xwrap) {
        if (part == 0) {
          rb = cell_start[row + cx - (need_l ? 1 : 0)];
          rlen = cell_start[row + cx + (need_r ? 2 : 1)] - rb;
        }
      } else if (!((part == 0 && !need_l) || (part == 2 && !need_r))) {
        int xx = cx + part - 1;
        xx += xx < 0 ? geom.ncx : (xx >= geom.ncx ? -geom.ncx : 0);
        rb = cell_start[row + xx];
        rlen = cell_start[row + xx + 1] - rb;
      }
    }
  }
  // the non-empty ranges, walked in order (every lane takes part in each shuffle); each candidate is
  // tested on every lane without a branch (the load index clamped into the range), and an accepted
  // pair's displacement and entry go to the stage as one 16-byte record in candidate order
  unsigned ne = __ballot_sync(0xffffffffu, rlen > 0);
  while (ne != 0u) {
    const int L = __ffs(ne) - 1;                       // warp-uniform
    ne &= ne - 1u;
    const int b = __shfl_sync(0xffffffffu, rb, L), e = b + __shfl_sync(0xffffffffu, rlen, L);
    const float oz = __shfl_sync(0xffffffffu, roz, L), oy = __shfl_sync(0xffffffffu, roy, L);
    const int code = __shfl_sync(0xffffffffu, rcode, L);
    const int shb = code & 255, part = code >> 8;
    for (int j0 = b; j0 < e; j0 += 32) {
      const int j = j0 + lane;
      const bool inr = j < e;
      const float4 pj = pos[inr ? j : e - 1];          // j0 < e: always inside the range
      const int dx = xwrap ? part - 1 : cell_x(pj.w) - cx;
      const float ox = (float)dx * geom.lx;            // exact: dx is -1, 0 or 1
      const float ddx = pj.x - pi.x + ox, ddy = pj.y - pi.y + oy, ddz = pj.z - pi.z + oz;
      const bool ok = inr && j != i && nb_r2(ddx, ddy, ddz) < B.b4;
      const uint32_t ent = (uint32_t)j | ((uint32_t)((dx + 1) + shb) << J_BITS);
      const unsigned m = __ballot_sync(0xffffffffu, ok);
      const int slot = acc + __popc(m & lower);
      if (ok && slot < NB_STAGE) stage[slot] = make_float4(ddx, ddy, ddz, __uint_as_float(ent));
      acc += __popc(m);
    }
  }
  __syncwarp();
  // Segments of the staged entries (classified here, 32 accepted pairs at a time, rather than in the
  // sparse candidate loop; the same float32 arithmetic as the acceptance test), their sizes and offsets,
  // then placement in candidate order within each segment.  Lane g < NB_SEG keeps segment g's count
  // and running offset; a chunk of 32 staged entries is counted with two warp reductions of one-hot
  // 6-bit fields (segments 0..4 and 5..9: at most 32 per field, no carries).
  const int ms = min(acc, NB_STAGE);
  const unsigned fsh = 6u * (unsigned)(lane % 5);
  int mycnt = 0;
  for (int s0 = 0; s0 < ms; s0 += 32) {
    int key = NB_SEG;
    if (s0 + lane < ms) {
      const float4 sd = stage[s0 + lane];
      key = segment_of(sd.x, sd.y, sd.z, nb_r2(sd.x, sd.y, sd.z), B);
      skey[s0 + lane] = (uint8_t)key;
    }
    mycnt += segment_counts(key, lane, fsh);
  }
  __syncwarp();
  if (lane >= NB_SEG) mycnt = 0;
  int incl = mycnt;                                    // inclusive prefix over lanes 0..NB_SEG-1
#pragma unroll
  for (int d = 1; d < 16; d <<= 1) {
    const int t = __shfl_up_sync(0xffffffffu, incl, d);
    if (lane >= d) incl += t;
  }
  int myrun = incl - mycnt;                            // next slot of segment `lane`
  for (int s0 = 0; s0 < ms; s0 += 32) {
    const bool valid = s0 + lane < ms;
    const int key = valid ? (int)skey[s0 + lane] : NB_SEG;
    const uint32_t ent = valid ? __float_as_uint(stage[s0 + lane].w) : 0u;
    const unsigned grp = __match_any_sync(0xffffffffu, key);
    const int k = __shfl_sync(0xffffffffu, myrun, key) + __popc(grp & lower);
    if (valid && k < limit) nbr[(size_t)k * n + i] = (int32_t)ent;
    myrun += segment_counts(key, lane, fsh);
  }
  const int c0 = __shfl_sync(0xffffffffu, mycnt, 0), c1 = __shfl_sync(0xffffffffu, mycnt, 1);
  const int c4 = __shfl_sync(0xffffffffu, mycnt, 4), c5 = __shfl_sync(0xffffffffu, mycnt, 5);
  const int c6 = __shfl_sync(0xffffffffu, mycnt, 6), c9 = __shfl_sync(0xffffffffu, mycnt, 9);
  const int n_own = __shfl_sync(0xffffffffu, incl, 4);
  if (lane == 0) {
    const int kept = min(acc, limit);
    if (acc > kept || acc > NB_STAGE) atomicOr(&ctrl->status, ST_OVERFLOW);
    nnum[i] = kept;
    nown[i] = min(n_own, kept);
    nang[i] = c0 + c1 + c5 + c6;
    nband0[i] = min(c0, kept);
    // far bands (each part's last): skippable while no atom moved far enough to bring them in range;
    // zero when the row overflowed (the evaluation then reports the overflow)
    nfar[i] = acc > kept ? 0 : (c4 | (c9 << 16));
  }
}

// One warp per atom i.  The lanes test 32 candidates at a time (coalesced position loads, the atom's
// own position broadcast): for each of the 9 (dy, dz) rows of the 27-cell stencil the three cells
// x-1, x, x+1 are consecutive in the cell-sorted arrays, so the row is one contiguous range and a
// candidate's x offset comes from its packed cell coordinate (rows that wrap around the periodic x
// boundary are walked cell by cell; the bounds of all ranges are read up front, one lane each).
// Accepted entries go to a per-warp shared-memory stage in
// candidate order (ballot + popc), then are placed by segment: [owned | not owned] x band, candidate
// order inside a segment -- the same row as the thread-per-atom formulation, with 32-wide work
// instead of divergent per-thread cell loops.
__global__ void __launch_bounds__(NB_WARPS * 32, 6)   // 40 registers at most: 6 resident blocks
k_neighbors(int n, const float4 *__restrict__ pos, const int *__restrict__ cell_start, const Geom geom, int cap,
            Bands B, int32_t *__restrict__ nbr, int32_t *__restrict__ nnum, int32_t *__restrict__ nang,
            int32_t *__restrict__ nown, int32_t *__restrict__ nband0, int32_t *__restrict__ nfar, Control *ctrl) {
  if (!ctrl->do_rebuild) return;
  __shared__ float4 stage[NB_WARPS][NB_STAGE];         // staged (displacement, entry)
  __shared__ uint8_t skey[NB_WARPS][NB_STAGE];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  // The grid is capped at the resident blocks (a launch on a step without a rebuild then costs a few
  // microseconds whatever the atom count); each block takes the next group of NB_WARPS consecutive
  // atoms from a counter, which keeps the order of the hardware's own block scheduling (a static
  // stride over the atoms measured 25 % slower).
  __shared__ int group;
  for (;;) {
    if (threadIdx.x == 0) group = atomicAdd(&ctrl->nb_next, 1);
    __syncthreads();
    const int g = group;
    __syncthreads();                                   // read by every warp before the next take
    if ((long long)g * NB_WARPS >= n) break;           // block-uniform
    const int i = g * NB_WARPS + w;                    // warp-uniform
    if (i < n)
      neighbors_of_atom(i, n, pos, cell_start, geom, B, min(cap, NB_STAGE), stage[w], skey[w], lane, nbr, nnum,
                        nang, nown, nband0, nfar, ctrl);
    __syncwarp();                                      // the stage is reused by the warp's next atom
  }
}

// ---------------------------------------------------------------------------------------------------
// Host launcher for the whole rebuild chain.


static int blocks_for(long long m, int b) { return (int)((m + b - 1) / b); }

// Grid of the rebuild-chain kernels: enough blocks for m items, at most what is resident at once (the
// occupancy calculator's blocks per SM x the SM count); the kernels loop over the rest.  Every step
// launches the chain and the kernels return at once when it does not rebuild, so the grid size is
// what such a step pays for.
static int sm_count() {
  static int sms = 0;
  if (sms <= 0) {
    int d = 0;
    if (cudaGetDevice(&d) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, d) != cudaSuccess ||
        sms <= 0)
      sms = 152;
  }
  return sms;
}
template <class K>
static int resident_grid(K kernel, long long m, int per_block, int threads) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, 0) != cudaSuccess || per_sm <= 0)
    per_sm = 1;
  return (int)std::min<long long>(blocks_for(m, per_block), (long long)sm_count() * per_sm);
}

cudaError_t launch_cell_sort(const RebuildArgs &a, cudaStream_t st) {
  if (a.n <= 0) return cudaSuccess;
  k_cell_zero<<<min(blocks_for(a.ncell, 256), 4096), 256, 0, st>>>(a.ncell, a.count, a.cursor, a.ctrl);
  k_cell_assign<<<resident_grid(k_cell_assign, a.n, 256, 256), 256, 0, st>>>(a.n, a.x, a.y, a.z, a.L[0], a.L[1], a.L[2], a.l[0], a.l[1],
                                                      a.l[2], a.nc[0], a.nc[1], a.nc[2], a.cell_of, a.count, a.ctrl);
  const int ntiles = blocks_for(a.ncell, SCAN_TILE);
  k_scan_tiles<<<ntiles, SCAN_THREADS, 0, st>>>(a.ncell, a.count, a.start, a.tile_sums, a.ctrl);
  k_scan_carry<<<1, 32, 0, st>>>(ntiles, a.tile_sums, a.ncell, a.start, a.ctrl);
  k_scan_add<<<resident_grid(k_scan_add, a.ncell, 256, 256), 256, 0, st>>>(a.ncell, a.start, a.tile_sums, a.ctrl);
  k_scatter<<<resident_grid(k_scatter, a.n, 256, 256), 256, 0, st>>>(a.n, a.cell_of, a.start, a.cursor, a.perm, a.ctrl);
  k_cell_sort<<<resident_grid(k_cell_sort, a.ncell, 128, 128), 128, 0, st>>>(a.ncell, a.start, a.perm, a.id, a.ctrl);
  k_permute<<<resident_grid(k_permute, a.n, 256, 256), 256, 0, st>>>(a.n, a.perm, a.x, a.y, a.z, a.vx, a.vy, a.vz, a.id, a.cell_of, a.xb,
                                                  a.yb, a.zb, a.vxb, a.vyb, a.vzb, a.idb, a.pos, a.pos_ref, a.l[0],
                                                  a.l[1], a.l[2], a.nc[0], a.nc[1], a.ctrl);
  k_copy_back<<<resident_grid(k_copy_back, a.n, 256, 256), 256, 0, st>>>(a.n, a.x, a.y, a.z, a.vx, a.vy, a.vz, a.id, a.xb, a.yb, a.zb,
                                                    a.vxb, a.vyb, a.vzb, a.idb, a.ctrl);
  return cudaGetLastError();
}

cudaError_t launch_neighbors(const RebuildArgs &a, cudaStream_t st) {
  if (a.n <= 0) return cudaSuccess;
  Geom g;
  g.lx = (float)a.l[0]; g.ly = (float)a.l[1]; g.lz = (float)a.l[2];
  g.ncx = a.nc[0]; g.ncy = a.nc[1]; g.ncz = a.nc[2];
  Bands B;
  B.b0 = a.ba2; B.b1 = a.ra2; B.b2 = a.br2; B.b3 = std::min(a.fs2, a.rl2); B.b4 = a.rl2;
  k_neighbors<<<resident_grid(k_neighbors, a.n, NB_WARPS, NB_WARPS * 32), NB_WARPS * 32, 0, st>>>(
      a.n, a.pos, a.start, g, a.cap, B, a.nbr, a.nnum, a.nang, a.nown, a.nband0, a.nfar, a.ctrl);
  return cudaGetLastError();
}

int scan_tiles(int ncell) { return blocks_for(ncell, SCAN_TILE); }

}  // namespace nep
