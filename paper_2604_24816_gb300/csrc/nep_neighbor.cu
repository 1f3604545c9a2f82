// nep_neighbor.cu -- cell binning, cell sort and distance-sorted neighbour lists on sm_103a.
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
//   k_neighbors     for each atom (one warp per atom), every j with |r_ij| < rc_R + skin among the 27
//                   neighbouring cell images, sorted by (float32 distance^2, packed j) so that the
//                   entries inside the angular and radial cutoffs come first and the per-pair branches
//                   in the force kernels stay warp-uniform; the prefix with |r_ij| < rc_A + skin is
//                   the angular list.
// Distances use cell-relative float32 coordinates plus the image offset of the neighbouring cell, so
// their error does not grow with the box size (float64 appears only in the wrap and cell assignment).
#include "nep_common.cuh"

namespace nep {

constexpr int SCAN_THREADS = 1024;
constexpr int SCAN_ITEMS = 4;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

__global__ void k_cell_zero(int ncell, int *__restrict__ count, int *__restrict__ cursor, const Control *ctrl) {
  if (!ctrl->do_rebuild) return;
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
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
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
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx < m) out[idx] += tile_sums[idx / SCAN_TILE];
}

__global__ void k_scatter(int n, const int *__restrict__ cell_of, const int *__restrict__ start, int *__restrict__ cursor,
                          int *__restrict__ perm, const Control *ctrl) {
  if (!ctrl->do_rebuild) return;
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  const int c = cell_of[s];
  perm[start[c] + atomicAdd(cursor + c, 1)] = s;
}

// One thread per cell: insertion sort of the cell's slots by original id (ids are unique).
__global__ void k_cell_sort(int ncell, const int *__restrict__ start, int *__restrict__ perm, const int *__restrict__ id,
                            const Control *ctrl) {
  if (!ctrl->do_rebuild) return;
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= ncell) return;
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

__global__ void k_permute(int n, const int *__restrict__ perm, const double *__restrict__ x, const double *__restrict__ y,
                          const double *__restrict__ z, const double *__restrict__ vx, const double *__restrict__ vy,
                          const double *__restrict__ vz, const int *__restrict__ id, const int *__restrict__ cell_of,
                          double *__restrict__ xb, double *__restrict__ yb, double *__restrict__ zb,
                          double *__restrict__ vxb, double *__restrict__ vyb, double *__restrict__ vzb,
                          int *__restrict__ idb, float4 *__restrict__ pos, float4 *__restrict__ pos_ref, double lx,
                          double ly, double lz, int ncx, int ncy, const Control *ctrl) {
  if (!ctrl->do_rebuild) return;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const int s = perm[t];
  const double px = x[s], py = y[s], pz = z[s];
  xb[t] = px; yb[t] = py; zb[t] = pz;
  vxb[t] = vx[s]; vyb[t] = vy[s]; vzb[t] = vz[s];
  idb[t] = id[s];
  const int c = cell_of[s];
  const int cx = c % ncx, cy = (c / ncx) % ncy, cz = c / (ncx * ncy);
  const float4 p = make_float4((float)(px - cx * lx), (float)(py - cy * ly), (float)(pz - cz * lz),
                               __int_as_float(cx | (cy << 10) | (cz << 20)));
  pos[t] = p;
  pos_ref[t] = p;
}

__global__ void k_copy_back(int n, double *__restrict__ x, double *__restrict__ y, double *__restrict__ z,
                            double *__restrict__ vx, double *__restrict__ vy, double *__restrict__ vz,
                            int *__restrict__ id, const double *__restrict__ xb, const double *__restrict__ yb,
                            const double *__restrict__ zb, const double *__restrict__ vxb,
                            const double *__restrict__ vyb, const double *__restrict__ vzb,
                            const int *__restrict__ idb, const Control *ctrl) {
  if (!ctrl->do_rebuild) return;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  x[t] = xb[t]; y[t] = yb[t]; z[t] = zb[t];
  vx[t] = vxb[t]; vy[t] = vyb[t]; vz[t] = vzb[t];
  id[t] = idb[t];
}

// One warp per atom, 32 consecutive atoms (a tile) per warp.  Lanes test the candidates of each of the
// 27 neighbouring cell images in parallel; accepted entries are compacted with a ballot into a
// per-warp key buffer (key = float32 distance^2 bits << 32 | packed entry), bitonic-sorted in shared
// memory, and staged in a [32][CAP+1] tile so the list is written row-coalesced ([cap][N] layout).
template <int CAP>
__global__ void __launch_bounds__(32)
k_neighbors(int n, const float4 *__restrict__ pos, const int *__restrict__ cell_start, const Geom geom, int cap,
            float rl2, float ra2, int32_t *__restrict__ nbr, int32_t *__restrict__ nnum, int32_t *__restrict__ nang,
            Control *ctrl) {
  if (!ctrl->do_rebuild) return;
  __shared__ float4 shift[27];
  __shared__ unsigned long long keys[CAP];
  __shared__ uint32_t tile[32][CAP + 1];
  __shared__ int tile_cnt[32];
  fill_shift_table(shift, geom);
  __syncwarp();
  const int lane = threadIdx.x;
  const unsigned lt_mask = (1u << lane) - 1u;
  const int base = blockIdx.x * 32;
  const int limit = min(cap, CAP);
  for (int t = 0; t < 32; ++t) {
    const int i = base + t;
    if (i >= n) {
      if (lane == 0) tile_cnt[t] = 0;
      continue;
    }
    const float4 pi = pos[i];
    const int cx = cell_x(pi.w), cy = cell_y(pi.w), cz = cell_z(pi.w);
    int cnt = 0;
    for (int dz = -1; dz <= 1; ++dz) {
      const int zz = (cz + dz + geom.ncz) % geom.ncz;
      for (int dy = -1; dy <= 1; ++dy) {
        const int yy = (cy + dy + geom.ncy) % geom.ncy;
        for (int dx = -1; dx <= 1; ++dx) {
          const int xx = (cx + dx + geom.ncx) % geom.ncx;
          const int sh = (dx + 1) + 3 * (dy + 1) + 9 * (dz + 1);
          const float4 o = shift[sh];
          const int c = (zz * geom.ncy + yy) * geom.ncx + xx;
          const int b = cell_start[c], e = cell_start[c + 1];
          for (int j0 = b; j0 < e; j0 += 32) {
            const int j = j0 + lane;
            bool ok = false;
            unsigned long long key = 0ull;
            if (j < e && !(j == i && sh == 13)) {
              const float4 pj = pos[j];
              const float ddx = pj.x - pi.x + o.x, ddy = pj.y - pi.y + o.y, ddz = pj.z - pi.z + o.z;
              const float r2 = ddx * ddx + ddy * ddy + ddz * ddz;
              ok = r2 < rl2;
              key = ((unsigned long long)__float_as_uint(r2) << 32) | (unsigned long long)((uint32_t)j | ((uint32_t)sh << J_BITS));
            }
            const unsigned m = __ballot_sync(0xffffffffu, ok);
            if (ok) {
              const int slot = cnt + __popc(m & lt_mask);
              if (slot < CAP) keys[slot] = key;
            }
            cnt += __popc(m);
          }
        }
      }
    }
    const int kept = min(cnt, limit);
    if (lane == 0 && cnt > kept) atomicOr(&ctrl->status, ST_OVERFLOW);
    for (int s = min(cnt, CAP) + lane; s < CAP; s += 32) keys[s] = ~0ull;
    __syncwarp();
    // bitonic sort of keys[0..CAP) ascending
    for (int size = 2; size <= CAP; size <<= 1) {
      for (int stride = size >> 1; stride > 0; stride >>= 1) {
        for (int p = lane; p < CAP / 2; p += 32) {
          const int lo = 2 * p - (p & (stride - 1));
          const int hi = lo + stride;
          const unsigned long long a = keys[lo], bb = keys[hi];
          const bool up = (lo & size) == 0;
          if ((a > bb) == up) { keys[lo] = bb; keys[hi] = a; }
        }
        __syncwarp();
      }
    }
    int na = 0;
    for (int k = lane; k < kept; k += 32) {
      const unsigned long long key = keys[k];
      tile[t][k] = (uint32_t)(key & 0xffffffffull);
      na += __uint_as_float((uint32_t)(key >> 32)) < ra2 ? 1 : 0;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) na += __shfl_xor_sync(0xffffffffu, na, o);
    if (lane == 0) {
      tile_cnt[t] = kept;
      nnum[i] = kept;
      nang[i] = na;
    }
    __syncwarp();
  }
  // flush: row k of the tile is 32 consecutive atoms -> one coalesced 128-byte store
  const int i = base + lane;
  const int mine = tile_cnt[lane];
  int kmax = mine;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) kmax = max(kmax, __shfl_xor_sync(0xffffffffu, kmax, o));
  for (int k = 0; k < kmax; ++k)
    if (k < mine && i < n) nbr[(size_t)k * n + i] = (int32_t)tile[lane][k];
}

// ---------------------------------------------------------------------------------------------------
// Host launcher for the whole rebuild chain.


static int blocks_for(long long m, int b) { return (int)((m + b - 1) / b); }

cudaError_t launch_cell_sort(const RebuildArgs &a, cudaStream_t st) {
  if (a.n <= 0) return cudaSuccess;
  k_cell_zero<<<min(blocks_for(a.ncell, 256), 4096), 256, 0, st>>>(a.ncell, a.count, a.cursor, a.ctrl);
  k_cell_assign<<<blocks_for(a.n, 256), 256, 0, st>>>(a.n, a.x, a.y, a.z, a.L[0], a.L[1], a.L[2], a.l[0], a.l[1],
                                                      a.l[2], a.nc[0], a.nc[1], a.nc[2], a.cell_of, a.count, a.ctrl);
  const int ntiles = blocks_for(a.ncell, SCAN_TILE);
  k_scan_tiles<<<ntiles, SCAN_THREADS, 0, st>>>(a.ncell, a.count, a.start, a.tile_sums, a.ctrl);
  k_scan_carry<<<1, 32, 0, st>>>(ntiles, a.tile_sums, a.ncell, a.start, a.ctrl);
  k_scan_add<<<blocks_for(a.ncell, 256), 256, 0, st>>>(a.ncell, a.start, a.tile_sums, a.ctrl);
  k_scatter<<<blocks_for(a.n, 256), 256, 0, st>>>(a.n, a.cell_of, a.start, a.cursor, a.perm, a.ctrl);
  k_cell_sort<<<blocks_for(a.ncell, 128), 128, 0, st>>>(a.ncell, a.start, a.perm, a.id, a.ctrl);
  k_permute<<<blocks_for(a.n, 256), 256, 0, st>>>(a.n, a.perm, a.x, a.y, a.z, a.vx, a.vy, a.vz, a.id, a.cell_of, a.xb,
                                                  a.yb, a.zb, a.vxb, a.vyb, a.vzb, a.idb, a.pos, a.pos_ref, a.l[0],
                                                  a.l[1], a.l[2], a.nc[0], a.nc[1], a.ctrl);
  k_copy_back<<<blocks_for(a.n, 256), 256, 0, st>>>(a.n, a.x, a.y, a.z, a.vx, a.vy, a.vz, a.id, a.xb, a.yb, a.zb,
                                                    a.vxb, a.vyb, a.vzb, a.idb, a.ctrl);
  return cudaGetLastError();
}

cudaError_t launch_neighbors(const RebuildArgs &a, cudaStream_t st) {
  if (a.n <= 0) return cudaSuccess;
  Geom g;
  g.lx = (float)a.l[0]; g.ly = (float)a.l[1]; g.lz = (float)a.l[2];
  g.ncx = a.nc[0]; g.ncy = a.nc[1]; g.ncz = a.nc[2];
  const int grid = blocks_for(a.n, 32);
  if (a.cap <= 128)
    k_neighbors<128><<<grid, 32, 0, st>>>(a.n, a.pos, a.start, g, a.cap, a.rl2, a.ra2, a.nbr, a.nnum, a.nang, a.ctrl);
  else
    k_neighbors<256><<<grid, 32, 0, st>>>(a.n, a.pos, a.start, g, a.cap, a.rl2, a.ra2, a.nbr, a.nnum, a.nang, a.ctrl);
  return cudaGetLastError();
}

int scan_tiles(int ncell) { return blocks_for(ncell, SCAN_TILE); }

}  // namespace nep
