// nep_noalloc.cu -- one force evaluation that allocates no memory (nep_compute_noalloc).
//
// Some callers cannot allocate GPU memory at the point where they need forces: a plugin running
// inside another program's memory pool or allocator budget, or an embedded runtime that forbids
// cudaMalloc after start-up.  For them this entry point evaluates E, F and the virial of a small system
// of the float32 teacher shape with the separate descriptor and full-row force kernels, but every
// intermediate buffer (cell lists, neighbour lists, adjoint rows, partial sums, status word) lives in
// one file-scope __device__ array of fixed size, created when the library is loaded and kept by every
// GPU that loads it until the process exits.
//
// The device address of that array is looked up once per device with cudaGetSymbolAddress (in host
// code the symbol name is only a host-side stand-in, never a device address), in the first call on
// each device.  The call waits for its work by polling the stream and reads results with synchronous
// copies, so it is not for use while a stream is being captured.  All calls share the array and it
// keeps the previous call's contents: every piece that must start from zero is cleared by the call
// itself, and calls that overlap on the GPU (on different streams, or from different threads) race on
// the array -- serialize them.  A call whose wait timed out leaves its work running on the array; the
// next call refuses to start (NEP_ERR_STATE) until that stream is idle.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <mutex>
#include <thread>

#include "nep_common.cuh"
#include "nep_descriptor.cuh"
#include "nep_gb300.h"

namespace nep {
template <class S>
cudaError_t launch_descriptor(const Model<S> &, const Geom &, int, const float4 *, const int32_t *, const RowExt &,
                              float *, float *, float *, long long *, long long *, int *, const Fallback &,
                              cudaStream_t);
template <class S, class GT>
cudaError_t launch_force(const Model<S> &, const Geom &, int, const float4 *, const int32_t *, const RowExt &,
                         const GT *, long long *, long long *, int *, cudaStream_t);
int descriptor_blocks(int n);
int force_blocks(int n);
cudaError_t launch_cell_sort(const RebuildArgs &, cudaStream_t);
cudaError_t launch_neighbors(const RebuildArgs &, cudaStream_t);
int scan_tiles(int ncell);
cudaError_t launch_control(Control *, bool, cudaStream_t);
cudaError_t launch_finalize(const long long *, int, const long long *, int, const long long *, int, double *,
                            long long *, cudaStream_t);
cudaError_t launch_load_state(int, const double *, const double *, double *, double *, double *, double *, double *,
                              double *, int *, int *, cudaStream_t);
cudaError_t launch_store_force(int, const int *, const long long *, double *, cudaStream_t);
}  // namespace nep

using namespace nep;

namespace {

using S = CuShape;
constexpr int NA_MAX = NEP_NOALLOC_MAX_ATOMS;
constexpr int NC_MAX = NEP_NOALLOC_MAX_CELLS;
constexpr int CAP = 128;

constexpr size_t up256(size_t b) { return (b + 255) / 256 * 256; }

// Byte offsets of the pieces inside the scratch array.
struct Layout {
  size_t x, y, z, vx, vy, vz, xb, yb, zb, vxb, vyb, vzb, id, idb, cell_of, perm, pos, pos_ref, F, usite, G, nbr,
      nnum, nang, nown, nband0, nfar, count, cursor, start, tile_sums, part_d, part_f, sums, counters, ctrl, io, total;
};

constexpr Layout make_layout() {
  Layout L{};
  size_t o = 0;
  auto take = [&o](size_t bytes) { const size_t at = o; o += up256(bytes); return at; };
  const size_t N = NA_MAX;
  L.x = take(N * 8); L.y = take(N * 8); L.z = take(N * 8);
  L.vx = take(N * 8); L.vy = take(N * 8); L.vz = take(N * 8);
  L.xb = take(N * 8); L.yb = take(N * 8); L.zb = take(N * 8);
  L.vxb = take(N * 8); L.vyb = take(N * 8); L.vzb = take(N * 8);
  L.id = take(N * 4); L.idb = take(N * 4); L.cell_of = take(N * 4); L.perm = take(N * 4);
  L.pos = take(N * 16); L.pos_ref = take(N * 16);
  L.F = take(N * 3 * 8); L.usite = take(N * 4); L.G = take(N * S::GS * 4); L.nbr = take(N * CAP * 4);
  L.nnum = take(N * 4); L.nang = take(N * 4); L.nown = take(N * 4); L.nband0 = take(N * 4); L.nfar = take(N * 4);
  L.count = take((size_t)NC_MAX * 4); L.cursor = take((size_t)NC_MAX * 4); L.start = take(((size_t)NC_MAX + 1) * 4);
  L.tile_sums = take(((size_t)NC_MAX / 4096 + 2) * 4);
  L.part_d = take(((size_t)N / 64 + 2) * 5 * 8); L.part_f = take(((size_t)N / 64 + 2) * 13 * 8);
  L.sums = take(32 * 8); L.counters = take(16 * 8); L.ctrl = take(sizeof(Control)); L.io = take(N * 3 * 8);
  L.total = o;
  return L;
}

constexpr Layout LAYOUT = make_layout();

// The scratch memory of nep_compute_noalloc (about 11 MB for 8,192 atoms).
static __device__ __align__(256) unsigned char g_noalloc_scratch[LAYOUT.total];

constexpr int MAX_DEVICES = 64;
constexpr double WAIT_LIMIT_S = 900.0;
std::mutex g_mutex;
unsigned char *g_scratch_addr[MAX_DEVICES] = {nullptr};
// stream of a call whose wait timed out, per device (its work may still use the array)
cudaStream_t g_busy_stream[MAX_DEVICES] = {nullptr};
bool g_busy[MAX_DEVICES] = {false};

// NEP_OK when no timed-out call's work is still running on this device's array.
nep_status previous_call_done() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) return NEP_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_busy[dev]) return NEP_OK;
  const cudaError_t e = cudaStreamQuery(g_busy_stream[dev]);
  if (e == cudaErrorNotReady) return NEP_ERR_STATE;
  if (e != cudaSuccess) cudaGetLastError();
  g_busy[dev] = false;
  return NEP_OK;
}

void mark_busy(cudaStream_t st) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) return;
  std::lock_guard<std::mutex> lock(g_mutex);
  g_busy[dev] = true;
  g_busy_stream[dev] = st;
}

// Device address of the scratch array on the current device (looked up once per device).
cudaError_t scratch_address(unsigned char **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= MAX_DEVICES) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mutex);
  if (g_scratch_addr[dev] == nullptr) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[dev] = static_cast<unsigned char *>(p);
  }
  *out = g_scratch_addr[dev];
  return cudaSuccess;
}

bool device_pointer(const void *p) {
  if (p == nullptr) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Bounded wait on the stream (no event objects are created).
nep_status wait_bounded(cudaStream_t st) {
  const auto t0 = std::chrono::steady_clock::now();
  for (int spins = 0;; ++spins) {
    const cudaError_t e = cudaStreamQuery(st);
    if (e == cudaSuccess) return NEP_OK;
    if (e != cudaErrorNotReady) return NEP_ERR_CUDA;
    const double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (el > WAIT_LIMIT_S) return NEP_ERR_TIMEOUT;
    if (spins > 64) {                       // yield for the first 2 ms, then sleep between polls
      if (el < 2e-3) std::this_thread::yield();
      else std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
  }
}

}  // namespace

#define NA_CUDA(call)                                 \
  do {                                                \
    if ((call) != cudaSuccess) return NEP_ERR_CUDA;   \
  } while (0)

extern "C" nep_status nep_compute_noalloc(const nep_params *p, int64_t n, const double *x, const double *box,
                                          double *E, double *F, double *virial, void *cuda_stream) {
  if (!p || !box) return NEP_ERR_ARG;
  if (p->n_max_R + 1 != S::NR || p->n_max_A + 1 != S::NA || p->basis_R != S::KR || p->basis_A != S::KA ||
      p->l_max_3b != S::LMAX || p->l_max_4b != (S::FOURBODY ? 2 : 0) || p->n_neu != S::NNEU || p->precision != NEP_FP32)
    return NEP_ERR_UNSUPPORTED;
  if (!p->c_R || !p->c_A || !p->W0 || !p->b0 || !p->w1 || !p->q_scale) return NEP_ERR_ARG;
  if (!(p->rc_R > 0.f) || !(p->rc_A > 0.f) || p->rc_A > p->rc_R || !(p->skin >= 0.f)) return NEP_ERR_ARG;
  if (p->lj_eps != 0.f && (!(p->lj_rc > 0.f) || p->lj_rc > p->rc_R || !(p->lj_sigma > 0.f))) return NEP_ERR_ARG;
  if (n < 0 || n > NEP_NOALLOC_MAX_ATOMS) return NEP_ERR_ARG;       // beyond the fixed scratch size
  if (n > 0 && !x) return NEP_ERR_ARG;
  const double rl = (double)p->rc_R + (double)p->skin;
  double l[3];
  int nc[3];
  long long ncell = 1;
  for (int d = 0; d < 3; ++d) {
    if (!(box[d] > 0.0) || !std::isfinite(box[d])) return NEP_ERR_ARG;
    if (box[d] < 2.0 * rl) return NEP_ERR_BOX_TOO_SMALL;
    nc[d] = std::max(2, std::min((int)std::floor(box[d] / rl), 1023));
    l[d] = box[d] / nc[d];
    ncell *= nc[d];
  }
  if (ncell > NEP_NOALLOC_MAX_CELLS) return NEP_ERR_ARG;              // beyond the fixed scratch size
  if (n == 0) {
    if (E) { const double z = 0.0; NA_CUDA(cudaMemcpy(E, &z, sizeof(double), cudaMemcpyDefault)); }
    if (virial) { const double z[9] = {0}; NA_CUDA(cudaMemcpy(virial, z, sizeof(z), cudaMemcpyDefault)); }
    return NEP_OK;
  }

  // Model parameters (kernel argument, no device memory).
  Model<S> M{};
  for (int a = 0; a < S::NR; ++a)
    for (int b = 0; b < S::KR; ++b) M.cR[a][b] = p->c_R[a * S::KR + b];
  for (int a = 0; a < S::NA; ++a)
    for (int b = 0; b < S::KA; ++b) M.cA[a][b] = p->c_A[a * S::KA + b];
  for (int m = 0; m < S::NNEU; ++m) {
    for (int v = 0; v < S::NDES; ++v) M.W0[m][v] = p->W0[m * S::NDES + v];
    M.b0[m] = p->b0[m];
    M.w1[m] = p->w1[m];
  }
  for (int v = 0; v < S::NDES; ++v) M.qs[v] = p->q_scale[v];
  M.b1 = p->b1;
  M.rcR = p->rc_R; M.rcA = p->rc_A; M.rcR2 = p->rc_R * p->rc_R; M.rcA2 = p->rc_A * p->rc_A;
  M.inv_rcR = 1.f / p->rc_R; M.inv_rcA = 1.f / p->rc_A;
  const double eps = p->lj_eps, sig = p->lj_sigma, rc = p->lj_rc;
  M.lj_on = eps != 0.0 ? 1.f : 0.f;
  if (eps != 0.0) {
    const double s6 = std::pow(sig, 6.0), sr6 = std::pow(sig / rc, 6.0);
    M.lj_c12 = (float)(4.0 * eps * s6 * s6);
    M.lj_c6 = (float)(4.0 * eps * s6);
    M.lj_e_rc = (float)(4.0 * eps * (sr6 * sr6 - sr6));
    M.lj_de_rc = (float)(4.0 * eps * (-12.0 * sr6 * sr6 + 6.0 * sr6) / rc);
    M.lj_e0 = (float)(4.0 * eps * ((-12.0 * sr6 * sr6 + 6.0 * sr6) - (sr6 * sr6 - sr6)));   // rc E'(rc) - E(rc)
    M.lj_m12 = (float)(-12.0 * 4.0 * eps * s6 * s6);
    M.lj_p6 = (float)(6.0 * 4.0 * eps * s6);
    M.lj_rc = (float)rc;
    M.lj_rc2 = (float)(rc * rc);
  }
  const float rmax = std::max(p->rc_R, eps != 0.0 ? p->lj_rc : 0.f);
  M.rmax2 = rmax * rmax;

  const nep_status prev = previous_call_done();
  if (prev != NEP_OK) return prev;
  unsigned char *base = nullptr;
  NA_CUDA(scratch_address(&base));
  auto at = [base](size_t off) { return static_cast<void *>(base + off); };
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  const int N = (int)n;

  RebuildArgs a{};
  a.n = N;
  a.ncell = (int)ncell;
  for (int d = 0; d < 3; ++d) { a.L[d] = box[d]; a.l[d] = l[d]; a.nc[d] = nc[d]; }
  a.x = (double *)at(LAYOUT.x); a.y = (double *)at(LAYOUT.y); a.z = (double *)at(LAYOUT.z);
  a.vx = (double *)at(LAYOUT.vx); a.vy = (double *)at(LAYOUT.vy); a.vz = (double *)at(LAYOUT.vz);
  a.xb = (double *)at(LAYOUT.xb); a.yb = (double *)at(LAYOUT.yb); a.zb = (double *)at(LAYOUT.zb);
  a.vxb = (double *)at(LAYOUT.vxb); a.vyb = (double *)at(LAYOUT.vyb); a.vzb = (double *)at(LAYOUT.vzb);
  a.id = (int *)at(LAYOUT.id); a.idb = (int *)at(LAYOUT.idb); a.cell_of = (int *)at(LAYOUT.cell_of);
  a.count = (int *)at(LAYOUT.count); a.cursor = (int *)at(LAYOUT.cursor); a.start = (int *)at(LAYOUT.start);
  a.tile_sums = (int *)at(LAYOUT.tile_sums); a.perm = (int *)at(LAYOUT.perm);
  a.pos = (float4 *)at(LAYOUT.pos); a.pos_ref = (float4 *)at(LAYOUT.pos_ref);
  a.nbr = (int32_t *)at(LAYOUT.nbr); a.nnum = (int32_t *)at(LAYOUT.nnum); a.nang = (int32_t *)at(LAYOUT.nang);
  a.nown = (int32_t *)at(LAYOUT.nown); a.nband0 = (int32_t *)at(LAYOUT.nband0); a.nfar = (int32_t *)at(LAYOUT.nfar);
  a.cap = CAP;
  const float rlf = p->rc_R + p->skin, raf = p->rc_A + p->skin, fsf = p->rc_R + FAR_EDGE * p->skin;
  a.rl2 = rlf * rlf; a.ra2 = raf * raf; a.ba2 = p->rc_A * p->rc_A; a.br2 = p->rc_R * p->rc_R; a.fs2 = fsf * fsf;
  Control *ctrl = (Control *)at(LAYOUT.ctrl);
  a.ctrl = ctrl;
  long long *Ffix = (long long *)at(LAYOUT.F);
  long long *pd = (long long *)at(LAYOUT.part_d), *pf = (long long *)at(LAYOUT.part_f);
  double *sums = (double *)at(LAYOUT.sums);
  long long *counters = (long long *)at(LAYOUT.counters);
  double *io = (double *)at(LAYOUT.io);
  Geom g;
  g.lx = (float)l[0]; g.ly = (float)l[1]; g.lz = (float)l[2];
  g.ncx = nc[0]; g.ncy = nc[1]; g.ncz = nc[2];

  // The array keeps the previous call's contents: clear the status word, control block and counters
  // (cell counters, force accumulators and partial sums are cleared or overwritten by the kernels).
  NA_CUDA(cudaMemsetAsync(ctrl, 0, sizeof(Control), st));
  NA_CUDA(cudaMemsetAsync(counters, 0, 16 * sizeof(long long), st));
  const double *xin = x;
  if (!device_pointer(x)) {
    NA_CUDA(cudaMemcpyAsync(io, x, 3 * (size_t)N * sizeof(double), cudaMemcpyHostToDevice, st));
    xin = io;
  }
  NA_CUDA(launch_load_state(N, xin, nullptr, a.x, a.y, a.z, a.vx, a.vy, a.vz, a.id, &ctrl->status, st));
  NA_CUDA(launch_control(ctrl, true, st));
  NA_CUDA(launch_cell_sort(a, st));
  NA_CUDA(launch_neighbors(a, st));
  const RowExt rows{a.nnum, a.nown, a.nband0, a.nfar, nullptr};   // one evaluation: the whole rows
  NA_CUDA(launch_descriptor<S>(M, g, N, a.pos, a.nbr, rows, (float *)at(LAYOUT.G), (float *)at(LAYOUT.usite),
                               nullptr, Ffix, pd, &ctrl->status, Fallback{}, st));
  NA_CUDA((launch_force<S, float>(M, g, N, a.pos, a.nbr, rows, (const float *)at(LAYOUT.G), Ffix, pf, &ctrl->status,
                                  st)));
  NA_CUDA(launch_finalize(pd, descriptor_blocks(N), pf, force_blocks(N), nullptr, 0, sums, counters, st));
  const bool f_dev = F && device_pointer(F);
  const bool e_dev = E && device_pointer(E);
  const bool w_dev = virial && device_pointer(virial);
  if (F) NA_CUDA(launch_store_force(N, a.id, Ffix, f_dev ? F : io, st));
  if (e_dev) NA_CUDA(cudaMemcpyAsync(E, sums, sizeof(double), cudaMemcpyDeviceToDevice, st));
  if (w_dev) NA_CUDA(cudaMemcpyAsync(virial, sums + 1, 9 * sizeof(double), cudaMemcpyDeviceToDevice, st));
  // Wait (bounded) for the work, then copy host-side results from the now idle scratch array.
  const nep_status w = wait_bounded(st);
  if (w == NEP_ERR_TIMEOUT) mark_busy(st);
  if (w != NEP_OK) return w;
  int status = 0;
  NA_CUDA(cudaMemcpy(&status, &ctrl->status, sizeof(int), cudaMemcpyDeviceToHost));
  if (F && !f_dev) NA_CUDA(cudaMemcpy(F, io, 3 * (size_t)N * sizeof(double), cudaMemcpyDeviceToHost));
  if (E && !e_dev) NA_CUDA(cudaMemcpy(E, sums, sizeof(double), cudaMemcpyDeviceToHost));
  if (virial && !w_dev) NA_CUDA(cudaMemcpy(virial, sums + 1, 9 * sizeof(double), cudaMemcpyDeviceToHost));
  if (status & ST_OVERFLOW) return NEP_ERR_NEIGH_OVERFLOW;
  if (status & ST_NAN) return NEP_ERR_NAN;
  return NEP_OK;
}
