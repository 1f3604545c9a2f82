// nep_api.cu -- the C ABI declared in include/nep_gb300.h: handle, device buffers, step sequencing.
//
// One MD step enqueues: kick+drift -> step control -> rebuild chain (kernels return at once unless
// the control kernel asked for a rebuild) -> descriptors+network -> forces -> kick -> reductions.
// Because the rebuild decision is taken on the device, a step has a fixed launch sequence: it is
// captured once as a CUDA graph and replayed, with no host synchronisation inside an md_verlet_step
// call.  With timing enabled the same sequence is launched eagerly with CUDA events around each
// kernel class.  The only host waits are bounded polls of a stream event (NEP_ERR_TIMEOUT).
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <thread>
#include <type_traits>
#include <vector>

#include "nep_gb300.h"
#include "nep_common.cuh"
#include "nep_descriptor.cuh"
#include "nep_tc.cuh"

namespace nep {
// nep_force.cu
template <class S>
cudaError_t launch_descriptor(const Model<S> &, const Geom &, int, const float4 *, const int32_t *, const RowExt &,
                              float *, float *, float *, long long *, long long *, int *, const Fallback &,
                              cudaStream_t);
template <class S, class GT>
cudaError_t launch_force(const Model<S> &, const Geom &, int, const float4 *, const int32_t *, const RowExt &,
                         const GT *, long long *, long long *, int *, cudaStream_t);
template <class S>
cudaError_t launch_fused(const Model<S> &, const Geom &, int, const float4 *, const int32_t *, const RowExt &, float *,
                         float *, long long *, long long *, long long *, int *, const PairCache &, cudaStream_t);
template <class S, class MT>
cudaError_t launch_fused_mixed(const Model<S> &, const Geom &, int, const float4 *, const int32_t *, const RowExt &,
                               float *, float *, long long *, long long *, long long *, int *, const PairCache &,
                               cudaStream_t);
template <class S>
cudaError_t launch_fused_reg(const Model<S> &, const Geom &, int, const float4 *, const int32_t *, const RowExt &,
                             float *, float *, long long *, long long *, long long *, int *, const Fallback &,
                             const PairCache &, cudaStream_t);
cudaError_t pair_cache_sm_bound(int *nsm);
size_t pair_cache_region_elems(int pmax);
#ifndef NEP_FUSED
#define NEP_FUSED 1
#endif
int descriptor_blocks(int n);
int force_blocks(int n);
// nep_mixed.cu
template <class S, class MT>
cudaError_t launch_descriptor_mixed(const Model<S> &, const Geom &, int, const float4 *, const int32_t *,
                                    const RowExt &, __half *, float *, float *, long long *, long long *, int *,
                                    const Fallback &, cudaStream_t);
int mixed_descriptor_blocks(int n);
template <class S>
cudaError_t launch_fallback_descriptor(const Model<S> &, const Geom &, int, const float4 *, const int32_t *,
                                       const int32_t *, const int *, const int *, int, float *, float *, long long *,
                                       long long *, int *, cudaStream_t);
template <class S>
cudaError_t launch_fallback_force(const Model<S> &, const Geom &, int, const float4 *, const int32_t *,
                                  const int32_t *, const int *, const int *, int, const float *, long long *,
                                  long long *, int *, cudaStream_t);
cudaError_t launch_fallback_flags(const int *, const int *, int, const int *, int *, cudaStream_t);
// nep_force.cu / nep_ablation.cu: kernel variants for ablation
template <class S>
cudaError_t launch_force_float_scatter(const Model<S> &, const Geom &, int, const float4 *, const int32_t *,
                                       const RowExt &, const float *, float *, long long *, int *, cudaStream_t);
template <class S>
cudaError_t launch_force_half_list(const Model<S> &, const Geom &, int, const float4 *, const int32_t *,
                                   const RowExt &, const float *, long long *, long long *, int *, cudaStream_t);
template <class S, int NT>
cudaError_t launch_descriptor_tiled(const Model<S> &, const Geom &, int, const float4 *, const int32_t *,
                                    const RowExt &, float *, float *, long long *, long long *, int *, float *,
                                    cudaStream_t);
cudaError_t launch_store_float3(int, const int *, const float *, double *, cudaStream_t);
template <class S>
cudaError_t launch_force_cpb(int, const Model<S> &, const Geom &, int, const float4 *, const int32_t *, const RowExt &,
                             const float *, long long *, long long *, int *, cudaStream_t);
cudaError_t launch_angular_counts(int, const float4 *, const int32_t *, const RowExt &, const Geom &, float, int *,
                                  cudaStream_t);
// nep_neighbor.cu
cudaError_t launch_cell_sort(const RebuildArgs &, cudaStream_t);
cudaError_t launch_neighbors(const RebuildArgs &, cudaStream_t);
int scan_tiles(int ncell);
// nep_md.cu
int md_blocks(int n);
cudaError_t launch_kick_drift(int, double *, double *, double *, double *, double *, double *, const long long *, float4 *,
                              const float4 *, double, double, const double *, float, Control *, cudaStream_t);
cudaError_t launch_control(Control *, bool, cudaStream_t);
cudaError_t launch_control_cond(Control *, cudaGraphConditionalHandle, cudaStream_t);
cudaError_t launch_control_check(Control *, cudaStream_t);
cudaError_t launch_inverse_order(int, const int *, int *, cudaStream_t);
cudaError_t launch_load_state_sorted(int, const double *, const double *, const int *, double *, double *, double *,
                                     double *, double *, double *, float4 *, const float4 *, const double *,
                                     const double *, float, Control *, cudaStream_t);
cudaError_t launch_kick(int, double *, double *, double *, const long long *, double, double, long long *, Control *,
                        cudaStream_t);
cudaError_t launch_kinetic(int, const double *, const double *, const double *, double, long long *, cudaStream_t);
cudaError_t launch_finalize(const long long *, int, const long long *, int, const long long *, int, double *,
                            long long *, cudaStream_t);
cudaError_t launch_load_state(int, const double *, const double *, double *, double *, double *, double *, double *,
                              double *, int *, int *, cudaStream_t);
cudaError_t launch_store_vec(int, const int *, const double *, const double *, const double *, const double *, int,
                             double *, cudaStream_t);
cudaError_t launch_store_force(int, const int *, const long long *, double *, cudaStream_t);
cudaError_t launch_store_scalar(int, const int *, const float *, double *, cudaStream_t);
cudaError_t launch_store_rows(int, int, const int *, const float *, float *, cudaStream_t);
cudaError_t launch_store_neighbors(int, int, int, const int *, const int32_t *, const int32_t *, const int32_t *,
                                   const int32_t *, int32_t *, int32_t *, int32_t *, int32_t *, cudaStream_t);
}  // namespace nep

using namespace nep;

namespace {

constexpr double KB_EV = 8.617333262e-5;
constexpr double ACC_CONV = 9.64853321233100e-3;
constexpr double WAIT_LIMIT_S = 900.0;

enum KClass {
  KC_DRIFT = 0, KC_CELL = 1, KC_NEIGH = 2, KC_DESC = 3, KC_FORCE = 4, KC_KICK = 5, KC_RED = 6, KC_OTHER = 7, KC_FB = 8
};

struct Timer {
  int cls;
  cudaEvent_t a, b;
};

}  // namespace

struct nep_handle {
  cudaStream_t stream = nullptr;
  cudaStream_t aux = nullptr;            // auxiliary stream: the rebuild chain's capture, nep_get_state's second
                                         // copy (created on first use)
  cudaEvent_t aux_ev[2] = {nullptr, nullptr};
  bool own_stream = false;
  int shape = 0;                   // 0: teacher shape (CuShape), 1: student shape (StudentShape)
  Model<CuShape> model_t{};
  Model<StudentShape> model_s{};
  double mass = 1.0;
  float skin = 1.0f, rcR = 0.f, rcA = 0.f;
  int cap = 128;
  int rebuild_every = 0;
  int precision = NEP_FP32;
  std::string err;

  // system
  int n = 0;
  double L[3] = {0, 0, 0}, l[3] = {0, 0, 0};
  int nc[3] = {0, 0, 0};
  int ncell = 0;
  bool have_state = false, have_nlist = false, have_forces = false;
  bool recheck = false;   // an upload kept the list: check the displacements before the next evaluation

  // device buffers
  double *x = nullptr, *y = nullptr, *z = nullptr, *vx = nullptr, *vy = nullptr, *vz = nullptr;
  double *xb = nullptr, *yb = nullptr, *zb = nullptr, *vxb = nullptr, *vyb = nullptr, *vzb = nullptr;
  int *id = nullptr, *idb = nullptr, *cell_of = nullptr, *perm = nullptr;
  float4 *pos = nullptr, *pos_ref = nullptr;
  long long *F = nullptr;          // fixed-point forces [3][n]
  float *usite = nullptr, *qbuf = nullptr;
  void *G = nullptr;               // adjoint rows: float32 (plain) or float16 (mixed) [n][GS]
  int32_t *nbr = nullptr, *nnum = nullptr, *nang = nullptr, *nown = nullptr, *nband0 = nullptr, *nfar = nullptr;
  int *count = nullptr, *cursor = nullptr, *start = nullptr, *tile_sums = nullptr;
  long long *part_d = nullptr, *part_f = nullptr, *part_k = nullptr;   // per-block int64 partial sums
  double *sums = nullptr;
  long long *counters = nullptr;   // pair counts (descriptor, force) and evaluations
  Control *ctrl = nullptr;
  double *io = nullptr;            // staging 2 x [n][3] float64 for host transfers
  int32_t *io_i = nullptr;         // staging for neighbour output
  size_t io_i_elems = 0;
  int nb_d = 0, nb_f = 0, nb_k = 0;

  // host mirrors (pinned)
  double *h_sums = nullptr;
  Control *h_ctrl = nullptr;
  long long *h_counters = nullptr;
  cudaEvent_t done = nullptr;

  // graph of one MD step
  cudaGraphExec_t graph = nullptr;
  double graph_dt = 0.0;
  long long graph_launches = 0;   // our kernel launches in one captured step, outside the rebuild chain
  long long graph_rebuild_launches = 0;   // those of the rebuild chain (run on rebuild steps only)

  // timing
  bool timing = false;
  std::vector<Timer> timers;
  size_t timers_used = 0;
  double ms[NEP_N_KERNEL_CLASSES] = {0};
  long long launches[NEP_N_KERNEL_CLASSES] = {0};
  long long launch_total = 0;

  // per-atom fallback to the teacher (student shape only)
  bool fb_on = false;
  Model<CuShape> fb_model{};
  float fb_lo[16] = {0}, fb_hi[16] = {0};
  double fb_frac = 1.0 / 16.0;
  int fb_cap = 0;
  int *fb_list = nullptr, *fb_count = nullptr;
  float *fb_G = nullptr;

  // buffers of the ablation variants (allocated on first use)
  float *abl_f = nullptr, *abl_s = nullptr;
  int *abl_cnt = nullptr;

  // pair records of the fused kernels (allocated with the system for the teacher and the float32 student)
  float4 *pc_rec = nullptr;
  int *inv = nullptr;                   // cell-order slot of each atom (filled by nep_set_state / nep_get_state)
  unsigned *pc_mask = nullptr;
  int pc_nsm = 0, pc_slots = 0;         // SM index bound and record regions per SM index

  int ndes() const { return shape == 0 ? CuShape::NDES : StudentShape::NDES; }
  int gs() const { return shape == 0 ? CuShape::GS : StudentShape::GS; }
};

namespace {

nep_status fail(nep_handle *h, nep_status s, const std::string &msg) {
  if (h) h->err = msg;
  return s;
}

nep_status cuda_fail(nep_handle *h, cudaError_t e, const char *where) {
  return fail(h, NEP_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define NEP_CUDA(h, call)                                   \
  do {                                                      \
    cudaError_t e_ = (call);                                \
    if (e_ != cudaSuccess) return cuda_fail(h, e_, #call);  \
  } while (0)

bool is_device_ptr(const void *p) {
  if (p == nullptr) return false;
  cudaPointerAttributes a;
  cudaError_t e = cudaPointerGetAttributes(&a, p);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// The device address of page-locked host memory (cudaHostAlloc / cudaHostRegister: kernels read and
// write it directly), else nullptr.
template <class T>
T *pinned_alias(T *p) {
  if (p == nullptr) return nullptr;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return a.type == cudaMemoryTypeHost ? static_cast<T *>(a.devicePointer) : nullptr;
}

template <class T>
void dfree(T *&p) {
  if (p) cudaFree((void *)p);
  p = nullptr;
}

void free_system(nep_handle *h) {
  if (h->graph) { cudaGraphExecDestroy(h->graph); h->graph = nullptr; }
  dfree(h->x); dfree(h->y); dfree(h->z); dfree(h->vx); dfree(h->vy); dfree(h->vz);
  dfree(h->xb); dfree(h->yb); dfree(h->zb); dfree(h->vxb); dfree(h->vyb); dfree(h->vzb);
  dfree(h->id); dfree(h->idb); dfree(h->cell_of); dfree(h->perm);
  dfree(h->pos); dfree(h->pos_ref); dfree(h->F); dfree(h->usite); dfree(h->G); dfree(h->qbuf);
  dfree(h->nbr); dfree(h->nnum); dfree(h->nang); dfree(h->nown); dfree(h->nband0); dfree(h->nfar);
  dfree(h->count); dfree(h->cursor); dfree(h->start); dfree(h->tile_sums);
  dfree(h->part_d); dfree(h->part_f); dfree(h->part_k); dfree(h->io); dfree(h->io_i);
  dfree(h->fb_list); dfree(h->fb_count); dfree(h->fb_G);
  dfree(h->abl_f); dfree(h->abl_s); dfree(h->abl_cnt);
  dfree(h->pc_rec); dfree(h->pc_mask); dfree(h->inv);
  h->pc_nsm = 0;
  h->fb_cap = 0;
  h->io_i_elems = 0;
  h->n = 0;
  h->have_state = h->have_nlist = h->have_forces = false;
}

template <class T>
cudaError_t dalloc(T *&p, size_t elems) {
  return cudaMalloc((void **)&p, std::max<size_t>(elems, 1) * sizeof(T));
}

// Bounded wait for all work enqueued so far on the handle's stream.
nep_status wait_stream(nep_handle *h) {
  NEP_CUDA(h, cudaEventRecord(h->done, h->stream));
  auto t0 = std::chrono::steady_clock::now();
  int spins = 0;
  for (;;) {
    cudaError_t e = cudaEventQuery(h->done);
    if (e == cudaSuccess) break;
    if (e != cudaErrorNotReady) return cuda_fail(h, e, "cudaEventQuery");
    // yield for the first 2 ms (a sleep costs 50-100 us of wake-up latency per wait, ~3 % of an
    // upload + MD step + download cycle on 1M atoms), then sleep between polls
    double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (++spins > 64) {
      if (el < 2e-3) std::this_thread::yield();
      else std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
    if (el > WAIT_LIMIT_S) return fail(h, NEP_ERR_TIMEOUT, "stream wait exceeded its limit");
  }
  return NEP_OK;
}

// Timer helpers: record an event pair around a kernel class when timing is on.
struct Scope {
  nep_handle *h;
  int cls, nlaunch;
  Timer *t = nullptr;
  Scope(nep_handle *h_, int cls_, int nlaunch_) : h(h_), cls(cls_), nlaunch(nlaunch_) {
    h->launch_total += nlaunch;
    if (!h->timing) return;
    if (h->timers_used == h->timers.size()) {
      Timer nt{cls, nullptr, nullptr};
      cudaEventCreate(&nt.a);
      cudaEventCreate(&nt.b);
      h->timers.push_back(nt);
    }
    t = &h->timers[h->timers_used++];
    t->cls = cls;
    cudaEventRecord(t->a, h->stream);
  }
  ~Scope() {
    if (t) cudaEventRecord(t->b, h->stream);
    if (h->timing) h->launches[cls] += nlaunch;
  }
};

void collect_timers(nep_handle *h) {
  for (size_t k = 0; k < h->timers_used; ++k) {
    float m = 0.f;
    if (cudaEventElapsedTime(&m, h->timers[k].a, h->timers[k].b) == cudaSuccess) h->ms[h->timers[k].cls] += m;
    else cudaGetLastError();
  }
  h->timers_used = 0;
}

// Largest squared displacement since the build (Angstrom^2) below which the far band (list entries
// built at r >= rc_R + FAR_EDGE skin) cannot hold a pair inside rc_R: two atoms close by at most twice
// the largest displacement, with a 0.02 Angstrom margin for float32 coordinates.  -1: never skip.
float far_dmax2(float skin) {
  const float d = 0.5f * (FAR_EDGE * skin - 0.02f);
  return d > 0.f ? d * d : -1.f;
}

RebuildArgs rebuild_args(nep_handle *h) {
  RebuildArgs a;
  a.n = h->n; a.ncell = h->ncell;
  for (int d = 0; d < 3; ++d) { a.L[d] = h->L[d]; a.l[d] = h->l[d]; a.nc[d] = h->nc[d]; }
  a.x = h->x; a.y = h->y; a.z = h->z; a.vx = h->vx; a.vy = h->vy; a.vz = h->vz;
  a.xb = h->xb; a.yb = h->yb; a.zb = h->zb; a.vxb = h->vxb; a.vyb = h->vyb; a.vzb = h->vzb;
  a.id = h->id; a.idb = h->idb; a.cell_of = h->cell_of; a.count = h->count; a.cursor = h->cursor;
  a.start = h->start; a.tile_sums = h->tile_sums; a.perm = h->perm;
  a.pos = h->pos; a.pos_ref = h->pos_ref; a.nbr = h->nbr; a.nnum = h->nnum; a.nang = h->nang; a.nown = h->nown; a.nband0 = h->nband0;
  a.nfar = h->nfar;
  a.cap = h->cap;
  const float rl = h->rcR + h->skin, ra = h->rcA + h->skin, fs = h->rcR + FAR_EDGE * h->skin;
  a.rl2 = rl * rl; a.ra2 = ra * ra; a.fs2 = fs * fs;
  a.ba2 = h->rcA * h->rcA; a.br2 = h->rcR * h->rcR;
  a.ctrl = h->ctrl;
  return a;
}

// The list extents the row walks read; the far bands are left out while ctrl->skip_far is set.
RowExt rows_of(nep_handle *h) { return RowExt{h->nnum, h->nown, h->nband0, h->nfar, h->ctrl}; }

Geom geom_of(nep_handle *h) {
  Geom g;
  g.lx = (float)h->l[0]; g.ly = (float)h->l[1]; g.lz = (float)h->l[2];
  g.ncx = h->nc[0]; g.ncy = h->nc[1]; g.ncz = h->nc[2];
  return g;
}

// Rebuild chain (cell sort + neighbour list); kernels act only if ctrl->do_rebuild is set.
cudaError_t enqueue_rebuild(nep_handle *h) {
  RebuildArgs a = rebuild_args(h);
  cudaError_t e;
  {
    Scope sc(h, KC_CELL, 9);
    e = launch_cell_sort(a, h->stream);
  }
  if (e != cudaSuccess) return e;
  Scope sc(h, KC_NEIGH, 1);
  return launch_neighbors(a, h->stream);
}

// Descriptors + network + forces; partial sums reduced with KE partials pk (may be null).
template <class S>
cudaError_t forces_of(nep_handle *h, const Model<S> &M, float *qout) {
  const Geom g = geom_of(h);
  if constexpr (std::is_same<S, CuShape>::value && NEP_FUSED) {
    if (!h->fb_on) {
      // the teacher: descriptors, network and forces in one kernel (forces zeroed first); the network in
      // float32, or as two tensor-core GEMMs with bf16 / f16 operands in the mixed-precision forms
      Scope sc(h, KC_FORCE, 1);
      cudaError_t e = cudaMemsetAsync(h->F, 0, 3 * (size_t)h->n * sizeof(long long), h->stream);
      if (e != cudaSuccess) return e;
      const PairCache pc{h->pc_rec, h->pc_mask, h->pc_nsm, h->cap, h->pc_slots};
      if (h->precision == NEP_FP32)
        return launch_fused<CuShape>(M, g, h->n, h->pos, h->nbr, rows_of(h), h->usite, qout, h->F, h->part_d,
                                     h->part_f, &h->ctrl->status, pc, h->stream);
      if (h->precision == NEP_MIX_BF16)
        return launch_fused_mixed<CuShape, __nv_bfloat16>(M, g, h->n, h->pos, h->nbr, rows_of(h), h->usite, qout, h->F,
                                                          h->part_d, h->part_f, &h->ctrl->status, pc, h->stream);
      return launch_fused_mixed<CuShape, __half>(M, g, h->n, h->pos, h->nbr, rows_of(h), h->usite, qout, h->F,
                                                 h->part_d, h->part_f, &h->ctrl->status, pc, h->stream);
    }
  }
  Fallback fb{};
  fb.on = h->fb_on ? 1 : 0;
  if (fb.on) {
    fb.cap = h->fb_cap; fb.list = h->fb_list; fb.count = h->fb_count;
    for (int v = 0; v < 16; ++v) { fb.lo[v] = h->fb_lo[v]; fb.hi[v] = h->fb_hi[v]; }
  }
  cudaError_t e;
  if (fb.on && (e = cudaMemsetAsync(h->fb_count, 0, sizeof(int), h->stream)) != cudaSuccess) return e;
  if constexpr (std::is_same<S, StudentShape>::value && NEP_FUSED) {
    if (h->precision == NEP_FP32) {
      // the student in float32: descriptors, network and full-row forces in one kernel (forces zeroed
      // first), then the teacher on the flagged atoms
      {
        Scope sc(h, KC_FORCE, 1);
        if ((e = cudaMemsetAsync(h->F, 0, 3 * (size_t)h->n * sizeof(long long), h->stream)) != cudaSuccess) return e;
        const PairCache pc{h->pc_rec, h->pc_mask, h->pc_nsm, h->cap, h->pc_slots};
        e = launch_fused_reg<StudentShape>(M, g, h->n, h->pos, h->nbr, rows_of(h), h->usite, qout, h->F, h->part_d,
                                           h->part_f, &h->ctrl->status, fb, pc, h->stream);
      }
      if (e == cudaSuccess && fb.on) {
        Scope sc(h, KC_FB, 2);
        e = launch_fallback_descriptor<CuShape>(h->fb_model, g, h->n, h->pos, h->nbr, h->nnum, h->fb_list,
                                                h->fb_count, h->fb_cap, h->fb_G, h->usite, h->part_d, h->counters,
                                                &h->ctrl->status, h->stream);
        if (e == cudaSuccess)
          e = launch_fallback_force<CuShape>(h->fb_model, g, h->n, h->pos, h->nbr, h->nnum, h->fb_list, h->fb_count,
                                             h->fb_cap, h->fb_G, h->F, h->part_f, &h->ctrl->status, h->stream);
      }
      return e;
    }
  }
  {
    Scope sc(h, KC_DESC, 1);
    if (h->precision == NEP_FP32)
      e = launch_descriptor<S>(M, g, h->n, h->pos, h->nbr, rows_of(h), static_cast<float *>(h->G), h->usite, qout, h->F,
                               h->part_d, &h->ctrl->status, fb, h->stream);
    else if (h->precision == NEP_MIX_BF16)
      e = launch_descriptor_mixed<S, __nv_bfloat16>(M, g, h->n, h->pos, h->nbr, rows_of(h), static_cast<__half *>(h->G),
                                                     h->usite, qout, h->F, h->part_d, &h->ctrl->status, fb, h->stream);
    else
      e = launch_descriptor_mixed<S, __half>(M, g, h->n, h->pos, h->nbr, rows_of(h), static_cast<__half *>(h->G),
                                              h->usite, qout, h->F, h->part_d, &h->ctrl->status, fb, h->stream);
  }
  if (e != cudaSuccess) return e;
  if (fb.on) {
    Scope sc(h, KC_FB, 1);
    e = launch_fallback_descriptor<CuShape>(h->fb_model, g, h->n, h->pos, h->nbr, h->nnum, h->fb_list, h->fb_count,
                                            h->fb_cap, h->fb_G, h->usite, h->part_d, h->counters, &h->ctrl->status,
                                            h->stream);
    if (e != cudaSuccess) return e;
  }
  {
    Scope sc(h, KC_FORCE, 1);
    if (h->precision == NEP_FP32)
      e = launch_force<S, float>(M, g, h->n, h->pos, h->nbr, rows_of(h), static_cast<const float *>(h->G),
                                 h->F, h->part_f, &h->ctrl->status, h->stream);
    else
      e = launch_force<S, __half>(M, g, h->n, h->pos, h->nbr, rows_of(h), static_cast<const __half *>(h->G),
                                  h->F, h->part_f, &h->ctrl->status, h->stream);
  }
  if (e == cudaSuccess && fb.on) {
    Scope sc(h, KC_FB, 1);
    e = launch_fallback_force<CuShape>(h->fb_model, g, h->n, h->pos, h->nbr, h->nnum, h->fb_list, h->fb_count,
                                       h->fb_cap, h->fb_G, h->F, h->part_f, &h->ctrl->status, h->stream);
  }
  return e;
}

cudaError_t enqueue_forces(nep_handle *h, float *qout) {
  return h->shape == 0 ? forces_of<CuShape>(h, h->model_t, qout) : forces_of<StudentShape>(h, h->model_s, qout);
}

cudaError_t enqueue_finalize(nep_handle *h, bool with_kinetic) {
  Scope sc(h, KC_RED, 1);
  return launch_finalize(h->part_d, h->nb_d, h->part_f, h->nb_f, with_kinetic ? h->part_k : nullptr, h->nb_k, h->sums,
                         h->counters, h->stream);
}

// One velocity-Verlet step.
// One MD step.  Launched eagerly (capture = false) the rebuild chain's kernels run every step and
// return at once unless the control kernel decided to rebuild.  Under stream capture (capture = true)
// the chain is the body of a conditional graph node whose condition the control kernel sets, so a
// step without a rebuild launches none of its kernels; the chain is captured from the auxiliary stream
// into the node's body graph.
cudaError_t enqueue_step(nep_handle *h, double dt, bool capture = false) {
  const double kick = 0.5 * dt * ACC_CONV / h->mass;
  const float hs = 0.5f * h->skin;
  cudaError_t e;
  {
    Scope sc(h, KC_DRIFT, 1);
    e = launch_kick_drift(h->n, h->x, h->y, h->z, h->vx, h->vy, h->vz, h->F, h->pos, h->pos_ref, kick, dt, h->l,
                          hs * hs, h->ctrl, h->stream);
  }
  if (e != cudaSuccess) return e;
  if (!capture) {
    {
      Scope sc(h, KC_CELL, 1);
      e = launch_control(h->ctrl, false, h->stream);
    }
    if (e != cudaSuccess) return e;
    if ((e = enqueue_rebuild(h)) != cudaSuccess) return e;
  } else {
    cudaStreamCaptureStatus cs;
    cudaGraph_t graph = nullptr;
    const cudaGraphNode_t *deps = nullptr;
    size_t nd = 0;
    if ((e = cudaStreamGetCaptureInfo(h->stream, &cs, nullptr, &graph, &deps, nullptr, &nd)) != cudaSuccess) return e;
    cudaGraphConditionalHandle cond;
    if ((e = cudaGraphConditionalHandleCreate(&cond, graph, 0, cudaGraphCondAssignDefault)) != cudaSuccess) return e;
    {
      Scope sc(h, KC_CELL, 1);
      e = launch_control_cond(h->ctrl, cond, h->stream);
    }
    if (e != cudaSuccess) return e;
    if ((e = cudaStreamGetCaptureInfo(h->stream, &cs, nullptr, &graph, &deps, nullptr, &nd)) != cudaSuccess) return e;
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = cond;
    cp.conditional.type = cudaGraphCondTypeIf;
    cp.conditional.size = 1;
    cudaGraphNode_t node;
    if ((e = cudaGraphAddNode(&node, graph, deps, nullptr, nd, &cp)) != cudaSuccess) return e;
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    if ((e = cudaStreamUpdateCaptureDependencies(h->stream, &node, nullptr, 1, cudaStreamSetCaptureDependencies)) !=
        cudaSuccess)
      return e;
    if (!h->aux && (e = cudaStreamCreateWithFlags(&h->aux, cudaStreamNonBlocking)) != cudaSuccess) return e;
    if ((e = cudaStreamBeginCaptureToGraph(h->aux, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal)) !=
        cudaSuccess)
      return e;
    const long long before = h->launch_total;
    cudaStream_t main = h->stream;
    h->stream = h->aux;                       // the chain's launches go to the body graph
    const cudaError_t eb = enqueue_rebuild(h);
    h->stream = main;
    cudaGraph_t captured = nullptr;
    const cudaError_t ee = cudaStreamEndCapture(h->aux, &captured);
    h->graph_rebuild_launches = h->launch_total - before;
    h->launch_total = before;
    if (eb != cudaSuccess) return eb;
    if (ee != cudaSuccess) return ee;
  }
  if ((e = enqueue_forces(h, nullptr)) != cudaSuccess) return e;
  // the energy, virial and pair counts of this evaluation (the kinetic energy is the one of the last
  // closing kick, refreshed by enqueue_step_end); the closing half kick is left to the next step's
  // opening kick, which applies both at once
  Scope sc(h, KC_RED, 1);
  return launch_finalize(h->part_d, h->nb_d, h->part_f, h->nb_f, nullptr, h->nb_k, h->sums, h->counters, h->stream);
}

// The closing half kick of the last step of md_verlet_step, its kinetic energy, and the sums again
// with it (no counters: the evaluation was counted by its own step).
cudaError_t enqueue_step_end(nep_handle *h, double dt) {
  const double kick = 0.5 * dt * ACC_CONV / h->mass;
  cudaError_t e;
  {
    Scope sc(h, KC_KICK, 1);
    e = launch_kick(h->n, h->vx, h->vy, h->vz, h->F, kick, h->mass, h->part_k, h->ctrl, h->stream);
  }
  if (e != cudaSuccess) return e;
  Scope sc(h, KC_RED, 1);
  return launch_finalize(h->part_d, h->nb_d, h->part_f, h->nb_f, h->part_k, h->nb_k, h->sums, nullptr, h->stream);
}

// Read back the control block and translate device-detected conditions into a status.
nep_status check_device_status(nep_handle *h) {
  NEP_CUDA(h, cudaMemcpyAsync(h->h_ctrl, h->ctrl, sizeof(Control), cudaMemcpyDeviceToHost, h->stream));
  NEP_CUDA(h, cudaMemcpyAsync(h->h_sums, h->sums, 32 * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  NEP_CUDA(h, cudaMemcpyAsync(h->h_counters, h->counters, 16 * sizeof(long long), cudaMemcpyDeviceToHost, h->stream));
  nep_status s = wait_stream(h);
  if (s != NEP_OK) return s;
  if (h->timing) collect_timers(h);
  const int st = h->h_ctrl->status;
  if (st & ST_OVERFLOW)
    return fail(h, NEP_ERR_NEIGH_OVERFLOW, "an atom has more neighbours within rc_R + skin than max_neighbors");
  if (st & ST_NAN) return fail(h, NEP_ERR_NAN, "non-finite position, energy or force");
  if (st & ST_TIMEOUT) return fail(h, NEP_ERR_TIMEOUT, "a bounded wait on the tensor cores ran out");
  if (st & ST_FB_OVERFLOW)
    return fail(h, NEP_ERR_FALLBACK_OVERFLOW, "more atoms left the student's range than the fallback list holds");
  if (st & ST_SLOT) return fail(h, NEP_ERR_CUDA, "a block of the fused force kernel found no free pair-record slot");
  return NEP_OK;
}

nep_status ensure_nlist(nep_handle *h) {
  if (h->have_nlist && h->recheck) {
    // an upload kept the list: rebuild (on the device) only if an atom moved more than skin/2
    {
      Scope sc(h, KC_CELL, 1);
      NEP_CUDA(h, launch_control_check(h->ctrl, h->stream));
    }
    NEP_CUDA(h, enqueue_rebuild(h));
    h->recheck = false;
    return NEP_OK;
  }
  if (h->have_nlist) return NEP_OK;
  h->recheck = false;
  {
    Scope sc(h, KC_CELL, 1);
    NEP_CUDA(h, launch_control(h->ctrl, true, h->stream));
  }
  NEP_CUDA(h, enqueue_rebuild(h));
  h->have_nlist = true;
  h->have_forces = false;
  return NEP_OK;
}

nep_status compute_internal(nep_handle *h, float *qout) {
  nep_status s = ensure_nlist(h);
  if (s != NEP_OK) return s;
  NEP_CUDA(h, enqueue_forces(h, qout));
  {
    Scope sc(h, KC_OTHER, 1);
    NEP_CUDA(h, launch_kinetic(h->n, h->vx, h->vy, h->vz, h->mass, h->part_k, h->stream));
  }
  NEP_CUDA(h, enqueue_finalize(h, true));
  h->have_forces = true;
  return NEP_OK;
}

nep_status build_graph(nep_handle *h, double dt) {
  if (h->graph) { cudaGraphExecDestroy(h->graph); h->graph = nullptr; }
  cudaGraph_t g = nullptr;
  const long long before = h->launch_total;
  NEP_CUDA(h, cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
  cudaError_t e = enqueue_step(h, dt, true);
  cudaError_t e2 = cudaStreamEndCapture(h->stream, &g);
  h->graph_launches = h->launch_total - before;   // kernels of one captured step, without the rebuild chain
  h->launch_total = before;
  if (e != cudaSuccess) { if (g) cudaGraphDestroy(g); return cuda_fail(h, e, "capture step"); }
  if (e2 != cudaSuccess) return cuda_fail(h, e2, "cudaStreamEndCapture");
  e = cudaGraphInstantiate(&h->graph, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) { h->graph = nullptr; return cuda_fail(h, e, "cudaGraphInstantiate"); }
  h->graph_dt = dt;
  return NEP_OK;
}

// Copy [n][3] positions/velocities (host or device) into the SoA state, ids = 0..n-1, and reset the
// device status word.
nep_status upload_state(nep_handle *h, const double *x, const double *v) {
  if (h->n > 0) {
    const size_t N = (size_t)h->n;
    NEP_CUDA(h, cudaMemsetAsync(&h->ctrl->status, 0, sizeof(int), h->stream));
    const double *xs = x, *vs = v;
    if (!is_device_ptr(x)) {
      NEP_CUDA(h, cudaMemcpyAsync(h->io, x, 3 * N * sizeof(double), cudaMemcpyHostToDevice, h->stream));
      xs = h->io;
    }
    if (v && !is_device_ptr(v)) {
      NEP_CUDA(h, cudaMemcpyAsync(h->io + 3 * N, v, 3 * N * sizeof(double), cudaMemcpyHostToDevice, h->stream));
      vs = h->io + 3 * N;
    }
    {
      Scope sc(h, KC_OTHER, 1);
      NEP_CUDA(h, launch_load_state(h->n, xs, vs, h->x, h->y, h->z, h->vx, h->vy, h->vz, h->id, &h->ctrl->status,
                                    h->stream));
    }
    nep_status s = check_device_status(h);
    if (s != NEP_OK) return s;
  }
  h->have_state = true;
  return NEP_OK;
}

// Upload into the current cell-sorted order (the list is kept; see k_load_state_sorted).  When no
// atom's float32 cell-relative position changed (for instance, the state just read back with
// nep_get_state is uploaded again, velocities possibly altered) the forces, energy and virial of the
// last evaluation still hold: they are kept, and only the kinetic energy is summed again.
nep_status upload_state_sorted(nep_handle *h, const double *x, const double *v) {
  const size_t N = (size_t)h->n;
  const bool had_forces = h->have_forces, had_recheck = h->recheck;
  h->have_forces = false;
  NEP_CUDA(h, cudaMemsetAsync(&h->ctrl->status, 0, sizeof(int), h->stream));
  NEP_CUDA(h, cudaMemsetAsync(&h->ctrl->changed, 0, sizeof(int), h->stream));
  // device arrays and page-locked host arrays are read by the kernel itself (in the caller's order,
  // contiguously); other host arrays are copied to the device first
  const double *xs = x, *vs = v;
  if (!is_device_ptr(x) && !(xs = pinned_alias(x))) {
    NEP_CUDA(h, cudaMemcpyAsync(h->io, x, 3 * N * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    xs = h->io;
  }
  if (v && !is_device_ptr(v) && !(vs = pinned_alias(v))) {
    NEP_CUDA(h, cudaMemcpyAsync(h->io + 3 * N, v, 3 * N * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    vs = h->io + 3 * N;
  }
  const float hs = 0.5f * h->skin;
  {
    Scope sc(h, KC_OTHER, 2);
    NEP_CUDA(h, launch_inverse_order(h->n, h->id, h->inv, h->stream));
    NEP_CUDA(h, launch_load_state_sorted(h->n, xs, vs, h->inv, h->x, h->y, h->z, h->vx, h->vy, h->vz, h->pos,
                                         h->pos_ref, h->l, h->L, hs * hs, h->ctrl, h->stream));
  }
  h->recheck = true;
  nep_status s = check_device_status(h);
  if (s != NEP_OK || h->h_ctrl->changed || !had_forces) return s;
  // positions unchanged: keep the list state and the forces; refresh the kinetic energy sum (the
  // evaluation counters are not touched: no force evaluation ran)
  h->recheck = had_recheck;
  h->have_forces = true;
  {
    Scope sc(h, KC_OTHER, 1);
    NEP_CUDA(h, launch_kinetic(h->n, h->vx, h->vy, h->vz, h->mass, h->part_k, h->stream));
  }
  {
    Scope sc(h, KC_RED, 1);
    NEP_CUDA(h, launch_finalize(h->part_d, h->nb_d, h->part_f, h->nb_f, h->part_k, h->nb_k, h->sums, nullptr,
                                h->stream));
  }
  return NEP_OK;
}

// Fallback buffers for the current system: flagged-atom list, its length, teacher adjoint rows.
cudaError_t alloc_fallback(nep_handle *h) {
  dfree(h->fb_list); dfree(h->fb_count); dfree(h->fb_G);
  const size_t N = (size_t)std::max(h->n, 1);
  h->fb_cap = (int)std::min<double>((double)N, std::max(1.0, std::ceil((double)N * h->fb_frac)));
  cudaError_t e = dalloc(h->fb_list, (size_t)h->fb_cap);
  if (e == cudaSuccess) e = dalloc(h->fb_count, 1);
  if (e == cudaSuccess) e = dalloc(h->fb_G, (size_t)h->fb_cap * CuShape::GS);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->fb_count, 0, sizeof(int), h->stream);
  return e;
}


}  // namespace

// =====================================================================================================
namespace {

template <class S>
bool shape_matches(const nep_params *p) {
  return p->n_max_R + 1 == S::NR && p->n_max_A + 1 == S::NA && p->basis_R == S::KR && p->basis_A == S::KA &&
         p->l_max_3b == S::LMAX && p->l_max_4b == (S::FOURBODY ? 2 : 0) && p->n_neu == S::NNEU;
}

// Model parameters in the kernels' layout (float32, LJ shifted-force constants precomputed in float64).
template <class S>
void fill_model(Model<S> &M, const nep_params *p) {
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
  M.rcR = p->rc_R; M.rcA = p->rc_A;
  M.rcR2 = p->rc_R * p->rc_R; M.rcA2 = p->rc_A * p->rc_A;
  M.inv_rcR = 1.f / p->rc_R; M.inv_rcA = 1.f / p->rc_A;
  const double eps = p->lj_eps, sig = p->lj_sigma, rc = p->lj_rc;
  M.lj_on = eps != 0.0 ? 1.f : 0.f;
  if (eps != 0.0) {
    const double s6 = std::pow(sig, 6.0);
    const double sr6 = std::pow(sig / rc, 6.0);
    M.lj_c12 = (float)(4.0 * eps * s6 * s6);
    M.lj_c6 = (float)(4.0 * eps * s6);
    M.lj_e_rc = (float)(4.0 * eps * (sr6 * sr6 - sr6));
    M.lj_de_rc = (float)(4.0 * eps * (-12.0 * sr6 * sr6 + 6.0 * sr6) / rc);
    M.lj_e0 = (float)(4.0 * eps * ((-12.0 * sr6 * sr6 + 6.0 * sr6) - (sr6 * sr6 - sr6)));   // rc E'(rc) - E(rc)
    M.lj_m12 = (float)(-12.0 * 4.0 * eps * s6 * s6);
    M.lj_p6 = (float)(6.0 * 4.0 * eps * s6);
    M.lj_rc = (float)rc;
    M.lj_rc2 = (float)(rc * rc);
  } else {
    M.lj_c12 = M.lj_c6 = M.lj_e_rc = M.lj_de_rc = 0.f;
    M.lj_e0 = M.lj_m12 = M.lj_p6 = 0.f;
    M.lj_rc = 0.f; M.lj_rc2 = 0.f;
  }
  const float rmax = std::max(p->rc_R, eps != 0.0 ? p->lj_rc : 0.f);
  M.rmax2 = rmax * rmax;
}

}  // namespace

extern "C" {

const char *nep_status_string(nep_status s) {
  switch (s) {
    case NEP_OK: return "NEP_OK";
    case NEP_ERR_ARG: return "NEP_ERR_ARG";
    case NEP_ERR_CUDA: return "NEP_ERR_CUDA";
    case NEP_ERR_NEIGH_OVERFLOW: return "NEP_ERR_NEIGH_OVERFLOW";
    case NEP_ERR_BOX_TOO_SMALL: return "NEP_ERR_BOX_TOO_SMALL";
    case NEP_ERR_NAN: return "NEP_ERR_NAN";
    case NEP_ERR_TIMEOUT: return "NEP_ERR_TIMEOUT";
    case NEP_ERR_STATE: return "NEP_ERR_STATE";
    case NEP_ERR_UNSUPPORTED: return "NEP_ERR_UNSUPPORTED";
    case NEP_ERR_OOM: return "NEP_ERR_OOM";
    case NEP_ERR_FALLBACK_OVERFLOW: return "NEP_ERR_FALLBACK_OVERFLOW";
  }
  return "NEP_ERR_UNKNOWN";
}

const char *nep_last_error(nep_handle *h) {
  if (!h) return "null handle";
  return h->err.c_str();
}

nep_status nep_create(const nep_params *p, void *cuda_stream, nep_handle **out) {
  if (!p || !out) return NEP_ERR_ARG;
  *out = nullptr;
  int shape;
  if (shape_matches<CuShape>(p)) shape = 0;
  else if (shape_matches<StudentShape>(p)) shape = 1;
  else return NEP_ERR_UNSUPPORTED;
  if (p->precision != NEP_FP32 && p->precision != NEP_MIX_BF16 && p->precision != NEP_MIX_FP16)
    return NEP_ERR_UNSUPPORTED;
  if (!p->c_R || !p->c_A || !p->W0 || !p->b0 || !p->w1 || !p->q_scale) return NEP_ERR_ARG;
  if (!(p->rc_R > 0.f) || !(p->rc_A > 0.f) || p->rc_A > p->rc_R || !(p->skin >= 0.f) || !(p->mass_amu > 0.0))
    return NEP_ERR_ARG;
  if (p->lj_eps != 0.f && (!(p->lj_rc > 0.f) || p->lj_rc > p->rc_R || !(p->lj_sigma > 0.f))) return NEP_ERR_ARG;
  if (p->max_neighbors < 0 || p->max_neighbors > 128 || p->rebuild_every < 0) return NEP_ERR_ARG;

  nep_handle *h = new (std::nothrow) nep_handle();
  if (!h) return NEP_ERR_OOM;
  h->shape = shape;
  if (shape == 0) fill_model(h->model_t, p);
  else fill_model(h->model_s, p);
  h->mass = p->mass_amu;
  h->skin = p->skin;
  h->rcR = p->rc_R;
  h->rcA = p->rc_A;
  h->cap = p->max_neighbors ? p->max_neighbors : 128;
  h->rebuild_every = p->rebuild_every;
  h->precision = p->precision;

  cudaError_t e;
  if (cuda_stream) {
    h->stream = (cudaStream_t)cuda_stream;
  } else {
    e = cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) { delete h; return NEP_ERR_CUDA; }
    h->own_stream = true;
  }
  if ((e = cudaEventCreateWithFlags(&h->done, cudaEventDisableTiming)) != cudaSuccess ||
      (e = dalloc(h->sums, 32)) != cudaSuccess || (e = dalloc(h->counters, 16)) != cudaSuccess ||
      (e = dalloc(h->ctrl, 1)) != cudaSuccess || (e = cudaMallocHost((void **)&h->h_sums, 32 * sizeof(double))) != cudaSuccess ||
      (e = cudaMallocHost((void **)&h->h_ctrl, sizeof(Control))) != cudaSuccess ||
      (e = cudaMallocHost((void **)&h->h_counters, 16 * sizeof(long long))) != cudaSuccess) {
    nep_destroy(h);
    return NEP_ERR_CUDA;
  }
  cudaMemsetAsync(h->sums, 0, 32 * sizeof(double), h->stream);
  cudaMemsetAsync(h->counters, 0, 16 * sizeof(long long), h->stream);
  Control c0{};
  c0.rebuild_every = h->rebuild_every;
  c0.far_dmax2 = far_dmax2(h->skin);
  cudaMemcpyAsync(h->ctrl, &c0, sizeof(Control), cudaMemcpyHostToDevice, h->stream);
  if ((e = cudaStreamSynchronize(h->stream)) != cudaSuccess) { nep_destroy(h); return NEP_ERR_CUDA; }
  *out = h;
  return NEP_OK;
}

nep_status nep_destroy(nep_handle *h) {
  if (!h) return NEP_OK;
  if (h->stream) cudaStreamSynchronize(h->stream);
  free_system(h);
  dfree(h->sums); dfree(h->counters); dfree(h->ctrl);
  if (h->h_sums) cudaFreeHost(h->h_sums);
  if (h->h_ctrl) cudaFreeHost(h->h_ctrl);
  if (h->h_counters) cudaFreeHost(h->h_counters);
  for (auto &t : h->timers) { cudaEventDestroy(t.a); cudaEventDestroy(t.b); }
  if (h->done) cudaEventDestroy(h->done);
  for (cudaEvent_t ev : h->aux_ev)
    if (ev) cudaEventDestroy(ev);
  if (h->aux) cudaStreamDestroy(h->aux);
  if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
  delete h;
  return NEP_OK;
}

nep_status nep_set_state(nep_handle *h, int64_t n, const double *x, const double *v, const double *box) {
  if (!h) return NEP_ERR_ARG;
  if (n < 0 || n > NEP_MAX_ATOMS) return fail(h, NEP_ERR_ARG, "atom count out of range");
  if (n > 0 && !x) return fail(h, NEP_ERR_ARG, "positions are NULL");
  if (!box) return fail(h, NEP_ERR_ARG, "box is NULL");
  const double rl = (double)h->rcR + (double)h->skin;
  for (int d = 0; d < 3; ++d) {
    if (!(box[d] > 0.0) || !std::isfinite(box[d])) return fail(h, NEP_ERR_ARG, "box edges must be positive and finite");
    if (box[d] < 2.0 * rl) return fail(h, NEP_ERR_BOX_TOO_SMALL, "every box edge must be >= 2 (rc_R + skin)");
  }
  cudaStreamSynchronize(h->stream);
  const bool same = h->have_state && h->n == (int)n && h->L[0] == box[0] && h->L[1] == box[1] && h->L[2] == box[2];
  if (same && h->have_nlist) {
    // Same size and box with a neighbour list: keep the list and the cell order; the next
    // evaluation rebuilds only if an atom moved more than skin/2 from where the list was built.
    return upload_state_sorted(h, x, v);
  }
  if (same) {
    // Same size and box: keep every buffer (and the captured step graph); upload and invalidate.
    h->have_nlist = h->have_forces = false;
    return upload_state(h, x, v);
  }
  free_system(h);
  h->n = (int)n;
  int64_t ncell = 1;
  for (int d = 0; d < 3; ++d) {
    h->L[d] = box[d];
    int nc = (int)std::floor(box[d] / rl);
    nc = std::max(2, std::min(nc, 1023));
    h->nc[d] = nc;
    h->l[d] = box[d] / nc;
    ncell *= nc;
  }
  if (ncell > (int64_t)1 << 30) return fail(h, NEP_ERR_ARG, "too many cells");
  h->ncell = (int)ncell;
  h->nb_d = h->precision == NEP_FP32 ? descriptor_blocks(h->n) : mixed_descriptor_blocks(h->n);
  h->nb_f = force_blocks(h->n);
  h->nb_k = md_blocks(h->n);
  const size_t N = (size_t)std::max(h->n, 1);
  cudaError_t e = cudaSuccess;
  auto A = [&](cudaError_t r) { if (e == cudaSuccess) e = r; };
  A(dalloc(h->x, N)); A(dalloc(h->y, N)); A(dalloc(h->z, N)); A(dalloc(h->vx, N)); A(dalloc(h->vy, N)); A(dalloc(h->vz, N));
  A(dalloc(h->xb, N)); A(dalloc(h->yb, N)); A(dalloc(h->zb, N)); A(dalloc(h->vxb, N)); A(dalloc(h->vyb, N)); A(dalloc(h->vzb, N));
  A(dalloc(h->id, N)); A(dalloc(h->idb, N)); A(dalloc(h->cell_of, N)); A(dalloc(h->perm, N)); A(dalloc(h->inv, N));
  A(dalloc(h->pos, N)); A(dalloc(h->pos_ref, N));
  A(dalloc(h->F, 3 * N)); A(dalloc(h->usite, N));
  A(dalloc(reinterpret_cast<char *&>(h->G), N * (size_t)h->gs() * (h->precision == NEP_FP32 ? 4 : 2)));
  A(dalloc(h->nbr, N * (size_t)h->cap)); A(dalloc(h->nnum, N)); A(dalloc(h->nang, N)); A(dalloc(h->nown, N));
  A(dalloc(h->nband0, N)); A(dalloc(h->nfar, N));
  A(dalloc(h->count, (size_t)h->ncell)); A(dalloc(h->cursor, (size_t)h->ncell)); A(dalloc(h->start, (size_t)h->ncell + 1));
  A(dalloc(h->tile_sums, (size_t)scan_tiles(h->ncell) + 1));
  A(dalloc(h->part_d, (size_t)h->nb_d * 5 + 1)); A(dalloc(h->part_f, (size_t)h->nb_f * 13 + 1));
  A(dalloc(h->part_k, (size_t)h->nb_k + 1)); A(dalloc(h->io, 6 * N));
  if (h->fb_on) A(alloc_fallback(h));
  if (e == cudaSuccess && (h->shape == 0 || h->precision == NEP_FP32)) {
    // pair records of the fused kernels: pc_slots regions per SM index, list capacity records per atom
    h->pc_slots = h->shape == 0 ? PC_SLOTS : PC_SLOTS_REG;
    A(pair_cache_sm_bound(&h->pc_nsm));
    // record offsets are 32-bit: nsm * slots (<= 8) * cap (<= 128) * 128 < 2^32 for nsm <= 4096
    if (e == cudaSuccess && (h->pc_nsm <= 0 || h->pc_nsm > 4096)) e = cudaErrorInvalidValue;
    if (e == cudaSuccess) {
      A(dalloc(h->pc_rec, (size_t)h->pc_nsm * h->pc_slots * pair_cache_region_elems(h->cap)));
      A(dalloc(h->pc_mask, (size_t)h->pc_nsm));
      if (e == cudaSuccess) A(cudaMemsetAsync(h->pc_mask, 0, (size_t)h->pc_nsm * sizeof(unsigned), h->stream));
    }
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    free_system(h);
    return fail(h, e == cudaErrorMemoryAllocation ? NEP_ERR_OOM : NEP_ERR_CUDA,
                std::string("allocation failed: ") + cudaGetErrorString(e));
  }
  NEP_CUDA(h, cudaMemsetAsync(h->F, 0, 3 * N * sizeof(long long), h->stream));
  NEP_CUDA(h, cudaMemsetAsync(h->sums, 0, 32 * sizeof(double), h->stream));
  NEP_CUDA(h, cudaMemsetAsync(h->counters, 0, 16 * sizeof(long long), h->stream));
  Control c0{};
  c0.rebuild_every = h->rebuild_every;
  c0.far_dmax2 = far_dmax2(h->skin);
  NEP_CUDA(h, cudaMemcpyAsync(h->ctrl, &c0, sizeof(Control), cudaMemcpyHostToDevice, h->stream));
  return upload_state(h, x, v);
}

nep_status nep_build_neighbors(nep_handle *h) {
  if (!h) return NEP_ERR_ARG;
  if (!h->have_state) return fail(h, NEP_ERR_STATE, "nep_set_state has not been called");
  if (h->n == 0) return NEP_OK;
  h->have_nlist = false;
  nep_status s = ensure_nlist(h);
  if (s != NEP_OK) return s;
  return check_device_status(h);
}

nep_status nep_compute(nep_handle *h, double *E, double *F, double *virial) {
  if (!h) return NEP_ERR_ARG;
  if (!h->have_state) return fail(h, NEP_ERR_STATE, "nep_set_state has not been called");
  if (h->n == 0) {
    if (E) *E = 0.0;
    if (virial) for (int k = 0; k < 9; ++k) virial[k] = 0.0;
    return NEP_OK;
  }
  nep_status s = compute_internal(h, nullptr);
  if (s != NEP_OK) return s;
  const bool fdev = F && is_device_ptr(F);
  if (F) {
    Scope sc(h, KC_OTHER, 1);
    NEP_CUDA(h, launch_store_force(h->n, h->id, h->F, fdev ? F : h->io, h->stream));
    if (!fdev)
      NEP_CUDA(h, cudaMemcpyAsync(F, h->io, 3 * (size_t)h->n * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  }
  s = check_device_status(h);
  if (s != NEP_OK) return s;
  if (E) *E = h->h_sums[0];
  if (virial) for (int k = 0; k < 9; ++k) virial[k] = h->h_sums[1 + k];
  return NEP_OK;
}

nep_status md_verlet_step(nep_handle *h, double dt_fs, int n_steps) {
  if (!h) return NEP_ERR_ARG;
  if (!h->have_state) return fail(h, NEP_ERR_STATE, "nep_set_state has not been called");
  if (n_steps < 0 || !(std::isfinite(dt_fs))) return fail(h, NEP_ERR_ARG, "bad dt or step count");
  if (h->n == 0 || n_steps == 0) return NEP_OK;
  if (!h->have_forces) {
    nep_status s = compute_internal(h, nullptr);
    if (s == NEP_OK && !h->timing) s = check_device_status(h);   // the host copy of the rebuild count
    if (s != NEP_OK) return s;
  }
  if (h->timing) {
    for (int k = 0; k < n_steps; ++k) NEP_CUDA(h, enqueue_step(h, dt_fs));
    NEP_CUDA(h, enqueue_step_end(h, dt_fs));
  } else {
    if (!h->graph || h->graph_dt != dt_fs) {
      nep_status s = build_graph(h, dt_fs);
      if (s != NEP_OK) return s;
    }
    const long long rebuilds_before = h->h_ctrl->rebuilds;
    for (int k = 0; k < n_steps; ++k) NEP_CUDA(h, cudaGraphLaunch(h->graph, h->stream));
    NEP_CUDA(h, enqueue_step_end(h, dt_fs));
    nep_status s = check_device_status(h);
    // the rebuild chain's kernels ran on the rebuild steps only
    h->launch_total += h->graph_launches * n_steps + h->graph_rebuild_launches * (h->h_ctrl->rebuilds - rebuilds_before);
    return s;
  }
  return check_device_status(h);
}

nep_status nep_get_state(nep_handle *h, double *x, double *v) {
  if (!h) return NEP_ERR_ARG;
  if (!h->have_state) return fail(h, NEP_ERR_STATE, "nep_set_state has not been called");
  if (h->n == 0) return NEP_OK;
  const size_t N3 = 3 * (size_t)h->n;
  {
    Scope sc(h, KC_OTHER, 1);
    NEP_CUDA(h, launch_inverse_order(h->n, h->id, h->inv, h->stream));
  }
  // device arrays and page-locked host arrays are written by the store kernel itself (16-byte stores of
  // whole rows: over the host link this outruns a staging buffer and a copy); pageable host arrays
  // through the staging buffer and a copy, the positions' copy on a second stream beside the
  // velocities' store and copy.
  if (!h->aux) NEP_CUDA(h, cudaStreamCreateWithFlags(&h->aux, cudaStreamNonBlocking));
  for (cudaEvent_t &ev : h->aux_ev)
    if (!ev) NEP_CUDA(h, cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
  bool aux_used = false;
  for (int which = 0; which < 2; ++which) {
    double *out = which == 0 ? x : v;
    if (!out) continue;
    double *direct = is_device_ptr(out) ? out : pinned_alias(out);
    const bool dev = direct != nullptr;
    double *stage = dev ? direct : h->io + which * N3;
    {
      Scope sc(h, KC_OTHER, 1);
      if (which == 0) NEP_CUDA(h, launch_store_vec(h->n, h->inv, h->x, h->y, h->z, h->L, 1, stage, h->stream));
      else NEP_CUDA(h, launch_store_vec(h->n, h->inv, h->vx, h->vy, h->vz, h->L, 0, stage, h->stream));
    }
    if (dev) continue;
    if (which == 0) {
      NEP_CUDA(h, cudaEventRecord(h->aux_ev[0], h->stream));
      NEP_CUDA(h, cudaStreamWaitEvent(h->aux, h->aux_ev[0], 0));
      NEP_CUDA(h, cudaMemcpyAsync(out, stage, N3 * sizeof(double), cudaMemcpyDeviceToHost, h->aux));
      NEP_CUDA(h, cudaEventRecord(h->aux_ev[1], h->aux));
      aux_used = true;
    } else {
      NEP_CUDA(h, cudaMemcpyAsync(out, stage, N3 * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    }
  }
  if (aux_used) NEP_CUDA(h, cudaStreamWaitEvent(h->stream, h->aux_ev[1], 0));
  return wait_stream(h);
}

nep_status nep_get_thermo(nep_handle *h, double out[8]) {
  if (!h || !out) return NEP_ERR_ARG;
  if (!h->have_state) return fail(h, NEP_ERR_STATE, "nep_set_state has not been called");
  nep_status s = check_device_status(h);
  if (s != NEP_OK) return s;
  const double pe = h->h_sums[0], ke = h->h_sums[10];
  const double V = h->L[0] * h->L[1] * h->L[2];
  const double trW = h->h_sums[1] + h->h_sums[5] + h->h_sums[9];
  out[0] = pe;
  out[1] = ke;
  out[2] = h->n > 1 ? 2.0 * ke / ((3.0 * h->n - 3.0) * KB_EV) : 0.0;
  out[3] = (2.0 * ke + trW) / (3.0 * V);
  out[4] = h->h_sums[1]; out[5] = h->h_sums[5]; out[6] = h->h_sums[9];
  out[7] = (double)h->h_ctrl->rebuilds;
  return NEP_OK;
}

nep_status nep_get_neighbors(nep_handle *h, int32_t *counts, int32_t *n_ang, int32_t *n_own, int32_t *list, int cap) {
  if (!h || !counts || !n_ang || !n_own || !list || cap <= 0) return NEP_ERR_ARG;
  if (!h->have_state) return fail(h, NEP_ERR_STATE, "nep_set_state has not been called");
  if (h->n == 0) return NEP_OK;
  nep_status s = ensure_nlist(h);
  if (s != NEP_OK) return s;
  const size_t N = (size_t)h->n;
  const size_t elems = N * 3 + N * (size_t)cap;
  if (h->io_i_elems < elems) {
    dfree(h->io_i);
    NEP_CUDA(h, dalloc(h->io_i, elems));
    h->io_i_elems = elems;
  }
  {
    Scope sc(h, KC_OTHER, 1);
    NEP_CUDA(h, launch_store_neighbors(h->n, h->cap, cap, h->id, h->nbr, h->nnum, h->nang, h->nown, h->io_i,
                                       h->io_i + N, h->io_i + 2 * N, h->io_i + 3 * N, h->stream));
  }
  NEP_CUDA(h, cudaMemcpyAsync(counts, h->io_i, N * sizeof(int32_t), cudaMemcpyDefault, h->stream));
  NEP_CUDA(h, cudaMemcpyAsync(n_ang, h->io_i + N, N * sizeof(int32_t), cudaMemcpyDefault, h->stream));
  NEP_CUDA(h, cudaMemcpyAsync(n_own, h->io_i + 2 * N, N * sizeof(int32_t), cudaMemcpyDefault, h->stream));
  NEP_CUDA(h, cudaMemcpyAsync(list, h->io_i + 3 * N, N * (size_t)cap * sizeof(int32_t), cudaMemcpyDefault, h->stream));
  return check_device_status(h);
}

nep_status nep_get_descriptors(nep_handle *h, float *q) {
  if (!h || !q) return NEP_ERR_ARG;
  if (!h->have_state) return fail(h, NEP_ERR_STATE, "nep_set_state has not been called");
  if (h->n == 0) return NEP_OK;
  const size_t N = (size_t)h->n;
  const size_t D = (size_t)h->ndes();
  if (!h->qbuf) NEP_CUDA(h, dalloc(h->qbuf, 2 * N * D));
  nep_status s = compute_internal(h, h->qbuf);
  if (s != NEP_OK) return s;
  {
    Scope sc(h, KC_OTHER, 1);
    NEP_CUDA(h, launch_store_rows(h->n, (int)D, h->id, h->qbuf, h->qbuf + N * D, h->stream));
  }
  NEP_CUDA(h, cudaMemcpyAsync(q, h->qbuf + N * D, N * D * sizeof(float), cudaMemcpyDefault, h->stream));
  return check_device_status(h);
}

nep_status nep_get_site_energies(nep_handle *h, double *U) {
  if (!h || !U) return NEP_ERR_ARG;
  if (!h->have_state) return fail(h, NEP_ERR_STATE, "nep_set_state has not been called");
  if (h->n == 0) return NEP_OK;
  if (!h->have_forces) {
    nep_status s = compute_internal(h, nullptr);
    if (s != NEP_OK) return s;
  }
  const bool dev = is_device_ptr(U);
  {
    Scope sc(h, KC_OTHER, 1);
    NEP_CUDA(h, launch_store_scalar(h->n, h->id, h->usite, dev ? U : h->io, h->stream));
  }
  if (!dev) NEP_CUDA(h, cudaMemcpyAsync(U, h->io, (size_t)h->n * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  return check_device_status(h);
}

nep_status nep_set_timing(nep_handle *h, int enable) {
  if (!h) return NEP_ERR_ARG;
  cudaStreamSynchronize(h->stream);
  h->timing = enable != 0;
  h->timers_used = 0;
  for (int k = 0; k < NEP_N_KERNEL_CLASSES; ++k) { h->ms[k] = 0.0; h->launches[k] = 0; }
  return NEP_OK;
}

nep_status nep_get_timing(nep_handle *h, double ms[NEP_N_KERNEL_CLASSES], int64_t launches[NEP_N_KERNEL_CLASSES]) {
  if (!h || !ms || !launches) return NEP_ERR_ARG;
  nep_status s = wait_stream(h);
  if (s != NEP_OK) return s;
  collect_timers(h);
  for (int k = 0; k < NEP_N_KERNEL_CLASSES; ++k) { ms[k] = h->ms[k]; launches[k] = h->launches[k]; }
  return NEP_OK;
}

nep_status nep_get_counters(nep_handle *h, int64_t out[13]) {
  if (!h || !out) return NEP_ERR_ARG;
  nep_status s = check_device_status(h);
  if (s != NEP_OK && s != NEP_ERR_NEIGH_OVERFLOW && s != NEP_ERR_NAN) return s;
  const long long *c = h->h_counters;
  out[0] = c[0];                // descriptor: radial pairs
  out[1] = c[1];                // descriptor: angular pairs
  out[2] = c[8];                // force evaluations
  out[3] = h->h_ctrl->rebuilds;
  out[4] = h->h_ctrl->steps;
  out[5] = h->launch_total;
  out[6] = c[2];                // descriptor: list entries
  out[7] = c[3];                // descriptor: active pairs
  out[8] = c[4];                // force: owned list entries
  out[9] = c[5];                // force: owned active pairs
  out[10] = c[6];               // force: owned radial pairs
  out[11] = c[7];               // force: owned angular pairs
  out[12] = c[9];               // atom evaluations by the fallback model
  return NEP_OK;
}

nep_status nep_set_fallback(nep_handle *h, const nep_params *teacher, const float *q_lo, const float *q_hi,
                            float margin, double max_fraction) {
  if (!h) return NEP_ERR_ARG;
  if (teacher == nullptr) {
    h->fb_on = false;
    if (h->graph) { cudaGraphExecDestroy(h->graph); h->graph = nullptr; }
    return NEP_OK;
  }
  if (h->shape != 1) return fail(h, NEP_ERR_UNSUPPORTED, "the fallback is for a student-shaped model");
  if (!shape_matches<CuShape>(teacher)) return fail(h, NEP_ERR_UNSUPPORTED, "the fallback model must have the teacher shape");
  if (!q_lo || !q_hi || !(margin >= 0.f) || !(max_fraction >= 0.0) || max_fraction > 1.0)
    return fail(h, NEP_ERR_ARG, "invalid fallback range");
  if (!teacher->c_R || !teacher->c_A || !teacher->W0 || !teacher->b0 || !teacher->w1 || !teacher->q_scale)
    return fail(h, NEP_ERR_ARG, "fallback model arrays are NULL");
  if (teacher->rc_R != h->rcR || teacher->rc_A > h->rcR)
    return fail(h, NEP_ERR_ARG, "the fallback model must use the student's radial cutoff");
  nep_params t = *teacher;
  t.lj_eps = 0.f;                                  // the LJ term stays with the student's kernels
  fill_model(h->fb_model, &t);
  for (int v = 0; v < 16; ++v) { h->fb_lo[v] = -INFINITY; h->fb_hi[v] = INFINITY; }
  for (int v = 0; v < StudentShape::NDES; ++v) {
    const float w = q_hi[v] - q_lo[v];
    h->fb_lo[v] = q_lo[v] - margin * w;
    h->fb_hi[v] = q_hi[v] + margin * w;
  }
  h->fb_frac = max_fraction > 0.0 ? max_fraction : 1.0 / 16.0;
  h->fb_on = true;
  if (h->graph) { cudaGraphExecDestroy(h->graph); h->graph = nullptr; }
  h->have_forces = false;
  if (h->have_state) {
    cudaError_t e = alloc_fallback(h);
    if (e != cudaSuccess) {
      cudaGetLastError();
      h->fb_on = false;
      return fail(h, e == cudaErrorMemoryAllocation ? NEP_ERR_OOM : NEP_ERR_CUDA, "fallback allocation failed");
    }
  }
  return NEP_OK;
}

nep_status nep_angular_p90(nep_handle *h, int *p90, int *cpb) {
  if (!h || !p90 || !cpb) return NEP_ERR_ARG;
  if (!h->have_state) return fail(h, NEP_ERR_STATE, "nep_set_state has not been called");
  if (h->shape != 0) return fail(h, NEP_ERR_UNSUPPORTED, "the CPB variants exist for the teacher shape");
  *p90 = 0;
  *cpb = 3;
  if (h->n == 0) return NEP_OK;
  nep_status s = ensure_nlist(h);
  if (s != NEP_OK) return s;
  const size_t N = (size_t)h->n;
  if (!h->abl_cnt) NEP_CUDA(h, dalloc(h->abl_cnt, N));
  int *counts = h->abl_cnt;
  NEP_CUDA(h, launch_angular_counts(h->n, h->pos, h->nbr, rows_of(h), geom_of(h), h->rcA * h->rcA, counts, h->stream));
  std::vector<int> hc(N);
  NEP_CUDA(h, cudaMemcpyAsync(hc.data(), counts, N * sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  s = wait_stream(h);
  if (s != NEP_OK) return s;
  const size_t k = std::min(N - 1, (size_t)std::ceil(0.9 * (double)N) - 1);
  std::nth_element(hc.begin(), hc.begin() + (long)k, hc.end());
  *p90 = hc[k];
  *cpb = *p90 <= 10 ? 3 : (*p90 < 24 ? 2 : 1);
  return NEP_OK;
}

nep_status nep_run_variant(nep_handle *h, int variant, double *ms, double *F) {
  if (!h || !ms) return NEP_ERR_ARG;
  if (!h->have_state) return fail(h, NEP_ERR_STATE, "nep_set_state has not been called");
  if (variant < NEP_VARIANT_FLOAT_SCATTER || variant > NEP_VARIANT_CPB_AUTO)
    return fail(h, NEP_ERR_ARG, "unknown variant");
  if (h->shape != 0 || h->precision != NEP_FP32 || h->fb_on)
    return fail(h, NEP_ERR_UNSUPPORTED, "the variants exist for the plain float32 teacher path");
  if (h->n == 0) { *ms = 0.0; return NEP_OK; }
  nep_status s = ensure_nlist(h);
  if (s != NEP_OK) return s;
  const Geom g = geom_of(h);
  const size_t N = (size_t)h->n;
  float *G = static_cast<float *>(h->G);
  cudaEvent_t a = nullptr, b = nullptr;
  NEP_CUDA(h, cudaEventCreate(&a));
  NEP_CUDA(h, cudaEventCreate(&b));
  cudaError_t e = cudaSuccess;
  {
    Scope sc(h, KC_OTHER, 3);
    if (variant == NEP_VARIANT_FLOAT_SCATTER) {
      if (!h->abl_f) e = dalloc(h->abl_f, 3 * N);
      if (e == cudaSuccess)
        e = launch_descriptor<CuShape>(h->model_t, g, h->n, h->pos, h->nbr, rows_of(h), G, h->usite, nullptr, h->F,
                                       h->part_d, &h->ctrl->status, Fallback{}, h->stream);
      if (e == cudaSuccess) e = cudaMemsetAsync(h->abl_f, 0, 3 * N * sizeof(float), h->stream);
      if (e == cudaSuccess) e = cudaEventRecord(a, h->stream);
      if (e == cudaSuccess)
        e = launch_force_float_scatter<CuShape>(h->model_t, g, h->n, h->pos, h->nbr, rows_of(h), G, h->abl_f,
                                                h->part_f, &h->ctrl->status, h->stream);
      if (e == cudaSuccess) e = cudaEventRecord(b, h->stream);
      if (e == cudaSuccess) e = launch_store_float3(h->n, h->id, h->abl_f, h->io, h->stream);
    } else if (variant == NEP_VARIANT_HALF_LIST || variant == NEP_VARIANT_SEPARATE_FORCE) {
      e = launch_descriptor<CuShape>(h->model_t, g, h->n, h->pos, h->nbr, rows_of(h), G, h->usite, nullptr, h->F,
                                     h->part_d, &h->ctrl->status, Fallback{}, h->stream);
      if (e == cudaSuccess) e = cudaEventRecord(a, h->stream);
      if (e == cudaSuccess && variant == NEP_VARIANT_HALF_LIST)
        e = launch_force_half_list<CuShape>(h->model_t, g, h->n, h->pos, h->nbr, rows_of(h), G, h->F,
                                            h->part_f, &h->ctrl->status, h->stream);
      if (e == cudaSuccess && variant == NEP_VARIANT_SEPARATE_FORCE)
        e = launch_force<CuShape, float>(h->model_t, g, h->n, h->pos, h->nbr, rows_of(h), G, h->F,
                                         h->part_f, &h->ctrl->status, h->stream);
      if (e == cudaSuccess) e = cudaEventRecord(b, h->stream);
      if (e == cudaSuccess) e = launch_store_force(h->n, h->id, h->F, h->io, h->stream);
    } else if (variant >= NEP_VARIANT_CPB1 && variant <= NEP_VARIANT_CPB_AUTO) {
      int cpb = variant - NEP_VARIANT_CPB1 + 1;
      if (variant == NEP_VARIANT_CPB_AUTO) {
        int p90 = 0;
        const nep_status ps = nep_angular_p90(h, &p90, &cpb);
        if (ps != NEP_OK) {
          cudaEventDestroy(a); cudaEventDestroy(b);
          return ps;
        }
      }
      e = launch_descriptor<CuShape>(h->model_t, g, h->n, h->pos, h->nbr, rows_of(h), G, h->usite, nullptr, h->F,
                                     h->part_d, &h->ctrl->status, Fallback{}, h->stream);
      if (e == cudaSuccess) e = cudaEventRecord(a, h->stream);
      if (e == cudaSuccess)
        e = launch_force_cpb<CuShape>(cpb, h->model_t, g, h->n, h->pos, h->nbr, rows_of(h), G, h->F, h->part_f,
                                      &h->ctrl->status, h->stream);
      if (e == cudaSuccess) e = cudaEventRecord(b, h->stream);
      if (e == cudaSuccess) e = launch_store_force(h->n, h->id, h->F, h->io, h->stream);
    } else if (variant == NEP_VARIANT_SEPARATE_DESCRIPTOR) {
      e = cudaEventRecord(a, h->stream);
      if (e == cudaSuccess)
        e = launch_descriptor<CuShape>(h->model_t, g, h->n, h->pos, h->nbr, rows_of(h), G, h->usite, nullptr, h->F,
                                       h->part_d, &h->ctrl->status, Fallback{}, h->stream);
      if (e == cudaSuccess) e = cudaEventRecord(b, h->stream);
      if (e == cudaSuccess)
        e = launch_force<CuShape, float>(h->model_t, g, h->n, h->pos, h->nbr, rows_of(h), G, h->F,
                                         h->part_f, &h->ctrl->status, h->stream);
      if (e == cudaSuccess) e = launch_store_force(h->n, h->id, h->F, h->io, h->stream);
    } else {
      if (!h->abl_s) e = dalloc(h->abl_s, (size_t)CuShape::NA * CuShape::NLM * N);
      if (e == cudaSuccess) e = cudaEventRecord(a, h->stream);
      if (e == cudaSuccess) {
        if (variant == NEP_VARIANT_TILE1)
          e = launch_descriptor_tiled<CuShape, 1>(h->model_t, g, h->n, h->pos, h->nbr, rows_of(h), G, h->usite, h->F,
                                                  h->part_d, &h->ctrl->status, h->abl_s, h->stream);
        else
          e = launch_descriptor_tiled<CuShape, 3>(h->model_t, g, h->n, h->pos, h->nbr, rows_of(h), G, h->usite, h->F,
                                                  h->part_d, &h->ctrl->status, h->abl_s, h->stream);
      }
      if (e == cudaSuccess) e = cudaEventRecord(b, h->stream);
      if (e == cudaSuccess)
        e = launch_force<CuShape, float>(h->model_t, g, h->n, h->pos, h->nbr, rows_of(h), G, h->F, h->part_f,
                                         &h->ctrl->status, h->stream);
      if (e == cudaSuccess) e = launch_store_force(h->n, h->id, h->F, h->io, h->stream);
    }
  }
  if (e == cudaSuccess && F) e = cudaMemcpyAsync(F, h->io, 3 * N * sizeof(double), cudaMemcpyDefault, h->stream);
  h->have_forces = false;              // the handle's own results are recomputed on the next request
  if (e != cudaSuccess) {
    cudaEventDestroy(a); cudaEventDestroy(b);
    return cuda_fail(h, e, "variant");
  }
  s = check_device_status(h);
  float m = 0.f;
  if (s == NEP_OK && cudaEventElapsedTime(&m, a, b) != cudaSuccess) s = cuda_fail(h, cudaGetLastError(), "timing");
  cudaEventDestroy(a); cudaEventDestroy(b);
  *ms = m;
  return s;
}

nep_status nep_get_fallback(nep_handle *h, int *flags, int64_t *count) {
  if (!h) return NEP_ERR_ARG;
  if (!h->fb_on) return fail(h, NEP_ERR_STATE, "no fallback model is set");
  if (!h->have_forces) return fail(h, NEP_ERR_STATE, "no force evaluation since the last state change");
  int hc = 0;
  NEP_CUDA(h, cudaMemcpyAsync(&hc, h->fb_count, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  if (flags && h->n > 0) {
    const size_t N = (size_t)h->n;
    if (h->io_i_elems < N) {
      dfree(h->io_i);
      NEP_CUDA(h, dalloc(h->io_i, N));
      h->io_i_elems = N;
    }
    NEP_CUDA(h, cudaMemsetAsync(h->io_i, 0, N * sizeof(int32_t), h->stream));
    {
      Scope sc(h, KC_OTHER, 1);
      NEP_CUDA(h, launch_fallback_flags(h->fb_list, h->fb_count, h->fb_cap, h->id, h->io_i, h->stream));
    }
    NEP_CUDA(h, cudaMemcpyAsync(flags, h->io_i, N * sizeof(int32_t), cudaMemcpyDefault, h->stream));
  }
  nep_status s = check_device_status(h);
  if (s != NEP_OK) return s;
  if (count) *count = std::min(hc, h->fb_cap);
  return NEP_OK;
}

}  // extern "C"
