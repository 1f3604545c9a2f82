/*
 * nep_gb300.h -- C ABI of the GB300 (sm_103a) NEP molecular-dynamics library.
 *
 * The library evaluates the Neuroevolution Potential (NEP) of one atomic species and integrates
 * Newton's equations with velocity Verlet, all on one GPU:
 *   cell-list neighbour build -> radial + angular (3-body, 4-body) descriptors -> single-hidden-layer
 *   tanh network giving site energies U_i -> chain-rule forces and virial -> velocity Verlet.
 * The method follows "Trillion-atom molecular dynamics simulations with ab initio accuracy"
 * (NEP energy formula and descriptor definitions in Section III.B and Fig. 1; model hyper-
 * parameters and MD protocol in Section VI.A; the five evaluation stages in Section V.B and Table 2).
 *
 * Conventions shared by every entry point
 *   - Units: Angstrom, eV, fs, amu.  Forces eV/Angstrom, virial eV.
 *   - Array pointers may be host or device memory; the library detects which with
 *     cudaPointerGetAttributes.  Host pointers make the call synchronous.  Device pointers are used
 *     on the handle's stream; the call returns once the work is enqueued unless it also returns a
 *     host scalar.
 *   - Per-atom arrays are in the caller's atom order ("original order", index 0..n-1 as passed to
 *     nep_set_state), row-major [n][3] for vectors.  Internally atoms are kept sorted by cell; the
 *     library permutes back on output.
 *   - The caller owns every pointer it passes; pointers are read or written only during the call.
 *     The library owns all of its internal device memory (allocated by nep_set_state, released by
 *     nep_destroy).
 *   - Errors are returned as nep_status; nep_last_error(h) gives a message.  No entry point exits,
 *     traps or spins without a bound.  Conditions detected on the device (neighbour-list overflow,
 *     non-finite values) are reported through a status word read back by the host.
 *   - Orthorhombic periodic box only; every edge must be >= 2 * (rc_R + skin).
 *   - At most NEP_MAX_ATOMS atoms (a neighbour entry packs a 27-bit atom index with a 5-bit
 *     periodic-shift code).
 */
#ifndef NEP_GB300_H
#define NEP_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define NEP_MAX_ATOMS 134217727LL   /* 2^27 - 1 */
#define NEP_N_KERNEL_CLASSES 9

typedef enum {
    NEP_OK = 0,
    NEP_ERR_ARG = 1,              /* invalid argument (NULL handle, bad size, bad model shape) */
    NEP_ERR_CUDA = 2,             /* CUDA runtime error; message via nep_last_error */
    NEP_ERR_NEIGH_OVERFLOW = 3,   /* an atom had more neighbours within rc_R + skin than max_neighbors */
    NEP_ERR_BOX_TOO_SMALL = 4,    /* some box edge < 2 * (rc_R + skin) */
    NEP_ERR_NAN = 5,              /* non-finite position or force detected */
    NEP_ERR_TIMEOUT = 6,          /* a bounded wait (host on the stream, or a kernel on the tensor cores) expired */
    NEP_ERR_STATE = 7,            /* call out of order (e.g. nep_compute before nep_set_state) */
    NEP_ERR_UNSUPPORTED = 8,      /* model shape without a compiled kernel instance */
    NEP_ERR_OOM = 9,              /* device allocation failed */
    NEP_ERR_FALLBACK_OVERFLOW = 10 /* more atoms flagged for the fallback model than its list holds */
} nep_status;

/* Arithmetic of the force evaluation.  NEP_FP32: everything in float32 (float64 integration and sums).
 * NEP_MIX_BF16 / NEP_MIX_FP16: descriptors in float32; the network GEMMs (forward and gradient) on the
 * tensor cores with bf16 / f16 operands and float32 accumulation (the paper's mixed precision, Section
 * V.B Optimization 4 and Section VII.A).  The teacher keeps its per-atom adjoint rows in float32 (in
 * tensor memory) and takes the network's tanh from the special-function unit (relative error about
 * 2^-11, below that of the 16-bit GEMM inputs); the student's mixed form stores its adjoint rows in
 * float16 between its two kernels. */
enum { NEP_FP32 = 0, NEP_MIX_BF16 = 1, NEP_MIX_FP16 = 2 };

/* Model and run parameters.  Host memory; copied by nep_create, the caller keeps ownership.
 * Descriptor order (n_des = (n_max_R+1) + (n_max_A+1)*l_max_3b + (n_max_A+1) if l_max_4b == 2):
 *   [ q_n, n = 0..n_max_R | q_nl, n-major, l = 1..l_max_3b | q4_n, n = 0..n_max_A ].
 * Radial functions g_n(r) = sum_k c[n][k] f_k(r), f_k = (T_k(x) + 1)/2 * f_c(r),
 * x = 2 (r/rc - 1)^2 - 1, f_c(r) = (1 + cos(pi r/rc))/2 (Section III.B: Chebyshev basis of the
 * first kind times a smooth cutoff).  Angular: q_nl = sum_{j,k} g_n(r_ij) g_n(r_ik) P_l(cos theta_jik)
 * (the m-contraction of spherical-harmonic sums, Section III.B); 4-body q4_n = tr(T_n^3),
 * T_n = sum_j g_n(r_ij)(u_ij u_ij^T - I/3) (the "four-body L_max = 2" of Section VI.A).
 * Site energy U_i = sum_mu w1[mu] tanh(sum_nu W0[mu][nu] q_nu * q_scale[nu] - b0[mu]) - b1
 * (Section III.B equation), plus half of each shifted-force Lennard-Jones pair energy. */
typedef struct nep_params {
    int n_max_R, n_max_A;     /* compiled instance: 4, 4 */
    int basis_R, basis_A;     /* compiled instance: 8, 8 (number of Chebyshev basis functions) */
    int l_max_3b, l_max_4b;   /* compiled instance: 4, 2 */
    int n_neu;                /* compiled instance: 30 */
    float rc_R, rc_A;         /* radial and angular cutoffs, rc_A <= rc_R */
    const float *c_R;         /* [n_max_R+1][basis_R] */
    const float *c_A;         /* [n_max_A+1][basis_A] */
    const float *W0;          /* [n_neu][n_des] */
    const float *b0;          /* [n_neu] */
    const float *w1;          /* [n_neu] */
    float b1;
    const float *q_scale;     /* [n_des] */
    float lj_eps, lj_sigma, lj_rc;   /* shifted-force LJ pair term; lj_eps = 0 disables it; lj_rc <= rc_R */
    double mass_amu;
    float skin;               /* neighbour-list skin (Angstrom); list radius rc_R + skin */
    int precision;            /* NEP_FP32, NEP_MIX_BF16 or NEP_MIX_FP16 */
    int max_neighbors;        /* per-atom list capacity, 1..128; 0 selects 128 */
    int rebuild_every;        /* MD: rebuild at least every k steps (0: only when an atom moved > skin/2) */
} nep_params;

typedef struct nep_handle nep_handle;

/* Create a handle.  cuda_stream: a cudaStream_t to enqueue on, or NULL for a library-owned stream.
 * Validates the model shape (NEP_ERR_UNSUPPORTED if no kernel instance matches). */
nep_status nep_create(const nep_params *params, void *cuda_stream, nep_handle **out);

/* Release every device buffer and the handle.  NULL is accepted. */
nep_status nep_destroy(nep_handle *h);

/* Load a configuration.  x: [n][3] positions (need not be wrapped), v: [n][3] velocities in
 * Angstrom/fs or NULL for zero, box: host [3] edge lengths.  Allocates device buffers for n atoms
 * (kept when n and the box are unchanged since the last call) and invalidates the forces.  When n and
 * the box are unchanged and a neighbour list exists, the list and the internal cell order are kept:
 * the next evaluation rebuilds the list only if an atom moved more than skin/2 from the positions it
 * was built for (the same test as between MD steps; positions are taken at their periodic image
 * nearest the previous ones, and a coordinate within 8 eps L of the current one, eps the float64
 * machine epsilon and L the box edge -- the rounding of the wrap applied by nep_get_state -- is the
 * current one).  Otherwise the neighbour list is invalidated.  n = 0 is accepted (every
 * later call is a no-op).  x and v may be host or device memory; when the list is kept, device and
 * page-locked host arrays are read by the GPU directly (other host arrays are copied first).  Returns
 * after the upload has completed, so the caller may reuse the arrays. */
nep_status nep_set_state(nep_handle *h, int64_t n, const double *x, const double *v, const double *box);

/* Build the cell list and the neighbour list (cutoff rc_R + skin) for the current positions:
 * atoms are sorted by cell, then each atom's list holds every j with |r_ij| < rc_R + skin (minimum
 * image), grouped by distance band -- r < rc_A, r < rc_A + skin, r < rc_R, r < rc_R + skin -- in a
 * fixed cell-stencil order inside each band; its prefix with |r_ij| < rc_A + skin is the angular list. */
nep_status nep_build_neighbors(nep_handle *h);

/* Energy, forces and virial of the current positions (builds the neighbour list first if needed).
 * E: host scalar, total potential energy; F: [n][3] (host or device, float64, original order);
 * virial: host [9], W[a][b] = -sum_i sum_j r_ij[a] dU_i/dr_ij[b].  Any of the three may be NULL. */
nep_status nep_compute(nep_handle *h, double *E, double *F, double *virial);

/* n_steps velocity-Verlet NVE steps of dt_fs each: half kick, drift, neighbour rebuild when an atom
 * moved more than skin/2 since the last build (or every rebuild_every steps), forces, half kick.
 * Positions/velocities are integrated in float64; forces are evaluated in float32 with float64
 * energy and virial sums.  Returns after enqueueing; the status word is checked at the end. */
nep_status md_verlet_step(nep_handle *h, double dt_fs, int n_steps);

/* Copy positions (wrapped into the box) and velocities out, [n][3] each, original order; either may
 * be NULL.  Device arrays and page-locked host arrays are written by the GPU directly (16-byte stores
 * of whole rows when the array is 16-byte aligned), pageable host arrays through a device staging
 * buffer and copies (the two arrays' copies run concurrently); returns when the data is in place. */
nep_status nep_get_state(nep_handle *h, double *x, double *v);

/* Thermodynamics of the last force evaluation: out = {potential energy, kinetic energy,
 * temperature (3N-3 dof), pressure (eV/Angstrom^3), W_xx, W_yy, W_zz, rebuild count}. */
nep_status nep_get_thermo(nep_handle *h, double out[8]);

/* Neighbour lists in original atom ids: counts[n], n_ang[n] (entries with |r_ij| < rc_A + skin),
 * n_own[n] (length of the owned part: each unordered pair is owned by exactly one of its two atoms)
 * and list[n][cap] (row i holds the ids of i's neighbours in list order -- owned part first, each part
 * grouped by distance band -- and -1 past the count). */
nep_status nep_get_neighbors(nep_handle *h, int32_t *counts, int32_t *n_ang, int32_t *n_own, int32_t *list, int cap);

/* Unscaled descriptors of the last evaluation, [n][n_des] float32, original order. */
nep_status nep_get_descriptors(nep_handle *h, float *q);

/* Site energies (NEP plus half of each LJ pair) of the last evaluation, [n] float64, original order. */
nep_status nep_get_site_energies(nep_handle *h, double *U);

/* Per-kernel-class CUDA-event timing of later calls: enable = 1 turns it on (and resets the sums). */
nep_status nep_set_timing(nep_handle *h, int enable);

/* Accumulated milliseconds and launch counts per kernel class since timing was enabled:
 * classes 0 drift, 1 cell sort, 2 neighbour list, 3 descriptors+network, 4 forces, 5 kick,
 * 6 reductions, 7 un-permute/other, 8 fallback model (descriptors, network and forces of the flagged
 * atoms, nep_set_fallback). */
nep_status nep_get_timing(nep_handle *h, double ms[NEP_N_KERNEL_CLASSES], int64_t launches[NEP_N_KERNEL_CLASSES]);

/* Counters since nep_set_state: out = {radial pairs (r < rc_R) and angular pairs (r < rc_A) seen by the
 * descriptor kernel, force evaluations, neighbour rebuilds, MD steps, kernel launches enqueued by the
 * library, list entries and pairs inside the largest cutoff seen by the descriptor kernel, then the
 * same four counts for the rows walked by the force kernel (whole rows for the float32 teacher, the
 * owned half of each row otherwise): list entries, pairs inside the largest cutoff, radial pairs,
 * angular pairs, then the atom evaluations done by the fallback model (nep_set_fallback)}.  Pair and
 * atom counts sum over evaluations.  List entries count the entries walked: the far band of each row
 * part (entries built beyond rc_R + 0.4 skin) is left out while no atom has moved more than
 * (0.4 skin - 0.02 A)/2 since the last rebuild, since none of its pairs can then be inside rc_R. */
nep_status nep_get_counters(nep_handle *h, int64_t out[13]);

/* Per-atom fallback from a student-shaped model (n_max 3/3, l_max 2, no 4-body, 16 neurons) to a
 * teacher-shaped model (the handle's model must be the student).  Every force evaluation flags each atom
 * whose scaled descriptors q~_nu = q_scale_nu q_nu leave [q_lo_nu - margin w_nu, q_hi_nu + margin w_nu]
 * (w = q_hi - q_lo; q_lo/q_hi: 12 floats, host memory, the student's training range) and takes that
 * atom's site energy from the teacher: E = sum_i U_i^(model of i), F = -grad E with each atom's own model
 * differentiated (the LJ term is shared and evaluated once).  The teacher runs in float32 on the
 * flagged atoms only (compacted list).  max_fraction (0 < f <= 1; 0 = 1/16) sizes the flagged-atom list
 * as a fraction of n; more flagged atoms in one evaluation returns NEP_ERR_FALLBACK_OVERFLOW.
 * teacher == NULL switches the fallback off.  The teacher's rc_R must equal the student's.  Parameters
 * are copied; the caller keeps ownership.  Because the flags can change from step to step, the energy is
 * not conserved across a switch (reported, not corrected). */
nep_status nep_set_fallback(nep_handle *h, const nep_params *teacher, const float *q_lo, const float *q_hi,
                            float margin, double max_fraction);

/* After a force evaluation: flags [n] (host or device, may be NULL; original order; 1 = teacher) and the
 * number of flagged atoms of the last evaluation.  NEP_ERR_STATE without a fallback or before the first
 * evaluation of the current state. */
nep_status nep_get_fallback(nep_handle *h, int *flags, int64_t *count);

/* Kernel variants kept for ablation (plain float32 teacher path only):
 *   NEP_VARIANT_FLOAT_SCATTER  the force kernel with float atomicAdd scatter (Section V.B, Optimization 1)
 *                              instead of 64-bit fixed-point integer atomics: the result depends on the
 *                              order in which additions arrive, so repeated runs may differ in the last bits;
 *   NEP_VARIANT_TILE1 / TILE3  the descriptor kernel with channel tiling (Algorithm 1): the angular
 *                              neighbours are walked once per tile of 1 or 3 channels, with s_nlm passed
 *                              through a global array (the paper's sum_fxyz) instead of registers;
 *   NEP_VARIANT_HALF_LIST      the force kernel over the owned half of each row: every unordered pair once,
 *                              with the adjoint rows of both atoms (the neighbour's gathered), instead of
 *                              every ordered pair with the own row only;
 *   NEP_VARIANT_SEPARATE_DESCRIPTOR / _FORCE  the descriptor kernel and the full-row force kernel as two
 *                              launches with the adjoint rows through device memory, instead of the fused
 *                              kernel (*ms = the named kernel's time; the other variants' force and
 *                              descriptor kernels are these, with one part changed).
 * The float-scatter and half-list variants run after the separate descriptor kernel.
 * One force evaluation on the current state with the variant; *ms = the variant kernel's time (CUDA
 * events), F (may be NULL; host or device; [n][3], caller's order) = the forces it produced.  The
 * handle's own results are recomputed on the next request. */
enum {
  NEP_VARIANT_FLOAT_SCATTER = 1,
  NEP_VARIANT_TILE1 = 2,
  NEP_VARIANT_TILE3 = 3,
  NEP_VARIANT_HALF_LIST = 4,
  NEP_VARIANT_SEPARATE_DESCRIPTOR = 5,
  NEP_VARIANT_SEPARATE_FORCE = 6,
  NEP_VARIANT_CPB1 = 7,
  NEP_VARIANT_CPB2 = 8,
  NEP_VARIANT_CPB3 = 9,
  NEP_VARIANT_CPB_AUTO = 10
};
/* NEP_VARIANT_CPB1/2/3/AUTO: the force kernel in the paper's thread-per-neighbour form with its adaptive
 * centres-per-block scheduling (Section V.B, Optimization 3): a 32-lane warp takes 1, 2 or 3 centre
 * atoms at a time, its lanes split into as many groups; a group strides over its centre's row (radial
 * and LJ pairs) and then over the centre's angular pairs (the three-body backward) with the adjoint row
 * in shared memory.  AUTO picks CPB from the 90th percentile of the angular pair count (nep_angular_p90).
 * Run after the separate descriptor kernel, like the other force variants. */
nep_status nep_run_variant(nep_handle *h, int variant, double *ms, double *F);

/* Diagnostic of the CPB variants: the 90th percentile p90 of the per-atom angular pair count (r < rc_A)
 * of the current state, and the centres per warp the paper's rule gives for 32-lane warps (its 64-lane
 * thresholds halved): 3 if p90 <= 10, 2 if p90 < 24, else 1.  Synchronous; host outputs. */
nep_status nep_angular_p90(nep_handle *h, int *p90, int *cpb);

/* Upper limits of nep_compute_noalloc: the size of its fixed scratch array. */
#define NEP_NOALLOC_MAX_ATOMS 8192
#define NEP_NOALLOC_MAX_CELLS 32768

/* One energy/force/virial evaluation that allocates no memory (no paper counterpart: it is a
 * deployment aid).  It is meant for callers that cannot allocate GPU memory where they need forces -- a
 * plugin that must stay inside a host program's memory pool or allocation budget, or an embedded
 * runtime that forbids cudaMalloc after start-up -- and so cannot create a handle (nep_create and
 * nep_set_state allocate).  It evaluates the float32 teacher shape only (params as for nep_create with
 * precision NEP_FP32; another shape or precision returns NEP_ERR_UNSUPPORTED; max_neighbors and
 * rebuild_every are ignored, the list capacity is 128), on up to NEP_NOALLOC_MAX_ATOMS atoms in boxes of
 * up to NEP_NOALLOC_MAX_CELLS neighbour cells, with the separate descriptor and full-row force kernels
 * (not the fused kernel of nep_compute, whose pair records would need more scratch), and keeps every
 * intermediate buffer in one fixed file-scope device array (about 11 MB, held by every GPU that loads
 * the library until the process exits); it calls no cudaMalloc, cudaFree or other allocating routine.
 * x: [n][3] positions, E: scalar, F: [n][3] float64 in the caller's order, virial: [9]; each pointer
 * host or device, E/F/virial may be NULL.  cuda_stream: the stream to run on (NULL = the legacy default
 * stream).  The call waits for its own work (polling the stream, 900 s limit) and reads its status and
 * host-side results with synchronous copies, so it must not run while any stream of the process is
 * being captured into a CUDA graph.  Sizes above the limits return NEP_ERR_ARG before any GPU work.  The
 * first call on each device looks up the array's device address.  All calls share the array and it
 * keeps the last call's contents (the call clears what must start at zero); calls that overlap on the
 * GPU race on it: do not run two at once.  After NEP_ERR_TIMEOUT the timed-out work may still be running
 * on the array: the next call returns NEP_ERR_STATE until that stream is idle. */
nep_status nep_compute_noalloc(const nep_params *params, int64_t n, const double *x, const double *box, double *E,
                               double *F, double *virial, void *cuda_stream);

/* Last error message of the handle (never NULL). */
const char *nep_last_error(nep_handle *h);

/* Self-test of the failure path of the tensor-core kernels' bounded waits: one block waits on an
 * mbarrier that nothing arrives on, with the same helper and at most `polls` polls (1 .. 2^24), and
 * *timed_out = 1 when the wait ran out and the kernel ended normally (0 would mean the barrier
 * completed).  Synchronous; uses the current device; no handle. */
nep_status nep_selftest_bounded_wait(int64_t polls, int *timed_out);

/* FP32 throughput microbenchmark of the current device (a measurement aid with no paper counterpart;
 * it gives the denominator of the FP32 roofline the force kernels are reported against).  Every SM is
 * filled with resident blocks whose threads run 16 independent multiply-add chains: scalar FMAs
 * (packed = 0), packed float2 FMAs, two per instruction (packed = 1), or, for comparison with the
 * 16-bit rate of the CUDA cores, packed half2 FMAs (packed = 2; any other value: NEP_ERR_ARG).  Each launch is sized to about
 * launch_ms (0 < launch_ms <= 1000) and timed with CUDA events on cuda_stream (NULL = legacy default
 * stream); after a calibration, `reps` launches (1..10000) are timed.  Outputs (host, may be NULL):
 * *best_tflops and *median_tflops = FLOP/s over the timed launches (FMA = 2 FLOP), in 10^12;
 * *fma_per_clock_sm = FMAs per SM clock cycle of the last launch (from clock64 in every block), which
 * does not depend on the clock frequency; *sm_count = multiprocessor count read from the device.
 * Synchronous; allocates and frees small buffers; NEP_ERR_ARG for bad sizes, NEP_ERR_CUDA / NEP_ERR_OOM
 * on runtime failures. */
nep_status nep_fp32_peak(int packed, double launch_ms, int reps, void *cuda_stream, double *best_tflops,
                         double *median_tflops, double *fma_per_clock_sm, int *sm_count);

/* Name of a status code (never NULL). */
const char *nep_status_string(nep_status s);

#ifdef __cplusplus
}
#endif

#endif /* NEP_GB300_H */
