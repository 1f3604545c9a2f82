/*
 * nep_student.h -- C ABI of the student-NEP training kernels (sm_103a).
 *
 * A student NEP (radial n_max 3, angular n_max 3, l_max 2, no 4-body term, 16 tanh neurons; the model
 * form of Section III.B) is fitted to energies and forces that the teacher NEP assigns to a set of
 * small periodic cells.  The training pass is split into hand-written kernels:
 *
 *   st_pairs        neighbour lists of every cell (brute force, minimum image; built once)
 *   st_basis        per-atom basis sums   Q_k = sum_j f^R_k(r_ij),  S_klm = sum_j f^A_k(r_ij) Y_lm(u_ij)
 *                   (built once: they depend on positions only)
 *   st_forward      per-atom descriptors q(theta; Q, S), network, site energy U_i and the adjoint row
 *                   G_i = [dU_i/ds_nlm | dU_i/dq_n]
 *   st_energy       E_s = sum of U_i over cell s
 *   st_force        F_i = sum_j D_ij from the adjoint rows of i and j (a gather: no atomics)
 *   st_jvp          directional derivatives of the basis sums along the force cotangent v = dL/dF:
 *                   dQ_k = sum_i v_i . dQ_k/dr_i, dS_klm likewise
 *   st_grad         dL/dtheta = sum_i [ gE_s(i) dU_i/dtheta - d(Fp_i . dq_i)/dtheta ]  (dq_i = the
 *                   directional derivative of q_i along v), reduced over atoms in a fixed order
 *   st_adam         one Adam update of the parameter vector
 *
 * Parameter vector theta (float32, ST_NPAR = 289 values, in this order):
 *   c_R [4][8] | c_A [4][8] | W0 [16][12] | b0 [16] | w1 [16] | b1
 * with descriptors q = [q_n (n < 4) | q_nl (n-major, l = 1, 2)] scaled by a fixed q_scale [12], and
 * U_i = sum_mu w1_mu tanh(sum_nu W0_mu,nu q_scale_nu q_nu - b0_mu) - b1.
 *
 * Data layout (all device memory, cells stored one after another):
 *   pos     float4 [n]: x, y, z (Angstrom, wrapped into the cell's box) and w = the cell index as
 *           int bits (__int_as_float).
 *   start   int [n_cells + 1]: first atom of each cell.
 *   boxes   float [n_cells][3]: orthorhombic box edges; each must be >= 2 * rc_R.
 *   nbr     int [cap][n], dvec float4 [cap][n] (neighbour-major): neighbour index j (global) and
 *           d_ij = r_j - r_i (minimum image); nnum int [n]: row lengths.  All j with r_ij < rc_R.
 *   Q       float [n][8], S float [n][64] (index k * 8 + lm), dQ, dS likewise.
 *   G       float [n][40]: dU_i/ds_nlm (index n * 8 + lm) then dU_i/dq_n (4) and padding.
 *   F, v    float [n][3].
 * Kernels that take [a0, a1) work on that atom range (a mini-batch of whole cells); neighbour indices
 * stay global.  Every call is asynchronous on `stream` (a cudaStream_t, NULL = default stream) and
 * returns a CUDA error code (0 = success) for the launch; device-detected conditions go to `status`
 * (bit 1: a neighbour row longer than cap).  The caller owns every buffer.
 */
#ifndef NEP_STUDENT_H
#define NEP_STUDENT_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ST_NPAR 289
#define ST_NDES 12
#define ST_GS 40

/* Cutoffs of the student (the teacher's: rc_R radial, rc_A angular). */
typedef struct {
    float rc_R, rc_A;
} st_cutoffs;

/* Neighbour lists of all cells: for each atom, every other atom of its cell with minimum-image
 * distance < rc_R, in ascending index order.  Rows longer than cap are truncated and set status bit 1. */
int st_pairs(int n, const float *pos, const int *start, const float *boxes, st_cutoffs rc, int cap,
             int *nbr, float *dvec, int *nnum, int *status, void *stream);

/* Basis sums Q, S of atoms [a0, a1) (Chebyshev basis times cosine cutoff; normalised real harmonics
 * l = 1, 2 with sum_m Y_lm(u) Y_lm(v) = P_l(u . v)). */
int st_basis(int a0, int a1, int n, int cap, const int *nbr, const float *dvec, const int *nnum, st_cutoffs rc,
             float *Q, float *S, void *stream);

/* Descriptors, network, site energies U [n] and adjoint rows G [n][40] of atoms [a0, a1).
 * q_out (may be NULL): the unscaled descriptors [n][12]. */
int st_forward(int a0, int a1, const float *theta, const float *q_scale, const float *Q, const float *S,
               float *U, float *G, float *q_out, void *stream);

/* E [s] = sum of U over the atoms of cell s, for cells [s0, s1) (float64 accumulation). */
int st_energy(int s0, int s1, const int *start, const float *U, double *E, void *stream);

/* Forces F [n][3] of atoms [a0, a1) from the adjoint rows G of the atoms and their neighbours. */
int st_force(int a0, int a1, int n, int cap, const int *nbr, const float *dvec, const int *nnum, st_cutoffs rc,
             const float *theta, const float *G, float *F, void *stream);

/* Directional derivatives dQ, dS of the basis sums of atoms [a0, a1) along v [n][3]. */
int st_jvp(int a0, int a1, int n, int cap, const int *nbr, const float *dvec, const int *nnum, st_cutoffs rc,
           const float *v, float *dQ, float *dS, void *stream);

/* Scratch floats st_grad needs for atoms [a0, a1). */
int64_t st_grad_scratch(int a0, int a1);

/* grad [ST_NPAR] = dL/dtheta for the atoms [a0, a1), given gE [n_cells] = dL/dE_s (indexed by the cell
 * index in pos.w), the basis sums and their directional derivatives along v = dL/dF.  Per-block partial
 * sums go to scratch (st_grad_scratch floats); the final sum over blocks runs in a fixed order in
 * float64, so the gradient is bitwise reproducible. */
int st_grad(int a0, int a1, const float *theta, const float *q_scale, const float *pos, const float *Q,
            const float *S, const float *dQ, const float *dS, const double *gE, float *scratch, float *grad,
            void *stream);

/* One Adam step on theta [npar] with moment buffers m, v (float32), step count t >= 1. */
int st_adam(int npar, float *theta, const float *grad, float *m, float *v, float lr, float beta1, float beta2,
            float eps, int t, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* NEP_STUDENT_H */
