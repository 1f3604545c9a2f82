/*
 * nep_oracle.c -- plain FP64 CPU oracle for NEP molecular dynamics of a single-species system.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the benchmark's CPU-baseline
 * leg may load this library.  It shares no code with the CUDA path: it is a slow, direct transcription
 * of the definitions, in double precision, with plain loops.
 *
 * What it computes (paper: "Trillion-atom molecular dynamics simulations with ab initio accuracy"):
 *   - site energy  U_i = sum_mu w1_mu tanh(sum_nu W0_{mu nu} q~_nu - b0_mu) - b1       (Section III.B eq.)
 *   - radial descriptors q_n = sum_j g_n(r_ij), g_n a linear combination of Chebyshev-of-the-
 *     first-kind basis functions times a smooth cutoff                                 (Section III.B)
 *   - angular descriptors: sums of radial functions times spherical harmonics, contracted over m
 *     to rotation invariants, with a shorter cutoff r_c < R_c                          (Section III.B, Fig. 1)
 *     The contraction is written in its plain two-neighbour form through the addition theorem:
 *       q_nl = sum_{j,k} g_n(r_ij) g_n(r_ik) P_l(cos theta_jik),  l = 1..4  (j = k included)
 *   - 4-body descriptor ("four-body L_max = 2", Section VI.A; the paper prints no formula):
 *       q4_n = tr(T_n^3),  T_n = sum_j g_n(r_ij) (u_ij u_ij^T - I/3)
 *   - a shifted-force Lennard-Jones Cu pair term (the workload's stability term)
 *   - forces F = -grad E by the explicit chain rule, the 3x3 virial, velocity-Verlet NVE.
 * Readings where the paper is silent (cosine cutoff, Chebyshev argument, 8 basis functions, l from 1,
 * the 4-body form, the descriptor order) are the ones listed in the design notes; each is a plain
 * formula below.
 *
 * Parity status: every routine here is pinned by the tests against finite differences, closed forms,
 * invariances, brute force, an independent spherical-harmonic route and an independent Wigner-3j
 * route.  Nothing here is pinned to a value printed in the paper (it prints no worked example).
 *
 * Units: Angstrom, eV, fs, amu.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

#define ACC_CONV 9.64853321233100e-3     /* 1 eV/(Angstrom amu) in Angstrom/fs^2 */
#define KE_CONV 103.642696562             /* 1 amu Angstrom^2/fs^2 in eV */
#define MAXK 16
#define MAXN 16
#define MAXL 4
#define MAXDES 128
#define MAXNEU 128

typedef struct {
    int nR, nA, kR, kA, lmax, nneu, ndes; /* nR = n_max_R + 1, nA = n_max_A + 1; ndes = nR + nA*lmax (+ nA) */
    int fourbody;                         /* 1: the 4-body descriptors q4_n are present (teacher), 0: absent */
    double rcR, rcA;
    const double *cR;    /* [nR][kR] */
    const double *cA;    /* [nA][kA] */
    const double *W0;    /* [nneu][ndes] */
    const double *b0;    /* [nneu] */
    const double *w1;    /* [nneu] */
    double b1;
    const double *qscale; /* [ndes] */
    double lj_eps, lj_sigma, lj_rc;
} onep;

/* ------------------------------------------------------------------------------------------------ */
/* Geometry                                                                                          */

static void min_image(double d[3], const double box[3]) {
    for (int a = 0; a < 3; ++a) d[a] -= box[a] * nearbyint(d[a] / box[a]);
}

/* Neighbour list (CSR): for each atom i, every j != i whose minimum-image distance is < rc. */
typedef struct {
    int n;
    int64_t *off;    /* [n+1] */
    int32_t *j;      /* [nnz] */
    double *d;       /* [nnz][3]  r_j - r_i (minimum image) */
} nlist;

static void nlist_free(nlist *L) {
    free(L->off); free(L->j); free(L->d);
    L->off = NULL; L->j = NULL; L->d = NULL;
}

typedef struct {
    int nc[3];
    int64_t *start;  /* [ncell+1] */
    int32_t *atoms;  /* [n] atoms sorted by cell, ascending index within a cell */
} cellgrid;

static int cell_coord(double x, double L, int nc) {
    double s = x / L;
    s -= floor(s);
    int c = (int)(s * nc);
    if (c >= nc) c = nc - 1;
    if (c < 0) c = 0;
    return c;
}

/* Cells of edge >= rc; returns 0 when some dimension has fewer than 3 cells (brute force then). */
static int cellgrid_build(cellgrid *G, int n, const double *x, const double box[3], double rc) {
    for (int a = 0; a < 3; ++a) {
        G->nc[a] = (int)floor(box[a] / rc);
        if (G->nc[a] < 3) return 0;
    }
    int64_t ncell = (int64_t)G->nc[0] * G->nc[1] * G->nc[2];
    G->start = (int64_t *)calloc((size_t)ncell + 1, sizeof(int64_t));
    G->atoms = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    int64_t *cid = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    for (int i = 0; i < n; ++i) {
        int cx = cell_coord(x[3 * i + 0], box[0], G->nc[0]);
        int cy = cell_coord(x[3 * i + 1], box[1], G->nc[1]);
        int cz = cell_coord(x[3 * i + 2], box[2], G->nc[2]);
        cid[i] = ((int64_t)cz * G->nc[1] + cy) * G->nc[0] + cx;
        G->start[cid[i] + 1]++;
    }
    for (int64_t c = 0; c < ncell; ++c) G->start[c + 1] += G->start[c];
    int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (size_t)ncell);
    memcpy(fill, G->start, sizeof(int64_t) * (size_t)ncell);
    for (int i = 0; i < n; ++i) G->atoms[fill[cid[i]]++] = i;   /* ascending i within each cell */
    free(fill);
    free(cid);
    return 1;
}

static void cellgrid_free(cellgrid *G) { free(G->start); free(G->atoms); G->start = NULL; G->atoms = NULL; }

static int cmp_int(const void *a, const void *b) {
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

/* Neighbours of one atom i (ascending j), using the grid when available, else all atoms.
 * Returns the count; fills js (and ds if non-NULL) up to cap entries. */
static int neighbors_of(int i, int n, const double *x, const double box[3], double rc,
                        const cellgrid *G, int use_grid, int32_t *js, int cap) {
    int cnt = 0;
    double rc2 = rc * rc;
    if (!use_grid) {
        for (int j = 0; j < n; ++j) {
            if (j == i) continue;
            double d[3] = {x[3 * j] - x[3 * i], x[3 * j + 1] - x[3 * i + 1], x[3 * j + 2] - x[3 * i + 2]};
            min_image(d, box);
            if (d[0] * d[0] + d[1] * d[1] + d[2] * d[2] < rc2) {
                if (cnt < cap) js[cnt] = j;
                cnt++;
            }
        }
        return cnt;
    }
    int c[3] = {cell_coord(x[3 * i], box[0], G->nc[0]), cell_coord(x[3 * i + 1], box[1], G->nc[1]),
                cell_coord(x[3 * i + 2], box[2], G->nc[2])};
    for (int dz = -1; dz <= 1; ++dz)
        for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
                int cx = (c[0] + dx + G->nc[0]) % G->nc[0];
                int cy = (c[1] + dy + G->nc[1]) % G->nc[1];
                int cz = (c[2] + dz + G->nc[2]) % G->nc[2];
                int64_t cc = ((int64_t)cz * G->nc[1] + cy) * G->nc[0] + cx;
                for (int64_t p = G->start[cc]; p < G->start[cc + 1]; ++p) {
                    int j = G->atoms[p];
                    if (j == i) continue;
                    double d[3] = {x[3 * j] - x[3 * i], x[3 * j + 1] - x[3 * i + 1], x[3 * j + 2] - x[3 * i + 2]};
                    min_image(d, box);
                    if (d[0] * d[0] + d[1] * d[1] + d[2] * d[2] < rc2) {
                        if (cnt < cap) js[cnt] = j;
                        cnt++;
                    }
                }
            }
    if (cnt <= cap) qsort(js, (size_t)cnt, sizeof(int32_t), cmp_int);
    return cnt;
}

#define NB_CAP 1024

/* Full CSR list for all atoms; use_cells = 0 forces the O(N^2) brute-force search. */
static int nlist_build(nlist *L, int n, const double *x, const double box[3], double rc, int use_cells) {
    cellgrid G = {{0, 0, 0}, NULL, NULL};
    int grid = use_cells ? cellgrid_build(&G, n, x, box, rc) : 0;
    L->n = n;
    L->off = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    int *cnt = (int *)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
    int bad = 0;
#pragma omp parallel for schedule(static) reduction(| : bad)
    for (int i = 0; i < n; ++i) {
        int32_t js[NB_CAP];
        cnt[i] = neighbors_of(i, n, x, box, rc, &G, grid, js, NB_CAP);
        if (cnt[i] > NB_CAP) bad |= 1;
    }
    if (bad) { free(cnt); if (grid) cellgrid_free(&G); return -1; }
    for (int i = 0; i < n; ++i) L->off[i + 1] = L->off[i] + cnt[i];
    int64_t nnz = L->off[n];
    L->j = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nnz > 0 ? nnz : 1));
    L->d = (double *)malloc(sizeof(double) * 3 * (size_t)(nnz > 0 ? nnz : 1));
#pragma omp parallel for schedule(static)
    for (int i = 0; i < n; ++i) {
        int32_t *js = L->j + L->off[i];
        neighbors_of(i, n, x, box, rc, &G, grid, js, cnt[i]);
        for (int p = 0; p < cnt[i]; ++p) {
            int j = js[p];
            double *d = L->d + 3 * (L->off[i] + p);
            d[0] = x[3 * j] - x[3 * i]; d[1] = x[3 * j + 1] - x[3 * i + 1]; d[2] = x[3 * j + 2] - x[3 * i + 2];
            min_image(d, box);
        }
    }
    free(cnt);
    if (grid) cellgrid_free(&G);
    return 0;
}

/* ------------------------------------------------------------------------------------------------ */
/* Radial functions: cosine cutoff, Chebyshev basis, linear combination                              */

/* f_c(r) = (1 + cos(pi r / rc)) / 2 for r < rc, else 0; and its derivative. */
static void cutoff_fn(double r, double rc, double *fc, double *dfc) {
    if (r >= rc) { *fc = 0.0; *dfc = 0.0; return; }
    *fc = 0.5 * (1.0 + cos(M_PI * r / rc));
    *dfc = -0.5 * M_PI / rc * sin(M_PI * r / rc);
}

/* f_k(r) = (T_k(x) + 1)/2 * f_c(r), x = 2 (r/rc - 1)^2 - 1, k = 0..K-1, with derivatives in r.
 * T_k by the three-term recurrence T_{k+1} = 2 x T_k - T_{k-1}. */
static void basis_fn(double r, double rc, int K, double *f, double *df) {
    double fc, dfc;
    cutoff_fn(r, rc, &fc, &dfc);
    double t = r / rc - 1.0;
    double x = 2.0 * t * t - 1.0;
    double dxdr = 4.0 * t / rc;
    double T[MAXK], dT[MAXK];
    T[0] = 1.0; dT[0] = 0.0;
    if (K > 1) { T[1] = x; dT[1] = 1.0; }
    for (int k = 2; k < K; ++k) {
        T[k] = 2.0 * x * T[k - 1] - T[k - 2];
        dT[k] = 2.0 * T[k - 1] + 2.0 * x * dT[k - 1] - dT[k - 2];
    }
    for (int k = 0; k < K; ++k) {
        f[k] = 0.5 * (T[k] + 1.0) * fc;
        df[k] = 0.5 * dT[k] * dxdr * fc + 0.5 * (T[k] + 1.0) * dfc;
    }
}

/* g_n(r) = sum_k c[n][k] f_k(r) for n = 0..nn-1, with derivatives. */
static void radial_fn(double r, double rc, int nn, int K, const double *c, double *g, double *dg) {
    double f[MAXK], df[MAXK];
    basis_fn(r, rc, K, f, df);
    for (int n = 0; n < nn; ++n) {
        double s = 0.0, ds = 0.0;
        for (int k = 0; k < K; ++k) { s += c[n * K + k] * f[k]; ds += c[n * K + k] * df[k]; }
        g[n] = s; dg[n] = ds;
    }
}

/* Legendre P_l(c) and P_l'(c), l = 0..lmax, Bonnet recurrence. */
static void legendre(double c, int lmax, double *P, double *dP) {
    P[0] = 1.0; dP[0] = 0.0;
    if (lmax >= 1) { P[1] = c; dP[1] = 1.0; }
    for (int l = 1; l < lmax; ++l) {
        P[l + 1] = ((2.0 * l + 1.0) * c * P[l] - l * P[l - 1]) / (l + 1.0);
        dP[l + 1] = c * dP[l] + (l + 1.0) * P[l];
    }
}

/* Shifted-force LJ: E(r) = phi(r) - phi(rc) - (r - rc) phi'(rc), phi = 4 eps [(s/r)^12 - (s/r)^6]. */
static void lj_pair(const onep *P, double r, double *e, double *de) {
    if (P->lj_eps == 0.0 || r >= P->lj_rc) { *e = 0.0; *de = 0.0; return; }
    double s = P->lj_sigma, eps = P->lj_eps, rc = P->lj_rc;
    double sr6 = pow(s / r, 6.0), sc6 = pow(s / rc, 6.0);
    double phi = 4.0 * eps * (sr6 * sr6 - sr6);
    double dphi = 4.0 * eps * (-12.0 * sr6 * sr6 + 6.0 * sr6) / r;
    double phic = 4.0 * eps * (sc6 * sc6 - sc6);
    double dphic = 4.0 * eps * (-12.0 * sc6 * sc6 + 6.0 * sc6) / rc;
    *e = phi - phic - (r - rc) * dphic;
    *de = dphi - dphic;
}

/* ------------------------------------------------------------------------------------------------ */
/* One atom: descriptors, site energy, and dU_i/dr_ij for each neighbour j                           */

/* Descriptor order: [q_n (n < nR) | q_nl, n-major, l = 1..lmax | q4_n (n < nA)]. */
static int idx_3b(const onep *P, int n, int l) { return P->nR + n * P->lmax + (l - 1); }
static int idx_4b(const onep *P, int n) { return P->nR + P->nA * P->lmax + n; }

/* Unscaled descriptors of an atom whose neighbours (within max cutoff) are given as vectors d[nn][3]. */
static void atom_descriptors(const onep *P, int nn, const double *d, double *q) {
    for (int v = 0; v < P->ndes; ++v) q[v] = 0.0;
    double g[MAXN], dg[MAXN];
    for (int a = 0; a < nn; ++a) {
        const double *da = d + 3 * a;
        double r = sqrt(da[0] * da[0] + da[1] * da[1] + da[2] * da[2]);
        if (r < P->rcR) {
            radial_fn(r, P->rcR, P->nR, P->kR, P->cR, g, dg);
            for (int n = 0; n < P->nR; ++n) q[n] += g[n];
        }
    }
    /* angular: two-neighbour sum with Legendre polynomials; 4-body: tr(T^3) */
    double T[MAXN][3][3];
    memset(T, 0, sizeof(T));
    for (int a = 0; a < nn; ++a) {
        const double *da = d + 3 * a;
        double ra = sqrt(da[0] * da[0] + da[1] * da[1] + da[2] * da[2]);
        if (ra >= P->rcA) continue;
        double ga[MAXN], dga[MAXN];
        radial_fn(ra, P->rcA, P->nA, P->kA, P->cA, ga, dga);
        double ua[3] = {da[0] / ra, da[1] / ra, da[2] / ra};
        for (int n = 0; n < P->nA; ++n)
            for (int s = 0; s < 3; ++s)
                for (int t = 0; t < 3; ++t) T[n][s][t] += ga[n] * (ua[s] * ua[t] - (s == t ? 1.0 / 3.0 : 0.0));
        for (int b = 0; b < nn; ++b) {
            const double *db = d + 3 * b;
            double rb = sqrt(db[0] * db[0] + db[1] * db[1] + db[2] * db[2]);
            if (rb >= P->rcA) continue;
            double gb[MAXN], dgb[MAXN];
            radial_fn(rb, P->rcA, P->nA, P->kA, P->cA, gb, dgb);
            double c = (da[0] * db[0] + da[1] * db[1] + da[2] * db[2]) / (ra * rb);
            double Pl[MAXL + 1], dPl[MAXL + 1];
            legendre(c, P->lmax, Pl, dPl);
            for (int n = 0; n < P->nA; ++n)
                for (int l = 1; l <= P->lmax; ++l) q[idx_3b(P, n, l)] += ga[n] * gb[n] * Pl[l];
        }
    }
    for (int n = 0; P->fourbody && n < P->nA; ++n) {
        double T2[3][3], tr3 = 0.0;
        for (int s = 0; s < 3; ++s)
            for (int t = 0; t < 3; ++t) {
                T2[s][t] = 0.0;
                for (int u = 0; u < 3; ++u) T2[s][t] += T[n][s][u] * T[n][u][t];
            }
        for (int s = 0; s < 3; ++s)
            for (int u = 0; u < 3; ++u) tr3 += T2[s][u] * T[n][u][s];
        q[idx_4b(P, n)] = tr3;
    }
}

/* Network: U = sum_mu w1 tanh(sum_nu W0 q~ - b0) - b1 with q~ = qscale * q; Fp = dU/dq (unscaled q). */
static double network(const onep *P, const double *q, double *Fp) {
    double qs[MAXDES];
    for (int v = 0; v < P->ndes; ++v) qs[v] = q[v] * P->qscale[v];
    double U = -P->b1;
    if (Fp) for (int v = 0; v < P->ndes; ++v) Fp[v] = 0.0;
    for (int mu = 0; mu < P->nneu; ++mu) {
        double z = -P->b0[mu];
        for (int v = 0; v < P->ndes; ++v) z += P->W0[mu * P->ndes + v] * qs[v];
        double h = tanh(z);
        U += P->w1[mu] * h;
        if (Fp) {
            double dz = P->w1[mu] * (1.0 - h * h);
            for (int v = 0; v < P->ndes; ++v) Fp[v] += dz * P->W0[mu * P->ndes + v] * P->qscale[v];
        }
    }
    return U;
}

/* Site energy (NEP + half of each LJ pair) and, if dU != NULL, dU_i/dr_ij per neighbour (dU[nn][3]),
 * including the LJ half-pair term.  q_out (unscaled descriptors) may be NULL. */
static double atom_site(const onep *P, int nn, const double *d, double *dU, double *q_out) {
    double q[MAXDES], Fp[MAXDES];
    atom_descriptors(P, nn, d, q);
    if (q_out) memcpy(q_out, q, sizeof(double) * (size_t)P->ndes);
    double U = network(P, q, dU ? Fp : NULL);
    double elj = 0.0;
    for (int a = 0; a < nn; ++a) {
        const double *da = d + 3 * a;
        double r = sqrt(da[0] * da[0] + da[1] * da[1] + da[2] * da[2]);
        double e, de;
        lj_pair(P, r, &e, &de);
        elj += 0.5 * e;
        if (dU) for (int s = 0; s < 3; ++s) dU[3 * a + s] = 0.5 * de * da[s] / r;
    }
    U += elj;
    if (!dU) return U;

    /* 4-body: M_n = 3 Fp_4n T_n^2 (gradient of tr(T^3) w.r.t. the symmetric T). */
    double T[MAXN][3][3];
    memset(T, 0, sizeof(T));
    for (int a = 0; a < nn; ++a) {
        const double *da = d + 3 * a;
        double ra = sqrt(da[0] * da[0] + da[1] * da[1] + da[2] * da[2]);
        if (ra >= P->rcA) continue;
        double ga[MAXN], dga[MAXN];
        radial_fn(ra, P->rcA, P->nA, P->kA, P->cA, ga, dga);
        double ua[3] = {da[0] / ra, da[1] / ra, da[2] / ra};
        for (int n = 0; n < P->nA; ++n)
            for (int s = 0; s < 3; ++s)
                for (int t = 0; t < 3; ++t) T[n][s][t] += ga[n] * (ua[s] * ua[t] - (s == t ? 1.0 / 3.0 : 0.0));
    }
    double M[MAXN][3][3];
    memset(M, 0, sizeof(M));
    for (int n = 0; P->fourbody && n < P->nA; ++n)
        for (int s = 0; s < 3; ++s)
            for (int t = 0; t < 3; ++t) {
                double v = 0.0;
                for (int u = 0; u < 3; ++u) v += T[n][s][u] * T[n][u][t];
                M[n][s][t] = 3.0 * Fp[idx_4b(P, n)] * v;
            }

    for (int a = 0; a < nn; ++a) {
        const double *da = d + 3 * a;
        double ra = sqrt(da[0] * da[0] + da[1] * da[1] + da[2] * da[2]);
        double ua[3] = {da[0] / ra, da[1] / ra, da[2] / ra};
        double *out = dU + 3 * a;
        /* radial: sum_n Fp_n g_n'(r) u */
        if (ra < P->rcR) {
            double g[MAXN], dg[MAXN];
            radial_fn(ra, P->rcR, P->nR, P->kR, P->cR, g, dg);
            double s = 0.0;
            for (int n = 0; n < P->nR; ++n) s += Fp[n] * dg[n];
            for (int t = 0; t < 3; ++t) out[t] += s * ua[t];
        }
        if (ra >= P->rcA) continue;
        double ga[MAXN], dga[MAXN];
        radial_fn(ra, P->rcA, P->nA, P->kA, P->cA, ga, dga);
        /* 3-body: dq_nl/dr_a = 2 sum_b g_n(b) [g_n'(a) P_l(c_ab) u_a + g_n(a) P_l'(c_ab) (u_b - c_ab u_a)/r_a] */
        double along_u = 0.0;          /* coefficient of u_a */
        double perp[3] = {0.0, 0.0, 0.0};
        for (int b = 0; b < nn; ++b) {
            const double *db = d + 3 * b;
            double rb = sqrt(db[0] * db[0] + db[1] * db[1] + db[2] * db[2]);
            if (rb >= P->rcA) continue;
            double gb[MAXN], dgb[MAXN];
            radial_fn(rb, P->rcA, P->nA, P->kA, P->cA, gb, dgb);
            double ub[3] = {db[0] / rb, db[1] / rb, db[2] / rb};
            double c = ua[0] * ub[0] + ua[1] * ub[1] + ua[2] * ub[2];
            double Pl[MAXL + 1], dPl[MAXL + 1];
            legendre(c, P->lmax, Pl, dPl);
            double cu = 0.0, cp = 0.0;
            for (int n = 0; n < P->nA; ++n)
                for (int l = 1; l <= P->lmax; ++l) {
                    double f = Fp[idx_3b(P, n, l)];
                    cu += 2.0 * f * dga[n] * gb[n] * Pl[l];
                    cp += 2.0 * f * ga[n] * gb[n] * dPl[l];
                }
            along_u += cu;
            for (int t = 0; t < 3; ++t) perp[t] += cp * (ub[t] - c * ua[t]) / ra;
        }
        for (int t = 0; t < 3; ++t) out[t] += along_u * ua[t] + perp[t];
        /* 4-body: sum_ab M_ab dT_ab/dr_a, T_ab = g (u_a u_b - delta/3) */
        for (int n = 0; P->fourbody && n < P->nA; ++n) {
            double Mu[3], uMu = 0.0, trM = M[n][0][0] + M[n][1][1] + M[n][2][2];
            for (int s = 0; s < 3; ++s) {
                Mu[s] = M[n][s][0] * ua[0] + M[n][s][1] * ua[1] + M[n][s][2] * ua[2];
                uMu += ua[s] * Mu[s];
            }
            for (int t = 0; t < 3; ++t)
                out[t] += dga[n] * ua[t] * (uMu - trM / 3.0) + 2.0 * ga[n] / ra * (Mu[t] - ua[t] * uMu);
        }
    }
    return U;
}

static double max_cut(const onep *P) {
    double rc = P->rcR;
    if (P->rcA > rc) rc = P->rcA;
    if (P->lj_eps != 0.0 && P->lj_rc > rc) rc = P->lj_rc;
    return rc;
}

/* ------------------------------------------------------------------------------------------------ */
/* Exported entry points                                                                             */

void oracle_set_threads(int t) {
#ifdef _OPENMP
    if (t > 0) omp_set_num_threads(t);
#else
    (void)t;
#endif
}

int oracle_get_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Neighbour counts per atom for distance < rc (strict). use_cells = 0: brute force O(N^2). */
int oracle_neighbor_counts(int n, const double *x, const double *box, double rc, int use_cells, int32_t *counts) {
    nlist L;
    if (nlist_build(&L, n, x, box, rc, use_cells) != 0) return -1;
    for (int i = 0; i < n; ++i) counts[i] = (int32_t)(L.off[i + 1] - L.off[i]);
    nlist_free(&L);
    return 0;
}

/* Neighbour lists (ascending j per row) in CSR form; offsets [n+1], list [nnz]. */
int oracle_neighbor_lists(int n, const double *x, const double *box, double rc, int use_cells, int64_t *offsets,
                          int32_t *list) {
    nlist L;
    if (nlist_build(&L, n, x, box, rc, use_cells) != 0) return -1;
    memcpy(offsets, L.off, sizeof(int64_t) * (size_t)(n + 1));
    memcpy(list, L.j, sizeof(int32_t) * (size_t)L.off[n]);
    nlist_free(&L);
    return 0;
}

/* Unscaled descriptors q[n][ndes]. */
int oracle_descriptors(const onep *P, int n, const double *x, const double *box, double *q) {
    nlist L;
    if (nlist_build(&L, n, x, box, max_cut(P), 1) != 0) return -1;
#pragma omp parallel for schedule(dynamic, 16)
    for (int i = 0; i < n; ++i) {
        int nn = (int)(L.off[i + 1] - L.off[i]);
        atom_descriptors(P, nn, L.d + 3 * L.off[i], q + (size_t)i * P->ndes);
    }
    nlist_free(&L);
    return 0;
}

/* Energy, site energies, forces and virial of the whole system.
 * W[a][b] = - sum_i sum_j r_ij[a] dU_i/dr_ij[b].  Any output pointer may be NULL. */
/* Energy, site energies, forces and virial.  Atom i's site energy comes from model Pb when flags[i] is
 * nonzero and from Pa otherwise (flags == NULL: Pa everywhere): E = sum_i U_i^(model of i), and the
 * forces are -dE/dr with each atom's own model differentiated (the per-atom teacher fallback). */
static int energy_forces_select(const onep *Pa, const onep *Pb, const int *flags, int n, const double *x,
                                const double *box, double *E, double *U, double *F, double *W) {
    double rc = max_cut(Pa);
    if (Pb && max_cut(Pb) > rc) rc = max_cut(Pb);
    nlist L;
    if (nlist_build(&L, n, x, box, rc, 1) != 0) return -1;
    int64_t nnz = L.off[n];
    double *dU = (double *)malloc(sizeof(double) * 3 * (size_t)(nnz > 0 ? nnz : 1));
    double *Us = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
#pragma omp parallel for schedule(dynamic, 16)
    for (int i = 0; i < n; ++i) {
        int nn = (int)(L.off[i + 1] - L.off[i]);
        const onep *P = (flags && flags[i]) ? Pb : Pa;
        Us[i] = atom_site(P, nn, L.d + 3 * L.off[i], dU + 3 * L.off[i], NULL);
    }
    /* serial, fixed-order accumulation */
    double Esum = 0.0, Wl[9] = {0};
    if (F) memset(F, 0, sizeof(double) * 3 * (size_t)n);
    for (int i = 0; i < n; ++i) {
        Esum += Us[i];
        for (int64_t p = L.off[i]; p < L.off[i + 1]; ++p) {
            int j = L.j[p];
            const double *g = dU + 3 * p, *d = L.d + 3 * p;
            if (F)
                for (int t = 0; t < 3; ++t) { F[3 * i + t] += g[t]; F[3 * j + t] -= g[t]; }
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) Wl[3 * a + b] -= d[a] * g[b];
        }
    }
    if (E) *E = Esum;
    if (U) memcpy(U, Us, sizeof(double) * (size_t)n);
    if (W) memcpy(W, Wl, sizeof(double) * 9);
    free(dU); free(Us);
    nlist_free(&L);
    return 0;
}

int oracle_energy_forces(const onep *P, int n, const double *x, const double *box, double *E, double *U,
                         double *F, double *W) {
    return energy_forces_select(P, NULL, NULL, n, x, box, E, U, F, W);
}

int oracle_energy_forces_select(const onep *Pa, const onep *Pb, const int *flags, int n, const double *x,
                                const double *box, double *E, double *U, double *F, double *W) {
    return energy_forces_select(Pa, Pb, flags, n, x, box, E, U, F, W);
}

/* Forces and site energies on a sample of atoms only, for large systems:
 * F_k = sum_{j in N(k)} dU_k/dr_kj - sum_{i : k in N(i)} dU_i/dr_ik. */
int oracle_forces_sampled(const onep *P, int n, const double *x, const double *box, int ns, const int64_t *idx,
                          double *F, double *U) {
    double rc = max_cut(P);
    cellgrid G = {{0, 0, 0}, NULL, NULL};
    int grid = cellgrid_build(&G, n, x, box, rc);
    int bad = 0;
#pragma omp parallel for schedule(dynamic, 4) reduction(| : bad)
    for (int s = 0; s < ns; ++s) {
        int k = (int)idx[s];
        int32_t jk[NB_CAP], ji[NB_CAP];
        double dk[3 * NB_CAP], di[3 * NB_CAP], gk[3 * NB_CAP], gi[3 * NB_CAP];
        int nk = neighbors_of(k, n, x, box, rc, &G, grid, jk, NB_CAP);
        if (nk > NB_CAP) { bad |= 1; continue; }
        for (int p = 0; p < nk; ++p) {
            int j = jk[p];
            for (int t = 0; t < 3; ++t) dk[3 * p + t] = x[3 * j + t] - x[3 * k + t];
            min_image(dk + 3 * p, box);
        }
        double Uk = atom_site(P, nk, dk, gk, NULL);
        double f[3] = {0, 0, 0};
        for (int p = 0; p < nk; ++p)
            for (int t = 0; t < 3; ++t) f[t] += gk[3 * p + t];
        for (int p = 0; p < nk; ++p) {
            int i = jk[p];
            int ni = neighbors_of(i, n, x, box, rc, &G, grid, ji, NB_CAP);
            if (ni > NB_CAP) { bad |= 1; break; }
            int pos = -1;
            for (int q = 0; q < ni; ++q) {
                int j = ji[q];
                for (int t = 0; t < 3; ++t) di[3 * q + t] = x[3 * j + t] - x[3 * i + t];
                min_image(di + 3 * q, box);
                if (j == k) pos = q;
            }
            atom_site(P, ni, di, gi, NULL);
            if (pos >= 0)
                for (int t = 0; t < 3; ++t) f[t] -= gi[3 * pos + t];
        }
        for (int t = 0; t < 3; ++t) F[3 * s + t] = f[t];
        if (U) U[s] = Uk;
    }
    if (grid) cellgrid_free(&G);
    return bad ? -1 : 0;
}

/* 3-body descriptors through real spherical harmonics (an independent route, for the addition-theorem
 * check): q_nl = 4 pi/(2l+1) sum_m s_nlm^2, s_nlm = sum_j g_n(r_ij) Y_lm(u_ij).  Output [n][nA*lmax]. */
static void real_ylm(const double u[3], double *Y /* 24 for l = 1..4 */) {
    double x = u[0], y = u[1], z = u[2];
    double pi = M_PI;
    int k = 0;
    /* l = 1 */
    double c1 = sqrt(3.0 / (4.0 * pi));
    Y[k++] = c1 * y; Y[k++] = c1 * z; Y[k++] = c1 * x;
    /* l = 2 */
    Y[k++] = 0.5 * sqrt(15.0 / pi) * x * y;
    Y[k++] = 0.5 * sqrt(15.0 / pi) * y * z;
    Y[k++] = 0.25 * sqrt(5.0 / pi) * (3.0 * z * z - 1.0);
    Y[k++] = 0.5 * sqrt(15.0 / pi) * x * z;
    Y[k++] = 0.25 * sqrt(15.0 / pi) * (x * x - y * y);
    /* l = 3 */
    Y[k++] = 0.25 * sqrt(35.0 / (2.0 * pi)) * y * (3.0 * x * x - y * y);
    Y[k++] = 0.5 * sqrt(105.0 / pi) * x * y * z;
    Y[k++] = 0.25 * sqrt(21.0 / (2.0 * pi)) * y * (5.0 * z * z - 1.0);
    Y[k++] = 0.25 * sqrt(7.0 / pi) * (5.0 * z * z * z - 3.0 * z);
    Y[k++] = 0.25 * sqrt(21.0 / (2.0 * pi)) * x * (5.0 * z * z - 1.0);
    Y[k++] = 0.25 * sqrt(105.0 / pi) * z * (x * x - y * y);
    Y[k++] = 0.25 * sqrt(35.0 / (2.0 * pi)) * x * (x * x - 3.0 * y * y);
    /* l = 4 */
    Y[k++] = 0.75 * sqrt(35.0 / pi) * x * y * (x * x - y * y);
    Y[k++] = 0.75 * sqrt(35.0 / (2.0 * pi)) * y * z * (3.0 * x * x - y * y);
    Y[k++] = 0.75 * sqrt(5.0 / pi) * x * y * (7.0 * z * z - 1.0);
    Y[k++] = 0.75 * sqrt(5.0 / (2.0 * pi)) * y * z * (7.0 * z * z - 3.0);
    Y[k++] = 3.0 / 16.0 * sqrt(1.0 / pi) * (35.0 * z * z * z * z - 30.0 * z * z + 3.0);
    Y[k++] = 0.75 * sqrt(5.0 / (2.0 * pi)) * x * z * (7.0 * z * z - 3.0);
    Y[k++] = 3.0 / 8.0 * sqrt(5.0 / pi) * (x * x - y * y) * (7.0 * z * z - 1.0);
    Y[k++] = 0.75 * sqrt(35.0 / (2.0 * pi)) * x * z * (x * x - 3.0 * y * y);
    Y[k++] = 3.0 / 16.0 * sqrt(35.0 / pi) * (x * x * (x * x - 3.0 * y * y) - y * y * (3.0 * x * x - y * y));
}

int oracle_q3b_ylm(const onep *P, int n, const double *x, const double *box, double *q3) {
    if (P->lmax != 4) return -2;
    nlist L;
    if (nlist_build(&L, n, x, box, max_cut(P), 1) != 0) return -1;
#pragma omp parallel for schedule(dynamic, 16)
    for (int i = 0; i < n; ++i) {
        double s[MAXN][24];
        memset(s, 0, sizeof(s));
        for (int64_t p = L.off[i]; p < L.off[i + 1]; ++p) {
            const double *d = L.d + 3 * p;
            double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
            if (r >= P->rcA) continue;
            double g[MAXN], dg[MAXN], Y[24], u[3] = {d[0] / r, d[1] / r, d[2] / r};
            radial_fn(r, P->rcA, P->nA, P->kA, P->cA, g, dg);
            real_ylm(u, Y);
            for (int nn = 0; nn < P->nA; ++nn)
                for (int c = 0; c < 24; ++c) s[nn][c] += g[nn] * Y[c];
        }
        for (int nn = 0; nn < P->nA; ++nn) {
            int c = 0;
            for (int l = 1; l <= 4; ++l) {
                double acc = 0.0;
                for (int m = 0; m < 2 * l + 1; ++m, ++c) acc += s[nn][c] * s[nn][c];
                q3[(size_t)i * P->nA * 4 + nn * 4 + (l - 1)] = 4.0 * M_PI / (2.0 * l + 1.0) * acc;
            }
        }
    }
    nlist_free(&L);
    return 0;
}

/* Radial functions g_n(r) and derivatives, for closed-form checks: which = 0 radial, 1 angular. */
void oracle_radial(const onep *P, int which, double r, double *g, double *dg) {
    if (which == 0) radial_fn(r, P->rcR, P->nR, P->kR, P->cR, g, dg);
    else radial_fn(r, P->rcA, P->nA, P->kA, P->cA, g, dg);
}

/* Shifted-force LJ pair energy and derivative, for closed-form checks. */
void oracle_lj(const onep *P, double r, double *e, double *de) { lj_pair(P, r, e, de); }

/* Site energy and dU/dr_ij of one atom from explicit neighbour vectors d[nn][3] (in any box). */
double oracle_atom_site(const onep *P, int nn, const double *d, double *dU, double *q) {
    return atom_site(P, nn, d, dU, q);
}

/* Velocity-Verlet NVE with masses m (amu) and dt (fs).  x, v are updated in place ([n][3], x wrapped
 * into the box).  thermo[(nsteps+1)][4] = (potential, kinetic, total, temperature) after each step,
 * row 0 the initial state.  Forces are recomputed from scratch (fresh neighbour search) every step. */
int oracle_md_nve(const onep *P, int n, double *x, double *v, const double *box, double mass, double dt, int nsteps,
                  double *thermo) {
    double *F = (double *)malloc(sizeof(double) * 3 * (size_t)(n > 0 ? n : 1));
    double E;
    const double kB = 8.617333262e-5;
    if (oracle_energy_forces(P, n, x, box, &E, NULL, F, NULL) != 0) { free(F); return -1; }
    for (int s = 0; s <= nsteps; ++s) {
        if (s > 0) {
            for (int i = 0; i < 3 * n; ++i) v[i] += 0.5 * dt * F[i] / mass * ACC_CONV;
            for (int i = 0; i < n; ++i)
                for (int t = 0; t < 3; ++t) {
                    double y = x[3 * i + t] + dt * v[3 * i + t];
                    y -= box[t] * floor(y / box[t]);
                    if (y >= box[t]) y -= box[t];
                    x[3 * i + t] = y;
                }
            if (oracle_energy_forces(P, n, x, box, &E, NULL, F, NULL) != 0) { free(F); return -1; }
            for (int i = 0; i < 3 * n; ++i) v[i] += 0.5 * dt * F[i] / mass * ACC_CONV;
        }
        if (thermo) {
            double ke = 0.0;
            for (int i = 0; i < 3 * n; ++i) ke += 0.5 * mass * v[i] * v[i] * KE_CONV;
            double* row = thermo + 4 * (size_t)s;
            row[0] = E; row[1] = ke; row[2] = E + ke;
            row[3] = n > 1 ? 2.0 * ke / ((3.0 * n - 3.0) * kB) : 0.0;
        }
    }
    free(F);
    return 0;
}
