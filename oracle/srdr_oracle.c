/*
 * srdr_oracle.c — plain FP64 CPU oracle of the splitting random-choice dynamic
 * relaxation method for TL-SPH (Zhu, Zhang & Hu, arXiv 2103.08932).
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the tests, the smoke check and the
 * benchmark's CPU-baseline leg, never by the product path.  It shares no code
 * with the CUDA library.
 *
 * Build: gcc -O2 -std=c11 -ffp-contract=off -fPIC -shared -lm
 *
 * Readings of points where the paper is silent, garbled or self-contradictory
 * (each one is repeated where it is used):
 *   R1  E = 2G(1+nu) (the printed 2G(1+2nu) is a typo; Eq. modulus-relation).
 *   R2  2D is plane strain: the 3D Lame constants act on the 2x2 tensors.
 *   R3  Wendland C2 normalisation alpha_2 = 7/(4 pi h^2), alpha_3 = 21/(16 pi h^3),
 *       support q = r/h < 2; cut-off r_c = 2h = cell edge.
 *   R4  Neo-Hookean S = dW/dE = mu (I - C^-1) + lambda ln J C^-1, C = F^T F.
 *   R5  Second position half-step uses v^{n+1}; dF/dt at n+1/2 uses v^{n+1}.
 *   R6  Damping S_d sits after the velocity update and before the second
 *       half-step (Lie-Trotter on v, Eq. operator-splitting).
 *   R7  Each of the forward and backward sweeps uses dt_loc = dt/2 in B_j.
 *   R8  Random choice: damp iff phi < alpha, with eta~ = eta/alpha (the printed
 *       "alpha < phi" would damp 80 % of steps, contradicting Sec. 3.3's "small
 *       fraction" and the 20 % cost of Table 1).  One draw per time step,
 *       phi = Philox4x64-10(counter = (step,0,0,0), key = (seed,0)) word 0,
 *       top 53 bits / 2^53.
 *   R9  Sweep order: colours 0..3^d-1 (colour = sum_a (i_a mod 3) 3^a), cells of
 *       a colour in ascending id, particles of a cell in ascending id; the
 *       backward sweep is the exact reverse.
 *   R10 The corrector (Eq. second-step) uses the pre-update v_j^n on the right.
 *   R11 Constrained particles are neighbours in every sum, are processed by
 *       S_d like any particle, and get v = 0 (u fixed) after S_m and after S_d.
 *   R12 dt fixed per body: Eq. time-step-criterion with |v|max = 0 and
 *       |a|max = the largest body-force magnitude, min'd with the implicit
 *       viscous limit 50 h^2 / (nu~ D), nu~ = eta / (alpha rho0).
 *   R13 Neighbour order within a row: ascending particle id (the pairwise
 *       scheme's pair updates, Sec. 3.2, depend on it; in the particle
 *       scheme it only orders the roundings of the sums).
 *   R14 Cell index ix = floor((x - x0)/r_c) in FP64, x0 = min_i x_i, clamped
 *       to [0, n_x - 1] with n_x = floor((max - min)/r_c) + 1.
 *   R15 Convergence (the paper runs to a fixed time): a relaxation stops after
 *       the first step with KE < tol KE_max, KE_max the largest KE so far.
 *   R16 Explicit-viscosity comparator (ORA_DAMP_EXPLICIT, Sec. 3): the term of
 *       Eq. damping-term with eta itself (no random choice) is evaluated at
 *       v^n and added to the acceleration of S_m; dt is min'd with the
 *       explicit limit 0.5 h^2 / (nu D), nu = eta / rho0 (Eq.
 *       viscous-criteria-o).
 *   R17 Twisting body force (Sec. 4.2): the printed g = (0, y gamma, z gamma)
 *       is radial, at odds with the "rotational body-force" that "twists"
 *       the cantilever.  Read it as the rotation about the cantilever axis
 *       (y_c, z_c): g = gamma (0, -(z - z_c), y - y_c), gamma = gamma0
 *       sin(pi x / (2L)), x from the clamped face; gamma0 = 20 g / H with the
 *       thickness H for "h" (the paper's "h" there is a length of the body, not
 *       the smoothing length).  It is added to gravity on every particle;
 *       dt's |a|max is the largest |g + end load + g_t| over the particles.
 *   R18 2^d-colour sweep layout (ORA_SWEEP_2D, an option; Sec. 3.4 keeps the
 *       3^d colours the default): the splitting cell-linked list with cells of
 *       edge 2 r_c = 4h, colour sum_a (i_a mod 2) 2^a.  Same-colour cells are
 *       then at least one cell of edge 2 r_c apart, so no particle is within
 *       r_c of both, and the cells of a colour touch disjoint particles as in
 *       the paper's layout.  The canonical order is colour, cell, particle id
 *       as in R9, over these cells; it differs from the default order, so the
 *       result of S_d differs too (another order of the same local operators).
 */
#include "srdr_oracle.h"

#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Threads.  The same source builds serially and, with -fopenmp, with the
 * per-particle loops of the stress and force evaluation and the cells of one
 * colour of the damping sweep spread over threads.  Neither changes a
 * rounding: every particle's sums run in the same order on one thread, the
 * cells of one colour touch disjoint particles (Sec. 3.4), and the kinetic
 * energy is summed serially.  The two builds give identical bits. */
void ora_set_threads(int nthreads)
{
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
}

int ora_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

#define ORA_PI 3.14159265358979323846

/* ======================================================================= */
/* Smoothing kernel: 5th-order Wendland C2 with h = 1.3 dp (Sec. 4 intro).  */
/* W(q) = alpha_d (1 - q/2)^4 (1 + 2q), q = r/h in [0, 2]  (reading R3).    */
/* ======================================================================= */
static double wendland_alpha(int dim, double h)
{
    if (dim == 2) return 7.0 / (4.0 * ORA_PI * h * h);
    return 21.0 / (16.0 * ORA_PI * h * h * h);
}

double ora_kernel_W(int dim, double h, double r)
{
    double q = r / h;
    if (q >= 2.0) return 0.0;
    double t = 1.0 - 0.5 * q;
    return wendland_alpha(dim, h) * t * t * t * t * (1.0 + 2.0 * q);
}

/* dW/dr = (alpha_d / h) * d/dq[(1-q/2)^4 (1+2q)] = (alpha_d / h) (-5 q) (1-q/2)^3 */
double ora_kernel_dW(int dim, double h, double r)
{
    double q = r / h;
    if (q >= 2.0) return 0.0;
    double t = 1.0 - 0.5 * q;
    return wendland_alpha(dim, h) / h * (-5.0 * q) * t * t * t;
}

/* ======================================================================= */
/* Material constants (Sec. 2.1, Eq. modulus-relation with reading R1).      */
/* ======================================================================= */
void ora_lame(double E, double nu, double* lambda, double* mu)
{
    *mu = E / (2.0 * (1.0 + nu));
    *lambda = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu));
}

/* Eq. viscous-parameter: eta = beta/4 sqrt(rho0 E) L */
double ora_eta(double beta, double rho0, double E, double L)
{
    return 0.25 * beta * sqrt(rho0 * E) * L;
}

/* ======================================================================= */
/* Small dense algebra on row-major 3x3 storage, restricted to dim x dim.   */
/* ======================================================================= */
static void mat_zero(double A[9]) { for (int k = 0; k < 9; ++k) A[k] = 0.0; }

static void mat_identity(int dim, double A[9])
{
    mat_zero(A);
    for (int a = 0; a < dim; ++a) A[a * 3 + a] = 1.0;
}

static void mat_mul(int dim, const double A[9], const double B[9], double C[9])
{
    double T[9];
    mat_zero(T);
    for (int a = 0; a < dim; ++a)
        for (int b = 0; b < dim; ++b) {
            double s = 0.0;
            for (int c = 0; c < dim; ++c) s += A[a * 3 + c] * B[c * 3 + b];
            T[a * 3 + b] = s;
        }
    memcpy(C, T, sizeof(T));
}

static void mat_transpose(int dim, const double A[9], double T[9])
{
    mat_zero(T);
    for (int a = 0; a < dim; ++a)
        for (int b = 0; b < dim; ++b) T[b * 3 + a] = A[a * 3 + b];
}

static double mat_det(int dim, const double A[9])
{
    if (dim == 2) return A[0] * A[4] - A[1] * A[3];
    return A[0] * (A[4] * A[8] - A[5] * A[7])
         - A[1] * (A[3] * A[8] - A[5] * A[6])
         + A[2] * (A[3] * A[7] - A[4] * A[6]);
}

/* inverse by the adjugate; returns the determinant */
static double mat_inverse(int dim, const double A[9], double Ainv[9])
{
    double d = mat_det(dim, A);
    mat_zero(Ainv);
    if (d == 0.0) return d;
    if (dim == 2) {
        Ainv[0] = A[4] / d;
        Ainv[1] = -A[1] / d;
        Ainv[3] = -A[3] / d;
        Ainv[4] = A[0] / d;
        return d;
    }
    Ainv[0] = (A[4] * A[8] - A[5] * A[7]) / d;
    Ainv[1] = (A[2] * A[7] - A[1] * A[8]) / d;
    Ainv[2] = (A[1] * A[5] - A[2] * A[4]) / d;
    Ainv[3] = (A[5] * A[6] - A[3] * A[8]) / d;
    Ainv[4] = (A[0] * A[8] - A[2] * A[6]) / d;
    Ainv[5] = (A[2] * A[3] - A[0] * A[5]) / d;
    Ainv[6] = (A[3] * A[7] - A[4] * A[6]) / d;
    Ainv[7] = (A[1] * A[6] - A[0] * A[7]) / d;
    Ainv[8] = (A[0] * A[4] - A[1] * A[3]) / d;
    return d;
}

/* ======================================================================= */
/* Constitutive laws (Sec. 2.1).                                            */
/* ======================================================================= */
/* Green-Lagrange strain, Eq. strain-tensor-e: E = 1/2 (F^T F - I) */
static void green_strain(int dim, const double F[9], double E[9])
{
    double Ft[9], C[9];
    mat_transpose(dim, F, Ft);
    mat_mul(dim, Ft, F, C);
    mat_zero(E);
    for (int a = 0; a < dim; ++a)
        for (int b = 0; b < dim; ++b)
            E[a * 3 + b] = 0.5 * (C[a * 3 + b] - (a == b ? 1.0 : 0.0));
}

void ora_pk2(int dim, int material, double lambda, double mu, const double F[9], double S[9])
{
    mat_zero(S);
    if (material == ORA_SVK) {
        /* Eq. constitutive-equation: S = lambda tr(E) I + 2 mu E  (reading: the
         * "linear elastic" law is Saint-Venant-Kirchhoff on the Green strain) */
        double E[9];
        green_strain(dim, F, E);
        double trE = 0.0;
        for (int a = 0; a < dim; ++a) trE += E[a * 3 + a];
        for (int a = 0; a < dim; ++a)
            for (int b = 0; b < dim; ++b)
                S[a * 3 + b] = 2.0 * mu * E[a * 3 + b] + (a == b ? lambda * trE : 0.0);
    } else {
        /* Eqs. strain-density, PK-stress (reading R4):
         * S = dW/dE = mu (I - C^-1) + lambda ln J C^-1 */
        double Ft[9], C[9], Cinv[9];
        mat_transpose(dim, F, Ft);
        mat_mul(dim, Ft, F, C);
        mat_inverse(dim, C, Cinv);
        double J = mat_det(dim, F);
        double lnJ = log(J);
        for (int a = 0; a < dim; ++a)
            for (int b = 0; b < dim; ++b)
                S[a * 3 + b] = mu * ((a == b ? 1.0 : 0.0) - Cinv[a * 3 + b])
                             + lambda * lnJ * Cinv[a * 3 + b];
    }
}

/* Eq. strain-density: W = mu tr(E) - mu ln J + lambda/2 (ln J)^2 */
double ora_nh_energy(int dim, double lambda, double mu, const double F[9])
{
    double E[9];
    green_strain(dim, F, E);
    double trE = 0.0;
    for (int a = 0; a < dim; ++a) trE += E[a * 3 + a];
    double lnJ = log(mat_det(dim, F));
    return mu * trE - mu * lnJ + 0.5 * lambda * lnJ * lnJ;
}

/* ======================================================================= */
/* Philox4x64-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as  */
/* easy as 1, 2, 3", SC'11), written from its published definition.        */
/* ======================================================================= */
static void mulhilo64(uint64_t a, uint64_t b, uint64_t* hi, uint64_t* lo)
{
    unsigned __int128 p = (unsigned __int128)a * (unsigned __int128)b;
    *hi = (uint64_t)(p >> 64);
    *lo = (uint64_t)p;
}

void ora_philox4x64_10(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4])
{
    const uint64_t M0 = 0xD2E7470EE14C6C93ULL, M1 = 0xCA5A826395121157ULL;
    const uint64_t W0 = 0x9E3779B97F4A7C15ULL, W1 = 0xBB67AE8584CAA73BULL;
    uint64_t x[4] = {ctr[0], ctr[1], ctr[2], ctr[3]};
    uint64_t k[2] = {key[0], key[1]};
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k[0] += W0;
            k[1] += W1;
        }
        uint64_t hi0, lo0, hi1, lo1;
        mulhilo64(M0, x[0], &hi0, &lo0);
        mulhilo64(M1, x[2], &hi1, &lo1);
        uint64_t y0 = hi1 ^ x[1] ^ k[0];
        uint64_t y2 = hi0 ^ x[3] ^ k[1];
        x[0] = y0;
        x[1] = lo1;
        x[2] = y2;
        x[3] = lo0;
    }
    memcpy(out, x, sizeof(x));
}

/* Reading R8: one uniform draw per time step, from word 0 of the block. */
double ora_phi(uint64_t seed, uint64_t step)
{
    uint64_t ctr[4] = {step, 0, 0, 0}, key[2] = {seed, 0}, out[4];
    ora_philox4x64_10(ctr, key, out);
    return (double)(out[0] >> 11) * (1.0 / 9007199254740992.0);
}

/* ======================================================================= */
/* Splitting cell-linked list (Sec. 3.4).                                   */
/* Cells of edge r_c = cut-off radius; 3^d blocks ("colours") whose cells   */
/* are pairwise non-adjacent.  Cell index ix = floor((x - x0)/r_c) in FP64, */
/* x0 = min_i x_i, clamped to [0, n_x - 1]; cell id = ix + nx (iy + ny iz); */
/* colour = sum_a (i_a mod 3) 3^a (reading R9).                              */
/* ======================================================================= */
typedef struct {
    int64_t key0, key1, id;
} sortkey3;

static int cmp_sortkey3(const void* a, const void* b)
{
    const sortkey3* x = (const sortkey3*)a;
    const sortkey3* y = (const sortkey3*)b;
    if (x->key0 != y->key0) return x->key0 < y->key0 ? -1 : 1;
    if (x->key1 != y->key1) return x->key1 < y->key1 ? -1 : 1;
    if (x->id != y->id) return x->id < y->id ? -1 : 1;
    return 0;
}

static void cell_coords(int dim, int64_t n, const double* r0, double rc, int64_t* ic,
                        int64_t ncell[3])
{
    double lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
    for (int a = 0; a < dim; ++a) {
        lo[a] = r0[a];
        hi[a] = r0[a];
        for (int64_t i = 1; i < n; ++i) {
            double x = r0[i * 3 + a];
            if (x < lo[a]) lo[a] = x;
            if (x > hi[a]) hi[a] = x;
        }
    }
    for (int a = 0; a < 3; ++a) ncell[a] = 1;
    for (int a = 0; a < dim; ++a) ncell[a] = (int64_t)floor((hi[a] - lo[a]) / rc) + 1;
    for (int64_t i = 0; i < n; ++i)
        for (int a = 0; a < 3; ++a) {
            int64_t c = 0;
            if (a < dim) {
                c = (int64_t)floor((r0[i * 3 + a] - lo[a]) / rc);
                if (c < 0) c = 0;
                if (c > ncell[a] - 1) c = ncell[a] - 1;
            }
            ic[i * 3 + a] = c;
        }
}

void ora_cells(int dim, int64_t n, const double* r0, double rc, int64_t* cell, int* colour,
               int64_t ncell_out[3], int64_t* order)
{
    ora_cells_base(dim, n, r0, rc, 3, cell, colour, ncell_out, order);
}

/* The same with colour sum_a (i_a mod base) base^a (base 3: Sec. 3.4; base
 * 2: the 2^d-colour layout of reading R18, cells of edge 2 r_c) */
void ora_cells_base(int dim, int64_t n, const double* r0, double rc, int base, int64_t* cell,
                    int* colour, int64_t ncell_out[3], int64_t* order)
{
    int64_t* ic = (int64_t*)malloc(sizeof(int64_t) * 3 * (size_t)(n > 0 ? n : 1));
    int64_t ncell[3];
    cell_coords(dim, n, r0, rc, ic, ncell);
    for (int64_t i = 0; i < n; ++i) {
        cell[i] = ic[i * 3 + 0] + ncell[0] * (ic[i * 3 + 1] + ncell[1] * ic[i * 3 + 2]);
        int c = 0, p = 1;
        for (int a = 0; a < dim; ++a) {
            c += (int)(ic[i * 3 + a] % base) * p;
            p *= base;
        }
        colour[i] = c;
    }
    for (int a = 0; a < 3; ++a) ncell_out[a] = ncell[a];
    if (order) {
        sortkey3* k = (sortkey3*)malloc(sizeof(sortkey3) * (size_t)(n > 0 ? n : 1));
        for (int64_t i = 0; i < n; ++i) {
            k[i].key0 = colour[i];
            k[i].key1 = cell[i];
            k[i].id = i;
        }
        qsort(k, (size_t)n, sizeof(sortkey3), cmp_sortkey3);
        for (int64_t i = 0; i < n; ++i) order[i] = k[i].id;
        free(k);
    }
    free(ic);
}

/* ======================================================================= */
/* Neighbour test: 0 < |r0_i - r0_j| < 2h, squared distance summed x,y,z.   */
/* ======================================================================= */
static double dist2(int dim, const double* a, const double* b)
{
    double s = 0.0;
    for (int c = 0; c < dim; ++c) {
        double d = a[c] - b[c];
        s = s + d * d;
    }
    return s;
}

int64_t ora_neighbours_brute(int dim, int64_t n, const double* r0, double cutoff,
                             int64_t* row_ptr, int64_t* col)
{
    double c2 = cutoff * cutoff;
    int64_t nnz = 0;
    for (int64_t i = 0; i < n; ++i) {
        if (row_ptr) row_ptr[i] = nnz;
        for (int64_t j = 0; j < n; ++j) {
            if (j == i) continue;
            double d2 = dist2(dim, r0 + i * 3, r0 + j * 3);
            if (d2 > 0.0 && d2 < c2) {
                if (col) col[nnz] = j;
                ++nnz;
            }
        }
    }
    if (row_ptr) row_ptr[n] = nnz;
    return nnz;
}

static int cmp_i64(const void* a, const void* b)
{
    int64_t x = *(const int64_t*)a, y = *(const int64_t*)b;
    return x < y ? -1 : (x > y ? 1 : 0);
}

/* ======================================================================= */
/* The body.                                                                */
/* ======================================================================= */
struct ora_body {
    ora_params p;
    int64_t n, nnz;
    double *r0, *vol, *mass;
    uint8_t* flags;
    double lambda, mu, eta, dt;
    /* neighbours: row_ptr[n+1], col[nnz] (ascending j), and per pair
     * dW = (dW/dr)^0 at |r0_ij|, rij = |r0_ij|, e = r0_ij / |r0_ij| */
    int64_t *row_ptr, *col;
    double *dW, *rij, *e;
    double* B0;  /* [n][9] */
    /* cells */
    int64_t* cell;
    int* colour;
    int64_t* order; /* canonical sweep order */
    int64_t ncell[3];
    /* the cells of the sweep as runs of the canonical order: run r covers
     * order[run[r] .. run[r+1]-1]; colour c owns runs colour_run[c] ..
     * colour_run[c+1]-1 */
    int64_t nrun;
    int64_t *run, *colour_run;
    int ncolours;
    /* state */
    double *u, *v, *F, *PB, *acc;
    int64_t step;
    int64_t damped;
    double ke, ke_max;
};

static void body_free(ora_body* b)
{
    if (!b) return;
    free(b->r0); free(b->vol); free(b->mass); free(b->flags);
    free(b->row_ptr); free(b->col); free(b->dW); free(b->rij); free(b->e);
    free(b->B0); free(b->cell); free(b->colour); free(b->order);
    free(b->run); free(b->colour_run);
    free(b->u); free(b->v); free(b->F); free(b->PB); free(b->acc);
    free(b);
}

void ora_body_destroy(ora_body* b) { body_free(b); }

/* gradient of the reference kernel, Eq. correction-matrix1:
 * grad0_i W_ij = (dW/dr)^0 e0_ij, e0_ij = r0_ij / |r0_ij|, r0_ij = r0_i - r0_j */
static void grad_w(const ora_body* b, int64_t k, double g[3])
{
    for (int c = 0; c < 3; ++c) g[c] = b->dW[k] * b->e[k * 3 + c];
}

/* Eq. correction-matrix: B0_i = ( - sum_j V0_j r0_ij (x) grad0_i W_ij )^-1 */
static int build_B0(ora_body* b, char* err, int errlen)
{
    int dim = b->p.dim;
    for (int64_t i = 0; i < b->n; ++i) {
        double M[9];
        mat_zero(M);
        for (int64_t k = b->row_ptr[i]; k < b->row_ptr[i + 1]; ++k) {
            int64_t j = b->col[k];
            double g[3], r[3];
            grad_w(b, k, g);
            for (int c = 0; c < 3; ++c) r[c] = b->r0[i * 3 + c] - b->r0[j * 3 + c];
            for (int a = 0; a < dim; ++a)
                for (int c = 0; c < dim; ++c) M[a * 3 + c] -= b->vol[j] * r[a] * g[c];
        }
        /* reading: a neighbourhood too flat to invert is an input error */
        double d = mat_inverse(dim, M, b->B0 + i * 9);
        if (!(fabs(d) >= 1e-8)) {
            if (err) snprintf(err, (size_t)errlen, "singular correction matrix at particle %lld (det %g)",
                              (long long)i, d);
            return -1;
        }
    }
    return 0;
}

static void build_neighbours_cll(ora_body* b)
{
    int dim = b->p.dim;
    int64_t n = b->n;
    double rc = 2.0 * b->p.h;
    int64_t* ic = (int64_t*)malloc(sizeof(int64_t) * 3 * (size_t)(n > 0 ? n : 1));
    int64_t ncell[3];
    cell_coords(dim, n, b->r0, rc, ic, ncell);
    int64_t nc = ncell[0] * ncell[1] * ncell[2];
    /* cells of edge r_c (the search grid, whatever the sweep's layout) and
     * their particles, ascending id (counting sort) */
    int64_t* cid = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    for (int64_t i = 0; i < n; ++i) cid[i] = ic[i * 3 + 0] + ncell[0] * (ic[i * 3 + 1] + ncell[1] * ic[i * 3 + 2]);
    int64_t* start = (int64_t*)calloc((size_t)nc + 1, sizeof(int64_t));
    int64_t* list = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    for (int64_t i = 0; i < n; ++i) start[cid[i] + 1]++;
    for (int64_t c = 0; c < nc; ++c) start[c + 1] += start[c];
    int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * (size_t)(nc + 1));
    memcpy(fill, start, sizeof(int64_t) * (size_t)(nc + 1));
    for (int64_t i = 0; i < n; ++i) list[fill[cid[i]]++] = i;
    free(fill);
    free(cid);

    double c2 = rc * rc;
    int64_t cap = 64;
    int64_t* buf = (int64_t*)malloc(sizeof(int64_t) * (size_t)cap);
    int64_t nnz = 0, nnz_cap = n * 32 + 16;
    int64_t* col = (int64_t*)malloc(sizeof(int64_t) * (size_t)nnz_cap);
    b->row_ptr = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n + 1));
    for (int64_t i = 0; i < n; ++i) {
        b->row_ptr[i] = nnz;
        int64_t cnt = 0;
        int64_t lo[3], hi[3];
        for (int a = 0; a < 3; ++a) {
            lo[a] = ic[i * 3 + a] - 1;
            hi[a] = ic[i * 3 + a] + 1;
            if (lo[a] < 0) lo[a] = 0;
            if (hi[a] > ncell[a] - 1) hi[a] = ncell[a] - 1;
        }
        for (int64_t z = lo[2]; z <= hi[2]; ++z)
            for (int64_t y = lo[1]; y <= hi[1]; ++y)
                for (int64_t x = lo[0]; x <= hi[0]; ++x) {
                    int64_t c = x + ncell[0] * (y + ncell[1] * z);
                    for (int64_t s = start[c]; s < start[c + 1]; ++s) {
                        int64_t j = list[s];
                        if (j == i) continue;
                        double d2 = dist2(dim, b->r0 + i * 3, b->r0 + j * 3);
                        if (d2 > 0.0 && d2 < c2) {
                            if (cnt == cap) {
                                cap *= 2;
                                buf = (int64_t*)realloc(buf, sizeof(int64_t) * (size_t)cap);
                            }
                            buf[cnt++] = j;
                        }
                    }
                }
        qsort(buf, (size_t)cnt, sizeof(int64_t), cmp_i64);
        if (nnz + cnt > nnz_cap) {
            while (nnz + cnt > nnz_cap) nnz_cap *= 2;
            col = (int64_t*)realloc(col, sizeof(int64_t) * (size_t)nnz_cap);
        }
        memcpy(col + nnz, buf, sizeof(int64_t) * (size_t)cnt);
        nnz += cnt;
    }
    b->row_ptr[n] = nnz;
    b->col = col;
    b->nnz = nnz;
    free(buf);
    free(start);
    free(list);
    free(ic);
}

static double vec_norm(int dim, const double* x)
{
    double s = 0.0;
    for (int c = 0; c < dim; ++c) s += x[c] * x[c];
    return sqrt(s);
}

/* reading R12 */
static double body_dt(const ora_body* b)
{
    const ora_params* p = &b->p;
    int dim = p->dim;
    double K = b->lambda + 2.0 * b->mu / 3.0;
    double c = sqrt(K / p->rho0);
    double amax = vec_norm(dim, p->gravity);
    if (p->twist[0] != 0.0) {
        for (int64_t i = 0; i < b->n; ++i) {
            double t[3], a[3];
            ora_twist_force(p, b->r0 + i * 3, t);
            for (int k = 0; k < 3; ++k)
                a[k] = p->gravity[k] + ((b->flags[i] & ORA_FLAG_END_LOAD) ? p->end_load[k] : 0.0) + t[k];
            double m = vec_norm(dim, a);
            if (m > amax) amax = m;
        }
    }
    for (int64_t i = 0; i < b->n; ++i)
        if (b->flags[i] & ORA_FLAG_END_LOAD) {
            double a[3];
            for (int k = 0; k < 3; ++k) a[k] = p->gravity[k] + p->end_load[k];
            double m = vec_norm(dim, a);
            if (m > amax) amax = m;
            break;
        }
    double dt = p->h / c;
    if (amax > 0.0) {
        double t = sqrt(p->h / amax);
        if (t < dt) dt = t;
    }
    dt *= 0.6;
    if (p->damping == ORA_DAMP_EXPLICIT) {
        if (b->eta > 0.0) {
            double nu = b->eta / p->rho0;
            double tv = 0.5 * p->h * p->h / (nu * (double)dim); /* Eq. viscous-criteria-o */
            if (tv < dt) dt = tv;
        }
    } else if (p->damping != ORA_DAMP_NONE && p->alpha > 0.0 && b->eta > 0.0) {
        double nu_t = b->eta / (p->alpha * p->rho0);
        double tv = 50.0 * p->h * p->h / (nu_t * (double)dim); /* Eq. viscous-criteria */
        if (tv < dt) dt = tv;
    }
    return dt;
}

ora_body* ora_body_create(const ora_params* p, int64_t n, const double* r0, const double* vol,
                          double vol_default, const uint8_t* flags, const double* u0, char* err,
                          int errlen)
{
    if (p->dim != 2 && p->dim != 3) {
        if (err) snprintf(err, (size_t)errlen, "dim must be 2 or 3");
        return NULL;
    }
    if (n < 1) {
        if (err) snprintf(err, (size_t)errlen, "empty body");
        return NULL;
    }
    ora_body* b = (ora_body*)calloc(1, sizeof(ora_body));
    b->p = *p;
    b->n = n;
    size_t n3 = (size_t)n * 3, n9 = (size_t)n * 9;
    b->r0 = (double*)calloc(n3, sizeof(double));
    for (int64_t i = 0; i < n; ++i)
        for (int a = 0; a < p->dim; ++a) b->r0[i * 3 + a] = r0[i * 3 + a];
    b->vol = (double*)malloc(sizeof(double) * (size_t)n);
    b->mass = (double*)malloc(sizeof(double) * (size_t)n);
    b->flags = (uint8_t*)calloc((size_t)n, 1);
    for (int64_t i = 0; i < n; ++i) {
        b->vol[i] = vol ? vol[i] : vol_default;
        b->mass[i] = p->rho0 * b->vol[i];
        if (flags) b->flags[i] = flags[i];
    }
    ora_lame(p->E, p->nu, &b->lambda, &b->mu);
    b->eta = ora_eta(p->beta, p->rho0, p->E, p->L_char);

    /* splitting cell-linked list and canonical order */
    b->cell = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
    b->colour = (int*)malloc(sizeof(int) * (size_t)n);
    b->order = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
    /* reading R18: the 2^d-colour layout takes cells of edge 2 r_c = 4h,
     * coloured by parity; the paper's layout (Sec. 3.4) cells of edge r_c =
     * 2h in 3^d colours */
    b->ncolours = p->sweep_layout == ORA_SWEEP_2D ? (p->dim == 2 ? 4 : 8) : (p->dim == 2 ? 9 : 27);
    ora_cells_base(p->dim, n, b->r0, p->sweep_layout == ORA_SWEEP_2D ? 4.0 * p->h : 2.0 * p->h,
                   p->sweep_layout == ORA_SWEEP_2D ? 2 : 3, b->cell, b->colour, b->ncell, b->order);
    {
        int ncol = b->ncolours;
        b->run = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n + 1));
        b->colour_run = (int64_t*)calloc((size_t)ncol + 1, sizeof(int64_t));
        int64_t r = 0;
        for (int64_t s = 0; s < n; ++s) {
            int64_t i = b->order[s];
            if (s == 0 || b->cell[i] != b->cell[b->order[s - 1]]) {
                b->run[r++] = s;
                b->colour_run[b->colour[i] + 1] = r;
            }
        }
        b->run[r] = n;
        b->nrun = r;
        for (int c = 1; c <= ncol; ++c)
            if (b->colour_run[c] < b->colour_run[c - 1]) b->colour_run[c] = b->colour_run[c - 1];
    }

    /* fixed reference neighbours and reference kernel gradients */
    build_neighbours_cll(b);
    b->dW = (double*)malloc(sizeof(double) * (size_t)(b->nnz + 1));
    b->rij = (double*)malloc(sizeof(double) * (size_t)(b->nnz + 1));
    b->e = (double*)calloc((size_t)(b->nnz + 1) * 3, sizeof(double));
    for (int64_t i = 0; i < n; ++i)
        for (int64_t k = b->row_ptr[i]; k < b->row_ptr[i + 1]; ++k) {
            int64_t j = b->col[k];
            double r[3];
            for (int c = 0; c < 3; ++c) r[c] = b->r0[i * 3 + c] - b->r0[j * 3 + c];
            double d = vec_norm(p->dim, r);
            b->rij[k] = d;
            b->dW[k] = ora_kernel_dW(p->dim, p->h, d);
            for (int c = 0; c < 3; ++c) b->e[k * 3 + c] = r[c] / d;
        }
    b->B0 = (double*)calloc(n9, sizeof(double));
    if (build_B0(b, err, errlen) != 0) {
        body_free(b);
        return NULL;
    }
    b->u = (double*)calloc(n3, sizeof(double));
    b->v = (double*)calloc(n3, sizeof(double));
    b->F = (double*)calloc(n9, sizeof(double));
    b->PB = (double*)calloc(n9, sizeof(double));
    b->acc = (double*)calloc(n3, sizeof(double));
    if (u0)
        for (int64_t i = 0; i < n; ++i)
            for (int a = 0; a < p->dim; ++a) b->u[i * 3 + a] = u0[i * 3 + a];
    ora_body_F_from_u(b, b->u, b->F);
    b->dt = p->dt > 0.0 ? p->dt : body_dt(b);
    return b;
}

int64_t ora_body_n(const ora_body* b) { return b->n; }
int64_t ora_body_nnz(const ora_body* b) { return b->nnz; }
double ora_body_dt(const ora_body* b) { return b->dt; }
double ora_body_eta(const ora_body* b) { return b->eta; }
int64_t ora_body_step_index(const ora_body* b) { return b->step; }
double ora_body_ke(const ora_body* b) { return b->ke; }
double ora_body_ke_max(const ora_body* b) { return b->ke_max; }
int64_t ora_body_damped_steps(const ora_body* b) { return b->damped; }

void ora_body_get(const ora_body* b, int what, double* out)
{
    size_t n3 = (size_t)b->n * 3, n9 = (size_t)b->n * 9;
    switch (what) {
    case ORA_U: memcpy(out, b->u, n3 * sizeof(double)); break;
    case ORA_V: memcpy(out, b->v, n3 * sizeof(double)); break;
    case ORA_ACC: memcpy(out, b->acc, n3 * sizeof(double)); break;
    case ORA_F: memcpy(out, b->F, n9 * sizeof(double)); break;
    case ORA_PB: memcpy(out, b->PB, n9 * sizeof(double)); break;
    case ORA_B0: memcpy(out, b->B0, n9 * sizeof(double)); break;
    default: break;
    }
}

void ora_body_set(ora_body* b, int what, const double* in)
{
    size_t n3 = (size_t)b->n * 3, n9 = (size_t)b->n * 9;
    switch (what) {
    case ORA_U: memcpy(b->u, in, n3 * sizeof(double)); break;
    case ORA_V: memcpy(b->v, in, n3 * sizeof(double)); break;
    case ORA_F: memcpy(b->F, in, n9 * sizeof(double)); break;
    default: break;
    }
}

void ora_body_neighbours(const ora_body* b, int64_t* row_ptr, int64_t* col)
{
    memcpy(row_ptr, b->row_ptr, sizeof(int64_t) * (size_t)(b->n + 1));
    memcpy(col, b->col, sizeof(int64_t) * (size_t)b->nnz);
}

void ora_body_cells(const ora_body* b, int64_t* cell, int* colour, int64_t* order)
{
    memcpy(cell, b->cell, sizeof(int64_t) * (size_t)b->n);
    memcpy(colour, b->colour, sizeof(int) * (size_t)b->n);
    memcpy(order, b->order, sizeof(int64_t) * (size_t)b->n);
}

/* ======================================================================= */
/* Kinematics (Sec. 2.2, Eq. deformation-gradient and the rate equation).   */
/* ======================================================================= */
/* F_i = I + grad0 u, with the corrected gradient
 * grad0 u_i = -(sum_j V0_j u_ij (x) grad0_i W_ij) B0_i  (reading R5: the
 * displacement form of the same discrete operator as dF/dt) */
void ora_body_F_from_u(const ora_body* b, const double* u, double* F_out)
{
    int dim = b->p.dim;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < b->n; ++i) {
        double G[9], GB[9];
        mat_zero(G);
        for (int64_t k = b->row_ptr[i]; k < b->row_ptr[i + 1]; ++k) {
            int64_t j = b->col[k];
            double g[3];
            grad_w(b, k, g);
            for (int a = 0; a < dim; ++a)
                for (int c = 0; c < dim; ++c)
                    G[a * 3 + c] += b->vol[j] * (u[i * 3 + a] - u[j * 3 + a]) * g[c];
        }
        mat_mul(dim, G, b->B0 + i * 9, GB);
        double* F = F_out + i * 9;
        mat_identity(dim, F);
        for (int a = 0; a < dim; ++a)
            for (int c = 0; c < dim; ++c) F[a * 3 + c] -= GB[a * 3 + c];
    }
}

/* dF_i/dt = -(sum_j V0_j v_ij (x) grad0_i W_ij) B0_i */
void ora_body_Fdot(const ora_body* b, const double* v, double* Fdot_out)
{
    int dim = b->p.dim;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < b->n; ++i) {
        double G[9], GB[9];
        mat_zero(G);
        for (int64_t k = b->row_ptr[i]; k < b->row_ptr[i + 1]; ++k) {
            int64_t j = b->col[k];
            double g[3];
            grad_w(b, k, g);
            for (int a = 0; a < dim; ++a)
                for (int c = 0; c < dim; ++c)
                    G[a * 3 + c] += b->vol[j] * (v[i * 3 + a] - v[j * 3 + a]) * g[c];
        }
        mat_mul(dim, G, b->B0 + i * 9, GB);
        for (int k = 0; k < 9; ++k) Fdot_out[i * 9 + k] = -GB[k];
    }
}

/* Eq. evaluate-momentum with Eq. averaged-Piola-Kirchhoff:
 * dv_i/dt = 2/m_i sum_j V0_i V0_j 1/2 (P_i B0_i + P_j B0_j) grad0_i W_ij + g,
 * P = F S (Eq. piola).  Also stores P B0 per particle in b->PB. */
void ora_body_acc(const ora_body* b, const double* F, double* acc_out)
{
    int dim = b->p.dim;
    ora_body* bm = (ora_body*)b;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < b->n; ++i) {
        double S[9], P[9];
        ora_pk2(dim, b->p.material, b->lambda, b->mu, F + i * 9, S);
        mat_mul(dim, F + i * 9, S, P);
        mat_mul(dim, P, b->B0 + i * 9, bm->PB + i * 9);
    }
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < b->n; ++i) {
        double a[3] = {0, 0, 0};
        for (int64_t k = b->row_ptr[i]; k < b->row_ptr[i + 1]; ++k) {
            int64_t j = b->col[k];
            double g[3];
            grad_w(b, k, g);
            for (int r = 0; r < dim; ++r) {
                double s = 0.0;
                for (int c = 0; c < dim; ++c)
                    s += 0.5 * (b->PB[i * 9 + r * 3 + c] + b->PB[j * 9 + r * 3 + c]) * g[c];
                a[r] += b->vol[i] * b->vol[j] * s;
            }
        }
        double tw[3] = {0, 0, 0};
        if (b->p.twist[0] != 0.0) ora_twist_force(&b->p, b->r0 + i * 3, tw);
        for (int r = 0; r < 3; ++r) {
            double extra = b->p.gravity[r] + tw[r];
            if (b->flags[i] & ORA_FLAG_END_LOAD) extra += b->p.end_load[r];
            acc_out[i * 3 + r] = (r < dim ? 2.0 / b->mass[i] * a[r] : 0.0) + (r < dim ? extra : 0.0);
        }
    }
}

/* ======================================================================= */
/* Damping (Sec. 3).                                                         */
/* ======================================================================= */
/* Eq. parameters1: B_j = 2 eta V0_i V0_j (1/r_ij) (dW/dr)^0 dt */
static double coeff_B(const ora_body* b, int64_t i, int64_t k, double eta, double dt)
{
    int64_t j = b->col[k];
    return 2.0 * eta * b->vol[i] * b->vol[j] * (1.0 / b->rij[k]) * b->dW[k] * dt;
}

/* Eq. rotation-body-force with reading R17 */
void ora_twist_force(const ora_params* p, const double r[3], double out[3])
{
    double gamma = p->twist[0] * sin(ORA_PI * r[0] / (2.0 * p->twist[1]));
    out[0] = 0.0;
    out[1] = -gamma * (r[2] - p->twist[3]);
    out[2] = gamma * (r[1] - p->twist[2]);
}

/* Eq. damping-term: a_i = (2 eta / m_i) sum_j V_i V_j v_ij / r_ij (dW/dr)_ij */
void ora_body_viscous_acc(const ora_body* b, double eta, const double* v, double* out)
{
    int dim = b->p.dim;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < b->n; ++i) {
        double a[3] = {0, 0, 0};
        double Vi = b->mass[i] / b->p.rho0;
        for (int64_t k = b->row_ptr[i]; k < b->row_ptr[i + 1]; ++k) {
            int64_t j = b->col[k];
            double Vj = b->mass[j] / b->p.rho0;
            double f = Vi * Vj * b->dW[k] / b->rij[k];
            for (int c = 0; c < dim; ++c) a[c] += f * (v[i * 3 + c] - v[j * 3 + c]);
        }
        for (int c = 0; c < 3; ++c) out[i * 3 + c] = c < dim ? 2.0 * eta / b->mass[i] * a[c] : 0.0;
    }
}

/* Sec. 3.1, particle-by-particle scheme: Eqs. parameters1, parameters2,
 * learning-rate-solve, first-step and second-step. */
static void local_update_particle(const ora_body* b, int64_t i, double eta, double dt, double* v)
{
    int dim = b->p.dim;
    int64_t k0 = b->row_ptr[i], k1 = b->row_ptr[i + 1];
    double mi = b->mass[i];
    double sumB = 0.0, sumB2 = 0.0, E[3] = {0, 0, 0};
    for (int64_t k = k0; k < k1; ++k) {
        int64_t j = b->col[k];
        double Bj = coeff_B(b, i, k, eta, dt);
        sumB += Bj;
        sumB2 += Bj * Bj;
        /* E_i = - sum_j B_j v_ij^n */
        for (int c = 0; c < dim; ++c) E[c] -= Bj * (v[i * 3 + c] - v[j * 3 + c]);
    }
    /* learning rate k = ((sum B_j - m_i)^2 + sum B_j^2)^-1 E_i */
    double denom = (sumB - mi) * (sumB - mi) + sumB2;
    double kv[3] = {0, 0, 0};
    for (int c = 0; c < dim; ++c) kv[c] = E[c] / denom;
    /* first step: v_i^{n+1} = v_i^n + (sum B - m_i) k;  v_j^p = v_j^n - B_j k */
    double vi_new[3] = {0, 0, 0};
    for (int c = 0; c < dim; ++c) vi_new[c] = v[i * 3 + c] + (sumB - mi) * kv[c];
    /* second step (reading R10): v_j^{n+1} = v_j^n - B_j (v_i^{n+1} - v_j^p) / m_j */
    for (int64_t k = k0; k < k1; ++k) {
        int64_t j = b->col[k];
        double Bj = coeff_B(b, i, k, eta, dt);
        for (int c = 0; c < dim; ++c) {
            double vp = v[j * 3 + c] - Bj * kv[c];
            v[j * 3 + c] = v[j * 3 + c] - Bj * (vi_new[c] - vp) / b->mass[j];
        }
    }
    for (int c = 0; c < dim; ++c) v[i * 3 + c] = vi_new[c];
}

/* Sec. 3.2, pairwise scheme: D_i = D_{i,1}..D_{i,N} D_{i,N}..D_{i,1}, each pair
 * over dt/2, solved in closed form by Eq. pairwise-solve. */
static void pair_update(const ora_body* b, int64_t i, int64_t k, double eta, double dt, double* v)
{
    int dim = b->p.dim;
    int64_t j = b->col[k];
    double Bj = coeff_B(b, i, k, eta, dt);
    double mi = b->mass[i], mj = b->mass[j];
    double den = mi * mj - (mi + mj) * Bj;
    for (int c = 0; c < dim; ++c) {
        double vij = v[i * 3 + c] - v[j * 3 + c];
        double dvi = mj * Bj * vij / den;
        double dvj = -mi * Bj * vij / den;
        v[i * 3 + c] += dvi;
        v[j * 3 + c] += dvj;
    }
}

static void local_update_pairwise(const ora_body* b, int64_t i, double eta, double dt, double* v)
{
    int64_t k0 = b->row_ptr[i], k1 = b->row_ptr[i + 1];
    for (int64_t k = k0; k < k1; ++k) pair_update(b, i, k, eta, 0.5 * dt, v);
    for (int64_t k = k1 - 1; k >= k0; --k) pair_update(b, i, k, eta, 0.5 * dt, v);
}

void ora_body_local_update(const ora_body* b, int64_t i, double eta_tilde, double dt_loc, double* v)
{
    if (b->p.damping == ORA_DAMP_PAIRWISE)
        local_update_pairwise(b, i, eta_tilde, dt_loc, v);
    else
        local_update_particle(b, i, eta_tilde, dt_loc, v);
}

/* Eq. particle-by-particle-splitting: forward sweep over the canonical order
 * with dt/2, then the exact reverse with dt/2 (reading R7, R9).  dt_loc here
 * is already the half step. */
void ora_body_damp(ora_body* b, double eta_tilde, double dt_loc)
{
    /* The canonical order, taken colour by colour: the runs (cells) of one
     * colour touch disjoint particles, so they may run in any order or at the
     * same time and give the serial result. */
    int ncol = b->ncolours;
    for (int c = 0; c < ncol; ++c) {
#pragma omp parallel for schedule(dynamic, 1)
        for (int64_t r = b->colour_run[c]; r < b->colour_run[c + 1]; ++r)
            for (int64_t s = b->run[r]; s < b->run[r + 1]; ++s)
                ora_body_local_update(b, b->order[s], eta_tilde, dt_loc, b->v);
    }
    for (int c = ncol - 1; c >= 0; --c) {
#pragma omp parallel for schedule(dynamic, 1)
        for (int64_t r = b->colour_run[c + 1] - 1; r >= b->colour_run[c]; --r)
            for (int64_t s = b->run[r + 1] - 1; s >= b->run[r]; --s)
                ora_body_local_update(b, b->order[s], eta_tilde, dt_loc, b->v);
    }
}

static void impose_constraints(ora_body* b)
{
    for (int64_t i = 0; i < b->n; ++i)
        if (b->flags[i] & ORA_FLAG_CONSTRAINED)
            for (int c = 0; c < 3; ++c) b->v[i * 3 + c] = 0.0;
}

static double kinetic_energy(const ora_body* b)
{
    double ke = 0.0;
    for (int64_t i = 0; i < b->n; ++i) {
        if (b->flags[i] & ORA_FLAG_CONSTRAINED) continue;
        double s = 0.0;
        for (int c = 0; c < b->p.dim; ++c) s += b->v[i * 3 + c] * b->v[i * 3 + c];
        ke += 0.5 * b->mass[i] * s;
    }
    return ke;
}

/* One time step: position Verlet (Sec. 2.3) with the Lie-Trotter split
 * v(t+dt) = S_d o S_m v(t) (Eq. operator-splitting) and the random choice of
 * Eq. viscosity-reset (reading R8). */
static void one_step(ora_body* b)
{
    int dim = b->p.dim;
    int64_t n = b->n;
    double dt = b->dt;
    size_t n9 = (size_t)n * 9;
    double* Fd = (double*)malloc(n9 * sizeof(double));
    double* Fh = (double*)malloc(n9 * sizeof(double));
    double* uh = (double*)malloc((size_t)n * 3 * sizeof(double));

    /* Eq. timestep-1: F^{n+1/2} = F^n + dt/2 dF/dt(v^n); r^{n+1/2} = r^n + dt/2 v^n */
    for (int64_t i = 0; i < n; ++i)
        for (int c = 0; c < 3; ++c) uh[i * 3 + c] = b->u[i * 3 + c] + 0.5 * dt * b->v[i * 3 + c];
    if (b->p.f_form == ORA_F_RATE) {
        ora_body_Fdot(b, b->v, Fd);
        for (size_t k = 0; k < n9; ++k) Fh[k] = b->F[k] + 0.5 * dt * Fd[k];
    } else {
        ora_body_F_from_u(b, uh, Fh);
    }

    /* S_m: v^* = v^n + dt dv/dt, dv/dt from the stress at F^{n+1/2}; the
     * explicit comparator adds the viscous term at v^n (reading R16) */
    ora_body_acc(b, Fh, b->acc);
    if (b->p.damping == ORA_DAMP_EXPLICIT && b->eta > 0.0) {
        double* av = (double*)malloc((size_t)n * 3 * sizeof(double));
        ora_body_viscous_acc(b, b->eta, b->v, av);
        for (int64_t i = 0; i < n; ++i)
            for (int c = 0; c < dim; ++c) b->acc[i * 3 + c] += av[i * 3 + c];
        free(av);
    }
    for (int64_t i = 0; i < n; ++i)
        for (int c = 0; c < dim; ++c) b->v[i * 3 + c] += dt * b->acc[i * 3 + c];
    impose_constraints(b);

    /* S_d on a randomly chosen step, eta~ = eta / alpha (reading R8) */
    if ((b->p.damping == ORA_DAMP_PARTICLE || b->p.damping == ORA_DAMP_PAIRWISE) && b->p.alpha > 0.0 &&
        b->eta > 0.0) {
        double phi = ora_phi(b->p.seed, (uint64_t)b->step);
        if (phi < b->p.alpha) {
            ora_body_damp(b, b->eta / b->p.alpha, 0.5 * dt);
            impose_constraints(b);
            b->damped++;
        }
    }

    /* Eq. timestep-3 with reading R5 */
    if (b->p.f_form == ORA_F_RATE) {
        ora_body_Fdot(b, b->v, Fd);
        for (size_t k = 0; k < n9; ++k) b->F[k] = Fh[k] + 0.5 * dt * Fd[k];
    }
    for (int64_t i = 0; i < n; ++i)
        for (int c = 0; c < 3; ++c) b->u[i * 3 + c] = uh[i * 3 + c] + 0.5 * dt * b->v[i * 3 + c];
    if (b->p.f_form != ORA_F_RATE) ora_body_F_from_u(b, b->u, b->F);

    b->ke = kinetic_energy(b);
    if (b->ke > b->ke_max) b->ke_max = b->ke;
    b->step++;
    free(Fd);
    free(Fh);
    free(uh);
}

int ora_body_step(ora_body* b, int64_t nsteps)
{
    for (int64_t s = 0; s < nsteps; ++s) one_step(b);
    return isfinite(b->ke) ? 0 : 2;
}

int ora_body_relax(ora_body* b, double tol, int64_t max_steps, int64_t* steps_taken, double* ratio)
{
    int64_t s = 0;
    int status = 1;
    while (s < max_steps) {
        one_step(b);
        ++s;
        if (!isfinite(b->ke)) {
            status = 2;
            break;
        }
        if (b->ke < tol * b->ke_max) {
            status = 0;
            break;
        }
    }
    if (steps_taken) *steps_taken = s;
    if (ratio) *ratio = b->ke_max > 0.0 ? b->ke / b->ke_max : 0.0;
    return status;
}
