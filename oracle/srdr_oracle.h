/*
 * srdr_oracle.h — plain, slow FP64 CPU oracle of the splitting random-choice
 * dynamic relaxation method for Total-Lagrangian SPH (Zhu, Zhang & Hu,
 * arXiv 2103.08932).
 *
 * TEST INFRASTRUCTURE ONLY.  This code exists to check the CUDA library against
 * the paper.  Only the test suite, the smoke check and the benchmark's CPU
 * baseline may load it; the product path never does.  It shares no code,
 * header, table or constant with the CUDA library.
 *
 * Every routine is written from the paper's equations in the paper's order,
 * with no blocking, fusion or reordering.  All arithmetic is IEEE binary64 and
 * the file must be compiled with -ffp-contract=off so that no fused
 * multiply-add changes a rounding (the neighbour test |r|^2 < (2h)^2 and the
 * cell index floor((x - x0) / r_c) are integer decisions taken in FP64).
 *
 * Particle arrays are in ORIGINAL order (index = particle id) and row-major:
 * vectors are [n][3], tensors [n][3][3]; in 2D the third component/row/column
 * is present and zero.
 */
#ifndef SRDR_ORACLE_H
#define SRDR_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { ORA_SVK = 0, ORA_NEO_HOOKEAN = 1 };
/* ORA_DAMP_EXPLICIT: the comparator of Sec. 3 -- the viscous term of
 * Eq. damping-term added to dv/dt with eta (no random choice), evaluated
 * at v^n, under the explicit limit of Eq. viscous-criteria-o */
enum { ORA_DAMP_NONE = 0, ORA_DAMP_PARTICLE = 1, ORA_DAMP_PAIRWISE = 2, ORA_DAMP_EXPLICIT = 3 };
enum { ORA_F_RATE = 0, ORA_F_DISPLACEMENT = 1 };
/* sweep layout: the paper's 3^d colours over cells of edge 2h (Sec. 3.4), or
 * 2^d colours over cells of edge 4h (reading R18) */
enum { ORA_SWEEP_3D = 0, ORA_SWEEP_2D = 1 };
/* particle flag bits */
enum { ORA_FLAG_CONSTRAINED = 1, ORA_FLAG_END_LOAD = 2 };

typedef struct {
    int dim;               /* 2 (plane strain) or 3 */
    int material;          /* ORA_SVK | ORA_NEO_HOOKEAN */
    double rho0, E, nu;    /* reference density, Young's modulus, Poisson ratio */
    double h;              /* smoothing length; support radius 2h */
    double gravity[3];     /* body force per unit mass */
    double end_load[3];    /* extra acceleration on ORA_FLAG_END_LOAD particles */
    double beta, L_char;   /* eta = beta/4 sqrt(rho0 E) L (Sec. 3.1, Eq. viscous-parameter) */
    double alpha;          /* random-choice probability (Sec. 3.3) */
    uint64_t seed;         /* Philox key */
    int damping;           /* ORA_DAMP_* */
    int f_form;            /* ORA_F_RATE (paper, Sec. 2.3) | ORA_F_DISPLACEMENT */
    double dt;             /* > 0: use this time step; 0: Eq. time-step-criterion */
    /* rotational body force of the twisting cantilever (Sec. 4.2, Eq.
     * rotation-body-force, reading R17): twist = (gamma0, L, y_c, z_c),
     * g_t = gamma0 sin(pi x / (2 L)) (0, -(z - z_c), y - y_c); gamma0 = 0: none */
    double twist[4];
    int sweep_layout;      /* ORA_SWEEP_3D (default) | ORA_SWEEP_2D */
} ora_params;

/* threads of the OpenMP build (ignored by the serial build); identical bits */
void ora_set_threads(int nthreads);
int  ora_threads(void);

/* ---- closed pieces ---------------------------------------------------- */
double ora_kernel_W(int dim, double h, double r);    /* Wendland C2 */
double ora_kernel_dW(int dim, double h, double r);   /* dW/dr */
void   ora_lame(double E, double nu, double* lambda, double* mu);
double ora_eta(double beta, double rho0, double E, double L);
/* second Piola-Kirchhoff stress S(F) for a dim x dim F (row-major 3x3 storage) */
void   ora_pk2(int dim, int material, double lambda, double mu, const double F[9], double S[9]);
/* strain energy density of the neo-Hookean law (Eq. strain-density) */
double ora_nh_energy(int dim, double lambda, double mu, const double F[9]);
/* Philox4x64-10 (Salmon et al., SC'11): out[4] from counter[4], key[2] */
void   ora_philox4x64_10(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4]);
/* uniform draw phi_n in [0,1) for step n of a body with this seed */
double ora_phi(uint64_t seed, uint64_t step);

/* ---- splitting cell-linked list (Sec. 3.4) ---------------------------- */
/* cell[i], colour[i] per particle; ncell_out[3] = cells per axis;
 * order[k] = particle id of the k-th particle in canonical sweep order. */
void ora_cells(int dim, int64_t n, const double* r0, double rc,
               int64_t* cell, int* colour, int64_t ncell_out[3], int64_t* order);
/* the same with colour base 3 (Sec. 3.4) or 2 (reading R18, cells of edge 4h) */
void ora_cells_base(int dim, int64_t n, const double* r0, double rc, int base,
                    int64_t* cell, int* colour, int64_t ncell_out[3], int64_t* order);

/* ---- neighbour lists: 0 < |r0_i - r0_j| < 2h -------------------------- */
/* brute force O(N^2).  row_ptr has n+1 entries; col has row_ptr[n] entries.
 * Call with col == NULL to count only.  Each row is ascending in j. */
int64_t ora_neighbours_brute(int dim, int64_t n, const double* r0, double cutoff,
                             int64_t* row_ptr, int64_t* col);

/* ---- the body ----------------------------------------------------------- */
typedef struct ora_body ora_body;

/* vol may be NULL (then every V0 = vol_default); flags may be NULL (all free);
 * u0 may be NULL (zero).  Returns NULL and writes err on failure. */
ora_body* ora_body_create(const ora_params* p, int64_t n, const double* r0,
                          const double* vol, double vol_default,
                          const uint8_t* flags, const double* u0,
                          char* err, int errlen);
void    ora_body_destroy(ora_body* b);
int64_t ora_body_n(const ora_body* b);
int64_t ora_body_nnz(const ora_body* b);
double  ora_body_dt(const ora_body* b);
double  ora_body_eta(const ora_body* b);
int64_t ora_body_step_index(const ora_body* b);
double  ora_body_ke(const ora_body* b);
double  ora_body_ke_max(const ora_body* b);
int64_t ora_body_damped_steps(const ora_body* b);

enum { ORA_U = 0, ORA_V = 1, ORA_F = 2, ORA_PB = 3, ORA_B0 = 4, ORA_ACC = 5 };
/* copy a state array out ([n][3] for U,V,ACC; [n][9] for F,PB,B0) */
void ora_body_get(const ora_body* b, int what, double* out);
/* overwrite U or V (and, for U in displacement form, nothing else); for F the
 * deformation gradient used by the rate form */
void ora_body_set(ora_body* b, int what, const double* in);
/* neighbour CSR built through the cell-linked list (rows ascending in j) */
void ora_body_neighbours(const ora_body* b, int64_t* row_ptr, int64_t* col);
void ora_body_cells(const ora_body* b, int64_t* cell, int* colour, int64_t* order);

/* one or more full time steps (Sec. 2.3 with the split damping of Sec. 3). */
int ora_body_step(ora_body* b, int64_t nsteps);
/* steps until KE < tol * KE_max (tested after each step) or max_steps.
 * returns 0 converged, 1 not converged, 2 non-finite KE */
int ora_body_relax(ora_body* b, double tol, int64_t max_steps, int64_t* steps_taken,
                   double* ratio);

/* building blocks exposed for the tests */
/* F from the current displacement: F = I - (sum_j V_j u_ij (x) gradW_ij) B0 */
void ora_body_F_from_u(const ora_body* b, const double* u, double* F_out);
/* dF/dt from a velocity field (Sec. 2.2) */
void ora_body_Fdot(const ora_body* b, const double* v, double* Fdot_out);
/* dv/dt from a deformation-gradient field (Eq. evaluate-momentum) */
void ora_body_acc(const ora_body* b, const double* F, double* acc_out);
/* rotational body force of reading R17 at reference position r (3 doubles) */
void ora_twist_force(const ora_params* p, const double r[3], double out[3]);
/* viscous acceleration of Eq. damping-term for a velocity field v[n][3]:
 * a_i = (2 eta / m_i) sum_j V_i V_j (v_i - v_j) / r_ij dW/dr (r_ij) */
void ora_body_viscous_acc(const ora_body* b, double eta, const double* v, double* acc_out);
/* apply the damping operator S_d (forward then backward sweep) to b's v */
void ora_body_damp(ora_body* b, double eta_tilde, double dt_loc);
/* one local update D_i on an arbitrary velocity array v[n][3] */
void ora_body_local_update(const ora_body* b, int64_t i, double eta_tilde, double dt_loc,
                           double* v);

#ifdef __cplusplus
}
#endif
#endif
