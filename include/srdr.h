/*
 * srdr.h — C ABI of the GB300 (sm_103a) library for the splitting
 * random-choice dynamic relaxation of Total-Lagrangian SPH
 * (Zhu, Zhang & Hu, "A splitting random-choice dynamic relaxation method for
 * smoothed particle hydrodynamics", arXiv 2103.08932).
 *
 * Problem statement (Sec. 2.1, Sec. 4 intro): an elastic body given by
 * particles on its reference configuration, smoothing length h = 1.3 dp,
 * fixed reference neighbours 0 < |r0_ij| < 2h, loaded by a body force, is
 * relaxed to static equilibrium by the TL-SPH step (Sec. 2.2-2.3) plus the
 * operator-split implicit artificial-viscosity damping (Sec. 3.1) applied on
 * randomly chosen steps (Sec. 3.3) and swept colour by colour over the
 * splitting cell-linked list (Sec. 3.4).
 *
 * Conventions for every entry point:
 *  - Every call returns an srdr_status; no C++ exception crosses the ABI.
 *    On failure srdr_last_error() returns a message (thread-local, valid
 *    until the next call on the same thread).
 *  - Host arrays passed in are caller-owned and only read during the call.
 *    Host arrays passed out are caller-owned and must hold the stated number
 *    of elements; the library never keeps a pointer to them.
 *  - Particle arrays are in ORIGINAL particle order, FP64, row-major [n][3]
 *    for vectors (the third component is ignored / written as 0 in 2D).
 *  - The library owns all device memory of a body (and of a server) and frees
 *    it in the matching destroy call.
 *  - A handle is not thread-safe; the server is internally synchronised.
 *  - cuda_stream is a cudaStream_t (NULL = the legacy default stream); all
 *    device work of a handle is ordered on it.
 */
#ifndef SRDR_H
#define SRDR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SRDR_OK = 0,
    SRDR_ERR_INVALID = -1,       /* bad argument or body (e.g. singular correction matrix) */
    SRDR_ERR_NO_MEMORY = -2,     /* device allocation or memory admission refused */
    SRDR_ERR_CUDA = -3,          /* a CUDA runtime call failed */
    SRDR_ERR_NOT_CONVERGED = -4, /* step cap reached before the KE criterion */
    SRDR_ERR_NONFINITE = -5,     /* kinetic energy became NaN or Inf */
    SRDR_ERR_TIMEOUT = -6,       /* a bounded device-side wait gave up */
    SRDR_ERR_BUSY = -7           /* server queue full / result not ready */
} srdr_status;

enum { SRDR_LINEAR_SVK = 0, SRDR_NEO_HOOKEAN = 1 };
enum { SRDR_FP64 = 0, SRDR_FP32_MIXED = 1 };
enum { SRDR_DAMP_NONE = 0, SRDR_DAMP_PARTICLE = 1, SRDR_DAMP_PAIRWISE = 2, SRDR_DAMP_EXPLICIT = 3 };
enum { SRDR_FLAG_CONSTRAINED = 1, SRDR_FLAG_END_LOAD = 2 };
enum { SRDR_SWEEP_LAYOUT_3D = 0, SRDR_SWEEP_LAYOUT_2D = 1 };

/*
 * Body description (POD, caller-owned, copied by the create calls).
 *
 * Lattice bodies (srdr_body_create): particles at (i + 1/2) dp filling
 * [0, extent[a]) on each axis; clamp_layers extra layers below 0 on
 * clamp_axis are constrained (v = 0, u = 0); presc_layers extra layers beyond
 * extent on clamp_axis are held at displacement presc_disp and the body
 * starts from the linear interpolation between the two faces;
 * end_load_layer != 0 adds end_load to the last body layer on clamp_axis.
 * Particle order: z outermost, y, x innermost, constrained layers included.
 *
 * material, rho0, E, nu: Sec. 2.1 (Eqs. constitutive-equation, strain-density;
 *   E = 2 mu (1 + nu), 2D is plane strain).
 * h_over_dp: smoothing length h = h_over_dp * dp (1.3 in Sec. 4).
 * beta, L_char: eta = beta/4 sqrt(rho0 E) L_char (Eq. viscous-parameter).
 * alpha, seed: random choice (Eq. viscosity-reset): step n is damped with
 *   eta~ = eta / alpha iff phi_n < alpha, phi_n from Philox4x64-10 with
 *   counter (n, 0, 0, 0) and key (seed, 0), top 53 bits of word 0 / 2^53.
 * damping: SRDR_DAMP_PARTICLE is the particle-by-particle scheme (Sec. 3.1),
 *   SRDR_DAMP_PAIRWISE the pairwise scheme (Sec. 3.2).  SRDR_DAMP_EXPLICIT is
 *   the comparator of Sec. 3: the viscous term of Eq. damping-term with eta
 *   (no random choice, alpha unused) evaluated at v^n and added to dv/dt, with
 *   dt limited by Eq. viscous-criteria-o, 0.5 h^2 / (nu D), nu = eta / rho0.
 *   Explicit bodies step alone (batches refuse them).
 * precision: SRDR_FP64 computes everything in FP64; SRDR_FP32_MIXED runs the
 *   neighbour sums, stress and damping in FP32 and keeps the displacement as
 *   an FP32 hi plus an FP32 lo per component (about 48 significant bits) and the kinetic-energy
 *   reduction in FP64.
 * dt: > 0 fixes the time step; 0 uses Eq. time-step-criterion with
 *   |v|max = 0 and |a|max = the largest body force, min'd with the implicit
 *   viscous limit 50 h^2 / (nu~ D) of Eq. viscous-criteria, nu~ = eta/(alpha rho0).
 * twist: the rotational body force of the twisting cantilever (Sec. 4.2,
 *   Eq. rotation-body-force) read as a rotation about the axis through
 *   (y, z) = (twist[2], twist[3]): g_t = twist[0] sin(pi x / (2 twist[1]))
 *   (0, -(z - twist[3]), y - twist[2]) per unit mass, x from the clamped face
 *   (the printed (0, y gamma, z gamma) is radial, not rotational).  Added to
 *   gravity on every particle; 3D only; twist[0] = 0: none.
 * sweep_layout: the splitting cell-linked list that orders the damping sweep
 *   (Sec. 3.4).  SRDR_SWEEP_LAYOUT_3D (0, the paper's): cells of edge
 *   r_c = 2h in 3^d colours, colour sum_a (i_a mod 3) 3^a.
 *   SRDR_SWEEP_LAYOUT_2D: cells of edge 2 r_c in 2^d colours, colour
 *   sum_a (i_a mod 2) 2^a; same-colour cells are still a cell of edge 2 r_c
 *   apart, so no particle is within r_c of two of them and they commute.
 *   Fewer colour phases (2^(d+1) - 1 instead of 2 3^d - 1) of cells 2^d times
 *   larger; the sweep order, and so the damped velocities, differ from the
 *   paper's layout within the method (the same static state).  The stress and
 *   force passes do not depend on it.  Batches refuse these bodies, and the
 *   sweep's footprint must fit in shared memory (FP64 3D does not).
 */
typedef struct {
    int dim;
    double extent[3];
    double dp;
    int clamp_axis;     /* -1: none */
    int clamp_layers;
    int presc_layers;
    double presc_disp[3];
    int end_load_layer;
    int material;
    double rho0, E, nu;
    double h_over_dp;
    double gravity[3];
    double end_load[3];
    double beta, L_char, alpha;
    uint64_t seed;
    int damping;
    int precision;
    double dt;
    double twist[4];
    int sweep_layout;
    int pass_layout;    /* SRDR_PASS_LAYOUT_AUTO (0) or SRDR_PASS_LAYOUT_SELL, see below */
} srdr_body_desc;

/* pass_layout: how the stress and force passes (Secs. 2.2-2.3, the momentum
 *   equation) enumerate a particle's neighbours.
 *   SRDR_PASS_LAYOUT_AUTO (0): a body whose reference positions form a box
 *   lattice of spacing dp (x fastest, then y, then z: the order that
 *   srdr_body_create builds), with one particle volume, takes the lattice
 *   stencil (SRDR_PASS_STENCIL below) when the stencil reproduces every
 *   particle's neighbour list (checked at creation); any other body takes
 *   the sliced-ELL mapping.  SRDR_PASS_LAYOUT_SELL: the sliced-ELL mapping
 *   (and the brick mapping of srdr_body_pass_mapping) for every body.  The
 *   pair gradients of the stencil are evaluated once per lattice offset from
 *   the exact offset, those of the sliced-ELL layout once per pair from the
 *   positions: the two agree to rounding. */
enum { SRDR_PASS_LAYOUT_AUTO = 0, SRDR_PASS_LAYOUT_SELL = 1 };

typedef struct srdr_body srdr_body;

/* Build a lattice body from desc: particles (Sec. 4), splitting cell-linked
 * list and colour split (Sec. 3.4), neighbour CSR and kernel-gradient weights
 * (Eqs. correction-matrix1), correction matrices B0 (Eq. correction-matrix).
 * SRDR_ERR_INVALID on a bad desc or a singular correction matrix. */
srdr_status srdr_body_create(const srdr_body_desc* desc, void* cuda_stream, srdr_body** out);

/* The same from explicit particles: r0[n][3] reference positions, vol[n]
 * volumes (NULL: dp^dim), flags[n] SRDR_FLAG_* bits (NULL: all free), u0[n][3]
 * initial displacements (NULL: zero; constrained particles keep theirs).
 * The lattice fields of desc (extent, clamp_*, presc_*, end_load_layer) are
 * ignored; dp still sets h and the default volume. */
srdr_status srdr_body_create_particles(const srdr_body_desc* desc, int64_t n, const double* r0,
                                       const double* vol, const uint8_t* flags, const double* u0,
                                       void* cuda_stream, srdr_body** out);

/* Advance nsteps time steps (Sec. 2.3 position-Verlet with the Lie-Trotter
 * split v(t+dt) = S_d o S_m v(t), Eq. operator-splitting).  Asynchronous on
 * the body's stream; errors of the device work surface at the next
 * synchronising call. */
srdr_status srdr_body_step(srdr_body* body, int64_t nsteps);

/* Step until KE < ke_ratio * KE_max (KE over free particles, FP64, tested
 * after every step) or max_steps more steps; the state stops at the step that
 * met the criterion.  SRDR_ERR_NOT_CONVERGED at the cap, SRDR_ERR_NONFINITE if
 * KE became non-finite, SRDR_ERR_TIMEOUT if a bounded wait of the damping
 * sweep ran out (see srdr_body_sweep_sync).  steps_taken / final_ke_ratio may
 * be NULL. */
srdr_status srdr_body_relax(srdr_body* body, double ke_ratio, int64_t max_steps,
                            int64_t* steps_taken, double* final_ke_ratio);

/* Displacement u^n (resp. velocity v^n) at the current full step into
 * host_out[n][3], original order; n_doubles must be >= 3 n. Synchronises. */
srdr_status srdr_body_read_displacement(const srdr_body* body, double* host_out, size_t n_doubles);
srdr_status srdr_body_read_velocity(const srdr_body* body, double* host_out, size_t n_doubles);

/* Overwrite the state at the current full step (checkpoint restore / test
 * set-up): u[n][3] and v[n][3] in original order, either may be NULL. */
srdr_status srdr_body_write_state(srdr_body* body, const double* u, const double* v,
                                  int64_t step_index, double ke_max);

/* Sizes: particles, neighbour pairs, non-empty cells, time step; any may be NULL. */
srdr_status srdr_body_info(const srdr_body* body, int64_t* n_particles, int64_t* nnz,
                           int* n_cells, double* dt);

typedef struct {
    int64_t step;          /* steps taken since creation */
    int64_t damped_steps;  /* steps on which S_d ran */
    double ke, ke_max;     /* last step's KE and the running maximum */
    double eta, dt;        /* artificial viscosity and time step */
    int converged;         /* last relax met its criterion */
    int64_t launches;      /* kernels launched by step / relax calls since creation */
    int sweep_cells_per_warp; /* damping-sweep mapping picked by the autotuner (1, 2, 4) */
    int pass_mapping;      /* mapping the stress and force passes use: SRDR_PASS_STENCIL,
                              SRDR_PASS_SELL or SRDR_PASS_BRICKS (SRDR_PASS_AUTO before
                              the first step of a body without the stencil) */
    int sweep_sync;        /* synchronisation of the sweep's colour phases in use:
                              SRDR_SWEEP_CELLS or SRDR_SWEEP_BARRIER (SRDR_SWEEP_AUTO
                              before the first damped step) */
} srdr_stats;
srdr_status srdr_body_stats(const srdr_body* body, srdr_stats* out);

/* Inspection of the build for tests: neighbour CSR (row_ptr[n+1], col[nnz],
 * original ids, rows ascending), cell id and colour per particle, and the
 * canonical sweep order (original ids sorted by colour, cell, id). */
srdr_status srdr_body_read_neighbours(const srdr_body* body, int64_t* row_ptr, int64_t* col);
srdr_status srdr_body_read_cells(const srdr_body* body, int64_t* cell, int* colour,
                                 int64_t* order);

enum { SRDR_FIELD_PB = 0, SRDR_FIELD_B0 = 1 };
/* Per-particle 3x3 fields, row-major [n][3][3], original order: P B0 from the
 * last stress pass, or the correction matrix B0. */
srdr_status srdr_body_read_field(const srdr_body* body, int field, double* host_out,
                                 size_t n_doubles);

/* Kernel timing with CUDA events recorded on the body's stream around each
 * kernel class of the timed steps (the damping sweep class spans the whole
 * S_d of a damped step).  srdr_body_profile(body, k) with k > 0 clears the
 * records and times every k-th step (steps whose index is a multiple of k:
 * k = 1 times all of them; a larger k keeps the events' own cost out of most
 * steps, and the random choice makes the sample of damped steps unbiased);
 * k = 0 stops.  srdr_body_kernel_times synchronises and returns the
 * accumulated device milliseconds and timed intervals per class and the
 * launches of all steps since the profile call.  Profiled stepping launches
 * every step directly (no graph replay).  The kinetic-energy reduction is
 * part of the force pass (undamped step) or of the finish pass (damped step)
 * on the sliced-ELL mapping; SRDR_K_KE times the separate KE kernels of the
 * brick-tiled mapping. */
enum { SRDR_K_PASS_A = 0, SRDR_K_PASS_B = 1, SRDR_K_SWEEP = 2, SRDR_K_FINISH = 3, SRDR_K_KE = 4,
       SRDR_K_NCLASS = 5 };
typedef struct {
    double ms[SRDR_K_NCLASS];
    int64_t launches[SRDR_K_NCLASS];
    int64_t intervals[SRDR_K_NCLASS];
} srdr_kernel_times;
srdr_status srdr_body_profile(srdr_body* body, int enable);

/* Kernel mapping of the damping sweep: sweep_cells_per_warp = 1, 2 or 4 cells
 * per warp and sweep_warps_per_block = 1 or 4, or both 0 to let the
 * autotuner time G = 1, 2 with W = 1, 4 on the body's first damped step (the
 * default).  The choice changes speed only: the sweep's sums follow one fixed
 * order, so results are bitwise the same. */
srdr_status srdr_body_tune(srdr_body* body, int sweep_cells_per_warp, int sweep_warps_per_block);

/* Synchronisation of the damping sweep's colour phases (Sec. 3.4: cells of
 * one colour run concurrently, colours one after another).
 * SRDR_SWEEP_BARRIER: a grid barrier between consecutive colour phases.
 * SRDR_SWEEP_CELLS: no barrier; before each of its phases a cell waits only
 * for the cells whose footprints overlap its own (within 2 cells on every
 * axis) to have finished their earlier phases, so the order of every pair of
 * cells that interact is the canonical one.  SRDR_SWEEP_AUTO (the default):
 * the autotuner times cell-wise waits with one cell per warp and grid
 * barriers with one or two (with more cells per warp, a warp's groups would
 * take turns: one polling while the other's chain waits); a mapping fixed by
 * srdr_body_tune uses cell-wise waits for one cell per warp and grid
 * barriers otherwise.  A batch uses the mode all of its bodies ask for, else
 * its own autotuner's choice.
 * Results are bitwise the same under every choice.  Every wait is bounded
 * (five seconds); a sweep whose wait runs out sets the body's status, and
 * srdr_body_relax returns SRDR_ERR_TIMEOUT after resetting the
 * synchronisation words (the velocity state is then that of a partial sweep:
 * restore it with srdr_body_write_state).  Returns SRDR_ERR_INVALID for
 * another mode. */
enum { SRDR_SWEEP_AUTO = 0, SRDR_SWEEP_BARRIER = 1, SRDR_SWEEP_CELLS = 2 };
srdr_status srdr_body_sweep_sync(srdr_body* body, int mode);

/* Width of the damping sweep's serial chain (Sec. 3.1's local update of one
 * particle after another, Sec. 3.4's colour sweep): the cell-wise sweep runs
 * one cell per warp, and the chain of a cell's particle updates uses 32 lanes
 * (each row's neighbours spread over 32 lanes, a 5-level reduction per
 * update) or 16 (one reduction level fewer, the whole warp still waiting,
 * copying and writing back).  The sums follow the same 32-lane order either
 * way, so results are bitwise the same.  lanes = 0 (the default) lets the
 * autotuner choose; 16 or 32 fixes it (with cell-wise waits, one cell per
 * warp, the warps per block of srdr_body_tune).  SRDR_ERR_INVALID for another
 * value or when the body asks for grid barriers (srdr_body_sweep_sync). */
srdr_status srdr_body_sweep_lanes(srdr_body* body, int lanes);

/* Test hook of the failure path above: makes every wait of the body's next
 * damping sweep run out (it sets the synchronisation words to counts that no
 * cell reaches), so that the sweep ends with the body's status set after
 * about five seconds.  Nothing else changes; the next srdr_body_relax reports
 * SRDR_ERR_TIMEOUT and resets the words. */
srdr_status srdr_body_debug_stall_sweep(srdr_body* body);

/* Kernel mapping of the stress and force passes (Sec. 2.2-2.3 and the
 * momentum equation).  SRDR_PASS_SELL: each thread streams its particle's
 * neighbour row from a sliced-ELL layout and gathers the neighbours' data
 * from global memory.  SRDR_PASS_BRICKS: one thread block per brick of
 * brick_x x brick_y x brick_z cells stages the data of the brick's cell
 * halo in shared memory and streams 16-bit halo indices; the layout is built
 * on the first step after the call (brick sizes 1..4 cells, 0 = default
 * 2 x 2 x 2 in 3D, 4 x 4 in 2D; SRDR_ERR_INVALID at that step if a brick's
 * halo does not fit in shared memory).  SRDR_PASS_AUTO (the default): the
 * sliced-ELL mapping, measured faster on GB300 for every body tried (the
 * brick layout is then not built).  Both visit a row's neighbours in the
 * same order with the same roundings, so results are bitwise the same; the
 * choice changes speed only.  SRDR_PASS_STENCIL is the mapping of bodies that
 * took the lattice stencil at creation (pass_layout above): neighbour k of
 * the particle at lattice point p is the particle at p + o_k when that point
 * lies in the box, with the pair gradient of offset o_k from a table; no
 * neighbour stream is read, and a warp's 32 threads are consecutive lattice
 * points, so a warp's gathers of one offset are consecutive records.  Such a
 * body keeps its particle arrays in lattice order and refuses the other two
 * mappings (SRDR_ERR_INVALID); create it with pass_layout =
 * SRDR_PASS_LAYOUT_SELL to use them. */
enum { SRDR_PASS_AUTO = 0, SRDR_PASS_SELL = 1, SRDR_PASS_BRICKS = 2, SRDR_PASS_STENCIL = 3 };
srdr_status srdr_body_pass_mapping(srdr_body* body, int mapping, int brick_x, int brick_y,
                                   int brick_z);
srdr_status srdr_body_kernel_times(const srdr_body* body, srdr_kernel_times* out);

void srdr_body_destroy(srdr_body* body);

/* Particles of the lattice body that srdr_body_create would build from desc. */
srdr_status srdr_desc_particle_count(const srdr_body_desc* desc, int64_t* n_particles);

/* ---------------------------------------------------------------- batches
 * Many bodies of uneven sizes relaxed together.  Each body keeps its own
 * device arrays; one batched step runs the stress pass, the force pass, the
 * damping sweep (Sec. 3.1, on the bodies whose random choice damps this
 * step, Sec. 3.3) colour-synchronised across the whole batch in one
 * cooperative launch (Sec. 3.4), the displacement update and a per-body FP64
 * kinetic-energy reduction, all bodies in shared launches captured as CUDA
 * graphs.  A body's result is bitwise the same alone or in a batch.  The
 * bodies must share dimension and precision; material, damping, alpha, seed,
 * time step and size may differ. */
typedef struct srdr_batch srdr_batch;

/* Group existing bodies (caller-owned; they must outlive the batch).  The
 * batch works on cuda_stream, or on a stream of its own if it is NULL. */
srdr_status srdr_batch_create(srdr_body* const* bodies, int nbodies, void* cuda_stream,
                              srdr_batch** out);
/* nsteps batched steps of every body. */
srdr_status srdr_batch_step(srdr_batch* batch, int64_t nsteps);
/* Relax: every body retires at its own criterion KE < ke_ratio * KE_max
 * (its work is then skipped and the work lists compacted); at most max_steps
 * steps.  per_body_status[n] (SRDR_OK, SRDR_ERR_NOT_CONVERGED,
 * SRDR_ERR_NONFINITE) and per_body_steps[n] may be NULL.  Returns the first
 * non-OK per-body status, or SRDR_ERR_TIMEOUT if a grid barrier gave up. */
srdr_status srdr_batch_run(srdr_batch* batch, double ke_ratio, int64_t max_steps,
                           srdr_status* per_body_status, int64_t* per_body_steps);
/* How a batch runs its bodies' steps.
 * SRDR_BATCH_SHARED: the shared launches described above (one stress pass,
 * one force pass, one colour-synchronised sweep ... per step for all bodies).
 * SRDR_BATCH_STREAMS: every body runs its own step kernels (those of
 * srdr_body_step, graph replays for small bodies) on one of up to 64 streams
 * of the batch, all bodies at the same time, in chunks of steps after which
 * the host retires the bodies that met their criterion.  A damped step's
 * sweep is a chain of dependent colour phases (Sec. 3.4) about as long for a
 * small body as for a large one; concurrent bodies overlap these chains,
 * where shared launches make every body wait at every step for the slowest
 * damped body.  SRDR_BATCH_AUTO (the default) is SRDR_BATCH_STREAMS, measured
 * faster on GB300 (2x to 4.5x on uneven bodies).  Results are bitwise the same
 * in every mode and equal to the bodies relaxed alone.  SRDR_BATCH_SHARED
 * takes sliced-ELL bodies only (bodies created with pass_layout =
 * SRDR_PASS_LAYOUT_SELL, or not on a box lattice); a batch holding a
 * lattice-stencil body refuses it.  SRDR_ERR_INVALID for another mode. */
enum { SRDR_BATCH_AUTO = 0, SRDR_BATCH_SHARED = 1, SRDR_BATCH_STREAMS = 2 };
srdr_status srdr_batch_mode(srdr_batch* batch, int mode);
/* Steps run, kernels launched, and the autotuner's choices (damping-sweep
 * cells per warp, threads per block of the passes); any may be NULL. */
srdr_status srdr_batch_info(const srdr_batch* batch, int64_t* steps, int64_t* launches,
                            int* sweep_cells_per_warp, int* pass_threads);
/* Frees the batch (not the bodies it was created from). */
void srdr_batch_destroy(srdr_batch* batch);

/* ---------------------------------------------------------------- serving
 * Relaxation requests served with continuous batching.  submit() queues a
 * lattice body description (any host thread).  A worker thread admits queued
 * requests while the number of live bodies is below max_bodies and their
 * estimated device memory fits the budget, relaxes all live bodies together
 * as one batch in chunks of steps, retires each body when its own KE falls
 * below ke_ratio * KE_max (or after max_steps: SRDR_ERR_NOT_CONVERGED),
 * copies its displacement to the host, frees its memory and admits the next
 * requests.  Each result is bitwise the same as the same body relaxed alone
 * (srdr_body_relax).  Internally synchronised. */
typedef struct srdr_server srdr_server;
typedef struct {
    int64_t submitted;
    int64_t completed;            /* solves: requests that met their KE criterion (SRDR_OK) */
    int64_t refused, queued, in_flight;
    int peak_concurrent;          /* most bodies live at once */
    size_t bytes_in_use;          /* admitted device-memory estimate */
    int64_t particle_steps;       /* over all finished chunks */
    double p50_latency_s, p99_latency_s;  /* submit -> result, solves only */
    double solves_per_s;          /* completed / (last retirement of any request - first submit) */
    int64_t not_converged;        /* retired at max_steps (SRDR_ERR_NOT_CONVERGED): not solves */
    int64_t failed;               /* retired with another error (non-finite KE, build failure) */
} srdr_server_report;

/* device_mem_budget: bytes the live bodies may hold; cuda_stream as for bodies
 * (NULL: the server makes its own).  Defaults: ke_ratio 1e-8, max_steps 1e6,
 * max_bodies 256, chunks of 256 steps, queue of 4096. */
srdr_status srdr_server_create(size_t device_mem_budget, void* cuda_stream, srdr_server** out);
srdr_status srdr_server_configure(srdr_server* server, double ke_ratio, int64_t max_steps,
                                  int max_bodies, int64_t chunk_steps, size_t queue_capacity);
/* SRDR_ERR_BUSY if the queue is full, SRDR_ERR_NO_MEMORY if the request alone
 * exceeds the budget. */
srdr_status srdr_server_submit(srdr_server* server, const srdr_body_desc* desc, uint64_t* ticket);
/* SRDR_ERR_BUSY while the request is unfinished; else its final status, with
 * the displacement (3 n doubles, original order) in host_disp_out (may be
 * NULL) and the submit-to-result latency.  A result is handed out once. */
srdr_status srdr_server_poll(srdr_server* server, uint64_t ticket, double* host_disp_out, size_t n,
                             double* latency_s);
/* As poll, blocking up to timeout_s; steps (may be NULL) = steps taken. */
srdr_status srdr_server_wait(srdr_server* server, uint64_t ticket, double timeout_s,
                             double* host_disp_out, size_t n, double* latency_s, int64_t* steps);
srdr_status srdr_server_stats(srdr_server* server, srdr_server_report* out);
/* Stops the worker after its current chunk; unfinished requests are dropped. */
void srdr_server_destroy(srdr_server* server);

/* One call: build lattice bodies from descs[nbodies], relax them as a batch,
 * copy each displacement into host_disp_out[b] (caller-owned, 3 n_b doubles
 * with n_b from srdr_desc_particle_count; NULL entries are skipped), free
 * everything. */
srdr_status srdr_batch_relax(const srdr_body_desc* descs, int nbodies, double ke_ratio,
                             int64_t max_steps, double** host_disp_out,
                             srdr_status* per_body_status);
const char* srdr_last_error(void);

/* Kinetic energy sum_i 1/2 m_i |v_i|^2 over the particles without
 * SRDR_FLAG_CONSTRAINED, in FP64, computed WITHOUT ALLOCATING any device
 * memory.  The paper has no counterpart: this entry point exists for callers
 * that cannot call cudaMalloc, such as codes whose device memory all belongs
 * to their own pool or arena, or services that fix their device-memory
 * footprint at start-up and refuse allocations afterwards.
 *
 * v: device array [3][n] (SoA: all x, then all y, then all z), mass: device
 * [n], both FP64 when precision == SRDR_FP64 and FP32 when
 * precision == SRDR_FP32_MIXED; flags: device [n] uint8 SRDR_FLAG_* bits or
 * NULL (all free); ke_out: device pointer to one double.  All are owned by
 * the caller.  The work is queued on cuda_stream and is complete when that
 * stream is.
 *
 * The scratch space is a fixed array of 16384 FP64 partial sums (128 KiB)
 * compiled into the library; every GPU that loads the library holds it until
 * the process exits.  One partial covers 256 particles, so n may be at most
 * 4,194,304; larger n returns SRDR_ERR_INVALID.  Every call made outside
 * stream capture looks up the array's device address in the current context
 * (cudaGetSymbolAddress; the address changes with the context, e.g. after
 * cudaDeviceReset); a call on a capturing stream reuses the address of the
 * last call on that device outside capture, so make the first call on each
 * device before any stream capture.  Each particle's term 1/2 m |v|^2 is
 * rounded as in the library's own reduction.  All calls
 * share the one array: calls whose GPU work overlaps (different streams, or
 * different host threads on one device) race and may return wrong sums, so
 * order them on one stream.  Each call writes every partial it reads before
 * reading it, so nothing is left over from an earlier call. */
srdr_status srdr_kinetic_energy_noalloc(const void* v, const void* mass, const uint8_t* flags,
                                        int64_t n, int precision, double* ke_out,
                                        void* cuda_stream);

/* The library's own Philox4x64-10 (host side of the device routine):
 * out[4] = Philox4x64-10(counter, key) and phi_n of the random choice. */
void srdr_philox4x64_10(const uint64_t counter[4], const uint64_t key[2], uint64_t out[4]);
double srdr_random_phi(uint64_t seed, uint64_t step);

#ifdef __cplusplus
}
#endif
#endif
