// srdr_internal.cuh — internal types and device helpers of the srdr library
// (splitting random-choice dynamic relaxation for TL-SPH, arXiv 2103.08932).
//
// Data layout in HBM (all per-particle arrays in SORTED order: particles
// sorted by (cell id, original id), the canonical order of the splitting
// cell-linked list):
//   r0    FP64 [3][n] SoA reference positions
//   u     FP64 [n][4] (FP64 mode) or FP32 hi and lo (FP32 mode: (hi x, y,
//         z, lo x) [n][4] and (lo y, lo z) [n][2], u = hi + lo), held at
//         the half step u^{n+1/2}; AoS so that one neighbour gather is a
//         16-byte and an 8-byte load (FP32) or two 16-byte loads (FP64)
//   v     T [n][4] velocity records (vx, vy, vz, 1/m): one 16-byte (FP32) or
//         two 16-byte (FP64) accesses per particle
//   B0    T [D*D][n] row-major tensor components, SoA (read by the owner only)
//   PB    T [pb_full][n] 16-byte chunks of the row-major entries, then
//         [pb_tail][n] leftover entries (gathered)
//   G     T [3][n]   sum_j V_j grad W_ij (for the difference form of the force)
//   CSR   row_ptr int32 [n+1], col int32 [nnz] (sorted ids, ascending),
//         loc uint16 [nnz] (index of j inside the 3^d-cell footprint of
//         cell(i)), w T [nnz] = V_i V_j W'(r)/r  (damping sweep)
//   SELL  32-row slices: sell_ptr int32 [nslices+1], sell_col int32 [slots],
//         sell_g T [3][slots] = g_ij = V_j grad0_i W_ij (stress and force passes)
//   cpos  T [n][4] offset inside its cell and volume V; ccell int32 [n]
//         packed cell coordinates: g_ij and G_i = sum_j g_ij are evaluated
//         from them by one rounding-exact formula (pairg.cuh)
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/srdr.h"

namespace srdr {

void set_error(const char* fmt, ...);

#define SRDR_CK(call)                                                                      \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess) {                                                           \
            ::srdr::set_error("%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, \
                              __LINE__);                                                   \
            return SRDR_ERR_CUDA;                                                          \
        }                                                                                  \
    } while (0)

#define SRDR_TRY(call)                         \
    do {                                       \
        srdr_status s_ = (call);               \
        if (s_ != SRDR_OK) return s_;          \
    } while (0)

// device-side scalars of one body, updated by the kernels
struct DevScalars {
    double ke;
    double ke_max;
    double tol;            // relax criterion (0: never done)
    long long step;        // steps completed
    long long damped;      // damped steps completed
    int done;              // criterion met or error: later step kernels skip
    int status;            // 0, or a device error code (SRDR_ERR_*)
    long long err_index;   // first offending particle / cell for status
    unsigned ke_ticket;    // blocks of the current KE-writing kernel that have finished (0 between kernels)
    int pad_;
};

// FP32-mixed displacement: u = hi + lo per component, hi = fl(u) and
// lo = fl(u - hi), stored as uhi [n][4] = (hi x, hi y, hi z, lo x) and
// ulo [n][2] = (lo y, lo z).  u then carries about 48 significant bits; a
// neighbour gather is one 16-byte and one 8-byte load with nothing to decode.

// 1/2 m |v|^2 of one particle with explicit roundings: the same bits in
// every kernel that evaluates it (no contraction choice left to the
// compiler)
template <typename T>
__device__ inline double ke_particle(T m, const T (&v)[3])
{
    if constexpr (sizeof(T) == 4) {
        const float s = __fmaf_rn(v[2], v[2], __fmaf_rn(v[1], v[1], __fmul_rn(v[0], v[0])));
        return (double)__fmul_rn(__fmul_rn(0.5f, m), s);
    } else {
        const double s = __fma_rn(v[2], v[2], __fma_rn(v[1], v[1], __dmul_rn(v[0], v[0])));
        return __dmul_rn(__dmul_rn(0.5, m), s);
    }
}

// grid-barrier buffer: kBarSub arrival sub-counters, a top counter and a
// generation word, each on its own 128-byte line
constexpr int kBarSub = 32;
constexpr int kBarWords = 32 * (kBarSub + 2);

// One brick of the tiled passes: its index in the brick grid, the offsets of
// its own particles (brick order), halo list and brick-sliced-ELL slices,
// and its particle counts.
struct BrickInfo {
    int q, own_base, halo_base, slice_base, nown, nhalo, pad0, pad1;
};

// device error codes written to DevScalars::status
enum { DEV_OK = 0, DEV_SINGULAR_B0 = 1, DEV_NONFINITE = 2, DEV_TIMEOUT = 3 };

// neighbour slots per batch of loads in the passes; lattice-stencil tables
// are padded to a multiple of it
constexpr int kStencilBatch = 8;

// The lattice stencil as a kernel parameter (constant bank), for the usual
// offset counts: K offsets with their index delta, lattice step and pair
// gradient.  K = 80 in 3D and 24 in 2D for h = 1.3 dp (20 offsets padded).
template <typename T, int K>
struct StencilTab {
    int delta[K];
    int dx[K], dy[K], dz[K];
    T g[K][3];
    int reach;  // the largest |component| of an offset
};
constexpr int kStencilK3 = 80;
constexpr int kStencilK2 = 24;

template <typename T>
struct StepArgs {
    int n;
    const int* __restrict__ sell_ptr;
    const int* __restrict__ sell_col;
    const T* __restrict__ g0;   // [slots] V_j grad0_i W_ij, x component (sliced ELL)
    const T* __restrict__ g1;   // y component
    const T* __restrict__ g2;   // z component
    const T* __restrict__ cpos;   // [n][4] offset in its cell (x, y, z) and volume
    const int* __restrict__ ccell; // [n] packed cell coordinates x | y << 10 | z << 20
    const T* __restrict__ B0;   // [D*D][n]
    T* __restrict__ PB;         // [pb_full][n] 16-byte chunks, [pb_tail][n] entries
    const T* __restrict__ Gs;   // [3][n]
    const T* __restrict__ dvisc; // [n][4] explicit comparator: dt a_visc(v^n), else null
    const T* __restrict__ bf;    // [n][4] per-particle body force (twist), else null
    const int* dflag;            // device-decided damping of this step (graph replay), else null
    T* __restrict__ v;          // [n][4] (vx, vy, vz, 1/m)
    double* __restrict__ u;     // [3][n] FP64 mode
    float* __restrict__ uhi;    // [n][4] FP32 mode: (hi x, y, z, lo x), u = hi + lo
    float* __restrict__ ulo;    // [n][2] FP32 mode: (lo y, lo z)
    const uint8_t* __restrict__ flags;
    const T* __restrict__ mass;
    double* __restrict__ ke_part;
    DevScalars* sc;
    T lambda, mu, inv_rho0, dt;
    T rc, inv_h, kc;             // cell edge, 1/h, -5 alpha_d / h^2
    T grav[3];
    T endl[3];
    // lattice stencil (bodies on a box lattice of lx x ly x lz points, x
    // fastest, particle index = lattice index): neighbour k of particle i is
    // i + st_off[k].w where the lattice point (x, y, z) + st_off[k].xyz lies
    // in the box, with the pair gradient st_g[k] (T [st_k][4]); st_k is a
    // multiple of the passes' batch, padded with zero offsets.  Null for the
    // sliced-ELL and brick mappings.
    const int4* __restrict__ st_off;
    const T* __restrict__ st_g;
    int st_k;
    int lx, ly, lz;
    // stencil bodies: the damping sweep's copy of the velocity records in
    // sorted order (T [n][4]) and particle -> sorted index.  The force pass
    // of a damped step writes v* there, the sweep works on it, and the
    // finish pass copies the damped velocities back to v.  Null otherwise.
    T* __restrict__ vs;
    const int* __restrict__ inv;
};

// One slot of a damping-sweep row: B_j = c w_ij, pre-scaled by the body's
// c = eta~ dt (the same product the sweep would form, rounded once), and the
// footprint-local index of j, so that the sweep reads a slot with one 8-byte
// (FP32) or 16-byte (FP64) shared-memory load
template <typename T>
struct SweepSlot;
template <>
struct __align__(8) SweepSlot<float> {
    float B;
    unsigned loc;
};
template <>
struct __align__(16) SweepSlot<double> {
    double B;
    unsigned loc;
    unsigned pad;
};

template <typename T>
struct SweepArgs {
    int n;
    int dim;
    int nx, ny, nz;
    const int* __restrict__ cell_start;
    const int* __restrict__ colour_cells;  // cells of this colour
    const int* __restrict__ row_ptr;
    const uint16_t* __restrict__ loc;
    const T* __restrict__ w;
    const SweepSlot<T>* __restrict__ rec;  // [nnz + 2] (B_j, footprint-local j) per row entry
    const T* __restrict__ mass;  // [n] sorted order
    const T* __restrict__ sbm;   // [n] sum_j B_j - m_i of the local solve (Sec. 3.1)
    const T* __restrict__ srd;   // [n] 1 / ((sum_j B_j - m_i)^2 + sum_j B_j^2)
    T* __restrict__ v;           // [n][4] sorted order (a stencil body's sorted copy)
    DevScalars* sc;
    const int* dflag;  // device-decided damping of this step (graph replay), else null
    T c;          // 2 eta~ dt_loc, so that B_j = c w_ij
    int cbase;    // colour base: 3 (3^d colours) or 2 (2^d colours over cells of edge 2 r_c)
    int wrad;     // cells within wrad on every axis may touch common particles (2, or 1)
    const int* __restrict__ foot_ptr;  // 2^d layout: touched lists per cell, else null
    const int* __restrict__ foot_tab;
    const int* __restrict__ own_off;
    int rows_global;  // 1: the cells' slot records are read from global memory, not staged
    int pairwise;
    int max_foot;
    int max_pairs;
    int max_cell;
};

}  // namespace srdr

// ---------------------------------------------------------------- the body
struct srdr_body {
    srdr_body_desc desc;
    int dim = 3;
    int prec = SRDR_FP64;
    int64_t n = 0, nnz = 0;
    int nc[3] = {1, 1, 1};
    int ncells = 0, ncells_nonempty = 0, ncolours = 0;
    cudaStream_t stream = nullptr;
    double h = 0, rc = 0, lambda = 0, mu = 0, eta = 0, dt = 0, vol0 = 0;
    double cut = 0;   // neighbour cut-off 2h (rc is the cell edge: cut, or 2 cut in the 2^d layout)
    int cbase = 3;    // colour base of the sweep layout: 3 (3^d colours) or 2 (2^d colours)
    // 2^d layout: the particles each cell's sweep touches (its own and their
    // neighbours, ascending sorted index), foot_tab[foot_ptr[c] ..
    // foot_ptr[c+1]-1], and the position of the cell's first particle in it;
    // null in the paper's layout, whose footprint is the 3^d neighbour cells
    int* foot_ptr = nullptr;
    int* foot_tab = nullptr;
    int* own_off = nullptr;
    double lo[3] = {0, 0, 0};
    // lattice stencil of the passes (bodies on a box lattice whose neighbour
    // lists the stencil reproduces): the particle arrays are then in lattice
    // (= original) order; the sweep keeps sorted-order copies of the masses
    // and velocity records
    int stencil = 0;
    int lat[3] = {0, 0, 0};     // lattice points per axis (0: not a lattice body)
    int st_k = 0;               // offsets, padded to a multiple of the passes' batch
    int4* st_off = nullptr;     // [st_k] (dx, dy, dz, index delta)
    void* st_g = nullptr;       // T [st_k][4] pair gradient of each offset
    std::vector<int4> st_off_h;    // host copies of the table (kernel-parameter tables)
    std::vector<double> st_g_h;    // [st_k][4], the values st_g holds before rounding to T
    int* pidx = nullptr;        // sorted -> particle index (= perm), stencil bodies only
    void* mass_sw = nullptr;    // T [n] masses in sorted order (the sweep's), stencil bodies only
    void* vs = nullptr;         // T [n][4] velocity records in sorted order (the sweep's), stencil bodies only

    // device arrays
    int* perm = nullptr;        // sorted -> original
    int* inv = nullptr;         // original -> sorted
    // particle-array index -> original (perm, or null: the identity for
    // lattice-stencil bodies, whose arrays are in original order)
    const int* io_perm() const { return stencil ? nullptr : perm; }
    int* cell_start = nullptr;  // [ncells+1]
    int* cell_of = nullptr;     // [n] cell id, sorted order
    int* colour_cells = nullptr;
    std::vector<int> colour_ptr;  // host [ncolours+1]
    double* r0 = nullptr;       // [3][n]
    uint8_t* flags = nullptr;   // [n]
    void* mass = nullptr;       // T [n]
    void* minv = nullptr;       // T [n] 1 / mass
    int* row_ptr = nullptr;
    int* col = nullptr;
    uint16_t* loc = nullptr;
    void* w = nullptr;          // T [nnz]
    int nslices = 0;
    int64_t nslots = 0;
    int* sell_ptr = nullptr;
    int* sell_col = nullptr;
    void* sell_g = nullptr;     // T [3][slots] pair gradients in sliced-ELL order
    void* cpos = nullptr;       // T [n][4] offset in its cell and volume
    int* ccell = nullptr;       // [n] packed cell coordinates
    void* B0 = nullptr;         // T [D*D][n]
    void* PB = nullptr;
    void* Gs = nullptr;         // T [3][n]
    void* sumw = nullptr;
    void* sumw2 = nullptr;
    void* srec = nullptr;        // SweepSlot<T> [nnz + 2] pre-scaled sweep slots (prepare_sweep)
    void* sbm = nullptr;         // T [n] per-particle constants of the local solve
    void* srd = nullptr;         //   (prepare_sweep; B_j = c w_ij with the body's c)
    void* v = nullptr;          // T [n][4] (vx, vy, vz, 1/m)
    double* u = nullptr;        // FP64 [3][n]
    float* uhi = nullptr;       // [n][4] FP32 mode: (hi x, y, z, lo x)
    float* ulo = nullptr;       // [n][2] FP32 mode: (lo y, lo z)
    double* ke_part = nullptr;
    int ke_blocks = 0;
    srdr::DevScalars* sc = nullptr;
    srdr::DevScalars* sc_host = nullptr;  // pinned mirror

    int pb_stride = 0;               // T elements per particle in PB
    int max_foot = 0, max_pairs = 0, max_cell = 0;  // per-cell maxima
    int* colour_ptr_d = nullptr;     // device copy of colour_ptr
    unsigned* bar = nullptr;         // grid-barrier counters and generation [kBarWords]
    // brick-tiled passes (built lazily on the first step that needs them)
    int pass_mapping = SRDR_PASS_AUTO;  // requested
    int pass_tiled = -1;             // in use: -1 undecided, 0 sliced ELL, 1 bricks
    int brick[3] = {0, 0, 0};        // requested brick size in cells (0: default)
    int bricks_built = 0;            // 1 built, -1 does not fit
    int nbricks = 0, max_halo = 0, max_own = 0, nbslices = 0;
    int64_t bslots = 0;
    srdr::BrickInfo* binfo = nullptr;  // [nbricks]
    int* bown = nullptr;             // [n] sorted index of own particle k (brick order)
    uint16_t* bown_h = nullptr;      // [n] its halo index
    int* bhalo = nullptr;            // [sum of halos] sorted index of halo particle h
    int* bsell_ptr = nullptr;        // [nbslices + 1] slot offsets of the brick slices
    uint16_t* blidx = nullptr;       // [bslots] halo index of the neighbour in each slot
    void* bg = nullptr;              // T [3][bslots] pair gradients
    double* ke_pp = nullptr;         // [n] kinetic energy per particle (tiled pass B)
    void* dvisc = nullptr;           // T [n][4] explicit comparator: dt a_visc(v^n)
    void* bf = nullptr;              // T [n][4] rotational body force per particle (twist)
    int sweep_cells_per_warp = 2;    // cells per warp of the sweep kernel (1, 2, 4)
    int sweep_warps_per_block = 1;   // warps per block of the sweep kernel (1, 4)
    int sweep_chain16 = 0;           // cell-wise sweep with the chain on 16 lanes of each warp
    int sweep_tuned = 0;
    int sweep_smem = 0;
    int sweep_rows_global = 0;       // slot records read from global memory (staging does not fit)
    int sweep_sync = SRDR_SWEEP_AUTO;  // requested synchronisation of the sweep's colour phases
    int sweep_cellwise = 1;            // the one in use: cell-wise waits (1) or grid barriers (0)
    unsigned* flow = nullptr;          // cell-wise synchronisation words (k_sweep_flow)

    // host mirrors
    int64_t step = 0;
    int converged = 0;
    int64_t launches = 0;

    // kernel-class timing (CUDA events on the body stream)
    int profiling = 0;               // 0 off, k > 0: time every k-th step
    int prof_active = 0;             // the step being enqueued is timed
    // replay of captured multi-step graphs (small bodies, damping decided on
    // the device): the flag word, the graph, its step count, availability
    int* dflag_d = nullptr;
    cudaGraphExec_t graph = nullptr;
    int graphs_ok = 1;
    int64_t graph_launches[SRDR_K_NCLASS] = {0, 0, 0, 0, 0};  // kernels per graph replay
    std::vector<cudaEvent_t> ev_pool;
    std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> ev_marks;
    size_t ev_next = 0;
    int64_t k_launch[SRDR_K_NCLASS] = {0, 0, 0, 0, 0};

    std::vector<void*> allocs;
};

namespace srdr {

srdr_status dev_alloc(srdr_body* b, void** p, size_t bytes);
// a tuned batch's launch configuration (batch.cu), for the next batch of a
// continuous-batching loop: {tuned, cells per warp, cell-wise, pass threads}
void batch_get_tuning(const srdr_batch* bt, int cfg[4]);
void batch_set_tuning(srdr_batch* bt, const int cfg[4]);
srdr_status dev_free(srdr_body* b, void* p);
template <typename P>
inline srdr_status dalloc(srdr_body* b, P** p, size_t count)
{
    return dev_alloc(b, reinterpret_cast<void**>(p), count * sizeof(P));
}

// -5 alpha_d / h^2 of the Wendland C2 kernel: W'(r)/r = kc (1 - r/(2h))^3,
// alpha_2 = 7 / (4 pi h^2), alpha_3 = 21 / (16 pi h^3)
inline double kernel_kc(int dim, double h)
{
    const double pi = 3.14159265358979323846;
    const double a = dim == 2 ? 7.0 / (4.0 * pi * h * h) : 21.0 / (16.0 * pi * h * h * h);
    return -5.0 * a / (h * h);
}

// cell-wise synchronisation words of the sweep: a counter per cell of the
// grid, then the epoch at flow_epoch_word and the finished-group count 32
// words later (each on its own 128-byte line)
__host__ __device__ inline int flow_epoch_word(int ncells) { return (ncells + 31) & ~31; }
__host__ __device__ inline int flow_words(int ncells) { return flow_epoch_word(ncells) + 64; }

// P B0 layout: the dim x dim entries of a particle, row-major, as pb_full
// whole 16-byte chunks (FP32 3D: 2, FP64 3D: 4, FP32 2D: 1, FP64 2D: 2) and
// pb_tail leftover entries (3D: 1, 2D: 0).  Chunk c of all particles is one
// dense array (chunk c of particle j at 16-byte index c n + j); leftover
// entry t of particle j sits at T index (pb_full E + t) n + j, E = 16 / T.
__host__ __device__ constexpr int pb_full(size_t tsize, int dim) { return (int)(dim * dim * tsize / 16); }
__host__ __device__ constexpr int pb_tail(size_t tsize, int dim)
{
    return dim * dim - pb_full(tsize, dim) * (int)(16 / tsize);
}
// 16-byte chunks covering one particle's entries (a padded record in the
// brick-tiled passes' shared memory: FP32 3D: 3, FP64 3D: 5, 2D: 1 or 2)
__host__ __device__ constexpr int pb_chunks(size_t tsize, int dim)
{
    return (int)((dim * dim * tsize + 15) / 16);
}
// T elements per particle in PB
inline int pb_stride(size_t tsize, int dim) { return pb_full(tsize, dim) * (int)(16 / tsize) + pb_tail(tsize, dim); }

// setup (setup.cu)
srdr_status build_body(srdr_body* b, int64_t n, const double* r0, const double* vol,
                       const uint8_t* flags, const double* u0);
// per-particle constants of the damping sweep's local solve for the body's
// current eta~ and dt (setup.cu): sbm = c sum_j w_ij - m_i and
// srd = 1 / (sbm^2 + c^2 sum_j w_ij^2) with c = 2 eta~ dt_loc; and the
// sweep's slot records (B_j = c w_ij, footprint-local j)
srdr_status prepare_sweep(srdr_body* b);
// brick layout of the tiled passes (setup.cu): builds it for the requested
// brick size; b->bricks_built = 1 when built, -1 when a halo does not fit
srdr_status build_bricks(srdr_body* b);
// shared memory of the tiled passes per block for a halo of h particles
inline size_t tile_smem_a(size_t tsize, int h) { return (tsize == 4 ? (size_t)24 : (size_t)32) * h; }
inline size_t tile_smem_b(size_t tsize, int dim, int h) { return 16 * (size_t)pb_chunks(tsize, dim) * h; }
constexpr size_t kTileSmemMax = 200 * 1024;
// kernel-class timing (api.cu): begin/end an interval of class k
void prof_begin(srdr_body* b, int k, cudaEvent_t* ev);
void prof_end(srdr_body* b, int k, cudaEvent_t ev);
// stepping (step.cu)
srdr_status launch_steps(srdr_body* b, int64_t nsteps);
// zero the damping sweep's synchronisation words after a wait ran out (api.cu)
srdr_status reset_sync_words(srdr_body* b);
srdr_status sync_scalars(const srdr_body* b);
srdr_status reset_scalars(srdr_body* b, double tol);

// ------------------------------------------------------------ Philox4x64-10
// Salmon, Moraes, Dror & Shaw, "Parallel random numbers: as easy as 1, 2, 3"
// (SC'11).  Round: (hi0,lo0) = M0*x0, (hi1,lo1) = M1*x2,
// x <- (hi1 ^ x1 ^ k0, lo1, hi0 ^ x3 ^ k1, lo0); key += Weyl constants
// between rounds.
__host__ __device__ inline uint64_t mul_hi64(uint64_t a, uint64_t b)
{
#ifdef __CUDA_ARCH__
    return __umul64hi(a, b);
#else
    return (uint64_t)(((unsigned __int128)a * (unsigned __int128)b) >> 64);
#endif
}

__host__ __device__ inline void philox4x64_10(const uint64_t c[4], const uint64_t k[2],
                                              uint64_t out[4])
{
    uint64_t x0 = c[0], x1 = c[1], x2 = c[2], x3 = c[3];
    uint64_t k0 = k[0], k1 = k[1];
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint64_t m0 = 0xD2E7470EE14C6C93ULL, m1 = 0xCA5A826395121157ULL;
        uint64_t h0 = mul_hi64(m0, x0), l0 = m0 * x0;
        uint64_t h1 = mul_hi64(m1, x2), l1 = m1 * x2;
        uint64_t y0 = h1 ^ x1 ^ k0, y2 = h0 ^ x3 ^ k1;
        x0 = y0;
        x1 = l1;
        x2 = y2;
        x3 = l0;
        k0 += 0x9E3779B97F4A7C15ULL;
        k1 += 0xBB67AE8584CAA73BULL;
    }
    out[0] = x0;
    out[1] = x1;
    out[2] = x2;
    out[3] = x3;
}

// phi_n of the random choice: one draw per step from word 0
__host__ __device__ inline double random_phi(uint64_t seed, uint64_t step)
{
    uint64_t c[4] = {step, 0, 0, 0}, k[2] = {seed, 0}, o[4];
    philox4x64_10(c, k, o);
    return (double)(o[0] >> 11) * 0x1.0p-53;
}

}  // namespace srdr
