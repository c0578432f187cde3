// batch.cu — many bodies of uneven sizes relaxed together.
//
// Every body keeps its own device arrays (built by srdr_body_create*).  A
// batch walks them through flat work lists: (body, 32-particle slice) for
// the stress, force and finish passes, and, per colour, (body, cell) for the
// damping sweep.  One batched step is
//   k_batch_decide   Philox random choice of every body (Eq. viscosity-reset)
//   k_batch_pass_a   stress pass over all slices of all active bodies
//   k_batch_pass_b   force pass, v* = v^n + dt a
//   k_batch_sweep    S_d of every damped body, all colours forward then
//                    backward in one cooperative launch (Sec. 3.4), either
//                    with grid barriers between colour phases or, in
//                    k_batch_sweep_flow, with each cell waiting only for the
//                    overlapping cells of its own body
//   k_batch_finish   constraints, displacement update, KE slice partials
//   k_batch_ke       per-body FP64 KE, KE_max, retirement test
// The per-particle arithmetic is the single-body code (passes.cuh,
// sweep.cuh) and every body keeps its own reduction order, so a body's
// result is bitwise the same alone or in a batch.  Converged bodies retire
// (their work items are skipped and the lists are compacted); chunks of
// steps are captured in CUDA graphs; an autotuner picks the sweep's cells
// per warp and the passes' threads per block.
#include <math.h>

#include <algorithm>
#include <new>
#include <vector>

#include "srdr_internal.cuh"

namespace srdr {
namespace {

constexpr int kThreads = 256;
constexpr int kUnroll = 8;  // sliced-ELL slots per batch of loads in the passes

#include "passes.cuh"
#include "sweep.cuh"

template <typename T>
struct BatchEntry {
    StepArgs<T> step;
    SweepArgs<T> sweep;
    int material;
    int damping_on;
    double alpha;
    unsigned long long seed;
    int nslices;
    int ncells_nonempty;
    unsigned* flow;  // the body's cell-wise synchronisation words
};

// one block: damping decision of every body; any[0] = some body is damped
template <typename T>
__global__ void k_batch_decide(const BatchEntry<T>* __restrict__ tab, int nb, int* __restrict__ damp,
                               int* __restrict__ any)
{
    __shared__ int s_any;
    if (threadIdx.x == 0) s_any = 0;
    __syncthreads();
    for (int b = threadIdx.x; b < nb; b += blockDim.x) {
        const DevScalars* sc = tab[b].step.sc;
        int d = 0;
        if (!sc->done && tab[b].damping_on)
            d = random_phi(tab[b].seed, (unsigned long long)sc->step) < tab[b].alpha;
        damp[b] = d;
        if (d) s_any = 1;
    }
    __syncthreads();
    if (threadIdx.x == 0) *any = s_any;
}

template <typename T, int D>
__global__ void k_batch_pass_a(const BatchEntry<T>* __restrict__ tab, const int2* __restrict__ items,
                               int nitems)
{
    const int w = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5);
    if (w >= nitems) return;
    const int2 e = items[w];
    const StepArgs<T>& a = tab[e.x].step;
    if (a.sc->done) return;
    const int i = e.y * 32 + (threadIdx.x & 31);
    if (i >= a.n) return;
    if (tab[e.x].material == SRDR_NEO_HOOKEAN)
        pass_a_particle<T, D, SRDR_NEO_HOOKEAN>(a, i);
    else
        pass_a_particle<T, D, SRDR_LINEAR_SVK>(a, i);
}

template <typename T, int D>
__global__ void k_batch_pass_b(const BatchEntry<T>* __restrict__ tab, const int2* __restrict__ items,
                               int nitems)
{
    const int w = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5);
    if (w >= nitems) return;
    const int2 e = items[w];
    const StepArgs<T>& a = tab[e.x].step;
    if (a.sc->done) return;
    const int i = e.y * 32 + (threadIdx.x & 31);
    if (i >= a.n) return;
    pass_b_particle<T, D>(a, i, 0);
}

template <typename T>
__global__ void k_batch_finish(const BatchEntry<T>* __restrict__ tab, const int2* __restrict__ items,
                               int nitems)
{
    const int w = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5);
    if (w >= nitems) return;
    const int2 e = items[w];
    const StepArgs<T>& a = tab[e.x].step;
    if (a.sc->done) return;
    const int i = e.y * 32 + (threadIdx.x & 31);
    const double ke = i < a.n ? finish_particle<T>(a, i) : 0.0;
    slice_partial_store(ke, a.ke_part, i, a.n);
}

template <typename T>
__global__ void __launch_bounds__(kKeThreads) k_batch_ke(const BatchEntry<T>* __restrict__ tab,
                                                        const int* __restrict__ bodies,
                                                        const int* __restrict__ damp)
{
    const int b = bodies[blockIdx.x];
    DevScalars* sc = tab[b].step.sc;
    if (sc->done) return;
    ke_finalize(tab[b].step.ke_part, tab[b].nslices, sc, damp[b]);
}

// The next work item of a group at or after item k of phase ph (k < 0: from
// the start of phase ph) that belongs to a damped body, and its phase; -1
// when there is none.  Group q0 takes items q0, q0 + qs, ... of each colour.
__device__ inline int batch_next(const int2* __restrict__ cells, const int* __restrict__ damp,
                                 const int* __restrict__ colour_ptr, int ncolours, int clast, int ph, int k,
                                 int q0, int qs, int* item_ph)
{
    for (int p = ph; p < 2 * ncolours; ++p) {
        const int col = phase_colour(p, ncolours);
        if (p >= ncolours && col == clast) continue;  // fused into the forward phase
        const int c0 = __ldg(colour_ptr + col), c1 = __ldg(colour_ptr + col + 1);
        for (int kk = (p == ph && k >= 0) ? k + qs : c0 + q0; kk < c1; kk += qs)
            if (damp[cells[kk].x]) {
                *item_ph = p;
                return kk;
            }
    }
    return -1;
}

// S_d of every damped body: colour c of all bodies, then c+1, ...; forward
// then backward (the last colour's two phases fused); group g of block bb
// takes work items bb*G+g, +gridDim*G, ...
// As in the single-body sweep, the read-only data of a group's next item is
// staged between the barrier's arrive and wait.
template <typename T, int D, int G>
__global__ void __launch_bounds__(32) k_batch_sweep(const BatchEntry<T>* __restrict__ tab,
                                                    const int2* __restrict__ cells,
                                                    const int* __restrict__ colour_ptr, int ncolours,
                                                    const int* __restrict__ damp,
                                                    const int* __restrict__ any, unsigned* bar,
                                                    DevScalars* status, int F, int P, int C)
{
    constexpr int L = 32 / G;
    if (!*(volatile const int*)any) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ unsigned s_gen;
    __shared__ int s_ok;
    const int g = threadIdx.x / L, gl = threadIdx.x % L;
    const unsigned gmask = (L == 32) ? 0xffffffffu : (((1u << L) - 1u) << (g * L));
    const CellSmem<T, D> s =
        cell_smem<T, D>(smem_raw + (size_t)g * cell_smem_bytes<T, D>(F, P, C), F, P, C);
    const int q0 = blockIdx.x * G + g, qs = gridDim.x * G;
    int sph = 0;
    const int clast = last_colour(colour_ptr, ncolours);
    int staged = batch_next(cells, damp, colour_ptr, ncolours, clast, 0, -1, q0, qs, &sph);
    CellStage st{};
    if (staged >= 0) {
        const int2 e = cells[staged];
        st = stage_cell<T, D, L>(tab[e.x].sweep, e.y, s, gl, gmask);
    }
    bool restage = false;
    int phases = 0;
    for (int ph = 0; ph < 2 * ncolours; ++ph) {
        const int backward = ph >= ncolours;
        const int col = backward ? 2 * ncolours - 1 - ph : ph;
        const int c0 = __ldg(colour_ptr + col), c1 = __ldg(colour_ptr + col + 1);
        if (c1 == c0 || (backward && col == clast)) continue;
        const int mode = col == clast ? 2 : backward;
        if (phases++ > 0) {
            __syncthreads();
            if (threadIdx.x == 0) s_gen = bar_arrive(bar, gridDim.x);
            if (restage && staged >= 0) {
                const int2 e = cells[staged];
                st = stage_cell<T, D, L>(tab[e.x].sweep, e.y, s, gl, gmask);
            }
            restage = false;
            if (threadIdx.x == 0) s_ok = bar_wait(bar, s_gen, status) ? 1 : 0;
            __syncthreads();
            if (!s_ok) {
                cp_async_wait_all();  // no copy may land after the block has left
                return;
            }
        }
        while (staged >= 0 && sph == ph) {
            const int2 e = cells[staged];
            run_cell<T, D, L>(tab[e.x].sweep, st, mode, s, gl, gmask);
            staged = batch_next(cells, damp, colour_ptr, ncolours, clast, ph, staged, q0, qs, &sph);
            if (staged >= 0 && sph == ph) {
                const int2 e2 = cells[staged];
                st = stage_cell<T, D, L>(tab[e2.x].sweep, e2.y, s, gl, gmask);
            } else {
                restage = true;
            }
        }
        __syncwarp();
    }
    cp_async_wait_all();
}

// The batched S_d with cell-wise waits instead of grid barriers (the
// single-body k_sweep_flow, per body): before each of its phases a cell
// waits for the cells of its own body whose footprints overlap its own to
// have finished their earlier phases.  The cell that finishes its body's
// last direction advances the body's epoch.  Same parameters as
// k_batch_sweep (bar unused) and bitwise the same results.
template <typename T, int D, int G>
__global__ void __launch_bounds__(32) k_batch_sweep_flow(const BatchEntry<T>* __restrict__ tab,
                                                         const int2* __restrict__ cells,
                                                         const int* __restrict__ colour_ptr, int ncolours,
                                                         const int* __restrict__ damp,
                                                         const int* __restrict__ any, unsigned* bar,
                                                         DevScalars* status, int F, int P, int C)
{
    constexpr int L = 32 / G;
    (void)bar;
    if (!*(volatile const int*)any) return;
    if (*(volatile int*)&status->status == DEV_TIMEOUT) return;  // words left mid-sweep: host resets them
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int g = threadIdx.x / L, gl = threadIdx.x % L;
    const unsigned gmask = (L == 32) ? 0xffffffffu : (((1u << L) - 1u) << (g * L));
    const CellSmem<T, D> s =
        cell_smem<T, D>(smem_raw + (size_t)g * cell_smem_bytes<T, D>(F, P, C), F, P, C);
    const int q0 = blockIdx.x * G + g, qs = gridDim.x * G;
    int sph = 0;
    const int clast = last_colour(colour_ptr, ncolours);
    int staged = batch_next(cells, damp, colour_ptr, ncolours, clast, 0, -1, q0, qs, &sph);
    CellStage st{};
    if (staged >= 0) {
        const int2 e = cells[staged];
        st = stage_cell<T, D, L>(tab[e.x].sweep, e.y, s, gl, gmask);
    }
    bool ok = true;
    for (int ph = 0; ph < 2 * ncolours && ok; ++ph) {
        const int backward = ph >= ncolours;
        const int col = backward ? 2 * ncolours - 1 - ph : ph;
        const int c0 = __ldg(colour_ptr + col), c1 = __ldg(colour_ptr + col + 1);
        if (c1 == c0 || (backward && col == clast)) continue;
        const int mode = col == clast ? 2 : backward;
        while (staged >= 0 && sph == ph) {
            const int2 e = cells[staged];
            const SweepArgs<T>& a = tab[e.x].sweep;
            unsigned* flow = tab[e.x].flow;
            const int fo = flow_epoch_word(a.nx * a.ny * a.nz);
            const unsigned epoch = *(volatile const unsigned*)(flow + fo);
            if (!flow_wait<T, L>(a, flow, epoch, e.y, ph, ncolours, clast, status, gl, gmask)) {
                ok = false;
                break;
            }
            run_cell<T, D, L>(a, st, mode, s, gl, gmask);
            if (gl == 0) {
                __threadfence();  // the group's write-back (ordered by run_cell's __syncwarp) first
                atomicAdd(flow + e.y, mode == 2 ? 2u : 1u);
                // the body's last cell to finish its last direction ends the body's sweep
                if (mode != 0 && atomicAdd(flow + fo + 32, 1u) == (unsigned)tab[e.x].ncells_nonempty - 1u) {
                    atomicExch(flow + fo + 32, 0u);
                    __threadfence();
                    atomicAdd(flow + fo, 1u);
                }
            }
            staged = batch_next(cells, damp, colour_ptr, ncolours, clast, ph, staged, q0, qs, &sph);
            if (staged >= 0) {
                const int2 e2 = cells[staged];
                st = stage_cell<T, D, L>(tab[e2.x].sweep, e2.y, s, gl, gmask);
            }
        }
    }
    cp_async_wait_all();  // no copy may land after the group has left
}

__global__ void k_batch_set_tol(DevScalars* const* scs, int nb, double tol)
{
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < nb; b += gridDim.x * blockDim.x) {
        scs[b]->tol = tol;
        if (scs[b]->status == DEV_OK) scs[b]->done = 0;
    }
}

// out[0..nb) = every body's scalars, out[nb] = the batch's own status word
__global__ void k_batch_gather(DevScalars* const* scs, int nb, const DevScalars* batch_status,
                               DevScalars* out)
{
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b <= nb; b += gridDim.x * blockDim.x)
        out[b] = b < nb ? *scs[b] : *batch_status;
}

}  // namespace
}  // namespace srdr

// ---------------------------------------------------------------- the batch
struct srdr_batch {
    std::vector<srdr_body*> bodies;
    bool owns_bodies = false;
    bool owns_stream = false;
    cudaStream_t stream = nullptr;
    int prec = SRDR_FP64, dim = 3, ncolours = 27;
    int F = 0, P = 0, C = 0;
    int G = 1;            // sweep cells per warp
    int cellwise = 1;     // sweep synchronised by cell-wise waits (1) or grid barriers (0)
    int pass_threads = 256;
    int tuned = 0;
    // device
    void* tab = nullptr;             // BatchEntry<T>[nb]
    int2* items = nullptr;           // (body, slice) of active bodies
    int nitems = 0;
    int2* cells = nullptr;           // (body, cell) per colour
    int* cptr_d = nullptr;
    int* active_d = nullptr;         // active body indices (for k_batch_ke)
    int nactive = 0;
    int* damp = nullptr;
    int* any = nullptr;
    unsigned* bar = nullptr;
    srdr::DevScalars* status = nullptr;
    srdr::DevScalars** scs = nullptr;  // device array of the bodies' scalar pointers
    srdr::DevScalars* gathered = nullptr;
    srdr::DevScalars* gathered_h = nullptr;
    std::vector<int> active;         // host copy of the active list
    std::vector<int> cptr;
    int sweep_grid = 0;
    size_t sweep_smem = 0;
    int64_t steps = 0;
    int64_t launches = 0;
    // graphs of chunks of steps for the current work lists
    cudaGraphExec_t graph = nullptr;
    int graph_steps = 0;
    int graphs_ok = 1;
    std::vector<void*> allocs;
    // SRDR_BATCH_STREAMS: each body steps with its own kernels on one of
    // these streams, all bodies at once
    int mode = SRDR_BATCH_AUTO;
    std::vector<cudaStream_t> pool;
};

namespace srdr {
namespace {

srdr_status balloc(srdr_batch* bt, void** p, size_t bytes)
{
    *p = nullptr;
    cudaError_t e = cudaMalloc(p, bytes ? bytes : 16);
    if (e != cudaSuccess) {
        cudaGetLastError();
        set_error("cudaMalloc(%zu bytes) failed: %s", bytes, cudaGetErrorString(e));
        return e == cudaErrorMemoryAllocation ? SRDR_ERR_NO_MEMORY : SRDR_ERR_CUDA;
    }
    bt->allocs.push_back(*p);
    return SRDR_OK;
}
template <typename P>
srdr_status balloc_n(srdr_batch* bt, P** p, size_t count)
{
    return balloc(bt, reinterpret_cast<void**>(p), count * sizeof(P));
}
void bfree(srdr_batch* bt, void* p)
{
    if (!p) return;
    auto it = std::find(bt->allocs.begin(), bt->allocs.end(), p);
    if (it != bt->allocs.end()) bt->allocs.erase(it);
    cudaFree(p);
}


template <typename T>
SweepArgs<T> sweep_args(srdr_body* b, int F, int P, int C)
{
    SweepArgs<T> s{};
    s.n = (int)b->n;
    s.dim = b->dim;
    s.nx = b->nc[0];
    s.ny = b->nc[1];
    s.nz = b->nc[2];
    s.cell_start = b->cell_start;
    s.colour_cells = b->colour_cells;
    s.row_ptr = b->row_ptr;
    s.loc = b->loc;
    s.w = static_cast<const T*>(b->w);
    s.rec = static_cast<const SweepSlot<T>*>(b->srec);
    s.mass = static_cast<const T*>(b->stencil ? b->mass_sw : b->mass);
    s.sbm = static_cast<const T*>(b->sbm);
    s.srd = static_cast<const T*>(b->srd);
    s.v = static_cast<T*>(b->stencil ? b->vs : b->v);
    s.sc = b->sc;
    s.c = b->desc.alpha > 0 ? (T)(b->eta / b->desc.alpha * b->dt) : T(0);
    s.pairwise = b->desc.damping == SRDR_DAMP_PAIRWISE;
    s.cbase = b->cbase;
    s.wrad = b->cbase == 3 ? 2 : 1;
    s.foot_ptr = b->foot_ptr;
    s.foot_tab = b->foot_tab;
    s.own_off = b->own_off;
    s.max_foot = F;  // one shared-memory layout for the whole batch
    s.max_pairs = P;
    s.max_cell = C;
    return s;
}

template <typename T>
srdr_status upload_table(srdr_batch* bt)
{
    const int nb = (int)bt->bodies.size();
    std::vector<BatchEntry<T>> tab(nb);
    for (int k = 0; k < nb; ++k) {
        srdr_body* b = bt->bodies[k];
        tab[k].step = make_step_args<T>(b);
        if (b->desc.damping != SRDR_DAMP_NONE && b->desc.alpha > 0.0 && b->eta > 0.0 && !b->sbm)
            SRDR_TRY(prepare_sweep(b));
        tab[k].sweep = sweep_args<T>(b, bt->F, bt->P, bt->C);
        tab[k].material = b->desc.material;
        tab[k].damping_on = b->desc.damping != SRDR_DAMP_NONE && b->desc.alpha > 0 && b->eta > 0;
        tab[k].alpha = b->desc.alpha;
        tab[k].seed = b->desc.seed;
        tab[k].nslices = b->nslices;
        tab[k].ncells_nonempty = b->ncells_nonempty;
        tab[k].flow = b->flow;
    }
    if (!bt->tab) SRDR_TRY(balloc(bt, &bt->tab, sizeof(BatchEntry<T>) * (size_t)nb));
    SRDR_CK(cudaMemcpyAsync(bt->tab, tab.data(), sizeof(BatchEntry<T>) * (size_t)nb,
                            cudaMemcpyHostToDevice, bt->stream));
    return SRDR_OK;
}

// Work lists of the active bodies: their slices, their cells by colour.
srdr_status build_lists(srdr_batch* bt, const std::vector<int>& active)
{
    std::vector<int2> items, cells;
    std::vector<std::vector<int2>> by_colour(bt->ncolours);
    for (int b : active) {
        srdr_body* body = bt->bodies[b];
        for (int s = 0; s < body->nslices; ++s) items.push_back(make_int2(b, s));
        std::vector<int> cc(std::max(1, body->ncells_nonempty));
        if (body->ncells_nonempty > 0)
            SRDR_CK(cudaMemcpy(cc.data(), body->colour_cells, sizeof(int) * body->ncells_nonempty,
                               cudaMemcpyDeviceToHost));
        for (int col = 0; col < body->ncolours; ++col)
            for (int k = body->colour_ptr[col]; k < body->colour_ptr[col + 1]; ++k)
                by_colour[col].push_back(make_int2(b, cc[k]));
    }
    bt->cptr.assign(bt->ncolours + 1, 0);
    for (int col = 0; col < bt->ncolours; ++col) {
        bt->cptr[col + 1] = bt->cptr[col] + (int)by_colour[col].size();
        cells.insert(cells.end(), by_colour[col].begin(), by_colour[col].end());
    }
    bfree(bt, bt->items);
    bfree(bt, bt->cells);
    bfree(bt, bt->active_d);
    bt->items = nullptr;
    bt->cells = nullptr;
    bt->active_d = nullptr;
    SRDR_TRY(balloc_n(bt, &bt->items, std::max<size_t>(items.size(), 1)));
    SRDR_TRY(balloc_n(bt, &bt->cells, std::max<size_t>(cells.size(), 1)));
    SRDR_TRY(balloc_n(bt, &bt->active_d, std::max<size_t>(active.size(), 1)));
    if (!items.empty())
        SRDR_CK(cudaMemcpy(bt->items, items.data(), sizeof(int2) * items.size(), cudaMemcpyHostToDevice));
    if (!cells.empty())
        SRDR_CK(cudaMemcpy(bt->cells, cells.data(), sizeof(int2) * cells.size(), cudaMemcpyHostToDevice));
    if (!active.empty())
        SRDR_CK(cudaMemcpy(bt->active_d, active.data(), sizeof(int) * active.size(),
                           cudaMemcpyHostToDevice));
    SRDR_CK(cudaMemcpy(bt->cptr_d, bt->cptr.data(), sizeof(int) * (bt->ncolours + 1),
                       cudaMemcpyHostToDevice));
    bt->nitems = (int)items.size();
    bt->active = active;
    bt->nactive = (int)active.size();
    if (bt->graph) {
        cudaGraphExecDestroy(bt->graph);
        bt->graph = nullptr;
        bt->graph_steps = 0;
    }
    return SRDR_OK;
}

template <typename T, int D, int G>
srdr_status sweep_config_g(srdr_batch* bt, const void** fn)
{
    const size_t smem = (size_t)G * cell_smem_bytes<T, D>(bt->F, bt->P, bt->C);
    if (smem > 227 * 1024) {
        set_error("batched sweep needs %zu bytes of shared memory per block", smem);
        return SRDR_ERR_INVALID;
    }
    *fn = bt->cellwise ? (const void*)k_batch_sweep_flow<T, D, G> : (const void*)k_batch_sweep<T, D, G>;
    if (smem > 48 * 1024)
        SRDR_CK(cudaFuncSetAttribute(*fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0, dev = 0, nsm = 0;
    SRDR_CK(cudaGetDevice(&dev));
    SRDR_CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    SRDR_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, *fn, 32, smem));
    if (per_sm < 1) {
        set_error("batched sweep kernel does not fit on an SM");
        return SRDR_ERR_INVALID;
    }
    int widest = 0;
    for (int c = 0; c < bt->ncolours; ++c) widest = std::max(widest, bt->cptr[c + 1] - bt->cptr[c]);
    bt->sweep_smem = smem;
    bt->sweep_grid = std::max(1, std::min((widest + G - 1) / G, per_sm * nsm));
    return SRDR_OK;
}

template <typename T, int D>
srdr_status sweep_config(srdr_batch* bt, const void** fn)
{
    switch (bt->G) {
    case 1: return sweep_config_g<T, D, 1>(bt, fn);
    case 4: return sweep_config_g<T, D, 4>(bt, fn);
    default: return sweep_config_g<T, D, 2>(bt, fn);
    }
}

// Enqueue nsteps batched steps on the batch stream.
template <typename T, int D>
srdr_status enqueue_steps(srdr_batch* bt, int64_t nsteps, const void* sweep_fn)
{
    if (bt->nactive == 0) return SRDR_OK;
    const BatchEntry<T>* tab = static_cast<const BatchEntry<T>*>(bt->tab);
    const int nb = (int)bt->bodies.size();
    const int tpb = bt->pass_threads;
    const int pblocks = (int)(((int64_t)bt->nitems * 32 + tpb - 1) / tpb);
    const int2* items = bt->items;
    int nitems = bt->nitems;
    const int2* cells = bt->cells;
    const int* cptr = bt->cptr_d;
    int ncol = bt->ncolours;
    const int* damp = bt->damp;
    const int* any = bt->any;
    unsigned* bar = bt->bar;
    DevScalars* status = bt->status;
    int F = bt->F, P = bt->P, C = bt->C;
    void* sweep_params[] = {&tab, &cells, &cptr, &ncol, &damp, &any, &bar, &status, &F, &P, &C};
    for (int64_t s = 0; s < nsteps; ++s) {
        k_batch_decide<T><<<1, 1024, 0, bt->stream>>>(tab, nb, bt->damp, bt->any);
        k_batch_pass_a<T, D><<<pblocks, tpb, 0, bt->stream>>>(tab, items, nitems);
        k_batch_pass_b<T, D><<<pblocks, tpb, 0, bt->stream>>>(tab, items, nitems);
        SRDR_CK(cudaLaunchCooperativeKernel(sweep_fn, dim3(bt->sweep_grid), dim3(32), sweep_params,
                                            bt->sweep_smem, bt->stream));
        k_batch_finish<T><<<pblocks, tpb, 0, bt->stream>>>(tab, items, nitems);
        k_batch_ke<T><<<bt->nactive, kKeThreads, 0, bt->stream>>>(tab, bt->active_d, bt->damp);
        bt->launches += 6;
    }
    SRDR_CK(cudaGetLastError());
    return SRDR_OK;
}

// A chunk of steps: replay a captured graph when one exists for this chunk
// length and these work lists, else capture one (falling back to direct
// launches if capture is not available).
template <typename T, int D>
srdr_status run_chunk(srdr_batch* bt, int64_t nsteps)
{
    // kernel attributes and occupancy are set up outside any stream capture
    const void* sweep_fn = nullptr;
    SRDR_TRY((sweep_config<T, D>(bt, &sweep_fn)));
    if (bt->graphs_ok && nsteps > 1) {
        if (!bt->graph || bt->graph_steps != nsteps) {
            if (bt->graph) {
                cudaGraphExecDestroy(bt->graph);
                bt->graph = nullptr;
            }
            cudaGraph_t g = nullptr;
            if (cudaStreamBeginCapture(bt->stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
                const int64_t l0 = bt->launches;
                srdr_status st = enqueue_steps<T, D>(bt, nsteps, sweep_fn);
                bt->launches = l0;
                cudaError_t e = cudaStreamEndCapture(bt->stream, &g);
                if (st == SRDR_OK && e == cudaSuccess && g &&
                    cudaGraphInstantiate(&bt->graph, g, 0) == cudaSuccess) {
                    bt->graph_steps = (int)nsteps;
                } else {
                    bt->graph = nullptr;
                    bt->graphs_ok = 0;
                }
                if (g) cudaGraphDestroy(g);
                cudaGetLastError();
            } else {
                cudaGetLastError();
                bt->graphs_ok = 0;
            }
        }
        if (bt->graph) {
            SRDR_CK(cudaGraphLaunch(bt->graph, bt->stream));
            bt->launches += 6 * nsteps;
            bt->steps += nsteps;
            return SRDR_OK;
        }
    }
    SRDR_TRY((enqueue_steps<T, D>(bt, nsteps, sweep_fn)));
    bt->steps += nsteps;
    return SRDR_OK;
}

// Autotuner: on fresh bodies (v = 0, where the sweep leaves every velocity
// at exactly 0 and the stress pass only rewrites P B0) time the sweep (on
// the bodies the first step damps) with
// 1, 2, 4 cells per warp, with cell-wise waits and with grid barriers, and
// the stress pass with 128, 256, 512 threads per block, and keep the
// fastest.  Bodies that already moved keep the defaults.  When every body
// asks for the same synchronisation (srdr_body_sweep_sync), the batch uses it.
template <typename T, int D>
srdr_status autotune(srdr_batch* bt)
{
    bt->tuned = 1;
    int want = bt->bodies.empty() ? SRDR_SWEEP_AUTO : bt->bodies[0]->sweep_sync;
    for (srdr_body* b : bt->bodies)
        if (b->sweep_sync != want) want = SRDR_SWEEP_AUTO;
    if (want != SRDR_SWEEP_AUTO) bt->cellwise = want == SRDR_SWEEP_CELLS;
    for (srdr_body* b : bt->bodies)
        if (b->step != 0) return SRDR_OK;
    const BatchEntry<T>* tab = static_cast<const BatchEntry<T>*>(bt->tab);
    const int nb = (int)bt->bodies.size();
    // the sweep is timed on the bodies the first step's random choice damps
    // (the share of damped bodies decides between cell-wise waits and grid
    // barriers), or on all of them when it damps none
    k_batch_decide<T><<<1, 1024, 0, bt->stream>>>(tab, nb, bt->damp, bt->any);
    int any_h = 0;
    SRDR_CK(cudaMemcpyAsync(&any_h, bt->any, sizeof(int), cudaMemcpyDeviceToHost, bt->stream));
    SRDR_CK(cudaStreamSynchronize(bt->stream));
    if (!any_h) {
        std::vector<int> ones(nb, 1);
        int one = 1;
        SRDR_CK(cudaMemcpyAsync(bt->damp, ones.data(), sizeof(int) * nb, cudaMemcpyHostToDevice, bt->stream));
        SRDR_CK(cudaMemcpyAsync(bt->any, &one, sizeof(int), cudaMemcpyHostToDevice, bt->stream));
    }
    cudaEvent_t e0, e1;
    SRDR_CK(cudaEventCreate(&e0));
    SRDR_CK(cudaEventCreate(&e1));
    auto timed = [&](auto&& launch, float* ms) -> srdr_status {
        launch();
        SRDR_CK(cudaEventRecord(e0, bt->stream));
        launch();
        launch();
        SRDR_CK(cudaEventRecord(e1, bt->stream));
        SRDR_CK(cudaEventSynchronize(e1));
        SRDR_CK(cudaGetLastError());
        SRDR_CK(cudaEventElapsedTime(ms, e0, e1));
        return SRDR_OK;
    };
    const int2* cells = bt->cells;
    const int* cptr = bt->cptr_d;
    int ncol = bt->ncolours;
    const int* damp = bt->damp;
    const int* any = bt->any;
    unsigned* bar = bt->bar;
    DevScalars* status = bt->status;
    int F = bt->F, P = bt->P, C = bt->C;
    void* sweep_params[] = {&tab, &cells, &cptr, &ncol, &damp, &any, &bar, &status, &F, &P, &C};
    float best = 3.0e38f;
    int best_g = bt->G, best_c = bt->cellwise;
    for (int cw : {1, 0})
        for (int g : {1, 2, 4}) {
            if (want != SRDR_SWEEP_AUTO && cw != (want == SRDR_SWEEP_CELLS)) continue;
            // cell-wise waits with one cell per warp only: two groups of a
            // warp would take turns, one polling while the other's chain waits
            if (cw && g > 1) continue;
            bt->G = g;
            bt->cellwise = cw;
            const void* fn = nullptr;
            if (sweep_config<T, D>(bt, &fn) != SRDR_OK) continue;
            float ms = 0;
            SRDR_TRY(timed([&] {
                cudaLaunchCooperativeKernel(fn, dim3(bt->sweep_grid), dim3(32), sweep_params, bt->sweep_smem,
                                            bt->stream);
            }, &ms));
            if (ms < best) {
                best = ms;
                best_g = g;
                best_c = cw;
            }
        }
    bt->G = best_g;
    bt->cellwise = best_c;
    best = 3.0e38f;
    int best_t = bt->pass_threads;
    // the block size must fit the register use of both passes (FP64 3D uses
    // more than 128 registers per thread, so 512 threads do not fit)
    int limit = 1024;
    for (const void* fn : {(const void*)k_batch_pass_a<T, D>, (const void*)k_batch_pass_b<T, D>}) {
        cudaFuncAttributes fa;
        SRDR_CK(cudaFuncGetAttributes(&fa, fn));
        limit = std::min(limit, fa.maxThreadsPerBlock);
    }
    for (int tpb : {128, 256, 512}) {
        if (tpb > limit) continue;
        const int blocks = (int)(((int64_t)bt->nitems * 32 + tpb - 1) / tpb);
        float ms = 0;
        // the stress pass only: it rewrites P B0 and leaves the state alone
        SRDR_TRY(timed([&] { k_batch_pass_a<T, D><<<blocks, tpb, 0, bt->stream>>>(tab, bt->items, bt->nitems); },
                       &ms));
        if (ms < best) {
            best = ms;
            best_t = tpb;
        }
    }
    bt->pass_threads = best_t;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return SRDR_OK;
}

// Run up to nsteps batched steps.  tol > 0: a body retires when its KE drops
// below tol * KE_max; the batch stops when every body has retired.  The
// host looks at the bodies' scalars after every chunk (chunks double up to
// check_every steps), retires bodies and compacts the work lists once they
// have shrunk by a fifth.
template <typename T, int D>
srdr_status batch_steps(srdr_batch* bt, int64_t nsteps, double tol, int64_t check_every,
                        srdr_status* per_status, int64_t* per_steps)
{
    const int nb = (int)bt->bodies.size();
    if (!bt->tuned) SRDR_TRY((autotune<T, D>(bt)));
    k_batch_set_tol<<<(nb + 255) / 256, 256, 0, bt->stream>>>(bt->scs, nb, tol);
    std::vector<int64_t> start(nb);
    for (int b = 0; b < nb; ++b) start[b] = bt->bodies[b]->step;
    int64_t left = nsteps;
    int64_t chunk = std::min<int64_t>(check_every, 64);
    bool gathered = false;
    while (left > 0 && bt->nactive > 0) {
        const int64_t k = std::min(left, chunk);
        SRDR_TRY((run_chunk<T, D>(bt, k)));
        left -= k;
        k_batch_gather<<<(nb + 256) / 256, 256, 0, bt->stream>>>(bt->scs, nb, bt->status, bt->gathered);
        SRDR_CK(cudaMemcpyAsync(bt->gathered_h, bt->gathered, sizeof(DevScalars) * (nb + 1),
                                cudaMemcpyDeviceToHost, bt->stream));
        SRDR_CK(cudaStreamSynchronize(bt->stream));
        gathered = true;
        if (bt->gathered_h[nb].status == DEV_TIMEOUT) {
            // the barrier words are left mid-sweep: reset them and the status
            DevScalars z{};
            SRDR_CK(cudaMemsetAsync(bt->bar, 0, kBarWords * sizeof(unsigned), bt->stream));
            for (srdr_body* b : bt->bodies)
                SRDR_CK(cudaMemsetAsync(b->flow, 0, sizeof(unsigned) * flow_words(b->ncells), bt->stream));
            SRDR_CK(cudaMemcpyAsync(bt->status, &z, sizeof(z), cudaMemcpyHostToDevice, bt->stream));
            SRDR_CK(cudaStreamSynchronize(bt->stream));
            set_error("batched damping sweep: a grid barrier timed out");
            return SRDR_ERR_TIMEOUT;
        }
        std::vector<int> still;
        for (int b : bt->active)
            if (!bt->gathered_h[b].done) still.push_back(b);
        if (still.empty()) break;
        if (still.size() != bt->active.size()) {
            size_t before = 0, after = 0;
            for (int b : bt->active) before += bt->bodies[b]->nslices;
            for (int b : still) after += bt->bodies[b]->nslices;
            if (after * 5 < before * 4) SRDR_TRY(build_lists(bt, still));
        }
        chunk = std::min<int64_t>(chunk * 2, check_every);
    }
    if (!gathered) {
        k_batch_gather<<<(nb + 256) / 256, 256, 0, bt->stream>>>(bt->scs, nb, bt->status, bt->gathered);
        SRDR_CK(cudaMemcpyAsync(bt->gathered_h, bt->gathered, sizeof(DevScalars) * (nb + 1),
                                cudaMemcpyDeviceToHost, bt->stream));
        SRDR_CK(cudaStreamSynchronize(bt->stream));
    }
    k_batch_set_tol<<<(nb + 255) / 256, 256, 0, bt->stream>>>(bt->scs, nb, 0.0);
    SRDR_CK(cudaStreamSynchronize(bt->stream));
    for (int b = 0; b < nb; ++b) {
        srdr_body* body = bt->bodies[b];
        const DevScalars& s = bt->gathered_h[b];
        body->step = s.step;
        body->converged = s.done && s.status == DEV_OK && tol > 0;
        if (per_steps) per_steps[b] = s.step - start[b];
        if (per_status) {
            if (s.status == DEV_NONFINITE) per_status[b] = SRDR_ERR_NONFINITE;
            else if (tol > 0 && !s.done) per_status[b] = SRDR_ERR_NOT_CONVERGED;
            else per_status[b] = SRDR_OK;
        }
    }
    // a fresh list of every body for the next call
    std::vector<int> all(nb);
    for (int b = 0; b < nb; ++b) all[b] = b;
    if ((int)bt->active.size() != nb) SRDR_TRY(build_lists(bt, all));
    return SRDR_OK;
}

template <typename T>
srdr_status batch_dispatch(srdr_batch* bt, int64_t nsteps, double tol, srdr_status* st, int64_t* steps)
{
    if (bt->dim == 2) return batch_steps<T, 2>(bt, nsteps, tol, 4096, st, steps);
    return batch_steps<T, 3>(bt, nsteps, tol, 4096, st, steps);
}

// Concurrent mode: every body runs its own step kernels (srdr_body_step's,
// graph replays for small bodies) on one of a pool of streams, all bodies at
// once, in chunks of steps; after each chunk the host reads each body's
// scalars and retires the ones that met their criterion.  A damped step's
// sweep is a chain of dependent colour phases whose length does not shrink
// with the body; bodies on different streams overlap those chains instead of
// waiting for each other's at every step, as shared launches must.  Each
// body's kernels and their order are those of srdr_body_relax, so its result
// is bitwise the same as alone.
constexpr int kPoolStreams = 64;

srdr_status batch_run_streams(srdr_batch* bt, int64_t nsteps, double tol, srdr_status* per_status,
                              int64_t* per_steps)
{
    const int nb = (int)bt->bodies.size();
    const int ns = std::min(nb, kPoolStreams);
    while ((int)bt->pool.size() < ns) {
        cudaStream_t q = nullptr;
        SRDR_CK(cudaStreamCreateWithFlags(&q, cudaStreamNonBlocking));
        bt->pool.push_back(q);
    }
    std::vector<cudaStream_t> saved(nb);
    std::vector<int64_t> start(nb);
    for (int b = 0; b < nb; ++b) {
        srdr_body* body = bt->bodies[b];
        SRDR_CK(cudaStreamSynchronize(body->stream));  // the body's earlier work first
        saved[b] = body->stream;
        body->stream = bt->pool[b % ns];
        start[b] = body->step;
    }
    srdr_status result = SRDR_OK;
    std::vector<int> live;
    for (int b = 0; b < nb; ++b) {
        srdr_status r = reset_scalars(bt->bodies[b], tol);
        if (r != SRDR_OK && result == SRDR_OK) result = r;
        live.push_back(b);
    }
    int64_t left = nsteps, chunk = 64;
    while (result == SRDR_OK && left > 0 && !live.empty()) {
        const int64_t k = std::min(left, chunk);
        for (int b : live) {
            srdr_body* body = bt->bodies[b];
            srdr_status r = launch_steps(body, k);
            if (r == SRDR_OK && cudaMemcpyAsync(body->sc_host, body->sc, sizeof(DevScalars),
                                                cudaMemcpyDeviceToHost, body->stream) != cudaSuccess) {
                set_error("reading the scalars of a batched body failed");
                r = SRDR_ERR_CUDA;
            }
            if (r != SRDR_OK) {
                result = r;
                break;
            }
        }
        std::vector<int> keep;
        for (int b : live) {
            srdr_body* body = bt->bodies[b];
            if (cudaStreamSynchronize(body->stream) != cudaSuccess) {
                set_error("a batched body's stream failed: %s", cudaGetErrorString(cudaGetLastError()));
                if (result == SRDR_OK) result = SRDR_ERR_CUDA;
                continue;
            }
            body->step = body->sc_host->step;
            if (body->sc_host->status == DEV_TIMEOUT) {
                reset_sync_words(body);
                set_error("a bounded wait of a batched body's damping sweep ran out");
                if (result == SRDR_OK) result = SRDR_ERR_TIMEOUT;
                continue;
            }
            if (!(tol > 0 && body->sc_host->done) && body->sc_host->status != DEV_NONFINITE) keep.push_back(b);
        }
        live.swap(keep);
        left -= k;
        bt->steps += k;
        chunk = std::min<int64_t>(chunk * 2, 4096);
    }
    for (int b = 0; b < nb; ++b) {
        srdr_body* body = bt->bodies[b];
        if (cudaMemcpyAsync(body->sc_host, body->sc, sizeof(DevScalars), cudaMemcpyDeviceToHost,
                            body->stream) == cudaSuccess)
            cudaStreamSynchronize(body->stream);
        const DevScalars& s = *body->sc_host;
        body->step = s.step;
        body->converged = s.done && s.status == DEV_OK && tol > 0;
        if (per_steps) per_steps[b] = s.step - start[b];
        if (per_status) {
            if (s.status == DEV_NONFINITE) per_status[b] = SRDR_ERR_NONFINITE;
            else if (tol > 0 && !s.done) per_status[b] = SRDR_ERR_NOT_CONVERGED;
            else per_status[b] = SRDR_OK;
        }
        reset_scalars(body, 0.0);
        cudaStreamSynchronize(body->stream);
        body->stream = saved[b];
    }
    return result;
}

srdr_status batch_run(srdr_batch* bt, int64_t nsteps, double tol, srdr_status* st, int64_t* steps)
{
    if (bt->mode != SRDR_BATCH_SHARED) {
        std::vector<int64_t> l0(bt->bodies.size());
        for (size_t b = 0; b < bt->bodies.size(); ++b) l0[b] = bt->bodies[b]->launches;
        const int64_t before = bt->launches;
        srdr_status r = batch_run_streams(bt, nsteps, tol, st, steps);
        bt->launches = before;
        for (size_t b = 0; b < bt->bodies.size(); ++b) bt->launches += bt->bodies[b]->launches - l0[b];
        return r;
    }
    if (bt->prec == SRDR_FP64) return batch_dispatch<double>(bt, nsteps, tol, st, steps);
    return batch_dispatch<float>(bt, nsteps, tol, st, steps);
}

void batch_free(srdr_batch* bt)
{
    if (!bt) return;
    if (bt->stream) cudaStreamSynchronize(bt->stream);
    if (bt->graph) cudaGraphExecDestroy(bt->graph);
    for (void* p : bt->allocs) cudaFree(p);
    if (bt->gathered_h) cudaFreeHost(bt->gathered_h);
    if (bt->owns_stream && bt->stream) cudaStreamDestroy(bt->stream);
    for (cudaStream_t q : bt->pool) {
        cudaStreamSynchronize(q);
        cudaStreamDestroy(q);
    }
    if (bt->owns_bodies)
        for (srdr_body* b : bt->bodies) srdr_body_destroy(b);
    delete bt;
}

srdr_status batch_create(srdr_body* const* bodies, int nb, void* stream, bool owns, srdr_batch** out)
{
    if (!out || !bodies || nb < 1) {
        set_error("need at least one body");
        return SRDR_ERR_INVALID;
    }
    *out = nullptr;
    for (int b = 0; b < nb; ++b)
        if (!bodies[b] || bodies[b]->dim != bodies[0]->dim || bodies[b]->prec != bodies[0]->prec ||
            bodies[b]->desc.damping == SRDR_DAMP_EXPLICIT ||
            bodies[b]->desc.sweep_layout != SRDR_SWEEP_LAYOUT_3D) {
            set_error("batched bodies must all exist, share dimension and precision, use "
                      "split damping or none, and the paper's 3^d-colour sweep layout");
            return SRDR_ERR_INVALID;
        }
    srdr_batch* bt = new (std::nothrow) srdr_batch();
    if (!bt) {
        set_error("host allocation failed");
        return SRDR_ERR_NO_MEMORY;
    }
    bt->bodies.assign(bodies, bodies + nb);
    bt->owns_bodies = owns;
    bt->dim = bodies[0]->dim;
    bt->prec = bodies[0]->prec;
    bt->ncolours = bt->dim == 2 ? 9 : 27;
    for (srdr_body* b : bt->bodies) {
        bt->F = std::max(bt->F, b->max_foot);
        bt->P = std::max(bt->P, b->max_pairs);
        bt->C = std::max(bt->C, b->max_cell);
        if (b->stream) cudaStreamSynchronize(b->stream);
    }
    cudaDeviceSynchronize();
    srdr_status st = SRDR_OK;
    auto fail = [&](srdr_status s) {
        batch_free(bt);
        return s;
    };
    // graphs need a capturable stream: use the caller's unless it is the
    // legacy default stream
    if (stream) {
        bt->stream = static_cast<cudaStream_t>(stream);
    } else {
        if (cudaStreamCreateWithFlags(&bt->stream, cudaStreamNonBlocking) != cudaSuccess) {
            set_error("cudaStreamCreate failed");
            return fail(SRDR_ERR_CUDA);
        }
        bt->owns_stream = true;
    }
    if ((st = balloc_n(bt, &bt->damp, nb)) != SRDR_OK) return fail(st);
    if ((st = balloc_n(bt, &bt->any, 1)) != SRDR_OK) return fail(st);
    if ((st = balloc_n(bt, &bt->bar, kBarWords)) != SRDR_OK) return fail(st);
    if ((st = balloc_n(bt, &bt->status, 1)) != SRDR_OK) return fail(st);
    if ((st = balloc_n(bt, &bt->scs, nb)) != SRDR_OK) return fail(st);
    if ((st = balloc_n(bt, &bt->gathered, nb + 1)) != SRDR_OK) return fail(st);
    if ((st = balloc_n(bt, &bt->cptr_d, bt->ncolours + 1)) != SRDR_OK) return fail(st);
    if (cudaMallocHost(&bt->gathered_h, sizeof(DevScalars) * (nb + 1)) != cudaSuccess) {
        bt->gathered_h = nullptr;
        set_error("pinned host allocation failed");
        return fail(SRDR_ERR_NO_MEMORY);
    }
    std::vector<DevScalars*> scs(nb);
    for (int b = 0; b < nb; ++b) scs[b] = bt->bodies[b]->sc;
    DevScalars z{};
    if (cudaMemset(bt->bar, 0, kBarWords * sizeof(unsigned)) != cudaSuccess ||
        cudaMemcpy(bt->status, &z, sizeof(z), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(bt->scs, scs.data(), sizeof(DevScalars*) * nb, cudaMemcpyHostToDevice) != cudaSuccess) {
        set_error("batch initialisation copies failed");
        return fail(SRDR_ERR_CUDA);
    }
    st = bt->prec == SRDR_FP64 ? upload_table<double>(bt) : upload_table<float>(bt);
    if (st != SRDR_OK) return fail(st);
    std::vector<int> all(nb);
    for (int b = 0; b < nb; ++b) all[b] = b;
    if ((st = build_lists(bt, all)) != SRDR_OK) return fail(st);
    if (cudaStreamSynchronize(bt->stream) != cudaSuccess) {
        set_error("batch set-up failed");
        return fail(SRDR_ERR_CUDA);
    }
    *out = bt;
    return SRDR_OK;
}

}  // namespace
}  // namespace srdr

using namespace srdr;

extern "C" {

srdr_status srdr_batch_create(srdr_body* const* bodies, int nbodies, void* cuda_stream,
                              srdr_batch** out)
{
    return batch_create(bodies, nbodies, cuda_stream, false, out);
}

srdr_status srdr_batch_step(srdr_batch* bt, int64_t nsteps)
{
    if (!bt || nsteps < 0) {
        set_error("bad batch or step count");
        return SRDR_ERR_INVALID;
    }
    return batch_run(bt, nsteps, 0.0, nullptr, nullptr);
}

srdr_status srdr_batch_run(srdr_batch* bt, double ke_ratio, int64_t max_steps,
                           srdr_status* per_body_status, int64_t* per_body_steps)
{
    if (!bt || !(ke_ratio > 0) || max_steps < 0) {
        set_error("bad batch, ratio or step cap");
        return SRDR_ERR_INVALID;
    }
    SRDR_TRY(batch_run(bt, max_steps, ke_ratio, per_body_status, per_body_steps));
    if (per_body_status)
        for (size_t b = 0; b < bt->bodies.size(); ++b)
            if (per_body_status[b] != SRDR_OK) return per_body_status[b];
    return SRDR_OK;
}

srdr_status srdr_batch_mode(srdr_batch* bt, int mode)
{
    if (!bt || mode < SRDR_BATCH_AUTO || mode > SRDR_BATCH_STREAMS) {
        set_error("batch mode must be SRDR_BATCH_AUTO, _SHARED or _STREAMS");
        return SRDR_ERR_INVALID;
    }
    if (mode == SRDR_BATCH_SHARED)
        for (const srdr_body* b : bt->bodies)
            if (b->stencil) {
                set_error("shared launches take sliced-ELL bodies only: create the batch's bodies with "
                          "pass_layout = SRDR_PASS_LAYOUT_SELL");
                return SRDR_ERR_INVALID;
            }
    bt->mode = mode;
    return SRDR_OK;
}

srdr_status srdr_batch_info(const srdr_batch* bt, int64_t* steps, int64_t* launches,
                            int* sweep_cells_per_warp, int* pass_threads)
{
    if (!bt) {
        set_error("batch is NULL");
        return SRDR_ERR_INVALID;
    }
    if (steps) *steps = bt->steps;
    if (launches) *launches = bt->launches;
    if (sweep_cells_per_warp) *sweep_cells_per_warp = bt->G;
    if (pass_threads) *pass_threads = bt->pass_threads;
    return SRDR_OK;
}

void srdr_batch_destroy(srdr_batch* bt) { batch_free(bt); }

}  // extern "C"

namespace srdr {
// launch configuration of a tuned batch, carried over to the next batch of
// a continuous-batching loop (whose bodies have moved, so it cannot tune)
void batch_get_tuning(const srdr_batch* bt, int cfg[4])
{
    cfg[0] = bt->tuned;
    cfg[1] = bt->G;
    cfg[2] = bt->cellwise;
    cfg[3] = bt->pass_threads;
}
void batch_set_tuning(srdr_batch* bt, const int cfg[4])
{
    if (!cfg[0]) return;
    bt->tuned = 1;
    bt->G = cfg[1];
    bt->cellwise = cfg[2];
    bt->pass_threads = cfg[3];
}
}  // namespace srdr

extern "C" {

srdr_status srdr_desc_particle_count(const srdr_body_desc* d, int64_t* n)
{
    if (!d || !n || (d->dim != 2 && d->dim != 3) || !(d->dp > 0)) {
        set_error("bad description");
        return SRDR_ERR_INVALID;
    }
    int64_t c = 1;
    for (int a = 0; a < d->dim; ++a) {
        int64_t k = llround(d->extent[a] / d->dp);
        if (a == d->clamp_axis) k += d->clamp_layers + d->presc_layers;
        c *= k;
    }
    *n = c;
    return SRDR_OK;
}

srdr_status srdr_batch_relax(const srdr_body_desc* descs, int nbodies, double ke_ratio,
                             int64_t max_steps, double** host_disp_out, srdr_status* per_body_status)
{
    if (!descs || nbodies < 1) {
        set_error("need at least one description");
        return SRDR_ERR_INVALID;
    }
    cudaStream_t s = nullptr;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
        set_error("cudaStreamCreate failed");
        return SRDR_ERR_CUDA;
    }
    std::vector<srdr_body*> bodies(nbodies, nullptr);
    srdr_status st = SRDR_OK;
    for (int b = 0; b < nbodies && st == SRDR_OK; ++b) st = srdr_body_create(&descs[b], s, &bodies[b]);
    srdr_batch* bt = nullptr;
    if (st == SRDR_OK) st = batch_create(bodies.data(), nbodies, s, true, &bt);
    if (st != SRDR_OK) {
        for (srdr_body* b : bodies) srdr_body_destroy(b);
        cudaStreamDestroy(s);
        return st;
    }
    std::vector<srdr_status> per(nbodies, SRDR_OK);
    st = batch_run(bt, max_steps, ke_ratio, per.data(), nullptr);
    for (int b = 0; b < nbodies && st == SRDR_OK; ++b) {
        if (per_body_status) per_body_status[b] = per[b];
        if (host_disp_out && host_disp_out[b])
            st = srdr_body_read_displacement(bodies[b], host_disp_out[b], (size_t)bodies[b]->n * 3);
    }
    batch_free(bt);  // owns the bodies
    cudaStreamDestroy(s);
    if (st != SRDR_OK) return st;
    for (int b = 0; b < nbodies; ++b)
        if (per[b] != SRDR_OK) return per[b];
    return SRDR_OK;
}

}  // extern "C"
