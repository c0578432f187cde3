// step.cu — the per-step hot path of the splitting random-choice dynamic
// relaxation (arXiv 2103.08932):
//   k_pass_a   corrected deformation gradient at u^{n+1/2} (Sec. 2.2-2.3),
//              stress S(F) (Sec. 2.1), P = F S, and P B0 per particle
//   k_pass_b   momentum sum (Eqs. evaluate-momentum, averaged-Piola-Kirchhoff),
//              velocity update, constraints, fused displacement half-steps,
//              per-block kinetic-energy partials
//   k_sweep    one colour of the forward or backward damping sweep S_d
//              (Eq. particle-by-particle-splitting, Sec. 3.1 / 3.2) over the
//              splitting cell-linked list (Sec. 3.4)
//   k_finish   constraints and displacement update after a damped step
//   k_ke_final FP64 kinetic energy, its running maximum and the relax test
#include <math.h>

#include <algorithm>
#include <type_traits>

#include "srdr_internal.cuh"

namespace srdr {

namespace {

constexpr int kThreads = 256;
constexpr int kUnroll = 8;  // sliced-ELL slots per batch of loads in the passes
constexpr int kGraphSteps = 32;       // steps per captured graph (small bodies)
constexpr int64_t kGraphMaxN = 65536;  // bodies up to this size replay graphs
inline int nblocks(int64_t n, int t = kThreads) { return (int)((n + t - 1) / t); }

#include "passes.cuh"

// ------------------------------------------------------------------ damping sweep
template <typename T>
__device__ inline T warp_allsum(T x)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

#include "sweep.cuh"
#include "tiles.cuh"

__global__ void k_set_tol(DevScalars* sc, double tol)
{
    sc->tol = tol;
    if (sc->status == DEV_OK) sc->done = 0;
}

// clears a DEV_TIMEOUT left by an autotuner's timing launch (on a scratch
// copy of v: the state is untouched); reports it in *out
__global__ void k_take_timeout(DevScalars* sc, int* out)
{
    *out = sc->status == DEV_TIMEOUT;
    if (sc->status == DEV_TIMEOUT) sc->status = DEV_OK;
}

// ------------------------------------------------------------------ host side

template <typename T>
SweepArgs<T> make_sweep_args(srdr_body* b)
{
    SweepArgs<T> s{};
    s.n = (int)b->n;
    s.dim = b->dim;
    s.nx = b->nc[0];
    s.ny = b->nc[1];
    s.nz = b->nc[2];
    s.cell_start = b->cell_start;
    s.colour_cells = b->colour_cells;  // all colours; colour_ptr_d indexes into it
    s.row_ptr = b->row_ptr;
    s.loc = b->loc;
    s.w = static_cast<const T*>(b->w);
    s.rec = static_cast<const SweepSlot<T>*>(b->srec);
    s.mass = static_cast<const T*>(b->stencil ? b->mass_sw : b->mass);
    s.sbm = static_cast<const T*>(b->sbm);
    s.srd = static_cast<const T*>(b->srd);
    s.v = static_cast<T*>(b->stencil ? b->vs : b->v);
    s.sc = b->sc;
    // B_j = 2 eta~ V_i V_j W'/r dt_loc with eta~ = eta / alpha, dt_loc = dt / 2
    s.c = (T)(b->eta / b->desc.alpha * b->dt);
    s.pairwise = b->desc.damping == SRDR_DAMP_PAIRWISE;
    s.cbase = b->cbase;
    s.wrad = b->cbase == 3 ? 2 : 1;
    s.foot_ptr = b->foot_ptr;
    s.foot_tab = b->foot_tab;
    s.own_off = b->own_off;
    s.max_foot = b->max_foot;
    s.rows_global = b->sweep_rows_global;
    s.max_pairs = b->sweep_rows_global ? 0 : b->max_pairs;  // no staged rows then
    s.max_cell = b->max_cell;
    return s;
}

// The sweep kernel for G cells per warp and W warps per block with grid
// barriers or cell-wise waits, its shared memory, its grid (co-resident
// blocks, at most one group per cell of the widest colour) and its
// synchronisation words (its last argument).
template <typename T, int D>
struct SweepLaunch {
    const void* fn = nullptr;
    size_t smem = 0;
    int grid = 0;
    int threads = 32;
    unsigned* sync = nullptr;
};

template <typename T, int D, int G, int W, int H = 0>
srdr_status sweep_launch_gw(srdr_body* b, SweepLaunch<T, D>* out)
{
    // the rows are staged in shared memory when a cell's fit, else read
    // through the caches (large cells of the 2^d layout)
    size_t smem = (size_t)G * W * cell_smem_bytes<T, D>(b->max_foot, b->max_pairs, b->max_cell);
    b->sweep_rows_global = 0;
    if (smem > 227 * 1024 && b->cbase == 2) {
        smem = (size_t)G * W * cell_smem_bytes<T, D>(b->max_foot, 0, b->max_cell);
        b->sweep_rows_global = 1;
    }
    if (smem > 227 * 1024) {
        set_error("damping sweep needs %zu bytes of shared memory per block (limit 227 KB)", smem);
        return SRDR_ERR_INVALID;
    }
    const void* fn = b->sweep_cellwise ? (const void*)k_sweep_flow<T, D, G, W, H>
                                       : (const void*)k_sweep_all<T, D, G, W>;
    if (smem > 48 * 1024)
        SRDR_CK(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0, dev = 0, nsm = 0;
    SRDR_CK(cudaGetDevice(&dev));
    SRDR_CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    SRDR_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, 32 * W, smem));
    if (per_sm < 1) {
        set_error("damping sweep kernel does not fit on an SM (%zu bytes of shared memory)", smem);
        return SRDR_ERR_INVALID;
    }
    int widest = 0;
    for (int c = 0; c < b->ncolours; ++c)
        widest = std::max(widest, b->colour_ptr[c + 1] - b->colour_ptr[c]);
    out->fn = fn;
    out->smem = smem;
    out->threads = 32 * W;
    out->sync = b->sweep_cellwise ? b->flow : b->bar;
    out->grid = std::max(1, std::min((widest + G * W - 1) / (G * W), per_sm * nsm));
    return SRDR_OK;
}

template <typename T, int D>
srdr_status sweep_launch(srdr_body* b, SweepLaunch<T, D>* out)
{
    if (b->sweep_chain16 && b->sweep_cellwise && b->sweep_cells_per_warp == 1)
        return b->sweep_warps_per_block == 4 ? sweep_launch_gw<T, D, 1, 4, 1>(b, out)
                                             : sweep_launch_gw<T, D, 1, 1, 1>(b, out);
    const int key = b->sweep_cells_per_warp * 10 + b->sweep_warps_per_block;
    switch (key) {
    case 11: return sweep_launch_gw<T, D, 1, 1>(b, out);
    case 14: return sweep_launch_gw<T, D, 1, 4>(b, out);
    case 21: return sweep_launch_gw<T, D, 2, 1>(b, out);
    case 24: return sweep_launch_gw<T, D, 2, 4>(b, out);
    case 41: return sweep_launch_gw<T, D, 4, 1>(b, out);
    default: return sweep_launch_gw<T, D, 4, 4>(b, out);
    }
}

// Autotuner of the sweep's mapping: time G = 1 or 2 cells per warp with
// W = 1 or 4 warps per block, with cell-wise waits and with grid barriers
// (unless one of them is asked for), and the cell-wise sweep with its chain
// on 16 lanes of each warp, one warm-up and one timed launch each,
// on a scratch copy of v (the sweep writes v, the body's state must not
// change) and keep the fastest.  G = 4 (measured slower on every body tried) stays
// available through srdr_body_tune.  The sweep's
// arithmetic does not depend on the mapping (its reductions follow one
// 32-lane order), so the choice changes speed, never results.
template <typename T, int D>
srdr_status autotune_sweep(srdr_body* b)
{
    b->sweep_tuned = 1;
    T* vtmp = nullptr;
    SRDR_TRY(dalloc(b, &vtmp, (size_t)4 * b->n));
    int* tflag = nullptr;
    SRDR_TRY(dalloc(b, &tflag, 1));
    SRDR_CK(cudaMemcpyAsync(vtmp, b->v, sizeof(T) * 4 * (size_t)b->n, cudaMemcpyDeviceToDevice,
                            b->stream));
    SweepArgs<T> sw = make_sweep_args<T>(b);
    sw.v = vtmp;
    const int* cptr = b->colour_ptr_d;
    int ncol = b->ncolours;
    unsigned* sync = nullptr;
    void* params[] = {&sw, &cptr, &ncol, &sync};
    cudaEvent_t e0, e1;
    SRDR_CK(cudaEventCreate(&e0));
    SRDR_CK(cudaEventCreate(&e1));
    float best = 3.0e38f;
    int best_g = b->sweep_cells_per_warp, best_w = b->sweep_warps_per_block, best_c = b->sweep_cellwise;
    int best_h = 0;
    for (int cw : {1, 0})
    for (int g : {1, 2})
    for (int h : {0, 1})
        for (int w : {1, 4}) {
            if ((cw && b->sweep_sync == SRDR_SWEEP_BARRIER) || (!cw && b->sweep_sync == SRDR_SWEEP_CELLS))
                continue;
            // cell-wise waits with one cell per warp only: two groups of a
            // warp would take turns, one polling while the other's chain waits
            if (cw && g > 1) continue;
            // the 16-lane chain: cell-wise waits, one cell per warp
            if (h && (!cw || g != 1)) continue;
            b->sweep_cellwise = cw;
            b->sweep_cells_per_warp = g;
            b->sweep_warps_per_block = w;
            b->sweep_chain16 = h;
            SweepLaunch<T, D> sl;
            if (sweep_launch<T, D>(b, &sl) != SRDR_OK) continue;  // e.g. too much shared memory
            sw.rows_global = b->sweep_rows_global;  // the staging this mapping can afford
            sw.max_pairs = b->sweep_rows_global ? 0 : b->max_pairs;
            sync = sl.sync;
            SRDR_CK(cudaLaunchCooperativeKernel(sl.fn, dim3(sl.grid), dim3(sl.threads), params, sl.smem,
                                                b->stream));
            SRDR_CK(cudaEventRecord(e0, b->stream));
            SRDR_CK(cudaLaunchCooperativeKernel(sl.fn, dim3(sl.grid), dim3(sl.threads), params, sl.smem,
                                                b->stream));
            SRDR_CK(cudaEventRecord(e1, b->stream));
            k_take_timeout<<<1, 1, 0, b->stream>>>(b->sc, tflag);
            int ran_out = 0;
            SRDR_CK(cudaMemcpyAsync(&ran_out, tflag, sizeof(int), cudaMemcpyDeviceToHost, b->stream));
            SRDR_CK(cudaEventSynchronize(e1));
            SRDR_CK(cudaStreamSynchronize(b->stream));
            if (ran_out) {
                // a wait of this mapping ran out: its words are mid-sweep and
                // the mapping is not a candidate
                SRDR_TRY(reset_sync_words(b));
                continue;
            }
            float ms = 0.f;
            SRDR_CK(cudaEventElapsedTime(&ms, e0, e1));
            if (ms < best) {
                best = ms;
                best_g = g;
                best_w = w;
                best_c = cw;
                best_h = h;
            }
        }
    b->sweep_cells_per_warp = best_g;
    b->sweep_warps_per_block = best_w;
    b->sweep_cellwise = best_c;
    b->sweep_chain16 = best_h;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    SRDR_TRY(dev_free(b, tflag));
    return dev_free(b, vtmp);
}

// Mapping of the stress and force passes: sliced ELL or brick tiles (see
// srdr_body_pass_mapping).  The automatic choice is the sliced-ELL mapping,
// the faster of the two on every body measured on GB300 (the brick layout is
// then never built).
template <typename T, int D, int MAT>
srdr_status choose_pass_mapping(srdr_body* b)
{
    if (b->stencil) {
        b->pass_tiled = 0;
        return SRDR_OK;
    }
    if (b->pass_mapping != SRDR_PASS_BRICKS) {
        b->pass_tiled = 0;
        return SRDR_OK;
    }
    if (b->bricks_built == 0) SRDR_TRY(build_bricks(b));
    if (b->bricks_built < 0) {
        set_error("a brick halo does not fit in shared memory: use smaller bricks or sliced ELL");
        return SRDR_ERR_INVALID;
    }
    b->pass_tiled = 1;
    return SRDR_OK;
}

template <typename T, int D, int MAT>
srdr_status steps_typed(srdr_body* b, int64_t nsteps)
{
    cudaStream_t st = b->stream;
    const bool explicit_visc = b->desc.damping == SRDR_DAMP_EXPLICIT && b->eta > 0.0;
    if (explicit_visc && !b->dvisc) {
        T* dv = nullptr;
        SRDR_TRY(dalloc(b, &dv, (size_t)4 * b->n));
        b->dvisc = dv;
    }
    StepArgs<T> a = make_step_args<T>(b);
    const int nb = nblocks(b->n);
    const bool damping = (b->desc.damping == SRDR_DAMP_PARTICLE || b->desc.damping == SRDR_DAMP_PAIRWISE) &&
                         b->desc.alpha > 0.0 && b->eta > 0.0;
    const T c2eta_dt = (T)(2.0 * b->eta * b->dt);
    if (damping && !b->sbm) SRDR_TRY(prepare_sweep(b));
    SweepLaunch<T, D> sl;
    if (damping && !b->sweep_tuned) SRDR_TRY((autotune_sweep<T, D>(b)));
    if (damping) SRDR_TRY((sweep_launch<T, D>(b, &sl)));
    SweepArgs<T> sw = make_sweep_args<T>(b);  // after sweep_launch chose the staging
    const size_t smem = sl.smem;
    const int grid = sl.grid;
    const int* cptr = b->colour_ptr_d;
    int ncol = b->ncolours;
    unsigned* bar = damping ? sl.sync : b->bar;  // grid barrier or cell-wise words
    if (damping && (!sw.colour_cells || !sw.cell_start || !sw.row_ptr || !sw.loc || !sw.w || !sw.rec ||
                    !sw.mass || !sw.sbm || !sw.srd || !sw.v || !cptr || !bar)) {
        set_error("damping sweep tables are not built");
        return SRDR_ERR_INVALID;
    }
    void* sweep_params[] = {&sw, &cptr, &ncol, &bar};
    if (b->pass_tiled < 0) SRDR_TRY((choose_pass_mapping<T, D, MAT>(b)));
    const bool tiled = b->pass_tiled == 1;
    // stencil bodies with the usual offset count take the table as a kernel
    // parameter, the others read it from global memory
    constexpr int KD = D == 3 ? kStencilK3 : kStencilK2;
    const bool tab = b->stencil && b->st_k == KD;
    const StencilTab<T, KD> stab = tab ? make_stencil_tab<T, KD>(b) : StencilTab<T, KD>{};
    TileArgs<T> tl{};
    size_t smem_a = 0, smem_b = 0;
    if (tiled) {
        tl = make_tile_args<T>(b);
        smem_a = tile_smem_a(sizeof(T), b->max_halo);
        smem_b = tile_smem_b(sizeof(T), D, b->max_halo);
        SRDR_CK(cudaFuncSetAttribute((const void*)k_pass_a_tiled<T, D, MAT>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_a));
        SRDR_CK(cudaFuncSetAttribute((const void*)k_pass_b_tiled<T, D>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_b));
    }
    cudaEvent_t ev = nullptr;
    auto counted = [&](int k, int nlaunch) {
        b->k_launch[k] += nlaunch;
        b->launches += nlaunch;
    };
    // device-decided copies of the arguments (multi-step graph replay)
    StepArgs<T> ad = a;
    SweepArgs<T> swd = sw;
    void* sweep_params_d[] = {&swd, &cptr, &ncol, &bar};

    // One step on stream q.  dev: the random choice is drawn on the device
    // (k_decide_one) and every kernel of the step reads it, so the launch
    // sequence is the same for every step; otherwise the host draws it and
    // launches only what the step needs.  Both give the same bits.
    auto one_step = [&](cudaStream_t q, bool dev, bool damp) -> srdr_status {
        const StepArgs<T>& A = dev ? ad : a;
        if (dev && damping)
            k_decide_one<<<1, 1, 0, q>>>(b->sc, (unsigned long long)b->desc.seed, b->desc.alpha, b->dflag_d);
        prof_begin(b, SRDR_K_PASS_A, &ev);
        if (tiled)
            k_pass_a_tiled<T, D, MAT><<<b->nbricks, kTileThreads, smem_a, q>>>(A, tl);
        else if (tab)
            k_pass_a_tab<T, D, MAT, KD><<<nb, kThreads, 0, q>>>(A, stab);
        else if (b->stencil)
            k_pass_a<T, D, MAT, 1><<<nb, kThreads, 0, q>>>(A);
        else
            k_pass_a<T, D, MAT, 0><<<nb, kThreads, 0, q>>>(A);
        prof_end(b, SRDR_K_PASS_A, ev);
        counted(SRDR_K_PASS_A, 1);
        if (explicit_visc) {
            // the explicit comparator's damping, at v^n, before the force pass
            prof_begin(b, SRDR_K_SWEEP, &ev);
            k_visc<T, D><<<nb, kThreads, 0, q>>>((int)b->n, b->row_ptr, b->col,
                                                 static_cast<const T*>(b->w), static_cast<const T*>(b->v),
                                                 static_cast<const T*>(b->stencil ? b->mass_sw : b->mass),
                                                 b->pidx, c2eta_dt, static_cast<T*>(b->dvisc), b->sc);
            prof_end(b, SRDR_K_SWEEP, ev);
            counted(SRDR_K_SWEEP, 1);
        }
        prof_begin(b, SRDR_K_PASS_B, &ev);
        if (tiled)
            k_pass_b_tiled<T, D><<<b->nbricks, kTileThreads, smem_b, q>>>(A, tl, damp ? 0 : 1);
        else if (tab)
            k_pass_b_tab<T, D, KD><<<nb, kThreads, 0, q>>>(A, stab, damp ? 0 : 1);
        else if (b->stencil)
            k_pass_b<T, D, 1><<<nb, kThreads, 0, q>>>(A, damp ? 0 : 1);
        else
            k_pass_b<T, D, 0><<<nb, kThreads, 0, q>>>(A, damp ? 0 : 1);
        prof_end(b, SRDR_K_PASS_B, ev);
        counted(SRDR_K_PASS_B, 1);
        if (dev ? damping : damp) {
            prof_begin(b, SRDR_K_SWEEP, &ev);
            SRDR_CK(cudaLaunchCooperativeKernel(sl.fn, dim3(grid), dim3(sl.threads),
                                                dev ? sweep_params_d : sweep_params, smem, q));
            prof_end(b, SRDR_K_SWEEP, ev);
            counted(SRDR_K_SWEEP, 1);
            prof_begin(b, SRDR_K_FINISH, &ev);
            k_finish<T><<<nb, kThreads, 0, q>>>(A);
            prof_end(b, SRDR_K_FINISH, ev);
            counted(SRDR_K_FINISH, 1);
        }
        // the KE: reduced by the last block of the sliced-ELL force pass
        // (undamped step) or of the finish pass (damped step); after the
        // brick-tiled force pass, by two kernels of its own
        if (tiled && (dev || !damp)) {
            prof_begin(b, SRDR_K_KE, &ev);
            k_ke_slices<<<nb, kThreads, 0, q>>>(b->ke_pp, (int)b->n, b->ke_part, b->sc, A.dflag);
            k_ke_final<<<1, kKeThreads, 0, q>>>(b->ke_part, b->nslices, b->sc, A.dflag);
            prof_end(b, SRDR_K_KE, ev);
            counted(SRDR_K_KE, 2);
        }
        return SRDR_OK;
    };

    int64_t s0 = 0;
    // small bodies: replay a captured graph of kGraphSteps device-decided
    // steps (their steps are short enough for launch overhead to dominate)
    if (!b->profiling && b->graphs_ok && b->n <= kGraphMaxN && nsteps >= kGraphSteps) {
        if (!b->dflag_d) {
            SRDR_TRY(dalloc(b, &b->dflag_d, 1));
            SRDR_CK(cudaMemsetAsync(b->dflag_d, 0, sizeof(int), st));
        }
        ad.dflag = b->dflag_d;
        swd.dflag = b->dflag_d;
        if (!b->graph) {
            // captured on a private stream (the body's may be the legacy
            // default stream, which cannot be captured); launches are not
            // counted while capturing
            cudaStream_t cs = nullptr;
            cudaGraph_t g = nullptr;
            const int64_t l0 = b->launches;
            int64_t k0[SRDR_K_NCLASS];
            for (int k = 0; k < SRDR_K_NCLASS; ++k) k0[k] = b->k_launch[k];
            bool ok = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) == cudaSuccess &&
                      cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
            if (ok) {
                for (int k = 0; k < kGraphSteps && ok; ++k) ok = one_step(cs, true, false) == SRDR_OK;
                ok = (cudaStreamEndCapture(cs, &g) == cudaSuccess) && ok && g &&
                     cudaGraphInstantiate(&b->graph, g, 0) == cudaSuccess;
            }
            if (g) cudaGraphDestroy(g);
            if (cs) cudaStreamDestroy(cs);
            cudaGetLastError();
            b->launches = l0;
            for (int k = 0; k < SRDR_K_NCLASS; ++k) b->graph_launches[k] = b->k_launch[k] - k0[k];
            for (int k = 0; k < SRDR_K_NCLASS; ++k) b->k_launch[k] = k0[k];
            if (!ok) {
                b->graph = nullptr;
                b->graphs_ok = 0;
            }
        }
        if (b->graph) {
            const int64_t ng = nsteps / kGraphSteps;
            for (int64_t g = 0; g < ng; ++g) {
                SRDR_CK(cudaGraphLaunch(b->graph, st));
                for (int k = 0; k < SRDR_K_NCLASS; ++k) counted(k, (int)b->graph_launches[k]);
            }
            s0 = ng * kGraphSteps;
        }
    }
    for (int64_t s = s0; s < nsteps; ++s) {
        const uint64_t step = (uint64_t)(b->step + s);
        const bool damp = damping && random_phi(b->desc.seed, step) < b->desc.alpha;
        b->prof_active = b->profiling > 0 && step % (uint64_t)b->profiling == 0;
        const srdr_status r = one_step(st, false, damp);
        b->prof_active = 0;
        SRDR_TRY(r);
    }
    SRDR_CK(cudaGetLastError());
    b->step += nsteps;
    return SRDR_OK;
}

template <typename T>
srdr_status steps_dispatch(srdr_body* b, int64_t nsteps)
{
    int mat = b->desc.material == SRDR_NEO_HOOKEAN ? 1 : 0;
    if (b->dim == 2)
        return mat ? steps_typed<T, 2, 1>(b, nsteps) : steps_typed<T, 2, 0>(b, nsteps);
    return mat ? steps_typed<T, 3, 1>(b, nsteps) : steps_typed<T, 3, 0>(b, nsteps);
}

}  // namespace

srdr_status launch_steps(srdr_body* b, int64_t nsteps)
{
    if (nsteps <= 0) return SRDR_OK;
    if (b->prec == SRDR_FP64) return steps_dispatch<double>(b, nsteps);
    return steps_dispatch<float>(b, nsteps);
}

srdr_status reset_scalars(srdr_body* b, double tol)
{
    k_set_tol<<<1, 1, 0, b->stream>>>(b->sc, tol);
    SRDR_CK(cudaGetLastError());
    return SRDR_OK;
}

srdr_status sync_scalars(const srdr_body* b)
{
    SRDR_CK(cudaMemcpyAsync(b->sc_host, b->sc, sizeof(DevScalars), cudaMemcpyDeviceToHost, b->stream));
    SRDR_CK(cudaStreamSynchronize(b->stream));
    return SRDR_OK;
}

}  // namespace srdr
