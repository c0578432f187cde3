// tiles.cuh — brick-tiled stress and force passes (included by step.cu
// after passes.cuh, inside its anonymous namespace).
//
// One block per brick of cells.  The block copies the data its particles'
// neighbours need (u for the stress pass, P B0 for the force pass) for the
// brick's whole cell halo into shared memory with 16-byte asynchronous
// copies, then each thread takes one own particle and streams its row from
// the brick sliced-ELL layout: a 16-bit halo index and g_ij per slot.  The
// rows keep the neighbour order of the sliced-ELL layout and the per-slot
// arithmetic is the same explicitly rounded code (acc_grad, acc_force), so
// the results are bitwise those of k_pass_a / k_pass_b; only the gathers
// move from L1/L2 to shared memory.

constexpr int kTileThreads = 256;
constexpr int kTileUnroll = 8;  // slots per batch of stream loads (shared-memory gathers are cheap)

template <typename T>
struct TileArgs {
    const BrickInfo* __restrict__ info;
    const int* __restrict__ own;         // [n] sorted index of own particle (brick order)
    const uint16_t* __restrict__ own_h;  // [n] its halo index
    const int* __restrict__ halo;        // halo particle lists
    const int* __restrict__ sell_ptr;    // brick slice slot offsets
    const uint16_t* __restrict__ lidx;   // [slots] neighbour halo index
    const T* __restrict__ g0;            // [slots] pair gradient components
    const T* __restrict__ g1;
    const T* __restrict__ g2;
    double* __restrict__ ke_pp;          // [n] kinetic energy per particle
};

__device__ inline void cp_async16(void* dst, const void* src)
{
    const unsigned d = static_cast<unsigned>(__cvta_generic_to_shared(dst));
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ inline void cp_async_wait_all_t() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// halo copy of P B0: record h of the block's halo (pb_chunks x 16 bytes,
// entries in row-major order) <- the pb_full whole chunks of particle
// halo[h] (chunk c of particle j at 16-byte index c n + j of src) and its
// pb_tail leftover entries (entry t at T index (pb_full E + t) n + j)
template <typename T, int D>
__device__ inline void stage_halo_pb(unsigned char* dst, const T* src, int n, const int* __restrict__ halo,
                                     int nh)
{
    constexpr int C = pb_chunks(sizeof(T), D), F = pb_full(sizeof(T), D), TL = pb_tail(sizeof(T), D);
    constexpr int E = 16 / (int)sizeof(T);
    constexpr int K = F + TL;  // copies per halo particle
    const unsigned char* sb = reinterpret_cast<const unsigned char*>(src);
    for (int q = threadIdx.x; q < nh * K; q += blockDim.x) {
        const int h = q / K, c = q - h * K;
        const int j = __ldg(halo + h);
        if (c < F)
            cp_async16(dst + ((size_t)h * C + c) * 16, sb + ((size_t)c * n + j) * 16);
        else
            cp_async_t<T>(reinterpret_cast<T*>(dst + (size_t)h * C * 16) + F * E + (c - F),
                          src + (size_t)(F * E + c - F) * n + j);
    }
    cp_async_wait_all_t();
    __syncthreads();
}

// halo copy of FP64 u records (two 16-byte chunks each)
__device__ inline void stage_halo_u64(unsigned char* dst, const unsigned char* src, const int* __restrict__ halo,
                                      int nh)
{
    for (int q = threadIdx.x; q < 2 * nh; q += blockDim.x) {
        const int h = q >> 1, c = q & 1;
        const int j = __ldg(halo + h);
        cp_async16(dst + ((size_t)h * 2 + c) * 16, src + ((size_t)j * 2 + c) * 16);
    }
    cp_async_wait_all_t();
    __syncthreads();
}

// u of halo record l from shared memory (FP32: (hi, lo x) records, then the
// (lo y, lo z) pairs after all nh of them)
template <typename T>
__device__ inline void u_smem(const unsigned char* s, int nh, int l, T (&x)[3], T (&lo)[3])
{
    if constexpr (sizeof(T) == 4) {
        const float4 a = reinterpret_cast<const float4*>(s)[l];
        const float2 b = reinterpret_cast<const float2*>(s + (size_t)nh * 16)[l];
        x[0] = a.x; x[1] = a.y; x[2] = a.z;
        lo[0] = a.w; lo[1] = b.x; lo[2] = b.y;
    } else {
        const double2* q = reinterpret_cast<const double2*>(s) + (size_t)l * 2;
        const double2 a = q[0], b = q[1];
        x[0] = a.x; x[1] = a.y; x[2] = b.x;
        lo[0] = lo[1] = lo[2] = 0;
    }
}

// P B0 of halo record l from shared memory: the D x D entries row-major in
// pb_chunks 16-byte chunks
template <typename T, int D>
__device__ inline void pb_smem(const T* s, int l, T (&m)[D][D])
{
    constexpr int C = pb_chunks(sizeof(T), D);
    constexpr int E = C * 16 / (int)sizeof(T);
    T e[E];
    if constexpr (sizeof(T) == 4) {
        const float4* q = reinterpret_cast<const float4*>(s + (size_t)l * E);
#pragma unroll
        for (int c = 0; c < C; ++c) {
            const float4 x = q[c];
            e[4 * c] = x.x;
            e[4 * c + 1] = x.y;
            e[4 * c + 2] = x.z;
            e[4 * c + 3] = x.w;
        }
    } else {
        const double2* q = reinterpret_cast<const double2*>(s + (size_t)l * E);
#pragma unroll
        for (int c = 0; c < C; ++c) {
            const double2 x = q[c];
            e[2 * c] = x.x;
            e[2 * c + 1] = x.y;
        }
    }
#pragma unroll
    for (int p = 0; p < D; ++p)
#pragma unroll
        for (int q = 0; q < D; ++q) m[p][q] = e[p * D + q];
}

template <typename T, int D, int MAT>
__global__ void __launch_bounds__(kTileThreads) k_pass_a_tiled(StepArgs<T> a, TileArgs<T> tl)
{
    if (a.sc->done) return;
    extern __shared__ __align__(16) unsigned char tsm[];
    const BrickInfo bi = tl.info[blockIdx.x];
    const int nh = bi.nhalo;
    if constexpr (sizeof(T) == 4) {
        // a 16-byte (hi, lo x) record and an 8-byte (lo y, lo z) pair per
        // halo particle
        const int* hl = tl.halo + bi.halo_base;
        for (int h = threadIdx.x; h < nh; h += blockDim.x) {
            const size_t j = (size_t)__ldg(hl + h);
            cp_async16(tsm + (size_t)h * 16, a.uhi + j * 4);
            cp_async8(tsm + (size_t)nh * 16 + (size_t)h * 8, a.ulo + j * 2);
        }
        cp_async_wait_all_t();
        __syncthreads();
    } else {
        stage_halo_u64(tsm, reinterpret_cast<const unsigned char*>(a.u), tl.halo + bi.halo_base, nh);
    }
    const int lane = threadIdx.x & 31;
    for (int k0 = 0; k0 < bi.nown; k0 += blockDim.x) {
        const int k = k0 + threadIdx.x;
        if (k - lane >= bi.nown) break;  // the warp's slice is past the brick's particles
        const bool own = k < bi.nown;
        const int hi = own ? tl.own_h[bi.own_base + k] : 0;
        const int sl = bi.slice_base + (k >> 5);
        const int base = __ldg(tl.sell_ptr + sl);
        const int width = (__ldg(tl.sell_ptr + sl + 1) - base) >> 5;
        T xi[3], li[3];
        u_smem<T>(tsm, nh, hi, xi, li);
        T G[D][D];
#pragma unroll
        for (int p = 0; p < D; ++p)
#pragma unroll
            for (int q = 0; q < D; ++q) G[p][q] = 0;
        for (int t0 = 0; t0 < width; t0 += kTileUnroll) {
            int ll[kTileUnroll];
            T gg[kTileUnroll][D];
#pragma unroll
            for (int u = 0; u < kTileUnroll; ++u) {
                const int kk = base + (t0 + u) * 32 + lane;
                const bool in = t0 + u < width;
                ll[u] = in ? (int)ld_stream(tl.lidx + kk) : hi;
                gg[u][0] = in ? ld_stream(tl.g0 + kk) : T(0);
                gg[u][1] = in ? ld_stream(tl.g1 + kk) : T(0);
                if constexpr (D == 3) gg[u][2] = in ? ld_stream(tl.g2 + kk) : T(0);
            }
            T xj[kTileUnroll][3], lj[kTileUnroll][3];
#pragma unroll
            for (int u = 0; u < kTileUnroll; ++u) u_smem<T>(tsm, nh, ll[u], xj[u], lj[u]);
#pragma unroll
            for (int u = 0; u < kTileUnroll; ++u) acc_grad<T, D>(G, xi, li, xj[u], lj[u], gg[u]);
        }
        if (own) pass_a_epilogue<T, D, MAT>(a, tl.own[bi.own_base + k], G);
    }
}

template <typename T, int D>
__global__ void __launch_bounds__(kTileThreads) k_pass_b_tiled(StepArgs<T> a, TileArgs<T> tl, int final_step)
{
    if (a.sc->done) return;
    if (a.dflag) final_step = *a.dflag == 0;
    extern __shared__ __align__(16) unsigned char tsm[];
    const BrickInfo bi = tl.info[blockIdx.x];
    stage_halo_pb<T, D>(tsm, a.PB, a.n, tl.halo + bi.halo_base, bi.nhalo);
    const T* spb = reinterpret_cast<const T*>(tsm);
    const int lane = threadIdx.x & 31;
    for (int k0 = 0; k0 < bi.nown; k0 += blockDim.x) {
        const int k = k0 + threadIdx.x;
        if (k - lane >= bi.nown) break;
        const bool own = k < bi.nown;
        const int hi = own ? tl.own_h[bi.own_base + k] : 0;
        const int sl = bi.slice_base + (k >> 5);
        const int base = __ldg(tl.sell_ptr + sl);
        const int width = (__ldg(tl.sell_ptr + sl + 1) - base) >> 5;
        T Pi[D][D];
        pb_smem<T, D>(spb, hi, Pi);
        T acc[D];
#pragma unroll
        for (int p = 0; p < D; ++p) acc[p] = 0;
        for (int t0 = 0; t0 < width; t0 += kTileUnroll) {
            int ll[kTileUnroll];
            T gg[kTileUnroll][D];
#pragma unroll
            for (int u = 0; u < kTileUnroll; ++u) {
                const int kk = base + (t0 + u) * 32 + lane;
                const bool in = t0 + u < width;
                ll[u] = in ? (int)ld_stream(tl.lidx + kk) : hi;
                gg[u][0] = in ? ld_stream(tl.g0 + kk) : T(0);
                gg[u][1] = in ? ld_stream(tl.g1 + kk) : T(0);
                if constexpr (D == 3) gg[u][2] = in ? ld_stream(tl.g2 + kk) : T(0);
            }
            T Pj[kTileUnroll][D][D];
#pragma unroll
            for (int u = 0; u < kTileUnroll; ++u) pb_smem<T, D>(spb, ll[u], Pj[u]);
#pragma unroll
            for (int u = 0; u < kTileUnroll; ++u) acc_force<T, D>(acc, Pi, Pj[u], gg[u]);
        }
        if (own) {
            const int i = tl.own[bi.own_base + k];
            const double ke = pass_b_epilogue<T, D>(a, i, acc, Pi, final_step);
            if (final_step) tl.ke_pp[i] = ke;
        }
    }
}

// KE slice partials (sorted order) from the per-particle energies of a tiled
// final force pass: the warp sums of slice_partial_store, so the body's KE
// has the same bits as with the sliced-ELL force pass
__global__ void __launch_bounds__(kThreads) k_ke_slices(const double* __restrict__ ke_pp, int n,
                                                         double* __restrict__ part, const DevScalars* sc,
                                                         const int* dflag)
{
    if (sc->done || (dflag && *dflag)) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    slice_partial_store(i < n ? ke_pp[i] : 0.0, part, i, n);
}

template <typename T>
TileArgs<T> make_tile_args(srdr_body* b)
{
    TileArgs<T> t{};
    t.info = b->binfo;
    t.own = b->bown;
    t.own_h = b->bown_h;
    t.halo = b->bhalo;
    t.sell_ptr = b->bsell_ptr;
    t.lidx = b->blidx;
    t.g0 = static_cast<const T*>(b->bg);
    t.g1 = t.g0 + b->bslots;
    t.g2 = t.g1 + b->bslots;
    t.ke_pp = b->ke_pp;
    return t;
}
