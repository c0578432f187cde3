// sweep.cuh — the damping operator S_d of one damped step (included by
// step.cu inside its anonymous namespace).
//
// Eq. particle-by-particle-splitting: the local operators D_i run over all
// particles in the canonical order (colour, cell, particle id) with dt/2,
// then in the exact reverse order with dt/2 (Sec. 3.1; pairwise variant
// Sec. 3.2).  Cells of one colour have disjoint 3^d footprints (Sec. 3.4), so
// they run concurrently and commute; the colours run one after another with
// a bounded grid barrier in one cooperative launch.
//
// Mapping: one warp per block holds G cells, one group of L = 32/G lanes per
// cell.  A group stages its cell's footprint velocities and inverse masses
// (through L2: other SMs wrote them in earlier colour phases), the cell's CSR
// rows and per-particle constants (read-only: cp.async, no register staging)
// in shared memory, then updates the cell's particles one after another,
// its lanes spread over each particle's neighbours.  More cells per warp give
// each warp independent work to overlap the serial in-cell chain; fewer give
// fewer shuffle levels per reduction.  G is chosen by the autotuner.

// ---------------------------------------------------------------- async copies
__device__ inline void cp_async4(void* dst, const void* src)
{
    const unsigned d = static_cast<unsigned>(__cvta_generic_to_shared(dst));
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ inline void cp_async8(void* dst, const void* src)
{
    const unsigned d = static_cast<unsigned>(__cvta_generic_to_shared(dst));
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(src) : "memory");
}
template <typename T>
__device__ inline void cp_async_t(T* dst, const T* src)
{
    if constexpr (sizeof(T) == 8)
        cp_async8(dst, src);
    else
        cp_async4(dst, src);
}
__device__ inline void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// ---------------------------------------------------------------- footprint runs
// The <= 9 runs of a cell's footprint (same z-outer, y-inner order as the
// footprint-local indices written at set-up), known to every lane of the
// group: run r covers sorted particles [a[r], a[r] + off[r+1] - off[r]) and
// sits at footprint-local offset off[r].
struct FootRuns {
    int nruns;
    int total;
    int a[9];
    int off[10];
    __device__ int particle(int q) const
    {
        int j = 0;
#pragma unroll
        for (int r = 0; r < 9; ++r)
            if (r < nruns && q >= off[r]) j = a[r] + (q - off[r]);
        return j;
    }
};

template <int L>
__device__ inline FootRuns foot_runs_group(int c, int dim, int nx, int ny, int nz,
                                           const int* __restrict__ start, int gl, unsigned gmask)
{
    const int cx = c % nx, cy = (c / nx) % ny, cz = c / (nx * ny);
    const int xlo = max(cx - 1, 0), xhi = min(cx + 1, nx - 1);
    const int ylo = dim >= 2 ? max(cy - 1, 0) : 0, yhi = dim >= 2 ? min(cy + 1, ny - 1) : 0;
    const int zlo = dim >= 3 ? max(cz - 1, 0) : 0, zhi = dim >= 3 ? min(cz + 1, nz - 1) : 0;
    const int ny_r = yhi - ylo + 1;
    FootRuns f;
    f.nruns = ny_r * (zhi - zlo + 1);
    // with L < 9 lanes some lanes find more than one run
    int ra[(9 + L - 1) / L], len[(9 + L - 1) / L];
#pragma unroll
    for (int q = 0; q < (9 + L - 1) / L; ++q) {
        const int r = gl + q * L;
        ra[q] = 0;
        len[q] = 0;
        if (r < f.nruns) {
            const int y = ylo + r % ny_r, z = zlo + r / ny_r;
            const int c0 = xlo + nx * (y + ny * z), c1 = xhi + nx * (y + ny * z);
            ra[q] = __ldg(start + c0);
            len[q] = __ldg(start + c1 + 1) - ra[q];
        }
    }
    int run = 0;
#pragma unroll
    for (int r = 0; r < 9; ++r) {
        const int aa = __shfl_sync(gmask, ra[r / L], r % L, L);
        const int ll = __shfl_sync(gmask, len[r / L], r % L, L);
        f.a[r] = aa;
        f.off[r] = run;
        run += r < f.nruns ? ll : 0;
    }
    f.off[9] = run;
    f.total = run;
    return f;
}

// ---------------------------------------------------------------- grid barrier
// Bounded grid barrier of a cooperative launch (all blocks co-resident).  The
// last block to arrive resets the count and bumps the generation; the others
// wait on the generation with a sleep, and give up after 2^24 polls, setting
// DEV_TIMEOUT in sc->status so that the host gets an error instead of a hung
// GPU.  Thread 0 of the block does the protocol; every thread of the block
// must call it.
__device__ inline bool grid_barrier(unsigned* count, volatile unsigned* gen, unsigned nblocks,
                                    DevScalars* sc)
{
    __shared__ int s_ok;
    __syncthreads();
    int ok = 1;
    if (threadIdx.x == 0) {
        unsigned g = *gen;
        __threadfence();
        if (atomicAdd(count, 1u) == nblocks - 1) {
            atomicExch(count, 0u);
            __threadfence();
            atomicAdd(const_cast<unsigned*>(gen), 1u);
        } else {
            long long polls = 0;
            while (*gen == g) {
                if (++polls > (1LL << 24)) {
                    atomicCAS(&sc->status, DEV_OK, DEV_TIMEOUT);
                    ok = 0;
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
        if (*(volatile int*)&sc->status == DEV_TIMEOUT) ok = 0;
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// ---------------------------------------------------------------- shared memory
// Per cell (group):
//   sv [D][F] footprint velocities, sminv [F] inverse masses, sw [P] weights,
//   sm / s1 / s2 [C] mass, sum w, sum w^2 of the cell's particles,
//   srow [C+1] absolute row starts, sl [P+4] footprint-local indices (uint16)
template <typename T, int D>
struct CellSmem {
    T* sv;
    T* sminv;
    T* sw;
    T* sm;
    T* s1;
    T* s2;
    int* srow;
    uint16_t* sl;
};

template <typename T, int D>
__host__ __device__ inline size_t cell_smem_bytes(int F, int P, int C)
{
    size_t b = sizeof(T) * ((size_t)(D + 1) * F + (size_t)P + 3 * (size_t)C);
    b = (b + 3) & ~size_t(3);
    b += sizeof(int) * ((size_t)C + 1);
    b += sizeof(uint16_t) * ((size_t)P + 4);
    return (b + 15) & ~size_t(15);
}

template <typename T, int D>
__device__ inline CellSmem<T, D> cell_smem(unsigned char* raw, int F, int P, int C)
{
    CellSmem<T, D> s;
    s.sv = reinterpret_cast<T*>(raw);
    s.sminv = s.sv + (size_t)D * F;
    s.sw = s.sminv + F;
    s.sm = s.sw + P;
    s.s1 = s.sm + C;
    s.s2 = s.s1 + C;
    size_t off = sizeof(T) * ((size_t)(D + 1) * F + (size_t)P + 3 * (size_t)C);
    off = (off + 3) & ~size_t(3);
    s.srow = reinterpret_cast<int*>(raw + off);
    s.sl = reinterpret_cast<uint16_t*>(s.srow + C + 1);
    return s;
}

template <typename T, int L>
__device__ inline T group_allsum(T x, unsigned gmask)
{
#pragma unroll
    for (int o = L / 2; o > 0; o >>= 1) x += __shfl_xor_sync(gmask, x, o, L);
    return x;
}

// ---------------------------------------------------------------- one cell
template <typename T, int D, int L>
__device__ inline void sweep_cell(const SweepArgs<T>& a, int c, int backward, const CellSmem<T, D>& s,
                                  int gl, unsigned gmask)
{
    const int n = a.n;
    const int cs = __ldg(a.cell_start + c), ce = __ldg(a.cell_start + c + 1);
    const int np = ce - cs;
    const int F = a.max_foot;
    T* sv = s.sv;
    T* sminv = s.sminv;
    T* sw = s.sw;
    const T cc = a.c;

    const FootRuns fr = foot_runs_group<L>(c, a.dim, a.nx, a.ny, a.nz, a.cell_start, gl, gmask);
    const int Ftot = fr.total;
    int my_off = 0;
#pragma unroll
    for (int r = 0; r < 9; ++r)
        if (r < fr.nruns && cs >= fr.a[r] && cs < fr.a[r] + (fr.off[r + 1] - fr.off[r]))
            my_off = fr.off[r] + (cs - fr.a[r]);
    const int p0 = __ldg(a.row_ptr + cs), p1 = __ldg(a.row_ptr + ce);

    // read-only data by asynchronous copies: CSR weights, footprint-local
    // indices (as 32-bit words from an even start), rows, masses, sums
    for (int k = p0 + gl; k < p1; k += L) cp_async_t(sw + (k - p0), a.w + k);
    {
        const int w0 = p0 >> 1, w1 = (p1 + 1) >> 1;
        const uint32_t* lw = reinterpret_cast<const uint32_t*>(a.loc);
        uint32_t* sw32 = reinterpret_cast<uint32_t*>(s.sl);
        for (int k = w0 + gl; k < w1; k += L) cp_async4(sw32 + (k - w0), lw + k);
    }
    for (int p = gl; p <= np; p += L) cp_async4(s.srow + p, a.row_ptr + cs + p);
    for (int p = gl; p < np; p += L) {
        cp_async_t(s.sm + p, a.mass + cs + p);
        cp_async_t(s.s1 + p, a.sumw + cs + p);
        cp_async_t(s.s2 + p, a.sumw2 + cs + p);
    }
    // velocities through L2 (ld.cg) and inverse masses, in register batches:
    // every load of a batch is issued before its shared-memory stores
    constexpr int U = 16;
    for (int base = 0; base < Ftot; base += L * U) {
        T tv[U][D], tm[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int q = base + u * L + gl;
            if (q < Ftot) {
                const int j = fr.particle(q);
#pragma unroll
                for (int d = 0; d < D; ++d) tv[u][d] = __ldcg(a.v + (size_t)d * n + j);
                tm[u] = __ldg(a.minv + j);
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int q = base + u * L + gl;
            if (q < Ftot) {
#pragma unroll
                for (int d = 0; d < D; ++d) sv[d * F + q] = tv[u][d];
                sminv[q] = tm[u];
            }
        }
    }
    cp_async_wait_all();
    __syncwarp(gmask);
    const uint16_t* sl = s.sl + (p0 & 1);  // entry k at sl[k - p0]

    for (int t = 0; t < np; ++t) {
        const int p = backward ? np - 1 - t : t;
        const int li = my_off + p;
        const int k0 = s.srow[p] - p0, k1 = s.srow[p + 1] - p0;
        if (!a.pairwise) {
            const T mi = s.sm[p];
            const T SB = cc * s.s1[p];
            const T SB2 = cc * cc * s.s2[p];
            T vi[D], E[D];
#pragma unroll
            for (int d = 0; d < D; ++d) {
                vi[d] = sv[d * F + li];
                E[d] = 0;
            }
            // E_i = -sum_j B_j (v_i - v_j), summed in the order of a 32-lane
            // butterfly whatever L is: lane gl of the group keeps the 32/L
            // "virtual lanes" gl + w L (neighbours k = virtual lane mod 32)
            // and combines them as the first butterfly levels would, so the
            // result does not depend on the cells-per-warp choice.  Rows of up
            // to L*NK neighbours keep their indices, weights and velocities in
            // registers: every shared-memory load of the particle is issued
            // before any of its stores.
            constexpr int V = 32 / L;
            constexpr int NK = L == 32 ? 4 : (L == 16 ? 8 : 12);
            T acc[V][D];
#pragma unroll
            for (int w = 0; w < V; ++w)
#pragma unroll
                for (int d = 0; d < D; ++d) acc[w][d] = 0;
            const bool in_regs = k1 - k0 <= L * NK;
            int jj[NK];
            T BB[NK], vj[NK][D], im[NK];
            if (in_regs) {
#pragma unroll
                for (int m = 0; m < NK; ++m) {
                    const int k = k0 + gl + m * L;
                    const bool ok = k < k1;
                    jj[m] = ok ? (int)sl[k] : li;
                    BB[m] = ok ? cc * sw[k] : T(0);
                }
#pragma unroll
                for (int m = 0; m < NK; ++m) {
#pragma unroll
                    for (int d = 0; d < D; ++d) vj[m][d] = sv[d * F + jj[m]];
                    im[m] = sminv[jj[m]];
                }
#pragma unroll
                for (int m = 0; m < NK; ++m)
                    if (k0 + gl + m * L < k1)
#pragma unroll
                        for (int d = 0; d < D; ++d) acc[m % V][d] -= BB[m] * (vi[d] - vj[m][d]);
            } else {
                for (int kb = k0 + gl; kb < k1; kb += 32) {
#pragma unroll
                    for (int w = 0; w < V; ++w) {
                        const int k = kb + w * L;
                        if (k < k1) {
                            const int j = sl[k];
                            const T B = cc * sw[k];
#pragma unroll
                            for (int d = 0; d < D; ++d) acc[w][d] -= B * (vi[d] - sv[d * F + j]);
                        }
                    }
                }
            }
#pragma unroll
            for (int o = 16; o >= L; o >>= 1) {
                const int sft = o / L;
#pragma unroll
                for (int w = 0; w < V; ++w)
                    if ((w & sft) == 0 && (w | sft) < V)
#pragma unroll
                        for (int d = 0; d < D; ++d) acc[w][d] = acc[w][d] + acc[w | sft][d];
            }
#pragma unroll
            for (int d = 0; d < D; ++d) E[d] = group_allsum<T, L>(acc[0][d], gmask);
            // k = E_i / ((sum B - m_i)^2 + sum B^2);  v_i += (sum B - m_i) k
            const T sbm = SB - mi;
            const T rden = T(1) / (sbm * sbm + SB2);
            T kk[D], vin[D];
#pragma unroll
            for (int d = 0; d < D; ++d) {
                kk[d] = E[d] * rden;
                vin[d] = vi[d] + sbm * kk[d];
            }
            // v_j <- v_j - B_j (v_i^new - v_j^p) / m_j,  v_j^p = v_j - B_j k
            if (in_regs) {
#pragma unroll
                for (int m = 0; m < NK; ++m)
                    if (k0 + gl + m * L < k1)
#pragma unroll
                        for (int d = 0; d < D; ++d)
                            sv[d * F + jj[m]] = vj[m][d] - BB[m] * (vin[d] - vj[m][d] + BB[m] * kk[d]) * im[m];
            } else {
                for (int k = k0 + gl; k < k1; k += L) {
                    const int j = sl[k];
                    const T B = cc * sw[k];
                    const T imj = sminv[j];
#pragma unroll
                    for (int d = 0; d < D; ++d) {
                        const T vjd = sv[d * F + j];
                        sv[d * F + j] = vjd - B * (vin[d] - vjd + B * kk[d]) * imj;
                    }
                }
            }
            __syncwarp(gmask);
            if (gl == 0) {
#pragma unroll
                for (int d = 0; d < D; ++d) sv[d * F + li] = vin[d];
            }
            __syncwarp(gmask);
        } else {
            // pairwise (Sec. 3.2): pairs in row order, then reversed, each
            // solved in closed form (Eq. pairwise-solve) over half the step
            if (gl == 0) {
                const T mi = s.sm[p];
                const T ch = T(0.5) * cc;
                for (int pass = 0; pass < 2; ++pass) {
                    for (int t2 = 0; t2 < k1 - k0; ++t2) {
                        const int k = pass == 0 ? k0 + t2 : k1 - 1 - t2;
                        const int j = sl[k];
                        const T B = ch * sw[k];
                        const T mj = T(1) / sminv[j];
                        const T den = mi * mj - (mi + mj) * B;
#pragma unroll
                        for (int d = 0; d < D; ++d) {
                            const T vij = sv[d * F + li] - sv[d * F + j];
                            sv[d * F + li] += mj * B * vij / den;
                            sv[d * F + j] += -mi * B * vij / den;
                        }
                    }
                }
            }
            __syncwarp(gmask);
        }
    }
    // write the footprint back (through L2: other SMs read it after the barrier)
    for (int q = gl; q < Ftot; q += L) {
        const int j = fr.particle(q);
#pragma unroll
        for (int d = 0; d < D; ++d) __stcg(a.v + (size_t)d * n + j, sv[d * F + q]);
    }
    __syncwarp(gmask);
}

// The whole S_d of one damped step in one cooperative launch: colours
// 0..3^d-1 forward, then 3^d-1..0 backward, a bounded grid barrier between
// colour phases.  Blocks of W warps, G cell groups per warp; group number
// q = (block * W + warp) * G + g takes the colour's cells q, q + gridDim*W*G, ...
// More warps per block means fewer blocks arriving at the grid barrier.
template <typename T, int D, int G, int W>
__global__ void __launch_bounds__(32 * W) k_sweep_all(SweepArgs<T> a, const int* __restrict__ colour_ptr,
                                                      int ncolours, unsigned* bar)
{
    constexpr int L = 32 / G;
    if (*(volatile int*)&a.sc->done) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int wb = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g = lane / L, gl = lane % L;
    const unsigned gmask = (L == 32) ? 0xffffffffu : (((1u << L) - 1u) << (g * L));
    const size_t cell_bytes = cell_smem_bytes<T, D>(a.max_foot, a.max_pairs, a.max_cell);
    const CellSmem<T, D> s = cell_smem<T, D>(smem_raw + (size_t)(wb * G + g) * cell_bytes, a.max_foot,
                                             a.max_pairs, a.max_cell);
    const int q0 = (blockIdx.x * W + wb) * G + g, qs = gridDim.x * W * G;
    int phases = 0;
    for (int ph = 0; ph < 2 * ncolours; ++ph) {
        const int backward = ph >= ncolours;
        const int col = backward ? 2 * ncolours - 1 - ph : ph;
        const int c0 = __ldg(colour_ptr + col), c1 = __ldg(colour_ptr + col + 1);
        if (c1 == c0) continue;
        if (phases++ > 0 && !grid_barrier(bar, bar + 1, gridDim.x, a.sc)) return;
        for (int cid = c0 + q0; cid < c1; cid += qs)
            sweep_cell<T, D, L>(a, __ldg(a.colour_cells + cid), backward, s, gl, gmask);
        __syncwarp();
    }
}
