// sweep.cuh — the damping operator S_d of one damped step (included by
// step.cu inside its anonymous namespace).
//
// Eq. particle-by-particle-splitting: the local operators D_i run over all
// particles in the canonical order (colour, cell, particle id) with dt/2,
// then in the exact reverse order with dt/2 (Sec. 3.1; pairwise variant
// Sec. 3.2).  Cells of one colour have disjoint 3^d footprints (Sec. 3.4), so
// they run concurrently and commute.  All colour phases run in one
// cooperative launch, ordered either by a bounded grid barrier between
// consecutive phases (k_sweep_all) or by each cell waiting only for the
// cells whose footprints overlap its own (k_sweep_flow); both give the same
// bits.
//
// Mapping: a warp holds G cells, one group of L = 32/G lanes per cell.  A
// group stages in shared memory its cell's CSR rows, weights and per-particle
// constants (read-only, by cp.async), a table of its footprint's particle
// indices, and its footprint's velocity records (v, 1/m) (cp.async from L2: other SMs
// wrote them in earlier colour phases), then updates the cell's particles
// one after another, its lanes spread over each particle's neighbours, each
// particle's loop only as long as its row.  The read-only part of the group's
// next cell is requested before the grid barrier that precedes it, so only
// the velocities are fetched after the barrier; inside the chain the
// next particle's neighbour indices and weights are read while the current
// particle's sums are reduced.  More cells per warp give each warp
// independent work to overlap the serial in-cell chain; fewer give fewer
// shuffle levels per reduction.  G is chosen by the autotuner.

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
__device__ inline void cp_async16s(void* dst, const void* src)
{
    const unsigned d = static_cast<unsigned>(__cvta_generic_to_shared(dst));
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
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
// Bounded, split-phase grid barrier of a cooperative launch (all blocks
// co-resident); the wait gives up after kWaitNs or kWaitPolls.  Words of the barrier buffer (kBarWords unsigned, zeroed at
// creation), each group on its own 128-byte line:
//   sub-counter k (k < kBarSub) at 32 k, top counter at 32 kBarSub,
//   generation at 32 (kBarSub + 1).
// Block b arrives at sub-counter b mod S (S = min(kBarSub, blocks)); the last
// arrival of a sub-counter resets it and arrives at the top counter; the last
// arrival there resets it and bumps the generation.  Waiters poll the
// generation (its own line, so polling does not slow the counters) with a
// sleep and give up after five seconds, setting DEV_TIMEOUT in sc->status, so
// the host gets an error instead of a hung GPU.  Between arrive and wait a
// block may do work that does not depend on other blocks.
__device__ inline unsigned bar_arrive(unsigned* bar, unsigned nblocks)
{
    volatile unsigned* gen = bar + 32 * (kBarSub + 1);
    const unsigned g = *gen;
    __threadfence();  // the block's writes (ordered by the block barrier) before the arrival
    const unsigned ns = nblocks < (unsigned)kBarSub ? nblocks : (unsigned)kBarSub;
    const unsigned k = blockIdx.x % ns;
    const unsigned nk = nblocks / ns + (k < nblocks % ns ? 1u : 0u);
    unsigned* sub = bar + 32 * k;
    if (atomicAdd(sub, 1u) == nk - 1) {
        atomicExch(sub, 0u);
        __threadfence();
        unsigned* top = bar + 32 * kBarSub;
        if (atomicAdd(top, 1u) == ns - 1) {
            atomicExch(top, 0u);
            __threadfence();
            atomicAdd(const_cast<unsigned*>(gen), 1u);
        }
    }
    return g;
}

// device clock in nanoseconds
__device__ inline unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// bound of every wait of the sweep: far above the sweep of any body that
// fits on the device (a cell-wise wait may span all earlier colour phases:
// about 0.6 s for FP64 pairwise updates of the 2^d layout's large cells),
// short enough for a test to run one out; the poll count bounds the wait
// too, set above what the time bound allows
constexpr unsigned long long kWaitNs = 5000000000ull;
constexpr long long kWaitPolls = 1LL << 27;

__device__ inline bool bar_wait(unsigned* bar, unsigned g, DevScalars* sc)
{
    volatile unsigned* gen = bar + 32 * (kBarSub + 1);
    long long polls = 0;
    bool ok = true;
    const unsigned long long t0 = global_ns();
    while (*gen == g) {
        if ((++polls & 63) == 0 && (global_ns() - t0 > kWaitNs || polls > kWaitPolls)) {
            atomicCAS(&sc->status, DEV_OK, DEV_TIMEOUT);
            ok = false;
            break;
        }
        __nanosleep(100);
    }
    __threadfence();
    if (*(volatile int*)&sc->status == DEV_TIMEOUT) ok = false;
    return ok;
}

// ---------------------------------------------------------------- shared memory
// Per cell (group), each section on a 16-byte boundary:
//   sv [F + 1] footprint velocity records (vx, vy, vz, 1/m) and a zero
//   record at F that padded neighbour slots point at,
//   srec [P + 2] the rows' slot records (B_j pre-scaled, footprint-local j),
//   copied in 16-byte chunks from the chunk holding the cell's first row
//   entry (R = 16 / sizeof(SweepSlot<T>) records per chunk),
//   sm / sbm / srd [C] per particle of the cell: mass, sum_B - m_i and
//   1 / ((sum_B - m_i)^2 + sum_B^2) (precomputed per body),
//   srow [C+1] absolute row starts,
//   sfoot [F] the sorted particle index of each footprint-local index.
template <typename T, int D>
struct CellSmem {
    vec4_t<T>* sv;
    SweepSlot<T>* srec;
    T* sm;
    T* sbm;
    T* srd;
    int* srow;
    int* sfoot;
};

__host__ __device__ inline size_t align16(size_t b) { return (b + 15) & ~size_t(15); }

// byte offsets of the sections after sv: srec, sm (then sbm, srd), srow,
// sfoot, end
template <typename T, int D>
__host__ __device__ inline void cell_smem_offsets(int F, int P, int C, size_t (&o)[5])
{
    o[0] = align16(sizeof(T) * 4 * ((size_t)F + 1));
    o[1] = o[0] + align16(sizeof(SweepSlot<T>) * ((size_t)P + 2));
    o[2] = o[1] + align16(sizeof(T) * 3 * (size_t)C);
    o[3] = o[2] + align16(sizeof(int) * ((size_t)C + 1));
    o[4] = o[3] + align16(sizeof(int) * (size_t)F);
}

template <typename T, int D>
__host__ __device__ inline size_t cell_smem_bytes(int F, int P, int C)
{
    size_t o[5];
    cell_smem_offsets<T, D>(F, P, C, o);
    return o[4];
}

template <typename T, int D>
__device__ inline CellSmem<T, D> cell_smem(unsigned char* raw, int F, int P, int C)
{
    size_t o[5];
    cell_smem_offsets<T, D>(F, P, C, o);
    CellSmem<T, D> s;
    s.sv = reinterpret_cast<vec4_t<T>*>(raw);
    s.srec = reinterpret_cast<SweepSlot<T>*>(raw + o[0]);
    s.sm = reinterpret_cast<T*>(raw + o[1]);
    s.sbm = s.sm + C;
    s.srd = s.sbm + C;
    s.srow = reinterpret_cast<int*>(raw + o[2]);
    s.sfoot = reinterpret_cast<int*>(raw + o[3]);
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
// What a group knows about its staged cell.
struct CellStage {
    int cs, np, p0, p1, my_off;
    FootRuns fr;
};

// Stage the read-only data of cell c: footprint runs, row starts, CSR weights
// and footprint-local indices (16-byte chunks), masses and the local solve's
// constants, and the footprint index table (plain shared-memory stores).  The
// copies are asynchronous; run_cell waits for them.
template <typename T, int D, int L>
__device__ inline CellStage stage_cell(const SweepArgs<T>& a, int c, const CellSmem<T, D>& s, int gl,
                                       unsigned gmask)
{
    CellStage st;
    st.cs = __ldg(a.cell_start + c);
    const int ce = __ldg(a.cell_start + c + 1);
    st.np = ce - st.cs;
    if (a.foot_tab) {
        // 2^d layout: the cell's touched particles, listed at set-up
        const int f0 = __ldg(a.foot_ptr + c);
        st.fr.nruns = 0;
        st.fr.total = __ldg(a.foot_ptr + c + 1) - f0;
        st.my_off = __ldg(a.own_off + c);
        for (int q = gl; q < st.fr.total; q += L) cp_async4(s.sfoot + q, a.foot_tab + f0 + q);
    } else {
        st.fr = foot_runs_group<L>(c, a.dim, a.nx, a.ny, a.nz, a.cell_start, gl, gmask);
        st.my_off = 0;
#pragma unroll
        for (int r = 0; r < 9; ++r)
            if (r < st.fr.nruns && st.cs >= st.fr.a[r] && st.cs < st.fr.a[r] + (st.fr.off[r + 1] - st.fr.off[r]))
                st.my_off = st.fr.off[r] + (st.cs - st.fr.a[r]);
    }
    st.p0 = __ldg(a.row_ptr + st.cs);
    st.p1 = __ldg(a.row_ptr + ce);
    const int p0 = st.p0, p1 = st.p1, np = st.np;
    if (!a.rows_global) {
        // slot records in 16-byte chunks from the chunk holding entry p0
        // (the array has two spare records, so the last chunk stays inside it)
        constexpr int R = 16 / (int)sizeof(SweepSlot<T>);
        const int rb = p0 & ~(R - 1);
        for (int k = rb + gl * R; k < p1; k += L * R) cp_async16s(s.srec + (k - rb), a.rec + k);
    }
    // footprint-local index -> sorted particle index (the 3^d neighbour
    // cells' runs; the 2^d layout's list is being copied above)
#pragma unroll
    for (int r = 0; r < 9; ++r) {
        if (r < st.fr.nruns) {
            const int o = st.fr.off[r], len = st.fr.off[r + 1] - o, a0 = st.fr.a[r];
            for (int q = gl; q < len; q += L) s.sfoot[o + q] = a0 + q;
        }
    }
    for (int p = gl; p <= np; p += L) cp_async4(s.srow + p, a.row_ptr + st.cs + p);
    for (int p = gl; p < np; p += L) {
        cp_async_t(s.sm + p, a.mass + st.cs + p);
        cp_async_t(s.sbm + p, a.sbm + st.cs + p);
        cp_async_t(s.srd + p, a.srd + st.cs + p);
    }
    return st;
}

// The serial chain of a staged cell (run_cell): the local operators of its
// particles in order, in reverse order, or both (mode 0, 1, 2), on L lanes
// (gmask) of the group.
template <typename T, int D, int L>
__device__ inline void chain_cell(const SweepArgs<T>& a, const CellStage& st, int mode, const CellSmem<T, D>& s,
                                  const SweepSlot<T>* __restrict__ rec, int gl, unsigned gmask)
{
    using V4 = vec4_t<T>;
    const int np = st.np, p0 = st.p0, my_off = st.my_off;
    V4* sv = s.sv;
    const int pad = a.max_foot;  // the zero record: padded slots read and write it with B = 0
    for (int dir = mode == 1 ? 1 : 0; dir <= (mode == 0 ? 0 : 1); ++dir) {
    const int backward = dir;
    if (!a.pairwise) {
        // E_i = -sum_j B_j (v_i - v_j), summed in the order of a 32-lane
        // butterfly whatever L is: lane gl of the group keeps the 32/L
        // "virtual lanes" gl + w L (neighbours k = virtual lane mod 32) and
        // combines them as the first butterfly levels would, so the result
        // does not depend on the cells-per-warp choice.  Rows of up to L*NK
        // neighbours keep their indices and weights in registers, read for
        // the next particle while the current one is reduced.
        constexpr int V = 32 / L;
        constexpr int NK = L == 32 ? 4 : (L == 16 ? 8 : 12);
        int jj[NK];
        T BB[NK];
        int k0 = 0, k1 = 0;
        auto slots = [&](int t, int (&j_)[NK], T (&b_)[NK], int& a0, int& a1) {
            const int p = backward ? np - 1 - t : t;
            a0 = s.srow[p] - p0;
            a1 = s.srow[p + 1] - p0;
#pragma unroll
            for (int m = 0; m < NK; ++m) {
                const int k = a0 + gl + m * L;
                j_[m] = pad;
                b_[m] = T(0);
                if (k < a1) {
                    const SweepSlot<T> r = rec[k];
                    j_[m] = (int)r.loc;
                    b_[m] = r.B;
                }
            }
        };
        if (np > 0) slots(0, jj, BB, k0, k1);
        for (int t = 0; t < np; ++t) {
            const int p = backward ? np - 1 - t : t;
            const int li = my_off + p;
            const T sbm = s.sbm[p], rden = s.srd[p];
            const V4 vi4 = sv[li];
            const T vi[3] = {vi4.x, vi4.y, vi4.z};
            const bool in_regs = k1 - k0 <= L * NK;
            // slot batches holding row entries (the same for every lane of
            // the group); later batches are all padding and are skipped
            const int nk = (k1 - k0 + L - 1) / L;
            T acc[V][D];
#pragma unroll
            for (int w = 0; w < V; ++w)
#pragma unroll
                for (int d = 0; d < D; ++d) acc[w][d] = 0;
            V4 vj[NK];
            if (in_regs) {
#pragma unroll
                for (int m = 0; m < NK; ++m)
                    if (m < nk) vj[m] = sv[jj[m]];
            }
            // the next particle's slots (read-only data)
            int jn[NK];
            T Bn[NK];
            int k0n = 0, k1n = 0;
            if (t + 1 < np) slots(t + 1, jn, Bn, k0n, k1n);
            if (in_regs) {
#pragma unroll
                for (int m = 0; m < NK; ++m) {
                    if (m < nk) {
                        const T vjd[3] = {vj[m].x, vj[m].y, vj[m].z};
#pragma unroll
                        for (int d = 0; d < D; ++d) acc[m % V][d] -= BB[m] * (vi[d] - vjd[d]);
                    }
                }
            } else {
                for (int kb = k0 + gl; kb < k1; kb += 32) {
#pragma unroll
                    for (int w = 0; w < V; ++w) {
                        const int k = kb + w * L;
                        if (k < k1) {
                            const SweepSlot<T> r = rec[k];
                            const V4 x = sv[r.loc];
                            const T xd[3] = {x.x, x.y, x.z};
                            const T B = r.B;
#pragma unroll
                            for (int d = 0; d < D; ++d) acc[w][d] -= B * (vi[d] - xd[d]);
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
            // k = E_i / ((sum B - m_i)^2 + sum B^2);  v_i += (sum B - m_i) k
            T kk[3] = {0, 0, 0}, vin[3] = {vi[0], vi[1], vi[2]};
#pragma unroll
            for (int d = 0; d < D; ++d) {
                const T E = group_allsum<T, L>(acc[0][d], gmask);
                kk[d] = E * rden;
                vin[d] = vi[d] + sbm * kk[d];
            }
            // v_j <- v_j - B_j (v_i^new - v_j^p) / m_j,  v_j^p = v_j - B_j k
            if (in_regs) {
                // padded slots write the zero record back unchanged (B = 0)
#pragma unroll
                for (int m = 0; m < NK; ++m) {
                    if (m < nk) {
                        const T vjd[3] = {vj[m].x, vj[m].y, vj[m].z};
                        T o[3] = {vjd[0], vjd[1], vjd[2]};
#pragma unroll
                        for (int d = 0; d < D; ++d)
                            o[d] = vjd[d] - BB[m] * (vin[d] - vjd[d] + BB[m] * kk[d]) * vj[m].w;
                        sv[jj[m]] = V4{o[0], o[1], o[2], vj[m].w};
                    }
                }
            } else {
                for (int k = k0 + gl; k < k1; k += L) {
                    const SweepSlot<T> r = rec[k];
                    const int j = (int)r.loc;
                    const T B = r.B;
                    const V4 x = sv[j];
                    const T xd[3] = {x.x, x.y, x.z};
                    T o[3] = {xd[0], xd[1], xd[2]};
#pragma unroll
                    for (int d = 0; d < D; ++d) o[d] = xd[d] - B * (vin[d] - xd[d] + B * kk[d]) * x.w;
                    sv[j] = V4{o[0], o[1], o[2], x.w};
                }
            }
            // no lane writes record li above (rows exclude the particle
            // itself) and every lane read it before the reduction's shuffles
            if (gl == 0) sv[li] = V4{vin[0], vin[1], vin[2], vi4.w};
            __syncwarp(gmask);
#pragma unroll
            for (int m = 0; m < NK; ++m) {
                jj[m] = jn[m];
                BB[m] = Bn[m];
            }
            k0 = k0n;
            k1 = k1n;
        }
    } else {
        // pairwise (Sec. 3.2): for each particle, its pairs in row order,
        // then reversed, each solved in closed form (Eq. pairwise-solve) over
        // half the step
        if (gl == 0) {
            for (int t = 0; t < np; ++t) {
                const int p = backward ? np - 1 - t : t;
                const int li = my_off + p;
                const int k0 = s.srow[p] - p0, k1 = s.srow[p + 1] - p0;
                const T mi = s.sm[p];
                for (int pass = 0; pass < 2; ++pass) {
                    for (int t2 = 0; t2 < k1 - k0; ++t2) {
                        const int k = pass == 0 ? k0 + t2 : k1 - 1 - t2;
                        const SweepSlot<T> r = rec[k];
                        const int j = (int)r.loc;
                        // half the step: (c/2) w = B/2 exactly (a power-of-two scaling)
                        const T B = T(0.5) * r.B;
                        V4 xi = sv[li], xj = sv[j];
                        // m_j B / den and m_i B / den, den = m_i m_j - (m_i + m_j) B,
                        // multiplied through by w_j = 1 / m_j (the record's fourth
                        // entry): one division per pair
                        const T wj = xj.w;
                        const T q = B / (mi - (mi * wj + T(1)) * B);
                        const T qj = mi * wj * q;
                        T pi_[3] = {xi.x, xi.y, xi.z}, pj_[3] = {xj.x, xj.y, xj.z};
#pragma unroll
                        for (int d = 0; d < D; ++d) {
                            const T vij = pi_[d] - pj_[d];
                            pi_[d] += q * vij;
                            pj_[d] -= qj * vij;
                        }
                        sv[li] = V4{pi_[0], pi_[1], pi_[2], xi.w};
                        sv[j] = V4{pj_[0], pj_[1], pj_[2], xj.w};
                    }
                }
            }
        }
        __syncwarp(gmask);
    }
    }  // dir
}

// Sweep the staged cell: copy the footprint's velocity records from L2 into
// shared memory, then apply the local operators of its particles in order
// (mode 0), in reverse order (mode 1) or in order and then in reverse order
// (mode 2: the last colour's forward and backward phases, fused since its
// cells' footprints are disjoint), then write the footprint back through L2.
// The copies and the write-back use the group's L lanes, the chain CL of
// them (CL < L only for a group that is a whole warp: lanes 0..CL-1).
template <typename T, int D, int L, int CL = L>
__device__ inline void run_cell(const SweepArgs<T>& a, const CellStage& st, int mode,
                                const CellSmem<T, D>& s, int gl, unsigned gmask)
{
    static_assert(CL == L || L == 32, "a shorter chain needs a whole-warp group");
    using V4 = vec4_t<T>;
    const int p0 = st.p0;
    const int Ftot = st.fr.total;
    V4* sv = s.sv;
    // entry k of the cell's rows at rec[k - p0]: staged in shared memory, or
    // (cells whose rows do not fit) read through the caches
    const SweepSlot<T>* rec =
        a.rows_global ? a.rec + p0 : s.srec + (p0 & (16 / (int)sizeof(SweepSlot<T>) - 1));
    const int* sfoot = s.sfoot;
    if (a.foot_tab) cp_async_wait_all();  // the touched list arrives by cp.async
    __syncwarp(gmask);  // the footprint table written by other lanes of the group

    // velocity records from L2 straight into shared memory
    for (int q = gl; q < Ftot; q += L) {
        const T* src = a.v + (size_t)sfoot[q] * 4;
        if constexpr (sizeof(T) == 4) {
            cp_async16s(sv + q, src);
        } else {
            cp_async16s(reinterpret_cast<double2*>(sv + q), src);
            cp_async16s(reinterpret_cast<double2*>(sv + q) + 1, src + 2);
        }
    }
    if (gl == 0) sv[a.max_foot] = V4{T(0), T(0), T(0), T(0)};
    cp_async_wait_all();
    __syncwarp(gmask);
    // the chain on CL lanes: all L lanes of the group (one shuffle level per
    // halving of the lanes fewer with CL < L; the sums follow the same 32-lane
    // order either way), the others wait for it before the write-back
    if constexpr (CL == L)
        chain_cell<T, D, L>(a, st, mode, s, rec, gl, gmask);
    else if (gl < CL)
        chain_cell<T, D, CL>(a, st, mode, s, rec, gl, (1u << CL) - 1u);
    __syncwarp(gmask);
    // write the footprint back (through L2: other SMs read it after the barrier)
    for (int q = gl; q < Ftot; q += L) stcg_v4<T>(a.v, sfoot[q], sv[q]);
    __syncwarp(gmask);
}

// Colour of phase ph (forward colours 0..nc-1, then backward nc-1..0).
__device__ inline int phase_colour(int ph, int ncolours) { return ph >= ncolours ? 2 * ncolours - 1 - ph : ph; }

// The last colour with cells: its backward phase is fused into its forward
// phase (mode 2 of run_cell) and skipped.
__device__ inline int last_colour(const int* __restrict__ colour_ptr, int ncolours)
{
    int c = -1;
    for (int k = 0; k < ncolours; ++k)
        if (__ldg(colour_ptr + k + 1) > __ldg(colour_ptr + k)) c = k;
    return c;
}

// The first item of group q0 at or after phase ph (its first cell of that
// phase), or -1 when there is none; the fused backward phase of colour
// clast is skipped.
__device__ inline int first_item(const int* __restrict__ colour_ptr, int ncolours, int clast, int ph, int q0)
{
    for (int p = ph; p < 2 * ncolours; ++p) {
        const int c = phase_colour(p, ncolours);
        if (p >= ncolours && c == clast) continue;
        const int c0 = __ldg(colour_ptr + c), c1 = __ldg(colour_ptr + c + 1);
        if (c0 + q0 < c1) return c0 + q0;
    }
    return -1;
}

// The item a group takes after item cid of phase ph: the next of the same
// phase (stride qs), else its first of a later phase.
__device__ inline int next_item(const int* __restrict__ colour_ptr, int ncolours, int clast, int ph, int cid,
                                int q0, int qs)
{
    const int col = phase_colour(ph, ncolours);
    if (cid + qs < __ldg(colour_ptr + col + 1)) return cid + qs;
    return first_item(colour_ptr, ncolours, clast, ph + 1, q0);
}

// The whole S_d of one damped step in one cooperative launch: colours
// 0..3^d-1 forward, then 3^d-1..0 backward, a bounded grid barrier between
// colour phases; the last colour runs both directions in one phase.  Blocks
// of W warps, G cell groups per warp; group number
// q = (block * W + warp) * G + g takes the colour's cells q, q + gridDim*W*G, ...
// More warps per block means fewer blocks arriving at the grid barrier.
template <typename T, int D, int G, int W>
__global__ void __launch_bounds__(32 * W) k_sweep_all(SweepArgs<T> a, const int* __restrict__ colour_ptr,
                                                      int ncolours, unsigned* bar)
{
    constexpr int L = 32 / G;
    if (*(volatile int*)&a.sc->done) return;
    if (a.dflag && *a.dflag == 0) return;  // every block reads the same word: no barrier is left waiting
    if (*(volatile int*)&a.sc->status == DEV_TIMEOUT) return;  // barrier left mid-sweep: host resets it
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int wb = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g = lane / L, gl = lane % L;
    const unsigned gmask = (L == 32) ? 0xffffffffu : (((1u << L) - 1u) << (g * L));
    const size_t cell_bytes = cell_smem_bytes<T, D>(a.max_foot, a.max_pairs, a.max_cell);
    const CellSmem<T, D> s = cell_smem<T, D>(smem_raw + (size_t)(wb * G + g) * cell_bytes, a.max_foot,
                                             a.max_pairs, a.max_cell);
    const int q0 = (blockIdx.x * W + wb) * G + g, qs = gridDim.x * W * G;
    __shared__ unsigned s_gen;
    __shared__ int s_ok;
    const int clast = last_colour(colour_ptr, ncolours);
    // the group's first cell, staged before the first phase
    int staged = first_item(colour_ptr, ncolours, clast, 0, q0);
    CellStage st{};
    if (staged >= 0) st = stage_cell<T, D, L>(a, __ldg(a.colour_cells + staged), s, gl, gmask);
    int phases = 0;
    bool restage = false;  // staging of the next item waits for the barrier's arrive
    for (int ph = 0; ph < 2 * ncolours; ++ph) {
        const int backward = ph >= ncolours;
        const int col = backward ? 2 * ncolours - 1 - ph : ph;
        const int c0 = __ldg(colour_ptr + col), c1 = __ldg(colour_ptr + col + 1);
        if (c1 == c0 || (backward && col == clast)) continue;
        const int mode = col == clast ? 2 : backward;
        if (phases++ > 0) {
            // arrive, stage the next cell while the other blocks finish, wait
            __syncthreads();
            if (threadIdx.x == 0) s_gen = bar_arrive(bar, gridDim.x);
            if (restage && staged >= 0)
                st = stage_cell<T, D, L>(a, __ldg(a.colour_cells + staged), s, gl, gmask);
            restage = false;
            if (threadIdx.x == 0) s_ok = bar_wait(bar, s_gen, a.sc) ? 1 : 0;
            __syncthreads();
            if (!s_ok) {
                cp_async_wait_all();  // no copy may land after the block has left
                return;
            }
        }
        for (int cid = c0 + q0; cid < c1; cid += qs) {
            // staged == cid here: items are visited in the order next_item gives
            run_cell<T, D, L>(a, st, mode, s, gl, gmask);
            staged = next_item(colour_ptr, ncolours, clast, ph, cid, q0, qs);
            if (staged >= 0 && staged < c1 && staged >= c0)
                st = stage_cell<T, D, L>(a, __ldg(a.colour_cells + staged), s, gl, gmask);
            else
                restage = true;  // a later phase: staged between arrive and wait
        }
        __syncwarp();
    }
    cp_async_wait_all();
}

// ---------------------------------------------------------------- cell-wise synchronisation
// The same S_d without grid barriers.  The canonical order only constrains
// cells whose footprints overlap, i.e. cells within 2 cells of each other on
// every axis (5^d - 1 of them; same-colour cells are 3 apart, so none of them
// shares a colour with the cell).  Each cell counts the sweep directions it
// has finished; before its phase ph a cell waits until every non-empty cell
// of its 5^d neighbourhood has finished all of its own phases that precede ph,
// and its later phases wait in turn for this one.  Every pair of overlapping
// cells is therefore ordered as in the canonical order, so the result is
// bitwise that of k_sweep_all; regions of the body that are ready run ahead
// instead of waiting for the slowest cell of the grid at every phase.
// Groups take their cells in phase order and all of them are co-resident
// (cooperative launch), so the lowest unfinished phase always progresses.
//
// flow buffer (unsigned, zeroed at creation): done[c] for every cell of the
// grid (sweep directions finished, counted over all sweeps: the fused phase
// of the last colour counts both), then at word fo = ncells rounded up to 32
// the epoch (sweeps finished), and at fo + 32 a count of finishers of this
// sweep, the last of which advances the epoch (the groups of a single-body
// sweep; the cells of the body in a batched sweep).  After e sweeps
// done[c] = 2 e for every cell, whichever colour a launch fuses.

// directions of a cell of colour cy finished before phase ph (the colour
// clast runs both in its forward phase)
__device__ inline unsigned phases_before(int cy, int ph, int ncolours, int clast)
{
    if (cy == clast) return cy < ph ? 2u : 0u;
    return (cy < ph ? 1u : 0u) + (2 * ncolours - 1 - cy < ph ? 1u : 0u);
}

// Wait until the neighbourhood of cell c is ready for its phase ph.  Each
// lane polls its share of the neighbour cells; a poll gives up after one
// second (DEV_TIMEOUT) or when another group has already given up.
template <typename T, int L>
__device__ inline bool flow_wait(const SweepArgs<T>& a, const unsigned* done, unsigned epoch, int c, int ph,
                                 int ncolours, int clast, DevScalars* status, int gl, unsigned gmask)
{
    const int nx = a.nx, ny = a.ny, nz = a.nz;
    const int cx = c % nx, cy = (c / nx) % ny, cz = c / (nx * ny);
    // cells within wrad on every axis: 2 for cells of edge r_c (3^d
    // footprints overlap up to 2 cells apart), 1 for cells of edge 2 r_c
    // (what they touch lies within r_c of them)
    const int wr = a.wrad, ww = 2 * wr + 1, q = a.cbase;
    const int nb = a.dim == 3 ? ww * ww * ww : ww * ww;
    bool ok = true;
    for (int o = gl; o < nb && ok; o += L) {
        const int dx = o % ww - wr, dy = (o / ww) % ww - wr, dz = a.dim == 3 ? o / (ww * ww) - wr : 0;
        const int x = cx + dx, y = cy + dy, z = cz + dz;
        if ((dx | dy | dz) == 0 || x < 0 || x >= nx || y < 0 || y >= ny || z < 0 || z >= nz) continue;
        const int d = x + nx * (y + ny * z);
        if (__ldg(a.cell_start + d + 1) == __ldg(a.cell_start + d)) continue;  // empty: never runs
        const int col = x % q + q * (y % q) + q * q * (z % q);
        const unsigned need = 2u * epoch + phases_before(col, ph, ncolours, clast);
        long long polls = 0;
        unsigned long long t0 = 0;
        while (*(volatile const unsigned*)(done + d) < need) {
            if (polls == 0) t0 = global_ns();
            if ((++polls & 63) == 0) {
                if (*(volatile int*)&status->status != DEV_OK) {
                    ok = false;
                    break;
                }
                if (global_ns() - t0 > kWaitNs || polls > kWaitPolls) {
                    atomicCAS(&status->status, DEV_OK, DEV_TIMEOUT);
                    ok = false;
                    break;
                }
            }
            __nanosleep(64);
        }
    }
    __threadfence();  // the neighbours' velocity writes before this group's reads
    return __all_sync(gmask, ok);
}

// H: one cell per warp whose chain runs on 16 lanes (G = 1), the whole warp
// waiting, copying and writing back
template <typename T, int D, int G, int W, int H = 0>
__global__ void __launch_bounds__(32 * W) k_sweep_flow(SweepArgs<T> a, const int* __restrict__ colour_ptr,
                                                       int ncolours, unsigned* flow)
{
    static_assert(H == 0 || G == 1, "the 16-lane chain takes one cell per warp");
    constexpr int L = 32 / G;
    constexpr int CL = H ? 16 : L;
    if (*(volatile int*)&a.sc->done) return;
    if (a.dflag && *a.dflag == 0) return;
    if (*(volatile int*)&a.sc->status == DEV_TIMEOUT) return;  // counts left inconsistent: host resets them
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int wb = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g = lane / L, gl = lane % L;
    const unsigned gmask = (L == 32) ? 0xffffffffu : (((1u << L) - 1u) << (g * L));
    const size_t cell_bytes = cell_smem_bytes<T, D>(a.max_foot, a.max_pairs, a.max_cell);
    const CellSmem<T, D> s = cell_smem<T, D>(smem_raw + (size_t)(wb * G + g) * cell_bytes, a.max_foot,
                                             a.max_pairs, a.max_cell);
    const int q0 = (blockIdx.x * W + wb) * G + g, qs = gridDim.x * W * G;
    const int fo = flow_epoch_word(a.nx * a.ny * a.nz);
    unsigned* done = flow;
    const unsigned epoch = *(volatile const unsigned*)(flow + fo);
    const int clast = last_colour(colour_ptr, ncolours);
    int staged = first_item(colour_ptr, ncolours, clast, 0, q0);
    CellStage st{};
    if (staged >= 0) st = stage_cell<T, D, L>(a, __ldg(a.colour_cells + staged), s, gl, gmask);
    bool ok = true;
    for (int ph = 0; ph < 2 * ncolours && ok; ++ph) {
        const int backward = ph >= ncolours;
        const int col = backward ? 2 * ncolours - 1 - ph : ph;
        const int c0 = __ldg(colour_ptr + col), c1 = __ldg(colour_ptr + col + 1);
        if (c1 == c0 || (backward && col == clast)) continue;
        const int mode = col == clast ? 2 : backward;
        for (int cid = c0 + q0; cid < c1; cid += qs) {
            // staged == cid here: items are visited in the order next_item gives
            const int cell = __ldg(a.colour_cells + cid);
            if (!flow_wait<T, L>(a, done, epoch, cell, ph, ncolours, clast, a.sc, gl, gmask)) {
                ok = false;
                break;
            }
            run_cell<T, D, L, CL>(a, st, mode, s, gl, gmask);
            if (gl == 0) {
                __threadfence();  // the group's write-back (ordered by run_cell's __syncwarp) first
                atomicAdd(done + cell, mode == 2 ? 2u : 1u);
            }
            staged = next_item(colour_ptr, ncolours, clast, ph, cid, q0, qs);
            if (staged >= 0) st = stage_cell<T, D, L>(a, __ldg(a.colour_cells + staged), s, gl, gmask);
        }
    }
    cp_async_wait_all();  // no copy may land after the group has left
    if (!ok) return;
    if (gl == 0) {
        const unsigned total = gridDim.x * W * G;
        __threadfence();
        if (atomicAdd(flow + fo + 32, 1u) == total - 1) {
            atomicExch(flow + fo + 32, 0u);
            __threadfence();
            atomicAdd(flow + fo, 1u);
        }
    }
}
