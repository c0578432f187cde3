#include "pairg.cuh"

// Loads of the neighbour streams (read once per pass): not allocated in L1,
// which then holds the neighbours' gathered records (measured 6 % faster
// passes on GB300)
__device__ inline int ld_stream(const int* p)
{
    int r;
    asm volatile("ld.global.nc.L1::no_allocate.b32 %0, [%1];" : "=r"(r) : "l"(p));
    return r;
}
__device__ inline float ld_stream(const float* p)
{
    float r;
    asm volatile("ld.global.nc.L1::no_allocate.f32 %0, [%1];" : "=f"(r) : "l"(p));
    return r;
}
__device__ inline double ld_stream(const double* p)
{
    double r;
    asm volatile("ld.global.nc.L1::no_allocate.f64 %0, [%1];" : "=d"(r) : "l"(p));
    return r;
}
__device__ inline uint16_t ld_stream(const uint16_t* p)
{
    unsigned short r;
    asm volatile("ld.global.nc.L1::no_allocate.u16 %0, [%1];" : "=h"(r) : "l"(p));
    return r;
}

// ------------------------------------------------------------------ layouts
// u at the half step: FP64 [n][4] (x, y, z, 0), or FP32 (hi x, y, z, lo x)
// [n][4] and (lo y, lo z) [n][2], u = hi + lo.
// PB (P B0): the D x D entries of a particle, row-major, in pb_full whole
// 16-byte chunks and pb_tail leftover entries; chunk c of all particles forms
// one dense array (chunk c of particle j at 16-byte index c n + j), each
// leftover entry another.  A neighbour gather then reads one 16-byte vector
// from each of a few dense arrays and one scalar for the leftover, so a
// warp's gathers touch fewer cache lines than with a padded record per
// particle (36 bytes per FP32 3D neighbour instead of 48).
template <typename T, int D>
struct PBL {
    static constexpr int C = pb_full(sizeof(T), D);
    static constexpr int TL = pb_tail(sizeof(T), D);
    static constexpr int E = 16 / (int)sizeof(T);  // entries per chunk
    __device__ static void load(const T* p, int n, int j, T (&m)[D][D])
    {
        T e[C * E + TL];
#pragma unroll
        for (int t = 0; t < TL; ++t) e[C * E + t] = __ldg(p + (size_t)(C * E + t) * n + j);
        if constexpr (sizeof(T) == 4) {
#pragma unroll
            for (int c = 0; c < C; ++c) {
                const float4 x = __ldg(reinterpret_cast<const float4*>(p) + (size_t)c * n + j);
                e[4 * c] = x.x;
                e[4 * c + 1] = x.y;
                e[4 * c + 2] = x.z;
                e[4 * c + 3] = x.w;
            }
        } else {
#pragma unroll
            for (int c = 0; c < C; ++c) {
                const double2 x = __ldg(reinterpret_cast<const double2*>(p) + (size_t)c * n + j);
                e[2 * c] = x.x;
                e[2 * c + 1] = x.y;
            }
        }
#pragma unroll
        for (int r = 0; r < D; ++r)
#pragma unroll
            for (int q = 0; q < D; ++q) m[r][q] = e[r * D + q];
    }
    __device__ static void store(T* p, int n, int j, const T (&m)[D][D])
    {
        T e[C * E + TL];
#pragma unroll
        for (int k = 0; k < C * E + TL; ++k) e[k] = m[k / D][k % D];
#pragma unroll
        for (int t = 0; t < TL; ++t) p[(size_t)(C * E + t) * n + j] = e[C * E + t];
        if constexpr (sizeof(T) == 4) {
#pragma unroll
            for (int c = 0; c < C; ++c)
                reinterpret_cast<float4*>(p)[(size_t)c * n + j] =
                    make_float4(e[4 * c], e[4 * c + 1], e[4 * c + 2], e[4 * c + 3]);
        } else {
#pragma unroll
            for (int c = 0; c < C; ++c)
                reinterpret_cast<double2*>(p)[(size_t)c * n + j] = make_double2(e[2 * c], e[2 * c + 1]);
        }
    }
};

// displacement access
template <typename T>
struct UAcc;
template <>
struct UAcc<double> {
    // FP64: [n][4]
    __device__ static void load(const double* u, const float*, const float*, int j, double (&x)[3],
                                double (&)[3])
    {
        const double2* q = reinterpret_cast<const double2*>(u + (size_t)j * 4);
        double2 a = __ldg(q), b = __ldg(q + 1);
        x[0] = a.x; x[1] = a.y; x[2] = b.x;
    }
    // u_i - u_j
    __device__ static double diff(const double (&xi)[3], const double (&)[3], const double (&xj)[3],
                                  const double (&)[3], int c)
    {
        return xi[c] - xj[c];
    }
};
template <>
struct UAcc<float> {
    // FP32 mixed: (hi x, y, z, lo x) and (lo y, lo z), u = hi + lo
    __device__ static void load(const double*, const float* hi, const float* lo, int j, float (&h)[3],
                                float (&l)[3])
    {
        const float4 a = __ldg(reinterpret_cast<const float4*>(hi) + j);
        const float2 b = __ldg(reinterpret_cast<const float2*>(lo) + j);
        h[0] = a.x; h[1] = a.y; h[2] = a.z;
        l[0] = a.w; l[1] = b.x; l[2] = b.y;
    }
    // (hi_i - hi_j) + (lo_i - lo_j): the hi difference is exact when the two
    // displacements are within a factor of two (Sterbenz), which is exactly
    // the case where a plain FP32 difference would cancel
    __device__ static float diff(const float (&hi)[3], const float (&li)[3], const float (&hj)[3],
                                 const float (&lj)[3], int c)
    {
        return (hi[c] - hj[c]) + (li[c] - lj[c]);
    }
};

// ------------------------------------------------------------------ stress
// Given H = F - I, return P B0 with P = F S (Eq. piola), S from
//   SVK (Eq. constitutive-equation): S = lambda tr(E) I + 2 mu E
//   neo-Hookean (Eqs. strain-density, PK-stress): S = mu (I - C^-1) + lambda ln J C^-1
// evaluated in forms free of cancellation at small strain:
//   E = (H + H^T + H^T H) / 2, mu (I - C^-1) = 2 mu C^-1 E,
//   J - 1 from the invariants of H, ln J = log1p(J - 1).
template <typename T, int D, int MAT>
__device__ inline void stress_PB(const T (&H)[D][D], const T (&B)[D][D], T lambda, T mu,
                                 T (&PB)[D][D])
{
    T E[D][D];
#pragma unroll
    for (int p = 0; p < D; ++p)
#pragma unroll
        for (int q = 0; q < D; ++q) {
            T s = H[p][q] + H[q][p];
#pragma unroll
            for (int r = 0; r < D; ++r) s += H[r][p] * H[r][q];
            E[p][q] = T(0.5) * s;
        }
    T S[D][D];
    if constexpr (MAT == SRDR_LINEAR_SVK) {
        T tr = 0;
#pragma unroll
        for (int p = 0; p < D; ++p) tr += E[p][p];
#pragma unroll
        for (int p = 0; p < D; ++p)
#pragma unroll
            for (int q = 0; q < D; ++q) S[p][q] = T(2) * mu * E[p][q] + (p == q ? lambda * tr : T(0));
    } else {
        // J - 1 = det(I + H) - 1
        T jm1;
        if constexpr (D == 2) {
            jm1 = H[0][0] + H[1][1] + (H[0][0] * H[1][1] - H[0][1] * H[1][0]);
        } else {
            T tr = H[0][0] + H[1][1] + H[2][2];
            T tr2 = 0;
#pragma unroll
            for (int p = 0; p < D; ++p)
#pragma unroll
                for (int q = 0; q < D; ++q) tr2 += H[p][q] * H[q][p];
            T det = H[0][0] * (H[1][1] * H[2][2] - H[1][2] * H[2][1]) -
                    H[0][1] * (H[1][0] * H[2][2] - H[1][2] * H[2][0]) +
                    H[0][2] * (H[1][0] * H[2][1] - H[1][1] * H[2][0]);
            jm1 = tr + T(0.5) * (tr * tr - tr2) + det;
        }
        T lnJ = log1p(jm1);
        T J = T(1) + jm1;
        T invdetC = T(1) / (J * J);  // det C = J^2
        // C = I + 2E, C^-1 = adj(C) / det C
        T C[D][D], Ci[D][D];
#pragma unroll
        for (int p = 0; p < D; ++p)
#pragma unroll
            for (int q = 0; q < D; ++q) C[p][q] = (p == q ? T(1) : T(0)) + T(2) * E[p][q];
        if constexpr (D == 2) {
            Ci[0][0] = C[1][1] * invdetC;
            Ci[0][1] = -C[0][1] * invdetC;
            Ci[1][0] = -C[1][0] * invdetC;
            Ci[1][1] = C[0][0] * invdetC;
        } else {
            constexpr int P = 2;
            Ci[0][0] = (C[1][1] * C[P][P] - C[1][P] * C[P][1]) * invdetC;
            Ci[0][1] = (C[0][P] * C[P][1] - C[0][1] * C[P][P]) * invdetC;
            Ci[0][P] = (C[0][1] * C[1][P] - C[0][P] * C[1][1]) * invdetC;
            Ci[1][0] = (C[1][P] * C[P][0] - C[1][0] * C[P][P]) * invdetC;
            Ci[1][1] = (C[0][0] * C[P][P] - C[0][P] * C[P][0]) * invdetC;
            Ci[1][P] = (C[0][P] * C[1][0] - C[0][0] * C[1][P]) * invdetC;
            Ci[P][0] = (C[1][0] * C[P][1] - C[1][1] * C[P][0]) * invdetC;
            Ci[P][1] = (C[0][1] * C[P][0] - C[0][0] * C[P][1]) * invdetC;
            Ci[P][P] = (C[0][0] * C[1][1] - C[0][1] * C[1][0]) * invdetC;
        }
#pragma unroll
        for (int p = 0; p < D; ++p)
#pragma unroll
            for (int q = 0; q < D; ++q) {
                T ce = 0;
#pragma unroll
                for (int r = 0; r < D; ++r) ce += Ci[p][r] * E[r][q];
                S[p][q] = T(2) * mu * ce + lambda * lnJ * Ci[p][q];
            }
    }
    // P = F S = S + H S;  PB = P B0
    T P[D][D];
#pragma unroll
    for (int p = 0; p < D; ++p)
#pragma unroll
        for (int q = 0; q < D; ++q) {
            T s = S[p][q];
#pragma unroll
            for (int r = 0; r < D; ++r) s += H[p][r] * S[r][q];
            P[p][q] = s;
        }
#pragma unroll
    for (int p = 0; p < D; ++p)
#pragma unroll
        for (int q = 0; q < D; ++q) {
            T s = 0;
#pragma unroll
            for (int r = 0; r < D; ++r) s += P[p][r] * B[r][q];
            PB[p][q] = s;
        }
}

// ------------------------------------------------------------------ pass A
// H_i = -(sum_j u_ij (x) g_ij) B0_i with g_ij = V_j grad0_i W_ij, i.e. the
// corrected displacement gradient at u^{n+1/2}; F = I + H.
//
// The per-neighbour accumulations use explicit roundings (no contraction
// left to the compiler), so the sliced-ELL kernels and the brick-tiled
// kernels, which visit a row's neighbours in the same order, give the same
// bits.
__device__ inline float fma_t(float x, float y, float z) { return __fmaf_rn(x, y, z); }
__device__ inline double fma_t(double x, double y, double z) { return __fma_rn(x, y, z); }
__device__ inline float sub_t(float x, float y) { return __fsub_rn(x, y); }
__device__ inline double sub_t(double x, double y) { return __dsub_rn(x, y); }

// G += (u_i - u_j) (x) g_ij
template <typename T, int D>
__device__ inline void acc_grad(T (&G)[D][D], const T (&xi)[3], const T (&li)[3], const T (&xj)[3],
                                const T (&lj)[3], const T (&g)[D])
{
#pragma unroll
    for (int p = 0; p < D; ++p) {
        const T du = UAcc<T>::diff(xi, li, xj, lj, p);
#pragma unroll
        for (int q = 0; q < D; ++q) G[p][q] = fma_t(du, g[q], G[p][q]);
    }
}

// H = -G B0, stress, P B0 stored
template <typename T, int D, int MAT>
__device__ inline void pass_a_epilogue(const StepArgs<T>& a, int i, const T (&G)[D][D])
{
    const int n = a.n;
    T B[D][D], H[D][D], PB[D][D];
#pragma unroll
    for (int p = 0; p < D; ++p)
#pragma unroll
        for (int q = 0; q < D; ++q) B[p][q] = a.B0[(size_t)(p * D + q) * n + i];
#pragma unroll
    for (int p = 0; p < D; ++p)
#pragma unroll
        for (int q = 0; q < D; ++q) {
            T s2 = 0;
#pragma unroll
            for (int r = 0; r < D; ++r) s2 += G[p][r] * B[r][q];
            H[p][q] = -s2;
        }
    stress_PB<T, D, MAT>(H, B, a.lambda, a.mu, PB);
    PBL<T, D>::store(a.PB, n, i, PB);
}

template <typename T, int D, int MAT>
__device__ inline void pass_a_particle(const StepArgs<T>& a, int i)
{
    int s = i >> 5, lane = i & 31;
    int base = __ldg(a.sell_ptr + s);
    int width = (__ldg(a.sell_ptr + s + 1) - base) >> 5;
    T xi[3], li[3];
    UAcc<T>::load(a.u, a.uhi, a.ulo, i, xi, li);
    T G[D][D];
#pragma unroll
    for (int p = 0; p < D; ++p)
#pragma unroll
        for (int q = 0; q < D; ++q) G[p][q] = 0;
    // slots in batches of kUnroll: all stream loads, then all gathers, then
    // the arithmetic, so each batch costs two memory round trips.  Padding
    // slots point at i itself with g = 0.
    for (int t0 = 0; t0 < width; t0 += kUnroll) {
        int jj[kUnroll];
        T gg[kUnroll][D];
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
            const int k = base + (t0 + u) * 32 + lane;
            const bool in = t0 + u < width;
            jj[u] = in ? ld_stream(a.sell_col + k) : i;
            gg[u][0] = in ? ld_stream(a.g0 + k) : T(0);
            gg[u][1] = in ? ld_stream(a.g1 + k) : T(0);
            if constexpr (D == 3) gg[u][2] = in ? ld_stream(a.g2 + k) : T(0);
        }
        T xj[kUnroll][3], lj[kUnroll][3];
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) UAcc<T>::load(a.u, a.uhi, a.ulo, jj[u], xj[u], lj[u]);
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) acc_grad<T, D>(G, xi, li, xj[u], lj[u], gg[u]);
    }
    pass_a_epilogue<T, D, MAT>(a, i, G);
}

// ------------------------------------------------------------------ lattice stencil
// A body on a box lattice has the same neighbour offsets at every particle
// away from its faces, and the same pair gradient for every pair with the
// same offset (g_ij depends on r0_ij only, Eq. correction-matrix1, with one
// particle volume).  Neighbour k of particle i is then j = i + delta_k when
// the lattice point of j lies in the box; the offsets are ordered by delta,
// i.e. by ascending neighbour index, the order of the neighbour lists, and
// the set-up checks that the stencil reproduces every particle's list.  An
// offset that leaves the box (and the zero padding of the table) takes j = i,
// whose difference terms below are exactly zero.  No neighbour stream is
// read; the 32 threads of a warp are consecutive lattice points, so their
// gathers of one offset are consecutive records.
static_assert(kUnroll == kStencilBatch, "stencil tables are padded to the passes' batch");

template <typename T, int D>
__device__ inline void stencil_slots(const StepArgs<T>& a, int i, int x, int y, int z, int k0,
                                     int (&jj)[kUnroll], T (&gg)[kUnroll][D])
{
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
        const int4 o = __ldg(a.st_off + k0 + u);
        const bool in = (unsigned)(x + o.x) < (unsigned)a.lx && (unsigned)(y + o.y) < (unsigned)a.ly &&
                        (unsigned)(z + o.z) < (unsigned)a.lz;
        jj[u] = in ? i + o.w : i;
        const vec4_t<T> g = load_cpos<T>(a.st_g, k0 + u);
        gg[u][0] = g.x;
        gg[u][1] = g.y;
        if constexpr (D == 3) gg[u][2] = g.z;
    }
}

__device__ inline void lattice_xyz(int i, int lx, int ly, int& x, int& y, int& z)
{
    const int r = i / lx;
    x = i - r * lx;
    z = r / ly;
    y = r - z * ly;
}

template <typename T, int D, int MAT>
__device__ inline void pass_a_particle_st(const StepArgs<T>& a, int i)
{
    int x, y, z;
    lattice_xyz(i, a.lx, a.ly, x, y, z);
    T xi[3], li[3];
    UAcc<T>::load(a.u, a.uhi, a.ulo, i, xi, li);
    T G[D][D];
#pragma unroll
    for (int p = 0; p < D; ++p)
#pragma unroll
        for (int q = 0; q < D; ++q) G[p][q] = 0;
    for (int k0 = 0; k0 < a.st_k; k0 += kUnroll) {
        int jj[kUnroll];
        T gg[kUnroll][D];
        stencil_slots<T, D>(a, i, x, y, z, k0, jj, gg);
        T xj[kUnroll][3], lj[kUnroll][3];
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) UAcc<T>::load(a.u, a.uhi, a.ulo, jj[u], xj[u], lj[u]);
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) acc_grad<T, D>(G, xi, li, xj[u], lj[u], gg[u]);
    }
    pass_a_epilogue<T, D, MAT>(a, i, G);
}

// ST: the lattice stencil instead of the sliced-ELL stream
template <typename T, int D, int MAT, int ST>
__global__ void __launch_bounds__(kThreads) k_pass_a(StepArgs<T> a)
{
    if (a.sc->done) return;
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.n) return;
    if constexpr (ST)
        pass_a_particle_st<T, D, MAT>(a, i);
    else
        pass_a_particle<T, D, MAT>(a, i);
}

// The stress pass with the stencil table as a kernel parameter: K offsets,
// the loop fully unrolled so that every table read is a constant-bank load at
// a fixed offset (the same for the whole warp), leaving the L1 path to the
// neighbour gathers.  Same table values in the same order as the global
// table above, so the same bits.
// CHECK: test each offset against the box; a warp whose lattice points all
// lie at least the table's reach inside the box skips the test (every
// neighbour exists).
template <typename T, int D, int K, bool CHECK>
__device__ inline void stencil_slots_tab(const StencilTab<T, K>& tb, const StepArgs<T>& a, int i, int x, int y,
                                         int z, int k0, int (&jj)[kUnroll], T (&gg)[kUnroll][D])
{
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
        const int k = k0 + u;
        if constexpr (CHECK) {
            const bool in = (unsigned)(x + tb.dx[k]) < (unsigned)a.lx &&
                            (unsigned)(y + tb.dy[k]) < (unsigned)a.ly && (unsigned)(z + tb.dz[k]) < (unsigned)a.lz;
            jj[u] = in ? i + tb.delta[k] : i;
        } else {
            jj[u] = i + tb.delta[k];
        }
        gg[u][0] = tb.g[k][0];
        gg[u][1] = tb.g[k][1];
        if constexpr (D == 3) gg[u][2] = tb.g[k][2];
    }
}

// lattice point (x, y, z) lies at least r points inside the box
template <int D>
__device__ inline bool lattice_inner(int x, int y, int z, int lx, int ly, int lz, int r)
{
    return x >= r && x < lx - r && y >= r && y < ly - r && (D == 2 || (z >= r && z < lz - r));
}

template <typename T, int D, int K, bool CHECK>
__device__ inline void pass_a_sum_tab(const StencilTab<T, K>& tb, const StepArgs<T>& a, int i, int x, int y, int z,
                                      const T (&xi)[3], const T (&li)[3], T (&G)[D][D])
{
#pragma unroll
    for (int k0 = 0; k0 < K; k0 += kUnroll) {
        int jj[kUnroll];
        T gg[kUnroll][D];
        stencil_slots_tab<T, D, K, CHECK>(tb, a, i, x, y, z, k0, jj, gg);
        T xj[kUnroll][3], lj[kUnroll][3];
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) UAcc<T>::load(a.u, a.uhi, a.ulo, jj[u], xj[u], lj[u]);
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) acc_grad<T, D>(G, xi, li, xj[u], lj[u], gg[u]);
    }
}

template <typename T, int D, int MAT, int K>
__global__ void __launch_bounds__(kThreads) k_pass_a_tab(StepArgs<T> a, const __grid_constant__ StencilTab<T, K> tb)
{
    static_assert(K % kUnroll == 0, "stencil tables are padded to the passes' batch");
    if (a.sc->done) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    int x, y, z;
    lattice_xyz(i, a.lx, a.ly, x, y, z);
    // one choice per warp (every lane votes before any leaves)
    const bool inner = __all_sync(0xffffffffu, i < a.n && lattice_inner<D>(x, y, z, a.lx, a.ly, a.lz, tb.reach));
    if (i >= a.n) return;
    T xi[3], li[3];
    UAcc<T>::load(a.u, a.uhi, a.ulo, i, xi, li);
    T G[D][D];
#pragma unroll
    for (int p = 0; p < D; ++p)
#pragma unroll
        for (int q = 0; q < D; ++q) G[p][q] = 0;
    if (inner)
        pass_a_sum_tab<T, D, K, false>(tb, a, i, x, y, z, xi, li, G);
    else
        pass_a_sum_tab<T, D, K, true>(tb, a, i, x, y, z, xi, li, G);
    pass_a_epilogue<T, D, MAT>(a, i, G);
}

// ------------------------------------------------------------------ reductions
__device__ inline double warp_sum(double x)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    return x;
}

// Kinetic-energy partials: one per 32-particle slice, summed in a fixed
// order by its warp (every lane of the warp must call this).  A body's KE is
// then the same whether it is stepped alone or inside a batch.
__device__ inline void slice_partial_store(double x, double* out, int i, int n)
{
    x = warp_sum(x);
    const int slice = i >> 5;
    if ((threadIdx.x & 31) == 0 && (slice << 5) < n) out[slice] = x;
}

// threads of the one-block kinetic-energy reductions (single body and batch
// use the same count, so a body's KE has the same bits in both); the block
// also updates the running maximum, the step counters and the relax test
constexpr int kKeThreads = 256;

// The body's FP64 kinetic energy in one fixed order, whichever kernels
// produced its parts.  The slice partials (32 particles each) form groups of
// kKeGroup consecutive slices, each summed in slice order; thread t of the
// kKeThreads adds groups t, t + B, ... in order; a warp butterfly and
// thread 0's sum of the warp totals finish it.  group(k) returns group k.
constexpr int kKeGroup = 8;
template <typename G>
__device__ inline void ke_reduce(G group, int ng, DevScalars* sc, int damped)
{
    __shared__ double s[kKeThreads / 32];
    double x = 0.0;
    for (int k0 = threadIdx.x; k0 < ng; k0 += 8 * blockDim.x) {
        double g[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int k = k0 + u * blockDim.x;
            g[u] = k < ng ? group(k) : 0.0;
        }
#pragma unroll
        for (int u = 0; u < 8; ++u)
            if (k0 + u * (int)blockDim.x < ng) x += g[u];
    }
    x = warp_sum(x);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) s[w] = x;
    __syncthreads();
    if (threadIdx.x == 0) {
        double ke = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) ke += s[k];
        sc->ke = ke;
        if (ke > sc->ke_max) sc->ke_max = ke;
        sc->step += 1;
        sc->damped += damped;
        if (!isfinite(ke)) {
            sc->status = DEV_NONFINITE;
            sc->done = 1;
        } else if (sc->tol > 0.0 && ke < sc->tol * sc->ke_max) {
            sc->done = 1;
        }
    }
}

// from the np slice partials (groups summed here)
__device__ inline void ke_finalize(const double* __restrict__ part, int np, DevScalars* sc, int damped)
{
    ke_reduce(
        [&](int k) {
            double v[kKeGroup];
#pragma unroll
            for (int u = 0; u < kKeGroup; ++u) v[u] = k * kKeGroup + u < np ? __ldcg(part + k * kKeGroup + u) : 0.0;
            double g = 0.0;
#pragma unroll
            for (int u = 0; u < kKeGroup; ++u)
                if (k * kKeGroup + u < np) g += v[u];
            return g;
        },
        (np + kKeGroup - 1) / kKeGroup, sc, damped);
}

// from group sums already formed (through L2: other blocks wrote them)
__device__ inline void ke_finalize_groups(const double* __restrict__ gpart, int ng, DevScalars* sc,
                                          int damped)
{
    ke_reduce([&](int k) { return __ldcg(gpart + k); }, ng, sc, damped);
}

// A block of kThreads = kKeGroup warps (the slices kKeGroup b ... of block
// b): its group sum, the warp sums (slice partials) added in slice order.
__device__ inline void group_partial_store(double x, double* gpart, int n)
{
    __shared__ double s[kKeGroup];
    x = warp_sum(x);
    if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = x;
    __syncthreads();
    if (threadIdx.x == 0) {
        const int np = (n + 31) >> 5;
        double g = 0.0;
        for (int u = 0; u < kKeGroup; ++u)
            if ((int)blockIdx.x * kKeGroup + u < np) g += s[u];
        gpart[blockIdx.x] = g;
    }
}

// The sliced-ELL force pass and the finish pass (blocks of kThreads =
// kKeGroup warps, so block b holds group b): each block stores its group
// sum; the block that finishes last reduces the group sums with the same
// threads and order as ke_finalize, so the KE has the same bits as in a
// batch, without a launch of its own and with a kKeGroup-th of the FP64
// additions left for one SM.  Every block has written its group sum
// (ordered by the block barrier and the fence) before it takes its ticket.
template <typename T>
__device__ inline void ke_last_block(const StepArgs<T>& a, double ke, int damped)
{
    static_assert(kThreads == kKeThreads && kThreads == 32 * kKeGroup,
                  "a block is one KE group and reduces with the KE kernel's threads");
    const int np = (a.n + 31) >> 5;
    double* gpart = a.ke_part + np;  // group sums after the slice partials
    group_partial_store(ke, gpart, a.n);
    __shared__ int s_last;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        s_last = atomicAdd(&a.sc->ke_ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    ke_finalize_groups(gpart, (np + kKeGroup - 1) / kKeGroup, a.sc, damped);
    if (threadIdx.x == 0) a.sc->ke_ticket = 0;
}

// u <- u + d, FP64, or FP32 hi + lo (two-sum with renormalisation,
// both parts stored as floats)
template <typename T>
__device__ inline void u_add(const StepArgs<T>& a, int i, const T (&d)[3]);
template <>
__device__ inline void u_add<double>(const StepArgs<double>& a, int i, const double (&d)[3])
{
    double2* q = reinterpret_cast<double2*>(a.u + (size_t)i * 4);
    double2 x = q[0], y = q[1];
    x.x += d[0];
    x.y += d[1];
    y.x += d[2];
    q[0] = x;
    q[1] = y;
}
__device__ inline void two_sum_add(float& hi, float& lo, float d)
{
    float s = hi + d;
    float bb = s - hi;
    float e = (hi - (s - bb)) + (d - bb);
    float l2 = lo + e;
    float h2 = s + l2;
    lo = l2 - (h2 - s);
    hi = h2;
}
template <>
__device__ inline void u_add<float>(const StepArgs<float>& a, int i, const float (&d)[3])
{
    float4* ph = reinterpret_cast<float4*>(a.uhi) + i;
    float2* pl = reinterpret_cast<float2*>(a.ulo) + i;
    const float4 r = *ph;
    const float2 q = *pl;
    float h[3] = {r.x, r.y, r.z}, l[3] = {r.w, q.x, q.y};
#pragma unroll
    for (int c = 0; c < 3; ++c) two_sum_add(h[c], l[c], d[c]);
    *ph = make_float4(h[0], h[1], h[2], l[0]);
    *pl = make_float2(l[1], l[2]);
}

// ------------------------------------------------------------------ pass B
// dv_i/dt = (1/rho0) sum_j (PB_i + PB_j) g_ij + g, evaluated as
// (1/rho0) [ sum_j (PB_j - PB_i) g_ij + 2 PB_i G_i ] + g with G_i = sum_j g_ij,
// the same sum written without the cancellation of a nearly uniform stress.
// Then v* = v^n + dt dv/dt (constrained: v = 0); on an undamped step also
// u^{n+3/2} = u^{n+1/2} + dt v^{n+1} and the particle's kinetic energy.

// acc += (PB_j - PB_i) g_ij
template <typename T, int D>
__device__ inline void acc_force(T (&acc)[D], const T (&Pi)[D][D], const T (&Pj)[D][D], const T (&g)[D])
{
#pragma unroll
    for (int p = 0; p < D; ++p)
#pragma unroll
        for (int q = 0; q < D; ++q) acc[p] = fma_t(sub_t(Pj[p][q], Pi[p][q]), g[q], acc[p]);
}

// the 2 PB_i G_i term, velocity update and constraints, and on an undamped
// step the displacement update; returns the particle's kinetic energy (0 if
// not final or constrained)
template <typename T, int D>
__device__ inline double pass_b_epilogue(const StepArgs<T>& a, int i, T (&acc)[D], const T (&Pi)[D][D],
                                         int final_step)
{
    const int n = a.n;
    double ke = 0.0;
    T Gi[D];
#pragma unroll
    for (int q = 0; q < D; ++q) Gi[q] = a.Gs[(size_t)q * n + i];
#pragma unroll
    for (int p = 0; p < D; ++p)
#pragma unroll
        for (int q = 0; q < D; ++q) acc[p] += T(2) * Pi[p][q] * Gi[q];
    uint8_t f = a.flags[i];
    vec4_t<T> v4 = ld_v4<T>(a.v, i);
    T vi[3] = {v4.x, v4.y, v4.z};
    if (f & SRDR_FLAG_CONSTRAINED) {
        vi[0] = vi[1] = vi[2] = 0;
    } else {
#pragma unroll
        for (int p = 0; p < D; ++p) {
            T ap = acc[p] * a.inv_rho0 + a.grav[p];
            if (a.bf) ap += a.bf[(size_t)i * 4 + p];
            if (f & SRDR_FLAG_END_LOAD) ap += a.endl[p];
            vi[p] += a.dt * ap;
            if (a.dvisc) vi[p] += a.dvisc[(size_t)i * 4 + p];
        }
    }
    v4.x = vi[0];
    v4.y = vi[1];
    v4.z = vi[2];
    // a damped step of a stencil body: v* goes to the sweep's sorted copy
    if (a.vs && !final_step)
        st_v4<T>(a.vs, __ldg(a.inv + i), v4);
    else
        st_v4<T>(a.v, i, v4);
    if (final_step && !(f & SRDR_FLAG_CONSTRAINED)) {
        T d[3] = {a.dt * vi[0], a.dt * vi[1], a.dt * vi[2]};
        u_add<T>(a, i, d);
        ke = ke_particle<T>(a.mass[i], vi);
    }
    return ke;
}

template <typename T, int D>
__device__ inline double pass_b_particle(const StepArgs<T>& a, int i, int final_step)
{
    int s = i >> 5, lane = i & 31;
    int base = __ldg(a.sell_ptr + s);
    int width = (__ldg(a.sell_ptr + s + 1) - base) >> 5;
    T Pi[D][D];
    PBL<T, D>::load(a.PB, a.n, i, Pi);
    T acc[D];
#pragma unroll
    for (int p = 0; p < D; ++p) acc[p] = 0;
    for (int t0 = 0; t0 < width; t0 += kUnroll) {
        int jj[kUnroll];
        T gg[kUnroll][D];
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
            const int k = base + (t0 + u) * 32 + lane;
            const bool in = t0 + u < width;
            jj[u] = in ? ld_stream(a.sell_col + k) : i;
            gg[u][0] = in ? ld_stream(a.g0 + k) : T(0);
            gg[u][1] = in ? ld_stream(a.g1 + k) : T(0);
            if constexpr (D == 3) gg[u][2] = in ? ld_stream(a.g2 + k) : T(0);
        }
        T Pj[kUnroll][D][D];
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) PBL<T, D>::load(a.PB, a.n, jj[u], Pj[u]);
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) acc_force<T, D>(acc, Pi, Pj[u], gg[u]);
    }
    return pass_b_epilogue<T, D>(a, i, acc, Pi, final_step);
}

template <typename T, int D>
__device__ inline double pass_b_particle_st(const StepArgs<T>& a, int i, int final_step)
{
    int x, y, z;
    lattice_xyz(i, a.lx, a.ly, x, y, z);
    T Pi[D][D];
    PBL<T, D>::load(a.PB, a.n, i, Pi);
    T acc[D];
#pragma unroll
    for (int p = 0; p < D; ++p) acc[p] = 0;
    for (int k0 = 0; k0 < a.st_k; k0 += kUnroll) {
        int jj[kUnroll];
        T gg[kUnroll][D];
        stencil_slots<T, D>(a, i, x, y, z, k0, jj, gg);
        T Pj[kUnroll][D][D];
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) PBL<T, D>::load(a.PB, a.n, jj[u], Pj[u]);
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) acc_force<T, D>(acc, Pi, Pj[u], gg[u]);
    }
    return pass_b_epilogue<T, D>(a, i, acc, Pi, final_step);
}

template <typename T, int D, int K, bool CHECK>
__device__ inline void pass_b_sum_tab(const StencilTab<T, K>& tb, const StepArgs<T>& a, int i, int x, int y, int z,
                                      const T (&Pi)[D][D], T (&acc)[D])
{
#pragma unroll
    for (int k0 = 0; k0 < K; k0 += kUnroll) {
        int jj[kUnroll];
        T gg[kUnroll][D];
        stencil_slots_tab<T, D, K, CHECK>(tb, a, i, x, y, z, k0, jj, gg);
        T Pj[kUnroll][D][D];
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) PBL<T, D>::load(a.PB, a.n, jj[u], Pj[u]);
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) acc_force<T, D>(acc, Pi, Pj[u], gg[u]);
    }
}

// the force pass with the stencil table as a kernel parameter (see
// k_pass_a_tab)
template <typename T, int D, int K>
__global__ void __launch_bounds__(kThreads, 4) k_pass_b_tab(StepArgs<T> a, const __grid_constant__ StencilTab<T, K> tb,
                                                           int final_step)
{
    static_assert(K % kUnroll == 0, "stencil tables are padded to the passes' batch");
    if (a.sc->done) return;
    if (a.dflag) final_step = *a.dflag == 0;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    double ke = 0.0;
    if (i < a.n) {
        // every offset tested against the box: a second, untested copy of
        // the loop (as in the stress pass) spills at this kernel's 80
        // registers and measured slower
        int x, y, z;
        lattice_xyz(i, a.lx, a.ly, x, y, z);
        T Pi[D][D];
        PBL<T, D>::load(a.PB, a.n, i, Pi);
        T acc[D];
#pragma unroll
        for (int p = 0; p < D; ++p) acc[p] = 0;
        pass_b_sum_tab<T, D, K, true>(tb, a, i, x, y, z, Pi, acc);
        ke = pass_b_epilogue<T, D>(a, i, acc, Pi, final_step);
    }
    if (final_step) ke_last_block(a, ke, 0);
}

template <typename T, int D, int ST>
__global__ void __launch_bounds__(kThreads, 3) k_pass_b(StepArgs<T> a, int final_step)
{
    if (a.sc->done) return;
    if (a.dflag) final_step = *a.dflag == 0;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    double ke = 0.0;
    if (i < a.n) {
        if constexpr (ST)
            ke = pass_b_particle_st<T, D>(a, i, final_step);
        else
            ke = pass_b_particle<T, D>(a, i, final_step);
    }
    if (final_step) ke_last_block(a, ke, 0);
}

// after S_d: constraints, u^{n+3/2} = u^{n+1/2} + dt v^{n+1}, KE contribution
template <typename T>
__device__ inline double finish_particle(const StepArgs<T>& a, int i)
{
    const int n = a.n;
    double ke = 0.0;
    {
        uint8_t f = a.flags[i];
        // a stencil body's damped velocities come from the sweep's sorted
        // copy and go back to v
        vec4_t<T> v4 = a.vs ? ld_v4<T>(a.vs, __ldg(a.inv + i)) : ld_v4<T>(a.v, i);
        if (f & SRDR_FLAG_CONSTRAINED) {
            v4.x = v4.y = v4.z = 0;
            st_v4<T>(a.v, i, v4);
        } else {
            if (a.vs) st_v4<T>(a.v, i, v4);
            const T vi[3] = {v4.x, v4.y, v4.z};
            T d[3] = {a.dt * vi[0], a.dt * vi[1], a.dt * vi[2]};
            u_add<T>(a, i, d);
            ke = ke_particle<T>(a.mass[i], vi);
        }
    }
    return ke;
}

template <typename T>
__global__ void __launch_bounds__(kThreads) k_finish(StepArgs<T> a)
{
    if (a.sc->done || (a.dflag && *a.dflag == 0)) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const double ke = i < a.n ? finish_particle<T>(a, i) : 0.0;
    ke_last_block(a, ke, 1);
}

// one block: KE of the body, KE_max, step counters, relax test, after the
// brick-tiled force pass of an undamped step (the sliced-ELL force pass and
// the finish pass reduce the KE in their last block instead)
__global__ void __launch_bounds__(kKeThreads) k_ke_final(const double* __restrict__ part, int np,
                                                        DevScalars* sc, const int* dflag)
{
    if (sc->done || (dflag && *dflag)) return;  // a damped step: k_finish reduced it
    ke_finalize(part, np, sc, 0);
}

// the random choice of the step (Eq. viscosity-reset) on the device, for
// replayed multi-step graphs: the same Philox draw as the host's
__global__ void k_decide_one(const DevScalars* sc, unsigned long long seed, double alpha, int* dflag)
{
    *dflag = !sc->done && random_phi(seed, (unsigned long long)sc->step) < alpha;
}


// ------------------------------------------------------------------ explicit comparator
// dv_i = dt (2 eta / m_i) sum_j V_i V_j (v_i - v_j) / r_ij dW/dr (Eq.
// damping-term at v^n) over the sweep's CSR rows, w_ij = V_i V_j W'(r)/r;
// the force pass adds it to v* (Sec. 3: the explicit scheme the split
// random-choice scheme replaces).  Rows, columns and mass_s are in sorted
// order; v and dv in particle order, reached through pidx when it is set.
template <typename T, int D>
__global__ void __launch_bounds__(kThreads) k_visc(int n, const int* __restrict__ row_ptr,
                                                    const int* __restrict__ col, const T* __restrict__ w,
                                                    const T* __restrict__ v, const T* __restrict__ mass_s,
                                                    const int* __restrict__ pidx, T c2eta_dt,
                                                    T* __restrict__ dv, const DevScalars* sc)
{
    if (sc->done) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int pi = pidx ? __ldg(pidx + i) : i;
    const vec4_t<T> vi4 = ld_v4<T>(v, pi);
    const T vi[3] = {vi4.x, vi4.y, vi4.z};
    T e[3] = {0, 0, 0};
    for (int k = __ldg(row_ptr + i); k < __ldg(row_ptr + i + 1); ++k) {
        const int j = __ldg(col + k);
        const vec4_t<T> vj4 = ld_v4<T>(v, pidx ? __ldg(pidx + j) : j);
        const T vj[3] = {vj4.x, vj4.y, vj4.z};
        const T wk = __ldg(w + k);
#pragma unroll
        for (int d = 0; d < D; ++d) e[d] = fma_t(wk, sub_t(vi[d], vj[d]), e[d]);
    }
    const T s = c2eta_dt / mass_s[i];
#pragma unroll
    for (int d = 0; d < 3; ++d) dv[(size_t)pi * 4 + d] = d < D ? s * e[d] : T(0);
    dv[(size_t)pi * 4 + 3] = T(0);
}

// ------------------------------------------------------------------ host: kernel arguments
template <typename T>
StepArgs<T> make_step_args(srdr_body* b)
{
    StepArgs<T> a{};
    a.n = (int)b->n;
    a.sell_ptr = b->sell_ptr;
    a.sell_col = b->sell_col;
    a.g0 = static_cast<const T*>(b->sell_g);
    a.g1 = a.g0 + b->nslots;
    a.g2 = a.g1 + b->nslots;
    a.cpos = static_cast<const T*>(b->cpos);
    a.ccell = b->ccell;
    a.B0 = static_cast<const T*>(b->B0);
    a.PB = static_cast<T*>(b->PB);
    a.Gs = static_cast<const T*>(b->Gs);
    a.dvisc = static_cast<const T*>(b->dvisc);
    a.bf = static_cast<const T*>(b->bf);
    a.v = static_cast<T*>(b->v);
    a.u = b->u;
    a.uhi = b->uhi;
    a.ulo = b->ulo;
    a.flags = b->flags;
    a.mass = static_cast<const T*>(b->mass);
    a.ke_part = b->ke_part;
    a.sc = b->sc;
    a.lambda = (T)b->lambda;
    a.mu = (T)b->mu;
    a.inv_rho0 = (T)(1.0 / b->desc.rho0);
    a.dt = (T)b->dt;
    a.rc = (T)b->rc;
    a.inv_h = (T)(1.0 / b->h);
    a.kc = (T)kernel_kc(b->dim, b->h);
    for (int p = 0; p < 3; ++p) {
        a.grav[p] = (T)(p < b->dim ? b->desc.gravity[p] : 0.0);
        a.endl[p] = (T)(p < b->dim ? b->desc.end_load[p] : 0.0);
    }
    if (b->stencil) {
        a.st_off = b->st_off;
        a.st_g = static_cast<const T*>(b->st_g);
        a.st_k = b->st_k;
        a.lx = b->lat[0];
        a.ly = b->lat[1];
        a.lz = b->lat[2];
        a.vs = static_cast<T*>(b->vs);
        a.inv = b->inv;
    }
    return a;
}

// the body's stencil as a kernel-parameter table of K offsets (the same
// values, rounded to T once, as its device table)
template <typename T, int K>
StencilTab<T, K> make_stencil_tab(const srdr_body* b)
{
    StencilTab<T, K> t{};
    for (int k = 0; k < K && k < (int)b->st_off_h.size(); ++k) {
        const int4 o = b->st_off_h[k];
        t.reach = std::max(t.reach, std::max(std::abs(o.x), std::max(std::abs(o.y), std::abs(o.z))));
        t.delta[k] = o.w;
        t.dx[k] = o.x;
        t.dy[k] = o.y;
        t.dz[k] = o.z;
        for (int c = 0; c < 3; ++c) t.g[k][c] = (T)b->st_g_h[(size_t)k * 4 + c];
    }
    return t;
}
