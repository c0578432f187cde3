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
constexpr int kUnroll = 4;  // sliced-ELL slots per batch of loads in the passes
inline int nblocks(int64_t n, int t = kThreads) { return (int)((n + t - 1) / t); }

// ------------------------------------------------------------------ layouts
// u at the half step: FP64 [n][4] (x, y, z, 0), or FP32 hi/lo float4 [n] each.
// PB (P B0): AoS, padded to whole 16-byte vectors: stride pb_stride<T, D>.
template <typename T, int D>
struct PBL;
template <>
struct PBL<float, 3> {
    static constexpr int S = 12;
    __device__ static void load(const float* p, int j, float (&m)[3][3])
    {
        const float4* q = reinterpret_cast<const float4*>(p + (size_t)j * S);
        float4 a = __ldg(q), b = __ldg(q + 1), c = __ldg(q + 2);
        m[0][0] = a.x; m[0][1] = a.y; m[0][2] = a.z;
        m[1][0] = a.w; m[1][1] = b.x; m[1][2] = b.y;
        m[2][0] = b.z; m[2][1] = b.w; m[2][2] = c.x;
    }
    __device__ static void store(float* p, int j, const float (&m)[3][3])
    {
        float4* q = reinterpret_cast<float4*>(p + (size_t)j * S);
        q[0] = make_float4(m[0][0], m[0][1], m[0][2], m[1][0]);
        q[1] = make_float4(m[1][1], m[1][2], m[2][0], m[2][1]);
        q[2] = make_float4(m[2][2], 0.f, 0.f, 0.f);
    }
};
template <>
struct PBL<float, 2> {
    static constexpr int S = 4;
    __device__ static void load(const float* p, int j, float (&m)[2][2])
    {
        float4 a = __ldg(reinterpret_cast<const float4*>(p + (size_t)j * S));
        m[0][0] = a.x; m[0][1] = a.y; m[1][0] = a.z; m[1][1] = a.w;
    }
    __device__ static void store(float* p, int j, const float (&m)[2][2])
    {
        *reinterpret_cast<float4*>(p + (size_t)j * S) = make_float4(m[0][0], m[0][1], m[1][0], m[1][1]);
    }
};
template <>
struct PBL<double, 3> {
    static constexpr int S = 10;
    __device__ static void load(const double* p, int j, double (&m)[3][3])
    {
        const double2* q = reinterpret_cast<const double2*>(p + (size_t)j * S);
        double2 a = __ldg(q), b = __ldg(q + 1), c = __ldg(q + 2), d = __ldg(q + 3), e = __ldg(q + 4);
        m[0][0] = a.x; m[0][1] = a.y; m[0][2] = b.x;
        m[1][0] = b.y; m[1][1] = c.x; m[1][2] = c.y;
        m[2][0] = d.x; m[2][1] = d.y; m[2][2] = e.x;
    }
    __device__ static void store(double* p, int j, const double (&m)[3][3])
    {
        double2* q = reinterpret_cast<double2*>(p + (size_t)j * S);
        q[0] = make_double2(m[0][0], m[0][1]);
        q[1] = make_double2(m[0][2], m[1][0]);
        q[2] = make_double2(m[1][1], m[1][2]);
        q[3] = make_double2(m[2][0], m[2][1]);
        q[4] = make_double2(m[2][2], 0.0);
    }
};
template <>
struct PBL<double, 2> {
    static constexpr int S = 4;
    __device__ static void load(const double* p, int j, double (&m)[2][2])
    {
        const double2* q = reinterpret_cast<const double2*>(p + (size_t)j * S);
        double2 a = __ldg(q), b = __ldg(q + 1);
        m[0][0] = a.x; m[0][1] = a.y; m[1][0] = b.x; m[1][1] = b.y;
    }
    __device__ static void store(double* p, int j, const double (&m)[2][2])
    {
        double2* q = reinterpret_cast<double2*>(p + (size_t)j * S);
        q[0] = make_double2(m[0][0], m[0][1]);
        q[1] = make_double2(m[1][0], m[1][1]);
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
    // FP32 mixed: u = hi + lo, two float4 arrays (about 48 significant bits)
    __device__ static void load(const double*, const float* hi, const float* lo, int j, float (&h)[3],
                                float (&l)[3])
    {
        float4 a = __ldg(reinterpret_cast<const float4*>(hi) + j);
        float4 b = __ldg(reinterpret_cast<const float4*>(lo) + j);
        h[0] = a.x; h[1] = a.y; h[2] = a.z;
        l[0] = b.x; l[1] = b.y; l[2] = b.z;
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
template <typename T, int D, int MAT>
__global__ void __launch_bounds__(kThreads) k_pass_a(StepArgs<T> a)
{
    if (a.sc->done) return;
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.n) return;
    const int n = a.n;
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
    // the arithmetic, so each batch costs two memory round trips
    for (int t0 = 0; t0 < width; t0 += kUnroll) {
        int jj[kUnroll];
        T gg[kUnroll][D];
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
            const int k = base + (t0 + u) * 32 + lane;
            const bool in = t0 + u < width;
            jj[u] = in ? __ldg(a.sell_col + k) : i;
            gg[u][0] = in ? __ldg(a.g0 + k) : T(0);
            gg[u][1] = in ? __ldg(a.g1 + k) : T(0);
            if constexpr (D == 3) gg[u][2] = in ? __ldg(a.g2 + k) : T(0);
        }
        T xj[kUnroll][3], lj[kUnroll][3];
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) UAcc<T>::load(a.u, a.uhi, a.ulo, jj[u], xj[u], lj[u]);
#pragma unroll
        for (int u = 0; u < kUnroll; ++u)
#pragma unroll
            for (int p = 0; p < D; ++p) {
                T du = UAcc<T>::diff(xi, li, xj[u], lj[u], p);
#pragma unroll
                for (int q = 0; q < D; ++q) G[p][q] += du * gg[u][q];
            }
    }
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
    PBL<T, D>::store(a.PB, i, PB);
}

// ------------------------------------------------------------------ reductions
__device__ inline double warp_sum(double x)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    return x;
}

// fixed-order block sum of one double per thread into out[blockIdx.x]
__device__ inline void block_sum_store(double x, double* out)
{
    __shared__ double s[kThreads / 32];
    x = warp_sum(x);
    int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) s[w] = x;
    __syncthreads();
    if (w == 0) {
        double y = l < (int)(blockDim.x >> 5) ? s[l] : 0.0;
        y = warp_sum(y);
        if (l == 0) out[blockIdx.x] = y;
    }
}

// u <- u + d, FP64 or FP32 hi/lo (two-sum with renormalisation)
template <typename T>
__device__ inline void u_add(StepArgs<T>& a, int i, const T (&d)[3]);
template <>
__device__ inline void u_add<double>(StepArgs<double>& a, int i, const double (&d)[3])
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
__device__ inline void u_add<float>(StepArgs<float>& a, int i, const float (&d)[3])
{
    float4* ph = reinterpret_cast<float4*>(a.uhi) + i;
    float4* pl = reinterpret_cast<float4*>(a.ulo) + i;
    float4 h = *ph, l = *pl;
    two_sum_add(h.x, l.x, d[0]);
    two_sum_add(h.y, l.y, d[1]);
    two_sum_add(h.z, l.z, d[2]);
    *ph = h;
    *pl = l;
}

// ------------------------------------------------------------------ pass B
// dv_i/dt = (1/rho0) sum_j (PB_i + PB_j) g_ij + g, evaluated as
// (1/rho0) [ sum_j (PB_j - PB_i) g_ij + 2 PB_i G_i ] + g with G_i = sum_j g_ij,
// the same sum written without the cancellation of a nearly uniform stress.
// Then v* = v^n + dt dv/dt (constrained: v = 0); on an undamped step also
// u^{n+3/2} = u^{n+1/2} + dt v^{n+1} and the KE partials.
template <typename T, int D>
__global__ void __launch_bounds__(kThreads) k_pass_b(StepArgs<T> a, int final_step)
{
    if (a.sc->done) return;
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int n = a.n;
    double ke = 0.0;
    if (i < n) {
        int s = i >> 5, lane = i & 31;
        int base = __ldg(a.sell_ptr + s);
        int width = (__ldg(a.sell_ptr + s + 1) - base) >> 5;
        T Pi[D][D];
        PBL<T, D>::load(a.PB, i, Pi);
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
                jj[u] = in ? __ldg(a.sell_col + k) : i;
                gg[u][0] = in ? __ldg(a.g0 + k) : T(0);
                gg[u][1] = in ? __ldg(a.g1 + k) : T(0);
                if constexpr (D == 3) gg[u][2] = in ? __ldg(a.g2 + k) : T(0);
            }
            T Pj[kUnroll][D][D];
#pragma unroll
            for (int u = 0; u < kUnroll; ++u) PBL<T, D>::load(a.PB, jj[u], Pj[u]);
#pragma unroll
            for (int u = 0; u < kUnroll; ++u)
#pragma unroll
                for (int p = 0; p < D; ++p)
#pragma unroll
                    for (int q = 0; q < D; ++q) acc[p] += (Pj[u][p][q] - Pi[p][q]) * gg[u][q];
        }
        T Gi[D];
#pragma unroll
        for (int q = 0; q < D; ++q) Gi[q] = a.Gs[(size_t)q * n + i];
#pragma unroll
        for (int p = 0; p < D; ++p)
#pragma unroll
            for (int q = 0; q < D; ++q) acc[p] += T(2) * Pi[p][q] * Gi[q];
        uint8_t f = a.flags[i];
        T vi[3];
#pragma unroll
        for (int p = 0; p < 3; ++p) vi[p] = a.v[(size_t)p * n + i];
        if (f & SRDR_FLAG_CONSTRAINED) {
            vi[0] = vi[1] = vi[2] = 0;
        } else {
#pragma unroll
            for (int p = 0; p < D; ++p) {
                T ap = acc[p] * a.inv_rho0 + a.grav[p];
                if (f & SRDR_FLAG_END_LOAD) ap += a.endl[p];
                vi[p] += a.dt * ap;
            }
        }
#pragma unroll
        for (int p = 0; p < 3; ++p) a.v[(size_t)p * n + i] = vi[p];
        if (final_step && !(f & SRDR_FLAG_CONSTRAINED)) {
            T d[3] = {a.dt * vi[0], a.dt * vi[1], a.dt * vi[2]};
            u_add<T>(a, i, d);
            T m = a.mass[i];
            ke = (double)(T(0.5) * m * (vi[0] * vi[0] + vi[1] * vi[1] + vi[2] * vi[2]));
        }
    }
    if (final_step) block_sum_store(ke, a.ke_part);
}

// after S_d: constraints, u^{n+3/2} = u^{n+1/2} + dt v^{n+1}, KE partials
template <typename T>
__global__ void __launch_bounds__(kThreads) k_finish(StepArgs<T> a)
{
    if (a.sc->done) return;
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int n = a.n;
    double ke = 0.0;
    if (i < n) {
        uint8_t f = a.flags[i];
        if (f & SRDR_FLAG_CONSTRAINED) {
#pragma unroll
            for (int p = 0; p < 3; ++p) a.v[(size_t)p * n + i] = 0;
        } else {
            T vi[3];
#pragma unroll
            for (int p = 0; p < 3; ++p) vi[p] = a.v[(size_t)p * n + i];
            T d[3] = {a.dt * vi[0], a.dt * vi[1], a.dt * vi[2]};
            u_add<T>(a, i, d);
            T m = a.mass[i];
            ke = (double)(T(0.5) * m * (vi[0] * vi[0] + vi[1] * vi[1] + vi[2] * vi[2]));
        }
    }
    block_sum_store(ke, a.ke_part);
}

// one block: KE in a fixed order, KE_max, step counters, relax test
__global__ void __launch_bounds__(kThreads) k_ke_final(const double* __restrict__ part, int nb,
                                                        DevScalars* sc, int damped)
{
    if (sc->done) return;
    double x = 0.0;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) x += part[b];
    __shared__ double s[kThreads / 32];
    x = warp_sum(x);
    int w = threadIdx.x >> 5, l = threadIdx.x & 31;
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

// ------------------------------------------------------------------ damping sweep
template <typename T>
__device__ inline T warp_allsum(T x)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

// The <= 9 runs of a cell's footprint, known to every lane of the warp:
// run r covers sorted particles [a[r], a[r] + off[r+1] - off[r]) and sits at
// footprint-local offset off[r].
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

__device__ inline FootRuns foot_runs_warp(int c, int dim, int nx, int ny, int nz,
                                          const int* __restrict__ start, int lane)
{
    const int cx = c % nx, cy = (c / nx) % ny, cz = c / (nx * ny);
    const int xlo = max(cx - 1, 0), xhi = min(cx + 1, nx - 1);
    const int ylo = dim >= 2 ? max(cy - 1, 0) : 0, yhi = dim >= 2 ? min(cy + 1, ny - 1) : 0;
    const int zlo = dim >= 3 ? max(cz - 1, 0) : 0, zhi = dim >= 3 ? min(cz + 1, nz - 1) : 0;
    const int ny_r = yhi - ylo + 1;
    FootRuns f;
    f.nruns = ny_r * (zhi - zlo + 1);
    int ra = 0, len = 0;
    if (lane < f.nruns) {
        const int y = ylo + lane % ny_r, z = zlo + lane / ny_r;
        const int c0 = xlo + nx * (y + ny * z), c1 = xhi + nx * (y + ny * z);
        ra = __ldg(start + c0);
        len = __ldg(start + c1 + 1) - ra;
    }
    int run = 0;
#pragma unroll
    for (int r = 0; r < 9; ++r) {
        f.a[r] = __shfl_sync(0xffffffffu, ra, r);
        const int l = __shfl_sync(0xffffffffu, len, r);
        f.off[r] = run;
        run += r < f.nruns ? l : 0;
    }
    f.off[9] = run;
    f.total = run;
    return f;
}

// Bounded grid barrier of a cooperative launch (all blocks co-resident).  The
// last block to arrive resets the count and bumps the generation; the others
// wait on the generation with a sleep, and give up after `limit` polls,
// setting DEV_TIMEOUT in sc->status so that the host gets an error instead of
// a hung GPU.  One warp per block: lane 0 does the protocol.
__device__ inline bool grid_barrier(unsigned* count, volatile unsigned* gen, unsigned nblocks,
                                    DevScalars* sc)
{
    __syncwarp();
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
    }
    ok = __shfl_sync(0xffffffffu, ok, 0);
    return ok != 0;
}

// Shared-memory layout of one cell (one warp):
//   sv [D][F] footprint velocities, sminv [F] inverse masses,
//   sw [P] weights, sl [P] footprint-local neighbour indices,
//   srow [C+1] row starts (relative), sm/ssb/ssb2 [C] mass, sum B, sum B^2
template <typename T, int D>
struct CellSmem {
    T* sv;
    T* sminv;
    T* sw;
    T* sm;
    T* ssb;
    T* ssb2;
    int* srow;
    uint16_t* sl;
};

template <typename T, int D>
__device__ inline CellSmem<T, D> cell_smem(unsigned char* raw, int F, int P, int C)
{
    CellSmem<T, D> s;
    s.sv = reinterpret_cast<T*>(raw);
    s.sminv = s.sv + (size_t)D * F;
    s.sw = s.sminv + F;
    s.sm = s.sw + P;
    s.ssb = s.sm + C;
    s.ssb2 = s.ssb + C;
    s.srow = reinterpret_cast<int*>(s.ssb2 + C);
    s.sl = reinterpret_cast<uint16_t*>(s.srow + C + 1);
    return s;
}

template <typename T, int D>
__device__ inline void sweep_cell(const SweepArgs<T>& a, int c, int backward, const CellSmem<T, D>& s)
{
    const int lane = threadIdx.x;
    const int n = a.n;
    const int cs = __ldg(a.cell_start + c), ce = __ldg(a.cell_start + c + 1);
    const int F = a.max_foot;
    T* sv = s.sv;
    T* sminv = s.sminv;
    T* sw = s.sw;
    uint16_t* sl = s.sl;
    const T cc = a.c;

    // The footprint's runs (same z-outer, y-inner order as the setup's
    // footprint-local indices): lane r < 9 finds run r, then every lane gets
    // all run starts and offsets by shuffles.
    const FootRuns fr = foot_runs_warp(c, a.dim, a.nx, a.ny, a.nz, a.cell_start, lane);
    const int Ftot = fr.total;
    int my_off = 0;
#pragma unroll
    for (int r = 0; r < 9; ++r)
        if (r < fr.nruns && cs >= fr.a[r] && cs < fr.a[r] + (fr.off[r + 1] - fr.off[r]))
            my_off = fr.off[r] + (cs - fr.a[r]);
    const int np = ce - cs;
    const int p0 = __ldg(a.row_ptr + cs), p1 = __ldg(a.row_ptr + ce);

    // Staging in register batches: all loads of a batch are issued before
    // any shared-memory store, so a batch costs one memory round trip.  v is
    // read through L2 (ld.cg): other SMs wrote it in earlier colour phases.
    constexpr int U = 8;
    for (int base = 0; base < Ftot; base += 32 * U) {
        T tv[U][D], tm[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int q = base + u * 32 + lane;
            if (q < Ftot) {
                const int j = fr.particle(q);
#pragma unroll
                for (int d = 0; d < D; ++d) tv[u][d] = __ldcg(a.v + (size_t)d * n + j);
                tm[u] = __ldg(a.minv + j);
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int q = base + u * 32 + lane;
            if (q < Ftot) {
#pragma unroll
                for (int d = 0; d < D; ++d) sv[d * F + q] = tv[u][d];
                sminv[q] = tm[u];
            }
        }
    }
    constexpr int U2 = 16;
    for (int base = p0; base < p1; base += 32 * U2) {
        T tw[U2];
        uint16_t tl[U2];
#pragma unroll
        for (int u = 0; u < U2; ++u) {
            const int k = base + u * 32 + lane;
            if (k < p1) {
                tw[u] = __ldg(a.w + k);
                tl[u] = __ldg(a.loc + k);
            }
        }
#pragma unroll
        for (int u = 0; u < U2; ++u) {
            const int k = base + u * 32 + lane;
            if (k < p1) {
                sw[k - p0] = tw[u];
                sl[k - p0] = tl[u];
            }
        }
    }
    for (int base = 0; base <= np; base += 32) {
        const int p = base + lane;
        int rp = 0;
        T m = 0, s1 = 0, s2 = 0;
        if (p <= np) rp = __ldg(a.row_ptr + cs + p) - p0;
        if (p < np) {
            m = __ldg(a.mass + cs + p);
            s1 = __ldg(a.sumw + cs + p);
            s2 = __ldg(a.sumw2 + cs + p);
        }
        if (p <= np) s.srow[p] = rp;
        if (p < np) {
            s.sm[p] = m;
            s.ssb[p] = cc * s1;
            s.ssb2[p] = cc * cc * s2;
        }
    }
    __syncwarp();

    for (int t = 0; t < np; ++t) {
        const int p = backward ? np - 1 - t : t;
        const int li = my_off + p;
        const int k0 = s.srow[p], k1 = s.srow[p + 1];
        if (!a.pairwise) {
            const T mi = s.sm[p];
            const T SB = s.ssb[p];
            const T SB2 = s.ssb2[p];
            T vi[D], E[D];
#pragma unroll
            for (int d = 0; d < D; ++d) {
                vi[d] = sv[d * F + li];
                E[d] = 0;
            }
            for (int k = k0 + lane; k < k1; k += 32) {
                const int j = sl[k];
                const T B = cc * sw[k];
#pragma unroll
                for (int d = 0; d < D; ++d) E[d] -= B * (vi[d] - sv[d * F + j]);
            }
#pragma unroll
            for (int d = 0; d < D; ++d) E[d] = warp_allsum(E[d]);
            const T sbm = SB - mi;
            const T rden = T(1) / (sbm * sbm + SB2);
            T kk[D], vin[D];
#pragma unroll
            for (int d = 0; d < D; ++d) {
                kk[d] = E[d] * rden;
                vin[d] = vi[d] + sbm * kk[d];
            }
            for (int k = k0 + lane; k < k1; k += 32) {
                const int j = sl[k];
                const T B = cc * sw[k];
                const T im = sminv[j];
#pragma unroll
                for (int d = 0; d < D; ++d) {
                    T vj = sv[d * F + j];
                    sv[d * F + j] = vj - B * (vin[d] - vj + B * kk[d]) * im;
                }
            }
            __syncwarp();
            if (lane == 0) {
#pragma unroll
                for (int d = 0; d < D; ++d) sv[d * F + li] = vin[d];
            }
            __syncwarp();
        } else {
            if (lane == 0) {
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
                            T vij = sv[d * F + li] - sv[d * F + j];
                            sv[d * F + li] += mj * B * vij / den;
                            sv[d * F + j] += -mi * B * vij / den;
                        }
                    }
                }
            }
            __syncwarp();
        }
    }
    // write the footprint back (through L2: other SMs read it after the barrier)
    for (int q = lane; q < Ftot; q += 32) {
        const int j = fr.particle(q);
#pragma unroll
        for (int d = 0; d < D; ++d) __stcg(a.v + (size_t)d * n + j, sv[d * F + q]);
    }
    __syncwarp();
}

// The whole damping operator S_d of one damped step in one cooperative
// launch: colours 0..3^d-1 forward, then 3^d-1..0 backward, with a bounded
// grid barrier between colour phases.  Each block (one warp) takes cells of
// the current colour in a grid-stride loop.
template <typename T, int D>
__global__ void __launch_bounds__(32) k_sweep_all(SweepArgs<T> a, const int* __restrict__ colour_ptr,
                                                  int ncolours, unsigned* bar)
{
    if (*(volatile int*)&a.sc->done) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const CellSmem<T, D> s = cell_smem<T, D>(smem_raw, a.max_foot, a.max_pairs, a.max_cell);
    int phases = 0;
    for (int ph = 0; ph < 2 * ncolours; ++ph) {
        const int backward = ph >= ncolours;
        const int col = backward ? 2 * ncolours - 1 - ph : ph;
        const int c0 = __ldg(colour_ptr + col), c1 = __ldg(colour_ptr + col + 1);
        if (c1 == c0) continue;
        if (phases++ > 0 && !grid_barrier(bar, bar + 1, gridDim.x, a.sc)) return;
        for (int cid = c0 + blockIdx.x; cid < c1; cid += gridDim.x)
            sweep_cell<T, D>(a, __ldg(a.colour_cells + cid), backward, s);
    }
}

__global__ void k_set_tol(DevScalars* sc, double tol)
{
    sc->tol = tol;
    if (sc->status == DEV_OK) sc->done = 0;
}

// ------------------------------------------------------------------ host side
template <typename T>
StepArgs<T> make_step_args(srdr_body* b)
{
    StepArgs<T> a{};
    a.n = (int)b->n;
    a.sell_ptr = b->sell_ptr;
    a.sell_col = b->sell_col;
    const T* sg = static_cast<const T*>(b->sell_g);
    size_t ns = (size_t)std::max<int64_t>(b->nslots, 1);
    a.g0 = sg;
    a.g1 = sg + ns;
    a.g2 = sg + 2 * ns;
    a.B0 = static_cast<const T*>(b->B0);
    a.PB = static_cast<T*>(b->PB);
    a.Gs = static_cast<const T*>(b->Gs);
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
    for (int p = 0; p < 3; ++p) {
        a.grav[p] = (T)(p < b->dim ? b->desc.gravity[p] : 0.0);
        a.endl[p] = (T)(p < b->dim ? b->desc.end_load[p] : 0.0);
    }
    return a;
}

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
    s.ncells_colour = b->ncells_nonempty;
    s.row_ptr = b->row_ptr;
    s.loc = b->loc;
    s.w = static_cast<const T*>(b->w);
    s.mass = static_cast<const T*>(b->mass);
    s.minv = static_cast<const T*>(b->minv);
    s.sumw = static_cast<const T*>(b->sumw);
    s.sumw2 = static_cast<const T*>(b->sumw2);
    s.v = static_cast<T*>(b->v);
    s.sc = b->sc;
    // B_j = 2 eta~ V_i V_j W'/r dt_loc with eta~ = eta / alpha, dt_loc = dt / 2
    s.c = (T)(b->eta / b->desc.alpha * b->dt);
    s.pairwise = b->desc.damping == SRDR_DAMP_PAIRWISE;
    s.max_foot = b->max_foot;
    s.max_pairs = b->max_pairs;
    s.max_cell = b->max_cell;
    return s;
}

template <typename T, int D>
size_t sweep_smem_bytes(const srdr_body* b)
{
    size_t C = (size_t)b->max_cell;
    size_t bytes = sizeof(T) * ((size_t)(D + 1) * b->max_foot + b->max_pairs + 3 * C) +
                   sizeof(int) * (C + 1) + sizeof(uint16_t) * b->max_pairs;
    return (bytes + 15) & ~size_t(15);
}

template <typename T, int D, int MAT>
srdr_status steps_typed(srdr_body* b, int64_t nsteps)
{
    cudaStream_t st = b->stream;
    StepArgs<T> a = make_step_args<T>(b);
    SweepArgs<T> sw = make_sweep_args<T>(b);
    const int nb = nblocks(b->n);
    const bool damping = b->desc.damping != SRDR_DAMP_NONE && b->desc.alpha > 0.0 && b->eta > 0.0;
    size_t smem = 0;
    int grid = 0;
    if (damping) {
        smem = sweep_smem_bytes<T, D>(b);
        if (smem > 227 * 1024) {
            set_error("damping sweep needs %zu bytes of shared memory per cell (limit 227 KB)", smem);
            return SRDR_ERR_INVALID;
        }
        if (smem > 48 * 1024)
            SRDR_CK(cudaFuncSetAttribute(k_sweep_all<T, D>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem));
        if (b->sweep_grid == 0) {
            int per_sm = 0, dev = 0, nsm = 0;
            SRDR_CK(cudaGetDevice(&dev));
            SRDR_CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
            SRDR_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_sweep_all<T, D>, 32, smem));
            int widest = 0;
            for (int c = 0; c < b->ncolours; ++c)
                widest = std::max(widest, b->colour_ptr[c + 1] - b->colour_ptr[c]);
            b->sweep_grid = std::max(1, std::min(widest, per_sm * nsm));
        }
        grid = b->sweep_grid;
    }
    const int* cptr = b->colour_ptr_d;
    int ncol = b->ncolours;
    unsigned* bar = b->bar;
    if (damping && (!sw.colour_cells || !sw.cell_start || !sw.row_ptr || !sw.loc || !sw.w ||
                    !sw.mass || !sw.minv || !sw.sumw || !sw.sumw2 || !sw.v || !cptr || !bar)) {
        set_error("damping sweep tables are not built");
        return SRDR_ERR_INVALID;
    }
    void* sweep_params[] = {&sw, &cptr, &ncol, &bar};
    cudaEvent_t ev = nullptr;
    auto counted = [&](int k, int nlaunch) {
        b->k_launch[k] += nlaunch;
        b->launches += nlaunch;
    };
    for (int64_t s = 0; s < nsteps; ++s) {
        const uint64_t step = (uint64_t)(b->step + s);
        const bool damp = damping && random_phi(b->desc.seed, step) < b->desc.alpha;
        prof_begin(b, SRDR_K_PASS_A, &ev);
        k_pass_a<T, D, MAT><<<nb, kThreads, 0, st>>>(a);
        prof_end(b, SRDR_K_PASS_A, ev);
        counted(SRDR_K_PASS_A, 1);
        prof_begin(b, SRDR_K_PASS_B, &ev);
        k_pass_b<T, D><<<nb, kThreads, 0, st>>>(a, damp ? 0 : 1);
        prof_end(b, SRDR_K_PASS_B, ev);
        counted(SRDR_K_PASS_B, 1);
        if (damp) {
            prof_begin(b, SRDR_K_SWEEP, &ev);
            const int nl = 1;
            SRDR_CK(cudaLaunchCooperativeKernel((const void*)k_sweep_all<T, D>, dim3(grid), dim3(32),
                                                sweep_params, smem, st));
            prof_end(b, SRDR_K_SWEEP, ev);
            counted(SRDR_K_SWEEP, nl);
            prof_begin(b, SRDR_K_FINISH, &ev);
            k_finish<T><<<nb, kThreads, 0, st>>>(a);
            prof_end(b, SRDR_K_FINISH, ev);
            counted(SRDR_K_FINISH, 1);
        }
        prof_begin(b, SRDR_K_KE, &ev);
        k_ke_final<<<1, kThreads, 0, st>>>(b->ke_part, nb, b->sc, damp ? 1 : 0);
        prof_end(b, SRDR_K_KE, ev);
        counted(SRDR_K_KE, 1);
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
