// pairg.cuh — the pair kernel gradient g_ij = V_j grad0_i W_ij (Eq.
// correction-matrix1), recomputed wherever it is needed instead of stored per
// pair.  Included inside an anonymous namespace by each translation unit.
//
// W'(r)/r = kc (1 - r/(2h))^3 with kc = -5 alpha_d / h^2 (Wendland C2).  Each
// particle carries its offset inside its cell, cpos = (ox, oy, oz, V), and its
// cell coordinates packed 10 bits per axis (modulo 1024).  Neighbours lie in
// the same or an adjacent cell, so the sign-extended 10-bit difference of two
// coordinates is the exact cell difference for a grid of any size, and
//   r0_ij = (c_i - c_j) r_c + (o_i - o_j)
// carries only the rounding of two small offsets.  The arithmetic uses
// explicit rounding intrinsics (no contraction left to the compiler), so g is
// bitwise the same in every kernel that computes it.

// sign-extended difference of one 10-bit cell coordinate, at bit offset S
template <int S>
__device__ inline int cell_diff(int ci, int cj)
{
    const int d = ((ci >> S) & 1023) - ((cj >> S) & 1023);
    return (int)((unsigned)d << 22) >> 22;
}

// four doubles, 16-byte aligned (two 16-byte accesses)
struct __align__(16) Dbl4 {
    double x, y, z, w;
};

template <typename T>
struct PairG;
template <>
struct PairG<float> {
    template <int D>
    __device__ static void g(const float4& pi, int ci, const float4& pj, int cj, float rc,
                             float inv_h, float kc, float (&out)[D])
    {
        const float dx = __fmaf_rn((float)cell_diff<0>(ci, cj), rc, __fsub_rn(pi.x, pj.x));
        const float dy = __fmaf_rn((float)cell_diff<10>(ci, cj), rc, __fsub_rn(pi.y, pj.y));
        float r2 = __fmaf_rn(dy, dy, __fmul_rn(dx, dx));
        float dz = 0.f;
        if constexpr (D == 3) {
            dz = __fmaf_rn((float)cell_diff<20>(ci, cj), rc, __fsub_rn(pi.z, pj.z));
            r2 = __fmaf_rn(dz, dz, r2);
        }
        const float t = fmaxf(__fmaf_rn(-0.5f, __fmul_rn(__fsqrt_rn(r2), inv_h), 1.0f), 0.0f);
        const float w = __fmul_rn(__fmul_rn(kc, __fmul_rn(t, __fmul_rn(t, t))), pj.w);
        out[0] = __fmul_rn(w, dx);
        out[1] = __fmul_rn(w, dy);
        if constexpr (D == 3) out[2] = __fmul_rn(w, dz);
    }
};
template <>
struct PairG<double> {
    template <int D>
    __device__ static void g(const Dbl4& pi, int ci, const Dbl4& pj, int cj, double rc,
                             double inv_h, double kc, double (&out)[D])
    {
        const double dx = __fma_rn((double)cell_diff<0>(ci, cj), rc, __dsub_rn(pi.x, pj.x));
        const double dy = __fma_rn((double)cell_diff<10>(ci, cj), rc, __dsub_rn(pi.y, pj.y));
        double r2 = __fma_rn(dy, dy, __dmul_rn(dx, dx));
        double dz = 0.0;
        if constexpr (D == 3) {
            dz = __fma_rn((double)cell_diff<20>(ci, cj), rc, __dsub_rn(pi.z, pj.z));
            r2 = __fma_rn(dz, dz, r2);
        }
        const double t = fmax(__fma_rn(-0.5, __dmul_rn(__dsqrt_rn(r2), inv_h), 1.0), 0.0);
        const double w = __dmul_rn(__dmul_rn(kc, __dmul_rn(t, __dmul_rn(t, t))), pj.w);
        out[0] = __dmul_rn(w, dx);
        out[1] = __dmul_rn(w, dy);
        if constexpr (D == 3) out[2] = __dmul_rn(w, dz);
    }
};

template <typename T>
struct Vec4;
template <>
struct Vec4<float> {
    using type = float4;
};
template <>
struct Vec4<double> {
    using type = Dbl4;
};
template <typename T>
using vec4_t = typename Vec4<T>::type;

template <typename T>
__device__ inline vec4_t<T> load_cpos(const T* cpos, int j)
{
    if constexpr (sizeof(T) == 4) {
        return __ldg(reinterpret_cast<const float4*>(cpos) + j);
    } else {
        const double2* q = reinterpret_cast<const double2*>(cpos + (size_t)j * 4);
        double2 a = __ldg(q), b = __ldg(q + 1);
        return Dbl4{a.x, a.y, b.x, b.y};
    }
}

// velocity records [n][4] = (vx, vy, vz, 1/m): the owner's access (read-only
// cache), and the damping sweep's accesses through L2 (other SMs write them
// between its colour phases)
template <typename T>
__device__ inline vec4_t<T> ld_v4(const T* v, int j)
{
    if constexpr (sizeof(T) == 4) {
        return *reinterpret_cast<const float4*>(v + (size_t)j * 4);
    } else {
        const double2* q = reinterpret_cast<const double2*>(v + (size_t)j * 4);
        const double2 a = q[0], b = q[1];
        return Dbl4{a.x, a.y, b.x, b.y};
    }
}
template <typename T>
__device__ inline void st_v4(T* v, int j, const vec4_t<T>& x)
{
    if constexpr (sizeof(T) == 4) {
        *reinterpret_cast<float4*>(v + (size_t)j * 4) = x;
    } else {
        double2* q = reinterpret_cast<double2*>(v + (size_t)j * 4);
        q[0] = make_double2(x.x, x.y);
        q[1] = make_double2(x.z, x.w);
    }
}
template <typename T>
__device__ inline vec4_t<T> ldcg_v4(const T* v, int j)
{
    if constexpr (sizeof(T) == 4) {
        return __ldcg(reinterpret_cast<const float4*>(v + (size_t)j * 4));
    } else {
        const double2* q = reinterpret_cast<const double2*>(v + (size_t)j * 4);
        const double2 a = __ldcg(q), b = __ldcg(q + 1);
        return Dbl4{a.x, a.y, b.x, b.y};
    }
}
template <typename T>
__device__ inline void stcg_v4(T* v, int j, const vec4_t<T>& x)
{
    if constexpr (sizeof(T) == 4) {
        __stcg(reinterpret_cast<float4*>(v + (size_t)j * 4), x);
    } else {
        double2* q = reinterpret_cast<double2*>(v + (size_t)j * 4);
        __stcg(q, make_double2(x.x, x.y));
        __stcg(q + 1, make_double2(x.z, x.w));
    }
}

// packed cell coordinates of linear cell c (x fastest), 10 bits per axis
__device__ inline int pack_cell(int c, int nx, int ny)
{
    const int cx = c % nx, cy = (c / nx) % ny, cz = c / (nx * ny);
    return (cx & 1023) | ((cy & 1023) << 10) | ((cz & 1023) << 20);
}
