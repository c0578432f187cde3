// setup.cu — body construction on the GPU: splitting cell-linked list and
// colour split (Sec. 3.4), fixed reference neighbours with kernel-gradient
// weights (Eq. correction-matrix1), correction matrices (Eq. correction-matrix)
// and the sliced-ELL layout streamed by the stress and force passes.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <vector>

#include "srdr_internal.cuh"

namespace srdr {

namespace {

constexpr int kThreads = 256;

inline int nblocks(int64_t n, int t = kThreads) { return (int)((n + t - 1) / t); }

#include "pairg.cuh"

// Wendland C2 (h = support / 2): W(q) = a_d (1 - q/2)^4 (1 + 2q), q = r/h < 2, with
// a_2 = 7 / (4 pi h^2), a_3 = 21 / (16 pi h^3).  Its radial derivative divided
// by r is W'(r)/r = -5 a_d / h^2 (1 - q/2)^3, free of a division by r.
__device__ inline double wendland_dw_over_r(int dim, double h, double r)
{
    const double pi = 3.14159265358979323846;
    double a = dim == 2 ? 7.0 / (4.0 * pi * h * h) : 21.0 / (16.0 * pi * h * h * h);
    double t = 1.0 - 0.5 * (r / h);
    if (t <= 0.0) return 0.0;
    return -5.0 * a / (h * h) * t * t * t;
}

// squared distance, IEEE ops in x, y, z order (no contraction), so that the
// integer decision 0 < d2 < rc2 is reproducible bit for bit
__device__ inline double dist2(int dim, const double* r0, int n, int i, int j)
{
    double s = 0.0;
    for (int a = 0; a < dim; ++a) {
        double d = __dsub_rn(r0[(size_t)a * n + i], r0[(size_t)a * n + j]);
        s = __dadd_rn(s, __dmul_rn(d, d));
    }
    return s;
}

// Neighbour test 0 < |r0_i - r0_j|^2 < rc2, decided exactly by the FP64
// operations above; an FP32 estimate from the cell offsets and packed cells
// (error below 1e-6 rc2 for any body size) settles the clear cases first, so
// FP64 work is spent only near the cut-off and on the pairs that are kept.
// Returns 1 clearly inside, 0 clearly outside, -1 undecided.
__device__ inline int near_prefilter(int dim, const float4& oi, int ci, const float4& oj, int cj, float rcf,
                                     float rc2f)
{
    const float dx = fmaf((float)cell_diff<0>(ci, cj), rcf, oi.x - oj.x);
    const float dy = fmaf((float)cell_diff<10>(ci, cj), rcf, oi.y - oj.y);
    float d2 = dx * dx + dy * dy;
    if (dim == 3) {
        const float dz = fmaf((float)cell_diff<20>(ci, cj), rcf, oi.z - oj.z);
        d2 += dz * dz;
    }
    if (d2 > rc2f * 1.00001f) return 0;
    if (d2 < rc2f * 0.99999f && d2 > rc2f * 1e-5f) return 1;
    return -1;
}

// ------------------------------------------------------------------ bbox
__global__ void k_bbox_partial(const double* __restrict__ r0aos, int n, double* __restrict__ part)
{
    __shared__ double smin[3][kThreads], smax[3][kThreads];
    int t = threadIdx.x;
    double mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int i = blockIdx.x * blockDim.x + t; i < n; i += gridDim.x * blockDim.x)
        for (int a = 0; a < 3; ++a) {
            double x = r0aos[(size_t)i * 3 + a];
            mn[a] = fmin(mn[a], x);
            mx[a] = fmax(mx[a], x);
        }
    for (int a = 0; a < 3; ++a) {
        smin[a][t] = mn[a];
        smax[a][t] = mx[a];
    }
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (t < s)
            for (int a = 0; a < 3; ++a) {
                smin[a][t] = fmin(smin[a][t], smin[a][t + s]);
                smax[a][t] = fmax(smax[a][t], smax[a][t + s]);
            }
        __syncthreads();
    }
    if (t == 0)
        for (int a = 0; a < 3; ++a) {
            part[blockIdx.x * 6 + a] = smin[a][0];
            part[blockIdx.x * 6 + 3 + a] = smax[a][0];
        }
}

__global__ void k_bbox_final(const double* __restrict__ part, int nb, double* __restrict__ out)
{
    __shared__ double smin[3][kThreads], smax[3][kThreads];
    const int t = threadIdx.x;
    double mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int b = t; b < nb; b += blockDim.x)
        for (int a = 0; a < 3; ++a) {
            mn[a] = fmin(mn[a], part[b * 6 + a]);
            mx[a] = fmax(mx[a], part[b * 6 + 3 + a]);
        }
    for (int a = 0; a < 3; ++a) {
        smin[a][t] = mn[a];
        smax[a][t] = mx[a];
    }
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (t < s)
            for (int a = 0; a < 3; ++a) {
                smin[a][t] = fmin(smin[a][t], smin[a][t + s]);
                smax[a][t] = fmax(smax[a][t], smax[a][t + s]);
            }
        __syncthreads();
    }
    if (t == 0)
        for (int a = 0; a < 3; ++a) {
            out[a] = smin[a][0];
            out[3 + a] = smax[a][0];
        }
}

// ------------------------------------------------------------------ cells
struct Grid {
    int dim;
    int nx, ny, nz;
    double lo0, lo1, lo2;
    double rc;
};

// FP32 cell offsets (for the prefilter) and packed cell coordinates
__global__ void k_cell_pos_f(const double* __restrict__ r0, int n, Grid g, const int* __restrict__ cell_of,
                             float4* __restrict__ of, int* __restrict__ ccell)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int c = cell_of[i];
    const int cc[3] = {c % g.nx, (c / g.nx) % g.ny, c / (g.nx * g.ny)};
    const double lo[3] = {g.lo0, g.lo1, g.lo2};
    float o[3] = {0.f, 0.f, 0.f};
    for (int a = 0; a < g.dim; ++a) o[a] = (float)fma(-(double)cc[a], g.rc, r0[(size_t)a * n + i] - lo[a]);
    of[i] = make_float4(o[0], o[1], o[2], 0.f);
    ccell[i] = pack_cell(c, g.nx, g.ny);
}


__device__ inline int cell_coord(double x, double lo, double rc, int ncell)
{
    double q = floor(__ddiv_rn(__dsub_rn(x, lo), rc));
    int c = (int)q;
    if (q < 0.0) c = 0;
    if (c > ncell - 1) c = ncell - 1;
    return c;
}

__global__ void k_cell_hash(const double* __restrict__ r0aos, int n, Grid g, int* __restrict__ cell,
                            int* __restrict__ count)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int cx = cell_coord(r0aos[(size_t)i * 3 + 0], g.lo0, g.rc, g.nx);
    int cy = g.dim >= 2 ? cell_coord(r0aos[(size_t)i * 3 + 1], g.lo1, g.rc, g.ny) : 0;
    int cz = g.dim >= 3 ? cell_coord(r0aos[(size_t)i * 3 + 2], g.lo2, g.rc, g.nz) : 0;
    int c = cx + g.nx * (cy + g.ny * cz);
    cell[i] = c;
    atomicAdd(&count[c], 1);
}

// exclusive scan over int counts, three kernels: per-block scan (1024
// elements, 512 threads), scan of block totals (one block, sequential
// chunks), add block offsets.
constexpr int kScanBlock = 1024;

__global__ void k_scan_local(const int* __restrict__ in, int* __restrict__ out, int count,
                             int* __restrict__ totals)
{
    __shared__ int s[kScanBlock];
    int base = blockIdx.x * kScanBlock;
    for (int k = threadIdx.x; k < kScanBlock; k += blockDim.x)
        s[k] = base + k < count ? in[base + k] : 0;
    __syncthreads();
    // Hillis-Steele inclusive scan
    for (int off = 1; off < kScanBlock; off <<= 1) {
        int vals[2];
        for (int q = 0; q < 2; ++q) {
            int k = threadIdx.x + q * blockDim.x;
            vals[q] = k >= off ? s[k - off] : 0;
        }
        __syncthreads();
        for (int q = 0; q < 2; ++q) s[threadIdx.x + q * blockDim.x] += vals[q];
        __syncthreads();
    }
    for (int k = threadIdx.x; k < kScanBlock; k += blockDim.x)
        if (base + k < count) out[base + k] = k == 0 ? 0 : s[k - 1];
    if (threadIdx.x == 0) totals[blockIdx.x] = s[kScanBlock - 1];
}

__global__ void k_scan_totals(int* __restrict__ totals, int nb, int* __restrict__ grand)
{
    if (threadIdx.x != 0) return;
    long long run = 0;
    for (int b = 0; b < nb; ++b) {
        long long t = totals[b];
        totals[b] = (int)run;
        run += t;
    }
    *grand = run > 0x7fffffffLL ? -1 : (int)run;
}

__global__ void k_scan_add(int* __restrict__ out, int count, const int* __restrict__ totals,
                           const int* __restrict__ grand)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < count) out[k] += totals[k / kScanBlock];
    if (k == 0) out[count] = *grand;
}

__global__ void k_scatter(const int* __restrict__ cell, int n, const int* __restrict__ start,
                          int* __restrict__ fill, int* __restrict__ perm)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int c = cell[i];
    perm[start[c] + atomicAdd(&fill[c], 1)] = i;
}

// stable order inside each cell: ascending original id (insertion sort)
__global__ void k_cell_sort(const int* __restrict__ start, int ncells, int* __restrict__ perm)
{
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncells) return;
    int a = start[c], b = start[c + 1];
    for (int k = a + 1; k < b; ++k) {
        int x = perm[k];
        int m = k - 1;
        while (m >= a && perm[m] > x) {
            perm[m + 1] = perm[m];
            --m;
        }
        perm[m + 1] = x;
    }
}

template <typename T>
__global__ void k_gather(const int* __restrict__ perm, int n, const double* __restrict__ r0aos,
                         const double* __restrict__ vol, double vol0, const uint8_t* __restrict__ fl,
                         const double* __restrict__ u0, const int* __restrict__ cell_orig,
                         double rho0, int* __restrict__ inv, int* __restrict__ cell_of,
                         double* __restrict__ r0, uint8_t* __restrict__ flags, T* __restrict__ mass,
                         T* __restrict__ minv, double* __restrict__ u, float* __restrict__ uhi, float* __restrict__ ulo)
{
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    int i = perm[s];
    inv[i] = s;
    cell_of[s] = cell_orig[i];
    for (int a = 0; a < 3; ++a) r0[(size_t)a * n + s] = r0aos[(size_t)i * 3 + a];
    flags[s] = fl ? fl[i] : 0;
    const double m = rho0 * (vol ? vol[i] : vol0);
    mass[s] = (T)m;
    minv[s] = (T)(1.0 / m);
    // u at the half step, AoS padded to 4: FP64 [n][4], or FP32 hi and lo
    // ((hi x, y, z, lo x) [n][4] and (lo y, lo z) [n][2])
    float h[3], l[3];
    for (int a = 0; a < 4; ++a) {
        double x = (u0 && a < 3) ? u0[(size_t)i * 3 + a] : 0.0;
        if (u) u[(size_t)s * 4 + a] = x;
        if (a < 3) {
            h[a] = (float)x;
            l[a] = (float)(x - (double)h[a]);
        }
    }
    if (uhi) {
        reinterpret_cast<float4*>(uhi)[s] = make_float4(h[0], h[1], h[2], l[0]);
        reinterpret_cast<float2*>(ulo)[s] = make_float2(l[1], l[2]);
    }
}

// per particle: offset inside its cell and volume, cpos = (r0 - lo - c r_c, V),
// and the packed cell coordinates read by the pair kernel gradient
template <typename T>
__global__ void k_cell_pos(const double* __restrict__ r0, int n, Grid g, const int* __restrict__ cell_of,
                           const T* __restrict__ mass, double rho0, T* __restrict__ cpos,
                           int* __restrict__ ccell)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int c = cell_of[i];
    const int cc[3] = {c % g.nx, (c / g.nx) % g.ny, c / (g.nx * g.ny)};
    const double lo[3] = {g.lo0, g.lo1, g.lo2};
    for (int a = 0; a < 3; ++a) {
        double o = 0.0;
        if (a < g.dim) o = fma(-(double)cc[a], g.rc, r0[(size_t)a * n + i] - lo[a]);
        cpos[(size_t)i * 4 + a] = (T)o;
    }
    cpos[(size_t)i * 4 + 3] = (T)((double)mass[i] / rho0);
    ccell[i] = pack_cell(c, g.nx, g.ny);
}

// G_i = sum_j g_ij with the pair gradient the passes compute (FP64 sum), so
// that sum_j (P_i + P_j) g_ij = sum_j (P_j - P_i) g_ij + 2 P_i G_i holds to
// the rounding of the sums
template <typename T, int D>
__global__ void k_gsum(int n, const int* __restrict__ row_ptr, const int* __restrict__ col,
                       const T* __restrict__ cpos, const int* __restrict__ ccell, T rc, T inv_h,
                       T kc, T* __restrict__ Gs)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const vec4_t<T> pi = load_cpos<T>(cpos, i);
    const int ci = ccell[i];
    double G[3] = {0, 0, 0};
    for (int k = row_ptr[i]; k < row_ptr[i + 1]; ++k) {
        const int j = col[k];
        T gg[D];
        PairG<T>::template g<D>(pi, ci, load_cpos<T>(cpos, j), ccell[j], rc, inv_h, kc, gg);
        for (int p = 0; p < D; ++p) G[p] += (double)gg[p];
    }
    for (int p = 0; p < 3; ++p) Gs[(size_t)p * n + i] = (T)G[p];
}

// rotational body force of the twisting cantilever per particle (sorted
// order), from the FP64 reference positions: g_t = gamma0 sin(pi x / 2L)
// (0, -(z - z_c), y - y_c)
template <typename T>
__global__ void k_twist(int n, const double* __restrict__ r0, double g0, double L, double yc, double zc,
                        T* __restrict__ bf)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double x = r0[i], y = r0[(size_t)n + i], z = r0[(size_t)2 * n + i];
    const double gamma = g0 * sin(3.14159265358979323846 * x / (2.0 * L));
    bf[(size_t)i * 4 + 0] = T(0);
    bf[(size_t)i * 4 + 1] = (T)(-gamma * (z - zc));
    bf[(size_t)i * 4 + 2] = (T)(gamma * (y - yc));
    bf[(size_t)i * 4 + 3] = T(0);
}

// velocity records (0, 0, 0, 1/m)
template <typename T>
__global__ void k_v_init(int n, const T* __restrict__ minv, T* __restrict__ v)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int a = 0; a < 3; ++a) v[(size_t)i * 4 + a] = T(0);
    v[(size_t)i * 4 + 3] = minv[i];
}

// colour = sum_a (i_a mod q) q^a per non-empty cell: q = 3 (Sec. 3.4) or
// q = 2 (the 2^d layout over cells of edge 2 r_c)
__device__ inline int cell_colour(int c, int dim, int nx, int ny, int q)
{
    int cx = c % nx, cy = (c / nx) % ny, cz = c / (nx * ny);
    int col = cx % q;
    if (dim >= 2) col += q * (cy % q);
    if (dim >= 3) col += q * q * (cz % q);
    return col;
}

__global__ void k_colour_count(const int* __restrict__ start, int ncells, int dim, int nx, int ny, int q,
                               int* __restrict__ ccount)
{
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncells) return;
    if (start[c + 1] == start[c]) return;
    atomicAdd(&ccount[cell_colour(c, dim, nx, ny, q)], 1);
}

__global__ void k_colour_fill(const int* __restrict__ start, int ncells, int dim, int nx, int ny, int q,
                              const int* __restrict__ cptr, int* __restrict__ cfill,
                              int* __restrict__ ccells)
{
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncells) return;
    if (start[c + 1] == start[c]) return;
    int col = cell_colour(c, dim, nx, ny, q);
    ccells[cptr[col] + atomicAdd(&cfill[col], 1)] = c;
}

// The 3^d-cell footprint of a cell is at most 9 runs of consecutive cells
// (x-neighbours are consecutive ids), each a contiguous range of sorted
// particles.  Calls f(range_begin, range_end, offset_in_footprint).
template <typename F>
__device__ inline int for_footprint(int c, int dim, int nx, int ny, int nz,
                                    const int* __restrict__ start, F f)
{
    int cx = c % nx, cy = (c / nx) % ny, cz = c / (nx * ny);
    int xlo = max(cx - 1, 0), xhi = min(cx + 1, nx - 1);
    int ylo = dim >= 2 ? max(cy - 1, 0) : 0, yhi = dim >= 2 ? min(cy + 1, ny - 1) : 0;
    int zlo = dim >= 3 ? max(cz - 1, 0) : 0, zhi = dim >= 3 ? min(cz + 1, nz - 1) : 0;
    int off = 0;
    for (int z = zlo; z <= zhi; ++z)
        for (int y = ylo; y <= yhi; ++y) {
            int c0 = xlo + nx * (y + ny * z), c1 = xhi + nx * (y + ny * z);
            int a = start[c0], b = start[c1 + 1];
            f(a, b, off);
            off += b - a;
        }
    return off;
}

__global__ void k_csr_count(const double* __restrict__ r0, int n, int dim, int nx, int ny, int nz,
                            const int* __restrict__ start, const int* __restrict__ cell_of,
                            const float4* __restrict__ of, const int* __restrict__ ccell, float rcf,
                            float rc2f, double rc2, int* __restrict__ deg)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int cnt = 0;
    const float4 oi = of[i];
    const int ci = ccell[i];
    for_footprint(cell_of[i], dim, nx, ny, nz, start, [&](int a, int b, int) {
        for (int j = a; j < b; ++j) {
            if (j == i) continue;
            const int pre = near_prefilter(dim, oi, ci, of[j], ccell[j], rcf, rc2f);
            if (pre == 0) continue;
            if (pre == 1) {
                ++cnt;
                continue;
            }
            double d2 = dist2(dim, r0, n, i, j);
            if (d2 > 0.0 && d2 < rc2) ++cnt;
        }
    });
    deg[i] = cnt;
}

// neighbours (ascending original id), footprint-local index, damping weight
// w_ij = V_i V_j W'(r)/r, and per particle: sum w, sum w^2 and
// B0_i = (-sum_j V_j r0_ij (x) grad0_i W_ij)^-1 (in FP64).
template <typename T>
__global__ void k_csr_fill(const double* __restrict__ r0, int n, int dim, int nx, int ny, int nz,
                           const int* __restrict__ start, const int* __restrict__ cell_of,
                           double rc2, double h, double rho0, const T* __restrict__ mass,
                           const int* __restrict__ row_ptr, int* __restrict__ col,
                           uint16_t* __restrict__ loc, T* __restrict__ w, T* __restrict__ sumw,
                           T* __restrict__ sumw2, T* __restrict__ B0,
                           const int* __restrict__ perm, const float4* __restrict__ of,
                           const int* __restrict__ ccell, float rcf, float rc2f, DevScalars* sc)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int k = row_ptr[i];
    double Vi = (double)mass[i] / rho0;
    double M[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
    double sw = 0.0, sw2 = 0.0;
    const float4 oi = of[i];
    const int ci = ccell[i];
    const int row_end = row_ptr[i + 1];
    for_footprint(cell_of[i], dim, nx, ny, nz, start, [&](int a, int b, int off) {
        for (int j = a; j < b; ++j) {
            if (j == i) continue;
            // the same decisions as k_csr_count, so the row fills exactly
            const int pre = near_prefilter(dim, oi, ci, of[j], ccell[j], rcf, rc2f);
            if (pre == 0) continue;
            double d2 = dist2(dim, r0, n, i, j);
            if (pre < 0 && !(d2 > 0.0 && d2 < rc2)) continue;
            if (k >= row_end) {  // cannot happen with count's decisions; never write past the row
                if (atomicCAS(&sc->status, DEV_OK, DEV_NONFINITE) == DEV_OK) sc->err_index = i;
                continue;
            }
            double r = sqrt(d2);
            double f = wendland_dw_over_r(dim, h, r);
            double Vj = (double)mass[j] / rho0;
            double x[3] = {0, 0, 0};
            for (int q = 0; q < dim; ++q) x[q] = r0[(size_t)q * n + i] - r0[(size_t)q * n + j];
            for (int p = 0; p < dim; ++p)
                for (int q = 0; q < dim; ++q) M[p][q] -= Vj * f * x[p] * x[q];
            double wij = Vi * Vj * f;
            sw += wij;
            sw2 += wij * wij;
            col[k] = j;
            loc[k] = (uint16_t)(off + (j - a));
            w[k] = (T)wij;
            ++k;
        }
    });
    // Canonical neighbour order of a row: ascending ORIGINAL particle id.  The
    // pairwise local operator applies its pair updates in row order (Sec. 3.2),
    // so the order is part of the result; insertion sort by perm[col], on a
    // thread-local copy of the row when it fits (keys read once), else in place.
    constexpr int kSortCap = 160;
    if (k - row_ptr[i] <= kSortCap) {
        const int k0 = row_ptr[i], deg = k - k0;
        int key[kSortCap], cj[kSortCap];
        uint16_t lj[kSortCap];
        T wj[kSortCap];
        for (int a = 0; a < deg; ++a) {
            cj[a] = col[k0 + a];
            lj[a] = loc[k0 + a];
            wj[a] = w[k0 + a];
            key[a] = perm[cj[a]];
        }
        for (int a = 1; a < deg; ++a) {
            const int kk = key[a], cc = cj[a];
            const uint16_t ll = lj[a];
            const T ww = wj[a];
            int m = a - 1;
            while (m >= 0 && key[m] > kk) {
                key[m + 1] = key[m];
                cj[m + 1] = cj[m];
                lj[m + 1] = lj[m];
                wj[m + 1] = wj[m];
                --m;
            }
            key[m + 1] = kk;
            cj[m + 1] = cc;
            lj[m + 1] = ll;
            wj[m + 1] = ww;
        }
        for (int a = 0; a < deg; ++a) {
            col[k0 + a] = cj[a];
            loc[k0 + a] = lj[a];
            w[k0 + a] = wj[a];
        }
    } else {
        const int k0 = row_ptr[i];
        for (int a = k0 + 1; a < k; ++a) {
            int cj = col[a];
            uint16_t lj = loc[a];
            T wj = w[a];
            int key = perm[cj];
            int m = a - 1;
            while (m >= k0 && perm[col[m]] > key) {
                col[m + 1] = col[m];
                loc[m + 1] = loc[m];
                w[m + 1] = w[m];
                --m;
            }
            col[m + 1] = cj;
            loc[m + 1] = lj;
            w[m + 1] = wj;
        }
    }
    sumw[i] = (T)sw;
    sumw2[i] = (T)sw2;
    double inv[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
    double det;
    if (dim == 2) {
        det = M[0][0] * M[1][1] - M[0][1] * M[1][0];
        inv[0][0] = M[1][1] / det;
        inv[0][1] = -M[0][1] / det;
        inv[1][0] = -M[1][0] / det;
        inv[1][1] = M[0][0] / det;
    } else {
        double c00 = M[1][1] * M[2][2] - M[1][2] * M[2][1];
        double c01 = M[1][2] * M[2][0] - M[1][0] * M[2][2];
        double c02 = M[1][0] * M[2][1] - M[1][1] * M[2][0];
        det = M[0][0] * c00 + M[0][1] * c01 + M[0][2] * c02;
        inv[0][0] = c00 / det;
        inv[1][0] = c01 / det;
        inv[2][0] = c02 / det;
        inv[0][1] = (M[0][2] * M[2][1] - M[0][1] * M[2][2]) / det;
        inv[1][1] = (M[0][0] * M[2][2] - M[0][2] * M[2][0]) / det;
        inv[2][1] = (M[0][1] * M[2][0] - M[0][0] * M[2][1]) / det;
        inv[0][2] = (M[0][1] * M[1][2] - M[0][2] * M[1][1]) / det;
        inv[1][2] = (M[0][2] * M[1][0] - M[0][0] * M[1][2]) / det;
        inv[2][2] = (M[0][0] * M[1][1] - M[0][1] * M[1][0]) / det;
    }
    if (!(fabs(det) >= 1e-8)) {
        if (atomicCAS(&sc->status, DEV_OK, DEV_SINGULAR_B0) == DEV_OK) sc->err_index = i;
    }
    for (int p = 0; p < dim; ++p)
        for (int q = 0; q < dim; ++q) B0[(size_t)(p * dim + q) * n + i] = (T)inv[p][q];
}

__global__ void k_sell_width(const int* __restrict__ row_ptr, int n, int nslices,
                             int* __restrict__ slots)
{
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nslices) return;
    int wmax = 0;
    for (int l = 0; l < 32; ++l) {
        int i = s * 32 + l;
        if (i < n) wmax = max(wmax, row_ptr[i + 1] - row_ptr[i]);
    }
    slots[s] = wmax * 32;
}

// sliced ELL: slot (slice s, column t, lane l) holds neighbour t of particle
// 32 s + l and g_ij from the same formula that gives G_i; padding slots hold
// the particle itself with g = 0
template <typename T, int D>
__global__ void k_sell_fill(int n, const int* __restrict__ row_ptr, const int* __restrict__ col,
                            const int* __restrict__ sell_ptr, const T* __restrict__ cpos,
                            const int* __restrict__ ccell, T rc, T inv_h, T kc,
                            int* __restrict__ scol, T* __restrict__ sg, int64_t nslots)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int s = i >> 5, lane = i & 31;
    int base = sell_ptr[s], width = (sell_ptr[s + 1] - base) >> 5;
    int k0 = row_ptr[i], deg = row_ptr[i + 1] - k0;
    const vec4_t<T> pi = load_cpos<T>(cpos, i);
    const int ci = ccell[i];
    for (int t = 0; t < width; ++t) {
        int64_t slot = (int64_t)base + t * 32 + lane;
        T g[3] = {0, 0, 0};
        int j = i;
        if (t < deg) {
            j = col[k0 + t];
            T gg[D];
            PairG<T>::template g<D>(pi, ci, load_cpos<T>(cpos, j), ccell[j], rc, inv_h, kc, gg);
            for (int q = 0; q < D; ++q) g[q] = gg[q];
        }
        scol[slot] = j;
        for (int q = 0; q < 3; ++q) sg[(size_t)q * nslots + slot] = g[q];
    }
}

__global__ void k_foot_stats(const int* __restrict__ start, int ncells, int dim, int nx, int ny,
                             int nz, const int* __restrict__ row_ptr, int* __restrict__ out)
{
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncells) return;
    int a = start[c], b = start[c + 1];
    if (a == b) return;
    int foot = for_footprint(c, dim, nx, ny, nz, start, [](int, int, int) {});
    atomicMax(&out[0], foot);
    atomicMax(&out[1], row_ptr[b] - row_ptr[a]);
    atomicMax(&out[2], b - a);
}

// 2^d layout: the particles a cell's sweep touches (its own particles and
// their neighbours), as ranks among the positions of its 3^d-cell footprint.
// One block per cell of the grid.  fill = 0 counts them (and their maximum);
// fill = 1 rewrites the cell's row entries' footprint-local indices into
// ranks, stores the touched particles' sorted indices at foot_tab[foot_ptr[c]
// + rank] (ascending: footprint positions follow the sorted order) and the
// rank of the cell's first particle.  Shared memory: one flag and one rank
// per footprint position (maxf of them).
__global__ void __launch_bounds__(256) k_touch(const int* __restrict__ start, int dim, int nx, int ny, int nz,
                                               const int* __restrict__ row_ptr, uint16_t* __restrict__ loc,
                                               int maxf, int fill, int* __restrict__ count,
                                               int* __restrict__ maxcount, const int* __restrict__ foot_ptr,
                                               int* __restrict__ foot_tab, int* __restrict__ own_off)
{
    extern __shared__ int tsm[];
    int* rank = tsm;                  // [maxf]
    int* part = tsm + maxf;           // [256] per-thread counts
    const int c = blockIdx.x;
    const int cs = start[c], ce = start[c + 1];
    if (cs == ce) return;
    int a_r[9], off_r[10], nr = 0;
    int own = 0;
    const int F = for_footprint(c, dim, nx, ny, nz, start, [&](int a, int b, int off) {
        if (cs >= a && cs < b) own = off + (cs - a);
        a_r[nr] = a;
        off_r[nr] = off;
        ++nr;
    });
    off_r[nr] = F;
    for (int f = threadIdx.x; f < F; f += blockDim.x) rank[f] = 0;
    __syncthreads();
    for (int q = threadIdx.x; q < ce - cs; q += blockDim.x) rank[own + q] = 1;
    for (int k = row_ptr[cs] + threadIdx.x; k < row_ptr[ce]; k += blockDim.x) rank[loc[k]] = 1;
    __syncthreads();
    // exclusive scan of the flags: each thread a contiguous chunk
    const int chunk = (F + blockDim.x - 1) / blockDim.x;
    const int f0 = min(F, (int)threadIdx.x * chunk), f1 = min(F, f0 + chunk);
    int cnt = 0;
    for (int f = f0; f < f1; ++f) cnt += rank[f];
    part[threadIdx.x] = cnt;
    __syncthreads();
    if (threadIdx.x == 0) {
        int run = 0;
        for (int t = 0; t < (int)blockDim.x; ++t) {
            const int x = part[t];
            part[t] = run;
            run += x;
        }
        if (!fill) {
            count[c] = run;
            atomicMax(maxcount, run);
        }
    }
    __syncthreads();
    if (!fill) return;
    int run = part[threadIdx.x];
    for (int f = f0; f < f1; ++f) {
        const int flag = rank[f];
        rank[f] = flag ? run : -1;
        if (flag) {
            int r = 0;
            while (r + 1 < nr && f >= off_r[r + 1]) ++r;
            foot_tab[foot_ptr[c] + run] = a_r[r] + (f - off_r[r]);
        }
        run += flag;
    }
    __syncthreads();
    for (int k = row_ptr[cs] + threadIdx.x; k < row_ptr[ce]; k += blockDim.x) loc[k] = (uint16_t)rank[loc[k]];
    if (threadIdx.x == 0) own_off[c] = rank[own];
}

srdr_status scan_exclusive(const int* in, int* out, int count, int* tmp, cudaStream_t st)
{
    // tmp holds nb totals followed by 1 grand total
    int nb = (count + kScanBlock - 1) / kScanBlock;
    if (nb < 1) nb = 1;
    k_scan_local<<<nb, kScanBlock / 2, 0, st>>>(in, out, count, tmp);
    k_scan_totals<<<1, 32, 0, st>>>(tmp, nb, tmp + nb);
    k_scan_add<<<nblocks(count + 1), kThreads, 0, st>>>(out, count, tmp, tmp + nb);
    SRDR_CK(cudaGetLastError());
    return SRDR_OK;
}

// ------------------------------------------------------------------ lattice stencil
// Lattice coordinates of particle index i of a box of lx x ly points per plane.
__device__ inline void lat_xyz(int i, int lx, int ly, int& x, int& y, int& z)
{
    const int r = i / lx;
    x = i - r * lx;
    z = r / ly;
    y = r - z * ly;
}

__device__ inline bool lat_in(const int4& o, int x, int y, int z, int lx, int ly, int lz)
{
    return (unsigned)(x + o.x) < (unsigned)lx && (unsigned)(y + o.y) < (unsigned)ly &&
           (unsigned)(z + o.z) < (unsigned)lz;
}

// The neighbour list of sorted particle s (its CSR row, ascending original
// index) against the stencil's in-box offsets in table order (zero offsets
// are padding); the first difference sets *bad.
__global__ void k_stencil_check(int n, const int* __restrict__ perm, const int* __restrict__ row_ptr,
                                const int* __restrict__ col, const int4* __restrict__ off, int K, int lx,
                                int ly, int lz, int* __restrict__ bad)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    const int i = perm[s];
    int x, y, z;
    lat_xyz(i, lx, ly, x, y, z);
    int k = row_ptr[s];
    const int k1 = row_ptr[s + 1];
    for (int t = 0; t < K; ++t) {
        const int4 o = off[t];
        if ((o.x | o.y | o.z) == 0 || !lat_in(o, x, y, z, lx, ly, lz)) continue;
        if (k >= k1 || perm[col[k]] != i + o.w) {
            atomicExch(bad, 1);
            return;
        }
        ++k;
    }
    if (k != k1) atomicExch(bad, 1);
}

// G_i = sum_j g_ij over the in-box offsets of particle i (lattice order), in
// FP64 from the table values the passes use, in table order
template <typename T, int D>
__global__ void k_stencil_gsum(int n, const int4* __restrict__ off, const T* __restrict__ g, int K, int lx,
                               int ly, int lz, T* __restrict__ Gs)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int x, y, z;
    lat_xyz(i, lx, ly, x, y, z);
    double G[3] = {0, 0, 0};
    for (int t = 0; t < K; ++t)
        if (lat_in(off[t], x, y, z, lx, ly, lz))
            for (int a = 0; a < D; ++a) G[a] += (double)g[(size_t)t * 4 + a];
    for (int a = 0; a < 3; ++a) Gs[(size_t)a * n + i] = (T)G[a];
}

// sorted -> particle order: rows of w elements (dst row perm[s] = src row s)
// and columns of an [m][n] array
template <typename E>
__global__ void k_perm_rows(const int* __restrict__ perm, int n, int w, const E* __restrict__ src,
                            E* __restrict__ dst)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    const size_t i = (size_t)perm[s];
    for (int c = 0; c < w; ++c) dst[i * w + c] = src[(size_t)s * w + c];
}

template <typename E>
__global__ void k_perm_cols(const int* __restrict__ perm, int n, int m, const E* __restrict__ src,
                            E* __restrict__ dst)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    const int i = perm[s];
    for (int c = 0; c < m; ++c) dst[(size_t)c * n + i] = src[(size_t)c * n + s];
}

// The stencil of a lattice body (b->lat set by the create path): every
// offset o with |o| dp below the cut-off, ordered by index delta (ascending
// neighbour index), with the pair gradient of the neighbour rows (Eq.
// correction-matrix1 with the Wendland C2 kernel, the formula of pairg.cuh)
// evaluated once in FP64 at r0_ij = -o dp, padded with zero offsets to a
// multiple of the passes' batch.  *ok is set when the stencil reproduces the
// neighbour list of every particle.
template <typename T>
srdr_status try_stencil(srdr_body* b, double vol, bool* ok)
{
    *ok = false;
    cudaStream_t st = b->stream;
    const int dim = b->dim, lx = b->lat[0], ly = b->lat[1], lz = b->lat[2];
    const double dp = b->desc.dp, cut = b->cut;
    const int R = (int)std::floor(cut / dp) + 1;
    struct Off {
        int x, y, z;
        long long d;
    };
    std::vector<Off> offs;
    for (int dz = dim == 3 ? -R : 0; dz <= (dim == 3 ? R : 0); ++dz)
        for (int dy = -R; dy <= R; ++dy)
            for (int dx = -R; dx <= R; ++dx) {
                if ((dx | dy | dz) == 0) continue;
                const double r2 = ((double)dx * dx + (double)dy * dy + (double)dz * dz) * dp * dp;
                if (!(r2 < cut * cut)) continue;
                offs.push_back({dx, dy, dz, dx + (long long)lx * (dy + (long long)ly * dz)});
            }
    std::sort(offs.begin(), offs.end(), [](const Off& p, const Off& q) { return p.d < q.d; });
    const int K = (int)((offs.size() + kStencilBatch - 1) / kStencilBatch * kStencilBatch);
    if (K == 0 || K > 4096) return SRDR_OK;
    std::vector<int4> ho(K, int4{0, 0, 0, 0});
    std::vector<T> hg((size_t)K * 4, T(0));
    std::vector<double> hgd((size_t)K * 4, 0.0);
    const double kc = kernel_kc(dim, b->h);
    for (size_t t = 0; t < offs.size(); ++t) {
        const Off& o = offs[t];
        if (o.d < INT32_MIN || o.d > INT32_MAX) return SRDR_OK;
        ho[t] = int4{o.x, o.y, o.z, (int)o.d};
        const double rx = -o.x * dp, ry = -o.y * dp, rz = -o.z * dp;
        const double r = std::sqrt(rx * rx + ry * ry + rz * rz);
        const double tt = std::max(1.0 - 0.5 * r / b->h, 0.0);
        const double w = kc * tt * tt * tt * vol;
        hgd[t * 4 + 0] = w * rx;
        hgd[t * 4 + 1] = w * ry;
        hgd[t * 4 + 2] = dim == 3 ? w * rz : 0.0;
        for (int c = 0; c < 3; ++c) hg[t * 4 + c] = (T)hgd[t * 4 + c];
    }
    int4* doff = nullptr;
    T* dg = nullptr;
    int* bad = nullptr;
    SRDR_TRY(dalloc(b, &doff, K));
    SRDR_TRY(dalloc(b, &dg, (size_t)K * 4));
    SRDR_TRY(dalloc(b, &bad, 1));
    SRDR_CK(cudaMemcpyAsync(doff, ho.data(), sizeof(int4) * K, cudaMemcpyHostToDevice, st));
    SRDR_CK(cudaMemcpyAsync(dg, hg.data(), sizeof(T) * 4 * K, cudaMemcpyHostToDevice, st));
    SRDR_CK(cudaMemsetAsync(bad, 0, sizeof(int), st));
    const int n = (int)b->n;
    k_stencil_check<<<nblocks(n), kThreads, 0, st>>>(n, b->perm, b->row_ptr, b->col, doff, K, lx, ly, lz, bad);
    SRDR_CK(cudaGetLastError());
    int hbad = 1;
    SRDR_CK(cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, st));
    SRDR_CK(cudaStreamSynchronize(st));
    SRDR_TRY(dev_free(b, bad));
    if (hbad) {
        SRDR_TRY(dev_free(b, doff));
        SRDR_TRY(dev_free(b, dg));
        return SRDR_OK;
    }
    b->st_off = doff;
    b->st_g = dg;
    b->st_k = K;
    b->st_off_h = ho;
    b->st_g_h = hgd;
    *ok = true;
    return SRDR_OK;
}

// Move the particle arrays of a stencil body from sorted to lattice (=
// original) order: flags, masses, 1/m, u, v, B0, body force, and G_i from
// the stencil.  The sweep keeps its structures (cells, rows, slot records)
// and sorted copies of the masses and velocity records; pidx = perm maps
// its sorted index to the particle arrays (the explicit comparator's rows).
template <typename T>
srdr_status relayout_stencil(srdr_body* b)
{
    cudaStream_t st = b->stream;
    const int n = (int)b->n, nb = nblocks(n), dim = b->dim;
    const int* perm = b->perm;
    uint8_t* fl = nullptr;
    SRDR_TRY(dalloc(b, &fl, n));
    k_perm_rows<uint8_t><<<nb, kThreads, 0, st>>>(perm, n, 1, b->flags, fl);
    T *m = nullptr, *mi = nullptr, *v = nullptr, *B0 = nullptr;
    SRDR_TRY(dalloc(b, &m, n));
    SRDR_TRY(dalloc(b, &mi, n));
    SRDR_TRY(dalloc(b, &v, (size_t)n * 4));
    SRDR_TRY(dalloc(b, &B0, (size_t)n * dim * dim));
    k_perm_rows<T><<<nb, kThreads, 0, st>>>(perm, n, 1, static_cast<const T*>(b->mass), m);
    k_perm_rows<T><<<nb, kThreads, 0, st>>>(perm, n, 1, static_cast<const T*>(b->minv), mi);
    k_perm_rows<T><<<nb, kThreads, 0, st>>>(perm, n, 4, static_cast<const T*>(b->v), v);
    k_perm_cols<T><<<nb, kThreads, 0, st>>>(perm, n, dim * dim, static_cast<const T*>(b->B0), B0);
    double* u = nullptr;
    float *uhi = nullptr, *ulo = nullptr;
    if (b->u) {
        SRDR_TRY(dalloc(b, &u, (size_t)n * 4));
        k_perm_rows<double><<<nb, kThreads, 0, st>>>(perm, n, 4, b->u, u);
    } else {
        SRDR_TRY(dalloc(b, &uhi, (size_t)n * 4));
        SRDR_TRY(dalloc(b, &ulo, (size_t)n * 2));
        k_perm_rows<float><<<nb, kThreads, 0, st>>>(perm, n, 4, b->uhi, uhi);
        k_perm_rows<float><<<nb, kThreads, 0, st>>>(perm, n, 2, b->ulo, ulo);
    }
    T* bf = nullptr;
    if (b->bf) {
        SRDR_TRY(dalloc(b, &bf, (size_t)n * 4));
        k_perm_rows<T><<<nb, kThreads, 0, st>>>(perm, n, 4, static_cast<const T*>(b->bf), bf);
    }
    if (dim == 2)
        k_stencil_gsum<T, 2><<<nb, kThreads, 0, st>>>(n, b->st_off, static_cast<const T*>(b->st_g), b->st_k,
                                                      b->lat[0], b->lat[1], b->lat[2], static_cast<T*>(b->Gs));
    else
        k_stencil_gsum<T, 3><<<nb, kThreads, 0, st>>>(n, b->st_off, static_cast<const T*>(b->st_g), b->st_k,
                                                      b->lat[0], b->lat[1], b->lat[2], static_cast<T*>(b->Gs));
    SRDR_CK(cudaGetLastError());
    SRDR_CK(cudaStreamSynchronize(st));
    SRDR_TRY(dev_free(b, b->flags));
    SRDR_TRY(dev_free(b, b->minv));
    SRDR_TRY(dev_free(b, b->B0));
    SRDR_TRY(dev_free(b, b->u));
    SRDR_TRY(dev_free(b, b->uhi));
    SRDR_TRY(dev_free(b, b->ulo));
    SRDR_TRY(dev_free(b, b->bf));
    b->mass_sw = b->mass;
    b->vs = b->v;  // the sorted records become the sweep's copy
    b->flags = fl;
    b->mass = m;
    b->minv = mi;
    b->v = v;
    b->B0 = B0;
    b->u = u;
    b->uhi = uhi;
    b->ulo = ulo;
    b->bf = bf;
    b->pidx = b->perm;
    b->stencil = 1;
    b->pass_tiled = 0;
    return SRDR_OK;
}

template <typename T>
srdr_status build_typed(srdr_body* b, int64_t n64, const double* r0_host, const double* vol_host,
                        const uint8_t* flags_host, const double* u0_host)
{
    cudaStream_t st = b->stream;
    int n = (int)n64;
    int dim = b->dim;
    // staging of the caller's arrays (original order)
    double *r0aos = nullptr, *vol = nullptr, *u0 = nullptr;
    uint8_t* fl = nullptr;
    std::vector<double> r0pad((size_t)n * 3, 0.0);
    for (int64_t i = 0; i < n; ++i)
        for (int a = 0; a < dim; ++a) r0pad[(size_t)i * 3 + a] = r0_host[(size_t)i * 3 + a];
    SRDR_TRY(dalloc(b, &r0aos, (size_t)n * 3));
    SRDR_CK(cudaMemcpyAsync(r0aos, r0pad.data(), sizeof(double) * 3 * n, cudaMemcpyHostToDevice, st));
    if (vol_host) {
        SRDR_TRY(dalloc(b, &vol, n));
        SRDR_CK(cudaMemcpyAsync(vol, vol_host, sizeof(double) * n, cudaMemcpyHostToDevice, st));
    }
    if (flags_host) {
        SRDR_TRY(dalloc(b, &fl, n));
        SRDR_CK(cudaMemcpyAsync(fl, flags_host, n, cudaMemcpyHostToDevice, st));
    }
    std::vector<double> u0pad;
    if (u0_host) {
        u0pad.assign((size_t)n * 3, 0.0);
        for (int64_t i = 0; i < n; ++i)
            for (int a = 0; a < dim; ++a) u0pad[(size_t)i * 3 + a] = u0_host[(size_t)i * 3 + a];
        SRDR_TRY(dalloc(b, &u0, (size_t)n * 3));
        SRDR_CK(cudaMemcpyAsync(u0, u0pad.data(), sizeof(double) * 3 * n, cudaMemcpyHostToDevice, st));
    }

    // bounding box -> cell grid
    int nbb = std::min(nblocks(n), 1024);
    double *bpart = nullptr, *bbox = nullptr;
    SRDR_TRY(dalloc(b, &bpart, (size_t)nbb * 6));
    SRDR_TRY(dalloc(b, &bbox, 6));
    k_bbox_partial<<<nbb, kThreads, 0, st>>>(r0aos, n, bpart);
    k_bbox_final<<<1, kThreads, 0, st>>>(bpart, nbb, bbox);
    double hb[6];
    SRDR_CK(cudaMemcpyAsync(hb, bbox, sizeof(hb), cudaMemcpyDeviceToHost, st));
    SRDR_CK(cudaStreamSynchronize(st));
    int64_t total = 1;
    for (int a = 0; a < 3; ++a) {
        b->lo[a] = hb[a];
        b->nc[a] = 1;
        if (a < dim) {
            double span = floor((hb[3 + a] - hb[a]) / b->rc);
            if (!(span >= 0.0) || span > 1e8) {
                set_error("body extent / cut-off out of range on axis %d", a);
                return SRDR_ERR_INVALID;
            }
            b->nc[a] = (int)span + 1;
        }
        total *= b->nc[a];
    }
    if (total > (1 << 28)) {
        set_error("too many cells (%lld): body too sparse for its cut-off", (long long)total);
        return SRDR_ERR_INVALID;
    }
    b->ncells = (int)total;
    int ncells = b->ncells;
    Grid g{dim, b->nc[0], b->nc[1], b->nc[2], b->lo[0], b->lo[1], b->lo[2], b->rc};

    int *cell_orig = nullptr, *count = nullptr, *fill = nullptr, *tmp = nullptr;
    int ntmp = (std::max<int64_t>(ncells, n) + 1) / kScanBlock + 4;
    SRDR_TRY(dalloc(b, &cell_orig, n));
    SRDR_TRY(dalloc(b, &count, ncells));
    SRDR_TRY(dalloc(b, &fill, ncells));
    SRDR_TRY(dalloc(b, &tmp, ntmp));
    SRDR_TRY(dalloc(b, &b->cell_start, (size_t)ncells + 1));
    SRDR_TRY(dalloc(b, &b->perm, n));
    SRDR_TRY(dalloc(b, &b->inv, n));
    SRDR_TRY(dalloc(b, &b->cell_of, n));
    SRDR_CK(cudaMemsetAsync(count, 0, sizeof(int) * ncells, st));
    SRDR_CK(cudaMemsetAsync(fill, 0, sizeof(int) * ncells, st));
    k_cell_hash<<<nblocks(n), kThreads, 0, st>>>(r0aos, n, g, cell_orig, count);
    SRDR_TRY(scan_exclusive(count, b->cell_start, ncells, tmp, st));
    k_scatter<<<nblocks(n), kThreads, 0, st>>>(cell_orig, n, b->cell_start, fill, b->perm);
    k_cell_sort<<<nblocks(ncells), kThreads, 0, st>>>(b->cell_start, ncells, b->perm);

    // sorted particle arrays and the initial (half-step) displacement
    SRDR_TRY(dalloc(b, &b->r0, (size_t)n * 3));
    SRDR_TRY(dalloc(b, &b->flags, n));
    T* mass = nullptr;
    SRDR_TRY(dalloc(b, &mass, n));
    b->mass = mass;
    T* minv = nullptr;
    SRDR_TRY(dalloc(b, &minv, n));
    b->minv = minv;
    if (b->prec == SRDR_FP64) {
        SRDR_TRY(dalloc(b, &b->u, (size_t)n * 4));
    } else {
        SRDR_TRY(dalloc(b, &b->uhi, (size_t)n * 4));
        SRDR_TRY(dalloc(b, &b->ulo, (size_t)n * 2));
    }
    k_gather<T><<<nblocks(n), kThreads, 0, st>>>(b->perm, n, r0aos, vol, b->vol0, fl, u0, cell_orig,
                                                 b->desc.rho0, b->inv, b->cell_of, b->r0, b->flags,
                                                 mass, minv, b->u, b->uhi, b->ulo);
    SRDR_CK(cudaGetLastError());

    // colour split: non-empty cells grouped by colour
    b->ncolours = b->cbase == 3 ? (dim == 2 ? 9 : 27) : (dim == 2 ? 4 : 8);
    int *ccount = nullptr, *cfill = nullptr, *cptr = nullptr;
    SRDR_TRY(dalloc(b, &ccount, 27));
    SRDR_TRY(dalloc(b, &cfill, 27));
    SRDR_TRY(dalloc(b, &cptr, 28));
    b->colour_ptr_d = cptr;
    SRDR_CK(cudaMemsetAsync(ccount, 0, sizeof(int) * 27, st));
    SRDR_CK(cudaMemsetAsync(cfill, 0, sizeof(int) * 27, st));
    k_colour_count<<<nblocks(ncells), kThreads, 0, st>>>(b->cell_start, ncells, dim, g.nx, g.ny,
                                                         b->cbase, ccount);
    int hcount[27];
    SRDR_CK(cudaMemcpyAsync(hcount, ccount, sizeof(hcount), cudaMemcpyDeviceToHost, st));
    SRDR_CK(cudaStreamSynchronize(st));
    b->colour_ptr.assign(b->ncolours + 1, 0);
    for (int c = 0; c < b->ncolours; ++c) b->colour_ptr[c + 1] = b->colour_ptr[c] + hcount[c];
    b->ncells_nonempty = b->colour_ptr[b->ncolours];
    SRDR_TRY(dalloc(b, &b->colour_cells, std::max(1, b->ncells_nonempty)));
    SRDR_CK(cudaMemcpyAsync(cptr, b->colour_ptr.data(), sizeof(int) * (b->ncolours + 1),
                            cudaMemcpyHostToDevice, st));
    k_colour_fill<<<nblocks(ncells), kThreads, 0, st>>>(b->cell_start, ncells, dim, g.nx, g.ny,
                                                        b->cbase, cptr, cfill, b->colour_cells);

    // neighbour CSR
    int* deg = nullptr;
    SRDR_TRY(dalloc(b, &deg, n));
    SRDR_TRY(dalloc(b, &b->row_ptr, (size_t)n + 1));
    double rc2 = b->cut * b->cut;  // the neighbour cut-off (the cell edge rc may be larger)
    float4* pof = nullptr;
    SRDR_TRY(dalloc(b, &pof, n));
    SRDR_TRY(dalloc(b, &b->ccell, n));
    k_cell_pos_f<<<nblocks(n), kThreads, 0, st>>>(b->r0, n, g, b->cell_of, pof, b->ccell);
    const float rcf = (float)b->rc, rc2f = (float)rc2;
    k_csr_count<<<nblocks(n), kThreads, 0, st>>>(b->r0, n, dim, g.nx, g.ny, g.nz, b->cell_start,
                                                 b->cell_of, pof, b->ccell, rcf, rc2f, rc2, deg);
    SRDR_TRY(scan_exclusive(deg, b->row_ptr, n, tmp, st));
    int nnz = 0;
    SRDR_CK(cudaMemcpyAsync(&nnz, b->row_ptr + n, sizeof(int), cudaMemcpyDeviceToHost, st));
    SRDR_CK(cudaStreamSynchronize(st));
    if (nnz < 0) {
        set_error("more than 2^31 neighbour pairs");
        return SRDR_ERR_INVALID;
    }
    b->nnz = nnz;
    T *w = nullptr, *sumw = nullptr, *sumw2 = nullptr, *Gs = nullptr, *B0 = nullptr, *PB = nullptr;
    SRDR_TRY(dalloc(b, &b->col, std::max(nnz, 1)));
    // a spare 16-byte chunk each: the sweep stages loc and w in 16-byte chunks
    SRDR_TRY(dalloc(b, &b->loc, (size_t)nnz + 8));
    SRDR_TRY(dalloc(b, &w, (size_t)nnz + 16 / sizeof(T)));
    SRDR_TRY(dalloc(b, &sumw, n));
    SRDR_TRY(dalloc(b, &sumw2, n));
    SRDR_TRY(dalloc(b, &Gs, (size_t)n * 3));
    SRDR_TRY(dalloc(b, &B0, (size_t)n * dim * dim));
    b->pb_stride = pb_stride(sizeof(T), dim);
    SRDR_TRY(dalloc(b, &PB, (size_t)n * b->pb_stride));
    b->w = w;
    b->sumw = sumw;
    b->sumw2 = sumw2;
    b->Gs = Gs;
    b->B0 = B0;
    b->PB = PB;
    SRDR_CK(cudaMemsetAsync(PB, 0, sizeof(T) * (size_t)n * b->pb_stride, st));
    k_csr_fill<T><<<nblocks(n), kThreads, 0, st>>>(b->r0, n, dim, g.nx, g.ny, g.nz, b->cell_start,
                                                   b->cell_of, rc2, b->h, b->desc.rho0, mass,
                                                   b->row_ptr, b->col, b->loc, w, sumw, sumw2, B0,
                                                   b->perm, pof, b->ccell, rcf, rc2f, b->sc);
    SRDR_CK(cudaGetLastError());

    // per-particle cell offsets and packed cells, then G_i from the same pair
    // gradient the passes evaluate
    T* cpos = nullptr;
    SRDR_TRY(dalloc(b, &cpos, (size_t)n * 4));
    b->cpos = cpos;
    k_cell_pos<T><<<nblocks(n), kThreads, 0, st>>>(b->r0, n, g, b->cell_of, mass, b->desc.rho0, cpos,
                                                   b->ccell);
    const T rcT = (T)b->rc, ihT = (T)(1.0 / b->h), kcT = (T)kernel_kc(dim, b->h);
    if (dim == 2)
        k_gsum<T, 2><<<nblocks(n), kThreads, 0, st>>>(n, b->row_ptr, b->col, cpos, b->ccell, rcT, ihT,
                                                      kcT, Gs);
    else
        k_gsum<T, 3><<<nblocks(n), kThreads, 0, st>>>(n, b->row_ptr, b->col, cpos, b->ccell, rcT, ihT,
                                                      kcT, Gs);
    SRDR_CK(cudaGetLastError());

    // the passes' neighbour enumeration: the lattice stencil (lattice bodies
    // whose neighbour lists it reproduces), else the sliced ELL
    b->nslices = (n + 31) / 32;
    bool stencil = false;
    if (b->lat[0] > 0) SRDR_TRY(try_stencil<T>(b, vol_host ? vol_host[0] : b->vol0, &stencil));
    int* slots = nullptr;
    if (!stencil) {
        SRDR_TRY(dalloc(b, &slots, b->nslices));
        SRDR_TRY(dalloc(b, &b->sell_ptr, (size_t)b->nslices + 1));
        k_sell_width<<<nblocks(b->nslices), kThreads, 0, st>>>(b->row_ptr, n, b->nslices, slots);
        SRDR_TRY(scan_exclusive(slots, b->sell_ptr, b->nslices, tmp, st));
        int nslots = 0;
        SRDR_CK(cudaMemcpyAsync(&nslots, b->sell_ptr + b->nslices, sizeof(int), cudaMemcpyDeviceToHost, st));
        SRDR_CK(cudaStreamSynchronize(st));
        if (nslots < 0) {
            set_error("sliced-ELL layout exceeds 2^31 slots");
            return SRDR_ERR_INVALID;
        }
        b->nslots = nslots;
        const int64_t ns = std::max(nslots, 1);
        SRDR_TRY(dalloc(b, &b->sell_col, ns));
        T* sg = nullptr;
        SRDR_TRY(dalloc(b, &sg, (size_t)ns * 3));
        b->sell_g = sg;
        if (dim == 2)
            k_sell_fill<T, 2><<<nblocks(n), kThreads, 0, st>>>(n, b->row_ptr, b->col, b->sell_ptr, cpos, b->ccell,
                                                               rcT, ihT, kcT, b->sell_col, sg, ns);
        else
            k_sell_fill<T, 3><<<nblocks(n), kThreads, 0, st>>>(n, b->row_ptr, b->col, b->sell_ptr, cpos, b->ccell,
                                                               rcT, ihT, kcT, b->sell_col, sg, ns);
    }

    // footprint maxima size the damping sweep's shared memory
    int* fs = nullptr;
    SRDR_TRY(dalloc(b, &fs, 3));
    SRDR_CK(cudaMemsetAsync(fs, 0, sizeof(int) * 3, st));
    k_foot_stats<<<nblocks(ncells), kThreads, 0, st>>>(b->cell_start, ncells, dim, g.nx, g.ny, g.nz,
                                                       b->row_ptr, fs);
    int hfs[3];
    SRDR_CK(cudaMemcpyAsync(hfs, fs, sizeof(hfs), cudaMemcpyDeviceToHost, st));
    SRDR_CK(cudaStreamSynchronize(st));
    SRDR_CK(cudaGetLastError());
    b->max_foot = hfs[0];
    b->max_pairs = hfs[1];
    b->max_cell = hfs[2];
    if (b->max_foot >= 65536) {
        set_error("a cell footprint holds %d particles (limit 65535)", b->max_foot);
        return SRDR_ERR_INVALID;
    }
    if (b->cbase == 2) {
        // 2^d layout: the sweep stages only the particles each cell touches
        // (same-colour cells' 3^d footprints overlap; what they touch does not)
        const size_t tsm = sizeof(int) * ((size_t)b->max_foot + 256);
        if (tsm > 200 * 1024) {
            set_error("a cell footprint of %d particles is too large for the 2^d sweep layout", b->max_foot);
            return SRDR_ERR_INVALID;
        }
        if (tsm > 48 * 1024)
            SRDR_CK(cudaFuncSetAttribute((const void*)k_touch, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)tsm));
        int *tcount = nullptr, *tmax = nullptr;
        SRDR_TRY(dalloc(b, &tcount, ncells));
        SRDR_TRY(dalloc(b, &tmax, 1));
        SRDR_TRY(dalloc(b, &b->foot_ptr, (size_t)ncells + 1));
        SRDR_TRY(dalloc(b, &b->own_off, ncells));
        SRDR_CK(cudaMemsetAsync(tcount, 0, sizeof(int) * ncells, st));
        SRDR_CK(cudaMemsetAsync(tmax, 0, sizeof(int), st));
        SRDR_CK(cudaMemsetAsync(b->own_off, 0, sizeof(int) * ncells, st));
        k_touch<<<ncells, 256, tsm, st>>>(b->cell_start, dim, g.nx, g.ny, g.nz, b->row_ptr, b->loc,
                                          b->max_foot, 0, tcount, tmax, nullptr, nullptr, nullptr);
        SRDR_TRY(scan_exclusive(tcount, b->foot_ptr, ncells, tmp, st));
        int total = 0, mx = 0;
        SRDR_CK(cudaMemcpyAsync(&total, b->foot_ptr + ncells, sizeof(int), cudaMemcpyDeviceToHost, st));
        SRDR_CK(cudaMemcpyAsync(&mx, tmax, sizeof(int), cudaMemcpyDeviceToHost, st));
        SRDR_CK(cudaStreamSynchronize(st));
        if (total < 0) {
            set_error("touched lists of the 2^d sweep layout exceed 2^31 entries");
            return SRDR_ERR_INVALID;
        }
        SRDR_TRY(dalloc(b, &b->foot_tab, std::max(total, 1)));
        k_touch<<<ncells, 256, tsm, st>>>(b->cell_start, dim, g.nx, g.ny, g.nz, b->row_ptr, b->loc,
                                          b->max_foot, 1, tcount, tmax, b->foot_ptr, b->foot_tab,
                                          b->own_off);
        SRDR_CK(cudaGetLastError());
        SRDR_CK(cudaStreamSynchronize(st));
        SRDR_TRY(dev_free(b, tcount));
        SRDR_TRY(dev_free(b, tmax));
        b->max_foot = mx;
    }
    SRDR_TRY(dalloc(b, &b->bar, kBarWords));
    SRDR_CK(cudaMemsetAsync(b->bar, 0, sizeof(unsigned) * kBarWords, st));
    SRDR_TRY(dalloc(b, &b->flow, flow_words(ncells)));
    SRDR_CK(cudaMemsetAsync(b->flow, 0, sizeof(unsigned) * flow_words(ncells), st));
    if (b->max_foot >= 65536) {
        set_error("a cell footprint holds %d particles (limit 65535)", b->max_foot);
        return SRDR_ERR_INVALID;
    }
    // velocity state and KE partials
    T* v = nullptr;
    SRDR_TRY(dalloc(b, &v, (size_t)n * 4));
    b->v = v;
    k_v_init<T><<<nblocks(n), kThreads, 0, st>>>(n, minv, v);
    if (b->desc.twist[0] != 0.0) {
        T* bf = nullptr;
        SRDR_TRY(dalloc(b, &bf, (size_t)n * 4));
        b->bf = bf;
        k_twist<T><<<nblocks(n), kThreads, 0, st>>>(n, b->r0, b->desc.twist[0], b->desc.twist[1],
                                                   b->desc.twist[2], b->desc.twist[3], bf);
    }
    // one FP64 partial per 32-particle slice, then one per group of 8 slices
    b->ke_blocks = b->nslices + (b->nslices + 7) / 8;
    SRDR_TRY(dalloc(b, &b->ke_part, b->ke_blocks));
    SRDR_CK(cudaMemsetAsync(b->ke_part, 0, sizeof(double) * b->ke_blocks, st));

    // release the staging buffers
    SRDR_CK(cudaStreamSynchronize(st));
    for (void* p : {(void*)r0aos, (void*)vol, (void*)u0, (void*)fl, (void*)bpart, (void*)bbox,
                    (void*)cell_orig, (void*)count, (void*)fill, (void*)ccount, (void*)cfill,
                    (void*)deg, (void*)slots, (void*)fs, (void*)tmp, (void*)pof})
        SRDR_TRY(dev_free(b, p));
    SRDR_CK(cudaStreamSynchronize(st));
    if (b->sc_host) {
        SRDR_CK(cudaMemcpy(b->sc_host, b->sc, sizeof(DevScalars), cudaMemcpyDeviceToHost));
        if (b->sc_host->status == DEV_SINGULAR_B0) {
            set_error("singular correction matrix at particle (sorted index) %lld",
                      (long long)b->sc_host->err_index);
            return SRDR_ERR_INVALID;
        }
        if (b->sc_host->status != DEV_OK) {
            set_error("neighbour rows inconsistent at particle (sorted index) %lld",
                      (long long)b->sc_host->err_index);
            return SRDR_ERR_INVALID;
        }
    }
    if (stencil) SRDR_TRY(relayout_stencil<T>(b));
    return SRDR_OK;
}


// ------------------------------------------------------------------ brick tiles
// Bricks of bx x by x bz cells tile the cell grid (brick q = qx + nbx (qy +
// nby qz)).  A brick's own particles are those of its cells, in rows of
// cells along x (z outer, y inner), each row a contiguous range of sorted
// particles; its halo is the box of cells one cell wider on every side
// (clipped to the grid), again as rows.  Every neighbour of an own particle
// lies in the halo.
constexpr int kMaxHaloRows = 36;  // (4 + 2) x (4 + 2)

struct BrickGeo {
    int x0, x1, y0, y1, z0, z1;        // own cell box (inclusive)
    int hx0, hx1, hy0, hy1, hz0, hz1;  // halo cell box (inclusive)
};

__device__ inline BrickGeo brick_geo(int q, const int* bd, const int* nb, int nx, int ny, int nz)
{
    BrickGeo g;
    const int qx = q % nb[0], qy = (q / nb[0]) % nb[1], qz = q / (nb[0] * nb[1]);
    g.x0 = qx * bd[0];
    g.x1 = min(g.x0 + bd[0], nx) - 1;
    g.y0 = qy * bd[1];
    g.y1 = min(g.y0 + bd[1], ny) - 1;
    g.z0 = qz * bd[2];
    g.z1 = min(g.z0 + bd[2], nz) - 1;
    g.hx0 = max(g.x0 - 1, 0);
    g.hx1 = min(g.x1 + 1, nx - 1);
    g.hy0 = max(g.y0 - 1, 0);
    g.hy1 = min(g.y1 + 1, ny - 1);
    g.hz0 = max(g.z0 - 1, 0);
    g.hz1 = min(g.z1 + 1, nz - 1);
    return g;
}

struct BrickDims {
    int bd[3], nb[3];
};

__global__ void k_brick_count(const int* __restrict__ start, int nx, int ny, int nz, BrickDims d, int nball,
                              int* __restrict__ nown, int* __restrict__ nhalo)
{
    int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nball) return;
    const BrickGeo g = brick_geo(q, d.bd, d.nb, nx, ny, nz);
    int own = 0, halo = 0;
    for (int z = g.z0; z <= g.z1; ++z)
        for (int y = g.y0; y <= g.y1; ++y)
            own += start[g.x1 + nx * (y + ny * z) + 1] - start[g.x0 + nx * (y + ny * z)];
    for (int z = g.hz0; z <= g.hz1; ++z)
        for (int y = g.hy0; y <= g.hy1; ++y)
            halo += start[g.hx1 + nx * (y + ny * z) + 1] - start[g.hx0 + nx * (y + ny * z)];
    nown[q] = own;
    nhalo[q] = halo;
}

// halo rows of a brick: first sorted particle hst[r] and halo offset hoff[r]
struct HaloRows {
    int nr, hny;
    int hst[kMaxHaloRows];
    int hoff[kMaxHaloRows + 1];
};

__device__ inline void halo_rows(const BrickGeo& g, const int* start, int nx, int ny, HaloRows& h)
{
    h.hny = g.hy1 - g.hy0 + 1;
    h.nr = 0;
    h.hoff[0] = 0;
    for (int z = g.hz0; z <= g.hz1; ++z)
        for (int y = g.hy0; y <= g.hy1; ++y) {
            const int a = start[g.hx0 + nx * (y + ny * z)], e = start[g.hx1 + nx * (y + ny * z) + 1];
            h.hst[h.nr] = a;
            h.hoff[h.nr + 1] = h.hoff[h.nr] + (e - a);
            ++h.nr;
        }
}

// bown / bown_h (own particles in brick order and their halo indices) and
// bhalo (halo particles), one block per non-empty brick
__global__ void k_brick_fill(const BrickInfo* __restrict__ info, const int* __restrict__ start, int nx,
                             int ny, int nz, BrickDims d, int* __restrict__ bown,
                             uint16_t* __restrict__ bown_h, int* __restrict__ bhalo)
{
    __shared__ HaloRows h;
    const BrickInfo bi = info[blockIdx.x];
    const BrickGeo g = brick_geo(bi.q, d.bd, d.nb, nx, ny, nz);
    if (threadIdx.x == 0) halo_rows(g, start, nx, ny, h);
    __syncthreads();
    for (int r = 0; r < h.nr; ++r)
        for (int e = threadIdx.x; e < h.hoff[r + 1] - h.hoff[r]; e += blockDim.x)
            bhalo[bi.halo_base + h.hoff[r] + e] = h.hst[r] + e;
    int ko = 0;
    for (int z = g.z0; z <= g.z1; ++z)
        for (int y = g.y0; y <= g.y1; ++y) {
            const int a = start[g.x0 + nx * (y + ny * z)], e = start[g.x1 + nx * (y + ny * z) + 1];
            const int r = (z - g.hz0) * h.hny + (y - g.hy0);
            for (int t = threadIdx.x; t < e - a; t += blockDim.x) {
                bown[bi.own_base + ko + t] = a + t;
                bown_h[bi.own_base + ko + t] = (uint16_t)(h.hoff[r] + (a + t - h.hst[r]));
            }
            ko += e - a;
        }
}

// slots of each brick slice (32 own particles): 32 x the longest row
__global__ void k_bslice_width(const BrickInfo* __restrict__ info, const int* __restrict__ bown,
                               const int* __restrict__ row_ptr, int* __restrict__ slots)
{
    const BrickInfo bi = info[blockIdx.x];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int ns = (bi.nown + 31) >> 5;
    for (int sl = w; sl < ns; sl += blockDim.x >> 5) {
        const int k = sl * 32 + lane;
        int deg = 0;
        if (k < bi.nown) {
            const int i = bown[bi.own_base + k];
            deg = row_ptr[i + 1] - row_ptr[i];
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) deg = max(deg, __shfl_xor_sync(0xffffffffu, deg, o));
        if (lane == 0) slots[bi.slice_base + sl] = deg * 32;
    }
}

// brick sliced ELL: slot (slice, column t, lane) holds the halo index of
// neighbour t of the lane's own particle and g_ij (the formula of the
// sliced-ELL layout, so both layouts hold the same bits); padding: the
// particle itself (lanes past the brick's particles: index 0) with g = 0
template <typename T, int D>
__global__ void k_bsell_fill(const BrickInfo* __restrict__ info, const int* __restrict__ start, int nx,
                             int ny, int nz, BrickDims d, const int* __restrict__ bown,
                             const uint16_t* __restrict__ bown_h, const int* __restrict__ row_ptr,
                             const int* __restrict__ col, const int* __restrict__ cell_of,
                             const int* __restrict__ bsell_ptr, const T* __restrict__ cpos,
                             const int* __restrict__ ccell, T rc, T inv_h, T kc,
                             uint16_t* __restrict__ lidx, T* __restrict__ sg, int64_t nslots)
{
    __shared__ HaloRows h;
    const BrickInfo bi = info[blockIdx.x];
    const BrickGeo g = brick_geo(bi.q, d.bd, d.nb, nx, ny, nz);
    if (threadIdx.x == 0) halo_rows(g, start, nx, ny, h);
    __syncthreads();
    const int ns = (bi.nown + 31) >> 5;
    for (int k = threadIdx.x; k < ns * 32; k += blockDim.x) {
        const int sl = bi.slice_base + (k >> 5), lane = k & 31;
        const int base = bsell_ptr[sl], width = (bsell_ptr[sl + 1] - base) >> 5;
        const bool own = k < bi.nown;
        int i = 0, hi = 0, k0 = 0, deg = 0;
        vec4_t<T> pi{};
        int ci = 0;
        if (own) {
            i = bown[bi.own_base + k];
            hi = bown_h[bi.own_base + k];
            k0 = row_ptr[i];
            deg = row_ptr[i + 1] - k0;
            pi = load_cpos<T>(cpos, i);
            ci = ccell[i];
        }
        for (int t = 0; t < width; ++t) {
            const int64_t slot = (int64_t)base + t * 32 + lane;
            T gq[3] = {0, 0, 0};
            int l = hi;
            if (t < deg) {
                const int j = col[k0 + t];
                const int c = cell_of[j];
                const int cy = (c / nx) % ny, cz = c / (nx * ny);
                const int r = (cz - g.hz0) * h.hny + (cy - g.hy0);
                l = h.hoff[r] + (j - h.hst[r]);
                T gg[D];
                PairG<T>::template g<D>(pi, ci, load_cpos<T>(cpos, j), ccell[j], rc, inv_h, kc, gg);
                for (int q = 0; q < D; ++q) gq[q] = gg[q];
            }
            lidx[slot] = (uint16_t)l;
            for (int q = 0; q < 3; ++q) sg[(size_t)q * nslots + slot] = gq[q];
        }
    }
}

template <typename T>
srdr_status build_bricks_typed(srdr_body* b)
{
    cudaStream_t st = b->stream;
    const int dim = b->dim;
    BrickDims d;
    for (int a = 0; a < 3; ++a) {
        int e = b->brick[a];
        if (e == 0) e = dim == 2 ? (a < 2 ? 4 : 1) : 2;
        if (a >= dim) e = 1;
        d.bd[a] = e;
        d.nb[a] = (b->nc[a] + e - 1) / e;
    }
    const int nball = d.nb[0] * d.nb[1] * d.nb[2];
    int *nown_d = nullptr, *nhalo_d = nullptr;
    SRDR_TRY(dalloc(b, &nown_d, nball));
    SRDR_TRY(dalloc(b, &nhalo_d, nball));
    k_brick_count<<<nblocks(nball), kThreads, 0, st>>>(b->cell_start, b->nc[0], b->nc[1], b->nc[2], d, nball,
                                                       nown_d, nhalo_d);
    std::vector<int> nown(nball), nhalo(nball);
    SRDR_CK(cudaMemcpyAsync(nown.data(), nown_d, sizeof(int) * nball, cudaMemcpyDeviceToHost, st));
    SRDR_CK(cudaMemcpyAsync(nhalo.data(), nhalo_d, sizeof(int) * nball, cudaMemcpyDeviceToHost, st));
    SRDR_CK(cudaStreamSynchronize(st));
    SRDR_TRY(dev_free(b, nown_d));
    SRDR_TRY(dev_free(b, nhalo_d));
    std::vector<BrickInfo> info;
    int64_t own = 0, halo = 0, slices = 0;
    int max_halo = 0, max_own = 0;
    for (int q = 0; q < nball; ++q) {
        if (nown[q] == 0) continue;
        BrickInfo bi{q, (int)own, (int)halo, (int)slices, nown[q], nhalo[q], 0, 0};
        info.push_back(bi);
        own += nown[q];
        halo += nhalo[q];
        slices += (nown[q] + 31) / 32;
        max_halo = std::max(max_halo, nhalo[q]);
        max_own = std::max(max_own, nown[q]);
    }
    const size_t smem = std::max(tile_smem_a(sizeof(T), max_halo), tile_smem_b(sizeof(T), dim, max_halo));
    if (own != b->n || halo > 0x7fffffffLL || max_halo >= 65536 || smem > kTileSmemMax) {
        b->bricks_built = -1;
        return SRDR_OK;
    }
    b->nbricks = (int)info.size();
    b->max_halo = max_halo;
    b->max_own = max_own;
    b->nbslices = (int)slices;
    SRDR_TRY(dalloc(b, &b->binfo, info.size()));
    SRDR_CK(cudaMemcpyAsync(b->binfo, info.data(), sizeof(BrickInfo) * info.size(), cudaMemcpyHostToDevice,
                            st));
    SRDR_TRY(dalloc(b, &b->bown, b->n));
    SRDR_TRY(dalloc(b, &b->bown_h, b->n));
    SRDR_TRY(dalloc(b, &b->bhalo, std::max<int64_t>(halo, 1)));
    const int nbk = b->nbricks;
    k_brick_fill<<<nbk, 128, 0, st>>>(b->binfo, b->cell_start, b->nc[0], b->nc[1], b->nc[2], d, b->bown,
                                      b->bown_h, b->bhalo);
    int *slots = nullptr, *tmp = nullptr;
    SRDR_TRY(dalloc(b, &slots, std::max<int64_t>(slices, 1)));
    SRDR_TRY(dalloc(b, &tmp, (slices + 1) / kScanBlock + 4));
    SRDR_TRY(dalloc(b, &b->bsell_ptr, slices + 1));
    k_bslice_width<<<nbk, 128, 0, st>>>(b->binfo, b->bown, b->row_ptr, slots);
    SRDR_TRY(scan_exclusive(slots, b->bsell_ptr, (int)slices, tmp, st));
    int nslots = 0;
    SRDR_CK(cudaMemcpyAsync(&nslots, b->bsell_ptr + slices, sizeof(int), cudaMemcpyDeviceToHost, st));
    SRDR_CK(cudaStreamSynchronize(st));
    if (nslots < 0) {
        set_error("brick sliced-ELL layout exceeds 2^31 slots");
        return SRDR_ERR_INVALID;
    }
    const int64_t ns = std::max(nslots, 1);
    b->bslots = ns;
    T* sg = nullptr;
    SRDR_TRY(dalloc(b, &b->blidx, ns));
    SRDR_TRY(dalloc(b, &sg, (size_t)ns * 3));
    b->bg = sg;
    const T rcT = (T)b->rc, ihT = (T)(1.0 / b->h), kcT = (T)kernel_kc(dim, b->h);
    if (dim == 2)
        k_bsell_fill<T, 2><<<nbk, 128, 0, st>>>(b->binfo, b->cell_start, b->nc[0], b->nc[1], b->nc[2], d,
                                                b->bown, b->bown_h, b->row_ptr, b->col, b->cell_of,
                                                b->bsell_ptr, static_cast<const T*>(b->cpos), b->ccell, rcT,
                                                ihT, kcT, b->blidx, sg, ns);
    else
        k_bsell_fill<T, 3><<<nbk, 128, 0, st>>>(b->binfo, b->cell_start, b->nc[0], b->nc[1], b->nc[2], d,
                                                b->bown, b->bown_h, b->row_ptr, b->col, b->cell_of,
                                                b->bsell_ptr, static_cast<const T*>(b->cpos), b->ccell, rcT,
                                                ihT, kcT, b->blidx, sg, ns);
    SRDR_CK(cudaGetLastError());
    SRDR_TRY(dalloc(b, &b->ke_pp, b->n));
    SRDR_CK(cudaStreamSynchronize(st));
    SRDR_TRY(dev_free(b, slots));
    SRDR_TRY(dev_free(b, tmp));
    b->bricks_built = 1;
    return SRDR_OK;
}

}  // namespace

srdr_status build_body(srdr_body* b, int64_t n, const double* r0, const double* vol,
                       const uint8_t* flags, const double* u0)
{
    if (n < 1 || n > 0x7fffffffLL / 3) {
        set_error("particle count %lld out of range", (long long)n);
        return SRDR_ERR_INVALID;
    }
    b->n = n;
    if (b->prec == SRDR_FP64) return build_typed<double>(b, n, r0, vol, flags, u0);
    return build_typed<float>(b, n, r0, vol, flags, u0);
}

template <typename T>
__global__ void k_sweep_consts(int n, T c, const T* __restrict__ mass, const T* __restrict__ sumw,
                               const T* __restrict__ sumw2, T* __restrict__ sbm, T* __restrict__ srd)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if constexpr (sizeof(T) == 4) {
        const float sb = __fmul_rn(c, sumw[i]), sb2 = __fmul_rn(__fmul_rn(c, c), sumw2[i]);
        const float d = __fsub_rn(sb, mass[i]);
        sbm[i] = d;
        srd[i] = __fdiv_rn(1.0f, __fmaf_rn(d, d, sb2));
    } else {
        const double sb = __dmul_rn(c, sumw[i]), sb2 = __dmul_rn(__dmul_rn(c, c), sumw2[i]);
        const double d = __dsub_rn(sb, mass[i]);
        sbm[i] = d;
        srd[i] = __ddiv_rn(1.0, __fma_rn(d, d, sb2));
    }
}

// slot records of the sweep: B = c w (one rounding, as the sweep would form
// it) and the footprint-local index; the two spare records after the last
// entry are zero (16-byte staging may read them)
template <typename T>
__global__ void k_sweep_slots(int64_t nnz, T c, const T* __restrict__ w, const uint16_t* __restrict__ loc,
                              SweepSlot<T>* __restrict__ rec)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nnz + 2) return;
    SweepSlot<T> r{};
    if (k < nnz) {
        if constexpr (sizeof(T) == 4)
            r.B = __fmul_rn(c, w[k]);
        else
            r.B = __dmul_rn(c, w[k]);
        r.loc = loc[k];
    }
    rec[k] = r;
}

template <typename T>
srdr_status prepare_sweep_typed(srdr_body* b)
{
    if (!b->sbm) {
        T *x = nullptr, *y = nullptr;
        SRDR_TRY(dalloc(b, &x, b->n));
        SRDR_TRY(dalloc(b, &y, b->n));
        b->sbm = x;
        b->srd = y;
        SweepSlot<T>* r = nullptr;
        SRDR_TRY(dalloc(b, &r, (size_t)b->nnz + 2));
        b->srec = r;
    }
    const T c = (T)(b->eta / b->desc.alpha * b->dt);
    k_sweep_consts<T><<<nblocks(b->n), kThreads, 0, b->stream>>>(
        (int)b->n, c, static_cast<const T*>(b->stencil ? b->mass_sw : b->mass), static_cast<const T*>(b->sumw),
        static_cast<const T*>(b->sumw2), static_cast<T*>(b->sbm), static_cast<T*>(b->srd));
    k_sweep_slots<T><<<nblocks(b->nnz + 2), kThreads, 0, b->stream>>>(
        b->nnz, c, static_cast<const T*>(b->w), b->loc, static_cast<SweepSlot<T>*>(b->srec));
    SRDR_CK(cudaGetLastError());
    return SRDR_OK;
}

srdr_status prepare_sweep(srdr_body* b)
{
    if (b->prec == SRDR_FP64) return prepare_sweep_typed<double>(b);
    return prepare_sweep_typed<float>(b);
}

srdr_status build_bricks(srdr_body* b)
{
    for (int a = 0; a < 3; ++a)
        if (b->brick[a] < 0 || b->brick[a] > 4) {
            set_error("brick size must be 1..4 cells (0: default)");
            return SRDR_ERR_INVALID;
        }
    if (b->prec == SRDR_FP64) return build_bricks_typed<double>(b);
    return build_bricks_typed<float>(b);
}

}  // namespace srdr
