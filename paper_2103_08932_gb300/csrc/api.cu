// api.cu — the C ABI of include/srdr.h: body creation from a lattice
// description or explicit particles, stepping, relaxation to equilibrium,
// state read/write and build inspection.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <new>
#include <vector>

#include "srdr_internal.cuh"

namespace srdr {

static thread_local char g_err[512] = "";

void set_error(const char* fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

srdr_status dev_alloc(srdr_body* b, void** p, size_t bytes)
{
    *p = nullptr;
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        set_error("cudaMalloc(%zu bytes) failed: %s", bytes, cudaGetErrorString(e));
        return e == cudaErrorMemoryAllocation ? SRDR_ERR_NO_MEMORY : SRDR_ERR_CUDA;
    }
    b->allocs.push_back(*p);
    return SRDR_OK;
}

// zero the damping sweep's grid-barrier and cell-wise words (left mid-sweep
// by a wait that ran out)
srdr_status reset_sync_words(srdr_body* b)
{
    if (b->bar) SRDR_CK(cudaMemsetAsync(b->bar, 0, sizeof(unsigned) * kBarWords, b->stream));
    if (b->flow) SRDR_CK(cudaMemsetAsync(b->flow, 0, sizeof(unsigned) * flow_words(b->ncells), b->stream));
    SRDR_CK(cudaStreamSynchronize(b->stream));
    return SRDR_OK;
}

srdr_status dev_free(srdr_body* b, void* p)
{
    if (!p) return SRDR_OK;
    auto it = std::find(b->allocs.begin(), b->allocs.end(), p);
    if (it != b->allocs.end()) b->allocs.erase(it);
    SRDR_CK(cudaFree(p));
    return SRDR_OK;
}

void prof_begin(srdr_body* b, int k, cudaEvent_t* ev)
{
    (void)k;
    *ev = nullptr;
    if (!b->prof_active) return;
    if (b->ev_next >= b->ev_pool.size()) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return;
        b->ev_pool.push_back(e);
    }
    *ev = b->ev_pool[b->ev_next++];
    cudaEventRecord(*ev, b->stream);
}

void prof_end(srdr_body* b, int k, cudaEvent_t ev)
{
    if (!b->prof_active || !ev) return;
    if (b->ev_next >= b->ev_pool.size()) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return;
        b->ev_pool.push_back(e);
    }
    cudaEvent_t e2 = b->ev_pool[b->ev_next++];
    cudaEventRecord(e2, b->stream);
    b->ev_marks.push_back({k, {ev, e2}});
}

namespace {

// Lame constants from E and nu (E = 2 mu (1 + nu), E = 3 K (1 - 2 nu)).
void lame(double E, double nu, double* lambda, double* mu)
{
    *mu = E / (2.0 * (1.0 + nu));
    *lambda = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu));
}

srdr_status check_desc(const srdr_body_desc* d)
{
    if (!d) {
        set_error("desc is NULL");
        return SRDR_ERR_INVALID;
    }
    if (d->dim != 2 && d->dim != 3) {
        set_error("dim must be 2 or 3 (got %d)", d->dim);
        return SRDR_ERR_INVALID;
    }
    if (!(d->dp > 0) || !(d->rho0 > 0) || !(d->E > 0) || !(d->nu > -1.0 && d->nu < 0.5) ||
        !(d->h_over_dp > 0)) {
        set_error("dp, rho0, E, h_over_dp must be positive and -1 < nu < 0.5");
        return SRDR_ERR_INVALID;
    }
    if (d->material != SRDR_LINEAR_SVK && d->material != SRDR_NEO_HOOKEAN) {
        set_error("unknown material %d", d->material);
        return SRDR_ERR_INVALID;
    }
    if (d->precision != SRDR_FP64 && d->precision != SRDR_FP32_MIXED) {
        set_error("unknown precision %d", d->precision);
        return SRDR_ERR_INVALID;
    }
    if (d->damping < SRDR_DAMP_NONE || d->damping > SRDR_DAMP_EXPLICIT) {
        set_error("unknown damping scheme %d", d->damping);
        return SRDR_ERR_INVALID;
    }
    if (d->damping != SRDR_DAMP_NONE && !(d->alpha >= 0.0 && d->alpha <= 1.0)) {
        set_error("alpha must lie in [0, 1]");
        return SRDR_ERR_INVALID;
    }
    if (d->twist[0] != 0.0 && (d->dim != 3 || !(d->twist[1] > 0.0) || !std::isfinite(d->twist[0]) ||
                               !std::isfinite(d->twist[2]) || !std::isfinite(d->twist[3]))) {
        set_error("the twisting body force needs dim 3, a finite amplitude and axis, and L > 0");
        return SRDR_ERR_INVALID;
    }
    if (d->sweep_layout != SRDR_SWEEP_LAYOUT_3D && d->sweep_layout != SRDR_SWEEP_LAYOUT_2D) {
        set_error("unknown sweep layout %d", d->sweep_layout);
        return SRDR_ERR_INVALID;
    }
    if (d->pass_layout != SRDR_PASS_LAYOUT_AUTO && d->pass_layout != SRDR_PASS_LAYOUT_SELL) {
        set_error("unknown pass layout %d", d->pass_layout);
        return SRDR_ERR_INVALID;
    }
    return SRDR_OK;
}

// Box lattice of spacing dp in x-fastest order (the order srdr_body_create
// builds): lx points along x, then ly rows, then lz planes, every position
// within 1e-9 dp of r0[0] + (ix, iy, iz) dp and one volume.  Returns false
// for any other particle set.
bool detect_lattice(const srdr_body_desc* d, int64_t n, const double* r0, const double* vol, int lat[3])
{
    lat[0] = lat[1] = lat[2] = 0;
    if (n < 1 || n > INT32_MAX) return false;
    const int dim = d->dim;
    const double dp = d->dp, tol = 1e-9 * dp;
    auto same = [&](int64_t i, int64_t j, int a) { return std::fabs(r0[i * 3 + a] - r0[j * 3 + a]) <= tol; };
    int64_t nx = 1;
    while (nx < n && same(nx, 0, 1) && (dim == 2 || same(nx, 0, 2))) ++nx;
    int64_t np = nx;
    if (dim == 3)
        while (np < n && same(np, 0, 2)) ++np;
    else
        np = n;
    if (np % nx != 0 || n % np != 0) return false;
    const int64_t ny = np / nx, nz = n / np;
    if (dim == 2 && nz != 1) return false;
    for (int64_t i = 0; i < n; ++i) {
        const int64_t c[3] = {i % nx, (i / nx) % ny, i / np};
        for (int a = 0; a < dim; ++a)
            if (std::fabs(r0[i * 3 + a] - (r0[a] + (double)c[a] * dp)) > tol) return false;
        if (vol && vol[i] != vol[0]) return false;
    }
    lat[0] = (int)nx;
    lat[1] = (int)ny;
    lat[2] = (int)nz;
    return true;
}

// time step: 0.6 min(h / c, sqrt(h / |a|max)) with c = sqrt(K / rho0)
// (Eq. time-step-criterion at |v|max = 0), and the implicit viscous limit
// 50 h^2 / (nu~ D), nu~ = eta / (alpha rho0) (Eq. viscous-criteria).
// rotational body force of the twisting cantilever (the reading of Eq.
// rotation-body-force stated in srdr.h)
void twist_force(const srdr_body_desc& d, const double* r, double* g)
{
    const double gamma = d.twist[0] * sin(3.14159265358979323846 * r[0] / (2.0 * d.twist[1]));
    g[0] = 0.0;
    g[1] = -gamma * (r[2] - d.twist[3]);
    g[2] = gamma * (r[1] - d.twist[2]);
}

double auto_dt(const srdr_body* b, bool has_end_load, int64_t n, const double* r0, const uint8_t* flags)
{
    const srdr_body_desc& d = b->desc;
    double K = b->lambda + 2.0 * b->mu / 3.0;
    double c = sqrt(K / d.rho0);
    auto norm = [&](const double* x) {
        double s = 0;
        for (int a = 0; a < b->dim; ++a) s += x[a] * x[a];
        return sqrt(s);
    };
    double amax = norm(d.gravity);
    if (has_end_load) {
        double ge[3] = {d.gravity[0] + d.end_load[0], d.gravity[1] + d.end_load[1],
                        d.gravity[2] + d.end_load[2]};
        amax = std::max(amax, norm(ge));
    }
    if (d.twist[0] != 0.0) {
        // the largest |g + end load + g_t| over the particles
        for (int64_t i = 0; i < n; ++i) {
            double t[3], a[3];
            twist_force(d, r0 + i * 3, t);
            const bool end = flags && (flags[i] & SRDR_FLAG_END_LOAD);
            for (int k = 0; k < 3; ++k) a[k] = d.gravity[k] + (end ? d.end_load[k] : 0.0) + t[k];
            amax = std::max(amax, norm(a));
        }
    }
    double dt = b->h / c;
    if (amax > 0) dt = std::min(dt, sqrt(b->h / amax));
    dt *= 0.6;
    if (d.damping == SRDR_DAMP_EXPLICIT) {
        // Eq. viscous-criteria-o
        if (b->eta > 0) dt = std::min(dt, 0.5 * b->h * b->h / (b->eta / d.rho0 * b->dim));
    } else if (d.damping != SRDR_DAMP_NONE && d.alpha > 0 && b->eta > 0) {
        double nut = b->eta / (d.alpha * d.rho0);
        dt = std::min(dt, 50.0 * b->h * b->h / (nut * b->dim));
    }
    return dt;
}

srdr_status create_common(const srdr_body_desc* desc, int64_t n, const double* r0,
                          const double* vol, const uint8_t* flags, const double* u0, void* stream,
                          srdr_body** out)
{
    if (!out) {
        set_error("out is NULL");
        return SRDR_ERR_INVALID;
    }
    *out = nullptr;
    SRDR_TRY(check_desc(desc));
    if (!r0) {
        set_error("r0 is NULL");
        return SRDR_ERR_INVALID;
    }
    srdr_body* b = new (std::nothrow) srdr_body();
    if (!b) {
        set_error("host allocation failed");
        return SRDR_ERR_NO_MEMORY;
    }
    b->desc = *desc;
    b->dim = desc->dim;
    b->prec = desc->precision;
    b->stream = static_cast<cudaStream_t>(stream);
    b->h = desc->h_over_dp * desc->dp;
    b->cut = 2.0 * b->h;
    // the splitting cell-linked list: cells of edge r_c in 3^d colours (Sec.
    // 3.4), or of edge 2 r_c in 2^d colours (SRDR_SWEEP_LAYOUT_2D)
    b->cbase = desc->sweep_layout == SRDR_SWEEP_LAYOUT_2D ? 2 : 3;
    b->rc = desc->sweep_layout == SRDR_SWEEP_LAYOUT_2D ? 2.0 * b->cut : b->cut;
    b->vol0 = b->dim == 2 ? desc->dp * desc->dp : desc->dp * desc->dp * desc->dp;
    lame(desc->E, desc->nu, &b->lambda, &b->mu);
    b->eta = 0.25 * desc->beta * sqrt(desc->rho0 * desc->E) * desc->L_char;
    bool has_end = false;
    if (flags)
        for (int64_t i = 0; i < n && !has_end; ++i) has_end = (flags[i] & SRDR_FLAG_END_LOAD) != 0;
    b->dt = desc->dt > 0 ? desc->dt : auto_dt(b, has_end, n, r0, flags);
    if (desc->pass_layout == SRDR_PASS_LAYOUT_AUTO) detect_lattice(desc, n, r0, vol, b->lat);

    srdr_status st = dalloc(b, &b->sc, 1);
    if (st == SRDR_OK) {
        if (cudaMallocHost(&b->sc_host, sizeof(DevScalars)) != cudaSuccess) {
            b->sc_host = nullptr;
            set_error("pinned host allocation failed");
            st = SRDR_ERR_NO_MEMORY;
        }
    }
    if (st == SRDR_OK) {
        DevScalars z{};
        if (cudaMemcpyAsync(b->sc, &z, sizeof(z), cudaMemcpyHostToDevice, b->stream) != cudaSuccess ||
            cudaStreamSynchronize(b->stream) != cudaSuccess) {
            set_error("initialising device scalars failed");
            st = SRDR_ERR_CUDA;
        }
    }
    if (st == SRDR_OK) st = build_body(b, n, r0, vol, flags, u0);
    if (st != SRDR_OK) {
        srdr_body_destroy(b);
        return st;
    }
    *out = b;
    return SRDR_OK;
}

// lattice body of the description (the same particle order as documented
// in srdr.h: z outermost, y, x innermost)
void lattice(const srdr_body_desc* d, std::vector<double>& r0, std::vector<uint8_t>& flags,
             std::vector<double>& u0, bool& any_presc)
{
    int cnt[3] = {1, 1, 1}, lo[3] = {0, 0, 0}, hi[3] = {1, 1, 1};
    for (int a = 0; a < d->dim; ++a) {
        cnt[a] = (int)llround(d->extent[a] / d->dp);
        lo[a] = 0;
        hi[a] = cnt[a];
    }
    int ax = d->clamp_axis;
    if (ax >= 0 && ax < d->dim) {
        lo[ax] = -d->clamp_layers;
        hi[ax] = cnt[ax] + d->presc_layers;
    } else {
        ax = -1;
    }
    any_presc = ax >= 0 && d->presc_layers > 0;
    for (int z = lo[2]; z < hi[2]; ++z)
        for (int y = lo[1]; y < hi[1]; ++y)
            for (int x = lo[0]; x < hi[0]; ++x) {
                int ijk[3] = {x, y, z};
                double p[3] = {(x + 0.5) * d->dp, (y + 0.5) * d->dp, d->dim == 3 ? (z + 0.5) * d->dp : 0.0};
                uint8_t f = 0;
                double frac = 0.0;
                if (ax >= 0) {
                    int k = ijk[ax];
                    if (k < 0 || k >= cnt[ax]) f |= SRDR_FLAG_CONSTRAINED;
                    if (d->end_load_layer && k == cnt[ax] - 1) f |= SRDR_FLAG_END_LOAD;
                    if (any_presc) {
                        double length = cnt[ax] * d->dp;
                        frac = std::min(std::max(p[ax] / length, 0.0), 1.0);
                        if (k < 0) frac = 0.0;
                        if (k >= cnt[ax]) frac = 1.0;
                    }
                }
                for (int a = 0; a < 3; ++a) r0.push_back(p[a]);
                flags.push_back(f);
                for (int a = 0; a < 3; ++a)
                    u0.push_back(any_presc && a < d->dim ? frac * d->presc_disp[a] : 0.0);
            }
}

template <typename T>
__global__ void k_read_uv(const int* __restrict__ perm, int n, const double* __restrict__ u,
                          const float* __restrict__ uhi, const float* __restrict__ ulo,
                          const T* __restrict__ v, double half_dt, int what, double* __restrict__ out)
{
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    const int i = perm ? perm[s] : s;  // null: arrays in original order
    float hf[3] = {0, 0, 0}, lf[3] = {0, 0, 0};
    if (!u) {
        const float4 r = reinterpret_cast<const float4*>(uhi)[s];
        const float2 q = reinterpret_cast<const float2*>(ulo)[s];
        hf[0] = r.x;
        hf[1] = r.y;
        hf[2] = r.z;
        lf[0] = r.w;
        lf[1] = q.x;
        lf[2] = q.y;
    }
    for (int a = 0; a < 3; ++a) {
        double vv = (double)v[(size_t)s * 4 + a];
        double x;
        if (what == 0) {
            double uh = u ? u[(size_t)s * 4 + a] : (double)hf[a] + (double)lf[a];
            x = uh - half_dt * vv;  // u^n = u^{n+1/2} - dt/2 v^n
        } else {
            x = vv;
        }
        out[(size_t)i * 3 + a] = x;
    }
}

template <typename T>
__global__ void k_write_uv(const int* __restrict__ perm, int n, const double* __restrict__ uin,
                           const double* __restrict__ vin, double half_dt, double* __restrict__ u,
                           float* __restrict__ uhi, float* __restrict__ ulo, T* __restrict__ v)
{
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    const int i = perm ? perm[s] : s;  // null: arrays in original order
    float h[3] = {0, 0, 0}, l[3] = {0, 0, 0};
    for (int a = 0; a < 3; ++a) {
        double vv = vin ? vin[(size_t)i * 3 + a] : (double)v[(size_t)s * 4 + a];
        if (vin) v[(size_t)s * 4 + a] = (T)vv;
        if (uin) {
            double x = uin[(size_t)i * 3 + a] + half_dt * vv;  // u^{n+1/2}
            if (u) {
                u[(size_t)s * 4 + a] = x;
            } else {
                h[a] = (float)x;
                l[a] = (float)(x - (double)h[a]);
            }
        }
    }
    if (uin && !u) {
        reinterpret_cast<float4*>(uhi)[s] = make_float4(h[0], h[1], h[2], l[0]);
        reinterpret_cast<float2*>(ulo)[s] = make_float2(l[1], l[2]);
    }
}

template <typename T>
__global__ void k_read_field(const int* __restrict__ perm, int n, int dim, const T* __restrict__ src,
                             int aos_stride, double* __restrict__ out)
{
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    const int i = perm ? perm[s] : s;  // null: arrays in original order
    for (int p = 0; p < 3; ++p)
        for (int q = 0; q < 3; ++q) {
            double x = 0.0;
            if (p < dim && q < dim) {
                int k = p * dim + q;
                if (aos_stride > 0) {
                    // PB: entry k < F E in 16-byte chunk k / E (E = 16 /
                    // sizeof(T) entries per chunk, F whole chunks), chunk c
                    // of particle s at c n + s; leftover entry t = k - F E at
                    // T index (F E + t) n + s
                    const int E = 16 / (int)sizeof(T), F = pb_full(sizeof(T), dim);
                    x = k < F * E ? (double)src[((size_t)(k / E) * n + s) * E + k % E]
                                  : (double)src[(size_t)k * n + s];
                } else {
                    x = (double)src[(size_t)k * n + s];
                }
            }
            out[(size_t)i * 9 + p * 3 + q] = x;
        }
}

}  // namespace
}  // namespace srdr

using namespace srdr;

extern "C" {

const char* srdr_last_error(void) { return g_err; }

srdr_status srdr_body_create_particles(const srdr_body_desc* desc, int64_t n, const double* r0,
                                       const double* vol, const uint8_t* flags, const double* u0,
                                       void* cuda_stream, srdr_body** out)
{
    return create_common(desc, n, r0, vol, flags, u0, cuda_stream, out);
}

srdr_status srdr_body_create(const srdr_body_desc* desc, void* cuda_stream, srdr_body** out)
{
    SRDR_TRY(check_desc(desc));
    for (int a = 0; a < desc->dim; ++a)
        if (!(desc->extent[a] > 0) || llround(desc->extent[a] / desc->dp) < 1) {
            set_error("extent[%d] holds no lattice layer", a);
            return SRDR_ERR_INVALID;
        }
    std::vector<double> r0, u0;
    std::vector<uint8_t> flags;
    bool presc = false;
    lattice(desc, r0, flags, u0, presc);
    return create_common(desc, (int64_t)flags.size(), r0.data(), nullptr, flags.data(),
                         presc ? u0.data() : nullptr, cuda_stream, out);
}

void srdr_body_destroy(srdr_body* b)
{
    if (!b) return;
    if (b->stream) cudaStreamSynchronize(b->stream);
    else cudaDeviceSynchronize();
    if (b->graph) cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
    for (void* p : b->allocs) cudaFree(p);
    b->allocs.clear();
    for (cudaEvent_t e : b->ev_pool) cudaEventDestroy(e);
    b->ev_pool.clear();
    if (b->sc_host) cudaFreeHost(b->sc_host);
    delete b;
}

srdr_status srdr_body_step(srdr_body* b, int64_t nsteps)
{
    if (!b || nsteps < 0) {
        set_error("bad body or step count");
        return SRDR_ERR_INVALID;
    }
    SRDR_TRY(reset_scalars(b, 0.0));
    return launch_steps(b, nsteps);
}

srdr_status srdr_body_relax(srdr_body* b, double ke_ratio, int64_t max_steps, int64_t* steps_taken,
                            double* final_ke_ratio)
{
    if (!b || !(ke_ratio > 0) || max_steps < 0) {
        set_error("bad body, ratio or step cap");
        return SRDR_ERR_INVALID;
    }
    SRDR_TRY(reset_scalars(b, ke_ratio));
    const int64_t start = b->step;
    int64_t left = max_steps;
    int64_t chunk = 64;
    b->converged = 0;
    srdr_status result = SRDR_ERR_NOT_CONVERGED;
    while (left > 0) {
        int64_t k = std::min(left, chunk);
        SRDR_TRY(launch_steps(b, k));
        left -= k;
        SRDR_TRY(sync_scalars(b));
        b->step = b->sc_host->step;
        if (b->sc_host->status == DEV_TIMEOUT) {
            SRDR_TRY(reset_sync_words(b));
            set_error("a bounded wait of the damping sweep ran out (before step %lld)", (long long)b->step);
            result = SRDR_ERR_TIMEOUT;
            break;
        }
        if (b->sc_host->done) {
            if (b->sc_host->status == DEV_NONFINITE) {
                set_error("kinetic energy became non-finite at step %lld", (long long)b->step);
                result = SRDR_ERR_NONFINITE;
            } else {
                b->converged = 1;
                result = SRDR_OK;
            }
            break;
        }
        chunk = std::min<int64_t>(chunk * 2, 4096);
    }
    if (steps_taken) *steps_taken = b->step - start;
    if (final_ke_ratio)
        *final_ke_ratio = b->sc_host->ke_max > 0 ? b->sc_host->ke / b->sc_host->ke_max : 0.0;
    SRDR_TRY(reset_scalars(b, 0.0));
    if (result == SRDR_ERR_NOT_CONVERGED) set_error("no convergence in %lld steps", (long long)max_steps);
    return result;
}

static srdr_status read_uv(const srdr_body* b, double* out, size_t nd, int what)
{
    if (!b || !out || nd < (size_t)b->n * 3) {
        set_error("output buffer too small (need %lld doubles)", b ? (long long)b->n * 3 : 0LL);
        return SRDR_ERR_INVALID;
    }
    srdr_body* m = const_cast<srdr_body*>(b);
    double* d = nullptr;
    SRDR_TRY(dalloc(m, &d, (size_t)b->n * 3));
    int nb = (int)((b->n + 255) / 256);
    if (b->prec == SRDR_FP64)
        k_read_uv<double><<<nb, 256, 0, b->stream>>>(b->io_perm(), (int)b->n, b->u, nullptr, nullptr,
                                                     (const double*)b->v, 0.5 * b->dt, what, d);
    else
        k_read_uv<float><<<nb, 256, 0, b->stream>>>(b->io_perm(), (int)b->n, nullptr, b->uhi, b->ulo,
                                                    (const float*)b->v, 0.5 * b->dt, what, d);
    SRDR_CK(cudaGetLastError());
    SRDR_CK(cudaMemcpyAsync(out, d, sizeof(double) * 3 * b->n, cudaMemcpyDeviceToHost, b->stream));
    SRDR_CK(cudaStreamSynchronize(b->stream));
    return dev_free(m, d);
}

srdr_status srdr_body_read_displacement(const srdr_body* b, double* out, size_t nd)
{
    return read_uv(b, out, nd, 0);
}

srdr_status srdr_body_read_velocity(const srdr_body* b, double* out, size_t nd)
{
    return read_uv(b, out, nd, 1);
}

srdr_status srdr_body_write_state(srdr_body* b, const double* u, const double* v, int64_t step_index,
                                  double ke_max)
{
    if (!b) {
        set_error("body is NULL");
        return SRDR_ERR_INVALID;
    }
    size_t bytes = sizeof(double) * 3 * (size_t)b->n;
    double *du = nullptr, *dv = nullptr;
    if (u) {
        SRDR_TRY(dalloc(b, &du, (size_t)b->n * 3));
        SRDR_CK(cudaMemcpyAsync(du, u, bytes, cudaMemcpyHostToDevice, b->stream));
    }
    if (v) {
        SRDR_TRY(dalloc(b, &dv, (size_t)b->n * 3));
        SRDR_CK(cudaMemcpyAsync(dv, v, bytes, cudaMemcpyHostToDevice, b->stream));
    }
    int nb = (int)((b->n + 255) / 256);
    if (!u) {
        // keep u^n: rebuild the half step from the current state first
        double* cur = nullptr;
        SRDR_TRY(dalloc(b, &cur, (size_t)b->n * 3));
        if (b->prec == SRDR_FP64)
            k_read_uv<double><<<nb, 256, 0, b->stream>>>(b->io_perm(), (int)b->n, b->u, nullptr, nullptr,
                                                         (const double*)b->v, 0.5 * b->dt, 0, cur);
        else
            k_read_uv<float><<<nb, 256, 0, b->stream>>>(b->io_perm(), (int)b->n, nullptr, b->uhi, b->ulo,
                                                        (const float*)b->v, 0.5 * b->dt, 0, cur);
        du = cur;
    }
    if (b->prec == SRDR_FP64)
        k_write_uv<double><<<nb, 256, 0, b->stream>>>(b->io_perm(), (int)b->n, du, dv, 0.5 * b->dt, b->u,
                                                      nullptr, nullptr, (double*)b->v);
    else
        k_write_uv<float><<<nb, 256, 0, b->stream>>>(b->io_perm(), (int)b->n, du, dv, 0.5 * b->dt, nullptr,
                                                     b->uhi, b->ulo, (float*)b->v);
    SRDR_CK(cudaGetLastError());
    SRDR_CK(cudaStreamSynchronize(b->stream));
    SRDR_TRY(dev_free(b, du));
    SRDR_TRY(dev_free(b, dv));
    SRDR_TRY(sync_scalars(b));
    if (b->sc_host->status == DEV_TIMEOUT) SRDR_TRY(reset_sync_words(b));
    DevScalars s = *b->sc_host;
    s.step = step_index;
    s.ke_max = ke_max;
    s.done = 0;
    s.status = DEV_OK;
    SRDR_CK(cudaMemcpyAsync(b->sc, &s, sizeof(s), cudaMemcpyHostToDevice, b->stream));
    SRDR_CK(cudaStreamSynchronize(b->stream));
    b->step = step_index;
    return SRDR_OK;
}

srdr_status srdr_body_info(const srdr_body* b, int64_t* n, int64_t* nnz, int* ncells, double* dt)
{
    if (!b) {
        set_error("body is NULL");
        return SRDR_ERR_INVALID;
    }
    if (n) *n = b->n;
    if (nnz) *nnz = b->nnz;
    if (ncells) *ncells = b->ncells_nonempty;
    if (dt) *dt = b->dt;
    return SRDR_OK;
}

srdr_status srdr_body_stats(const srdr_body* b, srdr_stats* out)
{
    if (!b || !out) {
        set_error("body or out is NULL");
        return SRDR_ERR_INVALID;
    }
    SRDR_TRY(sync_scalars(b));
    out->step = b->sc_host->step;
    out->damped_steps = b->sc_host->damped;
    out->ke = b->sc_host->ke;
    out->ke_max = b->sc_host->ke_max;
    out->eta = b->eta;
    out->dt = b->dt;
    out->converged = b->converged;
    out->launches = b->launches;
    out->sweep_cells_per_warp = b->sweep_cells_per_warp;
    out->pass_mapping = b->stencil ? SRDR_PASS_STENCIL
                                   : (b->pass_tiled < 0 ? SRDR_PASS_AUTO
                                                        : (b->pass_tiled ? SRDR_PASS_BRICKS : SRDR_PASS_SELL));
    out->sweep_sync = !b->sweep_tuned ? SRDR_SWEEP_AUTO : (b->sweep_cellwise ? SRDR_SWEEP_CELLS : SRDR_SWEEP_BARRIER);
    return SRDR_OK;
}

srdr_status srdr_body_tune(srdr_body* b, int cells_per_warp, int warps_per_block)
{
    const bool autotune = cells_per_warp == 0 && warps_per_block == 0;
    const bool fixed = (cells_per_warp == 1 || cells_per_warp == 2 || cells_per_warp == 4) &&
                       (warps_per_block == 1 || warps_per_block == 4);
    if (!b || !(autotune || fixed)) {
        set_error("sweep mapping must be (0, 0) for the autotuner, or cells per warp 1, 2, 4 "
                  "and warps per block 1, 4");
        return SRDR_ERR_INVALID;
    }
    if (b->graph) {
        cudaGraphExecDestroy(b->graph);  // captured with the old mapping
        b->graph = nullptr;
    }
    if (autotune) {
        b->sweep_tuned = 0;
    } else {
        b->sweep_tuned = 1;
        b->sweep_cells_per_warp = cells_per_warp;
        b->sweep_warps_per_block = warps_per_block;
        b->sweep_chain16 = 0;
        // cell-wise waits pair with one cell per warp unless asked for
        b->sweep_cellwise = b->sweep_sync == SRDR_SWEEP_CELLS ||
                            (b->sweep_sync == SRDR_SWEEP_AUTO && cells_per_warp == 1);
    }
    return SRDR_OK;
}

srdr_status srdr_body_sweep_sync(srdr_body* b, int mode)
{
    if (!b || mode < SRDR_SWEEP_AUTO || mode > SRDR_SWEEP_CELLS) {
        set_error("sweep synchronisation must be SRDR_SWEEP_AUTO, SRDR_SWEEP_BARRIER or SRDR_SWEEP_CELLS");
        return SRDR_ERR_INVALID;
    }
    if (b->graph) {
        cudaGraphExecDestroy(b->graph);  // captured with the old kernel
        b->graph = nullptr;
    }
    b->sweep_sync = mode;
    if (mode == SRDR_SWEEP_AUTO)
        b->sweep_tuned = 0;
    else
        b->sweep_cellwise = mode == SRDR_SWEEP_CELLS;
    return SRDR_OK;
}

srdr_status srdr_body_sweep_lanes(srdr_body* b, int lanes)
{
    if (!b || (lanes != 0 && lanes != 16 && lanes != 32)) {
        set_error("sweep chain lanes must be 0 (autotuned), 16 or 32");
        return SRDR_ERR_INVALID;
    }
    if (lanes != 0 && b->sweep_sync == SRDR_SWEEP_BARRIER) {
        set_error("the chain width is a choice of the cell-wise sweep (the body asks for grid barriers)");
        return SRDR_ERR_INVALID;
    }
    if (b->graph) {
        cudaGraphExecDestroy(b->graph);  // captured with the old kernel
        b->graph = nullptr;
    }
    if (lanes == 0) {
        b->sweep_tuned = 0;
        return SRDR_OK;
    }
    b->sweep_tuned = 1;
    b->sweep_cells_per_warp = 1;
    b->sweep_cellwise = 1;
    b->sweep_chain16 = lanes == 16;
    return SRDR_OK;
}

srdr_status srdr_body_debug_stall_sweep(srdr_body* b)
{
    if (!b || !b->bar || !b->flow) {
        set_error("bad body");
        return SRDR_ERR_INVALID;
    }
    // a grid-barrier sub-counter that its last arrival never matches, and an
    // epoch far above every cell's count: every wait of the next sweep runs out
    const unsigned big = 0x40000000u;
    SRDR_CK(cudaMemcpyAsync(b->bar, &big, sizeof(unsigned), cudaMemcpyHostToDevice, b->stream));
    SRDR_CK(cudaMemcpyAsync(b->flow + flow_epoch_word(b->ncells), &big, sizeof(unsigned),
                            cudaMemcpyHostToDevice, b->stream));
    SRDR_CK(cudaStreamSynchronize(b->stream));
    return SRDR_OK;
}

srdr_status srdr_body_pass_mapping(srdr_body* b, int mapping, int bx, int by, int bz)
{
    if (!b || mapping < SRDR_PASS_AUTO || mapping > SRDR_PASS_STENCIL || bx < 0 || bx > 4 || by < 0 ||
        by > 4 || bz < 0 || bz > 4) {
        set_error("pass mapping must be SRDR_PASS_AUTO, _SELL, _BRICKS or _STENCIL with brick sizes 0..4");
        return SRDR_ERR_INVALID;
    }
    if (b->stencil != (mapping == SRDR_PASS_STENCIL) && mapping != SRDR_PASS_AUTO) {
        set_error(b->stencil ? "the body took the lattice stencil at creation (its arrays are in lattice "
                               "order): create it with pass_layout = SRDR_PASS_LAYOUT_SELL for this mapping"
                             : "the lattice stencil is chosen at creation (pass_layout = "
                               "SRDR_PASS_LAYOUT_AUTO, a box lattice)");
        return SRDR_ERR_INVALID;
    }
    if (b->stencil) return SRDR_OK;
    if (mapping == SRDR_PASS_BRICKS && b->desc.sweep_layout != SRDR_SWEEP_LAYOUT_3D) {
        set_error("brick-tiled passes need the 3^d-colour sweep layout (bricks of cells of edge r_c)");
        return SRDR_ERR_INVALID;
    }
    const bool resize = bx != b->brick[0] || by != b->brick[1] || bz != b->brick[2];
    if (resize && b->bricks_built != 0) {
        // drop the old layout; the next step that needs bricks rebuilds it
        for (void* p : {(void*)b->binfo, (void*)b->bown, (void*)b->bown_h, (void*)b->bhalo,
                        (void*)b->bsell_ptr, (void*)b->blidx, b->bg, (void*)b->ke_pp})
            SRDR_TRY(dev_free(b, p));
        b->binfo = nullptr;
        b->bown = nullptr;
        b->bown_h = nullptr;
        b->bhalo = nullptr;
        b->bsell_ptr = nullptr;
        b->blidx = nullptr;
        b->bg = nullptr;
        b->ke_pp = nullptr;
        b->bricks_built = 0;
    }
    if (b->graph) {
        cudaGraphExecDestroy(b->graph);  // captured with the old mapping
        b->graph = nullptr;
    }
    b->brick[0] = bx;
    b->brick[1] = by;
    b->brick[2] = bz;
    b->pass_mapping = mapping;
    b->pass_tiled = -1;
    return SRDR_OK;
}

srdr_status srdr_body_profile(srdr_body* b, int enable)
{
    if (!b) {
        set_error("body is NULL");
        return SRDR_ERR_INVALID;
    }
    if (enable) {
        SRDR_CK(cudaStreamSynchronize(b->stream));
        b->ev_marks.clear();
        b->ev_next = 0;
        for (int k = 0; k < SRDR_K_NCLASS; ++k) b->k_launch[k] = 0;
    }
    b->profiling = enable > 0 ? enable : 0;
    return SRDR_OK;
}

srdr_status srdr_body_kernel_times(const srdr_body* b, srdr_kernel_times* out)
{
    if (!b || !out) {
        set_error("body or out is NULL");
        return SRDR_ERR_INVALID;
    }
    SRDR_CK(cudaStreamSynchronize(b->stream));
    *out = srdr_kernel_times{};
    for (const auto& m : b->ev_marks) {
        float ms = 0.f;
        SRDR_CK(cudaEventElapsedTime(&ms, m.second.first, m.second.second));
        out->ms[m.first] += ms;
        out->intervals[m.first] += 1;
    }
    for (int k = 0; k < SRDR_K_NCLASS; ++k) out->launches[k] = b->k_launch[k];
    return SRDR_OK;
}

srdr_status srdr_body_read_neighbours(const srdr_body* b, int64_t* row_ptr, int64_t* col)
{
    if (!b || !row_ptr || !col) {
        set_error("NULL argument");
        return SRDR_ERR_INVALID;
    }
    int n = (int)b->n;
    std::vector<int> rp(n + 1), c(std::max<int64_t>(b->nnz, 1)), perm(n), inv(n);
    SRDR_CK(cudaStreamSynchronize(b->stream));
    SRDR_CK(cudaMemcpy(rp.data(), b->row_ptr, sizeof(int) * (n + 1), cudaMemcpyDeviceToHost));
    SRDR_CK(cudaMemcpy(c.data(), b->col, sizeof(int) * b->nnz, cudaMemcpyDeviceToHost));
    SRDR_CK(cudaMemcpy(perm.data(), b->perm, sizeof(int) * n, cudaMemcpyDeviceToHost));
    SRDR_CK(cudaMemcpy(inv.data(), b->inv, sizeof(int) * n, cudaMemcpyDeviceToHost));
    int64_t k = 0;
    for (int i = 0; i < n; ++i) {
        row_ptr[i] = k;
        int s = inv[i];
        int64_t a = k;
        for (int q = rp[s]; q < rp[s + 1]; ++q) col[k++] = perm[c[q]];
        std::sort(col + a, col + k);
    }
    row_ptr[n] = k;
    return SRDR_OK;
}

srdr_status srdr_body_read_cells(const srdr_body* b, int64_t* cell, int* colour, int64_t* order)
{
    if (!b || !cell || !colour || !order) {
        set_error("NULL argument");
        return SRDR_ERR_INVALID;
    }
    int n = (int)b->n;
    std::vector<int> cof(n), perm(n), inv(n);
    SRDR_CK(cudaStreamSynchronize(b->stream));
    SRDR_CK(cudaMemcpy(cof.data(), b->cell_of, sizeof(int) * n, cudaMemcpyDeviceToHost));
    SRDR_CK(cudaMemcpy(perm.data(), b->perm, sizeof(int) * n, cudaMemcpyDeviceToHost));
    SRDR_CK(cudaMemcpy(inv.data(), b->inv, sizeof(int) * n, cudaMemcpyDeviceToHost));
    auto col_of = [&](int c) {
        const int q = b->cbase;
        int cx = c % b->nc[0], cy = (c / b->nc[0]) % b->nc[1], cz = c / (b->nc[0] * b->nc[1]);
        return cx % q + (b->dim >= 2 ? q * (cy % q) : 0) + (b->dim >= 3 ? q * q * (cz % q) : 0);
    };
    for (int i = 0; i < n; ++i) {
        cell[i] = cof[inv[i]];
        colour[i] = col_of(cof[inv[i]]);
    }
    // sorted positions are ordered by (cell, id); a stable sort by colour
    // gives the sweep order (colour, cell, id)
    std::vector<int> pos(n);
    for (int s = 0; s < n; ++s) pos[s] = s;
    std::stable_sort(pos.begin(), pos.end(), [&](int x, int y) { return col_of(cof[x]) < col_of(cof[y]); });
    for (int s = 0; s < n; ++s) order[s] = perm[pos[s]];
    return SRDR_OK;
}

srdr_status srdr_body_read_field(const srdr_body* b, int field, double* out, size_t nd)
{
    if (!b || !out || nd < (size_t)b->n * 9 || (field != SRDR_FIELD_PB && field != SRDR_FIELD_B0)) {
        set_error("bad field request");
        return SRDR_ERR_INVALID;
    }
    srdr_body* m = const_cast<srdr_body*>(b);
    double* d = nullptr;
    SRDR_TRY(dalloc(m, &d, (size_t)b->n * 9));
    int nb = (int)((b->n + 255) / 256);
    const void* src = field == SRDR_FIELD_PB ? b->PB : b->B0;
    int stride = field == SRDR_FIELD_PB ? b->pb_stride : 0;
    if (b->prec == SRDR_FP64)
        k_read_field<double><<<nb, 256, 0, b->stream>>>(b->io_perm(), (int)b->n, b->dim,
                                                        (const double*)src, stride, d);
    else
        k_read_field<float><<<nb, 256, 0, b->stream>>>(b->io_perm(), (int)b->n, b->dim,
                                                       (const float*)src, stride, d);
    SRDR_CK(cudaGetLastError());
    SRDR_CK(cudaMemcpyAsync(out, d, sizeof(double) * 9 * b->n, cudaMemcpyDeviceToHost, b->stream));
    SRDR_CK(cudaStreamSynchronize(b->stream));
    return dev_free(m, d);
}

void srdr_philox4x64_10(const uint64_t counter[4], const uint64_t key[2], uint64_t out[4])
{
    philox4x64_10(counter, key, out);
}

double srdr_random_phi(uint64_t seed, uint64_t step) { return random_phi(seed, step); }

}  // extern "C"
