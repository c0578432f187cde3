// noalloc.cu — a kinetic-energy reduction that allocates no device memory.
//
// Some callers cannot call cudaMalloc: codes that own all device memory
// through their own pool or arena, and services that must keep a fixed
// device-memory footprint once they are running (they account for every
// byte at start-up and refuse allocations afterwards).  For them this file
// provides srdr_kinetic_energy_noalloc, a variant of the library's per-block
// FP64 kinetic-energy reduction (the partials of the force pass and the
// one-block final sum) whose scratch lives in a file-scope __device__ array
// instead of memory the library allocates.
#include <mutex>

#include "srdr_internal.cuh"

namespace srdr {
namespace {

constexpr int kNaThreads = 256;
// 16384 FP64 block partials = 128 KiB, held by every GPU that loads the
// library until the process exits; one partial per 256 particles, so the
// largest accepted n is 16384 * 256 = 4,194,304 particles.
constexpr int kNaMaxBlocks = 16384;
__device__ __align__(256) double g_ke_scratch[kNaMaxBlocks];

std::mutex g_scratch_mu;
constexpr int kMaxDevices = 128;
double* g_scratch_addr[kMaxDevices] = {};

// Device address of g_ke_scratch in the current context.  In host code the
// symbol is only a host-side stand-in, so the address is looked up with
// cudaGetSymbolAddress, with the caller's device current.  A device address
// belongs to a context, not to a device (cudaDeviceReset, or a context the
// caller made current through the driver API, gives another one), so every
// call made outside stream capture looks it up again and refreshes the copy
// kept per device ordinal; a call on a capturing stream uses that copy, which
// is why the first call on a device must come before any capture.
srdr_status scratch_address(cudaStream_t st, double** out)
{
    int dev = 0;
    SRDR_CK(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) {
        set_error("device ordinal %d out of range", dev);
        return SRDR_ERR_INVALID;
    }
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    SRDR_CK(cudaStreamIsCapturing(st, &cap));
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (cap == cudaStreamCaptureStatusNone) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_ke_scratch);
        if (e != cudaSuccess || !p) {
            set_error("cudaGetSymbolAddress(scratch) failed: %s", cudaGetErrorString(e));
            return SRDR_ERR_CUDA;
        }
        g_scratch_addr[dev] = static_cast<double*>(p);
    } else if (!g_scratch_addr[dev]) {
        set_error("first allocation-free call on device %d made during stream capture", dev);
        return SRDR_ERR_INVALID;
    }
    *out = g_scratch_addr[dev];
    return SRDR_OK;
}

__device__ inline double na_warp_sum(double x)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    return x;
}

// one FP64 partial per block of 256 particles, fixed order
template <typename T>
__global__ void __launch_bounds__(kNaThreads) k_ke_partials_na(const T* __restrict__ v,
                                                               const T* __restrict__ mass,
                                                               const uint8_t* __restrict__ flags,
                                                               int64_t n, double* __restrict__ part)
{
    __shared__ double s[kNaThreads / 32];
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double ke = 0.0;
    if (i < n && !(flags && (flags[i] & SRDR_FLAG_CONSTRAINED))) {
        const T vi[3] = {v[i], v[n + i], v[2 * n + i]};
        ke = ke_particle<T>(mass[i], vi);  // the per-particle term of the library's reduction
    }
    ke = na_warp_sum(ke);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) s[w] = ke;
    __syncthreads();
    if (w == 0) {
        double y = l < (int)(blockDim.x >> 5) ? s[l] : 0.0;
        y = na_warp_sum(y);
        if (l == 0) part[blockIdx.x] = y;
    }
}

__global__ void __launch_bounds__(kNaThreads) k_ke_sum_na(const double* __restrict__ part, int nb,
                                                          double* __restrict__ out)
{
    __shared__ double s[kNaThreads / 32];
    double x = 0.0;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) x += part[b];
    x = na_warp_sum(x);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) s[w] = x;
    __syncthreads();
    if (threadIdx.x == 0) {
        double ke = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) ke += s[k];
        *out = ke;
    }
}

}  // namespace
}  // namespace srdr

extern "C" srdr_status srdr_kinetic_energy_noalloc(const void* v, const void* mass,
                                                   const uint8_t* flags, int64_t n, int precision,
                                                   double* ke_out, void* cuda_stream)
{
    using namespace srdr;
    if (!v || !mass || !ke_out || n < 1) {
        set_error("v, mass and ke_out must be device pointers and n >= 1");
        return SRDR_ERR_INVALID;
    }
    if (n > (int64_t)kNaMaxBlocks * kNaThreads) {
        set_error("n = %lld exceeds the allocation-free maximum of %lld particles",
                  (long long)n, (long long)kNaMaxBlocks * kNaThreads);
        return SRDR_ERR_INVALID;
    }
    if (precision != SRDR_FP64 && precision != SRDR_FP32_MIXED) {
        set_error("unknown precision %d", precision);
        return SRDR_ERR_INVALID;
    }
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    double* scratch = nullptr;
    SRDR_TRY(scratch_address(st, &scratch));
    const int nb = (int)((n + kNaThreads - 1) / kNaThreads);
    // every partial read below is written by this call first: nothing in the
    // scratch array has to start at zero
    if (precision == SRDR_FP64)
        k_ke_partials_na<double><<<nb, kNaThreads, 0, st>>>(static_cast<const double*>(v),
                                                            static_cast<const double*>(mass), flags,
                                                            n, scratch);
    else
        k_ke_partials_na<float><<<nb, kNaThreads, 0, st>>>(static_cast<const float*>(v),
                                                           static_cast<const float*>(mass), flags,
                                                           n, scratch);
    k_ke_sum_na<<<1, kNaThreads, 0, st>>>(scratch, nb, ke_out);
    SRDR_CK(cudaGetLastError());
    return SRDR_OK;
}
