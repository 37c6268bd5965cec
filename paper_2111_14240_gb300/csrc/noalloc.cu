// pmace_amplitude_energy_noalloc: the total measured energy sum_j ||y_j||^2
// without any device allocation.
//
// pmace_create computes this sum (it sets the energy-matched starting
// constant) with per-block partial sums in memory the job allocates.  This
// entry point computes the same sum for callers that cannot allocate device
// memory themselves: code running under a device-memory budget that another
// allocator owns (a framework's caching allocator, or a serving process that
// reserved all free HBM up front), and code that must not call cudaMalloc or
// cudaFree because those calls can synchronise the whole device.  The
// caller passes the amplitudes and a one-double output; the per-window
// partial sums live in a fixed array in the library's device image.
#include "pmace.h"
#include "pmace_internal.h"

#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstdio>
#include <mutex>

namespace {

// Largest number of windows one call accepts: one FP64 partial per window.
constexpr int kNoAllocMaxWindows = 65536;
constexpr int kEnergyThreads = 256;
constexpr int kMaxDevices = 64;

// Per-window partial sums.  Every GPU that loads the library holds these
// 512 KB until the process exits; all calls share them.
static __device__ __align__(256) double g_window_energy[kNoAllocMaxWindows];

// One CTA per window: the window's sum of y^2 in FP64, in a fixed order.
__global__ void __launch_bounds__(kEnergyThreads)
window_energy_kernel(const void* __restrict__ amps, int f16, const float* __restrict__ scales, int np,
                     double* __restrict__ partial) {
    const size_t P = (size_t)np * np;
    const size_t j = blockIdx.x;
    const float sc = f16 ? scales[j] : 1.0f;
    double s = 0.0;
    for (size_t e = threadIdx.x; e < P; e += kEnergyThreads) {
        const float v = f16 ? __half2float(static_cast<const __half*>(amps)[j * P + e]) * sc
                            : static_cast<const float*>(amps)[j * P + e];
        s += (double)v * (double)v;
    }
    __shared__ double red[kEnergyThreads];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = kEnergyThreads / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[j] = red[0];   // written, not accumulated: nothing to clear
}

// One CTA: out[0] = sum of the J partials, in a fixed order.
__global__ void __launch_bounds__(kEnergyThreads)
energy_total_kernel(const double* __restrict__ partial, int J, double* __restrict__ out) {
    double s = 0.0;
    for (int j = threadIdx.x; j < J; j += kEnergyThreads) s += partial[j];
    __shared__ double red[kEnergyThreads];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = kEnergyThreads / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[0] = red[0];
}

// Device address of g_window_energy on each device, looked up once per
// device with that device current (in host code the symbol itself is only a
// host-side stand-in and must not be handed to a kernel).
std::mutex g_setup_mutex;
double* g_scratch_addr[kMaxDevices] = {};

pmace_status fail(pmace_status st, const char* what) {
    pmace::set_unbound_error(what);
    return st;
}

}  // namespace

extern "C" pmace_status pmace_amplitude_energy_noalloc(const void* amps, pmace_amp_format fmt,
                                                        const float* scales, int32_t J, int32_t np,
                                                        double* out, void* stream) {
    pmace::set_unbound_error("");
    if (!amps || !out) return fail(PMACE_ERR_INVALID_ARG, "amps and out are required");
    if (fmt != PMACE_AMP_F32 && fmt != PMACE_AMP_F16_SCALED)
        return fail(PMACE_ERR_INVALID_ARG, "unknown amplitude format");
    if (fmt == PMACE_AMP_F16_SCALED && !scales)
        return fail(PMACE_ERR_INVALID_ARG, "FP16 amplitudes need per-pattern scales");
    if (np < 1 || J < 1) return fail(PMACE_ERR_INVALID_ARG, "J and np must be positive");
    if (J > kNoAllocMaxWindows) {
        char msg[160];
        snprintf(msg, sizeof msg, "J=%d exceeds the %d windows the fixed scratch of this entry point holds",
                 (int)J, kNoAllocMaxWindows);
        return fail(PMACE_ERR_INVALID_ARG, msg);
    }
    if ((size_t)np * (size_t)np > (size_t)1 << 30)
        return fail(PMACE_ERR_INVALID_ARG, "np too large");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(PMACE_ERR_CUDA, cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return fail(PMACE_ERR_CUDA, "device index out of range");
    double* scratch = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_setup_mutex);
        if (!g_scratch_addr[dev]) {
            e = cudaGetSymbolAddress(reinterpret_cast<void**>(&g_scratch_addr[dev]), g_window_energy);
            if (e != cudaSuccess) {
                g_scratch_addr[dev] = nullptr;
                return fail(PMACE_ERR_CUDA, cudaGetErrorString(e));
            }
        }
        scratch = g_scratch_addr[dev];
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    window_energy_kernel<<<J, kEnergyThreads, 0, s>>>(amps, fmt == PMACE_AMP_F16_SCALED, scales, np, scratch);
    e = cudaGetLastError();
    if (e != cudaSuccess) return fail(PMACE_ERR_CUDA, cudaGetErrorString(e));
    energy_total_kernel<<<1, kEnergyThreads, 0, s>>>(scratch, J, out);
    e = cudaGetLastError();
    if (e != cudaSuccess) return fail(PMACE_ERR_CUDA, cudaGetErrorString(e));
    return PMACE_OK;
}
