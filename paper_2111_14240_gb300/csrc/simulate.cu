// Data simulator on the GPU: the forward model of Section II and the photon
// scaling of Section IV, so that measurements for a job can be made where
// the job runs instead of on the host.
//
//   intensity  I_j = |F D P_j x|^2, F the 2-D orthonormal DFT (DC at index 0);
//   amplitudes y_j = sqrt(I_j) without noise, else
//              y_j = sqrt(Pois(I_j r / M_j)) * sqrt(M_j / r), M_j = max of I_j
//              (y_j = 0 where M_j = 0), r the peak count.
//
// Kernels: a row pass and a column pass, each CTA holding 16 rows (or 16
// columns) of one window in shared memory and running the two DIF radix
// stages of the agent sweep's plan; the column pass writes the intensity in
// natural frequency order and takes the window maximum with an atomic max
// on the float bits (exact, order independent); a noise kernel draws the
// Poisson counts.  Random numbers: the counter-based generator Philox4x32-10
// (Salmon, Moraes, Dror, Shaw, SC 2011) from its published definition; draw
// n of pixel p of window j uses counter (p, j, n, 0x504d4143) and key (seed
// low, seed high), two 32-bit words (a, b) give the double ((a >> 5) 2^26 +
// (b >> 6)) / 2^53, two doubles per call.  Poisson sampling in FP64:
// Knuth's multiplication method below lambda = 10, W. Hoermann's
// transformed rejection with squeeze (PTRS, 1993) above; every FP64 step is
// written with round-to-nearest intrinsics, so no contraction into fused
// multiply-adds changes a decision.
#include "fft_smem.cuh"
#include "pmace.h"
#include "pmace_internal.h"

#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

namespace pmace {
namespace {

constexpr int kSimThreads = 128;
constexpr int kSimRows = 16;   // rows (columns) of a window per CTA
constexpr uint32_t kStreamTag = 0x504D4143u;

// ---------------------------------------------------------------------------
// Philox4x32-10 and the per-pixel uniform stream.
__device__ __forceinline__ void philox4x32_10(uint32_t (&c)[4], uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        const uint32_t hi0 = __umulhi(0xD2511F53u, c[0]), lo0 = 0xD2511F53u * c[0];
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c[2]), lo1 = 0xCD9E8D57u * c[2];
        const uint32_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
        c[0] = n0;
        c[1] = lo1;
        c[2] = n2;
        c[3] = lo0;
    }
}

__device__ __forceinline__ double words_to_double(uint32_t a, uint32_t b) {
    return ((double)(a >> 5) * 67108864.0 + (double)(b >> 6)) * (1.0 / 9007199254740992.0);
}

struct PixelStream {
    uint32_t p, j, n, k0, k1;
    double spare;
    bool have;
    __device__ double next() {
        if (have) {
            have = false;
            return spare;
        }
        uint32_t c[4] = {p, j, n, kStreamTag};
        philox4x32_10(c, k0, k1);
        ++n;
        spare = words_to_double(c[2], c[3]);
        have = true;
        return words_to_double(c[0], c[1]);
    }
};

__device__ double poisson_draw(double lam, PixelStream& s) {
    if (!(lam > 0.0)) return 0.0;
    if (lam < 10.0) {   // Knuth: uniforms multiplied while the product stays above exp(-lambda)
        const double lim = exp(-lam);
        double prod = 1.0, k = 0.0;
        for (int it = 0; it < 4096; ++it) {   // P(k >= 4096) is far below 1e-300 here
            prod = __dmul_rn(prod, s.next());
            if (!(prod > lim)) return k;
            k += 1.0;
        }
        return k;
    }
    // PTRS (Hoermann 1993)
    const double slam = __dsqrt_rn(lam), loglam = log(lam);
    const double b = __dadd_rn(0.931, __dmul_rn(2.53, slam));
    const double a = __dadd_rn(-0.059, __dmul_rn(0.02483, b));
    const double invalpha = __dadd_rn(1.1239, __ddiv_rn(1.1328, __dadd_rn(b, -3.4)));
    const double vr = __dadd_rn(0.9277, -__ddiv_rn(3.6224, __dadd_rn(b, -2.0)));
    const double log_invalpha = log(invalpha);
    for (int it = 0; it < (1 << 20); ++it) {   // acceptance is above 0.88 per try
        const double u = __dadd_rn(s.next(), -0.5);
        const double v = s.next();
        const double us = __dadd_rn(0.5, -fabs(u));
        const double kk =
            floor(__dadd_rn(__dadd_rn(__dmul_rn(__dadd_rn(__ddiv_rn(__dmul_rn(2.0, a), us), b), u), lam), 0.43));
        if (us >= 0.07 && v <= vr) return kk;
        if (kk < 0.0 || (us < 0.013 && v > us)) continue;
        const double lhs = __dadd_rn(__dadd_rn(log(v), log_invalpha), -log(__dadd_rn(__ddiv_rn(a, __dmul_rn(us, us)), b)));
        const double rhs = __dadd_rn(__dadd_rn(-lam, __dmul_rn(kk, loglam)), -lgamma(__dadd_rn(kk, 1.0)));
        if (lhs <= rhs) return kk;
    }
    return floor(lam);   // not reached in practice
}

// ---------------------------------------------------------------------------
// Row pass: CTA (window j, rows 16 rb .. 16 rb + 15): a = d . P_j x, the two
// DIF row stages; the rows go to the scratch stack in storage order.
template <int N>
__global__ void __launch_bounds__(kSimThreads) sim_rows_kernel(const float2* __restrict__ x, int n2,
                                                               const float2* __restrict__ probe,
                                                               const int2* __restrict__ offs,
                                                               const float2* __restrict__ tw_g, float2* __restrict__ S) {
    constexpr RadixPlan P = radix_plan(N);
    constexpr int r1 = P.first, r2 = P.second, S1 = N / r1, RS = TileGeom<N>::RS;
    __shared__ float2 tile[kSimRows * RS];
    __shared__ float2 tw[N];
    const int j = blockIdx.x / (N / kSimRows), row0 = (blockIdx.x % (N / kSimRows)) * kSimRows;
    const int2 off = offs[j];
    for (int i = threadIdx.x; i < N; i += kSimThreads) tw[i] = tw_g[i];
    for (int e = threadIdx.x; e < kSimRows * N; e += kSimThreads) {
        const int k = e / N, c = e % N;
        const float2 xv = __ldg(x + (size_t)(off.x + row0 + k) * n2 + off.y + c);
        tile[k * RS + pcol(c)] = cmul(__ldg(probe + (size_t)(row0 + k) * N + c), xv);
    }
    __syncthreads();
    for (int id = threadIdx.x; id < kSimRows * S1; id += kSimThreads) {
        const int k = id / S1, b = id % S1;
        float2 v[r1];
#pragma unroll
        for (int t = 0; t < r1; ++t) v[t] = tile[k * RS + pcol(b + S1 * t)];
        Dft<r1, false>::run(v);
#pragma unroll
        for (int t = 1; t < r1; ++t) v[t] = cmul(v[t], tw[b * t]);
#pragma unroll
        for (int t = 0; t < r1; ++t) tile[k * RS + pcol(b + S1 * t)] = v[t];
    }
    __syncthreads();
    for (int id = threadIdx.x; id < kSimRows * r1; id += kSimThreads) {
        const int k = id / r1, m = id % r1;
        float2 v[r2];
#pragma unroll
        for (int i = 0; i < r2; ++i) v[i] = tile[k * RS + pcol(m * r2 + i)];
        Dft<r2, false>::run(v);
#pragma unroll
        for (int i = 0; i < r2; ++i) tile[k * RS + pcol(m * r2 + i)] = v[i];
    }
    __syncthreads();
    float2* out = S + ((size_t)j * N + row0) * N;
    for (int e = threadIdx.x; e < kSimRows * N; e += kSimThreads) {
        const int k = e / N, c = e % N;
        out[(size_t)k * N + c] = tile[k * RS + pcol(c)];
    }
}

// Column pass: CTA (window j, storage columns 16 cb .. 16 cb + 15): the two
// DIF column stages, I = |A|^2 / Np^2 written at the natural frequencies
// (perm: storage index -> frequency), and the window maximum.
template <int N>
__global__ void __launch_bounds__(kSimThreads) sim_cols_kernel(const float2* __restrict__ S,
                                                               const float2* __restrict__ tw_g,
                                                               const int* __restrict__ perm,
                                                               float* __restrict__ inten,
                                                               unsigned* __restrict__ wmax) {
    constexpr RadixPlan P = radix_plan(N);
    constexpr int r1 = P.first, r2 = P.second, S1 = N / r1, CS = kSimRows + 1;
    __shared__ float2 col[N * CS];
    __shared__ float2 tw[N];
    __shared__ unsigned smax;
    const int j = blockIdx.x / (N / kSimRows), c0 = (blockIdx.x % (N / kSimRows)) * kSimRows;
    if (threadIdx.x == 0) smax = 0u;
    for (int i = threadIdx.x; i < N; i += kSimThreads) tw[i] = tw_g[i];
    const float2* in = S + (size_t)j * N * N + c0;
    for (int e = threadIdx.x; e < N * kSimRows; e += kSimThreads) {
        const int g = e / kSimRows, c = e % kSimRows;
        col[g * CS + c] = in[(size_t)g * N + c];
    }
    __syncthreads();
    for (int id = threadIdx.x; id < kSimRows * S1; id += kSimThreads) {
        const int c = id % kSimRows, b = id / kSimRows;
        float2 v[r1];
#pragma unroll
        for (int t = 0; t < r1; ++t) v[t] = col[(b + S1 * t) * CS + c];
        Dft<r1, false>::run(v);
#pragma unroll
        for (int t = 1; t < r1; ++t) v[t] = cmul(v[t], tw[b * t]);
#pragma unroll
        for (int t = 0; t < r1; ++t) col[(b + S1 * t) * CS + c] = v[t];
    }
    __syncthreads();
    const float norm = 1.0f / ((float)N * (float)N);
    float lmax = 0.f;
    float* out = inten + (size_t)j * N * N;
    for (int id = threadIdx.x; id < kSimRows * r1; id += kSimThreads) {
        const int c = id % kSimRows, m = id / kSimRows;
        float2 v[r2];
#pragma unroll
        for (int i = 0; i < r2; ++i) v[i] = col[(m * r2 + i) * CS + c];
        Dft<r2, false>::run(v);
        const int fc = __ldg(perm + c0 + c);
#pragma unroll
        for (int i = 0; i < r2; ++i) {
            const float I = fmaf(v[i].x, v[i].x, v[i].y * v[i].y) * norm;
            out[(size_t)__ldg(perm + m * r2 + i) * N + fc] = I;
            lmax = fmaxf(lmax, I);
        }
    }
    atomicMax(&smax, __float_as_uint(lmax));   // non-negative floats order like their bits
    __syncthreads();
    if (threadIdx.x == 0) atomicMax(wmax + j, smax);
}

// Window maxima of given intensities (non-negative floats).
__global__ void window_max_kernel(const float* __restrict__ inten, int64_t total, int P, unsigned* __restrict__ wmax) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x)
        atomicMax(wmax + i / P, __float_as_uint(fmaxf(inten[i], 0.f)));
}

// Amplitudes from intensities: sqrt(I), or the photon-scaled Poisson draw.
__global__ void photon_noise_kernel(const float* __restrict__ inten, int64_t total, int P,
                                    const unsigned* __restrict__ wmax, double peak, uint32_t k0, uint32_t k1,
                                    float* __restrict__ y) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const float I = inten[i];
        if (!(peak > 0.0)) {
            y[i] = sqrtf(I);
            continue;
        }
        const int j = (int)(i / P), p = (int)(i % P);
        const double M = (double)__uint_as_float(wmax[j]);
        if (!(M > 0.0)) {
            y[i] = 0.f;
            continue;
        }
        PixelStream s{(uint32_t)p, (uint32_t)j, 0u, k0, k1, 0.0, false};
        const double n = poisson_draw(__dmul_rn((double)I, __ddiv_rn(peak, M)), s);
        y[i] = (float)__dmul_rn(__dsqrt_rn(n), __dsqrt_rn(__ddiv_rn(M, peak)));
    }
}

template <int N>
cudaError_t launch_forward(const float2* x, int n2, const float2* probe, const int2* offs, const float2* tw,
                           const int* perm, int J, float2* S, float* inten, unsigned* wmax, cudaStream_t s) {
    const unsigned blocks = (unsigned)J * (N / kSimRows);
    sim_rows_kernel<N><<<blocks, kSimThreads, 0, s>>>(x, n2, probe, offs, tw, S);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    sim_cols_kernel<N><<<blocks, kSimThreads, 0, s>>>(S, tw, perm, inten, wmax);
    return cudaGetLastError();
}

unsigned noise_blocks(int64_t total) {
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>((total + 255) / 256, 152 * 32));
}

// Device buffers of one call, freed on every path.
struct Buffers {
    std::vector<void*> p;
    template <typename T>
    cudaError_t get(T** out, size_t count) {
        void* q = nullptr;
        cudaError_t e = cudaMalloc(&q, std::max<size_t>(count * sizeof(T), 16));
        if (e == cudaSuccess) p.push_back(q);
        *out = static_cast<T*>(q);
        return e;
    }
    ~Buffers() {
        for (void* q : p) cudaFree(q);
    }
};

pmace_status sim_fail(pmace_status st, const char* msg) {
    set_unbound_error(msg);
    return st;
}

pmace_status cuda_status(cudaError_t e) {
    set_unbound_error(cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? PMACE_ERR_OOM : PMACE_ERR_CUDA;
}

}  // namespace
}  // namespace pmace

using namespace pmace;

extern "C" {

pmace_status pmace_simulate(const pmace_dims* dims, const float* probe, const int32_t* offsets, const float* object,
                            double peak, uint64_t seed, float* amps_out, int on_device, void* stream) {
    if (!dims || !probe || !offsets || !object || !amps_out) return sim_fail(PMACE_ERR_INVALID_ARG, "NULL argument");
    const pmace_dims D = *dims;
    const int np = D.np, J = D.J;
    if (D.n1 <= 0 || D.n2 <= 0 || np <= 0 || J <= 0) return sim_fail(PMACE_ERR_INVALID_ARG, "sizes must be positive");
    if (np != 32 && np != 64 && np != 128 && np != 256)
        return sim_fail(PMACE_ERR_UNSUPPORTED_SIZE, "np not in {32, 64, 128, 256}");
    if (np > D.n1 || np > D.n2) return sim_fail(PMACE_ERR_INVALID_ARG, "np exceeds the image");
    if (!std::isfinite(peak)) return sim_fail(PMACE_ERR_INVALID_ARG, "peak must be finite");
    for (int j = 0; j < J; ++j) {
        const int r = offsets[2 * j], c = offsets[2 * j + 1];
        if (r < 0 || c < 0 || r > D.n1 - np || c > D.n2 - np)
            return sim_fail(PMACE_ERR_INVALID_ARG, "window offset out of range");
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const size_t P = (size_t)np * np, JP = (size_t)J * P, NI = (size_t)D.n1 * D.n2;
    const cudaMemcpyKind kin = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    // twiddles exp(-2 pi i m / np) from double, and the DIF storage order of
    // the two radix stages: position k r2 + p holds frequency k + r1 p
    std::vector<float2> tw(np);
    for (int m = 0; m < np; ++m) {
        const double ang = -2.0 * M_PI * (double)m / (double)np;
        tw[m] = make_float2((float)std::cos(ang), (float)std::sin(ang));
    }
    const RadixPlan rp = radix_plan(np);
    std::vector<int> perm(np);
    for (int k = 0; k < rp.first; ++k)
        for (int p = 0; p < rp.second; ++p) perm[k * rp.second + p] = k + rp.first * p;
    Buffers buf;
    float2 *x_d = nullptr, *probe_d = nullptr, *tw_d = nullptr, *S = nullptr;
    int2* offs_d = nullptr;
    int* perm_d = nullptr;
    float *inten = nullptr, *y_d = nullptr;
    unsigned* wmax = nullptr;
    cudaError_t e = buf.get(&S, JP);
    if (e == cudaSuccess) e = buf.get(&inten, JP);
    if (e == cudaSuccess) e = buf.get(&wmax, (size_t)J);
    if (e == cudaSuccess) e = buf.get(&tw_d, (size_t)np);
    if (e == cudaSuccess) e = buf.get(&perm_d, (size_t)np);
    if (e == cudaSuccess) e = buf.get(&offs_d, (size_t)J);
    if (e == cudaSuccess && !on_device) e = buf.get(&x_d, NI);
    if (e == cudaSuccess && !on_device) e = buf.get(&probe_d, P);
    if (e == cudaSuccess && !on_device) e = buf.get(&y_d, JP);
    if (e == cudaSuccess && !on_device) e = cudaMemcpyAsync(x_d, object, NI * sizeof(float2), kin, s);
    if (e == cudaSuccess && !on_device) e = cudaMemcpyAsync(probe_d, probe, P * sizeof(float2), kin, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(offs_d, offsets, (size_t)J * sizeof(int2), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(tw_d, tw.data(), np * sizeof(float2), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(perm_d, perm.data(), np * sizeof(int), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(wmax, 0, (size_t)J * sizeof(unsigned), s);
    const float2* xs = on_device ? reinterpret_cast<const float2*>(object) : x_d;
    const float2* ps = on_device ? reinterpret_cast<const float2*>(probe) : probe_d;
    if (e == cudaSuccess) {
        switch (np) {
            case 32: e = launch_forward<32>(xs, D.n2, ps, offs_d, tw_d, perm_d, J, S, inten, wmax, s); break;
            case 64: e = launch_forward<64>(xs, D.n2, ps, offs_d, tw_d, perm_d, J, S, inten, wmax, s); break;
            case 128: e = launch_forward<128>(xs, D.n2, ps, offs_d, tw_d, perm_d, J, S, inten, wmax, s); break;
            default: e = launch_forward<256>(xs, D.n2, ps, offs_d, tw_d, perm_d, J, S, inten, wmax, s); break;
        }
    }
    float* yo = on_device ? amps_out : y_d;
    if (e == cudaSuccess) {
        photon_noise_kernel<<<noise_blocks((int64_t)JP), 256, 0, s>>>(inten, (int64_t)JP, (int)P, wmax, peak,
                                                                      (uint32_t)seed, (uint32_t)(seed >> 32), yo);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess && !on_device) e = cudaMemcpyAsync(amps_out, y_d, JP * sizeof(float), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);   // the scratch is freed on return
    if (e != cudaSuccess) {
        cudaStreamSynchronize(s);
        return cuda_status(e);
    }
    return PMACE_OK;
}

pmace_status pmace_photon_noise(const float* intensity, int32_t J, int32_t np, double peak, uint64_t seed,
                                float* amps_out, int on_device, void* stream) {
    if (!intensity || !amps_out) return sim_fail(PMACE_ERR_INVALID_ARG, "NULL argument");
    if (J <= 0 || np <= 0) return sim_fail(PMACE_ERR_INVALID_ARG, "sizes must be positive");
    if (!std::isfinite(peak)) return sim_fail(PMACE_ERR_INVALID_ARG, "peak must be finite");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const size_t P = (size_t)np * np, JP = (size_t)J * P;
    Buffers buf;
    float *in_d = nullptr, *y_d = nullptr;
    unsigned* wmax = nullptr;
    cudaError_t e = buf.get(&wmax, (size_t)J);
    if (e == cudaSuccess && !on_device) e = buf.get(&in_d, JP);
    if (e == cudaSuccess && !on_device) e = buf.get(&y_d, JP);
    if (e == cudaSuccess && !on_device)
        e = cudaMemcpyAsync(in_d, intensity, JP * sizeof(float), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(wmax, 0, (size_t)J * sizeof(unsigned), s);
    const float* is = on_device ? intensity : in_d;
    float* yo = on_device ? amps_out : y_d;
    if (e == cudaSuccess) {
        window_max_kernel<<<noise_blocks((int64_t)JP), 256, 0, s>>>(is, (int64_t)JP, (int)P, wmax);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        photon_noise_kernel<<<noise_blocks((int64_t)JP), 256, 0, s>>>(is, (int64_t)JP, (int)P, wmax, peak,
                                                                      (uint32_t)seed, (uint32_t)(seed >> 32), yo);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess && !on_device) e = cudaMemcpyAsync(amps_out, y_d, JP * sizeof(float), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        cudaStreamSynchronize(s);
        return cuda_status(e);
    }
    return PMACE_OK;
}

}  // extern "C"
