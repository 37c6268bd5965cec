// The fused agent sweep: steps S0-S5 of one PMACE iteration for every patch.
//
// For patch j (one cluster of C CTAs; CTA `rank` owns rows
// [rank*Np/C, (rank+1)*Np/C) of the patch) the kernel computes, entirely in
// shared memory and registers:
//   S0  v_j = q_j + 2 rho_prev P_j xbar   (closes the previous Mann step,
//       Algorithm 1: v <- v + 2 rho (z - w) with q = v - 2 rho w, z = P_j xbar)
//   S1  a = d . v_j
//   S2  A = F a                 (2-D DFT, in-place DIF stages)
//   S3  A' = y_j A / |A|, 0 where A = 0   (Section III-A)
//   S4  w_j = (alpha v_j + D^-1 F^* A') / (1 + alpha)   (equation F-interpolate)
//   S5  u_j = 2 w_j - v_j (input of G), q_j <- v_j - 2 rho_cur w_j
// and per-CTA FP64 partial sums of |z - w|^2, |w|^2, (y - |A|)^2, y^2.
#pragma once

#include "fft_smem.cuh"
#include "pmace_internal.h"

#include <cuda_fp16.h>

namespace pmace {

namespace cg = cooperative_groups;

template <int N, int C>
struct AgentGeom {
    static constexpr int R = N / C;                 // rows per CTA
    static constexpr int RS = TileGeom<N>::RS;
    static constexpr int kThreads = (N == 32) ? 128 : 256;
    static constexpr int kSmem = (R * RS + N) * (int)sizeof(float2);
    static constexpr RadixPlan kRow = radix_plan(N);
    static constexpr RadixPlan kCol = radix_plan(R);  // local part of the column transform
};

template <int AMP>
__device__ __forceinline__ float load_amp(const void* y, size_t idx, float scale) {
    if constexpr (AMP == 0) {
        return __ldg(static_cast<const float*>(y) + idx);
    } else {
        return __half2float(__ldg(static_cast<const __half*>(y) + idx)) * scale;
    }
}

template <int T>
__device__ __forceinline__ void block_reduce4(float (&acc)[4], double* red /* [T/32][4] */,
                                              double* out) {
    double v[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) v[i] = (double)acc[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
        for (int i = 0; i < 4; ++i) v[i] += __shfl_xor_sync(0xffffffffu, v[i], o);
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) {
#pragma unroll
        for (int i = 0; i < 4; ++i) red[warp * 4 + i] = v[i];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double s[4] = {0, 0, 0, 0};
        for (int w = 0; w < T / 32; ++w) {
#pragma unroll
            for (int i = 0; i < 4; ++i) s[i] += red[w * 4 + i];
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) out[i] = s[i];
    }
}

template <int N, int C, int AMP>
__global__ void __launch_bounds__(AgentGeom<N, C>::kThreads)
agent_kernel(const AgentArgs a) {
    using G = AgentGeom<N, C>;
    constexpr int R = G::R, RS = G::RS, T = G::kThreads;
    constexpr int r1 = G::kRow.first, r2 = G::kRow.second;
    constexpr int c1 = G::kCol.first, c2 = G::kCol.second;
    constexpr int S1 = N / r1;
    static_assert(r2 > 1, "row transform needs two stages");
    static_assert(R % C == 0, "cross-CTA stage needs C | rows per CTA");

    extern __shared__ float4 smem_raw[];
    float2* tile = reinterpret_cast<float2*>(smem_raw);
    float2* tw = tile + R * RS;
    __shared__ double red[(T / 32) * 4];

    int rank = 0;
    if constexpr (C > 1) rank = (int)cg::this_cluster().block_rank();
    const int j = blockIdx.x / C;

    for (int i = threadIdx.x; i < N; i += T) tw[i] = a.tw[i];
    const int2 off = a.offs[j];
    const size_t pbase = ((size_t)j * N + (size_t)rank * R) * N;   // first element of my rows
    float2* qp = a.q + pbase;   // read (S0) and overwritten (S5) element by element by one thread
    float2* __restrict__ uo = a.u + pbase;
    const float2* __restrict__ xb = a.xbar + (size_t)(off.x + rank * R) * a.n2 + off.y;
    const float2* __restrict__ pr = a.probe + (size_t)rank * R * N;
    const float2* __restrict__ di = a.dinv + (size_t)rank * R * N;
    const size_t ybase = pbase;
    float yscale = 1.0f;
    if constexpr (AMP == 1) yscale = __ldg(a.yscale + j);
    const float two_rho_prev = 2.0f * a.rho_prev;
    __syncthreads();

    // ---- S0 + S1 + first row DIF stage (span N, radix r1), straight from HBM.
    for (int t = threadIdx.x; t < R * S1; t += T) {
        const int row = t / S1, b = t % S1;
        float2 x[r1];
#pragma unroll
        for (int k = 0; k < r1; ++k) {
            const int col = b + k * S1;
            const float2 qv = qp[row * N + col];
            const float2 xv = __ldg(xb + (size_t)row * a.n2 + col);
            const float2 v = make_float2(fmaf(two_rho_prev, xv.x, qv.x), fmaf(two_rho_prev, xv.y, qv.y));
            x[k] = cmul(__ldg(pr + row * N + col), v);
        }
        Dft<r1, false>::run(x);
#pragma unroll
        for (int k = 1; k < r1; ++k) x[k] = cmul(x[k], tw[b * k]);
        float2* rp = tile + row * RS;
#pragma unroll
        for (int k = 0; k < r1; ++k) rp[pcol(b + k * S1)] = x[k];
    }
    __syncthreads();
    // ---- rest of the row DIF (span r2)
    row_stage<N, R, r2, r2, false, T>(tile, tw);
    __syncthreads();

    // ---- column DIF: cross-CTA stage (span N, radix C), then local stages
    float2* peer[C];
    if constexpr (C > 1) {
        cg::cluster_group cl = cg::this_cluster();
#pragma unroll
        for (int k = 0; k < C; ++k) peer[k] = cl.map_shared_rank(tile, k);
        cl.sync();
        cross_stage<N, R, C, false, T>(peer, tw, rank);
        cl.sync();
    }
    if constexpr (c2 > 1) {
        col_stage<N, R, R, c1, false, T>(tile, tw);
        __syncthreads();
    }

    // ---- last column DIF stage + S3 magnitude replacement + first column DIT stage
    float acc_d = 0.f, acc_y = 0.f;
    {
        constexpr int rl = (c2 > 1) ? c2 : c1;
        constexpr int NB = (R / rl) * N;
        const float inv_n = 1.0f / (float)N;
        for (int t = threadIdx.x; t < NB; t += T) {
            const int col = t % N, rbase = (t / N) * rl;
            float2* cp = tile + pcol(col);
            float2 x[rl];
#pragma unroll
            for (int k = 0; k < rl; ++k) x[k] = cp[(rbase + k) * RS];
            Dft<rl, false>::run(x);
#pragma unroll
            for (int k = 0; k < rl; ++k) {
                const float yv = load_amp<AMP>(a.y, ybase + (size_t)(rbase + k) * N + col, yscale);
                // phase A/|A| (0 only where A = 0); coefficients whose squared
                // magnitude would underflow are rescaled by 2^100 first
                float2 xa = x[k];
                float m2 = fmaf(xa.x, xa.x, xa.y * xa.y);
                float unscale = inv_n;
                if (m2 < 0x1p-100f) {
                    xa = xa * 0x1p100f;
                    m2 = fmaf(xa.x, xa.x, xa.y * xa.y);
                    unscale = inv_n * 0x1p-100f;
                }
                float2 o = make_float2(0.f, 0.f);
                float mag = 0.f;
                if (m2 > 0.f) {
                    const float rs = rsqrtf(m2);
                    mag = m2 * rs * unscale;
                    o = xa * (yv * rs);
                }
                const float e = yv - mag;
                acc_d = fmaf(e, e, acc_d);
                acc_y = fmaf(yv, yv, acc_y);
                x[k] = o;
            }
            Dft<rl, true>::run(x);
#pragma unroll
            for (int k = 0; k < rl; ++k) cp[(rbase + k) * RS] = x[k];
        }
    }
    __syncthreads();

    // ---- column DIT: remaining local stage, then the cross-CTA stage
    if constexpr (c2 > 1) {
        col_stage<N, R, R, c1, true, T>(tile, tw);
        __syncthreads();
    }
    if constexpr (C > 1) {
        cg::cluster_group cl = cg::this_cluster();
        cl.sync();
        cross_stage<N, R, C, true, T>(peer, tw, rank);
        cl.sync();   // also keeps every tile alive until the peers are done with it
    }
    // ---- row DIT (span r2), then the last row stage fused with S4 + S5
    row_stage<N, R, r2, r2, true, T>(tile, tw);
    __syncthreads();

    float acc_z = 0.f, acc_w = 0.f;
    {
        const float scale = 1.0f / (float)N;          // orthonormal F^*
        const float inv1pa = 1.0f / (1.0f + a.alpha);
        const float alpha = a.alpha;
        const float two_rho = 2.0f * a.rho_cur;
        const bool first = a.first != 0;
        for (int t = threadIdx.x; t < R * S1; t += T) {
            const int row = t / S1, b = t % S1;
            const float2* rp = tile + row * RS;
            float2 x[r1];
#pragma unroll
            for (int k = 0; k < r1; ++k) x[k] = rp[pcol(b + k * S1)];
#pragma unroll
            for (int k = 1; k < r1; ++k) x[k] = cmulc(x[k], tw[b * k]);
            Dft<r1, true>::run(x);
#pragma unroll
            for (int k = 0; k < r1; ++k) {
                const int col = b + k * S1;
                const int e = row * N + col;
                const float2 qv = qp[e];
                const float2 xv = __ldg(xb + (size_t)row * a.n2 + col);
                const float2 v = make_float2(fmaf(two_rho_prev, xv.x, qv.x), fmaf(two_rho_prev, xv.y, qv.y));
                const float2 dv = __ldg(di + e);
                float2 w;
                if (dv.x == 0.f && dv.y == 0.f) {
                    w = v;                                    // d treated as absent here
                } else {
                    const float2 g = cmul(dv, x[k] * scale);  // D^-1 F^* A'
                    w = make_float2(fmaf(alpha, v.x, g.x) * inv1pa, fmaf(alpha, v.y, g.y) * inv1pa);
                }
                const float2 uu = make_float2(2.f * w.x - v.x, 2.f * w.y - v.y);
                const float2 qn = make_float2(fmaf(-two_rho, w.x, v.x), fmaf(-two_rho, w.y, v.y));
                const float2 z = first ? v : xv;
                const float dzx = z.x - w.x, dzy = z.y - w.y;
                acc_z = fmaf(dzx, dzx, fmaf(dzy, dzy, acc_z));
                acc_w = fmaf(w.x, w.x, fmaf(w.y, w.y, acc_w));
                uo[e] = uu;
                qp[e] = qn;
            }
        }
    }
    float acc[4] = {acc_z, acc_w, acc_d, acc_y};
    block_reduce4<T>(acc, red, a.partials + ((size_t)j * C + rank) * 4);
}

template <int N, int C>
cudaError_t launch_agent_impl(const AgentArgs& a, int amp_f16, cudaStream_t s) {
    using G = AgentGeom<N, C>;
    void (*fn)(const AgentArgs) = amp_f16 ? agent_kernel<N, C, 1> : agent_kernel<N, C, 0>;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, G::kSmem);
    if (e != cudaSuccess) return e;
    if constexpr (C > 1) {
        e = cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e != cudaSuccess) return e;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(a.J * C), 1, 1);
    cfg.blockDim = dim3(G::kThreads, 1, 1);
    cfg.dynamicSmemBytes = G::kSmem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, fn, a);
}

template <int N, int C>
bool plan_launchable_impl();

template <int N, int C>
cudaError_t agent_entry_impl(const AgentArgs* a, int amp_f16, cudaStream_t s, AgentPlanInfo* info) {
    using G = AgentGeom<N, C>;
    if (a == nullptr) {
        if (info) {
            info->threads = G::kThreads;
            info->smem_bytes = G::kSmem;
            info->launchable = plan_launchable_impl<N, C>() ? 1 : 0;
        }
        return cudaSuccess;
    }
    return launch_agent_impl<N, C>(*a, amp_f16, s);
}

template <int N, int C>
bool plan_launchable_impl() {
    using G = AgentGeom<N, C>;
    void (*fn)(const AgentArgs) = agent_kernel<N, C, 0>;
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, G::kSmem) != cudaSuccess)
        return false;
    if (C == 1) return true;
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess)
        return false;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(C * 64), 1, 1);
    cfg.blockDim = dim3(G::kThreads, 1, 1);
    cfg.dynamicSmemBytes = G::kSmem;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int nclusters = 0;
    if (cudaOccupancyMaxActiveClusters(&nclusters, fn, &cfg) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return nclusters > 0;
}

}  // namespace pmace
