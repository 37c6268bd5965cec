// The fused agent sweep: steps S0-S5 of one PMACE iteration for every patch.
//
// For patch j (one cluster of C CTAs; CTA `rank` owns rows
// [rank*R, (rank+1)*R) of the Np x Np patch, R = Np/C) the kernel computes,
// entirely in shared memory and registers:
//   S0  v_j = q_j + 2 rho_prev P_j xbar   (closes the previous Mann step,
//       Algorithm 1: v <- v + 2 rho (z - w) with q = v - 2 rho w, z = P_j xbar)
//   S1  a = d . v_j
//   S2  A = F a                 (2-D DFT)
//   S3  A' = y_j A / |A|, 0 where A = 0   (Section III-A)
//   S4  w_j = (alpha v_j + D^-1 F^* A') / (1 + alpha)   (equation F-interpolate)
//   S5  u_j = 2 w_j - v_j (input of G), q_j <- v_j - 2 rho_cur w_j
// and per-CTA FP64 partial sums of |z - w|^2, |w|^2, (y - |A|)^2, y^2.
//
// Phases (Np threads per CTA):
//   copy-in  the CTA's amplitude rows go to shared memory with asynchronous
//            16-byte copies while every thread streams its element pairs of
//            q, xbar and d (16-byte loads, several pairs in flight), forms
//            a = d . v and stores it to the tile;
//   rows     each warp owns the rows r with r % warps == warp; the two
//            in-place row stages touch only the warp's own rows (__syncwarp);
//   columns  the column transform of length Np = C * R is one radix-C stage
//            across the cluster (distributed shared memory) and an R-point
//            DFT that each thread runs on its own column in registers,
//            together with the magnitude replacement and the inverse DFT;
//   copy-out the inverse row stages leave w's data term in the tile in
//            natural order; every thread then streams its element pairs of
//            q, xbar, 1/d and writes u and q (16-byte stores).
#pragma once

#include "fft_smem.cuh"
#include "pmace_internal.h"

#include <cuda_fp16.h>

namespace pmace {

namespace cg = cooperative_groups;

// Geometry of one plan: N x N probe, C CTAs per window, CPT columns per
// thread in the column step (N / CPT threads per CTA), YST = 1 to stage the
// amplitude rows in shared memory with asynchronous copies at kernel start
// (0: the column step loads them itself), PPC windows per cluster (every
// barrier then serves PPC windows).
template <int N, int C, int CPT, int YST, int PPC, int AMP>
struct AgentGeom {
    static constexpr int R = N / C;                 // rows per CTA = column DFT length
    static constexpr int RS = TileGeom<N>::RS;
    static constexpr int kThreads = N / CPT;
    static constexpr int kWarps = kThreads / 32;
    static constexpr int kTileBytes = PPC * R * RS * (int)sizeof(float2);
    static constexpr int kTwBytes = N * (int)sizeof(float2);
    static constexpr int kYBytes = YST ? PPC * R * N * (AMP ? 2 : 4) : 0;
    static constexpr int kSmem = kTileBytes + kTwBytes + kYBytes;
    static constexpr RadixPlan kRow = radix_plan(N);
    // resident CTAs per SM the shared memory allows (228 KB per SM, 1 KB
    // reserved per CTA plus the static reduction buffer), capped so that no
    // thread gets fewer than 96 registers
    static constexpr int kBySmem = (228 * 1024) / (kSmem + 2048);
    static constexpr int kByRegs = 65536 / (kThreads * 96);
    static constexpr int kMinBlocks = kBySmem < kByRegs ? (kBySmem > 0 ? kBySmem : 1) : kByRegs;
};

template <int AMP>
__device__ __forceinline__ float load_amp(const void* y, size_t idx, float scale) {
    if constexpr (AMP == 0) {
        return __ldg(static_cast<const float*>(y) + idx);
    } else {
        return __half2float(__ldg(static_cast<const __half*>(y) + idx)) * scale;
    }
}

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_addr(smem)), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// S3 for one spectrum coefficient A (unnormalised 2-D DFT): y A / |A|, 0
// where A = 0; coefficients whose squared magnitude would underflow are
// rescaled by 2^100 first.  With RES, also adds (y - |A|/Np)^2 and y^2 to
// the residual sums; the returned value is the same either way.
template <bool RES = true>
__device__ __forceinline__ float2 replace_magnitude(float2 xa, float y, float inv_n, float& acc_d, float& acc_y) {
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
        if constexpr (RES) mag = m2 * rs * unscale;
        o = xa * (y * rs);
    }
    if constexpr (RES) {
        const float e = y - mag;
        acc_d = fmaf(e, e, acc_d);
        acc_y = fmaf(y, y, acc_y);
    }
    return o;
}

// 1/sqrt(m) by the hardware approximation, for a normal m: there it is the
// value rsqrtf gives, without rsqrtf's handling of subnormal arguments.
__device__ __forceinline__ float rsqrt_normal(float m) {
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(m));
    return r;
}

// S3 for the R coefficients of one butterfly, with the arithmetic of
// replace_magnitude.  When every |A|^2 is at least 2^-100 (a normal number,
// so neither the rescaling nor the zero test applies) a coefficient costs
// its squared magnitude, one reciprocal square root and three
// multiplications; otherwise (rare: a coefficient that is tiny, zero or
// not finite) all R take the general path.
template <bool RES, int R>
__device__ __forceinline__ void replace_magnitudes(float2 (&x)[R], const float (&y)[R], float inv_n, float& acc_d,
                                                   float& acc_y) {
    float m2[R];
    bool general = false;
#pragma unroll
    for (int i = 0; i < R; ++i) {
        m2[i] = fmaf(x[i].x, x[i].x, x[i].y * x[i].y);
        general |= !(m2[i] >= 0x1p-100f);
    }
    if (general) {
#pragma unroll
        for (int i = 0; i < R; ++i) x[i] = replace_magnitude<RES>(x[i], y[i], inv_n, acc_d, acc_y);
        return;
    }
#pragma unroll
    for (int i = 0; i < R; ++i) {
        const float rs = rsqrt_normal(m2[i]);
        if constexpr (RES) {
            const float e = y[i] - m2[i] * rs * inv_n;
            acc_d = fmaf(e, e, acc_d);
            acc_y = fmaf(y[i], y[i], acc_y);
        }
        x[i] = x[i] * (y[i] * rs);
    }
}

// Window corner j of the job, checked against the image in the PMACE_DEBUG
// build (a corner outside [0, n1 - N] x [0, n2 - N] sets the bounds bit of
// the error word and is clamped into range).
template <int N>
__device__ __forceinline__ int2 window_corner(const AgentArgs& a, int j) {
    int2 off = a.offs[j];
#ifdef PMACE_DEBUG
    if (off.x < 0 || off.x > a.n1 - N || off.y < 0 || off.y > a.n2 - N) {
        atomicOr(a.err, kErrBoundsBit);
        off = make_int2(min(max(off.x, 0), a.n1 - N), min(max(off.y, 0), a.n2 - N));
    }
#endif
    return off;
}

// S0 for one pixel: v = q + 2 rho_prev xv (closes the previous Mann step).
__device__ __forceinline__ float2 mann_close(float2 q, float2 xv, float two_rho_prev) {
    return make_float2(fmaf(two_rho_prev, xv.x, q.x), fmaf(two_rho_prev, xv.y, q.y));
}

// S4 + S5 for one pixel: g = F^* A' unnormalised, v the agent input, dv =
// 1/d ((0, 0) where d is treated as absent).  w = (alpha v + D^-1 g / Np) /
// (1 + alpha) (w = v where d is absent); u = 2w - v; q' = v - 2 rho w.
// Returns w.
__device__ __forceinline__ float2 agent_step(float2 g, float2 v, float2 dv, float scale, float alpha, float inv1pa,
                                             float two_rho, float2& u, float2& qn) {
    float2 w;
    if (dv.x == 0.f && dv.y == 0.f) {
        w = v;                                    // d treated as absent here
    } else {
        const float2 h = cmul(dv, g * scale);     // D^-1 F^* A'
        w = make_float2(fmaf(alpha, v.x, h.x) * inv1pa, fmaf(alpha, v.y, h.y) * inv1pa);
    }
    u = make_float2(2.f * w.x - v.x, 2.f * w.y - v.y);
    qn = make_float2(fmaf(-two_rho, w.x, v.x), fmaf(-two_rho, w.y, v.y));
    return w;
}

// mann_close and agent_step with packed FP32 instructions (each lane
// rounded exactly as the scalar form); the constants come as lane pairs:
// trp2 = (2 rho_prev, 2 rho_prev), scale2 = (1/Np, 1/Np), alpha2, inv1pa2
// = (1/(1+alpha), 1/(1+alpha)), m2rho2 = (-2 rho, -2 rho).  CHECK: test
// for a probe value treated as absent (dv = 0) at this pixel; without it
// the caller knows there is none.
__device__ __forceinline__ float2 mann_close2(float2 q, float2 xv, float2 trp2) { return __ffma2_rn(trp2, xv, q); }
template <bool CHECK>
__device__ __forceinline__ float2 agent_step2(float2 g, float2 v, float2 dv, float2 scale2, float2 alpha2,
                                              float2 inv1pa2, float2 m2rho2, float2& u, float2& qn) {
    float2 w = __fmul2_rn(__ffma2_rn(alpha2, v, cmul(dv, __fmul2_rn(g, scale2))), inv1pa2);
    if constexpr (CHECK) {
        if (dv.x == 0.f && dv.y == 0.f) w = v;
    }
    u = __ffma2_rn(make_float2(2.f, 2.f), w, make_float2(-v.x, -v.y));
    qn = __ffma2_rn(m2rho2, w, v);
    return w;
}

// Residual sums of one pixel: |z - w|^2 and |w|^2 (z = v on the first
// iteration, else the consensus value).
__device__ __forceinline__ void residual_sums(float2 z, float2 w, float& az, float& aw) {
    const float dzx = z.x - w.x, dzy = z.y - w.y;
    az = fmaf(dzx, dzx, fmaf(dzy, dzy, az));
    aw = fmaf(w.x, w.x, fmaf(w.y, w.y, aw));
}

// Per-CTA sums of four FP32 per-thread partials: warp sums in FP32 (32
// terms), the warp totals added in FP64 in warp order by one thread.
template <int T>
__device__ __forceinline__ void block_reduce4(float (&acc)[4], double* red /* [T/32][4] */,
                                              double* out) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
        for (int i = 0; i < 4; ++i) acc[i] += __shfl_xor_sync(0xffffffffu, acc[i], o);
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) {
#pragma unroll
        for (int i = 0; i < 4; ++i) red[warp * 4 + i] = (double)acc[i];
    }
    __syncthreads();
    if (threadIdx.x < 4) {
        double s = 0.0;
        for (int w = 0; w < T / 32; ++w) s += red[w * 4 + threadIdx.x];
        out[threadIdx.x] = s;
    }
}

// Iterate over the butterflies of one row stage with radix RADIX that fall
// on the rows this warp owns: calls f(row, m) with m the butterfly index
// inside the row (N / RADIX per row).
template <int N, int NROWS, int NW, int RADIX, typename F>
__device__ __forceinline__ void for_warp_rows(F&& f) {
    constexpr int TPR = N / RADIX;              // threads per row
    static_assert(TPR <= 32 && 32 % TPR == 0, "a row stage must fit a warp");
    constexpr int RPI = 32 / TPR;               // rows per warp per step
    constexpr int ROWS_PER_WARP = NROWS / NW;
    static_assert(NROWS % NW == 0 && ROWS_PER_WARP % RPI == 0, "rows must split evenly over warps");
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
    for (int i = 0; i < ROWS_PER_WARP / RPI; ++i) {
        const int row = warp + NW * (i * RPI + lane / TPR);
        f(row, lane % TPR);
    }
}

// Element pairs (2p, 2p+1) of the CTA's rows, the unit of the copy phases:
// pair t = threadIdx.x + i*T covers row t / (N/2), columns 2 (t % (N/2)) + {0,1}.
template <int N, int NROWS, int T, int BATCH, typename F>
__device__ __forceinline__ void for_pairs(F&& f) {
    constexpr int PPT = NROWS * N / 2 / T;      // pairs per thread
    static_assert(PPT % BATCH == 0, "pairs must split into batches");
#pragma unroll 1
    for (int i0 = 0; i0 < PPT; i0 += BATCH) f(i0);
}

// The sweep of one cluster: windows j0 .. j0 + PPC - 1 of the job `a`.
template <int N, int C, int CPT, int YST, int PPC, int AMP>
__device__ __forceinline__ void agent_body(const AgentArgs& a, const int j0) {
    using G = AgentGeom<N, C, CPT, YST, PPC, AMP>;
    constexpr int R = G::R, RS = G::RS, T = G::kThreads, NW = G::kWarps;
    constexpr int r1 = G::kRow.first, r2 = G::kRow.second;
    constexpr int S1 = N / r1;
    constexpr int HALF = N / 2;
    constexpr int BATCH = 4;                       // element pairs in flight per thread, copy-in
    constexpr int BATCH_OUT = 4;                   // and copy-out
    constexpr int ROWS = PPC * R;                  // tile rows: PPC windows of R rows
    static_assert(r2 > 1, "row transform needs two stages");
    static_assert(R == 16 || R == 32, "column DFT length must be 16 or 32");
    static_assert(C == 1 || R % C == 0, "cross-CTA stage needs C | rows per CTA");

    extern __shared__ float4 smem_raw[];
    float2* tile = reinterpret_cast<float2*>(smem_raw);
    float2* tw = tile + ROWS * RS;
    char* ybuf = reinterpret_cast<char*>(tw + N);
    __shared__ double red[(T / 32) * 4];

    int rank = 0;
    if constexpr (C > 1) rank = (int)cg::this_cluster().block_rank();

    // window p of the cluster: j0 + p; it may lie past the end (J not a
    // multiple of PPC), in which case its rows are computed on zeros and
    // nothing of it is loaded or stored
    auto valid = [&](int p) { return j0 + p < a.J; };
    auto pbase_of = [&](int p) { return ((size_t)(j0 + p) * N + (size_t)rank * R) * N; };

    // ---- amplitude rows of this CTA -> shared memory, asynchronously
    if constexpr (YST) {
        constexpr int CH = G::kYBytes / PPC / 16;
#pragma unroll
        for (int p = 0; p < PPC; ++p) {
            if (!valid(p)) continue;
            const char* ysrc = static_cast<const char*>(a.y) + pbase_of(p) * (AMP ? 2 : 4);
            char* ydst = ybuf + p * (G::kYBytes / PPC);
            for (int c = threadIdx.x; c < CH; c += T) cp_async16(ydst + 16 * c, ysrc + 16 * c);
        }
        cp_async_commit();
    }
    for (int i = threadIdx.x; i < N; i += T) tw[i] = a.tw[i];
    const float2* __restrict__ pr = a.probe + (size_t)rank * R * N;
    const float2* __restrict__ di = a.dinv + (size_t)rank * R * N;
    const float two_rho_prev = 2.0f * a.rho_prev;

    // ---- S0 + S1: a = d . (q + 2 rho_prev xbar) into the tile, natural order
#pragma unroll
    for (int p = 0; p < PPC; ++p) {
        float2* tp = tile + p * R * RS;
        if (!valid(p)) {
            for (int e = threadIdx.x; e < R * RS; e += T) tp[e] = make_float2(0.f, 0.f);
            continue;
        }
        const int2 off = window_corner<N>(a, j0 + p);
        float2* qp = a.q + pbase_of(p);   // q in, v out: the copy-out reads v back (same thread, same pair)
        const float2* __restrict__ xb = a.xbar + (size_t)(off.x + rank * R) * a.n2 + off.y;
        for_pairs<N, R, T, BATCH>([&](int i0) {
            float4 qv[BATCH], dv[BATCH];
            float2 x0[BATCH], x1[BATCH];
#pragma unroll
            for (int i = 0; i < BATCH; ++i) {
                const int t = threadIdx.x + (i0 + i) * T;
                const int row = t / HALF, c = 2 * (t % HALF);
                qv[i] = *reinterpret_cast<const float4*>(qp + row * N + c);
                dv[i] = __ldg(reinterpret_cast<const float4*>(pr + row * N + c));
                x0[i] = __ldg(xb + (size_t)row * a.n2 + c);
                x1[i] = __ldg(xb + (size_t)row * a.n2 + c + 1);
            }
#pragma unroll
            for (int i = 0; i < BATCH; ++i) {
                const int t = threadIdx.x + (i0 + i) * T;
                const int row = t / HALF, c = 2 * (t % HALF);
                const float2 v0 = mann_close(make_float2(qv[i].x, qv[i].y), x0[i], two_rho_prev);
                const float2 v1 = mann_close(make_float2(qv[i].z, qv[i].w), x1[i], two_rho_prev);
                *reinterpret_cast<float4*>(qp + row * N + c) = make_float4(v0.x, v0.y, v1.x, v1.y);
                float2* dst = tp + row * RS + pcol(c);
                dst[0] = cmul(make_float2(dv[i].x, dv[i].y), v0);
                dst[1] = cmul(make_float2(dv[i].z, dv[i].w), v1);
            }
        });
    }
    __syncthreads();

    // ---- row DIF: span N (radix r1), then span r2, on the warp's own rows
    for_warp_rows<N, ROWS, NW, r1>([&](int row, int b) {
        float2* rp = tile + row * RS;
        float2 x[r1];
#pragma unroll
        for (int k = 0; k < r1; ++k) x[k] = rp[pcol(b + k * S1)];
        Dft<r1, false>::run(x);
#pragma unroll
        for (int k = 1; k < r1; ++k) x[k] = cmul(x[k], tw[b * k]);
#pragma unroll
        for (int k = 0; k < r1; ++k) rp[pcol(b + k * S1)] = x[k];
    });
    __syncwarp();
    for_warp_rows<N, ROWS, NW, r2>([&](int row, int m) {
        float2* rp = tile + row * RS;
        float2 x[r2];
#pragma unroll
        for (int k = 0; k < r2; ++k) x[k] = rp[pcol(m * r2 + k)];
        Dft<r2, false>::run(x);
#pragma unroll
        for (int k = 0; k < r2; ++k) rp[pcol(m * r2 + k)] = x[k];
    });

    // ---- column DIF, cross-CTA stage (span N, radix C)
    if constexpr (C > 1) {
        cg::cluster_group cl = cg::this_cluster();
        cl.sync();
        cross_stage<N, ROWS, R, C, false, T>(tile, tw, rank);
        if constexpr (YST) cp_async_wait_all();
        cl.sync();
    } else {
        if constexpr (YST) cp_async_wait_all();
        __syncthreads();
    }

    // ---- R-point column DFT in registers + S3 + inverse R-point DFT.
    // Thread `col` (CPT columns per thread) holds local rows 0..R-1 of its
    // column of window p; after the forward DFT register k2 holds frequency
    // row rank + C*k2, which is where the amplitudes were stored (kernel
    // order: row rank*R + k2).
    float acc_d[PPC], acc_y[PPC];
#pragma unroll
    for (int p = 0; p < PPC; ++p) {
        acc_d[p] = 0.f;
        acc_y[p] = 0.f;
        float yscale = 1.0f;
        if constexpr (AMP == 1) yscale = valid(p) ? __ldg(a.yscale + j0 + p) : 0.f;
        const size_t pb = pbase_of(p);
#pragma unroll 1
        for (int ci = 0; ci < CPT; ++ci) {
            const int col = threadIdx.x + ci * T;
            float yv[R];
#pragma unroll
            for (int k = 0; k < R; ++k) {
                if constexpr (YST) {
                    const char* yb = ybuf + p * (G::kYBytes / PPC);
                    if constexpr (AMP == 0) yv[k] = reinterpret_cast<const float*>(yb)[k * N + col];
                    else yv[k] = __half2float(reinterpret_cast<const __half*>(yb)[k * N + col]) * yscale;
                } else {
                    yv[k] = valid(p) ? load_amp<AMP>(a.y, pb + (size_t)k * N + col, yscale) : 0.f;
                }
            }
            float2* cp = tile + p * R * RS + pcol(col);
            float2 x[R];
#pragma unroll
            for (int k = 0; k < R; ++k) x[k] = cp[k * RS];
            Dft<R, false>::run(x);
            const float inv_n = 1.0f / (float)N;
            if (a.residual != 0) {
#pragma unroll
                for (int k = 0; k < R; ++k) x[k] = replace_magnitude<true>(x[k], yv[k], inv_n, acc_d[p], acc_y[p]);
            } else {
#pragma unroll
                for (int k = 0; k < R; ++k) x[k] = replace_magnitude<false>(x[k], yv[k], inv_n, acc_d[p], acc_y[p]);
            }
            Dft<R, true>::run(x);
#pragma unroll
            for (int k = 0; k < R; ++k) cp[k * RS] = x[k];
        }
    }

    // ---- column DIT, cross-CTA stage
    if constexpr (C > 1) {
        cg::cluster_group cl = cg::this_cluster();
        cl.sync();
        cross_stage<N, ROWS, R, C, true, T>(tile, tw, rank);
        cl.sync();   // also keeps every tile alive until the peers are done with it
    } else {
        __syncthreads();
    }

    // ---- row DIT: span r2, then span N; result back in the tile, natural order
    for_warp_rows<N, ROWS, NW, r2>([&](int row, int m) {
        float2* rp = tile + row * RS;
        float2 x[r2];
#pragma unroll
        for (int k = 0; k < r2; ++k) x[k] = rp[pcol(m * r2 + k)];
        Dft<r2, true>::run(x);
#pragma unroll
        for (int k = 0; k < r2; ++k) rp[pcol(m * r2 + k)] = x[k];
    });
    __syncwarp();
    for_warp_rows<N, ROWS, NW, r1>([&](int row, int b) {
        float2* rp = tile + row * RS;
        float2 x[r1];
#pragma unroll
        for (int k = 0; k < r1; ++k) x[k] = rp[pcol(b + k * S1)];
#pragma unroll
        for (int k = 1; k < r1; ++k) x[k] = cmulc(x[k], tw[b * k]);
        Dft<r1, true>::run(x);
#pragma unroll
        for (int k = 0; k < r1; ++k) rp[pcol(b + k * S1)] = x[k];
    });
    __syncthreads();

    // ---- S4 + S5, pair by pair
    float acc_z[PPC], acc_w[PPC];
    {
        const float scale = 1.0f / (float)N;          // orthonormal F^*
        const float inv1pa = 1.0f / (1.0f + a.alpha);
        const float alpha = a.alpha;
        const float two_rho = 2.0f * a.rho_cur;
        const bool first = a.first != 0;
        const bool res = a.residual != 0;
#pragma unroll
        for (int p = 0; p < PPC; ++p) {
            float az = 0.f, aw = 0.f;
            if (valid(p)) {
                const int2 off = window_corner<N>(a, j0 + p);
                float2* qp = a.q + pbase_of(p);   // v (written by the copy-in), overwritten by q' pair by pair by one thread
                float2* __restrict__ uo = a.u + pbase_of(p);
                const float2* __restrict__ xb = a.xbar + (size_t)(off.x + rank * R) * a.n2 + off.y;
                const float2* tp = tile + p * R * RS;
                for_pairs<N, R, T, BATCH_OUT>([&](int i0) {
                    float4 qv[BATCH_OUT], dv[BATCH_OUT];
                    float2 x0[BATCH_OUT], x1[BATCH_OUT];
#pragma unroll
                    for (int i = 0; i < BATCH_OUT; ++i) {
                        const int t = threadIdx.x + (i0 + i) * T;
                        const int row = t / HALF, c = 2 * (t % HALF);
                        qv[i] = *reinterpret_cast<const float4*>(qp + row * N + c);
                        dv[i] = __ldg(reinterpret_cast<const float4*>(di + row * N + c));
                        if (res) {   // the consensus values only feed the residual now
                            x0[i] = __ldg(xb + (size_t)row * a.n2 + c);
                            x1[i] = __ldg(xb + (size_t)row * a.n2 + c + 1);
                        }
                    }
#pragma unroll
                    for (int i = 0; i < BATCH_OUT; ++i) {
                        const int t = threadIdx.x + (i0 + i) * T;
                        const int row = t / HALF, c = 2 * (t % HALF);
                        const float2* src = tp + row * RS + pcol(c);
                        const float2 v0 = make_float2(qv[i].x, qv[i].y), v1 = make_float2(qv[i].z, qv[i].w);
                        float2 u0, u1, q0, q1;
                        const float2 w0 = agent_step(src[0], v0, make_float2(dv[i].x, dv[i].y), scale, alpha, inv1pa,
                                                     two_rho, u0, q0);
                        const float2 w1 = agent_step(src[1], v1, make_float2(dv[i].z, dv[i].w), scale, alpha, inv1pa,
                                                     two_rho, u1, q1);
                        if (res) {
                            residual_sums(first ? v0 : x0[i], w0, az, aw);
                            residual_sums(first ? v1 : x1[i], w1, az, aw);
                        }
                        *reinterpret_cast<float4*>(uo + row * N + c) = make_float4(u0.x, u0.y, u1.x, u1.y);
                        *reinterpret_cast<float4*>(qp + row * N + c) = make_float4(q0.x, q0.y, q1.x, q1.y);
                    }
                });
            }
            acc_z[p] = az;
            acc_w[p] = aw;
        }
    }
    if (a.residual == 0) return;      // only the residual iteration writes partial sums
#pragma unroll
    for (int p = 0; p < PPC; ++p) {
        float acc[4] = {acc_z[p], acc_w[p], acc_d[p], acc_y[p]};
        if (p > 0) __syncthreads();   // the reduction buffer is reused
        if (valid(p)) block_reduce4<T>(acc, red, a.partials + ((size_t)(j0 + p) * C + rank) * 4);
        else __syncthreads();         // keep the barrier count uniform
    }
}

// One job: cluster k processes windows k*PPC .. k*PPC + PPC - 1.
// MINB: resident CTAs per SM the register allocation is sized for.
template <int N, int C, int CPT, int YST, int PPC, int AMP, int MINB>
__global__ void __launch_bounds__(AgentGeom<N, C, CPT, YST, PPC, AMP>::kThreads, MINB)
agent_kernel(const __grid_constant__ AgentArgs a) {
    agent_body<N, C, CPT, YST, PPC, AMP>(a, (int)(blockIdx.x / C) * PPC);
}

// Several jobs in one launch: cluster k processes job work[k].x from window
// work[k].y on, with that job's arguments descs[work[k].x].
template <int N, int C, int CPT, int YST, int PPC, int AMP, int MINB>
__global__ void __launch_bounds__(AgentGeom<N, C, CPT, YST, PPC, AMP>::kThreads, MINB)
agent_kernel_batched(const AgentArgs* __restrict__ descs, const int2* __restrict__ work) {
    const int2 w = work[blockIdx.x / C];
    agent_body<N, C, CPT, YST, PPC, AMP>(descs[w.x], w.y);
}

template <int N, int C, int CPT, int YST, int PPC, int AMP, int MINB>
cudaError_t launch_agent_impl(const AgentArgs& a, cudaStream_t s) {
    using G = AgentGeom<N, C, CPT, YST, PPC, AMP>;
    void (*fn)(const AgentArgs) = agent_kernel<N, C, CPT, YST, PPC, AMP, MINB>;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, G::kSmem);
    if (e != cudaSuccess) return e;
    if constexpr (C > 1) {
        e = cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e != cudaSuccess) return e;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(((a.J + PPC - 1) / PPC) * C), 1, 1);
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

template <int N, int C, int CPT, int YST, int PPC, int AMP, int MINB>
cudaError_t launch_agent_batched_impl(const AgentArgs* descs, const int2* work, int nclusters, cudaStream_t s) {
    using G = AgentGeom<N, C, CPT, YST, PPC, AMP>;
    void (*fn)(const AgentArgs*, const int2*) = agent_kernel_batched<N, C, CPT, YST, PPC, AMP, MINB>;
    if (nclusters <= 0) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, G::kSmem);
    if (e != cudaSuccess) return e;
    if constexpr (C > 1) {
        e = cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e != cudaSuccess) return e;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(nclusters * C), 1, 1);
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
    return cudaLaunchKernelEx(&cfg, fn, descs, work);
}

// How many clusters of this plan the device holds at once (0: not launchable).
template <int N, int C, int CPT, int YST, int PPC, int AMP, int MINB>
int plan_max_clusters_impl() {
    using G = AgentGeom<N, C, CPT, YST, PPC, AMP>;
    void (*fn)(const AgentArgs) = agent_kernel<N, C, CPT, YST, PPC, AMP, MINB>;
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, G::kSmem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    if (C == 1) {
        int per_sm = 0, dev = 0, nsm = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, G::kThreads, G::kSmem) != cudaSuccess ||
            cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
            cudaGetLastError();
            return 0;
        }
        return per_sm * nsm;
    }
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
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
        return 0;
    }
    return nclusters;
}

// One plan, several jobs: `work` holds nclusters (job, first window) pairs.
template <int N, int C, int CPT, int YST, int PPC>
cudaError_t agent_variant_batched(const AgentArgs* descs, const int2* work, int nclusters, int amp_f16,
                                  cudaStream_t s) {
    if (amp_f16)
        return launch_agent_batched_impl<N, C, CPT, YST, PPC, 1, AgentGeom<N, C, CPT, YST, PPC, 1>::kMinBlocks>(
            descs, work, nclusters, s);
    return launch_agent_batched_impl<N, C, CPT, YST, PPC, 0, AgentGeom<N, C, CPT, YST, PPC, 0>::kMinBlocks>(
        descs, work, nclusters, s);
}

// One plan: query (a == nullptr) or launch, for either amplitude format.
template <int N, int C, int CPT, int YST, int PPC>
cudaError_t agent_variant(const AgentArgs* a, int amp_f16, cudaStream_t s, AgentPlanInfo* info) {
    if (amp_f16) {
        using G = AgentGeom<N, C, CPT, YST, PPC, 1>;
        if (a == nullptr) {
            info->threads = G::kThreads;
            info->smem_bytes = G::kSmem;
            info->max_clusters = plan_max_clusters_impl<N, C, CPT, YST, PPC, 1, G::kMinBlocks>();
            info->launchable = info->max_clusters > 0;
            return cudaSuccess;
        }
        return launch_agent_impl<N, C, CPT, YST, PPC, 1, G::kMinBlocks>(*a, s);
    }
    using G = AgentGeom<N, C, CPT, YST, PPC, 0>;
    if (a == nullptr) {
        info->threads = G::kThreads;
        info->smem_bytes = G::kSmem;
        info->max_clusters = plan_max_clusters_impl<N, C, CPT, YST, PPC, 0, G::kMinBlocks>();
        info->launchable = info->max_clusters > 0;
        return cudaSuccess;
    }
    return launch_agent_impl<N, C, CPT, YST, PPC, 0, G::kMinBlocks>(*a, s);
}

}  // namespace pmace
