// The fused agent sweep (steps S0-S5 of one PMACE iteration, the same
// arithmetic as agent.cuh) with the 2-D DFT split over a cluster by a
// transposing exchange instead of an in-place cross-CTA stage.
//
// A window is Np x Np; its cluster has C = Np / 16 CTAs.  CTA `rank` holds
// two 16 Np-element slabs in shared memory:
//   A  window rows [16 rank, 16 rank + 16), all Np columns (row slab);
//   B  all Np rows of storage columns [16 rank, 16 rank + 16) (column slab).
// Both are stored as C blocks of 16 x 16 elements; block p of A holds
// columns [16 p, 16 p + 16) of the CTA's rows, block r of B holds rows
// [16 r, 16 r + 16) of the CTA's columns, and inside a block element
// (k, c) sits at k * 17 + c (rows padded to 17 elements, 2176 bytes a
// block).  Every access pattern of the radix stages is then free of bank
// conflicts, and each address is a per-thread base plus a constant.  Block
// p of A is exactly block `rank` of CTA p's B, so one bulk copy per peer
// moves the row slabs into the column slabs, and one per peer moves them
// back.
//
// Per window:
//   rows   copy-in fused with the first (span Np) DIF row stage, in
//          registers; second row stage in A;
//   A -> B bulk copies (cp.async.bulk shared::cta -> shared::cluster), each
//          counted on the receiving CTA's mbarrier; where a warp's
//          second-stage butterflies cover whole blocks (Np >= 64) the warp
//          sends them as soon as it has written them;
//   cols   first DIF column stage in B; second column stage, magnitude
//          replacement (S3) and the inverse second stage in registers;
//          inverse first column stage in B;
//   B -> A bulk copies back;
//   rows   inverse second row stage in A; inverse first row stage fused
//          with the agent update and the stores of u and q (S4, S5).
//
// No cluster-wide barrier is needed between windows: a CTA sends block p of
// a slab only after it has received everything it needs from the previous
// exchange, and every CTA receives a block into exactly the region whose
// previous contents it has already sent on, so the mbarrier of the
// receiving slab is the only synchronisation (see the ordering notes at
// the sends).  A cluster processes a contiguous run of windows; it meets
// at the hardware cluster barrier once, after the barrier initialisation at
// kernel start, which every CTA reaches before any data moves.  Every later
// wait is bounded in polls and clock cycles.  A wait that gives up sets bit
// 2 of *err (the host reports PMACE_ERR_TIMEOUT); the CTA's threads agree at
// the next block barrier and stop: no further bulk copy is sent and the
// remaining windows are skipped.  The end of a run is an all-to-all arrival
// on a third mbarrier per CTA with a bounded wait: a CTA leaves only when
// every CTA of the cluster has passed its last receive wait or stopped.
#pragma once

#include "agent.cuh"
#include "cache_hints.cuh"
#include "tmem.cuh"

#include <type_traits>


namespace pmace {

template <int N>
struct XposeGeom {
    static constexpr int R = 16;                    // rows (and columns) per CTA
    static constexpr int C = N / R;                 // CTAs per window
    static constexpr int kThreads = N;
    static constexpr int kBlk = R * (R + 1);        // elements per exchange block (rows padded to 17)
    static constexpr int kSlab = C * kBlk;          // elements per slab (17 N)
    static constexpr int kBlkBytes = kBlk * (int)sizeof(float2);
    static constexpr RadixPlan kRad = radix_plan(N);
    static constexpr int r1 = kRad.first, r2 = kRad.second;
    static constexpr int S1 = N / r1;               // stride of the first stage (= r2)
    static constexpr int NB1 = R * S1;              // first-stage butterflies per slab
    static constexpr int NB2 = R * r1;              // second-stage butterflies per slab
    // first-stage twiddles: one row of r1 values per butterfly, padded to
    // kTwP elements (16-byte aligned rows; the 16-byte loads of the S1 rows
    // fall in distinct banks)
    static constexpr int kTwP = r1 + 2;
    static constexpr int kTwElems = S1 * kTwP;
    static constexpr int kSmem = 2 * kSlab * (int)sizeof(float2) + kTwElems * (int)sizeof(float2) + 32;
    // resident CTAs per SM: shared memory (228 KB, 1 KB reserved per CTA plus
    // the static reduction buffer), threads, and at least kRegFloor
    // registers a thread.  For 128 x 128 windows 96 registers (5 CTAs) keep
    // every value in registers; with 80 (6 CTAs) some spill to local memory,
    // which missed L1 and made the sweep 4 % slower.
    static constexpr int kRegFloor = N == 128 ? 96 : 64;
    static constexpr int kBySmem = (228 * 1024) / (kSmem + 2048);
    static constexpr int kByThreads = 2048 / kThreads;
    static constexpr int kByRegs = 65536 / (kThreads * kRegFloor);
    static constexpr int kMinBlocks0 = kBySmem < kByThreads ? kBySmem : kByThreads;
    static constexpr int kMinBlocks = kMinBlocks0 < kByRegs ? kMinBlocks0 : kByRegs;
    // the dynamic shared memory a launch asks for: padded so that no more
    // than kMinBlocks CTAs share an SM, which bounds the TMEM they allocate
    static constexpr int kSmemLaunch0 = (228 * 1024) / (kMinBlocks + 1) - 1024 + 64;
    static constexpr int kSmemLaunch = kSmem > kSmemLaunch0 ? kSmem : kSmemLaunch0;
    static_assert((kMinBlocks + 1) * (kSmemLaunch + 1024) > 228 * 1024, "one more CTA must not fit an SM");
    // (1 KB reserved per CTA, at most 320 bytes of static shared memory)
    static_assert(kMinBlocks * (kSmemLaunch + 1024 + 320) <= 228 * 1024, "kMinBlocks CTAs must fit an SM");
    static_assert(r1 * r2 == N && r2 > 1, "two radix stages per axis");
    static_assert(NB1 % kThreads == 0 && NB2 % kThreads == 0, "stages must split evenly over threads");
    static_assert(C >= 2 && C <= 16, "one block per CTA of the cluster");
    static_assert(kBlkBytes % 16 == 0, "bulk copies move multiples of 16 bytes between 16-byte aligned blocks");
    static_assert(S1 * r1 == N, "one twiddle table entry per (stage output, butterfly)");
    static_assert(S1 <= 16 && 16 % r2 == 0, "stage offsets split into a base and a constant");
    static_assert(r1 % 2 == 0 && kTwP % 2 == 0, "twiddles are read in 16-byte pairs from 16-byte aligned rows");
};

// First-stage butterfly of a row stage handled by thread slot id (0 ..
// 16 S1 - 1): slab row k, butterfly b (elements b + S1 t).  A half-warp
// takes 16 / S1 rows S1 apart (k = id / 16 + S1 * row of the half-warp),
// so that with rows padded to 17 elements its 16 eight-byte accesses fall
// in 16 different bank pairs (rows k and k + 1 side by side would share
// seven of them), while a warp still reads S1 consecutive elements of each
// of its rows from global memory.
__device__ __forceinline__ void row_butterfly(int id, int S1, int& k, int& b) {
    k = id / 16 + S1 * ((id % 16) / S1);
    b = id % S1;
}

// Slab index of element (k, c) of block blk (16 rows of 17 elements).
__device__ __forceinline__ int xslab(int blk, int k, int c) { return blk * 272 + k * 17 + c; }
// Row slab: window row k of the CTA, storage column s.
__device__ __forceinline__ int xrow(int k, int s) { return xslab(s >> 4, k, s & 15); }
// Column slab: storage row g, column c of the CTA.
__device__ __forceinline__ int xcol(int g, int c) { return xslab(g >> 4, g & 15, c); }

// The same offsets split into a per-thread base and a part that depends
// only on the unrolled loop index, a compile-time constant, so that every
// access of a stage is the base register plus an immediate.
// First stages, element b + S1 t (b < S1 <= 16): block and position of t.
template <int S1>
__device__ __forceinline__ constexpr int x1_blk(int t) { return S1 >= 16 ? t * (S1 / 16) : t / (16 / S1); }
template <int S1>
__device__ __forceinline__ constexpr int x1_pos(int t) { return S1 >= 16 ? 0 : S1 * (t % (16 / S1)); }
// xrow(k, b + S1 t) = xrow1_base(k, b) + xrow1_off<S1>(t)
__device__ __forceinline__ int xrow1_base(int k, int b) { return k * 17 + b; }
template <int S1>
__device__ __forceinline__ constexpr int xrow1_off(int t) { return x1_blk<S1>(t) * 272 + x1_pos<S1>(t); }
// xcol(b + S1 t, c) = xcol1_base(b, c) + xcol1_off<S1>(t)
__device__ __forceinline__ int xcol1_base(int b, int c) { return b * 17 + c; }
template <int S1>
__device__ __forceinline__ constexpr int xcol1_off(int t) { return x1_blk<S1>(t) * 272 + x1_pos<S1>(t) * 17; }
// Second stages, element m R2 + i (i < R2 <= 16):
// xrow(k, m R2 + i) = xrow2_base<R2>(k, m) + i, xcol(m R2 + i, c) = xcol2_base<R2>(m, c) + 17 i
template <int R2>
__device__ __forceinline__ int xrow2_base(int k, int m) {
    return (m / (16 / R2)) * 272 + k * 17 + R2 * (m % (16 / R2));
}
template <int R2>
__device__ __forceinline__ int xcol2_base(int m, int c) {
    return (m / (16 / R2)) * 272 + R2 * (m % (16 / R2)) * 17 + c;
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
// Make this thread's generic-proxy shared-memory writes visible to the bulk
// copies (async proxy) issued after the next barrier.
__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
// Copy `bytes` from this CTA's shared memory to shared memory of a CTA of
// the cluster; completion is counted on that CTA's mbarrier `bar`.
__device__ __forceinline__ void bulk_copy_to_peer(uint32_t dst, uint32_t src, uint32_t bytes, uint32_t bar) {
    asm volatile("cp.async.bulk.shared::cluster.shared::cta.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "r"(src), "r"(bytes), "r"(bar)
                 : "memory");
}

// Hint the L2 to fetch `bytes` (a multiple of 16) from global address p.
__device__ __forceinline__ void prefetch_l2(const void* p, uint32_t bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

// A wait gives up after kXposeSpinLimit polls or kXposeWaitCycles SM
// cycles, whichever comes first (try_wait may suspend the thread for a
// hardware-dependent time on each poll, so the cycle bound is what caps
// the wait at about a second).
constexpr uint32_t kXposeSpinLimit = 1u << 22;
constexpr long long kXposeWaitCycles = 1ll << 31;

// Bounded wait on an mbarrier phase; returns false (and sets bit 2 of
// *err) when it gives up.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity, int* err) {
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    for (uint32_t it = 1; it < kXposeSpinLimit; ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if (clock64() - t0 > kXposeWaitCycles) break;
    }
    if (err) atomicOr(err, 2);
    return false;
}
// Arrive (release, cluster scope) on an mbarrier of a CTA of the cluster.
__device__ __forceinline__ void mbar_remote_arrive(uint32_t cluster_bar) {
    asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(cluster_bar) : "memory");
}

// The 16 amplitudes a thread of the column step needs in one window, in
// the exchange variants' thread order (16-byte chunks, chunk k of thread t
// at element base + (k * T + t) * chunk): FP32 values, or FP16 codes
// converted to float (unscaled).  base: the window's first element plus
// rank * 16 * T.
template <int AMP, int T>
__device__ __forceinline__ void load_amps16(const void* y, size_t base, uint64_t pol, float (&out)[16]) {
    const uint4* p = reinterpret_cast<const uint4*>(static_cast<const char*>(y) + base * (AMP ? 2 : 4)) + threadIdx.x;
    constexpr int NCH = AMP ? 2 : 4;
#pragma unroll
    for (int k = 0; k < NCH; ++k) {
        const uint4 v = ld_nc_l2_hint(p + (size_t)k * T, pol);
        const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            if constexpr (AMP == 1) {
                const float2 f = __half22float2(*reinterpret_cast<const __half2*>(&w[q]));
                out[8 * k + 2 * q] = f.x;
                out[8 * k + 2 * q + 1] = f.y;
            } else {
                out[4 * k + q] = __uint_as_float(w[q]);
            }
        }
    }
}

// x[t] *= W^(b t) (CONJ: its conjugate) for t = 1 .. R - 1, from the
// butterfly's row of the twiddle table, two values per 16-byte load.
template <int R, bool CONJ>
__device__ __forceinline__ void twiddle_row(float2 (&x)[R], const float2* row) {
    const float4* w4 = reinterpret_cast<const float4*>(row);
#pragma unroll
    for (int p = 0; p < R / 2; ++p) {
        const float4 w = w4[p];
        if (p > 0) x[2 * p] = CONJ ? cmulc(x[2 * p], make_float2(w.x, w.y)) : cmul(x[2 * p], make_float2(w.x, w.y));
        x[2 * p + 1] = CONJ ? cmulc(x[2 * p + 1], make_float2(w.z, w.w)) : cmul(x[2 * p + 1], make_float2(w.z, w.w));
    }
}

// Windows j0 .. jn - 1 of the job `a` on one cluster.  TMC: keep 1/d and v
// in TMEM where the geometry allows (the launched kernels); the twin
// without it only serves the occupancy query (see agent_xpose).
template <int N, int AMP, bool TMC>
__device__ __forceinline__ void xpose_body(const AgentArgs& a, const int j0, const int jn) {
    using G = XposeGeom<N>;
    constexpr int C = G::C, T = G::kThreads, r1 = G::r1, r2 = G::r2, S1 = G::S1;
    constexpr int U2 = G::NB2 / T;   // second-stage butterflies per thread
    constexpr uint32_t kBlkBytes = G::kBlkBytes, kBytes = C * G::kBlkBytes;

    extern __shared__ float4 smem_raw[];
    float2* sA = reinterpret_cast<float2*>(smem_raw);
    float2* sB = sA + G::kSlab;
    float2* tw = sB + G::kSlab;
    uint64_t* bars = reinterpret_cast<uint64_t*>(tw + G::kTwElems);   // [0]: B slab filled, [1]: A slab filled, [2]: run done
    __shared__ double red[(T / 32) * 4];

    cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank();
    const uint32_t a_base = smem_addr(sA), b_base = smem_addr(sB);
    const uint32_t bar_b = smem_addr(bars), bar_a = smem_addr(bars + 1), bar_done = smem_addr(bars + 2);
    if (threadIdx.x == 0) {
        mbar_init(bar_b, 1);
        mbar_init(bar_a, 1);
        mbar_init(bar_done, C);
        mbar_fence_init();
        mbar_arrive_expect_tx(bar_b, kBytes);
        mbar_arrive_expect_tx(bar_a, kBytes);
    }
    // twiddles of the first-stage butterflies, by butterfly b then stage
    // output t: tw[b kTwP + t] = W_N^(b t)
    for (int i = threadIdx.x; i < N; i += T) tw[(i / r1) * G::kTwP + i % r1] = a.tw[(i / r1) * (i % r1)];
    cl.sync();   // every CTA's barriers are armed before any copy or arrival can land

    const float two_rho_prev = 2.0f * a.rho_prev;
    const float inv_n = 1.0f / (float)N;
    const float scale = 1.0f / (float)N;            // orthonormal F^*
    const float inv1pa = 1.0f / (1.0f + a.alpha);
    const float alpha = a.alpha;
    const float two_rho = 2.0f * a.rho_cur;
    const float2 trp2 = make_float2(two_rho_prev, two_rho_prev), scale2 = make_float2(scale, scale);
    const float2 alpha2 = make_float2(alpha, alpha), inv1pa2 = make_float2(inv1pa, inv1pa);
    const float2 m2rho2 = make_float2(-two_rho, -two_rho);
    const bool first = a.first != 0;
    const bool res = a.residual != 0;
    const int row0 = rank * G::R;
    const uint64_t pol_u = a.keep_u ? l2_policy_evict_last() : l2_policy_evict_normal();
    const uint64_t pol_first = l2_policy_evict_first();
    uint32_t parity = 0;

    // With one first-stage butterfly per thread (Np >= 128), a thread's 16
    // values of 1/d are the same in every window and its 16 values of v are
    // needed again in the copy-out of the same window: both are kept in
    // TMEM, 64 columns of the thread's lane (1/d in 0..31, v in 32..63), so
    // the copy-out loads nothing from memory outside the residual iteration.
    constexpr bool kTm = TMC && G::NB1 == T && r1 == 16;
    constexpr uint32_t kQuads = (uint32_t)((T / 32 + 3) / 4);   // warps sharing one lane quadrant
    constexpr uint32_t kTmCols = kTm ? 64u * kQuads : 32u;
    // the probe d itself in a second allocation of 32 columns a quadrant,
    // where the resident CTAs' columns allow it (else d = conj(1/d) / |1/d|^2)
    constexpr bool kTmD = kTm && (kTmCols + 32u * kQuads) * (uint32_t)G::kMinBlocks <= 512u;
    constexpr uint32_t kTmDCols = 32u * kQuads;
    static_assert(!kTm || kTmCols * G::kMinBlocks <= 512, "TMEM of the resident CTAs must fit an SM");
    __shared__ uint32_t tm_sh, tm_sh_d;
    uint32_t tm_addr = 0, tm_d = 0;
    // whether one of the thread's pixels has its probe value treated as
    // absent (1/d = 0): only then does the update test for it
    bool absent = !kTm;
    if constexpr (kTm) {
        if (threadIdx.x < 32) {
            if constexpr (kTmD) tmem_alloc2(smem_addr(&tm_sh), kTmCols, smem_addr(&tm_sh_d), kTmDCols);
            else tmem_alloc(smem_addr(&tm_sh), kTmCols);
        }
        tmem_fence_before_sync();
        __syncthreads();
        tmem_fence_after_sync();
        const int warp = threadIdx.x >> 5;
        const uint32_t lanes = (uint32_t)(32 * (warp & 3)) << 16;
        tm_addr = tm_sh + lanes + 64u * (uint32_t)(warp >> 2);
        if constexpr (kTmD) tm_d = tm_sh_d + lanes + 32u * (uint32_t)(warp >> 2);
        int k, b;
        row_butterfly(threadIdx.x, S1, k, b);
        const float2* dr = a.dinv + (size_t)(row0 + k) * N;
        const float2* pr = a.probe + (size_t)(row0 + k) * N;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            uint32_t r[16], p[16];
#pragma unroll
            for (int t = 0; t < 8; ++t) {
                const float2 di = __ldg(dr + b + S1 * (8 * h + t));
                absent |= di.x == 0.f && di.y == 0.f;
                r[2 * t] = __float_as_uint(di.x);
                r[2 * t + 1] = __float_as_uint(di.y);
                if constexpr (kTmD) {
                    const float2 d = __ldg(pr + b + S1 * (8 * h + t));
                    p[2 * t] = __float_as_uint(d.x);
                    p[2 * t + 1] = __float_as_uint(d.y);
                }
            }
            tmem_st16(tm_addr + 16u * h, r);
            if constexpr (kTmD) tmem_st16(tm_d + 16u * h, p);
        }
        tmem_wait_st();
    }

    // the CTA's stack rows and amplitudes of a window (one thread each)
    static_assert(G::NB2 / T * r2 == 16, "16 amplitudes per thread in the column step");
    auto prefetch_window = [&](int jw) {
        const size_t rb = ((size_t)jw * N + row0) * N;
        if (threadIdx.x == 0) prefetch_l2(a.q + rb, G::R * N * (uint32_t)sizeof(float2));
        else if (threadIdx.x == T - 1)
            prefetch_l2(static_cast<const char*>(a.y) + ((size_t)jw * N * N + (size_t)rank * 16 * T) * (AMP ? 2 : 4),
                        16 * T * (AMP ? 2 : 4));
    };
    prefetch_window(j0);

    // the window corner is loaded a window ahead, so the consensus loads of
    // the copy-in do not wait for it
    int2 off_next = window_corner<N>(a, j0);
#pragma unroll 1
    for (int j = j0; j < jn; ++j) {
        const int2 off = off_next;
        if (j + 1 < jn) off_next = window_corner<N>(a, j + 1);
        const size_t wbase = (size_t)j * N * N;
        float yscale = 1.0f;
        if constexpr (AMP == 1) yscale = __ldg(a.yscale + j);
        if (j + 1 < jn) prefetch_window(j + 1);   // while this window is in flight

        // ---- S0 + S1 fused with the first DIF row stage (span N, radix r1)
#pragma unroll 1
        for (int it = 0; it < G::NB1 / T; ++it) {
            const int id = threadIdx.x + it * T;
            int k, b;
            row_butterfly(id, S1, k, b);
            const int row = row0 + k;
            const float2* qr = a.q + wbase + (size_t)row * N;
            const float2* __restrict__ dr = a.probe + (size_t)row * N;
            const float2* __restrict__ xr = a.xbar + (size_t)(off.x + row) * a.n2 + off.y;
            // all stack loads first (one memory round trip), then the
            // L2-resident consensus and probe values
            float2 x[r1];
#pragma unroll
            for (int t = 0; t < r1; ++t) x[t] = qr[b + S1 * t];
#pragma unroll
            for (int t = 0; t < r1; ++t) x[t] = mann_close2(x[t], __ldg(xr + b + S1 * t), trp2);
            if constexpr (kTm) {
#pragma unroll
                for (int h = 0; h < 2; ++h) {   // keep v for the copy-out
                    uint32_t r[16];
#pragma unroll
                    for (int t = 0; t < 8; ++t) {
                        r[2 * t] = __float_as_uint(x[8 * h + t].x);
                        r[2 * t + 1] = __float_as_uint(x[8 * h + t].y);
                    }
                    tmem_st16(tm_addr + 32u + 16u * h, r);
                }
            }
            if constexpr (kTmD) {
                // d from TMEM
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    uint32_t r[16];
                    tmem_ld16(tm_d + 16u * h, r);
#pragma unroll
                    for (int t = 0; t < 8; ++t)
                        x[8 * h + t] = cmul(make_float2(__uint_as_float(r[2 * t]), __uint_as_float(r[2 * t + 1])),
                                            x[8 * h + t]);
                }
            } else if constexpr (kTm) {
                // d from the 1/d in TMEM: d = conj(1/d) / |1/d|^2 (0 where d is
                // treated as absent, where the table holds 0), one approximate
                // reciprocal per pixel instead of a load round
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    uint32_t r[16];
                    tmem_ld16(tm_addr + 16u * h, r);
#pragma unroll
                    for (int t = 0; t < 8; ++t) {
                        const float ix = __uint_as_float(r[2 * t]), iy = __uint_as_float(r[2 * t + 1]);
                        const float m2 = fmaf(ix, ix, iy * iy);
                        const float rm = m2 > 0.f ? __fdividef(1.0f, m2) : 0.f;
                        x[8 * h + t] = cmul(make_float2(ix * rm, -iy * rm), x[8 * h + t]);
                    }
                }
            } else {
#pragma unroll
                for (int t = 0; t < r1; ++t) x[t] = cmul(__ldg(dr + b + S1 * t), x[t]);
            }
            Dft<r1, false>::run(x);
            twiddle_row<r1, false>(x, tw + b * G::kTwP);
#pragma unroll
            for (int t = 0; t < r1; ++t) sA[xrow1_base(k, b) + xrow1_off<S1>(t)] = x[t];
        }
        __syncthreads();
        // ---- second DIF row stage (span r2), and A -> B.  Block `rank` of
        // peer p's B was last read by p's own copy of it back to this CTA in
        // the previous window, which landed before this CTA passed its wait
        // on the A slab: p's region is free.  A warp's butterflies of one
        // iteration cover all 16 rows of 2 r2 whole columns; where that is a
        // whole number of blocks (r2 >= 8), the warp sends them itself as
        // soon as it has written them, without a block barrier.
        constexpr bool kWarpSends = (2 * r2) % 16 == 0;
#pragma unroll 1
        for (int it = 0; it < G::NB2 / T; ++it) {
            const int id = threadIdx.x + it * T;
            const int k = id % 16, m = id / 16;
            float2 x[r2];
#pragma unroll
            for (int i = 0; i < r2; ++i) x[i] = sA[xrow2_base<r2>(k, m) + i];
            Dft<r2, false>::run(x);
#pragma unroll
            for (int i = 0; i < r2; ++i) sA[xrow2_base<r2>(k, m) + i] = x[i];
            if constexpr (kWarpSends) {
                constexpr int kBlocksPerWarp = 2 * r2 / 16;
                fence_proxy_async_smem();
                __syncwarp();
                const int lane = threadIdx.x & 31;
                const int p = ((id & ~31) / 16) * r2 / 16 + lane;   // first column of the warp / 16, + lane
                if (lane < kBlocksPerWarp)
                    bulk_copy_to_peer(cluster_addr(b_base + (uint32_t)rank * kBlkBytes, (uint32_t)p),
                                      a_base + (uint32_t)p * kBlkBytes, kBlkBytes, cluster_addr(bar_b, (uint32_t)p));
            }
        }
        if constexpr (!kWarpSends) {
            fence_proxy_async_smem();
            __syncthreads();
            if (threadIdx.x < C) {
                const uint32_t p = threadIdx.x;
                bulk_copy_to_peer(cluster_addr(b_base + (uint32_t)rank * kBlkBytes, p), a_base + p * kBlkBytes,
                                  kBlkBytes, cluster_addr(bar_b, p));
            }
        }
        // amplitudes of this thread's column butterflies (value u r2 + i of
        // the thread order is element i of butterfly u), loaded while the
        // exchange is in flight
        float yv[U2][r2];
        {
            float ya[16];
            load_amps16<AMP, T>(a.y, wbase + (size_t)rank * 16 * T, pol_first, ya);
#pragma unroll
            for (int u = 0; u < U2; ++u)
#pragma unroll
                for (int i = 0; i < r2; ++i) yv[u][i] = AMP ? ya[u * r2 + i] * yscale : ya[u * r2 + i];
        }
        const bool got_b = mbar_wait_bounded(bar_b, parity, a.err);
        // re-arm for the next window before this CTA's next send: every
        // peer's next A -> B copy comes after it has received that send.
        // Only after a completed phase: a wait that gave up leaves the
        // barrier as it is (its phase still counts the missing bytes), and
        // the CTA stops at the next block barrier.
        if (threadIdx.x == 0 && got_b && j + 1 < jn) mbar_arrive_expect_tx(bar_b, kBytes);

        // ---- first DIF column stage (span N, radix r1)
#pragma unroll 1
        for (int it = 0; it < G::NB1 / T; ++it) {
            const int id = threadIdx.x + it * T;
            const int c = id % 16, b = id / 16;
            float2 x[r1];
#pragma unroll
            for (int t = 0; t < r1; ++t) x[t] = sB[xcol1_base(b, c) + xcol1_off<S1>(t)];
            Dft<r1, false>::run(x);
            twiddle_row<r1, false>(x, tw + b * G::kTwP);
#pragma unroll
            for (int t = 0; t < r1; ++t) sB[xcol1_base(b, c) + xcol1_off<S1>(t)] = x[t];
        }
        // a wait that gave up stops the CTA before it sends anything more
        if (__syncthreads_or(!got_b)) break;
        // ---- second column stage, S3, inverse second column stage (the
        // data-misfit sums only on the residual iteration)
        float acc_d = 0.f, acc_y = 0.f;
        auto column_step = [&](auto with_res) {
            constexpr bool kRes = decltype(with_res)::value;
#pragma unroll
            for (int u = 0; u < U2; ++u) {
                const int id = threadIdx.x + u * T;
                const int c = id % 16, m = id / 16;
                float2 x[r2];
#pragma unroll
                for (int i = 0; i < r2; ++i) x[i] = sB[xcol2_base<r2>(m, c) + 17 * i];
                Dft<r2, false>::run(x);
                if (a.spectrum) {   // check of the forward transform (kernel row m r2 + i, column row0 + c)
#pragma unroll
                    for (int i = 0; i < r2; ++i) a.spectrum[wbase + (size_t)(m * r2 + i) * N + row0 + c] = x[i];
                }
                replace_magnitudes<kRes>(x, yv[u], inv_n, acc_d, acc_y);
                Dft<r2, true>::run(x);
#pragma unroll
                for (int i = 0; i < r2; ++i) sB[xcol2_base<r2>(m, c) + 17 * i] = x[i];
            }
        };
        if (res) column_step(std::true_type{});
        else column_step(std::false_type{});
        __syncthreads();
        // ---- inverse first column stage (DIT, span N)
#pragma unroll 1
        for (int it = 0; it < G::NB1 / T; ++it) {
            const int id = threadIdx.x + it * T;
            const int c = id % 16, b = id / 16;
            float2 x[r1];
#pragma unroll
            for (int t = 0; t < r1; ++t) x[t] = sB[xcol1_base(b, c) + xcol1_off<S1>(t)];
            twiddle_row<r1, true>(x, tw + b * G::kTwP);
            Dft<r1, true>::run(x);
#pragma unroll
            for (int t = 0; t < r1; ++t) sB[xcol1_base(b, c) + xcol1_off<S1>(t)] = x[t];
        }
        fence_proxy_async_smem();
        __syncthreads();
        // ---- B -> A.  Block `rank` of peer p's A is the block p sent here
        // in this window, which has landed (this CTA passed its wait on B).
        if (threadIdx.x < C) {
            const uint32_t p = threadIdx.x;
            bulk_copy_to_peer(cluster_addr(a_base + (uint32_t)rank * kBlkBytes, p), b_base + p * kBlkBytes, kBlkBytes,
                              cluster_addr(bar_a, p));
        }
        const bool got_a = mbar_wait_bounded(bar_a, parity, a.err);
        if (threadIdx.x == 0 && got_a && j + 1 < jn) mbar_arrive_expect_tx(bar_a, kBytes);

        // ---- inverse second row stage (span r2)
#pragma unroll 1
        for (int it = 0; it < G::NB2 / T; ++it) {
            const int id = threadIdx.x + it * T;
            const int k = id % 16, m = id / 16;
            float2 x[r2];
#pragma unroll
            for (int i = 0; i < r2; ++i) x[i] = sA[xrow2_base<r2>(k, m) + i];
            Dft<r2, true>::run(x);
#pragma unroll
            for (int i = 0; i < r2; ++i) sA[xrow2_base<r2>(k, m) + i] = x[i];
        }
        if (__syncthreads_or(!got_a)) break;
        // ---- inverse first row stage fused with S4 + S5 (the consensus
        // loads and the residual sums only on the residual iteration)
        float acc_z = 0.f, acc_w = 0.f;
        auto update = [&](auto with_res) {
            constexpr bool kRes = decltype(with_res)::value;
#pragma unroll 1
            for (int it = 0; it < G::NB1 / T; ++it) {
                const int id = threadIdx.x + it * T;
                int k, b;
                row_butterfly(id, S1, k, b);
                const int row = row0 + k;
                float2 x[r1];
#pragma unroll
                for (int t = 0; t < r1; ++t) x[t] = sA[xrow1_base(k, b) + xrow1_off<S1>(t)];
                twiddle_row<r1, true>(x, tw + b * G::kTwP);
                Dft<r1, true>::run(x);
                float2* qr = a.q + wbase + (size_t)row * N;   // read (S0) and overwritten (S5) by this thread only
                float2* __restrict__ ur = a.u + wbase + (size_t)row * N;
                const float2* __restrict__ xr = a.xbar + (size_t)(off.x + row) * a.n2 + off.y;
                // in quarters: the loads of a quarter are issued together
                constexpr int H = r1 / 4;
                if constexpr (kTm) tmem_wait_st();   // v of the copy-in has landed
#pragma unroll
                for (int h0 = 0; h0 < r1; h0 += H) {
                    float2 qv[H], xv[H], dv[H];
                    if constexpr (kTm) {
                        // v and 1/d from TMEM; the consensus values only feed the residual
                        static_assert(H == 4, "one 8-column TMEM load per quarter and table");
                        uint32_t rv[8], rd[8];
                        tmem_ld8x2(tm_addr + 32u + 2u * (uint32_t)h0, rv, tm_addr + 2u * (uint32_t)h0, rd);
#pragma unroll
                        for (int t = 0; t < H; ++t) {
                            qv[t] = make_float2(__uint_as_float(rv[2 * t]), __uint_as_float(rv[2 * t + 1]));
                            dv[t] = make_float2(__uint_as_float(rd[2 * t]), __uint_as_float(rd[2 * t + 1]));
                            if constexpr (kRes) xv[t] = __ldg(xr + b + S1 * (h0 + t));
                        }
                    } else {
                        const float2* __restrict__ dr = a.dinv + (size_t)row * N;
#pragma unroll
                        for (int t = 0; t < H; ++t) {
                            const int s = b + S1 * (h0 + t);
                            qv[t] = qr[s];
                            xv[t] = __ldg(xr + s);
                            dv[t] = __ldg(dr + s);
                        }
                    }
                    auto pixels = [&](auto check) {
                        constexpr bool kCheck = decltype(check)::value;
#pragma unroll
                        for (int t = 0; t < H; ++t) {
                            const int s = b + S1 * (h0 + t);
                            float2 u, qn;
                            // v: kept from the copy-in (TMEM), else q + 2 rho_prev xbar again
                            const float2 v = kTm ? qv[t] : mann_close2(qv[t], xv[t], trp2);
                            const float2 w =
                                agent_step2<kCheck>(x[h0 + t], v, dv[t], scale2, alpha2, inv1pa2, m2rho2, u, qn);
                            if constexpr (kRes) residual_sums(first ? v : xv[t], w, acc_z, acc_w);
                            st_l2_hint(ur + s, u, pol_u);       // read by the consensus gather next
                            st_l2_hint(qr + s, qn, pol_first);  // read again only next iteration
                        }
                    };
                    if (absent) pixels(std::true_type{});
                    else pixels(std::false_type{});
                }
            }
        };
        if (res) update(std::true_type{});
        else update(std::false_type{});
        // No barrier is needed before the next window: its copy-in writes
        // exactly the A rows this thread's warp has just read (the same
        // (k, b) butterflies), and the reduction buffer is only used here.
        float acc[4] = {acc_z, acc_w, acc_d, acc_y};
        if (res) block_reduce4<T>(acc, red, a.partials + ((size_t)j * C + rank) * 4);
        parity ^= 1u;
    }
    // End of the run: arrive on every CTA's done barrier (this CTA has passed
    // its last receive wait, or stopped), then wait until every CTA of the
    // cluster has.  After a full run no bulk copy into or out of this CTA is
    // then in flight: every copy it sent was received before its receiver
    // arrived.  The wait is bounded like the others.
    if constexpr (kTm) {
        tmem_wait_st();   // a stopped run may leave its last v stores outstanding
        tmem_fence_before_sync();
    }
    __syncthreads();
    if (threadIdx.x < C) mbar_remote_arrive(cluster_addr(bar_done, threadIdx.x));
    mbar_wait_bounded(bar_done, 0, a.err);
    __syncthreads();
    if constexpr (kTm) {
        if (threadIdx.x < 32) {
            tmem_fence_after_sync();
            tmem_dealloc(tm_sh, kTmCols);
            if constexpr (kTmD) tmem_dealloc(tm_sh_d, kTmDCols);
        }
    }
}

// One job: cluster k processes windows [k wpc, min((k + 1) wpc, J)).
template <int N, int AMP, bool TMC = true>
__global__ void __launch_bounds__(XposeGeom<N>::kThreads, XposeGeom<N>::kMinBlocks)
agent_xpose_kernel(const __grid_constant__ AgentArgs a) {
    const int j0 = (int)(blockIdx.x / XposeGeom<N>::C) * a.wpc;
    xpose_body<N, AMP, TMC>(a, j0, min(j0 + a.wpc, a.J));
}

// Several jobs: cluster k processes job work[k].x from window work[k].y on,
// that job's wpc windows at most.
template <int N, int AMP>
__global__ void __launch_bounds__(XposeGeom<N>::kThreads, XposeGeom<N>::kMinBlocks)
agent_xpose_kernel_batched(const AgentArgs* __restrict__ descs, const int2* __restrict__ work) {
    const int2 w = work[blockIdx.x / XposeGeom<N>::C];
    const AgentArgs& a = descs[w.x];
    xpose_body<N, AMP, true>(a, w.y, min(w.y + a.wpc, a.J));
}

template <int N, typename K>
cudaLaunchConfig_t xpose_config(K, int nclusters, cudaStream_t s, cudaLaunchAttribute* attr) {
    using G = XposeGeom<N>;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(nclusters * G::C), 1, 1);
    cfg.blockDim = dim3(G::kThreads, 1, 1);
    cfg.dynamicSmemBytes = G::kSmemLaunch;
    cfg.stream = s;
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = G::C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cfg;
}

template <typename K>
cudaError_t xpose_attributes(K fn, int smem, int cluster) {
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess && cluster > 8) e = cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    return e;
}

// Query (a == nullptr: fills info, max_clusters from the occupancy API) or
// launch ceil(J / a->wpc) clusters.
template <int N>
cudaError_t agent_xpose(const AgentArgs* a, int amp_f16, cudaStream_t s, AgentPlanInfo* info) {
    using G = XposeGeom<N>;
    void (*fn)(const AgentArgs) = amp_f16 ? agent_xpose_kernel<N, 1> : agent_xpose_kernel<N, 0>;
    cudaError_t e = xpose_attributes(fn, G::kSmemLaunch, G::C);
    if (a == nullptr) {
        // The occupancy API counts a kernel that allocates TMEM as one CTA
        // per SM.  The TMEM cache takes at most 1.9 columns per KB of shared
        // memory, so 426 of an SM's 512 columns in any mix of resident CTAs,
        // and never limits residency: ask for the same kernel without it.
        void (*twin)(const AgentArgs) = agent_xpose_kernel<N, 0, false>;
        cudaError_t et = xpose_attributes(twin, G::kSmemLaunch, G::C);
        info->threads = G::kThreads;
        info->smem_bytes = G::kSmemLaunch;
        info->max_clusters = 0;
        if (e == cudaSuccess && et == cudaSuccess) {
            cudaLaunchAttribute attr[1];
            cudaLaunchConfig_t cfg = xpose_config<N>(twin, 64, nullptr, attr);
            int n = 0;
            if (cudaOccupancyMaxActiveClusters(&n, twin, &cfg) == cudaSuccess) info->max_clusters = n;
        }
        cudaGetLastError();
        info->launchable = info->max_clusters > 0;
        return cudaSuccess;
    }
    if (e != cudaSuccess) return e;
    if (a->wpc <= 0) return cudaErrorInvalidValue;
    const int nclusters = (a->J + a->wpc - 1) / a->wpc;
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = xpose_config<N>(fn, nclusters, s, attr);
    return cudaLaunchKernelEx(&cfg, fn, *a);
}

template <int N>
cudaError_t agent_xpose_batched(const AgentArgs* descs, const int2* work, int nclusters, int amp_f16,
                                cudaStream_t s) {
    using G = XposeGeom<N>;
    if (nclusters <= 0) return cudaSuccess;
    void (*fn)(const AgentArgs*, const int2*) =
        amp_f16 ? agent_xpose_kernel_batched<N, 1> : agent_xpose_kernel_batched<N, 0>;
    cudaError_t e = xpose_attributes(fn, G::kSmemLaunch, G::C);
    if (e != cudaSuccess) return e;
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = xpose_config<N>(fn, nclusters, s, attr);
    return cudaLaunchKernelEx(&cfg, fn, descs, work);
}

}  // namespace pmace
