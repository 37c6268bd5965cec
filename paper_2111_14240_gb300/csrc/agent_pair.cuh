// The fused agent sweep (steps S0-S5 of one PMACE iteration) with two
// windows per cluster in packed single-precision lanes.
//
// Same data flow as the transposing-exchange sweep (agent_xpose.cuh): a
// window is Np x Np, its cluster has C = Np / 16 CTAs, CTA `rank` holds the
// row slab A (window rows [16 rank, 16 rank + 16)) and the column slab B
// (all rows of storage columns [16 rank, 16 rank + 16)), both as C blocks
// of 16 x 17 elements, and bulk copies between the CTAs transpose A into B
// and back.  Here every element of the slabs holds the same pixel of two
// windows j and j + 1 as (Re_j, Re_j+1, Im_j, Im_j+1): one 16-byte
// shared-memory access moves two complex values, and every butterfly,
// twiddle and agent update runs on the pair (Re_j, Re_j+1) and the pair
// (Im_j, Im_j+1) with the packed FP32 instructions of sm_100 and later
// (add, multiply and fused multiply-add on two floats at once, each lane
// rounded exactly as the scalar instruction).  The index arithmetic, the
// shared-memory instructions and the two exchanges are shared by the two
// windows, and the butterflies of the two windows are independent, so the
// instruction count per pixel is about half that of one window at a time.
//
// Per pair of windows:
//   rows   copy-in (S0: v = q + 2 rho_prev xbar, S1: a = d v, with v kept in
//          TMEM for the agent update) fused with the first DIF row stage;
//          second row stage in A;
//   A -> B bulk copies, each counted on the receiving CTA's mbarrier;
//   cols   first DIF column stage in B; second column stage, magnitude
//          replacement (S3) and the inverse second stage in registers;
//          inverse first column stage in B;
//   B -> A bulk copies back;
//   rows   inverse second row stage in A; inverse first row stage fused
//          with the agent update and the stores of u and q (S4, S5).
//
// Odd run lengths: the last pair of a run may hold one window; its second
// lane then repeats the first window (same loads, same values stored to
// the same addresses by the same thread) and writes no residual sums.
//
// Waits: every CTA waits on its two receive mbarriers, bounded in polls and
// in clock cycles.  A wait that gives up sets bit 2 of *err; the CTA's
// threads agree at the next block barrier (block-wide OR) and stop: no
// further bulk copy is sent and the remaining windows are skipped.  The end of a run is a bounded
// all-to-all arrival on a third mbarrier per CTA instead of a cluster
// barrier: a CTA leaves only when every CTA of the cluster has passed its
// last receive wait, so no bulk copy into or out of its shared memory is
// still in flight.  The only unbounded wait is the hardware cluster
// barrier after the barrier initialisation at kernel start, which every
// CTA of the cluster reaches before any data moves.
#pragma once

#include "agent.cuh"
#include "agent_xpose.cuh"
#include "cache_hints.cuh"
#include "tmem.cuh"

#include <type_traits>

namespace pmace {

// ------------------------------------------------------------------ packed lanes
__device__ __forceinline__ float2 padd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 psub(float2 a, float2 b) { return __fadd2_rn(a, make_float2(-b.x, -b.y)); }
__device__ __forceinline__ float2 pmul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 pfma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 pneg(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ constexpr float2 pdup(float s) { return float2{s, s}; }

// The same complex element of two windows: re = (Re_0, Re_1), im = (Im_0, Im_1).
struct cp2 {
    float2 re, im;
};
__device__ __forceinline__ cp2 cadd(cp2 a, cp2 b) { return {padd(a.re, b.re), padd(a.im, b.im)}; }
__device__ __forceinline__ cp2 csub(cp2 a, cp2 b) { return {psub(a.re, b.re), psub(a.im, b.im)}; }
// a + rot(b) and a - rot(b), rot = -i (forward) or +i (inverse)
template <bool INV>
__device__ __forceinline__ cp2 cadd_rot(cp2 a, cp2 b) {
    return INV ? cp2{psub(a.re, b.im), padd(a.im, b.re)} : cp2{padd(a.re, b.im), psub(a.im, b.re)};
}
template <bool INV>
__device__ __forceinline__ cp2 csub_rot(cp2 a, cp2 b) {
    return INV ? cp2{padd(a.re, b.im), psub(a.im, b.re)} : cp2{psub(a.re, b.im), padd(a.im, b.re)};
}
// a * w and a * conj(w) for a factor w = (c, s) shared by both lanes, given
// as the pairs (c, c) and (s, s)
__device__ __forceinline__ cp2 cmul_w(cp2 a, float2 c, float2 s) {
    return {pfma(a.re, c, pneg(pmul(a.im, s))), pfma(a.re, s, pmul(a.im, c))};
}
__device__ __forceinline__ cp2 cmulc_w(cp2 a, float2 c, float2 s) {
    return {pfma(a.im, s, pmul(a.re, c)), pfma(a.re, pneg(s), pmul(a.im, c))};
}
__device__ __forceinline__ cp2 ld_cp2(const float4* p) {
    const float4 v = *p;
    return {make_float2(v.x, v.y), make_float2(v.z, v.w)};
}
__device__ __forceinline__ void st_cp2(float4* p, cp2 a) { *p = make_float4(a.re.x, a.re.y, a.im.x, a.im.y); }

// ------------------------------------------------------------------ DFTs on lane pairs
// In-register DFT of length R on two windows at once, natural order in and
// out: X[k] = sum_j x[j] exp(-+2 pi i j k / R).  The same splits as Dft<R>
// (fft_smem.cuh); the multiplications by +-i are folded into the adds.
template <int R, bool INV>
struct PDft;

template <bool INV>
struct PDft<2, INV> {
    __device__ __forceinline__ static void run(cp2 (&x)[2]) {
        const cp2 a = x[0];
        x[0] = cadd(a, x[1]);
        x[1] = csub(a, x[1]);
    }
};

template <bool INV>
struct PDft<4, INV> {
    __device__ __forceinline__ static void run(cp2 (&x)[4]) {
        const cp2 a = cadd(x[0], x[2]), b = csub(x[0], x[2]), c = cadd(x[1], x[3]), e = csub(x[1], x[3]);
        x[0] = cadd(a, c);
        x[2] = csub(a, c);
        x[1] = cadd_rot<INV>(b, e);
        x[3] = csub_rot<INV>(b, e);
    }
};

// Radix 8 as 4 x 2 (index j = 2 j1 + j2, k = k1 + 4 k2): radix-4 over j1
// for j2 = 0, 1, the factors W_8^(j2 k1), radix 2 over j2.  The factor
// 1/sqrt(2) of W_8^1 and W_8^3 rides on the fused multiply-adds of the
// radix-2 step.
template <bool INV>
struct PDft<8, INV> {
    __device__ __forceinline__ static void run(cp2 (&x)[8]) {
        constexpr float kR = 0.70710678118654752440f;
        const float2 R = pdup(kR), NR = pdup(-kR);
        cp2 t[4] = {x[0], x[2], x[4], x[6]};
        cp2 s[4] = {x[1], x[3], x[5], x[7]};
        PDft<4, INV>::run(t);
        PDft<4, INV>::run(s);
        x[0] = cadd(t[0], s[0]);
        x[4] = csub(t[0], s[0]);
        x[2] = cadd_rot<INV>(t[2], s[2]);
        x[6] = csub_rot<INV>(t[2], s[2]);
        {   // k1 = 1: W_8^1 s = r (P, -M) forward, r (M, P) inverse
            const float2 P = padd(s[1].re, s[1].im), M = psub(s[1].re, s[1].im);
            if (INV) {
                x[1] = {pfma(M, R, t[1].re), pfma(P, R, t[1].im)};
                x[5] = {pfma(M, NR, t[1].re), pfma(P, NR, t[1].im)};
            } else {
                x[1] = {pfma(P, R, t[1].re), pfma(M, NR, t[1].im)};
                x[5] = {pfma(P, NR, t[1].re), pfma(M, R, t[1].im)};
            }
        }
        {   // k1 = 3: W_8^3 s = r (-M, -P) forward, r (-P, M) inverse
            const float2 P = padd(s[3].re, s[3].im), M = psub(s[3].re, s[3].im);
            if (INV) {
                x[3] = {pfma(P, NR, t[3].re), pfma(M, R, t[3].im)};
                x[7] = {pfma(P, R, t[3].re), pfma(M, NR, t[3].im)};
            } else {
                x[3] = {pfma(M, NR, t[3].re), pfma(P, NR, t[3].im)};
                x[7] = {pfma(M, R, t[3].re), pfma(P, R, t[3].im)};
            }
        }
    }
};

// Radix 16: the four-step split 4 x 4 with the inner twiddles folded into
// the second radix-4 pass, as Dft<16> (fft_smem.cuh): every nontrivial
// W_16^m is a real scale times a factor whose parts are +-1 or
// +-tan(pi/8), and the scales ride on the fused multiply-adds of the pass
// that follows.
template <bool INV>
struct PDft<16, INV> {
    static constexpr float kC = 0.92387953251128675613f;   // cos(pi/8)
    static constexpr float kT = 0.41421356237309504880f;   // tan(pi/8)
    static constexpr float kR = 0.70710678118654752440f;   // 1/sqrt(2)
    static constexpr float sg = INV ? 1.0f : -1.0f;         // sign of the twiddles' imaginary parts

    __device__ __forceinline__ static cp2 by_w1(cp2 a) {   // (1 + i sg t)
        return {pfma(a.im, pdup(-sg * kT), a.re), pfma(a.re, pdup(sg * kT), a.im)};
    }
    __device__ __forceinline__ static cp2 by_w3(cp2 a) {   // (t + i sg)
        return INV ? cp2{pfma(a.re, pdup(kT), pneg(a.im)), pfma(a.im, pdup(kT), a.re)}
                   : cp2{pfma(a.re, pdup(kT), a.im), pfma(a.im, pdup(kT), pneg(a.re))};
    }
    __device__ __forceinline__ static cp2 by_w9(cp2 a) {   // (-1 - i sg t)
        return {pfma(a.im, pdup(sg * kT), pneg(a.re)), pfma(a.re, pdup(-sg * kT), pneg(a.im))};
    }
    __device__ __forceinline__ static cp2 by_w2(cp2 a) {   // (1 + i sg)
        return INV ? cp2{psub(a.re, a.im), padd(a.im, a.re)} : cp2{padd(a.re, a.im), psub(a.im, a.re)};
    }
    __device__ __forceinline__ static cp2 by_w6(cp2 a) {   // (-1 + i sg)
        return INV ? cp2{pneg(padd(a.re, a.im)), psub(a.re, a.im)} : cp2{psub(a.im, a.re), pneg(padd(a.re, a.im))};
    }
    __device__ __forceinline__ static cp2 rot(cp2 a) {      // (-+ i) a
        return INV ? cp2{pneg(a.im), a.re} : cp2{a.im, pneg(a.re)};
    }
    // Radix-4 DFT of (i0, k2 u2, k13 u1, k13 u3) into x[k1 + 4 k2]
    template <int K1>
    __device__ __forceinline__ static void pass2(cp2 (&x)[16], cp2 i0, cp2 u1, cp2 u2, cp2 u3, float k2, float k13) {
        const float2 K2 = pdup(k2), NK2 = pdup(-k2), K13 = pdup(k13), NK13 = pdup(-k13);
        const cp2 a = {pfma(u2.re, K2, i0.re), pfma(u2.im, K2, i0.im)};
        const cp2 b = {pfma(u2.re, NK2, i0.re), pfma(u2.im, NK2, i0.im)};
        const cp2 c = cadd(u1, u3), e = csub(u1, u3);
        x[K1] = {pfma(c.re, K13, a.re), pfma(c.im, K13, a.im)};
        x[K1 + 8] = {pfma(c.re, NK13, a.re), pfma(c.im, NK13, a.im)};
        if (INV) {   // d = rot(e) = (-e.im, e.re)
            x[K1 + 4] = {pfma(e.im, NK13, b.re), pfma(e.re, K13, b.im)};
            x[K1 + 12] = {pfma(e.im, K13, b.re), pfma(e.re, NK13, b.im)};
        } else {     // d = rot(e) = (e.im, -e.re)
            x[K1 + 4] = {pfma(e.im, K13, b.re), pfma(e.re, NK13, b.im)};
            x[K1 + 12] = {pfma(e.im, NK13, b.re), pfma(e.re, K13, b.im)};
        }
    }
    __device__ __forceinline__ static void run(cp2 (&x)[16]) {
        cp2 t[4][4];
#pragma unroll
        for (int j2 = 0; j2 < 4; ++j2) {
            cp2 s[4] = {x[j2], x[4 + j2], x[8 + j2], x[12 + j2]};
            PDft<4, INV>::run(s);
#pragma unroll
            for (int k1 = 0; k1 < 4; ++k1) t[j2][k1] = s[k1];
        }
        {
            cp2 s[4] = {t[0][0], t[1][0], t[2][0], t[3][0]};
            PDft<4, INV>::run(s);
#pragma unroll
            for (int k2 = 0; k2 < 4; ++k2) x[4 * k2] = s[k2];
        }
        pass2<1>(x, t[0][1], by_w1(t[1][1]), by_w2(t[2][1]), by_w3(t[3][1]), kR, kC);
        pass2<2>(x, t[0][2], by_w2(t[1][2]), rot(t[2][2]), by_w6(t[3][2]), 1.0f, kR);
        pass2<3>(x, t[0][3], by_w3(t[1][3]), by_w6(t[2][3]), by_w9(t[3][3]), kR, kC);
    }
};

// S3 on a lane pair (y: the two windows' amplitudes): y A / |A|, 0 where
// A = 0, per lane exactly as replace_magnitude (agent.cuh); a lane whose
// squared magnitude is below 2^-100 takes that function's rescaling path.
template <bool RES>
__device__ __forceinline__ cp2 replace_magnitude2(cp2 a, float2 y, float inv_n, float2& acc_d, float2& acc_y) {
    const float2 m2 = pfma(a.re, a.re, pmul(a.im, a.im));
    if (m2.x < 0x1p-100f || m2.y < 0x1p-100f) {
        const float2 o0 = replace_magnitude<RES>(make_float2(a.re.x, a.im.x), y.x, inv_n, acc_d.x, acc_y.x);
        const float2 o1 = replace_magnitude<RES>(make_float2(a.re.y, a.im.y), y.y, inv_n, acc_d.y, acc_y.y);
        return {make_float2(o0.x, o1.x), make_float2(o0.y, o1.y)};
    }
    const float2 rs = make_float2(rsqrtf(m2.x), rsqrtf(m2.y));
    if constexpr (RES) {
        const float2 e = pfma(pmul(m2, rs), pdup(-inv_n), y);
        acc_d = pfma(e, e, acc_d);
        acc_y = pfma(y, y, acc_y);
    }
    const float2 f = pmul(y, rs);
    return {pmul(a.re, f), pmul(a.im, f)};
}

// ------------------------------------------------------------------ geometry
template <int N>
struct PairGeom {
    static constexpr int R = 16;                    // rows (and columns) per CTA
    static constexpr int C = N / R;                 // CTAs per window
    static constexpr int kThreads = N;
    static constexpr int kBlk = R * (R + 1);        // elements per exchange block (rows padded to 17)
    static constexpr int kSlab = C * kBlk;          // elements (float4: two windows) per slab
    static constexpr int kBlkBytes = kBlk * (int)sizeof(float4);
    static constexpr RadixPlan kRad = radix_plan(N);
    static constexpr int r1 = kRad.first, r2 = kRad.second;
    static constexpr int S1 = N / r1;               // stride of the first stage (= r2)
    static constexpr int NB1 = R * S1;              // first-stage butterflies per slab
    static constexpr int NB2 = R * r1;              // second-stage butterflies per slab
    // slabs, the first-stage twiddles as (c, c, s, s), three mbarriers
    static constexpr int kSmem = 2 * kSlab * (int)sizeof(float4) + N * (int)sizeof(float4) + 32;
    static constexpr int kBySmem = (228 * 1024) / (kSmem + 2048);
    static constexpr int kByThreads = 2048 / kThreads;
    static constexpr int kMinBlocks = kBySmem < kByThreads ? kBySmem : kByThreads;
    // TMEM per four warps: 1/d (scaled) 32 columns, d 32, v of both windows 64
    static constexpr uint32_t kTmCols = 128u * (uint32_t)((kThreads / 32 + 3) / 4);
    static_assert(r1 == 16 && NB1 == kThreads, "one first-stage butterfly (16 pixels) per thread");
    static_assert(NB2 % kThreads == 0, "second stage must split evenly over threads");
    static_assert(C >= 2 && C <= 16, "one block per CTA of the cluster");
    static_assert(kBlkBytes % 16 == 0, "bulk copies move multiples of 16 bytes between 16-byte aligned blocks");
    static_assert(kMinBlocks >= 1, "the slabs must fit one SM");
    static_assert(kTmCols * kMinBlocks <= 512, "TMEM of the resident CTAs must fit an SM");
};

// Per-CTA residual sums of two windows: lane 0 to out0, lane 1 to out1
// (out1 == nullptr: lane 1 repeats lane 0 and is not written).
template <int T>
__device__ __forceinline__ void block_reduce4_pair(float2 (&acc)[4], double* red, double* out0, double* out1) {
    float a0[4] = {acc[0].x, acc[1].x, acc[2].x, acc[3].x};
    float a1[4] = {acc[0].y, acc[1].y, acc[2].y, acc[3].y};
    block_reduce4<T>(a0, red, out0);
    __syncthreads();
    if (out1) {
        block_reduce4<T>(a1, red, out1);
        __syncthreads();
    }
}

// Windows j0 .. jn - 1 of the job `a` on one cluster, two at a time.  TMC:
// keep 1/d, d and v in TMEM (the launched kernels); the twin without it
// loads them from memory and only serves the occupancy query.
template <int N, int AMP, bool TMC>
__device__ __forceinline__ void pair_body(const AgentArgs& a, const int j0, const int jn) {
    using G = PairGeom<N>;
    constexpr int C = G::C, T = G::kThreads, r2 = G::r2, S1 = G::S1;
    constexpr int U2 = G::NB2 / T;   // second-stage butterflies per thread
    constexpr uint32_t kBlkBytes = G::kBlkBytes, kBytes = C * G::kBlkBytes;

    extern __shared__ float4 smem_raw[];
    float4* sA = smem_raw;
    float4* sB = sA + G::kSlab;
    float4* tw = sB + G::kSlab;
    uint64_t* bars = reinterpret_cast<uint64_t*>(tw + N);   // [0] B filled, [1] A filled, [2] run done
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
    // twiddles of the first-stage butterflies, by stage output t then
    // butterfly b: W_N^(b t) as (c, c, s, s)
    for (int i = threadIdx.x; i < N; i += T) {
        const float2 w = a.tw[(i % S1) * (i / S1)];
        tw[i] = make_float4(w.x, w.x, w.y, w.y);
    }
    cl.sync();   // every CTA's barriers are armed before any copy or arrival can land

    const float two_rho_prev = 2.0f * a.rho_prev;
    const float inv_n = 1.0f / (float)N;
    // w = alpha' v + h with alpha' = alpha / (1 + alpha) and h = (1/d) F^*A' / (N (1 + alpha))
    const float2 ALPHA1 = pdup(a.alpha / (1.0f + a.alpha));
    const float hscale = 1.0f / ((float)N * (1.0f + a.alpha));
    const float two_rho = 2.0f * a.rho_cur;
    const bool first = a.first != 0;
    const bool res = a.residual != 0;
    const int row0 = rank * G::R;
    const uint64_t pol_u = a.keep_u ? l2_policy_evict_last() : l2_policy_evict_normal();
    const uint64_t pol_first = l2_policy_evict_first();
    uint32_t parity = 0;

    // thread (k, b): first-stage butterfly b of slab row k, pixels (row0 + k, b + S1 t)
    const int k1 = threadIdx.x / S1, b1 = threadIdx.x % S1;
    const int row1 = row0 + k1;

    // TMEM: per thread 1/d * hscale (columns 0..31), d (32..63), v of the
    // window pair (64..127); also the positions where d is treated as
    // absent (1/d = 0), where the agent returns v
    __shared__ uint32_t tm_sh;
    uint32_t tm_addr = 0;
    uint32_t absent = 0;
    {
        const float2* dr = a.dinv + (size_t)row1 * N;
        const float2* pr = a.probe + (size_t)row1 * N;
#pragma unroll
        for (int t = 0; t < 16; ++t) {
            const float2 di = __ldg(dr + b1 + S1 * t);
            if (di.x == 0.f && di.y == 0.f) absent |= 1u << t;
        }
        if constexpr (TMC) {
            if (threadIdx.x < 32) tmem_alloc(smem_addr(&tm_sh), G::kTmCols);
            tmem_fence_before_sync();
            __syncthreads();
            tmem_fence_after_sync();
            const int warp = threadIdx.x >> 5;
            tm_addr = tm_sh + ((uint32_t)(32 * (warp & 3)) << 16) + 128u * (uint32_t)(warp >> 2);
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                uint32_t r[16], p[16];
#pragma unroll
                for (int t = 0; t < 8; ++t) {
                    const float2 di = __ldg(dr + b1 + S1 * (8 * h + t));
                    const float2 d = __ldg(pr + b1 + S1 * (8 * h + t));
                    r[2 * t] = __float_as_uint(di.x * hscale);
                    r[2 * t + 1] = __float_as_uint(di.y * hscale);
                    p[2 * t] = __float_as_uint(d.x);
                    p[2 * t + 1] = __float_as_uint(d.y);
                }
                tmem_st16(tm_addr + 16u * h, r);
                tmem_st16(tm_addr + 32u + 16u * h, p);
            }
            tmem_wait_st();
        }
    }

    // the CTA's stack rows and amplitudes of a window (one thread each)
    auto prefetch_window = [&](int jw, int slot) {
        const size_t rb = ((size_t)jw * N + row0) * N;
        if (threadIdx.x == 2 * slot) prefetch_l2(a.q + rb, G::R * N * (uint32_t)sizeof(float2));
        else if (threadIdx.x == 2 * slot + 1)
            prefetch_l2(static_cast<const char*>(a.y) + ((size_t)jw * N * N + (size_t)rank * 16 * T) * (AMP ? 2 : 4),
                        16 * T * (AMP ? 2 : 4));
    };
    prefetch_window(j0, 0);
    if (j0 + 1 < jn) prefetch_window(j0 + 1, 1);

    // Stack values of the thread's 16 pixels in the pair being loaded.  The
    // loads of pair p + 1 are issued quarter by quarter during the agent
    // update of pair p, so their latency overlaps that update; the consensus
    // values (mostly L2 hits) are loaded at the copy-in itself.
    float2 qa[16], qb[16];
    struct PairSrc {
        const float2 *q0, *q1;
    };
    auto pair_src = [&](int jj) {
        const int jjb = jj + 1 < jn ? jj + 1 : jj;
        return PairSrc{a.q + (size_t)jj * N * N + (size_t)row1 * N + b1,
                       a.q + (size_t)jjb * N * N + (size_t)row1 * N + b1};
    };
    auto load_quarter = [&](const PairSrc& ps, int h) {
#pragma unroll
        for (int t = 4 * h; t < 4 * h + 4; ++t) {
            qa[t] = ps.q0[S1 * t];
            qb[t] = ps.q1[S1 * t];
        }
    };
    {
        const PairSrc ps = pair_src(j0);
#pragma unroll
        for (int h = 0; h < 4; ++h) load_quarter(ps, h);
    }

    // window corners loaded a pair ahead, so the consensus loads of the
    // copy-in do not wait for them
    int2 off_next0 = window_corner<N>(a, j0), off_next1 = window_corner<N>(a, j0 + 1 < jn ? j0 + 1 : j0);
#pragma unroll 1
    for (int j = j0; j < jn; j += 2) {
        const bool two = j + 1 < jn;
        const int jb = two ? j + 1 : j;   // lane 1 repeats lane 0 at an odd end
        const int2 off0 = off_next0, off1 = off_next1;
        if (j + 2 < jn) {   // the next pair's corners, a pair ahead
            off_next0 = window_corner<N>(a, j + 2);
            off_next1 = window_corner<N>(a, j + 3 < jn ? j + 3 : j + 2);
        }
        const size_t wb0 = (size_t)j * N * N, wb1 = (size_t)jb * N * N;
        float2 ysc = make_float2(1.f, 1.f);
        if constexpr (AMP == 1) ysc = make_float2(__ldg(a.yscale + j), __ldg(a.yscale + jb));
        if (j + 2 < jn) prefetch_window(j + 2, 0);
        if (j + 3 < jn) prefetch_window(j + 3, 1);

        // ---- S0 + S1 fused with the first DIF row stage (span N, radix 16),
        // from the stack values loaded during the previous pair (or before
        // the loop)
        {
            const float2* __restrict__ xc0 = a.xbar + (size_t)(off0.x + row1) * a.n2 + off0.y + b1;
            const float2* __restrict__ xc1 = a.xbar + (size_t)(off1.x + row1) * a.n2 + off1.y + b1;
            cp2 x[16];
#pragma unroll
            for (int t = 0; t < 16; ++t) {
                const float2 va = mann_close(qa[t], __ldg(xc0 + S1 * t), two_rho_prev);
                const float2 vb = mann_close(qb[t], __ldg(xc1 + S1 * t), two_rho_prev);
                x[t] = {make_float2(va.x, vb.x), make_float2(va.y, vb.y)};
            }
            if constexpr (TMC) {
#pragma unroll
                for (int h = 0; h < 4; ++h) {   // keep v for the agent update
                    uint32_t r[16];
#pragma unroll
                    for (int t = 0; t < 4; ++t) {
                        const cp2 v = x[4 * h + t];
                        r[4 * t] = __float_as_uint(v.re.x);
                        r[4 * t + 1] = __float_as_uint(v.re.y);
                        r[4 * t + 2] = __float_as_uint(v.im.x);
                        r[4 * t + 3] = __float_as_uint(v.im.y);
                    }
                    tmem_st16(tm_addr + 64u + 16u * h, r);
                }
#pragma unroll
                for (int h = 0; h < 2; ++h) {   // a = d v
                    uint32_t r[16];
                    tmem_ld16(tm_addr + 32u + 16u * h, r);
#pragma unroll
                    for (int t = 0; t < 8; ++t) {
                        const float dx = __uint_as_float(r[2 * t]), dy = __uint_as_float(r[2 * t + 1]);
                        x[8 * h + t] = cmul_w(x[8 * h + t], pdup(dx), pdup(dy));
                    }
                }
            } else {
                const float2* __restrict__ pr = a.probe + (size_t)row1 * N + b1;
#pragma unroll
                for (int t = 0; t < 16; ++t) {
                    const float2 d = __ldg(pr + S1 * t);
                    x[t] = cmul_w(x[t], pdup(d.x), pdup(d.y));
                }
            }
            PDft<16, false>::run(x);
#pragma unroll
            for (int t = 1; t < 16; ++t) {
                const float4 w = tw[t * S1 + b1];
                x[t] = cmul_w(x[t], make_float2(w.x, w.y), make_float2(w.z, w.w));
            }
#pragma unroll
            for (int t = 0; t < 16; ++t) st_cp2(sA + xrow(k1, b1 + S1 * t), x[t]);
        }
        __syncthreads();
        // ---- second DIF row stage (span r2)
#pragma unroll
        for (int u = 0; u < U2; ++u) {
            const int id = threadIdx.x + u * T;
            const int k = id % 16, m = id / 16;
            cp2 x[r2];
#pragma unroll
            for (int i = 0; i < r2; ++i) x[i] = ld_cp2(sA + xrow(k, m * r2 + i));
            PDft<r2, false>::run(x);
#pragma unroll
            for (int i = 0; i < r2; ++i) st_cp2(sA + xrow(k, m * r2 + i), x[i]);
        }
        fence_proxy_async_smem();
        __syncthreads();
        // ---- A -> B (block `rank` of peer p's B was last read by p's own
        // copy of it back here in the previous pair, which landed before this
        // CTA passed its wait on the A slab: p's region is free)
        if (threadIdx.x < C) {
            const uint32_t p = threadIdx.x;
            bulk_copy_to_peer(cluster_addr(b_base + (uint32_t)rank * kBlkBytes, p), a_base + p * kBlkBytes, kBlkBytes,
                              cluster_addr(bar_b, p));
        }
        // amplitudes of this thread's column butterflies in both windows
        // (thread order: value u r2 + i is element i of butterfly u), loaded
        // while the exchange is in flight
        static_assert(U2 * r2 == 16, "16 amplitudes per thread in the column step");
        float2 yv[U2][r2];
        {
            float y0[16], y1[16];
            load_amps16<AMP, T>(a.y, wb0 + (size_t)rank * 16 * T, pol_first, y0);
            load_amps16<AMP, T>(a.y, wb1 + (size_t)rank * 16 * T, pol_first, y1);
#pragma unroll
            for (int u = 0; u < U2; ++u)
#pragma unroll
                for (int i = 0; i < r2; ++i) yv[u][i] = make_float2(y0[u * r2 + i], y1[u * r2 + i]);
        }
        const bool got_b = mbar_wait_bounded(bar_b, parity, a.err);
        // re-arm for the next pair before this CTA's next send: every peer's
        // next A -> B copy comes after it has received that send
        if (threadIdx.x == 0 && got_b && j + 2 < jn) mbar_arrive_expect_tx(bar_b, kBytes);

        // ---- first DIF column stage (span N, radix 16)
        {
            const int c = threadIdx.x % 16, b = threadIdx.x / 16;
            cp2 x[16];
#pragma unroll
            for (int t = 0; t < 16; ++t) x[t] = ld_cp2(sB + xcol(b + S1 * t, c));
            PDft<16, false>::run(x);
#pragma unroll
            for (int t = 1; t < 16; ++t) {
                const float4 w = tw[t * S1 + b];
                x[t] = cmul_w(x[t], make_float2(w.x, w.y), make_float2(w.z, w.w));
            }
#pragma unroll
            for (int t = 0; t < 16; ++t) st_cp2(sB + xcol(b + S1 * t, c), x[t]);
        }
        // a wait that gave up stops the CTA before it sends anything more
        if (__syncthreads_or(!got_b)) break;
        // ---- second column stage, S3, inverse second column stage
        float2 acc_d = make_float2(0.f, 0.f), acc_y = make_float2(0.f, 0.f);
        auto column_step = [&](auto with_res) {
            constexpr bool kRes = decltype(with_res)::value;
#pragma unroll
            for (int u = 0; u < U2; ++u) {
                const int id = threadIdx.x + u * T;
                const int c = id % 16, m = id / 16;
                cp2 x[r2];
#pragma unroll
                for (int i = 0; i < r2; ++i) x[i] = ld_cp2(sB + xcol(m * r2 + i, c));
                PDft<r2, false>::run(x);
                if (a.spectrum) {   // check of the forward transform (kernel row m r2 + i, column row0 + c)
#pragma unroll
                    for (int i = 0; i < r2; ++i) {
                        const size_t o = (size_t)(m * r2 + i) * N + row0 + c;
                        a.spectrum[wb0 + o] = make_float2(x[i].re.x, x[i].im.x);
                        a.spectrum[wb1 + o] = make_float2(x[i].re.y, x[i].im.y);
                    }
                }
#pragma unroll
                for (int i = 0; i < r2; ++i) {
                    const float2 y = AMP ? pmul(yv[u][i], ysc) : yv[u][i];
                    x[i] = replace_magnitude2<kRes>(x[i], y, inv_n, acc_d, acc_y);
                }
                PDft<r2, true>::run(x);
#pragma unroll
                for (int i = 0; i < r2; ++i) st_cp2(sB + xcol(m * r2 + i, c), x[i]);
            }
        };
        if (res) column_step(std::true_type{});
        else column_step(std::false_type{});
        __syncthreads();
        // ---- inverse first column stage (DIT, span N)
        {
            const int c = threadIdx.x % 16, b = threadIdx.x / 16;
            cp2 x[16];
#pragma unroll
            for (int t = 0; t < 16; ++t) x[t] = ld_cp2(sB + xcol(b + S1 * t, c));
#pragma unroll
            for (int t = 1; t < 16; ++t) {
                const float4 w = tw[t * S1 + b];
                x[t] = cmulc_w(x[t], make_float2(w.x, w.y), make_float2(w.z, w.w));
            }
            PDft<16, true>::run(x);
#pragma unroll
            for (int t = 0; t < 16; ++t) st_cp2(sB + xcol(b + S1 * t, c), x[t]);
        }
        fence_proxy_async_smem();
        __syncthreads();
        // ---- B -> A (block `rank` of peer p's A is the block p sent here in
        // this pair, which has landed: this CTA passed its wait on B)
        if (threadIdx.x < C) {
            const uint32_t p = threadIdx.x;
            bulk_copy_to_peer(cluster_addr(a_base + (uint32_t)rank * kBlkBytes, p), b_base + p * kBlkBytes, kBlkBytes,
                              cluster_addr(bar_a, p));
        }
        const bool got_a = mbar_wait_bounded(bar_a, parity, a.err);
        if (threadIdx.x == 0 && got_a && j + 2 < jn) mbar_arrive_expect_tx(bar_a, kBytes);

        // ---- inverse second row stage (span r2)
#pragma unroll
        for (int u = 0; u < U2; ++u) {
            const int id = threadIdx.x + u * T;
            const int k = id % 16, m = id / 16;
            cp2 x[r2];
#pragma unroll
            for (int i = 0; i < r2; ++i) x[i] = ld_cp2(sA + xrow(k, m * r2 + i));
            PDft<r2, true>::run(x);
#pragma unroll
            for (int i = 0; i < r2; ++i) st_cp2(sA + xrow(k, m * r2 + i), x[i]);
        }
        if (__syncthreads_or(!got_a)) break;
        // ---- inverse first row stage fused with S4 + S5
        float2 acc_z = make_float2(0.f, 0.f), acc_w = make_float2(0.f, 0.f);
        {
            cp2 x[16];
#pragma unroll
            for (int t = 0; t < 16; ++t) x[t] = ld_cp2(sA + xrow(k1, b1 + S1 * t));
#pragma unroll
            for (int t = 1; t < 16; ++t) {
                const float4 w = tw[t * S1 + b1];
                x[t] = cmulc_w(x[t], make_float2(w.x, w.y), make_float2(w.z, w.w));
            }
            PDft<16, true>::run(x);
            float2* q0 = a.q + wb0 + (size_t)row1 * N + b1;   // read (S0) and overwritten (S5) by this thread only
            float2* q1 = a.q + wb1 + (size_t)row1 * N + b1;
            float2* __restrict__ u0 = a.u + wb0 + (size_t)row1 * N + b1;
            float2* __restrict__ u1 = a.u + wb1 + (size_t)row1 * N + b1;
            const float2* __restrict__ x0 = a.xbar + (size_t)(off0.x + row1) * a.n2 + off0.y + b1;
            const float2* __restrict__ x1 = a.xbar + (size_t)(off1.x + row1) * a.n2 + off1.y + b1;
            const float2* __restrict__ dvp = a.dinv + (size_t)row1 * N + b1;
            if constexpr (TMC) tmem_wait_st();   // v of the copy-in has landed
            const bool more = j + 2 < jn;
            const PairSrc nxt = pair_src(more ? j + 2 : j);
            auto update = [&](auto check_absent) {
                constexpr bool kAbs = decltype(check_absent)::value;
#pragma unroll
                for (int h = 0; h < 4; ++h) {
                    cp2 v[4];
                    float2 dv[4];
                    if constexpr (TMC) {
                        uint32_t rv[16], rd[8];
                        tmem_ld16(tm_addr + 64u + 16u * h, rv);
                        tmem_ld8(tm_addr + 8u * h, rd);
#pragma unroll
                        for (int t = 0; t < 4; ++t) {
                            v[t] = {make_float2(__uint_as_float(rv[4 * t]), __uint_as_float(rv[4 * t + 1])),
                                    make_float2(__uint_as_float(rv[4 * t + 2]), __uint_as_float(rv[4 * t + 3]))};
                            dv[t] = make_float2(__uint_as_float(rd[2 * t]), __uint_as_float(rd[2 * t + 1]));
                        }
                    } else {
#pragma unroll
                        for (int t = 0; t < 4; ++t) {
                            const int s = S1 * (4 * h + t);
                            const float2 va = mann_close(q0[s], __ldg(x0 + s), two_rho_prev);
                            const float2 vb = mann_close(q1[s], __ldg(x1 + s), two_rho_prev);
                            v[t] = {make_float2(va.x, vb.x), make_float2(va.y, vb.y)};
                            const float2 di = __ldg(dvp + s);
                            dv[t] = make_float2(di.x * hscale, di.y * hscale);
                        }
                    }
#pragma unroll
                    for (int t = 0; t < 4; ++t) {
                        const int tt = 4 * h + t, s = S1 * tt;
                        const cp2 hh = cmul_w(x[tt], pdup(dv[t].x), pdup(dv[t].y));
                        cp2 w = {pfma(v[t].re, ALPHA1, hh.re), pfma(v[t].im, ALPHA1, hh.im)};
                        if constexpr (kAbs) {
                            if ((absent >> tt) & 1u) w = v[t];   // d treated as absent here
                        }
                        // u = 2w - v and q' = v - 2 rho w, per window as (re, im)
                        const float2 ua = make_float2(fmaf(2.f, w.re.x, -v[t].re.x), fmaf(2.f, w.im.x, -v[t].im.x));
                        const float2 ub = make_float2(fmaf(2.f, w.re.y, -v[t].re.y), fmaf(2.f, w.im.y, -v[t].im.y));
                        const float2 qn0 = make_float2(fmaf(-two_rho, w.re.x, v[t].re.x), fmaf(-two_rho, w.im.x, v[t].im.x));
                        const float2 qn1 = make_float2(fmaf(-two_rho, w.re.y, v[t].re.y), fmaf(-two_rho, w.im.y, v[t].im.y));
                        if (res) {
                            const float2 za = first ? make_float2(v[t].re.x, v[t].im.x) : __ldg(x0 + s);
                            const float2 zb = first ? make_float2(v[t].re.y, v[t].im.y) : __ldg(x1 + s);
                            float az = acc_z.x, aw = acc_w.x, bz = acc_z.y, bw = acc_w.y;
                            residual_sums(za, make_float2(w.re.x, w.im.x), az, aw);
                            residual_sums(zb, make_float2(w.re.y, w.im.y), bz, bw);
                            acc_z = make_float2(az, bz);
                            acc_w = make_float2(aw, bw);
                        }
                        st_l2_hint(u0 + s, ua, pol_u);      // read by the consensus gather next
                        st_l2_hint(u1 + s, ub, pol_u);
                        st_l2_hint(q0 + s, qn0, pol_first);  // read again only next iteration
                        st_l2_hint(q1 + s, qn1, pol_first);
                    }
                    // the next pair's values of these four pixels (the last
                    // pair of a run reloads its own, which keeps the loads
                    // unconditional, so the values are dead between the
                    // copy-in and this point)
                    load_quarter(nxt, h);
                }
            };
            if (absent) update(std::true_type{});
            else update(std::false_type{});
        }
        // No barrier is needed before the next pair: its copy-in writes
        // exactly the A elements this thread has just read (the same (k, b)
        // butterfly), and the reduction buffer is only used here.
        if (res) {
            float2 acc[4] = {acc_z, acc_w, acc_d, acc_y};
            block_reduce4_pair<T>(acc, red, a.partials + ((size_t)j * C + rank) * 4,
                                  two ? a.partials + ((size_t)jb * C + rank) * 4 : nullptr);
        }
        parity ^= 1u;
    }
    // End of the run: arrive on every CTA's done barrier (this CTA has passed
    // its last receive wait, or stopped), then wait until every CTA of the
    // cluster has: no bulk copy into or out of this CTA is in flight after.
    if constexpr (TMC) {
        tmem_wait_st();   // a stopped run may leave its last v stores outstanding
        tmem_fence_before_sync();
    }
    __syncthreads();
    if (threadIdx.x < C) mbar_remote_arrive(cluster_addr(bar_done, threadIdx.x));
    mbar_wait_bounded(bar_done, 0, a.err);
    __syncthreads();
    if constexpr (TMC) {
        if (threadIdx.x < 32) {
            tmem_fence_after_sync();
            tmem_dealloc(tm_sh, G::kTmCols);
        }
    }
}

// One job: cluster k processes windows [k wpc, min((k + 1) wpc, J)), wpc even.
template <int N, int AMP, bool TMC = true>
__global__ void __launch_bounds__(PairGeom<N>::kThreads, PairGeom<N>::kMinBlocks)
agent_pair_kernel(const __grid_constant__ AgentArgs a) {
    const int j0 = (int)(blockIdx.x / PairGeom<N>::C) * a.wpc;
    pair_body<N, AMP, TMC>(a, j0, min(j0 + a.wpc, a.J));
}

// Several jobs: cluster k processes job work[k].x from window work[k].y on,
// that job's wpc windows at most.
template <int N, int AMP>
__global__ void __launch_bounds__(PairGeom<N>::kThreads, PairGeom<N>::kMinBlocks)
agent_pair_kernel_batched(const AgentArgs* __restrict__ descs, const int2* __restrict__ work) {
    const int2 w = work[blockIdx.x / PairGeom<N>::C];
    const AgentArgs& a = descs[w.x];
    pair_body<N, AMP, true>(a, w.y, min(w.y + a.wpc, a.J));
}

template <int N>
cudaLaunchConfig_t pair_config(int nclusters, cudaStream_t s, cudaLaunchAttribute* attr) {
    using G = PairGeom<N>;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(nclusters * G::C), 1, 1);
    cfg.blockDim = dim3(G::kThreads, 1, 1);
    cfg.dynamicSmemBytes = G::kSmem;
    cfg.stream = s;
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = G::C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cfg;
}

// Query (a == nullptr: fills info, max_clusters from the occupancy API) or
// launch ceil(J / a->wpc) clusters (a->wpc must be even).
template <int N>
cudaError_t agent_pair(const AgentArgs* a, int amp_f16, cudaStream_t s, AgentPlanInfo* info) {
    using G = PairGeom<N>;
    void (*fn)(const AgentArgs) = amp_f16 ? agent_pair_kernel<N, 1> : agent_pair_kernel<N, 0>;
    cudaError_t e = xpose_attributes(fn, G::kSmem, G::C);
    if (a == nullptr) {
        // The occupancy API counts a kernel that allocates TMEM as one CTA
        // per SM; kTmCols per CTA fit the resident CTAs (static_assert), so
        // ask about the same kernel without the TMEM cache.
        void (*twin)(const AgentArgs) = agent_pair_kernel<N, 0, false>;
        cudaError_t et = xpose_attributes(twin, G::kSmem, G::C);
        info->threads = G::kThreads;
        info->smem_bytes = G::kSmem;
        info->max_clusters = 0;
        if (e == cudaSuccess && et == cudaSuccess) {
            cudaLaunchAttribute attr[1];
            cudaLaunchConfig_t cfg = pair_config<N>(64, nullptr, attr);
            int n = 0;
            if (cudaOccupancyMaxActiveClusters(&n, twin, &cfg) == cudaSuccess) info->max_clusters = n;
        }
        cudaGetLastError();
        info->launchable = info->max_clusters > 0;
        return cudaSuccess;
    }
    if (e != cudaSuccess) return e;
    if (a->wpc <= 0 || (a->wpc & 1)) return cudaErrorInvalidValue;
    const int nclusters = (a->J + a->wpc - 1) / a->wpc;
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = pair_config<N>(nclusters, s, attr);
    return cudaLaunchKernelEx(&cfg, fn, *a);
}

template <int N>
cudaError_t agent_pair_batched(const AgentArgs* descs, const int2* work, int nclusters, int amp_f16,
                               cudaStream_t s) {
    using G = PairGeom<N>;
    if (nclusters <= 0) return cudaSuccess;
    void (*fn)(const AgentArgs*, const int2*) =
        amp_f16 ? agent_pair_kernel_batched<N, 1> : agent_pair_kernel_batched<N, 0>;
    cudaError_t e = xpose_attributes(fn, G::kSmem, G::C);
    if (e != cudaSuccess) return e;
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = pair_config<N>(nclusters, s, attr);
    return cudaLaunchKernelEx(&cfg, fn, descs, work);
}

}  // namespace pmace
