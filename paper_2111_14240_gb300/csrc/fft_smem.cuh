// Register butterflies and in-place shared-memory FFT stages for the agent
// kernel.  The 2-D orthonormal DFT F of Section II is applied as a sequence
// of in-place radix-r stages: decimation in frequency (DIF, butterfly then
// twiddle) for the forward transform, which leaves the spectrum in
// digit-reversed order, and decimation in time (DIT, conjugate twiddle then
// inverse butterfly) in the reverse stage order for F^*, which takes the
// digit-reversed spectrum back to natural order.  The magnitude replacement
// between them is pointwise, so no reordering pass is ever needed; the
// measured amplitudes are stored in the same digit-reversed order once, at
// job creation.
#pragma once

#include <cuda_runtime.h>
#include <cooperative_groups.h>

namespace pmace {

// Complex addition and subtraction as one packed FP32 instruction (sm_100
// and later: two lanes, each rounded exactly as the scalar instruction).
__device__ __forceinline__ float2 operator+(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 operator-(float2 a, float2 b) { return __fadd2_rn(a, make_float2(-b.x, -b.y)); }
// a + rot(b) and a - rot(b) with rot = -i (forward) or +i (inverse), in
// scalar form: the rotation swaps the lanes of b, which a packed
// instruction cannot absorb.
template <bool INV>
__device__ __forceinline__ float2 add_rot(float2 a, float2 b) {
    return INV ? make_float2(a.x - b.y, a.y + b.x) : make_float2(a.x + b.y, a.y - b.x);
}
template <bool INV>
__device__ __forceinline__ float2 sub_rot(float2 a, float2 b) {
    return INV ? make_float2(a.x + b.y, a.y - b.x) : make_float2(a.x - b.y, a.y + b.x);
}
// c + k a on both lanes (k real)
__device__ __forceinline__ float2 fma_real(float k, float2 a, float2 c) { return __ffma2_rn(a, make_float2(k, k), c); }
__device__ __forceinline__ float2 operator*(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
// a * conj(b)
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.y, b.x, -a.x * b.y));
}

// cos(2 pi m / 32) for m = 0..31, built from cos(pi k / 16), k = 0..8, given
// as decimal values of the mathematical constants (rounded at compile time).
__host__ __device__ constexpr double k_cos32(int m) {
    constexpr double c[9] = {1.0,
                             0.98078528040323044913,
                             0.92387953251128675613,
                             0.83146961230254523708,
                             0.70710678118654752440,
                             0.55557023301960222474,
                             0.38268343236508977173,
                             0.19509032201612826785,
                             0.0};
    const int k = m & 31;                        // angle 2 pi k / 32 = pi k / 16
    return k <= 8 ? c[k] : k <= 16 ? -c[16 - k] : k <= 24 ? -c[k - 16] : c[32 - k];
}
__host__ __device__ constexpr double k_sin32(int m) { return k_cos32((m + 24) & 31); }

// a * W_D^M with W_D = exp(-2 pi i / D) (forward) or exp(+2 pi i / D) (INV),
// D in {2, 4, 8, 16, 32}; trivial factors are applied without multiplications.
template <int M, int D, bool INV>
__device__ __forceinline__ float2 twiddle(float2 a) {
    constexpr int m = (M * (32 / D)) & 31;      // in units of 2 pi / 32
    if constexpr (m == 0) {
        return a;
    } else if constexpr (m == 16) {
        return make_float2(-a.x, -a.y);
    } else if constexpr ((m == 8 && !INV) || (m == 24 && INV)) {
        return make_float2(a.y, -a.x);   // * (-i)
    } else if constexpr ((m == 24 && !INV) || (m == 8 && INV)) {
        return make_float2(-a.y, a.x);   // * (+i)
    } else {
        constexpr float c = (float)k_cos32(m);
        constexpr float s = INV ? (float)k_sin32(m) : -(float)k_sin32(m);
        return make_float2(fmaf(a.x, c, -a.y * s), fmaf(a.x, s, a.y * c));
    }
}

// In-register DFT of length R (2, 4, 8, 16, 32), natural order in and out:
// X[k] = sum_j x[j] exp(-+2 pi i j k / R).
template <int R, bool INV>
struct Dft;

template <bool INV>
struct Dft<2, INV> {
    __device__ __forceinline__ static void run(float2 (&x)[2]) {
        float2 a = x[0];
        x[0] = a + x[1];
        x[1] = a - x[1];
    }
};

template <bool INV>
struct Dft<4, INV> {
    __device__ __forceinline__ static void run(float2 (&x)[4]) {
        const float2 a = x[0] + x[2], b = x[0] - x[2], c = x[1] + x[3], e = x[1] - x[3];
        x[0] = a + c;
        x[2] = a - c;
        x[1] = add_rot<INV>(b, e);   // b + W_4 e
        x[3] = sub_rot<INV>(b, e);
    }
};

// Four-step split R = R1 * R2 with index maps j = R2*j1 + j2, k = k1 + R1*k2:
// X[k1 + R1 k2] = sum_j2 W_R2^{j2 k2} W_R^{j2 k1} sum_j1 x[R2 j1 + j2] W_R1^{j1 k1}.
template <int R1, int R2, bool INV>
struct FourStep {
    static constexpr int R = R1 * R2;
    template <int J2>
    __device__ __forceinline__ static void inner(const float2 (&x)[R], float2 (&t)[R]) {
        float2 s[R1];
#pragma unroll
        for (int j1 = 0; j1 < R1; ++j1) s[j1] = x[R2 * j1 + J2];
        Dft<R1, INV>::run(s);
        apply_tw<J2, 0>(s, t);
    }
    template <int J2, int K1>
    __device__ __forceinline__ static void apply_tw(const float2 (&s)[R1], float2 (&t)[R]) {
        if constexpr (K1 < R1) {
            t[J2 * R1 + K1] = twiddle<J2 * K1, R, INV>(s[K1]);
            apply_tw<J2, K1 + 1>(s, t);
        }
    }
    template <int J2>
    __device__ __forceinline__ static void all_inner(const float2 (&x)[R], float2 (&t)[R]) {
        if constexpr (J2 < R2) {
            inner<J2>(x, t);
            all_inner<J2 + 1>(x, t);
        }
    }
    __device__ __forceinline__ static void run(float2 (&x)[R]) {
        float2 t[R];
        all_inner<0>(x, t);
#pragma unroll
        for (int k1 = 0; k1 < R1; ++k1) {
            float2 s[R2];
#pragma unroll
            for (int j2 = 0; j2 < R2; ++j2) s[j2] = t[j2 * R1 + k1];
            Dft<R2, INV>::run(s);
#pragma unroll
            for (int k2 = 0; k2 < R2; ++k2) x[k1 + R1 * k2] = s[k2];
        }
    }
};

// Radix 8 as 4 x 2 (index j = 2 j1 + j2, k = k1 + 4 k2): radix-4 over j1
// for j2 = 0, 1, the factors W_8^k1 on the odd half, radix 2 over j2.  The
// factor 1/sqrt(2) of W_8^1 and W_8^3 rides on the fused multiply-adds of
// the radix-2 step: W_8^1 s = r (P, -M) forward and r (M, P) inverse,
// W_8^3 s = r (-M, -P) forward and r (-P, M) inverse, with P = s.x + s.y,
// M = s.x - s.y.
template <bool INV>
struct Dft<8, INV> {
    __device__ __forceinline__ static void run(float2 (&x)[8]) {
        constexpr float r = 0.70710678118654752440f;
        float2 t[4] = {x[0], x[2], x[4], x[6]};
        float2 s[4] = {x[1], x[3], x[5], x[7]};
        Dft<4, INV>::run(t);
        Dft<4, INV>::run(s);
        x[0] = t[0] + s[0];
        x[4] = t[0] - s[0];
        x[2] = add_rot<INV>(t[2], s[2]);
        x[6] = sub_rot<INV>(t[2], s[2]);
        {
            const float P = s[1].x + s[1].y, M = s[1].x - s[1].y;
            if (INV) {
                x[1] = make_float2(fmaf(M, r, t[1].x), fmaf(P, r, t[1].y));
                x[5] = make_float2(fmaf(M, -r, t[1].x), fmaf(P, -r, t[1].y));
            } else {
                x[1] = make_float2(fmaf(P, r, t[1].x), fmaf(M, -r, t[1].y));
                x[5] = make_float2(fmaf(P, -r, t[1].x), fmaf(M, r, t[1].y));
            }
        }
        {
            const float P = s[3].x + s[3].y, M = s[3].x - s[3].y;
            if (INV) {
                x[3] = make_float2(fmaf(P, -r, t[3].x), fmaf(M, r, t[3].y));
                x[7] = make_float2(fmaf(P, r, t[3].x), fmaf(M, -r, t[3].y));
            } else {
                x[3] = make_float2(fmaf(M, -r, t[3].x), fmaf(P, -r, t[3].y));
                x[7] = make_float2(fmaf(M, r, t[3].x), fmaf(P, r, t[3].y));
            }
        }
    }
};

// Radix 16: the four-step split 4 x 4, with the inner twiddles folded into
// the second radix-4 pass.  Every nontrivial W_16^m (m = j2 k1 in {1, 2, 3,
// 6, 9}) is a real scale times a factor whose parts are +-1 or +-tan(pi/8):
//   W^1 = c (1 - i t),  W^3 = c (t - i),  W^9 = c (-1 + i t),
//   W^2 = r (1 - i),    W^6 = r (-1 - i),  W^4 = -i
// (forward; F^* takes the conjugates), c = cos(pi/8), t = tan(pi/8),
// r = 1/sqrt(2).  The factors cost two adds or two fused multiply-adds a
// coefficient, and the scales ride on the multiply-adds of the pass that
// follows (its inputs 1 and 3 share one scale): 144 instructions instead of
// 160 for the plain four-step form.
template <bool INV>
struct Dft<16, INV> {
    static constexpr float kC = 0.92387953251128675613f;   // cos(pi/8)
    static constexpr float kT = 0.41421356237309504880f;   // tan(pi/8) = sqrt(2) - 1
    static constexpr float kR = 0.70710678118654752440f;   // 1/sqrt(2)
    static constexpr float sg = INV ? 1.0f : -1.0f;         // sign of the twiddles' imaginary parts

    // a * (p + i q) for q = sg * kT (p = 1) or p = kT (q = sg): two FMAs
    __device__ __forceinline__ static float2 by_w1(float2 a) {   // (1 + i sg t)
        return make_float2(fmaf(-sg * kT, a.y, a.x), fmaf(sg * kT, a.x, a.y));
    }
    __device__ __forceinline__ static float2 by_w3(float2 a) {   // (t + i sg)
        return make_float2(fmaf(kT, a.x, -sg * a.y), fmaf(kT, a.y, sg * a.x));
    }
    __device__ __forceinline__ static float2 by_w9(float2 a) {   // (-1 - i sg t)
        return make_float2(fmaf(sg * kT, a.y, -a.x), fmaf(-sg * kT, a.x, -a.y));
    }
    __device__ __forceinline__ static float2 by_w2(float2 a) {   // (1 + i sg)
        return INV ? make_float2(a.x - a.y, a.y + a.x) : make_float2(a.x + a.y, a.y - a.x);
    }
    __device__ __forceinline__ static float2 by_w6(float2 a) {   // (-1 + i sg)
        return INV ? make_float2(-a.x - a.y, a.x - a.y) : make_float2(a.y - a.x, -a.x - a.y);
    }
    // (-+ i) a: the radix-4 rotation
    __device__ __forceinline__ static float2 rot(float2 a) {
        return INV ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
    }
    // Radix-4 DFT of (i0, k2 * u2, k13 * u1, k13 * u3) into x[k1 + 4 k2];
    // ROT2: the second input is rot(u2) with k2 = 1 (u2 is passed with its
    // lanes unswapped; the rotation goes into scalar instructions)
    template <int K1, bool ROT2 = false>
    __device__ __forceinline__ static void pass2(float2 (&x)[16], float2 i0, float2 u1, float2 u2, float2 u3,
                                                 float k2, float k13) {
        float2 a, b;
        if constexpr (ROT2) {
            a = add_rot<INV>(i0, u2);
            b = sub_rot<INV>(i0, u2);
        } else {
            a = fma_real(k2, u2, i0);
            b = fma_real(-k2, u2, i0);
        }
        const float2 c = u1 + u3;
        const float2 e = u1 - u3;   // d = rot(e)
        x[K1] = fma_real(k13, c, a);
        x[K1 + 8] = fma_real(-k13, c, a);
        x[K1 + 4] = INV ? make_float2(fmaf(-k13, e.y, b.x), fmaf(k13, e.x, b.y))
                        : make_float2(fmaf(k13, e.y, b.x), fmaf(-k13, e.x, b.y));
        x[K1 + 12] = INV ? make_float2(fmaf(k13, e.y, b.x), fmaf(-k13, e.x, b.y))
                         : make_float2(fmaf(-k13, e.y, b.x), fmaf(k13, e.x, b.y));
    }
    __device__ __forceinline__ static void run(float2 (&x)[16]) {
        // first pass: t[j2][k1] = sum_j1 x[4 j1 + j2] W_4^(j1 k1)
        float2 t[4][4];
#pragma unroll
        for (int j2 = 0; j2 < 4; ++j2) {
            float2 s[4] = {x[j2], x[4 + j2], x[8 + j2], x[12 + j2]};
            Dft<4, INV>::run(s);
#pragma unroll
            for (int k1 = 0; k1 < 4; ++k1) t[j2][k1] = s[k1];
        }
        // second pass over j2, twiddle W_16^(j2 k1) folded in
        {
            float2 s[4] = {t[0][0], t[1][0], t[2][0], t[3][0]};
            Dft<4, INV>::run(s);
#pragma unroll
            for (int k2 = 0; k2 < 4; ++k2) x[4 * k2] = s[k2];
        }
        pass2<1>(x, t[0][1], by_w1(t[1][1]), by_w2(t[2][1]), by_w3(t[3][1]), kR, kC);
        pass2<2, true>(x, t[0][2], by_w2(t[1][2]), t[2][2], by_w6(t[3][2]), 1.0f, kR);
        pass2<3>(x, t[0][3], by_w3(t[1][3]), by_w6(t[2][3]), by_w9(t[3][3]), kR, kC);
    }
};

template <bool INV>
struct Dft<32, INV> {
    __device__ __forceinline__ static void run(float2 (&x)[32]) { FourStep<8, 4, INV>::run(x); }
};

// Padded shared-memory column index: one float2 of padding after every 16,
// which makes the stride-16 accesses of the short-span stages conflict free.
__device__ __forceinline__ int pcol(int c) { return c + (c >> 4); }
template <int N>
struct TileGeom {
    static constexpr int RS = N + N / 16;  // padded row stride in float2
};

// Distributed shared memory access through 32-bit shared::cluster addresses.
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
// Address of the same shared-memory location in CTA `rank` of the cluster.
__device__ __forceinline__ uint32_t cluster_addr(uint32_t local, uint32_t rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(local), "r"(rank));
    return r;
}
__device__ __forceinline__ float2 ld_cluster(uint32_t addr) {
    float2 v;
    asm volatile("ld.shared::cluster.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(addr) : "memory");
    return v;
}
__device__ __forceinline__ void st_cluster(uint32_t addr, float2 v) {
    asm volatile("st.shared::cluster.v2.f32 [%0], {%1, %2};" ::"r"(addr), "f"(v.x), "f"(v.y) : "memory");
}

// The column-axis stage of span N and radix C across the C CTAs of a
// cluster: CTA k holds global rows [k*NROWS, (k+1)*NROWS), so the butterfly
// at local row b combines row b of every CTA.  Each CTA takes NROWS/C of the
// butterflies, reading and writing the peers' tiles through distributed
// shared memory; a butterfly's elements are read and written by one thread
// only, so the stage is in place without staging.  `tile` is this CTA's
// tile; the peers' copies are addressed through mapa.
// The tile may hold several windows of WR rows each (NROWS = windows * WR);
// the twiddle of local row b is that of row b % WR of its window.
template <int N, int NROWS, int WR, int C, bool INV, int T>
__device__ __forceinline__ void cross_stage(const float2* tile, const float2* __restrict__ tw, int rank) {
    constexpr int RS = TileGeom<N>::RS;
    constexpr int BR = NROWS / C;         // butterfly rows per CTA
    constexpr int NB = BR * N;            // butterflies per CTA
    static_assert(NB % T == 0, "butterflies must split evenly over threads");
    constexpr int PER = NB / T;           // butterflies per thread
    // butterflies whose remote loads are issued together (up to 16 values in flight)
    constexpr int BB = (16 / C) < PER ? (16 / C > 0 ? 16 / C : 1) : PER;
    static_assert(PER % BB == 0, "butterfly batches must divide the per-thread count");
    const uint32_t mine = smem_addr(tile);
#pragma unroll 1
    for (int p0 = 0; p0 < PER; p0 += BB) {
        float2 x[BB][C];
        uint32_t off[BB];
        int bidx[BB];
#pragma unroll
        for (int i = 0; i < BB; ++i) {
            const int t = threadIdx.x + (p0 + i) * T;
            const int col = t % N;
            bidx[i] = rank * BR + t / N;
            off[i] = (uint32_t)(bidx[i] * RS + pcol(col)) * (uint32_t)sizeof(float2);
#pragma unroll
            for (int k = 0; k < C; ++k) x[i][k] = ld_cluster(cluster_addr(mine + off[i], (uint32_t)k));
        }
#pragma unroll
        for (int i = 0; i < BB; ++i) {
            const int b = bidx[i] % WR;
            if constexpr (INV) {
#pragma unroll
                for (int k = 1; k < C; ++k) x[i][k] = cmulc(x[i][k], tw[b * k]);
                Dft<C, true>::run(x[i]);
            } else {
                Dft<C, false>::run(x[i]);
#pragma unroll
                for (int k = 1; k < C; ++k) x[i][k] = cmul(x[i][k], tw[b * k]);
            }
#pragma unroll
            for (int k = 0; k < C; ++k) st_cluster(cluster_addr(mine + off[i], (uint32_t)k), x[i][k]);
        }
    }
}

}  // namespace pmace
