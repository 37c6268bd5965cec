// Support kernels of the PMACE hot path: the pixel-owner consensus gather
// (step S6, equation xjbar), the weight image Lambda, the Algorithm 1
// readout, the amplitude layout pass, the deterministic FP64 reduction of the
// residual partials, and the stack initialisation of Algorithm 1.
#include "pmace_internal.h"
#include "cache_hints.cuh"

#include <cuda_fp16.h>

namespace pmace {

// ---------------------------------------------------------------------------
// Pixel-owner gather over the scan-overlap lists.  The image is cut into
// TH x kGatherTileW tiles; every tile has the ascending list of the windows
// that intersect it, cut into runs ("units", one CTA each) of windows of the
// same index block i / B.  Every pixel sums |d(p - o_i)|^kappa * src_i(p - o_i)
// over the windows i that contain it, in ascending i within a block and then
// over the blocks in ascending order (a block with no such window adds an
// exact 0), so the result is deterministic, the same for every tile height,
// and needs no float atomics.
//   MODE 0: Lambda = sum_i |d|^kappa (FP64), writes Lambda^-1 (0 where Lambda = 0)
//   MODE 1: xbar = Lambda^-1 sum_i P_i^t |D|^kappa u_i                 (G, S6)
//   MODE 2: x_hat = Lambda^-1 sum_i P_i^t |D|^kappa q_i + 2 rho xbar   (readout)
// A tile cut into several units: each unit stores its partial sums in its
// scratch slot, fences, and counts itself in the tile's counter; the unit
// that brings the counter to the tile's unit count resets it to 0, reads
// the slots back from L2 in ascending order and writes the pixels.
// ---------------------------------------------------------------------------
template <int MODE, int TH>
__device__ __forceinline__ void gather_body(const GatherArgs& g, const int unit) {
    constexpr int TW = kGatherTileW;
    constexpr int NT = gather_threads(TH);
    constexpr int RPT = kGatherRowsPerThread;       // rows per thread
    static_assert(NT >= kGatherStage, "one thread stages one window of a chunk");
    __shared__ int s_i[kGatherStage];
    __shared__ int2 s_o[kGatherStage];
    __shared__ int s_last;

    const int4 un = __ldg(g.units + unit);          // (tile, lb, le, slot)
#ifdef PMACE_DEBUG
    // the unit must lie inside the tables (else the CTA flags it and stops)
    if (un.x < 0 || un.x >= g.ntiles || un.y < 0 || un.y > un.z || un.z > g.list_len || un.w < -1 ||
        un.w >= g.nslots) {
        if (threadIdx.x == 0) atomicOr(g.err, kErrBoundsBit);
        return;
    }
#endif
    const int tile = un.x;
    const int ty0 = (tile / g.tiles_x) * TH, tx0 = (tile % g.tiles_x) * TW;
    const int lane = threadIdx.x % TW, grp = threadIdx.x / TW;
    const int px = tx0 + lane;
    const int np = g.np;
    const size_t P = (size_t)np * np;

    const uint64_t pol_first = l2_policy_evict_first();   // u: this is its last read
    using Acc = typename std::conditional<MODE == 0, double, float2>::type;
    Acc acc[RPT];
#pragma unroll
    for (int r = 0; r < RPT; ++r) {
        if constexpr (MODE == 0) acc[r] = 0.0;
        else acc[r] = make_float2(0.f, 0.f);
    }
    for (int cb = un.y; cb < un.z; cb += kGatherStage) {
        const int n = min(kGatherStage, un.z - cb);
        if (cb != un.y) __syncthreads();            // the previous chunk is consumed
        if (threadIdx.x < n) {
            int i = __ldg(g.tile_list + cb + threadIdx.x);
#ifdef PMACE_DEBUG
            // a window index outside [0, J) or a corner outside the image is
            // flagged and the window left out (a corner far outside every tile)
            const bool bad_i = i < 0 || i >= g.J;
            if (bad_i) i = 0;
            int2 o = __ldg(g.offs + i);
            if (bad_i || o.x < 0 || o.x > g.n1 - np || o.y < 0 || o.y > g.n2 - np) {
                atomicOr(g.err, kErrBoundsBit);
                o = make_int2(-(1 << 29), -(1 << 29));
            }
            s_i[threadIdx.x] = i;
            s_o[threadIdx.x] = o;
#else
            s_i[threadIdx.x] = i;
            s_o[threadIdx.x] = __ldg(g.offs + i);
#endif
        }
        __syncthreads();
        // Windows are taken U at a time so that U * RPT loads are in flight
        // per thread; the accumulation still runs over ascending window index.
        // (U = 3 keeps 8 CTAs an SM; U = 4 with 7 was 4 % slower on the
        // 8192 x 8192 / 64009-window consensus, U = 8 with 4 CTAs 30 %.)
        constexpr int U = 3;
        for (int k0 = 0; k0 < n; k0 += U) {
            float wgt[U][RPT];
            float2 val[U][RPT];
#pragma unroll
            for (int k = 0; k < U; ++k) {
                const bool have = k0 + k < n;
                const int i = have ? s_i[k0 + k] : 0;
                const int2 o = have ? s_o[k0 + k] : make_int2(-(1 << 29), -(1 << 29));
                const int lx = px - o.y;
                const bool inx = have && (unsigned)lx < (unsigned)np;
#pragma unroll
                for (int r = 0; r < RPT; ++r) {
                    const int py = ty0 + grp + r * (NT / TW);
                    const int ly = py - o.x;
                    wgt[k][r] = 0.f;
                    val[k][r] = make_float2(0.f, 0.f);
                    if (inx && (unsigned)ly < (unsigned)np) {
                        const int e = ly * np + lx;
                        wgt[k][r] = __ldg(g.wk + e);
                        if constexpr (MODE == 1) val[k][r] = ld_nc_l2_hint(g.src + (size_t)i * P + e, pol_first);
                        else if constexpr (MODE == 2) val[k][r] = __ldg(g.src + (size_t)i * P + e);
                    }
                }
            }
#pragma unroll
            for (int k = 0; k < U; ++k) {
#pragma unroll
                for (int r = 0; r < RPT; ++r) {
                    if (wgt[k][r] != 0.f) {
                        if constexpr (MODE == 0) {
                            acc[r] += (double)wgt[k][r];
                        } else {
                            acc[r].x = fmaf(wgt[k][r], val[k][r].x, acc[r].x);
                            acc[r].y = fmaf(wgt[k][r], val[k][r].y, acc[r].y);
                        }
                    }
                }
            }
        }
    }
    if (un.w >= 0) {                                 // tile split over several units
        Acc* mine = reinterpret_cast<Acc*>(g.scratch) + (size_t)un.w * (TH * TW);
#pragma unroll
        for (int r = 0; r < RPT; ++r) mine[r * NT + threadIdx.x] = acc[r];
        __threadfence();
        __syncthreads();
        const int2 ts = __ldg(g.tile_seg + tile);    // (first slot, units)
        if (threadIdx.x == 0) {
            const int done = atomicAdd(g.counters + tile, 1);
            s_last = done == ts.y - 1;
            if (s_last) g.counters[tile] = 0;        // every unit of the tile has counted
        }
        __syncthreads();
        if (!s_last) return;
        __threadfence();
        const Acc* part = reinterpret_cast<const Acc*>(g.scratch) + (size_t)ts.x * (TH * TW);
#pragma unroll
        for (int r = 0; r < RPT; ++r) acc[r] = __ldcg(part + r * NT + threadIdx.x);
        for (int sl = 1; sl < ts.y; ++sl) {
#pragma unroll
            for (int r = 0; r < RPT; ++r) {
                const Acc v = __ldcg(part + (size_t)sl * (TH * TW) + r * NT + threadIdx.x);
                if constexpr (MODE == 0) {
                    acc[r] += v;
                } else {
                    acc[r].x += v.x;
                    acc[r].y += v.y;
                }
            }
        }
    }
    if (px >= g.n2) return;
#pragma unroll
    for (int r = 0; r < RPT; ++r) {
        const int py = ty0 + grp + r * (NT / TW);
        if (py >= g.n1) continue;
        const size_t p = (size_t)py * g.n2 + px;
        if constexpr (MODE == 0) {
            g.lam_out[p] = acc[r] > 0.0 ? (float)(1.0 / acc[r]) : 0.f;
        } else {
            const float li = __ldg(g.laminv + p);
            float2 v = make_float2(acc[r].x * li, acc[r].y * li);
            if constexpr (MODE == 2) {
                const float2 xb = __ldg(g.xbar_in + p);
                v.x = fmaf(g.two_rho, xb.x, v.x);
                v.y = fmaf(g.two_rho, xb.y, v.y);
            }
            g.out[p] = v;
        }
    }
}

template <int MODE, int TH>
__global__ void __launch_bounds__(gather_threads(TH)) gather_kernel(const __grid_constant__ GatherArgs g) {
    gather_body<MODE, TH>(g, blockIdx.x);
}

// Several jobs' units in one launch: CTA k gathers unit work[k].y of job work[k].x.
template <int MODE, int TH>
__global__ void __launch_bounds__(gather_threads(TH))
gather_kernel_batched(const GatherArgs* __restrict__ descs, const int2* __restrict__ work) {
    const int2 w = work[blockIdx.x];
    gather_body<MODE, TH>(descs[w.x], w.y);
}

template <int MODE>
static cudaError_t launch_gather(const GatherArgs& g, int nunits, int tile_h, cudaStream_t s) {
    if (nunits <= 0) return cudaSuccess;
    switch (tile_h) {
        case 8: gather_kernel<MODE, 8><<<nunits, gather_threads(8), 0, s>>>(g); break;
        case 16: gather_kernel<MODE, 16><<<nunits, gather_threads(16), 0, s>>>(g); break;
        case 32: gather_kernel<MODE, 32><<<nunits, gather_threads(32), 0, s>>>(g); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}
cudaError_t launch_gather_weights(const GatherArgs& g, int n, int th, cudaStream_t s) { return launch_gather<0>(g, n, th, s); }
cudaError_t launch_gather_consensus(const GatherArgs& g, int n, int th, cudaStream_t s) { return launch_gather<1>(g, n, th, s); }
cudaError_t launch_gather_readout(const GatherArgs& g, int n, int th, cudaStream_t s) { return launch_gather<2>(g, n, th, s); }

cudaError_t launch_gather_consensus_batched(const GatherArgs* descs, const int2* work, int nunits, int tile_h,
                                            cudaStream_t s) {
    if (nunits <= 0) return cudaSuccess;
    switch (tile_h) {
        case 8: gather_kernel_batched<1, 8><<<nunits, gather_threads(8), 0, s>>>(descs, work); break;
        case 16: gather_kernel_batched<1, 16><<<nunits, gather_threads(16), 0, s>>>(descs, work); break;
        case 32: gather_kernel_batched<1, 32><<<nunits, gather_threads(32), 0, s>>>(descs, work); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Amplitudes to the agent kernel's layout: y_k[j][e] = y[j][layout[e]], where
// layout[e] is the natural index (frequency row * np + frequency column) of
// stored position e (the digit-reversed order the in-place DIF stages leave
// the spectrum in, in the agent variant's thread order), validating
// finiteness and sign, and FP64 partial sums of y^2 per block.
// ---------------------------------------------------------------------------
constexpr int kPrepThreads = 256;

template <int F16>
__global__ void __launch_bounds__(kPrepThreads)
prep_amps_kernel(const void* __restrict__ in, const float* __restrict__ scales, void* __restrict__ out,
                 const int* __restrict__ layout, int J, int np, double* __restrict__ partials,
                 int* __restrict__ err) {
    const size_t P = (size_t)np * np;
    const size_t total = (size_t)J * P;
    double s = 0.0;
    int bad = 0;
    for (size_t idx = (size_t)blockIdx.x * kPrepThreads + threadIdx.x; idx < total;
         idx += (size_t)gridDim.x * kPrepThreads) {
        const size_t j = idx / P;
        const int e = (int)(idx % P);
        const size_t src = j * P + (size_t)layout[e];
        float v;
        if constexpr (F16) {
            const __half h = static_cast<const __half*>(in)[src];
            const float sc = scales[j];
            const float hv = __half2float(h);
            if (!(hv >= 0.f) || !(sc >= 0.f) || isinf(hv) || isinf(sc)) bad = 1;
            static_cast<__half*>(out)[idx] = h;
            v = hv * sc;
        } else {
            v = static_cast<const float*>(in)[src];
            if (!(v >= 0.f) || isinf(v)) bad = 1;
            static_cast<float*>(out)[idx] = v;
        }
        s += (double)v * (double)v;
    }
    if (bad) atomicOr(err, 1);
    __shared__ double red[kPrepThreads];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = kPrepThreads / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) partials[blockIdx.x] = red[0];
}

cudaError_t launch_prep_amps(const void* amps_in, int amp_f16, const float* scales, void* y_out,
                             const int* layout, int J, int np, double* partials, int* err, int nblocks,
                             cudaStream_t s) {
    if (amp_f16)
        prep_amps_kernel<1><<<nblocks, kPrepThreads, 0, s>>>(amps_in, scales, y_out, layout, J, np, partials, err);
    else
        prep_amps_kernel<0><<<nblocks, kPrepThreads, 0, s>>>(amps_in, scales, y_out, layout, J, np, partials, err);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Fixed-order FP64 reduction of an [nrows][ncols] table of partial sums
// (ncols <= 4): out[c] = sum_r partials[r][c].  One CTA; each thread sums a
// strided subset in order, then a fixed tree.  Deterministic run to run.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256)
reduce_partials_kernel(const double* __restrict__ p, int nrows, int ncols, double* __restrict__ out) {
    __shared__ double red[256][4];
    double s[4] = {0, 0, 0, 0};
    for (int r = threadIdx.x; r < nrows; r += 256) {
        for (int c = 0; c < ncols; ++c) s[c] += p[(size_t)r * ncols + c];
    }
    for (int c = 0; c < 4; ++c) red[threadIdx.x][c] = s[c];
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            for (int c = 0; c < 4; ++c) red[threadIdx.x][c] += red[threadIdx.x + o][c];
        }
        __syncthreads();
    }
    if (threadIdx.x < ncols) out[threadIdx.x] = red[0][threadIdx.x];
}

cudaError_t launch_reduce_partials(const double* partials, int nrows, int ncols, double* out,
                                   cudaStream_t s) {
    reduce_partials_kernel<<<1, 256, 0, s>>>(partials, nrows, ncols, out);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Algorithm 1 initialisation w = v = [P_j x^(0)]_j, stored as the pending
// stack q (the consensus image starts at 0, so v = q + 2 rho P xbar = q).
// init == NULL means the constant image cval.
// ---------------------------------------------------------------------------
__global__ void init_stack_kernel(float2* __restrict__ q, const float2* __restrict__ init, float2 cval,
                                  const int2* __restrict__ offs, int J, int np, int n2) {
    const size_t P = (size_t)np * np;
    const size_t total = (size_t)J * P;
    for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (size_t)gridDim.x * blockDim.x) {
        if (init == nullptr) {
            q[idx] = cval;
        } else {
            const size_t j = idx / P;
            const int e = (int)(idx % P);
            const int2 o = offs[j];
            q[idx] = init[(size_t)(o.x + e / np) * n2 + (o.y + e % np)];
        }
    }
}

cudaError_t launch_init_stack(float2* q, const float2* init, float2 cval, const int2* offs, int J,
                              int np, int n2, cudaStream_t s) {
    init_stack_kernel<<<1216, 256, 0, s>>>(q, init, cval, offs, J, np, n2);
    return cudaGetLastError();
}

// v = q + 2 rho P_j xbar, the current Algorithm 1 stack.
__global__ void patches_kernel(const float2* __restrict__ q, const float2* __restrict__ xbar,
                               const int2* __restrict__ offs, float2* __restrict__ v, int J, int np,
                               int n1, int n2, float two_rho, int* __restrict__ err) {
    const size_t P = (size_t)np * np;
    const size_t total = (size_t)J * P;
    for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (size_t)gridDim.x * blockDim.x) {
        const size_t j = idx / P;
        const int e = (int)(idx % P);
        int2 o = offs[j];
#ifdef PMACE_DEBUG
        if (o.x < 0 || o.x > n1 - np || o.y < 0 || o.y > n2 - np) {
            atomicOr(err, kErrBoundsBit);
            o = make_int2(min(max(o.x, 0), n1 - np), min(max(o.y, 0), n2 - np));
        }
#endif
        const float2 xb = xbar[(size_t)(o.x + e / np) * n2 + (o.y + e % np)];
        const float2 qv = q[idx];
        v[idx] = make_float2(fmaf(two_rho, xb.x, qv.x), fmaf(two_rho, xb.y, qv.y));
    }
}

cudaError_t launch_patches_from_state(const float2* q, const float2* xbar, const int2* offs,
                                      float2* v, int J, int np, int n1, int n2, float two_rho,
                                      int* err, cudaStream_t s) {
    patches_kernel<<<1216, 256, 0, s>>>(q, xbar, offs, v, J, np, n1, n2, two_rho, err);
    return cudaGetLastError();
}

// Per-window permutation of a [J][np * np] stack of elem-byte values:
// dst[j][e] = src[j][map[e]] (elem 2, 4 or 8).
template <typename E>
__global__ void relayout_window_kernel(E* __restrict__ dst, const E* __restrict__ src, const int* __restrict__ map,
                                       int J, int np) {
    const size_t P = (size_t)np * np, total = (size_t)J * P;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const size_t j = i / P;
        dst[i] = src[j * P + map[i % P]];
    }
}

cudaError_t launch_relayout_window(void* dst, const void* src, const int* map, int J, int np, int elem,
                                   cudaStream_t s) {
    if (elem == 2)
        relayout_window_kernel<unsigned short><<<1216, 256, 0, s>>>(static_cast<unsigned short*>(dst),
                                                                    static_cast<const unsigned short*>(src), map, J, np);
    else if (elem == 4)
        relayout_window_kernel<float><<<1216, 256, 0, s>>>(static_cast<float*>(dst), static_cast<const float*>(src),
                                                           map, J, np);
    else if (elem == 8)
        relayout_window_kernel<float2><<<1216, 256, 0, s>>>(static_cast<float2*>(dst), static_cast<const float2*>(src),
                                                            map, J, np);
    else
        return cudaErrorInvalidValue;
    return cudaGetLastError();
}

__global__ void check_finite_kernel(const float* __restrict__ d, int64_t n, int* __restrict__ err) {
    int bad = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        if (!isfinite(d[i])) bad = 1;
    }
    if (bad) atomicOr(err, 2);
}

cudaError_t launch_check_finite(const float* data, int64_t n, int* err, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    check_finite_kernel<<<304, 256, 0, s>>>(data, n, err);
    return cudaGetLastError();
}

}  // namespace pmace
