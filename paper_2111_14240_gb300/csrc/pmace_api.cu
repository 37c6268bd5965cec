// Host runtime and C ABI of the PMACE hot path (declared in include/pmace.h).
//
// A job keeps its whole working set resident on one GPU:
//   q     [J][Np][Np] complex64  pending Mann stack q = v - 2 rho w
//   u     [J][Np][Np] complex64  agent reflection u = 2w - v (input of G)
//   y     [J][Np][Np] f32 or f16 amplitudes, digit-reversed kernel order
//   xbar  [n1][n2]    complex64  consensus image of the last iteration
//   laminv[n1][n2]    f32        Lambda^-1 (0 where Lambda = 0)
// plus the probe tables (d, 1/d, |d|^kappa, twiddles) and the scan-overlap
// lists.  One iteration of Algorithm 1 is two launches: the fused agent
// sweep (agent.cuh) and the pixel-owner consensus gather (support.cu).
#include "pmace.h"
#include "job.h"
#include "pmace_internal.h"

#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>
#include <vector>

using namespace pmace;

namespace {

constexpr int kMaxCluster = 16;
constexpr int kPrepBlocks = 608;
constexpr int kGraphIters = 8;   // iterations per replay of the captured graph

thread_local std::string g_create_error;


}  // namespace


namespace {

pmace_status fail(pmace_job* h, pmace_status st, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    if (h) h->error = buf;
    else g_create_error = buf;
    return st;
}

pmace_status cuda_fail(pmace_job* h, cudaError_t e, const char* what) {
    return fail(h, e == cudaErrorMemoryAllocation ? PMACE_ERR_OOM : PMACE_ERR_CUDA, "%s: %s (%s)",
                what, cudaGetErrorName(e), cudaGetErrorString(e));
}

#define PM_CUDA(h, call)                                            \
    do {                                                            \
        cudaError_t e_ = (call);                                    \
        if (e_ != cudaSuccess) return cuda_fail((h), e_, #call);    \
    } while (0)

template <typename T>
cudaError_t dalloc(pmace_job* h, T** p, size_t count) {
    const size_t bytes = std::max<size_t>(count * sizeof(T), 16);
    cudaError_t e = cudaMalloc(reinterpret_cast<void**>(p), bytes);
    if (e == cudaSuccess) h->bytes += (int64_t)bytes;
    return e;
}

bool np_supported(int np) { return np == 32 || np == 64 || np == 128 || np == 256; }

cudaError_t agent_entry(int np, const AgentArgs* a, int variant, int amp, cudaStream_t s,
                        AgentPlanInfo* info) {
    switch (np) {
        case 32: return agent_entry_32(a, variant, amp, s, info);
        case 64: return agent_entry_64(a, variant, amp, s, info);
        case 128: return agent_entry_128(a, variant, amp, s, info);
        case 256: return agent_entry_256(a, variant, amp, s, info);
        default: return cudaErrorInvalidValue;
    }
}

// Agent variant to start from: PMACE_AGENT_PLAN (an index into
// agent_variant_of) when set and valid, else PMACE_AGENT_CLUSTER selects the
// first variant with that cluster size, else the probe size's default
// (default_agent_variant).
int default_variant(int np, int J) {
    if (const char* env = std::getenv("PMACE_AGENT_PLAN")) {
        const int v = std::atoi(env);
        if (v >= 0 && v < kAgentVariants) return v;
    }
    if (const char* env = std::getenv("PMACE_AGENT_CLUSTER")) {
        const int c = std::atoi(env);
        for (int v = 0; v < kAgentVariants; ++v)
            if (agent_variant_of(np, v).cluster == c) return v;
    }
    return default_agent_variant(np, J);
}

// Row order of the amplitudes for a cluster size: kernel row g holds
// frequency row (g / rows) + cluster * (g % rows), rows = np / cluster.
std::vector<int> column_order(int np, int cluster) {
    std::vector<int> perm(np);
    const int rows = np / cluster;
    for (int g = 0; g < np; ++g) perm[g] = g / rows + cluster * (g % rows);
    return perm;
}

// Frequency index held at each position after in-place DIF stages with the
// given radices (outer stage first): position k*(L/r) + p of a span-L block
// holds frequency k + r * (frequency of p in the span-L/r sub-transform).
void dif_order(const std::vector<int>& radices, size_t level, int L, std::vector<int>& out) {
    if (L == 1) {
        out.assign(1, 0);
        return;
    }
    const int r = radices[level];
    std::vector<int> sub;
    dif_order(radices, level + 1, L / r, sub);
    out.assign(L, 0);
    for (int k = 0; k < r; ++k)
        for (int p = 0; p < L / r; ++p) out[k * (L / r) + p] = k + r * sub[p];
}

std::vector<int> radices_of(int L) {
    const RadixPlan p = radix_plan(L);
    std::vector<int> v{p.first};
    if (p.second > 1) v.push_back(p.second);
    return v;
}

// Row order of the amplitudes for an agent variant: the in-place cross-CTA
// variants leave the column axis in column_order; the transposing exchange
// runs the same two DIF stages along columns as along rows, so both axes end
// in the DIF order.
std::vector<int> amp_row_order(int np, int variant) {
    const AgentVariant v = agent_variant_of(np, variant);
    if (!v.exchange) return column_order(np, v.cluster);
    std::vector<int> perm;
    dif_order(radices_of(np), 0, np, perm);
    return perm;
}

// Layout of one window's stored amplitudes for an agent variant: for every
// stored position, the natural index (frequency row * np + frequency
// column) of the amplitude held there.  The in-place cross-CTA variants
// store kernel rows (amp_row_order) of kernel columns (the DIF order of the
// row stages), row-major.  The exchange variants store each thread's values
// contiguously ("thread order"): CTA `rank` of the window's cluster reads
// the 16 amplitudes of its column-step butterflies as 16-byte chunks, chunk
// k of thread t at ((rank * chunks + k) * threads + t) * 16 bytes, so a warp
// loads 512 contiguous bytes per instruction.  Value f of a thread (f = u r2
// + i: butterfly u of the thread, element i) sits at kernel row
// m r2 + i, column 16 rank + c, with m = (t + u threads) / 16 and
// c = (t + u threads) % 16 (the column step's own indexing).
std::vector<int> amp_layout(int np, int variant, int elem) {
    const AgentVariant v = agent_variant_of(np, variant);
    const std::vector<int> rows = amp_row_order(np, variant);
    std::vector<int> cols;
    dif_order(radices_of(np), 0, np, cols);
    std::vector<int> out((size_t)np * np);
    if (!v.exchange) {
        for (int g = 0; g < np; ++g)
            for (int c = 0; c < np; ++c) out[(size_t)g * np + c] = rows[g] * np + cols[c];
        return out;
    }
    const RadixPlan rp = radix_plan(np);
    const int T = np, C = np / 16, U2 = 16 * rp.first / T, F = U2 * rp.second, CH = 16 / elem, NCH = F / CH;
    for (int rank = 0; rank < C; ++rank)
        for (int k = 0; k < NCH; ++k)
            for (int t = 0; t < T; ++t)
                for (int e = 0; e < CH; ++e) {
                    const int f = k * CH + e, u = f / rp.second, i = f % rp.second;
                    const int id = t + u * T, m = id / 16, c = id % 16;
                    const int g = m * rp.second + i, col = 16 * rank + c;
                    out[(((size_t)rank * NCH + k) * T + t) * CH + e] = rows[g] * np + cols[col];
                }
    return out;
}

// Windows each agent cluster processes: the variant's own count, or for the
// transposing exchange (a run of windows per cluster) J spread over four
// times the clusters the device holds at once, and at most 16: runs short
// enough that the clusters that finish early take up the remaining ones,
// which balances SMs that hold different numbers of CTAs, and long enough
// to amortise a cluster's start (TMEM and twiddle tables, the cluster
// barrier); on the 64009-window scan runs of 4, 8, 16 and 32 windows took
// 8.27, 8.03, 7.93 and 7.92 ms (PMACE_AGENT_WPC fixes the run).
// The packed-lane sweep counts in pairs of windows, so its runs are even.
int windows_per_cluster(int np, int variant, int J, const AgentPlanInfo& info) {
    const AgentVariant v = agent_variant_of(np, variant);
    if (!v.exchange) return v.windows;
    const int unit = v.exchange == 2 ? 2 : 1;   // the packed-lane sweep takes windows in pairs
    if (const char* env = std::getenv("PMACE_AGENT_WPC")) {   // fixed run length (rounded up to the unit)
        const int w = std::atoi(env);
        if (w > 0) return (w + unit - 1) / unit * unit;
    }
    const int m = 4 * std::max(info.max_clusters, 1) * unit;
    return unit * std::max(1, std::min(16 / unit, (J + m - 1) / m));
}

// Gather tables of one tile height: for every tile_h x kGatherTileW image
// tile the ascending list of the windows that intersect it (CSR: cnt[t] ..
// cnt[t + 1]), cut into units where the window index crosses a multiple of
// the job's block length B (windows [kB, (k+1)B) of the list form one
// unit).  Every pixel's sum is then the ascending-block sum of per-block
// partial sums, whatever the tile shape, so a job's results do not depend
// on the gather tile height.
struct GatherTables {
    int tile_h = 16, tiles_x = 0, tiles_y = 0, ntiles = 0, nslots = 0;
    std::vector<int> cnt, list;
    std::vector<int4> units;   // (tile, lb, le, slot or -1)
    std::vector<int2> seg;     // (first slot or -1, units) per tile
};

void overlap_lists(const pmace_dims& d, const std::vector<int32_t>& offs_h, GatherTables& t) {
    const int np = d.np, J = d.J;
    const int TH = t.tile_h, TW = kGatherTileW;
    t.tiles_y = (d.n1 + TH - 1) / TH;
    t.tiles_x = (d.n2 + TW - 1) / TW;
    t.ntiles = t.tiles_x * t.tiles_y;
    t.cnt.assign(t.ntiles + 1, 0);
    auto tile_range = [&](int j, int& y0, int& y1, int& x0, int& x1) {
        const int r = offs_h[2 * j], c = offs_h[2 * j + 1];
        y0 = r / TH;
        y1 = (r + np - 1) / TH;
        x0 = c / TW;
        x1 = (c + np - 1) / TW;
    };
    for (int j = 0; j < J; ++j) {
        int y0, y1, x0, x1;
        tile_range(j, y0, y1, x0, x1);
        for (int ty = y0; ty <= y1; ++ty)
            for (int tx = x0; tx <= x1; ++tx) t.cnt[ty * t.tiles_x + tx + 1]++;
    }
    for (int k = 0; k < t.ntiles; ++k) t.cnt[k + 1] += t.cnt[k];
    t.list.assign(std::max(t.cnt[t.ntiles], 1), 0);
    std::vector<int> fill(t.cnt.begin(), t.cnt.end() - 1);
    for (int j = 0; j < J; ++j) {   // ascending j, so every list is ascending
        int y0, y1, x0, x1;
        tile_range(j, y0, y1, x0, x1);
        for (int ty = y0; ty <= y1; ++ty)
            for (int tx = x0; tx <= x1; ++tx) t.list[fill[ty * t.tiles_x + tx]++] = j;
    }
}

// Units of the tables' lists for block length B (empty tiles keep one unit).
int64_t count_units(const GatherTables& t, int B) {
    int64_t n = 0;
    for (int k = 0; k < t.ntiles; ++k) {
        int64_t runs = 1;
        for (int a = t.cnt[k] + 1; a < t.cnt[k + 1]; ++a) runs += t.list[a] / B != t.list[a - 1] / B;
        n += runs;
    }
    return n;
}

void cut_units(GatherTables& t, int B) {
    t.seg.resize(t.ntiles);
    t.units.clear();
    t.units.reserve(t.ntiles);
    t.nslots = 0;
    for (int k = 0; k < t.ntiles; ++k) {
        const int lb = t.cnt[k], le = t.cnt[k + 1];
        const size_t first = t.units.size();
        int a = lb;
        do {
            int b = a + 1;
            while (b < le && t.list[b] / B == t.list[a] / B) ++b;
            t.units.push_back(make_int4(k, a, std::min(b, le), -1));
            a = b;
        } while (a < le);
        const int ns = (int)(t.units.size() - first);
        if (ns == 1) {
            t.seg[k] = make_int2(-1, 1);
        } else {
            t.seg[k] = make_int2(t.nslots, ns);
            for (int u = 0; u < ns; ++u) t.units[first + u].w = t.nslots + u;
            t.nslots += ns;
        }
    }
}

// Gather CTAs per launch the block length aims for: enough to fill the GPU
// several times over even when the image has few tiles, so that the long
// lists of interior tiles do not set the launch's duration.
constexpr int64_t kGatherTargetUnits = 3072;
// Fewest windows per unit on average the block length allows.
constexpr int64_t kGatherMinWindows = 16;

// The job's block length B: the smallest B whose cut of the 16-row tiles'
// lists gives at most max(tiles, min(kGatherTargetUnits, windows /
// kGatherMinWindows)) units (PMACE_GATHER_UNITS and PMACE_GATHER_SEG, if
// set, replace the two constants); J when the image alone has that many
// tiles.  A function of the job's scan alone.
int gather_block_length(const pmace_dims& d, const std::vector<int32_t>& offs_h) {
    GatherTables t;
    t.tile_h = 16;
    overlap_lists(d, offs_h, t);
    int64_t minw = kGatherMinWindows, units = kGatherTargetUnits;
    if (const char* env = std::getenv("PMACE_GATHER_SEG")) {
        const int v = std::atoi(env);
        if (v > 0) minw = v;
    }
    if (const char* env = std::getenv("PMACE_GATHER_UNITS")) {
        const int v = std::atoi(env);
        if (v > 0) units = v;
    }
    const int64_t total = t.cnt[t.ntiles];
    const int64_t target = std::max<int64_t>(t.ntiles, std::min<int64_t>(units, total / minw));
    if (t.ntiles >= target) return std::max(d.J, 1);
    int lo = 1, hi = std::max(d.J, 1);   // count_units(hi) = ntiles <= target
    while (lo < hi) {
        const int mid = lo + (hi - lo) / 2;
        if (count_units(t, mid) <= target) hi = mid;
        else lo = mid + 1;
    }
    return lo;
}

GatherTables make_gather_tables(const pmace_dims& d, const std::vector<int32_t>& offs_h, int tile_h, int B) {
    GatherTables t;
    t.tile_h = tile_h;
    overlap_lists(d, offs_h, t);
    cut_units(t, B);
    return t;
}

// Build the gather tables for tile height tile_h, upload them, and replace
// the job's current ones (freed after `s` has been synchronised).
pmace_status install_gather_tables(pmace_job* h, int tile_h, cudaStream_t s) {
    if (h->gblock <= 0) h->gblock = gather_block_length(h->dims, h->offs_host);
    const GatherTables t = make_gather_tables(h->dims, h->offs_host, tile_h, h->gblock);
    int* list = nullptr;
    int4* units = nullptr;
    int2* seg = nullptr;
    float2* scratch = nullptr;
    int* counters = nullptr;
    const size_t slot = (size_t)tile_h * kGatherTileW;
    const size_t b_list = t.list.size() * sizeof(int), b_units = t.units.size() * sizeof(int4),
                 b_seg = t.seg.size() * sizeof(int2),
                 b_scr = std::max<size_t>((size_t)t.nslots * slot, 1) * sizeof(float2),
                 b_cnt = (size_t)t.ntiles * sizeof(int);
    cudaError_t e = cudaMalloc(&list, b_list);
    if (e == cudaSuccess) e = cudaMalloc(&units, b_units);
    if (e == cudaSuccess) e = cudaMalloc(&seg, b_seg);
    if (e == cudaSuccess) e = cudaMalloc(&scratch, b_scr);
    if (e == cudaSuccess) e = cudaMalloc(&counters, b_cnt);
    if (e == cudaSuccess) e = cudaMemcpyAsync(list, t.list.data(), b_list, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(units, t.units.data(), b_units, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(seg, t.seg.data(), b_seg, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(counters, 0, b_cnt, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);   // the host tables die on return
    if (e != cudaSuccess) {
        for (void* p : {(void*)list, (void*)units, (void*)seg, (void*)scratch, (void*)counters})
            if (p) cudaFree(p);
        return cuda_fail(h, e, "gather tables");
    }
    for (void* p : {(void*)h->tile_list, (void*)h->units, (void*)h->tile_seg, (void*)h->gscratch,
                    (void*)h->gcounters})
        if (p) cudaFree(p);
    const int64_t bytes = (int64_t)(b_list + b_units + b_seg + b_scr + b_cnt);
    h->bytes += bytes - h->gather_bytes;
    h->gather_bytes = bytes;
    h->tile_list = list;
    h->list_len = (int)t.list.size();
    h->units = units;
    h->tile_seg = seg;
    h->gscratch = scratch;
    h->gcounters = counters;
    h->tile_h = t.tile_h;
    h->tiles_x = t.tiles_x;
    h->tiles_y = t.tiles_y;
    h->ntiles = t.ntiles;
    h->nunits = (int)t.units.size();
    h->nslots = t.nslots;
    return PMACE_OK;
}

pmace_status build_tables(pmace_job* h, const std::vector<float>& probe_h,
                          const std::vector<int32_t>& offs_h, cudaStream_t s,
                          std::vector<std::vector<char>>& keep, int** perm_out) {
    const int np = h->dims.np, J = h->dims.J;
    const size_t P = (size_t)np * np;
    // probe tables in double, rounded once
    std::vector<float2> d(P), dinv(P), tw(np);
    std::vector<float> wk(P);
    double amax = 0.0;
    for (size_t i = 0; i < P; ++i)
        amax = std::max(amax, std::hypot((double)probe_h[2 * i], (double)probe_h[2 * i + 1]));
    for (size_t i = 0; i < P; ++i) {
        const double re = probe_h[2 * i], im = probe_h[2 * i + 1];
        const double m = std::hypot(re, im);
        d[i] = make_float2((float)re, (float)im);
        wk[i] = (float)std::pow(m, (double)h->dims.kappa);
        if (m > 1e-30 * amax && m > 0.0) {
            const double m2 = re * re + im * im;
            dinv[i] = make_float2((float)(re / m2), (float)(-im / m2));
        } else {
            dinv[i] = make_float2(0.f, 0.f);
        }
    }
    for (int m = 0; m < np; ++m) {
        const double ang = -2.0 * M_PI * (double)m / (double)np;
        tw[m] = make_float2((float)std::cos(ang), (float)std::sin(ang));
    }
    // where the agent kernel reads each amplitude (spectrum orders of its
    // stages, and for the exchange variants the thread order)
    const std::vector<int> layout = amp_layout(np, h->variant, h->amp_f16 ? 2 : 4);

    PM_CUDA(h, dalloc(h, &h->probe, P));
    PM_CUDA(h, dalloc(h, &h->dinv, P));
    PM_CUDA(h, dalloc(h, &h->tw, (size_t)np));
    PM_CUDA(h, dalloc(h, &h->wk, P));
    PM_CUDA(h, dalloc(h, &h->offs, (size_t)J));
    auto up = [&](void* dst, const void* src, size_t bytes) -> cudaError_t {
        keep.emplace_back((const char*)src, (const char*)src + bytes);   // alive until the sync
        return cudaMemcpyAsync(dst, keep.back().data(), bytes, cudaMemcpyHostToDevice, s);
    };
    PM_CUDA(h, up(h->probe, d.data(), P * sizeof(float2)));
    PM_CUDA(h, up(h->dinv, dinv.data(), P * sizeof(float2)));
    PM_CUDA(h, up(h->tw, tw.data(), np * sizeof(float2)));
    PM_CUDA(h, up(h->wk, wk.data(), P * sizeof(float)));
    PM_CUDA(h, up(h->offs, offs_h.data(), (size_t)J * 2 * sizeof(int32_t)));
    // the layout table lives only until the amplitude pass
    PM_CUDA(h, cudaMalloc(perm_out, P * sizeof(int)));
    PM_CUDA(h, up(*perm_out, layout.data(), P * sizeof(int)));
    return PMACE_OK;
}


void free_job(pmace_job* h) {
    if (!h) return;
    void* ptrs[] = {h->q, h->u, h->xbar, h->probe, h->dinv, h->tw, h->img_tmp, h->y, h->yscale,
                    h->laminv, h->wk, h->offs, h->tile_list, h->units, h->tile_seg, h->gscratch,
                    h->gcounters, h->err, h->partials, h->red_out};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    for (auto* v : {&h->ev_agent, &h->ev_cons})
        for (auto& e : *v) {
            if (e.a) cudaEventDestroy(e.a);
            if (e.b) cudaEventDestroy(e.b);
        }
    if (h->graph) cudaGraphExecDestroy(h->graph);
    if (h->capture_stream) cudaStreamDestroy(h->capture_stream);
    delete h;
}

cudaError_t record_pair(std::vector<EventPair>& pool, size_t& n, bool start, cudaStream_t s) {
    if (start) {
        if (n == pool.size()) {
            EventPair p;
            cudaError_t e = cudaEventCreate(&p.a);
            if (e != cudaSuccess) return e;
            e = cudaEventCreate(&p.b);
            if (e != cudaSuccess) return e;
            pool.push_back(p);
        }
        return cudaEventRecord(pool[n].a, s);
    }
    cudaError_t e = cudaEventRecord(pool[n].b, s);
    ++n;
    return e;
}

}  // namespace

namespace pmace {
// Record the message pmace_last_error(NULL) returns, for entry points that
// have no handle.
void set_unbound_error(const char* msg) { g_create_error = msg ? msg : ""; }

GatherArgs gather_args(const pmace_job* h) {
    GatherArgs g{};
    g.wk = h->wk;
    g.offs = h->offs;
    g.tile_list = h->tile_list;
    g.units = h->units;
    g.tile_seg = h->tile_seg;
    g.scratch = h->gscratch;
    g.counters = h->gcounters;
    g.laminv = h->laminv;
    g.n1 = h->dims.n1;
    g.n2 = h->dims.n2;
    g.np = h->dims.np;
    g.tiles_x = h->tiles_x;
    g.J = h->dims.J;
    g.list_len = h->list_len;
    g.ntiles = h->ntiles;
    g.nslots = h->nslots;
    g.err = h->err;
    return g;
}

AgentArgs agent_args(const pmace_job* h, float alpha, float rho) {
    AgentArgs a{};
    a.q = h->q;
    a.u = h->u;
    a.xbar = h->xbar;
    a.y = h->y;
    a.yscale = h->yscale;
    a.probe = h->probe;
    a.dinv = h->dinv;
    a.tw = h->tw;
    a.offs = h->offs;
    a.partials = h->partials;
    a.n2 = h->dims.n2;
    a.n1 = h->dims.n1;
    a.J = h->dims.J;
    a.alpha = alpha;
    a.rho_cur = rho;
    a.rho_prev = h->rho_pending;
    a.first = h->iterations == 0 ? 1 : 0;
    a.wpc = h->wpc;
    a.err = h->err;
    a.residual = 1;
    a.keep_u = h->keep_u;
    return a;
}
}  // namespace pmace

namespace {


// One iteration of Algorithm 1: agent sweep (S0-S5) then consensus (S6);
// `residual`: the sweep also writes the residual partial sums.
pmace_status launch_iteration(pmace_job* h, float alpha, float rho, cudaStream_t s, bool events, bool residual,
                              float2* spectrum = nullptr) {
    AgentArgs a = agent_args(h, alpha, rho);
    a.residual = residual ? 1 : 0;
    a.spectrum = spectrum;
    GatherArgs g = gather_args(h);
    g.src = h->u;
    g.out = h->xbar;
    if (events) PM_CUDA(h, record_pair(h->ev_agent, h->n_agent, true, s));
    PM_CUDA(h, agent_entry(h->dims.np, &a, h->variant, h->amp_f16, s, nullptr));
    if (events) {
        PM_CUDA(h, record_pair(h->ev_agent, h->n_agent, false, s));
        PM_CUDA(h, record_pair(h->ev_cons, h->n_cons, true, s));
    }
    PM_CUDA(h, launch_gather_consensus(g, h->nunits, h->tile_h, s));
    if (events) PM_CUDA(h, record_pair(h->ev_cons, h->n_cons, false, s));
    h->rho_pending = rho;
    h->iterations++;
    return PMACE_OK;
}

// Capture kGraphIters steady-state iterations (rho_prev = rho, not the
// first iteration) for (alpha, rho) on the job's own stream, once.
pmace_status ensure_graph(pmace_job* h, float alpha, float rho) {
    if (h->graph && h->graph_alpha == alpha && h->graph_rho == rho) return PMACE_OK;
    if (h->graph) {
        cudaGraphExecDestroy(h->graph);
        h->graph = nullptr;
    }
    if (!h->capture_stream) PM_CUDA(h, cudaStreamCreateWithFlags(&h->capture_stream, cudaStreamNonBlocking));
    const int64_t it_saved = h->iterations;
    const float rho_saved = h->rho_pending;
    h->iterations = std::max<int64_t>(it_saved, 1);
    h->rho_pending = rho;
    cudaGraph_t graph = nullptr;
    PM_CUDA(h, cudaStreamBeginCapture(h->capture_stream, cudaStreamCaptureModeThreadLocal));
    pmace_status st = PMACE_OK;
    for (int i = 0; i < kGraphIters && st == PMACE_OK; ++i)
        st = launch_iteration(h, alpha, rho, h->capture_stream, false, false);
    cudaError_t e = cudaStreamEndCapture(h->capture_stream, &graph);
    h->iterations = it_saved;
    h->rho_pending = rho_saved;
    if (st != PMACE_OK) {
        if (graph) cudaGraphDestroy(graph);
        return st;
    }
    if (e != cudaSuccess) return cuda_fail(h, e, "graph capture");
    e = cudaGraphInstantiate(&h->graph, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
        h->graph = nullptr;
        return cuda_fail(h, e, "graph instantiate");
    }
    h->graph_alpha = alpha;
    h->graph_rho = rho;
    return PMACE_OK;
}

// Switch the agent variant and the gather tile height.  A variant with
// another amplitude layout (amp_layout) has them re-laid out on the device
// (through u, which is dead between iterations).
pmace_status switch_plan(pmace_job* h, int variant, int tile_h, cudaStream_t s) {
    const int np = h->dims.np, J = h->dims.J;
    if (variant < 0 || variant >= kAgentVariants)
        return fail(h, PMACE_ERR_INVALID_ARG, "variant %d not in [0, %d)", variant, kAgentVariants);
    if (tile_h != 8 && tile_h != 16 && tile_h != 32)
        return fail(h, PMACE_ERR_INVALID_ARG, "tile_h %d not in {8, 16, 32}", tile_h);
    if (variant != h->variant) {
        AgentPlanInfo info{};
        if (agent_entry(np, nullptr, variant, h->amp_f16, s, &info) != cudaSuccess || !info.launchable) {
            cudaGetLastError();
            return fail(h, PMACE_ERR_UNSUPPORTED_SIZE, "agent variant %d cannot run on this device", variant);
        }
        const int c_new = agent_variant_of(np, variant).cluster;
        const int elem = h->amp_f16 ? 2 : 4;
        const std::vector<int> l_old = amp_layout(np, h->variant, elem), l_new = amp_layout(np, variant, elem);
        if (l_old != l_new) {
            const size_t P = (size_t)np * np;
            std::vector<int> inv(P), map(P);
            for (size_t e = 0; e < P; ++e) inv[l_old[e]] = (int)e;
            for (size_t e = 0; e < P; ++e) map[e] = inv[l_new[e]];   // new position e <- old position map[e]
            int* map_d = nullptr;
            PM_CUDA(h, cudaMalloc(&map_d, P * sizeof(int)));
            const size_t ybytes = (size_t)J * P * elem;
            cudaError_t e = cudaMemcpyAsync(map_d, map.data(), P * sizeof(int), cudaMemcpyHostToDevice, s);
            if (e == cudaSuccess) e = cudaMemcpyAsync(h->u, h->y, ybytes, cudaMemcpyDeviceToDevice, s);
            if (e == cudaSuccess) e = launch_relayout_window(h->y, h->u, map_d, J, np, elem, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            cudaFree(map_d);
            if (e != cudaSuccess) return cuda_fail(h, e, "amplitude re-layout");
        }
        h->variant = variant;
        h->cluster = c_new;
        h->plan = info;
        h->wpc = windows_per_cluster(np, variant, J, info);
    }
    if (tile_h != h->tile_h) {
        const pmace_status st = install_gather_tables(h, tile_h, s);
        if (st != PMACE_OK) return st;
    }
    if (h->graph) {   // the captured launches refer to the old plan
        cudaGraphExecDestroy(h->graph);
        h->graph = nullptr;
    }
    return PMACE_OK;
}

}  // namespace

extern "C" {

int32_t pmace_abi_version(void) { return 2; }

const char* pmace_status_string(pmace_status s) {
    switch (s) {
        case PMACE_OK: return "ok";
        case PMACE_ERR_INVALID_ARG: return "invalid argument";
        case PMACE_ERR_OOM: return "out of memory";
        case PMACE_ERR_CUDA: return "CUDA error";
        case PMACE_ERR_UNSUPPORTED_SIZE: return "unsupported size";
        case PMACE_ERR_TIMEOUT: return "device wait timed out";
        case PMACE_ERR_STATE: return "invalid state";
    }
    return "unknown status";
}

const char* pmace_last_error(pmace_handle h) {
    return h ? h->error.c_str() : g_create_error.c_str();
}

pmace_status pmace_create(const pmace_dims* dims, const float* probe, const int32_t* offsets,
                          const void* amps, pmace_amp_format fmt, const float* scales,
                          const float* init, int inputs_on_device, void* stream,
                          pmace_handle* out) {
    g_create_error.clear();
    if (!out) return fail(nullptr, PMACE_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!dims || !probe || !offsets || !amps)
        return fail(nullptr, PMACE_ERR_INVALID_ARG, "dims, probe, offsets and amps are required");
    const pmace_dims D = *dims;
    if (D.n1 <= 0 || D.n2 <= 0 || D.np <= 0 || D.J <= 0)
        return fail(nullptr, PMACE_ERR_INVALID_ARG, "sizes must be positive (n1=%d n2=%d np=%d J=%d)",
                    D.n1, D.n2, D.np, D.J);
    if (!np_supported(D.np))
        return fail(nullptr, PMACE_ERR_UNSUPPORTED_SIZE, "np=%d not in {32, 64, 128, 256}", D.np);
    if (D.np > D.n1 || D.np > D.n2)
        return fail(nullptr, PMACE_ERR_INVALID_ARG, "np=%d exceeds the image %dx%d", D.np, D.n1, D.n2);
    if (!std::isfinite(D.kappa))
        return fail(nullptr, PMACE_ERR_INVALID_ARG, "kappa must be finite");
    if (fmt != PMACE_AMP_F32 && fmt != PMACE_AMP_F16_SCALED)
        return fail(nullptr, PMACE_ERR_INVALID_ARG, "unknown amplitude format %d", (int)fmt);
    if (fmt == PMACE_AMP_F16_SCALED && !scales)
        return fail(nullptr, PMACE_ERR_INVALID_ARG, "FP16 amplitudes need per-pattern scales");
    if ((size_t)D.J * D.np * D.np > (size_t)INT32_MAX * 8)
        return fail(nullptr, PMACE_ERR_INVALID_ARG, "stack too large");
    for (int j = 0; j < D.J; ++j) {
        const int r = offsets[2 * j], c = offsets[2 * j + 1];
        if (r < 0 || c < 0 || r > D.n1 - D.np || c > D.n2 - D.np)
            return fail(nullptr, PMACE_ERR_INVALID_ARG,
                        "offset %d = (%d, %d) outside [0, %d] x [0, %d]", j, r, c, D.n1 - D.np,
                        D.n2 - D.np);
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int np = D.np, J = D.J;
    const size_t P = (size_t)np * np, JP = (size_t)J * P, NI = (size_t)D.n1 * D.n2;

    pmace_job* h = new (std::nothrow) pmace_job();
    if (!h) return fail(nullptr, PMACE_ERR_OOM, "host allocation failed");
    h->dims = D;
    h->amp_f16 = fmt == PMACE_AMP_F16_SCALED;
    cudaGetDevice(&h->device);
    {
        int l2 = 0;
        if (cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, h->device) != cudaSuccess) cudaGetLastError();
        h->keep_u = l2 > 0 && JP * sizeof(float2) <= 2 * (size_t)l2;
    }

    auto bail = [&](pmace_status st) {
        g_create_error = h->error;
        free_job(h);
        return st;
    };

    // plan: the requested variant if the device can run it, else the first that it can
    {
        const int v0 = default_variant(np, J);
        int chosen = -1;
        for (int i = 0; i < kAgentVariants && chosen < 0; ++i) {
            const int v = (v0 + i) % kAgentVariants;
            AgentPlanInfo info{};
            if (agent_entry(np, nullptr, v, h->amp_f16, s, &info) == cudaSuccess && info.launchable) {
                h->plan = info;
                chosen = v;
            }
            cudaGetLastError();
        }
        if (chosen < 0)
            return bail(fail(h, PMACE_ERR_UNSUPPORTED_SIZE, "no launchable agent plan for np=%d", np));
        h->variant = chosen;
        h->cluster = agent_variant_of(np, chosen).cluster;
        h->wpc = windows_per_cluster(np, chosen, J, h->plan);
    }
    // gather tile height: PMACE_GATHER_TILE_H in {8, 16, 32}, default 16
    if (const char* env = std::getenv("PMACE_GATHER_TILE_H")) {
        const int th = std::atoi(env);
        if (th == 8 || th == 16 || th == 32) h->tile_h = th;
    }

    // host copies of the small inputs
    std::vector<float> probe_h(2 * P);
    std::vector<int32_t> offs_h(offsets, offsets + 2 * (size_t)J);
    h->offs_host = offs_h;
    if (const char* env = std::getenv("PMACE_GRAPHS")) h->use_graphs = std::atoi(env) != 0;
    if (inputs_on_device) {
        cudaError_t e = cudaMemcpy(probe_h.data(), probe, 2 * P * sizeof(float), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return bail(cuda_fail(h, e, "probe copy"));
    } else {
        std::memcpy(probe_h.data(), probe, 2 * P * sizeof(float));
    }
    for (float v : probe_h)
        if (!std::isfinite(v)) return bail(fail(h, PMACE_ERR_INVALID_ARG, "probe has non-finite values"));

    std::vector<std::vector<char>> keep;
    keep.reserve(16);
    int* perm_d = nullptr;
    auto bail_perm = [&](pmace_status st2) {
        cudaStreamSynchronize(s);
        if (perm_d) cudaFree(perm_d);
        return bail(st2);
    };
    pmace_status st = build_tables(h, probe_h, offs_h, s, keep, &perm_d);
    if (st == PMACE_OK) st = install_gather_tables(h, h->tile_h, s);
    if (st != PMACE_OK) return bail_perm(st);

    cudaError_t e;
#define PM_CREATE(call)                                                    \
    do {                                                                   \
        e = (call);                                                        \
        if (e != cudaSuccess) return bail_perm(cuda_fail(h, e, #call));   \
    } while (0)
    PM_CREATE(dalloc(h, &h->q, JP));
    PM_CREATE(dalloc(h, &h->u, JP));
    PM_CREATE(dalloc(h, &h->xbar, NI));
    PM_CREATE(dalloc(h, &h->laminv, NI));
    PM_CREATE(dalloc(h, &h->partials, (size_t)J * kMaxCluster * 4 + kPrepBlocks));
    PM_CREATE(dalloc(h, &h->red_out, (size_t)4));
    PM_CREATE(dalloc(h, &h->err, (size_t)1));
    PM_CREATE(cudaMemsetAsync(h->err, 0, sizeof(int), s));
    const size_t ybytes = JP * (h->amp_f16 ? sizeof(__half) : sizeof(float));
    PM_CREATE(cudaMalloc(&h->y, std::max<size_t>(ybytes, 16)));
    h->bytes += (int64_t)ybytes;

    // amplitudes to kernel order (staged through u when they come from the host)
    const void* amps_dev = amps;
    if (!inputs_on_device) {
        PM_CREATE(cudaMemcpyAsync(h->u, amps, ybytes, cudaMemcpyHostToDevice, s));
        amps_dev = h->u;
    }
    if (h->amp_f16) {
        PM_CREATE(dalloc(h, &h->yscale, (size_t)J));
        PM_CREATE(cudaMemcpyAsync(h->yscale, scales, J * sizeof(float),
                                  inputs_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
    }
    double* sum_partials = h->partials + (size_t)J * kMaxCluster * 4;
    PM_CREATE(launch_prep_amps(amps_dev, h->amp_f16, h->yscale, h->y, perm_d, J, np,
                               sum_partials, h->err, kPrepBlocks, s));
    PM_CREATE(launch_reduce_partials(sum_partials, kPrepBlocks, 1, h->red_out, s));

    // weight image Lambda^-1
    GatherArgs g = gather_args(h);
    g.lam_out = h->laminv;
    PM_CREATE(launch_gather_weights(g, h->nunits, h->tile_h, s));

    // initial stacks
    double sumsq = 0.0;
    PM_CREATE(cudaMemcpyAsync(&sumsq, h->red_out, sizeof(double), cudaMemcpyDeviceToHost, s));
    PM_CREATE(cudaStreamSynchronize(s));
    int errflag = 0;
    PM_CREATE(cudaMemcpy(&errflag, h->err, sizeof(int), cudaMemcpyDeviceToHost));
    if (errflag & 1) return bail_perm(fail(h, PMACE_ERR_INVALID_ARG, "amplitudes must be finite and >= 0"));
    double dsq = 0.0;
    for (size_t i = 0; i < 2 * P; ++i) dsq += (double)probe_h[i] * probe_h[i];
    const float cval = (dsq > 0.0) ? (float)std::sqrt(sumsq / ((double)J * dsq)) : 0.f;
    const float2* init_dev = nullptr;
    if (init) {
        if (inputs_on_device) {
            init_dev = reinterpret_cast<const float2*>(init);
        } else {
            PM_CREATE(cudaMemcpyAsync(h->xbar, init, NI * sizeof(float2), cudaMemcpyHostToDevice, s));
            init_dev = h->xbar;
        }
        PM_CREATE(launch_check_finite(reinterpret_cast<const float*>(init_dev), (int64_t)NI * 2, h->err, s));
    }
    PM_CREATE(launch_init_stack(h->q, init_dev, make_float2(cval, 0.f), h->offs, J, np, D.n2, s));
    PM_CREATE(cudaMemsetAsync(h->xbar, 0, NI * sizeof(float2), s));
    PM_CREATE(cudaStreamSynchronize(s));
    PM_CREATE(cudaMemcpy(&errflag, h->err, sizeof(int), cudaMemcpyDeviceToHost));
    if (errflag & 2) return bail_perm(fail(h, PMACE_ERR_INVALID_ARG, "init has non-finite values"));
    // Host-side fault injection for the tests of the error paths:
    // PMACE_INJECT_WAIT_TIMEOUT=1 marks the new job as if a bounded exchange
    // wait of its agent sweep had given up (bit 2 of the error word); no
    // device-side wait is involved.
    if (const char* env = std::getenv("PMACE_INJECT_WAIT_TIMEOUT")) {
        if (std::atoi(env) != 0) {
            const int bit = 2;
            PM_CREATE(cudaMemcpy(h->err, &bit, sizeof(int), cudaMemcpyHostToDevice));
        }
    }
#ifdef PMACE_DEBUG
    // Bounds-checking build only: PMACE_INJECT_BAD_OFFSET=1 overwrites the
    // last window's corner on the device with one past the image, after the
    // stacks were initialised, for the tests of the device-side checks (a
    // release build has no checks and must never see it).
    if (const char* env = std::getenv("PMACE_INJECT_BAD_OFFSET")) {
        if (std::atoi(env) != 0) {
            const int2 bad = make_int2(D.n1, D.n2);
            PM_CREATE(cudaMemcpy(h->offs + (J - 1), &bad, sizeof(int2), cudaMemcpyHostToDevice));
        }
    }
#endif
#undef PM_CREATE
    cudaFree(perm_d);
    h->iterations = 0;
    h->rho_pending = 0.5f;
    *out = h;
    return PMACE_OK;
}

pmace_status pmace_iterate(pmace_handle h, int32_t n, const pmace_step* step, void* stream) {
    if (!h) return fail(nullptr, PMACE_ERR_INVALID_ARG, "NULL handle");
    if (!step || n < 0) return fail(h, PMACE_ERR_INVALID_ARG, "step must be non-NULL and n >= 0");
    const float alpha = step->alpha, rho = step->rho;
    if (!(alpha >= 0.f) || !std::isfinite(alpha))
        return fail(h, PMACE_ERR_INVALID_ARG, "alpha must be finite and >= 0 (got %g)", alpha);
    if (!(rho > 0.f && rho < 1.f)) return fail(h, PMACE_ERR_INVALID_ARG, "rho must be in (0, 1) (got %g)", rho);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int32_t done = 0;
    // Iterations that open with the pending rho of an earlier call (or the
    // job's first iteration) are launched directly; the steady state
    // (rho_prev == rho) replays a captured graph of kGraphIters iterations.
    // Only the call's last iteration, always launched directly, writes the
    // residual partial sums that pmace_residual reduces.
    while (done < n && (h->iterations == 0 || h->rho_pending != rho)) {
        pmace_status st = launch_iteration(h, alpha, rho, s, h->profiling, done + 1 == n);
        if (st != PMACE_OK) return st;
        ++done;
    }
    if (!h->profiling && h->use_graphs && n - 1 - done >= kGraphIters) {
        pmace_status st = ensure_graph(h, alpha, rho);
        if (st != PMACE_OK) return st;
        for (; done + kGraphIters <= n - 1; done += kGraphIters) {
            PM_CUDA(h, cudaGraphLaunch(h->graph, s));
            h->iterations += kGraphIters;
        }
    }
    for (; done < n; ++done) {
        pmace_status st = launch_iteration(h, alpha, rho, s, h->profiling, done + 1 == n);
        if (st != PMACE_OK) return st;
    }
    return PMACE_OK;
}

pmace_status pmace_set_plan(pmace_handle h, int32_t variant, int32_t tile_h, void* stream) {
    if (!h) return fail(nullptr, PMACE_ERR_INVALID_ARG, "NULL handle");
    return switch_plan(h, variant, tile_h, static_cast<cudaStream_t>(stream));
}

pmace_status pmace_autotune(pmace_handle h, const pmace_step* step, int32_t iters, void* stream,
                            pmace_plan* chosen) {
    if (!h) return fail(nullptr, PMACE_ERR_INVALID_ARG, "NULL handle");
    if (!step || iters < 1) return fail(h, PMACE_ERR_INVALID_ARG, "step must be non-NULL and iters >= 1");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const size_t JP = (size_t)h->dims.J * h->dims.np * h->dims.np, NI = (size_t)h->dims.n1 * h->dims.n2;
    // save the state; every trial starts from it and it is restored at the end
    float2 *q0 = nullptr, *x0 = nullptr;
    cudaError_t e = cudaMalloc(&q0, JP * sizeof(float2));
    if (e == cudaSuccess) e = cudaMalloc(&x0, NI * sizeof(float2));
    if (e != cudaSuccess) {
        if (q0) cudaFree(q0);
        return cuda_fail(h, e, "autotune state copy");
    }
    const int64_t it0 = h->iterations;
    const float rho0 = h->rho_pending;
    const bool prof0 = h->profiling, graphs0 = h->use_graphs;
    pmace_status st = PMACE_OK;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    auto restore = [&]() -> cudaError_t {
        cudaError_t r = cudaMemcpyAsync(h->q, q0, JP * sizeof(float2), cudaMemcpyDeviceToDevice, s);
        if (r == cudaSuccess) r = cudaMemcpyAsync(h->xbar, x0, NI * sizeof(float2), cudaMemcpyDeviceToDevice, s);
        h->iterations = it0;
        h->rho_pending = rho0;
        return r;
    };
    // time `iters` iterations (after two untimed ones) of the current plan, ms per iteration
    auto trial = [&](double* ms) -> pmace_status {
        pmace_status r = pmace_iterate(h, 2, step, s);
        if (r != PMACE_OK) return r;
        PM_CUDA(h, cudaEventRecord(e0, s));
        r = pmace_iterate(h, iters, step, s);
        if (r != PMACE_OK) return r;
        PM_CUDA(h, cudaEventRecord(e1, s));
        PM_CUDA(h, cudaEventSynchronize(e1));
        float t = 0.f;
        PM_CUDA(h, cudaEventElapsedTime(&t, e0, e1));
        *ms = t / iters;
        PM_CUDA(h, restore());
        return PMACE_OK;
    };
    int best_v = h->variant, best_th = h->tile_h;
    double best = 1e300;
    h->profiling = false;
    h->use_graphs = true;
    e = cudaMemcpyAsync(q0, h->q, JP * sizeof(float2), cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(x0, h->xbar, NI * sizeof(float2), cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e != cudaSuccess) st = cuda_fail(h, e, "autotune setup");
    // agent variants at the current tile height, then tile heights for the best variant
    for (int v = 0; v < kAgentVariants && st == PMACE_OK; ++v) {
        AgentPlanInfo info{};
        if (agent_entry(h->dims.np, nullptr, v, h->amp_f16, s, &info) != cudaSuccess || !info.launchable) {
            cudaGetLastError();
            continue;
        }
        st = switch_plan(h, v, h->tile_h, s);
        double ms = 0.0;
        if (st == PMACE_OK) st = trial(&ms);
        if (st == PMACE_OK && ms < best) {
            best = ms;
            best_v = v;
        }
    }
    if (st == PMACE_OK) st = switch_plan(h, best_v, h->tile_h, s);
    for (int th : {8, 16, 32}) {
        if (st != PMACE_OK) break;
        st = switch_plan(h, best_v, th, s);
        double ms = 0.0;
        if (st == PMACE_OK) st = trial(&ms);
        if (st == PMACE_OK && ms < best) {
            best = ms;
            best_th = th;
        }
    }
    if (st == PMACE_OK) st = switch_plan(h, best_v, best_th, s);
    if (restore() != cudaSuccess && st == PMACE_OK) st = fail(h, PMACE_ERR_CUDA, "autotune restore failed");
    cudaStreamSynchronize(s);
    h->profiling = prof0;
    h->use_graphs = graphs0;
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(q0);
    cudaFree(x0);
    if (st == PMACE_OK && chosen) st = pmace_get_plan(h, chosen);
    return st;
}

pmace_status pmace_get_image(pmace_handle h, float* out, int out_on_device, void* stream) {
    if (!h) return fail(nullptr, PMACE_ERR_INVALID_ARG, "NULL handle");
    if (!out) return fail(h, PMACE_ERR_INVALID_ARG, "out is NULL");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const size_t NI = (size_t)h->dims.n1 * h->dims.n2;
    float2* dst = reinterpret_cast<float2*>(out);
    if (!out_on_device) {
        if (!h->img_tmp) PM_CUDA(h, dalloc(h, &h->img_tmp, NI));
        dst = h->img_tmp;
    }
    GatherArgs g = gather_args(h);
    g.src = h->q;
    g.xbar_in = h->xbar;
    g.out = dst;
    g.two_rho = 2.0f * h->rho_pending;
    PM_CUDA(h, launch_gather_readout(g, h->nunits, h->tile_h, s));
    if (!out_on_device) {
        int errflag = 0;
        PM_CUDA(h, cudaMemcpyAsync(out, dst, NI * sizeof(float2), cudaMemcpyDeviceToHost, s));
        PM_CUDA(h, cudaMemcpyAsync(&errflag, h->err, sizeof(int), cudaMemcpyDeviceToHost, s));
        PM_CUDA(h, cudaStreamSynchronize(s));
        if (errflag & 2)
            return fail(h, PMACE_ERR_TIMEOUT, "a bounded wait of the agent sweep's exchange gave up: the image may be wrong");
        if (errflag & kErrBoundsBit)
            return fail(h, PMACE_ERR_STATE, "a device-side bounds check failed (bounds-checking build): the image may be wrong");
    }
    return PMACE_OK;
}

pmace_status pmace_debug_spectra(pmace_handle h, const pmace_step* step, float* out, void* stream) {
    if (!h) return fail(nullptr, PMACE_ERR_INVALID_ARG, "NULL handle");
    if (!out || !step) return fail(h, PMACE_ERR_INVALID_ARG, "out and step are required");
    if (!(step->alpha >= 0.f) || !std::isfinite(step->alpha) || !(step->rho > 0.f && step->rho < 1.f))
        return fail(h, PMACE_ERR_INVALID_ARG, "invalid step");
    const int np = h->dims.np, J = h->dims.J;
    if (!agent_variant_of(np, h->variant).exchange)
        return fail(h, PMACE_ERR_UNSUPPORTED_SIZE, "the spectrum check needs an exchange plan (variant %d is not)",
                    h->variant);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    float2* dst = reinterpret_cast<float2*>(out);
    pmace_status st = launch_iteration(h, step->alpha, step->rho, s, false, true, dst);
    if (st != PMACE_OK) return st;
    // kernel order (row g, column c hold frequencies rows[g], cols[c]) to natural order, through u (dead now)
    const size_t P = (size_t)np * np;
    std::vector<int> rows = amp_row_order(np, h->variant), cols, map(P);
    dif_order(radices_of(np), 0, np, cols);
    for (int g = 0; g < np; ++g)
        for (int c = 0; c < np; ++c) map[(size_t)rows[g] * np + cols[c]] = g * np + c;
    int* map_d = nullptr;
    PM_CUDA(h, cudaMalloc(&map_d, P * sizeof(int)));
    cudaError_t e = cudaMemcpyAsync(map_d, map.data(), P * sizeof(int), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h->u, dst, (size_t)J * P * sizeof(float2), cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = launch_relayout_window(dst, h->u, map_d, J, np, (int)sizeof(float2), s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(map_d);
    if (e != cudaSuccess) return cuda_fail(h, e, "spectrum reordering");
    return PMACE_OK;
}

pmace_status pmace_get_patches(pmace_handle h, float* out, int out_on_device, void* stream) {
    if (!h) return fail(nullptr, PMACE_ERR_INVALID_ARG, "NULL handle");
    if (!out) return fail(h, PMACE_ERR_INVALID_ARG, "out is NULL");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const size_t JP = (size_t)h->dims.J * h->dims.np * h->dims.np;
    // u is dead between iterations (G consumed it), so it serves as staging
    float2* dst = out_on_device ? reinterpret_cast<float2*>(out) : h->u;
    PM_CUDA(h, launch_patches_from_state(h->q, h->xbar, h->offs, dst, h->dims.J, h->dims.np, h->dims.n1,
                                         h->dims.n2, 2.0f * h->rho_pending, h->err, s));
    if (!out_on_device) {
        PM_CUDA(h, cudaMemcpyAsync(out, dst, JP * sizeof(float2), cudaMemcpyDeviceToHost, s));
        PM_CUDA(h, cudaStreamSynchronize(s));
    }
    return PMACE_OK;
}

pmace_status pmace_residual(pmace_handle h, double out[2], void* stream) {
    if (!h) return fail(nullptr, PMACE_ERR_INVALID_ARG, "NULL handle");
    if (!out) return fail(h, PMACE_ERR_INVALID_ARG, "out is NULL");
    if (h->iterations == 0) return fail(h, PMACE_ERR_STATE, "no iteration has run yet");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    double r[4] = {0, 0, 0, 0};
    int errflag = 0;
    PM_CUDA(h, launch_reduce_partials(h->partials, h->dims.J * h->cluster, 4, h->red_out, s));
    PM_CUDA(h, cudaMemcpyAsync(r, h->red_out, sizeof(r), cudaMemcpyDeviceToHost, s));
    PM_CUDA(h, cudaMemcpyAsync(&errflag, h->err, sizeof(int), cudaMemcpyDeviceToHost, s));
    PM_CUDA(h, cudaStreamSynchronize(s));
    if (errflag & 2) return fail(h, PMACE_ERR_TIMEOUT, "a bounded wait of the agent sweep's exchange gave up");
    if (errflag & kErrBoundsBit)
        return fail(h, PMACE_ERR_STATE, "a device-side bounds check failed (bounds-checking build)");
    out[0] = r[1] > 0 ? std::sqrt(r[0] / r[1]) : 0.0;
    out[1] = r[3] > 0 ? r[2] / r[3] : 0.0;
    return PMACE_OK;
}

pmace_status pmace_get_state(pmace_handle h, float* q, float* xbar, pmace_state_info* info,
                             int on_device, void* stream) {
    if (!h) return fail(nullptr, PMACE_ERR_INVALID_ARG, "NULL handle");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    const size_t JP = (size_t)h->dims.J * h->dims.np * h->dims.np, NI = (size_t)h->dims.n1 * h->dims.n2;
    if (q) PM_CUDA(h, cudaMemcpyAsync(q, h->q, JP * sizeof(float2), k, s));
    if (xbar) PM_CUDA(h, cudaMemcpyAsync(xbar, h->xbar, NI * sizeof(float2), k, s));
    if (info) {
        info->iterations = h->iterations;
        info->rho_pending = h->rho_pending;
        info->reserved = 0;
    }
    if (!on_device) PM_CUDA(h, cudaStreamSynchronize(s));
    return PMACE_OK;
}

pmace_status pmace_set_state(pmace_handle h, const float* q, const float* xbar,
                             const pmace_state_info* info, int on_device, void* stream) {
    if (!h) return fail(nullptr, PMACE_ERR_INVALID_ARG, "NULL handle");
    if (!q || !xbar || !info) return fail(h, PMACE_ERR_INVALID_ARG, "q, xbar and info are required");
    if (info->iterations < 0 || !(info->rho_pending > 0.f && info->rho_pending < 1.f))
        return fail(h, PMACE_ERR_INVALID_ARG, "invalid state info");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    const size_t JP = (size_t)h->dims.J * h->dims.np * h->dims.np, NI = (size_t)h->dims.n1 * h->dims.n2;
    PM_CUDA(h, cudaMemcpyAsync(h->q, q, JP * sizeof(float2), k, s));
    PM_CUDA(h, cudaMemcpyAsync(h->xbar, xbar, NI * sizeof(float2), k, s));
    if (!on_device) PM_CUDA(h, cudaStreamSynchronize(s));
    h->iterations = info->iterations;
    h->rho_pending = info->rho_pending;
    return PMACE_OK;
}

pmace_status pmace_set_profiling(pmace_handle h, int enable) {
    if (!h) return fail(nullptr, PMACE_ERR_INVALID_ARG, "NULL handle");
    h->profiling = enable != 0;
    return PMACE_OK;
}

pmace_status pmace_kernel_times(pmace_handle h, double* agent_ms, int64_t* agent_launches,
                                double* consensus_ms, int64_t* consensus_launches, int reset) {
    if (!h) return fail(nullptr, PMACE_ERR_INVALID_ARG, "NULL handle");
    double ta = 0.0, tc = 0.0;
    for (size_t i = 0; i < h->n_agent; ++i) {
        float ms = 0.f;
        PM_CUDA(h, cudaEventSynchronize(h->ev_agent[i].b));
        PM_CUDA(h, cudaEventElapsedTime(&ms, h->ev_agent[i].a, h->ev_agent[i].b));
        ta += ms;
    }
    for (size_t i = 0; i < h->n_cons; ++i) {
        float ms = 0.f;
        PM_CUDA(h, cudaEventSynchronize(h->ev_cons[i].b));
        PM_CUDA(h, cudaEventElapsedTime(&ms, h->ev_cons[i].a, h->ev_cons[i].b));
        tc += ms;
    }
    if (agent_ms) *agent_ms = ta;
    if (agent_launches) *agent_launches = (int64_t)h->n_agent;
    if (consensus_ms) *consensus_ms = tc;
    if (consensus_launches) *consensus_launches = (int64_t)h->n_cons;
    if (reset) h->n_agent = h->n_cons = 0;
    return PMACE_OK;
}

pmace_status pmace_get_plan(pmace_handle h, pmace_plan* plan) {
    if (!h) return fail(nullptr, PMACE_ERR_INVALID_ARG, "NULL handle");
    if (!plan) return fail(h, PMACE_ERR_INVALID_ARG, "plan is NULL");
    const AgentVariant v = agent_variant_of(h->dims.np, h->variant);
    plan->cluster = h->cluster;
    plan->threads = h->plan.threads;
    plan->smem_bytes = h->plan.smem_bytes;
    plan->tile_h = h->tile_h;
    plan->tile_w = kGatherTileW;
    plan->variant = h->variant;
    plan->cols_per_thread = v.cols_per_thread;
    plan->stage_y = v.stage_y;
    plan->max_clusters = h->plan.max_clusters;
    plan->exchange = v.exchange;
    plan->windows_per_cluster = h->wpc;
    return PMACE_OK;
}

int64_t pmace_device_bytes(pmace_handle h) { return h ? h->bytes : 0; }

void pmace_destroy(pmace_handle h) {
    if (!h) return;
    int cur = 0;
    const int dev = h->device;
    cudaGetDevice(&cur);
    if (cur != dev) cudaSetDevice(dev);
    cudaDeviceSynchronize();
    free_job(h);
    if (cur != dev) cudaSetDevice(cur);
}

}  // extern "C"
