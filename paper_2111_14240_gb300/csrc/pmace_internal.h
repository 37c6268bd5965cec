// Internal interfaces between the host runtime (pmace_api.cu) and the CUDA
// kernels.  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace pmace {

// Radix plan of a length-L transform: at most two in-place stages,
// radices (first, second); second == 1 means a single stage.
struct RadixPlan {
    int first, second;
};
__host__ __device__ constexpr RadixPlan radix_plan(int L) {
    return L == 256 ? RadixPlan{16, 16}
         : L == 128 ? RadixPlan{16, 8}
         : L == 64  ? RadixPlan{8, 8}
         : L == 32  ? RadixPlan{8, 4}
         : L == 16  ? RadixPlan{16, 1}
         : L == 8   ? RadixPlan{8, 1}
                    : RadixPlan{0, 0};
}

// Bit of the job's error word that the bounds checks of the PMACE_DEBUG
// build set (a window offset outside the image, a window index outside
// [0, J), a gather unit outside its tables); the checked access is then
// clamped or skipped, so the build never reads or writes outside a job's
// arrays, and the host reports PMACE_ERR_STATE.
constexpr int kErrBoundsBit = 8;

// Arguments of one agent sweep (steps S0-S5 of one iteration, all patches).
struct AgentArgs {
    float2* q;              // [J][Np][Np] pending stack q = v - 2 rho w (read, then overwritten; the
                            // in-place variant keeps v there between its copy-in and copy-out)
    float2* u;              // [J][Np][Np] written: u = 2w - v
    const float2* xbar;     // [n1][n2] consensus image of the previous iteration
    const void* y;          // [J][Np][Np] amplitudes in kernel (digit-reversed) order
    const float* yscale;    // [J] per-pattern scale (FP16 codes only)
    const float2* probe;    // [Np][Np] d
    const float2* dinv;     // [Np][Np] 1/d, (0,0) where d is treated as absent
    const float2* tw;       // [Np] W_Np^m = exp(-2 pi i m / Np)
    const int2* offs;       // [J] (row, col) window corners
    double* partials;       // [J * cluster][4] residual partial sums
    int n2;                 // image row stride (columns)
    int n1;                 // image rows (bounds checks of the PMACE_DEBUG build)
    int J;
    float alpha, rho_prev, rho_cur;
    int first;              // 1 on the first iteration of the job
    int residual;           // 1: write the residual partial sums (else they are left untouched)
    int keep_u;             // 1: store u with the L2 evict-last hint (u fits about twice the L2)
    int wpc;                // windows per cluster (transposing-exchange variant)
    int* err;               // bit 2: a bounded device-side wait gave up; bit 3: a bounds check of the
                            // PMACE_DEBUG build failed
    float2* spectrum;       // when set (exchange variants): the unnormalised forward 2-D DFT of d v of every
                            // window, [J][Np][Np] in kernel order, written as the column step computes it
};

// Arguments of the pixel-owner gathers (weight image, consensus, readout).
struct GatherArgs {
    const float2* src;      // [J][Np][Np] stack to average (u or q)
    const float* wk;        // [Np][Np] |d|^kappa
    const int2* offs;       // [J]
    const int* tile_list;   // patch indices per tile, ascending, tiles one after another
    const int4* units;      // [nunits] CTA k: (tile, lb, le, slot), windows tile_list[lb..le)
    const int2* tile_seg;   // [ntiles] (first scratch slot, CTAs) of every tile
    float2* scratch;        // [nslots][tile_h * kGatherTileW] partial sums of split tiles
    int* counters;          // [ntiles] CTAs of a split tile finished; 0 between launches
    const float* laminv;    // [n1][n2] Lambda^-1 (0 where Lambda = 0)
    const float2* xbar_in;  // readout: consensus image
    float2* out;            // [n1][n2]
    float* lam_out;         // weight-image mode: Lambda^-1 written here
    int n1, n2, np, tiles_x;
    float two_rho;          // readout: 2 rho
    // bounds of the tables, checked by the PMACE_DEBUG build (bit 3 of *err)
    int J, list_len, ntiles, nslots;
    int* err;
};

// Gather tiles are kGatherTileW = 32 pixels wide (one warp per tile row
// segment) and tile_h rows high, tile_h in {8, 16, 32}; every thread owns
// kGatherRowsPerThread rows of its column, so a tile has tile_h * 8 threads.
constexpr int kGatherTileW = 32;
constexpr int kGatherRowsPerThread = 4;
// A tile's ascending window list is gathered by one CTA ("unit") per run
// of windows with the same index block i / B (B is fixed per job), so
// interior tiles with long lists are spread over several CTAs.  Unit
// `slot` >= 0 writes its partial sums to scratch slot `slot`; the unit that
// finishes last (a counter per tile) adds the tile's partials in ascending
// block order, so the sum order is fixed by the tables, not by timing.
// slot = -1: the tile has one unit, which writes the result.
// Windows of a unit are staged in shared memory kGatherStage at a time.
constexpr int kGatherStage = 64;
__host__ __device__ constexpr int gather_threads(int tile_h) {
    return tile_h / kGatherRowsPerThread * kGatherTileW;
}

// Agent kernel variants compiled for each probe size: CTAs per window,
// columns per thread in the column step, amplitude staging in shared memory,
// windows per cluster, and how the 2-D DFT is split over the cluster
// (exchange 0: an in-place cross-CTA butterfly stage through distributed
// shared memory, agent.cuh; 1: a transposing exchange of 16 x 16 blocks by
// bulk copies, Np / 16 CTAs, a run of windows per cluster, agent_xpose.cuh;
// 2: the same exchange with two windows at a time in packed FP32 lanes,
// agent_pair.cuh, compiled for 128 x 128 probes only).
// default_agent_variant is where a job starts; pmace_autotune and
// PMACE_AGENT_PLAN pick others.  A variant a probe size does not compile
// reports cudaErrorInvalidValue from its agent entry and is never chosen.
struct AgentVariant {
    int cluster, cols_per_thread, stage_y, windows, exchange;
};
constexpr int kAgentVariants = 6;
__host__ __device__ constexpr AgentVariant agent_variant_of(int np, int v) {
    constexpr AgentVariant t32[kAgentVariants] = {
        {2, 1, 1, 1, 0}, {1, 1, 1, 1, 0}, {2, 1, 0, 2, 0}, {1, 1, 0, 1, 0}, {2, 1, 0, 1, 1}, {2, 1, 0, 2, 2}};
    constexpr AgentVariant t64[kAgentVariants] = {
        {4, 1, 1, 1, 0}, {4, 2, 0, 1, 0}, {2, 1, 1, 1, 0}, {4, 1, 0, 2, 0}, {4, 1, 0, 1, 1}, {4, 1, 0, 2, 2}};
    constexpr AgentVariant t128[kAgentVariants] = {
        {8, 2, 0, 1, 0}, {8, 1, 1, 1, 0}, {4, 1, 1, 1, 0}, {8, 2, 0, 2, 0}, {8, 1, 0, 1, 1}, {8, 1, 0, 2, 2}};
    constexpr AgentVariant t256[kAgentVariants] = {
        {16, 2, 0, 1, 0}, {16, 2, 0, 2, 0}, {8, 1, 1, 1, 0}, {8, 2, 0, 1, 0}, {16, 1, 0, 1, 1}, {16, 1, 0, 2, 2}};
    return np == 32 ? t32[v] : np == 64 ? t64[v] : np == 128 ? t128[v] : t256[v];
}
// The fastest variant measured on GB300 for each probe size and J windows:
// the transposing exchange (variant 4) for 64 x 64 and larger probes (on a
// 1024^2 / 3600-window scan 0.174 ms against 0.179 ms for the best in-place
// variant); for 32 x 32 probes one CTA per window (variant 1) once J fills
// the GPU (0.042 ms against 0.066 ms on a 512^2 / 3600-window scan), else
// two CTAs per window (variant 0: 0.0121 ms against 0.0140 ms for 169
// windows).
__host__ __device__ constexpr int default_agent_variant(int np, int J) {
    return np >= 64 ? 4 : J >= 1024 ? 1 : 0;
}

// Geometry of one agent plan (probe size, CTAs per patch).
struct AgentPlanInfo {
    int threads;      // threads per CTA
    int smem_bytes;   // dynamic shared memory per CTA
    int launchable;   // the device can co-schedule at least one cluster
    int max_clusters; // clusters the device can hold at once
};

// Agent entry points, one per probe size (each in its own translation unit).
// With a == nullptr they only fill `info` for variant `v` of
// agent_variant_of (cudaErrorInvalidValue for an unknown variant);
// otherwise they launch the sweep.
cudaError_t agent_entry_32(const AgentArgs* a, int v, int amp_f16, cudaStream_t s, AgentPlanInfo* info);
cudaError_t agent_entry_64(const AgentArgs* a, int v, int amp_f16, cudaStream_t s, AgentPlanInfo* info);
cudaError_t agent_entry_128(const AgentArgs* a, int v, int amp_f16, cudaStream_t s, AgentPlanInfo* info);
cudaError_t agent_entry_256(const AgentArgs* a, int v, int amp_f16, cudaStream_t s, AgentPlanInfo* info);
// Several jobs of one probe size and amplitude format in one launch:
// `descs` (device) holds each job's arguments, `work` (device) the
// (job, first window) pair of each of the nclusters clusters.
cudaError_t agent_entry_batched_32(const AgentArgs* descs, const int2* work, int nclusters, int v, int amp_f16, cudaStream_t s);
cudaError_t agent_entry_batched_64(const AgentArgs* descs, const int2* work, int nclusters, int v, int amp_f16, cudaStream_t s);
cudaError_t agent_entry_batched_128(const AgentArgs* descs, const int2* work, int nclusters, int v, int amp_f16, cudaStream_t s);
cudaError_t agent_entry_batched_256(const AgentArgs* descs, const int2* work, int nclusters, int v, int amp_f16, cudaStream_t s);

// Support kernels (support.cu).
// nunits CTAs, one per entry of g.units.
cudaError_t launch_gather_weights(const GatherArgs& g, int nunits, int tile_h, cudaStream_t s);
cudaError_t launch_gather_consensus(const GatherArgs& g, int nunits, int tile_h, cudaStream_t s);
cudaError_t launch_gather_readout(const GatherArgs& g, int nunits, int tile_h, cudaStream_t s);
// Consensus of several jobs in one launch: `work` (device) holds the
// (job, unit) pair of each of the nunits CTAs, `descs` (device) each job's
// arguments; every job uses the same tile height.
cudaError_t launch_gather_consensus_batched(const GatherArgs* descs, const int2* work, int nunits, int tile_h,
                                            cudaStream_t s);
cudaError_t launch_prep_amps(const void* amps_in, int amp_f16, const float* scales, void* y_out,
                             const int* layout, int J, int np, double* sumsq_partials, int* err_flag,
                             int nblocks, cudaStream_t s);
cudaError_t launch_reduce_partials(const double* partials, int nrows, int ncols, double* out,
                                   cudaStream_t s);
cudaError_t launch_init_stack(float2* q, const float2* init, float2 cval, const int2* offs,
                              int J, int np, int n2, cudaStream_t s);
cudaError_t launch_patches_from_state(const float2* q, const float2* xbar, const int2* offs,
                                      float2* v, int J, int np, int n1, int n2, float two_rho,
                                      int* err, cudaStream_t s);
cudaError_t launch_check_finite(const float* data, int64_t n, int* err_flag, cudaStream_t s);
// dst[j][e] = src[j][map[e]] for every window j and stored position e
// (elem bytes per value: 2, 4 or 8).
cudaError_t launch_relayout_window(void* dst, const void* src, const int* map, int J, int np, int elem,
                                   cudaStream_t s);

// Message returned by pmace_last_error(NULL) (pmace_api.cu).
void set_unbound_error(const char* msg);

}  // namespace pmace
