// Internal: state of one reconstruction job (shared by the C ABI runtime in
// pmace_api.cu and the serving loop in server.cu).  Not part of the public ABI.
#pragma once

#include "pmace.h"
#include "pmace_internal.h"

#include <cuda_runtime.h>

#include <string>
#include <vector>

namespace pmace {

struct EventPair {
    cudaEvent_t a = nullptr, b = nullptr;
};

}  // namespace pmace

struct pmace_job {
    int device = 0;
    pmace_dims dims{};
    int amp_f16 = 0;
    int cluster = 1;
    int variant = 0;
    int wpc = 1;              // windows per agent cluster
    int keep_u = 0;           // u small enough to favour it in L2 for the gather
    pmace::AgentPlanInfo plan{};
    int tiles_x = 0, tiles_y = 0, ntiles = 0;
    int tile_h = 16;          // gather tile height (rows), width kGatherTileW
    int nunits = 0;           // gather CTAs (tiles with long lists are split)
    int list_len = 0;         // entries of the gather's window lists
    int gblock = 0;           // gather block length B: units split lists at multiples of B
    int nslots = 0;           // scratch slots of split tiles

    float2 *q = nullptr, *u = nullptr, *xbar = nullptr, *probe = nullptr, *dinv = nullptr,
           *tw = nullptr, *img_tmp = nullptr;
    void* y = nullptr;
    float *yscale = nullptr, *laminv = nullptr, *wk = nullptr;
    int2* offs = nullptr;
    int *tile_list = nullptr, *gcounters = nullptr, *err = nullptr;
    int4* units = nullptr;
    int2* tile_seg = nullptr;
    float2* gscratch = nullptr;
    int64_t gather_bytes = 0; // device bytes of the gather tables, included in `bytes`
    double *partials = nullptr, *red_out = nullptr;
    int64_t bytes = 0;

    int64_t iterations = 0;
    float rho_pending = 0.5f;

    std::vector<int32_t> offs_host;   // window corners, for rebuilding the overlap lists

    // CUDA graph of kGraphIters steady-state iterations for one (alpha, rho)
    bool use_graphs = true;
    cudaStream_t capture_stream = nullptr;
    cudaGraphExec_t graph = nullptr;
    float graph_alpha = -1.f, graph_rho = -1.f;

    bool profiling = false;
    std::vector<pmace::EventPair> ev_agent, ev_cons;
    size_t n_agent = 0, n_cons = 0;

    std::string error;
};

namespace pmace {

// Kernel arguments of one iteration of job h (pmace_api.cu).
AgentArgs agent_args(const pmace_job* h, float alpha, float rho);
GatherArgs gather_args(const pmace_job* h);

}  // namespace pmace
