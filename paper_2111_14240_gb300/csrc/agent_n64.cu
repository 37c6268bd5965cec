// Agent sweep instantiations for 64 x 64 probes (the variants of
// agent_variant_of(64, .)).
#include "agent.cuh"
#include "agent_xpose.cuh"

namespace pmace {

static_assert(agent_variant_of(64, 0).cluster == 4 && agent_variant_of(64, 0).cols_per_thread == 1 &&
              agent_variant_of(64, 0).stage_y == 1 && agent_variant_of(64, 0).windows == 1,
              "variant table mismatch");
static_assert(agent_variant_of(64, 1).cluster == 4 && agent_variant_of(64, 1).cols_per_thread == 2 &&
              agent_variant_of(64, 1).stage_y == 0 && agent_variant_of(64, 1).windows == 1,
              "variant table mismatch");
static_assert(agent_variant_of(64, 2).cluster == 2 && agent_variant_of(64, 2).cols_per_thread == 1 &&
              agent_variant_of(64, 2).stage_y == 1 && agent_variant_of(64, 2).windows == 1,
              "variant table mismatch");
static_assert(agent_variant_of(64, 3).cluster == 4 && agent_variant_of(64, 3).cols_per_thread == 1 &&
              agent_variant_of(64, 3).stage_y == 0 && agent_variant_of(64, 3).windows == 2,
              "variant table mismatch");

static_assert(agent_variant_of(64, 4).cluster == XposeGeom<64>::C && agent_variant_of(64, 4).exchange == 1,
              "variant table mismatch");

cudaError_t agent_entry_64(const AgentArgs* a, int v, int amp_f16, cudaStream_t s, AgentPlanInfo* info) {
    switch (v) {
        case 0: return agent_variant<64, 4, 1, 1, 1>(a, amp_f16, s, info);
        case 1: return agent_variant<64, 4, 2, 0, 1>(a, amp_f16, s, info);
        case 2: return agent_variant<64, 2, 1, 1, 1>(a, amp_f16, s, info);
        case 3: return agent_variant<64, 4, 1, 0, 2>(a, amp_f16, s, info);
        case 4: return agent_xpose<64>(a, amp_f16, s, info);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t agent_entry_batched_64(const AgentArgs* descs, const int2* work, int nclusters, int v, int amp_f16,
                                  cudaStream_t s) {
    switch (v) {
        case 0: return agent_variant_batched<64, 4, 1, 1, 1>(descs, work, nclusters, amp_f16, s);
        case 1: return agent_variant_batched<64, 4, 2, 0, 1>(descs, work, nclusters, amp_f16, s);
        case 2: return agent_variant_batched<64, 2, 1, 1, 1>(descs, work, nclusters, amp_f16, s);
        case 3: return agent_variant_batched<64, 4, 1, 0, 2>(descs, work, nclusters, amp_f16, s);
        case 4: return agent_xpose_batched<64>(descs, work, nclusters, amp_f16, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace pmace
