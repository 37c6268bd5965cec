// Agent sweep instantiations for 256 x 256 probes (the variants of
// agent_variant_of(256, .)).
#include "agent.cuh"
#include "agent_xpose.cuh"

namespace pmace {

static_assert(agent_variant_of(256, 0).cluster == 16 && agent_variant_of(256, 0).cols_per_thread == 2 &&
              agent_variant_of(256, 0).stage_y == 0 && agent_variant_of(256, 0).windows == 1,
              "variant table mismatch");
static_assert(agent_variant_of(256, 1).cluster == 16 && agent_variant_of(256, 1).cols_per_thread == 2 &&
              agent_variant_of(256, 1).stage_y == 0 && agent_variant_of(256, 1).windows == 2,
              "variant table mismatch");
static_assert(agent_variant_of(256, 2).cluster == 8 && agent_variant_of(256, 2).cols_per_thread == 1 &&
              agent_variant_of(256, 2).stage_y == 1 && agent_variant_of(256, 2).windows == 1,
              "variant table mismatch");
static_assert(agent_variant_of(256, 3).cluster == 8 && agent_variant_of(256, 3).cols_per_thread == 2 &&
              agent_variant_of(256, 3).stage_y == 0 && agent_variant_of(256, 3).windows == 1,
              "variant table mismatch");

static_assert(agent_variant_of(256, 4).cluster == XposeGeom<256>::C && agent_variant_of(256, 4).exchange == 1,
              "variant table mismatch");

cudaError_t agent_entry_256(const AgentArgs* a, int v, int amp_f16, cudaStream_t s, AgentPlanInfo* info) {
    switch (v) {
        case 0: return agent_variant<256, 16, 2, 0, 1>(a, amp_f16, s, info);
        case 1: return agent_variant<256, 16, 2, 0, 2>(a, amp_f16, s, info);
        case 2: return agent_variant<256, 8, 1, 1, 1>(a, amp_f16, s, info);
        case 3: return agent_variant<256, 8, 2, 0, 1>(a, amp_f16, s, info);
        case 4: return agent_xpose<256>(a, amp_f16, s, info);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t agent_entry_batched_256(const AgentArgs* descs, const int2* work, int nclusters, int v, int amp_f16,
                                  cudaStream_t s) {
    switch (v) {
        case 0: return agent_variant_batched<256, 16, 2, 0, 1>(descs, work, nclusters, amp_f16, s);
        case 1: return agent_variant_batched<256, 16, 2, 0, 2>(descs, work, nclusters, amp_f16, s);
        case 2: return agent_variant_batched<256, 8, 1, 1, 1>(descs, work, nclusters, amp_f16, s);
        case 3: return agent_variant_batched<256, 8, 2, 0, 1>(descs, work, nclusters, amp_f16, s);
        case 4: return agent_xpose_batched<256>(descs, work, nclusters, amp_f16, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace pmace
