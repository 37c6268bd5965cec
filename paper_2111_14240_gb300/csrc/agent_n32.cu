// Agent sweep instantiations for 32 x 32 probes (the variants of
// agent_variant_of(32, .)).
#include "agent.cuh"
#include "agent_xpose.cuh"

namespace pmace {

static_assert(agent_variant_of(32, 0).cluster == 2 && agent_variant_of(32, 0).cols_per_thread == 1 &&
              agent_variant_of(32, 0).stage_y == 1 && agent_variant_of(32, 0).windows == 1,
              "variant table mismatch");
static_assert(agent_variant_of(32, 1).cluster == 1 && agent_variant_of(32, 1).cols_per_thread == 1 &&
              agent_variant_of(32, 1).stage_y == 1 && agent_variant_of(32, 1).windows == 1,
              "variant table mismatch");
static_assert(agent_variant_of(32, 2).cluster == 2 && agent_variant_of(32, 2).cols_per_thread == 1 &&
              agent_variant_of(32, 2).stage_y == 0 && agent_variant_of(32, 2).windows == 2,
              "variant table mismatch");
static_assert(agent_variant_of(32, 3).cluster == 1 && agent_variant_of(32, 3).cols_per_thread == 1 &&
              agent_variant_of(32, 3).stage_y == 0 && agent_variant_of(32, 3).windows == 1,
              "variant table mismatch");

static_assert(agent_variant_of(32, 4).cluster == XposeGeom<32>::C && agent_variant_of(32, 4).exchange == 1,
              "variant table mismatch");

cudaError_t agent_entry_32(const AgentArgs* a, int v, int amp_f16, cudaStream_t s, AgentPlanInfo* info) {
    switch (v) {
        case 0: return agent_variant<32, 2, 1, 1, 1>(a, amp_f16, s, info);
        case 1: return agent_variant<32, 1, 1, 1, 1>(a, amp_f16, s, info);
        case 2: return agent_variant<32, 2, 1, 0, 2>(a, amp_f16, s, info);
        case 3: return agent_variant<32, 1, 1, 0, 1>(a, amp_f16, s, info);
        case 4: return agent_xpose<32>(a, amp_f16, s, info);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t agent_entry_batched_32(const AgentArgs* descs, const int2* work, int nclusters, int v, int amp_f16,
                                  cudaStream_t s) {
    switch (v) {
        case 0: return agent_variant_batched<32, 2, 1, 1, 1>(descs, work, nclusters, amp_f16, s);
        case 1: return agent_variant_batched<32, 1, 1, 1, 1>(descs, work, nclusters, amp_f16, s);
        case 2: return agent_variant_batched<32, 2, 1, 0, 2>(descs, work, nclusters, amp_f16, s);
        case 3: return agent_variant_batched<32, 1, 1, 0, 1>(descs, work, nclusters, amp_f16, s);
        case 4: return agent_xpose_batched<32>(descs, work, nclusters, amp_f16, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace pmace
