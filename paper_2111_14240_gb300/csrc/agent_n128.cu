// Agent sweep instantiations for 128 x 128 probes (the variants of
// agent_variant_of(128, .)), including the two-window packed-lane sweep.
#include "agent.cuh"
#include "agent_xpose.cuh"
#include "agent_pair.cuh"

namespace pmace {

static_assert(agent_variant_of(128, 0).cluster == 8 && agent_variant_of(128, 0).cols_per_thread == 2 &&
              agent_variant_of(128, 0).stage_y == 0 && agent_variant_of(128, 0).windows == 1,
              "variant table mismatch");
static_assert(agent_variant_of(128, 1).cluster == 8 && agent_variant_of(128, 1).cols_per_thread == 1 &&
              agent_variant_of(128, 1).stage_y == 1 && agent_variant_of(128, 1).windows == 1,
              "variant table mismatch");
static_assert(agent_variant_of(128, 2).cluster == 4 && agent_variant_of(128, 2).cols_per_thread == 1 &&
              agent_variant_of(128, 2).stage_y == 1 && agent_variant_of(128, 2).windows == 1,
              "variant table mismatch");
static_assert(agent_variant_of(128, 3).cluster == 8 && agent_variant_of(128, 3).cols_per_thread == 2 &&
              agent_variant_of(128, 3).stage_y == 0 && agent_variant_of(128, 3).windows == 2,
              "variant table mismatch");

static_assert(agent_variant_of(128, 4).cluster == XposeGeom<128>::C && agent_variant_of(128, 4).exchange == 1,
              "variant table mismatch");
static_assert(agent_variant_of(128, 5).cluster == PairGeom<128>::C && agent_variant_of(128, 5).exchange == 2 &&
              agent_variant_of(128, 5).windows == 2, "variant table mismatch");

cudaError_t agent_entry_128(const AgentArgs* a, int v, int amp_f16, cudaStream_t s, AgentPlanInfo* info) {
    switch (v) {
        case 0: return agent_variant<128, 8, 2, 0, 1>(a, amp_f16, s, info);
        case 1: return agent_variant<128, 8, 1, 1, 1>(a, amp_f16, s, info);
        case 2: return agent_variant<128, 4, 1, 1, 1>(a, amp_f16, s, info);
        case 3: return agent_variant<128, 8, 2, 0, 2>(a, amp_f16, s, info);
        case 4: return agent_xpose<128>(a, amp_f16, s, info);
        case 5: return agent_pair<128>(a, amp_f16, s, info);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t agent_entry_batched_128(const AgentArgs* descs, const int2* work, int nclusters, int v, int amp_f16,
                                  cudaStream_t s) {
    switch (v) {
        case 0: return agent_variant_batched<128, 8, 2, 0, 1>(descs, work, nclusters, amp_f16, s);
        case 1: return agent_variant_batched<128, 8, 1, 1, 1>(descs, work, nclusters, amp_f16, s);
        case 2: return agent_variant_batched<128, 4, 1, 1, 1>(descs, work, nclusters, amp_f16, s);
        case 3: return agent_variant_batched<128, 8, 2, 0, 2>(descs, work, nclusters, amp_f16, s);
        case 4: return agent_xpose_batched<128>(descs, work, nclusters, amp_f16, s);
        case 5: return agent_pair_batched<128>(descs, work, nclusters, amp_f16, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace pmace
