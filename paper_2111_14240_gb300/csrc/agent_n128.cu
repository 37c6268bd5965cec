// Agent sweep instantiations for 128 x 128 probes.
#include "agent.cuh"

namespace pmace {

cudaError_t agent_entry_128(const AgentArgs* a, int cluster, int amp_f16, cudaStream_t s,
                           AgentPlanInfo* info) {
    switch (cluster) {
        case 1: return agent_entry_impl<128, 1>(a, amp_f16, s, info);
        case 2: return agent_entry_impl<128, 2>(a, amp_f16, s, info);
        case 4: return agent_entry_impl<128, 4>(a, amp_f16, s, info);
        case 8: return agent_entry_impl<128, 8>(a, amp_f16, s, info);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace pmace
