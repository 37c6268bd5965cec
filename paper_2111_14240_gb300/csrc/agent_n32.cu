// Agent sweep instantiations for 32 x 32 probes.
#include "agent.cuh"

namespace pmace {

cudaError_t agent_entry_32(const AgentArgs* a, int cluster, int amp_f16, cudaStream_t s,
                           AgentPlanInfo* info) {
    switch (cluster) {
        case 1: return agent_entry_impl<32, 1>(a, amp_f16, s, info);
        case 2: return agent_entry_impl<32, 2>(a, amp_f16, s, info);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace pmace
