// Agent sweep instantiations for 256 x 256 probes.
#include "agent.cuh"

namespace pmace {

cudaError_t agent_entry_256(const AgentArgs* a, int cluster, int amp_f16, cudaStream_t s,
                           AgentPlanInfo* info) {
    switch (cluster) {
        case 4: return agent_entry_impl<256, 4>(a, amp_f16, s, info);
        case 8: return agent_entry_impl<256, 8>(a, amp_f16, s, info);
        case 16: return agent_entry_impl<256, 16>(a, amp_f16, s, info);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace pmace
