// Instantiation of the resident crowd kernel with 8 lanes per agent (its own
// translation unit so that the instantiations compile in parallel).
#include "crowd_resident_impl.cuh"

namespace crowd {

cudaError_t launch_resident_lanes8(const ResidentArgs& a, int grid, int block, cudaStream_t stream) {
    return launch_lanes<8>(a, grid, block, stream);
}

int resident_ctas_lanes8(int max_agents, int block, int K) { return ctas_lanes<8>(max_agents, block, K); }

}  // namespace crowd
