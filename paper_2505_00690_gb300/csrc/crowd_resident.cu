// Shared-memory-resident crowd step: one CTA owns one environment for a whole
// multi-step rollout.
//
// The paper advances the dynamic agents of many parallel environments on
// the GPU each simulation step (Sec. 3.2, "Interactive Dynamics
// Generation"), with environments of uneven size (Sec. 3.3).  Environments
// never interact, so a CTA loads an environment's agents into shared memory
// once, runs every step there (hash build, neighbour search, half-planes,
// LP, integration, with a __syncthreads between steps), and writes the state
// back once.  HBM traffic per rollout is the state, parameters and goals in
// and the state out; per step only the robot commands are read.  CTAs pull
// environments from an atomic queue (largest first) so uneven batches stay
// balanced.
//
// Per step, inside the CTA:
//   1. robot slots take their commanded velocity;
//   2. bounding box of the agents (warp shuffles) -> uniform grid with cell
//      size c >= R, at most kGridMax x kGridMax cells;
//   3. counting sort by cell: shared-memory atomics give each agent its rank
//      in its cell, a warp scan turns counts into cell starts, a scatter
//      writes the sorted copy of positions/velocities;
//   4. each thread takes agents in cell order, scans the 3 contiguous
//      sorted ranges of its 3x3 cell block, keeps the K nearest by the FP64
//      ranking key, builds segment and agent half-planes and solves the LP;
//   5. the new state goes to a second buffer; the buffers swap.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "crowd_internal.h"
#include "crowd_resident_impl.cuh"

namespace crowd {

size_t resident_smem_bytes(int max_agents, int K, int block) {
    return smem_layout(max_agents, resident_kmax(K), block / 32, nullptr, nullptr);
}

int resident_block_threads(int max_agents) {
    int b = ((max_agents + 31) / 32) * 32;
    return b < 64 ? 64 : (b > kMaxThreads ? kMaxThreads : b);
}

int resident_kmax(int K) { return K <= 8 ? 8 : (K <= 10 ? 10 : (K <= 16 ? 16 : 32)); }

cudaError_t launch_resident(const ResidentArgs& a, int grid, int block, cudaStream_t stream) {
    switch (a.lanes) {
        case 2: return launch_resident_lanes2(a, grid, block, stream);
        case 4: return launch_resident_lanes4(a, grid, block, stream);
        case 8: return launch_resident_lanes8(a, grid, block, stream);
        default: return launch_lanes<1>(a, grid, block, stream);
    }
}

int resident_ctas_per_sm(int max_agents, int block, int K, int lanes) {
    switch (lanes) {
        case 2: return resident_ctas_lanes2(max_agents, block, K);
        case 4: return resident_ctas_lanes4(max_agents, block, K);
        case 8: return resident_ctas_lanes8(max_agents, block, K);
        default: return ctas_lanes<1>(max_agents, block, K);
    }
}

}  // namespace crowd
