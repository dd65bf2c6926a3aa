// Internal host/device interfaces shared by the crowd library's translation
// units (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace crowd {

// Device error word bits.
enum : int {
    kErrObstacleOverflow = 1,  // an agent had more segments in reach than the line buffer holds
    kErrTooManyCells = 2,      // internal: grid larger than the shared-memory cell table
};

constexpr int kMaxObstacleLines = 32;
// Penetration depth (m) from which two agents, or an agent and a segment,
// count as colliding in the statistics: 1 mm, well above the FP32 resolution
// of positions (about 4 um at 40 m), so that agents ORCA leaves exactly
// touching are not counted on rounding noise.
constexpr float kCollideDepth = 1e-3f;
// Largest environment the shared-memory-resident kernel takes.
constexpr int kResidentMaxAgents = 2048;
// Cell table of the resident kernel: at most kGridMax x kGridMax cells.
constexpr int kGridMax = 32;
constexpr int kMaxCells = kGridMax * kGridMax;

struct EnvStats {
    unsigned long long agent_collisions;
    unsigned long long segment_collisions;
    double speed_sum;
    unsigned long long steps;
};

// Work counters (mirrors crowd_work of the public header).
struct WorkCount {
    unsigned long long agent_steps, candidates, agent_lines, obstacle_lines, segment_tests, lp_checks, lp_solves,
        lp_solve_lines, fallbacks;
};

// Arguments of one launch of the resident kernel: every listed environment
// is advanced n_steps steps, reading and writing `state` in place.
struct ResidentArgs {
    int n_work;             // environments in `order`
    const int* order;       // [n_work] environment ids, processed in this order
    int* queue;             // work counter (zeroed before launch)
    const int* env_start;   // [E+1]
    const int* seg_start;   // [E+1]
    const int* robot_index; // [E] env-local or -1
    const float4* segs;     // [S] (ax, ay, bx, by)
    const float4* par;      // [N] (radius, v_max, preferred speed, 0)
    const float2* goal;     // [N]
    float4* state;          // [N] (px, py, vx, vy)
    const float2* robot_vel;  // [n_steps][robot_stride] or null (keep current)
    int robot_stride;       // entries per step in robot_vel (normally E)
    int n_steps;
    float dt, tau, tau_o, R, robot_alpha;
    int K;
    int* nbr_out;           // [N][K] or null: neighbour lists of the last step
    EnvStats* stats;        // [E] or null: accumulate statistics
    int* reach;             // [N] or null: 1-based step of first goal reach
    long long step_base;    // global index of the first step of this launch
    WorkCount* work;        // or null: count work items
    int* err;               // device error word
    int max_agents;         // largest environment in `order` (sizes shared memory)
};

size_t resident_smem_bytes(int max_agents);
int resident_block_threads(int max_agents);
int resident_kmax(int K);
// Launch on `stream`; `grid` CTAs pull environments from the queue.
cudaError_t launch_resident(const ResidentArgs& a, int grid, int block, cudaStream_t stream);
// CTAs of the resident kernel that fit on one SM for this configuration.
int resident_ctas_per_sm(int max_agents, int block, int K);

}  // namespace crowd
