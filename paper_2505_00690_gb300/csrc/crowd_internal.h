// Internal host/device interfaces shared by the crowd library's translation
// units (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace crowd {

// Goal queue or goal pool of a handle (see crowd_set_goal_queue and
// crowd_set_goal_pool; at most one of the two is set).
struct GoalQueue {
    const float2* queue;  // [N][q]
    int* idx;             // [N] goals reached (queue) or drawn (pool) since set
    int q;                // goals per agent (0: no queue)
    int cyclic;           // 1: after the last goal the queue starts again
    const int* pool_start;  // [E + 1] each environment's points in `pool` (null: no pool)
    const float2* pool;     // [P] goal points
    uint2 seed;             // Philox key of the draws
    __host__ __device__ bool active() const { return q > 0 || pool_start != nullptr; }
};

// Lane-following vehicles of a handle (see crowd_set_vehicles).
struct VehicleArgs {
    int n;                  // vehicles (0: none)
    const int* start;       // [E + 1]: the vehicles of env e are [start[e], start[e + 1])
    const int* agent;       // [V] global agent slot
    const int* lane;        // [V]
    float* s;               // [V] arc position on the lane (updated in place)
    float* v;               // [V] speed (updated in place)
    const float4* par_a;    // [V] (v0, T, a, b)
    const float2* par_b;    // [V] (s0, length)
    const float2* pts;      // [P] lane points
    const int* lane_start;  // [n_lanes + 1]
    const float* cum;       // [P + n_lanes] cumulative lengths; lane l's start at lane_start[l] + l
    float half_width, lookahead;
};

// Episodes of a handle (see crowd_set_episodes): environment e starts over
// at the start of step t of the episode clock when steps[e] > 0, t > 0 and
// t % steps[e] == 0, restoring its rows from the snapshot taken when the
// episodes were set.
struct EpisodeArgs {
    const int* steps;     // [E] episode length in steps (0: never); null: no episodes
    const float4* state;  // [N] agent rows at the start of an episode
    const float2* goal;   // [N] goals at the start of an episode
    const int* gidx;      // [N] goal-queue counters at the start (null: no queue)
    const float* veh_s;   // [V] car arc positions at the start (null: no cars)
    const float* veh_v;   // [V] car speeds at the start
    long long origin;     // global step index of the episode clock's t = 0
};

__host__ __device__ inline bool episode_restart(int steps, long long global_step, long long origin) {
    const long long t = global_step - origin;
    return steps > 0 && t > 0 && t % steps == 0;
}

// Device error word bits.
enum : int {
    kErrObstacleOverflow = 1,  // an agent had more segments in reach than the line buffer holds
    kErrTooManyCells = 2,      // internal: grid larger than the shared-memory cell table
};

constexpr int kMaxObstacleLines = 64;
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
        lp_solve_lines, fallbacks, pairs_in_range;
};

// Static grid over an environment's segments with, per cell, the ascending
// list of segments that can come within reach (r + tau_obst v_max, maximised
// over the environment's agents) of a point of the cell; agents outside the
// grid use the nearest border cell.  Lists of cell k of the environment are
// seg_cell_ids[seg_cell_start[off + k] .. seg_cell_start[off + k + 1]).
struct SegGrid {
    float x0, y0, inv_c;
    int W, H;
    int off;
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
    const SegGrid* seg_grid;      // [E]
    const int* seg_cell_start;    // per-cell segment lists (see SegGrid)
    const int* seg_cell_ids;
    const float4* par;      // [N] (radius, v_max, preferred speed, 0)
    float2* goal;           // [N] current goals (advanced in place with a goal queue)
    GoalQueue goals;        // goal queue (q = 0: none)
    VehicleArgs veh;        // lane-following vehicles (n = 0: none)
    float4* state;          // [N] (px, py, vx, vy)
    const float2* robot_vel;  // [n_steps][robot_stride] or null (keep current)
    int robot_stride;       // entries per step in robot_vel (normally E)
    int n_steps;
    float dt, tau, tau_o, R, robot_alpha;
    int K;
    int seg_vd;             // 1: velocity-dependent segment half-planes
    int* nbr_out;           // [N][K] or null: neighbour lists of the last step
    EnvStats* stats;        // [E] or null: accumulate statistics
    int* reach;             // [N] or null: 1-based step of first goal reach
    long long step_base;    // global index of the first step of this launch
    WorkCount* work;        // or null: count work items
    int* err;               // device error word
    int max_agents;         // largest environment in `order` (sizes shared memory)
    int cell_split;         // grid cells >= R / cell_split (1: 3x3 search, 2: 5x5)
    int coop_fallback;      // infeasible LPs: in place (0), by whole warps after the pass (1), by one
                            // lane each after the pass, spread over the warps (2)
    int lanes;              // lanes per agent: 1, 2, 4 or 8 (groups of lanes share an agent's work)
    int agent_order;        // one lane per agent: 0 = warps take runs of cell order, 1 = interleaved
    // Per-environment overrides (all null for a batch handle; set by the
    // serving loop, whose environments are slots of fixed capacity):
    const int* env_count;   // [E] agents, instead of env_start differences
    const int* seg_count;   // [E] segments, instead of seg_start differences
    const int* env_steps;   // [E] steps of this launch, instead of n_steps
    const int* env_step0;   // [E] steps already done: robot command of step s is
                            //     robot_vel[e * rv_env_stride + step0 + s], reach steps offset by step0
    int rv_env_stride;
};

// Launch-shape knobs of the resident kernel (chosen by crowd_autotune).
struct Tuning {
    int block_threads;  // 0: one group of lanes per agent of the largest environment (64..512 threads)
    int coop_fallback;  // only with one lane per agent
    int cell_split;
    int lanes;          // lanes per agent: 1, 2, 4 or 8
    int order;          // agent order over the warps (one lane per agent only)
    int tiled_queue;    // tiled path: 1 = persistent work-queue update, 0 = one CTA per tile
};

// One large environment of the tiled path (static uniform grid, cell >= R).
// Order in which the persistent tiled update hands out its work items:
// longest first, so that the step does not end waiting for a costly item
// taken last.  Each item's cost (clock cycles of its warp) in one step puts
// it in one of kItemBuckets classes relative to the previous step's mean
// cost (>= 2, 1.4, 1, 0.7 times the mean, and below); the next step hands
// out the classes in that order.  The order changes no result: every agent
// is computed the same way whichever warp takes it and when.
constexpr int kItemBuckets = 5;
struct ItemSched {
    unsigned long long cost_sum;  // cycles of the items of the step in progress
    float mean;                   // mean item cost of the last finished step (0: none yet)
    int count_next[kItemBuckets]; // items per class in the step in progress
    int count[kItemBuckets];      // items per class of the last finished step (the order being handed out)
    int cursor[kItemBuckets];     // placement cursors of the order being built
};

struct TiledEnv {
    int e;          // environment id
    int base, n;    // agents [base, base + n)
    int seg0;       // first segment of the environment
    int robot;      // environment-local robot index or -1
    int co;         // offset of the environment's cells in count/start/segment-list arrays
    int W, H;       // grid cells
    float x0, y0, inv_c;
    int tx, ty;     // cells per tile of the update kernel (choose_tile)
    int span;       // cells searched on each side of an agent's cell (cells >= R / span)
};

// Largest side, in cells, of a tile of the tiled update kernel.
constexpr int kTileMax = 8;
// Largest neighbour-search span of a tiled environment (cells of R / 2).
constexpr int kTiledSpanMax = 2;
// Threads of a CTA of the tiled update kernel.
constexpr int kTiledUpdateThreads = 256;
// Threads of a CTA of the persistent (work-queue) tiled update kernel, and
// agents per work item (one warp).
constexpr int kQueueThreads = 128;
constexpr int kQueueItem = 32;
// CTAs of the persistent update per SM the compiler budgets registers for.
// With the statistics and work-count code (65,536 / (6 x 128) = 85, 80 a
// thread): on the 500-step 16 x 20,000 crowd 6 CTAs (24 warps per SM) ran
// 257.1 ms, 5 CTAs (96 registers) 265.9 ms, 7 (72 registers, more spills)
// 266.4 ms; 4 (128 registers) was slower than 5.  The plain form (neither,
// so fewer live values) at 8 CTAs (64 registers, 32 warps) ran 238.4 ms,
// against 247.9 ms at 6, 242.1 ms at 7, 245.6 ms at 9 (56 registers) and
// 262.6 ms at 10 (48 registers): below 64 registers the spills cost more
// than the added warps hide.
#ifndef CROWD_QUEUE_MINB
#define CROWD_QUEUE_MINB 6
#endif
#ifndef CROWD_QUEUE_PLAIN_MINB
#define CROWD_QUEUE_PLAIN_MINB 8
#endif
constexpr int kQueueMinBlocks = CROWD_QUEUE_MINB;
constexpr int kQueuePlainMinBlocks = CROWD_QUEUE_PLAIN_MINB;
// Cells of R / 2 are used when the tiled agents of a handle number at least
// this many rounds of kTiledUpdateThreads on every SM.
constexpr int kFineCellRounds = 4;
// Agents a tile of the update kernel (256 threads) should hold on average.
constexpr double kTileFill = 230.0;

// Tile of a tiled environment: the largest near-square block of cells
// (tx = ty or ty + 1, at most kTileMax a side) whose expected agents, n
// spread evenly over the W x H grid, fit one round of the update kernel's
// threads with a margin.  A tile of 4 x 4 cells in a crowd of 2 agents per
// m^2 (R = 3 m) holds about 290 agents, and its second round kept one warp
// of eight busy; 4 x 3 cells run the 20,000-agent crowd 10 % faster.
inline void choose_tile(int n, int W, int H, int& tx, int& ty) {
    const double per_cell = (double)n / ((double)W * (double)H);
    tx = ty = 1;
    for (int t = 3; t <= 2 * kTileMax; ++t) {  // t = tx + ty
        const int a = (t + 1) / 2, b = t / 2;
        if (a * b * per_cell > kTileFill) break;
        tx = a;
        ty = b;
    }
}
// Largest grid side of a tiled environment.
constexpr int kTiledGridMax = 512;

enum : int { kTiledStep = 0, kTiledStepCount = 1, kTiledStatsOnly = 2 };

// Arguments of one step of the tiled path.
struct TiledStepArgs {
    const TiledEnv* envs;
    int n_envs;
    float4* state_in;         // [N] state at the start of the step (robot slots get their command)
    float4* state_out;        // [N] state after the step
    const float2* robot_vel;  // [E] commands of this step, or null (keep current)
    const float4* par;
    float2* goal;             // [N] current goals (advanced in tiled_count with a goal queue)
    GoalQueue goals;
    EpisodeArgs ep;
    VehicleArgs veh;          // cars (stepped by tiled_vehicles when veh_on)
    int veh_on;               // some tiled environment has cars
    const float4* segs;
    const int* seg_cell_start;  // [cells + 1 per env] per-cell segment lists
    const int* seg_cell_ids;
    int* key;                 // [N] scratch: cell of each agent
    int* rank;                // [N] scratch: rank inside the cell
    int* count;               // [cells] scratch: zero between steps
    int* start;               // [cells + 1 per env] scratch: cell starts (global sorted slots)
    float4* sorted_pv;        // [N] scratch: state in cell order
    int* sorted_id;           // [N] scratch: environment-local index of each sorted slot
    int halo_cap;             // agents the update kernel stages in shared memory
    // persistent update (use_queue != 0): work items of 32 consecutive sorted
    // slots of one environment, item_start[t] the first item of tiled
    // environment t ([n_envs + 1]), taken from the counter *queue (zeroed by
    // tiled_scan) by the warps of queue_grid CTAs (queue_grid_plain for the
    // form without statistics and work counts)
    int use_queue;
    const int* item_start;
    int n_items;
    int* queue;
    int queue_grid, queue_grid_plain;
    // dispatch order of the items (longest first, by the cost each item took
    // in the previous step; see ItemSched), or null for item order
    int* item_order;
    unsigned char* item_bucket;  // [n_items] cost class of each item in the previous step
    ItemSched* sched;
    float R, dt, tau, tau_o, robot_alpha;
    int K;
    int seg_vd;               // 1: velocity-dependent segment half-planes
    int mode;                 // kTiledStep / kTiledStepCount / kTiledStatsOnly
    int* nbr_out;             // [N][K] or null
    EnvStats* stats;          // [E] or null
    int* reach;               // [N] (with stats)
    long long* step_index;    // device step counter (reach steps are 1-based from it)
    WorkCount* work;
    int* err;
};

// Halo agents the tiled update kernel stages in shared memory (60 KB).
constexpr int kHaloCap = 3072;

size_t tiled_smem_bytes(int halo_cap);
// CTAs of the persistent tiled update kernel for neighbour cap K that fit on
// one SM (0 on error).
int tiled_queue_blocks_per_sm(int K, bool plain);
// One-time kernel attributes of the tiled path (before any capture).
cudaError_t tiled_init(int halo_cap);
// Enqueue one thread setting the device step counter.
cudaError_t launch_set_step(long long* p, long long value, cudaStream_t s);
// Enqueue one step of the tiled path (4 kernels + bookkeeping).
// Enqueues one tiled step; *n_kernels (if given) receives how many kernels it
// launched.
cudaError_t launch_tiled_step(const TiledStepArgs& a, int max_agents, int max_tiles, cudaStream_t s,
                              int* n_kernels = nullptr);

size_t resident_smem_bytes(int max_agents, int K, int block);

}  // namespace crowd

#include <vector>

#include <nvtx3/nvToolsExt.h>

namespace crowd {

// An NVTX range over a scope of host code (the library's calls and the
// stages of a step show up by name under a profiler; without one attached a
// push or pop costs a call that returns).
struct TraceRange {
    explicit TraceRange(const char* name) { nvtxRangePushA(name); }
    ~TraceRange() { nvtxRangePop(); }
    TraceRange(const TraceRange&) = delete;
    TraceRange& operator=(const TraceRange&) = delete;
};

// Host-side construction of the static segment lists (crowd_api.cu).
double seg_reach(int base, int n, const float* radii, const float* vmax, float tau, float tau_obst);
void build_seg_lists(const float* segs, int seg0, int ns, double x0, double y0, double cc, int W, int H, double reach,
                     int off, std::vector<int>& seg_cell_start, std::vector<int>& seg_cell_ids);
SegGrid build_seg_grid(int base, int n, int seg0, int ns, const float* radii, const float* vmax, const float* segs,
                       float tau, float tau_obst, int off, std::vector<int>& seg_cell_start,
                       std::vector<int>& seg_cell_ids);
int resident_block_threads(int max_agents);
int resident_kmax(int K);
// Launch on `stream`; `grid` CTAs pull environments from the queue.
cudaError_t launch_resident(const ResidentArgs& a, int grid, int block, cudaStream_t stream);
// CTAs of the resident kernel that fit on one SM for this configuration.
int resident_ctas_per_sm(int max_agents, int block, int K, int lanes);
cudaError_t launch_resident_lanes2(const ResidentArgs& a, int grid, int block, cudaStream_t stream);
cudaError_t launch_resident_lanes4(const ResidentArgs& a, int grid, int block, cudaStream_t stream);
cudaError_t launch_resident_lanes8(const ResidentArgs& a, int grid, int block, cudaStream_t stream);
int resident_ctas_lanes2(int max_agents, int block, int K);
int resident_ctas_lanes4(int max_agents, int block, int K);
int resident_ctas_lanes8(int max_agents, int block, int K);

}  // namespace crowd
