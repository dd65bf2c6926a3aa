// C ABI of the crowd library: argument checks, device memory, launches.
//
// Every call validates its arguments on the host before anything is
// enqueued, returns a crowd_status, and records a message for
// crowd_last_error().  The handle owns all device memory; inputs are copied.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <numeric>
#include <string>
#include <vector>

#include "../../include/crowd.h"
#include "crowd_internal.h"

using namespace crowd;

namespace {

thread_local std::string g_last_error;

crowd_status fail(crowd_status st, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return st;
}

crowd_status cuda_fail(cudaError_t e, const char* what) {
    if (e == cudaErrorMemoryAllocation) return fail(CROWD_ENOMEM, "%s: %s", what, cudaGetErrorString(e));
    return fail(CROWD_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define CUDA_TRY(expr, what)                         \
    do {                                             \
        cudaError_t e_ = (expr);                     \
        if (e_ != cudaSuccess) return cuda_fail(e_, what); \
    } while (0)

bool finite_all(const float* p, size_t n) {
    for (size_t i = 0; i < n; ++i)
        if (!std::isfinite(p[i])) return false;
    return true;
}

template <class T>
cudaError_t dev_alloc(T** p, size_t count) {
    *p = nullptr;
    if (count == 0) count = 1;
    return cudaMalloc((void**)p, sizeof(T) * count);
}

}  // namespace

struct crowd_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    int32_t E = 0;
    int64_t N = 0, S = 0;
    int max_agents = 0;
    crowd_params p{};
    int64_t step_index = 0;
    bool broken = false;

    // device arrays
    int* env_start = nullptr;
    int* seg_start = nullptr;
    int* robot_index = nullptr;
    int* order = nullptr;
    int* queue = nullptr;
    int* err = nullptr;
    float4* state = nullptr;
    float4* par = nullptr;
    float2* goal = nullptr;
    float2* goal_queue = nullptr;  // [N][goal_q] (crowd_set_goal_queue)
    int* goal_idx = nullptr;       // [N]
    int goal_q = 0, goal_cyclic = 0;
    int* pool_start = nullptr;     // [E + 1] goal pool (crowd_set_goal_pool); null: no pool
    float2* pool = nullptr;        // [P]
    uint64_t pool_seed = 0;
    size_t goal_queue_cap = 0;     // entries allocated in goal_queue
    int* ep_steps = nullptr;       // [E] episode lengths (crowd_set_episodes); null: no episodes
    float4* ep_state = nullptr;    // [N] agent rows at the start of an episode
    float2* ep_goal = nullptr;     // [N] goals at the start of an episode
    int* ep_gidx = nullptr;        // [N] goal-queue counters at the start (with a queue)
    float* ep_veh = nullptr;       // [2V] car arcs at the start (with cars): s | v
    unsigned char* ep_mask = nullptr;  // [E] environments to start over now (crowd_restart_envs)
    int64_t ep_origin = 0;         // step_index at which the episode clock reads 0
    std::vector<int> h_ep_steps;   // host copy of ep_steps (empty: no episodes)
    // lane-following vehicles (crowd_set_vehicles)
    int n_veh = 0;
    int* veh_start = nullptr;      // [E + 1]
    int* veh_agent = nullptr;      // [V]
    int* veh_lane = nullptr;       // [V]
    float* veh_s = nullptr;        // [V]
    float* veh_v = nullptr;        // [V]
    float* veh_pref = nullptr;     // [V] preferred speeds of the car agents before they became cars
    float4* veh_par_a = nullptr;   // [V]
    float2* veh_par_b = nullptr;   // [V]
    float2* lane_pts = nullptr;    // [P]
    int* lane_start = nullptr;     // [n_lanes + 1]
    float* lane_cum = nullptr;     // [P + n_lanes]
    float veh_half_width = 0.f, veh_lookahead = 0.f;
    std::vector<int> h_env_start;  // [E + 1] host copy
    std::vector<char> h_env_tiled; // [E] environment stepped by the tiled path
    bool tiled_cars = false;       // some tiled environment has cars
    float4* segs = nullptr;
    float2* robot_vel = nullptr;
    size_t robot_vel_cap = 0;
    int* nbr = nullptr;
    int* reach = nullptr;
    EnvStats* stats = nullptr;
    WorkCount* work = nullptr;

    // resident path: environments that fit one CTA (the first n_res of `order`)
    int n_res = 0;
    std::vector<int> h_res_envs;  // host copy of the first n_res entries of `order`
    int res_max_agents = 0;
    int res_max_work = 0;  // largest count of solved (non-robot) agents of a resident environment
    int block = 0, grid = 0;  // resident launch shape for `tune`
    Tuning tune{0, 0, 1, 1, 0, 1};
    int sms = 0;

    // tiled path: larger environments (or all, with CROWD_FLAG_FORCE_TILED)
    int n_tiled = 0, tiled_max_agents = 0, tiled_max_tiles = 0, halo_cap = 0;
    std::vector<TiledEnv> h_tenvs;
    TiledEnv* tenvs = nullptr;
    float4* state_b = nullptr;
    float4* sorted_pv = nullptr;
    int* key = nullptr;
    int* rank = nullptr;
    int* count = nullptr;
    int* start = nullptr;
    int* sorted_id = nullptr;
    int* seg_cell_start = nullptr;
    int* seg_cell_ids = nullptr;
    SegGrid* seg_grid = nullptr;
    long long* d_step = nullptr;
    cudaStream_t cap_stream = nullptr;
    int* item_start = nullptr;  // [n_tiled + 1] work items (32 sorted slots) of the persistent update
    int n_items = 0;
    int* tqueue = nullptr;      // work-item counter of the persistent update
    int* item_order = nullptr;  // [n_items] dispatch order of the items (ItemSched)
    unsigned char* item_bucket = nullptr;  // [n_items] cost class of each item in the last step
    ItemSched* sched = nullptr;
    int queue_grid = 0;         // its CTAs: as many as fit on the GPU
    int queue_grid_plain = 0;   // the same for its form without statistics and work counts
    cudaGraphExec_t graph = nullptr;
    int64_t graph_kernels = 0;    // kernel launches one replay of `graph` performs
    int64_t kernel_launches = 0;  // kernels this handle's steps enqueued (graph replays by their kernels)
    struct GraphKey {
        int n_steps = 0;
        float dt = 0.f;
        const void* rv = nullptr;
        std::vector<int> stats_before;  // steps preceded by a statistics pass (episode starts)
        bool operator==(const GraphKey& o) const {
            return n_steps == o.n_steps && dt == o.dt && rv == o.rv && stats_before == o.stats_before;
        }
    } gkey;

    ~crowd_ctx() {
        if (graph) cudaGraphExecDestroy(graph);
        if (cap_stream) cudaStreamDestroy(cap_stream);
        void* ptrs[] = {env_start, seg_start, robot_index, order, queue, err, state, par, goal, goal_queue, goal_idx,
                        veh_start, veh_agent, veh_lane, veh_s, veh_v, veh_par_a, veh_par_b, lane_pts, lane_start,
                        lane_cum, veh_pref, ep_steps, ep_state, ep_goal, ep_gidx, ep_veh, ep_mask, pool_start, pool,
                        segs, robot_vel, nbr, reach, stats, work, tenvs, state_b, sorted_pv, key, rank,
                        count, start, sorted_id, seg_cell_start, seg_cell_ids, seg_grid, d_step, item_start,
                        tqueue, item_order, item_bucket, sched};
        for (void* q : ptrs)
            if (q) cudaFree(q);
    }
};

namespace crowd {

// Error reporting shared with the serving loop (crowd_server.cu).
crowd_status api_fail(crowd_status st, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return st;
}

// Largest r + tau_obst v_max over an environment's agents, with a margin.
double seg_reach(int base, int n, const float* radii, const float* vmax, float tau, float tau_obst) {
    double reach = 0.0;
    const double tau_o = tau_obst > 0.f ? tau_obst : tau;
    for (int i = 0; i < n; ++i) reach = std::max(reach, (double)radii[base + i] + tau_o * (double)vmax[base + i]);
    return reach * (1.0 + 1e-5) + 1e-6;
}

// Per-cell segment lists of a W x H grid (origin x0, y0, cell size cc) at
// offset `off`: segment s is listed in a cell when it comes within
// reach + half the cell diagonal of the cell's centre, hence within reach of
// some point of the cell.  Agents clamped into a border cell from outside the
// grid are covered too as long as the grid contains every segment: clamping
// onto a box does not increase distances to points inside it.
void build_seg_lists(const float* segs, int seg0, int ns, double x0, double y0, double cc, int W, int H, double reach,
                     int off, std::vector<int>& seg_cell_start, std::vector<int>& seg_cell_ids) {
    const double half_diag = 0.5 * std::sqrt(2.0) * cc;
    std::vector<std::vector<int>> lists((size_t)W * H);
    for (int s = 0; s < ns; ++s) {
        const float* q = segs + 4 * (seg0 + s);
        const double ax = q[0], ay = q[1], bx = q[2], by = q[3];
        const int cx0 = std::max(0, (int)std::floor((std::min(ax, bx) - reach - x0) / cc) - 1);
        const int cx1 = std::min(W - 1, (int)std::floor((std::max(ax, bx) + reach - x0) / cc) + 1);
        const int cy0 = std::max(0, (int)std::floor((std::min(ay, by) - reach - y0) / cc) - 1);
        const int cy1 = std::min(H - 1, (int)std::floor((std::max(ay, by) + reach - y0) / cc) + 1);
        const double ex = bx - ax, ey = by - ay, e2 = ex * ex + ey * ey;
        for (int cy = cy0; cy <= cy1; ++cy)
            for (int cx = cx0; cx <= cx1; ++cx) {
                const double px = x0 + (cx + 0.5) * cc, py = y0 + (cy + 0.5) * cc;
                double t = ((px - ax) * ex + (py - ay) * ey) / e2;
                t = std::min(1.0, std::max(0.0, t));
                const double dx = ax + t * ex - px, dy = ay + t * ey - py;
                if (std::sqrt(dx * dx + dy * dy) < reach + half_diag) lists[(size_t)cy * W + cx].push_back(s);
            }
    }
    if ((int)seg_cell_start.size() < off + W * H + 1) seg_cell_start.resize(off + W * H + 1);
    for (size_t k = 0; k < lists.size(); ++k) {
        seg_cell_start[off + k] = (int)seg_cell_ids.size();
        seg_cell_ids.insert(seg_cell_ids.end(), lists[k].begin(), lists[k].end());
    }
    seg_cell_start[off + lists.size()] = (int)seg_cell_ids.size();
}

// Segment grid of a resident environment: the bounding box of its segments
// padded by reach, cells of at least reach/2 and at most 64 a side.
SegGrid build_seg_grid(int base, int n, int seg0, int ns, const float* radii, const float* vmax, const float* segs,
                       float tau, float tau_obst, int off, std::vector<int>& seg_cell_start,
                       std::vector<int>& seg_cell_ids) {
    SegGrid g{};
    g.off = off;
    if (ns == 0) {
        g.x0 = g.y0 = 0.f;
        g.inv_c = 1.f;
        g.W = g.H = 1;
        build_seg_lists(segs, seg0, 0, 0.0, 0.0, 1.0, 1, 1, 0.0, off, seg_cell_start, seg_cell_ids);
        return g;
    }
    const double reach = seg_reach(base, n, radii, vmax, tau, tau_obst);
    double x0 = 1e300, y0 = 1e300, x1 = -1e300, y1 = -1e300;
    for (int s = 0; s < ns; ++s) {
        const float* q = segs + 4 * (seg0 + s);
        x0 = std::min({x0, (double)q[0], (double)q[2]});
        x1 = std::max({x1, (double)q[0], (double)q[2]});
        y0 = std::min({y0, (double)q[1], (double)q[3]});
        y1 = std::max({y1, (double)q[1], (double)q[3]});
    }
    x0 -= reach;
    y0 -= reach;
    x1 += reach;
    y1 += reach;
    const double ext = std::max(x1 - x0, y1 - y0);
    const float c = (float)std::max(std::max(reach * 0.5, 1e-3), ext / 63.0);
    g.x0 = (float)x0;
    g.y0 = (float)y0;
    g.inv_c = std::nextafter(1.0f / c, 0.0f);
    const double cc = 1.0 / (double)g.inv_c;
    g.W = std::min(64, (int)((x1 - x0) / cc) + 1);
    g.H = std::min(64, (int)((y1 - y0) / cc) + 1);
    build_seg_lists(segs, seg0, ns, x0, y0, cc, g.W, g.H, reach, off, seg_cell_start, seg_cell_ids);
    return g;
}

}  // namespace crowd

namespace {

// Cached tiled graphs bake the kernel arguments in, goal queue included.
void drop_graph(crowd_t h) {
    if (h->graph) {
        cudaGraphExecDestroy(h->graph);
        h->graph = nullptr;
    }
}

// Episodes snapshot goals, goal-queue counters and cars: setting any of them
// again removes the episodes.
void drop_episodes(crowd_t h) {
    if (h->h_ep_steps.empty()) return;
    void** ps[] = {(void**)&h->ep_steps, (void**)&h->ep_state, (void**)&h->ep_goal, (void**)&h->ep_gidx,
                   (void**)&h->ep_veh};
    cudaStreamSynchronize(h->stream);
    for (void** q : ps)
        if (*q) {
            cudaFree(*q);
            *q = nullptr;
        }
    h->h_ep_steps.clear();
    drop_graph(h);
}

EpisodeArgs episode_args(crowd_t h) {
    EpisodeArgs ep{};
    if (h->h_ep_steps.empty()) return ep;
    ep.steps = h->ep_steps;
    ep.state = h->ep_state;
    ep.goal = h->ep_goal;
    ep.gidx = h->ep_gidx;
    ep.veh_s = h->ep_veh;
    ep.veh_v = h->ep_veh ? h->ep_veh + h->n_veh : nullptr;
    ep.origin = h->ep_origin;
    return ep;
}

// Episodes of the resident environments: environment order[blockIdx.x]
// takes its episode-start rows, goals, goal-queue counters and car arcs when
// its episode starts at global step `step`.
__global__ void restart_resident_envs(EpisodeArgs ep, const int* order, const int* env_start, VehicleArgs veh,
                                      float4* state, float2* goal, int* gidx, long long step) {
    const int e = order[blockIdx.x];
    if (!episode_restart(ep.steps[e], step, ep.origin)) return;
    const int i = blockIdx.y * blockDim.x + threadIdx.x;
    const int g = env_start[e] + i;
    if (g < env_start[e + 1]) {
        state[g] = ep.state[g];
        goal[g] = ep.goal[g];
        if (ep.gidx) gidx[g] = ep.gidx[g];
    }
    if (ep.veh_s) {
        const int vi = veh.start[e] + i;
        if (vi < veh.start[e + 1]) {
            veh.s[vi] = ep.veh_s[vi];
            veh.v[vi] = ep.veh_v[vi];
        }
    }
}

// Environment blockIdx.x, when mask[e] is set, takes its episode-start rows,
// goals, goal-queue counters and car arcs (crowd_restart_envs).
__global__ void restart_masked_envs(EpisodeArgs ep, const unsigned char* mask, const int* env_start, VehicleArgs veh,
                                    float4* state, float2* goal, int* gidx) {
    const int e = blockIdx.x;
    if (!mask[e]) return;
    const int i = blockIdx.y * blockDim.x + threadIdx.x;
    const int g = env_start[e] + i;
    if (g < env_start[e + 1]) {
        state[g] = ep.state[g];
        goal[g] = ep.goal[g];
        if (ep.gidx) gidx[g] = ep.gidx[g];
    }
    if (ep.veh_s) {
        const int vi = veh.start[e] + i;
        if (vi < veh.start[e + 1]) {
            veh.s[vi] = ep.veh_s[vi];
            veh.v[vi] = ep.veh_v[vi];
        }
    }
}

// Goals that move on inside the kernels: a queue or a pool.
bool goals_move(crowd_t h) { return h->goal_q > 0 || h->pool_start != nullptr; }

GoalQueue goal_args(crowd_t h) {
    GoalQueue g{h->goal_queue, h->goal_idx, h->goal_q, h->goal_cyclic, h->pool_start, h->pool,
                make_uint2((unsigned)(h->pool_seed & 0xFFFFFFFFu), (unsigned)(h->pool_seed >> 32))};
    return g;
}

// A fixed goal set or a queue replaces a pool.
void drop_pool(crowd_t h) {
    if (!h->pool_start) return;
    cudaStreamSynchronize(h->stream);
    cudaFree(h->pool_start);
    cudaFree(h->pool);
    h->pool_start = nullptr;
    h->pool = nullptr;
    drop_graph(h);
}

crowd_status check_handle(crowd_t h) {
    if (!h) return fail(CROWD_EINVAL, "null handle");
    if (h->broken) return fail(CROWD_ESTATE, "handle is unusable after an earlier CUDA failure");
    return CROWD_OK;
}

// Copy a host or device buffer of `bytes` into the device buffer `dst`.
crowd_status copy_in(crowd_t h, void* dst, const void* src, size_t bytes, int32_t kind, const char* what) {
    if (kind != CROWD_HOST && kind != CROWD_DEVICE) return fail(CROWD_EINVAL, "%s: ptr_kind must be 0 or 1", what);
    if (bytes == 0) return CROWD_OK;
    cudaError_t e = cudaMemcpyAsync(dst, src, bytes, kind == CROWD_HOST ? cudaMemcpyHostToDevice
                                                                         : cudaMemcpyDeviceToDevice,
                                    h->stream);
    if (e != cudaSuccess) return cuda_fail(e, what);
    return CROWD_OK;
}

crowd_status read_err_word(crowd_t h) {
    int err = 0;
    CUDA_TRY(cudaMemcpyAsync(&err, h->err, sizeof(int), cudaMemcpyDeviceToHost, h->stream), "read error word");
    CUDA_TRY(cudaStreamSynchronize(h->stream), "synchronize");
    if (err) {
        CUDA_TRY(cudaMemsetAsync(h->err, 0, sizeof(int), h->stream), "clear error word");
        if (err & kErrObstacleOverflow)
            return fail(CROWD_EDEVICE, "an agent had more than %d static segments in reach in one step",
                        kMaxObstacleLines);
        return fail(CROWD_EDEVICE, "device error word 0x%x", err);
    }
    return CROWD_OK;
}


// Static grid of a tiled environment: the bounding box of its agents' start
// positions and its segments, padded by R, with cells of at least R / span
// (times a margin for FP32 rounding of cell coordinates) and at most
// kTiledGridMax a side; and for every cell the ascending list of the
// environment's segments that can come within r + tau_obst v_max of a point
// of the cell.  Agents that leave the box are clamped into its border cells,
// which keeps both the (2 span + 1)^2-cell neighbour search and the segment
// lists exact.
void build_tiled_env(int e, int base, int n, int seg0, int ns, int robot, const float* pos, const float* radii,
                     const float* vmax, const float* segs, const crowd_params& p, int co, bool fine_cells,
                     TiledEnv& te, std::vector<int>& seg_cell_start, std::vector<int>& seg_cell_ids) {
    const double R = p.neighbor_dist;
    double x0 = 1e300, y0 = 1e300, x1 = -1e300, y1 = -1e300;
    for (int i = 0; i < n; ++i) {
        x0 = std::min(x0, (double)pos[2 * (base + i)]);
        x1 = std::max(x1, (double)pos[2 * (base + i)]);
        y0 = std::min(y0, (double)pos[2 * (base + i) + 1]);
        y1 = std::max(y1, (double)pos[2 * (base + i) + 1]);
    }
    for (int s = 0; s < ns; ++s) {
        const float* q = segs + 4 * (seg0 + s);
        x0 = std::min({x0, (double)q[0], (double)q[2]});
        x1 = std::max({x1, (double)q[0], (double)q[2]});
        y0 = std::min({y0, (double)q[1], (double)q[3]});
        y1 = std::max({y1, (double)q[1], (double)q[3]});
    }
    if (!(x1 >= x0)) x0 = x1 = y0 = y1 = 0.0;
    x0 -= R;
    y0 -= R;
    x1 += R;
    y1 += R;
    const double ext = std::max(x1 - x0, y1 - y0);
    // with fine_cells, cells of R / 2 (5 x 5 cells searched, about 30 % fewer
    // candidates than 3 x 3 cells of R) when a cell still holds every
    // colliding pair, so that the +-1-cell collision count stays exact
    double rmax = 0.0;
    for (int i = 0; i < n; ++i) rmax = std::max(rmax, (double)radii[base + i]);
    te.span = fine_cells && R * 0.5 >= 2.0 * rmax ? kTiledSpanMax : 1;
    const float c = (float)std::max(R * 1.0001 / te.span, ext / (kTiledGridMax - 1));
    te.e = e;
    te.base = base;
    te.n = n;
    te.seg0 = seg0;
    te.robot = robot;
    te.co = co;
    te.x0 = (float)x0;
    te.y0 = (float)y0;
    // round toward zero so that the cell size in use is >= c
    te.inv_c = std::nextafter(1.0f / c, 0.0f);
    const double cc = 1.0 / (double)te.inv_c;
    te.W = std::min(kTiledGridMax, (int)((x1 - x0) / cc) + 1);
    te.H = std::min(kTiledGridMax, (int)((y1 - y0) / cc) + 1);
    choose_tile(n, te.W, te.H, te.tx, te.ty);

    build_seg_lists(segs, seg0, ns, x0, y0, cc, te.W, te.H,
                    seg_reach(base, n, radii, vmax, p.time_horizon, p.time_horizon_obst), co, seg_cell_start,
                    seg_cell_ids);
}


// Launch shape of the resident kernel for a tuning: block threads (0: one per
// agent of the largest environment, 64..512) and as many CTAs as fit.
void apply_tuning(crowd_t h, const Tuning& t) {
    if (t.tiled_queue != h->tune.tiled_queue) drop_graph(h);  // cached tiled graphs hold the update kernel
    h->tune = t;
    // default: one thread per agent, or one group of lanes per solved agent
    // (the robot is integrated apart in that mode)
    h->block = t.block_threads > 0 ? t.block_threads
               : t.lanes == 1      ? resident_block_threads(h->res_max_agents)
                                   : resident_block_threads(std::min(std::max(h->res_max_work, 1) * t.lanes, 512));
    const int per_sm =
        std::max(1, resident_ctas_per_sm(h->res_max_agents, h->block, h->p.max_neighbors, t.lanes));
    h->grid = std::max(1, std::min(std::max(h->n_res, 1), per_sm * std::max(h->sms, 1)));
}

// Enqueue n steps of the resident environments on `s`.
crowd_status resident_launch(crowd_t h, float dt, const float2* rv, int n_steps, int64_t step_base, bool stats,
                             float tau_o, cudaStream_t s) {
    ResidentArgs a{};
    a.n_work = h->n_res;
    a.order = h->order;
    a.queue = h->queue;
    a.env_start = h->env_start;
    a.seg_start = h->seg_start;
    a.robot_index = h->robot_index;
    a.segs = h->segs;
    a.seg_grid = h->seg_grid;
    a.seg_cell_start = h->seg_cell_start;
    a.seg_cell_ids = h->seg_cell_ids;
    a.par = h->par;
    a.goal = h->goal;
    a.goals = goal_args(h);
    a.seg_vd = (h->p.flags & CROWD_FLAG_VELOCITY_SEGMENTS) ? 1 : 0;
    a.veh = VehicleArgs{h->n_veh, h->veh_start, h->veh_agent, h->veh_lane, h->veh_s, h->veh_v, h->veh_par_a,
                        h->veh_par_b, h->lane_pts, h->lane_start, h->lane_cum, h->veh_half_width, h->veh_lookahead};
    a.state = h->state;
    a.robot_vel = rv;
    a.robot_stride = h->E;
    a.n_steps = n_steps;
    a.dt = dt;
    a.tau = h->p.time_horizon;
    a.tau_o = tau_o;
    a.R = h->p.neighbor_dist;
    a.robot_alpha = h->p.robot_responsibility;
    a.K = h->p.max_neighbors;
    a.nbr_out = h->nbr;
    a.stats = stats ? h->stats : nullptr;
    a.reach = stats ? h->reach : nullptr;
    a.step_base = step_base;
    a.work = h->work;
    a.err = h->err;
    a.max_agents = h->res_max_agents;
    a.cell_split = h->tune.cell_split;
    a.coop_fallback = h->tune.lanes == 1 ? h->tune.coop_fallback : 0;
    a.lanes = h->tune.lanes;
    a.agent_order = h->tune.lanes == 1 ? h->tune.order : 0;
    CUDA_TRY(cudaMemsetAsync(h->queue, 0, sizeof(int), s), "reset work queue");
    cudaError_t e = launch_resident(a, h->grid, h->block, s);
    if (e != cudaSuccess) {
        h->broken = e != cudaErrorInvalidValue && e != cudaErrorInvalidConfiguration;
        return cuda_fail(e, "launch crowd step");
    }
    h->kernel_launches += 1;
    return CROWD_OK;
}

// Steps k in [0, n_steps) of a call at whose start a resident environment
// starts over (episodes).
std::vector<int> resident_restart_steps(crowd_t h, int n_steps) {
    if (h->h_ep_steps.empty()) return {};
    std::vector<char> mark(n_steps, 0);
    const long long t0 = h->step_index - h->ep_origin;  // clock at k = 0
    for (int e : h->h_res_envs) {
        const long long L = h->h_ep_steps[e];
        if (L <= 0) continue;
        long long t = t0 <= 0 ? L : ((t0 + L - 1) / L) * L;  // first start at a clock reading > 0
        for (; t - t0 < n_steps; t += L) mark[t - t0] = 1;
    }
    std::vector<int> out;
    for (int k = 0; k < n_steps; ++k)
        if (mark[k]) out.push_back(k);
    return out;
}

// n steps of the resident environments.  With episodes the call is split at
// the steps where a resident environment starts over, and the starts run
// between the launches, so the step kernel carries no episode code: each
// launch counts its final state in the statistics and the next one does not
// count its first, so an episode's last state is counted and the restored
// start not.
crowd_status resident_steps(crowd_t h, float dt, const float2* rv, int n_steps, bool stats, float tau_o,
                            cudaStream_t s) {
    const std::vector<int> starts = resident_restart_steps(h, n_steps);
    if (starts.empty()) return resident_launch(h, dt, rv, n_steps, h->step_index, stats, tau_o, s);
    const EpisodeArgs ep = episode_args(h);
    const VehicleArgs veh{h->n_veh, h->veh_start, h->veh_agent, h->veh_lane, h->veh_s, h->veh_v, h->veh_par_a,
                          h->veh_par_b, h->lane_pts, h->lane_start, h->lane_cum, h->veh_half_width, h->veh_lookahead};
    const int span = std::max(h->res_max_agents, CROWD_MAX_VEHICLES_PER_ENV);
    int k = 0;
    size_t q = 0;
    while (k < n_steps) {
        if (q < starts.size() && starts[q] == k) {
            ++q;
            restart_resident_envs<<<dim3(h->n_res, (span + 255) / 256), 256, 0, s>>>(
                ep, h->order, h->env_start, veh, h->state, h->goal, h->goal_idx, h->step_index + k);
            CUDA_TRY(cudaGetLastError(), "episode start");
            h->kernel_launches += 1;
        }
        const int next = q < starts.size() ? starts[q] : n_steps;
        crowd_status st = resident_launch(h, dt, rv ? rv + (size_t)k * h->E : nullptr, next - k, h->step_index + k,
                                          stats, tau_o, s);
        if (st) return st;
        k = next;
    }
    return CROWD_OK;
}

// Arguments of step s (0-based) of an n-step tiled sequence.
TiledStepArgs tiled_args(crowd_t h, float dt, const float2* rv, int s, int n_steps, bool stats, float tau_o,
                         int mode) {
    TiledStepArgs a{};
    a.envs = h->tenvs;
    a.n_envs = h->n_tiled;
    a.state_in = (s & 1) ? h->state_b : h->state;
    a.state_out = (s & 1) ? h->state : h->state_b;
    a.robot_vel = (rv && mode != kTiledStatsOnly) ? rv + (size_t)s * h->E : nullptr;
    a.par = h->par;
    a.goal = h->goal;
    a.goals = goal_args(h);
    a.ep = episode_args(h);
    a.veh = VehicleArgs{h->n_veh, h->veh_start, h->veh_agent, h->veh_lane, h->veh_s, h->veh_v, h->veh_par_a,
                        h->veh_par_b, h->lane_pts, h->lane_start, h->lane_cum, h->veh_half_width, h->veh_lookahead};
    a.veh_on = h->tiled_cars ? 1 : 0;
    a.seg_vd = (h->p.flags & CROWD_FLAG_VELOCITY_SEGMENTS) ? 1 : 0;
    a.segs = h->segs;
    a.seg_cell_start = h->seg_cell_start;
    a.seg_cell_ids = h->seg_cell_ids;
    a.key = h->key;
    a.rank = h->rank;
    a.count = h->count;
    a.start = h->start;
    a.sorted_pv = h->sorted_pv;
    a.sorted_id = h->sorted_id;
    a.halo_cap = h->halo_cap;
    a.use_queue = h->tune.tiled_queue;
    a.item_start = h->item_start;
    a.n_items = h->n_items;
    a.queue = h->tqueue;
    a.item_order = a.use_queue ? h->item_order : nullptr;
    a.item_bucket = a.use_queue ? h->item_bucket : nullptr;
    a.sched = a.use_queue ? h->sched : nullptr;
    a.queue_grid = h->queue_grid;
    a.queue_grid_plain = h->queue_grid_plain;
    a.R = h->p.neighbor_dist;
    a.dt = dt;
    a.tau = h->p.time_horizon;
    a.tau_o = tau_o;
    a.robot_alpha = h->p.robot_responsibility;
    a.K = h->p.max_neighbors;
    a.mode = mode;
    a.nbr_out = (s == n_steps - 1 && mode != kTiledStatsOnly) ? h->nbr : nullptr;
    a.stats = stats ? h->stats : nullptr;
    a.reach = h->reach;
    a.step_index = h->d_step;
    a.work = mode == kTiledStatsOnly ? nullptr : h->work;
    a.err = h->err;
    return a;
}

// Steps k (0 < k < n_steps) of an n-step tiled call at whose start a tiled
// environment starts over, when statistics are on.
std::vector<int> tiled_stats_before(crowd_t h, int n_steps, bool stats) {
    std::vector<int> out;
    if (!stats || h->h_ep_steps.empty()) return out;
    for (int k = 1; k < n_steps; ++k)
        for (const TiledEnv& te : h->h_tenvs)
            if (te.n && episode_restart(h->h_ep_steps[te.e], h->step_index + k, h->ep_origin)) {
                out.push_back(k);
                break;
            }
    return out;
}

// Enqueue an n-step tiled sequence on `s`: the steps alternate between the
// two state buffers; an odd count ends with the tiled environments copied
// back; with statistics a last pass counts the collisions of the final state.
cudaError_t enqueue_tiled(crowd_t h, float dt, const float2* rv, int n_steps, bool stats, float tau_o,
                          cudaStream_t s, int64_t& kernels) {
    const std::vector<int> before = tiled_stats_before(h, n_steps, stats);
    size_t nb = 0;
    int nk = 0;
    for (int k = 0; k < n_steps; ++k) {
        const bool apart = nb < before.size() && before[nb] == k;
        if (apart) {
            // an environment starts over at step k: the statistics of every
            // environment's state at the start of k are counted first, so
            // that an episode's last state is counted and its restart not
            ++nb;
            cudaError_t e = launch_tiled_step(tiled_args(h, dt, nullptr, k, n_steps, stats, tau_o, kTiledStatsOnly),
                                              h->tiled_max_agents, h->tiled_max_tiles, s, &nk);
            kernels += nk;
            if (e != cudaSuccess) return e;
        }
        const int mode = (stats && k > 0 && !apart) ? kTiledStepCount : kTiledStep;
        cudaError_t e = launch_tiled_step(tiled_args(h, dt, rv, k, n_steps, stats, tau_o, mode), h->tiled_max_agents,
                                          h->tiled_max_tiles, s, &nk);
        kernels += nk;
        if (e != cudaSuccess) return e;
    }
    if (n_steps & 1) {
        for (const TiledEnv& te : h->h_tenvs) {
            if (!te.n) continue;
            cudaError_t e = cudaMemcpyAsync(h->state + te.base, h->state_b + te.base, sizeof(float4) * te.n,
                                            cudaMemcpyDeviceToDevice, s);
            if (e != cudaSuccess) return e;
        }
    }
    if (stats) {
        cudaError_t e = launch_tiled_step(tiled_args(h, dt, nullptr, 0, 1, stats, tau_o, kTiledStatsOnly),
                                          h->tiled_max_agents, h->tiled_max_tiles, s, &nk);
            kernels += nk;
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// Run the tiled environments n steps: a single step is launched directly;
// longer calls replay a CUDA graph of the whole sequence, captured once per
// (n_steps, dt, command buffer) and cached.
crowd_status tiled_steps(crowd_t h, float dt, const float2* rv, int n_steps, bool stats, float tau_o) {
    cudaError_t e = launch_set_step(h->d_step, h->step_index, h->stream);
    if (e != cudaSuccess) return cuda_fail(e, "set step index");
    h->kernel_launches += 1;
    if (n_steps == 1) {
        int64_t nk = 0;
        e = enqueue_tiled(h, dt, rv, n_steps, stats, tau_o, h->stream, nk);
        h->kernel_launches += nk;
        if (e != cudaSuccess) return cuda_fail(e, "launch tiled step");
        return CROWD_OK;
    }
    crowd_ctx::GraphKey key;
    key.n_steps = n_steps;
    key.dt = dt;
    key.rv = rv;
    key.stats_before = tiled_stats_before(h, n_steps, stats);
    if (!h->graph || !(key == h->gkey)) {
        if (h->graph) {
            cudaGraphExecDestroy(h->graph);
            h->graph = nullptr;
        }
        cudaGraph_t g = nullptr;
        e = cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return cuda_fail(e, "begin graph capture");
        int64_t nk = 0;
        cudaError_t le = enqueue_tiled(h, dt, rv, n_steps, stats, tau_o, h->cap_stream, nk);
        e = cudaStreamEndCapture(h->cap_stream, &g);
        if (le != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            return cuda_fail(le, "capture tiled steps");
        }
        if (e != cudaSuccess) return cuda_fail(e, "end graph capture");
        e = cudaGraphInstantiate(&h->graph, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            h->graph = nullptr;
            return cuda_fail(e, "instantiate graph");
        }
        h->gkey = key;
        h->graph_kernels = nk;
    }
    e = cudaGraphLaunch(h->graph, h->stream);
    if (e != cudaSuccess) return cuda_fail(e, "launch graph");
    h->kernel_launches += h->graph_kernels;
    return CROWD_OK;
}

}  // namespace

extern "C" {

int32_t crowd_abi_version(void) { return 5; }  // 5: crowd_read_launches, crowd_tuning.tiled_queue

const char* crowd_last_error(void) { return g_last_error.c_str(); }

int64_t crowd_num_agents(crowd_t h) { return h ? h->N : 0; }
int32_t crowd_num_envs(crowd_t h) { return h ? h->E : 0; }

crowd_status crowd_create(int32_t n_envs, const int32_t* agents_per_env, const float* radii,
                          const float* max_speeds, const float* pref_speeds, const float* init_pos,
                          const int32_t* robot_index, const int32_t* segs_per_env, const float* segments,
                          const crowd_params* p, void* cuda_stream, crowd_t* out) {
    const TraceRange trace("crowd_create");
    if (!out) return fail(CROWD_EINVAL, "out is null");
    *out = nullptr;
    if (!p) return fail(CROWD_EINVAL, "params is null");
    if (n_envs < 0) return fail(CROWD_EINVAL, "n_envs < 0");
    if (n_envs > 0 && !agents_per_env) return fail(CROWD_EINVAL, "agents_per_env is null");
    if (!(p->time_horizon > 0.f) || !std::isfinite(p->time_horizon))
        return fail(CROWD_EINVAL, "time_horizon must be finite and > 0");
    if (!(p->time_horizon_obst >= 0.f) || !std::isfinite(p->time_horizon_obst))
        return fail(CROWD_EINVAL, "time_horizon_obst must be finite and >= 0");
    if (!(p->neighbor_dist > 0.f) || !std::isfinite(p->neighbor_dist))
        return fail(CROWD_EINVAL, "neighbor_dist must be finite and > 0");
    if (p->max_neighbors < 0 || p->max_neighbors > CROWD_MAX_NEIGHBORS)
        return fail(CROWD_EINVAL, "max_neighbors must be in [0, %d]", CROWD_MAX_NEIGHBORS);
    if (!(p->robot_responsibility >= 0.f && p->robot_responsibility <= 1.f))
        return fail(CROWD_EINVAL, "robot_responsibility must be in [0, 1]");

    int64_t N = 0, S = 0;
    int max_agents = 0;
    for (int e = 0; e < n_envs; ++e) {
        if (agents_per_env[e] < 0) return fail(CROWD_EINVAL, "agents_per_env[%d] < 0", e);
        N += agents_per_env[e];
        max_agents = std::max(max_agents, (int)agents_per_env[e]);
        if (segs_per_env) {
            if (segs_per_env[e] < 0) return fail(CROWD_EINVAL, "segs_per_env[%d] < 0", e);
            S += segs_per_env[e];
        }
        if (robot_index && (robot_index[e] < -1 || robot_index[e] >= agents_per_env[e]))
            return fail(CROWD_EINVAL, "robot_index[%d] out of range", e);
    }
    if (N >= (int64_t)1 << 31 || S >= (int64_t)1 << 31) return fail(CROWD_EINVAL, "too many agents or segments");
    if (N > 0 && (!radii || !max_speeds || !init_pos)) return fail(CROWD_EINVAL, "agent arrays are null");
    if (S > 0 && !segments) return fail(CROWD_EINVAL, "segments is null");
    if (!finite_all(init_pos, (size_t)N * 2)) return fail(CROWD_EINVAL, "init_pos holds NaN/Inf");
    for (int64_t i = 0; i < N; ++i) {
        if (!(radii[i] > 0.f) || !std::isfinite(radii[i])) return fail(CROWD_EINVAL, "radius[%lld] must be > 0", (long long)i);
        if (!(max_speeds[i] >= 0.f) || !std::isfinite(max_speeds[i]))
            return fail(CROWD_EINVAL, "max_speed[%lld] must be >= 0", (long long)i);
        if (pref_speeds && (!(pref_speeds[i] >= 0.f) || !std::isfinite(pref_speeds[i])))
            return fail(CROWD_EINVAL, "pref_speed[%lld] must be >= 0", (long long)i);
    }
    if (!finite_all(segments, (size_t)S * 4)) return fail(CROWD_EINVAL, "segments hold NaN/Inf");
    for (int64_t s = 0; s < S; ++s) {
        const float* q = segments + 4 * s;
        if (q[0] == q[2] && q[1] == q[3]) return fail(CROWD_EINVAL, "segment %lld has zero length", (long long)s);
    }

    crowd_ctx* h = new (std::nothrow) crowd_ctx();
    if (!h) return fail(CROWD_ENOMEM, "host allocation failed");
    auto bail = [&](crowd_status st) {
        delete h;
        return st;
    };
    CUDA_TRY(cudaGetDevice(&h->device), "cudaGetDevice");
    h->stream = (cudaStream_t)cuda_stream;
    h->E = n_envs;
    h->N = N;
    h->S = S;
    h->max_agents = max_agents;
    h->p = *p;

    std::vector<int> env_start(n_envs + 1, 0), seg_start(n_envs + 1, 0), robot(n_envs, -1);
    for (int e = 0; e < n_envs; ++e) {
        env_start[e + 1] = env_start[e] + agents_per_env[e];
        seg_start[e + 1] = seg_start[e] + (segs_per_env ? segs_per_env[e] : 0);
        if (robot_index) robot[e] = robot_index[e];
    }
    // environments that fit one CTA go to the resident kernel (largest first,
    // so that its queue balances uneven batches); the others to the tiled path
    const bool force_tiled = (p->flags & CROWD_FLAG_FORCE_TILED) != 0;
    std::vector<int> order, tiled;
    h->h_env_start = env_start;
    h->h_env_tiled.assign(n_envs, 0);
    for (int e = 0; e < n_envs; ++e) {
        if (!force_tiled && agents_per_env[e] <= kResidentMaxAgents) order.push_back(e);
        else {
            tiled.push_back(e);
            h->h_env_tiled[e] = 1;
        }
    }
    std::stable_sort(order.begin(), order.end(),
                     [&](int a, int b) { return agents_per_env[a] > agents_per_env[b]; });
    for (int e : order) {
        h->res_max_agents = std::max(h->res_max_agents, (int)agents_per_env[e]);
        const bool has_robot = robot[e] >= 0 && robot[e] < agents_per_env[e];
        h->res_max_work = std::max(h->res_max_work, (int)agents_per_env[e] - (has_robot ? 1 : 0));
    }
    h->n_res = (int)order.size();
    h->h_res_envs = order;
    h->n_tiled = (int)tiled.size();
    std::vector<int> seg_cell_start, seg_cell_ids;
    int total_cells = 0;
    // Cells of R / 2 cut the instructions of the tiled update by about 14 %
    // but lengthen each agent's scan (five cell rows instead of three): they
    // pay when the tiled agents fill the GPU several times over (16 x 20,000
    // agents: 261 -> 272 M agent-steps/s) and cost a lone 20,000-agent
    // environment, one partial wave of tiles, 25 % (132 -> 164 us a step).
    // The neighbour lists, hence the results, are the same either way.
    long long tiled_agents = 0;
    for (int e : tiled) tiled_agents += agents_per_env[e];
    int sm_count = 0;
    if (!tiled.empty()) {
        const cudaError_t ea = cudaDeviceGetAttribute(&sm_count, cudaDevAttrMultiProcessorCount, h->device);
        if (ea != cudaSuccess) {
            cuda_fail(ea, "device attributes");
            return bail(CROWD_ECUDA);
        }
    }
    const bool fine_cells = tiled_agents >= (long long)kFineCellRounds * sm_count * kTiledUpdateThreads;
    for (int e : tiled) {
        TiledEnv te{};
        build_tiled_env(e, env_start[e], agents_per_env[e], seg_start[e], segs_per_env ? segs_per_env[e] : 0,
                        robot[e], init_pos, radii, max_speeds, segments, *p, total_cells, fine_cells, te,
                        seg_cell_start, seg_cell_ids);
        total_cells += te.W * te.H + 1;
        h->tiled_max_agents = std::max(h->tiled_max_agents, te.n);
        h->tiled_max_tiles = std::max(h->tiled_max_tiles, ((te.W + te.tx - 1) / te.tx) * ((te.H + te.ty - 1) / te.ty));
        h->h_tenvs.push_back(te);
    }
    // work items of the persistent update: kQueueItem consecutive sorted
    // slots of one environment
    std::vector<int> item_start(1, 0);
    for (const TiledEnv& te : h->h_tenvs) item_start.push_back(item_start.back() + (te.n + kQueueItem - 1) / kQueueItem);
    h->n_items = item_start.back();
    std::vector<SegGrid> seg_grids(std::max(n_envs, 1));
    int seg_off = total_cells;
    for (int e : order) {
        seg_grids[e] = build_seg_grid(env_start[e], agents_per_env[e], seg_start[e], segs_per_env ? segs_per_env[e] : 0,
                                      radii, max_speeds, segments, p->time_horizon, p->time_horizon_obst, seg_off,
                                      seg_cell_start, seg_cell_ids);
        seg_off += seg_grids[e].W * seg_grids[e].H + 1;
    }
    if (seg_cell_ids.empty()) seg_cell_ids.push_back(0);
    if (seg_cell_start.empty()) seg_cell_start.push_back(0);
    std::vector<float4> par((size_t)N), state((size_t)N);
    std::vector<float2> goal((size_t)N);
    for (int64_t i = 0; i < N; ++i) {
        par[i] = make_float4(radii[i], max_speeds[i], pref_speeds ? pref_speeds[i] : max_speeds[i], 0.f);
        state[i] = make_float4(init_pos[2 * i], init_pos[2 * i + 1], 0.f, 0.f);
        goal[i] = make_float2(init_pos[2 * i], init_pos[2 * i + 1]);
    }

    cudaError_t e = cudaSuccess;
#define ALLOC(ptr, n)                                              \
    if ((e = dev_alloc(&h->ptr, (size_t)(n))) != cudaSuccess) {    \
        cuda_fail(e, "cudaMalloc " #ptr);                          \
        return bail(e == cudaErrorMemoryAllocation ? CROWD_ENOMEM : CROWD_ECUDA); \
    }
    ALLOC(seg_grid, n_envs);
    ALLOC(seg_cell_start, seg_cell_start.size());
    ALLOC(seg_cell_ids, seg_cell_ids.size());
    if (h->n_tiled) {
        ALLOC(tenvs, h->n_tiled);
        ALLOC(state_b, N);
        ALLOC(sorted_pv, N);
        ALLOC(key, N);
        ALLOC(rank, N);
        ALLOC(sorted_id, N);
        ALLOC(count, total_cells);
        ALLOC(start, total_cells);
        ALLOC(d_step, 1);
        ALLOC(item_start, item_start.size());
        ALLOC(tqueue, 1);
        ALLOC(item_order, std::max(h->n_items, 1));
        ALLOC(item_bucket, std::max(h->n_items, 1));
        ALLOC(sched, 1);
    }
    ALLOC(env_start, n_envs + 1);
    ALLOC(seg_start, n_envs + 1);
    ALLOC(robot_index, n_envs);
    ALLOC(order, n_envs);
    ALLOC(queue, 1);
    ALLOC(err, 1);
    ALLOC(state, N);
    ALLOC(par, N);
    ALLOC(goal, N);
    ALLOC(segs, S);
    ALLOC(reach, N);
    ALLOC(stats, n_envs);
    if (p->flags & CROWD_FLAG_EXPORT_NEIGHBORS) ALLOC(nbr, (size_t)N * std::max(1, (int)p->max_neighbors));
    if (p->flags & CROWD_FLAG_COUNT_WORK) ALLOC(work, 1);
#undef ALLOC

    struct Copy {
        void* dst;
        const void* src;
        size_t bytes;
    } copies[] = {
        {h->env_start, env_start.data(), sizeof(int) * (n_envs + 1)},
        {h->seg_start, seg_start.data(), sizeof(int) * (n_envs + 1)},
        {h->robot_index, robot.data(), sizeof(int) * n_envs},
        {h->order, order.data(), sizeof(int) * order.size()},
        {h->tenvs, h->h_tenvs.data(), sizeof(TiledEnv) * h->h_tenvs.size()},
        {h->item_start, item_start.data(), h->n_tiled ? sizeof(int) * item_start.size() : 0},
        {h->seg_cell_start, seg_cell_start.data(), sizeof(int) * seg_cell_start.size()},
        {h->seg_cell_ids, seg_cell_ids.data(), sizeof(int) * seg_cell_ids.size()},
        {h->seg_grid, seg_grids.data(), sizeof(SegGrid) * n_envs},
        {h->state, state.data(), sizeof(float4) * N},
        {h->par, par.data(), sizeof(float4) * N},
        {h->goal, goal.data(), sizeof(float2) * N},
        {h->segs, segments, sizeof(float4) * S},
    };
    for (const Copy& c : copies) {
        if (c.bytes == 0) continue;
        if ((e = cudaMemcpyAsync(c.dst, c.src, c.bytes, cudaMemcpyHostToDevice, h->stream)) != cudaSuccess) {
            cuda_fail(e, "copy inputs");
            return bail(CROWD_ECUDA);
        }
    }
    if ((e = cudaMemsetAsync(h->err, 0, sizeof(int), h->stream)) != cudaSuccess ||
        (e = cudaMemsetAsync(h->reach, 0xff, sizeof(int) * std::max<int64_t>(N, 1), h->stream)) != cudaSuccess ||
        (e = cudaMemsetAsync(h->stats, 0, sizeof(EnvStats) * std::max(n_envs, 1), h->stream)) != cudaSuccess) {
        cuda_fail(e, "initialise buffers");
        return bail(CROWD_ECUDA);
    }
    ItemSched sched0{};
    sched0.count[0] = h->n_items;  // no costs yet: every item in the first class
    if (h->sched && ((e = cudaMemsetAsync(h->item_bucket, 0, std::max(h->n_items, 1), h->stream)) != cudaSuccess ||
                     (e = cudaMemcpyAsync(h->sched, &sched0, sizeof(ItemSched), cudaMemcpyHostToDevice, h->stream)) !=
                         cudaSuccess)) {
        cuda_fail(e, "initialise the item order");
        return bail(CROWD_ECUDA);
    }
    if (h->count && (e = cudaMemsetAsync(h->count, 0, sizeof(int) * total_cells, h->stream)) != cudaSuccess) {
        cuda_fail(e, "initialise cell counts");
        return bail(CROWD_ECUDA);
    }
    if (h->n_tiled && (e = tiled_init(kHaloCap)) != cudaSuccess) {
        cuda_fail(e, "tiled kernel attributes");
        return bail(CROWD_ECUDA);
    }
    if (h->n_tiled && (e = cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking)) != cudaSuccess) {
        cuda_fail(e, "create capture stream");
        return bail(CROWD_ECUDA);
    }
    if (h->work && (e = cudaMemsetAsync(h->work, 0, sizeof(WorkCount), h->stream)) != cudaSuccess) {
        cuda_fail(e, "initialise work counters");
        return bail(CROWD_ECUDA);
    }
    if (h->nbr &&
        (e = cudaMemsetAsync(h->nbr, 0xff, sizeof(int) * (size_t)N * std::max(1, (int)p->max_neighbors),
                             h->stream)) != cudaSuccess) {
        cuda_fail(e, "initialise neighbour buffer");
        return bail(CROWD_ECUDA);
    }

    // launch shape: one CTA per environment, as many resident per SM as fit
    h->halo_cap = kHaloCap;
    int sms = 0;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device)) != cudaSuccess) {
        cuda_fail(e, "device attributes");
        return bail(CROWD_ECUDA);
    }
    h->sms = sms;
    if (h->n_tiled) {
        const int per_sm = tiled_queue_blocks_per_sm(p->max_neighbors, false);
        const int per_sm_plain = tiled_queue_blocks_per_sm(p->max_neighbors, true);
        if (per_sm < 1 || per_sm_plain < 1) {
            cuda_fail(cudaGetLastError(), "occupancy of the persistent tiled update");
            return bail(CROWD_ECUDA);
        }
        h->queue_grid = per_sm * sms;
        h->queue_grid_plain = per_sm_plain * sms;
    }
    apply_tuning(h, h->tune);

    if ((e = cudaStreamSynchronize(h->stream)) != cudaSuccess) {
        cuda_fail(e, "synchronize after create");
        return bail(CROWD_ECUDA);
    }
    *out = h;
    return CROWD_OK;
}

crowd_status crowd_set_goals(crowd_t h, const float* goals, int32_t ptr_kind) {
    crowd_status st = check_handle(h);
    if (st) return st;
    if (h->N == 0) return CROWD_OK;
    if (!goals) return fail(CROWD_EINVAL, "goals is null");
    if (ptr_kind == CROWD_HOST && !finite_all(goals, (size_t)h->N * 2)) return fail(CROWD_EINVAL, "goals hold NaN/Inf");
    drop_episodes(h);
    drop_pool(h);
    if (h->goal_q) {
        h->goal_q = 0;  // fixed goals replace a goal queue
        drop_graph(h);
    }
    return copy_in(h, h->goal, goals, sizeof(float2) * h->N, ptr_kind, "copy goals");
}

crowd_status crowd_set_goal_queue(crowd_t h, int32_t n_goals, const float* goals, int32_t cyclic, int32_t ptr_kind) {
    crowd_status st = check_handle(h);
    if (st) return st;
    if (n_goals < 1 || n_goals > CROWD_MAX_GOALS) return fail(CROWD_EINVAL, "n_goals must be in [1, %d]", CROWD_MAX_GOALS);
    if (ptr_kind != CROWD_HOST && ptr_kind != CROWD_DEVICE) return fail(CROWD_EINVAL, "ptr_kind must be 0 or 1");
    if (h->N == 0) return CROWD_OK;
    if (!goals) return fail(CROWD_EINVAL, "goals is null");
    const size_t count = (size_t)h->N * n_goals;
    if (ptr_kind == CROWD_HOST && !finite_all(goals, count * 2)) return fail(CROWD_EINVAL, "goals hold NaN/Inf");
    CUDA_TRY(cudaStreamSynchronize(h->stream), "synchronize");
    drop_episodes(h);
    drop_pool(h);
    if (h->goal_queue && h->goal_queue_cap < count) {
        cudaFree(h->goal_queue);
        h->goal_queue = nullptr;
        h->goal_queue_cap = 0;
    }
    if (!h->goal_queue) {
        CUDA_TRY(dev_alloc(&h->goal_queue, count), "allocate goal queue");
        h->goal_queue_cap = count;
    }
    if (!h->goal_idx) CUDA_TRY(dev_alloc(&h->goal_idx, (size_t)h->N), "allocate goal counters");
    h->goal_q = 0;  // until the copies below succeed
    st = copy_in(h, h->goal_queue, goals, sizeof(float2) * count, ptr_kind, "copy goal queue");
    if (st) return st;
    CUDA_TRY(cudaMemsetAsync(h->goal_idx, 0, sizeof(int) * h->N, h->stream), "clear goal counters");
    // the current goal of every agent becomes the first of its queue
    CUDA_TRY(cudaMemcpy2DAsync(h->goal, sizeof(float2), h->goal_queue, sizeof(float2) * n_goals, sizeof(float2),
                               (size_t)h->N, cudaMemcpyDeviceToDevice, h->stream),
             "set first goals");
    h->goal_q = n_goals;
    h->goal_cyclic = cyclic ? 1 : 0;
    drop_graph(h);
    return CROWD_OK;
}

crowd_status crowd_set_goal_pool(crowd_t h, const int32_t* pool_start, const float* points, uint64_t seed) {
    crowd_status st = check_handle(h);
    if (st) return st;
    if (pool_start) {
        if (pool_start[0] != 0) return fail(CROWD_EINVAL, "pool_start[0] must be 0");
        for (int e = 0; e < h->E; ++e)
            if (pool_start[e + 1] < pool_start[e]) return fail(CROWD_EINVAL, "pool_start must not decrease");
        if (pool_start[h->E] > 0 && !points) return fail(CROWD_EINVAL, "points is null");
        if (pool_start[h->E] > 0 && !finite_all(points, (size_t)pool_start[h->E] * 2))
            return fail(CROWD_EINVAL, "pool points hold NaN/Inf");
    }
    CUDA_TRY(cudaStreamSynchronize(h->stream), "synchronize");
    drop_episodes(h);  // their snapshot holds the counters of the goals replaced here
    drop_pool(h);
    if (!pool_start || h->N == 0) return CROWD_OK;
    if (h->goal_q) {
        h->goal_q = 0;  // a pool replaces a goal queue
        drop_graph(h);
    }
    const int P = pool_start[h->E];
    CUDA_TRY(dev_alloc(&h->pool_start, (size_t)h->E + 1), "allocate goal pool");
    cudaError_t e = dev_alloc(&h->pool, (size_t)std::max(P, 1));
    if (e == cudaSuccess) e = cudaMemcpy(h->pool_start, pool_start, sizeof(int) * (h->E + 1), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && P) e = cudaMemcpy(h->pool, points, sizeof(float2) * P, cudaMemcpyHostToDevice);
    if (e == cudaSuccess && !h->goal_idx) e = dev_alloc(&h->goal_idx, (size_t)h->N);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->goal_idx, 0, sizeof(int) * h->N, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) {
        drop_pool(h);
        return cuda_fail(e, "set goal pool");
    }
    h->pool_seed = seed;
    drop_graph(h);
    return CROWD_OK;
}

namespace {
// A car's agent carries w = 1 and a negative preferred speed (the kernels
// test the sign of the value they hold anyway); `saved` keeps the speed.
__global__ void mark_vehicles(float4* par, const int* agent, int n, int mark, float* saved) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    float4& p = par[agent[k]];
    if (mark) {
        saved[k] = p.z;
        p.z = -1.f;
        p.w = 1.f;
    } else {
        p.z = saved[k];
        p.w = 0.f;
    }
}
}  // namespace

crowd_status crowd_set_vehicles(crowd_t h, int32_t n_lanes, const int32_t* lane_start, const float* points,
                                int32_t n_vehicles, const int32_t* agent, const int32_t* lane, const float* s,
                                const float* v, const float* params, float half_width, float lookahead) {
    crowd_status st = check_handle(h);
    if (st) return st;
    if (n_vehicles < 0 || n_lanes < 0) return fail(CROWD_EINVAL, "n_vehicles and n_lanes must be >= 0");
    if (n_vehicles > 0 && (!lane_start || !points || !agent || !lane || !s || !v || !params || n_lanes < 1))
        return fail(CROWD_EINVAL, "vehicle arrays are null or no lane is given");
    if (!(half_width >= 0.f) || !(lookahead > 0.f) || !std::isfinite(half_width) || !std::isfinite(lookahead))
        return fail(CROWD_EINVAL, "half_width >= 0 and lookahead > 0 (finite) required");
    // validate on the host
    std::vector<double> cum;
    std::vector<float> cumf;
    int P = 0;
    if (n_vehicles > 0) {
        if (lane_start[0] != 0) return fail(CROWD_EINVAL, "lane_start[0] must be 0");
        for (int l = 0; l < n_lanes; ++l)
            if (lane_start[l + 1] - lane_start[l] < 2) return fail(CROWD_EINVAL, "lane %d has fewer than 2 points", l);
        P = lane_start[n_lanes];
        if (!finite_all(points, (size_t)P * 2)) return fail(CROWD_EINVAL, "lane points hold NaN/Inf");
        for (int l = 0; l < n_lanes; ++l) {
            const int p0 = lane_start[l], m = lane_start[l + 1] - p0;
            double c = 0.0;
            cum.push_back(0.0);
            for (int k = 0; k < m; ++k) {
                const int q = p0 + (k + 1 == m ? 0 : k + 1);
                const double ex = (double)points[2 * q] - points[2 * (p0 + k)];
                const double ey = (double)points[2 * q + 1] - points[2 * (p0 + k) + 1];
                const double ln = std::sqrt(ex * ex + ey * ey);
                if (!(ln > 0.0)) return fail(CROWD_EINVAL, "lane %d has a zero-length segment", l);
                c += ln;
                cum.push_back(c);
            }
        }
        std::vector<int> per_env(h->E, 0);
        for (int k = 0; k < n_vehicles; ++k) {
            if (agent[k] < 0 || agent[k] >= h->N) return fail(CROWD_EINVAL, "vehicle %d: agent out of range", k);
            if (k > 0 && agent[k] <= agent[k - 1]) return fail(CROWD_EINVAL, "vehicle agents must ascend");
            if (lane[k] < 0 || lane[k] >= n_lanes) return fail(CROWD_EINVAL, "vehicle %d: lane out of range", k);
            const int e = (int)(std::upper_bound(h->h_env_start.begin(), h->h_env_start.end(), agent[k]) -
                                h->h_env_start.begin()) - 1;
            if (++per_env[e] > CROWD_MAX_VEHICLES_PER_ENV)
                return fail(CROWD_EINVAL, "more than %d vehicles in environment %d", CROWD_MAX_VEHICLES_PER_ENV, e);
            int32_t robot = -1;
            CUDA_TRY(cudaMemcpy(&robot, h->robot_index + e, sizeof(int32_t), cudaMemcpyDeviceToHost), "read robot");
            if (agent[k] - h->h_env_start[e] == robot) return fail(CROWD_EINVAL, "vehicle %d is the robot slot", k);
            const double L = cum[lane_start[lane[k] + 1] + lane[k]];
            const float* pr = params + 6 * k;
            if (!(s[k] >= 0.f) || !(s[k] < L) || !(v[k] >= 0.f) || !std::isfinite(v[k]))
                return fail(CROWD_EINVAL, "vehicle %d: s in [0, lane length) and v >= 0 required", k);
            for (int q = 0; q < 6; ++q)
                if (!(pr[q] > 0.f) || !std::isfinite(pr[q]))
                    return fail(CROWD_EINVAL, "vehicle %d: parameters must be finite and > 0", k);
        }
        cumf.assign(cum.begin(), cum.end());
    }
    CUDA_TRY(cudaStreamSynchronize(h->stream), "synchronize");
    drop_episodes(h);
    // unmark the old cars, release the old arrays
    if (h->n_veh > 0) {
        mark_vehicles<<<(h->n_veh + 255) / 256, 256, 0, h->stream>>>(h->par, h->veh_agent, h->n_veh, 0, h->veh_pref);
        CUDA_TRY(cudaGetLastError(), "unmark vehicles");
        CUDA_TRY(cudaStreamSynchronize(h->stream), "synchronize");
    }
    void** olds[] = {(void**)&h->veh_start, (void**)&h->veh_agent, (void**)&h->veh_lane, (void**)&h->veh_s,
                     (void**)&h->veh_v, (void**)&h->veh_par_a, (void**)&h->veh_par_b, (void**)&h->lane_pts,
                     (void**)&h->lane_start, (void**)&h->lane_cum, (void**)&h->veh_pref};
    for (void** q : olds)
        if (*q) {
            cudaFree(*q);
            *q = nullptr;
        }
    h->n_veh = 0;
    h->tiled_cars = false;
    drop_graph(h);  // cached tiled graphs hold the car arrays
    if (n_vehicles == 0) return CROWD_OK;
    std::vector<int> start(h->E + 1, 0);
    for (int k = 0; k < n_vehicles; ++k) {
        const int e = (int)(std::upper_bound(h->h_env_start.begin(), h->h_env_start.end(), agent[k]) -
                            h->h_env_start.begin()) - 1;
        ++start[e + 1];
    }
    for (int e = 0; e < h->E; ++e) start[e + 1] += start[e];
    std::vector<float4> pa(n_vehicles);
    std::vector<float2> pb(n_vehicles);
    for (int k = 0; k < n_vehicles; ++k) {
        const float* pr = params + 6 * k;
        pa[k] = make_float4(pr[0], pr[1], pr[2], pr[3]);
        pb[k] = make_float2(pr[4], pr[5]);
    }
    CUDA_TRY(dev_alloc(&h->veh_start, (size_t)h->E + 1), "allocate vehicles");
    CUDA_TRY(dev_alloc(&h->veh_agent, (size_t)n_vehicles), "allocate vehicles");
    CUDA_TRY(dev_alloc(&h->veh_lane, (size_t)n_vehicles), "allocate vehicles");
    CUDA_TRY(dev_alloc(&h->veh_s, (size_t)n_vehicles), "allocate vehicles");
    CUDA_TRY(dev_alloc(&h->veh_v, (size_t)n_vehicles), "allocate vehicles");
    CUDA_TRY(dev_alloc(&h->veh_par_a, (size_t)n_vehicles), "allocate vehicles");
    CUDA_TRY(dev_alloc(&h->veh_par_b, (size_t)n_vehicles), "allocate vehicles");
    CUDA_TRY(dev_alloc(&h->lane_pts, (size_t)P), "allocate lanes");
    CUDA_TRY(dev_alloc(&h->lane_start, (size_t)n_lanes + 1), "allocate lanes");
    CUDA_TRY(dev_alloc(&h->lane_cum, cumf.size()), "allocate lanes");
    CUDA_TRY(dev_alloc(&h->veh_pref, (size_t)n_vehicles), "allocate vehicles");
    struct Copy {
        void* dst;
        const void* src;
        size_t bytes;
    } copies[] = {{h->veh_start, start.data(), sizeof(int) * (h->E + 1)},
                  {h->veh_agent, agent, sizeof(int) * n_vehicles},
                  {h->veh_lane, lane, sizeof(int) * n_vehicles},
                  {h->veh_s, s, sizeof(float) * n_vehicles},
                  {h->veh_v, v, sizeof(float) * n_vehicles},
                  {h->veh_par_a, pa.data(), sizeof(float4) * n_vehicles},
                  {h->veh_par_b, pb.data(), sizeof(float2) * n_vehicles},
                  {h->lane_pts, points, sizeof(float2) * P},
                  {h->lane_start, lane_start, sizeof(int) * (n_lanes + 1)},
                  {h->lane_cum, cumf.data(), sizeof(float) * cumf.size()}};
    for (const Copy& c : copies) CUDA_TRY(cudaMemcpy(c.dst, c.src, c.bytes, cudaMemcpyHostToDevice), "copy vehicles");
    mark_vehicles<<<(n_vehicles + 255) / 256, 256, 0, h->stream>>>(h->par, h->veh_agent, n_vehicles, 1, h->veh_pref);
    CUDA_TRY(cudaGetLastError(), "mark vehicles");
    CUDA_TRY(cudaStreamSynchronize(h->stream), "synchronize");
    h->n_veh = n_vehicles;
    h->veh_half_width = half_width;
    h->veh_lookahead = lookahead;
    for (int e = 0; e < h->E; ++e)
        if (h->h_env_tiled[e] && start[e + 1] > start[e]) h->tiled_cars = true;
    return CROWD_OK;
}

crowd_status crowd_vehicle_state(crowd_t h, int32_t write, float* s, float* v) {
    crowd_status st = check_handle(h);
    if (st) return st;
    if (h->n_veh == 0) return CROWD_OK;
    if (!s || !v) return fail(CROWD_EINVAL, "s and v must not be null");
    if (write) {
        for (int k = 0; k < h->n_veh; ++k)
            if (!(s[k] >= 0.f) || !(v[k] >= 0.f) || !std::isfinite(s[k]) || !std::isfinite(v[k]))
                return fail(CROWD_EINVAL, "vehicle %d: s and v must be finite and >= 0", k);
        CUDA_TRY(cudaStreamSynchronize(h->stream), "synchronize");
        CUDA_TRY(cudaMemcpy(h->veh_s, s, sizeof(float) * h->n_veh, cudaMemcpyHostToDevice), "copy vehicle s");
        CUDA_TRY(cudaMemcpy(h->veh_v, v, sizeof(float) * h->n_veh, cudaMemcpyHostToDevice), "copy vehicle v");
    } else {
        CUDA_TRY(cudaStreamSynchronize(h->stream), "synchronize");
        CUDA_TRY(cudaMemcpy(s, h->veh_s, sizeof(float) * h->n_veh, cudaMemcpyDeviceToHost), "copy vehicle s");
        CUDA_TRY(cudaMemcpy(v, h->veh_v, sizeof(float) * h->n_veh, cudaMemcpyDeviceToHost), "copy vehicle v");
    }
    return CROWD_OK;
}

crowd_status crowd_read_goal_index(crowd_t h, int32_t* out) {
    crowd_status st = check_handle(h);
    if (st) return st;
    if (!out) return fail(CROWD_EINVAL, "out is null");
    if (h->N == 0) return CROWD_OK;
    if (!h->goal_idx || !goals_move(h)) {
        std::fill(out, out + h->N, 0);
        return CROWD_OK;
    }
    CUDA_TRY(cudaMemcpyAsync(out, h->goal_idx, sizeof(int) * h->N, cudaMemcpyDeviceToHost, h->stream), "copy goal counters");
    CUDA_TRY(cudaStreamSynchronize(h->stream), "synchronize");
    return CROWD_OK;
}

crowd_status crowd_set_episodes(crowd_t h, const int32_t* steps, const float* init_state, int32_t ptr_kind) {
    const TraceRange trace("crowd_set_episodes");
    crowd_status st = check_handle(h);
    if (st) return st;
    if (ptr_kind != CROWD_HOST && ptr_kind != CROWD_DEVICE) return fail(CROWD_EINVAL, "ptr_kind must be 0 or 1");
    if (steps)
        for (int e = 0; e < h->E; ++e)
            if (steps[e] < 0) return fail(CROWD_EINVAL, "steps[%d] must be >= 0", e);
    if (init_state && ptr_kind == CROWD_HOST && !finite_all(init_state, (size_t)h->N * 4))
        return fail(CROWD_EINVAL, "init_state holds NaN/Inf");
    CUDA_TRY(cudaStreamSynchronize(h->stream), "synchronize");
    drop_episodes(h);
    if (!steps || h->N == 0) return CROWD_OK;
    // the episodes exist once every snapshot below is in place
    auto undo = [&](crowd_status s) {
        h->h_ep_steps.assign(1, 0);
        drop_episodes(h);
        return s;
    };
    cudaError_t e = dev_alloc(&h->ep_steps, (size_t)h->E);
    if (e == cudaSuccess) e = dev_alloc(&h->ep_state, (size_t)h->N);
    if (e == cudaSuccess) e = dev_alloc(&h->ep_goal, (size_t)h->N);
    if (e == cudaSuccess && goals_move(h)) e = dev_alloc(&h->ep_gidx, (size_t)h->N);
    if (e == cudaSuccess && h->n_veh) e = dev_alloc(&h->ep_veh, 2 * (size_t)h->n_veh);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(h->ep_steps, steps, sizeof(int) * h->E, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess && !init_state)
        e = cudaMemcpyAsync(h->ep_state, h->state, sizeof(float4) * h->N, cudaMemcpyDeviceToDevice, h->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(h->ep_goal, h->goal, sizeof(float2) * h->N, cudaMemcpyDeviceToDevice, h->stream);
    if (e == cudaSuccess && goals_move(h))
        e = cudaMemcpyAsync(h->ep_gidx, h->goal_idx, sizeof(int) * h->N, cudaMemcpyDeviceToDevice, h->stream);
    if (e == cudaSuccess && h->n_veh)
        e = cudaMemcpyAsync(h->ep_veh, h->veh_s, sizeof(float) * h->n_veh, cudaMemcpyDeviceToDevice, h->stream);
    if (e == cudaSuccess && h->n_veh)
        e = cudaMemcpyAsync(h->ep_veh + h->n_veh, h->veh_v, sizeof(float) * h->n_veh, cudaMemcpyDeviceToDevice,
                            h->stream);
    if (e != cudaSuccess) return undo(cuda_fail(e, "set episodes"));
    if (init_state) {
        st = copy_in(h, h->ep_state, init_state, sizeof(float4) * h->N, ptr_kind, "copy episode state");
        if (st) return undo(st);
    }
    e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return undo(cuda_fail(e, "set episodes"));
    h->h_ep_steps.assign(steps, steps + h->E);
    h->ep_origin = h->step_index;
    drop_graph(h);
    return CROWD_OK;
}

crowd_status crowd_restart_envs(crowd_t h, const uint8_t* mask) {
    const TraceRange trace("crowd_restart_envs");
    crowd_status st = check_handle(h);
    if (st) return st;
    if (!mask) return fail(CROWD_EINVAL, "mask is null");
    if (h->h_ep_steps.empty()) return fail(CROWD_ESTATE, "no episode snapshot: call crowd_set_episodes first");
    if (h->N == 0) return CROWD_OK;
    if (!h->ep_mask) CUDA_TRY(dev_alloc(&h->ep_mask, (size_t)h->E), "allocate restart mask");
    CUDA_TRY(cudaMemcpyAsync(h->ep_mask, mask, (size_t)h->E, cudaMemcpyHostToDevice, h->stream), "copy restart mask");
    const VehicleArgs veh{h->n_veh, h->veh_start, h->veh_agent, h->veh_lane, h->veh_s, h->veh_v, h->veh_par_a,
                          h->veh_par_b, h->lane_pts, h->lane_start, h->lane_cum, h->veh_half_width, h->veh_lookahead};
    const int span = std::max(h->max_agents, CROWD_MAX_VEHICLES_PER_ENV);
    restart_masked_envs<<<dim3(h->E, (span + 255) / 256), 256, 0, h->stream>>>(episode_args(h), h->ep_mask, h->env_start,
                                                                              veh, h->state, h->goal, h->goal_idx);
    CUDA_TRY(cudaGetLastError(), "restart environments");
    // the host buffer may be reused once the copy has been made
    CUDA_TRY(cudaStreamSynchronize(h->stream), "synchronize");
    return CROWD_OK;
}

crowd_status crowd_set_state(crowd_t h, const float* state, int32_t ptr_kind) {
    crowd_status st = check_handle(h);
    if (st) return st;
    if (h->N == 0) return CROWD_OK;
    if (!state) return fail(CROWD_EINVAL, "state is null");
    if (ptr_kind == CROWD_HOST && !finite_all(state, (size_t)h->N * 4)) return fail(CROWD_EINVAL, "state holds NaN/Inf");
    return copy_in(h, h->state, state, sizeof(float4) * h->N, ptr_kind, "copy state");
}

crowd_status crowd_step(crowd_t h, float dt, const float* robot_vel, int32_t ptr_kind, int32_t n_steps) {
    const TraceRange trace("crowd_step");
    crowd_status st = check_handle(h);
    if (st) return st;
    if (!(dt > 0.f) || !std::isfinite(dt)) return fail(CROWD_EINVAL, "dt must be finite and > 0");
    if (n_steps < 1) return fail(CROWD_EINVAL, "n_steps must be >= 1");
    if (ptr_kind != CROWD_HOST && ptr_kind != CROWD_DEVICE) return fail(CROWD_EINVAL, "ptr_kind must be 0 or 1");
    if (h->E == 0) return CROWD_OK;
    const float2* rv = nullptr;
    if (robot_vel) {
        const size_t count = (size_t)n_steps * h->E;
        if (ptr_kind == CROWD_HOST) {
            if (!finite_all(robot_vel, count * 2)) return fail(CROWD_EINVAL, "robot_vel holds NaN/Inf");
            if (count > h->robot_vel_cap) {
                if (h->robot_vel) cudaFree(h->robot_vel);
                h->robot_vel = nullptr;
                h->robot_vel_cap = 0;
                CUDA_TRY(dev_alloc(&h->robot_vel, count), "cudaMalloc robot_vel");
                h->robot_vel_cap = count;
            }
            CUDA_TRY(cudaMemcpyAsync(h->robot_vel, robot_vel, sizeof(float2) * count, cudaMemcpyHostToDevice,
                                     h->stream),
                     "copy robot_vel");
            rv = h->robot_vel;
        } else {
            rv = (const float2*)robot_vel;
        }
    }
    const bool stats = (h->p.flags & CROWD_FLAG_STATS) != 0;
    const float tau_o = h->p.time_horizon_obst > 0.f ? h->p.time_horizon_obst : h->p.time_horizon;
    if (h->n_res) {
        const TraceRange stage("crowd_step/resident");
        st = resident_steps(h, dt, rv, n_steps, stats, tau_o, h->stream);
        if (st) return st;
    }
    if (h->n_tiled) {
        const TraceRange stage("crowd_step/tiled");
        st = tiled_steps(h, dt, rv, n_steps, stats, tau_o);
        if (st) return st;
    }
    h->step_index += n_steps;
    return CROWD_OK;
}

crowd_status crowd_read_state(crowd_t h, float* out, int32_t ptr_kind) {
    const TraceRange trace("crowd_read_state");
    crowd_status st = check_handle(h);
    if (st) return st;
    if (!out && h->N) return fail(CROWD_EINVAL, "out is null");
    if (ptr_kind != CROWD_HOST && ptr_kind != CROWD_DEVICE) return fail(CROWD_EINVAL, "ptr_kind must be 0 or 1");
    if (h->N)
        CUDA_TRY(cudaMemcpyAsync(out, h->state, sizeof(float4) * h->N,
                                 ptr_kind == CROWD_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice,
                                 h->stream),
                 "copy state out");
    return read_err_word(h);
}

crowd_status crowd_read_neighbors(crowd_t h, int32_t* out, int32_t ptr_kind) {
    crowd_status st = check_handle(h);
    if (st) return st;
    if (!h->nbr) return fail(CROWD_ESTATE, "created without CROWD_FLAG_EXPORT_NEIGHBORS");
    if (!out && h->N) return fail(CROWD_EINVAL, "out is null");
    if (ptr_kind != CROWD_HOST && ptr_kind != CROWD_DEVICE) return fail(CROWD_EINVAL, "ptr_kind must be 0 or 1");
    const size_t bytes = sizeof(int) * (size_t)h->N * h->p.max_neighbors;
    if (bytes)
        CUDA_TRY(cudaMemcpyAsync(out, h->nbr, bytes,
                                 ptr_kind == CROWD_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice,
                                 h->stream),
                 "copy neighbours out");
    return read_err_word(h);
}

crowd_status crowd_read_stats(crowd_t h, crowd_env_stats* env_stats, int32_t* reach_step) {
    crowd_status st = check_handle(h);
    if (st) return st;
    std::vector<EnvStats> tmp(std::max(h->E, 1));
    if (env_stats && h->E)
        CUDA_TRY(cudaMemcpyAsync(tmp.data(), h->stats, sizeof(EnvStats) * h->E, cudaMemcpyDeviceToHost, h->stream),
                 "copy stats out");
    if (reach_step && h->N)
        CUDA_TRY(cudaMemcpyAsync(reach_step, h->reach, sizeof(int) * h->N, cudaMemcpyDeviceToHost, h->stream),
                 "copy reach out");
    st = read_err_word(h);
    if (env_stats)
        for (int e = 0; e < h->E; ++e) {
            env_stats[e].agent_collisions = (int64_t)tmp[e].agent_collisions;
            env_stats[e].segment_collisions = (int64_t)tmp[e].segment_collisions;
            env_stats[e].speed_sum = tmp[e].speed_sum;
            env_stats[e].steps = (int64_t)tmp[e].steps;
        }
    return st;
}

crowd_status crowd_read_launches(crowd_t h, int64_t* out) {
    crowd_status st = check_handle(h);
    if (st) return st;
    if (!out) return fail(CROWD_EINVAL, "out is null");
    *out = h->kernel_launches;
    return CROWD_OK;
}

crowd_status crowd_read_work(crowd_t h, crowd_work* out) {
    crowd_status st = check_handle(h);
    if (st) return st;
    if (!h->work) return fail(CROWD_ESTATE, "created without CROWD_FLAG_COUNT_WORK");
    if (!out) return fail(CROWD_EINVAL, "out is null");
    static_assert(sizeof(WorkCount) == sizeof(crowd_work), "work counter layout");
    CUDA_TRY(cudaMemcpyAsync(out, h->work, sizeof(WorkCount), cudaMemcpyDeviceToHost, h->stream), "copy work out");
    return read_err_word(h);
}

crowd_status crowd_get_tuning(crowd_t h, crowd_tuning* out) {
    crowd_status st = check_handle(h);
    if (st) return st;
    if (!out) return fail(CROWD_EINVAL, "out is null");
    out->block_threads = h->block;
    out->coop_fallback = h->tune.coop_fallback;
    out->cell_split = h->tune.cell_split;
    out->lanes_per_agent = h->tune.lanes;
    out->agent_order = h->tune.order;
    out->tiled_queue = h->tune.tiled_queue;
    return CROWD_OK;
}

crowd_status crowd_set_tuning(crowd_t h, const crowd_tuning* t) {
    crowd_status st = check_handle(h);
    if (st) return st;
    if (!t) return fail(CROWD_EINVAL, "tuning is null");
    if (t->block_threads != 0 && (t->block_threads < 32 || t->block_threads > 512 || t->block_threads % 32))
        return fail(CROWD_EINVAL, "block_threads must be 0 or a multiple of 32 in [32, 512]");
    if (t->cell_split < 1 || t->cell_split > 3) return fail(CROWD_EINVAL, "cell_split must be 1, 2 or 3");
    const int lanes = t->lanes_per_agent == 0 ? 1 : t->lanes_per_agent;
    if (lanes != 1 && lanes != 2 && lanes != 4 && lanes != 8)
        return fail(CROWD_EINVAL, "lanes_per_agent must be 1, 2, 4 or 8");
    if (t->coop_fallback < 0 || t->coop_fallback > 2) return fail(CROWD_EINVAL, "coop_fallback must be 0, 1 or 2");
    if (t->agent_order != 0 && t->agent_order != 1) return fail(CROWD_EINVAL, "agent_order must be 0 or 1");
    if (t->tiled_queue != 0 && t->tiled_queue != 1) return fail(CROWD_EINVAL, "tiled_queue must be 0 or 1");
    apply_tuning(h, Tuning{t->block_threads, t->coop_fallback, t->cell_split, lanes, t->agent_order, t->tiled_queue});
    return CROWD_OK;
}

crowd_status crowd_autotune(crowd_t h, float dt, int32_t n_steps, crowd_tuning* chosen) {
    const TraceRange trace("crowd_autotune");
    crowd_status st = check_handle(h);
    if (st) return st;
    if (!(dt > 0.f) || !std::isfinite(dt) || n_steps < 1) return fail(CROWD_EINVAL, "dt > 0 and n_steps >= 1 required");
    if ((h->n_res || h->n_tiled) && h->N) {
        // save everything a trial step touches, time each candidate, restore
        float4* saved = nullptr;
        EnvStats* saved_stats = nullptr;
        int* saved_reach = nullptr;
        float2* saved_goal = nullptr;  // with a goal queue, trials move goals on
        int* saved_gidx = nullptr;
        float* saved_veh = nullptr;    // with vehicles, trials move the cars: [s | v]
        WorkCount saved_work{};
        CUDA_TRY(dev_alloc(&saved, h->N), "autotune scratch");
        cudaError_t e = dev_alloc(&saved_stats, h->E);
        if (e == cudaSuccess) e = dev_alloc(&saved_reach, h->N);
        if (e == cudaSuccess && goals_move(h)) e = dev_alloc(&saved_goal, h->N);
        if (e == cudaSuccess && goals_move(h)) e = dev_alloc(&saved_gidx, h->N);
        if (e == cudaSuccess && goals_move(h))
            e = cudaMemcpyAsync(saved_goal, h->goal, sizeof(float2) * h->N, cudaMemcpyDeviceToDevice, h->stream);
        if (e == cudaSuccess && goals_move(h))
            e = cudaMemcpyAsync(saved_gidx, h->goal_idx, sizeof(int) * h->N, cudaMemcpyDeviceToDevice, h->stream);
        if (e == cudaSuccess && h->n_veh) e = dev_alloc(&saved_veh, 2 * (size_t)h->n_veh);
        if (e == cudaSuccess && h->n_veh)
            e = cudaMemcpyAsync(saved_veh, h->veh_s, sizeof(float) * h->n_veh, cudaMemcpyDeviceToDevice, h->stream);
        if (e == cudaSuccess && h->n_veh)
            e = cudaMemcpyAsync(saved_veh + h->n_veh, h->veh_v, sizeof(float) * h->n_veh, cudaMemcpyDeviceToDevice,
                                h->stream);
        auto restore_start = [&]() {
            cudaError_t r = cudaMemcpyAsync(h->state, saved, sizeof(float4) * h->N, cudaMemcpyDeviceToDevice, h->stream);
            if (r == cudaSuccess && goals_move(h))
                r = cudaMemcpyAsync(h->goal, saved_goal, sizeof(float2) * h->N, cudaMemcpyDeviceToDevice, h->stream);
            if (r == cudaSuccess && goals_move(h))
                r = cudaMemcpyAsync(h->goal_idx, saved_gidx, sizeof(int) * h->N, cudaMemcpyDeviceToDevice, h->stream);
            if (r == cudaSuccess && h->n_veh)
                r = cudaMemcpyAsync(h->veh_s, saved_veh, sizeof(float) * h->n_veh, cudaMemcpyDeviceToDevice, h->stream);
            if (r == cudaSuccess && h->n_veh)
                r = cudaMemcpyAsync(h->veh_v, saved_veh + h->n_veh, sizeof(float) * h->n_veh,
                                    cudaMemcpyDeviceToDevice, h->stream);
            return r;
        };
        cudaEvent_t t0 = nullptr, t1 = nullptr;
        if (e == cudaSuccess) e = cudaEventCreate(&t0);
        if (e == cudaSuccess) e = cudaEventCreate(&t1);
        if (e == cudaSuccess) e = cudaMemcpyAsync(saved, h->state, sizeof(float4) * h->N, cudaMemcpyDeviceToDevice, h->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(saved_stats, h->stats, sizeof(EnvStats) * h->E, cudaMemcpyDeviceToDevice, h->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(saved_reach, h->reach, sizeof(int) * h->N, cudaMemcpyDeviceToDevice, h->stream);
        if (e == cudaSuccess && h->work)
            e = cudaMemcpyAsync(&saved_work, h->work, sizeof(WorkCount), cudaMemcpyDeviceToHost, h->stream);
        const Tuning before = h->tune;
        Tuning best = before;
        float best_ms = 1e30f;
        const float tau_o = h->p.time_horizon_obst > 0.f ? h->p.time_horizon_obst : h->p.time_horizon;
        // candidates: one lane per agent with every block size, in-place or
        // deferred one-lane fallbacks, cell splits 1-3 and both agent orders;
        // groups of 2, 4 and 8 lanes with a block of one group per agent
        // (capped at 512 threads) or 512 threads
        std::vector<Tuning> cands;
        const int blocks[] = {0, 64, 128, 256, 512};
        const int tq = before.tiled_queue;
        if (h->n_res) {
            for (int bi = 0; bi < 5; ++bi)
                for (int coop : {0, 2})
                    for (int split = 1; split <= 3; ++split)
                        for (int order = 0; order <= 1; ++order)
                            cands.push_back(Tuning{blocks[bi], coop, split, 1, order, tq});
            for (int lanes : {2, 4, 8})
                for (int split = 1; split <= 2; ++split) {
                    cands.push_back(Tuning{0, 0, split, lanes, 0, tq});
                    cands.push_back(Tuning{512, 0, split, lanes, 0, tq});
                }
        }
        // the tiled path's update kernel (persistent work queue or one CTA
        // per tile), with the resident shape as it stands
        if (h->n_tiled)
            for (int q : {0, 1}) {
                Tuning t = before;
                t.tiled_queue = q;
                cands.push_back(t);
            }
        // one timed run (after an untimed one) of a candidate from the saved start
        auto time_once = [&](const Tuning& t, float& ms) {
            apply_tuning(h, t);
            ms = 0.f;
            for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {
                e = restore_start();
                if (e != cudaSuccess) break;
                if (rep == 1) e = cudaEventRecord(t0, h->stream);
                if (e != cudaSuccess) break;
                if (h->n_res && resident_steps(h, dt, nullptr, n_steps, false, tau_o, h->stream) != CROWD_OK) {
                    e = cudaErrorLaunchFailure;
                    break;
                }
                if (h->n_tiled && tiled_steps(h, dt, nullptr, n_steps, false, tau_o) != CROWD_OK) {
                    e = cudaErrorLaunchFailure;
                    break;
                }
                if (rep == 1) {
                    e = cudaEventRecord(t1, h->stream);
                    if (e == cudaSuccess) e = cudaEventSynchronize(t1);
                    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, t0, t1);
                }
            }
        };
        // every candidate once, then the four fastest three times more each,
        // ranked by the median of their four times: a single timing is a few
        // per cent noisy, about the gap between the leading shapes
        std::vector<std::pair<float, size_t>> first;
        for (size_t ci = 0; ci < cands.size() && e == cudaSuccess; ++ci) {
            float ms = 0.f;
            time_once(cands[ci], ms);
            if (e == cudaSuccess) first.emplace_back(ms, ci);
        }
        std::sort(first.begin(), first.end());
        const size_t finalists = std::min<size_t>(4, first.size());
        for (size_t f = 0; f < finalists && e == cudaSuccess; ++f) {
            std::vector<float> times{first[f].first};
            for (int r = 0; r < 3 && e == cudaSuccess; ++r) {
                float ms = 0.f;
                time_once(cands[first[f].second], ms);
                times.push_back(ms);
            }
            if (e != cudaSuccess) break;
            std::sort(times.begin(), times.end());
            const float med = 0.5f * (times[1] + times[2]);
            if (med < best_ms) {
                best_ms = med;
                best = cands[first[f].second];
            }
        }
        if (e == cudaSuccess) e = restore_start();
        if (e == cudaSuccess) e = cudaMemcpyAsync(h->stats, saved_stats, sizeof(EnvStats) * h->E, cudaMemcpyDeviceToDevice, h->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(h->reach, saved_reach, sizeof(int) * h->N, cudaMemcpyDeviceToDevice, h->stream);
        if (e == cudaSuccess && h->work)
            e = cudaMemcpyAsync(h->work, &saved_work, sizeof(WorkCount), cudaMemcpyHostToDevice, h->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
        if (t0) cudaEventDestroy(t0);
        if (t1) cudaEventDestroy(t1);
        cudaFree(saved);
        if (saved_stats) cudaFree(saved_stats);
        if (saved_reach) cudaFree(saved_reach);
        if (saved_goal) cudaFree(saved_goal);
        if (saved_gidx) cudaFree(saved_gidx);
        if (saved_veh) cudaFree(saved_veh);
        apply_tuning(h, e == cudaSuccess ? best : before);
        if (e != cudaSuccess) return cuda_fail(e, "autotune");
    }
    if (chosen) return crowd_get_tuning(h, chosen);
    return CROWD_OK;
}

crowd_status crowd_reset_stats(crowd_t h) {
    crowd_status st = check_handle(h);
    if (st) return st;
    if (h->N) CUDA_TRY(cudaMemsetAsync(h->reach, 0xff, sizeof(int) * h->N, h->stream), "reset reach");
    if (h->E) CUDA_TRY(cudaMemsetAsync(h->stats, 0, sizeof(EnvStats) * h->E, h->stream), "reset stats");
    h->ep_origin -= h->step_index;  // the episode clock runs on
    h->step_index = 0;
    if (!h->h_ep_steps.empty()) drop_graph(h);  // cached tiled graphs hold the clock's origin
    return CROWD_OK;
}

crowd_status crowd_synchronize(crowd_t h) {
    crowd_status st = check_handle(h);
    if (st) return st;
    return read_err_word(h);
}

crowd_status crowd_destroy(crowd_t h) {
    if (!h) return CROWD_OK;
    cudaError_t e = cudaStreamSynchronize(h->stream);
    delete h;
    if (e != cudaSuccess) return cuda_fail(e, "synchronize before destroy");
    return CROWD_OK;
}

}  // extern "C"
