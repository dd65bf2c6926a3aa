// Serving loop with continuous batching: rollout requests of different sizes
// arrive over time; each is admitted into a device slot as soon as a slot and
// the memory budget allow, keeps its state resident on the device, and is
// stepped together with every other live request by the resident kernel, a
// chunk of steps per tick.  Requests that arrive while others run are
// admitted at the next tick, so their work overlaps on the device; each
// request's result depends on nothing but its own inputs (a slot is an
// environment of the batched step, and environments never interact).
//
// The paper samples many uneven scene instances per GPU and steps their
// dynamic agents together (Sec. 3.2-3.3); a request here is one such scene
// instance with its own step budget.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <new>
#include <numeric>
#include <string>
#include <vector>

#include "../../include/crowd.h"
#include "crowd_internal.h"

using namespace crowd;

namespace crowd {
crowd_status api_fail(crowd_status st, const char* fmt, ...);
}

namespace {

crowd_status sfail(crowd_status st, const char* what, cudaError_t e) {
    return api_fail(e == cudaErrorMemoryAllocation ? CROWD_ENOMEM : st, "%s: %s", what, cudaGetErrorString(e));
}

#define S_TRY(expr, what)                                      \
    do {                                                       \
        cudaError_t e_ = (expr);                               \
        if (e_ != cudaSuccess) return sfail(CROWD_ECUDA, what, e_); \
    } while (0)

bool finite_n(const float* p, size_t n) {
    for (size_t i = 0; i < n; ++i)
        if (!std::isfinite(p[i])) return false;
    return true;
}

// A request as kept on the host: inputs packed for the slot's device layout.
struct Req {
    int64_t id;
    int n, ns, steps, robot;
    size_t bytes;  // device bytes the request accounts for
    std::vector<float4> state, par;
    std::vector<float2> goal, rv;
    std::vector<float4> segs;
    SegGrid sg;
    std::vector<int> cell_start, cell_ids;  // lists relative to the slot's own id region
    std::vector<float> result;
    int status = CROWD_REQ_QUEUED;
    int slot = -1;
    int done = 0;  // steps run
};

}  // namespace

struct crowd_server_ctx {
    crowd_params p{};
    float dt = 0.f;
    crowd_server_config cfg{};
    cudaStream_t stream = nullptr;
    int sms = 0;
    int cells_stride = 0, ids_stride = 0;
    size_t bytes_in_use = 0;
    int64_t next_id = 1;
    bool broken = false;

    // device slot arena (slot k owns [k * stride, (k + 1) * stride) of each array)
    float4* state = nullptr;
    float4* par = nullptr;
    float2* goal = nullptr;
    float2* rv = nullptr;
    float4* segs = nullptr;
    int* cell_start = nullptr;
    int* cell_ids = nullptr;
    SegGrid* sg = nullptr;
    int* env_start = nullptr;   // k * max_agents
    int* seg_start = nullptr;   // k * max_segments
    int* env_count = nullptr;
    int* seg_count = nullptr;
    int* robot = nullptr;
    int* reach = nullptr;
    EnvStats* stats = nullptr;
    int* err = nullptr;
    int* queue = nullptr;
    // per-tick arrays (device) and their pinned host mirrors
    int* order = nullptr;
    int* env_steps = nullptr;
    int* env_step0 = nullptr;
    int* h_tick = nullptr;  // pinned: order | env_steps | env_step0
    float4* h_result = nullptr;  // pinned: max_slots * max_agents
    cudaEvent_t tick_done = nullptr;
    bool tick_in_flight = false;

    std::deque<int64_t> waiting;
    std::map<int64_t, Req> reqs;
    std::vector<int64_t> slot_req;  // request in each slot (0: free)
    std::vector<int> finishing;     // slots whose request ends with the tick in flight
    std::vector<int64_t> finished;  // requests completed and not yet reported by crowd_server_finished

    ~crowd_server_ctx() {
        if (tick_done) cudaEventDestroy(tick_done);
        void* d[] = {state, par, goal, rv, segs, cell_start, cell_ids, sg, env_start, seg_start, env_count, seg_count,
                     robot, reach, stats, err, queue, order, env_steps, env_step0};
        for (void* q : d)
            if (q) cudaFree(q);
        if (h_tick) cudaFreeHost(h_tick);
        if (h_result) cudaFreeHost(h_result);
    }
};

namespace {

template <class T>
cudaError_t dalloc(T** p, size_t n) {
    *p = nullptr;
    return cudaMalloc((void**)p, sizeof(T) * (n ? n : 1));
}

// Retire the requests of the tick in flight once it has finished.
crowd_status finish_tick(crowd_server_t s) {
    if (!s->tick_in_flight) return CROWD_OK;
    S_TRY(cudaEventSynchronize(s->tick_done), "wait for tick");
    s->tick_in_flight = false;
    int err = 0;
    S_TRY(cudaMemcpy(&err, s->err, sizeof(int), cudaMemcpyDeviceToHost), "read error word");
    if (err) {
        S_TRY(cudaMemset(s->err, 0, sizeof(int)), "clear error word");
        return api_fail(CROWD_EDEVICE, "device error word 0x%x during a serving tick", err);
    }
    for (int k : s->finishing) {
        Req& r = s->reqs[s->slot_req[k]];
        r.result.resize((size_t)r.n * 4);
        std::memcpy(r.result.data(), s->h_result + (size_t)k * s->cfg.max_agents, sizeof(float4) * r.n);
        r.status = CROWD_REQ_DONE;
        r.slot = -1;
        s->finished.push_back(r.id);
        s->bytes_in_use -= r.bytes;
        s->slot_req[k] = 0;
    }
    s->finishing.clear();
    return CROWD_OK;
}

crowd_status admit(crowd_server_t s, Req& r, int k) {
    const crowd_server_config& c = s->cfg;
    const size_t A = (size_t)k * c.max_agents, Sg = (size_t)k * c.max_segments;
    S_TRY(cudaMemcpyAsync(s->state + A, r.state.data(), sizeof(float4) * r.n, cudaMemcpyHostToDevice, s->stream), "admit");
    S_TRY(cudaMemcpyAsync(s->par + A, r.par.data(), sizeof(float4) * r.n, cudaMemcpyHostToDevice, s->stream), "admit");
    S_TRY(cudaMemcpyAsync(s->goal + A, r.goal.data(), sizeof(float2) * r.n, cudaMemcpyHostToDevice, s->stream), "admit");
    S_TRY(cudaMemcpyAsync(s->rv + (size_t)k * c.max_steps, r.rv.data(), sizeof(float2) * r.steps,
                          cudaMemcpyHostToDevice, s->stream), "admit");
    if (r.ns)
        S_TRY(cudaMemcpyAsync(s->segs + Sg, r.segs.data(), sizeof(float4) * r.ns, cudaMemcpyHostToDevice, s->stream),
              "admit");
    // lists are stored relative to the slot's regions: shift to absolute indices
    std::vector<int> starts(r.cell_start);
    for (int& v : starts) v += k * s->ids_stride;
    SegGrid g = r.sg;
    g.off = k * s->cells_stride;
    S_TRY(cudaMemcpyAsync(s->cell_start + (size_t)k * s->cells_stride, starts.data(), sizeof(int) * starts.size(),
                          cudaMemcpyHostToDevice, s->stream), "admit");
    if (!r.cell_ids.empty())
        S_TRY(cudaMemcpyAsync(s->cell_ids + (size_t)k * s->ids_stride, r.cell_ids.data(),
                              sizeof(int) * r.cell_ids.size(), cudaMemcpyHostToDevice, s->stream), "admit");
    S_TRY(cudaMemcpyAsync(s->sg + k, &g, sizeof(SegGrid), cudaMemcpyHostToDevice, s->stream), "admit");
    const int meta[3] = {r.n, r.ns, r.robot};
    S_TRY(cudaMemcpyAsync(s->env_count + k, &meta[0], sizeof(int), cudaMemcpyHostToDevice, s->stream), "admit");
    S_TRY(cudaMemcpyAsync(s->seg_count + k, &meta[1], sizeof(int), cudaMemcpyHostToDevice, s->stream), "admit");
    S_TRY(cudaMemcpyAsync(s->robot + k, &meta[2], sizeof(int), cudaMemcpyHostToDevice, s->stream), "admit");
    S_TRY(cudaMemsetAsync(s->stats + k, 0, sizeof(EnvStats), s->stream), "admit");
    S_TRY(cudaMemsetAsync(s->reach + A, 0xff, sizeof(int) * r.n, s->stream), "admit");
    r.slot = k;
    r.status = CROWD_REQ_RUNNING;
    s->slot_req[k] = r.id;
    s->bytes_in_use += r.bytes;
    return CROWD_OK;
}

}  // namespace

extern "C" {

crowd_status crowd_server_create(const crowd_params* p, float dt, const crowd_server_config* cfg, void* stream,
                                 crowd_server_t* out) {
    if (!out) return api_fail(CROWD_EINVAL, "out is null");
    *out = nullptr;
    if (!p || !cfg) return api_fail(CROWD_EINVAL, "params or config is null");
    if (!(dt > 0.f) || !std::isfinite(dt)) return api_fail(CROWD_EINVAL, "dt must be finite and > 0");
    if (!(p->time_horizon > 0.f) || !(p->neighbor_dist > 0.f) || !(p->time_horizon_obst >= 0.f) ||
        !std::isfinite(p->time_horizon) || !std::isfinite(p->neighbor_dist) || !std::isfinite(p->time_horizon_obst))
        return api_fail(CROWD_EINVAL, "time horizons and neighbor_dist must be finite and positive");
    if (p->max_neighbors < 0 || p->max_neighbors > CROWD_MAX_NEIGHBORS)
        return api_fail(CROWD_EINVAL, "max_neighbors must be in [0, %d]", CROWD_MAX_NEIGHBORS);
    if (cfg->max_slots < 1 || cfg->max_slots > 65536) return api_fail(CROWD_EINVAL, "max_slots must be in [1, 65536]");
    if (cfg->max_agents < 1 || cfg->max_agents > kResidentMaxAgents)
        return api_fail(CROWD_EINVAL, "max_agents must be in [1, %d]", kResidentMaxAgents);
    if (cfg->max_segments < 0 || cfg->max_steps < 1 || cfg->chunk_steps < 1)
        return api_fail(CROWD_EINVAL, "max_segments >= 0, max_steps >= 1 and chunk_steps >= 1 required");
    crowd_server_ctx* s = new (std::nothrow) crowd_server_ctx();
    if (!s) return api_fail(CROWD_ENOMEM, "host allocation failed");
    s->p = *p;
    s->p.flags &= CROWD_FLAG_STATS;
    s->dt = dt;
    s->cfg = *cfg;
    s->stream = (cudaStream_t)stream;
    s->cells_stride = 64 * 64 + 1;
    // segment-list capacity of a slot: each segment is listed in the cells
    // within reach of it, a few dozen on the 64 x 64 slot grid
    s->ids_stride = std::max(4096, 96 * cfg->max_segments);
    const size_t M = cfg->max_slots, A = (size_t)cfg->max_agents;
    auto bail = [&](cudaError_t e, const char* w) {
        delete s;
        return sfail(CROWD_ECUDA, w, e);
    };
    cudaError_t e = cudaSuccess;
#define SALLOC(f, n) \
    if ((e = dalloc(&s->f, (n))) != cudaSuccess) return bail(e, "cudaMalloc " #f);
    SALLOC(state, M * A);
    SALLOC(par, M * A);
    SALLOC(goal, M * A);
    SALLOC(reach, M * A);
    SALLOC(rv, M * cfg->max_steps);
    SALLOC(segs, M * std::max(1, cfg->max_segments));
    SALLOC(cell_start, M * s->cells_stride);
    SALLOC(cell_ids, M * s->ids_stride);
    SALLOC(sg, M);
    SALLOC(env_start, M);
    SALLOC(seg_start, M);
    SALLOC(env_count, M);
    SALLOC(seg_count, M);
    SALLOC(robot, M);
    SALLOC(stats, M);
    SALLOC(err, 1);
    SALLOC(queue, 1);
    SALLOC(order, M);
    SALLOC(env_steps, M);
    SALLOC(env_step0, M);
#undef SALLOC
    if ((e = cudaMallocHost((void**)&s->h_tick, sizeof(int) * 3 * M)) != cudaSuccess) return bail(e, "pinned tick");
    if ((e = cudaMallocHost((void**)&s->h_result, sizeof(float4) * M * A)) != cudaSuccess) return bail(e, "pinned result");
    if ((e = cudaEventCreateWithFlags(&s->tick_done, cudaEventDisableTiming)) != cudaSuccess) return bail(e, "event");
    std::vector<int> es(M), ss(M);
    for (size_t k = 0; k < M; ++k) {
        es[k] = (int)(k * A);
        ss[k] = (int)(k * std::max(1, cfg->max_segments));
    }
    if ((e = cudaMemcpy(s->env_start, es.data(), sizeof(int) * M, cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(s->seg_start, ss.data(), sizeof(int) * M, cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemset(s->err, 0, sizeof(int))) != cudaSuccess ||
        (e = cudaMemset(s->reach, 0xff, sizeof(int) * M * A)) != cudaSuccess)
        return bail(e, "initialise server");
    int dev = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess ||
        (e = cudaDeviceGetAttribute(&s->sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
        return bail(e, "device attributes");
    s->slot_req.assign(M, 0);
    *out = s;
    return CROWD_OK;
}

crowd_status crowd_server_submit(crowd_server_t s, const crowd_request* r, int64_t* id) {
    const TraceRange trace("crowd_server_submit");
    if (!s || !r || !id) return api_fail(CROWD_EINVAL, "null argument");
    if (s->broken) return api_fail(CROWD_ESTATE, "server is unusable after an earlier CUDA failure");
    const crowd_server_config& c = s->cfg;
    if (r->n_agents < 1 || r->n_agents > c.max_agents)
        return api_fail(CROWD_EINVAL, "n_agents must be in [1, %d]", c.max_agents);
    if (r->n_segments < 0 || r->n_segments > c.max_segments)
        return api_fail(CROWD_EINVAL, "n_segments must be in [0, %d]", c.max_segments);
    if (r->n_steps < 1 || r->n_steps > c.max_steps) return api_fail(CROWD_EINVAL, "n_steps must be in [1, %d]", c.max_steps);
    if (r->robot_index < -1 || r->robot_index >= r->n_agents) return api_fail(CROWD_EINVAL, "robot_index out of range");
    const int n = r->n_agents;
    if (!r->radii || !r->max_speeds || !r->init_pos || !r->goals) return api_fail(CROWD_EINVAL, "agent arrays are null");
    if (r->n_segments && !r->segments) return api_fail(CROWD_EINVAL, "segments is null");
    if (!finite_n(r->init_pos, 2 * n) || !finite_n(r->goals, 2 * n) || !finite_n(r->segments, 4 * (size_t)r->n_segments) ||
        (r->robot_vel && !finite_n(r->robot_vel, 2 * (size_t)r->n_steps)))
        return api_fail(CROWD_EINVAL, "inputs hold NaN/Inf");
    for (int i = 0; i < n; ++i) {
        if (!(r->radii[i] > 0.f) || !std::isfinite(r->radii[i])) return api_fail(CROWD_EINVAL, "radius must be > 0");
        if (!(r->max_speeds[i] >= 0.f) || !std::isfinite(r->max_speeds[i]))
            return api_fail(CROWD_EINVAL, "max_speed must be >= 0");
        if (r->pref_speeds && (!(r->pref_speeds[i] >= 0.f) || !std::isfinite(r->pref_speeds[i])))
            return api_fail(CROWD_EINVAL, "pref_speed must be >= 0");
    }
    for (int q = 0; q < r->n_segments; ++q) {
        const float* g = r->segments + 4 * q;
        if (g[0] == g[2] && g[1] == g[3]) return api_fail(CROWD_EINVAL, "segment %d has zero length", q);
    }
    Req q;
    q.id = s->next_id++;
    q.n = n;
    q.ns = r->n_segments;
    q.steps = r->n_steps;
    q.robot = r->robot_index;
    q.state.resize(n);
    q.par.resize(n);
    q.goal.resize(n);
    for (int i = 0; i < n; ++i) {
        q.state[i] = make_float4(r->init_pos[2 * i], r->init_pos[2 * i + 1], 0.f, 0.f);
        q.par[i] = make_float4(r->radii[i], r->max_speeds[i], r->pref_speeds ? r->pref_speeds[i] : r->max_speeds[i], 0.f);
        q.goal[i] = make_float2(r->goals[2 * i], r->goals[2 * i + 1]);
    }
    q.rv.assign(r->n_steps, make_float2(0.f, 0.f));
    if (r->robot_vel)
        for (int k = 0; k < r->n_steps; ++k) q.rv[k] = make_float2(r->robot_vel[2 * k], r->robot_vel[2 * k + 1]);
    q.segs.resize(q.ns);
    for (int k = 0; k < q.ns; ++k)
        q.segs[k] = make_float4(r->segments[4 * k], r->segments[4 * k + 1], r->segments[4 * k + 2], r->segments[4 * k + 3]);
    q.sg = build_seg_grid(0, n, 0, q.ns, r->radii, r->max_speeds, r->segments, s->p.time_horizon,
                          s->p.time_horizon_obst, 0, q.cell_start, q.cell_ids);
    if ((int)q.cell_ids.size() > s->ids_stride || q.sg.W * q.sg.H + 1 > s->cells_stride)
        return api_fail(CROWD_EINVAL, "segment lists exceed the slot capacity (too many segments)");
    q.bytes = (size_t)n * (sizeof(float4) * 2 + sizeof(float2) + sizeof(int)) + sizeof(float2) * q.steps +
              sizeof(float4) * q.ns + sizeof(int) * (q.cell_start.size() + q.cell_ids.size());
    if (q.bytes > c.mem_budget) return api_fail(CROWD_EINVAL, "request larger than the memory budget");
    *id = q.id;
    s->waiting.push_back(q.id);
    s->reqs.emplace(q.id, std::move(q));
    return CROWD_OK;
}

crowd_status crowd_server_tick(crowd_server_t s, int32_t* n_live, int32_t* n_finished) {
    const TraceRange trace("crowd_server_tick");
    if (!s) return api_fail(CROWD_EINVAL, "null server");
    if (s->broken) return api_fail(CROWD_ESTATE, "server is unusable after an earlier CUDA failure");
    const size_t done_before = s->finishing.size();
    crowd_status st = finish_tick(s);
    if (st) return st;
    if (n_finished) *n_finished = (int32_t)done_before;
    // admit waiting requests, first come first served, while slot and budget allow
    const crowd_server_config& c = s->cfg;
    int free_slot = 0;
    while (!s->waiting.empty()) {
        Req& r = s->reqs[s->waiting.front()];
        if (s->bytes_in_use + r.bytes > c.mem_budget) break;
        while (free_slot < c.max_slots && s->slot_req[free_slot]) ++free_slot;
        if (free_slot >= c.max_slots) break;
        st = admit(s, r, free_slot);
        if (st) {
            s->broken = true;
            return st;
        }
        s->waiting.pop_front();
    }
    // one chunk for every live request, largest first
    std::vector<int> live;
    int max_agents = 0;
    for (int k = 0; k < c.max_slots; ++k)
        if (s->slot_req[k]) {
            live.push_back(k);
            max_agents = std::max(max_agents, s->reqs[s->slot_req[k]].n);
        }
    if (n_live) *n_live = (int32_t)live.size();
    if (live.empty()) return CROWD_OK;
    std::stable_sort(live.begin(), live.end(),
                     [&](int a, int b) { return s->reqs[s->slot_req[a]].n > s->reqs[s->slot_req[b]].n; });
    const int L = (int)live.size(), M = c.max_slots;
    int* h_order = s->h_tick;
    int* h_steps = s->h_tick + M;
    int* h_step0 = s->h_tick + 2 * M;
    for (int q = 0; q < L; ++q) {
        const int k = live[q];
        Req& r = s->reqs[s->slot_req[k]];
        h_order[q] = k;
        h_steps[k] = std::min(c.chunk_steps, r.steps - r.done);
        h_step0[k] = r.done;
    }
    S_TRY(cudaMemcpyAsync(s->order, h_order, sizeof(int) * L, cudaMemcpyHostToDevice, s->stream), "tick arrays");
    S_TRY(cudaMemcpyAsync(s->env_steps, h_steps, sizeof(int) * M, cudaMemcpyHostToDevice, s->stream), "tick arrays");
    S_TRY(cudaMemcpyAsync(s->env_step0, h_step0, sizeof(int) * M, cudaMemcpyHostToDevice, s->stream), "tick arrays");
    S_TRY(cudaMemsetAsync(s->queue, 0, sizeof(int), s->stream), "tick queue");
    ResidentArgs a{};
    a.n_work = L;
    a.order = s->order;
    a.queue = s->queue;
    a.env_start = s->env_start;
    a.seg_start = s->seg_start;
    a.robot_index = s->robot;
    a.segs = s->segs;
    a.seg_grid = s->sg;
    a.seg_cell_start = s->cell_start;
    a.seg_cell_ids = s->cell_ids;
    a.par = s->par;
    a.goal = s->goal;
    a.state = s->state;
    a.robot_vel = s->rv;
    a.robot_stride = 0;
    a.n_steps = c.chunk_steps;
    a.dt = s->dt;
    a.tau = s->p.time_horizon;
    a.tau_o = s->p.time_horizon_obst > 0.f ? s->p.time_horizon_obst : s->p.time_horizon;
    a.R = s->p.neighbor_dist;
    a.robot_alpha = s->p.robot_responsibility;
    a.seg_vd = (s->p.flags & CROWD_FLAG_VELOCITY_SEGMENTS) ? 1 : 0;
    a.K = s->p.max_neighbors;
    const bool stats = (s->p.flags & CROWD_FLAG_STATS) != 0;
    a.stats = stats ? s->stats : nullptr;
    a.reach = stats ? s->reach : nullptr;
    a.err = s->err;
    a.max_agents = max_agents;
    a.cell_split = 1;
    a.coop_fallback = 0;
    a.lanes = 1;
    a.env_count = s->env_count;
    a.seg_count = s->seg_count;
    a.env_steps = s->env_steps;
    a.env_step0 = s->env_step0;
    a.rv_env_stride = c.max_steps;
    const int block = resident_block_threads(max_agents);
    const int per_sm = std::max(1, resident_ctas_per_sm(max_agents, block, a.K, 1));
    const int grid = std::max(1, std::min(L, per_sm * s->sms));
    cudaError_t e = launch_resident(a, grid, block, s->stream);
    if (e != cudaSuccess) {
        s->broken = true;
        return sfail(CROWD_ECUDA, "launch serving tick", e);
    }
    // results of the requests this chunk completes go back right behind it
    for (int k : live) {
        Req& r = s->reqs[s->slot_req[k]];
        r.done += h_steps[k];
        if (r.done >= r.steps) {
            S_TRY(cudaMemcpyAsync(s->h_result + (size_t)k * c.max_agents, s->state + (size_t)k * c.max_agents,
                                  sizeof(float4) * r.n, cudaMemcpyDeviceToHost, s->stream),
                  "copy result");
            s->finishing.push_back(k);
        }
    }
    S_TRY(cudaEventRecord(s->tick_done, s->stream), "record tick");
    s->tick_in_flight = true;
    return CROWD_OK;
}

crowd_status crowd_server_poll(crowd_server_t s, int64_t id, float* out_state, int32_t* status) {
    if (!s || !status) return api_fail(CROWD_EINVAL, "null argument");
    auto it = s->reqs.find(id);
    if (it == s->reqs.end()) return api_fail(CROWD_EINVAL, "unknown request id %lld", (long long)id);
    Req& r = it->second;
    if (r.status != CROWD_REQ_DONE && s->tick_in_flight && cudaEventQuery(s->tick_done) == cudaSuccess) {
        crowd_status st = finish_tick(s);
        if (st) return st;
    }
    *status = r.status;
    if (r.status == CROWD_REQ_DONE) {
        if (out_state) std::memcpy(out_state, r.result.data(), sizeof(float) * r.result.size());
        s->reqs.erase(it);
    }
    return CROWD_OK;
}

crowd_status crowd_server_finished(crowd_server_t s, int64_t* ids, int32_t cap, int32_t* n) {
    if (!s || !n || (cap > 0 && !ids)) return api_fail(CROWD_EINVAL, "null argument");
    if (s->tick_in_flight && cudaEventQuery(s->tick_done) == cudaSuccess) {
        crowd_status st = finish_tick(s);
        if (st) return st;
    }
    const int32_t k = (int32_t)std::min<size_t>((size_t)std::max(cap, 0), s->finished.size());
    for (int32_t q = 0; q < k; ++q) ids[q] = s->finished[q];
    s->finished.erase(s->finished.begin(), s->finished.begin() + k);
    *n = k;
    return CROWD_OK;
}

crowd_status crowd_server_info(crowd_server_t s, crowd_server_stats* out) {
    if (!s || !out) return api_fail(CROWD_EINVAL, "null argument");
    out->waiting = (int32_t)s->waiting.size();
    int live = 0;
    for (int64_t q : s->slot_req) live += q ? 1 : 0;
    out->live = live;
    out->bytes_in_use = s->bytes_in_use;
    return CROWD_OK;
}

crowd_status crowd_server_destroy(crowd_server_t s) {
    if (!s) return CROWD_OK;
    cudaError_t e = cudaStreamSynchronize(s->stream);
    delete s;
    if (e != cudaSuccess) return sfail(CROWD_ECUDA, "synchronize before destroy", e);
    return CROWD_OK;
}

}  // extern "C"
