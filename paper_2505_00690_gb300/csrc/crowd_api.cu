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
    float4* segs = nullptr;
    float2* robot_vel = nullptr;
    size_t robot_vel_cap = 0;
    int* nbr = nullptr;
    int* reach = nullptr;
    EnvStats* stats = nullptr;
    WorkCount* work = nullptr;

    // launch configuration
    int block = 0, grid = 0;

    ~crowd_ctx() {
        void* ptrs[] = {env_start, seg_start, robot_index, order, queue, err, state, par, goal,
                        segs, robot_vel, nbr, reach, stats, work};
        for (void* q : ptrs)
            if (q) cudaFree(q);
    }
};

namespace {

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

}  // namespace

extern "C" {

int32_t crowd_abi_version(void) { return 1; }

const char* crowd_last_error(void) { return g_last_error.c_str(); }

int64_t crowd_num_agents(crowd_t h) { return h ? h->N : 0; }
int32_t crowd_num_envs(crowd_t h) { return h ? h->E : 0; }

crowd_status crowd_create(int32_t n_envs, const int32_t* agents_per_env, const float* radii,
                          const float* max_speeds, const float* pref_speeds, const float* init_pos,
                          const int32_t* robot_index, const int32_t* segs_per_env, const float* segments,
                          const crowd_params* p, void* cuda_stream, crowd_t* out) {
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
    if (max_agents > kResidentMaxAgents)
        return fail(CROWD_EINVAL, "an environment has %d agents; at most %d per environment are supported",
                    max_agents, kResidentMaxAgents);
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
    // largest environments first: the queue then balances uneven batches
    std::vector<int> order(n_envs);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(),
                     [&](int a, int b) { return agents_per_env[a] > agents_per_env[b]; });
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
        {h->order, order.data(), sizeof(int) * n_envs},
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
    h->block = resident_block_threads(max_agents);
    int sms = 0;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device)) != cudaSuccess) {
        cuda_fail(e, "device attributes");
        return bail(CROWD_ECUDA);
    }
    const int per_sm = std::max(1, resident_ctas_per_sm(max_agents, h->block, p->max_neighbors));
    h->grid = std::max(1, std::min(n_envs, per_sm * sms));

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
    return copy_in(h, h->goal, goals, sizeof(float2) * h->N, ptr_kind, "copy goals");
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
    ResidentArgs a{};
    a.n_work = h->E;
    a.order = h->order;
    a.queue = h->queue;
    a.env_start = h->env_start;
    a.seg_start = h->seg_start;
    a.robot_index = h->robot_index;
    a.segs = h->segs;
    a.par = h->par;
    a.goal = h->goal;
    a.state = h->state;
    a.robot_vel = rv;
    a.robot_stride = h->E;
    a.n_steps = n_steps;
    a.dt = dt;
    a.tau = h->p.time_horizon;
    a.tau_o = h->p.time_horizon_obst > 0.f ? h->p.time_horizon_obst : h->p.time_horizon;
    a.R = h->p.neighbor_dist;
    a.robot_alpha = h->p.robot_responsibility;
    a.K = h->p.max_neighbors;
    a.nbr_out = h->nbr;
    const bool stats = (h->p.flags & CROWD_FLAG_STATS) != 0;
    a.stats = stats ? h->stats : nullptr;
    a.reach = stats ? h->reach : nullptr;
    a.step_base = h->step_index;
    a.work = h->work;
    a.err = h->err;
    a.max_agents = h->max_agents;
    CUDA_TRY(cudaMemsetAsync(h->queue, 0, sizeof(int), h->stream), "reset work queue");
    cudaError_t e = launch_resident(a, h->grid, h->block, h->stream);
    if (e != cudaSuccess) {
        h->broken = e != cudaErrorInvalidValue && e != cudaErrorInvalidConfiguration;
        return cuda_fail(e, "launch crowd step");
    }
    h->step_index += n_steps;
    return CROWD_OK;
}

crowd_status crowd_read_state(crowd_t h, float* out, int32_t ptr_kind) {
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

crowd_status crowd_read_work(crowd_t h, crowd_work* out) {
    crowd_status st = check_handle(h);
    if (st) return st;
    if (!h->work) return fail(CROWD_ESTATE, "created without CROWD_FLAG_COUNT_WORK");
    if (!out) return fail(CROWD_EINVAL, "out is null");
    static_assert(sizeof(WorkCount) == sizeof(crowd_work), "work counter layout");
    CUDA_TRY(cudaMemcpyAsync(out, h->work, sizeof(WorkCount), cudaMemcpyDeviceToHost, h->stream), "copy work out");
    return read_err_word(h);
}

crowd_status crowd_reset_stats(crowd_t h) {
    crowd_status st = check_handle(h);
    if (st) return st;
    if (h->N) CUDA_TRY(cudaMemsetAsync(h->reach, 0xff, sizeof(int) * h->N, h->stream), "reset reach");
    if (h->E) CUDA_TRY(cudaMemsetAsync(h->stats, 0, sizeof(EnvStats) * h->E, h->stream), "reset stats");
    h->step_index = 0;
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
