// crowd_step_noalloc: one crowd step of one environment that allocates no
// memory.
//
// Some callers cannot call cudaMalloc at all: code that runs inside another
// framework's memory pool or a fixed device-memory budget, real-time loops
// that must not allocate after start-up, and plug-ins handed only raw device
// pointers by their host.  For them this entry point runs the tiled step
// (the same kernels as large environments of a crowd handle) with every
// intermediate buffer -- cell keys and ranks, cell counts and starts, the
// state in cell order, the per-cell segment lists, the grid descriptor -- in
// one file-scope __device__ array of fixed size, g_noalloc_scratch below.
//
// Every GPU that loads the library holds that array until the process
// exits.  All calls share it and it keeps the last call's contents, so the
// parts that must start at zero are cleared by each call, and calls whose
// work overlaps on the GPU (other streams, other host threads) race on it:
// serialise them.  The first call on a device looks up the array's device
// address (cudaGetSymbolAddress, with that device current) and sets the
// tiled kernel's shared-memory attribute; make that first call before any
// stream capture.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstring>
#include <mutex>

#include "../../include/crowd.h"
#include "crowd_internal.h"

using namespace crowd;

namespace crowd {
crowd_status api_fail(crowd_status st, const char* fmt, ...);
}

namespace {

constexpr int kNaAgents = CROWD_NOALLOC_MAX_AGENTS;
constexpr int kNaCells = CROWD_NOALLOC_MAX_CELLS;
constexpr int kNaSegIds = CROWD_NOALLOC_MAX_SEGMENT_CELLS;
constexpr int kNaGridSide = 256;

// Byte layout of the scratch array (each part 256-byte aligned).
constexpr size_t align256(size_t b) { return (b + 255) & ~size_t(255); }
constexpr size_t kOffEnv = 0;                                          // TiledEnv
constexpr size_t kOffMisc = align256(kOffEnv + sizeof(TiledEnv));      // step counter, error word, reach, total
constexpr size_t kOffKey = align256(kOffMisc + 64);
constexpr size_t kOffRank = align256(kOffKey + sizeof(int) * kNaAgents);
constexpr size_t kOffSid = align256(kOffRank + sizeof(int) * kNaAgents);
constexpr size_t kOffSpv = align256(kOffSid + sizeof(int) * kNaAgents);
constexpr size_t kOffCount = align256(kOffSpv + sizeof(float4) * kNaAgents);
constexpr size_t kOffStart = align256(kOffCount + sizeof(int) * kNaCells);
constexpr size_t kOffSegStart = align256(kOffStart + sizeof(int) * (kNaCells + 1));
constexpr size_t kOffSegIds = align256(kOffSegStart + sizeof(int) * (kNaCells + 1));
constexpr size_t kScratchBytes = align256(kOffSegIds + sizeof(int) * kNaSegIds);

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

struct Misc {
    long long step;
    int err;
    float reach;
    int seg_total;
    int seg_outside;  // a segment endpoint lies outside the caller's box
};

std::mutex g_setup_mutex;
unsigned char* g_scratch_addr[64] = {};

// Device address of the scratch array on the current device (set up once).
crowd_status scratch_address(unsigned char** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return api_fail(CROWD_ECUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
    if (dev < 0 || dev >= 64) return api_fail(CROWD_EINVAL, "device ordinal %d out of range", dev);
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return api_fail(CROWD_ECUDA, "cudaGetSymbolAddress: %s", cudaGetErrorString(e));
        e = tiled_init(kHaloCap);
        if (e != cudaSuccess) return api_fail(CROWD_ECUDA, "tiled kernel attributes: %s", cudaGetErrorString(e));
        g_scratch_addr[dev] = (unsigned char*)p;
    }
    *out = g_scratch_addr[dev];
    return CROWD_OK;
}

// Largest r + tau_o v_max over the agents (one CTA), into misc->reach; a
// segment with an endpoint outside the box [x0, x1] x [y0, y1] sets
// misc->seg_outside (an agent outside the grid is clamped into a border
// cell, whose segment list is complete for it only when every segment lies
// inside the grid).
__global__ void na_reach(const float4* par, int n, float tau_o, const float4* segs, int ns, float x0, float y0,
                         float x1, float y1, Misc* misc) {
    __shared__ float red[32];
    float m = 0.f;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const float4 q = par[i];
        m = fmaxf(m, q.x + tau_o * q.y);
    }
    for (int s = threadIdx.x; s < ns; s += blockDim.x) {
        const float4 g = segs[s];
        if (!(fminf(g.x, g.z) >= x0 && fmaxf(g.x, g.z) <= x1 && fminf(g.y, g.w) >= y0 && fmaxf(g.y, g.w) <= y1))
            misc->seg_outside = 1;
    }
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) m = fmaxf(m, red[w]);
        misc->reach = m * (1.f + 1e-5f) + 1e-6f;
    }
}

// Segment s is listed in a cell when it comes within reach + half the cell
// diagonal of the cell's centre (so within reach of every point the cell
// holds, clamped agents from outside the grid included).  The test runs in
// coordinates relative to the grid origin, so that the cell centres carry no
// rounding error of a large offset; the margin still covers the FP32 error
// of moving the endpoints there, a few units of 2^-24 of |x0| + |y0| + the
// grid's extent.
__device__ __forceinline__ bool seg_near_cell(const TiledEnv& te, float4 sg, int cell, float reach) {
    const float c = 1.f / te.inv_c;
    const float px = ((cell % te.W) + 0.5f) * c, py = ((cell / te.W) + 0.5f) * c;
    const float ax = sg.x - te.x0, ay = sg.y - te.y0, bx = sg.z - te.x0, by = sg.w - te.y0;
    const float ex = bx - ax, ey = by - ay;
    float t = ((px - ax) * ex + (py - ay) * ey) / (ex * ex + ey * ey);
    t = fminf(1.f, fmaxf(0.f, t));
    const float dx = ax + t * ex - px, dy = ay + t * ey - py;
    const float slack = 1e-6f * (fabsf(te.x0) + fabsf(te.y0) + (float)max(te.W, te.H) * c);
    return sqrtf(dx * dx + dy * dy) < (reach + 0.7072f * c) * 1.0001f + 1e-5f + slack;
}

__global__ void na_seg_count(const TiledEnv* env, const float4* segs, int ns, const Misc* misc, int* seg_start) {
    const TiledEnv te = *env;
    const int cell = blockIdx.x * blockDim.x + threadIdx.x;
    if (cell >= te.W * te.H) return;
    int cnt = 0;
    for (int s = 0; s < ns; ++s) cnt += seg_near_cell(te, segs[s], cell, misc->reach) ? 1 : 0;
    seg_start[cell] = cnt;
}

// Exclusive scan of the per-cell counts (one CTA); the total goes to misc.
__global__ void na_seg_scan(const TiledEnv* env, int* seg_start, Misc* misc) {
    __shared__ int warp_sum[32];
    __shared__ int carry;
    const int C = env->W * env->H;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int c0 = 0; c0 < C; c0 += blockDim.x) {
        const int c = c0 + threadIdx.x;
        const int v = c < C ? seg_start[c] : 0;
        int incl = v;
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        if (lane == 31) warp_sum[warp] = incl;
        __syncthreads();
        if (warp == 0) {
            const int nw = blockDim.x >> 5;
            const int ws = lane < nw ? warp_sum[lane] : 0;
            int wincl = ws;
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, wincl, o);
                if (lane >= o) wincl += y;
            }
            if (lane < nw) warp_sum[lane] = wincl - ws;
        }
        __syncthreads();
        const int base = carry;
        if (c < C) seg_start[c] = base + warp_sum[warp] + incl - v;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry = base + warp_sum[warp] + incl;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        seg_start[C] = carry;
        misc->seg_total = carry;
    }
}

__global__ void na_seg_fill(const TiledEnv* env, const float4* segs, int ns, const Misc* misc, const int* seg_start,
                            int* seg_ids) {
    const TiledEnv te = *env;
    const int cell = blockIdx.x * blockDim.x + threadIdx.x;
    if (cell >= te.W * te.H) return;
    int at = seg_start[cell];
    const int end = min(seg_start[cell + 1], kNaSegIds);
    for (int s = 0; s < ns && at < end; ++s)
        if (seg_near_cell(te, segs[s], cell, misc->reach)) seg_ids[at++] = s;
}

}  // namespace

extern "C" crowd_status crowd_step_noalloc(int32_t n_agents, const float* state_in, float* state_out,
                                           const float* agent_params, const float* goals, int32_t robot_index,
                                           int32_t n_segments, const float* segments, const float* box,
                                           const crowd_params* p, float dt, void* cuda_stream) {
    if (!p || !box) return api_fail(CROWD_EINVAL, "params and box are required");
    if (n_agents < 0 || n_agents > kNaAgents)
        return api_fail(CROWD_EINVAL, "n_agents must be in [0, %d] for the allocation-free step", kNaAgents);
    if (n_segments < 0) return api_fail(CROWD_EINVAL, "n_segments < 0");
    if (n_agents > 0 && (!state_in || !state_out || !agent_params || !goals))
        return api_fail(CROWD_EINVAL, "agent buffers are null");
    if (n_segments > 0 && !segments) return api_fail(CROWD_EINVAL, "segments is null");
    if (robot_index < -1 || robot_index >= std::max(n_agents, 1)) return api_fail(CROWD_EINVAL, "robot_index out of range");
    if (!(dt > 0.f) || !std::isfinite(dt)) return api_fail(CROWD_EINVAL, "dt must be finite and > 0");
    if (!(p->time_horizon > 0.f) || !(p->neighbor_dist > 0.f) || !(p->time_horizon_obst >= 0.f) ||
        !std::isfinite(p->time_horizon) || !std::isfinite(p->neighbor_dist) || !std::isfinite(p->time_horizon_obst))
        return api_fail(CROWD_EINVAL, "time horizons and neighbor_dist must be finite and positive");
    if (p->max_neighbors < 0 || p->max_neighbors > CROWD_MAX_NEIGHBORS)
        return api_fail(CROWD_EINVAL, "max_neighbors must be in [0, %d]", CROWD_MAX_NEIGHBORS);
    for (int k = 0; k < 4; ++k)
        if (!std::isfinite(box[k])) return api_fail(CROWD_EINVAL, "box holds NaN/Inf");
    if (!(box[2] >= box[0]) || !(box[3] >= box[1])) return api_fail(CROWD_EINVAL, "box must have x1 >= x0, y1 >= y0");
    if (n_agents == 0) return CROWD_OK;

    // grid over the box: cells of at least R (times a margin for FP32
    // rounding of cell coordinates), at most 256 per side
    const double R = p->neighbor_dist;
    const double ext = std::max(box[2] - box[0], box[3] - box[1]);
    const float c = (float)std::max(R * 1.0001, ext / (kNaGridSide - 1));
    TiledEnv te{};
    te.e = 0;
    te.base = 0;
    te.n = n_agents;
    te.seg0 = 0;
    te.robot = robot_index;
    te.co = 0;
    te.x0 = box[0];
    te.y0 = box[1];
    te.inv_c = std::nextafter(1.0f / c, 0.0f);
    const double cc = 1.0 / (double)te.inv_c;
    te.W = std::min(kNaGridSide, (int)((box[2] - box[0]) / cc) + 1);
    te.H = std::min(kNaGridSide, (int)((box[3] - box[1]) / cc) + 1);
    choose_tile(n_agents, te.W, te.H, te.tx, te.ty);
    te.span = 1;
    const int C = te.W * te.H;
    if (C > kNaCells) return api_fail(CROWD_EINVAL, "grid of %d cells exceeds %d", C, kNaCells);

    unsigned char* base = nullptr;
    crowd_status st = scratch_address(&base);
    if (st) return st;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    TiledEnv* d_env = (TiledEnv*)(base + kOffEnv);
    Misc* misc = (Misc*)(base + kOffMisc);
    int* count = (int*)(base + kOffCount);
    int* seg_start = (int*)(base + kOffSegStart);
    int* seg_ids = (int*)(base + kOffSegIds);
    const float tau_o = p->time_horizon_obst > 0.f ? p->time_horizon_obst : p->time_horizon;

#define NA_TRY(expr, what)                                                                    \
    do {                                                                                      \
        cudaError_t e_ = (expr);                                                              \
        if (e_ != cudaSuccess) return api_fail(CROWD_ECUDA, "%s: %s", what, cudaGetErrorString(e_)); \
    } while (0)
    NA_TRY(cudaMemcpyAsync(d_env, &te, sizeof(TiledEnv), cudaMemcpyHostToDevice, s), "write grid");
    NA_TRY(cudaMemsetAsync(misc, 0, sizeof(Misc), s), "clear scratch");
    NA_TRY(cudaMemsetAsync(count, 0, sizeof(int) * C, s), "clear cell counts");
    // per-cell segment lists, checked against the scratch capacity
    na_reach<<<1, 1024, 0, s>>>((const float4*)agent_params, n_agents, tau_o, (const float4*)segments, n_segments,
                                box[0], box[1], box[2], box[3], misc);
    na_seg_count<<<(C + 255) / 256, 256, 0, s>>>(d_env, (const float4*)segments, n_segments, misc, seg_start);
    na_seg_scan<<<1, 1024, 0, s>>>(d_env, seg_start, misc);
    NA_TRY(cudaGetLastError(), "segment lists");
    Misc h_misc{};
    NA_TRY(cudaMemcpyAsync(&h_misc, misc, sizeof(Misc), cudaMemcpyDeviceToHost, s), "read list size");
    NA_TRY(cudaStreamSynchronize(s), "synchronize");
    if (h_misc.seg_outside)
        return api_fail(CROWD_EINVAL, "a segment lies outside the box: the box must contain every segment");
    if (h_misc.seg_total > kNaSegIds)
        return api_fail(CROWD_EINVAL, "%d segment-cell pairs exceed the allocation-free capacity %d", h_misc.seg_total,
                        kNaSegIds);
    na_seg_fill<<<(C + 255) / 256, 256, 0, s>>>(d_env, (const float4*)segments, n_segments, misc, seg_start, seg_ids);
    NA_TRY(cudaGetLastError(), "segment lists");

    TiledStepArgs a{};
    a.envs = d_env;
    a.n_envs = 1;
    a.state_in = (float4*)state_in;  // read only: no robot command is written back (robot_vel is null)
    a.state_out = (float4*)state_out;
    a.robot_vel = nullptr;
    a.par = (const float4*)agent_params;
    a.goal = const_cast<float2*>((const float2*)goals);  // read only: no goal queue here (a.goals.q == 0)
    a.segs = (const float4*)segments;
    a.seg_cell_start = seg_start;
    a.seg_cell_ids = seg_ids;
    a.key = (int*)(base + kOffKey);
    a.rank = (int*)(base + kOffRank);
    a.count = count;
    a.start = (int*)(base + kOffStart);
    a.sorted_pv = (float4*)(base + kOffSpv);
    a.sorted_id = (int*)(base + kOffSid);
    a.halo_cap = kHaloCap;
    a.R = p->neighbor_dist;
    a.dt = dt;
    a.tau = p->time_horizon;
    a.tau_o = tau_o;
    a.robot_alpha = p->robot_responsibility;
    a.seg_vd = (p->flags & CROWD_FLAG_VELOCITY_SEGMENTS) ? 1 : 0;
    a.K = p->max_neighbors;
    a.mode = kTiledStep;
    a.step_index = &misc->step;
    a.err = &misc->err;
    const int max_tiles = ((te.W + te.tx - 1) / te.tx) * ((te.H + te.ty - 1) / te.ty);
    NA_TRY(launch_tiled_step(a, n_agents, max_tiles, s), "allocation-free step");
    // the device error word of this step (an agent with more segments in
    // reach than its line buffer holds kept the nearest ones): reported
    // here, before the next call clears it
    int h_err = 0;
    NA_TRY(cudaMemcpyAsync(&h_err, &misc->err, sizeof(int), cudaMemcpyDeviceToHost, s), "read error word");
    NA_TRY(cudaStreamSynchronize(s), "synchronize");
#undef NA_TRY
    if (h_err & kErrObstacleOverflow)
        return api_fail(CROWD_EDEVICE, "an agent had more than %d static segments in reach; the nearest were kept",
                        kMaxObstacleLines);
    if (h_err) return api_fail(CROWD_EDEVICE, "device error word 0x%x", h_err);
    return CROWD_OK;
}
