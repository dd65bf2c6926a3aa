// Shared-memory-resident crowd step (kernel templates; included by the
// translation units that instantiate it for each lanes-per-agent count).
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "crowd_agent.cuh"
#include "crowd_group.cuh"
#include "crowd_internal.h"
#include "crowd_vehicles.cuh"
#include "orca_device.cuh"

namespace crowd {

namespace {

constexpr int kMaxThreads = 512;
constexpr int kMaxWarps = kMaxThreads / 32;

struct Smem {
    float4* pv;    // [Nm] current state
    float4* nv;    // [Nm] next state
    float4* par;   // [Nm] (r, v_max, preferred speed, 0)
    float4* spv;   // [Nm] state in cell order
    float2* goal;  // [Nm]
    int* sid;      // [Nm] agent index of each sorted slot
    int* cell;     // [kMaxCells + 1] counts, then starts
    unsigned short* key;   // [Nm] cell of each agent
    unsigned short* rank;  // [Nm] rank of each agent inside its cell
    unsigned char* pend;   // [Nm] agents deferred to the next fallback round
    FbEntry* fb;           // [fb_cap] agents queued for the cooperative fallback
    Line* fb_lines;        // [fb_cap][lmax] their lines
    Line* fb_scratch;      // [warps][lmax] subproblem lines of each warp
    int fb_cap, lmax;
};

// Fallback queue capacity: about 1/16 of the agents, 8..16 (the urban block
// has ~2.5% infeasible LPs per step; agents that find it full run again in
// another cooperative round).
__host__ __device__ inline int fb_capacity(int max_agents) {
    const int c = (max_agents + 15) / 16;
    return c < 8 ? 8 : (c > 16 ? 16 : c);
}

__host__ __device__ inline int round_up4(int n) { return (n + 3) & ~3; }

__host__ __device__ inline size_t smem_layout(int max_agents, int kmax, int warps, Smem* s, unsigned char* base) {
    const int nm = round_up4(max_agents > 0 ? max_agents : 1);
    const int lmax = kmax + kMaxObstacleLines;
    const int fb_cap = fb_capacity(max_agents);
    size_t off = 0;
    auto take = [&](size_t bytes) {
        unsigned char* p = base ? base + off : nullptr;
        off += (bytes + 15) & ~size_t(15);
        return p;
    };
    unsigned char* pv = take(sizeof(float4) * nm);
    unsigned char* nv = take(sizeof(float4) * nm);
    unsigned char* par = take(sizeof(float4) * nm);
    unsigned char* spv = take(sizeof(float4) * nm);
    unsigned char* goal = take(sizeof(float2) * nm);
    unsigned char* sid = take(sizeof(int) * nm);
    unsigned char* cell = take(sizeof(int) * (kMaxCells + 1));
    unsigned char* key = take(sizeof(unsigned short) * nm);
    unsigned char* rank = take(sizeof(unsigned short) * nm);
    unsigned char* pend = take(nm);
    unsigned char* fb = take(sizeof(FbEntry) * fb_cap);
    unsigned char* fb_lines = take(sizeof(Line) * fb_cap * lmax);
    unsigned char* fb_scratch = take(sizeof(Line) * warps * lmax);
    if (s) {
        s->pv = (float4*)pv;
        s->nv = (float4*)nv;
        s->par = (float4*)par;
        s->spv = (float4*)spv;
        s->goal = (float2*)goal;
        s->sid = (int*)sid;
        s->cell = (int*)cell;
        s->key = (unsigned short*)key;
        s->rank = (unsigned short*)rank;
        s->pend = pend;
        s->fb = (FbEntry*)fb;
        s->fb_lines = (Line*)fb_lines;
        s->fb_scratch = (Line*)fb_scratch;
        s->fb_cap = fb_cap;
        s->lmax = lmax;
    }
    return off;
}

struct Grid {
    float x0, y0, inv_c;
    int W, H;
};

__device__ __forceinline__ int cell_coord(float v, float v0, float inv_c, int n) {
    int c = __float2int_rd((v - v0) * inv_c);
    return min(max(c, 0), n - 1);
}

// Block-wide bounding box -> grid with cell size >= R / split (times a margin
// that covers FP32 rounding of the cell coordinate), at most kGridMax per
// side; neighbours then lie within `split` cells.
__device__ __forceinline__ void build_grid(const Smem& S, int n, float R, int split, float* red, Grid* g) {
    float xl = INFINITY, xh = -INFINITY, yl = INFINITY, yh = -INFINITY;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const float4 p = S.pv[i];
        xl = fminf(xl, p.x);
        xh = fmaxf(xh, p.x);
        yl = fminf(yl, p.y);
        yh = fmaxf(yh, p.y);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        xl = fminf(xl, __shfl_xor_sync(0xffffffffu, xl, o));
        xh = fmaxf(xh, __shfl_xor_sync(0xffffffffu, xh, o));
        yl = fminf(yl, __shfl_xor_sync(0xffffffffu, yl, o));
        yh = fmaxf(yh, __shfl_xor_sync(0xffffffffu, yh, o));
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) {
        red[4 * warp + 0] = xl;
        red[4 * warp + 1] = xh;
        red[4 * warp + 2] = yl;
        red[4 * warp + 3] = yh;
    }
    for (int c = threadIdx.x; c <= kMaxCells; c += blockDim.x) S.cell[c] = 0;
    __syncthreads();
    if (threadIdx.x == 0) {
        const int nw = (blockDim.x + 31) >> 5;
        for (int w = 1; w < nw; ++w) {
            xl = fminf(xl, red[4 * w + 0]);
            xh = fmaxf(xh, red[4 * w + 1]);
            yl = fminf(yl, red[4 * w + 2]);
            yh = fmaxf(yh, red[4 * w + 3]);
        }
        if (!(xh >= xl)) { xl = 0.f; xh = 0.f; }
        if (!(yh >= yl)) { yl = 0.f; yh = 0.f; }
        const float ext = fmaxf(xh - xl, yh - yl);
        const float c = fmaxf(R * 1.0001f / (float)split, ext / (float)(kGridMax - 1));
        g->x0 = xl;
        g->y0 = yl;
        g->inv_c = __frcp_rz(c);
        g->W = 1 + (int)fminf(fmaxf((xh - xl) * g->inv_c, 0.f), (float)(kGridMax - 1));
        g->H = 1 + (int)fminf(fmaxf((yh - yl) * g->inv_c, 0.f), (float)(kGridMax - 1));
    }
    __syncthreads();
}

// Counting sort of the environment's agents by cell into S.spv / S.sid.
__device__ __forceinline__ void sort_by_cell(const Smem& S, int n, const Grid& g) {
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const float4 p = S.pv[i];
        const int k = cell_coord(p.y, g.y0, g.inv_c, g.H) * g.W + cell_coord(p.x, g.x0, g.inv_c, g.W);
        S.key[i] = (unsigned short)k;
        S.rank[i] = (unsigned short)atomicAdd(&S.cell[k], 1);
    }
    __syncthreads();
    if (threadIdx.x < 32) {
        // exclusive scan of the cell counts by warp 0: each lane owns a run of cells
        const int C = g.W * g.H;
        const int lane = threadIdx.x;
        const int per = (C + 31) / 32;
        const int lo = min(C, lane * per), hi = min(C, lo + per);
        int sum = 0;
        for (int c = lo; c < hi; ++c) sum += S.cell[c];
        int incl = sum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        int run = incl - sum;
        for (int c = lo; c < hi; ++c) {
            const int cnt = S.cell[c];
            S.cell[c] = run;
            run += cnt;
        }
        if (lane == 31) S.cell[C] = incl;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const int slot = S.cell[S.key[i]] + S.rank[i];
        S.spv[slot] = S.pv[i];
        S.sid[slot] = i;
    }
    __syncthreads();
}

struct StepCtx {
    int e, base, n, robot, seg0, ns;
    long long step_base;  // global index of the first step of this launch
    SegGrid sg;
    int step;  // 0-based step inside this launch
    bool last;  // last step of the launch
    Grid g;
};

// Candidates of the environment in cell order, in shared memory.
struct SmemSource {
    const float4* spv;
    const int* sid;
    const int* cell;
    int W;
    __device__ __forceinline__ int2 row(int yy, int xa, int xb) const {
        return make_int2(cell[yy * W + xa], cell[yy * W + xb + 1]);
    }
    __device__ __forceinline__ float4 cand(int u) const { return spv[u]; }
    __device__ __forceinline__ int cand_id(int u) const { return sid[u]; }
};

// Agents of the environment by index, in shared memory.
struct SmemAgents {
    const float4* pv;
    const float4* par;
    __device__ __forceinline__ float4 state(int j) const { return pv[j]; }
    __device__ __forceinline__ float radius(int j) const { return par[j].x; }
    __device__ __forceinline__ bool vehicle(int j) const { return par[j].w != 0.f; }
    __device__ __forceinline__ float4 params(int j) const { return par[j]; }
};

// The environment's crowd as the car update reads it (shared memory).
struct SmemCrowd {
    const float4* pv_;
    const float4* par_;
    __device__ __forceinline__ float4 pv(int k) const { return pv_[k]; }
    __device__ __forceinline__ float4 par(int k) const { return par_[k]; }
};

// The segment list of the static segment-grid cell holding position `me`.
__device__ __forceinline__ ListedSegments cell_segments(const ResidentArgs& a, const StepCtx& c, float4 me) {
    const int k = cell_coord(me.y, c.sg.y0, c.sg.inv_c, c.sg.H) * c.sg.W + cell_coord(me.x, c.sg.x0, c.sg.inv_c, c.sg.W);
    const int s0 = __ldg(&a.seg_cell_start[c.sg.off + k]), s1 = __ldg(&a.seg_cell_start[c.sg.off + k + 1]);
    return ListedSegments{a.seg_cell_ids + s0, s1 - s0};
}

// A6 for agent i: integrate into the next-state buffer, statistics.
__device__ __forceinline__ void integrate(const ResidentArgs& a, const Smem& S, const StepCtx& c, int i, float4 me,
                                          float r, float2 v, double& speed_acc) {
    float4 nx;
    nx.x = fmaf(a.dt, v.x, me.x);
    nx.y = fmaf(a.dt, v.y, me.y);
    nx.z = v.x;
    nx.w = v.y;
    S.nv[i] = nx;
    if (a.stats && i != c.robot && S.par[i].z >= 0.f) {
        speed_acc += (double)sqrtf(v.x * v.x + v.y * v.y);
        if (a.reach) {
            int* rp = a.reach + c.base + i;
            const float2 gl = S.goal[i];
            const float gx = gl.x - nx.x, gy = gl.y - nx.y;
            if (*rp < 0 && sqrtf(gx * gx + gy * gy) <= r) *rp = (int)(c.step_base + c.step + 1);
        }
    }
}

// Returns true when the agent's infeasible LP found the fallback queue full
// (the agent then runs again in the next round).
template <int KMAX>
__device__ __forceinline__ bool agent_update(const ResidentArgs& a, const AgentParams& ap, const Smem& S,
                                             const StepCtx& c, int t, double& speed_acc, Tally& w,
                                             const FbQueue& fbq, bool export_nbrs) {
    const int i = S.sid[t];
    const float4 me = S.spv[t];
    const float4 pr = S.par[i];

    // A1/A2: K nearest within R, ranked by (FP64 key, index)
    NbList<KMAX> nb;
    const SmemSource src{S.spv, S.sid, S.cell, c.g.W};
    select_neighbors<KMAX, false>(src, CellGeom{c.g.x0, c.g.y0, c.g.inv_c}, cell_coord(me.x, c.g.x0, c.g.inv_c, c.g.W),
                           cell_coord(me.y, c.g.y0, c.g.inv_c, c.g.H), c.g.W, c.g.H, i, me, a.R, a.K, nb, w,
                           a.cell_split, a.work != nullptr);
    const int K = a.K;
    if (c.last && a.nbr_out && export_nbrs) {
        int* out = a.nbr_out + (size_t)(c.base + i) * K;
#pragma unroll
        for (int s = 0; s < KMAX; ++s)
            if (s < K) out[s] = s < nb.cnt ? nb.id[s] : -1;
    }

    // A3-A5 (the robot is not solved: it keeps its command); an infeasible
    // LP is queued for the warp-cooperative fallback, integrated there
    ++w.agent_steps;
    if (i == c.robot) {
        integrate(a, S, c, i, me, pr.x, make_float2(me.z, me.w), speed_acc);
        return false;
    }
    bool queued, deferred;
    const float2 v = solve_velocity<KMAX, false>(ap, SmemAgents{S.pv, S.par}, i, c.robot, me, pr, S.goal[i], c.seg0,
                                          cell_segments(a, c, me), nb, w, a.coop_fallback ? &fbq : nullptr, queued,
                                          deferred);
    if (!queued && !deferred) integrate(a, S, c, i, me, pr.x, v, speed_acc);
    return deferred;
}

// A car's slot in the agent pass (cars are dispatched here by the kernel, so
// that the agent update itself carries no test for them, which measurably
// slowed it): the car's neighbour list when the lists are exported this
// step, then the move of its commanded velocity.
template <int KMAX>
__device__ __noinline__ void vehicle_update(const ResidentArgs& a, const Smem& S, const StepCtx& c, int t,
                                            double& speed_acc, Tally& w) {
    const int i = S.sid[t];
    const float4 me = S.spv[t];
    if (c.last && a.nbr_out) {
        NbList<KMAX> nb;
        const SmemSource src{S.spv, S.sid, S.cell, c.g.W};
        select_neighbors<KMAX, false>(src, CellGeom{c.g.x0, c.g.y0, c.g.inv_c}, cell_coord(me.x, c.g.x0, c.g.inv_c, c.g.W),
                               cell_coord(me.y, c.g.y0, c.g.inv_c, c.g.H), c.g.W, c.g.H, i, me, a.R, a.K, nb, w,
                               a.cell_split, a.work != nullptr);
        int* out = a.nbr_out + (size_t)(c.base + i) * a.K;
        for (int s = 0; s < a.K; ++s) out[s] = s < nb.cnt ? nb.id[s] : -1;
    }
    ++w.agent_steps;
    integrate(a, S, c, i, me, S.par[i].x, make_float2(me.z, me.w), speed_acc);
}

// One agent by a group of G lanes (see crowd_group.cuh); lane 0 writes.
template <int KMAX, int G>
__device__ __forceinline__ void agent_update_group(const ResidentArgs& a, const AgentParams& ap, const Smem& S,
                                                   const StepCtx& c, int t, double& speed_acc, Tally& w) {
    const Grp<G> g;
    const int i = S.sid[t];
    const float4 me = S.spv[t];
    const float4 pr = S.par[i];
    NbList<KMAX> nb;
    const SmemSource src{S.spv, S.sid, S.cell, c.g.W};
    group_select<KMAX, G>(g, src, cell_coord(me.x, c.g.x0, c.g.inv_c, c.g.W), cell_coord(me.y, c.g.y0, c.g.inv_c, c.g.H),
                          c.g.W, c.g.H, i, me, a.R, a.K, nb, w, a.cell_split);
    if (g.lane == 0) {
        ++w.agent_steps;
        if (c.last && a.nbr_out) {
            int* out = a.nbr_out + (size_t)(c.base + i) * a.K;
#pragma unroll
            for (int s = 0; s < KMAX; ++s)
                if (s < a.K) out[s] = s < nb.cnt ? nb.id[s] : -1;
        }
    }
    if (i == c.robot || pr.z < 0.f) {
        if (g.lane == 0) integrate(a, S, c, i, me, pr.x, make_float2(me.z, me.w), speed_acc);
        return;
    }
    const float2 v = group_solve<KMAX, G>(g, ap, SmemAgents{S.pv, S.par}, i, c.robot, me, pr, S.goal[i], c.seg0,
                                          cell_segments(a, c, me), nb, w);
    if (g.lane == 0) integrate(a, S, c, i, me, pr.x, v, speed_acc);
}

// The queued fallbacks of this step, one warp per agent.
__device__ __forceinline__ void run_fallbacks(const ResidentArgs& a, const Smem& S, const StepCtx& c, int n_queued,
                                              double& speed_acc) {
    const int warp = threadIdx.x >> 5, warps = blockDim.x >> 5;
    Line* scratch = S.fb_scratch + (size_t)warp * S.lmax;
    for (int q = warp; q < n_queued; q += warps) {
        const FbEntry f = S.fb[q];
        const float2 v = coop_fallback(S.fb_lines + (size_t)q * S.lmax, f.n, f.n_hard, f.vmax, f.pref, scratch);
        if ((threadIdx.x & 31) == 0) integrate(a, S, c, f.agent, f.me, S.par[f.agent].x, v, speed_acc);
        __syncwarp();
    }
}

// Collision events of the current (post-integration) state: agent pairs
// i < j closer than r_i + r_j - kCollideDepth, agents closer than
// r_i - kCollideDepth to a segment.
__device__ __forceinline__ void count_collisions(const ResidentArgs& a, const Smem& S, const StepCtx& c, int t,
                                                 unsigned long long& ca, unsigned long long& cs) {
    const int i = S.sid[t];
    const float4 me = S.spv[t];
    const float ri = S.par[i].x;
    const int cx = cell_coord(me.x, c.g.x0, c.g.inv_c, c.g.W);
    const int cy = cell_coord(me.y, c.g.y0, c.g.inv_c, c.g.H);
    const int sp = a.cell_split;
    const int xa = max(cx - sp, 0), xb = min(cx + sp, c.g.W - 1);
    for (int yy = max(cy - sp, 0); yy <= min(cy + sp, c.g.H - 1); ++yy) {
        const int b0 = S.cell[yy * c.g.W + xa], b1 = S.cell[yy * c.g.W + xb + 1];
        for (int u = b0; u < b1; ++u) {
            const int j = S.sid[u];
            if (j <= i) continue;
            const float4 o = S.spv[u];
            const float dx = o.x - me.x, dy = o.y - me.y;
            if (sqrtf(dx * dx + dy * dy) < ri + S.par[j].x - kCollideDepth) ++ca;
        }
    }
    const float lim = ri - kCollideDepth;
    const ListedSegments sl = cell_segments(a, c, me);
    for (int q = 0; q < sl.count(); ++q) {
        const float4 sg = __ldg(&a.segs[c.seg0 + sl.id(q)]);
        if (box_dist2(me.x, me.y, sg) >= lim * lim) continue;
        float qx, qy;
        if (sqrtf(seg_dist2(me.x, me.y, sg, qx, qy)) < lim) ++cs;
    }
}

// Groups of 4 and 8 lanes run 512-thread blocks for 128 or 64 solved agents;
// two such blocks per SM need at most 64 registers a thread.
template <int KMAX, int G>
__global__ void __launch_bounds__(kMaxThreads, G >= 4 ? 2 : 1) resident_kernel(ResidentArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ float red[4 * kMaxWarps];
    __shared__ Grid grid;
    __shared__ int s_work;
    __shared__ unsigned long long s_ca, s_cs;
    __shared__ double s_speed;
    Smem S;
    smem_layout(a.max_agents, KMAX, blockDim.x >> 5, &S, smem_raw);
    __shared__ int s_fb_count, s_pend, s_item;

    for (;;) {
        if (threadIdx.x == 0) s_work = atomicAdd(a.queue, 1);
        __syncthreads();
        const int w = s_work;
        if (w >= a.n_work) break;
        StepCtx c;
        c.e = a.order[w];
        c.base = a.env_start[c.e];
        c.n = a.env_count ? a.env_count[c.e] : a.env_start[c.e + 1] - c.base;
        c.robot = a.robot_index[c.e];
        c.seg0 = a.seg_start[c.e];
        c.ns = a.seg_count ? a.seg_count[c.e] : a.seg_start[c.e + 1] - c.seg0;
        c.sg = a.seg_grid[c.e];
        const int n_steps = a.env_steps ? a.env_steps[c.e] : a.n_steps;
        const int step0 = a.env_step0 ? a.env_step0[c.e] : 0;
        c.step_base = a.step_base + step0;
        for (int i = threadIdx.x; i < c.n; i += blockDim.x) {
            S.pv[i] = a.state[c.base + i];
            S.par[i] = __ldg(&a.par[c.base + i]);
            S.goal[i] = __ldg(&a.goal[c.base + i]);
        }
        if (threadIdx.x == 0) {
            s_ca = 0;
            s_cs = 0;
            s_speed = 0.0;
        }
        __syncthreads();

        double speed_acc = 0.0;
        unsigned long long ca = 0, cs = 0;
        Tally tally;
        // cars are looked for only in environments that have some (a test per
        // agent in the others cost the dense crowd a third of its time)
        const bool env_veh = a.veh.n > 0 && a.veh.start[c.e + 1] > a.veh.start[c.e];
        const AgentParams ap{a.R, a.dt, a.tau, a.tau_o, a.robot_alpha, a.K, a.segs, a.err, a.seg_vd};
        // the queue capacity depends on this environment alone, so that its
        // results do not depend on the batch it runs in
        const FbQueue fbq{&s_fb_count, min(S.fb_cap, fb_capacity(c.n)), S.lmax, S.fb, S.fb_lines,
                          a.coop_fallback == 2};
        const int passes = n_steps + (a.stats ? 1 : 0);
        for (int step = 0; step < passes; ++step) {
            const bool compute = step < n_steps;
            if (compute && a.goals.active()) {
                // goal queue: agents within reach of their goal move on to the next
                for (int i = threadIdx.x; i < c.n; i += blockDim.x) {
                    if (i == c.robot || S.par[i].w != 0.f) continue;
                    const float2 cur = S.goal[i];
                    const float2 nx = advance_goal(a.goals, c.base + i, c.e, S.pv[i], S.par[i].x, cur);
                    if (nx.x != cur.x || nx.y != cur.y) {
                        S.goal[i] = nx;
                        a.goal[c.base + i] = nx;
                    }
                }
            }
            if (compute && a.veh.n > 0) {
                // cars: all of them from the step-start state, then written
                const int vb = a.veh.start[c.e], ve = a.veh.start[c.e + 1];
                const int vi = vb + (int)threadIdx.x;
                float s_new = 0.f, v_new = 0.f;
                if (vi < ve) idm_vehicle(a.veh, vi, vb, ve, SmemCrowd{S.pv, S.par}, c.n, a.dt, s_new, v_new);
                __syncthreads();
                if (vi < ve) place_vehicle(a.veh, vi, s_new, v_new, a.dt, S.pv + (a.veh.agent[vi] - c.base));
            }
            if (compute && c.robot >= 0 && c.robot < c.n && a.robot_vel && threadIdx.x == 0) {
                const size_t at = a.env_step0 ? (size_t)c.e * a.rv_env_stride + step0 + step
                                              : (size_t)step * a.robot_stride + c.e;
                const float2 cmd = __ldg(&a.robot_vel[at]);
                S.pv[c.robot].z = cmd.x;
                S.pv[c.robot].w = cmd.y;
            }
            __syncthreads();
            build_grid(S, c.n, a.R, a.cell_split, red, &grid);
            c.g = grid;
            sort_by_cell(S, c.n, c.g);
            c.step = step;
            c.last = step == n_steps - 1;
            if (a.stats && step > 0)
                for (int t = threadIdx.x; t < c.n; t += blockDim.x) count_collisions(a, S, c, t, ca, cs);
            if (!compute) break;
            if (threadIdx.x == 0) {
                s_fb_count = 0;
                s_pend = 0;
                s_item = 0;
            }
            __syncthreads();
            if (G == 1) {
                // each warp takes the environment's agents 32 at a time from
                // a shared counter (items = ceil(n / 32)), so that a warp done
                // early takes the next item instead of waiting for a round:
                // item k is the slots 32 k .. 32 k + 31 in cell order, or with
                // agent_order 1 the slots k, k + items, k + 2 items, ..., so
                // that the agents of a crowded region (adjacent in cell order,
                // and the costliest) are spread over the items
                const int lane = threadIdx.x & 31;
                const int items = (c.n + 31) >> 5;
                for (;;) {
                    int item = 0;
                    if (lane == 0) item = atomicAdd(&s_item, 1);
                    item = __shfl_sync(0xffffffffu, item, 0);
                    if (item >= items) break;
                    const int t = a.agent_order ? item + lane * items : (item << 5) + lane;
                    if (t >= c.n) continue;
                    if (env_veh && S.par[S.sid[t]].z < 0.f) {  // a car (negative preferred speed)
                        vehicle_update<KMAX>(a, S, c, t, speed_acc, tally);
                        S.pend[t] = 0;
                        continue;
                    }
                    const bool def = agent_update<KMAX>(a, ap, S, c, t, speed_acc, tally, fbq, true);
                    S.pend[t] = def ? 1 : 0;
                    if (def) atomicAdd(&s_pend, 1);
                }
            } else {
                // one group of G lanes per agent (all lanes of a group take the
                // same slot); the robot, which is not solved, is integrated by
                // thread 0 apart unless its neighbour list is exported
                const int groups = blockDim.x / G;
                const int tr = (c.robot >= 0 && c.robot < c.n) ? S.cell[S.key[c.robot]] + S.rank[c.robot] : c.n;
                const bool apart = tr < c.n && !(c.last && a.nbr_out);
                const int items = c.n - (apart ? 1 : 0);
                for (int k = threadIdx.x / G; k < items; k += groups)
                    agent_update_group<KMAX, G>(a, ap, S, c, (apart && k >= tr) ? k + 1 : k, speed_acc, tally);
                if (apart && threadIdx.x == 0) {
                    const float4 me = S.spv[tr];
                    ++tally.agent_steps;
                    integrate(a, S, c, c.robot, me, S.par[c.robot].x, make_float2(me.z, me.w), speed_acc);
                }
            }
            __syncthreads();
            if (a.coop_fallback == 2) {
                // deferred fallbacks, one lane each, spread over the warps
                // (queue entry q on warp q % warps, lane q / warps) so that no
                // warp runs several of them one after the other
                const int warps = blockDim.x >> 5;
                const int q = (threadIdx.x & 31) * warps + (threadIdx.x >> 5);
                if (q < min(s_fb_count, fbq.cap)) {
                    const FbEntry f = S.fb[q];
                    Line scratch[KMAX + kMaxObstacleLines];
                    const float2 v = lp_fallback(S.fb_lines + (size_t)q * S.lmax, f.n, f.n_hard, f.vmax, f.pref, scratch);
                    integrate(a, S, c, f.agent, f.me, S.par[f.agent].x, v, speed_acc);
                }
                __syncthreads();
            }
            // cooperative fallbacks; agents that found the queue full run
            // again, round after round, until every fallback went through it
            for (int round = 0; round <= c.n && a.coop_fallback == 1; ++round) {
                const int n_queued = min(s_fb_count, fbq.cap);
                const int n_pend = s_pend;
                if (n_queued) run_fallbacks(a, S, c, n_queued, speed_acc);
                __syncthreads();
                if (n_pend == 0) break;
                if (threadIdx.x == 0) {
                    s_fb_count = 0;
                    s_pend = 0;
                }
                __syncthreads();
                Tally redo;  // the work of a rerun is not counted twice
                for (int t = threadIdx.x; t < c.n; t += blockDim.x) {
                    if (!S.pend[t]) continue;
                    const bool def = agent_update<KMAX>(a, ap, S, c, t, speed_acc, redo, fbq, false);
                    S.pend[t] = def ? 1 : 0;
                    if (def) atomicAdd(&s_pend, 1);
                }
                __syncthreads();
            }
            float4* tmp = S.pv;
            S.pv = S.nv;
            S.nv = tmp;
            if (a.work) {  // the 32-bit tallies cover one step
                flush_tally(tally, a.work);
                tally = Tally{};
            }
        }
        __syncthreads();
        for (int i = threadIdx.x; i < c.n; i += blockDim.x) a.state[c.base + i] = S.pv[i];
        if (a.work) flush_tally(tally, a.work);
        if (a.stats) {
            if (ca) atomicAdd(&s_ca, ca);
            if (cs) atomicAdd(&s_cs, cs);
            if (speed_acc != 0.0) atomicAdd(&s_speed, speed_acc);
            __syncthreads();
            if (threadIdx.x == 0) {
                EnvStats* st = a.stats + c.e;
                st->agent_collisions += s_ca;
                st->segment_collisions += s_cs;
                st->speed_sum += s_speed;
                st->steps += (unsigned long long)n_steps;
            }
        }
        __syncthreads();
    }
}

template <int KMAX, int G>
cudaError_t launch_k(const ResidentArgs& a, int grid, int block, cudaStream_t stream) {
    const size_t smem = smem_layout(a.max_agents, KMAX, block / 32, nullptr, nullptr);
    cudaError_t err = cudaFuncSetAttribute(resident_kernel<KMAX, G>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)smem);
    if (err != cudaSuccess) return err;
    resident_kernel<KMAX, G><<<grid, block, smem, stream>>>(a);
    return cudaGetLastError();
}

template <int KMAX, int G>
int ctas_k(int max_agents, int block) {
    const size_t smem = smem_layout(max_agents, KMAX, block / 32, nullptr, nullptr);
    if (cudaFuncSetAttribute(resident_kernel<KMAX, G>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
        return 0;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, resident_kernel<KMAX, G>, block, smem) != cudaSuccess)
        return 0;
    return n;
}

// Launch / occupancy for lanes-per-agent G, one K instantiation each.
template <int G>
cudaError_t launch_lanes(const ResidentArgs& a, int grid, int block, cudaStream_t stream) {
    switch (resident_kmax(a.K)) {
        case 8: return launch_k<8, G>(a, grid, block, stream);
        case 10: return launch_k<10, G>(a, grid, block, stream);
        case 16: return launch_k<16, G>(a, grid, block, stream);
        default: return launch_k<32, G>(a, grid, block, stream);
    }
}

template <int G>
int ctas_lanes(int max_agents, int block, int K) {
    switch (resident_kmax(K)) {
        case 8: return ctas_k<8, G>(max_agents, block);
        case 10: return ctas_k<10, G>(max_agents, block);
        case 16: return ctas_k<16, G>(max_agents, block);
        default: return ctas_k<32, G>(max_agents, block);
    }
}


}  // namespace
}  // namespace crowd
