// Tiled crowd step for environments too large to live in one CTA.
//
// The paper's simulator advances every dynamic agent of every environment
// each step (Sec. 3.2); a city-scale scene (Appendix "Data") holds far more
// agents than one SM's shared memory.  For such environments one step is
// four kernels over global memory:
//   tiled_count    robot command, cell key (static per-environment grid with
//                  cells >= R / span, span 1 or 2) and rank inside the cell
//                  (atomic count);
//   tiled_scan     one CTA per environment turns the counts into cell starts
//                  (block scan) and clears the counts for the next step;
//   tiled_scatter  writes the state in cell order;
//   tiled_update   one CTA per (environment, tile of tx x ty cells, sized on
//                  the host so that a tile's agents fill one round of threads):
//                  stages the tile's halo cells (already contiguous in cell
//                  order) into shared memory, then each thread takes the
//                  tile's agents: K nearest from the staged halo, segment
//                  half-planes from the cell's precomputed segment list,
//                  agent half-planes, LP, integration into the other buffer.
// Multi-step calls replay these launches from a CUDA graph (captured by the
// host side).  Agents outside the grid are clamped into the border cells,
// which keeps the (2 span + 1)^2-cell search exact (clamping onto a box is
// non-expansive).
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>

#include "../../include/crowd.h"
#include "crowd_agent.cuh"
#include "crowd_internal.h"
#include "crowd_vehicles.cuh"
#include "orca_device.cuh"

namespace crowd {

namespace {

constexpr int kCountThreads = 256;
constexpr int kScanThreads = 1024;
constexpr int kUpdateThreads = kTiledUpdateThreads;

__device__ __forceinline__ int clamp_cell(float v, float v0, float inv_c, int n) {
    const int c = __float2int_rd((v - v0) * inv_c);
    return min(max(c, 0), n - 1);
}

__device__ __forceinline__ int cell_of(const TiledEnv& te, float x, float y) {
    return clamp_cell(y, te.y0, te.inv_c, te.H) * te.W + clamp_cell(x, te.x0, te.inv_c, te.W);
}

__global__ void __launch_bounds__(kCountThreads) tiled_count(TiledStepArgs a) {
    const TiledEnv te = a.envs[blockIdx.y];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= te.n) return;
    const int g = te.base + i;
    float4 p = a.state_in[g];
    const bool car = __ldg(&a.par[g]).w != 0.f;
    if (a.mode != kTiledStatsOnly && a.ep.steps && episode_restart(a.ep.steps[te.e], *a.step_index, a.ep.origin)) {
        // episodes: the environment starts over (the host counted the
        // statistics of the episode's last state before this step); a car's
        // row was placed from its restored arc by tiled_vehicles already
        if (!car) {
            p = a.ep.state[g];
            a.state_in[g] = p;
        }
        a.goal[g] = a.ep.goal[g];
        if (a.ep.gidx) a.goals.idx[g] = a.ep.gidx[g];
    }
    if (i == te.robot && a.robot_vel) {
        const float2 cmd = __ldg(&a.robot_vel[te.e]);
        p.z = cmd.x;
        p.w = cmd.y;
        a.state_in[g] = p;
    }
    if (a.goals.active() && i != te.robot && !car && a.mode != kTiledStatsOnly) {
        const float2 cur = a.goal[g];
        const float2 nx = advance_goal(a.goals, g, te.e, p, __ldg(&a.par[g]).x, cur);
        if (nx.x != cur.x || nx.y != cur.y) a.goal[g] = nx;
    }
    const int k = cell_of(te, p.x, p.y);
    a.key[g] = k;
    a.rank[g] = atomicAdd(&a.count[te.co + k], 1);
}

// Exclusive scan of one environment's cell counts into global sorted slots;
// start[co + W*H] closes the last cell.  Counts are cleared for the next step.
__global__ void __launch_bounds__(kScanThreads) tiled_scan(TiledStepArgs a) {
    __shared__ int warp_sum[kScanThreads / 32];
    __shared__ int carry;
    const TiledEnv te = a.envs[blockIdx.x];
    const int C = te.W * te.H;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) carry = te.base;
    if (blockIdx.x == 0 && threadIdx.x == 0 && a.queue) *a.queue = 0;  // work items of this step's update
    __syncthreads();
    for (int c0 = 0; c0 < C; c0 += blockDim.x) {
        const int c = c0 + threadIdx.x;
        const int v = c < C ? a.count[te.co + c] : 0;
        int incl = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        if (lane == 31) warp_sum[warp] = incl;
        __syncthreads();
        if (warp == 0) {
            const int nw = blockDim.x >> 5;
            int ws = lane < nw ? warp_sum[lane] : 0;
            int wincl = ws;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, wincl, o);
                if (lane >= o) wincl += y;
            }
            if (lane < nw) warp_sum[lane] = wincl - ws;  // exclusive warp offsets
        }
        __syncthreads();
        const int base = carry;
        if (c < C) {
            a.start[te.co + c] = base + warp_sum[warp] + incl - v;
            a.count[te.co + c] = 0;
        }
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry = base + warp_sum[warp] + incl;
        __syncthreads();
    }
    if (threadIdx.x == 0) a.start[te.co + C] = carry;
    if (a.item_order) {
        // this environment's work items into the dispatch order, by the cost
        // class each took in the previous step (classes in order, the items
        // of a class in any order)
        __shared__ int s_off[kItemBuckets];
        if (threadIdx.x == 0) {
            int o = 0;
            for (int b = 0; b < kItemBuckets; ++b) {
                s_off[b] = o;
                o += a.sched->count[b];
            }
        }
        __syncthreads();
        const int i1 = a.item_start[blockIdx.x + 1];
        for (int i = a.item_start[blockIdx.x] + threadIdx.x; i < i1; i += blockDim.x) {
            const int b = a.item_bucket[i];
            a.item_order[s_off[b] + atomicAdd(&a.sched->cursor[b], 1)] = i;
        }
    }
}

__global__ void __launch_bounds__(kCountThreads) tiled_scatter(TiledStepArgs a) {
    const TiledEnv te = a.envs[blockIdx.y];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= te.n) return;
    const int g = te.base + i;
    const int slot = a.start[te.co + a.key[g]] + a.rank[g];
    a.sorted_pv[slot] = a.state_in[g];
    a.sorted_id[slot] = i;
}

// Candidates of the tile's halo staged in shared memory.  Global sorted
// slots of halo row r (cells hx0..hx1) start at row_slot[r] and sit at
// smem offset row_off[r].
struct HaloSource {
    const float4* pv;
    const int* id;
    const int* start;  // global cell starts of the environment (start + co)
    const int* row_slot;
    const int* row_off;
    int W, hy0;
    __device__ __forceinline__ int2 row(int yy, int xa, int xb) const {
        const int r = yy - hy0;
        const int d = row_off[r] - row_slot[r];
        return make_int2(start[yy * W + xa] + d, start[yy * W + xb + 1] + d);
    }
    __device__ __forceinline__ float4 cand(int u) const { return pv[u]; }
    __device__ __forceinline__ int cand_id(int u) const { return id[u]; }
};

// Candidates read straight from the global sorted arrays (halo too large).
struct GlobalSource {
    const float4* pv;
    const int* id;
    const int* start;
    int W;
    __device__ __forceinline__ int2 row(int yy, int xa, int xb) const {
        return make_int2(start[yy * W + xa], start[yy * W + xb + 1]);
    }
    __device__ __forceinline__ float4 cand(int u) const { return pv[u]; }
    __device__ __forceinline__ int cand_id(int u) const { return id[u]; }
};

// Neighbour states by environment-local index from the step's input buffer.
struct GlobalAgents {
    const float4* pv;
    const float4* par;
    __device__ __forceinline__ float4 state(int j) const { return pv[j]; }
    __device__ __forceinline__ float4 params(int j) const { return __ldg(&par[j]); }
};

// INSTR: compiled with the statistics and work-count code (false: a launch
// with neither, whose work tallies are then dead code, so that the plain
// step holds no registers for them).
template <int KMAX, class Src, bool INSTR = true>
__device__ __forceinline__ void tile_agent(const TiledStepArgs& a, const AgentParams& ap, const TiledEnv& te,
                                           const Src& src, int slot, Tally& w, unsigned long long& ca,
                                           unsigned long long& cs, double& speed) {
    const int i = a.sorted_id[slot];
    const float4 me = a.sorted_pv[slot];
    const int g = te.base + i;
    const float4 pr = __ldg(&a.par[g]);
    const int k = cell_of(te, me.x, me.y);
    const int cx = k % te.W, cy = k / te.W;

    if (INSTR && a.mode != kTiledStep) {
        // collision events of the input state (the previous step's result)
        const int xa = max(cx - 1, 0), xb = min(cx + 1, te.W - 1);
        for (int yy = max(cy - 1, 0); yy <= min(cy + 1, te.H - 1); ++yy) {
            const int2 r = src.row(yy, xa, xb);
            for (int u = r.x; u < r.y; ++u) {
                const int j = src.cand_id(u);
                if (j <= i) continue;
                const float4 o = src.cand(u);
                const float dx = o.x - me.x, dy = o.y - me.y;
                if (sqrtf(dx * dx + dy * dy) < pr.x + __ldg(&a.par[te.base + j]).x - kCollideDepth) ++ca;
            }
        }
        const float lim = pr.x - kCollideDepth;
        const int s0 = a.seg_cell_start[te.co + k], s1 = a.seg_cell_start[te.co + k + 1];
        for (int q = s0; q < s1; ++q) {
            const float4 sg = __ldg(&a.segs[te.seg0 + a.seg_cell_ids[q]]);
            if (box_dist2(me.x, me.y, sg) >= lim * lim) continue;
            float qx, qy;
            if (sqrtf(seg_dist2(me.x, me.y, sg, qx, qy)) < lim) ++cs;
        }
        if (a.mode == kTiledStatsOnly) return;
    }

    NbList<KMAX> nb;
    select_neighbors<KMAX, true>(src, CellGeom{te.x0, te.y0, te.inv_c}, cx, cy, te.W, te.H, i, me, ap.R, ap.K, nb, w,
                           te.span, INSTR && a.work != nullptr);
    if (a.nbr_out) {
        int* out = a.nbr_out + (size_t)g * ap.K;
#pragma unroll
        for (int s = 0; s < KMAX; ++s)
            if (s < ap.K) out[s] = s < nb.cnt ? nb.id[s] : -1;
    }
    float2 v;
    if (i == te.robot || pr.w != 0.f) {  // the robot and the cars move as commanded
        v = make_float2(me.z, me.w);
    } else {
        // segment candidates: the cell's precomputed list
        const int s0 = a.seg_cell_start[te.co + k], s1 = a.seg_cell_start[te.co + k + 1];
        bool queued, deferred;
        v = solve_velocity<KMAX, true>(ap, GlobalAgents{a.state_in + te.base, a.par + te.base}, i, te.robot, me, pr,
                                 __ldg(&a.goal[g]), te.seg0, ListedSegments{a.seg_cell_ids + s0, s1 - s0}, nb, w,
                                 nullptr, queued, deferred);
    }
    ++w.agent_steps;
    float4 nx;
    nx.x = fmaf(ap.dt, v.x, me.x);
    nx.y = fmaf(ap.dt, v.y, me.y);
    nx.z = v.x;
    nx.w = v.y;
    a.state_out[g] = nx;
    if (INSTR && a.stats && i != te.robot && pr.w == 0.f) {
        speed += (double)sqrtf(v.x * v.x + v.y * v.y);
        const float2 gl = __ldg(&a.goal[g]);
        const float gx = gl.x - nx.x, gy = gl.y - nx.y;
        if (a.reach[g] < 0 && sqrtf(gx * gx + gy * gy) <= pr.x) a.reach[g] = (int)(*a.step_index + 1);
    }
}

template <int KMAX>
__global__ void __launch_bounds__(kUpdateThreads) tiled_update(TiledStepArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int s_row_slot[kTileMax + 2 * kTiledSpanMax], s_row_off[kTileMax + 2 * kTiledSpanMax],
        s_row_cnt[kTileMax + 2 * kTiledSpanMax];
    __shared__ int s_tile_row_slot[kTileMax], s_tile_row_cnt[kTileMax];
    __shared__ int s_total, s_tile_total;
    __shared__ unsigned long long s_ca, s_cs;
    __shared__ double s_speed;
    const TiledEnv te = a.envs[blockIdx.y];
    const int tile = blockIdx.x;
    const int tiles_x = (te.W + te.tx - 1) / te.tx, tiles_y = (te.H + te.ty - 1) / te.ty;
    if (tile >= tiles_x * tiles_y) return;
    const int tx0 = (tile % tiles_x) * te.tx, ty0 = (tile / tiles_x) * te.ty;
    const int tx1 = min(tx0 + te.tx, te.W) - 1, ty1 = min(ty0 + te.ty, te.H) - 1;
    const int hx0 = max(tx0 - te.span, 0), hx1 = min(tx1 + te.span, te.W - 1);
    const int hy0 = max(ty0 - te.span, 0), hy1 = min(ty1 + te.span, te.H - 1);
    const int* start = a.start + te.co;
    float4* s_pv = (float4*)smem_raw;
    int* s_id = (int*)(s_pv + a.halo_cap);

    if (threadIdx.x == 0) {
        int off = 0;
        for (int r = 0; r <= hy1 - hy0; ++r) {
            const int yy = hy0 + r;
            const int b0 = start[yy * te.W + hx0], b1 = start[yy * te.W + hx1 + 1];
            s_row_slot[r] = b0;
            s_row_off[r] = off;
            s_row_cnt[r] = b1 - b0;
            off += b1 - b0;
        }
        s_total = off;
        int tot = 0;
        for (int r = 0; r <= ty1 - ty0; ++r) {
            const int yy = ty0 + r;
            const int b0 = start[yy * te.W + tx0], b1 = start[yy * te.W + tx1 + 1];
            s_tile_row_slot[r] = b0;
            s_tile_row_cnt[r] = b1 - b0;
            tot += b1 - b0;
        }
        s_tile_total = tot;
        s_ca = 0;
        s_cs = 0;
        s_speed = 0.0;
    }
    __syncthreads();
    const bool staged = s_total <= a.halo_cap;
    if (staged) {
        for (int r = 0; r <= hy1 - hy0; ++r) {
            const int b0 = s_row_slot[r], n = s_row_cnt[r], o = s_row_off[r];
            for (int q = threadIdx.x; q < n; q += blockDim.x) {
                s_pv[o + q] = a.sorted_pv[b0 + q];
                s_id[o + q] = a.sorted_id[b0 + q];
            }
        }
    }
    __syncthreads();

    const AgentParams ap{a.R, a.dt, a.tau, a.tau_o, a.robot_alpha, a.K, a.segs, a.err, a.seg_vd};
    Tally w;
    unsigned long long ca = 0, cs = 0;
    double speed = 0.0;
    const int total = s_tile_total;
    for (int q = threadIdx.x; q < total; q += blockDim.x) {
        int r = 0, qq = q;
        while (qq >= s_tile_row_cnt[r]) {
            qq -= s_tile_row_cnt[r];
            ++r;
        }
        const int slot = s_tile_row_slot[r] + qq;
        if (staged) {
            const HaloSource src{s_pv, s_id, start, s_row_slot, s_row_off, te.W, hy0};
            tile_agent<KMAX>(a, ap, te, src, slot, w, ca, cs, speed);
        } else {
            const GlobalSource src{a.sorted_pv, a.sorted_id, start, te.W};
            tile_agent<KMAX>(a, ap, te, src, slot, w, ca, cs, speed);
        }
    }
    if (a.work) flush_tally(w, a.work);
    if (a.stats) {
        if (ca) atomicAdd(&s_ca, ca);
        if (cs) atomicAdd(&s_cs, cs);
        if (speed != 0.0) atomicAdd(&s_speed, speed);
        __syncthreads();
        if (threadIdx.x == 0) {
            EnvStats* st = a.stats + te.e;
            if (s_ca) atomicAdd(&st->agent_collisions, s_ca);
            if (s_cs) atomicAdd(&st->segment_collisions, s_cs);
            if (s_speed != 0.0) atomicAdd(&st->speed_sum, s_speed);
        }
    }
}

// Warp sums (all lanes get the total).
__device__ __forceinline__ unsigned long long warp_sum(unsigned long long v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Persistent form of the update (one launch for every tiled environment):
// as many CTAs as fit on the GPU, and every warp takes work items from one
// counter shared by all environments, an item being kQueueItem consecutive
// sorted slots (agents in cell order) of one environment.  Candidates and
// neighbours are read from the step's global arrays through L1/L2 (an item's
// agents share most of their candidate cells).  Warps never wait for one
// another: a crowded item holds up only its own warp, where a CTA per tile
// held its whole CTA until its slowest warp was done, and environments of
// any size share the launch.  The per-agent work is tile_agent's, so the
// results are those of tiled_update bit for bit.
template <int KMAX, bool INSTR>
__global__ void __launch_bounds__(kQueueThreads, INSTR ? kQueueMinBlocks : kQueuePlainMinBlocks)
    tiled_update_queue(TiledStepArgs a) {
    const int lane = threadIdx.x & 31;
    const AgentParams ap{a.R, a.dt, a.tau, a.tau_o, a.robot_alpha, a.K, a.segs, a.err, a.seg_vd};
    __shared__ long long s_t0[kQueueThreads / 32];  // start clock of each warp's item
    Tally w;
    for (;;) {
        int item = 0;
        if (lane == 0) item = atomicAdd(a.queue, 1);
        item = __shfl_sync(0xffffffffu, item, 0);
        if (item >= a.n_items) break;
        if (a.item_order) {
            item = a.item_order[item];
            if (lane == 0) s_t0[threadIdx.x >> 5] = clock64();  // kept in shared memory, not a register
        }
        int lo = 0, hi = a.n_envs - 1;  // environment of the item
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (__ldg(&a.item_start[mid]) <= item) lo = mid;
            else hi = mid - 1;
        }
        const TiledEnv te = a.envs[lo];
        const int q = (item - __ldg(&a.item_start[lo])) * kQueueItem + lane;
        unsigned long long ca = 0, cs = 0;
        double speed = 0.0;
        if (q < te.n) {
            const GlobalSource src{a.sorted_pv, a.sorted_id, a.start + te.co, te.W};
            tile_agent<KMAX, GlobalSource, INSTR>(a, ap, te, src, te.base + q, w, ca, cs, speed);
        }
        if (a.item_order) {
            // the item's cost class for the next step's dispatch order
            __syncwarp();
            if (lane == 0) {
                const long long c = clock64() - s_t0[threadIdx.x >> 5];
                const float m = a.sched->mean, cf = (float)c;
                const int b = cf >= 2.f * m ? 0 : cf >= 1.4f * m ? 1 : cf >= m ? 2 : cf >= 0.7f * m ? 3 : 4;
                a.item_bucket[item] = (unsigned char)b;
                atomicAdd(&a.sched->count_next[b], 1);
                atomicAdd(&a.sched->cost_sum, (unsigned long long)(c > 0 ? c : 0));
            }
        }
        if (INSTR && a.stats) {
            ca = warp_sum(ca);
            cs = warp_sum(cs);
            speed = warp_sum(speed);
            if (lane == 0) {
                EnvStats* st = a.stats + te.e;
                if (ca) atomicAdd(&st->agent_collisions, ca);
                if (cs) atomicAdd(&st->segment_collisions, cs);
                if (speed != 0.0) atomicAdd(&st->speed_sum, speed);
            }
        }
    }
    if (INSTR && a.work) flush_tally(w, a.work);
}

constexpr int kVehicleThreads = 256;

// Cars of tiled environment blockIdx.x (at most CROWD_MAX_VEHICLES_PER_ENV),
// ahead of the step's other kernels.  All threads: for every (car, crowd
// agent) pair, the distance ahead on the car's lane when the agent blocks
// it, reduced per car to the smallest (distance, agent index), the order the
// sequential scan keeps, by a shared 64-bit minimum.  One thread per car:
// the IDM step from the step-start state.  Then the arcs and the cars'
// agent rows are committed.  An environment that starts over at this step
// gives its cars their snapshot arcs and shows them the snapshot's crowd
// (which tiled_count restores right after).
__global__ void __launch_bounds__(kVehicleThreads) tiled_vehicles(TiledStepArgs a) {
    __shared__ unsigned long long s_best[CROWD_MAX_VEHICLES_PER_ENV];
    const TiledEnv te = a.envs[blockIdx.x];
    const VehicleArgs V = a.veh;
    const int vb = V.start[te.e], nv = min(V.start[te.e + 1] - vb, CROWD_MAX_VEHICLES_PER_ENV);
    if (nv <= 0) return;
    const bool restart = a.ep.steps && episode_restart(a.ep.steps[te.e], *a.step_index, a.ep.origin);
    const int t = threadIdx.x;
    if (t < nv) {
        s_best[t] = ~0ull;
        if (restart && a.ep.veh_s) {
            V.s[vb + t] = a.ep.veh_s[vb + t];
            V.v[vb + t] = a.ep.veh_v[vb + t];
        }
    }
    __syncthreads();
    const float4* rows = (restart ? a.ep.state : a.state_in) + te.base;
    const float4* par = a.par + te.base;
    for (int k = t; k < te.n; k += blockDim.x) {
        const float4 pk = __ldg(&par[k]);
        if (pk.w != 0.f) continue;  // cars are leaders through their lane only
        const float4 q = rows[k];
        for (int c = 0; c < nv; ++c) {
            float ds;
            if (agent_ahead(V, vb + c, make_float2(q.x, q.y), pk.x, ds))
                atomicMin(&s_best[c], ((unsigned long long)__float_as_uint(ds) << 32) | (unsigned)k);
        }
    }
    __syncthreads();
    float s_new = 0.f, v_new = 0.f;
    if (t < nv) {
        const unsigned long long b = s_best[t];
        const bool blocked = b != ~0ull;
        const float ds = blocked ? __uint_as_float((unsigned)(b >> 32)) : INFINITY;
        const float r = blocked ? __ldg(&par[(int)(unsigned)(b & 0xFFFFFFFFull)]).x : 0.f;
        idm_with_blocker(V, vb + t, vb, vb + nv, ds, r, a.dt, s_new, v_new);
    }
    __syncthreads();
    if (t < nv) place_vehicle(V, vb + t, s_new, v_new, a.dt, a.state_in + V.agent[vb + t]);
}

__global__ void tiled_finish_step(TiledStepArgs a) {
    // one thread: count the step in the statistics and advance the step index
    if (a.stats && a.mode != kTiledStatsOnly)
        for (int k = 0; k < a.n_envs; ++k) a.stats[a.envs[k].e].steps += 1;
    if (a.mode != kTiledStatsOnly) *a.step_index += 1;
    if (a.sched) {
        // the classes of this step's items become the next step's order; the
        // counts move only when the update classed every item
        ItemSched& q = *a.sched;
        int n = 0;
        for (int b = 0; b < kItemBuckets; ++b) n += q.count_next[b];
        if (n == a.n_items) {
            q.mean = a.n_items > 0 ? (float)((double)q.cost_sum / (double)a.n_items) : 0.f;
            for (int b = 0; b < kItemBuckets; ++b) q.count[b] = q.count_next[b];
        }
        for (int b = 0; b < kItemBuckets; ++b) {
            q.count_next[b] = 0;
            q.cursor[b] = 0;
        }
        q.cost_sum = 0;
    }
}

template <int KMAX>
cudaError_t update_k(const TiledStepArgs& a, int max_tiles, cudaStream_t s) {
    if (a.use_queue) {
        const int warps = kQueueThreads / 32;
        const int need = (a.n_items + warps - 1) / warps;
        if (a.work || a.stats || a.mode != kTiledStep)
            tiled_update_queue<KMAX, true><<<std::max(1, std::min(a.queue_grid, need)), kQueueThreads, 0, s>>>(a);
        else
            tiled_update_queue<KMAX, false><<<std::max(1, std::min(a.queue_grid_plain, need)), kQueueThreads, 0, s>>>(
                a);
    } else {
        tiled_update<KMAX><<<dim3(max_tiles, a.n_envs), kUpdateThreads, tiled_smem_bytes(a.halo_cap), s>>>(a);
    }
    return cudaGetLastError();
}

template <int KMAX>
int queue_blocks(bool plain) {
    int n = 0;
    const cudaError_t e =
        plain ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, tiled_update_queue<KMAX, false>, kQueueThreads, 0)
              : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, tiled_update_queue<KMAX, true>, kQueueThreads, 0);
    return e == cudaSuccess ? n : 0;
}

}  // namespace

__global__ void set_step_kernel(long long* p, long long v) { *p = v; }

cudaError_t launch_set_step(long long* p, long long value, cudaStream_t s) {
    set_step_kernel<<<1, 1, 0, s>>>(p, value);
    return cudaGetLastError();
}

size_t tiled_smem_bytes(int halo_cap) { return (size_t)halo_cap * (sizeof(float4) + sizeof(int)); }

int tiled_queue_blocks_per_sm(int K, bool plain) {
    switch (resident_kmax(K)) {
        case 8: return queue_blocks<8>(plain);
        case 10: return queue_blocks<10>(plain);
        case 16: return queue_blocks<16>(plain);
        default: return queue_blocks<32>(plain);
    }
}

cudaError_t tiled_init(int halo_cap) {
    const int smem = (int)tiled_smem_bytes(halo_cap);
    cudaError_t e = cudaFuncSetAttribute(tiled_update<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(tiled_update<10>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(tiled_update<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(tiled_update<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    return e;
}

cudaError_t launch_tiled_step(const TiledStepArgs& a, int max_agents, int max_tiles, cudaStream_t s, int* n_kernels) {
    if (n_kernels) *n_kernels = 0;
    if (a.n_envs == 0) return cudaSuccess;
    if (n_kernels) *n_kernels = (a.veh_on && a.mode != kTiledStatsOnly) ? 6 : 5;
    const dim3 agrid((max_agents + kCountThreads - 1) / kCountThreads, a.n_envs);
    if (a.veh_on && a.mode != kTiledStatsOnly) tiled_vehicles<<<a.n_envs, kVehicleThreads, 0, s>>>(a);
    tiled_count<<<agrid, kCountThreads, 0, s>>>(a);
    tiled_scan<<<a.n_envs, kScanThreads, 0, s>>>(a);
    tiled_scatter<<<agrid, kCountThreads, 0, s>>>(a);
    cudaError_t e;
    switch (resident_kmax(a.K)) {
        case 8: e = update_k<8>(a, max_tiles, s); break;
        case 10: e = update_k<10>(a, max_tiles, s); break;
        case 16: e = update_k<16>(a, max_tiles, s); break;
        default: e = update_k<32>(a, max_tiles, s); break;
    }
    if (e != cudaSuccess) return e;
    tiled_finish_step<<<1, 1, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace crowd
