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
};

__host__ __device__ inline int round_up4(int n) { return (n + 3) & ~3; }

__host__ __device__ inline size_t smem_layout(int max_agents, Smem* s, unsigned char* base) {
    const int nm = round_up4(max_agents > 0 ? max_agents : 1);
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

// Block-wide bounding box -> grid with cell size >= R (times a margin that
// covers FP32 rounding of the cell coordinate), at most kGridMax per side.
__device__ __forceinline__ void build_grid(const Smem& S, int n, float R, float* red, Grid* g) {
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
        const float c = fmaxf(R * 1.0001f, ext / (float)(kGridMax - 1));
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

// Distance from p to the bounding box of a segment, squared (a cheap lower
// bound of the segment distance used to skip far segments).
__device__ __forceinline__ float box_dist2(float px, float py, float4 s) {
    const float dx = fmaxf(fmaxf(fminf(s.x, s.z) - px, px - fmaxf(s.x, s.z)), 0.f);
    const float dy = fmaxf(fmaxf(fminf(s.y, s.w) - py, py - fmaxf(s.y, s.w)), 0.f);
    return dx * dx + dy * dy;
}

// Per-thread work tallies (only kept when counting is on).
struct Tally {
    unsigned long long agent_steps = 0, candidates = 0, agent_lines = 0, obstacle_lines = 0, segment_tests = 0,
                       lp_checks = 0, lp_solves = 0, lp_solve_lines = 0, fallbacks = 0;
};

struct StepCtx {
    int e, base, n, robot, seg0, ns;
    int step;        // 0-based step inside this launch
    bool last;       // last step of the launch
    Grid g;
};

template <int KMAX>
struct NbList {
    int id[KMAX];
    int cnt;
};

// K nearest agents within R of the agent in sorted slot t, ordered by
// (FP64 key, index) exactly as the definition ranks them.  Candidates are
// ranked by their FP32 squared distance (packed with the index into one
// 64-bit key); FP32 and FP64 keys further apart than kKeyRelErr order alike,
// so the FP32 order is exact unless two of the first K+1 keys are closer than
// that, in which case the block is rescanned with FP64 keys.  Candidates
// within kKeyRelErr of R^2 are admitted by their FP64 key.
template <int KMAX>
__device__ __forceinline__ void select_neighbors(const Smem& S, const StepCtx& c, int t, float4 me, float R, int K,
                                                 NbList<KMAX>& out, Tally& w) {
    const float R2 = R * R;
    const float R2hi = R2 * (1.f + kKeyRelErr), R2lo = R2 * (1.f - kKeyRelErr);
    const double Rd = (double)R;
    const unsigned long long R2bits = (unsigned long long)__double_as_longlong(__dmul_rn(Rd, Rd));
    const double xi = (double)me.x, yi = (double)me.y;
    const int cx = cell_coord(me.x, c.g.x0, c.g.inv_c, c.g.W);
    const int cy = cell_coord(me.y, c.g.y0, c.g.inv_c, c.g.H);
    const int xa = max(cx - 1, 0), xb = min(cx + 1, c.g.W - 1);
    const int ya = max(cy - 1, 0), yb = min(cy + 1, c.g.H - 1);
    TopK32<KMAX + 1> top;
    top.init();
    for (int yy = ya; yy <= yb; ++yy) {
        const int b0 = S.cell[yy * c.g.W + xa], b1 = S.cell[yy * c.g.W + xb + 1];
        w.candidates += (unsigned long long)(b1 - b0);
        for (int u = b0; u < b1; ++u) {
            const float4 o = S.spv[u];
            const float dx = o.x - me.x, dy = o.y - me.y;
            const float d2 = dx * dx + dy * dy;
            if (d2 < R2hi && u != t) {
                if (d2 > R2lo && !(rank_key(xi, yi, o.x, o.y) < R2bits)) continue;
                top.insert(((unsigned long long)__float_as_uint(d2) << 32) | (unsigned)S.sid[u], K + 1);
            }
        }
    }
    bool near_tie = false;
#pragma unroll
    for (int s = 0; s < KMAX; ++s) {
        if (s < K && s + 1 < top.cnt) {
            const float ka = TopK32<KMAX + 1>::key_of(top.e[s]), kb = TopK32<KMAX + 1>::key_of(top.e[s + 1]);
            if (kb - ka <= kKeyRelErr * kb) near_tie = true;
        }
    }
    if (!near_tie) {
        out.cnt = min(top.cnt, K);
#pragma unroll
        for (int s = 0; s < KMAX; ++s) out.id[s] = (int)(unsigned)(top.e[s] & 0xffffffffull);
        return;
    }
    TopK64<KMAX> nb;
    nb.init();
    for (int yy = ya; yy <= yb; ++yy) {
        const int b0 = S.cell[yy * c.g.W + xa], b1 = S.cell[yy * c.g.W + xb + 1];
        for (int u = b0; u < b1; ++u) {
            if (u == t) continue;
            const float4 o = S.spv[u];
            const unsigned long long k = rank_key(xi, yi, o.x, o.y);
            if (k < R2bits) nb.insert(k, S.sid[u], K);
        }
    }
    out.cnt = nb.cnt;
#pragma unroll
    for (int s = 0; s < KMAX; ++s) out.id[s] = nb.id[s];
}

template <int KMAX>
__device__ __forceinline__ void agent_update(const ResidentArgs& a, const Smem& S, const StepCtx& c, int t,
                                             double& speed_acc, Tally& w) {
    const int i = S.sid[t];
    const float4 me = S.spv[t];
    const float4 pr = S.par[i];

    // ---- A1/A2: K nearest within R, ranked by (FP64 key, index)
    NbList<KMAX> nb;
    select_neighbors<KMAX>(S, c, t, me, a.R, a.K, nb, w);
    const int K = a.K;
    if (c.last && a.nbr_out) {
        int* out = a.nbr_out + (size_t)(c.base + i) * K;
#pragma unroll
        for (int s = 0; s < KMAX; ++s)
            if (s < K) out[s] = s < nb.cnt ? nb.id[s] : -1;
    }

    float2 v;
    if (i == c.robot) {
        v = make_float2(me.z, me.w);  // commanded, not solved
    } else {
        const float2 gl = S.goal[i];
        const float2 pref = pref_velocity(me.x, me.y, gl.x, gl.y, pr.z, a.dt);
        Line L[KMAX + kMaxObstacleLines];

        // ---- A4: segments within r + tau_o v_max, ordered by (distance^2, id)
        const float reach = pr.x + a.tau_o * pr.y;
        const float reach2 = reach * reach;
        float okey[kMaxObstacleLines];
        int oid[kMaxObstacleLines];
        int no = 0;
        for (int s = 0; s < c.ns; ++s) {
            const float4 sg = __ldg(&a.segs[c.seg0 + s]);
            if (box_dist2(me.x, me.y, sg) >= reach2) continue;
            ++w.segment_tests;
            float qx, qy;
            const float d2 = seg_dist2(me.x, me.y, sg, qx, qy);
            if (!(d2 < reach2)) continue;
            if (no == kMaxObstacleLines) {
                atomicOr(a.err, kErrObstacleOverflow);
                if (!(d2 < okey[no - 1])) continue;
                --no;  // drop the farthest
            }
            int p = no;
            while (p > 0 && okey[p - 1] > d2) {
                okey[p] = okey[p - 1];
                oid[p] = oid[p - 1];
                --p;
            }
            okey[p] = d2;
            oid[p] = s;
            ++no;
        }
        for (int k = 0; k < no; ++k)
            L[k] = obstacle_line(me.x, me.y, me.z, me.w, pr.x, pr.y, __ldg(&a.segs[c.seg0 + oid[k]]), a.tau_o,
                                 a.dt);

        // ---- A3: one reciprocal half-plane per neighbour, in list order
#pragma unroll
        for (int s = 0; s < KMAX; ++s) {
            if (s < nb.cnt) {
                const int j = nb.id[s];
                const float4 o = S.pv[j];
                const float alpha = (j == c.robot) ? a.robot_alpha : 0.5f;
                L[no + s] = agent_line(me.x, me.y, me.z, me.w, pr.x, o.x, o.y, o.z, o.w, S.par[j].x, a.tau, a.dt,
                                       alpha, i < j);
            }
        }

        // ---- A5: LP, fallback when infeasible
        const int nl = no + nb.cnt;
        int solves = 0, solve_lines = 0;
        const bool feasible = lp2(L, nl, pr.y, pref, v, solves, solve_lines) == nl;
        if (!feasible) {
            Line scratch[KMAX + kMaxObstacleLines];
            v = lp_fallback(L, nl, no, pr.y, pref, scratch);
        }
        w.agent_lines += nb.cnt;
        w.obstacle_lines += no;
        w.lp_checks += nl;
        w.lp_solves += solves;
        w.lp_solve_lines += solve_lines;
        w.fallbacks += feasible ? 0 : 1;
    }
    ++w.agent_steps;

    // ---- A6: integrate into the next-state buffer
    float4 nx;
    nx.x = fmaf(a.dt, v.x, me.x);
    nx.y = fmaf(a.dt, v.y, me.y);
    nx.z = v.x;
    nx.w = v.y;
    S.nv[i] = nx;
    if (a.stats && i != c.robot) {
        speed_acc += (double)sqrtf(v.x * v.x + v.y * v.y);
        if (a.reach) {
            int* rp = a.reach + c.base + i;
            const float2 gl = S.goal[i];
            const float gx = gl.x - nx.x, gy = gl.y - nx.y;
            if (*rp < 0 && sqrtf(gx * gx + gy * gy) <= pr.x) *rp = (int)(a.step_base + c.step + 1);
        }
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
    const int xa = max(cx - 1, 0), xb = min(cx + 1, c.g.W - 1);
    for (int yy = max(cy - 1, 0); yy <= min(cy + 1, c.g.H - 1); ++yy) {
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
    for (int s = 0; s < c.ns; ++s) {
        const float4 sg = __ldg(&a.segs[c.seg0 + s]);
        if (box_dist2(me.x, me.y, sg) >= lim * lim) continue;
        float qx, qy;
        if (sqrtf(seg_dist2(me.x, me.y, sg, qx, qy)) < lim) ++cs;
    }
}

template <int KMAX>
__global__ void __launch_bounds__(kMaxThreads) resident_kernel(ResidentArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ float red[4 * kMaxWarps];
    __shared__ Grid grid;
    __shared__ int s_work;
    __shared__ unsigned long long s_ca, s_cs;
    __shared__ double s_speed;
    Smem S;
    smem_layout(a.max_agents, &S, smem_raw);

    for (;;) {
        if (threadIdx.x == 0) s_work = atomicAdd(a.queue, 1);
        __syncthreads();
        const int w = s_work;
        if (w >= a.n_work) break;
        StepCtx c;
        c.e = a.order[w];
        c.base = a.env_start[c.e];
        c.n = a.env_start[c.e + 1] - c.base;
        c.robot = a.robot_index[c.e];
        c.seg0 = a.seg_start[c.e];
        c.ns = a.seg_start[c.e + 1] - c.seg0;
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
        const int passes = a.n_steps + (a.stats ? 1 : 0);
        for (int step = 0; step < passes; ++step) {
            const bool compute = step < a.n_steps;
            if (compute && c.robot >= 0 && c.robot < c.n && a.robot_vel && threadIdx.x == 0) {
                const float2 cmd = __ldg(&a.robot_vel[(size_t)step * a.robot_stride + c.e]);
                S.pv[c.robot].z = cmd.x;
                S.pv[c.robot].w = cmd.y;
            }
            __syncthreads();
            build_grid(S, c.n, a.R, red, &grid);
            c.g = grid;
            sort_by_cell(S, c.n, c.g);
            c.step = step;
            c.last = step == a.n_steps - 1;
            if (a.stats && step > 0)
                for (int t = threadIdx.x; t < c.n; t += blockDim.x) count_collisions(a, S, c, t, ca, cs);
            if (!compute) break;
            for (int t = threadIdx.x; t < c.n; t += blockDim.x) agent_update<KMAX>(a, S, c, t, speed_acc, tally);
            __syncthreads();
            float4* tmp = S.pv;
            S.pv = S.nv;
            S.nv = tmp;
        }
        __syncthreads();
        for (int i = threadIdx.x; i < c.n; i += blockDim.x) a.state[c.base + i] = S.pv[i];
        if (a.work) {
            unsigned long long* dst = &a.work->agent_steps;
            const unsigned long long vals[9] = {tally.agent_steps, tally.candidates, tally.agent_lines,
                                                tally.obstacle_lines, tally.segment_tests, tally.lp_checks,
                                                tally.lp_solves, tally.lp_solve_lines, tally.fallbacks};
#pragma unroll
            for (int q = 0; q < 9; ++q) {
                unsigned long long v = vals[q];
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                if ((threadIdx.x & 31) == 0 && v) atomicAdd(dst + q, v);
            }
        }
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
                st->steps += (unsigned long long)a.n_steps;
            }
        }
        __syncthreads();
    }
}

template <int KMAX>
cudaError_t launch_k(const ResidentArgs& a, int grid, int block, cudaStream_t stream) {
    const size_t smem = resident_smem_bytes(a.max_agents);
    cudaError_t err = cudaFuncSetAttribute(resident_kernel<KMAX>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)smem);
    if (err != cudaSuccess) return err;
    resident_kernel<KMAX><<<grid, block, smem, stream>>>(a);
    return cudaGetLastError();
}

template <int KMAX>
int ctas_k(int max_agents, int block) {
    const size_t smem = resident_smem_bytes(max_agents);
    if (cudaFuncSetAttribute(resident_kernel<KMAX>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
        return 0;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, resident_kernel<KMAX>, block, smem) != cudaSuccess) return 0;
    return n;
}

}  // namespace

size_t resident_smem_bytes(int max_agents) { return smem_layout(max_agents, nullptr, nullptr); }

int resident_block_threads(int max_agents) {
    int b = ((max_agents + 31) / 32) * 32;
    return b < 64 ? 64 : (b > kMaxThreads ? kMaxThreads : b);
}

int resident_kmax(int K) { return K <= 8 ? 8 : (K <= 16 ? 16 : 32); }

cudaError_t launch_resident(const ResidentArgs& a, int grid, int block, cudaStream_t stream) {
    switch (resident_kmax(a.K)) {
        case 8: return launch_k<8>(a, grid, block, stream);
        case 16: return launch_k<16>(a, grid, block, stream);
        default: return launch_k<32>(a, grid, block, stream);
    }
}

int resident_ctas_per_sm(int max_agents, int block, int K) {
    switch (resident_kmax(K)) {
        case 8: return ctas_k<8>(max_agents, block);
        case 16: return ctas_k<16>(max_agents, block);
        default: return ctas_k<32>(max_agents, block);
    }
}

}  // namespace crowd
