// One agent's crowd update (steps A2-A6), shared by the kernels.
//
// The kernels differ only in where candidates and neighbour states live
// (shared memory for an environment resident in one CTA, global memory for
// large environments); they pass that in as small accessor objects:
//   Src    (candidates, in cell order):
//            int2 row(yy, xa, xb)   sorted-slot range of cells xa..xb of row yy
//            float4 cand(u)         (px, py, vx, vy) of sorted slot u
//            int cand_id(u)         environment-local index of sorted slot u
//   Agents (neighbour lookup by environment-local index):
//            float4 state(j)        (px, py, vx, vy), robot velocity = command
//            float radius(j)
#pragma once

#include <cuda_runtime.h>

#include "crowd_internal.h"
#include "orca_device.cuh"
#include "philox.cuh"

namespace crowd {

// Agents whose LP was infeasible, queued with their lines for the
// warp-cooperative fallback (see coop_fallback).
struct FbEntry {
    int agent;     // environment-local index
    int n, n_hard; // lines, of which the first n_hard are static segments
    float vmax;
    float2 pref;
    float4 me;     // step-start state
};
struct FbQueue {
    int* count;
    int cap, lmax;
    FbEntry* entries;
    Line* pool;      // cap x lmax lines
    bool in_place;   // a full queue sends the agent to the in-place fallback (else it runs again)
    __device__ __forceinline__ bool push(const Line* L, int n, int n_hard, float vmax, float2 pref, int agent,
                                         float4 me) const {
        const int slot = atomicAdd(count, 1);
        if (slot >= cap) return false;
        Line* dst = pool + (size_t)slot * lmax;
        for (int k = 0; k < n; ++k) dst[k] = L[k];
        entries[slot] = FbEntry{agent, n, n_hard, vmax, pref, me};
        return true;
    }
};

// Goal queues: agent g walks to queue[g][0], queue[g][1], ... and moves on to
// its next goal at the start of a step in which its position lies within its
// radius of the current goal, (g - p)^2 <= r^2, decided exactly as an FP64
// evaluation of the FP32 inputs decides it (exact differences and squares,
// one rounding of the sum): FP32 settles it unless d^2 is within 1e-5 of r^2
// relative, where the FP32 error (< 1e-6 relative) could flip it.
__device__ __forceinline__ bool goal_reached(float px, float py, float gx, float gy, float r) {
    const float dx = gx - px, dy = gy - py;
    const float d2 = dx * dx + dy * dy, r2 = r * r;
    if (fabsf(d2 - r2) > 1e-5f * r2) return d2 < r2;
    const double ex = __dsub_rn((double)gx, (double)px), ey = __dsub_rn((double)gy, (double)py);
    const double dr = (double)r;
    return __dadd_rn(__dmul_rn(ex, ex), __dmul_rn(ey, ey)) <= __dmul_rn(dr, dr);
}

// Advance agent g (global index, environment e) past a reached goal; returns
// its goal.  With a pool the next goal is drawn: with k the draws so far,
// u = Philox4x32-10(counter (g, k, 0, 0), key seed), point floor(u0 n / 2^32)
// of the environment's n points.
__device__ __forceinline__ float2 advance_goal(const GoalQueue& gq, int g, int e, float4 p, float r, float2 cur) {
    if (!gq.active() || !goal_reached(p.x, p.y, cur.x, cur.y, r)) return cur;
    const int k = gq.idx[g];
    if (gq.pool_start) {
        const int b = gq.pool_start[e], n = gq.pool_start[e + 1] - b;
        if (n <= 0) return cur;
        const uint4 u = philox4x32_10(make_uint4((unsigned)g, (unsigned)k, 0u, 0u), gq.seed);
        gq.idx[g] = k + 1;
        return gq.pool[b + (int)(((unsigned long long)u.x * (unsigned long long)n) >> 32)];
    }
    if (!gq.cyclic && k + 1 >= gq.q) return cur;  // stays at its last goal
    gq.idx[g] = k + 1;
    return gq.queue[(size_t)g * gq.q + (gq.cyclic ? (k + 1) % gq.q : k + 1)];
}

// Per-thread work tallies (only reported when counting is on).  32-bit: ten
// 64-bit counters live through the whole update held 20 registers and made
// the persistent tiled update spill more (16 x 20,000 crowd 2.7 % slower).
// A thread's counts cover one step: a tiled launch is one step, and the
// shared-memory kernel flushes them after every step when counting, so a
// count would need over 4e9 items of one kind in one step of one thread
// (tens of millions of agents at one point) to wrap.
struct Tally {
    unsigned agent_steps = 0, candidates = 0, agent_lines = 0, obstacle_lines = 0, segment_tests = 0,
             lp_checks = 0, lp_solves = 0, lp_solve_lines = 0, fallbacks = 0, pairs_in_range = 0;
};

template <int KMAX>
struct NbList {
    int id[KMAX];
    int cnt;
};

// Parameters of the step shared by all agents.
struct AgentParams {
    float R, dt, tau, tau_o, robot_alpha;
    int K;
    const float4* segs;  // segments of all environments
    int* err;            // device error word
    int seg_vd;          // 1: velocity-dependent segment half-planes (obstacle_line_vd)
};

// Velocity-dependent mode: segment s gets no line when an earlier segment
// line (one that leaves 0 allowed) forbids both end disks of its cutoff
// capsule, (X - q).n + r/tau_o <= 1e-5 for X = (a - p)/tau_o, (b - p)/tau_o:
// its whole velocity obstacle already lies in that line's forbidden
// half-plane.  At a convex corner this drops the second edge, whose line
// would nearly coincide with the first one's.  The agent must be clear of s.
__device__ __forceinline__ bool segment_covered(float px, float py, float r, float4 s, float tau_o, const Line* L,
                                                int m) {
    float cx, cy;
    if (!(seg_dist2(px, py, s, cx, cy) > r * r)) return false;
    const float a0 = (s.x - px) / tau_o, a1 = (s.y - py) / tau_o, b0 = (s.z - px) / tau_o, b1 = (s.w - py) / tau_o;
    const float rt = r / tau_o;
    for (int l = 0; l < m; ++l) {
        const Line ll = L[l];
        if (-(ll.qx * ll.nx + ll.qy * ll.ny) < -1e-5f) continue;  // 0 not allowed
        const float va = (a0 - ll.qx) * ll.nx + (a1 - ll.qy) * ll.ny + rt;
        const float vb = (b0 - ll.qx) * ll.nx + (b1 - ll.qy) * ll.ny + rt;
        if (va <= 1e-5f && vb <= 1e-5f) return true;
    }
    return false;
}

// Squared distance from p to segment s as the definition evaluates it in
// FP64 (projection parameter clamped to [0, 1], closest point, squared
// distance; every operation rounded separately).
__device__ __forceinline__ double seg_dist2_fp64(float px, float py, float4 s) {
    const double ex = __dsub_rn((double)s.z, (double)s.x), ey = __dsub_rn((double)s.w, (double)s.y);
    const double dx = __dsub_rn((double)px, (double)s.x), dy = __dsub_rn((double)py, (double)s.y);
    double t = __ddiv_rn(__dadd_rn(__dmul_rn(dx, ex), __dmul_rn(dy, ey)), __dadd_rn(__dmul_rn(ex, ex), __dmul_rn(ey, ey)));
    t = t < 0.0 ? 0.0 : (t > 1.0 ? 1.0 : t);
    const double cx = __dadd_rn((double)s.x, __dmul_rn(t, ex)), cy = __dadd_rn((double)s.y, __dmul_rn(t, ey));
    const double qx = __dsub_rn((double)px, cx), qy = __dsub_rn((double)py, cy);
    return __dadd_rn(__dmul_rn(qx, qx), __dmul_rn(qy, qy));
}

// With the covered rule the order of the segment lines matters, so runs of
// FP32 keys within 1e-5 relative of their neighbour are ranked again by
// (FP64 squared distance, id), the definition's order.
static __device__ __noinline__ void repair_segment_order(float px, float py, const float4* segs, const float* okey,
                                                         int* oid, int n) {
    int s = 0;
    while (s < n) {
        int e = s;
        while (e + 1 < n && okey[e + 1] - okey[e] <= 1e-5f * okey[e + 1]) ++e;
        if (e > s) {
            double kk[kMaxObstacleLines];
            for (int q = s; q <= e; ++q) kk[q] = seg_dist2_fp64(px, py, __ldg(&segs[oid[q]]));
            for (int q = s + 1; q <= e; ++q)
                for (int z = q; z > s && (kk[z] < kk[z - 1] || (kk[z] == kk[z - 1] && oid[z] < oid[z - 1])); --z) {
                    const double tk = kk[z];
                    kk[z] = kk[z - 1];
                    kk[z - 1] = tk;
                    const int ti = oid[z];
                    oid[z] = oid[z - 1];
                    oid[z - 1] = ti;
                }
        }
        s = e + 1;
    }
}

// A4 line of one segment, in the mode of the step.
__device__ __forceinline__ Line segment_line(const AgentParams& a, float4 me, float4 pr, float4 sg) {
    return a.seg_vd ? obstacle_line_vd(me.x, me.y, me.z, me.w, pr.x, pr.y, sg, a.tau_o, a.dt)
                    : obstacle_line(me.x, me.y, me.z, me.w, pr.x, pr.y, sg, a.tau_o, a.dt);
}

// Distance from p to the bounding box of a segment, squared (a cheap lower
// bound of the segment distance used to skip far segments).
__device__ __forceinline__ float box_dist2(float px, float py, float4 s) {
    const float dx = fmaxf(fmaxf(fminf(s.x, s.z) - px, px - fmaxf(s.x, s.z)), 0.f);
    const float dy = fmaxf(fmaxf(fminf(s.y, s.w) - py, py - fmaxf(s.y, s.w)), 0.f);
    return dx * dx + dy * dy;
}

// Rows of the (2 span + 1)^2 block round cell (cx, cy) of a W x H grid,
// nearest first: the agent's row, then the rows 1, 2, ... above and below it
// (cy, cy - 1, cy + 1, cy - 2, ...), each as one run of cells cx - span ..
// cx + span (contiguous in cell order, hence in sorted slots); every cell of
// the block comes exactly once.
struct RowWalk {
    int cx, cy, W, H, span, k;
    __device__ __forceinline__ RowWalk(int cx_, int cy_, int W_, int H_, int span_)
        : cx(cx_), cy(cy_), W(W_), H(H_), span(span_), k(0) {}
    __device__ __forceinline__ bool next(int& row, int& c0, int& c1) {
        while (k <= 2 * span) {
            const int off = (k & 1) ? -((k + 1) >> 1) : (k >> 1);
            ++k;
            const int y = cy + off;
            if (y < 0 || y >= H) continue;
            row = y;
            c0 = max(cx - span, 0);
            c1 = min(cx + span, W - 1);
            return true;
        }
        return false;
    }
};

// Placement of a uniform grid: an agent at (x, y) lies in cell
// (clamp(floor((x - x0) inv_c)), clamp(floor((y - y0) inv_c))).
struct CellGeom {
    float x0, y0, inv_c;
};

// Smallest squared distance from the agent at (mx, my), in cell (cx, cy), to
// a point of cells c0..c1 of row `row`, from the cell edges facing it less
// `margin` (which covers the FP32 rounding of the edges against the clamped
// floor map that placed the agents).  A border cell also holds the agents
// clamped into it from outside the grid, which lie beyond its outer edge,
// away from an agent inside, so the edge facing the agent still bounds them.
__device__ __forceinline__ float run_dist2(const CellGeom& g, float c, float margin, float mx, float my, int cx,
                                           int cy, int row, int c0, int c1) {
    float gx = 0.f, gy = 0.f;
    if (row < cy) gy = my - fmaf((float)(row + 1), c, g.y0);
    else if (row > cy) gy = fmaf((float)row, c, g.y0) - my;
    if (c1 < cx) gx = mx - fmaf((float)(c1 + 1), c, g.x0);
    else if (c0 > cx) gx = fmaf((float)c0, c, g.x0) - mx;
    gx = fmaxf(gx - margin, 0.f);
    gy = fmaxf(gy - margin, 0.f);
    return gx * gx + gy * gy;
}

// A2: the K nearest agents within R of agent `self` (in cell (cx, cy) of a
// W x H grid with cell size >= R / span, so that every neighbour lies within
// `span` cells), ordered by (FP64 key, index) exactly as the definition
// ranks them.
//
// Candidates are ranked by their FP32 squared distance, kept with their slot
// in the candidate source (TopKSplit: the index is loaded only for the K
// kept, and for candidates at distance 0, which may be the agent itself).
// FP32 and FP64 keys further apart than kKeyRelErr order alike, so
// the FP32 order is exact except inside runs of consecutive keys closer than
// that ("near ties"); such runs among the first K + 1 are re-sorted by
// (FP64 key, index), computed for their members only.  A run that reaches the
// end of a full list may continue past it: then the block of cells is
// rescanned with FP64 keys.  Candidates within kKeyRelErr of R^2 are admitted
// by their FP64 key.  The list keeps KMAX + 2 >= K + 2 entries.
template <int KMAX, bool NEAR_FIRST, class Src>
__device__ __forceinline__ void select_neighbors(const Src& src, const CellGeom& geom, int cx, int cy, int W, int H,
                                                 int self, float4 me, float R, int K, NbList<KMAX>& out, Tally& w,
                                                 int span, bool counting) {
    constexpr int CAP = KMAX + 2;
    const float R2 = R * R;
    const float R2hi = R2 * (1.f + kKeyRelErr), R2lo = R2 * (1.f - kKeyRelErr);
    const double Rd = (double)R;
    const unsigned long long R2bits = (unsigned long long)__double_as_longlong(__dmul_rn(Rd, Rd));
    const double xi = (double)me.x, yi = (double)me.y;
    const int xa = max(cx - span, 0), xb = min(cx + span, W - 1);
    const int ya = max(cy - span, 0), yb = min(cy + span, H - 1);
    // keys and slots in two 32-bit arrays (fewer integer operations per
    // insertion than the packed 64-bit list: dense crowd 8 %, uneven batch
    // and urban block 4-5 % faster)
    TopKSplit<CAP> top;
    top.init();
    // candidate o at sorted slot cu: ranked when within R (FP64 key near R^2)
    auto consider = [&](const float4& o, int cu) {
        const float dx = o.x - me.x, dy = o.y - me.y;
        const float d2 = dx * dx + dy * dy;
        if (d2 < R2hi) {
            if (d2 == 0.f && src.cand_id(cu) == self) return;
            if (d2 > R2lo && !(rank_key(xi, yi, o.x, o.y) < R2bits)) return;
            ++w.pairs_in_range;
            top.put(d2, cu);
        }
    };
    unsigned long long ncand = 0;
    if constexpr (NEAR_FIRST) {
        // The rows of the block are walked nearest first (the agent's row,
        // then outwards), as one sequence (a warp then iterates as often as
        // its longest sequence), and the next candidate is loaded while this
        // one is ranked.  Near candidates fill the list early; once it is
        // full, a row all of whose points lie farther than its last key is
        // skipped, as none of its candidates could enter the list.  The kept
        // set, the K + 2 smallest (key, slot), does not depend on the order.
        // (Dense crowds: 42 % fewer candidates; sparse ones, whose lists
        // seldom fill, pay for the row bookkeeping, so the shared-memory
        // kernel keeps the plain row order.)
        RowWalk walk(cx, cy, W, H, span);
        const float csz = 1.f / geom.inv_c;
        const float margin = 1e-3f * csz + 1e-6f * (fabsf(geom.x0) + fabsf(geom.y0) + fabsf(me.x) + fabsf(me.y));
        int row = cy, c0 = cx, c1 = cx;
        int u = 0, end = 0;
        while (u == end && walk.next(row, c0, c1)) {
            const int2 rg = src.row(row, c0, c1);
            u = rg.x;
            end = rg.y;
            ncand += (unsigned long long)(end - u);
        }
        float4 nxt = u < end ? src.cand(u) : make_float4(0.f, 0.f, 0.f, 0.f);
        while (u < end) {
            const float4 o = nxt;
            const int cu = u;
            if (++u == end) {
                while (u == end && walk.next(row, c0, c1)) {
                    if (top.cnt == CAP &&
                        run_dist2(geom, csz, margin, me.x, me.y, cx, cy, row, c0, c1) > top.key(CAP - 1)) {
                        // counting work: the pairs within R of a skipped row
                        // are still counted, so that the count is the
                        // definition's (every pair within R), not the search's
                        if (counting) {
                            const int2 rg = src.row(row, c0, c1);
                            for (int q = rg.x; q < rg.y; ++q) {
                                const float4 oq = src.cand(q);
                                const float dx = oq.x - me.x, dy = oq.y - me.y;
                                const float d2 = dx * dx + dy * dy;
                                if (d2 < R2hi && !(d2 == 0.f && src.cand_id(q) == self) &&
                                    !(d2 > R2lo && !(rank_key(xi, yi, oq.x, oq.y) < R2bits)))
                                    ++w.pairs_in_range;
                            }
                        }
                        continue;
                    }
                    const int2 rg = src.row(row, c0, c1);
                    u = rg.x;
                    end = rg.y;
                    ncand += (unsigned long long)(end - u);
                }
            }
            if (u < end) nxt = src.cand(u);
            consider(o, cu);
        }
    } else {
        // the rows of the cell block are walked bottom to top as one sequence
        // (a warp then iterates as often as its longest sequence, not its
        // longest row per row), and the next candidate is loaded while this
        // one is ranked
        int yy = ya;
        int2 r = src.row(yy, xa, xb);
        ncand = (unsigned long long)(r.y - r.x);
        while (r.x == r.y && yy < yb) {
            r = src.row(++yy, xa, xb);
            ncand += (unsigned long long)(r.y - r.x);
        }
        int u = r.x, end = r.y;
        float4 nxt = u < end ? src.cand(u) : make_float4(0.f, 0.f, 0.f, 0.f);
        while (u < end) {
            const float4 o = nxt;
            const int cu = u;
            if (++u == end && yy < yb) {
                do {
                    r = src.row(++yy, xa, xb);
                    ncand += (unsigned long long)(r.y - r.x);
                } while (r.x == r.y && yy < yb);
                u = r.x;
                end = r.y;
            }
            if (u < end) nxt = src.cand(u);
            consider(o, cu);
        }
    }
    w.candidates += (unsigned)ncand;
    const int cnt = top.cnt;
    // tie[s]: keys s and s + 1 are near-equal (s + 1 < cnt)
    bool any_tie = false;
    unsigned tie = 0u;
#pragma unroll
    for (int s = 0; s + 1 < CAP; ++s) {
        if (s + 1 < cnt && s < K) {
            const float ka = top.key(s), kb = top.key(s + 1);
            if (kb - ka <= kKeyRelErr * kb) {
                tie |= 1u << s;
                any_tie = true;
            }
        }
    }
    if (!any_tie) {
        out.cnt = min(cnt, K);
#pragma unroll
        for (int s = 0; s < KMAX; ++s) out.id[s] = s < out.cnt ? src.cand_id(top.slot(s)) : -1;
        return;
    }
    // extend the run through position K - 1 to its end
    int e = min(cnt, K) - 1;
    if (e >= 0 && (tie >> e) & 1u) {
#pragma unroll
        for (int s = 0; s + 1 < CAP; ++s) {
            if (s >= e && s + 1 < cnt && s + 1 == e + 1) {
                const float ka = top.key(s), kb = top.key(s + 1);
                if (kb - ka <= kKeyRelErr * kb) {
                    tie |= 1u << s;
                    e = s + 1;
                }
            }
        }
    }
    if (e == CAP - 1 && cnt == CAP) {
        // the run may continue past the list: rescan with FP64 keys
        TopK64<KMAX> nb;
        nb.init();
        for (int yy = ya; yy <= yb; ++yy) {
            const int2 r = src.row(yy, xa, xb);
            for (int u = r.x; u < r.y; ++u) {
                const int j = src.cand_id(u);
                if (j == self) continue;
                const float4 o = src.cand(u);
                const unsigned long long k = rank_key(xi, yi, o.x, o.y);
                if (k < R2bits) nb.insert(k, j, K);
            }
        }
        out.cnt = nb.cnt;
#pragma unroll
        for (int s = 0; s < KMAX; ++s) out.id[s] = nb.id[s];
        return;
    }
    // positions 0..e: FP64 keys for the members of runs, then each run sorted
    // by (FP64 key, index) in place
    unsigned long long kk[CAP];
    int id[CAP];
#pragma unroll
    for (int s = 0; s < CAP; ++s) {
        kk[s] = 0ull;
        id[s] = -1;
        if (s <= e) {
            const int u = top.slot(s);
            id[s] = src.cand_id(u);
            const bool member = ((tie >> s) & 1u) || (s > 0 && ((tie >> (s - 1)) & 1u));
            if (member) {
                const float4 o = src.cand(u);
                kk[s] = rank_key(xi, yi, o.x, o.y);
            }
        }
    }
#pragma unroll 1
    for (int s = 1; s <= e; ++s) {
        if (!((tie >> (s - 1)) & 1u)) continue;
        for (int q = s; q > 0 && ((tie >> (q - 1)) & 1u) &&
                        TopK64<CAP>::less(kk[q], id[q], kk[q - 1], id[q - 1]);
             --q) {
            const unsigned long long tk = kk[q];
            kk[q] = kk[q - 1];
            kk[q - 1] = tk;
            const int ti = id[q];
            id[q] = id[q - 1];
            id[q - 1] = ti;
        }
    }
    out.cnt = min(cnt, K);
#pragma unroll
    for (int s = 0; s < KMAX; ++s) out.id[s] = s < out.cnt ? id[s] : -1;
}

// Segment candidates of an agent: all segments of its environment, or a
// precomputed per-cell list (indices relative to the environment's first
// segment, ascending).
struct AllSegments {
    int ns;
    __device__ __forceinline__ int count() const { return ns; }
    __device__ __forceinline__ int id(int q) const { return q; }
};
struct ListedSegments {
    const int* ids;
    int n;
    __device__ __forceinline__ int count() const { return n; }
    __device__ __forceinline__ int id(int q) const { return __ldg(&ids[q]); }
};

// A0, A3-A5: the new velocity of non-robot agent i (environment-local index)
// with state `me` (px, py, vx, vy), parameters `pr` (r, v_max, preferred
// speed, 0), goal `gl`, its neighbour list, and the segment candidates
// `sl` of its environment (whose first segment is seg0).
// With a queue, an infeasible LP is queued for the warp-cooperative fallback
// (`queued` set, the returned velocity meaningless); when the queue is full,
// `deferred` is set instead and the caller runs the agent again in a later
// round (so that every fallback of a queued run takes the same cooperative
// path, whatever the thread order).  Without a queue the fallback runs here.
// WARM: an infeasible LP's fallback starts where the LP failed (lp_fallback's
// warm start).  The persistent tiled update takes it (16 x 20,000 crowd 9 %
// faster, the uneven batch on that path 9 %); the shared-memory kernel, whose
// step waits for its slowest agent, ran the uneven batch 23 % slower with it
// (same results) and is compiled without it.
template <int KMAX, bool WARM, class Agents, class SegList>
__device__ __forceinline__ float2 solve_velocity(const AgentParams& a, const Agents& ag, int i, int robot, float4 me,
                                                 float4 pr, float2 gl, int seg0, const SegList& sl,
                                                 const NbList<KMAX>& nb, Tally& w, const FbQueue* fbq,
                                                 bool& queued, bool& deferred) {
    queued = false;
    deferred = false;
    const float2 pref = pref_velocity(me.x, me.y, gl.x, gl.y, pr.z, a.dt);
    Line L[KMAX + kMaxObstacleLines];

    // A4: segments within r + tau_o v_max, ordered by (distance^2, id)
    const float reach = pr.x + a.tau_o * pr.y;
    const float reach2 = reach * reach;
    float okey[kMaxObstacleLines];
    int oid[kMaxObstacleLines];
    int no = 0;
    const int ns = sl.count();
    for (int q = 0; q < ns; ++q) {
        const int s = sl.id(q);
        const float4 sg = __ldg(&a.segs[seg0 + s]);
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
    if (a.seg_vd) {
        repair_segment_order(me.x, me.y, a.segs + seg0, okey, oid, no);
        int kept = 0;
        for (int k = 0; k < no; ++k) {
            const float4 sg = __ldg(&a.segs[seg0 + oid[k]]);
            if (!segment_covered(me.x, me.y, pr.x, sg, a.tau_o, L, kept)) L[kept++] = segment_line(a, me, pr, sg);
        }
        no = kept;
    } else {
        for (int k = 0; k < no; ++k) L[k] = segment_line(a, me, pr, __ldg(&a.segs[seg0 + oid[k]]));
    }

    // A3: one reciprocal half-plane per neighbour, in list order (a rolled
    // loop: one copy of agent_line keeps the kernel's code small)
#pragma unroll 1
    for (int s = 0; s < KMAX; ++s) {
        if (s < nb.cnt) {
            const int j = nb.id[s];
            const float4 o = ag.state(j);
            // (r, v_max, preferred speed, car flag) of j in one load; all of
            // the avoidance against a car, which does not react
            const float4 pj = ag.params(j);
            const float alpha = (j == robot) ? a.robot_alpha : (pj.w != 0.f ? 1.f : 0.5f);
            L[no + s] = agent_line(me.x, me.y, me.z, me.w, pr.x, o.x, o.y, o.z, o.w, pj.x, a.tau, a.dt,
                                   alpha, i < j);
        }
    }

    // A5: LP, fallback when infeasible
    const int nl = no + nb.cnt;
    int solves = 0, solve_lines = 0;
    float2 v;
    const int fail = lp2(L, nl, pr.y, pref, v, solves, solve_lines);
    const bool feasible = fail == nl;
    if (!feasible) {
        if (fbq) queued = fbq->push(L, nl, no, pr.y, pref, i, me);
        if (fbq && !queued && !fbq->in_place) {
            deferred = true;
        } else if (!queued) {
            Line scratch[KMAX + kMaxObstacleLines];
            if constexpr (WARM) {
                // the fallback starts where the 2D LP failed, from its last
                // iterate, when every static line lies before that point
                v = lp_fallback_warm(L, nl, no, pr.y, pref, scratch, fail >= no ? fail : -1, v);
            } else {
                v = lp_fallback(L, nl, no, pr.y, pref, scratch);
            }
        }
    }
    w.agent_lines += nb.cnt;
    w.obstacle_lines += no;
    w.lp_checks += nl;
    w.lp_solves += solves;
    w.lp_solve_lines += solve_lines;
    w.fallbacks += feasible ? 0 : 1;
    return v;
}

// Warp-reduce the tallies and add them to the global counters.
__device__ __forceinline__ void flush_tally(const Tally& tally, WorkCount* work) {
    unsigned long long* dst = &work->agent_steps;
    const unsigned long long vals[10] = {tally.agent_steps, tally.candidates, tally.agent_lines,
                                         tally.obstacle_lines, tally.segment_tests, tally.lp_checks,
                                         tally.lp_solves, tally.lp_solve_lines, tally.fallbacks,
                                         tally.pairs_in_range};
#pragma unroll
    for (int q = 0; q < 10; ++q) {
        unsigned long long v = vals[q];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if ((threadIdx.x & 31) == 0 && v) atomicAdd(dst + q, v);
    }
}

}  // namespace crowd
