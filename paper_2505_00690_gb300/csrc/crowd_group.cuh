// One agent's crowd update by a group of G lanes of a warp (G = 1, 2, 4,
// 8, 16 or 32), the alternative to one thread per agent.
//
// With one thread per agent, the 32 agents of a warp take different branches
// (candidate counts, LP paths, fallbacks) and the warp runs the union of
// them; with a group of G lanes per agent the lanes of a group take the same
// branches, share the work of each agent, and only the 32/G agents of a warp
// diverge.  Work split inside a group:
//   - neighbour candidates: strided over the lanes, each keeps its own
//     top-(K+1), merged by K+1 rounds of a group minimum;
//   - half-planes: line k is built and kept by lane k % G;
//   - LP: every lane follows the same incremental solve; each 1D interval is
//     clipped by every lane against its own earlier lines and the bounds meet
//     in a group reduction; the infeasible fallback runs the same way.
// Every lane returns the same velocity.
#pragma once

#include <cuda_runtime.h>

#include "crowd_agent.cuh"
#include "orca_device.cuh"

namespace crowd {

template <int G>
struct Grp {
    int lane;       // index inside the group
    unsigned mask;  // the group's lanes in the warp
    __device__ __forceinline__ Grp() {
        lane = threadIdx.x & (G - 1);
        const unsigned base = (threadIdx.x & 31u) & ~(unsigned)(G - 1);
        mask = (G == 32) ? 0xffffffffu : (((1u << G) - 1u) << base);
    }
    __device__ __forceinline__ float bcast(float v, int src) const { return __shfl_sync(mask, v, src, G); }
    __device__ __forceinline__ float max(float v) const {
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(mask, v, o, G));
        return v;
    }
    __device__ __forceinline__ float min(float v) const {
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) v = fminf(v, __shfl_xor_sync(mask, v, o, G));
        return v;
    }
    __device__ __forceinline__ unsigned long long min(unsigned long long v) const {
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) {
            const unsigned long long w = __shfl_xor_sync(mask, v, o, G);
            v = w < v ? w : v;
        }
        return v;
    }
    __device__ __forceinline__ bool any(bool p) const { return (__ballot_sync(mask, p) & mask) != 0u; }
};

// Line k of a group's line set, held by lane k % G at slot k / G.
template <int G>
__device__ __forceinline__ Line group_line(const Grp<G>& g, const Line* mine, int k) {
    const int owner = k & (G - 1);
    Line l{};
    if (g.lane == owner) l = mine[k / G];
    l.qx = g.bcast(l.qx, owner);
    l.qy = g.bcast(l.qy, owner);
    l.nx = g.bcast(l.nx, owner);
    l.ny = g.bcast(l.ny, owner);
    return l;
}

// line_interval for a group: line k (given) against the disk and the group's
// lines 0..k-1 (each lane clips with its own); the same slack rules.
template <int G>
__device__ __forceinline__ bool group_interval(const Grp<G>& g, const Line* mine, const Line& lk, int k, float vmax,
                                               float& tl, float& tr) {
    const float dx = -lk.ny, dy = lk.nx;
    const float qd = lk.qx * dx + lk.qy * dy;
    float disc = qd * qd - (lk.qx * lk.qx + lk.qy * lk.qy) + vmax * vmax;
    if (disc < 0.f) {
        if (disc < -2.f * kIntervalSlack * vmax) return false;
        disc = 0.f;
    }
    if (disc <= kTangentDisc * vmax * vmax) disc = 0.f;
    const float sq = sqrtf(disc);
    float lo = -qd - sq, hi = -qd + sq;
    bool bad = false;
    for (int l = g.lane; l < k; l += G) {
        const Line ll = mine[l / G];
        const float den = dx * ll.nx + dy * ll.ny;
        const float num = (ll.qx - lk.qx) * ll.nx + (ll.qy - lk.qy) * ll.ny;
        if (fabsf(den) < 1e-4f) {
            bad |= clip_near_parallel(lk, ll, lo, hi);
        } else {
            const float t = num / den;
            if (den > 0.f) lo = fmaxf(lo, t);
            else hi = fminf(hi, t);
        }
    }
    lo = g.max(lo);
    hi = g.min(hi);
    if (g.any(bad)) return false;
    if (lo > hi) {
        if (lo - hi > kIntervalSlack) return false;
        lo = hi = 0.5f * (lo + hi);
    }
    tl = lo;
    tr = hi;
    return true;
}

// Incremental LP over the group's lines 0..n-1 (least distance to pref).
template <int G>
__device__ __forceinline__ int group_lp2(const Grp<G>& g, const Line* mine, int n, float vmax, float2 pref, float2& v,
                                         int& solves, int& solve_lines) {
    const float pl2 = pref.x * pref.x + pref.y * pref.y;
    if (pl2 > vmax * vmax) {
        const float k = vmax * rsqrtf(pl2);
        v = make_float2(pref.x * k, pref.y * k);
    } else {
        v = pref;
    }
    for (int k = 0; k < n; ++k) {
        const Line lk = group_line(g, mine, k);
        if ((v.x - lk.qx) * lk.nx + (v.y - lk.qy) * lk.ny < 0.f) {
            ++solves;
            solve_lines += k;
            float tl, tr;
            if (!group_interval(g, mine, lk, k, vmax, tl, tr)) return k;
            const float dx = -lk.ny, dy = lk.nx;
            float t = (pref.x - lk.qx) * dx + (pref.y - lk.qy) * dy;
            t = fminf(fmaxf(t, tl), tr);
            v = make_float2(lk.qx + t * dx, lk.qy + t * dy);
        }
    }
    return n;
}

// Directional LP (maximise v.o) over the group's lines 0..m-1.
template <int G>
__device__ __forceinline__ bool group_lp_dir(const Grp<G>& g, const Line* mine, int m, float vmax, float ox, float oy,
                                             float2 pref, float2& v) {
    v = make_float2(vmax * ox, vmax * oy);
    for (int k = 0; k < m; ++k) {
        const Line lk = group_line(g, mine, k);
        if ((v.x - lk.qx) * lk.nx + (v.y - lk.qy) * lk.ny < 0.f) {
            float tl, tr;
            if (!group_interval(g, mine, lk, k, vmax, tl, tr)) return false;
            const float dx = -lk.ny, dy = lk.nx;
            const float dd = dx * ox + dy * oy;
            float t;
            if (dd > 1e-6f) t = tr;
            else if (dd < -1e-6f) t = tl;
            else t = fminf(fmaxf((pref.x - lk.qx) * dx + (pref.y - lk.qy) * dy, tl), tr);
            v = make_float2(lk.qx + t * dx, lk.qy + t * dy);
        }
    }
    return true;
}

// lp_fallback for a group: `mine` holds the group's lines, `sub` (same
// layout) the subproblem lines; a same-direction pair gives an inert line.
template <int G>
__device__ __forceinline__ float2 group_fallback(const Grp<G>& g, const Line* mine, Line* sub, int n, int n_hard,
                                                 float vmax, float2 pref) {
    float2 v;
    int solves = 0, solve_lines = 0;
    if (group_lp2(g, mine, n_hard, vmax, pref, v, solves, solve_lines) < n_hard) {
        n_hard = 0;
        const float pl2 = pref.x * pref.x + pref.y * pref.y;
        const float k = pl2 > vmax * vmax ? vmax * rsqrtf(pl2) : 1.f;
        v = make_float2(pref.x * k, pref.y * k);
    }
    float dist = -INFINITY;
    for (int i = n_hard; i < n; ++i) {
        const Line li = group_line(g, mine, i);
        const float viol = -((v.x - li.qx) * li.nx + (v.y - li.qy) * li.ny);
        if (viol > dist) {
            const float ci = li.qx * li.nx + li.qy * li.ny;
            for (int m = g.lane; m < i; m += G) {
                const Line lj = mine[m / G];
                if (m < n_hard) {
                    sub[m / G] = lj;
                } else {
                    float nx = lj.nx - li.nx, ny = lj.ny - li.ny;
                    const float nl2 = nx * nx + ny * ny;
                    if (nl2 < 1e-12f) {
                        sub[m / G] = Line{0.f, 0.f, 0.f, 0.f};
                    } else {
                        const float inv = rsqrtf(nl2);
                        nx *= inv;
                        ny *= inv;
                        const float c = ((lj.qx * lj.nx + lj.qy * lj.ny) - ci) * inv;
                        sub[m / G] = Line{c * nx, c * ny, nx, ny};
                    }
                }
            }
            float2 t;
            if (group_lp_dir(g, sub, i, vmax, li.nx, li.ny, pref, t)) v = t;
            dist = -((v.x - li.qx) * li.nx + (v.y - li.qy) * li.ny);
        }
    }
    return v;
}

// A2 for a group: candidates strided over the lanes, each lane's top-(K+1)
// merged by K+1 rounds of a group minimum (keys are unique: index in the low
// bits).  The near-tie rescan with FP64 keys runs redundantly in every lane.
template <int KMAX, int G, class Src>
__device__ __forceinline__ void group_select(const Grp<G>& g, const Src& src, int cx, int cy, int W, int H, int self,
                                             float4 me, float R, int K, NbList<KMAX>& out, Tally& w, int span) {
    const float R2 = R * R;
    const float R2hi = R2 * (1.f + kKeyRelErr), R2lo = R2 * (1.f - kKeyRelErr);
    const double Rd = (double)R;
    const unsigned long long R2bits = (unsigned long long)__double_as_longlong(__dmul_rn(Rd, Rd));
    const double xi = (double)me.x, yi = (double)me.y;
    const int xa = max(cx - span, 0), xb = min(cx + span, W - 1);
    const int ya = max(cy - span, 0), yb = min(cy + span, H - 1);
    TopK32<KMAX + 1> top;
    top.init();
    for (int yy = ya; yy <= yb; ++yy) {
        const int2 r = src.row(yy, xa, xb);
        if (g.lane == 0) w.candidates += (unsigned)(r.y - r.x);
        for (int u = r.x + g.lane; u < r.y; u += G) {
            const float4 o = src.cand(u);
            const float dx = o.x - me.x, dy = o.y - me.y;
            const float d2 = dx * dx + dy * dy;
            if (d2 < R2hi) {
                const int j = src.cand_id(u);
                if (j == self) continue;
                if (d2 > R2lo && !(rank_key(xi, yi, o.x, o.y) < R2bits)) continue;
                ++w.pairs_in_range;
                top.insert(((unsigned long long)__float_as_uint(d2) << 32) | (unsigned)j);
            }
        }
    }
    // merge: round s takes the smallest head of all lanes
    unsigned long long merged[KMAX + 1];
#pragma unroll
    for (int s = 0; s <= KMAX; ++s) {
        const unsigned long long m = g.min(top.e[0]);
        merged[s] = m;
        if (top.e[0] == m && m != ~0ull) {
#pragma unroll
            for (int q = 0; q < KMAX; ++q) top.e[q] = top.e[q + 1];
            top.e[KMAX] = ~0ull;
        }
    }
    int cnt = 0;
#pragma unroll
    for (int s = 0; s <= KMAX; ++s) cnt += merged[s] != ~0ull ? 1 : 0;
    bool near_tie = false;
#pragma unroll
    for (int s = 0; s < KMAX; ++s) {
        if (s < K && s + 1 < cnt) {
            const float ka = __uint_as_float((unsigned)(merged[s] >> 32));
            const float kb = __uint_as_float((unsigned)(merged[s + 1] >> 32));
            if (kb - ka <= kKeyRelErr * kb) near_tie = true;
        }
    }
    if (!near_tie) {
        out.cnt = min(cnt, K);
#pragma unroll
        for (int s = 0; s < KMAX; ++s) out.id[s] = (int)(unsigned)(merged[s] & 0xffffffffull);
        return;
    }
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
}

// A0, A3-A5 for a group (non-robot agent); every lane returns the velocity.
template <int KMAX, int G, class Agents, class SegList>
__device__ __forceinline__ float2 group_solve(const Grp<G>& g, const AgentParams& a, const Agents& ag, int i, int robot,
                                              float4 me, float4 pr, float2 gl, int seg0, const SegList& sl,
                                              const NbList<KMAX>& nb, Tally& w) {
    constexpr int kSlots = (KMAX + kMaxObstacleLines + G - 1) / G;
    const float2 pref = pref_velocity(me.x, me.y, gl.x, gl.y, pr.z, a.dt);
    Line mine[kSlots];

    // A4: segments within reach, ordered by (distance^2, id); every lane scans
    // the (short) cell list, lane k % G builds line k
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
        if (g.lane == 0) ++w.segment_tests;
        float qx, qy;
        const float d2 = seg_dist2(me.x, me.y, sg, qx, qy);
        if (!(d2 < reach2)) continue;
        if (no == kMaxObstacleLines) {
            if (g.lane == 0) atomicOr(a.err, kErrObstacleOverflow);
            if (!(d2 < okey[no - 1])) continue;
            --no;
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
        // the kept set depends on the lines before it: every lane builds all
        // of them, then keeps its share
        repair_segment_order(me.x, me.y, a.segs + seg0, okey, oid, no);
        Line all[kMaxObstacleLines];
        int kept = 0;
        for (int k = 0; k < no; ++k) {
            const float4 sg = __ldg(&a.segs[seg0 + oid[k]]);
            if (!segment_covered(me.x, me.y, pr.x, sg, a.tau_o, all, kept)) all[kept++] = segment_line(a, me, pr, sg);
        }
        no = kept;
        for (int k = g.lane; k < no; k += G) mine[k / G] = all[k];
    } else {
        for (int k = g.lane; k < no; k += G)
            mine[k / G] = segment_line(a, me, pr, __ldg(&a.segs[seg0 + oid[k]]));
    }

    // A3: agent line s is global line no + s
#pragma unroll
    for (int s = 0; s < KMAX; ++s) {
        if (s < nb.cnt && ((no + s) & (G - 1)) == g.lane) {
            const int j = nb.id[s];
            const float4 o = ag.state(j);
            // all of the avoidance against a vehicle, which does not react
            const float alpha = (j == robot) ? a.robot_alpha : (ag.vehicle(j) ? 1.f : 0.5f);
            mine[(no + s) / G] = agent_line(me.x, me.y, me.z, me.w, pr.x, o.x, o.y, o.z, o.w, ag.radius(j), a.tau,
                                            a.dt, alpha, i < j);
        }
    }
    __syncwarp(g.mask);

    // A5
    const int nl = no + nb.cnt;
    int solves = 0, solve_lines = 0;
    float2 v;
    const bool feasible = group_lp2(g, mine, nl, pr.y, pref, v, solves, solve_lines) == nl;
    if (!feasible) {
        Line sub[kSlots];
        v = group_fallback(g, mine, sub, nl, no, pr.y, pref);
    }
    if (g.lane == 0) {
        w.agent_lines += nb.cnt;
        w.obstacle_lines += no;
        w.lp_checks += nl;
        w.lp_solves += solves;
        w.lp_solve_lines += solve_lines;
        w.fallbacks += feasible ? 0 : 1;
    }
    return v;
}

}  // namespace crowd
