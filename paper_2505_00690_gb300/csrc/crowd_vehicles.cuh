// Lane-following vehicles under the Intelligent Driver Model (Treiber,
// Hennecke and Helbing, 2000), shared by the resident and the tiled kernels:
// the point of a lane at an arc position, the corridor test for crowd agents
// blocking a lane, one IDM step of a car, and the commit of a car's step.
#pragma once

#include <cuda_runtime.h>
#include <math.h>

#include "crowd_internal.h"

namespace crowd {

// Point of lane l (closed polyline) at arc position s.
__device__ __forceinline__ float2 lane_point(const VehicleArgs& V, int l, float s) {
    const int p0 = V.lane_start[l], m = V.lane_start[l + 1] - p0;
    const float* cum = V.cum + p0 + l;
    int k = 0;
    while (k + 1 < m && cum[k + 1] <= s) ++k;
    const float2 a = V.pts[p0 + k], b = V.pts[p0 + (k + 1 == m ? 0 : k + 1)];
    const float t = (s - cum[k]) / (cum[k + 1] - cum[k]);
    return make_float2(a.x + t * (b.x - a.x), a.y + t * (b.y - a.y));
}

// Whether a crowd agent at q (radius r) lies within half_width + r of the
// lane segment from a along e (length ln), and its arc position there.
// Near the corridor's edge the distance is taken again in FP64, as the
// definition evaluates it.
__device__ __forceinline__ bool lane_blocker(float2 q, float r, float2 a, float2 e, float ln, float c0,
                                             float half_width, float& s_at) {
    const float dx = q.x - a.x, dy = q.y - a.y;
    const float t = fminf(fmaxf((dx * e.x + dy * e.y) / (ln * ln), 0.f), 1.f);
    const float cx = a.x + t * e.x, cy = a.y + t * e.y;
    const float lat = sqrtf((q.x - cx) * (q.x - cx) + (q.y - cy) * (q.y - cy));
    const float thr = half_width + r;
    bool in = lat <= thr;
    if (fabsf(lat - thr) <= 1e-4f * thr) {
        const double ex = e.x, ey = e.y, l2 = (double)ln * (double)ln;
        const double ddx = (double)q.x - (double)a.x, ddy = (double)q.y - (double)a.y;
        double td = (ddx * ex + ddy * ey) / l2;
        td = td < 0.0 ? 0.0 : (td > 1.0 ? 1.0 : td);
        const double ox = (double)q.x - ((double)a.x + td * ex), oy = (double)q.y - ((double)a.y + td * ey);
        in = sqrt(ox * ox + oy * oy) <= (double)half_width + (double)r;
    }
    s_at = c0 + t * ln;
    return in;
}

// IDM step of vehicle vi of an environment (crowd agents [0, n)): the
// nearest thing ahead on its lane, a car of the lane or a crowd agent within
// the lane's corridor and `lookahead`, sets the interaction term of
// a (1 - (v/v0)^4 - (s*/gap)^2), s* = s0 + max(0, v T + v dv / (2 sqrt(a b)));
// v' = max(0, v + acc dt), s' = s + v' dt wrapped onto the lane.
// `ag` gives the environment's crowd agents k in [0, n): ag.par(k), ag.pv(k).
template <class Agents>
__device__ __forceinline__ void idm_vehicle(const VehicleArgs& V, int vi, int v_begin, int v_end, const Agents& ag,
                                            int n, float dt, float& s_new, float& v_new) {
    const int l = V.lane[vi];
    const int p0 = V.lane_start[l], m = V.lane_start[l + 1] - p0;
    const float* cum = V.cum + p0 + l;
    const float L = cum[m];
    const float s = V.s[vi], v = V.v[vi];
    const float4 pa = V.par_a[vi];
    const float2 pb = V.par_b[vi];
    float best = INFINITY, gap = 0.f, dv = 0.f;
    bool has = false;
    for (int j = v_begin; j < v_end; ++j) {
        if (j == vi || V.lane[j] != l) continue;
        float ds = V.s[j] - s;
        if (ds <= 0.f) ds += L;
        if (ds < best) {
            best = ds;
            gap = ds - 0.5f * (pb.y + V.par_b[j].y);
            dv = v - V.v[j];
            has = true;
        }
    }
    for (int k = 0; k < n; ++k) {
        const float4 pk = ag.par(k);
        if (pk.w != 0.f) continue;  // cars are leaders through their lane only
        const float4 q = ag.pv(k);
        for (int seg = 0; seg < m; ++seg) {
            const float2 a = V.pts[p0 + seg], b = V.pts[p0 + (seg + 1 == m ? 0 : seg + 1)];
            const float2 e = make_float2(b.x - a.x, b.y - a.y);
            float s_at;
            if (!lane_blocker(make_float2(q.x, q.y), pk.x, a, e, cum[seg + 1] - cum[seg], cum[seg], V.half_width,
                              s_at))
                continue;
            float ds = s_at - s;
            if (ds <= 0.f) ds += L;
            if (ds <= V.lookahead && ds < best) {
                best = ds;
                gap = ds - 0.5f * pb.y - pk.x;
                dv = v;
                has = true;
            }
        }
    }
    const float vr = v / pa.x;
    const float vr2 = vr * vr;
    const float free_term = 1.f - vr2 * vr2;
    float acc;
    if (has) {
        const float star = pb.x + fmaxf(0.f, v * pa.y + v * dv / (2.f * sqrtf(pa.z * pa.w)));
        const float q = star / fmaxf(gap, 0.01f);
        acc = pa.z * (free_term - q * q);
    } else {
        acc = pa.z * free_term;
    }
    v_new = fmaxf(0.f, v + acc * dt);
    s_new = s + v_new * dt;
    if (s_new >= L) s_new -= L;
}

// Commit the step of car vi: its arc state, and its agent row (position p(s),
// velocity (p(s') - p(s)) / dt).
__device__ __forceinline__ void place_vehicle(const VehicleArgs& V, int vi, float s_new, float v_new, float dt,
                                                  float4* row) {
    const int l = V.lane[vi];
    const float2 p_now = lane_point(V, l, V.s[vi]), p_next = lane_point(V, l, s_new);
    V.s[vi] = s_new;
    V.v[vi] = v_new;
    const float inv_dt = 1.f / dt;
    *row = make_float4(p_now.x, p_now.y, (p_next.x - p_now.x) * inv_dt, (p_next.y - p_now.y) * inv_dt);
}

// The nearest point of car vi's lane ahead of it, within `lookahead`, at
// which a crowd agent at q (radius r) blocks the lane: the smallest arc
// distance over the lane's segments whose corridor holds the agent; false
// when there is none.
__device__ __forceinline__ bool agent_ahead(const VehicleArgs& V, int vi, float2 q, float r, float& ds_min) {
    const int l = V.lane[vi];
    const int p0 = V.lane_start[l], m = V.lane_start[l + 1] - p0;
    const float* cum = V.cum + p0 + l;
    const float L = cum[m], s = V.s[vi];
    bool any = false;
    ds_min = INFINITY;
    for (int seg = 0; seg < m; ++seg) {
        const float2 a = V.pts[p0 + seg], b = V.pts[p0 + (seg + 1 == m ? 0 : seg + 1)];
        const float2 e = make_float2(b.x - a.x, b.y - a.y);
        float s_at;
        if (!lane_blocker(q, r, a, e, cum[seg + 1] - cum[seg], cum[seg], V.half_width, s_at)) continue;
        float ds = s_at - s;
        if (ds <= 0.f) ds += L;
        if (ds <= V.lookahead && ds < ds_min) {
            ds_min = ds;
            any = true;
        }
    }
    return any;
}

// IDM step of car vi when the nearest blocking crowd agent ahead is known
// (agent_ds, radius agent_r; agent_ds infinite when none blocks): the
// nearest car of the lane ahead first, replaced by the agent when the agent
// is strictly nearer, as idm_vehicle's scan (cars, then agents) decides.
__device__ __forceinline__ void idm_with_blocker(const VehicleArgs& V, int vi, int v_begin, int v_end,
                                                 float agent_ds, float agent_r, float dt, float& s_new,
                                                 float& v_new) {
    const int l = V.lane[vi];
    const int p0 = V.lane_start[l], m = V.lane_start[l + 1] - p0;
    const float L = V.cum[p0 + l + m];
    const float s = V.s[vi], v = V.v[vi];
    const float4 pa = V.par_a[vi];
    const float2 pb = V.par_b[vi];
    float best = INFINITY, gap = 0.f, dv = 0.f;
    bool has = false;
    for (int j = v_begin; j < v_end; ++j) {
        if (j == vi || V.lane[j] != l) continue;
        float ds = V.s[j] - s;
        if (ds <= 0.f) ds += L;
        if (ds < best) {
            best = ds;
            gap = ds - 0.5f * (pb.y + V.par_b[j].y);
            dv = v - V.v[j];
            has = true;
        }
    }
    if (agent_ds < best) {
        gap = agent_ds - 0.5f * pb.y - agent_r;
        dv = v;
        has = true;
    }
    const float vr = v / pa.x;
    const float vr2 = vr * vr;
    const float free_term = 1.f - vr2 * vr2;
    float acc;
    if (has) {
        const float star = pb.x + fmaxf(0.f, v * pa.y + v * dv / (2.f * sqrtf(pa.z * pa.w)));
        const float q = star / fmaxf(gap, 0.01f);
        acc = pa.z * (free_term - q * q);
    } else {
        acc = pa.z * free_term;
    }
    v_new = fmaxf(0.f, v + acc * dt);
    s_new = s + v_new * dt;
    if (s_new >= L) s_new -= L;
}

}  // namespace crowd
