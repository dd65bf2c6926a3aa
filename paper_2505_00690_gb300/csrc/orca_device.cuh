// Per-agent device arithmetic of the ORCA crowd step (sm_103a).
//
// FP32 throughout, except where a discrete decision or an ill-conditioned
// quantity must come out as the FP64 definition says:
//   - the neighbour ranking key (squared distance rounded in FP64 with no
//     fused multiply-add), so that neighbour lists are bit-exact;
//   - the leg choice (sign of det(p, w)) and the colliding test
//     (|p|^2 <= r^2) when the FP32 value is within its rounding error of 0;
//   - the near-parallel test of two LP lines (|det| <= 1e-9) and the
//     intersection parameter when |det| is small;
//   - the infeasible-LP fallback (min-max penetration, then the point closest
//     to the preferred velocity).
// The geometry is that of ORCA (van den Berg et al., ISRR 2011), the
// collision-avoidance rule the paper uses for its dynamic agents (Sec. 3.2).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace crowd {

constexpr float kEpsGoal = 1e-6f;  // preferred velocity is 0 closer than this to the goal
constexpr double kEpsParallel = 1e-9;  // |det(n_k, n_l)| at or below: parallel lines

// Half-plane {v : (v - q) . n >= 0}, n a unit vector.
struct Line {
    float qx, qy, nx, ny;
};

// ---------------------------------------------------------------- A0 ----
// Preferred velocity toward the goal: full speed along the direction, or
// exactly onto the goal when it is within one step, or 0 once on it.
__device__ __forceinline__ float2 pref_velocity(float px, float py, float gx, float gy, float speed,
                                                float dt) {
    float dx = gx - px, dy = gy - py;
    float dist = sqrtf(dx * dx + dy * dy);
    if (dist < kEpsGoal) return make_float2(0.f, 0.f);
    if (dist <= speed * dt) return make_float2(__fdiv_rn(dx, dt), __fdiv_rn(dy, dt));
    float k = __fdiv_rn(speed, dist);
    return make_float2(k * dx, k * dy);
}

// ---------------------------------------------------------------- A2 ----
// Ranking key: ((double)xj - xi)^2 + ((double)yj - yi)^2 with every product
// and the sum rounded separately in FP64.  Non-negative, so its bit pattern
// orders like the value.
__device__ __forceinline__ unsigned long long rank_key(double xi, double yi, float xj, float yj) {
    double dx = __dsub_rn((double)xj, xi);
    double dy = __dsub_rn((double)yj, yi);
    double k = __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy));
    return (unsigned long long)__double_as_longlong(k);
}

// Sorted list of the KMAX smallest (key, id) pairs; only the first K slots
// (runtime K <= KMAX) are used.  All indices are compile-time so that the
// list lives in registers.
template <int KMAX>
struct TopK {
    unsigned long long key[KMAX];
    int id[KMAX];
    int cnt;

    __device__ __forceinline__ void init() {
        cnt = 0;
#pragma unroll
        for (int s = 0; s < KMAX; ++s) {
            key[s] = ~0ull;
            id[s] = 0x7fffffff;
        }
    }
    __device__ __forceinline__ static bool less(unsigned long long ka, int ia, unsigned long long kb, int ib) {
        return ka < kb || (ka == kb && ia < ib);
    }
    // Insert (k, j) if it ranks among the first K.
    __device__ __forceinline__ void insert(unsigned long long k, int j, int K) {
        if (K <= 0) return;
        // the last used slot holds the current K-th element (or the sentinel)
        unsigned long long lk = ~0ull;
        int li = 0x7fffffff;
#pragma unroll
        for (int s = 0; s < KMAX; ++s)
            if (s == K - 1) { lk = key[s]; li = id[s]; }
        if (!less(k, j, lk, li)) return;
        int p = 0;  // insertion position = number of entries ranking before (k, j)
#pragma unroll
        for (int s = 0; s < KMAX; ++s) p += (s < cnt && less(key[s], id[s], k, j)) ? 1 : 0;
#pragma unroll
        for (int s = KMAX - 1; s >= 1; --s) {
            if (s > p) { key[s] = key[s - 1]; id[s] = id[s - 1]; }
            else if (s == p) { key[s] = k; id[s] = j; }
        }
        if (p == 0) { key[0] = k; id[0] = j; }
        cnt = cnt < K ? cnt + 1 : K;
    }
};

// ---------------------------------------------------------------- A3 ----
// Reciprocal half-plane of agent i against agent j (current velocities):
// u = (nearest point of the boundary of the truncated velocity obstacle to
// v = v_i - v_j) - v, n = the outward normal there, line through v_i + alpha u.
__device__ __forceinline__ Line agent_line(float pix, float piy, float vix, float viy, float ri, float pjx,
                                           float pjy, float vjx, float vjy, float rj, float tau, float dt,
                                           float alpha, bool i_before_j) {
    const float px = pjx - pix, py = pjy - piy;
    const float vx = vix - vjx, vy = viy - vjy;
    const float r = ri + rj;
    const float dist2 = px * px + py * py;
    const float r2 = r * r;
    bool apart = dist2 > r2;
    if (fabsf(dist2 - r2) <= 1e-5f * r2) {
        // too close to call in FP32: decide as FP64 does
        double dpx = (double)pjx - (double)pix, dpy = (double)pjy - (double)piy;
        double dr = (double)ri + (double)rj;
        apart = __dadd_rn(__dmul_rn(dpx, dpx), __dmul_rn(dpy, dpy)) > __dmul_rn(dr, dr);
    }
    float ux, uy, nx, ny;
    if (apart) {
        const float inv_tau = __frcp_rn(tau);
        const float wx = vx - __fdiv_rn(px, tau), wy = vy - __fdiv_rn(py, tau);
        const float w2 = wx * wx + wy * wy;
        const float wp = wx * px + wy * py;
        if (wp < 0.f && wp * wp > r2 * w2) {
            // nearest boundary point on the cut-off arc of D(p/tau, r/tau)
            const float wl = sqrtf(w2);
            const float inv = __frcp_rn(wl);
            const float wnx = wx * inv, wny = wy * inv;
            const float m = r * inv_tau - wl;
            ux = m * wnx;
            uy = m * wny;
            nx = wnx;
            ny = wny;
        } else {
            // nearest boundary point on a leg (ray from 0 tangent to D(p, r))
            const float leg = sqrtf(dist2 - r2);
            const float inv_d2 = __frcp_rn(dist2);
            float det = px * wy - py * wx;
            const float scale = fabsf(px * wy) + fabsf(py * wx);
            bool left = det > 0.f;
            if (fabsf(det) <= 1e-5f * scale) {
                // near the tie: take the FP64 sign, ties to the right leg
                double dpx = (double)pjx - (double)pix, dpy = (double)pjy - (double)piy;
                double dvx = (double)vix - (double)vjx, dvy = (double)viy - (double)vjy;
                double dt_ = (double)tau;
                double dwx = __dsub_rn(dvx, __ddiv_rn(dpx, dt_)), dwy = __dsub_rn(dvy, __ddiv_rn(dpy, dt_));
                left = __dsub_rn(__dmul_rn(dpx, dwy), __dmul_rn(dpy, dwx)) > 0.0;
            }
            float lx, ly;
            if (left) {
                lx = (px * leg - py * r) * inv_d2;
                ly = (px * r + py * leg) * inv_d2;
                nx = -ly;
                ny = lx;
            } else {
                lx = (px * leg + py * r) * inv_d2;
                ly = (-px * r + py * leg) * inv_d2;
                nx = ly;
                ny = -lx;
            }
            const float s = vx * lx + vy * ly;
            ux = s * lx - vx;
            uy = s * ly - vy;
        }
    } else {
        // already overlapping: leave D(p/dt, r/dt) within this step
        const float wx = vx - __fdiv_rn(px, dt), wy = vy - __fdiv_rn(py, dt);
        const float wl = sqrtf(wx * wx + wy * wy);
        float wnx, wny;
        if (wl > 0.f) {
            const float inv = __frcp_rn(wl);
            wnx = wx * inv;
            wny = wy * inv;
        } else if (dist2 > 0.f) {
            const float inv = rsqrtf(dist2);
            wnx = -px * inv;
            wny = -py * inv;
        } else {
            wnx = i_before_j ? 1.f : -1.f;
            wny = 0.f;
        }
        const float m = __fdiv_rn(r, dt) - wl;
        ux = m * wnx;
        uy = m * wny;
        nx = wnx;
        ny = wny;
    }
    Line L;
    L.qx = vix + alpha * ux;
    L.qy = viy + alpha * uy;
    L.nx = nx;
    L.ny = ny;
    return L;
}

// ---------------------------------------------------------------- A4 ----
// Squared distance from p to the segment (a, b) and the closest point.
__device__ __forceinline__ float seg_dist2(float px, float py, float4 s, float& cx, float& cy) {
    const float ex = s.z - s.x, ey = s.w - s.y;
    float t = __fdiv_rn((px - s.x) * ex + (py - s.y) * ey, ex * ex + ey * ey);
    t = fminf(fmaxf(t, 0.f), 1.f);
    cx = s.x + t * ex;
    cy = s.y + t * ey;
    const float dx = cx - px, dy = cy - py;
    return dx * dx + dy * dy;
}

// Half-plane of an agent against a static segment, full responsibility: the
// tangent of the truncated velocity obstacle at its point nearest 0,
// v.m <= (d - r)/tau_o (m: unit vector toward the closest point); when
// overlapping, v.m <= max((d - r)/dt, -v_max).  On the segment (d = 0) m is
// the segment normal on the side the agent's velocity points to (the left
// normal of a->b when undecided).
__device__ __forceinline__ Line obstacle_line(float px, float py, float vx, float vy, float r, float vmax,
                                              float4 s, float tau_o, float dt) {
    float cx, cy;
    const float d2 = seg_dist2(px, py, s, cx, cy);
    const float d = sqrtf(d2);
    float mx, my;
    if (d > 0.f) {
        const float inv = __frcp_rn(d);
        mx = (cx - px) * inv;
        my = (cy - py) * inv;
    } else {
        const float ex = s.z - s.x, ey = s.w - s.y;
        const float inv = rsqrtf(ex * ex + ey * ey);
        const float lx = -ey * inv, ly = ex * inv;
        const bool keep = vx * lx + vy * ly >= 0.f;
        mx = keep ? lx : -lx;
        my = keep ? ly : -ly;
    }
    float b;
    if (d > r) {
        b = __fdiv_rn(d - r, tau_o);
    } else {
        b = fmaxf(__fdiv_rn(d - r, dt), -vmax);
    }
    Line L;
    L.qx = b * mx;
    L.qy = b * my;
    L.nx = -mx;
    L.ny = -my;
    return L;
}

// ---------------------------------------------------------------- A5 ----
// Minimise |v - pref| on line k inside the speed disk and lines 0..k-1.
__device__ __forceinline__ bool lp1(const Line* L, int k, float vmax, float2 pref, float2& v) {
    const Line lk = L[k];
    const float dx = -lk.ny, dy = lk.nx;  // direction along line k
    const float qd = lk.qx * dx + lk.qy * dy;
    const float disc = qd * qd - (lk.qx * lk.qx + lk.qy * lk.qy) + vmax * vmax;
    if (disc < 0.f) return false;
    const float sq = sqrtf(disc);
    float tl = -qd - sq, tr = -qd + sq;
    for (int l = 0; l < k; ++l) {
        const Line ll = L[l];
        const float den = dx * ll.nx + dy * ll.ny;  // det(n_k, n_l)
        const float num = (ll.qx - lk.qx) * ll.nx + (ll.qy - lk.qy) * ll.ny;
        if (fabsf(den) < 1e-4f) {
            // near-parallel: classify and intersect in FP64
            const double ddx = -(double)lk.ny, ddy = (double)lk.nx;
            const double dden = ddx * (double)ll.nx + ddy * (double)ll.ny;
            const double dnum = ((double)ll.qx - (double)lk.qx) * (double)ll.nx +
                                ((double)ll.qy - (double)lk.qy) * (double)ll.ny;
            if (fabs(dden) <= kEpsParallel) {
                if (dnum > 0.0) return false;
                continue;
            }
            const float t = (float)(dnum / dden);
            if (dden > 0.0) tl = fmaxf(tl, t);
            else tr = fminf(tr, t);
        } else {
            const float t = __fdiv_rn(num, den);
            if (den > 0.f) tl = fmaxf(tl, t);
            else tr = fminf(tr, t);
        }
        if (tl > tr) return false;
    }
    float t = (pref.x - lk.qx) * dx + (pref.y - lk.qy) * dy;
    t = fminf(fmaxf(t, tl), tr);
    v.x = lk.qx + t * dx;
    v.y = lk.qy + t * dy;
    return true;
}

// Incremental 2D LP.  Returns n if feasible, else the failing line index.
// `solves` / `solve_lines` count the 1D sub-solves and the previous lines
// they scan.
__device__ __forceinline__ int lp2(const Line* L, int n, float vmax, float2 pref, float2& v, int& solves,
                                   int& solve_lines) {
    const float pl2 = pref.x * pref.x + pref.y * pref.y;
    if (pl2 > vmax * vmax) {
        const float k = vmax * rsqrtf(pl2);
        v = make_float2(pref.x * k, pref.y * k);
    } else {
        v = pref;
    }
    for (int k = 0; k < n; ++k) {
        const Line lk = L[k];
        if ((v.x - lk.qx) * lk.nx + (v.y - lk.qy) * lk.ny < 0.f) {
            float2 nv;
            ++solves;
            solve_lines += k;
            if (!lp1(L, k, vmax, pref, nv)) return k;
            v = nv;
        }
    }
    return n;
}

// ---------------------------------------------------------------- A5 fallback (FP64) ----
struct DLine {
    double qx, qy, nx, ny;
};

// Line k of the FP64 problems: the FP32 line k as is (k < n_hard), or shifted
// outward by `shift` (agent lines, relaxed to viol_k <= shift).
__device__ __forceinline__ DLine shifted_line(const Line* L, int k, int n_hard, double shift) {
    const Line l = L[k];
    DLine d{(double)l.qx, (double)l.qy, (double)l.nx, (double)l.ny};
    if (k >= n_hard) {
        d.qx -= shift * d.nx;
        d.qy -= shift * d.ny;
    }
    return d;
}

// Line m of the directional subproblem of agent line i: hard lines first,
// then for each agent line j in [n_hard, i) the half-plane viol_j <= viol_i,
// i.e. v.(n_j - n_i) >= q_j.n_j - q_i.n_i.  `valid` is false when n_j ~ n_i
// (the constraint cannot bind at the optimum then).
__device__ __forceinline__ DLine sub_line(const Line* L, int n_hard, int i, int m, bool& valid) {
    valid = true;
    if (m < n_hard) return shifted_line(L, m, n_hard, 0.0);
    const Line a = L[i], b = L[m];  // agent line m < i
    const double nx = (double)b.nx - (double)a.nx, ny = (double)b.ny - (double)a.ny;
    const double c = ((double)b.qx * b.nx + (double)b.qy * b.ny) - ((double)a.qx * a.nx + (double)a.qy * a.ny);
    const double nl = sqrt(nx * nx + ny * ny);
    if (nl < 1e-12) {
        valid = false;
        return DLine{0, 0, 1, 0};
    }
    const double inx = nx / nl, iny = ny / nl, off = c / nl;
    return DLine{off * inx, off * iny, inx, iny};
}

// 1D step shared by the FP64 LPs: interval of line `lk` inside the disk and
// the previous lines given by `prev(l, valid)`.
template <class Prev>
__device__ __forceinline__ bool interval_d(const DLine& lk, int k, double vmax, Prev prev, double& tl, double& tr) {
    const double dx = -lk.ny, dy = lk.nx;
    const double qd = lk.qx * dx + lk.qy * dy;
    const double disc = qd * qd - (lk.qx * lk.qx + lk.qy * lk.qy) + vmax * vmax;
    if (disc < 0.0) return false;
    const double sq = sqrt(disc);
    tl = -qd - sq;
    tr = -qd + sq;
    for (int l = 0; l < k; ++l) {
        bool valid;
        const DLine ll = prev(l, valid);
        if (!valid) continue;
        const double den = dx * ll.nx + dy * ll.ny;
        const double num = (ll.qx - lk.qx) * ll.nx + (ll.qy - lk.qy) * ll.ny;
        if (fabs(den) <= kEpsParallel) {
            if (num > 0.0) return false;
            continue;
        }
        const double t = num / den;
        if (den > 0.0) tl = fmax(tl, t);
        else tr = fmin(tr, t);
        if (tl > tr) return false;
    }
    return true;
}

// Least-distance FP64 LP over lines 0..n-1 (agent lines shifted by `shift`).
__device__ __forceinline__ bool lp2_d(const Line* L, int n, int n_hard, double shift, double vmax, double px,
                                      double py, double& vx, double& vy) {
    const double pl2 = px * px + py * py;
    if (pl2 > vmax * vmax) {
        const double k = vmax / sqrt(pl2);
        vx = px * k;
        vy = py * k;
    } else {
        vx = px;
        vy = py;
    }
    for (int k = 0; k < n; ++k) {
        const DLine lk = shifted_line(L, k, n_hard, shift);
        if ((vx - lk.qx) * lk.nx + (vy - lk.qy) * lk.ny < 0.0) {
            double tl, tr;
            auto prev = [&](int l, bool& valid) {
                valid = true;
                return shifted_line(L, l, n_hard, shift);
            };
            if (!interval_d(lk, k, vmax, prev, tl, tr)) return false;
            const double dx = -lk.ny, dy = lk.nx;
            double t = (px - lk.qx) * dx + (py - lk.qy) * dy;
            t = fmin(fmax(t, tl), tr);
            vx = lk.qx + t * dx;
            vy = lk.qy + t * dy;
        }
    }
    return true;
}

// Directional FP64 LP: maximise v.(ox, oy) over the disk and the
// subproblem lines of agent line i.
__device__ __forceinline__ bool lp_dir_d(const Line* L, int n_hard, int i, double vmax, double ox, double oy,
                                         double& vx, double& vy) {
    vx = vmax * ox;
    vy = vmax * oy;
    for (int k = 0; k < i; ++k) {  // hard lines, then agent lines before i
        bool valid;
        const DLine lk = sub_line(L, n_hard, i, k, valid);
        if (!valid) continue;
        if ((vx - lk.qx) * lk.nx + (vy - lk.qy) * lk.ny < 0.0) {
            double tl, tr;
            auto prev = [&](int l, bool& v) { return sub_line(L, n_hard, i, l, v); };
            if (!interval_d(lk, k, vmax, prev, tl, tr)) return false;
            const double dx = -lk.ny, dy = lk.nx;
            const double t = (dx * ox + dy * oy) > 0.0 ? tr : tl;
            vx = lk.qx + t * dx;
            vy = lk.qy + t * dy;
        }
    }
    return true;
}

// Fallback for an infeasible LP (FP64).  Lines [0, n_hard) are static
// (hard), the rest agent lines (soft).  If the disk and the hard lines leave
// nothing, all lines are soft.  d* = min over the hard region of the largest
// agent-line penetration, found by an incremental 3D LP (one directional 2D
// LP per line that the current point violates by more than the current d);
// the result is the point closest to pref with every penetration <= d*.
__device__ __forceinline__ float2 lp_fallback(const Line* L, int n, int n_hard, float vmax_f, float2 pref) {
    const double vmax = vmax_f, px = pref.x, py = pref.y;
    double vx, vy;
    if (!lp2_d(L, n_hard, n_hard, 0.0, vmax, px, py, vx, vy)) {
        n_hard = 0;
        const double pl2 = px * px + py * py;
        const double k = pl2 > vmax * vmax ? vmax / sqrt(pl2) : 1.0;
        vx = px * k;
        vy = py * k;
    }
    double dist = -1e300;
    for (int i = n_hard; i < n; ++i) {
        const Line li = L[i];
        const double viol = -((vx - li.qx) * li.nx + (vy - li.qy) * li.ny);
        if (viol > dist + 1e-12) {
            double tx, ty;
            if (lp_dir_d(L, n_hard, i, vmax, (double)li.nx, (double)li.ny, tx, ty)) {
                vx = tx;
                vy = ty;
            }
            dist = -((vx - li.qx) * li.nx + (vy - li.qy) * li.ny);
        }
    }
    // d* at the point found, then the closest point to pref within it
    double dstar = 0.0;
    for (int k = n_hard; k < n; ++k) {
        const Line lk = L[k];
        dstar = fmax(dstar, -((vx - lk.qx) * lk.nx + (vy - lk.qy) * lk.ny));
    }
    double rx, ry;
    if (lp2_d(L, n, n_hard, dstar + 1e-10, vmax, px, py, rx, ry)) return make_float2((float)rx, (float)ry);
    return make_float2((float)vx, (float)vy);
}

}  // namespace crowd
