// Per-agent device arithmetic of the ORCA crowd step (sm_103a).
//
// FP32 throughout, except where a discrete decision or an ill-conditioned
// quantity must come out as the FP64 definition says:
//   - the neighbour ranking key (squared distance rounded in FP64 with no
//     fused multiply-add) for candidates whose FP32 keys are too close to
//     order, so that neighbour lists are bit-exact;
//   - near contact, |p|^2 - r^2 in compensated FP32 (FP64 within 1e-6);
//   - the leg choice (sign of det(p, w)) and the colliding test
//     (|p|^2 <= r^2) when the FP32 value is within its rounding error of 0;
//   - the near-parallel test of two LP lines (|det| <= 1e-9) and the
//     intersection parameter when |det| is small.
// The geometry is that of ORCA (van den Berg et al., ISRR 2011), the
// collision-avoidance rule the paper uses for its dynamic agents (Sec. 3.2).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace crowd {

constexpr float kEpsGoal = 1e-6f;  // preferred velocity is 0 closer than this to the goal

// Reciprocal and quotients: the library is built with -prec-div=false and
// -prec-sqrt=false, so FP32 division, reciprocal and square root are the
// hardware approximations (about 1 ulp).  The contract needs FP32-level
// accuracy, not correctly rounded results; FP64 and the compensated
// sums are unaffected.
__device__ __forceinline__ float __frcp_fast(float x) { return 1.0f / x; }

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
    if (dist <= speed * dt) return make_float2(dx / dt, dy / dt);
    float k = speed / dist;
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

// Sorted list of the CAP smallest (FP64 key, id) pairs; only the first K
// slots (runtime K <= CAP) are used.  All indices are compile-time so that
// the list lives in registers.  Used when FP32 keys cannot order the
// candidates (near ties), see select_neighbors.
template <int CAP>
struct TopK64 {
    unsigned long long key[CAP];
    int id[CAP];
    int cnt;

    __device__ __forceinline__ void init() {
        cnt = 0;
#pragma unroll
        for (int s = 0; s < CAP; ++s) {
            key[s] = ~0ull;
            id[s] = 0x7fffffff;
        }
    }
    __device__ __forceinline__ static bool less(unsigned long long ka, int ia, unsigned long long kb, int ib) {
        return ka < kb || (ka == kb && ia < ib);
    }
    __device__ __forceinline__ void insert(unsigned long long k, int j, int K) {
        if (K <= 0) return;
        unsigned long long lk = ~0ull;
        int li = 0x7fffffff;
#pragma unroll
        for (int s = 0; s < CAP; ++s)
            if (s == K - 1) { lk = key[s]; li = id[s]; }
        if (!less(k, j, lk, li)) return;
        int p = 0;
#pragma unroll
        for (int s = 0; s < CAP; ++s) p += (s < cnt && less(key[s], id[s], k, j)) ? 1 : 0;
#pragma unroll
        for (int s = CAP - 1; s >= 1; --s) {
            if (s > p) { key[s] = key[s - 1]; id[s] = id[s - 1]; }
            else if (s == p) { key[s] = k; id[s] = j; }
        }
        if (p == 0) { key[0] = k; id[0] = j; }
        cnt = cnt < K ? cnt + 1 : K;
    }
};

// Sorted list of the CAP smallest packed (FP32 key bits << 32 | id) values:
// one 64-bit compare orders by key then id (keys are non-negative floats,
// whose bit patterns order like their values).
template <int CAP>
struct TopK32 {
    unsigned long long e[CAP];
    int cnt;

    __device__ __forceinline__ void init() {
        cnt = 0;
#pragma unroll
        for (int s = 0; s < CAP; ++s) e[s] = ~0ull;
    }
    // Keep the CAP smallest.  Every slot compares with x at once (the list is
    // sorted, so "greater than x" holds for a suffix of the slots): slot s
    // takes its left neighbour when that one is greater than x, x when it is
    // the first greater slot, else keeps its value.  No slot waits on another.
    __device__ __forceinline__ void insert(unsigned long long x) {
        if (x >= e[CAP - 1]) return;
        bool gt[CAP];
#pragma unroll
        for (int s = 0; s < CAP; ++s) gt[s] = e[s] > x;
#pragma unroll
        for (int s = CAP - 1; s >= 1; --s) e[s] = gt[s - 1] ? e[s - 1] : (gt[s] ? x : e[s]);
        e[0] = gt[0] ? x : e[0];
        cnt = cnt < CAP ? cnt + 1 : CAP;
    }
    __device__ __forceinline__ static float key_of(unsigned long long x) { return __uint_as_float((unsigned)(x >> 32)); }
    __device__ __forceinline__ void put(float d2, int slot) {
        insert(((unsigned long long)__float_as_uint(d2) << 32) | (unsigned)slot);
    }
    __device__ __forceinline__ float key(int s) const { return key_of(e[s]); }
    __device__ __forceinline__ int slot(int s) const { return (int)(unsigned)e[s]; }
};

// The same list with the FP32 keys and the candidate slots in two 32-bit
// arrays: one 32-bit compare and two selects per word and entry instead of
// a 64-bit compare and four selects (the insertion network is the update's
// busiest integer work).  Equal keys keep their order of insertion, and a
// key equal to the last one is not taken: exactly equal FP32 keys are near
// ties, which the caller ranks again by (FP64 key, index), so the kept
// neighbours are the same.
template <int CAP>
struct TopKSplit {
    unsigned k[CAP];
    int u[CAP];
    int cnt;

    __device__ __forceinline__ void init() {
        cnt = 0;
#pragma unroll
        for (int s = 0; s < CAP; ++s) {
            k[s] = 0xffffffffu;
            u[s] = 0;
        }
    }
    __device__ __forceinline__ void put(float d2, int slot) {
        const unsigned x = __float_as_uint(d2);
        if (x >= k[CAP - 1]) return;
        bool gt[CAP];
#pragma unroll
        for (int s = 0; s < CAP; ++s) gt[s] = k[s] > x;
#pragma unroll
        for (int s = CAP - 1; s >= 1; --s) {
            k[s] = gt[s - 1] ? k[s - 1] : (gt[s] ? x : k[s]);
            u[s] = gt[s - 1] ? u[s - 1] : (gt[s] ? slot : u[s]);
        }
        k[0] = gt[0] ? x : k[0];
        u[0] = gt[0] ? slot : u[0];
        cnt = cnt < CAP ? cnt + 1 : CAP;
    }
    __device__ __forceinline__ float key(int s) const { return __uint_as_float(k[s]); }
    __device__ __forceinline__ int slot(int s) const { return u[s]; }
};

// Relative error bound of the FP32 squared distance against the FP64
// ranking key (a few units of 2^-24, with margin): FP32 keys further apart
// than this order exactly like the FP64 keys.
constexpr float kKeyRelErr = 1e-6f;

// ---------------------------------------------------------------- A3 ----
// s + e = a + b exactly (Knuth's two-sum).
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

// (pj - pi)^2 - (ri + rj)^2 in compensated FP32: the differences and the sum
// are split into exact two-float pairs, the squares into product + FMA
// residual, and the cancelling sum is carried with its error terms, so the
// result is accurate to a few units in its last place even at contact.
__device__ __forceinline__ float contact_gap2(float pix, float piy, float pjx, float pjy, float ri, float rj) {
    float xh, xl, yh, yl, rh, rl;
    two_sum(pjx, -pix, xh, xl);
    two_sum(pjy, -piy, yh, yl);
    two_sum(ri, rj, rh, rl);
    const float h1 = __fmul_rn(xh, xh), l1 = fmaf(xh, xh, -h1) + 2.f * xh * xl;
    const float h2 = __fmul_rn(yh, yh), l2 = fmaf(yh, yh, -h2) + 2.f * yh * yl;
    const float h3 = __fmul_rn(rh, rh), l3 = fmaf(rh, rh, -h3) + 2.f * rh * rl;
    float s, e1, t, e2;
    two_sum(h1, h2, s, e1);
    two_sum(s, -h3, t, e2);
    return t + (((e1 + e2) + (l1 + l2)) - l3);
}

// FP64 evaluation of the agent half-plane (same geometry as agent_line),
// used for pairs within a relative 1e-6 of contact.  Every product and sum is rounded
// separately so that the colliding and leg decisions match an FP64
// evaluation of the definition exactly.
static __device__ __noinline__ Line agent_line_fp64(float pix, float piy, float vix, float viy, float ri, float pjx,
                                             float pjy, float vjx, float vjy, float rj, float tau, float dt,
                                             float alpha, bool i_before_j) {
    const double px = __dsub_rn((double)pjx, (double)pix), py = __dsub_rn((double)pjy, (double)piy);
    const double vx = __dsub_rn((double)vix, (double)vjx), vy = __dsub_rn((double)viy, (double)vjy);
    const double r = __dadd_rn((double)ri, (double)rj);
    const double dist2 = __dadd_rn(__dmul_rn(px, px), __dmul_rn(py, py));
    const double r2 = __dmul_rn(r, r);
    const double T = (double)tau, D = (double)dt;
    double ux, uy, nx, ny;
    if (dist2 > r2) {
        const double wx = __dsub_rn(vx, __ddiv_rn(px, T)), wy = __dsub_rn(vy, __ddiv_rn(py, T));
        const double w2 = __dadd_rn(__dmul_rn(wx, wx), __dmul_rn(wy, wy));
        const double wp = __dadd_rn(__dmul_rn(wx, px), __dmul_rn(wy, py));
        if (wp < 0.0 && __dmul_rn(wp, wp) > __dmul_rn(r2, w2)) {
            const double wl = sqrt(w2);
            const double wnx = wx / wl, wny = wy / wl;
            const double m = r / T - wl;
            ux = m * wnx;
            uy = m * wny;
            nx = wnx;
            ny = wny;
        } else {
            const double leg = sqrt(dist2 - r2);
            const bool left = __dsub_rn(__dmul_rn(px, wy), __dmul_rn(py, wx)) > 0.0;
            double lx, ly;
            if (left) {
                lx = (px * leg - py * r) / dist2;
                ly = (px * r + py * leg) / dist2;
                nx = -ly;
                ny = lx;
            } else {
                lx = (px * leg + py * r) / dist2;
                ly = (-px * r + py * leg) / dist2;
                nx = ly;
                ny = -lx;
            }
            const double s = vx * lx + vy * ly;
            ux = s * lx - vx;
            uy = s * ly - vy;
        }
    } else {
        const double wx = __dsub_rn(vx, __ddiv_rn(px, D)), wy = __dsub_rn(vy, __ddiv_rn(py, D));
        const double wl = sqrt(wx * wx + wy * wy);
        double wnx, wny;
        if (wl > 0.0) {
            wnx = wx / wl;
            wny = wy / wl;
        } else if (dist2 > 0.0) {
            const double pl = sqrt(dist2);
            wnx = -px / pl;
            wny = -py / pl;
        } else {
            wnx = i_before_j ? 1.0 : -1.0;
            wny = 0.0;
        }
        const double m = r / D - wl;
        ux = m * wnx;
        uy = m * wny;
        nx = wnx;
        ny = wny;
    }
    Line L;
    L.qx = (float)((double)vix + (double)alpha * ux);
    L.qy = (float)((double)viy + (double)alpha * uy);
    L.nx = (float)nx;
    L.ny = (float)ny;
    return L;
}

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
    // gap2 = |p|^2 - r^2: near contact it cancels, so there it is evaluated in
    // compensated FP32 (the colliding test and the legs' length depend on it)
    float gap2 = dist2 - r2;
    if (fabsf(gap2) <= 1e-2f * r2) {
        gap2 = contact_gap2(pix, piy, pjx, pjy, ri, rj);
        if (fabsf(gap2) <= 1e-6f * r2) {
            // closer to contact than compensated FP32 can decide like FP64
            return agent_line_fp64(pix, piy, vix, viy, ri, pjx, pjy, vjx, vjy, rj, tau, dt, alpha, i_before_j);
        }
    }
    const bool apart = gap2 > 0.f;
    float ux, uy, nx, ny;
    if (apart) {
        const float inv_tau = __frcp_fast(tau);
        const float wx = vx - px / tau, wy = vy - py / tau;
        const float w2 = wx * wx + wy * wy;
        const float wp = wx * px + wy * py;
        if (wp < 0.f && wp * wp > r2 * w2) {
            // nearest boundary point on the cut-off arc of D(p/tau, r/tau)
            const float wl = sqrtf(w2);
            const float inv = __frcp_fast(wl);
            const float wnx = wx * inv, wny = wy * inv;
            const float m = r * inv_tau - wl;
            ux = m * wnx;
            uy = m * wny;
            nx = wnx;
            ny = wny;
        } else {
            // nearest boundary point on a leg (ray from 0 tangent to D(p, r))
            const float leg = sqrtf(gap2);
            const float inv_d2 = __frcp_fast(dist2);
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
        const float wx = vx - px / dt, wy = vy - py / dt;
        const float wl = sqrtf(wx * wx + wy * wy);
        float wnx, wny;
        if (wl > 0.f) {
            const float inv = __frcp_fast(wl);
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
        const float m = r / dt - wl;
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
// a*d - b*c with one rounding's worth of error (Kahan's FMA scheme).
__device__ __forceinline__ float det2(float a, float b, float c, float d) {
    const float w = b * c;
    const float e = fmaf(-b, c, w);
    const float f = fmaf(a, d, -w);
    return f + e;
}

// Squared distance from p to the segment (a, b) and the closest point,
// relative to p, so that its rounding error scales with the distance and not
// with the coordinates or the segment length: inside the segment the closest
// point is det(a - p, e) / |e|^2 * (e_y, -e_x), the perpendicular foot, with
// the determinant evaluated by Kahan's scheme.  A clamped projection returns
// the endpoint itself, so that two segments meeting at a vertex give
// bit-identical closest points (and lines).
__device__ __forceinline__ float seg_dist2(float px, float py, float4 s, float& cx, float& cy) {
    const float ax = s.x - px, ay = s.y - py;
    const float ex = s.z - s.x, ey = s.w - s.y;
    const float e2 = ex * ex + ey * ey;
    const float t = -(ax * ex + ay * ey) / e2;
    if (t <= 0.f) {
        cx = ax;
        cy = ay;
    } else if (t >= 1.f) {
        cx = s.z - px;
        cy = s.w - py;
    } else {
        const float k = det2(ax, ay, ex, ey) / e2;
        cx = k * ey;
        cy = -k * ex;
    }
    return cx * cx + cy * cy;
}

// Half-plane of an agent against a static segment, full responsibility: the
// tangent of the truncated velocity obstacle at its point nearest 0,
// v.m <= (d - r)/tau_o (m: unit vector toward the closest point); when
// overlapping, v.m <= max((d - r)/dt, -v_max).  On the segment (d = 0) m is
// the segment normal on the side the agent's velocity points to (the left
// normal of a->b when undecided).
__device__ __forceinline__ Line obstacle_line(float px, float py, float vx, float vy, float r, float vmax,
                                              float4 s, float tau_o, float dt) {
    float cx, cy;  // closest point relative to p
    const float d2 = seg_dist2(px, py, s, cx, cy);
    const float d = sqrtf(d2);
    float mx, my;
    if (d > 0.f) {
        const float inv = __frcp_fast(d);
        mx = cx * inv;
        my = cy * inv;
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
        b = (d - r) / tau_o;
    } else {
        b = fmaxf((d - r) / dt, -vmax);
    }
    Line L;
    L.qx = b * mx;
    L.qy = b * my;
    L.nx = -mx;
    L.ny = -my;
    return L;
}

// ---------------------------------------------------------------- A4v ---
// Velocity-dependent half-plane against a static segment (full
// responsibility): the tangent of the segment's truncated velocity obstacle
// at its boundary point X nearest the current velocity v, (v' - X).n >= 0.
// The obstacle is the capsule C = [a - p, b - p] + D(r); its truncated VO is
// bounded by the two legs (rays from 0 tangent to C beyond the tangent
// points) and by the part of C / tau_o that faces 0.  Candidates, each the
// nearest point of one piece: the flat side of C / tau_o towards 0 (when it
// faces 0), the end-cap arcs that face 0 (their radial point, when it lies
// on the arc), and the two legs; the first of equally near pieces wins (flat,
// cap a, cap b, left, right).  Overlapping (d <= r): as obstacle_line.  When
// the two nearest pieces are within 2e-5 m/s, FP32 rounding could pick the
// other one, so the choice is made again in FP64.

// Unit tangent direction from 0 to the disk D(X, r) (left or right) and the
// tangent length; gap2 = |X|^2 - r^2 (compensated by the caller).
__device__ __forceinline__ void vd_leg(float x0, float x1, float r, float gap2, bool left, float& ux, float& uy,
                                       float& len) {
    const float l = sqrtf(fmaxf(gap2, 0.f));
    const float inv = __frcp_fast(x0 * x0 + x1 * x1);
    if (left) {
        ux = (x0 * l - x1 * r) * inv;
        uy = (x0 * r + x1 * l) * inv;
    } else {
        ux = (x0 * l + x1 * r) * inv;
        uy = (-x0 * r + x1 * l) * inv;
    }
    len = l;
}

struct VdBest {
    float best = INFINITY, second = INFINITY;
    Line L{0.f, 0.f, 0.f, 0.f};
    __device__ __forceinline__ void take(float dd, float x0, float x1, float n0, float n1) {
        if (dd < best) {
            second = best;
            best = dd;
            L = Line{x0, x1, n0, n1};
        } else if (dd < second) {
            second = dd;
        }
    }
};

static __device__ __noinline__ Line obstacle_line_vd_fp64(float px, float py, float vxf, float vyf, float rf,
                                                          float4 s, float tau_of) {
    const double vx = vxf, vy = vyf, r = rf, tau = tau_of;
    const double A0 = (double)s.x - (double)px, A1 = (double)s.y - (double)py;
    const double B0 = (double)s.z - (double)px, B1 = (double)s.w - (double)py;
    double L0, L1, Ll, R0, R1, Rl;
    {
        double la[3], lb[3], ra[3], rb[3];
        const double XA[2] = {A0, A1}, XB[2] = {B0, B1};
        for (int k = 0; k < 4; ++k) {
            const double* X = (k & 1) ? XB : XA;
            const bool left = k < 2;
            const double d2 = X[0] * X[0] + X[1] * X[1];
            const double l = sqrt(fmax(d2 - r * r, 0.0));
            double* o = left ? ((k & 1) ? lb : la) : ((k & 1) ? rb : ra);
            o[0] = left ? (X[0] * l - X[1] * r) / d2 : (X[0] * l + X[1] * r) / d2;
            o[1] = left ? (X[0] * r + X[1] * l) / d2 : (-X[0] * r + X[1] * l) / d2;
            o[2] = l;
        }
        if (la[0] * lb[1] - la[1] * lb[0] > 0.0) { L0 = lb[0]; L1 = lb[1]; Ll = lb[2]; }
        else { L0 = la[0]; L1 = la[1]; Ll = la[2]; }
        if (ra[0] * rb[1] - ra[1] * rb[0] < 0.0) { R0 = rb[0]; R1 = rb[1]; Rl = rb[2]; }
        else { R0 = ra[0]; R1 = ra[1]; Rl = ra[2]; }
    }
    double best = 1e300, X0 = 0.0, X1 = 0.0, N0 = 0.0, N1 = 0.0;
    const double rt = r / tau;
    const double a0 = A0 / tau, a1 = A1 / tau, b0 = B0 / tau, b1 = B1 / tau;
    const double e0 = B0 - A0, e1 = B1 - A1, el = sqrt(e0 * e0 + e1 * e1);
    if (el > 0.0) {
        double m0 = -e1 / el, m1 = e0 / el;
        if (m0 * A0 + m1 * A1 > 0.0) { m0 = -m0; m1 = -m1; }
        if (m0 * A0 + m1 * A1 < -r) {
            const double f0 = a0 + rt * m0, f1 = a1 + rt * m1, g0 = b0 - a0, g1 = b1 - a1;
            double t = ((vx - f0) * g0 + (vy - f1) * g1) / (g0 * g0 + g1 * g1);
            t = fmin(fmax(t, 0.0), 1.0);
            const double x0 = f0 + t * g0, x1 = f1 + t * g1;
            const double dd = sqrt((vx - x0) * (vx - x0) + (vy - x1) * (vy - x1));
            if (dd < best) { best = dd; X0 = x0; X1 = x1; N0 = m0; N1 = m1; }
        }
    }
    for (int cap = 0; cap < 2; ++cap) {
        const double c0 = cap ? b0 : a0, c1 = cap ? b1 : a1;
        const double o0 = cap ? A0 - B0 : B0 - A0, o1 = cap ? A1 - B1 : B1 - A1;
        const double w0 = vx - c0, w1 = vy - c1, wl = sqrt(w0 * w0 + w1 * w1);
        if (!(wl > 0.0)) continue;
        const double u0 = w0 / wl, u1 = w1 / wl;
        if (u0 * o0 + u1 * o1 > 0.0) continue;
        if (!(u0 * c0 + u1 * c1 < -rt)) continue;
        const double dd = fabs(wl - rt);
        if (dd < best) { best = dd; X0 = c0 + rt * u0; X1 = c1 + rt * u1; N0 = u0; N1 = u1; }
    }
    {
        const double t = fmax(vx * L0 + vy * L1, Ll / tau);
        const double x0 = t * L0, x1 = t * L1;
        const double dd = sqrt((vx - x0) * (vx - x0) + (vy - x1) * (vy - x1));
        if (dd < best) { best = dd; X0 = x0; X1 = x1; N0 = -L1; N1 = L0; }
    }
    {
        const double t = fmax(vx * R0 + vy * R1, Rl / tau);
        const double x0 = t * R0, x1 = t * R1;
        const double dd = sqrt((vx - x0) * (vx - x0) + (vy - x1) * (vy - x1));
        if (dd < best) { best = dd; X0 = x0; X1 = x1; N0 = R1; N1 = -R0; }
    }
    return Line{(float)X0, (float)X1, (float)N0, (float)N1};
}

// Kept out of line: the default segment lines do not pay for its registers.
static __device__ __noinline__ Line obstacle_line_vd(float px, float py, float vx, float vy, float r, float vmax,
                                                     float4 s, float tau_o, float dt) {
    float cx, cy;
    if (!(seg_dist2(px, py, s, cx, cy) > r * r)) return obstacle_line(px, py, vx, vy, r, vmax, s, tau_o, dt);
    const float A0 = s.x - px, A1 = s.y - py, B0 = s.z - px, B1 = s.w - py;
    float L0, L1, Ll, R0, R1, Rl;
    {
        const float ga = contact_gap2(px, py, s.x, s.y, r, 0.f), gb = contact_gap2(px, py, s.z, s.w, r, 0.f);
        float la0, la1, lal, lb0, lb1, lbl, ra0, ra1, ral, rb0, rb1, rbl;
        vd_leg(A0, A1, r, ga, true, la0, la1, lal);
        vd_leg(B0, B1, r, gb, true, lb0, lb1, lbl);
        vd_leg(A0, A1, r, ga, false, ra0, ra1, ral);
        vd_leg(B0, B1, r, gb, false, rb0, rb1, rbl);
        const bool lb_out = la0 * lb1 - la1 * lb0 > 0.f, rb_out = ra0 * rb1 - ra1 * rb0 < 0.f;
        L0 = lb_out ? lb0 : la0;
        L1 = lb_out ? lb1 : la1;
        Ll = lb_out ? lbl : lal;
        R0 = rb_out ? rb0 : ra0;
        R1 = rb_out ? rb1 : ra1;
        Rl = rb_out ? rbl : ral;
    }
    const float inv_tau = __frcp_fast(tau_o);
    const float rt = r * inv_tau;
    const float a0 = A0 * inv_tau, a1 = A1 * inv_tau, b0 = B0 * inv_tau, b1 = B1 * inv_tau;
    VdBest vb;
    const float e0 = B0 - A0, e1 = B1 - A1, ee = e0 * e0 + e1 * e1;
    if (ee > 0.f) {
        const float ie = rsqrtf(ee);
        float m0 = -e1 * ie, m1 = e0 * ie;
        if (m0 * A0 + m1 * A1 > 0.f) {
            m0 = -m0;
            m1 = -m1;
        }
        if (m0 * A0 + m1 * A1 < -r) {
            const float f0 = a0 + rt * m0, f1 = a1 + rt * m1, g0 = b0 - a0, g1 = b1 - a1;
            const float t = fminf(fmaxf(((vx - f0) * g0 + (vy - f1) * g1) / (g0 * g0 + g1 * g1), 0.f), 1.f);
            const float x0 = f0 + t * g0, x1 = f1 + t * g1;
            vb.take(sqrtf((vx - x0) * (vx - x0) + (vy - x1) * (vy - x1)), x0, x1, m0, m1);
        }
    }
#pragma unroll
    for (int cap = 0; cap < 2; ++cap) {
        const float c0 = cap ? b0 : a0, c1 = cap ? b1 : a1;
        const float o0 = cap ? -e0 : e0, o1 = cap ? -e1 : e1;
        const float w0 = vx - c0, w1 = vy - c1, wl = sqrtf(w0 * w0 + w1 * w1);
        if (!(wl > 0.f)) continue;
        const float iw = __frcp_fast(wl);
        const float u0 = w0 * iw, u1 = w1 * iw;
        if (u0 * o0 + u1 * o1 > 0.f || !(u0 * c0 + u1 * c1 < -rt)) continue;
        vb.take(fabsf(wl - rt), c0 + rt * u0, c1 + rt * u1, u0, u1);
    }
    {
        const float t = fmaxf(vx * L0 + vy * L1, Ll * inv_tau);
        const float x0 = t * L0, x1 = t * L1;
        vb.take(sqrtf((vx - x0) * (vx - x0) + (vy - x1) * (vy - x1)), x0, x1, -L1, L0);
    }
    {
        const float t = fmaxf(vx * R0 + vy * R1, Rl * inv_tau);
        const float x0 = t * R0, x1 = t * R1;
        vb.take(sqrtf((vx - x0) * (vx - x0) + (vy - x1) * (vy - x1)), x0, x1, R1, -R0);
    }
    if (vb.second - vb.best <= 2e-5f) return obstacle_line_vd_fp64(px, py, vx, vy, r, s, tau_o);
    return vb.L;
}

// ---------------------------------------------------------------- A5 ----
// Slack of the FP32 interval tests, in m/s: an interval that comes out empty
// by less than this (a line touching the speed disk, three lines through one
// point) is taken as the single point it is in exact arithmetic, instead of
// sending an LP that FP32 rounding alone made infeasible to the fallback.
constexpr float kIntervalSlack = 1e-5f;
// disc / v_max^2 at or below which a line counts as tangent to the speed disk
// (a few times the FP32 rounding of disc).
constexpr float kTangentDisc = 2e-6f;

// |det(n_k, n_l)| at or below which two lines count as parallel.
constexpr float kEpsParallelF = 1e-9f;

// p + e = a * b exactly (the FMA gives the rounding error of the product;
// p is rounded on its own, never fused into the sum that consumes it).
__device__ __forceinline__ void two_prod(float a, float b, float& p, float& e) {
    p = __fmul_rn(a, b);
    e = fmaf(a, b, -p);
}

// The LP below writes every a*b + c*d as fma(a, b, round(c*d)) and every
// q + t*d as one FMA.  Left to itself the compiler picks which product of a
// sum to fuse from the code around it, so two inlined copies of the same LP
// (the fallback run in place and the one run later from the queue) could
// round differently; with the pattern fixed they give the same bits.
__device__ __forceinline__ float fdot2(float a, float b, float c, float d) { return __fmaf_rn(a, b, __fmul_rn(c, d)); }
// (v - q).n for a point v and a line through q with normal n
__device__ __forceinline__ float side_of(float vx, float vy, float qx, float qy, float nx, float ny) {
    return fdot2(vx - qx, nx, vy - qy, ny);
}

// Clip [lo, hi] on line k by a line l nearly parallel to it (|det| < 1e-4 in
// plain FP32, where det and the offset cancel).  det(n_k, n_l) and
// (q_l - q_k).n_l are evaluated in compensated FP32: exact differences
// (two_sum) and products (two_prod), summed with their error terms, so both
// are accurate to a few units of 2^-48 of their terms, as close as an FP64
// evaluation of the same FP32 inputs for the parallel test (|det| <= 1e-9)
// and the signs it decides.  GB300 runs FP64 at 1/64 of the FP32 rate, so
// this branch stays in FP32.  Returns true when l is parallel to k and
// excludes it entirely.
__device__ __forceinline__ bool clip_near_parallel(const Line& lk, const Line& ll, float& lo, float& hi) {
    float p1, e1, p2, e2, den, e3;
    two_prod(-lk.ny, ll.nx, p1, e1);
    two_prod(lk.nx, ll.ny, p2, e2);
    two_sum(p1, p2, den, e3);
    den += (e1 + e2) + e3;
    float ax, axe, ay, aye;
    two_sum(ll.qx, -lk.qx, ax, axe);
    two_sum(ll.qy, -lk.qy, ay, aye);
    float q1, f1, q2, f2, num, f3;
    two_prod(ax, ll.nx, q1, f1);
    two_prod(ay, ll.ny, q2, f2);
    two_sum(q1, q2, num, f3);
    num += ((f1 + f2) + f3) + fdot2(axe, ll.nx, aye, ll.ny);
    if (fabsf(den) <= kEpsParallelF) return num > 0.f;
    const float t = num / den;
    if (den > 0.f) lo = fmaxf(lo, t);
    else hi = fminf(hi, t);
    return false;
}

// Interval [tl, tr] of the parameter t along line k (point q_k + t d_k,
// d_k = (-n_y, n_x)) inside the speed disk and the lines 0..k-1; false if
// empty by more than kIntervalSlack.  Near-parallel pairs (|det| < 1e-4 in
// FP32) go through clip_near_parallel, parallel meaning |det| <= 1e-9.
__device__ __forceinline__ bool line_interval(const Line* L, int k, float vmax, float& tl, float& tr) {
    const Line lk = L[k];
    const float dx = -lk.ny, dy = lk.nx;
    const float qd = fdot2(lk.qx, dx, lk.qy, dy);
    float disc = __fadd_rn(__fmaf_rn(qd, qd, -fdot2(lk.qx, lk.qx, lk.qy, lk.qy)), __fmul_rn(vmax, vmax));
    if (disc < 0.f) {
        // the line misses the disk by about -disc / (2 vmax)
        if (disc < -2.f * kIntervalSlack * vmax) return false;
        disc = 0.f;
    }
    // a line tangent to the disk (an overlapping agent's segment line capped
    // at -v_max is tangent by construction) meets it in one point; FP32
    // rounding of the line would open a chord of half-length sqrt(disc), so
    // chords within the rounding of disc are closed
    if (disc <= kTangentDisc * vmax * vmax) disc = 0.f;
    const float sq = sqrtf(disc);
    tl = -qd - sq;
    tr = -qd + sq;
    // the next line is loaded while this one clips
    Line nxt = k > 0 ? L[0] : lk;
    for (int l = 0; l < k; ++l) {
        const Line ll = nxt;
        if (l + 1 < k) nxt = L[l + 1];
        const float den = fdot2(dx, ll.nx, dy, ll.ny);  // det(n_k, n_l)
        const float num = side_of(ll.qx, ll.qy, lk.qx, lk.qy, ll.nx, ll.ny);
        if (fabsf(den) < 1e-4f) {
            if (clip_near_parallel(lk, ll, tl, tr)) return false;
        } else {
            const float t = num / den;
            if (den > 0.f) tl = fmaxf(tl, t);
            else tr = fminf(tr, t);
        }
        if (tl > tr) {
            if (tl - tr > kIntervalSlack) return false;
            tl = tr = 0.5f * (tl + tr);
        }
    }
    return true;
}

// Minimise |v - pref| on line k inside the speed disk and lines 0..k-1.
__device__ __forceinline__ bool lp1(const Line* L, int k, float vmax, float2 pref, float2& v) {
    float tl, tr;
    if (!line_interval(L, k, vmax, tl, tr)) return false;
    const Line lk = L[k];
    const float dx = -lk.ny, dy = lk.nx;
    float t = side_of(pref.x, pref.y, lk.qx, lk.qy, dx, dy);
    t = fminf(fmaxf(t, tl), tr);
    v.x = __fmaf_rn(t, dx, lk.qx);
    v.y = __fmaf_rn(t, dy, lk.qy);
    return true;
}

// Incremental 2D LP.  Returns n if feasible, else the failing line index.
// `solves` / `solve_lines` count the 1D sub-solves and the previous lines
// they scan.
__device__ __forceinline__ int lp2(const Line* L, int n, float vmax, float2 pref, float2& v, int& solves,
                                   int& solve_lines) {
    const float pl2 = fdot2(pref.x, pref.x, pref.y, pref.y);
    if (pl2 > __fmul_rn(vmax, vmax)) {
        const float k = vmax * rsqrtf(pl2);
        v = make_float2(pref.x * k, pref.y * k);
    } else {
        v = pref;
    }
    Line nxt = n > 0 ? L[0] : Line{0.f, 0.f, 0.f, 0.f};
    for (int k = 0; k < n; ++k) {
        const Line lk = nxt;
        if (k + 1 < n) nxt = L[k + 1];
        if (side_of(v.x, v.y, lk.qx, lk.qy, lk.nx, lk.ny) < 0.f) {
            float2 nv;
            ++solves;
            solve_lines += k;
            if (!lp1(L, k, vmax, pref, nv)) return k;
            v = nv;
        }
    }
    return n;
}

// ---------------------------------------------------------------- A5 fallback ----
// Maximise v.o over the speed disk and lines 0..m-1 (incremental, like lp2
// with a linear objective).  When the objective is perpendicular to the line
// the optimum lies on (|d.o| <= 1e-6), every point of the interval is
// optimal and the one closest to pref is taken.
__device__ __forceinline__ bool lp_dir(const Line* S, int m, float vmax, float ox, float oy, float2 pref, float2& v) {
    v = make_float2(vmax * ox, vmax * oy);
    for (int k = 0; k < m; ++k) {
        const Line lk = S[k];
        if (side_of(v.x, v.y, lk.qx, lk.qy, lk.nx, lk.ny) < 0.f) {
            float tl, tr;
            if (!line_interval(S, k, vmax, tl, tr)) return false;
            const float dx = -lk.ny, dy = lk.nx;
            const float dd = fdot2(dx, ox, dy, oy);
            float t;
            if (dd > 1e-6f) t = tr;
            else if (dd < -1e-6f) t = tl;
            else t = fminf(fmaxf(side_of(pref.x, pref.y, lk.qx, lk.qy, dx, dy), tl), tr);
            v.x = __fmaf_rn(t, dx, lk.qx);
            v.y = __fmaf_rn(t, dy, lk.qy);
        }
    }
    return true;
}

// Fallback for an infeasible LP.  Lines [0, n_hard) are static (hard), the
// rest agent lines (soft), penetration viol_k(v) = -(v - q_k).n_k.  If the
// disk and the hard lines leave nothing, all lines are soft.  The velocity of
// least maximal penetration is found by an incremental 3D LP over (v, t):
// while the current point penetrates agent line i by more than the current
// maximum, the optimum moves onto viol_i = t, where it maximises v.n_i subject
// to the hard lines and viol_j <= viol_i (j < i), i.e. the half-planes
// v.(n_j - n_i) >= q_j.n_j - q_i.n_i.  The least-penetration point is
// unique except when that subproblem's optimum is a whole interval, where
// lp_dir takes the point closest to pref.  S is scratch for the subproblem
// lines (at least n entries).
//
// The increments from line i0 on, from point v with penetration bound dist
// (shared by both starts below).
__device__ __forceinline__ float2 fallback_increments(const Line* L, int n, int n_hard, float vmax, float2 pref,
                                                      Line* S, float2 v, float dist, int i0) {
    for (int i = i0; i < n; ++i) {
        const Line li = L[i];
        const float viol = -side_of(v.x, v.y, li.qx, li.qy, li.nx, li.ny);
        if (viol > dist) {
            int m = 0;
            for (int k = 0; k < n_hard; ++k) S[m++] = L[k];
            const float ci = fdot2(li.qx, li.nx, li.qy, li.ny);
            for (int j = n_hard; j < i; ++j) {
                const Line lj = L[j];
                float nx = lj.nx - li.nx, ny = lj.ny - li.ny;
                const float nl2 = fdot2(nx, nx, ny, ny);
                if (nl2 < 1e-12f) continue;  // same direction: cannot bind at the optimum
                const float inv = rsqrtf(nl2);
                nx *= inv;
                ny *= inv;
                const float c = (fdot2(lj.qx, lj.nx, lj.qy, lj.ny) - ci) * inv;
                S[m++] = Line{c * nx, c * ny, nx, ny};
            }
            float2 t;
            if (lp_dir(S, m, vmax, li.nx, li.ny, pref, t)) v = t;
            dist = -side_of(v.x, v.y, li.qx, li.qy, li.nx, li.ny);
        }
    }
    return v;
}

// Cold start: from the hard lines' LP (all lines soft when it is empty),
// penetration bound -infinity, first agent line.
__device__ __forceinline__ float2 lp_fallback(const Line* L, int n, int n_hard, float vmax, float2 pref, Line* S) {
    float2 v;
    int solves = 0, solve_lines = 0;
    if (lp2(L, n_hard, vmax, pref, v, solves, solve_lines) < n_hard) {
        n_hard = 0;
        const float pl2 = fdot2(pref.x, pref.x, pref.y, pref.y);
        const float k = pl2 > __fmul_rn(vmax, vmax) ? vmax * rsqrtf(pl2) : 1.f;
        v = make_float2(pref.x * k, pref.y * k);
    }
    return fallback_increments(L, n, n_hard, vmax, pref, S, v, -INFINITY, n_hard);
}

// Warm start: when the 2D LP failed at line `begin` >= n_hard, its last
// iterate `v_begin` satisfies every line before `begin` (the hard ones
// among them), so the least maximal penetration, which is positive, is
// found by the same increments started there with penetration bound 0 and
// line `begin`: the lines before it cannot be penetrated more than 0 by
// that point.  The optimum is the same; the increments over the lines the
// 2D LP already satisfied are skipped.  Otherwise the cold start.
__device__ __forceinline__ float2 lp_fallback_warm(const Line* L, int n, int n_hard, float vmax, float2 pref,
                                                   Line* S, int begin, float2 v_begin) {
    if (begin >= n_hard && begin < n) return fallback_increments(L, n, n_hard, vmax, pref, S, v_begin, 0.f, begin);
    return lp_fallback(L, n, n_hard, vmax, pref, S);
}

// ---------------------------------------------------------------- A5, warp-cooperative ----
// The same LPs with the 32 lanes of a warp sharing each 1D sub-solve: lines
// live in shared memory, every lane clips the interval by a strided subset
// of the previous lines, and the bounds meet in a shuffle reduction.  All
// lanes call with identical arguments and return identical results.

__device__ __forceinline__ bool coop_line_interval(const Line* L, int k, float vmax, float& tl, float& tr) {
    const int lane = threadIdx.x & 31;
    const Line lk = L[k];
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
    for (int l = lane; l < k; l += 32) {
        const Line ll = L[l];
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
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        lo = fmaxf(lo, __shfl_xor_sync(0xffffffffu, lo, o));
        hi = fminf(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    }
    if (__any_sync(0xffffffffu, bad)) return false;
    if (lo > hi) {
        if (lo - hi > kIntervalSlack) return false;
        lo = hi = 0.5f * (lo + hi);
    }
    tl = lo;
    tr = hi;
    return true;
}

// Warp-cooperative lp2 (least distance to pref); returns n or the failing line.
__device__ __forceinline__ int coop_lp2(const Line* L, int n, float vmax, float2 pref, float2& v) {
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
            float tl, tr;
            if (!coop_line_interval(L, k, vmax, tl, tr)) return k;
            const float dx = -lk.ny, dy = lk.nx;
            float t = (pref.x - lk.qx) * dx + (pref.y - lk.qy) * dy;
            t = fminf(fmaxf(t, tl), tr);
            v = make_float2(lk.qx + t * dx, lk.qy + t * dy);
        }
    }
    return n;
}

// Warp-cooperative lp_dir.
__device__ __forceinline__ bool coop_lp_dir(const Line* S, int m, float vmax, float ox, float oy, float2 pref,
                                            float2& v) {
    v = make_float2(vmax * ox, vmax * oy);
    for (int k = 0; k < m; ++k) {
        const Line lk = S[k];
        if ((v.x - lk.qx) * lk.nx + (v.y - lk.qy) * lk.ny < 0.f) {
            float tl, tr;
            if (!coop_line_interval(S, k, vmax, tl, tr)) return false;
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

// Warp-cooperative lp_fallback; L and S (scratch, >= n lines) in shared
// memory.  A same-direction pair gives an inert line (zero normal).
__device__ __forceinline__ float2 coop_fallback(const Line* L, int n, int n_hard, float vmax, float2 pref, Line* S) {
    const int lane = threadIdx.x & 31;
    float2 v;
    if (coop_lp2(L, n_hard, vmax, pref, v) < n_hard) {
        n_hard = 0;
        const float pl2 = pref.x * pref.x + pref.y * pref.y;
        const float k = pl2 > vmax * vmax ? vmax * rsqrtf(pl2) : 1.f;
        v = make_float2(pref.x * k, pref.y * k);
    }
    float dist = -INFINITY;
    for (int i = n_hard; i < n; ++i) {
        const Line li = L[i];
        const float viol = -((v.x - li.qx) * li.nx + (v.y - li.qy) * li.ny);
        if (viol > dist) {
            const float ci = li.qx * li.nx + li.qy * li.ny;
            for (int m = lane; m < i; m += 32) {
                if (m < n_hard) {
                    S[m] = L[m];
                } else {
                    const Line lj = L[m];
                    float nx = lj.nx - li.nx, ny = lj.ny - li.ny;
                    const float nl2 = nx * nx + ny * ny;
                    if (nl2 < 1e-12f) {
                        S[m] = Line{0.f, 0.f, 0.f, 0.f};
                    } else {
                        const float inv = rsqrtf(nl2);
                        nx *= inv;
                        ny *= inv;
                        const float c = ((lj.qx * lj.nx + lj.qy * lj.ny) - ci) * inv;
                        S[m] = Line{c * nx, c * ny, nx, ny};
                    }
                }
            }
            __syncwarp();
            float2 t;
            if (coop_lp_dir(S, i, vmax, li.nx, li.ny, pref, t)) v = t;
            dist = -((v.x - li.qx) * li.nx + (v.y - li.qy) * li.ny);
            __syncwarp();
        }
    }
    return v;
}

}  // namespace crowd
