/*
 * FP64 CPU oracle for the batched ORCA crowd step.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the timed CPU
 * baseline of the benchmark may load this library; the product path never
 * calls it and shares no code with it.
 *
 * What it computes: the per-step update of the dynamic agents of the paper's
 * simulator (Sec. 3.2, "Interactive Dynamics Generation": agents adjust their
 * positions each step from proximity and relative velocity, with ORCA as the
 * collision-avoidance rule, avoiding both static and dynamic objects and
 * reacting to the trained robot).  The ORCA geometry is the cited method's
 * (van den Berg et al., "Reciprocal n-body collision avoidance", ISRR 2011):
 * truncated velocity obstacles, reciprocal half-planes, a per-agent linear
 * program with a min-max-penetration fallback.  Each stage below is written
 * plainly, in FP64, agent by agent, with no blocking or reordering.  Build
 * with -ffp-contract=off so that the neighbour ranking key rounds exactly as
 * written (Stage O2).
 *
 * Readings taken where the paper is silent (each one is listed with the
 * design notes): the "arrive exactly" preferred velocity (O1); neighbour
 * ranking by (FP64 squared distance, id) capped at K (O2); the right leg on a
 * det = 0 tie and the colliding-case degenerate normals (O3); the
 * "tangent at the nearest velocity-obstacle point" static-segment line with
 * full responsibility (O4); obstacle lines before agent lines in the LP (O5);
 * the fallback as min-max penetration, ties broken by distance to the
 * preferred velocity (O6).
 *
 * Parity pins: the closed forms (lone agent, symmetric head-on pair),
 * brute-force vertex enumeration of the LP, the corridor and equilateral
 * fallback closed forms, brute-force geometry of the velocity obstacle and the
 * half-plane / speed / no-overlap invariants all live in the tests.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_EPS_GOAL 1e-6 /* O1: distance under which the agent has arrived */
#define OR_EPS_PAR 1e-9  /* O5: |det| at or below which two lines are parallel */
#define OR_MAX_K 32
#define OR_COLLIDE_DEPTH 1e-3 /* O8: penetration counted as a collision, metres */

typedef struct {
    double tau;         /* time horizon for agents */
    double tau_obst;    /* time horizon for static segments (0 => tau) */
    double neighbor_dist; /* R */
    double dt;
    double robot_alpha; /* share of responsibility an agent takes against the robot */
    int32_t max_neighbors; /* K */
    int32_t seg_mode;   /* 0: O4 segment half-plane; 1: O4v velocity-dependent */
} or_params;

typedef struct {
    double qx, qy; /* a point on the boundary line */
    double nx, ny; /* unit normal pointing into the allowed side: (v - q).n >= 0 */
} or_line;

/* ---------------------------------------------------------------- O1 ---- */
/* Preferred velocity toward the goal, stopping exactly on it. */
void or_pref_velocity(double px, double py, double gx, double gy, double speed, double dt,
                      double* vx, double* vy)
{
    double dx = gx - px, dy = gy - py;
    double dist = sqrt(dx * dx + dy * dy);
    if (dist < OR_EPS_GOAL) {
        *vx = 0.0; *vy = 0.0;
    } else if (dist <= speed * dt) {
        *vx = dx / dt; *vy = dy / dt;
    } else {
        *vx = speed * dx / dist; *vy = speed * dy / dist;
    }
}

/* ---------------------------------------------------------------- O2 ---- */
/* Ranking key of neighbour j seen from agent i: squared distance, each
 * product and the sum rounded to FP64 (no fused multiply-add). */
double or_rank_key(double xi, double yi, double xj, double yj)
{
    double dx = xj - xi;
    double dy = yj - yi;
    double ax = dx * dx;
    double ay = dy * dy;
    return ax + ay;
}

typedef struct { double key; int32_t id; } or_cand;

static int or_cand_cmp(const void* a, const void* b)
{
    const or_cand* x = (const or_cand*)a;
    const or_cand* y = (const or_cand*)b;
    if (x->key < y->key) return -1;
    if (x->key > y->key) return 1;
    return (x->id > y->id) - (x->id < y->id);
}

/* All agents j != i of the env with key < R^2, ordered by (key, j), first K
 * kept.  ids are env-local.  Returns the count; *in_range (if given) gets
 * the number of agents with key < R^2 before the cap. */
static int neighbors_counted(int n, const double* pos, int i, double R, int K, int32_t* out_ids, double* out_keys,
                             int* in_range)
{
    or_cand* c = (or_cand*)malloc(sizeof(or_cand) * (size_t)(n > 0 ? n : 1));
    int m = 0;
    double R2 = R * R;
    for (int j = 0; j < n; ++j) {
        if (j == i) continue;
        double k = or_rank_key(pos[2 * i], pos[2 * i + 1], pos[2 * j], pos[2 * j + 1]);
        if (k < R2) { c[m].key = k; c[m].id = j; ++m; }
    }
    qsort(c, (size_t)m, sizeof(or_cand), or_cand_cmp);
    int cnt = m < K ? m : K;
    for (int t = 0; t < cnt; ++t) {
        out_ids[t] = c[t].id;
        if (out_keys) out_keys[t] = c[t].key;
    }
    free(c);
    if (in_range) *in_range = m;
    return cnt;
}

int or_neighbors(int n, const double* pos, int i, double R, int K, int32_t* out_ids, double* out_keys)
{
    return neighbors_counted(n, pos, i, R, K, out_ids, out_keys, NULL);
}

/* Closest point of segment [a,b] to p. */
static void or_closest_on_segment(double px, double py, const double* s, double* cx, double* cy)
{
    double ex = s[2] - s[0], ey = s[3] - s[1];
    double t = ((px - s[0]) * ex + (py - s[1]) * ey) / (ex * ex + ey * ey);
    if (t < 0.0) t = 0.0;
    if (t > 1.0) t = 1.0;
    *cx = s[0] + t * ex;
    *cy = s[1] + t * ey;
}

double or_seg_dist2(double px, double py, const double* s)
{
    double cx, cy;
    or_closest_on_segment(px, py, s, &cx, &cy);
    return (px - cx) * (px - cx) + (py - cy) * (py - cy);
}

/* Segments whose squared distance from p is below (r + tau_o * vmax)^2,
 * ordered by (squared distance, segment id). */
int or_obstacles(int ns, const double* segs, double px, double py, double reach, int32_t* out_ids)
{
    or_cand* c = (or_cand*)malloc(sizeof(or_cand) * (size_t)(ns > 0 ? ns : 1));
    int m = 0;
    for (int s = 0; s < ns; ++s) {
        double d2 = or_seg_dist2(px, py, segs + 4 * s);
        if (d2 < reach * reach) { c[m].key = d2; c[m].id = s; ++m; }
    }
    qsort(c, (size_t)m, sizeof(or_cand), or_cand_cmp);
    for (int t = 0; t < m; ++t) out_ids[t] = c[t].id;
    free(c);
    return m;
}

/* ---------------------------------------------------------------- O3 ---- */
/* Reciprocal half-plane of agent i against agent j.
 *   p = p_j - p_i, v = v_i - v_j, r = r_i + r_j.
 *   u = (closest point of the boundary of the truncated velocity obstacle to
 *        v) - v, n = outward normal there;
 *   line: (v' - (v_i + alpha u)) . n >= 0.
 * Not colliding: horizon tau; colliding: horizon dt, the obstacle is then the
 * disk D(p/dt, r/dt).  id_i/id_j only break the p = 0 tie. */
void or_agent_line(double pix, double piy, double vix, double viy, double ri,
                   double pjx, double pjy, double vjx, double vjy, double rj,
                   double tau, double dt, double alpha, int id_i, int id_j, or_line* out)
{
    double px = pjx - pix, py = pjy - piy;
    double vx = vix - vjx, vy = viy - vjy;
    double r = ri + rj;
    double dist2 = px * px + py * py;
    double r2 = r * r;
    double ux, uy, nx, ny;

    if (dist2 > r2) {
        /* w: relative velocity measured from the centre of the cut-off disk D(p/tau, r/tau) */
        double wx = vx - px / tau, wy = vy - py / tau;
        double w2 = wx * wx + wy * wy;
        double wp = wx * px + wy * py;
        if (wp < 0.0 && wp * wp > r2 * w2) {
            /* nearest boundary point lies on the cut-off arc */
            double wl = sqrt(w2);
            double wnx = wx / wl, wny = wy / wl;
            ux = (r / tau - wl) * wnx;
            uy = (r / tau - wl) * wny;
            nx = wnx; ny = wny;
        } else {
            /* nearest boundary point lies on a leg: the rays from 0 tangent to D(p, r) */
            double leg = sqrt(dist2 - r2);
            double lx, ly;
            double det = px * wy - py * wx;
            if (det > 0.0) {
                /* left leg: p rotated counter-clockwise by asin(r/|p|) */
                lx = (px * leg - py * r) / dist2;
                ly = (px * r + py * leg) / dist2;
                nx = -ly; ny = lx;
            } else {
                /* right leg: p rotated clockwise by asin(r/|p|) */
                lx = (px * leg + py * r) / dist2;
                ly = (-px * r + py * leg) / dist2;
                nx = ly; ny = -lx;
            }
            double s = vx * lx + vy * ly;
            ux = s * lx - vx;
            uy = s * ly - vy;
        }
    } else {
        /* colliding: leave the disk D(p/dt, r/dt) within one step */
        double wx = vx - px / dt, wy = vy - py / dt;
        double wl = sqrt(wx * wx + wy * wy);
        double wnx, wny;
        if (wl > 0.0) {
            wnx = wx / wl; wny = wy / wl;
        } else if (dist2 > 0.0) {
            double pl = sqrt(dist2);
            wnx = -px / pl; wny = -py / pl;
        } else {
            wnx = id_i < id_j ? 1.0 : -1.0; wny = 0.0;
        }
        ux = (r / dt - wl) * wnx;
        uy = (r / dt - wl) * wny;
        nx = wnx; ny = wny;
    }
    out->qx = vix + alpha * ux;
    out->qy = viy + alpha * uy;
    out->nx = nx;
    out->ny = ny;
}

/* ---------------------------------------------------------------- O4 ---- */
/* Half-plane of agent i against the static segment s (full responsibility):
 * the tangent to the truncated velocity obstacle at its point nearest the
 * origin, v'.m <= (d - r)/tau_o with m the unit vector from p to the closest
 * point; overlapping (d <= r): v'.m <= max((d - r)/dt, -vmax).  d = 0: m is
 * the segment normal on the side away from where the agent came from (the
 * side its current velocity points to), the left normal of a->b when that is
 * undecided. */
void or_obstacle_line(double px, double py, double vx, double vy, double r, double vmax,
                      const double* s, double tau_o, double dt, or_line* out)
{
    double cx, cy;
    or_closest_on_segment(px, py, s, &cx, &cy);
    double dx = cx - px, dy = cy - py;
    double d = sqrt(dx * dx + dy * dy);
    double mx, my;
    if (d > 0.0) {
        mx = dx / d; my = dy / d;
    } else {
        double ex = s[2] - s[0], ey = s[3] - s[1];
        double el = sqrt(ex * ex + ey * ey);
        double lx = -ey / el, ly = ex / el; /* left normal of a->b */
        if (vx * lx + vy * ly >= 0.0) { mx = lx; my = ly; } else { mx = -lx; my = -ly; }
    }
    double b;
    if (d > r) {
        b = (d - r) / tau_o;
    } else {
        b = (d - r) / dt;
        if (b < -vmax) b = -vmax;
    }
    /* v'.m <= b  <=>  (v' - b m).(-m) >= 0 */
    out->qx = b * mx;
    out->qy = b * my;
    out->nx = -mx;
    out->ny = -my;
}

/* ---------------------------------------------------------------- O4v --- */
/* Velocity-dependent half-plane of agent p (radius r, velocity v) against
 * segment s (the obstacle treatment of the method the paper cites, for one
 * segment on its own).  When the agent is clear of the segment (d > r):
 *   C = the capsule [a - p, b - p] + D(r); its truncated velocity obstacle
 *   is the union of s*C for s >= 1/tau_o, bounded by the two legs (the rays
 *   from 0 tangent to C, beyond the tangent points) and by the part of
 *   C/tau_o that faces 0 (outward normal u with u.X < 0).  X = the point of
 *   that boundary nearest v, n = the outward normal there; the agent takes
 *   the whole responsibility: (v' - X).n >= 0.  Candidates, each the nearest
 *   point of one piece: the flat side of C/tau_o towards 0 (when it faces
 *   0), the two end-cap arcs that face 0 (the radial point, when it lies on
 *   the arc; otherwise an end of the arc, which the flat side or a leg
 *   covers), and the two leg rays; the first of equally near pieces wins
 *   (flat, cap a, cap b, left, right).
 * When it overlaps (d <= r): as O4. */
static void or_leg(double X0, double X1, double r, int left, double* ux, double* uy, double* len)
{
    double d2 = X0 * X0 + X1 * X1;
    double l = sqrt(d2 - r * r);
    if (left) { *ux = (X0 * l - X1 * r) / d2; *uy = (X0 * r + X1 * l) / d2; }
    else      { *ux = (X0 * l + X1 * r) / d2; *uy = (-X0 * r + X1 * l) / d2; }
    *len = l;
}

void or_obstacle_line_vd(double px, double py, double vx, double vy, double r, double vmax,
                         const double* s, double tau_o, double dt, or_line* out)
{
    double cx, cy;
    or_closest_on_segment(px, py, s, &cx, &cy);
    double dx = cx - px, dy = cy - py;
    if (sqrt(dx * dx + dy * dy) <= r) {
        or_obstacle_line(px, py, vx, vy, r, vmax, s, tau_o, dt, out);
        return;
    }
    double A0 = s[0] - px, A1 = s[1] - py, B0 = s[2] - px, B1 = s[3] - py;
    /* legs: of the two end disks' tangents, the outermost on each side */
    double la0, la1, lal, lb0, lb1, lbl, ra0, ra1, ral, rb0, rb1, rbl;
    or_leg(A0, A1, r, 1, &la0, &la1, &lal);
    or_leg(B0, B1, r, 1, &lb0, &lb1, &lbl);
    or_leg(A0, A1, r, 0, &ra0, &ra1, &ral);
    or_leg(B0, B1, r, 0, &rb0, &rb1, &rbl);
    double L0, L1, Ll, R0, R1, Rl;
    if (la0 * lb1 - la1 * lb0 > 0.0) { L0 = lb0; L1 = lb1; Ll = lbl; } else { L0 = la0; L1 = la1; Ll = lal; }
    if (ra0 * rb1 - ra1 * rb0 < 0.0) { R0 = rb0; R1 = rb1; Rl = rbl; } else { R0 = ra0; R1 = ra1; Rl = ral; }
    double best = INFINITY, X0 = 0.0, X1 = 0.0, N0 = 0.0, N1 = 0.0;
    /* the part of C / tau_o that faces 0: the flat side towards 0 (if it
     * faces 0) and the arcs of the two end caps that face 0 */
    {
        double rt = r / tau_o;
        double a0 = A0 / tau_o, a1 = A1 / tau_o, b0 = B0 / tau_o, b1 = B1 / tau_o;
        double e0 = B0 - A0, e1 = B1 - A1, el = sqrt(e0 * e0 + e1 * e1);
        if (el > 0.0) {
            double m0 = -e1 / el, m1 = e0 / el;       /* unit normal of the segment, towards 0 */
            if (m0 * A0 + m1 * A1 > 0.0) { m0 = -m0; m1 = -m1; }
            if (m0 * A0 + m1 * A1 < -r) {            /* the flat side faces 0 */
                double f0 = a0 + rt * m0, f1 = a1 + rt * m1, g0 = b0 - a0, g1 = b1 - a1;
                double t = ((vx - f0) * g0 + (vy - f1) * g1) / (g0 * g0 + g1 * g1);
                if (t < 0.0) t = 0.0;
                if (t > 1.0) t = 1.0;
                double x0 = f0 + t * g0, x1 = f1 + t * g1;
                double dd = sqrt((vx - x0) * (vx - x0) + (vy - x1) * (vy - x1));
                if (dd < best) { best = dd; X0 = x0; X1 = x1; N0 = m0; N1 = m1; }
            }
        }
        for (int cap = 0; cap < 2; ++cap) {
            double c0 = cap ? b0 : a0, c1 = cap ? b1 : a1;        /* cap centre (scaled) */
            double o0 = cap ? A0 - B0 : B0 - A0, o1 = cap ? A1 - B1 : B1 - A1; /* towards the other end */
            double w0 = vx - c0, w1 = vy - c1, wl = sqrt(w0 * w0 + w1 * w1);
            if (!(wl > 0.0)) continue;
            double u0 = w0 / wl, u1 = w1 / wl;
            /* on this cap's half circle, and facing 0: u.(centre) < -r/tau_o */
            if (u0 * o0 + u1 * o1 > 0.0) continue;
            if (!(u0 * c0 + u1 * c1 < -rt)) continue;
            double dd = fabs(wl - rt);
            if (dd < best) { best = dd; X0 = c0 + rt * u0; X1 = c1 + rt * u1; N0 = u0; N1 = u1; }
        }
    }
    /* left leg: outward normal to its left */
    {
        double t = vx * L0 + vy * L1, tmin = Ll / tau_o;
        if (t < tmin) t = tmin;
        double x0 = t * L0, x1 = t * L1;
        double dd = sqrt((vx - x0) * (vx - x0) + (vy - x1) * (vy - x1));
        if (dd < best) { best = dd; X0 = x0; X1 = x1; N0 = -L1; N1 = L0; }
    }
    /* right leg: outward normal to its right */
    {
        double t = vx * R0 + vy * R1, tmin = Rl / tau_o;
        if (t < tmin) t = tmin;
        double x0 = t * R0, x1 = t * R1;
        double dd = sqrt((vx - x0) * (vx - x0) + (vy - x1) * (vy - x1));
        if (dd < best) { best = dd; X0 = x0; X1 = x1; N0 = R1; N1 = -R0; }
    }
    out->qx = X0;
    out->qy = X1;
    out->nx = N0;
    out->ny = N1;
}

/* O4v, segments already taken care of: segment s is given no line when an
 * earlier segment line of the agent (one that leaves 0 allowed) forbids both
 * end disks of s's cutoff capsule, (X - q).n + r/tau_o <= OR_EPS_COVERED for
 * X = (a - p)/tau_o and (b - p)/tau_o: the whole velocity obstacle of s then
 * lies in that line's forbidden half-plane (it is the union of the cutoff
 * capsule scaled away from 0).  The agent must be clear of s. */
#define OR_EPS_COVERED 1e-5
int or_segment_covered(double px, double py, double r, const double* s, double tau_o, const or_line* L,
                              int m)
{
    double cx, cy;
    or_closest_on_segment(px, py, s, &cx, &cy);
    if (sqrt((cx - px) * (cx - px) + (cy - py) * (cy - py)) <= r) return 0;
    double a0 = (s[0] - px) / tau_o, a1 = (s[1] - py) / tau_o, b0 = (s[2] - px) / tau_o, b1 = (s[3] - py) / tau_o;
    double rt = r / tau_o;
    for (int l = 0; l < m; ++l) {
        if (-(L[l].qx * L[l].nx + L[l].qy * L[l].ny) < -OR_EPS_COVERED) continue;  /* 0 not allowed */
        double va = (a0 - L[l].qx) * L[l].nx + (a1 - L[l].qy) * L[l].ny + rt;
        double vb = (b0 - L[l].qx) * L[l].nx + (b1 - L[l].qy) * L[l].ny + rt;
        if (va <= OR_EPS_COVERED && vb <= OR_EPS_COVERED) return 1;
    }
    return 0;
}

/* ---------------------------------------------------------------- O5 ---- */
/* Minimise |v' - pref| on line k, inside the disk of radius vmax and the
 * previous lines 0..k-1.  Returns 0 if that set is empty. */
static int or_lp1(const or_line* L, int k, double vmax, double prefx, double prefy,
                  double* vx, double* vy)
{
    const or_line* lk = &L[k];
    /* direction along line k */
    double dx = -lk->ny, dy = lk->nx;
    double qd = lk->qx * dx + lk->qy * dy;
    double disc = qd * qd - (lk->qx * lk->qx + lk->qy * lk->qy) + vmax * vmax;
    if (disc < 0.0) return 0;
    double sq = sqrt(disc);
    double tl = -qd - sq, tr = -qd + sq;
    for (int l = 0; l < k; ++l) {
        const or_line* ll = &L[l];
        double den = dx * ll->nx + dy * ll->ny; /* det(n_k, n_l) */
        double num = (ll->qx - lk->qx) * ll->nx + (ll->qy - lk->qy) * ll->ny;
        if (fabs(den) <= OR_EPS_PAR) {
            if (num > 0.0) return 0; /* line k lies wholly outside line l */
            continue;
        }
        double t = num / den;
        if (den > 0.0) { if (t > tl) tl = t; }
        else { if (t < tr) tr = t; }
        if (tl > tr) return 0;
    }
    double t = (prefx - lk->qx) * dx + (prefy - lk->qy) * dy;
    if (t < tl) t = tl;
    if (t > tr) t = tr;
    *vx = lk->qx + t * dx;
    *vy = lk->qy + t * dy;
    return 1;
}

/* Incremental 2D LP: argmin |v' - pref| over the disk and lines 0..n-1.
 * Returns n when feasible, else the index of the line at which it failed
 * (v holds the last feasible iterate then).  When given, *solves counts the
 * lines found violated (each starts a 1D solve on it) and *solve_lines the
 * earlier lines those solves take into account. */
static int lp2_counted(const or_line* L, int n, double vmax, double prefx, double prefy, double* vx, double* vy,
                       int64_t* solves, int64_t* solve_lines)
{
    double pl2 = prefx * prefx + prefy * prefy;
    if (pl2 > vmax * vmax) {
        double pl = sqrt(pl2);
        *vx = prefx / pl * vmax; *vy = prefy / pl * vmax;
    } else {
        *vx = prefx; *vy = prefy;
    }
    for (int k = 0; k < n; ++k) {
        double s = (*vx - L[k].qx) * L[k].nx + (*vy - L[k].qy) * L[k].ny;
        if (s < 0.0) {
            double nx, ny;
            if (solves) { *solves += 1; *solve_lines += k; }
            if (!or_lp1(L, k, vmax, prefx, prefy, &nx, &ny)) return k;
            *vx = nx; *vy = ny;
        }
    }
    return n;
}

int or_lp2(const or_line* L, int n, double vmax, double prefx, double prefy, double* vx, double* vy)
{
    return lp2_counted(L, n, vmax, prefx, prefy, vx, vy, NULL, NULL);
}

/* ---------------------------------------------------------------- O6 ---- */
/* Fallback when the LP is infeasible.  H = the first n_hard lines (static
 * obstacles), A = the rest (agents), viol_k(v) = -(v - q_k).n_k.
 *   d* = min over v in disk & H of max_k viol_k(v);
 *   result = the point of disk & H & {viol_k <= d*} closest to pref.
 * If disk & H is empty, H joins A.  d* is found by bisection on the
 * feasibility of the relaxed LP; the result is that LP at the upper end of
 * the final bracket.  Writes d* (the bracket's upper end) if dstar != NULL. */
void or_fallback(const or_line* L, int n, int n_hard, double vmax, double prefx, double prefy,
                 double* vx, double* vy, double* dstar)
{
    or_line* S = (or_line*)malloc(sizeof(or_line) * (size_t)(n > 0 ? n : 1));
    double v0x, v0y;
    int nh = n_hard;
    memcpy(S, L, sizeof(or_line) * (size_t)n);
    if (or_lp2(S, nh, vmax, prefx, prefy, &v0x, &v0y) < nh) {
        nh = 0; /* the static lines alone leave nothing: make them soft as well */
        double pl2 = prefx * prefx + prefy * prefy;
        if (pl2 > vmax * vmax) {
            double pl = sqrt(pl2);
            v0x = prefx / pl * vmax; v0y = prefy / pl * vmax;
        } else {
            v0x = prefx; v0y = prefy;
        }
    }
    double hi = 0.0;
    for (int k = nh; k < n; ++k) {
        double vk = -((v0x - L[k].qx) * L[k].nx + (v0y - L[k].qy) * L[k].ny);
        if (vk > hi) hi = vk;
    }
    hi += 1e-12;
    double lo = 0.0;
    for (int it = 0; it < 200 && hi - lo > 1e-13 * (hi > 1.0 ? hi : 1.0); ++it) {
        double mid = 0.5 * (lo + hi);
        for (int k = nh; k < n; ++k) {
            S[k].qx = L[k].qx - mid * L[k].nx;
            S[k].qy = L[k].qy - mid * L[k].ny;
        }
        double tx, ty;
        if (or_lp2(S, n, vmax, prefx, prefy, &tx, &ty) == n) hi = mid;
        else lo = mid;
    }
    for (int k = nh; k < n; ++k) {
        S[k].qx = L[k].qx - hi * L[k].nx;
        S[k].qy = L[k].qy - hi * L[k].ny;
    }
    if (or_lp2(S, n, vmax, prefx, prefy, vx, vy) < n) {
        /* cannot happen for a feasible upper end; keep the last iterate */
    }
    if (dstar) *dstar = hi;
    free(S);
}

/* --------------------------------------------------------- O1..O7 step -- */
/* One simultaneous step of every selected agent (all agents if sel == NULL).
 * Agents are env-major: env e owns agents [env_start[e], env_start[e+1]) and
 * segments [seg_start[e], seg_start[e+1]).  The robot slot of env e
 * (robot_index[e] >= 0, env-local) moves with robot_vel[e] and is not solved;
 * every other agent sees that commanded velocity.
 * Outputs (indexed by global agent id, only selected agents written):
 *   pos_out/vel_out [N][2]; nbr_out [N][K] env-local ids, -1 padded (may be
 *   NULL); status_out [N]: 0 LP feasible, 1 fallback, 2 robot, 3 vehicle (may be NULL).
 * kind [N] (may be NULL): 1 marks a vehicle, which keeps its given velocity
 * (set by its lane model) and which the others avoid with full
 * responsibility.
 * work [8] (may be NULL): work items of this step added in, for the operation
 * count of the step: agent updates, pairs j != i within R (key < R^2), agent
 * lines, segment lines, LP line checks, LP 1D solves, earlier lines those
 * solves take into account, infeasible LPs (fallbacks).
 * Returns 0, or -1 on bad arguments. */
int or_step(int32_t n_envs, const int64_t* env_start, const double* radius, const double* vmax,
            const double* pref_speed, const int32_t* robot_index, const int64_t* seg_start,
            const double* segs, const or_params* prm, const double* pos, const double* vel,
            const double* goal, const double* robot_vel, const int32_t* kind, int64_t n_sel, const int64_t* sel,
            double* pos_out, double* vel_out, int32_t* nbr_out, int32_t* status_out, int n_threads,
            int64_t* work)
{
    if (!prm || prm->max_neighbors < 0 || prm->max_neighbors > OR_MAX_K) return -1;
    const int K = prm->max_neighbors;
    const double tau_o = prm->tau_obst > 0.0 ? prm->tau_obst : prm->tau;
    int64_t n_total = env_start[n_envs];
    int64_t count = sel ? n_sel : n_total;
    int bad = 0;
    int64_t w_steps = 0, w_pairs = 0, w_alines = 0, w_olines = 0, w_checks = 0, w_solves = 0, w_solve_lines = 0,
            w_fallbacks = 0;
#ifdef _OPENMP
    if (n_threads > 0) omp_set_num_threads(n_threads);
#pragma omp parallel for schedule(dynamic, 8) \
    reduction(| : bad) reduction(+ : w_steps, w_pairs, w_alines, w_olines, w_checks, w_solves, w_solve_lines, w_fallbacks)
#endif
    for (int64_t t = 0; t < count; ++t) {
        int64_t g = sel ? sel[t] : t;
        if (g < 0 || g >= n_total) { bad |= 1; continue; }
        /* env of agent g */
        int e = 0, lo = 0, hi = n_envs - 1;
        while (lo <= hi) {
            int mid = (lo + hi) / 2;
            if (env_start[mid] <= g) { e = mid; lo = mid + 1; } else hi = mid - 1;
        }
        int64_t base = env_start[e];
        int n = (int)(env_start[e + 1] - base);
        int i = (int)(g - base);
        int robot = robot_index ? robot_index[e] : -1;

        /* step-start state of the env; the robot's velocity is its command */
        const double* P = pos + 2 * base;
#define OR_VEL(j, c) ((j) == robot ? robot_vel[2 * e + (c)] : vel[2 * (base + (j)) + (c)])

        int32_t ids[OR_MAX_K];
        int in_range = 0;
        int nn = neighbors_counted(n, P, i, prm->neighbor_dist, K, ids, NULL, &in_range);
        w_steps += 1;
        w_pairs += in_range;
        if (nbr_out) {
            for (int k = 0; k < K; ++k) nbr_out[g * K + k] = k < nn ? ids[k] : -1;
        }

        double nvx, nvy;
        int status = 0;
        if (i == robot) {
            nvx = OR_VEL(i, 0); nvy = OR_VEL(i, 1);
            status = 2;
        } else if (kind && kind[g] == 1) {
            /* a vehicle: moved by its lane model, not solved */
            nvx = OR_VEL(i, 0); nvy = OR_VEL(i, 1);
            status = 3;
        } else {
            double prefx, prefy;
            or_pref_velocity(P[2 * i], P[2 * i + 1], goal[2 * g], goal[2 * g + 1], pref_speed[g],
                             prm->dt, &prefx, &prefy);
            int ns = (int)(seg_start[e + 1] - seg_start[e]);
            const double* S = segs + 4 * seg_start[e];
            int32_t* oids = (int32_t*)malloc(sizeof(int32_t) * (size_t)(ns > 0 ? ns : 1));
            int no = or_obstacles(ns, S, P[2 * i], P[2 * i + 1], radius[g] + tau_o * vmax[g], oids);
            or_line* L = (or_line*)malloc(sizeof(or_line) * (size_t)(no + nn + 1));
            int kept = 0;
            for (int k = 0; k < no; ++k) {
                const double* sg = S + 4 * oids[k];
                if (prm->seg_mode == 1) {
                    if (or_segment_covered(P[2 * i], P[2 * i + 1], radius[g], sg, tau_o, L, kept)) continue;
                    or_obstacle_line_vd(P[2 * i], P[2 * i + 1], OR_VEL(i, 0), OR_VEL(i, 1), radius[g], vmax[g], sg,
                                        tau_o, prm->dt, &L[kept]);
                } else {
                    or_obstacle_line(P[2 * i], P[2 * i + 1], OR_VEL(i, 0), OR_VEL(i, 1), radius[g], vmax[g], sg,
                                     tau_o, prm->dt, &L[kept]);
                }
                ++kept;
            }
            no = kept;
            for (int k = 0; k < nn; ++k) {
                int j = ids[k];
                /* half the avoidance against another agent, the robot's share
                 * against the robot, all of it against a vehicle */
                double alpha = (j == robot) ? prm->robot_alpha : (kind && kind[base + j] == 1) ? 1.0 : 0.5;
                or_agent_line(P[2 * i], P[2 * i + 1], OR_VEL(i, 0), OR_VEL(i, 1), radius[g],
                              P[2 * j], P[2 * j + 1], OR_VEL(j, 0), OR_VEL(j, 1), radius[base + j],
                              prm->tau, prm->dt, alpha, i, j, &L[no + k]);
            }
            int nl = no + nn;
            int64_t solves = 0, solve_lines = 0;
            if (lp2_counted(L, nl, vmax[g], prefx, prefy, &nvx, &nvy, &solves, &solve_lines) < nl) {
                or_fallback(L, nl, no, vmax[g], prefx, prefy, &nvx, &nvy, NULL);
                status = 1;
                w_fallbacks += 1;
            }
            w_alines += nn;
            w_olines += no;
            w_checks += nl;
            w_solves += solves;
            w_solve_lines += solve_lines;
            free(L);
            free(oids);
        }
        vel_out[2 * g] = nvx;
        vel_out[2 * g + 1] = nvy;
        pos_out[2 * g] = P[2 * i] + prm->dt * nvx;
        pos_out[2 * g + 1] = P[2 * i + 1] + prm->dt * nvy;
        if (status_out) status_out[g] = status;
#undef OR_VEL
    }
    if (work) {
        work[0] += w_steps;
        work[1] += w_pairs;
        work[2] += w_alines;
        work[3] += w_olines;
        work[4] += w_checks;
        work[5] += w_solves;
        work[6] += w_solve_lines;
        work[7] += w_fallbacks;
    }
    return bad ? -1 : 0;
}

/* ---------------------------------------------------------------- O8 ---- */
/* Collision events of one post-integration state, per env: pairs i < j with
 * |p_i - p_j| < r_i + r_j - OR_COLLIDE_DEPTH and agent-segment pairs with
 * distance < r_i - OR_COLLIDE_DEPTH (the collision indicator of the paper's
 * metric table, counted from a penetration depth of 1 mm so that agents left
 * exactly touching by ORCA are not counted on rounding noise). */
void or_collisions(int32_t n_envs, const int64_t* env_start, const double* radius,
                   const int64_t* seg_start, const double* segs, const double* pos,
                   int64_t* agent_pairs_out, int64_t* seg_pairs_out)
{
    for (int e = 0; e < n_envs; ++e) {
        int64_t a = 0, s = 0;
        for (int64_t i = env_start[e]; i < env_start[e + 1]; ++i) {
            for (int64_t j = i + 1; j < env_start[e + 1]; ++j) {
                double dx = pos[2 * j] - pos[2 * i], dy = pos[2 * j + 1] - pos[2 * i + 1];
                double lim = radius[i] + radius[j] - OR_COLLIDE_DEPTH;
                if (sqrt(dx * dx + dy * dy) < lim) ++a;
            }
            for (int64_t k = seg_start[e]; k < seg_start[e + 1]; ++k) {
                double d = sqrt(or_seg_dist2(pos[2 * i], pos[2 * i + 1], segs + 4 * k));
                if (d < radius[i] - OR_COLLIDE_DEPTH) ++s;
            }
        }
        agent_pairs_out[e] = a;
        seg_pairs_out[e] = s;
    }
}

int or_abi_version(void) { return 1; }
