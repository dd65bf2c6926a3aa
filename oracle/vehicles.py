"""FP64 oracle of the lane-following vehicles (test infrastructure).

The paper's city scenes run vehicles beside the ORCA crowd, "controlled by
IDM policy" (the Intelligent Driver Model of Treiber, Hennecke and Helbing,
Phys. Rev. E 62, 2000), in the appendix's description of its Urban-Tra-City
scene.  This module states one step of such vehicles plainly:

  - each vehicle follows a closed lane polyline at arc position s with speed
    v >= 0;
  - its leader is the nearest thing ahead on its lane: another vehicle of
    the lane (arc distance ds in (0, L], gap ds - (len_i + len_j)/2,
    approach rate v_i - v_j), or an agent of the crowd (pedestrian or robot)
    whose closest point on a lane segment lies within half_width + r of the
    lane and at most `lookahead` ahead (gap ds - len_i/2 - r, approach rate
    v_i: it counts as standing still);
  - IDM acceleration a (1 - (v/v0)^4 - (s*/gap)^2) with
    s* = s0 + max(0, v T + v dv / (2 sqrt(a b))), the interaction term
    dropped when nothing is ahead, the gap floored at 0.01 m;
  - v' = max(0, v + acc dt), s' = s + v' dt (wrapped onto [0, L)); during the
    step the vehicle is the crowd agent at p(s) with velocity
    (p(s') - p(s)) / dt, which every pedestrian avoids with full
    responsibility.

Only tests/ import this module; the product path never does.
"""
from __future__ import annotations

import math

import numpy as np


class Lanes:
    """Closed polylines: lane l has points pts[start[l]:start[l+1]] (FP32
    values held in FP64) and segment k runs from point k to point k + 1
    (the last one back to point 0)."""

    def __init__(self, points, lane_start):
        self.pts = np.asarray(points, np.float32).astype(np.float64).reshape(-1, 2)
        self.start = np.asarray(lane_start, np.int64)
        self.seg = []   # per lane: (a [m,2], e [m,2], length [m], cumulative [m+1])
        for l in range(len(self.start) - 1):
            p = self.pts[self.start[l]:self.start[l + 1]]
            a = p
            b = np.roll(p, -1, axis=0)
            e = b - a
            ln = np.sqrt(e[:, 0] * e[:, 0] + e[:, 1] * e[:, 1])
            cum = np.zeros(len(p) + 1)
            for k in range(len(p)):
                cum[k + 1] = cum[k] + ln[k]
            self.seg.append((a, e, ln, cum))

    def length(self, l):
        return self.seg[l][3][-1]

    def point(self, l, s):
        a, e, ln, cum = self.seg[l]
        k = int(np.searchsorted(cum, s, side="right") - 1)
        k = min(max(k, 0), len(ln) - 1)
        t = (s - cum[k]) / ln[k]
        return a[k] + t * e[k]


def idm_step(lanes, veh_lane, veh_s, veh_v, veh_params, agents_pos, agents_r, blocker_mask, half_width, lookahead, dt):
    """One step of all vehicles (one environment's).  veh_params [V][6]:
    (v0, T, a, b, s0, length).  blocker_mask [M] selects the crowd agents
    that can block (pedestrians and the robot).  Returns (s', v', p(s), p(s'),
    velocity during the step)."""
    V = len(veh_s)
    s_new, v_new = np.zeros(V), np.zeros(V)
    p_now, p_next, vel = np.zeros((V, 2)), np.zeros((V, 2)), np.zeros((V, 2))
    q_all = np.asarray(agents_pos, np.float64).reshape(-1, 2)
    r_all = np.asarray(agents_r, np.float64).reshape(-1)
    for i in range(V):
        l = int(veh_lane[i])
        L = lanes.length(l)
        s, v = float(veh_s[i]), float(veh_v[i])
        v0, T, a, b, s0, length = (float(x) for x in veh_params[i])
        best_ds, gap, dv = math.inf, None, None
        for j in range(V):
            if j == i or int(veh_lane[j]) != l:
                continue
            ds = float(veh_s[j]) - s
            if ds <= 0.0:
                ds += L
            if ds < best_ds:
                best_ds = ds
                gap = ds - 0.5 * (length + float(veh_params[j][5]))
                dv = v - float(veh_v[j])
        a_pts, e_seg, ln, cum = lanes.seg[l]
        for k in np.nonzero(np.asarray(blocker_mask, bool))[0]:
            q, r = q_all[k], r_all[k]
            for m in range(len(ln)):
                d = q - a_pts[m]
                t = (d[0] * e_seg[m, 0] + d[1] * e_seg[m, 1]) / (ln[m] * ln[m])
                t = min(max(t, 0.0), 1.0)
                c = a_pts[m] + t * e_seg[m]
                lat = math.sqrt((q[0] - c[0]) ** 2 + (q[1] - c[1]) ** 2)
                if lat > half_width + r:
                    continue
                ds = cum[m] + t * ln[m] - s
                if ds <= 0.0:
                    ds += L
                if ds <= lookahead and ds < best_ds:
                    best_ds = ds
                    gap = ds - 0.5 * length - r
                    dv = v
        free = 1.0 - (v / v0) ** 4
        if gap is None:
            acc = a * free
        else:
            star = s0 + max(0.0, v * T + v * dv / (2.0 * math.sqrt(a * b)))
            acc = a * (free - (star / max(gap, 0.01)) ** 2)
        vn = max(0.0, v + acc * dt)
        sn = s + vn * dt
        if sn >= L:
            sn -= L
        s_new[i], v_new[i] = sn, vn
        p_now[i] = lanes.point(l, s)
        p_next[i] = lanes.point(l, sn)
        vel[i] = (p_next[i] - p_now[i]) / dt
    return s_new, v_new, p_now, p_next, vel
