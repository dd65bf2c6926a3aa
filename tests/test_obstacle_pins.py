"""Pins of the oracle's static-segment selection (no GPU).

The oracle gives agent i a half-plane for every segment whose squared
distance from p_i is below (r_i + tau_o v_max,i)^2, ordered by (squared
distance, segment id) (the reading of Sec. 3.2's "collision avoidance with
static objects" that the design notes list).  A segment farther than that
cannot bind: its line, v.m <= (d - r)/tau_o with (d - r)/tau_o >= v_max,
leaves the whole speed disk allowed.  So each agent's new velocity must not
change when the lines of ALL of its environment's segments are added; this
is checked here with an LP solved by brute-force vertex enumeration and a
fallback solved by bisection over it, both written from the definitions
only (the closest point to v_pref over the disk and the half-planes; the
least maximal penetration of the agent lines, segment lines kept hard).  A
wrong reach (r + v_max, or a missing radius) drops binding segments and
fails the first test; the hand case fails it on one wall.  The order is
checked against distances found by sampling each segment densely.
"""
import dataclasses
import math

import numpy as np
import pytest

import oracle
from paper_2505_00690_gb300 import scenes
from paper_2505_00690_gb300.scenes import Scene


def lp_vertices(Q, N, vmax, pref, tol=1e-12):
    """argmin |v - pref| over {|v| <= vmax} and {(v - q_k).n_k >= 0}, by
    enumerating every point where the optimum can sit (pref itself, its
    radial projection onto the circle, its projection onto each line, each
    line-circle and line-line intersection) and keeping the closest feasible
    one.  Returns None when no candidate is feasible."""
    pref = np.asarray(pref, float)
    Q = np.asarray(Q, float).reshape(-1, 2)
    N = np.asarray(N, float).reshape(-1, 2)
    c = [pref[None]]
    pl = np.linalg.norm(pref)
    if pl > 0:
        c.append((pref / pl * vmax)[None])
    if len(Q):
        off = ((pref - Q) * N).sum(1)
        c.append(pref - off[:, None] * N)
        D = np.stack([-N[:, 1], N[:, 0]], 1)
        qd = (Q * D).sum(1)
        disc = qd * qd - (Q * Q).sum(1) + vmax * vmax
        ok = disc >= 0
        sq = np.sqrt(np.where(ok, disc, 0.0))
        for sgn in (-1.0, 1.0):
            c.append((Q + ((-qd + sgn * sq)[:, None]) * D)[ok])
        a, b = np.triu_indices(len(Q), 1)
        det = N[a, 0] * N[b, 1] - N[a, 1] * N[b, 0]
        keep = np.abs(det) >= 1e-12
        a, b, det = a[keep], b[keep], det[keep]
        ra, rb = (Q[a] * N[a]).sum(1), (Q[b] * N[b]).sum(1)
        x = (ra * N[b, 1] - rb * N[a, 1]) / det
        y = (N[a, 0] * rb - N[b, 0] * ra) / det
        c.append(np.stack([x, y], 1))
    C = np.concatenate(c)
    feas = (C * C).sum(1) <= vmax * vmax * (1 + tol) + tol
    if len(Q):
        feas &= (((C[:, None, :] - Q[None]) * N[None]).sum(2) >= -tol).all(1)
    if not feas.any():
        return None
    C = C[feas]
    return C[np.argmin(((C - pref) ** 2).sum(1))]


def fallback_bisection(Q, N, n_hard, vmax, pref):
    """Least maximal penetration of the soft (agent) lines over the disk and
    the hard (segment) lines, by bisection on the penetration d with
    lp_vertices as the feasibility test; the hard lines become soft when
    they leave nothing.  Returns (velocity, d)."""
    Q = np.asarray(Q, float).reshape(-1, 2)
    N = np.asarray(N, float).reshape(-1, 2)
    if lp_vertices(Q[:n_hard], N[:n_hard], vmax, pref) is None:
        n_hard = 0
    shift = lambda d: np.concatenate([Q[:n_hard], Q[n_hard:] - d * N[n_hard:]])
    lo, hi = 0.0, 4 * vmax + 10
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if lp_vertices(shift(mid), N, vmax, pref, tol=1e-13) is None:
            lo = mid
        else:
            hi = mid
        if hi - lo < 1e-13:
            break
    return lp_vertices(shift(hi), N, vmax, pref, tol=1e-12), hi


def _check_all_segments(sc, steps, every, max_agents=None, seed=0):
    o = oracle.OracleScene(sc)
    prm = o.params  # the FP32-rounded parameters the oracle steps with
    tau_o, tau, dt, R, K = prm.tau_obst, prm.tau, prm.dt, prm.neighbor_dist, sc.max_neighbors
    pos, vel = sc.pos.astype(np.float64), sc.vel.astype(np.float64)
    rng = np.random.default_rng(seed)
    checked = changed = fallbacks = 0
    for k in range(steps):
        rv = sc.robot_vel_at(k).astype(np.float64) if sc.robot_vel is not None else None
        npos, nvel, _, st = o.step(pos, vel, rv)
        if k % every == 0:
            for e in range(sc.n_envs):
                base, n = sc.env_start[e], sc.env_start[e + 1] - sc.env_start[e]
                segs = sc.segments[sc.seg_start[e]:sc.seg_start[e + 1]].astype(np.float64)
                if not len(segs):
                    continue
                robot = sc.robot_index[e]
                V = vel[base:base + n].copy()
                if robot >= 0:
                    V[robot] = rv[e]
                agents = [i for i in range(n) if i != robot]
                if max_agents and len(agents) > max_agents:
                    agents = sorted(rng.choice(agents, max_agents, replace=False))
                for i in agents:
                    g = base + i
                    vmax, r = float(sc.max_speed[g]), float(sc.radius[g])
                    pref = oracle.pref_velocity(pos[g], sc.goal[g].astype(np.float64), float(sc.pref_speed[g]), dt)
                    lines = [oracle.obstacle_line(pos[g], V[i], r, vmax, s, tau_o, dt) for s in segs]
                    n_hard = len(lines)
                    ids, _ = oracle.neighbors(pos[base:base + n], i, R, K)
                    for j in ids:
                        alpha = prm.robot_alpha if j == robot else 0.5
                        lines.append(oracle.agent_line(pos[g], V[i], r, pos[base + j], V[j],
                                                       float(sc.radius[base + j]), tau, dt, alpha, i, j))
                    Q = np.array([q for q, _ in lines])
                    N = np.array([nn for _, nn in lines])
                    if st[g] == 0:
                        v = lp_vertices(Q, N, vmax, pref)
                        assert v is not None, (k, g)
                        assert np.linalg.norm(v - nvel[g]) < 1e-12, (k, g, v, nvel[g])
                    else:
                        fallbacks += 1
                        v, _ = fallback_bisection(Q, N, n_hard, vmax, pref)
                        assert np.linalg.norm(v - nvel[g]) < 1e-6, (k, g, v, nvel[g])
                    # the velocity differs from the unconstrained one: a line binds
                    changed += int(np.linalg.norm(nvel[g] - pref) > 1e-9)
                    checked += 1
        pos, vel = npos, nvel
    return checked, changed, fallbacks


def test_all_segment_lp_equals_oracle_step_urban_block():
    """Urban blocks (36 segments each): every agent's oracle velocity equals
    the LP over the lines of all 36 segments plus its agent lines."""
    sc = scenes.urban_block(3, n_envs=2, n_peds=48, steps=60)
    checked, changed, _ = _check_all_segments(sc, 60, 6)
    assert checked >= 900 and changed > 100


def test_all_segment_lp_equals_oracle_step_polygons():
    """Uneven polygon environments (convex polygons, many short edges near
    each other): the same check on a sample of agents per step."""
    sc = scenes.uneven_batch(5, n_envs=2, n_lo=40, n_hi=80, max_polys=12, steps=30)
    checked, changed, _ = _check_all_segments(sc, 30, 5, max_agents=25)
    assert checked >= 200 and changed > 20


def _wall_scene(d, r=0.3, vmax=1.4, tau=2.0):
    """One agent at the origin walking along +x at v_max toward a 4 m wall
    across its path at x = d (segment id 1), and a second wall far behind
    it (id 0)."""
    segs = np.array([[-40.0, -2.0, -40.0, 2.0], [d, -2.0, d, 2.0]], np.float32)
    return Scene(name="wall", agents_per_env=np.array([1], np.int32), radius=np.array([r], np.float32),
                 max_speed=np.array([vmax], np.float32), pref_speed=np.array([vmax], np.float32),
                 pos=np.zeros((1, 2), np.float32), vel=np.array([[vmax, 0.0]], np.float32),
                 goal=np.array([[50.0, 0.0]], np.float32), robot_index=np.array([-1], np.int32),
                 segs_per_env=np.array([2], np.int32), segments=segs, tau=tau, tau_obst=tau,
                 neighbor_dist=5.0, max_neighbors=10, dt=0.1)


@pytest.mark.parametrize("d", [2.0, 3.0, 3.05, 3.09, 3.2, 6.0])
def test_wall_just_inside_reach_binds(d):
    """Hand-derived: the wall's line is v_x <= (d - r)/tau_o, which binds iff
    d < r + tau_o v_max = 3.1 m; the agent then walks at exactly (d - r)/tau_o,
    else at v_max.  The walls at 3.05 and 3.09 m lie just inside the reach and
    change the answer; a reach of r + v_max (1.7 m) would miss them."""
    sc = _wall_scene(d)
    o = oracle.OracleScene(sc)
    r, vmax, tau = float(np.float32(0.3)), float(np.float32(1.4)), 2.0
    dd = float(np.float32(d))
    _, v, _, st = o.step(sc.pos.astype(np.float64), sc.vel.astype(np.float64))
    expect = min(vmax, (dd - r) / tau)
    assert st[0] == 0
    assert abs(v[0, 0] - expect) < 1e-12 and abs(v[0, 1]) < 1e-12
    ids = oracle.obstacles(sc.segments.astype(np.float64), np.zeros(2), r + tau * vmax)
    assert list(ids) == ([1] if dd < r + tau * vmax else [])


def _sampled_dist2(p, s, m=20001):
    t = np.linspace(0.0, 1.0, m)[:, None]
    pts = s[:2] + t * (s[2:] - s[:2])
    return float(((pts - p) ** 2).sum(1).min())


@pytest.mark.parametrize("seed", range(6))
def test_segment_order_by_sampled_distance(seed):
    """The oracle's segment list for a point: exactly the segments whose
    distance (found by sampling 20,001 points along each) is inside the reach,
    in increasing distance (up to the sampling resolution)."""
    rng = np.random.default_rng(77 + seed)
    segs = rng.uniform(-6, 6, (40, 4))
    p = rng.uniform(-3, 3, 2)
    reach = 3.0
    ids = list(oracle.obstacles(segs, p, reach))
    d2 = np.array([_sampled_dist2(p, s) for s in segs])
    res = np.array([(np.linalg.norm(s[2:] - s[:2]) / 20000.0) for s in segs])
    margin = (2 * np.sqrt(d2) + res) * res + 1e-12  # sampled d^2 overestimates by at most this
    inside = [k for k in range(len(segs)) if d2[k] - margin[k] < reach * reach]
    surely = [k for k in range(len(segs)) if d2[k] < reach * reach]
    assert set(surely) <= set(ids) <= set(inside)
    for a, b in zip(ids, ids[1:]):
        assert d2[a] - margin[a] <= d2[b] + 1e-12


def test_segment_ties_ordered_by_id():
    """Two walls at the same distance on either side: the lower id comes
    first, whichever side it is on."""
    left, right = [-1.0, -1.0, -1.0, 1.0], [1.0, -1.0, 1.0, 1.0]
    for segs, expect in (([left, right], [0, 1]), ([right, left], [0, 1])):
        ids = oracle.obstacles(np.array(segs, float), np.zeros(2), 2.0)
        assert list(ids) == expect
