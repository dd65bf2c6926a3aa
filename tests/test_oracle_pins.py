"""Pins of the FP64 oracle against what the definitions fix (no GPU).

Every check here comes from something other than the oracle itself: closed
forms derived by hand from the ORCA geometry, brute-force geometry built only
from the velocity-obstacle definition (a relative velocity v is in VO^tau when
t*v lands in D(p, r) for some t in [0, tau]), brute-force vertex enumeration
of the LP, and invariants ORCA guarantees (Sec. 3.2 of the paper with the
method it cites for the collision-avoidance rule).
"""
import dataclasses
import math

import numpy as np
import pytest

import oracle
from paper_2505_00690_gb300.scenes import Scene, plain_square, urban_block


def f32(x):
    return float(np.float32(x))


def one_env(pos, vel, goal, radius, vmax, segs=(), robot=-1, R=5.0, K=10, tau=2.0, dt=0.1, pref=None):
    n = len(pos)
    pref = vmax if pref is None else pref
    return Scene(name="t", agents_per_env=np.array([n], np.int32),
                 radius=np.full(n, radius, np.float32) if np.isscalar(radius) else np.asarray(radius, np.float32),
                 max_speed=np.full(n, vmax, np.float32) if np.isscalar(vmax) else np.asarray(vmax, np.float32),
                 pref_speed=np.full(n, pref, np.float32) if np.isscalar(pref) else np.asarray(pref, np.float32),
                 pos=np.asarray(pos, np.float32).reshape(-1, 2), vel=np.asarray(vel, np.float32).reshape(-1, 2),
                 goal=np.asarray(goal, np.float32).reshape(-1, 2), robot_index=np.array([robot], np.int32),
                 segs_per_env=np.array([len(segs)], np.int32),
                 segments=np.asarray(segs, np.float32).reshape(-1, 4), tau=tau, tau_obst=tau,
                 neighbor_dist=R, max_neighbors=K, dt=dt)


# ----------------------------------------------------------------------------- O1

def test_pref_velocity_arrive_rule():
    # far: speed along the unit direction; near: exactly onto the goal in one step; on it: zero
    v = oracle.pref_velocity((1.0, 2.0), (4.0, 6.0), 1.5, 0.1)
    assert np.allclose(v, [1.5 * 0.6, 1.5 * 0.8], atol=1e-15)
    v = oracle.pref_velocity((1.0, 2.0), (1.03, 2.04), 1.5, 0.1)
    assert np.allclose(v, [0.3, 0.4], atol=1e-12)
    assert np.all(oracle.pref_velocity((1.0, 2.0), (1.0, 2.0), 1.5, 0.1) == 0.0)
    # exactly s*dt away counts as "near"
    v = oracle.pref_velocity((0.0, 0.0), (0.15, 0.0), 1.5, 0.1)
    assert np.allclose(v, [1.5, 0.0], atol=1e-14)


def test_lone_agent_closed_form():
    """A lone agent walks at its preferred speed on the straight line to its goal
    and stops exactly on it (p_k = p_0 + k dt s g_hat until arrival)."""
    p0 = np.array([1.0, 2.0])
    g = np.array([f32(7.0), f32(10.0)])  # 6-8-10 triangle: distance 10
    s, dt = f32(1.25), f32(0.1)
    sc = one_env([p0], [[0, 0]], [g], 0.3, s)
    o = oracle.OracleScene(sc)
    pos, vel = p0[None].copy(), np.zeros((1, 2))
    ghat = (g - p0) / np.linalg.norm(g - p0)
    arrive = None
    for k in range(1, 120):
        pos, vel, nb, st = o.step(pos, vel)
        assert nb[0, 0] == -1 and st[0] == 0
        if arrive is None:
            expect = p0 + k * dt * s * ghat
            if np.linalg.norm(g - (p0 + (k - 1) * dt * s * ghat)) <= s * dt:
                arrive = k
                expect = g
                assert np.allclose(pos[0], g, atol=1e-12)
            else:
                assert np.allclose(vel[0], s * ghat, atol=1e-12), k
                assert np.allclose(pos[0], expect, atol=1e-12), k
        else:
            assert np.all(vel[0] == 0.0) or np.linalg.norm(vel[0]) < 1e-9
            assert np.allclose(pos[0], g, atol=1e-12)
    assert arrive == 80  # 10 m at 0.125 m per step: the 80th step starts exactly s*dt away and lands


# ----------------------------------------------------------------------------- goal queues

def _walk_queue(queue, cyclic, steps, r=0.35, s=1.0, dt=0.1):
    """A lone agent from (0, 0) through a goal queue; returns the goal index at
    the start of every step and the final position."""
    q = np.asarray(queue, np.float32)[None]
    sc = one_env([(0.0, 0.0)], [(0.0, 0.0)], [q[0, 0]], r, s, dt=dt)
    o = oracle.OracleScene(sc)
    pos, vel = np.zeros((1, 2)), np.zeros((1, 2))
    goal, idx = q[:, 0].astype(np.float64), np.zeros(1, np.int64)
    seen = []
    for _ in range(steps):
        goal, idx = oracle.advance_goals(pos, sc.radius, goal, idx, q, cyclic)
        seen.append(int(idx[0]))
        pos, vel, _, _ = o.step(pos, vel, goal=goal)
    return np.array(seen), pos[0]


def test_goal_queue_lone_agent_turns_within_reach():
    """Speed 1 m/s, dt 0.1 s, r 0.35 m, goals (10, 0) -> (10, 10) -> (0, 10).
    Hand-derived: the start of step k finds the agent 0.1 k m along the first
    leg, so it is within 0.35 m of (10, 0) first at k = 97 (x = 9.7); the
    second leg from (9.7, 0) is sqrt(0.3^2 + 10^2) = 10.0045 m long, so the
    agent is within reach of (10, 10) after ceil((10.0045 - 0.35) / 0.1) = 97
    more steps, at k = 194.  The queue is not cyclic: (0, 10) stays the goal,
    the agent lands on it by the arrive rule and stops."""
    seen, final = _walk_queue([(10.0, 0.0), (10.0, 10.0), (0.0, 10.0)], cyclic=False, steps=400)
    assert np.nonzero(seen == 1)[0][0] == 97
    assert np.nonzero(seen == 2)[0][0] == 194
    assert seen[-1] == 2 and seen.max() == 2
    assert np.allclose(final, [0.0, 10.0], atol=1e-12)


def test_goal_queue_cyclic_shuttle():
    """Goals (1, 0) and (0, 0), cyclic: out to x = 0.7 (within 0.35 of 1, step
    7), back to x = 0.3 (step 11), out again to 0.7 (step 15): the index grows
    every 4 steps after the first 7."""
    seen, _ = _walk_queue([(1.0, 0.0), (0.0, 0.0)], cyclic=True, steps=40)
    steps_at = [int(np.nonzero(seen == k)[0][0]) for k in range(1, 9)]
    assert steps_at == [7, 11, 15, 19, 23, 27, 31, 35]


def test_goal_queue_reach_boundary_and_robot():
    """|g - p|^2 == r^2 exactly moves on (<=); one ulp beyond does not; the
    robot row never moves on."""
    q = np.array([[[0.375, 0.0], [5.0, 5.0]], [[np.nextafter(np.float32(0.375), np.float32(1)), 0.0], [5.0, 5.0]],
                  [[0.0, 0.0], [5.0, 5.0]]], np.float32)
    pos = np.zeros((3, 2))
    g, k = oracle.advance_goals(pos, np.full(3, 0.375, np.float32), q[:, 0], np.zeros(3), q, cyclic=True,
                                skip=[False, False, True])
    assert list(k) == [1, 0, 0]
    assert np.array_equal(g[0], [5.0, 5.0]) and np.array_equal(g[1], q[1, 0]) and np.array_equal(g[2], [0.0, 0.0])


# ----------------------------------------------------------------------------- O3 closed form

@pytest.mark.parametrize("half_gap,steps", [((4.0, 0.0), 400), ((0.0, -4.0), 400), ((3.0, 4.0), 20),
                                            ((-2.5, 6.0), 30)])
def test_head_on_pair_closed_form(half_gap, steps):
    """Symmetric head-on pair, neighbour distance 15 m > 2 s tau + gap: every
    interaction is in the cut-off case, the lateral velocity stays 0, and with
    d the centre distance v_k = min(s, (d_k - (r_i + r_j)) / (2 tau)),
    d_{k+1} = d_k - 2 dt v_k (the reciprocal half of the cut-off disk's
    u = (r/tau - |w|) w_hat, w = v - p/tau).  On a coordinate axis the
    arithmetic is exactly symmetric; on an oblique axis rounding seeds a
    lateral offset that the head-on configuration amplifies once the line
    binds (it is an unstable equilibrium), so there only the approach is
    compared.  Axes with exact float32 coordinates keep the pair collinear
    with its goals."""
    h = np.array(half_gap)
    e = h / np.linalg.norm(h)
    r, s, tau, dt = f32(0.3), f32(1.4), 2.0, f32(0.1)
    pos = np.stack([-h, h])
    vel = np.stack([s * e, -s * e])
    goal = np.stack([100.0 * h, -100.0 * h])
    sc = one_env(pos, vel, goal, r, s, R=15.0, tau=tau, dt=dt)
    o = oracle.OracleScene(sc)
    P = sc.pos.astype(np.float64)
    V = sc.vel.astype(np.float64)
    d = float(np.linalg.norm(P[1] - P[0]))
    for k in range(steps):
        P, V, nb, st = o.step(P, V)
        assert st[0] == 0 and st[1] == 0
        v = min(s, (d - 2 * r) / (2 * tau))
        d = d - 2 * dt * v
        along = V[0] @ e
        lateral = V[0] @ np.array([-e[1], e[0]])
        assert abs(along - v) < 1e-12, k
        assert abs(lateral) < (1e-12 if steps >= 400 else 1e-9), k
        assert np.allclose(V[1], -V[0], atol=1e-12)
        assert abs(np.linalg.norm(P[1] - P[0]) - d) < 1e-11
    assert d > 2 * r  # never touches
    if steps >= 400:
        assert d - 2 * r < 1e-6  # converged onto contact
    else:
        assert (d - 2 * r) / (2 * tau) < s  # the line binds within the compared steps


@pytest.mark.parametrize("alpha", [1.0, 0.5])
def test_robot_pair_closed_form(alpha):
    """A pedestrian walking at the robot, which moves at its command
    (-1.4, 0) and does not react.  With the pedestrian's share alpha of the
    cut-off disk's u = (r/tau - |w|) w_hat, w = v - p/tau, the line bounds its
    velocity along the axis by v_k - alpha (v_k + 1.4 - (d_k - r)/tau); with
    alpha = 1 (the robot non-reactive, the pedestrian taking all of the
    avoidance) that is (d_k - r)/tau - 1.4, independent of v_k, and the gap
    d - r then shrinks by (1 - dt/tau) every step.  The lateral velocity stays
    0; d_{k+1} = d_k - dt (v_{k+1} + 1.4)."""
    r, s, tau, dt, vr = f32(0.3), f32(1.4), 2.0, f32(0.1), f32(1.4)
    pos = np.array([[0.0, 0.0], [8.0, 0.0]])
    vel = np.array([[s, 0.0], [-vr, 0.0]])
    goal = np.array([[100.0, 0.0], [-100.0, 0.0]])
    sc = dataclasses.replace(one_env(pos, vel, goal, r, s, robot=1, R=15.0, tau=tau, dt=dt),
                             robot_responsibility=alpha)
    o = oracle.OracleScene(sc)
    P, V = sc.pos.astype(np.float64), sc.vel.astype(np.float64)
    rv = np.array([[-vr, 0.0]], np.float32)
    d, v = 8.0, float(s)
    gaps = []
    for k in range(300):
        P, V, nb, st = o.step(P, V, rv)
        v = min(s, v - alpha * (v + vr - (d - 2 * r) / tau))
        d = d - dt * (v + vr)
        assert abs(V[0, 0] - v) < 1e-12 and abs(V[0, 1]) < 1e-12, k
        assert abs(P[1, 0] - P[0, 0] - d) < 1e-10 and np.array_equal(V[1], [-vr, 0.0])
        gaps.append(d - 2 * r)
    assert min(gaps) > 0  # never touches
    if alpha == 1.0:
        g = np.array(gaps)
        k0 = int(np.argmax(g < (s + vr) * tau))  # the line binds from here on
        assert np.allclose(g[k0 + 1:] / g[k0:-1], 1 - dt / tau, rtol=1e-9)


# ----------------------------------------------------------------------------- O3 brute force

def _in_vo(v, p, r, tau):
    """Definition: v is in the truncated VO iff t*v enters D(p, r) for some t in [0, tau]."""
    vv = v @ v
    t = 0.0 if vv == 0 else min(max((p @ v) / vv, 0.0), tau)
    return np.linalg.norm(t * v - p) < r


def _in_vo_many(P, p, r, tau):
    vv = (P * P).sum(-1)
    t = np.where(vv > 0, np.clip((P @ p) / np.where(vv > 0, vv, 1.0), 0.0, tau), 0.0)
    return np.linalg.norm(t[..., None] * P - p, axis=-1) < r


def _nearest_boundary(v, p, r, tau, ndir=512, reach=12.0, step=2e-3):
    """Brute force: shortest ray from v to a change of VO membership (a fine
    linear scan along each ray, so that thin parts of the VO are not stepped
    over, then bisection; the best direction is refined by golden section)."""
    inside = _in_vo(v, p, r, tau)
    s = np.arange(step, reach, step)

    def cross(thetas):
        d = np.stack([np.cos(thetas), np.sin(thetas)], -1)
        P = v[None, None, :] + s[None, :, None] * d[:, None, :]
        change = _in_vo_many(P, p, r, tau) != inside
        first = np.where(change.any(1), change.argmax(1), -1)
        out = np.full(len(thetas), np.inf)
        for k in np.nonzero(first >= 0)[0]:
            lo = 0.0 if first[k] == 0 else s[first[k] - 1]
            hi = s[first[k]]
            for _ in range(60):
                mid = 0.5 * (lo + hi)
                if _in_vo(v + mid * d[k], p, r, tau) == inside:
                    lo = mid
                else:
                    hi = mid
            out[k] = hi
        return out

    thetas = np.linspace(0, 2 * math.pi, ndir, endpoint=False)
    dists = cross(thetas)
    k = int(np.argmin(dists))
    a, b = thetas[k] - 2 * math.pi / ndir, thetas[k] + 2 * math.pi / ndir
    g = (math.sqrt(5) - 1) / 2
    c, d = b - g * (b - a), a + g * (b - a)
    fc, fd = cross(np.array([c]))[0], cross(np.array([d]))[0]
    for _ in range(50):
        if fc < fd:
            b, d, fd = d, c, fc
            c = b - g * (b - a)
            fc = cross(np.array([c]))[0]
        else:
            a, c, fc = c, d, fd
            d = a + g * (b - a)
            fd = cross(np.array([d]))[0]
    th = 0.5 * (a + b)
    dist = cross(np.array([th]))[0]
    u = dist * np.array([math.cos(th), math.sin(th)])
    return u, inside


@pytest.mark.parametrize("seed", range(12))
def test_agent_line_matches_vo_geometry(seed):
    """u and n of the agent half-plane equal the nearest point of the boundary
    of the truncated VO (found by brute force from the definition) and the
    outward normal there; the line passes through v_i + u/2."""
    rng = np.random.default_rng(seed)
    while True:
        pi = rng.uniform(-3, 3, 2)
        pj = pi + rng.uniform(-4, 4, 2)
        ri, rj = rng.uniform(0.2, 0.5, 2)
        vi, vj = rng.uniform(-1.5, 1.5, 2), rng.uniform(-1.5, 1.5, 2)
        tau = 2.0
        p = pj - pi
        if np.linalg.norm(p) > ri + rj + 0.05:
            break
    q, n = oracle.agent_line(pi, vi, ri, pj, vj, rj, tau, 0.1)
    v = vi - vj
    u_bf, inside = _nearest_boundary(v, p, ri + rj, tau)
    # the oracle's u, recovered from its line: q = v_i + u/2
    u = 2.0 * (q - vi)
    assert np.linalg.norm(u - u_bf) < 1e-6, (u, u_bf)
    n_bf = u_bf / np.linalg.norm(u_bf) * (1.0 if inside else -1.0)
    assert np.allclose(n, n_bf, atol=1e-4)
    assert abs(np.linalg.norm(n) - 1.0) < 1e-12


def _seg_dist_many(X, A, B):
    """Distance from points X [..., 2] to segment [A, B]."""
    e = B - A
    t = np.clip(((X - A) @ e) / (e @ e), 0.0, 1.0)
    return np.linalg.norm(X - (A + t[..., None] * e), axis=-1)


def _in_cvo_many(P, A, B, r, tau):
    """Definition for a segment: v is in the truncated VO of the capsule
    [A, B] + D(r) iff t*v comes within r of [A, B] for some t in [0, tau],
    i.e. iff the segments [0, tau v] and [A, B] are closer than r."""
    T = tau * P
    d = np.minimum(_seg_dist_many(T, A, B), _seg_dist_many(np.zeros_like(T), A, B))
    zero = np.zeros(2)
    for X in (A, B):
        e = T
        ee = np.where((e * e).sum(-1) > 0, (e * e).sum(-1), 1.0)
        t = np.clip((e @ X) / ee, 0.0, 1.0)
        d = np.minimum(d, np.linalg.norm(X - t[..., None] * e, axis=-1))
    # proper crossing of the two segments: distance 0
    cr = lambda o, a, b: (a[..., 0] - o[..., 0]) * (b[..., 1] - o[..., 1]) - (a[..., 1] - o[..., 1]) * (b[..., 0] - o[..., 0])
    Z = np.broadcast_to(zero, T.shape)
    Ab, Bb = np.broadcast_to(A, T.shape), np.broadcast_to(B, T.shape)
    crossing = (np.sign(cr(Z, T, Ab)) * np.sign(cr(Z, T, Bb)) < 0) & (np.sign(cr(Ab, Bb, Z)) * np.sign(cr(Ab, Bb, T)) < 0)
    return (d < r) | crossing


def _nearest_cvo_boundary(v, A, B, r, tau, ndir=512, reach=12.0, step=2e-3):
    """_nearest_boundary for the segment's VO (same search)."""
    inside = bool(_in_cvo_many(v[None], A, B, r, tau)[0])
    s = np.arange(step, reach, step)

    def cross(thetas):
        d = np.stack([np.cos(thetas), np.sin(thetas)], -1)
        P = v[None, None, :] + s[None, :, None] * d[:, None, :]
        change = _in_cvo_many(P, A, B, r, tau) != inside
        first = np.where(change.any(1), change.argmax(1), -1)
        out = np.full(len(thetas), np.inf)
        for k in np.nonzero(first >= 0)[0]:
            lo = 0.0 if first[k] == 0 else s[first[k] - 1]
            hi = s[first[k]]
            for _ in range(60):
                mid = 0.5 * (lo + hi)
                if bool(_in_cvo_many((v + mid * d[k])[None], A, B, r, tau)[0]) == inside:
                    lo = mid
                else:
                    hi = mid
            out[k] = hi
        return out

    thetas = np.linspace(0, 2 * math.pi, ndir, endpoint=False)
    dists = cross(thetas)
    k = int(np.argmin(dists))
    a, b = thetas[k] - 2 * math.pi / ndir, thetas[k] + 2 * math.pi / ndir
    g = (math.sqrt(5) - 1) / 2
    c, d = b - g * (b - a), a + g * (b - a)
    fc, fd = cross(np.array([c]))[0], cross(np.array([d]))[0]
    for _ in range(50):
        if fc < fd:
            b, d, fd = d, c, fc
            c = b - g * (b - a)
            fc = cross(np.array([c]))[0]
        else:
            a, c, fc = c, d, fd
            d = a + g * (b - a)
            fd = cross(np.array([d]))[0]
    th = 0.5 * (a + b)
    dist = cross(np.array([th]))[0]
    return dist * np.array([math.cos(th), math.sin(th)]), inside


def test_velocity_segment_line_long_wall_closed_form():
    """O4v against a long wall 5 m ahead (r 0.3, tau_o 2): the face of the VO
    is the line v_y = (5 - 0.3) / 2 = 2.35, so walking at it or along it the
    nearest boundary point is v's projection on that line and the normal -y
    (the velocity-independent O4 line is the same there)."""
    for v in ((0.0, 1.2), (1.2, 0.0), (-0.7, 0.4)):
        q, n = oracle.obstacle_line_vd((0.0, 0.0), v, 0.3, 1.4, (-50.0, 5.0, 50.0, 5.0), 2.0, 0.1)
        assert np.allclose(q, [v[0], 2.35], atol=1e-12) and np.allclose(n, [0.0, -1.0], atol=1e-12)


def test_velocity_segment_line_leg_hand_case():
    """Segment (-0.5, 3)-(0.5, 3), r 0.3, tau_o 2, v = (0.2, 2.0), inside the
    VO: by hand, the right leg (tangent to the disk at (0.5, 3): direction
    angle atan2(3, 0.5) - asin(0.3 / |(0.5, 3)|) = 1.3070 rad) is 0.328 m/s
    away, the left one 0.714 and the face behind v does not face 0, so X is
    v's projection on the right leg, (0.517, 1.914), with normal
    (0.9654, -0.2607)."""
    q, n = oracle.obstacle_line_vd((0.0, 0.0), (0.2, 2.0), 0.3, 1.4, (-0.5, 3.0, 0.5, 3.0), 2.0, 0.1)
    assert np.allclose(q, [0.517, 1.914], atol=2e-3) and np.allclose(n, [0.9654, -0.2607], atol=2e-4)


@pytest.mark.parametrize("seed", range(16))
def test_velocity_segment_line_matches_vo_geometry(seed):
    """X and n of O4v equal the nearest point of the segment VO's boundary
    (brute force from the definition) and the outward normal there."""
    rng = np.random.default_rng(500 + seed)
    while True:
        p = rng.uniform(-2, 2, 2)
        a = p + rng.uniform(-4, 4, 2)
        b = a + rng.uniform(-3, 3, 2)
        r = rng.uniform(0.2, 0.45)
        seg = np.concatenate([a, b])
        e = b - a
        t = np.clip(((p - a) @ e) / (e @ e), 0, 1)
        if np.linalg.norm(a + t * e - p) > r + 0.1:
            break
    v = rng.uniform(-1.5, 1.5, 2)
    tau = 2.0
    q, n = oracle.obstacle_line_vd(p, v, r, 1.6, seg, tau, 0.1)
    u_bf, inside = _nearest_cvo_boundary(v, a - p, b - p, r, tau)
    assert np.linalg.norm(q - (v + u_bf)) < 1e-5, (q, v + u_bf)
    n_bf = u_bf / np.linalg.norm(u_bf) * (1.0 if inside else -1.0)
    assert np.allclose(n, n_bf, atol=1e-3), (n, n_bf)


def test_velocity_segment_covered_at_polygon_vertex():
    """A square's corner nearest the agent: the first edge's line (tangent at
    the corner's cap, normal in the corner's normal cone) forbids both end
    disks of the other edge's cutoff capsule, which then gets no line; an edge
    facing away is not covered by a leg it does not lie behind."""
    p, r, tau = np.array([0.0, 0.0]), 0.3, 2.0
    e1 = (2.0, 2.0, 4.0, 2.0)   # bottom edge of the square [2,4] x [2,4]
    e2 = (2.0, 2.0, 2.0, 4.0)   # left edge, sharing the corner (2, 2)
    line1 = oracle.obstacle_line_vd(p, (0.0, 0.0), r, 1.5, e1, tau, 0.1)
    assert np.allclose(line1[1], -np.array([1.0, 1.0]) / np.sqrt(2), atol=1e-12)  # the corner cap, towards 0
    assert oracle.segment_covered(p, r, e2, tau, [line1])
    far = (-6.0, -1.0, -6.0, 1.0)  # a segment on the other side
    assert not oracle.segment_covered(p, r, far, tau, [line1])


def test_velocity_segment_line_overlap_is_o4():
    for v in ((0.3, -0.2), (0.0, 0.0)):
        q1, n1 = oracle.obstacle_line_vd((0.0, 0.1), v, 0.3, 1.4, (-1.0, 0.0, 1.0, 0.0), 2.0, 0.1)
        q0, n0 = oracle.obstacle_line((0.0, 0.1), v, 0.3, 1.4, (-1.0, 0.0, 1.0, 0.0), 2.0, 0.1)
        assert np.array_equal(q1, q0) and np.array_equal(n1, n0)


@pytest.mark.parametrize("seed", range(20))
def test_agent_line_reciprocity(seed):
    """The pair's two half-planes are mirror images: u_ji = -u_ij, n_ji = -n_ij."""
    rng = np.random.default_rng(100 + seed)
    pi, pj = rng.uniform(-3, 3, 2), rng.uniform(-3, 3, 2)
    vi, vj = rng.uniform(-1.5, 1.5, 2), rng.uniform(-1.5, 1.5, 2)
    ri, rj = rng.uniform(0.2, 0.5, 2)
    qi, ni = oracle.agent_line(pi, vi, ri, pj, vj, rj, 2.0, 0.1, 0.5, 0, 1)
    qj, nj = oracle.agent_line(pj, vj, rj, pi, vi, ri, 2.0, 0.1, 0.5, 1, 0)
    assert np.allclose(ni, -nj, atol=1e-12)
    assert np.allclose(2 * (qi - vi), -2 * (qj - vj), atol=1e-12)


def test_agent_line_colliding_closed_form():
    """Overlapping agents: horizon dt, u = (r/dt - |w|) w_hat with w = v - p/dt."""
    q, n = oracle.agent_line((0, 0), (0, 0), 0.3, (0.3, 0), (0, 0), 0.3, 2.0, 0.1)
    # w = -p/dt = (-3, 0); u = (6 - 3) * (-1, 0); q = u/2
    assert np.allclose(n, [-1, 0], atol=1e-15)
    assert np.allclose(q, [-1.5, 0], atol=1e-12)
    # w = 0 -> n = -p_hat
    q, n = oracle.agent_line((0, 0), (2.0, 0), 0.25, (0.25, 0), (0, 0), 0.25, 2.0, 0.125)
    # w = (2, 0) - (0.25, 0)/0.125 = 0 exactly; u = (0.5/0.125) * (-1, 0); q = v_i + u/2
    assert np.allclose(n, [-1, 0], atol=0) and np.allclose(q, [2.0 - 2.0, 0], atol=1e-15)
    # p = 0 -> +-x by id order, mirrored
    q0, n0 = oracle.agent_line((1, 1), (0, 0), 0.3, (1, 1), (0, 0), 0.3, 2.0, 0.1, 0.5, 0, 1)
    q1, n1 = oracle.agent_line((1, 1), (0, 0), 0.3, (1, 1), (0, 0), 0.3, 2.0, 0.1, 0.5, 1, 0)
    assert np.allclose(n0, [1, 0]) and np.allclose(n1, [-1, 0])
    assert np.allclose(q0, [3.0, 0]) and np.allclose(q1, [-3.0, 0])


def test_agent_line_leg_tie_takes_right_leg():
    # w parallel to p in the leg region: det = 0, the right leg (clockwise) is used
    q, n = oracle.agent_line((0, 0), (3.0, 0), 0.5, (4.0, 0), (0, 0), 0.5, 2.0, 0.1)
    # p = (4,0), r = 1: right leg direction (sqrt(15), -1)/4, outward normal (-1, -sqrt(15))/4
    assert np.allclose(n, [-1 / 4, -math.sqrt(15) / 4], atol=1e-12)


# ----------------------------------------------------------------------------- O4

def test_obstacle_line_closed_form():
    seg = (-1.0, 2.0, 1.0, 2.0)
    q, n = oracle.obstacle_line((0, 0), (0, 0), 0.5, 1.4, seg, 2.0, 0.1)
    # closest point (0, 2), d = 2, m = (0, 1): allowed v_y <= (2 - 0.5)/2
    assert np.allclose(n, [0, -1]) and np.allclose(q, [0, 0.75])
    # endpoint region: closest point is the endpoint a
    q, n = oracle.obstacle_line((-4, 2), (0, 0), 0.5, 1.4, seg, 2.0, 0.1)
    assert np.allclose(n, [-1, 0]) and np.allclose(q, [1.25, 0])
    # overlapping: (d - r)/dt, capped at -vmax
    q, n = oracle.obstacle_line((0, 1.9), (0, 0), 0.5, 1.4, seg, 2.0, 0.1)
    assert np.allclose(n, [0, -1]) and np.allclose(q, [0, -1.4])
    q, n = oracle.obstacle_line((0, 1.52), (0, 0), 0.5, 1.4, seg, 2.0, 0.1)
    assert np.allclose(q, [0, (0.48 - 0.5) / 0.1], atol=1e-12)
    # on the segment: the normal faces away from the side the velocity came from
    q, n = oracle.obstacle_line((0, 2), (0, 1.0), 0.5, 1.4, seg, 2.0, 0.1)
    assert np.allclose(n, [0, -1])  # moving up: pushed back down
    q, n = oracle.obstacle_line((0, 2), (0, -1.0), 0.5, 1.4, seg, 2.0, 0.1)
    assert np.allclose(n, [0, 1])
    q, n = oracle.obstacle_line((0, 2), (1.0, 0), 0.5, 1.4, seg, 2.0, 0.1)
    assert np.allclose(n, [0, -1])  # undecided: m = left normal of a->b = (0, 1)


@pytest.mark.parametrize("seed", range(10))
def test_obstacle_line_excludes_segment_vo(seed):
    """Every velocity that reaches the segment's r-capsule within tau_o is cut
    off by the line, the nearest such velocity lies on the line, and v = 0 is
    allowed when not overlapping."""
    rng = np.random.default_rng(seed)
    p = rng.uniform(-2, 2, 2)
    seg = np.concatenate([rng.uniform(-3, 3, 2), rng.uniform(-3, 3, 2)])
    r, tau_o = 0.4, 2.0
    a, b = seg[:2], seg[2:]
    t = np.clip(((p - a) @ (b - a)) / ((b - a) @ (b - a)), 0, 1)
    if np.linalg.norm(a + t * (b - a) - p) <= r + 0.05:
        pytest.skip("overlapping draw")
    q, n = oracle.obstacle_line(p, (0, 0), r, 1.4, seg, tau_o, 0.1)
    assert (np.zeros(2) - q) @ n > 0
    # sample the capsule and scale into the VO: v = (x - p)/t, t in (0, tau_o]
    s = rng.uniform(0, 1, 4000)
    ang = rng.uniform(0, 2 * math.pi, 4000)
    rad = r * np.sqrt(rng.uniform(0, 1, 4000))
    x = a[None] + s[:, None] * (b - a)[None] + rad[:, None] * np.stack([np.cos(ang), np.sin(ang)], 1)
    tt = tau_o * rng.uniform(1e-3, 1, 4000)
    vo = (x - p[None]) / tt[:, None]
    assert np.all((vo - q[None]) @ n <= 1e-12)
    # nearest VO velocity m (d - r)/tau_o is on the line
    c = a + t * (b - a)
    d = np.linalg.norm(c - p)
    vnear = (c - p) / d * (d - r) / tau_o
    assert abs((vnear - q) @ n) < 1e-12


# ----------------------------------------------------------------------------- O5 brute force

def brute_lp(lines, vmax, pref, tol=1e-12):
    """Closest feasible point to pref among all candidate optimum locations."""
    pref = np.asarray(pref, float)
    cands = [pref.copy()]
    pl = np.linalg.norm(pref)
    if pl > 0:
        cands.append(pref / pl * vmax)
    L = [(np.asarray(q, float), np.asarray(n, float)) for q, n in lines]
    for q, n in L:
        cands.append(pref - ((pref - q) @ n) * n)  # projection onto the line
        # line x circle
        d = np.array([-n[1], n[0]])
        qd = q @ d
        disc = qd * qd - q @ q + vmax * vmax
        if disc >= 0:
            for sgn in (-1, 1):
                cands.append(q + (-qd + sgn * math.sqrt(disc)) * d)
    for a in range(len(L)):
        for b in range(a + 1, len(L)):
            (qa, na), (qb, nb) = L[a], L[b]
            A = np.array([na, nb])
            if abs(np.linalg.det(A)) < 1e-12:
                continue
            cands.append(np.linalg.solve(A, [qa @ na, qb @ nb]))
    best = None
    for c in cands:
        if c @ c > vmax * vmax * (1 + tol) + tol:
            continue
        if any((c - q) @ n < -tol for q, n in L):
            continue
        dist = np.linalg.norm(c - pref)
        if best is None or dist < best[0]:
            best = (dist, c)
    return None if best is None else best[1]


def _random_lines(rng, m, spread=1.0):
    lines = []
    for _ in range(m):
        th = rng.uniform(0, 2 * math.pi)
        n = np.array([math.cos(th), math.sin(th)])
        q = rng.uniform(-spread, spread, 2)
        lines.append((q, n))
    return lines


def _margin(lines, vmax):
    """Largest slack of the feasible set (LP on a fine grid): >0 feasible, <0 infeasible."""
    g = np.linspace(-vmax, vmax, 401)
    X, Y = np.meshgrid(g, g)
    P = np.stack([X.ravel(), Y.ravel()], 1)
    P = P[(P ** 2).sum(1) <= vmax * vmax]
    s = np.full(len(P), np.inf)
    for q, n in lines:
        s = np.minimum(s, (P - q) @ n)
    return s.max()


@pytest.mark.parametrize("seed", range(60))
def test_lp_matches_vertex_enumeration(seed):
    rng = np.random.default_rng(1000 + seed)
    m = int(rng.integers(1, 7))
    vmax = rng.uniform(0.8, 2.0)
    lines = _random_lines(rng, m, 0.8)
    pref = rng.uniform(-2.5, 2.5, 2)
    if abs(_margin(lines, vmax)) < 0.02:
        pytest.skip("near the feasibility boundary")
    v, k = oracle.lp2(lines, vmax, pref)
    bf = brute_lp(lines, vmax, pref)
    if bf is None:
        assert k < m
    else:
        assert k == m
        assert np.linalg.norm(v - bf) < 1e-12


def test_lp_order_invariance():
    """The optimum is unique, so the line order changes only rounding."""
    rng = np.random.default_rng(7)
    hits = 0
    for _ in range(200):
        lines = _random_lines(rng, 5, 0.5)
        pref = rng.uniform(-2, 2, 2)
        v, k = oracle.lp2(lines, 1.5, pref)
        if k < 5:
            continue
        hits += 1
        v2, k2 = oracle.lp2(lines[::-1], 1.5, pref)
        assert k2 == 5 and np.linalg.norm(v - v2) < 1e-12
    assert hits > 20


# ----------------------------------------------------------------------------- O6

def test_fallback_corridor_closed_form():
    """Two parallel opposing agent lines with a gap of -1: the least maximal
    penetration is 1/2 on the mid line; the tie along it goes to pref."""
    lines = [((0.0, 0.5), (0.0, 1.0)), ((0.0, -0.5), (0.0, -1.0))]
    v, k = oracle.lp2(lines, 2.0, (1.0, 0.3))
    assert k < 2
    v, ds = oracle.fallback(lines, 0, 2.0, (1.0, 0.3))
    assert abs(ds - 0.5) < 1e-12
    assert np.allclose(v, [1.0, 0.0], atol=1e-11)


def test_fallback_equilateral_closed_form():
    """Three lines v.n_k >= c with n_k 120 degrees apart: d* = c at v = 0."""
    c = 0.3
    lines = []
    for k in range(3):
        th = 2 * math.pi * k / 3 + 0.4
        n = np.array([math.cos(th), math.sin(th)])
        lines.append((c * n, n))
    v, ds = oracle.fallback(lines, 0, 1.5, (0.7, -0.2))
    assert abs(ds - c) < 1e-12
    assert np.linalg.norm(v) < 1e-11


def test_fallback_hard_lines_respected():
    """Static lines stay hard: the agent lines give way."""
    hard = [((0.0, -0.2), (0.0, -1.0))]  # v_y <= -0.2
    soft = [((0.0, 0.4), (0.0, 1.0)), ((0.5, 0.0), (1.0, 0.0))]  # v_y >= 0.4, v_x >= 0.5
    v, ds = oracle.fallback(hard + soft, 1, 2.0, (0.0, 1.0))
    # best max-penetration: v_y = -0.2 (penetration 0.6 of the first soft line), v_x free >= 0.5 - 0.6
    assert abs(ds - 0.6) < 1e-12
    assert abs(v[1] + 0.2) < 1e-11 and abs(v[0] - 0.0) < 1e-11


def _brute_fallback(lines, n_hard, vmax, pref):
    """Bisection on d with the brute-force LP as feasibility test, then the closest point."""
    hard, soft = lines[:n_hard], lines[n_hard:]
    if brute_lp(hard, vmax, pref) is None:
        hard, soft = [], lines
    shift = lambda d: [(np.asarray(q) - d * np.asarray(n), np.asarray(n)) for q, n in soft]
    lo, hi = 0.0, 4 * vmax + 10
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if brute_lp(hard + shift(mid), vmax, pref, tol=1e-13) is None:
            lo = mid
        else:
            hi = mid
        if hi - lo < 1e-13:
            break
    return brute_lp(hard + shift(hi), vmax, pref, tol=1e-12), hi


@pytest.mark.parametrize("seed", range(30))
def test_fallback_matches_brute_force(seed):
    rng = np.random.default_rng(5000 + seed)
    found = False
    for _ in range(200):
        m = int(rng.integers(3, 6))
        lines = _random_lines(rng, m, 1.5)
        vmax = rng.uniform(0.8, 1.6)
        if _margin(lines, vmax) < -0.05:
            found = True
            break
    assert found
    n_hard = int(rng.integers(0, 2))
    pref = rng.uniform(-1.5, 1.5, 2)
    v, ds = oracle.fallback(lines, n_hard, vmax, pref)
    bv, bd = _brute_fallback(lines, n_hard, vmax, pref)
    assert abs(ds - bd) < 1e-9
    assert np.linalg.norm(v - bv) < 1e-6


# ----------------------------------------------------------------------------- O2

def test_neighbor_order_and_ties():
    # agent 0 at the origin; others at distances 1 (ids 5 and 3: tie -> 3 first), 2, 3, 4.9, 5 (excluded: key < R^2), 6
    pos = np.zeros((8, 2))
    pos[5] = (1, 0)
    pos[3] = (0, -1)
    pos[1] = (2, 0)
    pos[7] = (0, 3)
    pos[2] = (-4.9, 0)
    pos[4] = (5, 0)
    pos[6] = (6, 0)
    ids, keys = oracle.neighbors(pos, 0, 5.0, 10)
    assert list(ids) == [3, 5, 1, 7, 2]
    ids, _ = oracle.neighbors(pos, 0, 5.0, 3)
    assert list(ids) == [3, 5, 1]
    ids, _ = oracle.neighbors(pos, 0, 5.0, 0)
    assert list(ids) == []


def test_rank_key_has_no_fused_multiply_add():
    """The key rounds dx*dx and dy*dy separately (two roundings, then the sum)."""
    rng = np.random.default_rng(3)
    differ = 0
    for _ in range(2000):
        xi, yi, xj, yj = (float(np.float32(v)) for v in rng.uniform(-50, 50, 4))
        dx, dy = xj - xi, yj - yi
        k = oracle.rank_key((xi, yi), (xj, yj))
        assert k == np.float64(dx) * np.float64(dx) + np.float64(dy) * np.float64(dy)
        # the exactly rounded sum of exact squares differs in some cases: the key is not that
        from fractions import Fraction
        exact = Fraction(dx) ** 2 + Fraction(dy) ** 2
        differ += float(exact) != k
    assert differ > 0


@pytest.mark.parametrize("seed", range(3))
def test_neighbor_lists_are_the_k_smallest(seed):
    sc = plain_square(seed, n=64, side=12.0)
    pos = sc.pos.astype(np.float64)
    R, K = 3.0, 6
    for i in range(len(pos)):
        ids, keys = oracle.neighbors(pos, i, R, K)
        d2 = ((pos - pos[i]) ** 2).sum(1)
        order = sorted((d2[j], j) for j in range(len(pos)) if j != i and d2[j] < R * R)
        assert [j for _, j in order[:K]] == list(ids)


# ----------------------------------------------------------------------------- invariants

def _check_step_invariants(o, sc, pos, vel, robot_vel, nv, st):
    K = sc.max_neighbors
    es = sc.env_start
    prm = o.params  # the FP32-rounded parameters the oracle steps with
    tau_o, tau, dt, R, ra = prm.tau_obst, prm.tau, prm.dt, prm.neighbor_dist, prm.robot_alpha
    for e in range(sc.n_envs):
        base, n = es[e], es[e + 1] - es[e]
        segs = sc.segments[sc.seg_start[e]:sc.seg_start[e + 1]].astype(np.float64)
        robot = sc.robot_index[e]
        V = vel[base:base + n].copy()
        if robot >= 0:
            V[robot] = robot_vel[e]
        for i in range(n):
            g = base + i
            if i == robot:
                continue
            vmax = float(sc.max_speed[g])
            assert np.linalg.norm(nv[g]) <= vmax * (1 + 1e-12) + 1e-15
            ids, _ = oracle.neighbors(pos[base:base + n], i, R, K)
            oids = oracle.obstacles(segs, pos[g], float(sc.radius[g]) + tau_o * vmax) if len(segs) else []
            lines = []
            for s in oids:
                if prm.seg_mode == 1:
                    if oracle.segment_covered(pos[g], sc.radius[g], segs[s], tau_o, lines):
                        continue
                    lines.append(oracle.obstacle_line_vd(pos[g], V[i], sc.radius[g], vmax, segs[s], tau_o, dt))
                else:
                    lines.append(oracle.obstacle_line(pos[g], V[i], sc.radius[g], vmax, segs[s], tau_o, dt))
            n_hard = len(lines)
            for j in ids:
                alpha = ra if j == robot else 0.5
                lines.append(oracle.agent_line(pos[g], V[i], sc.radius[g], pos[base + j], V[j],
                                               sc.radius[base + j], tau, dt, alpha, i, j))
            if st[g] == 0:
                for q, nrm in lines:
                    assert (nv[g] - q) @ nrm >= -1e-9
            else:
                assert st[g] == 1
                hard = lines[:n_hard]
                if brute_lp(hard, vmax, (0.0, 0.0)) is not None:
                    for q, nrm in hard:
                        assert (nv[g] - q) @ nrm >= -1e-9


@pytest.mark.parametrize("maker", ["plain", "urban", "urban_velocity_segments"])
def test_rollout_invariants(maker):
    sc = plain_square(1, n=32) if maker == "plain" else urban_block(1, n_envs=2, n_peds=48, steps=40)
    if maker == "urban_velocity_segments":
        sc = dataclasses.replace(sc, segment_mode=1)
    o = oracle.OracleScene(sc)
    pos, vel = sc.pos.astype(np.float64), sc.vel.astype(np.float64)
    for k in range(40):
        rv = sc.robot_vel_at(k).astype(np.float64)
        npos, nvel, nb, st = o.step(pos, vel, rv)
        _check_step_invariants(o, sc, pos, vel, rv, nvel, st)
        assert np.allclose(npos, pos + o.params.dt * nvel, atol=1e-14)
        pos, vel = npos, nvel


def test_no_overlap_guarantee():
    """ORCA's pairwise guarantee: when i and j list each other, both LPs are
    feasible (each new velocity lies in its reciprocal half-plane) and they do
    not overlap now, they do not overlap after the step."""
    checked = 0
    for seed in range(4):
        sc = plain_square(10 + seed, n=40, side=10.0)
        o = oracle.OracleScene(sc)
        pos, vel = sc.pos.astype(np.float64), sc.vel.astype(np.float64)
        r = sc.radius.astype(np.float64)
        for k in range(120):
            npos, nvel, nb, st = o.step(pos, vel)
            n = len(pos)
            lists = [set(nb[i][nb[i] >= 0]) for i in range(n)]
            for i in range(n):
                for j in lists[i]:
                    if j <= i or i not in lists[j] or st[i] != 0 or st[j] != 0:
                        continue
                    lim = r[i] + r[j]
                    if np.linalg.norm(pos[i] - pos[j]) < lim:
                        continue
                    assert np.linalg.norm(npos[i] - npos[j]) >= lim - 1e-9, (k, i, j)
                    checked += 1
            pos, vel = npos, nvel
    assert checked > 1000


def test_collision_counter_hand_case():
    sc = one_env([[0, 0], [0.5, 0], [3, 0], [10, 0], [10.5995, 0], [20, 0]], [[0, 0]] * 6, [[0, 0]] * 6, 0.3, 1.0,
                 segs=[(2.8, -1, 2.8, 1), (20.2995, -1, 20.2995, 1)])
    o = oracle.OracleScene(sc)
    a, s = o.collisions(sc.pos.astype(np.float64))
    assert a[0] == 1  # agents 0 and 1 overlap by 0.1 m; 3 and 4 by 0.5 mm only (below the 1 mm depth)
    assert s[0] == 1  # agent 2 is 0.2 from a segment (< 0.3); agent 5 penetrates the other by 0.5 mm only
