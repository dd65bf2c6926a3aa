"""FP64 CPU oracle for the batched ORCA crowd step (test infrastructure).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path (the CUDA library and
its binding) never imports it, and the two share no code: the arithmetic here
lives in ``orca_oracle.c`` (plain C, FP64, compiled with -ffp-contract=off),
loaded with ctypes.

Stages follow the per-step update of the paper's dynamic agents (Sec. 3.2,
"Interactive Dynamics Generation") with the ORCA geometry of the method the
paper cites for it (van den Berg et al., ISRR 2011):
  O1 preferred velocity, O2 neighbours and nearby segments, O3 reciprocal agent
  half-planes, O4 static-segment half-planes, O5 incremental 2D LP, O6
  min-max-penetration fallback, O7 explicit Euler integration, O8 rollout
  statistics (collision indicator and speed of the paper's metric table,
  Appendix "Evaluation Metrics").
Around the step: goal queues (advance_goals), goal pools drawn with
Philox4x32-10 (advance_goals_pool), episodes that start
environments over on their own schedules or by a mask (episode_restarts,
restart_rows, restart_masked; Sec. 3.3), lane-following cars (``oracle.vehicles``) and the occupancy-map
front end (``oracle.frontend``).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "orca_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liborca_oracle.so")
_lock = threading.Lock()
_lib = None

ROBOT_STATUS = 2
FALLBACK_STATUS = 1


class Params(C.Structure):
    _fields_ = [("tau", C.c_double), ("tau_obst", C.c_double), ("neighbor_dist", C.c_double),
                ("dt", C.c_double), ("robot_alpha", C.c_double), ("max_neighbors", C.c_int32),
                ("seg_mode", C.c_int32)]


class Line(C.Structure):
    _fields_ = [("qx", C.c_double), ("qy", C.c_double), ("nx", C.c_double), ("ny", C.c_double)]


def build(force: bool = False) -> str:
    """Compile the oracle library (gcc, FP64, no FMA contraction, OpenMP)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC",
                               "-shared", "-std=c11", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            d, i32, i64, pd = C.c_double, C.c_int32, C.c_int64, C.POINTER(C.c_double)
            pi32, pi64 = C.POINTER(C.c_int32), C.POINTER(C.c_int64)
            L.or_pref_velocity.argtypes = [d, d, d, d, d, d, pd, pd]
            L.or_rank_key.argtypes = [d, d, d, d]
            L.or_rank_key.restype = d
            L.or_neighbors.argtypes = [C.c_int, pd, C.c_int, d, C.c_int, pi32, pd]
            L.or_neighbors.restype = C.c_int
            L.or_seg_dist2.argtypes = [d, d, pd]
            L.or_seg_dist2.restype = d
            L.or_obstacles.argtypes = [C.c_int, pd, d, d, d, pi32]
            L.or_obstacles.restype = C.c_int
            L.or_agent_line.argtypes = [d] * 13 + [C.c_int, C.c_int, C.POINTER(Line)]
            L.or_obstacle_line.argtypes = [d] * 6 + [pd, d, d, C.POINTER(Line)]
            L.or_obstacle_line_vd.argtypes = [d] * 6 + [pd, d, d, C.POINTER(Line)]
            L.or_segment_covered.argtypes = [d, d, d, pd, d, C.POINTER(Line), C.c_int]
            L.or_segment_covered.restype = C.c_int
            L.or_lp2.argtypes = [C.POINTER(Line), C.c_int, d, d, d, pd, pd]
            L.or_lp2.restype = C.c_int
            L.or_fallback.argtypes = [C.POINTER(Line), C.c_int, C.c_int, d, d, d, pd, pd, pd]
            L.or_step.argtypes = [i32, pi64, pd, pd, pd, pi32, pi64, pd, C.POINTER(Params), pd, pd, pd, pd,
                                  pi32, i64, pi64, pd, pd, pi32, pi32, C.c_int, pi64]
            L.or_step.restype = C.c_int
            L.or_collisions.argtypes = [i32, pi64, pd, pi64, pd, pd, pi64, pi64]
            _lib = L
    return _lib


def _p(a, ct):
    return a.ctypes.data_as(C.POINTER(ct))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


# ------------------------------------------------------------------ single stages

def pref_velocity(p, g, speed, dt):
    """O1."""
    vx, vy = C.c_double(), C.c_double()
    lib().or_pref_velocity(float(p[0]), float(p[1]), float(g[0]), float(g[1]), float(speed), float(dt),
                           C.byref(vx), C.byref(vy))
    return np.array([vx.value, vy.value])


def advance_goals(pos, radius, goal, idx, queue, cyclic, skip=None):
    """Goal queues (a reading: the paper's agents walk between sampled start
    and end points, Sec. 3.2, and the simulation runs on past an arrival).

    At the start of a step, every agent (rows of `skip` excepted: the robot)
    whose position p lies within its radius r of its current goal g,
    (gx - px)^2 + (gy - py)^2 <= r^2 in FP64 with each operation rounded once,
    moves on to the next goal of its queue: queue[i][idx + 1], wrapping to
    the start when `cyclic`, else staying at the last goal.  Returns the new
    (goal [N][2], idx [N]); the inputs are not modified."""
    p = np.asarray(pos, np.float64).reshape(-1, 2)
    g = np.array(goal, np.float64).reshape(-1, 2)
    k = np.array(idx, np.int64).reshape(-1)
    qu = np.asarray(queue, np.float64)
    n_goals = qu.shape[1]
    r = np.asarray(radius, np.float64).reshape(-1)
    dx = g[:, 0] - p[:, 0]
    dy = g[:, 1] - p[:, 1]
    reached = dx * dx + dy * dy <= r * r
    if skip is not None:
        reached &= ~np.asarray(skip, bool)
    move = reached & (bool(cyclic) | (k + 1 < n_goals))
    k[move] += 1
    rows = np.nonzero(move)[0]
    g[rows] = qu[rows, k[rows] % n_goals]
    return g, k


def advance_goals_pool(pos, radius, goal, idx, pool_start, pool, env_of, seed, skip=None):
    """Goal pools (a reading: the paper samples agents' start and end points
    on the traversable ground, Sec. 3.2, and its simulation runs on past an
    arrival): at the start of a step every agent g (rows of `skip` excepted)
    within its radius of its goal, decided as advance_goals decides it, draws
    its next goal from its environment's pool of points: with k = idx[g] the
    draws it made so far, u = Philox4x32-10(counter (g, k, 0, 0), key (seed
    low 32 bits, seed high 32 bits)), the pick is floor(u0 * n / 2^32) of the
    n points of environment env_of[g] (none when n = 0), and idx[g] = k + 1.
    Returns the new (goal [N][2], idx [N]); the inputs are not modified."""
    from .frontend import philox4x32_10

    p = np.asarray(pos, np.float64).reshape(-1, 2)
    g = np.array(goal, np.float64).reshape(-1, 2)
    k = np.array(idx, np.int64).reshape(-1)
    ps = np.asarray(pool_start, np.int64).reshape(-1)
    pl = np.asarray(pool, np.float64).reshape(-1, 2)
    r = np.asarray(radius, np.float64).reshape(-1)
    dx = g[:, 0] - p[:, 0]
    dy = g[:, 1] - p[:, 1]
    reached = dx * dx + dy * dy <= r * r
    if skip is not None:
        reached &= ~np.asarray(skip, bool)
    key = (int(seed) & 0xFFFFFFFF, (int(seed) >> 32) & 0xFFFFFFFF)
    for a in np.nonzero(reached)[0]:
        e = int(env_of[a])
        n = int(ps[e + 1] - ps[e])
        if n == 0:
            continue
        u0 = philox4x32_10((int(a), int(k[a]), 0, 0), key)[0]
        g[a] = pl[ps[e] + ((u0 * n) >> 32)]
        k[a] += 1
    return g, k


def episode_restarts(t, steps):
    """Episodes (Sec. 3.3: asynchronous scene sampling trains on many
    environments at once whose episodes differ, so each environment starts
    over on its own schedule).  Environment e with steps[e] > 0 starts over at
    the start of step t of the episode clock (the first step after the
    episodes are set up is t = 0) when t > 0 and t is a multiple of steps[e];
    steps[e] = 0 never starts over.  Returns the [E] bool mask."""
    st = np.asarray(steps, np.int64).reshape(-1)
    t = int(t)
    return (st > 0) & (t > 0) & (t % np.maximum(st, 1) == 0)


def restart_masked(mask, owner, current, snapshot):
    """Environments e with mask[e] set start over: the rows of `current`
    whose environment owner[row] is masked take the rows of `snapshot`; the
    others are kept.  Returns a new array."""
    out = np.array(current, copy=True)
    sel = np.asarray(mask, bool).reshape(-1)[np.asarray(owner, np.int64).reshape(-1)]
    out[sel] = np.asarray(snapshot)[sel]
    return out


def restart_rows(t, steps, owner, current, snapshot):
    """The rows of `current` whose environment owner[row] starts over at step
    t (episode_restarts) take the rows of `snapshot`; the others are kept.
    Applied at the start of the step, before anything else of it (goal queues,
    cars, the robot command), so the state read after the step that ends an
    episode is that episode's last state.  Returns a new array."""
    return restart_masked(episode_restarts(t, steps), owner, current, snapshot)


def rank_key(pi, pj):
    """O2 ranking key (FP64 squared distance, no FMA)."""
    return lib().or_rank_key(float(pi[0]), float(pi[1]), float(pj[0]), float(pj[1]))


def neighbors(pos, i, R, K):
    """O2: env-local ids of the K nearest agents within R, ordered by (key, id)."""
    pos = _f64(pos).reshape(-1, 2)
    ids = np.zeros(max(K, 1), np.int32)
    keys = np.zeros(max(K, 1), np.float64)
    n = lib().or_neighbors(len(pos), _p(pos, C.c_double), int(i), float(R), int(K), _p(ids, C.c_int32),
                           _p(keys, C.c_double))
    return ids[:n].copy(), keys[:n].copy()


def obstacles(segs, p, reach):
    """O2 (segments): ids of segments closer than reach, ordered by (distance, id)."""
    segs = _f64(segs).reshape(-1, 4)
    ids = np.zeros(max(len(segs), 1), np.int32)
    n = lib().or_obstacles(len(segs), _p(segs, C.c_double), float(p[0]), float(p[1]), float(reach),
                           _p(ids, C.c_int32))
    return ids[:n].copy()


def agent_line(pi, vi, ri, pj, vj, rj, tau, dt, alpha=0.5, id_i=0, id_j=1):
    """O3: returns (q, n) with the allowed side (v - q).n >= 0."""
    ln = Line()
    lib().or_agent_line(float(pi[0]), float(pi[1]), float(vi[0]), float(vi[1]), float(ri),
                        float(pj[0]), float(pj[1]), float(vj[0]), float(vj[1]), float(rj),
                        float(tau), float(dt), float(alpha), int(id_i), int(id_j), C.byref(ln))
    return np.array([ln.qx, ln.qy]), np.array([ln.nx, ln.ny])


def obstacle_line(p, v, r, vmax, seg, tau_o, dt):
    """O4: returns (q, n)."""
    ln = Line()
    s = _f64(seg).reshape(4)
    lib().or_obstacle_line(float(p[0]), float(p[1]), float(v[0]), float(v[1]), float(r), float(vmax),
                           _p(s, C.c_double), float(tau_o), float(dt), C.byref(ln))
    return np.array([ln.qx, ln.qy]), np.array([ln.nx, ln.ny])


def obstacle_line_vd(p, v, r, vmax, seg, tau_o, dt):
    """O4v (velocity-dependent segment half-plane): returns (q, n)."""
    ln = Line()
    s = _f64(seg).reshape(4)
    lib().or_obstacle_line_vd(float(p[0]), float(p[1]), float(v[0]), float(v[1]), float(r), float(vmax),
                              _p(s, C.c_double), float(tau_o), float(dt), C.byref(ln))
    return np.array([ln.qx, ln.qy]), np.array([ln.nx, ln.ny])


def segment_covered(p, r, seg, tau_o, lines):
    """O4v: whether an earlier segment line (q, n) already forbids the whole
    velocity obstacle of `seg` (then the segment gets no line)."""
    arr = (Line * max(1, len(lines)))()
    for k, (q, n) in enumerate(lines):
        arr[k] = Line(float(q[0]), float(q[1]), float(n[0]), float(n[1]))
    s = _f64(seg).reshape(4)
    return bool(lib().or_segment_covered(float(p[0]), float(p[1]), float(r), _p(s, C.c_double), float(tau_o), arr,
                                         len(lines)))


def _lines(lines):
    arr = (Line * max(len(lines), 1))()
    for k, (q, n) in enumerate(lines):
        arr[k] = Line(float(q[0]), float(q[1]), float(n[0]), float(n[1]))
    return arr


def lp2(lines, vmax, pref):
    """O5: returns (v, fail_index) with fail_index == len(lines) when feasible."""
    arr = _lines(lines)
    vx, vy = C.c_double(), C.c_double()
    k = lib().or_lp2(arr, len(lines), float(vmax), float(pref[0]), float(pref[1]), C.byref(vx), C.byref(vy))
    return np.array([vx.value, vy.value]), k


def fallback(lines, n_hard, vmax, pref):
    """O6: returns (v, d_star)."""
    arr = _lines(lines)
    vx, vy, ds = C.c_double(), C.c_double(), C.c_double()
    lib().or_fallback(arr, len(lines), int(n_hard), float(vmax), float(pref[0]), float(pref[1]),
                      C.byref(vx), C.byref(vy), C.byref(ds))
    return np.array([vx.value, vy.value]), ds.value


# ------------------------------------------------------------------ whole step

def _f32(x):
    return float(np.float32(x))


def scene_params(scene):
    """Scene parameters as the FP32 values the crowd library receives, held in FP64."""
    return Params(_f32(scene.tau), _f32(scene.tau_obst), _f32(scene.neighbor_dist), _f32(scene.dt),
                  _f32(scene.robot_responsibility), scene.max_neighbors, int(getattr(scene, "segment_mode", 0)))


class OracleScene:
    """FP64 copies of a Scene's static arrays, ready for repeated steps."""

    def __init__(self, scene):
        self.scene = scene
        self.E = scene.n_envs
        self.N = scene.n_agents
        self.K = scene.max_neighbors
        self.env_start = np.ascontiguousarray(scene.env_start, np.int64)
        self.seg_start = np.ascontiguousarray(scene.seg_start, np.int64)
        self.radius = _f64(scene.radius)
        self.vmax = _f64(scene.max_speed)
        self.pref = _f64(scene.pref_speed)
        self.robot = np.ascontiguousarray(scene.robot_index, np.int32)
        self.segs = _f64(scene.segments).reshape(-1, 4)
        if self.segs.size == 0:
            self.segs = np.zeros((1, 4))
        self.goal = _f64(scene.goal)
        self.params = scene_params(scene)
        self.dt = self.params.dt

    WORK_KEYS = ("agent_steps", "pairs_in_range", "agent_lines", "obstacle_lines", "lp_checks", "lp_solves",
                 "lp_solve_lines", "fallbacks")

    def step(self, pos, vel, robot_vel=None, sel=None, threads=1, goal=None, kind=None, work=None):
        """O1-O7 for the selected agents (all when sel is None).  `kind` [N]:
        1 marks vehicles, which keep the given velocity (their lane model's).
        `work` (a dict, may be None): the step's work items (WORK_KEYS) are
        added into it.

        Returns (pos_out, vel_out, nbrs [N,K] env-local ids -1 padded, status [N]);
        rows of unselected agents are left as NaN / -9."""
        kd = None if kind is None else np.ascontiguousarray(kind, np.int32)
        pos, vel = _f64(pos).reshape(-1, 2), _f64(vel).reshape(-1, 2)
        goal = self.goal if goal is None else _f64(goal).reshape(-1, 2)
        rv = _f64(np.zeros((self.E, 2)) if robot_vel is None else robot_vel).reshape(-1, 2)
        po = np.full((self.N, 2), np.nan)
        vo = np.full((self.N, 2), np.nan)
        nb = np.full((self.N, max(self.K, 1)), -9, np.int32)
        st = np.full(self.N, -9, np.int32)
        wk = np.zeros(8, np.int64)
        if sel is None:
            ns, sp = 0, None
        else:
            s = np.ascontiguousarray(sel, np.int64)
            ns, sp = len(s), _p(s, C.c_int64)
        rc = lib().or_step(self.E, _p(self.env_start, C.c_int64), _p(self.radius, C.c_double),
                           _p(self.vmax, C.c_double), _p(self.pref, C.c_double), _p(self.robot, C.c_int32),
                           _p(self.seg_start, C.c_int64), _p(self.segs, C.c_double), C.byref(self.params),
                           _p(pos, C.c_double), _p(vel, C.c_double), _p(goal, C.c_double), _p(rv, C.c_double),
                           None if kd is None else _p(kd, C.c_int32),
                           ns, sp, _p(po, C.c_double), _p(vo, C.c_double), _p(nb, C.c_int32),
                           _p(st, C.c_int32), int(threads), _p(wk, C.c_int64))
        if rc != 0:
            raise ValueError("oracle step rejected its arguments")
        if work is not None:
            for key, v in zip(self.WORK_KEYS, wk):
                work[key] = work.get(key, 0) + int(v)
        return po, vo, nb[:, : self.K], st

    def collisions(self, pos):
        """O8: per-env (agent-pair, agent-segment) collision events of one state."""
        pos = _f64(pos).reshape(-1, 2)
        a = np.zeros(self.E, np.int64)
        s = np.zeros(self.E, np.int64)
        lib().or_collisions(self.E, _p(self.env_start, C.c_int64), _p(self.radius, C.c_double),
                            _p(self.seg_start, C.c_int64), _p(self.segs, C.c_double), _p(pos, C.c_double),
                            _p(a, C.c_int64), _p(s, C.c_int64))
        return a, s


def rollout(scene, steps, threads=1, record=False, fp32_state=False):
    """Free-running FP64 rollout from the scene's initial state.

    O8 statistics over the non-robot agents: collision events summed over the
    post-integration states of every step (pairs involving the robot count),
    mean speed over agents and steps, goal reach (first step with
    |g - p| <= r), mean reach time in seconds and fraction reached.

    fp32_state: hold the state between steps in FP32, the format the crowd
    library's boundary stores and exchanges it in (each step still computes
    in FP64 from that state, as under teacher forcing); the statistics are
    then taken on the rounded state.
    """
    o = OracleScene(scene)
    pos = _f64(scene.pos).copy()
    vel = _f64(scene.vel).copy()
    ped = np.ones(o.N, bool)
    for e in range(o.E):
        if scene.robot_index[e] >= 0:
            ped[o.env_start[e] + scene.robot_index[e]] = False
    reach = np.full(o.N, -1, np.int64)
    coll_a = coll_s = 0
    speed_sum = 0.0
    states = []
    for k in range(steps):
        pos, vel, _, _ = o.step(pos, vel, scene.robot_vel_at(k), threads=threads)
        if fp32_state:
            pos = pos.astype(np.float32).astype(np.float64)
            vel = vel.astype(np.float32).astype(np.float64)
        a, s = o.collisions(pos)
        coll_a += int(a.sum())
        coll_s += int(s.sum())
        speed_sum += float(np.sqrt((vel[ped] ** 2).sum(1)).sum())
        d = np.sqrt(((o.goal - pos) ** 2).sum(1))
        newly = (reach < 0) & (d <= o.radius) & ped
        reach[newly] = k + 1
        if record:
            states.append(np.concatenate([pos, vel], 1))
    return _stats(reach, ped, coll_a, coll_s, speed_sum, steps, o.dt, pos, vel, states if record else None)


def _stats(reach, ped, coll_a, coll_s, speed_sum, steps, dt, pos, vel, states):
    n_ped = int(ped.sum())
    reached = (reach > 0) & ped
    return dict(
        collisions=coll_a + coll_s, agent_collisions=coll_a, segment_collisions=coll_s,
        mean_speed=speed_sum / max(1, n_ped * steps),
        reach_fraction=float(reached.sum()) / max(1, n_ped),
        mean_reach_time=float(reach[reached].mean() * dt) if reached.any() else float("nan"),
        reach_step=reach, final_pos=pos, final_vel=vel, states=states,
    )
