"""Seeded synthetic crowd scenes (inputs only; no ORCA arithmetic lives here).

The paper builds its crowds by sampling random start and end points for each
agent on the traversable part of a generated urban block (Sec. 3.2,
"Interactive Dynamics Generation") and batches many uneven scene instances per
GPU (Sec. 3.3, "Asynchronous Scene Sampling").  Its scene datasets are not
available, so these generators stand in for them with seeded, synthetic
scenes of the shapes the paper describes: open squares, urban blocks with
rectangular buildings and sidewalk edges, uneven batches with convex polygon
obstacles, dense crowds, and a Poisson stream of rollout requests.

Both the FP64 oracle and the CUDA path consume these arrays; this module only
draws random numbers and does rejection sampling for spawn clearance.

Every generator uses ``numpy.random.Generator(PCG64(seed))``.
"""
from __future__ import annotations

from dataclasses import dataclass, field
import math

import numpy as np

# default crowd parameters shared by the plain, uneven and serving workloads
TAU = 2.0
NEIGHBOR_DIST = 5.0
MAX_NEIGHBORS = 10
DT = 0.1
CLEARANCE = 0.05  # extra spacing at spawn between agents and from obstacles


@dataclass
class Scene:
    """A batch of independent crowd environments, agents ordered env-major."""

    name: str
    agents_per_env: np.ndarray  # int32 [E]
    radius: np.ndarray  # float32 [N]
    max_speed: np.ndarray  # float32 [N]
    pref_speed: np.ndarray  # float32 [N]
    pos: np.ndarray  # float32 [N, 2]
    vel: np.ndarray  # float32 [N, 2]
    goal: np.ndarray  # float32 [N, 2]
    robot_index: np.ndarray  # int32 [E], env-local index or -1
    segs_per_env: np.ndarray  # int32 [E]
    segments: np.ndarray  # float32 [S, 4] (ax, ay, bx, by)
    tau: float = TAU
    tau_obst: float = TAU
    neighbor_dist: float = NEIGHBOR_DIST
    max_neighbors: int = MAX_NEIGHBORS
    dt: float = DT
    robot_responsibility: float = 0.5
    segment_mode: int = 0  # 0: segment half-plane tangent at the VO point nearest 0; 1: velocity-dependent
    steps: int = 1
    robot_vel: np.ndarray | None = None  # float32 [steps, E, 2] m/s (commanded)
    meta: dict = field(default_factory=dict)

    @property
    def n_envs(self) -> int:
        return int(self.agents_per_env.shape[0])

    @property
    def n_agents(self) -> int:
        return int(self.pos.shape[0])

    @property
    def env_start(self) -> np.ndarray:
        return np.concatenate([[0], np.cumsum(self.agents_per_env)]).astype(np.int64)

    @property
    def seg_start(self) -> np.ndarray:
        return np.concatenate([[0], np.cumsum(self.segs_per_env)]).astype(np.int64)

    def state(self) -> np.ndarray:
        """[N, 4] float32 (px, py, vx, vy)."""
        return np.concatenate([self.pos, self.vel], axis=1).astype(np.float32)

    def robot_vel_at(self, step: int) -> np.ndarray:
        if self.robot_vel is None:
            return np.zeros((self.n_envs, 2), np.float32)
        return self.robot_vel[step % self.robot_vel.shape[0]]

    def subset(self, envs) -> "Scene":
        """The scene restricted to the listed environments (same arrays, re-packed)."""
        envs = np.asarray(envs, dtype=np.int64)
        es, ss = self.env_start, self.seg_start
        ai = np.concatenate([np.arange(es[e], es[e + 1]) for e in envs]) if len(envs) else np.zeros(0, np.int64)
        si = np.concatenate([np.arange(ss[e], ss[e + 1]) for e in envs]) if len(envs) else np.zeros(0, np.int64)
        return Scene(
            name=f"{self.name}[{len(envs)} envs]",
            agents_per_env=self.agents_per_env[envs].copy(),
            radius=self.radius[ai].copy(), max_speed=self.max_speed[ai].copy(),
            pref_speed=self.pref_speed[ai].copy(), pos=self.pos[ai].copy(), vel=self.vel[ai].copy(),
            goal=self.goal[ai].copy(), robot_index=self.robot_index[envs].copy(),
            segs_per_env=self.segs_per_env[envs].copy(),
            segments=self.segments[si].copy() if len(si) else np.zeros((0, 4), np.float32),
            tau=self.tau, tau_obst=self.tau_obst, neighbor_dist=self.neighbor_dist,
            max_neighbors=self.max_neighbors, dt=self.dt,
            robot_responsibility=self.robot_responsibility, segment_mode=self.segment_mode, steps=self.steps,
            robot_vel=None if self.robot_vel is None else self.robot_vel[:, envs].copy(),
            meta=dict(self.meta),
        )


# ----------------------------------------------------------------------------
# spawn helpers (rejection sampling; plain geometry for clearance only)
# ----------------------------------------------------------------------------

def _seg_point_dist(px, py, segs):
    """Distance from each point to the nearest of ``segs`` (spawn clearance)."""
    if len(segs) == 0:
        return np.full(np.shape(px), np.inf)
    ax, ay, bx, by = (segs[:, k][None, :] for k in range(4))
    px = np.asarray(px, np.float64)[..., None]
    py = np.asarray(py, np.float64)[..., None]
    ex, ey = bx - ax, by - ay
    t = np.clip(((px - ax) * ex + (py - ay) * ey) / (ex * ex + ey * ey), 0.0, 1.0)
    cx, cy = ax + t * ex, ay + t * ey
    return np.sqrt((px - cx) ** 2 + (py - cy) ** 2).min(axis=-1)


def _inside_any(px, py, polys):
    """True where the point lies inside one of the convex CCW polygons."""
    inside = np.zeros(np.shape(px), bool)
    for poly in polys:
        n = len(poly)
        ok = np.ones(np.shape(px), bool)
        for k in range(n):
            ax, ay = poly[k]
            bx, by = poly[(k + 1) % n]
            ok &= (bx - ax) * (py - ay) - (by - ay) * (px - ax) >= 0.0
        inside |= ok
    return inside


def _sample_points(rng, n, radii, lo, hi, segs, polys, separate=True, max_tries=200000):
    """Draw n points in [lo, hi]^2 clear of obstacles and (optionally) of each other.

    Candidates come in batches; obstacle clearance is tested for the whole
    batch at once and mutual separation through a uniform hash of the points
    already placed."""
    radii = np.asarray(radii, np.float64)
    pts = np.zeros((n, 2), np.float64)
    placed = 0
    tries = 0
    rmax = float(radii.max()) if n else 0.0
    cell = 2.0 * rmax + CLEARANCE if rmax > 0 else 1.0
    buckets = {}
    batch = 256
    while placed < n:
        cand = rng.uniform(lo, hi, size=(batch, 2))
        tries += batch
        if tries > max_tries * max(1, n // 64 + 1):
            raise RuntimeError("spawn rejection sampling did not converge")
        clear = np.ones(batch, bool)
        if len(segs):
            clear &= _seg_point_dist(cand[:, 0], cand[:, 1], segs) >= rmax + CLEARANCE
        if polys:
            clear &= ~_inside_any(cand[:, 0], cand[:, 1], polys)
        for c in cand[clear]:
            if placed >= n:
                break
            if separate:
                cx, cy = int(math.floor(c[0] / cell)), int(math.floor(c[1] / cell))
                ok = True
                for gx in (cx - 1, cx, cx + 1):
                    for gy in (cy - 1, cy, cy + 1):
                        for k in buckets.get((gx, gy), ()):
                            if math.hypot(pts[k, 0] - c[0], pts[k, 1] - c[1]) < radii[k] + radii[placed] + CLEARANCE:
                                ok = False
                                break
                        if not ok:
                            break
                    if not ok:
                        break
                if not ok:
                    continue
                buckets.setdefault((cx, cy), []).append(placed)
            pts[placed] = c
            placed += 1
    return pts


def _rect_segments(x0, y0, x1, y1):
    """Four edges of an axis-aligned rectangle, counter-clockwise."""
    return [(x0, y0, x1, y0), (x1, y0, x1, y1), (x1, y1, x0, y1), (x0, y1, x0, y0)]


def _poly_segments(poly):
    n = len(poly)
    return [(poly[k][0], poly[k][1], poly[(k + 1) % n][0], poly[(k + 1) % n][1]) for k in range(n)]


def _random_convex_polygon(rng, cx, cy, rho):
    nv = int(rng.integers(3, 7))
    ang = np.sort(rng.uniform(0.0, 2 * math.pi, nv))
    # keep vertices distinct so that no edge is degenerate
    while np.min(np.diff(np.concatenate([ang, [ang[0] + 2 * math.pi]]))) < 0.2:
        ang = np.sort(rng.uniform(0.0, 2 * math.pi, nv))
    return [(cx + rho * math.cos(a), cy + rho * math.sin(a)) for a in ang]


def _pack(name, envs, **kw) -> Scene:
    """Concatenate per-env dicts into one env-major Scene."""
    cat = lambda key, dt, shape: (np.concatenate([e[key] for e in envs]).astype(dt)
                                  if envs else np.zeros(shape, dt))
    segs = [np.asarray(e["segments"], np.float32).reshape(-1, 4) for e in envs]
    return Scene(
        name=name,
        agents_per_env=np.array([len(e["radius"]) for e in envs], np.int32),
        radius=cat("radius", np.float32, (0,)),
        max_speed=cat("max_speed", np.float32, (0,)),
        pref_speed=cat("pref_speed", np.float32, (0,)),
        pos=cat("pos", np.float32, (0, 2)).reshape(-1, 2),
        vel=cat("vel", np.float32, (0, 2)).reshape(-1, 2),
        goal=cat("goal", np.float32, (0, 2)).reshape(-1, 2),
        robot_index=np.array([e.get("robot", -1) for e in envs], np.int32),
        segs_per_env=np.array([len(s) for s in segs], np.int32),
        segments=np.concatenate(segs).astype(np.float32) if segs else np.zeros((0, 4), np.float32),
        **kw,
    )


# ----------------------------------------------------------------------------
# workloads
# ----------------------------------------------------------------------------

def plain_square(seed=0, n=32, side=20.0, steps=200) -> Scene:
    """One env, n pedestrians in an open side x side square, no obstacles.

    r 0.3 m, v_max = preferred speed 1.4 m/s, tau 2 s, neighbour distance 5 m,
    10 neighbours, dt 0.1 s.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    r = np.full(n, 0.3)
    pos = _sample_points(rng, n, r, 0.0, side, [], [])
    goal = _sample_points(rng, n, r, 0.0, side, [], [])
    env = dict(radius=r, max_speed=np.full(n, 1.4), pref_speed=np.full(n, 1.4), pos=pos,
               vel=np.zeros((n, 2)), goal=goal, segments=np.zeros((0, 4)))
    return _pack("plain_square", [env], steps=steps, meta=dict(seed=seed, side=side))


def urban_block(seed=0, n_envs=256, n_peds=128, side=40.0, n_buildings=8, steps=1000,
                robot=True, robot_vmax=1.0, robot_radius=0.4, action_steps=None) -> Scene:
    """Urban blocks: side x side m, rectangular buildings (sides U[4,10] m, four
    segments each) plus the four block-perimeter sidewalk edges; pedestrians as
    in the plain square; one robot agent per env whose commanded velocity is a
    seeded action in [-1,1]^2 scaled by its max speed.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    envs = []
    for _ in range(n_envs):
        rects = []
        tries = 0
        while len(rects) < n_buildings:
            tries += 1
            if tries > 10000:
                raise RuntimeError("building placement did not converge")
            w, h = rng.uniform(4.0, 10.0, 2)
            x0 = rng.uniform(1.0, side - 1.0 - w)
            y0 = rng.uniform(1.0, side - 1.0 - h)
            cand = (x0, y0, x0 + w, y0 + h)
            if all(cand[2] + 1.0 <= r[0] or r[2] + 1.0 <= cand[0] or
                   cand[3] + 1.0 <= r[1] or r[3] + 1.0 <= cand[1] for r in rects):
                rects.append(cand)
        segs = []
        for rc in rects:
            segs += _rect_segments(*rc)
        segs += _rect_segments(0.0, 0.0, side, side)  # sidewalk edges
        segs = np.array(segs, np.float64)
        polys = [[(r[0], r[1]), (r[2], r[1]), (r[2], r[3]), (r[0], r[3])] for r in rects]
        n = n_peds + (1 if robot else 0)
        rad = np.full(n, 0.3)
        vmax = np.full(n, 1.4)
        if robot:
            rad[-1] = robot_radius
            vmax[-1] = robot_vmax
        pos = _sample_points(rng, n, rad, 0.0, side, segs, polys)
        goal = _sample_points(rng, n, rad, 0.0, side, segs, polys)
        envs.append(dict(radius=rad, max_speed=vmax, pref_speed=vmax.copy(), pos=pos,
                         vel=np.zeros((n, 2)), goal=goal, segments=segs,
                         robot=(n - 1) if robot else -1))
    robot_vel = None
    if robot:
        na = steps if action_steps is None else action_steps
        actions = rng.uniform(-1.0, 1.0, size=(na, n_envs, 2))
        robot_vel = (actions * robot_vmax).astype(np.float32)
    return _pack("urban_block", envs, steps=steps, robot_vel=robot_vel,
                 meta=dict(seed=seed, side=side, n_buildings=n_buildings))


def _polygon_env(rng, n, density, max_polys, r_lo=0.25, r_hi=0.4, v_lo=1.0, v_hi=1.8):
    side = math.sqrt(n / density)
    n_poly = int(rng.integers(0, max_polys + 1))
    polys = []
    centres = []
    tries = 0
    while len(polys) < n_poly and tries < 20 * (n_poly + 1):
        tries += 1
        rho = rng.uniform(0.5, 3.0)
        cx, cy = rng.uniform(0.0, side, 2)
        if any(math.hypot(cx - c[0], cy - c[1]) < rho + c[2] + 1.0 for c in centres):
            continue
        centres.append((cx, cy, rho))
        polys.append(_random_convex_polygon(rng, cx, cy, rho))
    segs = []
    for p in polys:
        segs += _poly_segments(p)
    segs = np.array(segs, np.float64).reshape(-1, 4)
    rad = rng.uniform(r_lo, r_hi, n)
    vmax = rng.uniform(v_lo, v_hi, n)
    pos = _sample_points(rng, n, rad, 0.0, side, segs, polys)
    goal = _sample_points(rng, n, rad, 0.0, side, segs, polys)
    return dict(radius=rad, max_speed=vmax, pref_speed=vmax.copy(), pos=pos, vel=np.zeros((n, 2)),
                goal=goal, segments=segs)


def uneven_batch(seed=0, n_envs=1024, n_lo=16, n_hi=512, max_polys=40, density=0.25, steps=50) -> Scene:
    """Uneven batch: agent count U{n_lo..n_hi} per env, square side sqrt(N/density),
    0..max_polys random convex polygons (3-6 vertices, circumradius U[0.5,3] m),
    radii U[0.25,0.4] m, max speed U[1.0,1.8] m/s.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    envs = [_polygon_env(rng, int(rng.integers(n_lo, n_hi + 1)), density, max_polys) for _ in range(n_envs)]
    return _pack("uneven_batch", envs, steps=steps, meta=dict(seed=seed, density=density))


def dense_crowd(seed=0, n_envs=16, n_peds=20000, side=100.0, n_segs=200, steps=500,
                radius=0.25) -> Scene:
    """Dense crowd: n_peds at ~2 per m^2 in side x side m with n_segs random
    segments (length U[1,5] m).  Starts are a jittered hex lattice minus points
    near segments, subsampled; goals uniform clear of segments.  R 3 m, K 16.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    envs = []
    for _ in range(n_envs):
        a0 = rng.uniform(0.0, side, (n_segs, 2))
        ang = rng.uniform(0.0, 2 * math.pi, n_segs)
        ln = rng.uniform(1.0, 5.0, n_segs)
        segs = np.stack([a0[:, 0], a0[:, 1], a0[:, 0] + ln * np.cos(ang), a0[:, 1] + ln * np.sin(ang)], 1)
        # hex lattice slightly denser than the target so that removal near segments still leaves n_peds
        target = n_peds / (side * side) * 1.15
        a = math.sqrt(2.0 / (math.sqrt(3.0) * target))
        xs = np.arange(a / 2, side, a)
        ys = np.arange(a / 2, side, a * math.sqrt(3.0) / 2)
        gx, gy = np.meshgrid(xs, ys)
        gx = gx + (np.arange(len(ys))[:, None] % 2) * (a / 2)
        pts = np.stack([gx.ravel(), gy.ravel()], 1)
        jit = max(0.0, (a - 2 * radius - CLEARANCE) / 2 - 1e-3)
        rr = jit * np.sqrt(rng.uniform(0, 1, len(pts)))
        th = rng.uniform(0, 2 * math.pi, len(pts))
        pts = pts + np.stack([rr * np.cos(th), rr * np.sin(th)], 1)
        keep = (pts[:, 0] >= 0) & (pts[:, 0] <= side) & (pts[:, 1] >= 0) & (pts[:, 1] <= side)
        pts = pts[keep]
        clear = np.ones(len(pts), bool)
        for k in range(0, len(pts), 4096):
            clear[k:k + 4096] = _seg_point_dist(pts[k:k + 4096, 0], pts[k:k + 4096, 1], segs) >= radius + CLEARANCE
        pts = pts[clear]
        if len(pts) < n_peds:
            raise RuntimeError("dense lattice too sparse")
        pts = pts[np.sort(rng.choice(len(pts), n_peds, replace=False))]
        rad = np.full(n_peds, radius)
        goal = np.zeros((n_peds, 2))
        todo = np.arange(n_peds)
        while len(todo):
            g = rng.uniform(0.0, side, (len(todo), 2))
            ok = np.ones(len(todo), bool)
            for k in range(0, len(todo), 4096):
                ok[k:k + 4096] = _seg_point_dist(g[k:k + 4096, 0], g[k:k + 4096, 1], segs) >= radius + CLEARANCE
            goal[todo[ok]] = g[ok]
            todo = todo[~ok]
        envs.append(dict(radius=rad, max_speed=np.full(n_peds, 1.4), pref_speed=np.full(n_peds, 1.4),
                         pos=pts, vel=np.zeros((n_peds, 2)), goal=goal, segments=segs))
    return _pack("dense_crowd", envs, steps=steps, neighbor_dist=3.0, max_neighbors=16,
                 meta=dict(seed=seed, side=side))


@dataclass
class Request:
    """One rollout request of the serving workload."""

    arrival_s: float
    scene: Scene  # one env
    steps: int


def serving_stream(seed=0, rate=200.0, duration_s=10.0, n_lo=32, n_hi=2048, max_polys=60,
                   steps_lo=100, steps_hi=1000, density=0.25, max_requests=None):
    """Poisson arrivals (rate per second) of single-env rollout requests with
    log-uniform agent count in [n_lo, n_hi], 0..max_polys convex polygons and
    U{steps_lo..steps_hi} steps."""
    rng = np.random.Generator(np.random.PCG64(seed))
    t = 0.0
    reqs = []
    while True:
        t += rng.exponential(1.0 / rate)
        if t >= duration_s or (max_requests is not None and len(reqs) >= max_requests):
            break
        n = int(round(math.exp(rng.uniform(math.log(n_lo), math.log(n_hi)))))
        env = _polygon_env(rng, n, density, max_polys)
        steps = int(rng.integers(steps_lo, steps_hi + 1))
        reqs.append(Request(arrival_s=t, scene=_pack("request", [env], steps=steps), steps=steps))
    return reqs


def goal_queue(scene: Scene, n_goals: int, seed: int = 0, hop: float | None = None) -> np.ndarray:
    """Goal queues [N][n_goals][2] for crowd_set_goal_queue: goal 0 is the
    scene's goal; each later goal is drawn uniformly in the environment's
    box of starts and goals (or, with `hop`, within +-hop m of the previous
    goal, clipped to that box), at least r + CLEARANCE from every segment."""
    rng = np.random.Generator(np.random.PCG64(seed))
    q = np.zeros((scene.n_agents, n_goals, 2), np.float32)
    q[:, 0] = scene.goal
    es, ss = scene.env_start, scene.seg_start
    for e in range(scene.n_envs):
        a, b = int(es[e]), int(es[e + 1])
        if a == b:
            continue
        pts = np.concatenate([scene.pos[a:b], scene.goal[a:b]])
        lo, hi = pts.min(0), pts.max(0)
        segs = scene.segments[ss[e]:ss[e + 1]]
        for i in range(a, b):
            for k in range(1, n_goals):
                for _ in range(1000):
                    if hop is None:
                        c = rng.uniform(lo, hi)
                    else:
                        c = np.clip(q[i, k - 1] + rng.uniform(-hop, hop, 2), lo, hi)
                    if len(segs) == 0 or _seg_point_dist(c[0], c[1], segs).min() >= scene.radius[i] + CLEARANCE:
                        break
                q[i, k] = c
    return q


@dataclass
class Vehicles:
    """Lane-following vehicles of a Scene (crowd_set_vehicles): closed lane
    polylines, and per vehicle its agent slot (global index), lane, arc
    position, speed and IDM parameters (v0, T, a, b, s0, length)."""

    lane_start: np.ndarray  # int32 [n_lanes + 1]
    points: np.ndarray      # float32 [P][2]
    agent: np.ndarray       # int32 [V]
    lane: np.ndarray        # int32 [V]
    s: np.ndarray           # float32 [V]
    v: np.ndarray           # float32 [V]
    params: np.ndarray      # float32 [V][6]
    half_width: float = 1.5
    lookahead: float = 25.0


def urban_block_with_vehicles(seed=0, n_envs=16, n_peds=96, n_vehicles=5, steps=300, **kw):
    """Urban blocks with a one-lane ring road 3 m inside the block edge and
    `n_vehicles` cars per block on it (equally spaced, speed U[0, 6] m/s,
    desired speed U[8, 12] m/s, T 1.5 s, a 1.5 m/s^2, b 2 m/s^2, s0 2 m,
    length 4.5 m; the crowd sees each car as an agent of radius 1.2 m).
    Returns (Scene, Vehicles); the cars are the last agents of each env."""
    base = urban_block(seed, n_envs=n_envs, n_peds=n_peds, steps=steps, **kw)
    rng = np.random.Generator(np.random.PCG64(seed + 7919))
    side = float(kw.get("side", 40.0))
    envs, lane_pts, lane_start = [], [], [0]
    agent, lane, s0, v0, params = [], [], [], [], []
    total = 0
    for e in range(base.n_envs):
        a, b = int(base.env_start[e]), int(base.env_start[e + 1])
        m = 3.0
        ring = np.array([(m, m), (side - m, m), (side - m, side - m), (m, side - m)], np.float32)
        lane_pts.append(ring)
        lane_start.append(lane_start[-1] + len(ring))
        L = 4 * (side - 2 * m)
        offs = (np.arange(n_vehicles) + rng.uniform(0, 0.3)) * L / n_vehicles
        pos = []
        for k in range(n_vehicles):
            sk = offs[k] % L
            seg, t = int(sk // (side - 2 * m)), (sk % (side - 2 * m)) / (side - 2 * m)
            pos.append(ring[seg] + t * (ring[(seg + 1) % 4] - ring[seg]))
            agent.append(total + (b - a) + k)
            lane.append(e)
            s0.append(sk)
            v0.append(rng.uniform(0.0, 6.0))
            params.append((rng.uniform(8.0, 12.0), 1.5, 1.5, 2.0, 2.0, 4.5))
        envs.append(dict(radius=np.concatenate([base.radius[a:b], np.full(n_vehicles, 1.2, np.float32)]),
                         max_speed=np.concatenate([base.max_speed[a:b], np.full(n_vehicles, 12.0, np.float32)]),
                         pref_speed=np.concatenate([base.pref_speed[a:b], np.zeros(n_vehicles, np.float32)]),
                         pos=np.concatenate([base.pos[a:b], np.array(pos, np.float32)]),
                         vel=np.concatenate([base.vel[a:b], np.zeros((n_vehicles, 2), np.float32)]),
                         goal=np.concatenate([base.goal[a:b], np.array(pos, np.float32)]),
                         segments=base.segments[base.seg_start[e]:base.seg_start[e + 1]],
                         robot=int(base.robot_index[e])))
        total += (b - a) + n_vehicles
    sc = _pack(base.name + "+vehicles", envs, robot_vel=base.robot_vel, steps=steps)
    veh = Vehicles(lane_start=np.array(lane_start, np.int32), points=np.concatenate(lane_pts).astype(np.float32),
                   agent=np.array(agent, np.int32), lane=np.array(lane, np.int32),
                   s=np.array(s0, np.float32), v=np.array(v0, np.float32), params=np.array(params, np.float32))
    return sc, veh


def make(name: str, seed: int = 0, **kw) -> Scene:
    return {"plain_square": plain_square, "urban_block": urban_block, "uneven_batch": uneven_batch,
            "dense_crowd": dense_crowd}[name](seed=seed, **kw)
