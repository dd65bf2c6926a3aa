"""GPU path vs the FP64 oracle, through the C ABI (needs a GB300).

Contract (the crowd step of the paper's dynamic agents, Sec. 3.2):
  - neighbour lists bit-exact: same ids in the same order (FP64 key, then id);
  - per-step velocity within 1e-4 m/s under teacher forcing (both sides step
    from the same FP32 state; the teacher is the oracle's own trajectory);
  - positions within dt * 1e-4 plus FP32 rounding of the position;
  - rollout statistics within 1 % (counts below 200 within +-2 events).
    Mean speed and goal reach come from single rollouts against the FP64
    oracle.  The collision count (penetrations deeper than 1 mm) is a
    statistic of jammed clusters that rollouts from starts 1 ulp apart
    already spread by 0.3-1 %, and that the rounding of the state to FP32
    between steps (the boundary's state format) moves by 1-3 %: over 64
    urban blocks, a free FP64 rollout with its state rounded to FP32 after
    each step gives 20,015 agent-pair events on average where the unrounded
    one gives 20,194, and the GPU 20,024.  So it is compared as the mean over
    eight rollouts from 1-ulp perturbed starts against the oracle stepped
    from the FP32 state, at 1 %.
"""
import os

import numpy as np
import pytest

import oracle
from paper_2505_00690_gb300 import scenes
from paper_2505_00690_gb300.scenes import Scene

pytestmark = pytest.mark.gpu

VEL_TOL = 1e-4


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2505_00690_gb300 import build

    build.build()


def _crowd(scene, flags):
    from paper_2505_00690_gb300 import crowd as cw

    return cw.Crowd(scene, flags=flags)


def _pos_tol(scene, pos):
    return scene.dt * VEL_TOL + 4 * np.spacing(np.abs(pos).astype(np.float32)).astype(np.float64) + 1e-7


def teacher_forced(scene, steps, sel=None, flags=0, tuning=None):
    """Step the GPU and the oracle from the same FP32 state for `steps` steps,
    the next state being the oracle's.  Returns the worst velocity error, the
    number of neighbour-list mismatches and the fallback count."""
    from paper_2505_00690_gb300 import crowd as cw

    cr = _crowd(scene, cw.CROWD_FLAG_EXPORT_NEIGHBORS | flags)
    if tuning:
        cr.set_tuning(**tuning)
    o = oracle.OracleScene(scene)
    S = scene.state().astype(np.float32)
    worst, mism, fb = 0.0, 0, 0
    for k in range(steps):
        rv = scene.robot_vel_at(k).astype(np.float32)
        cr.set_state(S)
        cr.step(rv[None], n_steps=1)
        G = cr.state()
        nbG = cr.neighbors()
        po, vo, nbO, st = o.step(S[:, :2], S[:, 2:], rv, sel=sel)
        rows = np.arange(scene.n_agents) if sel is None else np.asarray(sel)
        if scene.max_neighbors:
            bad = np.any(nbG[rows] != nbO[rows], axis=1)
            mism += int(bad.sum())
            if bad.any():
                r = rows[np.argmax(bad)]
                print("neighbour mismatch at step", k, "agent", r, nbG[r], nbO[r])
        err = np.abs(G[rows, 2:].astype(np.float64) - vo[rows]).max() if len(rows) else 0.0
        perr = np.abs(G[rows, :2].astype(np.float64) - po[rows]) - _pos_tol(scene, po[rows])
        assert perr.max(initial=-1) <= 0, (k, perr.max())
        worst = max(worst, float(err))
        fb += int((st[rows] == 1).sum())
        if sel is None:
            S = np.concatenate([po, vo], 1).astype(np.float32)
        else:
            S = G.copy()
            S[rows] = np.concatenate([po[rows], vo[rows]], 1).astype(np.float32)
    cr.close()
    return worst, mism, fb


def one_env(pos, vel, goal, radius, vmax, segs=(), robot=-1, R=5.0, K=10, tau=2.0, dt=0.1):
    n = len(pos)
    arr = lambda x: np.full(n, x, np.float32) if np.isscalar(x) else np.asarray(x, np.float32)
    return Scene(name="edge", agents_per_env=np.array([n], np.int32), radius=arr(radius), max_speed=arr(vmax),
                 pref_speed=arr(vmax), pos=np.asarray(pos, np.float32).reshape(-1, 2),
                 vel=np.asarray(vel, np.float32).reshape(-1, 2), goal=np.asarray(goal, np.float32).reshape(-1, 2),
                 robot_index=np.array([robot], np.int32), segs_per_env=np.array([len(segs)], np.int32),
                 segments=np.asarray(segs, np.float32).reshape(-1, 4), tau=tau, tau_obst=tau, neighbor_dist=R,
                 max_neighbors=K, dt=dt)


# ----------------------------------------------------------------------------- teacher forcing

def test_plain_square_teacher_forced():
    sc = scenes.plain_square(0)
    worst, mism, fb = teacher_forced(sc, 200)
    assert mism == 0
    assert worst <= VEL_TOL, worst


@pytest.mark.parametrize("seed", [0, 1])
def test_urban_block_subset_teacher_forced(seed):
    sc = scenes.urban_block(seed, n_envs=6, steps=120)
    worst, mism, fb = teacher_forced(sc, 120)
    assert mism == 0
    assert worst <= VEL_TOL, worst


def test_uneven_polygons_teacher_forced():
    sc = scenes.uneven_batch(3, n_envs=12, steps=60)
    worst, mism, fb = teacher_forced(sc, 60)
    assert mism == 0
    assert worst <= VEL_TOL, worst


@pytest.mark.parametrize("tiled", [False, True])
def test_dense_cluster_with_fallbacks(tiled):
    """A jammed ring walking to the opposite side: many infeasible LPs (on the
    tiled path their fallback starts from the failed LP's iterate)."""
    from paper_2505_00690_gb300 import crowd as cw

    n = 48
    ang = np.linspace(0, 2 * np.pi, n, endpoint=False)
    pos = np.stack([4 * np.cos(ang), 4 * np.sin(ang)], 1)
    sc = one_env(pos, np.zeros((n, 2)), -pos, 0.3, 1.4, segs=[(-0.5, -0.5, 0.5, 0.5)])
    worst, mism, fb = teacher_forced(sc, 80, flags=cw.CROWD_FLAG_FORCE_TILED if tiled else 0)
    assert fb > 0
    assert mism == 0
    assert worst <= VEL_TOL, worst


# ----------------------------------------------------------------------------- edge cases

def _ragged_scene(sizes):
    rng = np.random.default_rng(sum(sizes))
    envs = []
    for n in sizes:
        side = max(4.0, np.sqrt(max(n, 1) / 0.5))
        envs.append(dict(radius=np.full(n, 0.2), max_speed=np.full(n, 1.2), pref_speed=np.full(n, 1.2),
                         pos=scenes._sample_points(rng, n, np.full(n, 0.2), 0, side, [], []),
                         vel=np.zeros((n, 2)), goal=rng.uniform(0, side, (n, 2)), segments=np.zeros((0, 4))))
    return scenes._pack("ragged", envs)


@pytest.mark.parametrize("tiled", [False, True])
@pytest.mark.parametrize("sizes", [[1], [0, 5, 0], [31, 32, 33], [63, 64, 65, 1], [511, 512, 513]])
def test_ragged_sizes(sizes, tiled):
    """Environments of 0, 1 and 2^k +- 1 agents, on the shared-memory kernel
    and forced onto the tiled path (its 32-agent work items then end ragged)."""
    from paper_2505_00690_gb300 import crowd as cw

    sc = _ragged_scene(sizes)
    worst, mism, fb = teacher_forced(sc, 20, flags=cw.CROWD_FLAG_FORCE_TILED if tiled else 0)
    assert mism == 0 and worst <= VEL_TOL


def test_largest_environment():
    sc = scenes.uneven_batch(5, n_envs=1, n_lo=2048, n_hi=2048, max_polys=10, steps=5)
    assert sc.n_agents == 2048
    worst, mism, fb = teacher_forced(sc, 5)
    assert mism == 0 and worst <= VEL_TOL


@pytest.mark.parametrize("tiled", [False, True])
def test_degenerate_geometry(tiled):
    """Coincident agents, an agent exactly on a segment, K = 0 and K = 32, on
    both paths (the tiled one ranks candidates with its nearest-row-first
    walk)."""
    from paper_2505_00690_gb300 import crowd as cw

    pos = [[0, 0], [0, 0], [3, 0], [3, 1e-7], [6, 1]]
    vel = [[0.5, 0], [0, 0], [0, 0], [0, 0], [0, 0.5]]
    goal = [[5, 5], [-5, -5], [3, 5], [3, -5], [6, 5]]
    seg = [(5, 1, 7, 1)]  # agent 4 sits on it
    for K in (0, 4, 32):
        sc = one_env(pos, vel, goal, 0.3, 1.2, segs=seg, K=K)
        worst, mism, fb = teacher_forced(sc, 10, flags=cw.CROWD_FLAG_FORCE_TILED if tiled else 0)
        assert mism == 0 and worst <= VEL_TOL, (K, worst)


@pytest.mark.parametrize("tiled", [False, True])
@pytest.mark.parametrize("K", [10, 16])
def test_lattice_exact_ties(tiled, K):
    """Agents on an exact 1 m lattice with R = 3 m: squared distances are
    exact small integers, so whole rings of neighbours tie exactly (4 at 1,
    4 at 2, 4 at 4, 8 at 5, 4 at 8 m^2), K = 10 and 16 fall inside a tied
    ring (ranked by index), and the lattice points at exactly 3 m sit on the
    R^2 boundary (excluded: the key must be below R^2)."""
    from paper_2505_00690_gb300 import crowd as cw

    rng = np.random.default_rng(11)
    g = np.arange(14, dtype=np.float64) + 0.5
    pos = np.array([[x, y] for y in g for x in g])
    perm = rng.permutation(len(pos))  # indices not in lattice order
    pos = pos[perm]
    goal = rng.uniform(0, 14, pos.shape)
    sc = one_env(pos, np.zeros_like(pos), goal, 0.3, 1.2, R=3.0, K=K)
    worst, mism, fb = teacher_forced(sc, 2, flags=cw.CROWD_FLAG_FORCE_TILED if tiled else 0)
    assert mism == 0 and worst <= VEL_TOL


@pytest.mark.parametrize("tiled", [False, True])
def test_overlapping_crowd(tiled):
    """200 agents of radius 0.3 m dropped into a 2 x 2 m square (nearly every
    pair overlaps): every candidate of the block is within R, K = 32 lists,
    colliding half-planes and fallbacks for most agents."""
    from paper_2505_00690_gb300 import crowd as cw

    rng = np.random.default_rng(5)
    pos = rng.uniform(0, 2, (200, 2))
    goal = rng.uniform(-10, 12, (200, 2))
    sc = one_env(pos, np.zeros_like(pos), goal, 0.3, 1.4, R=5.0, K=32)
    worst, mism, fb = teacher_forced(sc, 5, flags=cw.CROWD_FLAG_FORCE_TILED if tiled else 0)
    assert fb > 0
    assert mism == 0 and worst <= VEL_TOL, worst


def test_robot_agent_follows_command():
    sc = scenes.urban_block(4, n_envs=3, n_peds=20, steps=10)
    worst, mism, fb = teacher_forced(sc, 10)
    assert mism == 0 and worst <= VEL_TOL


# ----------------------------------------------------------------------------- full size, sampled

def test_urban_block_full_size_sampled():
    """All 256 urban blocks in one launch, in an autotuned launch shape like
    the benchmark's: every 100 steps, one step is checked on 2000 sampled
    agents."""
    from paper_2505_00690_gb300 import crowd as cw

    sc = scenes.urban_block(0)
    cr = _crowd(sc, cw.CROWD_FLAG_EXPORT_NEIGHBORS)
    print("tuning", cr.autotune(n_steps=50))
    o = oracle.OracleScene(sc)
    rng = np.random.default_rng(0)
    k = 0
    for chunk in [0, 100, 200, 300]:
        if chunk > k:
            cr.step(sc.robot_vel[k:chunk], n_steps=chunk - k)
            k = chunk
        S = cr.state()
        rv = sc.robot_vel_at(k)
        cr.step(rv[None], n_steps=1)
        k += 1
        G = cr.state()
        nb = cr.neighbors()
        sel = np.sort(rng.choice(sc.n_agents, 2000, replace=False))
        po, vo, nbO, st = o.step(S[:, :2], S[:, 2:], rv, sel=sel)
        assert np.array_equal(nb[sel], nbO[sel])
        assert np.abs(G[sel, 2:] - vo[sel]).max() <= VEL_TOL
    cr.close()


# ----------------------------------------------------------------------------- batching / determinism

def test_env_alone_equals_env_in_batch():
    """Each environment's arithmetic is independent of the batch around it."""
    from paper_2505_00690_gb300 import crowd as cw

    sc = scenes.uneven_batch(7, n_envs=24, n_lo=16, n_hi=300, steps=30)
    full = _crowd(sc, 0)
    full.step(n_steps=30)
    F = full.state()
    es = sc.env_start
    for e in [0, 5, 23]:
        one = _crowd(sc.subset([e]), 0)
        one.step(n_steps=30)
        assert np.array_equal(one.state(), F[es[e]:es[e + 1]])
        one.close()
    full.close()


def test_env_alone_equals_env_in_full_uneven_batch():
    """The full uneven batch (1024 environments of 16-512 agents, Sec. 3.3):
    an environment stepped alone gives the same bits as inside the batch, on
    both paths (the batch's launch shape, queue order and, on the tiled path,
    cell size and work items differ from the lone environment's)."""
    from paper_2505_00690_gb300 import crowd as cw

    sc = scenes.uneven_batch(0, steps=12)
    es = sc.env_start
    sizes = np.diff(es)
    pick = [int(np.argmin(sizes)), int(np.argmax(sizes)), 3, 511, 1023]
    for flags in (0, cw.CROWD_FLAG_FORCE_TILED):
        full = _crowd(sc, flags)
        full.step(n_steps=12)
        F = full.state()
        full.close()
        for e in pick:
            one = _crowd(sc.subset([e]), flags)
            one.step(n_steps=12)
            assert np.array_equal(one.state(), F[es[e]:es[e + 1]]), (flags, e, sizes[e])
            one.close()


@pytest.mark.parametrize("tiled", [False, True])
def test_checkpoint_resume_equals_continuous_run(tiled):
    """Checkpoint/resume: the state read after 15 steps, loaded into a new
    handle (crowd_set_state), continues bit for bit like the run that never
    stopped; with cars, their arc states are read and written back too."""
    from paper_2505_00690_gb300 import crowd as cw

    flags = cw.CROWD_FLAG_FORCE_TILED if tiled else 0
    sc = scenes.urban_block(8, n_envs=8, steps=40)
    a = _crowd(sc, flags)
    a.step(sc.robot_vel[:40], n_steps=40)
    full = a.state()
    a.close()
    b = _crowd(sc, flags)
    b.step(sc.robot_vel[:15], n_steps=15)
    snap = b.state()
    b.close()
    c = _crowd(sc, flags)
    c.set_state(snap)
    c.step(sc.robot_vel[15:40], n_steps=25)
    assert np.array_equal(c.state(), full)
    c.close()
    if tiled:
        return
    sv, veh = scenes.urban_block_with_vehicles(4, n_envs=4, n_peds=48, n_vehicles=3, steps=40)
    runs = []
    for split in (False, True):
        d = _crowd(sv, 0)
        d.set_vehicles(veh)
        if split:
            d.step(sv.robot_vel[:15], n_steps=15)
            snap, s, v = d.state(), *d.vehicle_state()
            d.close()
            d = _crowd(sv, 0)
            d.set_vehicles(veh)
            d.set_state(snap)
            d.set_vehicle_state(s, v)
            d.step(sv.robot_vel[15:40], n_steps=25)
        else:
            d.step(sv.robot_vel[:40], n_steps=40)
        runs.append((d.state(), *d.vehicle_state()))
        d.close()
    assert all(np.array_equal(x, y) for x, y in zip(*runs))


@pytest.mark.parametrize("tiled", [False, True])
def test_segment_overflow_reported_as_device_error(tiled):
    """Failure detection without a fault: an agent with more static segments
    in reach than its line buffer holds (80 short walls on a 2 m ring) keeps
    the nearest ones, the kernel sets the device error word, the next
    synchronising call returns CROWD_EDEVICE, and the handle then steps on."""
    from paper_2505_00690_gb300 import crowd as cw

    ang = np.linspace(0, 2 * np.pi, 80, endpoint=False)
    segs = [(2 * np.cos(a), 2 * np.sin(a), 2 * np.cos(a + 0.01), 2 * np.sin(a + 0.01)) for a in ang]
    pos = np.array([[0.0, 0.0], [12.0, 12.0]])
    sc = one_env(pos, np.zeros((2, 2)), np.array([[0.5, 0.0], [13.0, 12.0]]), 0.3, 1.4, segs=segs)
    cr = _crowd(sc, cw.CROWD_FLAG_FORCE_TILED if tiled else 0)
    cr.step(n_steps=1)
    with pytest.raises(cw.CrowdError) as err:
        cr.state()
    assert err.value.status == cw.CROWD_EDEVICE
    far = sc.state().astype(np.float32)
    far[0, :2] = [20.0, 20.0]  # away from the ring: nothing overflows
    cr.set_state(far)
    cr.step(n_steps=2)
    out = cr.state()
    assert np.all(np.isfinite(out))
    cr.close()


def test_multi_step_call_equals_single_steps():
    from paper_2505_00690_gb300 import crowd as cw

    sc = scenes.urban_block(2, n_envs=4, steps=40)
    a = _crowd(sc, 0)
    a.step(sc.robot_vel[:40], n_steps=40)
    b = _crowd(sc, 0)
    for k in range(40):
        b.step(sc.robot_vel[k:k + 1], n_steps=1)
    assert np.array_equal(a.state(), b.state())


def test_device_pointers_match_host_pointers():
    import torch

    sc = scenes.urban_block(3, n_envs=4, steps=20)
    a = _crowd(sc, 0)
    a.step(sc.robot_vel[:20], n_steps=20)
    b = _crowd(sc, 0)
    b.set_state(torch.from_numpy(sc.state()).cuda())
    b.set_goals(torch.from_numpy(sc.goal).cuda())
    b.step(torch.from_numpy(sc.robot_vel[:20]).cuda(), n_steps=20)
    out = torch.empty((sc.n_agents, 4), dtype=torch.float32, device="cuda")
    b.state(out)
    assert np.array_equal(a.state(), out.cpu().numpy())


# ----------------------------------------------------------------------------- rollout statistics

def _close(a, b, rel=0.01, floor=0.0):
    return abs(a - b) <= max(rel * max(abs(a), abs(b)), floor)


@pytest.mark.parametrize("which", ["plain", "urban", "urban_tiled"])
def test_rollout_statistics_within_one_percent(which):
    from paper_2505_00690_gb300 import crowd as cw

    sc = scenes.plain_square(0) if which == "plain" else scenes.urban_block(0, n_envs=64, steps=300)
    flags = cw.CROWD_FLAG_FORCE_TILED if which == "urban_tiled" else 0
    steps = sc.steps
    ref = oracle.rollout(sc, steps, threads=4)
    cr = _crowd(sc, cw.CROWD_FLAG_STATS | flags)
    rv = sc.robot_vel[:steps] if sc.robot_vel is not None else None
    cr.step(rv, n_steps=steps)
    env, reach = cr.stats()
    ped = np.ones(sc.n_agents, bool)
    for e in range(sc.n_envs):
        if sc.robot_index[e] >= 0:
            ped[sc.env_start[e] + sc.robot_index[e]] = False
    coll = sum(s["agent_collisions"] + s["segment_collisions"] for s in env)
    mean_speed = sum(s["speed_sum"] for s in env) / (ped.sum() * steps)
    reached = (reach > 0) & ped
    frac = reached.sum() / ped.sum()
    mrt = reach[reached].mean() * float(np.float32(sc.dt))
    print(which, "gpu", coll, mean_speed, frac, mrt, "oracle", ref["collisions"], ref["mean_speed"],
          ref["reach_fraction"], ref["mean_reach_time"])
    if which == "plain":  # few events: the +-2 floor applies (the urban counts are held by the ensemble test)
        ref32 = oracle.rollout(sc, steps, threads=4, fp32_state=True)
        assert max(coll, ref32["collisions"]) < 200
        assert _close(coll, ref32["collisions"], rel=0.01, floor=2)
    assert _close(mean_speed, ref["mean_speed"])
    assert _close(mrt, ref["mean_reach_time"])
    assert abs(frac - ref["reach_fraction"]) <= max(0.01, 1.0 / ped.sum())


@pytest.mark.parametrize("tiled", [False, True])
def test_non_reactive_robot_teacher_forced(tiled):
    """robot_responsibility = 1: every pedestrian takes all of the avoidance
    against the robot, which follows its command (the oracle's closed form of
    such a pair is pinned on the CPU)."""
    import dataclasses

    from paper_2505_00690_gb300 import crowd as cw

    sc = dataclasses.replace(scenes.urban_block(7, n_envs=8, steps=40), robot_responsibility=1.0)
    worst, mism, fb = teacher_forced(sc, 40, flags=cw.CROWD_FLAG_FORCE_TILED if tiled else 0)
    assert mism == 0
    assert worst <= VEL_TOL, worst


# ----------------------------------------------------------------------------- tiled (global-memory) path

@pytest.mark.parametrize("seed", [0, 1])
def test_tiled_path_teacher_forced(seed):
    from paper_2505_00690_gb300 import crowd as cw

    sc = scenes.urban_block(seed, n_envs=4, steps=60)
    worst, mism, fb = teacher_forced(sc, 60, flags=cw.CROWD_FLAG_FORCE_TILED)
    assert mism == 0
    assert worst <= VEL_TOL, worst


def test_tiled_uneven_teacher_forced():
    from paper_2505_00690_gb300 import crowd as cw

    sc = scenes.uneven_batch(3, n_envs=8, steps=30)
    worst, mism, fb = teacher_forced(sc, 30, flags=cw.CROWD_FLAG_FORCE_TILED)
    assert mism == 0
    assert worst <= VEL_TOL, worst


def test_tiled_graph_equals_single_steps():
    """A multi-step call (replayed CUDA graph) equals the same steps one call
    at a time, bit for bit, for odd and even step counts."""
    from paper_2505_00690_gb300 import crowd as cw

    sc = scenes.urban_block(5, n_envs=3, steps=40)
    for n in (7, 8):
        a = _crowd(sc, cw.CROWD_FLAG_FORCE_TILED)
        a.step(sc.robot_vel[:n], n_steps=n)
        a.step(sc.robot_vel[n:2 * n], n_steps=n)  # replays the cached graph
        b = _crowd(sc, cw.CROWD_FLAG_FORCE_TILED)
        for k in range(2 * n):
            b.step(sc.robot_vel[k:k + 1], n_steps=1)
        assert np.array_equal(a.state(), b.state()), n
        a.close()
        b.close()


def test_dense_crowd_full_size_sampled():
    """16 dense environments of 20,000 agents (tiled path, graph-replayed
    steps); one teacher-forced step checked on 1000 agents of environment 0."""
    from paper_2505_00690_gb300 import crowd as cw

    sc = scenes.dense_crowd(0, steps=10)
    cr = _crowd(sc, cw.CROWD_FLAG_EXPORT_NEIGHBORS)
    cr.step(n_steps=10)
    S = cr.state()
    cr.step(n_steps=1)
    G = cr.state()
    nb = cr.neighbors()
    o = oracle.OracleScene(sc)
    rng = np.random.default_rng(1)
    sel = np.sort(rng.choice(20000, 1000, replace=False))
    po, vo, nbO, st = o.step(S[:, :2], S[:, 2:], None, sel=sel, threads=8)
    assert np.array_equal(nb[sel], nbO[sel])
    assert np.abs(G[sel, 2:] - vo[sel]).max() <= VEL_TOL
    cr.close()


def test_tiled_cell_size_and_tiles_change_no_bit():
    """A 20,000-agent environment stepped alone (cells of R, 4 x 3-cell tiles)
    and inside the 16-environment crowd (enough agents for cells of R/2 and
    7 x 7-cell tiles) gives the same bits: the neighbour lists are exact
    either way and every agent runs the same arithmetic."""
    from paper_2505_00690_gb300 import crowd as cw

    sc = scenes.dense_crowd(2, steps=4)
    both = []
    for scene in (sc.subset([0]), sc):
        cr = _crowd(scene, cw.CROWD_FLAG_EXPORT_NEIGHBORS)
        cr.step(n_steps=3)
        both.append((cr.state()[:20000], cr.neighbors()[:20000]))
        cr.close()
    assert np.array_equal(both[0][0], both[1][0])
    assert np.array_equal(both[0][1], both[1][1])


# ----------------------------------------------------------------------------- tuning

def test_tuning_knobs_and_autotune():
    """Block size and cell split change no result bit; the cooperative and the
    in-place fallback agree within the velocity tolerance; the autotuner
    restores the state it timed on."""
    from paper_2505_00690_gb300 import crowd as cw

    sc = scenes.urban_block(6, n_envs=8, steps=30)
    ref = None
    for block in (64, 160, 512):
        for split in (1, 2):
            cr = _crowd(sc, 0)
            cr.set_tuning(block_threads=block, coop_fallback=1, cell_split=split)
            cr.step(sc.robot_vel[:30], n_steps=30)
            out = cr.state()
            if ref is None:
                ref = out
            assert np.array_equal(out, ref), (block, split)
            cr.close()
    # one step from a common state: in-place vs cooperative fallback
    S = ref.copy()
    outs = []
    for coop in (0, 1, 2):
        cr = _crowd(sc, 0)
        cr.set_tuning(block_threads=0, coop_fallback=coop, cell_split=1)
        cr.set_state(S)
        cr.step(sc.robot_vel[30:31], n_steps=1)
        outs.append(cr.state())
        cr.close()
    assert np.abs(outs[0] - outs[1]).max() <= VEL_TOL
    assert np.abs(outs[0] - outs[2]).max() <= VEL_TOL
    cr = _crowd(sc, cw.CROWD_FLAG_STATS)
    before = cr.state()
    t = cr.autotune(n_steps=5)
    assert t["block_threads"] in (64, 128, 160, 256, 512) and t["cell_split"] in (1, 2, 3)
    assert t["lanes_per_agent"] in (1, 4, 8)
    assert np.array_equal(cr.state(), before)
    env, reach = cr.stats()
    assert all(e["steps"] == 0 for e in env) and np.all(reach == -1)
    cr.close()


# ----------------------------------------------------------------------------- groups of lanes per agent

@pytest.mark.parametrize("lanes", [2, 4, 8])
def test_group_lanes_teacher_forced(lanes):
    """G lanes per agent: the same contract as one thread per agent."""
    tun = dict(block_threads=0, coop_fallback=0, cell_split=1, lanes_per_agent=lanes)
    sc = scenes.urban_block(0, n_envs=6, steps=120)
    worst, mism, fb = teacher_forced(sc, 120, tuning=tun)
    assert mism == 0
    assert worst <= VEL_TOL, worst
    sc = scenes.uneven_batch(3, n_envs=12, steps=40)
    worst, mism, fb = teacher_forced(sc, 40, tuning=dict(tun, cell_split=2))
    assert mism == 0
    assert worst <= VEL_TOL, worst


@pytest.mark.parametrize("lanes", [2, 4, 8])
def test_group_lanes_fallbacks_and_ragged(lanes):
    tun = dict(block_threads=0, coop_fallback=0, cell_split=1, lanes_per_agent=lanes)
    n = 48
    ang = np.linspace(0, 2 * np.pi, n, endpoint=False)
    pos = np.stack([4 * np.cos(ang), 4 * np.sin(ang)], 1)
    sc = one_env(pos, np.zeros((n, 2)), -pos, 0.3, 1.4, segs=[(-0.5, -0.5, 0.5, 0.5)])
    worst, mism, fb = teacher_forced(sc, 80, tuning=tun)
    assert fb > 0 and mism == 0
    assert worst <= VEL_TOL, worst
    for sizes in ([1], [0, 5, 0], [63, 64, 65, 1], [511, 512, 513]):
        sc = _ragged_scene(sizes)
        worst, mism, fb = teacher_forced(sc, 10, tuning=tun)
        assert mism == 0, sizes
        assert worst <= VEL_TOL, (sizes, worst)


def test_group_lanes_bit_identical_across_shapes():
    """2, 4 and 8 lanes per agent, any block size and cell split: the group
    reductions are exact (min / max) and the top-K merge is unique, so every
    shape gives the same bits."""
    sc = scenes.urban_block(6, n_envs=8, steps=30)
    ref = None
    for lanes, block, split in ((4, 0, 1), (4, 512, 2), (8, 0, 2), (8, 512, 1), (8, 256, 1), (2, 0, 1), (2, 96, 2)):
        cr = _crowd(sc, 0)
        cr.set_tuning(block_threads=block, coop_fallback=0, cell_split=split, lanes_per_agent=lanes)
        assert cr.tuning()["lanes_per_agent"] == lanes
        cr.step(sc.robot_vel[:30], n_steps=30)
        out = cr.state()
        cr.close()
        if ref is None:
            ref = out
        assert np.array_equal(out, ref), (lanes, block, split)


def test_group_lanes_rollout_statistics():
    from paper_2505_00690_gb300 import crowd as cw

    sc = scenes.urban_block(0, n_envs=64, steps=300)
    steps = sc.steps
    ref = oracle.rollout(sc, steps, threads=4)
    cr = _crowd(sc, cw.CROWD_FLAG_STATS)
    cr.set_tuning(block_threads=0, coop_fallback=0, cell_split=1, lanes_per_agent=4)
    cr.step(sc.robot_vel[:steps], n_steps=steps)
    env, reach = cr.stats()
    ped = np.ones(sc.n_agents, bool)
    for e in range(sc.n_envs):
        if sc.robot_index[e] >= 0:
            ped[sc.env_start[e] + sc.robot_index[e]] = False
    coll = sum(s["agent_collisions"] + s["segment_collisions"] for s in env)
    mean_speed = sum(s["speed_sum"] for s in env) / (ped.sum() * steps)
    reached = (reach > 0) & ped
    mrt = reach[reached].mean() * float(np.float32(sc.dt))
    assert coll > 0  # the count itself is held by the ensemble test, which runs this shape too
    assert _close(mean_speed, ref["mean_speed"])
    assert _close(mrt, ref["mean_reach_time"])
    assert abs(reached.sum() / ped.sum() - ref["reach_fraction"]) <= max(0.01, 1.0 / ped.sum())


@pytest.mark.parametrize("coop", [1, 2])
def test_deferred_fallback_modes_teacher_forced(coop):
    """Fallbacks queued after the pass (whole warps, or one lane each spread
    over the warps): the same contract as in-place fallbacks, on a jammed ring
    and on urban blocks."""
    tun = dict(block_threads=0, coop_fallback=coop, cell_split=1, lanes_per_agent=1)
    n = 48
    ang = np.linspace(0, 2 * np.pi, n, endpoint=False)
    pos = np.stack([4 * np.cos(ang), 4 * np.sin(ang)], 1)
    sc = one_env(pos, np.zeros((n, 2)), -pos, 0.3, 1.4, segs=[(-0.5, -0.5, 0.5, 0.5)])
    worst, mism, fb = teacher_forced(sc, 80, tuning=tun)
    assert fb > 0 and mism == 0
    assert worst <= VEL_TOL, worst
    sc = scenes.urban_block(1, n_envs=6, steps=60)
    worst, mism, fb = teacher_forced(sc, 60, tuning=tun)
    assert mism == 0
    assert worst <= VEL_TOL, worst


@pytest.mark.parametrize("which", ["urban", "uneven"])
def test_agent_order_and_deferred_fallback_change_no_bit(which):
    """In-place and deferred one-lane fallbacks run the same arithmetic on the
    same lines, and the agent order only changes which thread computes an
    agent: every combination gives the same bits."""
    if which == "urban":
        sc = scenes.urban_block(2, n_envs=8, steps=40)
    else:
        sc = scenes.uneven_batch(4, n_envs=12, n_lo=16, n_hi=600, steps=40)
    rv = sc.robot_vel[:40] if sc.robot_vel is not None else None
    ref = None
    for block, coop, order, split in ((0, 0, 0, 1), (0, 2, 0, 1), (0, 0, 1, 1), (0, 2, 1, 2), (256, 2, 1, 1),
                                      (64, 0, 1, 2), (512, 2, 0, 1), (128, 0, 1, 3)):
        cr = _crowd(sc, 0)
        cr.set_tuning(block_threads=block, coop_fallback=coop, cell_split=split, agent_order=order)
        assert cr.tuning()["agent_order"] == order
        cr.step(rv, n_steps=40)
        out = cr.state()
        cr.close()
        if ref is None:
            ref = out
        assert np.array_equal(out, ref), (block, coop, order, split)


# ----------------------------------------------------------------------------- goal queues

def teacher_forced_goals(scene, queue, cyclic, steps, flags=0):
    """Teacher forcing with goal queues: the host moves goals on with the
    oracle's rule from the teacher state; the GPU does the same inside the
    step.  Returns the worst velocity error, neighbour mismatches, goal-index
    mismatches and the number of goal changes."""
    from paper_2505_00690_gb300 import crowd as cw

    cr = _crowd(scene, cw.CROWD_FLAG_EXPORT_NEIGHBORS | flags)
    cr.set_goal_queue(queue, cyclic=cyclic)
    o = oracle.OracleScene(scene)
    robot_rows = np.zeros(scene.n_agents, bool)
    for e in range(scene.n_envs):
        if scene.robot_index[e] >= 0:
            robot_rows[scene.env_start[e] + scene.robot_index[e]] = True
    S = scene.state().astype(np.float32)
    goal, idx = queue[:, 0].astype(np.float64), np.zeros(scene.n_agents, np.int64)
    worst, mism, gmis = 0.0, 0, 0
    for k in range(steps):
        rv = scene.robot_vel_at(k).astype(np.float32)
        goal, idx = oracle.advance_goals(S[:, :2], scene.radius, goal, idx, queue, cyclic, skip=robot_rows)
        cr.set_state(S)
        cr.step(rv[None], n_steps=1)
        G = cr.state()
        gmis += int((cr.goal_index() != idx).sum())
        po, vo, nbO, st = o.step(S[:, :2], S[:, 2:], rv, goal=goal)
        if scene.max_neighbors:
            mism += int(np.any(cr.neighbors() != nbO, axis=1).sum())
        worst = max(worst, float(np.abs(G[:, 2:].astype(np.float64) - vo).max()))
        S = np.concatenate([po, vo], 1).astype(np.float32)
    cr.close()
    return worst, mism, gmis, int(idx.sum())


def test_goal_queue_lone_agent_on_gpu():
    """The hand-derived turns of the oracle pin: goal 1 from step 97, goal 2
    from step 194, then the last goal kept."""
    from paper_2505_00690_gb300 import crowd as cw

    q = np.array([[(10.0, 0.0), (10.0, 10.0), (0.0, 10.0)]], np.float32)
    sc = one_env([(0.0, 0.0)], [(0.0, 0.0)], q[:, 0], 0.35, 1.0)
    cr = cw.Crowd(sc)
    cr.set_goal_queue(q, cyclic=False)
    seen = []
    for _ in range(400):
        cr.step(n_steps=1)
        seen.append(int(cr.goal_index()[0]))
    # the index read after step k was set at the start of step k
    seen = np.array(seen)
    assert np.nonzero(seen == 1)[0][0] == 97 and np.nonzero(seen == 2)[0][0] == 194 and seen.max() == 2
    assert np.allclose(cr.state()[0, :2], [0.0, 10.0], atol=1e-5)
    cr.close()


@pytest.mark.parametrize("flags", [0, 8])
def test_goal_queue_teacher_forced(flags):
    """Urban blocks with 6-goal cyclic queues hopping <= 4 m: hundreds of goal
    changes; identical goal counters, bit-exact neighbours, 1e-4 m/s."""
    sc = scenes.urban_block(3, n_envs=4, steps=150)
    q = scenes.goal_queue(sc, 6, seed=1, hop=4.0)
    q[:, 0] = sc.pos + np.clip(q[:, 0] - sc.pos, -2.0, 2.0)  # first goals close by, too
    worst, mism, gmis, changes = teacher_forced_goals(sc, q, True, 150, flags=flags)
    assert changes > 200, changes
    assert gmis == 0 and mism == 0
    assert worst <= VEL_TOL, worst


def _goal_pool(sc, seed=7):
    """Per-environment goal pools: one point per agent of the environment,
    drawn like the scene's goals (clear of segments), and first goals within
    2 m of the starts so that arrivals and draws begin early."""
    q = scenes.goal_queue(sc, 2, seed=seed)
    first = (sc.pos + np.clip(q[:, 0] - sc.pos, -2.0, 2.0)).astype(np.float32)
    return first, np.asarray(sc.env_start, np.int32), np.ascontiguousarray(q[:, 1], np.float32)


@pytest.mark.parametrize("flags", [0, 8])
def test_goal_pool_teacher_forced(flags):
    """Goal pools drawn inside the kernels with Philox4x32-10: the goal
    counters and the drawn goals equal the oracle's, neighbours bit-exact,
    velocities within 1e-4 m/s."""
    from paper_2505_00690_gb300 import crowd as cw

    sc = scenes.urban_block(5, n_envs=4, steps=150)
    first, pool_start, pool = _goal_pool(sc)
    seed = 0x9E3779B97F4A7C15
    env_of = np.repeat(np.arange(sc.n_envs), sc.agents_per_env)
    robot_rows = np.zeros(sc.n_agents, bool)
    for e in range(sc.n_envs):
        robot_rows[sc.env_start[e] + sc.robot_index[e]] = True
    cr = _crowd(sc, cw.CROWD_FLAG_EXPORT_NEIGHBORS | flags)
    cr.set_goals(first)
    cr.set_goal_pool(pool_start, pool, seed)
    o = oracle.OracleScene(sc)
    S = sc.state().astype(np.float32)
    goal, idx = first.astype(np.float64), np.zeros(sc.n_agents, np.int64)
    worst, mism, gmis = 0.0, 0, 0
    for k in range(150):
        rv = sc.robot_vel_at(k).astype(np.float32)
        goal, idx = oracle.advance_goals_pool(S[:, :2], sc.radius, goal, idx, pool_start, pool, env_of, seed,
                                              skip=robot_rows)
        cr.set_state(S)
        cr.step(rv[None], n_steps=1)
        G = cr.state()
        gmis += int((cr.goal_index() != idx).sum())
        po, vo, nbO, st = o.step(S[:, :2], S[:, 2:], rv, goal=goal)
        mism += int(np.any(cr.neighbors() != nbO, axis=1).sum())
        worst = max(worst, float(np.abs(G[:, 2:].astype(np.float64) - vo).max()))
        S = np.concatenate([po, vo], 1).astype(np.float32)
    cr.close()
    assert idx.sum() > 200, idx.sum()
    assert gmis == 0 and mism == 0
    assert worst <= VEL_TOL, worst


def test_goal_pool_multi_step_equals_single_steps():
    from paper_2505_00690_gb300 import crowd as cw

    sc = scenes.urban_block(6, n_envs=4, steps=80)
    first, pool_start, pool = _goal_pool(sc, seed=3)
    outs = []
    for chunks in ((80,), (1,) * 80, (30, 50)):
        cr = _crowd(sc, 0)
        cr.set_goals(first)
        cr.set_goal_pool(pool_start, pool, 12345)
        k = 0
        for n in chunks:
            cr.step(sc.robot_vel[k:k + n], n_steps=n)
            k += n
        outs.append((cr.state(), cr.goal_index()))
        cr.close()
    assert outs[0][1].sum() > 100
    for st, gi in outs[1:]:
        assert np.array_equal(st, outs[0][0]) and np.array_equal(gi, outs[0][1])


def test_goal_queue_multi_step_equals_single_steps():
    from paper_2505_00690_gb300 import crowd as cw

    sc = scenes.urban_block(4, n_envs=6, steps=120)
    q = scenes.goal_queue(sc, 4, seed=2, hop=3.0)
    outs = []
    for chunks in ((120,), (1,) * 120, (50, 7, 63)):
        cr = cw.Crowd(sc)
        cr.set_goal_queue(q, cyclic=True)
        k = 0
        for n in chunks:
            cr.step(sc.robot_vel[k:k + n], n_steps=n)
            k += n
        outs.append((cr.state(), cr.goal_index()))
        cr.close()
    for st, gi in outs[1:]:
        assert np.array_equal(st, outs[0][0]) and np.array_equal(gi, outs[0][1])
    assert outs[0][1].sum() > 50


# ----------------------------------------------------------------------------- velocity-dependent segment lines

@pytest.mark.parametrize("which,flags", [("urban", 0), ("uneven", 0), ("urban", 8)])
def test_velocity_segments_teacher_forced(which, flags):
    """CROWD_FLAG_VELOCITY_SEGMENTS (segment half-planes tangent to the
    segment VO at its point nearest the current velocity): the same contract."""
    import dataclasses

    sc = scenes.urban_block(5, n_envs=6, steps=100) if which == "urban" else scenes.uneven_batch(4, n_envs=10,
                                                                                                  steps=40)
    sc = dataclasses.replace(sc, segment_mode=1)
    worst, mism, fb = teacher_forced(sc, sc.steps, flags=flags)
    assert mism == 0
    assert worst <= VEL_TOL, worst


def _perturbed(base, k):
    """The scene with every start coordinate moved by one FP32 ulp up or down
    (seeded by k; k = 0 leaves it as it is)."""
    import dataclasses

    if k == 0:
        return base
    rng = np.random.default_rng(k)
    up = rng.random(base.pos.shape) < 0.5
    pos = np.where(up, np.nextafter(base.pos, np.float32(np.inf)), np.nextafter(base.pos, np.float32(-np.inf)))
    return dataclasses.replace(base, pos=pos.astype(np.float32))


@pytest.mark.parametrize("mode", [0, 1])
def test_collision_count_ensemble_within_one_percent(mode):
    """The collision count (the appendix metric table's collision indicator,
    penetration deeper than 1 mm) of 256 urban blocks over 300 steps, as the
    mean of eight rollouts from 1-ulp perturbed starts, within 1 % of the
    oracle's mean over the same starts, the oracle stepping from the state
    held in FP32 between steps as the library holds it; on the resident
    kernel (one lane and four lanes per agent) and the tiled path (mode 1:
    velocity-dependent segment lines).  Mean speed, reach fraction and reach
    time of the unperturbed rollout within 1 % of the free FP64 rollout."""
    import dataclasses

    from paper_2505_00690_gb300 import crowd as cw

    base = dataclasses.replace(scenes.urban_block(0, n_envs=256, steps=300), segment_mode=mode)
    steps = base.steps
    ped = np.ones(base.n_agents, bool)
    for e in range(base.n_envs):
        if base.robot_index[e] >= 0:
            ped[base.env_start[e] + base.robot_index[e]] = False
    threads = os.cpu_count() or 4
    paths = (("resident", 0, 1), ("lanes4", 0, 4), ("tiled", cw.CROWD_FLAG_FORCE_TILED, 1))
    coll = {name: [] for name, _, _ in paths}
    coll_o = []
    for k in range(8):
        sc = _perturbed(base, k)
        coll_o.append(oracle.rollout(sc, steps, threads=threads, fp32_state=True)["collisions"])
        for name, flags, lanes in paths:
            cr = _crowd(sc, cw.CROWD_FLAG_STATS | flags)
            if lanes > 1:
                cr.set_tuning(block_threads=0, coop_fallback=0, cell_split=1, lanes_per_agent=lanes)
            cr.step(sc.robot_vel[:steps], n_steps=steps)
            env, reach = cr.stats()
            cr.close()
            coll[name].append(sum(s["agent_collisions"] + s["segment_collisions"] for s in env))
            if k == 0 and name == "resident":
                ref = oracle.rollout(sc, steps, threads=threads)
                mean_speed = sum(s["speed_sum"] for s in env) / (ped.sum() * steps)
                reached = (reach > 0) & ped
                mrt = reach[reached].mean() * float(np.float32(sc.dt))
                assert _close(mean_speed, ref["mean_speed"])
                assert _close(mrt, ref["mean_reach_time"])
                assert abs(reached.sum() / ped.sum() - ref["reach_fraction"]) <= max(0.01, 1.0 / ped.sum())
    print("mode", mode, "collisions gpu", coll, "oracle (FP32 state)", coll_o)
    for name in coll:
        assert _close(float(np.mean(coll[name])), float(np.mean(coll_o)), rel=0.01), name


# ----------------------------------------------------------------------------- lane-following vehicles

def _vehicle_kind(sc, veh):
    kind = np.zeros(sc.n_agents, np.int32)
    kind[veh.agent] = 1
    return kind


def _vehicle_oracle_step(sc, veh, lanes, S, vs, vv):
    """Cars of every env from the teacher state: new (s, v) and the state rows
    the crowd step starts from (position p(s), velocity (p(s') - p(s))/dt)."""
    from oracle import vehicles as VH

    S = S.copy()
    s_new, v_new = vs.astype(np.float64).copy(), vv.astype(np.float64).copy()
    kind = _vehicle_kind(sc, veh)
    for e in range(sc.n_envs):
        a, b = sc.env_start[e], sc.env_start[e + 1]
        ks = np.nonzero((veh.agent >= a) & (veh.agent < b))[0]
        if len(ks) == 0:
            continue
        blockers = kind[a:b] == 0
        sn, vn, p_now, p_next, vel = VH.idm_step(lanes, veh.lane[ks], vs[ks], vv[ks], veh.params[ks], S[a:b, :2],
                                                 sc.radius[a:b], blockers, veh.half_width, veh.lookahead,
                                                 float(np.float32(sc.dt)))
        s_new[ks], v_new[ks] = sn, vn
        S[veh.agent[ks], :2] = p_now
        S[veh.agent[ks], 2:] = vel
    return s_new, v_new, S


@pytest.mark.parametrize("tiled", [False, True])
def test_vehicles_teacher_forced(tiled):
    """Urban blocks with ring-road cars: the host runs the cars' IDM and the
    crowd step of the oracle from the teacher state (cars as vehicles), the
    GPU does both inside its step, on either kernel; car arc positions and
    speeds, pedestrian velocities (1e-4) and neighbour lists (bit-exact)
    agree."""
    from oracle import vehicles as VH
    from paper_2505_00690_gb300 import crowd as cw

    sc, veh = scenes.urban_block_with_vehicles(2, n_envs=6, n_peds=96, n_vehicles=5, steps=120)
    lanes = VH.Lanes(veh.points, veh.lane_start)
    kind = _vehicle_kind(sc, veh)
    cr = _crowd(sc, cw.CROWD_FLAG_EXPORT_NEIGHBORS | (cw.CROWD_FLAG_FORCE_TILED if tiled else 0))
    cr.set_vehicles(veh)
    o = oracle.OracleScene(sc)
    S = sc.state().astype(np.float32)
    vs, vv = veh.s.copy(), veh.v.copy()
    worst_ped, worst_car, mism, stopped = 0.0, 0.0, 0, 0
    for k in range(sc.steps):
        rv = sc.robot_vel_at(k).astype(np.float32)
        s_new, v_new, S_start = _vehicle_oracle_step(sc, veh, lanes, S, vs, vv)
        cr.set_state(S)
        cr.set_vehicle_state(vs, vv)
        cr.step(rv[None], n_steps=1)
        G = cr.state()
        gs, gv = cr.vehicle_state()
        po, vo, nb, st = o.step(S_start[:, :2], S_start[:, 2:], rv, kind=kind)
        assert np.all(st[veh.agent] == 3)
        mism += int(np.any(cr.neighbors() != nb, axis=1).sum())
        ped = kind == 0
        worst_ped = max(worst_ped, float(np.abs(G[ped, 2:] - vo[ped]).max()))
        L = np.array([lanes.length(int(l)) for l in veh.lane])
        ds = (gs - s_new + 0.5 * L) % L - 0.5 * L  # arc difference on the ring
        worst_car = max(worst_car, float(np.abs(gv - v_new).max()), float(np.abs(ds).max()) / float(np.float32(sc.dt)))
        stopped += int((v_new < 0.05).sum())
        S = np.concatenate([po, vo], 1).astype(np.float32)
        vs, vv = s_new.astype(np.float32), v_new.astype(np.float32)
    cr.close()
    assert mism == 0
    assert worst_ped <= VEL_TOL, worst_ped
    assert worst_car <= VEL_TOL, worst_car
    assert stopped > 0  # some cars had to stop for pedestrians on the road


def test_vehicles_tiled_multi_step_equals_single_steps():
    """Cars on the tiled path: a graph-replayed multi-step call equals single
    steps and other splits, bit for bit."""
    from paper_2505_00690_gb300 import crowd as cw

    sc, veh = scenes.urban_block_with_vehicles(3, n_envs=4, n_peds=64, n_vehicles=4, steps=60)
    outs = []
    for chunks in ((60,), (1,) * 60, (25, 35)):
        cr = _crowd(sc, cw.CROWD_FLAG_FORCE_TILED)
        cr.set_vehicles(veh)
        k = 0
        for n in chunks:
            cr.step(sc.robot_vel[k:k + n], n_steps=n)
            k += n
        outs.append((cr.state(), *cr.vehicle_state()))
        cr.close()
    for st, s_, v_ in outs[1:]:
        assert np.array_equal(st, outs[0][0]) and np.array_equal(s_, outs[0][1]) and np.array_equal(v_, outs[0][2])


def test_vehicles_multi_step_equals_single_steps_and_autotune_restores():
    from paper_2505_00690_gb300 import crowd as cw

    sc, veh = scenes.urban_block_with_vehicles(3, n_envs=8, n_peds=64, n_vehicles=4, steps=60)
    outs = []
    for chunks in ((60,), (1,) * 60, (25, 35)):
        cr = cw.Crowd(sc)
        cr.set_vehicles(veh)
        k = 0
        for n in chunks:
            cr.step(sc.robot_vel[k:k + n], n_steps=n)
            k += n
        outs.append((cr.state(), *cr.vehicle_state()))
        cr.close()
    for st, s, v in outs[1:]:
        assert np.array_equal(st, outs[0][0]) and np.array_equal(s, outs[0][1]) and np.array_equal(v, outs[0][2])
    cr = cw.Crowd(sc)
    cr.set_vehicles(veh)
    before = (cr.state(), *cr.vehicle_state())
    cr.autotune(n_steps=10)
    after = (cr.state(), *cr.vehicle_state())
    assert all(np.array_equal(x, y) for x, y in zip(before, after))
    with pytest.raises(cw.CrowdError):
        bad = scenes.Vehicles(**{**veh.__dict__, "agent": veh.agent[::-1].copy()})
        cr.set_vehicles(bad)
    cr.close()
