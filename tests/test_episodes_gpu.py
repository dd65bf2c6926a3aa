"""Episodes on the GPU (crowd_set_episodes; the oracle's rule is
episode_restarts / restart_rows, Sec. 3.3), on both kernels: the
shared-memory-resident one and the tiled one (forced with
CROWD_FLAG_FORCE_TILED).

  - a multi-step call equals the same steps taken one call at a time, bit for
    bit, and an environment's states repeat episode after episode when the
    robot's commands do;
  - teacher forcing across episode starts, with goal queues: neighbour lists
    bit-exact, velocities within 1e-4 m/s, goal counters equal to the
    oracle's;
  - statistics count every post-integration state once (an episode's last
    state included, the restored start not), however the steps are split
    into calls, also when the restored start holds overlapping agents;
  - crowd_set_goals removes the episodes; crowd_reset_stats keeps the clock;
  - cars start over with their environment (arc positions and speeds).
"""
import numpy as np
import pytest

import oracle
from paper_2505_00690_gb300 import scenes

pytestmark = pytest.mark.gpu

VEL_TOL = 1e-4
PATHS = ["resident", "tiled"]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2505_00690_gb300 import build

    build.build()


def _flags(path, extra=0):
    from paper_2505_00690_gb300 import crowd as cw

    return extra | (cw.CROWD_FLAG_FORCE_TILED if path == "tiled" else 0)


def _periodic_commands(sc, steps, T):
    """Robot commands [T][E][2] that repeat with each environment's episode."""
    base = np.stack([sc.robot_vel_at(t) for t in range(T)]).astype(np.float32)
    rv = base.copy()
    for e, L in enumerate(steps):
        if L:
            rv[:, e] = base[np.arange(T) % L, e]
    return rv


def _owner(sc):
    return np.repeat(np.arange(sc.n_envs), sc.agents_per_env)


@pytest.mark.parametrize("path", PATHS)
def test_episodes_multistep_equals_single_steps_and_repeat(path):
    from paper_2505_00690_gb300 import crowd as cw

    sc = scenes.urban_block(3, n_envs=6, n_peds=40, steps=40)
    steps = np.array([5, 0, 8, 3, 13, 1], np.int32)
    T = 27
    rv = _periodic_commands(sc, steps, T)
    a = cw.Crowd(sc, flags=_flags(path))
    a.set_episodes(steps)
    states = [a.state()]
    for t in range(T):
        a.step(rv[t:t + 1], n_steps=1)
        states.append(a.state())
    a.close()
    b = cw.Crowd(sc, flags=_flags(path))
    b.set_episodes(steps)
    b.step(rv, n_steps=T)
    assert np.array_equal(b.state(), states[T])
    b.close()
    plain = cw.Crowd(sc, flags=_flags(path))
    ref = [plain.state()]
    for t in range(T):
        plain.step(rv[t:t + 1], n_steps=1)
        ref.append(plain.state())
    plain.close()
    es = sc.env_start
    for e, L in enumerate(steps):
        rows = slice(es[e], es[e + 1])
        if L == 0:
            assert all(np.array_equal(states[t][rows], ref[t][rows]) for t in range(T + 1))
            continue
        for t in range(min(L, T) + 1):  # before the first start the run is the plain one
            assert np.array_equal(states[t][rows], ref[t][rows]), (e, t)
        if L > 1:
            assert not np.array_equal(states[L][rows], states[0][rows])
        for t in range(L + 1, T + 1):
            j = (t - 1) % L + 1
            assert np.array_equal(states[t][rows], states[j][rows]), (e, t, j)


@pytest.mark.parametrize("path", PATHS)
def test_episodes_teacher_forced_with_goal_queues(path):
    from paper_2505_00690_gb300 import crowd as cw

    sc = scenes.urban_block(4, n_envs=4, n_peds=48, steps=40)
    steps = np.array([4, 7, 0, 1], np.int32)
    T = 22
    queue = scenes.goal_queue(sc, 4, seed=2, hop=3.0)
    robot_rows = np.zeros(sc.n_agents, bool)
    for e in range(sc.n_envs):
        if sc.robot_index[e] >= 0:
            robot_rows[sc.env_start[e] + sc.robot_index[e]] = True
    owner = _owner(sc)
    cr = cw.Crowd(sc, flags=_flags(path, cw.CROWD_FLAG_EXPORT_NEIGHBORS))
    cr.set_goal_queue(queue, cyclic=True)
    cr.set_episodes(steps)
    o = oracle.OracleScene(sc)
    S0 = sc.state().astype(np.float32)
    goal0, idx0 = queue[:, 0].astype(np.float64), np.zeros(sc.n_agents, np.int64)
    S, goal, idx = S0.copy(), goal0.copy(), idx0.copy()
    worst, mism, gmis, starts, moved = 0.0, 0, 0, 0, 0
    for t in range(T):
        rv = sc.robot_vel_at(t).astype(np.float32)
        starts += int(oracle.episode_restarts(t, steps).sum())
        Sr = oracle.restart_rows(t, steps, owner, S, S0)
        goal = oracle.restart_rows(t, steps, owner, goal, goal0)
        idx = oracle.restart_rows(t, steps, owner, idx, idx0)
        before = idx.copy()
        goal, idx = oracle.advance_goals(Sr[:, :2], sc.radius, goal, idx, queue, True, skip=robot_rows)
        moved += int((idx != before).sum())
        cr.set_state(S)  # the episode's state: the GPU starts over by itself
        cr.step(rv[None], n_steps=1)
        G = cr.state()
        gmis += int((cr.goal_index() != idx).sum())
        po, vo, nbO, st = o.step(Sr[:, :2], Sr[:, 2:], rv, goal=goal)
        mism += int(np.any(cr.neighbors() != nbO, axis=1).sum())
        worst = max(worst, float(np.abs(G[:, 2:].astype(np.float64) - vo).max()))
        S = np.concatenate([po, vo], 1).astype(np.float32)
    cr.close()
    assert starts >= 20 and moved > 0
    assert mism == 0 and gmis == 0
    assert worst <= VEL_TOL, worst


def _overlapping_start(sc):
    """The scene's start with agent 1 of every environment placed 0.1 m from
    agent 0 (deep overlap: counted as a collision in the start state)."""
    S = sc.state().astype(np.float32)
    for e in range(sc.n_envs):
        a = int(sc.env_start[e])
        S[a + 1, :2] = S[a, :2] + np.float32([0.1, 0.0])
        S[a + 1, 2:] = 0
    return S


@pytest.mark.parametrize("path", PATHS)
def test_episode_statistics_count_every_step_once(path):
    from paper_2505_00690_gb300 import crowd as cw

    sc = scenes.urban_block(5, n_envs=4, n_peds=48, steps=40)
    steps = np.array([3, 5, 0, 2], np.int32)
    T = 16
    rv = np.stack([sc.robot_vel_at(t) for t in range(T)]).astype(np.float32)
    start = _overlapping_start(sc)
    runs = []
    for split in (False, True):
        cr = cw.Crowd(sc, flags=_flags(path, cw.CROWD_FLAG_STATS))
        cr.set_state(start)
        cr.set_episodes(steps)
        if split:
            for t in range(T):
                cr.step(rv[t:t + 1], n_steps=1)
        else:
            cr.step(rv, n_steps=T)
        env, _ = cr.stats()
        runs.append((env, cr.state()))
        cr.close()
    (one, s_one), (many, s_many) = runs
    assert np.array_equal(s_one, s_many)
    for e in range(sc.n_envs):
        assert one[e]["steps"] == many[e]["steps"] == T
        assert one[e]["agent_collisions"] == many[e]["agent_collisions"], (e, one[e], many[e])
        assert one[e]["segment_collisions"] == many[e]["segment_collisions"]
        assert one[e]["speed_sum"] == pytest.approx(many[e]["speed_sum"], rel=1e-9)
    # the restored start overlaps: had it been counted, the environments that
    # start over would show at least one extra collision per start
    d = np.linalg.norm(start[1, :2] - start[0, :2])
    assert d < sc.radius[0] + sc.radius[1] - 1e-3


@pytest.mark.parametrize("path", PATHS)
def test_set_goals_removes_episodes_and_reset_stats_keeps_clock(path):
    from paper_2505_00690_gb300 import crowd as cw

    sc = scenes.urban_block(6, n_envs=3, n_peds=40, steps=30)
    steps = np.array([4, 6, 5], np.int32)
    T = 15
    rv = np.stack([sc.robot_vel_at(t) for t in range(T)]).astype(np.float32)

    def run(setup, calls):
        cr = cw.Crowd(sc, flags=_flags(path, cw.CROWD_FLAG_STATS))
        setup(cr)
        t = 0
        for n, reset in calls:
            cr.step(rv[t:t + n], n_steps=n)
            if reset:
                cr.reset_stats()
            t += n
        out = cr.state()
        cr.close()
        return out

    plain = run(lambda c: None, [(T, False)])
    removed = run(lambda c: (c.set_episodes(steps), c.set_goals(sc.goal)), [(T, False)])
    assert np.array_equal(removed, plain)
    straight = run(lambda c: c.set_episodes(steps), [(T, False)])
    assert not np.array_equal(straight, plain)
    with_reset = run(lambda c: c.set_episodes(steps), [(3, True), (7, True), (T - 10, False)])
    assert np.array_equal(with_reset, straight)
    # calls of one length after each reset replay one cached graph on the tiled path
    same_len = run(lambda c: c.set_episodes(steps), [(5, True), (5, True), (5, False)])
    assert np.array_equal(same_len, straight)


def test_episode_arguments_are_checked():
    from paper_2505_00690_gb300 import crowd as cw

    sc = scenes.urban_block(6, n_envs=2, n_peds=20, steps=5)
    cr = cw.Crowd(sc)
    with pytest.raises(cw.CrowdError):
        cr.set_episodes(np.array([3, -1], np.int32))
    bad = sc.state().astype(np.float32)
    bad[0, 0] = np.nan
    with pytest.raises(cw.CrowdError):
        cr.set_episodes(np.array([3, 1], np.int32), init_state=bad)
    cr.set_episodes(None)
    cr.close()


@pytest.mark.parametrize("path", PATHS)
def test_episodes_with_cars_repeat_and_split_alike(path):
    """Cars start over with their environment: arc positions and speeds come
    back to their values at crowd_set_episodes, so with repeating robot
    commands the cars' and the crowd's states repeat episode after episode;
    one call and single steps agree bit for bit."""
    from paper_2505_00690_gb300 import crowd as cw

    sc, veh = scenes.urban_block_with_vehicles(3, n_envs=4, n_peds=48, n_vehicles=4, steps=40)
    steps = np.array([6, 0, 9, 4], np.int32)
    T = 20
    rv = _periodic_commands(sc, steps, T)
    runs = []
    for single in (True, False):
        cr = cw.Crowd(sc, flags=_flags(path))
        cr.set_vehicles(veh)
        cr.set_episodes(steps)
        seen = [(cr.state(), *cr.vehicle_state())]
        if single:
            for t in range(T):
                cr.step(rv[t:t + 1], n_steps=1)
                seen.append((cr.state(), *cr.vehicle_state()))
        else:
            cr.step(rv, n_steps=T)
            seen.append((cr.state(), *cr.vehicle_state()))
        runs.append(seen)
        cr.close()
    assert all(np.array_equal(x, y) for x, y in zip(runs[0][-1], runs[1][-1]))
    states = runs[0]
    es = sc.env_start
    car_env = np.searchsorted(es, veh.agent, side="right") - 1
    for e, L in enumerate(steps):
        if L == 0:
            continue
        rows = slice(es[e], es[e + 1])
        cars = car_env == e
        assert cars.any()
        assert not np.array_equal(states[L][2][cars], states[0][2][cars])  # the cars moved
        for t in range(L + 1, T + 1):
            j = (t - 1) % L + 1
            assert np.array_equal(states[t][0][rows], states[j][0][rows]), (e, t)
            assert np.array_equal(states[t][1][cars], states[j][1][cars]), (e, t)
            assert np.array_equal(states[t][2][cars], states[j][2][cars]), (e, t)


@pytest.mark.parametrize("path", PATHS)
def test_restart_mask_starts_chosen_environments_over(path):
    """crowd_restart_envs: the masked environments take the snapshot's rows
    and goal counters (the oracle's restart_masked), the others keep theirs,
    bit for bit.  Stepping on, the masked environments run like a handle of
    those environments started from the snapshot, the others like a handle
    that never stopped."""
    from paper_2505_00690_gb300 import crowd as cw

    sc = scenes.urban_block(9, n_envs=5, n_peds=40, steps=40)
    queue = scenes.goal_queue(sc, 3, seed=4, hop=2.0)
    owner = _owner(sc)
    mask = np.array([1, 0, 1, 0, 1], np.uint8)
    rv = np.stack([sc.robot_vel_at(t) for t in range(20)]).astype(np.float32)
    cr = cw.Crowd(sc, flags=_flags(path))
    with pytest.raises(cw.CrowdError) as err:
        cr.restart_envs(mask)  # no snapshot yet
    assert err.value.status == cw.CROWD_ESTATE
    cr.set_goal_queue(queue, cyclic=True)
    cr.set_episodes(np.zeros(sc.n_envs, np.int32))  # a snapshot, no scheduled starts
    snap = cr.state()
    cr.step(rv[:12], n_steps=12)
    before, idx_before = cr.state(), cr.goal_index()
    assert idx_before.any()  # some agents moved on along their queues
    cr.restart_envs(mask)
    assert np.array_equal(cr.state(), oracle.restart_masked(mask, owner, before, snap))
    assert np.array_equal(cr.goal_index(), oracle.restart_masked(mask, owner, idx_before, np.zeros_like(idx_before)))
    cr.step(rv[12:20], n_steps=8)
    out = cr.state()
    cr.close()
    es = sc.env_start

    def rows(a, envs):
        return np.concatenate([a[es[e]:es[e + 1]] for e in envs])

    for envs, start, cmds in ((np.flatnonzero(mask), 12, 8), (np.flatnonzero(mask == 0), 0, 20)):
        sub = cw.Crowd(sc.subset([int(e) for e in envs]), flags=_flags(path))
        sub.set_goal_queue(rows(queue, envs), cyclic=True)
        sub.set_state(rows(snap, envs))
        sub.step(np.ascontiguousarray(rv[start:start + cmds][:, envs]), n_steps=cmds)
        assert np.array_equal(sub.state(), rows(out, envs)), envs
        sub.close()


@pytest.mark.parametrize("path", PATHS)
def test_episodes_with_goal_pools_repeat(path):
    """A goal pool's draws are counted per agent from the snapshot's counters,
    so with repeating robot commands an environment draws the same goals in
    every episode and its states and counters repeat."""
    from paper_2505_00690_gb300 import crowd as cw

    sc = scenes.urban_block(10, n_envs=3, n_peds=40, steps=40)
    q = scenes.goal_queue(sc, 2, seed=5)
    first = (sc.pos + np.clip(q[:, 0] - sc.pos, -1.5, 1.5)).astype(np.float32)
    steps = np.array([12, 0, 9], np.int32)
    T = 30
    rv = _periodic_commands(sc, steps, T)
    cr = cw.Crowd(sc, flags=_flags(path))
    cr.set_goals(first)
    cr.set_goal_pool(np.asarray(sc.env_start, np.int32), np.ascontiguousarray(q[:, 1]), 99)
    cr.set_episodes(steps)
    seen = [(cr.state(), cr.goal_index())]
    for t in range(T):
        cr.step(rv[t:t + 1], n_steps=1)
        seen.append((cr.state(), cr.goal_index()))
    cr.close()
    es = sc.env_start
    drew = False
    for e, L in enumerate(steps):
        if L == 0:
            continue
        rows = slice(es[e], es[e + 1])
        drew |= bool(seen[L][1][rows].any())
        for t in range(L + 1, T + 1):
            j = (t - 1) % L + 1
            assert np.array_equal(seen[t][0][rows], seen[j][0][rows]), (e, t)
            assert np.array_equal(seen[t][1][rows], seen[j][1][rows]), (e, t)
    assert drew  # goals were drawn within the episodes
