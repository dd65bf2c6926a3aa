"""Pins of the episode rule of the oracle (CPU only): the restart schedule by
hand, the row selection by hand, and rollouts of the oracle step with restarts
that must repeat exactly, episode after episode, when the robot's commands
repeat with the episode."""
import numpy as np

import oracle
from paper_2505_00690_gb300 import scenes


def test_restart_schedule_by_hand():
    steps = [0, 1, 3, 5]
    assert oracle.episode_restarts(0, steps).tolist() == [False, False, False, False]
    assert oracle.episode_restarts(1, steps).tolist() == [False, True, False, False]
    assert oracle.episode_restarts(3, steps).tolist() == [False, True, True, False]
    assert oracle.episode_restarts(7, steps).tolist() == [False, True, False, False]
    assert oracle.episode_restarts(15, steps).tolist() == [False, True, True, True]


def test_restart_rows_by_hand():
    owner = [0, 0, 1, 2]
    cur = np.arange(8.0).reshape(4, 2)
    snap = -np.arange(8.0).reshape(4, 2) - 1
    out = oracle.restart_rows(6, [2, 0, 3], owner, cur, snap)  # envs 0 and 2 start over at t = 6
    assert out.tolist() == [[-1, -2], [-3, -4], [4, 5], [-7, -8]]
    assert cur[0, 0] == 0  # the input is not modified
    assert np.array_equal(oracle.restart_rows(5, [2, 0, 3], owner, cur, snap), cur)


def test_restart_masked_by_hand():
    owner = [0, 0, 1, 2, 2]
    cur = np.arange(5.0)
    snap = -np.arange(5.0) - 1
    assert oracle.restart_masked([0, 1, 0], owner, cur, snap).tolist() == [0, 1, -3, 3, 4]
    assert oracle.restart_masked([1, 0, 1], owner, cur, snap).tolist() == [-1, -2, 2, -4, -5]
    assert oracle.restart_masked([0, 0, 0], owner, cur, snap).tolist() == cur.tolist()


def _run(scene, steps, T, rv):
    """States after 1..T oracle steps from the scene's start, environments
    starting over by `steps`; rv[t] is the robot command of step t."""
    o = oracle.OracleScene(scene)
    owner = np.repeat(np.arange(scene.n_envs), scene.agents_per_env)
    s0 = scene.state().astype(np.float64)
    S, out = s0.copy(), [s0.copy()]
    for t in range(T):
        S = oracle.restart_rows(t, steps, owner, S, s0)
        pos, vel, _, _ = o.step(S[:, :2], S[:, 2:], rv[t])
        S = np.concatenate([pos, vel], 1)
        out.append(S)
    return out


def test_episodes_repeat_exactly():
    """With commands that repeat with the episode, an environment's states
    repeat: the state after L + j steps is the state after j steps, for
    j = 1..L (the episode's last state included, since the restart happens at
    the start of the next step, not at the end of the last one).  An
    environment without episodes runs as if none were set."""
    sc = scenes.urban_block(3, n_envs=3, n_peds=40, steps=40)
    steps = [5, 0, 8]
    T = 19
    base = np.stack([sc.robot_vel_at(t) for t in range(T)])
    rv = base.copy()
    for e, L in enumerate(steps):
        if L:
            rv[:, e] = base[np.arange(T) % L, e]
    out = _run(sc, steps, T, rv)
    plain = _run(sc, [0, 0, 0], T, rv)
    es = sc.env_start
    for e, L in enumerate(steps):
        rows = slice(es[e], es[e + 1])
        if L == 0:
            for t in range(T + 1):
                assert np.array_equal(out[t][rows], plain[t][rows])
            continue
        assert not np.array_equal(out[L][rows], out[0][rows])  # the episode moved the crowd
        for k in range(1, (T - 1) // L + 1):
            for j in range(1, L + 1):
                if k * L + j <= T:
                    assert np.array_equal(out[k * L + j][rows], out[j][rows]), (e, k, j)
        # before the first restart the run is the plain one
        for t in range(L + 1):
            assert np.array_equal(out[t][rows], plain[t][rows])
