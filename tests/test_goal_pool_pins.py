"""Pins of the goal-pool rule of the oracle (CPU only): the first draw of
agent 0 under seed 0 is fixed by Philox4x32-10's published known-answer
vector for a zero counter and key; pools of one point and of none; the robot
row; and picks spread evenly over a pool."""
import numpy as np

import oracle

KAT0 = 0x6627E8D5  # first word of Philox4x32-10(0, 0): Random123 known-answer vectors


def _one(n_pool, seed=0, agent=0, k=0, n_agents=1):
    pos = np.zeros((n_agents, 2))
    goal = np.zeros((n_agents, 2))  # reached: the agent stands on its goal
    idx = np.full(n_agents, k)
    pool = np.stack([np.arange(n_pool, dtype=float) + 10.0, np.zeros(n_pool)], 1)
    return oracle.advance_goals_pool(pos, np.full(n_agents, 0.3), goal, idx, [0, n_pool], pool,
                                     np.zeros(n_agents, int), seed)


def test_first_draw_matches_the_known_answer():
    for n in (1, 2, 7, 10, 1000):
        g, k = _one(n)
        pick = (KAT0 * n) >> 32
        assert g[0, 0] == 10.0 + pick and k[0] == 1
    g, _ = _one(10)
    assert g[0, 0] == 13.0  # floor(0x6627E8D5 * 10 / 2^32) = 3


def test_empty_pool_robot_and_not_reached():
    g, k = _one(0)
    assert g[0].tolist() == [0.0, 0.0] and k[0] == 0
    pos = np.array([[0.0, 0.0], [5.0, 5.0], [1.0, 1.0]])
    goal = np.array([[0.0, 0.0], [0.0, 0.0], [1.2, 1.0]])  # reached, far, within r = 0.3
    g, k = oracle.advance_goals_pool(pos, np.full(3, 0.3), goal, np.zeros(3), [0, 4], np.ones((4, 2)),
                                     np.zeros(3, int), 5, skip=[True, False, False])
    assert k.tolist() == [0, 0, 1]
    assert g[0].tolist() == [0.0, 0.0] and g[1].tolist() == [0.0, 0.0] and g[2].tolist() == [1.0, 1.0]


def test_picks_spread_evenly():
    """2000 agents on their goals draw from a pool of 8 points: every point
    is taken, with counts within a chi-square bound (7 degrees of freedom,
    p = 0.999: 24.3)."""
    n = 2000
    g, k = _one(8, seed=0x1234_5678_9ABC, n_agents=n)
    counts = np.bincount((g[:, 0] - 10.0).astype(int), minlength=8)
    chi2 = ((counts - n / 8) ** 2 / (n / 8)).sum()
    assert counts.min() > 0 and chi2 < 24.3 and (k == 1).all()
    g2, _ = _one(8, seed=0x1234_5678_9ABC, k=1, n_agents=n)  # the next draw differs
    assert (g2[:, 0] != g[:, 0]).sum() > n / 2
