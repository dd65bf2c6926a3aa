"""Pins of the oracle's work counts (no GPU): the units the roofline's
operation count is built from, checked against brute-force counts and hand
cases, not against the oracle's own arithmetic."""
import numpy as np

import oracle
from paper_2505_00690_gb300 import scenes


def test_pairs_in_range_match_brute_force():
    sc = scenes.urban_block(4, n_envs=3, n_peds=40, steps=5)
    o = oracle.OracleScene(sc)
    work = {}
    o.step(sc.pos, sc.vel, sc.robot_vel_at(0), work=work)
    R2 = float(np.float32(sc.neighbor_dist)) ** 2
    pairs = lines = 0
    for e in range(sc.n_envs):
        P = sc.pos[sc.env_start[e]:sc.env_start[e + 1]].astype(np.float64)
        d2 = ((P[:, None, :] - P[None]) ** 2).sum(2)
        np.fill_diagonal(d2, np.inf)
        inr = (d2 < R2).sum(1)
        pairs += int(inr.sum())
        robot = sc.robot_index[e]
        lines += int(sum(min(sc.max_neighbors, int(c)) for i, c in enumerate(inr) if i != robot))
    assert work["agent_steps"] == sc.n_agents
    assert work["pairs_in_range"] == pairs
    assert work["agent_lines"] == lines
    assert work["lp_checks"] == work["agent_lines"] + work["obstacle_lines"]
    assert 0 < work["lp_solves"] <= work["lp_checks"]


def test_lone_agent_and_wall_counts():
    """A lone agent in the open: one update, nothing else.  Facing a wall
    inside its reach: one segment line, checked once, violated once (the
    preferred velocity runs into it), no earlier line for that solve."""
    from tests.test_obstacle_pins import _wall_scene

    sc = _wall_scene(60.0)
    o = oracle.OracleScene(sc)
    w = {}
    o.step(sc.pos, sc.vel, work=w)
    assert w == dict(agent_steps=1, pairs_in_range=0, agent_lines=0, obstacle_lines=0, lp_checks=0, lp_solves=0,
                     lp_solve_lines=0, fallbacks=0)
    sc = _wall_scene(2.0)
    o = oracle.OracleScene(sc)
    w = {}
    o.step(sc.pos, sc.vel, work=w)
    assert w == dict(agent_steps=1, pairs_in_range=0, agent_lines=0, obstacle_lines=1, lp_checks=1, lp_solves=1,
                     lp_solve_lines=0, fallbacks=0)
