"""Throughput of the crowd step on every workload of the benchmark table.

    python -m paper_2505_00690_gb300.configs [--only NAME ...]

For each workload: the batched path (autotuned launch shape, the timed
launches on the GPU bracketed by synchronisation, inputs resident), the
plain form (one environment per launch, one step per launch, on a bounded
sample), and the serving stream.  One JSON line per workload.  The CPU
oracle is not timed here (bench.py times it on the default workload).
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

UNIT = "agent-steps/s"


def _time_rollouts(cr, rv, steps, reps, init):
    ms = []
    for _ in range(reps):
        cr.set_state(init)
        cr.synchronize()
        t0 = time.perf_counter()
        cr.step(rv, n_steps=steps)
        cr.synchronize()
        ms.append((time.perf_counter() - t0) * 1e3)
    return ms


def batched(sc, steps, reps=3, autotune_steps=None, flags=0):
    from . import crowd as cw

    rv = None if sc.robot_vel is None else np.ascontiguousarray(sc.robot_vel[:steps])
    cr = cw.Crowd(sc, flags=flags)
    tuning = cr.autotune(n_steps=autotune_steps) if autotune_steps else cr.tuning()
    init = sc.state()
    _time_rollouts(cr, rv, steps, 1, init)  # warm (graphs, caches)
    ms = _time_rollouts(cr, rv, steps, reps, init)
    cr.close()
    best = min(ms)
    return {"value": sc.n_agents * steps / (best / 1e3), "unit": UNIT, "ms_per_rollout": best,
            "ms_all": ms, "steps": steps, "tuning": tuning}


def plain(sc, steps, max_envs=32):
    """One environment per launch, one step per launch (same kernels)."""
    from . import crowd as cw

    envs = list(range(min(sc.n_envs, max_envs)))
    handles = [cw.Crowd(sc.subset([e]), flags=0) for e in envs]
    rvs = [None if sc.robot_vel is None else np.ascontiguousarray(sc.robot_vel[:steps, e:e + 1]) for e in envs]
    for h, rv in zip(handles, rvs):
        h.step(None if rv is None else rv[:1], n_steps=1)
        h.synchronize()
    t0 = time.perf_counter()
    for k in range(steps):
        for h, rv in zip(handles, rvs):
            h.step(None if rv is None else rv[k:k + 1], n_steps=1)
    for h in handles:
        h.synchronize()
    dt = time.perf_counter() - t0
    agents = sum(int(sc.agents_per_env[e]) for e in envs)
    for h in handles:
        h.close()
    return {"value": agents * steps / dt, "unit": UNIT, "envs": len(envs), "steps": steps}


def run(only=None):
    from . import build as B
    from . import crowd as cw
    from . import scenes, serve

    B.build()
    out = []
    cases = [
        ("plain_square", lambda: scenes.plain_square(0), 200, 20, 0),
        ("urban_block", lambda: scenes.urban_block(0), 1000, 400, 0),
        ("uneven_batch", lambda: scenes.uneven_batch(0), 50, 50, 0),
        ("dense_crowd", lambda: scenes.dense_crowd(0), 500, None, 0),
    ]
    for name, mk, steps, tune, flags in cases:
        if only and name not in only:
            continue
        sc = mk()
        b = batched(sc, steps, autotune_steps=tune, flags=flags)
        p = plain(sc, min(steps, 20), max_envs=16 if name == "dense_crowd" else 64)
        line = {"workload": name, "envs": sc.n_envs, "agents": sc.n_agents, "batched": b, "plain": p,
                "batched_over_plain": b["value"] / p["value"]}
        print(json.dumps(line), flush=True)
        out.append(line)
    if not only or "serving" in only:
        reqs = scenes.serving_stream(seed=0, rate=200.0, duration_s=10.0)
        params = cw.params_for(reqs[0].scene)
        s = serve.run_stream(reqs, params, reqs[0].scene.dt, chunk_steps=50, max_slots=1024, mem_budget=4 << 30)
        s.pop("results", None)
        s["plain_agent_steps_per_s"] = serve.run_plain(reqs[:20], params, reqs[0].scene.dt)
        line = {"workload": "serving", "serving": s}
        print(json.dumps(line), flush=True)
        out.append(line)
    return out


if __name__ == "__main__":
    ap = argparse.ArgumentParser()
    ap.add_argument("--only", nargs="*", default=None)
    a = ap.parse_args()
    run(a.only)
