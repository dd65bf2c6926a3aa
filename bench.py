"""Benchmark of the batched ORCA crowd step (agent-steps/s).

Headline workload (the largest single-GPU configuration): the dense crowd,
16 environments x 20,000 pedestrians at 2 per m^2 in 100 x 100 m with 200
random segment obstacles each, K = 16 neighbours within R = 3 m, dt 0.1 s.
One benchmark step = one 500-step rollout of all 16 environments from the
initial state (320,000 agents x 500 steps), issued as one
``crowd_step(n_steps=500)`` call (graph-replayed tiled kernels).

Timed region: the K rollouts, each bracketed by CUDA events on the crowd
stream; between rollouts (untimed) the state is reset on the device and a
256 MiB buffer is written to flush L2.  ``e2e`` repeats the measurement
through the C ABI with host buffers: per step the initial state goes
host->device from pinned memory and the final state comes back
device->host, inside the timed region.

The same line carries the serving workload (Poisson request stream at
200 req/s: p50/p99 latency and throughput, plus a sweep of arrival rates),
the urban block and the uneven batch (batched and plain forms), the plain
form of the headline, the CPU oracle on the host cores, the roofline of the
update kernel and the sampled clocks.

``--impl reference`` times the FP64 CPU oracle (the parity reference) on a
bounded sample of the same workload on the host cores.
"""
from __future__ import annotations

import argparse
import json
import os
import socket
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "agent-steps/sec at <=1e-4 m/s vs FP64 oracle, batched vs plain; p50/p99 latency"
UNIT = "agent-steps/s"
WORKLOAD = ("dense_crowd: 16 envs x 20,000 pedestrians (2 per m^2 in 100x100 m, 200 segments/env), K 16, "
            "R 3 m, 500-step rollout, dt 0.1")
ROLLOUT = 500
# dram__bytes_read.sum + dram__bytes_write.sum of one launch of the update
# kernel on this workload (ncu, one pass, `bench.py --profile-case dense`:
# the second step of the rollout), or None when the kernel has changed since
# the counters were taken
UPDATE_DRAM_BYTES = 146_685_184
FP32_LANES_PER_SM = 128
N_SMS = 152
SERVE_RATES = (200.0, 400.0, 800.0, 1600.0)


def _dist_env():
    from paper_2505_00690_gb300 import replicas

    return replicas.dist_env()


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "50"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.path or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(smax)), "reasons": sorted(reasons),
                "samples": len(sm)}


def algorithmic_flops(work):
    """Algorithmic FP32 operations of the counted work, in units the oracle
    counts identically on the same states (tests/test_work_counts_gpu.py):
    7 per pair within R (the pairs an exact neighbour search must test; the
    cells searched hold more, which is not counted), 35 per agent half-plane,
    20 per segment half-plane, 4 per LP line check, 15 + 10k per 1D sub-solve
    taking k earlier lines into account.  The fallback's own work is not
    counted."""
    return (7 * work["pairs_in_range"] + 35 * work["agent_lines"] + 20 * work["obstacle_lines"]
            + 4 * work["lp_checks"] + 15 * work["lp_solves"] + 10 * work["lp_solve_lines"])


def time_rollouts(cr, rv_dev, init, steps, n_timed, n_warm, stream, flush, dist=False):
    """Rollouts from `init` of `steps` steps: n_warm untimed, then n_timed each
    bracketed by CUDA events on the crowd stream (state reset and L2 flush
    between them, untimed).  Returns (per-rollout ms, wall seconds, kernels
    the library launched in the timed region)."""
    import torch

    def reset():
        cr.set_state(init)
        with torch.cuda.stream(stream):
            flush.fill_(1.0)

    for _ in range(n_warm):
        reset()
        cr.step(rv_dev, n_steps=steps)
    torch.cuda.synchronize()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(n_timed)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(n_timed)]
    if dist:
        import torch.distributed as tdist

        tdist.barrier()
    torch.cuda.synchronize()
    launches0 = cr.launches()
    t0 = time.perf_counter()
    for k in range(n_timed):
        reset()
        starts[k].record(stream)
        cr.step(rv_dev, n_steps=steps)
        ends[k].record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    launches = cr.launches() - launches0
    if dist:
        tdist.barrier()
    return [s.elapsed_time(e) for s, e in zip(starts, ends)], wall, launches


def plain_form(sc, steps, max_envs, stream):
    """The plain form: the same kernels, one environment per launch and one
    step per launch, on the first max_envs environments."""
    import torch

    from paper_2505_00690_gb300 import crowd as cw

    envs = list(range(min(sc.n_envs, max_envs)))
    handles = [cw.Crowd(sc.subset([e]), flags=0, stream=stream.cuda_stream) for e in envs]
    rvs = [None if sc.robot_vel is None else
           torch.from_numpy(np.ascontiguousarray(sc.robot_vel[:steps, e:e + 1])).cuda() for e in envs]
    for h, rv in zip(handles, rvs):  # warm
        h.step(None if rv is None else rv[:1], n_steps=1)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in range(steps):
        for h, rv in zip(handles, rvs):
            h.step(None if rv is None else rv[k:k + 1], n_steps=1)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    agents = sum(int(sc.agents_per_env[e]) for e in envs)
    for h in handles:
        h.close()
    return {"value": agents * steps / dt, "unit": UNIT, "envs": len(envs), "steps": steps,
            "launches": steps * len(envs)}


def side_workload(name, sc, steps, tune_steps, plain_envs, stream, flush, reps=3):
    """Batched (autotuned, best of `reps` rollouts by CUDA events) and plain
    forms of one more workload of the benchmark table."""
    import torch

    from paper_2505_00690_gb300 import crowd as cw

    with torch.cuda.stream(stream):
        cr = cw.Crowd(sc, flags=0, stream=stream.cuda_stream)
        init = torch.from_numpy(sc.state()).cuda()
        rv = None if sc.robot_vel is None else torch.from_numpy(np.ascontiguousarray(sc.robot_vel[:steps])).cuda()
    tuning = cr.autotune(n_steps=tune_steps) if tune_steps else cr.tuning()
    ms, _, _ = time_rollouts(cr, rv, init, steps, reps, 1, stream, flush)
    cr.close()
    best = min(ms)
    value = sc.n_agents * steps / (best / 1e3)
    # the same rollout once more (untimed) with the work counted, so that
    # workloads of different density compare by work rate as well
    counted = cw.Crowd(sc, flags=cw.CROWD_FLAG_COUNT_WORK, stream=stream.cuda_stream)
    counted.step(rv, n_steps=steps)
    work = counted.work()
    counted.close()
    flops = algorithmic_flops(work)
    plain = plain_form(sc, min(steps, 20), plain_envs, stream)
    return {"workload": name, "envs": sc.n_envs, "agents": sc.n_agents, "rollout_steps": steps,
            "value": value, "unit": UNIT, "ms_per_rollout": best, "ms_all": ms, "tuning": tuning,
            "counted_flop_per_agent_step": flops / max(1, work["agent_steps"]),
            "counted_tflops": flops / (best / 1e3) / 1e12,
            "plain": plain, "batched_over_plain": value / plain["value"]}


def run_ours(args):
    import torch

    from paper_2505_00690_gb300 import crowd as cw
    from paper_2505_00690_gb300 import replicas
    from paper_2505_00690_gb300 import scenes

    ws, rank, local = _dist_env()
    dist = ws > 1
    if dist:
        import torch.distributed as tdist

        tdist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(device=dev)

    from paper_2505_00690_gb300 import build as B

    B.build()
    sc = scenes.dense_crowd(seed=replicas.replica_seed(rank), steps=ROLLOUT)
    n_agents = sc.n_agents
    with torch.cuda.stream(stream):
        cr = cw.Crowd(sc, flags=0, stream=stream.cuda_stream)
        init = torch.from_numpy(sc.state()).to(dev)
        flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    torch.cuda.synchronize(dev)
    tuning = cr.autotune(n_steps=ROLLOUT)  # resident shapes only; the dense crowd runs on the tiled path

    with Clocks(local) as clk:
        per, wall, launches = time_rollouts(cr, None, init, ROLLOUT, args.steps, args.warmup, stream, flush, dist)
    clocks = clk.summary()
    my_ms = float(sum(per))
    my_agent_steps = n_agents * ROLLOUT * args.steps
    value = replicas.aggregate_throughput(my_agent_steps, my_ms / 1e3, device=dev)
    total_agent_steps = replicas.sum_over_ranks(my_agent_steps, device=dev)
    dev_ms = replicas.max_over_ranks(my_ms, device=dev)

    # ---- e2e: the same rollouts through the C ABI with pinned host buffers
    init_h = torch.from_numpy(sc.state()).pin_memory()
    out_h = torch.empty((n_agents, 4), dtype=torch.float32).pin_memory()
    lib = cw.load()
    import ctypes as C

    def e2e_step():
        cw._check(lib.crowd_set_state(cr.h, C.c_void_p(init_h.data_ptr()), cw.CROWD_HOST))
        cw._check(lib.crowd_step(cr.h, C.c_float(sc.dt), None, cw.CROWD_HOST, ROLLOUT))
        cw._check(lib.crowd_read_state(cr.h, C.c_void_p(out_h.data_ptr()), cw.CROWD_HOST))

    e2e_step()
    torch.cuda.synchronize(dev)
    if dist:
        tdist.barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        e2e_step()
    torch.cuda.synchronize(dev)
    e2e_s = replicas.max_over_ranks(time.perf_counter() - t0, device=dev)
    e2e = {"value": total_agent_steps / e2e_s, "unit": UNIT,
           "h2d_bytes_per_step": int(init_h.numel() * 4), "d2h_bytes_per_step": int(out_h.numel() * 4)}

    # ---- roofline of the update kernel (FP32 issue): counted work of one rollout
    counted = cw.Crowd(sc, flags=cw.CROWD_FLAG_COUNT_WORK, stream=stream.cuda_stream)
    counted.step(None, n_steps=ROLLOUT)
    work = counted.work()
    counted.close()
    flops = algorithmic_flops(work)
    step_s = dev_ms / 1e3 / args.steps / ROLLOUT
    sm_mhz = 2070.0
    fp32_peak = N_SMS * FP32_LANES_PER_SM * 2 * sm_mhz * 1e6 / 1e12  # TFLOP/s
    achieved = flops / ROLLOUT / step_s / 1e12
    roofline = {"bound": "alu", "achieved": achieved, "peak": fp32_peak, "unit": "TFLOP/s",
                "frac": achieved / fp32_peak,
                "traffic": UPDATE_DRAM_BYTES,
                "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 flop x 2070 MHz max SM clock",
                "launch": "one step of all 16 environments (the update kernel and its sort kernels, timed together)",
                "flops_per_launch": flops / ROLLOUT,
                "work_per_agent_step": {k: v / max(1, work["agent_steps"])
                                        for k, v in work.items() if k != "agent_steps"}}

    extra = {}
    if rank == 0 and not args.no_plain:
        p = plain_form(sc, 20, sc.n_envs, stream)
        p["batched_over_plain"] = value / ws / p["value"]
        extra["plain"] = p
    if rank == 0 and not args.no_side:
        extra["urban_block"] = side_workload("urban_block: 256 envs x (128 peds + 1 robot), 40x40 m, 36 segments/env",
                                             scenes.urban_block(0), 1000, 1000, 64, stream, flush)
        extra["uneven_batch"] = side_workload("uneven_batch: 1024 envs, 16-512 agents, 0-40 polygons",
                                              scenes.uneven_batch(0), 50, 50, 64, stream, flush)
    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu:
        cpu = cpu_baseline(sc, budget_s=args.cpu_seconds)
    serving = None
    if rank == 0 and not args.no_serve:
        serving = serve_workload(args.serve_seconds)

    cr.close()
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": dev_ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": WORKLOAD, "envs": sc.n_envs, "agents": n_agents, "rollout_steps": ROLLOUT,
                           "step": f"one {ROLLOUT}-step rollout of all envs (crowd_step n_steps={ROLLOUT})",
                           "l2": "256 MiB buffer written between timed rollouts",
                           "parallelism": f"env replicas x{ws}"},
                "wall_s": wall, "clocks": clocks, "e2e": e2e, "gpu_launches": launches,
                "tuning": tuning, "roofline": roofline, "cpu_baseline": cpu, "serving": serving,
                "kernel_ms": per, **extra}
        print(json.dumps(line))
    if dist:
        tdist.destroy_process_group()


def serve_workload(duration_s):
    """Serving workload: Poisson arrivals at 200 requests/s for duration_s,
    one environment each (32..2048 agents log-uniform, 0..60 convex polygons,
    100..1000 steps), through the continuous-batching server (4 GiB budget,
    1024 slots, 50 steps per tick); the plain form (one request at a time,
    one step per launch) on the first 20 requests; and a sweep of arrival
    rates over the same requests, their arrival times scaled by 200/rate
    (a Poisson stream at that rate), so that the sustainable throughput and
    the latency knee show."""
    from paper_2505_00690_gb300 import crowd as cw
    from paper_2505_00690_gb300 import scenes
    from paper_2505_00690_gb300 import serve

    reqs = scenes.serving_stream(seed=0, rate=SERVE_RATES[0], duration_s=duration_s)
    sc0 = reqs[0].scene
    params = cw.params_for(sc0)
    out = serve.run_stream(reqs, params, sc0.dt, chunk_steps=50, max_slots=1024, mem_budget=4 << 30)
    out.pop("results", None)
    out["rate_req_per_s"] = SERVE_RATES[0]
    out["plain_agent_steps_per_s"] = serve.run_plain(reqs[:20], params, sc0.dt)
    sweep = []
    for rate in SERVE_RATES:
        scaled = [scenes.Request(arrival_s=r.arrival_s * SERVE_RATES[0] / rate, scene=r.scene, steps=r.steps)
                  for r in reqs]
        s = serve.run_stream(scaled, params, sc0.dt, chunk_steps=50, max_slots=1024, mem_budget=4 << 30)
        sweep.append({"rate_req_per_s": rate, "p50_s": s["p50_s"], "p99_s": s["p99_s"],
                      "agent_steps_per_s": s["agent_steps_per_s"], "requests": s["requests"],
                      "max_live": s["max_live"], "wall_s": s["wall_s"]})
    out["sweep"] = sweep
    return out


def cpu_baseline(sc, budget_s=12.0, threads=None):
    """The FP64 oracle as it stands, on the host cores, on a bounded sample of
    the headline workload: consecutive steps of environment 0 (20,000
    agents, all of them) from the initial state until about budget_s; beside
    it the 1000-agent subset the teacher-forced parity test uses."""
    import oracle

    threads = threads or os.cpu_count() or 1
    one = sc.subset([0])
    o = oracle.OracleScene(one)
    pos = one.pos.astype(np.float64)
    vel = one.vel.astype(np.float64)
    steps = 0
    t0 = time.perf_counter()
    while True:
        pos, vel, _, _ = o.step(pos, vel, None, threads=threads)
        steps += 1
        if time.perf_counter() - t0 >= budget_s or steps >= ROLLOUT:
            break
    dt = time.perf_counter() - t0
    sel = np.random.default_rng(0).choice(one.n_agents, 1000, replace=False)
    t1 = time.perf_counter()
    o.step(one.pos.astype(np.float64), one.vel.astype(np.float64), None, sel=sel, threads=threads)
    sub_dt = time.perf_counter() - t1
    return {"value": one.n_agents * steps / dt, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"{steps} consecutive steps of env 0 ({one.n_agents} agents) from the initial state, FP64, "
                      f"OpenMP over agents",
            "subset_1000_agents": {"value": 1000 / sub_dt, "unit": UNIT, "steps": 1}}


def cpu_table(budget_s=6.0):
    """The FP64 oracle as it stands on each workload of the benchmark table,
    one thread and all host threads, on bounded samples (consecutive steps
    of the whole batch, or of its first environments where one step of the
    whole batch takes longer than the budget).  One JSON line per workload."""
    import oracle
    from paper_2505_00690_gb300 import scenes

    cores = os.cpu_count() or 1
    cases = [("plain_square", scenes.plain_square(0), None), ("urban_block", scenes.urban_block(0), None),
             ("uneven_batch", scenes.uneven_batch(0), None),
             ("dense_crowd", scenes.dense_crowd(0), 1)]  # one 20,000-agent env of the 16
    for name, sc, n_env in cases:
        if n_env is not None:
            sc = sc.subset(list(range(n_env)))
        o = oracle.OracleScene(sc)
        res = {}
        for threads in (1, cores):
            pos, vel = sc.pos.astype(np.float64), sc.vel.astype(np.float64)
            steps = 0
            t0 = time.perf_counter()
            while True:
                rv = sc.robot_vel_at(steps) if sc.robot_vel is not None else None
                pos, vel, _, _ = o.step(pos, vel, rv, threads=threads)
                steps += 1
                if time.perf_counter() - t0 >= budget_s or steps >= sc.steps:
                    break
            dt = time.perf_counter() - t0
            res[threads] = {"value": sc.n_agents * steps / dt, "steps": steps}
        print(json.dumps({"workload": name, "unit": UNIT, "kind": "oracle", "agents_in_sample": sc.n_agents,
                          "one_core": res[1], "all_cores": res[cores], "cores": cores}), flush=True)


def run_reference(args):
    """The reference arm: the FP64 oracle as it stands on the host cores.  Each
    benchmark step is a bounded sample of the headline workload: one ORCA
    step of all 16 environments (320,000 agents) from the initial state on."""
    ws, rank, local = _dist_env()
    if rank != 0:
        return
    from paper_2505_00690_gb300 import scenes

    sc = scenes.dense_crowd(seed=0, steps=ROLLOUT)
    import oracle

    threads = os.cpu_count() or 1
    o = oracle.OracleScene(sc)
    pos = sc.pos.astype(np.float64)
    vel = sc.vel.astype(np.float64)
    for _ in range(args.warmup):
        pos, vel, _, _ = o.step(pos, vel, None, threads=threads)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        pos, vel, _, _ = o.step(pos, vel, None, threads=threads)
    dt = time.perf_counter() - t0
    value = sc.n_agents * args.steps / dt
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": WORKLOAD, "envs": sc.n_envs, "agents": sc.n_agents,
                       "step": "one ORCA step of all envs (bounded sample of the 500-step rollout)"},
            "cpu_baseline": {"value": value, "unit": UNIT, "kind": "oracle", "cores": threads,
                             "sample": f"1 step x {args.steps} timed of all {sc.n_envs} envs ({sc.n_agents} agents)"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def profile_case(which):
    """Launches for ncu captures: `resident` = one 20-step launch of the
    256-env urban block (after one warm launch); `rollout` = the same with the
    full 1000-step rollout (for one-pass counters only); `tiled` = two single
    steps of one 20,000-agent dense-crowd environment (the second is
    captured); `dense` = two single steps of the 16-environment dense crowd
    (the headline workload; the second step's update is captured);
    `dense_rollout` = the headline workload's timed form on a short rollout:
    one warm single step, then one 20-step call (graph-replayed), every
    launch of which a one-pass launch list can take; `dense_jam` = the
    headline workload's jammed phase: a 300-step call, then two single steps
    (capture the last update, the 302nd)."""
    from paper_2505_00690_gb300 import build as B
    from paper_2505_00690_gb300 import crowd as cw
    from paper_2505_00690_gb300 import scenes

    B.build()
    if which == "resident":
        sc = scenes.urban_block(0, steps=20)
        cr = cw.Crowd(sc)
        cr.step(sc.robot_vel[:20], n_steps=20)
        cr.set_state(sc.state())
        cr.step(sc.robot_vel[:20], n_steps=20)
    elif which == "rollout":
        sc = scenes.urban_block(0, steps=1000)
        cr = cw.Crowd(sc)
        cr.step(sc.robot_vel[:1000], n_steps=1000)
        cr.set_state(sc.state())
        cr.step(sc.robot_vel[:1000], n_steps=1000)
    elif which == "dense":
        sc = scenes.dense_crowd(0, steps=4)
        cr = cw.Crowd(sc)
        cr.step(n_steps=1)
        cr.step(n_steps=1)
    elif which == "dense_jam":
        sc = scenes.dense_crowd(0, steps=300)
        cr = cw.Crowd(sc)
        cr.step(n_steps=300)
        cr.step(n_steps=1)
        cr.step(n_steps=1)
    elif which == "dense_rollout":
        sc = scenes.dense_crowd(0, steps=20)
        cr = cw.Crowd(sc)
        cr.step(n_steps=1)
        cr.step(n_steps=20)
    else:
        sc = scenes.dense_crowd(0, n_envs=1, steps=4)
        cr = cw.Crowd(sc)
        cr.step(n_steps=1)
        cr.step(n_steps=1)
    cr.synchronize()
    cr.close()
    print(json.dumps({"profile_case": which, "agents": sc.n_agents}))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def launch_replicas(args):
    """`--gpus N` outside a launcher: one replica process per GPU through
    torch.distributed.run (the same launch the contract uses), or an error
    when fewer than N GPUs are visible.  Returns the exit code."""
    try:
        import torch

        visible = torch.cuda.device_count()
    except Exception:
        visible = 0
    if visible < args.gpus:
        print(f"bench.py: --gpus {args.gpus} requested but {visible} GPU(s) visible", file=sys.stderr)
        return 2
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", f"--nproc-per-node={args.gpus}",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()), os.path.abspath(__file__)]
    cmd += [a for a in sys.argv[1:]]
    return subprocess.call(cmd)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-side", action="store_true", help="leave out the urban-block and uneven-batch keys")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-serve", action="store_true", help="leave out the serving replay and its rate sweep")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--serve-seconds", type=float, default=10.0)
    ap.add_argument("--cpu-table", action="store_true",
                    help="time the FP64 oracle on every workload (1 and all host threads) and exit")
    ap.add_argument("--profile-case", choices=["resident", "rollout", "tiled", "dense", "dense_rollout", "dense_jam"], default=None,
                    help="run a small case for an ncu capture and exit")
    args = ap.parse_args()
    if args.cpu_table:
        cpu_table()
        return 0
    if args.profile_case:
        profile_case(args.profile_case)
        return 0
    ws, rank, _ = _dist_env()
    launched = "LOCAL_RANK" in os.environ and "WORLD_SIZE" in os.environ
    if args.gpus < 1:
        print("bench.py: --gpus must be >= 1", file=sys.stderr)
        return 2
    if launched and ws != args.gpus:
        print(f"bench.py: --gpus {args.gpus} differs from the launcher's WORLD_SIZE {ws}", file=sys.stderr)
        return 2
    if not launched and args.gpus > 1:
        return launch_replicas(args)
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)
    return 0


if __name__ == "__main__":
    sys.exit(main())
