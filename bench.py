"""Benchmark of the batched ORCA crowd step (agent-steps/s).

Workload: 256 urban blocks (40 x 40 m, 8 rectangular buildings + 4 sidewalk
edges = 36 segments each), 128 pedestrians + 1 robot agent per block, robot
commands from a seeded action tensor, 1000-step rollouts, dt 0.1 s, tau 2 s,
R 5 m, K 10.  One benchmark step = one full 1000-step rollout of all 256
blocks from the initial state (33,024 agents x 1000 steps), issued as one
``crowd_step(n_steps=1000)`` call.

Timed region: the K rollouts, each bracketed by CUDA events on the crowd
stream; between rollouts (untimed) the state is reset on the device and a
256 MiB buffer is written to flush L2.  ``e2e`` repeats the measurement
through the C ABI with host buffers: per step the initial state and the
robot commands go host->device from pinned memory and the final state comes
back device->host, all inside the timed region.

``--impl reference`` times the FP64 CPU oracle (the parity reference) on a
bounded sample of the same workload on the host cores.
"""
from __future__ import annotations

import argparse
import json
import os
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
WORKLOAD = "urban_block: 256 envs x (128 peds + 1 robot), 40x40 m, 36 segments/env, 1000-step rollout, dt 0.1"
ROLLOUT = 1000
# dram__bytes_read.sum + dram__bytes_write.sum of one 1000-step rollout launch of
# the resident kernel (ncu, `bench.py --profile-case rollout`, one pass), or None
# when the kernel has changed since the counters were taken: the last capture
# (22.49e6 B) predates the flush-to-zero build, so `traffic` is null and that
# capture is reported beside it as `traffic_last_capture`
ROLLOUT_DRAM_BYTES = None
ROLLOUT_DRAM_BYTES_LAST_CAPTURE = {"bytes": 22.49e6, "build": "before -ftz=true"}
FP32_LANES_PER_SM = 128
N_SMS = 152


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


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return None


def algorithmic_flops(work):
    """Algorithmic FP32 operations of the counted work (per-unit costs of the
    crowd step: 7 per neighbour candidate, 35 per agent half-plane, 20 per
    segment half-plane, 12 per segment distance test, 4 per LP check, 15 + 10k
    per 1D sub-solve scanning k previous lines)."""
    return (7 * work["candidates"] + 35 * work["agent_lines"] + 20 * work["obstacle_lines"]
            + 12 * work["segment_tests"] + 4 * work["lp_checks"] + 15 * work["lp_solves"]
            + 10 * work["lp_solve_lines"])


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
    sc = scenes.urban_block(seed=replicas.replica_seed(rank), steps=ROLLOUT)
    n_agents = sc.n_agents
    with torch.cuda.stream(stream):
        cr = cw.Crowd(sc, flags=0, stream=stream.cuda_stream)
        init = torch.from_numpy(sc.state()).to(dev)
        rv_dev = torch.from_numpy(np.ascontiguousarray(sc.robot_vel[:ROLLOUT])).to(dev)
        flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    torch.cuda.synchronize(dev)

    # launch shape chosen by the library's autotuner (untimed), each candidate
    # timed on a whole rollout: the crowded regions that set the rollout time
    # form over hundreds of steps
    tuning = cr.autotune(n_steps=ROLLOUT)

    def one_rollout():
        cr.step(rv_dev, n_steps=ROLLOUT)

    def reset():
        cr.set_state(init)
        with torch.cuda.stream(stream):
            flush.fill_(1.0)

    for _ in range(args.warmup):
        reset()
        one_rollout()
    torch.cuda.synchronize(dev)

    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    if dist:
        tdist.barrier()
    torch.cuda.synchronize(dev)
    with Clocks(local) as clk:
        t0 = time.perf_counter()
        for k in range(args.steps):
            reset()
            starts[k].record(stream)
            one_rollout()
            ends[k].record(stream)
        torch.cuda.synchronize(dev)
        wall = time.perf_counter() - t0
    if dist:
        tdist.barrier()
    per = [s.elapsed_time(e) for s, e in zip(starts, ends)]  # ms
    my_ms = float(sum(per))
    clocks = clk.summary()
    # replicas: this rank's agent-steps, the slowest rank's time
    my_agent_steps = n_agents * ROLLOUT * args.steps
    value = replicas.aggregate_throughput(my_agent_steps, my_ms / 1e3, device=dev)
    total_agent_steps = replicas.sum_over_ranks(my_agent_steps, device=dev)
    dev_ms = replicas.max_over_ranks(my_ms, device=dev)

    # ---- e2e: same rollouts through the C ABI with pinned host buffers
    init_h = torch.from_numpy(sc.state()).pin_memory()
    rv_h = torch.from_numpy(np.ascontiguousarray(sc.robot_vel[:ROLLOUT])).pin_memory()
    out_h = torch.empty((n_agents, 4), dtype=torch.float32).pin_memory()
    lib = cw.load()
    import ctypes as C

    def e2e_step():
        cw._check(lib.crowd_set_state(cr.h, C.c_void_p(init_h.data_ptr()), cw.CROWD_HOST))
        cw._check(lib.crowd_step(cr.h, C.c_float(sc.dt), C.c_void_p(rv_h.data_ptr()), cw.CROWD_HOST, ROLLOUT))
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
           "h2d_bytes_per_step": int(init_h.numel() * 4 + rv_h.numel() * 4),
           "d2h_bytes_per_step": int(out_h.numel() * 4)}

    # ---- roofline of the resident kernel (FP32 issue): counted work of one rollout
    counted = cw.Crowd(sc, flags=cw.CROWD_FLAG_COUNT_WORK, stream=stream.cuda_stream)
    counted.step(rv_dev, n_steps=ROLLOUT)
    work = counted.work()
    counted.close()
    flops = algorithmic_flops(work)
    launch_s = dev_ms / 1e3 / args.steps
    peaks = measured_peaks()
    sm_mhz = 2070.0
    fp32_peak = N_SMS * FP32_LANES_PER_SM * 2 * sm_mhz * 1e6 / 1e12  # TFLOP/s
    achieved = flops / launch_s / 1e12
    roofline = {"bound": "alu", "achieved": achieved, "peak": fp32_peak, "unit": "TFLOP/s",
                "frac": achieved / fp32_peak, "traffic": ROLLOUT_DRAM_BYTES,
                "traffic_last_capture": ROLLOUT_DRAM_BYTES_LAST_CAPTURE,
                "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 flop x 2070 MHz max SM clock",
                "flops_per_launch": flops, "work_per_agent_step": {k: v / max(1, work["agent_steps"])
                                                                   for k, v in work.items() if k != "agent_steps"}}

    # ---- plain form: one environment per launch, one step per launch, same kernel
    plain = None
    if rank == 0 and not args.no_plain:
        plain_steps = 20
        handles = [cw.Crowd(sc.subset([e]), flags=0, stream=stream.cuda_stream) for e in range(sc.n_envs)]
        rv1 = [torch.from_numpy(np.ascontiguousarray(sc.robot_vel[:plain_steps, e:e + 1])).to(dev)
               for e in range(sc.n_envs)]
        for e, h in enumerate(handles):  # warm
            h.step(rv1[e][:1], n_steps=1)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        for k in range(plain_steps):
            for e, h in enumerate(handles):
                h.step(rv1[e][k:k + 1], n_steps=1)
        torch.cuda.synchronize(dev)
        pt = time.perf_counter() - t0
        plain_value = n_agents * plain_steps / pt
        plain = {"value": plain_value, "unit": UNIT, "steps": plain_steps,
                 "launches": plain_steps * sc.n_envs, "batched_over_plain": value / ws / plain_value}
        for h in handles:
            h.close()

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu:
        cpu = cpu_baseline(sc, budget_s=args.cpu_seconds)

    serving = None
    if rank == 0 and args.serve:
        serving = serve_workload(args.serve_seconds)

    cr.close()
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": dev_ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": WORKLOAD, "envs": sc.n_envs, "agents": n_agents, "rollout_steps": ROLLOUT,
                           "step": "one 1000-step rollout of all envs (crowd_step n_steps=1000)",
                           "l2": "256 MiB buffer written between timed rollouts",
                           "parallelism": f"env replicas x{ws}"},
                "wall_s": wall, "clocks": clocks, "e2e": e2e, "gpu_launches": args.steps, "tuning": tuning,
                "roofline": roofline, "cpu_baseline": cpu, "plain": plain, "serving": serving,
                "kernel_ms": per}
        print(json.dumps(line))
    if dist:
        tdist.destroy_process_group()


def serve_workload(duration_s):
    """Serving workload: Poisson arrivals at 200 requests/s for duration_s,
    one environment each (32..2048 agents log-uniform, 0..60 convex polygons,
    100..1000 steps), through the continuous-batching server (4 GiB budget,
    1024 slots, 50 steps per tick); plus the plain form (one request at a
    time, one step per launch) on the first 20 requests."""
    from paper_2505_00690_gb300 import crowd as cw
    from paper_2505_00690_gb300 import scenes
    from paper_2505_00690_gb300 import serve

    reqs = scenes.serving_stream(seed=0, rate=200.0, duration_s=duration_s)
    sc0 = reqs[0].scene
    params = cw.params_for(sc0)
    out = serve.run_stream(reqs, params, sc0.dt, chunk_steps=50, max_slots=1024, mem_budget=4 << 30)
    out.pop("results", None)
    plain = serve.run_plain(reqs[:20], params, sc0.dt)
    out["plain_agent_steps_per_s"] = plain
    out["rate_req_per_s"] = 200.0
    return out


def cpu_baseline(sc, budget_s=12.0, threads=None):
    """The FP64 oracle as it stands, on the host cores, on a bounded sample:
    consecutive steps of the full 256-env batch until about budget_s."""
    import oracle

    threads = threads or os.cpu_count() or 1
    o = oracle.OracleScene(sc)
    pos = sc.pos.astype(np.float64)
    vel = sc.vel.astype(np.float64)
    steps = 0
    t0 = time.perf_counter()
    while True:
        pos, vel, _, _ = o.step(pos, vel, sc.robot_vel_at(steps), threads=threads)
        steps += 1
        if time.perf_counter() - t0 >= budget_s or steps >= ROLLOUT:
            break
    dt = time.perf_counter() - t0
    return {"value": sc.n_agents * steps / dt, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"{steps} consecutive steps of all {sc.n_envs} envs ({sc.n_agents} agents), FP64, OpenMP over agents"}


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
    ws, rank, local = _dist_env()
    if rank != 0:
        return
    from paper_2505_00690_gb300 import scenes

    sc = scenes.urban_block(seed=0, steps=ROLLOUT)
    import oracle

    threads = os.cpu_count() or 1
    o = oracle.OracleScene(sc)
    pos = sc.pos.astype(np.float64)
    vel = sc.vel.astype(np.float64)
    sample_steps = 2  # each benchmark step: 2 ORCA steps of the full batch
    k = 0
    for _ in range(args.warmup):
        for _ in range(sample_steps):
            pos, vel, _, _ = o.step(pos, vel, sc.robot_vel_at(k), threads=threads)
            k += 1
    t0 = time.perf_counter()
    for _ in range(args.steps):
        for _ in range(sample_steps):
            pos, vel, _, _ = o.step(pos, vel, sc.robot_vel_at(k), threads=threads)
            k += 1
    dt = time.perf_counter() - t0
    value = sc.n_agents * sample_steps * args.steps / dt
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": WORKLOAD, "envs": sc.n_envs, "agents": sc.n_agents,
                       "step": f"{sample_steps} ORCA steps of all envs (bounded sample of the 1000-step rollout)"},
            "cpu_baseline": {"value": value, "unit": UNIT, "kind": "oracle", "cores": threads,
                             "sample": f"{sample_steps} steps x {args.steps} timed of all {sc.n_envs} envs"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def profile_case(which):
    """Launches for ncu captures: `resident` = one 20-step launch of the
    256-env urban block (after one warm launch); `rollout` = the same with the
    full 1000-step rollout (for one-pass counters only); `tiled` = two single
    steps of one 20,000-agent dense-crowd environment (the second is
    captured)."""
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
        # the timed launch of the default run: one 1000-step rollout of the
        # 256-env urban block (default launch shape), after a warm one
        sc = scenes.urban_block(0, steps=ROLLOUT)
        cr = cw.Crowd(sc)
        cr.step(sc.robot_vel[:ROLLOUT], n_steps=ROLLOUT)
        cr.set_state(sc.state())
        cr.step(sc.robot_vel[:ROLLOUT], n_steps=ROLLOUT)
    else:
        sc = scenes.dense_crowd(0, n_envs=1, steps=4)
        cr = cw.Crowd(sc)
        cr.step(n_steps=1)
        cr.step(n_steps=1)
    cr.synchronize()
    cr.close()
    print(json.dumps({"profile_case": which, "agents": sc.n_agents}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--serve", action="store_true",
                    help="also replay the serving workload (Poisson request stream) and report p50/p99 latency")
    ap.add_argument("--serve-seconds", type=float, default=10.0)
    ap.add_argument("--cpu-table", action="store_true",
                    help="time the FP64 oracle on every workload (1 and all host threads) and exit")
    ap.add_argument("--profile-case", choices=["resident", "rollout", "tiled"], default=None,
                    help="run a small case for an ncu capture and exit")
    args = ap.parse_args()
    if args.cpu_table:
        cpu_table()
    elif args.profile_case:
        profile_case(args.profile_case)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
