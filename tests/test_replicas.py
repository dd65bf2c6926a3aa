"""Host logic of the multi-GPU form (environment replicas, one process per
rank): two gloo ranks on the CPU build their batches, exchange only the
timing, and aggregate it the way bench.py does."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    from paper_2505_00690_gb300 import replicas, scenes

    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        assert replicas.dist_env() == (world, rank, rank)
        sc = scenes.urban_block(seed=replicas.replica_seed(rank), n_envs=2, steps=3)
        # each rank's batch is its own: gather a fingerprint of the start states
        fp = torch.tensor([float(np.float64(sc.pos).sum())], dtype=torch.float64)
        fps = [torch.zeros(1, dtype=torch.float64) for _ in range(world)]
        dist.all_gather(fps, fp)
        seconds = 1.0 + rank  # rank 1 is the slowest
        agent_steps = sc.n_agents * 3
        value = replicas.aggregate_throughput(agent_steps, seconds)
        out[rank] = (float(fps[0]), float(fps[1]), value, replicas.max_over_ranks(seconds),
                     replicas.sum_over_ranks(agent_steps), float(agent_steps))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_aggregate_like_bench():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    out = ctx.Manager().dict()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=240)
    assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
    r0, r1 = out[0], out[1]
    assert r0[0] == r1[0] and r0[1] == r1[1]      # both ranks saw both fingerprints
    assert r0[0] != r0[1]                         # distinct batches per rank
    assert r0[3] == r1[3] == 2.0                  # slowest rank's time
    assert r0[4] == r1[4] == r0[5] + r1[5]        # agent-steps summed
    assert r0[2] == pytest.approx((r0[5] + r1[5]) / 2.0)
    assert r0[2] == r1[2]


def test_single_process_is_identity():
    from paper_2505_00690_gb300 import replicas

    assert not dist.is_initialized()
    assert replicas.max_over_ranks(3.5) == 3.5
    assert replicas.aggregate_throughput(100.0, 4.0) == 25.0


def _bench(args, env=None):
    import subprocess
    import sys

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    e = {k: v for k, v in os.environ.items() if k not in ("WORLD_SIZE", "RANK", "LOCAL_RANK")}
    e.update(env or {})
    return subprocess.run([sys.executable, os.path.join(root, "bench.py")] + args, capture_output=True, text=True,
                          timeout=300, cwd=root, env=e)


def test_bench_gpus_without_enough_gpus_refuses():
    """`bench.py --gpus 2` outside a launcher starts one replica process per
    GPU; with fewer GPUs visible (none here) it exits non-zero instead of
    timing one GPU and calling it two."""
    if torch.cuda.is_available() and torch.cuda.device_count() >= 2:
        pytest.skip("enough GPUs: the spawn path would run the benchmark")
    r = _bench(["--gpus", "2", "--steps", "1", "--warmup", "0"])
    assert r.returncode == 2, (r.returncode, r.stderr[-500:])
    assert "--gpus 2 requested" in r.stderr
    assert not [l for l in r.stdout.splitlines() if l.startswith("{")]


def test_bench_gpus_must_match_launcher_world_size():
    """Under a launcher, --gpus must equal WORLD_SIZE (else the line's n_gpus
    and the ranks that ran would disagree)."""
    r = _bench(["--gpus", "1", "--steps", "1", "--warmup", "0"],
               env={"WORLD_SIZE": "2", "RANK": "0", "LOCAL_RANK": "0"})
    assert r.returncode == 2 and "differs from the launcher's WORLD_SIZE 2" in r.stderr, r.stderr[-500:]
