"""Host-side logic of the library, compiled with g++ and run without a GPU:
the tile shape of the tiled update kernel (hand-derived cases) and the
episode schedule (against the oracle's episode_restarts)."""
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CUDA = os.environ.get("CUDA_HOME", "/usr/local/cuda")


@pytest.fixture(scope="module")
def probe(tmp_path_factory):
    if shutil.which("g++") is None or not os.path.exists(os.path.join(CUDA, "include", "cuda_runtime.h")):
        pytest.skip("g++ or the CUDA headers missing")
    exe = str(tmp_path_factory.mktemp("host") / "host_logic")
    r = subprocess.run(["g++", "-std=c++17", "-O1", "-I", os.path.join(CUDA, "include"),
                        "-I", os.path.join(ROOT, "paper_2505_00690_gb300", "csrc"),
                        os.path.join(HERE, "host", "host_logic.cpp"), "-o", exe, "-ldl"],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-3000:]
    return exe


def _run(exe, *args):
    r = subprocess.run([exe, *args], capture_output=True, text=True)
    assert r.returncode == 0
    return r.stdout.split("\n")


@pytest.mark.parametrize("n,W,H,expect", [
    (20000, 34, 34, (4, 3)),    # 17.3 agents a cell: 4 x 3 = 208 <= 230 < 4 x 4 = 277
    (20000, 68, 68, (7, 7)),    # cells of R/2: 4.3 a cell, 7 x 7 = 212
    (129, 10, 10, (8, 8)),      # sparse: the largest tile
    (100000, 20, 20, (1, 1)),   # 250 a cell: one cell per tile
    (920, 2, 2, (1, 1)),        # 230 a cell exactly still fits one round
    (1000, 2, 2, (1, 1)),       # more than 230 a cell: a single cell per tile all the same
])
def test_tile_choice(probe, n, W, H, expect):
    out = _run(probe, "tile", f"{n},{W},{H}")
    assert out[0] == f"tile {expect[0]} {expect[1]}"


def test_episode_schedule_matches_the_oracle(probe):
    steps = [0, 1, 3, 7]
    args = []
    cases = []
    for origin in (0, 5, -4):
        for t in range(0, 22):
            for L in steps:
                args += ["restart", f"{L},{origin + t},{origin}"]
                cases.append((L, t))
    out = _run(probe, *args)
    got = [int(l.split()[1]) for l in out if l.startswith("restart")]
    want = [int(oracle.episode_restarts(t, [L])[0]) for L, t in cases]
    assert got == want
