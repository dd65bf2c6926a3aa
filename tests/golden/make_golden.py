"""Write the oracle fixtures of this folder (run from the repository root:
``python tests/golden/make_golden.py``).  Only the oracle and the seeded scene
generator are called; the fixtures pin the oracle against later changes of
its arithmetic (a change that moves them must say, in its commit, which
reading of the paper justifies it)."""
import dataclasses
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_2505_00690_gb300 import scenes  # noqa: E402

CASES = {
    # name: (scene, steps, description)
    "oracle_plain_square_seed0_10steps": (lambda: scenes.plain_square(0), 10,
                                          "plain square, seed 0: 32 agents, 20 x 20 m, no obstacles"),
    "oracle_urban_block_seed1_env0_8steps": (lambda: scenes.urban_block(1, n_envs=1, steps=8), 8,
                                             "urban block, seed 1, one environment: 128 pedestrians, a robot, 36 walls"),
    "oracle_urban_block_seed2_env0_8steps_vd": (
        lambda: dataclasses.replace(scenes.urban_block(2, n_envs=1, steps=8), segment_mode=1), 8,
        "urban block, seed 2, one environment, velocity-dependent segment half-planes"),
}


def run(scene, steps):
    o = oracle.OracleScene(scene)
    pos, vel = scene.pos.astype(np.float64), scene.vel.astype(np.float64)
    for k in range(steps):
        pos, vel, _, _ = o.step(pos, vel, scene.robot_vel_at(k))
    return np.concatenate([pos, vel], 1)


def main():
    for name, (make, steps, desc) in CASES.items():
        out = run(make(), steps)
        with open(os.path.join(HERE, name + ".txt"), "w") as f:
            f.write(f"# FP64 oracle state after {steps} steps: {desc}.\n")
            f.write("# Written by tests/golden/make_golden.py from the oracle alone; rows px py vx vy.\n")
            for row in out:
                f.write(" ".join(repr(float(x)) for x in row) + "\n")


if __name__ == "__main__":
    main()
