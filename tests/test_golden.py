"""The fixtures under tests/golden (CPU only): Philox4x32-10's published
known-answer vectors against both the oracle's generator and the stored
text, and the oracle's state after a few steps of two seeded scenes against
the values tests/golden/make_golden.py stored from it (any change of the
oracle's arithmetic shows here)."""
import os

import numpy as np
import pytest

from oracle import frontend as F

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _rows(name):
    with open(os.path.join(HERE, name)) as f:
        return [line.split() for line in f if line.strip() and not line.startswith("#")]


def test_philox_known_answer_vectors():
    rows = _rows("philox4x32_10_kat.txt")
    assert len(rows) == 3
    for r in rows:
        w = [int(x, 16) for x in r]
        assert F.philox4x32_10(w[0:4], w[4:6]) == tuple(w[6:10])


@pytest.mark.parametrize("name", ["oracle_plain_square_seed0_10steps", "oracle_urban_block_seed1_env0_8steps",
                                  "oracle_urban_block_seed2_env0_8steps_vd"])
def test_oracle_reproduces_its_fixture(name):
    import importlib.util

    spec = importlib.util.spec_from_file_location("make_golden", os.path.join(HERE, "make_golden.py"))
    mg = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mg)
    make, steps, _ = mg.CASES[name]
    stored = np.array([[float(x) for x in r] for r in _rows(name + ".txt")])
    assert np.array_equal(mg.run(make(), steps), stored)
