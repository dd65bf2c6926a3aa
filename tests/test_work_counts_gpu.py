"""The kernels' own work counters (CROWD_FLAG_COUNT_WORK), which the
benchmark's roofline operation count is built from, against the oracle's
counts of the same units on the same states (teacher forcing).

Exact: agent updates, pairs within R (the FP64 key decides admission on both
sides), agent lines (the neighbour lists are bit-exact) and segment lines.
The LP's counts (line checks follow from the lines; violated lines and the
earlier lines their 1D solves scan; infeasible LPs) are decided in FP32 on
the GPU and FP64 in the oracle, so a violation test within rounding of zero
can go either way: held within 1 %."""
import numpy as np
import pytest

import oracle
from paper_2505_00690_gb300 import scenes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2505_00690_gb300 import build

    build.build()


@pytest.mark.parametrize("case", ["urban_resident", "urban_tiled", "dense_tiled"])
def test_kernel_work_counts_equal_oracle_counts(case):
    from paper_2505_00690_gb300 import crowd as cw

    if case.startswith("urban"):
        sc = scenes.urban_block(5, n_envs=8, steps=6)
    else:
        sc = scenes.dense_crowd(2, n_envs=1, n_peds=3000, side=40.0, n_segs=30, steps=6)
    flags = cw.CROWD_FLAG_COUNT_WORK | (cw.CROWD_FLAG_FORCE_TILED if case.endswith("tiled") else 0)
    cr = cw.Crowd(sc, flags=flags)
    o = oracle.OracleScene(sc)
    S = sc.state().astype(np.float32)
    ow = {}
    for k in range(6):
        rv = sc.robot_vel_at(k).astype(np.float32) if sc.robot_vel is not None else None
        cr.set_state(S)
        cr.step(None if rv is None else rv[None], n_steps=1)
        po, vo, _, _ = o.step(S[:, :2], S[:, 2:], rv, threads=8, work=ow)
        S = np.concatenate([po, vo], 1).astype(np.float32)
    w = cr.work()
    cr.close()
    print(case, "gpu", w, "oracle", ow)
    for key in ("agent_steps", "pairs_in_range", "agent_lines", "obstacle_lines", "lp_checks"):
        assert w[key] == ow[key], key
    for key in ("lp_solves", "lp_solve_lines", "fallbacks"):
        assert abs(w[key] - ow[key]) <= 0.01 * ow[key] + 2, key
    assert w["candidates"] >= w["pairs_in_range"]  # the cell search tests a superset of the pairs in range
