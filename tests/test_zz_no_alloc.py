"""crowd_step_noalloc, the allocation-free entry point, against crowd_step
and the FP64 oracle.

Callers that cannot allocate device memory (inside another framework's
memory pool, under a fixed budget, in loops that must not allocate after
start-up) use crowd_step_noalloc, whose scratch lives in a fixed device array
of the library.  Here it is called through the C ABI twice in a row (the
second call starting from the first one's output) and compared, call by
call, with the regular handle-based crowd_step on the same environment and
with the oracle stepped from the same FP32 state (1e-4 m/s).
"""
import ctypes as C

import numpy as np
import pytest

import oracle
from paper_2505_00690_gb300 import scenes
from paper_2505_00690_gb300.scenes import Scene

pytestmark = pytest.mark.gpu

VEL_TOL = 1e-4


@pytest.fixture(scope="module")
def lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2505_00690_gb300 import build
    from paper_2505_00690_gb300 import crowd as cw

    build.build()
    L = cw.load()
    vp = C.c_void_p
    L.crowd_step_noalloc.argtypes = [C.c_int32, vp, vp, vp, vp, C.c_int32, C.c_int32, vp, vp,
                                     C.POINTER(cw.crowd_params), C.c_float, vp]
    L.crowd_step_noalloc.restype = C.c_int
    return L


def _box(sc):
    pts = np.concatenate([sc.pos, sc.goal, sc.segments[:, :2], sc.segments[:, 2:]]) if sc.segments.size else \
        np.concatenate([sc.pos, sc.goal])
    lo, hi = pts.min(0) - 1.0, pts.max(0) + 1.0
    return np.array([lo[0], lo[1], hi[0], hi[1]], np.float32)


def _shifted(sc, dx, dy):
    """The scene moved by (dx, dy): positions, goals and segments."""
    import dataclasses

    off = np.array([dx, dy], np.float32)
    segs = sc.segments.reshape(-1, 4) + np.concatenate([off, off])
    return dataclasses.replace(sc, pos=(sc.pos + off).astype(np.float32), goal=(sc.goal + off).astype(np.float32),
                               segments=segs.astype(np.float32))


@pytest.mark.parametrize("which", ["urban_block", "dense_patch", "urban_block_far"])
def test_noalloc_matches_crowd_step_two_calls(lib, which):
    """urban_block_far: the block 12 km east and 7 km south of the origin,
    where FP32 coordinates step by 1 mm, so that the per-cell segment lists
    (built on the GPU relative to the grid origin) must still hold every
    segment within reach of any point of the cell."""
    import torch

    from paper_2505_00690_gb300 import crowd as cw

    if which == "urban_block":
        sc = scenes.urban_block(7, n_envs=1, steps=2)
    elif which == "urban_block_far":
        sc = _shifted(scenes.urban_block(7, n_envs=1, steps=2), 12000.0, -7000.0)
    else:
        sc = scenes.dense_crowd(3, n_envs=1, n_peds=3000, side=40.0, n_segs=30, steps=2)
    n = sc.n_agents
    robot = int(sc.robot_index[0])
    rv = sc.robot_vel[:2] if sc.robot_vel is not None else np.zeros((2, 1, 2), np.float32)

    # regular entry point: a handle, two calls of one step
    h = cw.Crowd(sc, flags=0)
    ref = []
    for k in range(2):
        h.step(rv[k:k + 1] if sc.robot_vel is not None else None, n_steps=1)
        ref.append(h.state())
    h.close()

    # allocation-free entry point: same inputs, device buffers owned by the caller
    dev = torch.device("cuda")
    state = torch.from_numpy(sc.state()).to(dev)
    par = torch.from_numpy(np.stack([sc.radius, sc.max_speed, sc.pref_speed, np.zeros(n, np.float32)], 1)).to(dev)
    goal = torch.from_numpy(np.ascontiguousarray(sc.goal)).to(dev)
    segs = torch.from_numpy(np.ascontiguousarray(sc.segments.reshape(-1, 4))).to(dev) if sc.segments.size else None
    box = _box(sc)
    params = cw.params_for(sc)
    o = oracle.OracleScene(sc)
    outs = [torch.empty_like(state), torch.empty_like(state)]
    src = state
    for k in range(2):
        if robot >= 0:
            src[robot, 2:] = torch.from_numpy(rv[k, 0]).to(dev)  # the robot moves with the velocity in its slot
        st = lib.crowd_step_noalloc(n, src.data_ptr(), outs[k].data_ptr(), par.data_ptr(), goal.data_ptr(), robot,
                                    int(sc.segs_per_env[0]), None if segs is None else segs.data_ptr(),
                                    box.ctypes.data, C.byref(params), C.c_float(sc.dt), None)
        assert st == 0, lib.crowd_last_error().decode()
        torch.cuda.synchronize()
        got = outs[k].cpu().numpy()
        # positions: dt * 1e-4 plus a few units in the last place of the coordinate
        ptol = sc.dt * VEL_TOL + 1e-5 + 4 * np.spacing(np.abs(got[:, :2]).astype(np.float32)).astype(np.float64)
        assert np.abs(got[:, 2:] - ref[k][:, 2:]).max() <= VEL_TOL, k
        assert np.all(np.abs(got[:, :2] - ref[k][:, :2]) <= ptol), k
        # the oracle from the same FP32 state (the robot's slot holds its command)
        S = src.cpu().numpy()
        rvk = S[robot, 2:][None] if robot >= 0 else None
        po, vo, _, _ = o.step(S[:, :2], S[:, 2:], rvk, threads=4)
        assert np.abs(got[:, 2:].astype(np.float64) - vo).max() <= VEL_TOL, k
        assert np.all(np.abs(got[:, :2].astype(np.float64) - po) <= ptol), k
        src = outs[k].clone()


def test_noalloc_rejects_oversize(lib):
    from paper_2505_00690_gb300 import crowd as cw

    params = cw.crowd_params(2.0, 2.0, 5.0, 10, 0.5, 0)
    box = np.array([0, 0, 10, 10], np.float32)
    st = lib.crowd_step_noalloc(70000, 1, 1, 1, 1, -1, 0, None, box.ctypes.data, C.byref(params), C.c_float(0.1),
                                None)
    assert st == cw.CROWD_EINVAL and "allocation-free" in lib.crowd_last_error().decode()
    wide = np.array([0, 0, 1e6, 10], np.float32)  # 256 x 1 cells: fine; the agent limit still applies
    st = lib.crowd_step_noalloc(0, None, None, None, None, -1, 0, None, wide.ctypes.data, C.byref(params),
                                C.c_float(0.1), None)
    assert st == 0


def _noalloc_call(lib, sc, box, state=None):
    """One call on scene `sc` (one environment) with device copies of its
    inputs; returns (status, message, output state)."""
    import torch

    from paper_2505_00690_gb300 import crowd as cw

    dev = torch.device("cuda")
    n = sc.n_agents
    state = torch.from_numpy(sc.state() if state is None else state).to(dev)
    par = torch.from_numpy(np.stack([sc.radius, sc.max_speed, sc.pref_speed, np.zeros(n, np.float32)], 1)).to(dev)
    goal = torch.from_numpy(np.ascontiguousarray(sc.goal)).to(dev)
    segs = torch.from_numpy(np.ascontiguousarray(sc.segments.reshape(-1, 4))).to(dev)
    out = torch.empty_like(state)
    params = cw.params_for(sc)
    st = lib.crowd_step_noalloc(n, state.data_ptr(), out.data_ptr(), par.data_ptr(), goal.data_ptr(), -1,
                                int(sc.segs_per_env[0]), segs.data_ptr(), np.asarray(box, np.float32).ctypes.data,
                                C.byref(params), C.c_float(sc.dt), None)
    torch.cuda.synchronize()
    return st, lib.crowd_last_error().decode(), out.cpu().numpy()


def _ring_scene():
    """Two agents; 80 short walls on a 2 m ring round the first one, more
    than an agent's segment line buffer holds (CROWD_MAX_OBSTACLE_LINES)."""
    ang = np.linspace(0, 2 * np.pi, 80, endpoint=False)
    segs = np.array([(2 * np.cos(a), 2 * np.sin(a), 2 * np.cos(a + 0.01), 2 * np.sin(a + 0.01)) for a in ang],
                    np.float32)
    pos = np.array([[0.0, 0.0], [12.0, 12.0]], np.float32)
    n = 2
    return Scene(name="ring", agents_per_env=np.array([n], np.int32), pos=pos, vel=np.zeros((n, 2), np.float32),
                 goal=np.array([[0.5, 0.0], [13.0, 12.0]], np.float32), radius=np.full(n, 0.3, np.float32),
                 max_speed=np.full(n, 1.4, np.float32), pref_speed=np.full(n, 1.4, np.float32),
                 robot_index=np.array([-1], np.int32), segs_per_env=np.array([len(segs)], np.int32), segments=segs,
                 tau=2.0, tau_obst=2.0, neighbor_dist=5.0, max_neighbors=10, dt=0.1, robot_vel=None, steps=2)


def test_noalloc_reports_segment_overflow(lib):
    """More segments in one agent's reach than its line buffer holds: the call
    keeps the nearest ones and returns CROWD_EDEVICE, like crowd_step's next
    synchronising call; the next call, with the agent away from the ring,
    starts from a clear error word and succeeds."""
    from paper_2505_00690_gb300 import crowd as cw

    sc = _ring_scene()
    box = [-3.0, -3.0, 25.0, 25.0]
    st, msg, out = _noalloc_call(lib, sc, box)
    assert st == cw.CROWD_EDEVICE and "segments in reach" in msg, msg
    far = sc.state().copy()
    far[0, :2] = [20.0, 20.0]
    st, msg, out = _noalloc_call(lib, sc, box, far)
    assert st == 0, msg
    assert np.all(np.isfinite(out))


def test_noalloc_rejects_segment_outside_box(lib):
    """The grid covers the caller's box; a segment outside it could be missed
    by an agent clamped into a border cell, so the call refuses it."""
    from paper_2505_00690_gb300 import crowd as cw

    sc = _ring_scene()
    st, msg, _ = _noalloc_call(lib, sc, [-1.0, -1.0, 25.0, 25.0])  # the ring reaches x = -2
    assert st == cw.CROWD_EINVAL and "outside the box" in msg, msg
