"""Occupancy-map front end on the GPU against its oracle (bit-exact), through
the C ABI (crowd_map_segments, crowd_map_sample)."""
import ctypes as C

import numpy as np
import pytest

from oracle import frontend as F

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2505_00690_gb300 import build

    build.build()
    return t


def _blobs(rng, H, W, frac):
    occ = (rng.random((H, W)) < frac).astype(np.uint8)
    # grow a few rectangles so that long runs appear
    for _ in range(max(1, H * W // 400)):
        y, x = rng.integers(0, H), rng.integers(0, W)
        occ[y:y + rng.integers(1, 8), x:x + rng.integers(1, 12)] = 1
    return occ


@pytest.mark.parametrize("shape,frac,closed", [((1, 1), 0.0, True), ((1, 1), 1.0, False), ((1, 37), 0.3, True),
                                               ((29, 1), 0.3, False), ((61, 97), 0.15, True),
                                               ((61, 97), 0.15, False), ((200, 300), 0.05, True),
                                               ((64, 64), 1.0, True), ((64, 64), 0.0, False)])
def test_segments_bit_exact(torch, shape, frac, closed):
    from paper_2505_00690_gb300 import frontend

    rng = np.random.default_rng(sum(shape))
    occ = _blobs(rng, *shape, frac) if 0 < frac < 1 else np.full(shape, int(frac), np.uint8)
    cell, x0, y0 = 0.37, -12.5, 3.25
    ref = F.map_segments(occ, cell, x0, y0, closed)
    got = frontend.map_segments(torch.from_numpy(occ).cuda(), cell, x0, y0, closed).cpu().numpy()
    assert got.shape == ref.shape
    assert np.array_equal(got.view(np.uint32), ref.view(np.uint32))


@pytest.mark.parametrize("clearance,closed", [(0, True), (1, True), (2, False), (3, True)])
def test_sample_bit_exact(torch, clearance, closed):
    from paper_2505_00690_gb300 import frontend

    rng = np.random.default_rng(7 + clearance)
    occ = _blobs(rng, 83, 71, 0.08)
    ref, M = F.map_sample(occ, 0.5, 1.0, -4.0, closed, clearance, seed=0xDEADBEEF12345, stream=2, n=3000)
    got, m = frontend.map_sample(torch.from_numpy(occ).cuda(), 0.5, 3000, 1.0, -4.0, closed, clearance,
                                 seed=0xDEADBEEF12345, stream_id=2)
    assert m == M > 0
    assert np.array_equal(got.cpu().numpy().view(np.uint32), ref.view(np.uint32))


def test_errors_and_limits(torch):
    from paper_2505_00690_gb300 import crowd as cw
    from paper_2505_00690_gb300 import frontend

    L = frontend._lib()
    occ = torch.zeros((4, 5), dtype=torch.uint8, device="cuda")
    n = C.c_int32()
    out = torch.empty((2, 4), device="cuda")
    # a closed empty map has 4 walls: 2 slots are too few; the count comes back
    st = L.crowd_map_segments(occ.data_ptr(), 5, 4, 1.0, 0.0, 0.0, 1, 2, out.data_ptr(), C.byref(n), None)
    assert st == cw.CROWD_EINVAL and n.value == 4
    assert L.crowd_map_segments(occ.data_ptr(), 0, 4, 1.0, 0.0, 0.0, 1, 2, out.data_ptr(), C.byref(n),
                                None) == cw.CROWD_EINVAL
    assert L.crowd_map_segments(occ.data_ptr(), 5, 4, -1.0, 0.0, 0.0, 1, 2, out.data_ptr(), C.byref(n),
                                None) == cw.CROWD_EINVAL
    m = C.c_int32()
    pts = torch.empty((3, 2), device="cuda")
    st = L.crowd_map_sample(occ.data_ptr(), 5, 4, 1.0, 0.0, 0.0, 1, 2, 1, 0, 3, pts.data_ptr(), C.byref(m), None)
    assert st == cw.CROWD_EINVAL and m.value == 0  # clearance 2 leaves no cell of a 5 x 4 walled map
    st = L.crowd_map_sample(occ.data_ptr(), 5, 4, 1.0, 0.0, 0.0, 1, 1, 1, 0, 0, None, C.byref(m), None)
    assert st == cw.CROWD_OK and m.value == 6


def test_front_end_feeds_the_crowd_step(torch):
    """A walled map with two obstacle blocks: segments and sampled starts and
    goals from the front end, stepped by the crowd library and by the oracle
    (teacher forcing, 30 steps, 1e-4 m/s)."""
    import oracle
    from paper_2505_00690_gb300 import crowd as cw
    from paper_2505_00690_gb300 import frontend
    from paper_2505_00690_gb300.scenes import Scene

    occ = np.zeros((40, 40), np.uint8)
    occ[10:18, 8:20] = 1
    occ[24:30, 22:34] = 1
    d = torch.from_numpy(occ).cuda()
    segs = frontend.map_segments(d, 0.5, 0.0, 0.0, closed=True).cpu().numpy()
    n = 60
    starts, _ = frontend.map_sample(d, 0.5, n, closed=True, clearance=1, seed=11, stream_id=0)
    goals, _ = frontend.map_sample(d, 0.5, n, closed=True, clearance=1, seed=11, stream_id=1)
    starts, goals = starts.cpu().numpy(), goals.cpu().numpy()
    sc = Scene(name="map", agents_per_env=np.array([n], np.int32), radius=np.full(n, 0.2, np.float32),
               max_speed=np.full(n, 1.3, np.float32), pref_speed=np.full(n, 1.3, np.float32), pos=starts,
               vel=np.zeros((n, 2), np.float32), goal=goals, robot_index=np.array([-1], np.int32),
               segs_per_env=np.array([len(segs)], np.int32), segments=segs, tau=2.0, tau_obst=2.0,
               neighbor_dist=5.0, max_neighbors=10, dt=0.1)
    cr = cw.Crowd(sc, flags=cw.CROWD_FLAG_EXPORT_NEIGHBORS)
    o = oracle.OracleScene(sc)
    S = sc.state()
    worst = 0.0
    for _ in range(30):
        cr.set_state(S)
        cr.step(n_steps=1)
        G = cr.state()
        po, vo, nb, st = o.step(S[:, :2], S[:, 2:])
        assert np.array_equal(cr.neighbors(), nb)
        worst = max(worst, float(np.abs(G[:, 2:] - vo).max()))
        S = np.concatenate([po, vo], 1).astype(np.float32)
    cr.close()
    assert worst <= 1e-4, worst


def test_map_to_crowd_pipeline(torch):
    """The paper's pipeline on one environment (Sec. 3.2): an occupancy map
    -> its boundary segments and start points sampled on free cells with a
    clearance (front end) -> a crowd whose goals are drawn inside the step
    from a pool of free-cell samples -> 200 steps: every agent's centre stays
    on free ground, goals are drawn, and the run equals single steps."""
    from paper_2505_00690_gb300 import crowd as cw
    from paper_2505_00690_gb300 import frontend as FE
    from paper_2505_00690_gb300.scenes import Scene

    H, W, cell = 40, 40, 0.5
    occ = np.zeros((H, W), np.uint8)
    occ[6:12, 8:22] = 1
    occ[20:34, 26:31] = 1
    occ[25:29, 4:16] = 1
    occ_t = torch.from_numpy(occ).cuda()
    segs = FE.map_segments(occ_t, cell).cpu().numpy()
    starts = FE.map_sample(occ_t, cell, 48, clearance=2, seed=11, stream_id=0)[0].cpu().numpy()
    pool = FE.map_sample(occ_t, cell, 200, clearance=2, seed=11, stream_id=1)[0].cpu().numpy()
    n = len(starts)
    sc = Scene(name="map", agents_per_env=np.array([n], np.int32), radius=np.full(n, 0.2, np.float32),
               max_speed=np.full(n, 1.2, np.float32), pref_speed=np.full(n, 1.2, np.float32), pos=starts,
               vel=np.zeros((n, 2), np.float32), goal=starts.copy(), robot_index=np.array([-1], np.int32),
               segs_per_env=np.array([len(segs)], np.int32), segments=segs.astype(np.float32), tau=2.0,
               tau_obst=2.0, neighbor_dist=3.0, max_neighbors=10, dt=0.1)
    outs = []
    for chunks in ((200,), (1,) * 200):
        cr = cw.Crowd(sc)
        cr.set_goal_pool(np.array([0, len(pool)], np.int32), pool, seed=5)
        for k in chunks:
            cr.step(n_steps=k)
        outs.append((cr.state(), cr.goal_index()))
        cr.close()
    (S, drawn), (S1, drawn1) = outs
    assert np.array_equal(S, S1) and np.array_equal(drawn, drawn1)
    assert drawn.sum() > n  # every agent arrives at least about once and draws again
    cx = np.floor(S[:, 0] / cell).astype(int)
    cy = np.floor(S[:, 1] / cell).astype(int)
    inside = (cx >= 0) & (cx < W) & (cy >= 0) & (cy < H)
    assert inside.all()
    assert (occ[cy, cx] == 0).all()
