"""Continuous-batching server (crowd_server_*): admission, batching, results.

GPU tests check that every request's final state is bit-identical to the
same request stepped alone by a batch handle, whatever else shares the
device, and that the memory budget bounds what is admitted at once.
"""
import ctypes as C

import numpy as np
import pytest

from paper_2505_00690_gb300 import build as B
from paper_2505_00690_gb300 import crowd as cw
from paper_2505_00690_gb300 import scenes


def _params(K=10):
    return cw.crowd_params(2.0, 2.0, 5.0, K, 0.5, 0)


def test_server_rejects_bad_config():
    B.build()
    from paper_2505_00690_gb300 import serve

    L = serve._lib()
    h = C.c_void_p()
    p = _params()
    for cfg in [serve.crowd_server_config(0, 128, 10, 100, 1 << 20, 10),
                serve.crowd_server_config(4, 4096, 10, 100, 1 << 20, 10),
                serve.crowd_server_config(4, 128, 10, 0, 1 << 20, 10),
                serve.crowd_server_config(4, 128, 10, 100, 1 << 20, 0)]:
        assert L.crowd_server_create(C.byref(p), C.c_float(0.1), C.byref(cfg), None, C.byref(h)) == cw.CROWD_EINVAL
    cfg = serve.crowd_server_config(4, 128, 10, 100, 1 << 20, 10)
    assert L.crowd_server_create(C.byref(p), C.c_float(0.0), C.byref(cfg), None, C.byref(h)) == cw.CROWD_EINVAL
    bad = cw.crowd_params(2.0, 2.0, 5.0, 40, 0.5, 0)
    assert L.crowd_server_create(C.byref(bad), C.c_float(0.1), C.byref(cfg), None, C.byref(h)) == cw.CROWD_EINVAL


@pytest.fixture(scope="module")
def gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    B.build()


def _alone(scene, steps):
    h = cw.Crowd(scene, flags=0)
    h.step(n_steps=steps)
    out = h.state()
    h.close()
    return out


@pytest.mark.gpu
def test_results_equal_alone_and_in_the_mix(gpu):
    from paper_2505_00690_gb300 import serve

    reqs = scenes.serving_stream(seed=3, rate=400.0, duration_s=0.2, n_hi=600, steps_lo=20, steps_hi=140)
    assert len(reqs) >= 20
    sc0 = reqs[0].scene
    out = serve.run_stream(reqs, cw.params_for(sc0), sc0.dt, chunk_steps=25, max_slots=64, keep_results=True)
    assert out["max_live"] > 1  # requests really shared the device
    for k, r in enumerate(reqs):
        assert np.array_equal(out["results"][k], _alone(r.scene, r.steps)), k


@pytest.mark.gpu
def test_memory_budget_limits_admission(gpu):
    from paper_2505_00690_gb300 import serve

    reqs = scenes.serving_stream(seed=4, rate=1000.0, duration_s=0.05, n_lo=200, n_hi=200, steps_lo=60, steps_hi=60,
                                 max_polys=0)
    sc0 = reqs[0].scene
    per_req = 200 * (16 * 2 + 8 + 4) + 8 * 60 + 4 * (1 + 0)
    srv = serve.Server(cw.params_for(sc0), sc0.dt, max_slots=64, max_segments=1, max_steps=60,
                       mem_budget=3 * per_req + 100, chunk_steps=20)
    ids = [srv.submit(r.scene, n_steps=r.steps) for r in reqs]
    live, _ = srv.tick()
    assert live == 3
    info = srv.info()
    assert info["live"] == 3 and info["waiting"] == len(reqs) - 3
    done = {}
    while len(done) < len(ids):
        live, _ = srv.tick()
        assert live <= 3
        for k, rid in enumerate(ids):
            if k in done:
                continue
            st, res = srv.poll(rid, 200)
            if st == serve.CROWD_REQ_DONE:
                done[k] = res
    for k, r in enumerate(reqs):
        assert np.array_equal(done[k], _alone(r.scene, r.steps))
    srv.close()


@pytest.mark.gpu
def test_robot_commands_per_request(gpu):
    from paper_2505_00690_gb300 import serve

    sc = scenes.urban_block(2, n_envs=2, n_peds=40, steps=30)
    srv = serve.Server(cw.params_for(sc), sc.dt, max_slots=4, max_agents=64, max_segments=64, max_steps=30,
                       chunk_steps=7)
    ids = [srv.submit(sc.subset([e]), robot_vel=sc.robot_vel[:, e], n_steps=30) for e in range(2)]
    res = {}
    while len(res) < 2:
        srv.tick()
        for k, rid in enumerate(ids):
            if k not in res:
                st, out = srv.poll(rid, 41)
                if st == serve.CROWD_REQ_DONE:
                    res[k] = out
    batch = cw.Crowd(sc, flags=0)
    batch.step(sc.robot_vel[:30], n_steps=30)
    ref = batch.state()
    assert np.array_equal(np.concatenate([res[0], res[1]]), ref)
    srv.close()
