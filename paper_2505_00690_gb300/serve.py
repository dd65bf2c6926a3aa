"""Serving driver: a Poisson stream of rollout requests through the library's
continuous-batching server (crowd_server_* in include/crowd.h).

Marshalling and timing only: admission, slotting, batched stepping and
result copies all happen in the C++/CUDA server.  Latency of a request is
the wall time from its arrival to the moment its final state is on the host.
"""
from __future__ import annotations

import ctypes as C
import time

import numpy as np

from . import crowd as cw

CROWD_REQ_QUEUED, CROWD_REQ_RUNNING, CROWD_REQ_DONE = 0, 1, 2


class crowd_server_config(C.Structure):
    _fields_ = [("max_slots", C.c_int32), ("max_agents", C.c_int32), ("max_segments", C.c_int32),
                ("max_steps", C.c_int32), ("mem_budget", C.c_size_t), ("chunk_steps", C.c_int32)]


class crowd_request(C.Structure):
    _fields_ = [("n_agents", C.c_int32), ("radii", C.c_void_p), ("max_speeds", C.c_void_p),
                ("pref_speeds", C.c_void_p), ("init_pos", C.c_void_p), ("goals", C.c_void_p),
                ("robot_index", C.c_int32), ("n_segments", C.c_int32), ("segments", C.c_void_p),
                ("n_steps", C.c_int32), ("robot_vel", C.c_void_p)]


class crowd_server_stats(C.Structure):
    _fields_ = [("waiting", C.c_int32), ("live", C.c_int32), ("bytes_in_use", C.c_size_t)]


def _lib():
    L = cw.load()
    if not getattr(L, "_server_bound", False):
        vp, i32 = C.c_void_p, C.c_int32
        L.crowd_server_create.argtypes = [vp, C.c_float, vp, vp, C.POINTER(vp)]
        L.crowd_server_submit.argtypes = [vp, vp, C.POINTER(C.c_int64)]
        L.crowd_server_tick.argtypes = [vp, C.POINTER(i32), C.POINTER(i32)]
        L.crowd_server_poll.argtypes = [vp, C.c_int64, vp, C.POINTER(i32)]
        L.crowd_server_info.argtypes = [vp, vp]
        L.crowd_server_finished.argtypes = [vp, vp, i32, C.POINTER(i32)]
        L.crowd_server_destroy.argtypes = [vp]
        for n in ("crowd_server_create", "crowd_server_submit", "crowd_server_tick", "crowd_server_poll",
                  "crowd_server_info", "crowd_server_destroy", "crowd_server_finished"):
            getattr(L, n).restype = C.c_int
        L._server_bound = True
    return L


class Server:
    """One continuous-batching server (see crowd_server_create)."""

    def __init__(self, params, dt, max_slots=1024, max_agents=2048, max_segments=360, max_steps=1000,
                 mem_budget=4 << 30, chunk_steps=50, stream=None):
        L = _lib()
        self.cfg = crowd_server_config(max_slots, max_agents, max_segments, max_steps, mem_budget, chunk_steps)
        self.h = C.c_void_p()
        self.params = params
        cw._check(L.crowd_server_create(C.byref(params), C.c_float(dt), C.byref(self.cfg), C.c_void_p(stream or 0),
                                        C.byref(self.h)))
        self._keep = {}

    def submit(self, scene, robot_vel=None, n_steps=None):
        """Submit a one-environment Scene; returns the request id."""
        assert scene.n_envs == 1
        f = lambda a: np.ascontiguousarray(a, np.float32)
        arrs = dict(r=f(scene.radius), v=f(scene.max_speed), s=f(scene.pref_speed), p=f(scene.pos), g=f(scene.goal),
                    seg=f(scene.segments.reshape(-1, 4)) if scene.segments.size else None,
                    rv=None if robot_vel is None else f(robot_vel))
        ptr = lambda a: None if a is None else a.ctypes.data
        steps = int(n_steps if n_steps is not None else scene.steps)
        req = crowd_request(scene.n_agents, ptr(arrs["r"]), ptr(arrs["v"]), ptr(arrs["s"]), ptr(arrs["p"]),
                            ptr(arrs["g"]), int(scene.robot_index[0]), int(scene.segs_per_env[0]), ptr(arrs["seg"]),
                            steps, ptr(arrs["rv"]))
        rid = C.c_int64()
        cw._check(_lib().crowd_server_submit(self.h, C.byref(req), C.byref(rid)))
        return rid.value

    def tick(self):
        live, fin = C.c_int32(), C.c_int32()
        cw._check(_lib().crowd_server_tick(self.h, C.byref(live), C.byref(fin)))
        return live.value, fin.value

    def poll(self, rid, n_agents=None):
        """(status, state or None)."""
        st = C.c_int32()
        out = None if n_agents is None else np.empty((n_agents, 4), np.float32)
        cw._check(_lib().crowd_server_poll(self.h, C.c_int64(rid), None if out is None else out.ctypes.data,
                                           C.byref(st)))
        return st.value, (out if st.value == CROWD_REQ_DONE else None)

    def finished(self, cap=4096):
        """Ids of requests completed since the last call."""
        ids = np.empty(cap, np.int64)
        n = C.c_int32()
        cw._check(_lib().crowd_server_finished(self.h, ids.ctypes.data, cap, C.byref(n)))
        return ids[:n.value].tolist()

    def info(self):
        s = crowd_server_stats()
        cw._check(_lib().crowd_server_info(self.h, C.byref(s)))
        return dict(waiting=s.waiting, live=s.live, bytes_in_use=s.bytes_in_use)

    def close(self):
        if self.h is not None and self.h.value:
            cw._check(_lib().crowd_server_destroy(self.h))
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def run_stream(requests, params, dt, chunk_steps=50, max_slots=1024, mem_budget=4 << 30, keep_results=False,
               time_scale=1.0):
    """Replay a request stream (scenes.serving_stream) in real time.

    Returns latency percentiles (seconds), throughput (agent-steps/s over the
    wall time from the first arrival to the last completion) and, if asked,
    every result."""
    srv = Server(params, dt, max_slots=max_slots, max_segments=max(1, max(int(r.scene.segs_per_env[0]) for r in requests)),
                 max_steps=max(r.steps for r in requests), mem_budget=mem_budget, chunk_steps=chunk_steps)
    order = sorted(range(len(requests)), key=lambda k: requests[k].arrival_s)
    pending = {}
    latency = np.zeros(len(requests))
    results = {}
    nxt = 0
    t0 = time.perf_counter()
    done = 0
    max_live = 0
    while done < len(requests):
        now = (time.perf_counter() - t0) / time_scale
        while nxt < len(order) and requests[order[nxt]].arrival_s <= now:
            k = order[nxt]
            pending[srv.submit(requests[k].scene, n_steps=requests[k].steps)] = k
            nxt += 1
        live, _ = srv.tick()
        max_live = max(max_live, live)
        for rid in srv.finished():
            k = pending.pop(rid)
            latency[k] = (time.perf_counter() - t0) / time_scale - requests[k].arrival_s
            st, out = srv.poll(rid, requests[k].scene.n_agents if keep_results else None)
            if keep_results:
                results[k] = out
            done += 1
        if not pending and nxt < len(order):
            # idle until the next arrival
            wait = requests[order[nxt]].arrival_s - (time.perf_counter() - t0) / time_scale
            if wait > 0:
                time.sleep(min(wait * time_scale, 0.05))
    wall = time.perf_counter() - t0
    srv.close()
    work = sum(r.scene.n_agents * r.steps for r in requests)
    return dict(p50_s=float(np.percentile(latency, 50)), p99_s=float(np.percentile(latency, 99)),
                mean_s=float(latency.mean()), requests=len(requests), agent_steps=int(work),
                wall_s=wall, agent_steps_per_s=work / wall, max_live=max_live, results=results if keep_results else None)


def run_plain(requests, params, dt):
    """The plain form on the same requests: one request at a time, one
    environment per launch and one step per launch (no batching, no
    persistence).  Returns agent-steps/s."""
    t0 = time.perf_counter()
    work = 0
    for r in requests:
        h = cw.Crowd(r.scene, flags=0)
        for _ in range(r.steps):
            h.step(n_steps=1)
        h.state()
        h.close()
        work += r.scene.n_agents * r.steps
    return work / (time.perf_counter() - t0)
