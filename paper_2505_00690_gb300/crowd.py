"""Thin Python binding of the crowd C ABI (include/crowd.h).

Argument marshalling only: every step of the crowd update runs in the CUDA
library ``_build/libcrowd.so``.  The functions keep the C names; ``Crowd``
wraps one handle.  Host arrays are numpy; device arrays are torch CUDA
tensors (torch supplies device memory and streams, nothing else).  There is no
CPU fallback: without the built library every call raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libcrowd.so")

CROWD_OK, CROWD_EINVAL, CROWD_ENOMEM, CROWD_ECUDA, CROWD_EDEVICE, CROWD_ESTATE = range(6)
CROWD_HOST, CROWD_DEVICE = 0, 1
CROWD_FLAG_EXPORT_NEIGHBORS = 1
CROWD_FLAG_STATS = 2
CROWD_FLAG_COUNT_WORK = 4
CROWD_FLAG_FORCE_TILED = 8
CROWD_FLAG_VELOCITY_SEGMENTS = 16
STATUS_NAMES = {0: "CROWD_OK", 1: "CROWD_EINVAL", 2: "CROWD_ENOMEM", 3: "CROWD_ECUDA", 4: "CROWD_EDEVICE",
                5: "CROWD_ESTATE"}

EXPORTED = ["crowd_create", "crowd_set_goals", "crowd_set_state", "crowd_step", "crowd_read_state",
            "crowd_read_neighbors", "crowd_read_stats", "crowd_read_work", "crowd_reset_stats", "crowd_synchronize",
            "crowd_destroy", "crowd_num_agents", "crowd_num_envs", "crowd_last_error", "crowd_abi_version",
            "crowd_get_tuning", "crowd_set_tuning", "crowd_autotune", "crowd_set_goal_queue",
            "crowd_read_goal_index", "crowd_set_vehicles", "crowd_vehicle_state", "crowd_set_episodes",
            "crowd_restart_envs", "crowd_set_goal_pool", "crowd_read_launches"]


class CrowdError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class crowd_params(C.Structure):
    _fields_ = [("time_horizon", C.c_float), ("time_horizon_obst", C.c_float), ("neighbor_dist", C.c_float),
                ("max_neighbors", C.c_int32), ("robot_responsibility", C.c_float), ("flags", C.c_int32)]


class crowd_env_stats(C.Structure):
    _fields_ = [("agent_collisions", C.c_int64), ("segment_collisions", C.c_int64), ("speed_sum", C.c_double),
                ("steps", C.c_int64)]


class crowd_work(C.Structure):
    _fields_ = [(n, C.c_uint64) for n in ("agent_steps", "candidates", "agent_lines", "obstacle_lines",
                                          "segment_tests", "lp_checks", "lp_solves", "lp_solve_lines",
                                          "fallbacks", "pairs_in_range")]


class crowd_tuning(C.Structure):
    _fields_ = [("block_threads", C.c_int32), ("coop_fallback", C.c_int32), ("cell_split", C.c_int32),
                ("lanes_per_agent", C.c_int32), ("agent_order", C.c_int32), ("tiled_queue", C.c_int32)]


_lib = None


def load(path: str = LIB_PATH):
    """Load libcrowd.so (raises if it was not built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"crowd CUDA library not built ({path}); run paper_2505_00690_gb300.build.build()")
    L = C.CDLL(path)
    vp, fp, ip, i32 = C.c_void_p, C.POINTER(C.c_float), C.POINTER(C.c_int32), C.c_int32
    L.crowd_create.argtypes = [i32, vp, vp, vp, vp, vp, vp, vp, vp, C.POINTER(crowd_params), vp, C.POINTER(vp)]
    L.crowd_set_goals.argtypes = [vp, vp, i32]
    L.crowd_set_goal_queue.argtypes = [vp, i32, vp, i32, i32]
    L.crowd_read_goal_index.argtypes = [vp, vp]
    L.crowd_set_episodes.argtypes = [vp, vp, vp, i32]
    L.crowd_restart_envs.argtypes = [vp, vp]
    L.crowd_set_goal_pool.argtypes = [vp, vp, vp, C.c_uint64]
    L.crowd_set_vehicles.argtypes = [vp, i32, vp, vp, i32, vp, vp, vp, vp, vp, C.c_float, C.c_float]
    L.crowd_vehicle_state.argtypes = [vp, i32, vp, vp]
    L.crowd_set_state.argtypes = [vp, vp, i32]
    L.crowd_step.argtypes = [vp, C.c_float, vp, i32, i32]
    L.crowd_read_state.argtypes = [vp, vp, i32]
    L.crowd_read_neighbors.argtypes = [vp, vp, i32]
    L.crowd_read_stats.argtypes = [vp, vp, vp]
    L.crowd_read_work.argtypes = [vp, vp]
    L.crowd_read_launches.argtypes = [vp, vp]
    L.crowd_reset_stats.argtypes = [vp]
    L.crowd_get_tuning.argtypes = [vp, vp]
    L.crowd_set_tuning.argtypes = [vp, vp]
    L.crowd_autotune.argtypes = [vp, C.c_float, i32, vp]
    L.crowd_synchronize.argtypes = [vp]
    L.crowd_destroy.argtypes = [vp]
    L.crowd_num_agents.argtypes = [vp]
    L.crowd_num_agents.restype = C.c_int64
    L.crowd_num_envs.argtypes = [vp]
    L.crowd_num_envs.restype = C.c_int32
    L.crowd_last_error.restype = C.c_char_p
    for name in EXPORTED:
        if name not in ("crowd_num_agents", "crowd_num_envs", "crowd_last_error"):
            getattr(L, name).restype = C.c_int
    _lib = L
    return L


def _check(st):
    if st != CROWD_OK:
        raise CrowdError(st, (load().crowd_last_error() or b"").decode())


def _host_ptr(a, dtype):
    if a is None:
        return None, None
    arr = np.ascontiguousarray(a, dtype=dtype)
    return arr, arr.ctypes.data_as(C.c_void_p)


def _ptr(a, dtype):
    """(keep-alive, pointer, ptr_kind) for a numpy array or a torch CUDA tensor."""
    if a is None:
        return None, None, CROWD_HOST
    if hasattr(a, "is_cuda") and a.is_cuda:
        import torch

        want = {np.float32: torch.float32, np.int32: torch.int32}[dtype]
        if a.dtype != want or not a.is_contiguous():
            raise TypeError(f"device tensor must be contiguous {want}")
        return a, C.c_void_p(a.data_ptr()), CROWD_DEVICE
    arr, p = _host_ptr(a, dtype)
    return arr, p, CROWD_HOST


# ------------------------------------------------------------------ C names

def crowd_create(n_envs, agents_per_env, radii, max_speeds, pref_speeds, init_pos, robot_index, segs_per_env,
                 segments, params, cuda_stream=None):
    L = load()
    keep = []
    ptrs = []
    for a, dt in ((agents_per_env, np.int32), (radii, np.float32), (max_speeds, np.float32),
                  (pref_speeds, np.float32), (init_pos, np.float32), (robot_index, np.int32),
                  (segs_per_env, np.int32), (segments, np.float32)):
        arr, p = _host_ptr(a, dt)
        keep.append(arr)
        ptrs.append(p)
    h = C.c_void_p()
    _check(L.crowd_create(int(n_envs), *ptrs, C.byref(params), C.c_void_p(cuda_stream or 0), C.byref(h)))
    return h


def crowd_set_goals(h, goals):
    keep, p, kind = _ptr(goals, np.float32)
    _check(load().crowd_set_goals(h, p, kind))


def crowd_set_state(h, state):
    keep, p, kind = _ptr(state, np.float32)
    _check(load().crowd_set_state(h, p, kind))


def crowd_step(h, dt, robot_vel=None, n_steps=1):
    keep, p, kind = _ptr(robot_vel, np.float32)
    _check(load().crowd_step(h, C.c_float(dt), p, kind, int(n_steps)))


def crowd_read_state(h, out=None):
    n = load().crowd_num_agents(h)
    if out is None:
        out = np.empty((n, 4), np.float32)
    keep, p, kind = _ptr(out, np.float32)
    if kind == CROWD_HOST and keep is not out:
        raise TypeError("out must be a contiguous float32 array")
    _check(load().crowd_read_state(h, p, kind))
    return out


def crowd_read_neighbors(h, K, out=None):
    n = load().crowd_num_agents(h)
    if out is None:
        out = np.empty((n, K), np.int32)
    keep, p, kind = _ptr(out, np.int32)
    if kind == CROWD_HOST and keep is not out:
        raise TypeError("out must be a contiguous int32 array")
    _check(load().crowd_read_neighbors(h, p, kind))
    return out


def crowd_read_stats(h):
    L = load()
    E, N = L.crowd_num_envs(h), L.crowd_num_agents(h)
    st = (crowd_env_stats * max(E, 1))()
    reach = np.empty(max(N, 1), np.int32)
    _check(L.crowd_read_stats(h, C.cast(st, C.c_void_p), reach.ctypes.data_as(C.c_void_p)))
    env = [dict(agent_collisions=s.agent_collisions, segment_collisions=s.segment_collisions,
                speed_sum=s.speed_sum, steps=s.steps) for s in st[:E]]
    return env, reach[:N]


def crowd_read_work(h):
    w = crowd_work()
    _check(load().crowd_read_work(h, C.byref(w)))
    return {n: int(getattr(w, n)) for n, _ in crowd_work._fields_}


def crowd_read_launches(h):
    n = C.c_int64()
    _check(load().crowd_read_launches(h, C.byref(n)))
    return int(n.value)


def crowd_get_tuning(h):
    t = crowd_tuning()
    _check(load().crowd_get_tuning(h, C.byref(t)))
    return dict(block_threads=t.block_threads, coop_fallback=t.coop_fallback, cell_split=t.cell_split,
                lanes_per_agent=t.lanes_per_agent, agent_order=t.agent_order, tiled_queue=t.tiled_queue)


def crowd_set_tuning(h, block_threads=0, coop_fallback=0, cell_split=1, lanes_per_agent=1, agent_order=0,
                     tiled_queue=1):
    t = crowd_tuning(block_threads, coop_fallback, cell_split, lanes_per_agent, agent_order, tiled_queue)
    _check(load().crowd_set_tuning(h, C.byref(t)))


def crowd_autotune(h, dt, n_steps):
    t = crowd_tuning()
    _check(load().crowd_autotune(h, C.c_float(dt), int(n_steps), C.byref(t)))
    return dict(block_threads=t.block_threads, coop_fallback=t.coop_fallback, cell_split=t.cell_split,
                lanes_per_agent=t.lanes_per_agent, agent_order=t.agent_order, tiled_queue=t.tiled_queue)


def crowd_reset_stats(h):
    _check(load().crowd_reset_stats(h))


def crowd_synchronize(h):
    _check(load().crowd_synchronize(h))


def crowd_destroy(h):
    _check(load().crowd_destroy(h))


def crowd_last_error():
    return (load().crowd_last_error() or b"").decode()


# ------------------------------------------------------------------ convenience

def params_for(scene, flags=0):
    f = lambda x: float(np.float32(x))
    if getattr(scene, "segment_mode", 0) == 1:
        flags |= CROWD_FLAG_VELOCITY_SEGMENTS
    return crowd_params(f(scene.tau), f(scene.tau_obst), f(scene.neighbor_dist), int(scene.max_neighbors),
                        f(scene.robot_responsibility), int(flags))


class Crowd:
    """One crowd handle built from a Scene (see scenes.py)."""

    def __init__(self, scene, flags=0, stream=None):
        self.scene = scene
        self.K = int(scene.max_neighbors)
        self.N = scene.n_agents
        self.E = scene.n_envs
        self.params = params_for(scene, flags)
        segs = scene.segments.reshape(-1, 4) if scene.segments.size else None
        self.h = crowd_create(scene.n_envs, scene.agents_per_env, scene.radius, scene.max_speed, scene.pref_speed,
                              scene.pos, scene.robot_index, scene.segs_per_env, segs, self.params, stream)
        crowd_set_goals(self.h, scene.goal)
        if np.any(scene.vel != 0):
            crowd_set_state(self.h, scene.state())

    def set_state(self, state):
        crowd_set_state(self.h, state)

    def set_goals(self, goals):
        crowd_set_goals(self.h, goals)

    def set_goal_queue(self, queue, cyclic=True):
        """queue [N][Q][2]: each agent's goals in order (see crowd_set_goal_queue)."""
        q = np.ascontiguousarray(queue, np.float32)
        assert q.ndim == 3 and q.shape[0] == self.N and q.shape[2] == 2
        _check(load().crowd_set_goal_queue(self.h, int(q.shape[1]), q.ctypes.data, int(bool(cyclic)), CROWD_HOST))

    def set_episodes(self, steps, init_state=None):
        """Per-environment episode lengths [E] (0: never; None: remove) and the
        rows they start from (None: the current state); see crowd_set_episodes."""
        st = None if steps is None else np.ascontiguousarray(steps, np.int32)
        assert st is None or st.shape == (self.E,)
        init = None if init_state is None else np.ascontiguousarray(init_state, np.float32)
        assert init is None or init.shape == (self.N, 4)
        _check(load().crowd_set_episodes(self.h, None if st is None else st.ctypes.data,
                                         None if init is None else init.ctypes.data, CROWD_HOST))

    def set_goal_pool(self, pool_start, points, seed):
        """Per-environment goal pools (see crowd_set_goal_pool); None removes."""
        if pool_start is None:
            _check(load().crowd_set_goal_pool(self.h, None, None, 0))
            return
        ps = np.ascontiguousarray(pool_start, np.int32)
        pts = np.ascontiguousarray(points, np.float32).reshape(-1, 2)
        assert ps.shape == (self.E + 1,)
        _check(load().crowd_set_goal_pool(self.h, ps.ctypes.data, pts.ctypes.data, int(seed)))

    def restart_envs(self, mask):
        """Start the environments with mask[e] set over now (see crowd_restart_envs)."""
        m = np.ascontiguousarray(mask, np.uint8)
        assert m.shape == (self.E,)
        _check(load().crowd_restart_envs(self.h, m.ctypes.data))

    def set_vehicles(self, veh):
        """Lane-following cars (scenes.Vehicles; see crowd_set_vehicles)."""
        i32 = lambda a: np.ascontiguousarray(a, np.int32)
        f32 = lambda a: np.ascontiguousarray(a, np.float32)
        arrs = [i32(veh.lane_start), f32(veh.points), i32(veh.agent), i32(veh.lane), f32(veh.s), f32(veh.v),
                f32(veh.params)]
        self._veh_n = len(arrs[2])
        _check(load().crowd_set_vehicles(self.h, len(arrs[0]) - 1, arrs[0].ctypes.data, arrs[1].ctypes.data,
                                         self._veh_n, arrs[2].ctypes.data, arrs[3].ctypes.data, arrs[4].ctypes.data,
                                         arrs[5].ctypes.data, arrs[6].ctypes.data, C.c_float(veh.half_width),
                                         C.c_float(veh.lookahead)))

    def vehicle_state(self):
        n = getattr(self, "_veh_n", 0)
        s, v = np.zeros(n, np.float32), np.zeros(n, np.float32)
        if n:
            _check(load().crowd_vehicle_state(self.h, 0, s.ctypes.data, v.ctypes.data))
        return s, v

    def set_vehicle_state(self, s, v):
        s, v = np.ascontiguousarray(s, np.float32), np.ascontiguousarray(v, np.float32)
        _check(load().crowd_vehicle_state(self.h, 1, s.ctypes.data, v.ctypes.data))

    def goal_index(self):
        out = np.zeros(self.N, np.int32)
        _check(load().crowd_read_goal_index(self.h, out.ctypes.data))
        return out

    def step(self, robot_vel=None, n_steps=1, dt=None):
        crowd_step(self.h, self.scene.dt if dt is None else dt, robot_vel, n_steps)

    def state(self, out=None):
        return crowd_read_state(self.h, out)

    def neighbors(self):
        return crowd_read_neighbors(self.h, self.K)

    def stats(self):
        return crowd_read_stats(self.h)

    def work(self):
        return crowd_read_work(self.h)

    def launches(self):
        """Kernels this handle's steps have enqueued so far (graph replays by
        their kernels)."""
        return crowd_read_launches(self.h)

    def tuning(self):
        return crowd_get_tuning(self.h)

    def set_tuning(self, **kw):
        crowd_set_tuning(self.h, **kw)

    def autotune(self, n_steps=20, dt=None):
        return crowd_autotune(self.h, self.scene.dt if dt is None else dt, n_steps)

    def reset_stats(self):
        crowd_reset_stats(self.h)

    def synchronize(self):
        crowd_synchronize(self.h)

    def close(self):
        if self.h is not None:
            crowd_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
