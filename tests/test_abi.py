"""The C-ABI library builds, loads, exports every call its header declares,
and rejects bad arguments on the host before touching the GPU (no GPU needed)."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from paper_2505_00690_gb300 import build as B
from paper_2505_00690_gb300 import crowd as cw

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return cw.load()


def declared_functions():
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if h.endswith(".h"):
            text = open(os.path.join(ROOT, "include", h)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names += re.findall(r"^\s*[A-Za-z_][\w\s\*]*?\b(crowd_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ["crowd_create", "crowd_set_goals", "crowd_step", "crowd_read_state", "crowd_destroy"]:
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name
    assert lib.crowd_abi_version() == 5


def _params(**kw):
    p = dict(time_horizon=2.0, time_horizon_obst=2.0, neighbor_dist=5.0, max_neighbors=10,
             robot_responsibility=0.5, flags=0)
    p.update(kw)
    return cw.crowd_params(**p)


def _create(lib, n=3, **over):
    args = dict(agents_per_env=np.array([n], np.int32), radii=np.full(n, 0.3, np.float32),
                max_speeds=np.full(n, 1.4, np.float32), pref=None,
                pos=np.arange(2 * n, dtype=np.float32).reshape(n, 2), robot=np.array([-1], np.int32),
                segs_per_env=np.array([0], np.int32), segs=None, params=_params())
    args.update(over)
    keep = [np.ascontiguousarray(a) if isinstance(a, np.ndarray) else a for a in args.values()]
    ptr = lambda a: None if a is None else a.ctypes.data_as(C.c_void_p)
    h = C.c_void_p()
    st = lib.crowd_create(1, ptr(args["agents_per_env"]), ptr(args["radii"]), ptr(args["max_speeds"]),
                          ptr(args["pref"]), ptr(args["pos"]), ptr(args["robot"]), ptr(args["segs_per_env"]),
                          ptr(args["segs"]), C.byref(args["params"]), None, C.byref(h))
    return st, h, keep


@pytest.mark.parametrize("over,msg", [
    (dict(radii=np.array([0.3, 0.0, 0.3], np.float32)), "radius"),
    (dict(radii=np.array([0.3, -1.0, 0.3], np.float32)), "radius"),
    (dict(max_speeds=np.array([1.0, -0.1, 1.0], np.float32)), "max_speed"),
    (dict(pos=np.array([[0, 0], [np.nan, 1], [2, 2]], np.float32)), "NaN"),
    (dict(pos=np.array([[0, 0], [np.inf, 1], [2, 2]], np.float32)), "NaN"),
    (dict(params=_params(max_neighbors=33)), "max_neighbors"),
    (dict(params=_params(max_neighbors=-1)), "max_neighbors"),
    (dict(params=_params(neighbor_dist=0.0)), "neighbor_dist"),
    (dict(params=_params(time_horizon=0.0)), "time_horizon"),
    (dict(params=_params(time_horizon=float("nan"))), "time_horizon"),
    (dict(params=_params(robot_responsibility=1.5)), "robot_responsibility"),
    (dict(robot=np.array([3], np.int32)), "robot_index"),
    (dict(segs_per_env=np.array([1], np.int32), segs=np.array([[1, 1, 1, 1]], np.float32)), "zero length"),
    (dict(segs_per_env=np.array([1], np.int32), segs=np.array([[1, np.nan, 1, 2]], np.float32)), "NaN"),
])
def test_bad_arguments_rejected_on_host(lib, over, msg):
    st, h, keep = _create(lib, **over)
    assert st == cw.CROWD_EINVAL
    assert msg in lib.crowd_last_error().decode()
    assert not h.value


def test_null_handle_calls_fail_cleanly(lib):
    assert lib.crowd_step(None, C.c_float(0.1), None, 0, 1) == cw.CROWD_EINVAL
    assert lib.crowd_read_state(None, None, 0) == cw.CROWD_EINVAL
    assert lib.crowd_set_goal_queue(None, 2, None, 1, 0) == cw.CROWD_EINVAL
    assert lib.crowd_read_goal_index(None, None) == cw.CROWD_EINVAL
    assert lib.crowd_set_episodes(None, None, None, 0) == cw.CROWD_EINVAL
    assert lib.crowd_restart_envs(None, None) == cw.CROWD_EINVAL
    assert lib.crowd_set_goal_pool(None, None, None, 0) == cw.CROWD_EINVAL
    assert lib.crowd_vehicle_state(None, 0, None, None) == cw.CROWD_EINVAL
    assert lib.crowd_destroy(None) == cw.CROWD_OK
    assert lib.crowd_num_agents(None) == 0


def _preceding_comments():
    """Each declared call with the comment block that comes right before its
    declaration in the header (the block that documents it)."""
    out = {}
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not h.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", h)).read()
        for m in re.finditer(r"^\s*[A-Za-z_][\w\s\*]*?\b(crowd_\w+)\s*\(", text, flags=re.M):
            before = text[:m.start(1)]
            end = before.rfind("*/")
            start = before.rfind("/*", 0, end)
            out[m.group(1)] = before[start:end + 2] if end >= 0 and start >= 0 else ""
    return out


def test_every_call_cites_the_passage_that_defines_it():
    """Every boundary call names the paper section (or appendix subsection)
    that defines the operation, or says that the paper has none."""
    cites = re.compile(r"Sec\. 3\.[1-3]|Appendix \"|[Nn]o counterpart")
    blocks = _preceding_comments()
    for name in declared_functions():
        assert cites.search(blocks.get(name, "")), name
    for name in ["crowd_create", "crowd_set_goals", "crowd_step", "crowd_read_state"]:
        assert re.search(r"Sec\. 3\.2", blocks[name]), name
