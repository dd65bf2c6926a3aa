"""Pins of the lane-following vehicle oracle (CPU only): the free-road and
standstill behaviour the Intelligent Driver Model is built to have, the
steady state of a ring platoon, the corridor in which crowd agents block a
vehicle, and the arc-length placement on the lane polyline."""
import math

import numpy as np
import pytest

from oracle import vehicles as VH

SQ = [(0.0, 0.0), (100.0, 0.0), (100.0, 100.0), (0.0, 100.0)]  # ring of length 400
P = (10.0, 1.5, 1.0, 2.0, 2.0, 4.5)  # v0, T, a, b, s0, length


def _ring():
    return VH.Lanes(np.array(SQ, np.float32), [0, 4])


def test_polyline_arc_length():
    ln = _ring()
    assert ln.length(0) == 400.0
    assert np.allclose(ln.point(0, 0.0), [0, 0]) and np.allclose(ln.point(0, 100.0), [100, 0])
    assert np.allclose(ln.point(0, 150.0), [100, 50]) and np.allclose(ln.point(0, 399.0), [0, 1])


def test_free_road_from_rest_and_desired_speed():
    """Alone on the lane: from rest the first step accelerates at a exactly;
    the speed then rises to the desired speed v0 and stays there."""
    ln = _ring()
    s, v = np.array([0.0]), np.array([0.0])
    prm = np.array([P])
    s1, v1, *_ = VH.idm_step(ln, [0], s, v, prm, np.zeros((0, 2)), np.zeros(0), np.zeros(0, bool), 1.5, 25.0, 0.1)
    assert v1[0] == pytest.approx(P[2] * 0.1, abs=1e-15) and s1[0] == pytest.approx(P[2] * 0.1 * 0.1, abs=1e-15)
    for _ in range(3000):
        s, v, *_ = VH.idm_step(ln, [0], s, v, prm, np.zeros((0, 2)), np.zeros(0), np.zeros(0, bool), 1.5, 25.0, 0.1)
    assert v[0] == pytest.approx(10.0, abs=1e-6)


def test_ring_platoon_steady_state():
    """N equal cars spaced evenly on a ring keep the spacing and settle where
    the IDM acceleration vanishes: (s0 + v T) / sqrt(1 - (v/v0)^4) equals the
    gap L/N - length; that speed is found here by bisection."""
    ln = _ring()
    N = 16
    s = np.arange(N) * 400.0 / N
    v = np.full(N, 3.0)
    prm = np.tile(P, (N, 1))
    for _ in range(4000):
        s, v, *_ = VH.idm_step(ln, np.zeros(N, int), s, v, prm, np.zeros((0, 2)), np.zeros(0), np.zeros(0, bool),
                               1.5, 25.0, 0.1)
    gap = 400.0 / N - 4.5
    lo, hi = 0.0, 10.0
    for _ in range(100):
        mid = 0.5 * (lo + hi)
        if (2.0 + mid * 1.5) / math.sqrt(1 - (mid / 10.0) ** 4) < gap:
            lo = mid
        else:
            hi = mid
    assert np.allclose(v, lo, atol=1e-6)
    d = np.diff(np.sort(s))
    assert np.allclose(d, 400.0 / N, atol=1e-6)


def test_stops_behind_a_standing_pedestrian():
    """A pedestrian standing on the lane 60 m ahead: the car brakes to a stop
    without reaching it, ending near the jam distance s0 (where the IDM
    acceleration at rest vanishes)."""
    ln = _ring()
    s, v = np.array([0.0]), np.array([10.0])
    prm = np.array([P])
    ped, r = np.array([[60.0, 0.3]]), np.array([0.3])
    for _ in range(600):
        s, v, *_ = VH.idm_step(ln, [0], s, v, prm, ped, r, np.array([True]), 1.5, 80.0, 0.1)
    gap = 60.0 - s[0] - 0.5 * 4.5 - 0.3
    assert v[0] == 0.0 and 1.9 <= gap <= 2.6


@pytest.mark.parametrize("lat,ahead,blocks", [(1.5 + 0.3 - 1e-3, 10.0, True), (1.5 + 0.3 + 1e-3, 10.0, False),
                                              (0.5, 24.9, True), (0.5, 25.1, False), (0.5, -3.0, False)])
def test_blocking_corridor(lat, ahead, blocks):
    """Crowd agents block when within half_width + r of the lane and at most
    `lookahead` ahead; behind the car they do not."""
    ln = _ring()
    s, v = np.array([50.0]), np.array([5.0])
    prm = np.array([P])
    ped = np.array([[50.0 + ahead, lat]])
    _, v_blk, *_ = VH.idm_step(ln, [0], s, v, prm, ped, [0.3], [True], 1.5, 25.0, 0.1)
    _, v_free, *_ = VH.idm_step(ln, [0], s, v, prm, np.zeros((0, 2)), np.zeros(0), np.zeros(0, bool), 1.5, 25.0, 0.1)
    assert (v_blk[0] < v_free[0]) == blocks
