"""Pins of the occupancy-map front end's oracle (CPU only).

The generator is pinned by the known-answer vectors published with the
Philox family (Random123's kat_vectors, Philox4x32-10); the segment
extraction by hand-drawn maps and by invariants that hold for any map (the
free side of every segment is free, the obstacle side is not, the segments
tile the free/obstacle boundary exactly); the sampler by the cells it may
use and by uniformity over them."""
import numpy as np
import pytest

from oracle import frontend as F


@pytest.mark.parametrize("counter,key,expect", [
    ((0, 0, 0, 0), (0, 0), (0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8)),
    ((0xFFFFFFFF,) * 4, (0xFFFFFFFF, 0xFFFFFFFF), (0x408F276D, 0x41C83B0E, 0xA20BC7C6, 0x6D5451FD)),
    ((0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344), (0xA4093822, 0x299F31D0),
     (0xD16CFE09, 0x94FDCCEB, 0x5001E420, 0x24126EA1)),
])
def test_philox_known_answers(counter, key, expect):
    assert F.philox4x32_10(counter, key) == expect


def test_single_obstacle_cell_open_map():
    """One obstacle cell in a 3 x 3 free map, unit cells: its four edges,
    bottom and top first (horizontal lines), then left and right, each with
    the free side on its left."""
    occ = np.zeros((3, 3), np.uint8)
    occ[1, 1] = 1
    seg = F.map_segments(occ, 1.0, 0.0, 0.0, closed=False)
    assert seg.tolist() == [[2, 1, 1, 1],   # y = 1, free below: runs -x
                            [1, 2, 2, 2],   # y = 2, free above: runs +x
                            [1, 1, 1, 2],   # x = 1, free on the left: runs +y
                            [2, 2, 2, 1]]   # x = 2, free on the right: runs -y


def test_closed_empty_map_is_walled():
    seg = F.map_segments(np.zeros((2, 3), np.uint8), 0.5, -1.0, 2.0, closed=True)
    assert seg.tolist() == [[-1.0, 2.0, 0.5, 2.0],    # bottom wall, free above
                            [0.5, 3.0, -1.0, 3.0],    # top wall, free below
                            [-1.0, 3.0, -1.0, 2.0],   # left wall, free on the right
                            [0.5, 2.0, 0.5, 3.0]]     # right wall, free on the left
    assert F.map_segments(np.zeros((2, 3), np.uint8), 0.5, -1.0, 2.0, closed=False).shape == (0, 4)


def test_runs_merge_and_split_by_side():
    """An obstacle row of 3 cells gives one bottom and one top segment of
    length 3; a checkerboard gives unit segments only."""
    occ = np.zeros((3, 5), np.uint8)
    occ[1, 1:4] = 1
    seg = F.map_segments(occ, 1.0, 0.0, 0.0, closed=False)
    lengths = np.hypot(seg[:, 2] - seg[:, 0], seg[:, 3] - seg[:, 1])
    assert sorted(lengths.tolist()) == [1, 1, 3, 3]
    cb = (np.indices((4, 4)).sum(0) % 2).astype(np.uint8)
    seg = F.map_segments(cb, 1.0, 0.0, 0.0, closed=True)
    assert np.all(np.hypot(seg[:, 2] - seg[:, 0], seg[:, 3] - seg[:, 1]) == 1.0)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_segments_separate_free_from_obstacle(seed):
    """Any map: every unit edge between a free and an obstacle cell is covered
    exactly once, nothing else is, and the left of each segment is free."""
    rng = np.random.default_rng(seed)
    occ = (rng.random((13, 17)) < 0.35).astype(np.uint8)
    for closed in (False, True):
        seg = F.map_segments(occ, 1.0, 0.0, 0.0, closed=closed)
        f = F._free(occ, closed)
        covered = 0
        for ax, ay, bx, by in seg.astype(int):
            n = max(abs(bx - ax), abs(by - ay))
            dx, dy = np.sign(bx - ax), np.sign(by - ay)
            for t in range(n):
                x, y = ax + t * dx, ay + t * dy
                # unit edge from (x, y) in direction (dx, dy): cells on its left and right
                if dx:
                    cx = min(x, x + dx)
                    left_cell, right_cell = ((cx, y), (cx, y - 1)) if dx > 0 else ((cx, y - 1), (cx, y))
                else:
                    cy = min(y, y + dy)
                    left_cell, right_cell = ((x - 1, cy), (x, cy)) if dy > 0 else ((x, cy), (x - 1, cy))
                assert f[left_cell[1] + 1, left_cell[0] + 1] and not f[right_cell[1] + 1, right_cell[0] + 1]
                covered += 1
        boundary = int((f[1:, 1:-1] != f[:-1, 1:-1]).sum() + (f[1:-1, 1:] != f[1:-1, :-1]).sum())
        assert covered == boundary


def test_sample_stays_in_eligible_cells_and_is_uniform():
    rng = np.random.default_rng(5)
    occ = (rng.random((10, 12)) < 0.2).astype(np.uint8)
    cells = F.eligible_cells(occ, closed=True, clearance=1)
    assert len(cells) > 5
    n = 4000
    pts, M = F.map_sample(occ, 0.5, 3.0, -2.0, True, 1, seed=0x1234567890, stream=3, n=n)
    assert M == len(cells)
    cx = np.floor((pts[:, 0] - 3.0) / 0.5).astype(int)
    cy = np.floor((pts[:, 1] + 2.0) / 0.5).astype(int)
    lin = cy * 12 + cx
    assert np.isin(lin, cells).all()
    counts = np.array([(lin == c).sum() for c in cells])
    expect = n / len(cells)
    chi2 = ((counts - expect) ** 2 / expect).sum()
    assert chi2 < len(cells) + 6 * np.sqrt(2 * len(cells))  # about 6 sigma of a chi-square
    # another stream or seed gives another sequence; the same gives the same
    again, _ = F.map_sample(occ, 0.5, 3.0, -2.0, True, 1, seed=0x1234567890, stream=3, n=50)
    other, _ = F.map_sample(occ, 0.5, 3.0, -2.0, True, 1, seed=0x1234567890, stream=4, n=50)
    assert np.array_equal(again, pts[:50]) and not np.array_equal(other, pts[:50])


def test_clearance_and_empty_cases():
    occ = np.zeros((5, 5), np.uint8)
    assert len(F.eligible_cells(occ, closed=True, clearance=0)) == 25
    assert F.eligible_cells(occ, closed=True, clearance=1).tolist() == [6, 7, 8, 11, 12, 13, 16, 17, 18]
    assert F.eligible_cells(occ, closed=True, clearance=2).tolist() == [12]
    assert len(F.eligible_cells(occ, closed=True, clearance=3)) == 0
    pts, M = F.map_sample(occ, 1.0, 0.0, 0.0, True, 3, seed=1, stream=0, n=4)
    assert M == 0 and not pts.any()
