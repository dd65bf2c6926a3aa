"""FP32/integer oracle of the occupancy-map front end (test infrastructure).

The paper's scenes come from generated maps of traversable ground and static
objects, on which the dynamic agents get sampled start and end points (Sec.
3.1 "Hierarchical Urban Generation", Sec. 3.2 "Interactive Dynamics
Generation").  The front end turns such a map, given as a raster, into the
static segments of the crowd step and samples points on its traversable
ground.  This module states both plainly (loops over cells and lines, no
blocking) so that the CUDA kernels can be checked bit for bit:

  map_segments: the boundary between free and obstacle cells as maximal
      axis-aligned segments, each directed with the free side on its left;
  map_sample:   points drawn uniformly over the cells that are free with a
      clearance of c cells (Chebyshev), with the counter-based generator
      Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC 2011) written from its
      published definition.

Only tests/ import this module; the product path never does.
"""
from __future__ import annotations

import numpy as np

M32 = 0xFFFFFFFF
# Philox4x32 round multipliers and Weyl key increments (SC 2011, Table 2 /
# Section 5): the multipliers M0, M1 and the golden-ratio and sqrt(3)-1 bumps
PHILOX_M0, PHILOX_M1 = 0xD2511F53, 0xCD9E8D57
PHILOX_W0, PHILOX_W1 = 0x9E3779B9, 0xBB67AE85


def philox4x32_10(counter, key):
    """Philox4x32 with 10 rounds: 4 x 32-bit counter, 2 x 32-bit key ->
    4 x 32-bit outputs.  Each round multiplies two words by the round
    constants, takes high and low halves of the 64-bit products, and mixes
    them with the other two words and the round key; the key is bumped by the
    Weyl constants between rounds."""
    c0, c1, c2, c3 = (int(x) & M32 for x in counter)
    k0, k1 = (int(x) & M32 for x in key)
    for r in range(10):
        if r:
            k0 = (k0 + PHILOX_W0) & M32
            k1 = (k1 + PHILOX_W1) & M32
        p0 = PHILOX_M0 * c0
        p1 = PHILOX_M1 * c2
        hi0, lo0 = p0 >> 32, p0 & M32
        hi1, lo1 = p1 >> 32, p1 & M32
        c0, c1, c2, c3 = (hi1 ^ c1 ^ k0) & M32, lo1, (hi0 ^ c3 ^ k1) & M32, lo0
    return c0, c1, c2, c3


def _free(occ, closed):
    """Free flags with a one-cell frame: outside the map counts as obstacle
    when `closed`, else as free."""
    occ = np.asarray(occ)
    H, W = occ.shape
    f = np.full((H + 2, W + 2), not closed, bool)
    f[1:-1, 1:-1] = occ == 0
    return f


def _f32(x):
    return np.float32(x)


def _coord(o, i, h):
    # o + i * h, the product and the sum rounded to FP32 separately
    return _f32(_f32(o) + _f32(_f32(i) * _f32(h)))


def map_segments(occ, cell, x0, y0, closed):
    """Boundary segments [n][4] (ax, ay, bx, by) float32 of raster `occ`
    ([H][W], nonzero = obstacle; cell (x, y) covers [x0 + x h, x0 + (x+1) h)
    x [y0 + y h, y0 + (y+1) h)).  Horizontal lines y = y0 + j h (j = 0..H)
    first, then vertical lines x = x0 + i h (i = 0..W); along each line the
    maximal runs of unit edges that separate a free from an obstacle cell
    with the free cell on the same side, in increasing coordinate.  Each
    segment runs with its free side on the left."""
    f = _free(occ, closed)
    H, W = np.asarray(occ).shape
    out = []
    for j in range(H + 1):  # between row j-1 (below) and row j (above)
        x = 0
        while x < W:
            below, above = f[j, x + 1], f[j + 1, x + 1]
            if below == above:
                x += 1
                continue
            side = above  # free above
            xs = x
            while x < W and f[j, x + 1] != f[j + 1, x + 1] and f[j + 1, x + 1] == side:
                x += 1
            a = (_coord(x0, xs, cell), _coord(y0, j, cell))
            b = (_coord(x0, x, cell), _coord(y0, j, cell))
            out.append(a + b if side else b + a)  # free above: +x; free below: -x
    for i in range(W + 1):  # between column i-1 (left) and column i (right)
        y = 0
        while y < H:
            left, right = f[y + 1, i], f[y + 1, i + 1]
            if left == right:
                y += 1
                continue
            side = left  # free on the left of the line
            ys = y
            while y < H and f[y + 1, i] != f[y + 1, i + 1] and f[y + 1, i] == side:
                y += 1
            a = (_coord(x0, i, cell), _coord(y0, ys, cell))
            b = (_coord(x0, i, cell), _coord(y0, y, cell))
            out.append(a + b if side else b + a)  # free left: +y; free right: -y
    return np.array(out, np.float32).reshape(-1, 4)


def eligible_cells(occ, closed, clearance):
    """Row-major linear indices of the free cells with no obstacle cell (and,
    when `closed`, no outside) within `clearance` cells in x and y."""
    occ = np.asarray(occ)
    H, W = occ.shape
    c = int(clearance)
    f = np.full((H + 2 * c + 2, W + 2 * c + 2), not closed, bool)
    f[c + 1:c + 1 + H, c + 1:c + 1 + W] = occ == 0
    cells = []
    for y in range(H):
        for x in range(W):
            win = f[y + 1:y + 2 * c + 2, x + 1:x + 2 * c + 2]
            if win.all():
                cells.append(y * W + x)
    return np.array(cells, np.int64)


def map_sample(occ, cell, x0, y0, closed, clearance, seed, stream, n):
    """Points [n][2] float32: point k draws (u0, u1, u2, u3) = Philox4x32-10(
    counter (k, stream, 0, 0), key (seed & 0xffffffff, seed >> 32)); it lies
    in eligible cell number floor(u0 M / 2^32) (M eligible cells, row-major
    order) at offsets (u1 >> 8) 2^-24 and (u2 >> 8) 2^-24 of the cell."""
    occ = np.asarray(occ)
    W = occ.shape[1]
    cells = eligible_cells(occ, closed, clearance)
    M = len(cells)
    pts = np.zeros((n, 2), np.float32)
    if M == 0:
        return pts, 0
    key = (seed & M32, (seed >> 32) & M32)
    for k in range(n):
        u0, u1, u2, _ = philox4x32_10((k, stream, 0, 0), key)
        idx = (u0 * M) >> 32
        cx, cy = int(cells[idx] % W), int(cells[idx] // W)
        fx = _f32((u1 >> 8) * 2.0 ** -24)
        fy = _f32((u2 >> 8) * 2.0 ** -24)
        tx = _f32(_f32(cx) + fx)
        ty = _f32(_f32(cy) + fy)
        pts[k, 0] = _f32(_f32(x0) + _f32(tx * _f32(cell)))
        pts[k, 1] = _f32(_f32(y0) + _f32(ty * _f32(cell)))
    return pts, M
