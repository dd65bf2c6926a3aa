"""Binding of the occupancy-map front end (crowd_map_segments,
crowd_map_sample in include/crowd.h): marshalling only.

Maps and outputs are PyTorch CUDA tensors (the calls take device pointers);
all arithmetic runs in the library's kernels."""
from __future__ import annotations

import ctypes as C

from . import crowd as cw


def _lib():
    L = cw.load()
    if not getattr(L, "_map_bound", False):
        vp, i32, f32 = C.c_void_p, C.c_int32, C.c_float
        L.crowd_map_segments.argtypes = [vp, i32, i32, f32, f32, f32, i32, i32, vp, C.POINTER(i32), vp]
        L.crowd_map_sample.argtypes = [vp, i32, i32, f32, f32, f32, i32, i32, C.c_uint64, C.c_uint32, i32, vp,
                                       C.POINTER(i32), vp]
        L.crowd_map_segments.restype = C.c_int
        L.crowd_map_sample.restype = C.c_int
        L._map_bound = True
    return L


def _check_map(occ):
    import torch

    if not (isinstance(occ, torch.Tensor) and occ.is_cuda and occ.dtype == torch.uint8 and occ.dim() == 2):
        raise TypeError("occ must be a CUDA uint8 tensor [H][W]")
    return occ.contiguous()


def map_segments(occ, cell, x0=0.0, y0=0.0, closed=True, stream=None):
    """Boundary segments [n][4] (CUDA float32 tensor) of map `occ`."""
    import torch

    occ = _check_map(occ)
    H, W = occ.shape
    L = _lib()
    n = C.c_int32()
    s = C.c_void_p(stream or torch.cuda.current_stream(occ.device).cuda_stream)
    st = L.crowd_map_segments(occ.data_ptr(), W, H, cell, x0, y0, int(bool(closed)), 0, None, C.byref(n), s)
    if st not in (cw.CROWD_OK, cw.CROWD_EINVAL) or (st == cw.CROWD_EINVAL and n.value == 0):
        cw._check(st)
    out = torch.empty((max(n.value, 1), 4), dtype=torch.float32, device=occ.device)
    cw._check(L.crowd_map_segments(occ.data_ptr(), W, H, cell, x0, y0, int(bool(closed)), n.value, out.data_ptr(),
                                   C.byref(n), s))
    return out[: n.value]


def map_sample(occ, cell, n, x0=0.0, y0=0.0, closed=True, clearance=0, seed=0, stream_id=0, stream=None):
    """(points [n][2] CUDA float32 tensor, number of eligible cells)."""
    import torch

    occ = _check_map(occ)
    H, W = occ.shape
    out = torch.empty((max(int(n), 1), 2), dtype=torch.float32, device=occ.device)
    m = C.c_int32()
    s = C.c_void_p(stream or torch.cuda.current_stream(occ.device).cuda_stream)
    cw._check(_lib().crowd_map_sample(occ.data_ptr(), W, H, cell, x0, y0, int(bool(closed)), int(clearance),
                                      int(seed), int(stream_id), int(n), out.data_ptr(), C.byref(m), s))
    return out[: int(n)], m.value
