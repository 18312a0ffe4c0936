"""Python layer of depth-map mean fusion and TSDF integration (Sec. 4.4):
argument marshalling over libpgsag's pgsag_depth_fuse / pgsag_tsdf_integrate."""
from __future__ import annotations

import ctypes
from typing import Optional, Sequence, Tuple

import numpy as np
import torch

from . import _lib as L


def _ptr(t: Optional[torch.Tensor]):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream_ptr(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def fuse(maps: torch.Tensor, out: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
    """Mean of the valid (> 0, finite) depths of maps [n_maps, ...] per pixel."""
    lib = L.load()
    maps = maps.contiguous()
    assert maps.dtype == torch.float32 and maps.is_cuda
    n_maps = int(maps.shape[0])
    n_pix = maps[0].numel()
    if out is None:
        out = torch.empty(maps.shape[1:], dtype=torch.float32, device=maps.device)
    L.check(lib.pgsag_depth_fuse(n_maps, _ptr(maps), n_pix, _ptr(out), _stream_ptr(stream)), "pgsag_depth_fuse")
    return out


def depth_views(cams, offsets: Sequence[int]):
    """ctypes array of pgsag_depth_view (cameras with R, t, fx, fy, cx, cy, znear,
    width, height; offsets = first float of each view's map in the depth buffer)."""
    arr = (L.PgsagDepthView * max(len(cams), 1))()
    for v, c in enumerate(cams):
        V = arr[v]
        R = np.asarray(c.R, np.float32).reshape(9)
        t = np.asarray(c.t, np.float32).reshape(3)
        for k in range(9):
            V.R[k] = float(R[k])
        for k in range(3):
            V.t[k] = float(t[k])
        V.fx, V.fy, V.cx, V.cy, V.znear = float(c.fx), float(c.fy), float(c.cx), float(c.cy), float(c.znear)
        V.width, V.height = int(c.width), int(c.height)
        V.depth_offset = int(offsets[v])
    return arr


def grid(origin, voxel: float, dims, trunc: float):
    g = L.PgsagTsdfGrid()
    for a in range(3):
        g.origin[a] = float(origin[a])
    g.voxel, g.trunc = float(voxel), float(trunc)
    g.nx, g.ny, g.nz = (int(d) for d in dims)
    return g


def integrate(g, cams, depth: torch.Tensor, offsets: Sequence[int], tsdf: torch.Tensor, weight: torch.Tensor,
              accumulate: bool = False, status: Optional[torch.Tensor] = None, table=None, stream=None):
    """Integrate the views' depth maps (depth: one float32 device buffer, view v's
    map [H, W] at offsets[v]) into tsdf / weight [nz, ny, nx] (float32 device), in
    calls of at most 256 views."""
    lib = L.load()
    if status is None:
        status = torch.zeros(1, dtype=torch.int32, device=tsdf.device)
    arr = depth_views(cams, offsets) if table is None else table
    nv = len(cams)
    first = True
    s = _stream_ptr(stream)
    for v0 in range(0, max(nv, 1), L.TSDF_MAX_VIEWS):
        n = min(L.TSDF_MAX_VIEWS, nv - v0)
        sub = ctypes.cast(ctypes.addressof(arr) + v0 * ctypes.sizeof(L.PgsagDepthView),
                          ctypes.POINTER(L.PgsagDepthView))
        acc = 1 if (accumulate or not first) else 0
        L.check(lib.pgsag_tsdf_integrate(ctypes.byref(g), n, sub, _ptr(depth), acc, _ptr(tsdf), _ptr(weight),
                                         _ptr(status), s), "pgsag_tsdf_integrate")
        first = False
    return status
