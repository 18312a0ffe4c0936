"""Python layer of the multi-view voting filter (Sec. 4.1, Eq. 5-7): argument
marshalling over libpgsag's pgsag_vote_* calls.  The masks are bit-packed once
on the device (they are fixed over training); every vote then runs in the
library's kernels.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass
from typing import List, Optional, Sequence

import numpy as np
import torch

from . import _lib as L


def _ptr(t: Optional[torch.Tensor]):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream_ptr(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


@dataclass
class PackedMasks:
    """Bit-packed masks of a set of views in one device buffer."""
    bits: torch.Tensor          # int32 words (bit x & 31 of word y * wpr + x >> 5)
    offsets: List[int]          # first word of each view
    words_per_row: List[int]
    widths: List[int]
    heights: List[int]


def pack_masks(masks: Sequence[torch.Tensor], words_per_row: Optional[Sequence[int]] = None,
               stream=None) -> PackedMasks:
    """Pack uint8 [H, W] device masks (nonzero = building) with pgsag_vote_pack_mask."""
    lib = L.load()
    wprs, offs, Ws, Hs = [], [], [], []
    total = 0
    for i, m in enumerate(masks):
        H, W = int(m.shape[0]), int(m.shape[1])
        wpr = (W + 31) // 32 if words_per_row is None else int(words_per_row[i])
        offs.append(total)
        wprs.append(wpr)
        Ws.append(W)
        Hs.append(H)
        total += H * wpr
    dev = masks[0].device if len(masks) else torch.device("cuda")
    bits = torch.empty(max(total, 1), dtype=torch.int32, device=dev)
    s = _stream_ptr(stream)
    for i, m in enumerate(masks):
        m = m.contiguous()
        assert m.dtype == torch.uint8 and m.is_cuda
        L.check(lib.pgsag_vote_pack_mask(Ws[i], Hs[i], _ptr(m), wprs[i],
                                         ctypes.c_void_p(bits.data_ptr() + 4 * offs[i]), s),
                "pgsag_vote_pack_mask")
    return PackedMasks(bits, offs, wprs, Ws, Hs)


def vote_views(cams, packed: PackedMasks):
    """ctypes array of pgsag_vote_view for cameras with .R, .t, .fx, .fy, .cx, .cy,
    .znear (the pinhole camera of the renderer) and their packed masks."""
    arr = (L.PgsagVoteView * max(len(cams), 1))()
    for v, c in enumerate(cams):
        V = arr[v]
        R = np.asarray(c.R, np.float32).reshape(9)
        t = np.asarray(c.t, np.float32).reshape(3)
        for k in range(9):
            V.R[k] = float(R[k])
        for k in range(3):
            V.t[k] = float(t[k])
        V.fx, V.fy, V.cx, V.cy, V.znear = float(c.fx), float(c.fy), float(c.cx), float(c.cy), float(c.znear)
        if int(c.width) != packed.widths[v] or int(c.height) != packed.heights[v]:
            raise ValueError(f"view {v}: camera {c.width}x{c.height} vs mask {packed.widths[v]}x{packed.heights[v]}")
        V.width, V.height = int(c.width), int(c.height)
        V.words_per_row = packed.words_per_row[v]
        V.mask_offset = packed.offsets[v]
    return arr


@dataclass
class VoteResult:
    in_mask: torch.Tensor   # int32 [M] (uint32 counts): views whose mask holds the point (Eq. 5/6)
    us: torch.Tensor        # int32 [M]: unreliability score (Eq. 7)
    reliable: torch.Tensor  # uint8 [M]: potential and US < tau
    status: Optional[torch.Tensor] = None  # int32 [1] device status flags of the call


def vote_filter(points: torch.Tensor, cams, packed: PackedMasks, tau: int, out: Optional[VoteResult] = None,
                stream=None, table=None) -> VoteResult:
    """Eq. 5-7 for points float32 [M, 3] (device) against all views (in calls of
    at most 256 views, counts accumulated).  `table`: a prebuilt vote_views()
    array for these cameras (built here if omitted); `out`: result buffers to
    reuse (their status tensor is kept, not cleared)."""
    lib = L.load()
    points = points.contiguous()
    assert points.dtype == torch.float32 and points.is_cuda and points.shape[-1] == 3
    M = int(points.shape[0])
    dev = points.device
    if out is None:
        out = VoteResult(torch.empty(M, dtype=torch.int32, device=dev), torch.empty(M, dtype=torch.int32, device=dev),
                         torch.empty(M, dtype=torch.uint8, device=dev))
    if out.status is None:
        out.status = torch.zeros(1, dtype=torch.int32, device=dev)
    arr = vote_views(cams, packed) if table is None else table
    s = _stream_ptr(stream)
    nv = len(cams)
    first = True
    for v0 in range(0, max(nv, 1), L.VOTE_MAX_VIEWS):
        n = min(L.VOTE_MAX_VIEWS, nv - v0)
        sub = ctypes.cast(ctypes.addressof(arr) + v0 * ctypes.sizeof(L.PgsagVoteView), ctypes.POINTER(L.PgsagVoteView))
        L.check(lib.pgsag_vote_filter(M, _ptr(points), n, sub, _ptr(packed.bits), int(tau), 0 if first else 1,
                                      _ptr(out.in_mask), _ptr(out.us), _ptr(out.reliable), _ptr(out.status), s),
                "pgsag_vote_filter")
        first = False
    return out


def compact_async(reliable: torch.Tensor, idx: torch.Tensor, n_out: torch.Tensor, workspace: torch.Tensor,
                  status: torch.Tensor, stream=None) -> None:
    """Enqueue pgsag_vote_compact: the ascending indices of the nonzero entries of
    reliable into idx (int32, >= len(reliable) entries) and their number into
    n_out (int32 [1]); no host synchronisation."""
    lib = L.load()
    M = int(reliable.shape[0])
    ws_bytes = workspace.numel() * workspace.element_size()
    L.check(lib.pgsag_vote_compact(M, _ptr(reliable), _ptr(idx), _ptr(n_out), _ptr(workspace), ws_bytes,
                                   _ptr(status), _stream_ptr(stream)), "pgsag_vote_compact")


def compact_workspace(n: int, device="cuda") -> torch.Tensor:
    """Workspace tensor for compact_async over n entries."""
    ws_bytes = int(L.load().pgsag_vote_compact_workspace_size(n))
    return torch.empty((ws_bytes + 3) // 4, dtype=torch.int32, device=device)


def compact(reliable: torch.Tensor, stream=None) -> torch.Tensor:
    """Ascending indices of the nonzero entries (pgsag_vote_compact); reads the
    count back to the host."""
    M = int(reliable.shape[0])
    dev = reliable.device
    reliable = reliable.contiguous()
    idx = torch.empty(max(M, 1), dtype=torch.int32, device=dev)
    n_out = torch.zeros(1, dtype=torch.int32, device=dev)
    status = torch.zeros(1, dtype=torch.int32, device=dev)
    compact_async(reliable, idx, n_out, compact_workspace(M, dev), status, stream)
    return idx[:int(n_out.item())]
