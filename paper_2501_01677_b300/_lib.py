"""ctypes binding of libpgsag.so (include/pgsag.h): argument marshalling only.

The shared library is built in-tree by paper_2501_01677_b300.build.  Loading
fails loudly if it is missing; there is no fallback implementation.
"""
from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, c_double, c_float, c_int, c_int32, c_size_t, c_uint32, c_uint64, c_void_p

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libpgsag.so")

PGSAG_OK = 0
PGSAG_DEV_CAPACITY = 1
PGSAG_DEV_TIMEOUT = 2
PGSAG_DEV_BOUNDS = 4
MAX_VIEWS = 256
CHUNK = 32
PIX_MASK, PIX_EDGE, PIX_RENDER = 1, 2, 4
NOALLOC_MAX_CHUNKS = 1 << 20

# Every entry point declared in include/pgsag.h
EXPORTS = (
    "pgsag_status_str", "pgsag_build_info", "pgsag_prep_flags", "pgsag_prep_lists", "pgsag_prep_neighbours",
    "pgsag_prep_gc_weight",
    "pgsag_preprocess", "pgsag_bin_workspace_size", "pgsag_bin", "pgsag_render_fwd", "pgsag_loss_ban",
    "pgsag_render_bwd", "pgsag_preprocess_bwd", "pgsag_tile_stats", "pgsag_tile_stats_noalloc",
    "pgsag_schedule_lpt", "pgsag_adam",
    "pgsag_vote_pack_mask", "pgsag_vote_filter", "pgsag_vote_compact_workspace_size", "pgsag_vote_compact",
    "pgsag_depth_fuse", "pgsag_tsdf_integrate", "pgsag_adam_multi",
)
TSDF_MAX_VIEWS = 256
VOTE_MAX_VIEWS = 256


class PgsagView(ctypes.Structure):
    _fields_ = [
        ("R", c_float * 9), ("t", c_float * 3),
        ("fx", c_float), ("fy", c_float), ("cx", c_float), ("cy", c_float),
        ("znear", c_float), ("reserved0", c_float * 3),
        ("width", c_int32), ("height", c_int32), ("tile_w", c_int32), ("tile_h", c_int32),
        ("tiles_x", c_int32), ("tiles_y", c_int32),
        ("g_begin", c_uint32), ("g_end", c_uint32), ("pair_base", c_uint32), ("tile_base", c_uint32),
        ("sat_base", c_uint32), ("act_base", c_uint32), ("n_active", c_uint32), ("n_mask", c_uint32),
        ("chunk_base", c_uint32), ("n_chunks", c_uint32), ("pix_base", c_uint64),
    ]


assert ctypes.sizeof(PgsagView) == 152


class PgsagSched(ctypes.Structure):
    _fields_ = [("order", c_void_p), ("counter", c_void_p), ("ctas_per_sm", c_int32), ("reserved", c_int32)]


class PgsagBanGather(ctypes.Structure):
    """pgsag_ban_gather: the deferred Eq. 8 gather done by the render adjoint (and,
    for the Eq. 11 objective, the soft-count GC-load gradient)."""
    _fields_ = [("flags_c", c_void_p), ("nbr", c_void_p), ("scratch", c_void_p), ("acc", c_void_p),
                ("lambda_ban", ctypes.c_float), ("objective", ctypes.c_uint32), ("gc_weight", c_void_p),
                ("lambda_gc", ctypes.c_float), ("reserved", ctypes.c_uint32), ("depth", c_void_p)]


assert ctypes.sizeof(PgsagBanGather) == 64
CLEAR_MAX = 5


class PgsagClear(ctypes.Structure):
    """pgsag_clear: float buffers the render adjoint sets to zero on the side."""
    _fields_ = [("ptr", c_void_p * CLEAR_MAX), ("n", c_uint64 * CLEAR_MAX)]


assert ctypes.sizeof(PgsagClear) == 80
OBJ_PG, OBJ_EQ11 = 0, 1
RENDER_SOFT_COUNT = 1
LAMBDA_GC, LAMBDA_FLAT = 0.41, 100.0


class PgsagVoteView(ctypes.Structure):
    """pgsag_vote_view: one camera of the multi-view voting filter (Sec. 4.1)."""
    _fields_ = [
        ("R", c_float * 9), ("t", c_float * 3),
        ("fx", c_float), ("fy", c_float), ("cx", c_float), ("cy", c_float), ("znear", c_float),
        ("width", c_int32), ("height", c_int32), ("words_per_row", c_uint32), ("reserved", c_uint32 * 2),
        ("mask_offset", c_uint64),
    ]


assert ctypes.sizeof(PgsagVoteView) == 96


class PgsagDepthView(ctypes.Structure):
    """pgsag_depth_view: one camera and depth map of the TSDF integration (Sec. 4.4)."""
    _fields_ = [
        ("R", c_float * 9), ("t", c_float * 3),
        ("fx", c_float), ("fy", c_float), ("cx", c_float), ("cy", c_float), ("znear", c_float),
        ("width", c_int32), ("height", c_int32), ("reserved", c_uint32 * 3), ("depth_offset", c_uint64),
    ]


assert ctypes.sizeof(PgsagDepthView) == 96


class PgsagDssim(ctypes.Structure):
    """pgsag_dssim: the masked D-SSIM term of L_rgb."""
    _fields_ = [("pidx", c_void_p), ("scratch", c_void_p), ("n_active_total", c_uint32), ("tile_w", c_int32),
                ("tile_h", c_int32), ("lam", c_float)]


assert ctypes.sizeof(PgsagDssim) == 32
LAMBDA_DSSIM = 0.2


class PgsagAdamTensor(ctypes.Structure):
    _fields_ = [("p", c_void_p), ("g", c_void_p), ("m", c_void_p), ("v", c_void_p), ("n", c_uint64),
                ("lr", c_float), ("reserved", c_uint32)]


assert ctypes.sizeof(PgsagAdamTensor) == 48


class PgsagTsdfGrid(ctypes.Structure):
    _fields_ = [("origin", c_float * 3), ("voxel", c_float), ("nx", c_uint32), ("ny", c_uint32), ("nz", c_uint32),
                ("trunc", c_float)]


assert ctypes.sizeof(PgsagTsdfGrid) == 32


_lib = None


def _sig(lib, name, res, args):
    f = getattr(lib, name)
    f.restype = res
    f.argtypes = args


def load(path: str = LIB_PATH):
    """Load libpgsag.so (raises if it is absent)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"libpgsag.so not built at {path}; run `python -m paper_2501_01677_b300.build`")
    lib = ctypes.CDLL(path)
    P = c_void_p
    _sig(lib, "pgsag_status_str", ctypes.c_char_p, [c_int])
    _sig(lib, "pgsag_build_info", ctypes.c_char_p, [])
    _sig(lib, "pgsag_prep_flags", c_int, [POINTER(PgsagView), P, P, P, P, P])
    _sig(lib, "pgsag_prep_lists", c_int, [POINTER(PgsagView), c_uint32, P, P, c_uint32, c_uint32, P, P, P, P, P, P, P])
    _sig(lib, "pgsag_prep_neighbours", c_int, [POINTER(PgsagView), P, c_uint32, c_uint32, P, P, P, P, P])
    _sig(lib, "pgsag_prep_gc_weight", c_int, [POINTER(PgsagView), P, P, c_uint32, c_uint32, P, P, P])
    _sig(lib, "pgsag_preprocess", c_int, [c_uint32, P, P, P, P, P, c_uint32, P, P, P, P, P, P, P, P, P, P])
    _sig(lib, "pgsag_bin_workspace_size", c_size_t, [c_uint32, c_uint32, c_uint64])
    _sig(lib, "pgsag_bin", c_int, [c_uint32, c_uint32, P, c_uint32, P, P, P, P, c_uint64, P, c_size_t, P, P, P, P, P])
    _sig(lib, "pgsag_render_fwd", c_int,
         [c_uint32, P, P, P, P, P, c_uint32, P, POINTER(PgsagSched), c_uint32, P, P, P, P, P])
    _sig(lib, "pgsag_loss_ban", c_int,
         [c_uint32, P, c_uint32, P, P, P, P, P, P, P, P, P, c_float, P, c_int, P, P, P, P, P, P, c_uint32, c_uint32, P,
          POINTER(PgsagDssim), P, P])
    _sig(lib, "pgsag_render_bwd", c_int,
         [c_uint32, P, P, P, P, P, c_uint32, P, POINTER(PgsagSched), P, P, P, P, POINTER(PgsagBanGather), P,
          c_uint32, P, POINTER(PgsagClear), P, P])
    _sig(lib, "pgsag_preprocess_bwd", c_int,
         [c_uint32, P, P, P, P, P, c_uint32, P, P, P, c_int, P, P, P, P, P, P, c_float, P, P])
    _sig(lib, "pgsag_tile_stats", c_int, [c_uint32, P, c_uint32, P, c_uint32, P, P, P, P, P, P, P, P, P, P, P])
    _sig(lib, "pgsag_tile_stats_noalloc", c_int, [c_uint32, P, c_uint32, P, c_uint32, P, P, P, P, P, P, P, P, P])
    _sig(lib, "pgsag_schedule_lpt", c_int, [c_uint32, P, P, P, P, P, P])
    _sig(lib, "pgsag_adam", c_int, [c_uint64, P, P, P, P, c_float, c_float, c_float, c_float, c_int32, P])
    _sig(lib, "pgsag_vote_pack_mask", c_int, [c_int32, c_int32, P, c_uint32, P, P])
    _sig(lib, "pgsag_vote_filter", c_int,
         [c_uint32, P, c_uint32, POINTER(PgsagVoteView), P, c_uint32, c_int, P, P, P, P, P])
    _sig(lib, "pgsag_vote_compact_workspace_size", c_size_t, [c_uint32])
    _sig(lib, "pgsag_vote_compact", c_int, [c_uint32, P, P, P, P, c_size_t, P, P])
    _sig(lib, "pgsag_depth_fuse", c_int, [c_uint32, P, c_uint64, P, P])
    _sig(lib, "pgsag_adam_multi", c_int, [c_uint32, POINTER(PgsagAdamTensor), c_float, c_float, c_float, P, P, P])
    _sig(lib, "pgsag_tsdf_integrate", c_int,
         [POINTER(PgsagTsdfGrid), c_uint32, POINTER(PgsagDepthView), P, c_int, P, P, P, P])
    _lib = lib
    return lib


class PgsagError(RuntimeError):
    pass


def check(rc: int, what: str):
    if rc != PGSAG_OK:
        msg = load().pgsag_status_str(rc).decode()
        raise PgsagError(f"{what} failed: {rc} ({msg})")
