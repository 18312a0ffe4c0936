"""Python layer over libpgsag: a Plan owns the device buffers of one set of views,
and two autograd Functions expose the differentiable renderer and the fused
render + loss step.  PyTorch supplies device memory and the stream only; every
step of the computation runs in the library's CUDA kernels.

Paper passages: Sec. 3.1 (Eq. 1-4, rendering), Sec. 4.2 (Eq. 8, boundary-aware
normal loss), Sec. 4.3 (Eq. 9, GC-load statistic; Eq. 10-11 weights).
"""
from __future__ import annotations

import ctypes
import math
from dataclasses import dataclass
from typing import List, Optional, Sequence, Tuple

import numpy as np
import torch

from . import _lib as L

LAMBDA_BAN = 0.01  # Eq. 10-11: lambda_4


def _ptr(t: Optional[torch.Tensor]):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream_ptr(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


@dataclass
class GaussianParams:
    """Raw Gaussian parameters on the GPU (float32, contiguous)."""
    means: torch.Tensor          # [N,3]
    log_scales: torch.Tensor     # [N,3]
    quats: torch.Tensor          # [N,4] (w,x,y,z)
    opacity_logit: torch.Tensor  # [N]
    sh: torch.Tensor             # [N,16,3]

    @property
    def n(self) -> int:
        return int(self.means.shape[0])

    def tensors(self):
        return (self.means, self.log_scales, self.quats, self.opacity_logit, self.sh)

    @staticmethod
    def from_numpy(g, device="cuda", requires_grad=False) -> "GaussianParams":
        ts = [torch.from_numpy(np.ascontiguousarray(getattr(g, k), np.float32)).to(device)
              for k in ("means", "log_scales", "quats", "opacity_logit", "sh")]
        if requires_grad:
            for t in ts:
                t.requires_grad_(True)
        return GaussianParams(*ts)


class Plan:
    """Device state for rendering a fixed set of views.

    cams: objects with R [3,3], t [3], fx, fy, cx, cy, width, height, znear
    masks: uint8 [H,W] building masks (host numpy or device tensors)
    targets: float32 [H,W,3] photometric targets
    g_ranges: per view (g_begin, g_end) into the shared Gaussian arrays; default
      every view renders all n_gauss Gaussians.  The plan's calls cover only the
      span [min g_begin, max g_end) of the arrays (offset pointers): a plan of one
      sub-region of a large shared array does not touch the other Gaussians; its
      gradients outside the span are left as they are (see new_grads)
    tile: (tile_w, tile_h), each in {8, 16, 32}
    capacity: maximum number of (tile, Gaussian) duplicates; None sizes it on the
      first forward (one host synchronisation) and grows it on overflow.

    Outputs of forward() live in this plan's buffers and stay valid until the
    next forward on the same plan; backward must run before that.  One plan
    therefore holds one forward in flight: the autograd Functions record the
    plan's forward count and their backward raises if another forward ran on
    the same plan in between (use one plan per concurrently live graph).
    """

    def __init__(self, cams, masks, targets, n_gauss: int, g_ranges: Optional[Sequence[Tuple[int, int]]] = None,
                 tile=(16, 16), capacity: Optional[int] = None, device="cuda"):
        self.lib = L.load()
        self.device = torch.device(device)
        V = len(cams)
        if V == 0 or V > L.MAX_VIEWS:
            raise ValueError("number of views must be in [1, 256]")
        self.n_views = V
        self.n_gauss = int(n_gauss)
        self.tile = (int(tile[0]), int(tile[1]))
        tw, th = self.tile
        views = (L.PgsagView * V)()
        pix_base = tile_base = sat_base = pair_base = 0
        self.shapes = []
        spans = [(g_ranges[v] if g_ranges is not None else (0, self.n_gauss)) for v in range(V)]
        self.g_lo = min(int(a) for a, _ in spans) if V else 0
        self.g_hi = max(int(b) for _, b in spans) if V else 0
        if not (0 <= self.g_lo <= self.g_hi <= self.n_gauss):
            raise ValueError("bad Gaussian range")
        for v, cam in enumerate(cams):
            vw = views[v]
            R = np.asarray(cam.R, np.float32).reshape(9)
            t = np.asarray(cam.t, np.float32).reshape(3)
            for i in range(9):
                vw.R[i] = float(R[i])
            for i in range(3):
                vw.t[i] = float(t[i])
            vw.fx, vw.fy, vw.cx, vw.cy = float(cam.fx), float(cam.fy), float(cam.cx), float(cam.cy)
            vw.znear = float(cam.znear)
            W, H = int(cam.width), int(cam.height)
            vw.width, vw.height, vw.tile_w, vw.tile_h = W, H, tw, th
            vw.tiles_x, vw.tiles_y = (W + tw - 1) // tw, (H + th - 1) // th
            gb, ge = spans[v]
            if not (0 <= gb <= ge <= self.n_gauss):
                raise ValueError("bad Gaussian range")
            vw.g_begin, vw.g_end = gb - self.g_lo, ge - self.g_lo  # relative to the span
            vw.pair_base = pair_base
            vw.tile_base = tile_base
            vw.sat_base = sat_base
            vw.pix_base = pix_base
            pair_base += ge - gb
            tile_base += vw.tiles_x * vw.tiles_y
            sat_base += (vw.tiles_x + 1) * (vw.tiles_y + 1)
            pix_base += W * H
            self.shapes.append((H, W))
        self.views_host = views
        self.n_pairs, self.n_tiles, self.n_sat, self.n_pix = pair_base, tile_base, sat_base, pix_base
        if self.n_pairs >= 2 ** 32 or self.n_pix >= 2 ** 40:
            raise ValueError("problem too large")
        dev = self.device
        s = _stream_ptr()
        u8, i32, f32 = torch.uint8, torch.int32, torch.float32

        # ---- mask preparation (outside the timed step)
        self.flags = torch.zeros(self.n_pix, dtype=u8, device=dev)
        self.tile_npix = torch.zeros(max(self.n_tiles, 1), dtype=i32, device=dev)
        totals = torch.zeros((V, 4), dtype=i32, device=dev)
        for v in range(V):
            m = masks[v]
            m = m if torch.is_tensor(m) else torch.from_numpy(np.ascontiguousarray(m, np.uint8))
            m = m.to(dev, torch.uint8).contiguous()
            L.check(self.lib.pgsag_prep_flags(ctypes.byref(views[v]), _ptr(m), _ptr(self.flags), _ptr(self.tile_npix),
                                                  _ptr(totals[v]), s), "pgsag_prep_flags")
        tot = totals.cpu().numpy().astype(np.int64)
        self.n_active_v = tot[:, 0].copy()
        self.n_render_v = tot[:, 1].copy()
        self.n_chunks_v = tot[:, 2].copy()
        self.n_mask_v = tot[:, 3].copy()
        self.n_active = int(tot[:, 0].sum())
        self.n_render = int(tot[:, 1].sum())
        self.n_chunks = int(tot[:, 2].sum())
        self.n_mask = int(tot[:, 3].sum())
        if self.n_render >= 2 ** 32:
            raise ValueError("too many rendered pixels for 32-bit compact indices")
        self.tile_act = torch.empty(max(self.n_tiles, 1), dtype=i32, device=dev)
        self.sat = torch.empty(max(self.n_sat, 1), dtype=i32, device=dev)
        self.act_tiles = torch.empty((max(self.n_active, 1), 4), dtype=i32, device=dev)
        self.px_list = torch.empty(max(self.n_render, 1), dtype=i32, device=dev)
        self.chunks = torch.empty((max(self.n_chunks, 1), 4), dtype=i32, device=dev)
        self.pidx = torch.empty(self.n_pix, dtype=i32, device=dev)
        self.px_base_v = np.zeros(V, np.int64)
        act_base = px_base = chunk_base = 0
        for v in range(V):
            views[v].act_base = act_base
            views[v].n_active = int(self.n_active_v[v])
            views[v].n_mask = int(self.n_mask_v[v])
            views[v].chunk_base = chunk_base
            views[v].n_chunks = int(self.n_chunks_v[v])
            self.px_base_v[v] = px_base
            L.check(self.lib.pgsag_prep_lists(ctypes.byref(views[v]), v, _ptr(self.flags), _ptr(self.tile_npix),
                                                  px_base, chunk_base, _ptr(self.tile_act), _ptr(self.sat),
                                                  _ptr(self.act_tiles), _ptr(self.px_list), _ptr(self.chunks),
                                                  _ptr(self.pidx), s),
                        "pgsag_prep_lists")
            act_base += int(self.n_active_v[v])
            px_base += int(self.n_render_v[v])
            chunk_base += int(self.n_chunks_v[v])
        # compact neighbour table and flags of the rendered pixels
        nr = max(self.n_render, 1)
        self.nbr = torch.empty((nr, 4), dtype=i32, device=dev)
        self.flags_c = torch.zeros(nr, dtype=u8, device=dev)
        for v in range(V):
            L.check(self.lib.pgsag_prep_neighbours(ctypes.byref(views[v]), _ptr(self.px_list), int(self.px_base_v[v]),
                                                       int(self.n_render_v[v]), _ptr(self.flags), _ptr(self.pidx),
                                                       _ptr(self.nbr), _ptr(self.flags_c), s),
                        "pgsag_prep_neighbours")
        # targets and GC weights of the rendered pixels (compact layout); each
        # view's full image is on the device only while it is gathered
        self.target = torch.zeros(nr * 3, dtype=f32, device=dev)
        self.gc_weight = torch.ones(nr, dtype=f32, device=dev)
        for v in range(V):
            tg = targets[v]
            tg = tg if torch.is_tensor(tg) else torch.from_numpy(np.ascontiguousarray(tg, np.float32))
            H, W = self.shapes[v]
            tg = tg.reshape(H * W * 3).to(dev, f32).contiguous()
            L.check(self.lib.pgsag_prep_gc_weight(ctypes.byref(views[v]), _ptr(tg), _ptr(self.px_list),
                                                      int(self.px_base_v[v]), int(self.n_render_v[v]),
                                                      _ptr(self.target), _ptr(self.gc_weight), s),
                        "pgsag_prep_gc_weight")
            del tg
        raw = bytes(views)
        self.views_dev = torch.frombuffer(bytearray(raw), dtype=torch.uint8).to(dev)

        # ---- per-pixel buffers, compact: row q belongs to the pixel px_list[q]
        self.out8 = torch.zeros((nr, 8), dtype=f32, device=dev)
        self.depth = torch.zeros(nr, dtype=f32, device=dev)
        self.aux = torch.zeros((nr, 4), dtype=i32, device=dev)
        self.dout8 = torch.zeros((nr, 8), dtype=f32, device=dev)
        self.scratch = torch.zeros((nr, 6), dtype=f32, device=dev)
        # ---- per-pair buffers
        npairs = max(self.n_pairs, 1)
        self.rec = torch.empty((npairs, 16), dtype=f32, device=dev)
        self.dkey = torch.empty(npairs, dtype=i32, device=dev)
        self.bininfo = torch.empty((npairs, 4), dtype=i32, device=dev)
        self.tile_mask = torch.empty(npairs, dtype=torch.int64, device=dev)
        self.grad2d = torch.empty((npairs, 16), dtype=f32, device=dev)
        self._grad2d_clear = False  # True between a projection and the next render adjoint
        # ---- per-tile / per-view
        self.ranges = torch.zeros((max(self.n_active, 1), 2), dtype=i32, device=dev)
        self.tile_counts = torch.zeros(max(self.n_active, 1), dtype=i32, device=dev)
        self.k_out = torch.zeros(1, dtype=torch.int64, device=dev)
        self.status = torch.zeros(1, dtype=i32, device=dev)
        self.acc_loss = torch.zeros(8 * (V + 1), dtype=torch.float64, device=dev)
        self.objective = "pg"
        self.dssim_lambda = 0.0
        self.ssim_scratch = None
        self.acc_gc = torch.zeros(3 * V, dtype=torch.float64, device=dev)
        self.chunk_scratch = torch.zeros((max(self.n_chunks, 1), 8), dtype=f32, device=dev)
        self.gc_load = torch.zeros(V, dtype=f32, device=dev)
        self.loss_buf = torch.zeros(3 * V + 1, dtype=f32, device=dev)
        self.sched = None
        self.sched_order = None
        self.sched_counter = torch.zeros(1, dtype=i32, device=dev)
        self.stage_events = None  # list -> (name, start event, end event) per step call
        self.forward_count = 0  # projections run on this plan (each starts a new forward)
        self._auto_capacity = capacity is None
        self._alloc_capacity(int(capacity) if capacity is not None else max(4 * self.n_pairs, 1 << 16))

    # ------------------------------------------------------------------ buffers
    def _alloc_capacity(self, cap: int):
        self.capacity = int(max(cap, 1))
        self.dup_pairs = torch.empty(self.capacity, dtype=torch.int32, device=self.device)
        nbytes = int(self.lib.pgsag_bin_workspace_size(self.n_pairs, self.n_active, self.capacity))
        self.ws = torch.empty(nbytes, dtype=torch.uint8, device=self.device)

    def use_persistent_schedule(self, ctas_per_sm: int = 0, lpt: bool = True):
        """Render with a persistent grid (ctas_per_sm x SMs CTAs; 0: as many as
        the kernels' occupancy allows) pulling active tiles from a device work
        counter; with lpt=True the tiles are handed out longest first
        (pgsag_schedule_lpt, recomputed after every binning)."""
        self.lpt = bool(lpt)
        if self.lpt:
            self.sched_order = torch.empty(max(self.n_active, 1), dtype=torch.int32, device=self.device)
            self.lpt_ws = torch.zeros(64, dtype=torch.int32, device=self.device)
        else:
            self.sched_order = None
        self.sched = L.PgsagSched(self.sched_order.data_ptr() if self.lpt else None, self.sched_counter.data_ptr(),
                                  int(ctas_per_sm), 0)

    def use_plain_schedule(self):
        self.sched = None
        self.sched_order = None
        self.lpt = False

    def schedule(self, stream=None):
        """Longest-first tile order for the persistent render launches."""
        if self.sched is None or not getattr(self, "lpt", False):
            return
        s = _stream_ptr(stream)
        with self._ev('schedule'):
            L.check(self.lib.pgsag_schedule_lpt(self.n_active, _ptr(self.ranges), _ptr(self.act_tiles),
                                                _ptr(self.lpt_ws), _ptr(self.sched_order), _ptr(self.status), s),
                    "pgsag_schedule_lpt")

    def _sched_arg(self):
        return ctypes.byref(self.sched) if self.sched is not None else None

    # ------------------------------------------------------------------ step calls
    def _ev(self, name):
        """Record CUDA events around a step call on the current stream when
        stage_events is a list (profiling); a no-op otherwise."""
        plan = self

        class _Ctx:
            def __enter__(self_):
                if plan.stage_events is not None:
                    self_.a = torch.cuda.Event(enable_timing=True)
                    self_.a.record()

            def __exit__(self_, *exc):
                if plan.stage_events is not None:
                    b = torch.cuda.Event(enable_timing=True)
                    b.record()
                    plan.stage_events.append((name, self_.a, b))
        return _Ctx()

    def kernel_launches_per_step(self, with_stats=True) -> int:
        """Number of library kernels one step (step() / RenderLossFn) launches: the
        fused loss sums the GC-load and leaves the Eq. 8 gather to render_bwd."""
        n = 1  # preprocess
        if self.n_pairs and self.n_active:
            n += 7                              # bin: counter clear, emit, tile scan (2), scatter, sorts (2)
        if self.sched is not None and getattr(self, "lpt", False) and self.n_active:
            n += 3                              # schedule
        n += 1 if self.n_active else 0          # render_fwd
        n += (2 if self.n_chunks else 0) + 1    # loss pass A (+ GC-load sums), per-view reduce, final
        if self.objective == "eq11" and self.n_gauss:
            n += 1                              # flattening-loss sum
        if self.dssim_lambda and self.n_active:
            n += 2                              # D-SSIM window sums and their adjoint
        if with_stats:
            n += 1 if self.n_active else 0      # per-tile counts
        n += 1 if self.n_active else 0          # render_bwd
        n += 1 if self.n_gauss else 0           # preprocess_bwd
        return n

    def status_value(self) -> int:
        return int(self.status.item())

    def k_value(self) -> int:
        return int(self.k_out.item())

    def _span(self, P: GaussianParams):
        """(n, pointers of means, log_scales, quats, opacity_logit, sh) of the
        plan's Gaussian span of P's arrays (or of gradient arrays shaped like
        them)."""
        if P.n != self.n_gauss:
            raise ValueError(f"the plan was built for {self.n_gauss} Gaussians, got {P.n}")
        lo = self.g_lo
        ptrs = [ctypes.c_void_p(t.data_ptr() + lo * (t.numel() // max(P.n, 1)) * t.element_size())
                for t in P.tensors()]
        return (self.g_hi - lo, *ptrs)

    def new_grads(self, P: GaussianParams):
        """Gradient buffers for this plan's preprocess_bwd (accumulate=False):
        uninitialised when the plan's span covers all of P (every row is then
        written), zeros otherwise (rows outside the span are not touched)."""
        if (self.g_lo, self.g_hi) == (0, P.n):
            return new_param_grads(P)
        return [torch.zeros_like(t) for t in P.tensors()]

    def clearable(self, grads: Sequence[torch.Tensor]):
        """grads if the render adjoint can clear them for preprocess_bwd(cleared=True)
        (the plan's span covers every row and each buffer starts on 16 bytes), else
        None (preprocess_bwd then overwrites every row of the span itself)."""
        if (self.g_lo, self.g_hi) != (0, self.n_gauss) or any(t.data_ptr() % 16 for t in grads):
            return None
        return grads

    def backward_grads(self, P: GaussianParams):
        """(grads, clear, cleared) for an autograd backward: the buffers, what the
        render adjoint must clear, and whether preprocess_bwd may take them as
        zeros (new_grads returns zero-filled buffers for a partial span)."""
        grads = self.new_grads(P)
        full = (self.g_lo, self.g_hi) == (0, P.n)
        clear = self.clearable(grads) if full else None
        return grads, clear, (clear is not None) or not full

    def preprocess(self, P: GaussianParams, stream=None):
        s = _stream_ptr(stream)
        self.forward_count += 1
        with self._ev('preprocess'):
            n, means, log_scales, quats, opacity_logit, sh = self._span(P)
            L.check(self.lib.pgsag_preprocess(n, means, log_scales, quats, opacity_logit, sh, self.n_views, _ptr(self.views_dev), _ptr(self.tile_act),
                                              _ptr(self.sat), _ptr(self.rec), _ptr(self.dkey), _ptr(self.bininfo),
                                              _ptr(self.tile_mask), _ptr(self.grad2d), _ptr(self.status), s),
                    "pgsag_preprocess")
        # the binned pairs' rows of grad2d are zero until the next render adjoint
        self._grad2d_clear = True

    def bin(self, stream=None):
        s = _stream_ptr(stream)
        with self._ev('bin'):
            L.check(self.lib.pgsag_bin(self.n_pairs, self.n_views, _ptr(self.views_dev), self.n_active, _ptr(self.tile_act),
                                       _ptr(self.tile_mask), _ptr(self.bininfo), _ptr(self.dkey), self.capacity, _ptr(self.ws),
                                       self.ws.numel(),
                                       _ptr(self.dup_pairs), _ptr(self.ranges), _ptr(self.k_out), _ptr(self.status), s),
                    "pgsag_bin")

    def set_objective(self, objective: str):
        """"pg": the step differentiates L_rgb + lambda_4 L_ban (the GC-load is a
        value from the integer count).  "eq11": Eq. 10-11 over the locally defined
        terms, (1 - lambda)(L_rgb + lambda_3 L_s + lambda_4 L_ban) + lambda GC-load
        with the soft count, all differentiated."""
        if objective not in ("pg", "eq11"):
            raise ValueError(objective)
        self.objective = objective

    def set_dssim(self, lam: float = L.LAMBDA_DSSIM):
        """L_rgb = (1 - lam) L1 + lam (1 - SSIM_M) with the masked D-SSIM (3DGS's
        photometric loss restricted to the building mask); lam = 0 turns it off.
        Needs the dense pixel map (not released)."""
        if lam and self.pidx is None:
            raise ValueError("the D-SSIM term needs the dense pixel map (release_prep_buffers was called)")
        self.dssim_lambda = float(lam)
        if lam and self.ssim_scratch is None:
            self.ssim_scratch = torch.zeros(max(self.n_render, 1) * 9, dtype=torch.float32, device=self.device)

    def _dssim_arg(self):
        if not self.dssim_lambda:
            return None
        tw, th = self.tile
        return ctypes.byref(L.PgsagDssim(self.pidx.data_ptr(), self.ssim_scratch.data_ptr(), self.n_active, tw, th,
                                         self.dssim_lambda))

    def render_fwd(self, stream=None):
        s = _stream_ptr(stream)
        flags = L.RENDER_SOFT_COUNT if self.objective == "eq11" else 0
        with self._ev('render_fwd'):
            L.check(self.lib.pgsag_render_fwd(self.n_views, _ptr(self.views_dev), _ptr(self.rec), _ptr(self.dup_pairs),
                                              _ptr(self.ranges), _ptr(self.act_tiles), self.n_active,
                                              _ptr(self.px_list), self._sched_arg(), flags, _ptr(self.out8),
                                              _ptr(self.depth), _ptr(self.aux), _ptr(self.status), s),
                    "pgsag_render_fwd")

    def loss(self, lambda_ban=LAMBDA_BAN, loss_out: Optional[torch.Tensor] = None, stream=None,
             fused: bool = False, P: Optional[GaussianParams] = None):
        """L_rgb + lambda L_ban per view (Eq. 8) and its gradient on the rendered
        channels into dout8.  fused=True also sums the GC-load (Eq. 9) in the same
        pass and leaves the neighbour gather of Eq. 8 to the next render_bwd
        (which must then be called with ban=True).  With the "eq11" objective
        (fused only) the values follow Eq. 11 and P gives the flattening term."""
        s = _stream_ptr(stream)
        out = self.loss_buf if loss_out is None else loss_out
        self._lambda_ban = float(lambda_ban)
        eq11 = self.objective == "eq11"
        if eq11 and not fused:
            raise ValueError("the eq11 objective needs the fused loss")
        with self._ev('loss'):
            L.check(self.lib.pgsag_loss_ban(self.n_views, _ptr(self.views_dev), self.n_chunks, _ptr(self.chunks),
                                            _ptr(self.act_tiles), _ptr(self.px_list), _ptr(self.flags_c),
                                            _ptr(self.nbr), _ptr(self.out8), _ptr(self.depth), _ptr(self.aux),
                                            _ptr(self.target), float(lambda_ban),
                                            _ptr(self.gc_weight) if fused else None, 0 if fused else 1,
                                            _ptr(self.scratch), _ptr(self.acc_loss), _ptr(self.chunk_scratch),
                                            _ptr(out), _ptr(self.gc_load) if fused else None, _ptr(self.dout8),
                                            L.OBJ_EQ11 if eq11 else L.OBJ_PG,
                                            self.g_hi - self.g_lo if (eq11 and P is not None) else 0,
                                            self._span(P)[2] if (eq11 and P is not None) else None,
                                            self._dssim_arg(), _ptr(self.status), s), "pgsag_loss_ban")
        return out

    def tile_stats(self, stream=None, counts_only: bool = False):
        """Per-tile Gaussian counts and (unless counts_only) the per-view GC-load (Eq. 9)."""
        s = _stream_ptr(stream)
        with self._ev('tile_stats'):
            L.check(self.lib.pgsag_tile_stats(self.n_views, _ptr(self.views_dev), self.n_active, _ptr(self.ranges),
                                              self.n_chunks, _ptr(self.chunks), _ptr(self.act_tiles),
                                              _ptr(self.px_list), _ptr(self.aux), _ptr(self.gc_weight),
                                              _ptr(self.tile_counts), _ptr(self.acc_gc), _ptr(self.chunk_scratch),
                                              None if counts_only else _ptr(self.gc_load), _ptr(self.status), s),
                    "pgsag_tile_stats")

    def _ban_gather(self):
        eq11 = self.objective == "eq11"
        return L.PgsagBanGather(self.flags_c.data_ptr(), self.nbr.data_ptr(), self.scratch.data_ptr(),
                                self.acc_loss.data_ptr(), float(getattr(self, "_lambda_ban", LAMBDA_BAN)),
                                L.OBJ_EQ11 if eq11 else L.OBJ_PG, self.gc_weight.data_ptr() if eq11 else None,
                                L.LAMBDA_GC, 0, self.depth.data_ptr())

    def render_bwd(self, dout8: torch.Tensor, ddepth: Optional[torch.Tensor] = None,
                   dout_scale: Optional[torch.Tensor] = None, stream=None, ban: bool = False,
                   clear: Optional[Sequence[torch.Tensor]] = None):
        """Adjoint render into grad2d.  ban=True: dout8 comes from loss(fused=True)
        and the deferred Eq. 8 gather runs in this kernel's prologue.  clear: the
        raw-parameter gradient buffers of this step (shaped like P's tensors),
        whose rows in the plan's span the kernel sets to zero on the side, for a
        following preprocess_bwd(cleared=True)."""
        s = _stream_ptr(stream)
        bg = ctypes.byref(self._ban_gather()) if ban else None
        cl = None
        if clear is not None:
            n, *ptrs = self._span(GaussianParams(*clear))
            per_row = [t.numel() // max(self.n_gauss, 1) for t in clear]
            cl = ctypes.byref(L.PgsagClear((ctypes.c_void_p * L.CLEAR_MAX)(*[p.value for p in ptrs]),
                                           (ctypes.c_uint64 * L.CLEAR_MAX)(*[n * r for r in per_row])))
        # after a projection the binned rows are already zero: no full clear
        n_clear = 0 if self._grad2d_clear else self.n_pairs
        self._grad2d_clear = False
        with self._ev('render_bwd'):
            L.check(self.lib.pgsag_render_bwd(self.n_views, _ptr(self.views_dev), _ptr(self.rec), _ptr(self.dup_pairs),
                                              _ptr(self.ranges), _ptr(self.act_tiles), self.n_active,
                                              _ptr(self.px_list), self._sched_arg(), _ptr(self.out8), _ptr(self.aux),
                                              _ptr(dout8), _ptr(ddepth), bg, _ptr(dout_scale), n_clear,
                                              _ptr(self.grad2d), cl, _ptr(self.status), s), "pgsag_render_bwd")

    def preprocess_bwd(self, P: GaussianParams, grads: Sequence[torch.Tensor], accumulate=False, stream=None,
                       dout_scale: Optional[torch.Tensor] = None, cleared: bool = False):
        """Chain rule into the raw-parameter gradients `grads`: overwritten, added
        to (accumulate=True), or, with cleared=True, taken as zeros already (a
        render_bwd(clear=grads) or zero-filled buffers) so that only the rows of
        the Gaussians with a binned pair are written."""
        s = _stream_ptr(stream)
        mode = 1 if accumulate else (2 if cleared else 0)
        gm, gl, gq, go, gs = grads
        # Eq. 11: the flattening term (1 - lambda) lambda_3 L_s
        fw = (1.0 - L.LAMBDA_GC) * L.LAMBDA_FLAT if self.objective == "eq11" else 0.0
        with self._ev('preprocess_bwd'):
            n, means, log_scales, quats, opacity_logit, sh = self._span(P)
            _, gm, gl, gq, go, gs = self._span(GaussianParams(gm, gl, gq, go, gs))
            L.check(self.lib.pgsag_preprocess_bwd(n, means, log_scales, quats, opacity_logit, sh, self.n_views,
                                                  _ptr(self.views_dev), _ptr(self.bininfo), _ptr(self.grad2d),
                                                  mode, gm, gl, gq, go, gs, _ptr(dout_scale), fw,
                                                  _ptr(self.status), s),
                    "pgsag_preprocess_bwd")

    def forward(self, P: GaussianParams, check: bool = True, stream=None):
        """preprocess -> bin -> render_fwd.  With check=True (or while the capacity
        is being sized) the host synchronises once to read the device status and
        grows the duplicate capacity if it overflowed."""
        for _ in range(3):
            self.preprocess(P, stream)
            self.bin(stream)
            if not (check or self._auto_capacity):
                break
            st = self.status_value()
            if st & L.PGSAG_DEV_CAPACITY:
                self._alloc_capacity(int(self.k_value() * 1.25) + 1024)
                continue
            if st:
                raise L.PgsagError(f"device status {st} after binning")
            if self._auto_capacity:
                self._auto_capacity = False
            break
        self.schedule(stream)
        self.render_fwd(stream)

    def step(self, P: GaussianParams, grads: Sequence[torch.Tensor], lambda_ban: float = LAMBDA_BAN,
             loss_out: Optional[torch.Tensor] = None, accumulate: bool = False, stream=None):
        """One whole step through the library with no host synchronisation:
        preprocess, bin, (schedule), render, loss, statistics, render adjoint,
        preprocess adjoint into `grads`.  The duplicate capacity must already be
        sized (one forward(check=True) first)."""
        self.preprocess(P, stream)
        self.bin(stream)
        self.schedule(stream)
        self.render_fwd(stream)
        self.loss(lambda_ban, loss_out, stream, fused=True, P=P)
        self.tile_stats(stream, counts_only=True)
        clear = None if accumulate else self.clearable(grads)
        self.render_bwd(self.dout8, None, None, stream, ban=True, clear=clear)
        self.preprocess_bwd(P, grads, accumulate, stream, cleared=clear is not None)

    def capture(self, P: GaussianParams, grads: Sequence[torch.Tensor], lambda_ban: float = LAMBDA_BAN):
        """CUDA graph of one whole step (see step); replay() runs it."""
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            self.step(P, grads, lambda_ban)
        torch.cuda.current_stream().wait_stream(side)
        torch.cuda.synchronize()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph):
            self.step(P, grads, lambda_ban)
        return graph

    def release_prep_buffers(self):
        """Free the dense pixel-index map (4 B per image pixel): only mask
        preparation reads it; the step kernels use the compact neighbour table."""
        self.pidx = None
        torch.cuda.empty_cache()

    def device_bytes(self) -> dict:
        """Bytes of this plan's device buffers, grouped as: dense per image pixel
        (flags, pixel-index map), compact per rendered pixel, per (view,
        Gaussian) pair, per duplicate (tile lists and sort workspace), and the
        rest (per tile, per view)."""
        groups = {
            "dense_pixel": ("flags", "pidx"),
            "compact_pixel": ("px_list", "nbr", "flags_c", "target", "gc_weight", "out8", "depth", "aux", "dout8",
                              "scratch", "chunks", "chunk_scratch"),
            "pair": ("rec", "dkey", "bininfo", "tile_mask", "grad2d"),
            "duplicate": ("dup_pairs", "ws"),
        }
        out, seen = {}, set()
        for grp, names in groups.items():
            out[grp] = 0
            for n in names:
                t = getattr(self, n, None)
                if torch.is_tensor(t):
                    out[grp] += t.numel() * t.element_size()
                    seen.add(n)
        out["other"] = sum(t.numel() * t.element_size() for n, t in vars(self).items()
                           if torch.is_tensor(t) and t.is_cuda and n not in seen)
        return out

    def check_status(self):
        st = self.status_value()
        if st:
            raise L.PgsagError(f"device status {st}")

    # ------------------------------------------------------------------ views of outputs
    def pix_slice(self, v: int):
        """Slice of view v in the dense per-pixel arrays (flags, pidx)."""
        pb = int(self.views_host[v].pix_base)
        H, W = self.shapes[v]
        return slice(pb, pb + H * W)

    def px_slice(self, v: int):
        """Slice of view v in the compact per-pixel arrays (out8, depth, aux, ...)."""
        b = int(self.px_base_v[v])
        return slice(b, b + int(self.n_render_v[v]))

    def px_index(self, v: int) -> torch.Tensor:
        """Linear pixel index y * W + x (int64) of each of view v's compact rows."""
        return self.px_list[self.px_slice(v)].long()

    def scatter_image(self, v: int, rows: torch.Tensor) -> torch.Tensor:
        """Dense [H, W, ...] image of view v from its compact rows (zeros outside R)."""
        H, W = self.shapes[v]
        out = torch.zeros((H * W,) + tuple(rows.shape[1:]), dtype=rows.dtype, device=rows.device)
        out[self.px_index(v)] = rows
        return out.view((H, W) + tuple(rows.shape[1:]))

    def images(self, v: int):
        """Dense images of view v: rgb [H,W,3], dist [H,W], normal [H,W,3], alpha
        [H,W], depth [H,W], n_contrib [H,W], final_T, and soft_count (sum of the
        blended alphas) under the "eq11" objective or ray_dot (Eq. 4's -N . r)
        under the default one (zero outside the rendered set)."""
        sl = self.px_slice(v)
        o = self.scatter_image(v, self.out8[sl])
        aux = self.scatter_image(v, self.aux[sl])
        last = aux[..., 3].contiguous().view(torch.float32)
        out = dict(rgb=o[..., 0:3], dist=o[..., 3], normal=o[..., 4:7], alpha=o[..., 7],
                   depth=self.scatter_image(v, self.depth[sl]), n_contrib=aux[..., 2],
                   final_T=aux[..., 0].contiguous().view(torch.float32))
        out["soft_count" if self.objective == "eq11" else "ray_dot"] = last
        return out

    def flags_image(self, v: int):
        H, W = self.shapes[v]
        return self.flags[self.pix_slice(v)].view(H, W)


def new_param_grads(P: GaussianParams):
    """Gradient buffers for pgsag_preprocess_bwd, which overwrites every element
    (uninitialised: a step whose device status is set skips its kernels, so its
    gradients are meaningful only once the status reads zero)."""
    return [torch.empty_like(t) for t in P.tensors()]


def _check_same_forward(ctx):
    if ctx.plan.forward_count != ctx.forward_count:
        raise RuntimeError("another forward ran on this Plan after the one being differentiated: its buffers "
                           "(outputs, upstream gradients, projected records) now hold the newer forward; "
                           "use one Plan per live autograd graph")


def _finish_backward(ctx):
    """check=True: read the device status once (one host synchronisation) and
    raise if any kernel of the step flagged an error, since the kernels then
    skipped their work and the gradients are not valid.  check=False (CUDA-graph
    capture): the caller must call plan.check_status() before using them."""
    if ctx.check:
        ctx.plan.check_status()


class RenderLossFn(torch.autograd.Function):
    """Fused masked render + loss:  params -> sum over views of
    L_rgb + lambda_4 L_ban  (Eq. 8, Eq. 10 restricted to the L1 photometric and
    boundary-aware normal terms), or with plan.set_objective("eq11") Eq. 11's
    (1 - lambda)(L_rgb + lambda_3 L_s + lambda_4 L_ban) + lambda GC-load.  Backward runs the adjoint renderer on the
    gradient the loss kernel produced and the preprocess adjoint.

    The plan's buffers carry the state between forward and backward, so no other
    forward may run on the plan before this one's backward (it raises if one
    did).  With check=False the step never synchronises the host; the gradients
    are then valid only once plan.check_status() reports no device error."""

    @staticmethod
    def forward(ctx, plan: Plan, lambda_ban: float, check: bool, means, log_scales, quats, opacity_logit, sh):
        P = GaussianParams(means, log_scales, quats, opacity_logit, sh)
        plan.forward(P, check=check)
        out = torch.empty(3 * plan.n_views + 1, dtype=torch.float32, device=plan.device)
        plan.loss(lambda_ban, loss_out=out, fused=True, P=P)
        plan.tile_stats(counts_only=True)
        ctx.plan = plan
        ctx.P = P
        ctx.per_view = out
        ctx.check = bool(check)
        ctx.forward_count = plan.forward_count
        return out[3 * plan.n_views]

    @staticmethod
    def backward(ctx, g):
        plan, P = ctx.plan, ctx.P
        _check_same_forward(ctx)
        g = g.contiguous().to(torch.float32)
        grads, clear, cleared = plan.backward_grads(P)
        plan.render_bwd(plan.dout8, None, g, ban=True, clear=clear)
        plan.preprocess_bwd(P, grads, dout_scale=g, cleared=cleared)
        _finish_backward(ctx)
        return (None, None, None) + tuple(grads)


class RenderFn(torch.autograd.Function):
    """Differentiable masked renderer: params -> (out8 [n_render, 8] = {rgb, dist,
    normal, alpha}, depth [n_render]) for all views' rendered pixels (Eq. 1-4),
    row q holding the pixel plan.px_list[q] (view by plan.px_slice).

    The returned tensors are the plan's own output buffers (no copy): the next
    forward on the same plan overwrites them, and backward raises if such a
    forward ran before it.  With check=False the gradients are valid only once
    plan.check_status() reports no device error."""

    @staticmethod
    def forward(ctx, plan: Plan, check: bool, means, log_scales, quats, opacity_logit, sh):
        P = GaussianParams(means, log_scales, quats, opacity_logit, sh)
        plan.forward(P, check=check)
        ctx.plan = plan
        ctx.P = P
        ctx.check = bool(check)
        ctx.forward_count = plan.forward_count
        return plan.out8.detach(), plan.depth.detach()

    @staticmethod
    def backward(ctx, g_out8, g_depth):
        plan, P = ctx.plan, ctx.P
        _check_same_forward(ctx)
        if g_out8 is None:
            g_out8 = torch.zeros_like(plan.out8)
        g_out8 = g_out8.contiguous()
        if g_depth is not None:
            g_depth = g_depth.contiguous()
        grads, clear, cleared = plan.backward_grads(P)
        plan.render_bwd(g_out8, g_depth, None, clear=clear)
        plan.preprocess_bwd(P, grads, cleared=cleared)
        _finish_backward(ctx)
        return (None, None) + tuple(grads)


def render_loss(plan: Plan, P: GaussianParams, lambda_ban: float = LAMBDA_BAN, check: bool = True):
    return RenderLossFn.apply(plan, lambda_ban, check, *P.tensors())


def render(plan: Plan, P: GaussianParams, check: bool = True):
    return RenderFn.apply(plan, check, *P.tensors())


def adam_step(params: Sequence[torch.Tensor], grads: Sequence[torch.Tensor], m: Sequence[torch.Tensor],
              v: Sequence[torch.Tensor], lr, step: int, beta1=0.9, beta2=0.999, eps=1e-15, stream=None):
    """Fused Adam over each parameter tensor (per-tensor learning rates allowed)."""
    lib = L.load()
    s = _stream_ptr(stream)
    lrs = lr if isinstance(lr, (list, tuple)) else [lr] * len(params)
    for p, g, mm, vv, l in zip(params, grads, m, v, lrs):
        L.check(lib.pgsag_adam(p.numel(), _ptr(p), _ptr(g), _ptr(mm), _ptr(vv), float(l), float(beta1), float(beta2),
                               float(eps), int(step), s), "pgsag_adam")
