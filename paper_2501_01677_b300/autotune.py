"""Launch-shape autotuner for batched sub-region steps.

Picks the tile shape and the render queue depth (persistent CTAs per SM, with or
without the longest-first order) for a set of views by timing the whole
graph-captured training step of each candidate on the actual workload, and
caches the choice in a JSON file keyed by the workload's shape and the GPU.
Results do not depend on the tile shape (the binning rule is the alpha >= 1/255
ellipse, not a tile-sized box), so the tuner only changes speed.
"""
from __future__ import annotations

import hashlib
import json
import os
import time
from dataclasses import asdict, dataclass
from typing import Dict, List, Optional, Sequence, Tuple

import numpy as np
import torch

from . import raster

TILES: Tuple[Tuple[int, int], ...] = ((8, 8), (16, 16), (16, 32))
# None: one CTA per active tile, no queue; 0: persistent with as many CTAs as the
# occupancy allows; n > 0: persistent with n CTAs per SM
QUEUE_DEPTHS: Tuple[Optional[int], ...] = (None, 0, 4, 8)


@dataclass
class LaunchShape:
    tile_w: int
    tile_h: int
    ctas_per_sm: Optional[int]  # None: plain grid; else persistent queue depth
    lpt: bool

    @property
    def tile(self) -> Tuple[int, int]:
        return (self.tile_w, self.tile_h)


def default_cache_path() -> str:
    return os.environ.get("PGSAG_AUTOTUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "pgsag", "autotune.json"))


def workload_key(cams, masks, n_gauss: int, g_ranges) -> str:
    """Signature of a workload: GPU, Gaussian count, per-view image size, mask
    pixel count and Gaussian range length."""
    h = hashlib.sha1()
    h.update(torch.cuda.get_device_name().encode())
    h.update(str(int(n_gauss)).encode())
    for v, cam in enumerate(cams):
        m = masks[v]
        nm = int(m.sum().item()) if torch.is_tensor(m) else int(np.count_nonzero(m))
        gb, ge = g_ranges[v] if g_ranges is not None else (0, n_gauss)
        h.update(f"{int(cam.width)}x{int(cam.height)}:{nm}:{ge - gb};".encode())
    return h.hexdigest()


def _load_cache(path: str) -> Dict[str, dict]:
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store_cache(path: str, key: str, entry: dict) -> None:
    cache = _load_cache(path)
    cache[key] = entry
    os.makedirs(os.path.dirname(path) or ".", exist_ok=True)
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def time_step(plan: "raster.Plan", P: "raster.GaussianParams", shape: LaunchShape, replays: int = 5) -> float:
    """ms per graph replay of the whole step on `plan` with the given queue."""
    if shape.ctas_per_sm is None:
        plan.use_plain_schedule()
    else:
        plan.use_persistent_schedule(ctas_per_sm=shape.ctas_per_sm, lpt=shape.lpt)
    grads = raster.new_param_grads(P)
    graph = plan.capture(P, grads)
    graph.replay()
    torch.cuda.synchronize()
    plan.check_status()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(replays):
        graph.replay()
    b.record()
    torch.cuda.synchronize()
    plan.check_status()
    del graph
    return a.elapsed_time(b) / replays


def autotune(cams, masks, targets, P: "raster.GaussianParams", g_ranges=None,
             tiles: Sequence[Tuple[int, int]] = TILES, queue_depths: Sequence[Optional[int]] = QUEUE_DEPTHS,
             replays: int = 5, cache_path: Optional[str] = None, use_cache: bool = True):
    """Fastest LaunchShape for these views, and the table of timings (ms per
    step).  A cached choice for the same workload key is returned without
    timing when use_cache is set; the choice is stored either way."""
    path = cache_path or default_cache_path()
    key = workload_key(cams, masks, P.n, g_ranges)
    if use_cache:
        hit = _load_cache(path).get(key)
        if hit is not None:
            return LaunchShape(**hit["shape"]), hit["table"]
    table: List[dict] = []
    best, best_ms = None, float("inf")
    for tw, th in tiles:
        plan = raster.Plan(cams, masks, targets, P.n, g_ranges=g_ranges, tile=(tw, th))
        plan.forward(P)  # sizes the duplicate capacity
        for q in queue_depths:
            for lpt in ((False,) if q is None else (True, False)):
                shape = LaunchShape(tw, th, q, lpt)
                ms = time_step(plan, P, shape, replays)
                table.append({**asdict(shape), "ms": ms})
                if ms < best_ms:
                    best, best_ms = shape, ms
        del plan
        torch.cuda.empty_cache()
    _store_cache(path, key, {"shape": asdict(best), "table": table, "when": time.strftime("%Y-%m-%dT%H:%M:%S")})
    return best, table


def plan_for(cams, masks, targets, P: "raster.GaussianParams", shape: LaunchShape, g_ranges=None):
    """A Plan with the tuned tile shape and render queue."""
    plan = raster.Plan(cams, masks, targets, P.n, g_ranges=g_ranges, tile=shape.tile)
    plan.forward(P)
    if shape.ctas_per_sm is None:
        plan.use_plain_schedule()
    else:
        plan.use_persistent_schedule(ctas_per_sm=shape.ctas_per_sm, lpt=shape.lpt)
    return plan
