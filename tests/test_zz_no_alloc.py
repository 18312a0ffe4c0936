"""The allocation-free statistics entry point (pgsag_tile_stats_noalloc).

It serves callers that cannot allocate device memory -- an application or
plug-in that must take every device buffer from its own memory manager, or a
latency-critical loop that cannot afford a cudaMalloc -- by keeping its scratch
in a fixed array inside the library.  This test calls it through the C ABI and
checks it against pgsag_tile_stats (which takes its scratch from the caller) on
two calls in a row, since calls reuse the same internal array.
"""
import ctypes

import numpy as np
import pytest
import torch

import pgsag_synth as syn

pytestmark = pytest.mark.gpu


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def test_noalloc_tile_stats_matches_scratch_version_twice():
    from paper_2501_01677_b300 import _lib as L
    from paper_2501_01677_b300 import raster
    lib = L.load()
    g, views = syn.config0()
    P = raster.GaussianParams.from_numpy(g)
    plan = raster.Plan([views[0].cam], [views[0].mask], [views[0].target], g.n)
    plan.forward(P)
    plan.tile_stats()
    torch.cuda.synchronize()
    plan.check_status()
    ref_counts = plan.tile_counts.clone()
    ref_gc = plan.gc_load.clone()
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for _ in range(2):
        counts = torch.full_like(plan.tile_counts, -1)
        gc = torch.full_like(plan.gc_load, -1.0)
        rc = lib.pgsag_tile_stats_noalloc(plan.n_views, _ptr(plan.views_dev), plan.n_active, _ptr(plan.ranges),
                                          plan.n_chunks, _ptr(plan.chunks), _ptr(plan.act_tiles), _ptr(plan.px_list),
                                          _ptr(plan.aux), _ptr(plan.gc_weight), _ptr(counts), _ptr(gc),
                                          _ptr(plan.status), s)
        assert rc == 0
        torch.cuda.synchronize()
        plan.check_status()
        assert torch.equal(counts[:plan.n_active], ref_counts[:plan.n_active])
        np.testing.assert_allclose(gc.cpu().numpy(), ref_gc.cpu().numpy(), rtol=1e-6)
    # inputs beyond the fixed scratch are refused before any work is enqueued
    rc = lib.pgsag_tile_stats_noalloc(plan.n_views, _ptr(plan.views_dev), plan.n_active, _ptr(plan.ranges),
                                      L.NOALLOC_MAX_CHUNKS + 1, _ptr(plan.chunks), _ptr(plan.act_tiles),
                                      _ptr(plan.px_list), _ptr(plan.aux), _ptr(plan.gc_weight), _ptr(counts),
                                      _ptr(gc), _ptr(plan.status), s)
    assert rc == -2
