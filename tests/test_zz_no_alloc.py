"""The allocation-free statistics entry point (pgsag_tile_stats_noalloc).

It serves callers that cannot allocate device memory -- an application or
plug-in that must take every device buffer from its own memory manager, or a
latency-critical loop that cannot afford a cudaMalloc -- by keeping its scratch
in a fixed array inside the library.  This test calls it through the C ABI and
checks it against pgsag_tile_stats (which takes its scratch from the caller) on
two calls in a row, since calls reuse the same internal array, on one view and
on two views of different masks (the per-view reduction walks each view's slice
of the shared array).  Free device memory must not change across the calls, and
a refused call (more chunks than the array holds) must leave the outputs as
they were.
"""
import ctypes

import numpy as np
import pytest
import torch

import pgsag_synth as syn

pytestmark = pytest.mark.gpu


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def _noalloc(lib, plan, n_chunks, counts, gc, s):
    return lib.pgsag_tile_stats_noalloc(plan.n_views, _ptr(plan.views_dev), plan.n_active, _ptr(plan.ranges),
                                        n_chunks, _ptr(plan.chunks), _ptr(plan.act_tiles), _ptr(plan.px_list),
                                        _ptr(plan.aux), _ptr(plan.gc_weight), _ptr(counts), _ptr(gc),
                                        _ptr(plan.status), s)


@pytest.mark.parametrize("n_views", [1, 2])
def test_noalloc_tile_stats_matches_scratch_version_twice(n_views):
    from paper_2501_01677_b300 import _lib as L
    from paper_2501_01677_b300 import raster
    lib = L.load()
    g, views = syn.config0()
    v = views[0]
    vs = [v, syn.View(v.cam, np.ascontiguousarray(v.mask[::-1]), v.target)][:n_views]
    P = raster.GaussianParams.from_numpy(g)
    plan = raster.Plan([x.cam for x in vs], [x.mask for x in vs], [x.target for x in vs], g.n)
    plan.forward(P)
    plan.tile_stats()
    torch.cuda.synchronize()
    plan.check_status()
    ref_counts = plan.tile_counts.clone()
    ref_gc = plan.gc_load.clone()
    assert ref_gc.numel() == n_views and bool((ref_gc > 0).all())
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    outs = [(torch.full_like(plan.tile_counts, -1), torch.full_like(plan.gc_load, -1.0)) for _ in range(2)]
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for counts, gc in outs:
        assert _noalloc(lib, plan, plan.n_chunks, counts, gc, s) == 0
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free0
        plan.check_status()
        assert torch.equal(counts[:plan.n_active], ref_counts[:plan.n_active])
        np.testing.assert_allclose(gc.cpu().numpy(), ref_gc.cpu().numpy(), rtol=1e-6)
    # inputs beyond the fixed scratch are refused before any work is enqueued
    counts, gc = outs[1]
    before = (counts.clone(), gc.clone())
    assert _noalloc(lib, plan, L.NOALLOC_MAX_CHUNKS + 1, counts, gc, s) == -2
    torch.cuda.synchronize()
    assert torch.equal(counts, before[0]) and torch.equal(gc, before[1])
    plan.check_status()
