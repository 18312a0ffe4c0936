"""Depth fusion and TSDF integration (Sec. 4.4): CUDA path through the C-ABI vs
the oracle.  Weights are integer counts decided in float32 on both sides:
bit-exact; TSDF values: float32 sums of at most 256 terms in [-1, 1] against
float64, |error| <= 2e-5."""
from types import SimpleNamespace

import numpy as np
import pytest
import torch

import pgsag_synth as syn
from oracle import tsdf_oracle as TO

pytestmark = pytest.mark.gpu
TSDF_TOL = 2e-5


def gpu_tsdf(origin, voxel, dims, trunc, cams, depths, accumulate_from=None):
    from paper_2501_01677_b300 import tsdf as T
    sizes = [int(np.asarray(d).size) for d in depths]
    offs = np.concatenate([[0], np.cumsum(sizes)[:-1]]).astype(np.int64) if depths else []
    buf = torch.from_numpy(np.concatenate([np.asarray(d, np.float32).ravel() for d in depths])
                           if depths else np.zeros(1, np.float32)).cuda()
    nx, ny, nz = dims
    if accumulate_from is None:
        ts = torch.empty(nz, ny, nx, dtype=torch.float32, device="cuda")
        ws = torch.empty(nz, ny, nx, dtype=torch.float32, device="cuda")
    else:
        ts = torch.from_numpy(np.asarray(accumulate_from[0], np.float32)).cuda()
        ws = torch.from_numpy(np.asarray(accumulate_from[1], np.float32)).cuda()
    g = T.grid(origin, voxel, dims, trunc)
    st = T.integrate(g, cams, buf, offs, ts, ws, accumulate=accumulate_from is not None)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    return ts.cpu().numpy().astype(np.float64), ws.cpu().numpy().astype(np.float64)


def check(origin, voxel, dims, trunc, cams, depths):
    tg, wg = gpu_tsdf(origin, voxel, dims, trunc, cams, depths)
    to, wo = TO.integrate(origin, voxel, dims, trunc, cams, depths)
    np.testing.assert_array_equal(wg, wo)
    np.testing.assert_allclose(tg, to, atol=TSDF_TOL, rtol=0)
    return tg, wg


def fused_f32(w):
    # the oracle's mean fusion, handed to both sides as float32 input maps
    return [TO.fuse_mean([b, g]).astype(np.float32) for b, g in zip(w.building, w.background)]


@pytest.mark.parametrize("n_maps", [1, 2, 3, 8])
def test_depth_fuse(n_maps):
    from paper_2501_01677_b300 import tsdf as T
    rng = np.random.default_rng(n_maps)
    maps = rng.uniform(1, 100, (n_maps, 1000, 37)).astype(np.float32)
    maps[rng.random(maps.shape) < 0.3] = 0.0
    maps[rng.random(maps.shape) < 0.02] = np.nan
    maps[rng.random(maps.shape) < 0.02] = np.inf
    maps[rng.random(maps.shape) < 0.02] = -5.0
    out = T.fuse(torch.from_numpy(maps).cuda()).cpu().numpy()
    np.testing.assert_allclose(out, TO.fuse_mean(list(maps)), rtol=1e-6, atol=0)


def test_fronto_parallel_plane():
    cam = SimpleNamespace(R=np.eye(3, dtype=np.float32), t=np.zeros(3, np.float32), fx=8.0, fy=8.0, cx=8.0, cy=8.0,
                          znear=0.2, width=16, height=16)
    depth = np.full((16, 16), 5.0, np.float32)
    tg, wg = check((-0.4, -0.4, 3.0), 0.1, (8, 8, 40), 0.3, [cam], [depth])
    assert wg.sum() > 0 and (tg[wg == 0] == 1.0).all()


@pytest.mark.parametrize("dims,voxel", [((40, 40, 13), 4.0), ((37, 29, 11), 4.5), ((3, 2, 1), 30.0)])
def test_small_scene_parity(dims, voxel):
    w = syn.tsdf_workload(n_views=6, width=320, height=200, voxel=voxel, step=1)
    check(w.origin, w.voxel, dims, w.trunc, w.cams, fused_f32(w))


def test_accumulate_and_more_than_256_views():
    w = syn.tsdf_workload(n_views=300, width=64, height=40, voxel=5.0, step=1)
    maps = fused_f32(w)
    dims = (32, 32, 10)
    tg, wg = check(w.origin, w.voxel, dims, w.trunc, w.cams, maps)    # two calls inside the binding
    assert wg.max() >= 10
    # first half, then the second half on top of it
    ta, wa = gpu_tsdf(w.origin, w.voxel, dims, w.trunc, w.cams[:150], maps[:150])
    tb, wb = gpu_tsdf(w.origin, w.voxel, dims, w.trunc, w.cams[150:], maps[150:], accumulate_from=(ta, wa))
    np.testing.assert_array_equal(wb, wg)
    np.testing.assert_allclose(tb, tg, atol=TSDF_TOL)


def test_no_views_and_empty_maps():
    w = syn.tsdf_workload(n_views=2, width=64, height=40, voxel=5.0, step=1)
    tg, wg = gpu_tsdf(w.origin, w.voxel, (16, 16, 4), w.trunc, [], [])
    assert (wg == 0).all() and (tg == 1).all()
    tg, wg = check(w.origin, w.voxel, (16, 16, 4), w.trunc, w.cams, [np.zeros_like(m) for m in w.building])
    assert (wg == 0).all()


def test_full_size_sampled_voxels():
    """The bench workload (640 x 640 x 200 voxels at 0.25 m, 32 views at
    2736x1824): 1M sampled voxels against the oracle evaluated one by one."""
    w = syn.tsdf_workload()
    maps = fused_f32(w)
    tg, wg = gpu_tsdf(w.origin, w.voxel, w.dims, w.trunc, w.cams, maps)
    idx = np.random.default_rng(1).choice(tg.size, 1_000_000, replace=False)
    to, wo = TO.integrate(w.origin, w.voxel, w.dims, w.trunc, w.cams, maps, voxel_index=idx)
    np.testing.assert_array_equal(wg.ravel()[idx], wo)
    np.testing.assert_allclose(tg.ravel()[idx], to, atol=TSDF_TOL)
    assert (wo > 0).mean() > 0.05 and ((to < 0) & (wo > 0)).any()
