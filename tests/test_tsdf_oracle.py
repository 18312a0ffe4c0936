"""Pins of the depth-fusion / TSDF oracle (Sec. 4.4) against facts fixed outside
it: the closed-form TSDF of a fronto-parallel plane, the zero crossing at the
surface, the sign of the field around a tilted plane seen by a rotated camera
(depth maps from the inverse camera model in float64), weights of repeated
views, accumulation across calls, and the mean fusion closed form."""
from types import SimpleNamespace

import numpy as np
import pytest
from scipy.spatial.transform import Rotation

import pgsag_synth as syn
from oracle import tsdf_oracle as TO


def ident_cam(W=16, H=16, f=8.0):
    return SimpleNamespace(R=np.eye(3, dtype=np.float32), t=np.zeros(3, np.float32), fx=f, fy=f, cx=W / 2, cy=H / 2,
                           znear=0.2, width=W, height=H)


def test_fuse_mean_closed_form():
    a = np.array([[1.0, 0.0, 2.0, np.nan], [4.0, 0.0, -1.0, 3.0]], np.float32)
    b = np.array([[3.0, 0.0, 0.0, 5.0], [np.inf, 2.0, 1.0, 0.0]], np.float32)
    f = TO.fuse_mean([a, b])
    np.testing.assert_allclose(f, [[2.0, 0.0, 2.0, 5.0], [4.0, 2.0, 1.0, 3.0]])
    assert TO.fuse_mean([a])[0, 1] == 0.0


def test_fronto_parallel_plane_closed_form():
    D, mu, s = 5.0, 0.4, 0.1
    cam = ident_cam()
    depth = np.full((16, 16), D, np.float32)
    # one column of voxels on the optical axis, centres z = 3.05 .. 7.95
    origin, dims = (-0.05, -0.05, 3.0), (1, 1, 50)
    tsdf, w = TO.integrate(origin, s, dims, mu, [cam], [depth])
    z = 3.0 + (np.arange(50) + 0.5) * 0.1
    sdf = D - z
    used = sdf >= -mu - 1e-6
    np.testing.assert_array_equal(w[:, 0, 0], used.astype(float))
    np.testing.assert_allclose(tsdf[used, 0, 0], np.minimum(1.0, sdf[used] / mu), atol=2e-6)
    assert (tsdf[~used, 0, 0] == 1.0).all()
    # a mesher's zero crossing sits on the plane
    zc = TO.zero_crossing_along_z(tsdf[:, 0, 0], z)
    assert zc == pytest.approx(D, abs=1e-5)


def test_repeated_views_average_and_count():
    cam = ident_cam()
    depth = np.full((16, 16), 5.0, np.float32)
    args = ((-0.4, -0.4, 3.0), 0.1, (8, 8, 40), 0.3)
    t1, w1 = TO.integrate(*args, [cam], [depth])
    t2, w2 = TO.integrate(*args, [cam, cam], [depth, depth])
    np.testing.assert_allclose(t2, t1, atol=1e-15)
    np.testing.assert_array_equal(w2, 2 * w1)
    # a view without depth leaves the field untouched
    t3, w3 = TO.integrate(*args, [cam, cam], [depth, np.zeros_like(depth)])
    np.testing.assert_allclose(t3, t1, atol=1e-15)
    np.testing.assert_array_equal(w3, w1)


def test_accumulation_across_calls_equals_one_call():
    w = syn.tsdf_workload(n_views=4, width=160, height=120, voxel=4.0, step=1)
    args = (w.origin, w.voxel, w.dims, w.trunc)
    ta, wa = TO.integrate(*args, w.cams[:2], w.building[:2])
    tb, wb = TO.integrate(*args, w.cams[2:], w.building[2:], tsdf0=ta, weight0=wa)
    tc, wc = TO.integrate(*args, w.cams, w.building)
    np.testing.assert_array_equal(wb, wc)
    np.testing.assert_allclose(tb, tc, atol=1e-12)
    assert wc.max() >= 2 and (wc > 0).mean() > 0.001
    # subset evaluation equals the full grid at those voxels
    idx = np.random.default_rng(0).choice(wc.size, 500, replace=False)
    ts, ws = TO.integrate(*args, w.cams, w.building, voxel_index=idx)
    np.testing.assert_allclose(ts, tc.ravel()[idx], atol=1e-15)
    np.testing.assert_array_equal(ws, wc.ravel()[idx])


@pytest.mark.parametrize("seed", [0, 1])
def test_sign_around_a_tilted_plane_seen_by_a_rotated_camera(seed):
    """Depth maps from the inverse camera model (float64 ray-plane intersection
    through each pixel centre); voxels clearly in front of the plane (along the
    camera z) get a positive TSDF, voxels clearly behind (within the truncation)
    a negative one."""
    rng = np.random.default_rng(seed)
    W, H, f = 64, 48, 60.0
    Rm = Rotation.from_euler("xyz", rng.uniform(-0.3, 0.3, 3)).as_matrix()
    campos = np.array([0.0, 0.0, -10.0]) + rng.uniform(-1, 1, 3)
    t = -Rm @ campos
    cam = SimpleNamespace(R=Rm.astype(np.float32), t=t.astype(np.float32), fx=f, fy=f, cx=W / 2, cy=H / 2,
                          znear=0.2, width=W, height=H)
    n = np.array([0.2, -0.1, 1.0])
    n /= np.linalg.norm(n)
    p0 = np.zeros(3)                                   # plane n . (x - p0) = 0
    Rd, td = cam.R.astype(np.float64), cam.t.astype(np.float64)
    C = -Rd.T @ td
    uu, vv = np.meshgrid(np.arange(W) + 0.5, np.arange(H) + 0.5)
    dcam = np.stack([(uu - cam.cx) / f, (vv - cam.cy) / f, np.ones_like(uu)], -1)
    dw = dcam @ Rd                                     # R^T d: camera depth z at C + z dw
    z = (n @ (p0 - C)) / (dw @ n)
    depth = np.where(z > 0, z, 0.0).astype(np.float32)
    s, mu = 0.25, 1.5
    origin, dims = (-3.0, -2.0, -2.0), (24, 16, 16)
    tsdf, w = TO.integrate(origin, s, dims, mu, [cam], [depth])
    cen = TO.voxel_centres(origin, s, dims).astype(np.float64)
    zc = cen @ Rd.T[:, 2] + td[2]
    # camera depth of the plane along each voxel's own ray
    dv = (cen - C) / zc[:, None]
    zp = (n @ (p0 - C)) / (dv @ n)
    gap = zp - zc                                      # > 0: voxel in front of the plane
    foot = 2.0 * zc / f                                # two pixel footprints of depth change (slope < 1)
    ww, tt = w.ravel(), tsdf.ravel()
    front = (gap > foot) & (ww > 0)
    behind = (gap < -foot) & (gap > -mu + foot) & (ww > 0)
    assert front.sum() > 100 and behind.sum() > 50
    assert (tt[front] > 0).all() and (tt[behind] < 0).all()
    # voxels far behind the surface are not integrated
    assert (ww[gap < -mu - foot] == 0).all()
