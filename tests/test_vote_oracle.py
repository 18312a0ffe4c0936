"""Pins of the voting-filter oracle (Sec. 4.1, Eq. 5-7) against facts fixed
outside it: a hand-worked example, back-projection of pixel centres through the
inverse camera model (float64, independent of the forward formula), the
half-open image border, the near plane, and closed forms for constant and
complementary masks."""
import json
import os
from types import SimpleNamespace

import numpy as np
import pytest
from scipy.spatial.transform import Rotation

import pgsag_synth as syn
from oracle import vote_oracle as VO


def _load_json(path):
    with open(path) as f:
        return json.load(f)


GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def example():
    g = _load_json(os.path.join(GOLDEN, "vote_example.json"))
    cams = [SimpleNamespace(R=np.eye(3, dtype=np.float32), t=np.asarray(v["t"], np.float32), fx=2.0, fy=2.0,
                            cx=2.0, cy=2.0, znear=0.2, width=4, height=4) for v in g["views"]]
    masks = [np.asarray(v["mask"], np.uint8) for v in g["views"]]
    return g, np.asarray(g["points"], np.float32), cams, masks


def test_hand_worked_example():
    g, pts, cams, masks = example()
    cin, cout, rel, idx = VO.vote_filter(pts, cams, masks, 1)
    assert cin.tolist() == g["in_mask"]
    assert cout.tolist() == g["us"]
    assert rel.astype(int).tolist() == g["reliable_tau1"]
    assert idx.tolist() == [i for i, r in enumerate(g["reliable_tau1"]) if r]
    _, _, rel2, _ = VO.vote_filter(pts, cams, masks, 2)
    assert rel2.astype(int).tolist() == g["reliable_tau2"]


def random_camera(rng, W, H):
    R = Rotation.random(random_state=int(rng.integers(1 << 30))).as_matrix()
    return SimpleNamespace(R=R.astype(np.float32), t=rng.uniform(-50, 50, 3).astype(np.float32),
                           fx=float(np.float32(rng.uniform(200, 8000))), fy=float(np.float32(rng.uniform(200, 8000))),
                           cx=float(np.float32(rng.uniform(0, W))), cy=float(np.float32(rng.uniform(0, H))),
                           znear=0.2, width=W, height=H)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_backprojected_pixel_centres_land_in_their_pixel(seed):
    rng = np.random.default_rng(seed)
    W, H = 5472, 3648
    cam = random_camera(rng, W, H)
    n = 5000
    u = rng.integers(0, W, n)
    v = rng.integers(0, H, n)
    d = rng.uniform(1.0, 150.0, n)
    # inverse camera model in float64: centre (u + 1/2, v + 1/2) at depth d
    xc = np.stack([(u + 0.5 - cam.cx) / cam.fx * d, (v + 0.5 - cam.cy) / cam.fy * d, d], 1)
    Rd, td = cam.R.astype(np.float64), cam.t.astype(np.float64)
    Xw = (xc - td) @ Rd  # R^T (x_c - t)
    px, py, inside = VO.project_pixels(Xw.astype(np.float32), cam.R, cam.t, cam.fx, cam.fy, cam.cx, cam.cy,
                                       cam.znear, W, H)
    assert inside.all()
    np.testing.assert_array_equal(px, u)
    np.testing.assert_array_equal(py, v)


def test_image_border_is_half_open_and_near_plane_strict():
    # identity camera, fx = fy = 1, cx = cy = 0, z = 1: u = x and v = y exactly
    W, H = 8, 6
    pts = np.array([[0.0, 0.5, 1.0], [-2.0 ** -20, 0.5, 1.0], [8.0, 0.5, 1.0], [8.0 - 2.0 ** -10, 0.5, 1.0],
                    [0.5, 6.0, 1.0], [0.5, 6.0 - 2.0 ** -10, 1.0], [0.5, 0.5, 0.2], [0.5, 0.5, 0.2 + 2.0 ** -20]],
                   np.float32)
    px, py, inside = VO.project_pixels(pts, np.eye(3), np.zeros(3), 1.0, 1.0, 0.0, 0.0, 0.2, W, H)
    assert inside.tolist() == [True, False, False, True, False, True, False, True]
    # the last point sits just beyond the near plane: u = v = 0.5 / z = 2.5 - eps
    assert px[inside].tolist() == [0, 7, 0, 2]
    assert py[inside].tolist() == [0, 0, 5, 2]


def test_nan_and_infinite_points_never_count():
    pts = np.array([[np.nan, 0, 1], [0, np.inf, 1], [0, 0, np.inf], [0, 0, -np.inf]], np.float32)
    cam = SimpleNamespace(R=np.eye(3), t=np.zeros(3), fx=10.0, fy=10.0, cx=5.0, cy=5.0, znear=0.2, width=10, height=10)
    cin, cout = VO.vote_counts(pts, [cam], [np.ones((10, 10), np.uint8)])
    assert cin.tolist() == [0, 0, 0, 0] and cout.tolist() == [0, 0, 0, 0]


def small_workload():
    return syn.vote_workload(n_points=4000, n_views=5, width=320, height=240, mask_step=2)


def test_constant_and_complementary_masks():
    w = small_workload()
    ones = [np.ones_like(m) for m in w.masks]
    zeros = [np.zeros_like(m) for m in w.masks]
    c1, u1 = VO.vote_counts(w.points, w.cams, ones)
    c0, u0 = VO.vote_counts(w.points, w.cams, zeros)
    assert (u1 == 0).all() and (c0 == 0).all()
    np.testing.assert_array_equal(c1, u0)           # both count the views the point is inside
    assert c1.max() <= len(w.cams) and c1.sum() > 0
    cm, um = VO.vote_counts(w.points, w.cams, w.masks)
    cc, uc = VO.vote_counts(w.points, w.cams, [1 - m for m in w.masks])
    np.testing.assert_array_equal(cm, uc)
    np.testing.assert_array_equal(um, cc)
    np.testing.assert_array_equal(cm + um, c1)      # in image = in mask + outside mask
    # no potential point without a mask count; tau above the view count keeps every potential point
    rel = VO.reliable_points(cm, um, len(w.cams) + 1)
    np.testing.assert_array_equal(rel, cm > 0)
    assert not VO.reliable_points(cm, um, 0).any()


def test_view_and_point_permutation_invariance():
    w = small_workload()
    rng = np.random.default_rng(5)
    cm, um = VO.vote_counts(w.points, w.cams, w.masks)
    pv = rng.permutation(len(w.cams))
    cm2, um2 = VO.vote_counts(w.points, [w.cams[i] for i in pv], [w.masks[i] for i in pv])
    np.testing.assert_array_equal(cm, cm2)
    np.testing.assert_array_equal(um, um2)
    pp = rng.permutation(len(w.points))
    cm3, um3 = VO.vote_counts(w.points[pp], w.cams, w.masks)
    np.testing.assert_array_equal(cm[pp], cm3)
    np.testing.assert_array_equal(um[pp], um3)


def test_building_points_are_kept_more_often_than_ground_points():
    # the filter's purpose (Sec. 4.1): points on buildings pass, ground points
    # caught in false-positive blobs of a few views are rejected
    w = syn.vote_workload(n_points=20000, n_views=12, width=640, height=480, mask_step=2)
    cm, um, rel, _ = VO.vote_filter(w.points, w.cams, w.masks, w.tau)
    assert rel[w.on_building].mean() > 0.9
    assert rel[~w.on_building].mean() < rel[w.on_building].mean() - 0.2
