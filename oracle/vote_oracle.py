"""CPU oracle of PG-SAG's reliability-scored multi-view voting filter.

TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and bench.py's
cpu_baseline / reference leg may import or call this module.  It shares no code
with the CUDA library and never reads anything the CUDA path produced.

Passages followed (Sec. 4.1, "Reliability-scored Multi-view Voting Filter"):

* Eq. 5 / 6 -- a sparse point p_i is a potential building point iff
  sum_j I(p_i in M_j) > 0, the count over the N views of the masks that hold it.
* Eq. 7 -- its unreliability score US(p) = sum_j I(p in Image_j minus M_j), the
  number of views in which it lies inside the image but outside the mask.
* A potential point is reliable iff US < tau (tau is a tolerance chosen per
  scene; the paper gives no value).

Readings (the paper is silent on them):
* "p lies in M_j" means: p projects, through view j's pinhole camera
  (x_c = R x_w + t, in front iff z_c > znear), onto a pixel (floor(u),
  floor(v)) inside the image whose mask value is nonzero; no occlusion test.
* The three discrete decisions (in front, inside the image, which pixel) are
  taken in float32 with one correctly rounded operation per step, in the order
  x_c = ((R00 x + R01 y) + R02 z) + t0 (likewise y_c, z_c), iz = 1 / z_c,
  u = fx (x_c iz) + cx, v = fy (y_c iz) + cy, inside iff 0 <= u < W and
  0 <= v < H -- the precision of the kernel, so both sides decide alike.
  Everything else is integer counting.

Each view is processed as a whole array operation over the points (numpy float32
ufuncs round every operation to float32 and never fuse).
"""
from __future__ import annotations

from typing import Sequence, Tuple

import numpy as np

F32 = np.float32


def project_pixels(points: np.ndarray, R: np.ndarray, t: np.ndarray, fx, fy, cx, cy, znear, width, height):
    """Pixel (px, py) of every point in one view and whether it lands inside the
    image (in front of the camera and 0 <= u < W, 0 <= v < H)."""
    P = np.asarray(points, F32)
    R = np.asarray(R, F32).reshape(3, 3)
    t = np.asarray(t, F32).reshape(3)
    X, Y, Z = P[:, 0], P[:, 1], P[:, 2]
    with np.errstate(all="ignore"):
        xc = ((R[0, 0] * X + R[0, 1] * Y) + R[0, 2] * Z) + t[0]
        yc = ((R[1, 0] * X + R[1, 1] * Y) + R[1, 2] * Z) + t[1]
        zc = ((R[2, 0] * X + R[2, 1] * Y) + R[2, 2] * Z) + t[2]
        front = zc > F32(znear)
        iz = F32(1.0) / zc
        u = F32(fx) * (xc * iz) + F32(cx)
        v = F32(fy) * (yc * iz) + F32(cy)
        inside = front & (u >= F32(0.0)) & (u < F32(width)) & (v >= F32(0.0)) & (v < F32(height))
    for a in (xc, yc, zc, iz, u, v):
        assert a.dtype == F32
    px = np.where(inside, np.floor(np.where(inside, u, F32(0))), 0).astype(np.int64)
    py = np.where(inside, np.floor(np.where(inside, v, F32(0))), 0).astype(np.int64)
    return px, py, inside


def vote_counts(points: np.ndarray, cams: Sequence, masks: Sequence[np.ndarray]) -> Tuple[np.ndarray, np.ndarray]:
    """(in_mask, US) per point: the Eq. 5 / 6 mask count and the Eq. 7 score over
    all views.  cams: objects with R, t, fx, fy, cx, cy, znear, width, height;
    masks: uint8 [H, W] per view (nonzero = building)."""
    M = int(np.asarray(points).shape[0])
    cin = np.zeros(M, np.int64)
    cout = np.zeros(M, np.int64)
    for cam, mask in zip(cams, masks):
        mask = np.asarray(mask)
        assert mask.shape == (int(cam.height), int(cam.width))
        px, py, inside = project_pixels(points, cam.R, cam.t, cam.fx, cam.fy, cam.cx, cam.cy, cam.znear,
                                        int(cam.width), int(cam.height))
        m = np.zeros(M, bool)
        m[inside] = mask[py[inside], px[inside]] != 0
        cin += m
        cout += inside & ~m
    return cin, cout


def reliable_points(in_mask: np.ndarray, us: np.ndarray, tau: int) -> np.ndarray:
    """Eq. 6 and the tolerance rule: potential (in_mask > 0) and US < tau."""
    return (np.asarray(in_mask) > 0) & (np.asarray(us) < int(tau))


def vote_filter(points, cams, masks, tau: int):
    """in_mask, US, reliable flags and the ascending indices of the reliable points."""
    cin, cout = vote_counts(points, cams, masks)
    rel = reliable_points(cin, cout, tau)
    return cin, cout, rel, np.nonzero(rel)[0]
