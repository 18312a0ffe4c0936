"""CPU oracle of PG-SAG's depth-map fusion and TSDF integration (Sec. 4.4).

TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and bench.py's
cpu_baseline / reference leg may import or call this module.  It shares no code
with the CUDA library and never reads anything the CUDA path produced.

Passages followed (Sec. 4.4, "Mesh Extraction and Merge"): depth maps of the
buildings and of the background are rendered from several views; where the maps
overlap they are fused by their mean; the fused maps are integrated into a
truncated signed distance function (the TSDF method, by citation), from which a
mesh would be extracted (mesh extraction itself is not part of this module).

Readings (the paper is silent on them):
* Mean fusion: per pixel, the mean of the maps that hold a depth there (depth
  > 0 and finite); 0 where none does.
* TSDF (the volumetric method it cites): a regular grid of voxels, voxel
  (i, j, k) centred at origin + ((i, j, k) + 1/2) * voxel; per view, the voxel
  centre is projected through the pinhole camera (x_c = R x + t, in front iff
  z_c > znear, pixel (floor u, floor v) inside the image); where the pixel holds a
  depth d, the projective signed distance is sdf = d - z_c; the view is
  integrated iff sdf >= -trunc, with value min(1, sdf / trunc) and weight 1; the
  TSDF is the weighted mean of the integrated values (weight = their count);
  voxels no view integrates keep weight 0 and value 1.
* The discrete decisions (in front, inside the image, which pixel, d valid,
  sdf >= -trunc) are taken in float32, one correctly rounded operation per step
  in the order: voxel centre c = origin + ((i + 1/2) * voxel), x_c = ((R00 c_x +
  R01 c_y) + R02 c_z) + t0 (likewise y_c, z_c), iz = 1 / z_c, u = fx (x_c iz) + cx,
  v = fy (y_c iz) + cy, sdf = d - z_c -- the kernel's precision, so both sides
  integrate the same (voxel, view) pairs.  The values are then averaged in
  float64.
"""
from __future__ import annotations

from typing import Sequence, Tuple

import numpy as np

F32 = np.float32


def fuse_mean(maps: Sequence[np.ndarray]) -> np.ndarray:
    """Mean of the valid (> 0, finite) depths per pixel; 0 where no map has one."""
    M = np.stack([np.asarray(m, np.float64) for m in maps], 0)
    ok = np.isfinite(M) & (M > 0)
    s = np.where(ok, M, 0.0).sum(0)
    n = ok.sum(0)
    return np.where(n > 0, s / np.maximum(n, 1), 0.0)


def voxel_centres(origin, voxel, dims) -> np.ndarray:
    """float32 [nz*ny*nx, 3] centres, x fastest."""
    nx, ny, nz = (int(d) for d in dims)
    o = np.asarray(origin, F32)
    s = F32(voxel)
    ax = [o[a] + (np.arange(n, dtype=F32) + F32(0.5)) * s for a, n in enumerate((nx, ny, nz))]
    Z, Y, X = np.meshgrid(ax[2], ax[1], ax[0], indexing="ij")
    return np.stack([X.ravel(), Y.ravel(), Z.ravel()], 1)


def integrate(origin, voxel, dims, trunc, cams, depths, tsdf0=None, weight0=None,
              voxel_index=None) -> Tuple[np.ndarray, np.ndarray]:
    """TSDF and weight grids [nz, ny, nx] (float64) after integrating every view
    (cams: R, t, fx, fy, cx, cy, znear, width, height; depths: float32 [H, W]),
    optionally on top of an earlier (tsdf0, weight0).  voxel_index (linear
    indices, x fastest): evaluate only those voxels and return flat arrays."""
    nx, ny, nz = (int(d) for d in dims)
    C = voxel_centres(origin, voxel, dims)
    if voxel_index is not None:
        C = C[np.asarray(voxel_index, np.int64)]
    X, Y, Z = C[:, 0], C[:, 1], C[:, 2]
    mu = F32(trunc)
    ssum = np.zeros(len(C), np.float64)
    cnt = np.zeros(len(C), np.int64)
    for cam, dm in zip(cams, depths):
        R = np.asarray(cam.R, F32).reshape(3, 3)
        t = np.asarray(cam.t, F32).reshape(3)
        dm = np.asarray(dm, F32)
        W, H = int(cam.width), int(cam.height)
        assert dm.shape == (H, W)
        with np.errstate(all="ignore"):
            xc = ((R[0, 0] * X + R[0, 1] * Y) + R[0, 2] * Z) + t[0]
            yc = ((R[1, 0] * X + R[1, 1] * Y) + R[1, 2] * Z) + t[1]
            zc = ((R[2, 0] * X + R[2, 1] * Y) + R[2, 2] * Z) + t[2]
            iz = F32(1.0) / zc
            u = F32(cam.fx) * (xc * iz) + F32(cam.cx)
            v = F32(cam.fy) * (yc * iz) + F32(cam.cy)
            ins = (zc > F32(cam.znear)) & (u >= 0) & (u < F32(W)) & (v >= 0) & (v < F32(H))
        px = np.where(ins, np.floor(np.where(ins, u, F32(0))), 0).astype(np.int64)
        py = np.where(ins, np.floor(np.where(ins, v, F32(0))), 0).astype(np.int64)
        d = np.where(ins, dm[py, px], F32(0))
        ok = ins & np.isfinite(d) & (d > F32(0))
        with np.errstate(all="ignore"):
            sdf = d - zc                      # float32
            use = ok & (sdf >= -mu)
        val = np.minimum(1.0, sdf.astype(np.float64) / float(mu))
        ssum += np.where(use, val, 0.0)
        cnt += use
    if tsdf0 is None:
        w = cnt.astype(np.float64)
        tsdf = np.where(cnt > 0, ssum / np.maximum(cnt, 1), 1.0)
    else:
        t0 = np.asarray(tsdf0, np.float64).ravel()
        w0 = np.asarray(weight0, np.float64).ravel()
        if voxel_index is not None and t0.size != len(C):
            t0, w0 = t0[voxel_index], w0[voxel_index]
        w = w0 + cnt
        tsdf = np.where(cnt > 0, (t0 * w0 + ssum) / np.where(w > 0, w, 1.0), t0)
    if voxel_index is not None:
        return tsdf, w
    return tsdf.reshape(nz, ny, nx), w.reshape(nz, ny, nx)


def zero_crossing_along_z(tsdf_col: np.ndarray, z_centres: np.ndarray):
    """Linear interpolation of the first + to - sign change of a TSDF column
    (the surface a mesher would place); None if there is none."""
    s = np.asarray(tsdf_col, np.float64)
    for k in range(len(s) - 1):
        if s[k] > 0 >= s[k + 1]:
            a = s[k] / (s[k] - s[k + 1])
            return float(z_centres[k] + a * (z_centres[k + 1] - z_centres[k]))
    return None
