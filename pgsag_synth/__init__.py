"""Seeded synthetic inputs for the masked Gaussian-splat path.

This module only *draws* inputs: Gaussian parameters, pinhole cameras, binary
building masks and photometric targets.  It holds none of the method's
arithmetic (no projection, blending, loss or mask morphology), so both the
FP64 oracle and the CUDA path may use it.

Shapes and distributions follow the paper's workloads: aerial oblique views of
building clusters at the original GauU-Scene resolution (Sec. 5.1, 5468x3636
images, 120 m flight height) with building masks (Sec. 4.1).  The datasets
themselves are not available, so seeded stand-ins are drawn here.

All arrays are float32 (the kernels' input precision); the oracle upcasts the
same float32 values to float64.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence, Tuple

import numpy as np

BASE_SEED = 2025_0103
SH_COEFFS = 16  # degree 3


@dataclasses.dataclass
class Camera:
    """Pinhole camera, OpenCV axes (x right, y down, z forward).

    x_cam = R @ x_world + t.  Pixel (u, v) has its centre at (u+0.5, v+0.5).
    """
    R: np.ndarray          # float32 [3,3] world -> camera rotation
    t: np.ndarray          # float32 [3]
    fx: float
    fy: float
    cx: float
    cy: float
    width: int
    height: int
    znear: float = 0.2

    def __post_init__(self):
        self.R = np.asarray(self.R, dtype=np.float32).reshape(3, 3)
        self.t = np.asarray(self.t, dtype=np.float32).reshape(3)
        self.fx = float(np.float32(self.fx))
        self.fy = float(np.float32(self.fy))
        self.cx = float(np.float32(self.cx))
        self.cy = float(np.float32(self.cy))
        self.znear = float(np.float32(self.znear))


@dataclasses.dataclass
class Gaussians:
    """Raw (pre-activation) Gaussian parameters, SoA float32."""
    means: np.ndarray          # [N,3]
    log_scales: np.ndarray     # [N,3]
    quats: np.ndarray          # [N,4]  (w, x, y, z), not necessarily unit
    opacity_logit: np.ndarray  # [N]
    sh: np.ndarray             # [N,16,3]  coefficient-major, channel-minor

    @property
    def n(self) -> int:
        return int(self.means.shape[0])

    def subset(self, idx) -> "Gaussians":
        return Gaussians(self.means[idx], self.log_scales[idx], self.quats[idx],
                         self.opacity_logit[idx], self.sh[idx])

    @staticmethod
    def concat(parts: Sequence["Gaussians"]) -> "Gaussians":
        return Gaussians(*(np.ascontiguousarray(np.concatenate([getattr(p, f.name) for p in parts], 0))
                           for f in dataclasses.fields(Gaussians)))


@dataclasses.dataclass
class View:
    """One rendered view: camera, building mask (u8 0/1, [H,W]) and target RGB [H,W,3]."""
    cam: Camera
    mask: np.ndarray
    target: np.ndarray


def streams(config_index: int, n: int = 4) -> List[np.random.Generator]:
    """Independent PCG64 streams (scene, cameras, mask, target) for one config."""
    ss = np.random.SeedSequence(BASE_SEED + config_index)
    return [np.random.Generator(np.random.PCG64(s)) for s in ss.spawn(n)]


# --------------------------------------------------------------------------
# cameras
# --------------------------------------------------------------------------

def look_at_camera(campos, target, width, height, fx, fy=None, up=(0.0, 0.0, 1.0), znear=0.2) -> Camera:
    """Camera at `campos` looking at `target`; image principal point at the centre."""
    campos = np.asarray(campos, np.float64)
    fwd = np.asarray(target, np.float64) - campos
    fwd /= np.linalg.norm(fwd)
    right = np.cross(fwd, np.asarray(up, np.float64))
    if np.linalg.norm(right) < 1e-9:
        right = np.cross(fwd, np.array([0.0, 1.0, 0.0]))
    right /= np.linalg.norm(right)
    down = np.cross(fwd, right)
    R = np.stack([right, down, fwd], 0)
    t = -R @ campos
    fy = fx if fy is None else fy
    return Camera(R, t, fx, fy, width / 2.0, height / 2.0, width, height, znear)


def identity_camera(width, height, fx, fy=None, znear=0.2) -> Camera:
    fy = fx if fy is None else fy
    return Camera(np.eye(3), np.zeros(3), fx, fy, width / 2.0, height / 2.0, width, height, znear)


# --------------------------------------------------------------------------
# Gaussian attributes
# --------------------------------------------------------------------------

def random_quats(rng, n) -> np.ndarray:
    q = rng.standard_normal((n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    return q.astype(np.float32)


def _rotmat_to_quat(M: np.ndarray) -> np.ndarray:
    """Rotation matrices [n,3,3] -> quaternions (w,x,y,z) (input drawing only)."""
    from scipy.spatial.transform import Rotation
    xyzw = Rotation.from_matrix(M).as_quat()
    return np.concatenate([xyzw[:, 3:4], xyzw[:, :3]], 1)


def cube_scene(rng, n, cube=10.0, zmin=5.0, zmax=15.0) -> Gaussians:
    """Means uniform in a cube (side `cube`) spanning depth [zmin, zmax] in front of
    an identity camera; log-scales N(-3, 0.5); uniform unit quaternions; opacity
    logits N(0,1); SH degree-3 coefficients N(0, 0.2)."""
    means = np.empty((n, 3), np.float64)
    means[:, 0] = rng.uniform(-cube / 2, cube / 2, n)
    means[:, 1] = rng.uniform(-cube / 2, cube / 2, n)
    means[:, 2] = rng.uniform(zmin, zmax, n)
    log_scales = rng.normal(-3.0, 0.5, (n, 3))
    quats = random_quats(rng, n)
    opac = rng.normal(0.0, 1.0, n)
    sh = rng.normal(0.0, 0.2, (n, SH_COEFFS, 3))
    return Gaussians(means.astype(np.float32), log_scales.astype(np.float32), quats,
                     opac.astype(np.float32), sh.astype(np.float32))


# --------------------------------------------------------------------------
# masks and targets
# --------------------------------------------------------------------------

def rect_mask(rng, height, width, coverage=0.40, tol=0.03, nmin=3, nmax=6, max_tries=10000) -> np.ndarray:
    """Union of nmin..nmax random axis-aligned rectangles, rejection-sampled until the
    covered fraction is within coverage +- tol."""
    for _ in range(max_tries):
        m = np.zeros((height, width), np.uint8)
        k = int(rng.integers(nmin, nmax + 1))
        for _ in range(k):
            w = int(rng.integers(max(1, width // 8), max(2, (width * 3) // 4)))
            h = int(rng.integers(max(1, height // 8), max(2, (height * 3) // 4)))
            x0 = int(rng.integers(0, max(1, width - w + 1)))
            y0 = int(rng.integers(0, max(1, height - h + 1)))
            m[y0:y0 + h, x0:x0 + w] = 1
        if abs(m.mean() - coverage) <= tol:
            return m
    raise RuntimeError("rect_mask: coverage target not reached")


def random_target(rng, height, width) -> np.ndarray:
    return rng.random((height, width, 3), dtype=np.float32)


# --------------------------------------------------------------------------
# aerial building scenes
# --------------------------------------------------------------------------

@dataclasses.dataclass
class Box:
    x0: float
    y0: float
    x1: float
    y1: float
    h: float


def random_boxes(rng, n, area=160.0, fmin=8.0, fmax=30.0, hmin=8.0, hmax=45.0, gap=2.0,
                 footprint_scale=1.0, max_tries=200000) -> List[Box]:
    """n non-overlapping box 'buildings' with footprints U(fmin,fmax)*scale and heights
    U(hmin,hmax) inside an area x area square centred at the origin."""
    boxes: List[Box] = []
    tries = 0
    while len(boxes) < n:
        tries += 1
        if tries > max_tries:
            raise RuntimeError("random_boxes: could not place boxes")
        w = rng.uniform(fmin, fmax) * footprint_scale
        d = rng.uniform(fmin, fmax) * footprint_scale
        h = rng.uniform(hmin, hmax)
        if w >= area or d >= area:
            continue
        x0 = rng.uniform(-area / 2, area / 2 - w)
        y0 = rng.uniform(-area / 2, area / 2 - d)
        ok = all(x0 + w + gap <= b.x0 or b.x1 + gap <= x0 or y0 + d + gap <= b.y0 or b.y1 + gap <= y0
                 for b in boxes)
        if ok:
            boxes.append(Box(x0, y0, x0 + w, y0 + d, h))
    return boxes


def _surfaces(boxes: Sequence[Box], ground: float):
    """Rectangular surfaces (origin, edge u, edge v, outward normal)."""
    S = []
    g = ground / 2
    S.append((np.array([-g, -g, 0.0]), np.array([ground, 0, 0.0]), np.array([0, ground, 0.0]), np.array([0, 0, 1.0])))
    for b in boxes:
        w, d, h = b.x1 - b.x0, b.y1 - b.y0, b.h
        S.append((np.array([b.x0, b.y0, h]), np.array([w, 0, 0.0]), np.array([0, d, 0.0]), np.array([0, 0, 1.0])))
        S.append((np.array([b.x0, b.y0, 0.0]), np.array([w, 0, 0.0]), np.array([0, 0, h]), np.array([0, -1.0, 0])))
        S.append((np.array([b.x0, b.y1, 0.0]), np.array([w, 0, 0.0]), np.array([0, 0, h]), np.array([0, 1.0, 0])))
        S.append((np.array([b.x0, b.y0, 0.0]), np.array([0, d, 0.0]), np.array([0, 0, h]), np.array([-1.0, 0, 0])))
        S.append((np.array([b.x1, b.y0, 0.0]), np.array([0, d, 0.0]), np.array([0, 0, h]), np.array([1.0, 0, 0])))
    return S


def surface_gaussians(rng, boxes: Sequence[Box], n: int, ground: float = 200.0) -> Gaussians:
    """n flat, surface-hugging Gaussians on the box surfaces and the ground plane,
    placed proportionally to area; tangent log-scales N(-3,0.5), the normal axis
    ten times thinner; random in-plane twist; other attributes as cube_scene."""
    S = _surfaces(boxes, ground)
    areas = np.array([np.linalg.norm(np.cross(u, v)) for _, u, v, _ in S])
    counts = rng.multinomial(n, areas / areas.sum())
    means, rots = [], []
    for (o, u, v, nrm), c in zip(S, counts):
        if c == 0:
            continue
        a = rng.random((c, 1))
        b = rng.random((c, 1))
        means.append(o[None] + a * u[None] + b * v[None] + 1e-3 * nrm[None])
        tu = u / np.linalg.norm(u)
        tv = np.cross(nrm, tu)
        th = rng.uniform(0, 2 * np.pi, c)
        t1 = np.cos(th)[:, None] * tu[None] + np.sin(th)[:, None] * tv[None]
        t2 = np.cross(np.broadcast_to(nrm, t1.shape), t1)
        M = np.stack([t1, t2, np.broadcast_to(nrm, t1.shape)], axis=2)  # columns = axes
        rots.append(M)
    means = np.concatenate(means, 0)
    M = np.concatenate(rots, 0)
    perm = rng.permutation(n)
    means, M = means[perm], M[perm]
    quats = _rotmat_to_quat(M)
    ls = rng.normal(-3.0, 0.5, (n, 3))
    ls[:, 2] = rng.normal(-3.0, 0.5, n) - math.log(10.0)
    opac = rng.normal(0.0, 1.0, n)
    sh = rng.normal(0.0, 0.2, (n, SH_COEFFS, 3))
    return Gaussians(means.astype(np.float32), ls.astype(np.float32), quats.astype(np.float32),
                     opac.astype(np.float32), sh.astype(np.float32))


def raycast_box_mask(boxes: Sequence[Box], cam: Camera, step: int = 1) -> np.ndarray:
    """Binary mask of the pixels whose ray hits a box (boxes stand on the ground, so a
    box hit is always in front of the ground hit).  `step` > 1 casts a subsampled grid."""
    H, W = cam.height, cam.width
    R = cam.R.astype(np.float64)
    t = cam.t.astype(np.float64)
    C = -R.T @ t
    us = np.arange(0, W, step) + 0.5
    vs = np.arange(0, H, step) + 0.5
    m = np.zeros((len(vs), len(us)), np.uint8)
    for b in boxes:
        corners = np.array([[x, y, z] for x in (b.x0, b.x1) for y in (b.y0, b.y1) for z in (0.0, b.h)])
        pc = corners @ R.T + t
        if np.all(pc[:, 2] <= 1e-6):
            continue
        if np.any(pc[:, 2] <= 1e-6):
            ub = (0, W)
            vb = (0, H)
        else:
            px = cam.fx * pc[:, 0] / pc[:, 2] + cam.cx
            py = cam.fy * pc[:, 1] / pc[:, 2] + cam.cy
            ub = (max(0.0, px.min() - 2), min(float(W), px.max() + 2))
            vb = (max(0.0, py.min() - 2), min(float(H), py.max() + 2))
        iu = np.nonzero((us >= ub[0]) & (us <= ub[1]))[0]
        iv = np.nonzero((vs >= vb[0]) & (vs <= vb[1]))[0]
        if len(iu) == 0 or len(iv) == 0:
            continue
        uu, vv = np.meshgrid(us[iu], vs[iv])
        dcam = np.stack([(uu - cam.cx) / cam.fx, (vv - cam.cy) / cam.fy, np.ones_like(uu)], -1)
        dw = dcam @ R  # R^T d
        lo = np.array([b.x0, b.y0, 0.0])
        hi = np.array([b.x1, b.y1, b.h])
        with np.errstate(divide="ignore", invalid="ignore"):
            inv = 1.0 / dw
            t0 = (lo - C) * inv
            t1 = (hi - C) * inv
        tmin = np.nanmax(np.minimum(t0, t1), axis=-1)
        tmax = np.nanmin(np.maximum(t0, t1), axis=-1)
        hit = (tmax >= np.maximum(tmin, 0.0)).astype(np.uint8)
        sub = m[np.ix_(iv, iu)]
        m[np.ix_(iv, iu)] = np.maximum(sub, hit)
    return m


def aerial_views(rng_scene, rng_cam, n_gauss, n_boxes, area, cams_fn, coverage=None, cov_tol=0.05,
                 ground=None, max_iter=6):
    """Boxes + surface Gaussians + cameras + ray-cast masks.  If `coverage` is given,
    footprints are rescaled until the first view's mask covers coverage +- cov_tol."""
    ground = ground if ground is not None else area * 1.25
    scale = 1.0
    state = rng_scene.bit_generator.state
    for _ in range(max_iter):
        rng_scene.bit_generator.state = state
        boxes = random_boxes(rng_scene, n_boxes, area=area, footprint_scale=scale)
        cams = cams_fn(rng_cam)
        if coverage is None:
            break
        cov = raycast_box_mask(boxes, cams[0], step=8).mean()
        if abs(cov - coverage) <= cov_tol:
            break
        scale *= math.sqrt(coverage / max(cov, 1e-3))
    g = surface_gaussians(rng_scene, boxes, n_gauss, ground=ground)
    masks = [raycast_box_mask(boxes, c) for c in cams]
    return g, boxes, cams, masks


# --------------------------------------------------------------------------
# named workloads
# --------------------------------------------------------------------------

def config0() -> Tuple[Gaussians, List[View]]:
    """20k Gaussians in a 10 m cube 5-15 m in front of a 256x256 pinhole camera
    (fx = fy = 300), rectangle mask ~40%, uniform random target."""
    rs, rc, rm, rt = streams(0)
    g = cube_scene(rs, 20000)
    cam = identity_camera(256, 256, 300.0)
    mask = rect_mask(rm, 256, 256, 0.40, 0.03)
    return g, [View(cam, mask, random_target(rt, 256, 256))]


def aerial_camera(width, height, altitude=120.0, pitch_deg=45.0, azimuth_deg=0.0, look_at=(0.0, 0.0, 0.0),
                  fx_factor=1.2) -> Camera:
    """Oblique camera at `altitude` m, looking down at `pitch_deg` towards `look_at`."""
    dist = altitude / math.tan(math.radians(pitch_deg))
    az = math.radians(azimuth_deg)
    campos = np.array(look_at, np.float64) + np.array([-dist * math.cos(az), -dist * math.sin(az), altitude])
    return look_at_camera(campos, look_at, width, height, fx_factor * width)


def config1(n_gauss=1_500_000, width=5472, height=3648):
    """Single oblique aerial view at 5472x3648 of 40 box buildings (1.5M surface
    Gaussians over a ground plane), fx = 1.2 W, 120 m altitude, 45 deg pitch; the
    building mask (ray-cast) covers ~35% of the pixels."""
    rs, rc, rm, rt = streams(1)
    g, boxes, cams, masks = aerial_views(
        rs, rc, n_gauss, 40, 160.0,
        lambda r: [aerial_camera(width, height, 120.0, 45.0)], coverage=0.35, cov_tol=0.05, ground=200.0)
    return g, [View(cams[0], masks[0], random_target(rt, height, width))], boxes


def config2(n_gauss=300_000, width=1920, height=1080, n_views=4):
    """300k Gaussians on 8 buildings, 4 views at 1920x1080 (fx = 2304) around the block."""
    rs, rc, rm, rt = streams(2)
    area = 160.0 * math.sqrt(8 / 40)

    def cams_fn(r):
        return [aerial_camera(width, height, 60.0, 45.0, azimuth_deg=90.0 * j) for j in range(n_views)]
    g, boxes, cams, masks = aerial_views(rs, rc, n_gauss, 8, area, cams_fn, ground=area * 1.25)
    return g, [View(c, m, random_target(rt, height, width)) for c, m in zip(cams, masks)], boxes


CONFIG3_SIZES = (200_000, 400_000, 600_000, 900_000, 1_200_000, 1_800_000, 2_400_000, 3_000_000)
CONFIG3_RES = ((1920, 1080), (4000, 3000), (5472, 3648))


def config3(sizes=CONFIG3_SIZES, views_per_region=4, res=CONFIG3_RES, scale=1.0):
    """Uneven sub-regions: region s has sizes[s] Gaussians on its own building scene;
    its view j is at resolution res[(s+j) % 3], fx = 1.2 W; rectangle masks with
    coverage U(0.2, 0.6).  Returns (gaussians concatenated, per-region ranges, views,
    view -> region)."""
    rs, rc, rm, rt = streams(3)
    parts, ranges, views, owner = [], [], [], []
    start = 0
    for s, n in enumerate(sizes):
        n = max(1, int(n * scale))
        nb = max(2, int(round(40 * n / 1_500_000)))
        area = 160.0 * math.sqrt(nb / 40)
        boxes = random_boxes(rs, nb, area=area)
        g = surface_gaussians(rs, boxes, n, ground=area * 1.25)
        parts.append(g)
        ranges.append((start, start + n))
        start += n
        for j in range(views_per_region):
            w, h = res[(s + j) % len(res)]
            if scale < 1.0:
                w = max(64, int(w * math.sqrt(scale)))
                h = max(64, int(h * math.sqrt(scale)))
            alt = 120.0 * math.sqrt(nb / 40)
            cam = aerial_camera(w, h, alt, 45.0, azimuth_deg=90.0 * j + float(rc.uniform(-20, 20)))
            cov = float(rm.uniform(0.2, 0.6))
            mask = rect_mask(rm, h, w, cov, 0.03)
            views.append(View(cam, mask, random_target(rt, h, w)))
            owner.append(s)
    return Gaussians.concat(parts), ranges, views, owner


CONFIG4_TOTAL = 20_000_000
CONFIG4_REGIONS = 12
CONFIG4_RES = (6000, 4000)


def config4_sizes(total=CONFIG4_TOTAL, regions=CONFIG4_REGIONS):
    """Region sizes following the uneven config-3 pattern: the 8 sizes 200k..3M
    interpolated linearly at `regions` evenly spaced positions, then scaled so
    that they sum to `total`."""
    pat = np.asarray(CONFIG3_SIZES, np.float64)
    s = np.interp(np.linspace(0.0, len(pat) - 1.0, regions), np.arange(len(pat), dtype=np.float64), pat)
    sizes = np.floor(s / s.sum() * total).astype(np.int64)
    sizes[-1] += total - int(sizes.sum())
    return tuple(int(v) for v in sizes)


class LazyImages:
    """Per-view images made on demand from a per-view seed, so that a large batch
    of views never holds every mask or target in host memory at once."""

    def __init__(self, fn, n):
        self.fn, self.n = fn, n

    def __len__(self):
        return self.n

    def __getitem__(self, v):
        if not 0 <= v < self.n:
            raise IndexError(v)
        return self.fn(v)


def config4(scale=1.0, views_per_region=6, res=CONFIG4_RES, total=CONFIG4_TOTAL, regions=CONFIG4_REGIONS):
    """City block at HBM capacity: `regions` sub-regions totalling `total`
    Gaussians (config4_sizes), each on its own building scene, with
    views_per_region oblique views at 6000x4000 (fx = 1.2 W = 7200) and rectangle
    masks of coverage U(0.2, 0.6).  `scale` < 1 shrinks the Gaussian counts by
    scale and each image side by sqrt(scale) (same buildings and cameras).  Masks and targets are generated
    per view on access (LazyImages).  Returns (gaussians, per-region ranges,
    cameras, view -> region, masks, targets)."""
    rs, rc, _, _ = streams(4)
    parts, ranges, cams, owner = [], [], [], []
    start = 0
    for s, n_full in enumerate(config4_sizes(total, regions)):
        n = max(1, int(n_full * scale))
        nb = max(2, int(round(40 * n_full / 1_500_000)))  # the scene keeps its full-size layout
        area = 160.0 * math.sqrt(nb / 40)
        boxes = random_boxes(rs, nb, area=area)
        parts.append(surface_gaussians(rs, boxes, n, ground=area * 1.25))
        ranges.append((start, start + n))
        start += n
        w, h = res
        if scale < 1.0:
            w, h = max(64, int(w * math.sqrt(scale))), max(64, int(h * math.sqrt(scale)))
        alt = 120.0 * math.sqrt(nb / 40)
        for j in range(views_per_region):
            az = 360.0 / views_per_region * j + float(rc.uniform(-15, 15))
            cams.append(aerial_camera(w, h, alt, 45.0, azimuth_deg=az))
            owner.append(s)
    g = Gaussians.concat(parts)
    del parts

    def view_rng(v, what):
        return np.random.Generator(np.random.PCG64(np.random.SeedSequence([BASE_SEED + 4, what, v])))

    def mask(v):
        r = view_rng(v, 1)
        c = cams[v]
        return rect_mask(r, c.height, c.width, float(r.uniform(0.2, 0.6)), 0.03)

    def target(v):
        c = cams[v]
        return random_target(view_rng(v, 2), c.height, c.width)

    return g, ranges, cams, owner, LazyImages(mask, len(cams)), LazyImages(target, len(cams))


def tiny_scene(seed, n=48, width=32, height=32, fx=40.0, coverage=0.5, zmin=3.0, zmax=8.0, log_scale_mu=-1.5):
    """Small random scene for brute-force checks."""
    ss = np.random.SeedSequence([BASE_SEED, 7, seed])
    r1, r2, r3 = [np.random.Generator(np.random.PCG64(s)) for s in ss.spawn(3)]
    g = cube_scene(r1, n, cube=3.0, zmin=zmin, zmax=zmax)
    g.log_scales[:] = r1.normal(log_scale_mu, 0.4, (n, 3)).astype(np.float32)
    cam = identity_camera(width, height, fx)
    mask = rect_mask(r2, height, width, coverage, 0.1, nmin=1, nmax=3)
    return g, View(cam, mask, random_target(r3, height, width))


def crop_view(view: View, x0: int, y0: int, w: int, h: int) -> View:
    """The w x h window at (x0, y0) of a view, as a view of its own: the same
    camera with the principal point shifted by the window origin."""
    c = view.cam
    cam = Camera(c.R, c.t, c.fx, c.fy, c.cx - x0, c.cy - y0, w, h, c.znear)
    return View(cam, np.ascontiguousarray(view.mask[y0:y0 + h, x0:x0 + w]),
                np.ascontiguousarray(view.target[y0:y0 + h, x0:x0 + w]))


def densest_window(mask: np.ndarray, w: int, h: int, step: int = 64):
    """Top-left corner of the w x h window (on a `step` grid) with the most mask pixels."""
    H, W = mask.shape
    S = np.zeros((H + 1, W + 1), np.int64)
    S[1:, 1:] = np.cumsum(np.cumsum(mask.astype(np.int64), 0), 1)
    best, arg = -1, (0, 0)
    for y in range(0, max(1, H - h + 1), step):
        for x in range(0, max(1, W - w + 1), step):
            c = S[y + h, x + w] - S[y, x + w] - S[y + h, x] + S[y, x]
            if c > best:
                best, arg = c, (x, y)
    return arg


def hashed_uniform(index: np.ndarray, channel: int, seed: int = 0) -> np.ndarray:
    """Deterministic pseudo-random values in [-1, 1) per (index, channel), from a
    64-bit integer hash (splitmix64 finaliser) -- an upstream-gradient field that
    can be evaluated at any subset of pixels."""
    with np.errstate(over="ignore"):
        x = (np.asarray(index, np.uint64) * np.uint64(8) + np.uint64(channel)
             + np.uint64(seed) * np.uint64(0x9E3779B97F4A7C15))
        x = x + np.uint64(0x9E3779B97F4A7C15)
        x = (x ^ (x >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        x = (x ^ (x >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        x = x ^ (x >> np.uint64(31))
    return ((x >> np.uint64(40)).astype(np.float64) / float(1 << 24) * 2.0 - 1.0).astype(np.float32)


# --------------------------------------------------------------------------
# stand-in rendered channels (inputs of the loss pass alone)
# --------------------------------------------------------------------------

@dataclasses.dataclass
class RenderedChannels:
    """Dense [H,W] float32 stand-ins for what a render hands the loss: colour,
    blended plane distance, blended (not unit) normal, alpha, camera depth
    (0 = nothing rendered) and the blended count.  Drawn directly, so a test can
    give the loss kernels and the oracle's loss the same values."""
    rgb: np.ndarray        # [H,W,3]
    dist: np.ndarray       # [H,W]   > 0 where depth > 0
    normal: np.ndarray     # [H,W,3] facing the camera (z component < 0)
    alpha: np.ndarray      # [H,W]
    depth: np.ndarray      # [H,W]
    n_contrib: np.ndarray  # [H,W] int32, 0 exactly where depth = 0
    soft_count: np.ndarray  # [H,W] float32 in [0.3, 1] x n_contrib (a sum of blended alphas)


def rendered_channels(cam: Camera, boxes: Optional[Sequence[Box]] = None, seed: int = 0) -> RenderedChannels:
    """Depth: the ray-cast box scene when `boxes` are given, else two tilted
    planes with a step between them; a disc of unrendered pixels (depth 0) either
    way.  Normals: a smooth field (x, y components in [-0.32, 0.32], z = -1)
    with 1% noise, scaled by alpha in [0.6, 1]; colour uniform in [0, 1];
    counts uniform in 1..39 where rendered, the soft count 0.3-1 times the count."""
    ss = np.random.SeedSequence([BASE_SEED, 11, seed])
    rng = np.random.Generator(np.random.PCG64(ss))
    H, W = cam.height, cam.width
    vv, uu = np.mgrid[0:H, 0:W].astype(np.float64)
    if boxes is not None:
        depth = raycast_depth(boxes, cam)[0].astype(np.float64)
    else:
        a, b = rng.uniform(-2.0, 2.0, 2)
        depth = 8.0 + a * (uu / W - 0.5) + b * (vv / H - 0.5)
        depth = np.where(uu > rng.uniform(0.3, 0.7) * W, depth + 0.5, depth)
    cu, cv, rad = rng.uniform(0.2, 0.8) * W, rng.uniform(0.2, 0.8) * H, 0.08 * min(H, W)
    depth = np.where((uu - cu) ** 2 + (vv - cv) ** 2 < rad * rad, 0.0, depth)
    on = depth > 0
    p1, p2 = rng.uniform(0.0, 2.0 * math.pi, 2)
    nx = 0.3 * np.sin(2.0 * math.pi * 3.0 * uu / W + p1) + 0.02 * rng.uniform(-1.0, 1.0, (H, W))
    ny = 0.3 * np.cos(2.0 * math.pi * 2.0 * vv / H + p2) + 0.02 * rng.uniform(-1.0, 1.0, (H, W))
    alpha = np.where(on, rng.uniform(0.6, 1.0, (H, W)), 0.0)
    normal = np.stack([nx, ny, -np.ones((H, W))], -1) * alpha[..., None]
    dist = np.where(on, depth * rng.uniform(0.6, 1.0, (H, W)), 0.0)
    n_contrib = np.where(on, rng.integers(1, 40, (H, W)), 0).astype(np.int32)
    soft = n_contrib * rng.uniform(0.3, 1.0, (H, W))
    f32 = np.float32
    return RenderedChannels(rng.random((H, W, 3)).astype(f32), dist.astype(f32), normal.astype(f32),
                            alpha.astype(f32), depth.astype(f32), n_contrib, soft.astype(f32))


# --------------------------------------------------------------------------
# voting-filter workload (Sec. 4.1): sparse SfM points and coarse building
# masks of many views
# --------------------------------------------------------------------------

VOTE_CONFIG_INDEX = 5


@dataclasses.dataclass
class VoteWorkload:
    points: np.ndarray        # float32 [M,3] sparse points (surface samples + noise)
    on_building: np.ndarray   # bool [M]: drawn on a box surface (else on the ground)
    cams: List[Camera]
    masks: List[np.ndarray]   # uint8 [H,W] coarse building masks
    tau: int


def surface_points(rng, boxes: Sequence[Box], n: int, ground: float = 200.0, noise: float = 0.05):
    """n points on the box surfaces and the ground plane, placed proportionally to
    area, with isotropic N(0, noise) metres of jitter (SfM triangulation noise).
    Returns the points and whether each lies on a box."""
    S = _surfaces(boxes, ground)
    areas = np.array([np.linalg.norm(np.cross(u, v)) for _, u, v, _ in S])
    counts = rng.multinomial(n, areas / areas.sum())
    pts, onb = [], []
    for k, ((o, u, v, _), c) in enumerate(zip(S, counts)):
        if c == 0:
            continue
        a = rng.random((c, 1))
        b = rng.random((c, 1))
        pts.append(o[None] + a * u[None] + b * v[None] + rng.normal(0.0, noise, (c, 3)))
        onb.append(np.full(c, k > 0))
    perm = rng.permutation(n)
    return np.concatenate(pts, 0)[perm].astype(np.float32), np.concatenate(onb, 0)[perm]


def coarse_mask(rng, truth: np.ndarray, n_blobs=(3, 8), radius=(40.0, 250.0)) -> np.ndarray:
    """A coarse segmentation of the kind the voting filter cleans up: the true
    building mask plus a few false-positive ellipses (ground taken for building)."""
    H, W = truth.shape
    m = truth.copy()
    scale = W / 5472.0
    for _ in range(int(rng.integers(n_blobs[0], n_blobs[1] + 1))):
        cx, cy = rng.uniform(0, W), rng.uniform(0, H)
        rx, ry = rng.uniform(radius[0], radius[1], 2) * scale
        x0, x1 = int(max(0, cx - rx)), int(min(W, cx + rx + 1))
        y0, y1 = int(max(0, cy - ry)), int(min(H, cy + ry + 1))
        if x0 >= x1 or y0 >= y1:
            continue
        yy, xx = np.mgrid[y0:y1, x0:x1]
        blob = ((xx + 0.5 - cx) / rx) ** 2 + ((yy + 0.5 - cy) / ry) ** 2 <= 1.0
        m[y0:y1, x0:x1] |= blob.astype(np.uint8)
    return m


def vote_workload(n_points: int = 1_000_000, n_views: int = 32, width: int = 5472, height: int = 3648,
                  mask_step: int = 4, tau: int = 3, coverage: float = 0.35) -> VoteWorkload:
    """Sparse points of a 40-building scene (the config-1 scene generator) seen by
    n_views oblique aerial cameras circling it (azimuth spread over 360 deg,
    pitch 45 / 60 deg, altitude 120 +- 10 m, aim jittered by +-30 m), each with a
    coarse mask: the ray-cast building mask (cast on a mask_step grid and
    replicated to full resolution) plus false-positive blobs."""
    rs, rc, rm, _ = streams(VOTE_CONFIG_INDEX)

    def cams_fn(r):
        cams = []
        for j in range(n_views):
            az = 360.0 * j / max(n_views, 1) + r.uniform(-5.0, 5.0)
            look = (r.uniform(-30.0, 30.0), r.uniform(-30.0, 30.0), 0.0)
            cams.append(aerial_camera(width, height, 120.0 + r.uniform(-10.0, 10.0), (45.0, 60.0)[j % 2], az, look))
        return cams

    scale = 1.0
    state = rs.bit_generator.state
    cstate = rc.bit_generator.state
    for _ in range(6):
        rs.bit_generator.state = state
        rc.bit_generator.state = cstate
        boxes = random_boxes(rs, 40, area=160.0, footprint_scale=scale)
        cams = cams_fn(rc)
        step = max(1, min(16, width // 64))
        cov = raycast_box_mask(boxes, cams[0], step=step).mean() if cams else coverage
        if abs(cov - coverage) <= 0.05:
            break
        scale = min(2.0, max(0.25, scale * math.sqrt(coverage / max(cov, 1e-3))))
    pts, onb = surface_points(rs, boxes, n_points, ground=200.0)
    masks = []
    for c in cams:
        t = raycast_box_mask(boxes, c, step=mask_step)
        if mask_step > 1:
            t = np.repeat(np.repeat(t, mask_step, 0), mask_step, 1)[:height, :width]
        masks.append(coarse_mask(rm, np.ascontiguousarray(t)))
    return VoteWorkload(pts, onb, cams, masks, tau)


# --------------------------------------------------------------------------
# depth maps for the TSDF workload (Sec. 4.4): building and background depth
# maps of many views, ray-cast from the box scene
# --------------------------------------------------------------------------

TSDF_CONFIG_INDEX = 6


def raycast_depth(boxes: Sequence[Box], cam: Camera, ground: float = 200.0, step: int = 1):
    """Camera-z depth of the nearest hit (boxes and the ground square z = 0 of side
    `ground`) for each pixel centre of a `step` grid, 0 where the ray hits
    nothing, and whether that nearest hit is a box."""
    H, W = cam.height, cam.width
    R = cam.R.astype(np.float64)
    t = cam.t.astype(np.float64)
    C = -R.T @ t
    us = np.arange(0, W, step) + 0.5
    vs = np.arange(0, H, step) + 0.5
    uu, vv = np.meshgrid(us, vs)
    dcam = np.stack([(uu - cam.cx) / cam.fx, (vv - cam.cy) / cam.fy, np.ones_like(uu)], -1)
    dw = dcam @ R  # R^T d: a hit at C + z dw has camera depth z
    depth = np.full(uu.shape, np.inf)
    with np.errstate(divide="ignore", invalid="ignore"):
        zg = -C[2] / dw[..., 2]
        gx, gy = C[0] + zg * dw[..., 0], C[1] + zg * dw[..., 1]
        okg = (zg > 0) & (np.abs(gx) <= ground / 2) & (np.abs(gy) <= ground / 2)
    depth = np.where(okg, zg, depth)
    isbox = np.zeros(uu.shape, bool)
    for b in boxes:
        lo = np.array([b.x0, b.y0, 0.0])
        hi = np.array([b.x1, b.y1, b.h])
        # pixel rectangle of the projected box (whole grid if a corner is behind)
        corners = np.array([[x, y, z] for x in (b.x0, b.x1) for y in (b.y0, b.y1) for z in (0.0, b.h)])
        pc = corners @ R.T + t
        if np.all(pc[:, 2] <= 1e-6):
            continue
        if np.any(pc[:, 2] <= 1e-6):
            iu = np.arange(len(us))
            iv = np.arange(len(vs))
        else:
            px = cam.fx * pc[:, 0] / pc[:, 2] + cam.cx
            py = cam.fy * pc[:, 1] / pc[:, 2] + cam.cy
            iu = np.nonzero((us >= px.min() - 2) & (us <= px.max() + 2))[0]
            iv = np.nonzero((vs >= py.min() - 2) & (vs <= py.max() + 2))[0]
        if len(iu) == 0 or len(iv) == 0:
            continue
        sub = np.ix_(iv, iu)
        d = dw[sub]
        with np.errstate(divide="ignore", invalid="ignore"):
            inv = 1.0 / d
            t0 = (lo - C) * inv
            t1 = (hi - C) * inv
        tmin = np.nanmax(np.minimum(t0, t1), axis=-1)
        tmax = np.nanmin(np.maximum(t0, t1), axis=-1)
        cur = depth[sub]
        hit = (tmax >= np.maximum(tmin, 0.0)) & (tmin > 0) & (tmin < cur)
        depth[sub] = np.where(hit, tmin, cur)
        isbox[sub] |= hit
    depth = np.where(np.isfinite(depth), depth, 0.0)
    return depth.astype(np.float32), isbox


@dataclasses.dataclass
class TsdfWorkload:
    cams: List[Camera]
    building: List[np.ndarray]     # float32 [H,W] building depth maps (0 = none)
    background: List[np.ndarray]   # float32 [H,W] background depth maps (0 = none)
    origin: Tuple[float, float, float]
    voxel: float
    dims: Tuple[int, int, int]     # nx, ny, nz
    trunc: float


def tsdf_workload(n_views: int = 32, width: int = 2736, height: int = 1824, voxel: float = 0.25,
                  step: int = 2, band: int = 3, noise: float = 0.01, coverage: float = 0.35) -> TsdfWorkload:
    """The config-1 building scene (40 boxes, footprints rescaled to ~35% mask
    coverage in the first view) seen by n_views oblique aerial cameras circling
    it; per view a building depth map (the ray-cast depth on the building pixels
    dilated by `band` pixels) and a background depth map (on the pixels outside
    the building mask eroded by `band`), each with independent N(0, noise) m
    jitter, so they overlap in a band around every building outline.  The grid
    covers the 160 x 160 m block up to 50 m at `voxel` m, truncation 4 voxels."""
    from scipy import ndimage
    rs, rc, rm, _ = streams(TSDF_CONFIG_INDEX)

    def cams_fn(r):
        cams = []
        for j in range(n_views):
            az = 360.0 * j / max(n_views, 1) + r.uniform(-5.0, 5.0)
            look = (r.uniform(-30.0, 30.0), r.uniform(-30.0, 30.0), 0.0)
            cams.append(aerial_camera(width, height, 120.0 + r.uniform(-10.0, 10.0), (45.0, 60.0)[j % 2], az, look))
        return cams

    scale = 1.0
    state, cstate = rs.bit_generator.state, rc.bit_generator.state
    for _ in range(6):
        rs.bit_generator.state, rc.bit_generator.state = state, cstate
        boxes = random_boxes(rs, 40, area=160.0, footprint_scale=scale)
        cams = cams_fn(rc)
        cov = raycast_box_mask(boxes, cams[0], step=max(1, min(16, width // 64))).mean() if cams else coverage
        if abs(cov - coverage) <= 0.05:
            break
        scale = min(2.0, max(0.25, scale * math.sqrt(coverage / max(cov, 1e-3))))
    bld, bkg = [], []
    for c in cams:
        d, isbox = raycast_depth(boxes, c, 200.0, step)
        if step > 1:
            d = np.repeat(np.repeat(d, step, 0), step, 1)[:height, :width]
            isbox = np.repeat(np.repeat(isbox, step, 0), step, 1)[:height, :width]
        mb = ndimage.binary_dilation(isbox, iterations=band)
        mg = ~ndimage.binary_erosion(isbox, iterations=band)
        has = d > 0
        b = np.where(mb & has, d + rm.normal(0.0, noise, d.shape), 0.0)
        g = np.where(mg & has, d + rm.normal(0.0, noise, d.shape), 0.0)
        bld.append(np.maximum(b, 0.0).astype(np.float32))
        bkg.append(np.maximum(g, 0.0).astype(np.float32))
    nx = ny = int(round(160.0 / voxel))
    nz = int(round(50.0 / voxel))
    return TsdfWorkload(cams, bld, bkg, (-80.0, -80.0, -1.0), voxel, (nx, ny, nz), 4 * voxel)
