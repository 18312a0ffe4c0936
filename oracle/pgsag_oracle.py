"""FP64 CPU oracle for PG-SAG's masked differentiable Gaussian-splat step.

TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and bench.py's
cpu_baseline / reference leg may import or call this module.  It shares no code
with the CUDA library (no kernels, helpers, tables or constants generators) and
never reads anything the CUDA path produced.

It is the plain definition of what the path computes, written per stage in the
paper's notation, evaluated in float64 with PyTorch CPU ops; gradients are taken
by autograd through that definition (the derivative of the definition, exact up
to rounding).  Passages followed:

* Sec. 3.1, Eq. 1 -- front-to-back alpha blending C = sum c_i a_i T_i,
  T_i = prod_{j<i} (1 - a_j) (the product index of Eq. 1 read as j < i).
* Sec. 3.1 (by citation to 3DGS) -- EWA projection of each 3D Gaussian to a 2D
  Gaussian, spherical-harmonics colour, opacity.
* Sec. 3.1, Eq. 2 -- rendered normal N = sum R_c n_i a_i T_i.
* Sec. 3.1, Eq. 3 -- rendered plane distance D = sum d_i a_i T_i; the garbled
  d_i formula is read as the camera-centre-to-plane distance d_i = -n_c . mu_c
  with camera-frame normal n_c facing the camera.
* Sec. 3.1, Eq. 4 -- unbiased depth  Depth(p) = D / (-N(p) . K^-1 p~).
* Sec. 4.2, Eq. 8 -- boundary-aware normal loss, w = 0.1 on mask boundaries.
* Sec. 4.3, Eq. 9 -- GC-load statistic std_i(g_i / w_i).
* Sec. 4.3, Eq. 10-11 -- loss weights (lambda = 0.41, lambda_3 = 100,
  lambda_4 = 0.01) and the combined objective
  L = (1 - lambda) (L_rgb + lambda_3 L_s + lambda_4 L_ban) + lambda L_GC-load
  over the terms defined in the paper itself (L_mvgeo and L_mvrgb are defined
  only by citation and left out).
* Sec. 4.3 (by citation to PGSR) -- flattening loss L_s, read as the mean over
  the Gaussians of min(s_1, s_2, s_3), s = exp(log-scale).
* Sec. 4.3, Eq. 9 with a differentiable count: g~_i = sum of the alphas of the
  Gaussians blended into pixel i (the integer count g_i has no gradient; the
  soft count is the surrogate that lets the GC-load term shape the Gaussians).
* L_rgb with D-SSIM (3DGS by citation, "only the refined building masks are
  involved"): L_rgb = (1 - 0.2) L1 + 0.2 (1 - SSIM_M), SSIM_M = mean over the mask
  pixels and the 3 channels of the SSIM map; the SSIM window is 3DGS's 11 x 11
  Gaussian (sigma 1.5) restricted to the rendered set R and renormalised over it
  (the rendered image exists on R only), C1 = 0.01^2, C2 = 0.03^2.

Readings of passages where the paper is silent (3DGS constants by citation):
alpha = min(0.99, o exp(-1/2 d^T Q d)); a Gaussian enters a pixel iff
alpha >= 1/255; blending stops *before* the first entering Gaussian whose
T (1 - alpha) < 1e-4; near plane 0.2; 0.3 px^2 low-pass dilation; Jacobian
clamp 1.3 x half-FOV; SH colour offset +0.5 and clamp at 0; background 0.

Order of Gaussians along a pixel: ascending (depth key, Gaussian index), where
the depth key is the camera-space z evaluated in float32 in a fixed operation
order without fused multiply-add (`depth_key_f32`).  This discrete decision is
taken in the kernel's precision on both sides; everything else is float64.
"""
from __future__ import annotations

import math
from dataclasses import dataclass
from typing import Dict, Optional

import numpy as np
import torch

DT = torch.float64

# Rasteriser constants (3DGS by citation, Sec. 3.1)
ALPHA_MIN = 1.0 / 255.0
ALPHA_MAX = 0.99
T_MIN = 1e-4
COV_DILATION = 0.3
JAC_CLAMP = 1.3
SH_OFFSET = 0.5
# Loss constants (Sec. 4.2 Eq. 8, Sec. 4.3 Eq. 11)
W_BOUNDARY = 0.1
LAMBDA_GC = 0.41
LAMBDA_BAN = 0.01
LAMBDA_FLAT = 100.0
LAMBDA_DSSIM = 0.2          # 3DGS: L_rgb = (1 - 0.2) L1 + 0.2 D-SSIM
SSIM_C1, SSIM_C2 = 0.01 ** 2, 0.03 ** 2
SSIM_RADIUS, SSIM_SIGMA = 5, 1.5
# Validity threshold for Eq. 4 (ray-plane intersection must be in front)
RAY_DOT_MIN = 1e-8
# Relative window inside which a float32 threshold decision may legitimately flip
AMBIG_REL = 3e-5


# ---------------------------------------------------------------------------
# spherical harmonics (real, orthonormal, no Condon-Shortley phase)
# ---------------------------------------------------------------------------

def _legendre_deriv_poly(l: int, m: int) -> np.ndarray:
    """Power-series coefficients (ascending) of d^m/dz^m P_l(z)."""
    from numpy.polynomial import legendre as L
    c = np.zeros(l + 1)
    c[l] = 1.0
    if m > 0:
        c = L.legder(c, m)
    return L.leg2poly(c)


def sh_basis(dirs: torch.Tensor, degree: int = 3) -> torch.Tensor:
    """Real SH basis Y_lm at unit directions, index l*l + l + m.

    Y_lm = K_lm * (d^|m| P_l / dz^|m|)(z) * {sqrt2 Re((x+iy)^m), 1, sqrt2 Im((x+iy)^|m|)}
    for m > 0, m = 0, m < 0, with K_lm = sqrt((2l+1)/(4 pi) (l-|m|)!/(l+|m|)!).
    On the unit sphere (x+iy)^m = sin^m(theta) e^{i m phi}, so this is the
    textbook real harmonic written in Cartesian form (smooth everywhere).
    """
    x, y, z = dirs[..., 0], dirs[..., 1], dirs[..., 2]
    # (x + i y)^m  real / imaginary parts
    re = [torch.ones_like(x)]
    im = [torch.zeros_like(x)]
    for m in range(1, degree + 1):
        re.append(re[-1] * x - im[-1] * y)
        im.append(re[-2] * y + im[-1] * x)
    out = []
    for l in range(degree + 1):
        for m in range(-l, l + 1):
            am = abs(m)
            K = math.sqrt((2 * l + 1) / (4 * math.pi) * math.factorial(l - am) / math.factorial(l + am))
            coeffs = _legendre_deriv_poly(l, am)
            poly = torch.zeros_like(z)
            for c in coeffs[::-1]:
                poly = poly * z + float(c)
            if m > 0:
                out.append(math.sqrt(2.0) * K * poly * re[am])
            elif m == 0:
                out.append(K * poly)
            else:
                out.append(math.sqrt(2.0) * K * poly * im[am])
    return torch.stack(out, -1)


# ---------------------------------------------------------------------------
# per-Gaussian projection (Sec. 3.1)
# ---------------------------------------------------------------------------

def quat_to_rotmat(q: torch.Tensor) -> torch.Tensor:
    """Rotation by the unit quaternion q = (w, v):  R = I + 2 w [v]x + 2 [v]x^2."""
    w = q[..., 0]
    v = q[..., 1:]
    zero = torch.zeros_like(w)
    vx = torch.stack([
        torch.stack([zero, -v[..., 2], v[..., 1]], -1),
        torch.stack([v[..., 2], zero, -v[..., 0]], -1),
        torch.stack([-v[..., 1], v[..., 0], zero], -1)], -2)
    eye = torch.eye(3, dtype=q.dtype).expand(vx.shape)
    return eye + 2.0 * w[..., None, None] * vx + 2.0 * (vx @ vx)


def depth_key_f32(means_f32: np.ndarray, R_f32: np.ndarray, t_f32: np.ndarray) -> np.ndarray:
    """Camera-space z in float32, evaluated as ((R20*x + R21*y) + R22*z) + t2 with
    every product and sum rounded separately (no FMA).  Used only for the order
    of Gaussians and the near-plane test."""
    m = np.asarray(means_f32, np.float32)
    R = np.asarray(R_f32, np.float32)
    t = np.asarray(t_f32, np.float32)
    a = m[:, 0] * R[2, 0]
    b = m[:, 1] * R[2, 1]
    c = m[:, 2] * R[2, 2]
    with np.errstate(invalid="ignore", over="ignore"):
        return ((a + b) + c) + t[2]


@dataclass
class Cam:
    R: torch.Tensor   # [3,3] float64
    t: torch.Tensor   # [3]
    fx: float
    fy: float
    cx: float
    cy: float
    width: int
    height: int
    znear: float
    R32: np.ndarray
    t32: np.ndarray

    @staticmethod
    def from_synth(c) -> "Cam":
        return Cam(torch.tensor(np.asarray(c.R, np.float64), dtype=DT), torch.tensor(np.asarray(c.t, np.float64), dtype=DT),
                   float(c.fx), float(c.fy), float(c.cx), float(c.cy), int(c.width), int(c.height), float(c.znear),
                   np.asarray(c.R, np.float32), np.asarray(c.t, np.float32))


def params_from_synth(g, requires_grad=False) -> Dict[str, torch.Tensor]:
    p = {k: torch.tensor(np.asarray(getattr(g, k), np.float64), dtype=DT)
         for k in ("means", "log_scales", "quats", "opacity_logit", "sh")}
    if requires_grad:
        for v in p.values():
            v.requires_grad_(True)
    return p


def project(p: Dict[str, torch.Tensor], cam: Cam, means_f32: Optional[np.ndarray] = None) -> Dict[str, torch.Tensor]:
    """Per-Gaussian 2D quantities for one view.

    Returns mean2d [N,2] (pixels), conic [N,3] = (Q_xx, Q_xy, Q_yy) of Q = Sigma'^-1,
    cov2d [N,3], opacity [N], rgb [N,3], normal [N,3] (camera frame, facing the
    camera), dist [N] (= -n_c . mu_c), key [N] float32 depth key, visible [N] bool,
    flip_ambiguous [N] bool.
    """
    means, ls, quats = p["means"], p["log_scales"], p["quats"]
    n = means.shape[0]
    s = torch.exp(ls)
    qn = quats / torch.linalg.norm(quats, dim=-1, keepdim=True)
    Rq = quat_to_rotmat(qn)
    o = torch.sigmoid(p["opacity_logit"])
    mc = means @ cam.R.T + cam.t
    x, y, z = mc[:, 0], mc[:, 1], mc[:, 2]

    m32 = means_f32 if means_f32 is not None else means.detach().numpy().astype(np.float32)
    key = depth_key_f32(m32, cam.R32, cam.t32)
    finite = torch.isfinite(means).all(-1) & torch.isfinite(ls).all(-1) & torch.isfinite(quats).all(-1) \
        & torch.isfinite(p["opacity_logit"]) & torch.isfinite(p["sh"]).reshape(n, -1).all(-1)
    visible = torch.from_numpy(np.asarray(key > np.float32(cam.znear))) & finite

    # 3D covariance Sigma = R S S^T R^T
    M = Rq * s[:, None, :]
    Sigma = M @ M.transpose(1, 2)
    # EWA: Sigma' = J W Sigma W^T J^T + 0.3 I, J = Jacobian of the pinhole map
    zs = torch.where(visible, z, torch.ones_like(z))
    limx = JAC_CLAMP * 0.5 * cam.width / cam.fx
    limy = JAC_CLAMP * 0.5 * cam.height / cam.fy
    tx = torch.clamp(x / zs, -limx, limx) * zs
    ty = torch.clamp(y / zs, -limy, limy) * zs
    zero = torch.zeros_like(zs)
    J = torch.stack([torch.stack([cam.fx / zs, zero, -cam.fx * tx / zs ** 2], -1),
                     torch.stack([zero, cam.fy / zs, -cam.fy * ty / zs ** 2], -1)], -2)
    T2 = J @ cam.R
    cov = T2 @ Sigma @ T2.transpose(1, 2)
    a = cov[:, 0, 0] + COV_DILATION
    b = cov[:, 0, 1]
    c = cov[:, 1, 1] + COV_DILATION
    det = a * c - b * b
    conic = torch.stack([c / det, -b / det, a / det], -1)
    mean2d = torch.stack([cam.fx * x / zs + cam.cx, cam.fy * y / zs + cam.cy], -1)

    # colour from degree-3 SH at the viewing direction
    campos = -cam.R.T @ cam.t
    dvec = means - campos
    dirs = dvec / torch.linalg.norm(dvec, dim=-1, keepdim=True)
    Y = sh_basis(dirs, 3)
    rgb = torch.clamp_min(torch.einsum("nk,nkc->nc", Y, p["sh"]) + SH_OFFSET, 0.0)

    # flattened-Gaussian normal: axis of the smallest scale, turned to face the camera
    k = torch.argmin(ls.detach(), dim=1)
    n_w = Rq[torch.arange(n), :, k]
    n_c = n_w @ cam.R.T
    dot = (n_c * mc).sum(-1)
    sign = torch.where(dot.detach() > 0, -1.0, 1.0).to(DT)
    n_c = n_c * sign[:, None]
    dist = -(n_c * mc).sum(-1)
    cosang = dot.detach().abs() / (torch.linalg.norm(mc.detach(), dim=-1) + 1e-300)
    flip_amb = cosang < 1e-6
    return dict(mean2d=mean2d, conic=conic, cov2d=torch.stack([a, b, c], -1), opacity=o, rgb=rgb,
                normal=n_c, dist=dist, key=torch.from_numpy(np.asarray(key, np.float32)),
                visible=visible, flip_ambiguous=flip_amb, z=z, mc_norm=torch.linalg.norm(mc.detach(), dim=-1))


# ---------------------------------------------------------------------------
# mask preparation (Sec. 4.1 masks, Sec. 4.2 boundaries)
# ---------------------------------------------------------------------------

def mask_sets(mask: np.ndarray):
    """M = building mask; E = 3x3 morphological gradient (dilation - erosion) of M,
    the mask boundary of Eq. 8; R = 3x3 dilation of M, the rendered set (every M pixel
    has its 4 neighbours rendered).  Neighbours outside the image are ignored."""
    M = np.asarray(mask) != 0
    H, W = M.shape
    P = np.pad(M, 1, mode="edge")
    win = np.stack([P[dy:dy + H, dx:dx + W] for dy in range(3) for dx in range(3)], 0)
    dil = win.any(0)
    ero = win.all(0)
    return M, dil & ~ero, dil


# ---------------------------------------------------------------------------
# per-pixel compositing (Eq. 1-3)
# ---------------------------------------------------------------------------

def _ellipse_bbox(pr, visible):
    """Pixel-index bounds (inclusive) of the alpha >= 1/255 region, +1 px margin."""
    o = pr["opacity"].detach()
    cov = pr["cov2d"].detach()
    m = pr["mean2d"].detach()
    lg = torch.log(255.0 * o)
    ok = visible & (lg > 0)
    r2 = torch.clamp(2.0 * lg, min=0.0)
    ex = torch.sqrt(r2 * cov[:, 0]) + 1.0
    ey = torch.sqrt(r2 * cov[:, 2]) + 1.0
    u0 = torch.ceil(m[:, 0] - ex - 0.5)
    u1 = torch.floor(m[:, 0] + ex - 0.5)
    v0 = torch.ceil(m[:, 1] - ey - 0.5)
    v1 = torch.floor(m[:, 1] + ey - 0.5)
    return ok, u0, u1, v0, v1


def candidate_pairs(pr, width, height, pix_u=None, pix_v=None, chunk=64):
    """(pixel row, Gaussian) candidate pairs: every Gaussian whose alpha >= 1/255
    region may contain the pixel.  Either all image pixels (pix_u None) or the given
    pixel list.  Returns (pixel index into the list / linear image index, gaussian)."""
    ok, u0, u1, v0, v1 = _ellipse_bbox(pr, pr["visible"])
    if pix_u is None:
        u0c = torch.clamp(u0, 0, width - 1)
        u1c = torch.clamp(u1, 0, width - 1)
        v0c = torch.clamp(v0, 0, height - 1)
        v1c = torch.clamp(v1, 0, height - 1)
        ok = ok & (u1 >= 0) & (v1 >= 0) & (u0 <= width - 1) & (v0 <= height - 1)
        gid = torch.nonzero(ok).flatten()
        nu = (u1c[gid] - u0c[gid] + 1).long()
        nv = (v1c[gid] - v0c[gid] + 1).long()
        cnt = nu * nv
        g = torch.repeat_interleave(gid, cnt)
        start = torch.cumsum(cnt, 0) - cnt
        local = torch.arange(int(cnt.sum())) - torch.repeat_interleave(start, cnt)
        nu_r = torch.repeat_interleave(nu, cnt)
        uu = torch.repeat_interleave(u0c[gid].long(), cnt) + local % nu_r
        vv = torch.repeat_interleave(v0c[gid].long(), cnt) + local // nu_r
        return vv * width + uu, g
    pu = torch.as_tensor(pix_u, dtype=torch.long)
    pv = torch.as_tensor(pix_v, dtype=torch.long)
    gid = torch.nonzero(ok).flatten()
    U0, U1, V0, V1 = u0[gid], u1[gid], v0[gid], v1[gid]
    P_, G_ = [], []
    for s in range(0, len(pu), chunk):
        cu = pu[s:s + chunk, None].to(DT)
        cv = pv[s:s + chunk, None].to(DT)
        hit = (cu >= U0[None]) & (cu <= U1[None]) & (cv >= V0[None]) & (cv <= V1[None])
        pi, gi = torch.nonzero(hit, as_tuple=True)
        P_.append(pi + s)
        G_.append(gid[gi])
    return torch.cat(P_) if P_ else torch.zeros(0, dtype=torch.long), torch.cat(G_) if G_ else torch.zeros(0, dtype=torch.long)


def composite(pr, pu: torch.Tensor, pv: torch.Tensor, pair_pix: torch.Tensor, pair_g: torch.Tensor):
    """Front-to-back blending (Eq. 1-3) at pixel centres (pu+0.5, pv+0.5).

    pair_pix indexes into (pu, pv).  Returns dict with rgb [P,3], dist D [P],
    normal N [P,3], alpha A [P], n_contrib [P] (long), ambiguous [P] (bool),
    final_T [P], and mag: per channel the blended magnitude of the quantity's own
    rounding scale (|c| for colour, |n| for normal components, |mu_c| for the
    plane distance), which bounds the rounding error of any evaluation."""
    Pn = pu.shape[0]
    key = pr["key"].numpy()
    # order: pixel, then (depth key, gaussian index)
    if pair_g.numel():
        order = np.lexsort((pair_g.numpy(), key[pair_g.numpy()], pair_pix.numpy()))
        pair_pix = pair_pix[order]
        pair_g = pair_g[order]
    cnt = torch.bincount(pair_pix, minlength=Pn)
    L = int(cnt.max()) if Pn and pair_g.numel() else 0
    start = torch.cumsum(cnt, 0) - cnt
    slot = torch.arange(pair_pix.numel()) - start[pair_pix]
    idx = torch.full((Pn, max(L, 1)), -1, dtype=torch.long)
    idx[pair_pix, slot] = pair_g
    valid = idx >= 0
    gi = torch.clamp(idx, min=0)

    m2 = pr["mean2d"][gi]                  # [P,L,2]
    q = pr["conic"][gi]                    # [P,L,3]
    o = pr["opacity"][gi]
    dx = (pu.to(DT) + 0.5)[:, None] - m2[..., 0]
    dy = (pv.to(DT) + 0.5)[:, None] - m2[..., 1]
    power = -0.5 * (q[..., 0] * dx * dx + 2.0 * q[..., 1] * dx * dy + q[..., 2] * dy * dy)
    raw = o * torch.exp(power)
    alpha = torch.clamp_max(raw, ALPHA_MAX)
    enters = valid & (raw.detach() >= ALPHA_MIN)
    amb = (valid & ((raw.detach() * 255.0 - 1.0).abs() < AMBIG_REL)).any(1)
    amb = amb | (valid & enters & pr["flip_ambiguous"][gi]).any(1)

    T = torch.ones(Pn, dtype=DT)
    C = torch.zeros(Pn, 3, dtype=DT)
    N = torch.zeros(Pn, 3, dtype=DT)
    D = torch.zeros(Pn, dtype=DT)
    # magnitude sums sum_i w_i |x_i| of each blended channel: the scale of the
    # rounding error of any evaluation of these sums.  A normal component is
    # computed from a unit vector, so its error scales with |n| = 1; the plane
    # distance d = -n . mu_c is a dot product, so its error scales with |mu_c|.
    magC = torch.zeros(Pn, 3, dtype=DT)
    magN = torch.zeros(Pn, 3, dtype=DT)
    magD = torch.zeros(Pn, dtype=DT)
    mcn = pr["mc_norm"][gi]
    ncon = torch.zeros(Pn, dtype=torch.long)
    soft = torch.zeros(Pn, dtype=DT)
    done = torch.zeros(Pn, dtype=torch.bool)
    col = pr["rgb"][gi]
    nor = pr["normal"][gi]
    dst = pr["dist"][gi]
    for j in range(L):
        a = alpha[:, j]
        ent = enters[:, j] & ~done
        test = T * (1.0 - a)
        td = test.detach()
        amb = amb | (ent & ((td / T_MIN - 1.0).abs() < AMBIG_REL))
        stop = ent & (td < T_MIN)
        done = done | stop
        blend = ent & ~stop
        w = torch.where(blend, a * T, torch.zeros_like(a))
        C = C + w[:, None] * col[:, j]
        N = N + w[:, None] * nor[:, j]
        D = D + w * dst[:, j]
        wd = w.detach()
        magC = magC + wd[:, None] * col[:, j].detach().abs()
        magN = magN + wd[:, None] * torch.linalg.norm(nor[:, j].detach(), dim=-1, keepdim=True)
        magD = magD + wd * mcn[:, j]
        T = torch.where(blend, test, T)
        ncon = ncon + blend.long()
        soft = soft + torch.where(blend, a, torch.zeros_like(a))
    return dict(rgb=C, normal=N, dist=D, alpha=1.0 - T, final_T=T, n_contrib=ncon, soft_count=soft, ambiguous=amb,
                mag=dict(rgb=magC, normal=magN, dist=magD, alpha=(1.0 - T).detach()))


def pixel_rays(cam: Cam, pu: torch.Tensor, pv: torch.Tensor) -> torch.Tensor:
    """r = K^-1 (u+1/2, v+1/2, 1)."""
    return torch.stack([((pu.to(DT) + 0.5) - cam.cx) / cam.fx, ((pv.to(DT) + 0.5) - cam.cy) / cam.fy,
                        torch.ones(pu.shape[0], dtype=DT)], -1)


def unbiased_depth(out, cam: Cam, pu, pv):
    """Eq. 4: Depth = D / (-N . r).  A pixel is valid iff something was blended,
    -N.r > 1e-8 and D > 0; invalid pixels get depth 0."""
    r = pixel_rays(cam, pu, pv)
    sdot = -(out["normal"] * r).sum(-1)
    valid = (out["n_contrib"] > 0) & (sdot.detach() > RAY_DOT_MIN) & (out["dist"].detach() > 0)
    depth = torch.where(valid, out["dist"] / torch.where(valid, sdot, torch.ones_like(sdot)), torch.zeros_like(sdot))
    return depth, valid


def render_view(p, cam: Cam, mask: np.ndarray, means_f32=None):
    """Render every pixel of the render set R of one view.  Returns projection,
    per-pixel outputs scattered to dense [H, W, ...] images (zero outside R), and
    the sets M, E, R."""
    M, E, R = mask_sets(mask)
    pr = project(p, cam, means_f32)
    H, W = cam.height, cam.width
    pv_all, pu_all = np.nonzero(R)
    pu = torch.from_numpy(pu_all.astype(np.int64))
    pv = torch.from_numpy(pv_all.astype(np.int64))
    lin, g = candidate_pairs(pr, W, H)
    # keep pairs on R pixels only, re-indexed into the R pixel list
    rid = torch.full((H * W,), -1, dtype=torch.long)
    rid[pv * W + pu] = torch.arange(pu.shape[0])
    sel = rid[lin] >= 0
    out = composite(pr, pu, pv, rid[lin[sel]], g[sel])
    depth, valid = unbiased_depth(out, cam, pu, pv)
    return pr, out, depth, valid, (pu, pv), (M, E, R)


def dense(vals: torch.Tensor, pu, pv, H, W):
    """Scatter per-pixel values into a dense image (zeros elsewhere), differentiable."""
    shape = (H * W,) + tuple(vals.shape[1:])
    img = torch.zeros(shape, dtype=vals.dtype)
    img = img.index_put((pv * W + pu,), vals)
    return img.reshape((H, W) + tuple(vals.shape[1:]))


# ---------------------------------------------------------------------------
# losses (Eq. 8, L1 photometric term, Eq. 9)
# ---------------------------------------------------------------------------

def losses(out, depth, valid, pix, sets, cam: Cam, target: np.ndarray, dssim: bool = False):
    """L_rgb = mean over M of |C - C*|_1 / 3.

    L_ban (Eq. 8) = (1/|V|) sum_{i in V} w_i || n_depth,i - n_r,i ||^2 with
    n_depth = normalize((P[v+1]-P[v-1]) x (P[u+1]-P[u-1])), P = Depth * r,
    n_r = N / |N|, w_i = 0.1 on the mask boundary E and 1 elsewhere, and V the mask
    pixels off the image border that are valid, whose 4 neighbours are in R and
    valid, and whose cross product is non-zero.

    Returns dict of scalars (torch, differentiable) and |M|, |V|."""
    pu, pv = pix
    M, E, R = sets
    H, W = cam.height, cam.width
    C = dense(out["rgb"], pu, pv, H, W)
    N = dense(out["normal"], pu, pv, H, W)
    Dp = dense(depth, pu, pv, H, W)
    Vd = np.zeros((H, W), bool)
    Vd[pv.numpy(), pu.numpy()] = valid.numpy()
    Mt = torch.from_numpy(M)
    tgt = torch.from_numpy(np.asarray(target, np.float64))
    nM = int(M.sum())
    l_rgb = (C - tgt).abs().sum(-1)[Mt].sum() / (3.0 * max(nM, 1)) if nM else torch.zeros((), dtype=DT) + 0 * C.sum()
    ssim_m = None
    if dssim:
        l_rgb, ssim_m = l_rgb_dssim(C, tgt, M, R)

    # back-projected points
    uu = torch.arange(W, dtype=DT)[None, :].expand(H, W)
    vv = torch.arange(H, dtype=DT)[:, None].expand(H, W)
    ray = torch.stack([(uu + 0.5 - cam.cx) / cam.fx, (vv + 0.5 - cam.cy) / cam.fy, torch.ones(H, W, dtype=DT)], -1)
    P = Dp[..., None] * ray
    # interior candidate pixels
    cand = np.zeros((H, W), bool)
    if H >= 3 and W >= 3:
        inner = (slice(1, H - 1), slice(1, W - 1))
        nb_ok = (R[:-2, 1:-1] & Vd[:-2, 1:-1]) & (R[2:, 1:-1] & Vd[2:, 1:-1]) & \
                (R[1:-1, :-2] & Vd[1:-1, :-2]) & (R[1:-1, 2:] & Vd[1:-1, 2:])
        cand[inner] = M[inner] & Vd[inner] & nb_ok
    cv, cu = np.nonzero(cand)
    cvt, cut = torch.from_numpy(cv), torch.from_numpy(cu)
    a = P[cvt + 1, cut] - P[cvt - 1, cut]
    b = P[cvt, cut + 1] - P[cvt, cut - 1]
    cr = torch.cross(a, b, dim=-1)
    crn = torch.linalg.norm(cr, dim=-1)
    keep = crn.detach() > 0
    cvt, cut, cr, crn = cvt[keep], cut[keep], cr[keep], crn[keep]
    nd = cr / crn[:, None]
    Nv = N[cvt, cut]
    nr = Nv / torch.linalg.norm(Nv, dim=-1, keepdim=True)
    # weight built in float64 (a Python-scalar torch.where would round 0.1 to float32)
    w = torch.where(torch.from_numpy(E[cvt.numpy(), cut.numpy()]), torch.tensor(W_BOUNDARY, dtype=DT),
                    torch.tensor(1.0, dtype=DT))
    nV = int(cvt.shape[0])
    if nV:
        l_ban = (w * ((nd - nr) ** 2).sum(-1)).sum() / nV
    else:
        l_ban = torch.zeros((), dtype=DT) + 0 * C.sum()
    total = l_rgb + LAMBDA_BAN * l_ban
    return dict(l_rgb=l_rgb, l_ban=l_ban, total=total, n_mask=nM, n_valid=nV, ssim=ssim_m)


def ssim_window() -> torch.Tensor:
    """11 x 11 Gaussian window (sigma 1.5) summing to 1."""
    r = torch.arange(-SSIM_RADIUS, SSIM_RADIUS + 1, dtype=DT)
    g = torch.exp(-(r ** 2) / (2.0 * SSIM_SIGMA ** 2))
    g = g / g.sum()
    return g[:, None] * g[None, :]


def masked_ssim_map(C: torch.Tensor, T: torch.Tensor, R: np.ndarray) -> torch.Tensor:
    """SSIM per pixel and channel [H, W, 3] with the window restricted to the
    rendered set R and renormalised: every moment is the weighted mean over the
    rendered pixels of the window."""
    G = ssim_window()[None, None]
    Rt = torch.from_numpy(np.asarray(R, np.float64))
    pad = SSIM_RADIUS

    def blur(img):  # img [H, W] -> sum_k G(k - i) img(k), zero outside the image
        return torch.nn.functional.conv2d(img[None, None], G, padding=pad)[0, 0]

    Wsum = blur(Rt)
    Wd = torch.where(Wsum > 0, Wsum, torch.ones_like(Wsum))
    out = []
    for c in range(3):
        x, y = C[..., c] * Rt, T[..., c] * Rt
        mx, my = blur(x) / Wd, blur(y) / Wd
        sxx = blur(x * C[..., c]) / Wd - mx * mx
        syy = blur(y * T[..., c]) / Wd - my * my
        sxy = blur(x * T[..., c]) / Wd - mx * my
        num = (2 * mx * my + SSIM_C1) * (2 * sxy + SSIM_C2)
        den = (mx * mx + my * my + SSIM_C1) * (sxx + syy + SSIM_C2)
        out.append(num / den)
    return torch.stack(out, -1)


def l_rgb_dssim(C: torch.Tensor, T: torch.Tensor, M: np.ndarray, R: np.ndarray):
    """(1 - 0.2) L1 + 0.2 (1 - SSIM_M) over the mask pixels, and SSIM_M."""
    Mt = torch.from_numpy(M)
    nM = int(M.sum())
    if nM == 0:
        z = torch.zeros((), dtype=DT) + 0 * C.sum()
        return z, z
    l1 = (C - T).abs().sum(-1)[Mt].sum() / (3.0 * nM)
    ssim_m = masked_ssim_map(C, T, R)[Mt].mean()
    return (1.0 - LAMBDA_DSSIM) * l1 + LAMBDA_DSSIM * (1.0 - ssim_m), ssim_m


def luminance_gradient_weight(target: np.ndarray) -> np.ndarray:
    """w_i of Eq. 9, read as 1 + |Sobel(luminance)| of the target image with
    luminance Y = 0.299 R + 0.587 G + 0.114 B and replicated borders."""
    from scipy import ndimage
    t = np.asarray(target, np.float64)
    Y = 0.299 * t[..., 0] + 0.587 * t[..., 1] + 0.114 * t[..., 2]
    gx = ndimage.sobel(Y, axis=1, mode="nearest")
    gy = ndimage.sobel(Y, axis=0, mode="nearest")
    return 1.0 + np.hypot(gx, gy)


def gc_load(n_contrib: np.ndarray, weight: np.ndarray, R: np.ndarray) -> float:
    """Eq. 9: population standard deviation of g_i / w_i over the rendered pixels
    (g_i = number of Gaussians blended into pixel i)."""
    g = np.asarray(n_contrib, np.float64)[R]
    w = np.asarray(weight, np.float64)[R]
    if g.size == 0:
        return 0.0
    x = g / w
    return float(np.sqrt(np.mean((x - x.mean()) ** 2)))


def total_loss_with_gc(l_pg_geo: float, l_gc: float) -> float:
    """Eq. 11: L = (1 - lambda) L_PG-geo + lambda L_GC-load."""
    return (1.0 - LAMBDA_GC) * l_pg_geo + LAMBDA_GC * l_gc


def gc_load_soft(soft_count: torch.Tensor, weight_r: torch.Tensor) -> torch.Tensor:
    """Eq. 9 with the soft count, differentiable: population std over the
    rendered pixels of g~_i / w_i (soft_count and weight_r list the render set R)."""
    if soft_count.numel() == 0:
        return torch.zeros((), dtype=DT)
    x = soft_count / weight_r
    return torch.sqrt(torch.mean((x - x.mean()) ** 2))


def flatten_loss(log_scales: torch.Tensor) -> torch.Tensor:
    """L_s (PGSR by citation): mean over the Gaussians of their smallest scale
    min(exp(log_scales)) (the L1 norm of a positive scalar)."""
    if log_scales.shape[0] == 0:
        return torch.zeros((), dtype=DT)
    return torch.exp(log_scales).min(dim=1).values.mean()


def objective_eq11(l_rgb, l_ban, l_s, l_gc):
    """Eq. 10-11 over the locally defined terms:
    (1 - lambda) (L_rgb + lambda_3 L_s + lambda_4 L_ban) + lambda L_GC-load."""
    return (1.0 - LAMBDA_GC) * (l_rgb + LAMBDA_FLAT * l_s + LAMBDA_BAN * l_ban) + LAMBDA_GC * l_gc


# ---------------------------------------------------------------------------
# whole step
# ---------------------------------------------------------------------------

def step(g, view, need_grad=True, retain_intermediate=False, objective="pg", dssim=False):
    """Forward + loss (+ autograd backward) for one view of a synthetic scene `g`
    (pgsag_synth.Gaussians) and `view` (pgsag_synth.View).  Returns a dict with
    dense images, losses and parameter gradients.

    objective "pg": L_rgb + lambda_4 L_ban is differentiated (the GC-load value
    is reported by gc_load, without gradient).  "eq11": objective_eq11 with the
    flattening loss and the soft-count GC-load, all differentiated.  dssim: L_rgb
    takes the masked D-SSIM term (l_rgb_dssim)."""
    cam = Cam.from_synth(view.cam)
    p = params_from_synth(g, requires_grad=need_grad)
    pr, out, depth, valid, pix, sets = render_view(p, cam, view.mask, np.asarray(g.means, np.float32))
    if retain_intermediate and need_grad:
        for k in ("mean2d", "conic", "opacity", "rgb", "normal", "dist"):
            pr[k].retain_grad()
        for k in ("rgb", "normal", "dist"):
            out[k].retain_grad()
    L = losses(out, depth, valid, pix, sets, cam, view.target, dssim=dssim)
    if objective == "eq11":
        pu, pv = pix
        wts = torch.from_numpy(luminance_gradient_weight(view.target)[pv.numpy(), pu.numpy()])
        L["l_s"] = flatten_loss(p["log_scales"])
        L["l_gc_soft"] = gc_load_soft(out["soft_count"], wts)
        L["total"] = objective_eq11(L["l_rgb"], L["l_ban"], L["l_s"], L["l_gc_soft"])
    elif objective != "pg":
        raise ValueError(objective)
    res = dict(proj=pr, out=out, depth=depth, valid=valid, pix=pix, sets=sets, loss=L, cam=cam)
    if need_grad:
        L["total"].backward()
        res["grads"] = {k: (v.grad if v.grad is not None else torch.zeros_like(v)) for k, v in p.items()}
    res["params"] = p
    return res


def to_dense_np(vals: torch.Tensor, pix, H, W, fill=0.0):
    pu, pv = pix
    v = vals.detach().numpy()
    img = np.full((H, W) + v.shape[1:], fill, dtype=np.float64)
    img[pv.numpy(), pu.numpy()] = v
    return img
