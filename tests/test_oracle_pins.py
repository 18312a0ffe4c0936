"""Further pins of the FP64 oracle: parts whose plausible misreadings the
closed forms of test_oracle.py would not catch.  Each expected value comes from
a library routine (scipy), from hand arithmetic, or from a closed form of the
geometry, never from the oracle itself.

* Colour direction under a posed camera (Sec. 3.1, SH colour by citation to
  3DGS): the viewing direction is normalize(mu - c) with the camera centre
  c = -R^T t, checked against scipy's real SH at that direction.
* Jacobian clamp of the EWA projection (Sec. 3.1 by citation): x/z and y/z are
  clamped to 1.3 x the half field of view (width / 2 / fx, height / 2 / fy)
  inside the Jacobian only, and the clamped coordinate carries no gradient.
* Eq. 8 (Sec. 4.2) with a non-zero value: weight 0.1 on the boundary set E,
  mean over the valid interior mask pixels V (not over M), both normals of
  unit length.
* Near plane (Sec. 3.1 by citation): camera-space z <= 0.2 is culled.
* Eq. 9 weight (Sec. 4.3): w = 1 + |Sobel(Y)| with the unnormalised 3x3 Sobel
  kernels, the Euclidean magnitude, Y = 0.299 R + 0.587 G + 0.114 B and
  replicated borders.
"""
import math

import numpy as np
import pytest
import torch

import pgsag_synth as syn
from oracle import pgsag_oracle as O


# ----------------------------------------------------------------- colour direction

def _scipy_real_sh(dirs: np.ndarray) -> np.ndarray:
    """Real orthonormal SH (no Condon-Shortley phase), index l*l + l + m, from
    scipy's complex harmonics."""
    from scipy.special import sph_harm_y
    theta = np.arccos(np.clip(dirs[:, 2], -1, 1))
    phi = np.arctan2(dirs[:, 1], dirs[:, 0])
    out = np.zeros((len(dirs), 16))
    for l in range(4):
        for m in range(-l, l + 1):
            if m > 0:
                v = math.sqrt(2) * (-1) ** m * np.real(sph_harm_y(l, m, theta, phi))
            elif m == 0:
                v = np.real(sph_harm_y(l, 0, theta, phi))
            else:
                v = math.sqrt(2) * (-1) ** m * np.imag(sph_harm_y(l, -m, theta, phi))
            out[:, l * l + l + m] = v
    return out


def test_colour_direction_under_posed_camera():
    """Look-at camera away from the origin (t != 0), SH degree 3: the colour is
    max(0, sum_k sh_k Y_k(dir) + 0.5) at dir = normalize(mu - campos), where the
    test knows campos directly (it built the camera there)."""
    rng = np.random.default_rng(31)
    campos = np.array([3.0, -2.0, -4.0])
    cam = syn.look_at_camera(campos, [0.0, 0.0, 5.0], 64, 48, 60.0)
    assert np.linalg.norm(cam.t) > 1.0
    g = syn.cube_scene(rng, 40, cube=3.0, zmin=3.5, zmax=6.5)
    g.sh[:] = rng.normal(0.0, 0.4, g.sh.shape).astype(np.float32)
    pr = O.project(O.params_from_synth(g), O.Cam.from_synth(cam))
    mu = g.means.astype(np.float64)
    # the camera centre in float32 storage (R, t are float32 in the camera record)
    c32 = -(cam.R.astype(np.float64).T @ cam.t.astype(np.float64))
    np.testing.assert_allclose(c32, campos, atol=1e-5)
    d = mu - c32
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    Y = _scipy_real_sh(d)
    ref = np.maximum(np.einsum("nk,nkc->nc", Y, g.sh.astype(np.float64)) + 0.5, 0.0)
    np.testing.assert_allclose(pr["rgb"].detach().numpy(), ref, rtol=1e-10, atol=1e-12)
    # the direction matters: the mirrored centre gives other colours
    d2 = mu + c32
    d2 /= np.linalg.norm(d2, axis=1, keepdims=True)
    wrong = np.maximum(np.einsum("nk,nkc->nc", _scipy_real_sh(d2), g.sh.astype(np.float64)) + 0.5, 0.0)
    assert np.abs(wrong - ref).max() > 0.05


# ----------------------------------------------------------------- Jacobian clamp

def _one_gaussian(mean, ls=(-2.0, -2.5, -3.0), quat=(0.9, 0.2, -0.3, 0.1)):
    q = np.asarray(quat, np.float64)
    q /= np.linalg.norm(q)
    return syn.Gaussians(np.asarray([mean], np.float32), np.asarray([ls], np.float32), q[None].astype(np.float32),
                         np.zeros(1, np.float32), np.zeros((1, 16, 3), np.float32))


def _hand_cov2d(g, cam, xt, yt):
    """Sigma' = J W Sigma W^T J^T + 0.3 I with J built by hand at the given
    (clamped) x~, y~ (camera frame) and the true z."""
    from scipy.spatial.transform import Rotation
    q = g.quats[0].astype(np.float64)
    Rq = Rotation.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()
    s = np.exp(g.log_scales[0].astype(np.float64))
    Sig = Rq @ np.diag(s * s) @ Rq.T
    W = cam.R.astype(np.float64)
    z = (W @ g.means[0].astype(np.float64) + cam.t)[2]
    J = np.array([[cam.fx / z, 0.0, -cam.fx * xt / z ** 2], [0.0, cam.fy / z, -cam.fy * yt / z ** 2]])
    return J @ W @ Sig @ W.T @ J.T + 0.3 * np.eye(2), z


def test_jacobian_clamp_at_1p3_half_fov():
    """x/z = 1.2 lies beyond 1.3 (W/2)/fx = 0.832 but inside 1.3 W/fx = 1.664;
    y/z = -0.9 lies beyond -1.3 (H/2)/fy = -0.567 but inside -1.3 H/fy.  The
    Jacobian must use the clamped values 0.832 z and -0.567 z."""
    W, H, fx, fy = 64, 48, 50.0, 55.0
    cam = syn.identity_camera(W, H, fx, fy)
    z = 4.0
    g = _one_gaussian([1.2 * z, -0.9 * z, z])
    pr = O.project(O.params_from_synth(g), O.Cam.from_synth(cam))
    limx, limy = 1.3 * (W / 2) / fx, 1.3 * (H / 2) / fy
    ref, _ = _hand_cov2d(g, cam, limx * z, -limy * z)
    a, b, c = pr["cov2d"][0].numpy()
    np.testing.assert_allclose([a, b, c], [ref[0, 0], ref[0, 1], ref[1, 1]], rtol=1e-12)
    # without the clamp the covariance would differ clearly
    unc, _ = _hand_cov2d(g, cam, 1.2 * z, -0.9 * z)
    assert abs(unc[0, 0] - ref[0, 0]) > 1e-3 * ref[0, 0]
    # the 2-D mean is the true (unclamped) projection
    x, y, zz = g.means[0].astype(np.float64)
    np.testing.assert_allclose(pr["mean2d"][0].numpy(), [fx * x / zz + W / 2, fy * y / zz + H / 2], rtol=1e-12)


def test_jacobian_inside_clamp_is_unclamped():
    W, H, fx, fy = 64, 48, 50.0, 55.0
    cam = syn.identity_camera(W, H, fx, fy)
    z = 4.0
    g = _one_gaussian([0.5 * z, -0.3 * z, z])
    pr = O.project(O.params_from_synth(g), O.Cam.from_synth(cam))
    x, y, _ = g.means[0].astype(np.float64)
    ref, _ = _hand_cov2d(g, cam, x, y)
    a, b, c = pr["cov2d"][0].numpy()
    np.testing.assert_allclose([a, b, c], [ref[0, 0], ref[0, 1], ref[1, 1]], rtol=1e-12)


def test_clamped_coordinate_has_zero_gradient():
    """Where x/z is clamped, the covariance does not depend on x (camera frame =
    world frame for the identity camera); where it is not, it does."""
    W, H, fx, fy = 64, 48, 50.0, 55.0
    c = O.Cam.from_synth(syn.identity_camera(W, H, fx, fy))
    z = 4.0
    for xr, expect_zero in ((1.2, True), (0.5, False)):
        g = _one_gaussian([xr * z, 0.1 * z, z])
        p = O.params_from_synth(g, requires_grad=True)
        pr = O.project(p, c)
        pr["cov2d"].sum().backward()
        gx = float(p["means"].grad[0, 0])
        if expect_zero:
            assert gx == 0.0
        else:
            assert abs(gx) > 1e-6


# ----------------------------------------------------------------- Eq. 8 value

def _plane_depth_field(cam, n_p, d0, H, W):
    """Depth of every pixel on the plane {X : n_p . X = -d0} (ray X = Depth r)."""
    uu, vv = np.meshgrid(np.arange(W), np.arange(H))
    r = np.stack([(uu + 0.5 - cam.cx) / cam.fx, (vv + 0.5 - cam.cy) / cam.fy, np.ones((H, W))], -1)
    return d0 / (-(r @ n_p))


def _eq8_inputs(n_p, n_N, H=14, W=17, seed=3):
    """Hand-made forward outputs for Eq. 8: depth on a camera-facing plane,
    rendered normal N = A n_N with per-pixel A (so only its direction counts),
    one invalid rendered pixel, a mask touching the left image border."""
    rng = np.random.default_rng(seed)
    cam = syn.identity_camera(W, H, 20.0, 24.0)
    mask = np.zeros((H, W), np.uint8)
    mask[3:10, 0:9] = 1       # touches the border column x = 0
    mask[5:12, 9:14] = 1
    M, E, R = O.mask_sets(mask)
    pv, pu = np.nonzero(R)
    dep = _plane_depth_field(cam, n_p, 5.0, H, W)[pv, pu]
    A = rng.uniform(0.2, 1.0, len(pu))
    valid = np.ones(len(pu), bool)
    bad = int(np.nonzero((pu == 12) & (pv == 8))[0][0])   # an interior mask pixel
    valid[bad] = False
    dep[bad] = 0.0
    out = {"rgb": torch.zeros(len(pu), 3, dtype=torch.float64),
           "normal": torch.tensor(A[:, None] * np.asarray(n_N)[None], dtype=torch.float64)}
    pix = (torch.from_numpy(pu.astype(np.int64)), torch.from_numpy(pv.astype(np.int64)))
    return dict(cam=O.Cam.from_synth(cam), out=out, depth=torch.tensor(dep), valid=torch.from_numpy(valid), pix=pix,
                sets=(M, E, R), target=np.zeros((H, W, 3)), bad=(12, 8))


def _expected_V(M, R, bad, H, W):
    """Mask pixels off the image border whose 4 neighbours are rendered and valid,
    themselves valid (hand rule of the reading of Eq. 8)."""
    def ok(x, y):
        return bool(R[y, x]) and (x, y) != bad

    V = np.zeros((H, W), bool)
    for y in range(1, H - 1):
        for x in range(1, W - 1):
            if M[y, x] and ok(x, y) and ok(x, y - 1) and ok(x, y + 1) and ok(x - 1, y) and ok(x + 1, y):
                V[y, x] = True
    return V


@pytest.mark.parametrize("n_p,n_N", [((0.0, 0.0, -1.0), (0.3, -0.4, -0.8)),
                                     ((0.25, -0.35, -0.9), (-0.2, 0.1, -1.0))])
def test_eq8_value_weights_and_normalisation(n_p, n_N):
    n_p = np.asarray(n_p) / np.linalg.norm(n_p)
    nN = np.asarray(n_N) / np.linalg.norm(n_N)
    inp = _eq8_inputs(n_p, n_N)
    M, E, R = inp["sets"]
    H, W = M.shape
    L = O.losses(inp["out"], inp["depth"], inp["valid"], inp["pix"], inp["sets"], inp["cam"], inp["target"])
    V = _expected_V(M, R, inp["bad"], H, W)
    assert L["n_valid"] == V.sum() and V.sum() < M.sum()
    # on a plane the depth-derived normal is the plane's camera-facing unit normal
    c = float(((n_p - nN) ** 2).sum())
    w = np.where(E, 0.1, 1.0)[V]
    assert (w == 0.1).sum() > 5 and (w == 1.0).sum() > 5
    want = c * w.sum() / V.sum()
    assert float(L["l_ban"]) == pytest.approx(want, rel=1e-10)
    assert float(L["total"]) == pytest.approx(float(L["l_rgb"]) + 0.01 * want, rel=1e-12)


def test_eq8_boundary_weight_moves_by_exact_amount():
    """Taking one V pixel out of E raises L_ban by (1 - 0.1) c / |V|."""
    n_p = np.array([0.0, 0.0, -1.0])
    n_N = np.array([0.3, -0.4, -0.8])
    inp = _eq8_inputs(n_p, n_N)
    M, E, R = inp["sets"]
    H, W = M.shape
    V = _expected_V(M, R, inp["bad"], H, W)
    ys, xs = np.nonzero(V & E)
    E2 = E.copy()
    E2[ys[0], xs[0]] = False
    L1 = O.losses(inp["out"], inp["depth"], inp["valid"], inp["pix"], (M, E, R), inp["cam"], inp["target"])
    L2 = O.losses(inp["out"], inp["depth"], inp["valid"], inp["pix"], (M, E2, R), inp["cam"], inp["target"])
    c = float(((n_p - n_N / np.linalg.norm(n_N)) ** 2).sum())
    assert float(L2["l_ban"]) - float(L1["l_ban"]) == pytest.approx(0.9 * c / V.sum(), rel=1e-9)


# ----------------------------------------------------------------- near plane

def test_near_plane_culls_at_camera_z_0p2():
    """Camera-space z of 0.19 and 0.2 are culled, 0.21 is kept; with a camera
    looking along +x, camera z is world x whatever the world z."""
    g = _one_gaussian([0.0, 0.0, 0.19])
    for z, keep in ((0.19, False), (0.2, False), (0.21, True), (5.0, True)):
        g.means[0] = [0.0, 0.0, z]
        pr = O.project(O.params_from_synth(g), O.Cam.from_synth(syn.identity_camera(32, 32, 30.0)))
        assert bool(pr["visible"][0]) == keep, z
    cam = syn.look_at_camera([0.0, 0.0, 0.0], [10.0, 0.0, 0.0], 32, 32, 30.0)
    for pos, keep in (([0.19, 0.0, 0.05], False), ([0.21, 0.02, 3.0], True), ([-1.0, 0.0, 0.0], False)):
        g.means[0] = pos
        pr = O.project(O.params_from_synth(g), O.Cam.from_synth(cam))
        assert bool(pr["visible"][0]) == keep, pos


def test_near_plane_culled_gaussian_never_renders():
    """A large opaque Gaussian at z = 0.19 straight ahead leaves the image empty;
    at z = 0.21 it covers the centre pixel."""
    W = H = 16
    for z, lit in ((0.19, False), (0.21, True)):
        g = _one_gaussian([0.0, 0.0, z], ls=(-3.0, -3.0, -6.0), quat=(1.0, 0.0, 0.0, 0.0))
        g.opacity_logit[:] = 3.0
        v = syn.View(syn.identity_camera(W, H, 20.0), np.ones((H, W), np.uint8), np.zeros((H, W, 3), np.float32))
        res = O.step(g, v, need_grad=False)
        A = O.to_dense_np(res["out"]["alpha"], res["pix"], H, W)
        assert (A[H // 2, W // 2] > 0.5) == lit


# ----------------------------------------------------------------- Eq. 9 weight

def test_sobel_weight_unit_step_edge():
    """Vertical step of white (Y = 1): the unnormalised Sobel x-kernel sums
    (1 + 2 + 1) x 1 = 4 across the step, so w = 5 on the two columns beside it
    and 1 elsewhere."""
    t = np.zeros((9, 12, 3))
    t[:, 6:] = 1.0
    w = O.luminance_gradient_weight(t)
    for x, want in ((3, 1.0), (4, 1.0), (5, 5.0), (6, 5.0), (7, 1.0)):
        assert w[4, x] == pytest.approx(want, abs=1e-12), x


def test_sobel_weight_corner_euclidean_magnitude_and_luma():
    """Corner of a white quadrant (x >= 6, y >= 5): at (x, y) = (5, 4) only the
    diagonal neighbour is lit, gx = gy = 1, so w = 1 + sqrt(2) (the L1 norm would
    give 3).  A red step (Y = 0.299) gives w = 1 + 4 x 0.299."""
    t = np.zeros((10, 12, 3))
    t[5:, 6:] = 1.0
    w = O.luminance_gradient_weight(t)
    assert w[4, 5] == pytest.approx(1.0 + math.sqrt(2.0), abs=1e-12)
    t = np.zeros((6, 10, 3))
    t[:, 5:, 0] = 1.0
    w = O.luminance_gradient_weight(t)
    assert w[3, 4] == pytest.approx(1.0 + 4 * 0.299, abs=1e-12)
    t = np.zeros((6, 10, 3))
    t[:, 5:, 1] = 1.0
    assert O.luminance_gradient_weight(t)[3, 5] == pytest.approx(1.0 + 4 * 0.587, abs=1e-12)


def test_sobel_weight_replicated_border():
    """Only column 0 lit: with replicated borders the column left of the image
    repeats column 0, so gx(0) = 4 (0 - 1) and w = 5; zero padding would give 1."""
    t = np.zeros((6, 8, 3))
    t[:, 0] = 1.0
    w = O.luminance_gradient_weight(t)
    assert w[3, 0] == pytest.approx(5.0, abs=1e-12)
    assert w[3, 1] == pytest.approx(5.0, abs=1e-12)
    assert w[3, 2] == pytest.approx(1.0, abs=1e-12)
