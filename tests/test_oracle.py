"""Pins of the FP64 oracle against facts fixed outside it: library routines
(scipy real SH, scipy rotations, scipy morphology, autograd Jacobians), closed
forms, invariants, brute force on tiny inputs and finite differences."""
import json
import math
import os

import numpy as np
import pytest
import torch

import pgsag_synth as syn
from oracle import pgsag_oracle as O


def _load_json(path):
    with open(path) as f:
        return json.load(f)


GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ----------------------------------------------------------------- constants

def test_paper_constants_golden():
    g = _load_json(os.path.join(GOLDEN, "paper_constants.json"))
    assert O.W_BOUNDARY == g["boundary_weight"]["value"]
    assert O.LAMBDA_GC == g["lambda_gc"]["value"]
    assert O.LAMBDA_BAN == g["lambda_4_ban"]["value"]
    assert O.total_loss_with_gc(2.0, 3.0) == pytest.approx((1 - 0.41) * 2.0 + 0.41 * 3.0, rel=1e-15)


# ----------------------------------------------------------------- SH basis

def test_sh_basis_matches_scipy_real_combination():
    from scipy.special import sph_harm_y
    rng = np.random.default_rng(1)
    d = rng.standard_normal((200, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    theta = np.arccos(np.clip(d[:, 2], -1, 1))
    phi = np.arctan2(d[:, 1], d[:, 0])
    ours = O.sh_basis(torch.tensor(d), 3).numpy()
    for l in range(4):
        for m in range(-l, l + 1):
            if m > 0:
                ref = math.sqrt(2) * (-1) ** m * np.real(sph_harm_y(l, m, theta, phi))
            elif m == 0:
                ref = np.real(sph_harm_y(l, 0, theta, phi))
            else:
                ref = math.sqrt(2) * (-1) ** m * np.imag(sph_harm_y(l, -m, theta, phi))
            np.testing.assert_allclose(ours[:, l * l + l + m], ref, rtol=1e-10, atol=1e-12)


def test_sh_degree0_constant():
    d = torch.tensor([[0.0, 0.0, 1.0], [1.0, 0.0, 0.0]], dtype=torch.float64)
    Y = O.sh_basis(d, 3)
    assert Y[:, 0].numpy() == pytest.approx([0.28209479177387814] * 2, rel=1e-14)


# ----------------------------------------------------------------- rotations

def test_quat_rotmat_matches_scipy():
    from scipy.spatial.transform import Rotation
    rng = np.random.default_rng(2)
    q = rng.standard_normal((100, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    ours = O.quat_to_rotmat(torch.tensor(q)).numpy()
    ref = Rotation.from_quat(np.concatenate([q[:, 1:], q[:, :1]], 1)).as_matrix()
    np.testing.assert_allclose(ours, ref, atol=1e-13)


# ----------------------------------------------------------------- EWA Jacobian

def test_ewa_covariance_equals_projection_jacobian():
    """Sigma' - 0.3 I == Jp W Sigma W^T Jp^T with Jp the autograd Jacobian of the
    pinhole map (x, y, z) -> (fx x/z + cx, fy y/z + cy) (unclamped case)."""
    rng = np.random.default_rng(3)
    g = syn.cube_scene(rng, 16, cube=2.0, zmin=4.0, zmax=6.0)
    cam = syn.look_at_camera([0.3, -0.2, -1.0], [0.0, 0.0, 5.0], 64, 48, 50.0, 55.0)
    c = O.Cam.from_synth(cam)
    p = O.params_from_synth(g)
    pr = O.project(p, c)
    R = c.R
    for i in range(16):
        mc = (R @ p["means"][i] + c.t)
        Jp = torch.autograd.functional.jacobian(
            lambda v: torch.stack([c.fx * v[0] / v[2] + c.cx, c.fy * v[1] / v[2] + c.cy]), mc)
        s = torch.exp(p["log_scales"][i])
        q = p["quats"][i] / torch.linalg.norm(p["quats"][i])
        Rq = O.quat_to_rotmat(q)
        Sig = Rq @ torch.diag(s * s) @ Rq.T
        ref = Jp @ R @ Sig @ R.T @ Jp.T
        a, b, cc = pr["cov2d"][i]
        np.testing.assert_allclose([a - 0.3, b, cc - 0.3], [ref[0, 0], ref[0, 1], ref[1, 1]], rtol=1e-10, atol=1e-14)
        np.testing.assert_allclose(pr["mean2d"][i].numpy(),
                                   [c.fx * mc[0] / mc[2] + c.cx, c.fy * mc[1] / mc[2] + c.cy], rtol=1e-13)
        # conic is the inverse
        cov = torch.tensor([[a, b], [b, cc]])
        Q = torch.tensor([[pr["conic"][i, 0], pr["conic"][i, 1]], [pr["conic"][i, 1], pr["conic"][i, 2]]])
        np.testing.assert_allclose((Q @ cov).numpy(), np.eye(2), atol=1e-10)


# ----------------------------------------------------------------- mask sets

def test_mask_sets_match_scipy_morphology():
    from scipy import ndimage
    rng = np.random.default_rng(4)
    m = (rng.random((37, 29)) < 0.3).astype(np.uint8)
    M, E, R = O.mask_sets(m)
    st = np.ones((3, 3), bool)
    dil = ndimage.binary_dilation(m, st, border_value=0)
    ero = ndimage.binary_erosion(m, st, border_value=1)
    assert (R == dil).all()
    assert (E == (dil & ~ero)).all()
    assert (M == (m != 0)).all()


# ----------------------------------------------------------------- closed forms

def _single_gaussian(z0=5.0, s=0.05, sn=0.005, o=0.7, W=64, H=64, f=100.0, shift=(0.0, 0.0)):
    g = syn.Gaussians(
        means=np.array([[shift[0], shift[1], z0]], np.float32),
        log_scales=np.log(np.array([[s, s, sn]], np.float32)).astype(np.float32),
        quats=np.array([[1.0, 0, 0, 0]], np.float32),
        opacity_logit=np.array([math.log(o / (1 - o))], np.float32),
        sh=np.zeros((1, 16, 3), np.float32))
    g.sh[0, 0] = [0.3, -0.1, 0.6]
    cam = syn.identity_camera(W, H, f)
    mask = np.ones((H, W), np.uint8)
    return g, syn.View(cam, mask, np.zeros((H, W, 3), np.float32))


def test_single_gaussian_closed_form():
    z0, s, f, W, H = 5.0, 0.05, 100.0, 64, 64
    g, v = _single_gaussian(z0=z0, s=s, f=f, W=W, H=H)
    res = O.step(g, v, need_grad=False)
    o = float(torch.sigmoid(torch.tensor(float(g.opacity_logit[0]), dtype=torch.float64)))
    s32 = float(np.exp(np.float64(g.log_scales[0, 0])))
    sig2 = (f * s32 / z0) ** 2 + 0.3
    pu, pv = res["pix"]
    du = pu.numpy() + 0.5 - W / 2
    dv = pv.numpy() + 0.5 - H / 2
    raw = o * np.exp(-0.5 * (du ** 2 + dv ** 2) / sig2)
    alpha = np.where(raw >= 1 / 255, np.minimum(raw, 0.99), 0.0)
    Y00 = 0.28209479177387814
    col = np.maximum(np.array([0.3, -0.1, 0.6]) * Y00 + 0.5, 0)
    out = res["out"]
    np.testing.assert_allclose(out["alpha"].detach().numpy(), alpha, atol=1e-14)
    np.testing.assert_allclose(out["rgb"].detach().numpy(), alpha[:, None] * col[None], atol=1e-14)
    np.testing.assert_allclose(out["normal"].detach().numpy(), alpha[:, None] * np.array([[0, 0, -1.0]]), atol=1e-14)
    np.testing.assert_allclose(out["dist"].detach().numpy(), alpha * z0, atol=1e-12)
    val = res["valid"].numpy()
    assert val.sum() == (alpha > 0).sum()
    np.testing.assert_allclose(res["depth"].detach().numpy()[val], z0, rtol=1e-13)


def test_termination_special_case():
    """Identical centred Gaussians with alpha = 0.95 at the pixel: T goes
    1 -> 0.05 -> 0.0025 -> 1.25e-4; the 4th would leave 6.25e-6 < 1e-4 so exactly
    three are blended and A = 1 - 0.05^3."""
    k = 6
    W = H = 31
    g = syn.Gaussians(
        means=np.tile(np.array([[0.0, 0.0, 5.0]], np.float32), (k, 1)),
        log_scales=np.tile(np.log(np.array([[0.05, 0.05, 0.005]], np.float32)), (k, 1)).astype(np.float32),
        quats=np.tile(np.array([[1.0, 0, 0, 0]], np.float32), (k, 1)),
        opacity_logit=np.full(k, math.log(0.95 / 0.05), np.float32),
        sh=np.zeros((k, 16, 3), np.float32))
    v = syn.View(syn.identity_camera(W, H, 100.0), np.ones((H, W), np.uint8), np.zeros((H, W, 3), np.float32))
    res = O.step(g, v, need_grad=False)
    pu, pv = res["pix"]
    c = int(np.nonzero((pu.numpy() == 15) & (pv.numpy() == 15))[0][0])
    o = float(torch.sigmoid(torch.tensor(float(g.opacity_logit[0]), dtype=torch.float64)))
    assert o == pytest.approx(0.95, abs=1e-7)
    assert int(res["out"]["n_contrib"][c]) == 3
    assert float(res["out"]["alpha"][c]) == pytest.approx(1 - (1 - o) ** 3, rel=1e-14)
    assert not bool(res["out"]["ambiguous"][c])


def _flat_plane_scene(n, normal, d0, seed=5, W=48, H=40, f=60.0, o_mu=1.5):
    """n Gaussians on the plane {x : n . x = -d0} (camera at the origin), their
    smallest axis along the plane normal."""
    from scipy.spatial.transform import Rotation
    rng = np.random.default_rng(seed)
    nrm = np.asarray(normal, np.float64)
    nrm /= np.linalg.norm(nrm)
    t1 = np.cross(nrm, [0.0, 1.0, 0.0])
    t1 /= np.linalg.norm(t1)
    t2 = np.cross(nrm, t1)
    uv = rng.uniform(-2.5, 2.5, (n, 2))
    base = -d0 * nrm
    means = base[None] + uv[:, :1] * t1[None] + uv[:, 1:] * t2[None]
    Mrot = np.stack([t1, t2, nrm], axis=1)
    xyzw = Rotation.from_matrix(np.broadcast_to(Mrot, (n, 3, 3))).as_quat()
    quats = np.concatenate([xyzw[:, 3:], xyzw[:, :3]], 1)
    ls = np.stack([rng.normal(-1.5, 0.2, n), rng.normal(-1.5, 0.2, n), np.full(n, -6.0)], 1)
    g = syn.Gaussians(means.astype(np.float32), ls.astype(np.float32), quats.astype(np.float32),
                      rng.normal(o_mu, 0.5, n).astype(np.float32), rng.normal(0, 0.2, (n, 16, 3)).astype(np.float32))
    cam = syn.identity_camera(W, H, f)
    return g, syn.View(cam, np.ones((H, W), np.uint8), rng.random((H, W, 3), dtype=np.float32))


@pytest.mark.parametrize("normal", [(0.0, 0.0, -1.0), (0.3, -0.2, -1.0)])
def test_coplanar_gaussians_give_exact_plane_depth_and_zero_ban(normal):
    """Gaussians sharing one plane (normal along their thinnest axis): Eq. 4 returns
    the exact ray-plane depth, n_depth = n_rendered, so L_ban = 0."""
    d0 = 6.0
    g, v = _flat_plane_scene(300, normal, d0)
    res = O.step(g, v, need_grad=False)
    nrm = np.asarray(normal) / np.linalg.norm(normal)
    pu, pv = res["pix"]
    r = O.pixel_rays(res["cam"], pu, pv).numpy()
    val = res["valid"].numpy()
    assert val.sum() > 200
    expect = d0 / (-(r @ nrm))
    # float32 storage of the Gaussian means puts them within ~1e-6 of the plane
    np.testing.assert_allclose(res["depth"].detach().numpy()[val], expect[val], rtol=2e-5)
    assert res["loss"]["n_valid"] > 100
    assert float(res["loss"]["l_ban"]) < 1e-8
    A = res["out"]["alpha"].detach().numpy()
    Nn = res["out"]["normal"].detach().numpy()
    np.testing.assert_allclose(Nn[val], A[val, None] * nrm[None], atol=1e-5)


def test_blending_invariants_white_colour():
    """With every colour 1 the rendered colour equals A = 1 - prod(1 - alpha_k)
    (telescoping sum of alpha_k T_k); equal normals give N = A n."""
    g, v = syn.tiny_scene(11, n=64, width=40, height=36)
    g.sh[:] = 0
    g.sh[:, 0, :] = 0.5 / 0.28209479177387814
    g.quats[:] = [1, 0, 0, 0]
    g.log_scales[:, 2] = g.log_scales[:, :2].min(1) - 1.0
    res = O.step(g, v, need_grad=False)
    out = res["out"]
    A = out["alpha"].detach().numpy()
    C = out["rgb"].detach().numpy()
    np.testing.assert_allclose(C, np.repeat(A[:, None], 3, 1), atol=1e-13)
    np.testing.assert_allclose(out["normal"].detach().numpy(), A[:, None] * np.array([[0, 0, -1.0]]), atol=1e-13)
    np.testing.assert_allclose(A, 1 - out["final_T"].detach().numpy(), atol=1e-15)
    assert (A > 0.5).sum() > 50


# ----------------------------------------------------------------- brute force

def _brute_force(pr, pu, pv):
    """Per pixel, loop over all Gaussians sorted by (key, index) in pure Python."""
    n = pr["opacity"].shape[0]
    key = pr["key"].numpy()
    order = sorted([i for i in range(n) if bool(pr["visible"][i])], key=lambda i: (float(key[i]), i))
    m2 = pr["mean2d"].detach().numpy()
    q = pr["conic"].detach().numpy()
    o = pr["opacity"].detach().numpy()
    col = pr["rgb"].detach().numpy()
    nor = pr["normal"].detach().numpy()
    dst = pr["dist"].detach().numpy()
    res = []
    for u, v in zip(pu.tolist(), pv.tolist()):
        T = 1.0
        C = [0.0] * 3
        N = [0.0] * 3
        D = 0.0
        k = 0
        soft = 0.0
        for i in order:
            dx = u + 0.5 - m2[i, 0]
            dy = v + 0.5 - m2[i, 1]
            a = o[i] * math.exp(-0.5 * (q[i, 0] * dx * dx + 2 * q[i, 1] * dx * dy + q[i, 2] * dy * dy))
            if a < 1 / 255:
                continue
            a = min(a, 0.99)
            if T * (1 - a) < 1e-4:
                break
            w = a * T
            for c in range(3):
                C[c] += w * col[i, c]
                N[c] += w * nor[i, c]
            D += w * dst[i]
            T *= (1 - a)
            k += 1
            soft += a
        res.append(C + N + [D, 1 - T, k, soft])
    return np.array(res)


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_vectorised_compositing_equals_brute_force(seed):
    g, v = syn.tiny_scene(seed, n=64, width=32, height=28)
    res = O.step(g, v, need_grad=False)
    pu, pv = res["pix"]
    bf = _brute_force(res["proj"], pu, pv)
    out = res["out"]
    got = np.concatenate([out["rgb"].detach().numpy(), out["normal"].detach().numpy(),
                          out["dist"].detach().numpy()[:, None], out["alpha"].detach().numpy()[:, None],
                          out["n_contrib"].numpy()[:, None], out["soft_count"].detach().numpy()[:, None]], 1)
    np.testing.assert_allclose(got, bf, atol=1e-12, rtol=1e-12)
    assert (bf[:, -2] > 0).sum() > 30


def test_render_set_is_mask_dilation_and_pixels_outside_R_not_rendered():
    g, v = syn.tiny_scene(5, n=40, width=30, height=30)
    res = O.step(g, v, need_grad=False)
    pu, pv = res["pix"]
    M, E, R = res["sets"]
    assert len(pu) == R.sum()
    assert R[pv.numpy(), pu.numpy()].all()


# ----------------------------------------------------------------- normals

def test_flattened_normal_is_min_scale_axis_facing_camera():
    from scipy.spatial.transform import Rotation
    rng = np.random.default_rng(9)
    n = 50
    Rm = Rotation.random(n, random_state=10).as_matrix()
    xyzw = Rotation.from_matrix(Rm).as_quat()
    quats = np.concatenate([xyzw[:, 3:], xyzw[:, :3]], 1).astype(np.float32)
    q64 = quats.astype(np.float64)
    Rm = Rotation.from_quat(np.concatenate([q64[:, 1:], q64[:, :1]], 1)).as_matrix()
    ls = rng.normal(-2, 0.5, (n, 3)).astype(np.float32)
    g = syn.cube_scene(rng, n)
    g.quats[:] = quats
    g.log_scales[:] = ls
    cam = syn.look_at_camera([1.0, 0.5, -2.0], [0, 0, 10.0], 64, 64, 80.0)
    c = O.Cam.from_synth(cam)
    pr = O.project(O.params_from_synth(g), c)
    for i in range(n):
        k = int(np.argmin(ls[i]))
        nw = Rm[i][:, k]
        nc = c.R.numpy() @ nw
        mc = c.R.numpy() @ g.means[i].astype(np.float64) + c.t.numpy()
        if nc @ mc > 0:
            nc = -nc
        np.testing.assert_allclose(pr["normal"][i].numpy(), nc, atol=1e-12)
        assert float(pr["dist"][i]) == pytest.approx(-(nc @ mc), rel=1e-10, abs=1e-12)
        assert float(pr["dist"][i]) >= 0


# ----------------------------------------------------------------- losses

def test_l_rgb_closed_form():
    """Constant target vs a single Gaussian image: L_rgb = mean_M |C - C*| / 3."""
    g, v = _single_gaussian()
    v.target[:] = 0.25
    v.mask[:] = 0
    v.mask[20:44, 16:40] = 1
    res = O.step(g, v, need_grad=False)
    C = O.to_dense_np(res["out"]["rgb"], res["pix"], 64, 64)
    M = v.mask.astype(bool)
    ref = np.abs(C - 0.25).sum(-1)[M].sum() / (3 * M.sum())
    assert float(res["loss"]["l_rgb"]) == pytest.approx(ref, rel=1e-14)


def test_gc_load_population_std():
    g = np.array([[0, 1, 2], [3, 4, 5]])
    w = np.array([[1.0, 2.0, 1.0], [1.0, 2.0, 5.0]])
    R = np.array([[True, True, False], [True, True, True]])
    x = np.array([0, 0.5, 3, 2, 1.0])
    assert O.gc_load(g, w, R) == pytest.approx(float(np.std(x)), rel=1e-15)


def test_luminance_weight_flat_image_is_one_and_edge_positive():
    t = np.zeros((10, 12, 3), np.float32)
    assert np.allclose(O.luminance_gradient_weight(t), 1.0)
    t[:, 6:] = 1.0
    w = O.luminance_gradient_weight(t)
    assert w[5, 5] > 1.0 and w[5, 0] == 1.0


# ----------------------------------------------------------------- gradients

def _loss_at(g, v, name, idx, val):
    g2 = syn.Gaussians(*(np.array(getattr(g, f), copy=True) for f in ("means", "log_scales", "quats", "opacity_logit", "sh")))
    cam = O.Cam.from_synth(v.cam)
    p = O.params_from_synth(g2)
    p[name] = p[name].clone()
    p[name].view(-1)[idx] = val
    pr, out, depth, valid, pix, sets = O.render_view(p, cam, v.mask, np.asarray(g.means, np.float32))
    return float(O.losses(out, depth, valid, pix, sets, cam, v.target)["total"])


@pytest.mark.parametrize("seed", [0, 1])
def test_autograd_gradient_matches_central_differences(seed):
    """Central differences (h = 1e-6, float64) on sampled parameters; samples whose
    one-sided differences disagree (a threshold crossed) are skipped."""
    g, v = syn.tiny_scene(20 + seed, n=40, width=28, height=26, log_scale_mu=-1.2)
    res = O.step(g, v)
    grads = res["grads"]
    rng = np.random.default_rng(seed)
    h = 1e-6
    checked = 0
    for name in ("means", "log_scales", "quats", "opacity_logit", "sh"):
        base = res["params"][name].detach().reshape(-1).numpy()
        gr = grads[name].reshape(-1).numpy()
        cand = np.nonzero(np.abs(gr) > 1e-7)[0]
        if len(cand) == 0:
            continue
        for idx in rng.choice(cand, size=min(6, len(cand)), replace=False):
            x0 = base[idx]
            lp = _loss_at(g, v, name, idx, x0 + h)
            lm = _loss_at(g, v, name, idx, x0 - h)
            l0 = float(res["loss"]["total"].detach())
            fwd, bwd = (lp - l0) / h, (l0 - lm) / h
            if abs(fwd - bwd) > 1e-3 * max(abs(fwd), abs(bwd), 1e-6):
                continue
            fd = (lp - lm) / (2 * h)
            assert fd == pytest.approx(gr[idx], rel=2e-4, abs=1e-8), (name, idx)
            checked += 1
    assert checked >= 15


# ----------------------------------------------------------------- Eq. 10-11 terms

def test_flatten_loss_closed_form():
    ls = torch.tensor([[0.0, 1.0, 2.0], [3.0, -1.0, 5.0], [-2.0, -2.0, 0.5]], dtype=torch.float64)
    want = (1.0 + math.exp(-1.0) + math.exp(-2.0)) / 3.0
    assert float(O.flatten_loss(ls)) == pytest.approx(want, rel=1e-15)
    ls.requires_grad_(True)
    O.flatten_loss(ls).backward()
    g = ls.grad.numpy()
    # only the smallest axis of each Gaussian gets a gradient, exp(min) / N
    np.testing.assert_allclose(g[0], [1.0 / 3, 0, 0], rtol=1e-15)
    np.testing.assert_allclose(g[1], [0, math.exp(-1.0) / 3, 0], rtol=1e-15)
    assert g[2, 2] == 0.0 and g[2, :2].sum() == pytest.approx(math.exp(-2.0) / 3, rel=1e-15)


def test_soft_count_single_gaussian_is_alpha_and_bounds():
    g, v = _single_gaussian()
    out = O.step(g, v, need_grad=False)["out"]
    np.testing.assert_allclose(out["soft_count"].detach().numpy(), out["alpha"].detach().numpy(), atol=1e-15)
    g, v = syn.tiny_scene(3, n=64, width=32, height=28)
    out = O.step(g, v, need_grad=False)["out"]
    soft = out["soft_count"].detach().numpy()
    A = out["alpha"].detach().numpy()
    k = out["n_contrib"].numpy()
    # 1 - prod (1 - a_k) <= sum a_k <= 0.99 * count, equality with one Gaussian
    assert (soft >= A - 1e-12).all() and (soft <= 0.99 * k + 1e-12).all()
    one = k == 1
    assert one.any() and np.allclose(soft[one], A[one], atol=1e-14)
    assert (soft[k >= 2] > A[k >= 2]).all()


def test_gc_load_soft_is_population_std_and_matches_integer_counts():
    rng = np.random.default_rng(4)
    c = rng.integers(0, 20, 500).astype(np.float64)
    w = 1.0 + rng.random(500)
    got = float(O.gc_load_soft(torch.tensor(c), torch.tensor(w)))
    assert got == pytest.approx(float(np.std(c / w)), rel=1e-13)
    R = np.ones(500, bool)
    assert got == pytest.approx(O.gc_load(c, w, R), rel=1e-13)
    assert float(O.gc_load_soft(torch.ones(7, dtype=torch.float64), torch.full((7,), 2.0, dtype=torch.float64))) == 0.0


def test_objective_eq11_weights():
    l = O.objective_eq11(2.0, 3.0, 0.5, 7.0)
    assert l == pytest.approx((1 - 0.41) * (2.0 + 100.0 * 0.5 + 0.01 * 3.0) + 0.41 * 7.0, rel=1e-15)


def _eq11_at(g, v, name, idx, val):
    g2 = syn.Gaussians(*(np.array(getattr(g, f), copy=True) for f in ("means", "log_scales", "quats", "opacity_logit", "sh")))
    cam = O.Cam.from_synth(v.cam)
    p = O.params_from_synth(g2)
    p[name] = p[name].clone()
    p[name].view(-1)[idx] = val
    pr, out, depth, valid, pix, sets = O.render_view(p, cam, v.mask, np.asarray(g.means, np.float32))
    L = O.losses(out, depth, valid, pix, sets, cam, v.target)
    pu, pv = pix
    w = torch.from_numpy(O.luminance_gradient_weight(v.target)[pv.numpy(), pu.numpy()])
    return float(O.objective_eq11(L["l_rgb"], L["l_ban"], O.flatten_loss(p["log_scales"]),
                                  O.gc_load_soft(out["soft_count"], w)))


def test_eq11_autograd_gradient_matches_central_differences():
    """The Eq. 11 objective (with L_s and the soft-count GC-load) against central
    differences of its value, sampled over all parameter tensors."""
    g, v = syn.tiny_scene(31, n=40, width=28, height=26, log_scale_mu=-1.2)
    res = O.step(g, v, objective="eq11")
    rng = np.random.default_rng(7)
    h = 1e-6
    checked = 0
    l0 = float(res["loss"]["total"].detach())
    for name in ("means", "log_scales", "quats", "opacity_logit", "sh"):
        base = res["params"][name].detach().reshape(-1).numpy()
        gr = res["grads"][name].reshape(-1).numpy()
        cand = np.nonzero(np.abs(gr) > 1e-7)[0]
        for idx in rng.choice(cand, size=min(6, len(cand)), replace=False):
            lp = _eq11_at(g, v, name, idx, base[idx] + h)
            lm = _eq11_at(g, v, name, idx, base[idx] - h)
            fwd, bwd = (lp - l0) / h, (l0 - lm) / h
            if abs(fwd - bwd) > 1e-3 * max(abs(fwd), abs(bwd), 1e-6):
                continue
            assert (lp - lm) / (2 * h) == pytest.approx(gr[idx], rel=2e-4, abs=1e-8), (name, idx)
            checked += 1
    assert checked >= 15
    # the soft-count term alone moves opacities: its gradient is not zero
    g_only = O.step(g, v, need_grad=False, objective="eq11")
    assert float(g_only["loss"]["l_gc_soft"]) > 0


# ----------------------------------------------------------------- masked D-SSIM

def test_ssim_window_is_normalised_gaussian():
    G = O.ssim_window().numpy()
    assert G.shape == (11, 11) and G.sum() == pytest.approx(1.0, rel=1e-14)
    np.testing.assert_allclose(G, G.T, atol=1e-18)
    r = np.arange(-5, 6)
    g = np.exp(-r ** 2 / (2 * 1.5 ** 2))
    np.testing.assert_allclose(G, np.outer(g, g) / g.sum() ** 2, rtol=1e-13)


def test_ssim_identity_and_constant_images_closed_form():
    rng = np.random.default_rng(0)
    H, W = 20, 24
    R = np.ones((H, W), bool)
    x = torch.tensor(rng.random((H, W, 3)))
    np.testing.assert_allclose(O.masked_ssim_map(x, x, R).numpy(), 1.0, atol=1e-12)
    a, b = 0.3, 0.7
    S = O.masked_ssim_map(torch.full((H, W, 3), a, dtype=torch.float64), torch.full((H, W, 3), b, dtype=torch.float64),
                          R).numpy()
    np.testing.assert_allclose(S, (2 * a * b + O.SSIM_C1) / (a * a + b * b + O.SSIM_C1), rtol=1e-12)


def test_masked_ssim_matches_direct_windowed_moments():
    """Weighted moments written out per pixel over the 11 x 11 neighbourhood,
    restricted to R and the image, the Gaussian weights renormalised."""
    rng = np.random.default_rng(1)
    H, W = 17, 19
    R = rng.random((H, W)) < 0.7
    x = rng.random((H, W, 3))
    y = rng.random((H, W, 3))
    S = O.masked_ssim_map(torch.tensor(x), torch.tensor(y), R).numpy()
    for (i, j) in [(0, 0), (8, 9), (16, 18), (3, 14), (12, 2)]:
        for c in range(3):
            w = []
            xs, ys = [], []
            for di in range(-5, 6):
                for dj in range(-5, 6):
                    ii, jj = i + di, j + dj
                    if 0 <= ii < H and 0 <= jj < W and R[ii, jj]:
                        w.append(math.exp(-(di * di + dj * dj) / (2 * 1.5 ** 2)))
                        xs.append(x[ii, jj, c])
                        ys.append(y[ii, jj, c])
            w = np.array(w) / np.sum(w)
            xs, ys = np.array(xs), np.array(ys)
            mx, my = w @ xs, w @ ys
            vx, vy, cxy = w @ (xs - mx) ** 2, w @ (ys - my) ** 2, w @ ((xs - mx) * (ys - my))
            want = ((2 * mx * my + O.SSIM_C1) * (2 * cxy + O.SSIM_C2)) / \
                   ((mx * mx + my * my + O.SSIM_C1) * (vx + vy + O.SSIM_C2))
            assert S[i, j, c] == pytest.approx(want, rel=1e-10), (i, j, c)


def test_l_rgb_dssim_weights_and_gradient_central_differences():
    rng = np.random.default_rng(2)
    H, W = 14, 16
    M = rng.random((H, W)) < 0.5
    from scipy import ndimage
    R = ndimage.binary_dilation(M, structure=np.ones((3, 3), bool))
    C = torch.tensor(rng.random((H, W, 3)), requires_grad=True)
    T = torch.tensor(rng.random((H, W, 3)))
    l, s = O.l_rgb_dssim(C, T, M, R)
    l1 = float((C.detach() - T).abs().sum(-1)[torch.from_numpy(M)].sum() / (3 * M.sum()))
    assert float(l.detach()) == pytest.approx(0.8 * l1 + 0.2 * (1 - float(s.detach())), rel=1e-14)
    l.backward()
    g = C.grad.numpy()
    # pixels outside R do not enter the loss
    assert (g[~R] == 0).all()
    h = 1e-6
    for (i, j, c) in [(3, 4, 0), (7, 7, 2), (10, 12, 1), (0, 5, 1)]:
        if not R[i, j]:
            continue
        Cp = C.detach().clone()
        Cm = C.detach().clone()
        Cp[i, j, c] += h
        Cm[i, j, c] -= h
        fd = (float(O.l_rgb_dssim(Cp, T, M, R)[0]) - float(O.l_rgb_dssim(Cm, T, M, R)[0])) / (2 * h)
        assert fd == pytest.approx(g[i, j, c], rel=1e-5, abs=1e-9)
