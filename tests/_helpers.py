"""Shared helpers for the GPU parity tests: run the CUDA path and the oracle on
the same seeded inputs and compare with the tolerances the method fixes.

Forward tolerance (per pixel and channel): |g - o| / max(|o|, S) <= 1e-4 with
S = sum_i w_i s_i the blended rounding scale of the terms (s = |c| for colour,
|n| = 1 for normal components, |mu_c| for the plane distance d = -n . mu_c): a
floating-point sum of products has error bounded relative to S, not to |sum|
(normal components cancel, d cancels for planes seen edge-on), over pixels the
oracle does not flag as ambiguous (a float32
threshold decision within 3e-5 relative of alpha = 1/255 or T(1-alpha) = 1e-4,
or a normal flip within 1e-6 of edge-on).  Gradient tolerance: relative L2 per
parameter tensor <= 1e-3.

Eq. 4 depth = D / s, s = -N . r: its plain relative error must be <= 1e-4 on
the pixels valid on both sides, and validity must agree exactly.  Its float32
error is bounded by the rounding scales of D (the blended |mu_c|) and of s
(A |r|, N being a blend of unit normals); the error relative to |Depth|
(magD / |D| + A |r| / |s|) is reported (and asserted) beside it, as is each
channel's error under the fixed denominator max(|o|, 1e-3 max_R |o_ch|).

The ambiguous-pixel gate (AMBIG_FRAC_MAX) bounds how many pixels the exclusion
may remove.  The flagged fraction grows with the pairs evaluated per pixel (each
pair that lands within 3e-5 relative of alpha = 1/255 flags its pixel), so it is
a per-workload sanity bound, not a tolerance.
"""
from __future__ import annotations

import numpy as np
import torch

import pgsag_synth as syn
from oracle import pgsag_oracle as O

FWD_TOL = 1e-4
GRAD_TOL = 1e-3
AMBIG_FRAC_MAX = 2e-3


def gpu_run(g, views, tile=(16, 16), g_ranges=None, capacity=None, grad=True, lambda_ban=O.LAMBDA_BAN):
    from paper_2501_01677_b300 import raster
    P = raster.GaussianParams.from_numpy(g, requires_grad=grad)
    plan = raster.Plan([v.cam for v in views], [v.mask for v in views], [v.target for v in views], g.n,
                       g_ranges=g_ranges, tile=tile, capacity=capacity)
    if grad:
        loss = raster.render_loss(plan, P, lambda_ban)
        loss.backward()
    else:
        plan.forward(P)
        plan.loss(lambda_ban)
        plan.tile_stats()
    torch.cuda.synchronize()
    plan.check_status()
    return plan, P


def oracle_run(g, view, grad=True):
    return O.step(g, view, need_grad=grad)


def compare_forward(plan, v, res, tol=FWD_TOL):
    """Returns dict of max errors; asserts the bar."""
    im = {k: t.detach().cpu().numpy() for k, t in plan.images(v).items()}
    pu, pv = [t.numpy() for t in res["pix"]]
    out = res["out"]
    amb = out["ambiguous"].numpy()
    ok = ~amb
    frac = amb.mean() if len(amb) else 0.0
    assert frac <= AMBIG_FRAC_MAX, f"ambiguous fraction {frac}"
    ref = {
        "rgb": out["rgb"].detach().numpy(), "normal": out["normal"].detach().numpy(),
        "dist": out["dist"].detach().numpy(), "alpha": out["alpha"].detach().numpy(),
    }
    errs = {}
    for k, o in ref.items():
        gv = im[k][pv, pu]
        o2 = o.reshape(len(pu), -1)
        g2 = gv.reshape(len(pu), -1)
        S = out["mag"][k].numpy().reshape(len(pu), -1)
        den = np.maximum(np.abs(o2), S)
        e = np.where(den > 0, np.abs(g2 - o2) / np.where(den > 0, den, 1.0), np.abs(g2 - o2) * 1e30)
        e = e[ok]
        errs[k] = float(e.max()) if e.size else 0.0
        # the same error under the fixed per-channel denominator max(|o|, 1e-3 max_R |o_ch|)
        den_s = np.maximum(np.abs(o2), 1e-3 * np.abs(o2).max(0, keepdims=True))
        es = np.where(den_s > 0, np.abs(g2 - o2) / np.where(den_s > 0, den_s, 1.0), 0.0)[ok]
        errs[k + "_fixed_den"] = float(es.max()) if es.size else 0.0
    nc = im["n_contrib"][pv, pu]
    errs["n_contrib_mismatch"] = int((nc[ok] != out["n_contrib"].numpy()[ok]).sum())
    # unbiased depth (Eq. 4) where both sides find the pixel valid
    dg = im["depth"][pv, pu]
    do = res["depth"].detach().numpy()
    vo = res["valid"].numpy()
    vg = dg > 0
    errs["valid_mismatch"] = int((vo[ok] != vg[ok]).sum())
    both = ok & vo & vg
    errs["depth"], errs["depth_plain_rel"] = depth_errors(res, pu, pv, dg, both)
    errs["ambiguous_frac"] = float(frac)
    print("forward errors:", {k: (round(v, 9) if isinstance(v, float) else v) for k, v in errs.items()})
    for k in ("rgb", "normal", "dist", "alpha", "depth", "depth_plain_rel"):
        assert errs[k] <= tol, errs
    assert errs["n_contrib_mismatch"] == 0, errs
    assert errs["valid_mismatch"] == 0, errs
    return errs


def depth_errors(res, pu, pv, dg, sel):
    """Eq. 4 depth error on the selected pixels: (max error relative to the
    depth's rounding scale, max plain relative error)."""
    if not sel.any():
        return 0.0, 0.0
    out = res["out"]
    do = res["depth"].detach().numpy()[sel]
    D = out["dist"].detach().numpy()[sel]
    magD = out["mag"]["dist"].numpy()[sel]
    A = out["alpha"].detach().numpy()[sel]
    r = O.pixel_rays(res["cam"], torch.as_tensor(pu[sel]), torch.as_tensor(pv[sel])).numpy()
    s = -(out["normal"].detach().numpy()[sel] * r).sum(-1)
    kappa = magD / np.abs(D) + A * np.linalg.norm(r, axis=1) / np.abs(s)
    e = np.abs(dg[sel] - do)
    return float((e / (np.abs(do) * kappa)).max()), float((e / np.abs(do)).max())


def rel_l2(a: np.ndarray, b: np.ndarray) -> float:
    n = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / n) if n > 0 else float(np.linalg.norm(a))


def compare_grads(P, res, tol=GRAD_TOL):
    errs = {}
    for name, t in zip(("means", "log_scales", "quats", "opacity_logit", "sh"), P.tensors()):
        gg = t.grad.detach().cpu().numpy().astype(np.float64)
        go = res["grads"][name].numpy()
        errs[name] = rel_l2(gg.reshape(-1), go.reshape(-1))
    for k, e in errs.items():
        assert e <= tol, errs
    return errs



def write_stand_in(plan, v, ch):
    """Write the stand-in rendered channels `ch` (pgsag_synth.rendered_channels)
    into view v's compact rows of the plan's render outputs: out8, depth, the
    count (aux word 2) and, under the Eq. 11 objective, the soft count (aux word
    3).  Returns the rows' linear pixel indices."""
    sl = plan.px_slice(v)
    lin = plan.px_index(v).cpu().numpy()
    rows8 = np.concatenate([ch.rgb.reshape(-1, 3), ch.dist.reshape(-1, 1), ch.normal.reshape(-1, 3),
                            ch.alpha.reshape(-1, 1)], 1)[lin]
    plan.out8[sl] = torch.from_numpy(np.ascontiguousarray(rows8)).cuda()
    plan.depth[sl] = torch.from_numpy(ch.depth.reshape(-1)[lin]).cuda()
    plan.aux[sl, 2] = torch.from_numpy(ch.n_contrib.reshape(-1)[lin]).cuda()
    if plan.objective == "eq11":
        plan.aux[sl, 3] = torch.from_numpy(ch.soft_count.reshape(-1)[lin].view(np.int32)).cuda()
    return lin


def loss_pass_vs_oracle(plan, v, view, ch, lambda_ban=O.LAMBDA_BAN):
    """The loss pass alone (pgsag_loss_ban with its own gather, so dout8 is the
    complete dL/d(rendered channels)) against the oracle's L_rgb + lambda L_ban
    (Sec. 4.2 Eq. 8) and its autograd gradient, on the stand-in rendered
    channels `ch` (pgsag_synth.rendered_channels) written into view v's compact
    rows; the oracle takes the same float32 values in float64, on its own
    render set R.  Eq. 8 reads the depth values as given; their gradient reaches
    the plane distance and the normal through Eq. 4 (Depth = D / (-N . r)),
    differentiated at the given D and N.  Compared element by element over every
    rendered pixel.  Returns {loss relative errors, gradient rel-L2 per channel
    group, render-set and validity checks, alpha-channel gradient maximum}."""
    sl = plan.px_slice(v)
    H, W = plan.shapes[v]
    lin = write_stand_in(plan, v, ch)
    plan.loss(lambda_ban)
    torch.cuda.synchronize()
    plan.check_status()
    d8 = np.zeros((H * W, 8))
    d8[lin] = plan.dout8[sl].double().cpu().numpy()
    lb = plan.loss_buf.cpu().numpy().astype(np.float64)
    # the oracle's own render set and pixel order
    sets = O.mask_sets(view.mask)
    pv_np, pu_np = np.nonzero(sets[2])
    pu, pv = torch.from_numpy(pu_np), torch.from_numpy(pv_np)
    lin_o = pv_np * W + pu_np

    def leaf(a, k):
        return torch.from_numpy(a.reshape(H * W, k)[lin_o].astype(np.float64)).squeeze(-1).requires_grad_(True)

    rgb, dist, normal = leaf(ch.rgb, 3), leaf(ch.dist, 1), leaf(ch.normal, 3)
    out = dict(rgb=rgb, dist=dist, normal=normal, n_contrib=torch.from_numpy(ch.n_contrib.reshape(-1)[lin_o]))
    cam = O.Cam.from_synth(view.cam)
    chain, valid = O.unbiased_depth(out, cam, pu, pv)
    given = torch.from_numpy(ch.depth.reshape(-1)[lin_o].astype(np.float64))
    depth = torch.where(valid, given + (chain - chain.detach()), torch.zeros_like(given))
    lv = O.losses(out, depth, valid, (pu, pv), sets, cam, view.target)
    total = lv["l_rgb"] + lambda_ban * lv["l_ban"]
    total.backward()
    ref = dict(rgb=rgb.grad.numpy(), dist=dist.grad.numpy(), normal=normal.grad.numpy())
    got = dict(rgb=d8[lin_o, 0:3], dist=d8[lin_o, 3], normal=d8[lin_o, 4:7])
    errs = {"grad_" + k: rel_l2(got[k].ravel(), ref[k].ravel()) for k in ref}
    want = (float(lv["l_rgb"].detach()), float(lv["l_ban"].detach()), float(total.detach()))
    for i, (name, w) in enumerate(zip(("l_rgb", "l_ban", "total"), want)):
        errs[name] = abs(lb[3 * v + i] - w) / abs(w) if w != 0 else abs(lb[3 * v + i])
    errs["render_set_equal"] = bool(np.array_equal(np.sort(lin), lin_o))
    errs["valid_is_depth_positive"] = bool(np.array_equal(valid.numpy(), given.numpy() > 0))
    errs["alpha_grad_max"] = float(np.abs(d8[:, 7]).max())
    errs["n_valid"] = int(lv["n_valid"])
    errs["n_mask"] = int(lv["n_mask"])
    return errs


def check_projection(plan, pr):
    """Projection records of every binned pair of the plan's first view against
    the oracle's projection pr (Sec. 3.1, Eq. 2-3): the 2D mean (integer part +
    fraction, compensated) within 2e-6 px, the Cholesky factor of the conic
    within 1e-5 of its scale, opacity, colour, plane distance, the flattened
    normal (off flip-ambiguous Gaussians) and the float32 depth key bit for bit.
    Returns the number of pairs checked."""
    rec = plan.rec.cpu().numpy()
    bi = plan.bininfo.cpu().numpy()
    n = pr["visible"].shape[0]
    rec, bi = rec[:n], bi[:n]
    vis = pr["visible"].numpy() & (bi[:, 3] > 0)
    m2 = pr["mean2d"].detach().numpy()
    q = pr["conic"].detach().numpy()
    # 2D mean = integer part + fraction (compensated evaluation): the integer part
    # is the float32 value s = f x/z + c rounded to an integer, and the fraction
    # also carries the compensation terms (the rounding errors of f x/z and of
    # the sum, each within an ulp of |f x/z| <= |s| + |c|), so |fraction| <= 1/2
    # + a few ulps of (|s| + image size)
    H, W = plan.shapes[0]
    for j, fj in ((0, 14), (1, 15)):
        ip, fp = rec[vis, j], rec[vis, fj]
        assert (ip == np.rint(ip)).all()
        excess = (np.abs(fp) - 0.5) / np.spacing(np.abs(ip) + np.float32(max(W, H)))
        k = int(np.argmax(excess))
        assert excess[k] <= 4.0, (j, float(excess[k]), float(ip[k]), float(fp[k]))
    mean = np.stack([rec[:, 0].astype(np.float64) + rec[:, 14], rec[:, 1].astype(np.float64) + rec[:, 15]], 1)
    err_mean = float(np.abs(mean[vis] - m2[vis]).max())
    assert err_mean < 2e-6, err_mean
    # the record holds the Cholesky factor of the conic: Q = L L^T
    l11 = np.sqrt(q[:, 0])
    l21 = q[:, 1] / l11
    l22 = np.sqrt(q[:, 2] - l21 * l21)
    for j, ref in ((2, l11), (3, l21), (4, l22)):
        scale = np.maximum(np.maximum(np.abs(l11), np.abs(l22))[vis], 1e-12)
        assert (np.abs(rec[vis, j] - ref[vis]) / scale).max() < 1e-5
    np.testing.assert_allclose(rec[vis, 5], pr["opacity"].detach().numpy()[vis], rtol=1e-5)
    np.testing.assert_allclose(rec[vis, 6:9], pr["rgb"].detach().numpy()[vis], rtol=1e-4, atol=1e-5)
    np.testing.assert_allclose(rec[vis, 9], pr["dist"].detach().numpy()[vis], rtol=1e-4, atol=1e-5)
    amb = pr["flip_ambiguous"].numpy()
    ok = vis & ~amb
    np.testing.assert_allclose(rec[ok, 10:13], pr["normal"].detach().numpy()[ok], atol=1e-5)
    # depth key is bit-identical to the oracle's float32 key
    assert (plan.dkey.cpu().numpy()[:n].view(np.float32)[vis] == pr["key"].numpy()[vis]).all()
    print("projection: pairs checked", int(vis.sum()), "max 2D-mean error", err_mean)
    return int(vis.sum())


def check_binning(plan, pr, R, n_sample=None, seed=0):
    """The duplicate lists of the plan's first view (tile size 16x16): ranges
    partition [0, K) in tile order and equal the tile counts; each tile's list
    is in strictly ascending (depth key, pair) order; each pair has `touched`
    duplicates, all inside its tile rectangle; and binning is conservative: every
    (active tile, Gaussian) with a rendered pixel where the oracle finds
    alpha >= 1/255 is a duplicate.  The last check takes every Gaussian
    (n_sample None) or a seeded sample of n_sample Gaussians, whose bounding-box
    pixels are evaluated one by one.  Returns (K, the duplicate set)."""
    K = plan.k_value()
    dup = plan.dup_pairs[:K].cpu().numpy().astype(np.int64)
    rg = plan.ranges.cpu().numpy().astype(np.int64)[:plan.n_active]
    key = plan.dkey.cpu().numpy().view(np.uint32).astype(np.int64)
    bi = plan.bininfo.cpu().numpy().astype(np.int64)
    at = plan.act_tiles.cpu().numpy().astype(np.int64)[:plan.n_active]
    ln = rg[:, 1] - rg[:, 0]
    assert ln.sum() == K and (ln >= 0).all()
    nz = ln > 0
    assert (rg[nz, 0] == np.concatenate([[0], np.cumsum(ln)[:-1]])[nz]).all()
    assert (plan.tile_counts.cpu().numpy()[:plan.n_active] == ln).all()
    tile_of = np.repeat(np.arange(plan.n_active), ln)
    same = tile_of[1:] == tile_of[:-1]
    k0, k1 = key[dup[:-1]], key[dup[1:]]
    assert (((k0 < k1) | ((k0 == k1) & (dup[:-1] < dup[1:])))[same]).all()
    assert (np.bincount(dup, minlength=len(bi)) == bi[:, 3]).all()
    tx, ty = at[tile_of, 1] & 0xFFFF, at[tile_of, 1] >> 16
    x0, y0, x1, y1 = bi[dup, 0] & 0xFFFF, bi[dup, 0] >> 16, bi[dup, 1] & 0xFFFF, bi[dup, 1] >> 16
    assert ((tx >= x0) & (tx <= x1) & (ty >= y0) & (ty <= y1)).all()
    H, W = plan.shapes[0]
    tiles_x = (W + 15) // 16
    ta = plan.tile_act.cpu().numpy()
    have = set(zip(tile_of.tolist(), dup.tolist()))
    assert len(have) == K
    m2, q, o = pr["mean2d"].detach().numpy(), pr["conic"].detach().numpy(), pr["opacity"].detach().numpy()
    if n_sample is None:
        lin, gid = O.candidate_pairs(pr, W, H)
        u, v, gid = (lin % W).numpy(), (lin // W).numpy(), gid.numpy()
    else:
        ok, u0, u1, v0, v1 = O._ellipse_bbox(pr, pr["visible"])
        ok = ok.numpy()
        u0, u1 = np.clip(u0.numpy(), 0, W - 1).astype(np.int64), np.clip(u1.numpy(), 0, W - 1).astype(np.int64)
        v0, v1 = np.clip(v0.numpy(), 0, H - 1).astype(np.int64), np.clip(v1.numpy(), 0, H - 1).astype(np.int64)
        cand = np.nonzero(ok & (u1 >= u0) & (v1 >= v0))[0]
        rng = np.random.default_rng(seed)
        gs = rng.choice(cand, size=min(n_sample, len(cand)), replace=False)
        w_, h_ = u1[gs] - u0[gs] + 1, v1[gs] - v0[gs] + 1
        gs, w_, h_ = gs[w_ * h_ <= 65536], w_[w_ * h_ <= 65536], h_[w_ * h_ <= 65536]
        npx = w_ * h_
        gid = np.repeat(gs, npx)
        off = np.arange(npx.sum()) - np.repeat(np.cumsum(npx) - npx, npx)
        u = u0[gid] + off % np.repeat(w_, npx)
        v = v0[gid] + off // np.repeat(w_, npx)
    keep = R[v, u]
    u, v, gid = u[keep], v[keep], gid[keep]
    dx, dy = u + 0.5 - m2[gid, 0], v + 0.5 - m2[gid, 1]
    a = o[gid] * np.exp(-0.5 * (q[gid, 0] * dx * dx + 2 * q[gid, 1] * dx * dy + q[gid, 2] * dy * dy))
    ent = a >= 1 / 255 * (1 + 1e-4)
    need = set(zip(ta[(v[ent] // 16) * tiles_x + u[ent] // 16].tolist(), gid[ent].tolist()))
    assert need <= have, len(need - have)
    print("binning: duplicates", K, "(tile, Gaussian) pairs the oracle requires", len(need))
    return K, have
