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
