"""CUDA path vs the FP64 oracle, through the C-ABI (ctypes binding)."""
import math

import numpy as np
import pytest
import torch

import pgsag_synth as syn
from oracle import pgsag_oracle as O
from tests._helpers import (FWD_TOL, GRAD_TOL, check_binning, check_projection, compare_forward, compare_grads,
                            gpu_run,
                            loss_pass_vs_oracle, oracle_run, rel_l2)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def config0():
    g, views = syn.config0()
    res = oracle_run(g, views[0])
    return g, views, res


def test_config0_forward_parity(config0):
    g, views, res = config0
    plan, P = gpu_run(g, views)
    errs = compare_forward(plan, 0, res)
    print("config0 forward errors", errs)


def test_config0_loss_and_gradients(config0):
    g, views, res = config0
    plan, P = gpu_run(g, views)
    lv = res["loss"]
    # per-view loss values from the loss kernel
    plan2, P2 = gpu_run(g, views, grad=False)
    lb = plan2.loss_buf.cpu().numpy()
    assert lb[0] == pytest.approx(float(lv["l_rgb"].detach()), rel=1e-4)
    assert lb[1] == pytest.approx(float(lv["l_ban"].detach()), rel=1e-3)
    assert lb[3] == pytest.approx(float(lv["total"].detach()), rel=1e-4)
    errs = compare_grads(P, res)
    print("config0 gradient rel-L2", errs)


def _assert_loss_pass(errs):
    """Same rendered channels on both sides, so only float32 arithmetic separates
    them: the L1 sum to 1e-5 (per-pixel rounding plus the float32 chunk sums),
    the Eq. 8 mean to 1e-4 (central differences of back-projected points cancel),
    the gradient groups to the gradient tolerance; validity (Eq. 4) and the zero
    alpha-channel gradient exactly."""
    print("loss pass vs oracle:", errs)
    assert errs["render_set_equal"] and errs["valid_is_depth_positive"], errs
    assert errs["n_valid"] > 0
    assert errs["alpha_grad_max"] == 0.0, errs
    assert errs["l_rgb"] <= 1e-5, errs
    assert errs["l_ban"] <= 1e-4 and errs["total"] <= 1e-4, errs
    for k in ("grad_rgb", "grad_dist", "grad_normal"):
        assert errs[k] <= GRAD_TOL, errs


def test_config0_loss_pass_matches_oracle_on_same_channels(config0):
    """pgsag_loss_ban alone, on stand-in rendered channels (two tilted planes
    with a step and an unrendered disc): the three loss values and the complete
    upstream gradient (L1 sign term, Eq. 8 own-normal term, Eq. 8 neighbour
    gather mapped through Eq. 4) against the oracle's autograd."""
    g, views, _ = config0
    plan, P = gpu_run(g, views, grad=False)
    _assert_loss_pass(loss_pass_vs_oracle(plan, 0, views[0], syn.rendered_channels(views[0].cam, None, seed=0)))


def test_loss_pass_second_view_of_a_ragged_two_view_plan():
    """Odd image sizes (ragged chunks and tiles) and the second view's rows of a
    two-view plan (non-zero compact and chunk bases)."""
    g, v = syn.tiny_scene(4, n=300, width=83, height=61, coverage=0.6)
    v2 = syn.View(v.cam, np.ascontiguousarray(v.mask[::-1, :]), np.ascontiguousarray(v.target[::-1, :]))
    plan, P = gpu_run(g, [v, v2], grad=False)
    for i, view in enumerate((v, v2)):
        _assert_loss_pass(loss_pass_vs_oracle(plan, i, view, syn.rendered_channels(view.cam, None, seed=3 + i)))


def test_config0_preprocess_parity(config0):
    g, views, res = config0
    plan, P = gpu_run(g, views, grad=False)
    n = check_projection(plan, res["proj"])
    assert n > 1000


def test_config0_rect_is_conservative(config0):
    """Every rendered pixel where the oracle finds alpha >= 1/255 lies in the GPU
    tile rect of that Gaussian."""
    g, views, res = config0
    plan, P = gpu_run(g, views, grad=False)
    pr = res["proj"]
    M, E, R = res["sets"]
    bi = plan.bininfo.cpu().numpy().astype(np.int64)
    lin, gid = O.candidate_pairs(pr, 256, 256)
    u = (lin % 256).numpy()
    v = (lin // 256).numpy()
    gid = gid.numpy()
    inR = R[v, u]
    u, v, gid = u[inR], v[inR], gid[inR]
    m2 = pr["mean2d"].detach().numpy()
    q = pr["conic"].detach().numpy()
    o = pr["opacity"].detach().numpy()
    dx = u + 0.5 - m2[gid, 0]
    dy = v + 0.5 - m2[gid, 1]
    a = o[gid] * np.exp(-0.5 * (q[gid, 0] * dx * dx + 2 * q[gid, 1] * dx * dy + q[gid, 2] * dy * dy))
    ent = a >= 1 / 255
    tx, ty = u[ent] // 16, v[ent] // 16
    gg = gid[ent]
    x0, y0 = bi[gg, 0] & 0xFFFF, bi[gg, 0] >> 16
    x1, y1 = bi[gg, 1] & 0xFFFF, bi[gg, 1] >> 16
    assert (bi[gg, 3] > 0).all() or not ent.any()
    inside = (tx >= x0) & (tx <= x1) & (ty >= y0) & (ty <= y1)
    assert inside.all()


def test_config0_bin_sort_and_binning(config0):
    """The duplicate lists: each tile's list is in strictly ascending (depth key,
    pair) order (the unique part, checked exactly); the emitted set is valid --
    it matches each pair's `touched`, lies inside the pair's tile rectangle on
    active tiles, and contains every (tile, Gaussian) with a rendered pixel where
    the oracle finds alpha >= 1/255 (binning is conservative)."""
    g, views, res = config0
    plan, P = gpu_run(g, views, grad=False)
    M, E, R = res["sets"]
    K, have = check_binning(plan, res["proj"], R)
    bi = plan.bininfo.cpu().numpy().astype(np.int64)
    ta = plan.tile_act.cpu().numpy()
    # the exact test prunes the axis-aligned rule
    aabb = 0
    for p in np.nonzero(bi[:, 3] > 0)[0]:
        x0, y0, x1, y1 = bi[p, 0] & 0xFFFF, bi[p, 0] >> 16, bi[p, 1] & 0xFFFF, bi[p, 1] >> 16
        blk = ta.reshape(16, 16)[y0:y1 + 1, x0:x1 + 1]
        aabb += int((blk >= 0).sum())
    print("duplicates", K, "axis-aligned rule", aabb)
    assert K <= aabb


def test_config0_gc_load(config0):
    g, views, res = config0
    plan, P = gpu_run(g, views, grad=False)
    M, E, R = res["sets"]
    nc = O.to_dense_np(res["out"]["n_contrib"].double(), res["pix"], 256, 256).astype(np.int64)
    w = O.luminance_gradient_weight(views[0].target)
    ref = O.gc_load(nc, w, R)
    assert float(plan.gc_load[0]) == pytest.approx(ref, rel=1e-4)
    lin = plan.px_index(0).cpu().numpy()
    np.testing.assert_allclose(plan.gc_weight[plan.px_slice(0)].cpu().numpy(), w.reshape(-1)[lin], rtol=1e-5, atol=1e-6)
    tc = plan.target.view(-1, 3)[plan.px_slice(0)].cpu().numpy()
    assert np.array_equal(tc, views[0].target.reshape(-1, 3)[lin])
    fl = plan.flags_image(0).cpu().numpy()
    assert ((fl & 1) != 0).sum() == M.sum() and (((fl & 2) != 0) == E).all() and (((fl & 4) != 0) == R).all()


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_tiny_scenes_forward_and_grad(seed):
    g, v = syn.tiny_scene(seed, n=64, width=37, height=29)
    res = oracle_run(g, v)
    plan, P = gpu_run(g, [v], tile=(8, 8))
    compare_forward(plan, 0, res)
    compare_grads(P, res)


def test_results_independent_of_tile_size(config0):
    g, views, res = config0
    outs = []
    for tile in ((8, 8), (16, 16), (16, 32), (32, 32), (32, 8)):
        plan, P = gpu_run(g, views, tile=tile, grad=False)
        im = plan.images(0)
        outs.append([im[k].cpu().numpy() for k in ("rgb", "dist", "normal", "alpha", "n_contrib", "depth")])
    for o in outs[1:]:
        for a, b in zip(o, outs[0]):
            assert np.array_equal(a, b)


@pytest.mark.parametrize("tile", [(8, 8), (16, 32), (32, 32), (32, 8)])
def test_gradients_independent_of_tile_size(config0, tile):
    """The adjoint at every supported tile shape -- tiles of more than 256
    rendered pixels take several pixel rounds per CTA, each reusing the staged
    list -- gives the oracle's gradients and, up to the order of the float
    atomics, the 16x16 tiles' gradients."""
    g, views, res = config0
    _, P16 = gpu_run(g, views, tile=(16, 16))
    _, P = gpu_run(g, views, tile=tile)
    compare_grads(P, res)
    for a, b in zip(P.tensors(), P16.tensors()):
        ga = a.grad.detach().cpu().numpy().astype(np.float64).ravel()
        gb = b.grad.detach().cpu().numpy().astype(np.float64).ravel()
        assert rel_l2(ga, gb) < 1e-5


def test_repeated_adjoint_after_one_forward(config0):
    """The projection clears the binned pairs' gradient rows, so the first render
    adjoint after it skips the full clear; a second adjoint on the same forward
    must clear them itself and give the same per-pair gradients (up to the order
    of the float atomics), not twice them."""
    from paper_2501_01677_b300 import raster
    g, views, _ = config0
    P = raster.GaussianParams.from_numpy(g)
    plan = raster.Plan([v.cam for v in views], [v.mask for v in views], [v.target for v in views], g.n)
    plan.forward(P)
    plan.loss(O.LAMBDA_BAN, fused=True, P=P)
    plan.render_bwd(plan.dout8, ban=True)
    torch.cuda.synchronize()
    binned = plan.bininfo[:, 3].cpu().numpy() > 0
    first = plan.grad2d.cpu().numpy()[binned]
    plan.render_bwd(plan.dout8, ban=True)
    torch.cuda.synchronize()
    plan.check_status()
    second = plan.grad2d.cpu().numpy()[binned]
    assert np.abs(first).max() > 0
    assert rel_l2(second.ravel().astype(np.float64), first.ravel().astype(np.float64)) < 1e-5


@pytest.mark.parametrize("objective", ["pg", "eq11"])
def test_gradient_rows_cleared_by_the_render_adjoint(objective):
    """The step's render adjoint clears the raw-parameter gradient buffers on the
    side (pgsag_clear: float4 bodies split over its CTAs, 1-3 trailing floats),
    and the projection adjoint over those zeros (accumulate = 2) writes only the
    Gaussians with a binned pair and the flattening term.  Buffers filled with
    NaN before the step end up bitwise equal to the mode that writes every row
    (accumulate = 0, same grad2d): no row is left uncleared or written twice."""
    from paper_2501_01677_b300 import raster
    n = 1001  # means / log-scales 3003 floats, opacity 1001: trailing floats
    g, v = syn.tiny_scene(21, n=n, width=83, height=61, coverage=0.4)
    g.means[:150, 2] = -3.0  # behind the camera: never binned
    P = raster.GaussianParams.from_numpy(g)
    plan = raster.Plan([v.cam], [v.mask], [v.target], g.n)
    plan.set_objective(objective)
    plan.forward(P)
    nan = [torch.full_like(t, float("nan")) for t in P.tensors()]
    assert plan.clearable(nan) is not None
    plan.step(P, nan)
    ref = [torch.full_like(t, float("nan")) for t in P.tensors()]
    plan.preprocess_bwd(P, ref)
    torch.cuda.synchronize()
    plan.check_status()
    binned = plan.bininfo[:, 3].cpu().numpy() > 0
    assert binned.sum() > 0 and not binned[:150].any()
    for a, b in zip(nan, ref):
        a, b = a.cpu().numpy(), b.cpu().numpy()
        assert np.isfinite(a).all()
        assert np.array_equal(a, b)
        rows = a.reshape(n, -1)
        assert np.abs(rows[binned]).max() > 0
    if objective == "pg":
        assert all(float(np.abs(t.cpu().numpy().reshape(n, -1)[~binned]).max()) == 0.0 for t in nan)
    else:  # the flattening term reaches every Gaussian's smallest log-scale
        assert np.abs(nan[1].cpu().numpy()[~binned]).max() > 0


def test_maximum_view_count():
    """PGSAG_MAX_VIEWS (256) views in one plan, each with its own principal point
    and mask: the view table fills 39 KB of the projection's shared memory and,
    with the SH slab, takes the projection adjoint past the 48 KB default.  Each
    sampled view renders bitwise as in a plan of its own, and the gradient of
    the 256-view loss equals the sum over four 64-view plans (float atomics
    order aside)."""
    n_max = 256
    g, v = syn.tiny_scene(8, n=300, width=24, height=20, coverage=0.7)
    c = v.cam
    views = []
    for k in range(n_max):
        cam = syn.Camera(c.R, c.t, c.fx, c.fy, c.cx + 0.7 * (k % 9 - 4), c.cy + 0.6 * (k // 9 % 7 - 3),
                         c.width, c.height, c.znear)
        views.append(syn.View(cam, np.ascontiguousarray(np.roll(v.mask, k, axis=1)),
                              np.ascontiguousarray(np.roll(v.target, k, axis=1))))
    plan, P = gpu_run(g, views)
    assert plan.n_views == n_max
    for k in (0, 131, n_max - 1):
        one, _ = gpu_run(g, [views[k]], grad=False)
        a, b = plan.images(k), one.images(0)
        for ch in ("rgb", "dist", "normal", "alpha", "n_contrib", "depth"):
            assert np.array_equal(a[ch].cpu().numpy(), b[ch].cpu().numpy()), (k, ch)
    parts = [gpu_run(g, views[i:i + 64])[1] for i in range(0, n_max, 64)]
    for name, t, *ts in zip(("means", "log_scales", "quats", "opacity_logit", "sh"), P.tensors(),
                            *[q.tensors() for q in parts]):
        ref = sum(x.grad.detach().cpu().numpy().astype(np.float64) for x in ts).ravel()
        got = t.grad.detach().cpu().numpy().astype(np.float64).ravel()
        assert np.abs(ref).max() > 0
        assert rel_l2(got, ref) < 1e-5, name


def test_batched_views_equal_plain_views():
    """Several views (different resolutions, Gaussian subsets) in one plan give the
    same per-view results as one plan per view; the sort is bit-identical."""
    g, ranges, views, owner = syn.config3(sizes=(3000, 5000, 2000), views_per_region=2, scale=0.2)
    g_ranges = [ranges[o] for o in owner]
    planb, Pb = gpu_run(g, views, g_ranges=g_ranges)
    for v in range(len(views)):
        plan1, P1 = gpu_run(g, [views[v]], g_ranges=[g_ranges[v]])
        sl, s1 = planb.px_slice(v), plan1.px_slice(0)
        assert np.array_equal(planb.px_list[sl].cpu().numpy(), plan1.px_list[s1].cpu().numpy())
        assert np.array_equal(planb.out8[sl].cpu().numpy(), plan1.out8[s1].cpu().numpy())
        assert np.array_equal(planb.aux[sl, 2].cpu().numpy(), plan1.aux[s1, 2].cpu().numpy())
    # gradients of the batch = sum of per-view gradients
    acc = [torch.zeros_like(t) for t in Pb.tensors()]
    for v in range(len(views)):
        plan1, P1 = gpu_run(g, [views[v]], g_ranges=[g_ranges[v]])
        for a, t in zip(acc, P1.tensors()):
            a += t.grad
    for a, t in zip(acc, Pb.tensors()):
        assert rel_l2(t.grad.cpu().numpy().ravel(), a.cpu().numpy().ravel()) < 1e-5


def test_empty_mask_and_no_gaussians():
    g, v = syn.tiny_scene(3, n=20, width=24, height=24)
    v.mask[:] = 0
    plan, P = gpu_run(g, [v])
    assert plan.n_render == 0 and plan.n_chunks == 0
    for t in P.tensors():
        assert float(t.grad.abs().max()) == 0.0
    g0, v0 = syn.tiny_scene(4, n=10)
    g0 = g0.subset(np.arange(0))
    plan, P = gpu_run(g0, [v0], grad=False)
    assert plan.k_value() == 0
    assert float(plan.out8.abs().max()) == 0.0


def test_culled_and_nonfinite_gaussians():
    g, v = syn.tiny_scene(6, n=40, width=32, height=32)
    g.means[:10, 2] = -3.0                 # behind the camera
    g.means[10, 0] = np.nan                # non-finite
    g.opacity_logit[11] = np.inf
    g.opacity_logit[12] = -20.0            # o < 1/255
    plan, P = gpu_run(g, [v], grad=False)
    bi = plan.bininfo.cpu().numpy()
    assert (bi[:13, 3] == 0).all()
    assert (plan.dkey.cpu().numpy().view(np.uint32)[:13] == 0xFFFFFFFF).all()
    assert np.isfinite(plan.out8.cpu().numpy()).all()


def test_capacity_overflow_reports_status_then_grows():
    g, views = syn.config0()
    from paper_2501_01677_b300 import raster
    P = raster.GaussianParams.from_numpy(g)
    plan = raster.Plan([views[0].cam], [views[0].mask], [views[0].target], g.n, capacity=1000)
    plan.preprocess(P)
    plan.bin()
    plan.render_fwd()
    torch.cuda.synchronize()
    assert plan.status_value() & 1
    assert plan.k_value() > 1000
    plan._auto_capacity = True
    plan.forward(P)
    torch.cuda.synchronize()
    assert plan.status_value() == 0 and plan.capacity >= plan.k_value()


def test_render_fn_upstream_gradient_matches_oracle():
    """Differentiable renderer with an arbitrary upstream gradient on the outputs
    (RGB, D, N, A and depth): gradient of <G, outputs> vs oracle autograd."""
    g, v = syn.tiny_scene(9, n=50, width=30, height=26)
    from paper_2501_01677_b300 import raster
    rng = np.random.default_rng(0)
    H, W = 26, 30
    G8 = rng.standard_normal((H * W, 8)).astype(np.float32)
    Gd = rng.standard_normal(H * W).astype(np.float32)
    P = raster.GaussianParams.from_numpy(g, requires_grad=True)
    plan = raster.Plan([v.cam], [v.mask], [v.target], g.n, tile=(16, 16))
    out8, depth = raster.render(plan, P)
    q = plan.px_index(0)  # compact rows -> linear pixel index
    (out8 * torch.from_numpy(G8).cuda()[q]).sum().add_((depth * torch.from_numpy(Gd).cuda()[q]).sum()).backward()
    # oracle
    cam = O.Cam.from_synth(v.cam)
    p = O.params_from_synth(g, requires_grad=True)
    pr, out, dep, valid, pix, sets = O.render_view(p, cam, v.mask, g.means)
    pu, pv = pix
    lin = (pv * W + pu).numpy()
    G8t = torch.from_numpy(G8.astype(np.float64))[lin]
    Gdt = torch.from_numpy(Gd.astype(np.float64))[lin]
    obj = (out["rgb"] * G8t[:, 0:3]).sum() + (out["dist"] * G8t[:, 3]).sum() + (out["normal"] * G8t[:, 4:7]).sum() \
        + (out["alpha"] * G8t[:, 7]).sum() + (dep * Gdt).sum()
    obj.backward()
    for name, t in zip(("means", "log_scales", "quats", "opacity_logit", "sh"), P.tensors()):
        e = rel_l2(t.grad.cpu().numpy().astype(np.float64).ravel(), p[name].grad.numpy().ravel())
        assert e < GRAD_TOL, (name, e)


def test_persistent_lpt_schedule_and_graph_replay_match_plain():
    """Persistent launches over a longest-first tile queue, and a CUDA-graph replay
    of the whole step, give the plain launch's outputs (forward bitwise; gradients
    up to float atomics order)."""
    from paper_2501_01677_b300 import raster
    g, ranges, views, owner = syn.config3(sizes=(3000, 5000, 2000), views_per_region=2, scale=0.2)
    g_ranges = [ranges[o] for o in owner]
    P = raster.GaussianParams.from_numpy(g)

    def run(mode):
        plan = raster.Plan([v.cam for v in views], [v.mask for v in views], [v.target for v in views], g.n,
                           g_ranges=g_ranges)
        plan.forward(P)  # sizes the capacity
        if mode != "plain":
            plan.use_persistent_schedule(ctas_per_sm=2, lpt=True)
        grads = raster.new_param_grads(P)
        if mode == "graph":
            graph = plan.capture(P, grads)
            graph.replay()
            graph.replay()
        else:
            plan.step(P, grads)
        torch.cuda.synchronize()
        plan.check_status()
        return plan, [t.cpu().numpy() for t in grads]

    plain, gp = run("plain")
    pers, gq = run("persistent")
    graph, gg = run("graph")
    order = pers.sched_order[:pers.n_active].cpu().numpy()
    assert sorted(order.tolist()) == list(range(pers.n_active))
    for other, go in ((pers, gq), (graph, gg)):
        assert np.array_equal(other.out8.cpu().numpy(), plain.out8.cpu().numpy())
        assert np.array_equal(other.aux.cpu().numpy(), plain.aux.cpu().numpy())
        assert np.allclose(other.loss_buf.cpu().numpy(), plain.loss_buf.cpu().numpy(), rtol=1e-6)
        for a, b in zip(go, gp):
            assert rel_l2(a.ravel().astype(np.float64), b.ravel().astype(np.float64)) < 1e-5


def test_city_block_small_scale_compact_memory():
    """All 72 views of the city-block workload (at 1/2000 of its Gaussians) in one
    plan: per-pixel memory is 5 B per image pixel plus a fixed record per rendered
    pixel, and every view's outputs land on its own rendered set."""
    from paper_2501_01677_b300 import raster
    g, ranges, cams, owner, masks, targets = syn.config4(scale=0.0005)
    plan = raster.Plan(cams, masks, targets, g.n, g_ranges=[ranges[o] for o in owner])
    P = raster.GaussianParams.from_numpy(g)
    plan.forward(P)
    plan.loss()
    torch.cuda.synchronize()
    plan.check_status()
    b = plan.device_bytes()
    assert b["dense_pixel"] == 5 * plan.n_pix
    assert b["compact_pixel"] == 145 * plan.n_render + 48 * plan.n_chunks
    for v in (0, 35, 71):
        R = (plan.flags_image(v).cpu().numpy() & 4) != 0
        a = plan.images(v)["alpha"].cpu().numpy()
        assert (a[~R] == 0).all() and a[R].max() > 0


def test_autotuner_picks_a_shape_and_caches_it(tmp_path, monkeypatch):
    """The autotuner times each (tile, queue depth) candidate on the workload,
    stores the fastest under the workload key, and a second call is served from
    the cache without timing anything."""
    from paper_2501_01677_b300 import autotune as AT, raster
    g, ranges, views, owner = syn.config3(sizes=(3000, 5000, 2000), views_per_region=2, scale=0.2)
    g_ranges = [ranges[o] for o in owner]
    P = raster.GaussianParams.from_numpy(g)
    cams, masks, targets = [v.cam for v in views], [v.mask for v in views], [v.target for v in views]
    path = str(tmp_path / "autotune.json")
    shape, table = AT.autotune(cams, masks, targets, P, g_ranges, tiles=((8, 8), (16, 16)),
                               queue_depths=(None, 2), replays=2, cache_path=path)
    assert len(table) == 2 * 3 and all(r["ms"] > 0 for r in table)
    assert shape.tile in ((8, 8), (16, 16))
    assert min(r["ms"] for r in table) == next(r["ms"] for r in table if (r["tile_w"], r["tile_h"], r["ctas_per_sm"],
                                                                            r["lpt"]) == (shape.tile_w, shape.tile_h,
                                                                                          shape.ctas_per_sm, shape.lpt))

    def no_timing(*a, **k):
        raise AssertionError("cache miss")
    monkeypatch.setattr(AT, "time_step", no_timing)
    shape2, table2 = AT.autotune(cams, masks, targets, P, g_ranges, tiles=((8, 8), (16, 16)),
                                 queue_depths=(None, 2), replays=2, cache_path=path)
    assert shape2 == shape and table2 == table
    plan = AT.plan_for(cams, masks, targets, P, shape, g_ranges)
    grads = raster.new_param_grads(P)
    plan.step(P, grads)
    torch.cuda.synchronize()
    plan.check_status()


@pytest.mark.parametrize("n,seed,kmin", [(400, 20, 257), (1500, 11, 513), (5000, 16, 4097), (9000, 14, 8193)])
def test_long_tile_lists_sorted_through_merges(n, seed, kmin):
    """Tile lists longer than a warp sorts on its own (256 entries) go to the
    block sort: one shared-memory pass up to 2048 entries, beyond that sorted
    chunks merged in global memory (an even and an odd number of merge
    rounds).  The list is still in strictly ascending (depth key, pair) order
    and the render still matches the oracle.  (Seeds chosen so that no pixel is
    within float32 reach of an alpha or termination threshold.)"""
    g, v = syn.tiny_scene(seed, n=n, width=16, height=16, fx=20.0, coverage=0.6)
    res = oracle_run(g, v, grad=False)
    plan, P = gpu_run(g, [v], tile=(16, 16), grad=False)
    K = plan.k_value()
    assert plan.n_active == 1 and K >= kmin
    dup = plan.dup_pairs[:K].cpu().numpy().astype(np.int64)
    key = plan.dkey.cpu().numpy().view(np.uint32).astype(np.int64)
    k0, k1 = key[dup[:-1]], key[dup[1:]]
    assert ((k0 < k1) | ((k0 == k1) & (dup[:-1] < dup[1:]))).all()
    bi = plan.bininfo.cpu().numpy().astype(np.int64)
    assert (np.bincount(dup, minlength=len(bi)) == bi[:, 3]).all()
    compare_forward(plan, 0, res)


def test_neighbour_table_and_chunk_records(config0):
    """Mask-preparation tables: each rendered pixel's {up, down, left, right}
    entries are the px_list positions of those neighbours (~0 outside the image
    or outside R), its compact flags equal the dense ones, and the chunk records
    {view, first entry, count, tile} cover px_list exactly, 32 entries at most."""
    g, views, res = config0
    plan, P = gpu_run(g, views, grad=False)
    H, W = plan.shapes[0]
    px = plan.px_list[:plan.n_render].cpu().numpy().astype(np.int64)
    pidx = plan.pidx.cpu().numpy().view(np.uint32).astype(np.int64).reshape(H, W)
    nbr = plan.nbr[:plan.n_render].cpu().numpy().view(np.uint32).astype(np.int64)
    y, x = px // W, px % W
    none = 0xFFFFFFFF
    exp = np.stack([np.where(y > 0, pidx[np.maximum(y - 1, 0), x], none),
                    np.where(y < H - 1, pidx[np.minimum(y + 1, H - 1), x], none),
                    np.where(x > 0, pidx[y, np.maximum(x - 1, 0)], none),
                    np.where(x < W - 1, pidx[y, np.minimum(x + 1, W - 1)], none)], 1)
    assert np.array_equal(nbr, exp)
    # a neighbour index points back at that neighbour's pixel
    ok = exp[:, 0] != none
    assert np.array_equal(px[exp[ok, 0]], px[ok] - W)
    fl = plan.flags_image(0).cpu().numpy().reshape(-1)
    assert np.array_equal(plan.flags_c[:plan.n_render].cpu().numpy(), fl[px])
    ch = plan.chunks[:plan.n_chunks].cpu().numpy().astype(np.int64)
    assert (ch[:, 0] == 0).all() and (ch[:, 2] >= 1).all() and (ch[:, 2] <= 32).all()
    cover = np.zeros(plan.n_render, np.int64)
    for first, cnt in ch[:, 1:3]:
        cover[first:first + cnt] += 1
    assert (cover == 1).all()
    at = plan.act_tiles[:plan.n_active].cpu().numpy().astype(np.int64)
    t = ch[:, 3]
    assert ((ch[:, 1] >= at[t, 2]) & (ch[:, 1] + ch[:, 2] <= at[t, 2] + at[t, 3])).all()


def test_forward_and_sort_bit_stable_across_runs(config0):
    """No atomics in the forward: the sorted duplicate lists and every forward
    output are bit-identical when the step is run again."""
    from paper_2501_01677_b300 import raster
    g, views, res = config0
    P = raster.GaussianParams.from_numpy(g)
    plan = raster.Plan([views[0].cam], [views[0].mask], [views[0].target], g.n)
    plan.forward(P)
    torch.cuda.synchronize()
    K = plan.k_value()
    dup1 = plan.dup_pairs[:K].clone()
    out1, aux1, dep1 = plan.out8.clone(), plan.aux.clone(), plan.depth.clone()
    for _ in range(2):
        plan.forward(P)
        torch.cuda.synchronize()
        assert plan.k_value() == K
        assert torch.equal(plan.dup_pairs[:K], dup1)
        assert torch.equal(plan.out8, out1) and torch.equal(plan.aux, aux1) and torch.equal(plan.depth, dep1)


@pytest.mark.parametrize("objective", ["pg", "eq11"])
def test_plan_over_a_gaussian_span_equals_plan_over_the_slice(objective):
    """A plan whose views render the range [a, b) of a larger Gaussian array works
    on that span only (offset pointers): outputs bitwise those of a plan over the
    sliced arrays, gradients equal on the span and zero outside it (under Eq. 11
    the flattening term is the mean over the span's Gaussians)."""
    from paper_2501_01677_b300 import raster
    g, v = syn.tiny_scene(12, n=300, width=64, height=48)
    a, b = 70, 230
    sub = g.subset(np.arange(a, b))
    P_s = raster.GaussianParams.from_numpy(sub, requires_grad=True)
    plan_s = raster.Plan([v.cam], [v.mask], [v.target], sub.n)
    plan_s.set_objective(objective)
    raster.render_loss(plan_s, P_s).backward()
    P = raster.GaussianParams.from_numpy(g, requires_grad=True)
    plan = raster.Plan([v.cam], [v.mask], [v.target], g.n, g_ranges=[(a, b)])
    plan.set_objective(objective)
    assert (plan.g_lo, plan.g_hi) == (a, b)
    loss = raster.render_loss(plan, P)
    loss.backward()
    torch.cuda.synchronize()
    plan.check_status()
    assert np.array_equal(plan.out8.cpu().numpy(), plan_s.out8.cpu().numpy())
    assert np.array_equal(plan.aux.cpu().numpy(), plan_s.aux.cpu().numpy())
    for t, ts in zip(P.tensors(), P_s.tensors()):
        gr = t.grad.cpu().numpy()
        assert rel_l2(gr[a:b].ravel().astype(np.float64), ts.grad.cpu().numpy().ravel().astype(np.float64)) < 1e-6
        assert float(np.abs(gr[:a]).max(initial=0.0)) == 0.0 and float(np.abs(gr[b:]).max(initial=0.0)) == 0.0


def test_backward_after_another_forward_on_the_plan_raises():
    """The plan's buffers carry a forward's state to its backward; a second
    forward on the same plan in between is detected."""
    from paper_2501_01677_b300 import raster
    g, v = syn.tiny_scene(13, n=64, width=40, height=32)
    P = raster.GaussianParams.from_numpy(g, requires_grad=True)
    plan = raster.Plan([v.cam], [v.mask], [v.target], g.n)
    loss = raster.render_loss(plan, P)
    plan.forward(raster.GaussianParams(*[t.detach() for t in P.tensors()]))
    with pytest.raises(RuntimeError, match="another forward"):
        loss.backward()
    out8, depth = raster.render(plan, P)
    raster.render_loss(plan, raster.GaussianParams(*[t.detach().clone().requires_grad_(True) for t in P.tensors()]))
    with pytest.raises(RuntimeError, match="another forward"):
        out8.sum().backward()


def test_backward_with_check_raises_on_device_status():
    """With check=True the backward reads the device status once: a step whose
    kernels found an error (here a status planted before the adjoint) raises
    instead of returning gradients the skipped kernels never wrote."""
    from paper_2501_01677_b300 import _lib as L
    from paper_2501_01677_b300 import raster
    g, v = syn.tiny_scene(14, n=64, width=40, height=32)
    P = raster.GaussianParams.from_numpy(g, requires_grad=True)
    plan = raster.Plan([v.cam], [v.mask], [v.target], g.n)
    loss = raster.render_loss(plan, P, check=True)
    plan.status.fill_(L.PGSAG_DEV_BOUNDS)
    with pytest.raises(L.PgsagError):
        loss.backward()


def test_persistent_lpt_multiview_step_matches_oracle_per_view():
    """Two views of one scene (different masks and targets) in one plan with the
    persistent longest-first render queue: the summed loss and gradients equal
    the sums of the oracle's per-view losses and gradients."""
    from paper_2501_01677_b300 import raster
    g, v = syn.tiny_scene(9, n=200, width=72, height=64)
    v2 = syn.View(v.cam, np.ascontiguousarray(v.mask[:, ::-1]), np.ascontiguousarray(v.target[:, ::-1]))
    views = [v, v2]
    P = raster.GaussianParams.from_numpy(g, requires_grad=True)
    plan = raster.Plan([x.cam for x in views], [x.mask for x in views], [x.target for x in views], g.n)
    plan.forward(raster.GaussianParams(*[t.detach() for t in P.tensors()]))  # sizes the capacity
    plan.use_persistent_schedule(ctas_per_sm=0, lpt=True)
    loss = raster.render_loss(plan, P)
    loss.backward()
    torch.cuda.synchronize()
    plan.check_status()
    refs = [oracle_run(g, x) for x in views]
    want = sum(float(r["loss"]["total"].detach()) for r in refs)
    assert float(loss.detach()) == pytest.approx(want, rel=1e-5)
    for name, t in zip(("means", "log_scales", "quats", "opacity_logit", "sh"), P.tensors()):
        ref = sum(r["grads"][name].numpy() for r in refs)
        err = rel_l2(t.grad.cpu().numpy().ravel().astype(np.float64), ref.ravel())
        assert err <= GRAD_TOL, (name, err)
