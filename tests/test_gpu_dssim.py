"""Masked D-SSIM term of L_rgb: CUDA path through the C-ABI vs the FP64 oracle
(loss values to 1e-4, gradients rel-L2 <= 1e-3)."""
import numpy as np
import pytest
import torch

import pgsag_synth as syn
from oracle import pgsag_oracle as O
from tests._helpers import compare_grads

pytestmark = pytest.mark.gpu


def gpu_dssim(g, views, tile=(16, 16), objective="pg", grad=True):
    from paper_2501_01677_b300 import raster
    P = raster.GaussianParams.from_numpy(g, requires_grad=grad)
    plan = raster.Plan([v.cam for v in views], [v.mask for v in views], [v.target for v in views], g.n, tile=tile)
    plan.set_objective(objective)
    plan.set_dssim(0.2)
    loss = raster.render_loss(plan, P)
    if grad:
        loss.backward()
    torch.cuda.synchronize()
    plan.check_status()
    return plan, P, float(loss.detach())


@pytest.fixture(scope="module")
def config0():
    g, views = syn.config0()
    return g, views, O.step(g, views[0], dssim=True)


def test_config0_dssim_loss_and_gradients(config0):
    g, views, res = config0
    plan, P, loss = gpu_dssim(g, views)
    L = res["loss"]
    assert loss == pytest.approx(float(L["total"].detach()), rel=1e-4)
    errs = compare_grads(P, res)
    print("dssim config0 gradient rel-L2", errs)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_tiny_scenes_dssim(seed):
    g, v = syn.tiny_scene(seed, n=64, width=40, height=32)
    res = O.step(g, v, dssim=True)
    plan, P, loss = gpu_dssim(g, [v])
    assert loss == pytest.approx(float(res["loss"]["total"].detach()), rel=1e-4)
    compare_grads(P, res)


@pytest.mark.parametrize("tile", [(8, 8), (16, 32), (32, 32)])
def test_dssim_independent_of_tile_shape(config0, tile):
    g, views, res = config0
    _, _, loss = gpu_dssim(g, views, tile=tile, grad=False)
    assert loss == pytest.approx(float(res["loss"]["total"].detach()), rel=1e-4)


def test_dssim_with_eq11_objective():
    g, v = syn.tiny_scene(5, n=64, width=40, height=32)
    res = O.step(g, v, objective="eq11", dssim=True)
    plan, P, loss = gpu_dssim(g, [v], objective="eq11")
    assert loss == pytest.approx(float(res["loss"]["total"].detach()), rel=1e-4)
    compare_grads(P, res)


def test_dssim_two_views_in_one_plan():
    g, views = syn.config2(n_gauss=20000, width=320, height=180, n_views=2)[:2]
    plan, P, loss = gpu_dssim(g, views, grad=False)
    want = sum(float(O.step(g, v, need_grad=False, dssim=True)["loss"]["total"]) for v in views)
    assert loss == pytest.approx(want, rel=1e-4)
