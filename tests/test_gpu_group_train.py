"""Parallel group training (Sec. 5.1): fused multi-tensor Adam with a device step
count vs torch.optim.Adam, and the GroupTrainer's graph-replayed iterations vs
the same iterations run eagerly."""
import numpy as np
import pytest
import torch

import pgsag_synth as syn

pytestmark = pytest.mark.gpu


def test_adam_multi_matches_torch_and_graph_replay():
    import ctypes
    from paper_2501_01677_b300 import _lib as L
    lib = L.load()
    torch.manual_seed(1)
    shapes = [(1003, 3), (1003, 4), (1003,), (1003, 16, 3), (7,)]
    lrs = [1.6e-4, 5e-3, 5e-2, 2.5e-3, 1e-2]
    ps = [torch.randn(s, device="cuda") for s in shapes]
    ref = [p.clone().requires_grad_(True) for p in ps]
    opt = torch.optim.Adam([{"params": [r], "lr": lr} for r, lr in zip(ref, lrs)], betas=(0.9, 0.999), eps=1e-15)
    gs = [torch.zeros_like(p) for p in ps]
    m = [torch.zeros_like(p) for p in ps]
    v = [torch.zeros_like(p) for p in ps]
    step = torch.zeros(4, dtype=torch.int32, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    tab = (L.PgsagAdamTensor * 5)()
    for k in range(5):
        tab[k] = L.PgsagAdamTensor(ps[k].data_ptr(), gs[k].data_ptr(), m[k].data_ptr(), v[k].data_ptr(),
                                   ps[k].numel(), lrs[k], 0)
    def call():
        s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)   # the capture stream inside a capture
        return lib.pgsag_adam_multi(5, tab, 0.9, 0.999, 1e-15, ctypes.c_void_p(step.data_ptr()),
                                    ctypes.c_void_p(status.data_ptr()), s)

    # steps 1-2 eagerly, then 3 graph replays of one captured call
    graph = None
    for it in range(5):
        g_new = [torch.randn_like(p) for p in ps]
        for a, b in zip(gs, g_new):
            a.copy_(b)
        if it < 2:
            assert call() == 0
        else:
            if graph is None:
                torch.cuda.synchronize()
                graph = torch.cuda.CUDAGraph()
                with torch.cuda.graph(graph):
                    assert call() == 0
            graph.replay()
        for r, gg in zip(ref, g_new):
            r.grad = gg.clone()
        opt.step()
    torch.cuda.synchronize()
    assert int(step[0].item()) == 5 and int(status.item()) == 0
    for p, r in zip(ps, ref):
        np.testing.assert_allclose(p.cpu().numpy(), r.detach().cpu().numpy(), rtol=2e-6, atol=2e-7)


def small_groups(scale=0.01, views=3):
    g, ranges, views_all, owner = syn.config3(scale=scale, views_per_region=views)
    by_group = [[vw for vw, o in zip(views_all, owner) if o == s] for s in range(len(ranges))]
    return g, ranges, by_group


def test_graph_replayed_iterations_equal_eager_iterations():
    from paper_2501_01677_b300 import raster, train
    g, ranges, by_group = small_groups()
    A = raster.GaussianParams.from_numpy(g)
    B = raster.GaussianParams.from_numpy(g)
    ta = train.GroupTrainer(A, by_group, ranges)
    tb = train.GroupTrainer(B, by_group, ranges)
    order = ta.schedule(9, seed=3)
    la, lb = [], []
    for j in order:
        la.append(float(ta.iteration(j)[-1].item()))
        lb.append(float(tb.eager_iteration(j)[-1].item()))
    ta.check_status()
    tb.check_status()
    assert all(x is not None for x in ta.graphs)       # every slot captured and replayed
    np.testing.assert_allclose(la, lb, rtol=1e-5)
    # the render adjoint sums gradients with float atomics, so the two runs differ
    # in the last bits; Adam turns such a difference in a near-zero gradient into
    # a different step of up to ~3.2 lr (bias-corrected |m| / sqrt(v) <= (1 - b1) /
    # sqrt(1 - b2)), so a few elements may differ by that much, the rest must not
    for a, b, lr in zip(A.tensors(), B.tensors(), train.DEFAULT_LRS):
        diff = (a - b).abs()
        tol = 1e-5 * max(1.0, b.abs().max().item())
        frac = (diff > tol).float().mean().item()
        assert frac <= 1e-3, frac
        assert diff.max().item() <= 2 * 3.2 * lr * len(order), diff.max().item()
    assert int(ta.step_dev[0].item()) == 9


def test_training_reduces_the_loss():
    from paper_2501_01677_b300 import raster, train
    g, ranges, by_group = small_groups(views=2)
    P = raster.GaussianParams.from_numpy(g)
    tr = train.GroupTrainer(P, by_group, ranges)
    losses = tr.run(60, seed=0).cpu().numpy()
    tr.check_status()
    assert np.isfinite(losses).all()
    first = losses[:4].mean()
    last = losses[-4:].mean()
    assert last < 0.9 * first, (first, last)


def test_checkpoint_resume_adam_bit_identical_and_trainer_resume(tmp_path):
    """A resumed Adam step is bit-identical to the uninterrupted one (same
    gradients); a trainer restored from a checkpoint continues like the original
    (to rounding: the render adjoint sums with float atomics)."""
    from paper_2501_01677_b300 import raster, train
    g, ranges, by_group = small_groups(views=2)
    A = raster.GaussianParams.from_numpy(g)
    ta = train.GroupTrainer(A, by_group, ranges)
    ta.run(4, seed=0)
    path = str(tmp_path / "ckpt.pt")
    ta.save(path)
    # Adam alone, same gradients: uninterrupted vs restored
    B = raster.GaussianParams.from_numpy(g)
    tb = train.GroupTrainer(B, by_group, ranges)
    tb.load(path)
    for a, b in zip(A.tensors(), B.tensors()):
        assert torch.equal(a, b)
    torch.manual_seed(5)
    for ga, gb in zip(ta.grads, tb.grads):
        r = torch.randn_like(ga)
        ga.copy_(r)
        gb.copy_(r)
    ta._adam()
    tb._adam()
    torch.cuda.synchronize()
    for a, b in zip(A.tensors(), B.tensors()):
        assert torch.equal(a, b)
    assert int(ta.step_dev[0].item()) == int(tb.step_dev[0].item()) == 5
    # whole iterations after the restore
    la = ta.run(4, seed=9).cpu().numpy()
    lb = tb.run(4, seed=9).cpu().numpy()
    np.testing.assert_allclose(la, lb, rtol=1e-5)
