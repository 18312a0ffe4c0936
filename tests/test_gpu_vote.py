"""Voting filter (Sec. 4.1, Eq. 5-7): CUDA path through the C-ABI vs the oracle.
Counts, flags and compacted indices are integers: bit-exact."""
import json
import os
from types import SimpleNamespace

import numpy as np
import pytest
import torch

import pgsag_synth as syn
from oracle import vote_oracle as VO


def _load_json(path):
    with open(path) as f:
        return json.load(f)


pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def gpu_vote(points, cams, masks, tau, words_per_row=None):
    from paper_2501_01677_b300 import vote
    md = [torch.from_numpy(np.ascontiguousarray(m, np.uint8)).cuda() for m in masks]
    packed = vote.pack_masks(md, words_per_row) if md else None
    if packed is None:
        packed = vote.PackedMasks(torch.zeros(1, dtype=torch.int32, device="cuda"), [], [], [], [])
    pts = torch.from_numpy(np.ascontiguousarray(points, np.float32).reshape(-1, 3)).cuda()
    res = vote.vote_filter(pts, cams, packed, tau)
    idx = vote.compact(res.reliable)
    torch.cuda.synchronize()
    assert int(res.status.item()) == 0
    return (res.in_mask.cpu().numpy().astype(np.int64), res.us.cpu().numpy().astype(np.int64),
            res.reliable.cpu().numpy().astype(bool), idx.cpu().numpy().astype(np.int64), packed)


def check(points, cams, masks, tau, **kw):
    ci, cu, rel, idx, packed = gpu_vote(points, cams, masks, tau, **kw)
    oi, ou, orel, oidx = VO.vote_filter(points, cams, masks, tau)
    np.testing.assert_array_equal(ci, oi)
    np.testing.assert_array_equal(cu, ou)
    np.testing.assert_array_equal(rel, orel)
    np.testing.assert_array_equal(idx, oidx)
    return ci, cu, rel, idx, packed


def test_pack_mask_bits_ragged_rows():
    from paper_2501_01677_b300 import vote
    rng = np.random.default_rng(3)
    masks = [(rng.random((7, w)) < 0.4).astype(np.uint8) * rng.integers(1, 255, (7, w)).astype(np.uint8)
             for w in (1, 31, 32, 37, 64, 100, 1000)]
    wprs = [(m.shape[1] + 31) // 32 + extra for m, extra in zip(masks, (0, 1, 0, 2, 0, 1, 3))]
    packed = vote.pack_masks([torch.from_numpy(m).cuda() for m in masks], wprs)
    bits = packed.bits.cpu().numpy().view(np.uint32)
    for m, off, wpr in zip(masks, packed.offsets, packed.words_per_row):
        H, W = m.shape
        want = np.zeros((H, wpr * 32), np.uint8)
        want[:, :W] = m != 0
        words = (want.reshape(H, wpr, 32).astype(np.uint64) << np.arange(32, dtype=np.uint64)).sum(-1)
        np.testing.assert_array_equal(bits[off:off + H * wpr].reshape(H, wpr), words.astype(np.uint32))


def test_hand_worked_example():
    g = _load_json(os.path.join(GOLDEN, "vote_example.json"))
    cams = [SimpleNamespace(R=np.eye(3, dtype=np.float32), t=np.asarray(v["t"], np.float32), fx=2.0, fy=2.0,
                            cx=2.0, cy=2.0, znear=0.2, width=4, height=4) for v in g["views"]]
    masks = [np.asarray(v["mask"], np.uint8) for v in g["views"]]
    pts = np.asarray(g["points"], np.float32)
    ci, cu, rel, idx, _ = check(pts, cams, masks, 1)
    assert ci.tolist() == g["in_mask"] and cu.tolist() == g["us"]
    assert rel.astype(int).tolist() == g["reliable_tau1"]
    _, _, rel2, _, _ = check(pts, cams, masks, 2)
    assert rel2.astype(int).tolist() == g["reliable_tau2"]


@pytest.mark.parametrize("n_points,n_views,W,H", [(20000, 6, 640, 480), (70001, 13, 1000, 750), (3, 1, 37, 5)])
def test_vote_parity_synthetic(n_points, n_views, W, H):
    w = syn.vote_workload(n_points=n_points, n_views=n_views, width=W, height=H, mask_step=1 if W < 64 else 2)
    ci, cu, rel, idx, _ = check(w.points, w.cams, w.masks, w.tau)
    if n_points > 1000:
        assert (ci > 0).mean() > 0.3 and rel.any() and not rel.all()


def test_edges_borders_near_plane_and_nonfinite_points():
    W, H = 37, 9   # width not a multiple of 32: a ragged last word
    cam = SimpleNamespace(R=np.eye(3, dtype=np.float32), t=np.zeros(3, np.float32), fx=1.0, fy=1.0, cx=0.0, cy=0.0,
                          znear=0.2, width=W, height=H)
    rng = np.random.default_rng(9)
    mask = (rng.random((H, W)) < 0.5).astype(np.uint8)
    pts = [[0.0, 0.5, 1.0], [-2.0 ** -20, 0.5, 1.0], [37.0, 0.5, 1.0], [37.0 - 2.0 ** -10, 8.5, 1.0],
           [0.5, 9.0, 1.0], [0.5, 9.0 - 2.0 ** -10, 1.0], [0.5, 0.5, 0.2], [0.5, 0.5, 0.2 + 2.0 ** -20],
           [np.nan, 0, 1], [0, np.inf, 1], [0, 0, np.inf], [0, 0, -np.inf], [1e30, 1e30, 1e-30]]
    pts += [[x + 0.5, y + 0.5, 1.0] for y in range(H) for x in range(W)]   # every pixel once
    pts = np.asarray(pts, np.float32)
    ci, cu, rel, idx, _ = check(pts, [cam], [mask], 1, words_per_row=[3])
    np.testing.assert_array_equal(ci[13:], mask.reshape(-1))


def test_degenerate_sizes_and_tau():
    w = syn.vote_workload(n_points=5000, n_views=4, width=320, height=240, mask_step=2)
    check(w.points[:0], w.cams, w.masks, w.tau)             # no points
    ci, cu, rel, idx, _ = check(w.points, [], [], w.tau)     # no views: zero counts
    assert ci.sum() == 0 and cu.sum() == 0 and idx.size == 0
    _, _, rel, idx, _ = check(w.points, w.cams, w.masks, 0)  # tau = 0 keeps nothing
    assert idx.size == 0
    _, _, rel, idx, _ = check(w.points, w.cams, w.masks, 1000)


def test_more_views_than_one_call_accumulates():
    # 300 views > 256 per call: the binding splits the views and accumulates the counts
    w = syn.vote_workload(n_points=3000, n_views=300, width=64, height=48, mask_step=1)
    ci, cu, rel, idx, _ = check(w.points, w.cams, w.masks, 40)
    assert ci.max() > 0


@pytest.mark.parametrize("n", [1, 4095, 4096, 4097, 1_000_003])
def test_compact_matches_nonzero(n):
    from paper_2501_01677_b300 import vote
    rng = np.random.default_rng(n)
    flags = (rng.random(n) < 0.37).astype(np.uint8)
    idx = vote.compact(torch.from_numpy(flags).cuda()).cpu().numpy()
    np.testing.assert_array_equal(idx, np.nonzero(flags)[0])


def test_vote_parity_full_size():
    # the bench workload: 1M points against 32 coarse masks at 5472x3648
    w = syn.vote_workload()
    ci, cu, rel, idx, _ = check(w.points, w.cams, w.masks, w.tau)
    assert rel[w.on_building].mean() > 0.9
