"""Host-side checks of the C-ABI library (no GPU): it loads, exports every entry
point declared in include/pgsag.h, its struct layout matches the binding and
its host-only queries answer."""
import ctypes
import os
import re

import pytest

from paper_2501_01677_b300 import _lib as L

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    with open(os.path.join(ROOT, "include", "pgsag.h")) as f:
        src = f.read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(pgsag_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(L.LIB_PATH):
        from paper_2501_01677_b300 import build
        build.build()
    return L.load()


def test_every_declared_symbol_is_exported(lib):
    names = header_functions()
    assert len(names) >= 14
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(L.EXPORTS) == names


def test_view_struct_layout(lib):
    assert ctypes.sizeof(L.PgsagView) == 152
    assert b"152" in lib.pgsag_build_info()


def test_struct_layouts(lib):
    assert ctypes.sizeof(L.PgsagBanGather) == 64
    assert ctypes.sizeof(L.PgsagClear) == 80
    assert ctypes.sizeof(L.PgsagDssim) == 32
    assert ctypes.sizeof(L.PgsagAdamTensor) == 48
    assert ctypes.sizeof(L.PgsagDepthView) == 96
    assert ctypes.sizeof(L.PgsagTsdfGrid) == 32
    assert ctypes.sizeof(L.PgsagVoteView) == 96
    assert ctypes.sizeof(L.PgsagSched) == 24


def test_status_strings(lib):
    assert lib.pgsag_status_str(0) == b"ok"
    assert b"argument" in lib.pgsag_status_str(-1)
    assert b"unknown" in lib.pgsag_status_str(17)


def test_bin_workspace_size_grows_with_sizes(lib):
    a = lib.pgsag_bin_workspace_size(1000, 100, 4000)
    b = lib.pgsag_bin_workspace_size(1000, 100000, 4000)
    c = lib.pgsag_bin_workspace_size(1000, 100000, 8000)
    assert 0 < a < b < c
    assert b - a >= 4 * (100000 - 100) - 512     # one counter per active tile
    assert c - b >= 3 * 4 * 4000 - 768           # three entries per duplicate


def test_invalid_arguments_rejected_on_host(lib):
    # argument errors are detected before any device work
    assert lib.pgsag_preprocess(10, None, None, None, None, None, 0, None, None, None, None, None, None, None,
                                None, None, None) == -5
    assert lib.pgsag_bin(10, 1, None, 0, None, None, None, None, 0, None, 0, None, None, None, None, None) == -1
    assert lib.pgsag_adam(10, None, None, None, None, 0.1, 0.9, 0.999, 1e-8, 1, None) == -1
    # unknown render flags / objective
    assert lib.pgsag_render_fwd(1, ctypes.c_void_p(16), None, None, None, None, 0, None, None, 8, None, None, None,
                                ctypes.c_void_p(16), None) == -5
    assert lib.pgsag_loss_ban(1, None, 0, None, None, None, None, None, None, None, None, None, 0.01, None, 0, None,
                              None, None, None, None, None, 7, 0, None, None, None, None) == -5
    # the Eq. 11 objective needs the GC weights and the deferred gather
    st = ctypes.c_void_p(16)
    assert lib.pgsag_loss_ban(1, st, 0, None, None, None, None, None, None, None, None, None, 0.01, None, 0, None,
                              st, None, st, None, None, 1, 0, None, None, st, None) == -1
    # D-SSIM needs the pixel map, its scratch and an aligned tile list
    d = L.PgsagDssim(None, None, 10, 16, 16, 0.2)
    assert lib.pgsag_loss_ban(1, st, 0, None, None, None, None, None, None, None, None, None, 0.01, None, 1, None,
                              st, None, st, None, None, 0, 0, None, ctypes.byref(d), st, None) == -1
    # voting filter: too many views, missing buffers, bad view table
    assert lib.pgsag_vote_filter(10, None, 300, None, None, 3, 0, None, None, None, st, None) == -5
    assert lib.pgsag_vote_filter(10, None, 1, None, None, 3, 0, None, None, None, st, None) == -1
    v = L.PgsagVoteView()
    v.width, v.height, v.words_per_row = 100, 10, 3   # 3 words < 100 pixels
    assert lib.pgsag_vote_filter(10, st, 1, ctypes.byref(v), st, 3, 0, st, st, st, st, None) == -1
    assert lib.pgsag_vote_pack_mask(100, 10, st, 3, st, None) == -1
    assert lib.pgsag_vote_compact_workspace_size(0) == 4


def test_adjoint_clear_and_accumulate_modes_checked_on_host(lib):
    """The render adjoint's side clear takes 16-byte aligned buffers and the
    projection adjoint's accumulate modes 0-2; a view count beyond
    PGSAG_MAX_VIEWS is refused; all before any device work."""
    st = ctypes.c_void_p(16)

    def render_bwd(n_views, clear):
        return lib.pgsag_render_bwd(n_views, st, None, None, None, None, 0, None, None, None, None, None, None, None,
                                    None, 0, None, clear, st, None)

    def clear_of(ptr, n):
        c = L.PgsagClear()
        c.ptr[0], c.n[0] = ptr, n
        return ctypes.byref(c)
    assert render_bwd(1, clear_of(24, 8)) == -1          # not 16-byte aligned
    assert render_bwd(1, clear_of(None, 8)) == -1        # null buffer with floats to clear
    assert render_bwd(L.MAX_VIEWS + 1, None) == -5
    args = [10, st, st, st, st, st, 1, st, st, st, None, st, st, st, st, st, None, 0.0, st, None]
    for bad in (-1, 3):
        a = list(args)
        a[10] = bad
        assert lib.pgsag_preprocess_bwd(*a) == -1
    a = list(args)
    a[6] = L.MAX_VIEWS + 1
    a[10] = 0
    assert lib.pgsag_preprocess_bwd(*a) == -5
    assert lib.pgsag_vote_compact_workspace_size(4097) == 8


def test_autograd_backward_asks_for_the_clear_only_where_it_can():
    """The autograd backward hands the render adjoint the gradient buffers to
    clear only when the plan spans every Gaussian and each buffer starts on 16
    bytes (the C ABI's alignment); a plan over a span gets zero-filled buffers
    instead, which the projection adjoint may also take as zeros."""
    import torch
    from paper_2501_01677_b300 import raster
    n = 10
    P = raster.GaussianParams(torch.zeros(n, 3), torch.zeros(n, 3), torch.zeros(n, 4), torch.zeros(n),
                              torch.zeros(n, 16, 3))

    def plan(lo, hi):
        p = raster.Plan.__new__(raster.Plan)  # host logic only: no device buffers
        p.g_lo, p.g_hi, p.n_gauss = lo, hi, n
        return p
    full, part = plan(0, n), plan(2, 7)
    grads = [torch.zeros_like(t) for t in P.tensors()]
    assert full.clearable(grads) is grads
    assert part.clearable(grads) is None
    shifted = [torch.zeros(t.numel() + 1)[1:].view(t.shape) for t in P.tensors()]  # 4 bytes past an allocation
    assert all(t.data_ptr() % 16 == 4 for t in shifted)
    assert full.clearable(shifted) is None
    g, clear, cleared = full.backward_grads(P)
    assert clear is g and cleared
    assert [t.shape for t in g] == [t.shape for t in P.tensors()]
    g, clear, cleared = part.backward_grads(P)
    assert clear is None and cleared
    assert all(float(t.abs().max()) == 0.0 for t in g)
