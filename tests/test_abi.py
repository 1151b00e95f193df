"""Host-side checks of the C ABI: the library loads, exports every function the header
declares, its struct layouts match the binding, and the host helpers behave.  No kernel
is launched (no GPU needed)."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "radsplat.h")


@pytest.fixture(scope="module")
def native():
    from paper_2403_13806_gb300 import build, _native
    build.build()
    return _native


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(rs_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_hot_path():
    fns = declared_functions()
    for name in ("rs_project", "rs_bin_sort", "rs_render", "rs_importance", "rs_filter", "rs_filter_nearest",
                 "rs_render_backward", "rs_workspace_size", "rs_status_str"):
        assert name in fns


def test_library_exports_every_declared_symbol(native):
    L = ctypes.CDLL(native.LIB_PATH)
    missing = [f for f in declared_functions() if not hasattr(L, f)]
    assert not missing, missing
    assert set(declared_functions()) == set(native.SIGNATURES), "binding signatures out of date"


def test_struct_layouts_match(native):
    L = native.lib()
    assert L.rs_abi_version() == 1
    assert ctypes.sizeof(native.RsView) == 128
    n = len(native.STRUCTS)
    sizes = (ctypes.c_int64 * n)()
    assert L.rs_struct_sizes(sizes, n) == n
    assert list(sizes) == [ctypes.sizeof(c) for c in native.STRUCTS]
    assert ctypes.sizeof(native.RsTuneResult) == 32


def test_autotune_host_checks(native):
    L = native.lib()
    assert L.rs_autotune_candidates(0) == 0
    # stage 1: three tile shapes x 1, 2, 4 staged records per thread; stage 2: views per launch
    assert L.rs_autotune_candidates(1) == 9 + 1
    assert L.rs_autotune_candidates(4) == 9 + 3      # 1, 2, 4
    assert L.rs_autotune_candidates(5) == 9 + 4      # 1, 2, 4, 5
    res = native.RsTuneResult()
    # argument checks happen before any device work
    assert L.rs_autotune(None, None, 1, None, None, None, 0, ctypes.byref(res), None, None) == native.RS_ERR_INVALID_ARG
    L.rs_autotune_clear()


def test_status_strings(native):
    assert native.status_str(0) == "ok"
    assert "capacity" in native.status_str(native.RS_ERR_CAPACITY)
    assert native.status_str(99) == "unknown status"


def test_config_defaults(native):
    c = native.lib().rs_config_default()
    assert c.eps2d == pytest.approx(0.3) and c.near_plane == pytest.approx(0.2)
    assert list(c.bg) == [0.0, 0.0, 0.0]
    assert c.batch == 0 and c.grad_overwrite == 0   # default staging; gradients are added


def make_cams(sizes):
    from paper_2403_13806_gb300 import synth
    return [synth.camera(synth.look_at((0, 0, -4.0 - i), (0, 0, 0)), 100.0 + i, 90.0, w / 2, h / 2, w, h)
            for i, (w, h) in enumerate(sizes)]


def prepare(native, cams, n_items, tile):
    from paper_2403_13806_gb300.api import _camera_struct
    V = len(cams)
    arr = (native.RsCamera * V)(*[_camera_struct(c) for c in cams])
    out = (native.RsView * V)()
    b = native.RsViewBatch()
    n = np.asarray(n_items, dtype=np.int64)
    rc = native.lib().rs_views_prepare(arr, V, n.ctypes.data_as(ctypes.c_void_p), tile[0], tile[1], out,
                                       ctypes.byref(b))
    return rc, out, b


def test_views_prepare_bases(native):
    cams = make_cams([(100, 50), (33, 17), (64, 64)])
    rc, out, b = prepare(native, cams, [10, 0, 7], (16, 16))
    assert rc == 0
    tiles = [(7, 4), (3, 2), (4, 4)]
    assert [(v.tiles_x, v.tiles_y) for v in out] == tiles
    assert [v.tile_base for v in out] == [0, 28, 34]
    assert [v.pixel_base for v in out] == [0, 5000, 5000 + 561]
    assert [v.item_base for v in out] == [0, 10, 10]
    assert b.n_tiles == 50 and b.n_items == 17 and b.n_pixels == 5000 + 561 + 4096
    # camera centre -R^T t and the J clamp limits
    vm = np.asarray(cams[0]["viewmat"], np.float64)
    np.testing.assert_allclose(list(out[0].campos), -vm[:, :3].T @ vm[:, 3], atol=1e-5)
    assert out[0].lim_x == pytest.approx(1.3 * 50 / 100.0)
    rc, out, b = prepare(native, cams, [10, 0, 7], (32, 8))
    assert rc == 0 and [(v.tiles_x, v.tiles_y) for v in out] == [(4, 7), (2, 3), (2, 8)]


def test_views_prepare_rejects_bad_input(native):
    cams = make_cams([(100, 50)])
    assert prepare(native, cams, [10], (16, 8))[0] == native.RS_ERR_UNSUPPORTED
    cams[0]["width"] = 0
    assert prepare(native, cams, [10], (16, 16))[0] == native.RS_ERR_INVALID_ARG
    cams = make_cams([(100, 50)])
    assert prepare(native, cams, [-1], (16, 16))[0] == native.RS_ERR_INVALID_ARG


def test_entry_points_reject_null_arguments(native):
    L = native.lib()
    assert L.rs_project(None, None, None, None, None, None) == native.RS_ERR_INVALID_ARG
    assert L.rs_bin_sort(None, None, None, None, 0, None, None) == native.RS_ERR_INVALID_ARG
    assert L.rs_render(None, None, None, None, None, None, None, None, 0, None) == native.RS_ERR_INVALID_ARG
    assert L.rs_importance(None, None, None, None, None, 0, None) == native.RS_ERR_INVALID_ARG
    assert L.rs_filter(None, 0, 0.0, 0, None, None, None, None, 0, None) == native.RS_ERR_INVALID_ARG
    assert L.rs_filter_nearest(None, 1, None, 1, None, None) == native.RS_ERR_INVALID_ARG
    assert L.rs_render_backward(*([None] * 10 + [0, None])) == native.RS_ERR_INVALID_ARG


def test_workspace_sizes_grow_with_the_problem(native):
    L = native.lib()
    b = native.RsViewBatch()
    b.n_items = 1000
    b.n_views = 1
    b.n_tiles = 64
    small = L.rs_workspace_size(native.RS_STAGE_BIN_SORT, ctypes.byref(b), 10_000)
    big = L.rs_workspace_size(native.RS_STAGE_BIN_SORT, ctypes.byref(b), 1_000_000)
    assert 0 < small < big
    assert big >= 4 * 4 * 1_000_000           # two key and two value buffers of super instances
    b.n_items = 10_000_000
    assert L.rs_workspace_size(native.RS_STAGE_FILTER, ctypes.byref(b), 0) >= 4 * (10_000_000 // 4096)
    assert L.rs_workspace_size(native.RS_STAGE_BACKWARD, ctypes.byref(b), 0) >= 36 * 10_000_000
    assert L.rs_workspace_size(native.RS_STAGE_PROJECT, ctypes.byref(b), 0) == 0


def test_staging_batch_values(native):
    """rs_config.batch: 0, or 1, 2 or 4 records per thread of the one-warp blend CTA (32, 64,
    128) for every tile shape; other values are rejected before anything is launched.  The
    batch below has no tiles, so an accepted call returns at once (the host pointers are
    only checked, never read)."""
    L = native.lib()
    mem = np.zeros(4096, np.float32)
    p = mem.ctypes.data
    assert p % 16 == 0
    proj = native.RsProjected(p, p, p, p, p)
    bins = native.RsBins(None, p, p, 0)
    for tile in ((16, 16), (32, 8), (8, 8)):
        b = native.RsViewBatch()
        b.views = p
        b.n_views = 1
        b.n_tiles = 0
        b.tile_w, b.tile_h = tile
        for batch, ok in ((0, True), (32, True), (64, True), (128, True), (96, False), (256, False), (16, False),
                          (-32, False)):
            cfg = L.rs_config_default()
            cfg.batch = batch
            want = native.RS_OK if ok else native.RS_ERR_UNSUPPORTED
            assert L.rs_render(ctypes.byref(proj), ctypes.byref(bins), ctypes.byref(b), ctypes.byref(cfg),
                               None, None, None, None, 0, None) == want, (tile, batch)
            assert L.rs_importance(ctypes.byref(proj), ctypes.byref(bins), ctypes.byref(b), ctypes.byref(cfg),
                                   p, 1, None) == want, (tile, batch)
