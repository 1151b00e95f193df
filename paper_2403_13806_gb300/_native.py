"""ctypes mirror of include/radsplat.h and the loader of the in-tree CUDA library.

Argument marshalling only: every step of the hot path runs in the library's kernels.
Loading fails loudly if the library has not been built; there is no fallback.
"""
from __future__ import annotations

import ctypes
import os

from ctypes import c_float, c_int32, c_int64, c_size_t, c_void_p

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libradsplat.so")

RS_OK, RS_ERR_INVALID_ARG, RS_ERR_WORKSPACE, RS_ERR_UNSUPPORTED, RS_ERR_CUDA, RS_ERR_CAPACITY, RS_ERR_TIMEOUT = range(7)
RS_PRUNE_BELOW, RS_KEEP_ABOVE, RS_PRUNE_KEEP = 0, 1, 2
RS_FILTER_NOALLOC_MAX_N = 1 << 26
RS_STAGE_PROJECT, RS_STAGE_BIN_SORT, RS_STAGE_RENDER, RS_STAGE_BACKWARD, RS_STAGE_FILTER = range(5)
RS_PROBE_FFMA, RS_PROBE_FFMA2, RS_PROBE_ALU, RS_PROBE_EX2, RS_PROBE_SMEM, RS_PROBE_L2 = range(6)


class RsGaussians(ctypes.Structure):
    _fields_ = [("means", c_void_p), ("log_scales", c_void_p), ("quats", c_void_p), ("opacity_logit", c_void_p),
                ("sh", c_void_p), ("n", c_int64), ("sh_degree", c_int32), ("reserved", c_int32)]


class RsCamera(ctypes.Structure):
    _fields_ = [("viewmat", c_float * 12), ("fx", c_float), ("fy", c_float), ("cx", c_float), ("cy", c_float),
                ("width", c_int32), ("height", c_int32)]


class RsView(ctypes.Structure):
    _fields_ = [("viewmat", c_float * 12), ("fx", c_float), ("fy", c_float), ("cx", c_float), ("cy", c_float),
                ("campos", c_float * 3), ("lim_x", c_float), ("lim_y", c_float), ("width", c_int32),
                ("height", c_int32), ("tiles_x", c_int32), ("tiles_y", c_int32), ("tile_base", c_int32),
                ("pixel_base", c_int64), ("item_base", c_int64), ("n_items", c_int64)]


class RsViewBatch(ctypes.Structure):
    _fields_ = [("views", c_void_p), ("subset_idx", c_void_p), ("n_views", c_int32), ("n_tiles", c_int32),
                ("n_items", c_int64), ("n_pixels", c_int64), ("tile_w", c_int32), ("tile_h", c_int32)]


class RsConfig(ctypes.Structure):
    _fields_ = [("eps2d", c_float), ("near_plane", c_float), ("bg", c_float * 3), ("batch", c_int32),
                ("grad_overwrite", c_int32), ("reserved", c_int32 * 1)]


class RsProjected(ctypes.Structure):
    _fields_ = [("xy", c_void_p), ("conic_o", c_void_p), ("rgb_d", c_void_p), ("rect", c_void_p),
                ("n_tiles", c_void_p)]


class RsBins(ctypes.Structure):
    _fields_ = [("keys", c_void_p), ("vals", c_void_p), ("ranges", c_void_p), ("capacity", c_int64)]


class RsGaussianGrads(ctypes.Structure):
    _fields_ = [("means", c_void_p), ("log_scales", c_void_p), ("quats", c_void_p), ("opacity_logit", c_void_p),
                ("sh", c_void_p)]


class RsImageGrads(ctypes.Structure):
    _fields_ = [("g_xy_ab", c_void_p), ("g_c_o_rg", c_void_p), ("g_b", c_void_p)]


class RsDeviceStatus(ctypes.Structure):
    _fields_ = [("code", c_int32), ("nonfinite", c_int32), ("required", c_int64), ("n_instances", c_int64),
                ("reserved", c_int64)]


class RsTuneResult(ctypes.Structure):
    _fields_ = [("tile_w", c_int32), ("tile_h", c_int32), ("smem_batch", c_int32), ("views_per_launch", c_int32),
                ("ms_per_view", c_float), ("cached", c_int32), ("n_candidates", c_int32), ("front_lists", c_int32)]


RS_TUNE_BACKWARD, RS_TUNE_FORCE, RS_TUNE_FRONT = 1, 2, 4


class RsAdamGroup(ctypes.Structure):
    _fields_ = [("param", c_void_p), ("grad", c_void_p), ("m", c_void_p), ("v", c_void_p), ("n", c_int64),
                ("lr", c_float), ("reserved", c_int32)]


class RsGatherDesc(ctypes.Structure):
    _fields_ = [("src", c_void_p), ("dst", c_void_p), ("rows", c_int64), ("src_stride", c_int64),
                ("dst_stride", c_int64)]

STRUCTS = [RsGaussians, RsCamera, RsView, RsViewBatch, RsConfig, RsProjected, RsBins, RsGaussianGrads, RsDeviceStatus,
           RsTuneResult, RsAdamGroup, RsGatherDesc, RsImageGrads]

# every function include/radsplat.h declares, with its ctypes signature
P = c_void_p
SIGNATURES = {
    "rs_abi_version": (c_int32, []),
    "rs_status_str": (ctypes.c_char_p, [ctypes.c_int]),
    "rs_config_default": (RsConfig, []),
    "rs_views_prepare": (ctypes.c_int, [P, c_int32, P, c_int32, c_int32, P, P]),
    "rs_workspace_size": (c_size_t, [ctypes.c_int, P, c_int64]),
    "rs_struct_sizes": (c_int32, [P, c_int32]),
    "rs_project": (ctypes.c_int, [P, P, P, P, P, P]),
    "rs_bin_sort": (ctypes.c_int, [P, P, P, P, c_size_t, P, P]),
    "rs_bin_sort_front": (ctypes.c_int, [P, P, P, P, c_size_t, P, P]),
    "rs_render": (ctypes.c_int, [P, P, P, P, P, P, P, P, c_int64, P]),
    "rs_importance": (ctypes.c_int, [P, P, P, P, P, c_int64, P]),
    "rs_filter": (ctypes.c_int, [P, c_int64, c_float, ctypes.c_int, P, P, P, P, c_size_t, P]),
    "rs_filter_nearest": (ctypes.c_int, [P, c_int32, P, c_int32, P, P]),
    "rs_kmeans": (ctypes.c_int, [P, c_int32, P, c_int32, c_int32, P, P]),
    "rs_nn_distance": (ctypes.c_int, [P, c_int64, P, P, c_size_t, P]),
    "rs_nn_workspace_size": (c_size_t, [c_int64]),
    "rs_filter_noalloc": (ctypes.c_int, [P, c_int64, c_float, ctypes.c_int, P, P, P, P]),
    "rs_render_backward": (ctypes.c_int, [P, P, P, P, P, P, P, P, P, P, c_size_t, P]),
    "rs_backward_image_grads": (ctypes.c_int, [P, P, c_size_t, P]),
    "rs_l1_loss": (ctypes.c_int, [P, P, c_int64, P, P, P]),
    "rs_autotune": (ctypes.c_int, [P, P, c_int32, P, P, P, c_int32, P, P, P]),
    "rs_adam_step": (ctypes.c_int, [P, c_int32, c_float, c_float, c_float, c_int32, P]),
    "rs_ssim_loss": (ctypes.c_int, [P, P, c_int32, c_int32, c_int32, c_float, P, P, P, c_size_t, P]),
    "rs_ssim_workspace_size": (c_size_t, [c_int32, c_int32, c_int32]),
    "rs_gather_columns": (ctypes.c_int, [P, c_int32, P, P, c_int64, P]),
    "rs_scatter_columns": (ctypes.c_int, [P, c_int32, P, P, c_int64, P]),
    "rs_touched_columns": (ctypes.c_int, [P, c_int64, c_int64, P, P]),
    "rs_autotune_candidates": (c_int32, [c_int32]),
    "rs_autotune_clear": (None, []),
    "rs_peak_probe": (ctypes.c_int, [c_int32, c_int32, P, c_int64, P, P]),
    "rs_peak_probe_sink_floats": (c_int64, []),
    "rs_profile_enable": (ctypes.c_int, [c_int32]),
    "rs_profile_count": (c_int32, []),
    "rs_profile_read": (ctypes.c_int, [c_int32, P, P]),
}

_lib = None


class RadsplatError(RuntimeError):
    def __init__(self, fn: str, code: int):
        super().__init__(f"{fn} failed: {status_str(code)} ({code})")
        self.code = code


def lib(path: str = LIB_PATH):
    """The loaded library.  Raises if it is missing (build with __graft_entry__.build())."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise RuntimeError(f"CUDA library not built: {path} is missing (run __graft_entry__.build())")
        L = ctypes.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
        sizes = (c_int64 * len(STRUCTS))()
        n = L.rs_struct_sizes(sizes, len(STRUCTS))
        for s, cls in zip(sizes[:n], STRUCTS):
            if s != ctypes.sizeof(cls):
                raise RuntimeError(f"ABI mismatch: {cls.__name__} is {ctypes.sizeof(cls)} bytes here, {s} in the library")
    return _lib


def status_str(code: int) -> str:
    return lib().rs_status_str(int(code)).decode()


def check(fn: str, code: int):
    if code != RS_OK:
        raise RadsplatError(fn, code)


def call(fn: str, *args):
    check(fn, getattr(lib(), fn)(*args))


def ref(x):
    return ctypes.byref(x)


def profile_enable(on: bool):
    call("rs_profile_enable", 1 if on else 0)


def profile_records():
    """[(kernel name, device ms)] of the launches recorded since profile_enable(True)."""
    L = lib()
    out = []
    for i in range(L.rs_profile_count()):
        name = ctypes.c_char_p()
        ms = ctypes.c_float()
        call("rs_profile_read", i, ctypes.byref(name), ctypes.byref(ms))
        out.append((name.value.decode(), ms.value))
    return out
