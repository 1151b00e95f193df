"""FP64 CPU oracle for the tile-based Gaussian-splatting hot path (RadSplat, arXiv 2403.13806).

TEST INFRASTRUCTURE ONLY.  The tests, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` use it; the product library never imports it, and it imports
nothing from the product library.  The arithmetic lives in ``radsplat_oracle.c``
(plain C, FP64, no FMA contraction) and ``grad.py`` (PyTorch FP64 autograd on the CPU);
this module only marshals numpy arrays through ctypes.

Pinned functions (see tests/test_oracle_*.py): projection, the FP32 image mean, SH
basis, per-pixel compositing, importance, integer binning stages, filter and nearest
centre, the FP64
gradient, and (``optim.py``) the Adam step and the compaction of pruned parameters.
No function here is unpinned.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "radsplat_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lib = None

ALPHA_MAX = 0.99
ALPHA_MIN = 1.0 / 255.0
T_MIN = 1e-4
DEFAULT_AMB_REL = 1e-5


def build(force: bool = False) -> str:
    """Compile the C oracle into oracle/_build/liboracle.so (gcc, OpenMP)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-shared", "-fPIC",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB_PATH)
        P = ctypes.c_void_p
        i64, i32, f64, f32 = ctypes.c_int64, ctypes.c_int32, ctypes.c_double, ctypes.c_float
        L.or_project.argtypes = [i64, P, P, P, P, P, ctypes.c_int, P, P, ctypes.c_int, ctypes.c_int,
                                 f64, f32, ctypes.c_int, ctypes.c_int] + [P] * 9
        L.or_project.restype = ctypes.c_int
        L.or_render.argtypes = [i64, P, P, P, P, P, P, P, ctypes.c_int, ctypes.c_int, P, i64, P,
                                ctypes.c_int, f64, P, P, P, P, P, P, P, P, P, P, ctypes.c_int]
        L.or_render.restype = ctypes.c_int
        L.or_bin_sort.argtypes = [i64, P, P, P, P, P, i64, P, P]
        L.or_bin_sort.restype = i64
        L.or_tile_ranges.argtypes = [i64, P, i64, P]
        L.or_tile_ranges.restype = None
        L.or_filter.argtypes = [i64, P, f32, ctypes.c_int, P, P]
        L.or_filter.restype = i64
        L.or_nearest.argtypes = [i32, P, i32, P, P]
        L.or_nearest.restype = None
        L.or_mean2d_f32.argtypes = [i64, P, P, P, P]
        L.or_mean2d_f32.restype = None
        L.or_sh_basis.argtypes = [ctypes.c_int, P, P]
        L.or_sh_basis.restype = None
        _lib = L
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def sh_basis(degree: int, d) -> np.ndarray:
    """Real orthonormal SH Y_lm(d) (Condon-Shortley phase) from the Legendre recurrence."""
    d = _c(d, np.float64)
    y = np.zeros(16, dtype=np.float64)
    lib().or_sh_basis(degree, _p(d), _p(y))
    return y[: (degree + 1) ** 2]


def project(scene, cam, eps2d=0.3, near=0.2, tile=(16, 16)) -> dict:
    """FP64 projection of every Gaussian for one camera (Sec. 3.2)."""
    n = scene.n
    means, ls, q, lg, sh = (_c(a, np.float64) for a in scene.arrays())
    vm = _c(cam["viewmat"], np.float32).reshape(12)
    intr = np.array([cam["fx"], cam["fy"], cam["cx"], cam["cy"]], dtype=np.float32)
    out = {
        "xy": np.zeros((n, 2)), "conic": np.zeros((n, 3)), "cov2d": np.zeros((n, 3)),
        "opacity": np.zeros(n), "rgb": np.zeros((n, 3)), "depth": np.zeros(n, dtype=np.float32),
        "ext": np.zeros((n, 2)), "rect": np.zeros((n, 4), dtype=np.int32),
        "valid": np.zeros(n, dtype=np.int32),
    }
    rc = lib().or_project(n, _p(means), _p(ls), _p(q), _p(lg), _p(sh), scene.sh_degree, _p(vm), _p(intr),
                          cam["width"], cam["height"], float(eps2d), np.float32(near),
                          tile[0], tile[1], _p(out["xy"]), _p(out["conic"]), _p(out["cov2d"]),
                          _p(out["opacity"]), _p(out["rgb"]), _p(out["depth"]), _p(out["ext"]),
                          _p(out["rect"]), _p(out["valid"]))
    if rc != 0:
        raise ValueError("oracle projection rejected its arguments")
    out["n_tiles"] = ((out["rect"][:, 2] - out["rect"][:, 0]) * (out["rect"][:, 3] - out["rect"][:, 1])).astype(np.int64)
    out["xy32"] = mean2d_f32(scene, cam)
    out["width"], out["height"] = cam["width"], cam["height"]
    return out


def mean2d_f32(scene, cam) -> np.ndarray:
    """FP32 image means [N, 2] of single-precision arithmetic on the FP32 inputs (reading C5:
    fma chains for t = M p + m, correctly rounded t_x / t_z, then fmaf(f, u, c))."""
    n = scene.n
    means = _c(np.asarray(scene.arrays()[0], dtype=np.float32), np.float32)
    vm = _c(cam["viewmat"], np.float32).reshape(12)
    intr = np.array([cam["fx"], cam["fy"], cam["cx"], cam["cy"]], dtype=np.float32)
    out = np.zeros((n, 2), dtype=np.float32)
    lib().or_mean2d_f32(n, _p(means), _p(vm), _p(intr), _p(out))
    return out


def render(proj: dict, pixels=None, mode: str = "bucketed", bg=(0.0, 0.0, 0.0),
           amb_rel: float = DEFAULT_AMB_REL, h=None, h_amb=None, threads: int = 0, alt_mean: bool = True) -> dict:
    """Composite the given pixels (all if None) front to back, Eq. (render-gs).

    ``h`` / ``h_amb`` (float64[N]) accumulate the importance max of Eq.
    (importance-score) across calls; fresh zero arrays are used when None.
    A pixel is flagged ``ambiguous`` when one of its skip/stop decisions lies within a
    relative ``amb_rel`` of its threshold (reading C6), evaluated at the FP64 image mean
    and, with ``alt_mean`` and the projection's ``xy32``, also at the FP32 image mean a
    single-precision renderer uses (flagged too where the two fall on different sides).
    ``T_amb`` / ``c_amb``: transmittance in front of the first flagged decision and the
    largest colour behind it, whose product bounds how far two renderings that agree
    before that decision can differ (0 on unflagged pixels).
    """
    n = proj["xy"].shape[0]
    W, H = proj["width"], proj["height"]
    if pixels is None:
        npix, pix = W * H, None
    else:
        pix = _c(pixels, np.int32).reshape(-1, 2)
        npix = pix.shape[0]
    h = np.zeros(n) if h is None else h
    h_amb = np.zeros(n) if h_amb is None else h_amb
    assert h.dtype == np.float64 and h_amb.dtype == np.float64
    out = {"image": np.zeros((npix, 3)), "T_final": np.zeros(npix),
           "last_id": np.zeros(npix, dtype=np.int32), "n_contrib": np.zeros(npix, dtype=np.int32),
           "ambiguous": np.zeros(npix, dtype=np.uint8), "T_amb": np.zeros(npix), "c_amb": np.zeros(npix)}
    bgv = _c(bg, np.float64)
    xy_alt = None
    if alt_mean and "xy32" in proj:
        xy_alt = _c(proj["xy32"], np.float64)
    rc = lib().or_render(n, _p(proj["xy"]), _p(proj["conic"]), _p(proj["opacity"]), _p(proj["rgb"]),
                         _p(proj["depth"]), _p(proj["valid"]), _p(proj["ext"]), W, H, _p(bgv), npix,
                         None if pix is None else _p(pix), 1 if mode == "bucketed" else 0, float(amb_rel),
                         None if xy_alt is None else _p(xy_alt),
                         _p(out["image"]), _p(out["T_final"]), _p(out["last_id"]), _p(out["n_contrib"]),
                         _p(out["ambiguous"]), _p(out["T_amb"]), _p(out["c_amb"]), _p(h), _p(h_amb), int(threads))
    if rc != 0:
        raise MemoryError("oracle render ran out of memory")
    out["h"], out["h_amb"] = h, h_amb
    if pixels is None:
        out["image_chw"] = out["image"].reshape(H, W, 3).transpose(2, 0, 1)
    return out


def bin_sort(depth, rect, item_view, view_tiles_x, view_tile_base):
    """Integer-stage mirror: duplicated (tile|depth) keys, stable sort (keys, vals)."""
    depth = _c(depth, np.float32)
    rect = _c(rect, np.uint16).reshape(-1, 4)
    item_view = _c(item_view, np.int32)
    tx = _c(view_tiles_x, np.int32)
    tb = _c(view_tile_base, np.int32)
    m = depth.shape[0]
    K = lib().or_bin_sort(m, _p(depth), _p(rect), _p(item_view), _p(tx), _p(tb), 0, None, None)
    keys = np.zeros(max(K, 1), dtype=np.uint64)
    vals = np.zeros(max(K, 1), dtype=np.uint32)
    K2 = lib().or_bin_sort(m, _p(depth), _p(rect), _p(item_view), _p(tx), _p(tb), K, _p(keys), _p(vals))
    assert K2 == K
    return keys[:K], vals[:K]


def tile_ranges(keys, n_tiles: int) -> np.ndarray:
    keys = _c(keys, np.uint64)
    ranges = np.zeros((n_tiles, 2), dtype=np.uint32)
    lib().or_tile_ranges(keys.shape[0], _p(keys), n_tiles, _p(ranges))
    return ranges


PRUNE_BELOW, KEEP_ABOVE, PRUNE_KEEP = 0, 1, 2


def filter_mask(h, t: float, mode: int):
    """Sec. 3.3 (mode PRUNE_BELOW: h < t; PRUNE_KEEP: h >= t, the survivors) /
    Eq. (importance-score-vis) (KEEP_ABOVE: h > t)."""
    h = _c(h, np.float32)
    mask = np.zeros(h.shape[0], dtype=np.uint8)
    idx = np.zeros(h.shape[0], dtype=np.uint32)
    cnt = lib().or_filter(h.shape[0], _p(h), np.float32(t), mode, _p(mask), _p(idx))
    return mask, idx[:cnt]


def nearest(centres, cams) -> np.ndarray:
    """Sec. 3.4: index of the nearest cluster centre for each camera centre."""
    centres = _c(centres, np.float32).reshape(-1, 3)
    cams = _c(cams, np.float32).reshape(-1, 3)
    out = np.zeros(cams.shape[0], dtype=np.int32)
    lib().or_nearest(centres.shape[0], _p(centres), cams.shape[0], _p(cams), _p(out))
    return out


def importance(scene, cams, eps2d=0.3, near=0.2, mode="bucketed", threads=0):
    """Eq. (importance-score): max over the given views and all their pixels of alpha*T."""
    h = np.zeros(scene.n)
    h_amb = np.zeros(scene.n)
    for cam in cams:
        render(project(scene, cam, eps2d, near), mode=mode, h=h, h_amb=h_amb, threads=threads)
    return h, h_amb
