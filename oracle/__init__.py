"""CPU oracle for the 3-D segmentation stage -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path (the CUDA library and
its Python binding) never imports it, and the two share no code.

The arithmetic lives in ``seg_oracle.c`` (plain single-threaded C, built by
``oracle/build.py``); this module only marshals numpy arrays through ctypes.
Every function follows the paper's Segmentation section (Otsu thresholding,
connected components, minimum volume, closing, distance map, each cell's
voxels as label runs) and Background
Noise Removal section (Eq. 1, Gaussian low-pass read as binomial smoothing;
the stem-cell denoise front end; the MRF vessel denoise of Eqs. 2-3); see
the C file for the exact readings.

Parity status: every function is pinned by tests/test_oracle_pins.py against
brute force, closed forms, exact-rational Otsu and library routines.
"""
import ctypes
import os

import numpy as np

from . import build as _build

CELL_DTYPE = np.dtype([
    ("count", "<u8"),
    ("sum", "<i8", (3,)),
    ("bbox_min", "<u4", (3,)),
    ("bbox_max", "<u4", (3,)),
    ("pad", "<u4", (2,)),
])
assert CELL_DTYPE.itemsize == 64

_lib = None


def _load():
    global _lib
    if _lib is None:
        path = _build.build()
        lib = ctypes.CDLL(path)
        u16p = ctypes.POINTER(ctypes.c_uint16)
        u32p = ctypes.POINTER(ctypes.c_uint32)
        u64p = ctypes.POINTER(ctypes.c_uint64)
        u8p = ctypes.POINTER(ctypes.c_uint8)
        vp = ctypes.c_void_p
        lib.oracle_smooth.argtypes = [u16p, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32, u16p]
        lib.oracle_smooth.restype = ctypes.c_int
        lib.oracle_histogram.argtypes = [u16p, ctypes.c_uint64, u64p]
        lib.oracle_histogram.restype = ctypes.c_int
        lib.oracle_otsu.argtypes = [u64p]
        lib.oracle_otsu.restype = ctypes.c_uint16
        lib.oracle_label26.argtypes = [u8p, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32, u32p]
        lib.oracle_label26.restype = ctypes.c_int64
        lib.oracle_filter_features.argtypes = [u32p, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                                               ctypes.c_uint32, ctypes.c_uint32, u32p, vp,
                                               ctypes.c_uint64, u64p]
        lib.oracle_filter_features.restype = ctypes.c_int
        lib.oracle_segment.argtypes = [u16p, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32,
                                       ctypes.c_uint32, ctypes.c_uint32, u32p, vp, ctypes.c_uint64, u64p,
                                       u16p, u64p, u16p]
        lib.oracle_segment.restype = ctypes.c_int
        for name in ("oracle_background", "oracle_denoise"):
            getattr(lib, name).argtypes = [u16p, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32,
                                           ctypes.c_uint32, u16p]
            getattr(lib, name).restype = ctypes.c_int
        lib.oracle_box_pass.argtypes = [u16p, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32,
                                        ctypes.c_int, ctypes.c_uint32, u16p]
        lib.oracle_box_pass.restype = ctypes.c_int
        lib.oracle_median27.argtypes = [u16p, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32, u16p]
        lib.oracle_median27.restype = ctypes.c_int
        lib.oracle_close.argtypes = [u8p, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32, u8p]
        lib.oracle_close.restype = ctypes.c_int
        lib.oracle_distance.argtypes = [u8p, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32,
                                        ctypes.c_uint32, ctypes.c_uint32, u32p]
        lib.oracle_distance.restype = ctypes.c_int
        lib.oracle_mrf_delta.argtypes = [u16p, ctypes.c_uint64]
        lib.oracle_mrf_delta.restype = ctypes.c_uint32
        lib.oracle_mrf_laplacian.argtypes = [u16p, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32, u64p]
        lib.oracle_mrf_laplacian.restype = ctypes.c_uint64
        lib.oracle_mrf_limit.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64]
        lib.oracle_mrf_limit.restype = ctypes.c_double
        lib.oracle_mrf_step.argtypes = [u16p, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32,
                                        u16p]
        lib.oracle_mrf_step.restype = ctypes.c_int
        lib.oracle_mrf.argtypes = [u16p, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32, u16p,
                                   u32p]
        lib.oracle_mrf.restype = ctypes.c_int
        lib.oracle_cell_distance.argtypes = [u32p, u32p, ctypes.c_uint64, ctypes.c_uint64, u32p]
        lib.oracle_cell_distance.restype = ctypes.c_int
        lib.oracle_label_runs.argtypes = [u32p, ctypes.c_uint32, ctypes.c_uint64, vp, ctypes.c_uint64, u64p]
        lib.oracle_label_runs.restype = ctypes.c_int
        i32p = ctypes.POINTER(ctypes.c_int32)
        lib.oracle_reg_sums.argtypes = [u16p, u16p, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32, i32p, u64p]
        lib.oracle_reg_sums.restype = None
        lib.oracle_normcov.argtypes = [u64p, ctypes.POINTER(ctypes.c_int)]
        lib.oracle_normcov.restype = ctypes.c_double
        lib.oracle_register.argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.c_uint32, ctypes.c_uint32,
                                        ctypes.c_uint32, ctypes.c_uint32, i32p, i32p, ctypes.c_uint32, i32p, vp,
                                        ctypes.c_uint32, u32p]
        lib.oracle_register.restype = ctypes.c_int
        _lib = lib
    return _lib


def _ptr(a, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct))


def _dims(vol):
    if vol.ndim != 3:
        raise ValueError("volume must be [Z][Y][X]")
    Z, Y, X = vol.shape
    return int(X), int(Y), int(Z)


def smooth(vol: np.ndarray) -> np.ndarray:
    """Binomial smoothing, uint16 [Z,Y,X] -> uint16 [Z,Y,X] (Eq. 1 low-pass)."""
    vol = np.ascontiguousarray(vol, dtype=np.uint16)
    X, Y, Z = _dims(vol)
    out = np.empty_like(vol)
    rc = _load().oracle_smooth(_ptr(vol, ctypes.c_uint16), X, Y, Z, _ptr(out, ctypes.c_uint16))
    if rc:
        raise RuntimeError("oracle_smooth failed: %d" % rc)
    return out


def histogram(s: np.ndarray) -> np.ndarray:
    """65536-bin uint64 histogram of a uint16 array."""
    s = np.ascontiguousarray(s, dtype=np.uint16)
    h = np.zeros(65536, dtype=np.uint64)
    rc = _load().oracle_histogram(_ptr(s, ctypes.c_uint16), s.size, _ptr(h, ctypes.c_uint64))
    if rc:
        raise RuntimeError("oracle_histogram failed: %d" % rc)
    return h


def otsu(h: np.ndarray) -> int:
    """Otsu level t* of a 65536-bin histogram (foreground is s > t*)."""
    h = np.ascontiguousarray(h, dtype=np.uint64)
    if h.shape != (65536,):
        raise ValueError("histogram must have 65536 bins")
    return int(_load().oracle_otsu(_ptr(h, ctypes.c_uint64)))


def label26(mask: np.ndarray):
    """26-connected labelling; returns (uint32 labels [Z,Y,X], n_components)."""
    m = np.ascontiguousarray(mask, dtype=np.uint8)
    X, Y, Z = _dims(m)
    lab = np.empty(m.shape, dtype=np.uint32)
    n = _load().oracle_label26(_ptr(m, ctypes.c_uint8), X, Y, Z, _ptr(lab, ctypes.c_uint32))
    if n < 0:
        raise RuntimeError("oracle_label26 failed: %d" % n)
    return lab, int(n)


def filter_features(prov: np.ndarray, ncomp: int, min_volume: int):
    """Minimum-volume filter + canonical numbering + features.

    Returns (labels uint32 [Z,Y,X], cells structured array of CELL_DTYPE)."""
    prov = np.ascontiguousarray(prov, dtype=np.uint32)
    X, Y, Z = _dims(prov)
    lab = np.empty_like(prov)
    cap = max(int(ncomp), 1)
    cells = np.zeros(cap, dtype=CELL_DTYPE)
    k = np.zeros(1, dtype=np.uint64)
    rc = _load().oracle_filter_features(_ptr(prov, ctypes.c_uint32), ncomp, X, Y, Z, min_volume,
                                        _ptr(lab, ctypes.c_uint32), cells.ctypes.data, cap,
                                        _ptr(k, ctypes.c_uint64))
    if rc:
        raise RuntimeError("oracle_filter_features failed: %d" % rc)
    return lab, cells[: int(k[0])].copy()


class OracleResult:
    __slots__ = ("labels", "cells", "threshold", "hist", "smoothed", "distance", "denoised", "mrf_steps")

    def __init__(self, labels, cells, threshold, hist, smoothed, distance=None):
        self.labels = labels
        self.cells = cells
        self.threshold = threshold
        self.hist = hist
        self.smoothed = smoothed
        self.distance = distance
        self.denoised = None
        self.mrf_steps = None

    @property
    def n_cells(self):
        return len(self.cells)


def _vol_op(name, vol, *args):
    vol = np.ascontiguousarray(vol, dtype=np.uint16)
    X, Y, Z = _dims(vol)
    out = np.empty_like(vol)
    rc = getattr(_load(), name)(_ptr(vol, ctypes.c_uint16), X, Y, Z, *args, _ptr(out, ctypes.c_uint16))
    if rc:
        raise RuntimeError("%s failed: %d" % (name, rc))
    return out


def box_pass(vol: np.ndarray, axis: int, r: int) -> np.ndarray:
    """One rounded box pass of radius r along axis 0 = x, 1 = y, 2 = z."""
    return _vol_op("oracle_box_pass", vol, int(axis), int(r))


def background(vol: np.ndarray, r: int) -> np.ndarray:
    """Background estimate of the denoise front end (Eq. 1): 3 box passes per axis."""
    return _vol_op("oracle_background", vol, int(r))


def median27(vol: np.ndarray) -> np.ndarray:
    """3x3x3 median with replicate edges."""
    return _vol_op("oracle_median27", vol)


def denoise(vol: np.ndarray, r: int) -> np.ndarray:
    """Denoised stem-cell image: median27(max(vol - background(vol, r), 0))."""
    return _vol_op("oracle_denoise", vol, int(r))


def close(mask: np.ndarray, rho: int) -> np.ndarray:
    """Closing of a boolean [Z,Y,X] mask with the ball of radius rho (padded)."""
    m = np.ascontiguousarray(mask, dtype=np.uint8)
    X, Y, Z = _dims(m)
    out = np.empty_like(m)
    rc = _load().oracle_close(_ptr(m, ctypes.c_uint8), X, Y, Z, int(rho), _ptr(out, ctypes.c_uint8))
    if rc:
        raise RuntimeError("oracle_close failed: %d" % rc)
    return out.astype(bool)


def distance(mask: np.ndarray, weights=(16, 16, 25)) -> np.ndarray:
    """Weighted squared distance (wx dx^2 + wy dy^2 + wz dz^2) of every voxel
    of a boolean [Z,Y,X] mask to its nearest foreground voxel (brute force;
    0xFFFFFFFF when there is no foreground)."""
    m = np.ascontiguousarray(mask, dtype=np.uint8)
    X, Y, Z = _dims(m)
    out = np.empty(m.shape, dtype=np.uint32)
    rc = _load().oracle_distance(_ptr(m, ctypes.c_uint8), X, Y, Z, int(weights[0]), int(weights[1]),
                                 int(weights[2]), _ptr(out, ctypes.c_uint32))
    if rc:
        raise RuntimeError("oracle_distance failed: %d" % rc)
    return out


def distance_at(mask: np.ndarray, points, weights=(16, 16, 25)) -> np.ndarray:
    """The same weighted squared distance, evaluated only at the given
    (z, y, x) points: for each, the minimum over all foreground voxels
    (brute force; 0xFFFFFFFF when there is no foreground)."""
    fz, fy, fx = (a.astype(np.int64) for a in np.nonzero(mask))
    wx, wy, wz = (int(w) for w in weights)
    out = np.empty(len(points), dtype=np.uint32)
    for i, (z, y, x) in enumerate(points):
        if len(fx) == 0:
            out[i] = 0xFFFFFFFF
            continue
        d = wx * (fx - int(x)) ** 2 + wy * (fy - int(y)) ** 2 + wz * (fz - int(z)) ** 2
        out[i] = int(d.min())
    return out


def mrf_delta(vol: np.ndarray) -> int:
    """Delta of Eq. 3: the smallest gap between two distinct voxel values (0: fewer than two)."""
    vol = np.ascontiguousarray(vol, dtype=np.uint16)
    return int(_load().oracle_mrf_delta(_ptr(vol, ctypes.c_uint16), vol.size))


def mrf_laplacian(vol: np.ndarray):
    """(S, M) of the noise estimate: the summed absolute response of the
    per-plane mask [1 -2 1; -2 4 -2; 1 -2 1] over plane interiors, and M,
    the number of interior voxels."""
    vol = np.ascontiguousarray(vol, dtype=np.uint16)
    X, Y, Z = _dims(vol)
    m = np.zeros(1, dtype=np.uint64)
    s = _load().oracle_mrf_laplacian(_ptr(vol, ctypes.c_uint16), X, Y, Z, _ptr(m, ctypes.c_uint64))
    return int(s), int(m[0])


def mrf_limit(s: int, m: int, n: int) -> float:
    """N sigma^2, sigma = sqrt(pi / 2) S / (6 M): the bound of Eq. 2 on the summed squares."""
    return float(_load().oracle_mrf_limit(int(s), int(m), int(n)))


def mrf_step(vol: np.ndarray, delta: int) -> np.ndarray:
    """One step of Eq. 3 (six neighbour sign votes, step delta, clamped)."""
    return _vol_op("oracle_mrf_step", vol, int(delta))


def mrf(vol: np.ndarray, max_iter: int):
    """The MRF vessel denoise of Eqs. 2-3: (denoised image, steps kept)."""
    vol = np.ascontiguousarray(vol, dtype=np.uint16)
    X, Y, Z = _dims(vol)
    out = np.empty_like(vol)
    it = np.zeros(1, dtype=np.uint32)
    rc = _load().oracle_mrf(_ptr(vol, ctypes.c_uint16), X, Y, Z, int(max_iter), _ptr(out, ctypes.c_uint16),
                            _ptr(it, ctypes.c_uint32))
    if rc:
        raise RuntimeError("oracle_mrf failed: %d" % rc)
    return out, int(it[0])


def cell_distance(labels: np.ndarray, dmap: np.ndarray, k: int) -> np.ndarray:
    """Per cell 1..k of `labels`, the smallest value of `dmap` over its voxels
    (the cell's distance to the nearest vessel when dmap is the vessel
    channel's distance map)."""
    lab = np.ascontiguousarray(labels, dtype=np.uint32)
    m = np.ascontiguousarray(dmap, dtype=np.uint32)
    if lab.shape != m.shape:
        raise ValueError("labels and map differ in shape")
    out = np.empty(max(int(k), 1), dtype=np.uint32)
    rc = _load().oracle_cell_distance(_ptr(lab, ctypes.c_uint32), _ptr(m, ctypes.c_uint32), lab.size, int(k),
                                      _ptr(out, ctypes.c_uint32))
    if rc:
        raise RuntimeError("oracle_cell_distance failed: %d" % rc)
    return out[: int(k)]


RUN_DTYPE = np.dtype([("label", "<u4"), ("row", "<u4"), ("x_begin", "<u2"), ("x_end", "<u2")])
assert RUN_DTYPE.itemsize == 12


def label_runs(labels: np.ndarray) -> np.ndarray:
    """Each cell's voxels (the set the Segmentation section hands to the
    convex hull step) as runs: the maximal stretches of equal non-zero label
    along x in one row (row = y + Y z), in order of row and x; a structured
    array of RUN_DTYPE (label, row, first x, last x inclusive)."""
    lab = np.ascontiguousarray(labels, dtype=np.uint32)
    X = lab.shape[-1] if lab.ndim else 1
    rows = lab.size // X if X else 0
    n = np.zeros(1, dtype=np.uint64)
    lib = _load()
    rc = lib.oracle_label_runs(_ptr(lab, ctypes.c_uint32), X, rows, None, 0, _ptr(n, ctypes.c_uint64))
    out = np.zeros(int(n[0]), dtype=RUN_DTYPE)
    if len(out):
        rc = lib.oracle_label_runs(_ptr(lab, ctypes.c_uint32), X, rows, ctypes.c_void_p(out.ctypes.data),
                                   len(out), _ptr(n, ctypes.c_uint64))
        if rc:
            raise RuntimeError("oracle_label_runs failed: %d" % rc)
    return out


EDGE_DTYPE = np.dtype([("a", "<u4"), ("b", "<u4"), ("shift", "<i4", (3,)), ("pad0", "<u4"),
                       ("score", "<f8"), ("in_tree", "<u4"), ("pad1", "<u4")])
assert EDGE_DTYPE.itemsize == 40


def reg_sums(A: np.ndarray, B: np.ndarray, d) -> np.ndarray:
    """(N, Sa, Sb, Saa, Sbb, Sab) over the voxels tile A (origin 0) shares with
    tile B placed at origin d = (dx, dy, dz) in A's coordinates."""
    A = np.ascontiguousarray(A, dtype=np.uint16)
    B = np.ascontiguousarray(B, dtype=np.uint16)
    X, Y, Z = _dims(A)
    dd = np.array(d, dtype=np.int32)
    out = np.zeros(6, dtype=np.uint64)
    _load().oracle_reg_sums(_ptr(A, ctypes.c_uint16), _ptr(B, ctypes.c_uint16), X, Y, Z,
                            _ptr(dd, ctypes.c_int32), _ptr(out, ctypes.c_uint64))
    return out


def normcov(sums):
    """Eq. 4 (Pearson correlation) from the six sums; None when undefined."""
    s = np.ascontiguousarray(sums, dtype=np.uint64)
    ok = ctypes.c_int()
    r = _load().oracle_normcov(_ptr(s, ctypes.c_uint64), ctypes.byref(ok))
    return float(r) if ok.value else None


def register(tiles, stage, radius, root=0):
    """Montage registration: (delta [n, 3] int32, edges structured array)."""
    tiles = [np.ascontiguousarray(t, dtype=np.uint16) for t in tiles]
    X, Y, Z = _dims(tiles[0])
    n = len(tiles)
    ptrs = (ctypes.c_void_p * n)(*[t.ctypes.data for t in tiles])
    st = np.ascontiguousarray(stage, dtype=np.int32).reshape(n, 3)
    rad = np.ascontiguousarray(radius, dtype=np.int32)
    delta = np.zeros((n, 3), dtype=np.int32)
    cap = n * (n - 1) // 2
    edges = np.zeros(max(cap, 1), dtype=EDGE_DTYPE)
    ne = np.zeros(1, dtype=np.uint32)
    rc = _load().oracle_register(ptrs, n, X, Y, Z, _ptr(st, ctypes.c_int32), _ptr(rad, ctypes.c_int32),
                                 int(root), _ptr(delta, ctypes.c_int32), edges.ctypes.data, cap,
                                 _ptr(ne, ctypes.c_uint32))
    if rc:
        raise RuntimeError("oracle_register failed: %d" % rc)
    return delta, edges[: int(ne[0])].copy()


def segment(vol: np.ndarray, min_volume: int = 30, keep_hist: bool = False,
            keep_smoothed: bool = False, denoise_radius: int = 0, closing_radius: int = 0,
            distance_weights=None, mrf_iterations: int = 0) -> OracleResult:
    """The whole stage for one frame and channel (uint16 [Z,Y,X]); with
    denoise_radius > 0 the denoise front end runs first, with mrf_iterations
    > 0 the MRF vessel denoise (at most that many steps), with closing_radius
    > 0 the foreground is closed with that ball before labelling, and with
    distance_weights the distance map of the (closed) foreground is added."""
    if mrf_iterations:
        den, it = mrf(vol, mrf_iterations)
        r = segment(den, min_volume, keep_hist, keep_smoothed, denoise_radius, closing_radius, distance_weights)
        r.denoised, r.mrf_steps = den, it
        return r
    if distance_weights is not None:
        r = segment(vol, min_volume, keep_hist, True, denoise_radius, closing_radius)
        fg = r.smoothed > r.threshold
        if closing_radius:
            fg = close(fg, closing_radius)
        r.distance = distance(fg, distance_weights)
        if not keep_smoothed:
            r.smoothed = None
        return r
    vol = np.ascontiguousarray(vol, dtype=np.uint16)
    if denoise_radius:
        vol = denoise(vol, denoise_radius)
    X, Y, Z = _dims(vol)
    n = vol.size
    labels = np.empty(vol.shape, dtype=np.uint32)
    # K can not exceed the number of components; each keeps >= 1 voxel and,
    # being 26-separated, components are at most ceil(X/2)ceil(Y/2)ceil(Z/2).
    cap = ((X + 1) // 2) * ((Y + 1) // 2) * ((Z + 1) // 2)
    if min_volume > 1:
        cap = min(cap, n // min_volume + 1)
    cells = np.zeros(max(cap, 1), dtype=CELL_DTYPE)
    k = np.zeros(1, dtype=np.uint64)
    t = np.zeros(1, dtype=np.uint16)
    hist = np.zeros(65536, dtype=np.uint64) if keep_hist else None
    sm = np.empty_like(vol) if keep_smoothed else None
    rc = _load().oracle_segment(
        _ptr(vol, ctypes.c_uint16), X, Y, Z, int(min_volume), int(closing_radius), _ptr(labels, ctypes.c_uint32),
        cells.ctypes.data, len(cells), _ptr(k, ctypes.c_uint64), _ptr(t, ctypes.c_uint16),
        _ptr(hist, ctypes.c_uint64) if hist is not None else None,
        _ptr(sm, ctypes.c_uint16) if sm is not None else None)
    if rc:
        raise RuntimeError("oracle_segment failed: %d" % rc)
    return OracleResult(labels, cells[: int(k[0])].copy(), int(t[0]), hist, sm)
