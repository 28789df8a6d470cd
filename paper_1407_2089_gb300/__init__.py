"""Python binding of libseg (include/seg.h): argument marshalling only.

Every step of the segmentation runs in the library's CUDA kernels; this module
loads ``libseg.so`` from this directory with ctypes and exposes the C entry
points under the same names.  There is no fallback: if the library is missing
or cannot be loaded, importing the binding raises.

Inputs may be numpy arrays (host) or torch CUDA tensors (device, passed by
data_ptr); torch is used only for device memory and streams.
"""
import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libseg.so")

SEG_OK = 0
SEG_EINVAL = -1
SEG_ETOOBIG = -2
SEG_EAGAIN = -3
SEG_ENOTREADY = -4
SEG_ETIMEOUT = -5
SEG_ECUDA = -6
SEG_ESMALL = -7
SEG_ENOENT = -8
SEG_EFAILED = -9
SEG_MAX_YZ = 2147483583

SEG_PENDING = 0
SEG_DONE = 1
SEG_FAILED = 2

SEG_FORCE_TILE = 0x1
SEG_PLAIN = 0x2
SEG_NO_GRAPH = 0x4
SEG_PROFILE = 0x8
SEG_TEST_UNION_FAIL = 0x10
SEG_KEEP_SMOOTHED = 0x20

SEG_MAX_KERNELS = 32
SEG_REG_MAX_RXY = 12
SEG_REG_MAX_RZ = 6


class seg_dims(ctypes.Structure):
    _fields_ = [("x", ctypes.c_uint32), ("y", ctypes.c_uint32), ("z", ctypes.c_uint32)]


class seg_cell_features(ctypes.Structure):
    _fields_ = [("count", ctypes.c_uint64), ("sum", ctypes.c_int64 * 3),
                ("bbox_min", ctypes.c_uint32 * 3), ("bbox_max", ctypes.c_uint32 * 3),
                ("pad", ctypes.c_uint32 * 2)]


FEATURE_DTYPE = np.dtype([
    ("count", "<u8"), ("sum", "<i8", (3,)), ("bbox_min", "<u4", (3,)),
    ("bbox_max", "<u4", (3,)), ("pad", "<u4", (2,))])
assert FEATURE_DTYPE.itemsize == ctypes.sizeof(seg_cell_features) == 64


class seg_config(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int), ("hbm_budget_bytes", ctypes.c_uint64),
                ("max_inflight", ctypes.c_uint32), ("flags", ctypes.c_uint32),
                ("tile_y", ctypes.c_uint32), ("tile_z", ctypes.c_uint32),
                ("max_batch_volumes", ctypes.c_uint32), ("batch_window_us", ctypes.c_uint32),
                ("host_queue", ctypes.c_uint32), ("order_stream", ctypes.c_void_p)]


class seg_channel_params(ctypes.Structure):
    _fields_ = [("min_volume_voxels", ctypes.c_uint32), ("denoise_radius", ctypes.c_uint32),
                ("closing_radius", ctypes.c_uint32), ("distance_weights", ctypes.c_uint32 * 3),
                ("mrf_iterations", ctypes.c_uint32)]


class seg_offset(ctypes.Structure):
    _fields_ = [("x", ctypes.c_int32), ("y", ctypes.c_int32), ("z", ctypes.c_int32)]


MONTAGE_EDGE_DTYPE = np.dtype([("a", "<u4"), ("b", "<u4"), ("shift", "<i4", (3,)), ("pad0", "<u4"),
                               ("score", "<f8"), ("in_tree", "<u4"), ("pad1", "<u4")])


LABEL_RUN_DTYPE = np.dtype([("label", "<u4"), ("row", "<u4"), ("x_begin", "<u2"), ("x_end", "<u2")])
assert LABEL_RUN_DTYPE.itemsize == 12


class seg_stats(ctypes.Structure):
    _fields_ = [("batches", ctypes.c_uint64), ("volumes", ctypes.c_uint64),
                ("voxels", ctypes.c_uint64), ("tile_y", ctypes.c_uint32),
                ("tile_z", ctypes.c_uint32), ("n_kernels", ctypes.c_uint32),
                ("names", (ctypes.c_char * 32) * SEG_MAX_KERNELS),
                ("launches", ctypes.c_uint64 * SEG_MAX_KERNELS),
                ("total_ms", ctypes.c_double * SEG_MAX_KERNELS),
                ("bytes_in_use", ctypes.c_uint64), ("budget_bytes", ctypes.c_uint64)]


EXPORTS = ["seg_create", "seg_destroy", "seg_submit_volume", "seg_flush", "seg_poll",
           "seg_enqueue_wait", "seg_read_labels", "seg_read_label_runs", "seg_read_distance", "seg_read_cell_distance", "seg_read_denoised",
           "seg_read_smoothed", "seg_read_features", "seg_release",
           "seg_request_times", "seg_get_stats", "seg_reset_stats", "seg_strerror",
           "seg_otsu_threshold_noalloc", "seg_register_montage"]


def _bind(lib):
    vp, u32, u64, i32 = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int
    P = ctypes.POINTER
    sig = {
        "seg_create": [P(seg_config), P(vp)],
        "seg_destroy": [vp],
        "seg_submit_volume": [vp, vp, i32, seg_dims, u32, P(seg_channel_params), P(u64)],
        "seg_flush": [vp],
        "seg_poll": [vp, u64, u32, P(i32)],
        "seg_enqueue_wait": [vp, u64, vp],
        "seg_read_labels": [vp, u64, u32, vp, u64, i32],
        "seg_read_label_runs": [vp, u64, u32, vp, u64, P(u64), i32],
        "seg_read_distance": [vp, u64, u32, vp, u64, i32],
        "seg_read_cell_distance": [vp, u64, u32, u32, vp, u64, P(u64)],
        "seg_read_denoised": [vp, u64, u32, vp, u64, i32, P(u32)],
        "seg_read_smoothed": [vp, u64, u32, vp, u64, i32],
        "seg_read_features": [vp, u64, u32, vp, u64, P(u64), P(ctypes.c_uint16)],
        "seg_release": [vp, u64],
        "seg_request_times": [vp, u64, P(ctypes.c_double), P(ctypes.c_double),
                              P(ctypes.c_double), P(ctypes.c_double)],
        "seg_get_stats": [vp, P(seg_stats)],
        "seg_reset_stats": [vp],
        "seg_otsu_threshold_noalloc": [vp, seg_dims, vp, vp],
        "seg_register_montage": [i32, P(vp), i32, u32, seg_dims, P(seg_offset), seg_offset, u32, P(seg_offset),
                                 vp, u32, P(u32)],
    }
    for name, args in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = ctypes.c_int
    lib.seg_strerror.argtypes = [ctypes.c_int]
    lib.seg_strerror.restype = ctypes.c_char_p
    return lib


def load_library(path: str = LIB_PATH):
    if not os.path.exists(path):
        raise ImportError("libseg.so not built (run __graft_entry__.build() or "
                          "python paper_1407_2089_gb300/build.py): %s" % path)
    return _bind(ctypes.CDLL(path))


_lib = load_library()


class SegError(RuntimeError):
    def __init__(self, code, what):
        super().__init__("%s: %s (%d)" % (what, _lib.seg_strerror(code).decode(), code))
        self.code = code


def _check(rc, what):
    if rc != SEG_OK:
        raise SegError(rc, what)
    return rc


def seg_strerror(code: int) -> str:
    return _lib.seg_strerror(code).decode()


def seg_create(device=0, max_inflight=0, hbm_budget_bytes=0, flags=0, tile_y=0, tile_z=0,
               max_batch_volumes=0, batch_window_us=0, host_queue=0, order_stream=None):
    """Returns an opaque context handle (int)."""
    cfg = seg_config(device, hbm_budget_bytes, max_inflight, flags, tile_y, tile_z,
                     max_batch_volumes, batch_window_us, host_queue,
                     ctypes.c_void_p(order_stream) if order_stream else None)
    out = ctypes.c_void_p()
    _check(_lib.seg_create(ctypes.byref(cfg), ctypes.byref(out)), "seg_create")
    return out.value


def seg_destroy(ctx):
    _check(_lib.seg_destroy(ctx), "seg_destroy")


def _voxel_ptr(voxels):
    """(pointer, on_device, dims) for a numpy array or a torch CUDA tensor."""
    if isinstance(voxels, np.ndarray):
        if voxels.dtype != np.uint16 or not voxels.flags["C_CONTIGUOUS"]:
            raise ValueError("voxels must be C-contiguous uint16")
        return voxels.ctypes.data, 0
    # torch tensor (host or device)
    if str(voxels.dtype) != "torch.uint16" and str(voxels.dtype) != "torch.int16":
        raise ValueError("voxels must be a uint16 (or int16-viewed) tensor")
    if not voxels.is_contiguous():
        raise ValueError("voxels must be contiguous")
    return voxels.data_ptr(), 1 if voxels.is_cuda else 0


def seg_submit_volume(ctx, voxels, dims=None, channels=None, min_volume=30, denoise_radius=0, closing_radius=0,
                      distance_weights=None, mrf_iterations=0, keep_host_input=False):
    """Submits [C][Z][Y][X] (or [Z][Y][X]) uint16 voxels; returns the request id.

    min_volume, denoise_radius, closing_radius: one int for every channel or
    a sequence of per-channel ints (0 = no denoise front end / no closing).
    distance_weights: None (no distance map), one (wx, wy, wz) for every
    channel, or a per-channel sequence of triples or None.  mrf_iterations:
    step limit of the MRF vessel denoise (0 = off), one int or per channel.
    keep_host_input: for a host input, only queue its copy; the caller then
    keeps it unchanged until the request is done (best with pinned memory)."""
    shape = tuple(voxels.shape)
    if dims is None:
        if len(shape) == 3:
            channels, (Z, Y, X) = 1, shape
        elif len(shape) == 4:
            channels, Z, Y, X = shape
        else:
            raise ValueError("voxels must be [Z][Y][X] or [C][Z][Y][X]")
        dims = (X, Y, Z)
    if channels is None:
        channels = 1
    ptr, on_dev = _voxel_ptr(voxels)
    if keep_host_input and not on_dev:
        on_dev = 2
    mv = [min_volume] * channels if np.isscalar(min_volume) else list(min_volume)
    dr = [denoise_radius] * channels if np.isscalar(denoise_radius) else list(denoise_radius)
    cr = [closing_radius] * channels if np.isscalar(closing_radius) else list(closing_radius)
    if distance_weights is None or (len(distance_weights) == 3 and np.isscalar(distance_weights[0])):
        dw = [distance_weights] * channels
    else:
        dw = list(distance_weights)
    dw = [(0, 0, 0) if w is None else tuple(int(a) for a in w) for w in dw]
    mi = [mrf_iterations] * channels if np.isscalar(mrf_iterations) else list(mrf_iterations)
    if any(len(a) != channels for a in (mv, dr, cr, dw, mi)):
        raise ValueError("per-channel parameter lists must have one entry per channel")
    params = (seg_channel_params * channels)(
        *[seg_channel_params(int(m), int(d), int(c), (ctypes.c_uint32 * 3)(*w), int(i))
          for m, d, c, w, i in zip(mv, dr, cr, dw, mi)])
    out = ctypes.c_uint64()
    _check(_lib.seg_submit_volume(ctx, ctypes.c_void_p(ptr), on_dev, seg_dims(*dims), channels,
                                  params, ctypes.byref(out)), "seg_submit_volume")
    return out.value


def seg_flush(ctx):
    _check(_lib.seg_flush(ctx), "seg_flush")


def seg_poll(ctx, req, timeout_ms=0):
    """Returns SEG_PENDING, SEG_DONE or SEG_FAILED."""
    st = ctypes.c_int()
    rc = _lib.seg_poll(ctx, req, timeout_ms, ctypes.byref(st))
    if rc not in (SEG_OK, SEG_ETIMEOUT):
        _check(rc, "seg_poll")
    return st.value


def seg_wait(ctx, req, timeout_ms=600000):
    st = seg_poll(ctx, req, timeout_ms)
    if st == SEG_PENDING:
        raise SegError(SEG_ETIMEOUT, "seg_wait")
    return st


def seg_enqueue_wait(ctx, req, stream_ptr):
    _check(_lib.seg_enqueue_wait(ctx, req, ctypes.c_void_p(stream_ptr or None)), "seg_enqueue_wait")


def seg_read_labels(ctx, req, channel, out):
    """Copies labels into `out`: a numpy uint32 array or a torch CUDA int32/uint32 tensor."""
    if isinstance(out, np.ndarray):
        if out.dtype != np.uint32 or not out.flags["C_CONTIGUOUS"]:
            raise ValueError("out must be C-contiguous uint32")
        ptr, n, dev = out.ctypes.data, out.size, 0
    else:
        ptr, n, dev = out.data_ptr(), out.numel(), 1 if out.is_cuda else 0
    _check(_lib.seg_read_labels(ctx, req, channel, ctypes.c_void_p(ptr), n, dev), "seg_read_labels")
    return out


def seg_read_label_runs(ctx, req, channel, out=None):
    """The channel's label image as runs (LABEL_RUN_DTYPE: label, row =
    y + Y*z, first and last x), in order of row and x.

    out=None: a new numpy array (the runs are counted first, then read).
    out: a C-contiguous numpy array of LABEL_RUN_DTYPE, or a uint8 torch
    tensor (host or CUDA) of 12 bytes per run; returns out[:n] (numpy) or the
    first 12*n bytes (torch).  Raises SegError(SEG_ESMALL) when out is too
    small."""
    n = ctypes.c_uint64()
    if out is None:
        _check(_lib.seg_read_label_runs(ctx, req, channel, None, 0, ctypes.byref(n), 0), "seg_read_label_runs")
        out = np.zeros(n.value, dtype=LABEL_RUN_DTYPE)
        if not n.value:
            return out
    if isinstance(out, np.ndarray):
        if out.dtype != LABEL_RUN_DTYPE or not out.flags["C_CONTIGUOUS"]:
            raise ValueError("out must be a C-contiguous array of LABEL_RUN_DTYPE")
        ptr, cap, dev = out.ctypes.data, out.size, 0
    else:
        if out.element_size() != 1 or not out.is_contiguous():
            raise ValueError("out must be a contiguous uint8 tensor")
        ptr, cap, dev = out.data_ptr(), out.numel() // LABEL_RUN_DTYPE.itemsize, 1 if out.is_cuda else 0
    _check(_lib.seg_read_label_runs(ctx, req, channel, ctypes.c_void_p(ptr) if cap else None, cap,
                                    ctypes.byref(n), dev), "seg_read_label_runs")
    return out[: n.value] if isinstance(out, np.ndarray) else out[: n.value * LABEL_RUN_DTYPE.itemsize]


def seg_read_distance(ctx, req, channel, out):
    """Copies the channel's distance map into `out` (as seg_read_labels)."""
    if isinstance(out, np.ndarray):
        if out.dtype != np.uint32 or not out.flags["C_CONTIGUOUS"]:
            raise ValueError("out must be C-contiguous uint32")
        ptr, n, dev = out.ctypes.data, out.size, 0
    else:
        ptr, n, dev = out.data_ptr(), out.numel(), 1 if out.is_cuda else 0
    _check(_lib.seg_read_distance(ctx, req, channel, ctypes.c_void_p(ptr), n, dev), "seg_read_distance")
    return out


def seg_read_cell_distance(ctx, req, cells_channel, map_channel):
    """Per cell of cells_channel, its distance to the nearest foreground voxel
    of map_channel (a uint32 array of K weighted squared distances)."""
    k = ctypes.c_uint64()
    _check(_lib.seg_read_cell_distance(ctx, req, cells_channel, map_channel, None, 0, ctypes.byref(k)),
           "seg_read_cell_distance")
    out = np.zeros(k.value, dtype=np.uint32)
    if k.value:
        _check(_lib.seg_read_cell_distance(ctx, req, cells_channel, map_channel, ctypes.c_void_p(out.ctypes.data),
                                           k.value, ctypes.byref(k)), "seg_read_cell_distance")
    return out


def seg_read_denoised(ctx, req, channel, out):
    """Copies the channel's denoised image into `out` (a numpy uint16 array or
    a torch int16/uint16 tensor); returns the number of MRF steps kept."""
    if isinstance(out, np.ndarray):
        if out.dtype != np.uint16 or not out.flags["C_CONTIGUOUS"]:
            raise ValueError("out must be C-contiguous uint16")
        ptr, n, dev = out.ctypes.data, out.size, 0
    else:
        ptr, n, dev = out.data_ptr(), out.numel(), 1 if out.is_cuda else 0
    steps = ctypes.c_uint32()
    _check(_lib.seg_read_denoised(ctx, req, channel, ctypes.c_void_p(ptr), n, dev, ctypes.byref(steps)),
           "seg_read_denoised")
    return steps.value


def seg_read_smoothed(ctx, req, channel, out):
    """Copies the channel's smoothed image into `out` (a numpy uint16 array or
    a torch int16/uint16 tensor); the context needs SEG_KEEP_SMOOTHED."""
    if isinstance(out, np.ndarray):
        if out.dtype != np.uint16 or not out.flags["C_CONTIGUOUS"]:
            raise ValueError("out must be C-contiguous uint16")
        ptr, n, dev = out.ctypes.data, out.size, 0
    else:
        ptr, n, dev = out.data_ptr(), out.numel(), 1 if out.is_cuda else 0
    _check(_lib.seg_read_smoothed(ctx, req, channel, ctypes.c_void_p(ptr), n, dev), "seg_read_smoothed")
    return out


def seg_read_features(ctx, req, channel):
    """Returns (cells structured array of FEATURE_DTYPE, otsu threshold)."""
    n = ctypes.c_uint64()
    t = ctypes.c_uint16()
    _check(_lib.seg_read_features(ctx, req, channel, None, 0, ctypes.byref(n), ctypes.byref(t)),
           "seg_read_features")
    cells = np.zeros(n.value, dtype=FEATURE_DTYPE)
    if n.value:
        _check(_lib.seg_read_features(ctx, req, channel, ctypes.c_void_p(cells.ctypes.data), n.value,
                                      ctypes.byref(n), ctypes.byref(t)), "seg_read_features")
    return cells, int(t.value)


def seg_release(ctx, req):
    _check(_lib.seg_release(ctx, req), "seg_release")


def seg_request_times(ctx, req):
    v = [ctypes.c_double() for _ in range(4)]
    _check(_lib.seg_request_times(ctx, req, *[ctypes.byref(x) for x in v]), "seg_request_times")
    return tuple(x.value for x in v)


def seg_get_stats(ctx):
    s = seg_stats()
    _check(_lib.seg_get_stats(ctx, ctypes.byref(s)), "seg_get_stats")
    names = [s.names[k].value.decode() for k in range(s.n_kernels)]
    return {
        "batches": s.batches, "volumes": s.volumes, "voxels": s.voxels,
        "tile_y": s.tile_y, "tile_z": s.tile_z,
        "kernels": {names[k]: {"launches": s.launches[k], "ms": s.total_ms[k]}
                    for k in range(s.n_kernels)},
        "bytes_in_use": s.bytes_in_use, "budget_bytes": s.budget_bytes,
    }


def seg_reset_stats(ctx):
    _check(_lib.seg_reset_stats(ctx), "seg_reset_stats")


def seg_otsu_threshold_noalloc(voxels_ptr, dims, result_ptr, stream_ptr=None):
    """Allocation-free Otsu level of one device volume (see include/seg.h).

    voxels_ptr / result_ptr are device addresses (uint16 volume, 2 x uint32
    result); dims = (X, Y, Z).  Enqueues on stream_ptr and returns."""
    _check(_lib.seg_otsu_threshold_noalloc(ctypes.c_void_p(voxels_ptr), seg_dims(*dims),
                                           ctypes.c_void_p(result_ptr),
                                           ctypes.c_void_p(stream_ptr or None)),
           "seg_otsu_threshold_noalloc")


def segment(ctx, voxels, min_volume=30, labels_out=None, timeout_ms=600000, denoise_radius=0, closing_radius=0,
            distance_weights=None, mrf_iterations=0):
    """Convenience: submit one volume, wait, read labels + cells of every channel, release.

    Returns a list (one entry per channel) of (labels, cells, threshold), with
    the distance map (or None) as a fourth entry when distance_weights is given."""
    req = seg_submit_volume(ctx, voxels, min_volume=min_volume, denoise_radius=denoise_radius,
                            closing_radius=closing_radius, distance_weights=distance_weights,
                            mrf_iterations=mrf_iterations)
    seg_flush(ctx)
    try:
        st = seg_wait(ctx, req, timeout_ms)
        if st != SEG_DONE:
            raise SegError(SEG_EFAILED, "segment")
        shape = tuple(voxels.shape)
        C = 1 if len(shape) == 3 else shape[0]
        out = []
        for c in range(C):
            lab = np.empty(shape[-3:], dtype=np.uint32) if labels_out is None else labels_out[c]
            seg_read_labels(ctx, req, c, lab)
            cells, t = seg_read_features(ctx, req, c)
            if distance_weights is None:
                out.append((lab, cells, t))
                continue
            wc = distance_weights
            if not (len(wc) == 3 and np.isscalar(wc[0])):
                wc = wc[c]
            dist = None
            if wc is not None and any(wc):
                dist = np.empty(shape[-3:], dtype=np.uint32)
                seg_read_distance(ctx, req, c, dist)
            out.append((lab, cells, t, dist))
        return out
    finally:
        seg_release(ctx, req)


def seg_register_montage(tiles, stage, radius, root=0, device=0):
    """Registers the montage tiles (a list of equal-shape [Z][Y][X] uint16
    numpy arrays, or CUDA int16/uint16 tensors on `device`) placed at
    stage[i] = (x, y, z); radius = (rx, ry, rz) half-widths of the search.
    Returns (delta [n, 3] int32, edges structured array of MONTAGE_EDGE_DTYPE)."""
    n = len(tiles)
    if n == 0:
        raise ValueError("no tiles")
    on_dev = not isinstance(tiles[0], np.ndarray)
    keep = []
    ptrs = (ctypes.c_void_p * n)()
    for i, t in enumerate(tiles):
        if on_dev:
            if not t.is_cuda or not t.is_contiguous():
                raise ValueError("device tiles must be contiguous CUDA tensors")
            ptrs[i] = t.data_ptr()
        else:
            a = np.ascontiguousarray(t, dtype=np.uint16)
            keep.append(a)
            ptrs[i] = a.ctypes.data
    Z, Y, X = tuple(tiles[0].shape)
    st = (seg_offset * n)(*[seg_offset(int(p[0]), int(p[1]), int(p[2])) for p in stage])
    delta = (seg_offset * n)()
    cap = n * (n - 1) // 2
    edges = np.zeros(max(cap, 1), dtype=MONTAGE_EDGE_DTYPE)
    ne = ctypes.c_uint32()
    _check(_lib.seg_register_montage(int(device), ptrs, 1 if on_dev else 0, n, seg_dims(X, Y, Z), st,
                                     seg_offset(*[int(v) for v in radius]), int(root), delta,
                                     ctypes.c_void_p(edges.ctypes.data), cap, ctypes.byref(ne)),
           "seg_register_montage")
    d = np.array([[o.x, o.y, o.z] for o in delta], dtype=np.int32)
    return d, edges[: ne.value].copy()
