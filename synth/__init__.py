"""Seeded synthetic inputs shaped like the paper's workloads.

The paper's data (18 5-D SVZ sequences, the 34-tile montage; Methods and
Registration sections) are not available, so every test and benchmark input is
drawn here from a seed.  This module holds no segmentation arithmetic: it draws
noise and renders nuclei and vessels (``synth.c``), and it chooses shapes,
positions and motion (numpy ``Generator(PCG64(seed))``).

Workloads (all uint16, planar [Z][Y][X] per channel):
  * single frame    128x128x32, 1 channel, background N(200,20), 40 nuclei with
                    radii U[4,8], peak 1500, blur sigma 1.5, >= 3 voxels apart.
  * time-lapse      512x512x64, 60 frames x 2 channels, noise N(200,25);
                    ch0: 300 nuclei (radii U[4,9]) random-walking 2 voxels per
                    frame, 5 % dividing per frame; ch1: static vessels (cubic
                    spline centrelines, radius U[3,6], intensity 2000).
  * batched uneven  48 volumes, X=Y=round(exp U[ln 64, ln 1024]), Z in 64..96,
                    first 64^3 and last 1024x1024x96, 1 nucleus per 40^3 voxels.
  * montage         5530x5530x80 x 2 channels, 20,000 nuclei + vessels.
  * serving stream  Poisson arrivals (mean 200/s), X=Y=round(128*16^u),
                    Z=round(128*0.5^u), u ~ U[0,1], 2 channels, 1 nucleus per 40^3.
"""
import ctypes
import math
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(HERE, "synth.c")
_LIB = os.path.join(HERE, "libsynth.so")
_lib = None


def build(force: bool = False) -> str:
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + ".tmp%d" % os.getpid()
    subprocess.run(["gcc", "-O2", "-std=c99", "-fopenmp", "-fPIC", "-shared", _SRC, "-o", tmp,
                    "-lm"], check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        vp = ctypes.c_void_p
        u32, u64, i64, f64 = ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int64, ctypes.c_double
        lib.synth_background.argtypes = [vp, u64, u64, f64, f64]
        lib.synth_add_ellipsoids.argtypes = [vp, u32, u32, u32, i64, vp, f64]
        lib.synth_tube_field.argtypes = [vp, u32, u32, u32, i64, vp, f64]
        lib.synth_add_field.argtypes = [vp, vp, u64]
        for f in (lib.synth_background, lib.synth_add_ellipsoids, lib.synth_tube_field,
                  lib.synth_add_field):
            f.restype = None
        _lib = lib
    return _lib


def mix_seed(*parts) -> int:
    """64-bit seed from integers (splitmix-style mixing, pure Python)."""
    h = 0x243F6A8885A308D3
    for p in parts:
        h = (h ^ (int(p) & 0xFFFFFFFFFFFFFFFF)) & 0xFFFFFFFFFFFFFFFF
        h = (h + 0x9E3779B97F4A7C15) & 0xFFFFFFFFFFFFFFFF
        h = ((h ^ (h >> 30)) * 0xBF58476D1CE4E5B9) & 0xFFFFFFFFFFFFFFFF
        h = ((h ^ (h >> 27)) * 0x94D049BB133111EB) & 0xFFFFFFFFFFFFFFFF
        h ^= h >> 31
    return h


# --------------------------------------------------------------------------
# primitives
# --------------------------------------------------------------------------

def background(dims, seed, mean=200.0, sigma=20.0, out=None):
    """uint16 [Z,Y,X] Gaussian noise N(mean, sigma) rounded and clipped."""
    X, Y, Z = dims
    if out is None:
        out = np.empty((Z, Y, X), dtype=np.uint16)
    _load().synth_background(out.ctypes.data, out.size, seed & 0xFFFFFFFFFFFFFFFF, mean, sigma)
    return out


def render_nuclei(vol, nuclei, sigma=1.5):
    """Adds blurred ellipsoids; nuclei is (n, 7): cx, cy, cz, rx, ry, rz, peak."""
    nuclei = np.ascontiguousarray(nuclei, dtype=np.float64)
    Z, Y, X = vol.shape
    if len(nuclei):
        _load().synth_add_ellipsoids(vol.ctypes.data, X, Y, Z, len(nuclei), nuclei.ctypes.data,
                                     sigma)
    return vol


def tube_field(dims, segments, sigma=1.0):
    """uint16 [Z,Y,X] field of tubes; segments is (n, 8): p0, p1, radius, intensity."""
    X, Y, Z = dims
    segs = np.ascontiguousarray(segments, dtype=np.float64)
    f = np.empty((Z, Y, X), dtype=np.uint16)
    _load().synth_tube_field(f.ctypes.data, X, Y, Z, len(segs), segs.ctypes.data, sigma)
    return f


def add_field(vol, field):
    _load().synth_add_field(vol.ctypes.data, field.ctypes.data, vol.size)
    return vol


def place_nuclei(rng, dims, n, r_lo, r_hi, min_sep, peak=1500.0, margin=None, max_tries=200000):
    """Rejection-sampled nucleus centres with surface separation >= min_sep.

    Returns (k, 7) float64 rows (cx, cy, cz, rx, ry, rz, peak); k <= n when the
    volume is too crowded to place them all within max_tries draws."""
    X, Y, Z = dims
    cell = 2.0 * r_hi + min_sep
    grid = {}
    out = []
    tries = 0
    while len(out) < n and tries < max_tries:
        tries += 1
        r = rng.uniform(r_lo, r_hi, size=3)
        m = np.max(r) if margin is None else margin
        lo = np.array([m, m, min(m, (Z - 1) / 2.0)])
        hi = np.array([X - 1 - m, Y - 1 - m, max(Z - 1 - m, (Z - 1) / 2.0)])
        if np.any(hi < lo):
            break
        c = rng.uniform(lo, hi)
        key = tuple((c // cell).astype(int))
        ok = True
        for dz in (-1, 0, 1):
            for dy in (-1, 0, 1):
                for dx in (-1, 0, 1):
                    for j in grid.get((key[0] + dx, key[1] + dy, key[2] + dz), ()):
                        o = out[j]
                        if np.linalg.norm(c - o[:3]) < np.max(r) + np.max(o[3:6]) + min_sep:
                            ok = False
                            break
                    if not ok:
                        break
                if not ok:
                    break
            if not ok:
                break
        if ok:
            grid.setdefault(key, []).append(len(out))
            out.append(np.concatenate([c, r, [peak]]))
    return np.array(out, dtype=np.float64).reshape(-1, 7)


def spline_vessels(rng, dims, n_vessels, r_lo=3.0, r_hi=6.0, intensity=2000.0, step=1.0):
    """Tubes around Catmull-Rom centrelines crossing the volume.

    Returns (m, 8) segment rows for tube_field."""
    X, Y, Z = dims
    rows = []
    size = np.array([X - 1, Y - 1, Z - 1], dtype=np.float64)
    for _ in range(n_vessels):
        radius = rng.uniform(r_lo, r_hi)
        k = 5
        pts = rng.uniform(0.0, 1.0, size=(k, 3)) * size
        # enter and leave through opposite x or y faces
        axis = rng.integers(0, 2)
        pts[0, axis] = 0.0
        pts[-1, axis] = size[axis]
        pts[:, 2] = np.clip(pts[:, 2], radius, max(size[2] - radius, radius))
        ctrl = np.vstack([2 * pts[0] - pts[1], pts, 2 * pts[-1] - pts[-2]])
        samples = []
        for i in range(1, len(ctrl) - 2):
            p0, p1, p2, p3 = ctrl[i - 1], ctrl[i], ctrl[i + 1], ctrl[i + 2]
            seg_len = np.linalg.norm(p2 - p1)
            m = max(2, int(math.ceil(seg_len / step)))
            for t in np.linspace(0.0, 1.0, m, endpoint=False):
                t2, t3 = t * t, t * t * t
                samples.append(0.5 * ((2 * p1) + (-p0 + p2) * t + (2 * p0 - 5 * p1 + 4 * p2 - p3) * t2
                                      + (-p0 + 3 * p1 - 3 * p2 + p3) * t3))
        samples.append(ctrl[-2])
        s = np.array(samples)
        for a, b in zip(s[:-1], s[1:]):
            rows.append(np.concatenate([a, b, [radius, intensity]]))
    return np.array(rows, dtype=np.float64).reshape(-1, 8)


def nuclei_volume(dims, seed, n_nuclei, r_lo=4.0, r_hi=8.0, min_sep=3.0, peak=1500.0,
                  noise_mean=200.0, noise_sigma=20.0, blur=1.5):
    """One channel: noise + blurred ellipsoidal nuclei.  Returns (vol, nuclei)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    nuc = place_nuclei(rng, dims, n_nuclei, r_lo, r_hi, min_sep, peak)
    vol = background(dims, mix_seed(seed, 1), noise_mean, noise_sigma)
    render_nuclei(vol, nuc, blur)
    return vol, nuc


def well_separated(dims, seed, n_nuclei, r_lo=4.0, r_hi=6.0):
    """Nuclei at >= 8 voxels surface separation, fully inside, noise sigma 20.

    Used for the whole-pipeline pin: every planted nucleus is one cell."""
    margin = r_hi + 4.0
    rng = np.random.Generator(np.random.PCG64(seed))
    nuc = place_nuclei(rng, dims, n_nuclei, r_lo, r_hi, 8.0, 1500.0, margin=margin)
    vol = background(dims, mix_seed(seed, 1), 200.0, 20.0)
    render_nuclei(vol, nuc, 1.5)
    return vol, nuc


# --------------------------------------------------------------------------
# the five workloads
# --------------------------------------------------------------------------

def single_frame(seed=1):
    """128x128x32, one channel, 40 nuclei."""
    vol, _ = nuclei_volume((128, 128, 32), mix_seed(1, seed), 40, 4.0, 8.0, 3.0)
    return vol


class TimeLapse:
    """512x512x64 x frames x 2 channels, nuclei random walk with divisions + static vessels."""

    def __init__(self, seed=2, dims=(512, 512, 64), n_nuclei=300, n_vessels=8, frames=60):
        self.dims = dims
        self.frames = frames
        self.seed = seed
        rng = np.random.Generator(np.random.PCG64(mix_seed(2, seed)))
        self.nuclei0 = place_nuclei(rng, dims, n_nuclei, 4.0, 9.0, 3.0, 1500.0)
        self._rng = rng
        self.vessel_segments = spline_vessels(rng, dims, n_vessels)
        self._vessel_field = None
        self._states = [self.nuclei0]

    def vessel_field(self):
        if self._vessel_field is None:
            self._vessel_field = tube_field(self.dims, self.vessel_segments, 1.0)
        return self._vessel_field

    def nuclei_at(self, t):
        X, Y, Z = self.dims
        cap = 2 * len(self.nuclei0)
        while len(self._states) <= t:
            prev = self._states[-1]
            rng = np.random.Generator(np.random.PCG64(mix_seed(2, self.seed, len(self._states))))
            cur = prev.copy()
            d = rng.normal(size=(len(cur), 3))
            d /= np.maximum(np.linalg.norm(d, axis=1, keepdims=True), 1e-9)
            cur[:, :3] += 2.0 * d
            lo = cur[:, 3:6].max(axis=1)
            for a, hi in enumerate((X - 1, Y - 1, Z - 1)):
                c = cur[:, a]
                lim_lo = np.minimum(lo, hi / 2.0)
                lim_hi = np.maximum(hi - lo, hi / 2.0)
                c = np.where(c < lim_lo, 2 * lim_lo - c, c)
                c = np.where(c > lim_hi, 2 * lim_hi - c, c)
                cur[:, a] = np.clip(c, lim_lo, lim_hi)
            divide = rng.uniform(size=len(cur)) < 0.05
            born = []
            for i in np.nonzero(divide)[0]:
                if len(cur) + len(born) >= cap:
                    break
                u = rng.normal(size=3)
                u /= max(np.linalg.norm(u), 1e-9)
                r = cur[i, 3:6] * 2.0 ** (-1.0 / 3.0)
                off = (r.max() + 1.0) * u
                child = cur[i].copy()
                child[3:6] = r
                child[:3] += off
                cur[i, 3:6] = r
                cur[i, :3] -= off
                born.append(child)
            if born:
                cur = np.vstack([cur, np.array(born)])
            self._states.append(cur)
        return self._states[t]

    def frame(self, t, channel):
        """uint16 [Z,Y,X] for frame t, channel 0 (nuclei) or 1 (vessels)."""
        s = mix_seed(2, self.seed, t, channel)
        vol = background(self.dims, s, 200.0, 25.0)
        if channel == 0:
            render_nuclei(vol, self.nuclei_at(t), 1.5)
        else:
            add_field(vol, self.vessel_field())
        return vol


def batched_uneven_dims(seed=3, n=48):
    """Dims of the batched-uneven workload: first 64^3, last 1024x1024x96."""
    rng = np.random.Generator(np.random.PCG64(mix_seed(3, seed)))
    dims = []
    for i in range(n):
        xy = int(round(math.exp(rng.uniform(math.log(64), math.log(1024)))))
        z = int(rng.integers(64, 97))
        dims.append((xy, xy, z))
    dims[0] = (64, 64, 64)
    dims[-1] = (1024, 1024, 96)
    return dims


def density_volume(dims, seed, per=40 ** 3):
    """Noise N(200,20) + nuclei at 1 per `per` voxels (radii U[4,8])."""
    X, Y, Z = dims
    n = max(1, int(round(X * Y * Z / per)))
    vol, _ = nuclei_volume(dims, seed, n, 4.0, 8.0, 3.0)
    return vol


def batched_uneven(seed=3, n=48):
    return [density_volume(d, mix_seed(3, seed, i)) for i, d in enumerate(batched_uneven_dims(seed, n))]


def serving_requests(seed=5, n=2000, rate=200.0):
    """Poisson request stream: list of (arrival_s, dims)."""
    rng = np.random.Generator(np.random.PCG64(mix_seed(5, seed)))
    t = np.cumsum(rng.exponential(1.0 / rate, size=n))
    out = []
    for i in range(n):
        u = rng.uniform()
        xy = int(round(128 * 16 ** u))
        z = max(1, int(round(128 * 0.5 ** u)))
        out.append((float(t[i]), (xy, xy, z)))
    return out


def serving_volume(dims, seed, index, channel):
    if channel == 0:
        return density_volume(dims, mix_seed(5, seed, index, 0))
    rng = np.random.Generator(np.random.PCG64(mix_seed(5, seed, index, 1)))
    X, Y, Z = dims
    vol = background(dims, mix_seed(5, seed, index, 2), 200.0, 25.0)
    nv = max(1, int(round(X * Y / (1024 * 1024))))
    add_field(vol, tube_field(dims, spline_vessels(rng, dims, nv), 1.0))
    return vol


def montage(seed=4, dims=(5530, 5530, 80), n_nuclei=20000, channel=0):
    """The stitched 6x6-tile montage as one global volume (one channel)."""
    if channel == 0:
        vol, _ = nuclei_volume(dims, mix_seed(4, seed), n_nuclei, 4.0, 9.0, 3.0,
                               noise_sigma=25.0)
        return vol
    rng = np.random.Generator(np.random.PCG64(mix_seed(4, seed, 1)))
    X, Y, Z = dims
    vol = background(dims, mix_seed(4, seed, 2), 200.0, 25.0)
    # about one long vessel per 1024 x 1024 of stage area
    nv = max(1, int(round(X * Y / (1024 * 1024))))
    add_field(vol, tube_field(dims, spline_vessels(rng, dims, nv), 1.0))
    return vol
