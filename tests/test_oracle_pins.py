"""Pins for the CPU oracle, independent of the oracle's own code.

Each test checks the oracle against something the paper or mathematics fixes:
brute-force definitions (the 125-term smoothing sum, iterative min-label
propagation, per-label enumeration), closed forms (impulse response, exact
rational Otsu, symmetric sums), invariants and library special cases
(numpy.bincount, scipy.ndimage.label with the full 3x3x3 structure).
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
B5 = np.array([1, 4, 6, 4, 1], dtype=np.int64)


# ----------------------------------------------------------------------------
# smoothing (Background Noise Removal, Eq. 1: Gaussian low-pass -> binomial)
# ----------------------------------------------------------------------------

def smooth_bruteforce(v):
    """The 125-term definition with per-axis edge clamping, int64, one rounding."""
    Z, Y, X = v.shape
    v = v.astype(np.int64)
    S = np.zeros_like(v)
    xs, ys, zs = np.arange(X), np.arange(Y), np.arange(Z)
    for c in range(5):
        zi = np.clip(zs + c - 2, 0, Z - 1)
        for b in range(5):
            yi = np.clip(ys + b - 2, 0, Y - 1)
            for a in range(5):
                xi = np.clip(xs + a - 2, 0, X - 1)
                S += B5[a] * B5[b] * B5[c] * v[np.ix_(zi, yi, xi)]
    assert S.max() < 2 ** 32
    return ((S + 2048) >> 12).astype(np.uint16)


@pytest.mark.parametrize("dims", [(1, 1, 1), (2, 3, 4), (5, 5, 5), (7, 3, 9), (13, 11, 6),
                                  (1, 17, 2), (33, 4, 3)])
def test_smooth_equals_125_term_sum(dims):
    X, Y, Z = dims
    rng = np.random.default_rng(hash(dims) & 0xFFFF)
    for kind in range(3):
        if kind == 0:
            v = rng.integers(0, 65536, size=(Z, Y, X), dtype=np.uint16)
        elif kind == 1:
            v = rng.choice(np.array([0, 65535], dtype=np.uint16), size=(Z, Y, X))
        else:
            v = rng.integers(150, 260, size=(Z, Y, X), dtype=np.uint16)
        np.testing.assert_array_equal(oracle.smooth(v), smooth_bruteforce(v))


def test_smooth_impulse_response():
    # an interior impulse of height 4096 returns exactly B[a]B[b]B[c]
    v = np.zeros((9, 9, 9), dtype=np.uint16)
    v[4, 4, 4] = 4096
    s = oracle.smooth(v).astype(np.int64)
    expect = np.zeros((9, 9, 9), dtype=np.int64)
    expect[2:7, 2:7, 2:7] = B5[:, None, None] * B5[None, :, None] * B5[None, None, :]
    np.testing.assert_array_equal(s, expect)


def test_smooth_constant_and_bounds():
    for c in (0, 1, 200, 4095, 65535):
        v = np.full((6, 7, 8), c, dtype=np.uint16)
        np.testing.assert_array_equal(oracle.smooth(v), v)
    rng = np.random.default_rng(7)
    v = rng.integers(1000, 3000, size=(10, 12, 14), dtype=np.uint16)
    s = oracle.smooth(v)
    assert s.min() >= v.min() and s.max() <= v.max()


def test_smooth_half_rounds_up():
    # S = 2048 exactly (half of 4096) must round up to 1: an impulse of height
    # 2048/(B[a]B[b]B[c]) with B=6*6*6=216 is not integral, so build S=2048 by
    # a single corner-adjacent value: impulse 8 at distance 2 in x and y and z
    # contributes 8*1*1*1*...; use height 2048 at a voxel seen with weight 1.
    v = np.zeros((5, 5, 5), dtype=np.uint16)
    v[0, 0, 0] = 2048
    s = smooth_bruteforce(v)
    # voxel (2,2,2) sees (0,0,0) with weight 1*1*1 -> S = 2048 -> s = 1
    assert s[2, 2, 2] == 1
    assert oracle.smooth(v)[2, 2, 2] == 1


# ----------------------------------------------------------------------------
# histogram
# ----------------------------------------------------------------------------

def test_histogram_matches_bincount():
    rng = np.random.default_rng(3)
    s = rng.integers(0, 65536, size=100000, dtype=np.uint16)
    h = oracle.histogram(s)
    np.testing.assert_array_equal(h, np.bincount(s, minlength=65536).astype(np.uint64))
    assert int(h.sum()) == s.size


# ----------------------------------------------------------------------------
# Otsu (Segmentation section, ref. [11])
# ----------------------------------------------------------------------------

def load_otsu_golden():
    cases = []
    with open(os.path.join(GOLDEN, "otsu_hand.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            lhs, rhs = line.split("->")
            h = np.zeros(65536, dtype=np.uint64)
            for tok in lhs.split():
                lvl, cnt = tok.split(":")
                h[int(lvl)] += int(cnt)
            cases.append((h, int(rhs)))
    return cases


def test_otsu_hand_worked():
    cases = load_otsu_golden()
    assert len(cases) >= 8
    for h, t in cases:
        assert oracle.otsu(h) == t


def otsu_exact(h):
    """Exact-rational Otsu: argmax of (S n0 - N s0)^2 / (n0 n1), ties -> lowest t.

    Returns (t*, best value, runner-up value among distinct classes)."""
    nz = np.nonzero(h)[0]
    N = int(h.sum())
    S = int(sum(int(u) * int(h[u]) for u in nz))
    best = None
    best_t = None
    values = []
    n0 = s0 = 0
    for u in nz:
        n0 += int(h[u])
        s0 += int(u) * int(h[u])
        n1 = N - n0
        if n1 == 0:
            break
        val = Fraction((S * n0 - N * s0) ** 2, n0 * n1)
        values.append(val)
        if best is None or val > best:
            best, best_t = val, int(u)
    if best_t is None:
        return int(nz[0]), None, None
    vs = sorted(set(values), reverse=True)
    return best_t, best, (vs[1] if len(vs) > 1 else None)


def test_otsu_vs_exact_rational():
    rng = np.random.default_rng(11)
    near_ties = 0
    for trial in range(400):
        h = np.zeros(65536, dtype=np.uint64)
        k = int(rng.integers(1, 12))
        span = int(rng.choice([8, 64, 4096, 65536]))
        lo = int(rng.integers(0, 65536 - span + 1))
        k = min(k, span)
        levels = rng.choice(np.arange(lo, lo + span), size=k, replace=False)
        h[levels] = rng.integers(1, 10 ** int(rng.integers(1, 7)), size=k).astype(np.uint64)
        t_exact, best, second = otsu_exact(h)
        t = oracle.otsu(h)
        if t != t_exact:
            # only admissible when binary64 cannot separate the top two values
            assert second is not None and abs(best - second) <= Fraction(1, 10 ** 12) * best
            near_ties += 1
    assert near_ties == 0


def test_otsu_two_spikes_and_scale():
    rng = np.random.default_rng(5)
    for _ in range(50):
        a, b = sorted(rng.choice(65536, size=2, replace=False))
        h = np.zeros(65536, dtype=np.uint64)
        h[a] = rng.integers(1, 10 ** 6)
        h[b] = rng.integers(1, 10 ** 6)
        assert oracle.otsu(h) == a
        # power-of-two scaling of all counts scales var exactly by 4^j
        h2 = h * np.uint64(1 << int(rng.integers(1, 8)))
        assert oracle.otsu(h2) == a


def test_otsu_empty_runs_pick_lowest():
    # levels between occupied bins repeat the same (n0, s0) -> same value;
    # the answer must be an occupied level
    rng = np.random.default_rng(9)
    for _ in range(50):
        h = np.zeros(65536, dtype=np.uint64)
        lv = rng.choice(65536, size=6, replace=False)
        h[lv] = rng.integers(1, 1000, size=6).astype(np.uint64)
        assert h[oracle.otsu(h)] > 0


# ----------------------------------------------------------------------------
# 26-connected labelling (Segmentation section, connected component filter)
# ----------------------------------------------------------------------------

def minlabel_propagation(mask):
    """Brute force: every foreground voxel repeatedly takes the minimum linear
    index over itself and its 26 neighbours until nothing changes; components
    are then numbered by that minimum."""
    Z, Y, X = mask.shape
    big = np.iinfo(np.int64).max
    idx = np.arange(mask.size, dtype=np.int64).reshape(mask.shape)
    cur = np.where(mask, idx, big)
    while True:
        pad = np.pad(cur, 1, constant_values=big)
        nxt = cur.copy()
        for dz in (-1, 0, 1):
            for dy in (-1, 0, 1):
                for dx in (-1, 0, 1):
                    sh = pad[1 + dz:1 + dz + Z, 1 + dy:1 + dy + Y, 1 + dx:1 + dx + X]
                    nxt = np.minimum(nxt, sh)
        nxt = np.where(mask, nxt, big)
        if np.array_equal(nxt, cur):
            break
        cur = nxt
    roots = np.unique(cur[mask])
    rank = {int(r): i + 1 for i, r in enumerate(roots)}
    out = np.zeros(mask.shape, dtype=np.uint32)
    out[mask] = [rank[int(r)] for r in cur[mask]]
    return out, len(roots)


@pytest.mark.parametrize("dims", [(1, 1, 1), (3, 3, 3), (12, 5, 1), (6, 7, 8), (12, 12, 12),
                                  (1, 9, 11), (10, 1, 10)])
def test_label26_vs_minlabel_propagation(dims):
    X, Y, Z = dims
    rng = np.random.default_rng(sum(dims))
    for p in (0.05, 0.1, 0.3, 0.5, 0.7, 0.95):
        mask = rng.uniform(size=(Z, Y, X)) < p
        lab, n = oracle.label26(mask)
        ref, nref = minlabel_propagation(mask)
        assert n == nref
        np.testing.assert_array_equal(lab, ref)


def test_label26_vs_scipy():
    ndimage = pytest.importorskip("scipy.ndimage")
    rng = np.random.default_rng(21)
    for trial in range(10):
        dims = rng.integers(5, 40, size=3)
        mask = rng.uniform(size=tuple(dims)) < rng.uniform(0.05, 0.6)
        lab, n = oracle.label26(mask)
        ref, nref = ndimage.label(mask, structure=np.ones((3, 3, 3), dtype=bool))
        assert n == nref
        np.testing.assert_array_equal(lab, ref.astype(np.uint32))


def load_label_golden():
    cases = []
    with open(os.path.join(GOLDEN, "label_tiny.txt")) as f:
        lines = [l.rstrip("\n") for l in f if l.strip() and not l.startswith("#")]
    i = 0
    while i < len(lines):
        _, X, Y, Z = lines[i].split()
        X, Y, Z = int(X), int(Y), int(Z)
        i += 1
        rows = lines[i:i + Y * Z]
        i += Y * Z
        assert lines[i] == "labels"
        i += 1
        lrows = lines[i:i + Y * Z]
        i += Y * Z
        assert lines[i] == "end"
        i += 1
        mask = np.array([[c == "o" for c in r] for r in rows]).reshape(Z, Y, X)
        lab = np.array([[0 if c == "." else int(c) for c in r] for r in lrows],
                       dtype=np.uint32).reshape(Z, Y, X)
        cases.append((mask, lab))
    return cases


def test_label26_hand_worked():
    cases = load_label_golden()
    assert len(cases) == 4
    for mask, expect in cases:
        lab, n = oracle.label26(mask)
        np.testing.assert_array_equal(lab, expect)
        assert n == expect.max()


def test_label26_connectivity_kinds():
    # face, edge and corner contacts all join under 26-connectivity
    for off in [(0, 0, 1), (0, 1, 1), (1, 1, 1), (1, -1, 1)]:
        m = np.zeros((3, 3, 3), dtype=bool)
        m[1, 1, 1] = True
        m[1 + off[0], 1 + off[1], 1 + off[2]] = True
        _, n = oracle.label26(m)
        assert n == 1
    # distance 2 never joins
    m = np.zeros((1, 1, 5), dtype=bool)
    m[0, 0, 0] = m[0, 0, 2] = m[0, 0, 4] = True
    lab, n = oracle.label26(m)
    assert n == 3 and list(lab[0, 0]) == [1, 0, 2, 0, 3]


# ----------------------------------------------------------------------------
# minimum volume, canonical numbering, features
# ----------------------------------------------------------------------------

def features_enumerated(labels, K):
    out = []
    for l in range(1, K + 1):
        z, y, x = np.nonzero(labels == l)
        out.append((len(x), (int(x.sum()), int(y.sum()), int(z.sum())),
                    (int(x.min()), int(y.min()), int(z.min())),
                    (int(x.max()), int(y.max()), int(z.max()))))
    return out


def check_cells(cells, labels):
    K = len(cells)
    assert labels.max() == K
    for c, (cnt, sums, mn, mx) in zip(cells, features_enumerated(labels, K)):
        assert int(c["count"]) == cnt
        assert tuple(int(v) for v in c["sum"]) == sums
        assert tuple(int(v) for v in c["bbox_min"]) == mn
        assert tuple(int(v) for v in c["bbox_max"]) == mx


@pytest.mark.parametrize("m", [0, 1, 2, 5, 30])
def test_filter_and_features(m):
    rng = np.random.default_rng(100 + m)
    mask = rng.uniform(size=(9, 14, 17)) < 0.25
    prov, n = oracle.label26(mask)
    lab, cells = oracle.filter_features(prov, n, m)
    counts = np.bincount(prov.ravel(), minlength=n + 1)
    keep = [c for c in range(1, n + 1) if counts[c] >= m]
    assert len(cells) == len(keep)
    # survivors keep their relative (lowest-index) order and become 1..K
    for new, old in enumerate(keep, start=1):
        np.testing.assert_array_equal(lab == new, prov == old)
    assert np.all(lab[np.isin(prov, [c for c in range(1, n + 1) if counts[c] < m])] == 0)
    check_cells(cells, lab)


def test_symmetric_shapes_closed_form():
    # digitised sphere centred on a voxel: sums are count * centre exactly
    Z, Y, X = 21, 23, 25
    zz, yy, xx = np.mgrid[0:Z, 0:Y, 0:X]
    c = (12, 11, 10)
    ball = (xx - c[0]) ** 2 + (yy - c[1]) ** 2 + (zz - c[2]) ** 2 <= 36
    box = (xx >= 1) & (xx <= 4) & (yy >= 2) & (yy <= 20) & (zz >= 18) & (zz <= 19)
    prov, n = oracle.label26(ball | box)
    lab, cells = oracle.filter_features(prov, n, 1)
    assert len(cells) == 2
    bi = 0 if cells[0]["bbox_min"][2] < 10 else 1
    b, q = cells[bi], cells[1 - bi]
    k = int(b["count"])
    assert k == int(ball.sum())
    assert tuple(int(v) for v in b["sum"]) == (k * c[0], k * c[1], k * c[2])
    assert tuple(int(v) for v in b["bbox_min"]) == (6, 5, 4)
    assert tuple(int(v) for v in b["bbox_max"]) == (18, 17, 16)
    # box 4 x 19 x 2: sum of x = 19*2*(1+2+3+4), y = 4*2*sum(2..20), z = 4*19*(18+19)
    assert int(q["count"]) == 4 * 19 * 2
    assert tuple(int(v) for v in q["sum"]) == (19 * 2 * 10, 4 * 2 * sum(range(2, 21)),
                                              4 * 19 * 37)


# ----------------------------------------------------------------------------
# whole pipeline
# ----------------------------------------------------------------------------

def test_segment_composes_the_steps():
    rng = np.random.default_rng(4)
    v = rng.integers(100, 400, size=(10, 20, 30), dtype=np.uint16)
    v[3:7, 5:12, 8:20] += 2000
    r = oracle.segment(v, min_volume=3, keep_hist=True, keep_smoothed=True)
    s = smooth_bruteforce(v)
    np.testing.assert_array_equal(r.smoothed, s)
    np.testing.assert_array_equal(r.hist, np.bincount(s.ravel(), minlength=65536))
    t_exact, _, _ = otsu_exact(r.hist)
    assert r.threshold == t_exact
    ref, _ = minlabel_propagation(s > r.threshold)
    counts = np.bincount(ref.ravel())
    keep = [c for c in range(1, len(counts)) if counts[c] >= 3]
    assert r.n_cells == len(keep)
    check_cells(r.cells, r.labels)


def test_blank_volume_has_no_cells():
    for c in (0, 200, 65535):
        v = np.full((8, 9, 10), c, dtype=np.uint16)
        r = oracle.segment(v)
        assert r.threshold == c and r.n_cells == 0 and not r.labels.any()


def test_well_separated_nuclei_counted_exactly():
    for seed in (1, 2, 3):
        vol, nuc = synth.well_separated((96, 96, 40), seed, 25)
        assert len(nuc) >= 15
        r = oracle.segment(vol, min_volume=30)
        assert r.n_cells == len(nuc)
        # each planted centre lies in the bbox of exactly one cell
        for c in nuc[:, :3]:
            inside = [(cell["bbox_min"] <= c).all() and (c <= cell["bbox_max"]).all()
                      for cell in r.cells]
            assert sum(inside) == 1


def test_single_frame_workload_counts():
    vol = synth.single_frame()
    r = oracle.segment(vol, min_volume=30)
    assert 30 <= r.n_cells <= 40
    assert 300 < r.threshold < 1500


# ---------------------------------------------------------------------------
# Denoise front end (Background Noise Removal, Eq. 1): background by box
# cascade, floor-at-zero subtraction, 3x3x3 median
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("r", [1, 2, 4, 8])
def test_box_pass_matches_uniform_filter(r):
    ndi = pytest.importorskip("scipy.ndimage")
    # one pass = the mean over 2r+1 replicate-padded neighbours, rounded to
    # nearest; w is odd, so no value lies exactly halfway
    rng = np.random.default_rng(40 + r)
    for shape in [(7, 9, 11), (3, 1, 20), (1, 5, 2)]:
        v = rng.integers(0, 65536, size=shape).astype(np.uint16)
        for axis in range(3):
            got = oracle.box_pass(v, axis, r)
            mean = ndi.uniform_filter1d(v.astype(np.float64), size=2 * r + 1, axis=2 - axis, mode="nearest")
            assert np.array_equal(got, np.floor(mean + 0.5).astype(np.uint16)), (shape, axis)


@pytest.mark.parametrize("r", [1, 3, 8])
def test_box_cascade_impulse_is_three_fold_convolution(r):
    # an impulse of height k w^3 far from the edges stays exact through three
    # passes (every intermediate sum divides by w), giving k times the
    # three-fold convolution of the box with itself
    w = 2 * r + 1
    k = 7
    X = 8 * w
    v = np.zeros((1, 1, X), dtype=np.uint16)
    c = X // 2
    v[0, 0, c] = k * w ** 3 if k * w ** 3 < 65536 else 0
    if v[0, 0, c] == 0:
        k = 65535 // w ** 3
        v[0, 0, c] = k * w ** 3
    out = v
    for _ in range(3):
        out = oracle.box_pass(out, 0, r)
    kern = np.convolve(np.convolve(np.ones(w, dtype=np.int64), np.ones(w, dtype=np.int64)), np.ones(w, dtype=np.int64))
    expect = np.zeros(X, dtype=np.int64)
    expect[c - 3 * r: c + 3 * r + 1] = k * kern
    assert np.array_equal(out[0, 0].astype(np.int64), expect)


def test_background_keeps_constants_and_interior_ramps():
    r = 3
    flat = np.full((12, 13, 14), 777, dtype=np.uint16)
    assert np.array_equal(oracle.background(flat, r), flat)
    # a ramp along each axis in turn is reproduced wherever the windows of
    # all nine passes stay inside the volume (symmetric sums of a linear
    # function are exact multiples of w)
    for axis in range(3):
        n = 6 * 3 * r + 5
        idx = np.arange(n, dtype=np.int64) * 5 + 100
        shape = [3, 3, 3]
        shape[2 - axis] = n
        ramp = np.broadcast_to(idx.reshape([-1 if i == 2 - axis else 1 for i in range(3)]), shape)
        ramp = np.ascontiguousarray(ramp, dtype=np.uint16)
        b = oracle.background(ramp, r)
        sl = [slice(None)] * 3
        sl[2 - axis] = slice(3 * r, n - 3 * r)
        assert np.array_equal(b[tuple(sl)], ramp[tuple(sl)]), axis


def test_median27_matches_scipy():
    ndi = pytest.importorskip("scipy.ndimage")
    rng = np.random.default_rng(44)
    for shape in [(6, 7, 8), (1, 1, 5), (2, 3, 1), (4, 4, 4)]:
        v = rng.integers(0, 65536, size=shape).astype(np.uint16)
        assert np.array_equal(oracle.median27(v), ndi.median_filter(v, size=3, mode="nearest")), shape
    # few distinct values: ties
    v = rng.integers(0, 3, size=(9, 10, 11)).astype(np.uint16)
    assert np.array_equal(oracle.median27(v), ndi.median_filter(v, size=3, mode="nearest"))


def test_denoise_is_median_of_floored_difference():
    ndi = pytest.importorskip("scipy.ndimage")
    rng = np.random.default_rng(45)
    v = rng.integers(0, 4000, size=(10, 12, 14)).astype(np.uint16)
    for r in (1, 4):
        b = oracle.background(v, r).astype(np.int64)
        d = np.maximum(v.astype(np.int64) - b, 0).astype(np.uint16)
        assert np.array_equal(oracle.denoise(v, r), ndi.median_filter(d, size=3, mode="nearest"))


def test_segment_with_denoise_is_segment_of_denoised():
    vol, _ = synth.well_separated((48, 40, 20), seed=9, n_nuclei=6)
    r = 4
    a = oracle.segment(vol, min_volume=5, denoise_radius=r)
    b = oracle.segment(oracle.denoise(vol, r), min_volume=5)
    assert a.threshold == b.threshold and np.array_equal(a.labels, b.labels)


# ---------------------------------------------------------------------------
# Closing with a binary ball (Segmentation): pinned to scipy on the padded
# volume, and to the algebra of a closing
# ---------------------------------------------------------------------------

def _ball(rho):
    g = np.arange(-rho, rho + 1)
    return (g[:, None, None] ** 2 + g[None, :, None] ** 2 + g[None, None, :] ** 2) <= rho * rho


@pytest.mark.parametrize("rho", [1, 2, 3])
def test_close_matches_scipy_on_padded_volume(rho):
    ndi = pytest.importorskip("scipy.ndimage")
    rng = np.random.default_rng(60 + rho)
    for shape, p in [((9, 11, 13), 0.3), ((4, 20, 7), 0.5), ((1, 6, 30), 0.4), ((12, 12, 12), 0.1)]:
        m = rng.uniform(size=shape) < p
        padded = np.pad(m, rho)
        ref = ndi.binary_closing(padded, structure=_ball(rho))[rho:-rho, rho:-rho, rho:-rho]
        assert np.array_equal(oracle.close(m, rho), ref), (shape, rho)


def test_close_algebra():
    rng = np.random.default_rng(66)
    m = rng.uniform(size=(10, 12, 14)) < 0.35
    for rho in (1, 2):
        c = oracle.close(m, rho)
        assert np.all(c[m])                                  # extensive
        assert np.array_equal(oracle.close(c, rho), c)       # idempotent
    assert np.array_equal(oracle.close(m, 0), m)             # radius 0: identity
    # a one-voxel hole inside a solid block is filled by the smallest ball
    b = np.zeros((9, 9, 9), dtype=bool)
    b[2:7, 2:7, 2:7] = True
    b[4, 4, 4] = False
    assert oracle.close(b, 1)[4, 4, 4]


def test_segment_with_closing_labels_the_closed_mask():
    ndi = pytest.importorskip("scipy.ndimage")
    vol, _ = synth.well_separated((40, 36, 18), seed=11, n_nuclei=5)
    r = oracle.segment(vol, min_volume=1, closing_radius=2, keep_smoothed=True)
    closed = oracle.close(r.smoothed > r.threshold, 2)
    lab, n = ndi.label(closed, structure=np.ones((3, 3, 3)))
    assert n == r.labels.max() and np.array_equal(r.labels > 0, closed)


# ---------------------------------------------------------------------------
# Distance map of the foreground (vasculature channel): brute-force minimum,
# pinned to scipy's exact Euclidean distance transform with the voxel spacing
# ---------------------------------------------------------------------------

def test_distance_matches_scipy_edt():
    ndi = pytest.importorskip("scipy.ndimage")
    rng = np.random.default_rng(70)
    for shape, p in [((6, 9, 11), 0.05), ((1, 7, 20), 0.1), ((9, 9, 9), 0.01), ((4, 13, 5), 0.3)]:
        m = rng.uniform(size=shape) < p
        m.flat[rng.integers(m.size)] = True
        d2 = oracle.distance(m, (16, 16, 25))
        # scipy: distance to the nearest zero, sampling per axis (z, y, x) in um
        e = ndi.distance_transform_edt(~m, sampling=(1.0, 0.8, 0.8))
        assert np.array_equal(d2, np.rint(25.0 * e * e).astype(np.uint32)), shape


def test_distance_special_cases():
    m = np.zeros((3, 4, 5), dtype=bool)
    assert np.all(oracle.distance(m) == 0xFFFFFFFF)         # no foreground
    m[1, 2, 3] = True
    d2 = oracle.distance(m, (1, 2, 3))
    z, y, x = np.meshgrid(np.arange(3), np.arange(4), np.arange(5), indexing="ij")
    assert np.array_equal(d2, (x - 3) ** 2 + 2 * (y - 2) ** 2 + 3 * (z - 1) ** 2)
    assert np.all(oracle.distance(np.ones((2, 2, 2), dtype=bool)) == 0)


def test_distance_at_agrees_with_the_full_map():
    # the sampled form used at full size gives the full map's values
    rng = np.random.default_rng(71)
    for shape, p in [((5, 8, 13), 0.03), ((3, 3, 3), 0.0), ((7, 2, 9), 0.2)]:
        m = rng.uniform(size=shape) < p
        pts = [tuple(int(rng.integers(s)) for s in shape) for _ in range(25)]
        d2 = oracle.distance(m, (7, 3, 11))
        assert np.array_equal(oracle.distance_at(m, pts, (7, 3, 11)), np.array([d2[q] for q in pts], np.uint32))


# ---- MRF vessel denoise (Background Noise Removal, Eqs. 2-3) ---------------

def test_mrf_delta_is_the_smallest_gap():
    rng = np.random.default_rng(80)
    for levels in ([7], [3, 10], [0, 65535], [5, 9, 12, 40000]):
        v = rng.choice(np.array(levels, np.uint16), size=(3, 4, 5))
        v.flat[: len(levels)] = levels  # every level present
        u = np.unique(v)
        want = int(np.diff(u.astype(np.int64)).min()) if len(u) > 1 else 0
        assert oracle.mrf_delta(v) == want
    v = rng.integers(100, 4000, size=(6, 7, 8)).astype(np.uint16)
    assert oracle.mrf_delta(v) == int(np.diff(np.unique(v).astype(np.int64)).min())


def test_mrf_laplacian_matches_convolution():
    ndi = pytest.importorskip("scipy.ndimage")
    mask = np.array([[1, -2, 1], [-2, 4, -2], [1, -2, 1]], np.int64)
    rng = np.random.default_rng(81)
    for shape in [(3, 9, 11), (1, 3, 3), (2, 5, 40), (4, 2, 7), (2, 8, 2)]:
        v = rng.integers(0, 65536, size=shape).astype(np.uint16)
        s = 0
        for plane in v.astype(np.int64):
            r = ndi.convolve(plane, mask, mode="constant")[1:-1, 1:-1]
            s += int(np.abs(r).sum())
        Z, Y, X = shape
        assert oracle.mrf_laplacian(v) == (s, Z * max(X - 2, 0) * max(Y - 2, 0)), shape


def test_mrf_noise_estimate_recovers_sigma():
    # Immerkaer's estimate is unbiased for white Gaussian noise on a flat image
    rng = np.random.default_rng(82)
    for sigma in (10.0, 30.0):
        v = np.rint(rng.normal(1000, sigma, size=(8, 96, 96))).astype(np.uint16)
        s, m = oracle.mrf_laplacian(v)
        est = math.sqrt(oracle.mrf_limit(s, m, v.size) / v.size)
        assert abs(est - sigma) < 0.05 * sigma, (sigma, est)


def test_mrf_limit_closed_form():
    # one spike of height h inside a zero plane: all nine mask responses are
    # interior, |response| sums to 16 h
    h = 300
    v = np.zeros((2, 7, 9), np.uint16)
    v[1, 3, 4] = h
    s, m = oracle.mrf_laplacian(v)
    assert (s, m) == (16 * h, 2 * 5 * 7)
    sigma = math.sqrt(math.pi / 2) * 16 * h / (6 * m)
    assert oracle.mrf_limit(s, m, v.size) == pytest.approx(v.size * sigma * sigma, rel=1e-15)
    assert oracle.mrf_limit(0, 0, 10) == 0.0


def test_mrf_step_special_cases():
    # constant: fixed
    c = np.full((3, 4, 5), 77, np.uint16)
    assert np.array_equal(oracle.mrf_step(c, 1), c)
    # spike: it drops by delta, its six face neighbours rise by delta
    v = np.zeros((5, 5, 5), np.uint16)
    v[2, 2, 2] = 9
    s = oracle.mrf_step(v, 4).astype(np.int64)
    want = np.zeros((5, 5, 5), np.int64)
    want[2, 2, 2] = 5
    for dz, dy, dx in [(1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)]:
        want[2 + dz, 2 + dy, 2 + dx] = 4
    assert np.array_equal(s, want)
    # ramp along x: the interior is fixed (one vote each way); the low end
    # rises and the high end falls (its outer neighbour votes 0)
    r = np.broadcast_to(np.arange(6, dtype=np.uint16) * 3, (2, 3, 6)).copy()
    s = oracle.mrf_step(r, 3)
    assert np.array_equal(s[..., 1:-1], r[..., 1:-1])
    assert np.all(s[..., 0] == 3) and np.all(s[..., -1] == 12)


def test_mrf_step_invariants():
    rng = np.random.default_rng(83)
    v = rng.integers(0, 50, size=(5, 6, 7)).astype(np.uint16)
    d = oracle.mrf_delta(v)
    s = oracle.mrf_step(v, d).astype(np.int64)
    diff = s - v.astype(np.int64)
    assert set(np.unique(diff)) <= {-d, 0, d}
    # strict local maxima (over in-volume face neighbours) fall, minima rise
    p = np.pad(v.astype(np.int64), 1, mode="edge")
    nb = [p[1:-1, 1:-1, :-2], p[1:-1, 1:-1, 2:], p[1:-1, :-2, 1:-1], p[1:-1, 2:, 1:-1], p[:-2, 1:-1, 1:-1],
          p[2:, 1:-1, 1:-1]]
    c = v.astype(np.int64)
    # (replicated edges equal the centre and vote 0, as the outside does)
    higher = sum((n > c).astype(int) for n in nb)
    lower = sum((n < c).astype(int) for n in nb)
    assert np.all(diff[(lower > 0) & (higher == 0)] == -d)
    assert np.all(diff[(higher > 0) & (lower == 0)] == d)
    # mirror symmetry along each axis
    for ax in range(3):
        assert np.array_equal(oracle.mrf_step(np.flip(v, ax).copy(), d), np.flip(s, ax).astype(np.uint16))


def test_mrf_iteration_stops():
    rng = np.random.default_rng(84)
    # constant: no step changes anything
    c = np.full((4, 5, 6), 300, np.uint16)
    out, it = oracle.mrf(c, 10)
    assert it == 0 and np.array_equal(out, c)
    # planes without interior (Y = 2): sigma = 0, the first step already
    # strays from the original, so nothing is kept
    v = rng.integers(0, 100, size=(3, 2, 9)).astype(np.uint16)
    out, it = oracle.mrf(v, 10)
    assert it == 0 and np.array_equal(out, v)
    # noisy flat image: the kept steps are exactly the repeated step while the
    # summed squares stay within N sigma^2, and fewer steps are a prefix
    v = np.rint(rng.normal(500, 20, size=(4, 24, 24))).astype(np.uint16)
    d = oracle.mrf_delta(v)
    s, m = oracle.mrf_laplacian(v)
    lim = oracle.mrf_limit(s, m, v.size)
    cur, want = v, 0
    while want < 200:
        nxt = oracle.mrf_step(cur, d)
        e = int(((nxt.astype(np.int64) - v.astype(np.int64)) ** 2).sum())
        if np.array_equal(nxt, cur) or float(e) > lim:
            break
        cur, want = nxt, want + 1
    out, it = oracle.mrf(v, 200)
    assert it == want and np.array_equal(out, cur) and 0 < it < 200
    out3, it3 = oracle.mrf(v, 3)
    assert it3 == 3
    p = v
    for _ in range(3):
        p = oracle.mrf_step(p, d)
    assert np.array_equal(out3, p)


def test_segment_with_mrf_is_segment_of_denoised():
    rng = np.random.default_rng(85)
    v = np.rint(rng.normal(200, 25, size=(12, 30, 40))).clip(0, 65535).astype(np.uint16)
    v[4:8, 10:20, 5:35] += 1500
    r = oracle.segment(v, min_volume=5, mrf_iterations=20)
    den, it = oracle.mrf(v, 20)
    assert r.mrf_steps == it and np.array_equal(r.denoised, den)
    ref = oracle.segment(den, min_volume=5)
    assert np.array_equal(r.labels, ref.labels) and r.threshold == ref.threshold


# ---- montage registration (Registration section, Eq. 4) --------------------

def _montage(rng, grid, dims, overlap, jitter, radius):
    """Tiles cut from one textured global volume at true positions; the stage
    positions are the true ones moved by at most `radius` voxels per axis."""
    X, Y, Z = dims
    nx, ny = grid
    step = (X - overlap[0], Y - overlap[1])
    true, stage = [], []
    for j in range(ny):
        for i in range(nx):
            s = np.array([i * step[0], j * step[1], 0])
            t = s + rng.integers(-jitter, jitter + 1, size=3) * np.array([1, 1, 0])
            t[2] = rng.integers(0, radius[2] + 1)
            true.append(t + np.array([radius[0], radius[1], 0]))
            stage.append(s + np.array([radius[0], radius[1], 0]))
    true, stage = np.array(true), np.array(stage)
    ext = true.max(axis=0) + np.array(dims) + 1
    G = rng.integers(0, 4000, size=(ext[2], ext[1], ext[0])).astype(np.uint16)
    tiles = [G[t[2]:t[2] + Z, t[1]:t[1] + Y, t[0]:t[0] + X].copy() for t in true]
    return tiles, true, stage


def test_reg_sums_brute_force():
    rng = np.random.default_rng(90)
    X, Y, Z = 9, 7, 5
    A = rng.integers(0, 65536, size=(Z, Y, X)).astype(np.uint16)
    B = rng.integers(0, 65536, size=(Z, Y, X)).astype(np.uint16)
    for d in [(0, 0, 0), (3, -2, 1), (-8, 6, -4), (9, 0, 0), (2, 2, 5), (-4, -6, 0)]:
        n = sa = sb = saa = sbb = sab = 0
        for z in range(Z):
            for y in range(Y):
                for x in range(X):
                    bx, by, bz = x - d[0], y - d[1], z - d[2]
                    if 0 <= bx < X and 0 <= by < Y and 0 <= bz < Z:
                        a, b = int(A[z, y, x]), int(B[bz, by, bx])
                        n, sa, sb, saa, sbb, sab = n + 1, sa + a, sb + b, saa + a * a, sbb + b * b, sab + a * b
        assert list(oracle.reg_sums(A, B, d)) == [n, sa, sb, saa, sbb, sab], d


def test_normcov_special_cases():
    rng = np.random.default_rng(91)
    A = rng.integers(0, 30000, size=(4, 6, 8)).astype(np.uint16)
    assert oracle.normcov(oracle.reg_sums(A, A, (0, 0, 0))) == pytest.approx(1.0, abs=1e-15)
    B = (2 * A.astype(np.int64) + 7).astype(np.uint16)
    assert oracle.normcov(oracle.reg_sums(A, B, (0, 0, 0))) == pytest.approx(1.0, abs=1e-15)
    C = (60000 - A.astype(np.int64)).astype(np.uint16)
    assert oracle.normcov(oracle.reg_sums(A, C, (0, 0, 0))) == pytest.approx(-1.0, abs=1e-15)
    assert oracle.normcov(oracle.reg_sums(A, np.full_like(A, 5), (0, 0, 0))) is None  # no variance
    assert oracle.normcov(oracle.reg_sums(A, A, (8, 0, 0))) is None                   # no overlap
    D = rng.integers(0, 65536, size=A.shape).astype(np.uint16)
    d = (2, -1, 1)
    a = A[1:, :5, 2:].astype(np.float64).ravel()
    b = D[:3, 1:, :6].astype(np.float64).ravel()
    assert oracle.normcov(oracle.reg_sums(A, D, d)) == pytest.approx(np.corrcoef(a, b)[0, 1], abs=1e-12)


def test_register_recovers_planted_offsets():
    rng = np.random.default_rng(92)
    radius = (3, 3, 2)
    # relative shifts of neighbours stay inside the window (jitter 1 per tile)
    tiles, true, stage = _montage(rng, (3, 2), (40, 36, 12), (9, 8), 1, radius)
    delta, edges = oracle.register(tiles, stage, radius, root=0)
    assert np.array_equal(delta, (true - stage) - (true - stage)[0])
    # a tree edge's shift is the difference of its tiles' corrections
    for e in edges[edges["in_tree"] == 1]:
        assert np.array_equal(delta[e["b"]] - delta[e["a"]], e["shift"])
    assert (edges["in_tree"] == 1).sum() == len(tiles) - 1
    # another root moves every correction by the same amount
    d2, _ = oracle.register(tiles, stage, radius, root=4)
    assert np.array_equal(d2 - d2[0], delta)


def test_register_tree_is_maximum():
    # the tree has the largest total score among all spanning trees of the
    # pair graph (brute force over edge subsets)
    import itertools
    rng = np.random.default_rng(93)
    radius = (2, 2, 1)
    tiles, true, stage = _montage(rng, (2, 2), (30, 30, 8), (8, 8), 1, radius)
    # noisier copies so that scores differ
    tiles = [np.clip(t.astype(np.int64) + rng.integers(-3000, 3000, size=t.shape), 0, 65535).astype(np.uint16)
             for t in tiles]
    _, edges = oracle.register(tiles, stage, radius, root=0)
    n = len(tiles)
    best = None
    for sub in itertools.combinations(range(len(edges)), n - 1):
        p = list(range(n))

        def f(i):
            while p[i] != i:
                i = p[i]
            return i
        ok = True
        for k in sub:
            ra, rb = f(int(edges[k]["a"])), f(int(edges[k]["b"]))
            if ra == rb:
                ok = False
                break
            p[ra] = rb
        if ok:
            w = sum(edges[k]["score"] for k in sub)
            best = w if best is None else max(best, w)
    chosen = edges[edges["in_tree"] == 1]["score"].sum()
    assert len(edges[edges["in_tree"] == 1]) == n - 1 and chosen == pytest.approx(best, abs=1e-12)


def test_cell_distance_is_the_smallest_map_value_per_cell():
    rng = np.random.default_rng(95)
    lab = rng.integers(0, 6, size=(5, 7, 9)).astype(np.uint32)
    lab[0, 0, 0] = 5
    m = rng.integers(0, 1 << 31, size=lab.shape).astype(np.uint32)
    got = oracle.cell_distance(lab, m, 7)  # labels 6 and 7 have no voxel
    for k in range(1, 8):
        sel = m[lab == k]
        assert got[k - 1] == (sel.min() if sel.size else 0xFFFFFFFF), k
    # a cell touching the vessel foreground is at distance 0; the whole
    # stage's cells against the oracle's vessel map
    vol = synth.single_frame()
    r = oracle.segment(vol, min_volume=30)
    vessel = np.zeros(vol.shape, bool)
    vessel[10:12, 40:90, 60:64] = True
    dmap = oracle.distance(vessel, (16, 16, 25))
    cd = oracle.cell_distance(r.labels, dmap, r.n_cells)
    for k in range(1, r.n_cells + 1):
        inside = (r.labels == k)
        assert cd[k - 1] == dmap[inside].min()
        assert (cd[k - 1] == 0) == bool((inside & vessel).any())


# ----------------------------------------------------------------------------
# label runs (Segmentation section: each cell's voxels, passed to the hulls)
# ----------------------------------------------------------------------------

def runs_bruteforce(lab):
    """Voxel by voxel: a run opens at a non-zero voxel whose left neighbour in
    the row differs, and every further voxel of equal label extends it."""
    X = lab.shape[-1]
    flat = lab.reshape(-1, X)
    out = []
    for row in range(flat.shape[0]):
        for x in range(X):
            v = int(flat[row, x])
            if v == 0:
                continue
            if x > 0 and int(flat[row, x - 1]) == v:
                out[-1][3] = x
            else:
                out.append([v, row, x, x])
    return out


def test_label_runs_brute_force_and_repaint():
    rng = np.random.default_rng(96)
    for shape in [(1, 1, 1), (1, 1, 9), (3, 4, 1), (2, 5, 17), (4, 3, 33)]:
        # few labels, zeros and equal neighbours, so runs of every length and
        # adjacent runs of different labels occur
        lab = rng.choice([0, 0, 0, 1, 2, 2, 3], size=shape).astype(np.uint32)
        got = oracle.label_runs(lab)
        want = runs_bruteforce(lab)
        assert [list(map(int, r)) for r in got] == want, shape
        # painting the runs back gives the label image
        X = shape[-1]
        paint = np.zeros(lab.size, np.uint32)
        for r in got:
            paint[int(r["row"]) * X + int(r["x_begin"]): int(r["row"]) * X + int(r["x_end"]) + 1] = r["label"]
        assert np.array_equal(paint.reshape(shape), lab)
    assert len(oracle.label_runs(np.zeros((3, 4, 5), np.uint32))) == 0
    full = np.full((2, 2, 6), 9, np.uint32)
    assert [tuple(map(int, r)) for r in oracle.label_runs(full)] == [(9, k, 0, 5) for k in range(4)]


def test_label_runs_carry_the_cell_features():
    # per cell, the run lengths add up to the cell's voxel count and the run
    # ends span its bounding box
    vol = synth.single_frame()
    r = oracle.segment(vol, min_volume=30)
    runs = oracle.label_runs(r.labels)
    Z, Y, X = vol.shape
    ln = runs["x_end"].astype(np.int64) - runs["x_begin"] + 1
    cnt = np.bincount(runs["label"], weights=ln, minlength=r.n_cells + 1)
    assert np.array_equal(cnt[1:].astype(np.uint64), r.cells["count"])
    for k in range(1, r.n_cells + 1):
        sel = runs[runs["label"] == k]
        y, z = sel["row"] % Y, sel["row"] // Y
        assert sel["x_begin"].min() == r.cells["bbox_min"][k - 1][0]
        assert sel["x_end"].max() == r.cells["bbox_max"][k - 1][0]
        assert (y.min(), z.min()) == tuple(r.cells["bbox_min"][k - 1][1:])
        assert (y.max(), z.max()) == tuple(r.cells["bbox_max"][k - 1][1:])
