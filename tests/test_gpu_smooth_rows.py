"""The smoothing kernel for row-aligned volumes (X % 8 == 0 with a 16-byte
aligned input, or an even X >= 10 with a 4-byte aligned input) against the
oracle: the smoothed image element by element (contexts
created with SEG_KEEP_SMOOTHED, read with seg_read_smoothed), then labels,
cells and t*.

The kernel sums the five rows of the y pass on packed 16-bit pairs, which is
exact while every raw value is below 4096, and a warp redoes a plane in
32-bit lanes when one of its values is not; x-neighbours come from the
neighbouring lanes, from the staged plane at a warp's ends, from the edge
voxel, or (x-tiled rows, X > 512) from halo chunks.  It also stores each mask
word's largest value, so that the threshold pass reads only the words above
t*.  The cases cover every tile shape class (one octet per row up to 64, rows
wider than a tile, a last x-tile of one octet), values at and above 4096
placed in a tile's own rows, in the halo rows shared with the next tile and
in the x-halo columns, planes split into z-chunks, rows of 256 .. 2048 voxels
over several row tiles (the word-maximum threshold pass), and batches that
mix these volumes with ones the other smoothing kernel takes (ragged X,
unaligned device input)."""
import numpy as np
import pytest

import oracle
from gpu_util import assert_matches_oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def seg():
    import torch
    assert torch.cuda.is_available()
    import paper_1407_2089_gb300 as seg
    return seg


@pytest.fixture(scope="module")
def ctx(seg):
    c = seg.seg_create(device=0, flags=seg.SEG_KEEP_SMOOTHED)
    yield c
    seg.seg_destroy(c)


def noisy(dims, seed, n_blobs=6, lo=1200, hi=3000):
    X, Y, Z = dims
    rng = np.random.default_rng(seed)
    v = rng.normal(200, 20, size=(Z, Y, X)).clip(0, 65535).astype(np.uint16)
    for _ in range(n_blobs):
        c = rng.integers(0, [Z, Y, X])
        r = rng.integers(1, 6, size=3)
        sl = tuple(slice(max(0, c[i] - r[i]), c[i] + r[i] + 1) for i in range(3))
        v[sl] = rng.integers(lo, hi)
    return v


def check(seg, c, vols, m=5, what=""):
    """Submits vols (host arrays) in one batch; compares each channel's
    smoothed image, labels, cells and t* with the oracle."""
    reqs = [seg.seg_submit_volume(c, v, min_volume=m) for v in vols]
    seg.seg_flush(c)
    for k, (v, r) in enumerate(zip(vols, reqs)):
        assert seg.seg_wait(c, r) == seg.SEG_DONE
        ref = oracle.segment(v, min_volume=m, keep_smoothed=True)
        sm = np.empty(v.shape, np.uint16)
        seg.seg_read_smoothed(c, r, 0, sm)
        if not np.array_equal(sm, ref.smoothed):
            d = np.argwhere(sm != ref.smoothed)
            raise AssertionError("%s #%d %s: %d smoothed voxels differ, first (z, y, x) %s: %d vs %d" % (
                what, k, v.shape, len(d), tuple(d[0]), sm[tuple(d[0])], ref.smoothed[tuple(d[0])]))
        lab = np.empty(v.shape, np.uint32)
        seg.seg_read_labels(c, r, 0, lab)
        cells, thr = seg.seg_read_features(c, r, 0)
        assert_matches_oracle(v, lab, cells, thr, min_volume=m, ref=ref, what="%s #%d %s" % (what, k, v.shape))
        seg.seg_release(c, r)


# (X, Y, Z): one octet per row (a 512-row tile), 25 and 31 octets per row
# (tiles of 20 and 16 rows, idle threads), full 512-voxel rows, rows wider
# than a tile with a last x-tile of 1 octet, 2 tiles, several tiles.
SHAPES = [(8, 1, 1), (8, 3, 2), (16, 40, 3), (64, 16, 5), (128, 70, 21), (200, 33, 9), (248, 5, 70),
          (512, 20, 9), (520, 11, 7), (1024, 9, 6), (1032, 17, 5), (1544, 5, 3)]


@pytest.mark.parametrize("dims", SHAPES)
def test_packed_path_shapes(seg, ctx, dims):
    check(seg, ctx, [noisy(dims, sum(dims), n_blobs=max(2, dims[0] * dims[1] * dims[2] // 3000))],
          what="packed")


def test_values_at_and_above_4096(seg, ctx):
    # 4095 keeps the packed sums at most 16 * 4095 per lane; 4096 and above
    # send the plane through the 32-bit y pass
    vols = []
    for dims, val in [((64, 16, 5), 4095), ((64, 16, 5), 4096), ((512, 20, 9), 40000), ((1032, 17, 5), 65535)]:
        X, Y, Z = dims
        v = noisy(dims, X + val)
        v[Z // 2, Y // 3, X // 5] = val
        v[Z // 2, Y // 3, X // 5 + 1] = val
        vols.append(v)
    vols.append(np.full((6, 10, 64), 65535, np.uint16))
    rng = np.random.default_rng(11)
    vols.append(rng.integers(0, 65536, size=(7, 19, 520), dtype=np.uint16))
    check(seg, ctx, vols, what="high values")


def test_high_values_in_halo_rows_and_columns(seg, ctx):
    # X = 512: tiles of 8 rows; a bright row that only the neighbouring tile
    # stages as halo (y = 8, 9 are halo rows of the tile y < 8; y = 6, 7 of
    # the tile y >= 8).  X = 1024: two x-tiles; bright voxels at x = 510, 511
    # (the right tile's left halo word) and x = 512, 513 (the left tile's
    # right halo word).
    vols = []
    for y in (6, 7, 8, 9):
        v = noisy((512, 24, 6), 100 + y, n_blobs=2)
        v[3, y, 100:104] = 30000
        vols.append(v)
    for x in (510, 511, 512, 513):
        v = noisy((1024, 12, 5), 200 + x, n_blobs=2)
        v[2, 5, x] = 50000
        vols.append(v)
    # the halo planes of a z-chunk: the only bright plane just outside a chunk
    v = noisy((64, 64, 300), 7, n_blobs=20)
    v[8, 30, 30] = 60000
    v[7, 31, 33] = 9000
    vols.append(v)
    check(seg, ctx, vols, m=1, what="halo")


def test_z_chunks_and_tall_volumes(seg, ctx):
    # a lone volume is cut into z-chunks so that every multiprocessor gets
    # tiles; chunks meet with two-plane halos
    check(seg, ctx, [noisy((64, 64, 300), 3, n_blobs=60)], what="z-chunks")
    check(seg, ctx, [noisy((8, 700, 40), 4, n_blobs=20)], what="one octet, tall")


def test_mixed_batch_with_other_kernel(seg):
    import torch
    c = seg.seg_create(device=0, flags=seg.SEG_KEEP_SMOOTHED, batch_window_us=10_000_000)
    try:
        vols = [noisy((512, 40, 12), 1), noisy((100, 37, 20), 2), noisy((1024, 16, 8), 3),
                noisy((33, 200, 9), 4), noisy((64, 64, 64), 5), noisy((520, 9, 3), 6)]
        check(seg, c, vols, what="mixed")
        # an aligned row width from a device pointer 2 bytes off 16 bytes
        v = noisy((512, 30, 10), 9)
        buf = torch.zeros(v.size + 8, dtype=torch.int16, device="cuda")
        buf[1:1 + v.size] = torch.from_numpy(v.view(np.int16).ravel().copy()).cuda()
        t = buf[1:1 + v.size]
        assert t.data_ptr() % 16 == 2
        r = seg.seg_submit_volume(c, t, dims=(512, 30, 10), channels=1, min_volume=5)
        seg.seg_flush(c)
        assert seg.seg_wait(c, r) == seg.SEG_DONE
        ref = oracle.segment(v, min_volume=5, keep_smoothed=True)
        sm = np.empty(v.shape, np.uint16)
        seg.seg_read_smoothed(c, r, 0, sm)
        assert np.array_equal(sm, ref.smoothed)
        lab = np.empty(v.shape, np.uint32)
        seg.seg_read_labels(c, r, 0, lab)
        cells, thr = seg.seg_read_features(c, r, 0)
        assert_matches_oracle(v, lab, cells, thr, min_volume=5, ref=ref, what="unaligned device input")
        seg.seg_release(c, r)
    finally:
        seg.seg_destroy(c)


def test_word_maxima_threshold_many_row_tiles(seg):
    # rows of 256 .. 2048 voxels take the threshold pass that reads only the
    # mask words whose maximum is above t*; several row tiles of 256 rows
    # per volume, in one batch and alone
    c = seg.seg_create(device=0, flags=seg.SEG_KEEP_SMOOTHED, batch_window_us=10_000_000)
    try:
        vols = [noisy((256, 300, 3), 21, n_blobs=30), noisy((512, 130, 4), 22, n_blobs=30),
                noisy((1024, 150, 3), 23, n_blobs=40), noisy((2048, 200, 2), 24, n_blobs=50)]
        check(seg, c, vols, m=1, what="word maxima, batch")
        for v in vols:
            check(seg, c, [v], m=1, what="word maxima, alone")
    finally:
        seg.seg_destroy(c)


def test_otsu_flat_maxima(seg, ctx):
    # Histograms whose between-class variance is nearly flat around its
    # maximum (unimodal noise of many widths, two modes of nearly equal
    # weight, a few isolated levels): many levels come close to the maximum,
    # so the binary64 Otsu sweep must still pick the oracle's level among
    # them.  Row-aligned and ragged shapes (both smoothing kernels).  The
    # uniform 16-bit noise and the ramp occupy 10000 to 65000 levels, more
    # than the Otsu kernel lists in shared memory (its per-thread path); the
    # others occupy 4 to 1400 (its listed path).
    rng = np.random.default_rng(123)
    vols = []
    for dims in [(64, 40, 9), (67, 40, 9), (256, 33, 5)]:
        X, Y, Z = dims
        for lo, hi in [(0, 65536), (1000, 1100), (30000, 30008), (0, 4096)]:
            vols.append(rng.integers(lo, hi, size=(Z, Y, X), dtype=np.uint16))
        a = np.full((Z, Y, X), 500, np.uint16)
        a[:, :, X // 2:] = 3000
        a[:, Y // 2:, :] += rng.integers(0, 3, size=(Z, Y - Y // 2, X), dtype=np.uint16)
        vols.append(a)
        b = rng.normal(800, 30, size=(Z, Y, X)).clip(0, 65535).astype(np.uint16)
        b[: Z // 2] = rng.normal(2000, 30, size=(Z // 2, Y, X)).clip(0, 65535).astype(np.uint16)
        vols.append(b)
    # a ramp through all 65536 values: the smoothing keeps its interior, so
    # almost every level is occupied about equally (the variance peaks in the
    # middle, where neighbouring levels come within rounding of each other)
    X, Y, Z = 256, 256, 3
    r = (np.arange(Y)[:, None] * X + np.arange(X)[None, :]).astype(np.uint16)
    vols.append(np.broadcast_to(r, (Z, Y, X)).copy())
    check(seg, ctx, vols, m=1, what="flat Otsu maxima")


def test_time_lapse_frame_smoothed(seg, ctx):
    import synth
    tl = synth.TimeLapse()
    check(seg, ctx, [tl.frame(5, 0), tl.frame(5, 1)], m=30, what="time-lapse")


# Even X that is not a multiple of 8: 4-byte copies and stores, a partial
# last octet of 2, 4 or 6 voxels whose missing neighbours repeat the last
# voxel; rows narrower than a tile (one tile row, several rows per tile, tile
# rows of 2 .. 64 octets), just below and above 512 (x-tiled rows with a
# partial last tile), and the montage's row width.  The threshold pass reads
# the word maxima with voxel pairs for these widths.
RAGGED_EVEN = [(10, 7, 3), (14, 40, 5), (18, 3, 9), (26, 33, 4), (34, 20, 6), (100, 17, 5), (250, 12, 7),
               (254, 9, 4), (506, 8, 5), (510, 11, 3), (514, 9, 4), (522, 6, 5), (1030, 7, 3), (2046, 4, 3),
               (5530, 5, 3)]


@pytest.mark.parametrize("dims", RAGGED_EVEN)
def test_ragged_even_rows(seg, ctx, dims):
    X, Y, Z = dims
    v = noisy(dims, X + 7 * Y + Z, n_blobs=max(3, X * Y * Z // 2000))
    # bright voxels at the row's last columns (the partial octet and its
    # left neighbour) and one value above 4096 there
    v[Z // 2, Y // 2, X - 1] = 3000
    v[Z // 2, Y // 2, X - 2] = 2800
    v[Z - 1, Y - 1, X - 3] = 50000
    check(seg, ctx, [v], m=1, what="ragged even")


def test_ragged_even_batch_and_alignment(seg):
    import torch
    c = seg.seg_create(device=0, flags=seg.SEG_KEEP_SMOOTHED, batch_window_us=10_000_000)
    try:
        # ragged and aligned widths and the other smoothing kernel (odd X)
        # in one batch; many row tiles per volume
        vols = [noisy((130, 200, 6), 31, n_blobs=30), noisy((512, 40, 5), 32), noisy((5530, 12, 3), 33, n_blobs=20),
                noisy((33, 50, 7), 34), noisy((1030, 60, 4), 35, n_blobs=25)]
        check(seg, c, vols, m=1, what="ragged batch")
        # device input 4 bytes off a 16-byte boundary (the 4-byte copies) and
        # 2 bytes off (the other smoothing kernel)
        for off in (2, 1):
            v = noisy((130, 30, 6), 40 + off)
            buf = torch.zeros(v.size + 16, dtype=torch.int16, device="cuda")
            buf[off:off + v.size] = torch.from_numpy(v.view(np.int16).ravel().copy()).cuda()
            t = buf[off:off + v.size]
            assert t.data_ptr() % 16 == 2 * off
            r = seg.seg_submit_volume(c, t, dims=(130, 30, 6), channels=1, min_volume=1)
            seg.seg_flush(c)
            assert seg.seg_wait(c, r) == seg.SEG_DONE
            ref = oracle.segment(v, min_volume=1, keep_smoothed=True)
            sm = np.empty(v.shape, np.uint16)
            seg.seg_read_smoothed(c, r, 0, sm)
            assert np.array_equal(sm, ref.smoothed)
            lab = np.empty(v.shape, np.uint32)
            seg.seg_read_labels(c, r, 0, lab)
            cells, thr = seg.seg_read_features(c, r, 0)
            assert_matches_oracle(v, lab, cells, thr, min_volume=1, ref=ref, what="device input offset %d" % (2 * off))
            seg.seg_release(c, r)
    finally:
        seg.seg_destroy(c)


def test_read_smoothed_needs_the_flag(seg):
    c = seg.seg_create(device=0)
    try:
        v = noisy((64, 8, 4), 1)
        r = seg.seg_submit_volume(c, v)
        seg.seg_flush(c)
        assert seg.seg_wait(c, r) == seg.SEG_DONE
        with pytest.raises(seg.SegError) as e:
            seg.seg_read_smoothed(c, r, 0, np.empty(v.shape, np.uint16))
        assert e.value.code == seg.SEG_EINVAL
        seg.seg_release(c, r)
    finally:
        seg.seg_destroy(c)
