"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle,
bit-exact on labels, cells and the Otsu level, on seeded synthetic inputs."""
import numpy as np
import pytest

import oracle
import synth
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
    c = seg.seg_create(device=0)
    yield c
    seg.seg_destroy(c)


def blobs(dims, seed, n=6, density_noise=(200, 20)):
    """Noise plus a few bright boxes and balls of random sizes (ragged, touching edges)."""
    X, Y, Z = dims
    rng = np.random.default_rng(seed)
    v = rng.normal(density_noise[0], density_noise[1], size=(Z, Y, X)).clip(0, 65535).astype(np.uint16)
    for _ in range(n):
        c = rng.integers(0, [Z, Y, X])
        r = rng.integers(1, 6, size=3)
        sl = tuple(slice(max(0, c[i] - r[i]), c[i] + r[i] + 1) for i in range(3))
        v[sl] = rng.integers(1200, 3000)
    return v


def run(seg, ctx, vol, m=30):
    (lab, cells, thr), = seg.segment(ctx, vol, min_volume=m)
    return lab, cells, thr


def test_single_frame_workload(seg, ctx):
    vol = synth.single_frame()
    lab, cells, thr = run(seg, ctx, vol)
    ref = assert_matches_oracle(vol, lab, cells, thr, what="single frame")
    assert ref.n_cells >= 30


# Row counts Y*Z that take each row-tile size on a 152-multiprocessor GPU: a
# batch with fewer than two row tiles per multiprocessor halves its tile
# (256 rows) down to 32, so the run kernels still fill the GPU.  Tall, narrow
# volumes with many runs per tile and cells that cross tile boundaries.
@pytest.mark.parametrize("dims", [(8, 100, 900), (16, 300, 200), (32, 200, 150), (40, 64, 100), (7, 33, 20)])
def test_row_tile_sizes(seg, ctx, dims):
    X, Y, Z = dims
    rng = np.random.default_rng(X * Y + Z)
    vol = rng.normal(300, 30, size=(Z, Y, X)).clip(0, 65535).astype(np.uint16)
    for _ in range(Y * Z // 400):
        c = rng.integers(0, [Z, Y, X])
        r = rng.integers(1, 4, size=3)
        sl = tuple(slice(max(0, c[i] - r[i]), c[i] + r[i] + 1) for i in range(3))
        vol[sl] = rng.integers(1500, 3000)
    for m in (1, 10):
        lab, cells, thr = run(seg, ctx, vol, m)
        assert_matches_oracle(vol, lab, cells, thr, min_volume=m, what="%s m=%d" % (dims, m))


@pytest.mark.parametrize("dims", [(1, 1, 1), (5, 3, 2), (31, 1, 7), (33, 40, 3), (64, 16, 5),
                                  (65, 17, 9), (130, 70, 21), (200, 3, 66), (97, 131, 40)])
def test_ragged_shapes(seg, ctx, dims):
    vol = blobs(dims, sum(dims), n=max(1, dims[0] * dims[1] * dims[2] // 4000))
    for m in (1, 30):
        lab, cells, thr = run(seg, ctx, vol, m)
        assert_matches_oracle(vol, lab, cells, thr, min_volume=m, what="%s m=%d" % (dims, m))


def test_dense_random_masks(seg, ctx):
    # high-density foreground: many runs per row, heavy union traffic
    rng = np.random.default_rng(5)
    for p in (0.3, 0.5, 0.7):
        vol = np.where(rng.uniform(size=(24, 50, 77)) < p, 3000, 100).astype(np.uint16)
        lab, cells, thr = run(seg, ctx, vol, 1)
        assert_matches_oracle(vol, lab, cells, thr, min_volume=1, what="p=%.1f" % p)


def test_blank_and_two_level_volumes(seg, ctx):
    for c in (0, 200, 65535):
        vol = np.full((9, 10, 11), c, dtype=np.uint16)
        lab, cells, thr = run(seg, ctx, vol)
        assert thr == c and len(cells) == 0 and not lab.any()
    vol = np.zeros((20, 30, 40), dtype=np.uint16)
    vol[5:15, 5:25, 10:30] = 65535
    lab, cells, thr = run(seg, ctx, vol, 1)
    assert_matches_oracle(vol, lab, cells, thr, min_volume=1, what="two-level")


def test_wide_rows_reach_65536(seg, ctx):
    rng = np.random.default_rng(8)
    vol = rng.normal(200, 20, size=(3, 2, 65536)).clip(0, 65535).astype(np.uint16)
    vol[:, :, 65500:] = 4000
    vol[:, :, 100:140] = 4000
    lab, cells, thr = run(seg, ctx, vol, 1)
    assert_matches_oracle(vol, lab, cells, thr, min_volume=1, what="X=65536")


@pytest.mark.parametrize("ty,tz", [(16, 1), (16, 7), (32, 3), (32, 64), (64, 5), (64, 200)])
def test_tile_shape_invariance(seg, ty, tz):
    c = seg.seg_create(device=0, flags=seg.SEG_FORCE_TILE, tile_y=ty, tile_z=tz)
    try:
        for dims in [(130, 70, 21), (64, 64, 64)]:
            vol = blobs(dims, 99 + tz, n=12)
            lab, cells, thr = run(seg, c, vol, 5)
            assert_matches_oracle(vol, lab, cells, thr, min_volume=5, what="tile %d/%d %s" % (ty, tz, dims))
    finally:
        seg.seg_destroy(c)


def test_time_lapse_frame_both_channels(seg, ctx):
    tl = synth.TimeLapse()
    vol = np.stack([tl.frame(3, 0), tl.frame(3, 1)])
    res = seg.segment(ctx, vol, min_volume=30)
    for c in range(2):
        lab, cells, thr = res[c]
        assert_matches_oracle(vol[c], lab, cells, thr, what="time-lapse ch%d" % c)


def test_batch_of_uneven_volumes_in_one_launch(seg):
    c = seg.seg_create(device=0, batch_window_us=10_000_000)
    try:
        dims = [(64, 64, 64), (100, 37, 20), (33, 200, 9), (256, 256, 40), (1, 1, 1), (5, 300, 2)]
        vols = [blobs(d, i, n=10) for i, d in enumerate(dims)]
        reqs = [seg.seg_submit_volume(c, v, min_volume=3) for v in vols]
        seg.seg_flush(c)
        for v, r in zip(vols, reqs):
            assert seg.seg_wait(c, r) == seg.SEG_DONE
            lab = np.empty(v.shape, dtype=np.uint32)
            seg.seg_read_labels(c, r, 0, lab)
            cells, thr = seg.seg_read_features(c, r, 0)
            assert_matches_oracle(v, lab, cells, thr, min_volume=3, what="batch %s" % (v.shape,))
            seg.seg_release(c, r)
        st = seg.seg_get_stats(c)
        assert st["batches"] == 1 and st["volumes"] == len(dims)
    finally:
        seg.seg_destroy(c)


def test_device_resident_input(seg, ctx):
    import torch
    vol = synth.single_frame()
    t = torch.from_numpy(vol.view(np.int16).copy()).cuda()
    req = seg.seg_submit_volume(ctx, t, dims=(vol.shape[2], vol.shape[1], vol.shape[0]), channels=1)
    seg.seg_flush(ctx)
    assert seg.seg_wait(ctx, req) == seg.SEG_DONE
    out = torch.empty(vol.size, dtype=torch.int32, device="cuda")
    seg.seg_read_labels(ctx, req, 0, out)
    cells, thr = seg.seg_read_features(ctx, req, 0)
    lab = out.cpu().numpy().view(np.uint32).reshape(vol.shape)
    assert_matches_oracle(vol, lab, cells, thr, what="device input")
    seg.seg_release(ctx, req)


def test_queued_host_input(seg):
    # host inputs whose copies are only queued (keep_host_input): pinned and
    # pageable sources, several requests in one batch, each equal to the oracle
    import ctypes
    import torch
    c = seg.seg_create(device=0, batch_window_us=30_000_000)
    try:
        vols = [blobs((70, 40, 9), 40 + k, n=10) for k in range(4)]
        srcs = [torch.from_numpy(v.view(np.int16).copy()).pin_memory() if k % 2 == 0 else v
                for k, v in enumerate(vols)]
        reqs = [seg.seg_submit_volume(c, s_, min_volume=5, keep_host_input=True) for s_ in srcs]
        seg.seg_flush(c)
        for k, (v, r) in enumerate(zip(vols, reqs)):
            assert seg.seg_wait(c, r) == seg.SEG_DONE
            lab = np.empty(v.shape, np.uint32)
            seg.seg_read_labels(c, r, 0, lab)
            cells, thr = seg.seg_read_features(c, r, 0)
            assert_matches_oracle(v, lab, cells, thr, min_volume=5, what="queued input %d" % k)
            seg.seg_release(c, r)
        # input modes other than 0, 1, 2 are rejected
        out = ctypes.c_uint64()
        for mode in (-1, 3):
            rc = seg._lib.seg_submit_volume(c, ctypes.c_void_p(vols[0].ctypes.data), mode,
                                            seg.seg_dims(70, 40, 9), 1, None, ctypes.byref(out))
            assert rc == seg.SEG_EINVAL, mode
    finally:
        seg.seg_destroy(c)


def test_union_find_stress(seg, ctx):
    # dense random masks in many shapes: every missed or wrong union changes
    # the labels (m = 1 keeps every fragment), so races show up here
    rng = np.random.default_rng(77)
    for trial in range(40):
        dims = tuple(int(v) for v in rng.integers(3, 90, size=3))
        X, Y, Z = dims
        p = float(rng.uniform(0.2, 0.6))
        vol = np.where(rng.uniform(size=(Z, Y, X)) < p, 3000, 100).astype(np.uint16)
        lab, cells, thr = run(seg, ctx, vol, 1)
        assert_matches_oracle(vol, lab, cells, thr, min_volume=1, what="stress %d %s p=%.2f" % (trial, dims, p))


def brick_run_counts(mask, by=32, bz=8):
    """x-runs per brick of by x bz rows of a [Z][Y][X] boolean mask."""
    starts = mask & ~np.concatenate([np.zeros_like(mask[..., :1]), mask[..., :-1]], axis=-1)
    per_row = starts.sum(axis=-1)  # [Z][Y]
    Z, Y = per_row.shape
    out = []
    for z0 in range(0, Z, bz):
        for y0 in range(0, Y, by):
            out.append(int(per_row[z0:z0 + bz, y0:y0 + by].sum()))
    return out


def test_union_bricks_shared_and_overflow(seg, ctx):
    # Bricks of 32 x 8 rows unite their runs in shared memory when they hold
    # at most 4096 runs; denser bricks go through the global union-find.  Here
    # stripes (period 8 along x) fill the bricks at y < 32, z < 8 with more
    # runs than that, blobs elsewhere cross brick faces, and the stripes'
    # components reach into neighbouring bricks.
    X, Y, Z = 300, 70, 20
    rng = np.random.default_rng(21)
    vol = rng.normal(100, 10, size=(Z, Y, X)).clip(0, 65535).astype(np.uint16)
    xs = np.arange(X)
    vol[:8, :32, :] = np.where((xs % 8) < 4, 3000, 100).astype(np.uint16)
    for c in [(8, 32, 50), (7, 31, 200), (15, 60, 280), (3, 45, 10), (12, 20, 150)]:
        z, y, x = c
        vol[max(0, z - 3):z + 4, max(0, y - 4):y + 5, max(0, x - 5):x + 6] = 2500
    ref = oracle.segment(vol, min_volume=1, keep_smoothed=True)
    counts = brick_run_counts(ref.smoothed > ref.threshold)
    assert max(counts) > 4096 and 0 < min(c for c in counts if c) <= 4096, counts
    lab, cells, thr = run(seg, ctx, vol, 1)
    assert_matches_oracle(vol, lab, cells, thr, min_volume=1, ref=ref, what="bricks")
