"""GPU parity of the label runs read (Segmentation section: each cell's
voxels, the set passed on to the convex hull step) against the oracle: the
runs of the label image bit for bit, in order, for host and device
destinations, ragged rows, empty and full rows and the widest rows."""
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


def blobs(dims, seed, n=6):
    """Noise N(200, 20) plus bright boxes; some reach the row ends."""
    X, Y, Z = dims
    rng = np.random.default_rng(seed)
    v = rng.normal(200, 20, size=(Z, Y, X))
    for k in range(n):
        c = rng.integers(0, [Z, Y, X])
        h = rng.integers(1, 4, size=3)
        sl = tuple(slice(max(0, c[i] - h[i]), c[i] + h[i] + 1) for i in range(3))
        v[sl] += 1500
    if X > 4:
        v[:, : max(1, Y // 3), X - 3:] += 1500  # runs ending at x = X - 1
    return np.rint(v).clip(0, 65535).astype(np.uint16)


def runs_of(seg, ctx, vol, min_volume=1, **kw):
    req = seg.seg_submit_volume(ctx, vol, min_volume=min_volume, **kw)
    seg.seg_flush(ctx)
    try:
        assert seg.seg_wait(ctx, req) == seg.SEG_DONE
        lab = np.empty(vol.shape, np.uint32)
        seg.seg_read_labels(ctx, req, 0, lab)
        cells, thr = seg.seg_read_features(ctx, req, 0)
        runs = seg.seg_read_label_runs(ctx, req, 0)
    finally:
        seg.seg_release(ctx, req)
    return lab, cells, thr, runs


def assert_runs_equal(got, want, what=""):
    assert got.dtype.itemsize == 12 and len(got) == len(want), "%s: %d runs vs %d" % (what, len(got), len(want))
    for f in ("label", "row", "x_begin", "x_end"):
        if not np.array_equal(got[f], want[f]):
            i = int(np.nonzero(got[f] != want[f])[0][0])
            raise AssertionError("%s: field %s differs first at run %d (gpu %s, oracle %s)" % (
                what, f, i, got[i], want[i]))


@pytest.mark.parametrize("dims", [(1, 1, 1), (7, 3, 2), (31, 9, 4), (32, 8, 5), (33, 17, 3), (64, 20, 6),
                                  (100, 13, 7), (256, 5, 3), (257, 6, 4), (300, 70, 3)])
def test_ragged_shapes(seg, ctx, dims):
    # rows cut at every remainder of 32 and 256, more than one block of rows
    vol = blobs(dims, sum(dims))
    lab, cells, thr, runs = runs_of(seg, ctx, vol)
    ref = assert_matches_oracle(vol, lab, cells, thr, min_volume=1, what=str(dims))
    assert_runs_equal(runs, oracle.label_runs(ref.labels), str(dims))


def test_empty_and_full(seg, ctx):
    # constant volume: one level, nothing above t*, no runs
    lab, _, _, runs = runs_of(seg, ctx, np.full((5, 6, 40), 300, np.uint16))
    assert not lab.any() and len(runs) == 0
    # two levels, the upper one filling whole rows: one run per row
    vol = np.full((3, 4, 70), 100, np.uint16)
    vol[1:, :, :] = 2000
    lab, _, _, runs = runs_of(seg, ctx, vol)
    assert_runs_equal(runs, oracle.label_runs(lab), "full rows")
    assert len(runs) > 0 and (runs["x_end"] - runs["x_begin"] == 69).all()


def test_widest_rows(seg, ctx):
    # X = 65536: x_end reaches the top of its 16-bit field
    vol = blobs((65536, 1, 2), 5, n=40)
    lab, cells, thr, runs = runs_of(seg, ctx, vol)
    ref = assert_matches_oracle(vol, lab, cells, thr, min_volume=1, what="X=65536")
    want = oracle.label_runs(ref.labels)
    assert_runs_equal(runs, want, "X=65536")
    assert want["x_end"].max() == 65535


def test_destinations_and_sizes(seg, ctx):
    import torch
    vol = blobs((90, 40, 8), 11, n=12)
    req = seg.seg_submit_volume(ctx, vol, min_volume=1)
    seg.seg_flush(ctx)
    try:
        assert seg.seg_wait(ctx, req) == seg.SEG_DONE
        lab = np.empty(vol.shape, np.uint32)
        seg.seg_read_labels(ctx, req, 0, lab)
        want = oracle.label_runs(lab)
        n = len(want)
        assert n > 10
        # exact-size numpy, oversized numpy (returns the first n), host and device tensors
        assert_runs_equal(seg.seg_read_label_runs(ctx, req, 0, np.zeros(n, seg.LABEL_RUN_DTYPE)), want, "exact")
        assert_runs_equal(seg.seg_read_label_runs(ctx, req, 0, np.zeros(n + 50, seg.LABEL_RUN_DTYPE)), want, "big")
        # pageable host, pinned host (written through its device mapping) and
        # device tensors, exact and oversized
        for kind in ("cpu", "pinned", "cuda:0"):
            for extra in (0, 3, 10_000):
                t = torch.zeros(12 * (n + extra), dtype=torch.uint8, device="cuda:0" if kind == "cuda:0" else "cpu")
                if kind == "pinned":
                    t = t.pin_memory()
                got = seg.seg_read_label_runs(ctx, req, 0, t)
                assert got.numel() == 12 * n
                assert_runs_equal(got.cpu().numpy().view(seg.LABEL_RUN_DTYPE), want, "%s +%d" % (kind, extra))
                assert not t[12 * n:].any(), kind  # nothing past the runs
        # too small: SEG_ESMALL and nothing written, for every kind of destination
        small = np.zeros(n - 1, seg.LABEL_RUN_DTYPE)
        with pytest.raises(seg.SegError) as e:
            seg.seg_read_label_runs(ctx, req, 0, small)
        assert e.value.code == seg.SEG_ESMALL
        assert not small["label"].any()
        for kind in ("pinned", "cuda:0"):
            t = torch.zeros(12 * (n - 1), dtype=torch.uint8, device="cuda:0" if kind == "cuda:0" else "cpu")
            if kind == "pinned":
                t = t.pin_memory()
            with pytest.raises(seg.SegError) as e:
                seg.seg_read_label_runs(ctx, req, 0, t)
            assert e.value.code == seg.SEG_ESMALL and not t.any(), kind
        with pytest.raises(seg.SegError) as e:
            seg.seg_read_label_runs(ctx, req, 1, None)
        assert e.value.code == seg.SEG_EINVAL
    finally:
        seg.seg_release(ctx, req)


def test_mixed_batch(seg):
    # several requests and channels in one batch, with the closing on one
    c = seg.seg_create(device=0, batch_window_us=30_000_000)
    try:
        a = np.stack([blobs((60, 30, 10), 21), blobs((60, 30, 10), 22)])
        b = blobs((45, 33, 7), 23)
        ra = seg.seg_submit_volume(c, a, min_volume=[3, 5], closing_radius=[0, 1])
        rb = seg.seg_submit_volume(c, b, min_volume=2)
        seg.seg_flush(c)
        for r in (ra, rb):
            assert seg.seg_wait(c, r) == seg.SEG_DONE
        for req, ch, vol, kw in [(ra, 0, a[0], dict(min_volume=3)), (ra, 1, a[1], dict(min_volume=5, closing_radius=1)),
                                 (rb, 0, b, dict(min_volume=2))]:
            ref = oracle.segment(vol, **kw)
            assert_runs_equal(seg.seg_read_label_runs(c, req, ch), oracle.label_runs(ref.labels), "ch%d" % ch)
        for r in (ra, rb):
            seg.seg_release(c, r)
    finally:
        seg.seg_destroy(c)


def test_time_lapse_frame_full_size(seg, ctx):
    # both channels of a 512 x 512 x 64 frame of the time-lapse workload
    tl = synth.TimeLapse(frames=1)
    vol = np.stack([tl.frame(0, 0), tl.frame(0, 1)])
    req = seg.seg_submit_volume(ctx, vol, min_volume=30)
    seg.seg_flush(ctx)
    try:
        assert seg.seg_wait(ctx, req) == seg.SEG_DONE
        for ch in range(2):
            ref = oracle.segment(vol[ch], min_volume=30)
            runs = seg.seg_read_label_runs(ctx, req, ch)
            assert_runs_equal(runs, oracle.label_runs(ref.labels), "frame ch%d" % ch)
            # the runs carry the cells: voxel counts per label
            ln = runs["x_end"].astype(np.int64) - runs["x_begin"] + 1
            cnt = np.bincount(runs["label"], weights=ln, minlength=ref.n_cells + 1)[1:]
            assert np.array_equal(cnt.astype(np.uint64), ref.cells["count"])
    finally:
        seg.seg_release(ctx, req)
