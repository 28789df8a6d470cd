"""GPU parity of the distance map of the final foreground (Segmentation
section: distance from every voxel to the nearest foreground voxel, here the
exact weighted squared Euclidean distance) against the oracle, bit-exact."""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import assert_matches_oracle

pytestmark = pytest.mark.gpu

INF = 0xFFFFFFFF


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


def boxes(dims, seed, n):
    """Noise plus n bright boxes (n = 0: noise only, an empty foreground)."""
    X, Y, Z = dims
    rng = np.random.default_rng(seed)
    v = rng.normal(200, 20, size=(Z, Y, X)).clip(0, 65535).astype(np.uint16)
    for _ in range(n):
        c = rng.integers(0, [Z, Y, X])
        r = rng.integers(1, 5, size=3)
        v[tuple(slice(max(0, c[i] - r[i]), c[i] + r[i] + 1) for i in range(3))] = 3000
    return v


def check(seg, ctx, vol, w, min_volume=1, closing_radius=0, what=""):
    ref = oracle.segment(vol, min_volume=min_volume, closing_radius=closing_radius, distance_weights=w)
    (lab, cells, thr, dist), = seg.segment(ctx, vol, min_volume=min_volume, closing_radius=closing_radius,
                                          distance_weights=w)
    assert_matches_oracle(vol, lab, cells, thr, ref=ref, what=what)
    if not np.array_equal(dist, ref.distance):
        d = np.argwhere(dist != ref.distance)
        raise AssertionError("%s: %d distance mismatches, first at %s (gpu %d, oracle %d)" % (
            what, len(d), tuple(d[0]), dist[tuple(d[0])], ref.distance[tuple(d[0])]))
    return ref


@pytest.mark.parametrize("dims", [(1, 1, 1), (5, 3, 2), (31, 1, 7), (33, 40, 3), (70, 9, 30), (1100, 6, 5),
                                  (64, 64, 16), (40, 300, 4), (9, 512, 3), (5, 700, 3), (4, 1024, 2),
                                  (4, 1100, 2), (40, 7, 80), (33, 9, 100), (35, 5, 200), (3, 5, 257),
                                  (3, 5, 600)])
@pytest.mark.parametrize("w", [(16, 16, 25), (1, 1, 1), (7, 3, 11)])
def test_ragged_shapes(seg, ctx, dims, w):
    # rows of 1..35 mask words (more than one warp chunk); lines along y up to
    # 512 and up to 1024 voxels (the fused x+y kernel's two block shapes) and
    # longer (the long-line kernels); lines along z for each tile height of
    # the z kernel (128, 96, 64 and 32 lines) and longer than 256; sparse
    # foreground (rows, lines and planes without any); unequal weights that
    # catch a swapped axis
    vol = boxes(dims, sum(dims) + w[1], n=3)
    check(seg, ctx, vol, w, what="%s w=%s" % (dims, w))


def test_widest_rows(seg, ctx):
    # X = 65536: x distances no longer fit 16 bits, so the long-line x and y
    # kernels take the volume
    vol = boxes((65536, 1, 1), 17, n=2)
    check(seg, ctx, vol, (1, 1, 1), what="X=65536")


def test_empty_foreground(seg, ctx):
    vol = np.full((20, 10, 6), 500, dtype=np.uint16)  # constant: no voxel above the level
    ref = check(seg, ctx, vol, (16, 16, 25), what="empty")
    assert np.all(ref.distance == INF)


def test_single_foreground_voxel(seg, ctx):
    # one bright voxel among zeros: after smoothing one voxel stays above the
    # level, so the map is the weighted paraboloid around it
    vol = np.zeros((11, 19, 37), dtype=np.uint16)
    vol[5, 7, 30] = 60000
    ref = check(seg, ctx, vol, (7, 3, 11), what="single voxel")
    assert (ref.distance == 0).sum() >= 1


def test_single_frame_with_closing(seg, ctx):
    vol = synth.single_frame()
    for rho in (0, 2):
        check(seg, ctx, vol, (16, 16, 25), min_volume=30, closing_radius=rho, what="single frame rho=%d" % rho)


def test_mixed_batch(seg):
    c = seg.seg_create(device=0, batch_window_us=30_000_000)
    try:
        a = np.stack([boxes((96, 80, 24), 3, 6), boxes((96, 80, 24), 4, 2)])
        b = boxes((64, 64, 40), 5, 4)
        ra = seg.seg_submit_volume(c, a, denoise_radius=[4, 0], closing_radius=[1, 0], min_volume=5,
                                   distance_weights=[None, (16, 16, 25)])
        rb = seg.seg_submit_volume(c, b, closing_radius=1, min_volume=5, distance_weights=(1, 2, 3))
        seg.seg_flush(c)
        assert seg.seg_wait(c, ra) == seg.SEG_DONE and seg.seg_wait(c, rb) == seg.SEG_DONE
        assert seg.seg_get_stats(c)["batches"] == 1
        cases = [(ra, 0, a[0], 4, 1, None), (ra, 1, a[1], 0, 0, (16, 16, 25)), (rb, 0, b, 0, 1, (1, 2, 3))]
        for req, ch, vol, dr, cr, w in cases:
            lab = np.empty(vol.shape, dtype=np.uint32)
            seg.seg_read_labels(c, req, ch, lab)
            cells, thr = seg.seg_read_features(c, req, ch)
            ref = oracle.segment(vol, min_volume=5, denoise_radius=dr, closing_radius=cr, distance_weights=w)
            assert_matches_oracle(vol, lab, cells, thr, ref=ref, what="mixed ch%d" % ch)
            dist = np.empty(vol.shape, dtype=np.uint32)
            if w is None:
                with pytest.raises(seg.SegError) as e:
                    seg.seg_read_distance(c, req, ch, dist)
                assert e.value.code == seg.SEG_EINVAL
            else:
                seg.seg_read_distance(c, req, ch, dist)
                assert np.array_equal(dist, ref.distance), "mixed ch%d" % ch
        seg.seg_release(c, ra)
        seg.seg_release(c, rb)
    finally:
        seg.seg_destroy(c)


def test_device_destination(seg, ctx):
    import torch
    vol = boxes((48, 40, 12), 9, 4)
    req = seg.seg_submit_volume(ctx, vol, min_volume=1, distance_weights=(16, 16, 25))
    seg.seg_flush(ctx)
    try:
        assert seg.seg_wait(ctx, req) == seg.SEG_DONE
        out = torch.empty(vol.shape, dtype=torch.int32, device="cuda:0")
        seg.seg_read_distance(ctx, req, 0, out)
        ref = oracle.segment(vol, min_volume=1, distance_weights=(16, 16, 25))
        assert np.array_equal(out.cpu().numpy().view(np.uint32), ref.distance)
        small = np.empty(10, dtype=np.uint32)
        with pytest.raises(seg.SegError) as e:
            seg.seg_read_distance(ctx, req, 0, small)
        assert e.value.code == seg.SEG_ESMALL
    finally:
        seg.seg_release(ctx, req)


def test_weight_validation(seg, ctx):
    vol = np.zeros((4, 4, 4), dtype=np.uint16)
    for w in [(0, 1, 1), (1, 0, 1), (1, 1, 0), (1 << 30, 1, 1), (1, 1, 0xFFFFFFFF)]:
        with pytest.raises(seg.SegError) as e:
            seg.seg_submit_volume(ctx, vol, distance_weights=w)
        assert e.value.code == seg.SEG_EINVAL, w
    # the largest distance just below the marker is accepted
    req = seg.seg_submit_volume(ctx, vol, distance_weights=((0xFFFFFFFE - 18) // 9, 1, 1))
    seg.seg_flush(ctx)
    assert seg.seg_wait(ctx, req) == seg.SEG_DONE
    seg.seg_release(ctx, req)


def test_vessel_frame_full_size(seg, ctx):
    # the 512 x 512 x 64 vessel channel of the time-lapse workload: exact on
    # sampled voxels (brute force over the oracle's foreground), zero exactly
    # on the foreground, and positive everywhere else
    tl = synth.TimeLapse(frames=1)
    vol = tl.frame(0, 1)
    w = (16, 16, 25)
    ref = oracle.segment(vol, min_volume=30, keep_smoothed=True)
    fg = ref.smoothed > ref.threshold
    (lab, cells, thr, dist), = seg.segment(ctx, vol, min_volume=30, distance_weights=w)
    assert_matches_oracle(vol, lab, cells, thr, ref=ref, what="vessel frame")
    assert np.all(dist[fg] == 0)
    assert np.all(dist[~fg] > 0)
    rng = np.random.default_rng(12)
    Z, Y, X = vol.shape
    pts = [(int(rng.integers(Z)), int(rng.integers(Y)), int(rng.integers(X))) for _ in range(500)]
    pts += [(0, 0, 0), (Z - 1, Y - 1, X - 1), (Z - 1, 0, X - 1), (0, Y - 1, 0)]
    exp = oracle.distance_at(fg, pts, w)
    got = np.array([dist[p] for p in pts], dtype=np.uint32)
    assert np.array_equal(got, exp)


def test_cell_to_vessel_distance(seg, ctx):
    # cells of a nuclei channel against the distance map of a vessel channel
    # of the same request (Fig. 4), against the oracle's full map
    X, Y, Z = 96, 80, 24
    rng = np.random.default_rng(41)
    nuc = boxes((X, Y, Z), 42, n=12)
    ves = rng.normal(200, 20, size=(Z, Y, X))
    ves[8:12, :, 30:34] += 2500
    ves[:, 50:53, 10:90] += 2500
    ves = np.rint(ves).clip(0, 65535).astype(np.uint16)
    vol = np.stack([nuc, ves])
    w = (16, 16, 25)
    req = seg.seg_submit_volume(ctx, vol, min_volume=5, distance_weights=[None, w])
    seg.seg_flush(ctx)
    try:
        assert seg.seg_wait(ctx, req) == seg.SEG_DONE
        cd = seg.seg_read_cell_distance(ctx, req, 0, 1)
        with pytest.raises(seg.SegError) as e:
            seg.seg_read_cell_distance(ctx, req, 1, 0)  # channel 0 has no map
        assert e.value.code == seg.SEG_EINVAL
    finally:
        seg.seg_release(ctx, req)
    r0 = oracle.segment(nuc, min_volume=5)
    r1 = oracle.segment(ves, min_volume=5, distance_weights=w)
    want = oracle.cell_distance(r0.labels, r1.distance, r0.n_cells)
    assert len(cd) == r0.n_cells > 0 and np.array_equal(cd, want)


def test_cell_to_vessel_distance_full_size(seg, ctx):
    # the time-lapse frame (nuclei and vessel channels): exact for the ten
    # smallest cells (brute force over the oracle's vessel foreground)
    tl = synth.TimeLapse(frames=1)
    vol = np.stack([tl.frame(0, 0), tl.frame(0, 1)])
    w = (16, 16, 25)
    req = seg.seg_submit_volume(ctx, vol, min_volume=30, distance_weights=[None, w])
    seg.seg_flush(ctx)
    try:
        assert seg.seg_wait(ctx, req) == seg.SEG_DONE
        cd = seg.seg_read_cell_distance(ctx, req, 0, 1)
    finally:
        seg.seg_release(ctx, req)
    r0 = oracle.segment(vol[0], min_volume=30)
    r1 = oracle.segment(vol[1], min_volume=30, keep_smoothed=True)
    fg = r1.smoothed > r1.threshold
    assert len(cd) == r0.n_cells
    for k in np.argsort(r0.cells["count"])[:10] + 1:
        pts = [tuple(p) for p in np.argwhere(r0.labels == k)]
        assert cd[k - 1] == oracle.distance_at(fg, pts, w).min(), k
