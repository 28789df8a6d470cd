"""GPU parity of the closing with a binary ball (Segmentation section)
between the threshold and the labelling, against the oracle, bit-exact."""
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


def holey(dims, seed, n=8):
    """Noise plus bright boxes with one-voxel and two-voxel holes and slits."""
    X, Y, Z = dims
    rng = np.random.default_rng(seed)
    v = rng.normal(200, 20, size=(Z, Y, X)).clip(0, 65535).astype(np.uint16)
    for _ in range(n):
        c = rng.integers(0, [Z, Y, X])
        r = rng.integers(2, 7, size=3)
        sl = tuple(slice(max(0, c[i] - r[i]), c[i] + r[i] + 1) for i in range(3))
        v[sl] = 3000
        h = tuple(min(max(c[i] + rng.integers(-1, 2), 0), v.shape[i] - 1) for i in range(3))
        v[h] = 200
    return v


def test_single_frame_closed(seg, ctx):
    vol = synth.single_frame()
    for rho in (1, 2):
        ref = oracle.segment(vol, min_volume=30, closing_radius=rho)
        (lab, cells, thr), = seg.segment(ctx, vol, min_volume=30, closing_radius=rho)
        assert_matches_oracle(vol, lab, cells, thr, ref=ref, what="single frame rho=%d" % rho)


@pytest.mark.parametrize("dims", [(1, 1, 1), (5, 3, 2), (31, 1, 7), (33, 40, 3), (70, 9, 30), (1100, 6, 5),
                                  (64, 64, 16)])
@pytest.mark.parametrize("rho", [1, 2, 3, 8])
def test_ragged_shapes(seg, ctx, dims, rho):
    # rows of 1..35 words (more than a warp), single rows and planes, balls
    # wider than the volume
    vol = holey(dims, sum(dims) + rho)
    ref = oracle.segment(vol, min_volume=1, closing_radius=rho)
    (lab, cells, thr), = seg.segment(ctx, vol, min_volume=1, closing_radius=rho)
    assert_matches_oracle(vol, lab, cells, thr, ref=ref, what="%s rho=%d" % (dims, rho))


def test_mixed_batch_with_denoise(seg):
    c = seg.seg_create(device=0, batch_window_us=30_000_000)
    try:
        a = np.stack([holey((96, 80, 24), 3), holey((96, 80, 24), 4)])
        b = holey((64, 64, 40), 5)
        ra = seg.seg_submit_volume(c, a, denoise_radius=[4, 0], closing_radius=[1, 2], min_volume=5)
        rb = seg.seg_submit_volume(c, b, closing_radius=0, min_volume=5)
        seg.seg_flush(c)
        assert seg.seg_wait(c, ra) == seg.SEG_DONE and seg.seg_wait(c, rb) == seg.SEG_DONE
        assert seg.seg_get_stats(c)["batches"] == 1
        cases = [(ra, 0, a[0], 4, 1), (ra, 1, a[1], 0, 2), (rb, 0, b, 0, 0)]
        for req, ch, vol, dr, cr in cases:
            lab = np.empty(vol.shape, dtype=np.uint32)
            seg.seg_read_labels(c, req, ch, lab)
            cells, thr = seg.seg_read_features(c, req, ch)
            ref = oracle.segment(vol, min_volume=5, denoise_radius=dr, closing_radius=cr)
            assert_matches_oracle(vol, lab, cells, thr, ref=ref, what="mixed dn=%d cl=%d" % (dr, cr))
        seg.seg_release(c, ra)
        seg.seg_release(c, rb)
    finally:
        seg.seg_destroy(c)


def test_radius_limit(seg, ctx):
    vol = np.zeros((4, 4, 4), dtype=np.uint16)
    with pytest.raises(seg.SegError) as e:
        seg.seg_submit_volume(ctx, vol, closing_radius=9)
    assert e.value.code == seg.SEG_EINVAL
