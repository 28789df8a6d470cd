"""GPU parity of the denoise front end (Background Noise Removal, Eq. 1):
box-cascade background, floored subtraction and 3x3x3 median in front of the
segmentation stage, against the oracle, bit-exact."""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import assert_cells_equal, assert_matches_oracle

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


def run(seg, ctx, vol, r, m=30):
    (lab, cells, thr), = seg.segment(ctx, vol, min_volume=m, denoise_radius=r)
    return lab, cells, thr


def test_single_frame_denoised(seg, ctx):
    vol = synth.single_frame()
    for r in (4, 8):
        ref = oracle.segment(vol, min_volume=30, denoise_radius=r)
        lab, cells, thr = run(seg, ctx, vol, r)
        assert_matches_oracle(vol, lab, cells, thr, ref=ref, what="single frame r=%d" % r)


@pytest.mark.parametrize("dims", [(1, 1, 1), (5, 3, 2), (31, 1, 7), (33, 40, 3), (70, 9, 300), (300, 17, 5),
                                  (257, 258, 3),
                                  # X % 8 == 0 (16-byte copies along y and z), lane groups cut short
                                  (8, 130, 7), (72, 9, 300), (200, 17, 5), (136, 258, 3)])
@pytest.mark.parametrize("r", [1, 3, 16])
def test_ragged_shapes(seg, ctx, dims, r):
    # lines shorter than the window, chunks of 256 with ragged tails, X not
    # a multiple of 8, single rows and planes
    X, Y, Z = dims
    rng = np.random.default_rng(sum(dims) + r)
    vol = rng.normal(300, 40, size=(Z, Y, X)).clip(0, 65535).astype(np.uint16)
    for _ in range(4):
        c = rng.integers(0, [Z, Y, X])
        sl = tuple(slice(max(0, c[i] - 3), c[i] + 4) for i in range(3))
        vol[sl] = rng.integers(1500, 4000)
    ref = oracle.segment(vol, min_volume=1, denoise_radius=r)
    lab, cells, thr = run(seg, ctx, vol, r, 1)
    assert_matches_oracle(vol, lab, cells, thr, ref=ref, what="%s r=%d" % (dims, r))


def test_mixed_batch(seg):
    # channels with and without the front end, and another request, in one launch
    c = seg.seg_create(device=0, batch_window_us=30_000_000)
    try:
        a = np.stack([synth.nuclei_volume((96, 80, 24), seed=3, n_nuclei=12)[0],
                      synth.nuclei_volume((96, 80, 24), seed=4, n_nuclei=12)[0]])
        b = synth.nuclei_volume((64, 64, 40), seed=5, n_nuclei=8)[0]
        ra = seg.seg_submit_volume(c, a, denoise_radius=[6, 0])
        rb = seg.seg_submit_volume(c, b, denoise_radius=2)
        seg.seg_flush(c)
        assert seg.seg_wait(c, ra) == seg.SEG_DONE and seg.seg_wait(c, rb) == seg.SEG_DONE
        assert seg.seg_get_stats(c)["batches"] == 1
        cases = [(ra, 0, a[0], 6), (ra, 1, a[1], 0), (rb, 0, b, 2)]
        for req, ch, vol, r in cases:
            lab = np.empty(vol.shape, dtype=np.uint32)
            seg.seg_read_labels(c, req, ch, lab)
            cells, thr = seg.seg_read_features(c, req, ch)
            ref = oracle.segment(vol, min_volume=30, denoise_radius=r)
            assert_matches_oracle(vol, lab, cells, thr, ref=ref, what="mixed r=%d" % r)
        seg.seg_release(c, ra)
        seg.seg_release(c, rb)
    finally:
        seg.seg_destroy(c)


def test_time_lapse_frame_stem_cell_channel(seg, ctx):
    # the paper applies this front end to the stem-cell channel
    vol = synth.TimeLapse(frames=1).frame(0, 0)
    ref = oracle.segment(vol, min_volume=30, denoise_radius=8)
    lab, cells, thr = run(seg, ctx, vol, 8)
    assert_matches_oracle(vol, lab, cells, thr, ref=ref, what="time-lapse ch0 r=8")


def test_radius_limit(seg, ctx):
    vol = np.zeros((4, 4, 4), dtype=np.uint16)
    with pytest.raises(seg.SegError) as e:
        seg.seg_submit_volume(ctx, vol, denoise_radius=17)
    assert e.value.code == seg.SEG_EINVAL
