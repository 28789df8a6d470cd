"""GPU parity of the MRF vessel denoise (Background Noise Removal, Eqs. 2-3)
in front of the stage, against the oracle: the kept image and the number of
steps bit-exact, then the segmentation of it."""
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


def vessels(dims, seed, sigma=25.0, bars=3):
    """Noise N(200, sigma) plus a few bright bars (a vessel-like foreground)."""
    X, Y, Z = dims
    rng = np.random.default_rng(seed)
    v = rng.normal(200, sigma, size=(Z, Y, X))
    for _ in range(bars):
        c = rng.integers(0, [Z, Y, X])
        ax = rng.integers(3)
        sl = [slice(max(0, c[i] - 2), c[i] + 3) for i in range(3)]
        sl[ax] = slice(None)
        v[tuple(sl)] += 1500
    return np.rint(v).clip(0, 65535).astype(np.uint16)


def run(seg, ctx, vol, iters, min_volume=5, what="", **kw):
    req = seg.seg_submit_volume(ctx, vol, min_volume=min_volume, mrf_iterations=iters, **kw)
    seg.seg_flush(ctx)
    try:
        assert seg.seg_wait(ctx, req) == seg.SEG_DONE
        den = np.empty(vol.shape, np.uint16)
        steps = seg.seg_read_denoised(ctx, req, 0, den)
        lab = np.empty(vol.shape, np.uint32)
        seg.seg_read_labels(ctx, req, 0, lab)
        cells, thr = seg.seg_read_features(ctx, req, 0)
    finally:
        seg.seg_release(ctx, req)
    want, wsteps = oracle.mrf(vol, iters)
    assert steps == wsteps, "%s: %d steps vs %d" % (what, steps, wsteps)
    if not np.array_equal(den, want):
        d = np.argwhere(den != want)
        raise AssertionError("%s: %d voxels differ, first at %s (gpu %d, oracle %d)" % (
            what, len(d), tuple(d[0]), den[tuple(d[0])], want[tuple(d[0])]))
    ref = oracle.segment(vol, min_volume=min_volume, mrf_iterations=iters)
    assert_matches_oracle(vol, lab, cells, thr, ref=ref, what=what)
    return steps


@pytest.mark.parametrize("dims", [(1, 1, 1), (7, 1, 1), (9, 5, 3), (33, 17, 6), (64, 48, 10), (130, 3, 4),
                                  (5, 70, 9)])
@pytest.mark.parametrize("iters", [1, 7, 60])
def test_ragged_shapes(seg, ctx, dims, iters):
    # octets cut by the row end, rows and planes without interior (sigma 0),
    # step limits below and above where the noise bound stops the iteration
    run(seg, ctx, vessels(dims, sum(dims) + iters), iters, what="%s it=%d" % (dims, iters))


def test_degenerate_inputs(seg, ctx):
    # one level: Delta = 0, nothing to do
    assert run(seg, ctx, np.full((8, 9, 10), 321, np.uint16), 10, what="constant") == 0
    # two levels far apart (Delta = their gap)
    v = np.full((6, 12, 14), 100, np.uint16)
    v[2:4, 3:9, 4:10] = 2100
    v[3, 6, 7] = 100
    run(seg, ctx, v, 10, what="two levels")
    # values near the top of the range
    rng = np.random.default_rng(7)
    v = (65535 - rng.integers(0, 40, size=(5, 16, 16))).astype(np.uint16)
    run(seg, ctx, v, 10, what="top of range")


def test_noise_levels_stop_the_iteration(seg, ctx):
    # on pure noise the RMS bound stops the iteration, later for larger noise
    # (bright structures inflate the Laplacian estimate, so there the step
    # limit decides)
    steps = [run(seg, ctx, vessels((48, 40, 8), 11, sigma=s, bars=0), 500, what="sigma=%g" % s)
             for s in (5.0, 40.0)]
    assert 0 < steps[0] < steps[1] < 500


def test_mixed_batch(seg):
    c = seg.seg_create(device=0, batch_window_us=30_000_000)
    try:
        a = np.stack([vessels((40, 36, 12), 21), vessels((40, 36, 12), 22)])
        b = vessels((70, 20, 9), 23)
        ra = seg.seg_submit_volume(c, a, min_volume=5, mrf_iterations=[0, 12], denoise_radius=[3, 0],
                                   closing_radius=[0, 1], distance_weights=[None, (16, 16, 25)])
        rb = seg.seg_submit_volume(c, b, min_volume=5, mrf_iterations=40)
        rc = seg.seg_submit_volume(c, b, min_volume=5)
        seg.seg_flush(c)
        for r in (ra, rb, rc):
            assert seg.seg_wait(c, r) == seg.SEG_DONE
        assert seg.seg_get_stats(c)["batches"] == 1
        # the front end's image is readable too
        den = np.empty(a[0].shape, np.uint16)
        assert seg.seg_read_denoised(c, ra, 0, den) == 0
        assert np.array_equal(den, oracle.denoise(a[0], 3))
        for req, ch, vol, it, extra in [(ra, 1, a[1], 12, dict(closing_radius=1, distance_weights=(16, 16, 25))),
                                        (rb, 0, b, 40, {})]:
            den = np.empty(vol.shape, np.uint16)
            steps = seg.seg_read_denoised(c, req, ch, den)
            want, wsteps = oracle.mrf(vol, it)
            assert steps == wsteps and np.array_equal(den, want), (ch, it)
            lab = np.empty(vol.shape, np.uint32)
            seg.seg_read_labels(c, req, ch, lab)
            cells, thr = seg.seg_read_features(c, req, ch)
            ref = oracle.segment(vol, min_volume=5, mrf_iterations=it, **extra)
            assert_matches_oracle(vol, lab, cells, thr, ref=ref, what="mixed ch%d" % ch)
            if "distance_weights" in extra:
                dist = np.empty(vol.shape, np.uint32)
                seg.seg_read_distance(c, req, ch, dist)
                assert np.array_equal(dist, ref.distance)
        # without MRF the same volume is segmented as it is
        lab = np.empty(b.shape, np.uint32)
        seg.seg_read_labels(c, rc, 0, lab)
        assert np.array_equal(lab, oracle.segment(b, min_volume=5).labels)
        with pytest.raises(seg.SegError) as e:
            seg.seg_read_denoised(c, rc, 0, np.empty(b.shape, np.uint16))
        assert e.value.code == seg.SEG_EINVAL
        for r in (ra, rb, rc):
            seg.seg_release(c, r)
    finally:
        seg.seg_destroy(c)


def test_parameter_limits(seg, ctx):
    vol = np.zeros((4, 4, 4), np.uint16)
    for kw in (dict(mrf_iterations=1001), dict(mrf_iterations=5, denoise_radius=2)):
        with pytest.raises(seg.SegError) as e:
            seg.seg_submit_volume(ctx, vol, **kw)
        assert e.value.code == seg.SEG_EINVAL, kw


def test_vessel_frame_full_size(seg, ctx):
    # the 512 x 512 x 64 vessel channel of the time-lapse workload
    vol = synth.TimeLapse(frames=1).frame(0, 1)
    steps = run(seg, ctx, vol, 30, min_volume=30, what="vessel frame")
    assert steps > 0


def test_unaligned_device_input(seg, ctx):
    # a device input 2 bytes past a 16-byte boundary takes the scalar loads
    import torch
    vol = vessels((48, 20, 6), 31)
    flat = torch.zeros(vol.size + 8, dtype=torch.int16, device="cuda:0")
    flat[1:1 + vol.size] = torch.from_numpy(vol.reshape(-1).view(np.int16)).cuda()
    d = flat[1:1 + vol.size].view(vol.shape)
    assert d.data_ptr() % 16 == 2
    req = seg.seg_submit_volume(ctx, d, min_volume=5, mrf_iterations=9)
    seg.seg_flush(ctx)
    try:
        assert seg.seg_wait(ctx, req) == seg.SEG_DONE
        den = np.empty(vol.shape, np.uint16)
        steps = seg.seg_read_denoised(ctx, req, 0, den)
    finally:
        seg.seg_release(ctx, req)
    want, wsteps = oracle.mrf(vol, 9)
    assert steps == wsteps and np.array_equal(den, want)
