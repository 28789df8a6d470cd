"""Error handling through the C ABI: argument checks, HBM-budget admission,
host-queue back-pressure, poll timeouts, reads of unfinished, failed or
released requests, and a request that fails on the device (through the
union-find error bit, raised by a test hook, with no device fault) while the
context stays usable."""
import numpy as np
import pytest

import synth
from gpu_util import assert_matches_oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def seg():
    import torch
    assert torch.cuda.is_available()
    import paper_1407_2089_gb300 as seg
    return seg


def code_of(seg, fn, *a, **k):
    with pytest.raises(seg.SegError) as e:
        fn(*a, **k)
    return e.value.code


def test_argument_checks(seg):
    ctx = seg.seg_create(device=0)
    try:
        v = np.zeros((4, 4, 4), dtype=np.uint16)
        assert code_of(seg, seg.seg_submit_volume, ctx, v, dims=(0, 4, 4), channels=1) == seg.SEG_EINVAL
        assert code_of(seg, seg.seg_submit_volume, ctx, v, dims=(4, 4, 4), channels=0) == seg.SEG_EINVAL
        assert code_of(seg, seg.seg_submit_volume, ctx, v, dims=(65537, 1, 1), channels=1) == seg.SEG_ETOOBIG
        assert code_of(seg, seg.seg_submit_volume, ctx, v, dims=(65536, 65536, 1), channels=1) == seg.SEG_ETOOBIG
        for big in [(1, 2 ** 31 + 5, 1), (1, 2 ** 32 - 1, 1), (1, 1, 2 ** 31 + 5)]:
            assert code_of(seg, seg.seg_submit_volume, ctx, v, dims=big, channels=1) == seg.SEG_ETOOBIG, big
        # a device input at an odd address is rejected before it is read
        import ctypes
        import torch
        t = torch.zeros(64, dtype=torch.int16, device="cuda")
        out = ctypes.c_uint64()
        rc = seg._lib.seg_submit_volume(ctx, ctypes.c_void_p(t.data_ptr() + 1), 1, seg.seg_dims(4, 4, 2), 1, None,
                                        ctypes.byref(out))
        assert rc == seg.SEG_EINVAL
        assert code_of(seg, seg.seg_release, ctx, 123456) == seg.SEG_ENOENT
        assert code_of(seg, seg.seg_read_features, ctx, 123456, 0) == seg.SEG_ENOENT
        assert code_of(seg, seg.seg_create, device=10 ** 6) == seg.SEG_EINVAL
        assert code_of(seg, seg.seg_create, device=0, flags=seg.SEG_FORCE_TILE, tile_y=7, tile_z=4) == seg.SEG_EINVAL
    finally:
        seg.seg_destroy(ctx)


def test_budget_too_small_is_too_big(seg):
    ctx = seg.seg_create(device=0, hbm_budget_bytes=1 << 20)
    try:
        v = np.zeros((64, 64, 64), dtype=np.uint16)
        assert code_of(seg, seg.seg_submit_volume, ctx, v) == seg.SEG_ETOOBIG
    finally:
        seg.seg_destroy(ctx)


def test_admission_waits_for_memory(seg):
    # learn one request's footprint: admitted at submit it holds its results
    # and its batch scratch (F); once its batch is done it holds results (p)
    v = synth.single_frame()
    probe = seg.seg_create(device=0, batch_window_us=30_000_000)
    try:
        r = seg.seg_submit_volume(probe, v)
        F = seg.seg_get_stats(probe)["bytes_in_use"]
        seg.seg_flush(probe)
        seg.seg_wait(probe, r)
        p = seg.seg_get_stats(probe)["bytes_in_use"]
        seg.seg_release(probe, r)
        assert seg.seg_get_stats(probe)["bytes_in_use"] == 0
    finally:
        seg.seg_destroy(probe)
    assert 0 < p < F
    # room for one request, not for a second while the first's results are held
    ctx = seg.seg_create(device=0, hbm_budget_bytes=F + p // 2)
    try:
        r1 = seg.seg_submit_volume(ctx, v)
        r2 = seg.seg_submit_volume(ctx, v)
        seg.seg_flush(ctx)
        assert seg.seg_wait(ctx, r1) == seg.SEG_DONE
        assert seg.seg_poll(ctx, r2, 300) == seg.SEG_PENDING
        st = seg.seg_get_stats(ctx)
        assert st["bytes_in_use"] <= st["budget_bytes"]
        seg.seg_release(ctx, r1)
        seg.seg_flush(ctx)
        assert seg.seg_wait(ctx, r2) == seg.SEG_DONE
        lab = np.empty(v.shape, dtype=np.uint32)
        seg.seg_read_labels(ctx, r2, 0, lab)
        cells, thr = seg.seg_read_features(ctx, r2, 0)
        assert_matches_oracle(v, lab, cells, thr, what="admitted after release")
        seg.seg_release(ctx, r2)
        assert seg.seg_get_stats(ctx)["bytes_in_use"] == 0
    finally:
        seg.seg_destroy(ctx)


def test_window_poll_timeout_and_not_ready(seg):
    ctx = seg.seg_create(device=0, batch_window_us=30_000_000, host_queue=2)
    try:
        v = synth.single_frame()
        r = seg.seg_submit_volume(ctx, v)
        assert seg.seg_poll(ctx, r, 50) == seg.SEG_PENDING
        lab = np.empty(v.shape, dtype=np.uint32)
        assert code_of(seg, seg.seg_read_labels, ctx, r, 0, lab) == seg.SEG_ENOTREADY
        r2 = seg.seg_submit_volume(ctx, v)
        # host queue of 2 is full
        assert code_of(seg, seg.seg_submit_volume, ctx, v) == seg.SEG_EAGAIN
        seg.seg_flush(ctx)
        assert seg.seg_wait(ctx, r) == seg.SEG_DONE
        assert seg.seg_wait(ctx, r2) == seg.SEG_DONE
        small = np.empty(10, dtype=np.uint32)
        assert code_of(seg, seg.seg_read_labels, ctx, r, 0, small) == seg.SEG_ESMALL
        assert code_of(seg, seg.seg_read_labels, ctx, r, 1, lab) == seg.SEG_EINVAL
        seg.seg_release(ctx, r)
        assert code_of(seg, seg.seg_read_labels, ctx, r, 0, lab) == seg.SEG_ENOENT
        seg.seg_release(ctx, r2)
    finally:
        seg.seg_destroy(ctx)


def test_features_destination_too_small(seg):
    import ctypes
    ctx = seg.seg_create(device=0)
    try:
        v = synth.single_frame()
        r = seg.seg_submit_volume(ctx, v)
        seg.seg_flush(ctx)
        seg.seg_wait(ctx, r)
        n = ctypes.c_uint64()
        t = ctypes.c_uint16()
        buf = (seg.seg_cell_features * 2)()
        rc = seg._lib.seg_read_features(ctx, r, 0, ctypes.cast(buf, ctypes.c_void_p), 2,
                                        ctypes.byref(n), ctypes.byref(t))
        assert rc == seg.SEG_ESMALL and n.value > 2 and buf[0].count > 0
        seg.seg_release(ctx, r)
    finally:
        seg.seg_destroy(ctx)


def test_device_error_bit_fails_request_context_survives(seg):
    ctx = seg.seg_create(device=0, flags=seg.SEG_TEST_UNION_FAIL)
    try:
        v = synth.single_frame()
        r = seg.seg_submit_volume(ctx, v)
        seg.seg_flush(ctx)
        assert seg.seg_wait(ctx, r) == seg.SEG_FAILED
        lab = np.empty(v.shape, dtype=np.uint32)
        assert code_of(seg, seg.seg_read_labels, ctx, r, 0, lab) == seg.SEG_EFAILED
        seg.seg_release(ctx, r)
        # a volume with no adjacent runs needs no union and still succeeds
        blank = np.full((8, 16, 32), 300, dtype=np.uint16)
        r2 = seg.seg_submit_volume(ctx, blank)
        seg.seg_flush(ctx)
        assert seg.seg_wait(ctx, r2) == seg.SEG_DONE
        seg.seg_release(ctx, r2)
    finally:
        seg.seg_destroy(ctx)
    # and a fresh context on the same device is unaffected
    ok = seg.seg_create(device=0)
    try:
        (lab, cells, thr), = seg.segment(ok, synth.single_frame())
        assert_matches_oracle(synth.single_frame(), lab, cells, thr, what="after failure")
    finally:
        seg.seg_destroy(ok)
