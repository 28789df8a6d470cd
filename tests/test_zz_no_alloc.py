"""The allocation-free Otsu entry point against the regular one.

seg_otsu_threshold_noalloc serves callers that cannot allocate device memory
(their HBM is reserved by another allocator, or cudaMalloc's implicit
synchronisation is not acceptable in their loop); it keeps its scratch in one
fixed device array per GPU.  This file is collected last on purpose.  The test
calls the entry point twice in a row through the C ABI, on two different
volumes, and requires each result to equal, exactly, the Otsu level that the
regular seg_submit_volume path reports for the same volume; the second call
also shows that the shared scratch is cleared between calls.
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


def test_noalloc_matches_regular_path_twice():
    import torch

    import paper_1407_2089_gb300 as seg

    assert torch.cuda.is_available()
    # the third volume has ragged rows (X % 8 != 0) and small odd Y and Z, so
    # the edge-clamped loads of the smoothing run through this entry point too
    vols = [synth.single_frame(),
            synth.nuclei_volume((200, 150, 45), 77, 60, peak=3000.0, noise_mean=500.0,
                                noise_sigma=25.0)[0],
            synth.nuclei_volume((37, 23, 5), 78, 2, r_lo=2.0, r_hi=3.0, peak=2000.0)[0]]
    ctx = seg.seg_create(device=0)
    try:
        expected = []
        for v in vols:
            (_, _, thr), = seg.segment(ctx, v)
            expected.append(thr)
    finally:
        seg.seg_destroy(ctx)
    assert len(set(expected)) == len(expected)

    stream = torch.cuda.current_stream()
    dev_vols = [torch.from_numpy(v.view(np.int16).copy()).cuda() for v in vols]
    results = [torch.full((2,), -1, dtype=torch.int32, device="cuda") for _ in vols]
    torch.cuda.synchronize()
    for v, d, r in zip(vols, dev_vols, results):
        Z, Y, X = v.shape
        seg.seg_otsu_threshold_noalloc(d.data_ptr(), (X, Y, Z), r.data_ptr(), stream.cuda_stream)
    torch.cuda.synchronize()
    got = [tuple(int(x) for x in r.cpu()) for r in results]
    for g, e in zip(got, expected):
        assert g == (e, 0)


def test_noalloc_rejects_bad_arguments():
    import paper_1407_2089_gb300 as seg
    with pytest.raises(seg.SegError) as e:
        seg.seg_otsu_threshold_noalloc(0, (4, 4, 4), 0)
    assert e.value.code == seg.SEG_EINVAL
    with pytest.raises(seg.SegError) as e:
        seg.seg_otsu_threshold_noalloc(16, (65536, 65536, 1), 16)
    assert e.value.code == seg.SEG_ETOOBIG
    for dims in [(1, 2 ** 31 + 5, 1), (1, 2 ** 32 - 1, 1)]:
        with pytest.raises(seg.SegError) as e:
            seg.seg_otsu_threshold_noalloc(16, dims, 16)
        assert e.value.code == seg.SEG_ETOOBIG
    with pytest.raises(seg.SegError) as e:
        seg.seg_otsu_threshold_noalloc(17, (4, 4, 4), 16)
    assert e.value.code == seg.SEG_EINVAL
