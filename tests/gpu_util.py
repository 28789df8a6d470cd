"""Helpers shared by the GPU tests: run the CUDA path through the C ABI and
compare it with the oracle element by element."""
import numpy as np

import oracle


def assert_cells_equal(gpu_cells, ref_cells, what=""):
    assert len(gpu_cells) == len(ref_cells), "%s: K %d vs %d" % (what, len(gpu_cells), len(ref_cells))
    for f in ("count", "sum", "bbox_min", "bbox_max"):
        a = np.asarray(gpu_cells[f])
        b = np.asarray(ref_cells[f])
        if not np.array_equal(a, b):
            bad = np.nonzero((a != b).reshape(len(a), -1).any(axis=1))[0]
            raise AssertionError("%s: field %s differs at cells %s" % (what, f, bad[:10]))


def assert_matches_oracle(vol, labels, cells, thr, min_volume=30, ref=None, what=""):
    if ref is None:
        ref = oracle.segment(vol, min_volume=min_volume)
    assert thr == ref.threshold, "%s: threshold %d vs %d" % (what, thr, ref.threshold)
    if not np.array_equal(labels, ref.labels):
        d = np.argwhere(labels != ref.labels)
        raise AssertionError("%s: %d label mismatches, first at %s (gpu %d, oracle %d)" % (
            what, len(d), tuple(d[0]), labels[tuple(d[0])], ref.labels[tuple(d[0])]))
    assert_cells_equal(cells, ref.cells, what)
    return ref
