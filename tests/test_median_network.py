"""The selection networks used by the CUDA 3x3x3 median (host-side check of
the generated comparator lists; no GPU)."""
import importlib.util
import os

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
GEN = os.path.join(ROOT, "paper_1407_2089_gb300", "csrc", "gen_median27.py")


def _gen():
    spec = importlib.util.spec_from_file_location("gen_median27", GEN)
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _apply(ops, w):
    for op in ops:
        a, b = op[0], op[1]
        na, nb = (op[2], op[3]) if len(op) == 4 else (True, True)
        lo, hi = np.minimum(w[a], w[b]), np.maximum(w[a], w[b])
        if na:
            w[a] = lo
        if nb:
            w[b] = hi
    return w


def test_sort9_sorts():
    ops, out = _gen().sort9()
    rng = np.random.default_rng(9)
    for hi in (2, 4, 65536):
        vals = rng.integers(0, hi, size=(20000, 9))
        w = {i: vals[:, i].copy() for i in range(9)}
        w = _apply(ops, w)
        got = np.stack([w[out[k]] for k in range(9)], axis=1)
        assert np.array_equal(got, np.sort(vals, axis=1)), hi


def test_median3x9_on_sorted_lists():
    ops, out = _gen().median3x9()
    rng = np.random.default_rng(27)
    for hi in (2, 3, 30, 65536):
        vals = rng.integers(0, hi, size=(20000, 27))
        lists = [np.sort(vals[:, 9 * k: 9 * k + 9], axis=1) for k in range(3)]
        w = {}
        for k in range(3):
            for i in range(9):
                w[16 * k + i] = lists[k][:, i].copy()
        w = _apply(ops, w)
        assert np.array_equal(w[out], np.sort(vals, axis=1)[:, 13]), hi


def test_median3x9_zero_one():
    # 0-1 inputs: each sorted list is a number of zeros then ones
    ops, out = _gen().median3x9()
    for z0 in range(10):
        for z1 in range(10):
            for z2 in range(10):
                w = {}
                for k, nz in enumerate((z0, z1, z2)):
                    for i in range(9):
                        w[16 * k + i] = np.array([0 if i < nz else 1])
                w = _apply(ops, w)
                assert w[out][0] == (0 if z0 + z1 + z2 >= 14 else 1)


def test_committed_header_is_current(tmp_path):
    out = tmp_path / "net.h"
    _gen().emit(str(out))
    committed = open(os.path.join(ROOT, "paper_1407_2089_gb300", "csrc", "median27_net.h")).read()
    assert out.read_text() == committed
