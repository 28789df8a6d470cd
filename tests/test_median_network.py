"""The selection network used by the CUDA 3x3x3 median (host-side check of
the generated comparator list; no GPU)."""
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


def _run(kept, out_var, vals):
    v = [vals[:, k].copy() for k in range(vals.shape[1])] + [None] * 5
    for a, b, na, nb in kept:
        lo, hi = np.minimum(v[a], v[b]), np.maximum(v[a], v[b])
        if na:
            v[a] = lo
        if nb:
            v[b] = hi
    return v[out_var]


def test_network_selects_the_median():
    kept, out_var = _gen().network()
    rng = np.random.default_rng(27)
    for hi in (2, 3, 30, 65536):  # many ties .. all distinct
        vals = rng.integers(0, hi, size=(20000, 27))
        assert np.array_equal(_run(kept, out_var, vals), np.sort(vals, axis=1)[:, 13]), hi


def test_network_on_zero_one_inputs():
    # 0-1 principle, restricted: every input with k ones at random positions
    kept, out_var = _gen().network()
    rng = np.random.default_rng(28)
    for k in range(28):
        vals = np.zeros((2000, 27), dtype=np.int64)
        for row in vals:
            row[rng.choice(27, size=k, replace=False)] = 1
        assert np.array_equal(_run(kept, out_var, vals), (np.arange(2000) * 0 + (1 if k >= 14 else 0))), k


def test_committed_header_is_current(tmp_path):
    out = tmp_path / "net.h"
    _gen().emit(str(out))
    committed = open(os.path.join(ROOT, "paper_1407_2089_gb300", "csrc", "median27_net.h")).read()
    assert out.read_text() == committed
