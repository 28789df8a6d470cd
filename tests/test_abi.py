"""Host-side checks of the C-ABI library: it loads without a GPU and exports
every entry point declared in include/seg.h (no compute calls here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "seg.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(seg_\w+)\s*\(", src, flags=re.M)))


@pytest.fixture(scope="module")
def lib():
    import importlib.util
    spec = importlib.util.spec_from_file_location(
        "segbuild", os.path.join(ROOT, "paper_1407_2089_gb300", "build.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    path = mod.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ["seg_create", "seg_destroy", "seg_submit_volume", "seg_poll", "seg_read_labels",
              "seg_read_features", "seg_release", "seg_strerror"]:
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_names_match_header():
    import paper_1407_2089_gb300 as seg
    for n in declared_functions():
        assert hasattr(seg, n), n
    assert set(seg.EXPORTS) == set(declared_functions())


def test_strerror_and_null_arguments(lib):
    lib.seg_strerror.restype = ctypes.c_char_p
    assert lib.seg_strerror(0) == b"ok"
    assert b"invalid" in lib.seg_strerror(-1)
    # null arguments are rejected before any CUDA call
    assert lib.seg_create(None, None) == -1
    assert lib.seg_destroy(None) == -1
    assert lib.seg_flush(None) == -1
    assert lib.seg_read_label_runs(None, ctypes.c_uint64(1), 0, None, ctypes.c_uint64(0), None, 0) == -1


def test_struct_layouts():
    import paper_1407_2089_gb300 as seg
    assert ctypes.sizeof(seg.seg_cell_features) == 64
    assert ctypes.sizeof(seg.seg_dims) == 12
    assert ctypes.sizeof(seg.seg_config) == 56
    assert ctypes.sizeof(seg.seg_channel_params) == 28
    assert ctypes.sizeof(seg.seg_offset) == 12
    assert seg.MONTAGE_EDGE_DTYPE.itemsize == 40
    assert seg.LABEL_RUN_DTYPE.itemsize == 12


def test_binding_constants_match_header():
    # the ctypes mirrors of the header's array sizes and flags
    hdr = open(os.path.join(ROOT, "include", "seg.h")).read()
    defs = dict(re.findall(r"#define\s+(SEG_[A-Z_]+)\s+\(?(-?0x[0-9a-fA-F]+|-?[0-9]+)u?\)?", hdr))
    import paper_1407_2089_gb300 as seg
    for name in ("SEG_MAX_KERNELS", "SEG_FORCE_TILE", "SEG_PLAIN", "SEG_NO_GRAPH", "SEG_PROFILE", "SEG_REG_MAX_RXY",
                 "SEG_REG_MAX_RZ", "SEG_TEST_UNION_FAIL", "SEG_KEEP_SMOOTHED", "SEG_MAX_YZ"):
        assert name in defs, name
        assert getattr(seg, name) == int(defs[name], 0), name


def test_noalloc_argument_checks_without_cuda(lib):
    # the allocation-free entry point validates its arguments before any CUDA
    # call, so these return at once on a machine without a GPU
    import paper_1407_2089_gb300 as seg
    f = lib.seg_otsu_threshold_noalloc
    f.argtypes = [ctypes.c_void_p, seg.seg_dims, ctypes.c_void_p, ctypes.c_void_p]
    f.restype = ctypes.c_int
    aligned, res = 1 << 20, 1 << 21
    assert f(None, seg.seg_dims(4, 4, 4), res, None) == seg.SEG_EINVAL
    assert f(aligned, seg.seg_dims(4, 0, 4), res, None) == seg.SEG_EINVAL
    assert f(aligned + 1, seg.seg_dims(4, 4, 4), res, None) == seg.SEG_EINVAL   # odd uint16 address
    assert f(aligned, seg.seg_dims(4, 4, 4), res + 2, None) == seg.SEG_EINVAL   # unaligned uint32 result
    for dims in [(1, 2 ** 31 + 5, 1), (1, 2 ** 32 - 1, 1), (1, 1, 2 ** 31 + 5), (1, seg.SEG_MAX_YZ + 1, 1),
                 (65537, 1, 1), (65536, 65536, 1)]:
        assert f(aligned, seg.seg_dims(*dims), res, None) == seg.SEG_ETOOBIG, dims
