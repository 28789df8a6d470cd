"""GPU parity of the montage registration (Registration section, Eq. 4)
against the oracle: every pair's best shift and score (bit-identical binary64),
the maximum spanning tree and the tile corrections."""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def seg():
    import torch
    assert torch.cuda.is_available()
    import paper_1407_2089_gb300 as seg
    return seg


def montage(rng, grid, dims, overlap, jitter, radius, noise=0):
    """Tiles cut from one textured global volume at true positions (stage
    positions moved by at most `jitter` voxels in x and y and up to the z
    radius in z), with optional independent noise per tile."""
    X, Y, Z = dims
    nx, ny = grid
    true, stage = [], []
    for j in range(ny):
        for i in range(nx):
            s = np.array([i * (X - overlap[0]) + radius[0], j * (Y - overlap[1]) + radius[1], 0])
            # neighbours' relative shifts stay inside the window
            jx, jy = min(jitter, radius[0] // 2), min(jitter, radius[1] // 2)
            t = s + np.array([rng.integers(-jx, jx + 1), rng.integers(-jy, jy + 1), rng.integers(0, radius[2] + 1)])
            true.append(t)
            stage.append(s)
    true, stage = np.array(true), np.array(stage)
    ext = true.max(axis=0) + np.array(dims) + 1
    # smooth-ish texture: noise plus blobs, so the correlation peaks sharply
    G = rng.integers(0, 3000, size=(ext[2], ext[1], ext[0])).astype(np.int64)
    tiles = []
    for t in true:
        a = G[t[2]:t[2] + Z, t[1]:t[1] + Y, t[0]:t[0] + X].copy()
        if noise:
            a = a + rng.integers(-noise, noise + 1, size=a.shape)
        tiles.append(np.clip(a, 0, 65535).astype(np.uint16))
    return tiles, true, stage


def check(seg, tiles, stage, radius, root=0, device_tiles=None, what=""):
    delta, edges = seg.seg_register_montage(device_tiles if device_tiles is not None else tiles, stage, radius,
                                            root=root)
    wd, we = oracle.register(tiles, stage, radius, root=root)
    assert len(edges) == len(we), what
    for k in ("a", "b", "shift", "in_tree"):
        assert np.array_equal(edges[k], we[k]), (what, k, edges[k], we[k])
    assert np.array_equal(edges["score"], we["score"]), (what, edges["score"] - we["score"])
    assert np.array_equal(delta, wd), (what, delta, wd)
    return delta, edges


@pytest.mark.parametrize("grid,dims,overlap,radius", [
    ((2, 2), (48, 40, 12), (10, 9), (3, 3, 2)),
    ((3, 2), (64, 33, 9), (12, 7), (4, 2, 1)),
    ((1, 3), (40, 70, 20), (6, 14), (0, 5, 3)),
    ((3, 3), (37, 35, 6), (9, 9), (2, 2, 0)),
])
def test_small_montages(seg, grid, dims, overlap, radius):
    rng = np.random.default_rng(sum(dims) + sum(radius))
    tiles, true, stage = montage(rng, grid, dims, overlap, 1, radius, noise=400)
    delta, edges = check(seg, tiles, stage, radius, what=str(grid))
    # the planted corrections come back (relative to the root)
    assert np.array_equal(delta, (true - stage) - (true - stage)[0])


def test_device_tiles_and_other_root(seg):
    import torch
    rng = np.random.default_rng(5)
    radius = (3, 3, 1)
    tiles, true, stage = montage(rng, (3, 2), (50, 44, 10), (11, 10), 1, radius, noise=200)
    dev = [torch.from_numpy(t.view(np.int16)).cuda() for t in tiles]
    check(seg, tiles, stage, radius, root=4, device_tiles=dev, what="device")


def test_degenerate_montages(seg):
    rng = np.random.default_rng(6)
    t = rng.integers(0, 1000, size=(8, 20, 20)).astype(np.uint16)
    # one tile: no pairs
    d, e = seg.seg_register_montage([t], [(0, 0, 0)], (2, 2, 1))
    assert len(e) == 0 and np.array_equal(d, np.zeros((1, 3), np.int32))
    # tiles far apart: no pairs, nobody moves
    d, e = seg.seg_register_montage([t, t], [(0, 0, 0), (100, 0, 0)], (2, 2, 1))
    assert len(e) == 0 and not d.any()
    # constant tiles: no score is defined, so the pair stays out of the tree
    c = np.full((8, 20, 20), 7, np.uint16)
    check(seg, [c, c], [(0, 0, 0), (15, 0, 0)], (2, 2, 1), what="constant")
    # search window of one shift
    tiles, true, stage = montage(rng, (2, 1), (30, 20, 6), (8, 0), 0, (0, 0, 0))
    check(seg, tiles, stage, (0, 0, 0), what="radius 0")


def test_argument_errors(seg):
    t = np.zeros((4, 8, 8), np.uint16)
    for args in [([t], [(0, 0, 0)], (13, 0, 0)), ([t], [(0, 0, 0)], (0, 0, 7)), ([t], [(0, 0, 0)], (-1, 0, 0))]:
        with pytest.raises(seg.SegError) as e:
            seg.seg_register_montage(*args)
        assert e.value.code == seg.SEG_EINVAL
    with pytest.raises(seg.SegError) as e:
        seg.seg_register_montage([t, t], [(0, 0, 0), (4, 0, 0)], (1, 1, 1), root=2)
    assert e.value.code == seg.SEG_EINVAL


def test_montage_512(seg):
    # 3 x 3 tiles of 512 x 512 x 32 with 10 % overlap and a (4, 4, 1) window
    rng = np.random.default_rng(7)
    radius = (4, 4, 1)
    tiles, true, stage = montage(rng, (3, 3), (512, 512, 32), (51, 51), 2, radius, noise=300)
    delta, edges = check(seg, tiles, stage, radius, what="512")
    assert np.array_equal(delta, (true - stage) - (true - stage)[0])
