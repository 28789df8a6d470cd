"""Checks for label images too large for the oracle: properties that hold at
any size, evaluated exactly on samples (no GPU code involved)."""
import numpy as np

B5 = np.array([1, 4, 6, 4, 1], dtype=np.int64)


def smoothed_at(vol, zyx):
    """Smoothed values at sample points, from the 125-term definition
    (per-axis edge clamping, one rounding), vectorised over the samples."""
    Z, Y, X = vol.shape
    z, y, x = zyx
    S = np.zeros(len(z), dtype=np.int64)
    for c in range(5):
        zi = np.clip(z + c - 2, 0, Z - 1)
        for b in range(5):
            yi = np.clip(y + b - 2, 0, Y - 1)
            for a in range(5):
                xi = np.clip(x + a - 2, 0, X - 1)
                S += B5[a] * B5[b] * B5[c] * vol[zi, yi, xi].astype(np.int64)
    return (S + 2048) >> 12


def smooth_histogram_slabs(vol, slab=8):
    """65536-bin histogram of the smoothed volume, computed slab by slab with
    scipy's correlate1d (replicate borders; exact integer sums in double)."""
    from scipy import ndimage
    Z = vol.shape[0]
    w = np.array([1, 4, 6, 4, 1], dtype=np.float64)
    h = np.zeros(65536, dtype=np.uint64)
    for z0 in range(0, Z, slab):
        z1 = min(z0 + slab, Z)
        zi = np.clip(np.arange(z0 - 2, z1 + 2), 0, Z - 1)
        part = vol[zi].astype(np.float64)
        part = ndimage.correlate1d(part, w, axis=2, mode="nearest")
        part = ndimage.correlate1d(part, w, axis=1, mode="nearest")
        part = ndimage.correlate1d(part, w, axis=0, mode="nearest")[2:2 + (z1 - z0)]
        s = (part.astype(np.int64) + 2048) >> 12
        h += np.bincount(s.ravel(), minlength=65536).astype(np.uint64)
    return h


def check_threshold_samples(vol, labels, t, rng, n=200000):
    Z, Y, X = vol.shape
    zyx = (rng.integers(0, Z, n), rng.integers(0, Y, n), rng.integers(0, X, n))
    s = smoothed_at(vol, zyx)
    lab = labels[zyx]
    # background voxels are unlabelled; labelled voxels are foreground (an
    # unlabelled foreground voxel belongs to a discarded small component)
    assert np.all(lab[s <= t] == 0)
    assert np.all(s[lab > 0] > t)
    return int((s > t).sum())


def check_adjacency_samples(labels, rng, n=100000):
    """Every labelled voxel's 26-neighbours carry its label or 0."""
    Z, Y, X = labels.shape
    fz, fy, fx = rng.integers(0, Z, n * 4), rng.integers(0, Y, n * 4), rng.integers(0, X, n * 4)
    keep = labels[fz, fy, fx] > 0
    fz, fy, fx = fz[keep][:n], fy[keep][:n], fx[keep][:n]
    own = labels[fz, fy, fx]
    for dz in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                qz, qy, qx = fz + dz, fy + dy, fx + dx
                ok = (qz >= 0) & (qz < Z) & (qy >= 0) & (qy < Y) & (qx >= 0) & (qx < X)
                nb = labels[qz[ok], qy[ok], qx[ok]]
                o = own[ok]
                assert np.all((nb == 0) | (nb == o))
    return len(own)


def check_cells_by_planes(labels, cells, min_volume):
    """Counts, z sums and z ranges per cell by plane-wise bincounts, plus the
    ordering proxy: a cell's first plane never decreases with its label."""
    K = len(cells)
    Z = labels.shape[0]
    cnt = np.zeros(K + 1, dtype=np.int64)
    sz = np.zeros(K + 1, dtype=np.int64)
    zmin = np.full(K + 1, Z, dtype=np.int64)
    zmax = np.full(K + 1, -1, dtype=np.int64)
    for z in range(Z):
        c = np.bincount(labels[z].ravel(), minlength=K + 1).astype(np.int64)
        assert len(c) == K + 1, "label above K"
        cnt += c
        sz += c * z
        present = c > 0
        zmin[present] = np.minimum(zmin[present], z)
        zmax[present] = np.maximum(zmax[present], z)
    assert np.array_equal(cnt[1:], cells["count"].astype(np.int64))
    assert np.all(cnt[1:] >= min_volume)
    assert np.array_equal(sz[1:], cells["sum"][:, 2].astype(np.int64))
    assert np.array_equal(zmin[1:], cells["bbox_min"][:, 2].astype(np.int64))
    assert np.array_equal(zmax[1:], cells["bbox_max"][:, 2].astype(np.int64))
    assert np.all(np.diff(cells["bbox_min"][:, 2].astype(np.int64)) >= 0)


def first_index(labels, cell, lab):
    """Lowest linear index of label lab, searched inside its bounding box."""
    (x0, y0, z0), (x1, y1, z1) = cell["bbox_min"], cell["bbox_max"]
    Z, Y, X = labels.shape
    sub = labels[z0:z1 + 1, y0:y1 + 1, x0:x1 + 1] == lab
    zz, yy, xx = np.nonzero(sub)
    idx = (xx + x0) + X * ((yy + y0) + Y * (zz + z0))
    return int(idx.min()), sub, (x0, y0, z0)


def check_sampled_cells(labels, cells, rng, n=150):
    """For sampled cells: exact x/y sums and boxes from their bounding box, and
    canonical order (lowest linear index increases with the label)."""
    K = len(cells)
    Z, Y, X = labels.shape
    picks = rng.choice(max(K - 1, 1), size=min(n, max(K - 1, 1)), replace=False) + 1 if K > 1 else []
    for l in picks:
        c = cells[l - 1]
        i0, sub, (x0, y0, z0) = first_index(labels, c, l)
        zz, yy, xx = np.nonzero(sub)
        assert int((xx + x0).sum()) == int(c["sum"][0])
        assert int((yy + y0).sum()) == int(c["sum"][1])
        assert int(xx.min() + x0) == int(c["bbox_min"][0]) and int(xx.max() + x0) == int(c["bbox_max"][0])
        if l < K:
            i1, _, _ = first_index(labels, cells[l], l + 1)
            assert i0 < i1
