/*
 * seg_oracle.c -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, single-threaded CPU statement of the per-frame, per-channel
 * 3-D segmentation stage (smooth -> histogram -> Otsu -> threshold ->
 * 26-connected labelling -> minimum-volume filter -> canonical numbering ->
 * per-cell features).  It exists so that the CUDA path can be checked against
 * something written independently of it.  Only the test suite, the smoke
 * check and the CPU-baseline leg of the benchmark may load this file; the
 * product path never calls it and shares no code, header or table with it.
 *
 * Sources (Wait et al., "Visualization and Correction of Automated
 * Segmentation, Tracking and Lineaging from 5-D Stem Cell Image Sequences"):
 *   - Background Noise Removal, Eq. 1: the stem-cell channel is low-pass
 *     (Gaussian) filtered.  Read here as integer separable binomial smoothing
 *     [1 4 6 4 1] per axis (the binomial kernel is the integer form of a
 *     Gaussian with sigma = 1 voxel), uint32 accumulation, one final rounding
 *     (S + 2048) >> 12, replicate-edge borders.
 *   - Segmentation: adaptive Otsu thresholding of every channel (Otsu 1979,
 *     the paper's ref. [11]) giving a binary foreground image; a connected
 *     component filter; components below 19 um^3 discarded (user settable).
 *     Read here as a global Otsu over the frame's 65536-level integer
 *     histogram (FP64 between-class variance, ties to the lowest level,
 *     foreground strictly above the level), 26-connectivity, components
 *     numbered 1..K in increasing order of their lowest linear voxel index
 *     after dropping those with fewer than m voxels (m = 30 voxels is
 *     19 um^3 at the 0.8 x 0.8 x 1.0 um spacing of the Methods section).
 *   - Per-cell features (voxel count, inclusive bounding box, int64 coordinate
 *     sums) stand in for the per-cell voxel sets used by tracking (Eq. 6 uses
 *     the voxel count).
 *
 * Linear index i = x + X*(y + Y*z), x fastest.
 *
 * Build with -O2 -ffp-contract=off and without -ffast-math: the Otsu
 * variance must be evaluated in IEEE binary64 exactly in the order written.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_OK 0
#define ORACLE_EINVAL (-1)
#define ORACLE_ENOMEM (-2)
#define ORACLE_ESMALL (-3)

/* Per-cell record, 64 bytes, defined here independently of the CUDA path. */
typedef struct {
    uint64_t count;
    int64_t sum[3];      /* sum of x, y, z over the cell's voxels */
    uint32_t bbox_min[3];/* inclusive */
    uint32_t bbox_max[3];/* inclusive */
    uint32_t pad[2];
} oracle_cell;

static const uint32_t BINOM5[5] = {1u, 4u, 6u, 4u, 1u};

static int64_t clamp_i64(int64_t k, int64_t n) {
    if (k < 0) return 0;
    if (k >= n) return n - 1;
    return k;
}

/* Background Noise Removal (Eq. 1, Gaussian low-pass) as binomial smoothing:
 *   S(x,y,z) = sum_{a,b,c in -2..2} B[a] B[b] B[c] v(cl(x+a), cl(y+b), cl(z+c))
 *   s = (S + 2048) >> 12
 * computed as three 1-D passes (x, then y, then z) in uint32 with the single
 * rounding at the end, which equals the 125-term sum exactly. */
int oracle_smooth(const uint16_t *v, uint32_t X, uint32_t Y, uint32_t Z, uint16_t *s) {
    if (!v || !s || X == 0 || Y == 0 || Z == 0) return ORACLE_EINVAL;
    uint64_t n = (uint64_t)X * Y * Z;
    uint32_t *a = (uint32_t *)malloc(n * sizeof(uint32_t));
    uint32_t *b = (uint32_t *)malloc(n * sizeof(uint32_t));
    if (!a || !b) { free(a); free(b); return ORACLE_ENOMEM; }
    /* pass along x */
    for (uint64_t z = 0; z < Z; ++z)
        for (uint64_t y = 0; y < Y; ++y)
            for (uint64_t x = 0; x < X; ++x) {
                uint32_t acc = 0;
                for (int k = 0; k < 5; ++k) {
                    int64_t xx = clamp_i64((int64_t)x + k - 2, X);
                    acc += BINOM5[k] * (uint32_t)v[xx + X * (y + Y * z)];
                }
                a[x + X * (y + Y * z)] = acc;
            }
    /* pass along y */
    for (uint64_t z = 0; z < Z; ++z)
        for (uint64_t y = 0; y < Y; ++y)
            for (uint64_t x = 0; x < X; ++x) {
                uint32_t acc = 0;
                for (int k = 0; k < 5; ++k) {
                    int64_t yy = clamp_i64((int64_t)y + k - 2, Y);
                    acc += BINOM5[k] * a[x + X * (yy + Y * z)];
                }
                b[x + X * (y + Y * z)] = acc;
            }
    /* pass along z, then the one rounding */
    for (uint64_t z = 0; z < Z; ++z)
        for (uint64_t y = 0; y < Y; ++y)
            for (uint64_t x = 0; x < X; ++x) {
                uint32_t acc = 0;
                for (int k = 0; k < 5; ++k) {
                    int64_t zz = clamp_i64((int64_t)z + k - 2, Z);
                    acc += BINOM5[k] * b[x + X * (y + Y * zz)];
                }
                s[x + X * (y + Y * z)] = (uint16_t)((acc + 2048u) >> 12);
            }
    free(a);
    free(b);
    return ORACLE_OK;
}

/* Histogram of the smoothed frame: h[u] = number of voxels with value u. */
int oracle_histogram(const uint16_t *s, uint64_t n, uint64_t *h) {
    if (!s || !h) return ORACLE_EINVAL;
    memset(h, 0, 65536 * sizeof(uint64_t));
    for (uint64_t i = 0; i < n; ++i) h[s[i]] += 1;
    return ORACLE_OK;
}

/* Otsu's threshold (Segmentation section, ref. [11]).
 * For every level t = 0..65534 with C0 = {u <= t}, C1 = {u > t}:
 *   n0 = sum_{u<=t} h[u], s0 = sum_{u<=t} u h[u], n1 = N - n0, s1 = S - s0,
 *   skip t when n0 == 0 or n1 == 0, else
 *   var(t) = ((n0 * n1) * (s1/n1 - s0/n0)) * (s1/n1 - s0/n0)   in binary64,
 * which is N^2 times Otsu's between-class variance (the same argmax).
 * t* = the lowest t attaining the maximum.  A frame with one distinct value has
 * no admissible t; then t* is that value, so nothing lies strictly above it. */
uint16_t oracle_otsu(const uint64_t *h) {
    uint64_t N = 0, S = 0;
    for (uint32_t u = 0; u < 65536u; ++u) {
        N += h[u];
        S += (uint64_t)u * h[u];
    }
    uint64_t n0 = 0, s0 = 0;
    double best = -1.0;
    int found = 0;
    uint32_t best_t = 0;
    for (uint32_t t = 0; t < 65535u; ++t) {
        n0 += h[t];
        s0 += (uint64_t)t * h[t];
        uint64_t n1 = N - n0;
        uint64_t s1 = S - s0;
        if (n0 == 0 || n1 == 0) continue;
        double m0 = (double)s0 / (double)n0;
        double m1 = (double)s1 / (double)n1;
        double d = m1 - m0;
        double var = (((double)n0 * (double)n1) * d) * d;
        if (!found || var > best) {
            best = var;
            best_t = t;
            found = 1;
        }
    }
    if (!found) {
        for (uint32_t u = 0; u < 65536u; ++u)
            if (h[u]) return (uint16_t)u;
        return 0;
    }
    return (uint16_t)best_t;
}

/* 26-connected component labelling of a binary volume (Segmentation section,
 * "connected component image filter").  Voxels are scanned in increasing
 * linear index; each unlabelled foreground voxel starts a breadth-first flood
 * over its 26 neighbours (in bounds, no wrap).  Provisional ids are 1, 2, ...
 * in discovery order, i.e. in increasing order of each component's lowest
 * linear index.  Returns the number of components, or a negative error. */
int64_t oracle_label26(const uint8_t *mask, uint32_t X, uint32_t Y, uint32_t Z, uint32_t *lab) {
    if (!mask || !lab || X == 0 || Y == 0 || Z == 0) return ORACLE_EINVAL;
    uint64_t n = (uint64_t)X * Y * Z;
    uint64_t *queue = (uint64_t *)malloc(n * sizeof(uint64_t));
    if (!queue) return ORACLE_ENOMEM;
    memset(lab, 0, n * sizeof(uint32_t));
    uint32_t next = 0;
    for (uint64_t i = 0; i < n; ++i) {
        if (!mask[i] || lab[i]) continue;
        next += 1;
        uint64_t head = 0, tail = 0;
        lab[i] = next;
        queue[tail++] = i;
        while (head < tail) {
            uint64_t p = queue[head++];
            int64_t px = (int64_t)(p % X);
            int64_t py = (int64_t)((p / X) % Y);
            int64_t pz = (int64_t)(p / ((uint64_t)X * Y));
            for (int dz = -1; dz <= 1; ++dz)
                for (int dy = -1; dy <= 1; ++dy)
                    for (int dx = -1; dx <= 1; ++dx) {
                        if (!dx && !dy && !dz) continue;
                        int64_t qx = px + dx, qy = py + dy, qz = pz + dz;
                        if (qx < 0 || qy < 0 || qz < 0) continue;
                        if (qx >= X || qy >= Y || qz >= Z) continue;
                        uint64_t q = (uint64_t)qx + X * ((uint64_t)qy + (uint64_t)Y * qz);
                        if (mask[q] && !lab[q]) {
                            lab[q] = next;
                            queue[tail++] = q;
                        }
                    }
        }
    }
    free(queue);
    return (int64_t)next;
}

/* Minimum-volume filter, canonical numbering and per-cell features
 * (Segmentation section: components under the user-set volume are discarded).
 * A provisional component survives iff its voxel count >= min_volume; the
 * survivors are numbered 1..K keeping the provisional (lowest-index) order.
 * labels_out may alias prov.  Features are gathered by visiting every voxel. */
int oracle_filter_features(const uint32_t *prov, uint64_t ncomp, uint32_t X, uint32_t Y, uint32_t Z,
                           uint32_t min_volume, uint32_t *labels_out, oracle_cell *cells,
                           uint64_t cap, uint64_t *k_out) {
    if (!prov || !labels_out || !k_out || X == 0 || Y == 0 || Z == 0) return ORACLE_EINVAL;
    uint64_t n = (uint64_t)X * Y * Z;
    uint64_t *count = (uint64_t *)calloc(ncomp + 1, sizeof(uint64_t));
    uint32_t *remap = (uint32_t *)calloc(ncomp + 1, sizeof(uint32_t));
    if (!count || !remap) { free(count); free(remap); return ORACLE_ENOMEM; }
    for (uint64_t i = 0; i < n; ++i) count[prov[i]] += 1;
    uint64_t K = 0;
    for (uint64_t c = 1; c <= ncomp; ++c)
        if (count[c] >= min_volume) remap[c] = (uint32_t)(++K);
    *k_out = K;
    int rc = ORACLE_OK;
    if (cells && cap < K) rc = ORACLE_ESMALL;
    if (cells && rc == ORACLE_OK) {
        for (uint64_t k = 0; k < K; ++k) {
            memset(&cells[k], 0, sizeof(oracle_cell));
            for (int a = 0; a < 3; ++a) cells[k].bbox_min[a] = 0xFFFFFFFFu;
        }
    }
    for (uint64_t z = 0; z < Z; ++z)
        for (uint64_t y = 0; y < Y; ++y)
            for (uint64_t x = 0; x < X; ++x) {
                uint64_t i = x + X * (y + Y * z);
                uint32_t l = remap[prov[i]];
                labels_out[i] = l;
                if (!l || !cells || rc != ORACLE_OK) continue;
                oracle_cell *c = &cells[l - 1];
                uint64_t p[3] = {x, y, z};
                c->count += 1;
                for (int a = 0; a < 3; ++a) {
                    c->sum[a] += (int64_t)p[a];
                    if (p[a] < c->bbox_min[a]) c->bbox_min[a] = (uint32_t)p[a];
                    if (p[a] > c->bbox_max[a]) c->bbox_max[a] = (uint32_t)p[a];
                }
            }
    free(count);
    free(remap);
    return rc;
}

/* ------------------------------------------------------------------------
 * Denoise front end for the stem-cell channel (Background Noise Removal,
 * Eq. 1: observed = background + shot noise + signal).  The background B is
 * a low-pass of the observed image; the paper names a Gaussian without a
 * width.  Read here as three box filters of width w = 2r + 1 along x, then
 * three along y, then three along z (three boxes approximate a Gaussian of
 * variance 3 (w^2 - 1) / 12 per axis), each pass rounding to nearest,
 * (sum + r) / w, with replicate edges.  The background is subtracted with a
 * floor at 0 and the shot noise removed by the 3x3x3 median (the 14th of the
 * 27 values, replicate edges).
 * ------------------------------------------------------------------------ */

/* One box pass of radius r along `axis` (0 = x, 1 = y, 2 = z). */
int oracle_box_pass(const uint16_t *in, uint32_t X, uint32_t Y, uint32_t Z, int axis, uint32_t r,
                    uint16_t *out) {
    if (!in || !out || X == 0 || Y == 0 || Z == 0 || axis < 0 || axis > 2) return ORACLE_EINVAL;
    const uint64_t w = 2 * (uint64_t)r + 1;
    const int64_t len = axis == 0 ? X : (axis == 1 ? Y : Z);
    for (uint64_t z = 0; z < Z; ++z)
        for (uint64_t y = 0; y < Y; ++y)
            for (uint64_t x = 0; x < X; ++x) {
                const int64_t pos = axis == 0 ? (int64_t)x : (axis == 1 ? (int64_t)y : (int64_t)z);
                uint64_t sum = 0;
                for (int64_t k = -(int64_t)r; k <= (int64_t)r; ++k) {
                    const int64_t q = clamp_i64(pos + k, len);
                    const uint64_t xx = axis == 0 ? (uint64_t)q : x;
                    const uint64_t yy = axis == 1 ? (uint64_t)q : y;
                    const uint64_t zz = axis == 2 ? (uint64_t)q : z;
                    sum += in[xx + X * (yy + Y * zz)];
                }
                out[x + X * (y + Y * z)] = (uint16_t)((sum + r) / w);
            }
    return ORACLE_OK;
}

/* Background estimate B: three box passes along x, three along y, three
 * along z. */
int oracle_background(const uint16_t *v, uint32_t X, uint32_t Y, uint32_t Z, uint32_t r, uint16_t *b) {
    if (!v || !b || X == 0 || Y == 0 || Z == 0) return ORACLE_EINVAL;
    uint64_t n = (uint64_t)X * Y * Z;
    uint16_t *t = (uint16_t *)malloc(n * sizeof(uint16_t));
    if (!t) return ORACLE_ENOMEM;
    memcpy(b, v, n * sizeof(uint16_t));
    int rc = ORACLE_OK;
    for (int axis = 0; axis < 3 && rc == ORACLE_OK; ++axis)
        for (int p = 0; p < 3 && rc == ORACLE_OK; ++p) {
            rc = oracle_box_pass(b, X, Y, Z, axis, r, t);
            memcpy(b, t, n * sizeof(uint16_t));
        }
    free(t);
    return rc;
}

/* 3x3x3 median with replicate edges: the 14th smallest of the 27 values. */
int oracle_median27(const uint16_t *d, uint32_t X, uint32_t Y, uint32_t Z, uint16_t *out) {
    if (!d || !out || X == 0 || Y == 0 || Z == 0) return ORACLE_EINVAL;
    for (int64_t z = 0; z < Z; ++z)
        for (int64_t y = 0; y < Y; ++y)
            for (int64_t x = 0; x < X; ++x) {
                uint16_t w[27];
                int m = 0;
                for (int c = -1; c <= 1; ++c)
                    for (int b = -1; b <= 1; ++b)
                        for (int a = -1; a <= 1; ++a)
                            w[m++] = d[clamp_i64(x + a, X) + X * (clamp_i64(y + b, Y) + Y * clamp_i64(z + c, Z))];
                /* insertion sort */
                for (int i = 1; i < 27; ++i) {
                    uint16_t key = w[i];
                    int j = i - 1;
                    while (j >= 0 && w[j] > key) {
                        w[j + 1] = w[j];
                        --j;
                    }
                    w[j + 1] = key;
                }
                out[x + X * (y + Y * z)] = w[13];
            }
    return ORACLE_OK;
}

/* The denoised image: median27(max(v - B, 0)). */
int oracle_denoise(const uint16_t *v, uint32_t X, uint32_t Y, uint32_t Z, uint32_t r, uint16_t *out) {
    if (!v || !out || X == 0 || Y == 0 || Z == 0) return ORACLE_EINVAL;
    uint64_t n = (uint64_t)X * Y * Z;
    uint16_t *b = (uint16_t *)malloc(n * sizeof(uint16_t));
    if (!b) return ORACLE_ENOMEM;
    int rc = oracle_background(v, X, Y, Z, r, b);
    if (rc == ORACLE_OK) {
        for (uint64_t i = 0; i < n; ++i) b[i] = v[i] > b[i] ? (uint16_t)(v[i] - b[i]) : 0;
        rc = oracle_median27(b, X, Y, Z, out);
    }
    free(b);
    return rc;
}

/* ------------------------------------------------------------------------
 * Morphological closing of the foreground (Segmentation: a closing with a
 * binary ball removes holes before the connected components).  The ball of
 * radius rho holds the offsets with dx^2 + dy^2 + dz^2 <= rho^2 (voxel
 * units).  The closing is taken on the volume padded with rho voxels of
 * background on every side -- dilation, then erosion, then the original box
 * -- so it contains the foreground it started from and has no border
 * artefacts.
 * ------------------------------------------------------------------------ */
int oracle_close(const uint8_t *m, uint32_t X, uint32_t Y, uint32_t Z, uint32_t rho, uint8_t *out) {
    if (!m || !out || X == 0 || Y == 0 || Z == 0) return ORACLE_EINVAL;
    const int64_t r = rho;
    const int64_t PX = X + 2 * r, PY = Y + 2 * r, PZ = Z + 2 * r;
    const uint64_t pn = (uint64_t)PX * PY * PZ;
    uint8_t *a = (uint8_t *)calloc(pn, 1), *d = (uint8_t *)calloc(pn, 1);
    if (!a || !d) { free(a); free(d); return ORACLE_ENOMEM; }
    for (int64_t z = 0; z < Z; ++z)
        for (int64_t y = 0; y < Y; ++y)
            for (int64_t x = 0; x < X; ++x)
                a[(x + r) + PX * ((y + r) + PY * (z + r))] = m[x + X * (y + Y * z)] ? 1 : 0;
    /* dilation: any ball neighbour inside the padded box set */
    for (int64_t z = 0; z < PZ; ++z)
        for (int64_t y = 0; y < PY; ++y)
            for (int64_t x = 0; x < PX; ++x) {
                uint8_t v = 0;
                for (int64_t c = -r; c <= r && !v; ++c)
                    for (int64_t b = -r; b <= r && !v; ++b)
                        for (int64_t e = -r; e <= r && !v; ++e) {
                            if (e * e + b * b + c * c > r * r) continue;
                            const int64_t xx = x + e, yy = y + b, zz = z + c;
                            if (xx < 0 || yy < 0 || zz < 0 || xx >= PX || yy >= PY || zz >= PZ) continue;
                            v = a[xx + PX * (yy + PY * zz)];
                        }
                d[x + PX * (y + PY * z)] = v;
            }
    /* erosion, read back inside the original box: every ball neighbour set
     * (all of them lie inside the padded box) */
    for (int64_t z = 0; z < Z; ++z)
        for (int64_t y = 0; y < Y; ++y)
            for (int64_t x = 0; x < X; ++x) {
                uint8_t v = 1;
                for (int64_t c = -r; c <= r && v; ++c)
                    for (int64_t b = -r; b <= r && v; ++b)
                        for (int64_t e = -r; e <= r && v; ++e) {
                            if (e * e + b * b + c * c > r * r) continue;
                            v = d[(x + r + e) + PX * ((y + r + b) + PY * (z + r + c))];
                        }
                out[x + X * (y + Y * z)] = v;
            }
    free(a);
    free(d);
    return ORACLE_OK;
}

/* ------------------------------------------------------------------------
 * Distance map of the foreground (Segmentation: the vasculature channel's
 * distance map gives every voxel its distance to the nearest foreground
 * voxel).  Squared Euclidean distance with integer axis weights (wx, wy,
 * wz): d2(p) = min over foreground q of wx dx^2 + wy dy^2 + wz dz^2; with
 * weights 16, 16, 25 this is 25 times the squared distance in um at the
 * 0.8 x 0.8 x 1.0 um spacing.  No foreground at all: 0xFFFFFFFF everywhere.
 * Plain definition: the minimum over every foreground voxel.
 * ------------------------------------------------------------------------ */
int oracle_distance(const uint8_t *m, uint32_t X, uint32_t Y, uint32_t Z, uint32_t wx, uint32_t wy,
                    uint32_t wz, uint32_t *d2) {
    if (!m || !d2 || X == 0 || Y == 0 || Z == 0) return ORACLE_EINVAL;
    const uint64_t n = (uint64_t)X * Y * Z;
    uint64_t nf = 0;
    for (uint64_t i = 0; i < n; ++i) nf += m[i] ? 1 : 0;
    uint32_t *fx = (uint32_t *)malloc((nf ? nf : 1) * 3 * sizeof(uint32_t));
    if (!fx) return ORACLE_ENOMEM;
    uint64_t k = 0;
    for (uint64_t z = 0; z < Z; ++z)
        for (uint64_t y = 0; y < Y; ++y)
            for (uint64_t x = 0; x < X; ++x)
                if (m[x + X * (y + Y * z)]) {
                    fx[3 * k] = (uint32_t)x;
                    fx[3 * k + 1] = (uint32_t)y;
                    fx[3 * k + 2] = (uint32_t)z;
                    ++k;
                }
    for (uint64_t z = 0; z < Z; ++z)
        for (uint64_t y = 0; y < Y; ++y)
            for (uint64_t x = 0; x < X; ++x) {
                uint64_t best = UINT64_MAX;
                for (uint64_t j = 0; j < nf; ++j) {
                    const int64_t dx = (int64_t)x - fx[3 * j], dy = (int64_t)y - fx[3 * j + 1];
                    const int64_t dz = (int64_t)z - fx[3 * j + 2];
                    const uint64_t v = (uint64_t)(wx * dx * dx + wy * dy * dy + wz * dz * dz);
                    if (v < best) best = v;
                }
                d2[x + X * (y + Y * z)] = nf ? (uint32_t)best : 0xFFFFFFFFu;
            }
    free(fx);
    return ORACLE_OK;
}

/* ---- MRF vessel denoise (Background Noise Removal, Eqs. 2-3) -------------
 *
 * The vessel channel is denoised by an iteration that moves every voxel by a
 * fixed step Delta towards its six face neighbours (Eq. 3) and stops before
 * the image strays from the original by more than the noise level estimated
 * from the original (Eq. 2).  Readings of the passage:
 *   - Delta is the smallest difference between two distinct voxel values of
 *     the original image (0 when it holds fewer than two: nothing to do).
 *   - The noise level sigma is estimated "by convolving with a Laplacian":
 *     read as Immerkaer's estimate (Fast noise variance estimation, 1996) on
 *     every z-plane, the mask [1 -2 1; -2 4 -2; 1 -2 1] over the plane's
 *     interior, sigma = sqrt(pi / 2) * S / (6 M) with S the sum of the
 *     absolute responses and M the number of interior voxels (0 when M = 0).
 *   - The norm of Eq. 2 is the root-mean-square voxel difference, so the
 *     iterate I^{n+1} is kept while sum (I^{n+1} - I^0)^2 <= N sigma^2
 *     (N voxels), evaluated in binary64 in the order written below.
 *   - Each pair of terms of Eq. 3 is read as the votes of the two
 *     neighbours along an axis towards themselves, sgn(I_prev - I) +
 *     sgn(I_next - I): with the second term of a pair as printed,
 *     sgn(I - I_next), an isolated bright voxel would get +1 - 1 = 0 from
 *     every axis and never move, which is not a denoiser.  A neighbour
 *     outside the volume votes 0.  The step is clamped to [0, 65535].
 *   - The iteration also stops when a step changes no voxel (a fixed point)
 *     and after max_iter accepted steps. */

/* Delta of Eq. 3. */
uint32_t oracle_mrf_delta(const uint16_t *v, uint64_t n) {
    uint8_t *seen = (uint8_t *)calloc(65536, 1);
    if (!seen) return 0;
    for (uint64_t i = 0; i < n; ++i) seen[v[i]] = 1;
    int32_t prev = -1;
    uint32_t best = 0;
    for (int32_t level = 0; level < 65536; ++level) {
        if (!seen[level]) continue;
        if (prev >= 0) {
            const uint32_t gap = (uint32_t)(level - prev);
            if (best == 0 || gap < best) best = gap;
        }
        prev = level;
    }
    free(seen);
    return best;
}

/* S of the noise estimate: sum over every z-plane's interior of the absolute
 * response of the mask [1 -2 1; -2 4 -2; 1 -2 1]; *m_out gets M. */
uint64_t oracle_mrf_laplacian(const uint16_t *v, uint32_t X, uint32_t Y, uint32_t Z, uint64_t *m_out) {
    static const int32_t mask[3][3] = {{1, -2, 1}, {-2, 4, -2}, {1, -2, 1}};
    uint64_t s = 0, m = 0;
    for (uint64_t z = 0; z < Z; ++z)
        for (uint64_t y = 1; y + 1 < Y; ++y)
            for (uint64_t x = 1; x + 1 < X; ++x) {
                int64_t r = 0;
                for (int dy = -1; dy <= 1; ++dy)
                    for (int dx = -1; dx <= 1; ++dx)
                        r += mask[dy + 1][dx + 1] * (int64_t)v[(x + dx) + X * ((y + dy) + Y * z)];
                s += (uint64_t)(r < 0 ? -r : r);
                ++m;
            }
    if (m_out) *m_out = m;
    return s;
}

/* The bound N sigma^2 of Eq. 2 from S and M, for N voxels. */
double oracle_mrf_limit(uint64_t s, uint64_t m, uint64_t n) {
    if (m == 0) return 0.0;
    const double half_pi = 3.14159265358979323846 / 2.0;
    const double sigma = (sqrt(half_pi) * (double)s) / (6.0 * (double)m);
    return ((double)n * sigma) * sigma;
}

/* One step of Eq. 3 (reading above): next = clamp(cur + delta * sgn(votes)). */
int oracle_mrf_step(const uint16_t *cur, uint32_t X, uint32_t Y, uint32_t Z, uint32_t delta, uint16_t *next) {
    if (!cur || !next || X == 0 || Y == 0 || Z == 0) return ORACLE_EINVAL;
    for (int64_t z = 0; z < Z; ++z)
        for (int64_t y = 0; y < Y; ++y)
            for (int64_t x = 0; x < X; ++x) {
                const uint64_t i = (uint64_t)x + (uint64_t)X * ((uint64_t)y + (uint64_t)Y * (uint64_t)z);
                const int32_t c = cur[i];
                int32_t votes = 0;
                const int64_t nb[6][3] = {{x - 1, y, z}, {x + 1, y, z}, {x, y - 1, z},
                                          {x, y + 1, z}, {x, y, z - 1}, {x, y, z + 1}};
                for (int k = 0; k < 6; ++k) {
                    const int64_t a = nb[k][0], b = nb[k][1], d = nb[k][2];
                    if (a < 0 || a >= X || b < 0 || b >= Y || d < 0 || d >= Z) continue;
                    const int32_t o = cur[(uint64_t)a + (uint64_t)X * ((uint64_t)b + (uint64_t)Y * (uint64_t)d)];
                    votes += (o > c) - (o < c);
                }
                int32_t v = c + (int32_t)delta * ((votes > 0) - (votes < 0));
                if (v < 0) v = 0;
                if (v > 65535) v = 65535;
                next[i] = (uint16_t)v;
            }
    return ORACLE_OK;
}

/* The iteration of Eqs. 2-3 on one volume: out gets the last kept image,
 * *iters the number of steps kept (each at most max_iter). */
int oracle_mrf(const uint16_t *v, uint32_t X, uint32_t Y, uint32_t Z, uint32_t max_iter, uint16_t *out,
               uint32_t *iters) {
    if (!v || !out || X == 0 || Y == 0 || Z == 0) return ORACLE_EINVAL;
    const uint64_t n = (uint64_t)X * Y * Z;
    memcpy(out, v, n * sizeof(uint16_t));
    uint32_t kept = 0;
    const uint32_t delta = oracle_mrf_delta(v, n);
    if (delta > 0 && max_iter > 0) {
        uint64_t m = 0;
        const uint64_t s = oracle_mrf_laplacian(v, X, Y, Z, &m);
        const double limit = oracle_mrf_limit(s, m, n);
        uint16_t *next = (uint16_t *)malloc(n * sizeof(uint16_t));
        if (!next) return ORACLE_ENOMEM;
        while (kept < max_iter) {
            oracle_mrf_step(out, X, Y, Z, delta, next);
            int changed = 0;
            uint64_t e = 0;
            for (uint64_t i = 0; i < n; ++i) {
                changed |= next[i] != out[i];
                const int64_t d = (int64_t)next[i] - (int64_t)v[i];
                e += (uint64_t)(d * d);
            }
            if (!changed) break;           /* fixed point */
            if ((double)e > limit) break;  /* Eq. 2: keep the previous image */
            memcpy(out, next, n * sizeof(uint16_t));
            ++kept;
        }
        free(next);
    }
    if (iters) *iters = kept;
    return ORACLE_OK;
}

/* Cell-to-vessel distance (Segmentation section and Fig. 4: each stem cell's
 * distance to its nearest vessel): for cell k = 1..K of a label image, the
 * smallest value of a distance map over the cell's voxels (out[k - 1];
 * 0xFFFFFFFF for a label with no voxel). */
int oracle_cell_distance(const uint32_t *labels, const uint32_t *map, uint64_t n, uint64_t k, uint32_t *out) {
    if (!labels || !map || !out) return ORACLE_EINVAL;
    for (uint64_t c = 0; c < k; ++c) out[c] = 0xFFFFFFFFu;
    for (uint64_t i = 0; i < n; ++i) {
        const uint32_t l = labels[i];
        if (l == 0) continue;
        if (l > k) return ORACLE_EINVAL;
        if (map[i] < out[l - 1]) out[l - 1] = map[i];
    }
    return ORACLE_OK;
}

/* ---- Label runs (Segmentation section: each cell's voxels) ---------------
 *
 * The voxels of each cell, the set the Segmentation section passes on to the
 * convex hull step, written as runs: the maximal stretches of equal non-zero
 * label along x within one row (row = y + Y z), in order of row and then x.
 * One record per run: label, row, first x, last x (inclusive).  On return *n
 * is the number of runs; with cap < *n nothing past cap is written and the
 * call fails with ORACLE_ESMALL. */
typedef struct {
    uint32_t label;
    uint32_t row;
    uint16_t x_begin;
    uint16_t x_end;
} oracle_run;

int oracle_label_runs(const uint32_t *labels, uint32_t X, uint64_t rows, oracle_run *out, uint64_t cap,
                      uint64_t *n) {
    if (!labels || !n || X == 0 || X > 65536u) return ORACLE_EINVAL;
    uint64_t k = 0;
    for (uint64_t row = 0; row < rows; ++row) {
        const uint32_t *L = labels + row * X;
        uint32_t x = 0;
        while (x < X) {
            if (L[x] == 0) {
                ++x;
                continue;
            }
            uint32_t e = x;
            while (e + 1 < X && L[e + 1] == L[x]) ++e;
            if (k < cap && out) {
                out[k].label = L[x];
                out[k].row = (uint32_t)row;
                out[k].x_begin = (uint16_t)x;
                out[k].x_end = (uint16_t)e;
            }
            ++k;
            x = e + 1;
        }
    }
    *n = k;
    return k > cap ? ORACLE_ESMALL : ORACLE_OK;
}

/* ---- Montage registration (Registration section, Eq. 4) -------------------
 *
 * Overlapping tiles of a montage are placed at their stage positions; each
 * overlapping pair is scored at every shift of the second tile inside a
 * window around its stage position by the normalized covariance of Eq. 4
 * over the voxels the two tiles then share; each pair keeps its best shift;
 * a maximum spanning tree of the pair graph (dropping the lowest-scoring
 * edges) anchors one tile and gives every other tile the sum of the shifts
 * along its tree path.  Readings:
 *   - normcov(A, B) = sum (A - muA)(B - muB) / (sigmaA sigmaB) over the
 *     overlap is read as the Pearson correlation, sigma the root of the
 *     summed squared deviations, so the score does not grow with the size of
 *     the overlap (which changes with the shift).  From exact integer sums:
 *     num = N Sab - Sa Sb, va = N Saa - Sa^2, vb = N Sbb - Sb^2 (128-bit),
 *     rho = (double)num / sqrt((double)va * (double)vb); undefined when the
 *     overlap is empty or va or vb is 0.
 *   - A pair is an edge when its stage boxes overlap.  Its shift s (of the
 *     second tile, b > a) runs over [-r, r] per axis, z outermost, then y,
 *     then x; the first shift with the largest defined score is kept.  An
 *     edge with no defined score stays out of the tree.
 *   - The maximum spanning tree is Kruskal's: edges by score, highest first,
 *     ties by (a, b); the root keeps its stage position; delta(b) =
 *     delta(a) + s over a tree edge (a, b), delta(a) = delta(b) - s; tiles
 *     outside the root's tree keep delta 0.
 */
typedef struct {
    uint32_t a, b;
    int32_t shift[3];
    uint32_t pad0;
    double score;
    uint32_t in_tree;
    uint32_t pad1;
} oracle_edge;

/* Sums over the voxels shared by tile A (origin 0) and tile B placed with its
 * origin at d in A's coordinates: out = {N, Sa, Sb, Saa, Sbb, Sab}. */
void oracle_reg_sums(const uint16_t *A, const uint16_t *B, uint32_t X, uint32_t Y, uint32_t Z, const int32_t *d,
                     uint64_t *out) {
    int64_t lo[3], hi[3];
    const int64_t D[3] = {X, Y, Z};
    for (int k = 0; k < 3; ++k) {
        lo[k] = d[k] > 0 ? d[k] : 0;
        hi[k] = d[k] + D[k] < D[k] ? d[k] + D[k] : D[k];
    }
    uint64_t n = 0, sa = 0, sb = 0, saa = 0, sbb = 0, sab = 0;
    for (int64_t z = lo[2]; z < hi[2]; ++z)
        for (int64_t y = lo[1]; y < hi[1]; ++y)
            for (int64_t x = lo[0]; x < hi[0]; ++x) {
                const uint64_t a = A[x + X * (y + Y * z)];
                const uint64_t b = B[(x - d[0]) + X * ((y - d[1]) + Y * (z - d[2]))];
                ++n;
                sa += a;
                sb += b;
                saa += a * a;
                sbb += b * b;
                sab += a * b;
            }
    out[0] = n; out[1] = sa; out[2] = sb; out[3] = saa; out[4] = sbb; out[5] = sab;
}

/* Eq. 4 as read above from the six sums; *defined = 0 when undefined. */
double oracle_normcov(const uint64_t *s, int *defined) {
    const __int128 n = (__int128)s[0];
    const __int128 num = n * (__int128)s[5] - (__int128)s[1] * (__int128)s[2];
    const __int128 va = n * (__int128)s[3] - (__int128)s[1] * (__int128)s[1];
    const __int128 vb = n * (__int128)s[4] - (__int128)s[2] * (__int128)s[2];
    if (s[0] == 0 || va == 0 || vb == 0) {
        *defined = 0;
        return 0.0;
    }
    *defined = 1;
    return (double)num / sqrt((double)va * (double)vb);
}

static uint32_t uf_find(uint32_t *p, uint32_t i) {
    while (p[i] != i) i = p[i];
    return i;
}

int oracle_register(const uint16_t *const *tiles, uint32_t nt, uint32_t X, uint32_t Y, uint32_t Z,
                    const int32_t *stage, const int32_t *radius, uint32_t root, int32_t *delta,
                    oracle_edge *edges, uint32_t cap, uint32_t *n_edges) {
    if (!tiles || !stage || !radius || !delta || nt == 0 || root >= nt || X == 0 || Y == 0 || Z == 0)
        return ORACLE_EINVAL;
    const int64_t D[3] = {X, Y, Z};
    uint32_t ne = 0;
    for (uint32_t a = 0; a < nt; ++a)
        for (uint32_t b = a + 1; b < nt; ++b) {
            int overlap = 1;
            for (int k = 0; k < 3; ++k) {
                const int64_t o = (int64_t)stage[3 * b + k] - stage[3 * a + k];
                if (o >= D[k] || -o >= D[k]) overlap = 0;
            }
            if (!overlap) continue;
            if (ne < cap && edges) {
                oracle_edge *e = &edges[ne];
                memset(e, 0, sizeof(*e));
                e->a = a;
                e->b = b;
                e->score = -2.0;  /* no defined score */
                for (int32_t sz = -radius[2]; sz <= radius[2]; ++sz)
                    for (int32_t sy = -radius[1]; sy <= radius[1]; ++sy)
                        for (int32_t sx = -radius[0]; sx <= radius[0]; ++sx) {
                            const int32_t d[3] = {stage[3 * b] - stage[3 * a] + sx,
                                                  stage[3 * b + 1] - stage[3 * a + 1] + sy,
                                                  stage[3 * b + 2] - stage[3 * a + 2] + sz};
                            uint64_t sums[6];
                            oracle_reg_sums(tiles[a], tiles[b], X, Y, Z, d, sums);
                            int ok;
                            const double r = oracle_normcov(sums, &ok);
                            if (ok && r > e->score) {
                                e->score = r;
                                e->shift[0] = sx;
                                e->shift[1] = sy;
                                e->shift[2] = sz;
                            }
                        }
            }
            ++ne;
        }
    if (n_edges) *n_edges = ne;
    if (ne > cap || !edges) return ne > cap ? ORACLE_ESMALL : ORACLE_OK;
    /* Kruskal: edges by score, highest first, ties by (a, b) (selection order) */
    uint32_t *order = (uint32_t *)malloc((ne ? ne : 1) * sizeof(uint32_t));
    uint32_t *par = (uint32_t *)malloc(nt * sizeof(uint32_t));
    if (!order || !par) {
        free(order);
        free(par);
        return ORACLE_ENOMEM;
    }
    for (uint32_t i = 0; i < ne; ++i) order[i] = i;
    for (uint32_t i = 0; i < ne; ++i)  /* insertion sort: stable, so ties keep (a, b) order */
        for (uint32_t j = i; j > 0 && edges[order[j]].score > edges[order[j - 1]].score; --j) {
            const uint32_t t = order[j];
            order[j] = order[j - 1];
            order[j - 1] = t;
        }
    for (uint32_t i = 0; i < nt; ++i) par[i] = i;
    for (uint32_t i = 0; i < ne; ++i) {
        oracle_edge *e = &edges[order[i]];
        if (e->score < -1.5) continue;  /* undefined */
        const uint32_t ra = uf_find(par, e->a), rb = uf_find(par, e->b);
        if (ra == rb) continue;
        par[ra] = rb;
        e->in_tree = 1;
    }
    /* deltas along the tree from the root (repeated sweeps until nothing changes) */
    uint8_t *known = (uint8_t *)calloc(nt, 1);
    for (uint32_t i = 0; i < 3 * nt; ++i) delta[i] = 0;
    known[root] = 1;
    for (int grew = 1; grew;) {
        grew = 0;
        for (uint32_t i = 0; i < ne; ++i) {
            const oracle_edge *e = &edges[i];
            if (!e->in_tree || known[e->a] == known[e->b]) continue;
            if (known[e->a])
                for (int k = 0; k < 3; ++k) delta[3 * e->b + k] = delta[3 * e->a + k] + e->shift[k];
            else
                for (int k = 0; k < 3; ++k) delta[3 * e->a + k] = delta[3 * e->b + k] - e->shift[k];
            known[e->a] = known[e->b] = 1;
            grew = 1;
        }
    }
    free(known);
    free(order);
    free(par);
    return ORACLE_OK;
}

/* The whole stage for one frame and channel: smooth, histogram, Otsu,
 * threshold (foreground iff s > t*), label, filter, features.
 * hist (65536 entries) and smoothed (n entries) are optional outputs. */
int oracle_segment(const uint16_t *v, uint32_t X, uint32_t Y, uint32_t Z, uint32_t min_volume,
                   uint32_t closing_radius, uint32_t *labels, oracle_cell *cells, uint64_t cap,
                   uint64_t *k_out, uint16_t *t_out, uint64_t *hist, uint16_t *smoothed) {
    if (!v || !labels || !k_out || !t_out || X == 0 || Y == 0 || Z == 0) return ORACLE_EINVAL;
    uint64_t n = (uint64_t)X * Y * Z;
    uint16_t *s = smoothed ? smoothed : (uint16_t *)malloc(n * sizeof(uint16_t));
    uint64_t *h = hist ? hist : (uint64_t *)malloc(65536 * sizeof(uint64_t));
    uint8_t *m = (uint8_t *)malloc(n);
    int rc = ORACLE_OK;
    if (!s || !h || !m) { rc = ORACLE_ENOMEM; goto done; }
    rc = oracle_smooth(v, X, Y, Z, s);
    if (rc) goto done;
    rc = oracle_histogram(s, n, h);
    if (rc) goto done;
    uint16_t t = oracle_otsu(h);
    *t_out = t;
    for (uint64_t i = 0; i < n; ++i) m[i] = (uint8_t)(s[i] > t);
    if (closing_radius) {
        uint8_t *c = (uint8_t *)malloc(n);
        if (!c) { rc = ORACLE_ENOMEM; goto done; }
        rc = oracle_close(m, X, Y, Z, closing_radius, c);
        memcpy(m, c, n);
        free(c);
        if (rc) goto done;
    }
    int64_t nc = oracle_label26(m, X, Y, Z, labels);
    if (nc < 0) { rc = (int)nc; goto done; }
    rc = oracle_filter_features(labels, (uint64_t)nc, X, Y, Z, min_volume, labels, cells, cap, k_out);
done:
    if (!smoothed) free(s);
    if (!hist) free(h);
    free(m);
    return rc;
}
