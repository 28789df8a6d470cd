/*
 * synth.c -- seeded synthetic confocal volumes (uint16, [Z][Y][X], x fastest).
 *
 * Input generator shared by the tests, the benchmark and the CPU baseline.  It
 * holds none of the segmentation arithmetic: it only draws noise and renders
 * shapes.  Parallel loops split work by z-plane and every voxel's value is a
 * function of (seed, voxel index, shape list) only, so the output does not
 * depend on the thread count.
 *
 * Noise: splitmix64 counter stream (Steele, Lea, Flood 2014) -> Box-Muller.
 * Nuclei: solid ellipsoids blurred by a Gaussian of width sigma, rendered with
 *   the 1-D edge profile 0.5*erfc(d / (sigma*sqrt 2)) of the distance d to the
 *   surface (normalised radius - 1) * mean radius, summed over nuclei.
 * Vessels: tubes of radius r around polyline centrelines, profile
 *   0.5*erfc((dist - r) / (sigma*sqrt 2)), max-combined over segments.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

static inline uint64_t splitmix64(uint64_t x) {
    x += 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    return x ^ (x >> 31);
}

static inline double unit_open(uint64_t r) { /* (0, 1) */
    return ((double)(r >> 11) + 0.5) * (1.0 / 9007199254740992.0);
}

static inline uint16_t sat_u16(double v) {
    if (v <= 0.0) return 0;
    if (v >= 65535.0) return 65535;
    return (uint16_t)floor(v + 0.5);
}

/* out[i] = clip(round(mean + sigma * N_i)), N_i standard normal, i in [0, n). */
void synth_background(uint16_t *out, uint64_t n, uint64_t seed, double mean, double sigma) {
    const uint64_t key = splitmix64(seed ^ 0xA5A5A5A5DEADBEEFull);
    const int64_t npairs = (int64_t)((n + 1) / 2);
    const double two_pi = 6.283185307179586476925286766559;
#pragma omp parallel for schedule(static)
    for (int64_t p = 0; p < npairs; ++p) {
        uint64_t r1 = splitmix64(key + 0x9E3779B97F4A7C15ull * (uint64_t)(2 * p));
        uint64_t r2 = splitmix64(key + 0x9E3779B97F4A7C15ull * (uint64_t)(2 * p + 1));
        double rad = sqrt(-2.0 * log(unit_open(r1)));
        double ang = two_pi * unit_open(r2);
        uint64_t i = (uint64_t)(2 * p);
        out[i] = sat_u16(mean + sigma * rad * cos(ang));
        if (i + 1 < n) out[i + 1] = sat_u16(mean + sigma * rad * sin(ang));
    }
}

/* Adds blurred solid ellipsoids.  params: n rows of (cx, cy, cz, rx, ry, rz,
 * peak).  Values are accumulated in double per voxel in nucleus order and
 * saturated once, so the result is independent of threading. */
void synth_add_ellipsoids(uint16_t *vol, uint32_t X, uint32_t Y, uint32_t Z, int64_t n,
                          const double *params, double sigma) {
    const double inv = 1.0 / (sigma * 1.4142135623730950488);
    const double reach = 4.0 * sigma;
#pragma omp parallel
    {
        double *row = (double *)malloc(sizeof(double) * X);
        int64_t *sel = (int64_t *)malloc(sizeof(int64_t) * (n > 0 ? n : 1));
#pragma omp for schedule(dynamic, 1)
        for (int64_t z = 0; z < (int64_t)Z; ++z) {
            int64_t ns = 0;
            for (int64_t k = 0; k < n; ++k) {
                const double *p = params + 7 * k;
                double rmax = fmax(p[3], fmax(p[4], p[5])) + reach;
                if (fabs((double)z - p[2]) <= rmax) sel[ns++] = k;
            }
            if (!ns) continue;
            for (int64_t y = 0; y < (int64_t)Y; ++y) {
                int any = 0;
                int64_t xlo = X, xhi = -1;
                for (int64_t s = 0; s < ns; ++s) {
                    const double *p = params + 7 * sel[s];
                    double rmax = fmax(p[3], fmax(p[4], p[5])) + reach;
                    if (fabs((double)y - p[1]) > rmax) continue;
                    int64_t a = (int64_t)floor(p[0] - rmax), b = (int64_t)ceil(p[0] + rmax);
                    if (a < 0) a = 0;
                    if (b > (int64_t)X - 1) b = (int64_t)X - 1;
                    if (a > b) continue;
                    if (!any) { any = 1; }
                    if (a < xlo) xlo = a;
                    if (b > xhi) xhi = b;
                }
                if (!any) continue;
                for (int64_t x = xlo; x <= xhi; ++x) row[x] = 0.0;
                for (int64_t s = 0; s < ns; ++s) {
                    const double *p = params + 7 * sel[s];
                    double rmax = fmax(p[3], fmax(p[4], p[5])) + reach;
                    if (fabs((double)y - p[1]) > rmax) continue;
                    double rmean = (p[3] + p[4] + p[5]) / 3.0;
                    int64_t a = (int64_t)floor(p[0] - rmax), b = (int64_t)ceil(p[0] + rmax);
                    if (a < 0) a = 0;
                    if (b > (int64_t)X - 1) b = (int64_t)X - 1;
                    double dy = ((double)y - p[1]) / p[4], dz = ((double)z - p[2]) / p[5];
                    for (int64_t x = a; x <= b; ++x) {
                        double dx = ((double)x - p[0]) / p[3];
                        double rho = sqrt(dx * dx + dy * dy + dz * dz);
                        double d = (rho - 1.0) * rmean;
                        if (d > reach) continue;
                        row[x] += p[6] * 0.5 * erfc(d * inv);
                    }
                }
                uint16_t *dst = vol + (uint64_t)X * ((uint64_t)y + (uint64_t)Y * (uint64_t)z);
                for (int64_t x = xlo; x <= xhi; ++x)
                    if (row[x] > 0.0) dst[x] = sat_u16((double)dst[x] + row[x]);
            }
        }
        free(row);
        free(sel);
    }
}

static double seg_dist(double px, double py, double pz, const double *s) {
    double ax = s[0], ay = s[1], az = s[2];
    double bx = s[3] - ax, by = s[4] - ay, bz = s[5] - az;
    double qx = px - ax, qy = py - ay, qz = pz - az;
    double bb = bx * bx + by * by + bz * bz;
    double t = bb > 0.0 ? (qx * bx + qy * by + qz * bz) / bb : 0.0;
    if (t < 0.0) t = 0.0;
    if (t > 1.0) t = 1.0;
    double dx = qx - t * bx, dy = qy - t * by, dz = qz - t * bz;
    return sqrt(dx * dx + dy * dy + dz * dz);
}

/* Writes field[i] = round(max over segments of I * 0.5 erfc((dist - r)/(sigma sqrt2))).
 * segs: n rows of (x0, y0, z0, x1, y1, z1, radius, intensity). */
void synth_tube_field(uint16_t *field, uint32_t X, uint32_t Y, uint32_t Z, int64_t n,
                      const double *segs, double sigma) {
    const double inv = 1.0 / (sigma * 1.4142135623730950488);
    const double reach = 4.0 * sigma;
#pragma omp parallel
    {
        float *plane = (float *)malloc(sizeof(float) * (uint64_t)X * Y);
#pragma omp for schedule(dynamic, 1)
        for (int64_t z = 0; z < (int64_t)Z; ++z) {
            uint16_t *dst = field + (uint64_t)X * Y * (uint64_t)z;
            memset(plane, 0, sizeof(float) * (uint64_t)X * Y);
            for (int64_t k = 0; k < n; ++k) {
                const double *s = segs + 8 * k;
                double ext = s[6] + reach;
                double zlo = fmin(s[2], s[5]) - ext, zhi = fmax(s[2], s[5]) + ext;
                if ((double)z < zlo || (double)z > zhi) continue;
                int64_t ya = (int64_t)floor(fmin(s[1], s[4]) - ext), yb = (int64_t)ceil(fmax(s[1], s[4]) + ext);
                int64_t xa = (int64_t)floor(fmin(s[0], s[3]) - ext), xb = (int64_t)ceil(fmax(s[0], s[3]) + ext);
                if (ya < 0) ya = 0;
                if (xa < 0) xa = 0;
                if (yb > (int64_t)Y - 1) yb = (int64_t)Y - 1;
                if (xb > (int64_t)X - 1) xb = (int64_t)X - 1;
                for (int64_t y = ya; y <= yb; ++y)
                    for (int64_t x = xa; x <= xb; ++x) {
                        double d = seg_dist((double)x, (double)y, (double)z, s) - s[6];
                        if (d > reach) continue;
                        float v = (float)(s[7] * 0.5 * erfc(d * inv));
                        float *c = &plane[(uint64_t)y * X + (uint64_t)x];
                        if (v > *c) *c = v;
                    }
            }
            for (uint64_t i = 0; i < (uint64_t)X * Y; ++i) dst[i] = sat_u16((double)plane[i]);
        }
        free(plane);
    }
}

/* vol[i] = min(65535, vol[i] + field[i]) */
void synth_add_field(uint16_t *vol, const uint16_t *field, uint64_t n) {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < (int64_t)n; ++i) {
        uint32_t s = (uint32_t)vol[i] + field[i];
        vol[i] = (uint16_t)(s > 65535u ? 65535u : s);
    }
}
