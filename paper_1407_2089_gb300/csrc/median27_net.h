// Generated by gen_median27.py: sort9 (28 comparators) and the median of
// three sorted lists of 9 (55 comparators, pruned Batcher networks), on
// one voxel per 32-bit word and on two voxels per word (16-bit halves).
#pragma once

// Sorts v[0..8] in place (s[k] receives the k-th smallest).
__device__ __forceinline__ void sort9(const uint32_t *v, uint32_t *s) {
    uint32_t w[16];
    w[0] = v[0];
    w[1] = v[1];
    w[2] = v[2];
    w[3] = v[3];
    w[4] = v[4];
    w[5] = v[5];
    w[6] = v[6];
    w[7] = v[7];
    w[8] = v[8];
    { const uint32_t t = min(w[0], w[1]); w[1] = max(w[0], w[1]); w[0] = t; }
    { const uint32_t t = min(w[2], w[3]); w[3] = max(w[2], w[3]); w[2] = t; }
    { const uint32_t t = min(w[4], w[5]); w[5] = max(w[4], w[5]); w[4] = t; }
    { const uint32_t t = min(w[6], w[7]); w[7] = max(w[6], w[7]); w[6] = t; }
    { const uint32_t t = min(w[0], w[2]); w[2] = max(w[0], w[2]); w[0] = t; }
    { const uint32_t t = min(w[1], w[3]); w[3] = max(w[1], w[3]); w[1] = t; }
    { const uint32_t t = min(w[4], w[6]); w[6] = max(w[4], w[6]); w[4] = t; }
    { const uint32_t t = min(w[5], w[7]); w[7] = max(w[5], w[7]); w[5] = t; }
    { const uint32_t t = min(w[1], w[2]); w[2] = max(w[1], w[2]); w[1] = t; }
    { const uint32_t t = min(w[5], w[6]); w[6] = max(w[5], w[6]); w[5] = t; }
    { const uint32_t t = min(w[0], w[4]); w[4] = max(w[0], w[4]); w[0] = t; }
    { const uint32_t t = min(w[1], w[5]); w[5] = max(w[1], w[5]); w[1] = t; }
    { const uint32_t t = min(w[2], w[6]); w[6] = max(w[2], w[6]); w[2] = t; }
    { const uint32_t t = min(w[3], w[7]); w[7] = max(w[3], w[7]); w[3] = t; }
    { const uint32_t t = min(w[2], w[4]); w[4] = max(w[2], w[4]); w[2] = t; }
    { const uint32_t t = min(w[3], w[5]); w[5] = max(w[3], w[5]); w[3] = t; }
    { const uint32_t t = min(w[1], w[2]); w[2] = max(w[1], w[2]); w[1] = t; }
    { const uint32_t t = min(w[3], w[4]); w[4] = max(w[3], w[4]); w[3] = t; }
    { const uint32_t t = min(w[5], w[6]); w[6] = max(w[5], w[6]); w[5] = t; }
    { const uint32_t t = min(w[0], w[8]); w[8] = max(w[0], w[8]); w[0] = t; }
    { const uint32_t t = min(w[4], w[8]); w[8] = max(w[4], w[8]); w[4] = t; }
    { const uint32_t t = min(w[2], w[4]); w[4] = max(w[2], w[4]); w[2] = t; }
    { const uint32_t t = min(w[3], w[5]); w[5] = max(w[3], w[5]); w[3] = t; }
    { const uint32_t t = min(w[6], w[8]); w[8] = max(w[6], w[8]); w[6] = t; }
    { const uint32_t t = min(w[1], w[2]); w[2] = max(w[1], w[2]); w[1] = t; }
    { const uint32_t t = min(w[3], w[4]); w[4] = max(w[3], w[4]); w[3] = t; }
    { const uint32_t t = min(w[5], w[6]); w[6] = max(w[5], w[6]); w[5] = t; }
    { const uint32_t t = min(w[7], w[8]); w[8] = max(w[7], w[8]); w[7] = t; }
    s[0] = w[0];
    s[1] = w[1];
    s[2] = w[2];
    s[3] = w[3];
    s[4] = w[4];
    s[5] = w[5];
    s[6] = w[6];
    s[7] = w[7];
    s[8] = w[8];
}

// The 14th smallest of a[0..8], b[0..8], c[0..8], each sorted ascending.
__device__ __forceinline__ uint32_t median3x9(const uint32_t *a, const uint32_t *b, const uint32_t *c) {
    uint32_t w[64];
    w[0] = a[0];
    w[1] = a[1];
    w[2] = a[2];
    w[3] = a[3];
    w[4] = a[4];
    w[5] = a[5];
    w[6] = a[6];
    w[7] = a[7];
    w[8] = a[8];
    w[16] = b[0];
    w[17] = b[1];
    w[18] = b[2];
    w[19] = b[3];
    w[20] = b[4];
    w[21] = b[5];
    w[22] = b[6];
    w[23] = b[7];
    w[24] = b[8];
    w[32] = c[0];
    w[33] = c[1];
    w[34] = c[2];
    w[35] = c[3];
    w[36] = c[4];
    w[37] = c[5];
    w[38] = c[6];
    w[39] = c[7];
    w[40] = c[8];
    { const uint32_t t = min(w[0], w[16]); w[16] = max(w[0], w[16]); w[0] = t; }
    { const uint32_t t = min(w[1], w[17]); w[17] = max(w[1], w[17]); w[1] = t; }
    { const uint32_t t = min(w[2], w[18]); w[18] = max(w[2], w[18]); w[2] = t; }
    { const uint32_t t = min(w[3], w[19]); w[19] = max(w[3], w[19]); w[3] = t; }
    { const uint32_t t = min(w[4], w[20]); w[20] = max(w[4], w[20]); w[4] = t; }
    { const uint32_t t = min(w[5], w[21]); w[21] = max(w[5], w[21]); w[5] = t; }
    { const uint32_t t = min(w[6], w[22]); w[22] = max(w[6], w[22]); w[6] = t; }
    { const uint32_t t = min(w[7], w[23]); w[23] = max(w[7], w[23]); w[7] = t; }
    { const uint32_t t = min(w[8], w[24]); w[24] = max(w[8], w[24]); w[8] = t; }
    { const uint32_t t = min(w[8], w[16]); w[16] = max(w[8], w[16]); w[8] = t; }
    { const uint32_t t = min(w[4], w[8]); w[8] = max(w[4], w[8]); w[4] = t; }
    { const uint32_t t = min(w[5], w[17]); w[17] = max(w[5], w[17]); w[5] = t; }
    { const uint32_t t = min(w[6], w[18]); w[18] = max(w[6], w[18]); w[6] = t; }
    { const uint32_t t = min(w[7], w[19]); w[19] = max(w[7], w[19]); w[7] = t; }
    { const uint32_t t = min(w[20], w[16]); w[16] = max(w[20], w[16]); w[20] = t; }
    { const uint32_t t = min(w[2], w[4]); w[4] = max(w[2], w[4]); w[2] = t; }
    { const uint32_t t = min(w[3], w[5]); w[5] = max(w[3], w[5]); w[3] = t; }
    { const uint32_t t = min(w[6], w[8]); w[8] = max(w[6], w[8]); w[6] = t; }
    { const uint32_t t = min(w[7], w[17]); w[17] = max(w[7], w[17]); w[7] = t; }
    { const uint32_t t = min(w[18], w[20]); w[20] = max(w[18], w[20]); w[18] = t; }
    { const uint32_t t = min(w[19], w[21]); w[21] = max(w[19], w[21]); w[19] = t; }
    { const uint32_t t = min(w[22], w[16]); w[16] = max(w[22], w[16]); w[22] = t; }
    { const uint32_t t = min(w[1], w[2]); w[2] = max(w[1], w[2]); w[1] = t; }
    { const uint32_t t = min(w[3], w[4]); w[4] = max(w[3], w[4]); w[3] = t; }
    { const uint32_t t = min(w[5], w[6]); w[6] = max(w[5], w[6]); w[5] = t; }
    { const uint32_t t = min(w[7], w[8]); w[8] = max(w[7], w[8]); w[7] = t; }
    { const uint32_t t = min(w[17], w[18]); w[18] = max(w[17], w[18]); w[17] = t; }
    { const uint32_t t = min(w[19], w[20]); w[20] = max(w[19], w[20]); w[19] = t; }
    { const uint32_t t = min(w[21], w[22]); w[22] = max(w[21], w[22]); w[21] = t; }
    w[16] = max(w[23], w[16]);
    w[32] = max(w[0], w[32]);
    w[33] = max(w[1], w[33]);
    w[34] = max(w[2], w[34]);
    w[35] = max(w[3], w[35]);
    w[36] = max(w[4], w[36]);
    w[37] = max(w[5], w[37]);
    w[38] = max(w[6], w[38]);
    w[7] = min(w[7], w[39]);
    w[8] = min(w[8], w[40]);
    w[16] = min(w[16], w[32]);
    w[24] = min(w[24], w[33]);
    w[16] = max(w[8], w[16]);
    w[24] = max(w[17], w[24]);
    w[34] = max(w[18], w[34]);
    w[19] = min(w[19], w[35]);
    w[20] = min(w[20], w[36]);
    w[21] = min(w[21], w[37]);
    w[22] = min(w[22], w[38]);
    w[19] = max(w[7], w[19]);
    w[16] = max(w[20], w[16]);
    w[21] = min(w[21], w[24]);
    w[22] = min(w[22], w[34]);
    w[21] = max(w[19], w[21]);
    w[22] = min(w[22], w[16]);
    w[21] = min(w[21], w[22]);
    return w[21];
}

// Packed unsigned 16-bit min and max of both halves (sm_90 and later).
__device__ __forceinline__ uint32_t vmin16x2(uint32_t a, uint32_t b) {
    uint32_t d;
    asm("min.u16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
    return d;
}
__device__ __forceinline__ uint32_t vmax16x2(uint32_t a, uint32_t b) {
    uint32_t d;
    asm("max.u16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
    return d;
}

// sort9 on two voxels: every word of v holds one value of each.
__device__ __forceinline__ void sort9x2(const uint32_t *v, uint32_t *s) {
    uint32_t w[16];
    w[0] = v[0];
    w[1] = v[1];
    w[2] = v[2];
    w[3] = v[3];
    w[4] = v[4];
    w[5] = v[5];
    w[6] = v[6];
    w[7] = v[7];
    w[8] = v[8];
    { const uint32_t t = vmin16x2(w[0], w[1]); w[1] = vmax16x2(w[0], w[1]); w[0] = t; }
    { const uint32_t t = vmin16x2(w[2], w[3]); w[3] = vmax16x2(w[2], w[3]); w[2] = t; }
    { const uint32_t t = vmin16x2(w[4], w[5]); w[5] = vmax16x2(w[4], w[5]); w[4] = t; }
    { const uint32_t t = vmin16x2(w[6], w[7]); w[7] = vmax16x2(w[6], w[7]); w[6] = t; }
    { const uint32_t t = vmin16x2(w[0], w[2]); w[2] = vmax16x2(w[0], w[2]); w[0] = t; }
    { const uint32_t t = vmin16x2(w[1], w[3]); w[3] = vmax16x2(w[1], w[3]); w[1] = t; }
    { const uint32_t t = vmin16x2(w[4], w[6]); w[6] = vmax16x2(w[4], w[6]); w[4] = t; }
    { const uint32_t t = vmin16x2(w[5], w[7]); w[7] = vmax16x2(w[5], w[7]); w[5] = t; }
    { const uint32_t t = vmin16x2(w[1], w[2]); w[2] = vmax16x2(w[1], w[2]); w[1] = t; }
    { const uint32_t t = vmin16x2(w[5], w[6]); w[6] = vmax16x2(w[5], w[6]); w[5] = t; }
    { const uint32_t t = vmin16x2(w[0], w[4]); w[4] = vmax16x2(w[0], w[4]); w[0] = t; }
    { const uint32_t t = vmin16x2(w[1], w[5]); w[5] = vmax16x2(w[1], w[5]); w[1] = t; }
    { const uint32_t t = vmin16x2(w[2], w[6]); w[6] = vmax16x2(w[2], w[6]); w[2] = t; }
    { const uint32_t t = vmin16x2(w[3], w[7]); w[7] = vmax16x2(w[3], w[7]); w[3] = t; }
    { const uint32_t t = vmin16x2(w[2], w[4]); w[4] = vmax16x2(w[2], w[4]); w[2] = t; }
    { const uint32_t t = vmin16x2(w[3], w[5]); w[5] = vmax16x2(w[3], w[5]); w[3] = t; }
    { const uint32_t t = vmin16x2(w[1], w[2]); w[2] = vmax16x2(w[1], w[2]); w[1] = t; }
    { const uint32_t t = vmin16x2(w[3], w[4]); w[4] = vmax16x2(w[3], w[4]); w[3] = t; }
    { const uint32_t t = vmin16x2(w[5], w[6]); w[6] = vmax16x2(w[5], w[6]); w[5] = t; }
    { const uint32_t t = vmin16x2(w[0], w[8]); w[8] = vmax16x2(w[0], w[8]); w[0] = t; }
    { const uint32_t t = vmin16x2(w[4], w[8]); w[8] = vmax16x2(w[4], w[8]); w[4] = t; }
    { const uint32_t t = vmin16x2(w[2], w[4]); w[4] = vmax16x2(w[2], w[4]); w[2] = t; }
    { const uint32_t t = vmin16x2(w[3], w[5]); w[5] = vmax16x2(w[3], w[5]); w[3] = t; }
    { const uint32_t t = vmin16x2(w[6], w[8]); w[8] = vmax16x2(w[6], w[8]); w[6] = t; }
    { const uint32_t t = vmin16x2(w[1], w[2]); w[2] = vmax16x2(w[1], w[2]); w[1] = t; }
    { const uint32_t t = vmin16x2(w[3], w[4]); w[4] = vmax16x2(w[3], w[4]); w[3] = t; }
    { const uint32_t t = vmin16x2(w[5], w[6]); w[6] = vmax16x2(w[5], w[6]); w[5] = t; }
    { const uint32_t t = vmin16x2(w[7], w[8]); w[8] = vmax16x2(w[7], w[8]); w[7] = t; }
    s[0] = w[0];
    s[1] = w[1];
    s[2] = w[2];
    s[3] = w[3];
    s[4] = w[4];
    s[5] = w[5];
    s[6] = w[6];
    s[7] = w[7];
    s[8] = w[8];
}

// median3x9 on two voxels (packed as in sort9x2).
__device__ __forceinline__ uint32_t median3x9x2(const uint32_t *a, const uint32_t *b, const uint32_t *c) {
    uint32_t w[64];
    w[0] = a[0];
    w[1] = a[1];
    w[2] = a[2];
    w[3] = a[3];
    w[4] = a[4];
    w[5] = a[5];
    w[6] = a[6];
    w[7] = a[7];
    w[8] = a[8];
    w[16] = b[0];
    w[17] = b[1];
    w[18] = b[2];
    w[19] = b[3];
    w[20] = b[4];
    w[21] = b[5];
    w[22] = b[6];
    w[23] = b[7];
    w[24] = b[8];
    w[32] = c[0];
    w[33] = c[1];
    w[34] = c[2];
    w[35] = c[3];
    w[36] = c[4];
    w[37] = c[5];
    w[38] = c[6];
    w[39] = c[7];
    w[40] = c[8];
    { const uint32_t t = vmin16x2(w[0], w[16]); w[16] = vmax16x2(w[0], w[16]); w[0] = t; }
    { const uint32_t t = vmin16x2(w[1], w[17]); w[17] = vmax16x2(w[1], w[17]); w[1] = t; }
    { const uint32_t t = vmin16x2(w[2], w[18]); w[18] = vmax16x2(w[2], w[18]); w[2] = t; }
    { const uint32_t t = vmin16x2(w[3], w[19]); w[19] = vmax16x2(w[3], w[19]); w[3] = t; }
    { const uint32_t t = vmin16x2(w[4], w[20]); w[20] = vmax16x2(w[4], w[20]); w[4] = t; }
    { const uint32_t t = vmin16x2(w[5], w[21]); w[21] = vmax16x2(w[5], w[21]); w[5] = t; }
    { const uint32_t t = vmin16x2(w[6], w[22]); w[22] = vmax16x2(w[6], w[22]); w[6] = t; }
    { const uint32_t t = vmin16x2(w[7], w[23]); w[23] = vmax16x2(w[7], w[23]); w[7] = t; }
    { const uint32_t t = vmin16x2(w[8], w[24]); w[24] = vmax16x2(w[8], w[24]); w[8] = t; }
    { const uint32_t t = vmin16x2(w[8], w[16]); w[16] = vmax16x2(w[8], w[16]); w[8] = t; }
    { const uint32_t t = vmin16x2(w[4], w[8]); w[8] = vmax16x2(w[4], w[8]); w[4] = t; }
    { const uint32_t t = vmin16x2(w[5], w[17]); w[17] = vmax16x2(w[5], w[17]); w[5] = t; }
    { const uint32_t t = vmin16x2(w[6], w[18]); w[18] = vmax16x2(w[6], w[18]); w[6] = t; }
    { const uint32_t t = vmin16x2(w[7], w[19]); w[19] = vmax16x2(w[7], w[19]); w[7] = t; }
    { const uint32_t t = vmin16x2(w[20], w[16]); w[16] = vmax16x2(w[20], w[16]); w[20] = t; }
    { const uint32_t t = vmin16x2(w[2], w[4]); w[4] = vmax16x2(w[2], w[4]); w[2] = t; }
    { const uint32_t t = vmin16x2(w[3], w[5]); w[5] = vmax16x2(w[3], w[5]); w[3] = t; }
    { const uint32_t t = vmin16x2(w[6], w[8]); w[8] = vmax16x2(w[6], w[8]); w[6] = t; }
    { const uint32_t t = vmin16x2(w[7], w[17]); w[17] = vmax16x2(w[7], w[17]); w[7] = t; }
    { const uint32_t t = vmin16x2(w[18], w[20]); w[20] = vmax16x2(w[18], w[20]); w[18] = t; }
    { const uint32_t t = vmin16x2(w[19], w[21]); w[21] = vmax16x2(w[19], w[21]); w[19] = t; }
    { const uint32_t t = vmin16x2(w[22], w[16]); w[16] = vmax16x2(w[22], w[16]); w[22] = t; }
    { const uint32_t t = vmin16x2(w[1], w[2]); w[2] = vmax16x2(w[1], w[2]); w[1] = t; }
    { const uint32_t t = vmin16x2(w[3], w[4]); w[4] = vmax16x2(w[3], w[4]); w[3] = t; }
    { const uint32_t t = vmin16x2(w[5], w[6]); w[6] = vmax16x2(w[5], w[6]); w[5] = t; }
    { const uint32_t t = vmin16x2(w[7], w[8]); w[8] = vmax16x2(w[7], w[8]); w[7] = t; }
    { const uint32_t t = vmin16x2(w[17], w[18]); w[18] = vmax16x2(w[17], w[18]); w[17] = t; }
    { const uint32_t t = vmin16x2(w[19], w[20]); w[20] = vmax16x2(w[19], w[20]); w[19] = t; }
    { const uint32_t t = vmin16x2(w[21], w[22]); w[22] = vmax16x2(w[21], w[22]); w[21] = t; }
    w[16] = vmax16x2(w[23], w[16]);
    w[32] = vmax16x2(w[0], w[32]);
    w[33] = vmax16x2(w[1], w[33]);
    w[34] = vmax16x2(w[2], w[34]);
    w[35] = vmax16x2(w[3], w[35]);
    w[36] = vmax16x2(w[4], w[36]);
    w[37] = vmax16x2(w[5], w[37]);
    w[38] = vmax16x2(w[6], w[38]);
    w[7] = vmin16x2(w[7], w[39]);
    w[8] = vmin16x2(w[8], w[40]);
    w[16] = vmin16x2(w[16], w[32]);
    w[24] = vmin16x2(w[24], w[33]);
    w[16] = vmax16x2(w[8], w[16]);
    w[24] = vmax16x2(w[17], w[24]);
    w[34] = vmax16x2(w[18], w[34]);
    w[19] = vmin16x2(w[19], w[35]);
    w[20] = vmin16x2(w[20], w[36]);
    w[21] = vmin16x2(w[21], w[37]);
    w[22] = vmin16x2(w[22], w[38]);
    w[19] = vmax16x2(w[7], w[19]);
    w[16] = vmax16x2(w[20], w[16]);
    w[21] = vmin16x2(w[21], w[24]);
    w[22] = vmin16x2(w[22], w[34]);
    w[21] = vmax16x2(w[19], w[21]);
    w[22] = vmin16x2(w[22], w[16]);
    w[21] = vmin16x2(w[21], w[22]);
    return w[21];
}
