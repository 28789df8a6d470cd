// Generated by gen_median27.py: median (14th smallest) of 27 values by
// a pruned odd-even merge network (126 comparators).
#pragma once

__device__ __forceinline__ uint32_t median27_net(uint32_t *v) {
    { const uint32_t t = min(v[0], v[1]); v[1] = max(v[0], v[1]); v[0] = t; }
    { const uint32_t t = min(v[2], v[3]); v[3] = max(v[2], v[3]); v[2] = t; }
    { const uint32_t t = min(v[4], v[5]); v[5] = max(v[4], v[5]); v[4] = t; }
    { const uint32_t t = min(v[6], v[7]); v[7] = max(v[6], v[7]); v[6] = t; }
    { const uint32_t t = min(v[8], v[9]); v[9] = max(v[8], v[9]); v[8] = t; }
    { const uint32_t t = min(v[10], v[11]); v[11] = max(v[10], v[11]); v[10] = t; }
    { const uint32_t t = min(v[12], v[13]); v[13] = max(v[12], v[13]); v[12] = t; }
    { const uint32_t t = min(v[14], v[15]); v[15] = max(v[14], v[15]); v[14] = t; }
    { const uint32_t t = min(v[16], v[17]); v[17] = max(v[16], v[17]); v[16] = t; }
    { const uint32_t t = min(v[18], v[19]); v[19] = max(v[18], v[19]); v[18] = t; }
    { const uint32_t t = min(v[20], v[21]); v[21] = max(v[20], v[21]); v[20] = t; }
    { const uint32_t t = min(v[22], v[23]); v[23] = max(v[22], v[23]); v[22] = t; }
    { const uint32_t t = min(v[24], v[25]); v[25] = max(v[24], v[25]); v[24] = t; }
    { const uint32_t t = min(v[0], v[2]); v[2] = max(v[0], v[2]); v[0] = t; }
    { const uint32_t t = min(v[1], v[3]); v[3] = max(v[1], v[3]); v[1] = t; }
    { const uint32_t t = min(v[4], v[6]); v[6] = max(v[4], v[6]); v[4] = t; }
    { const uint32_t t = min(v[5], v[7]); v[7] = max(v[5], v[7]); v[5] = t; }
    { const uint32_t t = min(v[8], v[10]); v[10] = max(v[8], v[10]); v[8] = t; }
    { const uint32_t t = min(v[9], v[11]); v[11] = max(v[9], v[11]); v[9] = t; }
    { const uint32_t t = min(v[12], v[14]); v[14] = max(v[12], v[14]); v[12] = t; }
    { const uint32_t t = min(v[13], v[15]); v[15] = max(v[13], v[15]); v[13] = t; }
    { const uint32_t t = min(v[16], v[18]); v[18] = max(v[16], v[18]); v[16] = t; }
    { const uint32_t t = min(v[17], v[19]); v[19] = max(v[17], v[19]); v[17] = t; }
    { const uint32_t t = min(v[20], v[22]); v[22] = max(v[20], v[22]); v[20] = t; }
    { const uint32_t t = min(v[21], v[23]); v[23] = max(v[21], v[23]); v[21] = t; }
    { const uint32_t t = min(v[24], v[26]); v[26] = max(v[24], v[26]); v[24] = t; }
    { const uint32_t t = min(v[1], v[2]); v[2] = max(v[1], v[2]); v[1] = t; }
    { const uint32_t t = min(v[5], v[6]); v[6] = max(v[5], v[6]); v[5] = t; }
    { const uint32_t t = min(v[9], v[10]); v[10] = max(v[9], v[10]); v[9] = t; }
    { const uint32_t t = min(v[13], v[14]); v[14] = max(v[13], v[14]); v[13] = t; }
    { const uint32_t t = min(v[17], v[18]); v[18] = max(v[17], v[18]); v[17] = t; }
    { const uint32_t t = min(v[21], v[22]); v[22] = max(v[21], v[22]); v[21] = t; }
    { const uint32_t t = min(v[25], v[26]); v[26] = max(v[25], v[26]); v[25] = t; }
    { const uint32_t t = min(v[0], v[4]); v[4] = max(v[0], v[4]); v[0] = t; }
    { const uint32_t t = min(v[1], v[5]); v[5] = max(v[1], v[5]); v[1] = t; }
    { const uint32_t t = min(v[2], v[6]); v[6] = max(v[2], v[6]); v[2] = t; }
    { const uint32_t t = min(v[3], v[7]); v[7] = max(v[3], v[7]); v[3] = t; }
    { const uint32_t t = min(v[8], v[12]); v[12] = max(v[8], v[12]); v[8] = t; }
    { const uint32_t t = min(v[9], v[13]); v[13] = max(v[9], v[13]); v[9] = t; }
    { const uint32_t t = min(v[10], v[14]); v[14] = max(v[10], v[14]); v[10] = t; }
    { const uint32_t t = min(v[11], v[15]); v[15] = max(v[11], v[15]); v[11] = t; }
    { const uint32_t t = min(v[16], v[20]); v[20] = max(v[16], v[20]); v[16] = t; }
    { const uint32_t t = min(v[17], v[21]); v[21] = max(v[17], v[21]); v[17] = t; }
    { const uint32_t t = min(v[18], v[22]); v[22] = max(v[18], v[22]); v[18] = t; }
    { const uint32_t t = min(v[19], v[23]); v[23] = max(v[19], v[23]); v[19] = t; }
    { const uint32_t t = min(v[2], v[4]); v[4] = max(v[2], v[4]); v[2] = t; }
    { const uint32_t t = min(v[3], v[5]); v[5] = max(v[3], v[5]); v[3] = t; }
    { const uint32_t t = min(v[10], v[12]); v[12] = max(v[10], v[12]); v[10] = t; }
    { const uint32_t t = min(v[11], v[13]); v[13] = max(v[11], v[13]); v[11] = t; }
    { const uint32_t t = min(v[18], v[20]); v[20] = max(v[18], v[20]); v[18] = t; }
    { const uint32_t t = min(v[19], v[21]); v[21] = max(v[19], v[21]); v[19] = t; }
    { const uint32_t t = min(v[1], v[2]); v[2] = max(v[1], v[2]); v[1] = t; }
    { const uint32_t t = min(v[3], v[4]); v[4] = max(v[3], v[4]); v[3] = t; }
    { const uint32_t t = min(v[5], v[6]); v[6] = max(v[5], v[6]); v[5] = t; }
    { const uint32_t t = min(v[9], v[10]); v[10] = max(v[9], v[10]); v[9] = t; }
    { const uint32_t t = min(v[11], v[12]); v[12] = max(v[11], v[12]); v[11] = t; }
    { const uint32_t t = min(v[13], v[14]); v[14] = max(v[13], v[14]); v[13] = t; }
    { const uint32_t t = min(v[17], v[18]); v[18] = max(v[17], v[18]); v[17] = t; }
    { const uint32_t t = min(v[19], v[20]); v[20] = max(v[19], v[20]); v[19] = t; }
    { const uint32_t t = min(v[21], v[22]); v[22] = max(v[21], v[22]); v[21] = t; }
    { const uint32_t t = min(v[25], v[26]); v[26] = max(v[25], v[26]); v[25] = t; }
    { const uint32_t t = min(v[0], v[8]); v[8] = max(v[0], v[8]); v[0] = t; }
    { const uint32_t t = min(v[1], v[9]); v[9] = max(v[1], v[9]); v[1] = t; }
    { const uint32_t t = min(v[2], v[10]); v[10] = max(v[2], v[10]); v[2] = t; }
    { const uint32_t t = min(v[3], v[11]); v[11] = max(v[3], v[11]); v[3] = t; }
    { const uint32_t t = min(v[4], v[12]); v[12] = max(v[4], v[12]); v[4] = t; }
    { const uint32_t t = min(v[5], v[13]); v[13] = max(v[5], v[13]); v[5] = t; }
    { const uint32_t t = min(v[6], v[14]); v[14] = max(v[6], v[14]); v[6] = t; }
    v[7] = min(v[7], v[15]);
    { const uint32_t t = min(v[16], v[24]); v[24] = max(v[16], v[24]); v[16] = t; }
    { const uint32_t t = min(v[17], v[25]); v[25] = max(v[17], v[25]); v[17] = t; }
    { const uint32_t t = min(v[18], v[26]); v[26] = max(v[18], v[26]); v[18] = t; }
    { const uint32_t t = min(v[4], v[8]); v[8] = max(v[4], v[8]); v[4] = t; }
    { const uint32_t t = min(v[5], v[9]); v[9] = max(v[5], v[9]); v[5] = t; }
    { const uint32_t t = min(v[6], v[10]); v[10] = max(v[6], v[10]); v[6] = t; }
    { const uint32_t t = min(v[7], v[11]); v[11] = max(v[7], v[11]); v[7] = t; }
    { const uint32_t t = min(v[20], v[24]); v[24] = max(v[20], v[24]); v[20] = t; }
    { const uint32_t t = min(v[21], v[25]); v[25] = max(v[21], v[25]); v[21] = t; }
    { const uint32_t t = min(v[22], v[26]); v[26] = max(v[22], v[26]); v[22] = t; }
    { const uint32_t t = min(v[2], v[4]); v[4] = max(v[2], v[4]); v[2] = t; }
    { const uint32_t t = min(v[3], v[5]); v[5] = max(v[3], v[5]); v[3] = t; }
    { const uint32_t t = min(v[6], v[8]); v[8] = max(v[6], v[8]); v[6] = t; }
    { const uint32_t t = min(v[7], v[9]); v[9] = max(v[7], v[9]); v[7] = t; }
    { const uint32_t t = min(v[10], v[12]); v[12] = max(v[10], v[12]); v[10] = t; }
    { const uint32_t t = min(v[11], v[13]); v[13] = max(v[11], v[13]); v[11] = t; }
    { const uint32_t t = min(v[18], v[20]); v[20] = max(v[18], v[20]); v[18] = t; }
    { const uint32_t t = min(v[19], v[21]); v[21] = max(v[19], v[21]); v[19] = t; }
    { const uint32_t t = min(v[22], v[24]); v[24] = max(v[22], v[24]); v[22] = t; }
    { const uint32_t t = min(v[23], v[25]); v[25] = max(v[23], v[25]); v[23] = t; }
    { const uint32_t t = min(v[1], v[2]); v[2] = max(v[1], v[2]); v[1] = t; }
    { const uint32_t t = min(v[3], v[4]); v[4] = max(v[3], v[4]); v[3] = t; }
    { const uint32_t t = min(v[5], v[6]); v[6] = max(v[5], v[6]); v[5] = t; }
    { const uint32_t t = min(v[7], v[8]); v[8] = max(v[7], v[8]); v[7] = t; }
    { const uint32_t t = min(v[9], v[10]); v[10] = max(v[9], v[10]); v[9] = t; }
    { const uint32_t t = min(v[11], v[12]); v[12] = max(v[11], v[12]); v[11] = t; }
    { const uint32_t t = min(v[13], v[14]); v[14] = max(v[13], v[14]); v[13] = t; }
    { const uint32_t t = min(v[17], v[18]); v[18] = max(v[17], v[18]); v[17] = t; }
    { const uint32_t t = min(v[19], v[20]); v[20] = max(v[19], v[20]); v[19] = t; }
    { const uint32_t t = min(v[21], v[22]); v[22] = max(v[21], v[22]); v[21] = t; }
    { const uint32_t t = min(v[23], v[24]); v[24] = max(v[23], v[24]); v[23] = t; }
    { const uint32_t t = min(v[25], v[26]); v[26] = max(v[25], v[26]); v[25] = t; }
    v[16] = max(v[0], v[16]);
    v[17] = max(v[1], v[17]);
    v[18] = max(v[2], v[18]);
    v[19] = max(v[3], v[19]);
    v[20] = max(v[4], v[20]);
    v[21] = max(v[5], v[21]);
    v[22] = max(v[6], v[22]);
    v[7] = min(v[7], v[23]);
    v[8] = min(v[8], v[24]);
    v[9] = min(v[9], v[25]);
    v[10] = min(v[10], v[26]);
    v[16] = max(v[8], v[16]);
    v[17] = max(v[9], v[17]);
    v[18] = max(v[10], v[18]);
    v[11] = min(v[11], v[19]);
    v[12] = min(v[12], v[20]);
    v[13] = min(v[13], v[21]);
    v[14] = min(v[14], v[22]);
    v[11] = max(v[7], v[11]);
    v[16] = max(v[12], v[16]);
    v[13] = min(v[13], v[17]);
    v[14] = min(v[14], v[18]);
    v[13] = max(v[11], v[13]);
    v[14] = min(v[14], v[16]);
    v[13] = min(v[13], v[14]);
    return v[13];
}
