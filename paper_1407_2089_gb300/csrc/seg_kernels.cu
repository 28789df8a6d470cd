// seg_kernels.cu -- sm_103a kernels of the segmentation stage.
//
// Paper: Wait et al., LEVER 3-D.  Background Noise Removal (Eq. 1: Gaussian
// low-pass, here binomial [1 4 6 4 1] per axis) and Segmentation (Otsu
// thresholding, ref. [11]; connected component filter; components below the
// user-set volume discarded).  Linear index i = x + X*(y + Y*z).
//
// Pipeline for one batch of volume-channels (all kernels walk the batch
// descriptor, so one launch sequence serves any mix of volume sizes):
//   init            zero histograms and status words
//   smooth_rows /   the one pass over the raw voxels: binomial smoothing in
//   smooth_hist     shared memory and registers, the smoothed volume written
//                   as uint16 (with each 32-voxel word's maximum for
//                   row-aligned volumes), a 65536-bin shared histogram merged
//                   into the volume's bins
//   otsu            one block per volume: bins -> t*
//   threshold_runs  pass over the smoothed volume: foreground = s > t*,
//                   written as a bit mask (32 voxels per word along x),
//                   foreground runs counted per x-row
//   row_runs        run table (x0, x1) per row (offsets from the row tiles
//                   below and the row counts); union-find parent = self
//   union_local,    26-adjacency between runs of neighbouring rows, union by
//   union           minimum run index, so a component's root is its first
//                   run in raster order (in shared memory within bricks of
//                   rows, then across brick faces)
//   flatten         parent = root; voxel count accumulated at the root
//   keep_count      roots with count >= min_volume, per row
//   rank            label of each kept root = 1 + its rank in raster order
//   label_features  per-voxel labels (coalesced uint32 rows) and per-cell
//                   count / bbox / coordinate sums
#include <climits>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <mutex>

#include <algorithm>
#include <type_traits>

#include "median27_net.h"
#include "seg_internal.h"

namespace seg {

const char *const kKernelNames[NUM_KERNELS] = {
    "denoise_box", "denoise_median", "init",       "mrf_stats",        "mrf_iterate",
    "smooth_rows", "smooth_hist",  "otsu",       "threshold_runs",
    "dilate",      "erode",          "dist_xy",    "dist_xy_1024",     "dist_x",
    "dist_y",      "dist_z",         "dist_z_long", "row_runs",
    "union_local", "union",          "flatten",    "keep_count",
    "rank",        "label_features", "gather_stat"};

namespace {

constexpr unsigned FULL = 0xFFFFFFFFu;
// Shared histogram: levels below HIST_LOW have a 32-bit counter in each of
// two copies (one per half-warp, the second offset by 16 words so that equal
// levels in the two copies sit in different banks); the rest share words as
// two 16-bit counters.
constexpr int HIST_LOW = 4096;
constexpr int HIST_COPY1 = HIST_LOW + 16;         // word offset of the second copy
constexpr int HIST_PAIRS = 2 * HIST_LOW + 16;     // word offset of the 16-bit pairs
constexpr int HIST_WORDS = HIST_PAIRS + (HIST_BINS - HIST_LOW) / 2;


// ----------------------------------------------------------------------------
// small helpers
// ----------------------------------------------------------------------------

__device__ __forceinline__ uint32_t find_vol_tile(const BatchHdr *__restrict__ h, uint32_t t) {
    uint32_t lo = 0, hi = h->nvol;
    while (hi - lo > 1) {
        uint32_t mid = (lo + hi) >> 1;
        if (h->vol[mid].tile_base <= t) lo = mid; else hi = mid;
    }
    return lo;
}

// Volume lookup for the persistent loops: the blocks copy the volumes' first
// flat indices of one kind (row tiles, bricks, ...) into shared memory once,
// so each item's binary search runs on shared memory rather than on one
// header cache line per step.  Batches of more than SMEM_VOLS volumes search
// the header itself.
constexpr uint32_t SMEM_VOLS = 512;

template <uint32_t VolDev::*BASE>
struct VolIndex {
    uint32_t base[SMEM_VOLS];
    __device__ __forceinline__ void load(const BatchHdr *__restrict__ h) {
        if (h->nvol <= SMEM_VOLS)
            for (uint32_t i = threadIdx.x; i < h->nvol; i += blockDim.x) base[i] = h->vol[i].*BASE;
        __syncthreads();
    }
    __device__ __forceinline__ uint32_t find(const BatchHdr *__restrict__ h, uint32_t t) const {
        const uint32_t nv = h->nvol;
        uint32_t lo = 0, hi = nv;
        if (nv <= SMEM_VOLS) {
            while (hi - lo > 1) {
                const uint32_t mid = (lo + hi) >> 1;
                if (base[mid] <= t) lo = mid; else hi = mid;
            }
        } else {
            while (hi - lo > 1) {
                const uint32_t mid = (lo + hi) >> 1;
                if (h->vol[mid].*BASE <= t) lo = mid; else hi = mid;
            }
        }
        return lo;
    }
};

// Exclusive block scan of one uint32 per thread; *total gets the block sum.
// sbuf: 33 words of shared memory.  Contains the barriers needed so that
// values read before the call are not overwritten by writes after it.
template <int NT>
__device__ __forceinline__ uint32_t block_exscan(uint32_t x, uint32_t *total, uint32_t *sbuf) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    uint32_t inc = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t a = __shfl_up_sync(FULL, inc, o);
        if (lane >= o) inc += a;
    }
    if (lane == 31) sbuf[wid] = inc;
    __syncthreads();
    if (wid == 0) {
        uint32_t w = lane < NT / 32 ? sbuf[lane] : 0u;
        uint32_t wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t a = __shfl_up_sync(FULL, wi, o);
            if (lane >= o) wi += a;
        }
        if (lane < NT / 32) sbuf[lane] = wi - w;
        if (lane == 31) sbuf[32] = wi;
    }
    __syncthreads();
    uint32_t r = sbuf[wid] + inc - x;
    *total = sbuf[32];
    __syncthreads();
    return r;
}

template <int NT>
__device__ __forceinline__ uint32_t block_sum(uint32_t x, uint32_t *sbuf) {
    uint32_t t;
    block_exscan<NT>(x, &t, sbuf);
    return t;
}

// Sum of a volume's row-tile totals below row tile lt, by the whole block
// (each block scans the tiles before its own instead of a separate scan
// kernel: a volume has at most a few thousand row tiles).
__device__ __forceinline__ uint32_t tiles_below(const uint32_t *__restrict__ tot, uint32_t lt, uint32_t *sbuf) {
    uint32_t s = 0;
    for (uint32_t i = threadIdx.x; i < lt; i += ROW_TILE) s += tot[i];
    return block_sum<ROW_TILE>(s, sbuf);
}

// First x >= p in the row whose mask bit equals `want`; X if none.  Bits at
// x >= X are zero by construction.
__device__ __forceinline__ uint32_t find_bit(const uint32_t *__restrict__ row, uint32_t W,
                                             uint32_t X, uint32_t p, bool want) {
    if (p >= X) return X;
    uint32_t w = p >> 5;
    uint32_t word = row[w];
    if (!want) word = ~word;
    word &= FULL << (p & 31);
    while (!word) {
        if (++w >= W) return X;
        word = row[w];
        if (!want) word = ~word;
    }
    uint32_t x = (w << 5) + (__ffs(word) - 1);
    return x < X ? x : X;
}

// ----------------------------------------------------------------------------
// union-find over runs (parent index <= own index at all times)
// ----------------------------------------------------------------------------

// Root of x without writing.  k_flatten must use this: a compressing store
// racing with another thread's final "parent = root" store could replace the
// root by an intermediate ancestor.  Reads go through L2 (ld.cg) because
// parents change under other SMs.
__device__ __forceinline__ uint32_t uf_root(const uint32_t *P, uint32_t x) {
    uint32_t p = __ldcg(P + x);
    while (p != x) {
        x = p;
        p = __ldcg(P + x);
    }
    return x;
}

// Root of x with path halving, for the union phase only: every visited node
// is re-pointed at its grandparent.  The store can only replace a parent by
// one of its ancestors (all parents point to lower indices), so it never
// breaks a path; if it overwrites a concurrent atomicMin, that union sees
// old != root and retries from the old parent, so no link is lost.
__device__ __forceinline__ uint32_t uf_find(uint32_t *P, uint32_t x) {
    uint32_t p = __ldcg(P + x);
    while (p != x) {
        const uint32_t g = __ldcg(P + p);
        if (g == p) return p;
        __stcg(P + x, g);
        x = g;
        p = __ldcg(P + x);
    }
    return x;
}

// Union with the lower index as the surviving root.  atomicMin only ever
// lowers a parent, so each component ends rooted at its minimum run index
// whatever the interleaving.  Bounded retries; exhaustion raises ERR_UNION.
__device__ __forceinline__ void uf_union(uint32_t *P, uint32_t a, uint32_t b, uint32_t *err,
                                         uint32_t limit) {
    for (uint32_t it = 0; it < limit; ++it) {
        a = uf_find(P, a);
        b = uf_find(P, b);
        if (a == b) return;
        if (a < b) {
            const uint32_t old = atomicMin(P + b, a);
            if (old == b) return;
            b = old;
        } else {
            const uint32_t old = atomicMin(P + a, b);
            if (old == a) return;
            a = old;
        }
    }
    atomicOr(err, ERR_UNION);
}

// ----------------------------------------------------------------------------
// 16-byte asynchronous global -> shared copies (cp.async, LDGSTS)
// ----------------------------------------------------------------------------

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

// dst (a shared-memory address) and src 16-byte aligned; cached in L2 only.
__device__ __forceinline__ void cp_async16(uint32_t dst, uintptr_t src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}

// 4-byte copy; n = 4 copies, n = 0 writes zeros (the source is not read).
__device__ __forceinline__ void cp_async4(uint32_t dst, uintptr_t src, uint32_t n) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(dst), "l"(src), "r"(n) : "memory");
}

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }

// Waits until at most N of this thread's committed groups are outstanding.
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// ----------------------------------------------------------------------------
// separable binomial smoothing of one tile
// ----------------------------------------------------------------------------
//
// A block of 8*TY threads owns a TILE_X x TY column of outputs (each thread 8
// adjacent outputs of one row) and marches along z from z0 - 2 to z1 + 1.
// Input planes stream through a ring of S shared-memory stages, S - 1 planes
// ahead of use.  For each of the plane's TY+4 halo rows the 16-byte-aligned
// 160-byte window holding the row's 68 needed voxels is copied as ten 16-byte
// cp.async chunks; the row's offset inside its window (0..7 voxels) is kept
// per row, so any X and any base alignment work.  Rows whose window would
// leave the volume's buffer (first and last rows of a volume) are read with
// plain loads instead.  The x pass (8 adjacent outputs from 12 inputs, edges
// clamped per axis) writes one of two shared buffers while the y pass (5
// rows) of the previous plane reads the other; the z pass is in scatter form:
// with accumulators a0..a3 holding the partial sums of outputs zi-2..zi+1,
//     out(zi-2) = a0 + P, a0 <- a1 + 4P, a1 <- a2 + 6P, a2 <- a3 + 4P, a3 <- P.
// All sums are exact in uint32 (at most 4096 * 65535); the one rounding
// (S + 2048) >> 12 is applied to the completed sum, which equals the 125-term
// definition.
//
// x-pass buffer layout: the 8 outputs of octet o of a row sit at words 4o..4o+3
// (the first four) and 32+4o..32+4o+3 (the last four), so that the eight
// threads of one row read or write 8 distinct groups of 4 banks.

template <int TY>
struct Tile {
    static constexpr int NT = 8 * TY;
    static constexpr int RH = TY + 4;
    static constexpr int PX_WORDS = RH * TILE_X;
    static constexpr int XITEMS = RH * (TILE_X / 8);  // x-pass octets per plane
    static constexpr int S = 3;              // ring stages
    static constexpr int ROWB = 160;         // bytes staged per halo row
    static constexpr int ROWE = ROWB / 2;    // voxels per staged row
    static constexpr int CHUNKS = ROWB / 16; // 16-byte copies per row
    static constexpr int NCHUNK = RH * CHUNKS;
    static constexpr int STAGE_BYTES = RH * ROWB;
    static constexpr int RING_BYTES = S * STAGE_BYTES;
    static constexpr int SHIFT_BYTES = (S * RH + 15) / 16 * 16;
    // dynamic shared memory without / with the shared histogram
    static constexpr size_t MASK_SMEM = RING_BYTES + 8 * PX_WORDS + SHIFT_BYTES;  // two x-pass buffers
    static constexpr size_t HIST_SMEM = MASK_SMEM + 4 * (size_t)HIST_WORDS;
    static_assert(NCHUNK <= 2 * NT, "at most two copy chunks per thread per plane");
    static_assert(XITEMS <= 2 * NT, "at most two x-pass octets per thread per plane");
};

struct Ring {
    unsigned char *stage;  // S stages of RH rows x ROWB bytes
    int8_t *shift;         // per stage and row: voxel offset in the window, -1 = plain loads
    uint32_t pc;           // planes consumed by this block so far
};

// x pass of 8 adjacent outputs from the 12 inputs v[0..11].
__device__ __forceinline__ void xpass8(const uint32_t *v, uint32_t *o) {
#pragma unroll
    for (int j = 0; j < 8; ++j) o[j] = v[j] + 4u * v[j + 1] + 6u * v[j + 2] + 4u * v[j + 3] + v[j + 4];
}

// The 12 inputs of an octet from the 7 staged words that hold them, the
// first input at voxel offset `odd` (0 or 1) of the first word.
__device__ __forceinline__ void unpack12(const uint32_t *w, bool odd, uint32_t *v) {
    const uint32_t sel = odd ? 0x5432u : 0x3210u;
    uint32_t wd[7];
#pragma unroll
    for (int k = 0; k < 7; ++k) wd[k] = w[k];
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        const uint32_t p = __byte_perm(wd[k], wd[k + 1], sel);
        v[2 * k] = p & 0xFFFFu;
        v[2 * k + 1] = p >> 16;
    }
}

template <int TY, class Emit>
__device__ __forceinline__ void smooth_tile(const uint16_t *__restrict__ raw, uint32_t X, uint32_t Y,
                                            uint32_t Z, int x0, int y0, int z0, int z1,
                                            uint32_t *__restrict__ spx, Ring &R, Emit &emit) {
    using T = Tile<TY>;
    const int tid = threadIdx.x;
    const int q = tid & 7, ty = tid >> 3;
    const int n = z1 - z0 + 4;
    const uint64_t plane = (uint64_t)X * Y;
    const uintptr_t lo = (uintptr_t)raw, hi = lo + 2 * plane * Z;
    // Planes strictly between the first and the last cannot take a window
    // outside the buffer when a plane holds more than two windows.
    const bool mid_inside = plane >= (uint64_t)T::ROWB;
    // this thread's copy chunks (at most two): halo row cr, 16-byte piece cc;
    // address of the row's first needed voxel in plane 0 (may lie before the
    // buffer)
    int cr[2], cc[2];
    uintptr_t crow[2];
#pragma unroll
    for (int u = 0; u < 2; ++u) {
        const int c = tid + u * T::NT;
        cr[u] = c / T::CHUNKS;
        cc[u] = c - cr[u] * T::CHUNKS;
        crow[u] = lo + (uintptr_t)(2 * ((int64_t)min(max(y0 - 2 + cr[u], 0), (int)Y - 1) * X + (x0 - 2)));
    }
    const uint32_t ring0 = smem_addr(R.stage);
    auto issue = [&](int zi, uint32_t st) {
        const int zc = min(max(zi, 0), (int)Z - 1);
        const bool mid = mid_inside && zc > 0 && zc + 1 < (int)Z;
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            if (tid + u * T::NT >= T::NCHUNK) break;
            const uintptr_t addr = crow[u] + 2 * plane * (uint64_t)zc;
            const uintptr_t a16 = addr & ~(uintptr_t)15;
            const bool inside = mid || (a16 >= lo && a16 + T::ROWB <= hi);
            if (cc[u] == 0) R.shift[st * T::RH + cr[u]] = inside ? (int8_t)((addr & 15) >> 1) : (int8_t)-1;
            if (inside)
                cp_async16(ring0 + st * T::STAGE_BYTES + cr[u] * T::ROWB + cc[u] * 16, a16 + 16 * cc[u]);
        }
    };
    // this thread's x-pass octets (row r, octet o of the 8 in a row); the
    // second one only for the first XITEMS - NT threads
    constexpr int EXTRA = T::XITEMS - T::NT;
    // this thread's x-pass octets (row r, octet o of the 8 in a row); the
    // second one for the last EXTRA threads, which issue at most one copy
    const bool two = EXTRA > 0 && tid >= T::NT - EXTRA;
    const int rA = tid >> 3, oA = tid & 7, rB = (tid + EXTRA) >> 3, oB = tid & 7;
    // an octet reads inputs x0 + 8 o - 2 .. x0 + 8 o + 9; at a volume edge
    // the inputs outside [0, X) take the edge voxel's value
    const int xa = x0 + 8 * oA - 2;           // first input of this thread's octets
    const bool fA = xa >= 0 && xa + 12 <= (int)X;
    auto xitem = [&](const unsigned char *stage, const int8_t *sh, uint32_t *px, int r, int o, bool f, int zi) {
        const int s = sh[r];
        uint32_t v[12];
        if (f && s == 6) {
            // rows of a 16-byte-aligned volume with X % 8 == 0: the octet's 12
            // inputs are words 3..8 of the three 16-byte chunks o, o+1, o+2
            const uint4 *c = reinterpret_cast<const uint4 *>(stage + r * T::ROWB) + o;
            const uint4 c0 = c[0], c1 = c[1], c2 = c[2];
            const uint32_t wd[6] = {c0.w, c1.x, c1.y, c1.z, c1.w, c2.x};
#pragma unroll
            for (int k = 0; k < 6; ++k) {
                v[2 * k] = wd[k] & 0xFFFFu;
                v[2 * k + 1] = wd[k] >> 16;
            }
        } else if (s >= 0) {
            const int off = r * T::ROWE + s + 8 * o;
            unpack12(reinterpret_cast<const uint32_t *>(stage) + (off >> 1), off & 1, v);
            if (!f) {
                // the window also holds x = 0 and x = X - 1 when the octet
                // reaches past them (indices clamped for octets wholly past X,
                // whose outputs are not used)
                const uint16_t *st16 = reinterpret_cast<const uint16_t *>(stage) + r * T::ROWE;
                const int jr = (int)X - 1 - xa;  // last input inside the row
                const uint32_t vl = st16[min(max(2 - x0 + s, 0), T::ROWE - 1)];
                const uint32_t vr = st16[min(max((int)X + 1 - x0 + s, 0), T::ROWE - 1)];
#pragma unroll
                for (int j = 0; j < 12; ++j) {
                    if (xa + j < 0) v[j] = vl;
                    if (j > jr) v[j] = vr;
                }
            }
        } else {
            // a row read with plain loads: clamp every x
            const uint64_t rowg = ((uint64_t)min(max(zi, 0), (int)Z - 1) * Y +
                                   (uint64_t)min(max(y0 - 2 + r, 0), (int)Y - 1)) * X;
#pragma unroll
            for (int j = 0; j < 12; ++j) v[j] = __ldg(raw + rowg + min(max(x0 - 2 + 8 * o + j, 0), (int)X - 1));
        }
        uint32_t out[8];
        xpass8(v, out);
        uint32_t *d = px + r * TILE_X + 4 * o;
        *reinterpret_cast<uint4 *>(d) = make_uint4(out[0], out[1], out[2], out[3]);
        *reinterpret_cast<uint4 *>(d + 32) = make_uint4(out[4], out[5], out[6], out[7]);
    };
    const uint32_t *py = spx + ty * TILE_X + 4 * q;  // this thread's y-pass column
    emit.bind(x0 + 8 * q, y0 + ty);
    __syncthreads();  // the previous tile is done with the ring and spx
#pragma unroll
    for (int j = 0; j < T::S - 1; ++j) {
        if (j < n) issue(z0 - 2 + j, (R.pc + j) % T::S);
        cp_async_commit();
    }
    uint32_t a0[8], a1[8], a2[8], a3[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) a0[j] = a1[j] = a2[j] = a3[j] = 0u;
    // Iteration k runs the x pass of plane k into buffer k & 1 and the y and
    // z passes of plane k - 1 from the other buffer, so one barrier per plane
    // separates the two uses of each buffer and of each ring stage.
    for (int k = 0; k <= n; ++k) {
        if (k < n) cp_async_wait<T::S - 2>();  // this thread's chunks of plane k have landed
        __syncthreads();  // everyone's have; x pass k-1 is written; y pass k-2 is done
        if (k < n) {
            const int zi = z0 - 2 + k;
            const uint32_t st = (R.pc + k) % T::S;
            const unsigned char *stage = R.stage + st * T::STAGE_BYTES;
            const int8_t *sh = R.shift + st * T::RH;
            uint32_t *px = spx + (k & 1) * T::PX_WORDS;
            xitem(stage, sh, px, rA, oA, fA, zi);
            if (two) xitem(stage, sh, px, rB, oB, fA, zi);
            // the stage of plane k-1 was last read before the barrier above
            if (k + T::S - 1 < n) issue(zi + T::S - 1, (R.pc + k + T::S - 1) % T::S);
            cp_async_commit();
        }
        if (k > 0) {
            const uint32_t *pk = py + ((k - 1) & 1) * T::PX_WORDS;
            const int zi = z0 - 3 + k;  // plane k - 1
            uint32_t p[8];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const uint4 r0 = *reinterpret_cast<const uint4 *>(pk + 32 * h + 0 * TILE_X);
                const uint4 r1 = *reinterpret_cast<const uint4 *>(pk + 32 * h + 1 * TILE_X);
                const uint4 r2 = *reinterpret_cast<const uint4 *>(pk + 32 * h + 2 * TILE_X);
                const uint4 r3 = *reinterpret_cast<const uint4 *>(pk + 32 * h + 3 * TILE_X);
                const uint4 r4 = *reinterpret_cast<const uint4 *>(pk + 32 * h + 4 * TILE_X);
                p[4 * h + 0] = r0.x + 4u * r1.x + 6u * r2.x + 4u * r3.x + r4.x;
                p[4 * h + 1] = r0.y + 4u * r1.y + 6u * r2.y + 4u * r3.y + r4.y;
                p[4 * h + 2] = r0.z + 4u * r1.z + 6u * r2.z + 4u * r3.z + r4.z;
                p[4 * h + 3] = r0.w + 4u * r1.w + 6u * r2.w + 4u * r3.w + r4.w;
            }
            uint32_t s[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const uint32_t out = a0[j] + p[j];
                a0[j] = a1[j] + 4u * p[j];
                a1[j] = a2[j] + 6u * p[j];
                a2[j] = a3[j] + 4u * p[j];
                a3[j] = p[j];
                s[j] = (out + 2048u) >> 12;
            }
            emit(zi - 2, zi >= z0 + 2, s);
        }
    }
    cp_async_wait<0>();  // only empty groups remain; keeps the count at zero between tiles
    R.pc += (uint32_t)n;
}

// Histogram emit.  Levels below HIST_LOW (where microscope data live) count
// in 32-bit shared words; higher levels share words as two 16-bit counters,
// and the thread whose increment takes such a counter to 0x8000 moves 0x8000
// to the global bin, so a counter never exceeds 0x8000 + (increments in
// flight) < 0x10000 and never carries into its neighbour.  With STORE the
// smoothed voxels are also written (16-byte stores when rows are 16-byte
// aligned).  bind() fixes, per tile, which of the thread's 8 voxels lie
// inside the volume.
template <bool STORE>
struct HistEmit {
    uint32_t *sh;
    uint32_t *gh;
    uint16_t *sm;       // smoothed volume (STORE only)
    uint32_t X, Y;
    uint32_t valid;     // bit j: voxel j of the octet is inside the volume
    uint32_t copy;      // word offset of this half-warp's copy of the low levels
    uint16_t *row;      // &sm[y * X + xb] at z = 0
    size_t zstride;     // voxels per z-plane
    bool vec;           // all 8 inside and 16-byte aligned
    __device__ __forceinline__ void bind(int xb, int y) {
        valid = 0;
        if ((uint32_t)y < Y)
            for (int j = 0; j < 8; ++j) valid |= ((uint32_t)(xb + j) < X ? 1u : 0u) << j;
        copy = (threadIdx.x & 16u) ? (uint32_t)HIST_COPY1 : 0u;
        if (STORE) {
            zstride = (size_t)X * Y;
            row = sm + ((size_t)(valid ? (uint32_t)y : 0u) * X + (uint32_t)xb);
            vec = valid == 0xFFu && (X & 7u) == 0u;
        }
    }
    __device__ __forceinline__ void operator()(int z, bool live, const uint32_t *s) {
        if (!live) return;
        const uint32_t vmax = max(max(max(s[0], s[1]), max(s[2], s[3])), max(max(s[4], s[5]), max(s[6], s[7])));
        // warp-uniform fast path: 8 voxels inside, aligned row, low levels only
        const bool fast = __all_sync(FULL, valid == 0xFFu && (!STORE || vec) && vmax < (uint32_t)HIST_LOW);
        if (fast) {
            if (STORE)
                *reinterpret_cast<uint4 *>(row + (size_t)(uint32_t)z * zstride) =
                    make_uint4(s[0] | (s[1] << 16), s[2] | (s[3] << 16), s[4] | (s[5] << 16), s[6] | (s[7] << 16));
            uint32_t *hc = sh + copy;
#pragma unroll
            for (int j = 0; j < 8; ++j) atomicAdd(hc + s[j], 1u);
            return;
        }
        if (STORE) {
            uint16_t *p = row + (size_t)(uint32_t)z * zstride;
            if (vec) {
                *reinterpret_cast<uint4 *>(p) =
                    make_uint4(s[0] | (s[1] << 16), s[2] | (s[3] << 16), s[4] | (s[5] << 16), s[6] | (s[7] << 16));
            } else {
#pragma unroll
                for (int j = 0; j < 8; ++j)
                    if (valid & (1u << j)) p[j] = (uint16_t)s[j];
            }
        }
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            if (valid & (1u << j)) {
                const uint32_t v = s[j];
                if (v < (uint32_t)HIST_LOW) {
                    atomicAdd(sh + copy + v, 1u);
                } else {
                    const uint32_t w = HIST_PAIRS + ((v - HIST_LOW) >> 1);
                    const uint32_t sft = (v & 1u) << 4;
                    const uint32_t old = atomicAdd(sh + w, 1u << sft);
                    if (((old >> sft) & 0xFFFFu) == 0x7FFFu) {
                        atomicSub(sh + w, 0x8000u << sft);
                        atomicAdd(gh + v, 0x8000u);
                    }
                }
            }
        }
    }
};

// ----------------------------------------------------------------------------
// Otsu (Segmentation section, ref. [11]) over a finished histogram
// ----------------------------------------------------------------------------
//
// var(t) = ((n0*n1) * d) * d with d = s1/n1 - s0/n0 in binary64, all
// operations explicitly rounded (no contraction).  Only levels t with
// h[t] > 0 are evaluated: for an empty level (n0, s0) repeat those of t - 1,
// so the value repeats and t can never be the lowest maximiser.  Ties go to
// the lowest t.  With no admissible t (one distinct level) t* is that level.
//
// Binary64 arithmetic is slow on this GPU (a division takes about 650
// cycles of latency, an add or compare 70 to 175), so the binary64 formula is
// evaluated only where it can decide the maximum.  A first pass bounds every
// occupied level's variance in binary32: each operand is converted within
// 2 ulp (2^-23 relative) and each quotient is correctly rounded, so a class
// mean is within 5 * 2^-24 relative, i.e. 0.02 voxel-value units for values
// below 65536; the difference d of the means is off by less than 0.05, and
// n0*n1 by less than 10^-6 relative; hence
//     lo = n0 n1 (1 - 1e-5) max(|d~| - 0.05, 0)^2 <= var <= hi = n0 n1 (1 + 1e-5) (|d~| + 0.05)^2,
// where var is the exact (rational) variance, and the binary64 value is
// within 10^-13 relative of it.  Every level whose hi is below the largest
// lo is below the maximum and cannot win or tie (two distinct binary32
// values differ by at least 2^-24 relative, far more than the binary64
// values can move); the binary64 formula is evaluated, in the stated order,
// at the remaining levels only.

template <int NT>
__device__ void otsu_block(const uint32_t *__restrict__ gh, uint32_t *stat, uint64_t nvox,
                           unsigned char *scr, uint32_t scr_bytes) {
    constexpr int NW = NT / 32;
    constexpr int GL = 128;               // levels per group (one 16-byte load per lane)
    constexpr int NG = HIST_BINS / GL;    // groups
    constexpr int GPW = NG / NW;          // groups per warp
    constexpr int LF = NT >= 1024 ? 4 : 8;   // group loads in flight per lane
    static_assert(GPW % LF == 0 && NG <= NT, "group layout");
    __shared__ unsigned long long g_n[NG], g_s[NG];  // group totals, then exclusive prefixes
    __shared__ uint32_t g_k[NG];                      // occupied levels per group, then prefix
    __shared__ uint16_t g_id[NG];                     // the occupied groups, in level order
    __shared__ unsigned long long w_n[32], w_s[32];
    __shared__ uint32_t w_k[32], w_g[32];
    __shared__ unsigned long long s_tot[2];
    __shared__ uint32_t s_ktot, s_gtot, s_cnt;
    __shared__ unsigned long long s_best;  // largest binary64 variance (bits)
    __shared__ uint32_t s_lvl, s_only, s_lb;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const uint4 *h4 = reinterpret_cast<const uint4 *>(gh);
    if (tid == 0) { s_cnt = 0; s_best = 0ull; s_lvl = 0xFFFFFFFFu; s_only = 0u; s_lb = 0u; }
    // 1. totals of every group of 128 levels: warp wid reads groups wid,
    // wid + NW, wid + 2 NW, ... (the occupied levels, low in the range,
    // spread over all warps), one coalesced 512-byte load per group
#pragma unroll 1
    for (int r = 0; r < GPW; r += LF) {
        uint4 c[LF];
#pragma unroll
        for (int k = 0; k < LF; ++k) c[k] = __ldcg(h4 + (size_t)((r + k) * NW + wid) * 32 + lane);
#pragma unroll
        for (int k = 0; k < LF; ++k) {
            const int g = (r + k) * NW + wid;
            const uint32_t u0 = (uint32_t)g * GL + 4u * (uint32_t)lane;
            unsigned long long n = (unsigned long long)c[k].x + c[k].y + c[k].z + c[k].w;
            if (!__any_sync(FULL, n != 0)) {
                if (lane == 0) { g_n[g] = 0; g_s[g] = 0; g_k[g] = 0; }
                continue;
            }
            unsigned long long s = (unsigned long long)u0 * n + c[k].y + 2ull * c[k].z + 3ull * c[k].w;
            uint32_t o = (c[k].x != 0) + (c[k].y != 0) + (c[k].z != 0) + (c[k].w != 0);
#pragma unroll 1
            for (int off = 16; off > 0; off >>= 1) {
                n += __shfl_xor_sync(FULL, n, off);
                s += __shfl_xor_sync(FULL, s, off);
                o += __shfl_xor_sync(FULL, o, off);
            }
            if (lane == 0) { g_n[g] = n; g_s[g] = s; g_k[g] = o; }
        }
    }
    __syncthreads();
    // 2. exclusive prefixes over the groups (thread g holds group g), the
    // totals, and the list of occupied groups
    {
        unsigned long long gn = 0, gs = 0;
        uint32_t gk = 0;
        if (tid < NG) { gn = g_n[tid]; gs = g_s[tid]; gk = g_k[tid]; }
        const uint32_t ne = gk != 0u;
        unsigned long long in = gn, is = gs;
        uint32_t ik = gk, ie = ne;
#pragma unroll 1
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long a = __shfl_up_sync(FULL, in, o), b = __shfl_up_sync(FULL, is, o);
            const uint32_t c = __shfl_up_sync(FULL, ik, o), d = __shfl_up_sync(FULL, ie, o);
            if (lane >= o) { in += a; is += b; ik += c; ie += d; }
        }
        if (lane == 31) { w_n[wid] = in; w_s[wid] = is; w_k[wid] = ik; w_g[wid] = ie; }
        __syncthreads();
        // every warp scans the warp totals itself (no further barrier): its
        // own exclusive prefix sits in lane wid, the grand totals in lane 31
        {
            const unsigned long long wn = lane < NW ? w_n[lane] : 0ull, ws = lane < NW ? w_s[lane] : 0ull;
            const uint32_t wk = lane < NW ? w_k[lane] : 0u, wg = lane < NW ? w_g[lane] : 0u;
            unsigned long long an = wn, as = ws;
            uint32_t ak = wk, ag = wg;
#pragma unroll 1
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned long long a = __shfl_up_sync(FULL, an, o), b = __shfl_up_sync(FULL, as, o);
                const uint32_t c = __shfl_up_sync(FULL, ak, o), d = __shfl_up_sync(FULL, ag, o);
                if (lane >= o) { an += a; as += b; ak += c; ag += d; }
            }
            const unsigned long long bn = __shfl_sync(FULL, an - wn, wid), bs = __shfl_sync(FULL, as - ws, wid);
            const uint32_t bk = __shfl_sync(FULL, ak - wk, wid), bg = __shfl_sync(FULL, ag - wg, wid);
            if (tid == 31) { s_tot[0] = an; s_tot[1] = as; s_ktot = ak; s_gtot = ag; }
            if (tid < NG) {
                g_n[tid] = bn + in - gn;
                g_s[tid] = bs + is - gs;
                g_k[tid] = bk + ik - gk;
                if (ne) g_id[bg + ie - 1u] = (uint16_t)tid;
            }
        }
        __syncthreads();
    }
    const unsigned long long Nt = s_tot[0], St = s_tot[1];
    const uint32_t K = s_ktot;  // occupied levels
    // binary32 bounds of the variance at level u (classes n0, s0 / n1, s1);
    // each operand converted from its two 32-bit halves (one rounding of
    // the high half, one of the fused sum: within 2 ulp)
    auto f32 = [](unsigned long long x) {
        const uint32_t hi32 = (uint32_t)(x >> 32), lo32 = (uint32_t)x;
        return hi32 ? __fmaf_rn(__uint2float_rn(hi32), 4294967296.0f, __uint2float_rn(lo32)) : __uint2float_rn(lo32);
    };
    auto bounds = [&](unsigned long long n0, unsigned long long s0, unsigned long long n1, float &lo, float &hi) {
        const float d = __fsub_rn(__fdiv_rn(f32(St - s0), f32(n1)), __fdiv_rn(f32(s0), f32(n0)));
        const float nn = __fmul_rn(f32(n0), f32(n1));
        const float e = fmaxf(fabsf(d) - 0.05f, 0.0f), f = fabsf(d) + 0.05f;
        lo = __fmul_rn(__fmul_rn(nn, 0.99999f), __fmul_rn(e, e));
        hi = __fmul_rn(__fmul_rn(nn, 1.00001f), __fmul_rn(f, f));
    };
    // The variance is never negative (n0 n1 d d with n0, n1 > 0, and d d is
    // +0 at worst), so the order of the binary64 values is the order of
    // their bit patterns read as unsigned integers; the running maximum is
    // kept as those bits, with level 0xFFFFFFFF for "none yet".
    unsigned long long best = 0ull;
    uint32_t bt = 0xFFFFFFFFu;
    auto eval = [&](uint32_t u, unsigned long long n0, unsigned long long s0) {
        const unsigned long long n1 = Nt - n0, s1 = St - s0;
        const double m0 = __ddiv_rn(__ull2double_rn(s0), __ull2double_rn(n0));
        const double m1 = __ddiv_rn(__ull2double_rn(s1), __ull2double_rn(n1));
        const double d = __dsub_rn(m1, m0);
        const double var = __dmul_rn(__dmul_rn(__dmul_rn(__ull2double_rn(n0), __ull2double_rn(n1)), d), d);
        const unsigned long long vb = (unsigned long long)__double_as_longlong(var);
        if (vb > best || (vb == best && u < bt)) { best = vb; bt = u; }
    };
    // largest of the threads' non-negative binary32 values (their bit
    // patterns order as unsigned integers)
    auto block_max = [&](float x) {
        const uint32_t m = __reduce_max_sync(FULL, __float_as_uint(x));
        if (lane == 0 && m) atomicMax(&s_lb, m);
        __syncthreads();
        return __uint_as_float(s_lb);
    };
    // The occupied levels (a frame's values span a few thousand of the 65536)
    // are listed in the scratch with their class prefixes (n0, s0), each
    // occupied group by one warp; every later step runs over the list, NT
    // entries at a time.
    const uint32_t lcap = (scr_bytes / 22u) & ~7u;
    if (K <= lcap) {
        unsigned long long *ln = reinterpret_cast<unsigned long long *>(scr), *ls = ln + lcap;
        float *lh = reinterpret_cast<float *>(ls + lcap);
        uint16_t *lu = reinterpret_cast<uint16_t *>(lh + lcap);
        const uint32_t ng = s_gtot;
#pragma unroll 1
        for (uint32_t q = (uint32_t)wid; q < ng; q += NW) {
            const uint32_t g = g_id[q];
            const uint4 c = __ldcg(h4 + (size_t)g * 32 + lane);
            const uint32_t u0 = g * GL + 4u * (uint32_t)lane;
            const unsigned long long n = (unsigned long long)c.x + c.y + c.z + c.w;
            const unsigned long long s = (unsigned long long)u0 * n + c.y + 2ull * c.z + 3ull * c.w;
            const uint32_t o = (c.x != 0) + (c.y != 0) + (c.z != 0) + (c.w != 0);
            unsigned long long in = n, is = s;
            uint32_t io = o;
#pragma unroll 1
            for (int off = 1; off < 32; off <<= 1) {
                const unsigned long long a = __shfl_up_sync(FULL, in, off), b = __shfl_up_sync(FULL, is, off);
                const uint32_t d = __shfl_up_sync(FULL, io, off);
                if (lane >= off) { in += a; is += b; io += d; }
            }
            unsigned long long n0 = g_n[g] + in - n, s0 = g_s[g] + is - s;
            uint32_t k = g_k[g] + io - o;
            const uint32_t cs[4] = {c.x, c.y, c.z, c.w};
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                if (!cs[j]) continue;
                n0 += cs[j];
                s0 += (unsigned long long)(u0 + j) * cs[j];
                ln[k] = n0;
                ls[k] = s0;
                lu[k] = (uint16_t)(u0 + j);
                ++k;
            }
        }
        __syncthreads();
        if (tid == 0 && K == 1) s_only = lu[0];
        // bounds of every listed level, the largest lower bound
        float lo_max = 0.0f;
#pragma unroll 1
        for (uint32_t k = (uint32_t)tid; k < K; k += NT) {
            const unsigned long long n0 = ln[k];
            float lo = 0.0f, hi = -1.0f;  // the top level (empty upper class) is no candidate
            if (Nt - n0 != 0) bounds(n0, ls[k], Nt - n0, lo, hi);
            lh[k] = hi;
            lo_max = fmaxf(lo_max, lo);
        }
        const float LB = block_max(lo_max);
        // binary64 at the levels whose upper bound reaches LB
#pragma unroll 1
        for (uint32_t k = (uint32_t)tid; k < K; k += NT)
            if (lh[k] >= LB) eval(lu[k], ln[k], ls[k]);
    } else {
        // More occupied levels than the list holds: each thread takes PER
        // consecutive levels; its class prefixes start from its group's
        // prefix plus the sums of the group's levels below its own.
        constexpr int PER = HIST_BINS / NT;
        static_assert(GL % PER == 0, "whole threads per group");
        const uint32_t base = (uint32_t)tid * PER, g = base / GL;
        unsigned long long n0b = g_n[g], s0b = g_s[g];
        if (base % GL) {
#pragma unroll 4
            for (uint32_t q = g * (GL / 4); q < base / 4; ++q) {
                const uint4 c = __ldcg(h4 + q);
                const unsigned long long n = (unsigned long long)c.x + c.y + c.z + c.w;
                n0b += n;
                s0b += (unsigned long long)(4u * q) * n + c.y + 2ull * c.z + 3ull * c.w;
            }
        }
        // the thread's levels, four per load, the next load in flight
        auto sweep = [&](auto &&level) {
            uint4 nx = __ldcg(h4 + base / 4);
#pragma unroll 1
            for (uint32_t q = 0; q < PER / 4; ++q) {
                const uint4 c = nx;
                if (q + 1 < PER / 4) nx = __ldcg(h4 + base / 4 + q + 1);
                const uint32_t cs[4] = {c.x, c.y, c.z, c.w};
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    if (cs[j]) level(base + 4u * q + (uint32_t)j, cs[j]);
            }
        };
        float lo_max = 0.0f;
        {
            unsigned long long n0 = n0b, s0 = s0b;
            sweep([&](uint32_t u, uint32_t c) {
                n0 += c;
                s0 += (unsigned long long)u * c;
                if (Nt - n0 == 0) return;
                float lo, hi;
                bounds(n0, s0, Nt - n0, lo, hi);
                lo_max = fmaxf(lo_max, lo);
            });
        }
        const float LB = block_max(lo_max);
        // the levels whose upper bound reaches LB go to a list in the
        // scratch, so that all threads share their binary64 evaluations
        const uint32_t cap = scr_bytes / 20u;
        unsigned long long *cn = reinterpret_cast<unsigned long long *>(scr), *cs = cn + cap;
        uint32_t *cu = reinterpret_cast<uint32_t *>(cs + cap);
        {
            unsigned long long n0 = n0b, s0 = s0b;
            sweep([&](uint32_t u, uint32_t c) {
                n0 += c;
                s0 += (unsigned long long)u * c;
                if (Nt - n0 == 0) return;
                float lo, hi;
                bounds(n0, s0, Nt - n0, lo, hi);
                if (hi < LB) return;  // below the maximum
                const uint32_t k = atomicAdd(&s_cnt, 1u);
                if (k < cap) {
                    cu[k] = u;
                    cn[k] = n0;
                    cs[k] = s0;
                }
            });
        }
        __syncthreads();
        const uint32_t nc = s_cnt;
        if (nc <= cap) {
#pragma unroll 1
            for (uint32_t k = (uint32_t)tid; k < nc; k += NT) eval(cu[k], cn[k], cs[k]);
        } else {
            // more candidates than the scratch holds: each thread its own
            unsigned long long n0 = n0b, s0 = s0b;
            sweep([&](uint32_t u, uint32_t c) {
                n0 += c;
                s0 += (unsigned long long)u * c;
                if (Nt - n0 == 0) return;
                float lo, hi;
                bounds(n0, s0, Nt - n0, lo, hi);
                if (hi >= LB) eval(u, n0, s0);
            });
        }
    }
    // the largest variance, then the lowest level that reaches it.  With two
    // or more occupied levels some level survives the pruning (the one whose
    // lower bound is LB); with one, t* is that level, with none 0.
    if (bt != 0xFFFFFFFFu) atomicMax(&s_best, best);
    __syncthreads();
    if (bt != 0xFFFFFFFFu && best == s_best) atomicMin(&s_lvl, bt);
    __syncthreads();
    if (tid == 0) {
        stat[ST_THRESH] = s_lvl != 0xFFFFFFFFu ? s_lvl : s_only;
        if (Nt != nvox) atomicOr(stat + ST_ERROR, ERR_OTSU);
    }
    __syncthreads();
}

// Merge the block's shared histogram into the volume's bins (and leave it
// zero for the block's next volume).
template <int NT>
__device__ void flush_hist(const VolDev &V, uint32_t *sh) {
    __syncthreads();
    for (int i = threadIdx.x; i < HIST_LOW / 4; i += NT) {
        uint4 a = reinterpret_cast<uint4 *>(sh)[i];
        uint4 b = reinterpret_cast<uint4 *>(sh + HIST_COPY1)[i];
        a.x += b.x; a.y += b.y; a.z += b.z; a.w += b.w;
        if (a.x | a.y | a.z | a.w) {
            reinterpret_cast<uint4 *>(sh)[i] = make_uint4(0, 0, 0, 0);
            reinterpret_cast<uint4 *>(sh + HIST_COPY1)[i] = make_uint4(0, 0, 0, 0);
            const uint32_t ws[4] = {a.x, a.y, a.z, a.w};
#pragma unroll
            for (int j = 0; j < 4; ++j)
                if (ws[j]) atomicAdd(V.hist + 4u * i + j, ws[j]);
        }
    }
    for (int i = threadIdx.x; i < (HIST_WORDS - HIST_PAIRS) / 4; i += NT) {
        uint4 w = reinterpret_cast<uint4 *>(sh + HIST_PAIRS)[i];
        if (w.x | w.y | w.z | w.w) {
            reinterpret_cast<uint4 *>(sh + HIST_PAIRS)[i] = make_uint4(0, 0, 0, 0);
            const uint32_t ws[4] = {w.x, w.y, w.z, w.w};
            const uint32_t b = HIST_LOW + 8u * (uint32_t)i;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                if (ws[j] & 0xFFFFu) atomicAdd(V.hist + b + 2 * j, ws[j] & 0xFFFFu);
                if (ws[j] >> 16) atomicAdd(V.hist + b + 2 * j + 1, ws[j] >> 16);
            }
        }
    }
    __syncthreads();
}

// Otsu level of every volume of a batch (Segmentation section, ref. [11]:
// the level that maximises the between-class variance of the smoothed
// volume's histogram), one block per volume, after all smoothing tiles have
// merged their bins.  The dynamic shared memory holds the list of occupied
// levels.
constexpr int OTSU_NT = 512;
constexpr uint32_t OTSU_SMEM = 192u * 1024u;

__global__ void __launch_bounds__(OTSU_NT, 1) k_otsu(const BatchHdr *__restrict__ h) {
    extern __shared__ __align__(16) unsigned char oscr[];
    const uint32_t nv = h->nvol;
#pragma unroll 1
    for (uint32_t v = blockIdx.x; v < nv; v += gridDim.x) {
        const VolDev &V = h->vol[v];
        otsu_block<OTSU_NT>(V.hist, V.stat, (uint64_t)V.X * V.Y * V.Z, oscr, OTSU_SMEM);
    }
}

// The same for one volume given by its bins and status words.
__global__ void __launch_bounds__(OTSU_NT, 1) k_otsu_one(const uint32_t *__restrict__ hist, uint32_t *stat,
                                                         uint64_t nvox) {
    extern __shared__ __align__(16) unsigned char oscr[];
    otsu_block<OTSU_NT>(hist, stat, nvox, oscr, OTSU_SMEM);
}

// ----------------------------------------------------------------------------
// kernels
// ----------------------------------------------------------------------------

__global__ void k_init(const BatchHdr *__restrict__ h) {
    const uint32_t per = HIST_BINS / 4;
    const uint64_t total = (uint64_t)h->nvol * per;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t v = (uint32_t)(i / per), j = (uint32_t)(i % per);
        reinterpret_cast<uint4 *>(h->vol[v].hist)[j] = make_uint4(0, 0, 0, 0);
        if (j < ST_WORDS / 4) reinterpret_cast<uint4 *>(h->vol[v].stat)[j] = make_uint4(0, 0, 0, 0);
        if (j < 2048 / 4 && h->vol[v].mrf_bits)
            reinterpret_cast<uint4 *>(h->vol[v].mrf_bits)[j] = make_uint4(0, 0, 0, 0);
    }
}

template <int TY>
__global__ void __launch_bounds__(8 * TY, 1) k_smooth_hist(const BatchHdr *__restrict__ h) {
    using T = Tile<TY>;
    extern __shared__ __align__(128) unsigned char dsm[];
    unsigned char *ring = dsm;
    uint32_t *sh = reinterpret_cast<uint32_t *>(dsm + T::RING_BYTES);
    uint32_t *spx = sh + HIST_WORDS;
    int8_t *shift = reinterpret_cast<int8_t *>(spx + 2 * T::PX_WORDS);
    Ring R{ring, shift, 0};
    for (int i = threadIdx.x; i < HIST_WORDS / 4; i += T::NT)
        reinterpret_cast<uint4 *>(sh)[i] = make_uint4(0, 0, 0, 0);
    __syncthreads();
    const uint32_t nt = h->ntiles, G = gridDim.x;
    const uint32_t tb = (uint32_t)(((uint64_t)nt * blockIdx.x) / G);
    const uint32_t te = (uint32_t)(((uint64_t)nt * (blockIdx.x + 1)) / G);
    if (tb >= te) return;
    uint32_t v = find_vol_tile(h, tb);
    const int tz = (int)h->tile_z;
    for (uint32_t t = tb; t < te; ++t) {
        while (v + 1 < h->nvol && t >= h->vol[v + 1].tile_base) {
            flush_hist<T::NT>(h->vol[v], sh);
            ++v;
        }
        const VolDev &V = h->vol[v];
        const uint32_t tl = t - V.tile_base;
        const uint32_t ix = tl % V.ntx, rest = tl / V.ntx;
        const uint32_t iy = rest % V.nty, iz = rest / V.nty;
        const int z0 = (int)iz * tz;
        const int z1 = min(z0 + tz, (int)V.Z);
        HistEmit<true> e{sh, V.hist, V.smooth, V.X, V.Y, 0u, 0u, nullptr, 0, false};
        smooth_tile<TY>(V.raw, V.X, V.Y, V.Z, (int)ix * TILE_X, (int)iy * TY, z0, z1, spx, R, e);
    }
    flush_hist<T::NT>(h->vol[v], sh);
}

// ----------------------------------------------------------------------------
// Smoothing + histogram of volumes whose rows are 16-byte aligned
// (X % 8 == 0, 16-byte aligned input): k_smooth_rows
// ----------------------------------------------------------------------------
//
// The same arithmetic as smooth_tile (binomial [1 4 6 4 1] per axis, exact
// uint32 sums, one rounding (S + 2048) >> 12, replicate edges), arranged so
// that every warp works on its own:
//   y pass first, on the raw voxels as staged: a lane reads its octet of the
//     five rows around its own (five 16-byte loads) and sums the packed
//     16-bit pairs of each word at once; when every raw value is below 4096
//     no lane of a word can exceed 16 * 4095 = 65520, so the packed sum is
//     exact.  Each lane checks the words it reads; a warp in which one of
//     them is 4096 or more redoes that plane's y pass in 32-bit lanes.
//   x pass in registers: the y-sums left and right of a lane's octet come
//     from the neighbouring lanes by shuffles; a lane at the end of a warp
//     y-sums the neighbouring word itself from the staged plane (also the
//     halo chunks of x-tiled rows), and at the volume's x-edges the edge
//     voxel is repeated.
//   z pass in registers (scatter form, four running sums per output), with
//     the rounding constant carried in the newest running sum.
// A tile is FS_RT octets (512 voxels) wide, or the whole row when X <= 512,
// and FS_NT / octets-per-row rows high; it marches down z through a ring of
// FS_S staged planes filled with 16-byte cp.async copies by all threads.
// The ring is driven by mbarriers instead of block barriers: a stage's
// "full" barrier completes when every thread's copies of its plane have
// landed (cp.async.mbarrier.arrive), its "empty" barrier when every warp has
// read it, and a thread refills a stage only after the plane two behind its
// own is empty (five stages, three planes staged ahead), so warps drift up
// to two planes apart.  Every wait is bounded:
// a wait that runs out raises ERR_TIMEOUT for the volume and puts the block
// in a mode that skips the remaining work but still reaches every block
// barrier.  Consecutive tiles of a block are y-neighbours, so the rows two of
// them share are fetched again while still in L2.

constexpr int FS_S = 5;                  // ring stages
constexpr int FS_LEAD = 3;               // planes staged ahead of the one being read
// a thread refills the stage of plane k - (FS_S - FS_LEAD) while reading
// plane k: warps may drift FS_S - FS_LEAD planes apart
constexpr int FS_STAGE = 12 * 66 * 16;   // bytes per stage: 12 rows x 66 chunks (x-tiled) bound all shapes
constexpr int FS_WARPS = FS_NT / 32;
constexpr uint32_t FS_WAIT_LIMIT = 1u << 23;  // mbarrier polls (each suspends <= ~256 ns) before a wait gives up
constexpr size_t FS_SMEM = 4ull * HIST_WORDS + (size_t)FS_S * FS_STAGE + 16ull * 2 * FS_S + 16;
static_assert((8 * FS_RT / FS_RT + 4) * (FS_RT + 2) * 16 <= FS_STAGE, "x-tiled stage");
static_assert((FS_NT / FS_RT + 4) * FS_RT * 16 <= FS_STAGE && (FS_NT + 4) * 16 <= FS_STAGE, "stage bound");

__device__ __forceinline__ uint32_t find_vol_fs(const BatchHdr *__restrict__ h, uint32_t t) {
    uint32_t lo = 0, hi = h->nvol;
    while (hi - lo > 1) {
        uint32_t mid = (lo + hi) >> 1;
        if (h->vol[mid].fs_base <= t) lo = mid; else hi = mid;
    }
    return lo;
}

__device__ __forceinline__ uint32_t fs_ysum(uint32_t r0, uint32_t r1, uint32_t r2, uint32_t r3, uint32_t r4) {
    return r0 + r4 + 4u * (r1 + r3) + 6u * r2;
}

// y-sums (32-bit) of the low and high voxel of five staged words
__device__ __forceinline__ void fs_ysum32(uint32_t r0, uint32_t r1, uint32_t r2, uint32_t r3, uint32_t r4,
                                          uint32_t &lo, uint32_t &hi) {
    lo = fs_ysum(r0 & 0xFFFFu, r1 & 0xFFFFu, r2 & 0xFFFFu, r3 & 0xFFFFu, r4 & 0xFFFFu);
    hi = fs_ysum(r0 >> 16, r1 >> 16, r2 >> 16, r3 >> 16, r4 >> 16);
}

// ---- mbarriers ------------------------------------------------------------

__device__ __forceinline__ void mbar_init(uint64_t *b, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *b) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(b)) : "memory");
}
// arrives on b once all of this thread's earlier cp.async copies have landed
__device__ __forceinline__ void mbar_arrive_copies(uint64_t *b) {
    asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(smem_addr(b)) : "memory");
}
// non-blocking test of the given phase
__device__ __forceinline__ bool mbar_test(uint64_t *b, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(smem_addr(b)), "r"(parity)
        : "memory");
    return ok != 0;
}
// waits for the phase, suspending the thread for at most about 256 ns
__device__ __forceinline__ bool mbar_try(uint64_t *b, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(smem_addr(b)), "r"(parity), "r"(256u)
        : "memory");
    return ok != 0;
}

// Polls b until the given phase completes: false once the block has
// aborted, or when FS_WAIT_LIMIT polls have passed (then the block is
// aborted and the volume flagged).
__device__ __noinline__ bool fs_wait_slow(uint64_t *b, uint32_t parity, volatile uint32_t *abort, uint32_t *stat) {
    for (uint32_t i = 0; !mbar_try(b, parity); ++i) {
        if ((i & 63u) == 0u && *abort) return false;
        if (i >= FS_WAIT_LIMIT) {
            *abort = 1u;
            atomicOr(stat + ST_ERROR, ERR_TIMEOUT);
            return false;
        }
    }
    return true;
}

// The ring's synchronisation state of one block.
struct FsSync {
    uint64_t *full;           // FS_S barriers: the stage's plane has landed
    uint64_t *empty;          // FS_S barriers: every warp has read the stage
    volatile uint32_t *abort; // set when a wait ran out
    uint32_t g;               // planes this block has run through the ring
    __device__ __forceinline__ bool wait(uint64_t *b, uint32_t parity, uint32_t *stat) {
        return mbar_test(b, parity) || fs_wait_slow(b, parity, abort, stat);
    }
};

// One tile: octets [x0, x0 + 8 rte) of rows [y0, y0 + TYF) of planes [z0, z1).
// RTC = FS_RT: rows of 64 octets (8 rows per tile), HXC: halo chunks
// (x-tiled rows), both known at compile time; RTC = 0: the shape of V.
template <int RTC, int HXC, int RAG>
__device__ __forceinline__ void smooth_rows_tile(const VolDev &V, uint32_t ix, uint32_t iy, int z0, int z1,
                                                 unsigned char *ring, uint32_t *sh, FsSync &S) {
    const int tid = threadIdx.x, lane = tid & 31;
    const int X = (int)V.X, Y = (int)V.Y, Z = (int)V.Z;
    // the descriptor's fields in registers (the barrier operations below are
    // memory clobbers, which would reload them from global memory)
    const uint16_t *raw = V.raw;
    uint16_t *osm = V.smooth;
    uint32_t *stat = V.stat, *ghist = V.hist;
    uint16_t *wmax = V.wmax;
    const uint32_t W = V.W;
    const int RT = RTC ? RTC : (int)V.fs_rt;
    const int TYF = RTC ? FS_NT / RTC : (int)V.fs_ty;
    const int hx = RTC ? HXC : (int)V.fs_hx;
    const int RC = RT + 2 * hx;   // 16-byte chunks per staged row
    const int RB = 16 * RC;       // bytes per staged row
    const int x0 = (int)ix * 8 * RT, y0 = (int)iy * TYF;
    // octets of this tile; rows of X % 8 != 0 voxels (RAG) end in a partial
    // octet of nvl voxels (X even: 2, 4 or 6), whose missing voxels repeat
    // the last one in the x pass and are neither stored nor counted
    const int rte = RAG ? min(RT, (X - x0 + 7) >> 3) : min(RT, (X - x0) >> 3);
    const int q = RTC ? (tid & (RTC - 1)) : tid % RT;
    const int ty = RTC ? tid / RTC : tid / RT;
    const bool act = ty < TYF && q < rte;
    const int tyc = ty < TYF ? ty : 0;       // threads past the tile read a valid row
    const bool emit_ok = act && y0 + ty < Y;
    const bool haloL = x0 > 0, haloR = x0 + 8 * rte < X;
    const bool edgeL = q == 0, edgeR = q == rte - 1;
    const int nvl = RAG && edgeR ? min(8, X - (x0 + 8 * q)) : 8;  // valid voxels of this lane's octet
    // neighbour words this lane y-sums itself: at a warp's ends and at the
    // tile's ends of x-tiled rows (the halo chunks)
    const bool ownL = edgeL ? haloL : lane == 0;
    const bool ownR = edgeR ? haloR : lane == 31;
    const int colo = tyc * RB + (hx + q) * 16;                     // this lane's octet in a staged plane
    const int fixo = ownL ? colo - 4 : colo + 16;                  // the word it y-sums, if any
    // this thread's copy chunks (at most two per plane): staged row r, chunk
    // cc, as 32-bit voxel offsets from the volume's start at plane 0
    const int nchunk = (TYF + 4) * RC;
    uint32_t cdst[2], csrc[2];
    int cend[2];  // voxels of the chunk before the row's end (RAG)
    bool cok[2];
#pragma unroll
    for (int u = 0; u < 2; ++u) {
        const int c = tid + u * FS_NT;
        cok[u] = false;
        cdst[u] = 0;
        csrc[u] = 0;
        cend[u] = 0;
        if (c < nchunk) {
            const int r = c / RC, cc = c - r * RC;
            const int x = x0 - 8 * hx + 8 * cc;
            cok[u] = x >= 0 && x < X;
            cend[u] = X - x;
            const int yy = min(max(y0 - 2 + r, 0), Y - 1);
            cdst[u] = (uint32_t)(r * RB + cc * 16);
            csrc[u] = (uint32_t)yy * (uint32_t)X + (uint32_t)x;
        }
    }
    const uint32_t plane = (uint32_t)X * (uint32_t)Y;  // < 2^32 (X Y Z < 2^32)
    const int n = z1 - z0 + 4;
    const uint32_t ring0 = smem_addr(ring);
    // Tiles run through the ring in whole rounds of FS_S planes (a tile's
    // planes padded with planes that only keep the barriers' phases in step),
    // so that the stage of every plane is a compile-time constant; `par` is
    // the phase parity of the current round.
    const uint32_t g0 = S.g;                   // a multiple of FS_S
    const int npad = (n + FS_S - 1) / FS_S * FS_S;
    // tile plane k into stage ST (full phase fp), once every warp has read
    // the plane that stage held before (empty phase fp ^ 1, if there was one)
    auto issue = [&](int k, auto stc, uint32_t fp) {
        constexpr uint32_t ST = decltype(stc)::value;
        const bool ok = g0 + (uint32_t)k < (uint32_t)FS_S || S.wait(S.empty + ST, fp ^ 1u, stat);
        if (ok && k < n) {
            const uint32_t zoff = plane * (uint32_t)min(max(z0 - 2 + k, 0), Z - 1);
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                if (!cok[u]) continue;
                if (!RAG) {
                    cp_async16(ring0 + ST * FS_STAGE + cdst[u], reinterpret_cast<uintptr_t>(raw + (csrc[u] + zoff)));
                } else {
                    // rows start 4-byte aligned only: four pairs, those at
                    // or past the row's end zero-filled
#pragma unroll
                    for (int pq = 0; pq < 4; ++pq) {
                        const bool in = 2 * pq < cend[u];
                        cp_async4(ring0 + ST * FS_STAGE + cdst[u] + 4 * pq,
                                  reinterpret_cast<uintptr_t>(in ? raw + (csrc[u] + zoff + 2 * pq) : raw), in ? 4u : 0u);
                    }
                }
            }
        }
        mbar_arrive_copies(S.full + ST);
    };
    // x-sums of the last planes, plane k in slot k % 5 (the ring stage, a
    // compile-time index in every step)
    uint32_t pr[FS_S][8];
#pragma unroll
    for (int i = 0; i < FS_S; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) pr[i][j] = 0u;
    const uint32_t orow = (uint32_t)(y0 + tyc) * (uint32_t)X + (uint32_t)(x0 + 8 * q);
    uint32_t *hc = sh + ((threadIdx.x & 16u) ? (uint32_t)HIST_COPY1 : 0u);
    // plane k from stage ST (full phase fp): nothing but the barriers for
    // the padding planes k >= n
    auto step = [&](int k, auto stc, uint32_t fp) {
        constexpr uint32_t ST = decltype(stc)::value;
        const bool ok = S.wait(S.full + ST, fp, stat);
        // a warp whose wait gave up skips the work (the block stays in step
        // for its block barriers); warp-uniform, so that the shuffles below
        // see every lane
        if (!__all_sync(FULL, ok)) return;
        if (k >= n) {
            __syncwarp();
            if (lane == 0) mbar_arrive(S.empty + ST);
            return;
        }
            const unsigned char *stg = ring + ST * FS_STAGE;
            // y pass on packed pairs
            const unsigned char *cp = stg + colo;
            const uint4 r0 = *reinterpret_cast<const uint4 *>(cp);
            const uint4 r1 = *reinterpret_cast<const uint4 *>(cp + RB);
            const uint4 r2 = *reinterpret_cast<const uint4 *>(cp + 2 * RB);
            const uint4 r3 = *reinterpret_cast<const uint4 *>(cp + 3 * RB);
            const uint4 r4 = *reinterpret_cast<const uint4 *>(cp + 4 * RB);
            uint32_t yw[4];
            yw[0] = fs_ysum(r0.x, r1.x, r2.x, r3.x, r4.x);
            yw[1] = fs_ysum(r0.y, r1.y, r2.y, r3.y, r4.y);
            yw[2] = fs_ysum(r0.z, r1.z, r2.z, r3.z, r4.z);
            yw[3] = fs_ysum(r0.w, r1.w, r2.w, r3.w, r4.w);
            uint32_t chk = (r0.x | r0.y | r0.z | r0.w | r1.x | r1.y | r1.z | r1.w | r2.x | r2.y) |
                           (r2.z | r2.w | r3.x | r3.y | r3.z | r3.w | r4.x | r4.y | r4.z | r4.w);
            uint32_t hw = 0u;  // packed y-sum of the neighbour word this lane reads itself
            if (ownL || ownR) {
                const unsigned char *hp = stg + fixo;
                const uint32_t w0 = *reinterpret_cast<const uint32_t *>(hp);
                const uint32_t w1 = *reinterpret_cast<const uint32_t *>(hp + RB);
                const uint32_t w2 = *reinterpret_cast<const uint32_t *>(hp + 2 * RB);
                const uint32_t w3 = *reinterpret_cast<const uint32_t *>(hp + 3 * RB);
                const uint32_t w4 = *reinterpret_cast<const uint32_t *>(hp + 4 * RB);
                hw = fs_ysum(w0, w1, w2, w3, w4);
                chk |= w0 | w1 | w2 | w3 | w4;
            }
            const uint32_t nl = __shfl_up_sync(FULL, yw[3], 1);
            const uint32_t nr = __shfl_down_sync(FULL, yw[0], 1);
            uint32_t v[12];
            if (!__any_sync(FULL, act && (chk & 0xF000F000u) != 0u)) {
                const uint32_t wl = ownL ? hw : (edgeL ? __byte_perm(yw[0], 0u, 0x1010u) : nl);
                const uint32_t wr = ownR ? hw : (edgeR ? __byte_perm(yw[3], 0u, 0x3232u) : nr);
                v[0] = wl & 0xFFFFu;
                v[1] = wl >> 16;
    #pragma unroll
                for (int i = 0; i < 4; ++i) {
                    v[2 + 2 * i] = yw[i] & 0xFFFFu;
                    v[3 + 2 * i] = yw[i] >> 16;
                }
                v[10] = wr & 0xFFFFu;
                v[11] = wr >> 16;
            } else {
                // a raw value of 4096 or more in this warp's part of the plane:
                // its y pass again, in 32-bit lanes
    #pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const unsigned char *wp = cp + 4 * i;
                    fs_ysum32(*reinterpret_cast<const uint32_t *>(wp), *reinterpret_cast<const uint32_t *>(wp + RB),
                              *reinterpret_cast<const uint32_t *>(wp + 2 * RB),
                              *reinterpret_cast<const uint32_t *>(wp + 3 * RB),
                              *reinterpret_cast<const uint32_t *>(wp + 4 * RB), v[2 + 2 * i], v[3 + 2 * i]);
                }
                uint32_t hlo = 0u, hhi = 0u;
                if (ownL || ownR) {
                    const unsigned char *hp = stg + fixo;
                    fs_ysum32(*reinterpret_cast<const uint32_t *>(hp), *reinterpret_cast<const uint32_t *>(hp + RB),
                              *reinterpret_cast<const uint32_t *>(hp + 2 * RB),
                              *reinterpret_cast<const uint32_t *>(hp + 3 * RB),
                              *reinterpret_cast<const uint32_t *>(hp + 4 * RB), hlo, hhi);
                }
                const uint32_t l0 = __shfl_up_sync(FULL, v[8], 1), l1 = __shfl_up_sync(FULL, v[9], 1);
                const uint32_t q0 = __shfl_down_sync(FULL, v[2], 1), q1 = __shfl_down_sync(FULL, v[3], 1);
                v[0] = ownL ? hlo : (edgeL ? v[2] : l0);
                v[1] = ownL ? hhi : (edgeL ? v[2] : l1);
                v[10] = ownR ? hlo : (edgeR ? v[9] : q0);
                v[11] = ownR ? hhi : (edgeR ? v[9] : q1);
            }
            if (RAG && nvl < 8) {
                // the row's last octet is partial (nvl = 2, 4 or 6 for even
                // X): the voxels past the end repeat the last one
                const uint32_t e = nvl <= 2 ? v[3] : (nvl <= 4 ? v[5] : v[7]);
#pragma unroll
                for (int k = 4; k < 12; ++k)
                    if (k >= 2 + nvl) v[k] = e;
            }
            // this warp is done with the stage
            __syncwarp();
            if (lane == 0) mbar_arrive(S.empty + ST);
            // x pass, then the z pass over planes k-4 .. k in gather form; the
            // 2048 enters with the outer pair so that s = sum >> 12 rounds
            // half up
            uint32_t s[8];
    #pragma unroll
            for (int j = 0; j < 8; ++j) {
                const uint32_t p = v[j] + v[j + 4] + 4u * (v[j + 1] + v[j + 3]) + 6u * v[j + 2];
                const uint32_t A = pr[(ST + 1) % FS_S][j], B = pr[(ST + 2) % FS_S][j];
                const uint32_t C = pr[(ST + 3) % FS_S][j], D = pr[(ST + 4) % FS_S][j];
                s[j] = (A + p + 2048u + 4u * (B + D) + 6u * C) >> 12;
                pr[ST][j] = p;
            }
            if (k >= 4) {
                if (RAG) {
#pragma unroll
                    for (int j = 2; j < 8; ++j)
                        if (j >= nvl) s[j] = 0u;  // not emitted (and below any t*)
                }
                const uint32_t vmax = max(max(max(s[0], s[1]), max(s[2], s[3])), max(max(s[4], s[5]), max(s[6], s[7])));
                const bool fast = __all_sync(FULL, !emit_ok || vmax < (uint32_t)HIST_LOW);
                if (wmax) {
                    // the largest value of each 32-voxel mask word (four lanes),
                    // so that the threshold pass reads only words above t*
                    uint32_t wm = emit_ok ? vmax : 0u;
                    wm = max(wm, __shfl_xor_sync(FULL, wm, 1));
                    wm = max(wm, __shfl_xor_sync(FULL, wm, 2));
                    if (emit_ok && (q & 3) == 0)
                        wmax[(uint32_t)((z0 + k - 4) * Y + y0 + ty) * W + (uint32_t)((x0 + 8 * q) >> 5)] = (uint16_t)wm;
                }
                if (emit_ok) {
                    uint16_t *op = osm + (orow + plane * (uint32_t)(z0 + k - 4));
                    if (!RAG) {
                        *reinterpret_cast<uint4 *>(op) =
                            make_uint4(s[0] | (s[1] << 16), s[2] | (s[3] << 16), s[4] | (s[5] << 16), s[6] | (s[7] << 16));
                    } else {
                        // rows start 4-byte aligned only; the pairs past the end stay unwritten
#pragma unroll
                        for (int j = 0; j < 8; j += 2)
                            if (j < nvl) *reinterpret_cast<uint32_t *>(op + j) = s[j] | (s[j + 1] << 16);
                    }
                    if (fast) {
    #pragma unroll
                        for (int j = 0; j < 8; ++j)
                            if (!RAG || j < nvl) atomicAdd(hc + s[j], 1u);
                    } else {
    #pragma unroll
                        for (int j = 0; j < 8; ++j) {
                            if (RAG && j >= nvl) continue;
                            const uint32_t u = min(s[j], 65535u);  // (always true for exact sums)
                            if (u < (uint32_t)HIST_LOW) {
                                atomicAdd(hc + u, 1u);
                            } else {
                                const uint32_t w = HIST_PAIRS + ((u - HIST_LOW) >> 1);
                                const uint32_t sft = (u & 1u) << 4;
                                const uint32_t old = atomicAdd(sh + w, 1u << sft);
                                if (((old >> sft) & 0xFFFFu) == 0x7FFFu) {
                                    atomicSub(sh + w, 0x8000u << sft);
                                    atomicAdd(ghist + u, 0x8000u);
                                }
                            }
                        }
                    }
                }
            }
    };
    using C0 = std::integral_constant<uint32_t, 0>;
    using C1 = std::integral_constant<uint32_t, 1>;
    using C2 = std::integral_constant<uint32_t, 2>;
    using C3 = std::integral_constant<uint32_t, 3>;
    using C4 = std::integral_constant<uint32_t, 4>;
    static_assert(FS_S == 5 && FS_LEAD == 3, "the round below stages three planes ahead in a ring of five");
    uint32_t par = (g0 / FS_S) & 1u;
    issue(0, C0(), par);
    issue(1, C1(), par);
    issue(2, C2(), par);
    for (int k0 = 0; k0 < npad; k0 += FS_S) {
        if (k0 + 3 < npad) issue(k0 + 3, C3(), par);
        step(k0, C0(), par);
        if (k0 + 4 < npad) issue(k0 + 4, C4(), par);
        step(k0 + 1, C1(), par);
        if (k0 + 5 < npad) issue(k0 + 5, C0(), par ^ 1u);
        step(k0 + 2, C2(), par);
        if (k0 + 6 < npad) issue(k0 + 6, C1(), par ^ 1u);
        step(k0 + 3, C3(), par);
        if (k0 + 7 < npad) issue(k0 + 7, C2(), par ^ 1u);
        step(k0 + 4, C4(), par);
        par ^= 1u;
    }
    S.g = g0 + (uint32_t)npad;
}

constexpr uint32_t FS_GROUP = 4;

__global__ void __launch_bounds__(FS_NT, 1) k_smooth_rows(const BatchHdr *__restrict__ h) {
    extern __shared__ __align__(128) unsigned char dsm[];
    uint32_t *sh = reinterpret_cast<uint32_t *>(dsm);
    unsigned char *ring = dsm + 4 * HIST_WORDS;
    uint64_t *bars = reinterpret_cast<uint64_t *>(ring + FS_S * FS_STAGE);
    // Groups of FS_GROUP consecutive blocks share a contiguous range of
    // tiles and take its tiles in turn, so that y-adjacent tiles of a volume
    // are smoothed at the same time and the rows one stages as halo are
    // still in L2 when its neighbour stages them as its own.
    const uint32_t nt = h->fs_tiles, G = gridDim.x;
    const uint32_t gs = G % FS_GROUP == 0 ? FS_GROUP : 1u;
    const uint32_t nq = G / gs, q = blockIdx.x / gs, m = blockIdx.x % gs;
    const uint32_t tb = (uint32_t)(((uint64_t)nt * q) / nq) + m;
    const uint32_t te = (uint32_t)(((uint64_t)nt * (q + 1)) / nq);
    if (tb >= te) return;
    FsSync S{bars, bars + FS_S, reinterpret_cast<volatile uint32_t *>(bars + 2 * FS_S), 0u};
    if (threadIdx.x == 0) {
        for (int i = 0; i < FS_S; ++i) {
            mbar_init(S.full + i, FS_NT);
            mbar_init(S.empty + i, FS_WARPS);
        }
        *S.abort = 0u;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    for (int i = threadIdx.x; i < HIST_WORDS / 4; i += FS_NT)
        reinterpret_cast<uint4 *>(sh)[i] = make_uint4(0, 0, 0, 0);
    __syncthreads();
    uint32_t v = find_vol_fs(h, tb);
    for (uint32_t t = tb; t < te; t += gs) {
        while (v + 1 < h->nvol && t >= h->vol[v + 1].fs_base) {
            flush_hist<FS_NT>(h->vol[v], sh);
            ++v;
        }
        const VolDev &V = h->vol[v];
        const uint32_t tl = t - V.fs_base;
        const uint32_t iy = tl % V.fs_nty, rest = tl / V.fs_nty;
        const uint32_t ix = rest % V.fs_ntx, iz = rest / V.fs_ntx;
        const int z0 = (int)(iz * V.fs_tz);
        const int z1 = min(z0 + (int)V.fs_tz, (int)V.Z);
        if (V.fs_rag) {
            if (V.fs_hx) smooth_rows_tile<FS_RT, 1, 1>(V, ix, iy, z0, z1, ring, sh, S);
            else smooth_rows_tile<0, 0, 1>(V, ix, iy, z0, z1, ring, sh, S);
        } else if (V.fs_rt == (uint32_t)FS_RT) {
            if (V.fs_hx) smooth_rows_tile<FS_RT, 1, 0>(V, ix, iy, z0, z1, ring, sh, S);
            else smooth_rows_tile<FS_RT, 0, 0>(V, ix, iy, z0, z1, ring, sh, S);
        } else {
            smooth_rows_tile<0, 0, 0>(V, ix, iy, z0, z1, ring, sh, S);
        }
    }
    asm volatile("cp.async.wait_all;" ::: "memory");  // no copy into this block's shared memory outlives it
    flush_hist<FS_NT>(h->vol[v], sh);
}

// Foreground bits of 8 consecutive smoothed voxels (a 16-byte load, two per
// word, the lower x in the low half): bit j is set iff voxel j > t*.  The OR
// of the four words bounds every voxel from above, so an octet of background
// (almost all of a volume) is settled by one test.
__device__ __forceinline__ uint32_t octet_bits(uint4 q, uint32_t t) {
    const uint32_t ow = q.x | q.y | q.z | q.w;
    if ((ow & 0xFFFFu) <= t && (ow >> 16) <= t) return 0u;
    auto two = [t](uint32_t w) { return ((w & 0xFFFFu) > t ? 1u : 0u) | ((w >> 16) > t ? 2u : 0u); };
    return two(q.x) | (two(q.y) << 2) | (two(q.z) << 4) | (two(q.w) << 6);
}

// Threshold + run count, streaming over the smoothed volume.  One block per
// row tile, one warp per row at a time: foreground bits s > t* are gathered
// into mask words (ballot, or 8 voxels per lane with 16-byte loads when rows
// are 16-byte aligned), and run starts (a set bit whose left neighbour is
// clear, across word boundaries) are counted per row.  The row counts and the
// row tile's total feed the run scan.
__global__ void __launch_bounds__(ROW_TILE) k_threshold_runs(const BatchHdr *__restrict__ h) {
    __shared__ VolIndex<&VolDev::rt_base> VI;
    VI.load(h);
    constexpr int WARPS = ROW_TILE / 32;
    __shared__ uint32_t wsum[WARPS];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (uint32_t rt = blockIdx.x; rt < h->nrowtiles; rt += gridDim.x) {
        const VolDev &V = h->vol[VI.find(h, rt)];
        const uint32_t lt = rt - V.rt_base;
        const uint32_t row0 = lt * h->row_tile;
        const uint32_t nrows = min(h->row_tile, V.rows - row0);
        const uint32_t X = V.X, W = V.W, t = V.stat[ST_THRESH];
        const bool vec = (X & 7u) == 0u;
        uint32_t wtot = 0;
        const uint16_t *wmax = V.wmax;
        if (wmax && (X & 255u) == 0u && W <= 256u && ((W >> 3) & ((W >> 3) - 1u)) == 0u) {
            // Word maxima (rows of 256, 512, ..., 8192 voxels): a lane owns
            // 8 consecutive mask words of one row
            // (one 16-byte load of their maxima), reads the 64 bytes of each
            // word whose maximum is above t* (about one word in eight on
            // microscope data; the others are background) and writes its 8
            // words; a row is W / 8 consecutive lanes, a warp 256 / W rows.
            const uint32_t seg = W >> 3;             // lanes per row: 1, 2, 4, ..., 32
            const uint32_t rows_pw = 32u / seg;      // rows per warp step
            const uint32_t lrow = (uint32_t)lane / seg, lw = ((uint32_t)lane & (seg - 1u)) * 8u;
            for (uint32_t rb = warp * rows_pw; rb < nrows; rb += WARPS * rows_pw) {
                const uint32_t rr = rb + lrow;
                const bool live = rr < nrows;
                const size_t wbase = (size_t)(row0 + rr) * W + lw;
                uint4 mx = make_uint4(0, 0, 0, 0);
                if (live) mx = __ldcs(reinterpret_cast<const uint4 *>(wmax + wbase));
                const uint32_t mw[4] = {mx.x, mx.y, mx.z, mx.w};
                uint32_t act = 0;  // bit i: word lw + i has a voxel above t*
#pragma unroll
                for (int i = 0; i < 4; ++i)
                    act |= ((mw[i] & 0xFFFFu) > t ? 1u : 0u) << (2 * i) | ((mw[i] >> 16) > t ? 2u : 0u) << (2 * i);
                uint32_t word[8];
#pragma unroll
                for (int i = 0; i < 8; ++i) word[i] = 0u;
                const uint16_t *src = V.smooth + (size_t)(row0 + rr) * X + 32u * lw;
                for (uint32_t a = act; a; a &= a - 1u) {
                    const int i = __ffs(a) - 1;
                    const uint4 *p = reinterpret_cast<const uint4 *>(src + 32 * i);
                    const uint4 o0 = __ldcs(p), o1 = __ldcs(p + 1), o2 = __ldcs(p + 2), o3 = __ldcs(p + 3);
                    const uint32_t w = octet_bits(o0, t) | octet_bits(o1, t) << 8 | octet_bits(o2, t) << 16 |
                                       octet_bits(o3, t) << 24;
#pragma unroll
                    for (int j = 0; j < 8; ++j)
                        if (j == i) word[j] = w;
                }
                // run starts: a set bit whose left neighbour (across words,
                // and from the previous lane of the same row) is clear
                uint32_t left = __shfl_up_sync(FULL, word[7], 1) >> 31;
                if (lw == 0u) left = 0u;
                uint32_t cnt = 0;
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    cnt += __popc(word[i] & ~((word[i] << 1) | left));
                    left = word[i] >> 31;
                }
                for (uint32_t o = 1; o < seg; o <<= 1) cnt += __shfl_xor_sync(FULL, cnt, o);
                if (live) {
                    uint4 *dst = reinterpret_cast<uint4 *>(V.mask + wbase);
                    dst[0] = make_uint4(word[0], word[1], word[2], word[3]);
                    dst[1] = make_uint4(word[4], word[5], word[6], word[7]);
                    if (lw == 0u) {
                        V.rowoff[row0 + rr] = cnt;
                        wtot += cnt;
                    }
                }
            }
            // each row was counted by its first lane: the warp's total
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) wtot += __shfl_xor_sync(FULL, wtot, o);
        } else if (wmax && W <= 256u && (X & 1u) == 0u && ((X & 7u) != 0u || X > 512u)) {
            // Word maxima, the other row widths up to 8192 voxels that the
            // 16-byte loop below does not take (X % 8 != 0, or X > 512): a lane owns
            // 8 consecutive mask words (lanes past the row's words hold none),
            // a row is seg lanes (the power of two >= W / 8).  Each word
            // above t* is read as octets (16-byte aligned rows, X % 8 == 0)
            // or as voxel pairs (rows of an even X start 4-byte aligned);
            // the last word of a row stops at X.
            uint32_t seg = 1u;
            while (seg * 8u < W) seg <<= 1;
            const uint32_t rows_pw = 32u / seg;
            const uint32_t lrow = (uint32_t)lane / seg, lw = ((uint32_t)lane & (seg - 1u)) * 8u;
            for (uint32_t rb = warp * rows_pw; rb < nrows; rb += WARPS * rows_pw) {
                const uint32_t rr = rb + lrow;
                const bool live = rr < nrows;
                const uint16_t *mp = wmax + (size_t)(row0 + rr) * W;
                const uint16_t *src = V.smooth + (size_t)(row0 + rr) * X;
                uint32_t word[8];
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    word[i] = 0u;
                    const uint32_t w = lw + (uint32_t)i;
                    if (!live || w >= W || mp[w] <= t) continue;
                    const uint32_t xb = 32u * w, nv = min(32u, X - xb);  // voxels of word w
                    uint32_t bits = 0u;
                    if (vec) {
                        for (uint32_t o = 0; o < nv; o += 8u)
                            bits |= octet_bits(__ldcs(reinterpret_cast<const uint4 *>(src + xb + o)), t) << o;
                    } else {
                        for (uint32_t o = 0; o < nv; o += 2u) {
                            const uint32_t pr = __ldcs(reinterpret_cast<const unsigned int *>(src + xb + o));
                            bits |= (((pr & 0xFFFFu) > t ? 1u : 0u) | ((pr >> 16) > t ? 2u : 0u)) << o;
                        }
                    }
                    word[i] = bits;
                }
                uint32_t left = __shfl_up_sync(FULL, word[7], 1) >> 31;
                if (lw == 0u) left = 0u;
                uint32_t cnt = 0;
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    cnt += __popc(word[i] & ~((word[i] << 1) | left));
                    left = word[i] >> 31;
                }
                for (uint32_t o = 1; o < seg; o <<= 1) cnt += __shfl_xor_sync(FULL, cnt, o);
                if (live) {
                    uint32_t *dst = V.mask + (size_t)(row0 + rr) * W;
#pragma unroll
                    for (int i = 0; i < 8; ++i)
                        if (lw + (uint32_t)i < W) dst[lw + i] = word[i];
                    if (lw == 0u) {
                        V.rowoff[row0 + rr] = cnt;
                        wtot += cnt;
                    }
                }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) wtot += __shfl_xor_sync(FULL, wtot, o);
        } else if (vec && X <= 512u) {
            // 4 rows per warp at once, all 16-byte loads issued first
            for (uint32_t rb = warp; rb < nrows; rb += 4 * WARPS) {
                uint4 q4[4][2];
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const uint32_t rr = rb + k * WARPS;
#pragma unroll
                    for (int c = 0; c < 2; ++c) {
                        const uint32_t x = 256u * c + 8u * (uint32_t)lane;
                        q4[k][c] = (rr < nrows && x < X)
                                       ? __ldcs(reinterpret_cast<const uint4 *>(V.smooth + (size_t)(row0 + rr) * X + x))
                                       : make_uint4(0, 0, 0, 0);
                    }
                }
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const uint32_t rr = rb + k * WARPS;
                    if (rr >= nrows) break;
                    uint32_t *dst = V.mask + (size_t)(row0 + rr) * W;
                    uint32_t carry = 0, cnt = 0;
#pragma unroll
                    for (int c = 0; c < 2; ++c) {
                        const uint32_t xb = 256u * c;
                        if (xb >= X) break;
                        const uint32_t x = xb + 8u * (uint32_t)lane;
                        uint32_t bits = 0;
                        if (x < X) bits = octet_bits(q4[k][c], t);
                        uint32_t word = bits << (8 * (lane & 3));
                        word |= __shfl_xor_sync(FULL, word, 1);
                        word |= __shfl_xor_sync(FULL, word, 2);
                        const uint32_t prev = __shfl_up_sync(FULL, word, 4);
                        const uint32_t left = lane < 4 ? carry : (prev >> 31);
                        const uint32_t wi = (xb >> 5) + ((uint32_t)lane >> 2);
                        if ((lane & 3) == 0 && wi < W) {
                            dst[wi] = word;
                            cnt += __popc(word & ~((word << 1) | left));
                        }
                        carry = __shfl_sync(FULL, word, 28) >> 31;
                    }
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(FULL, cnt, o);
                    if (lane == 0) V.rowoff[row0 + rr] = cnt;
                    wtot += cnt;
                }
            }
        } else
        for (uint32_t rr = warp; rr < nrows; rr += WARPS) {
            const uint32_t row = row0 + rr;
            const uint16_t *src = V.smooth + (size_t)row * X;
            uint32_t *dst = V.mask + (size_t)row * W;
            uint32_t carry = 0, cnt = 0;
            if (vec) {
                // up to 4 x 256 voxels per lane batch: all loads first
                for (uint32_t xb0 = 0; xb0 < X; xb0 += 1024) {
                    uint4 q4[4];
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        const uint32_t x = xb0 + 256u * c + 8u * (uint32_t)lane;
                        q4[c] = x < X ? __ldcs(reinterpret_cast<const uint4 *>(src + x)) : make_uint4(0, 0, 0, 0);
                    }
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        const uint32_t xb = xb0 + 256u * c;
                        if (xb >= X) break;
                        const uint32_t x = xb + 8u * (uint32_t)lane;
                        uint32_t bits = 0;
                        if (x < X) bits = octet_bits(q4[c], t);
                        // lanes 4g..4g+3 hold the 32 bits of word g of this chunk
                        uint32_t word = bits << (8 * (lane & 3));
                        word |= __shfl_xor_sync(FULL, word, 1);
                        word |= __shfl_xor_sync(FULL, word, 2);
                        const uint32_t prev = __shfl_up_sync(FULL, word, 4);
                        const uint32_t left = lane < 4 ? carry : (prev >> 31);
                        const uint32_t wi = (xb >> 5) + ((uint32_t)lane >> 2);
                        if ((lane & 3) == 0 && wi < W) {
                            dst[wi] = word;
                            cnt += __popc(word & ~((word << 1) | left));
                        }
                        carry = __shfl_sync(FULL, word, 28) >> 31;
                    }
                }
            } else {
                for (uint32_t xb = 0; xb < X; xb += 32) {
                    const uint32_t x = xb + (uint32_t)lane;
                    const bool on = x < X && __ldcs(src + x) > t;
                    const uint32_t word = __ballot_sync(FULL, on);
                    if (lane == 0) {
                        dst[xb >> 5] = word;
                        cnt += __popc(word & ~((word << 1) | carry));
                    }
                    carry = word >> 31;
                }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(FULL, cnt, o);
            if (lane == 0) V.rowoff[row] = cnt;
            wtot += cnt;
        }
        if (lane == 0) wsum[warp] = wtot;
        __syncthreads();
        if (threadIdx.x == 0) {
            uint32_t tot = 0;
            for (int w = 0; w < WARPS; ++w) tot += wsum[w];
            V.tsum[lt] = tot;
        }
        __syncthreads();
    }
}

__global__ void __launch_bounds__(ROW_TILE) k_row_runs(const BatchHdr *__restrict__ h) {
    __shared__ VolIndex<&VolDev::rt_base> VI;
    VI.load(h);
    __shared__ uint32_t sbuf[33];
    for (uint32_t rt = blockIdx.x; rt < h->nrowtiles; rt += gridDim.x) {
        const VolDev &V = h->vol[VI.find(h, rt)];
        const uint32_t lt = rt - V.rt_base;
        const uint32_t row = lt * h->row_tile + threadIdx.x;
        const bool own = threadIdx.x < h->row_tile && row < V.rows;
        const uint32_t cnt = own ? V.rowoff[row] : 0u;
        const uint32_t base = tiles_below(V.tsum, lt, sbuf);
        uint32_t tot;
        const uint32_t ex = block_exscan<ROW_TILE>(cnt, &tot, sbuf);
        if (lt + 1 == V.nrt && threadIdx.x == 0) {  // the volume's run count R
            V.stat[ST_RUNS] = base + tot;
            if (base + tot > V.r_cap) atomicOr(V.stat + ST_ERROR, ERR_RCAP);
        }
        if (own) {
            const uint32_t off = base + ex;
            V.rowoff[row] = off;
            if (row == V.rows - 1) V.rowoff[V.rows] = off + cnt;
            if (cnt && off + cnt <= V.r_cap) {
                const uint32_t *m = V.mask + (size_t)row * V.W;
                uint32_t p = 0, k = off;
                const uint32_t kend = off + cnt;
                while (k < kend) {
                    const uint32_t s = find_bit(m, V.W, V.X, p, true);
                    if (s >= V.X) break;
                    const uint32_t e = find_bit(m, V.W, V.X, s, false) - 1;
                    V.run_x[k] = s | (e << 16);
                    V.run_par[k] = k;
                    V.run_aux[k] = 0;
                    ++k;
                    p = e + 1;
                }
            }
        }
    }
}

// Sweep two x-sorted run lists and unite every pair at x-distance <= 1
// (26-adjacency between runs of rows that differ by one in y and/or z).
__device__ __forceinline__ void unite_rows(uint32_t *P, const uint32_t *__restrict__ RX, uint32_t i,
                                           uint32_t ie, uint32_t j, uint32_t je, uint32_t *err,
                                           uint32_t limit) {
    while (i < ie && j < je) {
        const uint32_t a = RX[i], b = RX[j];
        const uint32_t a0 = a & 0xFFFFu, a1 = a >> 16, b0 = b & 0xFFFFu, b1 = b >> 16;
        if (b1 + 1 < a0) { ++j; continue; }
        if (a1 + 1 < b0) { ++i; continue; }
        uf_union(P, i, j, err, limit);
        if (a1 < b1) ++i; else ++j;
    }
}

// ---- brick-local union-find in shared memory ------------------------------
//
// Same rules as the global structure (parent index <= own index, union by
// atomicMin towards the lower index, halving only while uniting), on local
// run indices.  Local indices follow the global run order (brick rows are
// taken z-major, y-minor, like the rows themselves), so the lowest local
// index of a component is also its lowest global index within the brick.

__device__ __forceinline__ uint32_t sm_find(volatile uint32_t *P, uint32_t x) {
    uint32_t p = P[x];
    while (p != x) {
        const uint32_t g = P[p];
        if (g == p) return p;
        P[x] = g;
        x = g;
        p = P[x];
    }
    return x;
}

// Returns false when the retry limit is reached.
__device__ __forceinline__ bool sm_union(volatile uint32_t *P, uint32_t a, uint32_t b, uint32_t limit) {
    for (uint32_t it = 0; it < limit; ++it) {
        a = sm_find(P, a);
        b = sm_find(P, b);
        if (a == b) return true;
        if (a < b) {
            const uint32_t old = atomicMin(const_cast<uint32_t *>(P) + b, a);
            if (old == b) return true;
            b = old;
        } else {
            const uint32_t old = atomicMin(const_cast<uint32_t *>(P) + a, b);
            if (old == a) return true;
            a = old;
        }
    }
    return false;
}

__device__ __forceinline__ bool sm_unite_rows(volatile uint32_t *P, const uint32_t *RX, uint32_t i,
                                              uint32_t ie, uint32_t j, uint32_t je, uint32_t limit) {
    bool ok = true;
    while (i < ie && j < je) {
        const uint32_t a = RX[i], b = RX[j];
        const uint32_t a0 = a & 0xFFFFu, a1 = a >> 16, b0 = b & 0xFFFFu, b1 = b >> 16;
        if (b1 + 1 < a0) { ++j; continue; }
        if (a1 + 1 < b0) { ++i; continue; }
        ok &= sm_union(P, i, j, limit);
        if (a1 < b1) ++i; else ++j;
    }
    return ok;
}

// Every run's parent becomes its root.  Called between barriers, with no
// union in progress: a concurrent reader sees the old parent or the root,
// both ancestors of the node.
__device__ __forceinline__ void sm_compress(volatile uint32_t *P, uint32_t n, uint32_t t, uint32_t nt) {
    for (uint32_t l = t; l < n; l += nt) {
        uint32_t r = P[l];
        if (r == l) continue;
        uint32_t p = P[r];
        while (p != r) {
            r = p;
            p = P[r];
        }
        P[l] = r;
    }
}

// Global run index of local run l: the brick's runs of z-plane lz are one
// contiguous global range starting at gb[lz] (local start soff[lz * BRICK_Y]).
__device__ __forceinline__ uint32_t brick_global(uint32_t l, const uint32_t *soff, const uint32_t *gb) {
    uint32_t lz = 0;
#pragma unroll
    for (int k = 1; k < BRICK_Z; ++k) lz = soff[k * BRICK_Y] <= l ? (uint32_t)k : lz;
    return gb[lz] + (l - soff[lz * BRICK_Y]);
}

// One block per brick of BRICK_Y x BRICK_Z rows, one thread per row.  The
// brick's runs are copied to shared memory, every 26-adjacent pair of runs
// whose rows both lie in the brick is united there, and each run's global
// parent is set to its local root (a valid union-find state: the parent is
// a lower run of the same component).  A brick with more than BRICK_CAP runs
// unites the same pairs through the global structure instead; that touches
// only the brick's own runs, so it cannot interfere with other bricks.
// k_union then unites the pairs of rows that lie in different bricks.
__global__ void __launch_bounds__(BRICK_Y * BRICK_Z) k_union_local(const BatchHdr *__restrict__ h) {
    __shared__ VolIndex<&VolDev::bk_base> VI;
    VI.load(h);
    constexpr int NT = BRICK_Y * BRICK_Z;
    __shared__ uint32_t sx[BRICK_CAP];       // run x0 | x1 << 16
    __shared__ uint32_t sp[BRICK_CAP];       // local parent
    __shared__ uint32_t soff[NT + 1];        // local run offset of each brick row
    __shared__ uint32_t gb[BRICK_Z];         // global index of each plane's first run
    __shared__ uint32_t sbuf[33];
    const uint32_t t = threadIdx.x, ly = t % BRICK_Y, lz = t / BRICK_Y;
    for (uint32_t bk = blockIdx.x; bk < h->nbricks; bk += gridDim.x) {
        const VolDev &V = h->vol[VI.find(h, bk)];
        const uint32_t lb = bk - V.bk_base;
        const uint32_t y = (lb % V.nby) * BRICK_Y + ly, z = (lb / V.nby) * BRICK_Z + lz;
        const bool valid = y < V.Y && z < V.Z;
        const uint32_t row = z * V.Y + y;
        uint32_t ib = 0, cnt = 0;
        if (valid) {
            ib = V.rowoff[row];
            cnt = V.rowoff[row + 1] - ib;
        }
        uint32_t n;
        // the scan's barriers also order this iteration's shared writes after
        // the previous iteration's reads
        const uint32_t loc = block_exscan<NT>(cnt, &n, sbuf);
        if (n == 0) continue;  // n is the same in every thread
        if (n > (uint32_t)BRICK_CAP) {
            if (cnt) {
                const uint32_t ie = ib + cnt, lim = V.union_limit;
                uint32_t *err = V.stat + ST_ERROR;
                if (ly > 0) unite_rows(V.run_par, V.run_x, ib, ie, V.rowoff[row - 1], ib, err, lim);
                if (lz > 0) {
                    const uint32_t rz = row - V.Y;
                    if (ly > 0)
                        unite_rows(V.run_par, V.run_x, ib, ie, V.rowoff[rz - 1], V.rowoff[rz], err, lim);
                    unite_rows(V.run_par, V.run_x, ib, ie, V.rowoff[rz], V.rowoff[rz + 1], err, lim);
                    if (ly + 1 < (uint32_t)BRICK_Y && y + 1 < V.Y)
                        unite_rows(V.run_par, V.run_x, ib, ie, V.rowoff[rz + 1], V.rowoff[rz + 2], err, lim);
                }
            }
            continue;
        }
        soff[t] = loc;
        if (t == NT - 1) soff[NT] = n;
        if (ly == 0) gb[lz] = ib;
        // Each warp holds one plane of the brick (32 rows): it stages its own
        // runs and unites its rows with their (y-1) neighbours, which lie in
        // the same plane, synchronising with __syncwarp only.
        const uint32_t pbeg = __shfl_sync(FULL, loc, 0), pend = __shfl_sync(FULL, loc + cnt, 31);
        const uint32_t pg = __shfl_sync(FULL, ib, 0);  // global index of the plane's first run
        for (uint32_t l = pbeg + ly; l < pend; l += BRICK_Y) {
            sx[l] = V.run_x[pg + (l - pbeg)];
            sp[l] = l;
        }
        __syncwarp();
        // Three phases, each followed by a full compression (every run points
        // at its root) so that no phase walks long paths: rows of one plane,
        // then the same row of the plane below, then the two diagonals.
        const uint32_t i1 = loc + cnt, lim = V.union_limit, u = t - BRICK_Y;
        bool ok = true;
        if (cnt && ly > 0) ok &= sm_unite_rows(sp, sx, loc, i1, soff[t - 1], soff[t], lim);  // (y-1, z)
        __syncwarp();
        for (uint32_t l = pbeg + ly; l < pend; l += BRICK_Y) {  // compress this plane's runs
            uint32_t r = sp[l];
            if (r == l) continue;
            uint32_t q = sp[r];
            while (q != r) {
                r = q;
                q = sp[r];
            }
            sp[l] = r;
        }
        __syncthreads();
        if (cnt && lz > 0) ok &= sm_unite_rows(sp, sx, loc, i1, soff[u], soff[u + 1], lim);  // (y, z-1)
        __syncthreads();
        sm_compress(sp, n, t, NT);
        __syncthreads();
        if (cnt && lz > 0) {
            if (ly > 0) ok &= sm_unite_rows(sp, sx, loc, i1, soff[u - 1], soff[u], lim);     // (y-1, z-1)
            if (ly + 1 < (uint32_t)BRICK_Y)
                ok &= sm_unite_rows(sp, sx, loc, i1, soff[u + 1], soff[u + 2], lim);         // (y+1, z-1)
        }
        if (!ok) atomicOr(V.stat + ST_ERROR, ERR_UNION);
        __syncthreads();
        for (uint32_t l = t; l < n; l += NT) {
            uint32_t r = l, p = sp[r];
            while (p != r) {  // no writers any more; parents only decrease
                r = p;
                p = sp[r];
            }
            V.run_par[brick_global(l, soff, gb)] = brick_global(r, soff, gb);
        }
    }
}

// One thread per pair of 26-adjacent rows that lie in different bricks, in
// four groups (row y, plane z; neighbour rows (y-1,z), (y-1,z-1), (y,z-1),
// (y+1,z-1)):
//   planes z = 8k > 0: every row with each of its three neighbours in z-1;
//   rows y = 32k > 0, every plane: (y-1, z);
//   rows y = 32k > 0, the other planes z > 0: (y-1, z-1);
//   rows y = 32k - 1 (y+1 < Y), the other planes z > 0: (y+1, z-1).
// Consecutive threads take consecutive rows of a plane where they can.
__global__ void __launch_bounds__(ROW_TILE) k_union(const BatchHdr *__restrict__ h) {
    __shared__ VolIndex<&VolDev::bt_base> VI;
    VI.load(h);
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t gt = blockIdx.x * blockDim.x + threadIdx.x; gt < h->nbtasks; gt += stride) {
        const VolDev &V = h->vol[VI.find(h, gt)];
        uint32_t t = gt - V.bt_base;
        const uint32_t Y = V.Y, Z = V.Z;
        const uint32_t nzb = (Z - 1) / BRICK_Z, nyb = (Y - 1) / BRICK_Y, nzi = Z - 1 - nzb;
        uint32_t y, z, nb;
        if (t < nzb * Y * 3) {
            const uint32_t pz = t / (3 * Y), rem = t - pz * 3 * Y;
            z = BRICK_Z * (pz + 1);
            nb = 1 + rem / Y;
            y = rem % Y;
        } else {
            t -= nzb * Y * 3;
            if (t < nyb * Z) {
                z = t / nyb;
                y = BRICK_Y * (t % nyb + 1);
                nb = 0;
            } else {
                t -= nyb * Z;
                const uint32_t grp = t / (nyb * nzi);  // 0: (y-1, z-1) at y = 32k; 1: (y+1, z-1) at 32k - 1
                t -= grp * nyb * nzi;
                const uint32_t iz = t / nyb;
                z = iz + 1 + iz / (BRICK_Z - 1);  // the iz-th plane with z % 8 != 0, z > 0
                y = BRICK_Y * (t % nyb + 1) - grp;
                nb = grp ? 3u : 1u;
            }
        }
        if (nb == 1 && y == 0) continue;
        if (nb == 3 && y + 1 >= Y) continue;
        const uint32_t row = z * Y + y;
        const uint32_t ib = V.rowoff[row], ie = V.rowoff[row + 1];
        if (ib == ie) continue;
        const uint32_t r = nb == 0 ? row - 1 : row - Y + nb - 2;
        unite_rows(V.run_par, V.run_x, ib, ie, V.rowoff[r], V.rowoff[r + 1], V.stat + ST_ERROR, V.union_limit);
    }
}

// One thread per run (all volumes of the batch in turn): parent = root, and
// the run's voxels are added to the root's size, one atomic per warp when all
// its lanes share a root.
__global__ void __launch_bounds__(ROW_TILE) k_flatten(const BatchHdr *__restrict__ h) {
    const uint32_t stride = gridDim.x * blockDim.x;
    const uint32_t lane = threadIdx.x & 31;
    for (uint32_t v = 0; v < h->nvol; ++v) {
        const VolDev &V = h->vol[v];
        const uint32_t R = V.rowoff[V.rows];
        // whole warps stay in the loop so that the shuffles see every lane
        for (uint32_t j0 = blockIdx.x * blockDim.x + (threadIdx.x & ~31u); j0 < R; j0 += stride) {
            const uint32_t j = j0 + lane;
            uint32_t root = 0xFFFFFFFFu, len = 0;
            if (j < R) {
                root = uf_root(V.run_par, j);
                V.run_par[j] = root;
                const uint32_t x = V.run_x[j];
                len = (x >> 16) - (x & 0xFFFFu) + 1u;
            }
            const uint32_t r0 = __shfl_sync(FULL, root, 0);
            if (__all_sync(FULL, root == r0 || j >= R)) {
                uint32_t sum = len;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(FULL, sum, o);
                if (lane == 0) atomicAdd(V.run_aux + r0, sum);
            } else if (j < R) {
                atomicAdd(V.run_aux + root, len);
            }
        }
    }
}

__global__ void __launch_bounds__(ROW_TILE) k_keep_count(const BatchHdr *__restrict__ h) {
    __shared__ VolIndex<&VolDev::rt_base> VI;
    VI.load(h);
    __shared__ uint32_t sbuf[33];
    for (uint32_t rt = blockIdx.x; rt < h->nrowtiles; rt += gridDim.x) {
        const VolDev &V = h->vol[VI.find(h, rt)];
        const uint32_t lt = rt - V.rt_base;
        const uint32_t row = lt * h->row_tile + threadIdx.x;
        uint32_t cnt = 0;
        if (threadIdx.x < h->row_tile && row < V.rows) {
            const uint32_t ib = V.rowoff[row], ie = V.rowoff[row + 1];
            for (uint32_t r = ib; r < ie; ++r)
                cnt += (V.run_par[r] == r && V.run_aux[r] >= V.min_volume) ? 1u : 0u;
            V.rowk[row] = cnt;
        }
        const uint32_t tot = block_sum<ROW_TILE>(cnt, sbuf);
        if (threadIdx.x == 0) V.tkeep[lt] = tot;
    }
}

__global__ void __launch_bounds__(ROW_TILE) k_rank(const BatchHdr *__restrict__ h) {
    __shared__ VolIndex<&VolDev::rt_base> VI;
    VI.load(h);
    __shared__ uint32_t sbuf[33];
    for (uint32_t rt = blockIdx.x; rt < h->nrowtiles; rt += gridDim.x) {
        const VolDev &V = h->vol[VI.find(h, rt)];
        const uint32_t lt = rt - V.rt_base;
        const uint32_t row = lt * h->row_tile + threadIdx.x;
        const bool own = threadIdx.x < h->row_tile && row < V.rows;
        const uint32_t cnt = own ? V.rowk[row] : 0u;
        const uint32_t base = tiles_below(V.tkeep, lt, sbuf);
        uint32_t tot;
        const uint32_t ex = block_exscan<ROW_TILE>(cnt, &tot, sbuf);
        if (lt + 1 == V.nrt && threadIdx.x == 0) {  // the volume's cell count K
            V.stat[ST_CELLS] = base + tot;
            if (base + tot > V.k_cap) atomicOr(V.stat + ST_ERROR, ERR_KCAP);
        }
        if (own) {
            uint32_t lab = base + ex;
            const uint32_t ib = V.rowoff[row], ie = V.rowoff[row + 1];
            for (uint32_t r = ib; r < ie; ++r) {
                if (V.run_par[r] != r) continue;
                if (V.run_aux[r] >= V.min_volume) {
                    ++lab;
                    V.run_aux[r] = lab;
                    if (lab <= V.k_cap) {
                        seg_cell_features f;
                        f.count = 0;
                        f.sum[0] = f.sum[1] = f.sum[2] = 0;
                        f.bbox_min[0] = f.bbox_min[1] = f.bbox_min[2] = 0xFFFFFFFFu;
                        f.bbox_max[0] = f.bbox_max[1] = f.bbox_max[2] = 0;
                        f.pad[0] = f.pad[1] = 0;
                        V.feat[lab - 1] = f;
                    }
                } else {
                    V.run_aux[r] = 0;
                }
            }
        }
    }
}

// Per-block aggregation of cell features: an open-addressed table keyed by
// label in shared memory; a run whose label finds no slot within FEAT_PROBES
// probes goes straight to global atomics.
constexpr int FEAT_SLOTS = 256;
constexpr int FEAT_PROBES = 8;

// cx packs a cell's voxel count in a row tile (at most 256 * 65536 = 2^24,
// 25 bits) under its x-coordinate sum (at most 256 * (0 + ... + 65535) < 2^39),
// so one 64-bit add carries both exactly.
constexpr int CX_SHIFT = 25;

struct FeatTable {
    uint32_t key[FEAT_SLOTS];
    unsigned long long cx[FEAT_SLOTS], sy[FEAT_SLOTS], sz[FEAT_SLOTS];
    uint32_t mn[3][FEAT_SLOTS], mx[3][FEAT_SLOTS];
};

// Shared min / max that skip the atomic when the value cannot change the
// result: a stale read is never below the current minimum (above the
// current maximum), so a value it rules out is ruled out for good.
__device__ __forceinline__ void smin(uint32_t *a, uint32_t v) {
    if (v < *reinterpret_cast<volatile uint32_t *>(a)) atomicMin(a, v);
}
__device__ __forceinline__ void smax(uint32_t *a, uint32_t v) {
    if (v > *reinterpret_cast<volatile uint32_t *>(a)) atomicMax(a, v);
}

__device__ __forceinline__ void feat_global(seg_cell_features *f, unsigned long long cnt, unsigned long long sx,
                                            unsigned long long sy, unsigned long long sz, const uint32_t *mn,
                                            const uint32_t *mx) {
    atomicAdd(reinterpret_cast<unsigned long long *>(&f->count), cnt);
    atomicAdd(reinterpret_cast<unsigned long long *>(&f->sum[0]), sx);
    atomicAdd(reinterpret_cast<unsigned long long *>(&f->sum[1]), sy);
    atomicAdd(reinterpret_cast<unsigned long long *>(&f->sum[2]), sz);
    for (int a = 0; a < 3; ++a) {
        atomicMin(&f->bbox_min[a], mn[a]);
        atomicMax(&f->bbox_max[a], mx[a]);
    }
}

// One block per row tile (256 consecutive rows; their labels are one
// contiguous range).  The tile's runs (x extent and final label, the label
// being its root's, set by k_rank) are first loaded into shared memory by all
// threads at once, so that no row waits on its own chain of global loads;
// a tile with more than LABEL_RUNS runs reads them from global memory
// instead.  Labels: one warp per row, 16-byte streaming stores when rows are
// 16-byte aligned (X % 4 == 0), zeros between runs.  Then one thread per run
// folds the run's contribution to its cell (count, coordinate sums, bounding
// box) into a shared table; after a barrier the table goes to the global
// cells with one set of atomics per (tile, cell).
constexpr int LABEL_RUNS = 2048;

__global__ void __launch_bounds__(ROW_TILE, 6) k_label_features(const BatchHdr *__restrict__ h) {
    __shared__ VolIndex<&VolDev::rt_base> VI;
    VI.load(h);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    constexpr int WARPS = ROW_TILE / 32;
    __shared__ uint32_t soff[ROW_TILE + 1];
    __shared__ uint2 srl[LABEL_RUNS];  // staged runs: x0 | x1 << 16, final label
    __shared__ uint8_t srow[LABEL_RUNS];  // row of each staged run in the tile
    __shared__ FeatTable T;
    for (uint32_t rt = blockIdx.x; rt < h->nrowtiles; rt += gridDim.x) {
        const VolDev &V = h->vol[VI.find(h, rt)];
        const uint32_t lt = rt - V.rt_base;
        const uint32_t row0 = lt * h->row_tile;
        const uint32_t nrows = min(h->row_tile, V.rows - row0);
        __syncthreads();  // previous tile done with soff, srl and T
        for (uint32_t i = tid; i <= nrows; i += ROW_TILE) soff[i] = V.rowoff[row0 + i];
        T.key[tid] = 0u;
        T.cx[tid] = T.sy[tid] = T.sz[tid] = 0ull;
        for (int a = 0; a < 3; ++a) {
            T.mn[a][tid] = 0xFFFFFFFFu;
            T.mx[a][tid] = 0u;
        }
        __syncthreads();
        const uint32_t *__restrict__ RX = V.run_x;
        const uint32_t *__restrict__ RP = V.run_par;
        const uint32_t *__restrict__ RA = V.run_aux;
        const uint32_t rb = soff[0], re = soff[nrows];
        const bool staged = re - rb <= (uint32_t)LABEL_RUNS;  // the same in every thread
        if (staged) {
            for (uint32_t j = rb + tid; j < re; j += ROW_TILE) {
                srl[j - rb] = make_uint2(RX[j], RA[RP[j]]);
            }
            if ((uint32_t)tid < nrows)
                for (uint32_t j = soff[tid]; j < soff[tid + 1]; ++j) srow[j - rb] = (uint8_t)tid;
            __syncthreads();
        }
        auto run_x = [&](uint32_t j) { return staged ? srl[j - rb].x : RX[j]; };
        auto run_label = [&](uint32_t j) { return staged ? srl[j - rb].y : RA[RP[j]]; };
        // labels
        const uint32_t X = V.X;
        const bool vec = (X & 3u) == 0u;
        for (uint32_t rr = warp; rr < nrows; rr += WARPS) {
            uint32_t *out = V.labels + (size_t)(row0 + rr) * X;
            const uint32_t ib = soff[rr], ie = soff[rr + 1];
            if (vec) {
                uint4 *o4 = reinterpret_cast<uint4 *>(out);
                if (ib == ie) {
                    for (uint32_t x = lane; x < X / 4; x += 32) __stcs(o4 + x, make_uint4(0, 0, 0, 0));
                    continue;
                }
                if (staged && ie - ib <= 16u) {
                    // few runs: every lane goes through the row's runs in
                    // step (broadcast reads, no divergent walk) for each
                    // 128-voxel segment, and fills its 4-voxel chunk
                    uint32_t j = ib;
                    for (uint32_t sb = 0; sb < X; sb += 128) {
                        const uint32_t xb = sb + 4u * lane;
                        uint32_t v0 = 0, v1 = 0, v2 = 0, v3 = 0;
                        while (j < ie && (srl[j - rb].x >> 16) < sb) ++j;
                        for (uint32_t k = j; k < ie; ++k) {
                            const uint2 rl = srl[k - rb];  // one 8-byte load: extent and label
                            const uint32_t rx = rl.x;
                            const uint32_t x0 = rx & 0xFFFFu, x1 = rx >> 16;
                            if (x0 >= sb + 128u) break;
                            if (x1 < xb || x0 > xb + 3u) continue;
                            const uint32_t L = rl.y, w = x1 - x0;
                            if (xb - x0 <= w) v0 = L;
                            if (xb + 1u - x0 <= w) v1 = L;
                            if (xb + 2u - x0 <= w) v2 = L;
                            if (xb + 3u - x0 <= w) v3 = L;
                        }
                        if (xb < X) __stcs(o4 + xb / 4, make_uint4(v0, v1, v2, v3));
                    }
                    continue;
                }
                uint32_t j = ib, jx = run_x(ib), jl = run_label(ib);
                for (uint32_t xb = 4 * lane; xb < X; xb += 128) {
                    // j: the first run that does not end before xb
                    while (j < ie && (jx >> 16) < xb) {
                        if (++j < ie) {
                            jx = run_x(j);
                            jl = run_label(j);
                        }
                    }
                    uint4 o;
                    if (j >= ie || (jx & 0xFFFFu) > xb + 3u) {
                        o = make_uint4(0, 0, 0, 0);            // the 4 voxels lie before run j
                    } else if ((jx & 0xFFFFu) <= xb && (jx >> 16) >= xb + 3u) {
                        o = make_uint4(jl, jl, jl, jl);        // all 4 inside run j
                    } else {
                        uint32_t l4[4];
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            const uint32_t x = xb + q;
                            while (j < ie && (jx >> 16) < x) {
                                if (++j < ie) {
                                    jx = run_x(j);
                                    jl = run_label(j);
                                }
                            }
                            l4[q] = (j < ie && (jx & 0xFFFFu) <= x) ? jl : 0u;
                        }
                        o = make_uint4(l4[0], l4[1], l4[2], l4[3]);
                    }
                    __stcs(o4 + xb / 4, o);
                }
            } else {
                if (ib == ie) {
                    for (uint32_t x = lane; x < X; x += 32) __stcs(out + x, 0u);
                    continue;
                }
                uint32_t j = ib, jx = run_x(ib), jl = run_label(ib);
                for (uint32_t x = lane; x < X; x += 32) {
                    while (j < ie && (jx >> 16) < x) {
                        if (++j < ie) {
                            jx = run_x(j);
                            jl = run_label(j);
                        }
                    }
                    __stcs(out + x, (j < ie && (jx & 0xFFFFu) <= x) ? jl : 0u);
                }
            }
        }
        for (uint32_t j = rb + tid; j < re; j += ROW_TILE) {
            const uint32_t lab = run_label(j);
            if (!lab || lab > V.k_cap) continue;
            uint32_t lo;
            if (staged) {
                lo = srow[j - rb];
            } else {
                // row of run j: the last i with soff[i] <= j
                uint32_t hi = nrows;
                lo = 0;
                while (hi - lo > 1) {
                    const uint32_t mid = (lo + hi) >> 1;
                    if (soff[mid] <= j) lo = mid; else hi = mid;
                }
            }
            const uint32_t row = row0 + lo;
            const uint32_t y = row % V.Y, z = row / V.Y;
            const uint32_t rx = run_x(j);
            const uint32_t x0 = rx & 0xFFFFu, x1 = rx >> 16;
            const unsigned long long len = x1 - x0 + 1u;
            const unsigned long long sx = ((unsigned long long)(x0 + x1) * len) >> 1;
            uint32_t slot = (lab * 2654435761u) >> 24;
            bool done = false;
            for (int p = 0; p < FEAT_PROBES && !done; ++p, slot = (slot + 1) & (FEAT_SLOTS - 1)) {
                uint32_t k = *reinterpret_cast<volatile uint32_t *>(&T.key[slot]);
                if (k == 0u) k = atomicCAS(&T.key[slot], 0u, lab);
                if (k == 0u || k == lab) {
                    atomicAdd(&T.cx[slot], (sx << CX_SHIFT) | len);
                    atomicAdd(&T.sy[slot], len * y);
                    atomicAdd(&T.sz[slot], len * z);
                    smin(&T.mn[0][slot], x0);
                    smax(&T.mx[0][slot], x1);
                    smin(&T.mn[1][slot], y);
                    smax(&T.mx[1][slot], y);
                    smin(&T.mn[2][slot], z);
                    smax(&T.mx[2][slot], z);
                    done = true;
                }
            }
            if (!done) {
                const uint32_t mn[3] = {x0, y, z}, mx[3] = {x1, y, z};
                feat_global(V.feat + (lab - 1), len, sx, len * y, len * z, mn, mx);
            }
        }
        __syncthreads();
        {
            const uint32_t lab = T.key[tid];
            if (lab) {
                const uint32_t mn[3] = {T.mn[0][tid], T.mn[1][tid], T.mn[2][tid]};
                const uint32_t mx[3] = {T.mx[0][tid], T.mx[1][tid], T.mx[2][tid]};
                const unsigned long long cx = T.cx[tid];
                feat_global(V.feat + (lab - 1), cx & ((1ull << CX_SHIFT) - 1), cx >> CX_SHIFT, T.sy[tid],
                            T.sz[tid], mn, mx);
            }
        }
    }
}

// Copies every volume's status words to one contiguous buffer (fixed-size
// read-back for the host, independent of where the volumes live).
__global__ void k_gather_stat(const BatchHdr *__restrict__ h, uint32_t *out) {
    const uint32_t n = h->nvol * ST_WORDS;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        out[i] = h->vol[i / ST_WORDS].stat[i % ST_WORDS];
}

// ----------------------------------------------------------------------------
// Denoise front end of the stem-cell channel (Background Noise Removal,
// Eq. 1): background B by box passes, D = max(L - B, 0), 3x3x3 median of D
// ----------------------------------------------------------------------------

// (n + r) / w for n + r < 2^24 and w = 2r + 1 <= 65, as a multiply-high by
// mul = ceil(2^32 / w) (division by an invariant integer, Granlund and
// Montgomery 1994): the product's error n * (mul * w - 2^32) / (w 2^32) stays
// below 2^-8 < 1/w, so the floor is exact.
__device__ __forceinline__ uint32_t box_div(uint32_t n, uint32_t mul) { return __umulhi(n, mul); }

// The three rounded box passes of radius r along AXIS, for every tile of 64
// lines x DN_CHUNK positions of the volumes with the denoise front end.  A
// block loads its tile with a halo of 3r positions on each side (clamped to
// the line) into shared memory, runs the three passes there -- pass k over
// the positions the next one needs, each reading its input at positions
// clamped to the line, which is the replicate edge of every pass -- and
// writes the chunk.  Axis x reads dn_src and writes dn_a, y reads dn_a and
// writes dn_b, z reads dn_b and writes the background into dn_a.  Shared
// layout [position][lane], lanes padded to 66 so that both the lane-major
// passes and the position-major copies of axis x avoid bank conflicts.
constexpr int BOX_LANES = 64, BOX_PITCH = BOX_LANES + 2;
constexpr int BOX_POS = DN_CHUNK + 6 * DN_MAX_R;
constexpr size_t BOX_SMEM = 2ull * BOX_POS * BOX_PITCH * sizeof(uint16_t);

template <int AXIS>
__global__ void __launch_bounds__(256) k_box3(const BatchHdr *__restrict__ h) {
    __shared__ VolIndex<AXIS == 0 ? &VolDev::dn_base0 : (AXIS == 1 ? &VolDev::dn_base1 : &VolDev::dn_base2)> VI;
    extern __shared__ __align__(16) uint16_t bsm[];
    uint16_t *bufA = bsm, *bufB = bsm + BOX_POS * BOX_PITCH;
    VI.load(h);
    const int t = threadIdx.x;
    for (uint32_t it = blockIdx.x; it < h->dn_items[AXIS]; it += gridDim.x) {
        const VolDev &V = h->vol[VI.find(h, it)];
        const uint32_t li = it - (AXIS == 0 ? V.dn_base0 : (AXIS == 1 ? V.dn_base1 : V.dn_base2));
        const int X = (int)V.X, Y = (int)V.Y, Z = (int)V.Z;
        const int n = AXIS == 0 ? X : (AXIS == 1 ? Y : Z);
        const int nchunk = (n + DN_CHUNK - 1) / DN_CHUNK;
        const int group = (int)(li / (uint32_t)nchunk), chunk = (int)(li % (uint32_t)nchunk);
        const int r = (int)V.dn_r;
        const uint32_t mul = V.dn_mul;
        const int c0 = chunk * DN_CHUNK, c1 = min(c0 + DN_CHUNK, n), base = c0 - 3 * r;
        const int lo = max(base, 0), hi = min(c1 + 3 * r, n);  // loaded positions
        // lane l of this group: its line's first element and the step along it
        const int nxg = (X + BOX_LANES - 1) / BOX_LANES;
        int nl;            // lanes of this group that exist
        size_t gstart;     // element of lane 0 at position 0
        size_t lstride, pstride;
        if (AXIS == 0) {
            const int rows = Y * Z;
            nl = min(BOX_LANES, rows - group * BOX_LANES);
            gstart = (size_t)group * BOX_LANES * X;
            lstride = (size_t)X;
            pstride = 1;
        } else {
            const int gx = group % nxg, other = group / nxg;
            nl = min(BOX_LANES, X - gx * BOX_LANES);
            lstride = 1;
            if (AXIS == 1) {
                gstart = (size_t)gx * BOX_LANES + (size_t)X * Y * other;
                pstride = (size_t)X;
            } else {
                gstart = (size_t)gx * BOX_LANES + (size_t)X * other;
                pstride = (size_t)X * Y;
            }
        }
        const uint16_t *src = AXIS == 0 ? V.dn_src : (AXIS == 1 ? V.dn_a : V.dn_b);
        uint16_t *dst = AXIS == 1 ? V.dn_b : V.dn_a;
        const int np = hi - lo;
        __syncthreads();  // the previous tile is done with the buffers
        // load: consecutive threads on consecutive elements in memory, eight
        // independent loads in flight per thread before the shared stores
        constexpr int NB = 8;
        if (AXIS == 0) {
            // one warp per line (a row segment), lanes along it
            const int lane = t & 31, warp = t >> 5, nw = blockDim.x >> 5;
            for (int l = warp; l < nl; l += nw) {
                const uint16_t *row = src + gstart + (size_t)l * lstride;
                for (int q0 = lo + lane; q0 < hi; q0 += 32 * NB) {
                    uint16_t v[NB];
#pragma unroll
                    for (int j = 0; j < NB; ++j)
                        if (q0 + 32 * j < hi) v[j] = row[q0 + 32 * j];
#pragma unroll
                    for (int j = 0; j < NB; ++j)
                        if (q0 + 32 * j < hi) bufA[(q0 + 32 * j - base) * BOX_PITCH + l] = v[j];
                }
            }
        } else if ((X & 7) == 0) {
            // rows of 8-voxel octets (X % 8 == 0, scratch buffers 16-byte
            // aligned): thread t moves lanes 8 (t % 8) .. + 7 of positions
            // t / 8 + 32 i as one 16-byte load and four 4-byte shared stores
            // (pitch 66: the 32 threads of a warp hit 32 different banks)
            const int oct = t & 7, pr = t >> 3;
            constexpr int NV = 4;
            if (8 * oct < nl) {
                const uint16_t *col = src + gstart + 8 * oct;
                for (int q0 = lo + pr; q0 < hi; q0 += 32 * NV) {
                    uint4 v[NV];
#pragma unroll
                    for (int j = 0; j < NV; ++j)
                        if (q0 + 32 * j < hi)
                            v[j] = *reinterpret_cast<const uint4 *>(col + (size_t)(q0 + 32 * j) * pstride);
#pragma unroll
                    for (int j = 0; j < NV; ++j)
                        if (q0 + 32 * j < hi) {
                            uint32_t *w = reinterpret_cast<uint32_t *>(bufA + (q0 + 32 * j - base) * BOX_PITCH + 8 * oct);
                            w[0] = v[j].x; w[1] = v[j].y; w[2] = v[j].z; w[3] = v[j].w;
                        }
                }
            }
        } else {
            const int total = np * BOX_LANES, nt = blockDim.x;
            for (int i0 = t; i0 < total; i0 += nt * NB) {
                uint16_t v[NB];
#pragma unroll
                for (int j = 0; j < NB; ++j) {
                    const int i = i0 + j * nt, l = i % BOX_LANES, q = lo + i / BOX_LANES;
                    if (i < total && l < nl) v[j] = src[gstart + (size_t)l * lstride + (size_t)q * pstride];
                }
#pragma unroll
                for (int j = 0; j < NB; ++j) {
                    const int i = i0 + j * nt, l = i % BOX_LANES, q = lo + i / BOX_LANES;
                    if (i < total && l < nl) bufA[(q - base) * BOX_PITCH + l] = v[j];
                }
            }
        }
        __syncthreads();
        // three passes: A -> B over [c0-2r, c1+2r), B -> A over [c0-r, c1+r), A -> B over [c0, c1)
        const int l = t % BOX_LANES, seg = t / BOX_LANES;
        for (int k = 0; k < 3; ++k) {
            const uint16_t *in = (k == 1) ? bufB : bufA;
            uint16_t *out = (k == 1) ? bufA : bufB;
            const int p0 = max(c0 - (2 - k) * r, 0), p1 = min(c1 + (2 - k) * r, n);
            const int per = (p1 - p0 + 3) / 4;
            const int q0 = p0 + seg * per, q1 = min(q0 + per, p1);
            if (l < nl && q0 < q1) {
                // every read lies in [q0 - r, q1 - 1 + r] clamped to the line,
                // inside the positions the previous pass (or the load) covered
                auto at = [&](int q) { return (uint32_t)in[(min(max(q, 0), n - 1) - base) * BOX_PITCH + l]; };
                // sum holds the window sum plus the rounding term r
                uint32_t sum = (uint32_t)r;
                if (q0 - r >= 0 && q0 + r < n) {
                    const uint16_t *pw = in + (q0 - r - base) * BOX_PITCH + l;
                    for (int i = 0; i <= 2 * r; ++i) sum += pw[i * BOX_PITCH];
                } else {
                    for (int q = q0 - r; q <= q0 + r; ++q) sum += at(q);
                }
                out[(q0 - base) * BOX_PITCH + l] = (uint16_t)box_div(sum, mul);
                // positions q whose window [q - r - 1, q + r] needs no
                // clamping run through three moving pointers
                const int qa = min(max(q0 + 1, r + 1), q1), qb = max(min(q1, n - r), qa);
                int q = q0 + 1;
                for (; q < qa; ++q) {
                    sum += at(q + r) - at(q - r - 1);
                    out[(q - base) * BOX_PITCH + l] = (uint16_t)box_div(sum, mul);
                }
                const uint16_t *pin = in + (q + r - base) * BOX_PITCH + l;
                const uint16_t *pout = in + (q - r - 1 - base) * BOX_PITCH + l;
                uint16_t *po = out + (q - base) * BOX_PITCH + l;
#pragma unroll 4
                for (; q < qb; ++q) {
                    sum += (uint32_t)*pin - (uint32_t)*pout;
                    *po = (uint16_t)box_div(sum, mul);
                    pin += BOX_PITCH;
                    pout += BOX_PITCH;
                    po += BOX_PITCH;
                }
                for (; q < q1; ++q) {
                    sum += at(q + r) - at(q - r - 1);
                    out[(q - base) * BOX_PITCH + l] = (uint16_t)box_div(sum, mul);
                }
            }
            __syncthreads();
        }
        // store the chunk from B
        const int nc = c1 - c0;
        if (AXIS == 0) {
            const int lane = t & 31, warp = t >> 5, nw = blockDim.x >> 5;
            for (int ll = warp; ll < nl; ll += nw) {
                uint16_t *row = dst + gstart + (size_t)ll * lstride;
                for (int q = c0 + lane; q < c1; q += 32) row[q] = bufB[(q - base) * BOX_PITCH + ll];
            }
        } else if ((X & 7) == 0) {
            const int oct = t & 7, pr = t >> 3;
            if (8 * oct < nl) {
                uint16_t *col = dst + gstart + 8 * oct;
                for (int q = c0 + pr; q < c1; q += 32) {
                    const uint32_t *w = reinterpret_cast<const uint32_t *>(bufB + (q - base) * BOX_PITCH + 8 * oct);
                    *reinterpret_cast<uint4 *>(col + (size_t)q * pstride) = make_uint4(w[0], w[1], w[2], w[3]);
                }
            }
        } else {
            for (int i = t; i < nc * BOX_LANES; i += blockDim.x) {
                const int ll = i % BOX_LANES, q = c0 + i / BOX_LANES;
                if (ll < nl) dst[gstart + (size_t)ll * lstride + (size_t)q * pstride] = bufB[(q - base) * BOX_PITCH + ll];
            }
        }
    }
}

// D = max(L - B, 0) staged per tile of 64 x 8 x 8 voxels (plus a one-voxel
// halo, clamped), then the median of each voxel's 27 neighbours from the
// sorted 3x3 neighbourhoods of its three planes; the result is the volume
// the smoothing reads.  Each thread takes two neighbouring voxels along x:
// the comparator networks run on 16-bit halves of 32-bit words (packed min
// and max), and the pairs of a 3x3 row are two aligned shared-memory words
// and one byte permutation of them.
constexpr int MED_TX = 32, MED_TY = 8, MED_TZ = 8;  // threads along x and y; planes per tile
static_assert(2 * MED_TX == MED_TILE_X && MED_TY == MED_TILE_Y && MED_TZ == MED_TILE_Z, "median tile");

__global__ void __launch_bounds__(MED_TX * MED_TY, 4) k_median27(const BatchHdr *__restrict__ h) {
    __shared__ VolIndex<&VolDev::dn_tbase> VI;
    __shared__ __align__(16) uint16_t d[MED_TZ + 2][MED_TY + 2][MED_TILE_X + 2];  // rows of 132 bytes
    VI.load(h);
    const int tx = threadIdx.x % MED_TX, ty = threadIdx.x / MED_TX;
    for (uint32_t t = blockIdx.x; t < h->dn_tiles; t += gridDim.x) {
        const VolDev &V = h->vol[VI.find(h, t)];
        const uint32_t lt = t - V.dn_tbase;
        const int X = (int)V.X, Y = (int)V.Y, Z = (int)V.Z;
        const int ntx = (X + MED_TILE_X - 1) / MED_TILE_X, nty = (Y + MED_TY - 1) / MED_TY;
        const int x0 = (int)(lt % ntx) * MED_TILE_X, y0 = (int)((lt / ntx) % nty) * MED_TY;
        const int z0 = (int)(lt / ((uint32_t)ntx * nty)) * MED_TZ;
        __syncthreads();  // the previous tile is done with d
        constexpr int SXW = MED_TILE_X + 2;
        // Staging: one warp per staged row (MED_TZ + 2 planes x MED_TY + 2
        // rows of SXW voxels, x, y and z clamped to the volume); lane l takes
        // shared x indices 2l and 2l + 1 (one 32-bit shared word), lanes 0
        // and 1 also index 64 + l.  A row's clamped y and z and its base are
        // computed once; four rows' loads are in flight per lane.
        {
            static_assert(SXW == 66 && MED_TX * MED_TY == 256, "staging layout");
            constexpr int NROW = (MED_TZ + 2) * (MED_TY + 2), RB = 4, NW = MED_TX * MED_TY / 32;
            const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
            const int xa = min(max(x0 - 1 + 2 * lane, 0), X - 1), xb = min(max(x0 + 2 * lane, 0), X - 1);
            const int xc = min(max(x0 + 63 + lane, 0), X - 1);  // index 64 + lane (lanes 0, 1)
            uint16_t *ds = &d[0][0][0];
            for (int r0 = warp; r0 < NROW; r0 += NW * RB) {
                uint32_t la[RB], lb[RB], lc[RB], ba[RB], bb[RB], bc[RB];
#pragma unroll
                for (int j = 0; j < RB; ++j) {
                    const int rr = r0 + NW * j;
                    la[j] = lb[j] = lc[j] = ba[j] = bb[j] = bc[j] = 0u;
                    if (rr < NROW) {
                        const int sz = rr / (MED_TY + 2), sy = rr - sz * (MED_TY + 2);
                        const int y = min(max(y0 - 1 + sy, 0), Y - 1), z = min(max(z0 - 1 + sz, 0), Z - 1);
                        const size_t ro = (size_t)X * ((size_t)y + (size_t)Y * z);
                        const uint16_t *L = V.dn_src + ro, *B = V.dn_a + ro;
                        la[j] = L[xa];
                        lb[j] = L[xb];
                        ba[j] = B[xa];
                        bb[j] = B[xb];
                        if (lane < 2) {
                            lc[j] = L[xc];
                            bc[j] = B[xc];
                        }
                    }
                }
#pragma unroll
                for (int j = 0; j < RB; ++j) {
                    const int rr = r0 + NW * j;
                    if (rr < NROW) {
                        const uint32_t da = la[j] > ba[j] ? la[j] - ba[j] : 0u;
                        const uint32_t db = lb[j] > bb[j] ? lb[j] - bb[j] : 0u;
                        reinterpret_cast<uint32_t *>(ds + rr * SXW)[lane] = da | (db << 16);
                        if (lane < 2) ds[rr * SXW + 64 + lane] = (uint16_t)(lc[j] > bc[j] ? lc[j] - bc[j] : 0u);
                    }
                }
            }
        }
        __syncthreads();
        const int x = x0 + 2 * tx, y = y0 + ty;
        if (x >= X || y >= Y) continue;
        // the pair's 3x3 neighbourhood in plane c: shared x indices 2 tx + a
        // and 2 tx + 1 + a for a = 0, 1, 2, i.e. word tx, the middle of words
        // tx and tx + 1, and word tx + 1 of each row
        auto plane = [&](int c, uint32_t *srt) {
            uint32_t v[9];
#pragma unroll
            for (int b = 0; b < 3; ++b) {
                const uint32_t *row = reinterpret_cast<const uint32_t *>(&d[c][ty + b][0]);
                const uint32_t w0 = row[tx], w1 = row[tx + 1];
                v[3 * b] = w0;
                v[3 * b + 1] = __byte_perm(w0, w1, 0x5432);
                v[3 * b + 2] = w1;
            }
            sort9x2(v, srt);
        };
        const bool two = x + 1 < X, wide = two && (X & 1) == 0;  // 32-bit stores at even x of even rows
        uint32_t s0[9], s1[9], s2[9];
        plane(0, s0);
        plane(1, s1);
        for (int k = 0; k < MED_TZ && z0 + k < Z; ++k) {
            plane(k + 2, s2);
            const uint32_t m = median3x9x2(s0, s1, s2);
            uint16_t *o = V.dn_out + (size_t)x + (size_t)X * ((size_t)y + (size_t)Y * (z0 + k));
            if (wide) {
                *reinterpret_cast<uint32_t *>(o) = m;
            } else {
                o[0] = (uint16_t)(m & 0xFFFFu);
                if (two) o[1] = (uint16_t)(m >> 16);
            }
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                s0[i] = s1[i];
                s1[i] = s2[i];
            }
        }
    }
}

// ----------------------------------------------------------------------------
// Closing of the foreground with a binary ball (Segmentation section): the
// ball of radius rho holds the offsets with dx^2 + dy^2 + dz^2 <= rho^2.  It
// is split into rows: for each (dy, dz) with dy^2 + dz^2 <= rho^2 an x-run of
// half-width floor(sqrt(rho^2 - dy^2 - dz^2)).  Dilation (OR) fills the
// extended mask, which covers rho rows and planes of padding and one word
// of padding on each side of every row; erosion (AND) reads it back for the
// rows of the volume, so every ball around a voxel stays inside the
// extended mask -- the closing of the padded volume, cut to the volume.
// ----------------------------------------------------------------------------

// x-run half-widths of the balls, per radius and row offset (-1 outside the
// ball), filled once per block: rx^2 <= rho^2 - dy^2 - dz^2 < (rx + 1)^2.
constexpr int CL_SPAN = 2 * CL_MAX_R + 1;

struct BallTable {
    int8_t rx[CL_MAX_R + 1][CL_SPAN][CL_SPAN];
    __device__ __forceinline__ void fill() {
        for (int i = threadIdx.x; i < (CL_MAX_R + 1) * CL_SPAN * CL_SPAN; i += blockDim.x) {
            const int rho = i / (CL_SPAN * CL_SPAN), dy = (i / CL_SPAN) % CL_SPAN - CL_MAX_R;
            const int dz = i % CL_SPAN - CL_MAX_R;
            const int q = rho * rho - dy * dy - dz * dz;
            int r = -1;
            if (q >= 0)
                while ((r + 1) * (r + 1) <= q) ++r;
            (&rx[0][0][0])[i] = (int8_t)r;
        }
        __syncthreads();
    }
    __device__ __forceinline__ int get(int rho, int dy, int dz) const {
        return rx[rho][dy + CL_MAX_R][dz + CL_MAX_R];
    }
};

// OR (DIL) or AND of the 2 rx + 1 x-shifts of a bit word w1 with its
// neighbours w0 (lower x) and w2 (higher x).
template <bool DIL>
__device__ __forceinline__ uint32_t smear(uint32_t w0, uint32_t w1, uint32_t w2, int rx) {
    uint32_t acc = w1;
    for (int k = 1; k <= rx; ++k) {
        const uint32_t up = __funnelshift_r(w1, w2, k);    // bit b <- x + k
        const uint32_t dn = __funnelshift_l(w0, w1, k);    // bit b <- x - k
        acc = DIL ? (acc | up | dn) : (acc & up & dn);
    }
    return acc;
}

// One thread per word of the extended mask of every closing volume.
__global__ void __launch_bounds__(256) k_dilate(const BatchHdr *__restrict__ h) {
    __shared__ VolIndex<&VolDev::cl_base> VI;
    __shared__ BallTable BT;
    VI.load(h);
    BT.fill();
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t it = blockIdx.x * blockDim.x + threadIdx.x; it < h->cl_items; it += stride) {
        const VolDev &V = h->vol[VI.find(h, it)];
        const uint32_t li = it - V.cl_base;
        const int rho = (int)V.cl_r, W = (int)V.W, WE = W + 2, Y = (int)V.Y, Z = (int)V.Z;
        const int YE = Y + 2 * rho;
        const int we = (int)(li % (uint32_t)WE), er = (int)(li / (uint32_t)WE);
        const int y = er % YE - rho, z = er / YE - rho;
        const int w = we - 1;  // word of the row, -1 and W are the padding words
        uint32_t acc = 0;
        for (int dz = -rho; dz <= rho; ++dz) {
            const int zz = z + dz;
            if (zz < 0 || zz >= Z) continue;
            for (int dy = -rho; dy <= rho; ++dy) {
                const int rx = BT.get(rho, dy, dz), yy = y + dy;
                if (rx < 0 || yy < 0 || yy >= Y) continue;
                const uint32_t *row = V.mask + ((size_t)zz * Y + yy) * W;
                const uint32_t a0 = (w >= 1 && w - 1 < W) ? row[w - 1] : 0u;
                const uint32_t a1 = (w >= 0 && w < W) ? row[w] : 0u;
                const uint32_t a2 = (w + 1 >= 0 && w + 1 < W) ? row[w + 1] : 0u;
                acc |= smear<true>(a0, a1, a2, rx);
            }
        }
        V.cl_ext[(size_t)er * WE + we] = acc;
    }
}

// One block per row tile, one warp per row: the eroded row, its run starts
// and the tile's run total (the closed foreground replaces the threshold
// mask and the run counts of k_threshold_runs).
__global__ void __launch_bounds__(ROW_TILE) k_erode(const BatchHdr *__restrict__ h) {
    __shared__ VolIndex<&VolDev::rt_base> VI;
    __shared__ BallTable BT;
    __shared__ uint32_t wsum[ROW_TILE / 32];
    VI.load(h);
    BT.fill();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (uint32_t rt = blockIdx.x; rt < h->nrowtiles; rt += gridDim.x) {
        const VolDev &V = h->vol[VI.find(h, rt)];
        if (V.cl_r == 0) continue;  // the same for the whole block
        const uint32_t lt = rt - V.rt_base, row0 = lt * h->row_tile;
        const uint32_t nrows = min(h->row_tile, V.rows - row0);
        const int rho = (int)V.cl_r, W = (int)V.W, WE = W + 2, Y = (int)V.Y;
        const int YE = Y + 2 * rho;
        // rows of at most 16 words share a warp: segments of seg lanes
        // (a power of two >= W), one row per segment
        int seg = 32;
        while (seg / 2 >= W && seg > 1) seg /= 2;
        const int per = 32 / seg, sub = lane / seg, sl = lane % seg;
        uint32_t wtot = 0;
        for (uint32_t rb = (uint32_t)warp * per; rb < nrows; rb += (ROW_TILE / 32) * per) {
            const uint32_t rr = rb + (uint32_t)sub;
            const bool live = rr < nrows;
            const uint32_t row = row0 + (live ? rr : 0u);
            const int y = (int)(row % (uint32_t)Y), z = (int)(row / (uint32_t)Y);
            uint32_t carry = 0, cnt = 0;
            for (int w0 = 0; w0 < W; w0 += seg) {
                const int w = w0 + sl;
                uint32_t acc = 0u;
                if (live && w < W) {
                    acc = 0xFFFFFFFFu;
                    for (int dz = -rho; dz <= rho; ++dz)
                        for (int dy = -rho; dy <= rho; ++dy) {
                            const int rx = BT.get(rho, dy, dz);
                            if (rx < 0) continue;
                            const uint32_t *e = V.cl_ext + ((size_t)(z + dz + rho) * YE + (y + dy + rho)) * WE + (w + 1);
                            acc &= smear<false>(e[-1], e[0], e[1], rx);
                        }
                    const uint32_t x0 = 32u * (uint32_t)w;
                    if (x0 + 32u > V.X) acc &= (1u << (V.X - x0)) - 1u;  // no bits past the row
                    V.mask[(size_t)row * W + w] = acc;
                }
                const uint32_t prev = __shfl_up_sync(FULL, acc, 1, seg);
                const uint32_t left = sl == 0 ? carry : (prev >> 31);
                if (live && w < W) cnt += __popc(acc & ~((acc << 1) | left));
                carry = __shfl_sync(FULL, acc, seg - 1, seg) >> 31;
            }
            for (int o = seg / 2; o > 0; o >>= 1) cnt += __shfl_xor_sync(FULL, cnt, o);
            if (live && sl == 0) {
                V.rowoff[row] = cnt;
                wtot += cnt;
            }
        }
        for (int o = 16; o > 0; o >>= 1) wtot += __shfl_xor_sync(FULL, wtot, o);
        if (lane == 0) wsum[warp] = wtot;
        __syncthreads();
        if (threadIdx.x == 0) {
            uint32_t tot = 0;
            for (int i = 0; i < ROW_TILE / 32; ++i) tot += wsum[i];
            V.tsum[lt] = tot;
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// MRF vessel denoise (Background Noise Removal, Eqs. 2-3).  Every step moves
// each voxel by Delta towards the majority of its six face neighbours (Eq. 3:
// a neighbour votes +1 if higher, -1 if lower, 0 if equal or outside the
// volume; the paired terms of the printed equation read as the two
// neighbours' votes), all voxels at once, clamped to [0, 65535].  A step is
// kept while the root-mean-square difference from the input stays within the
// noise level sigma estimated from the input with a Laplacian mask (Eq. 2).
// Delta is the smallest gap between two distinct input levels.  One tile is
// MRF_TILE octets (8 x-consecutive voxels of a row) of one volume.

__device__ __forceinline__ int mrf_sgn(int32_t d) { return (d > 0) - (d < 0); }

// Block sum of one uint64 per thread (MRF_TILE threads); thread 0 gets it.
__device__ __forceinline__ unsigned long long mrf_block_sum(unsigned long long v, unsigned long long *red) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    unsigned long long s = 0;
    if (threadIdx.x == 0)
        for (int i = 0; i < MRF_TILE / 32; ++i) s += red[i];
    __syncthreads();
    return s;
}

// The 8 voxels of an octet at p (16-byte aligned when `vec`), else the first
// n of them.
__device__ __forceinline__ void mrf_load8(const uint16_t *p, bool vec, uint32_t n, int32_t *v) {
    if (vec) {
        const uint4 q = *reinterpret_cast<const uint4 *>(p);
        const uint32_t w[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            v[2 * j] = (int32_t)(w[j] & 0xFFFFu);
            v[2 * j + 1] = (int32_t)(w[j] >> 16);
        }
    } else {
#pragma unroll
        for (int j = 0; j < 8; ++j) v[j] = (uint32_t)j < n ? (int32_t)p[j] : 0;
    }
}

// Levels present in the input and the noise estimate's sum S over every
// z-plane's interior of |[1 -2 1; -2 4 -2; 1 -2 1] * I| (Immerkaer's mask),
// added into the volume's ST_MRF_E words.  The levels collect in a shared
// bitmap, merged into the volume's (nonzero words only) when the block moves
// to another volume and at its end.
__global__ void __launch_bounds__(MRF_TILE) k_mrf_stats(const BatchHdr *__restrict__ h) {
    __shared__ unsigned long long red[MRF_TILE / 32];
    __shared__ uint32_t sbits[2048];
    for (int i = threadIdx.x; i < 2048; i += MRF_TILE) sbits[i] = 0u;
    // a contiguous range of tiles per block, so it meets few volumes
    const uint32_t T = h->mrf_tiles, G = gridDim.x;
    const uint32_t tb = (uint32_t)(((uint64_t)T * blockIdx.x) / G);
    const uint32_t te = (uint32_t)(((uint64_t)T * (blockIdx.x + 1)) / G);
    uint32_t vi = 0;
    while (vi + 1 < h->nvol && tb >= h->vol[vi + 1].mrf_tbase) ++vi;
    unsigned long long s = 0;
    __syncthreads();
    auto flush = [&]() {  // this block's levels and sum for volume vi
        const unsigned long long tot = mrf_block_sum(s, red);  // (barriers order sbits too)
        s = 0;
        const VolDev &V = h->vol[vi];
        if (threadIdx.x == 0 && tot) atomicAdd(reinterpret_cast<unsigned long long *>(V.stat + ST_MRF_E), tot);
        for (int i = threadIdx.x; i < 2048; i += MRF_TILE) {
            const uint32_t w = sbits[i];
            if (w) {
                atomicOr(V.mrf_bits + i, w);
                sbits[i] = 0u;
            }
        }
        __syncthreads();
    };
    for (uint32_t t = tb; t < te; ++t) {
        if (vi + 1 < h->nvol && t >= h->vol[vi + 1].mrf_tbase) {
            flush();
            do ++vi; while (vi + 1 < h->nvol && t >= h->vol[vi + 1].mrf_tbase);
        }
        const VolDev &V = h->vol[vi];
        const uint32_t X = V.X, Y = V.Y, OX = (X + 7) >> 3;
        const uint32_t o = (t - V.mrf_tbase) * MRF_TILE + threadIdx.x;
        if (o >= V.rows * OX) continue;
        const uint32_t row = o / OX, x0 = 8 * (o % OX), y = row % Y;
        const uint16_t *r0 = V.mrf_in + (size_t)row * X + x0;
        const uint32_t n = min(8u, X - x0);
        const bool vec = n == 8u && V.mrf_vec;  // (mrf_buf is always aligned)
        int32_t c[8];
        mrf_load8(r0, vec, n, c);
        for (uint32_t j = 0; j < n; ++j) {  // most levels are already marked: test before setting
            const uint32_t bit = 1u << (c[j] & 31);
            if (!(sbits[c[j] >> 5] & bit)) atomicOr(sbits + (c[j] >> 5), bit);
        }
        if (y >= 1 && y + 1 < Y) {
            int32_t a[8], b[8];
            mrf_load8(r0 - X, vec, n, a);
            mrf_load8(r0 + X, vec, n, b);
            // second differences along x of the three rows, then along y
            int32_t l0 = 0, la = 0, lb = 0, r0v = 0, ra = 0, rb = 0;
            if (x0 > 0) {
                l0 = r0[-1];
                la = r0[-1 - (int)X];
                lb = r0[-1 + (int)X];
            }
            if (x0 + 8 < X) {
                r0v = r0[8];
                ra = r0[8 - (int)X];
                rb = r0[8 + (int)X];
            }
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const uint32_t x = x0 + j;
                if (x < 1 || x + 1 >= X || (uint32_t)j >= n) continue;
                const int32_t cl = j > 0 ? c[j - 1] : l0, cr = j < 7 ? c[j + 1] : r0v;
                const int32_t al = j > 0 ? a[j - 1] : la, ar = j < 7 ? a[j + 1] : ra;
                const int32_t bl = j > 0 ? b[j - 1] : lb, br = j < 7 ? b[j + 1] : rb;
                const int32_t da = al - 2 * a[j] + ar, dc = cl - 2 * c[j] + cr, db = bl - 2 * b[j] + br;
                s += (unsigned long long)abs(da - 2 * dc + db);
            }
        }
    }
    if (tb < te) flush();
}

// One warp per MRF volume: Delta from the levels present, and the bound
// N sigma^2 of Eq. 2 from S in binary64 with every operation rounded as
// written (sigma = (sqrt(pi/2) S) / (6 M), bound = (N sigma) sigma, M the
// number of plane-interior voxels).  Fewer than two levels: nothing to do,
// the input is kept.
__global__ void k_mrf_prep(const BatchHdr *__restrict__ h) {
    const int lane = threadIdx.x & 31;
    for (uint32_t v = blockIdx.x; v < h->nvol; v += gridDim.x) {
        const VolDev &V = h->vol[v];
        if (V.mrf_max == 0) continue;
        // lane l scans levels [2048 l, 2048 l + 2048)
        int first = -1, last = -1;
        uint32_t gap = 0xFFFFFFFFu;
        for (int i = 0; i < 64; ++i) {
            const uint32_t w = V.mrf_bits[64 * lane + i];
            if (!w) continue;
            const int pos0 = 32 * (64 * lane + i);
            const int lo = pos0 + __ffs(w) - 1, hi = pos0 + 31 - __clz(w);
            if (first < 0) first = lo;
            if (last >= 0) gap = min(gap, (uint32_t)(lo - last));
            int prev = lo;
            for (uint32_t m = w & (w - 1u); m && gap > 1u; m &= m - 1u) {
                const int p = pos0 + __ffs(m) - 1;
                gap = min(gap, (uint32_t)(p - prev));
                prev = p;
            }
            last = hi;
        }
        int gl = -1;  // last level seen over the lanes before
        uint32_t delta = 0xFFFFFFFFu;
        for (int l = 0; l < 32; ++l) {
            const int f = __shfl_sync(FULL, first, l), la = __shfl_sync(FULL, last, l);
            const uint32_t g = __shfl_sync(FULL, gap, l);
            if (f < 0) continue;
            if (gl >= 0) delta = min(delta, (uint32_t)(f - gl));
            delta = min(delta, g);
            gl = la;
        }
        if (lane == 0) {
            uint32_t *st = V.stat;
            unsigned long long *e = reinterpret_cast<unsigned long long *>(st + ST_MRF_E);
            const unsigned long long s = *e;
            const unsigned long long m =
                (unsigned long long)V.Z * (V.X >= 2 ? V.X - 2 : 0) * (V.Y >= 2 ? V.Y - 2 : 0);
            const unsigned long long n = (unsigned long long)V.X * V.Y * V.Z;
            double limit = 0.0;
            if (m) {
                const double half_pi = 3.14159265358979323846 / 2.0;
                const double sigma = __ddiv_rn(__dmul_rn(__dsqrt_rn(half_pi), __ull2double_rn(s)),
                                               __dmul_rn(6.0, __ull2double_rn(m)));
                limit = __dmul_rn(__dmul_rn(__ull2double_rn(n), sigma), sigma);
            }
            *reinterpret_cast<double *>(st + ST_MRF_LIMIT) = limit;
            *e = 0ull;
            st[ST_MRF_CNT] = 0u;
            st[ST_MRF_CHG] = 0u;
            st[ST_MRF_STEPS] = 0u;
            st[ST_MRF_SEL] = 0u;
            st[ST_MRF_DELTA] = delta == 0xFFFFFFFFu ? 0u : delta;
            st[ST_MRF_DONE] = delta == 0xFFFFFFFFu ? 1u : 0u;
        }
    }
}

// Octet helpers of the step kernel: 8 voxels packed two to a word.
__device__ __forceinline__ uint4 mrf_oct(const uint16_t *p, bool vec, uint32_t n) {
    if (vec) return *reinterpret_cast<const uint4 *>(p);
    uint32_t w[4] = {0u, 0u, 0u, 0u};
    for (uint32_t j = 0; j < n; ++j) w[j >> 1] |= (uint32_t)p[j] << (16 * (j & 1));
    return make_uint4(w[0], w[1], w[2], w[3]);
}
__device__ __forceinline__ void mrf_unpack(uint4 q, int32_t *v) {
    const uint32_t w[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        v[2 * j] = (int32_t)(w[j] & 0xFFFFu);
        v[2 * j + 1] = (int32_t)(w[j] >> 16);
    }
}

// Eq. 3 on one octet c (n voxels valid; FULL: n = 8): left / right are the
// x neighbours of its end voxels (-1: outside the volume), ym, yp, zm, zp
// the octets of the neighbouring rows and planes (null: outside).  Adds the
// octet's sum (I^{n+1} - I^0)^2 to e and whether it changed to `changed`;
// returns the new octet (voxels past n are zero).
template <bool FULL>
__device__ __forceinline__ uint4 mrf_update(uint4 c, int32_t left, int32_t right, const uint4 *ym, const uint4 *yp,
                                            const uint4 *zm, const uint4 *zp, uint4 org, int32_t delta, uint32_t n,
                                            unsigned long long &e, bool &changed) {
    int32_t v[8], nb[8];
    int votes[8];
    mrf_unpack(c, v);
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const int32_t l = k > 0 ? v[k - 1] : left;
        const int32_t r = k < 7 ? (FULL || (uint32_t)(k + 1) < n ? v[k + 1] : -1) : right;
        votes[k] = (l >= 0 ? mrf_sgn(l - v[k]) : 0) + (r >= 0 ? mrf_sgn(r - v[k]) : 0);
    }
    const uint4 *rows[4] = {ym, yp, zm, zp};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        if (!rows[q]) continue;
        mrf_unpack(*rows[q], nb);
#pragma unroll
        for (int k = 0; k < 8; ++k) votes[k] += mrf_sgn(nb[k] - v[k]);
    }
    mrf_unpack(org, nb);
    uint32_t w[4] = {0u, 0u, 0u, 0u};
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        if (!FULL && (uint32_t)k >= n) continue;
        const int32_t nv = min(max(v[k] + delta * mrf_sgn(votes[k]), 0), 65535);
        const uint32_t d = (uint32_t)abs(nv - nb[k]);
        e += (unsigned long long)d * d;
        changed |= nv != v[k];
        w[k >> 1] |= (uint32_t)nv << (16 * (k & 1));
    }
    return make_uint4(w[0], w[1], w[2], w[3]);
}

__device__ __forceinline__ int32_t mrf_clamp1(int32_t d) { return min(max(d, -1), 1); }  // sgn of an integer

// Eq. 3 on a whole octet with comparisons shared where two voxels compare
// with each other: inside the octet each x pair is compared once, and along
// z the comparison of a voxel with the plane above is, negated, the next
// plane's comparison with the plane below (za: in, the previous plane's
// comparisons with its plane above, or 0 at z = 0; out, this plane's).
__device__ __forceinline__ uint4 mrf_update_full(uint4 c, int32_t left, int32_t right, const uint4 *ym,
                                                 const uint4 *yp, const uint4 *zp, int32_t *za, uint4 org,
                                                 int32_t delta, unsigned long long &e, bool &changed) {
    int32_t v[8], nb[8], votes[8];
    mrf_unpack(c, v);
    int32_t px[7];
#pragma unroll
    for (int k = 0; k < 7; ++k) px[k] = mrf_clamp1(v[k + 1] - v[k]);
    votes[0] = (left >= 0 ? mrf_clamp1(left - v[0]) : 0) + px[0] - za[0];
#pragma unroll
    for (int k = 1; k < 7; ++k) votes[k] = px[k] - px[k - 1] - za[k];
    votes[7] = (right >= 0 ? mrf_clamp1(right - v[7]) : 0) - px[6] - za[7];
    if (ym) {
        mrf_unpack(*ym, nb);
#pragma unroll
        for (int k = 0; k < 8; ++k) votes[k] += mrf_clamp1(nb[k] - v[k]);
    }
    if (yp) {
        mrf_unpack(*yp, nb);
#pragma unroll
        for (int k = 0; k < 8; ++k) votes[k] += mrf_clamp1(nb[k] - v[k]);
    }
    if (zp) {
        mrf_unpack(*zp, nb);
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            za[k] = mrf_clamp1(nb[k] - v[k]);
            votes[k] += za[k];
        }
    } else {
#pragma unroll
        for (int k = 0; k < 8; ++k) za[k] = 0;
    }
    mrf_unpack(org, nb);
    uint32_t w[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int32_t a = min(max(v[2 * j] + delta * mrf_clamp1(votes[2 * j]), 0), 65535);
        const int32_t b = min(max(v[2 * j + 1] + delta * mrf_clamp1(votes[2 * j + 1]), 0), 65535);
        const uint32_t da = (uint32_t)abs(a - nb[2 * j]), db = (uint32_t)abs(b - nb[2 * j + 1]);
        e += (unsigned long long)da * da + (unsigned long long)db * db;
        w[j] = (uint32_t)a | (uint32_t)b << 16;
    }
    const uint4 r = make_uint4(w[0], w[1], w[2], w[3]);
    changed |= ((r.x ^ c.x) | (r.y ^ c.y) | (r.z ^ c.z) | (r.w ^ c.w)) != 0u;
    return r;
}

// Step `it` of every MRF volume not yet stopped: reads mrf_in (it = 0) or
// mrf_buf[it & 1], writes mrf_buf[(it + 1) & 1], and adds the step's
// sum (I^{it+1} - I^0)^2 and whether anything changed to the volume's
// status words.  A tile is MRF_TX octets x MRF_TY rows walked down z: each
// thread keeps its octet of planes z - 1, z, z + 1 in registers, the rows
// y - 1 and y + 1 come from the neighbouring threads through shared memory
// and the x neighbours by shuffles, so every voxel of the current image is
// read from memory about once per step.  Blocks take contiguous tile ranges
// and flush their sums once per volume; the block whose flush completes a
// volume decides: stop at a step that changes nothing or strays too far
// (keeping I^it), or at the step limit; when stopping it points the volume's
// raw input for the smoothing (in the device copy of the batch descriptor)
// at the kept image.
__global__ void __launch_bounds__(MRF_TX * MRF_TY, 3) k_mrf_step(const BatchHdr *__restrict__ h, uint32_t it) {
    __shared__ uint4 srow[MRF_TY + 2][MRF_TX];  // plane z, rows y0 - 1 .. y0 + MRF_TY
    __shared__ unsigned long long red[MRF_TX * MRF_TY / 32];
    __shared__ uint32_t chg_any;  // some voxel of the block's tiles changed (0 between volumes)
    if (threadIdx.x == 0) chg_any = 0u;
    const int lx = threadIdx.x & 31, ly = threadIdx.x >> 5;
    const uint32_t T = h->mrf_ctiles, G = gridDim.x;
    const uint32_t tb = (uint32_t)(((uint64_t)T * blockIdx.x) / G);
    const uint32_t te = (uint32_t)(((uint64_t)T * (blockIdx.x + 1)) / G);
    uint32_t vi = 0;
    while (vi + 1 < h->nvol && tb >= h->vol[vi + 1].mrf_cbase) ++vi;
    unsigned long long e = 0;
    bool changed = false;
    uint32_t ntile = 0;
    __syncthreads();
    auto flush = [&]() {  // this block's tiles of volume vi
        if (changed) chg_any = 1u;  // benign race: every writer stores 1
        const unsigned long long sum = mrf_block_sum(e, red);  // (its barriers also order chg_any)
        const VolDev &V = h->vol[vi];
        uint32_t *st = V.stat;
        if (threadIdx.x == 0 && ntile) {
            unsigned long long *E = reinterpret_cast<unsigned long long *>(st + ST_MRF_E);
            if (sum) atomicAdd(E, sum);
            if (chg_any) atomicOr(st + ST_MRF_CHG, 1u);
            __threadfence();
            if (atomicAdd(st + ST_MRF_CNT, ntile) + ntile == V.mrf_ctiles) {
                // every tile of this volume is in: decide
                __threadfence();
                const unsigned long long tot = atomicAdd(E, 0ull);
                const uint32_t chg = atomicAdd(st + ST_MRF_CHG, 0u);
                const double limit = *reinterpret_cast<const volatile double *>(st + ST_MRF_LIMIT);
                uint32_t sel, steps, done;
                if (!chg || __ull2double_rn(tot) > limit) {
                    done = 1u;  // keep I^it
                    steps = it;
                    sel = it == 0 ? 0u : 1u + (it & 1u);
                } else {
                    steps = it + 1u;
                    sel = 1u + ((it + 1u) & 1u);
                    done = it + 1u >= V.mrf_max ? 1u : 0u;
                }
                st[ST_MRF_STEPS] = steps;
                st[ST_MRF_SEL] = sel;
                st[ST_MRF_DONE] = done;
                if (done) {
                    // the smoothing reads the kept image: the descriptor is
                    // the device copy made for this launch sequence
                    VolDev &W = const_cast<VolDev &>(V);
                    W.raw = sel == 0 ? V.mrf_in : V.mrf_buf[sel - 1u];
                }
                *E = 0ull;
                st[ST_MRF_CHG] = 0u;
                st[ST_MRF_CNT] = 0u;
            }
        }
        if (threadIdx.x == 0) chg_any = 0u;
        e = 0;
        changed = false;
        ntile = 0;
        __syncthreads();
    };
    for (uint32_t t = tb; t < te; ++t) {
        if (vi + 1 < h->nvol && t >= h->vol[vi + 1].mrf_cbase) {
            flush();
            do ++vi; while (vi + 1 < h->nvol && t >= h->vol[vi + 1].mrf_cbase);
        }
        const VolDev &V = h->vol[vi];
        // volumes that stopped (or never started) are left alone; the flag
        // was set by an earlier launch, so it is the same for every thread
        if (it >= V.mrf_max || V.stat[ST_MRF_DONE]) continue;
        ++ntile;
        const uint32_t X = V.X, Y = V.Y, Z = V.Z, OX = (X + 7) >> 3;
        const uint32_t ntx = (OX + MRF_TX - 1) / MRF_TX;
        const uint32_t lt = t - V.mrf_cbase;
        const uint32_t ox = (lt % ntx) * MRF_TX + lx, y0 = (lt / ntx) * MRF_TY, y = y0 + ly;
        const uint32_t x0 = 8 * ox;
        const bool live = ox < OX && y < Y;
        const uint32_t n = live ? min(8u, X - x0) : 0u;
        const bool vec = n == 8u && V.mrf_vec;  // (mrf_buf is always aligned)
        const size_t plane = (size_t)X * Y;
        const uint16_t *cur = it == 0 ? V.mrf_in : V.mrf_buf[it & 1u];
        uint16_t *nxt = V.mrf_buf[(it + 1u) & 1u];
        const int32_t delta = (int32_t)V.stat[ST_MRF_DELTA];
        const size_t off = (size_t)y * X + x0;  // this octet in plane 0
        // halo rows of the tile (loaded by the first and last warp)
        const bool hrow = (ly == 0 && y0 > 0) || (ly == MRF_TY - 1 && y0 + MRF_TY < Y);
        const uint32_t hy = ly == 0 ? y0 - 1 : y0 + MRF_TY;
        const uint32_t hn = (hrow && ox < OX) ? min(8u, X - x0) : 0u;
        const size_t hoff = (size_t)hy * X + x0;
        uint4 below = make_uint4(0, 0, 0, 0), c = below, above = below;
        int32_t za[8] = {0, 0, 0, 0, 0, 0, 0, 0};  // full octets: comparisons with the plane above
        if (n) c = mrf_oct(cur + off, vec, n);
        if (n && Z > 1) above = mrf_oct(cur + plane + off, vec, n);
        for (uint32_t z = 0; z < Z; ++z) {
            const size_t zo = (size_t)z * plane;
            srow[ly + 1][lx] = c;
            if (hn) srow[ly == 0 ? 0 : MRF_TY + 1][lx] = mrf_oct(cur + zo + hoff, hn == 8u && V.mrf_vec, hn);
            // x neighbours: the next octets of the row, or memory at the tile's ends
            const uint32_t lnb = __shfl_up_sync(FULL, c.w >> 16, 1);
            const uint32_t rnb = __shfl_down_sync(FULL, c.x & 0xFFFFu, 1);
            __syncthreads();
            if (n) {
                const int32_t left = x0 == 0 ? -1 : (lx > 0 ? (int32_t)lnb : (int32_t)cur[zo + off - 1]);
                const int32_t right = x0 + 8 >= X ? -1 : (lx < 31 ? (int32_t)rnb : (int32_t)cur[zo + off + 8]);
                const uint4 *ym = y > 0 ? &srow[ly][lx] : nullptr;
                const uint4 *yp = y + 1 < Y ? &srow[ly + 2][lx] : nullptr;
                const uint4 org = mrf_oct(V.mrf_in + zo + off, vec, n);
                uint4 res;
                if (n == 8u)
                    res = mrf_update_full(c, left, right, ym, yp, z + 1 < Z ? &above : nullptr, za, org, delta, e,
                                          changed);
                else
                    res = mrf_update<false>(c, left, right, ym, yp, z > 0 ? &below : nullptr,
                                            z + 1 < Z ? &above : nullptr, org, delta, n, e, changed);
                uint16_t *dst = nxt + zo + off;
                if (vec) {
                    *reinterpret_cast<uint4 *>(dst) = res;
                } else {
                    const uint32_t w[4] = {res.x, res.y, res.z, res.w};
                    for (uint32_t k = 0; k < n; ++k) dst[k] = (uint16_t)(w[k >> 1] >> (16 * (k & 1)));
                }
            }
            below = c;
            c = above;
            if (n && z + 2 < Z) above = mrf_oct(cur + zo + 2 * plane + off, vec, n);
            __syncthreads();  // srow is rewritten for the next plane
        }
    }
    if (tb < te) flush();
}

// ---------------------------------------------------------------------------
// Distance map of the final foreground (Segmentation section: for every voxel
// the distance to the nearest foreground voxel of the vessel channel).  The
// weighted squared Euclidean distance min over foreground voxels p of
// wx (x - px)^2 + wy (y - py)^2 + wz (z - pz)^2 is separable: a pass along x
// gives, per row, the distance to the row's nearest foreground voxel; each
// following pass along an axis a takes, per line, the lower envelope
// out(q) = min_i f(i) + w_a (q - i)^2 of the previous pass's values f (the
// lower envelope of parabolas of Felzenszwalb and Huttenlocher, "Distance
// transforms of sampled functions").  Parabola i is A(i) - 2 w q i + w q^2
// with A(i) = f(i) + w i^2, so the parabolas lowest somewhere are the
// vertices of the lower convex hull of the points (i, A(i)).  Every
// comparison is exact in integers, so the map equals the brute-force minimum.
// Submission checks wx (X-1)^2 + wy (Y-1)^2 + wz (Z-1)^2 < 2^32 - 1, and f of
// a pass is at most the sum of the earlier axes' terms, so A(i) and every
// value f(i) + w (q - i)^2 at positions inside the volume fit in 32 bits.
//
// Paths: k_dist_xy (x and y passes fused, lines along y in shared memory)
// then k_dist_z (z pass in shared memory); for lines too long for a block,
// k_dist_x, k_dist_line<1> and k_dist_line<2> keep their stacks in global
// memory.

constexpr uint32_t DT_INF = 0xFFFFFFFFu;  // no foreground reachable
constexpr uint16_t DX_NONE = 0xFFFFu;     // row without foreground (k_dist_xy)

// Flat work index of DtKernel K over the batch (as VolIndex).
template <int K>
struct DtIndex {
    uint32_t base[SMEM_VOLS];
    __device__ __forceinline__ void load(const BatchHdr *__restrict__ h) {
        if (h->nvol <= SMEM_VOLS)
            for (uint32_t i = threadIdx.x; i < h->nvol; i += blockDim.x) base[i] = h->vol[i].dt_base[K];
        __syncthreads();
    }
    __device__ __forceinline__ uint32_t find(const BatchHdr *__restrict__ h, uint32_t t) const {
        const uint32_t nv = h->nvol;
        uint32_t lo = 0, hi = nv;
        while (hi - lo > 1) {
            const uint32_t mid = (lo + hi) >> 1;
            const uint32_t b = nv <= SMEM_VOLS ? base[mid] : h->vol[mid].dt_base[K];
            if (b <= t) lo = mid; else hi = mid;
        }
        return lo;
    }
};

// Point (pm, am) lies on or above the segment from (pa, aa) to (pc, ac),
// pa < pm < pc: parabola pm is nowhere strictly below both others and leaves
// the lower envelope.  In the form ac (pm - pa) + aa (pc - pm) <= am (pc - pa)
// every product is of two unsigned 32-bit numbers (A < 2^32, positions
// < 2^16), so each side stays below 2^49.
__device__ __forceinline__ bool dt_covered(uint32_t pa, uint32_t aa, uint32_t pm, uint32_t am, uint32_t pc,
                                           uint32_t ac) {
    const uint64_t lhs = (uint64_t)ac * (pm - pa) + (uint64_t)aa * (pc - pm);
    return lhs <= (uint64_t)am * (pc - pa);
}

__device__ __forceinline__ uint32_t dt_sq(int d) {
    const uint32_t u = (uint32_t)abs(d);
    return u * u;
}

// Long-line path, x pass.  One warp per mask row of every such volume:
// g(x) = wx d^2 with d the distance along the row to its nearest foreground
// voxel, DT_INF when the row has none.  Lane l of a step writes
// x = 32 w + l, so each store is 128 contiguous bytes.
__global__ void __launch_bounds__(256) k_dist_x(const BatchHdr *__restrict__ h) {
    __shared__ DtIndex<DT_X> VI;
    VI.load(h);
    const int lane = threadIdx.x & 31;
    const uint32_t nw = blockDim.x >> 5;
    for (uint32_t it = blockIdx.x * nw + (threadIdx.x >> 5); it < h->dt_items[DT_X]; it += gridDim.x * nw) {
        const VolDev &V = h->vol[VI.find(h, it)];
        const uint32_t row = it - V.dt_base[DT_X];
        const int W = (int)V.W, X = (int)V.X;
        const uint32_t wx = V.dt_w[0];
        const uint32_t *m = V.mask + (size_t)row * W;
        uint32_t *g = V.dt_g + (size_t)row * X;
        int left = -1;  // last foreground x before the current chunk of 32 words
        for (int c0 = 0; c0 < W; c0 += 32) {
            const int w = c0 + lane;
            const uint32_t word = w < W ? m[w] : 0u;
            // first foreground x after this chunk (INT_MAX: none)
            int right = INT_MAX;
            for (int c1 = c0 + 32; c1 < W; c1 += 32) {
                const uint32_t wd = c1 + lane < W ? m[c1 + lane] : 0u;
                const uint32_t b = __ballot_sync(FULL, wd != 0u);
                if (b) {
                    const int l = __ffs(b) - 1;
                    right = 32 * (c1 + l) + __ffs(__shfl_sync(FULL, wd, l)) - 1;
                    break;
                }
            }
            // last foreground x at or before word w; first one at or after it
            int pre = word ? 32 * w + 31 - __clz(word) : -1;
            int suf = word ? 32 * w + __ffs(word) - 1 : INT_MAX;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int a = __shfl_up_sync(FULL, pre, o);
                const int b = __shfl_down_sync(FULL, suf, o);
                if (lane >= o) pre = max(pre, a);
                if (lane + o < 32) suf = min(suf, b);
            }
            int lprev = __shfl_up_sync(FULL, pre, 1);
            int rnext = __shfl_down_sync(FULL, suf, 1);
            lprev = lane == 0 ? left : max(lprev, left);
            rnext = lane == 31 ? right : min(rnext, right);
            left = max(left, __shfl_sync(FULL, pre, 31));
            const int nword = min(32, W - c0);
            for (int j = 0; j < nword; ++j) {
                const uint32_t wd = __shfl_sync(FULL, word, j);
                const int lp = __shfl_sync(FULL, lprev, j), rn = __shfl_sync(FULL, rnext, j);
                const int xb = 32 * (c0 + j), x = xb + lane;
                if (x < X) {
                    const uint32_t lo = wd & (0xFFFFFFFFu >> (31 - lane));  // bits <= lane
                    const uint32_t hi = wd >> lane;                          // bits >= lane
                    const int l = lo ? xb + 31 - __clz(lo) : lp;
                    const int r = hi ? x + __ffs(hi) - 1 : rn;
                    uint32_t d = 0xFFFFFFFFu;
                    if (l >= 0) d = (uint32_t)(x - l);
                    if (r != INT_MAX) d = min(d, (uint32_t)(r - x));
                    g[x] = d == 0xFFFFFFFFu ? DT_INF : wx * d * d;
                }
            }
        }
    }
}

// Long-line path: lower envelope of one line of L values f (stride apart),
// weight w: out(q) = min_i f(i) + w (q - i)^2 over the i with f(i) != DT_INF,
// DT_INF when there is none.  The forward sweep keeps the hull vertices on a
// stack, dropping the top one while dt_covered; stack entry k is written over
// element k of the line itself (f value) and of sp (position): k <= q always,
// so no value still to be read is overwritten.  The second sweep walks the
// stack while the next parabola is no higher at q.
__device__ __forceinline__ void dist_line(uint32_t *__restrict__ f, uint16_t *__restrict__ sp,
                                          uint32_t *__restrict__ out, size_t stride, int L, uint32_t w) {
    int k = -1;
    uint32_t p0 = 0, a0 = 0, p1 = 0, a1 = 0;  // stack entries k - 1 and k
    for (int q = 0; q < L; ++q) {
        const uint32_t fq = f[(size_t)q * stride];
        if (fq == DT_INF) continue;
        const uint32_t aq = fq + w * dt_sq(q);
        while (k >= 1 && dt_covered(p0, a0, p1, a1, (uint32_t)q, aq)) {
            --k;
            p1 = p0;
            a1 = a0;
            if (k >= 1) {
                p0 = sp[(size_t)(k - 1) * stride];
                a0 = f[(size_t)(k - 1) * stride] + w * p0 * p0;
            }
        }
        ++k;
        sp[(size_t)k * stride] = (uint16_t)q;
        f[(size_t)k * stride] = fq;
        p0 = p1;
        a0 = a1;
        p1 = (uint32_t)q;
        a1 = aq;
    }
    if (k < 0) {
        for (int q = 0; q < L; ++q) out[(size_t)q * stride] = DT_INF;
        return;
    }
    const int top = k;
    int j = 0;
    uint32_t pj = sp[0], fj = f[0], pn = 0u, fn = 0u;
    if (top >= 1) {
        pn = sp[stride];
        fn = f[stride];
    }
    for (int q = 0; q < L; ++q) {
        uint32_t vj = fj + w * dt_sq(q - (int)pj);
        while (j < top) {
            const uint32_t vn = fn + w * dt_sq(q - (int)pn);
            if (vn > vj) break;
            ++j;
            pj = pn;
            fj = fn;
            vj = vn;
            if (j < top) {
                pn = sp[(size_t)(j + 1) * stride];
                fn = f[(size_t)(j + 1) * stride];
            }
        }
        out[(size_t)q * stride] = vj;
    }
}

// Long-line path: one thread per line along y (AXIS 1: g -> h) or z
// (AXIS 2: h -> the distance map); consecutive threads take consecutive x,
// so every step of a warp touches 32 neighbouring words.
template <int AXIS>
__global__ void __launch_bounds__(256) k_dist_line(const BatchHdr *__restrict__ h) {
    constexpr int K = AXIS == 1 ? DT_Y : DT_ZL;
    __shared__ DtIndex<K> VI;
    VI.load(h);
    for (uint32_t it = blockIdx.x * blockDim.x + threadIdx.x; it < h->dt_items[K]; it += gridDim.x * blockDim.x) {
        const VolDev &V = h->vol[VI.find(h, it)];
        const uint32_t li = it - V.dt_base[K];
        const uint32_t x = li % V.X, u = li / V.X;  // u = z (y lines) or y (z lines)
        const size_t plane = (size_t)V.X * V.Y;
        if (AXIS == 1) {
            const size_t o = (size_t)u * plane + x;
            dist_line(V.dt_g + o, V.dt_sp + o, V.dt_h + o, V.X, (int)V.Y, V.dt_w[1]);
        } else {
            const size_t o = (size_t)u * V.X + x;
            dist_line(V.dt_h + o, V.dt_sp + o, V.dt_out + o, plane, (int)V.Z, V.dt_w[2]);
        }
    }
}

// x and y passes fused: one block per (mask word w, plane z) of every volume
// whose lines along y fit (Y <= 32 NB, X < 65536).  Lane l follows the line
// x = 32 w + l along y; warp b holds band b of it, BL = ceil(Y / NB)
// consecutive y.
//   1. x pass: a warp reads each of its band's mask rows whole (so the
//      nearest foreground voxels left and right of the word are found too) and
//      stores dx, the distance along x to the row's nearest foreground voxel
//      (DX_NONE: none), in shared memory.
//   2. Each band builds the lower hull of its points (y, A(y)),
//      A(y) = wx dx(y)^2 + wy y^2, on a stack in shared memory.
//   3. Hulls of neighbouring band groups merge in log2(NB) rounds: the lower
//      common tangent of two hulls separated along y is found by dropping the
//      left hull's last vertex or the right hull's first while it is covered
//      by the segment from its neighbour to the other hull; each band keeps
//      the contiguous range [lo, hi) of its stack that survives.
//   4. Each band evaluates its outputs: the vertex lowest at the band's first
//      y is reached by walking from the band's own vertices (along the hull
//      the values at one y fall, then rise), then the walk goes on forward as
//      y grows.  Values at y inside the volume stay below 2^32 (the weights
//      were checked against the volume's extent), so step 4 is 32-bit.
// The result, min over foreground (x', y', z) of wx (x-x')^2 + wy (y-y')^2,
// goes to dt_h.
template <int NB>
__global__ void __launch_bounds__(NB * 32, NB == 16 ? 3 : 1) k_dist_xy(const BatchHdr *__restrict__ h) {
    constexpr int K = NB == 16 ? DT_XY16 : DT_XY32;
    constexpr int YCAP = 32 * NB;
    extern __shared__ __align__(16) uint16_t xsm[];
    uint16_t *sdx = xsm;              // [YCAP][32] x distances
    uint16_t *sst = xsm + YCAP * 32;  // [YCAP][32] band stacks (positions y)
    __shared__ uint16_t slo[NB][32], shi[NB][32];
    __shared__ DtIndex<K> VI;
    VI.load(h);
    const int lane = threadIdx.x & 31, b = threadIdx.x >> 5;
    for (uint32_t it = blockIdx.x; it < h->dt_items[K]; it += gridDim.x) {
        const VolDev &V = h->vol[VI.find(h, it)];
        const uint32_t li = it - V.dt_base[K];
        const int W = (int)V.W, X = (int)V.X, Y = (int)V.Y;
        const int w = (int)(li % (uint32_t)W), z = (int)(li / (uint32_t)W);
        const int BL = (Y + NB - 1) / NB;
        const int x = 32 * w + lane;
        const uint32_t wx = V.dt_w[0], wy = V.dt_w[1];
        const int ys = min(b * BL, Y), ye = min(ys + BL, Y);
        // 1. x distances of this band's rows
        auto put_dx = [&](int y, uint32_t own, int lc, int rc) {
            uint32_t dx = DX_NONE;
            if (x < X) {
                const uint32_t lo = own & (0xFFFFFFFFu >> (31 - lane));  // bits <= lane
                const uint32_t hi = own >> lane;                          // bits >= lane
                const int l = lo ? 32 * w + 31 - __clz(lo) : lc;
                const int r = hi ? x + __ffs(hi) - 1 : rc;
                uint32_t d = 0xFFFFFFFFu;
                if (l >= 0) d = (uint32_t)(x - l);
                if (r != INT_MAX) d = min(d, (uint32_t)(r - x));
                if (d != 0xFFFFFFFFu) dx = d;  // d <= X - 1 < DX_NONE
            }
            sdx[y * 32 + lane] = (uint16_t)dx;
        };
        const uint32_t *mb = V.mask + ((size_t)z * Y + ys) * W;
        if (W <= 32) {
            // rows of at most 32 words: lane l holds word l of 8 rows at a
            // time, the 8 loads issued before any is used
            for (int r0 = 0; r0 < ye - ys; r0 += 8) {
            uint32_t rw[8];
#pragma unroll
            for (int u = 0; u < 8; ++u)
                rw[u] = (r0 + u < ye - ys && lane < W) ? mb[(size_t)(r0 + u) * W + lane] : 0u;
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int r = r0 + u;
                if (r >= ye - ys) break;
                const uint32_t wd = rw[u];
                const uint32_t nz = __ballot_sync(FULL, wd != 0u);
                const uint32_t own = __shfl_sync(FULL, wd, w);
                const uint32_t below = nz & ((1u << w) - 1u);
                const uint32_t above = w >= 31 ? 0u : nz & ~((2u << w) - 1u);
                int lc = -1, rc = INT_MAX;  // nearest foreground x left / right of word w
                if (below) {
                    const int j = 31 - __clz(below);
                    lc = 32 * j + 31 - __clz(__shfl_sync(FULL, wd, j));
                }
                if (above) {
                    const int j = __ffs(above) - 1;
                    rc = 32 * j + __ffs(__shfl_sync(FULL, wd, j)) - 1;
                }
                put_dx(ys + r, own, lc, rc);
            }
            }
        } else {
            for (int y = ys; y < ye; ++y) {
                const uint32_t *m = mb + (size_t)(y - ys) * W;
                uint32_t own = 0u;
                int lc = -1, rc = INT_MAX;
                for (int c0 = 0; c0 < W; c0 += 32) {
                    const uint32_t wd = c0 + lane < W ? m[c0 + lane] : 0u;
                    const uint32_t nz = __ballot_sync(FULL, wd != 0u);
                    const int rel = w - c0;  // word w's place in this chunk
                    if (rel >= 0 && rel < 32) own = __shfl_sync(FULL, wd, rel);
                    const uint32_t below = rel <= 0 ? 0u : (rel >= 32 ? nz : nz & ((1u << rel) - 1u));
                    const uint32_t above = rel < 0 ? nz : (rel >= 31 ? 0u : nz & ~((2u << rel) - 1u));
                    if (below) {
                        const int j = 31 - __clz(below);
                        lc = 32 * (c0 + j) + 31 - __clz(__shfl_sync(FULL, wd, j));
                    }
                    if (above && rc == INT_MAX) {
                        const int j = __ffs(above) - 1;
                        rc = 32 * (c0 + j) + __ffs(__shfl_sync(FULL, wd, j)) - 1;
                    }
                }
                put_dx(y, own, lc, rc);
            }
        }
        // (own rows only: each lane reads back what it wrote)
        auto fval = [&](int p) -> uint32_t {  // wx dx(p)^2 of a row with foreground
            const uint32_t d = sdx[p * 32 + lane];
            return wx * d * d;
        };
        auto A = [&](uint32_t p) -> uint32_t { return fval((int)p) + wy * p * p; };
        // 2. the band's lower hull
        int k = -1;
        uint32_t p0 = 0, a0 = 0, p1 = 0, a1 = 0;  // stack entries k - 1 and k
        for (int q = ys; q < ye; ++q) {
            const uint32_t d = sdx[q * 32 + lane];
            if (d == DX_NONE) continue;
            const uint32_t aq = wx * d * d + wy * dt_sq(q);
            while (k >= 1 && dt_covered(p0, a0, p1, a1, (uint32_t)q, aq)) {
                --k;
                p1 = p0;
                a1 = a0;
                if (k >= 1) {
                    p0 = sst[(ys + k - 1) * 32 + lane];
                    a0 = A(p0);
                }
            }
            ++k;
            sst[(ys + k) * 32 + lane] = (uint16_t)q;
            p0 = p1;
            a0 = a1;
            p1 = (uint32_t)q;
            a1 = aq;
        }
        slo[b][lane] = 0;
        shi[b][lane] = (uint16_t)(k + 1);
        __syncthreads();
        auto pos = [&](int bb, int i) -> int { return sst[(min(bb * BL, Y) + i) * 32 + lane]; };
        auto empty = [&](int bb) -> bool { return slo[bb][lane] >= shi[bb][lane]; };
        // 3. merge rounds: band b = (2g + 1) s joins [b - s, b) and [b, b + s)
        for (int s = 1; s < NB; s <<= 1) {
            if ((b & (2 * s - 1)) == s) {
                int bl = b - 1, br = b;
                while (bl >= b - s && empty(bl)) --bl;
                while (br < b + s && empty(br)) ++br;
                if (bl >= b - s && br < b + s) {
                    int il = shi[bl][lane] - 1, ir = slo[br][lane];
                    uint32_t pL = pos(bl, il), aL = A(pL), pR = pos(br, ir), aR = A(pR);
                    for (bool moved = true; moved;) {
                        moved = false;
                        for (;;) {  // the left hull's last vertex
                            int pb = bl, pi = il - 1;
                            if (pi < (int)slo[pb][lane]) {
                                do --pb; while (pb >= b - s && empty(pb));
                                if (pb < b - s) break;
                                pi = shi[pb][lane] - 1;
                            }
                            const uint32_t pP = pos(pb, pi), aP = A(pP);
                            if (!dt_covered(pP, aP, pL, aL, pR, aR)) break;
                            bl = pb; il = pi; pL = pP; aL = aP;
                            moved = true;
                        }
                        for (;;) {  // the right hull's first vertex
                            int nb = br, ni = ir + 1;
                            if (ni >= (int)shi[nb][lane]) {
                                do ++nb; while (nb < b + s && empty(nb));
                                if (nb >= b + s) break;
                                ni = slo[nb][lane];
                            }
                            const uint32_t pN = pos(nb, ni), aN = A(pN);
                            if (!dt_covered(pL, aL, pR, aR, pN, aN)) break;
                            br = nb; ir = ni; pR = pN; aR = aN;
                            moved = true;
                        }
                    }
                    shi[bl][lane] = (uint16_t)(il + 1);
                    for (int bb = bl + 1; bb < b; ++bb) shi[bb][lane] = slo[bb][lane];
                    slo[br][lane] = (uint16_t)ir;
                    for (int bb = b; bb < br; ++bb) slo[bb][lane] = shi[bb][lane];
                }
            }
            __syncthreads();
        }
        // 4. outputs of this band
        if (x < X && ys < ye) {
            uint32_t *out = V.dt_h + (size_t)z * Y * X + x;
            // a surviving vertex near the band: its own first, else the
            // nearest band's to the left (last), else to the right (first)
            int cb = b, ci = 0;
            bool any = true;
            if (!empty(b)) {
                ci = slo[b][lane];
            } else {
                cb = b - 1;
                while (cb >= 0 && empty(cb)) --cb;
                if (cb >= 0) {
                    ci = shi[cb][lane] - 1;
                } else {
                    cb = b + 1;
                    while (cb < NB && empty(cb)) ++cb;
                    if (cb < NB) ci = slo[cb][lane]; else any = false;
                }
            }
            if (!any) {
                for (int q = ys; q < ye; ++q) out[(size_t)q * X] = DT_INF;
            } else {
                auto val = [&](uint32_t f, int p, int q) -> uint32_t {
                    const uint32_t d = (uint32_t)abs(q - p);
                    return f + wy * d * d;
                };
                int pc = pos(cb, ci);
                uint32_t fc = fval(pc);
                for (;;) {  // back while the previous vertex is lower at ys
                    int pb = cb, pi = ci - 1;
                    if (pi < (int)slo[pb][lane]) {
                        do --pb; while (pb >= 0 && empty(pb));
                        if (pb < 0) break;
                        pi = shi[pb][lane] - 1;
                    }
                    const int pp = pos(pb, pi);
                    const uint32_t fp = fval(pp);
                    if (val(fp, pp, ys) >= val(fc, pc, ys)) break;
                    cb = pb; ci = pi; pc = pp; fc = fp;
                }
                // the next vertex (none: pn < 0)
                int nb = cb, ni = ci + 1, pn = -1;
                uint32_t fn = 0u;
                auto load_next = [&]() {
                    if (ni >= (int)shi[nb][lane]) {
                        do ++nb; while (nb < NB && empty(nb));
                        if (nb >= NB) { pn = -1; return; }
                        ni = slo[nb][lane];
                    }
                    pn = pos(nb, ni);
                    fn = fval(pn);
                };
                load_next();
                for (int q = ys; q < ye; ++q) {
                    uint32_t vc = val(fc, pc, q);
                    while (pn >= 0) {
                        const uint32_t vn = val(fn, pn, q);
                        if (vn > vc) break;
                        pc = pn;
                        fc = fn;
                        vc = vn;
                        ++ni;
                        load_next();
                    }
                    out[(size_t)q * X] = vc;
                }
            }
        }
        __syncthreads();  // the next tile reuses the shared arrays
    }
}

// z pass: one block per (mask word w, group of lt / 32 rows) of every volume
// with Z <= 256 (lt lines, lt Z <= DZ_ELEMS).  Thread t < lt follows the
// line x = 32 w + (t & 31), y = y0 + (t >> 5) along z: it loads the line's
// dt_h values into shared memory (entry q at q lt + t, the loads independent
// of each other), builds the lower hull over them in place (as dist_line),
// then writes the distance map.  Positions (< 256) are bytes, four entries of
// a line to a 32-bit word, so a warp's lanes always touch distinct banks.
// Values at z inside the volume stay below 2^32, so the second sweep is
// 32-bit.  Each thread touches only its own entries.
__global__ void __launch_bounds__(128) k_dist_z(const BatchHdr *__restrict__ h) {
    extern __shared__ __align__(16) uint32_t zsm[];
    uint32_t *sf = zsm;                                              // [DZ_ELEMS] values
    uint8_t *spb = reinterpret_cast<uint8_t *>(zsm + DZ_ELEMS);      // positions
    __shared__ DtIndex<DT_Z> VI;
    VI.load(h);
    const int t = threadIdx.x;
    for (uint32_t it = blockIdx.x; it < h->dt_items[DT_Z]; it += gridDim.x) {
        const VolDev &V = h->vol[VI.find(h, it)];
        const uint32_t li = it - V.dt_base[DT_Z];
        const int W = (int)V.W, X = (int)V.X, Y = (int)V.Y, Z = (int)V.Z, lt = (int)V.dt_zlt;
        const int w = (int)(li % (uint32_t)W), y = (int)(li / (uint32_t)W) * (lt >> 5) + (t >> 5);
        const int x = 32 * w + (t & 31);
        if (t >= lt || x >= X || y >= Y) continue;
        const size_t plane = (size_t)X * Y;
        const uint32_t *in = V.dt_h + (size_t)y * X + x;
        uint32_t *out = V.dt_out + (size_t)y * X + x;
        uint32_t *f = sf + t;
        auto pos = [&](int k) -> uint8_t & { return spb[(((k >> 2) * lt + t) << 2) + (k & 3)]; };
#pragma unroll 8
        for (int q = 0; q < Z; ++q) f[q * lt] = in[(size_t)q * plane];
        const uint32_t wz = V.dt_w[2];
        int k = -1;
        uint32_t p0 = 0, a0 = 0, p1 = 0, a1 = 0;  // stack entries k - 1 and k
        for (int q = 0; q < Z; ++q) {
            const uint32_t fq = f[q * lt];
            if (fq == DT_INF) continue;
            const uint32_t aq = fq + wz * dt_sq(q);
            while (k >= 1 && dt_covered(p0, a0, p1, a1, (uint32_t)q, aq)) {
                --k;
                p1 = p0;
                a1 = a0;
                if (k >= 1) {
                    p0 = pos(k - 1);
                    a0 = f[(k - 1) * lt] + wz * p0 * p0;
                }
            }
            ++k;
            pos(k) = (uint8_t)q;
            f[k * lt] = fq;
            p0 = p1;
            a0 = a1;
            p1 = (uint32_t)q;
            a1 = aq;
        }
        if (k < 0) {
            for (int q = 0; q < Z; ++q) out[(size_t)q * plane] = DT_INF;
            continue;
        }
        const int top = k;
        int j = 0;
        uint32_t pj = pos(0), fj = f[0], pn = 0u, fn = 0u;
        if (top >= 1) {
            pn = pos(1);
            fn = f[lt];
        }
        for (int q = 0; q < Z; ++q) {
            uint32_t vj = fj + wz * dt_sq(q - (int)pj);
            while (j < top) {
                const uint32_t vn = fn + wz * dt_sq(q - (int)pn);
                if (vn > vj) break;
                ++j;
                pj = pn;
                fj = fn;
                vj = vn;
                if (j < top) {
                    pn = pos(j + 1);
                    fn = f[(j + 1) * lt];
                }
            }
            out[(size_t)q * plane] = vj;
        }
    }
}

// Cell-to-vessel distance (Fig. 4): out[k - 1] = min over the voxels of cell k
// of a distance map (out preset to DT_INF).  Each thread takes 8 consecutive
// voxels and flushes one atomic per run of equal labels.
__global__ void __launch_bounds__(256) k_cell_distance(const uint32_t *__restrict__ labels,
                                                       const uint32_t *__restrict__ map, uint64_t n, uint64_t k,
                                                       uint32_t *__restrict__ out) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x * 8;
    for (uint64_t i0 = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) * 8; i0 < n; i0 += stride) {
        const uint64_t e = i0 + 8 < n ? i0 + 8 : n;
        uint32_t cur = 0, best = 0xFFFFFFFFu;
        for (uint64_t i = i0; i < e; ++i) {
            const uint32_t l = labels[i];
            if (l != cur) {
                if (cur && cur <= k) atomicMin(out + (cur - 1), best);
                cur = l;
                best = 0xFFFFFFFFu;
            }
            if (l) best = min(best, map[i]);
        }
        if (cur && cur <= k) atomicMin(out + (cur - 1), best);
    }
}

// Label runs (read path; Segmentation section: each cell's voxels, the set
// handed to the convex hull step): the maximal runs of equal non-zero label
// along x, in order of (row, x).  With L = 0 outside the row, a run starts at
// x when L(x) != 0 and L(x) != L(x - 1), and ends at x - 1 when L(x - 1) != 0
// and L(x - 1) != L(x).  RUNS_ROWS rows per block, one warp per row, lanes on
// consecutive voxels, eight 32-voxel loads in flight before the boundaries
// are tested; ballots rank the starts and ends of a row.  The count pass
// stores each row's runs and each block's total; after the scan over blocks
// the write pass turns them into row offsets (a block scan) and writes the
// records, the start fields from the run's first voxel and x_end from the
// boundary after its last.
constexpr int RUNS_ROWS = 64;
constexpr int RUNS_THREADS = 256;

template <bool WRITE>
__global__ void __launch_bounds__(RUNS_THREADS) k_label_runs(const uint32_t *__restrict__ labels, uint32_t X,
                                                             uint32_t rows, uint32_t ntiles,
                                                             uint32_t *__restrict__ rowcnt,
                                                             uint32_t *__restrict__ tiles,
                                                             seg_label_run *__restrict__ out,
                                                             const uint32_t *__restrict__ total, uint64_t cap) {
    __shared__ uint32_t sbuf[33];
    __shared__ uint32_t soff[RUNS_ROWS];
    if (WRITE && *total > cap) return;  // the destination is too small: write nothing
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t below = (1u << lane) - 1u;
    for (uint32_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const uint32_t r0 = t * RUNS_ROWS;
        if (WRITE) {
            const uint32_t row = r0 + threadIdx.x;
            const uint32_t c = threadIdx.x < RUNS_ROWS && row < rows ? rowcnt[row] : 0u;
            uint32_t tot;
            const uint32_t ex = block_exscan<RUNS_THREADS>(c, &tot, sbuf);
            if (threadIdx.x < RUNS_ROWS) soff[threadIdx.x] = tiles[t] + ex;
            __syncthreads();
        }
        uint32_t cnt = 0;
        for (uint32_t rr = warp; rr < RUNS_ROWS; rr += RUNS_THREADS / 32) {
            const uint32_t row = r0 + rr;
            if (row >= rows) break;
            const uint32_t *L = labels + (uint64_t)row * X;
            const uint32_t base = WRITE ? soff[rr] : 0u;
            uint32_t carry = 0, ns = 0, ne = 0;
            for (uint32_t xb = 0; xb < X; xb += 256) {
                uint32_t v[8];
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const uint32_t x = xb + 32u * j + lane;
                    v[j] = x < X ? L[x] : 0u;
                }
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const uint32_t x = xb + 32u * j + lane;
                    if (xb + 32u * j >= X) break;
                    uint32_t prev = __shfl_up_sync(FULL, v[j], 1);
                    if (lane == 0) prev = carry;
                    const bool st = v[j] != 0u && v[j] != prev;
                    const bool en = prev != 0u && prev != v[j];
                    const uint32_t bs = __ballot_sync(FULL, st), be = __ballot_sync(FULL, en);
                    if (WRITE) {
                        if (st) {
                            seg_label_run *o = out + base + ns + __popc(bs & below);
                            o->label = v[j];
                            o->row = row;
                            o->x_begin = (uint16_t)x;
                        }
                        if (en) out[base + ne + __popc(be & below)].x_end = (uint16_t)(x - 1u);
                    }
                    ns += __popc(bs);
                    ne += __popc(be);
                    carry = __shfl_sync(FULL, v[j], 31);
                }
            }
            // a run reaching the row end (X a multiple of 32: the boundary
            // after the last voxel is in no step)
            if (carry) {
                if (WRITE && lane == 0) out[base + ne].x_end = (uint16_t)(X - 1u);
                ++ne;
            }
            if (!WRITE && lane == 0) rowcnt[row] = ns;
            cnt += ns;
        }
        if (!WRITE) {
            const uint32_t tot = block_sum<RUNS_THREADS>(lane == 0 ? cnt : 0u, sbuf);
            if (threadIdx.x == 0) tiles[t] = tot;
        }
        __syncthreads();  // soff and sbuf are reused by the next tile
    }
}

// The records to a destination the device reaches (mapped pinned host
// memory) as 4-byte words, coalesced; nothing when they do not fit.
__global__ void __launch_bounds__(256) k_label_runs_copy(const uint32_t *__restrict__ src, uint32_t *__restrict__ dst,
                                                         const uint32_t *__restrict__ total, uint64_t cap) {
    const uint64_t n = *total;
    if (n > cap) return;
    const uint64_t words = 3 * n;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < words; i += (uint64_t)gridDim.x * blockDim.x)
        dst[i] = src[i];
}

// Exclusive scan over the blocks' run counts (one block); *total = the sum.
__global__ void __launch_bounds__(1024) k_label_runs_scan(uint32_t *__restrict__ tiles, uint32_t ntiles,
                                                          uint32_t *__restrict__ total) {
    __shared__ uint32_t sbuf[33];
    uint32_t carry = 0;
    for (uint32_t b = 0; b < ntiles; b += 1024) {
        const uint32_t i = b + threadIdx.x;
        const uint32_t c = i < ntiles ? tiles[i] : 0u;
        uint32_t tot;
        const uint32_t ex = block_exscan<1024>(c, &tot, sbuf);
        if (i < ntiles) tiles[i] = carry + ex;
        carry += tot;
    }
    if (threadIdx.x == 0) *total = carry;
}

template <int TY>
cudaError_t launch_tile_kernels(const BatchHdr *d, const LaunchPlan &p, cudaStream_t s,
                                cudaEvent_t *ev, int &k) {
    auto rec = [&]() {
        if (ev) cudaEventRecordWithFlags(ev[k], s, cudaEventRecordExternal);
        ++k;
    };
    rec();
    if (p.rows) k_smooth_rows<<<p.grid_hist, FS_NT, FS_SMEM, s>>>(d);
    rec();
    if (p.tiles) k_smooth_hist<TY><<<p.grid_hist, Tile<TY>::NT, hist_smem_bytes(TY), s>>>(d);
    rec();
    k_otsu<<<p.grid_vols, OTSU_NT, OTSU_SMEM, s>>>(d);
    return cudaGetLastError();
}

}  // namespace

// k_dist_xy<NB>: x distances and band stacks, 32 lines x 32 NB rows, uint16
static size_t dxy_smem(int nb) { return 2ull * 2 * 32 * 32 * (size_t)nb; }
// k_dist_z: uint32 values and byte positions (rows of four, padded)
constexpr size_t DZ_SMEM = 5ull * DZ_ELEMS + 512;

size_t hist_smem_bytes(int tile_y) {
    return tile_y == 16 ? Tile<16>::HIST_SMEM : (tile_y == 32 ? Tile<32>::HIST_SMEM : Tile<64>::HIST_SMEM);
}

cudaError_t configure_kernels(int device, LaunchPlan &plan) {
    cudaError_t e = cudaSetDevice(device);
    if (e != cudaSuccess) return e;
#define SEG_CFG(TY)                                                                        \
    e = cudaFuncSetAttribute(k_smooth_hist<TY>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                             (int)hist_smem_bytes(TY));                                    \
    if (e != cudaSuccess) return e;                                                        \

    SEG_CFG(16)
    SEG_CFG(32)
    SEG_CFG(64)
#undef SEG_CFG
    e = cudaFuncSetAttribute(k_smooth_rows, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)FS_SMEM);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_otsu, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)OTSU_SMEM);
    if (e != cudaSuccess) return e;
    auto resident = [&](const void *fn, int threads, int *grid) -> cudaError_t {
        int per_sm = 0;
        const cudaError_t r = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, threads, 0);
        if (r != cudaSuccess) return r;
        *grid = plan.sms * (per_sm > 0 ? per_sm : 1);
        return cudaSuccess;
    };
    int g1 = 0, g2 = 0, g3 = 0;
    if ((e = resident((const void *)k_threshold_runs, ROW_TILE, &plan.grid_thr)) != cudaSuccess) return e;
    if ((e = resident((const void *)k_row_runs, ROW_TILE, &g1)) != cudaSuccess) return e;
    if ((e = resident((const void *)k_keep_count, ROW_TILE, &g2)) != cudaSuccess) return e;
    if ((e = resident((const void *)k_rank, ROW_TILE, &g3)) != cudaSuccess) return e;
    plan.grid_rows = std::min(g1, std::min(g2, g3));
    if ((e = resident((const void *)k_union_local, BRICK_Y * BRICK_Z, &plan.grid_ul)) != cudaSuccess) return e;
    if ((e = resident((const void *)k_union, ROW_TILE, &g1)) != cudaSuccess) return e;
    if ((e = resident((const void *)k_flatten, ROW_TILE, &g2)) != cudaSuccess) return e;
    plan.grid_task = std::min(g1, g2);
    if ((e = resident((const void *)k_label_features, ROW_TILE, &plan.grid_lab)) != cudaSuccess) return e;
    for (const void *fn : {(const void *)k_box3<0>, (const void *)k_box3<1>, (const void *)k_box3<2>})
        if ((e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)BOX_SMEM)) != cudaSuccess)
            return e;
    {
        int per_sm = 0;
        if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_box3<1>, 256, BOX_SMEM)) != cudaSuccess)
            return e;
        plan.grid_box = plan.sms * (per_sm > 0 ? per_sm : 1);
    }
    if ((e = resident((const void *)k_median27, MED_TX * MED_TY, &plan.grid_med)) != cudaSuccess) return e;
    if ((e = resident((const void *)k_dist_x, 256, &g1)) != cudaSuccess) return e;
    if ((e = resident((const void *)k_dist_line<2>, 256, &g2)) != cudaSuccess) return e;
    if ((e = resident((const void *)k_dist_line<1>, 256, &g3)) != cudaSuccess) return e;
    plan.grid_dist = std::min(g1, std::min(g2, g3));
    if ((e = resident((const void *)k_mrf_stats, MRF_TILE, &plan.grid_mrf)) != cudaSuccess) return e;
    if ((e = resident((const void *)k_mrf_step, MRF_TX * MRF_TY, &plan.grid_mrfs)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k_dist_z, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)DZ_SMEM)) !=
        cudaSuccess)
        return e;
    {
        int per_sm = 0;
        if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_dist_z, 128, DZ_SMEM)) != cudaSuccess)
            return e;
        plan.grid_dz = plan.sms * (per_sm > 0 ? per_sm : 1);
    }
    for (int nb : {16, 32}) {
        const void *fn = nb == 16 ? (const void *)k_dist_xy<16> : (const void *)k_dist_xy<32>;
        if ((e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dxy_smem(nb))) !=
            cudaSuccess)
            return e;
        int per_sm = 0;
        if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, nb * 32, dxy_smem(nb))) != cudaSuccess)
            return e;
        (nb == 16 ? plan.grid_dxy16 : plan.grid_dxy32) = plan.sms * (per_sm > 0 ? per_sm : 1);
    }
    return cudaSuccess;
}

cudaError_t launch_tile_probe(const BatchHdr *d, const LaunchPlan &p, cudaStream_t s) {
    k_init<<<p.grid_vols * 4, 256, 0, s>>>(d);
    switch (p.tile_y) {
        case 16: k_smooth_hist<16><<<p.grid_hist, Tile<16>::NT, hist_smem_bytes(16), s>>>(d); break;
        case 32: k_smooth_hist<32><<<p.grid_hist, Tile<32>::NT, hist_smem_bytes(32), s>>>(d); break;
        default: k_smooth_hist<64><<<p.grid_hist, Tile<64>::NT, hist_smem_bytes(64), s>>>(d); break;
    }
    return cudaGetLastError();
}

static void launch_box_passes(const BatchHdr *d, const LaunchPlan &p, cudaStream_t s) {
    k_box3<0><<<p.grid_box, 256, BOX_SMEM, s>>>(d);
    k_box3<1><<<p.grid_box, 256, BOX_SMEM, s>>>(d);
    k_box3<2><<<p.grid_box, 256, BOX_SMEM, s>>>(d);
}

cudaError_t launch_cell_distance(const uint32_t *labels, const uint32_t *map, uint64_t n, uint32_t *out, uint64_t k,
                                 int sms, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(out, 0xFF, 4 * (k ? k : 1), s);
    if (e != cudaSuccess || k == 0 || n == 0) return e;
    const uint64_t want = (n + 8 * 256 - 1) / (8 * 256);
    const int grid = (int)std::min<uint64_t>(want, (uint64_t)sms * 8);
    k_cell_distance<<<grid, 256, 0, s>>>(labels, map, n, k, out);
    return cudaGetLastError();
}

uint32_t label_runs_tiles(uint32_t rows) { return (rows + RUNS_ROWS - 1) / RUNS_ROWS; }

cudaError_t launch_label_runs_count(const uint32_t *labels, uint32_t X, uint32_t rows, uint32_t *rowcnt,
                                    uint32_t *tiles, uint32_t *total, int sms, cudaStream_t s) {
    const uint32_t nt = label_runs_tiles(rows);
    const int grid = (int)std::min<uint64_t>(nt, (uint64_t)sms * 8);
    k_label_runs<false><<<grid, RUNS_THREADS, 0, s>>>(labels, X, rows, nt, rowcnt, tiles, nullptr, nullptr, 0);
    k_label_runs_scan<<<1, 1024, 0, s>>>(tiles, nt, total);
    return cudaGetLastError();
}

cudaError_t launch_label_runs_write(const uint32_t *labels, uint32_t X, uint32_t rows, const uint32_t *rowcnt,
                                    const uint32_t *tiles, const uint32_t *total, uint64_t cap, seg_label_run *out,
                                    seg_label_run *mapped, int sms, cudaStream_t s) {
    const uint32_t nt = label_runs_tiles(rows);
    const int grid = (int)std::min<uint64_t>(nt, (uint64_t)sms * 8);
    k_label_runs<true><<<grid, RUNS_THREADS, 0, s>>>(labels, X, rows, nt, const_cast<uint32_t *>(rowcnt),
                                                     const_cast<uint32_t *>(tiles), out, total, cap);
    if (mapped) {
        const uint64_t words = 3 * cap;
        const int cg = (int)std::max<uint64_t>(1, std::min<uint64_t>((words + 255) / 256, (uint64_t)sms * 4));
        k_label_runs_copy<<<cg, 256, 0, s>>>(reinterpret_cast<const uint32_t *>(out),
                                             reinterpret_cast<uint32_t *>(mapped), total, cap);
    }
    return cudaGetLastError();
}

cudaError_t launch_denoise(const BatchHdr *d, const LaunchPlan &p, cudaStream_t s) {
    launch_box_passes(d, p, s);
    k_median27<<<p.grid_med, MED_TX * MED_TY, 0, s>>>(d);
    return cudaGetLastError();
}

cudaError_t launch_pipeline(const BatchHdr *d, const LaunchPlan &p, cudaStream_t s, cudaEvent_t *ev,
                            uint32_t *stat_out) {
    int k = 0;
    auto rec = [&]() {
        if (ev) cudaEventRecordWithFlags(ev[k], s, cudaEventRecordExternal);
        ++k;
    };
    // denoise front end, for batches in which some volume asks for it
    rec();
    if (p.denoise) launch_box_passes(d, p, s);
    rec();
    if (p.denoise) k_median27<<<p.grid_med, MED_TX * MED_TY, 0, s>>>(d);
    rec();
    k_init<<<p.grid_vols * 4, 256, 0, s>>>(d);
    // MRF vessel denoise, for batches in which some volume asks for it
    rec();
    if (p.mrf_iters) {
        k_mrf_stats<<<p.grid_mrf, MRF_TILE, 0, s>>>(d);
        k_mrf_prep<<<p.grid_vols, 32, 0, s>>>(d);
    }
    rec();
    for (uint32_t it = 0; it < p.mrf_iters; ++it) k_mrf_step<<<p.grid_mrfs, MRF_TX * MRF_TY, 0, s>>>(d, it);
    cudaError_t e;
    switch (p.tile_y) {
        case 16: e = launch_tile_kernels<16>(d, p, s, ev, k); break;
        case 32: e = launch_tile_kernels<32>(d, p, s, ev, k); break;
        default: e = launch_tile_kernels<64>(d, p, s, ev, k); break;
    }
    if (e != cudaSuccess) return e;
    rec();
    k_threshold_runs<<<p.grid_thr, ROW_TILE, 0, s>>>(d);
    // closing, for batches in which some volume asks for it
    rec();
    if (p.closing) k_dilate<<<p.grid_task, 256, 0, s>>>(d);
    rec();
    if (p.closing) k_erode<<<p.grid_thr, ROW_TILE, 0, s>>>(d);
    // distance map of the final foreground, for batches in which some volume
    // asks for it
    rec();
    if (p.distance) k_dist_xy<16><<<p.grid_dxy16, 16 * 32, dxy_smem(16), s>>>(d);
    rec();
    if (p.distance) k_dist_xy<32><<<p.grid_dxy32, 32 * 32, dxy_smem(32), s>>>(d);
    rec();
    if (p.distance) k_dist_x<<<p.grid_dist, 256, 0, s>>>(d);
    rec();
    if (p.distance) k_dist_line<1><<<p.grid_dist, 256, 0, s>>>(d);
    rec();
    if (p.distance) k_dist_z<<<p.grid_dz, 128, DZ_SMEM, s>>>(d);
    rec();
    if (p.distance) k_dist_line<2><<<p.grid_dist, 256, 0, s>>>(d);
    rec();
    k_row_runs<<<p.grid_rows, ROW_TILE, 0, s>>>(d);
    rec();
    k_union_local<<<p.grid_ul, BRICK_Y * BRICK_Z, 0, s>>>(d);
    rec();
    k_union<<<p.grid_task, ROW_TILE, 0, s>>>(d);
    rec();
    k_flatten<<<p.grid_task, ROW_TILE, 0, s>>>(d);
    rec();
    k_keep_count<<<p.grid_rows, ROW_TILE, 0, s>>>(d);
    rec();
    k_rank<<<p.grid_rows, ROW_TILE, 0, s>>>(d);
    rec();
    k_label_features<<<p.grid_lab, ROW_TILE, 0, s>>>(d);
    rec();
    k_gather_stat<<<p.grid_vols, 256, 0, s>>>(d, stat_out);
    if (ev) cudaEventRecordWithFlags(ev[k], s, cudaEventRecordExternal);
    return cudaGetLastError();
}

}  // namespace seg

// ----------------------------------------------------------------------------
// Allocation-free Otsu level (no counterpart in the paper).
//
// Some callers cannot allocate device memory: their HBM is fully reserved by
// another allocator (for example a framework's caching allocator), or they
// run latency-critical loops in which cudaMalloc / cudaFree, with their
// implicit synchronisation, are not acceptable.  seg_otsu_threshold_noalloc
// serves them: it runs the histogram + Otsu kernel on one device-resident
// volume with its scratch (the 65536-bin histogram and the status words) in
// the fixed array below, so it allocates nothing.
// ----------------------------------------------------------------------------

namespace seg {
namespace {

constexpr int NOALLOC_WORDS = HIST_BINS + ST_WORDS;  // 262,208 bytes per device

// Scratch of seg_otsu_threshold_noalloc: histogram bins, then status words.
// Every GPU that loads the library holds it until the process exits.
static __device__ __align__(256) uint32_t g_noalloc_scratch[NOALLOC_WORDS];

constexpr int NOALLOC_TY = 32;
constexpr int NOALLOC_TZ = 64;
constexpr int NOALLOC_MAX_DEVICES = 64;

// Device address of g_noalloc_scratch per device (host code must not use the
// symbol itself: in host code it names a host-side stand-in).
uint32_t *g_noalloc_ptr[NOALLOC_MAX_DEVICES] = {};
int g_noalloc_sms[NOALLOC_MAX_DEVICES] = {};
std::mutex g_noalloc_mu;

// The histogram kernel with its one-volume descriptor passed by value.
template <int TY>
__global__ void __launch_bounds__(8 * TY, 1) k_smooth_hist_noalloc(const __grid_constant__ BatchHdr hdr) {
    using T = Tile<TY>;
    const BatchHdr *h = &hdr;
    extern __shared__ __align__(128) unsigned char dsm[];
    unsigned char *ring = dsm;
    uint32_t *sh = reinterpret_cast<uint32_t *>(dsm + T::RING_BYTES);
    uint32_t *spx = sh + HIST_WORDS;
    int8_t *shift = reinterpret_cast<int8_t *>(spx + 2 * T::PX_WORDS);
    const VolDev &V = h->vol[0];
    Ring R{ring, shift, 0};
    for (int i = threadIdx.x; i < HIST_WORDS / 4; i += T::NT)
        reinterpret_cast<uint4 *>(sh)[i] = make_uint4(0, 0, 0, 0);
    __syncthreads();
    const uint32_t nt = h->ntiles, G = gridDim.x;
    const uint32_t tb = (uint32_t)(((uint64_t)nt * blockIdx.x) / G);
    const uint32_t te = (uint32_t)(((uint64_t)nt * (blockIdx.x + 1)) / G);
    if (tb >= te) return;
    const int tz = (int)h->tile_z;
    for (uint32_t t = tb; t < te; ++t) {
        const uint32_t ix = t % V.ntx, rest = t / V.ntx;
        const uint32_t iy = rest % V.nty, iz = rest / V.nty;
        const int z0 = (int)iz * tz;
        const int z1 = min(z0 + tz, (int)V.Z);
        HistEmit<false> e{sh, V.hist, nullptr, V.X, V.Y, 0u, 0u, nullptr, 0, false};
        smooth_tile<TY>(V.raw, V.X, V.Y, V.Z, (int)ix * TILE_X, (int)iy * TY, z0, z1, spx, R, e);
    }
    flush_hist<T::NT>(V, sh);
}

// Once per device, with that device current: resolve the scratch address and
// raise the kernel's dynamic shared-memory limit.
int noalloc_setup(int dev, uint32_t **ptr, int *sms) {
    if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) return SEG_EINVAL;
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) { cudaGetLastError(); return SEG_ECUDA; }
        e = cudaFuncSetAttribute(k_smooth_hist_noalloc<NOALLOC_TY>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)hist_smem_bytes(NOALLOC_TY));
        if (e != cudaSuccess) { cudaGetLastError(); return SEG_ECUDA; }
        e = cudaFuncSetAttribute(k_otsu_one, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)OTSU_SMEM);
        if (e != cudaSuccess) { cudaGetLastError(); return SEG_ECUDA; }
        int n = 0;
        e = cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) { cudaGetLastError(); return SEG_ECUDA; }
        g_noalloc_sms[dev] = n;
        g_noalloc_ptr[dev] = static_cast<uint32_t *>(p);
    }
    *ptr = g_noalloc_ptr[dev];
    *sms = g_noalloc_sms[dev];
    return SEG_OK;
}

}  // namespace

}  // namespace seg

extern "C" int seg_otsu_threshold_noalloc(const uint16_t *d_voxels, seg_dims dims, uint32_t *d_result,
                                          void *stream) {
    using namespace seg;
    if (!d_voxels || !d_result || dims.x == 0 || dims.y == 0 || dims.z == 0) return SEG_EINVAL;
    // uint16 voxels and uint32 results must be naturally aligned
    if ((reinterpret_cast<uintptr_t>(d_voxels) & 1u) || (reinterpret_cast<uintptr_t>(d_result) & 3u))
        return SEG_EINVAL;
    const uint64_t n = (uint64_t)dims.x * dims.y * dims.z;
    if (n > SEG_NOALLOC_MAX_VOXELS || dims.x > 65536u || dims.y > SEG_MAX_YZ || dims.z > SEG_MAX_YZ)
        return SEG_ETOOBIG;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) { cudaGetLastError(); return SEG_ECUDA; }
    uint32_t *scratch = nullptr;
    int sms = 0;
    int rc = noalloc_setup(dev, &scratch, &sms);
    if (rc != SEG_OK) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    BatchHdr hdr;
    std::memset(&hdr, 0, sizeof(hdr));
    VolDev &V = hdr.vol[0];
    V.raw = d_voxels;
    V.hist = scratch;
    V.stat = scratch + HIST_BINS;
    V.X = dims.x; V.Y = dims.y; V.Z = dims.z;
    V.ntx = (uint32_t)(((uint64_t)dims.x + TILE_X - 1) / TILE_X);
    V.nty = (uint32_t)(((uint64_t)dims.y + NOALLOC_TY - 1) / NOALLOC_TY);
    V.ntz = (uint32_t)(((uint64_t)dims.z + NOALLOC_TZ - 1) / NOALLOC_TZ);
    hdr.nvol = 1;
    hdr.ntiles = V.ntx * V.nty * V.ntz;
    hdr.tile_z = NOALLOC_TZ;
    hdr.tile_y = NOALLOC_TY;
    // the array keeps the previous call's contents: clear bins and counters
    cudaError_t e = cudaMemsetAsync(scratch, 0, sizeof(uint32_t) * NOALLOC_WORDS, s);
    if (e == cudaSuccess) {
        k_smooth_hist_noalloc<NOALLOC_TY><<<sms, Tile<NOALLOC_TY>::NT, hist_smem_bytes(NOALLOC_TY), s>>>(hdr);
        k_otsu_one<<<1, OTSU_NT, OTSU_SMEM, s>>>(V.hist, V.stat, n);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_result, scratch + HIST_BINS + ST_THRESH, sizeof(uint32_t),
                            cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_result + 1, scratch + HIST_BINS + ST_ERROR, sizeof(uint32_t),
                            cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) { cudaGetLastError(); return SEG_ECUDA; }
    return SEG_OK;
}
