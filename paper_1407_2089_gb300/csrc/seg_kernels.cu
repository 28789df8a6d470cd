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
//   smooth_hist     pass 1 over the raw voxels: binomial smoothing in
//                   registers/shared memory, 65536-bin shared histogram
//                   (two 16-bit counters per word), merge into the volume's
//                   histogram; the last block of a volume runs Otsu
//   smooth_mask     pass 2: smoothing again, foreground = s > t*, written as
//                   a bit mask (32 voxels per word along x)
//   row_count       foreground runs per x-row
//   scan_runs       per-volume scan of run counts over row tiles
//   row_runs        run table (x0, x1) per row; union-find parent = self
//   union           26-adjacency between runs of neighbouring rows, union by
//                   minimum run index (atomicMin), so a component's root is
//                   its first run in raster order
//   flatten         parent = root; voxel count accumulated at the root
//   keep_count      roots with count >= min_volume, per row
//   scan_keep       per-volume scan of kept roots -> K
//   rank            label of each kept root = 1 + its rank in raster order
//   label_features  per-voxel labels (coalesced uint32 rows) and per-cell
//                   count / bbox / coordinate sums
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "seg_internal.h"

namespace seg {

const char *const kKernelNames[NUM_KERNELS] = {
    "init",     "smooth_hist_otsu", "smooth_mask", "row_count", "scan_runs",      "row_runs", "union",
    "flatten",  "keep_count",       "scan_keep",   "rank",      "label_features", "gather_stat"};

namespace {

constexpr unsigned FULL = 0xFFFFFFFFu;
constexpr int HIST_WORDS = HIST_BINS / 2;  // two 16-bit counters per word
constexpr uint32_t UNION_LIMIT = 1u << 24;

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

__device__ __forceinline__ uint32_t find_vol_rt(const BatchHdr *__restrict__ h, uint32_t t) {
    uint32_t lo = 0, hi = h->nvol;
    while (hi - lo > 1) {
        uint32_t mid = (lo + hi) >> 1;
        if (h->vol[mid].rt_base <= t) lo = mid; else hi = mid;
    }
    return lo;
}

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

__device__ __forceinline__ uint32_t uf_find(const uint32_t *P, uint32_t x) {
    uint32_t p = __ldcg(P + x);
    while (p != x) {
        x = p;
        p = __ldcg(P + x);
    }
    return x;
}

// Union with the lower index as the surviving root.  atomicMin only ever
// lowers a parent, so each component ends rooted at its minimum run index
// whatever the interleaving.  Bounded retries; exhaustion raises ERR_UNION.
__device__ __forceinline__ void uf_union(uint32_t *P, uint32_t a, uint32_t b, uint32_t *err) {
    for (uint32_t it = 0; it < UNION_LIMIT; ++it) {
        a = uf_find(P, a);
        b = uf_find(P, b);
        if (a == b) return;
        if (a < b) {
            uint32_t old = atomicMin(P + b, a);
            if (old == b) return;
            b = old;
        } else {
            uint32_t old = atomicMin(P + a, b);
            if (old == a) return;
            a = old;
        }
    }
    atomicOr(err, ERR_UNION);
}

// ----------------------------------------------------------------------------
// separable binomial smoothing of one tile (shared by both passes)
// ----------------------------------------------------------------------------
//
// A block of 16*TY threads owns a TILE_X x TY column of outputs and marches
// along z from z0 - 2 to z1 + 1.  For each input plane it stages the
// (TY+4) x (TILE_X+4) clamped halo in shared memory as uint32, runs the x
// pass (each thread 4 adjacent outputs from 8 staged values), then the y pass
// (5 rows), and feeds the z pass in scatter form: with accumulators a0..a3
// holding the partial sums of outputs zi-2..zi+1,
//     out(zi-2) = a0 + P, a0 <- a1 + 4P, a1 <- a2 + 6P, a2 <- a3 + 4P, a3 <- P.
// All sums are exact in uint32 (at most 4096 * 65535); the one rounding
// (S + 2048) >> 12 is applied to the completed sum, which equals the 125-term
// definition.  Clamped coordinates replicate edge voxels per axis.

template <int TY>
struct Tile {
    static constexpr int NT = 16 * TY;
    static constexpr int RH = TY + 4;
    static constexpr int RW = TILE_X + 8;  // staged row stride in words
    static constexpr int CW = TILE_X + 4;  // staged columns
    static constexpr int NLOAD = RH * CW;
    static constexpr int LPT = (NLOAD + NT - 1) / NT;
    static constexpr int RAW_WORDS = RH * RW;
};

template <int TY, class Emit>
__device__ __forceinline__ void smooth_tile(const uint16_t *__restrict__ raw, uint32_t X, uint32_t Y,
                                            uint32_t Z, int x0, int y0, int z0, int z1,
                                            uint32_t *__restrict__ sraw, uint32_t *__restrict__ spx,
                                            Emit &emit) {
    using T = Tile<TY>;
    const int tid = threadIdx.x;
    const int q = tid & 15, ty = tid >> 4;
    uint32_t goff[T::LPT];
    int soff[T::LPT];
#pragma unroll
    for (int k = 0; k < T::LPT; ++k) {
        const int e = tid + k * T::NT;
        if (e < T::NLOAD) {
            const int r = e / T::CW, c = e - r * T::CW;
            const int gx = min(max(x0 - 2 + c, 0), (int)X - 1);
            const int gy = min(max(y0 - 2 + r, 0), (int)Y - 1);
            goff[k] = (uint32_t)gy * X + (uint32_t)gx;
            soff[k] = r * T::RW + c;
        } else {
            goff[k] = 0;
            soff[k] = -1;
        }
    }
    const size_t plane = (size_t)X * Y;
    uint32_t pre[T::LPT];
    auto fetch = [&](int zi) {
        const uint16_t *p = raw + (size_t)min(max(zi, 0), (int)Z - 1) * plane;
#pragma unroll
        for (int k = 0; k < T::LPT; ++k)
            if (soff[k] >= 0) pre[k] = __ldg(p + goff[k]);
    };
    uint32_t a0[4] = {0, 0, 0, 0}, a1[4] = {0, 0, 0, 0}, a2[4] = {0, 0, 0, 0}, a3[4] = {0, 0, 0, 0};
    fetch(z0 - 2);
    for (int zi = z0 - 2; zi < z1 + 2; ++zi) {
        __syncthreads();
#pragma unroll
        for (int k = 0; k < T::LPT; ++k)
            if (soff[k] >= 0) sraw[soff[k]] = pre[k];
        __syncthreads();
        if (zi + 1 < z1 + 2) fetch(zi + 1);
        for (int r = ty; r < T::RH; r += TY) {
            const uint4 u = *reinterpret_cast<const uint4 *>(sraw + r * T::RW + 4 * q);
            const uint4 w = *reinterpret_cast<const uint4 *>(sraw + r * T::RW + 4 * q + 4);
            uint4 o;
            o.x = u.x + 4u * u.y + 6u * u.z + 4u * u.w + w.x;
            o.y = u.y + 4u * u.z + 6u * u.w + 4u * w.x + w.y;
            o.z = u.z + 4u * u.w + 6u * w.x + 4u * w.y + w.z;
            o.w = u.w + 4u * w.x + 6u * w.y + 4u * w.z + w.w;
            *reinterpret_cast<uint4 *>(spx + r * TILE_X + 4 * q) = o;
        }
        __syncthreads();
        const uint4 r0 = *reinterpret_cast<const uint4 *>(spx + (ty + 0) * TILE_X + 4 * q);
        const uint4 r1 = *reinterpret_cast<const uint4 *>(spx + (ty + 1) * TILE_X + 4 * q);
        const uint4 r2 = *reinterpret_cast<const uint4 *>(spx + (ty + 2) * TILE_X + 4 * q);
        const uint4 r3 = *reinterpret_cast<const uint4 *>(spx + (ty + 3) * TILE_X + 4 * q);
        const uint4 r4 = *reinterpret_cast<const uint4 *>(spx + (ty + 4) * TILE_X + 4 * q);
        uint32_t p[4];
        p[0] = r0.x + 4u * r1.x + 6u * r2.x + 4u * r3.x + r4.x;
        p[1] = r0.y + 4u * r1.y + 6u * r2.y + 4u * r3.y + r4.y;
        p[2] = r0.z + 4u * r1.z + 6u * r2.z + 4u * r3.z + r4.z;
        p[3] = r0.w + 4u * r1.w + 6u * r2.w + 4u * r3.w + r4.w;
        uint32_t s[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const uint32_t out = a0[j] + p[j];
            a0[j] = a1[j] + 4u * p[j];
            a1[j] = a2[j] + 6u * p[j];
            a2[j] = a3[j] + 4u * p[j];
            a3[j] = p[j];
            s[j] = (out + 2048u) >> 12;
        }
        if (zi >= z0 + 2) emit(x0 + 4 * q, y0 + ty, zi - 2, s);
    }
}

// Histogram emit: two 16-bit counters per shared word.  The thread whose
// increment takes a counter to 0x8000 moves 0x8000 to the global bin, so a
// counter never exceeds 0x8000 + (increments in flight) < 0x10000 and never
// carries into its neighbour.
struct HistEmit {
    uint32_t *sh;
    uint32_t *gh;
    uint32_t X, Y;
    __device__ __forceinline__ void operator()(int xb, int y, int z, const uint32_t *s) {
        if ((uint32_t)y >= Y) return;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            if ((uint32_t)(xb + j) < X) {
                const uint32_t v = s[j];
                const uint32_t sft = (v & 1u) << 4;
                const uint32_t old = atomicAdd(sh + (v >> 1), 1u << sft);
                if (((old >> sft) & 0xFFFFu) == 0x7FFFu) {
                    atomicSub(sh + (v >> 1), 0x8000u << sft);
                    atomicAdd(gh + v, 0x8000u);
                }
            }
        }
    }
};

// Mask emit: 4 bits per thread, 8 lanes form one 32-bit word.
struct MaskEmit {
    uint32_t *mask;
    uint32_t X, Y, W, t;
    __device__ __forceinline__ void operator()(int xb, int y, int z, const uint32_t *s) {
        uint32_t nib = 0;
#pragma unroll
        for (int j = 0; j < 4; ++j)
            if ((uint32_t)(xb + j) < X && s[j] > t) nib |= 1u << j;
        const int lane = threadIdx.x & 31;
        uint32_t word = nib << (4 * (lane & 7));
        word |= __shfl_xor_sync(FULL, word, 1);
        word |= __shfl_xor_sync(FULL, word, 2);
        word |= __shfl_xor_sync(FULL, word, 4);
        if ((lane & 7) == 0 && (uint32_t)y < Y) {
            const uint32_t wi = (uint32_t)xb >> 5;
            if (wi < W) mask[((size_t)z * Y + (uint32_t)y) * W + wi] = word;
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

template <int NT>
__device__ void otsu_block(const uint32_t *__restrict__ gh, uint32_t *stat, uint64_t nvox) {
    constexpr int PER = HIST_BINS / NT;
    __shared__ unsigned long long s_n[32], s_s[32];
    __shared__ double s_bv[32];
    __shared__ uint32_t s_bt[32], s_mn[32];
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const uint32_t base = (uint32_t)tid * PER;
    unsigned long long n = 0, s = 0;
    for (int i = 0; i < PER; i += 4) {
        const uint4 c = __ldcg(reinterpret_cast<const uint4 *>(gh + base + i));
        const unsigned long long u = base + i;
        n += (unsigned long long)c.x + c.y + c.z + c.w;
        s += u * c.x + (u + 1) * c.y + (u + 2) * c.z + (u + 3) * c.w;
    }
    unsigned long long ni = n, si = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        unsigned long long a = __shfl_up_sync(FULL, ni, o), b = __shfl_up_sync(FULL, si, o);
        if (lane >= o) { ni += a; si += b; }
    }
    if (lane == 31) { s_n[wid] = ni; s_s[wid] = si; }
    __syncthreads();
    if (wid == 0) {
        unsigned long long wn = lane < NT / 32 ? s_n[lane] : 0ull;
        unsigned long long ws = lane < NT / 32 ? s_s[lane] : 0ull;
        unsigned long long in = wn, is = ws;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            unsigned long long a = __shfl_up_sync(FULL, in, o), b = __shfl_up_sync(FULL, is, o);
            if (lane >= o) { in += a; is += b; }
        }
        if (lane < NT / 32) { s_n[lane] = in - wn; s_s[lane] = is - ws; }
    }
    __syncthreads();
    __shared__ unsigned long long s_tot[2];
    if (tid == NT - 1) { s_tot[0] = s_n[wid] + ni; s_tot[1] = s_s[wid] + si; }
    __syncthreads();
    const unsigned long long Nt = s_tot[0], St = s_tot[1];
    unsigned long long n0 = s_n[wid] + ni - n;
    unsigned long long s0 = s_s[wid] + si - s;
    double best = -1.0;
    uint32_t bt = 0xFFFFFFFFu, mn = 0xFFFFFFFFu;
    for (int i = 0; i < PER; i += 4) {
        const uint4 c4 = __ldcg(reinterpret_cast<const uint4 *>(gh + base + i));
        const uint32_t cs[4] = {c4.x, c4.y, c4.z, c4.w};
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const uint32_t c = cs[j];
            if (!c) continue;
            const uint32_t u = base + i + j;
            if (mn == 0xFFFFFFFFu) mn = u;
            n0 += c;
            s0 += (unsigned long long)u * c;
            const unsigned long long n1 = Nt - n0;
            if (n1 == 0) continue;
            const unsigned long long s1 = St - s0;
            const double m0 = __ddiv_rn(__ull2double_rn(s0), __ull2double_rn(n0));
            const double m1 = __ddiv_rn(__ull2double_rn(s1), __ull2double_rn(n1));
            const double d = __dsub_rn(m1, m0);
            const double var =
                __dmul_rn(__dmul_rn(__dmul_rn(__ull2double_rn(n0), __ull2double_rn(n1)), d), d);
            if (var > best) { best = var; bt = u; }
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const double ov = __shfl_xor_sync(FULL, best, o);
        const uint32_t ot = __shfl_xor_sync(FULL, bt, o);
        const uint32_t om = __shfl_xor_sync(FULL, mn, o);
        if (ov > best || (ov == best && ot < bt)) { best = ov; bt = ot; }
        mn = min(mn, om);
    }
    if (lane == 0) { s_bv[wid] = best; s_bt[wid] = bt; s_mn[wid] = mn; }
    __syncthreads();
    if (wid == 0) {
        best = lane < NT / 32 ? s_bv[lane] : -1.0;
        bt = lane < NT / 32 ? s_bt[lane] : 0xFFFFFFFFu;
        mn = lane < NT / 32 ? s_mn[lane] : 0xFFFFFFFFu;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const double ov = __shfl_xor_sync(FULL, best, o);
            const uint32_t ot = __shfl_xor_sync(FULL, bt, o);
            const uint32_t om = __shfl_xor_sync(FULL, mn, o);
            if (ov > best || (ov == best && ot < bt)) { best = ov; bt = ot; }
            mn = min(mn, om);
        }
        if (lane == 0) {
            stat[ST_THRESH] = bt != 0xFFFFFFFFu ? bt : (mn != 0xFFFFFFFFu ? mn : 0u);
            if (Nt != nvox) atomicOr(stat + ST_ERROR, ERR_OTSU);
        }
    }
    __syncthreads();
}

// Merge the block's shared histogram into the volume's bins, then count the
// block's finished tiles; the block that completes the volume runs Otsu.
template <int NT>
__device__ void flush_hist(const BatchHdr *__restrict__ h, uint32_t v, uint32_t ndone, uint32_t *sh) {
    __shared__ uint32_t s_last;
    const VolDev &V = h->vol[v];
    __syncthreads();
    for (int i = threadIdx.x; i < HIST_WORDS / 4; i += NT) {
        uint4 w = reinterpret_cast<uint4 *>(sh)[i];
        if (w.x | w.y | w.z | w.w) {
            reinterpret_cast<uint4 *>(sh)[i] = make_uint4(0, 0, 0, 0);
            const uint32_t b = 8u * (uint32_t)i;
            const uint32_t ws[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                if (ws[j] & 0xFFFFu) atomicAdd(V.hist + b + 2 * j, ws[j] & 0xFFFFu);
                if (ws[j] >> 16) atomicAdd(V.hist + b + 2 * j + 1, ws[j] >> 16);
            }
        }
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        s_last = 0;
        if (ndone) {
            const uint32_t nt = V.ntx * V.nty * V.ntz;
            const uint32_t prev = atomicAdd(V.stat + ST_TILES_DONE, ndone);
            s_last = (prev + ndone == nt);
        }
    }
    __syncthreads();
    if (s_last) {
        __threadfence();
        otsu_block<NT>(V.hist, V.stat, (uint64_t)V.X * V.Y * V.Z);
    }
    __syncthreads();
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
    }
}

template <int TY>
__global__ void __launch_bounds__(16 * TY, 1) k_smooth_hist(const BatchHdr *__restrict__ h) {
    using T = Tile<TY>;
    extern __shared__ __align__(16) uint32_t smem[];
    uint32_t *sh = smem;
    uint32_t *sraw = sh + HIST_WORDS;
    uint32_t *spx = sraw + T::RAW_WORDS;
    for (int i = threadIdx.x; i < HIST_WORDS / 4; i += T::NT)
        reinterpret_cast<uint4 *>(sh)[i] = make_uint4(0, 0, 0, 0);
    __syncthreads();
    const uint32_t nt = h->ntiles, G = gridDim.x;
    const uint32_t tb = (uint32_t)(((uint64_t)nt * blockIdx.x) / G);
    const uint32_t te = (uint32_t)(((uint64_t)nt * (blockIdx.x + 1)) / G);
    if (tb >= te) return;
    uint32_t v = find_vol_tile(h, tb);
    uint32_t ndone = 0;
    const int tz = (int)h->tile_z;
    for (uint32_t t = tb; t < te; ++t) {
        while (v + 1 < h->nvol && t >= h->vol[v + 1].tile_base) {
            flush_hist<T::NT>(h, v, ndone, sh);
            ndone = 0;
            ++v;
        }
        const VolDev &V = h->vol[v];
        const uint32_t tl = t - V.tile_base;
        const uint32_t ix = tl % V.ntx, rest = tl / V.ntx;
        const uint32_t iy = rest % V.nty, iz = rest / V.nty;
        const int z0 = (int)iz * tz;
        const int z1 = min(z0 + tz, (int)V.Z);
        HistEmit e{sh, V.hist, V.X, V.Y};
        smooth_tile<TY>(V.raw, V.X, V.Y, V.Z, (int)ix * TILE_X, (int)iy * TY, z0, z1, sraw, spx, e);
        ++ndone;
    }
    flush_hist<T::NT>(h, v, ndone, sh);
}

template <int TY>
__global__ void __launch_bounds__(16 * TY) k_smooth_mask(const BatchHdr *__restrict__ h) {
    using T = Tile<TY>;
    extern __shared__ __align__(16) uint32_t smem[];
    uint32_t *sraw = smem;
    uint32_t *spx = sraw + T::RAW_WORDS;
    const int tz = (int)h->tile_z;
    for (uint32_t t = blockIdx.x; t < h->ntiles; t += gridDim.x) {
        const uint32_t v = find_vol_tile(h, t);
        const VolDev &V = h->vol[v];
        const uint32_t tl = t - V.tile_base;
        const uint32_t ix = tl % V.ntx, rest = tl / V.ntx;
        const uint32_t iy = rest % V.nty, iz = rest / V.nty;
        const int z0 = (int)iz * tz;
        const int z1 = min(z0 + tz, (int)V.Z);
        MaskEmit e{V.mask, V.X, V.Y, V.W, V.stat[ST_THRESH]};
        smooth_tile<TY>(V.raw, V.X, V.Y, V.Z, (int)ix * TILE_X, (int)iy * TY, z0, z1, sraw, spx, e);
    }
}

__global__ void __launch_bounds__(ROW_TILE) k_row_count(const BatchHdr *__restrict__ h) {
    __shared__ uint32_t sbuf[33];
    for (uint32_t rt = blockIdx.x; rt < h->nrowtiles; rt += gridDim.x) {
        const VolDev &V = h->vol[find_vol_rt(h, rt)];
        const uint32_t lt = rt - V.rt_base;
        const uint32_t row = lt * ROW_TILE + threadIdx.x;
        uint32_t cnt = 0;
        if (row < V.rows) {
            const uint32_t *m = V.mask + (size_t)row * V.W;
            uint32_t carry = 0;
            for (uint32_t w = 0; w < V.W; ++w) {
                const uint32_t x = m[w];
                cnt += __popc(x & ~((x << 1) | carry));
                carry = x >> 31;
            }
            V.rowoff[row] = cnt;
        }
        const uint32_t tot = block_sum<ROW_TILE>(cnt, sbuf);
        if (threadIdx.x == 0) V.tsum[lt] = tot;
    }
}

// Per-volume exclusive scan over row-tile totals; the grand total is R or K.
template <int WHICH>
__global__ void __launch_bounds__(1024) k_tile_scan(const BatchHdr *__restrict__ h) {
    __shared__ uint32_t sbuf[33];
    for (uint32_t v = blockIdx.x; v < h->nvol; v += gridDim.x) {
        const VolDev &V = h->vol[v];
        uint32_t *a = WHICH ? V.tkeep : V.tsum;
        uint32_t carry = 0;
        for (uint32_t b = 0; b < V.nrt; b += 1024) {
            const uint32_t i = b + threadIdx.x;
            const uint32_t x = i < V.nrt ? a[i] : 0u;
            uint32_t tot;
            const uint32_t ex = block_exscan<1024>(x, &tot, sbuf);
            if (i < V.nrt) a[i] = carry + ex;
            carry += tot;
        }
        if (threadIdx.x == 0) {
            if (WHICH == 0) {
                V.stat[ST_RUNS] = carry;
                if (carry > V.r_cap) atomicOr(V.stat + ST_ERROR, ERR_RCAP);
            } else {
                V.stat[ST_CELLS] = carry;
                if (carry > V.k_cap) atomicOr(V.stat + ST_ERROR, ERR_KCAP);
            }
        }
        __syncthreads();
    }
}

__global__ void __launch_bounds__(ROW_TILE) k_row_runs(const BatchHdr *__restrict__ h) {
    __shared__ uint32_t sbuf[33];
    for (uint32_t rt = blockIdx.x; rt < h->nrowtiles; rt += gridDim.x) {
        const VolDev &V = h->vol[find_vol_rt(h, rt)];
        const uint32_t lt = rt - V.rt_base;
        const uint32_t row = lt * ROW_TILE + threadIdx.x;
        const uint32_t cnt = row < V.rows ? V.rowoff[row] : 0u;
        uint32_t tot;
        const uint32_t ex = block_exscan<ROW_TILE>(cnt, &tot, sbuf);
        if (row < V.rows) {
            const uint32_t off = V.tsum[lt] + ex;
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
                                           uint32_t ie, uint32_t j, uint32_t je, uint32_t *err) {
    while (i < ie && j < je) {
        const uint32_t a = RX[i], b = RX[j];
        const uint32_t a0 = a & 0xFFFFu, a1 = a >> 16, b0 = b & 0xFFFFu, b1 = b >> 16;
        if (b1 + 1 < a0) { ++j; continue; }
        if (a1 + 1 < b0) { ++i; continue; }
        uf_union(P, i, j, err);
        if (a1 < b1) ++i; else ++j;
    }
}

__global__ void __launch_bounds__(ROW_TILE) k_union(const BatchHdr *__restrict__ h) {
    for (uint32_t rt = blockIdx.x; rt < h->nrowtiles; rt += gridDim.x) {
        const VolDev &V = h->vol[find_vol_rt(h, rt)];
        const uint32_t row = (rt - V.rt_base) * ROW_TILE + threadIdx.x;
        if (row >= V.rows) continue;
        const uint32_t ib = V.rowoff[row], ie = V.rowoff[row + 1];
        if (ib == ie) continue;
        const uint32_t y = row % V.Y, z = row / V.Y;
        uint32_t *err = V.stat + ST_ERROR;
        // backward neighbour rows: (y-1,z), (y-1,z-1), (y,z-1), (y+1,z-1)
        if (y > 0) {
            const uint32_t r = row - 1;
            unite_rows(V.run_par, V.run_x, ib, ie, V.rowoff[r], V.rowoff[r + 1], err);
        }
        if (z > 0) {
            const uint32_t rz = row - V.Y;
            if (y > 0) unite_rows(V.run_par, V.run_x, ib, ie, V.rowoff[rz - 1], V.rowoff[rz], err);
            unite_rows(V.run_par, V.run_x, ib, ie, V.rowoff[rz], V.rowoff[rz + 1], err);
            if (y + 1 < V.Y)
                unite_rows(V.run_par, V.run_x, ib, ie, V.rowoff[rz + 1], V.rowoff[rz + 2], err);
        }
    }
}

__global__ void __launch_bounds__(ROW_TILE) k_flatten(const BatchHdr *__restrict__ h) {
    for (uint32_t rt = blockIdx.x; rt < h->nrowtiles; rt += gridDim.x) {
        const VolDev &V = h->vol[find_vol_rt(h, rt)];
        const uint32_t row = (rt - V.rt_base) * ROW_TILE + threadIdx.x;
        if (row >= V.rows) continue;
        const uint32_t ib = V.rowoff[row], ie = V.rowoff[row + 1];
        for (uint32_t r = ib; r < ie; ++r) {
            const uint32_t root = uf_find(V.run_par, r);
            V.run_par[r] = root;
            const uint32_t x = V.run_x[r];
            atomicAdd(V.run_aux + root, (x >> 16) - (x & 0xFFFFu) + 1u);
        }
    }
}

__global__ void __launch_bounds__(ROW_TILE) k_keep_count(const BatchHdr *__restrict__ h) {
    __shared__ uint32_t sbuf[33];
    for (uint32_t rt = blockIdx.x; rt < h->nrowtiles; rt += gridDim.x) {
        const VolDev &V = h->vol[find_vol_rt(h, rt)];
        const uint32_t lt = rt - V.rt_base;
        const uint32_t row = lt * ROW_TILE + threadIdx.x;
        uint32_t cnt = 0;
        if (row < V.rows) {
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
    __shared__ uint32_t sbuf[33];
    for (uint32_t rt = blockIdx.x; rt < h->nrowtiles; rt += gridDim.x) {
        const VolDev &V = h->vol[find_vol_rt(h, rt)];
        const uint32_t lt = rt - V.rt_base;
        const uint32_t row = lt * ROW_TILE + threadIdx.x;
        const uint32_t cnt = row < V.rows ? V.rowk[row] : 0u;
        uint32_t tot;
        const uint32_t ex = block_exscan<ROW_TILE>(cnt, &tot, sbuf);
        if (row < V.rows) {
            uint32_t lab = V.tkeep[lt] + ex;
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

__global__ void __launch_bounds__(ROW_TILE) k_label_features(const BatchHdr *__restrict__ h) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr int WARPS = ROW_TILE / 32;
    for (uint32_t rt = blockIdx.x; rt < h->nrowtiles; rt += gridDim.x) {
        const VolDev &V = h->vol[find_vol_rt(h, rt)];
        const uint32_t lt = rt - V.rt_base;
        for (uint32_t rr = warp; rr < ROW_TILE; rr += WARPS) {
            const uint32_t row = lt * ROW_TILE + rr;
            if (row >= V.rows) break;
            const uint32_t X = V.X;
            uint32_t *out = V.labels + (size_t)row * X;
            const uint32_t ib = V.rowoff[row], ie = V.rowoff[row + 1];
            if (ib == ie) {
                for (uint32_t x = lane; x < X; x += 32) out[x] = 0u;
                continue;
            }
            const uint32_t y = row % V.Y, z = row / V.Y;
            for (uint32_t r = ib + lane; r < ie; r += 32) {
                const uint32_t lab = V.run_aux[V.run_par[r]];
                if (!lab || lab > V.k_cap) continue;
                const uint32_t rx = V.run_x[r];
                const uint32_t x0 = rx & 0xFFFFu, x1 = rx >> 16;
                const unsigned long long len = x1 - x0 + 1u;
                seg_cell_features *f = V.feat + (lab - 1);
                atomicAdd(reinterpret_cast<unsigned long long *>(&f->count), len);
                atomicAdd(reinterpret_cast<unsigned long long *>(&f->sum[0]),
                          ((unsigned long long)(x0 + x1) * len) >> 1);
                atomicAdd(reinterpret_cast<unsigned long long *>(&f->sum[1]), len * y);
                atomicAdd(reinterpret_cast<unsigned long long *>(&f->sum[2]), len * z);
                atomicMin(&f->bbox_min[0], x0);
                atomicMax(&f->bbox_max[0], x1);
                atomicMin(&f->bbox_min[1], y);
                atomicMax(&f->bbox_max[1], y);
                atomicMin(&f->bbox_min[2], z);
                atomicMax(&f->bbox_max[2], z);
            }
            uint32_t j = ib;
            for (uint32_t x = lane; x < X; x += 32) {
                while (j < ie && (V.run_x[j] >> 16) < x) ++j;
                uint32_t lab = 0;
                if (j < ie && (V.run_x[j] & 0xFFFFu) <= x) lab = V.run_aux[V.run_par[j]];
                out[x] = lab;
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

template <int TY>
cudaError_t launch_tile_kernels(const BatchHdr *d, const LaunchPlan &p, cudaStream_t s,
                                cudaEvent_t *ev, int &k) {
    auto rec = [&]() {
        if (ev) cudaEventRecordWithFlags(ev[k], s, cudaEventRecordExternal);
        ++k;
    };
    rec();
    k_smooth_hist<TY><<<p.grid_hist, 16 * TY, hist_smem_bytes(TY), s>>>(d);
    rec();
    k_smooth_mask<TY><<<p.grid_mask, 16 * TY, mask_smem_bytes(TY), s>>>(d);
    return cudaGetLastError();
}

}  // namespace

size_t hist_smem_bytes(int tile_y) {
    const int rh = tile_y + 4;
    return (size_t)4 * (HIST_WORDS + rh * (TILE_X + 8) + rh * TILE_X);
}

size_t mask_smem_bytes(int tile_y) {
    const int rh = tile_y + 4;
    return (size_t)4 * (rh * (TILE_X + 8) + rh * TILE_X);
}

cudaError_t configure_kernels(int device) {
    cudaError_t e = cudaSetDevice(device);
    if (e != cudaSuccess) return e;
#define SEG_CFG(TY)                                                                        \
    e = cudaFuncSetAttribute(k_smooth_hist<TY>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                             (int)hist_smem_bytes(TY));                                    \
    if (e != cudaSuccess) return e;                                                        \
    e = cudaFuncSetAttribute(k_smooth_mask<TY>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                             (int)mask_smem_bytes(TY));                                    \
    if (e != cudaSuccess) return e;
    SEG_CFG(8)
    SEG_CFG(16)
    SEG_CFG(32)
#undef SEG_CFG
    return cudaSuccess;
}

cudaError_t launch_pipeline(const BatchHdr *d, const LaunchPlan &p, cudaStream_t s, cudaEvent_t *ev,
                            uint32_t *stat_out) {
    int k = 0;
    auto rec = [&]() {
        if (ev) cudaEventRecordWithFlags(ev[k], s, cudaEventRecordExternal);
        ++k;
    };
    rec();
    k_init<<<p.grid_vols * 4, 256, 0, s>>>(d);
    cudaError_t e;
    switch (p.tile_y) {
        case 8: e = launch_tile_kernels<8>(d, p, s, ev, k); break;
        case 16: e = launch_tile_kernels<16>(d, p, s, ev, k); break;
        default: e = launch_tile_kernels<32>(d, p, s, ev, k); break;
    }
    if (e != cudaSuccess) return e;
    rec();
    k_row_count<<<p.grid_rows, ROW_TILE, 0, s>>>(d);
    rec();
    k_tile_scan<0><<<p.grid_vols, 1024, 0, s>>>(d);
    rec();
    k_row_runs<<<p.grid_rows, ROW_TILE, 0, s>>>(d);
    rec();
    k_union<<<p.grid_rows, ROW_TILE, 0, s>>>(d);
    rec();
    k_flatten<<<p.grid_rows, ROW_TILE, 0, s>>>(d);
    rec();
    k_keep_count<<<p.grid_rows, ROW_TILE, 0, s>>>(d);
    rec();
    k_tile_scan<1><<<p.grid_vols, 1024, 0, s>>>(d);
    rec();
    k_rank<<<p.grid_rows, ROW_TILE, 0, s>>>(d);
    rec();
    k_label_features<<<p.grid_rows, ROW_TILE, 0, s>>>(d);
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
__global__ void __launch_bounds__(16 * TY, 1) k_smooth_hist_noalloc(const __grid_constant__ BatchHdr hdr) {
    using T = Tile<TY>;
    const BatchHdr *h = &hdr;
    extern __shared__ __align__(16) uint32_t smem[];
    uint32_t *sh = smem;
    uint32_t *sraw = sh + HIST_WORDS;
    uint32_t *spx = sraw + T::RAW_WORDS;
    for (int i = threadIdx.x; i < HIST_WORDS / 4; i += T::NT)
        reinterpret_cast<uint4 *>(sh)[i] = make_uint4(0, 0, 0, 0);
    __syncthreads();
    const uint32_t nt = h->ntiles, G = gridDim.x;
    const uint32_t tb = (uint32_t)(((uint64_t)nt * blockIdx.x) / G);
    const uint32_t te = (uint32_t)(((uint64_t)nt * (blockIdx.x + 1)) / G);
    if (tb >= te) return;
    const VolDev &V = h->vol[0];
    const int tz = (int)h->tile_z;
    uint32_t ndone = 0;
    for (uint32_t t = tb; t < te; ++t) {
        const uint32_t ix = t % V.ntx, rest = t / V.ntx;
        const uint32_t iy = rest % V.nty, iz = rest / V.nty;
        const int z0 = (int)iz * tz;
        const int z1 = min(z0 + tz, (int)V.Z);
        HistEmit e{sh, V.hist, V.X, V.Y};
        smooth_tile<TY>(V.raw, V.X, V.Y, V.Z, (int)ix * TILE_X, (int)iy * TY, z0, z1, sraw, spx, e);
        ++ndone;
    }
    flush_hist<T::NT>(h, 0, ndone, sh);
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
    const uint64_t n = (uint64_t)dims.x * dims.y * dims.z;
    if (n > SEG_NOALLOC_MAX_VOXELS || dims.x > 65536u) return SEG_ETOOBIG;
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
    V.ntx = (dims.x + TILE_X - 1) / TILE_X;
    V.nty = (dims.y + NOALLOC_TY - 1) / NOALLOC_TY;
    V.ntz = (dims.z + NOALLOC_TZ - 1) / NOALLOC_TZ;
    hdr.nvol = 1;
    hdr.ntiles = V.ntx * V.nty * V.ntz;
    hdr.tile_z = NOALLOC_TZ;
    hdr.tile_y = NOALLOC_TY;
    // the array keeps the previous call's contents: clear bins and counters
    cudaError_t e = cudaMemsetAsync(scratch, 0, sizeof(uint32_t) * NOALLOC_WORDS, s);
    if (e == cudaSuccess) {
        k_smooth_hist_noalloc<NOALLOC_TY><<<sms, 16 * NOALLOC_TY, hist_smem_bytes(NOALLOC_TY), s>>>(hdr);
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
