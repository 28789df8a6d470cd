// seg_montage.cu -- montage registration (Registration section, Eq. 4):
// overlapping tiles are scored at every shift of a search window by the
// normalized covariance of their shared voxels, each overlapping pair keeps
// its best shift, and a maximum spanning tree of the pairs gives every tile
// its correction relative to an anchored one.
//
// Per pair and shift s the score needs six exact integer sums over the
// shared box: N, Sa, Sb, Saa, Sbb and Sab.  The GPU computes
//   * Sab for all shifts at once (k_reg_corr): a block stages a sub-box of
//     tile a and the matching region of tile b widened by the window (b
//     zero outside its box, so no bounds test per product), and each thread
//     takes shifts, summing the products over the sub-box from shared
//     memory;
//   * Sa, Saa (tile a) and Sb, Sbb (tile b) from the x-range sums of every
//     row (k_reg_rows), their prefixes along y per x-range and plane
//     (k_reg_q), then per shift a sum over the planes of its box
//     (k_reg_box), because the shared box varies only at its faces.
// The host then forms the Pearson correlation in 128-bit integers and
// binary64, picks the first best shift in z, y, x order, builds the maximum
// spanning tree (Kruskal) and sums the shifts from the root.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <numeric>
#include <utility>
#include <vector>

#include "seg.h"

namespace {

constexpr int RC_TX = 32, RC_TY = 8, RC_TZ = 8;  // tile-a sub-box of a k_reg_corr block
constexpr int RC_THREADS = 256;

// Half-open range [lo, hi) of one axis.
struct Range {
    int lo, hi;
};

// Shared range along one axis for tile b's origin at d in tile a's frame:
// in a's coordinates (side 0) or in b's (side 1).
__host__ __device__ inline Range shared_range(int d, int D, int side) {
    if (side == 0) return Range{d > 0 ? d : 0, d + D < D ? d + D : D};
    return Range{-d > 0 ? -d : 0, D - d < D ? D - d : D};
}

// Sab for every shift: block = sub-box (RC_TX x RC_TY x RC_TZ) of tile a's
// search region U (in a's coordinates).  Shift index
// si = ((sz + rz) SY + (sy + ry)) SX + (sx + rx).  Thread (g, c) takes the
// (y, z)-shift g = (sy, sz) for every x-shift (KX = 2 RX + 1 of them) over
// the sub-box rows c, c + C, ...: along a row the x-shifts need b values
// x + 2 RX - k, so a register window of KX b values slides with x and every
// product costs one multiply-add.  The threads' sums meet in shared memory
// and go out with one atomic per (block, shift).
template <int RX>
__global__ void __launch_bounds__(RC_THREADS) k_reg_corr(const uint16_t *__restrict__ A, const uint16_t *__restrict__ B,
                                                         int X, int Y, int Z, int3 u0, int3 u1, int3 d0, int ry,
                                                         int rz, unsigned long long *__restrict__ sab) {
    constexpr int KX = 2 * RX + 1;
    constexpr int BX = RC_TX + 2 * RX;
    extern __shared__ __align__(16) unsigned long long rsm64[];
    const int BY = RC_TY + 2 * ry, BZ = RC_TZ + 2 * rz, SY = 2 * ry + 1, G = SY * (2 * rz + 1);
    unsigned long long *red = rsm64;                                      // [G][KX]
    uint16_t *As = reinterpret_cast<uint16_t *>(rsm64 + (size_t)G * KX);  // [RC_TZ][RC_TY][RC_TX]
    uint16_t *Bs = As + RC_TX * RC_TY * RC_TZ;                            // [BZ][BY][BX]
    const int nbx = (u1.x - u0.x + RC_TX - 1) / RC_TX, nby = (u1.y - u0.y + RC_TY - 1) / RC_TY;
    const int bi = (int)blockIdx.x;
    const int ax0 = u0.x + (bi % nbx) * RC_TX, ay0 = u0.y + ((bi / nbx) % nby) * RC_TY;
    const int az0 = u0.z + (bi / (nbx * nby)) * RC_TZ;
    for (int i = threadIdx.x; i < G * KX; i += RC_THREADS) red[i] = 0ull;
    for (int i = threadIdx.x; i < RC_TX * RC_TY * RC_TZ; i += RC_THREADS) {
        const int x = ax0 + i % RC_TX, y = ay0 + (i / RC_TX) % RC_TY, z = az0 + i / (RC_TX * RC_TY);
        As[i] = (x < u1.x && y < u1.y && z < u1.z) ? A[((size_t)z * Y + y) * X + x] : (uint16_t)0;
    }
    // b coordinates of a's sub-box under every shift: a - d0 - s
    const int bx0 = ax0 - d0.x - RX, by0 = ay0 - d0.y - ry, bz0 = az0 - d0.z - rz;
    for (int i = threadIdx.x; i < BX * BY * BZ; i += RC_THREADS) {
        const int x = bx0 + i % BX, y = by0 + (i / BX) % BY, z = bz0 + i / (BX * BY);
        Bs[i] = (x >= 0 && x < X && y >= 0 && y < Y && z >= 0 && z < Z) ? B[((size_t)z * Y + y) * X + x]
                                                                       : (uint16_t)0;
    }
    __syncthreads();
    constexpr int ROWS = RC_TY * RC_TZ;
    const int C = G >= RC_THREADS ? 1 : min(ROWS, RC_THREADS / G);  // row chunks per shift group
    for (int w = threadIdx.x; w < G * C; w += RC_THREADS) {
        const int g = w % G, c = w / G;
        const int sy = g % SY - ry, sz = g / SY - rz;
        unsigned long long acc[KX];
#pragma unroll
        for (int k = 0; k < KX; ++k) acc[k] = 0ull;
        for (int row = c; row < ROWS; row += C) {
            const int y = row % RC_TY, z = row / RC_TY;
            const uint16_t *ar = As + row * RC_TX;
            const uint16_t *br = Bs + ((z - sz + rz) * BY + (y - sy + ry)) * BX;
            uint32_t win[KX];  // b at x .. x + 2 RX
#pragma unroll
            for (int j = 0; j < KX - 1; ++j) win[j + 1] = br[j];
#pragma unroll
            for (int x = 0; x < RC_TX; ++x) {
#pragma unroll
                for (int j = 0; j < KX - 1; ++j) win[j] = win[j + 1];
                win[KX - 1] = br[x + 2 * RX];
                const uint32_t a = ar[x];
#pragma unroll
                for (int k = 0; k < KX; ++k) acc[k] += (unsigned long long)(a * win[2 * RX - k]);
            }
        }
#pragma unroll
        for (int k = 0; k < KX; ++k)
            if (acc[k]) atomicAdd(red + g * KX + k, acc[k]);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < G * KX; i += RC_THREADS)
        if (red[i]) atomicAdd(sab + i, red[i]);
}

// Shared memory of k_reg_corr<RX>.
size_t reg_corr_smem(int rx, int ry, int rz) {
    const size_t G = (size_t)(2 * ry + 1) * (2 * rz + 1), KX = 2 * rx + 1;
    return 8 * G * KX + 2 * ((size_t)RC_TX * RC_TY * RC_TZ +
                             (size_t)(RC_TX + 2 * rx) * (RC_TY + 2 * ry) * (RC_TZ + 2 * rz));
}

using RegCorrFn = void (*)(const uint16_t *, const uint16_t *, int, int, int, int3, int3, int3, int, int,
                           unsigned long long *);
template <int... R>
RegCorrFn reg_corr_fn(int rx, std::integer_sequence<int, R...>) {
    RegCorrFn f = nullptr;
    ((rx == R ? (f = k_reg_corr<R>, 0) : 0), ...);
    return f;
}

// Per row (y, z) of the region U of one tile and x-shift sxi: the sums of v
// and v^2 over the shift's x-range, R[sxi rows + row] with row =
// (z - u0.z) UY + (y - u0.y).  One warp per row: the part of the row every
// x-range shares (the core) is summed by all lanes and reduced; lane sxi then
// adds its range's voxels outside the core (at most 2 rx of them).
__global__ void k_reg_rows(const uint16_t *__restrict__ T, int X, int Y, int3 u0, int3 u1, int d0x, int rx, int side,
                           unsigned long long *__restrict__ r1, unsigned long long *__restrict__ r2) {
    const int UY = u1.y - u0.y, rows = UY * (u1.z - u0.z), SX = 2 * rx + 1;
    const int lane = threadIdx.x & 31;
    const Range first = shared_range(d0x - rx, X, side), last = shared_range(d0x + rx, X, side);
    // ranges move monotonically with the shift: the core is [max lo, min hi)
    const int clo = max(first.lo, last.lo), chi = min(first.hi, last.hi);
    const int nw = (gridDim.x * blockDim.x) >> 5;
    for (int row = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; row < rows; row += nw) {
        const int y = u0.y + row % UY, z = u0.z + row / UY;
        const uint16_t *t = T + ((size_t)z * Y + y) * X;
        unsigned long long a = 0, b = 0;
        for (int x = clo + lane; x < chi; x += 32) {
            const unsigned long long v = t[x];
            a += v;
            b += v * v;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            a += __shfl_xor_sync(0xFFFFFFFFu, a, o);
            b += __shfl_xor_sync(0xFFFFFFFFu, b, o);
        }
        if (lane < SX) {
            const Range q = shared_range(d0x + lane - rx, X, side);
            if (clo >= chi) {  // no core: the whole range
                a = b = 0;
                for (int x = q.lo; x < q.hi; ++x) {
                    const unsigned long long v = t[x];
                    a += v;
                    b += v * v;
                }
            } else if (q.lo >= q.hi) {
                a = b = 0;
            } else {
                for (int x = q.lo; x < clo; ++x) {
                    const unsigned long long v = t[x];
                    a += v;
                    b += v * v;
                }
                for (int x = chi; x < q.hi; ++x) {
                    const unsigned long long v = t[x];
                    a += v;
                    b += v * v;
                }
            }
            r1[(size_t)lane * rows + row] = a;
            r2[(size_t)lane * rows + row] = b;
        }
    }
}

// For every x-shift and plane of U: prefix along y of the rows' sums over the
// shift's x-range.  Q[(sxi (UZ) + z - u0.z) (UY + 1) + j].  One block per
// (x-shift, plane): each thread sums a run of consecutive rows, a block scan
// of the run totals gives each run's start, then the runs are written.
constexpr int RQ_THREADS = 256;
__global__ void __launch_bounds__(RQ_THREADS) k_reg_q(const unsigned long long *__restrict__ r1,
                                                      const unsigned long long *__restrict__ r2, int3 u0, int3 u1,
                                                      unsigned long long *__restrict__ q1,
                                                      unsigned long long *__restrict__ q2) {
    __shared__ unsigned long long t1[RQ_THREADS], t2[RQ_THREADS];
    const int UY = u1.y - u0.y, UZ = u1.z - u0.z, rows = UY * UZ;
    const int i = (int)blockIdx.x, sxi = i / UZ, zz = i % UZ;
    const unsigned long long *s1 = r1 + (size_t)sxi * rows + (size_t)zz * UY;
    const unsigned long long *s2 = r2 + (size_t)sxi * rows + (size_t)zz * UY;
    const int per = (UY + RQ_THREADS - 1) / RQ_THREADS, j0 = threadIdx.x * per, j1 = min(j0 + per, UY);
    unsigned long long a = 0, b = 0;
    for (int j = j0; j < j1; ++j) {
        a += s1[j];
        b += s2[j];
    }
    t1[threadIdx.x] = a;
    t2[threadIdx.x] = b;
    __syncthreads();
    // inclusive scan of the run totals (Hillis-Steele)
    for (int o = 1; o < RQ_THREADS; o <<= 1) {
        const unsigned long long x = threadIdx.x >= o ? t1[threadIdx.x - o] : 0ull;
        const unsigned long long y = threadIdx.x >= o ? t2[threadIdx.x - o] : 0ull;
        __syncthreads();
        t1[threadIdx.x] += x;
        t2[threadIdx.x] += y;
        __syncthreads();
    }
    unsigned long long *o1 = q1 + (size_t)i * (UY + 1), *o2 = q2 + (size_t)i * (UY + 1);
    a = t1[threadIdx.x] - a;  // exclusive start of this run
    b = t2[threadIdx.x] - b;
    if (threadIdx.x == 0) {
        o1[0] = 0;
        o2[0] = 0;
    }
    for (int j = j0; j < j1; ++j) {
        a += s1[j];
        b += s2[j];
        o1[j + 1] = a;
        o2[j + 1] = b;
    }
}

// Per shift: the sums of v and v^2 over the tile's shared box; one warp per
// shift, lanes over the planes of the box.
__global__ void k_reg_box(const unsigned long long *__restrict__ q1, const unsigned long long *__restrict__ q2,
                          int X, int Y, int Z, int3 u0, int3 u1, int3 d0, int3 r, int side,
                          unsigned long long *__restrict__ s1, unsigned long long *__restrict__ s2) {
    const int UY = u1.y - u0.y, UZ = u1.z - u0.z, lane = threadIdx.x & 31;
    const int SX = 2 * r.x + 1, SY = 2 * r.y + 1, S = SX * SY * (2 * r.z + 1);
    const int nw = (gridDim.x * blockDim.x) >> 5;
    for (int si = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; si < S; si += nw) {
        const int sxi = si % SX, sy = (si / SX) % SY - r.y, sz = si / (SX * SY) - r.z;
        const Range xr = shared_range(d0.x + sxi - r.x, X, side);
        const Range yr = shared_range(d0.y + sy, Y, side), zr = shared_range(d0.z + sz, Z, side);
        unsigned long long a = 0, b = 0;
        if (xr.lo < xr.hi && yr.lo < yr.hi && zr.lo < zr.hi) {
            for (int z = zr.lo + lane; z < zr.hi; z += 32) {
                const size_t q = (size_t)(sxi * UZ + (z - u0.z)) * (UY + 1);
                a += q1[q + (yr.hi - u0.y)] - q1[q + (yr.lo - u0.y)];
                b += q2[q + (yr.hi - u0.y)] - q2[q + (yr.lo - u0.y)];
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            a += __shfl_xor_sync(0xFFFFFFFFu, a, o);
            b += __shfl_xor_sync(0xFFFFFFFFu, b, o);
        }
        if (lane == 0) {
            s1[si] = a;
            s2[si] = b;
        }
    }
}

int fail(cudaError_t e) {
    if (e == cudaSuccess) return SEG_OK;
    cudaGetLastError();
    return SEG_ECUDA;
}

#define RK(call)                                 \
    do {                                         \
        const cudaError_t e__ = (call);          \
        if (e__ != cudaSuccess) return fail(e__); \
    } while (0)

// Device buffers of one registration call, freed on every return path.
// Device scratch of one call, from the stream-ordered pool on stream s, and
// REG_STREAMS worker streams that take the pairs in turn.
constexpr int REG_STREAMS = 4;

struct Scratch {
    std::vector<void *> ptrs;
    cudaStream_t s = nullptr;
    cudaStream_t w[REG_STREAMS] = {};
    cudaEvent_t ev[REG_STREAMS + 1] = {};
    ~Scratch() {
        if (s && w[REG_STREAMS - 1] && ev[REG_STREAMS - 1]) join();  // frees wait for the worker streams too
        for (void *p : ptrs) cudaFreeAsync(p, s);
        if (s) cudaStreamSynchronize(s);
        for (int k = 0; k < REG_STREAMS; ++k)
            if (w[k]) cudaStreamDestroy(w[k]);
        for (int k = 0; k <= REG_STREAMS; ++k)
            if (ev[k]) cudaEventDestroy(ev[k]);
        if (s) cudaStreamDestroy(s);
    }
    cudaError_t init() {
        cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
        for (int k = 0; k < REG_STREAMS && e == cudaSuccess; ++k)
            e = cudaStreamCreateWithFlags(&w[k], cudaStreamNonBlocking);
        for (int k = 0; k <= REG_STREAMS && e == cudaSuccess; ++k)
            e = cudaEventCreateWithFlags(&ev[k], cudaEventDisableTiming);
        return e;
    }
    template <class T>
    cudaError_t alloc(T **p, size_t n) {
        void *q = nullptr;
        const cudaError_t e = cudaMallocAsync(&q, n ? n * sizeof(T) : 1, s);
        if (e == cudaSuccess) ptrs.push_back(q);
        *p = static_cast<T *>(q);
        return e;
    }
    // the worker streams wait for everything queued on s so far
    cudaError_t fork() {
        cudaError_t e = cudaEventRecord(ev[REG_STREAMS], s);
        for (int k = 0; k < REG_STREAMS && e == cudaSuccess; ++k) e = cudaStreamWaitEvent(w[k], ev[REG_STREAMS], 0);
        return e;
    }
    // s waits for everything queued on the worker streams so far
    cudaError_t join() {
        cudaError_t e = cudaSuccess;
        for (int k = 0; k < REG_STREAMS && e == cudaSuccess; ++k) {
            e = cudaEventRecord(ev[k], w[k]);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(s, ev[k], 0);
        }
        return e;
    }
};

// Search region of one side (0: tile a, 1: tile b) in that tile's frame:
// the union over the window of the shared boxes.
void side_region(const int *d0, const int *r, const int *D, int side, int3 &u0, int3 &u1) {
    int lo[3], hi[3];
    for (int k = 0; k < 3; ++k) {
        const Range a = shared_range(d0[k] - r[k], D[k], side), b = shared_range(d0[k] + r[k], D[k], side);
        lo[k] = std::min(a.lo, b.lo);
        hi[k] = std::max(a.hi, b.hi);
        if (lo[k] > hi[k]) hi[k] = lo[k];
    }
    u0 = make_int3(lo[0], lo[1], lo[2]);
    u1 = make_int3(hi[0], hi[1], hi[2]);
}

// Entries of the prefix buffers one side of a pair needs.
void side_sizes(const int *D, const int *d0, const int *r, int side, size_t &np, size_t &nq) {
    int3 u0, u1;
    side_region(d0, r, D, side, u0, u1);
    const size_t UX = (size_t)(u1.x - u0.x), UY = (size_t)(u1.y - u0.y), UZ = (size_t)(u1.z - u0.z);
    np = (size_t)(2 * r[0] + 1) * UY * UZ * (UX > 0 ? 1 : 0);
    nq = (size_t)(2 * r[0] + 1) * UZ * (UY + 1);
}

// Buffers (p1, p2: x-range sums per row; q1, q2: prefixes along y), sized
// for the largest side.
struct Prefix {
    unsigned long long *p1, *p2, *q1, *q2;
};

// Sa, Saa (side 0) or Sb, Sbb (side 1) of every shift.
int side_sums(cudaStream_t st, const Prefix &pf, const uint16_t *T, const int *D, const int *d0, const int *r,
              int side, unsigned long long *s1, unsigned long long *s2) {
    int3 u0, u1;
    side_region(d0, r, D, side, u0, u1);
    const int UX = u1.x - u0.x, UY = u1.y - u0.y, UZ = u1.z - u0.z;
    const int SX = 2 * r[0] + 1, S = SX * (2 * r[1] + 1) * (2 * r[2] + 1);
    if (UX <= 0 || UY <= 0 || UZ <= 0) {
        RK(cudaMemsetAsync(s1, 0, S * sizeof(unsigned long long), st));
        RK(cudaMemsetAsync(s2, 0, S * sizeof(unsigned long long), st));
        return SEG_OK;
    }
    unsigned long long *p1 = pf.p1, *p2 = pf.p2, *q1 = pf.q1, *q2 = pf.q2;
    const int rows = UY * UZ;
    k_reg_rows<<<(rows + 7) / 8, 256, 0, st>>>(T, D[0], D[1], u0, u1, d0[0], r[0], side, p1, p2);
    k_reg_q<<<SX * UZ, RQ_THREADS, 0, st>>>(p1, p2, u0, u1, q1, q2);
    k_reg_box<<<(S + 7) / 8, 256, 0, st>>>(q1, q2, D[0], D[1], D[2], u0, u1, make_int3(d0[0], d0[1], d0[2]),
                                             make_int3(r[0], r[1], r[2]), side, s1, s2);
    RK(cudaGetLastError());
    return SEG_OK;
}

uint32_t uf_root(std::vector<uint32_t> &p, uint32_t i) {
    while (p[i] != i) {
        p[i] = p[p[i]];
        i = p[i];
    }
    return i;
}

}  // namespace

extern "C" int seg_register_montage(int device, const uint16_t *const *tiles, int on_device, uint32_t n_tiles,
                                    seg_dims dims, const seg_offset *stage, seg_offset radius, uint32_t root,
                                    seg_offset *delta, seg_montage_edge *edges, uint32_t edges_cap,
                                    uint32_t *n_edges) {
    if (!tiles || !stage || !delta || !n_edges || n_tiles == 0 || root >= n_tiles || dims.x == 0 || dims.y == 0 ||
        dims.z == 0)
        return SEG_EINVAL;
    if (radius.x < 0 || radius.y < 0 || radius.z < 0 || radius.x > SEG_REG_MAX_RXY || radius.y > SEG_REG_MAX_RXY ||
        radius.z > SEG_REG_MAX_RZ)
        return SEG_EINVAL;
    for (uint32_t i = 0; i < n_tiles; ++i)
        if (!tiles[i]) return SEG_EINVAL;
    const uint64_t n = (uint64_t)dims.x * dims.y * dims.z;
    if (n >= (1ull << 32) || dims.x > 0x7FFFFFFFu || dims.y > 0x7FFFFFFFu || dims.z > 0x7FFFFFFFu)
        return SEG_ETOOBIG;
    const int D[3] = {(int)dims.x, (int)dims.y, (int)dims.z};
    const int r[3] = {radius.x, radius.y, radius.z};
    // pairs whose stage boxes overlap, in (a, b) order
    std::vector<seg_montage_edge> E;
    for (uint32_t a = 0; a < n_tiles; ++a)
        for (uint32_t b = a + 1; b < n_tiles; ++b) {
            const int64_t o[3] = {(int64_t)stage[b].x - stage[a].x, (int64_t)stage[b].y - stage[a].y,
                                  (int64_t)stage[b].z - stage[a].z};
            bool ov = true;
            for (int k = 0; k < 3; ++k) ov = ov && o[k] < D[k] && -o[k] < D[k];
            if (!ov) continue;
            seg_montage_edge e;
            std::memset(&e, 0, sizeof(e));
            e.a = a;
            e.b = b;
            e.score = -2.0;
            E.push_back(e);
        }
    *n_edges = (uint32_t)E.size();
    if (E.size() > edges_cap || (!edges && !E.empty())) return SEG_ESMALL;

    RK(cudaSetDevice(device));
    {
        // keep freed scratch in the pool between calls
        cudaMemPool_t pool;
        if (cudaDeviceGetDefaultMemPool(&pool, device) == cudaSuccess) {
            uint64_t thr = UINT64_MAX;
            cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
        }
        cudaGetLastError();
    }
    Scratch sc;
    RK(sc.init());
    // the tiles on the device
    std::vector<const uint16_t *> dt(n_tiles);
    if (on_device) {
        for (uint32_t i = 0; i < n_tiles; ++i) dt[i] = tiles[i];
    } else {
        for (uint32_t i = 0; i < n_tiles; ++i) {
            uint16_t *p;
            RK(sc.alloc(&p, n));
            RK(cudaMemcpyAsync(p, tiles[i], 2 * n, cudaMemcpyHostToDevice, sc.s));
            dt[i] = p;
        }
    }
    const int SX = 2 * r[0] + 1, SY = 2 * r[1] + 1, S = SX * SY * (2 * r[2] + 1);
    // Pairs go in groups of up to REG_GROUP: every pair of a group gets its
    // own slice of sums (Sab, Sa, Saa, Sb, Sbb of every shift), the group's
    // kernels are queued back to back, and one copy and one synchronisation
    // bring its sums to the host.
    constexpr size_t REG_GROUP = 64;
    const size_t per = 5 * (size_t)S;
    const size_t gmax = std::max<size_t>(1, std::min(E.size(), REG_GROUP));
    unsigned long long *dsum;
    RK(sc.alloc(&dsum, per * gmax));
    std::vector<unsigned long long> hs(per * gmax);
    size_t np = 1, nq = 1;
    for (const seg_montage_edge &e : E) {
        const int d0[3] = {stage[e.b].x - stage[e.a].x, stage[e.b].y - stage[e.a].y, stage[e.b].z - stage[e.a].z};
        for (int side = 0; side < 2; ++side) {
            size_t a, b;
            side_sizes(D, d0, r, side, a, b);
            np = std::max(np, a);
            nq = std::max(nq, b);
        }
    }
    Prefix pf[REG_STREAMS];
    for (int k = 0; k < REG_STREAMS; ++k) {
        RK(sc.alloc(&pf[k].p1, np));
        RK(sc.alloc(&pf[k].p2, np));
        RK(sc.alloc(&pf[k].q1, nq));
        RK(sc.alloc(&pf[k].q2, nq));
    }
    const size_t smem = reg_corr_smem(r[0], r[1], r[2]);
    const RegCorrFn corr = reg_corr_fn(r[0], std::make_integer_sequence<int, SEG_REG_MAX_RXY + 1>{});
    if (!corr) return SEG_EINVAL;
    RK(cudaFuncSetAttribute(corr, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    for (size_t g0 = 0; g0 < E.size(); g0 += REG_GROUP) {
        const size_t g1 = std::min(E.size(), g0 + REG_GROUP);
        RK(sc.fork());
        for (size_t ei = g0; ei < g1; ++ei) {
            const seg_montage_edge &e = E[ei];
            unsigned long long *ds = dsum + per * (ei - g0);
            const int k = (int)(ei % REG_STREAMS);
            const cudaStream_t st = sc.w[k];
            const int d0[3] = {stage[e.b].x - stage[e.a].x, stage[e.b].y - stage[e.a].y,
                               stage[e.b].z - stage[e.a].z};
            RK(cudaMemsetAsync(ds, 0, S * sizeof(unsigned long long), st));
            int3 u0, u1;
            side_region(d0, r, D, 0, u0, u1);
            if (u1.x > u0.x && u1.y > u0.y && u1.z > u0.z) {
                const int nb = ((u1.x - u0.x + RC_TX - 1) / RC_TX) * ((u1.y - u0.y + RC_TY - 1) / RC_TY) *
                               ((u1.z - u0.z + RC_TZ - 1) / RC_TZ);
                corr<<<nb, RC_THREADS, smem, st>>>(dt[e.a], dt[e.b], D[0], D[1], D[2], u0, u1,
                                                   make_int3(d0[0], d0[1], d0[2]), r[1], r[2], ds);
                RK(cudaGetLastError());
            }
            int rc = side_sums(st, pf[k], dt[e.a], D, d0, r, 0, ds + S, ds + 2 * (size_t)S);
            if (rc != SEG_OK) return rc;
            rc = side_sums(st, pf[k], dt[e.b], D, d0, r, 1, ds + 3 * (size_t)S, ds + 4 * (size_t)S);
            if (rc != SEG_OK) return rc;
        }
        RK(sc.join());
        RK(cudaMemcpyAsync(hs.data(), dsum, per * (g1 - g0) * sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                           sc.s));
        RK(cudaStreamSynchronize(sc.s));
        for (size_t ei = g0; ei < g1; ++ei) {
            seg_montage_edge &e = E[ei];
            const unsigned long long *h = hs.data() + per * (ei - g0);
            const int d0[3] = {stage[e.b].x - stage[e.a].x, stage[e.b].y - stage[e.a].y,
                               stage[e.b].z - stage[e.a].z};
            // the first best shift in z, y, x order
            for (int si = 0; si < S; ++si) {
                const int s[3] = {si % SX - r[0], (si / SX) % SY - r[1], si / (SX * SY) - r[2]};
                uint64_t cnt = 1;
                for (int k = 0; k < 3; ++k) {
                    const Range q = shared_range(d0[k] + s[k], D[k], 0);
                    cnt *= (uint64_t)(q.hi > q.lo ? q.hi - q.lo : 0);
                }
                if (cnt == 0) continue;
                const unsigned long long sab = h[si], sa = h[S + si], saa = h[2 * (size_t)S + si];
                const unsigned long long sb = h[3 * (size_t)S + si], sbb = h[4 * (size_t)S + si];
                const __int128 N = (__int128)cnt;
                const __int128 num = N * (__int128)sab - (__int128)sa * (__int128)sb;
                const __int128 va = N * (__int128)saa - (__int128)sa * (__int128)sa;
                const __int128 vb = N * (__int128)sbb - (__int128)sb * (__int128)sb;
                if (va == 0 || vb == 0) continue;
                const double rho = (double)num / std::sqrt((double)va * (double)vb);
                if (rho > e.score) {
                    e.score = rho;
                    e.shift.x = s[0];
                    e.shift.y = s[1];
                    e.shift.z = s[2];
                }
            }
        }
    }
    // maximum spanning tree: scores highest first, ties by (a, b)
    std::vector<uint32_t> order(E.size());
    std::iota(order.begin(), order.end(), 0u);
    std::stable_sort(order.begin(), order.end(), [&](uint32_t i, uint32_t j) { return E[i].score > E[j].score; });
    std::vector<uint32_t> par(n_tiles);
    std::iota(par.begin(), par.end(), 0u);
    std::vector<std::vector<uint32_t>> adj(n_tiles);
    for (uint32_t i : order) {
        seg_montage_edge &e = E[i];
        if (e.score < -1.5) continue;  // no defined score
        const uint32_t ra = uf_root(par, e.a), rb = uf_root(par, e.b);
        if (ra == rb) continue;
        par[ra] = rb;
        e.in_tree = 1;
        adj[e.a].push_back(i);
        adj[e.b].push_back(i);
    }
    // corrections from the root along the tree
    for (uint32_t i = 0; i < n_tiles; ++i) delta[i] = seg_offset{0, 0, 0};
    std::vector<uint8_t> seen(n_tiles, 0);
    std::vector<uint32_t> todo{root};
    seen[root] = 1;
    while (!todo.empty()) {
        const uint32_t t = todo.back();
        todo.pop_back();
        for (uint32_t i : adj[t]) {
            const seg_montage_edge &e = E[i];
            const uint32_t o = e.a == t ? e.b : e.a;
            if (seen[o]) continue;
            const int sg = e.a == t ? 1 : -1;  // delta(b) = delta(a) + shift
            delta[o] = seg_offset{delta[t].x + sg * e.shift.x, delta[t].y + sg * e.shift.y,
                                  delta[t].z + sg * e.shift.z};
            seen[o] = 1;
            todo.push_back(o);
        }
    }
    if (!E.empty()) std::memcpy(edges, E.data(), E.size() * sizeof(seg_montage_edge));
    return SEG_OK;
}
