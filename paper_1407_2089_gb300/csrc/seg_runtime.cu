// seg_runtime.cu -- host runtime behind the C ABI in include/seg.h.
//
// A context owns `max_inflight` launch slots (a CUDA stream each, a pinned +
// device batch descriptor, optional captured CUDA graphs, profiling events)
// and one scheduler thread.  Requests are admitted against an HBM budget
// (their own results plus the scratch of the batch that carries them),
// grouped into batches of up to max_batch_volumes volume-channels and
// launched on a free slot; every kernel walks the batch descriptor, so one
// launch sequence segments any mix of volume sizes.  Requests arriving while
// batches run are admitted into the next batch as slots and memory free up
// (continuous batching).  Completion is observed through a host function
// enqueued behind each batch.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <memory>
#include <map>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "seg.h"
#include "seg_internal.h"

namespace seg {
namespace {

using Clock = std::chrono::steady_clock;

constexpr size_t ALIGN = 256;
inline size_t al(size_t b) { return (b + ALIGN - 1) / ALIGN * ALIGN; }
inline uint64_t cdiv(uint64_t a, uint64_t b) { return (a + b - 1) / b; }

struct Batch;

// Geometry and footprint of one channel of a request.
struct VolGeom {
    uint32_t X, Y, Z, W, rows, nrt;
    uint32_t dn_r;   // denoise box radius, 0 = off
    uint32_t cl_r;   // closing ball radius, 0 = off
    uint64_t cl_words;  // words of the extended (padded) mask of the closing
    uint32_t dt_w[3];   // distance-map weights, {0, 0, 0} = off
    uint32_t mrf_max;   // MRF denoise step limit, 0 = off
    uint64_t n, r_cap, k_cap;
    size_t scratch;  // bytes of per-batch scratch for this volume-channel
};

// Distance-map path of a volume: the fused x+y kernel for lines along y of
// at most 512 or 1024 voxels (and X < 65536, so x distances fit 16 bits),
// else the long-line x and y kernels; the shared-memory z kernel for Z <= 256
// with `lt` lines per tile (32 x (lt / 32) rows, lt * Z <= DZ_ELEMS), else the
// long-line z kernel.
struct DtPath {
    int xy;     // DT_XY16, DT_XY32 or DT_X (long-line x and y kernels)
    int z;      // DT_Z or DT_ZL
    uint32_t lt;
    bool long_y() const { return xy == DT_X; }
    bool needs_stack() const { return xy == DT_X || z == DT_ZL; }
};

DtPath dt_path(uint32_t X, uint32_t Y, uint32_t Z) {
    DtPath p;
    p.xy = X >= 65536u ? DT_X : (Y <= 512u ? DT_XY16 : (Y <= 1024u ? DT_XY32 : DT_X));
    p.lt = std::min<uint32_t>(128u, (uint32_t)DZ_ELEMS / Z / 32u * 32u);
    p.z = p.lt >= 32u ? DT_Z : DT_ZL;
    return p;
}

VolGeom geom(seg_dims d, uint32_t min_volume, uint32_t dn_r, uint32_t cl_r, const uint32_t *dt_w,
             uint32_t mrf_max) {
    VolGeom g;
    g.X = d.x; g.Y = d.y; g.Z = d.z;
    g.W = (uint32_t)cdiv(d.x, 32);
    g.rows = d.y * d.z;
    g.nrt = (uint32_t)cdiv(g.rows, ROW_TILE_MIN);  // room for the smallest row tile
    g.n = (uint64_t)d.x * d.y * d.z;
    g.r_cap = (uint64_t)g.rows * cdiv(d.x, 2);
    // 26-separated components: at most one per 2x2x2 block; each surviving
    // cell also holds >= min_volume voxels.
    uint64_t kc = cdiv(d.x, 2) * cdiv(d.y, 2) * cdiv(d.z, 2);
    if (min_volume > 1) kc = std::min<uint64_t>(kc, g.n / min_volume + 1);
    g.k_cap = std::max<uint64_t>(kc, 1);
    g.scratch = al(4ull * HIST_BINS) + al(2ull * g.n) + al(2ull * g.rows * g.W) + al(4ull * g.rows * g.W) +
                al(4ull * (g.rows + 1)) +
                al(4ull * g.rows) + 2 * al(4ull * g.nrt) + 3 * al(4ull * g.r_cap);
    g.dn_r = dn_r;
    if (dn_r) g.scratch += 2 * al(2ull * g.n);  // two box-pass buffers (the denoised image persists)
    g.mrf_max = mrf_max;
    if (mrf_max) g.scratch += al(4ull * 2048);  // levels present in the input
    g.cl_r = cl_r;
    g.cl_words = cl_r ? (uint64_t)(d.y + 2 * cl_r) * (d.z + 2 * cl_r) * (g.W + 2) : 0;
    if (cl_r) g.scratch += al(4ull * g.cl_words);
    for (int a = 0; a < 3; ++a) g.dt_w[a] = dt_w ? dt_w[a] : 0u;
    // distance map: the x+y pass result; the long-line kernels also need the
    // x-pass result and the stack positions
    if (g.dt_w[0]) {
        const DtPath p = dt_path(d.x, d.y, d.z);
        g.scratch += al(4ull * g.n);
        if (p.long_y()) g.scratch += al(4ull * g.n);
        if (p.needs_stack()) g.scratch += al(2ull * g.n);
    }
    return g;
}

struct Request {
    seg_req id = 0;
    seg_dims dims{};
    uint32_t C = 0;
    std::vector<uint32_t> minvol;
    std::vector<VolGeom> g;
    const uint16_t *user_dev = nullptr;  // device input owned by the caller
    std::vector<uint16_t> host_copy;     // host input waiting for admission
    char *block = nullptr;               // labels | feat | stat | [input]
    size_t block_bytes = 0;
    size_t off_labels = 0, off_feat = 0, off_stat = 0, off_input = 0;
    std::vector<size_t> off_dist;         // per channel; SIZE_MAX = no distance map
    std::vector<size_t> off_den;          // per channel; SIZE_MAX = no denoise (front end: 1 image, MRF: 2)
    size_t off_smooth = SIZE_MAX;         // smoothed images of all channels (SEG_KEEP_SMOOTHED)
    std::vector<uint32_t> mrf_steps, mrf_sel;
    size_t per_labels = 0, per_feat = 0;  // bytes per channel
    bool owns_input = false;
    bool admitted = false;
    bool launched = false;
    bool issued = false;  // launch sequence (and done_ev record) enqueued
    int state = SEG_PENDING;
    int err = SEG_OK;
    size_t persist = 0, scratch = 0;
    std::vector<uint32_t> thresh, ncells, errbits;
    cudaEvent_t ready_ev = nullptr;  // order-stream point for device inputs, or the queued host copy
    cudaEvent_t done_ev = nullptr;
    double t_submit = -1, t_admit = -1, t_launch = -1, t_done = -1;

    const uint16_t *input(uint32_t c) const {
        const uint16_t *base = user_dev ? user_dev : reinterpret_cast<const uint16_t *>(block + off_input);
        return base + (size_t)c * g[0].n;
    }
    uint32_t *labels(uint32_t c) const {
        return reinterpret_cast<uint32_t *>(block + off_labels + c * per_labels);
    }
    uint16_t *den(uint32_t c, int k = 0) const {
        return off_den[c] == SIZE_MAX ? nullptr
                                      : reinterpret_cast<uint16_t *>(block + off_den[c]) + (size_t)k * g[c].n;
    }
    uint16_t *smoothed(uint32_t c) const {
        return off_smooth == SIZE_MAX ? nullptr
                                      : reinterpret_cast<uint16_t *>(block + off_smooth) + (size_t)c * g[0].n;
    }
    uint32_t *dist(uint32_t c) const {
        return off_dist[c] == SIZE_MAX ? nullptr : reinterpret_cast<uint32_t *>(block + off_dist[c]);
    }
    seg_cell_features *feat(uint32_t c) const {
        return reinterpret_cast<seg_cell_features *>(block + off_feat + c * per_feat);
    }
    uint32_t *stat(uint32_t c) const {
        return reinterpret_cast<uint32_t *>(block + off_stat) + (size_t)c * ST_WORDS;
    }
};

struct Slot {
    cudaStream_t stream = nullptr;
    BatchHdr *h_hdr = nullptr;  // pinned
    BatchHdr *d_hdr = nullptr;
    uint32_t *h_stat = nullptr;  // pinned
    uint32_t *d_stat = nullptr;
    std::map<uint64_t, cudaGraphExec_t> graph;  // by graph_key of the launch plan
    cudaEvent_t ev[NUM_KERNELS + 1] = {};
    Batch *busy = nullptr;
};

struct Batch {
    Slot *slot = nullptr;
    std::vector<Request *> reqs;
    char *scratch = nullptr;
    size_t scratch_bytes = 0;
    uint32_t nvol = 0;
    uint64_t voxels = 0;
    uint32_t mrf_iters = 0;  // MRF steps launched (the largest limit in the batch)
    std::atomic<bool> done{false};
    int launch_err = SEG_OK;
    struct seg_ctx *ctx = nullptr;
};

}  // namespace
}  // namespace seg

using namespace seg;

struct seg_ctx {
    seg_config cfg{};
    int device = 0;
    int sms = 0;
    LaunchPlan plan{};
    uint32_t tile_z = 64;
    uint64_t budget = 0;
    uint64_t used = 0;
    uint32_t cap_vols = 512;
    bool plain = false, graphs = true, profile = false;
    bool tuned = false;  // tile shape fixed (forced, or tuned on the first batch)
    cudaStream_t copy_stream = nullptr;
    cudaStream_t read_stream = nullptr;
    uint32_t *read_pin = nullptr;  // pinned words for small results of the read calls (one reader at a time)
    std::vector<Slot> slots;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<Request *> pending;
    std::unordered_map<seg_req, std::unique_ptr<Request>> reqs;
    seg_req next_id = 1;
    bool stop = false;
    bool flush = false;
    uint64_t flush_upto = 0;  // requests with a lower id are flushed
    Clock::time_point t0;
    Clock::time_point first_pending;
    std::thread worker;
    // stats
    uint64_t st_batches = 0, st_volumes = 0, st_voxels = 0;
    uint64_t st_launches[NUM_KERNELS] = {};
    double st_ms[NUM_KERNELS] = {};

    double now() const {
        return std::chrono::duration<double, std::milli>(Clock::now() - t0).count();
    }
};

namespace {

int cuda_fail(cudaError_t e, const char *what) {
    if (e == cudaSuccess) return SEG_OK;
    if (std::getenv("SEG_DEBUG")) std::fprintf(stderr, "libseg: %s: %s\n", what, cudaGetErrorString(e));
    return SEG_ECUDA;
}

#define CK(call)                                         \
    do {                                                 \
        cudaError_t e__ = (call);                        \
        if (e__ != cudaSuccess) return cuda_fail(e__, #call); \
    } while (0)

void CUDART_CB on_batch_done(void *p) {
    Batch *b = static_cast<Batch *>(p);
    seg_ctx *ctx = b->ctx;
    {
        std::lock_guard<std::mutex> lk(ctx->mu);
        b->done.store(true);
    }
    ctx->cv.notify_all();
}

// Lays out a request's device block: labels, features, status, [distance
// maps], [denoised images], [smoothed images], [input].
void layout_request(Request &r, bool keep_smoothed) {
    const VolGeom &g = r.g[0];
    r.per_labels = al(4ull * g.n);
    r.per_feat = al(sizeof(seg_cell_features) * g.k_cap);
    for (uint32_t c = 1; c < r.C; ++c) r.per_feat = std::max(r.per_feat, al(sizeof(seg_cell_features) * r.g[c].k_cap));
    size_t off = 0;
    r.off_labels = off;
    off += r.per_labels * r.C;
    r.off_feat = off;
    off += r.per_feat * r.C;
    r.off_stat = off;
    off += al(4ull * ST_WORDS * r.C);
    r.off_dist.assign(r.C, SIZE_MAX);
    for (uint32_t c = 0; c < r.C; ++c)
        if (r.g[c].dt_w[0]) {
            r.off_dist[c] = off;
            off += al(4ull * g.n);
        }
    r.off_den.assign(r.C, SIZE_MAX);
    for (uint32_t c = 0; c < r.C; ++c)
        if (r.g[c].dn_r || r.g[c].mrf_max) {
            r.off_den[c] = off;
            off += al(2ull * g.n * (r.g[c].mrf_max ? 2 : 1));
        }
    r.off_smooth = SIZE_MAX;
    if (keep_smoothed) {
        r.off_smooth = off;
        off += al(2ull * g.n * r.C);
    }
    r.off_input = off;
    if (r.owns_input) off += al(2ull * g.n * r.C);
    r.block_bytes = off;
    r.persist = off;
    r.scratch = 0;
    for (uint32_t c = 0; c < r.C; ++c) r.scratch += r.g[c].scratch;
}

// Builds the batch descriptor on the slot's pinned header.
// z-chunk for a batch: the tuned one, halved (down to 8 planes) while the
// batch would have fewer than two smoothing tiles per multiprocessor, so that
// small batches still spread over the whole GPU.  A forced shape is kept.
// Row-aligned volumes (X % 8 == 0, 16-byte aligned first input of the
// smoothing) take k_smooth_rows; the others k_smooth_hist.
// Volumes for k_smooth_rows: rows of X % 8 == 0 voxels from a 16-byte
// aligned input (16-byte copies), or of an even X >= 10 from a 4-byte aligned
// input (4-byte copies: every row start is then 4-byte aligned).
bool rows_aligned(const VolGeom &g, const void *smooth_in) {
    const uintptr_t a = reinterpret_cast<uintptr_t>(smooth_in);
    if (g.X % 8u == 0u) return (a & 15u) == 0u;
    return g.X % 2u == 0u && g.X >= 10u && (a & 3u) == 0u;
}

const void *smooth_input(const Request *r, uint32_t c) {
    return r->g[c].dn_r ? static_cast<const void *>(r->den(c)) : static_cast<const void *>(r->input(c));
}

uint32_t batch_tile_z(const seg_ctx *ctx, const Batch &b) {
    const uint32_t ty = (uint32_t)ctx->plan.tile_y;
    uint32_t tz = ctx->tile_z;
    if (ctx->cfg.flags & SEG_FORCE_TILE) return tz;
    for (;;) {
        uint64_t tiles = 0;
        for (const Request *r : b.reqs)
            for (uint32_t c = 0; c < r->C; ++c) {
                const VolGeom &g = r->g[c];
                if (rows_aligned(g, smooth_input(r, c))) continue;
                tiles += cdiv(g.X, TILE_X) * cdiv(g.Y, ty) * cdiv(g.Z, tz);
            }
        if (tz <= 8 || tiles >= 2ull * (uint64_t)ctx->sms) return tz;
        tz /= 2;
    }
}

// Planes per k_smooth_rows tile for a batch: as deep as 256 planes, halved
// (down to 1) while the batch has fewer than three tiles per multiprocessor
// (a lone small volume: more tiles, each with its four halo planes).
uint32_t batch_rows_tile_z(const seg_ctx *ctx, const Batch &b) {
    uint32_t tz = 256;
    for (;;) {
        uint64_t tiles = 0;
        for (const Request *r : b.reqs)
            for (uint32_t c = 0; c < r->C; ++c) {
                const VolGeom &g = r->g[c];
                if (!rows_aligned(g, smooth_input(r, c))) continue;
                const uint32_t rt = fs_rows_rt(g.X);
                tiles += cdiv(g.X, 8ull * rt) * cdiv(g.Y, FS_NT / rt) * cdiv(g.Z, tz);
            }
        if (tz <= 1 || tiles >= 3ull * (uint64_t)ctx->sms) return tz;
        tz /= 2;
    }
}

// Rows per row tile for a batch: ROW_TILE, halved while the batch has fewer
// than two row tiles per multiprocessor (a lone small volume), down to
// ROW_TILE_MIN.
uint32_t batch_row_tile(const seg_ctx *ctx, const Batch &b) {
    uint64_t rows = 0;
    for (const Request *r : b.reqs)
        for (uint32_t c = 0; c < r->C; ++c) rows += r->g[c].rows;
    uint32_t rt = ROW_TILE;
    while (rt > (uint32_t)ROW_TILE_MIN && cdiv(rows, rt) < 2ull * (uint64_t)ctx->sms) rt /= 2;
    return rt;
}

void build_header(seg_ctx *ctx, Batch &b) {
    BatchHdr *h = b.slot->h_hdr;
    const uint32_t ty = (uint32_t)ctx->plan.tile_y, tz = batch_tile_z(ctx, b), fz = batch_rows_tile_z(ctx, b);
    const uint32_t rtile = batch_row_tile(ctx, b);
    uint32_t fst = 0;
    uint32_t v = 0, tiles = 0, rts = 0, bks = 0, bts = 0, dn[3] = {0, 0, 0}, dnt = 0, cl = 0;
    uint32_t dtb[DT_NK] = {0, 0, 0, 0, 0, 0};
    uint32_t mrft = 0, mrfc = 0, mrf_iters = 0;
    char *sp = b.scratch;
    for (Request *r : b.reqs) {
        for (uint32_t c = 0; c < r->C; ++c) {
            const VolGeom &g = r->g[c];
            VolDev &V = h->vol[v++];
            V.raw = r->input(c);
            V.labels = r->labels(c);
            V.feat = r->feat(c);
            V.stat = r->stat(c);
            V.dn_r = g.dn_r;
            V.dn_src = V.raw;
            V.dn_a = V.dn_b = V.dn_out = nullptr;
            V.dn_mul = 0;
            V.dn_n[0] = V.dn_n[1] = V.dn_n[2] = 0;
            V.dn_tiles = 0;
            if (g.dn_r) {
                V.dn_a = reinterpret_cast<uint16_t *>(sp); sp += al(2ull * g.n);
                V.dn_b = reinterpret_cast<uint16_t *>(sp); sp += al(2ull * g.n);
                V.dn_out = r->den(c);
                V.raw = V.dn_out;  // the smoothing reads the denoised image
                const uint64_t w = 2ull * g.dn_r + 1;
                V.dn_mul = (uint32_t)(((1ull << 32) + w - 1) / w);
                // tiles of 64 lines x DN_CHUNK positions per axis
                V.dn_n[0] = (uint32_t)(cdiv((uint64_t)g.Y * g.Z, 64) * cdiv(g.X, DN_CHUNK));
                V.dn_n[1] = (uint32_t)(cdiv(g.X, 64) * g.Z * cdiv(g.Y, DN_CHUNK));
                V.dn_n[2] = (uint32_t)(cdiv(g.X, 64) * g.Y * cdiv(g.Z, DN_CHUNK));
                V.dn_tiles = (uint32_t)(cdiv(g.X, MED_TILE_X) * cdiv(g.Y, MED_TILE_Y) * cdiv(g.Z, MED_TILE_Z));
            }
            V.dn_base0 = dn[0];
            V.dn_base1 = dn[1];
            V.dn_base2 = dn[2];
            V.dn_tbase = dnt;
            dn[0] += V.dn_n[0];
            dn[1] += V.dn_n[1];
            dn[2] += V.dn_n[2];
            dnt += V.dn_tiles;
            V.cl_r = g.cl_r;
            V.cl_ext = nullptr;
            V.cl_n = 0;
            V.cl_pad = 0;
            if (g.cl_r) {
                V.cl_ext = reinterpret_cast<uint32_t *>(sp); sp += al(4ull * g.cl_words);
                V.cl_n = (uint32_t)g.cl_words;
            }
            V.cl_base = cl;
            cl += V.cl_n;
            V.mrf_in = V.raw;
            V.mrf_buf[0] = V.mrf_buf[1] = nullptr;
            V.mrf_bits = nullptr;
            V.mrf_max = g.mrf_max;
            V.mrf_tiles = 0;
            V.mrf_vec = (g.X % 8u == 0u && (reinterpret_cast<uintptr_t>(V.mrf_in) & 15u) == 0u) ? 1u : 0u;
            V.mrf_tbase = mrft;
            V.mrf_ctiles = 0;
            V.mrf_cbase = mrfc;
            if (g.mrf_max) {
                V.mrf_buf[0] = r->den(c, 0);
                V.mrf_buf[1] = r->den(c, 1);
                V.mrf_bits = reinterpret_cast<uint32_t *>(sp); sp += al(4ull * 2048);
                V.mrf_tiles = (uint32_t)cdiv((uint64_t)g.rows * cdiv(g.X, 8), MRF_TILE);
                mrft += V.mrf_tiles;
                V.mrf_ctiles = (uint32_t)(cdiv(cdiv(g.X, 8), MRF_TX) * cdiv(g.Y, MRF_TY));
                mrfc += V.mrf_ctiles;
                mrf_iters = std::max(mrf_iters, g.mrf_max);
            }
            V.dt_out = r->dist(c);
            V.dt_g = V.dt_h = nullptr;
            V.dt_sp = nullptr;
            V.dt_zlt = 0;
            V.dt_pad = 0;
            for (int a = 0; a < 3; ++a) V.dt_w[a] = g.dt_w[a];
            for (int k = 0; k < DT_NK; ++k) V.dt_base[k] = dtb[k];
            if (g.dt_w[0]) {
                const DtPath p = dt_path(g.X, g.Y, g.Z);
                V.dt_h = reinterpret_cast<uint32_t *>(sp); sp += al(4ull * g.n);
                if (p.long_y()) {
                    V.dt_g = reinterpret_cast<uint32_t *>(sp); sp += al(4ull * g.n);
                    dtb[DT_X] += g.rows;
                    dtb[DT_Y] += g.X * g.Z;
                } else {
                    dtb[p.xy] += g.W * g.Z;
                }
                if (p.needs_stack()) {
                    V.dt_sp = reinterpret_cast<uint16_t *>(sp); sp += al(2ull * g.n);
                }
                if (p.z == DT_Z) {
                    V.dt_zlt = p.lt;
                    dtb[DT_Z] += g.W * (uint32_t)cdiv(g.Y, p.lt / 32u);
                } else {
                    dtb[DT_ZL] += g.X * g.Y;
                }
            }
            V.hist = reinterpret_cast<uint32_t *>(sp); sp += al(4ull * HIST_BINS);
            V.smooth = reinterpret_cast<uint16_t *>(sp); sp += al(2ull * g.n);
            if (r->smoothed(c)) V.smooth = r->smoothed(c);
            V.wmax = reinterpret_cast<uint16_t *>(sp); sp += al(2ull * g.rows * g.W);
            V.mask = reinterpret_cast<uint32_t *>(sp); sp += al(4ull * g.rows * g.W);
            V.rowoff = reinterpret_cast<uint32_t *>(sp); sp += al(4ull * (g.rows + 1));
            V.rowk = reinterpret_cast<uint32_t *>(sp); sp += al(4ull * g.rows);
            V.tsum = reinterpret_cast<uint32_t *>(sp); sp += al(4ull * g.nrt);
            V.tkeep = reinterpret_cast<uint32_t *>(sp); sp += al(4ull * g.nrt);
            V.run_x = reinterpret_cast<uint32_t *>(sp); sp += al(4ull * g.r_cap);
            V.run_par = reinterpret_cast<uint32_t *>(sp); sp += al(4ull * g.r_cap);
            V.run_aux = reinterpret_cast<uint32_t *>(sp); sp += al(4ull * g.r_cap);
            V.k_cap = g.k_cap;
            V.r_cap = g.r_cap;
            V.X = g.X; V.Y = g.Y; V.Z = g.Z; V.W = g.W;
            V.rows = g.rows;
            V.min_volume = r->minvol[c];
            V.union_limit = (ctx->cfg.flags & SEG_TEST_UNION_FAIL) ? 0u : UNION_LIMIT;
            if (rows_aligned(g, V.raw)) {
                V.ntx = V.nty = V.ntz = 0;
                V.fs_rt = fs_rows_rt(g.X);
                V.fs_ty = (uint32_t)FS_NT / V.fs_rt;
                V.fs_hx = g.X > 8u * FS_RT ? 1u : 0u;
                V.fs_rag = g.X % 8u != 0u ? 1u : 0u;
                V.fs_tz = fz;
                V.fs_ntx = (uint32_t)cdiv(g.X, 8ull * V.fs_rt);
                V.fs_nty = (uint32_t)cdiv(g.Y, V.fs_ty);
                V.fs_ntz = (uint32_t)cdiv(g.Z, fz);
                // word maxima: groups of four octet lanes of one tile row hold
                // one mask word, so the tile's rows span whole groups
                if (V.fs_rt % 4u != 0u) V.wmax = nullptr;
            } else {
                V.wmax = nullptr;
                V.ntx = (uint32_t)cdiv(g.X, TILE_X);
                V.nty = (uint32_t)cdiv(g.Y, ty);
                V.ntz = (uint32_t)cdiv(g.Z, tz);
                V.fs_rt = V.fs_ty = V.fs_hx = V.fs_tz = V.fs_rag = 0;
                V.fs_ntx = V.fs_nty = V.fs_ntz = 0;
            }
            V.fs_base = fst;
            fst += V.fs_ntx * V.fs_nty * V.fs_ntz;
            V.nrt = (uint32_t)cdiv(g.rows, rtile);
            V.tile_base = tiles;
            V.rt_base = rts;
            V.nby = (uint32_t)cdiv(g.Y, BRICK_Y);
            V.nbk = V.nby * (uint32_t)cdiv(g.Z, BRICK_Z);
            V.bk_base = bks;
            {
                // row pairs across brick faces: every pair of a plane z = 8k
                // with the plane below; pairs (y, y-1) with y = 32k in every
                // plane; the two diagonals through y = 32k and y = 32k - 1 in
                // the other planes
                const uint32_t nzb = (g.Z - 1) / BRICK_Z, nyb = (g.Y - 1) / BRICK_Y;
                const uint32_t nzi = g.Z - 1 - nzb;
                V.nbt = nzb * g.Y * 3 + nyb * g.Z + 2 * nyb * nzi;
            }
            V.bt_base = bts;
            tiles += V.ntx * V.nty * V.ntz;
            rts += V.nrt;
            bks += V.nbk;
            bts += V.nbt;
        }
    }
    h->nvol = v;
    h->ntiles = tiles;
    h->fs_tiles = fst;
    h->nrowtiles = rts;
    h->row_tile = rtile;
    h->nbricks = bks;
    h->nbtasks = bts;
    h->dn_items[0] = dn[0];
    h->dn_items[1] = dn[1];
    h->dn_items[2] = dn[2];
    h->dn_tiles = dnt;
    h->cl_items = cl;
    for (int k = 0; k < DT_NK; ++k) h->dt_items[k] = dtb[k];
    h->mrf_tiles = mrft;
    h->mrf_ctiles = mrfc;
    b.mrf_iters = mrf_iters;
    h->tile_z = tz;
    h->tile_y = ty;
    b.nvol = v;
}

// A captured graph fixes which optional kernels launch and how many MRF steps.
uint64_t graph_key(const LaunchPlan &p) {
    return (uint64_t)p.tile_y | (uint64_t)p.rows << 11 | (uint64_t)p.tiles << 12 |
           (uint64_t)p.denoise << 8 | (uint64_t)p.closing << 9 | (uint64_t)p.distance << 10 |
           (uint64_t)p.mrf_iters << 16;
}

// Enqueues descriptor upload, the pipeline and the status read-back.
int enqueue_body(seg_ctx *ctx, Slot &s, uint32_t nvol) {
    const size_t hb = ctx->graphs ? batch_bytes(ctx->cap_vols) : batch_bytes(nvol);
    const size_t sb = 4ull * ST_WORDS * (ctx->graphs ? ctx->cap_vols : nvol);
    CK(cudaMemcpyAsync(s.d_hdr, s.h_hdr, hb, cudaMemcpyHostToDevice, s.stream));
    CK(launch_pipeline(s.d_hdr, ctx->plan, s.stream, ctx->profile ? s.ev : nullptr, s.d_stat));
    CK(cudaMemcpyAsync(s.h_stat, s.d_stat, sb, cudaMemcpyDeviceToHost, s.stream));
    return SEG_OK;
}

// Tile tuning on the first batch: time init + smoothing/histogram for each
// candidate tile shape on the batch's own data and keep the fastest.  The
// pipeline's results do not depend on the tile shape.
int tune_tiles(seg_ctx *ctx, Batch &b) {
    static const int kTy[] = {32, 64};
    static const uint32_t kTz[] = {16, 32, 64};
    Slot &s = *b.slot;
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    float best = 1e30f;
    int best_ty = ctx->plan.tile_y;
    uint32_t best_tz = ctx->tile_z;
    for (int ty : kTy) {
        for (uint32_t tz : kTz) {
            ctx->plan.tile_y = ty;
            ctx->tile_z = tz;
            build_header(ctx, b);
            float ms = 0.f;
            for (int rep = 0; rep < 2; ++rep) {  // first run warms caches and clocks
                CK(cudaMemcpyAsync(s.d_hdr, s.h_hdr, batch_bytes(b.nvol), cudaMemcpyHostToDevice, s.stream));
                CK(cudaEventRecord(e0, s.stream));
                CK(launch_tile_probe(s.d_hdr, ctx->plan, s.stream));
                CK(cudaEventRecord(e1, s.stream));
                CK(cudaEventSynchronize(e1));
                CK(cudaEventElapsedTime(&ms, e0, e1));
            }
            if (ms < best) {
                best = ms;
                best_ty = ty;
                best_tz = tz;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    ctx->plan.tile_y = best_ty;
    ctx->tile_z = best_tz;
    ctx->tuned = true;
    return SEG_OK;
}

int launch_batch(seg_ctx *ctx, Batch &b) {
    Slot &s = *b.slot;
    // Inputs that waited on the host are copied now (pageable source: the
    // call returns once the data is staged).
    for (Request *r : b.reqs) {
        if (!r->block) {
            CK(cudaMallocAsync(reinterpret_cast<void **>(&r->block), r->block_bytes, s.stream));
        }
        if (!r->host_copy.empty()) {
            CK(cudaMemcpyAsync(r->block + r->off_input, r->host_copy.data(), r->host_copy.size() * 2,
                               cudaMemcpyHostToDevice, s.stream));
        }
        if (r->ready_ev) CK(cudaStreamWaitEvent(s.stream, r->ready_ev, 0));
    }
    for (Request *r : b.reqs) std::vector<uint16_t>().swap(r->host_copy);
    CK(cudaMallocAsync(reinterpret_cast<void **>(&b.scratch), b.scratch_bytes, s.stream));
    build_header(ctx, b);
    if (!ctx->tuned && s.h_hdr->ntiles > 0) {
        // the tile shape only concerns k_smooth_hist: tune on the first
        // batch that has volumes for it
        const int rc = tune_tiles(ctx, b);
        if (rc != SEG_OK) return rc;
        build_header(ctx, b);
    }
    ctx->plan.rows = s.h_hdr->fs_tiles > 0;
    ctx->plan.tiles = s.h_hdr->ntiles > 0;
    ctx->plan.denoise = s.h_hdr->dn_tiles > 0;
    ctx->plan.closing = s.h_hdr->cl_items > 0;
    ctx->plan.distance = false;
    for (int k = 0; k < DT_NK; ++k) ctx->plan.distance |= s.h_hdr->dt_items[k] > 0;
    ctx->plan.mrf_iters = b.mrf_iters;
    if (ctx->graphs) {
        const uint64_t key = graph_key(ctx->plan);
        if (s.graph.size() >= 64 && !s.graph.count(key)) {
            // many distinct plans (e.g. varying MRF step limits): start over
            for (auto &g : s.graph)
                if (g.second) cudaGraphExecDestroy(g.second);
            s.graph.clear();
        }
        cudaGraphExec_t &ge = s.graph[key];
        if (!ge) {
            cudaGraph_t g = nullptr;
            CK(cudaStreamBeginCapture(s.stream, cudaStreamCaptureModeThreadLocal));
            int rc = enqueue_body(ctx, s, b.nvol);
            cudaError_t e = cudaStreamEndCapture(s.stream, &g);
            if (rc != SEG_OK) return rc;
            CK(e);
            e = cudaGraphInstantiate(&ge, g, 0);
            cudaGraphDestroy(g);
            CK(e);
        }
        CK(cudaGraphLaunch(ge, s.stream));
    } else {
        int rc = enqueue_body(ctx, s, b.nvol);
        if (rc != SEG_OK) return rc;
    }
    for (Request *r : b.reqs) CK(cudaEventRecord(r->done_ev, s.stream));
    CK(cudaFreeAsync(b.scratch, s.stream));
    b.scratch = nullptr;
    CK(cudaLaunchHostFunc(s.stream, on_batch_done, &b));
    return SEG_OK;
}

// Called with ctx->mu held, after the batch's host function ran.
void finalize_batch(seg_ctx *ctx, Slot &s) {
    Batch *b = s.busy;
    const double t = ctx->now();
    uint32_t v = 0;
    for (Request *r : b->reqs) {
        bool bad = b->launch_err != SEG_OK;
        for (uint32_t c = 0; c < r->C; ++c, ++v) {
            const uint32_t *w = s.h_stat + (size_t)v * ST_WORDS;
            r->thresh[c] = w[ST_THRESH];
            r->ncells[c] = w[ST_CELLS];
            r->errbits[c] = w[ST_ERROR];
            r->mrf_steps[c] = w[ST_MRF_STEPS];
            r->mrf_sel[c] = w[ST_MRF_SEL];
            if (w[ST_ERROR]) bad = true;
        }
        r->state = bad ? SEG_FAILED : SEG_DONE;
        r->err = bad ? (b->launch_err != SEG_OK ? b->launch_err : SEG_EFAILED) : SEG_OK;
        r->t_done = t;
    }
    if (ctx->profile && b->launch_err == SEG_OK) {
        for (int k = 0; k < NUM_KERNELS; ++k) {
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, s.ev[k], s.ev[k + 1]) == cudaSuccess) ctx->st_ms[k] += ms;
        }
    }
    for (int k = 0; k < NUM_KERNELS; ++k) ctx->st_launches[k] += 1;
    ctx->st_batches += 1;
    ctx->st_volumes += b->nvol;
    ctx->st_voxels += b->voxels;
    ctx->used -= b->scratch_bytes;
    s.busy = nullptr;
    delete b;
}

void worker_main(seg_ctx *ctx) {
    cudaSetDevice(ctx->device);
    std::unique_lock<std::mutex> lk(ctx->mu);
    for (;;) {
        bool progressed = false;
        for (Slot &s : ctx->slots) {
            if (s.busy && !s.busy->done.load()) {
                // a device fault leaves the context unusable and the batch's
                // host function never runs: fail the batch instead of waiting
                const cudaError_t e = cudaStreamQuery(s.stream);
                if (e != cudaSuccess && e != cudaErrorNotReady) {
                    s.busy->launch_err = SEG_ECUDA;
                    s.busy->done.store(true);
                }
            }
            if (s.busy && s.busy->done.load()) {
                finalize_batch(ctx, s);
                progressed = true;
            }
        }
        if (progressed) ctx->cv.notify_all();
        bool inflight = false;
        for (Slot &s : ctx->slots) inflight |= (s.busy != nullptr);
        if (ctx->stop && !inflight && ctx->pending.empty()) break;
        Slot *free_slot = nullptr;
        for (Slot &s : ctx->slots)
            if (!s.busy) { free_slot = &s; break; }
        if (free_slot && !ctx->pending.empty()) {
            bool go = ctx->stop || ctx->cfg.batch_window_us == 0;
            if (!go) {
                double waited = std::chrono::duration<double, std::micro>(Clock::now() - ctx->first_pending).count();
                go = waited >= ctx->cfg.batch_window_us;
            }
            // a flush launches what was submitted before it, not requests
            // that arrive while the batch is being formed
            const bool flush_only = !go && ctx->flush;
            go = go || ctx->flush;
            if (go) {
                Batch *b = new Batch();
                b->slot = free_slot;
                b->ctx = ctx;
                uint32_t nv = 0;
                uint64_t dt_lines = 0;
                const uint32_t max_req = ctx->plain ? 1u : 0xFFFFFFFFu;
                // FIFO, except that a request still waiting for memory does not
                // hold back admitted ones queued behind it
                std::deque<Request *> rest;
                while (!ctx->pending.empty() && b->reqs.size() < max_req) {
                    Request *r = ctx->pending.front();
                    ctx->pending.pop_front();
                    if (flush_only && r->id >= ctx->flush_upto) {
                        rest.push_back(r);
                        break;
                    }
                    if (nv + r->C > ctx->cap_vols) {
                        rest.push_back(r);
                        break;
                    }
                    // the distance map's flat line indices stay 32-bit
                    uint64_t rl = 0;
                    for (uint32_t c = 0; c < r->C; ++c)
                        if (r->g[c].dt_w[0]) rl += (uint64_t)r->g[c].X * std::max(r->g[c].Y, r->g[c].Z);
                    if (!b->reqs.empty() && dt_lines + rl > 0xFFFFFFFFull) {
                        rest.push_back(r);
                        break;
                    }
                    // an admitted request already holds its results and its
                    // scratch, so it can always launch
                    if (!r->admitted) {
                        if (ctx->used + r->persist + r->scratch > ctx->budget) {
                            rest.push_back(r);
                            continue;
                        }
                        ctx->used += r->persist + r->scratch;
                        r->admitted = true;
                        r->t_admit = ctx->now();
                    }
                    b->scratch_bytes += r->scratch;
                    r->launched = true;
                    r->t_launch = ctx->now();
                    nv += r->C;
                    dt_lines += rl;
                    b->voxels += r->g[0].n * r->C;
                    b->reqs.push_back(r);
                }
                while (!ctx->pending.empty()) {
                    rest.push_back(ctx->pending.front());
                    ctx->pending.pop_front();
                }
                ctx->pending.swap(rest);
                ctx->flush = !ctx->pending.empty() && ctx->pending.front()->id < ctx->flush_upto;
                if (!ctx->pending.empty()) ctx->first_pending = Clock::now();
                if (b->reqs.empty()) {
                    delete b;  // budget exhausted: wait for completions
                } else {
                    free_slot->busy = b;
                    lk.unlock();
                    int rc = launch_batch(ctx, *b);
                    lk.lock();
                    for (Request *r : b->reqs) r->issued = true;
                    if (rc != SEG_OK) {
                        b->launch_err = rc;
                        // the batch may be partly enqueued: wait for the stream
                        lk.unlock();
                        cudaStreamSynchronize(free_slot->stream);
                        cudaGetLastError();
                        lk.lock();
                        b->done.store(true);
                    }
                    ctx->cv.notify_all();
                    continue;
                }
            }
        }
        if (free_slot && !ctx->pending.empty() && !ctx->flush && ctx->cfg.batch_window_us) {
            ctx->cv.wait_for(lk, std::chrono::microseconds(std::max<uint32_t>(ctx->cfg.batch_window_us / 4, 20)));
        } else {
            ctx->cv.wait_for(lk, std::chrono::milliseconds(50));
        }
    }
}

Request *find_req(seg_ctx *ctx, seg_req id) {
    auto it = ctx->reqs.find(id);
    return it == ctx->reqs.end() ? nullptr : it->second.get();
}

}  // namespace

extern "C" {

const char *seg_strerror(int code) {
    switch (code) {
        case SEG_OK: return "ok";
        case SEG_EINVAL: return "invalid argument";
        case SEG_ETOOBIG: return "volume too large for the limits or the HBM budget";
        case SEG_EAGAIN: return "host queue full, retry later";
        case SEG_ENOTREADY: return "request not finished";
        case SEG_ETIMEOUT: return "timed out";
        case SEG_ECUDA: return "CUDA error";
        case SEG_ESMALL: return "destination too small";
        case SEG_ENOENT: return "unknown request";
        case SEG_EFAILED: return "request failed";
        default: return "unknown error code";
    }
}

int seg_create(const seg_config *cfg, seg_ctx **out) {
    if (!cfg || !out) return SEG_EINVAL;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || cfg->device < 0 || cfg->device >= ndev) {
        cudaGetLastError();
        return SEG_EINVAL;
    }
    if (cfg->flags & SEG_FORCE_TILE) {
        if (cfg->tile_y != 16 && cfg->tile_y != 32 && cfg->tile_y != 64) return SEG_EINVAL;
        if (cfg->tile_z == 0) return SEG_EINVAL;
    }
    std::unique_ptr<seg_ctx> ctx(new seg_ctx());
    ctx->cfg = *cfg;
    ctx->device = cfg->device;
    ctx->t0 = Clock::now();
    CK(cudaSetDevice(cfg->device));
    CK(cudaDeviceGetAttribute(&ctx->sms, cudaDevAttrMultiProcessorCount, cfg->device));

    ctx->plain = (cfg->flags & SEG_PLAIN) != 0;
    // the plain form runs one request per launch sequence, captured like the
    // batched form's (one graph per slot and launch plan)
    ctx->graphs = !(cfg->flags & SEG_NO_GRAPH);
    ctx->profile = (cfg->flags & SEG_PROFILE) != 0;
    ctx->cap_vols = cfg->max_batch_volumes ? cfg->max_batch_volumes : 512;
    const uint32_t nslots = ctx->plain ? 1 : (cfg->max_inflight ? cfg->max_inflight : 2);
    size_t fr = 0, tot = 0;
    CK(cudaMemGetInfo(&fr, &tot));
    ctx->budget = cfg->hbm_budget_bytes ? cfg->hbm_budget_bytes : (uint64_t)(0.8 * (double)fr);
    int ty = 64;
    uint32_t tz = 64;
    if (cfg->flags & SEG_FORCE_TILE) { ty = (int)cfg->tile_y; tz = cfg->tile_z; }
    ctx->tuned = (cfg->flags & SEG_FORCE_TILE) != 0;
    ctx->tile_z = tz;
    ctx->plan.sms = ctx->sms;
    ctx->plan.tile_y = ty;
    ctx->plan.grid_hist = ctx->sms;  // one resident block per SM (176 KiB histogram)
    ctx->plan.grid_vols = ctx->sms;
    ctx->plan.rows = ctx->plan.tiles = true;
    ctx->plan.denoise = false;
    ctx->plan.closing = false;
    ctx->plan.distance = false;
    ctx->plan.mrf_iters = 0;
    CK(configure_kernels(cfg->device, ctx->plan));
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, cfg->device) == cudaSuccess) {
        uint64_t thr = UINT64_MAX;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    cudaGetLastError();
    CK(cudaStreamCreateWithFlags(&ctx->copy_stream, cudaStreamNonBlocking));
    CK(cudaStreamCreateWithFlags(&ctx->read_stream, cudaStreamNonBlocking));
    CK(cudaMallocHost(reinterpret_cast<void **>(&ctx->read_pin), 64));
    ctx->slots.resize(nslots);
    for (Slot &s : ctx->slots) {
        CK(cudaStreamCreateWithFlags(&s.stream, cudaStreamNonBlocking));
        CK(cudaMallocHost(reinterpret_cast<void **>(&s.h_hdr), batch_bytes(ctx->cap_vols)));
        CK(cudaMalloc(reinterpret_cast<void **>(&s.d_hdr), batch_bytes(ctx->cap_vols)));
        CK(cudaMallocHost(reinterpret_cast<void **>(&s.h_stat), 4ull * ST_WORDS * ctx->cap_vols));
        CK(cudaMalloc(reinterpret_cast<void **>(&s.d_stat), 4ull * ST_WORDS * ctx->cap_vols));
        std::memset(s.h_hdr, 0, batch_bytes(ctx->cap_vols));
        for (auto &e : s.ev) CK(cudaEventCreate(&e));
    }
    ctx->worker = std::thread(worker_main, ctx.get());
    *out = ctx.release();
    return SEG_OK;
}

int seg_destroy(seg_ctx *ctx) {
    if (!ctx) return SEG_EINVAL;
    {
        std::lock_guard<std::mutex> lk(ctx->mu);
        ctx->stop = true;
    }
    ctx->cv.notify_all();
    if (ctx->worker.joinable()) ctx->worker.join();
    cudaSetDevice(ctx->device);
    for (auto &kv : ctx->reqs) {
        Request &r = *kv.second;
        if (r.block) cudaFree(r.block);
        if (r.ready_ev) cudaEventDestroy(r.ready_ev);
        if (r.done_ev) cudaEventDestroy(r.done_ev);
    }
    for (Slot &s : ctx->slots) {
        for (auto &g : s.graph)
            if (g.second) cudaGraphExecDestroy(g.second);
        for (auto &e : s.ev)
            if (e) cudaEventDestroy(e);
        if (s.h_hdr) cudaFreeHost(s.h_hdr);
        if (s.d_hdr) cudaFree(s.d_hdr);
        if (s.h_stat) cudaFreeHost(s.h_stat);
        if (s.d_stat) cudaFree(s.d_stat);
        if (s.stream) cudaStreamDestroy(s.stream);
    }
    if (ctx->copy_stream) cudaStreamDestroy(ctx->copy_stream);
    if (ctx->read_stream) cudaStreamDestroy(ctx->read_stream);
    if (ctx->read_pin) cudaFreeHost(ctx->read_pin);
    delete ctx;
    return SEG_OK;
}

int seg_submit_volume(seg_ctx *ctx, const uint16_t *voxels, int on_device, seg_dims dims,
                      uint32_t channels, const seg_channel_params *per_channel, seg_req *out) {
    if (!ctx || !voxels || !out || channels == 0 || dims.x == 0 || dims.y == 0 || dims.z == 0 || on_device < 0 ||
        on_device > 2)
        return SEG_EINVAL;
    // 0: host input copied before the call returns; 1: device input;
    // 2: host input whose copy is queued (the caller keeps it unchanged until
    // the request is done)
    const bool host_in = on_device != 1;
    const uint64_t n = (uint64_t)dims.x * dims.y * dims.z;
    // the kernels index rows and planes with int arithmetic (tile origins
    // plus halos): Y and Z stay below INT_MAX - 64
    if (n >= (1ull << 32) || dims.x > 65536u || dims.y > SEG_MAX_YZ || dims.z > SEG_MAX_YZ) return SEG_ETOOBIG;
    // uint16 voxels: a device input must be 2-byte aligned
    if (!host_in && (reinterpret_cast<uintptr_t>(voxels) & 1u)) return SEG_EINVAL;
    if (channels > ctx->cap_vols) return SEG_ETOOBIG;
    std::unique_ptr<Request> r(new Request());
    r->dims = dims;
    r->C = channels;
    r->minvol.resize(channels);
    for (uint32_t c = 0; c < channels; ++c) {
        uint32_t m = per_channel ? per_channel[c].min_volume_voxels : 30u;
        const uint32_t dr = per_channel ? per_channel[c].denoise_radius : 0u;
        const uint32_t cr = per_channel ? per_channel[c].closing_radius : 0u;
        if (dr > (uint32_t)DN_MAX_R || cr > (uint32_t)CL_MAX_R) return SEG_EINVAL;
        const uint32_t *dw = per_channel ? per_channel[c].distance_weights : nullptr;
        if (dw && (dw[0] | dw[1] | dw[2])) {
            // every weight >= 1 and the largest distance below the 0xFFFFFFFF marker
            if (!dw[0] || !dw[1] || !dw[2]) return SEG_EINVAL;
            const unsigned __int128 dmax =
                (unsigned __int128)dw[0] * (dims.x - 1ull) * (dims.x - 1ull) +
                (unsigned __int128)dw[1] * (dims.y - 1ull) * (dims.y - 1ull) +
                (unsigned __int128)dw[2] * (dims.z - 1ull) * (dims.z - 1ull);
            if (dmax >= 0xFFFFFFFFull) return SEG_EINVAL;
        } else {
            dw = nullptr;
        }
        const uint32_t mi = per_channel ? per_channel[c].mrf_iterations : 0u;
        if (mi > MRF_MAX_ITER || (mi && dr)) return SEG_EINVAL;
        r->minvol[c] = m ? m : 1u;  // a cell has at least one voxel
        r->g.push_back(geom(dims, r->minvol[c], dr, cr, dw, mi));
    }
    {
        uint64_t rl = 0;
        for (uint32_t c = 0; c < channels; ++c)
            if (r->g[c].dt_w[0]) rl += (uint64_t)dims.x * std::max(dims.y, dims.z);
        if (rl > 0xFFFFFFFFull) return SEG_ETOOBIG;  // distance-map lines of one launch
    }
    r->thresh.assign(channels, 0);
    r->ncells.assign(channels, 0);
    r->mrf_steps.assign(channels, 0);
    r->mrf_sel.assign(channels, 0);
    r->errbits.assign(channels, 0);
    r->owns_input = host_in;
    if (!host_in) r->user_dev = voxels;
    layout_request(*r, (ctx->cfg.flags & SEG_KEEP_SMOOTHED) != 0);
    if (r->persist + r->scratch > ctx->budget) return SEG_ETOOBIG;
    cudaSetDevice(ctx->device);
    if (cudaEventCreateWithFlags(&r->done_ev, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        return SEG_ECUDA;
    }
    if (!host_in && ctx->cfg.order_stream) {
        if (cudaEventCreateWithFlags(&r->ready_ev, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventRecord(r->ready_ev, static_cast<cudaStream_t>(ctx->cfg.order_stream)) != cudaSuccess) {
            cudaGetLastError();
            cudaEventDestroy(r->done_ev);
            return SEG_ECUDA;
        }
    }
    bool copy_now = false;
    {
        std::lock_guard<std::mutex> lk(ctx->mu);
        r->t_submit = ctx->now();
        uint32_t hq = ctx->cfg.host_queue ? ctx->cfg.host_queue : 4096u;
        if (ctx->pending.size() >= hq) {
            cudaEventDestroy(r->done_ev);
            if (r->ready_ev) cudaEventDestroy(r->ready_ev);
            return SEG_EAGAIN;
        }
        if (host_in && ctx->used + r->persist + r->scratch <= ctx->budget) {
            // admit now (its results and its batch scratch reserved) and copy
            // straight from the caller's buffer
            ctx->used += r->persist + r->scratch;
            r->admitted = true;
            r->t_admit = ctx->now();
            copy_now = true;
        }
    }
    if (host_in) {
        const size_t bytes = 2ull * n * channels;
        int rc = SEG_OK;
        if (copy_now) {
            cudaError_t e = cudaMallocAsync(reinterpret_cast<void **>(&r->block), r->block_bytes, ctx->copy_stream);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(r->block + r->off_input, voxels, bytes, cudaMemcpyHostToDevice, ctx->copy_stream);
            if (on_device == 2) {
                // the batch waits for the copy on the device
                if (e == cudaSuccess) e = cudaEventCreateWithFlags(&r->ready_ev, cudaEventDisableTiming);
                if (e == cudaSuccess) e = cudaEventRecord(r->ready_ev, ctx->copy_stream);
            } else if (e == cudaSuccess) {
                e = cudaStreamSynchronize(ctx->copy_stream);
            }
            if (e != cudaSuccess) rc = cuda_fail(e, "submit copy");
        } else {
            r->host_copy.assign(voxels, voxels + n * channels);
        }
        if (rc != SEG_OK) {
            std::lock_guard<std::mutex> lk(ctx->mu);
            if (r->admitted) ctx->used -= r->persist + r->scratch;
            if (r->block) cudaFreeAsync(r->block, ctx->copy_stream);
            cudaEventDestroy(r->done_ev);
            if (r->ready_ev) cudaEventDestroy(r->ready_ev);
            return rc;
        }
    }
    {
        std::lock_guard<std::mutex> lk(ctx->mu);
        r->id = ctx->next_id++;
        *out = r->id;
        if (ctx->pending.empty()) ctx->first_pending = Clock::now();
        ctx->pending.push_back(r.get());
        ctx->reqs.emplace(r->id, std::move(r));
    }
    ctx->cv.notify_all();
    return SEG_OK;
}

int seg_flush(seg_ctx *ctx) {
    if (!ctx) return SEG_EINVAL;
    {
        std::lock_guard<std::mutex> lk(ctx->mu);
        if (!ctx->pending.empty()) {
            ctx->flush = true;
            ctx->flush_upto = ctx->next_id;
        }
    }
    ctx->cv.notify_all();
    return SEG_OK;
}

int seg_poll(seg_ctx *ctx, seg_req req, uint32_t timeout_ms, int *state) {
    if (!ctx || !state) return SEG_EINVAL;
    std::unique_lock<std::mutex> lk(ctx->mu);
    Request *r = find_req(ctx, req);
    if (!r) return SEG_ENOENT;
    if (r->state == SEG_PENDING && timeout_ms) {
        ctx->cv.wait_for(lk, std::chrono::milliseconds(timeout_ms), [&] { return r->state != SEG_PENDING; });
    }
    *state = r->state;
    return r->state == SEG_PENDING ? SEG_ETIMEOUT : SEG_OK;
}

int seg_enqueue_wait(seg_ctx *ctx, seg_req req, void *stream) {
    if (!ctx) return SEG_EINVAL;
    std::unique_lock<std::mutex> lk(ctx->mu);
    Request *r = find_req(ctx, req);
    if (!r) return SEG_ENOENT;
    if (!r->issued && r->state == SEG_PENDING) {
        ctx->flush = true;
        ctx->flush_upto = std::max<uint64_t>(ctx->flush_upto, r->id + 1);
        ctx->cv.notify_all();
        ctx->cv.wait(lk, [&] { return r->issued || r->state != SEG_PENDING; });
    }
    cudaEvent_t ev = r->done_ev;
    lk.unlock();
    cudaSetDevice(ctx->device);
    cudaError_t e = cudaStreamWaitEvent(static_cast<cudaStream_t>(stream), ev, 0);
    return cuda_fail(e, "seg_enqueue_wait");
}

int seg_read_labels(seg_ctx *ctx, seg_req req, uint32_t channel, uint32_t *dst, uint64_t dst_elems,
                    int dst_on_device) {
    if (!ctx || !dst) return SEG_EINVAL;
    Request *r;
    {
        std::lock_guard<std::mutex> lk(ctx->mu);
        r = find_req(ctx, req);
        if (!r) return SEG_ENOENT;
        if (r->state == SEG_PENDING) return SEG_ENOTREADY;
        if (r->state == SEG_FAILED) return SEG_EFAILED;
    }
    if (channel >= r->C) return SEG_EINVAL;
    const uint64_t n = r->g[channel].n;
    if (dst_elems < n) return SEG_ESMALL;
    cudaSetDevice(ctx->device);
    cudaError_t e = cudaMemcpyAsync(dst, r->labels(channel), 4ull * n,
                                    dst_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                                    ctx->read_stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->read_stream);
    return cuda_fail(e, "seg_read_labels");
}

int seg_read_denoised(seg_ctx *ctx, seg_req req, uint32_t channel, uint16_t *dst, uint64_t dst_elems,
                      int dst_on_device, uint32_t *mrf_steps) {
    if (!ctx || !dst) return SEG_EINVAL;
    Request *r;
    {
        std::lock_guard<std::mutex> lk(ctx->mu);
        r = find_req(ctx, req);
        if (!r) return SEG_ENOENT;
        if (r->state == SEG_PENDING) return SEG_ENOTREADY;
        if (r->state == SEG_FAILED) return SEG_EFAILED;
    }
    if (channel >= r->C || !r->den(channel)) return SEG_EINVAL;
    const uint64_t n = r->g[channel].n;
    if (dst_elems < n) return SEG_ESMALL;
    // the front end's image, or the MRF image that was kept
    const uint16_t *src = r->den(channel);
    if (r->g[channel].mrf_max) {
        const uint32_t sel = r->mrf_sel[channel];
        src = sel == 0 ? r->input(channel) : r->den(channel, (int)sel - 1);
    }
    if (mrf_steps) *mrf_steps = r->mrf_steps[channel];
    cudaSetDevice(ctx->device);
    cudaError_t e = cudaMemcpyAsync(dst, src, 2ull * n,
                                    dst_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                                    ctx->read_stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->read_stream);
    return cuda_fail(e, "seg_read_denoised");
}

int seg_read_smoothed(seg_ctx *ctx, seg_req req, uint32_t channel, uint16_t *dst, uint64_t dst_elems,
                      int dst_on_device) {
    if (!ctx || !dst) return SEG_EINVAL;
    Request *r;
    {
        std::lock_guard<std::mutex> lk(ctx->mu);
        r = find_req(ctx, req);
        if (!r) return SEG_ENOENT;
        if (r->state == SEG_PENDING) return SEG_ENOTREADY;
        if (r->state == SEG_FAILED) return SEG_EFAILED;
    }
    if (channel >= r->C || !r->smoothed(channel)) return SEG_EINVAL;
    const uint64_t n = r->g[channel].n;
    if (dst_elems < n) return SEG_ESMALL;
    cudaSetDevice(ctx->device);
    cudaError_t e = cudaMemcpyAsync(dst, r->smoothed(channel), 2ull * n,
                                    dst_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                                    ctx->read_stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->read_stream);
    return cuda_fail(e, "seg_read_smoothed");
}

int seg_read_cell_distance(seg_ctx *ctx, seg_req req, uint32_t cells_channel, uint32_t map_channel, uint32_t *dst,
                           uint64_t cap, uint64_t *n_cells) {
    if (!ctx) return SEG_EINVAL;
    Request *r;
    {
        std::lock_guard<std::mutex> lk(ctx->mu);
        r = find_req(ctx, req);
        if (!r) return SEG_ENOENT;
        if (r->state == SEG_PENDING) return SEG_ENOTREADY;
        if (r->state == SEG_FAILED) return SEG_EFAILED;
    }
    if (cells_channel >= r->C || map_channel >= r->C || !r->dist(map_channel)) return SEG_EINVAL;
    const uint64_t k = r->ncells[cells_channel];
    if (n_cells) *n_cells = k;
    if (!dst) return cap == 0 ? SEG_OK : SEG_EINVAL;
    if (cap < k) return SEG_ESMALL;
    if (k == 0) return SEG_OK;
    cudaSetDevice(ctx->device);
    uint32_t *d = nullptr;
    cudaError_t e = cudaMallocAsync(reinterpret_cast<void **>(&d), 4 * k, ctx->read_stream);
    if (e == cudaSuccess)
        e = launch_cell_distance(r->labels(cells_channel), r->dist(map_channel), r->g[cells_channel].n, d, k,
                                 ctx->sms, ctx->read_stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dst, d, 4 * k, cudaMemcpyDeviceToHost, ctx->read_stream);
    if (d) cudaFreeAsync(d, ctx->read_stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->read_stream);
    return cuda_fail(e, "seg_read_cell_distance");
}

int seg_read_label_runs(seg_ctx *ctx, seg_req req, uint32_t channel, seg_label_run *dst, uint64_t cap,
                        uint64_t *n_runs, int dst_on_device) {
    if (!ctx) return SEG_EINVAL;
    Request *r;
    {
        std::lock_guard<std::mutex> lk(ctx->mu);
        r = find_req(ctx, req);
        if (!r) return SEG_ENOENT;
        if (r->state == SEG_PENDING) return SEG_ENOTREADY;
        if (r->state == SEG_FAILED) return SEG_EFAILED;
    }
    if (channel >= r->C || (!dst && cap)) return SEG_EINVAL;
    const VolGeom &g = r->g[channel];
    if (g.rows > 0xFFFFFFFFu - 64u) return SEG_ETOOBIG;  // row indices of the blocks stay in 32 bits
    const uint32_t nt = label_runs_tiles(g.rows);
    const size_t a_rows = al(4ull * g.rows), a_tiles = al(4ull * nt);
    const uint64_t most = (uint64_t)g.rows * ((g.X + 1) / 2);  // runs a label image can hold
    cudaSetDevice(ctx->device);
    cudaStream_t s = ctx->read_stream;
    // A destination the device reaches (device memory, or pinned host
    // memory through its mapping) takes the records in the same pass of
    // launches as the count, with one synchronisation; pageable memory is
    // filled by a copy once the count is known.
    seg_label_run *mapped = nullptr;
    if (dst && cap && !dst_on_device) {
        cudaPointerAttributes pa;
        if (cudaPointerGetAttributes(&pa, dst) == cudaSuccess && pa.type == cudaMemoryTypeHost && pa.devicePointer)
            mapped = static_cast<seg_label_run *>(pa.devicePointer);
        cudaGetLastError();
    }
    const bool one_pass = dst && cap && (dst_on_device || mapped);
    const uint64_t stage = mapped ? std::min<uint64_t>(cap, most) : 0;
    char *tmp = nullptr;
    seg_label_run *dev_out = nullptr;
    uint32_t total = 0;
    cudaError_t e = cudaMallocAsync(reinterpret_cast<void **>(&tmp), a_rows + a_tiles + 256, s);
    uint32_t *rowcnt = reinterpret_cast<uint32_t *>(tmp);
    uint32_t *tiles = reinterpret_cast<uint32_t *>(tmp + a_rows);
    uint32_t *d_total = reinterpret_cast<uint32_t *>(tmp + a_rows + a_tiles);
    if (e == cudaSuccess) e = launch_label_runs_count(r->labels(channel), g.X, g.rows, rowcnt, tiles, d_total,
                                                      ctx->sms, s);
    if (one_pass) {
        dev_out = dst_on_device ? dst : nullptr;
        if (e == cudaSuccess && mapped && stage)
            e = cudaMallocAsync(reinterpret_cast<void **>(&dev_out), sizeof(seg_label_run) * stage, s);
        if (e == cudaSuccess && dev_out)
            e = launch_label_runs_write(r->labels(channel), g.X, g.rows, rowcnt, tiles, d_total,
                                        mapped ? stage : cap, dev_out, mapped, ctx->sms, s);
        if (mapped && dev_out) cudaFreeAsync(dev_out, s);
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(ctx->read_pin, d_total, 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    int rc = SEG_OK;
    if (e == cudaSuccess) {
        total = ctx->read_pin[0];
        if (n_runs) *n_runs = total;
        if (cap < total) {
            rc = dst ? SEG_ESMALL : SEG_OK;
        } else if (total && !one_pass) {
            e = cudaMallocAsync(reinterpret_cast<void **>(&dev_out), sizeof(seg_label_run) * total, s);
            if (e == cudaSuccess)
                e = launch_label_runs_write(r->labels(channel), g.X, g.rows, rowcnt, tiles, d_total, total, dev_out,
                                            nullptr, ctx->sms, s);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(dst, dev_out, sizeof(seg_label_run) * total, cudaMemcpyDeviceToHost, s);
            if (dev_out) cudaFreeAsync(dev_out, s);
        }
    }
    if (tmp) cudaFreeAsync(tmp, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "seg_read_label_runs");
    return rc;
}

int seg_read_distance(seg_ctx *ctx, seg_req req, uint32_t channel, uint32_t *dst, uint64_t dst_elems,
                      int dst_on_device) {
    if (!ctx || !dst) return SEG_EINVAL;
    Request *r;
    {
        std::lock_guard<std::mutex> lk(ctx->mu);
        r = find_req(ctx, req);
        if (!r) return SEG_ENOENT;
        if (r->state == SEG_PENDING) return SEG_ENOTREADY;
        if (r->state == SEG_FAILED) return SEG_EFAILED;
    }
    if (channel >= r->C || !r->dist(channel)) return SEG_EINVAL;
    const uint64_t n = r->g[channel].n;
    if (dst_elems < n) return SEG_ESMALL;
    cudaSetDevice(ctx->device);
    cudaError_t e = cudaMemcpyAsync(dst, r->dist(channel), 4ull * n,
                                    dst_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                                    ctx->read_stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->read_stream);
    return cuda_fail(e, "seg_read_distance");
}

int seg_read_features(seg_ctx *ctx, seg_req req, uint32_t channel, seg_cell_features *dst, uint64_t cap,
                      uint64_t *n_cells, uint16_t *otsu_threshold) {
    if (!ctx) return SEG_EINVAL;
    Request *r;
    {
        std::lock_guard<std::mutex> lk(ctx->mu);
        r = find_req(ctx, req);
        if (!r) return SEG_ENOENT;
        if (r->state == SEG_PENDING) return SEG_ENOTREADY;
        if (r->state == SEG_FAILED) return SEG_EFAILED;
    }
    if (channel >= r->C) return SEG_EINVAL;
    const uint64_t k = r->ncells[channel];
    if (n_cells) *n_cells = k;
    if (otsu_threshold) *otsu_threshold = (uint16_t)r->thresh[channel];
    if (!dst) return cap == 0 ? SEG_OK : SEG_EINVAL;
    const uint64_t m = std::min<uint64_t>(k, cap);
    if (m) {
        cudaSetDevice(ctx->device);
        cudaError_t e = cudaMemcpyAsync(dst, r->feat(channel), m * sizeof(seg_cell_features),
                                        cudaMemcpyDeviceToHost, ctx->read_stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->read_stream);
        if (e != cudaSuccess) return cuda_fail(e, "seg_read_features");
    }
    return cap < k ? SEG_ESMALL : SEG_OK;
}

int seg_release(seg_ctx *ctx, seg_req req) {
    if (!ctx) return SEG_EINVAL;
    std::unique_ptr<Request> owned;
    {
        std::unique_lock<std::mutex> lk(ctx->mu);
        Request *r = find_req(ctx, req);
        if (!r) return SEG_ENOENT;
        if (!r->launched) {
            auto it = std::find(ctx->pending.begin(), ctx->pending.end(), r);
            if (it != ctx->pending.end()) ctx->pending.erase(it);
        } else {
            ctx->cv.wait(lk, [&] { return r->state != SEG_PENDING; });
        }
        if (r->admitted) ctx->used -= r->launched ? r->persist : r->persist + r->scratch;
        auto it = ctx->reqs.find(req);
        owned = std::move(it->second);
        ctx->reqs.erase(it);
    }
    cudaSetDevice(ctx->device);
    if (owned->block) cudaFreeAsync(owned->block, ctx->copy_stream);
    if (owned->ready_ev) cudaEventDestroy(owned->ready_ev);
    if (owned->done_ev) cudaEventDestroy(owned->done_ev);
    cudaGetLastError();
    ctx->cv.notify_all();
    return SEG_OK;
}

int seg_request_times(seg_ctx *ctx, seg_req req, double *submit_ms, double *admit_ms, double *launch_ms,
                      double *done_ms) {
    if (!ctx) return SEG_EINVAL;
    std::lock_guard<std::mutex> lk(ctx->mu);
    Request *r = find_req(ctx, req);
    if (!r) return SEG_ENOENT;
    if (submit_ms) *submit_ms = r->t_submit;
    if (admit_ms) *admit_ms = r->t_admit;
    if (launch_ms) *launch_ms = r->t_launch;
    if (done_ms) *done_ms = r->t_done;
    return SEG_OK;
}

int seg_get_stats(seg_ctx *ctx, seg_stats *out) {
    if (!ctx || !out) return SEG_EINVAL;
    std::lock_guard<std::mutex> lk(ctx->mu);
    std::memset(out, 0, sizeof(*out));
    out->batches = ctx->st_batches;
    out->volumes = ctx->st_volumes;
    out->voxels = ctx->st_voxels;
    out->tile_y = (uint32_t)ctx->plan.tile_y;
    out->tile_z = ctx->tile_z;
    static_assert(NUM_KERNELS <= SEG_MAX_KERNELS, "seg_stats holds SEG_MAX_KERNELS kernels");
    out->n_kernels = NUM_KERNELS;
    for (int k = 0; k < NUM_KERNELS; ++k) {
        std::snprintf(out->names[k], sizeof(out->names[k]), "%s", kKernelNames[k]);
        out->launches[k] = ctx->st_launches[k];
        out->total_ms[k] = ctx->st_ms[k];
    }
    out->bytes_in_use = ctx->used;
    out->budget_bytes = ctx->budget;
    return SEG_OK;
}

int seg_reset_stats(seg_ctx *ctx) {
    if (!ctx) return SEG_EINVAL;
    std::lock_guard<std::mutex> lk(ctx->mu);
    ctx->st_batches = ctx->st_volumes = ctx->st_voxels = 0;
    for (int k = 0; k < NUM_KERNELS; ++k) { ctx->st_launches[k] = 0; ctx->st_ms[k] = 0; }
    return SEG_OK;
}

}  // extern "C"
