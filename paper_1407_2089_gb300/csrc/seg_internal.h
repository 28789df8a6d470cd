// seg_internal.h -- device-side batch descriptors shared by the runtime and
// the kernels of libseg (not part of the public ABI).
#pragma once

#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>

#include "seg.h"

namespace seg {

// Per-volume status words (VolDev::stat).
enum StatWord : uint32_t {
    ST_THRESH = 0,     // Otsu level t* (foreground = s > t*)
    ST_RUNS = 1,       // number of foreground runs R
    ST_CELLS = 2,      // number of surviving cells K
    // word 3 unused
    ST_ERROR = 4,      // error bits (ERR_*)
    ST_MRF_STEPS = 5,  // MRF denoise: steps kept
    ST_MRF_SEL = 6,    // MRF denoise: result buffer (0 input, 1 mrf_buf[0], 2 mrf_buf[1])
    ST_MRF_DONE = 7,   // MRF denoise: stopped
    ST_MRF_DELTA = 8,  // MRF denoise: step size (0: fewer than two levels)
    ST_MRF_CNT = 9,    // MRF denoise: tiles done in the current launch
    ST_MRF_CHG = 10,   // MRF denoise: some voxel changed in the current step
    ST_MRF_E = 12,     // MRF denoise: uint64 at words 12-13, Laplacian sum S, then sum d^2
    ST_MRF_LIMIT = 14, // MRF denoise: binary64 bound N sigma^2 at words 14-15
    ST_WORDS = 16,
};

enum ErrBits : uint32_t {
    ERR_UNION = 1u << 0,   // union retry limit reached
    ERR_KCAP = 1u << 1,    // more cells than the feature buffer holds
    ERR_RCAP = 1u << 2,    // more runs than the run buffer holds
    ERR_OTSU = 1u << 3,    // histogram total differs from the voxel count
    ERR_TIMEOUT = 1u << 4, // a bounded wait on an asynchronous copy gave up
};

constexpr int TILE_X = 64;        // smoothing tile width (outputs along x)
constexpr uint32_t UNION_LIMIT = 1u << 24;  // union-find retries before ERR_UNION
constexpr int ROW_TILE = 256;     // rows per row tile (run kernels; their block size)
constexpr int ROW_TILE_MIN = 32;  // smallest row tile (batches with few rows)
constexpr int HIST_BINS = 65536;
// Union-find bricks: BRICK_Y x BRICK_Z rows (one thread each) whose runs are
// united in shared memory when there are at most BRICK_CAP of them.
constexpr int BRICK_Y = 32;
constexpr int BRICK_Z = 8;
constexpr int BRICK_CAP = 2048;

// One volume-channel inside a batch.  All pointers are device addresses.
struct VolDev {
    const uint16_t *raw;      // [Z][Y][X]
    uint32_t *labels;         // [Z][Y][X] output
    seg_cell_features *feat;  // k_cap cells output
    uint32_t *stat;           // ST_WORDS words
    uint32_t *hist;           // 65536 uint32 bins
    uint16_t *smooth;         // [Z][Y][X] smoothed voxels (pass 1 -> threshold pass)
    uint16_t *wmax;           // rows x W: largest smoothed value of each mask word (k_smooth_rows
                              // volumes with X % 32 == 0 or X > 512; else null)
    uint32_t *mask;           // rows x W words, bit b of word w is x = 32w + b
    uint32_t *rowoff;         // rows + 1: run count per row, then run offsets
    uint32_t *rowk;           // rows: kept-root count per row, then label base
    uint32_t *tsum;           // row tiles: run totals, then offsets
    uint32_t *tkeep;          // row tiles: kept-root totals, then offsets
    uint32_t *run_x;          // r_cap: x0 | x1 << 16 (inclusive run ends)
    uint32_t *run_par;        // r_cap: union-find parent (run index)
    uint32_t *run_aux;        // r_cap: voxel count at roots, then label
    uint64_t k_cap;
    uint64_t r_cap;
    uint32_t X, Y, Z, W;      // W = words per mask row
    uint32_t rows;            // Y * Z
    uint32_t min_volume;
    uint32_t union_limit;     // retries before a union gives up (ERR_UNION)
    uint32_t ntx, nty, ntz;   // smoothing tiles per axis (k_smooth_hist; 0 for row-aligned volumes)
    uint32_t nrt;             // row tiles (of BatchHdr::row_tile rows)
    uint32_t tile_base;       // first flat smoothing-tile index
    // k_smooth_rows (X % 8 == 0 with a 16-byte aligned input, or X even and
    // at least 10 with a 4-byte aligned input); fs_ntx = 0 for the other volumes
    uint32_t fs_rt;           // octets per tile row (min(ceil(X / 8), 64))
    uint32_t fs_ty;           // rows per tile (FS_NT / fs_rt)
    uint32_t fs_hx;           // 1: x-tiled (X > 512), staged rows carry a halo chunk on each side
    uint32_t fs_rag;          // 1: X % 8 != 0 (X even): 4-byte copies and stores, a partial last octet
    uint32_t fs_tz;           // planes per tile
    uint32_t fs_ntx, fs_nty, fs_ntz;  // tiles per axis
    uint32_t fs_base;         // first flat k_smooth_rows tile index
    uint32_t rt_base;         // first flat row-tile index
    uint32_t nby;             // union-find bricks along y
    uint32_t nbk;             // union-find bricks
    uint32_t bk_base;         // first flat brick index
    uint32_t nbt;             // row pairs that cross a brick face (k_union tasks)
    uint32_t bt_base;         // first flat k_union task index
    // denoise front end (dn_r > 0); raw then points at dn_out
    const uint16_t *dn_src;   // observed image [Z][Y][X]
    uint16_t *dn_a, *dn_b;    // box-pass ping-pong buffers (the background ends in dn_a)
    uint16_t *dn_out;         // denoised image (the smoothing's input)
    uint32_t dn_r;            // box radius, 0 = no denoise
    uint32_t dn_mul;          // ceil(2^32 / (2 dn_r + 1)): division by the box width
    uint32_t dn_n[3];         // box-pass items per axis (lines x chunks)
    uint32_t dn_base0, dn_base1, dn_base2;  // first flat box item per axis
    uint32_t dn_tiles;        // median tiles
    uint32_t dn_tbase;        // first flat median tile
    // closing of the foreground (cl_r > 0)
    uint32_t *cl_ext;         // dilated mask on rows y in [-r, Y+r), z in [-r, Z+r), W + 2 words each
    uint32_t cl_r;            // ball radius, 0 = no closing
    uint32_t cl_n;            // dilation items (words of the extended mask)
    uint32_t cl_base;         // first flat dilation item
    uint32_t cl_pad;
    // distance map of the final foreground (dt_w[0] > 0)
    uint32_t *dt_out;         // [Z][Y][X] weighted squared distances (output)
    uint32_t *dt_h;           // [Z][Y][X] distances of the x and y passes
    uint32_t *dt_g;           // [Z][Y][X] x-pass distances (long-line path only)
    uint16_t *dt_sp;          // [Z][Y][X] stack positions (long-line path only)
    uint32_t dt_w[3];         // weights of dx^2, dy^2, dz^2; 0 = no distance map
    uint32_t dt_base[6];      // first flat item of this volume in each DtKernel
    uint32_t dt_zlt;          // lines of a k_dist_z tile (32, 64, 96 or 128)
    uint32_t dt_pad;
    // MRF vessel denoise (mrf_max > 0); raw is rewritten on the device to the
    // kept image before the smoothing reads it
    const uint16_t *mrf_in;   // the input I^0 [Z][Y][X]
    uint16_t *mrf_buf[2];     // steps: it 0 reads mrf_in, it > 0 mrf_buf[it & 1]; writes mrf_buf[(it + 1) & 1]
    uint32_t *mrf_bits;       // 2048 words: levels present in the input
    uint32_t mrf_max;         // step limit, 0 = off
    uint32_t mrf_tiles;       // k_mrf_stats tiles of MRF_TILE octets (8 x-consecutive voxels)
    uint32_t mrf_tbase;       // first flat k_mrf_stats tile
    uint32_t mrf_ctiles;      // k_mrf_step tiles: MRF_TX octets x MRF_TY rows, all of z
    uint32_t mrf_cbase;       // first flat k_mrf_step tile
    uint32_t mrf_vec;         // 1: X % 8 == 0 and the input 16-byte aligned (octets load as uint4)
};

// The distance-map kernels and their work items.  A volume takes the fused
// x+y kernel when its lines along y fit one block (Y <= 1024, X < 65536), the
// shared-memory z kernel when its lines along z do (Z <= 256); otherwise the
// long-line kernels, which keep their stacks in global memory.
enum DtKernel : int {
    DT_XY16 = 0,  // k_dist_xy<16>: (mask word, z) tiles, Y <= 512
    DT_XY32 = 1,  // k_dist_xy<32>: (mask word, z) tiles, 512 < Y <= 1024
    DT_X = 2,     // k_dist_x: mask rows (long y lines)
    DT_Y = 3,     // k_dist_line<1>: y lines (long y lines)
    DT_Z = 4,     // k_dist_z: (mask word, y group) tiles, Z <= 256
    DT_ZL = 5,    // k_dist_line<2>: z lines (Z > 256)
    DT_NK = 6,
};
constexpr int DZ_ELEMS = 8192;   // k_dist_z shared stack entries per block
constexpr int MRF_TILE = 256;    // octets per k_mrf_stats tile (one per thread)
constexpr int MRF_TX = 32;       // k_mrf_step tile: octets along x (one warp) ...
constexpr int MRF_TY = 8;        // ... times rows, walked down z
constexpr uint32_t MRF_MAX_ITER = 1000;

// Batch header, followed in memory by VolDev[nvol].
struct BatchHdr {
    uint32_t nvol;
    uint32_t ntiles;     // smoothing tiles over the batch
    uint32_t nrowtiles;  // row tiles over the batch
    uint32_t tile_z;     // z-chunk of a smoothing tile
    uint32_t tile_y;     // rows of a smoothing tile
    uint32_t fs_tiles;   // k_smooth_rows tiles over the batch
    uint32_t nbricks;    // union-find bricks over the batch
    uint32_t nbtasks;    // k_union tasks over the batch
    uint32_t dn_items[3];// denoise box-pass items per axis over the batch
    uint32_t dn_tiles;   // denoise median tiles over the batch
    uint32_t cl_items;   // closing dilation items over the batch
    uint32_t dt_items[DT_NK]; // distance-map items per DtKernel over the batch
    uint32_t mrf_tiles;       // k_mrf_stats tiles over the batch
    uint32_t mrf_ctiles;      // k_mrf_step tiles over the batch
    uint32_t row_tile;        // rows per row tile: ROW_TILE, or down to ROW_TILE_MIN
                              // so that a batch with few rows still fills the GPU
    VolDev vol[1];       // nvol entries
};

inline size_t batch_bytes(uint32_t nvol) {
    return offsetof(BatchHdr, vol) + sizeof(VolDev) * (nvol ? nvol : 1);
}

// Host-side description of the kernels launched for one batch.
constexpr int NUM_KERNELS = 25;
extern const char *const kKernelNames[NUM_KERNELS];

struct LaunchPlan {
    int sms;             // multiprocessors on the device
    int tile_y;          // 8, 16 or 32
    int grid_hist;       // persistent grid of the histogram kernel
    int grid_vols;       // per-volume kernels
    // persistent grids of the row-tile, brick and run kernels: the blocks
    // that are resident at once (occupancy x SMs), so no block waits for a
    // slot while others already loop over their second item
    int grid_thr;        // k_threshold_runs
    int grid_rows;       // k_row_runs, k_keep_count, k_rank
    int grid_ul;         // k_union_local
    int grid_task;       // k_union, k_flatten
    int grid_lab;        // k_label_features
    int grid_box;        // k_box_pass
    int grid_med;        // k_median27
    bool rows;           // some volume of the batch takes k_smooth_rows
    bool tiles;          // some volume of the batch takes k_smooth_hist
    bool denoise;        // some volume of the batch runs the denoise front end
    bool closing;        // some volume of the batch closes its foreground
    bool distance;       // some volume of the batch has a distance map
    int grid_dist;       // k_dist_x, k_dist_line
    int grid_dxy16;      // k_dist_xy<16>
    int grid_dxy32;      // k_dist_xy<32>
    int grid_dz;         // k_dist_z
    int grid_mrf;        // k_mrf_stats
    int grid_mrfs;       // k_mrf_step
    uint32_t mrf_iters;  // k_mrf_step launches: the largest step limit in the batch (0: none)
};

// Enqueues the whole pipeline for a batch whose header lives at d_hdr (device)
// on `stream`.  ev, when non-null, holds NUM_KERNELS + 1 events recorded
// around the launches (external records, so they survive graph capture).
// stat_out receives nvol * ST_WORDS status words (volume-major).
cudaError_t launch_pipeline(const BatchHdr *d_hdr, const LaunchPlan &plan, cudaStream_t stream,
                            cudaEvent_t *ev, uint32_t *stat_out);

// Only the tile-dependent part (init + smoothing/histogram), for tile tuning.
cudaError_t launch_tile_probe(const BatchHdr *d_hdr, const LaunchPlan &plan, cudaStream_t stream);

// Denoise front end of the volumes with dn_r > 0 (none: the kernels exit).
constexpr int DN_CHUNK = 128;    // box-pass positions per tile along a line
constexpr int MED_TILE_X = 64, MED_TILE_Y = 8, MED_TILE_Z = 8;  // k_median27 tile (voxels)
constexpr int DN_MAX_R = 16;
constexpr int CL_MAX_R = 8;      // closing ball radius limit
cudaError_t launch_denoise(const BatchHdr *d_hdr, const LaunchPlan &plan, cudaStream_t stream);

// Cell-to-vessel distance: out[k - 1] = min of map over the voxels labelled k.
cudaError_t launch_cell_distance(const uint32_t *labels, const uint32_t *map, uint64_t n, uint32_t *out, uint64_t k,
                                 int sms, cudaStream_t s);
// Label runs of one label image (rows = Y*Z rows of X voxels): the count
// pass (per-row counts into rowcnt, per-block offsets into tiles, the total
// into *total) and the write pass (records into out, nothing when *total >
// cap; then, with mapped != null, the records copied on to that
// device-visible host memory).
uint32_t label_runs_tiles(uint32_t rows);
cudaError_t launch_label_runs_count(const uint32_t *labels, uint32_t X, uint32_t rows, uint32_t *rowcnt,
                                    uint32_t *tiles, uint32_t *total, int sms, cudaStream_t s);
cudaError_t launch_label_runs_write(const uint32_t *labels, uint32_t X, uint32_t rows, const uint32_t *rowcnt,
                                    const uint32_t *tiles, const uint32_t *total, uint64_t cap, seg_label_run *out,
                                    seg_label_run *mapped, int sms, cudaStream_t s);

// Histogram-kernel shared memory per block for a tile height.
size_t hist_smem_bytes(int tile_y);
// k_smooth_rows: threads per block, octets per tile row at most, and the
// tile shape of a row-aligned volume of width X.
constexpr int FS_NT = 512;
constexpr int FS_RT = 64;
inline uint32_t fs_rows_rt(uint32_t X) { return X >= 8u * FS_RT ? (uint32_t)FS_RT : (X + 7u) / 8u; }
// Sets kernel attributes on `device` and fills the persistent grid sizes of
// `plan` (plan.sms must be set).
cudaError_t configure_kernels(int device, LaunchPlan &plan);

}  // namespace seg
