/*
 * seg.h -- C ABI of libseg, a GB300 (sm_103a) library for the per-frame,
 * per-channel 3-D segmentation stage of LEVER 3-D (Wait et al.): smooth ->
 * histogram -> Otsu -> threshold -> 26-connected labelling -> minimum-volume
 * filter -> canonical numbering -> per-cell features.
 *
 * Paper passages the operations come from:
 *   - Background Noise Removal, Eq. 1: the stem-cell channel is low-pass
 *     (Gaussian) filtered.  Here: integer separable binomial smoothing
 *     [1 4 6 4 1] per axis, uint32 sums, one rounding (S + 2048) >> 12,
 *     replicate-edge borders.
 *   - Segmentation: adaptive Otsu thresholding of all channels (ref. [11])
 *     giving a binary foreground image; a connected component filter; cells
 *     below 19 um^3 discarded, the limit settable by the user before the run.
 *     Here: global Otsu over the frame's 65536-level histogram (binary64
 *     between-class variance, ties to the lowest level, foreground strictly
 *     above it), 26-connectivity, survivors numbered 1..K by their lowest
 *     linear voxel index.  The default limit, 30 voxels, is 19 um^3 at the
 *     0.8 x 0.8 x 1.0 um spacing of the Methods section.
 *     Optional steps of the same section: closing of the foreground with a
 *     binary ball before labelling, and (vessel channel) a distance map from
 *     every voxel to the nearest foreground voxel, here the exact weighted
 *     squared Euclidean distance.
 *   - Tracking, Eq. 6 uses each cell's voxel count; the per-cell record
 *     (count, inclusive bounding box, int64 coordinate sums) is what the
 *     later stages consume.
 *
 * Layout: a volume is uint16 [C][Z][Y][X] (channels planar, x fastest);
 * linear index i = x + X*(y + Y*z).  Labels are uint32 [Z][Y][X] per channel,
 * 0 = background, 1..K = cells.  Limits: X*Y*Z < 2^32, X <= 65536, Y and Z
 * <= SEG_MAX_YZ.
 *
 * Threading: one thread may submit while another polls and reads; calls on
 * one context are otherwise serialised by the caller.  No call throws; every
 * call returns SEG_OK (0) or a negative SEG_E* code.  Device pointers are
 * CUDA device addresses on the context's device.
 */
#ifndef SEG_H
#define SEG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- return codes ------------------------------------------------------- */
#define SEG_OK 0
#define SEG_EINVAL (-1)    /* null pointer, zero dimension, channels == 0, bad field */
#define SEG_ETOOBIG (-2)   /* X*Y*Z >= 2^32, X > 65536, or footprint > HBM budget  */
#define SEG_EAGAIN (-3)    /* host queue full: retry after polling / releasing      */
#define SEG_ENOTREADY (-4) /* read of a request that is not DONE                    */
#define SEG_ETIMEOUT (-5)  /* seg_poll timed out, or a bounded device wait gave up  */
#define SEG_ECUDA (-6)     /* a CUDA call failed; the request is FAILED             */
#define SEG_ESMALL (-7)    /* destination too small (n_cells is still reported)     */
#define SEG_ENOENT (-8)    /* unknown or released request handle                    */
#define SEG_EFAILED (-9)   /* the request FAILED (device error flag or CUDA error)  */

/* Largest Y and Z of a volume (row and plane indices stay int-sized with
 * their halos); larger extents give SEG_ETOOBIG. */
#define SEG_MAX_YZ 2147483583u

/* ---- request states (seg_poll) ------------------------------------------ */
#define SEG_PENDING 0
#define SEG_DONE 1
#define SEG_FAILED 2

/* ---- seg_config.flags ---------------------------------------------------- */
#define SEG_FORCE_TILE 0x1u /* use tile_y / tile_z as given, skip the autotuner   */
#define SEG_PLAIN 0x2u      /* plain per-frame form: one request per launch
                               sequence, one stream, no batching                 */
#define SEG_NO_GRAPH 0x4u   /* kernels launched one by one, without CUDA-graph
                               capture                                           */
#define SEG_PROFILE 0x8u    /* record CUDA events around every kernel launch     */
#define SEG_TEST_UNION_FAIL 0x10u /* test hook: every union-find union gives up at
                                     once and raises its error bit, so requests
                                     with adjacent runs end FAILED (error path
                                     without any device fault)                  */
#define SEG_KEEP_SMOOTHED 0x20u /* keep each channel's smoothed image (2 bytes per
                                   voxel more per request) for seg_read_smoothed */

typedef struct seg_ctx seg_ctx; /* opaque; owns streams, graphs, device state   */
typedef uint64_t seg_req;       /* request handle, never 0                       */

typedef struct {
    uint32_t x, y, z;
} seg_dims;

/* One cell, 64 bytes; cells are stored in label order 1..K. */
typedef struct {
    uint64_t count;       /* voxels in the cell                                 */
    int64_t sum[3];       /* sum of x, y, z over its voxels (0-based coords)   */
    uint32_t bbox_min[3]; /* inclusive                                          */
    uint32_t bbox_max[3]; /* inclusive                                          */
    uint32_t pad[2];
} seg_cell_features;

/* One run of a label image, 12 bytes: voxels x_begin..x_end (inclusive) of
 * row `row` (= y + Y*z) carry label `label` (>= 1). */
typedef struct {
    uint32_t label;
    uint32_t row;
    uint16_t x_begin;
    uint16_t x_end;
} seg_label_run;

typedef struct {
    int device;                /* CUDA ordinal                                   */
    uint64_t hbm_budget_bytes; /* admission limit for all device state; 0 -> 80 %
                                  of the device's free memory at seg_create      */
    uint32_t max_inflight;     /* batches in flight (streams); 0 -> 2            */
    uint32_t flags;            /* SEG_FORCE_TILE | SEG_PLAIN | ...               */
    uint32_t tile_y;           /* smoothing tile rows: 16, 32 or 64 (FORCE_TILE) */
    uint32_t tile_z;           /* smoothing z-chunk, >= 1 (FORCE_TILE)           */
    uint32_t max_batch_volumes;/* volume-channels per launch; 0 -> 512           */
    uint32_t batch_window_us;  /* wait this long for more requests before a
                                  launch when nothing is in flight; 0 -> launch
                                  at once                                        */
    uint32_t host_queue;       /* requests held on the host awaiting admission;
                                  0 -> 4096                                      */
    void *order_stream;        /* optional cudaStream_t: device inputs are read
                                  only after the work queued on it at submit    */
} seg_config;

typedef struct {
    uint32_t min_volume_voxels; /* keep cells with >= this many voxels (30)      */
    /* 0: off.  1..16: the denoise front end of the stem-cell channel
     * (Background Noise Removal, Eq. 1) runs before the smoothing: the
     * background is three box filters of width 2r+1 along x, then y, then z
     * (each rounding to nearest, replicate edges), it is subtracted with a
     * floor at 0, and the 3x3x3 median of the difference is segmented. */
    uint32_t denoise_radius;
    /* 0: off.  1..8: the foreground is closed with the binary ball of this
     * radius (offsets with dx^2 + dy^2 + dz^2 <= r^2) before labelling,
     * dilation then erosion on the volume padded with background, so the
     * closed foreground contains the original (Segmentation section). */
    uint32_t closing_radius;
    /* {0, 0, 0}: off.  Otherwise every voxel gets the weighted squared
     * distance wx*dx^2 + wy*dy^2 + wz*dz^2 (uint32, exact) to the nearest
     * voxel of the channel's final (closed) foreground, 0 on the foreground,
     * 0xFFFFFFFF everywhere when the foreground is empty: the vessel-channel
     * distance map of the Segmentation section, read back with
     * seg_read_distance.  Weights are the squared voxel spacing in any common
     * unit (16, 16, 25 is 0.8 x 0.8 x 1.0 um in units of 0.2 um); each must be
     * >= 1 and wx(X-1)^2 + wy(Y-1)^2 + wz(Z-1)^2 < 0xFFFFFFFF, else
     * seg_submit_volume returns SEG_EINVAL. */
    uint32_t distance_weights[3];
    /* 0: off.  1..1000: the MRF denoise of the vessel channel (Background
     * Noise Removal, Eqs. 2-3) runs before the smoothing, at most this many
     * steps: every voxel moves by Delta (the smallest gap between two
     * distinct input levels) towards the majority of its six face
     * neighbours (a neighbour votes +1 if higher, -1 if lower, 0 if equal
     * or outside the volume), all voxels at once, clamped to [0, 65535];
     * a step is kept while the root-mean-square difference from the input
     * stays within the noise level sigma = sqrt(pi/2) S / (6 M), S the
     * summed absolute response of the plane mask [1 -2 1; -2 4 -2; 1 -2 1]
     * over the M interior voxels of the z-planes (binary64: the step is kept
     * iff (double)sum d^2 <= (N sigma) sigma); the iteration also stops at a
     * step that changes nothing.  Not combined with denoise_radius
     * (SEG_EINVAL). */
    uint32_t mrf_iterations;
} seg_channel_params;

/* Creates a context on cfg->device.  Allocates streams and descriptor buffers;
 * runs the tile autotuner unless SEG_FORCE_TILE or SEG_PLAIN is set.
 * *out is set on success.  Errors: SEG_EINVAL, SEG_ECUDA. */
int seg_create(const seg_config *cfg, seg_ctx **out);

/* Waits for all in-flight work, frees every request and the context. */
int seg_destroy(seg_ctx *ctx);

/* Submits one volume of `channels` planar channels, each [Z][Y][X] uint16,
 * for the segmentation stage of each channel (Background Noise Removal,
 * Eq. 1: the binomial low-pass; Segmentation section: Otsu threshold (ref.
 * [11]), 26-connected components, components below the minimum volume
 * discarded, cells numbered by lowest linear index).
 *   voxels     host pointer (on_device = 0 or 2) or device pointer
 *              (on_device = 1, 2-byte aligned, else SEG_EINVAL; rows of
 *              X % 8 == 0 voxels from a 16-byte aligned pointer, or of an
 *              even X >= 10 from a 4-byte aligned one, take the faster
 *              smoothing kernel, the same results either way).  With 0 the input is copied before the call
 *              returns (the caller may free or reuse it).  With 2 the copy is
 *              only queued (pinned memory: it runs while the call returns and
 *              the batch waits for it on the device), so the host input, like
 *              a device input, must stay valid and unchanged until seg_poll
 *              reports DONE or FAILED.  Other values: SEG_EINVAL.
 *   per_channel  array of `channels` params, or NULL for the default (30).
 * On success *out is a new handle.  Results stay on the device until
 * seg_release.  Errors: SEG_EINVAL, SEG_ETOOBIG (can never be admitted),
 * SEG_EAGAIN (host queue full), SEG_ECUDA. */
int seg_submit_volume(seg_ctx *ctx, const uint16_t *voxels, int on_device, seg_dims dims,
                      uint32_t channels, const seg_channel_params *per_channel, seg_req *out);

/* Launches everything submitted so far without waiting for the batch window. */
int seg_flush(seg_ctx *ctx);

/* Waits up to timeout_ms for the request to leave PENDING; *state is set to
 * SEG_PENDING, SEG_DONE or SEG_FAILED.  Returns SEG_ETIMEOUT if still
 * pending, SEG_ENOENT for an unknown handle. */
int seg_poll(seg_ctx *ctx, seg_req req, uint32_t timeout_ms, int *state);

/* Makes `stream` (a cudaStream_t on the context's device; NULL is the legacy
 * default stream) wait until the request's results are complete.  If the
 * request has not been launched yet this flushes the queue and blocks the
 * host until its launch sequence is enqueued; the device wait itself never
 * blocks the host. */
int seg_enqueue_wait(seg_ctx *ctx, seg_req req, void *stream);

/* Copies channel `channel`'s label image (X*Y*Z uint32; Segmentation
 * section: 0 = background, 1..K = the cells in order of their lowest linear
 * index) to dst (host, or device when dst_on_device = 1).  Blocks until the
 * copy is complete.
 * Errors: SEG_ENOTREADY, SEG_EFAILED, SEG_ESMALL (dst_elems < X*Y*Z),
 * SEG_EINVAL, SEG_ENOENT, SEG_ECUDA. */
int seg_read_labels(seg_ctx *ctx, seg_req req, uint32_t channel, uint32_t *dst,
                    uint64_t dst_elems, int dst_on_device);

/* Channel `channel`'s label image as runs (Segmentation section: each
 * cell's voxels, the set the paper passes on to the convex hull step): the
 * maximal stretches of equal non-zero label along x within one row, in order
 * of row (y + Y*z) and then x, one seg_label_run each.  Painting the runs
 * into a zeroed X*Y*Z image gives exactly seg_read_labels' image; a row of
 * X voxels holds at most ceil(X/2) runs.  *n_runs gets the number of runs.
 * dst holds cap runs in host memory, or device memory when dst_on_device = 1;
 * dst = NULL with cap = 0 only reports the number.  Derived on the device
 * from the label image (two passes over it) and copied; blocks until done.
 * Errors: SEG_ESMALL (cap < *n_runs, nothing written); SEG_ETOOBIG for an
 * image of more than 2^32 - 65 rows; otherwise as seg_read_labels. */
int seg_read_label_runs(seg_ctx *ctx, seg_req req, uint32_t channel, seg_label_run *dst, uint64_t cap,
                        uint64_t *n_runs, int dst_on_device);

/* Copies channel `channel`'s distance map (X*Y*Z uint32, layout of the
 * labels) to dst (host, or device when dst_on_device = 1).  Blocks until the
 * copy is complete.  Errors: SEG_EINVAL also when the channel was submitted
 * without distance weights; otherwise as seg_read_labels. */
int seg_read_distance(seg_ctx *ctx, seg_req req, uint32_t channel, uint32_t *dst,
                      uint64_t dst_elems, int dst_on_device);

/* The distance of every cell of channel cells_channel to the nearest
 * foreground voxel of channel map_channel (Fig. 4: each stem cell's distance
 * to its nearest vessel): dst[k - 1] = the smallest value of map_channel's
 * distance map over the voxels of cell k (weighted squared distance, see
 * seg_channel_params.distance_weights), K = the cells of cells_channel
 * (*n_cells, optional).  dst is host memory of cap entries; dst = NULL with
 * cap = 0 only reports K.  Blocks until done.  Errors: SEG_EINVAL also when
 * map_channel has no distance map; SEG_ESMALL (cap < K); otherwise as
 * seg_read_labels. */
int seg_read_cell_distance(seg_ctx *ctx, seg_req req, uint32_t cells_channel, uint32_t map_channel, uint32_t *dst,
                           uint64_t cap, uint64_t *n_cells);

/* Copies the image channel `channel` was segmented from after its denoise
 * (front end or MRF; X*Y*Z uint16, layout of the input) to dst (host, or
 * device when dst_on_device = 1); *mrf_steps (optional) gets the number of
 * MRF steps kept (0 for the front end).  Blocks until the copy is complete.
 * Errors: SEG_EINVAL also when the channel has neither denoise; otherwise as
 * seg_read_labels. */
int seg_read_denoised(seg_ctx *ctx, seg_req req, uint32_t channel, uint16_t *dst, uint64_t dst_elems,
                      int dst_on_device, uint32_t *mrf_steps);

/* Copies the smoothed image of channel `channel` (X*Y*Z uint16, layout of the
 * input) to dst (host, or device when dst_on_device = 1): the low-pass of
 * Background Noise Removal, Eq. 1, as computed here -- the binomial
 * [1 4 6 4 1] along x, y and z, the uint32 sum S rounded once to
 * (S + 2048) >> 12, edges replicated -- which is the image the Otsu
 * histogram counts and the threshold compares.  Only for contexts created
 * with SEG_KEEP_SMOOTHED (otherwise SEG_EINVAL); blocks until the copy is
 * complete.  Other errors as seg_read_labels. */
int seg_read_smoothed(seg_ctx *ctx, seg_req req, uint32_t channel, uint16_t *dst, uint64_t dst_elems,
                      int dst_on_device);

/* Copies channel `channel`'s cells (label order; per cell the voxel count,
 * bounding box and coordinate sums, which stand in for the hull the
 * Segmentation section builds) to host memory dst (cap entries) and reports
 * n_cells and the Otsu level t* (foreground = s > t*).
 * dst may be NULL with cap 0 to query n_cells.  SEG_ESMALL if cap < n_cells
 * (n_cells and the threshold are still set). */
int seg_read_features(seg_ctx *ctx, seg_req req, uint32_t channel, seg_cell_features *dst,
                      uint64_t cap, uint64_t *n_cells, uint16_t *otsu_threshold);

/* Frees the request's device state and returns its bytes to the budget. */
int seg_release(seg_ctx *ctx, seg_req req);

/* Host timestamps of a request in milliseconds since seg_create: submitted,
 * admitted (device memory reserved), launched, completed (device work done,
 * observed by the runtime).  Values not reached yet are negative. */
int seg_request_times(seg_ctx *ctx, seg_req req, double *submit_ms, double *admit_ms,
                      double *launch_ms, double *done_ms);

#define SEG_MAX_KERNELS 32
typedef struct {
    uint64_t batches;                 /* launch sequences completed            */
    uint64_t volumes;                 /* volume-channels segmented             */
    uint64_t voxels;                  /* voxels segmented (all channels)       */
    uint32_t tile_y, tile_z;          /* tile shape in use                     */
    uint32_t n_kernels;
    char names[SEG_MAX_KERNELS][32];  /* kernel names, launch order            */
    uint64_t launches[SEG_MAX_KERNELS];
    double total_ms[SEG_MAX_KERNELS]; /* CUDA-event time (SEG_PROFILE only)    */
    uint64_t bytes_in_use;            /* budget accounting                     */
    uint64_t budget_bytes;
} seg_stats;

/* Counters since seg_create or the last seg_reset_stats. */
int seg_get_stats(seg_ctx *ctx, seg_stats *out);
int seg_reset_stats(seg_ctx *ctx);

/* Allocation-free Otsu level of one device-resident volume.  The paper has
 * no counterpart: this entry point exists for callers that cannot allocate
 * device memory -- their HBM is wholly reserved by another allocator (for
 * example a framework's caching allocator), or they run latency-critical
 * loops where cudaMalloc/cudaFree and their implicit synchronisation are not
 * acceptable.  It needs no seg_ctx and calls no allocating routine.
 *
 *   d_voxels  device pointer, uint16 [Z][Y][X] of the current device,
 *             2-byte aligned (else SEG_EINVAL).
 *   d_result  device pointer (4-byte aligned) to 2 uint32: [0] = Otsu level t* of the
 *             smoothed volume (the value seg_read_features reports for the
 *             same input), [1] = error bits (0 = ok).
 *   stream    cudaStream_t on the current device (NULL = legacy default).
 * Work is enqueued on `stream`; the call does not wait for it.
 *
 * Scratch: one fixed 262,208-byte device array per GPU (65536 histogram bins
 * and 16 status words), held by every GPU that loads the library until the
 * process exits.  Every call on a device shares it and it keeps the last
 * call's contents; the call clears it on `stream` first.  Calls whose work
 * overlaps on the GPU (different streams, or several host threads) race on it
 * and must be serialised by the caller.  The first call on a device (with
 * that device current) resolves the array's device address and sets kernel
 * attributes; make that first call before any stream capture.
 * Limits: X*Y*Z <= SEG_NOALLOC_MAX_VOXELS (the bins count in uint32),
 * X <= 65536 and Y, Z <= SEG_MAX_YZ, else SEG_ETOOBIG; these and the
 * argument checks are made before any CUDA call.  Other errors: SEG_EINVAL,
 * SEG_ECUDA. */
#define SEG_NOALLOC_MAX_VOXELS 4294967295ull
int seg_otsu_threshold_noalloc(const uint16_t *d_voxels, seg_dims dims, uint32_t *d_result,
                               void *stream);

/* Human-readable text for a return code (static storage). */
const char *seg_strerror(int code);

/* ---- montage registration (Registration section, Eq. 4) ----------------- */

typedef struct {
    int32_t x, y, z;
} seg_offset;

/* One overlapping pair of tiles, 40 bytes. */
typedef struct {
    uint32_t a, b;     /* tiles, a < b, whose stage boxes overlap          */
    seg_offset shift;  /* best shift of tile b away from its stage position */
    uint32_t pad0;
    double score;      /* normcov at that shift; -2 when no shift had one   */
    uint32_t in_tree;  /* 1: edge of the maximum spanning tree              */
    uint32_t pad1;
} seg_montage_edge;

#define SEG_REG_MAX_RXY 12 /* search half-width limits along x and y, and z */
#define SEG_REG_MAX_RZ 6

/* Registers n_tiles tiles of one montage (all dims.x * dims.y * dims.z
 * uint16, [Z][Y][X]; tiles[i] a host pointer, or a device pointer on
 * `device` when on_device = 1) placed at stage[i] (voxels, one global frame).
 * Every pair whose stage boxes overlap is scored at each shift s of the
 * second tile with |s.x|, |s.y| <= radius.x, radius.y (<= SEG_REG_MAX_RXY)
 * and |s.z| <= radius.z (<= SEG_REG_MAX_RZ): normcov (Eq. 4, read as the
 * Pearson correlation (N Sab - Sa Sb) / sqrt((N Saa - Sa^2)(N Sbb - Sb^2))
 * over the voxels the two tiles then share, exact integer sums, binary64
 * ratio), and keeps the first best shift in z, y, x order.  A maximum
 * spanning tree of the pairs (Kruskal, ties by (a, b)) anchors tile `root`;
 * delta[i] gets the correction of tile i (stage + delta is its registered
 * position; 0 for tiles the tree does not reach).  edges (cap edges_cap)
 * gets the pairs in (a, b) order and *n_edges their number.  Blocks until
 * done.  Errors: SEG_EINVAL (null pointer, zero size, root >= n_tiles, a
 * radius outside its limit), SEG_ETOOBIG (a tile of 2^32 voxels or more),
 * SEG_ESMALL (edges_cap < *n_edges: nothing else is written), SEG_ECUDA. */
int seg_register_montage(int device, const uint16_t *const *tiles, int on_device, uint32_t n_tiles,
                         seg_dims dims, const seg_offset *stage, seg_offset radius, uint32_t root,
                         seg_offset *delta, seg_montage_edge *edges, uint32_t edges_cap, uint32_t *n_edges);

#ifdef __cplusplus
}
#endif

#endif /* SEG_H */
