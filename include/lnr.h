/*
 * lnr.h -- C ABI of the GB300 render path of "Real-time Neural Rendering of LiDAR Point
 * Clouds" (arXiv 2502.11618): a coloured multi-scan LiDAR cloud is partitioned by a
 * uniform grid, culled against the view frustum, projected as 1x1 pixels into an RGBDA
 * image, pruned by the depth-guided filter and turned into the output frame by a
 * fully convolutional U-Net.
 *
 * Conventions shared by every call:
 *  - All pointers are plain host pointers unless an argument says "device".  Input
 *    buffers belong to the caller; the library copies what it needs during the call and
 *    keeps no pointer to them.  Output buffers are allocated by the caller.
 *  - Images are row-major, pixel (u, v) at index v*W + u; multi-channel images are
 *    interleaved (HWC).  Batched images are view-major (NHWC).
 *  - Every call returns an lnr_status.  No call aborts the process.  After an error,
 *    lnr_last_error() describes it.
 *  - A context owns one CUDA device and one stream; its calls are not thread-safe,
 *    except lnr_submit / lnr_poll / lnr_serve_stats, which may be called from any
 *    thread.
 */
#ifndef LNR_H
#define LNR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lnr_ctx lnr_ctx;

typedef enum {
    LNR_OK = 0,
    LNR_E_ARG = -1,      /* an argument is out of range, NULL or not finite */
    LNR_E_STATE = -2,    /* calls out of order (render before build_grid / set_unet) */
    LNR_E_OOM = -3,      /* device memory or the memory budget is exhausted */
    LNR_E_CUDA = -4,     /* a CUDA call failed */
    LNR_E_TIMEOUT = -5,  /* a bounded device or host wait ran out */
    LNR_E_BUSY = -6      /* lnr_poll: the request is not finished yet */
} lnr_status;

typedef enum { LNR_FP32 = 0, LNR_BF16 = 1, LNR_FP8 = 2 } lnr_precision;

/* A view: world-to-camera rotation R (row-major 3x3; camera x right, y down, z forward)
 * and camera centre C in world coordinates.  Both in FP64: with georeferenced clouds the
 * camera-relative geometry is formed in FP64 on the host before any FP32 rounding. */
typedef struct {
    double R[9];
    double C[3];
} lnr_view;

/* Pinhole intrinsics (pixels) and the depth range; a point is drawn when
 * znear < z < zfar.  zfar also normalises the depth channel of the U-Net input. */
typedef struct {
    float fx, fy, cx, cy, znear, zfar;
} lnr_intrinsics;

/* U-Net shape: `levels` resolution levels with ch[l] channels, in_ch = 5 (RGBDA),
 * out_ch = 3 (RGB); has_bn = 1 when the weight file carries batch-norm statistics for the
 * encoder convolutions. */
typedef struct {
    int levels;
    int ch[8];
    int in_ch;
    int out_ch;
    int has_bn;
} lnr_unet_desc;

/* Stages that lnr_render_stage can stop after (parity and debugging taps). */
typedef enum {
    LNR_STAGE_KEYS = 0,       /* uint64 [H*W]: (float bits of z << 32 | sorted position), ~0 = empty */
    LNR_STAGE_RGBDA_RAW = 1,  /* 8 bytes per pixel: float z (+inf empty), uint8 r, g, b, A */
    LNR_STAGE_FILTERED = 2,   /* float [H*W]: kept depth, +inf where empty or filtered out */
    LNR_STAGE_UNET_IN = 3,    /* float [H*W*5]: r/255, g/255, b/255, z/zfar, A (zero where A = 0) */
    LNR_STAGE_CULL = 4        /* uint64 [2]: visible non-empty cells, visible points */
} lnr_stage;

/* Create a context on CUDA device `device`.  cuda_stream (nullable) is a cudaStream_t the
 * context issues its work on; NULL makes the context create its own stream. */
lnr_status lnr_create(lnr_ctx** out, int device, void* cuda_stream);
lnr_status lnr_destroy(lnr_ctx* ctx);

/* Last error message of this context ("" when none).  Valid until the next call. */
const char* lnr_last_error(lnr_ctx* ctx);

/* Upload a cloud (Sec. 1: merged multi-scanner coloured points).  xyz: n x 3 FP64 world
 * coordinates; rgb: n x 3 uint8; scan_id: n uint8 source-scanner index (nullable: 0).
 * Invalidates any grid built before.  n must be in [1, 2^32 - 1]. */
lnr_status lnr_load_cloud(lnr_ctx* ctx, const double* xyz, const uint8_t* rgb,
                          const uint8_t* scan_id, uint64_t n);

/* Uniform-grid partition of the loaded cloud (Sec. 1; Sec. 3, "Point Cloud
 * Projection"), built on the device: grid origin g0 = floor(min/cell)*cell, stable
 * counting sort of the points by cell id (k*dy + j)*dx + i, and per point an FP32 offset to
 * its cell's FP64 origin.  cell_size > 0; at most 2^31 cells. */
lnr_status lnr_build_grid(lnr_ctx* ctx, double cell_size);

/* Grid summary: out_g0[3] (FP64 origin), out_dims[3] (cells per axis); nullable each. */
lnr_status lnr_grid_info(lnr_ctx* ctx, double* out_g0, int32_t* out_dims);

/* Load the U-Net (Fig. 1; Sec. 3, "U-Net Reconstruction").  weights: n_floats FP32 values;
 * for every convolution in network order (enc0a, enc0b, ..., the bottleneck pair, then
 * dec(L-2)a, dec(L-2)b, ..., dec0a, dec0b) its OIHW weight then its bias; then the 1x1 head
 * (OIHW, bias); then, if has_bn, (gamma, beta, mean, var) per encoder convolution (folded
 * into that convolution here, eps 1e-5).  A decoder "a" convolution reads the skip
 * tensor's channels first, the nearest-upsampled deeper tensor's after.  The weights are
 * converted for every precision; `precision` selects the one lnr_render uses. */
lnr_status lnr_set_unet(lnr_ctx* ctx, const lnr_unet_desc* desc, const float* weights,
                        size_t n_floats, lnr_precision precision);

/* Select the U-Net precision for later renders (weights must be loaded; LNR_FP8 also needs
 * lnr_calibrate).  lnr_set_unet with LNR_FP8 loads the weights, selects BF16 and returns
 * LNR_E_STATE until the net is calibrated. */
lnr_status lnr_set_precision(lnr_ctx* ctx, lnr_precision precision);

/* Network input of one synthetic training pair (Sec. 3, "Training Data Generation").  The frame is
 * projected and filtered at this view exactly as lnr_render does (n_levels, fs), then
 * composed with a caller's ground-truth photo gt_rgb (host, H*W*3 FP32 HWC, any range):
 *  - unfiltered = 0 (the filtered net's input): RGB = gt where the filter keeps the
 *    pixel (A^s = 1), D = z / zfar there, A = A^s; zero elsewhere;
 *  - unfiltered = 1 (the unfiltered net's input): every filled pixel, RGB = gt for pixels
 *    the filter keeps (foreground) and the projected point colour / 255 for pixels it
 *    drops (background), D = z / zfar, A = 1; zero where no point falls.
 * out: host, H*W*5 FP32 (r, g, b, D, A).  The ground truth of the pair is gt itself.
 * Errors as lnr_render_stage; LNR_E_ARG for null gt_rgb / out.  Allocates temporaries. */
lnr_status lnr_training_input(lnr_ctx* ctx, const lnr_view* view, const lnr_intrinsics* intr,
                              int W, int H, int n_levels, float fs, const float* gt_rgb,
                              int unfiltered, float* out);

/* ---- cloud shards: one cloud split over several contexts (GPUs) ----
 * A cloud too large for one GPU is split by cells: every shard holds the points of a range
 * of cells of one common grid frame.  Each shard splats its points into z-buffer keys
 * (lnr_render_stage, LNR_STAGE_KEYS) whose position field is the point's position in the
 * whole cloud's sorted order (lnr_set_shard).  The element-wise minimum of the shards' keys
 * is the whole cloud's z-buffer, bit for bit.  Each shard resolves the colours of its own
 * front points (lnr_shard_resolve); the element-wise sum (or maximum) of the shards'
 * colours is the whole cloud's.  Any one context then finishes the frame
 * (lnr_shard_finish).  The two exchanges (a u64 min and a u32 sum over the shards) belong
 * to the caller, e.g. NCCL all-reduces.  Not with the soft z-buffer. */

/* Build the grid in a given frame (cell size, origin g0[3] FP64, dims[3] cells), as
 * lnr_build_grid would for the whole cloud (lnr_grid_info of a context holding it, or the
 * same formulas): points are sorted by cell as usual, points outside the frame go to its
 * border cells.  Errors: LNR_E_STATE before load_cloud; LNR_E_ARG for a bad frame. */
lnr_status lnr_build_grid_frame(lnr_ctx* ctx, double cell_size, const double* g0, const int32_t* dims);

/* Make this context a cloud shard: key positions are its sorted positions + pos_base (the
 * number of the whole cloud's points in the cells before this shard's), and the resolve
 * colours only keys inside [pos_base, pos_base + n).  0 (the default) for a whole cloud.
 * Errors: LNR_E_ARG when positions would exceed 32 bits; LNR_E_STATE while serving. */
lnr_status lnr_set_shard(lnr_ctx* ctx, uint32_t pos_base);

/* A shard's colours for the whole cloud's keys.  keys: device, H*W uint64 (the shards'
 * minimum); rgba: device, H*W uint32 written: r | g << 8 | b << 16 | 1 << 24 where the
 * front point is this shard's, 0 elsewhere.  view / intr / W / H as lnr_render. */
lnr_status lnr_shard_resolve(lnr_ctx* ctx, const lnr_view* view, const lnr_intrinsics* intr, int W,
                             int H, const uint64_t* keys, uint32_t* rgba);

/* The frame from the whole cloud's keys and colours (device buffers as above): depth
 * filter (Fig. 2) with n_levels / fs, U-Net, out_rgb as lnr_render (host, or device when
 * out_on_device).  Equals lnr_render of a context holding the whole cloud, bit for bit. */
lnr_status lnr_shard_finish(lnr_ctx* ctx, const lnr_view* view, const lnr_intrinsics* intr, int W,
                            int H, int n_levels, float fs, const uint64_t* keys, const uint32_t* rgba,
                            float* out_rgb, int out_on_device);

/* Collision rule of the splat (Sec. 3, "Point Cloud Projection").  rel = 0 (the default):
 * hard z-buffer, each pixel keeps its nearest point (depth ties: lower sorted position).
 * rel > 0: soft z-buffer, the pixel's colour is the per-channel integer mean, rounded half
 * up, of every point that projects to it with depth z <= z_front * (1 + rel) (one FP32
 * multiply), z_front its nearest depth; depth and the filter are unchanged.  The paper
 * states no threshold.  Costs a second pass over the visible points and 16 bytes per
 * pixel.  Errors: LNR_E_ARG for rel negative, NaN or above 1e6; LNR_E_STATE while serving. */
lnr_status lnr_set_soft_zbuffer(lnr_ctx* ctx, float rel);

/* Render one frame (Fig. 1): cull, splat, filter (Fig. 2) with n_levels min-pool levels
 * and filter_strength fs, U-Net.  out_rgb: H*W*3 FP32 in [0, 1], HWC; host memory, or
 * device memory when out_on_device != 0 (then the call returns without waiting for the
 * GPU; the result is complete when the context's stream reaches it).
 * Errors: LNR_E_STATE before build_grid / set_unet; LNR_E_ARG when W or H is not a
 * positive multiple of 2^(levels-1), n_levels is outside [0, floor(log2(min(W, H)))] or
 * above 6, fs is negative or NaN, or the view is not finite. */
lnr_status lnr_render(lnr_ctx* ctx, const lnr_view* view, const lnr_intrinsics* intr, int W,
                      int H, int n_levels, float fs, float* out_rgb, int out_on_device);

/* The same path stopped after `stage`; `out` (host, or device when out_on_device) receives
 * the buffer lnr_stage describes.  Needs set_unet only for no stage. */
lnr_status lnr_render_stage(lnr_ctx* ctx, const lnr_view* view, const lnr_intrinsics* intr,
                            int W, int H, int n_levels, float fs, int stage, void* out,
                            int out_on_device);

/* Render nviews views of one resolution in one pass: every view's splat, filter and
 * U-Net run batched (the U-Net on an NHWC batch).  views, intr and fs are arrays of
 * nviews; out_rgb holds nviews*H*W*3 floats, view-major.  With out_on_device the U-Net
 * writes out_rgb directly (the frame's CUDA graph is kept per configuration and output
 * buffer, for up to 256 of them).  One resolution and pyramid depth per call: views of other sizes go to other
 * calls, or to the serving loop, which runs batches of different sizes side by side on
 * its slots.  Same errors as lnr_render. */
lnr_status lnr_render_batch(lnr_ctx* ctx, int nviews, const lnr_view* views,
                            const lnr_intrinsics* intr, int W, int H, int n_levels,
                            const float* fs, float* out_rgb, int out_on_device);

/* Calibrate the FP8 (E4M3) U-Net on one view (after set_unet): the view is rendered with
 * the BF16 U-Net, the largest magnitude of every convolution's output sets that tensor's
 * static scale (headroom x amax / 448; the headroom leaves room for views with larger
 * activations), and E4M3 weights with per-output-channel scales are built with the input
 * scales folded in; accumulation stays FP32 (the paper states no precision; reduced
 * precision is this library's addition).  Afterwards lnr_set_precision(LNR_FP8) is
 * allowed.  Arguments as lnr_render.  Errors: as lnr_render; LNR_E_ARG when a channel count
 * of the net is not a multiple of 32. */
lnr_status lnr_calibrate(lnr_ctx* ctx, const lnr_view* view, const lnr_intrinsics* intr, int W,
                         int H, int n_levels, float fs);

/* The same calibration over nviews views rendered as one batch (arrays as
 * lnr_render_batch): every tensor's scale comes from its largest magnitude over all of
 * them, so the scales cover the spread of activations between views. */
lnr_status lnr_calibrate_batch(lnr_ctx* ctx, int nviews, const lnr_view* views,
                               const lnr_intrinsics* intr, int W, int H, int n_levels,
                               const float* fs);

/* Autotune the tensor-core U-Net for batches of `batch` views at W x H (part of this
 * library's batching; the paper has no counterpart): for every convolution, every valid
 * kernel configuration (generic kernel; halo kernel over tile heights, parity classes per
 * tile, K-chunk widths, epilogue warps, direct or staged stores) is timed on the device
 * and the fastest is kept for that layer resolution; later renders and served batches at
 * that resolution use it.  Runs on the
 * context's stream and waits for it.  Needs set_unet; a no-op for the FP32 precision.
 * Errors: LNR_E_STATE before set_unet, LNR_E_ARG for sizes as lnr_render or batch outside
 * [1, 64], LNR_E_OOM / LNR_E_CUDA. */
lnr_status lnr_autotune(lnr_ctx* ctx, int W, int H, int batch);

/* ---- serving: continuous batching of render requests ------------------------------ */

/* Start the serving loop: up to max_batch requests of one resolution per launch, up to
 * `slots` launches in flight.  The frames run in launch order on one compute stream of the
 * loop; each slot copies its results to host memory on a stream of its own, overlapping
 * the next frames.  Uses the precision selected by set_unet / set_precision at this call.
 * Errors: LNR_E_STATE (already serving, or no grid / network), LNR_E_ARG (max_batch
 * outside [1, 64], slots outside [1, 16]), LNR_E_CUDA. */
lnr_status lnr_serve_start(lnr_ctx* ctx, int max_batch, int slots);
lnr_status lnr_serve_stop(lnr_ctx* ctx);
/* Device-memory budget of the serving loop's slots (0 = no bound): a batch is admitted when
 * the buffers of the slots already busy plus the batch's own need fit, and slots release
 * buffers they no longer need so that all slots together hold at most `bytes` (a single
 * request larger than the budget still runs, alone). */
lnr_status lnr_set_memory_budget(lnr_ctx* ctx, size_t bytes);

/* Queue one render request; *ticket identifies it.  Thread-safe.  Arguments as
 * lnr_render; they are copied. */
lnr_status lnr_submit(lnr_ctx* ctx, const lnr_view* view, const lnr_intrinsics* intr, int W,
                      int H, int n_levels, float fs, uint64_t* ticket);

/* As lnr_submit, with the result's destination given now: out_rgb (host, H*W*3 floats,
 * owned by the caller, valid and untouched until lnr_poll reports the request done).  When
 * out_rgb is page-locked (cudaHostAlloc / cudaHostRegister) the device copies the result
 * straight into it and lnr_poll copies nothing; otherwise the result goes through the
 * library's page-locked buffers and lnr_poll copies it into out_rgb (when its own out_rgb
 * is null).  Thread-safe.  Part of this library's serving; the paper has no counterpart. */
lnr_status lnr_submit_into(lnr_ctx* ctx, const lnr_view* view, const lnr_intrinsics* intr, int W,
                           int H, int n_levels, float fs, float* out_rgb, uint64_t* ticket);

/* Result of a request: LNR_E_BUSY until it is done, then copies H*W*3 floats to out_rgb
 * (host, nullable) and its latency (completion minus submission, seconds) to
 * *latency_s (nullable), and forgets the request.  Thread-safe. */
lnr_status lnr_poll(lnr_ctx* ctx, uint64_t ticket, float* out_rgb, double* latency_s);

/* Serving counters: out[0] requests done, out[1] launches, out[2] largest batch,
 * out[3] peak device bytes admitted (busy slots' buffers plus the batch being admitted),
 * out[4] peak device bytes held by all slots' buffers, out[5] peak number of slots with work
 * on the device at once.  out holds 6 values.  Thread-safe. */
lnr_status lnr_serve_stats(lnr_ctx* ctx, uint64_t out[6]);

/* ---- measurement ------------------------------------------------------------------- */

/* Measurements of the most recent lnr_render / lnr_render_batch with timing enabled.
 * Device time (ms) of each stage: out[0] cull, out[1] splat, out[2] resolve+pyramid,
 * out[3] upsample and pack, out[4] U-Net, out[5] whole frame.  out[6] the visible points
 * of the batch (the cull's totals, summed over the views); out[7] the number of kernels
 * the frame launched.  With timing on, frames run eagerly (not from a captured graph) and
 * the call waits for the device; enable = 0 turns it off. */
lnr_status lnr_set_timing(lnr_ctx* ctx, int enable);
lnr_status lnr_get_timing(lnr_ctx* ctx, double out[8]);

/* Throughput ceiling of the splat's z-buffer update (Sec. 3 "Point Cloud Projection": the
 * nearest point per pixel, here a 64-bit atomicMin per projected point), measured alone:
 * n_ops atomicMin of splat-shaped keys (depth bits << 32 | index) into a fresh buffer of
 * n_slots keys, coherent = 1 with neighbouring operations on neighbouring keys (as
 * cell-sorted points), 0 with hashed keys.  *ops_per_s: operations per second of the
 * fastest of five timed launches after a warm-up, with the splat's grid.  The probe
 * allocates and frees its own buffer and runs on the context's stream, after waiting for
 * it.  Errors: LNR_E_ARG for n_slots outside [1, 2^32] or n_ops outside [1, 2^34];
 * LNR_E_OOM; LNR_E_CUDA. */
lnr_status lnr_probe_atomic_rate(lnr_ctx* ctx, uint64_t n_slots, uint64_t n_ops, int coherent,
                                 double* ops_per_s);

/* ---- filter without allocation ------------------------------------------------------ */

/* The depth filter stage of lnr_render on its own, for callers that may not allocate
 * device memory -- e.g. a host application's real-time frame loop, where cudaMalloc can
 * synchronise the whole device and stall unrelated work, or a plug-in whose host owns every
 * allocation.  The paper has no counterpart of this entry point: it is a deployment variant
 * of lnr_render's filter stage, with the same arithmetic (kept depth bit-identical to
 * LNR_STAGE_FILTERED).
 * d_depth: device float [H*W], view-space depth, +inf where no point was projected.
 * d_kept:  device float [H*W] output, the kept depth, +inf where empty or filtered out.
 * n_levels, fs: as lnr_render.  cuda_stream: cudaStream_t (NULL = legacy default stream).
 * Runs on the current CUDA device and allocates nothing: the pyramid lives in a fixed
 * 12 MiB device array inside the library (held by every GPU that loads it until exit),
 * enough for images up to about 2560 x 1440 at 6 levels; larger images return LNR_E_ARG.
 * The first call on a device looks up that array's address; make it before any stream
 * capture.  Calls whose work overlaps on the GPU share the array and race; order them.
 * Returns without waiting for the GPU.  Errors: LNR_E_ARG (null pointer, bad size, level
 * count or strength), LNR_E_CUDA (a launch failed). */
lnr_status lnr_filter_static(const float* d_depth, int W, int H, int n_levels, float fs, float* d_kept,
                             void* cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* LNR_H */
