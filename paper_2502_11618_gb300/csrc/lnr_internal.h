// Internal declarations shared by the CUDA translation units of liblnr.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <condition_variable>
#include <deque>
#include <map>
#include <set>
#include <tuple>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "../../include/lnr.h"

namespace lnr {

constexpr int kMaxLevels = 6;      // filter pyramid depth handled by the 64x64 tile kernel
constexpr int kPyrTile = 64;       // resolve + min-pool tile side
constexpr int kMaxUnetLevels = 8;

// Kernels launched by the calling thread: every launch site of the frame path adds one, so
// that a frame's launch count is the difference across its enqueue.
inline thread_local uint64_t tl_launches = 0;
inline void count_launch() { ++tl_launches; }

// Parameters of one view on the device (filled by the host in FP64, then rounded once).
struct ViewDev {
    int32_t anchor[3];
    float d0[3];
    float s[9];      // s[3k + r]: component r of grid step k in camera space
    float Rf[9];     // world->camera rotation, row-major, FP32
    float fx, fy, cx, cy, znear, zfar;
    float S;         // keep scale 1 + fs * KEEP_REL
    float inv_pad;
};

// Tensor-core kernel choice for one convolution: mode 0 = built-in default, 1 = halo
// kernel with (R, P, CK), 2 = generic kernel.
struct TcConfig {
    int mode = 0;
    int R = 0, P = 0, CK = 0;
    int O = 0;  // halo kernel: 1 or 2 = epilogue stores through that many staging buffers and TMA
    int E = 8;  // halo kernel: epilogue warps (4, 8, or 12 for standard tiles)
    int F = 0;  // first conv only: 2 or 4 = fused with the second (k_enc0_fused, F output rows per tile)
};

// One convolution as the GPU runs it.
struct ConvLayer {
    int cin0 = 0;       // channels read from the same-resolution source
    int cin1 = 0;       // channels read from the half-resolution source (nearest 2x up)
    int cin_pad = 0;    // cin0 + cin1 rounded up to the kernel's K granularity
    int cout = 0;
    int level = 0;
    bool pool = false;  // also write the 2x2 max-pooled output (encoder convs below the bottom)
    bool head = false;  // fuse the 1x1 head + sigmoid (last decoder conv)
    float* w32 = nullptr;   // device, FP32 [tap][cin_pad][cout]
    float* b32 = nullptr;   // device, FP32 [cout]
    void* wtc = nullptr;    // device, tensor-core weights [cout][tap][cin_pad] (bf16 or fp8)
    void* wh[3] = {nullptr, nullptr, nullptr};  // device, halo-kernel weights for chunks of <= 16 / 32 / 64 channels
    std::map<std::pair<int, int>, TcConfig> tuned;  // autotuned kernel per layer resolution (W, H)
    std::map<std::pair<int, int>, TcConfig> tuned8; // the same for the FP8 precision
    // FP8 (E4M3): set by calibration.  Operands are E4M3 when fp8 (every conv but the
    // first, whose input is the BF16 RGBDA image); in_scale: activation scale of each K
    // segment's input; out_scale: of this conv's output; wscale8: per output channel.
    bool fp8 = false;
    bool out_bf16 = false;  // FP8 mode: a consumer of this conv's output reads BF16 operands
    bool pool_bf16 = false; // FP8 mode: the consumer of its pooled output reads BF16
    float in_scale[2] = {1.f, 1.f};
    float out_scale = 1.f;
    void* wh8[3] = {nullptr, nullptr, nullptr};
    float* wscale8 = nullptr;
    std::vector<float> wscale8_h;  // host copy of wscale8
    float* wscale = nullptr;  // device, per-output-channel dequant scale (fp8), else null
    std::vector<float> wf;  // host FP32 OIHW after batch-norm folding
    std::vector<float> bf;
};

struct Unet {
    int levels = 0;
    int ch[kMaxUnetLevels] = {0};
    int in_ch = 5, out_ch = 3;
    std::vector<ConvLayer> convs;   // network order
    float* head_w = nullptr;        // device FP32 [out_ch][ch0]
    float* head_b = nullptr;
    std::vector<float> head_wh, head_bh;
    bool fp8_ready = false;         // FP8 weights and activation scales calibrated
};

// Grow-only device buffer.
struct DBuf {
    void* p = nullptr;
    size_t bytes = 0;
    cudaError_t ensure(size_t n) {
        if (n <= bytes) return cudaSuccess;
        if (p) cudaFree(p);
        p = nullptr;
        bytes = 0;
        cudaError_t e = cudaMalloc(&p, n);
        if (e == cudaSuccess) bytes = n;
        return e;
    }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        bytes = 0;
    }
    template <class T> T* as() const { return static_cast<T*>(p); }
};

struct GraphKey {
    int B, W, H, nlev, prec;
    int vk;            // pinned view block the graph uploads from
    const void* out;   // where the graph's U-Net head writes
    bool operator<(const GraphKey& o) const {
        return std::tie(B, W, H, nlev, prec, vk, out) < std::tie(o.B, o.W, o.H, o.nlev, o.prec, o.vk, o.out);
    }
};

// Per-launch workspace: everything one batch of views needs on the device.
struct Workspace {
    int B = 0, W = 0, H = 0, nlev = 0;
    DBuf view;                              // ViewDev[B]
    DBuf cull_flag, cull_cnt, cull_bsum;    // per-cell temporaries
    DBuf vis_info, vis_pref, vis_tot;       // visible cells (camera-space origin, position offset), point prefix, totals
    DBuf chunk_cell;                        // per view: first visible cell of every splat chunk
    DBuf keys;                              // uint64 [B][P]
    bool keys_dirty = true;
    DBuf soft_acc;                          // soft z-buffer sums, uint64 [B][P][2] (soft mode only)
    bool soft_dirty = true;
    DBuf depth, rgba;                       // float / uint32 [B][P]
    DBuf pyr_m, pyr_u;                      // min-pooled and upsampled levels (all levels)
    DBuf u0;                                // float [B][P] kept depth (stage tap)
    DBuf act[4 * kMaxUnetLevels + 2];       // U-Net activations; [4 * kMaxUnetLevels] = U-Net input
    DBuf out;                               // float [B][P][3]
    float* out_ptr = nullptr;               // U-Net output of the next frame: a caller's device buffer, or null for out
    bool allow_fuse = true;                 // false: every conv runs apart (the FP8 calibration frame reads every output)
    // View parameters go up from two pinned host blocks in turn; view_ev[k] is recorded right
    // after block k's upload, so composing the next frame waits only for the upload that
    // last used its block, never for the frame still on the device.
    DBuf pinned_view[2];                    // host pinned ViewDev[B]
    cudaEvent_t view_ev[2] = {nullptr, nullptr};
    int vk = 0;                             // block of the frame being prepared
    uint64_t vcount = 0;
    cudaStream_t stream = nullptr;
    cudaEvent_t ev[16] = {nullptr};
    // CUDA graphs of whole frames, per (B, W, H, nlev, precision); valid while no buffer
    // they captured has been reallocated (alloc_gen) and the cloud / net are unchanged
    std::map<GraphKey, cudaGraphExec_t> graphs;
    std::map<GraphKey, int> graph_uses;     // eager runs of a configuration not captured yet
    uint64_t alloc_gen = 0, graph_gen = 0, graph_cloud = 0, graph_unet = 0;
    void release();
    size_t device_bytes() const;            // device memory held by the buffers above
};

struct Request {
    uint64_t ticket;
    lnr_view view;
    lnr_intrinsics intr;
    int W, H, nlev;
    float fs;
    double t_submit;
    double t_done = 0.0;
    bool done = false;
    std::vector<float> out;
    size_t act_bytes = 0;
};

struct Server;

}  // namespace lnr

struct lnr_ctx {
    int device = 0;
    int num_sms = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    std::string err;
    // cloud
    uint64_t n = 0;
    lnr::DBuf xyz, rgb, scan;
    uint64_t cloud_gen = 0;
    // grid
    bool grid_ok = false;
    double cell = 0.0;
    double g0[3] = {0, 0, 0};
    int32_t dims[3] = {0, 0, 0};
    int64_t ncells = 0;
    lnr::DBuf cell_start, ox, oy, oz, rgbs;
    // U-Net
    bool unet_ok = false;
    lnr::Unet unet;
    lnr_precision prec = LNR_FP32;
    uint64_t unet_gen = 0;
    // splat collision rule: 0 = hard z-buffer, > 0 = soft with this relative depth threshold
    float soft_rel = 0.0f;
    // cloud shard: keys carry sorted position + shard_base (the shard's first point in the
    // whole cloud's order); the resolve colours only this shard's points
    uint32_t shard_base = 0;
    // per-frame workspace of the synchronous calls
    lnr::Workspace ws;
    bool timing = false;
    double times[8] = {0};
    // serving
    lnr::Server* server = nullptr;  // owned; deleted by lnr_serve_stop
    size_t mem_budget = 0;
};

namespace lnr {

double now_s();
lnr_status fail(lnr_ctx* c, lnr_status s, const std::string& msg);
lnr_status cuda_fail(lnr_ctx* c, cudaError_t e, const char* where);

// grid.cu
cudaError_t grid_bbox(const double* xyz, uint64_t n, double* d_tmp, double out_lohi[6], cudaStream_t st);
cudaError_t grid_build(lnr_ctx* c, cudaStream_t st);

// raster.cu
int cull_blocks(int64_t ncells);
void launch_cull(const lnr_ctx* c, Workspace& ws, cudaStream_t st);
void launch_splat(const lnr_ctx* c, Workspace& ws, cudaStream_t st);
void launch_clear_keys(Workspace& ws, cudaStream_t st);
void launch_resolve_pyramid(const lnr_ctx* c, Workspace& ws, cudaStream_t st);
// One view from z-buffer keys (and, when rgba is non-null, resolved colours) computed
// elsewhere: resolve, pyramid, filter, packing and (stage < 0) the U-Net.
void enqueue_from_keys(lnr_ctx* c, Workspace& ws, cudaStream_t st, const uint64_t* keys, const uint32_t* rgba,
                       int stage, lnr_precision prec);
void launch_splat_soft(const lnr_ctx* c, Workspace& ws, cudaStream_t st);
size_t splat_max_chunks(uint64_t npoints);  // entries per view of the splat's chunk -> first cell table
void launch_training_input(const Workspace& ws, const float* gt, float zfar, int unfiltered, float* out,
                           cudaStream_t st);
// Upsample step from level l+1 to level l; at l == 0 also packs the U-Net input.
// unet_in_kind: 0 = FP32 NHWC8, 1 = BF16 NHWC16, 2 = none (stage taps only).
void launch_upsample(const lnr_ctx* c, Workspace& ws, int l, void* unet_in, int unet_in_kind,
                     bool write_u0, cudaStream_t st);
size_t pyramid_floats(int W, int H, int nlev);
size_t pyramid_offset(int W, int H, int l);
void launch_unet_in_extract(const void* unet_in, int kind, float* out5, int64_t npx, cudaStream_t st);
cudaError_t probe_atomic_rate(uint64_t n_slots, uint64_t n_ops, int coherent, int num_sms, cudaStream_t st,
                              double* ops_per_s);

// api.cu
lnr_status check_frame_args(lnr_ctx* c, int nviews, const lnr_view* views, const lnr_intrinsics* in, int W, int H,
                            int nlev, const float* fs, bool need_unet);
lnr_status prepare_views(lnr_ctx* c, Workspace& ws, int B, const lnr_view* views, const lnr_intrinsics* in, int W,
                         int H, int nlev, const float* fs, lnr_precision prec);
void enqueue_frame(lnr_ctx* c, Workspace& ws, cudaStream_t st, int stage, lnr_precision prec, bool timed);
cudaError_t run_frame(lnr_ctx* c, Workspace& ws, lnr_precision prec, bool use_graph);
size_t frame_bytes(const lnr_ctx* c, int B, int W, int H, bool soft);  // raster workspace bytes of a batch

// unet.cu
lnr_status unet_autotune(lnr_ctx* c, Workspace& ws, lnr_precision p, int reps);
lnr_status unet_calibrate_fp8(lnr_ctx* c, Workspace& ws);
cudaError_t unet_ensure(const Unet& u, Workspace& ws, lnr_precision p);
size_t unet_act_bytes(const Unet& u, int B, int W, int H, lnr_precision p);
lnr_status unet_prepare(lnr_ctx* c);
void unet_forward(const lnr_ctx* c, Workspace& ws, lnr_precision p, const void* in, float* out,
                  cudaStream_t st, cudaEvent_t* layer_ev);
int unet_in_kind(lnr_precision p);
size_t unet_in_bytes_per_px(lnr_precision p);  // network-input buffer bytes per pixel (32 in both layouts)

// conv_tc.cu
bool tc_available();
cudaError_t tc_prepare_layer(ConvLayer& L, lnr_precision p);
void tc_conv(const ConvLayer& L, lnr_precision p, const void* src0, const void* src1, void* out, void* pool_out,
             const float* head_w, const float* head_b, const float* head_wh, const float* head_bh, float* head_out, int B,
             int W, int H, int head_o, cudaStream_t st, const TcConfig* force = nullptr);
std::vector<TcConfig> tc_candidates(const ConvLayer& L, lnr_precision p);
// The first two encoder convs fused (R rows per tile, 2 or 4); false when they cannot be.
bool tc_fused_enc0(const ConvLayer& L0, const ConvLayer& L1, lnr_precision p, const void* in, void* out,
                   void* pool_out, int B, int W, int H, int R, cudaStream_t st);
cudaError_t tc_prepare_fp8(ConvLayer& L);
int tc_error_word();  // nonzero after a bounded wait in a tensor-core kernel ran out (then reset)

}  // namespace lnr
