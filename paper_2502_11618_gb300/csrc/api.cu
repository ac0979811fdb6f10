// C ABI of the render path (include/lnr.h): context, cloud upload, grid build, U-Net
// loading, the FP64 host composition of each view, and the per-frame launch sequence.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>

#include "lnr_internal.h"

namespace lnr {

constexpr float kKeepRel = 0.05f;  // keep tolerance per unit of filter_strength
constexpr double kBnEps = 1e-5;

double now_s() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

lnr_status fail(lnr_ctx* c, lnr_status s, const std::string& msg) {
    if (c) c->err = msg;
    return s;
}

lnr_status cuda_fail(lnr_ctx* c, cudaError_t e, const char* where) {
    return fail(c, e == cudaErrorMemoryAllocation ? LNR_E_OOM : LNR_E_CUDA,
                std::string(where) + ": " + cudaGetErrorString(e));
}

void Workspace::release() {
    DBuf* all[] = {&view, &cull_flag, &cull_cnt, &cull_bsum, &vis_info, &vis_pref, &vis_tot, &chunk_cell, &keys,
                   &soft_acc, &depth, &rgba, &pyr_m, &pyr_u, &u0, &out};
    for (DBuf* b : all) b->release();
    for (auto& a : act) a.release();
    for (auto& pv : pinned_view) {
        if (pv.p) cudaFreeHost(pv.p);
        pv.p = nullptr;
        pv.bytes = 0;
    }
    for (auto& e : ev)
        if (e) { cudaEventDestroy(e); e = nullptr; }
    for (auto& e : view_ev)
        if (e) { cudaEventDestroy(e); e = nullptr; }
    for (auto& kv : graphs) cudaGraphExecDestroy(kv.second);
    graphs.clear();
    graph_uses.clear();
}

size_t Workspace::device_bytes() const {
    const DBuf* all[] = {&view, &cull_flag, &cull_cnt, &cull_bsum, &vis_info, &vis_pref, &vis_tot, &chunk_cell,
                         &keys, &soft_acc, &depth, &rgba, &pyr_m, &pyr_u, &u0, &out};
    size_t n = 0;
    for (const DBuf* b : all) n += b->bytes;
    for (const auto& a : act) n += a.bytes;
    return n;
}

// FP64 composition of the view with the grid (once per view, on the host): the anchor
// cell holds the camera; d0 = R (origin(anchor) - C) and the grid steps R (cell e_k) are
// formed in FP64 and rounded once, so georeferenced coordinates keep their precision.
static void compose_view(const lnr_ctx* c, const lnr_view& v, const lnr_intrinsics& in, float fs, ViewDev& o) {
    double rel[3];
    for (int a = 0; a < 3; ++a) {
        double f = std::floor((v.C[a] - c->g0[a]) / c->cell);
        if (f < 0.0) f = 0.0;
        if (f > (double)(c->dims[a] - 1)) f = (double)(c->dims[a] - 1);
        o.anchor[a] = (int32_t)f;
        rel[a] = (c->g0[a] + (double)o.anchor[a] * c->cell) - v.C[a];
    }
    for (int r = 0; r < 3; ++r) {
        double acc = v.R[3 * r] * rel[0];
        acc = acc + v.R[3 * r + 1] * rel[1];
        acc = acc + v.R[3 * r + 2] * rel[2];
        o.d0[r] = (float)acc;
        for (int k = 0; k < 3; ++k) o.s[3 * k + r] = (float)(v.R[3 * r + k] * c->cell);
    }
    for (int e = 0; e < 9; ++e) o.Rf[e] = (float)v.R[e];
    o.fx = in.fx; o.fy = in.fy; o.cx = in.cx; o.cy = in.cy; o.znear = in.znear; o.zfar = in.zfar;
    const float prod = fs * kKeepRel;
    o.S = 1.0f + prod;
    o.inv_pad = 0.f;
}

static bool finite_view(const lnr_view& v) {
    for (double x : v.R) if (!std::isfinite(x)) return false;
    for (double x : v.C) if (!std::isfinite(x)) return false;
    return true;
}

lnr_status check_frame_args(lnr_ctx* c, int nviews, const lnr_view* views, const lnr_intrinsics* in,
                                   int W, int H, int nlev, const float* fs, bool need_unet) {
    if (!c->grid_ok) return fail(c, LNR_E_STATE, "render before build_grid");
    if (need_unet && !c->unet_ok) return fail(c, LNR_E_STATE, "render before set_unet");
    if (nviews < 1 || !views || !in || !fs) return fail(c, LNR_E_ARG, "null view, intrinsics or strength");
    if (W < 1 || H < 1 || (int64_t)W * H > (1ll << 31)) return fail(c, LNR_E_ARG, "bad image size");
    if (need_unet) {
        const int m = 1 << (c->unet.levels - 1);
        if (W % m || H % m) return fail(c, LNR_E_ARG, "W and H must be multiples of 2^(levels-1)");
    }
    int maxl = 0;
    while ((2 << maxl) <= std::min(W, H)) ++maxl;
    if (nlev < 0 || nlev > std::min(maxl, kMaxLevels))
        return fail(c, LNR_E_ARG, "n_levels outside [0, min(6, floor(log2(min(W, H))))]");
    for (int i = 0; i < nviews; ++i) {
        if (!(fs[i] >= 0.0f)) return fail(c, LNR_E_ARG, "filter_strength must be >= 0 and not NaN");
        if (!finite_view(views[i])) return fail(c, LNR_E_ARG, "view is not finite");
        const lnr_intrinsics& k = in[i];
        if (!(std::isfinite(k.fx) && std::isfinite(k.fy) && std::isfinite(k.cx) && std::isfinite(k.cy) &&
              k.znear > 0.0f && k.zfar > k.znear && std::isfinite(k.zfar)))
            return fail(c, LNR_E_ARG, "bad intrinsics");
    }
    return LNR_OK;
}

// Size every per-frame buffer for B views of W x H with nlev pyramid levels.
static cudaError_t ensure_ws(const lnr_ctx* c, Workspace& ws, int B, int W, int H, int nlev) {
    cudaError_t e;
    const void* before[] = {ws.view.p, ws.cull_flag.p, ws.cull_cnt.p, ws.cull_bsum.p, ws.vis_info.p, ws.vis_pref.p,
                            ws.vis_tot.p, ws.depth.p, ws.rgba.p, ws.pyr_m.p, ws.pyr_u.p, ws.u0.p, ws.out.p, ws.keys.p,
                            ws.soft_acc.p, ws.chunk_cell.p};
    const size_t P = (size_t)W * H;
    const int nb = cull_blocks(c->ncells);
    const size_t pf = pyramid_floats(W, H, kMaxLevels);
    if ((e = ws.view.ensure(sizeof(ViewDev) * B)) || (e = ws.cull_flag.ensure(4 * c->ncells * B)) ||
        (e = ws.cull_cnt.ensure(4 * c->ncells * B)) || (e = ws.cull_bsum.ensure(8 * (size_t)nb * B)) ||
        (e = ws.vis_info.ensure(16 * c->ncells * B)) || (e = ws.vis_pref.ensure(4 * c->ncells * B)) ||
        (e = ws.vis_tot.ensure(8 * B)) || (e = ws.chunk_cell.ensure(4 * splat_max_chunks(c->n) * B)) ||
        (e = ws.depth.ensure(4 * P * B)) || (e = ws.rgba.ensure(4 * P * B)) ||
        (e = ws.pyr_m.ensure(4 * pf * B)) || (e = ws.pyr_u.ensure(4 * pf * B)) || (e = ws.u0.ensure(4 * P * B)) ||
        (e = ws.out.ensure(12 * P * B)))
        return e;
    const bool new_keys = ws.keys.bytes < 8 * P * B;
    if ((e = ws.keys.ensure(8 * P * B))) return e;
    if (new_keys) ws.keys_dirty = true;
    if (c->soft_rel > 0.0f) {
        const bool new_acc = ws.soft_acc.bytes < 16 * P * B;
        if ((e = ws.soft_acc.ensure(16 * P * B))) return e;
        if (new_acc) ws.soft_dirty = true;
    }
    for (auto& pv : ws.pinned_view)
        if (pv.bytes < sizeof(ViewDev) * B) {
            if (pv.p) cudaFreeHost(pv.p);
            pv.p = nullptr;
            pv.bytes = 0;
            if ((e = cudaMallocHost(&pv.p, sizeof(ViewDev) * B))) return e;
            pv.bytes = sizeof(ViewDev) * B;
            ws.alloc_gen++;  // captured graphs upload from the old block
        }
    if (!ws.ev[0])
        for (auto& ev : ws.ev)
            if ((e = cudaEventCreate(&ev))) return e;
    if (!ws.view_ev[0])
        for (auto& ev : ws.view_ev)
            if ((e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming))) return e;
    const void* after[] = {ws.view.p, ws.cull_flag.p, ws.cull_cnt.p, ws.cull_bsum.p, ws.vis_info.p, ws.vis_pref.p,
                           ws.vis_tot.p, ws.depth.p, ws.rgba.p, ws.pyr_m.p, ws.pyr_u.p, ws.u0.p, ws.out.p, ws.keys.p,
                           ws.soft_acc.p, ws.chunk_cell.p};
    for (size_t i = 0; i < sizeof(before) / sizeof(before[0]); ++i)
        if (before[i] != after[i]) ws.alloc_gen++;
    ws.B = B;
    ws.W = W;
    ws.H = H;
    ws.nlev = nlev;
    return cudaSuccess;
}

// The upload of the frame's view block is done once view_ev[vk] completes.  Under stream
// capture the record becomes a node of its own (an external event record), so that every
// replay of the graph records it; outside capture it is a plain record.
static void record_view_uploaded(Workspace& ws, cudaStream_t st) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaStreamIsCapturing(st, &cs);
    if (cs == cudaStreamCaptureStatusActive) cudaEventRecordWithFlags(ws.view_ev[ws.vk], st, cudaEventRecordExternal);
    else cudaEventRecord(ws.view_ev[ws.vk], st);
}

// Enqueue one batch on `st`: params upload, cull, splat, resolve + pyramid, upsampling,
// U-Net.  stage < 0 runs the whole frame into ws.out; otherwise stops after that stage.
void enqueue_frame(lnr_ctx* c, Workspace& ws, cudaStream_t st, int stage, lnr_precision prec,
                          bool timed) {
    cudaEvent_t* ev = ws.ev;
    auto mark = [&](int i) {
        if (timed) cudaEventRecord(ev[i], st);
    };
    mark(0);
    cudaMemcpyAsync(ws.view.p, ws.pinned_view[ws.vk].p, sizeof(ViewDev) * ws.B, cudaMemcpyHostToDevice, st);
    record_view_uploaded(ws, st);
    if (ws.keys_dirty) launch_clear_keys(ws, st);
    launch_cull(c, ws, st);
    mark(1);
    if (stage == LNR_STAGE_CULL) return;
    launch_splat(c, ws, st);
    mark(2);
    if (stage == LNR_STAGE_KEYS) {
        ws.keys_dirty = true;  // the resolve that would clear the keys does not run
        return;
    }
    if (c->soft_rel > 0.0f) launch_splat_soft(c, ws, st);
    launch_resolve_pyramid(c, ws, st);
    mark(3);
    if (stage == LNR_STAGE_RGBDA_RAW) return;
    const int kind = (stage >= 0) ? 0 : unet_in_kind(prec);
    void* unet_in = ws.act[4 * kMaxUnetLevels].p;
    for (int l = ws.nlev - 1; l >= 1; --l) launch_upsample(c, ws, l, nullptr, 2, false, st);
    launch_upsample(c, ws, 0, unet_in, kind, stage == LNR_STAGE_FILTERED, st);
    mark(4);
    if (stage >= 0) return;
    unet_forward(c, ws, prec, unet_in, ws.out_ptr ? ws.out_ptr : ws.out.as<float>(), st, nullptr);
    mark(5);
}

void enqueue_from_keys(lnr_ctx* c, Workspace& ws, cudaStream_t st, const uint64_t* keys, const uint32_t* rgba,
                       int stage, lnr_precision prec) {
    const size_t P = (size_t)ws.W * ws.H;
    cudaMemcpyAsync(ws.view.p, ws.pinned_view[ws.vk].p, sizeof(ViewDev) * ws.B, cudaMemcpyHostToDevice, st);
    record_view_uploaded(ws, st);
    cudaMemcpyAsync(ws.keys.p, keys, 8 * P, cudaMemcpyDeviceToDevice, st);
    launch_resolve_pyramid(c, ws, st);  // depth, pyramid, this context's colours; clears the keys
    if (rgba) cudaMemcpyAsync(ws.rgba.p, rgba, 4 * P, cudaMemcpyDeviceToDevice, st);
    if (stage == LNR_STAGE_RGBDA_RAW) return;
    const int kind = (stage >= 0) ? 0 : unet_in_kind(prec);
    void* unet_in = ws.act[4 * kMaxUnetLevels].p;
    for (int l = ws.nlev - 1; l >= 1; --l) launch_upsample(c, ws, l, nullptr, 2, false, st);
    launch_upsample(c, ws, 0, unet_in, kind, stage == LNR_STAGE_FILTERED, st);
    if (stage >= 0) return;
    unet_forward(c, ws, prec, unet_in, ws.out.as<float>(), st, nullptr);
}

lnr_status prepare_views(lnr_ctx* c, Workspace& ws, int B, const lnr_view* views, const lnr_intrinsics* in,
                                int W, int H, int nlev, const float* fs, lnr_precision prec) {
    cudaError_t e = ensure_ws(c, ws, B, W, H, nlev);
    if (e != cudaSuccess) return cuda_fail(c, e, "workspace");
    const void* in_before = ws.act[4 * kMaxUnetLevels].p;
    e = ws.act[4 * kMaxUnetLevels].ensure((size_t)B * W * H * unet_in_bytes_per_px(prec) + 256);
    if (e != cudaSuccess) return cuda_fail(c, e, "U-Net input");
    if (in_before != ws.act[4 * kMaxUnetLevels].p) ws.alloc_gen++;
    if (c->unet_ok) {
        e = unet_ensure(c->unet, ws, prec);
        if (e != cudaSuccess) return cuda_fail(c, e, "U-Net activations");
    }
    ws.out_ptr = nullptr;
    // the block this frame's parameters go into: wait for the upload that used it last
    ws.vk = (int)(ws.vcount++ & 1);
    e = cudaEventSynchronize(ws.view_ev[ws.vk]);
    if (e != cudaSuccess) return cuda_fail(c, e, "stream");
    ViewDev* hv = ws.pinned_view[ws.vk].as<ViewDev>();
    for (int i = 0; i < B; ++i) compose_view(c, views[i], in[i], fs[i], hv[i]);
    return LNR_OK;
}

size_t frame_bytes(const lnr_ctx* c, int B, int W, int H, bool soft) {
    const size_t P = (size_t)B * W * H;
    // keys 8, depth 4, rgba 4, kept depth 4, output 12, U-Net input 32 bytes per pixel, pyramid;
    // soft z-buffer sums 16; per view the cull and compaction tables (28 bytes per cell, block
    // sums, the splat's chunk table) and the view parameters
    const size_t per_view = 28 * (size_t)c->ncells + 8 * (size_t)cull_blocks(c->ncells) +
                            4 * splat_max_chunks(c->n) + sizeof(ViewDev) + 8;
    return P * (soft ? 80 : 64) + 8 * (size_t)B * pyramid_floats(W, H, kMaxLevels) + (size_t)B * per_view + 16 * 256;
}

// Enqueue a whole frame batch on ws.stream: replayed from a CUDA graph captured for this
// (batch, size, levels, precision) once the configuration has run eagerly twice; graphs are
// dropped whenever a buffer they captured was reallocated or the cloud / net changed.
constexpr size_t kMaxGraphs = 256;

cudaError_t run_frame(lnr_ctx* c, Workspace& ws, lnr_precision prec, bool use_graph) {
    if (!use_graph) {
        enqueue_frame(c, ws, ws.stream, -1, prec, false);
        return cudaGetLastError();
    }
    const GraphKey key{ws.B, ws.W, ws.H, ws.nlev, (int)prec, ws.vk, ws.out_ptr};
    // at most kMaxGraphs configurations are kept (a served mix of 3 resolutions x 3 depths x
    // 8 batch sizes x 2 view blocks has 144); past that, start over
    if (ws.graph_gen != ws.alloc_gen || ws.graph_cloud != c->cloud_gen || ws.graph_unet != c->unet_gen ||
        ws.graphs.size() >= kMaxGraphs) {
        for (auto& kv : ws.graphs) cudaGraphExecDestroy(kv.second);
        ws.graphs.clear();
        ws.graph_uses.clear();
        ws.graph_gen = ws.alloc_gen;
        ws.graph_cloud = c->cloud_gen;
        ws.graph_unet = c->unet_gen;
    }
    auto it = ws.graphs.find(key);
    if (it == ws.graphs.end()) {
        // The first two runs of a configuration are eager: capturing costs more than an eager
        // run, so a configuration is captured only once it recurs (a served stream of mixed
        // resolutions, depths and batch sizes meets many configurations only once or twice).
        int& uses = ws.graph_uses[key];
        if (uses < 2 || ws.keys_dirty) {
            ++uses;
            enqueue_frame(c, ws, ws.stream, -1, prec, false);
            return cudaGetLastError();
        }
        cudaGraph_t g = nullptr;
        cudaGraphExec_t ex = nullptr;
        cudaError_t e = cudaStreamBeginCapture(ws.stream, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            enqueue_frame(c, ws, ws.stream, -1, prec, false);
            e = cudaStreamEndCapture(ws.stream, &g);
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&ex, g, 0);
        if (g) cudaGraphDestroy(g);
        if (e != cudaSuccess) {  // capture not possible on this stream: stay eager
            cudaGetLastError();
            enqueue_frame(c, ws, ws.stream, -1, prec, false);
            return cudaGetLastError();
        }
        it = ws.graphs.emplace(key, ex).first;
    }
    return cudaGraphLaunch(it->second, ws.stream);
}

static void read_timing(lnr_ctx* c, Workspace& ws) {
    float ms;
    for (int i = 0; i < 5; ++i) {
        cudaEventElapsedTime(&ms, ws.ev[i], ws.ev[i + 1]);
        c->times[i] = ms;
    }
    cudaEventElapsedTime(&ms, ws.ev[0], ws.ev[5]);
    c->times[5] = ms;
    // visible points of the batch: the cull's per-view totals {cells, points}
    std::vector<uint32_t> tot(2 * (size_t)ws.B);
    double nvis = 0.0;
    if (cudaMemcpy(tot.data(), ws.vis_tot.p, 8 * (size_t)ws.B, cudaMemcpyDeviceToHost) == cudaSuccess)
        for (int v = 0; v < ws.B; ++v) nvis += tot[2 * v + 1];
    c->times[6] = nvis;
}

static lnr_status finish_output(lnr_ctx* c, Workspace& ws, float* out, size_t nfloat, int on_device) {
    cudaError_t e = cudaSuccess;
    if (out != ws.out_ptr)  // else the U-Net wrote the caller's device buffer directly
        e = cudaMemcpyAsync(out, ws.out.p, nfloat * 4, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                            ws.stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "output copy");
    if (!on_device || c->timing) {
        e = cudaStreamSynchronize(ws.stream);
        if (e != cudaSuccess) return cuda_fail(c, e, "render");
    }
    if (c->timing) read_timing(c, ws);
    if ((!on_device || c->timing) && c->prec != LNR_FP32) {
        const int w = tc_error_word();
        if (w >= 5 && w <= 7) return fail(c, LNR_E_TIMEOUT, "a tensor-core kernel gave up waiting (bounded wait ran out)");
        if (w) return fail(c, LNR_E_CUDA, "a tensor-core convolution could not be launched (code " + std::to_string(w) + ")");
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(c, e, "render launch");
    return LNR_OK;
}

}  // namespace lnr

using namespace lnr;

extern "C" {

lnr_status lnr_create(lnr_ctx** out, int device, void* cuda_stream) {
    if (!out) return LNR_E_ARG;
    *out = nullptr;
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) return LNR_E_ARG;
    if (cudaSetDevice(device) != cudaSuccess) return LNR_E_CUDA;
    lnr_ctx* c = new lnr_ctx();
    c->device = device;
    cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device);
    if (cuda_stream) {
        c->stream = (cudaStream_t)cuda_stream;
    } else {
        if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) {
            delete c;
            return LNR_E_CUDA;
        }
        c->own_stream = true;
    }
    c->ws.stream = c->stream;
    *out = c;
    return LNR_OK;
}

lnr_status lnr_destroy(lnr_ctx* c) {
    if (!c) return LNR_E_ARG;
    cudaSetDevice(c->device);
    lnr_serve_stop(c);
    cudaStreamSynchronize(c->stream);
    c->ws.release();
    DBuf* all[] = {&c->xyz, &c->rgb, &c->scan, &c->cell_start, &c->ox, &c->oy, &c->oz, &c->rgbs};
    for (DBuf* b : all) b->release();
    for (auto& L : c->unet.convs) {
        if (L.w32) cudaFree(L.w32);
        if (L.b32) cudaFree(L.b32);
        if (L.wtc) cudaFree(L.wtc);
        for (void* w : L.wh)
            if (w) cudaFree(w);
        for (void* w : L.wh8)
            if (w) cudaFree(w);
        if (L.wscale8) cudaFree(L.wscale8);
        if (L.wscale) cudaFree(L.wscale);
    }
    if (c->unet.head_w) cudaFree(c->unet.head_w);
    if (c->unet.head_b) cudaFree(c->unet.head_b);
    if (c->own_stream) cudaStreamDestroy(c->stream);
    delete c;
    return LNR_OK;
}

const char* lnr_last_error(lnr_ctx* c) { return c ? c->err.c_str() : "null context"; }

lnr_status lnr_load_cloud(lnr_ctx* c, const double* xyz, const uint8_t* rgb, const uint8_t* scan_id, uint64_t n) {
    if (!c) return LNR_E_ARG;
    if (!xyz || !rgb) return fail(c, LNR_E_ARG, "null xyz or rgb");
    if (n < 1 || n > 0xffffffffull) return fail(c, LNR_E_ARG, "point count outside [1, 2^32-1]");
    cudaSetDevice(c->device);
    for (uint64_t i = 0; i < 3 * n; ++i)
        if (!std::isfinite(xyz[i])) return fail(c, LNR_E_ARG, "non-finite coordinate");
    cudaError_t e;
    c->grid_ok = false;
    if ((e = c->xyz.ensure(24 * n)) || (e = c->rgb.ensure(3 * n)) || (scan_id && (e = c->scan.ensure(n))))
        return cuda_fail(c, e, "cloud upload");
    if (!scan_id) c->scan.release();
    if ((e = cudaMemcpy(c->xyz.p, xyz, 24 * n, cudaMemcpyHostToDevice)) ||
        (e = cudaMemcpy(c->rgb.p, rgb, 3 * n, cudaMemcpyHostToDevice)) ||
        (scan_id && (e = cudaMemcpy(c->scan.p, scan_id, n, cudaMemcpyHostToDevice))))
        return cuda_fail(c, e, "cloud upload");
    c->n = n;
    c->cloud_gen++;
    return LNR_OK;
}

// Grid build in a given frame (origin g0, dims cells of size cell): points outside it are
// clamped into its border cells.
static lnr_status build_grid_in(lnr_ctx* c, double cell, const double g0[3], const int32_t dims[3]) {
    double total = 1.0;
    for (int a = 0; a < 3; ++a) {
        if (dims[a] < 1 || !std::isfinite(g0[a])) return fail(c, LNR_E_ARG, "bad grid frame");
        total *= (double)dims[a];
    }
    if (total > 2147483647.0) return fail(c, LNR_E_ARG, "too many cells (> 2^31)");
    std::memcpy(c->g0, g0, sizeof(c->g0));
    std::memcpy(c->dims, dims, sizeof(c->dims));
    c->cell = cell;
    c->ncells = (int64_t)total;
    cudaError_t e = grid_build(c, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "grid build");
    c->grid_ok = true;
    c->cloud_gen++;
    c->ws.keys_dirty = true;
    return LNR_OK;
}

lnr_status lnr_build_grid_frame(lnr_ctx* c, double cell, const double* g0, const int32_t* dims) {
    if (!c || !g0 || !dims) return LNR_E_ARG;
    if (!c->n) return fail(c, LNR_E_STATE, "build_grid before load_cloud");
    if (!(cell > 0.0) || !std::isfinite(cell)) return fail(c, LNR_E_ARG, "cell size must be > 0");
    cudaSetDevice(c->device);
    return build_grid_in(c, cell, g0, dims);
}

lnr_status lnr_build_grid(lnr_ctx* c, double cell) {
    if (!c) return LNR_E_ARG;
    if (!c->n) return fail(c, LNR_E_STATE, "build_grid before load_cloud");
    if (!(cell > 0.0) || !std::isfinite(cell)) return fail(c, LNR_E_ARG, "cell size must be > 0");
    cudaSetDevice(c->device);
    DBuf tmp;
    cudaError_t e = tmp.ensure(1024 * 6 * sizeof(double));
    if (e != cudaSuccess) return cuda_fail(c, e, "grid");
    double lohi[6];
    e = grid_bbox(c->xyz.as<double>(), c->n, tmp.as<double>(), lohi, c->stream);
    tmp.release();
    if (e != cudaSuccess) return cuda_fail(c, e, "grid bounds");
    double g0[3];
    int32_t dims[3];
    for (int a = 0; a < 3; ++a) {
        g0[a] = std::floor(lohi[a] / cell) * cell;
        const double d = std::floor((lohi[3 + a] - g0[a]) / cell) + 1.0;
        if (d > 2147483647.0) return fail(c, LNR_E_ARG, "too many cells");
        dims[a] = (int32_t)d;
    }
    return build_grid_in(c, cell, g0, dims);
}

lnr_status lnr_set_shard(lnr_ctx* c, uint32_t pos_base) {
    if (!c) return LNR_E_ARG;
    if (c->server) return fail(c, LNR_E_STATE, "cannot change the shard while serving");
    if ((uint64_t)pos_base + c->n > 0xffffffffull) return fail(c, LNR_E_ARG, "shard positions exceed 32 bits");
    if (pos_base != c->shard_base) {
        c->shard_base = pos_base;
        c->cloud_gen++;  // captured frame graphs hold the old base
    }
    return LNR_OK;
}

// One cloud shard's resolve against the whole cloud's z-buffer keys (device, H*W): the
// colours (r | g << 8 | b << 16 | 1 << 24) of the pixels whose front point is this shard's,
// zero elsewhere, into rgba (device, H*W).
lnr_status lnr_shard_resolve(lnr_ctx* c, const lnr_view* view, const lnr_intrinsics* in, int W, int H,
                             const uint64_t* keys, uint32_t* rgba) {
    if (!c) return LNR_E_ARG;
    const float fs = 0.0f;
    lnr_status s = check_frame_args(c, 1, view, in, W, H, 0, &fs, false);
    if (s != LNR_OK) return s;
    if (!keys || !rgba) return fail(c, LNR_E_ARG, "null keys or colours");
    if (c->soft_rel > 0.0f) return fail(c, LNR_E_STATE, "cloud shards use the hard z-buffer");
    cudaSetDevice(c->device);
    Workspace& ws = c->ws;
    s = prepare_views(c, ws, 1, view, in, W, H, 0, &fs, c->prec);
    if (s != LNR_OK) return s;
    enqueue_from_keys(c, ws, ws.stream, keys, nullptr, LNR_STAGE_RGBDA_RAW, c->prec);
    cudaError_t e = cudaMemcpyAsync(rgba, ws.rgba.p, 4 * (size_t)W * H, cudaMemcpyDeviceToDevice, ws.stream);
    if (!e) e = cudaStreamSynchronize(ws.stream);
    if (!e) e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(c, e, "shard_resolve");
    return LNR_OK;
}

// The rest of the frame from the whole cloud's keys and colours (both device, H*W): filter
// with n_levels / fs, U-Net, out_rgb as lnr_render.
lnr_status lnr_shard_finish(lnr_ctx* c, const lnr_view* view, const lnr_intrinsics* in, int W, int H, int nlev,
                            float fs, const uint64_t* keys, const uint32_t* rgba, float* out, int on_device) {
    if (!c) return LNR_E_ARG;
    lnr_status s = check_frame_args(c, 1, view, in, W, H, nlev, &fs, true);
    if (s != LNR_OK) return s;
    if (!keys || !rgba || !out) return fail(c, LNR_E_ARG, "null keys, colours or output");
    cudaSetDevice(c->device);
    Workspace& ws = c->ws;
    s = prepare_views(c, ws, 1, view, in, W, H, nlev, &fs, c->prec);
    if (s != LNR_OK) return s;
    enqueue_from_keys(c, ws, ws.stream, keys, rgba, -1, c->prec);
    const size_t bytes = 12 * (size_t)W * H;
    cudaError_t e = cudaMemcpyAsync(out, ws.out.p, bytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                                    ws.stream);
    if (!e) e = cudaStreamSynchronize(ws.stream);
    if (!e) e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(c, e, "shard_finish");
    if (c->prec != LNR_FP32) {
        const int w = tc_error_word();
        if (w >= 5 && w <= 7) return fail(c, LNR_E_TIMEOUT, "a tensor-core kernel gave up waiting (bounded wait ran out)");
        if (w) return fail(c, LNR_E_CUDA, "a tensor-core convolution could not be launched (code " + std::to_string(w) + ")");
    }
    return LNR_OK;
}

lnr_status lnr_grid_info(lnr_ctx* c, double* g0, int32_t* dims) {
    if (!c) return LNR_E_ARG;
    if (!c->grid_ok) return fail(c, LNR_E_STATE, "no grid");
    if (g0) std::memcpy(g0, c->g0, sizeof(c->g0));
    if (dims) std::memcpy(dims, c->dims, sizeof(c->dims));
    return LNR_OK;
}

lnr_status lnr_set_unet(lnr_ctx* c, const lnr_unet_desc* d, const float* w, size_t n_floats, lnr_precision prec) {
    if (!c) return LNR_E_ARG;
    if (!d || !w) return fail(c, LNR_E_ARG, "null descriptor or weights");
    if (d->levels < 1 || d->levels > kMaxUnetLevels) return fail(c, LNR_E_ARG, "levels outside [1, 8]");
    if (d->in_ch != 5 || d->out_ch < 1 || d->out_ch > 4) return fail(c, LNR_E_ARG, "in_ch must be 5, out_ch in [1, 4]");
    if (prec < LNR_FP32 || prec > LNR_FP8) return fail(c, LNR_E_ARG, "bad precision");
    for (int l = 0; l < d->levels; ++l)
        if (d->ch[l] < 16 || d->ch[l] > 256 || d->ch[l] % 16) return fail(c, LNR_E_ARG, "channels must be multiples of 16 in [16, 256]");
    const int L = d->levels;
    // count and locate
    size_t need = 0;
    int cin = d->in_ch;
    std::vector<std::pair<int, int>> shp;  // (cout, cin)
    for (int l = 0; l < L; ++l) {
        shp.push_back({d->ch[l], cin});
        shp.push_back({d->ch[l], d->ch[l]});
        cin = d->ch[l];
    }
    for (int l = L - 2; l >= 0; --l) {
        shp.push_back({d->ch[l], d->ch[l] + d->ch[l + 1]});
        shp.push_back({d->ch[l], d->ch[l]});
    }
    for (auto& s : shp) need += (size_t)s.first * s.second * 9 + s.first;
    need += (size_t)d->out_ch * d->ch[0] + d->out_ch;
    if (d->has_bn)
        for (int l = 0; l < L; ++l) need += 8 * (size_t)d->ch[l];
    if (n_floats != need) return fail(c, LNR_E_ARG, "weight count does not match the descriptor");
    for (size_t i = 0; i < n_floats; ++i)
        if (!std::isfinite(w[i])) return fail(c, LNR_E_ARG, "non-finite weight");
    cudaSetDevice(c->device);
    cudaStreamSynchronize(c->stream);
    for (auto& Lr : c->unet.convs) {
        if (Lr.w32) cudaFree(Lr.w32);
        if (Lr.b32) cudaFree(Lr.b32);
        if (Lr.wtc) cudaFree(Lr.wtc);
        for (void* w : Lr.wh)
            if (w) cudaFree(w);
        for (void* w : Lr.wh8)
            if (w) cudaFree(w);
        if (Lr.wscale8) cudaFree(Lr.wscale8);
        if (Lr.wscale) cudaFree(Lr.wscale);
    }
    Unet u;
    u.levels = L;
    for (int l = 0; l < L; ++l) u.ch[l] = d->ch[l];
    u.in_ch = d->in_ch;
    u.out_ch = d->out_ch;
    u.head_w = c->unet.head_w;
    u.head_b = c->unet.head_b;
    const float* p = w;
    for (size_t i = 0; i < shp.size(); ++i) {
        ConvLayer Lr;
        const int co = shp[i].first, ci = shp[i].second;
        Lr.cout = co;
        const bool enc = i < (size_t)2 * L;
        Lr.level = enc ? (int)(i / 2) : (int)(L - 2 - (i - 2 * L) / 2);
        const bool dec_a = !enc && ((i - 2 * L) % 2 == 0);
        Lr.cin0 = dec_a ? d->ch[Lr.level] : ci;
        Lr.cin1 = dec_a ? d->ch[Lr.level + 1] : 0;
        Lr.pool = enc && (i % 2 == 1) && Lr.level < L - 1;
        Lr.head = (i + 1 == shp.size()) && L > 1;
        Lr.wf.assign(p, p + (size_t)co * ci * 9);
        p += (size_t)co * ci * 9;
        Lr.bf.assign(p, p + co);
        p += co;
        u.convs.push_back(std::move(Lr));
    }
    u.head_wh.assign(p, p + (size_t)d->out_ch * d->ch[0]);
    p += (size_t)d->out_ch * d->ch[0];
    u.head_bh.assign(p, p + d->out_ch);
    p += d->out_ch;
    if (d->has_bn) {
        // fold y = gamma (conv - mean) / sqrt(var + eps) + beta into the encoder convs (FP64)
        for (int e = 0; e < 2 * L; ++e) {
            ConvLayer& Lr = u.convs[e];
            const int co = Lr.cout;
            const float *g = p, *be = p + co, *mu = p + 2 * co, *var = p + 3 * co;
            const size_t per = Lr.wf.size() / co;
            for (int o = 0; o < co; ++o) {
                const double sc = (double)g[o] / std::sqrt((double)var[o] + kBnEps);
                for (size_t k = 0; k < per; ++k) Lr.wf[o * per + k] = (float)((double)Lr.wf[o * per + k] * sc);
                Lr.bf[o] = (float)(((double)Lr.bf[o] - (double)mu[o]) * sc + (double)be[o]);
            }
            p += 4 * co;
        }
    }
    c->unet = std::move(u);
    c->unet_ok = false;
    lnr_status s = unet_prepare(c);
    if (s != LNR_OK) return s;
    c->unet_ok = true;
    c->prec = prec;
    c->unet_gen++;
    if ((prec != LNR_FP32 && !tc_available()) || (prec != LNR_FP32 && L < 2)) {
        c->prec = LNR_FP32;
        return fail(c, LNR_E_ARG, "precision not available for this net");
    }
    if (prec == LNR_FP8) {  // E4M3 needs calibrated activation scales first
        c->prec = LNR_BF16;
        return fail(c, LNR_E_STATE, "FP8 needs lnr_calibrate after set_unet (BF16 selected meanwhile)");
    }
    return LNR_OK;
}

lnr_status lnr_set_soft_zbuffer(lnr_ctx* c, float rel) {
    if (!c) return LNR_E_ARG;
    if (!(rel >= 0.0f && rel <= 1e6f)) return fail(c, LNR_E_ARG, "soft z-buffer threshold must be in [0, 1e6]");
    if (c->server) return fail(c, LNR_E_STATE, "cannot change the z-buffer rule while serving");
    if (rel != c->soft_rel) {
        c->soft_rel = rel;
        c->cloud_gen++;  // captured frame graphs hold the other splat sequence
    }
    return LNR_OK;
}

lnr_status lnr_set_precision(lnr_ctx* c, lnr_precision prec) {
    if (!c) return LNR_E_ARG;
    if (!c->unet_ok) return fail(c, LNR_E_STATE, "set_precision before set_unet");
    if (prec < LNR_FP32 || prec > LNR_FP8) return fail(c, LNR_E_ARG, "bad precision");
    if ((prec != LNR_FP32 && !tc_available()) || (prec != LNR_FP32 && c->unet.levels < 2))
        return fail(c, LNR_E_ARG, "precision not available for this net");
    if (prec == LNR_FP8 && !c->unet.fp8_ready) return fail(c, LNR_E_STATE, "FP8 needs lnr_calibrate first");
    c->prec = prec;
    return LNR_OK;
}

lnr_status lnr_render_batch(lnr_ctx* c, int nviews, const lnr_view* views, const lnr_intrinsics* in, int W, int H,
                            int nlev, const float* fs, float* out, int on_device) {
    if (!c) return LNR_E_ARG;
    lnr_status s = check_frame_args(c, nviews, views, in, W, H, nlev, fs, true);
    if (s != LNR_OK) return s;
    if (!out) return fail(c, LNR_E_ARG, "null output");
    cudaSetDevice(c->device);
    Workspace& ws = c->ws;
    s = prepare_views(c, ws, nviews, views, in, W, H, nlev, fs, c->prec);
    if (s != LNR_OK) return s;
    if (on_device) ws.out_ptr = out;  // the U-Net head writes the caller's buffer
    if (c->timing) {
        const uint64_t k0 = tl_launches;
        enqueue_frame(c, ws, ws.stream, -1, c->prec, true);
        c->times[7] = (double)(tl_launches - k0);
    } else {
        cudaError_t e = run_frame(c, ws, c->prec, true);
        if (e != cudaSuccess) return cuda_fail(c, e, "render launch");
    }
    return finish_output(c, ws, out, (size_t)nviews * W * H * 3, on_device);
}

lnr_status lnr_render(lnr_ctx* c, const lnr_view* view, const lnr_intrinsics* in, int W, int H, int nlev, float fs,
                      float* out, int on_device) {
    return lnr_render_batch(c, 1, view, in, W, H, nlev, &fs, out, on_device);
}

lnr_status lnr_training_input(lnr_ctx* c, const lnr_view* view, const lnr_intrinsics* in, int W, int H, int nlev,
                              float fs, const float* gt_rgb, int unfiltered, float* out) {
    if (!c) return LNR_E_ARG;
    lnr_status s = check_frame_args(c, 1, view, in, W, H, nlev, &fs, false);
    if (s != LNR_OK) return s;
    if (!gt_rgb || !out) return fail(c, LNR_E_ARG, "null ground truth or output");
    cudaSetDevice(c->device);
    Workspace& ws = c->ws;
    s = prepare_views(c, ws, 1, view, in, W, H, nlev, &fs, c->prec);
    if (s != LNR_OK) return s;
    enqueue_frame(c, ws, ws.stream, LNR_STAGE_FILTERED, c->prec, false);
    const size_t P = (size_t)W * H;
    DBuf gt, o5;
    cudaError_t e = gt.ensure(12 * P);
    if (!e) e = o5.ensure(20 * P);
    if (!e) e = cudaMemcpyAsync(gt.p, gt_rgb, 12 * P, cudaMemcpyHostToDevice, ws.stream);
    if (!e) {
        launch_training_input(ws, gt.as<float>(), in->zfar, unfiltered != 0, o5.as<float>(), ws.stream);
        e = cudaMemcpyAsync(out, o5.p, 20 * P, cudaMemcpyDeviceToHost, ws.stream);
    }
    if (!e) e = cudaStreamSynchronize(ws.stream);
    if (!e) e = cudaGetLastError();
    gt.release();
    o5.release();
    if (e != cudaSuccess) return cuda_fail(c, e, "training_input");
    return LNR_OK;
}

lnr_status lnr_render_stage(lnr_ctx* c, const lnr_view* view, const lnr_intrinsics* in, int W, int H, int nlev,
                            float fs, int stage, void* out, int on_device) {
    if (!c) return LNR_E_ARG;
    if (stage < LNR_STAGE_KEYS || stage > LNR_STAGE_CULL) return fail(c, LNR_E_ARG, "bad stage");
    lnr_status s = check_frame_args(c, 1, view, in, W, H, nlev, &fs, false);
    if (s != LNR_OK) return s;
    if (!out) return fail(c, LNR_E_ARG, "null output");
    cudaSetDevice(c->device);
    Workspace& ws = c->ws;
    s = prepare_views(c, ws, 1, view, in, W, H, nlev, &fs, c->prec);
    if (s != LNR_OK) return s;
    enqueue_frame(c, ws, ws.stream, stage, c->prec, false);
    const size_t P = (size_t)W * H;
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    cudaError_t e = cudaSuccess;
    std::vector<uint8_t> tmp;
    switch (stage) {
        case LNR_STAGE_CULL: {
            uint32_t t[2];
            e = cudaMemcpyAsync(t, ws.vis_tot.p, 8, cudaMemcpyDeviceToHost, ws.stream);
            if (!e) e = cudaStreamSynchronize(ws.stream);
            uint64_t r[2] = {t[0], t[1]};
            if (!e) e = cudaMemcpy(out, r, 16, on_device ? cudaMemcpyHostToDevice : cudaMemcpyHostToHost);
            break;
        }
        case LNR_STAGE_KEYS:
            e = cudaMemcpyAsync(out, ws.keys.p, 8 * P, kind, ws.stream);
            break;
        case LNR_STAGE_RGBDA_RAW: {
            std::vector<float> d(P);
            std::vector<uint32_t> col(P);
            e = cudaMemcpyAsync(d.data(), ws.depth.p, 4 * P, cudaMemcpyDeviceToHost, ws.stream);
            if (!e) e = cudaMemcpyAsync(col.data(), ws.rgba.p, 4 * P, cudaMemcpyDeviceToHost, ws.stream);
            if (!e) e = cudaStreamSynchronize(ws.stream);
            tmp.resize(8 * P);
            for (size_t q = 0; q < P; ++q) {
                std::memcpy(&tmp[8 * q], &d[q], 4);
                std::memcpy(&tmp[8 * q + 4], &col[q], 4);
            }
            if (!e) e = cudaMemcpy(out, tmp.data(), 8 * P, on_device ? cudaMemcpyHostToDevice : cudaMemcpyHostToHost);
            break;
        }
        case LNR_STAGE_FILTERED:
            e = cudaMemcpyAsync(out, ws.u0.p, 4 * P, kind, ws.stream);
            break;
        case LNR_STAGE_UNET_IN: {
            DBuf o5;
            e = o5.ensure(20 * P);
            if (!e) {
                launch_unet_in_extract(ws.act[4 * kMaxUnetLevels].p, 0, o5.as<float>(), (int64_t)P, ws.stream);
                e = cudaMemcpyAsync(out, o5.p, 20 * P, kind, ws.stream);
                if (!e) e = cudaStreamSynchronize(ws.stream);
            }
            o5.release();
            break;
        }
    }
    if (!e) e = cudaStreamSynchronize(ws.stream);
    if (!e) e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(c, e, "render_stage");
    return LNR_OK;
}

lnr_status lnr_calibrate(lnr_ctx* c, const lnr_view* view, const lnr_intrinsics* in, int W, int H, int nlev, float fs) {
    return lnr_calibrate_batch(c, 1, view, in, W, H, nlev, &fs);
}

lnr_status lnr_calibrate_batch(lnr_ctx* c, int nviews, const lnr_view* view, const lnr_intrinsics* in, int W, int H,
                               int nlev, const float* fs) {
    if (!c) return LNR_E_ARG;
    lnr_status s = check_frame_args(c, nviews, view, in, W, H, nlev, fs, true);
    if (s != LNR_OK) return s;
    if (c->prec == LNR_FP32 && !tc_available()) return fail(c, LNR_E_ARG, "no tensor-core path in this library");
    for (const auto& L : c->unet.convs)
        if (L.cout < 32 || (L.cin0 != 5 && L.cin0 % 32) || L.cin1 % 32)
            return fail(c, LNR_E_ARG, "FP8 needs every U-Net channel count to be a multiple of 32");
    cudaSetDevice(c->device);
    Workspace& ws = c->ws;
    s = prepare_views(c, ws, nviews, view, in, W, H, nlev, fs, LNR_BF16);  // the calibration frames run in BF16
    if (s != LNR_OK) return s;
    ws.allow_fuse = false;  // the calibration reads every conv's output
    enqueue_frame(c, ws, ws.stream, -1, LNR_BF16, false);
    ws.allow_fuse = true;
    cudaError_t e = cudaStreamSynchronize(ws.stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "calibration frame");
    return unet_calibrate_fp8(c, ws);
}

lnr_status lnr_autotune(lnr_ctx* c, int W, int H, int batch) {
    if (!c) return LNR_E_ARG;
    if (!c->unet_ok) return fail(c, LNR_E_STATE, "autotune before set_unet");
    const int m = 1 << (c->unet.levels - 1);
    if (W < m || H < m || W % m || H % m || batch < 1 || batch > 64 || (int64_t)W * H * batch > (1ll << 31))
        return fail(c, LNR_E_ARG, "autotune: W, H must be multiples of 2^(levels-1); batch in [1, 64]");
    if (c->prec == LNR_FP32) return LNR_OK;  // the FP32 path has one kernel per layer shape
    cudaSetDevice(c->device);
    Workspace& ws = c->ws;
    cudaError_t e = cudaStreamSynchronize(ws.stream);
    ws.B = batch;
    ws.W = W;
    ws.H = H;
    const void* in_before = ws.act[4 * kMaxUnetLevels].p;
    const void* out_before = ws.out.p;
    if (!e) e = ws.act[4 * kMaxUnetLevels].ensure((size_t)batch * W * H * unet_in_bytes_per_px(c->prec) + 256);
    if (!e) e = ws.out.ensure((size_t)batch * W * H * 12);
    if (!e) e = unet_ensure(c->unet, ws, LNR_FP32);
    if (e != cudaSuccess) return cuda_fail(c, e, "autotune buffers");
    if (in_before != ws.act[4 * kMaxUnetLevels].p || out_before != ws.out.p) ws.alloc_gen++;
    return unet_autotune(c, ws, c->prec, 3);
}

lnr_status lnr_set_timing(lnr_ctx* c, int enable) {
    if (!c) return LNR_E_ARG;
    c->timing = enable != 0;
    return LNR_OK;
}

lnr_status lnr_get_timing(lnr_ctx* c, double out[8]) {
    if (!c || !out) return LNR_E_ARG;
    std::memcpy(out, c->times, sizeof(c->times));
    return LNR_OK;
}

lnr_status lnr_probe_atomic_rate(lnr_ctx* c, uint64_t n_slots, uint64_t n_ops, int coherent, double* ops_per_s) {
    if (!c) return LNR_E_ARG;
    if (!ops_per_s || n_slots == 0 || n_slots > (1ull << 32) || n_ops == 0 || n_ops > (1ull << 34))
        return fail(c, LNR_E_ARG, "atomic probe: n_slots in [1, 2^32], n_ops in [1, 2^34]");
    cudaSetDevice(c->device);
    Workspace& ws = c->ws;
    cudaError_t e = cudaStreamSynchronize(ws.stream);
    if (!e) e = probe_atomic_rate(n_slots, n_ops, coherent != 0, c->num_sms, ws.stream, ops_per_s);
    if (e == cudaErrorMemoryAllocation) return fail(c, LNR_E_OOM, "atomic probe buffer");
    if (e != cudaSuccess) return cuda_fail(c, e, "atomic probe");
    return LNR_OK;
}

}  // extern "C"
