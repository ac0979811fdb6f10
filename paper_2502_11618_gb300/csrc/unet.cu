// U-Net reconstruction (Fig. 1; Sec. 3, "U-Net Reconstruction"): encoder of two 3x3
// convolutions + ReLU per level with 2x2 max pooling between levels, decoder of nearest
// 2x upsampling, concatenation [skip, upsampled] and two 3x3 convolutions + ReLU, then a
// 1x1 head with a sigmoid.  Batch norm after the encoder convolutions is folded into them
// when the weights are loaded.
//
// This file holds the FP32 path (CUDA-core implicit GEMM; the accuracy reference of the
// GPU) and the layer orchestration shared by every precision.  Pooling, upsampling and
// concatenation are fused into the convolutions: nothing but conv outputs is written.
#include <cmath>
#include <cuda_bf16.h>
#include <cstdio>
#include <cstdlib>
#include <cstring>

#include "lnr_internal.h"

namespace lnr {
namespace {

struct ConvArgsF32 {
    const float* src0;  // NHWC, c0 channels, output resolution
    const float* src1;  // NHWC, c1 channels, half resolution (read nearest-upsampled), or null
    int c0, c1;
    int W, H;
    const float* w;     // [9][c0 + c1][cout]
    const float* bias;  // [cout]
    int cout;
    float* out;         // NHWC, cout channels
    float* pool_out;    // NHWC, cout channels at W/2 x H/2, or null
};

// Tile: 2 rows x TW pixels x CT output channels.  Thread = one 2x2 pixel quad x 8 output
// channels; K is walked 8 input channels at a time, all 9 taps per chunk, from a shared
// halo tile of 4 rows x (TW+2) pixels.
template <int TW, int CT>
__global__ void __launch_bounds__(256) k_conv3x3_f32(const ConvArgsF32 a) {
    constexpr int NCOG = CT / 8;
    constexpr int HW = TW + 2;
    static_assert((TW / 2) * NCOG == 256, "256 threads");
    __shared__ float sin_[8][4][HW];
    __shared__ __align__(16) float sw[9][8][CT];
    const int cog = threadIdx.x % NCOG, q = threadIdx.x / NCOG;
    const int x0 = blockIdx.x * TW, y0 = blockIdx.y * 2;
    const int nco_blocks = a.cout / CT;
    const int view = blockIdx.z / nco_blocks;
    const int co0 = (blockIdx.z % nco_blocks) * CT;
    const int cin = a.c0 + a.c1;
    const size_t P = (size_t)a.W * a.H;
    const int Wh = a.W >> 1, Hh = a.H >> 1;
    const float* s0 = a.src0 + view * P * a.c0;
    const float* s1 = a.src1 ? a.src1 + view * (size_t)Wh * Hh * a.c1 : nullptr;
    float acc[4][8];
#pragma unroll
    for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[p][j] = 0.f;

    for (int cb = 0; cb < cin; cb += 8) {
        __syncthreads();
        for (int idx = threadIdx.x; idx < 4 * HW * 2; idx += 256) {
            const int h = idx & 1, j = (idx >> 1) % HW, r = (idx >> 1) / HW;
            const int gx = x0 - 1 + j, gy = y0 - 1 + r;
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (gx >= 0 && gx < a.W && gy >= 0 && gy < a.H) {
                if (cb < a.c0)
                    v = *reinterpret_cast<const float4*>(s0 + ((size_t)gy * a.W + gx) * a.c0 + cb + 4 * h);
                else
                    v = *reinterpret_cast<const float4*>(s1 + ((size_t)(gy >> 1) * Wh + (gx >> 1)) * a.c1 +
                                                         (cb - a.c0) + 4 * h);
            }
            sin_[4 * h + 0][r][j] = v.x;
            sin_[4 * h + 1][r][j] = v.y;
            sin_[4 * h + 2][r][j] = v.z;
            sin_[4 * h + 3][r][j] = v.w;
        }
        for (int idx = threadIdx.x; idx < 9 * 8 * (CT / 4); idx += 256) {
            const int c4 = idx % (CT / 4), ci = (idx / (CT / 4)) % 8, t = idx / (CT / 4) / 8;
            *reinterpret_cast<float4*>(&sw[t][ci][4 * c4]) =
                *reinterpret_cast<const float4*>(a.w + ((size_t)t * cin + cb + ci) * a.cout + co0 + 4 * c4);
        }
        __syncthreads();
#pragma unroll 2
        for (int ci = 0; ci < 8; ++ci) {
            float in[4][4];
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int c = 0; c < 4; ++c) in[r][c] = sin_[ci][r][2 * q + c];
#pragma unroll
            for (int ky = 0; ky < 3; ++ky)
#pragma unroll
                for (int kx = 0; kx < 3; ++kx) {
                    const float4 w0 = *reinterpret_cast<const float4*>(&sw[ky * 3 + kx][ci][cog * 8]);
                    const float4 w1 = *reinterpret_cast<const float4*>(&sw[ky * 3 + kx][ci][cog * 8 + 4]);
                    const float wv[8] = {w0.x, w0.y, w0.z, w0.w, w1.x, w1.y, w1.z, w1.w};
                    const float av[4] = {in[ky][kx], in[ky][kx + 1], in[ky + 1][kx], in[ky + 1][kx + 1]};
#pragma unroll
                    for (int p = 0; p < 4; ++p)
#pragma unroll
                        for (int j = 0; j < 8; ++j) acc[p][j] = fmaf(av[p], wv[j], acc[p][j]);
                }
        }
    }
    const int co = co0 + cog * 8;
    float b[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) b[j] = a.bias[co + j];
    float mx[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) mx[j] = 0.f;
#pragma unroll
    for (int p = 0; p < 4; ++p) {
        const int x = x0 + 2 * q + (p & 1), y = y0 + (p >> 1);
        float o[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            o[j] = fmaxf(acc[p][j] + b[j], 0.f);
            mx[j] = fmaxf(mx[j], o[j]);
        }
        if (x < a.W && y < a.H) {
            float4* dst = reinterpret_cast<float4*>(a.out + (view * P + (size_t)y * a.W + x) * a.cout + co);
            dst[0] = make_float4(o[0], o[1], o[2], o[3]);
            dst[1] = make_float4(o[4], o[5], o[6], o[7]);
        }
    }
    if (a.pool_out) {
        const int px = (x0 >> 1) + q, py = y0 >> 1;
        if (px < Wh && py < Hh) {
            float4* dst = reinterpret_cast<float4*>(a.pool_out + (view * (size_t)Wh * Hh + (size_t)py * Wh + px) * a.cout + co);
            dst[0] = make_float4(mx[0], mx[1], mx[2], mx[3]);
            dst[1] = make_float4(mx[4], mx[5], mx[6], mx[7]);
        }
    }
}

// 1x1 head + sigmoid: out[q][o] = 1 / (1 + exp(-(b[o] + sum_c w[o][c] x[q][c]))).
__global__ void k_head_f32(const float* __restrict__ x, int C, const float* __restrict__ w,
                           const float* __restrict__ b, int O, float* __restrict__ out, size_t npx) {
    size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (q >= npx) return;
    const float* xp = x + q * C;
    for (int o = 0; o < O; ++o) {
        float acc = b[o];
        for (int c = 0; c < C; ++c) acc = fmaf(w[o * C + c], xp[c], acc);
        out[q * O + o] = 1.0f / (1.0f + expf(-acc));
    }
}

void conv_f32(const ConvLayer& L, const float* src0, const float* src1, float* out, float* pool_out, int B,
              int W, int H, cudaStream_t st) {
    ConvArgsF32 a{src0, src1, L.cin0 == 5 ? 8 : L.cin0, L.cin1, W, H, L.w32, L.b32, L.cout, out, pool_out};
    if (L.cout % 64 == 0) {
        dim3 g((W + 63) / 64, (H + 1) / 2, B * (L.cout / 64));
        k_conv3x3_f32<64, 64><<<g, 256, 0, st>>>(a);
        count_launch();
    } else if (L.cout % 32 == 0) {
        dim3 g((W + 127) / 128, (H + 1) / 2, B * (L.cout / 32));
        k_conv3x3_f32<128, 32><<<g, 256, 0, st>>>(a);
        count_launch();
    } else {
        dim3 g((W + 255) / 256, (H + 1) / 2, B * (L.cout / 16));
        k_conv3x3_f32<256, 16><<<g, 256, 0, st>>>(a);
        count_launch();
    }
}

// Activation buffer slots: for level l, 4*l + {0: first conv out, 1: skip, 2: pooled, 3: decoder out}.
inline int slot(int l, int k) { return 4 * l + k; }

}  // namespace

int unet_in_kind(lnr_precision p) { return p == LNR_FP32 ? 0 : 1; }
// Bytes per pixel of the network-input buffer: 8 FP32 or 16 BF16 channels (the stage taps use
// the FP32 layout at every precision).
size_t unet_in_bytes_per_px(lnr_precision) { return 32; }

static size_t elem_bytes(lnr_precision p) { return p == LNR_FP32 ? 4 : 2; }

// Activation buffers of the forward pass (the network input and output are counted with the
// frame's raster buffers): four per level, each at most the level's size (+ 256 bytes).
size_t unet_act_bytes(const Unet& u, int B, int W, int H, lnr_precision p) {
    size_t tot = 0;
    for (int l = 0; l < u.levels; ++l) {
        size_t Pl = (size_t)B * (W >> l) * (H >> l);
        tot += (Pl * u.ch[l] * elem_bytes(p) + 256) * 4;
    }
    return tot;
}

// Ensure the activation buffers of the workspace for (B, W, H); a reallocation bumps the
// workspace's allocation generation (captured graphs must be rebuilt).
cudaError_t unet_ensure(const Unet& u, Workspace& ws, lnr_precision p) {
    const size_t e = elem_bytes(p);
    cudaError_t err;
    for (int l = 0; l < u.levels; ++l) {
        size_t Pl = (size_t)ws.B * (ws.W >> l) * (ws.H >> l);
        for (int k = 0; k < 4; ++k) {
            size_t n = (k == 2) ? (size_t)ws.B * (ws.W >> (l + 1)) * (ws.H >> (l + 1)) * u.ch[l] : Pl * u.ch[l];
            const void* before = ws.act[slot(l, k)].p;
            if ((err = ws.act[slot(l, k)].ensure(n * e + 256))) return err;
            if (before != ws.act[slot(l, k)].p) ws.alloc_gen++;
        }
    }
    return cudaSuccess;
}

// One convolution launch of the forward pass: layer, sources, outputs, resolution.
struct ConvCall {
    int layer;
    const void* src0;
    const void* src1;
    void* out;
    void* pool;
    const float* head_w;   // device
    const float* head_b;
    const float* head_wh;  // host copies
    const float* head_bh;
    float* head_out;
    int W, H;
};

// The forward pass as a list of convolution launches (encoder: conv, conv (+pool) per
// level; decoder: concat conv, conv (+head on the last)); buffers from the workspace.
static std::vector<ConvCall> unet_plan(const Unet& u, Workspace& ws, lnr_precision p, const void* in, float* out) {
    std::vector<ConvCall> calls;
    const int L = u.levels;
    int ci = 0;
    const void* x = in;
    for (int l = 0; l < L; ++l) {
        const int W = ws.W >> l, H = ws.H >> l;
        void* t = ws.act[slot(l, 0)].p;
        void* s = ws.act[slot(l, 1)].p;
        void* pl = (l < L - 1) ? ws.act[slot(l, 2)].p : nullptr;
        calls.push_back({ci, x, nullptr, t, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, W, H});
        calls.push_back({ci + 1, t, nullptr, s, pl, nullptr, nullptr, nullptr, nullptr, nullptr, W, H});
        ci += 2;
        x = pl;
    }
    const void* deep = ws.act[slot(L - 1, 1)].p;
    for (int l = L - 2; l >= 0; --l) {
        const int W = ws.W >> l, H = ws.H >> l;
        void* t = ws.act[slot(l, 0)].p;
        void* d = ws.act[slot(l, 3)].p;
        const void* skip = ws.act[slot(l, 1)].p;
        calls.push_back({ci, skip, deep, t, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, W, H});
        const bool fuse_head = (l == 0) && p != LNR_FP32;
        calls.push_back({ci + 1, t, nullptr, d, nullptr, fuse_head ? u.head_w : nullptr, fuse_head ? u.head_b : nullptr,
                         fuse_head ? u.head_wh.data() : nullptr, fuse_head ? u.head_bh.data() : nullptr,
                         fuse_head ? out : nullptr, W, H});
        ci += 2;
        deep = d;
    }
    return calls;
}

static void run_call(const Unet& u, const ConvCall& k, Workspace& ws, lnr_precision p, cudaStream_t st,
                     const TcConfig* force) {
    const ConvLayer& L = u.convs[k.layer];
    if (p == LNR_FP32)
        conv_f32(L, (const float*)k.src0, (const float*)k.src1, (float*)k.out, (float*)k.pool, ws.B, k.W, k.H, st);
    else
        tc_conv(L, p, k.src0, k.src1, k.out, k.pool, k.head_w, k.head_b, k.head_wh, k.head_bh, k.head_out, ws.B, k.W, k.H,
                u.out_ch, st, force);
}

// Rows per tile of the fused level-0 encoder for the layer resolution (W, H), or 0 to run
// the first two convs apart: the autotuner's choice, else LNR_CONV_FUSE0=2|4 (tests).
static int fuse_rows(const Unet& u, lnr_precision p, int W, int H) {
    if (p == LNR_FP32 || u.convs.size() < 2) return 0;
    static const int forced = [] {
        const char* e = getenv("LNR_CONV_FUSE0");
        const int v = e ? atoi(e) : 0;
        return v == 2 || v == 4 ? v : 0;
    }();
    const auto& table = p == LNR_FP8 ? u.convs[0].tuned8 : u.convs[0].tuned;
    auto it = table.find({W, H});
    if (it != table.end() && it->second.F) return it->second.F;
    return forced;
}

void unet_forward(const lnr_ctx* c, Workspace& ws, lnr_precision p, const void* in, float* out,
                  cudaStream_t st, cudaEvent_t* layer_ev) {
    const Unet& u = c->unet;
    if (unet_ensure(u, ws, p) != cudaSuccess) return;
    int ev = 0;
    if (layer_ev) cudaEventRecord(layer_ev[ev++], st);
    const std::vector<ConvCall> calls = unet_plan(u, ws, p, in, out);
    for (size_t i = 0; i < calls.size(); ++i) {
        const ConvCall& k = calls[i];
        if (k.layer == 0 && i + 1 < calls.size() && ws.allow_fuse) {
            const int R = fuse_rows(u, p, k.W, k.H);
            const ConvCall& k1 = calls[i + 1];
            if (R && tc_fused_enc0(u.convs[0], u.convs[1], p, k.src0, k1.out, k1.pool, ws.B, k.W, k.H, R, st)) {
                ++i;  // both convs done
                if (layer_ev) cudaEventRecord(layer_ev[ev++], st);
                if (layer_ev) cudaEventRecord(layer_ev[ev++], st);
                continue;
            }
        }
        run_call(u, k, ws, p, st, nullptr);
        if (layer_ev) cudaEventRecord(layer_ev[ev++], st);
    }
    if (p == LNR_FP32) {
        const void* deep = ws.act[slot(u.levels > 1 ? 0 : 0, u.levels > 1 ? 3 : 1)].p;
        size_t npx = (size_t)ws.B * ws.W * ws.H;
        k_head_f32<<<(unsigned)((npx + 255) / 256), 256, 0, st>>>((const float*)deep, u.ch[0], u.head_w, u.head_b,
                                                                  u.out_ch, out, npx);
        count_launch();
        if (layer_ev) cudaEventRecord(layer_ev[ev++], st);
    }
}

// FP8 policy.  Headroom of the static activation scales over the calibration frames'
// largest magnitudes, and the convolutions that keep BF16 operands: the full-resolution
// encoder convs (the first reads the BF16 RGBDA image) and every decoder conv at full and
// half resolution (the last one's features feed the output head).  E4M3's three mantissa
// bits cost the most accuracy there: on 16 1080p views keeping the second encoder conv in
// BF16 raised the minimum PSNR by 0.8 dB, and on a small frame with other weights the
// decoder's level-1 convs decided whether the 38 dB bar held.  Scale headroom between 2
// and 64 changed nothing measurable (E4M3 is floating point).  LNR_FP8_HEADROOM and
// LNR_FP8_BF16_LAYERS (comma-separated indices in network order, replacing the default
// set) override them for measurements.
constexpr float kFp8Headroom = 8.0f;

static float fp8_headroom() {
    const char* e = getenv("LNR_FP8_HEADROOM");
    const float v = e ? (float)atof(e) : kFp8Headroom;
    return v >= 1.0f && v <= 1e4f ? v : kFp8Headroom;
}

static bool fp8_layer_bf16(int layer, int level, bool decoder) {
    static const char* env = getenv("LNR_FP8_BF16_LAYERS");
    if (!env) return decoder ? level <= 1 : level == 0;
    static const std::vector<int> keep = [] {
        std::vector<int> v;
        for (const char* p = env; p && *p;) {
            v.push_back(atoi(p));
            p = strchr(p, ',');
            if (p) ++p;
        }
        return v;
    }();
    for (int k : keep)
        if (k == layer) return true;
    return false;
}

__global__ void k_amax_bf16(const __nv_bfloat16* __restrict__ x, size_t n, unsigned* __restrict__ out) {
    float m = 0.f;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        m = fmaxf(m, fabsf(__bfloat162float(x[i])));
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out, __float_as_uint(m));  // non-negative floats order as integers
}

// FP8 calibration, after a BF16 forward pass on ws: the largest magnitude of every
// convolution's output gives that tensor's E4M3 scale (amax / 448); each layer's E4M3
// weights then fold in the scales of its inputs.  The first conv keeps BF16 operands (its
// input is the RGBDA image) and writes E4M3.
lnr_status unet_calibrate_fp8(lnr_ctx* c, Workspace& ws) {
    Unet& u = c->unet;
    const void* in = ws.act[4 * kMaxUnetLevels].p;
    const std::vector<ConvCall> calls = unet_plan(u, ws, LNR_BF16, in, ws.out.as<float>());
    unsigned* d_amax = nullptr;
    cudaError_t e = cudaMalloc(&d_amax, sizeof(unsigned) * calls.size());
    if (e != cudaSuccess) return cuda_fail(c, e, "calibration");
    cudaMemsetAsync(d_amax, 0, sizeof(unsigned) * calls.size(), ws.stream);
    for (size_t i = 0; i < calls.size(); ++i) {
        const ConvCall& k = calls[i];
        if (k.head_out) continue;  // the last conv's features go straight into the head
        const size_t n = (size_t)ws.B * k.W * k.H * u.convs[k.layer].cout;
        k_amax_bf16<<<1024, 256, 0, ws.stream>>>(static_cast<const __nv_bfloat16*>(k.out), n, d_amax + i);
    }
    std::vector<unsigned> h(calls.size());
    e = cudaMemcpyAsync(h.data(), d_amax, sizeof(unsigned) * calls.size(), cudaMemcpyDeviceToHost, ws.stream);
    if (!e) e = cudaStreamSynchronize(ws.stream);
    cudaFree(d_amax);
    if (e != cudaSuccess) return cuda_fail(c, e, "calibration");
    // Buffers are reused across levels (an encoder and a decoder conv of one level write
    // the same slot), so the producer of an input is the LAST earlier call that wrote it.
    std::vector<float> sc(calls.size());
    for (size_t i = 0; i < calls.size(); ++i) {
        float a;
        std::memcpy(&a, &h[i], 4);
        // headroom of 8x over the calibration view's maximum: other views may see larger
        // activations, and E4M3 keeps its relative precision over a wide exponent range, so
        // the margin costs almost nothing while clipping would cost a lot
        sc[i] = std::max(a, 1e-6f) * fp8_headroom() / 448.0f;
        u.convs[calls[i].layer].out_scale = sc[i];
        u.convs[calls[i].layer].out_bf16 = false;
    }
    auto producer = [&](size_t i, const void* buf) -> int {
        for (size_t j = i; j-- > 0;)
            if (calls[j].out == buf || (calls[j].pool && calls[j].pool == buf)) return (int)j;
        return -1;  // the BF16 input image
    };
    // BF16 operands for the first conv (the BF16 input image) and the last one (its
    // features feed the output head directly) -- optionally the whole full-resolution
    // decoder level; E4M3 everywhere else.  A producer writes BF16 for a BF16 consumer.
    for (size_t i = 0; i < calls.size(); ++i) {
        const ConvCall& k = calls[i];
        ConvLayer& L = u.convs[k.layer];
        L.pool_bf16 = false;
        const int p0 = producer(i, k.src0);
        const bool bf16 = p0 < 0 || k.head_out || fp8_layer_bf16(k.layer, L.level, k.layer >= 2 * u.levels);
        L.fp8 = !bf16;
        if (bf16) {
            for (const void* src : {k.src0, k.src1}) {
                if (!src) continue;
                const int pj = producer(i, src);
                if (pj < 0) continue;
                if (calls[pj].out == src) u.convs[calls[pj].layer].out_bf16 = true;
                else u.convs[calls[pj].layer].pool_bf16 = true;
            }
        }
    }
    for (size_t i = 0; i < calls.size(); ++i) {
        const ConvCall& k = calls[i];
        ConvLayer& L = u.convs[k.layer];
        if (!L.fp8) continue;
        L.in_scale[0] = sc[producer(i, k.src0)];
        const int p1 = k.src1 ? producer(i, k.src1) : -1;
        L.in_scale[1] = p1 >= 0 ? sc[p1] : 1.f;
        if ((e = tc_prepare_fp8(L)) != cudaSuccess) return cuda_fail(c, e, "FP8 weights");
        L.fp8 = true;
    }
    u.fp8_ready = true;
    c->unet_gen++;
    return LNR_OK;
}

// Autotuner: for every tensor-core convolution of the forward pass at the workspace's
// (B, W, H), time each candidate kernel configuration (CUDA events, `reps` launches after a
// warm-up launch) on the layer's real buffers and keep the fastest for that layer
// resolution.  Contents of the buffers do not matter: the kernels are data-independent.
lnr_status unet_autotune(lnr_ctx* c, Workspace& ws, lnr_precision p, int reps) {
    Unet& u = c->unet;
    if (p == LNR_FP32) return LNR_OK;
    cudaError_t e = unet_ensure(u, ws, p);
    if (e != cudaSuccess) return cuda_fail(c, e, "autotune buffers");
    cudaStream_t st = ws.stream;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const void* in = ws.act[4 * kMaxUnetLevels].p;
    // LNR_TUNE_LOG=1: each layer's choice on stderr; =2: also every candidate's time
    static const int log = [] {
        const char* v = getenv("LNR_TUNE_LOG");
        return v ? std::max(1, atoi(v)) : 0;
    }();
    const std::vector<ConvCall> calls = unet_plan(u, ws, p, in, ws.out.as<float>());
    std::vector<float> best_ms(calls.size(), 0.f);
    for (size_t ci = 0; ci < calls.size(); ++ci) {
        const ConvCall& k = calls[ci];
        ConvLayer& L = u.convs[k.layer];
        float best = 1e30f;
        TcConfig best_cfg;
        for (const TcConfig& cfg : tc_candidates(L, p)) {
            run_call(u, k, ws, p, st, &cfg);  // warm-up (and first-use set-up)
            cudaEventRecord(e0, st);
            for (int r = 0; r < reps; ++r) run_call(u, k, ws, p, st, &cfg);
            cudaEventRecord(e1, st);
            if ((e = cudaEventSynchronize(e1)) != cudaSuccess) break;
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (tc_error_word()) continue;  // a configuration that failed is never chosen
            if (log >= 2)
                fprintf(stderr, "  candidate layer %d: mode %d R %d P %d ck %d O %d E %d  %.1f us\n", k.layer, cfg.mode,
                        cfg.R, cfg.P, cfg.CK, cfg.O, cfg.E, 1e3 * ms / reps);
            if (ms < best) {
                best = ms;
                best_cfg = cfg;
            }
        }
        if (e != cudaSuccess) break;
        best_ms[ci] = best;
        (p == LNR_FP8 ? L.tuned8 : L.tuned)[{k.W, k.H}] = best_cfg;
        if (log)
            fprintf(stderr, "autotune layer %d %dx%d: mode %d R %d P %d ck %d O %d E %d  %.1f us\n", k.layer, k.W, k.H,
                    best_cfg.mode, best_cfg.R, best_cfg.P, best_cfg.CK, best_cfg.O, best_cfg.E, 1e3 * best / reps);
    }
    // the first two convs fused, against the two best separate configurations
    if (e == cudaSuccess && calls.size() >= 2 && calls[0].layer == 0 && calls[1].layer == 1) {
        const ConvCall &k0 = calls[0], &k1 = calls[1];
        auto& entry = (p == LNR_FP8 ? u.convs[0].tuned8 : u.convs[0].tuned)[{k0.W, k0.H}];
        entry.F = 0;
        float best = best_ms[0] + best_ms[1];
        for (int R : {2, 4}) {
            if (!tc_fused_enc0(u.convs[0], u.convs[1], p, k0.src0, k1.out, k1.pool, ws.B, k0.W, k0.H, R, st)) continue;
            cudaEventRecord(e0, st);
            for (int r = 0; r < reps; ++r)
                tc_fused_enc0(u.convs[0], u.convs[1], p, k0.src0, k1.out, k1.pool, ws.B, k0.W, k0.H, R, st);
            cudaEventRecord(e1, st);
            if ((e = cudaEventSynchronize(e1)) != cudaSuccess) break;
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (tc_error_word()) continue;
            if (log) fprintf(stderr, "autotune fused layers 0+1 %dx%d: R %d  %.1f us (apart %.1f us)\n", k0.W, k0.H, R,
                             1e3 * ms / reps, 1e3 * (best_ms[0] + best_ms[1]) / reps);
            if (ms < best) {
                best = ms;
                entry.F = R;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) return cuda_fail(c, e, "autotune");
    c->unet_gen++;  // captured graphs hold the old kernel choices
    return LNR_OK;
}

// Convert the host weights (already batch-norm folded) to the device layouts.
lnr_status unet_prepare(lnr_ctx* c) {
    Unet& u = c->unet;
    for (auto& L : u.convs) {
        const int cin = L.cin0 + L.cin1;
        const int cin_pad = (L.cin0 == 5 ? 8 : L.cin0) + L.cin1;
        L.cin_pad = cin_pad;
        std::vector<float> w((size_t)9 * cin_pad * L.cout, 0.f);
        for (int co = 0; co < L.cout; ++co)
            for (int ci = 0; ci < cin; ++ci)
                for (int t = 0; t < 9; ++t) w[((size_t)t * cin_pad + ci) * L.cout + co] = L.wf[((size_t)co * cin + ci) * 9 + t];
        if (L.w32) cudaFree(L.w32);
        if (L.b32) cudaFree(L.b32);
        if (cudaMalloc(&L.w32, w.size() * 4) || cudaMalloc(&L.b32, L.cout * 4))
            return fail(c, LNR_E_OOM, "U-Net weight upload");
        cudaMemcpy(L.w32, w.data(), w.size() * 4, cudaMemcpyHostToDevice);
        cudaMemcpy(L.b32, L.bf.data(), L.cout * 4, cudaMemcpyHostToDevice);
        if (tc_available()) {
            for (lnr_precision p : {LNR_BF16}) {
                cudaError_t e = tc_prepare_layer(L, p);
                if (e != cudaSuccess) return cuda_fail(c, e, "tensor-core weight upload");
            }
        }
    }
    if (u.head_w) cudaFree(u.head_w);
    if (u.head_b) cudaFree(u.head_b);
    if (cudaMalloc(&u.head_w, u.head_wh.size() * 4) || cudaMalloc(&u.head_b, u.head_bh.size() * 4))
        return fail(c, LNR_E_OOM, "U-Net head upload");
    cudaMemcpy(u.head_w, u.head_wh.data(), u.head_wh.size() * 4, cudaMemcpyHostToDevice);
    cudaMemcpy(u.head_b, u.head_bh.data(), u.head_bh.size() * 4, cudaMemcpyHostToDevice);
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(c, e, "U-Net upload");
    return LNR_OK;
}

}  // namespace lnr
