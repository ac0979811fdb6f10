// Per-frame projection and depth filter of the render path:
//   cull     frustum culling of grid cells and compaction of the visible ones
//            (Sec. 1; Sec. 3, "Point Cloud Projection"; Fig. 1)
//   splat    1x1-pixel projection of the visible cells' points into a 64-bit z-buffer
//            keyed by (float bits of z << 32 | sorted position)        (Sec. 3)
//   resolve  keys -> depth D, colour and fill mask A, fused with the whole min-pool
//            pyramid of a 64x64 tile                                   (Fig. 1; Fig. 2)
//   upsample one Laplacian-edge-aware upsampling step per level, with the
//            linear-interpolation fill on non-final levels and, on the final level, the
//            packing of the U-Net's RGBDA input                        (Fig. 2; Sec. 3)
//
// Compiled with --fmad=false and written with explicit round-to-nearest intrinsics: the
// arithmetic of culling, projection and filtering is exactly the sequence of FP32
// operations of the method's definition, so the results are bit-exact against any
// implementation of that same sequence.
#include <cuda_bf16.h>

#include "lnr_internal.h"

namespace lnr {

void scan_exclusive_u32(const uint32_t* in, uint32_t* out, uint64_t n, uint32_t* tmp, cudaStream_t st);

namespace {

constexpr float kEdgeRel = 0.1f;         // edge when |Laplacian| > kEdgeRel * depth
constexpr float kCullPad = 1.0f / 64.0f; // cells grow by 1/64 of a step on every side
constexpr int kCullThreads = 256;
constexpr int kCullPer = 4;
constexpr int kCullTile = kCullThreads * kCullPer;
constexpr int kSplatThreads = 256;
constexpr int kSplatChunk = 1024;  // visible points per splat range (one warp's unit of work)
constexpr uint64_t kEmpty = ~0ull;

__device__ __forceinline__ void cell_cam(int64_t i, int64_t j, int64_t k, const ViewDev& v, float o[3]) {
    float di = (float)(i - v.anchor[0]), dj = (float)(j - v.anchor[1]), dk = (float)(k - v.anchor[2]);
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        float t = __fmaf_rn(di, v.s[0 + r], v.d0[r]);
        t = __fmaf_rn(dj, v.s[3 + r], t);
        o[r] = __fmaf_rn(dk, v.s[6 + r], t);
    }
}

// ---------------------------------------------------------------- culling ----

__device__ bool cell_visible(int64_t i, int64_t j, int64_t k, const ViewDev& v, int W, int H) {
    float o[3];
    cell_cam(i, j, k, v, o);
    const float cxw = __fsub_rn(v.cx, (float)W), cyh = __fsub_rn(v.cy, (float)H);
    bool out_all[6] = {true, true, true, true, true, true};
#pragma unroll
    for (int corner = 0; corner < 8; ++corner) {
        float tx = (corner & 1) ? 1.0f + kCullPad : -kCullPad;
        float ty = (corner & 2) ? 1.0f + kCullPad : -kCullPad;
        float tz = (corner & 4) ? 1.0f + kCullPad : -kCullPad;
        float p[3];
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            float t = __fmaf_rn(tx, v.s[0 + r], o[r]);
            t = __fmaf_rn(ty, v.s[3 + r], t);
            p[r] = __fmaf_rn(tz, v.s[6 + r], t);
        }
        const float x = p[0], y = p[1], z = p[2];
        float pl[6];
        pl[0] = __fsub_rn(z, v.znear);
        pl[1] = __fsub_rn(v.zfar, z);
        pl[2] = __fmaf_rn(v.fx, x, __fmul_rn(v.cx, z));
        pl[3] = -__fmaf_rn(v.fx, x, __fmul_rn(cxw, z));
        pl[4] = __fmaf_rn(v.fy, y, __fmul_rn(v.cy, z));
        pl[5] = -__fmaf_rn(v.fy, y, __fmul_rn(cyh, z));
#pragma unroll
        for (int q = 0; q < 6; ++q) out_all[q] = out_all[q] && (pl[q] < 0.0f);
    }
    bool culled = false;
#pragma unroll
    for (int q = 0; q < 6; ++q) culled |= out_all[q];
    return !culled;
}

__device__ __forceinline__ void block_scan2(uint32_t a, uint32_t b, uint32_t& ea, uint32_t& eb,
                                            uint32_t& ta, uint32_t& tb) {
    __shared__ uint32_t wa[kCullThreads / 32], wb[kCullThreads / 32];
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t xa = a, xb = b;
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t ya = __shfl_up_sync(0xffffffffu, xa, o), yb = __shfl_up_sync(0xffffffffu, xb, o);
        if (lane >= o) { xa += ya; xb += yb; }
    }
    if (lane == 31) { wa[warp] = xa; wb[warp] = xb; }
    __syncthreads();
    if (warp == 0) {
        const int nw = kCullThreads / 32;
        uint32_t sa = lane < nw ? wa[lane] : 0, sb = lane < nw ? wb[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t ya = __shfl_up_sync(0xffffffffu, sa, o), yb = __shfl_up_sync(0xffffffffu, sb, o);
            if (lane >= o) { sa += ya; sb += yb; }
        }
        if (lane < nw) { wa[lane] = sa; wb[lane] = sb; }
    }
    __syncthreads();
    ea = (warp ? wa[warp - 1] : 0) + xa - a;
    eb = (warp ? wb[warp - 1] : 0) + xb - b;
    ta = wa[kCullThreads / 32 - 1];
    tb = wb[kCullThreads / 32 - 1];
    __syncthreads();
}

// Phase 1: visibility of every cell, block-local ranks of the visible non-empty cells and
// of their points.  flag[c] = local rank or ~0; cnt[c] = local point prefix.
__global__ void __launch_bounds__(kCullThreads) k_cull_block(
    const ViewDev* __restrict__ views, const uint32_t* __restrict__ cell_start, int dx, int dy,
    int dz, int64_t C, int W, int H, uint32_t* __restrict__ flag, uint32_t* __restrict__ cnt,
    uint32_t* __restrict__ bsum, int nb) {
    const int view = blockIdx.y;
    const ViewDev v = views[view];
    int64_t c0 = (int64_t)blockIdx.x * kCullTile + (int64_t)threadIdx.x * kCullPer;
    uint32_t f[kCullPer], n[kCullPer], sf = 0, sn = 0;
#pragma unroll
    for (int e = 0; e < kCullPer; ++e) {
        int64_t c = c0 + e;
        f[e] = 0;
        n[e] = 0;
        if (c < C) {
            uint32_t cntc = cell_start[c + 1] - cell_start[c];
            if (cntc) {
                int64_t i = c % dx, j = (c / dx) % dy, k = c / ((int64_t)dx * dy);
                if (cell_visible(i, j, k, v, W, H)) {
                    f[e] = 1;
                    n[e] = cntc;
                }
            }
        }
        sf += f[e];
        sn += n[e];
    }
    uint32_t ef, en, tf, tn;
    block_scan2(sf, sn, ef, en, tf, tn);
    uint32_t* fl = flag + (size_t)view * C;
    uint32_t* ct = cnt + (size_t)view * C;
#pragma unroll
    for (int e = 0; e < kCullPer; ++e) {
        int64_t c = c0 + e;
        if (c < C) {
            fl[c] = f[e] ? ef : ~0u;
            ct[c] = en;
        }
        ef += f[e];
        en += n[e];
    }
    if (threadIdx.x == 0) {
        bsum[((size_t)view * nb + blockIdx.x) * 2 + 0] = tf;
        bsum[((size_t)view * nb + blockIdx.x) * 2 + 1] = tn;
    }
}

// Phase 2: one block per view scans the block sums in place and writes the totals
// tot[view] = {visible non-empty cells, visible points}.
__global__ void __launch_bounds__(kCullThreads) k_cull_scan(uint32_t* __restrict__ bsum, int nb,
                                                            uint32_t* __restrict__ tot) {
    const int view = blockIdx.x;
    uint32_t* bs = bsum + (size_t)view * nb * 2;
    uint32_t carry_a = 0, carry_b = 0;
    for (int base = 0; base < nb; base += kCullThreads) {
        int b = base + threadIdx.x;
        uint32_t a = b < nb ? bs[2 * b] : 0, p = b < nb ? bs[2 * b + 1] : 0;
        uint32_t ea, eb, ta, tb;
        block_scan2(a, p, ea, eb, ta, tb);
        if (b < nb) {
            bs[2 * b] = carry_a + ea;
            bs[2 * b + 1] = carry_b + eb;
        }
        carry_a += ta;
        carry_b += tb;
    }
    if (threadIdx.x == 0) {
        tot[2 * view] = carry_a;
        tot[2 * view + 1] = carry_b;
    }
}

// Phase 3: compaction.  For the r-th visible cell of a view: vis_info[view][r] = its
// camera-space origin and (sorted position of its first point - visible points before it),
// vis_pref[view][r] = visible points before it; and chunk_cell[view][k] = r for every
// splat range k (kSplatChunk visible points) whose first point lies in this cell, so that
// the splat finds a range's cells without searching.
__global__ void k_cull_compact(const ViewDev* __restrict__ views, const uint32_t* __restrict__ flag,
                               const uint32_t* __restrict__ cnt, const uint32_t* __restrict__ bsum, int nb,
                               int64_t C, int dx, int dy, const uint32_t* __restrict__ cell_start,
                               float4* __restrict__ vis_info, uint32_t* __restrict__ vis_pref,
                               uint32_t* __restrict__ chunk_cell, size_t max_chunks) {
    const int view = blockIdx.y;
    int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= C) return;
    uint32_t f = flag[(size_t)view * C + c];
    if (f == ~0u) return;
    int b = (int)(c / kCullTile);
    const uint32_t* bs = bsum + ((size_t)view * nb + b) * 2;
    uint32_t r = bs[0] + f;
    const uint32_t pref = bs[1] + cnt[(size_t)view * C + c];
    float o[3];
    cell_cam(c % dx, (c / dx) % dy, c / ((int64_t)dx * dy), views[view], o);
    vis_info[(size_t)view * C + r] = make_float4(o[0], o[1], o[2], __uint_as_float(cell_start[c] - pref));
    vis_pref[(size_t)view * C + r] = pref;
    const uint32_t n = cell_start[c + 1] - cell_start[c];  // > 0: only non-empty cells are visible
    uint32_t* cc = chunk_cell + (size_t)view * max_chunks;
    for (uint32_t k = (pref + kSplatChunk - 1) / kSplatChunk; k <= (pref + n - 1) / kSplatChunk; ++k) cc[k] = r;
}

// ------------------------------------------------------------------ splat ----
//
// Warps work independently (no block barriers) through ranges of kSplatChunk consecutive
// visible points, the ranges of all views of the batch in one list.  For a range, lane l
// holds visible cell (first cell of the range) + l: its camera-space origin, the offset
// from visible-point index to sorted position and its point prefix, loaded from the
// compaction's tables.  The points are taken 32 x kSplatBatch at a time (a batch); a
// batch's cells are the lanes from the one holding its first point on, found with warp
// votes: when the whole batch lies in one cell (the common case) every lane takes that
// cell's data with warp-uniform shuffles, else each point compares its index with the
// prefixes of the few cells that start inside the batch.  A range whose points span more
// than 32 cells is processed 32 cells at a time.  Each lane keeps kSplatBatch points'
// offset loads in flight before projecting them.  The views' parameters are staged in
// shared memory once per block.

constexpr int kSplatBatch = 4;
constexpr int kSplatMaxViews = 64;  // views per launch (their parameters are staged in shared memory)

template <bool SOFT>
__global__ void __launch_bounds__(kSplatThreads, 4) k_splat(
    const ViewDev* __restrict__ views, int nviews, int64_t C, const float4* __restrict__ vis_info,
    const uint32_t* __restrict__ vis_pref, const uint32_t* __restrict__ tot, const float* __restrict__ ox,
    const float* __restrict__ oy, const float* __restrict__ oz, int W, int H, unsigned long long* __restrict__ keys,
    const uint32_t* __restrict__ rgbs, unsigned long long* __restrict__ acc, float scale,
    const uint32_t* __restrict__ chunk_cell, size_t max_chunks, uint32_t pos_base) {
    __shared__ ViewDev sv[kSplatMaxViews];
    for (int i = threadIdx.x; i < nviews * (int)(sizeof(ViewDev) / 4); i += blockDim.x)
        reinterpret_cast<uint32_t*>(sv)[i] = reinterpret_cast<const uint32_t*>(views)[i];
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const uint64_t warp0 = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    const float Wf = (float)W, Hf = (float)H;
    int view = 0;
    uint64_t first = 0;  // global index of the view's first range
    for (uint64_t g = warp0;; g += nwarps) {
        // the view of global range g (ranges of view 0 first, then view 1, ...)
        uint32_t nr = (tot[2 * view + 1] + kSplatChunk - 1) / kSplatChunk;
        while (g >= first + nr) {
            first += nr;
            if (++view == nviews) return;
            nr = (tot[2 * view + 1] + kSplatChunk - 1) / kSplatChunk;
        }
        const ViewDev& v = sv[view];
        const uint32_t nvc = tot[2 * view], npts = tot[2 * view + 1];
        const float4* vi = vis_info + (size_t)view * C;
        const uint32_t* vp = vis_pref + (size_t)view * C;
        unsigned long long* kv = keys + (size_t)view * W * H;
        const uint32_t rg = (uint32_t)(g - first);
        const uint32_t start = rg * kSplatChunk;
        const uint32_t end = min(start + (uint32_t)kSplatChunk, npts);
        uint32_t cb = chunk_cell[(size_t)view * max_chunks + rg];  // the cell holding point `start`
        for (uint32_t a = start; a < end;) {
            // lane l: visible cell cb + l
            const uint32_t k = cb + (uint32_t)lane;
            float4 info = make_float4(0.f, 0.f, 0.f, 0.f);
            uint32_t pref = 0xffffffffu;
            if (k < nvc) {
                info = vi[k];
                pref = vp[k];
            }
            // points [a, b) lie in these 32 cells
            const uint32_t b = min(end, cb + 32 < nvc ? vp[cb + 32] : 0xffffffffu);
            for (uint32_t e0 = a; e0 < b; e0 += 32 * kSplatBatch) {
                const uint32_t elast = min(e0 + 32 * kSplatBatch, b) - 1;
                // the lane of the cell holding e0, and the cells starting later in the batch
                const int cur = __popc(__ballot_sync(0xffffffffu, pref <= e0)) - 1;
                const uint32_t starts = __ballot_sync(0xffffffffu, pref > e0 && pref <= elast);
                float px[kSplatBatch], py[kSplatBatch], pz[kSplatBatch];
                uint32_t pos[kSplatBatch];
                int cl[kSplatBatch];
                const uint32_t off0 = __float_as_uint(__shfl_sync(0xffffffffu, info.w, cur));
#pragma unroll
                for (int t = 0; t < kSplatBatch; ++t) {
                    const uint32_t e = e0 + (uint32_t)(32 * t + lane);
                    cl[t] = cur;
                    uint32_t off = off0;
                    if (starts) {  // warp-uniform: some cell starts inside the batch
                        for (uint32_t m = starts; m; m &= m - 1) {
                            const int j = __ffs(m) - 1;
                            if (__shfl_sync(0xffffffffu, pref, j) <= e) cl[t] = j;
                        }
                        off = __float_as_uint(__shfl_sync(0xffffffffu, info.w, cl[t]));
                    }
                    pos[t] = e + off;
                    if (e <= elast) {
                        px[t] = ox[pos[t]];
                        py[t] = oy[pos[t]];
                        pz[t] = oz[pos[t]];
                    }
                }
                float c0u = __shfl_sync(0xffffffffu, info.x, cur), c1u = __shfl_sync(0xffffffffu, info.y, cur),
                      c2u = __shfl_sync(0xffffffffu, info.z, cur);
#pragma unroll
                for (int t = 0; t < kSplatBatch; ++t) {
                    float c0 = c0u, c1 = c1u, c2 = c2u;
                    if (starts) {
                        c0 = __shfl_sync(0xffffffffu, info.x, cl[t]);
                        c1 = __shfl_sync(0xffffffffu, info.y, cl[t]);
                        c2 = __shfl_sync(0xffffffffu, info.z, cl[t]);
                    }
                    if (e0 + (uint32_t)(32 * t + lane) > elast) continue;
                    const float cell_o[3] = {c0, c1, c2};
                    float p[3];
#pragma unroll
                    for (int r = 0; r < 3; ++r) {
                        float q = __fmaf_rn(v.Rf[3 * r + 2], pz[t], cell_o[r]);
                        q = __fmaf_rn(v.Rf[3 * r + 1], py[t], q);
                        p[r] = __fmaf_rn(v.Rf[3 * r + 0], px[t], q);
                    }
                    const float z = p[2];
                    if (!(z > v.znear && z < v.zfar)) continue;
                    const float u = __fadd_rn(__fdiv_rn(__fmul_rn(v.fx, p[0]), z), v.cx);
                    const float w = __fadd_rn(__fdiv_rn(__fmul_rn(v.fy, p[1]), z), v.cy);
                    if (!(u >= 0.0f && u < Wf && w >= 0.0f && w < Hf)) continue;
                    const int64_t pix = (int64_t)floorf(w) * W + (int64_t)floorf(u);
                    if (!SOFT) {
                        const unsigned long long key = ((unsigned long long)__float_as_uint(z) << 32) | (pos[t] + pos_base);
                        atomicMin(&kv[pix], key);
                    } else {
                        const unsigned long long front = kv[pix];
                        if (front == kEmpty || !(z <= __fmul_rn(__uint_as_float((uint32_t)(front >> 32)), scale))) continue;
                        const uint32_t col = rgbs[pos[t]];
                        unsigned long long* ac = acc + 2 * ((size_t)view * W * H + pix);
                        atomicAdd(ac, ((unsigned long long)(col & 255u) << 32) | ((col >> 8) & 255u));
                        atomicAdd(ac + 1, ((unsigned long long)((col >> 16) & 255u) << 32) | 1ull);
                    }
                }
            }
            a = b;
            cb += 32;
        }
    }
}

__global__ void k_fill_u64(unsigned long long* __restrict__ p, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        p[i] = kEmpty;
}

// --------------------------------------------------- resolve + min-pool pyramid ----

// One 64x64 tile: keys -> depth (+inf empty) and rgba (r | g<<8 | b<<16 | A<<24), keys
// reset to empty for the next frame, then every min-pool level of the tile (kernel 2x2,
// stride 2; level sizes ceil(W/2^l) x ceil(H/2^l); pixels outside the image count as
// +inf, so each level pixel is the minimum over its clipped 2^l x 2^l block).  With the
// soft z-buffer's sums (acc non-null) the colour is their per-channel integer mean
// (sum + n/2) / n, and the sums are reset to zero.
__global__ void __launch_bounds__(256) k_resolve_pyramid(
    unsigned long long* __restrict__ keys, const uint32_t* __restrict__ rgbs, int W, int H, int nlev,
    float* __restrict__ depth, uint32_t* __restrict__ rgba, float* __restrict__ pyr, size_t pyr_stride,
    unsigned long long* __restrict__ acc, uint32_t pos_base, uint32_t n_local) {
    __shared__ float s[64][65];
    __shared__ float t[32][33];
    const int view = blockIdx.z;
    const size_t P = (size_t)W * H;
    unsigned long long* kv = keys + view * P;
    float* dv = depth + view * P;
    uint32_t* cv = rgba + view * P;
    const int x = threadIdx.x & 63, y0 = threadIdx.x >> 6;
    const int gx = blockIdx.x * 64 + x;
#pragma unroll 4
    for (int i = 0; i < 16; ++i) {
        const int y = y0 + 4 * i;
        const int gy = blockIdx.y * 64 + y;
        float d = INFINITY;
        if (gx < W && gy < H) {
            const size_t q = (size_t)gy * W + gx;
            const unsigned long long key = kv[q];
            uint32_t col = 0;
            if (key != kEmpty) {
                d = __uint_as_float((uint32_t)(key >> 32));
                // a cloud shard colours only its own points; another shard's front point
                // leaves the colour (and this buffer's A bit) zero
                const uint32_t idx = (uint32_t)key - pos_base;
                col = idx < n_local ? (rgbs[idx] & 0x00ffffffu) | (1u << 24) : 0u;
                kv[q] = kEmpty;
                if (acc) {
                    ulonglong2* a = reinterpret_cast<ulonglong2*>(acc) + view * P + q;
                    const ulonglong2 sums = *a;
                    const unsigned long long n = sums.y & 0xffffffffull;
                    if (n) {
                        const unsigned long long r = ((sums.x >> 32) + n / 2) / n, g = ((sums.x & 0xffffffffull) + n / 2) / n,
                                                 b = ((sums.y >> 32) + n / 2) / n;
                        col = (uint32_t)r | ((uint32_t)g << 8) | ((uint32_t)b << 16) | (1u << 24);
                    }
                    *a = make_ulonglong2(0ull, 0ull);
                }
            }
            dv[q] = d;
            cv[q] = col;
        }
        s[y][x] = d;
    }
    __syncthreads();
    float* lev = pyr + view * pyr_stride;
    int Wl = W, Hl = H;
    for (int l = 1; l <= nlev; ++l) {
        const int T = 64 >> l;                  // tile side at this level
        Wl = (Wl + 1) >> 1;
        Hl = (Hl + 1) >> 1;
        // read level l-1 from s (l odd) or t (l even), write level l into the other
        for (int idx = threadIdx.x; idx < T * T; idx += 256) {
            const int lx = idx % T, ly = idx / T;
            float m;
            if (l & 1) {
                m = fminf(fminf(s[2 * ly][2 * lx], s[2 * ly][2 * lx + 1]),
                          fminf(s[2 * ly + 1][2 * lx], s[2 * ly + 1][2 * lx + 1]));
                t[ly][lx] = m;
            } else {
                m = fminf(fminf(t[2 * ly][2 * lx], t[2 * ly][2 * lx + 1]),
                          fminf(t[2 * ly + 1][2 * lx], t[2 * ly + 1][2 * lx + 1]));
                s[ly][lx] = m;
            }
            const int ox_ = blockIdx.x * T + lx, oy_ = blockIdx.y * T + ly;
            if (ox_ < Wl && oy_ < Hl) lev[(size_t)oy_ * Wl + ox_] = m;
        }
        lev += (size_t)Wl * Hl;
        __syncthreads();
    }
}

// ------------------------------------------------------------------ upsample ----

struct UpArgs {
    const ViewDev* views;
    const float* Mf;     // fine min-pooled level (level 0: the depth image)
    const float* Mc;     // coarse min-pooled level
    const float* Uc;     // coarse upsampled level (the coarsest: Mc itself)
    float* Uf;           // fine upsampled level (levels > 0)
    size_t f_stride, c_stride, uc_stride, uf_stride;  // per-view strides (floats)
    int Wf, Hf, Wc, Hc;
    int fill;            // non-final level: fill empty pixels by interpolation
    // final level only
    const uint32_t* rgba;
    void* unet_in;       // NHWC: 8 FP32 channels (kind 0) or 16 BF16 channels (kind 1)
    int kind;            // 0 = FP32, 1 = BF16, 2 = none
    float* u0;           // kept depth tap (nullable)
};

// 32 bytes to a 32-byte-aligned global address in one store (a whole L2 sector).
__device__ __forceinline__ void st_sector(void* dst, uint32_t w0, uint32_t w1, uint32_t w2, uint32_t w3, uint32_t w4,
                                          uint32_t w5, uint32_t w6, uint32_t w7) {
    asm volatile("st.global.v8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"l"(dst), "r"(w0), "r"(w1), "r"(w2),
                 "r"(w3), "r"(w4), "r"(w5), "r"(w6), "r"(w7)
                 : "memory");
}

// One pixel of the network input: 8 FP32 channels or 16 BF16 channels (32 bytes in both
// layouts), written as one sector.
__device__ __forceinline__ void store_unet_in(void* base, int kind, size_t q, float r, float g, float b,
                                              float d, float a) {
    if (kind == 0) {
        st_sector(static_cast<float*>(base) + q * 8, __float_as_uint(r), __float_as_uint(g), __float_as_uint(b),
                  __float_as_uint(d), __float_as_uint(a), 0u, 0u, 0u);
    } else if (kind == 1) {
        __nv_bfloat162 v0 = __floats2bfloat162_rn(r, g), v1 = __floats2bfloat162_rn(b, d);
        __nv_bfloat162 v2 = __floats2bfloat162_rn(a, 0.f);
        st_sector(static_cast<uint4*>(base) + 2 * q, *reinterpret_cast<uint32_t*>(&v0), *reinterpret_cast<uint32_t*>(&v1),
                  *reinterpret_cast<uint32_t*>(&v2), 0u, 0u, 0u, 0u, 0u);
    }
}

__device__ __forceinline__ void pack_pixel(const UpArgs& a, const ViewDev& v, int view, size_t q, bool keep, float m) {
    const size_t P = (size_t)a.Wf * a.Hf;
    if (a.u0) a.u0[view * P + q] = keep ? m : INFINITY;
    if (a.kind == 2) return;
    if (keep) {
        const uint32_t c = a.rgba[view * P + q];
        store_unet_in(a.unet_in, a.kind, view * P + q, __fdiv_rn((float)(c & 255u), 255.0f),
                      __fdiv_rn((float)((c >> 8) & 255u), 255.0f), __fdiv_rn((float)((c >> 16) & 255u), 255.0f),
                      __fdiv_rn(m, v.zfar), 1.0f);
    } else {
        store_unet_in(a.unet_in, a.kind, view * P + q, 0.f, 0.f, 0.f, 0.f, 0.f);
    }
}

// One thread per coarse pixel p of a 32x8 tile; the coarse levels are staged with a
// one-pixel clamped halo, so replicated borders come for free.
__global__ void __launch_bounds__(256) k_upsample(const UpArgs a) {
    __shared__ float sM[10][34], sU[10][34];
    const int view = blockIdx.z;
    const ViewDev v = a.views[view];
    const float* Mc = a.Mc + view * a.c_stride;
    const float* Uc = a.Uc + view * a.uc_stride;
    const int tx0 = blockIdx.x * 32, ty0 = blockIdx.y * 8;
    for (int idx = threadIdx.x; idx < 340; idx += 256) {
        const int hx = idx % 34, hy = idx / 34;
        const int gx = min(max(tx0 + hx - 1, 0), a.Wc - 1), gy = min(max(ty0 + hy - 1, 0), a.Hc - 1);
        sM[hy][hx] = Mc[(size_t)gy * a.Wc + gx];
        sU[hy][hx] = Uc[(size_t)gy * a.Wc + gx];
    }
    __syncthreads();
    const int lx = threadIdx.x & 31, ly = threadIdx.x >> 5;
    const int cx = tx0 + lx, cy = ty0 + ly;
    if (cx >= a.Wc || cy >= a.Hc) return;
    const int sx = lx + 1, sy = ly + 1;
    const float d = sM[sy][sx];
    bool edge = false;
    if (d != INFINITY) {
        const float nb[4] = {sM[sy][sx - 1], sM[sy][sx + 1], sM[sy - 1][sx], sM[sy + 1][sx]};
        float te[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) te[e] = nb[e] == INFINITY ? 0.0f : __fsub_rn(nb[e], d);
        const float lap = __fadd_rn(__fadd_rn(te[0], te[1]), __fadd_rn(te[2], te[3]));
        edge = fabsf(lap) > __fmul_rn(kEdgeRel, d);
    }
    float ref;
    if (edge) {
        ref = INFINITY;
#pragma unroll
        for (int b = -1; b <= 1; ++b)
#pragma unroll
            for (int c = -1; c <= 1; ++c) ref = fminf(ref, sU[sy + b][sx + c]);
    } else {
        ref = sU[sy][sx];
    }
    const float thr = __fmul_rn(ref, v.S);
    const float* Mf = a.Mf + view * a.f_stride;
#pragma unroll
    for (int b = 0; b < 2; ++b)
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            const int fx = 2 * cx + c, fy = 2 * cy + b;
            if (fx >= a.Wf || fy >= a.Hf) continue;
            const size_t q = (size_t)fy * a.Wf + fx;
            const float m = Mf[q];
            const bool keep = (m <= thr) && (m != INFINITY);
            if (a.Uf) {
                float val = keep ? m : INFINITY;
                if (!keep && a.fill) {
                    const int fxs = c ? sx + 1 : sx - 1;   // far tap in x (clamped by the halo)
                    const int fys = b ? sy + 1 : sy - 1;
                    const float tap[4] = {sU[sy][sx], sU[sy][fxs], sU[fys][sx], sU[fys][fxs]};
                    const float wt[4] = {0.5625f, 0.1875f, 0.1875f, 0.0625f};
                    float num = 0.0f, den = 0.0f;
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        if (tap[e] == INFINITY) continue;
                        num = __fadd_rn(num, __fmul_rn(wt[e], tap[e]));
                        den = __fadd_rn(den, wt[e]);
                    }
                    if (den > 0.0f) val = __fdiv_rn(num, den);
                }
                a.Uf[view * a.uf_stride + q] = val;
            } else {
                pack_pixel(a, v, view, q, keep, m);
            }
        }
}

// n_levels = 0: no filter, every filled pixel is kept.
__global__ void k_pack_direct(const UpArgs a, int B) {
    const size_t P = (size_t)a.Wf * a.Hf;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < P * B; i += (size_t)gridDim.x * blockDim.x) {
        const int view = (int)(i / P);
        const size_t q = i % P;
        const float m = a.Mf[view * a.f_stride + q];
        pack_pixel(a, a.views[view], view, q, m != INFINITY, m);
    }
}

__global__ void k_extract5(const void* in, int kind, float* out, int64_t npx) {
    int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q >= npx) return;
    for (int c = 0; c < 5; ++c) {
        float v;
        if (kind == 0) v = static_cast<const float*>(in)[q * 8 + c];
        else v = __bfloat162float(static_cast<const __nv_bfloat16*>(in)[q * 16 + c]);
        out[q * 5 + c] = v;
    }
}

}  // namespace

size_t splat_max_chunks(uint64_t npoints) { return (size_t)(npoints / kSplatChunk) + 2; }

int cull_blocks(int64_t ncells) { return (int)((ncells + kCullTile - 1) / kCullTile); }

void launch_cull(const lnr_ctx* c, Workspace& ws, cudaStream_t st) {
    const int nb = cull_blocks(c->ncells);
    dim3 g1(nb, ws.B);
    k_cull_block<<<g1, kCullThreads, 0, st>>>(ws.view.as<ViewDev>(), c->cell_start.as<uint32_t>(), c->dims[0],
                                              c->dims[1], c->dims[2], c->ncells, ws.W, ws.H,
                                              ws.cull_flag.as<uint32_t>(), ws.cull_cnt.as<uint32_t>(),
                                              ws.cull_bsum.as<uint32_t>(), nb);
    count_launch();
    k_cull_scan<<<ws.B, kCullThreads, 0, st>>>(ws.cull_bsum.as<uint32_t>(), nb, ws.vis_tot.as<uint32_t>());
    count_launch();
    dim3 g3((unsigned)((c->ncells + 255) / 256), ws.B);
    k_cull_compact<<<g3, 256, 0, st>>>(ws.view.as<ViewDev>(), ws.cull_flag.as<uint32_t>(), ws.cull_cnt.as<uint32_t>(),
                                       ws.cull_bsum.as<uint32_t>(), nb, c->ncells, c->dims[0], c->dims[1],
                                       c->cell_start.as<uint32_t>(), ws.vis_info.as<float4>(), ws.vis_pref.as<uint32_t>(),
                                       ws.chunk_cell.as<uint32_t>(), splat_max_chunks(c->n));
    count_launch();
}

// Grid of the splat: as many blocks as fit on the GPU at once (the warps stride through the
// ranges of every view).
static int splat_blocks(const lnr_ctx* c, bool soft) {
    static int per_sm[2] = {0, 0};
    if (!per_sm[soft]) {
        int n = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, soft ? k_splat<true> : k_splat<false>, kSplatThreads, 0);
        per_sm[soft] = std::max(1, n);
    }
    return c->num_sms * per_sm[soft];
}

// One launch per group of up to kSplatMaxViews views.
template <bool SOFT>
static void splat_views(const lnr_ctx* c, Workspace& ws, cudaStream_t st, float scale) {
    const size_t P = (size_t)ws.W * ws.H, mc = splat_max_chunks(c->n);
    for (int v0 = 0; v0 < ws.B; v0 += kSplatMaxViews) {
        const int nv = std::min(kSplatMaxViews, ws.B - v0);
        k_splat<SOFT><<<splat_blocks(c, SOFT), kSplatThreads, 0, st>>>(
            ws.view.as<ViewDev>() + v0, nv, c->ncells, ws.vis_info.as<float4>() + (size_t)v0 * c->ncells,
            ws.vis_pref.as<uint32_t>() + (size_t)v0 * c->ncells,
            ws.vis_tot.as<uint32_t>() + 2 * v0, c->ox.as<float>(), c->oy.as<float>(), c->oz.as<float>(), ws.W, ws.H,
            ws.keys.as<unsigned long long>() + v0 * P, SOFT ? c->rgbs.as<uint32_t>() : nullptr,
            SOFT ? ws.soft_acc.as<unsigned long long>() + 2 * v0 * P : nullptr, scale,
            ws.chunk_cell.as<uint32_t>() + (size_t)v0 * mc, mc, SOFT ? 0u : c->shard_base);
        count_launch();
    }
}

void launch_splat(const lnr_ctx* c, Workspace& ws, cudaStream_t st) { splat_views<false>(c, ws, st, 1.0f); }

// Second pass of the soft z-buffer (after launch_splat has finished the keys).
void launch_splat_soft(const lnr_ctx* c, Workspace& ws, cudaStream_t st) {
    if (ws.soft_dirty) {  // fresh allocation: zero every sum once; the resolve re-zeroes what it reads
        cudaMemsetAsync(ws.soft_acc.p, 0, ws.soft_acc.bytes, st);
        ws.soft_dirty = false;
    }
    splat_views<true>(c, ws, st, 1.0f + c->soft_rel);
}

// ------------------------------------------------------- atomic throughput probe ----

// The output function of splitmix64 (Steele, Lea and Flood, OOPSLA 2014): a bijective mix of
// 64-bit integers, here only a source of scattered keys and depths.
__device__ __forceinline__ uint64_t mix64(uint64_t x) {
    x ^= x >> 30;
    x *= 0xbf58476d1ce4e5b9ull;
    x ^= x >> 27;
    x *= 0x94d049bb133111ebull;
    return x ^ (x >> 31);
}

// The splat's z-buffer update in isolation: n_ops 64-bit atomicMin of splat-shaped keys
// (depth bits << 32 | index) into n_slots keys.  coherent = 1: operation i updates key
// i mod n_slots, neighbouring threads neighbouring keys (as cell-sorted points do);
// coherent = 0: a hashed key.
__global__ void k_atomic_rate(unsigned long long* __restrict__ keys, uint64_t n_slots, uint64_t n_ops, int coherent) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n_ops; i += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t h = mix64(i);
        const uint64_t j = (coherent ? i : h) % n_slots;
        atomicMin(&keys[j], ((unsigned long long)(uint32_t)(h >> 34) << 32) | (uint32_t)i);
    }
}

cudaError_t probe_atomic_rate(uint64_t n_slots, uint64_t n_ops, int coherent, int num_sms, cudaStream_t st,
                              double* ops_per_s) {
    unsigned long long* keys = nullptr;
    cudaError_t e = cudaMalloc(&keys, n_slots * sizeof(unsigned long long));
    if (e != cudaSuccess) return e;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const unsigned grid = (unsigned)std::max(1, num_sms) * 8;  // the splat's grid for 8 views
    float best = 1e30f;
    for (int r = 0; r < 6 && e == cudaSuccess; ++r) {  // run 0 warms up; the fastest later run counts
        k_fill_u64<<<1024, 256, 0, st>>>(keys, n_slots);
        cudaEventRecord(e0, st);
        k_atomic_rate<<<grid, 256, 0, st>>>(keys, n_slots, n_ops, coherent);
        cudaEventRecord(e1, st);
        e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e == cudaSuccess && r > 0) best = std::min(best, ms);
    }
    if (e == cudaSuccess) e = cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(keys);
    if (e == cudaSuccess) *ops_per_s = (double)n_ops / (best * 1e-3);
    return e;
}

void launch_clear_keys(Workspace& ws, cudaStream_t st) {
    // the whole allocation: a tap that stopped after the splat may have left keys of an
    // earlier, larger frame behind
    size_t n = ws.keys.bytes / 8;
    k_fill_u64<<<1024, 256, 0, st>>>(ws.keys.as<unsigned long long>(), n);
    count_launch();
    ws.keys_dirty = false;
}

size_t pyramid_offset(int W, int H, int l) {
    size_t off = 0;
    for (int k = 1; k < l; ++k) {
        W = (W + 1) / 2;
        H = (H + 1) / 2;
        off += (size_t)W * H;
    }
    return off;
}
size_t pyramid_floats(int W, int H, int nlev) { return pyramid_offset(W, H, nlev + 1) + 1; }

void launch_resolve_pyramid(const lnr_ctx* c, Workspace& ws, cudaStream_t st) {
    dim3 g((ws.W + 63) / 64, (ws.H + 63) / 64, ws.B);
    k_resolve_pyramid<<<g, 256, 0, st>>>(ws.keys.as<unsigned long long>(), c->rgbs.as<uint32_t>(), ws.W, ws.H,
                                         ws.nlev, ws.depth.as<float>(), ws.rgba.as<uint32_t>(), ws.pyr_m.as<float>(),
                                         pyramid_floats(ws.W, ws.H, ws.nlev),
                                         c->soft_rel > 0.0f ? ws.soft_acc.as<unsigned long long>() : nullptr, c->shard_base,
                                         (uint32_t)c->n);
    count_launch();
}

void launch_upsample(const lnr_ctx* c, Workspace& ws, int l, void* unet_in, int kind, bool write_u0,
                     cudaStream_t st) {
    (void)c;
    const size_t P = (size_t)ws.W * ws.H;
    const size_t pstride = pyramid_floats(ws.W, ws.H, ws.nlev);
    UpArgs a{};
    a.views = ws.view.as<ViewDev>();
    a.rgba = ws.rgba.as<uint32_t>();
    a.unet_in = unet_in;
    a.kind = kind;
    a.u0 = write_u0 ? ws.u0.as<float>() : nullptr;
    int Wl = ws.W, Hl = ws.H;
    for (int k = 0; k < l; ++k) { Wl = (Wl + 1) / 2; Hl = (Hl + 1) / 2; }
    a.Wf = Wl; a.Hf = Hl;
    a.Wc = (Wl + 1) / 2; a.Hc = (Hl + 1) / 2;
    if (ws.nlev == 0) {
        a.Mf = ws.depth.as<float>();
        a.f_stride = P;
        k_pack_direct<<<2048, 256, 0, st>>>(a, ws.B);
        count_launch();
        return;
    }
    if (l == 0) { a.Mf = ws.depth.as<float>(); a.f_stride = P; }
    else { a.Mf = ws.pyr_m.as<float>() + pyramid_offset(ws.W, ws.H, l); a.f_stride = pstride; }
    a.Mc = ws.pyr_m.as<float>() + pyramid_offset(ws.W, ws.H, l + 1);
    a.c_stride = pstride;
    if (l + 1 == ws.nlev) { a.Uc = a.Mc; a.uc_stride = pstride; }
    else { a.Uc = ws.pyr_u.as<float>() + pyramid_offset(ws.W, ws.H, l + 1); a.uc_stride = pstride; }
    if (l > 0) { a.Uf = ws.pyr_u.as<float>() + pyramid_offset(ws.W, ws.H, l); a.uf_stride = pstride; a.fill = 1; }
    dim3 g((a.Wc + 31) / 32, (a.Hc + 7) / 8, ws.B);
    k_upsample<<<g, 256, 0, st>>>(a);
    count_launch();
}

// Network input of one synthetic training pair (Sec. 3, "Training Data Generation"): per pixel from the
// raw depth / colour of the projection, the kept depth of the filter and the ground-truth
// image gt (FP32 RGB).  filtered input: (gt * A^s, z / zfar, A^s) with A^s the kept mask;
// unfiltered input: every filled pixel, kept ones (foreground) with gt, filtered-out ones
// (background) with the projected colour / 255, D = z / zfar, A = 1; zero elsewhere.
__global__ void k_training_input(const float* __restrict__ depth, const uint32_t* __restrict__ rgba,
                                 const float* __restrict__ kept, const float* __restrict__ gt, float zfar,
                                 int unfiltered, int64_t npx, float* __restrict__ out) {
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < npx; q += (int64_t)gridDim.x * blockDim.x) {
        const float z = depth[q], zk = kept[q];
        const bool filled = z != INFINITY, fg = zk != INFINITY;
        float r = 0.f, g = 0.f, b = 0.f, d = 0.f, a = 0.f;
        if (fg || (unfiltered && filled)) {
            if (fg) {
                r = gt[3 * q];
                g = gt[3 * q + 1];
                b = gt[3 * q + 2];
            } else {
                const uint32_t c = rgba[q];
                r = __fdiv_rn((float)(c & 255u), 255.0f);
                g = __fdiv_rn((float)((c >> 8) & 255u), 255.0f);
                b = __fdiv_rn((float)((c >> 16) & 255u), 255.0f);
            }
            d = __fdiv_rn(z, zfar);
            a = 1.0f;
        }
        float* o = out + 5 * q;
        o[0] = r;
        o[1] = g;
        o[2] = b;
        o[3] = d;
        o[4] = a;
    }
}

void launch_training_input(const Workspace& ws, const float* gt, float zfar, int unfiltered, float* out,
                           cudaStream_t st) {
    const int64_t npx = (int64_t)ws.W * ws.H;
    k_training_input<<<(unsigned)std::min<int64_t>((npx + 255) / 256, 8192), 256, 0, st>>>(
        ws.depth.as<float>(), ws.rgba.as<uint32_t>(), ws.u0.as<float>(), gt, zfar, unfiltered, npx, out);
}

void launch_unet_in_extract(const void* unet_in, int kind, float* out5, int64_t npx, cudaStream_t st) {
    k_extract5<<<(unsigned)((npx + 255) / 256), 256, 0, st>>>(unet_in, kind, out5, npx);
}

}  // namespace lnr

// ============================================ depth filter into a static scratch array ==
//
// lnr_filter_static runs the depth-guided filter on a caller's device depth image without
// allocating any memory: its pyramid lives in the file-scope array below, which every GPU
// that loads the library holds until the process exits.  Every call overwrites the whole
// part of the array it uses, so nothing has to be cleared between calls; two calls whose
// work overlaps on the GPU (different streams, no ordering between them) share the array
// and race.

namespace lnr {
namespace {

// 3 Mi floats (12 MiB): one view parameter block, the min-pooled levels M1..Mn and the
// upsampled levels U1..U(n-1).  A 2560 x 1440 image with 6 levels needs about 2.5 Mi.
constexpr size_t kStaticFilterFloats = size_t(3) << 20;
constexpr size_t kStaticViewFloats = 64;  // ViewDev block at the front (256-byte aligned)
static_assert(sizeof(ViewDev) <= kStaticViewFloats * sizeof(float), "view block");

__device__ __align__(256) float g_filter_scratch[kStaticFilterFloats];

__global__ void k_static_view(ViewDev* v, float S, float zfar) {
    ViewDev d{};
    d.S = S;
    d.zfar = zfar;
    *v = d;
}

// Min-pool pyramid of a depth image, one 64 x 64 tile per block (the same levels as the
// resolve kernel computes from z-buffer keys).
__global__ void __launch_bounds__(256) k_pyramid_from_depth(const float* __restrict__ depth, int W, int H, int nlev,
                                                            float* __restrict__ pyr) {
    __shared__ float s[64][65];
    __shared__ float t[32][33];
    const int x = threadIdx.x & 63, y0 = threadIdx.x >> 6;
    const int gx = blockIdx.x * 64 + x;
    for (int i = 0; i < 16; ++i) {
        const int y = y0 + 4 * i, gy = blockIdx.y * 64 + y;
        s[y][x] = (gx < W && gy < H) ? depth[(size_t)gy * W + gx] : INFINITY;
    }
    __syncthreads();
    float* lev = pyr;
    int Wl = W, Hl = H;
    for (int l = 1; l <= nlev; ++l) {
        const int T = 64 >> l;
        Wl = (Wl + 1) >> 1;
        Hl = (Hl + 1) >> 1;
        for (int idx = threadIdx.x; idx < T * T; idx += 256) {
            const int lx = idx % T, ly = idx / T;
            float m;
            if (l & 1) {
                m = fminf(fminf(s[2 * ly][2 * lx], s[2 * ly][2 * lx + 1]), fminf(s[2 * ly + 1][2 * lx], s[2 * ly + 1][2 * lx + 1]));
                t[ly][lx] = m;
            } else {
                m = fminf(fminf(t[2 * ly][2 * lx], t[2 * ly][2 * lx + 1]), fminf(t[2 * ly + 1][2 * lx], t[2 * ly + 1][2 * lx + 1]));
                s[ly][lx] = m;
            }
            const int ox_ = blockIdx.x * T + lx, oy_ = blockIdx.y * T + ly;
            if (ox_ < Wl && oy_ < Hl) lev[(size_t)oy_ * Wl + ox_] = m;
        }
        lev += (size_t)Wl * Hl;
        __syncthreads();
    }
}

float* g_static_ptr[64] = {nullptr};
std::mutex g_static_mu;

}  // namespace
}  // namespace lnr

extern "C" lnr_status lnr_filter_static(const float* d_depth, int W, int H, int n_levels, float fs, float* d_kept,
                                        void* cuda_stream) {
    using namespace lnr;
    if (!d_depth || !d_kept || W < 1 || H < 1 || (int64_t)W * H > (1ll << 30)) return LNR_E_ARG;
    int maxl = 0;
    while ((2 << maxl) <= std::min(W, H)) ++maxl;
    if (n_levels < 0 || n_levels > std::min(maxl, kMaxLevels) || !(fs >= 0.0f)) return LNR_E_ARG;
    const size_t lev = pyramid_floats(W, H, n_levels);
    if (kStaticViewFloats + 2 * lev > kStaticFilterFloats) return LNR_E_ARG;  // beyond the static capacity
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return LNR_E_CUDA;
    float* scratch;
    {
        std::lock_guard<std::mutex> g(g_static_mu);
        if (!g_static_ptr[dev]) {
            void* ptr = nullptr;
            if (cudaGetSymbolAddress(&ptr, g_filter_scratch) != cudaSuccess || !ptr) return LNR_E_CUDA;
            g_static_ptr[dev] = static_cast<float*>(ptr);
        }
        scratch = g_static_ptr[dev];
    }
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    ViewDev* view = reinterpret_cast<ViewDev*>(scratch);
    float* M = scratch + kStaticViewFloats;
    float* U = M + lev;
    const float S = 1.0f + fs * 0.05f;  // keep scale, as for lnr_render
    k_static_view<<<1, 1, 0, st>>>(view, S, 1.0f);
    UpArgs a{};
    a.views = view;
    a.kind = 2;
    if (n_levels == 0) {
        a.Mf = d_depth;
        a.f_stride = (size_t)W * H;
        a.Wf = W;
        a.Hf = H;
        a.u0 = d_kept;
        k_pack_direct<<<2048, 256, 0, st>>>(a, 1);
        return cudaGetLastError() == cudaSuccess ? LNR_OK : LNR_E_CUDA;
    }
    dim3 g((W + 63) / 64, (H + 63) / 64, 1);
    k_pyramid_from_depth<<<g, 256, 0, st>>>(d_depth, W, H, n_levels, M);
    for (int l = n_levels - 1; l >= 0; --l) {
        int Wl = W, Hl = H;
        for (int k = 0; k < l; ++k) { Wl = (Wl + 1) / 2; Hl = (Hl + 1) / 2; }
        UpArgs u = a;
        u.Wf = Wl; u.Hf = Hl;
        u.Wc = (Wl + 1) / 2; u.Hc = (Hl + 1) / 2;
        u.Mf = l == 0 ? d_depth : M + pyramid_offset(W, H, l);
        u.Mc = M + pyramid_offset(W, H, l + 1);
        u.Uc = (l + 1 == n_levels) ? u.Mc : U + pyramid_offset(W, H, l + 1);
        u.f_stride = u.c_stride = u.uc_stride = u.uf_stride = 0;
        if (l > 0) { u.Uf = U + pyramid_offset(W, H, l); u.fill = 1; }
        else { u.Uf = nullptr; u.u0 = d_kept; u.fill = 0; }
        dim3 gu((u.Wc + 31) / 32, (u.Hc + 7) / 8, 1);
        k_upsample<<<gu, 256, 0, st>>>(u);
    }
    return cudaGetLastError() == cudaSuccess ? LNR_OK : LNR_E_CUDA;
}
