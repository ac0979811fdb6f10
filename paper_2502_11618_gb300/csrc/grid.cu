// Uniform-grid build on the device (Sec. 1; Sec. 3, "Point Cloud Projection"): the only
// preprocessing of the cloud.  Points are counting-sorted by linear cell id, stably, by
// a least-significant-digit radix sort on 8-bit digits; each sorted point then stores its
// FP32 offset to its cell's FP64 origin and its packed colour.
//
// Compiled with --fmad=false: every FP64 step below is one IEEE operation, rounded on
// its own, so the offsets match an FP64 host computation bit for bit.
#include "lnr_internal.h"

namespace lnr {
namespace {

constexpr int kThreads = 256;
constexpr int kItems = 16;
constexpr int kTile = kThreads * kItems;  // keys per radix tile
constexpr int kWarps = kThreads / 32;

__global__ void k_bbox_partial(const double* __restrict__ xyz, uint64_t n, double* __restrict__ part) {
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n;
         i += (uint64_t)gridDim.x * blockDim.x) {
        for (int a = 0; a < 3; ++a) {
            double v = xyz[3 * i + a];
            lo[a] = fmin(lo[a], v);
            hi[a] = fmax(hi[a], v);
        }
    }
    __shared__ double s[6][kThreads];
    for (int a = 0; a < 3; ++a) {
        s[a][threadIdx.x] = lo[a];
        s[3 + a][threadIdx.x] = hi[a];
    }
    __syncthreads();
    for (int w = kThreads / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w)
            for (int a = 0; a < 3; ++a) {
                s[a][threadIdx.x] = fmin(s[a][threadIdx.x], s[a][threadIdx.x + w]);
                s[3 + a][threadIdx.x] = fmax(s[3 + a][threadIdx.x], s[3 + a][threadIdx.x + w]);
            }
        __syncthreads();
    }
    if (threadIdx.x < 6) part[blockIdx.x * 6 + threadIdx.x] = s[threadIdx.x][0];
}

__global__ void k_cell_id(const double* __restrict__ xyz, uint64_t n, double g0x, double g0y,
                          double g0z, double cell, int dx, int dy, int dz, uint32_t* __restrict__ cid,
                          uint32_t* __restrict__ counts) {
    uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double g0[3] = {g0x, g0y, g0z};
    const int dim[3] = {dx, dy, dz};
    int64_t ijk[3];
    for (int a = 0; a < 3; ++a) {
        double f = floor(__ddiv_rn(__dsub_rn(xyz[3 * i + a], g0[a]), cell));
        f = fmax(f, 0.0);
        f = fmin(f, (double)(dim[a] - 1));
        ijk[a] = (int64_t)f;
    }
    uint32_t c = (uint32_t)((ijk[2] * dy + ijk[1]) * dx + ijk[0]);
    cid[i] = c;
    atomicAdd(&counts[c], 1u);
}

// ---- device-wide exclusive scan of uint32 (3 phases, recursive on the block sums) ----

constexpr int kScanItems = 8;
constexpr int kScanTile = kThreads * kScanItems;

__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t* total) {
    __shared__ uint32_t warp_sum[kWarps];
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t x = v;
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_sum[warp] = x;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = lane < kWarps ? warp_sum[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < kWarps) warp_sum[lane] = w;
    }
    __syncthreads();
    uint32_t base = warp ? warp_sum[warp - 1] : 0;
    *total = warp_sum[kWarps - 1];
    __syncthreads();
    return base + x - v;
}

__global__ void k_scan_reduce(const uint32_t* __restrict__ in, uint64_t n, uint32_t* __restrict__ bsum) {
    uint64_t base = (uint64_t)blockIdx.x * kScanTile;
    uint32_t s = 0;
    for (int k = 0; k < kScanItems; ++k) {
        uint64_t i = base + (uint64_t)k * kThreads + threadIdx.x;
        if (i < n) s += in[i];
    }
    uint32_t tot;
    block_exclusive_scan(s, &tot);
    if (threadIdx.x == 0) bsum[blockIdx.x] = tot;
}

__global__ void k_scan_apply(const uint32_t* __restrict__ in, uint64_t n, uint32_t* __restrict__ out,
                             const uint32_t* __restrict__ boff) {
    uint64_t base = (uint64_t)blockIdx.x * kScanTile + (uint64_t)threadIdx.x * kScanItems;
    uint32_t v[kScanItems];
    uint32_t s = 0;
    for (int k = 0; k < kScanItems; ++k) {
        uint64_t i = base + k;
        v[k] = i < n ? in[i] : 0;
        s += v[k];
    }
    uint32_t tot;
    uint32_t run = block_exclusive_scan(s, &tot) + (boff ? boff[blockIdx.x] : 0);
    for (int k = 0; k < kScanItems; ++k) {
        uint64_t i = base + k;
        if (i < n) out[i] = run;
        run += v[k];
    }
}

// Exclusive scan of n values; tmp must hold scan_tmp_words(n) words.
size_t scan_tmp_words(uint64_t n) {
    size_t w = 0;
    while (n > (uint64_t)kScanTile) {
        n = (n + kScanTile - 1) / kScanTile;
        w += 2 * n;
    }
    return w + 1;
}

void scan_exclusive(const uint32_t* in, uint32_t* out, uint64_t n, uint32_t* tmp, cudaStream_t st) {
    if (n == 0) return;
    if (n <= (uint64_t)kScanTile) {
        k_scan_apply<<<1, kThreads, 0, st>>>(in, n, out, nullptr);
        return;
    }
    uint64_t nb = (n + kScanTile - 1) / kScanTile;
    uint32_t* bsum = tmp;
    uint32_t* boff = tmp + nb;
    k_scan_reduce<<<(unsigned)nb, kThreads, 0, st>>>(in, n, bsum);
    scan_exclusive(bsum, boff, nb, tmp + 2 * nb, st);
    k_scan_apply<<<(unsigned)nb, kThreads, 0, st>>>(in, n, out, boff);
}

// ---- stable LSD radix sort of (cell id, point index) -----------------------------------

__global__ void k_radix_hist(const uint32_t* __restrict__ keys, uint64_t n, int shift,
                             uint32_t* __restrict__ hist, uint32_t nblocks) {
    __shared__ uint32_t h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    uint64_t base = (uint64_t)blockIdx.x * kTile;
    for (int k = 0; k < kItems; ++k) {
        uint64_t i = base + (uint64_t)k * kThreads + threadIdx.x;
        if (i < n) atomicAdd(&h[(keys[i] >> shift) & 255u], 1u);
    }
    __syncthreads();
    hist[(uint64_t)threadIdx.x * nblocks + blockIdx.x] = h[threadIdx.x];
}

// Stable scatter: warp w of a tile owns keys [w*512, (w+1)*512) of the tile and walks them
// 32 at a time in order, so ranks among equal digits follow the input order.
__global__ void __launch_bounds__(kThreads) k_radix_scatter(
    const uint32_t* __restrict__ kin, const uint32_t* __restrict__ vin, uint32_t* __restrict__ kout,
    uint32_t* __restrict__ vout, const uint32_t* __restrict__ offs, uint64_t n, int shift,
    uint32_t nblocks) {
    __shared__ uint32_t wcnt[kWarps][256];
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int d = threadIdx.x; d < kWarps * 256; d += kThreads) (&wcnt[0][0])[d] = 0;
    __syncthreads();
    uint64_t base = (uint64_t)blockIdx.x * kTile + (uint64_t)warp * (kItems * 32);
    uint32_t key[kItems], val[kItems], rank[kItems];
    const uint32_t lt = (1u << lane) - 1u;
#pragma unroll
    for (int r = 0; r < kItems; ++r) {
        uint64_t i = base + (uint64_t)r * 32 + lane;
        bool valid = i < n;
        key[r] = valid ? kin[i] : 0u;
        val[r] = valid ? (vin ? vin[i] : (uint32_t)i) : 0u;
        uint32_t mask = __ballot_sync(0xffffffffu, valid);
        rank[r] = 0;
        if (valid) {
            uint32_t d = (key[r] >> shift) & 255u;
            uint32_t peers = __match_any_sync(mask, d);
            uint32_t old = wcnt[warp][d];
            __syncwarp(mask);
            if (lane == __ffs(peers) - 1) wcnt[warp][d] = old + __popc(peers);
            __syncwarp(mask);
            rank[r] = old + __popc(peers & lt);
        }
    }
    __syncthreads();
    {
        uint32_t d = threadIdx.x, run = 0;
        for (int w = 0; w < kWarps; ++w) {
            uint32_t c = wcnt[w][d];
            wcnt[w][d] = run;
            run += c;
        }
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kItems; ++r) {
        uint64_t i = base + (uint64_t)r * 32 + lane;
        if (i < n) {
            uint32_t d = (key[r] >> shift) & 255u;
            uint32_t pos = offs[(uint64_t)d * nblocks + blockIdx.x] + wcnt[warp][d] + rank[r];
            kout[pos] = key[r];
            vout[pos] = val[r];
        }
    }
}

__global__ void k_offsets(const double* __restrict__ xyz, const uint8_t* __restrict__ rgb,
                          const uint8_t* __restrict__ scan, const uint32_t* __restrict__ skey,
                          const uint32_t* __restrict__ sval, uint64_t n, double g0x, double g0y,
                          double g0z, double cell, int dx, int dy, float* __restrict__ ox,
                          float* __restrict__ oy, float* __restrict__ oz, uint32_t* __restrict__ rgbs) {
    uint64_t pos = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    if (pos >= n) return;
    uint32_t c = skey[pos];
    uint64_t p = sval[pos];
    int64_t i = c % (uint32_t)dx;
    int64_t j = (c / (uint32_t)dx) % (uint32_t)dy;
    int64_t k = c / ((uint32_t)dx * (uint32_t)dy);
    double ogx = __dadd_rn(g0x, __dmul_rn((double)i, cell));
    double ogy = __dadd_rn(g0y, __dmul_rn((double)j, cell));
    double ogz = __dadd_rn(g0z, __dmul_rn((double)k, cell));
    ox[pos] = __double2float_rn(__dsub_rn(xyz[3 * p + 0], ogx));
    oy[pos] = __double2float_rn(__dsub_rn(xyz[3 * p + 1], ogy));
    oz[pos] = __double2float_rn(__dsub_rn(xyz[3 * p + 2], ogz));
    uint32_t s = scan ? scan[p] : 0u;
    rgbs[pos] = (uint32_t)rgb[3 * p] | ((uint32_t)rgb[3 * p + 1] << 8) | ((uint32_t)rgb[3 * p + 2] << 16) |
                (s << 24);
}

}  // namespace

cudaError_t grid_bbox(const double* xyz, uint64_t n, double* d_tmp, double out[6], cudaStream_t st) {
    const int nb = 1024;
    k_bbox_partial<<<nb, kThreads, 0, st>>>(xyz, n, d_tmp);
    std::vector<double> h(nb * 6);
    cudaError_t e = cudaMemcpyAsync(h.data(), d_tmp, sizeof(double) * nb * 6, cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) return e;
    e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return e;
    for (int a = 0; a < 3; ++a) {
        out[a] = INFINITY;
        out[3 + a] = -INFINITY;
    }
    for (int b = 0; b < nb; ++b)
        for (int a = 0; a < 3; ++a) {
            out[a] = fmin(out[a], h[b * 6 + a]);
            out[3 + a] = fmax(out[3 + a], h[b * 6 + 3 + a]);
        }
    return cudaGetLastError();
}

// Sort the loaded cloud into the grid described by c->g0 / c->dims / c->cell.
cudaError_t grid_build(lnr_ctx* c, cudaStream_t st) {
    const uint64_t n = c->n;
    const int64_t C = c->ncells;
    cudaError_t e;
    DBuf ka, kb, va, vb, counts, hist, hscan, tmp;
    auto cleanup = [&]() {
        ka.release(); kb.release(); va.release(); vb.release();
        counts.release(); hist.release(); hscan.release(); tmp.release();
    };
    uint64_t nblocks = (n + kTile - 1) / kTile;
    size_t tmp_words = scan_tmp_words(std::max<uint64_t>((uint64_t)C + 1, 256 * nblocks));
    if ((e = ka.ensure(4 * n)) || (e = kb.ensure(4 * n)) || (e = va.ensure(4 * n)) ||
        (e = vb.ensure(4 * n)) || (e = counts.ensure(4 * (C + 1))) ||
        (e = hist.ensure(4 * 256 * nblocks)) || (e = hscan.ensure(4 * 256 * nblocks)) ||
        (e = tmp.ensure(4 * tmp_words)) || (e = c->cell_start.ensure(4 * (C + 1))) ||
        (e = c->ox.ensure(4 * n)) || (e = c->oy.ensure(4 * n)) || (e = c->oz.ensure(4 * n)) ||
        (e = c->rgbs.ensure(4 * n))) {
        cleanup();
        return e;
    }
    cudaMemsetAsync(counts.p, 0, 4 * (C + 1), st);
    unsigned g = (unsigned)((n + kThreads - 1) / kThreads);
    k_cell_id<<<g, kThreads, 0, st>>>(c->xyz.as<double>(), n, c->g0[0], c->g0[1], c->g0[2], c->cell,
                                      c->dims[0], c->dims[1], c->dims[2], ka.as<uint32_t>(),
                                      counts.as<uint32_t>());
    scan_exclusive(counts.as<uint32_t>(), c->cell_start.as<uint32_t>(), (uint64_t)C + 1, tmp.as<uint32_t>(), st);
    int bits = 1;
    while (bits < 32 && ((uint64_t)1 << bits) < (uint64_t)C) ++bits;
    uint32_t *kin = ka.as<uint32_t>(), *kout = kb.as<uint32_t>();
    uint32_t *vin = nullptr, *vout = vb.as<uint32_t>();
    uint32_t* vspare = va.as<uint32_t>();
    for (int shift = 0; shift < bits; shift += 8) {
        k_radix_hist<<<(unsigned)nblocks, kThreads, 0, st>>>(kin, n, shift, hist.as<uint32_t>(), (uint32_t)nblocks);
        scan_exclusive(hist.as<uint32_t>(), hscan.as<uint32_t>(), 256 * nblocks, tmp.as<uint32_t>(), st);
        k_radix_scatter<<<(unsigned)nblocks, kThreads, 0, st>>>(kin, vin, kout, vout, hscan.as<uint32_t>(), n,
                                                               shift, (uint32_t)nblocks);
        std::swap(kin, kout);
        uint32_t* nv = vout;
        vout = vin ? vin : vspare;
        vin = nv;
    }
    k_offsets<<<g, kThreads, 0, st>>>(c->xyz.as<double>(), c->rgb.as<uint8_t>(),
                                      c->scan.p ? c->scan.as<uint8_t>() : nullptr, kin, vin, n, c->g0[0],
                                      c->g0[1], c->g0[2], c->cell, c->dims[0], c->dims[1], c->ox.as<float>(),
                                      c->oy.as<float>(), c->oz.as<float>(), c->rgbs.as<uint32_t>());
    e = cudaStreamSynchronize(st);
    cleanup();
    if (e == cudaSuccess) e = cudaGetLastError();
    return e;
}

// exported for the raster translation unit
void scan_exclusive_u32(const uint32_t* in, uint32_t* out, uint64_t n, uint32_t* tmp, cudaStream_t st) {
    scan_exclusive(in, out, n, tmp, st);
}
size_t scan_tmp_words_u32(uint64_t n) { return scan_tmp_words(n); }

}  // namespace lnr
