/*
 * lnr_oracle.c -- plain, slow, CPU reference of the per-frame render path of
 * "Real-time Neural Rendering of LiDAR Point Clouds" (arXiv 2502.11618).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the benchmark's CPU
 * baseline may load this file's library.  The GPU product path never calls it and
 * shares no code, header or constant with it.
 *
 * What it computes, with the passage each step follows:
 *   grid      uniform-grid spatial partition: stable counting sort of points by cell,
 *             FP32 offsets to FP64 cell origins               (Sec. 1; Sec. 3, "Point
 *                                                              Cloud Projection")
 *   view      FP64 composition of the view with the grid      (Sec. 3, projection)
 *   cull      frustum culling of grid cells, six planes       (Sec. 3; Fig. 1)
 *   splat     1x1-pixel projection with a hard z-buffer keyed by (depth, position)
 *                                                             (Sec. 3, projection)
 *   soft      soft z-buffer: the colours of the points that arrive within a small
 *             depth threshold of the front are averaged       (Sec. 3, projection)
 *   resolve   RGB, depth D and fill mask A                    (Fig. 1; Sec. 3 "U-Net")
 *   filter    min-pool pyramid, then Laplacian-edge-aware upsampling with
 *             filter_strength and linear-interpolation fill   (Fig. 2; Sec. 3, "Depth
 *                                                              filtering")
 *   pack      RGBDA input of the U-Net; filtered points get zero alpha
 *                                                             (Sec. 3, "U-Net")
 *   unet      fully convolutional U-Net in FP64, batch norm after each encoder
 *             convolution                                      (Fig. 1; Sec. 3, "U-Net")
 *
 * Readings where the paper is silent (each also listed in the design notes):
 *   - the front of a pixel is its hard z-buffer minimum (ties in depth break towards the
 *     lower sorted position); with the soft rule a point of the pixel contributes its
 *     colour when z <= z_front * (1 + rel) in FP32 (rel unstated; 0.01 by default in
 *     the tests), and the colour is the per-channel integer mean rounded half up;
 *   - D is view-space z; the U-Net's D channel is z / zfar;
 *   - the Laplacian is the 4-neighbour kernel on the coarser min-pooled level with
 *     replicated borders, and a pixel is an edge when |lap| > EDGE_REL * depth;
 *   - an edge pixel's reference is the minimum over its 3x3 window of the coarser
 *     upsampled level, a non-edge pixel's reference is its own value there;
 *   - a finer pixel is kept when its min-pooled depth <= reference * (1 + fs*KEEP_REL);
 *   - the fill is bilinear with weights {3/4, 1/4} per axis over non-empty taps;
 *   - cells are culled against the frustum after growing each cell by 1/64 of its size
 *     on every side, so rounding can never cull a cell that holds a visible point.
 *
 * Floating point: compiled with -ffp-contract=off; every fused multiply-add below is an
 * explicit fmaf, every other operation is rounded on its own.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define EDGE_REL 0.1f    /* edge threshold, relative to the coarse depth */
#define KEEP_REL 0.05f   /* keep tolerance per unit of filter_strength */
#define CULL_PAD (1.0f / 64.0f)
#define BN_EPS 1e-5

static const float INF = (float)INFINITY;

/* ------------------------------------------------------------------ grid ---- */

static int64_t cell_coord(double x, double g0, double cell, int32_t dim) {
    double f = floor((x - g0) / cell);
    if (f < 0.0) f = 0.0;
    if (f > (double)(dim - 1)) f = (double)(dim - 1);
    return (int64_t)f;
}

/* Grid origin g0 = floor(min/cell)*cell and dims = floor((max-g0)/cell)+1 per axis.
 * Returns 0, or -1 for an empty cloud, a non-positive cell or more than 2^31 cells. */
int orc_grid_dims(const double* xyz, uint64_t n, double cell, double g0[3], int32_t dims[3]) {
    if (n == 0 || !(cell > 0.0)) return -1;
    double lo[3] = {xyz[0], xyz[1], xyz[2]}, hi[3] = {xyz[0], xyz[1], xyz[2]};
    for (uint64_t i = 1; i < n; ++i)
        for (int a = 0; a < 3; ++a) {
            double v = xyz[3 * i + a];
            if (v < lo[a]) lo[a] = v;
            if (v > hi[a]) hi[a] = v;
        }
    double total = 1.0;
    for (int a = 0; a < 3; ++a) {
        g0[a] = floor(lo[a] / cell) * cell;
        double d = floor((hi[a] - g0[a]) / cell) + 1.0;
        if (d > 2147483647.0) return -1;
        dims[a] = (int32_t)d;
        total *= d;
    }
    return total > 2147483647.0 ? -1 : 0;
}

/* Stable counting sort of the points by linear cell id c = (k*dy + j)*dx + i.
 * Outputs: cell_start[C+1]; order[pos] = input index of the point at sorted position pos;
 * per position the FP32 offset (x - (g0 + i*cell)) and rgbs = r | g<<8 | b<<16 | scan<<24. */
void orc_grid_build(const double* xyz, const uint8_t* rgb, const uint8_t* scan, uint64_t n,
                    double cell, const double g0[3], const int32_t dims[3], uint32_t* cell_start,
                    uint32_t* order, float* ox, float* oy, float* oz, uint32_t* rgbs) {
    int64_t C = (int64_t)dims[0] * dims[1] * dims[2];
    uint32_t* cid = (uint32_t*)malloc(sizeof(uint32_t) * (n ? n : 1));
    uint32_t* fill = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)(C + 1));
    memset(cell_start, 0, sizeof(uint32_t) * (size_t)(C + 1));
    for (uint64_t p = 0; p < n; ++p) {
        int64_t i = cell_coord(xyz[3 * p + 0], g0[0], cell, dims[0]);
        int64_t j = cell_coord(xyz[3 * p + 1], g0[1], cell, dims[1]);
        int64_t k = cell_coord(xyz[3 * p + 2], g0[2], cell, dims[2]);
        cid[p] = (uint32_t)((k * dims[1] + j) * dims[0] + i);
        cell_start[cid[p] + 1] += 1;
    }
    for (int64_t c = 0; c < C; ++c) cell_start[c + 1] += cell_start[c];
    memcpy(fill, cell_start, sizeof(uint32_t) * (size_t)(C + 1));
    for (uint64_t p = 0; p < n; ++p) {
        uint32_t pos = fill[cid[p]]++;
        order[pos] = (uint32_t)p;
        int64_t c = cid[p];
        int64_t i = c % dims[0], j = (c / dims[0]) % dims[1], k = c / ((int64_t)dims[0] * dims[1]);
        double oxd = g0[0] + (double)i * cell;
        double oyd = g0[1] + (double)j * cell;
        double ozd = g0[2] + (double)k * cell;
        ox[pos] = (float)(xyz[3 * p + 0] - oxd);
        oy[pos] = (float)(xyz[3 * p + 1] - oyd);
        oz[pos] = (float)(xyz[3 * p + 2] - ozd);
        uint32_t s = scan ? scan[p] : 0u;
        rgbs[pos] = (uint32_t)rgb[3 * p] | ((uint32_t)rgb[3 * p + 1] << 8) |
                    ((uint32_t)rgb[3 * p + 2] << 16) | (s << 24);
    }
    free(cid);
    free(fill);
}

/* ------------------------------------------------------------------ view ---- */

/* FP64 composition of the view R (world->camera, row-major) and centre C with the grid:
 * anchor = cell of C (clamped); d0 = (float)(R * (origin(anchor) - C)); step k of the
 * grid in camera space s[3k+r] = (float)(R[r][k] * cell); Rf = (float)R. */
void orc_view_params(const double R[9], const double Cw[3], const double g0[3],
                     const int32_t dims[3], double cell, int32_t anchor[3], float d0[3],
                     float s[9], float Rf[9]) {
    double v[3];
    for (int a = 0; a < 3; ++a) {
        anchor[a] = (int32_t)cell_coord(Cw[a], g0[a], cell, dims[a]);
        v[a] = (g0[a] + (double)anchor[a] * cell) - Cw[a];
    }
    for (int r = 0; r < 3; ++r) {
        double acc = R[3 * r + 0] * v[0];
        acc = acc + R[3 * r + 1] * v[1];
        acc = acc + R[3 * r + 2] * v[2];
        d0[r] = (float)acc;
        for (int k = 0; k < 3; ++k) s[3 * k + r] = (float)(R[3 * r + k] * cell);
    }
    for (int e = 0; e < 9; ++e) Rf[e] = (float)R[e];
}

/* Camera-space position of a point t (in cell units, relative to cell (i,j,k)'s origin). */
static void cam_of(int64_t i, int64_t j, int64_t k, const int32_t a[3], const float d0[3],
                   const float s[9], float tx, float ty, float tz, float out[3]) {
    float di = (float)(i - a[0]), dj = (float)(j - a[1]), dk = (float)(k - a[2]);
    for (int r = 0; r < 3; ++r) {
        float o = fmaf(di, s[0 + r], d0[r]);
        o = fmaf(dj, s[3 + r], o);
        o = fmaf(dk, s[6 + r], o);
        if (tx != 0.0f || ty != 0.0f || tz != 0.0f) {
            o = fmaf(tx, s[0 + r], o);
            o = fmaf(ty, s[3 + r], o);
            o = fmaf(tz, s[6 + r], o);
        }
        out[r] = o;
    }
}

/* ------------------------------------------------------------------ cull ---- */

/* intr = {fx, fy, cx, cy, znear, zfar}.  visible[c] = 1 unless all 8 corners of the
 * grown cell lie strictly outside one frustum plane.  Returns the visible cell count. */
int64_t orc_cull(const int32_t dims[3], const int32_t anchor[3], const float d0[3],
                 const float s[9], const float intr[6], int W, int H, uint8_t* visible) {
    const float fx = intr[0], fy = intr[1], cx = intr[2], cy = intr[3], zn = intr[4], zf = intr[5];
    const float cxw = cx - (float)W, cyh = cy - (float)H;
    int64_t nvis = 0;
    for (int64_t k = 0; k < dims[2]; ++k)
        for (int64_t j = 0; j < dims[1]; ++j)
            for (int64_t i = 0; i < dims[0]; ++i) {
                int out_all[6] = {1, 1, 1, 1, 1, 1};
                for (int corner = 0; corner < 8; ++corner) {
                    float tx = (corner & 1) ? 1.0f + CULL_PAD : -CULL_PAD;
                    float ty = (corner & 2) ? 1.0f + CULL_PAD : -CULL_PAD;
                    float tz = (corner & 4) ? 1.0f + CULL_PAD : -CULL_PAD;
                    float p[3];
                    cam_of(i, j, k, anchor, d0, s, tx, ty, tz, p);
                    float x = p[0], y = p[1], z = p[2];
                    float pl[6];
                    pl[0] = z - zn;
                    pl[1] = zf - z;
                    pl[2] = fmaf(fx, x, cx * z);
                    pl[3] = -fmaf(fx, x, cxw * z);
                    pl[4] = fmaf(fy, y, cy * z);
                    pl[5] = -fmaf(fy, y, cyh * z);
                    for (int q = 0; q < 6; ++q)
                        if (!(pl[q] < 0.0f)) out_all[q] = 0;
                }
                int culled = 0;
                for (int q = 0; q < 6; ++q) culled |= out_all[q];
                int64_t c = (k * dims[1] + j) * dims[0] + i;
                visible[c] = (uint8_t)!culled;
                nvis += !culled;
            }
    return nvis;
}

/* ------------------------------------------------------------------ splat --- */

static uint32_t fbits(float f) {
    uint32_t u;
    memcpy(&u, &f, 4);
    return u;
}

/* Pixel of the point at sorted position pos of a cell whose camera-space origin is o:
 * -1 when it falls outside the near/far range or the image; its depth in *zout. */
static int64_t point_pixel(const float o[3], const float* ox, const float* oy, const float* oz,
                           uint32_t pos, const float Rf[9], const float intr[6], int W, int H,
                           float* zout) {
    const float fx = intr[0], fy = intr[1], cx = intr[2], cy = intr[3], zn = intr[4], zf = intr[5];
    float p[3];
    for (int r = 0; r < 3; ++r) {
        float t = fmaf(Rf[3 * r + 2], oz[pos], o[r]);
        t = fmaf(Rf[3 * r + 1], oy[pos], t);
        p[r] = fmaf(Rf[3 * r + 0], ox[pos], t);
    }
    float z = p[2];
    if (!(z > zn && z < zf)) return -1;
    float u = (fx * p[0]) / z + cx;
    float v = (fy * p[1]) / z + cy;
    if (!(u >= 0.0f && u < (float)W && v >= 0.0f && v < (float)H)) return -1;
    *zout = z;
    return (int64_t)floorf(v) * W + (int64_t)floorf(u);
}

/* keys[v*W+u] = min over the points of the visible cells (all cells when visible is
 * NULL) that project to pixel (u,v) of (bits(z) << 32 | pos); ~0 where none does.
 * Returns the number of points in the visited cells. */
uint64_t orc_splat(const uint8_t* visible, const int32_t dims[3], const uint32_t* cell_start,
                   const float* ox, const float* oy, const float* oz, const int32_t anchor[3],
                   const float d0[3], const float s[9], const float Rf[9], const float intr[6],
                   int W, int H, uint64_t* keys) {
    for (int64_t q = 0; q < (int64_t)W * H; ++q) keys[q] = ~(uint64_t)0;
    uint64_t nvis = 0;
    for (int64_t k = 0; k < dims[2]; ++k)
        for (int64_t j = 0; j < dims[1]; ++j)
            for (int64_t i = 0; i < dims[0]; ++i) {
                int64_t c = (k * dims[1] + j) * dims[0] + i;
                if (visible && !visible[c]) continue;
                float o[3];
                cam_of(i, j, k, anchor, d0, s, 0.0f, 0.0f, 0.0f, o);
                nvis += cell_start[c + 1] - cell_start[c];
                for (uint32_t pos = cell_start[c]; pos < cell_start[c + 1]; ++pos) {
                    float z;
                    int64_t pix = point_pixel(o, ox, oy, oz, pos, Rf, intr, W, H, &z);
                    if (pix < 0) continue;
                    uint64_t key = ((uint64_t)fbits(z) << 32) | pos;
                    if (key < keys[pix]) keys[pix] = key;
                }
            }
    return nvis;
}

/* Soft z-buffer colours (Sec. 3, "Point Cloud Projection": colours of points that arrive
 * at similar depths are averaged, given a small depth threshold).  keys are the hard
 * z-buffer of the same points; a point projecting to pixel q contributes when its depth
 * z <= z_front(q) * scale (one FP32 multiply, scale = 1 + rel), z_front the depth in
 * keys[q].  rgb[q] = per-channel mean of the contributors, (sum + n/2) / n in integers;
 * 0 where keys[q] is empty. */
void orc_soft_colours(const uint8_t* visible, const int32_t dims[3], const uint32_t* cell_start,
                      const float* ox, const float* oy, const float* oz, const uint32_t* rgbs,
                      const int32_t anchor[3], const float d0[3], const float s[9],
                      const float Rf[9], const float intr[6], int W, int H, const uint64_t* keys,
                      float scale, uint8_t* rgb) {
    const int64_t P = (int64_t)W * H;
    uint64_t* sum = (uint64_t*)calloc((size_t)P * 4, sizeof(uint64_t));  /* r, g, b, n */
    for (int64_t k = 0; k < dims[2]; ++k)
        for (int64_t j = 0; j < dims[1]; ++j)
            for (int64_t i = 0; i < dims[0]; ++i) {
                int64_t c = (k * dims[1] + j) * dims[0] + i;
                if (visible && !visible[c]) continue;
                float o[3];
                cam_of(i, j, k, anchor, d0, s, 0.0f, 0.0f, 0.0f, o);
                for (uint32_t pos = cell_start[c]; pos < cell_start[c + 1]; ++pos) {
                    float z;
                    int64_t pix = point_pixel(o, ox, oy, oz, pos, Rf, intr, W, H, &z);
                    if (pix < 0 || keys[pix] == ~(uint64_t)0) continue;
                    uint32_t zb = (uint32_t)(keys[pix] >> 32);
                    float zfront;
                    memcpy(&zfront, &zb, 4);
                    float thr = zfront * scale;
                    if (!(z <= thr)) continue;
                    uint32_t col = rgbs[pos];
                    sum[4 * pix + 0] += col & 255u;
                    sum[4 * pix + 1] += (col >> 8) & 255u;
                    sum[4 * pix + 2] += (col >> 16) & 255u;
                    sum[4 * pix + 3] += 1;
                }
            }
    for (int64_t q = 0; q < P; ++q) {
        uint64_t n = sum[4 * q + 3];
        for (int ch = 0; ch < 3; ++ch)
            rgb[3 * q + ch] = n ? (uint8_t)((sum[4 * q + ch] + n / 2) / n) : 0;
    }
    free(sum);
}

/* RGB, depth (+inf where empty) and fill mask from the z-buffer keys. */
void orc_resolve(const uint64_t* keys, const uint32_t* rgbs, int W, int H, uint8_t* rgb,
                 float* D, uint8_t* A) {
    for (int64_t q = 0; q < (int64_t)W * H; ++q) {
        uint64_t key = keys[q];
        if (key == ~(uint64_t)0) {
            rgb[3 * q] = rgb[3 * q + 1] = rgb[3 * q + 2] = 0;
            D[q] = INF;
            A[q] = 0;
        } else {
            uint32_t zb = (uint32_t)(key >> 32), pos = (uint32_t)key;
            float z;
            memcpy(&z, &zb, 4);
            uint32_t c = rgbs[pos];
            rgb[3 * q] = (uint8_t)c;
            rgb[3 * q + 1] = (uint8_t)(c >> 8);
            rgb[3 * q + 2] = (uint8_t)(c >> 16);
            D[q] = z;
            A[q] = 1;
        }
    }
}

/* ------------------------------------------------------------------ filter -- */

/* One min-pool step, kernel 2x2, stride 2; the coarse level has ceil(W/2) x ceil(H/2)
 * pixels and children outside the fine level are ignored. */
void orc_minpool(const float* fine, int W, int H, float* coarse) {
    int Wc = (W + 1) / 2, Hc = (H + 1) / 2;
    for (int y = 0; y < Hc; ++y)
        for (int x = 0; x < Wc; ++x) {
            float m = INF;
            for (int b = 0; b < 2; ++b)
                for (int a = 0; a < 2; ++a) {
                    int fx = 2 * x + a, fy = 2 * y + b;
                    if (fx < W && fy < H && fine[(int64_t)fy * W + fx] < m) m = fine[(int64_t)fy * W + fx];
                }
            coarse[(int64_t)y * Wc + x] = m;
        }
}

static int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

/* Edge flag of coarse pixel (x,y) from the 4-neighbour Laplacian of Mc. */
static int is_edge(const float* Mc, int Wc, int Hc, int x, int y) {
    float d = Mc[(int64_t)y * Wc + x];
    if (d == INF) return 0;
    float n[4];
    n[0] = Mc[(int64_t)y * Wc + clampi(x - 1, 0, Wc - 1)];
    n[1] = Mc[(int64_t)y * Wc + clampi(x + 1, 0, Wc - 1)];
    n[2] = Mc[(int64_t)clampi(y - 1, 0, Hc - 1) * Wc + x];
    n[3] = Mc[(int64_t)clampi(y + 1, 0, Hc - 1) * Wc + x];
    float t[4];
    for (int e = 0; e < 4; ++e) t[e] = (n[e] == INF) ? 0.0f : n[e] - d;
    float lap = (t[0] + t[1]) + (t[2] + t[3]);
    return fabsf(lap) > EDGE_REL * d;
}

/* One upsampling step (Fig. 2, right): from the coarse min-pooled level Mc and the
 * coarse upsampled level Uc to the fine upsampled level Uf, given the fine min-pooled
 * level Mf.  S = 1 + fs*KEEP_REL.  With fill != 0 the empty fine pixels are then filled
 * by bilinear interpolation of Uc. */
void orc_upsample(const float* Mf, int W, int H, const float* Mc, const float* Uc, float S,
                  int fill, float* Uf) {
    int Wc = (W + 1) / 2, Hc = (H + 1) / 2;
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            int px = x >> 1, py = y >> 1;
            float ref;
            if (is_edge(Mc, Wc, Hc, px, py)) {
                ref = INF;
                for (int b = -1; b <= 1; ++b)
                    for (int a = -1; a <= 1; ++a) {
                        float u = Uc[(int64_t)clampi(py + b, 0, Hc - 1) * Wc + clampi(px + a, 0, Wc - 1)];
                        if (u < ref) ref = u;
                    }
            } else {
                ref = Uc[(int64_t)py * Wc + px];
            }
            float m = Mf[(int64_t)y * W + x];
            int keep = (m <= ref * S) && (m != INF);
            Uf[(int64_t)y * W + x] = keep ? m : INF;
        }
    if (!fill) return;
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            if (Uf[(int64_t)y * W + x] != INF) continue;
            int nx = x >> 1, ny = y >> 1;
            int fxx = clampi((x & 1) ? nx + 1 : nx - 1, 0, Wc - 1);
            int fyy = clampi((y & 1) ? ny + 1 : ny - 1, 0, Hc - 1);
            const int tx[4] = {nx, fxx, nx, fxx};
            const int ty[4] = {ny, ny, fyy, fyy};
            const float w[4] = {0.5625f, 0.1875f, 0.1875f, 0.0625f};
            float num = 0.0f, den = 0.0f;
            for (int e = 0; e < 4; ++e) {
                float u = Uc[(int64_t)ty[e] * Wc + tx[e]];
                if (u == INF) continue;
                num = num + w[e] * u;
                den = den + w[e];
            }
            if (den > 0.0f) Uf[(int64_t)y * W + x] = num / den;
        }
}

/* The depth-guided filter: min-pool n_levels times, then upsample back to the full
 * resolution.  U0 receives the kept depth of every pixel (+inf where the pixel is empty
 * or was filtered out).  Returns 0, or -1 on a bad argument. */
int orc_filter(const float* D, int W, int H, int n_levels, float fs, float* U0) {
    if (W <= 0 || H <= 0 || n_levels < 0 || !(fs >= 0.0f)) return -1;
    float S = 1.0f + fs * KEEP_REL;
    int Ws[33], Hs[33];
    float* M[33];
    float* U[33];
    Ws[0] = W;
    Hs[0] = H;
    M[0] = (float*)D;
    for (int l = 0; l < n_levels; ++l) {
        Ws[l + 1] = (Ws[l] + 1) / 2;
        Hs[l + 1] = (Hs[l] + 1) / 2;
        M[l + 1] = (float*)malloc(sizeof(float) * (size_t)Ws[l + 1] * Hs[l + 1]);
        orc_minpool(M[l], Ws[l], Hs[l], M[l + 1]);
    }
    U[n_levels] = M[n_levels];
    for (int l = n_levels - 1; l >= 0; --l) {
        U[l] = (l == 0) ? U0 : (float*)malloc(sizeof(float) * (size_t)Ws[l] * Hs[l]);
        orc_upsample(M[l], Ws[l], Hs[l], M[l + 1], U[l + 1], S, l > 0, U[l]);
    }
    if (n_levels == 0) memcpy(U0, D, sizeof(float) * (size_t)W * H);
    for (int l = 1; l < n_levels; ++l) free(U[l]);
    for (int l = 1; l <= n_levels; ++l) free(M[l]);
    return 0;
}

/* U-Net input, channels [r/255, g/255, b/255, z/zfar, A]; all zero where A = 0. */
void orc_pack_input(const uint8_t* rgb, const float* U0, int W, int H, float zfar, float* out) {
    for (int64_t q = 0; q < (int64_t)W * H; ++q) {
        int a = U0[q] != INF;
        out[5 * q + 0] = a ? (float)rgb[3 * q + 0] / 255.0f : 0.0f;
        out[5 * q + 1] = a ? (float)rgb[3 * q + 1] / 255.0f : 0.0f;
        out[5 * q + 2] = a ? (float)rgb[3 * q + 2] / 255.0f : 0.0f;
        out[5 * q + 3] = a ? U0[q] / zfar : 0.0f;
        out[5 * q + 4] = a ? 1.0f : 0.0f;
    }
}

/* ------------------------------------------------------------------ U-Net --- */

/* 3x3 convolution, zero padding, stride 1, NHWC (one image), weights OIHW, FP64.
 * With bn (gamma, beta, mean, var per output channel) the batch norm follows the
 * convolution; relu applies max(0, .) last. */
static void conv3x3(const double* in, int W, int H, int cin, const float* w, const float* b,
                    int cout, const float* bn, int relu, double* out) {
    double* wt = (double*)malloc(sizeof(double) * (size_t)cout * 9 * cin);
    for (int co = 0; co < cout; ++co)
        for (int ci = 0; ci < cin; ++ci)
            for (int t = 0; t < 9; ++t) wt[((size_t)co * 9 + t) * cin + ci] = w[((size_t)co * cin + ci) * 9 + t];
#pragma omp parallel for schedule(static)
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x)
            for (int co = 0; co < cout; ++co) {
                double acc = (double)b[co];
                for (int ky = 0; ky < 3; ++ky) {
                    int yy = y + ky - 1;
                    if (yy < 0 || yy >= H) continue;
                    for (int kx = 0; kx < 3; ++kx) {
                        int xx = x + kx - 1;
                        if (xx < 0 || xx >= W) continue;
                        const double* ip = in + ((size_t)yy * W + xx) * cin;
                        const double* wp = wt + ((size_t)co * 9 + ky * 3 + kx) * cin;
                        for (int ci = 0; ci < cin; ++ci) acc += wp[ci] * ip[ci];
                    }
                }
                if (bn) {
                    double g = bn[co], be = bn[cout + co], mu = bn[2 * cout + co], var = bn[3 * cout + co];
                    acc = (acc - mu) / sqrt(var + BN_EPS) * g + be;
                }
                if (relu && acc < 0.0) acc = 0.0;
                out[((size_t)y * W + x) * cout + co] = acc;
            }
    free(wt);
}

static void maxpool2(const double* in, int W, int H, int c, double* out) {
    int Wo = W / 2, Ho = H / 2;
    for (int y = 0; y < Ho; ++y)
        for (int x = 0; x < Wo; ++x)
            for (int ch = 0; ch < c; ++ch) {
                double m = in[((size_t)(2 * y) * W + 2 * x) * c + ch];
                double v1 = in[((size_t)(2 * y) * W + 2 * x + 1) * c + ch];
                double v2 = in[((size_t)(2 * y + 1) * W + 2 * x) * c + ch];
                double v3 = in[((size_t)(2 * y + 1) * W + 2 * x + 1) * c + ch];
                if (v1 > m) m = v1;
                if (v2 > m) m = v2;
                if (v3 > m) m = v3;
                out[((size_t)y * Wo + x) * c + ch] = m;
            }
}

/* [skip (cs channels), nearest-2x-upsampled deep (cd channels)] at the skip's size. */
static void up_concat(const double* skip, int W, int H, int cs, const double* deep, int cd,
                      double* out) {
    int Wd = W / 2;
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            double* o = out + ((size_t)y * W + x) * (cs + cd);
            memcpy(o, skip + ((size_t)y * W + x) * cs, sizeof(double) * cs);
            memcpy(o + cs, deep + ((size_t)(y / 2) * Wd + x / 2) * cd, sizeof(double) * cd);
        }
}

/* Number of floats the weight file of this net holds. */
int64_t orc_unet_weight_count(int L, const int32_t* ch, int in_ch, int out_ch, int has_bn) {
    int64_t n = 0;
    int cin = in_ch;
    for (int l = 0; l < L; ++l) {
        n += (int64_t)ch[l] * cin * 9 + ch[l];
        n += (int64_t)ch[l] * ch[l] * 9 + ch[l];
        if (has_bn) n += 8 * (int64_t)ch[l];
        cin = ch[l];
    }
    for (int l = L - 2; l >= 0; --l) {
        n += (int64_t)ch[l] * (ch[l] + ch[l + 1]) * 9 + ch[l];
        n += (int64_t)ch[l] * ch[l] * 9 + ch[l];
    }
    n += (int64_t)out_ch * ch[0] + out_ch;
    return n;
}

/* FP64 U-Net on one W x H image (W, H multiples of 2^(L-1)); in is NHWC float with in_ch
 * channels, out is NHWC double with out_ch channels in (0, 1).  nthreads <= 0 keeps the
 * OpenMP default.  Returns 0, or -1 on a bad argument. */
int orc_unet(const float* in, int W, int H, int L, const int32_t* ch, int in_ch, int out_ch,
             int has_bn, const float* weights, double* out, int nthreads) {
    if (L < 1 || L > 8 || W <= 0 || H <= 0 || (W % (1 << (L - 1))) || (H % (1 << (L - 1)))) return -1;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
    /* locate every tensor of the weight file */
    const float* cw[32];
    const float* cb[32];
    const float* bnp[32];
    int ncv = 0;
    const float* p = weights;
    int cin = in_ch;
    for (int l = 0; l < L; ++l) {
        cw[ncv] = p; p += (size_t)ch[l] * cin * 9; cb[ncv++] = p; p += ch[l];
        cw[ncv] = p; p += (size_t)ch[l] * ch[l] * 9; cb[ncv++] = p; p += ch[l];
        cin = ch[l];
    }
    for (int l = L - 2; l >= 0; --l) {
        cw[ncv] = p; p += (size_t)ch[l] * (ch[l] + ch[l + 1]) * 9; cb[ncv++] = p; p += ch[l];
        cw[ncv] = p; p += (size_t)ch[l] * ch[l] * 9; cb[ncv++] = p; p += ch[l];
    }
    const float* hw = p; p += (size_t)out_ch * ch[0];
    const float* hb = p; p += out_ch;
    for (int e = 0; e < 2 * L; ++e) {
        bnp[e] = has_bn ? p : NULL;
        if (has_bn) p += 4 * (size_t)ch[e / 2];
    }

    size_t P = (size_t)W * H;
    double* x = (double*)malloc(sizeof(double) * P * in_ch);
    for (size_t q = 0; q < P * in_ch; ++q) x[q] = (double)in[q];
    double* skip[8];
    int Wl = W, Hl = H, c_in = in_ch, cv = 0;
    for (int l = 0; l < L; ++l) {
        size_t Pl = (size_t)Wl * Hl;
        double* t = (double*)malloc(sizeof(double) * Pl * ch[l]);
        conv3x3(x, Wl, Hl, c_in, cw[cv], cb[cv], ch[l], bnp[2 * l], 1, t);
        cv++;
        double* s = (double*)malloc(sizeof(double) * Pl * ch[l]);
        conv3x3(t, Wl, Hl, ch[l], cw[cv], cb[cv], ch[l], bnp[2 * l + 1], 1, s);
        cv++;
        free(t);
        free(x);
        c_in = ch[l];
        if (l == L - 1) { x = s; break; }
        skip[l] = s;
        x = (double*)malloc(sizeof(double) * (Pl / 4) * ch[l]);
        maxpool2(s, Wl, Hl, ch[l], x);
        Wl /= 2;
        Hl /= 2;
    }
    for (int l = L - 2; l >= 0; --l) {
        Wl *= 2;
        Hl *= 2;
        size_t Pl = (size_t)Wl * Hl;
        int cc = ch[l] + ch[l + 1];
        double* cat = (double*)malloc(sizeof(double) * Pl * cc);
        up_concat(skip[l], Wl, Hl, ch[l], x, ch[l + 1], cat);
        free(x);
        free(skip[l]);
        double* t = (double*)malloc(sizeof(double) * Pl * ch[l]);
        conv3x3(cat, Wl, Hl, cc, cw[cv], cb[cv], ch[l], NULL, 1, t);
        cv++;
        free(cat);
        x = (double*)malloc(sizeof(double) * Pl * ch[l]);
        conv3x3(t, Wl, Hl, ch[l], cw[cv], cb[cv], ch[l], NULL, 1, x);
        cv++;
        free(t);
    }
#pragma omp parallel for schedule(static)
    for (int64_t q = 0; q < (int64_t)P; ++q)
        for (int o = 0; o < out_ch; ++o) {
            double acc = (double)hb[o];
            for (int c = 0; c < ch[0]; ++c) acc += (double)hw[o * ch[0] + c] * x[(size_t)q * ch[0] + c];
            out[(size_t)q * out_ch + o] = 1.0 / (1.0 + exp(-acc));
        }
    free(x);
    return 0;
}

int orc_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
