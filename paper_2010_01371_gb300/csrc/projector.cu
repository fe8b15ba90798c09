// Joseph ray-driven projector A and its exact transpose A^T on the GPU.
//
// The paper leaves the system matrix A of the mean model (Eq. 1; A -> A for
// standard CT, Eq. 20, and A -> QA for one-step MBMD, Eq. 44) unspecified;
// this is Joseph's method on a pixel-centred grid.  For each ray the axis with
// the largest |u| component drives the march; at every driving-axis pixel
// index i the ray's coordinate along the other axis is interpolated linearly
// (2-D) between the two neighbouring pixel centres (zero outside the grid)
// and the samples are summed with weight (pixel size) / |u_axis|.
//
// Design (2-D):
//  * set-up: one FP64 thread per ray computes the interpolation coordinate at
//    i = 0, its increment per step, the weight and a conservative range of i
//    (outside it every sample is zero); stored as one float4 per ray and
//    shared by the forward and the transpose so both use identical weights;
//  * forward: one thread per ray (default; neighbouring threads =
//    neighbouring bins of one view) reading an x-driven copy [ix][iy][m] and a
//    y-driven copy [iy][ix][m] of the image (materials packed as
//    float/float2/float4) with Kahan-compensated FP32 accumulation along the
//    ray, or tile sums through shared memory (the tile decomposition below;
//    mbir_plan_set_projector);
//  * transpose: tile scatter into 32-bit fixed-point shared-memory
//    accumulators and a 64-bit fixed-point image (default; bitwise
//    reproducible), a pixel-driven gather (deterministic, no atomics) and a
//    ray-driven scatter with global FP32 atomics, all with the forward's
//    per-ray weights (mbir_plan_set_backprojector).
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdint>
#include <cstring>

#include "common.cuh"

namespace psps {
namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ void ray_2d(const mbir_geometry &g, int64_t ray, double &px, double &py, double &ux,
                                       double &uy) {
    const int view = (int)(ray / g.n_u);
    const int iu = (int)(ray % g.n_u);
    const double ang = g.angle0 + view * (g.angle_span / g.n_views);
    double c, s;
    sincos(ang, &s, &c);
    if (g.kind == MBIR_PAR2D) {
        const double t = (iu - 0.5 * (g.n_u - 1)) * g.du;
        px = -s * t;
        py = c * t;
        ux = -c;
        uy = -s;
    } else {
        const double ga = (iu - 0.5 * (g.n_u - 1)) * g.du / g.sdd;
        px = g.sid * c;
        py = g.sid * s;
        double sg, cg;
        sincos(ang - ga, &sg, &cg);
        ux = -cg;
        uy = -sg;
    }
}

// Conservative range of driving indices i in [0, n_drive-1] for which the
// interpolation coordinate f(i) = f0 + i*df lies in (-1, n_other).
__device__ __forceinline__ void drive_range(double f0, double df, int n_drive, int n_other, int &lo, int &hi) {
    double a, b;
    if (df == 0.0) {
        if (f0 > -1.0 && f0 < (double)n_other) {
            lo = 0;
            hi = n_drive - 1;
        } else {
            lo = 1;
            hi = 0;
        }
        return;
    }
    a = (-1.0 - f0) / df;
    b = ((double)n_other - f0) / df;
    if (a > b) {
        double t = a;
        a = b;
        b = t;
    }
    double l = floor(a) - 1.0, h = ceil(b) + 1.0;
    if (l < 0) l = 0;
    if (h > n_drive - 1) h = n_drive - 1;
    if (l > h) {
        lo = 1;
        hi = 0;
    } else {
        lo = (int)l;
        hi = (int)h;
    }
}

__global__ void setup_2d_kernel(mbir_geometry g, int64_t n_rays, float4 *tab) {
    const int64_t ray = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (ray >= n_rays) return;
    double px, py, ux, uy;
    ray_2d(g, ray, px, py, ux, uy);
    const double cx = 0.5 * (g.nx - 1), cy = 0.5 * (g.ny - 1);
    int axis, lo, hi;
    double f0, df, w;
    if (fabs(ux) >= fabs(uy)) {
        axis = 0;
        // f(i) = (py + ((i - cx) dx - px) uy/ux) / dy + cy
        df = g.dx * uy / ux / g.dy;
        f0 = (py + ((0.0 - cx) * g.dx - px) * uy / ux) / g.dy + cy;
        w = g.dx / fabs(ux);
        drive_range(f0, df, g.nx, g.ny, lo, hi);
    } else {
        axis = 1;
        df = g.dy * ux / uy / g.dx;
        f0 = (px + ((0.0 - cy) * g.dy - py) * ux / uy) / g.dx + cx;
        w = g.dy / fabs(uy);
        drive_range(f0, df, g.ny, g.nx, lo, hi);
    }
    const int bits = axis | (lo << 1) | (hi << 16);
    tab[ray] = make_float4((float)f0, (float)df, (float)w, __int_as_float(bits));
}

__global__ void setup_view_kernel(mbir_geometry g, float4 *vt) {
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= g.n_views) return;
    const double ang = g.angle0 + v * (g.angle_span / g.n_views);
    double s, c;
    sincos(ang, &s, &c);
    if (g.kind == MBIR_PAR2D) {
        vt[v] = make_float4((float)c, (float)s, 0.f, 0.f);
    } else {
        // reduce beta + pi into (-pi, pi]
        double a = ang + M_PI;
        a -= 2.0 * M_PI * rint(a / (2.0 * M_PI));
        vt[v] = make_float4((float)(g.sid * c), (float)(g.sid * s), (float)a, 0.f);
    }
}

template <int NM>
struct Pack;
template <>
struct Pack<1> {
    using T = float;
    static constexpr int P = 1;
    __device__ static void get(const T &v, float (&o)[1]) { o[0] = v; }
};
template <>
struct Pack<2> {
    using T = float2;
    static constexpr int P = 2;
    __device__ static void get(const T &v, float (&o)[2]) {
        o[0] = v.x;
        o[1] = v.y;
    }
};
template <>
struct Pack<3> {
    using T = float4;
    static constexpr int P = 4;
    __device__ static void get(const T &v, float (&o)[3]) {
        o[0] = v.x;
        o[1] = v.y;
        o[2] = v.z;
    }
};
template <>
struct Pack<4> {
    using T = float4;
    static constexpr int P = 4;
    __device__ static void get(const T &v, float (&o)[4]) {
        o[0] = v.x;
        o[1] = v.y;
        o[2] = v.z;
        o[3] = v.w;
    }
};

// x [m][ny][nx] -> xrow [iy][ix][P] and xcol [ix][iy][P] (P = packed stride).
// 32x32 tiles through shared memory for the transposed copy.
template <int NM>
__global__ void pack_kernel(const float *__restrict__ x, int nx, int ny, float *__restrict__ xrow,
                            float *__restrict__ xcol) {
    constexpr int P = Pack<NM>::P;
    __shared__ float tile[NM][32][33];
    const int bx = blockIdx.x * 32, by = blockIdx.y * 32;
    const int64_t npix = (int64_t)nx * ny;
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int iy = by + r, ix = bx + threadIdx.x;
        if (iy < ny && ix < nx) {
#pragma unroll
            for (int m = 0; m < NM; ++m) {
                const float v = x[m * npix + (int64_t)iy * nx + ix];
                tile[m][r][threadIdx.x] = v;
                if (xrow) xrow[((int64_t)iy * nx + ix) * P + m] = v;
            }
            if (xrow && P > NM) xrow[((int64_t)iy * nx + ix) * P + NM] = 0.f;
        }
    }
    __syncthreads();
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int ix = bx + r, iy = by + threadIdx.x;
        if (iy < ny && ix < nx) {
#pragma unroll
            for (int m = 0; m < NM; ++m) xcol[((int64_t)ix * ny + iy) * P + m] = tile[m][threadIdx.x][r];
            if (P > NM) xcol[((int64_t)ix * ny + iy) * P + NM] = 0.f;
        }
    }
}

// Neighbour pairs for the one-channel forward: pairs[i][j + 1] =
// (x(i, j), x(i, j + 1)) along the interpolated axis, j = -1 .. n_other - 1,
// zero outside the image, so every sample is one aligned 8-byte load.
// family 0: i = column, j = row; family 1: i = row, j = column.
__global__ void pair_pack_kernel(const float *__restrict__ x, int nx, int ny, float2 *__restrict__ pc,
                                 float2 *__restrict__ pr) {
    const int64_t ncol = (int64_t)nx * (ny + 1), nrow = (int64_t)ny * (nx + 1);
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < ncol + nrow;
         t += (int64_t)gridDim.x * blockDim.x) {
        if (t < ncol) {
            const int i = (int)(t / (ny + 1)), j = (int)(t % (ny + 1)) - 1;   // column i, rows j, j+1
            const float a = j >= 0 ? x[(int64_t)j * nx + i] : 0.f;
            const float b = j + 1 < ny ? x[(int64_t)(j + 1) * nx + i] : 0.f;
            pc[t] = make_float2(a, b);
        } else {
            const int64_t u = t - ncol;
            const int i = (int)(u / (nx + 1)), j = (int)(u % (nx + 1)) - 1;   // row i, columns j, j+1
            const float a = j >= 0 ? x[(int64_t)i * nx + j] : 0.f;
            const float b = j + 1 < nx ? x[(int64_t)i * nx + j + 1] : 0.f;
            pr[u] = make_float2(a, b);
        }
    }
}

__device__ __forceinline__ void decode(float4 r, int &axis, int &lo, int &hi) {
    const int bits = __float_as_int(r.w);
    axis = bits & 1;
    lo = (bits >> 1) & 0x7fff;
    hi = (bits >> 16) & 0x7fff;
}

template <int NM>
__global__ void __launch_bounds__(kThreads) fwd_2d_kernel(const float4 *__restrict__ tab, int64_t n_rays, int nx,
                                                          int ny, const typename Pack<NM>::T *__restrict__ xrow,
                                                          const typename Pack<NM>::T *__restrict__ xcol,
                                                          float *__restrict__ l) {
    const int64_t ray = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (ray >= n_rays) return;
    const float4 r = tab[ray];
    int axis, lo, hi;
    decode(r, axis, lo, hi);
    const typename Pack<NM>::T *src = axis == 0 ? xcol : xrow;
    const int n_other = axis == 0 ? ny : nx;
    const float f0h = r.x - 0.5f;
    float acc[NM], comp[NM];
#pragma unroll
    for (int m = 0; m < NM; ++m) acc[m] = comp[m] = 0.f;
    for (int i = lo; i <= hi; ++i) {
        float f;
        const int i0 = joseph_split(fmaf((float)i, r.y, f0h), f);
        const typename Pack<NM>::T *base = src + (int64_t)i * n_other;
        float a[NM], b[NM];
#pragma unroll
        for (int m = 0; m < NM; ++m) a[m] = b[m] = 0.f;
        if (i0 >= 0 && i0 < n_other) Pack<NM>::get(__ldg(base + i0), a);
        if (i0 + 1 >= 0 && i0 + 1 < n_other) Pack<NM>::get(__ldg(base + i0 + 1), b);
#pragma unroll
        for (int m = 0; m < NM; ++m) {
            const float v = __fadd_rn(__fmul_rn(1.f - f, a[m]), __fmul_rn(f, b[m]));
            const float yk = __fsub_rn(v, comp[m]);
            const float t = __fadd_rn(acc[m], yk);
            comp[m] = __fsub_rn(__fsub_rn(t, acc[m]), yk);
            acc[m] = t;
        }
    }
#pragma unroll
    for (int m = 0; m < NM; ++m) l[(int64_t)m * n_rays + ray] = acc[m] * r.z;
}

__global__ void __launch_bounds__(kThreads) fwd_2d_pair_kernel(const float4 *__restrict__ tab, int64_t n_rays, int nx,
                                                               int ny, const float2 *__restrict__ pc,
                                                               const float2 *__restrict__ pr, float *__restrict__ l) {
    const int64_t ray = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (ray >= n_rays) return;
    const float4 r = tab[ray];
    int axis, lo, hi;
    decode(r, axis, lo, hi);
    const int n_other = axis == 0 ? ny : nx;
    const int stride = n_other + 1;
    const float f0h = r.x - 0.5f;
    // joseph_split inlined, returning i0 + 1 (the pair index) directly
    const int rel = __float_as_int(kSplitMagic) - 1;
    const float2 *row = (axis == 0 ? pc : pr) + (int64_t)lo * stride;
    float acc = 0.f, comp = 0.f, fi = (float)lo;
    // Eight samples per step: their neighbour-pair loads are issued before
    // any is consumed, so a lane keeps eight independent gathers in flight;
    // the eight samples are summed in order in FP32 and that partial sum is
    // added to the Kahan-compensated total (error of a partial: 7 roundings
    // of at most 8 terms, then compensated across partials).
    constexpr int U = 8;
    int i = lo;
    for (; i + U - 1 <= hi; i += U, fi += (float)U, row += U * stride) {
        float2 ab[U];
        float f[U];
        bool ok[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const float h = fmaf(fi + (float)u, r.y, f0h);
            const float rn = h + kSplitMagic;
            const int k = __float_as_int(rn) - rel;
            ok[u] = (unsigned)k <= (unsigned)n_other;   // else both pixels are off the grid
            f[u] = (h - (rn - kSplitMagic)) + 0.5f;
            ab[u] = __ldg(row + u * stride + (ok[u] ? k : 0));
        }
        float part = 0.f;
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const float v = ok[u] ? fmaf(f[u], ab[u].y - ab[u].x, ab[u].x) : 0.f;
            part = __fadd_rn(part, v);
        }
        const float yk = __fsub_rn(part, comp);
        const float t = __fadd_rn(acc, yk);
        comp = __fsub_rn(__fsub_rn(t, acc), yk);
        acc = t;
    }
    for (; i <= hi; ++i, fi += 1.f, row += stride) {
        const float h = fmaf(fi, r.y, f0h);
        const float rn = h + kSplitMagic;
        const int k = __float_as_int(rn) - rel;
        if ((unsigned)k > (unsigned)n_other) continue;  // both pixels off the grid
        const float f = (h - (rn - kSplitMagic)) + 0.5f;
        const float2 ab = __ldg(row + k);
        const float v = fmaf(f, ab.y - ab.x, ab.x);
        const float yk = __fsub_rn(v, comp);
        const float t = __fadd_rn(acc, yk);
        comp = __fsub_rn(__fsub_rn(t, acc), yk);
        acc = t;
    }
    l[ray] = acc * r.z;
}

__global__ void __launch_bounds__(kThreads) back_2d_kernel(const float4 *__restrict__ tab, int64_t n_rays, int nx,
                                                           int ny, int n_mat, const float *__restrict__ sino,
                                                           float *__restrict__ x) {
    const int64_t ray = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (ray >= n_rays) return;
    const float4 r = tab[ray];
    int axis, lo, hi;
    decode(r, axis, lo, hi);
    const int64_t npix = (int64_t)nx * ny;
    for (int m = 0; m < n_mat; ++m) {
        const float ws = r.z * sino[(int64_t)m * n_rays + ray];
        if (ws == 0.f) continue;
        float *img = x + m * npix;
        const int n_other = axis == 0 ? ny : nx;
        for (int i = lo; i <= hi; ++i) {
            const float fy = fmaf((float)i, r.y, r.x);
            const float fl = floorf(fy);
            const int i0 = (int)fl;
            const float f = fy - fl;
            // pixel index of (driving i, other j)
            if (i0 >= 0 && i0 < n_other) {
                const int64_t idx = axis == 0 ? (int64_t)i0 * nx + i : (int64_t)i * nx + i0;
                atomicAdd(img + idx, (1.f - f) * ws);
            }
            if (i0 + 1 >= 0 && i0 + 1 < n_other) {
                const int64_t idx = axis == 0 ? (int64_t)(i0 + 1) * nx + i : (int64_t)i * nx + i0 + 1;
                atomicAdd(img + idx, f * ws);
            }
        }
    }
}

// Pixel-driven exact transpose: every pixel gathers, view by view, the rays
// whose Joseph samples touch it.  For x-driven rays that is the set crossing
// the vertical segment x = x_c, |y - y_c| < dy; for y-driven rays the
// horizontal segment y = y_c, |x - x_c| < dx.  The bin range of each segment
// is found from its end points (bin position is monotone along a segment) and
// widened by one bin; every candidate's weight is then recomputed from the same
// per-ray set-up as the forward projector, so candidates that do not touch
// the pixel contribute exactly zero and the weights equal the forward ones.
// Deterministic (no atomics), one write per pixel, Kahan sums over views.
template <int NC>
__global__ void __launch_bounds__(kThreads)
    back_gather_2d_kernel(const float4 *__restrict__ tab, const float4 *__restrict__ vt, mbir_geometry g,
                          const float *__restrict__ sino, int64_t n_rays, float *__restrict__ x, int accumulate) {
    const int ix = blockIdx.x * 16 + (threadIdx.x & 15);
    const int iy = blockIdx.y * 16 + (threadIdx.x >> 4);
    if (ix >= g.nx || iy >= g.ny) return;
    const float cxp = 0.5f * (g.nx - 1), cyp = 0.5f * (g.ny - 1);
    const float xc = (float)((ix - 0.5 * (g.nx - 1)) * g.dx), yc = (float)((iy - 0.5 * (g.ny - 1)) * g.dy);
    const float dx = (float)g.dx, dy = (float)g.dy;
    const float cu = 0.5f * (g.n_u - 1);
    const float inv_du = (float)(1.0 / g.du);
    const float fan_scale = (float)(g.sdd / g.du);
    const bool fan = g.kind == MBIR_FAN2D;
    float acc[NC], comp[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) acc[c] = comp[c] = 0.f;
    (void)cxp;
    (void)cyp;
    for (int v = 0; v < g.n_views; ++v) {
        const float4 V = vt[v];
        const float4 *trow = tab + (int64_t)v * g.n_u;
        const float *srow = sino + (int64_t)v * g.n_u;
#pragma unroll
        for (int fam = 0; fam < 2; ++fam) {
            // segment end points
            const float ax = fam == 0 ? xc : xc - dx, ay = fam == 0 ? yc - dy : yc;
            const float bx = fam == 0 ? xc : xc + dx, by = fam == 0 ? yc + dy : yc;
            float pa, pb;
            if (!fan) {
                pa = (-V.y * ax + V.x * ay) * inv_du + cu;
                pb = (-V.y * bx + V.x * by) * inv_du + cu;
            } else {
                float ga = V.z - atan2f(ay - V.y, ax - V.x);
                float gb = V.z - atan2f(by - V.y, bx - V.x);
                ga -= 6.283185307f * rintf(ga * 0.159154943f);
                gb -= 6.283185307f * rintf(gb * 0.159154943f);
                pa = ga * fan_scale + cu;
                pb = gb * fan_scale + cu;
            }
            int b0 = (int)floorf(fminf(pa, pb)) - 1, b1 = (int)ceilf(fmaxf(pa, pb)) + 1;
            if (b0 < 0) b0 = 0;
            if (b1 > g.n_u - 1) b1 = g.n_u - 1;
            for (int b = b0; b <= b1; ++b) {
                const float4 r = __ldg(trow + b);
                const int bits = __float_as_int(r.w);
                if ((bits & 1) != fam) continue;
                const int i = fam == 0 ? ix : iy;      // driving index of this pixel
                const int j = fam == 0 ? iy : ix;      // interpolated index
                const float fy = fmaf((float)i, r.y, r.x);
                const float fl = floorf(fy);
                const int i0 = (int)fl;
                const float f = fy - fl;
                float wgt;
                if (j == i0) wgt = 1.f - f;
                else if (j == i0 + 1) wgt = f;
                else continue;
                wgt *= r.z;
#pragma unroll
                for (int c = 0; c < NC; ++c) {
                    const float val = wgt * __ldg(srow + (int64_t)c * n_rays + b);
                    const float yk = __fsub_rn(val, comp[c]);
                    const float t = __fadd_rn(acc[c], yk);
                    comp[c] = __fsub_rn(__fsub_rn(t, acc[c]), yk);
                    acc[c] = t;
                }
            }
        }
    }
    const int64_t npix = (int64_t)g.nx * g.ny;
    const int64_t pix = (int64_t)iy * g.nx + ix;
#pragma unroll
    for (int c = 0; c < NC; ++c) {
        float *o = x + c * npix + pix;
        *o = accumulate ? *o + acc[c] : acc[c];
    }
}

// ---------------------------------------------------------------------------
// Tile decomposition shared by the forward projector and the transpose.
//
// One CTA owns a kBT x kBT image tile and a chunk of kBVsplit views.  A
// prologue finds, for every view, the bins whose rays can touch the tile (fan
// angle / offset of the tile corners widened by one pixel, plus two bins) and
// prefix-sums their counts; the threads then stride over the flattened
// (view, bin) items with no further barriers.  For one item the driving
// indices inside the tile where the interpolated coordinate can reach the
// tile are solved from the ray's own set-up (f0, df), and each Joseph sample
// is split into its two pixel terms; a CTA handles exactly the terms whose
// pixel lies in its tile, so every term is counted once over all CTAs:
//   forward:   partial sums over the tile's terms, one global atomic per
//              (tile, ray, channel) into l;
//   transpose: terms added into shared-memory accumulators (one per channel),
//              one global atomic per (pixel, channel) per CTA into x.
// Both use the same per-ray weights as the one-ray-per-thread forward, so the
// pair is an exact transpose up to FP32 rounding.
constexpr int kBT = 32;          // tile side (pixels)
constexpr int kBVsplit = 180;    // views per CTA

struct TileItems {
    int nv;                      // views in this chunk
    int v_begin;
    int b0[kBVsplit];
    int prefix[kBVsplit + 1];
};

// Prologue: bin ranges of all views of the chunk (all threads), prefix sum.
__device__ __forceinline__ void tile_items(TileItems &ti, const float4 *__restrict__ vt, const mbir_geometry &g,
                                           int c0, int r0) {
    const bool fan = g.kind == MBIR_FAN2D;
    const float cu = 0.5f * (g.n_u - 1);
    const float inv_du = (float)(1.0 / g.du), fan_scale = (float)(g.sdd / g.du);
    const float x_lo = (float)((c0 - 1 - 0.5 * (g.nx - 1)) * g.dx), x_hi = (float)((c0 + kBT - 0.5 * (g.nx - 1)) * g.dx);
    const float y_lo = (float)((r0 - 1 - 0.5 * (g.ny - 1)) * g.dy), y_hi = (float)((r0 + kBT - 0.5 * (g.ny - 1)) * g.dy);
    for (int k = threadIdx.x; k < ti.nv; k += blockDim.x) {
        const float4 V = vt[ti.v_begin + k];
        float bmin = 3e38f, bmax = -3e38f;
        for (int q = 0; q < 4; ++q) {
            const float px = (q & 1) ? x_hi : x_lo, py = (q & 2) ? y_hi : y_lo;
            float b;
            if (!fan) {
                b = (-V.y * px + V.x * py) * inv_du + cu;
            } else {
                float ga = V.z - atan2f(py - V.y, px - V.x);
                ga -= 6.283185307f * rintf(ga * 0.159154943f);
                b = ga * fan_scale + cu;
            }
            bmin = fminf(bmin, b);
            bmax = fmaxf(bmax, b);
        }
        const int b0 = max((int)floorf(bmin) - 2, 0), b1 = min((int)ceilf(bmax) + 2, g.n_u - 1);
        ti.b0[k] = b0;
        ti.prefix[k + 1] = max(0, b1 - b0 + 1);   // count, turned into a prefix below
    }
    __syncthreads();
    if (threadIdx.x < 32) {
        // warp-level inclusive scan over the counts, 32 views at a time
        int carry = 0;
        for (int base = 0; base < ti.nv; base += 32) {
            const int k = base + threadIdx.x;
            int v = k < ti.nv ? ti.prefix[k + 1] : 0;
            for (int o = 1; o < 32; o <<= 1) {
                const int t = __shfl_up_sync(0xffffffffu, v, o);
                if (threadIdx.x >= o) v += t;
            }
            if (k < ti.nv) ti.prefix[k + 1] = carry + v;
            carry += __shfl_sync(0xffffffffu, v, 31);
        }
        if (threadIdx.x == 0) ti.prefix[0] = 0;
    }
    __syncthreads();
}

// Driving-index range [ia, ib] of one ray inside the tile (empty: ia > ib);
// axis / d0 / o0: the ray's driving axis, the tile's first driving index and
// the tile's first interpolated index.
__device__ __forceinline__ void tile_ray_range(const float4 &r, int c0, int r0, int &axis, int &d0, int &o0, int &ia,
                                               int &ib) {
    const int bits = __float_as_int(r.w);
    axis = bits & 1;
    const int lo = (bits >> 1) & 0x7fff, hi = (bits >> 16) & 0x7fff;
    d0 = axis == 0 ? c0 : r0;
    o0 = axis == 0 ? r0 : c0;
    ia = max(lo, d0);
    ib = min(hi, d0 + kBT - 1);
    if (r.y != 0.f) {
        float ta = ((float)o0 - 1.f - r.x) / r.y, tb = ((float)(o0 + kBT) - r.x) / r.y;
        if (ta > tb) {
            const float t = ta;
            ta = tb;
            tb = t;
        }
        // nearly axis-aligned rays give huge |ta|, |tb|: clamp before
        // converting so that the integer bounds cannot overflow
        ta = fminf(fmaxf(ta, -1.0e8f), 1.0e8f);
        tb = fminf(fmaxf(tb, -1.0e8f), 1.0e8f);
        ia = max(ia, (int)floorf(ta) - 1);
        ib = min(ib, (int)ceilf(tb) + 1);
    }
}

// tile_ray_range with one approximate reciprocal instead of two divisions:
// the range only has to contain every driving index whose sample reaches the
// tile, and the one-index margins on both sides absorb the few-ulp error of
// the approximate reciprocal wherever the bound falls inside the tile.
__device__ __forceinline__ void tile_ray_range_approx(const float4 &r, int c0, int r0, int &axis, int &d0, int &o0,
                                                      int &ia, int &ib) {
    const int bits = __float_as_int(r.w);
    axis = bits & 1;
    const int lo = (bits >> 1) & 0x7fff, hi = (bits >> 16) & 0x7fff;
    d0 = axis == 0 ? c0 : r0;
    o0 = axis == 0 ? r0 : c0;
    ia = max(lo, d0);
    ib = min(hi, d0 + kBT - 1);
    if (r.y != 0.f) {
        const float inv = __fdividef(1.f, r.y);
        float ta = ((float)o0 - 1.f - r.x) * inv, tb = ((float)(o0 + kBT) - r.x) * inv;
        const float t0 = fminf(ta, tb), t1 = fmaxf(ta, tb);
        ia = max(ia, (int)floorf(fminf(fmaxf(t0, -1.0e8f), 1.0e8f)) - 1);
        ib = min(ib, (int)ceilf(fminf(fmaxf(t1, -1.0e8f), 1.0e8f)) + 1);
    }
}


// Tile transpose, lanes on driving indices.  Each warp takes 32 (view, bin)
// items at a time, keeps those whose ray crosses the tile (ballot +
// compaction into a per-warp staging area, x-driven rays from the front,
// y-driven rays from the back), then walks the kept rays one by one with lane
// l on driving index d0 + l.  The accumulators of both driving axes are
// stored with the driving index fastest ([axis][c][interpolated row -1..kBT]
// [driving index]), so the 32 lanes of one red.shared always hit 32 distinct
// banks whatever the ray's slope; rows -1 and kBT are padding for samples
// that straddle the tile edge (their other half belongs to the neighbouring
// tile, which handles the same sample).
//
// No per-lane range test is needed besides the row test: driving indices
// outside the ray's [lo, hi] only give samples whose interpolation pixels are
// both off the grid (the range is widened by one index on each side), and
// those, like lanes past the grid's edge, land in rows or columns that the
// epilogue drops.
//
// A sample at interpolated coordinate h goes to pixels floor(h) and
// floor(h) + 1 with weights 1 - f and f, f = h - floor(h): the same split as
// the forward projector's joseph_split, computed with one round-down add.
//
// The accumulators are 32-bit fixed point: shared-memory integer adds are
// native, while an FP32 shared-memory add costs a load and a compare-and-swap
// (three wavefronts of the shared-memory pipe that bounds this kernel against
// one).  Channel c uses the scale
//   sc = min(2^22, 2^30 / T) / M_c,  M_c = w_max max_i |s_c,i| >= |w_i s_c,i|,
// T = a bound on the terms one accumulator receives: a ray adds at most one
// term to a given accumulator, so T = min(the CTA's candidate rays, its
// views x the plan's bound on the rays of one view that reach one
// accumulator, cell_rays; one T, and so one scale, for the whole launch).  A
// sample's value v = sc w s is at most 2^22 (so
// the magic-number conversions below are exact rounding to nearest), its two
// terms round(f v) and round(v) - round(f v) at most min(2^22, 2^30 / T) + 1,
// and T of them stay below 2^30 + T < 2^31.  The terms carry at most one
// unit of 1 / sc (2^-22 M_c when T <= 256) of rounding.  Each CTA adds its
// tile sums into a 64-bit fixed-point image with integer atomics and a last
// pass divides by sc: every sum is exact, so the transpose is bitwise
// reproducible whatever order the adds run in.
constexpr float kFixMagic = 12582912.f;  // 1.5 * 2^23: x + magic rounds x (|x| <= 2^22) to an integer
constexpr int kFixMagicBits = 0x4B400000;

// The pair of adds of one sample: [addr] += lo, [addr + OFF] += hi.
template <int OFF>
__device__ __forceinline__ void red_shared_pair(unsigned addr, int lo, int hi) {
    asm volatile(
        "red.shared.add.s32 [%0], %1;\n\t"
        "red.shared.add.s32 [%0+%3], %2;" ::"r"(addr),
        "r"(lo), "r"(hi), "n"(OFF)
        : "memory");
}

// One channel of one sample: with v = the ray's scaled, weighted value, the
// upper term round(f v) comes from one FMA, hb = bits(f v + magic), and the
// lower one is round(v) - round(f v) = bits(v + magic) - hb, so the two terms
// of a ray add up to round(v) exactly.
template <int OFF>
__device__ __forceinline__ void fix_sample(unsigned addr, float f, float v) {
    const int hb = __float_as_int(fmaf(f, v, kFixMagic));
    red_shared_pair<OFF>(addr, __float_as_int(v + kFixMagic) - hb, hb - kFixMagicBits);
}

// Kept rays [j0, j1) of one driving axis: fi = this lane's driving index,
// rowbase = the tile's first interpolated index - 1, addr = byte address of
// this lane's column in the axis' first accumulator plane (rows of STRIDE
// words); ws holds (f0, df, v0, v1), ws2 v2, v3 (NC > 2).
template <int NC, int STRIDE>
__device__ __forceinline__ void tile_lane_pass(const float4 *__restrict__ ws, const float2 *__restrict__ ws2, int j0,
                                               int j1, float fi, int rowbase, unsigned addr) {
    constexpr unsigned kRowBytes = 4u * STRIDE;
    constexpr unsigned kPlaneBytes = kRowBytes * (kBT + 2);
#pragma unroll 4
    for (int j = j0; j < j1; ++j) {
        const float4 a = ws[j];
        // interpolated coordinate h = f0 + fi df: lower pixel floor(h), weight
        // of the upper one f = h - floor(h) (the magic add rounding down)
        const float h = fmaf(fi, a.y, a.x);
        const float rn = __fadd_rd(h, kFixMagic);
        const float f = h - (rn - kFixMagic);
        const int jr = (__float_as_int(rn) - kFixMagicBits) - rowbase;  // interpolated index - (first index - 1)
        if ((unsigned)jr <= (unsigned)kBT) {
            const unsigned q = addr + (unsigned)jr * kRowBytes;
            fix_sample<kRowBytes>(q, f, a.z);
            if (NC >= 2) fix_sample<kRowBytes>(q + kPlaneBytes, f, a.w);
            if (NC >= 3) {
                const float2 c = ws2[j];
                fix_sample<kRowBytes>(q + 2 * kPlaneBytes, f, c.x);
                if (NC == 4) fix_sample<kRowBytes>(q + 3 * kPlaneBytes, f, c.y);
            }
        }
    }
}

// Fixed-point scale of one channel (see above); 0 when M is not finite.
// M = w_max max|s| rounded up bounds every rounded product w_i s_i; the
// quotient is rounded down so that M sc never exceeds its limit.
__device__ __forceinline__ float fix_scale(unsigned sbits, float w_max, int bound) {
    const float M = __fmul_ru(w_max, __uint_as_float(sbits));
    if (!(M <= 3.0e38f)) return 0.f;
    if (M == 0.f) return 1.f;
    const float lim = fminf(4194304.f, 1073741824.f / (float)(bound > 1 ? bound : 1));
    return fminf(__fdiv_rd(lim, M), 0x1p126f);
}

// max_i |s_c,i| over the rays, as float bits (atomicMax on the bits orders
// non-negative floats; a NaN input propagates as NaN bits).
__global__ void __launch_bounds__(kThreads)
    tile_smax_kernel(const float *__restrict__ sino, int64_t n_rays, int nch, unsigned *__restrict__ out) {
    for (int c = 0; c < nch; ++c) {
        const float *sc = sino + (int64_t)c * n_rays;
        unsigned m = 0u;
        auto take = [&m](float v) {
            const float a = fabsf(v);
            const unsigned b = a != a ? 0x7fc00000u : __float_as_uint(a);
            m = b > m ? b : m;
        };
        // float4 loads from the first 16-byte boundary of the channel
        const int64_t head = ((16 - ((uintptr_t)sc & 15)) & 15) / 4;
        const int64_t h = head < n_rays ? head : n_rays;
        const int64_t n4 = (n_rays - h) / 4;
        const float4 *v4 = reinterpret_cast<const float4 *>(sc + h);
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4;
             i += (int64_t)gridDim.x * blockDim.x) {
            const float4 v = __ldg(v4 + i);
            take(v.x);
            take(v.y);
            take(v.z);
            take(v.w);
        }
        if (blockIdx.x == 0) {
            for (int64_t i = threadIdx.x; i < h; i += blockDim.x) take(sc[i]);
            for (int64_t i = h + 4 * n4 + threadIdx.x; i < n_rays; i += blockDim.x) take(sc[i]);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned t = __shfl_xor_sync(0xffffffffu, m, o);
            m = t > m ? t : m;
        }
        if ((threadIdx.x & 31) == 0 && m) atomicMax(out + c, m);
    }
}

// Largest |w| of the ray table (float bits), once per plan.
__global__ void __launch_bounds__(kThreads) ray_wmax_kernel(const float4 *__restrict__ tab, int64_t n_rays,
                                                            unsigned *__restrict__ out) {
    unsigned m = 0u;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_rays; i += (int64_t)gridDim.x * blockDim.x) {
        const unsigned b = __float_as_uint(fabsf(tab[i].z));
        m = b > m ? b : m;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned t = __shfl_xor_sync(0xffffffffu, m, o);
        m = t > m ? t : m;
    }
    if ((threadIdx.x & 31) == 0 && m) atomicMax(out, m);
}

template <int NC>
__global__ void __launch_bounds__(kThreads, 5)
    back_tile_2d_kernel(const float4 *__restrict__ tab, const float4 *__restrict__ vt, mbir_geometry g,
                        const float *__restrict__ sino, int64_t n_rays, int vs,
                        const unsigned *__restrict__ smax, float w_max, int T, long long *__restrict__ xfix) {
    static_assert(kBT == 32, "one lane per driving index of the tile");
    static_assert(NC >= 1 && NC <= 4, "one to four channels");
    constexpr int kRows = kBT + 2;
    // x-driven planes [row][32 columns]; y-driven planes [column][33]: the
    // pad word keeps the epilogue's transposed reads conflict-free
    constexpr int kSX = kBT, kSY = kBT;
    constexpr int kPX = kRows * kSX, kPY = kRows * kSY;
    __shared__ int acc[NC * (kPX + kPY)];
    __shared__ TileItems ti;
    __shared__ float4 stage[kThreads];
    __shared__ float2 stage2[NC > 2 ? kThreads : 1];
    __shared__ int tr[kBT * (kBT + 1)];
    const int c0 = blockIdx.x * kBT, r0 = blockIdx.y * kBT;
    if (threadIdx.x == 0) {
        ti.v_begin = blockIdx.z * vs;
        ti.nv = min(g.n_views - ti.v_begin, vs);
    }
    for (int k = threadIdx.x; k < NC * (kPX + kPY); k += blockDim.x) acc[k] = 0;
    __syncthreads();
    tile_items(ti, vt, g, c0, r0);
    const int total = ti.prefix[ti.nv];
    float sc[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) sc[c] = fix_scale(__ldg(smax + c), w_max, T);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const unsigned below = (1u << lane) - 1u;
    const unsigned colx = (unsigned)__cvta_generic_to_shared(acc) + 4u * (unsigned)lane;
    const unsigned coly = colx + 4u * NC * kPX;
    float4 *ws = stage + warp * 32;
    float2 *ws2 = stage2 + (NC > 2 ? warp * 32 : 0);
    int k = 0;
    for (int base = warp * 32; base < total; base += nwarps * 32) {
        const int item = base + lane;
        bool keep = false;
        int axis = 0;
        float v[4] = {0.f, 0.f, 0.f, 0.f};
        float4 r = make_float4(0.f, 0.f, 0.f, 0.f);
        if (item < total) {
            while (item >= ti.prefix[k + 1]) ++k;
            const int64_t ray = (int64_t)(ti.v_begin + k) * g.n_u + ti.b0[k] + (item - ti.prefix[k]);
            r = __ldg(tab + ray);
#pragma unroll
            for (int c = 0; c < NC; ++c) v[c] = r.z * __ldg(sino + c * n_rays + ray) * sc[c];
            int d0, o0, ia, ib;
            tile_ray_range_approx(r, c0, r0, axis, d0, o0, ia, ib);
            keep = ia <= ib;
        }
        const unsigned kx = __ballot_sync(0xffffffffu, keep && axis == 0);
        const unsigned ky = __ballot_sync(0xffffffffu, keep && axis == 1);
        if (keep) {
            const int pos = axis == 0 ? __popc(kx & below) : 31 - __popc(ky & below);
            ws[pos] = make_float4(r.x, r.y, v[0], v[1]);
            if (NC > 2) ws2[pos] = make_float2(v[2], v[3]);
        }
        __syncwarp();
        tile_lane_pass<NC, kSX>(ws, ws2, 0, __popc(kx), (float)(c0 + lane), r0 - 1, colx);
        tile_lane_pass<NC, kSY>(ws, ws2, 32 - __popc(ky), 32, (float)(r0 + lane), c0 - 1, coly);
        __syncwarp();
    }
    __syncthreads();
    if (total == 0) return;
    const int64_t npix = (int64_t)g.nx * g.ny;
    // y-driven planes are [column][row]: turn them around through a padded
    // buffer (reads along rows, writes with stride kBT + 1) so that neither
    // side has bank conflicts, then flush row-major with coalesced atomics
    for (int c = 0; c < NC; ++c) {
        for (int q = threadIdx.x; q < kBT * kBT; q += blockDim.x) {
            const int cc = q / kBT, rr = q % kBT;
            tr[rr * (kBT + 1) + cc] = acc[NC * kPX + c * kPY + (cc + 1) * kSY + rr];
        }
        __syncthreads();
        for (int q = threadIdx.x; q < kBT * kBT; q += blockDim.x) {
            const int rr = q / kBT, cc = q % kBT;
            const int iy = r0 + rr, ix = c0 + cc;
            if (iy >= g.ny || ix >= g.nx) continue;
            const long long v = (long long)acc[c * kPX + (rr + 1) * kSX + cc] + (long long)tr[rr * (kBT + 1) + cc];
            if (v)
                atomicAdd(reinterpret_cast<unsigned long long *>(xfix + c * npix + (int64_t)iy * g.nx + ix),
                          (unsigned long long)v);
        }
        __syncthreads();
    }
}

// x[c] (+)= xfix[c] / sc_c, the scale of the transpose launch.
__global__ void __launch_bounds__(kThreads)
    fix_to_float_kernel(const long long *__restrict__ xfix, float *__restrict__ x, int64_t npix, int nch,
                        const unsigned *__restrict__ smax, float w_max, int T, int accumulate) {
    for (int c = 0; c < nch; ++c) {
        const float sc = fix_scale(__ldg(smax + c), w_max, T);
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < npix;
             i += (int64_t)gridDim.x * blockDim.x) {
            const int64_t k = (int64_t)c * npix + i;
            const float v = sc > 0.f ? __fdiv_rn(__ll2float_rn(xfix[k]), sc) : __int_as_float(0x7fc00000);
            x[k] = accumulate ? x[k] + v : v;
        }
    }
}

template <int NC>
__global__ void __launch_bounds__(kThreads, 8)
    fwd_tile_2d_kernel(const float4 *__restrict__ tab, const float4 *__restrict__ vt, mbir_geometry g,
                       const float *__restrict__ x, int64_t n_rays, float *__restrict__ l) {
    __shared__ float img[NC][kBT][kBT + 1];
    __shared__ TileItems ti;
    const int c0 = blockIdx.x * kBT, r0 = blockIdx.y * kBT;
    if (threadIdx.x == 0) {
        ti.v_begin = blockIdx.z * kBVsplit;
        ti.nv = min(g.n_views - ti.v_begin, kBVsplit);
    }
    const int64_t npix = (int64_t)g.nx * g.ny;
    for (int q = threadIdx.x; q < kBT * kBT; q += blockDim.x) {
        const int rr = q / kBT, cc = q % kBT;
        const int iy = r0 + rr, ix = c0 + cc;
        const bool in = iy < g.ny && ix < g.nx;
#pragma unroll
        for (int c = 0; c < NC; ++c) img[c][rr][cc] = in ? x[c * npix + (int64_t)iy * g.nx + ix] : 0.f;
    }
    __syncthreads();
    tile_items(ti, vt, g, c0, r0);
    const int total = ti.prefix[ti.nv];
    int k = 0;
    for (int item = threadIdx.x; item < total; item += blockDim.x) {
        while (item >= ti.prefix[k + 1]) ++k;
        const int64_t ray = (int64_t)(ti.v_begin + k) * g.n_u + ti.b0[k] + (item - ti.prefix[k]);
        const float4 r = __ldg(tab + ray);
        int axis, d0, o0, ia, ib;
        tile_ray_range(r, c0, r0, axis, d0, o0, ia, ib);
        if (ia > ib) continue;
        float sum[NC];
#pragma unroll
        for (int c = 0; c < NC; ++c) sum[c] = 0.f;
        bool any = false;
        for (int i = ia; i <= ib; ++i) {
            const float fy = fmaf((float)i, r.y, r.x);
            const float fl = floorf(fy);
            const int j0 = (int)fl - o0;
            const float f = fy - fl;
            const int li = i - d0;
            if (j0 >= 0 && j0 < kBT) {
                any = true;
#pragma unroll
                for (int c = 0; c < NC; ++c) sum[c] = fmaf(1.f - f, axis == 0 ? img[c][j0][li] : img[c][li][j0], sum[c]);
            }
            if (j0 + 1 >= 0 && j0 + 1 < kBT) {
                any = true;
#pragma unroll
                for (int c = 0; c < NC; ++c) sum[c] = fmaf(f, axis == 0 ? img[c][j0 + 1][li] : img[c][li][j0 + 1], sum[c]);
            }
        }
        if (any) {
#pragma unroll
            for (int c = 0; c < NC; ++c)
                if (sum[c] != 0.f) atomicAdd(l + (int64_t)c * n_rays + ray, sum[c] * r.z);
        }
    }
}

// ---------------------------------------------------------------- strip forward
// One CTA owns kSV consecutive views x kSB consecutive bins (one ray per
// thread, lanes on neighbouring bins) and marches its rays through the image
// in strips of S driving indices (columns for x-driven rays, rows for
// y-driven ones).  For every strip the CTA finds the window of interpolated
// indices its rays touch there (block min/max of the sample splits at the
// strip ends; the split is monotone along a ray), stages that window of the
// strip in shared memory (zero outside the image, so samples need no bounds
// tests) and every lane then steps the same driving index: neighbouring lanes
// read neighbouring shared-memory words.  Windows taller than kSH rows are
// staged in part and the samples outside read global memory.  Sums: a plain
// FP32 sum per strip (at most S samples), strips Kahan-compensated.  Weights
// and the sample split are the per-ray table's, as in every other projector
// and transpose, so the result is the same operator.
// Views x bins per CTA: sb bins (a runtime choice among 32, 64, 128, 256,
// tuned per plan) and kThreads / sb views, one ray per thread.
constexpr int kSH = 256;           // staged window rows

template <int NM>
struct StripShape {
    static constexpr int S = NM == 1 ? 32 : (NM == 2 ? 16 : 8);   // strip width (driving indices)
    static constexpr size_t smem = sizeof(float) * NM * S * kSH;
};

// Planar transposed copies xt[m][ix][iy] of x[m][iy][ix] (the x-driven
// strips read columns contiguously), 32 x 32 tiles through shared memory.
__global__ void transpose_planes_kernel(const float *__restrict__ x, int nm, int nx, int ny, float *__restrict__ xt) {
    __shared__ float tile[32][33];
    const int64_t npix = (int64_t)nx * ny;
    const int bx = blockIdx.x * 32, by = blockIdx.y * 32, m = blockIdx.z;
    if (m >= nm) return;
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int iy = by + r, ix = bx + threadIdx.x;
        if (iy < ny && ix < nx) tile[r][threadIdx.x] = x[m * npix + (int64_t)iy * nx + ix];
    }
    __syncthreads();
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int ix = bx + r, iy = by + threadIdx.x;
        if (iy < ny && ix < nx) xt[m * npix + (int64_t)ix * ny + iy] = tile[threadIdx.x][r];
    }
}

__device__ __forceinline__ int block_min_int(int v, int *red) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = min(v, __shfl_xor_sync(0xffffffffu, v, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    int r = red[0];
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) r = min(r, red[w]);
    return r;
}

__device__ __forceinline__ int block_max_int(int v, int *red) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    int r = red[0];
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) r = max(r, red[w]);
    return r;
}

template <int NM>
__global__ void __launch_bounds__(kThreads) fwd_strip_2d_kernel(const float4 *__restrict__ tab, mbir_geometry g,
                                                                const float *__restrict__ x,
                                                                const float *__restrict__ xt, int64_t n_rays, int sb,
                                                                float *__restrict__ l) {
    constexpr int S = StripShape<NM>::S;
    extern __shared__ float sm[];   // [NM][S][kSH]
    __shared__ int red[4][kThreads / 32];
    const int tid = threadIdx.x;
    const int view = blockIdx.y * (kThreads / sb) + tid / sb, bin = blockIdx.x * sb + tid % sb;
    const bool valid = view < g.n_views && bin < g.n_u;
    const int64_t ray = (int64_t)view * g.n_u + bin;
    float4 r = make_float4(0.f, 0.f, 0.f, 0.f);
    int axis = 0, lo = 1, hi = 0;
    if (valid) {
        r = __ldg(tab + ray);
        decode(r, axis, lo, hi);
    }
    const float f0h = r.x - 0.5f;
    const int64_t npix = (int64_t)g.nx * g.ny;
    float acc[NM], comp[NM];
#pragma unroll
    for (int m = 0; m < NM; ++m) acc[m] = comp[m] = 0.f;
#pragma unroll 1
    for (int fam = 0; fam < 2; ++fam) {
        const bool mine = valid && lo <= hi && axis == fam;
        // driving-index range of this family's rays in the CTA (uniform)
        const int f_lo = block_min_int(mine ? lo : INT_MAX, red[0]);
        const int f_hi = block_max_int(mine ? hi : -1, red[1]);
        if (f_lo > f_hi) continue;
        const int n_drive = fam == 0 ? g.nx : g.ny, n_other = fam == 0 ? g.ny : g.nx;
        const float *src = fam == 0 ? xt : x;   // planar [m][driving][interpolated]
#pragma unroll 1
        for (int i0 = f_lo; i0 <= f_hi; i0 += S) {
            const int ia = max(lo, i0), ib = min(hi, i0 + S - 1);
            const bool has = mine && ia <= ib;
            int ka = INT_MAX, kb = INT_MIN;
            if (has) {
                float fa, fb;
                const int k1 = joseph_split(fmaf((float)ia, r.y, f0h), fa);
                const int k2 = joseph_split(fmaf((float)ib, r.y, f0h), fb);
                ka = min(k1, k2) - 1;       // one index of margin on each side
                kb = max(k1, k2) + 2;       // upper neighbour k + 1, plus margin
            }
            __syncthreads();   // previous strip's readers of sm and red are done
            const int w0 = block_min_int(ka, red[2]);
            const int w1 = block_max_int(kb, red[3]);
            if (w1 < w0) continue;                  // no ray of the CTA samples this strip
            const int hs = min(w1 - w0 + 1, kSH);   // staged rows [w0, w0 + hs)
            // one warp per (material, strip index), lanes down the window
            for (int mc = tid >> 5; mc < NM * S; mc += kThreads / 32) {
                const int m = mc / S, i = i0 + (mc - m * S);
                const float *col = src + m * npix + (int64_t)i * n_other;
                float *dst = sm + mc * kSH;
                const bool in_i = i < n_drive;
                for (int rr = tid & 31; rr < hs; rr += 32) {
                    const int row = w0 + rr;
                    dst[rr] = (in_i && row >= 0 && row < n_other) ? __ldg(col + row) : 0.f;
                }
            }
            __syncthreads();
            if (has) {
                float sum[NM];
#pragma unroll
                for (int m = 0; m < NM; ++m) sum[m] = 0.f;
                for (int i = ia; i <= ib; ++i) {
                    float f;
                    const int k = joseph_split(fmaf((float)i, r.y, f0h), f);
                    const int kl = k - w0, c = i - i0;
                    if (kl >= 0 && kl + 1 < hs) {
#pragma unroll
                        for (int m = 0; m < NM; ++m) {
                            const float a = sm[(m * S + c) * kSH + kl], b = sm[(m * S + c) * kSH + kl + 1];
                            sum[m] += fmaf(f, b - a, a);
                        }
                    } else {
                        // outside the staged part of a tall window
#pragma unroll
                        for (int m = 0; m < NM; ++m) {
                            const float *col = src + m * npix + (int64_t)i * n_other;
                            const float a = (k >= 0 && k < n_other) ? __ldg(col + k) : 0.f;
                            const float b = (k + 1 >= 0 && k + 1 < n_other) ? __ldg(col + k + 1) : 0.f;
                            sum[m] += fmaf(f, b - a, a);
                        }
                    }
                }
#pragma unroll
                for (int m = 0; m < NM; ++m) {
                    const float yk = __fsub_rn(sum[m], comp[m]);
                    const float t = __fadd_rn(acc[m], yk);
                    comp[m] = __fsub_rn(__fsub_rn(t, acc[m]), yk);
                    acc[m] = t;
                }
            }
        }
    }
    if (!valid) return;
#pragma unroll
    for (int m = 0; m < NM; ++m) l[(int64_t)m * n_rays + ray] = acc[m] * r.z;
}

template <int NM>
mbir_status project_strip_nm(mbir_plan *p, const float *x, float *l, cudaStream_t s) {
    const int nx = p->g.nx, ny = p->g.ny;
    const dim3 tb(32, 8), tg((unsigned)cdiv(nx, 32), (unsigned)cdiv(ny, 32), (unsigned)NM);
    transpose_planes_kernel<<<tg, tb, 0, s>>>(x, NM, nx, ny, p->xcol.p);
    PSPS_LAUNCH_CHECK();
    const int sb = p->strip_bins, sv = kThreads / sb;
    const dim3 grd((unsigned)cdiv(p->g.n_u, sb), (unsigned)cdiv(p->g.n_views, sv));
    fwd_strip_2d_kernel<NM><<<grd, kThreads, StripShape<NM>::smem, s>>>(p->ray.p, p->g, x, p->xcol.p, p->n_rays, sb,
                                                                        l);
    PSPS_LAUNCH_CHECK();
    return MBIR_OK;
}

template <int NM>
mbir_status project_2d_nm(mbir_plan *p, const float *x, float *l, cudaStream_t s) {
    constexpr int P = Pack<NM>::P;
    if (NM == 1) {
        const int nx = p->g.nx, ny = p->g.ny;
        float2 *pc = (float2 *)p->xcol.p, *pr = (float2 *)p->xrow.p;
        const int64_t tot = (int64_t)nx * (ny + 1) + (int64_t)ny * (nx + 1);
        const int64_t gb = cdiv(tot, kThreads) < 8192 ? cdiv(tot, kThreads) : 8192;
        pair_pack_kernel<<<(unsigned)gb, kThreads, 0, s>>>(x, nx, ny, pc, pr);
        PSPS_LAUNCH_CHECK();
        fwd_2d_pair_kernel<<<(unsigned)cdiv(p->n_rays, kThreads), kThreads, 0, s>>>(p->ray.p, p->n_rays, nx, ny, pc,
                                                                                   pr, l);
        PSPS_LAUNCH_CHECK();
        return MBIR_OK;
    }
    const int nx = p->g.nx, ny = p->g.ny;
    float *xrow = (NM == 1) ? nullptr : p->xrow.p;
    dim3 blk(32, 8), grd((unsigned)cdiv(nx, 32), (unsigned)cdiv(ny, 32));
    pack_kernel<NM><<<grd, blk, 0, s>>>(x, nx, ny, xrow, p->xcol.p);
    PSPS_LAUNCH_CHECK();
    const typename Pack<NM>::T *row = (NM == 1) ? (const typename Pack<NM>::T *)x
                                                : (const typename Pack<NM>::T *)p->xrow.p;
    (void)P;
    fwd_2d_kernel<NM><<<(unsigned)cdiv(p->n_rays, kThreads), kThreads, 0, s>>>(
        p->ray.p, p->n_rays, nx, ny, row, (const typename Pack<NM>::T *)p->xcol.p, l);
    PSPS_LAUNCH_CHECK();
    return MBIR_OK;
}

}  // namespace

mbir_status project(mbir_plan *p, const float *x, float *l, int n_mat, cudaStream_t s) {
    if (p->g.kind == MBIR_CONE3D) return project_cone(p, x, l, n_mat, s);
    if (p->fwd_mode == 0) {
        PSPS_CUDA(cudaMemsetAsync(l, 0, sizeof(float) * (size_t)n_mat * p->n_rays, s));
        const dim3 grd((unsigned)cdiv(p->g.nx, kBT), (unsigned)cdiv(p->g.ny, kBT),
                       (unsigned)cdiv(p->g.n_views, kBVsplit));
        for (int m0 = 0; m0 < n_mat;) {
            const int left = n_mat - m0;
            const float *xm = x + (int64_t)m0 * p->n_pix;
            float *lm = l + (int64_t)m0 * p->n_rays;
            if (left >= 2) {
                fwd_tile_2d_kernel<2><<<grd, kThreads, 0, s>>>(p->ray.p, p->view.p, p->g, xm, p->n_rays, lm);
                m0 += 2;
            } else {
                fwd_tile_2d_kernel<1><<<grd, kThreads, 0, s>>>(p->ray.p, p->view.p, p->g, xm, p->n_rays, lm);
                m0 += 1;
            }
            PSPS_LAUNCH_CHECK();
        }
        return MBIR_OK;
    }
    int done = 0;
    for (int m0 = 0; m0 < n_mat; m0 += 4) {
        const int nm = n_mat - m0 < 4 ? n_mat - m0 : 4;
        const float *xm = x + (int64_t)m0 * p->n_pix;
        float *lm = l + (int64_t)m0 * p->n_rays;
        if (p->fwd_mode == 2) {
            switch (nm) {
                case 1: PSPS_TRY(project_strip_nm<1>(p, xm, lm, s)); break;
                case 2: PSPS_TRY(project_strip_nm<2>(p, xm, lm, s)); break;
                case 3: PSPS_TRY(project_strip_nm<3>(p, xm, lm, s)); break;
                default: PSPS_TRY(project_strip_nm<4>(p, xm, lm, s)); break;
            }
            continue;
        }
        switch (nm) {
            case 1: PSPS_TRY(project_2d_nm<1>(p, xm, lm, s)); break;
            case 2: PSPS_TRY(project_2d_nm<2>(p, xm, lm, s)); break;
            case 3: PSPS_TRY(project_2d_nm<3>(p, xm, lm, s)); break;
            default: PSPS_TRY(project_2d_nm<4>(p, xm, lm, s)); break;
        }
        done += nm;
    }
    (void)done;
    return MBIR_OK;
}

mbir_status backproject(mbir_plan *p, const float *sino, float *x, int n_mat, int accumulate, cudaStream_t s) {
    if (p->g.kind == MBIR_CONE3D) return backproject_cone(p, sino, x, n_mat, accumulate, s);
    if (p->back_mode == 2) {
        if (!accumulate) PSPS_CUDA(cudaMemsetAsync(x, 0, sizeof(float) * (size_t)n_mat * p->n_pix, s));
        back_2d_kernel<<<(unsigned)cdiv(p->n_rays, kThreads), kThreads, 0, s>>>(p->ray.p, p->n_rays, p->g.nx,
                                                                               p->g.ny, n_mat, sino, x);
        PSPS_LAUNCH_CHECK();
        return MBIR_OK;
    }
    if (p->back_mode == 0) {
        const int vs = p->back_views;
        const dim3 grd((unsigned)cdiv(p->g.nx, kBT), (unsigned)cdiv(p->g.ny, kBT), (unsigned)cdiv(p->g.n_views, vs));
        if (n_mat > (int)p->wmax.n) return fail(MBIR_ERR_ARG, "backproject: %d channels exceed the plan's n_mat_max", n_mat);
        // one bound T for every CTA: vs views x the rays of one view that can
        // reach one accumulator (or all bins of the views when unknown)
        const int T = p->cell_rays > 0 ? vs * p->cell_rays : vs * p->g.n_u;
        PSPS_CUDA(cudaMemsetAsync(p->wmax.p, 0, sizeof(unsigned) * n_mat, s));
        PSPS_CUDA(cudaMemsetAsync(p->xfix.p, 0, sizeof(long long) * (size_t)n_mat * p->n_pix, s));
        {
            const int64_t b = cdiv(p->n_rays, kThreads);
            tile_smax_kernel<<<(unsigned)(b < 1024 ? b : 1024), kThreads, 0, s>>>(sino, p->n_rays, n_mat, p->wmax.p);
            PSPS_LAUNCH_CHECK();
        }
        for (int m0 = 0; m0 < n_mat;) {
            const int nc = n_mat - m0 < 4 ? n_mat - m0 : 4;   // channels of this launch
            const float *sm = sino + (int64_t)m0 * p->n_rays;
            long long *xm = p->xfix.p + (int64_t)m0 * p->n_pix;
            const unsigned *wm = p->wmax.p + m0;
            switch (nc) {
                case 4: back_tile_2d_kernel<4><<<grd, kThreads, 0, s>>>(p->ray.p, p->view.p, p->g, sm, p->n_rays, vs, wm, p->w_max, T, xm); break;
                case 3: back_tile_2d_kernel<3><<<grd, kThreads, 0, s>>>(p->ray.p, p->view.p, p->g, sm, p->n_rays, vs, wm, p->w_max, T, xm); break;
                case 2: back_tile_2d_kernel<2><<<grd, kThreads, 0, s>>>(p->ray.p, p->view.p, p->g, sm, p->n_rays, vs, wm, p->w_max, T, xm); break;
                default: back_tile_2d_kernel<1><<<grd, kThreads, 0, s>>>(p->ray.p, p->view.p, p->g, sm, p->n_rays, vs, wm, p->w_max, T, xm); break;
            }
            PSPS_LAUNCH_CHECK();
            m0 += nc;
        }
        const int64_t b = cdiv(p->n_pix, kThreads);
        fix_to_float_kernel<<<(unsigned)(b < 1024 ? b : 1024), kThreads, 0, s>>>(p->xfix.p, x, p->n_pix, n_mat,
                                                                                  p->wmax.p, p->w_max, T, accumulate);
        PSPS_LAUNCH_CHECK();
        return MBIR_OK;
    }
    const dim3 grd((unsigned)cdiv(p->g.nx, 16), (unsigned)cdiv(p->g.ny, 16));
    for (int m0 = 0; m0 < n_mat;) {
        const int left = n_mat - m0;
        const float *sm = sino + (int64_t)m0 * p->n_rays;
        float *xm = x + (int64_t)m0 * p->n_pix;
        if (left >= 4) {
            back_gather_2d_kernel<4><<<grd, kThreads, 0, s>>>(p->ray.p, p->view.p, p->g, sm, p->n_rays, xm, accumulate);
            m0 += 4;
        } else if (left >= 2) {
            back_gather_2d_kernel<2><<<grd, kThreads, 0, s>>>(p->ray.p, p->view.p, p->g, sm, p->n_rays, xm, accumulate);
            m0 += 2;
        } else {
            back_gather_2d_kernel<1><<<grd, kThreads, 0, s>>>(p->ray.p, p->view.p, p->g, sm, p->n_rays, xm, accumulate);
            m0 += 1;
        }
        PSPS_LAUNCH_CHECK();
    }
    return MBIR_OK;
}

}  // namespace psps

using namespace psps;

extern "C" mbir_status mbir_plan_create(const mbir_geometry *g, int n_mat_max, mbir_plan **out) {
    if (!g || !out) return fail(MBIR_ERR_ARG, "mbir_plan_create: null argument");
    *out = nullptr;
    if (g->kind != MBIR_PAR2D && g->kind != MBIR_FAN2D && g->kind != MBIR_CONE3D)
        return fail(MBIR_ERR_ARG, "mbir_plan_create: unknown geometry kind %d", g->kind);
    const bool cone = g->kind == MBIR_CONE3D;
    if (g->nx < 1 || g->ny < 1 || g->nx > 16384 || g->ny > 16384 || g->n_views < 1 || g->n_u < 1 ||
        (cone && (g->nz < 1 || g->nz > 16384 || g->n_v < 1)))
        return fail(MBIR_ERR_ARG, "mbir_plan_create: bad sizes nx=%d ny=%d nz=%d views=%d n_u=%d n_v=%d", g->nx, g->ny,
                    g->nz, g->n_views, g->n_u, g->n_v);
    if (!(g->dx > 0) || !(g->dy > 0) || !(g->du > 0) || !(g->angle_span != 0) || (cone && (!(g->dz > 0) || !(g->dv > 0))))
        return fail(MBIR_ERR_ARG, "mbir_plan_create: pixel/bin sizes must be > 0 and angle_span != 0");
    if (g->kind == MBIR_FAN2D || cone) {
        const double half = 0.5 * sqrt(g->nx * g->dx * g->nx * g->dx + g->ny * g->dy * g->ny * g->dy);
        if (!(g->sdd > 0) || !(g->sid > half))
            return fail(MBIR_ERR_ARG, "mbir_plan_create: divergent beams need sdd > 0 and the source outside the image");
    }
    if (n_mat_max < 1 || n_mat_max > 8) return fail(MBIR_ERR_ARG, "mbir_plan_create: n_mat_max must be 1..8");
    mbir_plan *p = new mbir_plan();
    p->g = *g;
    if (!cone) p->g.nz = 1, p->g.n_v = 1;
    p->n_mat_max = n_mat_max;
    p->n_rays = (int64_t)p->g.n_views * p->g.n_u * p->g.n_v;
    p->n_pix = (int64_t)p->g.nx * p->g.ny * p->g.nz;
    mbir_status st;
    const int64_t copy = cone ? std::max<int64_t>(p->n_pix * 4, cone_pack_floats(p->g)) : p->n_pix * 4;
    if ((st = p->xcol.alloc(copy)) != MBIR_OK || (st = p->xrow.alloc(copy)) != MBIR_OK ||
        (cone && (st = p->xcol3.alloc(copy)) != MBIR_OK)) {
        delete p;
        return st;
    }
    if (cone) {
        st = cone_setup(p);
        cudaError_t e = cudaDeviceSynchronize();
        if (st == MBIR_OK && e != cudaSuccess) st = fail(MBIR_ERR_CUDA, "mbir_plan_create: %s", cudaGetErrorString(e));
        if (st != MBIR_OK) {
            delete p;
            return st;
        }
        *out = p;
        return MBIR_OK;
    }
    {
        // Rays of one view reaching one tile accumulator: their samples at a
        // fixed driving index lie in a window two pixels wide, and adjacent
        // rays of a view are at least delta pixels apart there: parallel
        // beam du / pixel; fan beam (equiangular bins du / sdd) D du / sdd /
        // pixel with D >= sid - R the distance from the source to any point
        // within a pixel of the grid.
        const double pix = std::max(p->g.dx, p->g.dy);
        double delta = 0.0;
        if (p->g.kind == MBIR_PAR2D) {
            delta = p->g.du / pix;
        } else if (p->g.kind == MBIR_FAN2D && p->g.sdd > 0) {
            const double R = std::hypot((0.5 * p->g.nx + 1.0) * p->g.dx, (0.5 * p->g.ny + 1.0) * p->g.dy);
            if (p->g.sid > R) delta = (p->g.sid - R) * (p->g.du / p->g.sdd) / pix;
        }
        p->cell_rays = delta > 1e-3 ? (int)std::floor(2.0 / delta) + 2 : 0;
    }
    {
        // default views per CTA of the tile transpose: about six CTAs per SM
        // on a 152-SM GPU, between 4 and 60 views (mbir_plan_autotune refines)
        const int64_t tiles = cdiv(p->g.nx, kBT) * cdiv(p->g.ny, kBT);
        const int64_t v = tiles * p->g.n_views / (152 * 6);
        p->back_views = (int)(v < 4 ? 4 : (v > 60 ? 60 : v));
    }
    if ((st = p->ray.alloc(p->n_rays)) != MBIR_OK || (st = p->view.alloc(p->g.n_views)) != MBIR_OK ||
        (st = p->wmax.alloc(n_mat_max)) != MBIR_OK || (st = p->xfix.alloc((size_t)n_mat_max * p->n_pix)) != MBIR_OK) {
        delete p;
        return st;
    }
    setup_2d_kernel<<<(unsigned)cdiv(p->n_rays, kThreads), kThreads>>>(p->g, p->n_rays, p->ray.p);
    setup_view_kernel<<<(unsigned)cdiv(p->g.n_views, 128), 128>>>(p->g, p->view.p);
    cudaMemset(p->wmax.p, 0, sizeof(unsigned));
    ray_wmax_kernel<<<(unsigned)std::min<int64_t>(cdiv(p->n_rays, kThreads), 1024), kThreads>>>(p->ray.p, p->n_rays,
                                                                                              p->wmax.p);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    unsigned wbits = 0u;
    if (e == cudaSuccess) e = cudaMemcpy(&wbits, p->wmax.p, sizeof(unsigned), cudaMemcpyDeviceToHost);
    std::memcpy(&p->w_max, &wbits, sizeof(float));
    if (e != cudaSuccess) {
        delete p;
        return fail(MBIR_ERR_CUDA, "mbir_plan_create: set-up kernel: %s", cudaGetErrorString(e));
    }
    *out = p;
    return MBIR_OK;
}

extern "C" mbir_status mbir_plan_destroy(mbir_plan *p) {
    delete p;
    return MBIR_OK;
}

extern "C" int64_t mbir_plan_n_rays(const mbir_plan *p) { return p ? p->n_rays : -1; }
extern "C" int64_t mbir_plan_n_pix(const mbir_plan *p) { return p ? p->n_pix : -1; }

extern "C" mbir_status mbir_project(mbir_plan *p, const float *x, float *l, int n_mat, mbir_stream s) {
    if (!p || !x || !l) return fail(MBIR_ERR_ARG, "mbir_project: null argument");
    if (n_mat < 1 || n_mat > p->n_mat_max) return fail(MBIR_ERR_ARG, "mbir_project: n_mat %d not in 1..%d", n_mat, p->n_mat_max);
    return project(p, x, l, n_mat, (cudaStream_t)s);
}

extern "C" mbir_status mbir_backproject(mbir_plan *p, const float *sino, float *x, int n_mat, int accumulate,
                                        mbir_stream s) {
    if (!p || !x || !sino) return fail(MBIR_ERR_ARG, "mbir_backproject: null argument");
    if (n_mat < 1 || n_mat > p->n_mat_max)
        return fail(MBIR_ERR_ARG, "mbir_backproject: n_mat %d not in 1..%d", n_mat, p->n_mat_max);
    return backproject(p, sino, x, n_mat, accumulate, (cudaStream_t)s);
}

extern "C" mbir_status mbir_plan_set_backprojector(mbir_plan *p, int mode) {
    if (!p || mode < 0 || mode > (p->g.kind == MBIR_CONE3D ? 3 : 2))
        return fail(MBIR_ERR_ARG, "mbir_plan_set_backprojector: bad argument (0..2; 3 for cone plans)");
    p->back_mode = mode;
    return MBIR_OK;
}

extern "C" mbir_status mbir_plan_set_tiling(mbir_plan *p, int views_per_cta) {
    if (!p || views_per_cta < 1 || views_per_cta > kBVsplit)
        return fail(MBIR_ERR_ARG, "mbir_plan_set_tiling: views_per_cta must be 1..%d", kBVsplit);
    p->back_views = views_per_cta;
    return MBIR_OK;
}

namespace {

// Device time of `reps` calls of fn after one warm-up call (CUDA events on s).
template <class F>
mbir_status time_calls(F &&fn, cudaStream_t s, cudaEvent_t e0, cudaEvent_t e1, int reps, float &ms) {
    PSPS_TRY(fn());
    PSPS_CUDA(cudaEventRecord(e0, s));
    for (int r = 0; r < reps; ++r) PSPS_TRY(fn());
    PSPS_CUDA(cudaEventRecord(e1, s));
    PSPS_CUDA(cudaEventSynchronize(e1));
    PSPS_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    return MBIR_OK;
}

struct EventPair {
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    ~EventPair() {
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
    }
};

mbir_status autotune_impl(mbir_plan *p, int n_channels, cudaStream_t s) {
    EventPair ev;
    PSPS_CUDA(cudaEventCreate(&ev.e0));
    PSPS_CUDA(cudaEventCreate(&ev.e1));
    const int n_fwd = n_channels / 2 > 0 ? n_channels / 2 : 1;   // basis images of a 2 n_mat-channel transpose
    DBuf<float> sino, img;
    PSPS_TRY(sino.alloc((size_t)n_channels * p->n_rays));
    PSPS_TRY(img.alloc((size_t)n_channels * p->n_pix));
    PSPS_CUDA(cudaMemsetAsync(sino.p, 0, sizeof(float) * sino.n, s));
    PSPS_CUDA(cudaMemsetAsync(img.p, 0, sizeof(float) * img.n, s));
    float ms = 0.f, best_ms = 3.0e38f;
    if (p->g.kind == MBIR_CONE3D) {
        // the transpose's algorithm: fixed-point tile scatter (0, where the
        // plan bounds the rays reaching a voxel), direct gather (1) or
        // split-table gather (3)
        // (the tile scatter with tiles 16 or 8 voxels deep)
        int best = p->back_mode, best_tile = p->cone_tile;
        for (int cand : {0, 100, 1, 3}) {
            const int mode = cand == 100 ? 0 : cand;
            if (mode == 0 && p->cell_rays <= 0) continue;
            p->back_mode = mode;
            p->cone_tile = cand == 100 ? 8 : 16;
            PSPS_TRY(time_calls([&] { return backproject(p, sino.p, img.p, n_channels, 0, s); }, s, ev.e0, ev.e1, 1,
                                ms));
            if (ms < best_ms) best_ms = ms, best = mode, best_tile = p->cone_tile;
        }
        p->back_mode = best;
        p->cone_tile = best_tile;
        // the forward's march: each lane from its own range (1) or warp-aligned (2)
        best_ms = 3.0e38f;
        best = p->fwd_mode;
        for (int mode : {1, 2}) {
            p->fwd_mode = mode;
            PSPS_TRY(time_calls([&] { return project(p, img.p, sino.p, n_fwd, s); }, s, ev.e0, ev.e1, 1, ms));
            if (ms < best_ms) best_ms = ms, best = mode;
        }
        p->fwd_mode = best;
        return MBIR_OK;
    }
    // 2-D transpose: views per CTA of the tile kernel
    p->back_mode = 0;
    int best = p->back_views;
    const int cand[] = {4, 8, 15, 30, 45, 60, 90, 120, 180};
    for (int vs : cand) {
        if (vs > p->g.n_views && vs != cand[0]) continue;
        p->back_views = vs;
        PSPS_TRY(time_calls([&] { return backproject(p, sino.p, img.p, n_channels, 0, s); }, s, ev.e0, ev.e1, 3, ms));
        if (ms < best_ms) best_ms = ms, best = vs;
    }
    p->back_views = best;
    // 2-D forward: one thread per ray, or the strip kernel with 32 .. 256
    // bins per CTA
    best_ms = 3.0e38f;
    int best_mode = p->fwd_mode, best_sb = p->strip_bins;
    for (int c = 0; c < 5; ++c) {
        p->fwd_mode = c == 0 ? 1 : 2;
        if (c > 0) p->strip_bins = 16 << c;   // 32, 64, 128, 256
        PSPS_TRY(time_calls([&] { return project(p, img.p, sino.p, n_fwd, s); }, s, ev.e0, ev.e1, 3, ms));
        if (ms < best_ms) best_ms = ms, best_mode = p->fwd_mode, best_sb = p->strip_bins;
    }
    p->fwd_mode = best_mode;
    p->strip_bins = best_sb;
    return MBIR_OK;
}

}  // namespace

extern "C" mbir_status mbir_plan_autotune(mbir_plan *p, int n_channels, mbir_stream stream, int *views_per_cta) {
    if (!p || n_channels < 1 || n_channels > p->n_mat_max)
        return fail(MBIR_ERR_ARG, "mbir_plan_autotune: bad argument (n_channels must be 1..n_mat_max)");
    cudaStream_t s = (cudaStream_t)stream;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    PSPS_CUDA(cudaStreamIsCapturing(s, &cap));
    if (cap != cudaStreamCaptureStatusNone) return fail(MBIR_ERR_ARG, "mbir_plan_autotune: stream is capturing");
    const int back_mode = p->back_mode, back_views = p->back_views, fwd_mode = p->fwd_mode, sb = p->strip_bins;
    const int cone_tile = p->cone_tile;
    const mbir_status st = autotune_impl(p, n_channels, s);
    if (st != MBIR_OK) {   // keep the plan as it was
        p->back_mode = back_mode, p->back_views = back_views, p->fwd_mode = fwd_mode, p->strip_bins = sb;
        p->cone_tile = cone_tile;
        return st;
    }
    if (views_per_cta) *views_per_cta = p->back_views;
    return MBIR_OK;
}

extern "C" mbir_status mbir_plan_set_strip_bins(mbir_plan *p, int bins) {
    if (!p || (bins != 32 && bins != 64 && bins != 128 && bins != 256))
        return fail(MBIR_ERR_ARG, "mbir_plan_set_strip_bins: bins must be 32, 64, 128 or 256");
    p->strip_bins = bins;
    return MBIR_OK;
}

extern "C" mbir_status mbir_plan_set_cone_tile(mbir_plan *p, int depth) {
    if (!p || p->g.kind != MBIR_CONE3D || (depth != 8 && depth != 16))
        return fail(MBIR_ERR_ARG, "mbir_plan_set_cone_tile: a cone plan and a depth of 8 or 16");
    p->cone_tile = depth;
    return MBIR_OK;
}

extern "C" mbir_status mbir_plan_tuning(const mbir_plan *p, int *fwd_mode, int *strip_bins, int *back_mode,
                                        int *back_views, int *cone_tile) {
    if (!p) return fail(MBIR_ERR_ARG, "mbir_plan_tuning: null plan");
    if (fwd_mode) *fwd_mode = p->fwd_mode;
    if (strip_bins) *strip_bins = p->strip_bins;
    if (back_mode) *back_mode = p->back_mode;
    if (back_views) *back_views = p->back_views;
    if (cone_tile) *cone_tile = p->cone_tile;
    return MBIR_OK;
}

extern "C" mbir_status mbir_plan_set_projector(mbir_plan *p, int mode) {
    if (!p || mode < 0 || mode > 2) return fail(MBIR_ERR_ARG, "mbir_plan_set_projector: bad argument");
    p->fwd_mode = mode;
    return MBIR_OK;
}
