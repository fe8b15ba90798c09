// Cone-beam (flat detector) Joseph projector and its transpose on the GPU.
//
// Same method as the 2-D projector: the axis a with the largest |d_a| of the
// ray direction d drives the march (ties: x before y before z), every voxel
// plane i of that axis contributes one bilinear sample in the two other axes
// b, c (b = y for x-driven rays, else x; c = y for z-driven rays, else z),
// zero outside the volume, weight delta_a |d| / |d_a|.
//
// Per-ray set-up in FP32 without cancellation: the crossing of the ray with
// the central plane of its driving axis is written in closed form from the
// source-detector geometry (for an x-driven ray y0 = -sid u / d_x and
// z0 = -sid cos(beta) w / d_x, with u, w the detector offsets), so the
// interpolation coordinates f(i) = f_mid + (i - c_a) df carry no
// large-number rounding.
//
// The set-up runs once per plan and is stored per ray (24 bytes: 1.7 GB for
// 360 x 384 x 512 rays; the central-plane coordinates less 1/2, for the
// conversion-free sample split), so the forward and the transposes read
// bitwise the same interpolation coordinates and weights.
//
// Forward: one thread per ray (neighbouring threads = neighbouring detector
// columns of one row), reading a packed copy of the volume laid out so the
// two interpolated axes are the fastest (b fastest), for each driving axis;
// Kahan-compensated FP32 sums.
//
// Transpose (default): voxel-driven gather, one thread per voxel, no atomics
// (bitwise reproducible), reading a weighted copy of the sinogram with up to
// four channels interleaved per ray (16 bytes per ray of plan scratch).  For every view and every driving axis a that the
// view's rays use, the voxel's bilinear footprint on the plane of its own
// driving index (the voxel centre +- one voxel in the two interpolated axes)
// is projected onto the detector; every detector cell whose centre lies in the
// bounding box of the projected corners is a candidate ray, and a candidate
// contributes exactly the forward's weight of this voxel: its driving axis
// must be a and the ray's sample split must put the voxel on one of its four
// taps.  The ray-driven scatter with global FP32 atomics
// remains as the alternative (mbir_plan_set_backprojector mode 2).
#include <algorithm>
#include <cmath>
#include <type_traits>

#include "common.cuh"

namespace psps {
namespace {

constexpr int kThreads = 256;

struct ConeRay {
    int axis;      // driving axis
    int lo, hi;    // driving index range that can touch the volume
    float fb_mid, dfb, fc_mid, dfc, ca, w;
};

__device__ __forceinline__ void range_1d(float f_mid, float df, float ca, int n_other, int n_drive, float &lo,
                                         float &hi) {
    // indices i with f_mid + (i - ca) df in (-1, n_other)
    if (df == 0.f) {
        if (f_mid > -1.f && f_mid < (float)n_other) {
            lo = 0.f;
            hi = (float)(n_drive - 1);
        } else {
            lo = 1.f;
            hi = 0.f;
        }
        return;
    }
    float t0 = (-1.f - f_mid) / df + ca, t1 = ((float)n_other - f_mid) / df + ca;
    if (t0 > t1) {
        const float t = t0;
        t0 = t1;
        t1 = t;
    }
    lo = fmaxf(t0, -1.0e8f);
    hi = fminf(t1, 1.0e8f);
}

__device__ __forceinline__ ConeRay cone_ray(const mbir_geometry &g, float4 V, int iu, int iv) {
    // V = (sx, sy, cos beta, sin beta)
    const float u = (float)((iu - 0.5 * (g.n_u - 1)) * g.du), w = (float)((iv - 0.5 * (g.n_v - 1)) * g.dv);
    const float sdd = (float)g.sdd, sid = (float)g.sid;
    const float d0 = -sdd * V.z - u * V.w, d1 = -sdd * V.w + u * V.z, d2 = w;
    const float a0 = fabsf(d0), a1 = fabsf(d1), a2 = fabsf(d2);
    const float nd = sqrtf(d0 * d0 + d1 * d1 + d2 * d2);
    const float dx = (float)g.dx, dy = (float)g.dy, dz = (float)g.dz;
    const float cx = 0.5f * (g.nx - 1), cy = 0.5f * (g.ny - 1), cz = 0.5f * (g.nz - 1);
    ConeRay r;
    if (a0 >= a1 && a0 >= a2) {
        r.axis = 0;
        const float y0 = -sid * u / d0, z0 = -sid * V.z * w / d0;
        r.fb_mid = y0 / dy + cy;
        r.dfb = dx * (d1 / d0) / dy;
        r.fc_mid = z0 / dz + cz;
        r.dfc = dx * (d2 / d0) / dz;
        r.ca = cx;
        r.w = dx * nd / a0;
    } else if (a1 >= a2) {
        r.axis = 1;
        const float x0 = sid * u / d1, z0 = -sid * V.w * w / d1;
        r.fb_mid = x0 / dx + cx;
        r.dfb = dy * (d0 / d1) / dx;
        r.fc_mid = z0 / dz + cz;
        r.dfc = dy * (d2 / d1) / dz;
        r.ca = cy;
        r.w = dy * nd / a1;
    } else {
        r.axis = 2;
        // crossing of the source plane z = 0: the source itself
        r.fb_mid = V.x / dx + cx;
        r.dfb = dz * (d0 / d2) / dx;
        r.fc_mid = V.y / dy + cy;
        r.dfc = dz * (d1 / d2) / dy;
        r.ca = cz;   // plane z = 0 is index cz; the source sits there
        r.w = dz * nd / a2;
    }
    const int na = r.axis == 0 ? g.nx : (r.axis == 1 ? g.ny : g.nz);
    const int nb = r.axis == 0 ? g.ny : g.nx;
    const int nc = r.axis == 2 ? g.ny : g.nz;
    float l0, h0, l1, h1;
    range_1d(r.fb_mid, r.dfb, r.ca, nb, na, l0, h0);
    range_1d(r.fc_mid, r.dfc, r.ca, nc, na, l1, h1);
    const float lo = fmaxf(fmaxf(l0, l1), 0.f), hi = fminf(fminf(h0, h1), (float)(na - 1));
    r.lo = (int)floorf(lo) - 1;
    r.hi = (int)ceilf(hi) + 1;
    if (r.lo < 0) r.lo = 0;
    if (r.hi > na - 1) r.hi = na - 1;
    return r;
}

__global__ void setup_view3d_kernel(mbir_geometry g, float4 *vt) {
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= g.n_views) return;
    const double ang = g.angle0 + v * (g.angle_span / g.n_views);
    double s, c;
    sincos(ang, &s, &c);
    vt[v] = make_float4((float)(g.sid * c), (float)(g.sid * s), (float)c, (float)s);
}

__global__ void setup_rays3d_kernel(mbir_geometry g, const float4 *__restrict__ vt, int64_t n_rays,
                                    float4 *__restrict__ ta, float2 *__restrict__ tb, int *__restrict__ view_axes) {
    const int64_t ray = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (ray >= n_rays) return;
    const int per_view = g.n_u * g.n_v;
    const int v = (int)(ray / per_view);
    const int rem = (int)(ray % per_view);
    const ConeRay r = cone_ray(g, vt[v], rem % g.n_u, rem / g.n_u);
    ta[ray] = make_float4(r.fb_mid - 0.5f, r.dfb, r.fc_mid - 0.5f, r.dfc);
    const bool empty = r.lo > r.hi;
    const int bits = r.axis | ((empty ? 1 : r.lo) << 2) | ((empty ? 0 : r.hi) << 17);
    tb[ray] = make_float2(r.w, __int_as_float(bits));
    if (!empty) atomicOr(view_axes + v, 1 << r.axis);
}

__device__ __forceinline__ void decode3(float2 b, int &axis, int &lo, int &hi) {
    const int bits = __float_as_int(b.y);
    axis = bits & 3;
    lo = (bits >> 2) & 0x7fff;
    hi = (bits >> 17) & 0x7fff;
}

// Packed copies of x[m][z][y][x] for the three driving axes, materials
// innermost with stride P: layout[a][c][b][m] (see the file comment), each
// plane of the driving axis with kPad zero cells on both sides of b and c,
// so that every tap of every sample a ray's range can take lies inside the
// copy and reads the value or a zero (no bounds tests in the forward).
constexpr int kPad = 2;

__host__ __device__ inline int64_t pack3d_floats(int nx, int ny, int nz) {
    const int64_t a = (int64_t)nx * (nz + 2 * kPad) * (ny + 2 * kPad);   // a = x: [ix][iz][iy]
    const int64_t b = (int64_t)ny * (nz + 2 * kPad) * (nx + 2 * kPad);   // a = y: [iy][iz][ix]
    const int64_t c = (int64_t)nz * (ny + 2 * kPad) * (nx + 2 * kPad);   // a = z: [iz][iy][ix]
    return 4 * (a > b ? (a > c ? a : c) : (b > c ? b : c));
}

// Zero the kPad-wide borders of the three packed copies (the interiors are
// written by pack3d_kernel), P floats per cell.
__global__ void pack3d_border_kernel(int P, int nx, int ny, int nz, float *__restrict__ ox, float *__restrict__ oy,
                                     float *__restrict__ oz) {
    const int W = 2 * kPad;
    for (int a = 0; a < 3; ++a) {
        const int na = a == 0 ? nx : (a == 1 ? ny : nz);
        const int nb = a == 0 ? ny : nx, nc = a == 2 ? ny : nz;
        const int64_t plane = (int64_t)(nc + W) * (nb + W);
        float *o = a == 0 ? ox : (a == 1 ? oy : oz);
        const int64_t n = (int64_t)na * plane;
        for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
            const int rem = (int)(k % plane);
            const int c = rem / (nb + W), b = rem % (nb + W);
            if (c >= kPad && c < nc + kPad && b >= kPad && b < nb + kPad) continue;
            for (int m = 0; m < P; ++m) o[k * P + m] = 0.f;
        }
    }
}

__global__ void pack3d_kernel(const float *__restrict__ x, int nm, int P, int nx, int ny, int nz,
                              float *__restrict__ ox, float *__restrict__ oy, float *__restrict__ oz) {
    const int64_t n = (int64_t)nx * ny * nz;
    const int W = 2 * kPad;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
        const int ix = (int)(j % nx);
        const int iy = (int)((j / nx) % ny);
        const int iz = (int)(j / ((int64_t)nx * ny));
        const int64_t px = (((int64_t)ix * (nz + W) + iz + kPad) * (ny + W) + iy + kPad) * P;   // [ix][iz][iy]
        const int64_t py = (((int64_t)iy * (nz + W) + iz + kPad) * (nx + W) + ix + kPad) * P;   // [iy][iz][ix]
        const int64_t pz = (((int64_t)iz * (ny + W) + iy + kPad) * (nx + W) + ix + kPad) * P;   // [iz][iy][ix]
        for (int m = 0; m < P; ++m) {
            const float v = m < nm ? x[m * n + j] : 0.f;
            ox[px + m] = v;
            oy[py + m] = v;
            oz[pz + m] = v;
        }
    }
}

template <int NM>
struct P3;
template <>
struct P3<1> {
    using T = float;
    __device__ static void get(const T &v, float (&o)[1]) { o[0] = v; }
};
template <>
struct P3<2> {
    using T = float2;
    __device__ static void get(const T &v, float (&o)[2]) {
        o[0] = v.x;
        o[1] = v.y;
    }
};
template <>
struct P3<4> {
    using T = float4;
    __device__ static void get(const T &v, float (&o)[4]) {
        o[0] = v.x;
        o[1] = v.y;
        o[2] = v.z;
        o[3] = v.w;
    }
};

// ALIGNED: the lanes of a warp (neighbouring detector columns of one row)
// step the same driving index over the union of their ranges, each adding
// only inside its own range, so that one load instruction of the warp reads
// neighbouring voxels of one plane (a few cache lines) instead of one plane
// per lane.  Same samples, weights and summation order either way.
template <int NM, bool ALIGNED>
__global__ void __launch_bounds__(kThreads)
    fwd_cone_kernel(mbir_geometry g, const float4 *__restrict__ ta, const float2 *__restrict__ tb,
                    const typename P3<NM>::T *__restrict__ ox, const typename P3<NM>::T *__restrict__ oy,
                    const typename P3<NM>::T *__restrict__ oz, int nm, int64_t n_rays, float *__restrict__ l) {
    const int64_t ray = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (ALIGNED) {
        if (((int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31)) >= n_rays) return;   // whole warp past the end
    } else if (ray >= n_rays) {
        return;
    }
    const bool live = ray < n_rays;
    const float4 A = live ? ta[ray] : make_float4(0.f, 0.f, 0.f, 0.f);
    const float2 B = live ? tb[ray] : make_float2(0.f, __int_as_float(1 << 2));   // empty range lo 1 > hi 0
    int axis, lo, hi;
    decode3(B, axis, lo, hi);
    int i_lo = lo, i_hi = hi;
    if (ALIGNED) {
        // rays that miss the volume (lo > hi) do not widen the warp's range
        if (lo > hi) i_lo = 0x7fffffff, i_hi = -1;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            i_lo = min(i_lo, __shfl_xor_sync(0xffffffffu, i_lo, o));
            i_hi = max(i_hi, __shfl_xor_sync(0xffffffffu, i_hi, o));
        }
    }
    const typename P3<NM>::T *src = axis == 0 ? ox : (axis == 1 ? oy : oz);
    // padded plane: (nc + 2 kPad) rows of (nb + 2 kPad) cells.  A sample's
    // lower tap indices are clamped to [-kPad, n + kPad - 2]: a sample the
    // clamp moves lies wholly outside the volume (its taps are at <= -2 or
    // >= n), and the clamped taps then read border zeros, as the true ones
    // are; every other sample reads its own taps.
    const int nb = axis == 0 ? g.ny : g.nx, nc = axis == 2 ? g.ny : g.nz;
    const int nbp = nb + 2 * kPad, ncp = nc + 2 * kPad;
    const float ca = 0.5f * ((axis == 0 ? g.nx : (axis == 1 ? g.ny : g.nz)) - 1);
    float acc[NM], comp[NM];
#pragma unroll
    for (int m = 0; m < NM; ++m) acc[m] = comp[m] = 0.f;
    int i = i_lo;
    if (!ALIGNED) {
        // Two samples per step: their eight tap loads (addresses clamped into
        // the volume, values zeroed outside it) are issued before use; the
        // taps and samples are then added in the one-at-a-time order.
        using T = typename P3<NM>::T;
        for (; i + 1 <= i_hi; i += 2) {
            T v[2][4];
            float gb[2], gc[2];
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                const float t = (float)(i + u) - ca;
                const int ib0 = joseph_split(fmaf(t, A.y, A.x), gb[u]), ic0 = joseph_split(fmaf(t, A.w, A.z), gc[u]);
                const int ibc = min(max(ib0, -kPad), nb + kPad - 2), icc = min(max(ic0, -kPad), nc + kPad - 2);
                const T *tap = src + ((int64_t)(i + u) * ncp + icc + kPad) * nbp + ibc + kPad;
                v[u][0] = __ldg(tap);
                v[u][1] = __ldg(tap + 1);
                v[u][2] = __ldg(tap + nbp);
                v[u][3] = __ldg(tap + nbp + 1);
            }
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                float sm[NM];
#pragma unroll
                for (int m = 0; m < NM; ++m) sm[m] = 0.f;
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const float wc = (q >> 1) ? gc[u] : 1.f - gc[u];
                    const float wbc = ((q & 1) ? gb[u] : 1.f - gb[u]) * wc;
                    float val[NM];
                    P3<NM>::get(v[u][q], val);
#pragma unroll
                    for (int m = 0; m < NM; ++m) sm[m] = fmaf(wbc, val[m], sm[m]);
                }
#pragma unroll
                for (int m = 0; m < NM; ++m) {
                    const float yk = __fsub_rn(sm[m], comp[m]);
                    const float tt = __fadd_rn(acc[m], yk);
                    comp[m] = __fsub_rn(__fsub_rn(tt, acc[m]), yk);
                    acc[m] = tt;
                }
            }
        }
    }
    for (; i <= i_hi; ++i) {
        if (ALIGNED && (i < lo || i > hi)) continue;
        const float t = (float)i - ca;
        float gb, gc;
        const int ib0 = joseph_split(fmaf(t, A.y, A.x), gb), ic0 = joseph_split(fmaf(t, A.w, A.z), gc);
        float s[NM];
#pragma unroll
        for (int m = 0; m < NM; ++m) s[m] = 0.f;
        const int ibc = min(max(ib0, -kPad), nb + kPad - 2), icc = min(max(ic0, -kPad), nc + kPad - 2);
        const typename P3<NM>::T *tap = src + ((int64_t)i * ncp + icc + kPad) * nbp + ibc + kPad;
#pragma unroll
        for (int jc = 0; jc < 2; ++jc) {
            const float wc = jc ? gc : 1.f - gc;
#pragma unroll
            for (int jb = 0; jb < 2; ++jb) {
                const float wbc = (jb ? gb : 1.f - gb) * wc;
                float val[NM];
                P3<NM>::get(__ldg(tap + jc * nbp + jb), val);
#pragma unroll
                for (int m = 0; m < NM; ++m) s[m] = fmaf(wbc, val[m], s[m]);
            }
        }
#pragma unroll
        for (int m = 0; m < NM; ++m) {
            const float yk = __fsub_rn(s[m], comp[m]);
            const float tt = __fadd_rn(acc[m], yk);
            comp[m] = __fsub_rn(__fsub_rn(tt, acc[m]), yk);
            acc[m] = tt;
        }
    }
    if (!live) return;
#pragma unroll
    for (int m = 0; m < NM; ++m)
        if (m < nm) l[(int64_t)m * n_rays + ray] = acc[m] * B.x;
}

__global__ void __launch_bounds__(kThreads)
    back_cone_kernel(mbir_geometry g, const float4 *__restrict__ ta, const float2 *__restrict__ tb,
                     const float *__restrict__ sino, int nm, int64_t n_rays, float *__restrict__ x) {
    const int64_t ray = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (ray >= n_rays) return;
    const float4 A = ta[ray];
    const float2 B = tb[ray];
    ConeRay r;
    decode3(B, r.axis, r.lo, r.hi);
    r.fb_mid = A.x, r.dfb = A.y, r.fc_mid = A.z, r.dfc = A.w, r.w = B.x;
    r.ca = 0.5f * ((r.axis == 0 ? g.nx : (r.axis == 1 ? g.ny : g.nz)) - 1);
    const int nb = r.axis == 0 ? g.ny : g.nx;
    const int nc = r.axis == 2 ? g.ny : g.nz;
    // voxel strides of the driving axis and the two interpolated axes in x[z][y][x]
    const int64_t sx = 1, sy = g.nx, sz = (int64_t)g.nx * g.ny;
    const int64_t sa = r.axis == 0 ? sx : (r.axis == 1 ? sy : sz);
    const int64_t sb = r.axis == 0 ? sy : sx;
    const int64_t sc = r.axis == 2 ? sy : sz;
    const int64_t npix = (int64_t)g.nx * g.ny * g.nz;
    for (int m = 0; m < nm; ++m) {
        const float ws = r.w * sino[(int64_t)m * n_rays + ray];
        if (ws == 0.f) continue;
        float *img = x + m * npix;
        for (int i = r.lo; i <= r.hi; ++i) {
            const float t = (float)i - r.ca;
            float gb, gc;
            const int ib0 = joseph_split(fmaf(t, r.dfb, r.fb_mid), gb), ic0 = joseph_split(fmaf(t, r.dfc, r.fc_mid), gc);
            for (int jc = 0; jc < 2; ++jc) {
                const int ic = ic0 + jc;
                if (ic < 0 || ic >= nc) continue;
                const float wc = jc ? gc : 1.f - gc;
                for (int jb = 0; jb < 2; ++jb) {
                    const int ib = ib0 + jb;
                    if (ib < 0 || ib >= nb) continue;
                    atomicAdd(img + i * sa + ib * sb + ic * sc, (jb ? gb : 1.f - gb) * wc * ws);
                }
            }
        }
    }
}

template <int C>
struct Vec;
template <>
struct Vec<1> {
    using T = float;
    __device__ static void get(const T &v, float (&o)[1]) { o[0] = v; }
    __device__ static void put(T &v, const float (&o)[1]) { v = o[0]; }
};
template <>
struct Vec<2> {
    using T = float2;
    __device__ static void get(const T &v, float (&o)[2]) { o[0] = v.x, o[1] = v.y; }
    __device__ static void put(T &v, const float (&o)[2]) { v = make_float2(o[0], o[1]); }
};
template <>
struct Vec<4> {
    using T = float4;
    __device__ static void get(const T &v, float (&o)[4]) { o[0] = v.x, o[1] = v.y, o[2] = v.z, o[3] = v.w; }
    __device__ static void put(T &v, const float (&o)[4]) { v = make_float4(o[0], o[1], o[2], o[3]); }
};

// Weighted sinogram for the transposes: ws[ray][c] = w_ray * sino[c][ray],
// channels interleaved (C = 1, 2 or 4 floats per ray, one vector store;
// channels past nc are 0).  smax (optional, zeroed by the caller): per
// channel max_ray |ws| as float bits (atomicMax on the bits orders
// non-negative floats; a NaN makes it NaN bits, above every finite value).
template <int C>
__global__ void weigh_sino_kernel(const float2 *__restrict__ tb, const float *__restrict__ sino, int nc,
                                  int64_t n_rays, typename Vec<C>::T *__restrict__ ws, unsigned *__restrict__ smax) {
    unsigned mx[C];
#pragma unroll
    for (int c = 0; c < C; ++c) mx[c] = 0u;
    for (int64_t ray = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; ray < n_rays;
         ray += (int64_t)gridDim.x * blockDim.x) {
        const float w = tb[ray].x;
        float v[C];
#pragma unroll
        for (int c = 0; c < C; ++c) {
            v[c] = c < nc ? w * __ldg(sino + (int64_t)c * n_rays + ray) : 0.f;
            const float a = fabsf(v[c]);
            const unsigned bits = a != a ? 0x7fc00000u : __float_as_uint(a);
            mx[c] = bits > mx[c] ? bits : mx[c];
        }
        Vec<C>::put(ws[ray], v);
    }
    if (!smax) return;
#pragma unroll
    for (int c = 0; c < C; ++c) {
        const unsigned m = __reduce_max_sync(0xffffffffu, mx[c]);
        if ((threadIdx.x & 31) == 0 && m) atomicMax(smax + c, m);
    }
}

// Detector cells whose centres lie in the bounding box of the projections of
// points (x, y, z) with x in {xs}, y in {ys}, z in {zs} (2 values each) for
// view V (widened by 1e-3 of a cell for rounding; a ray outside the box has
// no point in the footprint), clipped to the detector; false if a point
// reaches the source plane (then the whole detector is returned).  NXY:
// distinct (x, y) corners (2 when xs or ys holds one value twice, as in a
// voxel's footprint for x- or y-driven rays; otherwise 4).
template <int NXY>
__device__ __forceinline__ bool footprint_box(const mbir_geometry &g, const float4 &V, const float (&xs)[2],
                                              const float (&ys)[2], const float (&zs)[2], int &iu0, int &iu1,
                                              int &iv0, int &iv1) {
    const float sdd = (float)g.sdd;
    float umin = 3.0e38f, umax = -3.0e38f, imin = 3.0e38f, imax = -3.0e38f;
    bool behind = false;
#pragma unroll
    for (int k = 0; k < NXY; ++k) {
        const float qx = xs[NXY == 4 ? (k & 1) : k] - V.x, qy = ys[NXY == 4 ? (k >> 1) : k] - V.y;
        const float depth = -(qx * V.z + qy * V.w);   // along the central ray, source to detector
        if (!(depth > 0.f)) behind = true;
        const float inv = sdd / depth;
        const float u = (-qx * V.w + qy * V.z) * inv;
        umin = fminf(umin, u), umax = fmaxf(umax, u), imin = fminf(imin, inv), imax = fmaxf(imax, inv);
    }
    if (behind) {
        iu0 = 0, iu1 = g.n_u - 1, iv0 = 0, iv1 = g.n_v - 1;
        return false;
    }
    // w = z * sdd / depth over the z values and the corner magnifications
    const float wmin = fminf(fminf(zs[0] * imin, zs[0] * imax), fminf(zs[1] * imin, zs[1] * imax));
    const float wmax = fmaxf(fmaxf(zs[0] * imin, zs[0] * imax), fmaxf(zs[1] * imin, zs[1] * imax));
    const float inv_du = (float)(1.0 / g.du), inv_dv = (float)(1.0 / g.dv);
    const float cu = 0.5f * (g.n_u - 1), cv = 0.5f * (g.n_v - 1);
    constexpr float eps = 1.0e-3f;
    iu0 = max((int)ceilf(fmaxf(umin * inv_du + cu - eps, -2.0e9f)), 0);
    iu1 = min((int)floorf(fminf(umax * inv_du + cu + eps, 2.0e9f)), g.n_u - 1);
    iv0 = max((int)ceilf(fmaxf(wmin * inv_dv + cv - eps, -2.0e9f)), 0);
    iv1 = min((int)floorf(fminf(wmax * inv_dv + cv + eps, 2.0e9f)), g.n_v - 1);
    return true;
}

// The footprint of voxel (px, py, pz) for rays driven along A: its own
// coordinate along A, +- one voxel along the two interpolated axes; for
// A = 0 / 1 the two (x, y) corners are (px, py -+ dy) / (px -+ dx, py).
template <int A>
__device__ __forceinline__ void voxel_footprint(const mbir_geometry &g, float px, float py, float pz, float (&xs)[2],
                                                float (&ys)[2], float (&zs)[2]) {
    const float dx = (float)g.dx, dy = (float)g.dy, dz = (float)g.dz;
    xs[0] = xs[1] = px, ys[0] = ys[1] = py, zs[0] = zs[1] = pz;
    if (A != 0) xs[0] = px - dx, xs[1] = px + dx;
    if (A != 1) ys[0] = py - dy, ys[1] = py + dy;
    if (A != 2) zs[0] = pz - dz, zs[1] = pz + dz;
}

// Adds the weights of the candidate rays in cells [iu0, iu1] x [iv0, iv1] of
// view v to sv.  Ray data come either from global memory (stage == nullptr)
// or from a shared-memory copy of the box [su0, su0 + sw) x [sv0, ...)
// (ray parameters, weighted channels and, for mixed views, axes).
template <int A, int C>
__device__ __forceinline__ void gather_cells(const mbir_geometry &g, int v, int ix, int iy, int iz, int iu0, int iu1,
                                             int iv0, int iv1, bool check_axis, const float4 *__restrict__ ta,
                                             const int *__restrict__ tbits, const typename Vec<C>::T *__restrict__ ws,
                                             const float4 *s_ta, const typename Vec<C>::T *s_ws, const int *s_ax,
                                             int su0, int sv0, int sw, float (&sv)[C]) {
    const int id = A == 0 ? ix : (A == 1 ? iy : iz);                   // driving index
    const int ib = A == 0 ? iy : ix, ic = A == 2 ? iy : iz;            // interpolated indices
    const float t = (float)id - 0.5f * ((A == 0 ? g.nx : (A == 1 ? g.ny : g.nz)) - 1);
    const int64_t view0 = (int64_t)v * g.n_u * g.n_v;
    for (int jv = iv0; jv <= iv1; ++jv) {
        for (int ju = iu0; ju <= iu1; ++ju) {
            float4 R;
            float val[C];
            if (s_ta) {
                const int k = (jv - sv0) * sw + (ju - su0);
                if (check_axis && s_ax[k] != A) continue;
                R = s_ta[k];
                Vec<C>::get(s_ws[k], val);
            } else {
                const int64_t ray = view0 + (int64_t)jv * g.n_u + ju;
                if (check_axis && (__ldg(tbits + 2 * ray + 1) & 3) != A) continue;
                R = __ldg(ta + ray);
                Vec<C>::get(__ldg(ws + ray), val);
            }
            float gb, gc;
            const int db = ib - joseph_split(fmaf(t, R.y, R.x), gb), dc = ic - joseph_split(fmaf(t, R.w, R.z), gc);
            if ((unsigned)db > 1u || (unsigned)dc > 1u) continue;
            const float wbc = (db ? gb : 1.f - gb) * (dc ? gc : 1.f - gc);
#pragma unroll
            for (int c = 0; c < C; ++c) sv[c] = fmaf(wbc, val[c], sv[c]);
        }
    }
}

// Voxel-driven exact transpose (see the file comment).  A CTA owns a tile of
// kGX x kGY x kGZ voxels; for every view and driving axis (x or y) it stages
// the rays of the detector box that covers the whole tile's footprint in
// shared memory once, and every thread gathers its own voxel's candidates
// from that copy (rays driven along z, and boxes larger than the staging
// area, are read from global memory instead).  C channels per launch from
// the weighted interleaved sinogram; the candidates of one view are summed
// in FP32 and the per-view sums Kahan-compensated; x[c] is written (or
// added to) for c < nc.
constexpr int kGX = 4, kGY = 4, kGZ = 16;   // 256 voxels per CTA
constexpr int kStageCap = 640;              // staged detector cells per view

template <int C>
__global__ void __launch_bounds__(kGX * kGY * kGZ, 4)
    back_cone_gather_kernel(mbir_geometry g, const float4 *__restrict__ vt, const float4 *__restrict__ ta,
                            const float2 *__restrict__ tb, const int *__restrict__ view_axes,
                            const typename Vec<C>::T *__restrict__ ws, int nc, float *__restrict__ x,
                            int accumulate) {
    __shared__ float4 s_ta[kStageCap];
    __shared__ typename Vec<C>::T s_ws[kStageCap];
    __shared__ int s_ax[kStageCap];
    __shared__ int s_box[5];
    const int tid = threadIdx.x;
    const int x0 = blockIdx.x * kGX, y0 = blockIdx.y * kGY, z0 = blockIdx.z * kGZ;
    const int ix = x0 + tid % kGX, iy = y0 + (tid / kGX) % kGY, iz = z0 + tid / (kGX * kGY);
    const bool inside = ix < g.nx && iy < g.ny && iz < g.nz;
    const float dx = (float)g.dx, dy = (float)g.dy, dz = (float)g.dz;
    const float cx = 0.5f * (g.nx - 1), cy = 0.5f * (g.ny - 1), cz = 0.5f * (g.nz - 1);
    const float px = (ix - cx) * dx, py = (iy - cy) * dy, pz = (iz - cz) * dz;
    // the tile's voxel-centre extent (clipped to the volume)
    const float tx0 = (x0 - cx) * dx, tx1 = (min(x0 + kGX, g.nx) - 1 - cx) * dx;
    const float ty0 = (y0 - cy) * dy, ty1 = (min(y0 + kGY, g.ny) - 1 - cy) * dy;
    const float tz0 = (z0 - cz) * dz, tz1 = (min(z0 + kGZ, g.nz) - 1 - cz) * dz;
    const int *tbits = reinterpret_cast<const int *>(tb);  // (w, bits) pairs: bits at odd indices
    float acc[C], comp[C];
#pragma unroll
    for (int c = 0; c < C; ++c) acc[c] = comp[c] = 0.f;
    for (int v = 0; v < g.n_views; ++v) {
        const int axes = view_axes[v];
        if (!axes) continue;
        const float4 V = vt[v];  // (sx, sy, cos beta, sin beta)
        const bool mixed = (axes & (axes - 1)) != 0;
        const int64_t view0 = (int64_t)v * g.n_u * g.n_v;
        float sv[C];
#pragma unroll
        for (int c = 0; c < C; ++c) sv[c] = 0.f;
#pragma unroll
        for (int A = 0; A < 3; ++A) {
            if (!((axes >> A) & 1)) continue;
            // this voxel's candidate box
            float xs[2], ys[2], zs[2];
            int iu0, iu1, iv0, iv1;
            if (A == 0) {
                voxel_footprint<0>(g, px, py, pz, xs, ys, zs);
                footprint_box<2>(g, V, xs, ys, zs, iu0, iu1, iv0, iv1);
            } else if (A == 1) {
                voxel_footprint<1>(g, px, py, pz, xs, ys, zs);
                footprint_box<2>(g, V, xs, ys, zs, iu0, iu1, iv0, iv1);
            } else {
                voxel_footprint<2>(g, px, py, pz, xs, ys, zs);
                footprint_box<4>(g, V, xs, ys, zs, iu0, iu1, iv0, iv1);
            }
            // the tile's box (same for every thread of the CTA: thread 0
            // computes it; the barrier below publishes it)
            __syncthreads();   // previous readers of the staging area and the box are done
            if (tid == 0) {
                int b0 = 0, b1 = -1, b2 = 0, b3 = -1;
                bool ok = false;
                if (A != 2) {
                    const float txs[2] = {A == 0 ? tx0 : tx0 - dx, A == 0 ? tx1 : tx1 + dx};
                    const float tys[2] = {A == 1 ? ty0 : ty0 - dy, A == 1 ? ty1 : ty1 + dy};
                    const float tzs[2] = {tz0 - dz, tz1 + dz};
                    ok = footprint_box<4>(g, V, txs, tys, tzs, b0, b1, b2, b3) &&
                         (b1 - b0 + 1) * (b3 - b2 + 1) <= kStageCap;
                }
                s_box[0] = b0, s_box[1] = b1, s_box[2] = b2, s_box[3] = b3, s_box[4] = ok;
            }
            __syncthreads();
            const int su0 = s_box[0], su1 = s_box[1], sv0 = s_box[2], sv1 = s_box[3];
            const bool staged = s_box[4] != 0;
            const int sw = su1 - su0 + 1;
            if (staged) {
                const int n = sw * (sv1 - sv0 + 1);
                for (int k = tid; k < n; k += blockDim.x) {
                    const int64_t ray = view0 + (int64_t)(sv0 + k / sw) * g.n_u + su0 + k % sw;
                    s_ta[k] = __ldg(ta + ray);
                    s_ws[k] = __ldg(ws + ray);
                    if (mixed) s_ax[k] = __ldg(tbits + 2 * ray + 1) & 3;
                }
                __syncthreads();
                iu0 = max(iu0, su0), iu1 = min(iu1, su1), iv0 = max(iv0, sv0), iv1 = min(iv1, sv1);
            }
            if (!inside) continue;
            if (A == 0)
                gather_cells<0, C>(g, v, ix, iy, iz, iu0, iu1, iv0, iv1, mixed, ta, tbits, ws,
                                   staged ? s_ta : nullptr, s_ws, s_ax, su0, sv0, sw, sv);
            else if (A == 1)
                gather_cells<1, C>(g, v, ix, iy, iz, iu0, iu1, iv0, iv1, mixed, ta, tbits, ws,
                                   staged ? s_ta : nullptr, s_ws, s_ax, su0, sv0, sw, sv);
            else
                gather_cells<2, C>(g, v, ix, iy, iz, iu0, iu1, iv0, iv1, mixed, ta, tbits, ws, nullptr, s_ws, s_ax,
                                   su0, sv0, sw, sv);
        }
#pragma unroll
        for (int c = 0; c < C; ++c) {
            const float yk = __fsub_rn(sv[c], comp[c]);
            const float tt = __fadd_rn(acc[c], yk);
            comp[c] = __fsub_rn(__fsub_rn(tt, acc[c]), yk);
            acc[c] = tt;
        }
    }
    if (!inside) return;
    const int64_t npix = (int64_t)g.nx * g.ny * g.nz;
    const int64_t j = ((int64_t)iz * g.ny + iy) * g.nx + ix;
#pragma unroll
    for (int c = 0; c < C; ++c) {
        if (c >= nc) break;
        float *o = x + (int64_t)c * npix + j;
        *o = accumulate ? *o + acc[c] : acc[c];
    }
}

// The detector box of the whole tile's footprint for driving axis A != 2,
// computed by the lanes of one warp (lanes 0-3 project one corner each) and
// shared by shuffles, so no barrier is needed for it: every warp gets the
// same box.  Same bounds as footprint_box<4> of the tile corners.
template <int A>
__device__ __forceinline__ bool tile_box_warp(const mbir_geometry &g, const float4 &V, float tx0, float tx1, float ty0,
                                              float ty1, float tz0, float tz1, int &iu0, int &iu1, int &iv0,
                                              int &iv1) {
    const float dx = (float)g.dx, dy = (float)g.dy, dz = (float)g.dz;
    const int lane = threadIdx.x & 31;
    const float xa = A == 0 ? tx0 : tx0 - dx, xb = A == 0 ? tx1 : tx1 + dx;
    const float ya = A == 1 ? ty0 : ty0 - dy, yb = A == 1 ? ty1 : ty1 + dy;
    const int k = lane & 3;
    const float qx = ((k & 1) ? xb : xa) - V.x, qy = ((k >> 1) ? yb : ya) - V.y;
    const float depth = -(qx * V.z + qy * V.w);
    const float inv = (float)g.sdd / depth;
    float u = (-qx * V.w + qy * V.z) * inv;
    float umin = u, umax = u, imin = inv, imax = inv;
    int behind = depth > 0.f ? 0 : 1;
#pragma unroll
    for (int o = 1; o <= 2; o <<= 1) {
        umin = fminf(umin, __shfl_xor_sync(0xffffffffu, umin, o));
        umax = fmaxf(umax, __shfl_xor_sync(0xffffffffu, umax, o));
        imin = fminf(imin, __shfl_xor_sync(0xffffffffu, imin, o));
        imax = fmaxf(imax, __shfl_xor_sync(0xffffffffu, imax, o));
        behind |= __shfl_xor_sync(0xffffffffu, behind, o);
    }
    if (behind) return false;
    const float za = tz0 - dz, zb = tz1 + dz;
    const float wmin = fminf(fminf(za * imin, za * imax), fminf(zb * imin, zb * imax));
    const float wmax = fmaxf(fmaxf(za * imin, za * imax), fmaxf(zb * imin, zb * imax));
    const float inv_du = (float)(1.0 / g.du), inv_dv = (float)(1.0 / g.dv);
    const float cu = 0.5f * (g.n_u - 1), cv = 0.5f * (g.n_v - 1);
    constexpr float eps = 1.0e-3f;
    iu0 = max((int)ceilf(fmaxf(umin * inv_du + cu - eps, -2.0e9f)), 0);
    iu1 = min((int)floorf(fminf(umax * inv_du + cu + eps, 2.0e9f)), g.n_u - 1);
    iv0 = max((int)ceilf(fmaxf(wmin * inv_dv + cv - eps, -2.0e9f)), 0);
    iv1 = min((int)floorf(fminf(wmax * inv_dv + cv + eps, 2.0e9f)), g.n_v - 1);
    return true;
}

// Voxel-driven exact transpose with split tables (default).  Same tiles,
// candidate boxes and staging as back_cone_gather_kernel, but the staging
// also evaluates, for every staged detector cell and each of the tile's
// kPlanes driving planes (x- or y-driven rays), the ray's Joseph split on
// that plane: lower indices (ib0, ic0) packed in one word and the upper
// weights (gb, gc).  Those are the same for every voxel of the plane, so a
// voxel's candidate test is two integer compares against its own indices and
// its weight two shared-memory loads -- the arithmetic of the split leaves
// the per-(voxel, cell) loop.  Cells of another driving axis, and samples
// whose taps cannot reach the volume, get a code no voxel matches.  Same
// weights and summation order as back_cone_gather_kernel, so the two give
// bitwise the same image; z-driven rays and boxes larger than the staging
// area take that kernel's global-memory path.
constexpr int kPlanes = 4;
static_assert(kGX == kPlanes && kGY == kPlanes, "one split table per driving plane of the tile");
constexpr unsigned kNoCell = 0xffffffffu;

template <int C>
__global__ void __launch_bounds__(kGX * kGY * kGZ, 4)
    back_cone_split_kernel(mbir_geometry g, const float4 *__restrict__ vt, const float4 *__restrict__ ta,
                           const float2 *__restrict__ tb, const int *__restrict__ view_axes,
                           const typename Vec<C>::T *__restrict__ ws, int nc, float *__restrict__ x,
                           int accumulate) {
    __shared__ unsigned s_ij[kPlanes][kStageCap];
    __shared__ float2 s_f[kPlanes][kStageCap];
    __shared__ typename Vec<C>::T s_ws[kStageCap];
    const int tid = threadIdx.x;
    const int x0 = blockIdx.x * kGX, y0 = blockIdx.y * kGY, z0 = blockIdx.z * kGZ;
    const int ix = x0 + tid % kGX, iy = y0 + (tid / kGX) % kGY, iz = z0 + tid / (kGX * kGY);
    const bool inside = ix < g.nx && iy < g.ny && iz < g.nz;
    const float dx = (float)g.dx, dy = (float)g.dy, dz = (float)g.dz;
    const float cx = 0.5f * (g.nx - 1), cy = 0.5f * (g.ny - 1), cz = 0.5f * (g.nz - 1);
    const float px = (ix - cx) * dx, py = (iy - cy) * dy, pz = (iz - cz) * dz;
    const float tx0 = (x0 - cx) * dx, tx1 = (min(x0 + kGX, g.nx) - 1 - cx) * dx;
    const float ty0 = (y0 - cy) * dy, ty1 = (min(y0 + kGY, g.ny) - 1 - cy) * dy;
    const float tz0 = (z0 - cz) * dz, tz1 = (min(z0 + kGZ, g.nz) - 1 - cz) * dz;
    const int *tbits = reinterpret_cast<const int *>(tb);  // (w, bits) pairs: bits at odd indices
    float acc[C], comp[C];
#pragma unroll
    for (int c = 0; c < C; ++c) acc[c] = comp[c] = 0.f;
    for (int v = 0; v < g.n_views; ++v) {
        const int axes = view_axes[v];
        if (!axes) continue;
        const float4 V = vt[v];  // (sx, sy, cos beta, sin beta)
        const bool mixed = (axes & (axes - 1)) != 0;
        const int64_t view0 = (int64_t)v * g.n_u * g.n_v;
        float sv[C];
#pragma unroll
        for (int c = 0; c < C; ++c) sv[c] = 0.f;
#pragma unroll
        for (int A = 0; A < 3; ++A) {
            if (!((axes >> A) & 1)) continue;
            float xs[2], ys[2], zs[2];
            int iu0, iu1, iv0, iv1;
            if (A == 0) {
                voxel_footprint<0>(g, px, py, pz, xs, ys, zs);
                footprint_box<2>(g, V, xs, ys, zs, iu0, iu1, iv0, iv1);
            } else if (A == 1) {
                voxel_footprint<1>(g, px, py, pz, xs, ys, zs);
                footprint_box<2>(g, V, xs, ys, zs, iu0, iu1, iv0, iv1);
            } else {
                voxel_footprint<2>(g, px, py, pz, xs, ys, zs);
                footprint_box<4>(g, V, xs, ys, zs, iu0, iu1, iv0, iv1);
            }
            int su0 = 0, su1 = -1, sv0 = 0, sv1 = -1;
            bool staged = false;
            if (A == 0)
                staged = tile_box_warp<0>(g, V, tx0, tx1, ty0, ty1, tz0, tz1, su0, su1, sv0, sv1);
            else if (A == 1)
                staged = tile_box_warp<1>(g, V, tx0, tx1, ty0, ty1, tz0, tz1, su0, su1, sv0, sv1);
            staged = staged && su1 >= su0 && sv1 >= sv0 && (su1 - su0 + 1) * (sv1 - sv0 + 1) <= kStageCap;
            const int sw = su1 - su0 + 1;
            if (staged) {
                __syncthreads();   // the previous staging's readers are done
                const int n = sw * (sv1 - sv0 + 1);
                const int pbase = A == 0 ? x0 : y0;
                const float ca = 0.5f * ((A == 0 ? g.nx : g.ny) - 1);
                const int nb = A == 0 ? g.ny : g.nx;   // interpolated axes b, c (c = z for A = 0, 1)
                for (int k = tid; k < n; k += blockDim.x) {
                    const int64_t ray = view0 + (int64_t)(sv0 + k / sw) * g.n_u + su0 + k % sw;
                    s_ws[k] = __ldg(ws + ray);
                    const bool same = (__ldg(tbits + 2 * ray + 1) & 3) == A;
                    const float4 R = __ldg(ta + ray);
#pragma unroll
                    for (int q = 0; q < kPlanes; ++q) {
                        const float t = (float)(pbase + q) - ca;
                        float gb, gc;
                        const int ib0 = joseph_split(fmaf(t, R.y, R.x), gb);
                        const int ic0 = joseph_split(fmaf(t, R.w, R.z), gc);
                        const bool ok = same && ib0 >= -1 && ib0 < nb && ic0 >= -1 && ic0 < g.nz;
                        s_ij[q][k] = ok ? (unsigned)(ib0 + 1) | ((unsigned)(ic0 + 1) << 16) : kNoCell;
                        s_f[q][k] = make_float2(gb, gc);
                    }
                }
                __syncthreads();
                iu0 = max(iu0, su0), iu1 = min(iu1, su1), iv0 = max(iv0, sv0), iv1 = min(iv1, sv1);
            }
            if (!inside) continue;
            if (staged) {
                const int q = A == 0 ? ix - x0 : iy - y0;
                const int ib = A == 0 ? iy : ix;
                const unsigned *tij = s_ij[q];
                const float2 *tf = s_f[q];
                for (int jv = iv0; jv <= iv1; ++jv) {
                    const int row = (jv - sv0) * sw - su0;
                    for (int ju = iu0; ju <= iu1; ++ju) {
                        const int k = row + ju;
                        const unsigned code = tij[k];
                        const int db = ib - ((int)(code & 0xffffu) - 1), dc = iz - ((int)(code >> 16) - 1);
                        if ((unsigned)db > 1u || (unsigned)dc > 1u) continue;
                        const float2 f = tf[k];
                        const float wbc = (db ? f.x : 1.f - f.x) * (dc ? f.y : 1.f - f.y);
                        float val[C];
                        Vec<C>::get(s_ws[k], val);
#pragma unroll
                        for (int c = 0; c < C; ++c) sv[c] = fmaf(wbc, val[c], sv[c]);
                    }
                }
            } else if (A == 0) {
                gather_cells<0, C>(g, v, ix, iy, iz, iu0, iu1, iv0, iv1, mixed, ta, tbits, ws, nullptr, s_ws, nullptr,
                                   su0, sv0, sw, sv);
            } else if (A == 1) {
                gather_cells<1, C>(g, v, ix, iy, iz, iu0, iu1, iv0, iv1, mixed, ta, tbits, ws, nullptr, s_ws, nullptr,
                                   su0, sv0, sw, sv);
            } else {
                gather_cells<2, C>(g, v, ix, iy, iz, iu0, iu1, iv0, iv1, mixed, ta, tbits, ws, nullptr, s_ws, nullptr,
                                   su0, sv0, sw, sv);
            }
        }
#pragma unroll
        for (int c = 0; c < C; ++c) {
            const float yk = __fsub_rn(sv[c], comp[c]);
            const float tt = __fadd_rn(acc[c], yk);
            comp[c] = __fsub_rn(__fsub_rn(tt, acc[c]), yk);
            acc[c] = tt;
        }
    }
    if (!inside) return;
    const int64_t npix = (int64_t)g.nx * g.ny * g.nz;
    const int64_t j = ((int64_t)iz * g.ny + iy) * g.nx + ix;
#pragma unroll
    for (int c = 0; c < C; ++c) {
        if (c >= nc) break;
        float *o = x + (int64_t)c * npix + j;
        *o = accumulate ? *o + acc[c] : acc[c];
    }
}

// Ray-driven tile transpose with fixed-point shared-memory sums (mode 0,
// the default).  A CTA owns a tile of 8 x 8 x TZ voxels (TZ = 16 or 8, chosen
// per plan) and runs over
// every view.  For each view and each driving axis a of its rays it stages,
// in chunks, the detector box that covers the tile's footprint (the gather's
// box), and every pair (staged ray, tile plane of axis a) takes the forward's
// sample split on that plane and adds the sample's bilinear terms, times the
// ray's weighted value of each channel, to the tile's accumulators of the
// taps that lie in the tile.  A voxel so receives exactly the terms of the
// forward's weights (A^T), without the gather's per-voxel candidate search;
// a sample whose taps straddle the tile's edge is taken by each tile it
// reaches, for its own taps.
//
// The accumulators are 32-bit fixed point, [C][TZ][kTY][kTX] with the x
// index XOR-swizzled by y, so that a warp's lanes (eight planes x four rays)
// fall in distinct banks for x- and y-driven rays.  Channel c uses the scale
//   sc = min(2^22, 2^30 / T) / M_c,  M_c = max_i |w_i s_c,i|,
// T = a bound on the terms one accumulator receives between two flushes: a
// ray adds at most one term to a voxel and at most cell_rays rays of a view
// reach one voxel (the plan's bound, from cone_setup), so with a flush every
// vb views T = vb * cell_rays (vb chosen so that T <= 256 where the bound
// allows: a grid of M_c 2^-22).  A ray's scaled value v = sc w s (rounded) is at
// most min(2^22, 2^30 / T), each term round(w_bc v) (one FMA with the magic
// number: exact rounding to nearest) at most that plus 1/2, and T of them
// stay below 2^31.  Channels c < nfine (the gradient numerators, which the
// cross-material preconditioners difference: there a grid of M_c 2^-22 shows
// in the step) also add each term's remainder w v - round(w v), rounded to
// 2^-11 units, to a second word: terms of at most 2^10 of those units, T of
// them below 2^31.  At every flush each thread moves its own voxels' words
// into 64-bit registers (exact integer sums in units of 2^-11 / sc) and
// clears them; the image is sum / sc.  Integer sums are exact, so the result
// is the same bit for bit whatever order the adds run in; its error is at
// most half a unit 1 / sc per term (2^-12 units for the fine channels),
// besides the FP32 roundings of the scaled value v and of the weight product
// (2^-24 of each term, as in the FP32 gather) and the final conversion's
// 2^-24 relative.  The 64-bit sums hold up to 2^20 flushes.
constexpr int kTX = 8, kTY = 8;               // tile width and height; depth TZ = 16 (default) or 8
template <int TZ>
struct Tile3 {
    static constexpr int Vox = kTX * kTY * TZ;     // voxels per CTA
    static constexpr int Plane = Vox;              // words per channel
    static constexpr int PerThread = Vox / 256;    // voxels per thread
};
constexpr int kTThreads = 256;                 // four voxels per thread
constexpr int kTCap = 512;                     // staged rays per chunk
constexpr int kTMaxVB = 32;                    // views per flush at most
constexpr float kFixMagic3 = 12582912.f;       // 1.5 * 2^23: x + magic rounds x (|x| <= 2^22) to an integer
constexpr int kFixMagic3Bits = 0x4B400000;

// Accumulator word of tile voxel (lx, ly, lz): x fastest, XOR-swizzled with
// y so that a warp's lanes -- eight consecutive planes of four rays -- fall
// in distinct banks for x- and y-driven rays.
__device__ __forceinline__ int tile3_word(int lx, int ly, int lz) {
    return (lz * kTY + ly) * kTX + (lx ^ (ly & (kTX - 1)));
}

// Fixed-point scale of one channel (see above) from M_c's float bits; 0 when
// M_c is not finite, 1 when the channel is all zero.  The quotient is rounded
// down so that M_c sc never exceeds the limit.
__device__ __forceinline__ float tile3_scale(unsigned mbits, int bound) {
    const float M = __uint_as_float(mbits);
    if (!(M <= 3.0e38f)) return 0.f;
    if (M == 0.f) return 1.f;
    const float lim = fminf(4194304.f, 1073741824.f / (float)(bound > 1 ? bound : 1));
    return fminf(__fdiv_rd(lim, M), 0x1p126f);
}

template <unsigned OFF>
__device__ __forceinline__ void red_word(unsigned addr, int v) {
    asm volatile("red.shared.add.s32 [%0+%2], %1;" ::"r"(addr), "r"(v), "n"(OFF) : "memory");
}

// The terms of one tap (byte address addr of channel 0's word) for every
// channel: round(w v_c) to the coarse words, and for the first NF channels
// the remainder w v_c - round(w v_c) on a grid 2^11 times finer to the low
// words (LO bytes further on).
template <int C, int NF, unsigned LO, int PL, int c = 0>
__device__ __forceinline__ void tile3_tap(unsigned addr, float w, const float (&v)[C]) {
    if constexpr (c < C) {
        const float h = fmaf(w, v[c], kFixMagic3);   // magic + round(w v), exact
        red_word<4u * c * PL>(addr, __float_as_int(h) - kFixMagic3Bits);
        if constexpr (c < NF) {
            const float r = fmaf(w, v[c], kFixMagic3 - h);   // w v - round(w v), |r| <= 1/2
            red_word<4u * c * PL + LO>(addr, __float_as_int(fmaf(r, 2048.f, kFixMagic3)) - kFixMagic3Bits);
        }
        tile3_tap<C, NF, LO, PL, c + 1>(addr, w, v);
    }
}

// The pairs (staged ray k < m, tile plane p) of driving axis A: the sample's
// split on plane a0 + p and its terms on the taps inside the tile (b in
// [b0, b0 + eb), c in [c0, c0 + ec); planes p < np).  NP consecutive
// threads take the NP planes (8, or the depth for z-driven rays) of one ray.
template <int A, int C, int NF, int TZ>
__device__ __forceinline__ void tile3_scatter(int m, const float4 *s_ta, const typename Vec<C>::T *s_ws,
                                              const int *s_ax, int a0, int np, float ca, int b0, int eb, int c0,
                                              int ec, unsigned acc) {
    constexpr int NP = A == 2 ? TZ : (A == 0 ? kTX : kTY);
    constexpr int PL = Tile3<TZ>::Plane;
    constexpr unsigned LO = 4u * C * PL;        // byte offset of the low words
    const int p = threadIdx.x % NP;
    if (p >= np) return;
    const float t = (float)(a0 + p) - ca;
    for (int k = threadIdx.x / NP; k < m; k += kTThreads / NP) {
        if (s_ax[k] != A) continue;
        const float4 R = s_ta[k];
        float gb, gc;
        const int lb = joseph_split(fmaf(t, R.y, R.x), gb) - b0;
        const int lc = joseph_split(fmaf(t, R.w, R.z), gc) - c0;
        if (lb < -1 || lb >= eb || lc < -1 || lc >= ec) continue;
        float v[C];
        Vec<C>::get(s_ws[k], v);
#pragma unroll
        for (int dc = 0; dc < 2; ++dc) {
            const int cc = lc + dc;
            if (cc < 0 || cc >= ec) continue;
            const float wc = dc ? gc : 1.f - gc;
#pragma unroll
            for (int db = 0; db < 2; ++db) {
                const int bb = lb + db;
                if (bb < 0 || bb >= eb) continue;
                const float wbc = (db ? gb : 1.f - gb) * wc;
                const int w = A == 0 ? tile3_word(p, bb, cc) : (A == 1 ? tile3_word(bb, p, cc) : tile3_word(bb, cc, p));
                tile3_tap<C, NF, LO, PL>(acc + 4u * (unsigned)w, wbc, v);
            }
        }
    }
}

template <int C, int NF, int TZ>
__global__ void __launch_bounds__(kTThreads, TZ == 16 ? 4 : 5)
    back_cone_tile_kernel(mbir_geometry g, const float4 *__restrict__ vt, const float4 *__restrict__ ta,
                          const float2 *__restrict__ tb, const int *__restrict__ view_axes,
                          const typename Vec<C>::T *__restrict__ ws, const unsigned *__restrict__ smax, int vb,
                          int T, int nc, float *__restrict__ x, int accumulate) {
    constexpr int kTPlane = Tile3<TZ>::Plane, kTZ = TZ, kPer = Tile3<TZ>::PerThread;
    __shared__ int acc[(C + NF) * kTPlane];   // C coarse planes, then the fine channels' low words
    __shared__ float4 s_ta[kTCap];
    __shared__ typename Vec<C>::T s_ws[kTCap];
    __shared__ int s_ax[kTCap];
    __shared__ int4 s_box[kTMaxVB * 3];
    const int tid = threadIdx.x;
    const int x0 = blockIdx.x * kTX, y0 = blockIdx.y * kTY, z0 = blockIdx.z * kTZ;
    const int ex = min(kTX, g.nx - x0), ey = min(kTY, g.ny - y0), ez = min(kTZ, g.nz - z0);
    const float dx = (float)g.dx, dy = (float)g.dy, dz = (float)g.dz;
    const float cx = 0.5f * (g.nx - 1), cy = 0.5f * (g.ny - 1), cz = 0.5f * (g.nz - 1);
    const float tx0 = (x0 - cx) * dx, tx1 = (x0 + ex - 1 - cx) * dx;
    const float ty0 = (y0 - cy) * dy, ty1 = (y0 + ey - 1 - cy) * dy;
    const float tz0 = (z0 - cz) * dz, tz1 = (z0 + ez - 1 - cz) * dz;
    const int *tbits = reinterpret_cast<const int *>(tb);
    float sc[C];
#pragma unroll
    for (int c = 0; c < C; ++c) sc[c] = tile3_scale(__ldg(smax + c), T);
    for (int k = tid; k < (C + NF) * kTPlane; k += kTThreads) acc[k] = 0;
    long long sum[kPer][C];
#pragma unroll
    for (int r = 0; r < kPer; ++r)
#pragma unroll
        for (int c = 0; c < C; ++c) sum[r][c] = 0;
    const unsigned acc_addr = (unsigned)__cvta_generic_to_shared(acc);
    for (int vb0 = 0; vb0 < g.n_views; vb0 += vb) {
        const int nvb = min(vb, g.n_views - vb0);
        // the detector boxes of the block's (view, axis) pairs, one lane each
        if (tid < 32) {
            for (int q = tid; q < 3 * nvb; q += 32) {
                const int v = vb0 + q / 3, A = q % 3;
                int4 b = make_int4(0, -1, 0, -1);
                if ((__ldg(view_axes + v) >> A) & 1) {
                    const float txs[2] = {A == 0 ? tx0 : tx0 - dx, A == 0 ? tx1 : tx1 + dx};
                    const float tys[2] = {A == 1 ? ty0 : ty0 - dy, A == 1 ? ty1 : ty1 + dy};
                    const float tzs[2] = {A == 2 ? tz0 : tz0 - dz, A == 2 ? tz1 : tz1 + dz};
                    footprint_box<4>(g, __ldg(vt + v), txs, tys, tzs, b.x, b.y, b.z, b.w);
                }
                s_box[q] = b;
            }
        }
        __syncthreads();   // boxes published; every flush of the previous block done
        for (int q = 0; q < 3 * nvb; ++q) {
            const int4 b = s_box[q];
            if (b.y < b.x || b.w < b.z) continue;
            const int v = vb0 + q / 3, A = q % 3;
            const int sw = b.y - b.x + 1, n = sw * (b.w - b.z + 1);
            const int64_t view0 = (int64_t)v * g.n_u * g.n_v;
            for (int k0 = 0; k0 < n; k0 += kTCap) {
                const int m = min(kTCap, n - k0);
                for (int k = tid; k < m; k += kTThreads) {
                    const int kk = k0 + k, row = kk / sw;
                    const int64_t ray = view0 + (int64_t)(b.z + row) * g.n_u + b.x + (kk - row * sw);
                    s_ta[k] = __ldg(ta + ray);
                    float val[C];
                    Vec<C>::get(__ldg(ws + ray), val);
#pragma unroll
                    for (int c = 0; c < C; ++c) val[c] *= sc[c];
                    Vec<C>::put(s_ws[k], val);
                    s_ax[k] = __ldg(tbits + 2 * ray + 1) & 3;   // every ray: a view's empty rays may use another axis
                }
                __syncthreads();
                if (A == 0)
                    tile3_scatter<0, C, NF, TZ>(m, s_ta, s_ws, s_ax, x0, ex, cx, y0, ey, z0, ez, acc_addr);
                else if (A == 1)
                    tile3_scatter<1, C, NF, TZ>(m, s_ta, s_ws, s_ax, y0, ey, cy, x0, ex, z0, ez, acc_addr);
                else
                    tile3_scatter<2, C, NF, TZ>(m, s_ta, s_ws, s_ax, z0, ez, cz, x0, ex, y0, ey, acc_addr);
                __syncthreads();
            }
        }
        // flush this thread's voxels (no other thread reads or writes their
        // words until the next block's first barrier)
#pragma unroll
        for (int r = 0; r < kPer; ++r) {
            const int j = tid + r * kTThreads;
            const int w = tile3_word(j % kTX, (j / kTX) % kTY, j / (kTX * kTY));
#pragma unroll
            for (int c = 0; c < C; ++c) {
                // sums in units of 2^-11 / sc
                long long u = (long long)acc[c * kTPlane + w] * 2048;
                acc[c * kTPlane + w] = 0;
                if (c < NF) {
                    u += acc[(C + c) * kTPlane + w];
                    acc[(C + c) * kTPlane + w] = 0;
                }
                sum[r][c] += u;
            }
        }
    }
    const int64_t npix = (int64_t)g.nx * g.ny * g.nz;
#pragma unroll
    for (int r = 0; r < kPer; ++r) {
        const int j = tid + r * kTThreads;
        const int lx = j % kTX, ly = (j / kTX) % kTY, lz = j / (kTX * kTY);
        if (lx >= ex || ly >= ey || lz >= ez) continue;
        const int64_t o = ((int64_t)(z0 + lz) * g.ny + y0 + ly) * g.nx + x0 + lx;
#pragma unroll
        for (int c = 0; c < C; ++c) {
            if (c >= nc) break;
            const float v = sc[c] > 0.f ? __fdiv_rn(__ll2float_rn(sum[r][c]), sc[c]) * 0x1p-11f : __int_as_float(0x7fc00000);
            float *dst = x + (int64_t)c * npix + o;
            *dst = accumulate ? *dst + v : v;
        }
    }
}

}  // namespace

int64_t cone_pack_floats(const mbir_geometry &g) { return pack3d_floats(g.nx, g.ny, g.nz); }

mbir_status cone_setup(mbir_plan *p) {
    PSPS_TRY(p->view.alloc(p->g.n_views));
    PSPS_TRY(p->ray.alloc(p->n_rays));
    PSPS_TRY(p->ray3b.alloc(p->n_rays));
    PSPS_TRY(p->view_axes.alloc(p->g.n_views));
    PSPS_TRY(p->view_axes.zero(0));
    PSPS_TRY(p->wsino.alloc((size_t)4 * p->n_rays));
    PSPS_TRY(p->wmax.alloc(4));
    {
        // Rays of one view that reach one voxel j (any driving axis), for the
        // fixed-point scale of the tile transpose.  A ray reaches j through its
        // sample on j's plane, which then lies within one voxel of j's centre
        // in the two interpolated axes, so inside the cube of half-side s
        // (the largest voxel side) around j, whatever the ray's axis.  Its
        // points are within R of the rotation axis and |z| <= Z, so at depth
        // D >= D_min = sid - R from the source along the central ray.  On the
        // flat detector u = sdd L / D and w = sdd z / D (L the lateral
        // offset, |L| <= R); across the cube L, D and z change by at most
        // 2 sqrt2 s, so its image spans at most
        //   E_u = sdd (1 + R / D_min) 2 sqrt2 s / D_min in u,
        //   E_v = sdd (1 + Z / D_min) 2 sqrt2 s / D_min in v,
        // and holds at most floor(E / pitch) + 1 cell centres along each (one
        // more for the FP32 set-up's rounding).
        const mbir_geometry &g = p->g;
        const double s = std::max(g.dx, std::max(g.dy, g.dz));
        const double R = std::hypot((0.5 * g.nx + 1.0) * g.dx, (0.5 * g.ny + 1.0) * g.dy);
        const double Z = (0.5 * g.nz + 1.0) * g.dz, D = g.sid - R;
        p->cell_rays = 0;
        if (D > 1e-6 * g.sid) {
            const double side = 2.0 * std::sqrt(2.0) * s;
            const double Eu = g.sdd * (1.0 + R / D) * side / D, Ev = g.sdd * (1.0 + Z / D) * side / D;
            const double cells = (std::floor(Eu / g.du) + 2.0) * (std::floor(Ev / g.dv) + 2.0);
            if (cells < 16384.0) p->cell_rays = (int)cells;
        }
    }
    setup_view3d_kernel<<<(unsigned)cdiv(p->g.n_views, 128), 128>>>(p->g, p->view.p);
    PSPS_LAUNCH_CHECK();
    setup_rays3d_kernel<<<(unsigned)cdiv(p->n_rays, kThreads), kThreads>>>(p->g, p->view.p, p->n_rays, p->ray.p,
                                                                          p->ray3b.p, p->view_axes.p);
    PSPS_LAUNCH_CHECK();
    return MBIR_OK;
}

mbir_status project_cone(mbir_plan *p, const float *x, float *l, int n_mat, cudaStream_t s) {
    const mbir_geometry &g = p->g;
    const int64_t n = p->n_pix;
    for (int m0 = 0; m0 < n_mat; m0 += 4) {
        const int nm = n_mat - m0 < 4 ? n_mat - m0 : 4;
        const int P = nm == 1 ? 1 : (nm == 2 ? 2 : 4);
        float *ox = p->xcol.p, *oy = p->xrow.p, *oz = p->xcol3.p;
        const int64_t grid = cdiv(n, kThreads) < 65535 * 8 ? cdiv(n, kThreads) : 65535 * 8;
        pack3d_border_kernel<<<1024, kThreads, 0, s>>>(P, g.nx, g.ny, g.nz, ox, oy, oz);
        PSPS_LAUNCH_CHECK();
        pack3d_kernel<<<(unsigned)grid, kThreads, 0, s>>>(x + m0 * n, nm, P, g.nx, g.ny, g.nz, ox, oy, oz);
        PSPS_LAUNCH_CHECK();
        const unsigned gr = (unsigned)cdiv(p->n_rays, kThreads);
        float *lm = l + (int64_t)m0 * p->n_rays;
        // fwd_mode 2: warp-aligned march; otherwise each lane from its own range
        if (p->fwd_mode == 2) {
            if (P == 1)
                fwd_cone_kernel<1, true><<<gr, kThreads, 0, s>>>(g, p->ray.p, p->ray3b.p, ox, oy, oz, nm, p->n_rays, lm);
            else if (P == 2)
                fwd_cone_kernel<2, true><<<gr, kThreads, 0, s>>>(g, p->ray.p, p->ray3b.p, (const float2 *)ox,
                                                                 (const float2 *)oy, (const float2 *)oz, nm,
                                                                 p->n_rays, lm);
            else
                fwd_cone_kernel<4, true><<<gr, kThreads, 0, s>>>(g, p->ray.p, p->ray3b.p, (const float4 *)ox,
                                                                 (const float4 *)oy, (const float4 *)oz, nm,
                                                                 p->n_rays, lm);
        } else {
            if (P == 1)
                fwd_cone_kernel<1, false><<<gr, kThreads, 0, s>>>(g, p->ray.p, p->ray3b.p, ox, oy, oz, nm, p->n_rays,
                                                                  lm);
            else if (P == 2)
                fwd_cone_kernel<2, false><<<gr, kThreads, 0, s>>>(g, p->ray.p, p->ray3b.p, (const float2 *)ox,
                                                                  (const float2 *)oy, (const float2 *)oz, nm,
                                                                  p->n_rays, lm);
            else
                fwd_cone_kernel<4, false><<<gr, kThreads, 0, s>>>(g, p->ray.p, p->ray3b.p, (const float4 *)ox,
                                                                  (const float4 *)oy, (const float4 *)oz, nm,
                                                                  p->n_rays, lm);
        }
        PSPS_LAUNCH_CHECK();
    }
    return MBIR_OK;
}

mbir_status backproject_cone(mbir_plan *p, const float *sino, float *x, int n_mat, int accumulate, cudaStream_t s) {
    if (p->back_mode == 2) {
        if (!accumulate) PSPS_CUDA(cudaMemsetAsync(x, 0, sizeof(float) * (size_t)n_mat * p->n_pix, s));
        back_cone_kernel<<<(unsigned)cdiv(p->n_rays, kThreads), kThreads, 0, s>>>(p->g, p->ray.p, p->ray3b.p, sino,
                                                                                 n_mat, p->n_rays, x);
        PSPS_LAUNCH_CHECK();
        return MBIR_OK;
    }
    // mode 0 (default): fixed-point tile scatter (the direct gather where the
    // plan has no bound on the rays reaching a voxel); 1: direct gather; 3:
    // split-table gather (1 and 3 bitwise equal)
    const int mode = p->back_mode == 0 && (p->cell_rays <= 0 || p->g.n_views > (1 << 20)) ? 1 : p->back_mode;
    const dim3 grd((unsigned)cdiv(p->g.nx, kGX), (unsigned)cdiv(p->g.ny, kGY), (unsigned)cdiv(p->g.nz, kGZ));
    const int tz = p->cone_tile == 8 ? 8 : 16;   // tile depth of the tile transpose
    const dim3 grt((unsigned)cdiv(p->g.nx, kTX), (unsigned)cdiv(p->g.ny, kTY), (unsigned)cdiv(p->g.nz, tz));
    const int nthr = kGX * kGY * kGZ;
    // the weighting pass: a grid-stride loop over 2048 CTAs at most, so that
    // its per-warp maxima meet in few same-address atomics
    const unsigned gw = (unsigned)(cdiv(p->n_rays, kThreads) < 2048 ? cdiv(p->n_rays, kThreads) : 2048);
    // tile transpose: a flush every vb views, T = vb * cell_rays terms per
    // accumulator between flushes (T <= 256, so a grid of M 2^-22, where the
    // bound allows)
    const int vb = mode == 0 ? std::max(1, std::min(kTMaxVB, 256 / p->cell_rays)) : 1;
    const int T = mode == 0 ? vb * p->cell_rays : 0;
    for (int m0 = 0; m0 < n_mat;) {
        const int left = n_mat - m0;
        const float *sm = sino + (int64_t)m0 * p->n_rays;
        float *xm = x + (int64_t)m0 * p->n_pix;
        const int nc = left >= 4 ? 4 : left;                 // channels of this launch
        const int C = nc == 1 ? 1 : (nc == 2 ? 2 : 4);      // interleaved floats per ray
        float *w = p->wsino.p;
        unsigned *smax = mode == 0 ? p->wmax.p : nullptr;
        const int nfine = std::max(0, std::min(nc, p->tile_fine - m0));   // leading channels with low words
        if (smax) PSPS_CUDA(cudaMemsetAsync(smax, 0, 4 * sizeof(unsigned), s));
        auto run = [&](auto cst) -> mbir_status {
            constexpr int CC = decltype(cst)::value;
            using V = typename Vec<CC>::T;
            weigh_sino_kernel<CC><<<gw, kThreads, 0, s>>>(p->ray3b.p, sm, nc, p->n_rays, reinterpret_cast<V *>(w), smax);
            PSPS_LAUNCH_CHECK();
            const V *wv = reinterpret_cast<const V *>(w);
            if (mode == 0) {
                // the fine channels' count rounded up to an instantiated one
                // (more fine channels only add precision)
                auto tile = [&](auto nf) {
                    constexpr int NF = decltype(nf)::value;
                    if (tz == 8)
                        back_cone_tile_kernel<CC, NF, 8><<<grt, kTThreads, 0, s>>>(
                            p->g, p->view.p, p->ray.p, p->ray3b.p, p->view_axes.p, wv, smax, vb, T, nc, xm, accumulate);
                    else
                        back_cone_tile_kernel<CC, NF, 16><<<grt, kTThreads, 0, s>>>(
                            p->g, p->view.p, p->ray.p, p->ray3b.p, p->view_axes.p, wv, smax, vb, T, nc, xm, accumulate);
                };
                if (nfine == 0)
                    tile(std::integral_constant<int, 0>{});
                else if (nfine <= CC / 2)
                    tile(std::integral_constant<int, CC / 2 ? CC / 2 : 1>{});
                else
                    tile(std::integral_constant<int, CC>{});
            } else if (mode == 3)
                back_cone_split_kernel<CC><<<grd, nthr, 0, s>>>(p->g, p->view.p, p->ray.p, p->ray3b.p,
                                                                p->view_axes.p, wv, nc, xm, accumulate);
            else
                back_cone_gather_kernel<CC><<<grd, nthr, 0, s>>>(p->g, p->view.p, p->ray.p, p->ray3b.p,
                                                                 p->view_axes.p, wv, nc, xm, accumulate);
            PSPS_LAUNCH_CHECK();
            return MBIR_OK;
        };
        if (C == 4)
            PSPS_TRY(run(std::integral_constant<int, 4>{}));
        else if (C == 2)
            PSPS_TRY(run(std::integral_constant<int, 2>{}));
        else
            PSPS_TRY(run(std::integral_constant<int, 1>{}));
        m0 += nc;
    }
    return MBIR_OK;
}

}  // namespace psps
