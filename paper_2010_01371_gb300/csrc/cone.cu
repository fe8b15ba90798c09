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
// Forward: one thread per ray (neighbouring threads = neighbouring detector
// columns of one row), reading a packed copy of the volume laid out so the
// two interpolated axes are the fastest (b fastest), for each driving axis;
// Kahan-compensated FP32 sums.  Transpose: the same walk scattering with
// FP32 atomics (exact transpose of the weights).
#include <cmath>

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

// Packed copies of x[m][z][y][x] for the three driving axes, materials
// innermost with stride P: layout[a][c][b][m] (see the file comment).
__global__ void pack3d_kernel(const float *__restrict__ x, int nm, int P, int nx, int ny, int nz,
                              float *__restrict__ ox, float *__restrict__ oy, float *__restrict__ oz) {
    const int64_t n = (int64_t)nx * ny * nz;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
        const int ix = (int)(j % nx);
        const int iy = (int)((j / nx) % ny);
        const int iz = (int)(j / ((int64_t)nx * ny));
        const int64_t px = (((int64_t)ix * nz + iz) * ny + iy) * P;   // a = x: [ix][iz][iy]
        const int64_t py = (((int64_t)iy * nz + iz) * nx + ix) * P;   // a = y: [iy][iz][ix]
        const int64_t pz = (((int64_t)iz * ny + iy) * nx + ix) * P;   // a = z: [iz][iy][ix]
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

template <int NM>
__global__ void __launch_bounds__(kThreads)
    fwd_cone_kernel(mbir_geometry g, const float4 *__restrict__ vt, const typename P3<NM>::T *__restrict__ ox,
                    const typename P3<NM>::T *__restrict__ oy, const typename P3<NM>::T *__restrict__ oz, int nm,
                    int64_t n_rays, float *__restrict__ l) {
    const int64_t ray = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (ray >= n_rays) return;
    const int per_view = g.n_u * g.n_v;
    const int v = (int)(ray / per_view);
    const int rem = (int)(ray % per_view);
    const ConeRay r = cone_ray(g, vt[v], rem % g.n_u, rem / g.n_u);
    const typename P3<NM>::T *src = r.axis == 0 ? ox : (r.axis == 1 ? oy : oz);
    const int nb = r.axis == 0 ? g.ny : g.nx;
    const int nc = r.axis == 2 ? g.ny : g.nz;
    float acc[NM], comp[NM];
#pragma unroll
    for (int m = 0; m < NM; ++m) acc[m] = comp[m] = 0.f;
    for (int i = r.lo; i <= r.hi; ++i) {
        const float t = (float)i - r.ca;
        const float fb = fmaf(t, r.dfb, r.fb_mid), fc = fmaf(t, r.dfc, r.fc_mid);
        const float flb = floorf(fb), flc = floorf(fc);
        const int ib0 = (int)flb, ic0 = (int)flc;
        const float gb = fb - flb, gc = fc - flc;
        float s[NM];
#pragma unroll
        for (int m = 0; m < NM; ++m) s[m] = 0.f;
#pragma unroll
        for (int jc = 0; jc < 2; ++jc) {
            const int ic = ic0 + jc;
            if (ic < 0 || ic >= nc) continue;
            const float wc = jc ? gc : 1.f - gc;
#pragma unroll
            for (int jb = 0; jb < 2; ++jb) {
                const int ib = ib0 + jb;
                if (ib < 0 || ib >= nb) continue;
                const float wbc = (jb ? gb : 1.f - gb) * wc;
                float val[NM];
                P3<NM>::get(__ldg(src + ((int64_t)i * nc + ic) * nb + ib), val);
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
#pragma unroll
    for (int m = 0; m < NM; ++m)
        if (m < nm) l[(int64_t)m * n_rays + ray] = acc[m] * r.w;
}

__global__ void __launch_bounds__(kThreads)
    back_cone_kernel(mbir_geometry g, const float4 *__restrict__ vt, const float *__restrict__ sino, int nm,
                     int64_t n_rays, float *__restrict__ x) {
    const int64_t ray = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (ray >= n_rays) return;
    const int per_view = g.n_u * g.n_v;
    const int v = (int)(ray / per_view);
    const int rem = (int)(ray % per_view);
    const ConeRay r = cone_ray(g, vt[v], rem % g.n_u, rem / g.n_u);
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
            const float fb = fmaf(t, r.dfb, r.fb_mid), fc = fmaf(t, r.dfc, r.fc_mid);
            const float flb = floorf(fb), flc = floorf(fc);
            const int ib0 = (int)flb, ic0 = (int)flc;
            const float gb = fb - flb, gc = fc - flc;
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

}  // namespace

mbir_status cone_setup(mbir_plan *p) {
    PSPS_TRY(p->view.alloc(p->g.n_views));
    setup_view3d_kernel<<<(unsigned)cdiv(p->g.n_views, 128), 128>>>(p->g, p->view.p);
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
        pack3d_kernel<<<(unsigned)grid, kThreads, 0, s>>>(x + m0 * n, nm, P, g.nx, g.ny, g.nz, ox, oy, oz);
        PSPS_LAUNCH_CHECK();
        const unsigned gr = (unsigned)cdiv(p->n_rays, kThreads);
        float *lm = l + (int64_t)m0 * p->n_rays;
        if (P == 1)
            fwd_cone_kernel<1><<<gr, kThreads, 0, s>>>(g, p->view.p, ox, oy, oz, nm, p->n_rays, lm);
        else if (P == 2)
            fwd_cone_kernel<2><<<gr, kThreads, 0, s>>>(g, p->view.p, (const float2 *)ox, (const float2 *)oy,
                                                       (const float2 *)oz, nm, p->n_rays, lm);
        else
            fwd_cone_kernel<4><<<gr, kThreads, 0, s>>>(g, p->view.p, (const float4 *)ox, (const float4 *)oy,
                                                       (const float4 *)oz, nm, p->n_rays, lm);
        PSPS_LAUNCH_CHECK();
    }
    return MBIR_OK;
}

mbir_status backproject_cone(mbir_plan *p, const float *sino, float *x, int n_mat, int accumulate, cudaStream_t s) {
    if (!accumulate) PSPS_CUDA(cudaMemsetAsync(x, 0, sizeof(float) * (size_t)n_mat * p->n_pix, s));
    back_cone_kernel<<<(unsigned)cdiv(p->n_rays, kThreads), kThreads, 0, s>>>(p->g, p->view.p, sino, n_mat, p->n_rays,
                                                                             x);
    PSPS_LAUNCH_CHECK();
    return MBIR_OK;
}

}  // namespace psps
