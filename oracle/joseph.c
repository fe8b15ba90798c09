/*
 * FP64 reference Joseph projector and its exact transpose.
 *
 * TEST INFRASTRUCTURE ONLY.  This file belongs to the oracle: a plain, slow,
 * obviously correct CPU statement of the ray-driven projector A that the
 * forward model y_bar = B exp(-A x) (Eq. 1; A -> A for standard CT, Eq. 20, QA for
 * one-step MBMD, Eq. 44) is built on.  Only tests, the smoke check and the CPU-baseline
 * leg of the benchmark may load it.  It shares no code with the CUDA library.
 *
 * Definition (the paper fixes no projector; this is the textbook Joseph
 * method).  A ray is a full line p0 + t*u with unit direction u.  The axis with
 * the largest |u| component drives the march (ties: x before y before z).  For
 * an x-driven ray every image column ix contributes once: the line is
 * evaluated at the column-centre plane x = xc(ix), the image is interpolated
 * linearly (2-D) or bilinearly (3-D) between the neighbouring pixel centres in
 * the other axes, pixels outside the grid count as zero, and the sum is scaled
 * by dx/|u_x|, the path length per column.  The transpose scatters the same
 * weights.
 *
 * Pixel (ix,iy,iz) has its centre at ((ix-(nx-1)/2)dx, (iy-(ny-1)/2)dy,
 * (iz-(nz-1)/2)dz); images are [iz][iy][ix], 2-D sinograms [view][bin] and 3-D
 * sinograms [view][row][col].  Ray geometry per kind:
 *   0 parallel 2-D: th_v = angle0 + v*span/n_views; u = -(cos th, sin th);
 *     p0 = t_b * (-sin th, cos th), t_b = (b-(n_u-1)/2) du.
 *   1 fan 2-D, curved detector: source s = sid (cos be, sin be); fan angle
 *     ga_b = (b-(n_u-1)/2) du/sdd; u = -(cos(be-ga_b), sin(be-ga_b)); p0 = s.
 *   2 cone 3-D, flat detector: s = (sid cos be, sid sin be, 0); detector
 *     point d = s - sdd e_r + u_b e_u + v_r e_z with e_r=(cos be, sin be, 0),
 *     e_u = (-sin be, cos be, 0); u = (d-s)/|d-s|; p0 = s.
 */
#include <math.h>
#include <stdint.h>
#include <string.h>

typedef struct {
    int kind;
    int nx, ny, nz;
    double dx, dy, dz;
    int n_views;
    double angle0, angle_span;
    int n_u, n_v;
    double du, dv;
    double sid, sdd;
} og_geom;

static void ray_of(const og_geom *g, int64_t ray, double p0[3], double u[3]) {
    int64_t per_view = (int64_t)g->n_u * (g->kind == 2 ? g->n_v : 1);
    int view = (int)(ray / per_view);
    int64_t rem = ray % per_view;
    int iv = (int)(rem / g->n_u);
    int iu = (int)(rem % g->n_u);
    double ang = g->angle0 + view * (g->angle_span / g->n_views);
    double c = cos(ang), s = sin(ang);
    p0[2] = 0.0;
    u[2] = 0.0;
    if (g->kind == 0) {
        double t = (iu - 0.5 * (g->n_u - 1)) * g->du;
        p0[0] = -s * t;
        p0[1] = c * t;
        u[0] = -c;
        u[1] = -s;
    } else if (g->kind == 1) {
        double ga = (iu - 0.5 * (g->n_u - 1)) * g->du / g->sdd;
        p0[0] = g->sid * c;
        p0[1] = g->sid * s;
        u[0] = -cos(ang - ga);
        u[1] = -sin(ang - ga);
    } else {
        double uu = (iu - 0.5 * (g->n_u - 1)) * g->du;
        double vv = (iv - 0.5 * (g->n_v - 1)) * g->dv;
        double d[3];
        p0[0] = g->sid * c;
        p0[1] = g->sid * s;
        d[0] = -g->sdd * c - uu * s;
        d[1] = -g->sdd * s + uu * c;
        d[2] = vv;
        double n = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
        u[0] = d[0] / n;
        u[1] = d[1] / n;
        u[2] = d[2] / n;
    }
}

/* Visit every (pixel index, weight) pair of one ray.  mode 0: return the
 * weighted sum of img; mode 1: img[pixel] += weight * val. */
static double march(const og_geom *g, const double p0[3], const double u[3],
                    double *img, int mode, double val) {
    const int nx = g->nx, ny = g->ny, nz = (g->kind == 2) ? g->nz : 1;
    const double cx = 0.5 * (nx - 1), cy = 0.5 * (ny - 1), cz = 0.5 * (nz - 1);
    double ax = fabs(u[0]), ay = fabs(u[1]), az = fabs(u[2]);
    double sum = 0.0;
    if (g->kind != 2) {
        if (ax >= ay) {
            double w = g->dx / ax;
            for (int ix = 0; ix < nx; ++ix) {
                double xc = (ix - cx) * g->dx;
                double t = (xc - p0[0]) / u[0];
                double fy = (p0[1] + t * u[1]) / g->dy + cy;
                double fl = floor(fy);
                int iy0 = (int)fl;
                double f = fy - fl;
                if (iy0 >= 0 && iy0 < ny) {
                    if (mode == 0) sum += (1.0 - f) * img[(int64_t)iy0 * nx + ix];
                    else img[(int64_t)iy0 * nx + ix] += w * (1.0 - f) * val;
                }
                if (iy0 + 1 >= 0 && iy0 + 1 < ny) {
                    if (mode == 0) sum += f * img[(int64_t)(iy0 + 1) * nx + ix];
                    else img[(int64_t)(iy0 + 1) * nx + ix] += w * f * val;
                }
            }
            return sum * w;
        } else {
            double w = g->dy / ay;
            for (int iy = 0; iy < ny; ++iy) {
                double yc = (iy - cy) * g->dy;
                double t = (yc - p0[1]) / u[1];
                double fx = (p0[0] + t * u[0]) / g->dx + cx;
                double fl = floor(fx);
                int ix0 = (int)fl;
                double f = fx - fl;
                if (ix0 >= 0 && ix0 < nx) {
                    if (mode == 0) sum += (1.0 - f) * img[(int64_t)iy * nx + ix0];
                    else img[(int64_t)iy * nx + ix0] += w * (1.0 - f) * val;
                }
                if (ix0 + 1 >= 0 && ix0 + 1 < nx) {
                    if (mode == 0) sum += f * img[(int64_t)iy * nx + ix0 + 1];
                    else img[(int64_t)iy * nx + ix0 + 1] += w * f * val;
                }
            }
            return sum * w;
        }
    }
    /* 3-D: driving axis a, the other two (b, c) are interpolated bilinearly. */
    int axis;
    if (ax >= ay && ax >= az) axis = 0;
    else if (ay >= az) axis = 1;
    else axis = 2;
    const int n[3] = {nx, ny, nz};
    const double d[3] = {g->dx, g->dy, g->dz};
    const double c[3] = {cx, cy, cz};
    const int64_t stride[3] = {1, nx, (int64_t)nx * ny};
    int b = (axis == 0) ? 1 : 0;
    int cc = (axis == 2) ? 1 : 2;
    double w = d[axis] / fabs(u[axis]);
    for (int ia = 0; ia < n[axis]; ++ia) {
        double pa = (ia - c[axis]) * d[axis];
        double t = (pa - p0[axis]) / u[axis];
        double fb = (p0[b] + t * u[b]) / d[b] + c[b];
        double fc = (p0[cc] + t * u[cc]) / d[cc] + c[cc];
        double flb = floor(fb), flc = floor(fc);
        int ib0 = (int)flb, ic0 = (int)flc;
        double gb = fb - flb, gc = fc - flc;
        for (int jb = 0; jb < 2; ++jb) {
            int ib = ib0 + jb;
            if (ib < 0 || ib >= n[b]) continue;
            double wb = jb ? gb : 1.0 - gb;
            for (int jc = 0; jc < 2; ++jc) {
                int ic = ic0 + jc;
                if (ic < 0 || ic >= n[cc]) continue;
                double wc = jc ? gc : 1.0 - gc;
                int64_t idx = ia * stride[axis] + ib * stride[b] + ic * stride[cc];
                if (mode == 0) sum += wb * wc * img[idx];
                else img[idx] += w * wb * wc * val;
            }
        }
    }
    return sum * w;
}

static int64_t n_rays_of(const og_geom *g) {
    return (int64_t)g->n_views * g->n_u * (g->kind == 2 ? g->n_v : 1);
}

/* l = A x for every ray. */
void og_project(const og_geom *g, const double *x, double *l) {
    int64_t nr = n_rays_of(g);
    double p0[3], u[3];
    for (int64_t r = 0; r < nr; ++r) {
        ray_of(g, r, p0, u);
        l[r] = march(g, p0, u, (double *)x, 0, 0.0);
    }
}

/* l[k] = [A x]_{rays[k]} for a list of rays (sampled checks at full size). */
void og_project_rays(const og_geom *g, const double *x, const int64_t *rays, int64_t n, double *l) {
    double p0[3], u[3];
    for (int64_t k = 0; k < n; ++k) {
        ray_of(g, rays[k], p0, u);
        l[k] = march(g, p0, u, (double *)x, 0, 0.0);
    }
}

/* x = A^T s (overwrites x). */
void og_backproject(const og_geom *g, const double *s, double *x) {
    int64_t nr = n_rays_of(g);
    int64_t np = (int64_t)g->nx * g->ny * (g->kind == 2 ? g->nz : 1);
    memset(x, 0, sizeof(double) * (size_t)np);
    double p0[3], u[3];
    for (int64_t r = 0; r < nr; ++r) {
        if (s[r] == 0.0) continue;
        ray_of(g, r, p0, u);
        march(g, p0, u, x, 1, s[r]);
    }
}

/* Ray origin and direction, exposed so tests can compute closed-form chords
 * for exactly the rays the projector uses. */
void og_ray(const og_geom *g, int64_t ray, double *p0, double *u) { ray_of(g, ray, p0, u); }
