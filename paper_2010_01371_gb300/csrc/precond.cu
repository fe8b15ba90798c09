// Preconditioners x = M x' (Sec. II-C to II-F): one-time build on the GPU and
// the per-iteration applies M, M^T, |M|, |M|^T.
//
// Build (Sec. II-C): the Hessian at the solution H = A^T F A + R is formed
// with the per-ray Fisher blocks F_i of the data approximated from the
// measurements (standard CT: D = y / I0; spectral: water-only fit), applied
// matrix-free (project, per-ray block multiply, backproject, penalty).
//  * M0 = blocks of (F+R)1_k raised to -1/2 (Eqs. 30, 42, 53-54): column k of
//    every per-pixel (per-ray) block is the response to the all-ones image of
//    material k; FP64 symmetric inverse square roots on the GPU with each
//    block's eigenvalues clamped to >= 1e-6 of its largest and blocks whose
//    trace is <= 1e-12 of the largest set to zero (outside the field of view).
//  * Fourier (Eqs. 28-29, 32-33): Lambda~ = |DFT(N delta_c) / DFT(delta_c)| for
//    the unit impulse at the centre pixel c (N = H, or M0 H M0); |DFT(delta)| =
//    1, so Lambda~ is the modulus of the response's DFT.  The modulus replaces
//    the real part: for a shift-variant H the phase-corrected ratio is complex
//    and its real part can be negative.
//  * Haar (Eqs. 18, 34): Lambda~_k = [U N U^T xi]_k / [U U^T xi]_k with xi
//    the indicator of one subband of one level restricted to one class of a
//    P x P position lattice (one test function per set; P = 0 is the single
//    all-ones test function U^T 1).
//  * Eigenvalues clamped to >= 1e-6 of the largest before the -1/2 power.
// |M| for the separable curvature: Fourier uses the circulant of the absolute
// kernel |IDFT(Lambda~^-1/2)|, Haar the all-positive taps |U|, blocks |M0|.
#include <cmath>
#include <vector>

#include "haar.cuh"
#include "model.cuh"
#include "precond.cuh"

namespace psps {
namespace {

constexpr int kThreads = 256;
inline unsigned nblk(int64_t n) { return (unsigned)cdiv(n, kThreads); }

__global__ void set_value_kernel(float *p, int64_t idx, float v) { p[idx] = v; }

__global__ void fill_kernel(float *p, int64_t n, float v) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        p[i] = v;
}

// out[c][j] = a[c][j] * b[j]  (b broadcast over channels)
__global__ void mul_bcast_kernel(const float *a, const float *b, float *out, int64_t n, int channels) {
    const int64_t tot = n * channels;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < tot; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = a[i] * b[i % n];
}

// u[p][m][i] = sum_k F_i[m][k] l[p][k][i]; F packed upper triangle [nm(nm+1)/2][n_rays]
__global__ void fisher_mul_kernel(int nm, int nprobe, int64_t n_rays, const float *__restrict__ F,
                                  const float *__restrict__ l, float *__restrict__ u) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_rays) return;
    float f[4][4];
    int k = 0;
    for (int a = 0; a < nm; ++a)
        for (int b = a; b < nm; ++b, ++k) f[a][b] = f[b][a] = F[(int64_t)k * n_rays + i];
    for (int p = 0; p < nprobe; ++p) {
        float lv[4];
        for (int m = 0; m < nm; ++m) lv[m] = l[((int64_t)p * nm + m) * n_rays + i];
        for (int m = 0; m < nm; ++m) {
            float acc = 0.f;
            for (int kk = 0; kk < nm; ++kk) acc = fmaf(f[m][kk], lv[kk], acc);
            u[((int64_t)p * nm + m) * n_rays + i] = acc;
        }
    }
}

__global__ void modulus_kernel(const float2 *Z, float *out, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = hypotf(Z[i].x, Z[i].y);
}

__global__ void real_part_kernel(const float2 *Z, float *out, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = Z[i].x;
}

__global__ void abs_copy_kernel(const float *in, float *out, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = fabsf(in[i]);
}

__global__ void abs_kernel(float *p, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        p[i] = fabsf(p[i]);
}

// s = max(|lam|, floor)^-1/2 (FP64 arithmetic)
__global__ void invsqrt_clamp_kernel(const float *lam, double floor_v, float *s, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double v = fabs((double)lam[i]);
        if (v < floor_v) v = floor_v;
        s[i] = (float)(1.0 / sqrt(v));
    }
}

// Indicator of one Haar test set in the Mallat layout of an n x n image:
// level block size h (n, n/2, ..., 2), band 0 = HL (top right), 1 = LH
// (bottom left), 2 = HH (bottom right), 3 = final low-pass block; lattice
// class (a, c) of the position inside the band modulo P (P = 0: all ones).
__global__ void haar_mask_kernel(int n, int h, int band, int a, int c, int P, float *out) {
    const int64_t nn = (int64_t)n * n;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nn; t += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(t / n), j = (int)(t % n);
        float v = 0.f;
        if (P == 0) {
            v = 1.f;
        } else {
            const int h2 = h / 2;
            int r0 = 0, c0 = 0;
            bool in;
            if (band == 3) {
                in = i < h2 && j < h2;
            } else {
                r0 = band == 0 ? 0 : h2;
                c0 = band == 1 ? 0 : h2;
                in = i >= r0 && i < r0 + h2 && j >= c0 && j < c0 + h2;
                if (in) in = ((i - r0) % P == a) && ((j - c0) % P == c);
            }
            v = in ? 1.f : 0.f;
        }
        out[t] = v;
    }
}

// 3-D: indicator of one test set of an n^3 volume: level block size h, detail
// octant (sz, sy, sx) = bits of band + 1 (band 0..6), band 7 = final
// low-pass block; lattice class (a, b, c) of the (z, y, x) position inside
// the octant modulo P (P = 0: all ones).
__global__ void haar_mask3_kernel(int n, int h, int band, int a, int b, int c, int P, float *out) {
    const int64_t nnn = (int64_t)n * n * n;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nnn; t += (int64_t)gridDim.x * blockDim.x) {
        const int z = (int)(t / ((int64_t)n * n)), y = (int)((t / n) % n), x = (int)(t % n);
        float v = 1.f;
        if (P != 0) {
            const int h2 = h / 2;
            bool in;
            if (band == 7) {
                in = z < h2 && y < h2 && x < h2;
            } else {
                const int oct = band + 1;
                const int z0 = (oct >> 2) * h2, y0 = ((oct >> 1) & 1) * h2, x0 = (oct & 1) * h2;
                in = z >= z0 && z < z0 + h2 && y >= y0 && y < y0 + h2 && x >= x0 && x < x0 + h2;
                if (in) in = ((z - z0) % P == a) && ((y - y0) % P == b) && ((x - x0) % P == c);
            }
            v = in ? 1.f : 0.f;
        }
        out[t] = v;
    }
}

__global__ void masked_ratio_kernel(const float *mask, const float *r, const float *den, float *lam, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        if (mask[i] != 0.f) lam[i] = r[i] / den[i];
}

// Column k of the cross-material wavelet blocks (Eqs. 59-60) at the
// coefficients of one test set: K[m][k][j] = r[m][j] / den[j] where mask[j].
__global__ void masked_block_ratio_kernel(const float *mask, const float *r, const float *den, float *K, int nm, int k,
                                          int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        if (mask[i] != 0.f)
            for (int m = 0; m < nm; ++m) K[((int64_t)m * nm + k) * n + i] = r[(int64_t)m * n + i] / den[i];
}

__global__ void to_complex_kernel(const float *in, float2 *out, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = make_float2(in[i], 0.f);
}

// Symmetric inverse square root of nm x nm blocks (FP64, cyclic Jacobi).
// H[a][b][j] full (both triangles); writes B and |B| as [a][b][j].
__global__ void block_invsqrt_kernel(int nm, int64_t n, const float *__restrict__ H, double max_trace,
                                     float *__restrict__ Bout, float *__restrict__ Babs) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    double A[4][4], V[4][4];
    double tr = 0.0;
    for (int a = 0; a < nm; ++a)
        for (int b = 0; b < nm; ++b) {
            A[a][b] = 0.5 * ((double)H[((int64_t)a * nm + b) * n + j] + (double)H[((int64_t)b * nm + a) * n + j]);
            V[a][b] = a == b ? 1.0 : 0.0;
        }
    for (int a = 0; a < nm; ++a) tr += A[a][a];
    const bool dead = !(tr > 1e-12 * max_trace);
    if (nm > 1 && !dead) {
        for (int sweep = 0; sweep < 20; ++sweep) {
            double off = 0.0;
            for (int p = 0; p < nm; ++p)
                for (int q = p + 1; q < nm; ++q) off += A[p][q] * A[p][q];
            if (off < 1e-30 * tr * tr) break;
            for (int p = 0; p < nm; ++p)
                for (int q = p + 1; q < nm; ++q) {
                    if (A[p][q] == 0.0) continue;
                    const double theta = (A[q][q] - A[p][p]) / (2.0 * A[p][q]);
                    const double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                    const double cs = 1.0 / sqrt(t * t + 1.0), sn = t * cs;
                    for (int k = 0; k < nm; ++k) {
                        const double akp = A[k][p], akq = A[k][q];
                        A[k][p] = cs * akp - sn * akq;
                        A[k][q] = sn * akp + cs * akq;
                    }
                    for (int k = 0; k < nm; ++k) {
                        const double apk = A[p][k], aqk = A[q][k];
                        A[p][k] = cs * apk - sn * aqk;
                        A[q][k] = sn * apk + cs * aqk;
                    }
                    for (int k = 0; k < nm; ++k) {
                        const double vkp = V[k][p], vkq = V[k][q];
                        V[k][p] = cs * vkp - sn * vkq;
                        V[k][q] = sn * vkp + cs * vkq;
                    }
                }
        }
    }
    double lam[4], lmax = 0.0;
    for (int a = 0; a < nm; ++a) {
        lam[a] = A[a][a];
        if (lam[a] > lmax) lmax = lam[a];
    }
    for (int a = 0; a < nm; ++a) {
        double v = lam[a];
        if (v < 1e-6 * lmax) v = 1e-6 * lmax;
        lam[a] = v > 0 ? 1.0 / sqrt(v) : 0.0;
    }
    for (int a = 0; a < nm; ++a)
        for (int b = 0; b < nm; ++b) {
            double v = 0.0;
            if (!dead)
                for (int k = 0; k < nm; ++k) v += V[a][k] * lam[k] * V[b][k];
            Bout[((int64_t)a * nm + b) * n + j] = (float)v;
            Babs[((int64_t)a * nm + b) * n + j] = (float)fabs(v);
        }
}

// out[m][j] = sum_k B[m][k][j] in[k][j]   (transpose: B[k][m][j])
__global__ void block_apply_kernel(int nm, int64_t n, const float *__restrict__ B, const float *__restrict__ in,
                                   float *__restrict__ out, int transpose) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
        float v[4];
        for (int k = 0; k < nm; ++k) v[k] = in[(int64_t)k * n + j];
        for (int m = 0; m < nm; ++m) {
            float acc = 0.f;
            for (int k = 0; k < nm; ++k) {
                const int64_t bi = transpose ? ((int64_t)k * nm + m) : ((int64_t)m * nm + k);
                acc = fmaf(B[bi * n + j], v[k], acc);
            }
            out[(int64_t)m * n + j] = acc;
        }
    }
}

// Cyclic Jacobi eigendecomposition of a symmetric n x n matrix (n <= 8, FP64):
// A is destroyed (its diagonal becomes the eigenvalues), V gets the
// eigenvectors as columns.
__device__ void sym_eig(int n, double (&A)[8][8], double (&V)[8][8]) {
    for (int a = 0; a < n; ++a)
        for (int b = 0; b < n; ++b) V[a][b] = a == b ? 1.0 : 0.0;
    double scale = 0.0;
    for (int a = 0; a < n; ++a) scale += A[a][a] * A[a][a];
    for (int sweep = 0; sweep < 30; ++sweep) {
        double off = 0.0;
        for (int p = 0; p < n; ++p)
            for (int q = p + 1; q < n; ++q) off += A[p][q] * A[p][q];
        if (off <= 1e-30 * scale || off == 0.0) break;
        for (int p = 0; p < n; ++p)
            for (int q = p + 1; q < n; ++q) {
                if (A[p][q] == 0.0) continue;
                const double theta = (A[q][q] - A[p][p]) / (2.0 * A[p][q]);
                const double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                const double cs = 1.0 / sqrt(t * t + 1.0), sn = t * cs;
                for (int k = 0; k < n; ++k) {
                    const double akp = A[k][p], akq = A[k][q];
                    A[k][p] = cs * akp - sn * akq;
                    A[k][q] = sn * akp + cs * akq;
                }
                for (int k = 0; k < n; ++k) {
                    const double apk = A[p][k], aqk = A[q][k];
                    A[p][k] = cs * apk - sn * aqk;
                    A[q][k] = sn * apk + cs * aqk;
                }
                for (int k = 0; k < n; ++k) {
                    const double vkp = V[k][p], vkq = V[k][q];
                    V[k][p] = cs * vkp - sn * vkq;
                    V[k][q] = sn * vkp + cs * vkq;
                }
            }
    }
}

// Z[a][f] <- sum_b L[a][b][f] Z[b][f] for every frequency f (nm <= 4).
__global__ void mix_kernel(int nm, int64_t n, const float *__restrict__ L, float2 *__restrict__ Z) {
    for (int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; f < n; f += (int64_t)gridDim.x * blockDim.x) {
        float2 v[4];
        for (int b = 0; b < nm; ++b) v[b] = Z[(int64_t)b * n + f];
        for (int a = 0; a < nm; ++a) {
            float2 acc = make_float2(0.f, 0.f);
            for (int b = 0; b < nm; ++b) {
                const float l = L[((int64_t)a * nm + b) * n + f];
                acc.x = fmaf(l, v[b].x, acc.x);
                acc.y = fmaf(l, v[b].y, acc.y);
            }
            Z[(int64_t)a * n + f] = acc;
        }
    }
}

// Lc[a][k][f] = Z[a][f] / DFT(delta_c)(f) = Z[a][f] exp(+2 pi i (fy cy/ny + fx cx/nx))
__global__ void phase_kernel(int nm, int nx, int ny, int nz, int cx, int cy, int cz, const float2 *__restrict__ Z,
                             int k, float2 *__restrict__ Lc) {
    const int64_t n = (int64_t)nx * ny * nz;
    for (int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; f < n; f += (int64_t)gridDim.x * blockDim.x) {
        const int fx = (int)(f % nx), fy = (int)((f / nx) % ny), fz = (int)(f / ((int64_t)nx * ny));
        const double ang = 2.0 * M_PI *
                           ((double)((int64_t)fz * cz % nz) / nz + (double)((int64_t)fy * cy % ny) / ny +
                            (double)((int64_t)fx * cx % nx) / nx);
        double sn, cs;
        sincos(ang, &sn, &cs);
        for (int a = 0; a < nm; ++a) {
            const float2 z = Z[(int64_t)a * n + f];
            Lc[((int64_t)a * nm + k) * n + f] = make_float2((float)(z.x * cs - z.y * sn), (float)(z.x * sn + z.y * cs));
        }
    }
}

// P = Re((L^H L)^1/2), symmetrised (the block analogue of |lambda|), and its
// largest eigenvalue, per frequency (FP64; the Hermitian square root through
// the real 2nm x 2nm embedding [[Re, -Im], [Im, Re]]).
__global__ void polar_kernel(int nm, int64_t n, const float2 *__restrict__ Lc, float *__restrict__ P,
                             float *__restrict__ lmax) {
    const int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= n) return;
    double Lr[4][4], Li[4][4];
    for (int a = 0; a < nm; ++a)
        for (int b = 0; b < nm; ++b) {
            const float2 z = Lc[((int64_t)a * nm + b) * n + f];
            Lr[a][b] = z.x;
            Li[a][b] = z.y;
        }
    double E[8][8], V[8][8];
    const int m2 = 2 * nm;
    for (int a = 0; a < nm; ++a)
        for (int b = 0; b < nm; ++b) {
            double gr = 0.0, gi = 0.0;  // G = L^H L: G_ab = sum_c conj(L_ca) L_cb
            for (int c = 0; c < nm; ++c) {
                gr += Lr[c][a] * Lr[c][b] + Li[c][a] * Li[c][b];
                gi += Lr[c][a] * Li[c][b] - Li[c][a] * Lr[c][b];
            }
            E[a][b] = gr;
            E[a + nm][b + nm] = gr;
            E[a][b + nm] = -gi;
            E[a + nm][b] = gi;
        }
    sym_eig(m2, E, V);
    double S[4][4];
    for (int a = 0; a < nm; ++a)
        for (int b = 0; b < nm; ++b) {
            double v = 0.0;
            for (int k = 0; k < m2; ++k) v += V[a][k] * sqrt(fmax(E[k][k], 0.0)) * V[b][k];
            S[a][b] = v;
        }
    double A[8][8];
    for (int a = 0; a < nm; ++a)
        for (int b = 0; b < nm; ++b) {
            A[a][b] = 0.5 * (S[a][b] + S[b][a]);
            P[((int64_t)a * nm + b) * n + f] = (float)A[a][b];
        }
    sym_eig(nm, A, V);
    double mx = A[0][0];
    for (int a = 1; a < nm; ++a) mx = fmax(mx, A[a][a]);
    lmax[f] = (float)mx;
}

// Largest eigenvalue of every symmetric block P[a][b][f] (FP64).
__global__ void block_lmax_kernel(int nm, int64_t n, const float *__restrict__ P, float *__restrict__ lmax) {
    const int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= n) return;
    double A[8][8], V[8][8];
    for (int a = 0; a < nm; ++a)
        for (int b = 0; b < nm; ++b)
            A[a][b] = 0.5 * ((double)P[((int64_t)a * nm + b) * n + f] + (double)P[((int64_t)b * nm + a) * n + f]);
    sym_eig(nm, A, V);
    double mx = A[0][0];
    for (int a = 1; a < nm; ++a) mx = fmax(mx, A[a][a]);
    lmax[f] = (float)mx;
}

// Li = P^-1/2 with every eigenvalue clamped to >= floor (FP64).
__global__ void invsqrt_floor_kernel(int nm, int64_t n, const float *__restrict__ P, double floor_v,
                                     float *__restrict__ Li) {
    const int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= n) return;
    double A[8][8], V[8][8];
    for (int a = 0; a < nm; ++a)
        for (int b = 0; b < nm; ++b)
            A[a][b] = 0.5 * ((double)P[((int64_t)a * nm + b) * n + f] + (double)P[((int64_t)b * nm + a) * n + f]);
    sym_eig(nm, A, V);
    double s[4];
    for (int a = 0; a < nm; ++a) s[a] = 1.0 / sqrt(fmax(A[a][a], floor_v));
    for (int a = 0; a < nm; ++a)
        for (int b = 0; b < nm; ++b) {
            double v = 0.0;
            for (int k = 0; k < nm; ++k) v += V[a][k] * s[k] * V[b][k];
            Li[((int64_t)a * nm + b) * n + f] = (float)v;
        }
}

// The Haar test sets of an n x n image: one per (level block h, detail band,
// lattice class (a, c) mod P), plus the final low-pass block; of an n^3
// volume: one per (h, detail octant, class (a, b, c) mod P), plus the final
// low-pass block.  P = 0 gives the paper's single all-ones set.
struct HaarSet {
    int h, band, a, b, c;
};

std::vector<HaarSet> haar_sets(int nx, int P, int nz) {
    std::vector<HaarSet> sets;
    if (P == 0) {
        sets.push_back({nx, 0, 0, 0, 0});
        return sets;
    }
    const bool vol = nz > 1;
    for (int h = nx; h >= 2; h /= 2) {
        const int h2 = h / 2, L = P < h2 ? P : h2;
        for (int band = 0; band < (vol ? 7 : 3); ++band)
            for (int a = 0; a < L; ++a)
                for (int b = 0; b < (vol ? L : 1); ++b)
                    for (int c = 0; c < L; ++c) sets.push_back({h, band, a, b, c});
    }
    sets.push_back({2, vol ? 7 : 3, 0, 0, 0});
    return sets;
}

void launch_haar_mask(int nx, int nz, const HaarSet &st, int P, float *out, cudaStream_t s);

unsigned gs(int64_t n) {
    int64_t b = cdiv(n, kThreads);
    return (unsigned)(b > 4096 ? 4096 : (b < 1 ? 1 : b));
}

void launch_haar_mask(int nx, int nz, const HaarSet &st, int P, float *out, cudaStream_t s) {
    if (nz > 1)
        haar_mask3_kernel<<<gs((int64_t)nx * nx * nx), kThreads, 0, s>>>(nx, st.h, st.band, st.a, st.b, st.c, P, out);
    else
        haar_mask_kernel<<<gs((int64_t)nx * nx), kThreads, 0, s>>>(nx, st.h, st.band, st.a, st.c, P, out);
}

// Matrix-free Hessian H v = A^T F A v + R v for nprobe stacked vectors of nm
// materials (images), or F v per ray in the projection domain.
struct HessOp {
    mbir_plan *plan;
    int nm;
    int64_t n_rays, n;
    const float *F;
    PenaltyDev pd;
    bool has_pen;
    DBuf<float> l, u;
    mbir_status init(int max_ch) {
        if (plan) {
            PSPS_TRY(l.alloc((size_t)max_ch * n_rays));
            PSPS_TRY(u.alloc((size_t)max_ch * n_rays));
        }
        return MBIR_OK;
    }
    // precise: sum the transpose in FP32 with the deterministic pixel / voxel
    // gather instead of the fixed-point tile kernel, for the build steps
    // with few probes (M0 blocks, Fourier impulses), where each pixel's
    // response spans many decades and a grid of the launch-wide largest term
    // would dominate the error of its small values.
    mbir_status apply(const float *v, float *out, int nprobe, cudaStream_t s, bool precise = false) {
        const int ch = nprobe * nm;
        if (!plan) {
            fisher_mul_kernel<<<nblk(n_rays), kThreads, 0, s>>>(nm, nprobe, n_rays, F, v, out);
            PSPS_LAUNCH_CHECK();
            return MBIR_OK;
        }
        PSPS_TRY(project(plan, v, l.p, ch, s));
        fisher_mul_kernel<<<nblk(n_rays), kThreads, 0, s>>>(nm, nprobe, n_rays, F, l.p, u.p);
        PSPS_LAUNCH_CHECK();
        const int mode = plan->back_mode;
        if (precise && mode == 0) plan->back_mode = 1;
        const mbir_status bs = backproject(plan, u.p, out, ch, 0, s);
        plan->back_mode = mode;
        PSPS_TRY(bs);
        if (has_pen)
            for (int p = 0; p < nprobe; ++p)
                PSPS_TRY(launch_penalty(pd, plan->g.nx, plan->g.ny, plan->g.nz, v + (int64_t)p * nm * n, nullptr,
                                        out + (int64_t)p * nm * n, 1, 0, nullptr, penalty_blocks(n), s));
        return MBIR_OK;
    }
};

mbir_status host_max_abs(const float *d, int64_t n, double &mx, cudaStream_t s) {
    std::vector<float> h(n);
    PSPS_CUDA(cudaMemcpyAsync(h.data(), d, sizeof(float) * n, cudaMemcpyDeviceToHost, s));
    PSPS_CUDA(cudaStreamSynchronize(s));
    mx = 0.0;
    for (int64_t i = 0; i < n; ++i) mx = fmax(mx, fabs((double)h[i]));
    return MBIR_OK;
}

// s = clamp(|lam|)^-1/2 in place of `s`; s_abs = Re DFT |IDFT(s)| (Fourier only)
mbir_status finish_scalar(psps_precond *pc, float *lam, bool fourier, cudaStream_t s) {
    double mx;
    PSPS_TRY(host_max_abs(lam, pc->n, mx, s));
    if (!(mx > 0) || !std::isfinite(mx)) return fail(MBIR_ERR_NONFINITE, "preconditioner eigenvalues are not positive");
    invsqrt_clamp_kernel<<<gs(pc->n), kThreads, 0, s>>>(lam, 1e-6 * mx, pc->s.p, pc->n);
    PSPS_LAUNCH_CHECK();
    if (fourier) {
        // kernel k = IDFT(s): filter the unit impulse at the origin
        float *imp = pc->tmp.p, *k = pc->tmp.p + pc->n;
        PSPS_CUDA(cudaMemsetAsync(imp, 0, sizeof(float) * pc->n, s));
        set_value_kernel<<<1, 1, 0, s>>>(imp, 0, 1.f);
        PSPS_TRY(pc->fft.filter(1, imp, pc->Z.p, k, nullptr, nullptr, pc->s.p, s));
        abs_kernel<<<gs(pc->n), kThreads, 0, s>>>(k, pc->n);
        PSPS_TRY(pc->fft.forward(1, k, pc->Z.p, s));
        real_part_kernel<<<gs(pc->n), kThreads, 0, s>>>(pc->Z.p, pc->s_abs.p, pc->n);
        PSPS_LAUNCH_CHECK();
    } else {
        PSPS_CUDA(cudaMemcpyAsync(pc->s_abs.p, pc->s.p, sizeof(float) * pc->n, cudaMemcpyDeviceToDevice, s));
    }
    return MBIR_OK;
}

}  // namespace

mbir_status launch_abs_copy(const float *in, float *out, int64_t n, cudaStream_t s) {
    abs_copy_kernel<<<gs(n), kThreads, 0, s>>>(in, out, n);
    PSPS_LAUNCH_CHECK();
    return MBIR_OK;
}
mbir_status launch_fill(float *p, int64_t n, float v, cudaStream_t s) {
    fill_kernel<<<gs(n), kThreads, 0, s>>>(p, n, v);
    PSPS_LAUNCH_CHECK();
    return MBIR_OK;
}
mbir_status finish_scalar_pub(psps_precond *pc, float *lam, bool fourier, cudaStream_t s) {
    return finish_scalar(pc, lam, fourier, s);
}

// Li = P^-1/2 (global eigenvalue floor 1e-6 of the largest) and its
// absolute-kernel spectra Li_abs[a][b] = Re DFT |IDFT(Li[a][b])|.
mbir_status finish_cross_fourier(psps_precond *pc, const float *P, const float *lmax, cudaStream_t s) {
    const int nm = pc->nm;
    const int64_t n = pc->n;
    double mx;
    PSPS_TRY(host_max_abs(lmax, n, mx, s));
    if (!(mx > 0) || !std::isfinite(mx)) return fail(MBIR_ERR_NONFINITE, "cross-material eigenvalues are not positive");
    PSPS_TRY(pc->Li.alloc((size_t)nm * nm * n));
    PSPS_TRY(pc->Li_abs.alloc((size_t)nm * nm * n));
    invsqrt_floor_kernel<<<(unsigned)cdiv(n, 128), 128, 0, s>>>(nm, n, P, 1e-6 * mx, pc->Li.p);
    PSPS_LAUNCH_CHECK();
    float *imp = pc->tmp.p, *k = pc->tmp.p + n;
    for (int ab = 0; ab < nm * nm; ++ab) {
        PSPS_CUDA(cudaMemsetAsync(imp, 0, sizeof(float) * n, s));
        set_value_kernel<<<1, 1, 0, s>>>(imp, 0, 1.f);
        PSPS_TRY(pc->fft.filter(1, imp, pc->Z.p, k, nullptr, nullptr, pc->Li.p + (int64_t)ab * n, s));
        abs_kernel<<<gs(n), kThreads, 0, s>>>(k, n);
        PSPS_TRY(pc->fft.forward(1, k, pc->Z.p, s));
        real_part_kernel<<<gs(n), kThreads, 0, s>>>(pc->Z.p, pc->Li_abs.p + (int64_t)ab * n, n);
        PSPS_LAUNCH_CHECK();
    }
    PSPS_CUDA(cudaStreamSynchronize(s));
    return MBIR_OK;
}

// Ki = P^-1/2 (global eigenvalue floor 1e-6 of the largest), |Ki| elementwise
// (the wavelet-domain operator is block diagonal, so |.| acts per block).
mbir_status finish_cross_haar(psps_precond *pc, const float *P, const float *lmax, cudaStream_t s) {
    const int nm = pc->nm;
    const int64_t n = pc->n;
    double mx;
    PSPS_TRY(host_max_abs(lmax, n, mx, s));
    if (!(mx > 0) || !std::isfinite(mx)) return fail(MBIR_ERR_NONFINITE, "cross-material eigenvalues are not positive");
    PSPS_TRY(pc->Li.alloc((size_t)nm * nm * n));
    PSPS_TRY(pc->Li_abs.alloc((size_t)nm * nm * n));
    invsqrt_floor_kernel<<<(unsigned)cdiv(n, 128), 128, 0, s>>>(nm, n, P, 1e-6 * mx, pc->Li.p);
    PSPS_LAUNCH_CHECK();
    abs_copy_kernel<<<gs((int64_t)nm * nm * n), kThreads, 0, s>>>(pc->Li.p, pc->Li_abs.p, (int64_t)nm * nm * n);
    PSPS_LAUNCH_CHECK();
    PSPS_CUDA(cudaStreamSynchronize(s));
    return MBIR_OK;
}

mbir_status launch_block_lmax(int nm, int64_t n, const float *P, float *lmax, cudaStream_t s) {
    block_lmax_kernel<<<(unsigned)cdiv(n, 128), 128, 0, s>>>(nm, n, P, lmax);
    PSPS_LAUNCH_CHECK();
    return MBIR_OK;
}

mbir_status launch_polar(int nm, int64_t n, const float2 *Lc, float *P, float *lmax, cudaStream_t s) {
    polar_kernel<<<(unsigned)cdiv(n, 128), 128, 0, s>>>(nm, n, Lc, P, lmax);
    PSPS_LAUNCH_CHECK();
    return MBIR_OK;
}

mbir_status launch_phase(int nm, int nx, int ny, int nz, const float2 *Z, int k, float2 *Lc, cudaStream_t s) {
    phase_kernel<<<gs((int64_t)nx * ny * nz), kThreads, 0, s>>>(nm, nx, ny, nz, nx / 2, ny / 2, nz / 2, Z, k, Lc);
    PSPS_LAUNCH_CHECK();
    return MBIR_OK;
}

mbir_status launch_block_apply(int nm, int64_t n, const float *B, const float *in, float *out, int transpose,
                               cudaStream_t s) {
    block_apply_kernel<<<gs(n), kThreads, 0, s>>>(nm, n, B, in, out, transpose);
    PSPS_LAUNCH_CHECK();
    return MBIR_OK;
}

mbir_status precond_apply(psps_precond *pc, int op, const float *in, float *out, cudaStream_t s) {
    const bool absm = (op == PSPS_APPLY_ABS_M || op == PSPS_APPLY_ABS_MT);
    const bool tr = (op == PSPS_APPLY_MT || op == PSPS_APPLY_ABS_MT);
    const int64_t tot = pc->n * pc->nm;
    // Where M0 enters the Fourier and wavelet kinds: one-sided M = M0 C
    // (M^T = C^T M0^T: M0 before the transform for M^T, after it for M) or
    // the literal two-sided M0^T C M0 (both).
    const bool m0_before = pc->sides == 2 || tr;
    const bool m0_after = pc->sides == 2 || !tr;
    switch (pc->kind) {
        case PSPS_PRECOND_NONE:
            if (in != out) PSPS_CUDA(cudaMemcpyAsync(out, in, sizeof(float) * tot, cudaMemcpyDeviceToDevice, s));
            return MBIR_OK;
        case PSPS_PRECOND_FOURIER:
        case PSPS_PRECOND_MOD_FOURIER: {
            // C and |C| are symmetric circulants
            const float *m0 = pc->kind == PSPS_PRECOND_MOD_FOURIER ? pc->m0.p : nullptr;
            return pc->fft.filter(pc->nm, in, pc->Z.p, out, m0_before ? m0 : nullptr, m0_after ? m0 : nullptr,
                                  absm ? pc->s_abs.p : pc->s.p, s);
        }
        case PSPS_PRECOND_HAAR:
            return haar_apply(pc->nx, pc->nm, in, pc->tmp.p, out, m0_before ? pc->m0.p : nullptr,
                              m0_after ? pc->m0.p : nullptr, pc->s.p, absm ? 0xffffffffu : 0u, s, pc->nz);
        case PSPS_PRECOND_BLOCK:
            block_apply_kernel<<<gs(pc->n), kThreads, 0, s>>>(pc->nm, pc->n, absm ? pc->Babs.p : pc->B.p, in, out,
                                                              tr ? 1 : 0);
            PSPS_LAUNCH_CHECK();
            return MBIR_OK;
        case PSPS_PRECOND_BLOCK_FOURIER: {
            // M = M0^T C M0 (Eq. 57) or M0^T C with C = U^H L^-1/2 U; the
            // per-frequency blocks are symmetric, so C^T = C; |M| uses |M0|
            // and the absolute-kernel spectra.  M^T applies M0 first.
            const float *Bm = absm ? pc->Babs.p : pc->B.p;
            float *t0 = pc->tmp.p, *t1 = pc->tmp.p + pc->n * pc->nm;
            const float *src = in;
            if (m0_before) {
                block_apply_kernel<<<gs(pc->n), kThreads, 0, s>>>(pc->nm, pc->n, Bm, in, t0, 0);
                PSPS_LAUNCH_CHECK();
                src = t0;
            }
            PSPS_TRY(pc->fft.forward(pc->nm, src, pc->Z.p, s));
            mix_kernel<<<gs(pc->n), kThreads, 0, s>>>(pc->nm, pc->n, absm ? pc->Li_abs.p : pc->Li.p, pc->Z.p);
            PSPS_LAUNCH_CHECK();
            PSPS_TRY(pc->fft.inverse(pc->nm, pc->Z.p, m0_after ? t1 : out, nullptr, s));
            if (m0_after) {
                block_apply_kernel<<<gs(pc->n), kThreads, 0, s>>>(pc->nm, pc->n, Bm, t1, out, 1);
                PSPS_LAUNCH_CHECK();
            }
            return MBIR_OK;
        }
        case PSPS_PRECOND_BLOCK_HAAR: {
            // M = M0^T U^T K^-1/2 U M0 (Eq. 61) or M0^T U^T K^-1/2 U, U per
            // material; M^T swaps the blocks of K^-1/2 and applies M0 first;
            // |M| uses |M0|, |U| and |K^-1/2|.
            const float *Bm = absm ? pc->Babs.p : pc->B.p;
            const unsigned amask = absm ? 0xffffffffu : 0u;
            float *t0 = pc->tmp.p, *t1 = pc->tmp.p + pc->n * pc->nm;
            const float *src = in;
            if (m0_before) {
                block_apply_kernel<<<gs(pc->n), kThreads, 0, s>>>(pc->nm, pc->n, Bm, in, t0, 0);
                PSPS_LAUNCH_CHECK();
                src = t0;
            }
            PSPS_TRY(haar_forward(pc->nx, pc->nm, src, t1, nullptr, nullptr, amask, s, pc->nz));
            block_apply_kernel<<<gs(pc->n), kThreads, 0, s>>>(pc->nm, pc->n, absm ? pc->Li_abs.p : pc->Li.p, t1, t0,
                                                              tr ? 1 : 0);
            PSPS_LAUNCH_CHECK();
            PSPS_TRY(haar_inverse(pc->nx, pc->nm, t0, m0_after ? t1 : out, nullptr, amask, s, pc->nz));
            if (m0_after) {
                block_apply_kernel<<<gs(pc->n), kThreads, 0, s>>>(pc->nm, pc->n, Bm, t1, out, 1);
                PSPS_LAUNCH_CHECK();
            }
            return MBIR_OK;
        }
        default:
            return fail(MBIR_ERR_UNIMPLEMENTED, "preconditioner kind %d not built", pc->kind);
    }
}

mbir_status precond_apply2(psps_precond *pc, int op0, const float *in0, float *out0, int op1, const float *in1,
                           float *out1, cudaStream_t s) {
    PSPS_TRY(precond_apply(pc, op0, in0, out0, s));
    return precond_apply(pc, op1, in1, out1, s);
}

}  // namespace psps

using namespace psps;

namespace {

// Where M0 enters by default: the literal two-sided M0^T C M0 for a scalar
// M0 (its remainder M0^2 in M^T H M is diagonal, absorbed by the separable
// curvature), the one-sided M0^T C for per-pixel blocks (the remainder
// M0^T M0 would couple the materials of a pixel).
int default_sides(int kind) {
    return (kind == PSPS_PRECOND_BLOCK_FOURIER || kind == PSPS_PRECOND_BLOCK_HAAR) ? 1 : 2;
}

mbir_status build_impl(mbir_plan *plan, const mbmd_spectrum *spec, int kind, const float *y, int64_t n_rays,
                       const double *beta, int haar_lattice, cudaStream_t s, psps_precond *pc) {
    const int nm = spec->n_mat;
    pc->kind = kind;
    pc->nm = nm;
    pc->sides = default_sides(kind);
    pc->image = plan != nullptr;
    if (plan) {
        pc->nx = plan->g.nx;
        pc->ny = plan->g.ny;
        pc->nz = plan->g.kind == MBIR_CONE3D ? plan->g.nz : 1;
        pc->n = plan->n_pix;
    } else {
        pc->nx = (int)n_rays;
        pc->ny = 1;
        pc->n = n_rays;
    }
    if (kind == PSPS_PRECOND_NONE) return MBIR_OK;
    if (!plan && kind != PSPS_PRECOND_BLOCK)
        return fail(MBIR_ERR_ARG, "projection-domain decomposition supports NONE and BLOCK preconditioners");
    if ((kind == PSPS_PRECOND_FOURIER || kind == PSPS_PRECOND_MOD_FOURIER || kind == PSPS_PRECOND_HAAR) && nm != 1)
        return fail(MBIR_ERR_ARG, "Fourier / modified Fourier / Haar preconditioners are single-material (n_mat = 1)");
    const bool haar_kind = kind == PSPS_PRECOND_HAAR || kind == PSPS_PRECOND_BLOCK_HAAR;
    if (haar_kind && !haar_supported(pc->nx, plan->g.ny, pc->nz))
        return fail(MBIR_ERR_ARG,
                    "Haar preconditioners need a square power-of-two image (<= 2048) or a cubic power-of-two volume "
                    "(<= 256)");
    if (haar_kind && (haar_lattice < 0 || haar_lattice > 64)) return fail(MBIR_ERR_ARG, "haar_lattice must be 0..64");
    if (kind == PSPS_PRECOND_FOURIER || kind == PSPS_PRECOND_MOD_FOURIER || kind == PSPS_PRECOND_BLOCK_FOURIER)
        PSPS_TRY(pc->fft.init(pc->nx, pc->ny, pc->nz));

    const int64_t n = pc->n;
    // the impulse of the Fourier estimates sits at the centre voxel
    const int64_t centre = ((int64_t)(pc->nz / 2) * pc->ny + pc->ny / 2) * pc->nx + pc->nx / 2;
    const int nF = nm * (nm + 1) / 2;
    DBuf<float> F;
    PSPS_TRY(F.alloc((size_t)nF * n_rays));
    PSPS_TRY(launch_fisher_blocks(spec, n_rays, y, F.p, s));

    HessOp H{plan, nm, n_rays, n, F.p, PenaltyDev{}, false};
    H.pd.nm = nm;
    for (int a = 0; a < 16; ++a) H.pd.beta[a] = 0.f;
    if (beta && plan) {
        for (int a = 0; a < nm; ++a)
            for (int b = 0; b < nm; ++b) {
                H.pd.beta[a * 4 + b] = (float)beta[a * nm + b];
                if (beta[a * nm + b] != 0.0) H.has_pen = true;
            }
    }
    const int max_ch = plan ? plan->n_mat_max : nm * nm;
    PSPS_TRY(H.init(max_ch));
    PSPS_TRY(pc->tmp.alloc((size_t)n * (nm * 2 > max_ch ? nm * 2 : max_ch) * 2));
    PSPS_TRY(pc->Z.alloc((size_t)n * nm * 2));
    PSPS_TRY(pc->s.alloc(n));
    PSPS_TRY(pc->s_abs.alloc(n));

    // ---- M0 blocks from (F+R) 1_k (Eqs. 30, 53-54): all nm probes at once
    {
        DBuf<float> ones, Hcols;
        PSPS_TRY(ones.alloc((size_t)nm * nm * n));
        PSPS_TRY(Hcols.alloc((size_t)nm * nm * n));
        PSPS_CUDA(cudaMemsetAsync(ones.p, 0, sizeof(float) * ones.n, s));
        for (int k = 0; k < nm; ++k)
            fill_kernel<<<gs(n), kThreads, 0, s>>>(ones.p + ((int64_t)k * nm + k) * n, n, 1.f);
        PSPS_LAUNCH_CHECK();
        // all nm probes at once when the plan has the channels, else one by one
        if (!plan || nm * nm <= max_ch) {
            PSPS_TRY(H.apply(ones.p, Hcols.p, nm, s, true));
        } else {
            for (int k = 0; k < nm; ++k)
                PSPS_TRY(H.apply(ones.p + (int64_t)k * nm * n, Hcols.p + (int64_t)k * nm * n, 1, s, true));
        }
        // Hcols[k][m][j] = (H 1_k)_m(j) = block[m][k] -> reorder to [m][k][j]
        // (kept with the preconditioner for psps_precondition_export)
        DBuf<float> &Hb = pc->Hblk;
        PSPS_TRY(Hb.alloc((size_t)nm * nm * n));
        for (int k = 0; k < nm; ++k)
            for (int m = 0; m < nm; ++m)
                PSPS_CUDA(cudaMemcpyAsync(Hb.p + ((int64_t)m * nm + k) * n, Hcols.p + ((int64_t)k * nm + m) * n,
                                          sizeof(float) * n, cudaMemcpyDeviceToDevice, s));
        // largest trace (host)
        std::vector<float> hb((size_t)nm * nm * n);
        PSPS_CUDA(cudaMemcpyAsync(hb.data(), Hb.p, sizeof(float) * hb.size(), cudaMemcpyDeviceToHost, s));
        PSPS_CUDA(cudaStreamSynchronize(s));
        double mt = 0.0;
        for (int64_t j = 0; j < n; ++j) {
            double t = 0.0;
            for (int a = 0; a < nm; ++a) t += hb[((size_t)a * nm + a) * n + j];
            mt = fmax(mt, t);
        }
        if (!(mt > 0) || !std::isfinite(mt)) return fail(MBIR_ERR_NONFINITE, "zero-frequency response is not positive");
        PSPS_TRY(pc->B.alloc((size_t)nm * nm * n));
        PSPS_TRY(pc->Babs.alloc((size_t)nm * nm * n));
        block_invsqrt_kernel<<<nblk(n), kThreads, 0, s>>>(nm, n, Hb.p, mt, pc->B.p, pc->Babs.p);
        PSPS_LAUNCH_CHECK();
        PSPS_CUDA(cudaStreamSynchronize(s));
    }
    if (kind == PSPS_PRECOND_BLOCK) return MBIR_OK;
    if (kind == PSPS_PRECOND_BLOCK_FOURIER) {
        // L_k of Eq. 56: DFT of M0^T H M0 delta_{c,k} over DFT(delta_c), for
        // each material k with the impulse at the centre pixel c
        DBuf<float2> Lc;
        DBuf<float> d, v, hv, P, lmax;
        PSPS_TRY(Lc.alloc((size_t)nm * nm * n));
        PSPS_TRY(d.alloc((size_t)nm * n));
        PSPS_TRY(v.alloc((size_t)nm * n));
        PSPS_TRY(hv.alloc((size_t)nm * n));
        for (int k = 0; k < nm; ++k) {
            PSPS_CUDA(cudaMemsetAsync(d.p, 0, sizeof(float) * nm * n, s));
            set_value_kernel<<<1, 1, 0, s>>>(d.p, (int64_t)k * n + centre, 1.f);
            PSPS_TRY(launch_block_apply(nm, n, pc->B.p, d.p, v.p, 0, s));
            PSPS_TRY(H.apply(v.p, hv.p, 1, s, true));
            PSPS_TRY(launch_block_apply(nm, n, pc->B.p, hv.p, v.p, 1, s));
            PSPS_TRY(pc->fft.forward(nm, v.p, pc->Z.p, s));
            PSPS_TRY(launch_phase(nm, pc->nx, pc->ny, pc->nz, pc->Z.p, k, Lc.p, s));
        }
        PSPS_TRY(P.alloc((size_t)nm * nm * n));
        PSPS_TRY(lmax.alloc(n));
        PSPS_TRY(launch_polar(nm, n, Lc.p, P.p, lmax.p, s));
        PSPS_TRY(pc->est.alloc(P.n));
        PSPS_CUDA(cudaMemcpyAsync(pc->est.p, P.p, sizeof(float) * P.n, cudaMemcpyDeviceToDevice, s));
        return finish_cross_fourier(pc, P.p, lmax.p, s);
    }
    if (kind == PSPS_PRECOND_BLOCK_HAAR) {
        // K_k of Eqs. 59-60 with the lattice test functions: for every test
        // set xi and material k, dx = U^T xi in material k; column k of the
        // blocks of the set's coefficients = U M0^T H M0 dx / (U dx).  The
        // (set, material) probes go through the Hessian in batches that fill
        // the plan's channels.
        const int nx = pc->nx, nz = pc->nz;
        const std::vector<HaarSet> sets = haar_sets(nx, haar_lattice, nz);
        const int np = max_ch / nm > 1 ? max_ch / nm : 1;
        DBuf<float> K, mask, coef, dx, den, d, v, hv, r;
        PSPS_TRY(K.alloc((size_t)nm * nm * n));
        PSPS_TRY(mask.alloc((size_t)np * n));
        PSPS_TRY(coef.alloc((size_t)np * n));
        PSPS_TRY(dx.alloc((size_t)np * n));
        PSPS_TRY(den.alloc((size_t)np * n));
        PSPS_TRY(d.alloc((size_t)np * nm * n));
        PSPS_TRY(v.alloc((size_t)np * nm * n));
        PSPS_TRY(hv.alloc((size_t)np * nm * n));
        PSPS_TRY(r.alloc((size_t)np * nm * n));
        PSPS_CUDA(cudaMemsetAsync(K.p, 0, sizeof(float) * K.n, s));
        const size_t n_pairs = sets.size() * (size_t)nm;
        for (size_t p0 = 0; p0 < n_pairs; p0 += np) {
            const int nb = (int)(n_pairs - p0 < (size_t)np ? n_pairs - p0 : np);
            for (int b = 0; b < nb; ++b)
                launch_haar_mask(nx, nz, sets[(p0 + b) / nm], haar_lattice, mask.p + (int64_t)b * n, s);
            PSPS_LAUNCH_CHECK();
            PSPS_CUDA(cudaMemcpyAsync(coef.p, mask.p, sizeof(float) * nb * n, cudaMemcpyDeviceToDevice, s));
            PSPS_TRY(haar_inverse(nx, nb, coef.p, dx.p, nullptr, 0u, s, nz));
            PSPS_TRY(haar_forward(nx, nb, dx.p, den.p, nullptr, nullptr, 0u, s, nz));
            PSPS_CUDA(cudaMemsetAsync(d.p, 0, sizeof(float) * nb * nm * n, s));
            for (int b = 0; b < nb; ++b) {
                const int k = (int)((p0 + b) % nm);
                PSPS_CUDA(cudaMemcpyAsync(d.p + ((int64_t)b * nm + k) * n, dx.p + (int64_t)b * n, sizeof(float) * n,
                                          cudaMemcpyDeviceToDevice, s));
            }
            for (int b = 0; b < nb; ++b)
                PSPS_TRY(launch_block_apply(nm, n, pc->B.p, d.p + (int64_t)b * nm * n, v.p + (int64_t)b * nm * n, 0, s));
            PSPS_TRY(H.apply(v.p, hv.p, nb, s));
            for (int b = 0; b < nb; ++b)
                PSPS_TRY(launch_block_apply(nm, n, pc->B.p, hv.p + (int64_t)b * nm * n, v.p + (int64_t)b * nm * n, 1, s));
            PSPS_TRY(haar_forward(nx, nb * nm, v.p, r.p, nullptr, nullptr, 0u, s, nz));
            for (int b = 0; b < nb; ++b) {
                const int k = (int)((p0 + b) % nm);
                masked_block_ratio_kernel<<<gs(n), kThreads, 0, s>>>(mask.p + (int64_t)b * n, r.p + (int64_t)b * nm * n,
                                                                     den.p + (int64_t)b * n, K.p, nm, k, n);
            }
            PSPS_LAUNCH_CHECK();
        }
        PSPS_TRY(pc->est.alloc(K.n));
        PSPS_CUDA(cudaMemcpyAsync(pc->est.p, K.p, sizeof(float) * K.n, cudaMemcpyDeviceToDevice, s));
        DBuf<float2> Kc;
        DBuf<float> P, lmax;
        PSPS_TRY(Kc.alloc((size_t)nm * nm * n));
        to_complex_kernel<<<gs((int64_t)nm * nm * n), kThreads, 0, s>>>(K.p, Kc.p, (int64_t)nm * nm * n);
        PSPS_LAUNCH_CHECK();
        PSPS_TRY(P.alloc((size_t)nm * nm * n));
        PSPS_TRY(lmax.alloc(n));
        PSPS_TRY(launch_polar(nm, n, Kc.p, P.p, lmax.p, s));
        return finish_cross_haar(pc, P.p, lmax.p, s);
    }
    // one material from here on: m0 = B
    PSPS_TRY(pc->m0.alloc(n));
    if (kind == PSPS_PRECOND_FOURIER) {
        fill_kernel<<<gs(n), kThreads, 0, s>>>(pc->m0.p, n, 1.f);
    } else {
        PSPS_CUDA(cudaMemcpyAsync(pc->m0.p, pc->B.p, sizeof(float) * n, cudaMemcpyDeviceToDevice, s));
    }
    const float *m0 = pc->m0.p;
    const int nx = pc->nx;
    // N v = m0 .* H (m0 .* v)
    auto applyN = [&](const float *v, float *out, int nprobe, bool precise) -> mbir_status {
        float *w = pc->tmp.p;  // nprobe * n
        mul_bcast_kernel<<<gs(n * nprobe), kThreads, 0, s>>>(v, m0, w, n, nprobe);
        PSPS_LAUNCH_CHECK();
        PSPS_TRY(H.apply(w, out, nprobe, s, precise));
        mul_bcast_kernel<<<gs(n * nprobe), kThreads, 0, s>>>(out, m0, out, n, nprobe);
        PSPS_LAUNCH_CHECK();
        return MBIR_OK;
    };
    DBuf<float> lam;
    PSPS_TRY(lam.alloc(n));
    if (kind == PSPS_PRECOND_FOURIER || kind == PSPS_PRECOND_MOD_FOURIER) {
        DBuf<float> d, r;
        PSPS_TRY(d.alloc(n));
        PSPS_TRY(r.alloc(n));
        PSPS_CUDA(cudaMemsetAsync(d.p, 0, sizeof(float) * n, s));
        set_value_kernel<<<1, 1, 0, s>>>(d.p, centre, 1.f);
        PSPS_TRY(applyN(d.p, r.p, 1, true));
        PSPS_TRY(pc->fft.forward(1, r.p, pc->Z.p, s));
        modulus_kernel<<<gs(n), kThreads, 0, s>>>(pc->Z.p, lam.p, n);
        PSPS_LAUNCH_CHECK();
        PSPS_TRY(pc->est.alloc(n));
        PSPS_CUDA(cudaMemcpyAsync(pc->est.p, lam.p, sizeof(float) * n, cudaMemcpyDeviceToDevice, s));
        PSPS_TRY(finish_scalar(pc, lam.p, true, s));
        PSPS_CUDA(cudaStreamSynchronize(s));
        return MBIR_OK;
    }
    // ---- Haar
    {
        const int P = haar_lattice;
        const int nz = pc->nz;
        const std::vector<HaarSet> sets = haar_sets(nx, P, nz);
        const int batch = plan->n_mat_max;
        DBuf<float> mask, dx, r, den, coef;
        PSPS_TRY(mask.alloc((size_t)batch * n));
        PSPS_TRY(dx.alloc((size_t)batch * n));
        PSPS_TRY(r.alloc((size_t)batch * n));
        PSPS_TRY(den.alloc((size_t)batch * n));
        PSPS_TRY(coef.alloc((size_t)batch * n));
        DBuf<float> tmp2;
        PSPS_TRY(tmp2.alloc((size_t)batch * n));
        PSPS_CUDA(cudaMemsetAsync(lam.p, 0, sizeof(float) * n, s));
        for (size_t s0 = 0; s0 < sets.size(); s0 += batch) {
            const int nb = (int)(sets.size() - s0 < (size_t)batch ? sets.size() - s0 : batch);
            for (int b = 0; b < nb; ++b) launch_haar_mask(nx, nz, sets[s0 + b], P, mask.p + (int64_t)b * n, s);
            PSPS_LAUNCH_CHECK();
            // dx = U^T xi  (haar_inverse uses its coefficient input as scratch)
            PSPS_CUDA(cudaMemcpyAsync(coef.p, mask.p, sizeof(float) * nb * n, cudaMemcpyDeviceToDevice, s));
            PSPS_TRY(haar_inverse(nx, nb, coef.p, dx.p, nullptr, 0u, s, nz));
            PSPS_TRY(applyN(dx.p, tmp2.p, nb, false));
            PSPS_TRY(haar_forward(nx, nb, tmp2.p, r.p, nullptr, nullptr, 0u, s, nz));
            PSPS_TRY(haar_forward(nx, nb, dx.p, den.p, nullptr, nullptr, 0u, s, nz));
            for (int b = 0; b < nb; ++b)
                masked_ratio_kernel<<<gs(n), kThreads, 0, s>>>(mask.p + (int64_t)b * n, r.p + (int64_t)b * n,
                                                               den.p + (int64_t)b * n, lam.p, n);
            PSPS_LAUNCH_CHECK();
        }
        PSPS_TRY(pc->est.alloc(n));
        PSPS_CUDA(cudaMemcpyAsync(pc->est.p, lam.p, sizeof(float) * n, cudaMemcpyDeviceToDevice, s));
        PSPS_TRY(finish_scalar(pc, lam.p, false, s));
        PSPS_CUDA(cudaStreamSynchronize(s));
    }
    return MBIR_OK;
}

}  // namespace

extern "C" mbir_status psps_precondition_build(mbir_plan *plan, const mbmd_spectrum *spec, int kind, const float *y,
                                               int64_t n_rays, const double *beta, int haar_lattice, mbir_stream stream,
                                               psps_precond **out) {
    if (!spec || !y || !out) return fail(MBIR_ERR_ARG, "psps_precondition_build: null argument");
    *out = nullptr;
    if (kind < PSPS_PRECOND_NONE || kind > PSPS_PRECOND_BLOCK_HAAR)
        return fail(MBIR_ERR_ARG, "psps_precondition_build: unknown kind %d", kind);
    if (plan && n_rays != plan->n_rays) return fail(MBIR_ERR_ARG, "psps_precondition_build: n_rays does not match plan");
    if (n_rays < 1) return fail(MBIR_ERR_ARG, "psps_precondition_build: n_rays must be >= 1");
    if (plan && spec->n_mat > plan->n_mat_max) return fail(MBIR_ERR_ARG, "psps_precondition_build: n_mat > n_mat_max");
    psps_precond *pc = new psps_precond();
    mbir_status st = build_impl(plan, spec, kind, y, n_rays, beta, haar_lattice, (cudaStream_t)stream, pc);
    if (st != MBIR_OK) {
        delete pc;
        return st;
    }
    *out = pc;
    return MBIR_OK;
}

namespace {
mbir_status create_impl(mbir_plan *plan, int kind, int nm, int64_t n, const float *lam, const float *m0,
                        const float *blocks, cudaStream_t s, psps_precond *pc) {
    pc->kind = kind;
    pc->nm = nm;
    pc->sides = default_sides(kind);
    pc->image = plan != nullptr;
    pc->n = n;
    pc->nx = plan ? plan->g.nx : (int)n;
    pc->ny = plan ? plan->g.ny : 1;
    pc->nz = plan && plan->g.kind == MBIR_CONE3D ? plan->g.nz : 1;
    if (kind == PSPS_PRECOND_NONE) return MBIR_OK;
    if (kind == PSPS_PRECOND_BLOCK) {
        if (!blocks) return fail(MBIR_ERR_ARG, "psps_precondition_create: BLOCK needs blocks");
        PSPS_TRY(pc->B.alloc((size_t)nm * nm * n));
        PSPS_TRY(pc->Babs.alloc((size_t)nm * nm * n));
        PSPS_CUDA(cudaMemcpyAsync(pc->B.p, blocks, sizeof(float) * pc->B.n, cudaMemcpyDeviceToDevice, s));
        PSPS_TRY(launch_abs_copy(blocks, pc->Babs.p, (int64_t)pc->B.n, s));
        PSPS_CUDA(cudaStreamSynchronize(s));
        return MBIR_OK;
    }
    if (kind == PSPS_PRECOND_BLOCK_FOURIER) {
        if (!plan || !lam || !blocks)
            return fail(MBIR_ERR_ARG, "psps_precondition_create: BLOCK_FOURIER needs a plan, lam (P blocks) and blocks");
        PSPS_TRY(pc->fft.init(pc->nx, pc->ny, pc->nz));
        PSPS_TRY(pc->B.alloc((size_t)nm * nm * n));
        PSPS_TRY(pc->Babs.alloc((size_t)nm * nm * n));
        PSPS_CUDA(cudaMemcpyAsync(pc->B.p, blocks, sizeof(float) * pc->B.n, cudaMemcpyDeviceToDevice, s));
        PSPS_TRY(launch_abs_copy(blocks, pc->Babs.p, (int64_t)pc->B.n, s));
        PSPS_TRY(pc->tmp.alloc((size_t)n * nm * 2));
        PSPS_TRY(pc->Z.alloc((size_t)n * nm));
        DBuf<float> lmax;
        PSPS_TRY(lmax.alloc(n));
        PSPS_TRY(launch_block_lmax(nm, n, lam, lmax.p, s));
        return finish_cross_fourier(pc, lam, lmax.p, s);
    }
    if (kind == PSPS_PRECOND_BLOCK_HAAR) {
        if (!plan || !lam || !blocks)
            return fail(MBIR_ERR_ARG, "psps_precondition_create: BLOCK_HAAR needs a plan, lam (P blocks) and blocks");
        if (!haar_supported(plan->g.nx, plan->g.ny, pc->nz))
            return fail(MBIR_ERR_ARG, "Haar preconditioners need a square power-of-two image (<= 2048) or a cubic "
                                      "power-of-two volume (<= 256)");
        PSPS_TRY(pc->B.alloc((size_t)nm * nm * n));
        PSPS_TRY(pc->Babs.alloc((size_t)nm * nm * n));
        PSPS_CUDA(cudaMemcpyAsync(pc->B.p, blocks, sizeof(float) * pc->B.n, cudaMemcpyDeviceToDevice, s));
        PSPS_TRY(launch_abs_copy(blocks, pc->Babs.p, (int64_t)pc->B.n, s));
        PSPS_TRY(pc->tmp.alloc((size_t)n * nm * 2));
        DBuf<float> lmax;
        PSPS_TRY(lmax.alloc(n));
        PSPS_TRY(launch_block_lmax(nm, n, lam, lmax.p, s));
        return finish_cross_haar(pc, lam, lmax.p, s);
    }
    if (!plan || nm != 1 || !lam)
        return fail(MBIR_ERR_ARG, "psps_precondition_create: Fourier/Haar kinds need a plan, n_mat = 1 and lam");
    if (kind == PSPS_PRECOND_HAAR && !haar_supported(plan->g.nx, plan->g.ny, pc->nz))
        return fail(MBIR_ERR_ARG, "Haar preconditioner needs a square power-of-two image (<= 2048) or a cubic "
                                  "power-of-two volume (<= 256)");
    if (kind == PSPS_PRECOND_FOURIER || kind == PSPS_PRECOND_MOD_FOURIER)
        PSPS_TRY(pc->fft.init(pc->nx, pc->ny, pc->nz));
    PSPS_TRY(pc->tmp.alloc((size_t)n * 4));
    PSPS_TRY(pc->Z.alloc((size_t)n * 2));
    PSPS_TRY(pc->s.alloc(n));
    PSPS_TRY(pc->s_abs.alloc(n));
    PSPS_TRY(pc->m0.alloc(n));
    if (m0 && kind != PSPS_PRECOND_FOURIER)
        PSPS_CUDA(cudaMemcpyAsync(pc->m0.p, m0, sizeof(float) * n, cudaMemcpyDeviceToDevice, s));
    else
        PSPS_TRY(launch_fill(pc->m0.p, n, 1.f, s));
    DBuf<float> l2;
    PSPS_TRY(l2.alloc(n));
    PSPS_CUDA(cudaMemcpyAsync(l2.p, lam, sizeof(float) * n, cudaMemcpyDeviceToDevice, s));
    PSPS_TRY(finish_scalar_pub(pc, l2.p, kind != PSPS_PRECOND_HAAR, s));
    PSPS_CUDA(cudaStreamSynchronize(s));
    return MBIR_OK;
}
}  // namespace

extern "C" mbir_status psps_precondition_create(mbir_plan *plan, int kind, int n_mat, int64_t n, const float *lam,
                                                const float *m0, const float *blocks, mbir_stream stream,
                                                psps_precond **out) {
    if (!out) return fail(MBIR_ERR_ARG, "psps_precondition_create: null out");
    *out = nullptr;
    if (kind < PSPS_PRECOND_NONE || kind > PSPS_PRECOND_BLOCK_HAAR)
        return fail(MBIR_ERR_ARG, "psps_precondition_create: unknown kind %d", kind);
    if (n_mat < 1 || n_mat > 4) return fail(MBIR_ERR_ARG, "psps_precondition_create: n_mat must be 1..4");
    if (plan && n != plan->n_pix) return fail(MBIR_ERR_ARG, "psps_precondition_create: n must equal the plan's pixels");
    if (n < 1) return fail(MBIR_ERR_ARG, "psps_precondition_create: n must be >= 1");
    psps_precond *pc = new psps_precond();
    mbir_status st = create_impl(plan, kind, n_mat, n, lam, m0, blocks, (cudaStream_t)stream, pc);
    if (st != MBIR_OK) {
        delete pc;
        return st;
    }
    *out = pc;
    return MBIR_OK;
}

extern "C" mbir_status psps_precondition_destroy(psps_precond *pc) {
    delete pc;
    return MBIR_OK;
}

extern "C" mbir_status psps_precondition(psps_precond *pc, int op, const float *in, float *out, mbir_stream s) {
    if (!pc || !in || !out) return fail(MBIR_ERR_ARG, "psps_precondition: null argument");
    if (op < PSPS_APPLY_M || op > PSPS_APPLY_ABS_MT) return fail(MBIR_ERR_ARG, "psps_precondition: bad op %d", op);
    if (in == out) return fail(MBIR_ERR_ARG, "psps_precondition: in and out must not alias");
    return precond_apply(pc, op, in, out, (cudaStream_t)s);
}

extern "C" mbir_status psps_precondition_export(psps_precond *pc, int what, float *out, int64_t n_out,
                                                mbir_stream stream) {
    if (!pc || !out) return fail(MBIR_ERR_ARG, "psps_precondition_export: null argument");
    const psps::DBuf<float> *src = nullptr;
    const bool cross = pc->kind == PSPS_PRECOND_BLOCK_FOURIER || pc->kind == PSPS_PRECOND_BLOCK_HAAR;
    switch (what) {
        case PSPS_EXPORT_SCALES: src = cross ? &pc->Li : &pc->s; break;
        case PSPS_EXPORT_BLOCKS: src = &pc->B; break;
        case PSPS_EXPORT_M0: src = &pc->m0; break;
        case PSPS_EXPORT_HBLOCKS: src = &pc->Hblk; break;
        case PSPS_EXPORT_ESTIMATE: src = &pc->est; break;
        default: return fail(MBIR_ERR_ARG, "psps_precondition_export: unknown array %d", what);
    }
    if (!src->p || src->n == 0)
        return fail(MBIR_ERR_ARG, "psps_precondition_export: preconditioner kind %d has no array %d", pc->kind, what);
    // the scalar kinds' scratch may be longer than the array itself
    const bool block_shaped = what == PSPS_EXPORT_BLOCKS || what == PSPS_EXPORT_HBLOCKS ||
                              ((what == PSPS_EXPORT_SCALES || what == PSPS_EXPORT_ESTIMATE) && cross);
    const int64_t n = block_shaped ? (int64_t)pc->nm * pc->nm * pc->n : pc->n;
    if (n_out != n)
        return fail(MBIR_ERR_ARG, "psps_precondition_export: array %d holds %lld values, n_out is %lld", what,
                    (long long)n, (long long)n_out);
    PSPS_CUDA(cudaMemcpyAsync(out, src->p, sizeof(float) * n, cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
    return MBIR_OK;
}

extern "C" mbir_status psps_precondition_set_sides(psps_precond *pc, int sides) {
    if (!pc) return fail(MBIR_ERR_ARG, "psps_precondition_set_sides: null preconditioner");
    if (sides != 1 && sides != 2) return fail(MBIR_ERR_ARG, "psps_precondition_set_sides: sides must be 1 or 2");
    pc->sides = sides;
    return MBIR_OK;
}
