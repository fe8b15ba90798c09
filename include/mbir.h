/*
 * mbir.h -- C ABI of the GB300 preconditioned-SPS library (libpsps.so).
 *
 * The library evaluates one preconditioned separable-parabolic-surrogates
 * (PSPS) iteration for penalized weighted least-squares CT reconstruction
 * (MBIR), projection-domain material decomposition and one-step model-based
 * material decomposition (MBMD), following Tivnan, Wang & Stayman,
 * "A Preconditioned Algorithm for Model-Based Iterative CT Reconstruction and
 * Material Decomposition from Spectral CT Data" (arXiv 2010.01371):
 *   mean model            y_bar = B exp(-A x)                    (Sec. II-A, Eq. 1)
 *   objective             1/2 (y - y_bar)^T Sigma^-1 (y - y_bar) + 1/2 x^T R x (Eqs. 2-3)
 *   SPS update            Sec. II-B, Eqs. 4-11
 *   preconditioned SPS    x = M x', operator A -> A M            (Sec. II-C)
 *   preconditioners       Fourier / modified Fourier / Haar wavelet (Sec. II-D),
 *                         per-ray cross-material blocks (Sec. II-E),
 *                         per-pixel blocks and cross-material Fourier (Sec. II-F)
 *
 * Conventions shared by every entry point:
 *   - Every function returns an mbir_status; on failure mbir_last_error()
 *     returns a thread-local message.  Invalid arguments return
 *     MBIR_ERR_ARG before anything is launched or written.
 *   - Array pointers named x, l, y, grad, ... are DEVICE pointers owned by the
 *     caller; they must stay valid until the work queued on `stream` is
 *     done.  Calls are asynchronous on `stream` unless documented otherwise.
 *   - Images are row-major [n_mat][nz][ny][nx] (2-D: [n_mat][ny][nx]) FP32;
 *     sinograms are [n_chan or n_mat][n_views][n_v][n_u] (2-D: [..][n_views][n_u]).
 *   - Handles (mbir_plan, mbmd_spectrum, psps_precond, psps_state) are owned by
 *     the library: created by *_create, released by *_destroy.  A handle may
 *     be used from one host thread at a time.
 *   - `stream` is a cudaStream_t (NULL = the legacy default stream).
 */
#ifndef MBIR_H
#define MBIR_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *mbir_stream; /* same type as cudaStream_t */

typedef enum {
    MBIR_OK = 0,
    MBIR_ERR_ARG = -1,            /* invalid argument or shape          */
    MBIR_ERR_CUDA = -2,           /* a CUDA runtime call failed         */
    MBIR_ERR_OOM = -3,            /* device allocation failed           */
    MBIR_ERR_NONFINITE = -4,      /* a reduction produced NaN / Inf     */
    MBIR_ERR_TIMEOUT = -5,        /* a bounded device wait gave up      */
    MBIR_ERR_UNIMPLEMENTED = -6   /* option not available in this build */
} mbir_status;

enum { MBIR_PAR2D = 0, MBIR_FAN2D = 1, MBIR_CONE3D = 2 };

/* Scan geometry (lengths in mm, angles in radians).
 * Pixel (ix,iy,iz) is centred at ((ix-(nx-1)/2)dx, (iy-(ny-1)/2)dy, (iz-(nz-1)/2)dz).
 * Views: angle_v = angle0 + v * angle_span / n_views.
 *   MBIR_PAR2D : ray direction -(cos a, sin a); bin b crosses the centre line at
 *                t_b = (b-(n_u-1)/2) du along (-sin a, cos a).
 *   MBIR_FAN2D : curved detector; source at sid (cos a, sin a); fan angle
 *                g_b = (b-(n_u-1)/2) du / sdd; direction -(cos(a-g_b), sin(a-g_b)).
 *   MBIR_CONE3D: flat detector at distance sdd from the source (sid from the
 *                centre), axes e_u = (-sin a, cos a, 0), e_v = (0, 0, 1); pixel
 *                (iu,iv) at ((iu-(n_u-1)/2) du, (iv-(n_v-1)/2) dv).
 * The projector is Joseph's method: the dominant direction axis drives the
 * march, one (bi)linearly interpolated sample per driving-axis pixel, scaled by
 * the pixel size over |u_axis|.  (The paper leaves A unspecified; Sec. II-D.) */
typedef struct {
    int kind;
    int nx, ny, nz;
    double dx, dy, dz;
    int n_views;
    double angle0, angle_span;
    int n_u, n_v;
    double du, dv;
    double sid, sdd;
} mbir_geometry;

typedef struct mbir_plan mbir_plan;
typedef struct mbmd_spectrum mbmd_spectrum;
typedef struct psps_precond psps_precond;
typedef struct psps_state psps_state;

/* ---------------------------------------------------------------- projector */

/* Create a projector plan for one geometry: the system matrix A of the mean
 * model (Eq. 1; A for standard CT, Eqs. 19-20; applied per basis material in
 * one-step MBMD, Eq. 44), which the paper leaves unspecified and this library
 * realises as Joseph's method (pixel-driven interpolation along each ray).
 * Precomputes the per-ray Joseph set-up (FP64 on the device, stored FP32) and
 * owns the projector's scratch.  n_mat_max bounds the number of channels
 * later calls may pass (1..8).  MBIR_ERR_ARG for an invalid geometry,
 * MBIR_ERR_OOM if device memory runs out; *out is NULL on error. */
mbir_status mbir_plan_create(const mbir_geometry *g, int n_mat_max, mbir_plan **out);
mbir_status mbir_plan_destroy(mbir_plan *plan);
/* Number of rays (sinogram entries per channel) and pixels of a plan. */
int64_t mbir_plan_n_rays(const mbir_plan *plan);
int64_t mbir_plan_n_pix(const mbir_plan *plan);

/* l[m] = A x[m] for m < n_mat (the operator A inside the exponential,
 * Sec. II-D; for one-step MBMD, A is applied per basis material, Sec. II-F).
 * x: [n_mat][image], l: [n_mat][n_rays] (overwritten). */
mbir_status mbir_project(mbir_plan *plan, const float *x, float *l, int n_mat, mbir_stream stream);

/* x[m] (+)= A^T s[m]: the exact transpose of mbir_project (same weights).
 * accumulate = 0 overwrites x, 1 adds to it. */
mbir_status mbir_backproject(mbir_plan *plan, const float *s, float *x, int n_mat, int accumulate,
                             mbir_stream stream);

/* Select the transpose's algorithm.  2-D: 0 = tile scatter through shared
 * memory (default; lanes of a warp on consecutive driving indices of one ray),
 * 1 = pixel-driven gather (deterministic: no atomics, bitwise reproducible),
 * 2 = ray-driven scatter with global FP32 atomics.  Mode 0 accumulates in
 * fixed point: each term is rounded to a grid of M max(2^-22, T 2^-30), M
 * a bound on |weight x value| over the call and T a bound on the terms one
 * pixel receives from one CTA's views (views per CTA x the rays of one view
 * that reach one pixel: a few for detector bins no finer than the pixels,
 * more for finer bins); the sums are exact integer sums, so the result is
 * bitwise reproducible.  A non-finite input makes its channel's image NaN.
 * It needs 8 bytes x n_mat_max x n_pix of plan scratch.  3-D (cone): 0 =
 * tile scatter (default): a CTA per 8 x 8 x 16-voxel tile runs over every
 * view, stages the rays of the tile's detector box and adds each (ray, tile
 * plane) sample's bilinear terms to 32-bit fixed-point shared-memory
 * accumulators, flushed into exact 64-bit sums every vb views; each term is
 * rounded to a grid of M max(2^-22, T 2^-30), M = max |weight x value| of
 * the channel over the call, T = vb x the plan's bound on the rays of one view
 * that reach one voxel (vb chosen so that T <= 256 where that bound allows),
 * bitwise reproducible, a non-finite input makes its channel's image NaN;
 * plans whose geometry gives no such bound (a source within the volume's
 * reach) run mode 1 instead.  1 = voxel-driven gather (FP32 sums per view,
 * Kahan-compensated across views; deterministic), 2 = ray-driven scatter with
 * global FP32 atomics, 3 = the voxel gather with per-plane split tables in
 * shared memory (bitwise equal to 1).  All use the forward projector's
 * per-ray weights and are the exact transpose of mbir_project up to
 * rounding.  MBIR_ERR_ARG for another mode (3 on a 2-D plan). */
mbir_status mbir_plan_set_backprojector(mbir_plan *plan, int mode);
/* Views handled by one CTA of the tile transpose (mode 0), 1..180: the
 * grid is (image tiles) x ceil(n_views / views_per_cta) CTAs.  The plan's
 * default aims at about six CTAs per SM (4..60 views).  Only changes
 * the work split (and the fixed-point grid, through the bound on the terms
 * one accumulator receives), not the result's definition.
 * MBIR_ERR_ARG outside 1..180. */
mbir_status mbir_plan_set_tiling(mbir_plan *plan, int views_per_cta);
/* Autotuner (the paper has no counterpart; it picks work shapes, never the
 * operator): times candidates with zero data (a warm-up and up to three
 * launches each, CUDA events on `stream`) and keeps the fastest in the plan.
 * 2-D plans: the tile transpose of n_channels channels for 4/8/15/30/45/60/
 * 90/120/180 views per CTA (written to *views_per_cta if non-NULL), then the
 * forward projection of n_channels / 2 (at least 1) basis images by one
 * thread per ray and by the strip kernel with 32/64/128/256 bins (and
 * 256 / that many views) per CTA.  Cone-beam plans: the tile scatter (where
 * available; 16- and 8-voxel-deep tiles), the direct voxel gather and the
 * split-table gather, then the
 * forward's per-lane and warp-aligned marches (mbir_plan_set_projector modes
 * 1 and 2; equal results).  Synchronises; allocates and
 * frees temporary device buffers; not allowed while `stream` is capturing
 * (MBIR_ERR_ARG).  MBIR_ERR_ARG if n_channels is outside 1..n_mat_max; on
 * any error the plan keeps its previous choices. */
mbir_status mbir_plan_autotune(mbir_plan *plan, int n_channels, mbir_stream stream, int *views_per_cta);
/* Bins per CTA of the strip forward (mode 2): 32, 64, 128 or 256, with
 * 256 / bins views per CTA; MBIR_ERR_ARG otherwise.  Work split only. */
mbir_status mbir_plan_set_strip_bins(mbir_plan *plan, int bins);
/* Depth of the cone tile transpose's tiles (mode 0): 8 x 8 x 16 voxels
 * (default; 256 threads, four voxels each) or 8 x 8 x 8 (two voxels per
 * thread, five CTAs per SM).  Work split only: both give the same terms and
 * the same fixed-point grid.  MBIR_ERR_ARG for a 2-D plan or another depth. */
mbir_status mbir_plan_set_cone_tile(mbir_plan *plan, int depth);
/* The plan's current choices (any pointer may be NULL): forward algorithm
 * (mbir_plan_set_projector's modes), strip bins per CTA, transpose mode,
 * tile-transpose views per CTA (2-D) and cone tile depth (3-D). */
mbir_status mbir_plan_tuning(const mbir_plan *plan, int *fwd_mode, int *strip_bins, int *back_mode, int *back_views,
                             int *cone_tile);
/* Select the forward projector's algorithm (Eq. 1's A).  2-D: 0 = per-tile
 * partial sums through shared memory, combined with one FP32 atomic per
 * (tile, ray); 1 = one thread per ray with Kahan-compensated sums, gathering
 * from L1/L2, eight samples summed before each compensated add
 * (deterministic); 2 = rays of a block of views and bins march
 * shared-memory strips of the image, every lane on the same driving index
 * (deterministic).  Cone beam: one thread per ray; 1 (and 0) = each lane
 * marches its own range, 2 = the lanes of a warp march the same plane index
 * (same samples and sums).  All use the same per-ray Joseph weights.
 * MBIR_ERR_ARG for other modes. */
mbir_status mbir_plan_set_projector(mbir_plan *plan, int mode);

/* ------------------------------------------------------- spectral model */

/* Spectral model of Sec. II-E/F: Q[E][m] (mass attenuation of material m at
 * energy E, per unit of x), S[c][E] (channel sensitivity with the gain folded
 * in).  Standard CT (Sec. II-D) is n_mat = n_energy = n_chan = 1, Q = 1,
 * S = I0.  Host FP64 arrays, copied; limits: n_mat <= 4, n_chan <= 8,
 * n_energy <= 256. */
mbir_status mbmd_spectrum_create(int n_mat, int n_energy, int n_chan, const double *Q, const double *S,
                                 mbmd_spectrum **out);
mbir_status mbmd_spectrum_destroy(mbmd_spectrum *spec);

/* Detector blur in the outer operator B S of the forward model (Eq. 1): the
 * mean counts become y_bar[c] = B (sum_E S[c][E] exp(-[Q l]_E)) with
 * [B v]_i = sum_{k=-radius..radius} taps[k + radius] v_{i+k}, taken within
 * detector rows of `row` consecutive rays (rays past a row's ends count as
 * zero).  The SPS numerators of Eqs. 8 and 10 then use B^T of the weighted
 * residual and of w .* B 1 (Sec. II-B's rank-one bound applied to the rows of
 * B S).  The preconditioners still use blur-free Fisher blocks.
 * radius 0..3 (0 removes the blur; taps and row are then ignored); taps:
 * host FP64 [2 radius + 1], finite and >= 0, stored in FP32; row >= 1.
 * Every model call, state and batch on this spectrum then needs n_rays to be
 * a multiple of row (MBIR_ERR_ARG otherwise).  A PSPS state keeps the blur
 * the spectrum had when it was created.  Bad arguments leave the spectrum
 * unchanged and return MBIR_ERR_ARG. */
mbir_status mbmd_spectrum_set_blur(mbmd_spectrum *spec, int radius, int row, const double *taps);

/* Correlated detector noise (Sec. II-A: the data covariance is known; Eq. 3
 * weights the residual by its inverse): Sigma_y = D^1/2 C D^1/2 with
 * D = diag(max(y, 1)) and, within each detector row of `row` consecutive rays
 * and in every channel, C[j][k] = a^|j - k|.  Its inverse W couples
 * neighbouring cells (tridiagonal), so the data term, its gradient, the
 * line-search terms and the SPS numerators (Eqs. 8 and 10, with the curvature
 * from |W|: W has negative entries next to the diagonal) couple row
 * neighbours.  a = 0 restores the diagonal covariance (row ignored);
 * 0 <= a < 0.99, row >= 2, equal to the blur's row when both are set.  Model
 * calls, states and batches then need n_rays to be a multiple of row.  The
 * forward model and the preconditioner builds do not change.  A PSPS state
 * keeps the setting the spectrum had when it was created.  Bad arguments
 * leave the spectrum unchanged and return MBIR_ERR_ARG. */
mbir_status mbmd_spectrum_set_noise(mbmd_spectrum *spec, double a, int row);

/* Mean counts y_bar[c][i] = sum_E S[c][E] exp(-sum_m Q[E][m] l[m][i]) (Eq. 1),
 * followed by the spectrum's detector blur B along detector rows when one is
 * set (mbmd_spectrum_set_blur; n_rays must then be a multiple of its row).
 * l: [n_mat][n_rays], ybar: [n_chan][n_rays]. */
mbir_status mbmd_forward_model(const mbmd_spectrum *spec, const float *l, float *ybar, int64_t n_rays,
                               mbir_stream stream);

/* PWLS data term L = 1/2 sum_{c,i} w (y - y_bar)^2 with w = 1/max(y, 1)
 * (Eq. 3, Sigma_y = diag(max(y,1))), y_bar as in mbmd_forward_model.  plan != NULL: x_or_l is an image
 * [n_mat][image] and l = A x is formed internally; plan == NULL: x_or_l is
 * the line-integral array [n_mat][n_rays] (projection-domain decomposition).
 * *objective is a DEVICE double written with the FP64-reduced value. */
mbir_status mbmd_objective(mbir_plan *plan, const mbmd_spectrum *spec, const float *x_or_l, const float *y,
                           int64_t n_rays, double *objective, mbir_stream stream);

/* Gradient of the data term with respect to x (plan != NULL: the adjoint
 * A^T of the per-ray derivative, recomputing l = A x and exp(-Q l) instead of
 * storing them) or l (plan == NULL).  grad has the shape of x_or_l
 * (overwritten); objective (device, nullable) receives L.  On a cone plan
 * whose transpose is the tile scatter, every gradient channel keeps its
 * terms to 2^-12 of the fixed-point unit (the low words of
 * mbir_plan_set_backprojector's mode 0). */
mbir_status mbmd_gradient(mbir_plan *plan, const mbmd_spectrum *spec, const float *x_or_l, const float *y,
                          int64_t n_rays, float *grad, double *objective, mbir_stream stream);

/* Plain-SPS separable curvature of the data term at x (Eqs. 6 and 8-11 with
 * M = I): curv = A^T kappa with, per ray and material,
 *   kappa[m][i] = sum_E Q[E][m] gamma[E][i] c[E][i],  gamma = Q (A 1),
 * c the maximum curvature of the per-ray, per-energy surrogate built from
 * eta and rho (with the spectrum's detector blur and correlated noise, if
 * set).  plan == NULL:
 * projection domain (A = I, gamma = Q 1) and curv = kappa per ray.  The PSPS
 * iteration forms the same numerators with gamma = Q A|M|1.  curv: device,
 * [n_mat][image] (plan) or [n_mat][n_rays], overwritten.  Errors as
 * mbmd_gradient. */
mbir_status mbmd_curvature(mbir_plan *plan, const mbmd_spectrum *spec, const float *x_or_l, const float *y,
                           int64_t n_rays, float *curv, mbir_stream stream);

/* mbmd_objective for projection-domain line integrals (the plan == NULL
 * case) that allocates no device memory.  The paper has no counterpart; this
 * entry point exists for callers that cannot allocate device memory: code
 * inside a host framework whose device memory belongs to another allocator,
 * deployments held to a fixed memory budget, and loops that must not call
 * cudaMalloc / cudaFree (they can block or synchronise the device).
 * Arguments: Q[n_energy][n_mat] and S[n_chan][n_energy] are HOST FP64 arrays
 * (as for mbmd_spectrum_create), l [n_mat][n_rays] and y [n_chan][n_rays] are
 * device arrays, *objective is a device double that receives
 * L = 1/2 sum w (y - y_bar)^2 (overwritten, not accumulated).
 * Scratch: a static 28,928-byte device array per GPU, held until the process
 * exits; limits n_mat <= 4, n_energy <= 256, n_chan <= 8 (larger sizes return
 * MBIR_ERR_ARG with a message); n_rays is not limited.  The first call on
 * each device looks up the array's address.  The call cannot be captured into
 * a CUDA graph (it stages the spectral table with a pageable host copy): on a
 * stream that is capturing it returns MBIR_ERR_ARG and enqueues nothing.
 * Every call shares the array: calls that overlap on the GPU race and must be
 * ordered by the caller (one stream, or events). */
mbir_status mbmd_objective_noalloc(int n_mat, int n_energy, int n_chan, const double *Q, const double *S,
                                   const float *l, const float *y, int64_t n_rays, double *objective,
                                   mbir_stream stream);

/* ----------------------------------------------------- preconditioners */

enum {
    PSPS_PRECOND_NONE = 0,          /* M = I: plain SPS (Sec. II-B)                   */
    PSPS_PRECOND_FOURIER = 1,       /* M = U^H Lambda^-1/2 U (Eq. 29)                 */
    PSPS_PRECOND_MOD_FOURIER = 2,   /* M = M0 U^H Lambda^-1/2 U M0 (Eqs. 30-33)       */
    PSPS_PRECOND_HAAR = 3,          /* M = M0 U_DWT^T Lambda^-1/2 U_DWT M0 (Eq. 34)   */
    PSPS_PRECOND_BLOCK = 4,         /* per-pixel / per-ray N_k x N_k M0 (Eqs. 42, 54) */
    PSPS_PRECOND_BLOCK_FOURIER = 5, /* cross-material Fourier (Eqs. 56-57)            */
    PSPS_PRECOND_BLOCK_HAAR = 6     /* cross-material wavelet (Eqs. 58-61)            */
};
enum { PSPS_APPLY_M = 0, PSPS_APPLY_MT = 1, PSPS_APPLY_ABS_M = 2, PSPS_APPLY_ABS_MT = 3 };

/* Build a preconditioner once, before iterating (Sec. II-C): the Hessian at
 * the solution is approximated with D from the data (standard CT: y / I0;
 * spectral: a per-ray water-only fit), M0 from (F+R)1_k, and the eigenvalues
 * from Eq. 18 taken in modulus (the phase-corrected ratio is complex for a
 * shift-variant Hessian), clamped to >= 1e-6 of the largest.  Haar
 * eigenvalues use Eq. 18 with one test function per (level, subband, class of
 * a P x P position lattice); the cross-material wavelet blocks (Eqs. 59-60)
 * use the same test functions once per material.  Cross-material blocks are
 * not symmetric: K^-1/2 and L^-1/2 are taken of their polar factors
 * (K^T K)^1/2, Re (L^H L)^1/2, with the eigenvalue floor 1e-6 of the largest
 * over all blocks.  HAAR and BLOCK_HAAR need a square power-of-two image;
 * FOURIER kinds need sides 2^a 3^b 5^c 7^d <= 1024; 3-D volumes take BLOCK
 * only (MBIR_ERR_UNIMPLEMENTED otherwise).
 * y: device [n_chan][n_rays]; beta: host [n_mat][n_mat] penalty strengths
 * (NULL = no penalty); haar_lattice: lattice size P of the Haar test
 * functions (0 = the paper's single U^T 1; 3 is the default); plan == NULL
 * selects projection-domain decomposition (only NONE and BLOCK).
 * Synchronises `stream`. */
mbir_status psps_precondition_build(mbir_plan *plan, const mbmd_spectrum *spec, int kind, const float *y,
                                    int64_t n_rays, const double *beta, int haar_lattice, mbir_stream stream,
                                    psps_precond **out);
/* Create a preconditioner from precomputed data instead of building it (to
 * reuse one across reconstructions, or to load one):
 *   FOURIER / MOD_FOURIER / HAAR (n_mat = 1, plan required): lam = the
 *     eigenvalue estimates (device, n values: the [ny][nx] DFT spectrum, or the
 *     Haar coefficients in the Mallat layout); m0 = the diagonal
 *     zero-frequency normalisation (device, n values; NULL = 1; ignored for
 *     FOURIER).  lam is taken in modulus, clamped to >= 1e-6 of its largest
 *     and raised to -1/2 exactly as psps_precondition_build does.
 *   BLOCK: blocks = the M0 blocks themselves (device [n_mat][n_mat][n]).
 *   BLOCK_FOURIER / BLOCK_HAAR (plan required): blocks = M0 as for BLOCK;
 *     lam = the symmetric polar factors of the cross-material blocks, one
 *     [n_mat][n_mat] block per DFT frequency ([ny][nx]) / Haar coefficient
 *     (Mallat layout), device [n_mat][n_mat][n]; inverted with the same
 *     global floor as the build.
 * n = pixels per material (plan) or rays (plan == NULL, BLOCK only).
 * Synchronises `stream`. */
mbir_status psps_precondition_create(mbir_plan *plan, int kind, int n_mat, int64_t n, const float *lam,
                                     const float *m0, const float *blocks, mbir_stream stream, psps_precond **out);
mbir_status psps_precondition_destroy(psps_precond *pc);

/* Where M0 enters the Fourier and wavelet kinds (MOD_FOURIER, HAAR,
 * BLOCK_FOURIER, BLOCK_HAAR; FOURIER and BLOCK are unaffected).  The paper
 * writes M = M0^T C M0 (Eqs. 33, 34, 57, 61) with C = U^H Lambda~^-1/2 U built
 * from the spectrum of N = M0^T H M0; then M^T H M = M0^T M0 where N is
 * diagonal in U, not the I that Sec. II-C aims for.  With one material that
 * remainder is diagonal and the separable curvature absorbs it: MOD_FOURIER
 * and HAAR default to the literal form (sides = 2).  With per-pixel blocks it
 * couples the materials of a pixel, which a separable surrogate cannot
 * absorb: BLOCK_FOURIER and BLOCK_HAAR default to the one-sided M = M0^T C
 * (sides = 1), for which M^T H M = C N C = I there.  This call overrides the
 * default.  Call it before psps_state_create: a state precomputes A|M|1 and
 * |M|^T|R||M|1 from the preconditioner it is given.  sides other than 1 or 2
 * return MBIR_ERR_ARG. */
mbir_status psps_precondition_set_sides(psps_precond *pc, int sides);

/* Copy one array of a preconditioner into caller-owned device memory (for
 * checking a build against an independent one element by element; the
 * arrays are those of psps_precondition_create):
 *   PSPS_EXPORT_SCALES  FOURIER / MOD_FOURIER / HAAR: the scales
 *                       clamp(Lambda~)^-1/2 of Eqs. 29, 33, 34, [n];
 *                       BLOCK_FOURIER / BLOCK_HAAR: the per-frequency /
 *                       per-coefficient blocks L^-1/2, K^-1/2 of Eqs. 57, 61,
 *                       [n_mat][n_mat][n];
 *   PSPS_EXPORT_BLOCKS  the M0 blocks of Eqs. 30, 42, 53-54, [n_mat][n_mat][n]
 *                       (built kinds other than FOURIER);
 *   PSPS_EXPORT_M0      the scalar M0 of the one-material kinds, [n] (ones
 *                       for FOURIER);
 *   PSPS_EXPORT_HBLOCKS built only: the blocks (F+R)1_k that M0 is the
 *                       inverse square root of, [n_mat][n_mat][n];
 *   PSPS_EXPORT_ESTIMATE built Fourier / wavelet kinds only: the Eq. 18
 *                       estimates before the modulus, floor and -1/2 power:
 *                       Lambda~ [n] (FOURIER, MOD_FOURIER: already the
 *                       modulus; HAAR: signed ratios), the polar factors
 *                       Re (L^H L)^1/2 (BLOCK_FOURIER) or the estimated blocks
 *                       K (BLOCK_HAAR), [n_mat][n_mat][n].
 * n_out must equal the array's length; a kind without the array returns
 * MBIR_ERR_ARG.  Asynchronous on `stream`. */
enum { PSPS_EXPORT_SCALES = 0, PSPS_EXPORT_BLOCKS = 1, PSPS_EXPORT_M0 = 2, PSPS_EXPORT_HBLOCKS = 3,
       PSPS_EXPORT_ESTIMATE = 4 };
mbir_status psps_precondition_export(psps_precond *pc, int what, float *out, int64_t n_out, mbir_stream stream);

/* out = op(M) in for op in PSPS_APPLY_*: the change of variables x = M x'
 * of Sec. II-C (Eq. 15) with the preconditioner's M (Eqs. 29, 33, 34, 42, 57,
 * 61), its transpose (the preconditioned gradient M^T grad, Eq. 5 for A M),
 * and the elementwise bounds |M|, |M|^T that the separable curvature of the
 * preconditioned problem uses (Eqs. 6 and 8 with A M).  Arrays device,
 * caller-owned, shaped like the unknowns ([n_mat][image] or
 * [n_mat][n_rays]); in and out must not alias (MBIR_ERR_ARG).  Asynchronous
 * on `stream`. */
mbir_status psps_precondition(psps_precond *pc, int op, const float *in, float *out, mbir_stream stream);

/* ------------------------------------------------------------ iteration */

enum {
    PSPS_FLAG_LINESEARCH = 1, /* safeguarded Newton line search on phi(alpha)  */
    PSPS_FLAG_NONNEG = 2,     /* clamp x >= 0 after each step (plain SPS only) */
    PSPS_FLAG_GRAPH = 4       /* replay each iteration as a captured CUDA graph */
};

/* Create an iteration state for the PWLS estimate of Eqs. 2-3 (penalty
 * Eqs. 26, 49-52) solved by SPS on x' with x = M x' (Sec. II-B, Eqs. 4-7, on
 * the preconditioned model of Eq. 15): copies y (device [n_chan][n_rays]),
 * beta (host [n_mat][n_mat], NULL = 0) and x0 (device image, NULL = 0);
 * pc == NULL runs plain SPS.  The state keeps x, l = A x (updated
 * incrementally, recomputed exactly every `reproject_every` iterations), the
 * precomputed gamma~ = A|M|1 (gamma of Eq. 9 for A M) and |M|^T|R||M|1, and
 * the objective history on the device.  The library owns the state (free it
 * with psps_state_destroy); the plan, spectrum and preconditioner must
 * outlive it.  MBIR_ERR_ARG on size or argument mismatches, MBIR_ERR_OOM if
 * device memory runs out.  Synchronises `stream`. */
mbir_status psps_state_create(mbir_plan *plan, const mbmd_spectrum *spec, psps_precond *pc, const float *y,
                              int64_t n_rays, const double *beta, const float *x0, int flags,
                              int reproject_every, mbir_stream stream, psps_state **out);
mbir_status psps_state_destroy(psps_state *st);

/* Run n_iter iterations on `stream` (asynchronous): per iteration the SPS
 * numerators (Eqs. 8-11), the preconditioned gradient and separable curvature
 * (Eqs. 5-6 for A M), the direction p' = -grad'/d' of the surrogate's
 * minimiser (Eq. 7), p = M p', the line search along p (with
 * PSPS_FLAG_LINESEARCH) and the update x += alpha p.  If objective_history
 * (HOST, length n_iter + 1) is non-NULL the call synchronises and writes
 * Phi before each iteration and after the last one (after an exact
 * re-projection).  On a cone plan whose transpose is the tile scatter, the
 * cross-material Fourier and wavelet preconditioners (which difference the
 * materials' gradient numerators after a spatial filter) get the gradient
 * channels to 2^-12 of the fixed-point unit (low words), the other kinds
 * the unit M 2^-22 of mbir_plan_set_backprojector's mode 0.  Returns
 * MBIR_ERR_NONFINITE if a reduction went non-finite, MBIR_ERR_ARG for
 * n_iter < 0. */
mbir_status psps_step(psps_state *st, int n_iter, double *objective_history, mbir_stream stream);

/* Replace the measured counts y of the state (n = n_chan * n_rays values,
 * [n_chan][n_rays]; HOST or device pointer: the copy direction follows the
 * pointer, pinned host memory keeps it asynchronous on `stream`).  The next
 * iterations fit the new data; the preconditioner, x, l and the line-search
 * state are kept (Eq. 3 with the new y).  MBIR_ERR_ARG if n does not match. */
mbir_status psps_state_set_data(psps_state *st, const float *y, int64_t n, mbir_stream stream);

/* Copy the current image x = M x' (Eq. 15: the estimate of Eq. 2 in the
 * original variables; device, caller-owned, [n_mat][image] or
 * [n_mat][n_rays], asynchronous on `stream`) / step lengths (host, the last n
 * alphas of the most recent psps_step call; synchronises).  MBIR_ERR_ARG for
 * NULL pointers or n outside the recorded range. */
mbir_status psps_get_image(psps_state *st, float *x, mbir_stream stream);
mbir_status psps_get_alphas(psps_state *st, double *alphas, int n, mbir_stream stream);

/* Batches: independent reconstructions (e.g. the slices of a volume, each
 * with its own plan, spectrum handle, preconditioner and state) advanced
 * together.  One CUDA graph per iteration holds every state's iteration as a
 * parallel branch, so the slices' kernels overlap on the GPU and the batch
 * costs one graph launch per iteration.  The paper has no counterpart: this
 * is the batched execution of its per-slice iteration (Eqs. 5-7 with the
 * preconditioned direction of Eq. 15).
 *
 * psps_batch_create keeps the n state pointers (the caller keeps ownership and
 * must keep them alive); MBIR_ERR_ARG if a state is NULL or repeated, if two
 * states share a plan or a preconditioner (their scratch buffers would race
 * in concurrent branches), or if their reproject_every differ.
 * psps_batch_step runs n_iter iterations of every state on `stream`; with
 * objective_history (HOST, n * (n_iter + 1) doubles, row i = state i, as
 * psps_step) it synchronises and returns MBIR_ERR_NONFINITE if a state went
 * non-finite.  Not thread-safe per batch; a state in a batch must not be
 * stepped on its own concurrently. */
typedef struct psps_batch psps_batch;
mbir_status psps_batch_create(psps_state *const *states, int n, psps_batch **out);
mbir_status psps_batch_destroy(psps_batch *batch);
mbir_status psps_batch_step(psps_batch *batch, int n_iter, double *objective_history, mbir_stream stream);
/* Kernels launched by psps_batch_step so far (graph kernel nodes x replays). */
mbir_status psps_batch_launch_count(psps_batch *batch, int64_t *count);

/* Stage timers.  psps_profile(st, 1) resets and enables CUDA-event timers
 * around the contiguous stages of an iteration (indices below); after every
 * psps_step call the stages of its LAST iteration are synchronised and added
 * to the totals that psps_profile_read returns (ms[k] summed milliseconds,
 * count[k] number of timed stage runs).  Enabling or disabling re-captures the
 * iteration graph. */
enum {
    PSPS_PROF_REPROJECT = 0,   /* exact re-projection l = A x            */
    PSPS_PROF_MODEL = 1,       /* per-ray gradient/curvature numerators  */
    PSPS_PROF_BACKPROJECT = 2, /* A^T of both numerators (2 n_mat ch.)   */
    PSPS_PROF_PRECOND = 3,     /* penalty, M^T, |M|^T, direction, M      */
    PSPS_PROF_PROJECT = 4,     /* q = A p                                */
    PSPS_PROF_LINESEARCH = 5,  /* phi(alpha) evaluations and control    */
    PSPS_PROF_UPDATE = 6,      /* x += alpha p, l += alpha q             */
    PSPS_PROF_STAGES = 7
};
mbir_status psps_profile(psps_state *st, int enable);
mbir_status psps_profile_read(psps_state *st, double *ms, int64_t *count);
/* Number of this library's kernels launched so far by graph replays of the
 * iteration (PSPS_FLAG_GRAPH), counted from the captured graphs' kernel nodes. */
mbir_status psps_launch_count(psps_state *st, int64_t *count);

/* Thread-local description of the last error (never NULL). */
const char *mbir_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* MBIR_H */
