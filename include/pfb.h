/*
 * libpfb: GB300 (sm_103a) implementation of the pfb-clean hot path
 * (Bester, Repetti, Perkins, Smirnov & Kenyon, "A practical preconditioner for
 * wide-field continuum imaging of radio interferometric data").
 *
 * The library evaluates the wide-field measurement operator R of Section 2
 * (Eq. 1), its weighted adjoint R^dagger Sigma^-1 (Eq. 3), the dirty image,
 * the PSF, the exact Hessian-vector product R^dagger Sigma^-1 R x (Eq. 3), the
 * PSF convolution I^psf * x (Eq. 4) and one preconditioned forward-backward
 * step (Eqs. 6-8 with the regulariser of Eq. 9).
 *
 * Conventions shared by every entry point
 * ----------------------------------------
 *  - Array arguments are DEVICE pointers to contiguous row-major memory owned by
 *    the caller (for example torch tensors on the context's device), unless an
 *    argument is marked "host".  The library never frees caller memory.
 *  - uvw     [nrow][3]  float64, metres (rows as in a Measurement Set).
 *  - freq    [nchan]    float64, Hz.
 *  - band_of_chan [nchan] int32 in [0, nband): imaging band of each channel
 *    (Section 2: n_b bands with n_b << n_nu channels).
 *  - vis     [nrow][nchan] complex, interleaved (re, im): complex64 for PFB_F32,
 *    complex128 for PFB_F64.
 *  - wgt     [nrow][nchan] real >= 0 (float32 for PFB_F32, float64 for PFB_F64),
 *    the diagonal of Sigma^-1; NULL means all ones.
 *  - image   [nband][nx][ny] real (float32 / float64).  Pixel (i, j) sits at
 *    l = l0 + (i - nx/2) dl, m = m0 + (j - ny/2) dm; n = sqrt(1 - l^2 - m^2).  The
 *    first image axis pairs with u, the second with v.  (l0, m0) = (0, 0) centres the
 *    image on the phase centre; otherwise the image is a facet of a wider field (the
 *    paper's route to cheaper wide-field operators): R of an image is the sum of R
 *    over facets that tile it, and R^dagger of a facet is the image's R^dagger on the
 *    facet's pixels.  A facet's w-stack spans only the facet (the part of n - 1 that is
 *    linear across it is applied as a shift of u and v by w dn/dl, w dn/dm at the
 *    facet centre), and its PSF (pfb_psf) is the PSF at the facet centre.
 *  - R x [d, nu] = sum_{i,j} x[b(nu),i,j] / n_ij exp(-2 pi i (u l_i + v m_j + w (n_ij - 1)))
 *    with (u, v, w) = uvw_d f_nu / c.  R^dagger is the transpose under the real
 *    inner products Re sum conj(a) b (visibilities) and sum x z (images).
 *  - Work is enqueued on `stream` (a cudaStream_t passed as void*; NULL is the
 *    legacy default stream).  Outputs are valid once the stream has completed
 *    the work, except where an entry point writes a host output: those return
 *    after synchronising the stream.
 *  - The first call for a new (geometry, precision, uvw/freq/band pointers,
 *    nrow, nchan) builds a plan (a device sort of the visibilities into uv tiles
 *    and w-planes, pixel correction tables): it reads freq and band_of_chan back
 *    to the host and synchronises the stream once.  The plan is cached in the
 *    context and reused while those pointers and sizes stay the same.  If the
 *    CONTENTS of uvw, freq or band_of_chan change under the same pointers, call
 *    pfb_plan_reset() first.
 *  - Return value: PFB_OK, or a negative PFB_ERR_* code; on error the outputs
 *    are unspecified and pfb_last_error() describes the failure.
 *  - A context is not thread-safe: use one context per host thread.
 *  - Accuracy: epsilon is the requested relative L2 error of R x and R^dagger y
 *    against the exact FP64 direct sum.  PFB_F32 keeps uvw x frequency -> grid
 *    coordinates and the w-plane phases in FP64 and everything else in FP32; it
 *    accepts epsilon >= 1e-6.  PFB_F64 computes in FP64 and accepts
 *    epsilon >= 1e-12.
 */
#ifndef PFB_H
#define PFB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pfb_ctx pfb_ctx;

typedef enum { PFB_F32 = 0, PFB_F64 = 1 } pfb_prec;

enum {
    PFB_OK = 0,
    PFB_ERR_ARG = -1,             /* invalid argument (null pointer, size, geometry, band id) */
    PFB_ERR_OOM = -2,             /* device memory (or the context's HBM budget) exhausted */
    PFB_ERR_CUDA = -3,            /* a CUDA runtime or cuFFT call failed */
    PFB_ERR_EPS = -4,             /* epsilon outside what the precision can reach */
    PFB_ERR_TIMEOUT = -5,         /* a bounded wait expired */
    PFB_ERR_NOT_IMPLEMENTED = -6
};

/* pfb_geom.flags (test switches; production calls pass 0) */
#define PFB_NO_DIVIDE_BY_N 1u     /* drop the 1/n factor of Eq. 1 */
#define PFB_NO_WTERM 2u           /* drop the w (n - 1) term (coplanar 2-D NUFFT) */
/* Memory/speed trade-off, no effect on the result beyond rounding: by default an
   FP32 plan whose budget has room also keeps 24 bytes of precomputed geometry per
   gridding item (first-tap cell, plane, flip, tap offsets, phase rotor), which the
   gridding and degridding kernels stream instead of recomputing it from uvw.  With
   this flag the plan never keeps them. */
#define PFB_NO_ITEM_RECORDS 4u
/* pfb_degrid adds R x into vis_out instead of overwriting it (vis_out += R x), so that
   R of a faceted image is the sum of the facets' calls.  Other entry points ignore it. */
#define PFB_ACCUMULATE 8u
/* Speed switch, no effect on the result beyond rounding: FP32 plans whose w-planes are
   powers of two of 1024..8192 cells per side transform only the image region and the
   32 x 32 uv tiles that some visibility touches, with the pre- and post-pass folded
   into the column transforms.  With this flag they take the full-plane transforms. */
#define PFB_NO_PRUNED_FFT 16u

typedef struct {
    int32_t nx, ny;      /* image pixels per band (even); the PSF is 2nx x 2ny */
    double dl, dm;       /* pixel size, radians */
    double fov_l, fov_m; /* field of view in radians: 0 = derive, else must equal nx*dl, ny*dm */
    double epsilon;      /* requested relative L2 accuracy of R and R^dagger */
    int32_t nband;       /* n_b imaging bands */
    uint32_t flags;      /* PFB_NO_DIVIDE_BY_N | PFB_NO_WTERM | PFB_NO_ITEM_RECORDS | PFB_ACCUMULATE |
                            PFB_NO_PRUNED_FFT */
    double l0, m0;       /* direction cosines of the image centre (facets); 0, 0 = the phase centre */
} pfb_geom;

/* Parameters of one pfb-clean step (Eqs. 6-9). */
typedef struct {
    double gamma;        /* step size (Eq. 6); the preconditioning allows gamma close to 1 */
    double sigma;        /* sigma > 0 of U = I^psf* + sigma Id (Eq. 8), in PSF-peak units */
    double lambda;       /* weight of the l2,1 term of Eq. 9 */
    double cg_tol;       /* CG stops when ||r|| <= cg_tol ||IR|| (0: run cg_iters) */
    double pd_tol;       /* reserved: the primal-dual solver runs pd_iters iterations */
    int32_t cg_iters;    /* conjugate-gradient iterations for U delta = IR */
    int32_t pd_iters;    /* Condat-Vu primal-dual iterations for Eq. 7 */
    int32_t nlevel;      /* wavelet decomposition levels (wavelet bases) */
    uint32_t basis_mask; /* bit 0 Dirac; bits 1..6 Daubechies db1..db6 (Eq. 9's dictionary) */
    double unorm;        /* ||U|| for the primal step; <= 0: max |PSF spectrum| + sigma */
    uint32_t flags;      /* PFB_STEP_* bits; 0 = the exact-gradient step */
} pfb_params;

/* pfb_params.flags */
/* Approximate gradient (Eq. 4): the step takes IR = I^d - I^psf * x_k, the PSF
   convolution standing in for the Hessian, instead of the exact IR = I^d - H x_k
   (Eq. 3).  No visibility is touched: the step costs only image-sized FFTs.  The
   paper notes that this gradient is inexact for wide fields (the w term breaks the
   convolution structure); it is offered as the cheap inner gradient of a major /
   minor cycle scheme, not as a replacement for the exact step. */
#define PFB_STEP_APPROX_GRADIENT 1u
/* pfb_clean only: before the steps, estimate L_U = lambda_max(U^-1 H) with
   pfb_step_bound (PFB_SAFE_GAMMA_ITERS power iterations, cg_iters CG iterations
   each, from the image 0.5 + u_e, u_e the SplitMix64 uniform of the flat pixel index
   e + 1 (Steele, Lea & Flood 2014): a generic positive start, since a constant one
   can miss the modes where H exceeds U most) and take gamma = min(gamma, 1.9 / L_U).
   Forward-backward in the metric U (Eqs. 6-7) converges for gamma < 2 / L_U; on wide
   fields the PSF-based U can fall short of the Hessian by more than a factor 2 in
   some directions, so a fixed gamma = 1 may diverge.  The estimate costs
   PFB_SAFE_GAMMA_ITERS Hessian applications, counted in n_hessian_out. */
#define PFB_STEP_SAFE_GAMMA 2u
#define PFB_SAFE_GAMMA_ITERS 30

/* Create a context on CUDA device `device`.  hbm_budget_bytes bounds the scratch
 * (w-plane stacks, sort tables); 0 means 85% of the device memory free at creation.
 * Returns PFB_OK and *ctx, or an error (then *ctx is NULL). */
int pfb_create(pfb_ctx **ctx, int device, size_t hbm_budget_bytes);

/* Free every device buffer the context owns.  The buffers are released in stream
 * order after the work of the context's last call; the function does not wait for
 * the device, and work of other contexts or streams is not held up. */
void pfb_destroy(pfb_ctx *ctx);

/* Message of the last failure on this context ("" if none).  The pointer stays
 * valid until the next call on the context.  With ctx == NULL: the last failure
 * of a context-free call (pfb_wsum_static) on the calling thread. */
const char *pfb_last_error(const pfb_ctx *ctx);

/* Drop cached plans, PSF spectra and scratch buffers (w-plane blocks and the
 * like), returning their memory to the context's budget; the next call rebuilds
 * what it needs.  Call it after changing uvw/freq/band or PSF contents in place,
 * or between the phases of a solve that use different geometries (the PSF's 2x
 * field, then the image).  The buffers are released in stream order after the
 * work of the context's last call (the context allocates from a memory pool of its
 * own, on the stream of each call), so the function neither waits for the device
 * nor holds up work on other streams.  Calls of one context are expected in the
 * order of one stream (or ordered by the caller), as before. */
int pfb_plan_reset(pfb_ctx *ctx);

/* R, degridding (Section 2, Eq. 1): image [nband][nx][ny] -> vis_out [nrow][nchan].
 * w-stacking with an exponential-of-semicircle kernel; accuracy epsilon. */
int pfb_degrid(pfb_ctx *ctx, const pfb_geom *geom, pfb_prec prec, int64_t nrow, int32_t nchan,
               const double *uvw, const double *freq, const int32_t *band_of_chan,
               const void *image, void *vis_out, void *stream);

/* R^dagger Sigma^-1, gridding (Eq. 3): image_out = R^dagger (wgt . vis).
 * image_out [nband][nx][ny] is overwritten. */
int pfb_grid(pfb_ctx *ctx, const pfb_geom *geom, pfb_prec prec, int64_t nrow, int32_t nchan,
             const double *uvw, const double *freq, const int32_t *band_of_chan,
             const void *vis, const void *wgt, void *image_out, void *stream);

/* Dirty image I^d = R^dagger Sigma^-1 V (Eq. 3) into image_out, and if wsum_out
 * (host, [nband]) is not NULL the per-band weight sums (then the call returns
 * after synchronising the stream). */
int pfb_dirty(pfb_ctx *ctx, const pfb_geom *geom, pfb_prec prec, int64_t nrow, int32_t nchan,
              const double *uvw, const double *freq, const int32_t *band_of_chan,
              const void *vis, const void *wgt, void *image_out, double *wsum_out, void *stream);

/* PSF I^psf (Eqs. 4 and 8): R'^dagger (wgt . 1) where R' is the operator on a
 * 2nx x 2ny grid with the same pixel size; psf_out [nband][2nx][2ny], centre
 * pixel (nx, ny), unnormalised (its centre value is the band's weight sum).
 * wsum_out as in pfb_dirty. */
int pfb_psf(pfb_ctx *ctx, const pfb_geom *geom, pfb_prec prec, int64_t nrow, int32_t nchan,
            const double *uvw, const double *freq, const int32_t *band_of_chan,
            const void *wgt, void *psf_out, double *wsum_out, void *stream);

/* Exact Hessian-vector product (Eq. 3): y_out = R^dagger Sigma^-1 R x, both [nband][nx][ny].  Arguments,
 * layouts and errors as pfb_degrid and pfb_grid (wgt may be NULL: unit weights).  The intermediate R x lives in
 * the context's scratch ([nrow][nchan] complex values); on FP32 plans with tile kernels it stays in the plan's
 * item order between R and R^dagger Sigma^-1, so the result equals pfb_grid(pfb_degrid(x)) up to rounding. */
int pfb_hessian(pfb_ctx *ctx, const pfb_geom *geom, pfb_prec prec, int64_t nrow, int32_t nchan,
                const double *uvw, const double *freq, const int32_t *band_of_chan,
                const void *wgt, const void *x, void *y_out, void *stream);

/* The Hessian of pfb_hessian (Eq. 3) from HOST buffers: uvw, freq, band_of_chan, wgt (may be NULL:
 * unit weights) and x are read from host memory, y_out is written to host memory; layouts as in
 * pfb_hessian.  uvw, freq, band_of_chan and x go in on `stream` before the computation; wgt goes in on an
 * internal copy stream, issued before R x (only R^dagger Sigma^-1 reads it, and waits for it); each band
 * of y_out comes back on the copy stream as soon as it is gridded.  With page-locked (pinned) host memory
 * the copies are asynchronous and may overlap the computation; pageable memory works but loses that.
 * The call enqueues work on `stream` (the copy stream is joined back to it); y_out holds the
 * result once `stream` has been synchronised, and the host buffers must stay valid until then.  The
 * device copies live in the context's scratch and the plan is built on them; it is reused while the
 * host pointers of uvw, freq and band_of_chan (and nrow, nchan) stay the same, so call
 * pfb_plan_reset() when their contents change under the same pointers.  Errors as pfb_hessian. */
int pfb_hessian_host(pfb_ctx *ctx, const pfb_geom *geom, pfb_prec prec, int64_t nrow, int32_t nchan,
                     const double *uvw, const double *freq, const int32_t *band_of_chan,
                     const void *wgt, const void *x, void *y_out, void *stream);

/* PSF convolution (Eq. 4): y_out[b,i,j] = sum_{i',j'} psf[b, i-i'+nx, j-j'+ny] x[b,i',j']
 * (linear convolution, psf [nband][2nx][2ny] as written by pfb_psf).  Uses the
 * geometry's nx, ny, nband only.  The PSF spectrum is cached per psf pointer. */
int pfb_psf_conv(pfb_ctx *ctx, const pfb_geom *geom, pfb_prec prec, const void *psf,
                 const void *x, void *y_out, void *stream);

/* One preconditioned forward-backward step (Eqs. 6-7):
 *   wbar = mean_b wsum[b]; I^d, I^psf and the Hessian are divided by wbar;
 *   IR = I^d - H x_k (one exact Hessian application, Eq. 3);
 *   delta = CG solve of U delta = IR per band, U = I^psf_sym * + sigma Id (Eq. 8),
 *           I^psf_sym the PSF symmetrised about its centre (the symmetric part of
 *           the PSF convolution; identical to it when w = 0);
 *   x_{k+1/2} = x_k + gamma delta (Eq. 6);
 *   x_{k+1} = prox^U_{gamma r}(x_{k+1/2}) by Condat-Vu primal-dual iterations with
 *             r(x) = lambda ||Psi^dagger x||_{2,1} + iota_+(x) (Eqs. 7 and 9).
 * dirty [nband][nx][ny] and psf [nband][2nx][2ny] as written by pfb_dirty / pfb_psf;
 * wsum (host, [nband]) the weight sums they returned; x_inout [nband][nx][ny];
 * dual_inout [nbasis][nband][nx][ny] (nbasis = bits set in basis_mask), zero on
 * the first step.  n_hessian_out (host, may be NULL) receives 1 (0 with
 * PFB_STEP_APPROX_GRADIENT, where IR = I^d - I^psf * x_k and the objective's data
 * term uses I^psf * x_k in place of H x_k); stats_out (host,
 * [3], may be NULL) receives [objective at x_k without the data constant,
 * ||x_{k+1} - x_k|| / ||x_{k+1}||, largest CG relative residual]; when stats_out
 * is given the call returns after synchronising the stream, otherwise it only
 * enqueues work. */
int pfb_step(pfb_ctx *ctx, const pfb_geom *geom, pfb_prec prec, const pfb_params *params,
             int64_t nrow, int32_t nchan, const double *uvw, const double *freq,
             const int32_t *band_of_chan, const void *wgt, const void *dirty, const void *psf,
             const double *wsum, void *x_inout, void *dual_inout, int64_t *n_hessian_out,
             double *stats_out, void *stream);

/* A whole pfb-clean solve from the data (Section 3: the PSF and dirty image, then
 * preconditioned forward-backward steps until the iterates settle):
 *   1. psf_out = I^psf on the 2nx x 2ny grid and wsum_out (host, [nband]) the
 *      per-band weight sums, exactly as pfb_psf writes them;
 *   2. the context's plans and scratch buffers are dropped (as pfb_plan_reset:
 *      the PSF's 2x-field plan is not reused), then dirty_out = I^d as pfb_dirty;
 *   3. up to max_outer calls of the step of pfb_step on x_inout / dual_inout (their
 *      contents on entry are the starting point: zeros for a cold start), stopping
 *      after the first step whose relative update ||x_{k+1} - x_k|| / ||x_{k+1}||
 *      is <= tol (tol <= 0: always max_outer steps).
 * params as for pfb_step (PFB_STEP_APPROX_GRADIENT makes every step use Eq. 4).
 * n_outer_out (host) receives the steps taken; n_hessian_out (host) the count of
 * full R^dagger Sigma^-1 R applications: one per exact-gradient step plus one for
 * the dirty image and the PSF together (each is one half: a gridding pass without
 * the degridding).  history_out (host, [max_outer][3], may be NULL) receives each
 * step's stats as pfb_step's stats_out.  Synchronises the stream after every step
 * (the stopping test reads the update on the host).
 * Arrays: vis, wgt as pfb_dirty; dirty_out [nband][nx][ny]; psf_out
 * [nband][2nx][2ny]; x_inout [nband][nx][ny]; dual_inout [nbasis][nband][nx][ny]. */
int pfb_clean(pfb_ctx *ctx, const pfb_geom *geom, pfb_prec prec, const pfb_params *params, int32_t max_outer,
              double tol, int64_t nrow, int32_t nchan, const double *uvw, const double *freq,
              const int32_t *band_of_chan, const void *vis, const void *wgt, void *dirty_out, void *psf_out,
              double *wsum_out, void *x_inout, void *dual_inout, int32_t *n_outer_out, int64_t *n_hessian_out,
              double *history_out, void *stream);

/* Step-size bound of the preconditioned forward-backward step (Eqs. 6-8):
 * *lmax_out = an estimate of L_U = lambda_max(U^-1 H) in the step's normalised units
 * (H and I^psf divided by wbar = mean_b wsum[b]; U = I^psf_sym * + sigma Id with
 * params->sigma), by `iters` power iterations: rho_k = z^T H z / z^T U z, then
 * z <- U^-1 H z (params->cg_iters CG iterations per band) normalised; the largest rho_k
 * is returned (each is a lower bound of L_U).  The step converges for gamma < 2 / L_U.
 * Data as pfb_hessian; psf [nband][2nx][2ny] (device), wsum [nband] (host), z0
 * [nband][nx][ny] (device) the start vector or NULL for 0.5 + u_e (the SplitMix64 start of
 * PFB_STEP_SAFE_GAMMA).  Costs `iters`
 * Hessian applications; returns after synchronising the stream. */
int pfb_step_bound(pfb_ctx *ctx, const pfb_geom *geom, pfb_prec prec, const pfb_params *params, int64_t nrow,
                   int32_t nchan, const double *uvw, const double *freq, const int32_t *band_of_chan,
                   const void *wgt, const void *psf, const double *wsum, const void *z0, int32_t iters,
                   double *lmax_out, void *stream);

/* The bound of the context's last pfb_step_bound, or of its last pfb_clean with
 * PFB_STEP_SAFE_GAMMA, and the step size that solve used (host doubles; 0 when none). */
int pfb_last_step_bound(pfb_ctx *ctx, double *lmax_out, double *gamma_out);

/* Per-kernel device timing (tracing; not part of the paper's method).
 * pfb_timing(ctx, 1) clears the totals and starts recording CUDA events around
 * every kernel group the library enqueues (on the caller's stream, so timings
 * reflect that stream's order); pfb_timing(ctx, 0) stops recording. */
int pfb_timing(pfb_ctx *ctx, int enable);

/* Totals since timing was enabled for one kernel group name ("grid_tiles",
 * "gather", "fft_fwd", ...), or "*" for all groups together (then *launches is
 * the number of this library's own kernel launches, cuFFT excluded).  bytes (may
 * be NULL) receives the algorithmic HBM traffic of those launches: the bytes the
 * operation must read and write at minimum, computed from the sizes.  Waits for
 * the recorded events. */
int pfb_timing_read(pfb_ctx *ctx, const char *kernel, int64_t *launches, double *total_ms, double *bytes);

/* Comma-separated names of the groups recorded so far, written into buf (len bytes). */
int pfb_timing_names(pfb_ctx *ctx, char *buf, size_t len);

/* Per-band weight sums with no device allocation (the paper has no counterpart:
 * this is a deployment variant of the weight-sum reduction behind pfb_dirty's and
 * pfb_psf's wsum_out).  For callers that may not call cudaMalloc at this point,
 * such as an engine that owns the whole HBM pool, or a stream where an allocation
 * could synchronise the device.
 *   wsum_out[b] = sum over rows and the channels c of band b of wgt[row][c]
 *   (1 per visibility when wgt is NULL).
 * device: CUDA device to run on; the calling thread's current device is restored
 * before the call returns.  band_of_chan [nchan] int32 (device memory); an id outside
 * [0, nband) makes the call return PFB_ERR_ARG, as pfb_dirty does.  wgt
 * [nrow][nchan] float32 (PFB_F32) / float64 (PFB_F64) (device memory) or NULL.
 * wsum_out [nband] float64, host or device memory owned by the caller (the result is
 * copied out with cudaMemcpyDefault); the call returns after `stream` has completed
 * its work, so wsum_out is valid on return (as with pfb_dirty's host wsum_out).
 * The accumulators are a fixed device array of 33 doubles inside the library (every
 * GPU that loads the library holds it until the process exits): nband > 32 returns
 * PFB_ERR_ARG.  The call clears them on `stream` before use.  All calls on a device
 * share that array, so calls whose work overlaps on the GPU (different streams, or
 * host threads without ordering) race: order them on one stream.  The first call on
 * a device looks up the array's device address (with that device current), which
 * may also load the library's device code on that device; make that first call
 * before any stream capture.  Errors: PFB_ERR_ARG for bad sizes, host pointers where
 * device memory is required, or out-of-range band ids; PFB_ERR_CUDA for a failed
 * launch; pfb_last_error(NULL) gives the message. */
int pfb_wsum_static(int device, pfb_prec prec, int64_t nrow, int32_t nchan, int32_t nband,
                    const int32_t *band_of_chan, const void *wgt, double *wsum_out, void *stream);

/* Support W (taps per axis, in u, v and w) of the ES kernel that the library picks
 * for a requested accuracy epsilon (Section 2; the smallest W whose worst-case
 * aliasing bound is <= epsilon at 2x oversampling).  Each visibility then costs
 * W^2 W_w multiply-adds per gridding or degridding pass (W_w = W with w-stacking,
 * 1 without).  Returns W (4..16), or PFB_ERR_EPS when epsilon is below what
 * `prec` reaches (1e-6 for PFB_F32, 1e-12 for PFB_F64) and PFB_ERR_ARG when it
 * is not positive and finite.  No device work. */
int pfb_kernel_support(double epsilon, pfb_prec prec);

/* Library version string. */
const char *pfb_version(void);

#ifdef __cplusplus
}
#endif

#endif /* PFB_H */
