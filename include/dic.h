/*
 * libdic: local-subset 2D digital image correlation on one GPU.
 *
 * The calls follow the paper's statement of the problem (Hirst et al., "Pyvale",
 * arXiv 2601.12941, Sec. 2.1, Listing 1): a reference image, a deformed image, a
 * region of interest, a seed, a subset size and a subset step; the result per
 * subset is the displacement (u, v), the shape-function parameters, a correlation
 * coefficient and convergence information (Sec. 4: "correlation coefficient
 * map", unconverged points optionally NaN).
 *
 * Method (all of it runs in this library's CUDA kernels):
 *   - cubic B-spline interpolation of gray levels at sub-pixel positions (Sec. 2.2),
 *     or Keys' bicubic convolution (dic_interp);
 *   - the ZNSSD cost (Eq. 4) minimised per subset over the rigid, affine or
 *     quadratic shape function (Eq. 5) by inverse-compositional Gauss-Newton;
 *   - reliability-guided propagation to the four nearest neighbours (Sec. 2.4,
 *     Fig. 3), run as deterministic frontier waves: every point on the frontier
 *     is correlated in one launch, starting from the warp of its accepted
 *     neighbour with the highest correlation coefficient;
 *   - an integer-pixel ZNCC search gives each seed its starting displacement.
 *
 * Conventions shared by every call:
 *   - Return value: DIC_OK (0) or a negative DIC_E* code; nothing is thrown
 *     across this interface. dic_last_error() gives the calling thread's last
 *     message.
 *   - Images are row-major. A dic_image with on_device = 1 is borrowed: the
 *     device buffer must stay valid and unchanged until it is replaced or the
 *     handle is destroyed. Host images (on_device = 0) are copied during the call
 *     and may be reused as soon as it returns.
 *   - Result pointers are owned by the handle and stay valid until the next
 *     dic_correlate or dic_destroy on it.
 *   - A handle is used by one host thread at a time. Different handles may be
 *     used at the same time from different host threads, each on its own stream.
 */
#ifndef DIC_H
#define DIC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- return codes -------------------------------------------------------- */
#define DIC_OK 0
#define DIC_EINVAL (-1)   /* an argument is out of range or inconsistent      */
#define DIC_ENOMEM (-2)   /* a device or pinned-host allocation failed         */
#define DIC_ECUDA (-3)    /* a CUDA call failed; see dic_last_error()          */
#define DIC_ETIMEOUT (-4) /* the wave loop exceeded its bound                  */
#define DIC_ENOSEED (-5)  /* no seed could start (all out of ROI or rejected)  */
#define DIC_ESTATE (-6)   /* call made in the wrong order (e.g. no images)     */

/* ---- enumerations -------------------------------------------------------- */
typedef enum { DIC_U8 = 0, DIC_U16 = 1, DIC_BF16 = 2, DIC_F32 = 3, DIC_F64 = 4 } dic_dtype;

/* Eq. 5: rigid uses p0..p1, affine p0..p5, quadratic p0..p11 (no 1/2 factor):
 *   x' = x_c + p0 + (1+p2) dx + p3 dy + p6 dx^2 + p7 dx dy + p8 dy^2
 *   y' = y_c + p1 + p4 dx + (1+p5) dy + p9 dx^2 + p10 dx dy + p11 dy^2
 * with (dx, dy) the pixel offset from the subset centre (x_c, y_c). */
typedef enum { DIC_RIGID = 0, DIC_AFFINE = 1, DIC_QUADRATIC = 2 } dic_shape;

/* Cost minimised per subset: ZNSSD (Eq. 4, the paper's default), NSSD (Eq. 3) or
 * SSD (Eq. 2). Each enters the IC-GN step through its residual: b = sum SD_i e_i with
 * e_i = fbar_i - (||fbar|| / ||gbar||) gbar_i, f_i - (||f|| / ||g||) g_i or f_i - g_i.
 * The reported coefficient and the acceptance test remain the ZNCC (see zncc in
 * dic_results for the warp it is taken at). */
typedef enum { DIC_COST_ZNSSD = 0, DIC_COST_NSSD = 1, DIC_COST_SSD = 2 } dic_cost;

/* Per-subset optimiser (Sec. 2.2 names Levenberg-Marquardt and leaves the details to
 * the literature): undamped inverse-compositional Gauss-Newton (default), or
 * Levenberg-Marquardt with Marquardt's diagonal damping H + lambda diag(H), lambda from
 * 1e-3. A trial warp is kept when it is the first, lowers the cost (Eq. 2-4) or
 * shortens the undamped Gauss-Newton step; keeping it divides lambda by 10, refusing
 * it multiplies lambda by 10, and the next step is always taken from the best trial
 * so far. A point has converged when the best trial's undamped step is below
 * conv_threshold (that step is then applied). Both optimisers reach the same root. */
typedef enum { DIC_OPT_GAUSS_NEWTON = 0, DIC_OPT_LEVENBERG_MARQUARDT = 1 } dic_optimizer;

/* Interpolant of the gray levels at sub-pixel positions.
 *   DIC_BSPLINE3: interpolating cubic B-spline, whole-sample mirror boundary
 *                 (Sec. 2.2, the default); the coefficient planes come from a
 *                 prefilter of each image.
 *   DIC_BICUBIC:  Keys' bicubic convolution, kernel parameter a = -1/2, on the gray
 *                 levels themselves (no prefilter), same 4 x 4 support, sampling
 *                 bounds and mirror boundary; the reference gradient is the
 *                 central difference (f[k+1] - f[k-1]) / 2. */
typedef enum { DIC_BSPLINE3 = 0, DIC_BICUBIC = 1 } dic_interp;

/* How the seeds of dic_correlate start (Sec. 2.2):
 *   DIC_INIT_SEARCH: the integer ZNCC search over |du|, |dv| <= search_radius;
 *   DIC_INIT_FFT:    the multi-window FFT initialiser (dic_fft_field, without the
 *                    sub-pixel fit) runs first and every seed starts from its
 *                    estimate at the seed's grid point, rounded to the nearest
 *                    integer, halves up (the paper's default MULTIWINDOW_RG). */
typedef enum { DIC_INIT_SEARCH = 0, DIC_INIT_FFT = 1 } dic_init;

/* DIC_MIXED: gray levels kept in their input type; interpolation coefficients,
 * samples, sums, the Jacobi-scaled Hessian inverse (FP64 when a scaled pivot falls
 * below 1e-5), the solve, the warp update and the ZNCC normalisation in FP32;
 * results stored as FP64. DIC_FP64: FP64 everywhere. DIC_MIXED_FP64_SOLVE: as
 * DIC_MIXED, except that each Gauss-Newton step solves H dp = -b beyond FP32
 * accuracy (the Hessian in FP64 from the FP32 moment sums; one step of iterative
 * refinement whose residual is evaluated in FP64, the FP32 inverse supplying the
 * first solution and the correction) and the final ZNCC is normalised in FP64 from
 * the FP32 sums; Gauss-Newton with ZNSSD on the B-spline only. */
typedef enum { DIC_FP64 = 0, DIC_MIXED = 1, DIC_MIXED_FP64_SOLVE = 2 } dic_precision;

/* per-point status (dic_results.status) */
enum {
  DIC_PT_OK = 0,            /* converged, ZNCC >= zncc_min, in bounds: accepted */
  DIC_PT_NOT_IN_ROI = 1,    /* part of the S x S subset is outside the ROI mask */
  DIC_PT_NOT_REACHED = 2,   /* no accepted neighbour ever led to this point     */
  DIC_PT_OUT_OF_BOUNDS = 3, /* a sample fell outside 1 <= x < W-2, 1 <= y < H-2 */
  DIC_PT_MAX_ITER = 4,      /* max_iter updates without meeting conv_threshold  */
  DIC_PT_LOW_ZNCC = 5,      /* converged but ZNCC < zncc_min                    */
  DIC_PT_SINGULAR = 6,      /* Hessian pivot <= 1e-12 * max diagonal            */
  DIC_PT_FLAT = 7           /* subset RMS contrast <= 1e-6 * max(|mean|, 1)     */
};

/* ---- structures ---------------------------------------------------------- */
typedef struct {
  const void* data;          /* first pixel                                          */
  int32_t width, height;     /* pixels                                               */
  int64_t row_stride_bytes;  /* 0 means width * element size                        */
  int32_t dtype;             /* dic_dtype                                            */
  int32_t on_device;         /* 1: device pointer (borrowed); 0: host (copied)      */
} dic_image;

typedef struct {
  int32_t max_iter;          /* Sec. 4 default 40                                    */
  int32_t search_radius;     /* seed search |du|, |dv| <= R (default 8)             */
  double conv_threshold;     /* Sec. 4 default 0.01, on ||dp|| (see below)          */
  double zncc_min;           /* Sec. 4 "precision" 0.70, read as the ZNCC cut-off   */
  int32_t precision;         /* dic_precision (default DIC_MIXED)                   */
  int32_t nan_unconverged;   /* Sec. 4: 1 sets u, v, p of rejected points to NaN    */
  int32_t profile;           /* 1: record CUDA-event stage timings (dic_get_timing) */
  int32_t cost;              /* dic_cost (default DIC_COST_ZNSSD)                    */
  int32_t optimizer;         /* dic_optimizer (default DIC_OPT_GAUSS_NEWTON)         */
  int32_t init;              /* dic_init: how seeds start (default DIC_INIT_SEARCH)  */
  int32_t max_displacement;  /* DIC_INIT_FFT: expected largest |u|, |v| in px,       */
                             /* 0 <= D <= 4095 (default 32); see dic_fft_params      */
  int32_t reserved;          /* 0                                                    */
  double mad_tau;            /* DIC_INIT_FFT: outlier cut (default 3; <= 0: off)     */
  double mad_eps;            /* DIC_INIT_FFT: px added to the scaled MAD (0.5)       */
} dic_params;
/* ||dp|| = sqrt(dp0^2 + dp1^2 + r^2 (dp2^2+..+dp5^2) + r^4 (dp6^2+..+dp11^2)),
 * r = (subset_size - 1) / 2; a subset has converged once ||dp|| < conv_threshold. */

typedef struct {
  int64_t n_points;          /* nx * ny; point q = j * nx + i                        */
  int32_t nx, ny;            /* grid: x = r + i * step, y = r + j * step             */
  int32_t n_params;          /* 2, 6 or 12                                           */
  int32_t n_waves;           /* propagation waves run (seeds are wave 0)             */
  int64_t n_accepted;        /* points with status DIC_PT_OK                         */
  const int32_t* x;          /* [n_points] subset centre, pixels                     */
  const int32_t* y;
  const double* u;           /* [n_points] p0: displacement at the centre, px        */
  const double* v;           /* [n_points] p1                                        */
  const double* p;           /* [n_points][n_params], Eq. 5 parameters               */
  const float* zncc;         /* [n_points] ZNCC = 1 - ZNSSD/2 (NaN if none): Gauss-Newton */
                             /* takes it from its last iteration's pass (the warp the  */
                             /* final, sub-threshold update was computed at; p includes */
                             /* that update), Levenberg-Marquardt at the final p        */
  const int32_t* iters;      /* [n_points] parameter updates applied                 */
  const uint8_t* converged;  /* [n_points] 1 if ||dp|| < conv_threshold was met      */
  const uint8_t* status;     /* [n_points] DIC_PT_*                                  */
  const int32_t* wave;       /* [n_points] propagation wave, -1 if never attempted   */
} dic_results;

typedef struct {
  double prefilter_ms;       /* spline prefilter of the images that changed          */
  double setup_ms;           /* ROI flags, point reset, seed search                  */
  double waves_ms;           /* first wave launch to last wave completion            */
  double icgn_kernel_ms;     /* sum of the wave kernels' own durations               */
  double seed_kernel_ms;     /* integer ZNCC search kernel                           */
  int32_t n_wave_launches;   /* wave kernels launched (some may find an empty front) */
  int32_t n_waves;
  int64_t n_points_attempted;
  int64_t sum_sample_passes; /* sum over attempted points of (iters + 1)            */
} dic_timing;

typedef struct dic_handle dic_handle;

/* ---- calls --------------------------------------------------------------- */

/* Sec. 4 defaults: max_iter 40, conv_threshold 0.01, zncc_min 0.70; search
 * radius 8; DIC_MIXED; no NaN; no profiling. */
dic_params dic_default_params(void);

/* Creates a handle for a reference/deformed pair (Sec. 2.1, Listing 1).
 *   ref, def     : same width and height (>= 8 each); any dic_dtype.
 *   roi          : NULL (every grid point) or a DIC_U8 mask of the same size,
 *                  nonzero = inside; a point is used iff its whole S x S subset is.
 *   subset_size  : odd, 3 <= S <= 61 and S <= min(width, height).
 *   subset_step  : >= 1.
 *   shape_fn     : dic_shape. interp: dic_interp (DIC_BSPLINE3 or DIC_BICUBIC).
 * Allocates every device buffer the correlation needs; host images are copied,
 * device images borrowed. No kernel runs until dic_correlate.
 * Errors: DIC_EINVAL, DIC_ENOMEM, DIC_ECUDA. On error *out is NULL. */
int dic_create(const dic_image* ref, const dic_image* def, const dic_image* roi,
               int32_t subset_size, int32_t subset_step, int32_t shape_fn, int32_t interp,
               dic_handle** out);

/* Replaces the parameters (validated: max_iter >= 1, conv_threshold > 0,
 * -1 <= zncc_min <= 1, 0 <= search_radius <= 256, precision valid). */
int dic_set_params(dic_handle* h, const dic_params* params);
int dic_get_params(const dic_handle* h, dic_params* out);

/* Replace the reference or the deformed image (same size and dtype as at
 * creation). The reference's spline coefficients stay resident across calls
 * until the reference changes; a sequence replaces only the deformed image. */
int dic_set_reference(dic_handle* h, const dic_image* ref);
int dic_set_deformed(dic_handle* h, const dic_image* def);

/* Runs the hot path on cuda_stream (NULL: the legacy default stream): spline
 * prefilter of whichever image changed, seed search, and every propagation wave
 * until the front is empty. seeds_xy holds n_seeds (x, y) pixel pairs, each
 * snapped to the nearest grid point (ties to the lower index); seeds outside the
 * ROI are skipped. Returns once the results are complete on the device.
 * Errors: DIC_EINVAL (no seeds), DIC_ENOSEED (no seed inside the ROI or every
 * seed rejected), DIC_ECUDA, DIC_ETIMEOUT. */
int dic_correlate(dic_handle* h, const int32_t* seeds_xy, int32_t n_seeds, void* cuda_stream);

/* Next frame of a sequence (Sec. 2.1: several deformed images against one
 * reference): correlates the handle's current deformed image (set it with
 * dic_set_deformed) against the resident reference, starting every point that the
 * previous correlation on this handle accepted from its previous warp, all in
 * wave 0; the other points are reached by propagation as in dic_correlate. The
 * reference coefficients are reused unless the reference changed. Same outputs
 * and errors as dic_correlate; DIC_ESTATE without an earlier correlation or after
 * a precision change. */
int dic_correlate_sequence(dic_handle* h, void* cuda_stream);

/* Fills *out with device pointers (on_device = 1) or with pointers to host copies
 * owned by the handle (on_device = 0; copied during the call, ordered on the
 * stream of the last correlation). DIC_ESTATE before the first correlation and
 * after dic_set_subsets. */
int dic_get_results(dic_handle* h, dic_results* out, int32_t on_device);

/* Device pointer to the interpolation coefficients (spline coefficients, or the
 * gray levels as T under DIC_BICUBIC) of the reference (which = 0) or the
 * deformed image (which = 1) as computed by the last dic_correlate: height rows of
 * *ld elements, each element *elem_bytes wide (4: FP32 under DIC_MIXED, 8: FP64).
 * Owned by the handle; for inspection and tests. DIC_ESTATE before any correlate. */
int dic_get_coefficients(const dic_handle* h, int32_t which, const void** plane, int64_t* ld,
                         int32_t* elem_bytes);

/* Stage timings of the last dic_correlate; zeros unless params.profile = 1. */
int dic_get_timing(const dic_handle* h, dic_timing* out);

/* ---- strain (Sec. 2.3) -----------------------------------------------------
 *
 * At every grid point: the displacement gradient of a least-squares fit
 * u(x, y) = P(x, y) c over the window x window grid points centred on it (Eq. 8-9),
 * the deformation gradient F = I + grad u (Eq. 6) and one strain measure. The
 * virtual strain gauge is (window - 1) subset_step + subset_size pixels (Eq. 7).
 * Readings where the paper is silent: the window is centred on its point and
 * grad u is the slope of the fit there; only accepted points (status 0) inside the
 * grid enter a window and the centre must be accepted; the fit needs at least as
 * many points as basis terms and a well-posed design (the unit-diagonal normal
 * matrix in grid units keeps every elimination pivot above 1e-5), otherwise the
 * point has no strain (NaN, valid 0). The bases are taken as printed (no xy term).
 * FP32 arithmetic on displacements taken relative to the window's centre. */
typedef enum { DIC_STRAIN_BILINEAR = 0, DIC_STRAIN_BIQUADRATIC = 1 } dic_strain_basis;

/* Sec. 2.3: Green-Lagrange (F^T F - I)/2; Hencky ln sqrt(F^T F); Euler-Almansi
 * (I - (F F^T)^-1)/2; Biot right sqrt(F^T F) - I; Biot left sqrt(F F^T) - I. */
typedef enum {
  DIC_GREEN_LAGRANGE = 0,
  DIC_HENCKY = 1,
  DIC_EULER_ALMANSI = 2,
  DIC_BIOT_RIGHT = 3,
  DIC_BIOT_LEFT = 4
} dic_strain_measure;

/* Device arrays of nx * ny elements in grid order, owned by the caller: the
 * displacement gradient (du/dx, du/dy, dv/dx, dv/dy), the strain tensor
 * components (exx, eyy and the tensor shear exy), and 1 where the point has them. */
typedef struct {
  float* dudx;
  float* dudy;
  float* dvdx;
  float* dvdy;
  float* exx;
  float* eyy;
  float* exy;
  uint8_t* valid;
} dic_strain_outputs;

/* Strain of a displacement field on the subset grid: u, v and status are device
 * arrays of nx * ny elements in grid order (as dic_get_results gives them on the
 * device), subset_step the grid step in pixels, window odd in [3, 31]. Launches one
 * kernel on cuda_stream and returns; allocates nothing. Errors: DIC_EINVAL (a NULL
 * pointer, an empty grid, step < 1, a bad window, basis or measure), DIC_ECUDA. */
int dic_strain_field(const double* u, const double* v, const uint8_t* status, int32_t nx, int32_t ny,
                     int32_t subset_step, int32_t window, int32_t basis, int32_t measure,
                     const dic_strain_outputs* out, void* cuda_stream);

/* ---- serving support (the paper has no counterpart) ----------------------
 *
 * A server that keeps one handle per reference image answers later jobs on the
 * same reference without uploading or prefiltering it again, whatever their
 * subset settings, and admits jobs against a device-memory budget. */

/* Re-grids a handle for another subset size, step, shape function or ROI (the
 * arguments and checks of dic_create) and keeps its images and the reference's
 * spline coefficients resident. Per-point arrays are reused when large enough,
 * re-allocated otherwise. The previous results and the sequence state are
 * dropped: dic_get_results and dic_correlate_sequence give DIC_ESTATE until the
 * next dic_correlate. Errors: DIC_EINVAL (the handle is unchanged); DIC_ENOMEM
 * or DIC_ECUDA (the handle keeps its images but has no grid, and dic_correlate
 * gives DIC_ESTATE, until a later dic_set_subsets succeeds). */
int dic_set_subsets(dic_handle* h, const dic_image* roi, int32_t subset_size, int32_t subset_step,
                    int32_t shape_fn);

/* Device bytes that dic_create with these arguments followed by one dic_correlate
 * with n_seeds seeds requests: owned copies of host images (on_device = 0, rows
 * padded to 128 bytes), the two coefficient planes in params' precision, the
 * per-point arrays, the ROI flags when has_roi, and the seed-search buffers. Only
 * width, height, dtype and on_device of ref and def are read (data may be NULL).
 * Not included: the driver's rounding of each allocation to its granularity, and
 * the transient copy of the ROI mask while flags are computed. Errors: DIC_EINVAL. */
int dic_estimate_device_bytes(const dic_image* ref, const dic_image* def, int32_t has_roi,
                              int32_t subset_size, int32_t subset_step, int32_t shape_fn,
                              const dic_params* params, int32_t n_seeds, int64_t* bytes);

/* Device bytes that h holds after dic_set_subsets with these settings,
 * dic_set_deformed(def) and one dic_correlate with n_seeds seeds: the reference
 * copy and, at an unchanged precision, the coefficient planes are kept, and
 * every other buffer keeps its current capacity unless the new settings need
 * more. Only width, height, dtype and on_device of def are read. Errors:
 * DIC_EINVAL. */
int dic_estimate_regrid_bytes(const dic_handle* h, const dic_image* def, int32_t has_roi,
                              int32_t subset_size, int32_t subset_step, int32_t shape_fn,
                              const dic_params* params, int32_t n_seeds, int64_t* bytes);

/* Device bytes the handle holds now: the requested sizes of its live allocations. */
int dic_get_device_bytes(const dic_handle* h, int64_t* bytes);

/* ---- multi-window FFT initialiser (Sec. 2.2, Eq. 1; Sec. 4) ---------------- */
/* Rigid displacement estimates by normalised FFT cross-correlation of square
 * windows that halve from above the expected maximum displacement down to the
 * subset size (window sizes: the powers of two above D, largest first, that exceed
 * the subset size S and fit in the image, then S). A power-of-two level tiles the
 * image (window (i, j) covers [iL, iL + L) x [jL, jL + L)); the last level's windows
 * are the S x S subsets of the correlation grid. Each window's deformed window is
 * moved by the previous level's estimate, interpolated bilinearly between the four
 * nearest window centres and rounded (halves up), and clamped into the image.
 * Eq. 1 is computed as the zero-normalised circular cross-correlation
 *   R(s) = sum_x (f(x) - f_m)(g(x - s) - g_m) / (||f - f_m|| ||g - g_m||)
 * through one packed complex 2-D transform per window; its largest value (ties to
 * the lower row-major index (s_y, s_x)) gives the shift d = -s wrapped into
 * [-floor(L/2), ceil(L/2) - 1], and the window's displacement is the deformed
 * window's offset plus d. After every level each value whose u or v differs from
 * the median over its 3 x 3 neighbourhood of windows (itself included) by more than
 * tau (1.4826 MAD + eps) takes the neighbourhood medians. A window with a constant
 * f or g gives d = 0 and peak 0. Sub-pixel (last level, optional): per axis the
 * vertex of the Gaussian through the peak and its two circular neighbours, kept at
 * 0 unless all three are positive. FP32 transforms, FP64 guesses and MAD tests. */
typedef struct {
  int32_t max_displacement;  /* D, px, 0 <= D <= 4095 (default 32)                   */
  int32_t subpixel;          /* 1: Gaussian peak fit on the last level (default 1)   */
  double mad_tau;            /* outlier cut (default 3); <= 0 switches it off        */
  double mad_eps;            /* px added to the scaled MAD (default 0.5)             */
} dic_fft_params;

typedef struct {
  int64_t n_points;          /* grid points, as in dic_results                       */
  int32_t nx, ny;
  int32_t n_levels;          /* window sizes used, coarse to fine; the last is S     */
  int32_t window[16];
  const float* u;            /* [n_points] last-level displacement, px (device)      */
  const float* v;
  const float* peak;         /* [n_points] R at the integer peak (Eq. 1)             */
  const uint8_t* status;     /* [n_points] DIC_PT_OK, or DIC_PT_NOT_IN_ROI           */
  const uint8_t* replaced;   /* [n_points] 1 where the MAD rule replaced the value   */
} dic_fft_results;

/* Sec. 2.2 defaults of this library: D = 32, sub-pixel fit on, tau = 3, eps = 0.5. */
dic_fft_params dic_fft_default_params(void);

/* Runs the whole initialiser (the paper's MULTIWINDOW method) on the handle's
 * reference and deformed images over its subset grid and ROI. Allocates, on first
 * use, a work buffer of up to 8 bytes per image pixel for windows above 64 px and
 * per-window arrays (kept until dic_destroy). Errors: DIC_EINVAL (D outside
 * [0, 4095], or no handle), DIC_ESTATE (no grid), DIC_ENOMEM, DIC_ECUDA. */
int dic_fft_field(dic_handle* h, const dic_fft_params* fp, void* cuda_stream);

/* Device arrays of the last dic_fft_field (or of the initialiser run by a
 * dic_correlate with DIC_INIT_FFT), owned by the handle. DIC_ESTATE before any. */
int dic_get_fft_results(const dic_handle* h, dic_fft_results* out);

/* Eq. 1 over explicit windows of side `window` (odd 3..63, or a power of two
 * 4..4096) on the handle's images: origins is a device array of n_windows
 * (x0, y0, gx0, gy0) int32 quadruples, reference and deformed window origins (each
 * window inside its image; x0 < 0 marks a window to skip, which gets 0s). Writes
 * device arrays u, v (the deformed offset plus the shift, sub-pixel when subpixel
 * = 1, which needs window <= 64) and peak. Errors: DIC_EINVAL, DIC_ENOMEM,
 * DIC_ECUDA. */
int dic_fftcc_windows(dic_handle* h, int32_t window, int64_t n_windows, const int32_t* origins,
                      int32_t subpixel, float* u, float* v, float* peak, void* cuda_stream);

/* The MAD rule above over an nx x ny field of device arrays u, v (valid: NULL, or
 * nonzero for the values that take part and get tested); writes u_out, v_out and,
 * when non-NULL, replaced. In-place calls (u_out == u) are not allowed. Errors:
 * DIC_EINVAL. */
int dic_mad_filter(const float* u, const float* v, const uint8_t* valid, int32_t nx, int32_t ny, double tau,
                   double eps, float* u_out, float* v_out, uint8_t* replaced, void* cuda_stream);

/* ---- incremental reference updating (planned in Sec. 6) --------------------- */
/* For sequences with large strains, after Pan et al. 2012: the reference image
 * evolves through the sequence. Every grid point of the first reference carries its
 * warp from the first frame; a frame correlated against the current reference gives
 * the point's total warp: x_r = X + (u_a, v_a) is its current position, the grid
 * point q nearest to x_r (per axis, ties to the lower index) must be accepted in the
 * frame, q's warp re-expanded at x_r - x_q gives (d, A_i), and
 *     (u, v) = (u_a, v_a) + d,     I + A = (I + A_i)(I + A_a)
 * with A = [[p2, p3], [p4, p5]] of Eq. 5 (A = 0 for the rigid shape function). The
 * first reference is the one of the last dic_correlate (or dic_set_reference, or
 * dic_set_subsets); until the first update the totals are the frame's own warps. */
typedef struct {
  int64_t n_points;          /* grid points, as in dic_results                       */
  int32_t nx, ny;
  int32_t n_params;
  int32_t n_updates;         /* reference updates since the first reference          */
  const double* u;           /* [n_points] total displacement, px (device)           */
  const double* v;
  const double* p;           /* [n_points][n_params] total warp; p2..p5 composed     */
  const uint8_t* status;     /* [n_points] DIC_PT_OK, DIC_PT_NOT_REACHED (no total   */
                             /* this frame, or lost at an earlier update), or        */
                             /* DIC_PT_NOT_IN_ROI                                    */
} dic_total_results;

/* Makes the handle's current deformed image the reference for the following frames:
 * the totals of the last correlation become the accumulated warps (points without
 * one drop out for good), the deformed image and its coefficients become the
 * reference's (a borrowed device image must stay valid while it is the reference),
 * and the next dic_correlate_sequence starts every in-ROI point from the identity
 * warp in wave 0 (dic_get_results shows that start until then). Rigid and affine
 * shape functions only: two quadratic warps of Eq. 5 do not compose into one.
 * Errors: DIC_EINVAL (no handle, quadratic), DIC_ESTATE (no correlation yet),
 * DIC_ENOMEM, DIC_ECUDA. */
int dic_update_reference(dic_handle* h, void* cuda_stream);

/* Computes, on cuda_stream, the total warps of the last correlated frame from the
 * first reference; device arrays owned by the handle, valid until its next
 * correlation, update or destroy. Errors: DIC_EINVAL, DIC_ESTATE, DIC_ENOMEM,
 * DIC_ECUDA. */
int dic_get_total_results(dic_handle* h, dic_total_results* out, void* cuda_stream);

/* ---- allocation-free correlation (the paper has no counterpart) ----------
 *
 * For callers that must not allocate device memory when they correlate: code
 * running inside an allocator's own callback, a real-time loop that cannot take
 * the driver's allocation locks, or a host that gives all device memory to its
 * own pool. dic_correlate_static runs the same kernels as dic_correlate (spline
 * prefilter, seed search, propagation waves) on caller-owned device images and
 * writes caller-owned device outputs; every intermediate buffer lives in one
 * file-scope device array of this library (about 10 MiB, held by every GPU that
 * loads the library until the process exits). It calls no cudaMalloc, cudaFree
 * or other allocating routine.
 *
 * Limits (larger problems return DIC_EINVAL and a message saying which):
 *   H * (W rounded up to 32) <= DIC_STATIC_MAX_PIXELS, grid points <=
 *   DIC_STATIC_MAX_POINTS, n_seeds <= DIC_STATIC_MAX_SEEDS, search_radius <=
 *   DIC_STATIC_MAX_RADIUS; precision must be DIC_MIXED; no ROI (every grid point);
 *   the interpolant is the cubic B-spline.
 * Shared state: all calls in the process use the same array and it keeps the
 * last call's contents (every call clears what must start from zero). Calls that
 * overlap on the GPU (other streams or host threads) race on it: serialise them.
 * The first call on each device looks up the array's device address and caches
 * it; make that first call before any stream capture.
 * Arguments: ref, def: device images (on_device = 1), same size and dtype;
 * subset_size, subset_step, shape_fn, params, seeds_xy, n_seeds as for
 * dic_create / dic_correlate; out: device arrays of n_points = nx * ny entries
 * (p: n_points * n_params doubles) in grid order, n_accepted an optional host
 * pointer; errbuf (optional, errlen bytes) receives the message of a failure.
 * Returns once the outputs are complete. Errors: DIC_EINVAL, DIC_ENOSEED,
 * DIC_ECUDA, DIC_ETIMEOUT. */
#define DIC_STATIC_MAX_PIXELS 1048576
#define DIC_STATIC_MAX_POINTS 65536
#define DIC_STATIC_MAX_SEEDS 16
#define DIC_STATIC_MAX_RADIUS 32

typedef struct {
  double* u;
  double* v;
  double* p;
  float* zncc;
  int32_t* iters;
  uint8_t* converged;
  uint8_t* status;
  int32_t* wave;
  int64_t* n_accepted;       /* host, optional */
} dic_static_outputs;

int dic_correlate_static(const dic_image* ref, const dic_image* def, int32_t subset_size,
                         int32_t subset_step, int32_t shape_fn, const dic_params* params,
                         const int32_t* seeds_xy, int32_t n_seeds, const dic_static_outputs* out,
                         void* cuda_stream, char* errbuf, int32_t errlen);

/* Test hook for the timeout path; the paper has no counterpart. Every wait inside a
 * kernel is bounded: the wave kernel polls the mbarrier of a tile load at most
 * 65,536 times, and a wait that runs out sets an error flag, lets the copy in
 * flight land (a second bounded wait), ends its block and makes dic_correlate /
 * dic_correlate_sequence return DIC_ETIMEOUT. on != 0 makes the first of those
 * waits give up at once in every wave launched afterwards by this process (the
 * second wait keeps its full bound, so no copy is left in flight); 0 restores
 * normal waits. Results of a run that timed out are incomplete; the handle stays
 * usable. Returns DIC_OK. Not for production use. */
int dic_test_expire_tile_waits(int32_t on);

/* Frees every buffer of the handle (NULL is ignored). */
void dic_destroy(dic_handle* h);

/* Thread-local text of the last error on the calling thread ("" if none). */
const char* dic_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* DIC_H */
