/*
 * ash.h -- C ABI of the aberration-space holography library (GB300, sm_103a).
 *
 * The library computes the compressed spot transform of aberration-space
 * holography (Christen et al., arXiv 2505.08777) and the weighted
 * Gerchberg-Saxton loop built on it, with hand-written CUDA kernels. It never
 * forms the N x M kernel matrix: every kernel value exp(-i C_n . Z_m) is
 * evaluated on the fly.
 *
 * Notation (paper Sec. II and Methods "Computational Scaling"):
 *   nx, ny  SLM grid; pixel (i, j) = column i, row j; M = nx*ny;
 *           per-pixel arrays are row-major [ny][nx], flat index m = j*nx + i.
 *   D       number of basis modes Z_d (Zernike polynomials in Noll order, or
 *           a caller-supplied basis).
 *   N       number of spots; C is the N x D coefficient matrix w_d^(n),
 *           row-major [N][D], radians per unit of basis value.
 *   A_m     illumination amplitude (real); phi_m SLM phase;
 *           f_m = A_m exp(i phi_m) the nearfield.
 *   Forward  E_n = sum_m f_m exp(-i C_n . Z_m)          (Sec. II, F_n = F_c{f})
 *   Adjoint  g_m = sum_n y_n exp(+i C_n . Z_m)          (Sec. II, f = F_c^-1{F})
 *   Sums are unnormalised (the paper writes them up to proportionality).
 *
 * Zernike basis (when a Noll list is given): pixel coordinates
 *   x = (i - (nx-1)/2)/R, y = (j - (ny-1)/2)/R, R = min(nx, ny)/2,
 *   Z = R_n^|m|(rho) cos(m theta) (m >= 0) or R_n^|m|(rho) sin(|m| theta)
 *   (m < 0), no RMS normalisation; pixels outside the unit disk keep their
 *   polynomial values. Noll 2/3 are the x/y tilts, Noll 4 defocus (Sec. II).
 *
 * Complex arrays are interleaved float pairs (re, im), i.e. complex64.
 *
 * Ownership: the caller owns every buffer passed in; all of them are device
 * pointers unless a parameter says "host". The handle owns its workspace
 * (basis in a tiled internal layout, copied coefficients, anchor table,
 * forward partial sums), allocated in ash_hologram_create (through the
 * allocator hook, see ash_set_allocator) and freed in ash_hologram_destroy.
 * The handle keeps no pointer to caller buffers after a call returns.
 *
 * Streams: every call enqueues its work on `stream` (a cudaStream_t; NULL =
 * legacy default stream) and returns without synchronising, except where a
 * description says otherwise. A handle must not be used from two streams at
 * once (calls share the handle's workspace). Different handles may be used
 * at the same time, from different streams and host threads (each owns its
 * workspace and loop graphs); ash_forward_noalloc calls must not overlap.
 *
 * Errors: every call returns an ash_status. Invalid arguments return
 * ASH_ERR_INVALID_ARG before anything is launched. CUDA failures return
 * ASH_ERR_CUDA; ash_last_error() gives a message (per host thread). Nothing
 * aborts the process. Kernels never spin on another CTA; device-side faults
 * that a kernel detects set an error word that ash_hologram_check() reports.
 *
 * Precision: inputs FP32, arithmetic FP32 with complex64 accumulation;
 * per-(spot, tile) base phases are reduced exactly in turns from FP64-derived
 * tables so that tilts of thousands of radians keep ~1e-6 rad phase error.
 * Transforms match the FP64 definition to 1e-4 (normwise) while
 * max |C_n . Z_m| <= 2.5e3 rad. Beyond that, as on very elongated grids
 * where R is half the short side and high-order modes grow on the long
 * axis, rounding Z_m to FP32 alone costs about 2^-24 max |C_n . Z_m|.
 */
#ifndef ASH_H
#define ASH_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ASH_ABI_VERSION 1

typedef enum {
  ASH_OK = 0,
  ASH_ERR_INVALID_ARG = 1,
  ASH_ERR_CUDA = 2,
  ASH_ERR_OOM = 3,
  ASH_ERR_TIMEOUT = 4,
  ASH_ERR_UNSUPPORTED = 5,
  ASH_ERR_INJECTED = 6,
  ASH_ERR_DEVICE = 7
} ash_status;

/* Opaque handle: one hologram (grid, amplitude, basis, coefficients). */
typedef struct ash_hologram ash_hologram;

/* Largest supported number of basis modes D. */
#define ASH_MAX_MODES 16

/* ABI version of the loaded library (ASH_ABI_VERSION at build time). */
int ash_abi_version(void);

/* Human-readable name of a status code (static string). */
const char *ash_status_string(ash_status s);

/* Last error message recorded on the calling host thread ("" if none). */
const char *ash_last_error(void);

/*
 * Allocator hook for the handle workspaces. alloc(ctx, bytes, stream) returns
 * a device pointer or NULL (reported as ASH_ERR_OOM); free(ctx, ptr, stream)
 * releases it. Passing NULL for both restores cudaMallocAsync/cudaFreeAsync.
 * Process-wide; set it before creating handles.
 */
typedef void *(*ash_alloc_fn)(void *ctx, size_t bytes, void *stream);
typedef void (*ash_free_fn)(void *ctx, void *ptr, void *stream);
ash_status ash_set_allocator(ash_alloc_fn alloc, ash_free_fn free_fn, void *ctx);

/*
 * Host-side fault injection for tests: the n-th API call from now (n >= 1)
 * that would launch work returns ASH_ERR_INJECTED without launching; n = 0
 * disables it. Process-wide.
 */
ash_status ash_debug_fail_after(int n_calls);

/*
 * The transforms' two sin / cos evaluations, for accuracy tests: path 0 the
 * MUFU approximations (sin.approx / cos.approx), path 1 the FP32-pipe
 * polynomial (half-angle reduction, degree-4 polynomials in r^2). x, s, c
 * are device float[n] (n >= 0); s_i = sin(x_i), c_i = cos(x_i). Enqueued on
 * `stream`; ASH_ERR_INVALID_ARG for a NULL pointer, n < 0 or another path.
 */
ash_status ash_debug_sincos(const float *x, int n, float *s, float *c, int path, void *stream);

/*
 * Per-SM unit rates that bound the transforms (Methods, "Computational
 * Scaling": every term needs a phase, a sine, a cosine and a complex
 * multiply-accumulate, so the chip's sin/cos and FP32 rates set the
 * roofline). Measured on the current device: one CTA of 1024 threads per SM,
 * independent chains of one operation, timed by the SM cycle counter.
 *   out  host double[ASH_PROBE_COUNT]:
 *        [0] sin.approx / cos.approx results per clock per SM (MUFU)
 *        [1] fma.rn.f32 lane results per clock per SM
 *        [2] fma.rn.f32x2 lane results per clock per SM (two per instruction)
 *        [3] ex2.approx results per clock per SM (MUFU)
 *        [4] SM clock during the probe, MHz (cycles / CUDA-event time)
 *        [5] SMs that ran the probe
 * Allocates two small device arrays on `stream` (stream-ordered) and
 * synchronises it; takes about 10 ms. ASH_ERR_INVALID_ARG for a NULL out,
 * ASH_ERR_CUDA if a launch fails.
 */
#define ASH_PROBE_COUNT 6
ash_status ash_probe_rates(double *out, void *stream);

/*
 * Create a hologram (paper Sec. II: kernels K_n built from the N x D matrix
 * w_d^(n) and the per-pixel basis, Methods "Computational Scaling").
 *   out     host: receives the handle.
 *   nx, ny  grid, 1 <= nx, ny <= 16384.
 *   amp     device float[ny*nx], illumination amplitude A (row-major).
 *   D       number of modes, 1 <= D <= ASH_MAX_MODES.
 *   noll    host int[D] Noll indices (>= 1, <= 231) of the Zernike modes, or
 *           NULL when `basis` is given.
 *   basis   device float[D*ny*nx], caller basis, row d = Z_d over the grid
 *           (row-major), or NULL when `noll` is given. Exactly one of noll /
 *           basis must be non-NULL.
 *   N       number of spots, 1 <= N <= 1<<20.
 *   coeff   device float[N*D], C row-major.
 *   stream  cudaStream_t for the set-up kernels.
 * The basis is materialised once, relative to per-tile anchor pixels, in a
 * tiled internal layout (FP64 evaluation of the monomial expansion for Noll
 * lists). Returns ASH_ERR_OOM if the workspace cannot be allocated.
 * Synchronises `stream` before returning (the set-up kernels and the
 * stream-ordered allocations are complete when the handle is returned).
 */
ash_status ash_hologram_create(ash_hologram **out, int nx, int ny, const float *amp, int D,
                               const int *noll, const float *basis, int N, const float *coeff,
                               void *stream);

/*
 * Create a hologram whose D modes are fixed combinations of Zernike modes
 * (paper Sec. III and Methods "Anisoplanatic Singular Value Decomposition":
 * principal isoplanatic modes are a rotation of the Zernike basis; Methods
 * "Computational Scaling": other bases can be used to reduce D).
 *   noll    host int[D_in] Noll indices of the input Zernike modes, 1 <= D_in <= 64.
 *   mix     host double[D*D_in], row-major: output mode k = sum_d mix[k][d] Z_{noll[d]}
 *           (e.g. the `mix` of ash_principal_modes).
 *   D       number of output modes, 1 <= D <= ASH_MAX_MODES.
 *   coeff   device float[N*D], coefficients of the output modes.
 * Other arguments as ash_hologram_create. The combined polynomials are
 * formed and evaluated in FP64, so the basis carries no extra rounding; an
 * output row that is a single input mode with weight 1 counts as that
 * Zernike (a pair of exact tilts keeps the one-K-atom tensor-core layout).
 */
ash_status ash_hologram_create_mixed(ash_hologram **out, int nx, int ny, const float *amp, int D_in,
                                     const int *noll, int D, const double *mix, int N,
                                     const float *coeff, void *stream);

/*
 * Create a band hologram: rows [row0, row1) of an SLM grid of nx x ny_full
 * pixels, for pixel-sharded transforms over several GPUs (Methods,
 * "Computational Scaling": each pixel's kernel values depend only on that
 * pixel and the global N x D matrix, so the forward is a sum over pixel
 * blocks and the adjoint is independent per pixel). The band uses the full
 * grid's coordinates (unit disk of radius min(nx, ny_full)/2 about the full
 * grid's centre), tiles and tile anchors, so that
 *   sum over bands of ash_forward(band)  ==  ash_forward(full grid)
 *   ash_adjoint(band)                    ==  the band's rows of ash_adjoint(full grid)
 * up to the summation order of fp32 partial sums.
 *   row0, row1  0 <= row0 < row1 <= ny_full; row0 a multiple of 32 and row1
 *               a multiple of 32 or ny_full (whole 32-row tile rows).
 *   amp     device float[(row1-row0)*nx]: the band's rows of the amplitude.
 *   basis   device float[D*(row1-row0)*nx] (the band's rows of each mode) or
 *           NULL with `noll`.
 * Phases, fields and outputs of the band's calls are (row1-row0) x nx.
 * Other arguments and behaviour as ash_hologram_create.
 */
ash_status ash_hologram_create_band(ash_hologram **out, int nx, int ny_full, int row0, int row1,
                                    const float *amp, int D, const int *noll, const float *basis, int N,
                                    const float *coeff, void *stream);

/*
 * Band of a handle: first row and rows of the full grid (0 and ny for a
 * handle that is not a band), and the handle's sum of A^2 over its own
 * pixels (host double). Any pointer may be NULL. Reading sum_a2
 * synchronises the device.
 */
ash_status ash_hologram_band(const ash_hologram *h, int *row0, int *ny_full, double *sum_a2);

/*
 * The weighted-GS spot update alone (Sec. II / Sec. III; rule and options as
 * in ash_wgs_iterate and ash_wgs_set_options): from the spot fields E,
 *   w <- w (T^ / E^)^p, renormalised;  y = w exp(i psi)  (psi = arg E, or the
 *   held phases when phase fixing is on).
 *   E       device float[2N] complex64 (e.g. the all-reduced partial fields
 *           of all bands of a sharded grid).
 *   w       device float[N], updated in place; target device float[N].
 *   y       device float[2N] complex64, written: the adjoint's spot weights.
 * Uses and updates the handle's held spot phases like ash_wgs_iterate. A
 * sharded loop runs it on every rank with the same E, so every rank holds
 * the same w and y.
 */
ash_status ash_spot_update(ash_hologram *h, const float *E, float *w, const float *target, float *y,
                           void *stream);

/*
 * Spot metrics of E (as ash_wgs_iterate's metrics_out): uniformity,
 * efficiency sum|E|^2 / (nx * ny_full * sum A^2), sum |E|^2, min |E|^2/T^2.
 *   sum_a2  the sum of A^2 over the whole grid (host double; for a sharded
 *           grid the sum over all bands), or 0 for the handle's own.
 *   metrics_out  device float[4].
 */
ash_status ash_spot_metrics(ash_hologram *h, const float *E, const float *target, double sum_a2,
                            float *metrics_out, void *stream);

/*
 * Principal isoplanatic modes (paper, Methods "Anisoplanatic Singular Value
 * Decomposition"; Sec. III "principal isoplanatic modes"): the SVD
 * W = U Sigma V^T of the N x ncols block W of the coefficient matrix formed
 * by the modes `cols`, truncated to the K largest singular values. Host
 * memory only, FP64, no GPU work.
 *   coeff      host float[N*D], C row-major.
 *   cols       host int[ncols], distinct mode positions in [0, D) to rotate
 *              (e.g. all but the tilts, which define the spot positions).
 *   K          principal modes kept, 0 <= K <= ncols.
 *   mix        host double[(D - ncols + K) * D] out: rows = output modes; first the
 *              modes not in `cols` (unit rows, original order), then the K
 *              principal modes (rows of V^T, by decreasing singular value; sign
 *              chosen so that each row's largest-magnitude entry is positive).
 *   coeff_out  host float[N * (D - ncols + K)] out: C of the output modes,
 *              untouched columns then (U Sigma)_k.
 *   sigma      host double[ncols] out (may be NULL): all singular values, decreasing.
 * With K = ncols, coeff_out . (mix . Z) equals C . Z up to rounding.
 */
ash_status ash_principal_modes(int N, int D, const float *coeff, int ncols, const int *cols, int K,
                               double *mix, float *coeff_out, double *sigma);

/* Destroy a handle (NULL is ignored). Synchronises the device (work on any
 * stream may still use the workspace), then frees the workspace. */
void ash_hologram_destroy(ash_hologram *h);

/* Sizes of a handle: any output pointer may be NULL. */
ash_status ash_hologram_info(const ash_hologram *h, int *nx, int *ny, int *N, int *D,
                             size_t *workspace_bytes);

/* Replace the coefficient matrix C (device float[N*D]); same N and D. */
ash_status ash_set_coefficients(ash_hologram *h, const float *coeff, void *stream);

/* Copy the coefficient matrix the handle holds into coeff (device
 * float[N*D], row-major), stream-ordered after the calls before it. */
ash_status ash_get_coefficients(const ash_hologram *h, float *coeff, void *stream);

/* Replace the illumination amplitude A (device float[ny*nx]). */
ash_status ash_set_amplitude(ash_hologram *h, const float *amp, void *stream);

/*
 * Forward transform of a phase-only hologram (Sec. II, F_n = F_c{f}):
 *   E_n = sum_m A_m exp(i phase_m) exp(-i C_n . Z_m).
 *   phase  device float[ny*nx].
 *   E      device float[2*N] (complex64), overwritten.
 * Deterministic: partial sums are reduced in a fixed order.
 */
ash_status ash_forward(ash_hologram *h, const float *phase, float *E, void *stream);

/*
 * Forward transform of a general complex nearfield (amplitude ignored):
 *   E_n = sum_m f_m exp(-i C_n . Z_m).
 *   field  device float[2*ny*nx] (complex64).
 *   E      device float[2*N] (complex64), overwritten.
 */
ash_status ash_forward_field(ash_hologram *h, const float *field, float *E, void *stream);

/*
 * Set the coefficients and run the forward in one call (ash_set_coefficients
 * then ash_forward, enqueued on `stream`): the forward pass of a gradient
 * step on C (Methods, gradients through the transform) with one call.
 *   coeff   device float[N*D]; phase device float[M]; E device float[2N].
 */
ash_status ash_forward_coeff(ash_hologram *h, const float *coeff, const float *phase, float *E, void *stream);

/*
 * Spot-intensity loss and its gradient (the objective of the gradient-descent
 * refinement; the paper gives none, so this is the reading used throughout):
 *   I_n = |E_n|^2, mu = mean I, r_n = I_n / mu - t_n, L = sum_n r_n^2,
 *   grad_E_n = dL/dRe E_n + i dL/dIm E_n = 2 G_n E_n,
 *   G_k = (2 / mu) (r_k - (1/N) sum_n r_n I_n / mu).
 *   E       device float[2N] complex64; t device float[N]; 1 <= N <= 2^20.
 *   loss    device float[1] or NULL; grad_E device float[2N] or NULL (not both NULL).
 * One CTA, sums in fp64 in a fixed order (deterministic).
 */
ash_status ash_spot_loss(const float *E, const float *t, int N, float *loss, float *grad_E, void *stream);

/*
 * Conjugate-gradient refinement of the SLM phase (paper Methods: precision
 * targets such as uniform top hats are refined by conjugate-gradient
 * descent through the transform's gradients). Loss: the spot-intensity
 * loss L = sum_n (I_n / mean I - t_n)^2, I = |E|^2 (the ash_grad loss).
 * Nonlinear CG with the Polak-Ribiere+ coefficient (restart to -g when the
 * direction does not descend) and a one-trial line search: the trial step
 * changes no pixel's phase by more than `theta`, and the step is the
 * minimum of the quadratic through L, its slope and the trial loss (twice
 * the trial step if that quadratic has no minimum). Each iteration runs two
 * forwards and one gradient adjoint; the loop is one CUDA graph per
 * iteration count. A call starts a fresh CG sequence (d = -g).
 *   phase     device float[ny*nx], in/out;  t  device float[N] loss targets;
 *   iters     0..1024;  theta  in (0, 3.2] rad;
 *   loss_out  device float[iters+1] or NULL: L before the first and after
 *             every iteration.
 */
ash_status ash_cg_refine(ash_hologram *h, float *phase, const float *t, int iters, float theta,
                         float *loss_out, void *stream);

/*
 * Simulated Zernike-subtraction calibration (paper Sec. III: a global
 * Zernike order is superimposed on the SLM with a swept amplitude, a
 * per-spot figure of merit gives each site's local contribution, which is
 * then subtracted spot by spot in aberration space). The handle `h` plays
 * the optical system (its coefficient matrix is the system's kernels).
 *
 * ash_zsub_sweep: for k = 0..K-1,
 *   intensity[k*N + n] = |E_n|^2,  E = K_h (A exp(i (phase + deltas[k] Z_mode))),
 * evaluated as the forward of `phase` through the coefficients with column
 * `mode` shifted by -deltas[k] for every spot (the same sum).
 *   phase      device float[ny*nx];  deltas  HOST float[K], 1 <= K <= 32;
 *   mode       column of the coefficient matrix, 0 <= mode < D;
 *   intensity  device float[K*N].
 * The handle's coefficients and operand images are restored afterwards (on
 * the stream), also when a launch fails.
 */
ash_status ash_zsub_sweep(ash_hologram *h, const float *phase, int mode, const float *deltas, int K,
                          float *intensity, void *stream);

/*
 * Per-spot estimate from a sweep: the least-squares parabola through
 * (deltas[k], ln max(intensity[k*N + n], 1e-37)) -- a Gaussian peak -- and
 * its vertex -b / (2 c), clipped to [min deltas, max deltas]; if the fitted
 * curvature c is not negative, the offset of the largest sample (the first
 * one on ties). Arithmetic in fp64.
 *   intensity  device float[K*N];  deltas HOST float[K], 3 <= K <= 32, at
 *              least three distinct values (else ASH_ERR_INVALID_ARG);
 *   delta_star device float[N], the estimates;
 *   coeff      device float[N*D] or NULL: if given, coeff[n*D + mode] +=
 *              delta_star[n] (the subtraction into the model's matrix).
 */
ash_status ash_zsub_estimate(const float *intensity, const float *deltas, int K, int N, float *delta_star,
                             float *coeff, int D, int mode, void *stream);

/*
 * Adjoint transform (Sec. II, f = F_c^-1{F}, the merge of all N kernels):
 *   g_m = sum_n y_n exp(+i C_n . Z_m).
 *   y          device float[2*N] (complex64).
 *   g          device float[2*ny*nx] (complex64) or NULL.
 *   phase_out  device float[ny*nx] or NULL: phase_out_m = arg g_m (0 where
 *              g_m == 0), the phase-only projection used by GS.
 * At least one of g / phase_out must be non-NULL.
 */
ash_status ash_adjoint(ash_hologram *h, const float *y, float *g, float *phase_out, void *stream);

/*
 * Weighted Gerchberg-Saxton iterations (Sec. II; Sec. III uses weighted GS).
 * The paper does not print the update rule; this library implements:
 *   init (caller): w = T, phase given.   T^ = T/||T||_2
 *   each iteration:  E = forward(phase);  E^ = |E|/||E||_2;
 *                    w <- w * T^ / max(E^, 1e-30);  w <- w/||w||_2;
 *                    phase <- arg adjoint(w exp(i arg E)).
 *   after the last iteration one more forward gives E_out and the metrics.
 *   phase        device float[ny*nx], in/out (the loop state).
 *   w            device float[N], in/out (the loop state).
 *   target       device float[N], target amplitudes T (> 0).
 *   iters        0 <= iters <= 1000000.
 *   E_out        device float[2*N] or NULL: field of the final phase.
 *   metrics_out  device float[4] or NULL: {uniformity, efficiency,
 *                sum |E|^2, min |E|^2/T^2}; uniformity
 *                U = 1 - (max I^ - min I^)/(max I^ + min I^), I^_n = |E_n|^2/T_n^2;
 *                efficiency = sum |E|^2 / (M sum A^2).
 * The state is exactly (phase, w), plus the held spot phases when phase
 * fixing is on (ash_wgs_set_options): running k iterations twice equals
 * running 2k iterations once, bit for bit. The loop is enqueued as a CUDA graph when
 * iters > 1 (captured on first use per handle and iteration count).
 */
ash_status ash_wgs_iterate(ash_hologram *h, float *phase, float *w, const float *target, int iters,
                           float *E_out, float *metrics_out, void *stream);

/*
 * Gradient through the forward transform (Methods: gradients propagated
 * forward and backward through the transform). Given grad_E = dL/dRe(E) +
 * i dL/dIm(E) for E = forward(phase):
 *   dphase_m = -Im(f_m conj(h_m)),  h = K^H grad_E      (adjoint pass)
 *   dcoeff_nd = Im(conj(grad_E_n) S_nd), S_nd = sum_m Z_dm f_m K_nm
 *               (forward pass with D moments, tiles recomputed; the phases
 *               C_n . Z_m come from the tensor cores when the operand row
 *               fits one K-atom, D <= 12 and the basis is a polynomial of
 *               total degree <= 4, else from the FMA pipe).
 * The tensor-core moment pass overwrites the handle's nearfield image (no
 * other state of the handle changes).
 *   phase   device float[ny*nx];  grad_E device float[2*N];
 *   dphase  device float[ny*nx] or NULL;  dcoeff device float[N*D] or NULL.
 */
ash_status ash_grad(ash_hologram *h, const float *phase, const float *grad_E, float *dphase,
                    float *dcoeff, void *stream);

/*
 * Launch shapes chosen for the handle, written to the host array out[8]:
 *   {CTAs of the FMA-pipe transform launches, their resident CTAs per SM
 *    (forward), (adjoint), CTAs of the tensor-core adjoint and of the
 *    tensor-core forward (0 if not available), split flags (bit 0: FMA schedule
 *    splits tiles, bit 1: tensor-core schedule splits sub-tiles, bit 2:
 *    the tensor-core forward splits spot blocks, bit 3: the tensor-core
 *    forward's CTAs claim their ranges by SM), kernels in use (adjoint:
 *    1 FMA or 2 tensor core, plus 4 if the forward and 8 if the
 *    coefficient-gradient moments use the tensor core), pixels per thread}.
 */
ash_status ash_hologram_launch_info(const ash_hologram *h, int *out);

/*
 * Kernel variant of the forward and adjoint transforms and of the
 * coefficient-gradient moments: 0 = automatic (the faster measured family
 * per pass: tensor cores when the operand row fits one K-atom, for the
 * forward and the moments from N = 64 spots, for the adjoint from N = 256),
 * 1 = FMA-pipe kernels, 2 = tensor-core kernels (available for every D a
 * handle accepts: one K-atom per operand row for D <= 10 and for D = 11
 * with both tilts, two otherwise; the moments stay on the FMA pipe where
 * their tensor-core pass is not available). Both
 * compute the same sums; the tensor-core variant forms the phases
 * C_n . dZ_m with split-tf32 tcgen05 MMAs into tensor memory. Drops the
 * handle's captured graphs.
 */
ash_status ash_set_kernel_variant(ash_hologram *h, int variant);

/*
 * WGS variants (the paper uses weighted GS after Kim et al., Sec. II "...with
 * the weighted Gerchberg-Saxton algorithm"): for the following
 * ash_wgs_iterate calls on this handle,
 *   feedback   exponent p of the weight update w <- w (T^/E^)^p, 0 <= p <= 16
 *              (1: the plain rule; 0: plain GS with the target amplitudes);
 *   fix_phase  1: hold every spot's phase psi_n at its value from the last
 *              update made with fix_phase = 0 (phase fixing), 0: psi_n = arg E_n.
 * The held phases live in the handle (they start at 0) and are the third part
 * of the WGS state besides (phase, w). Cached loop graphs are discarded.
 */
ash_status ash_wgs_set_options(ash_hologram *h, float feedback, int fix_phase);

/*
 * Number of kernel launches one ash_wgs_iterate call with `iters` iterations
 * enqueues (transform kernels, reductions, fix-ups, spot updates, metrics);
 * -1 on a NULL handle.
 */
int ash_wgs_launches(const ash_hologram *h, int iters);

/*
 * Kernel nodes of a graph the handle has captured and cached, counted when
 * it was captured (kernels of embedded child graphs included): key = iters
 * for the loop of ash_wgs_iterate(iters >= 2), key = -iters for that of
 * ash_cg_refine(iters >= 1). Every kernel of those calls runs inside that
 * graph. -1 if no graph is cached under key (none captured yet, or dropped
 * by ash_set_kernel_variant / ash_wgs_set_options) or h is NULL.
 */
int ash_graph_kernels(const ash_hologram *h, int key);

/*
 * Measurement helper: runs each kernel of one WGS iteration once on
 * `stream`, bracketed by CUDA events recorded on that stream, synchronises
 * it, and writes the durations in milliseconds to the host array ms_out[6]:
 *   {forward kernel, forward reduction, adjoint kernel (phase epilogue),
 *    adjoint fix-up (0 if not needed), spot update, coefficient-gradient
 *    kernel}.
 *   phase  device float[ny*nx] (forward input); y device float[2*N]
 *          (adjoint input and gradient input).
 * The handle's workspace is used; outputs are discarded.
 */
ash_status ash_profile(ash_hologram *h, const float *phase, const float *y, float *ms_out, void *stream);

/*
 * Synchronise `stream` and report device-side errors recorded by the
 * handle's kernels, clearing them: ASH_ERR_TIMEOUT if a bounded wait gave up
 * (every spin-wait of the tensor-core kernels has an iteration limit; on
 * reaching it the kernel records the timeout, stops waiting and returns, so
 * the context stays usable), ASH_ERR_DEVICE for any other recorded error.
 */
ash_status ash_hologram_check(ash_hologram *h, void *stream);

/*
 * For tests of that path: enqueue one kernel whose single bounded wait is
 * never released (a fresh mbarrier nothing arrives on). It gives up after
 * `polls` polls (1 <= polls <= 2^20) and records the timeout in the handle's
 * error word, as a transform kernel would; the next ash_hologram_check
 * returns ASH_ERR_TIMEOUT. No fault, no trap, nothing left running.
 */
ash_status ash_debug_wait_timeout(ash_hologram *h, unsigned polls, void *stream);

/* ------------------------------------------------------------------------
 * Batched uneven form: many holograms (different grids, spot counts and
 * mode counts) solved together, the whole loop one CUDA graph. Members
 * below a size threshold form the persistent group: each phase of a WGS
 * iteration (forward, reduction, spot update, adjoint, fix-up) is ONE launch
 * over the work units (hologram, tile, spot) of all of them, cut into equal
 * contiguous ranges per CTA. Larger members run their own single-hologram
 * loop inside the same graph (ash_batch_create_ex). Not in the paper (which
 * solves one hologram at a time); results equal the per-hologram path's up
 * to fp32 summation order, and bit for bit for standalone members.
 */
typedef struct ash_batch ash_batch;

/* One hologram of a batch: same meaning as the ash_hologram_create
 * arguments; 1 <= D <= 12 for the members of the persistent group (see
 * ash_batch_create_ex). */
typedef struct {
  int nx, ny;
  const float *amp;     /* device float[ny*nx] */
  int D;
  const int *noll;      /* host int[D] or NULL */
  const float *basis;   /* device float[D*ny*nx] or NULL */
  int N;
  const float *coeff;   /* device float[N*D] */
} ash_hologram_desc;

/* Create a batch of `count` holograms (descs: host array). Allocates one
 * handle workspace per hologram plus the batch's descriptor table and split
 * scratch; synchronises `stream`. Members with N * nx * ny >= 2^22 terms
 * run standalone (see ash_batch_create_ex); ASH_ERR_UNSUPPORTED if a member
 * of the persistent group has D > 12. */
ash_status ash_batch_create(ash_batch **out, int count, const ash_hologram_desc *descs, void *stream);

/* As ash_batch_create, with the standalone threshold given: a member with
 * N * nx * ny >= solo_terms runs its own single-hologram WGS loop (the
 * kernels and launch shapes ash_wgs_iterate would use) inside the batch's
 * CUDA graph; the others share the persistent launches. solo_terms = 0 makes
 * every member standalone, a value above every member's N * nx * ny none.
 * ASH_ERR_INVALID_ARG if solo_terms < 0. The grid, autotuner and resident
 * CTAs of ash_batch_info / _set_grid / _tune refer to the persistent group
 * (grid 0 when it is empty). */
ash_status ash_batch_create_ex(ash_batch **out, int count, const ash_hologram_desc *descs, long long solo_terms,
                               void *stream);

/* Number of standalone members (-1 for NULL). */
int ash_batch_standalone(const ash_batch *b);

/* Destroy (synchronises the device first); NULL is ignored. */
void ash_batch_destroy(ash_batch *b);

/* count, CTAs per transform launch, resident CTAs of the device, and the
 * total number of (hologram, tile, spot) work units; outputs may be NULL. */
ash_status ash_batch_info(const ash_batch *b, int *count, int *grid, int *resident_ctas, long long *units);

/* Override the CTA count of the transform launches (clamped to
 * [1, 4 x resident CTAs]); invalidates captured graphs. */
ash_status ash_batch_set_grid(ash_batch *b, int grid);

/* Kernel family of the batch: 0 automatic (the tensor-core transforms when
 * every hologram has tensor-core operand images with the same K-atom count,
 * else the FMA-pipe kernels), 1 FMA-pipe kernels, 2 tensor-core kernels
 * (ASH_ERR_UNSUPPORTED if not every hologram qualifies). Resets the grid to
 * the family's resident CTAs and invalidates captured graphs. */
ash_status ash_batch_set_variant(ash_batch *b, int variant);

/* Kernel launches one ash_batch_wgs call enqueues for `iters`; -1 if NULL. */
int ash_batch_wgs_launches(const ash_batch *b, int iters);

/* Kernel nodes of the graph ash_batch_wgs captured for `iters` (every
 * kernel of the call; the graph is captured on its first call with that
 * count); -1 if no such graph is cached or b is NULL. */
int ash_batch_graph_kernels(const ash_batch *b, int iters);

/*
 * Weighted GS on every hologram of the batch (same rule as
 * ash_wgs_iterate), in place on phases[i] / weights[i]:
 *   phases, weights, targets  host arrays of `count` device pointers
 *                             (float[ny_i*nx_i], float[N_i], float[N_i]).
 *   metrics_out  device float[4*count] or NULL ({uniformity, efficiency,
 *                sum |E|^2, min I^} per hologram).
 * The loop runs as one CUDA graph per iteration count (captured on first use).
 */
ash_status ash_batch_wgs(ash_batch *b, float *const *phases, float *const *weights, const float *const *targets,
                         int iters, float *metrics_out, void *stream);

/*
 * Autotuner (the batched form's "tile shapes picked by an autotuner"): for
 * each distinct grouping of the members (every member standalone; the
 * persistent group for members below 2^20, 2^22, 2^24, 2^26 terms; every
 * member the persistent kernels can take in the group) and each kernel
 * family of the persistent group (tensor-core and FMA-pipe, or only the one
 * forced with ash_batch_set_variant), it picks the group's CTA count among
 * 0.5x .. 4x the resident CTAs by timing one batched forward + adjoint, then
 * times two WGS iterations of the whole batch as the CUDA graph
 * ash_batch_wgs runs; the fastest (grouping, family, CTA count) is applied.
 * Phases: the caller's (host array of device pointers); weights and targets
 * are set to 1 for the timing, so the batch's WGS state is overwritten.
 * The choice is appended as "key solo_terms family grid" to the text file
 * cache_path (NULL: no cache); the key is the device's SM count and each
 * member's log2 pixel count, log2 spot count and mode count (rounded up),
 * plus the forced family. A cache line with this batch's key is applied
 * without timing. grid_out (host, may be NULL) receives the persistent
 * group's CTA count (0 if the choice makes every member standalone).
 * Synchronises the device.
 */
ash_status ash_batch_tune(ash_batch *b, const float *const *phases, const char *cache_path, int *grid_out,
                          void *stream);

/*
 * Allocation-free forward transform. The paper has no counterpart: this is
 * an interface for callers that cannot allocate device memory -- a host
 * framework that owns all device memory and forbids cudaMalloc once running,
 * a real-time SLM control loop that must not allocate, a plugin that only
 * receives pre-allocated buffers. Such callers cannot create a handle, so
 * every input is passed directly:
 *   E_n = sum_m amp_m exp(i phase_m) exp(-i coeff_n . basis_m)
 *   nx, ny  grid, 1 <= nx, ny <= 16384.
 *   amp, phase  device float[ny*nx] (row-major).
 *   D       1 <= D <= ASH_MAX_MODES.
 *   basis   device float[D*ny*nx], row d = Z_d over the grid (row-major).
 *   N       1 <= N <= 131072.
 *   coeff   device float[N*D] (row-major).
 *   E       device float[2*N] (complex64, 8-byte aligned), overwritten.
 * It calls no cudaMalloc, cudaFree or other allocating routine. Its split-M
 * partial sums live in a fixed 8 MiB __device__ array inside the library
 * (every GPU that loads the library holds it until the process exits); N is
 * limited so that at least one CTA's rows fit, and larger N returns
 * ASH_ERR_INVALID_ARG. All calls share that array and it keeps the last
 * call's contents (each call overwrites every row it later reads), so calls
 * whose kernels overlap on the GPU -- on different streams, or from several
 * host threads -- race; serialise them. The first call on each device does a
 * one-time set-up (it looks up the array's device address with that device
 * current); make that first call before any stream capture. Precision and
 * results match ash_forward on a handle created with the same basis, to fp32
 * rounding.
 */
ash_status ash_forward_noalloc(int nx, int ny, const float *amp, const float *phase, int D,
                               const float *basis, int N, const float *coeff, float *E,
                               void *stream);

#ifdef __cplusplus
}
#endif

#endif /* ASH_H */
