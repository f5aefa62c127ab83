/*
 * gspoisson: free-space Poisson solver on the GPU (Gaussian-sum FFT convolution).
 *
 * Solves -Laplace(u) = rho in R^3 with u -> 0 at infinity as u = U * rho,
 * U(x) = 1/(4 pi |x|) (Exl, arXiv:1612.01799, Sec. 1, eqs. problem1 and conv), for a
 * density sampled on the cube [-L, L]^3 with N cell-centred points per axis,
 * x_i = -L + (i + 1/2) * 2L/N.
 *
 * Method (Sec. 2): after scaling the box by lambda = L to [-1, 1]^3,
 *   u = lambda^2 (I_1 + I_delta),
 * where I_1 is the convolution with the Gaussian-sum kernel
 *   U_GS(y) = sum_j w_j exp(-tau_j^2 |y|^2)   (sinc quadrature, eq. approx)
 * done with zero padding to (2N)^3 and the FFT, with the symbol (the G-tensor)
 *   G_k = sum_j w_j prod_q A_j(k_q),  A_j(k) = 2 int_0^2 exp(-tau_j^2 t^2) cos(pi k t/2) dt,
 * and I_delta = C0 rho + C2 Laplace(rho) is the Taylor near-zone correction inside the
 * delta-ball (Sec. 2, last paragraph).  The correction enters the padded symbol as
 * C0 - C2 |kappa|^2 with kappa = pi k / 2, so one solve is
 *   u = lambda^2 Re IFFT_(2N)^3 [ G_tot . FFT_(2N)^3 (pad(rho)) ] cropped to N^3.
 * delta follows the Sec. 3 heuristic: min_q (b_q - a_q)/(50 n_q), at least 1e-3.
 * Setup (plan creation) is separate from the solve and a plan is reused for many
 * solves (Sec. 3 and Sec. 4: the solver object is set up once per geometry).
 *
 * Conventions for every call:
 *   - Return value: POISSON_OK (0) or a negative POISSON_ERR_* code; no call aborts
 *     the process or traps the device.  poisson_strerror() names a code.
 *   - Arrays: N^3 values, x fastest: index i + N*(j + N*k) for point (x_i, y_j, z_k).
 *   - Streams are cudaStream_t values passed as void*; NULL is the legacy default stream.
 *   - Device pointers must be device (or managed) memory of the plan's device.
 *   - A plan may be used by one stream at a time: its workspace is shared by its solves.
 */
#ifndef GSPOISSON_POISSON_H
#define GSPOISSON_POISSON_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct poisson_plan_s *poisson_plan;

/* Arithmetic of the solve.  POISSON_F32: FP32 data, FFT butterflies and symbol table;
 * twiddles and the symbol are computed in FP64 and rounded once.  POISSON_F64: FP64
 * throughout. */
typedef enum { POISSON_F32 = 0, POISSON_F64 = 1 } poisson_dtype;

enum {
    POISSON_OK = 0,
    POISSON_ERR_ARG = -1,         /* invalid argument (null pointer, N, L, tol, dtype) */
    POISSON_ERR_ALLOC = -2,       /* device or host allocation failed */
    POISSON_ERR_CUDA = -3,        /* a CUDA runtime call or kernel launch failed */
    POISSON_ERR_UNSUPPORTED = -4, /* N not in the supported set */
    POISSON_ERR_TIMEOUT = -5,     /* a bounded device-side wait gave up */
    POISSON_ERR_NUMERIC = -6      /* plan setup could not reach the requested accuracy */
};

/*
 * Create a plan: the setup phase of Sec. 3 (delta, the Gaussian sum, the per-axis
 * G-tensor factors by quadrature, C0 and C2, the symbol table, FFT twiddles) and the
 * device workspace for solves.  Runs on the current CUDA device, synchronously.
 *   out   [out] receives the plan; *out is set to NULL on failure.
 *   N     points per axis: even, 4 <= N <= 1024, with no prime factor above 5 (so that 2N
 *         factors into 2, 3 and 5), else POISSON_ERR_UNSUPPORTED; see poisson_supported_n().
 *   L     half-width of the cube [-L, L]^3, L > 0 and L < 25 N (the Sec. 3 condition
 *         lambda <= 25 min_q n_q that keeps delta inside the scaled box).
 *   tol   requested accuracy of the Gaussian sum: eps = clamp(tol/10, 1e-14, 1e-7) is
 *         the maximum relative error of U_GS on [delta, 2 sqrt(3)] (Sec. 2 and 3).
 *   dtype POISSON_F32 or POISSON_F64.
 * The plan owns its device memory; poisson_plan_destroy() frees it.
 * Kernel forms (the POISSON_KNOB_*_FORM knobs) are chosen by timing them on the first plan
 * of each (device, N, dtype) in the process.  If the environment variable
 * POISSON_TUNE_CACHE names a file, the choices persist across processes: the file is read
 * at the first plan creation, a shape found there (for a device of the same name) is not
 * timed again, and every new choice is appended (first line "gspoisson-tune 1", then one
 * line "N dtype zform yform xform xyform device-name" per choice).  Unreadable or invalid
 * lines are ignored; a missing or unwritable file only disables the persistence.
 */
int poisson_plan_create(poisson_plan *out, int N, double L, double tol, int dtype);

/*
 * A plan whose workspace holds up to max_batch densities (1 <= max_batch <= 64) of this
 * geometry, so that poisson_solve_batched solves all its entries with one launch per pass.
 * Same arguments and errors as poisson_plan_create; the workspace grows by max_batch.
 */
int poisson_plan_create_batched(poisson_plan *out, int N, double L, double tol, int dtype,
                                int max_batch);

/*
 * A plan for the rectangular box [-Lx, Lx] x [-Ly, Ly] x [-Lz, Lz] with N points on every
 * axis (spacings 2 Lx / N, 2 Ly / N, 2 Lz / N; a box off the origin gives the same grid
 * values, the potential depending only on the offsets between points).  Sec. 2's
 * standardised form: lambda = max_q L_q, scaled half-lengths l_q = L_q / lambda, one
 * G-tensor factor per axis, l_q A_j(tau_j l_q, k), kappa_q = pi k / (2 l_q) in the
 * correction, the Gaussian sum fitted on [delta, 2 |l|], delta = max(min_q 2 L_q / (50 N),
 * 1e-3) below min_q l_q (else POISSON_ERR_ARG).  The symbol is not symmetric in its three
 * indices, so the plan also keeps a copy with kz innermost for the z warp forms (the
 * table's memory counts twice in poisson_plan_info).  poisson_plan_axis_table returns the
 * x axis's factors.  Other
 * arguments, errors and use as for poisson_plan_create (one density per solve).
 */
int poisson_plan_create_box(poisson_plan *out, int N, double Lx, double Ly, double Lz, double tol, int dtype);

/*
 * A plan for the box [-Lx, Lx] x [-Ly, Ly] x [-Lz, Lz] with n_q points on axis q (Sec. 2's
 * standardised form with n_1, n_2, n_3 points per axis): spacings 2 Lx / nx, 2 Ly / ny,
 * 2 Lz / nz; each axis zero-padded to 2 n_q, so the padded period of axis q is 4 l_q and its
 * frequency k has kappa_q = pi k / (2 l_q); the G-tensor factor of axis q is
 * l_q A_j(tau_j l_q, k) for k = 0..n_q; delta = max(min_q 2 L_q / (50 n_q), 1e-3) (Sec. 3)
 * below min_q l_q (else POISSON_ERR_ARG).  Densities and potentials are nz x ny x nx
 * arrays, x fastest (index i + nx (j + ny k)).  Each n_q must be even, 4 <= n_q <= 1024,
 * with no prime factor above 5 (else POISSON_ERR_ARG or POISSON_ERR_UNSUPPORTED).  With
 * nx = ny = nz this is poisson_plan_create_box.  Plans whose counts differ (or whose common
 * count has no compiled transform schedule, poisson_supported_n() == 2) run the
 * runtime-length forms of the five passes: one form per pass (the form knobs have only
 * value 0), the same arithmetics, no TMA staging.  poisson_plan_axis_table returns the x
 * axis's factors (n_terms x (nx + 1)).  Other arguments, errors and use as for
 * poisson_plan_create (one density per solve).
 */
int poisson_plan_create_box_n(poisson_plan *out, int nx, int ny, int nz, double Lx, double Ly, double Lz,
                              double tol, int dtype);

/* Free a plan and its device memory.  NULL is accepted.  The caller must make sure no
 * solve on the plan is still running (synchronise its stream first). */
int poisson_plan_destroy(poisson_plan p);

/*
 * One solve (Sec. 2/3: I_1 by the padded FFT with the symbol, plus the near-zone
 * correction folded into the symbol), entirely on the device and stream ordered:
 * no host synchronisation and no host<->device traffic.
 *   rho_d  device pointer to N^3 values of the plan's dtype (input density).
 *   u_d    device pointer to N^3 values of the plan's dtype (output potential); may
 *          equal rho_d.
 *   stream cudaStream_t as void*.
 * The caller owns both buffers.  Launch errors are reported; errors of kernels still
 * running are reported by the next synchronising call.
 */
int poisson_solve(poisson_plan p, const void *rho_d, void *u_d, void *stream);

/*
 * The same solve on host buffers: copies rho_h to the device, solves, copies u back
 * and synchronises the stream before returning.  rho_h, u_h: host pointers to N^3
 * values of the plan's dtype (pinned memory gives full copy bandwidth).  Uses the
 * plan's own device staging buffers.  Where N is a multiple of 8 (N >= 16) and the x and y
 * passes are separate launches, the copies run in 8 z-slabs on a copy stream of the plan,
 * overlapped with the x and y passes of the neighbouring slabs (those passes transform
 * each z-plane on its own); they start after the work already queued on `stream`.  The result is the
 * same, bit for bit, as poisson_solve's on device copies of the buffers.
 */
int poisson_solve_host(poisson_plan p, const void *rho_h, void *u_h, void *stream);

/*
 * Solves of several independent densities, possibly of different N, stream ordered with
 * respect to `stream`.  plans[i], rho_d[i], u_d[i] as for poisson_solve; all plans on one
 * device; count >= 0.  Entries that share a plan are solved together, at most the plan's
 * max_batch at a time, with one launch per pass; the groups of different plans run
 * concurrently on streams forked from `stream` and joined back to it, so the call can be
 * captured into a CUDA graph (the fork streams are created with the device's first plan).
 */
int poisson_solve_batched(int count, const poisson_plan *plans, const void *const *rho_d,
                          void *const *u_d, void *stream);

/*
 * One solve as poisson_solve that also returns the a-posteriori indicator of the density's
 * resolution: eta = sqrt(E_shell / E_total), E the energy |F|^2 of the padded forward
 * spectrum of rho (all (2N)^3 frequencies, the Hermitian half counted twice) and E_shell its
 * part with max(|kx|, |ky|, |kz|) >= N - N/8.  The error of the method is driven by the
 * convergence of the density's finite Fourier series (Sec. 3); a tail that is not small
 * means N does not resolve rho.  eta: host pointer.  Synchronises `stream`.
 */
int poisson_solve_checked(poisson_plan p, const void *rho_d, void *u_d, double *eta, void *stream);

/*
 * count (1 <= count <= the plan's max_batch) checked solves of the plan's geometry with one
 * launch per pass: rho_d[i] -> u_d[i] as poisson_solve_batched, eta[i] (host array of count
 * doubles) as poisson_solve_checked for density i.  Synchronises `stream`.  The grid
 * selector's batched refinement runs on it: the densities that chose the same N solve
 * together, and those whose eta fails the check move to the next N together.
 */
int poisson_solve_checked_batched(poisson_plan p, int count, const void *const *rho_d, void *const *u_d,
                                  double *eta, void *stream);

/*
 * The final residual check: relative L2 and relative l-infinity differences of a against
 * b over n values, accumulated in FP64 on the device: rel_l2 = ||a - b||_2 / ||b||_2,
 * rel_linf = max|a - b| / max|b| (the paper's error measure E, Sec. 5, eq. error_infty).
 * a_d, b_d: device arrays of dtypes a_dtype, b_dtype (POISSON_F32 / POISSON_F64, may
 * differ); rel_l2, rel_linf: host pointers.  Synchronises `stream`; concurrent calls are
 * serialised by the library.
 */
int poisson_compare(const void *a_d, int a_dtype, const void *b_d, int b_dtype, size_t n,
                    double *rel_l2, double *rel_linf, void *stream);

/*
 * Per-pass device times of one solve, in milliseconds, measured with CUDA events
 * recorded on `stream` around each of the five passes (x forward, y forward, z
 * forward + symbol + z inverse, y inverse, x inverse).  ms[5] receives them.  With the
 * fused x-y form (POISSON_KNOB_XY_FORM = 1) the forward x and y passes are one kernel,
 * timed in ms[0] with ms[1] = 0, and the inverse y and x passes are one kernel, timed in
 * ms[3] with ms[4] = 0.  The call synchronises the stream.  Same arguments and aliasing
 * rules as poisson_solve.
 */
int poisson_solve_timed(poisson_plan p, const void *rho_d, void *u_d, void *stream, float *ms);

/*
 * Status of the plan's earlier solves: synchronises `stream` (cudaStream_t as void*),
 * reads the plan's device status word and clears it.  Returns POISSON_OK, or
 * POISSON_ERR_TIMEOUT if a bounded device-side wait of a solve gave up (its kernel
 * stopped early and its output is not valid).
 */
int poisson_last_status(poisson_plan p, void *stream);

/*
 * Test hook of the failure detection above (no counterpart in the paper): launches on
 * `stream` one device-side wait of the kind every TMA pass uses, on an mbarrier that nothing
 * completes, bounded at `polls` polls (1 <= polls <= 2^24).  The wait gives up, records the
 * timeout bit in the plan's status word and the kernel returns: no fault, no trap, no hang,
 * and the context stays usable.  The next poisson_last_status on the plan then returns
 * POISSON_ERR_TIMEOUT (and clears the word).  No solve output is touched.
 * Returns POISSON_ERR_ARG for a null plan or polls out of range.
 */
int poisson_selftest_wait(poisson_plan p, long long polls, void *stream);

/*
 * Facts of a plan, for checks and reports.  Any output pointer may be NULL.
 *   delta       near-zone radius in scaled coordinates (Sec. 3 heuristic).
 *   eps         Gaussian-sum accuracy actually requested.
 *   n_terms     S + 1, the number of Gaussian-sum terms.
 *   c0, c2      near-zone constants of I_delta = C0 rho + C2 Laplace(rho).
 *   ws_bytes    device workspace of one solve.
 *   table_bytes device bytes of the symbol table and twiddles.
 */
int poisson_plan_info(poisson_plan p, double *delta, double *eps, int *n_terms, double *c0,
                      double *c2, size_t *ws_bytes, size_t *table_bytes);

/*
 * Kernel-variant knobs of a plan.  poisson_plan_create times the variants a knob has for
 * the plan's N and dtype on the plan's own workspace and keeps the fastest; the choice is
 * cached per process, device, N and dtype, so every plan of a shape solves with the same
 * kernels (and gives bit-identical results).  Variants differ only in rounding order.
 *   POISSON_KNOB_Z_FORM  form of the fused z pass (Sec. 2, the convolution with the
 *       G-tensor along the last axis):
 *       0 = length-2N transforms, a column pair spread over the threads of a block;
 *       1 = the pruned length-2N transforms split into even- and odd-frequency length-N
 *           transforms, where the length-N schedule has fewer stages
 *           (N = 16, 80, 256, 320, 384);
 *       2 = one warp per column pair: an E1-point DFT (N = 16 E1) and a 16-point DFT in
 *           registers, a radix-2 step between lane pairs and one warp-local
 *           shared-memory exchange per direction (POISSON_F32, N = 64, 96, 128, 160,
 *           192, 256); at N = 512 one warp per column, two 32-point DFTs in registers
 *           and one warp-local exchange per direction (POISSON_F32).
 *   POISSON_KNOB_Y_FORM  form of the two y passes (Sec. 2, the zero-padded transforms
 *       along the middle axis): 0 = a column pair spread over the threads of a block;
 *       1 = one warp per column pair, as form 2 of the z pass (POISSON_F32, the same N;
 *       at N = 512 one warp per column).
 *   POISSON_KNOB_X_FORM  form of the two x passes (Sec. 2, the real transforms along the
 *       first axis and the crop): 0 = a tile of rows staged in shared memory; 1 = one
 *       half-warp (N = 64 ... 256 as for the z pass) or warp (N = 512) per pair of rows,
 *       read and written straight from device memory (POISSON_F32).
 *   POISSON_KNOB_XY_FORM  whether the x and y passes run as separate launches (0, in the
 *       forms of the two knobs above) or fused (1: one persistent kernel per direction
 *       whose row tasks (x) and column-tile tasks (y) hand each z-plane over through a
 *       ring of plane slots that stays in L2, so the x spectrum never goes to device
 *       memory; the bodies are the warp forms; POISSON_F32, N = 64, 96, 128, 160, 192,
 *       256).
 *   POISSON_KNOB_CORRECTION  where the near-field correction I_delta = C0 rho +
 *       C2 Laplace(rho) of Sec. 2 enters: 0 (the default) = in the symbol at every padded
 *       frequency, C0 - C2 |kappa|^2 (the Laplacian of the 2N-periodic series);
 *       1 = the paper's order, Laplace(rho) of the N-periodic series from an unpadded N^3
 *       transform pair; the plan gets it from the same padded transforms by placing
 *       8 (C0 - C2 |kappa|^2) at the frequencies whose three indices are all even (the
 *       N-point DFT is the padded DFT at even frequencies) and nothing elsewhere.  The two
 *       differ by terms of order C2 |kappa|^2 at high frequencies.  Setting it recomputes
 *       the plan's symbol table on its device (a temporary device allocation and a
 *       synchronisation) and is not timed; every dtype and N, every kernel form.
 *   POISSON_KNOB_ARITH  arithmetic of a POISSON_F64 plan: 0 = FP64 (the FP64 pipe);
 *       1 = double-float, each real an unevaluated sum hi + lo of two FP32 numbers (a
 *       48-bit significand, unit roundoff 2^-48 = 3.6e-15) computed on the FP32 pipe, with
 *       the workspace, twiddles and symbol table in that format and rho and u still FP64
 *       (converted where the x passes read and write them).  The forms of both are the
 *       block forms (knob value 0 or 1 of the z knob).  Timed at plan creation like the
 *       forms (the faster is kept); setting it rebuilds the plan's twiddles and symbol
 *       table on its device (temporary device memory, a synchronisation).  POISSON_F32
 *       plans have only 0.  The FP32 exponent range limits double-float to values of
 *       magnitude above about 1e-38 relative to the density's scale: smaller entries
 *       (deep in the symbol's decay) flush to zero, which is far below the FP64 path's
 *       1e-12 accuracy bar.
 * poisson_plan_get_knob stores the plan's current value in *value.
 * poisson_plan_set_knob selects a variant for this plan only (no other plan changes):
 * POISSON_ERR_ARG for an unknown knob or value, POISSON_ERR_UNSUPPORTED for a variant that
 * does not exist for the plan's N and dtype.  Not to be called while the plan has work in
 * flight.
 */
#define POISSON_KNOB_Z_FORM 0
#define POISSON_KNOB_Y_FORM 1
#define POISSON_KNOB_X_FORM 2
#define POISSON_KNOB_XY_FORM 3
#define POISSON_KNOB_CORRECTION 4
#define POISSON_KNOB_ARITH 5
int poisson_plan_get_knob(poisson_plan p, int knob, int *value);
int poisson_plan_set_knob(poisson_plan p, int knob, int value);

/* Copy the Gaussian sum of a plan: tau[j], w[j] for j < min(cap, n_terms). */
int poisson_plan_gauss_sum(poisson_plan p, double *tau, double *w, int cap);

/* Copy the per-axis G-tensor factors A_j(k), k = 0..N, row-major (n_terms x (N+1)),
 * into a[cap] (cap in doubles). */
int poisson_plan_axis_table(poisson_plan p, double *a, size_t cap);

/* How a plan with N points per axis runs: 1 in the compiled-length forms (a compiled
 * transform schedule for N and 2N: N = 4, 8, 16, 32, 48, 64, 80, 96, 128, 160, 192, 256,
 * 320, 384, 512, 1024), 2 in the runtime-length forms (every other even N in 4..1024 with
 * no prime factor above 5), 0 if N is not supported. */
int poisson_supported_n(int N);

/* Human-readable name of a return code. */
const char *poisson_strerror(int code);

/* Name of the last CUDA error behind a POISSON_ERR_CUDA or POISSON_ERR_ALLOC return on this
 * host thread ("none" if there was none). */
const char *poisson_last_cuda_error(void);

/* ---- Inputs and exact potentials for grid selection (not part of a solve) ---------- */

#define POISSON_MAX_GAUSSIANS 8

/*
 * Sample rho = sum_g q_g prod_q (2 pi s_gq^2)^(-1/2) exp(-(x_q - c_gq)^2 / (2 s_gq^2)) on the
 * cell-centred N^3 grid of [-L, L]^3 (x fastest) into out_d (device, dtype).  params (host):
 * ng <= POISSON_MAX_GAUSSIANS records (cx, cy, cz, sx, sy, sz, q).  Stream ordered.
 */
int poisson_sample_gaussians(int N, double L, int ng, const double *params, int dtype, void *out_d,
                             void *stream);

/*
 * Exact potential of the same Gaussian sum at npts grid points of the N^3 grid on
 * [-L, L]^3, in FP64: idx_d (device) holds (i, j, k) per point, out_d (device) receives u.
 * Evaluated through 1/(4 pi r) = (1/(2 pi^{3/2})) int_0^inf exp(-r^2 s^2) ds, which turns the
 * convolution with a normalised anisotropic Gaussian into a 1-D integral over s.
 */
int poisson_gaussian_potential(int N, double L, int ng, const double *params, int npts, const int *idx_d,
                               double *out_d, void *stream);

/* Relative L2 difference between u_d (N^3 grid, dtype) at the npts points idx_d and the FP64
 * reference values ref_d there, accumulated in FP64; synchronises `stream`. */
int poisson_compare_points(const void *u_d, int dtype, int N, int npts, const int *idx_d,
                           const double *ref_d, double *rel_l2, void *stream);

/* ---- Learned grid selection ------------------------------------------------------------- */

#define POISSON_FEATURES 64
#define POISSON_MAX_CANDIDATES 16

/*
 * Features of count 32^3 FP32 density samples (device, each x fastest): log10 of the
 * power spectrum averaged over 64 radial shells of |k|, relative to the mean power at
 * k = 0, clamped to [-30, 0].  feat_d: count x 64 (device).
 */
int poisson_features32(const float *sample_d, int count, float *feat_d, void *stream);

/* Parameters of the selector MLP 64 -> 64 -> 64 -> 64 -> K (ReLU hidden layers), or -1. */
int poisson_mlp_nparams(int K);

/* MLP forward for count inputs x_d (count x 64) into y_d (count x K); acts_d: null or
 * count x 3 x 64 floats that receive the hidden activations for the backward pass. */
int poisson_mlp_forward(const float *params_d, int K, const float *x_d, int count, float *y_d,
                        float *acts_d, void *stream);

/* Mean squared error over n outputs: dy_d = 2 (y - t) / n, *loss_d = mean (y - t)^2. */
int poisson_mlp_loss(const float *y_d, const float *target_d, int n, float *dy_d, float *loss_d,
                     void *stream);

/* Parameter gradients of the loss for count samples into grad_d (zeroed first). */
int poisson_mlp_backward(const float *params_d, int K, const float *x_d, const float *acts_d, int count,
                         const float *dy_d, float *grad_d, void *stream);

/* One Adam step (bias-corrected with step >= 1) on n parameters. */
int poisson_mlp_adam(float *params_d, const float *grad_d, float *m_d, float *v_d, int n, float lr,
                     float beta1, float beta2, float eps, int step, void *stream);

typedef struct poisson_selector_s *poisson_selector;

/*
 * Load a trained selector (file written by the package's training driver) with room for
 * `capacity` densities per poisson_select_n call.  Allocates device memory.
 */
int poisson_selector_load(poisson_selector *out, const char *path, int capacity);
int poisson_selector_destroy(poisson_selector s);

/*
 * Grid sizes for count densities from their 32^3 samples (device FP32): the network's
 * predicted log10 error at each candidate N; N_out[b] (host) is the smallest candidate whose
 * prediction is <= log10(tol) - margin, else the largest.  pred_out: null or host
 * count x K predictions.  Synchronises `stream` (N is a host-side shape).
 */
int poisson_select_n(poisson_selector s, const float *sample32_d, int count, double tol, int *N_out,
                     float *pred_out, void *stream);

/*
 * Slab decomposition of one solve over P ranks (one GPU each, one plan each; the paper has
 * one device, this spreads its convolution).  The x and y passes work plane by plane in z and
 * the fused z pass line by line in (kx, ky), so a rank r that owns density planes
 * [z0_r, z0_r + nz_r) and y-spectrum lines [ky0_r, ky0_r + nky_r) solves as:
 *   1. poisson_slab_forward: the x and y forward passes of its planes, into planes
 *      z0_r .. of its plan's y-spectrum buffer (buffer 0 below);
 *   2. the caller exchanges blocks: rank r sends buffer 0 [z in its planes][ky in rank s's
 *      lines] to every rank s and receives [z in s's planes][ky in its lines] into the same
 *      place of its own buffer 0 (an all-to-all);
 *   3. poisson_slab_z: the fused z pass (forward, symbol, inverse) of its lines, all z, from
 *      buffer 0 into buffer 1;
 *   4. the reverse exchange on buffer 1: it sends [z in s's planes][ky in its lines] and
 *      receives [z in its planes][ky in s's lines];
 *   5. poisson_slab_inverse: the y and x inverse passes of its planes, into u.
 * rho_slab_d / u_slab_d: device pointers to the slab's planes only (nz ny nx values of the
 * plan's dtype, x fastest).  0 <= z0, 1 <= nz, z0 + nz <= n_z; 0 <= ky0, 1 <= nky,
 * ky0 + nky <= 2 n_y; else POISSON_ERR_ARG.  Stream ordered, no host synchronisation.  The
 * z pass of a slab runs in the runtime-length form on the plan's tables (any plan, any
 * arithmetic).  Each rank's plan holds a whole workspace; the slabs divide the work, not the
 * memory.  The plan's first density only; not with work of the plan in flight.
 */
int poisson_slab_forward(poisson_plan p, const void *rho_slab_d, int z0, int nz, void *stream);
int poisson_slab_z(poisson_plan p, int ky0, int nky, void *stream);
int poisson_slab_inverse(poisson_plan p, void *u_slab_d, int z0, int nz, void *stream);

/*
 * The plan's y-spectrum buffers for the exchanges of a slab decomposition: which = 0 the
 * forward spectrum (the x and y passes write it, the z pass reads it), 1 the z pass's output.
 * *ptr receives the device pointer; layout [z < n_z][ky < 2 n_y][kx < Px] of complex values
 * (re, im of the dtype; double-float: four floats re.hi, re.lo, im.hi, im.lo); *plane_bytes
 * the bytes of one z plane, *row_bytes of one ky row (Px complex values; only kx <= n_x
 * matter).  Either size pointer may be NULL.
 */
int poisson_plan_spectrum(poisson_plan p, int which, void **ptr, size_t *plane_bytes, size_t *row_bytes);

/*
 * A solve that allocates nothing.  The paper has no counterpart: this entry point exists
 * for callers that may not allocate device memory when they solve, for example a
 * real-time loop that must not enter an allocator (an allocation can take unbounded
 * time), or a process whose device memory is reserved by a framework's caching allocator
 * (a cudaMalloc there fails, or forces the framework to give memory back).  It needs no
 * plan: the symbol table, the twiddles, the workspace and a status word live in one static
 * device array of POISSON_NOALLOC_SCRATCH_BYTES that every GPU loading this library holds
 * until exit, and the host-side setup uses fixed static host arrays.  No cudaMalloc,
 * cudaFree or other allocating routine is called.
 *   N, L, tol, dtype  as for poisson_plan_create, with N <= POISSON_NOALLOC_MAX_N;
 *                     a larger N returns POISSON_ERR_UNSUPPORTED.
 *   rho_d, u_d        device pointers to N^3 values of dtype (u_d may equal rho_d).
 *   stream            cudaStream_t as void*.
 * The first call on a device looks up the array's device address and clears its status
 * word; the first call with a given (N, L, tol, dtype) on a device (and the next one after
 * a call with other parameters) also computes the tables on the host, copies them into the
 * array and synchronises `stream`.  Make those set-up calls before any stream capture.
 * Later calls with the same parameters only launch the five solve kernels, stream ordered.
 * The near-field correction is the fused placement (POISSON_KNOB_CORRECTION = 0); the
 * kernel forms are the block forms (knob value 0 of each form knob).
 * All calls share the array and it keeps the last call's contents.  Only the status word
 * must start at zero (the first call on a device clears it, poisson_noalloc_last_status
 * clears it after reading); the tables and workspace need no clearing, since each pass
 * writes every element the next one reads.  Calls that overlap on the GPU (on different
 * streams, or from different threads) race on the array; serialise them.
 * A bounded device-side wait that gives up during such a solve sets the status word, and
 * the returned code (launch errors only) cannot show it: read it with
 * poisson_noalloc_last_status after the solve.
 */
#define POISSON_NOALLOC_MAX_N 64
#define POISSON_NOALLOC_SCRATCH_BYTES (32u << 20)
int poisson_solve_noalloc(int N, double L, double tol, int dtype, const void *rho_d, void *u_d,
                          void *stream);

/*
 * The status word of the allocation-free solves on the current device: POISSON_OK, or
 * POISSON_ERR_TIMEOUT if a bounded device-side wait of one of them gave up since the last
 * read (its result is then undefined).  A non-zero word is cleared.  Synchronises `stream`
 * (order it after the solves it reports on).  Allocates nothing.
 */
int poisson_noalloc_last_status(void *stream);

/*
 * Test hook: one bounded device-side wait that nothing completes, on the allocation-free
 * solves' status word, giving up after `polls` polls (1 <= polls <= 2^24, else
 * POISSON_ERR_ARG) so that poisson_noalloc_last_status then reports POISSON_ERR_TIMEOUT.
 * No fault, trap or hang.  Allocates nothing.
 */
int poisson_noalloc_selftest_wait(long long polls, void *stream);

/*
 * The bounds-check flags of the debug build (libgspoisson_debug.so, the same sources
 * compiled with GSP_DEBUG): in that build every shared-memory access of the pass kernels'
 * access helpers is checked against the CTA's dynamic shared memory and the
 * runtime-length forms check their computed row and symbol indices; an access that fails
 * is skipped (a load yields zero; no trap) and sets a bit of a device-wide word.
 *   flags   out: that word, bit 0 a shared-memory access out of bounds, bit 1 a global
 *           index out of bounds (0: no violation since the last read), then cleared.
 *   stream  synchronised before the read (order it after the solves it reports on).
 * Returns POISSON_OK, or POISSON_ERR_UNSUPPORTED in the release build (flags set to 0),
 * POISSON_ERR_ARG for a null flags pointer, POISSON_ERR_CUDA if the read fails.
 */
int poisson_debug_flags(unsigned int *flags, void *stream);

/*
 * Test hook of the debug build: one single-thread kernel evaluates the bounds checks on
 * an address inside its dynamic shared memory (must pass), on one past its end and on the
 * index -1 of a 10-element array (both must fail); the failing checks only set their
 * flag bits (1 and 2), no access is made.  Read the result with poisson_debug_flags.
 * Returns POISSON_ERR_UNSUPPORTED in the release build (nothing launched).
 */
int poisson_debug_selftest(void *stream);

#ifdef __cplusplus
}
#endif

#endif /* GSPOISSON_POISSON_H */
