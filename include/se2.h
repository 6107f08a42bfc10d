/*
 * se2.h -- C ABI of the GB300 (sm_103a) library for fast SE(2) convolutions
 * on the coset space Z^2\SE(2) (arXiv 2504.05149).
 *
 * The operation.  For f on Z^2\SE(2) and a kernel rho radial in translations,
 * the SE(2) convolution reduces to an abelian 3-D periodic convolution
 * (Theorem f*gP, Section 5.1), and its convolutional finite Fourier series on
 * the sampling grid Omega_L (Eq. OmL) is, at output grid N = L (Section 6.1,
 * closed form below Eq. MatSKfgonG; Algorithm 3):
 *
 *     out = iDFT( W . DFT(F) . C ),      C = DFT(P) / |L|,
 *
 * with F, P the samples of f and rho, W(k) = (-1)^(k1+k2) (Eq. W), |L| = N*N*M,
 * and DFT / iDFT as in Eqs. 3DFT / 3iDFT.  A chain of k kernels uses
 * W^k . DFT(F) . C_1 ... C_k (Eq. MatSqKfgG; Algorithms 4 and 6).
 *
 * Layout (all row-major, x fastest):
 *   real grid   [M][N][N]        = [theta_l][y_j][x_i], x_i = -1/2 + i/N,
 *                                  y_j = -1/2 + j/N, theta_l = 2 pi l / M
 *   spectrum    [M][N][N/2+1]    complex, interleaved (re, im); bins 0..N/2
 *                                  along x (the rest is the Hermitian mirror),
 *                                  all bins along y and theta.
 *   A batch of B problems is B such arrays back to back.
 *   Real type: double for SE2_F64, float for SE2_F32; complex = 2 of those.
 *
 * Sizes: N in {8, 16, ..., 512}, M in {2, 4, ..., 128} (powers of two), B >= 1.
 *
 * Ownership and streams.  The caller owns every data buffer (device memory,
 * e.g. from PyTorch).  A plan owns only its twiddle tables, its scratch
 * workspace and (with SE2_HOST_STAGING) the staging of se2_convolve_host, all
 * allocated in se2_plan_create; no call below allocates (grid plans: likewise
 * in se2_grid_plan_create).  Every compute call is asynchronous on the
 * caller's CUDA stream (`stream` is a cudaStream_t; NULL = legacy default
 * stream).
 *
 * Errors.  Every call returns an se2_status and never aborts or traps.
 * Argument errors are found on the host before anything is launched.
 * se2_last_error() returns a thread-local description of the last failure.
 */
#ifndef SE2_H
#define SE2_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct se2_plan_s* se2_plan_t;

typedef enum {
    SE2_OK = 0,
    SE2_ERR_INVALID_ARG = 1,  /* null/misaligned pointer, bad size, bad count */
    SE2_ERR_UNSUPPORTED = 2,  /* valid but not implemented (size, precision)  */
    SE2_ERR_OOM = 3,          /* plan allocation failed (nothing leaked)      */
    SE2_ERR_CUDA = 4,         /* a CUDA runtime call or launch failed         */
    SE2_ERR_TIMEOUT = 5,      /* a bounded device-side wait gave up           */
    SE2_ERR_NUMERIC = 6       /* non-finite output (flag SE2_CHECK_FINITE)    */
} se2_status;

typedef enum {
    SE2_F64 = 0,              /* double storage and arithmetic                */
    SE2_F32 = 1,              /* float storage and arithmetic, FP64 tables    */
    SE2_SPLIT_BF16 = 2,       /* float storage; the angular DFT (M = 64, 128)
                                 runs on the tensor cores with bf16 hi + lo
                                 operands (3 products), FP32 accumulation      */
    SE2_BF16 = 3,             /* as SE2_SPLIT_BF16 with one bf16 product      */
    SE2_SPLIT_F16 = 4         /* as SE2_SPLIT_BF16 with fp16 hi + lo operands;
                                 each line scaled by a power of two into the
                                 fp16 range first (about 22 bits kept)        */
} se2_precision;

/* Plan flags */
#define SE2_SHARED_KERNEL 0x1u  /* one coefficient array serves the whole batch */
#define SE2_PERSISTENT    0x2u  /* FP32: run se2_convolve(_chain) as one persistent dataflow kernel */
/* Grids (f, kernel samples, output) sampled at x_i = i/N instead of on
 * Omega_L (x_i = -1/2 + i/N, Eq. OmL), theta unchanged.  The rectangle rule of
 * the convolution is then the plain cyclic convolution
 *   out[n] = (1/|L|) sum_m F[m] P[n - m],
 * i.e. the scheme without the weight W of Eq. W (which undoes the -1/2
 * offset): convolutions, chains, separable chains and the adjoint drop W, and
 * the kernel samplers (se2_sample_radial_gaussian, se2_separable_tables)
 * sample at x_i = i/N.  se2_coeffs is unaffected (C = DFT(P)/|L| either way). */
#define SE2_GRID_ORIGIN_ZERO 0x4u
/* Mass renormalisation in FP64 (se2_convolve and se2_convolve_chain): the
 * total mass of each output, sum(out), is set to its exact value
 * sum(f) * C_1[0] ... C_k[0] * exp(sum of the log-scales) (the DC bin of the
 * product, Eq. MatSqKfgG; W = 1 there) by adding the difference, spread
 * evenly, to every sample; the rounding residual of each stored sample is
 * carried to the next one, so the stored samples keep the mass to about
 * 1e-10 relative.  Both sums are taken in FP64 on the device.  Costs one
 * extra read of f and a read-modify-write of out. */
#define SE2_MASS_RENORM   0x8u
/* The kernel spectra are mirror-symmetric in y, C(kt, ky, kx) = C(kt, N - ky, kx),
 * as for every kernel radial in translations sampled on Omega_L (or at
 * x_i = i/N): y_j -> -y_j maps the grid to itself.  The FP32 fast path of
 * se2_convolve, se2_convolve_chain and se2_convolve_chain_all then reads only
 * the rows ky <= N/2 of each coefficient array, about half of its bytes; the
 * other paths read all rows.  Results for kernels without the symmetry are
 * undefined. */
#define SE2_KERNEL_YSYM   0x10u
/* se2_convolve_host staging: three groups of f and out in device memory and
 * two copy streams, allocated by se2_plan_create; se2_convolve_host needs a
 * plan with this flag. */
#define SE2_HOST_STAGING  0x20u
/* Output check: after each se2_convolve / se2_convolve_chain /
 * se2_convolve_chain_all / se2_convolve_separable / se2_backward call, one
 * extra read of the output looks for NaN or infinity; if it finds one, the
 * plan's error word records it and se2_plan_status returns SE2_ERR_NUMERIC. */
#define SE2_CHECK_FINITE  0x40u

/*
 * se2_plan_create -- validate sizes, build FP64-accurate twiddle tables and
 * allocate the scratch workspace for batches of up to `batch` problems.
 *   plan   out: the new plan (NULL on failure)
 *   N, M   grid sizes (see above); batch >= 1
 *   device the CUDA device the plan and every buffer given to it live on
 * Synchronous.  Returns SE2_ERR_OOM if device memory runs out.
 */
se2_status se2_plan_create(se2_plan_t* plan, int N, int M, int batch,
                           se2_precision precision, unsigned flags, int device);

/* Frees the plan's tables and workspace (synchronises the device first). */
se2_status se2_plan_destroy(se2_plan_t plan);

/* Bytes of device workspace the plan holds (tables + scratch). */
size_t se2_plan_workspace_bytes(se2_plan_t plan);

/*
 * se2_coeffs -- scaled kernel spectra C = DFT(P) / |L| of n kernels
 * (Section 4.1, Eq. FkLv: C is W times the finite Fourier coefficients of
 * the kernel), for Algorithms 3, 4 and 6.
 *   samples   device, [n][M][N][N] real: P sampled on Omega_L
 *   n         number of kernels, >= 1 (processed in chunks of `batch`)
 *   coeffs    device, [n][M][N][N/2+1] complex, written
 *   log_scale device, [n] double, or NULL.  If non-NULL, coeffs are stored
 *             divided by s = mean(|P|) (so |C| <= 1) and log_scale[i] = ln s;
 *             s = 0 stores C unscaled and log_scale = 0.  Convolution calls
 *             multiply the result back by exp(sum of the log scales) in FP64,
 *             which keeps long chains inside the range of the real type.
 */
se2_status se2_coeffs(se2_plan_t plan, const void* samples, int n, void* coeffs,
                      double* log_scale, void* stream);

/*
 * se2_convolve -- S_K[f, rho] on Omega_L for a batch (Algorithm 3 at N = L):
 *   out_b = iDFT( W . DFT(F_b) . C_b ) * exp(log_scale_b)
 *   f         device, [B][M][N][N] real, B <= plan batch
 *   B         number of problems in this call
 *   coeffs    device, [B][M][N][N/2+1] complex (from se2_coeffs), or one
 *             [M][N][N/2+1] array for all problems with SE2_SHARED_KERNEL
 *   log_scale device, [B] (or [1]) double, or NULL (= 0)
 *   out       device, [B][M][N][N] real; may not alias f or coeffs
 */
se2_status se2_convolve(se2_plan_t plan, const void* f, int B, const void* coeffs,
                        const double* log_scale, void* out, void* stream);

/*
 * se2_convolve_chain -- f * rho_1 * ... * rho_k (Eq. MatSqKfgG with the
 * Hadamard power replaced by the product of k coefficient arrays; with k
 * equal kernels this is Algorithm 4, and the result equals the last V_k of
 * Algorithm 6):
 *   out_b = iDFT( W^k . DFT(F_b) . C_1,b ... C_k,b ) * exp(sum_i log_scale_i,b)
 *   coeffs     host array of k device pointers, each laid out as in se2_convolve
 *   log_scales host array of k device pointers ([B] or [1] doubles), or NULL;
 *              individual entries may be NULL
 *   k          1 <= k <= 32
 */
se2_status se2_convolve_chain(se2_plan_t plan, const void* f, int B,
                              const void* const* coeffs, const double* const* log_scales,
                              int k, void* out, void* stream);

/*
 * se2_convolve_chain_all -- every intermediate result of a chain (Algorithm 6,
 * the fast recursion): V_p = f * rho_1 * ... * rho_p for p = 1..k from one
 * forward transform, V_p = iDFT(W^p . DFT(f) . C_1 ... C_p) exp(ls_1 + ... + ls_p).
 * Arguments as se2_convolve_chain; out is [k][B][M][N][N] (V_p at p - 1).
 * On the FP32 fast path (N in {32, 64, 128, 256}) B runs in groups of half
 * the plan's scratch slots (the running product and its inverse y transform
 * live side by side).  Other plans (FP64, N = 512, tensor-core precisions)
 * compute each V_p as its own chain of the first p kernels.
 */
se2_status se2_convolve_chain_all(se2_plan_t plan, const void* f, int B, const void* const* coeffs,
                                  const double* const* log_scales, int k, void* out, void* stream);

/*
 * se2_backward -- adjoint of se2_convolve (not in the paper; derived from it):
 * for a loss with gradient G_b = dLoss/dout_b of out_b = iDFT(W . DFT(F_b) . C_b)
 * * exp(ls_b),
 *   grad_f_b  = iDFT( W . conj(C_b) . DFT(G_b) ) * exp(ls_b)     (a correlation)
 *   grad_params[i] += sum_b (1/|L|) sum_k W(k) dC_i,b(k) conj(DFT(G_b)(k)) DFT(F_b)(k)
 * (the sum over all bins, real; evaluated on the half spectrum with weights 1
 * at x bins 0 and N/2, 2 elsewhere).
 *   grad_out     device, [B][M][N][N] real (G)
 *   f            device, [B][M][N][N] real (needed when n_params > 0)
 *   coeffs, log_scale  as in se2_convolve (single kernel)
 *   n_params     0..4 kernel parameters
 *   dcoeffs      host array of n_params device pointers: DFT(dP/dp_i)/|L|, the
 *                derivative of the effective kernel spectrum exp(ls) C (use
 *                se2_coeffs without log_scale on the sampled derivative), laid
 *                out like coeffs
 *   grad_params  device, [n_params] double, ACCUMULATED (zero it first)
 *   grad_f       device, [B][M][N][N] real, or NULL (parameters only)
 */
se2_status se2_backward(se2_plan_t plan, const void* grad_out, const void* f, int B,
                        const void* coeffs, const double* log_scale, int n_params,
                        const void* const* dcoeffs, double* grad_params, void* grad_f,
                        void* stream);

/*
 * se2_sample_radial_gaussian -- the radial kernel family used for
 * differentiation, sampled on Omega_L: a Gaussian of width sigma in x
 * (normalised over R^2, periodised over Z^2) times 2 pi times a wrapped normal
 * of width sigma_theta centred at nu (unit mass under the Haar measure Eq. dg),
 * the radial Gaussians of Section 6.2.  Writes [M][N][N] arrays of the plan's
 * real type: P and its derivatives in sigma and sigma_theta (any may be NULL).
 * The 1-D factors are evaluated in FP64.
 */
se2_status se2_sample_radial_gaussian(se2_plan_t plan, double sigma, double sigma_theta, double nu,
                                      void* P, void* dP_dsigma, void* dP_dsigma_theta, void* stream);

/*
 * se2_sample_se2_gaussian -- the Gaussian on SE(2) with mean beta and
 * covariance Sigma (Section 5, Eq. fbS):
 *   f(g) = exp(-1/2 w^T Sigma^-1 w),  w = log(beta^-1 o g)^v = (v1, v2, phi),
 * with log the principal matrix logarithm of the matrices of Eq. gxyt (phi in
 * (-pi, pi]; +pi at the branch point) and ^v the identification se(2) -> R^3.
 * The kernel rho of Eq. gbS0 shifted by nu in the rotations (the paper's chain
 * experiments) is beta = {0, 0, nu}, Sigma = sigma^2 I.
 *   beta:   host, 3 doubles {b1, b2, nu}: beta = (b, R_nu).
 *   Sigma:  host, 9 doubles, row major, symmetric positive definite.
 *   images: 0..8; the samples sum the left translates by lattice vectors
 *           |n1|, |n2| <= images (0 samples the function on the grid as it is).
 *   P:      device, [M][N][N] of the plan's real type, on the plan's grid
 *           (Omega_L, or x_i = i/N with SE2_GRID_ORIGIN_ZERO).
 * Evaluated in FP64, rounded once.  Errors: SE2_ERR_INVALID_ARG for NULL or
 * misaligned pointers, a Sigma that is not symmetric positive definite, or
 * images out of range.
 */
se2_status se2_sample_se2_gaussian(se2_plan_t plan, const double* beta, const double* Sigma, int images, void* P,
                                   void* stream);

/*
 * se2_sample_deformed_gaussian -- the 3D deformed Gaussian of Eq. fHsnu,
 *   f(x, R_theta) = exp(-x^T H x) exp(-(theta - nu)^2 / s),
 * with theta the grid angle 2 pi l / M in [0, 2 pi) as printed (no wrapping).
 *   H: host, 4 doubles, row major 2x2; only its symmetric part enters and it
 *      must be positive definite.  s > 0.
 *   images, P, errors: as se2_sample_se2_gaussian.
 */
se2_status se2_sample_deformed_gaussian(se2_plan_t plan, const double* H, double nu, double s, int images, void* P,
                                        void* stream);

/*
 * se2_separable_tables -- coefficients of a chain of separable radial kernels
 * in factored form.  The kernel family of se2_sample_radial_gaussian is a
 * product of 1-D factors, so its C = DFT(P)/|L| is tt (x) ty (x) tx, and the
 * product over a chain (Eq. MatSqKfgG) stays factored.  For problem b with
 * k[b] kernels whose (sigma, sigma_theta, nu) are params[b][j][0..2] (j <
 * k[b], array [B][kmax][3]), writes tables[b] = [tx (N/2+1) | ty (N) | tt (M)]
 * complex (FP64 sampling and DFTs, rounded to the plan's type), with the
 * extra W^(k-1) folded into tx and ty so that se2_convolve_separable applies
 * W once.  params, k, tables: device memory.
 */
se2_status se2_separable_tables(se2_plan_t plan, const double* params, const int* k, int kmax, int B,
                                void* tables, void* stream);

/*
 * se2_convolve_separable -- se2_convolve with the coefficient array given by
 * factored tables (se2_separable_tables): the multiply step reads N/2+1+N+M
 * complex numbers per problem instead of M*N*(N/2+1), so a convolution moves
 * 8 bytes per grid point (read f, write out) in FP32.
 *   tables  device, [B][N/2+1+N+M] complex ([1][...] with SE2_SHARED_KERNEL)
 */
se2_status se2_convolve_separable(se2_plan_t plan, const void* f, int B, const void* tables, void* out,
                                  void* stream);

/*
 * Batch plans: many independent problems of uneven sizes (Algorithm 3 for
 * each problem, or Algorithm 4 / Eq. MatSqKfgG with a chain of separable
 * radial kernels in factored form, as se2_convolve_separable).
 *
 * se2_batch_plan_create -- a plan over n_problems problems, problem i on an
 * N x N x M grid given by shapes[i] (host array; each N, M as for
 * se2_plan_create).  Problems are grouped into size classes (equal (N, M)),
 * ordered by total work, largest first; each class gets its own plan, whose
 * scratch holds at most 512 MiB of problems at a time.  flags: 0,
 * SE2_GRID_ORIGIN_ZERO, SE2_CHECK_FINITE.  Synchronous.  Errors: as
 * se2_plan_create.
 *
 * Packed layout.  All grids of the batch live in one array and all tables in
 * another, class by class in class order and, inside a class, in the order of
 * `shapes`.  se2_batch_plan_layout returns, per problem (host arrays of
 * n_problems, each may be NULL): its position in that order, the offset of
 * its grid ([M][N][N] real elements) and of its tables (N/2+1+N+M complex
 * elements), and the two totals.  params and k of se2_batch_separable_tables
 * are indexed by position.
 *
 * se2_batch_separable_tables -- se2_separable_tables for every class:
 *   params  device, [n][kmax][3] double (sigma, sigma_theta, nu), by position
 *   k       device, [n] int, chain lengths 1..kmax, by position
 *   tables  device, the packed tables (written)
 * se2_batch_convolve_separable -- the convolution of every problem: f and out
 * the packed grids (device, must not overlap), tables the packed tables.
 * The classes run on `lanes` stream lanes: lane 0 is `stream`, the others
 * are plan-owned streams forked from it and joined back into it (events
 * only), so the call can be captured in a CUDA graph.  A new plan has one
 * lane (the classes one after another).
 *
 * se2_batch_tune -- the autotuner: for each class, time the candidate
 * schedules (`reps` calls each, on the given data, on `stream`) and keep the
 * fastest: FP32 fast path with pipeline depth 1 or depth 2 with groups of
 * 1, 2, 4, .. 64 problems, or the persistent dataflow kernel.  Then time the
 * whole batch on 1, 2, 3, 4 and n_classes lanes and keep the fastest, then
 * the one-launch kernel (below), kept if faster still.
 * Synchronous; not for stream capture.  se2_batch_plan_config reports per
 * class (host arrays of n_classes, each may be NULL): shape, count, pipeline
 * depth (0 for the persistent kernel), group, persistent (0/1) and the tuned
 * ms per call.
 *
 * se2_batch_plan_lanes -- set the number of lanes (lanes >= 1, clamped to
 * n_classes; classes are assigned longest first to the least-loaded lane,
 * by tuned ms once tuned, by grid points before) or, with lanes <= 0, leave
 * it.  Returns, each output may be NULL: *current, the lanes in force;
 * lane_of_class[n_classes]; lane_ms[n_classes], entry L - 1 the tuner's
 * whole-batch ms on L lanes (0 where not timed).  Host only.
 * se2_batch_plan_launches: kernels launched through the plan so far.
 *
 * se2_batch_plan_one_launch -- the whole batch as one persistent kernel: every
 * unit (x+theta pass, y pass, inverse theta+x pass) of every problem of every
 * class in one launch, ordered by a work list built at enabling (classes
 * largest first, each a pipeline of problems with per-problem completion
 * counters and a ring of scratch slots), after one memset of the counters.
 * FP32; classes N in {32, 64, 128, 256} x M in {16, 32, 64}, at most 16
 * classes and 65535 problems per class (else SE2_ERR_UNSUPPORTED).
 * mode 1 enables it (allocating its work list and scratch: not a convolve
 * call), 0 disables it, -1 leaves it; *current receives 1 if in force,
 * *tuned_ms the tuner's time for it (0 if not timed).  The tuner enables it
 * only when it beats the best lane schedule.  Every wait of the kernel is
 * bounded; one that gives up makes se2_batch_plan_status return
 * SE2_ERR_TIMEOUT.
 *
 * se2_batch_plan_status -- synchronises `stream`, then reports (and clears) a
 * timed-out wait of the one-launch kernel, then each class plan's status.
 *
 * se2_debug_batch_wait_timeout -- test hook: runs the one-launch kernel on the
 * given buffers with every y-pass wait asking for one unit more than exists,
 * so each such wait gives up after 4096 polls; the next
 * se2_batch_plan_status returns SE2_ERR_TIMEOUT and the plan stays usable.
 * out is overwritten with partial results.  Asynchronous on `stream`.
 *
 * se2_debug_batch_work_list -- the one-launch kernel's work list for classes
 * shapes[c] with counts[c] problems (in plan order) and `grid` resident
 * blocks, on the host (no device): with units == NULL, *n_units receives the
 * length; else units (host, *n_units entries) receives the codes, class << 28
 * | stage << 26 | block << 16 | problem in class (stage 0 x+theta, 1 y,
 * 2 inverse theta+x).  slots[c], lag[c] (each may be NULL) receive the ring
 * size D and lag L of each class.  For tests of the schedule.
 */
typedef struct { int N, M; } se2_shape;
typedef struct se2_batch_plan_s* se2_batch_plan_t;
se2_status se2_batch_plan_create(se2_batch_plan_t* plan, const se2_shape* shapes, int n_problems,
                                 se2_precision precision, unsigned flags, int device);
se2_status se2_batch_plan_destroy(se2_batch_plan_t plan);
se2_status se2_batch_plan_layout(se2_batch_plan_t plan, int* position, long long* grid_offset, long long* table_offset,
                                 long long* grid_total, long long* table_total);
se2_status se2_batch_separable_tables(se2_batch_plan_t plan, const double* params, const int* k, int kmax, void* tables,
                                      void* stream);
se2_status se2_batch_convolve_separable(se2_batch_plan_t plan, const void* f, const void* tables, void* out, void* stream);
se2_status se2_batch_tune(se2_batch_plan_t plan, const void* f, const void* tables, void* out, int reps, void* stream);
se2_status se2_batch_plan_config(se2_batch_plan_t plan, int* n_classes, se2_shape* shape, int* count, int* depth,
                                 int* group, int* persistent, double* tuned_ms);
se2_status se2_batch_plan_lanes(se2_batch_plan_t plan, int lanes, int* current, int* lane_of_class, double* lane_ms);
se2_status se2_batch_plan_one_launch(se2_batch_plan_t plan, int mode, int* current, double* tuned_ms);
se2_status se2_batch_plan_status(se2_batch_plan_t plan, void* stream);
se2_status se2_debug_batch_wait_timeout(se2_batch_plan_t plan, const void* f, const void* tables, void* out,
                                        void* stream);
se2_status se2_debug_batch_work_list(const se2_shape* shapes, const int* counts, int n_classes, int grid,
                                     unsigned* units, long long* n_units, int* slots, int* lag);
unsigned long long se2_batch_plan_launches(se2_batch_plan_t plan);

/*
 * se2_plan_launches -- the number of kernels the plan's entry points have
 * launched so far (host-side count, updated as launches are enqueued; plan
 * creation's own set-up launches are not counted).  0 for a NULL plan.
 * Lets a caller state how many kernels a call or a timed loop ran.  The paper
 * has no counterpart.
 */
unsigned long long se2_plan_launches(se2_plan_t plan);

/*
 * se2_plan_timing / se2_plan_timing_read -- per-launch durations of the FP32
 * fast path's kernels (0: forward x and theta transforms, kf_fwd_xt /
 * kf2_fwd_xt; 1: y pass with the product, kf_lines; 2: inverse theta and x
 * transforms, kf_inv_tx / kf2_inv_tx; 3: the whole-batch dataflow kernel
 * kflow_conv, which runs all three units).  With timing on, each launch is
 * bracketed by CUDA events recorded on the stream it runs on (the pipeline's
 * own streams included); se2_plan_timing(plan, 1) also clears what was
 * recorded.  _read waits for the recorded events and returns, per kind, the
 * summed milliseconds ms[4] and the launch counts count[4] (host arrays).
 * Not for use while a stream is being captured into a CUDA graph.  Up to
 * 32768 launches are recorded.
 */
se2_status se2_plan_timing(se2_plan_t plan, int on);
se2_status se2_plan_timing_read(se2_plan_t plan, double* ms, long long* count);

/*
 * se2_plan_status -- synchronise `stream`, then report and clear the plan's
 * device error word.  The persistent convolution kernel waits on counters
 * that other blocks of the same launch update and the tensor-core DFT on
 * its matrix products; each wait is bounded (about a second).  A wait that
 * gives up sets the error word, the kernel stops, and the call's output is
 * undefined.  Returns
 * SE2_ERR_TIMEOUT in that case, SE2_OK otherwise.  Until it is read, later
 * launches of the persistent kernel also stop at once.
 */
se2_status se2_plan_status(se2_plan_t plan, void* stream);

/*
 * se2_debug_wait_timeout -- test hook for the bounded-wait path: launches the
 * persistent kernel on one problem (f, coeffs, out as in se2_convolve) with a
 * dependency that is never met, so that its wait runs out after a few
 * thousand polls.  Afterwards se2_plan_status returns SE2_ERR_TIMEOUT.
 * SE2_ERR_UNSUPPORTED if the plan does not use the persistent kernel.
 */
se2_status se2_debug_wait_timeout(se2_plan_t plan, const void* f, const void* coeffs, void* out,
                                  void* stream);

/*
 * se2_convolve_host -- se2_convolve with f and out in HOST memory.  The batch
 * goes through device staging buffers owned by the plan in groups of
 * problems; the copy of one group to the device, the convolution of the
 * previous group and the copy of the one before back to the host run on
 * separate streams and overlap.  The paper has no counterpart: this is a
 * deployment variant of Algorithm 3 at N = L for data that lives on the host.
 *   f          host, [B][M][N][N] (float, or double for SE2_F64 plans);
 *              page-locked memory (cudaHostAlloc / cudaHostRegister) lets
 *              the copies run asynchronously, pageable memory works but the
 *              copies then serialise with the host
 *   coeffs     device, as in se2_convolve
 *   log_scale  device or NULL, as in se2_convolve
 *   out        host, [B][M][N][N], must not overlap f
 *   stream     the call is ordered after earlier work on `stream`; on
 *              return all of its work is enqueued and `stream` waits for it,
 *              so synchronise `stream` before reading out
 * The plan must have been created with SE2_HOST_STAGING (SE2_ERR_INVALID_ARG
 * otherwise): its staging buffers (three groups of f and out) and copy
 * streams come from se2_plan_create, and this call allocates nothing.
 * Not for stream capture.  Errors: as se2_convolve.
 */
se2_status se2_convolve_host(se2_plan_t plan, const void* f, int B, const void* coeffs, const double* log_scale,
                             void* out, void* stream);

/*
 * se2_convolve_noalloc -- the same result as se2_convolve (FP32, one kernel
 * spectrum per problem, no log scale) for callers that cannot create a plan
 * because creating one allocates device memory: for instance code running
 * inside a host framework's execution step where device allocation is not
 * allowed, or code that must not risk the implicit synchronisation that
 * cudaMalloc / cudaFree may cause.  The paper has no counterpart.
 *   f, coeffs, out  as in se2_convolve (float / complex float, caller-owned)
 *   N, M, B         sizes; the batch is processed in chunks that fit
 * Memory: the call uses a fixed 64 MiB device array defined in the library
 * (twiddle tables + scratch), present on every GPU that loads the library
 * until the process exits; it calls no cudaMalloc, cudaFree or other
 * allocating routine.  A problem whose scratch exceeds the array (e.g.
 * N = 512 with M = 128) is rejected with SE2_ERR_UNSUPPORTED.
 * The first call on a device sets the device up (looks up the array's
 * device address, writes the twiddle tables, synchronises the device once);
 * make that first call before any stream capture.  All calls share the one
 * array, so calls that may overlap on the GPU (different streams, or other
 * threads) race and must be serialised by the caller.  Nothing in the array
 * needs to start at zero.  Errors: as the other calls (se2_last_error()).
 */
se2_status se2_convolve_noalloc(const void* f, const void* coeffs, void* out, int N, int M, int B,
                                void* stream);

/*
 * Allocation accounting (tests and diagnostics).  Every device allocation the
 * library makes (plans, grid plans, host-call staging) goes through one
 * counter:
 *   se2_debug_alloc_stats -- live: allocations not yet freed; total: all made.
 *   se2_debug_fail_alloc  -- make the n-th next allocation fail as if device
 *                            memory had run out (n = 0: off).  The call that
 *                            meets it returns SE2_ERR_OOM and frees what it had
 *                            allocated.  Process-wide.
 * Host arrays; never fail except on NULL / negative arguments.
 */
se2_status se2_debug_alloc_stats(long long* live, long long* total);
se2_status se2_debug_fail_alloc(long long n);

/* Thread-local text of the last error (never NULL). */
/*
 * Odd sampling grids and upsampled output (Section 4.2, Eq. MatSKfonG and
 * Algorithm SKLAlg; Section 6.1, Eqs. Qf, W, MatSKfgonG).
 *
 * A grid plan samples on Omega_L with L = (Lx, Ly, Lr) = 2K + 1 per axis
 * (x_i = -1/2 + i/Lx, y_j = -1/2 + j/Ly, theta_l = 2 pi l / Lr) and evaluates
 * the convolutional finite Fourier series
 *   S_K[f, rho_1..rho_k](w) = sum_{|k| <= K} f^[k;L] rho_1^[k;L] .. rho_k^[k;L] phi_k(w)
 * on the N-grid (x'_n = -1/2 + n/Nx, y'_m = -1/2 + m/Ny, theta'_l = 2 pi l / Nr),
 * N >= L per axis.  With k = 0 the result is S_K[f] itself (the finite
 * Fourier series of f on the N-grid).  N = L gives the plain scheme on an odd
 * grid.  Arrays are x fastest: samples [n][Lr][Ly][Lx] and outputs
 * [B][Nr][Ny][Nx] of the plan's real type; coefficients [n][Lr][Ly][Kx+1]
 * complex (DFT bins; kx = 0..Kx, the rest follows from Hermitian symmetry).
 * The kernels must be radial in translations for S_K[f, rho] to approximate
 * f * rho (Theorem f*gP); the series itself is computed for any input.
 */
typedef struct se2_grid_plan_s* se2_grid_plan_t;

/*
 * se2_grid_plan_create -- L: host int[3] {Lx, Ly, Lr}, each odd in [1, 255];
 * N: host int[3] {Nx, Ny, Nr} with L <= N <= 1024 per axis; batch >= 1;
 * precision SE2_F32 or SE2_F64; flags 0 or SE2_SHARED_KERNEL (one coefficient
 * array per kernel for the whole batch).  Allocates the DFT tables (FP64
 * sincospi, rounded) and 2 * batch * Nr * Ny * (Kx+1) + batch * Lr * Ly * (Kx+1)
 * complex of workspace.
 * Calls on one grid plan share that workspace: order them on one stream.
 * Errors: SE2_ERR_UNSUPPORTED (even L, precision, flags), SE2_ERR_INVALID_ARG
 * (N < L, batch, device), SE2_ERR_OOM; *plan is NULL on failure.
 */
se2_status se2_grid_plan_create(se2_grid_plan_t* plan, const int* L, const int* N, int batch, int precision,
                                unsigned flags, int device);
se2_status se2_grid_plan_destroy(se2_grid_plan_t plan);

/* Kernel launches issued by this plan so far. */
unsigned long long se2_grid_plan_launches(se2_grid_plan_t plan);

/*
 * se2_grid_coeffs -- C = DFT(P) / |L| (Eq. FkLv without its sign) of n <= batch
 * real sample arrays [n][Lr][Ly][Lx] into coeffs [n][Lr][Ly][Kx+1] complex.
 * Device pointers; asynchronous on `stream`.
 */
se2_status se2_grid_coeffs(se2_grid_plan_t plan, const void* samples, int n, void* coeffs, void* stream);

/*
 * se2_grid_convolve_chain -- out = Re S_K[f, rho_1..rho_k] on the N-grid for
 * B <= batch problems: f [B][Lr][Ly][Lx] real, coeffs[t] from se2_grid_coeffs
 * ([B][..] or, with SE2_SHARED_KERNEL, [1][..]), 0 <= k <= 32, out
 * [B][Nr][Ny][Nx] real (must not alias f).  Computed as
 *   sum over the stored bins of W^k (DFT(F)/|L|) C_1 .. C_k e^{+2 pi i k.n/N}
 * (Proposition LtoN1D: the zero-padded iDFT of Eq. MatSKfgonG without forming
 * the padded array).  Device pointers (host array of k coefficient pointers);
 * asynchronous on `stream`.  Errors: SE2_ERR_INVALID_ARG.
 */
se2_status se2_grid_convolve_chain(se2_grid_plan_t plan, const void* f, int B, const void* const* coeffs, int k,
                                   void* out, void* stream);

/*
 * se2_grid_convolve_chain_all -- every intermediate V_p = Re S_K[f, rho_1..rho_p],
 * p = 1..k, on the N-grid from one forward transform (Algorithm 6, the fast
 * recursion): out is [k][B][Nr][Ny][Nx] (it must not overlap f); coeffs and
 * the other arguments as se2_grid_convolve_chain, 1 <= k <= 32.  The running
 * product is kept unscaled in the plan's workspace.
 */
se2_status se2_grid_convolve_chain_all(se2_grid_plan_t plan, const void* f, int B, const void* const* coeffs, int k,
                                       void* out, void* stream);

/*
 * se2_grid_sample_se2_gaussian / se2_grid_sample_deformed_gaussian -- the
 * samplers of se2_sample_se2_gaussian (Eq. fbS) and
 * se2_sample_deformed_gaussian (Eq. fHsnu) on a grid plan's sampling grid
 * Omega_L: P is [Lr][Ly][Lx] of the plan's real type (device).  Arguments
 * and errors as for the square-grid samplers.
 */
se2_status se2_grid_sample_se2_gaussian(se2_grid_plan_t plan, const double* beta, const double* Sigma, int images,
                                        void* P, void* stream);
se2_status se2_grid_sample_deformed_gaussian(se2_grid_plan_t plan, const double* H, double nu, double s, int images,
                                             void* P, void* stream);

/*
 * se2_grid_ffc_at -- one finite Fourier coefficient f^[k; L] (Eq. FkLv,
 * Section 4.1) read from grid coefficients C = DFT(P) / |L| of real samples:
 * (-1)^(k1 + k2) C(tau(k)), where tau maps the signed frequency to its DFT bin
 * (k mod L); C holds x bins 0 .. Kx only, so a negative k1 reads the
 * Hermitian partner -k and conjugates it.  The step of Algorithm 1 that reads
 * one entry of the transform.
 *   coeffs  device, [batch][Lr][Ly][Kx+1] complex as written by se2_grid_coeffs
 *   index   which problem of the batch, 0 <= index < batch
 *   k1..k3  |k1| <= Kx, |k2| <= Ky, |k3| <= Kr (K = (L - 1) / 2)
 *   out     device, 2 doubles: real and imaginary part (written on `stream`)
 * Errors: SE2_ERR_INVALID_ARG for k outside the range, NULL or misaligned
 * pointers.
 */
se2_status se2_grid_ffc_at(se2_grid_plan_t plan, const void* coeffs, int index, int k1, int k2, int k3, double* out,
                           void* stream);

/*
 * se2_accuracy_order -- Algorithm 1 (Section 4.2; Theorem fkLmain and the
 * remark after it): the smallest K in N with
 *   K >= max(c ||grad f||_inf / eps, ||k||_inf),
 * so that the finite Fourier coefficient f^[k; 2K+1] on the odd grid
 * L = 2K+1 is within eps of the Fourier coefficient f^[k] for f in C^1
 * supported in Omega.  c = `constant` if > 0, else the theorem's 32 (its
 * proof through Theorem UkL gives 36).  Host only; writes *K.  Errors:
 * SE2_ERR_INVALID_ARG (eps <= 0, grad_inf < 0, k_inf < 0, non-finite input,
 * NULL K), SE2_ERR_UNSUPPORTED (K beyond 4e18).  A K above 127 exceeds the
 * grid plans' largest L.
 */
se2_status se2_accuracy_order(double eps, double grad_inf, int k_inf, double constant, long long* K);

const char* se2_last_error(void);

/* Library version string. */
const char* se2_version(void);

#ifdef __cplusplus
}
#endif
#endif /* SE2_H */
