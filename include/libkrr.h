/*
 * libkrr -- preconditioned Krylov solvers for Gaussian-kernel regression on
 * NVIDIA GB300 (sm_103a).
 *
 * The method is that of "Preconditioned Krylov solvers for kernel regression"
 * (Srinivasan, Hu, Gumerov, Murtugudde, Duraiswami; arXiv:1408.1237):
 * solve K x = b with K = K_hat + gamma I (Eq. 3), K_hat the Gaussian kernel
 * matrix of Eqs. 1-2, by flexible GMRES (Algorithm 1) right-preconditioned by
 * a truncated conjugate-gradient solve with M = K + delta I (Sec. 5).  The
 * kernel matrix is never stored: every product K q is summed on the fly.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Arrays:     X is N x d row-major float32 (point i at X[i*d .. i*d+d-1]).
 *             Multi-column arrays (Q, Y, B, Xsol) are N x m column-major:
 *             column c starts at element c*N.  Inputs are float32; solver
 *             solutions are FP64 (the iterate is carried in float-float, and
 *             rounding it to float32 alone can cost more than a 1e-6 relative
 *             residual when K is ill-conditioned).
 * Pointers:   array pointers may be DEVICE pointers (cudaMalloc / PyTorch
 *             tensors on the handle's device) or HOST pointers (pageable or
 *             pinned).  Host arrays are staged through the handle's device
 *             workspace with copies on `stream`, and such a call synchronises
 *             `stream` before it returns.  Calls on device arrays are
 *             stream-ordered and return without waiting unless an `info`
 *             pointer asks for results (see each function).
 *             The caller owns every array; the library never frees one.
 *             No array may alias another unless a function says so.
 * Streams:    `stream` is a cudaStream_t passed as void* (NULL = legacy
 *             default stream).  All device work of a call runs on it.
 * Handle:     a krr_handle binds to the device that is current when it is
 *             created and owns the device workspace (grown on demand, freed by
 *             krr_destroy).  A handle is not thread-safe: use one per host
 *             thread, or serialise calls.
 * Errors:     every function returns a krr_status and never aborts or exits;
 *             krr_last_error(h) gives a message for the last failing call on h.
 *             Invalid arguments are rejected before any device work is queued.
 *             Scalar outputs (gradients of krr_mll_grad) are HOST pointers.
 * Limits:     1 <= d <= 64; N >= 1 (N = 0 returns KRR_OK with no work);
 *             sigma > 0; shifts (gamma, delta) >= 0; all finite.
 * Dimension:  up to 8 the kernels are specialised per d and compact target
 *             blocks use the expanded exponent form (tensor cores where it
 *             pays).  Above 8 the coordinates are held padded with zeros to
 *             16, 32, 48 or 64; single-column float32 products contract the
 *             cross term of compact blocks on the tensor cores, and every
 *             other pair takes the direct form (exact differences on the CUDA
 *             cores).
 */
#ifndef LIBKRR_H
#define LIBKRR_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct krr_handle_s* krr_handle;

typedef enum {
    KRR_OK = 0,
    KRR_ERR_INVALID_ARG = 1,   /* bad size, pointer, sigma, shift or option     */
    KRR_ERR_CUDA = 2,          /* a CUDA runtime call failed (message has it)   */
    KRR_ERR_OOM = 3,           /* workspace allocation failed                   */
    KRR_ERR_NONFINITE = 4,     /* NaN or Inf met in inputs or iterates          */
    KRR_NOT_CONVERGED = 5,     /* iteration cap reached before the tolerance    */
    KRR_ERR_BREAKDOWN = 6,     /* Krylov breakdown that is not a lucky one      */
    KRR_ERR_TIMEOUT = 7,       /* a bounded device wait ran out                 */
    KRR_ERR_UNIMPLEMENTED = 8, /* option combination not built                  */
    KRR_ERR_SIZE_LIMIT = 9     /* problem larger than krr_kernel_mvp_noalloc's
                                  fixed scratch array accepts                   */
} krr_status;

/* Arithmetic of the kernel product.  KRR_FP32 sums in float32 with a
 * compensated (Kahan) fold across source tiles; KRR_BF16 / KRR_FP16 evaluate
 * the kernel values at reduced precision with float32 accumulation (the
 * low-accuracy inner product that Sec. 5.1 allows for the preconditioner). */
typedef enum { KRR_FP32 = 0, KRR_BF16 = 1, KRR_FP16 = 2 } krr_precision;

/* Options of krr_fgmres_solve (defaults from Sec. 6 in brackets).
 * Fill with krr_fgmres_default_opts(). */
typedef struct {
    int restart;          /* m of FGMRES(m), 1..64                      [30]   */
    int max_cycles;       /* restart cycles before KRR_NOT_CONVERGED     [50]   */
    double tol;           /* outer tol on |b - K x| / |b|                [1e-6] */
    double delta;         /* preconditioner shift; < 0: 10 gamma, or 1e-3
                             when gamma = 0 (Sec. 6)                      [-1]   */
    double inner_tol;     /* inner CG tol on |v - M z| / |v|; < 0: 10 tol [-1]  */
    int inner_maxit;      /* inner CG iteration cap; 0 = no preconditioner
                             (plain GMRES)                               [100]  */
    krr_precision inner_prec; /* arithmetic of the inner product M p    [FP32] */
    int use_graph;        /* 1: run the whole solve as one CUDA graph with
                             device-side loop control; 0: host-driven loop
                             with one status read per step               [1]    */
    int x0_given;         /* 1: the solution array holds an initial guess x0
                             on entry and the solve starts from it: the first
                             cycle takes r0 = b - K x0 from the accurate
                             product, as every restart of Alg. 1 (x0 <- x_m)
                             does, so a capped solve resumes where it
                             stopped; 0: x0 = 0 and the array is output only
                                                                          [0]    */
} krr_fgmres_opts;

/* Per-right-hand-side solver report. */
typedef struct {
    int outer_iters;        /* Arnoldi steps over all cycles (FGMRES) or CG
                               iterations (krr_cg_solve)                        */
    int inner_iters;        /* inner CG iterations in total                     */
    int cycles;             /* restart cycles run                               */
    int breakdowns;         /* inner p^T M p <= 0 events (inner solve cut short) */
    double relres_est;      /* last residual estimate |g_{j+1}| / |b|           */
    double relres_true;     /* |b - K x| / |b| from a fresh product at exit     */
    double time_ms;         /* device time of the solve                         */
    krr_status status;
} krr_solve_info;

/* One problem of a batched solve.  All arrays are DEVICE pointers. */
typedef struct {
    const float* X;   /* N x d row-major                                       */
    const float* B;   /* N x m_rhs column-major right-hand sides               */
    double* Xsol;     /* N x m_rhs column-major FP64 solutions (in: the initial
                         guess when opts->x0_given, else ignored)            */
    int64_t N;
    float gamma;
} krr_problem;

/* ---------------------------------------------------------------- handle */
krr_status krr_create(krr_handle* out);
krr_status krr_destroy(krr_handle h);
const char* krr_last_error(krr_handle h);
const char* krr_status_string(krr_status s);
/* Library version as major*10000 + minor*100 + patch. */
int krr_version(void);
void krr_fgmres_default_opts(krr_fgmres_opts* opts);

/* Handle options. */
typedef enum {
    /* The kernel of the compact target blocks of multi-column products
     * (krr_kernel_mvp with m >= 2, block, batched and gradient solves):
     *  0: mma.sync for the exponent and for Y += P Q;
     *  1: mma.sync for the exponent into registers, P = 2^E stored to tensor
     *     memory (tcgen05.st), Y += P Q by tcgen05.mma with P read from
     *     tensor memory and accumulators in tensor memory;
     *  2: tcgen05.mma for the exponent into tensor memory, loaded,
     *     exponentiated and stored back as P, then Y += P Q as in 1;
     *  3 (default): 1 for float32 products of more than 8 columns with at
     *     least 65536 targets at d >= 5 or 131072 at d <= 4, else 0; the
     *     solvers (block, batched and gradient solves) instead time 0 and 1
     *     once per product shape when they reserve it (a few products,
     *     before any graph capture) and keep the faster.
     * Same results to the float32 bar (and the reduced-precision bars).  On
     * GB300, 16 columns at 2^20 points: float32 370 / 434 / 552 ms, f16
     * 260 / 261 / 378 ms for 1 / 0 / 2.  Other values: KRR_ERR_INVALID_ARG. */
    KRR_OPT_TCGEN05 = 1,
    /* value: a krr_kernel_family.  The kernel function every product and
     * solver of this handle uses (default KRR_KERNEL_GAUSSIAN).  Under
     * KRR_KERNEL_MATERN32 the `sigma` argument of every call is the Matern
     * length scale h.  krr_mll_grad supports the Gaussian only and returns
     * KRR_ERR_UNIMPLEMENTED otherwise. */
    KRR_OPT_KERNEL = 2,
    /* value != 0: autotune the kernel variant and the source split of
     * every product.  The first product of each shape (sizes, columns,
     * precision, kernel family) on this handle, outside a CUDA-graph
     * capture, times the real launch on scratch weights (a few launches per
     * candidate; waits for them):
     *  - first the kernel variants of the shape at the modelled split:
     *    multi-column Gaussian products up to 8 dimensions try the mma.sync
     *    and tcgen05 kernels for compact target blocks and the tensor-core
     *    and CUDA-core weighted sums for direct-form blocks (the settings of
     *    KRR_OPT_TCGEN05 and KRR_OPT_DIRECT_TENSOR); single-column float32
     *    products that would take the tensor-core exponent path also try
     *    the packed CUDA-core kernel;
     *  - then the source split of the fastest variant (the range of source
     *    tiles one CTA sums) at 1/4 to 4 times the modelled split count.
     * The handle's own settings win unless a candidate is 2% faster; the
     * pick is kept for later products of that shape.  Results stay within
     * the same error bars; the summation grouping, hence the last bits, may
     * differ. */
    KRR_OPT_AUTOTUNE = 3,
    /* Target-row shard emulation (the row partition a multi-GPU product
     * would use, run on one GPU): with SHARD_COUNT = P > 1, krr_kernel_mvp
     * on this handle computes and writes only shard SHARD_INDEX = k of its
     * target rows: the sorted (Morton-order) super-blocks
     * [k nsb / P, (k+1) nsb / P) of 256 targets, that is 1/P of the work.
     * The other rows of Y are left as they were (a host Y is uploaded
     * first).  The plans are those of the whole product, so the P shards
     * written into one Y equal the unsharded product bit for bit.  Other
     * entry points ignore the setting.  SHARD_COUNT: 1 (default) to 4096;
     * SHARD_INDEX: 0 to SHARD_COUNT - 1 (checked at the call). */
    KRR_OPT_SHARD_COUNT = 4,
    KRR_OPT_SHARD_INDEX = 5,
    /* value != 0 (default): single-column products above 8 dimensions
     * contract their compact super-blocks with tcgen05.mma into tensor
     * memory; 0: with mma.sync.  Same results to the float32 bar; on GB300
     * the default is faster (measured at N = 65536: d = 16 2685 vs 2500,
     * d = 32 1434 vs 1185, d = 64 739 vs 655 Gpairs/s). */
    KRR_OPT_HIGHD_TCGEN05 = 6,
    /* value != 0 (default): multi-column products (m >= 2, block solves,
     * the gradient's solves) up to 8 dimensions evaluate the kernel values of
     * their direct-form (non-compact) target blocks on the CUDA cores and run
     * the weighted sum P Q on the tensor cores (tf32 hi/lo split for KRR_FP32,
     * single f16 / bf16 for reduced precision); 0: the all-CUDA-core kernel
     * (one FMA per pair and column).  Same results to the float32 bar. */
    KRR_OPT_DIRECT_TENSOR = 7
} krr_option;

/* Kernel functions (KRR_OPT_KERNEL). */
typedef enum {
    /* exp(-|x_i - x_j|^2 / (2 sigma^2))  (Eq. 2) */
    KRR_KERNEL_GAUSSIAN = 0,
    /* Matern, smoothness 3/2 (Sec. 6.1, Eq. MaternKernel):
     * (1 + sqrt(3) r / h) exp(-sqrt(3) r / h), r = |x_i - x_j|, h = sigma.
     * Every pair takes the direct form (differences, sqrt, one exponential),
     * on the CUDA cores at float32 whatever `prec` asks; the accurate
     * products of the solvers evaluate it in float-float. */
    KRR_KERNEL_MATERN32 = 1
} krr_kernel_family;
/* Set option `option` of h to `value`.  Unknown options or values:
 * KRR_ERR_INVALID_ARG. */
krr_status krr_set_option(krr_handle h, int option, int value);

/* ----------------------------------------------------------- kernel MVP
 * Y = (K_hat + gamma I) Q  (Eqs. 1-3; the weighted kernel sum of Sec. 3.1):
 *     Y[i,c] = sum_j exp(-|x_i - x_j|^2 / (2 sigma^2)) Q[j,c] + gamma Q[i,c]
 * over all N^2 pairs (no cut-off), summed on the fly in O(N) memory.
 * X: N x d; Q, Y: N x m column-major, 1 <= m <= 64.  Y must not alias X or Q.
 * m = 1 takes one exponential per pair, with the exponent contraction on the
 * tensor cores for compact target blocks and the CUDA-core kernel for the
 * rest; m >= 2 evaluates each kernel value once for up to 16 columns
 * (tensor cores for compact target blocks).
 * prec: KRR_FP32 (max relative error per element, against the FP64 sum
 * scaled by sum_j |Q_jc| K_hat_ij + gamma |Q_ic|, below 1e-5) or KRR_BF16 /
 * KRR_FP16 (reduced-precision kernel values, float32 accumulation).
 * The call waits briefly for the point preparation (Morton sort and block
 * metadata) to read the block counts that size the product grids; the
 * product itself is asynchronous on device arrays. */
krr_status krr_kernel_mvp(krr_handle h, const float* X, int64_t N, int d,
                          float sigma, float gamma, const float* Q, int m,
                          float* Y, krr_precision prec, void* stream);

/* ----------------------------------------------------------- prepared point sets
 * Repeated products over one point set (a serving loop, a caller's own
 * iterative method, many weight vectors): the Morton sort, packing and block
 * metadata of krr_kernel_mvp are done once, and each product then runs with
 * no host synchronisation, so it can be captured in a CUDA graph.
 *
 * krr_points_create prepares X (N x d, host or device, row-major float32)
 * for the kernel width sigma and the handle's kernel family (KRR_OPT_KERNEL
 * at creation; later changes of the option do not affect the object).  Its
 * device buffers belong to the object, inside h's workspace; X may be
 * overwritten or freed once the call returns.  The call waits for the
 * preparation once, to read the block counts that size the product grids.
 * On success *out is the object; destroy it with krr_points_destroy before
 * krr_destroy(h), and use it only with h.  Errors as for krr_kernel_mvp. */
typedef struct krr_points_s* krr_points;
krr_status krr_points_create(krr_handle h, const float* X, int64_t N, int d,
                             float sigma, krr_points* out, void* stream);

/* Y = (K_hat + gamma I) Q over a prepared point set (Eqs. 1-3), as
 * krr_kernel_mvp computes it (the same kernels, hence the same results):
 * Q, Y: DEVICE arrays, N x m column-major, 1 <= m <= 64; Y must not alias
 * Q.  Host arrays: KRR_ERR_INVALID_ARG.  The handle's product options
 * (KRR_OPT_TCGEN05, _DIRECT_TENSOR, _HIGHD_TCGEN05, _AUTOTUNE, the row
 * shards) apply as at the call.  No host synchronisation.  The products'
 * scratch belongs to the point set: once a product of this (m, prec) has
 * run on it, a call allocates nothing and can be captured in a CUDA graph,
 * which stays valid until krr_points_destroy (the first call of a shape may
 * allocate and must not be captured; neither may a larger m or another
 * precision after the capture).  Device-side errors (a timed-out bounded
 * wait) are reported by krr_points_destroy. */
krr_status krr_kernel_mvp_points(krr_handle h, krr_points P, const float* Q,
                                 int m, float gamma, float* Y,
                                 krr_precision prec, void* stream);

/* Waits for the device, frees the object's device buffers and reports a
 * device-side error of its products (KRR_ERR_TIMEOUT; the object is freed
 * anyway).  NULL P: KRR_OK.  P from another handle: KRR_ERR_INVALID_ARG. */
krr_status krr_points_destroy(krr_handle h, krr_points P);

/* Prediction product of Eq. GPR_mean / Eq. Kriging:
 *     Y[t,c] = sum_j exp(-|xt_t - xs_j|^2 / (2 sigma^2)) Q[j,c]
 * Xt: Nt x d targets, Xs: Ns x d sources, Q: Ns x m, Y: Nt x m (no diagonal
 * term).  Asynchronous on device arrays. */
krr_status krr_kernel_mvp_rect(krr_handle h, const float* Xt, int64_t Nt,
                               const float* Xs, int64_t Ns, int d, float sigma,
                               const float* Q, int m, float* Y,
                               krr_precision prec, void* stream);

/* ----------------------------------------------------------- CG solve
 * Conjugate gradient (Sec. 3) on (K_hat + shift I) x = b: the unpreconditioned
 * baseline when shift = gamma, the inner preconditioner solve when shift =
 * gamma + delta.  x: FP64, in = initial guess, out = solution (length N).
 * Stops when the true residual |b - A x| / |b| <= tol or after maxit
 * iterations in total.
 * Returns KRR_NOT_CONVERGED if the cap is reached.  If info != NULL the call
 * waits for the solve and fills *info (relres_true from a fresh product). */
krr_status krr_cg_solve(krr_handle h, const float* X, int64_t N, int d,
                        float sigma, float shift, const float* b, double* x,
                        double tol, int maxit, krr_precision prec,
                        krr_solve_info* info, void* stream);

/* ----------------------------------------------------------- FGMRES solve
 * Algorithm 1 on K = K_hat + gamma I with the paper's preconditioner:
 * truncated CG on M = K + delta I (Sec. 5), restart m, x0 = 0 (or the
 * initial guess in Xsol when opts->x0_given).  Arnoldi
 * (classical Gram-Schmidt applied twice, equal to the modified Gram-Schmidt
 * of Alg. 1 to working precision) and the Givens least-squares update run in
 * FP64; the outer products K z_j and the true residual in float32 with
 * compensated (float-float) arithmetic; the inner products M p in
 * opts->inner_prec.
 * B: N x m_rhs right-hand sides (float32), Xsol: N x m_rhs FP64 solutions
 * (column-major), each column solved to |b - K x| / |b| <= opts->tol (true
 * residual).  Several right-hand sides are solved in lockstep blocks of at
 * most 16 columns (as few blocks as possible, of equal width): every column
 * runs its own Alg. 1 with its own Krylov basis and restarts, and each inner
 * CG step applies M to all columns' directions in one multi-column product.
 * info[c].time_ms is the time of the block that solved column c.
 * opts = NULL takes the defaults.  info: NULL or an array of m_rhs reports.
 * The call waits for the solve when info != NULL.  Returns the worst status
 * over the columns. */
krr_status krr_fgmres_solve(krr_handle h, const float* X, int64_t N, int d,
                            float sigma, float gamma, const float* B, int m_rhs,
                            double* Xsol, const krr_fgmres_opts* opts,
                            krr_solve_info* info, void* stream);

/* ------------------------------------------------------ flexible CG solve
 * Flexible CG (Notay; the paper's second outer iteration, Sec. 4.2) on
 * K = K_hat + gamma I with the same truncated-CG preconditioner on
 * M = K + delta I: each new search direction is the preconditioned residual
 * made K-orthogonal to the previous opts->restart directions (the window),
 * step lengths from the FP64 recursion, the iterate in float-float, products
 * K d with the compensated kernel.  When the recursive residual meets the
 * tolerance the true residual is computed; if it does not meet it, the
 * iteration restarts from it with an empty window.  At most
 * opts->restart * opts->max_cycles steps.  The paper pairs flexible CG with
 * an accurate inner solve (its experiments: delta = inner_tol = 1e-4).
 * Arguments and reports as krr_fgmres_solve (outer_iters = flexible-CG
 * steps, cycles = restarts + 1); right-hand sides are solved one after
 * another.  Waits for the solve. */
krr_status krr_fcg_solve(krr_handle h, const float* X, int64_t N, int d,
                         float sigma, float gamma, const float* B, int m_rhs,
                         double* Xsol, const krr_fgmres_opts* opts,
                         krr_solve_info* info, void* stream);

/* Many independent problems (same d, sigma, opts; own N_k, gamma_k, m_rhs
 * right-hand sides each) solved together: one lockstep block solve per
 * problem (and block of right-hand sides), each an independent branch with
 * its own workspace, launched as CUDA graphs of at most 32 concurrent
 * branches.  probs: HOST array of nprob krr_problem records whose arrays are
 * DEVICE pointers.  info: NULL or nprob * m_rhs reports (problem-major);
 * time_ms is the time of the whole batch.  Waits for the solve.  Returns the
 * worst status. */
krr_status krr_fgmres_solve_batched(krr_handle h, const krr_problem* probs,
                                    int nprob, int d, float sigma, int m_rhs,
                                    const krr_fgmres_opts* opts,
                                    krr_solve_info* info, void* stream);

/* ----------------------------------------------------- MLL gradient
 * Gradient of the GP log-marginal likelihood
 *     L = -1/2 y^T K^-1 y - 1/2 log det K - N/2 log 2 pi   (Sec. 2.1 ML fit)
 * with respect to log sigma, log gamma and the points X, using alpha = K^-1 y
 * and u_p = K^-1 z_p (FGMRES solves) for n_probes Rademacher probes z_p drawn
 * from SplitMix64 seeded with `seed` (element (i, p) is -1 when the top bit of
 * output number p*N + i + 1 is set), and the Hutchinson estimate
 * K^-1 ~ (1/P) sum_p u_p z_p^T in the trace term.
 * dlogsigma, dloggamma: HOST doubles; dX: N x d row-major float32 (device or
 * host), may be NULL.  Waits for the result before returning. */
krr_status krr_mll_grad(krr_handle h, const float* X, int64_t N, int d,
                        float sigma, float gamma, const float* y, int n_probes,
                        uint64_t seed, const krr_fgmres_opts* opts,
                        double* dlogsigma, double* dloggamma, float* dX,
                        krr_solve_info* info, void* stream);

/* ----------------------------------------------------- diagnostics
 * Issue-rate microbenchmarks that bound the kernel product (not part of the
 * paper's method): results per second of MUFU.EX2 (ex2.approx.ftz.f32), of
 * scalar FP32 FMA, and of FP32 lanes through packed f32x2 FMA, on the
 * handle's device at its current clocks (about 10 ms of GPU time; waits for
 * the result).  Outputs are HOST doubles; any may be NULL. */
krr_status krr_measure_alu_peaks(krr_handle h, double* ex2_per_s, double* ffma_per_s,
                                 double* ffma2_lanes_per_s, void* stream);
/* Reciprocal square roots (rsqrtf, the one the Matern kernel takes per pair)
 * per second on the handle's device at its current clocks, measured the same
 * way (a few ms of GPU time; waits).  rsqrt_per_s: HOST double, not NULL. */
krr_status krr_measure_rsqrt_rate(krr_handle h, double* rsqrt_per_s, void* stream);

/* Rates behind the reduced-precision design, measured the same way (a few
 * ms of GPU time; waits): exponential VALUES per second through the packed
 * half-precision instructions ex2.approx.f16x2 and ex2.approx.ftz.bf16x2 (two
 * values per instruction; on GB300 they give the same values per second as
 * ex2.approx.ftz.f32, so half-precision kernel values do not raise the
 * exponential bound), and dense f16 FLOP/s of the warp-level tensor-core MMA
 * mma.sync m16n8k16 with f32 accumulation.  Outputs: HOST doubles; any may
 * be NULL. */
krr_status krr_measure_half_rates(krr_handle h, double* ex2_f16x2_values_per_s,
                                  double* ex2_bf16x2_values_per_s,
                                  double* mma_sync_f16_flops_per_s, void* stream);

/* Failure-path self-test (not part of the method: failure detection checked
 * without a GPU fault).  Every device wait of the library is
 * bounded: a kernel whose wait runs out records it in the handle's error word,
 * drains what it has in flight and returns, and the call reports
 * KRR_ERR_TIMEOUT.  This entry point runs a one-thread kernel that waits, with
 * that same bounded routine, on an mbarrier phase nothing completes (no copy,
 * MMA or other warp is outstanding on it), giving up after limit_clocks SM
 * clocks (1 to 2e9; a few thousand take microseconds).  It waits for `stream`
 * and returns KRR_ERR_TIMEOUT, after which the handle stays usable: the error
 * word is cleared and later calls run normally. */
krr_status krr_selftest_wait_timeout(krr_handle h, long long limit_clocks, void* stream);

/* Launch and timing counters for measurement (not part of the method). */
typedef struct {
    long long launches;     /* kernels the library launched since it was loaded
                               (a launch captured into a CUDA graph counts once) */
    int product_launches;   /* fast-product launches (single- or multi-column
                               float32 / reduced-precision products, not the
                               accurate product) timed since the last read      */
    double product_ms;      /* their summed device time (CUDA events recorded
                               on the stream each launch ran on)                */
    double product_pairs;   /* target x source pairs they evaluated, per column */
    int tensor_exponent_launches; /* of the timed launches, those that took the
                               tensor-core exponent path (the exponent
                               contraction on the tensor cores, one MUFU.EX2
                               and one FMA per pair on the CUDA cores); the
                               rest ran the CUDA-core kernels                  */
} krr_profile;
/* Start (enable != 0) or stop timing the fast-product kernel on h; resets the
 * timed list.  Timing adds two event records per product launch. */
krr_status krr_profile_enable(krr_handle h, int enable);
/* Fill *out, waiting for the recorded events, and reset the timed list. */
krr_status krr_profile_read(krr_handle h, krr_profile* out);

/* ------------------------------------------------ tuning cache file
 * The autotuner's results on h (KRR_OPT_AUTOTUNE, and the solvers' timed
 * kernel choice): per product shape, the kernel variant and the source-split
 * scale.  A shape's key holds its sizes, columns, precision, kernel family,
 * planning slots, compact-block counts and the kernel-option mode, so an
 * entry is used only for the same shape under the same options.
 * krr_tune_save writes them to the text file `path` (a header with the
 * device's SM count, then one line per shape); KRR_ERR_INVALID_ARG when the
 * file cannot be written.  krr_tune_load reads such a file into h (its
 * entries replace h's for the same shapes), so that a later process skips
 * the timing; KRR_ERR_INVALID_ARG for a missing or malformed file or one
 * written on a device with another SM count.  Host-only: no device work. */
krr_status krr_tune_save(krr_handle h, const char* path);
krr_status krr_tune_load(krr_handle h, const char* path);

/* ------------------------------------------------ no-allocation product
 * The paper has no counterpart to this entry point.  It serves callers that
 * cannot allocate device memory: processes whose device memory pool belongs
 * to another framework (which forbids or is fragmented by foreign cudaMalloc
 * calls), and latency-bound paths where cudaMalloc's implicit device
 * synchronisation is not allowed.  Such callers cannot create a krr_handle
 * either, since a handle grows its workspace with cudaMalloc.
 * Result: that of krr_kernel_mvp with KRR_FP32, for DEVICE arrays X (N x d
 * row-major), Q and Y (N x m column-major) with N <= 16384, d <= 8 and
 * m <= 16.  Larger problems return KRR_ERR_SIZE_LIMIT; host arrays and bad
 * values return KRR_ERR_INVALID_ARG.
 * It allocates nothing.  Its scratch is one fixed device array of 10,415,872
 * bytes, held by every GPU that loads the library until the process exits;
 * an internal request beyond a region of it returns KRR_ERR_OOM instead of
 * allocating.  The first call made with a device current looks up that
 * array's device address (cudaGetSymbolAddress).  All calls on a device
 * share the array and it keeps the last call's contents; calls that overlap
 * on the GPU race on it and give wrong results.
 * The call waits for `stream`: the point preparation reads two block counts
 * back to the host before the product is queued.  So it returns
 * KRR_ERR_INVALID_ARG while `stream` is being captured into a CUDA graph,
 * and it must not be called from a host function enqueued on a stream
 * (CUDA forbids CUDA calls there). */
krr_status krr_kernel_mvp_noalloc(const float* X, int64_t N, int d, float sigma,
                                  float gamma, const float* Q, int m, float* Y,
                                  void* stream);

#ifdef __cplusplus
}
#endif

#endif /* LIBKRR_H */
