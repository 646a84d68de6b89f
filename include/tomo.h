/*
 * tomo.h -- C ABI of the GB300 detector-tomography solver.
 *
 * The library reconstructs the diagonal POVM matrix Theta (M photon numbers x
 * N outcomes, row-major) of a phase-insensitive detector from measured outcome
 * frequencies P (D coherent probes x N, row-major) by solving
 *
 *     min_Theta  ||P - F Theta||_2^2 + gamma sum_n sum_{i=0}^{M-2}
 *                (Theta_{i,n} - Theta_{i+1,n})^2
 *     subject to Theta_{i,n} >= 0,  sum_n Theta_{i,n} = 1 for every i,
 *
 * (Schapeler et al., arXiv 2404.02844: Eq. min, Eq. regul), where
 * F_{d,i} = lambda_d^i e^{-lambda_d} / i! (Eq. Fmatrix) is never stored: the
 * kernels regenerate it in log space inside every band contraction.  The
 * solver is the paper's two-stage, two-metric projected truncated Newton
 * method (App. B, Algorithms 1-3).
 *
 * Conventions for every entry point:
 *   - Return a tomo_status; nothing aborts, throws or exits across the ABI.
 *     tomo_last_error() gives a message for the last failure on this thread.
 *   - Matrices are dense, row-major, double precision, no padding.
 *   - "device" pointers are CUDA global-memory pointers of the current device;
 *     entry points documented as "host or device" accept either and detect the
 *     kind with cudaPointerGetAttributes (host buffers are staged through
 *     plan-owned device memory).
 *   - Work is ordered on the plan's stream; calls return after the results
 *     they report are complete (device outputs are complete on return).
 *   - The caller keeps ownership of every buffer it passes; the plan owns its
 *     workspaces and frees them in tomo_plan_destroy.
 *   - A plan is not thread-safe: one call at a time per plan.
 */
#ifndef TOMO_H
#define TOMO_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    TOMO_OK = 0,
    TOMO_EINVAL = 1,     /* invalid argument (sizes, non-finite lambda, NULL) */
    TOMO_ENOMEM = 2,     /* device or host allocation failed */
    TOMO_ECUDA = 3,      /* a CUDA runtime call failed */
    TOMO_ENOTCONV = 4,   /* iteration cap reached before the stopping rule */
    TOMO_ETIMEOUT = 5,   /* a bounded device wait (tensor-core pipeline) gave up */
    TOMO_ENONFINITE = 6  /* P or Theta holds NaN/Inf, or the objective became non-finite */
} tomo_status;

/* Arithmetic of the band contractions F X and F^T Y.
 *   FP64: every product in double ("plain" solver): the objective of every
 *         line-search trial is evaluated directly, f = ||F Theta' - P||^2 + g.
 *   FP32: products in single precision with FP32 accumulation; the residual
 *         R = F Theta - P is kept in double, refreshed by a double product
 *         every refresh_every Newton iterations and otherwise updated as
 *         R <- R + F s for each accepted step s; line searches use the exact
 *         quadratic expansion f(Theta + s) - f(Theta) = 2<R, F s> + ||F s||^2
 *         + g(Theta + s) - g(Theta) reduced in double. */
/*   MIXED: as FP32 for the CG Hessian products and the line-search products,
 *         but the gradient F^T R is contracted in double.
 *   TC:   the CG Hessian products run on the tensor cores (tcgen05.mma,
 *         bf16 operands split into hi + lo parts, three products per slice,
 *         f32 accumulation in tensor memory: ~17 significant bits, relative
 *         error ~8e-6) and the
 *         CG vectors (x, r, z, p) are float, their dot products summed per
 *         row in float and across rows in double; the line-search products
 *         F s and the gradient F^T R are contracted in float (the Armijo
 *         test needs float-grade F s); Theta, the gradient, residual
 *         refreshes, the objective and every other reduction in double. */
typedef enum {
    TOMO_PREC_FP64 = 0,
    TOMO_PREC_FP32 = 1,
    TOMO_PREC_MIXED = 2,
    TOMO_PREC_TC = 3
} tomo_precision;

typedef struct tomo_plan_s *tomo_plan_t;

/* tomo_desc.flags: time candidate schedule densities of the CG Hessian
 * product at plan time and keep the fastest (SIMT forms: work units per SM
 * and column block in {1, 2, 4, 8}; tensor-core form: persistent CTAs per
 * column block in {all SMs, 3/4, 1/2}).  Choices are cached per process by
 * (precision form, N, power-of-two class of M and of D), so a batch of
 * instances of one class tunes once.  The paper has no counterpart. */
#define TOMO_PLAN_AUTOTUNE 1u

/* Problem descriptor (Eq. min, Eq. Fmatrix, Eq. regul). */
typedef struct {
    int64_t M;             /* photon-number cutoff: i = 0..M-1, 1 <= M <= 2^30 */
    int64_t N;             /* outcomes, 2 <= N <= 1024 */
    int64_t D;             /* probes, 1 <= D <= 2^30 */
    const double *lambda;  /* HOST array of D mean photon numbers |alpha_d|^2,
                              finite, >= 0 and non-decreasing (probes sorted by
                              intensity); copied by tomo_plan */
    double band_k;         /* Poisson band half-width in standard deviations:
                              F_{d,i} is kept for lo_d <= i <= hi_d with
                              lo_d = max(0, floor(lambda - k sqrt(lambda))),
                              hi_d = min(M-1, max(16, ceil(lambda + k sqrt(lambda))));
                              band_k <= 0 keeps every i (dense F) */
    double gamma;          /* regularisation weight gamma >= 0 (Eq. regul) */
    int32_t precision;     /* tomo_precision */
    int32_t reserved;
    void *stream;          /* cudaStream_t to order work on; NULL: the plan
                              creates and owns a non-blocking stream */
    uint32_t flags;        /* 0 or TOMO_PLAN_AUTOTUNE */
} tomo_desc;

/* Builds a plan: validates the descriptor, computes the probe bands, the
 * log-space Poisson anchor table, the contraction tile schedule and the
 * Hessian diagonal on the device, and allocates every workspace (about
 * (3 D N + 13 M N) doubles).  Invalid input gives TOMO_EINVAL and leaves
 * *out == NULL.  (Eq. Fmatrix; Table ops "diagonal of Hessian".) */
tomo_status tomo_plan(tomo_plan_t *out, const tomo_desc *desc);

/* Frees the plan and everything it owns.  NULL is accepted. */
void tomo_plan_destroy(tomo_plan_t plan);

/* Objective value (Table ops "objective value"; Eq. min + Eq. regul):
 * *f_host = ||P - F Theta||^2 + gamma sum (Theta_{i,n} - Theta_{i+1,n})^2,
 * always in double.  P (D x N) and Theta (M x N) are host or device.  If
 * grad is not NULL it receives G = 2 F^T (F Theta - P) + 2 gamma L Theta
 * (M x N, same kind of memory as Theta), computed with the plan's
 * precision for F^T R and double for the residual. */
tomo_status tomo_objective(tomo_plan_t plan, const double *P, const double *Theta,
                           double *f_host, double *grad);

/* Solver options; tomo_fit_opts_default fills the defaults shown. */
typedef struct {
    double eps_kkt;        /* 1e-10: stop when the KKT residual of App. B,
                              sqrt(mean (Theta (G + lambda_i))^2) with
                              lambda_i = max(0, -min_n G_{i,n}), is <= eps_kkt */
    double eps_bar;        /* 1e-6: eps_k = min(eps_bar, w_k) in the index set I */
    double beta;           /* 0.75: backtracking factor (App. B) */
    double c;              /* 0.1: Armijo constant (App. B) */
    double switch_tol;     /* 1e-4: stage-1 -> stage-2 switch threshold (App. B) */
    double f_target;       /* 0: off; > 0: stop as soon as f <= f_target
                              (checked with a double-precision residual) */
    int32_t max_newton;    /* 1000: Newton iterations, both stages together */
    int32_t max_stage1;    /* 200: stage-1 iterations */
    int32_t max_cg;        /* 10000: cap on Hessian products per Newton iteration,
                              a safety bound (CG stops on its forcing rule) */
    int32_t ls_max;        /* 50: backtracking steps per line search */
    int32_t start_stage;   /* 1: Algorithm 3; 2: stage 2 only (Algorithm 1) */
    int32_t warm_start;    /* 0: Theta^(0) = 1/N; 1: start from Theta as passed */
    int32_t stall_iters;   /* 5: stop after this many iterations without decrease */
    int32_t refresh_every; /* 8: FP32 plans recompute R in double this often */
    int32_t profile;       /* 0; 1: time every band contraction of the CG loop
                              with CUDA events on the plan stream (report fields
                              fwd_ms / adj_ms); adds no synchronisation */
    int32_t trace_len;     /* 0; > 0: rows of `trace` (one per Newton iteration) */
    /* CG forcing term (App. B leaves the CG stop open): CG stops when
     * ||r|| <= eta ||b||, eta = min(cg_eta_max, ||b||^cg_eta_pow), b the
     * right-hand side (minus the free gradient); cg_eta_pow = 0 gives the
     * constant eta = cg_eta_max. */
    double cg_eta_max;     /* 0.5 */
    double cg_eta_pow;     /* 0.5 */
    double max_seconds;    /* 0: off; > 0: stop (stop code 2) once the solve has
                              run this long on the host clock */
    double *trace;         /* NULL, or a HOST array of trace_len x TOMO_TRACE_COLS
                              doubles: per Newton iteration k, row k receives
                              (stage, f before the step, KKT residual before the
                              step, CG products, ||r|| / ||b|| reached by the CG
                              recursion, accepted step length (0: none),
                              line-search trials, host ms since the start,
                              trials rejected for a negative implicit entry
                              (stage 2), how CG ended: 0 forcing test,
                              1 product cap, 2 non-positive curvature,
                              host ms spent in the CG loop) */
} tomo_fit_opts;

#define TOMO_TRACE_COLS 11

/* Result of a fit. */
typedef struct {
    double f;              /* final objective (double-precision residual) */
    double kkt;            /* final KKT residual */
    double time_ms;        /* wall time of the solve on the host clock */
    int32_t iters_s1, iters_s2;  /* Newton iterations per stage */
    int32_t cg_total;      /* Hessian products in CG */
    int32_t ls_total;      /* line-search trials */
    int32_t refreshes;     /* double-precision residual recomputations */
    int32_t stop;          /* 0 KKT reached, 1 f_target reached, 2 iteration cap,
                              3 stagnated (no decrease / line search failed) */
    int32_t stage_end;     /* stage at exit */
    int32_t kernels;       /* kernels launched by this call */
    int32_t fwd_count;     /* profiled CG products F p (opts.profile) */
    int32_t adj_count;     /* profiled CG products F^T (F p) */
    double fwd_ms;         /* summed device time of those launches */
    double adj_ms;
} tomo_fit_report;

void tomo_fit_opts_default(tomo_fit_opts *opts);

/* Two-stage two-metric projected truncated Newton fit (Algorithm 3: stage 1
 * = Algorithm 2 with the row-wise simplex projection P_{S^M}, stage 2 =
 * Algorithm 1 with the row-maximum transformation).  P (D x N) is read,
 * Theta (M x N) is read when opts->warm_start and always overwritten with
 * the result; both host or device.  opts may be NULL (defaults); report may
 * be NULL.  Theta is on the row simplices on every return except
 * TOMO_EINVAL.  Returns TOMO_OK for stop codes 0, 1 and 3, TOMO_ENOTCONV for
 * the iteration cap. */
tomo_status tomo_fit(tomo_plan_t plan, const double *P, double *Theta,
                     const tomo_fit_opts *opts, tomo_fit_report *report);

/* Batch of independent problems (for instance one data set at several gamma,
 * or many detectors): each instance k gets its own plan (built from
 * descs[k]) and is solved by tomo_fit(P[k], Theta[k], opts), up to
 * `concurrency` instances at a time (<= 0: 8), each on its plan's own work
 * stream so that small instances share the GPU.  Plans are built and freed
 * inside the call, so memory is bounded by the concurrent instances.  Every
 * plan fences descs[k].stream into its work stream on entry and back on exit.
 * statuses[k] receives each instance's status, reports[k] (may be NULL) its
 * report.  Returns TOMO_OK if every instance returned TOMO_OK or
 * TOMO_ENOTCONV, else the first other failure. */
tomo_status tomo_fit_batched(const tomo_desc *descs, const double *const *P, double *const *Theta,
                             int32_t count, const tomo_fit_opts *opts, tomo_fit_report *reports,
                             tomo_status *statuses, int32_t concurrency);

/* ---- single steps of the hot path (device pointers only) ----------------
 * Exposed so that every step can be checked on its own; the solver calls the
 * same kernels. */

/* O = F X (Table ops, the F Pi product of the objective): X M x N -> O D x N,
 * computed in the precision of the plan's Hessian products (double for FP64
 * plans, float otherwise), stored in double. */
tomo_status tomo_apply_F(tomo_plan_t plan, const double *X, double *O);

/* Z = F^T Y: Y D x N -> Z M x N, plan precision, stored in double. */
tomo_status tomo_apply_Ft(tomo_plan_t plan, const double *Y, double *Z);

/* Hessian product (Table ops): HV = 2 F^T F V + 2 gamma L V, M x N, in the
 * arithmetic of the plan's CG products (tensor cores for TC plans). */
tomo_status tomo_hvp(tomo_plan_t plan, const double *V, double *HV);

/* Schedule chosen for the plan's CG Hessian product. */
typedef struct {
    int32_t autotuned;      /* 1 if TOMO_PLAN_AUTOTUNE chose the density */
    int32_t from_cache;     /* 1 if the choice came from the per-process cache */
    int32_t tensor_cores;   /* 1 for the tensor-core form */
    int32_t density;        /* SIMT units per SM, or tensor-core CTAs per column block */
    double hvp_ms;          /* timed Hessian product of the chosen density (0 if not tuned) */
    int32_t units_fwd, units_adj;   /* work units of the forward / adjoint contraction */
    int32_t ctas_fwd, ctas_adj;     /* CTAs launched per column block */
} tomo_plan_info_t;

tomo_status tomo_plan_info(tomo_plan_t plan, tomo_plan_info_t *info);

/* The work-unit planning of the tensor-core contractions, host only (no
 * device work), exposed so that schedules can be checked without a GPU:
 * tile t reduces over [st[t], en[t]) (multiples of align; en <= st: empty);
 * the ranges, laid end to end, are cut into at most `ctas` equal shares
 * (multiples of align), a share crossing a tile boundary becoming one unit
 * per tile, no unit longer than max_unit (a multiple of align), empty tiles
 * one zero-length unit each, spread over the CTAs.  Writes up to `capacity`
 * units as (tile, chunk, k0, k1) int32 quadruples in CTA order, the CTA
 * boundaries (n_ctas + 1 entries, at most ctas + 1), the units per tile, and
 * n_ctas; returns the number of units, or -1 (EINVAL in tomo_last_error) on
 * invalid arguments or too small a capacity.  The paper has no counterpart. */
int64_t tomo_plan_tc_units(const int64_t *st, const int64_t *en, int32_t tiles, int32_t align,
                           int64_t max_unit, int64_t ctas, int32_t *units_out, int64_t capacity,
                           int32_t *cta_first_out, int32_t *nsplit_out, int32_t *n_ctas_out);

/* Self-test of the bounded device waits (no counterpart in the paper): runs
 * one tensor-core Hessian product whose tensor-core instructions are
 * withheld and whose mbarrier waits are bounded at 4096 polls, so every wait
 * gives up; the kernels flag it and return without faulting.  Returns what
 * a real timeout returns, TOMO_ETIMEOUT, after re-arming the plan (it stays
 * usable).  EINVAL for a plan not in the tensor-core form. */
tomo_status tomo_selftest_tc_timeout(tomo_plan_t plan);

/* Hessian diagonal h_i = 2 sum_d F_{d,i}^2 + 2 gamma L_ii (Table ops), M
 * doubles, always computed in double at plan time. */
tomo_status tomo_hess_diag(tomo_plan_t plan, double *h);

/* Row-wise projection onto the probability simplex (Eq. Mp1_proj):
 * Y_i = argmin_{y >= 0, sum y = 1} ||X_i - y||, M rows of N; double. */
tomo_status tomo_project_simplex(tomo_plan_t plan, const double *X, double *Y);

/* Long-range smoothing (Sec. "Regularisation and smoothing", Eq. smoothing):
 * Y_{i,n} = mean of X_{j,n} over j in [i - w, i + w], w = floor(i / div),
 * with the window clipped to [0, M-1] and the mean taken over the rows in it;
 * rows i < exclude are copied.  The paper uses div = 50 and excludes the
 * lowest ~100 photon numbers.  X, Y: M x N row-major doubles in device memory
 * (caller-owned; Y may equal X).  A mean of simplex rows is a simplex row, so
 * a feasible X gives a feasible Y: the warm start of the stage-2-only refit
 * (tomo_fit with start_stage = 2).  Computed from double-double column prefix
 * sums; each output is within a few units in the last place of the exact
 * window mean.  EINVAL: NULL pointer, exclude < 0 or div <= 0 (or NaN).
 * Uses plan workspaces: not concurrent with another call on the same plan. */
tomo_status tomo_smooth(tomo_plan_t plan, const double *X, double *Y, int64_t exclude, double div);

/* Infidelity 1 - F_n of Eq. fidelities between two POVMs (M x N doubles,
 * device, row-major; each column an operator diagonal in the photon-number
 * basis): F_n = (sum_i sqrt(Theta_in Ref_in))^2 / (sum_i Theta_in sum_i Ref_in),
 * the matrix-square-root definition for commuting operators.  infid_host
 * receives N doubles (nan for an all-zero column).  Uses plan workspaces. */
tomo_status tomo_infidelity(tomo_plan_t plan, const double *Theta, const double *Theta_ref,
                            double *infid_host);

/* KKT residual of App. B for (Theta, G), both M x N device; double. */
tomo_status tomo_kkt(tomo_plan_t plan, const double *Theta, const double *G,
                     double *kkt_host);

/* Poisson weights F_{d,i} as the kernels generate them, for `count` pairs
 * (d[k], i[k]) given in HOST arrays; out_host receives double values in the
 * plan's precision (0 outside the band). */
tomo_status tomo_poisson_weights(tomo_plan_t plan, const int64_t *d, const int64_t *i,
                                 int64_t count, double *out_host);

/* Band bounds lo_d, hi_d as computed by the plan (HOST arrays of D). */
tomo_status tomo_bands(tomo_plan_t plan, int64_t *lo_host, int64_t *hi_host);

/* ---- learned warm start ----------------------------------------------------
 * The paper has no counterpart: it starts Algorithm 3 from Theta^(0) = 1/N.
 * A small network maps measured frequencies P (D probes x C0 outcome columns,
 * the columns n >= ncols of a sample zero) to a starting POVM Theta0 (M x C0,
 * each row a softmax over its first ncols columns, hence on the simplex):
 *   Y1 = conv1d(P, W1, b1, stride S1)        (D/S1) x C1
 *   Y2 = conv1d(relu(Y1), W2, b2, stride S2) (D/S1/S2) x C2
 *   Y3 = W3 flat(relu(Y2)) + b3              H
 *   Z  = W4 relu(Y3) + b4                    M x C0 logits
 * conv1d(X, W, b, S)[t, co] = b[co] + sum_{ci,k} W[co,ci,k] X[S t + k - K/2, ci]
 * (zero padding).  Training minimises the row-wise cross-entropy against
 * target POVMs (mean over rows and samples) with Adam (beta1 0.9, beta2
 * 0.999, eps 1e-8); float arithmetic and float master weights; inference
 * reads a bf16 copy of the weights with float accumulation.  Parameters form
 * one float vector: W1 (C1 x C0 x K), b1, W2 (C2 x C1 x K), b2, W3 (H x F,
 * F = D/S1/S2 * C2, flattened t-major), b3, W4 (M C0 x H), b4 (M C0). */
typedef struct tomo_ws_s *tomo_ws_t;

typedef struct {
    int64_t D, C0, M;       /* probes, padded outcome columns (2..256), photon numbers */
    int64_t C1, C2, K;      /* conv channels and kernel width */
    int64_t S1, S2, H;      /* conv strides (D % S1 == 0, (D/S1) % S2 == 0), hidden width */
    int64_t max_batch;      /* largest training batch */
    uint64_t seed;          /* SplitMix64 seed of the He-uniform initialisation */
    void *stream;           /* cudaStream_t; NULL: the handle owns a stream */
} tomo_ws_desc;

/* Allocates the parameters, Adam state and activations (device) and
 * initialises the weights.  EINVAL on a shape out of range. */
tomo_status tomo_ws_create(tomo_ws_t *out, const tomo_ws_desc *desc);
void tomo_ws_destroy(tomo_ws_t ws);
/* Number of parameters (-1 for a NULL handle). */
int64_t tomo_ws_param_count(tomo_ws_t ws);
/* Copy the float parameters to / from HOST memory (set also resets Adam). */
tomo_status tomo_ws_get_params(tomo_ws_t ws, float *host);
tomo_status tomo_ws_set_params(tomo_ws_t ws, const float *host);
/* Mean cross-entropy of a batch and its gradient (no update).  P: B x D x C0,
 * T: B x M x C0 doubles in device memory (padded columns ignored); ncols:
 * HOST array of B column counts (1..C0); grad_host (nullable) receives
 * tomo_ws_param_count floats. */
tomo_status tomo_ws_loss_grad(tomo_ws_t ws, const double *P, const double *T, const int32_t *ncols,
                              int32_t B, float *loss_host, float *grad_host);
/* One Adam step on the batch (same inputs); loss_host (nullable) receives
 * the batch loss before the step. */
tomo_status tomo_ws_train_step(tomo_ws_t ws, const double *P, const double *T, const int32_t *ncols,
                               int32_t B, float lr, float *loss_host);
/* Theta0 (M x N doubles, device) for one problem's P (D x N doubles, device,
 * N <= C0 columns, unpadded): every row on the simplex. */
tomo_status tomo_ws_infer(tomo_ws_t ws, const double *P, int64_t N, double *Theta0);
/* Algorithm 3 started from the learned warm start, with its fallback: Theta0
 * = tomo_ws_infer(ws, P, N); with zero_below > 0, the entries of each row of
 * Theta0 below zero_below x the row's largest are set to 0 and the row is
 * rescaled to sum 1 (a softmax has no exact zeros, while most entries of a
 * detector POVM are zero at the optimum: the zeros start at their bound);
 * zero_below = 0 keeps the network's output.  When f(Theta0) < f(1/N) (both evaluated in
 * double, Eq. min + Eq. regul) the fit starts from Theta0 (warm_start = 1),
 * else from Theta = 1/N; a warm-started fit that fails (any status other
 * than TOMO_OK and TOMO_ENOTCONV, or a non-finite objective) is redone from
 * 1/N.  The handle must match the plan (same D and M, N <= C0).  P (D x N)
 * and Theta (M x N, receives the result) are DEVICE pointers; opts and
 * report as in tomo_fit (opts->warm_start is ignored); *used_warm (nullable)
 * receives 1 when the returned Theta comes from the warm-started fit.  The
 * paper has no counterpart (it starts from 1/N). */
tomo_status tomo_fit_warm(tomo_plan_t plan, tomo_ws_t ws, const double *P, double *Theta,
                          double zero_below, const tomo_fit_opts *opts, tomo_fit_report *report,
                          int32_t *used_warm);

/* Parameter file: magic "TOMOWS01", the nine shape fields, the floats. */
tomo_status tomo_ws_save(tomo_ws_t ws, const char *path);
tomo_status tomo_ws_load(tomo_ws_t ws, const char *path);

/* Kernel launches made by this library since it was loaded (all threads,
 * all entry points), for launch accounting. */
int64_t tomo_kernel_launches(void);

/* ---- objective without a plan, allocating nothing -----------------------
 * The paper has no counterpart of this entry point.  It is for callers that
 * cannot allocate device memory where they need the objective: code that
 * runs inside a memory pool or arena owning every allocation of the process,
 * code inside a framework that forbids allocation (and its device
 * synchronisation) in its hot loop, or callers whose memory is committed to
 * their own buffers.  tomo_plan allocates tables and workspaces; this call
 * allocates nothing and needs no plan.
 *
 * *f (one double, DEVICE memory) receives f = ||P - F Theta||^2 + gamma
 * sum_n sum_{i<M-1} (Theta_{i,n} - Theta_{i+1,n})^2 in double, with the band
 * of band_k as in tomo_desc.  lambda (D), P (D x N) and Theta (M x N) are
 * DEVICE pointers; lambda need not be sorted, and every entry must be
 * finite and >= 0 (it is in device memory, so the call cannot check it on
 * the host: an invalid entry makes *f NaN).  Work is queued on `stream`
 * (cudaStream_t, NULL: the legacy default stream); the call returns without
 * waiting, f is ready when the stream reaches it.
 *
 * Its only scratch is a static device array of TOMO_NOALLOC_MAX_ROWS doubles
 * (2 MiB) that every device loading the library holds until the library is
 * unloaded; D + M above TOMO_NOALLOC_MAX_ROWS gives TOMO_EINVAL.  The first
 * call on a device looks up that array's device address (make the first call
 * before any stream capture).  All calls share the array: calls whose work
 * overlaps on the GPU (different streams or threads) race and return wrong
 * values; order them on one stream.  2 <= N <= 1024, M, D >= 1. */
#define TOMO_NOALLOC_MAX_ROWS 262144
tomo_status tomo_objective_noalloc(int64_t M, int64_t N, int64_t D, const double *lambda,
                                   double band_k, double gamma, const double *P,
                                   const double *Theta, double *f, void *stream);

/* Message of the last failure on the calling thread ("" if none). */
const char *tomo_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* TOMO_H */
