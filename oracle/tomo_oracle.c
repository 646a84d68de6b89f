/*
 * tomo_oracle.c -- plain FP64 CPU oracle for phase-insensitive quantum
 * detector tomography (Schapeler, Schade, Lass, Plessl, Bartley,
 * "Scalable quantum detector tomography by high-performance computing",
 * arXiv 2404.02844).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  It shares no code,
 * header, table or helper with the CUDA library, and the CUDA library never
 * calls it.
 *
 * What it computes (each function cites the passage it follows):
 *   F_{d,i} = lambda_d^i e^{-lambda_d} / i!                  (Eq. Fmatrix)
 *   f(Theta) = ||P - F Theta||^2 + gamma sum_n sum_{i<M-1}
 *              (Theta_{i,n} - Theta_{i+1,n})^2                (Eq. min, Eq. regul)
 *   G = 2 F^T (F Theta - P) + 2 gamma L Theta, H v = 2 F^T F v + 2 gamma L v
 *   row-wise simplex projection P_{S^M}                        (Eq. Mp1_proj)
 *   two-stage two-metric projected truncated Newton            (Algorithms 1-3)
 *   KKT stopping residual                                      (App. B, KKT criterion)
 *
 * Everything is double precision.  The Poisson weights are evaluated from
 * their definition in long double (lgammal/logl/expl) so that the
 * cancellation in i*ln(lambda) - lambda - ln(i!) at large i does not dominate
 * the double result.  Parallel loops use OpenMP; no blocking, fusion or
 * reordering beyond summing each output in its natural index order.
 *
 * Readings of points the paper leaves open (identical on the GPU side, each
 * listed in the design notes):
 *   band:   F_{d,i} is kept for lo_d <= i <= hi_d with
 *           lo_d = max(0, floor(lambda - k sqrt(lambda))),
 *           hi_d = min(M-1, max(16, ceil(lambda + k sqrt(lambda)))), k > 0;
 *           k <= 0 keeps the full range (dense F).
 *   I set:  eps_k = min(eps_bar, w_k), w_k = || x - P(x - grad) ||_2 with P the
 *           stage's projection (simplex rows in stage 1, max(0,.) in stage 2).
 *   CG:     p0 = 0; stop when ||r|| <= eta ||b||, eta = min(eta_max,
 *           ||b||^eta_pow) (default min(0.5, sqrt(||b||))), or after max_cg
 *           (default 10000, a safety bound: the forcing test is the working
 *           rule) Hessian products; non-descent result ->
 *           p = -grad / diag.
 *   Armijo: accept the smallest m with f(x(beta^m)) <= f(x) + c grad^T
 *           (x(beta^m) - x) (projected-arc form), beta = 3/4, c = 1/10.
 *   switch: |grad^T (x_{k+1} - x_k) / alpha_k| <= 1e-4, or two failed stage-1
 *           line searches in a row.
 *   KKT:    sqrt(mean (Theta (G + lambda_i))^2), lambda_i = max(0, -min_n G_{i,n}).
 *   m(i):   lowest index among the row maxima, recomputed every iteration.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_API __attribute__((visibility("default")))

/* ---------------------------------------------------------------------- */
/* Problem                                                                 */
/* ---------------------------------------------------------------------- */

typedef struct {
    int64_t M, N, D;
    double gamma;
    double band_k;
    double *lam;      /* D */
    int64_t *lo, *hi; /* D: band of probe d, inclusive */
    int64_t *off;     /* D+1: offsets of the stored band values */
    double *F;        /* stored band values (NULL in lazy mode) */
    int64_t *dlo, *dhi; /* M: probes whose band contains i (range to scan) */
} orc_problem;

/* Eq. Fmatrix: F_{d,i} = lambda^i e^{-lambda} / i!, evaluated in log space in
 * long double; lambda = 0 gives the vacuum (F = 1 at i = 0, else 0). */
ORC_API double orc_poisson(int64_t i, double lam)
{
    if (lam == 0.0) return i == 0 ? 1.0 : 0.0;
    long double l = (long double)lam;
    long double lnF = (long double)i * logl(l) - l - lgammal((long double)i + 1.0L);
    return (double)expl(lnF);
}

/* Band of probe d (see the reading above). */
ORC_API void orc_band(int64_t M, double band_k, double lam, int64_t *lo, int64_t *hi)
{
    if (band_k <= 0.0) {
        *lo = 0;
        *hi = M - 1;
        return;
    }
    double s = sqrt(lam);
    double a = floor(lam - band_k * s);
    double b = ceil(lam + band_k * s);
    if (b < 16.0) b = 16.0;
    int64_t l = a < 0.0 ? 0 : (int64_t)a;
    int64_t h = b > (double)(M - 1) ? M - 1 : (int64_t)b;
    if (l > M - 1) l = M; /* empty band: lambda far beyond the cutoff */
    *lo = l;
    *hi = h;
}

ORC_API orc_problem *orc_create(int64_t M, int64_t N, int64_t D, const double *lam,
                                double band_k, double gamma, int store_F)
{
    orc_problem *p = (orc_problem *)calloc(1, sizeof(orc_problem));
    if (!p) return NULL;
    p->M = M; p->N = N; p->D = D; p->gamma = gamma; p->band_k = band_k;
    p->lam = (double *)malloc(sizeof(double) * D);
    p->lo = (int64_t *)malloc(sizeof(int64_t) * D);
    p->hi = (int64_t *)malloc(sizeof(int64_t) * D);
    p->off = (int64_t *)malloc(sizeof(int64_t) * (D + 1));
    p->dlo = (int64_t *)malloc(sizeof(int64_t) * M);
    p->dhi = (int64_t *)malloc(sizeof(int64_t) * M);
    memcpy(p->lam, lam, sizeof(double) * D);
    p->off[0] = 0;
    for (int64_t d = 0; d < D; ++d) {
        orc_band(M, band_k, lam[d], &p->lo[d], &p->hi[d]);
        int64_t cnt = p->hi[d] >= p->lo[d] ? p->hi[d] - p->lo[d] + 1 : 0;
        p->off[d + 1] = p->off[d] + cnt;
    }
    if (store_F) {
        for (int64_t i = 0; i < M; ++i) { p->dlo[i] = D; p->dhi[i] = -1; }
        for (int64_t d = 0; d < D; ++d)
            for (int64_t i = p->lo[d]; i <= p->hi[d]; ++i) {
                if (d < p->dlo[i]) p->dlo[i] = d;
                if (d > p->dhi[i]) p->dhi[i] = d;
            }
    } else {
        /* lazy mode (sampled outputs only): scan every probe */
        for (int64_t i = 0; i < M; ++i) { p->dlo[i] = 0; p->dhi[i] = D - 1; }
    }
    if (store_F) {
        p->F = (double *)malloc(sizeof(double) * (p->off[D] > 0 ? p->off[D] : 1));
        if (!p->F) { free(p); return NULL; }
#pragma omp parallel for schedule(dynamic, 4)
        for (int64_t d = 0; d < D; ++d)
            for (int64_t i = p->lo[d]; i <= p->hi[d]; ++i)
                p->F[p->off[d] + i - p->lo[d]] = orc_poisson(i, p->lam[d]);
    }
    return p;
}

ORC_API void orc_destroy(orc_problem *p)
{
    if (!p) return;
    free(p->lam); free(p->lo); free(p->hi); free(p->off);
    free(p->dlo); free(p->dhi); free(p->F); free(p);
}

ORC_API int64_t orc_band_nnz(const orc_problem *p) { return p->off[p->D]; }
ORC_API void orc_bands(const orc_problem *p, int64_t *lo, int64_t *hi)
{
    memcpy(lo, p->lo, sizeof(int64_t) * p->D);
    memcpy(hi, p->hi, sizeof(int64_t) * p->D);
}

static inline double Fval(const orc_problem *p, int64_t d, int64_t i)
{
    if (i < p->lo[d] || i > p->hi[d]) return 0.0;
    if (p->F) return p->F[p->off[d] + i - p->lo[d]];
    return orc_poisson(i, p->lam[d]);
}

/* Dense D x M copy of F (Eq. Fmatrix, zero outside the bands). */
ORC_API void orc_dense_F(const orc_problem *p, double *out)
{
    const int64_t M = p->M;
#pragma omp parallel for
    for (int64_t d = 0; d < p->D; ++d)
        for (int64_t i = 0; i < M; ++i) out[d * M + i] = Fval(p, d, i);
}

/* ---------------------------------------------------------------------- */
/* Products with F (Table ops: objective / gradient / Hessian products)    */
/* ---------------------------------------------------------------------- */

/* O = F X, O is D x N, X is M x N (row-major). */
ORC_API void orc_apply_F(const orc_problem *p, const double *X, double *O)
{
    const int64_t N = p->N;
#pragma omp parallel for schedule(dynamic, 8)
    for (int64_t d = 0; d < p->D; ++d) {
        double *restrict o = O + d * N;
        for (int64_t n = 0; n < N; ++n) o[n] = 0.0;
        for (int64_t i = p->lo[d]; i <= p->hi[d]; ++i) {
            const double f = Fval(p, d, i);
            const double *restrict x = X + i * N;
            for (int64_t n = 0; n < N; ++n) o[n] += f * x[n];
        }
    }
}

/* Rows `rows[k]` of O = F X only (out: nrows x N). */
ORC_API void orc_apply_F_rows(const orc_problem *p, const double *X, const int64_t *rows,
                              int64_t nrows, double *out)
{
    const int64_t N = p->N;
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t k = 0; k < nrows; ++k) {
        const int64_t d = rows[k];
        double *o = out + k * N;
        for (int64_t n = 0; n < N; ++n) o[n] = 0.0;
        for (int64_t i = p->lo[d]; i <= p->hi[d]; ++i) {
            double f = Fval(p, d, i);
            const double *x = X + i * N;
            for (int64_t n = 0; n < N; ++n) o[n] += f * x[n];
        }
    }
}

/* Rows `rows[k]` of Z = F^T Y only (out: nrows x N). */
ORC_API void orc_apply_Ft_rows(const orc_problem *p, const double *Y, const int64_t *rows,
                               int64_t nrows, double *out)
{
    const int64_t N = p->N;
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t k = 0; k < nrows; ++k) {
        const int64_t i = rows[k];
        double *z = out + k * N;
        for (int64_t n = 0; n < N; ++n) z[n] = 0.0;
        for (int64_t d = p->dlo[i]; d <= p->dhi[i]; ++d) {
            if (i < p->lo[d] || i > p->hi[d]) continue;
            double f = Fval(p, d, i);
            const double *y = Y + d * N;
            for (int64_t n = 0; n < N; ++n) z[n] += f * y[n];
        }
    }
}

/* Z = F^T Y, Z is M x N, Y is D x N. */
ORC_API void orc_apply_Ft(const orc_problem *p, const double *Y, double *Z)
{
    const int64_t N = p->N;
#pragma omp parallel for schedule(dynamic, 8)
    for (int64_t i = 0; i < p->M; ++i) {
        double *restrict z = Z + i * N;
        for (int64_t n = 0; n < N; ++n) z[n] = 0.0;
        for (int64_t d = p->dlo[i]; d <= p->dhi[i]; ++d) {
            if (i < p->lo[d] || i > p->hi[d]) continue;
            const double f = Fval(p, d, i);
            const double *restrict y = Y + d * N;
            for (int64_t n = 0; n < N; ++n) z[n] += f * y[n];
        }
    }
}

/* Eq. regul: g = gamma sum_n sum_{i=0}^{M-2} (X_{i,n} - X_{i+1,n})^2 */
ORC_API double orc_regulariser(const orc_problem *p, const double *X)
{
    const int64_t M = p->M, N = p->N;
    double s = 0.0;
#pragma omp parallel for reduction(+ : s)
    for (int64_t i = 0; i < M - 1; ++i)
        for (int64_t n = 0; n < N; ++n) {
            double t = X[i * N + n] - X[(i + 1) * N + n];
            s += t * t;
        }
    return p->gamma * s;
}

/* Y += 2 gamma L X, with (L X)_i = (X_i - X_{i+1})[i<M-1] + (X_i - X_{i-1})[i>0],
 * the derivative of Eq. regul. */
static void add_2gammaL(const orc_problem *p, const double *X, double *Y)
{
    const int64_t M = p->M, N = p->N;
    const double g2 = 2.0 * p->gamma;
    if (p->gamma == 0.0) return;
#pragma omp parallel for
    for (int64_t i = 0; i < M; ++i)
        for (int64_t n = 0; n < N; ++n) {
            double lx = 0.0;
            if (i < M - 1) lx += X[i * N + n] - X[(i + 1) * N + n];
            if (i > 0) lx += X[i * N + n] - X[(i - 1) * N + n];
            Y[i * N + n] += g2 * lx;
        }
}

/* Eq. min + Eq. regul: f = ||P - F Theta||^2 + g(Theta).  R (D x N, may be
 * NULL) receives F Theta - P. */
ORC_API double orc_objective(const orc_problem *p, const double *P, const double *Th,
                             double *R_out)
{
    const int64_t DN = p->D * p->N;
    double *O = R_out ? R_out : (double *)malloc(sizeof(double) * DN);
    orc_apply_F(p, Th, O);
    double s = 0.0;
#pragma omp parallel for reduction(+ : s)
    for (int64_t k = 0; k < DN; ++k) {
        O[k] -= P[k];
        s += O[k] * O[k];
    }
    if (!R_out) free(O);
    return s + orc_regulariser(p, Th);
}

/* Gradient of f (Table ops, "gradient"): G = 2 F^T (F Theta - P) + 2 gamma L Theta.
 * Returns f. */
ORC_API double orc_gradient(const orc_problem *p, const double *P, const double *Th,
                            double *G)
{
    const int64_t DN = p->D * p->N, MN = p->M * p->N;
    double *R = (double *)malloc(sizeof(double) * DN);
    double f = orc_objective(p, P, Th, R);
    orc_apply_Ft(p, R, G);
#pragma omp parallel for
    for (int64_t k = 0; k < MN; ++k) G[k] *= 2.0;
    add_2gammaL(p, Th, G);
    free(R);
    return f;
}

/* Hessian product (Table ops, "Hessian products"): H V = 2 F^T F V + 2 gamma L V. */
ORC_API void orc_hvp(const orc_problem *p, const double *V, double *HV)
{
    const int64_t DN = p->D * p->N, MN = p->M * p->N;
    double *O = (double *)malloc(sizeof(double) * DN);
    orc_apply_F(p, V, O);
    orc_apply_Ft(p, O, HV);
#pragma omp parallel for
    for (int64_t k = 0; k < MN; ++k) HV[k] *= 2.0;
    add_2gammaL(p, V, HV);
    free(O);
}

/* Diagonal of the Hessian (Table ops): h_i = 2 sum_d F_{d,i}^2 + 2 gamma L_ii,
 * the same for every column n. */
ORC_API void orc_hess_diag(const orc_problem *p, double *h)
{
    const int64_t M = p->M;
#pragma omp parallel for
    for (int64_t i = 0; i < M; ++i) {
        double s = 0.0;
        for (int64_t d = p->dlo[i]; d <= p->dhi[i]; ++d) {
            if (i < p->lo[d] || i > p->hi[d]) continue;
            double f = Fval(p, d, i);
            s += f * f;
        }
        double lii = (double)((i > 0) + (i < M - 1));
        h[i] = 2.0 * s + 2.0 * p->gamma * lii;
    }
}

/* ---------------------------------------------------------------------- */
/* Simplex projection (Eq. Mp1_proj)                                       */
/* ---------------------------------------------------------------------- */

static int cmp_desc(const void *a, const void *b)
{
    double x = *(const double *)a, y = *(const double *)b;
    return (x < y) - (x > y);
}

/* Euclidean projection of x (length n) onto {y >= 0, sum y = 1}: sort-based
 * closed form (Held, Wolfe & Crowder 1974): with u sorted descending, rho is
 * the largest k with u_k - (sum_{j<=k} u_j - 1)/k > 0 and
 * tau = (sum_{j<=rho} u_j - 1)/rho; y = max(x - tau, 0). */
ORC_API void orc_project_simplex_sort(const double *x, int64_t n, double *y)
{
    double *u = (double *)malloc(sizeof(double) * n);
    memcpy(u, x, sizeof(double) * n);
    qsort(u, (size_t)n, sizeof(double), cmp_desc);
    double cum = 0.0, tau = 0.0;
    for (int64_t k = 0; k < n; ++k) {
        cum += u[k];
        double t = (cum - 1.0) / (double)(k + 1);
        if (u[k] - t > 0.0) tau = t;
    }
    for (int64_t k = 0; k < n; ++k) {
        double v = x[k] - tau;
        y[k] = v > 0.0 ? v : 0.0;
    }
    free(u);
}

/* The same projection by Condat's algorithm (Condat 2016, "Fast projection
 * onto the simplex and the l1 ball"), the method the paper uses: a running
 * estimate rho of the threshold over a candidate list, a second pass over the
 * values set aside, then removal of candidates below the threshold until
 * nothing changes.  Used only as a cross-check of the sort-based form. */
ORC_API void orc_project_simplex_condat(const double *x, int64_t n, double *y)
{
    double *v = (double *)malloc(sizeof(double) * n);
    double *vt = (double *)malloc(sizeof(double) * n);
    int64_t nv = 0, nvt = 0;
    v[nv++] = x[0];
    double rho = x[0] - 1.0;
    for (int64_t k = 1; k < n; ++k) {
        double yk = x[k];
        if (yk > rho) {
            rho += (yk - rho) / (double)(nv + 1);
            if (rho > yk - 1.0) {
                v[nv++] = yk;
            } else {
                for (int64_t j = 0; j < nv; ++j) vt[nvt++] = v[j];
                nv = 0;
                v[nv++] = yk;
                rho = yk - 1.0;
            }
        }
    }
    for (int64_t j = 0; j < nvt; ++j) {
        double yk = vt[j];
        if (yk > rho) {
            v[nv++] = yk;
            rho += (yk - rho) / (double)nv;
        }
    }
    int changed = 1;
    while (changed) {
        changed = 0;
        int64_t w = 0, cur = nv;
        for (int64_t j = 0; j < nv; ++j) {
            double yk = v[j];
            if (yk <= rho && cur > 1) {
                /* remove yk; the threshold over the |v|-1 survivors grows */
                cur -= 1;
                rho += (rho - yk) / (double)cur;
                changed = 1;
            } else {
                v[w++] = yk;
            }
        }
        nv = w;
    }
    for (int64_t k = 0; k < n; ++k) {
        double t = x[k] - rho;
        y[k] = t > 0.0 ? t : 0.0;
    }
    free(v);
    free(vt);
}

/* P_{S^M}: every row of X (M x N) projected onto the simplex. */
ORC_API void orc_project_rows(const orc_problem *p, const double *X, double *Y)
{
#pragma omp parallel for
    for (int64_t i = 0; i < p->M; ++i)
        orc_project_simplex_sort(X + i * p->N, p->N, Y + i * p->N);
}

/* KKT residual (App. B, convergence criterion of stage 2). */
ORC_API double orc_kkt(const orc_problem *p, const double *Th, const double *G)
{
    const int64_t M = p->M, N = p->N;
    double s = 0.0;
#pragma omp parallel for reduction(+ : s)
    for (int64_t i = 0; i < M; ++i) {
        double mn = G[i * N];
        for (int64_t n = 1; n < N; ++n)
            if (G[i * N + n] < mn) mn = G[i * N + n];
        double lam = -mn > 0.0 ? -mn : 0.0;
        for (int64_t n = 0; n < N; ++n) {
            double t = Th[i * N + n] * (G[i * N + n] + lam);
            s += t * t;
        }
    }
    return sqrt(s / ((double)N * (double)M));
}

/* Frank-Wolfe duality gap of a feasible Theta: f is convex on the product of
 * row simplices, so for every feasible Theta', f(Theta') >= f(Theta) +
 * <G, Theta' - Theta>, whose minimum over the simplices puts each row's mass
 * on its smallest gradient entry.  Hence
 *     f(Theta) - f* <= sum_i ( <G_i, Theta_i> - min_n G_{i,n} ),
 * a certificate of the optimum that needs no knowledge of f*. */
ORC_API double orc_fw_gap(const orc_problem *p, const double *Th, const double *G)
{
    const int64_t M = p->M, N = p->N;
    double s = 0.0;
#pragma omp parallel for reduction(+ : s)
    for (int64_t i = 0; i < M; ++i) {
        double mn = G[i * N], dot = 0.0;
        for (int64_t n = 0; n < N; ++n) {
            if (G[i * N + n] < mn) mn = G[i * N + n];
            dot += G[i * N + n] * Th[i * N + n];
        }
        s += dot - mn;
    }
    return s;
}

/* Long-range smoothing (Eq. smoothing): for i >= exclude,
 *   Y_{i,n} = mean of X_{j,n} over j in [i - w, i + w], w = floor(i / div),
 * the window clipped to [0, M-1] (the mean is then over the rows present);
 * rows i < exclude are copied.  A mean of simplex rows is a simplex row. */
ORC_API void orc_smooth(const orc_problem *p, const double *X, double *Y, int64_t exclude,
                        double div)
{
    const int64_t M = p->M, N = p->N;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < M; ++i) {
        if (i < exclude) {
            for (int64_t n = 0; n < N; ++n) Y[i * N + n] = X[i * N + n];
            continue;
        }
        const int64_t w = (int64_t)floor((double)i / div);
        const int64_t a = i - w < 0 ? 0 : i - w;
        const int64_t b = i + w > M - 1 ? M - 1 : i + w;
        for (int64_t n = 0; n < N; ++n) {
            double s = 0.0;
            for (int64_t j = a; j <= b; ++j) s += X[j * N + n];
            Y[i * N + n] = s / (double)(b - a + 1);
        }
    }
}

/* ---------------------------------------------------------------------- */
/* Two-stage two-metric projected truncated Newton (Algorithms 1, 2, 3)    */
/* ---------------------------------------------------------------------- */

typedef struct {
    double eps_kkt;      /* KKT stopping threshold */
    double eps_bar;      /* upper bound of eps_k in the index set I */
    double beta;         /* backtracking factor, 3/4 */
    double c;            /* Armijo constant, 1/10 */
    double switch_tol;   /* stage-1 -> stage-2 switch threshold, 1e-4 */
    double f_target;     /* > 0: stop as soon as f <= f_target */
    int64_t max_newton;  /* cap on Newton iterations (both stages) */
    int64_t max_stage1;  /* cap on stage-1 iterations */
    int64_t max_cg;      /* cap on Hessian products per Newton iteration */
    int64_t ls_max;      /* cap on backtracking steps */
    int64_t start_stage; /* 1: Algorithm 3; 2: stage 2 only (Algorithm 1) */
    int64_t warm_start;  /* 0: Theta^(0) = 1/N, 1: use Theta as given */
    int64_t stall_iters; /* stop after this many iterations without decrease */
    double cg_eta_max;   /* CG forcing term eta = min(cg_eta_max, ||b||^cg_eta_pow) */
    double cg_eta_pow;
} orc_opts;

typedef struct {
    double f, kkt;
    int64_t iters_s1, iters_s2, cg_total, ls_total;
    int64_t status; /* 0 KKT reached, 1 f_target reached, 2 iteration cap,
                       3 stagnated (no decrease / line search failed) */
    int64_t stage_end;
} orc_report;

ORC_API void orc_default_opts(orc_opts *o)
{
    o->eps_kkt = 1e-10;
    o->eps_bar = 1e-6;
    o->beta = 0.75;
    o->c = 0.1;
    o->switch_tol = 1e-4;
    o->f_target = 0.0;
    o->max_newton = 1000;
    o->max_stage1 = 200;
    o->max_cg = 10000;
    o->ls_max = 50;
    o->start_stage = 1;
    o->warm_start = 0;
    o->stall_iters = 5;
    o->cg_eta_max = 0.5;
    o->cg_eta_pow = 0.5;
}

typedef struct {
    double *G, *g, *diag, *x, *r, *z, *pv, *q, *dir, *trial, *tmp, *hq;
    uint8_t *freem, *var;
    int64_t *mrow;
    double *h;
} orc_work;

static double dot(const double *a, const double *b, int64_t n)
{
    double s = 0.0;
#pragma omp parallel for reduction(+ : s)
    for (int64_t k = 0; k < n; ++k) s += a[k] * b[k];
    return s;
}

/* Apply the modified Hessian D^(k) restricted to the free variables
 * (Algorithm 1 / 2, "solve D P = G"): stage 1 uses H itself; stage 2 uses the
 * Hessian in the reduced variables, E^T H E, where E lifts a reduced vector by
 * filling column m(i) with minus the row sum of the others. */
static void apply_D_free(const orc_problem *p, int stage, const orc_work *w,
                         const double *v, double *q)
{
    const int64_t M = p->M, N = p->N, MN = M * N;
    if (stage == 1) {
        orc_hvp(p, v, q);
    } else {
        for (int64_t i = 0; i < M; ++i) {
            double s = 0.0;
            for (int64_t n = 0; n < N; ++n) {
                w->tmp[i * N + n] = v[i * N + n];
                if (n != w->mrow[i]) s += v[i * N + n];
            }
            w->tmp[i * N + w->mrow[i]] = -s;
        }
        orc_hvp(p, w->tmp, w->hq);
        for (int64_t i = 0; i < M; ++i) {
            double qm = w->hq[i * N + w->mrow[i]];
            for (int64_t n = 0; n < N; ++n)
                q[i * N + n] = (n == w->mrow[i]) ? 0.0 : w->hq[i * N + n] - qm;
        }
    }
    for (int64_t k = 0; k < MN; ++k)
        if (!w->freem[k]) q[k] = 0.0;
}

/* Newton direction of one iteration: diagonally preconditioned CG on the
 * free variables, -g/diag on the set I (two-metric D^(k) of Bertsekas). */
static int64_t newton_direction(const orc_problem *p, int stage, orc_work *w,
                                const orc_opts *o)
{
    const int64_t MN = p->M * p->N;
    for (int64_t k = 0; k < MN; ++k) {
        w->x[k] = 0.0;
        w->r[k] = w->freem[k] ? -w->g[k] : 0.0;
        w->z[k] = w->freem[k] ? w->r[k] / w->diag[k] : 0.0;
        w->pv[k] = w->z[k];
    }
    double bn = sqrt(dot(w->r, w->r, MN));
    /* forcing term: min(eta_max, ||b||^eta_pow); the default 0.5, 0.5 is the
     * truncated-Newton choice min(0.5, sqrt||b||) */
    double pw;
    if (o->cg_eta_pow == 0.5) pw = sqrt(bn);
    else if (o->cg_eta_pow == 1.0) pw = bn;
    else if (o->cg_eta_pow == 0.0) pw = 1.0;
    else pw = pow(bn, o->cg_eta_pow);
    double eta = pw < o->cg_eta_max ? pw : o->cg_eta_max;
    double tol = eta * bn;
    double rz = dot(w->r, w->z, MN);
    int64_t it = 0;
    for (; it < o->max_cg; ++it) {
        double rn = sqrt(dot(w->r, w->r, MN));
        if (rn <= tol) break;
        apply_D_free(p, stage, w, w->pv, w->q);
        double pq = dot(w->pv, w->q, MN);
        if (!(pq > 0.0)) break;
        double a = rz / pq;
        for (int64_t k = 0; k < MN; ++k) {
            w->x[k] += a * w->pv[k];
            w->r[k] -= a * w->q[k];
            w->z[k] = w->freem[k] ? w->r[k] / w->diag[k] : 0.0;
        }
        double rz_new = dot(w->r, w->z, MN);
        double b = rz_new / rz;
        rz = rz_new;
        for (int64_t k = 0; k < MN; ++k) w->pv[k] = w->z[k] + b * w->pv[k];
    }
    for (int64_t k = 0; k < MN; ++k) {
        if (!w->var[k]) w->dir[k] = 0.0;
        else if (w->freem[k]) w->dir[k] = w->x[k];
        else w->dir[k] = -w->g[k] / w->diag[k];
    }
    /* a direction that does not descend is replaced by the scaled gradient */
    if (!(dot(w->g, w->dir, MN) < 0.0))
        for (int64_t k = 0; k < MN; ++k)
            w->dir[k] = w->var[k] ? -w->g[k] / w->diag[k] : 0.0;
    return it;
}

/* Line search of Algorithm 2 (stage 1) or Algorithm 1 (stage 2) along dir,
 * Armijo rule of App. B.  On success Theta <- trial, returns 1. */
static int line_search(const orc_problem *p, int stage, const double *P, double *Th,
                       double f, orc_work *w, const orc_opts *o, double *f_new,
                       double *gts_out, double *alpha_out, int64_t *ls_count)
{
    const int64_t M = p->M, N = p->N, MN = M * N;
    double alpha = 1.0;
    for (int64_t m = 0; m < o->ls_max; ++m, alpha *= o->beta) {
        ++*ls_count;
        if (stage == 1) {
            for (int64_t k = 0; k < MN; ++k) w->tmp[k] = Th[k] + alpha * w->dir[k];
            orc_project_rows(p, w->tmp, w->trial);
        } else {
            int neg = 0;
            for (int64_t i = 0; i < M; ++i) {
                double s = 0.0;
                for (int64_t n = 0; n < N; ++n) {
                    if (n == w->mrow[i]) continue;
                    double t = Th[i * N + n] + alpha * w->dir[i * N + n];
                    t = t > 0.0 ? t : 0.0;
                    w->trial[i * N + n] = t;
                    s += t;
                }
                double tm = 1.0 - s;
                w->trial[i * N + w->mrow[i]] = tm;
                if (tm < 0.0) neg = 1;
            }
            if (neg) continue; /* implicit entries must stay non-negative */
        }
        double gts = 0.0;
        for (int64_t k = 0; k < MN; ++k)
            if (w->var[k]) gts += w->g[k] * (w->trial[k] - Th[k]);
        double ft = orc_objective(p, P, w->trial, NULL);
        if (ft <= f + o->c * gts) {
            memcpy(Th, w->trial, sizeof(double) * MN);
            *f_new = ft;
            *gts_out = gts;
            *alpha_out = alpha;
            return 1;
        }
    }
    return 0;
}

/* Set up one Newton iteration of the given stage: gradient in the stage's
 * variables (g), variable mask, eps_k, the index set I (free mask) and the
 * diagonal of D^(k). */
static void setup_iteration(const orc_problem *p, int stage, const double *Th,
                            orc_work *w, const orc_opts *o)
{
    const int64_t M = p->M, N = p->N, MN = M * N;
    if (stage == 1) {
        for (int64_t k = 0; k < MN; ++k) {
            w->g[k] = w->G[k];
            w->var[k] = 1;
            w->tmp[k] = Th[k] - w->G[k];
        }
        orc_project_rows(p, w->tmp, w->trial);
        double s = 0.0;
        for (int64_t k = 0; k < MN; ++k) {
            double t = Th[k] - w->trial[k];
            s += t * t;
        }
        double eps = sqrt(s) < o->eps_bar ? sqrt(s) : o->eps_bar;
        for (int64_t i = 0; i < M; ++i)
            for (int64_t n = 0; n < N; ++n) {
                int64_t k = i * N + n;
                int inI = Th[k] <= eps && w->g[k] > 0.0;
                w->freem[k] = !inI;
                w->diag[k] = w->h[i];
            }
    } else {
        /* transformation step: m(i) = argmax_n Theta_{i,n} (lowest index) */
        for (int64_t i = 0; i < M; ++i) {
            int64_t m = 0;
            for (int64_t n = 1; n < N; ++n)
                if (Th[i * N + n] > Th[i * N + m]) m = n;
            w->mrow[i] = m;
        }
        double s = 0.0;
        for (int64_t i = 0; i < M; ++i) {
            double gm = w->G[i * N + w->mrow[i]];
            for (int64_t n = 0; n < N; ++n) {
                int64_t k = i * N + n;
                if (n == w->mrow[i]) {
                    w->g[k] = 0.0;
                    w->var[k] = 0;
                } else {
                    w->g[k] = w->G[k] - gm;
                    w->var[k] = 1;
                    double pr = Th[k] - w->g[k];
                    pr = pr > 0.0 ? pr : 0.0;
                    s += (Th[k] - pr) * (Th[k] - pr);
                }
            }
        }
        double eps = sqrt(s) < o->eps_bar ? sqrt(s) : o->eps_bar;
        for (int64_t i = 0; i < M; ++i)
            for (int64_t n = 0; n < N; ++n) {
                int64_t k = i * N + n;
                int inI = Th[k] <= eps && w->g[k] > 0.0;
                w->freem[k] = w->var[k] && !inI;
                w->diag[k] = 2.0 * w->h[i];
            }
    }
}

/* Algorithm 3: stage 1 (Algorithm 2) from Theta^(0) = 1/N, then stage 2
 * (Algorithm 1) until the KKT residual is below eps_kkt.  Theta (M x N) is
 * updated in place; f_hist (may be NULL, capacity max_newton + 1) receives
 * f(Theta^(k)) at the start of every iteration and the final value. */
ORC_API int64_t orc_fit(const orc_problem *p, const double *P, double *Th,
                        const orc_opts *o, orc_report *rep, double *f_hist)
{
    const int64_t M = p->M, N = p->N, MN = M * N;
    orc_work w;
    double **bufs[] = {&w.G, &w.g, &w.diag, &w.x, &w.r, &w.z, &w.pv, &w.q,
                       &w.dir, &w.trial, &w.tmp, &w.hq};
    for (size_t b = 0; b < sizeof(bufs) / sizeof(bufs[0]); ++b)
        *bufs[b] = (double *)calloc((size_t)MN, sizeof(double));
    w.freem = (uint8_t *)calloc((size_t)MN, 1);
    w.var = (uint8_t *)calloc((size_t)MN, 1);
    w.mrow = (int64_t *)calloc((size_t)M, sizeof(int64_t));
    w.h = (double *)calloc((size_t)M, sizeof(double));
    orc_hess_diag(p, w.h);

    if (!o->warm_start)
        for (int64_t k = 0; k < MN; ++k) Th[k] = 1.0 / (double)N;

    memset(rep, 0, sizeof(*rep));
    int stage = o->start_stage == 2 ? 2 : 1;
    int64_t stall = 0, nh = 0;
    double f = 0.0, kkt = 0.0;
    rep->status = 2;
    for (int64_t k = 0; k < o->max_newton; ++k) {
        f = orc_gradient(p, P, Th, w.G);
        kkt = orc_kkt(p, Th, w.G);
        if (f_hist) f_hist[nh++] = f;
        if (kkt <= o->eps_kkt) { rep->status = 0; break; }
        if (o->f_target > 0.0 && f <= o->f_target) { rep->status = 1; break; }
        if (stage == 1 && rep->iters_s1 >= o->max_stage1) stage = 2;

        setup_iteration(p, stage, Th, &w, o);
        rep->cg_total += newton_direction(p, stage, &w, o);
        if (stage == 1) rep->iters_s1++; else rep->iters_s2++;

        double f_new = f, gts = 0.0, alpha = 0.0;
        int ok = line_search(p, stage, P, Th, f, &w, o, &f_new, &gts, &alpha, &rep->ls_total);
        if (!ok) {
            /* fallback: scaled gradient direction on the stage's variables */
            for (int64_t q = 0; q < MN; ++q)
                w.dir[q] = w.var[q] ? -w.g[q] / w.diag[q] : 0.0;
            ok = line_search(p, stage, P, Th, f, &w, o, &f_new, &gts, &alpha, &rep->ls_total);
        }
        if (!ok) {
            if (stage == 1) { stage = 2; continue; }
            rep->status = 3;
            break;
        }
        if (stage == 1 && fabs(gts / alpha) <= o->switch_tol) stage = 2;
        if (!(f_new < f * (1.0 - 1e-15))) {
            if (++stall >= o->stall_iters) {
                f = f_new;
                rep->status = 3;
                break;
            }
        } else {
            stall = 0;
        }
    }
    /* final state */
    f = orc_gradient(p, P, Th, w.G);
    kkt = orc_kkt(p, Th, w.G);
    if (f_hist) f_hist[nh++] = f;
    rep->f = f;
    rep->kkt = kkt;
    rep->stage_end = stage;
    for (size_t b = 0; b < sizeof(bufs) / sizeof(bufs[0]); ++b) free(*bufs[b]);
    free(w.freem); free(w.var); free(w.mrow); free(w.h);
    return nh;
}

ORC_API int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
