// rowops.cu -- row-wise and element-wise kernels of the two-stage two-metric
// projected truncated Newton solver (App. B, Algorithms 1-3): the simplex
// projection P_{S^M} (Eq. Mp1_proj), the row maxima m(i) of the transformation
// step, the index set I and the diagonal of D^(k), the preconditioned-CG vector
// updates, the line-search trial points with their Armijo terms, the KKT
// residual and the regulariser (Eq. regul).
//
// One warp owns one row of N <= MAX_N outcomes (each lane VPL values held in
// registers); rows are distributed grid-stride over a bounded grid so the
// number of per-CTA partial sums stays small.  Every reduction ends in the
// deterministic last-CTA finalisation of grid_reduce.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <type_traits>

#include "tomo_device.cuh"
#include "tomo_internal.cuh"

namespace tomo {

struct RowArgs {
    int64_t M, N;
    double gamma;
    const double *h;     // Hessian diagonal (M)
    const float *hinv;   // float 1/h (M) then 1/(2h) (M)
    double *partials;
    int64_t pstride;
    DevScalars *sc;
};

static RowArgs row_args(Plan &p)
{
    RowArgs a;
    a.M = p.M; a.N = p.N; a.gamma = p.gamma; a.h = p.h; a.hinv = p.hinv_f;
    a.partials = p.partials; a.pstride = p.max_partials; a.sc = p.sc;
    return a;
}

// Threshold tau of the projection of one row onto the probability simplex,
// y = max(x - tau, 0), by the fixed-point iteration of Michelot (1986): start
// from all entries, set tau = (sum of the kept entries - 1) / (number kept),
// keep the entries above tau, repeat until the kept set stops shrinking.  The
// set shrinks monotonically and always keeps the maximum, so at most N passes.
template <int VPL>
__device__ __forceinline__ double simplex_tau(const double (&y)[VPL], int64_t N, int lane)
{
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < VPL; ++k)
        if (lane + 32 * k < N) s += y[k];
    s = warp_sum(s);
    int cnt = int(N);
    double tau = (s - 1.0) / double(cnt);
    for (int it = 0; it <= int(N) + 1; ++it) {
        double sk = 0.0;
        int ck = 0;
#pragma unroll
        for (int k = 0; k < VPL; ++k)
            if (lane + 32 * k < N && y[k] > tau) { sk += y[k]; ++ck; }
        sk = warp_sum(sk);
        ck = warp_sum_int(ck);
        if (ck == cnt || ck == 0) break;
        cnt = ck;
        tau = (sk - 1.0) / double(cnt);
    }
    return tau;
}

// Lowest index n of the row maximum (ties -> lowest index).
template <int VPL>
__device__ __forceinline__ int row_argmax(const double (&x)[VPL], int64_t N, int lane)
{
    double best = -INFINITY;
    int bi = INT32_MAX;
#pragma unroll
    for (int k = 0; k < VPL; ++k) {
        const int n = lane + 32 * k;
        if (n < N && (x[k] > best)) { best = x[k]; bi = n; }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const double ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
    }
    return bi < N ? bi : 0;  // a row without any ordered value keeps column 0
}

template <int VPL, typename T>
__device__ __forceinline__ void load_row(const T *src, int64_t i, int64_t N, int lane, T (&v)[VPL])
{
#pragma unroll
    for (int k = 0; k < VPL; ++k) {
        const int64_t n = lane + 32 * k;
        v[k] = n < N ? src[i * N + n] : T(0);
    }
}

template <int VPL>
__device__ __forceinline__ void store_row(double *dst, int64_t i, int64_t N, int lane,
                                          const double (&v)[VPL])
{
#pragma unroll
    for (int k = 0; k < VPL; ++k) {
        const int64_t n = lane + 32 * k;
        if (n < N) dst[i * N + n] = v[k];
    }
}

#define ROW_LOOP_BEGIN                                                            \
    const int lane = threadIdx.x & 31;                                           \
    const int64_t warp0 = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5; \
    const int64_t nwarp = (int64_t(gridDim.x) * blockDim.x) >> 5;                \
    for (int64_t i = warp0; i < a.M; i += nwarp) {
#define ROW_LOOP_END }

// ---------------------------------------------------------------------------
// Sparsified start of a warm-started fit: in every row the entries below rel
// x the row's largest become 0 and the row is rescaled to sum 1 (rows of a
// softmax have no exact zeros).  Warp per row.
// ---------------------------------------------------------------------------
template <int VPL>
__global__ void k_zero_small_rows(RowArgs a, double *X, double rel)
{
    ROW_LOOP_BEGIN
    double x[VPL];
    load_row<VPL>(X, i, a.N, lane, x);
    double mx = 0.0;
#pragma unroll
    for (int k = 0; k < VPL; ++k) mx = fmax(mx, x[k]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < VPL; ++k) {
        if (x[k] < rel * mx) x[k] = 0.0;
        s += x[k];
    }
    s = warp_sum(s);
    if (s > 0.0) {
#pragma unroll
        for (int k = 0; k < VPL; ++k) x[k] /= s;
        store_row<VPL>(X, i, a.N, lane, x);
    }
    ROW_LOOP_END
}

// ---------------------------------------------------------------------------
// Projection of every row onto the simplex (Eq. Mp1_proj).
// ---------------------------------------------------------------------------
template <int VPL>
__global__ void k_project_rows(RowArgs a, const double *X, double *Y)
{
    ROW_LOOP_BEGIN
    double y[VPL];
    load_row<VPL>(X, i, a.N, lane, y);
    const double tau = simplex_tau<VPL>(y, a.N, lane);
#pragma unroll
    for (int k = 0; k < VPL; ++k) y[k] = fmax(y[k] - tau, 0.0);
    store_row<VPL>(Y, i, a.N, lane, y);
    ROW_LOOP_END
}

// ---------------------------------------------------------------------------
// KKT residual of App. B: sum over rows of (Theta (G + lambda_i))^2 with
// lambda_i = max(0, -min_n G_{i,n}).
// ---------------------------------------------------------------------------
template <int VPL>
__device__ __forceinline__ double kkt_row(const double (&th)[VPL], const double (&G)[VPL],
                                          int64_t N, int lane)
{
    double mn = INFINITY;
#pragma unroll
    for (int k = 0; k < VPL; ++k)
        if (lane + 32 * k < N) mn = fmin(mn, G[k]);
    mn = warp_min(mn);
    const double lam = -mn > 0.0 ? -mn : 0.0;
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < VPL; ++k)
        if (lane + 32 * k < N) {
            const double t = th[k] * (G[k] + lam);
            s += t * t;
        }
    return s;
}

template <int VPL>
__global__ void k_kkt(RowArgs a, const double *Th, const double *G)
{
    double acc = 0.0;
    ROW_LOOP_BEGIN
    double th[VPL], g[VPL];
    load_row<VPL>(Th, i, a.N, lane, th);
    load_row<VPL>(G, i, a.N, lane, g);
    acc += kkt_row<VPL>(th, g, a.N, lane);
    ROW_LOOP_END
    double v[1] = {acc};  // per-lane partial sums
    DevScalars *sc = a.sc;
    grid_reduce<1>(v, a.partials, a.pstride, &sc->ticket[0], [sc](const double *t) { sc->kkt2 = t[0]; });
}

// ---------------------------------------------------------------------------
// Newton iteration set-up, part 1: KKT residual, the stage's gradient g and
// variable mask, and w_k = ||x - P(x - g)|| for eps_k = min(eps_bar, w_k).
// Stage 1 (Algorithm 2): variables Theta, g = G, P = simplex rows.
// Stage 2 (Algorithm 1): m(i) = argmax_n Theta_{i,n}; variables Theta_{i,n},
// n != m(i); reduced gradient g_{i,n} = G_{i,n} - G_{i,m(i)}; P = max(0, .).
// ---------------------------------------------------------------------------
template <int VPL>
__global__ void k_setup1(RowArgs a, int stage, double eps_bar, const double *Th, const double *G,
                         double *g, uint8_t *var, int32_t *mrow)
{
    double kk = 0.0, ww = 0.0;
    ROW_LOOP_BEGIN
    double th[VPL], gg[VPL];
    load_row<VPL>(Th, i, a.N, lane, th);
    load_row<VPL>(G, i, a.N, lane, gg);
    kk += kkt_row<VPL>(th, gg, a.N, lane);  // per-lane partial sum
    if (stage == 1) {
        double y[VPL];
#pragma unroll
        for (int k = 0; k < VPL; ++k) y[k] = th[k] - gg[k];
        const double tau = simplex_tau<VPL>(y, a.N, lane);
#pragma unroll
        for (int k = 0; k < VPL; ++k) {
            const int64_t n = lane + 32 * k;
            if (n < a.N) {
                const double t = th[k] - fmax(y[k] - tau, 0.0);
                ww += t * t;
                g[i * a.N + n] = gg[k];
                var[i * a.N + n] = 1;
            }
        }
    } else {
        const int m = row_argmax<VPL>(th, a.N, lane);
        if (lane == 0) mrow[i] = m;
        const double gm = __shfl_sync(0xffffffffu, gg[(m / 32) % VPL], m % 32);
#pragma unroll
        for (int k = 0; k < VPL; ++k) {
            const int64_t n = lane + 32 * k;
            if (n < a.N) {
                if (n == m) {
                    g[i * a.N + n] = 0.0;
                    var[i * a.N + n] = 0;
                } else {
                    const double gr = gg[k] - gm;
                    g[i * a.N + n] = gr;
                    var[i * a.N + n] = 1;
                    const double pr = fmax(th[k] - gr, 0.0);
                    ww += (th[k] - pr) * (th[k] - pr);
                }
            }
        }
    }
    ROW_LOOP_END
    double v[2] = {kk, ww};
    DevScalars *sc = a.sc;
    grid_reduce<2>(v, a.partials, a.pstride, &sc->ticket[0], [sc, eps_bar](const double *t) {
        sc->kkt2 = t[0];
        sc->w2 = t[1];
        const double w = sqrt(t[1]);
        sc->eps = w < eps_bar ? w : eps_bar;
    });
}

// ---------------------------------------------------------------------------
// Set-up, part 2: index set I = {x <= eps_k, g > 0} (free = var and not in I),
// and the start of the diagonally preconditioned CG on the free variables:
// x = 0, r = -g (free), z = r / diag, p = z; stage 2 also lifts p into
// u = E p (column m(i) := -sum of the others).
// ---------------------------------------------------------------------------
template <int VPL, typename VT>
__global__ void k_setup2(RowArgs a, int stage, int max_cg, double eta_max, double eta_pow,
                         const double *Th, const double *g,
                         const uint8_t *var, const int32_t *mrow, uint8_t *freem, VT *x,
                         VT *r, VT *z, VT *p, VT *u)
{
    constexpr bool F32 = std::is_same<VT, float>::value;
    double rz = 0.0, rr = 0.0;
    const double eps = a.sc->eps;
    ROW_LOOP_BEGIN
    const double diag = stage == 1 ? a.h[i] : 2.0 * a.h[i];
    const float inv = F32 ? a.hinv[(stage == 1 ? 0 : a.M) + i] : 0.f;
    VT pv[VPL];
    VT psum = 0;
    float rz_row = 0.f, rr_row = 0.f;
#pragma unroll
    for (int k = 0; k < VPL; ++k) {
        const int64_t n = lane + 32 * k;
        pv[k] = 0;
        if (n < a.N) {
            const int64_t e = i * a.N + n;
            const double gv = g[e];
            const bool isv = var[e] != 0;
            const bool inI = Th[e] <= eps && gv > 0.0;
            const bool fr = isv && !inI;
            freem[e] = fr;
            if constexpr (F32) {
                const float rv = fr ? float(-gv) : 0.f;
                const float zv = rv * inv;
                x[e] = 0.f;
                r[e] = rv;
                z[e] = zv;
                p[e] = zv;
                pv[k] = zv;
                rz_row = fmaf(rv, zv, rz_row);
                rr_row = fmaf(rv, rv, rr_row);
                if (stage == 2) psum += zv;
            } else {
                const double rv = fr ? -gv : 0.0;
                const double zv = fr ? rv / diag : 0.0;
                x[e] = 0.0;
                r[e] = rv;
                z[e] = zv;
                p[e] = zv;
                pv[k] = zv;
                rz += rv * zv;
                rr += rv * rv;
                if (stage == 2) psum += zv;
            }
        }
    }
    if constexpr (F32) {
        rz += double(rz_row);
        rr += double(rr_row);
    }
    if (stage == 2) {
        const int m = mrow[i];
        psum = warp_sum(psum);
#pragma unroll
        for (int k = 0; k < VPL; ++k) {
            const int64_t n = lane + 32 * k;
            if (n < a.N) u[i * a.N + n] = (n == m) ? -psum : pv[k];
        }
    }
    ROW_LOOP_END
    double v[2] = {rz, rr};
    DevScalars *sc = a.sc;
    grid_reduce<2>(v, a.partials, a.pstride, &sc->ticket[0], [sc, max_cg, eta_max, eta_pow](const double *t) {
        sc->rz = t[0];
        sc->rr = t[1];
        const double bn = sqrt(t[1]);
        // forcing term eta = min(eta_max, ||b||^eta_pow) (reading R5: 0.5, 0.5)
        const double pw = eta_pow == 0.5 ? sqrt(bn) : eta_pow == 1.0 ? bn : eta_pow == 0.0 ? 1.0 : pow(bn, eta_pow);
        sc->bn = bn;
        sc->tol = (pw < eta_max ? pw : eta_max) * bn;
        sc->cg_iters = 0;
        sc->max_cg = max_cg;
        sc->use_grad_dir = 0;
        sc->cg_active = (max_cg > 0 && !(bn <= sc->tol)) ? 1 : 0;
    });
}

// ---------------------------------------------------------------------------
// CG: restrict the full Hessian product to the free variables, q = mask(E^T
// qfull) (stage 2: q_{i,n} = qfull_{i,n} - qfull_{i,m(i)}), and pq = p^T q.
// ---------------------------------------------------------------------------
template <int VPL, typename VT>
__global__ void k_cg_restrict(RowArgs a, int stage, const int32_t *mrow, const uint8_t *freem,
                              const VT *p, VT *q)
{
    constexpr bool F32 = std::is_same<VT, float>::value;
    if (a.sc->cg_active == 0) return;
    double pq = 0.0;
    ROW_LOOP_BEGIN
    VT qv[VPL];
    load_row<VPL>(q, i, a.N, lane, qv);
    VT qm = 0;
    if (stage == 2) {
        const int m = mrow[i];
        qm = __shfl_sync(0xffffffffu, qv[(m / 32) % VPL], m % 32);
    }
    float pq_row = 0.f;
#pragma unroll
    for (int k = 0; k < VPL; ++k) {
        const int64_t n = lane + 32 * k;
        if (n < a.N) {
            const int64_t e = i * a.N + n;
            const VT v = freem[e] ? qv[k] - qm : VT(0);
            q[e] = v;
            if constexpr (F32) pq_row = fmaf(p[e], v, pq_row);
            else pq += p[e] * v;
        }
    }
    if constexpr (F32) pq += double(pq_row);
    ROW_LOOP_END
    double v[1] = {pq};
    DevScalars *sc = a.sc;
    grid_reduce<1>(v, a.partials, a.pstride, &sc->ticket[0], [sc](const double *t) {
        sc->pq = t[0];
        if (!(t[0] > 0.0)) {
            sc->cg_active = 0;
        } else {
            sc->alpha = sc->rz / t[0];
        }
    });
}

// x += alpha p, r -= alpha q, z = r / diag (free), with r.z and r.r; warp per
// row (the diagonal is one value per row).  Float vectors scale by the
// row's reciprocal diagonal and sum each row in float before the double
// accumulation.
template <typename VT>
__global__ void k_cg_update_xr(RowArgs a, int stage, const uint8_t *freem, const VT *p,
                               const VT *q, VT *x, VT *r, VT *z)
{
    constexpr bool F32 = std::is_same<VT, float>::value;
    if (a.sc->cg_active == 0) return;
    const double al = a.sc->alpha;
    const float alf = float(al);
    const double scale = stage == 1 ? 1.0 : 2.0;
    double rz = 0.0, rr = 0.0;
    ROW_LOOP_BEGIN
    if constexpr (F32) {
        const float inv = a.hinv[(stage == 1 ? 0 : a.M) + i];
        float rz_row = 0.f, rr_row = 0.f;
        for (int64_t n = lane; n < a.N; n += 32) {
            const int64_t e = i * a.N + n;
            const float xv = fmaf(alf, p[e], x[e]);
            const float rv = fmaf(-alf, q[e], r[e]);
            const float zv = freem[e] ? rv * inv : 0.f;
            x[e] = xv;
            r[e] = rv;
            z[e] = zv;
            rz_row = fmaf(rv, zv, rz_row);
            rr_row = fmaf(rv, rv, rr_row);
        }
        rz += double(rz_row);
        rr += double(rr_row);
    } else {
        const double diag = scale * a.h[i];
        for (int64_t n = lane; n < a.N; n += 32) {
            const int64_t e = i * a.N + n;
            const double xv = x[e] + al * p[e];
            const double rv = r[e] - al * q[e];
            const double zv = freem[e] ? rv / diag : 0.0;
            x[e] = xv;
            r[e] = rv;
            z[e] = zv;
            rz += rv * zv;
            rr += rv * rv;
        }
    }
    ROW_LOOP_END
    double v[2] = {rz, rr};
    DevScalars *sc = a.sc;
    grid_reduce<2>(v, a.partials, a.pstride, &sc->ticket[0], [sc](const double *t) {
        sc->beta = t[0] / sc->rz;
        sc->rz = t[0];
        sc->rr = t[1];
        sc->cg_iters += 1;
        if (sqrt(t[1]) <= sc->tol || sc->cg_iters >= sc->max_cg) sc->cg_active = 0;
    });
}

// The same update for float vectors with N % 4 == 0, a float4 per lane: all
// loads of a row are issued before any is used (one memory round trip per
// row instead of one per 32 columns), and each lane sums its four values in
// float before the per-row double accumulation.
template <int CPL>
__global__ void k_cg_update_xr_f4(RowArgs a, int stage, const uint8_t *freem, const float4 *p,
                                  const float4 *q, float4 *x, float4 *r, float4 *z)
{
    if (a.sc->cg_active == 0) return;
    const float alf = float(a.sc->alpha);
    const int64_t nc = a.N / 4;
    const uchar4 *fm4 = reinterpret_cast<const uchar4 *>(freem);
    double rz = 0.0, rr = 0.0;
    ROW_LOOP_BEGIN
    const float inv = a.hinv[(stage == 1 ? 0 : a.M) + i];
    float4 pv[CPL], qv[CPL], xv[CPL], rv[CPL];
    uchar4 fv[CPL];
#pragma unroll
    for (int k = 0; k < CPL; ++k) {
        const int64_t c = lane + 32 * k;
        if (c < nc) {
            const int64_t e = i * nc + c;
            pv[k] = p[e];
            qv[k] = q[e];
            xv[k] = x[e];
            rv[k] = r[e];
            fv[k] = fm4[e];
        }
    }
    float rz_row = 0.f, rr_row = 0.f;
#pragma unroll
    for (int k = 0; k < CPL; ++k) {
        const int64_t c = lane + 32 * k;
        if (c < nc) {
            const int64_t e = i * nc + c;
            float4 xo, ro, zo;
            xo.x = fmaf(alf, pv[k].x, xv[k].x); ro.x = fmaf(-alf, qv[k].x, rv[k].x); zo.x = fv[k].x ? ro.x * inv : 0.f;
            xo.y = fmaf(alf, pv[k].y, xv[k].y); ro.y = fmaf(-alf, qv[k].y, rv[k].y); zo.y = fv[k].y ? ro.y * inv : 0.f;
            xo.z = fmaf(alf, pv[k].z, xv[k].z); ro.z = fmaf(-alf, qv[k].z, rv[k].z); zo.z = fv[k].z ? ro.z * inv : 0.f;
            xo.w = fmaf(alf, pv[k].w, xv[k].w); ro.w = fmaf(-alf, qv[k].w, rv[k].w); zo.w = fv[k].w ? ro.w * inv : 0.f;
            x[e] = xo;
            r[e] = ro;
            z[e] = zo;
            rz_row = fmaf(ro.x, zo.x, rz_row); rz_row = fmaf(ro.y, zo.y, rz_row);
            rz_row = fmaf(ro.z, zo.z, rz_row); rz_row = fmaf(ro.w, zo.w, rz_row);
            rr_row = fmaf(ro.x, ro.x, rr_row); rr_row = fmaf(ro.y, ro.y, rr_row);
            rr_row = fmaf(ro.z, ro.z, rr_row); rr_row = fmaf(ro.w, ro.w, rr_row);
        }
    }
    rz += double(rz_row);
    rr += double(rr_row);
    ROW_LOOP_END
    double v[2] = {rz, rr};
    DevScalars *sc = a.sc;
    grid_reduce<2>(v, a.partials, a.pstride, &sc->ticket[0], [sc](const double *t) {
        sc->beta = t[0] / sc->rz;
        sc->rz = t[0];
        sc->rr = t[1];
        sc->cg_iters += 1;
        if (sqrt(t[1]) <= sc->tol || sc->cg_iters >= sc->max_cg) sc->cg_active = 0;
    });
}

// p = z + beta p; stage 2 also u = E p.
template <int VPL, typename VT>
__global__ void k_cg_update_p(RowArgs a, int stage, const int32_t *mrow, const VT *z,
                              VT *p, VT *u)
{
    if (a.sc->cg_active == 0) return;
    const VT be = VT(a.sc->beta);
    ROW_LOOP_BEGIN
    VT pv[VPL];
    VT psum = 0;
#pragma unroll
    for (int k = 0; k < VPL; ++k) {
        const int64_t n = lane + 32 * k;
        pv[k] = 0;
        if (n < a.N) {
            const int64_t e = i * a.N + n;
            const VT v = z[e] + be * p[e];
            p[e] = v;
            pv[k] = v;
            psum += v;
        }
    }
    if (stage == 2) {
        const int m = mrow[i];
        const VT pm = __shfl_sync(0xffffffffu, pv[(m / 32) % VPL], m % 32);
        psum = warp_sum(psum) - pm;
#pragma unroll
        for (int k = 0; k < VPL; ++k) {
            const int64_t n = lane + 32 * k;
            if (n < a.N) u[i * a.N + n] = (n == m) ? -psum : pv[k];
        }
    }
    ROW_LOOP_END
}

// Newton direction: CG solution on the free variables, -g/diag on I, 0 on
// non-variables; g^T dir decides whether the scaled gradient replaces it.
template <typename VT>
__global__ void k_direction(RowArgs a, int stage, const uint8_t *var, const uint8_t *freem,
                            const VT *x, const double *g, double *dir)
{
    const double scale = stage == 1 ? 1.0 : 2.0;
    double gd = 0.0;
    ROW_LOOP_BEGIN
    const double diag = scale * a.h[i];
    for (int64_t n = lane; n < a.N; n += 32) {
        const int64_t e = i * a.N + n;
        double d;
        if (!var[e]) d = 0.0;
        else if (freem[e]) d = double(x[e]);
        else d = -g[e] / diag;
        dir[e] = d;
        gd += g[e] * d;
    }
    ROW_LOOP_END
    double v[1] = {gd};
    DevScalars *sc = a.sc;
    grid_reduce<1>(v, a.partials, a.pstride, &sc->ticket[0], [sc](const double *t) {
        sc->gdir = t[0];
        sc->use_grad_dir = (t[0] < 0.0) ? 0 : 1;
    });
}

// ---------------------------------------------------------------------------
// Line-search trial point Theta(alpha) of row i (returns it in t[], with the
// implicit-entry negativity flag for stage 2).
// Stage 1: t = P_S(Theta_i + alpha dir_i).
// Stage 2: t_n = max(0, Theta_{i,n} + alpha dir_{i,n}) for n != m(i),
//          t_m = 1 - sum_{n != m} t_n.
// ---------------------------------------------------------------------------
template <int VPL>
__device__ __forceinline__ void trial_row(const RowArgs &a, int stage, int64_t i, int lane,
                                          double alpha, bool graddir, const double *Th,
                                          const double *dir, const double *g,
                                          const int32_t *mrow, const uint8_t *var,
                                          double (&th)[VPL], double (&t)[VPL], bool &neg)
{
    load_row<VPL>(Th, i, a.N, lane, th);
    const double scale = stage == 1 ? 1.0 : 2.0;
    const double diag = scale * a.h[i];
    double y[VPL];
#pragma unroll
    for (int k = 0; k < VPL; ++k) {
        const int64_t n = lane + 32 * k;
        double dv = 0.0;
        if (n < a.N) {
            const int64_t e = i * a.N + n;
            dv = graddir ? (var[e] ? -g[e] / diag : 0.0) : dir[e];
        }
        y[k] = th[k] + alpha * dv;
    }
    neg = false;
    if (stage == 1) {
        const double tau = simplex_tau<VPL>(y, a.N, lane);
#pragma unroll
        for (int k = 0; k < VPL; ++k) t[k] = fmax(y[k] - tau, 0.0);
    } else {
        const int m = mrow[i];
        double s = 0.0;
#pragma unroll
        for (int k = 0; k < VPL; ++k) {
            const int64_t n = lane + 32 * k;
            t[k] = 0.0;
            if (n < a.N && n != m) {
                t[k] = fmax(y[k], 0.0);
                s += t[k];
            }
        }
        s = warp_sum(s);
        const double tm = 1.0 - s;
#pragma unroll
        for (int k = 0; k < VPL; ++k)
            if (lane + 32 * k == m) t[k] = tm;
        neg = tm < 0.0;
    }
}

// Trial point of the whole matrix with g^T (trial - Theta), the regulariser
// (direct mode: g(trial); delta mode: g(trial) - g(Theta) from the exact
// expansion) and the count of negative implicit entries.  A CTA owns blocks
// of ROW_WARPS consecutive rows (one warp per row) and keeps their Theta and
// trial rows, plus the next block's first row (recomputed by the last warp),
// in shared memory for the nearest-neighbour term.
template <int VPL>
__global__ void k_trial(RowArgs a, int stage, double alpha, int delta, const double *Th,
                        const double *dir, const double *g, const int32_t *mrow,
                        const uint8_t *var, double *trial, double *s_out)
{
    extern __shared__ double trial_sm[];
    double *sh_th = trial_sm;                              // [ROW_WARPS + 1][N]
    double *sh_t = trial_sm + (ROW_WARPS + 1) * a.N;        // [ROW_WARPS + 1][N]
    const bool graddir = a.sc->use_grad_dir != 0;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    double gts = 0.0, reg = 0.0, negc = 0.0;
    const int64_t nblocks = (a.M + ROW_WARPS - 1) / ROW_WARPS;
    for (int64_t b = blockIdx.x; b < nblocks; b += gridDim.x) {
        const int64_t i0 = b * ROW_WARPS;
        // own row, and the halo row (first row of the next block) by the last warp
        for (int pass = 0; pass < (w == ROW_WARPS - 1 ? 2 : 1); ++pass) {
            const int slot = pass == 0 ? w : ROW_WARPS;
            const int64_t i = i0 + slot;
            if (i >= a.M) continue;
            double th[VPL], t[VPL];
            bool neg;
            trial_row<VPL>(a, stage, i, lane, alpha, graddir, Th, dir, g, mrow, var, th, t, neg);
#pragma unroll
            for (int k = 0; k < VPL; ++k) {
                const int64_t n = lane + 32 * k;
                if (n < a.N) {
                    sh_th[slot * a.N + n] = th[k];
                    sh_t[slot * a.N + n] = t[k];
                }
            }
            if (pass == 0) {
                if (lane == 0 && neg) negc += 1.0;
#pragma unroll
                for (int k = 0; k < VPL; ++k) {
                    const int64_t n = lane + 32 * k;
                    if (n < a.N) {
                        const int64_t e = i * a.N + n;
                        const double sv = t[k] - th[k];
                        trial[e] = t[k];
                        s_out[e] = sv;
                        if (var[e]) gts += g[e] * sv;
                    }
                }
            }
        }
        __syncthreads();
        const int64_t i = i0 + w;
        if (a.gamma != 0.0 && i + 1 < a.M) {
            for (int64_t n = lane; n < a.N; n += 32) {
                const double t0 = sh_t[w * a.N + n], t1 = sh_t[(w + 1) * a.N + n];
                if (delta) {
                    const double th0 = sh_th[w * a.N + n], th1 = sh_th[(w + 1) * a.N + n];
                    const double ds = (t0 - th0) - (t1 - th1);
                    const double dth = th0 - th1;
                    reg += ds * ds + 2.0 * dth * ds;
                } else {
                    const double dt = t0 - t1;
                    reg += dt * dt;
                }
            }
        }
        __syncthreads();
    }
    double v[3] = {gts, a.gamma * reg, negc};
    DevScalars *sc = a.sc;
    grid_reduce<3>(v, a.partials, a.pstride, &sc->ticket[0], [sc, alpha](const double *t) {
        sc->gts = t[0];
        sc->reg = t[1];
        sc->neg = t[2] > 0.0 ? 1 : 0;
        sc->alpha_ls = alpha;
        sc->accept = 0;
        sc->f_trial = 0.0;
        sc->ls_go = t[2] > 0.0 ? 0 : 1;
    });
}

// ---------------------------------------------------------------------------
// Element-wise helpers
// ---------------------------------------------------------------------------
__global__ void k_fill(double *x, double v, int64_t n)
{
    for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < n;
         e += int64_t(gridDim.x) * blockDim.x)
        x[e] = v;
}

// Eq. regul: gamma sum_n sum_{i<M-1} (X_{i,n} - X_{i+1,n})^2.
__global__ void k_regulariser(RowArgs a, const double *X)
{
    double s = 0.0;
    const int64_t n1 = (a.M - 1) * a.N;
    for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < n1;
         e += int64_t(gridDim.x) * blockDim.x) {
        const double t = X[e] - X[e + a.N];
        s += t * t;
    }
    double v[1] = {s};
    DevScalars *sc = a.sc;
    const double gam = a.gamma;
    grid_reduce<1>(v, a.partials, a.pstride, &sc->ticket[0], [sc, gam](const double *t) {
        sc->regval = gam * t[0];
    });
}

__global__ void k_nonfinite(RowArgs a, const double *x, int64_t n)
{
    double c = 0.0;
    for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < n;
         e += int64_t(gridDim.x) * blockDim.x)
        if (!isfinite(x[e])) c += 1.0;
    double v[1] = {c};
    DevScalars *sc = a.sc;
    grid_reduce<1>(v, a.partials, a.pstride, &sc->ticket[0], [sc](const double *t) {
        sc->nonfinite = t[0];
    });
}

__global__ void k_set_grad_dir(DevScalars *sc) { sc->use_grad_dir = 1; }

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
static unsigned row_grid(const Plan &p)
{
    const int64_t rows_per_cta = ROW_WARPS;
    int64_t g = (p.M + rows_per_cta - 1) / rows_per_cta;
    const int64_t cap = int64_t(p.num_sms) * 8;
    if (g > cap) g = cap;
    if (g < 1) g = 1;
    return unsigned(g);
}

static unsigned elem_grid(const Plan &p, int64_t n)
{
    int64_t g = (n + 255) / 256;
    const int64_t cap = int64_t(p.num_sms) * 8;
    if (g > cap) g = cap;
    if (g < 1) g = 1;
    return unsigned(g);
}

#define VPL_DISPATCH_T(N, KERNEL, VT, GRID, ...)                                            \
    do {                                                                                    \
        const int64_t _n = (N);                                                             \
        if (_n <= 32) KERNEL<1, VT><<<GRID, ROW_WARPS * 32, 0, p.stream>>>(__VA_ARGS__);     \
        else if (_n <= 64) KERNEL<2, VT><<<GRID, ROW_WARPS * 32, 0, p.stream>>>(__VA_ARGS__); \
        else if (_n <= 128) KERNEL<4, VT><<<GRID, ROW_WARPS * 32, 0, p.stream>>>(__VA_ARGS__); \
        else if (_n <= 256) KERNEL<8, VT><<<GRID, ROW_WARPS * 32, 0, p.stream>>>(__VA_ARGS__); \
        else if (_n <= 512) KERNEL<16, VT><<<GRID, ROW_WARPS * 32, 0, p.stream>>>(__VA_ARGS__); \
        else KERNEL<32, VT><<<GRID, ROW_WARPS * 32, 0, p.stream>>>(__VA_ARGS__);             \
        count_launch();                                                                     \
    } while (0)

// CG vectors: float in the tensor-core form, double otherwise (same buffers)
#define CGV(ptr) reinterpret_cast<float *>(ptr)

#define VPL_DISPATCH(N, KERNEL, GRID, ...)                                                  \
    do {                                                                                    \
        const int64_t _n = (N);                                                             \
        if (_n <= 32) KERNEL<1><<<GRID, ROW_WARPS * 32, 0, p.stream>>>(__VA_ARGS__);         \
        else if (_n <= 64) KERNEL<2><<<GRID, ROW_WARPS * 32, 0, p.stream>>>(__VA_ARGS__);    \
        else if (_n <= 128) KERNEL<4><<<GRID, ROW_WARPS * 32, 0, p.stream>>>(__VA_ARGS__);   \
        else if (_n <= 256) KERNEL<8><<<GRID, ROW_WARPS * 32, 0, p.stream>>>(__VA_ARGS__);   \
        else if (_n <= 512) KERNEL<16><<<GRID, ROW_WARPS * 32, 0, p.stream>>>(__VA_ARGS__);  \
        else KERNEL<32><<<GRID, ROW_WARPS * 32, 0, p.stream>>>(__VA_ARGS__);                 \
        count_launch();                                                                     \
    } while (0)

cudaError_t launch_set_grad_dir(Plan &p)
{
    k_set_grad_dir<<<1, 1, 0, p.stream>>>(p.sc);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_fill(Plan &p, double *x, double v, int64_t n)
{
    k_fill<<<elem_grid(p, n), 256, 0, p.stream>>>(x, v, n);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_regulariser(Plan &p, const double *X)
{
    RowArgs a = row_args(p);
    k_regulariser<<<elem_grid(p, p.M * p.N), 256, 0, p.stream>>>(a, X);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_nonfinite_check(Plan &p, const double *x, int64_t n, int)
{
    RowArgs a = row_args(p);
    k_nonfinite<<<elem_grid(p, n), 256, 0, p.stream>>>(a, x, n);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_zero_small_rows(Plan &p, double *X, double rel)
{
    RowArgs a = row_args(p);
    VPL_DISPATCH(p.N, k_zero_small_rows, row_grid(p), a, X, rel);
    return cudaGetLastError();
}

cudaError_t launch_project_rows(Plan &p, const double *X, double *Y)
{
    RowArgs a = row_args(p);
    VPL_DISPATCH(p.N, k_project_rows, row_grid(p), a, X, Y);
    return cudaGetLastError();
}

cudaError_t launch_kkt(Plan &p, const double *Th, const double *G)
{
    RowArgs a = row_args(p);
    VPL_DISPATCH(p.N, k_kkt, row_grid(p), a, Th, G);
    return cudaGetLastError();
}

cudaError_t launch_setup1(Plan &p, int stage, double eps_bar)
{
    RowArgs a = row_args(p);
    VPL_DISPATCH(p.N, k_setup1, row_grid(p), a, stage, eps_bar, p.Th, p.G, p.g, p.var, p.mrow);
    return cudaGetLastError();
}

cudaError_t launch_setup2(Plan &p, int stage, int max_cg, double eta_max, double eta_pow)
{
    RowArgs a = row_args(p);
    if (p.cg_f32)
        VPL_DISPATCH_T(p.N, k_setup2, float, row_grid(p), a, stage, max_cg, eta_max, eta_pow, p.Th, p.g, p.var, p.mrow,
                       p.freem, CGV(p.x), CGV(p.r), CGV(p.z), CGV(p.p), CGV(p.u));
    else
        VPL_DISPATCH_T(p.N, k_setup2, double, row_grid(p), a, stage, max_cg, eta_max, eta_pow, p.Th, p.g, p.var, p.mrow,
                       p.freem, p.x, p.r, p.z, p.p, p.u);
    return cudaGetLastError();
}

cudaError_t launch_cg_restrict(Plan &p, int stage)
{
    RowArgs a = row_args(p);
    if (p.cg_f32)
        VPL_DISPATCH_T(p.N, k_cg_restrict, float, row_grid(p), a, stage, p.mrow, p.freem, CGV(p.p), CGV(p.q));
    else
        VPL_DISPATCH_T(p.N, k_cg_restrict, double, row_grid(p), a, stage, p.mrow, p.freem, p.p, p.q);
    return cudaGetLastError();
}

cudaError_t launch_cg_update_xr(Plan &p, int stage)
{
    RowArgs a = row_args(p);
    if (p.cg_f32 && (p.N % 4) == 0) {
        auto f4 = [](double *b) { return reinterpret_cast<float4 *>(b); };
        const int64_t cpl = (p.N / 4 + 31) / 32;
        auto kern = cpl <= 1 ? k_cg_update_xr_f4<1> : cpl <= 2 ? k_cg_update_xr_f4<2> : k_cg_update_xr_f4<8>;
        kern<<<row_grid(p), ROW_WARPS * 32, 0, p.stream>>>(a, stage, p.freem, f4(p.p), f4(p.q), f4(p.x), f4(p.r), f4(p.z));
        count_launch();
        return cudaGetLastError();
    }
    if (p.cg_f32)
        k_cg_update_xr<float><<<row_grid(p), ROW_WARPS * 32, 0, p.stream>>>(
            a, stage, p.freem, CGV(p.p), CGV(p.q), CGV(p.x), CGV(p.r), CGV(p.z));
    else
        k_cg_update_xr<double><<<row_grid(p), ROW_WARPS * 32, 0, p.stream>>>(a, stage, p.freem, p.p, p.q,
                                                                         p.x, p.r, p.z);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_cg_update_p(Plan &p, int stage)
{
    RowArgs a = row_args(p);
    if (p.cg_f32)
        VPL_DISPATCH_T(p.N, k_cg_update_p, float, row_grid(p), a, stage, p.mrow, CGV(p.z), CGV(p.p), CGV(p.u));
    else
        VPL_DISPATCH_T(p.N, k_cg_update_p, double, row_grid(p), a, stage, p.mrow, p.z, p.p, p.u);
    return cudaGetLastError();
}

cudaError_t launch_direction(Plan &p, int stage)
{
    RowArgs a = row_args(p);
    if (p.cg_f32)
        k_direction<float><<<row_grid(p), ROW_WARPS * 32, 0, p.stream>>>(a, stage, p.var, p.freem, CGV(p.x),
                                                                         p.g, p.dir);
    else
        k_direction<double><<<row_grid(p), ROW_WARPS * 32, 0, p.stream>>>(a, stage, p.var, p.freem, p.x,
                                                                          p.g, p.dir);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_trial(Plan &p, int stage, double alpha, bool delta_mode)
{
    RowArgs a = row_args(p);
    const size_t smem = sizeof(double) * 2 * (ROW_WARPS + 1) * size_t(p.N);
    const unsigned grid = row_grid(p);
    const int d = delta_mode ? 1 : 0;
#define TRIAL_LAUNCH(V)                                                                            \
    do {                                                                                           \
        static const cudaError_t cfg_ = cudaFuncSetAttribute(                                      \
            k_trial<V>, cudaFuncAttributeMaxDynamicSharedMemorySize,                               \
            int(2 * (ROW_WARPS + 1) * MAX_N * sizeof(double)));                                    \
        if (cfg_ != cudaSuccess) return cfg_;                                                      \
        k_trial<V><<<grid, ROW_WARPS * 32, smem, p.stream>>>(a, stage, alpha, d, p.Th, p.dir, p.g, \
                                                             p.mrow, p.var, p.trial, p.s);         \
    } while (0)
    if (p.N <= 32) TRIAL_LAUNCH(1);
    else if (p.N <= 64) TRIAL_LAUNCH(2);
    else if (p.N <= 128) TRIAL_LAUNCH(4);
    else if (p.N <= 256) TRIAL_LAUNCH(8);
    else if (p.N <= 512) TRIAL_LAUNCH(16);
    else TRIAL_LAUNCH(32);
#undef TRIAL_LAUNCH
    count_launch();
    return cudaGetLastError();
}

}  // namespace tomo
