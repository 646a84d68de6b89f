// plan.cu -- plan-time tables of the band contractions, built on the device:
//   * band of every probe (the truncation of F, Sec. Data distribution: F is
//     sparse and banded for large M),
//   * Poisson anchors F_{d,i} at every RUN-th photon number of each band
//     (Eq. Fmatrix) evaluated in log space in double,
//   * per-tile photon-number / probe ranges of the forward and adjoint tiles,
//   * the Hessian diagonal h_i = 2 sum_d F_{d,i}^2 + 2 gamma L_ii (Table ops).
//
// Log-space Poisson weights: poisson.cuh (saddle-point form of Loader).
#include <cub/device/device_scan.cuh>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "poisson.cuh"
#include "tomo_device.cuh"
#include "tomo_internal.cuh"

namespace tomo {

// Band of probe d.  The products and differences are rounded explicitly
// (no fused multiply-add) so that the integer bounds are those of the plain
// IEEE evaluation round(lambda - round(k sqrt(lambda))).
__global__ void k_bands(int64_t D, int64_t M, double band_k, const double *lam,
                        int32_t *lo, int32_t *hi, int64_t *cnt)
{
    const int64_t d = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    if (d >= D) return;
    int64_t l, h;
    if (band_k <= 0.0) {
        l = 0;
        h = M - 1;
    } else {
        const double x = lam[d];
        const double s = sqrt(x);
        const double ks = __dmul_rn(band_k, s);
        const double a = floor(__dsub_rn(x, ks));
        double b = ceil(__dadd_rn(x, ks));
        if (b < 16.0) b = 16.0;
        l = a < 0.0 ? 0 : int64_t(a);
        h = b > double(M - 1) ? M - 1 : int64_t(b);
        if (l > M - 1) l = M;
    }
    lo[d] = int32_t(l);
    hi[d] = int32_t(h);
    const int64_t a0 = l & ~int64_t(RUN - 1);
    cnt[d] = (l <= h) ? (h - a0) / RUN + 1 : 0;
}

__global__ void k_anchors(int64_t D, const double *lam, const int32_t *lo, const int32_t *hi,
                          const int64_t *aoff, double *anc, float *anc_f)
{
    const int64_t d = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    if (d >= D) return;
    const int64_t l = lo[d], h = hi[d];
    if (l > h) return;
    const int64_t a0 = l & ~int64_t(RUN - 1);
    const double x = lam[d];
    int64_t k = aoff[d];
    for (int64_t i = a0; i <= h; i += RUN, ++k) {
        const double v = poisson_weight(i, x);
        anc[k] = v;
        anc_f[k] = float(v);
    }
}

// 1/i in double and as a float pair hi + lo (hi = float(1/i), lo = float(1/i - hi)),
// and lambda_d as a float pair, so that the float weight recurrence can form
// lambda / (i + 1) to ~1e-14 before its single rounding (no systematic bias
// from rounding lambda or 1/i to float).
__global__ void k_ratio_inv(int64_t n, double *r, float2 *rf2)
{
    const int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    if (i >= n) return;
    const double v = i == 0 ? 0.0 : 1.0 / double(i);
    r[i] = v;
    const float hi = float(v);
    rf2[i] = make_float2(hi, float(v - double(hi)));
}

__global__ void k_lam_split(int64_t D, const double *lam, float2 *lam2)
{
    const int64_t d = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    if (d >= D) return;
    const float hi = float(lam[d]);
    lam2[d] = make_float2(hi, float(lam[d] - double(hi)));
}

// Forward tile t covers probes [TILE_R t, TILE_R (t+1)): union of their bands.
__global__ void k_fwd_tiles(int64_t D, int tiles, const int32_t *lo, const int32_t *hi,
                            int32_t *klo, int32_t *khi)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= tiles) return;
    int32_t a = INT32_MAX, b = -1;
    for (int64_t d = int64_t(t) * TILE_R; d < D && d < int64_t(t + 1) * TILE_R; ++d) {
        if (lo[d] > hi[d]) continue;
        a = min(a, lo[d]);
        b = max(b, hi[d]);
    }
    if (b < 0) { a = 1; b = 0; }
    klo[t] = a;
    khi[t] = b;
}

// Adjoint tile t covers photon numbers [TILE_R t, TILE_R (t+1)).  With probes
// sorted by intensity, lo_d and hi_d are non-decreasing in d, so the probes
// whose band meets the tile form the range [first d with hi_d >= i0,
// last d with lo_d <= i1] (binary searches).
__global__ void k_adj_tiles(int64_t D, int64_t M, int tiles, const int32_t *lo,
                            const int32_t *hi, int32_t *dlo, int32_t *dhi)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= tiles) return;
    const int64_t i0 = int64_t(t) * TILE_R;
    int64_t i1 = i0 + TILE_R - 1;
    if (i1 > M - 1) i1 = M - 1;
    int64_t a = 0, b = D;  // first d with hi_d >= i0
    while (a < b) {
        const int64_t mid = (a + b) / 2;
        if (hi[mid] >= i0) b = mid; else a = mid + 1;
    }
    const int64_t first = a;
    a = 0; b = D;          // first d with lo_d > i1
    while (a < b) {
        const int64_t mid = (a + b) / 2;
        if (lo[mid] > i1) b = mid; else a = mid + 1;
    }
    const int64_t last = a - 1;
    dlo[t] = int32_t(first);
    dhi[t] = int32_t(last);
}

// F_{d,i} expanded from its anchor exactly as the contraction kernels do
// (double version).
__device__ double weight_from_anchor_d(int64_t d, int64_t i, const double *lam,
                                       const int32_t *lo, const int32_t *hi,
                                       const int64_t *aoff, const double *anc,
                                       const double *rinv)
{
    if (i < lo[d] || i > hi[d]) return 0.0;
    const int64_t a0 = int64_t(lo[d]) & ~int64_t(RUN - 1);
    const int64_t ir = i & ~int64_t(RUN - 1);
    double v = anc[aoff[d] + (ir - a0) / RUN];
    const double x = lam[d];
    for (int64_t j = ir; j < i; ++j) v = v * (x * rinv[j + 1]);
    return v;
}

__device__ float weight_from_anchor_f(int64_t d, int64_t i, const float2 *lam2,
                                      const int32_t *lo, const int32_t *hi,
                                      const int64_t *aoff, const float *anc,
                                      const float2 *rinv2)
{
    if (i < lo[d] || i > hi[d]) return 0.0f;
    const int64_t a0 = int64_t(lo[d]) & ~int64_t(RUN - 1);
    const int64_t ir = i & ~int64_t(RUN - 1);
    float v = anc[aoff[d] + (ir - a0) / RUN];
    const float2 x = lam2[d];
    for (int64_t j = ir; j < i; ++j) {
        const float2 r = rinv2[j + 1];
        v = v * fmaf(x.x, r.x, fmaf(x.x, r.y, x.y * r.x));
    }
    return v;
}

// h_i = 2 sum_d F_{d,i}^2 + 2 gamma L_ii, one thread per photon number,
// probes in increasing order (deterministic).
__global__ void k_hess_diag(int64_t M, double gamma, const double *lam, const int32_t *lo,
                            const int32_t *hi, const int64_t *aoff, const double *anc,
                            const double *rinv, const int32_t *dlo, const int32_t *dhi,
                            double *h, float *hinv)
{
    const int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    if (i >= M) return;
    const int t = int(i / TILE_R);
    double s = 0.0;
    for (int64_t d = dlo[t]; d <= dhi[t]; ++d) {
        const double f = weight_from_anchor_d(d, i, lam, lo, hi, aoff, anc, rinv);
        s += f * f;
    }
    const double lii = double((i > 0) + (i < M - 1));
    const double hv = 2.0 * s + 2.0 * gamma * lii;
    h[i] = hv;
    // float reciprocals of the stage-1 and stage-2 preconditioner diagonals
    // (h and 2h), for the float CG vector updates
    hinv[i] = float(1.0 / hv);
    hinv[M + i] = float(1.0 / (2.0 * hv));
}

__global__ void k_poisson_weights(int64_t count, const int64_t *dd, const int64_t *ii,
                                  int prec, int64_t D, int64_t M, const double *lam,
                                  const float2 *lam2, const int32_t *lo, const int32_t *hi,
                                  const int64_t *aoff, const double *anc, const float *anc_f,
                                  const double *rinv, const float2 *rinv_f2, double *out)
{
    const int64_t k = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    if (k >= count) return;
    const int64_t d = dd[k], i = ii[k];
    if (d < 0 || d >= D || i < 0 || i >= M) { out[k] = 0.0; return; }
    out[k] = prec == TOMO_PREC_FP64
                 ? weight_from_anchor_d(d, i, lam, lo, hi, aoff, anc, rinv)
                 : double(weight_from_anchor_f(d, i, lam2, lo, hi, aoff, anc_f, rinv_f2));
}

static inline unsigned blocks_for(int64_t n, int t) { return unsigned((n + t - 1) / t); }

cudaError_t launch_plan_tables(Plan &p)
{
    cudaError_t e;
    int64_t *cnt = nullptr;
    void *tmp = nullptr;
    size_t tmp_bytes = 0;
    if ((e = cudaMalloc(&cnt, sizeof(int64_t) * (p.D + 1))) != cudaSuccess) return e;
    k_bands<<<blocks_for(p.D, 256), 256, 0, p.stream>>>(p.D, p.M, p.band_k, p.lam, p.lo, p.hi, cnt);
    count_launch();
    cudaMemsetAsync(cnt + p.D, 0, sizeof(int64_t), p.stream);
    cub::DeviceScan::ExclusiveSum(nullptr, tmp_bytes, cnt, p.aoff, p.D + 1, p.stream);
    if ((e = cudaMalloc(&tmp, tmp_bytes)) != cudaSuccess) { cudaFree(cnt); return e; }
    cub::DeviceScan::ExclusiveSum(tmp, tmp_bytes, cnt, p.aoff, p.D + 1, p.stream);
    count_launch();
    int64_t total = 0;
    cudaMemcpyAsync(&total, p.aoff + p.D, sizeof(int64_t), cudaMemcpyDeviceToHost, p.stream);
    e = cudaStreamSynchronize(p.stream);
    cudaFree(tmp);
    cudaFree(cnt);
    if (e != cudaSuccess) return e;
    p.n_anchor = total;
    const int64_t na = total > 0 ? total : 1;
    if ((e = cudaMalloc(&p.anchor, sizeof(double) * na)) != cudaSuccess) return e;
    if ((e = cudaMalloc(&p.anchor_f, sizeof(float) * na)) != cudaSuccess) return e;
    k_anchors<<<blocks_for(p.D, 128), 128, 0, p.stream>>>(p.D, p.lam, p.lo, p.hi, p.aoff,
                                                          p.anchor, p.anchor_f);
    count_launch();
    const int64_t nr = p.M + RUN + 1;
    k_ratio_inv<<<blocks_for(nr, 256), 256, 0, p.stream>>>(nr, p.ratio_inv, p.ratio_inv_f2);
    count_launch();
    k_lam_split<<<blocks_for(p.D, 256), 256, 0, p.stream>>>(p.D, p.lam, p.lam_f2);
    count_launch();
    k_fwd_tiles<<<blocks_for(p.fwd_tiles, 128), 128, 0, p.stream>>>(p.D, p.fwd_tiles, p.lo,
                                                                    p.hi, p.fwd_klo, p.fwd_khi);
    count_launch();
    k_adj_tiles<<<blocks_for(p.adj_tiles, 128), 128, 0, p.stream>>>(p.D, p.M, p.adj_tiles, p.lo,
                                                                    p.hi, p.adj_dlo, p.adj_dhi);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_hess_diag(Plan &p)
{
    k_hess_diag<<<blocks_for(p.M, 128), 128, 0, p.stream>>>(
        p.M, p.gamma, p.lam, p.lo, p.hi, p.aoff, p.anchor, p.ratio_inv, p.adj_dlo, p.adj_dhi, p.h,
        p.hinv_f);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_poisson_weights(Plan &p, const int64_t *d, const int64_t *i, int64_t count,
                                   double *out)
{
    if (count <= 0) return cudaSuccess;
    k_poisson_weights<<<blocks_for(count, 128), 128, 0, p.stream>>>(
        count, d, i, prec_products(p.precision), p.D, p.M, p.lam, p.lam_f2, p.lo, p.hi, p.aoff,
        p.anchor, p.anchor_f, p.ratio_inv, p.ratio_inv_f2, out);
    count_launch();
    return cudaGetLastError();
}

}  // namespace tomo
