// band_gemm.cu -- the banded contractions O = F X and Z = F^T Y of the
// detector-tomography objective (Table ops: objective value, gradient,
// Hessian products), with the Poisson weights F_{d,i} = lambda_d^i
// e^{-lambda_d} / i! (Eq. Fmatrix) regenerated inside every tile.
//
// Weight generation: the plan stores, for every probe d, the weight at every
// RUN-th photon number of its band (computed in log space in double, see
// plan.cu).  A thread expands one run of RUN consecutive weights from its
// anchor with the exact ratio F_{d,i+1} / F_{d,i} = lambda_d / (i + 1), in the
// arithmetic type T of the contraction (at most RUN - 1 roundings per value).
// Weights outside [lo_d, hi_d] are zero (band truncation).
//
// Tiles are dense in-band register-blocked SIMT GEMM tiles: the forward tile
// is FWD_BD probes x BN columns swept over the union band of its probes in
// steps of BK photon numbers; the adjoint tile is ADJ_BI photon numbers x BN
// columns swept over the probes whose band meets it.  Epilogues fuse the
// residual, the objective / line-search reductions and the smoothness term.
#include <cuda_runtime.h>
#include <stdint.h>

#include "tomo_device.cuh"
#include "tomo_internal.cuh"

namespace tomo {

template <typename T> struct BK_of;
template <> struct BK_of<float> { static constexpr int v = 32; };
template <> struct BK_of<double> { static constexpr int v = 16; };

struct BandArgs {
    int64_t M, N, D;
    const double *lam;
    const int32_t *lo, *hi;
    const int64_t *aoff;
    const void *anchor;  // T*
    const void *rinv;    // T*, M + RUN + 1 entries
    const int32_t *rlo, *rhi;  // per-tile range (photon numbers or probes)
    const int32_t *gate;       // NULL or pointer to a flag: run only if != 0
    double *partials;
    int64_t pstride;
    DevScalars *sc;
    double gamma;
};

// Expands the run of RUN weights of probe d starting at photon number i_r
// (i_r a multiple of RUN) into vals[].  Zero outside the band.
template <typename T>
__device__ __forceinline__ void gen_run(const BandArgs &a, int64_t d, int64_t i_r, T (&vals)[RUN])
{
    const int64_t lo = a.lo[d], hi = a.hi[d];
#pragma unroll
    for (int t = 0; t < RUN; ++t) vals[t] = T(0);
    if (i_r + RUN - 1 < lo || i_r > hi) return;
    const int64_t a0 = lo & ~int64_t(RUN - 1);
    const T *anc = reinterpret_cast<const T *>(a.anchor);
    const T *rinv = reinterpret_cast<const T *>(a.rinv);
    T v = anc[a.aoff[d] + (i_r - a0) / RUN];
    const T lam = T(a.lam[d]);
#pragma unroll
    for (int t = 0; t < RUN; ++t) {
        const int64_t i = i_r + t;
        vals[t] = (i >= lo && i <= hi) ? v : T(0);
        v = v * (lam * rinv[i + 1]);
    }
}

// ----------------------------------------------------------------------------
// Forward: O = F X.   grid (fwd_tiles, ceil(N / BN)), 256 threads.
// ----------------------------------------------------------------------------
template <typename T, int BN, int MODE>
__global__ void __launch_bounds__(GEMM_THREADS)
k_forward(BandArgs a, const double *__restrict__ X, double *__restrict__ out,
          const double *__restrict__ aux)
{
    constexpr int BD = FWD_BD;
    constexpr int BK = BK_of<T>::v;
    constexpr int TN = BN >= 64 ? (BN == 128 ? 8 : 4) : 4;   // columns per thread
    constexpr int TX = BN / TN;                               // threads along columns
    constexpr int TY = GEMM_THREADS / TX;                     // threads along probes
    constexpr int TM = BD / TY;                               // probes per thread
    static_assert(TX * TY == GEMM_THREADS && TM * TY == BD, "tile shape");
    constexpr int NRUN = BD * BK / RUN;                       // runs per K step

    if (a.gate && *a.gate == 0) return;

    __shared__ __align__(16) T Fs[BK][BD];
    __shared__ __align__(16) T Xs[BK][BN];

    const int tid = threadIdx.x;
    const int tx = tid % TX, ty = tid / TX;
    const int tile = blockIdx.x;
    const int64_t d0 = int64_t(tile) * BD;
    const int64_t n0 = int64_t(blockIdx.y) * BN;
    const int64_t M = a.M, N = a.N, D = a.D;
    const int32_t klo = a.rlo[tile], khi = a.rhi[tile];

    T acc[TM][TN];
#pragma unroll
    for (int m = 0; m < TM; ++m)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[m][j] = T(0);

    // generation role: probe dd, run r
    const int gdd = tid % BD, grr = tid / BD;
    const int64_t gd = d0 + gdd;

    if (klo <= khi) {
        const int64_t kbeg = int64_t(klo) & ~int64_t(BK - 1);
        for (int64_t k0 = kbeg; k0 <= khi; k0 += BK) {
            if (tid < NRUN) {
                T vals[RUN];
                if (gd < D) gen_run<T>(a, gd, k0 + int64_t(grr) * RUN, vals);
                else {
#pragma unroll
                    for (int t = 0; t < RUN; ++t) vals[t] = T(0);
                }
#pragma unroll
                for (int t = 0; t < RUN; ++t) Fs[grr * RUN + t][gdd] = vals[t];
            }
            for (int e = tid; e < BK * BN; e += GEMM_THREADS) {
                const int kk = e / BN, nn = e % BN;
                const int64_t i = k0 + kk, n = n0 + nn;
                Xs[kk][nn] = (i < M && n < N) ? T(X[i * N + n]) : T(0);
            }
            __syncthreads();
#pragma unroll 8
            for (int kk = 0; kk < BK; ++kk) {
                T af[TM], bf[TN];
#pragma unroll
                for (int m = 0; m < TM; ++m) af[m] = Fs[kk][ty * TM + m];
#pragma unroll
                for (int j = 0; j < TN; ++j) bf[j] = Xs[kk][tx * TN + j];
#pragma unroll
                for (int m = 0; m < TM; ++m)
#pragma unroll
                    for (int j = 0; j < TN; ++j) acc[m][j] = fma(af[m], bf[j], acc[m][j]);
            }
            __syncthreads();
        }
    }

    double part = 0.0;
#pragma unroll
    for (int m = 0; m < TM; ++m) {
        const int64_t d = d0 + ty * TM + m;
        if (d >= D) continue;
#pragma unroll
        for (int j = 0; j < TN; ++j) {
            const int64_t n = n0 + tx * TN + j;
            if (n >= N) continue;
            const double v = double(acc[m][j]);
            const int64_t k = d * N + n;
            if (MODE == FWD_STORE) {
                out[k] = v;
            } else if (MODE == FWD_RESID) {
                const double rv = v - aux[k];
                out[k] = rv;
                part += rv * rv;
            } else {
                const double rv = aux[k];
                out[k] = rv + v;
                part += 2.0 * rv * v + v * v;
            }
        }
    }
    if (MODE != FWD_STORE) {
        double vv[1] = {part};
        DevScalars *sc = a.sc;
        grid_reduce<1>(vv, a.partials, a.pstride, &sc->ticket[0], [sc](const double *t) {
            if (MODE == FWD_RESID) sc->res2 = t[0];
            else sc->dres = t[0];
        });
    }
}

// ----------------------------------------------------------------------------
// Adjoint: Z = F^T Y.   grid (adj_tiles, ceil(N / BN)), 256 threads.
// ADJ_GRAD / ADJ_HESS epilogue: out = 2 Z + 2 gamma L Xreg.
// ----------------------------------------------------------------------------
template <typename T, int BN, int MODE>
__global__ void __launch_bounds__(GEMM_THREADS)
k_adjoint(BandArgs a, const double *__restrict__ Y, double *__restrict__ out,
          const double *__restrict__ Xreg)
{
    constexpr int BI = ADJ_BI;
    constexpr int BKD = BK_of<T>::v;                          // probes per step
    constexpr int TN = BN >= 64 ? (BN == 128 ? 8 : 4) : 4;
    constexpr int TX = BN / TN;
    constexpr int TY = GEMM_THREADS / TX;
    constexpr int TM = BI / TY;                               // photon numbers per thread
    static_assert(TX * TY == GEMM_THREADS && TM * TY == BI, "tile shape");
    constexpr int RPP = BI / RUN;                             // runs per probe
    constexpr int NRUN = BKD * RPP;

    if (a.gate && *a.gate == 0) return;

    __shared__ T Fs[BKD][BI + 1];
    __shared__ __align__(16) T Ys[BKD][BN];

    const int tid = threadIdx.x;
    const int tx = tid % TX, ty = tid / TX;
    const int tile = blockIdx.x;
    const int64_t i0 = int64_t(tile) * BI;
    const int64_t n0 = int64_t(blockIdx.y) * BN;
    const int64_t M = a.M, N = a.N, D = a.D;
    const int32_t dlo = a.rlo[tile], dhi = a.rhi[tile];

    T acc[TM][TN];
#pragma unroll
    for (int m = 0; m < TM; ++m)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[m][j] = T(0);

    const int gpp = tid % BKD, grr = tid / BKD;

    if (dlo <= dhi) {
        for (int64_t dd0 = dlo; dd0 <= dhi; dd0 += BKD) {
            if (tid < NRUN) {
                const int64_t d = dd0 + gpp;
                T vals[RUN];
                if (d <= dhi) gen_run<T>(a, d, i0 + int64_t(grr) * RUN, vals);
                else {
#pragma unroll
                    for (int t = 0; t < RUN; ++t) vals[t] = T(0);
                }
#pragma unroll
                for (int t = 0; t < RUN; ++t) Fs[gpp][grr * RUN + t] = vals[t];
            }
            for (int e = tid; e < BKD * BN; e += GEMM_THREADS) {
                const int kk = e / BN, nn = e % BN;
                const int64_t d = dd0 + kk, n = n0 + nn;
                Ys[kk][nn] = (d <= dhi && n < N) ? T(Y[d * N + n]) : T(0);
            }
            __syncthreads();
#pragma unroll 8
            for (int kk = 0; kk < BKD; ++kk) {
                T af[TM], bf[TN];
#pragma unroll
                for (int m = 0; m < TM; ++m) af[m] = Fs[kk][ty * TM + m];
#pragma unroll
                for (int j = 0; j < TN; ++j) bf[j] = Ys[kk][tx * TN + j];
#pragma unroll
                for (int m = 0; m < TM; ++m)
#pragma unroll
                    for (int j = 0; j < TN; ++j) acc[m][j] = fma(af[m], bf[j], acc[m][j]);
            }
            __syncthreads();
        }
    }

    const double g2 = 2.0 * a.gamma;
#pragma unroll
    for (int m = 0; m < TM; ++m) {
        const int64_t i = i0 + ty * TM + m;
        if (i >= M) continue;
#pragma unroll
        for (int j = 0; j < TN; ++j) {
            const int64_t n = n0 + tx * TN + j;
            if (n >= N) continue;
            const int64_t k = i * N + n;
            const double v = double(acc[m][j]);
            if (MODE == ADJ_STORE) {
                out[k] = v;
            } else {
                double lx = 0.0;
                if (g2 != 0.0) {
                    const double xi = Xreg[k];
                    if (i < M - 1) lx += xi - Xreg[k + N];
                    if (i > 0) lx += xi - Xreg[k - N];
                }
                out[k] = 2.0 * v + g2 * lx;
            }
        }
    }
}

// ----------------------------------------------------------------------------
// launchers
// ----------------------------------------------------------------------------
static BandArgs band_args(Plan &p, int prec, bool fwd)
{
    BandArgs a;
    a.M = p.M; a.N = p.N; a.D = p.D;
    a.lam = p.lam; a.lo = p.lo; a.hi = p.hi; a.aoff = p.aoff;
    a.anchor = prec == TOMO_PREC_FP64 ? (const void *)p.anchor : (const void *)p.anchor_f;
    a.rinv = prec == TOMO_PREC_FP64 ? (const void *)p.ratio_inv : (const void *)p.ratio_inv_f;
    a.rlo = fwd ? p.fwd_klo : p.adj_dlo;
    a.rhi = fwd ? p.fwd_khi : p.adj_dhi;
    a.gate = nullptr;
    a.partials = p.partials;
    a.pstride = p.max_partials;
    a.sc = p.sc;
    a.gamma = p.gamma;
    return a;
}

// Column tile width: the widest of 128/64/32 that still gives at least
// 1.5 CTAs per SM, else 32.
static int pick_bn(const Plan &p, int tiles)
{
    const int64_t want = (3 * int64_t(p.num_sms)) / 2;
    if (p.N > 64 && int64_t(tiles) * ((p.N + 127) / 128) >= want) return 128;
    if (p.N > 32 && int64_t(tiles) * ((p.N + 63) / 64) >= want) return 64;
    return 32;
}

template <typename T, int MODE>
static cudaError_t fwd_dispatch(Plan &p, BandArgs a, const double *X, double *out,
                                const double *aux)
{
    const int bn = pick_bn(p, p.fwd_tiles);
    dim3 grid(p.fwd_tiles, unsigned((p.N + bn - 1) / bn));
    if (bn == 128) k_forward<T, 128, MODE><<<grid, GEMM_THREADS, 0, p.stream>>>(a, X, out, aux);
    else if (bn == 64) k_forward<T, 64, MODE><<<grid, GEMM_THREADS, 0, p.stream>>>(a, X, out, aux);
    else k_forward<T, 32, MODE><<<grid, GEMM_THREADS, 0, p.stream>>>(a, X, out, aux);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_forward(Plan &p, int prec, FwdMode mode, const double *X, double *out,
                           const double *P_or_R, bool gated)
{
    BandArgs a = band_args(p, prec, true);
    if (gated) a.gate = &p.sc->cg_active;
    if (prec == TOMO_PREC_FP64) {
        switch (mode) {
        case FWD_STORE: return fwd_dispatch<double, FWD_STORE>(p, a, X, out, P_or_R);
        case FWD_RESID: return fwd_dispatch<double, FWD_RESID>(p, a, X, out, P_or_R);
        default: return fwd_dispatch<double, FWD_DELTA>(p, a, X, out, P_or_R);
        }
    }
    switch (mode) {
    case FWD_STORE: return fwd_dispatch<float, FWD_STORE>(p, a, X, out, P_or_R);
    case FWD_RESID: return fwd_dispatch<float, FWD_RESID>(p, a, X, out, P_or_R);
    default: return fwd_dispatch<float, FWD_DELTA>(p, a, X, out, P_or_R);
    }
}

// Line-search product: runs only if the trial kernel cleared it (no negative
// implicit entry), so a rejected stage-2 trial costs no contraction.
cudaError_t launch_forward_gated_ls(Plan &p, int prec, FwdMode mode, const double *X, double *out,
                                   const double *P_or_R)
{
    BandArgs a = band_args(p, prec, true);
    a.gate = &p.sc->ls_go;
    if (prec == TOMO_PREC_FP64) {
        if (mode == FWD_RESID) return fwd_dispatch<double, FWD_RESID>(p, a, X, out, P_or_R);
        return fwd_dispatch<double, FWD_DELTA>(p, a, X, out, P_or_R);
    }
    if (mode == FWD_RESID) return fwd_dispatch<float, FWD_RESID>(p, a, X, out, P_or_R);
    return fwd_dispatch<float, FWD_DELTA>(p, a, X, out, P_or_R);
}

template <typename T, int MODE>
static cudaError_t adj_dispatch(Plan &p, BandArgs a, const double *Y, double *out,
                                const double *Xreg)
{
    const int bn = pick_bn(p, p.adj_tiles);
    dim3 grid(p.adj_tiles, unsigned((p.N + bn - 1) / bn));
    if (bn == 128) k_adjoint<T, 128, MODE><<<grid, GEMM_THREADS, 0, p.stream>>>(a, Y, out, Xreg);
    else if (bn == 64) k_adjoint<T, 64, MODE><<<grid, GEMM_THREADS, 0, p.stream>>>(a, Y, out, Xreg);
    else k_adjoint<T, 32, MODE><<<grid, GEMM_THREADS, 0, p.stream>>>(a, Y, out, Xreg);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_adjoint(Plan &p, int prec, AdjMode mode, const double *Y, double *out,
                           const double *Xreg, bool gated)
{
    BandArgs a = band_args(p, prec, false);
    if (gated) a.gate = &p.sc->cg_active;
    if (prec == TOMO_PREC_FP64) {
        if (mode == ADJ_STORE) return adj_dispatch<double, ADJ_STORE>(p, a, Y, out, Xreg);
        return adj_dispatch<double, ADJ_GRAD>(p, a, Y, out, Xreg);
    }
    if (mode == ADJ_STORE) return adj_dispatch<float, ADJ_STORE>(p, a, Y, out, Xreg);
    return adj_dispatch<float, ADJ_GRAD>(p, a, Y, out, Xreg);
}

}  // namespace tomo
