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
// Tiles: TILE_R output rows (probes for F X, photon numbers for F^T Y) x BN
// output columns (outcomes), 256 threads, each owning an 8 x 8 (or 8 x 4,
// 4 x 4) register micro-tile whose rows/columns are split in two halves so
// that 128-bit shared loads of a warp cover contiguous 256-byte spans.  The
// reduction dimension (the tile's union band, or its probe range) is cut into
// work units of equal length planned on the host (split-K) so that every SM
// gets the same amount of band work whatever the band shape; units of one
// tile write partial tiles and the unit that arrives last sums them in unit
// order (deterministic) and runs the epilogue.  Two shared-memory stages with
// register prefetch overlap the global loads of step k+1 with the FMAs of
// step k.  Epilogues fuse the residual, the objective / line-search
// reductions and the smoothness term.
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
    const void *anchor;        // T*
    const void *rinv;          // double*, M + RUN + 1 entries (double path)
    const float2 *rinv2;       // 1/i as float hi + lo (float path)
    const float2 *lam2;        // lambda_d as float hi + lo (float path)
    const WorkUnit *units;
    const int32_t *tile_first; // per tile: index of its first partial slot
    const int32_t *tile_nsplit;
    unsigned int *counters;    // per (tile, column block)
    void *part;                // partial tiles (T)
    const int32_t *gate;       // NULL or pointer to a flag: run only if != 0
    double *partials;
    int64_t pstride;
    DevScalars *sc;
    double gamma;
};

// Expands the run of RUN weights of probe d starting at photon number i_r
// (i_r a multiple of RUN) into vals[].  Zero outside the band.
// The float path forms the ratio lambda * (1/(i+1)) from float pairs
// (hi + lo) so it is rounded once, without the systematic per-probe bias a
// float lambda would carry along a run.
template <typename T>
__device__ __forceinline__ void gen_run(const BandArgs &a, int64_t d, int64_t i_r, T (&vals)[RUN])
{
    const int64_t lo = a.lo[d], hi = a.hi[d];
#pragma unroll
    for (int t = 0; t < RUN; ++t) vals[t] = T(0);
    if (i_r + RUN - 1 < lo || i_r > hi) return;
    const int64_t a0 = lo & ~int64_t(RUN - 1);
    const T *anc = reinterpret_cast<const T *>(a.anchor);
    T v = anc[a.aoff[d] + (i_r - a0) / RUN];
    if constexpr (sizeof(T) == 8) {
        const double *rinv = reinterpret_cast<const double *>(a.rinv);
        const double lam = a.lam[d];
#pragma unroll
        for (int t = 0; t < RUN; ++t) {
            const int64_t i = i_r + t;
            vals[t] = (i >= lo && i <= hi) ? v : T(0);
            v = v * (lam * rinv[i + 1]);
        }
    } else {
        const float2 lam = a.lam2[d];
#pragma unroll
        for (int t = 0; t < RUN; ++t) {
            const int64_t i = i_r + t;
            vals[t] = (i >= lo && i <= hi) ? v : T(0);
            const float2 r = a.rinv2[i + 1];
            v = v * fmaf(lam.x, r.x, fmaf(lam.x, r.y, lam.y * r.x));
        }
    }
}

// Micro-tile geometry: TM x TN per thread, two halves per dimension when 8.
template <int BN> struct Geo;
template <> struct Geo<128> { static constexpr int TM = 8, TN = 8; };
template <> struct Geo<64> { static constexpr int TM = 8, TN = 4; };
template <> struct Geo<32> { static constexpr int TM = 4, TN = 4; };

template <int TDIM, int EXT>
__device__ __forceinline__ int micro_index(int t, int j)
{
    // element j of thread t's micro-tile along a dimension of extent EXT:
    // TDIM == 8 -> {4t..4t+3} U {EXT/2 + 4t..EXT/2 + 4t+3}; TDIM == 4 -> 4t..4t+3
    if (TDIM == 8) return (j < 4) ? 4 * t + j : EXT / 2 + 4 * t + (j - 4);
    return 4 * t + j;
}

template <typename T, int BN>
struct SmemTile {
    static constexpr int BK = BK_of<T>::v;
    T A[2][BK][TILE_R];   // weights, reduction index major
    T B[2][BK][BN];       // X or Y rows
};

template <typename T>
__device__ __forceinline__ void load4(const T *p, T *v)
{
    if constexpr (sizeof(T) == 4) {
        const float4 t = *reinterpret_cast<const float4 *>(p);
        v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
    } else {
        const double2 t0 = *reinterpret_cast<const double2 *>(p);
        const double2 t1 = *reinterpret_cast<const double2 *>(p + 2);
        v[0] = t0.x; v[1] = t0.y; v[2] = t1.x; v[3] = t1.y;
    }
}

// One contraction kernel for both directions.
//   FWD: rows = probes d (tile of TILE_R), reduction over photon numbers i,
//        A[k][r] = F_{d0+r, k0+k}, B[k][n] = X[k0+k, n].
//   ADJ: rows = photon numbers i, reduction over probes d,
//        A[k][r] = F_{k0+k, i0+r}, B[k][n] = Y[k0+k, n].
template <typename T, int BN, bool FWD, int MODE>
__global__ void __launch_bounds__(GEMM_THREADS)
k_band(BandArgs a, const double *__restrict__ In, double *__restrict__ out,
       const double *__restrict__ aux)
{
    constexpr int BK = BK_of<T>::v;
    constexpr int TM = Geo<BN>::TM, TN = Geo<BN>::TN;
    constexpr int TX = BN / TN;                 // threads along columns
    constexpr int TY = GEMM_THREADS / TX;       // threads along rows
    static_assert(TY * TM == TILE_R, "tile rows");
    constexpr int NRUN = TILE_R * BK / RUN;     // weight runs per K step
    constexpr int RPT = NRUN / GEMM_THREADS;    // runs per thread
    static_assert(RPT * GEMM_THREADS == NRUN, "runs per thread");
    constexpr int BPT = BK * BN / GEMM_THREADS; // B values per thread
    static_assert(BPT * GEMM_THREADS == BK * BN, "B per thread");

    if (a.gate && *a.gate == 0) return;

    extern __shared__ __align__(16) unsigned char smem_raw[];
    SmemTile<T, BN> &S = *reinterpret_cast<SmemTile<T, BN> *>(smem_raw);

    const int tid = threadIdx.x;
    const int tx = tid % TX, ty = tid / TX;
    const WorkUnit wu = a.units[blockIdx.x];
    const int tile = wu.tile;
    const int64_t r0 = int64_t(tile) * TILE_R;
    const int64_t n0 = int64_t(blockIdx.y) * BN;
    const int64_t M = a.M, N = a.N, D = a.D;
    const int64_t rows = FWD ? D : M;           // output rows
    const int64_t kext = FWD ? M : D;           // reduction extent

    T acc[TM][TN];
#pragma unroll
    for (int m = 0; m < TM; ++m)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[m][j] = T(0);

    T rv[RPT][RUN];
    T bv[BPT];

    // stage loader: weights of step k0 into rv, B rows into bv
    auto fetch = [&](int64_t k0) {
#pragma unroll
        for (int q = 0; q < RPT; ++q) {
            const int run = tid + q * GEMM_THREADS;
            if (FWD) {
                // run = (row r, run index along k): probe d0 + r, photons k0 + 8j
                const int r = run % TILE_R, j = run / TILE_R;
                const int64_t d = r0 + r;
                if (d < D) gen_run<T>(a, d, k0 + int64_t(j) * RUN, rv[q]);
                else {
#pragma unroll
                    for (int t = 0; t < RUN; ++t) rv[q][t] = T(0);
                }
            } else {
                // run = (probe k, run index along rows): probe k0 + k, photons i0 + 8j
                constexpr int RPR = TILE_R / RUN;
                const int j = run % RPR, k = run / RPR;
                const int64_t d = k0 + k;
                if (d < D && d < wu.k1) gen_run<T>(a, d, r0 + int64_t(j) * RUN, rv[q]);
                else {
#pragma unroll
                    for (int t = 0; t < RUN; ++t) rv[q][t] = T(0);
                }
            }
        }
#pragma unroll
        for (int q = 0; q < BPT; ++q) {
            const int e = tid + q * GEMM_THREADS;
            const int kk = e / BN, nn = e % BN;
            const int64_t k = k0 + kk, n = n0 + nn;
            bv[q] = (k < kext && k < wu.k1 && n < N) ? T(In[k * N + n]) : T(0);
        }
    };
    auto stash = [&](int buf) {
#pragma unroll
        for (int q = 0; q < RPT; ++q) {
            const int run = tid + q * GEMM_THREADS;
            if (FWD) {
                const int r = run % TILE_R, j = run / TILE_R;
#pragma unroll
                for (int t = 0; t < RUN; ++t) S.A[buf][j * RUN + t][r] = rv[q][t];
            } else {
                constexpr int RPR = TILE_R / RUN;
                const int j = run % RPR, k = run / RPR;
                T *dst = &S.A[buf][k][j * RUN];
                if constexpr (sizeof(T) == 4) {
                    reinterpret_cast<float4 *>(dst)[0] = make_float4(rv[q][0], rv[q][1], rv[q][2], rv[q][3]);
                    reinterpret_cast<float4 *>(dst)[1] = make_float4(rv[q][4], rv[q][5], rv[q][6], rv[q][7]);
                } else {
#pragma unroll
                    for (int t = 0; t < RUN; t += 2)
                        reinterpret_cast<double2 *>(dst)[t / 2] = make_double2(rv[q][t], rv[q][t + 1]);
                }
            }
        }
#pragma unroll
        for (int q = 0; q < BPT; ++q) {
            const int e = tid + q * GEMM_THREADS;
            S.B[buf][e / BN][e % BN] = bv[q];
        }
    };

    int buf = 0;
    if (wu.k0 < wu.k1) {
        fetch(wu.k0);
        stash(0);
        __syncthreads();
        for (int64_t k0 = wu.k0; k0 < wu.k1; k0 += BK) {
            const bool more = k0 + BK < wu.k1;
            if (more) fetch(k0 + BK);
#pragma unroll 4
            for (int kk = 0; kk < BK; ++kk) {
                T af[TM], bf[TN];
                load4<T>(&S.A[buf][kk][micro_index<TM, TILE_R>(ty, 0)], af);
                if constexpr (TM == 8) load4<T>(&S.A[buf][kk][micro_index<TM, TILE_R>(ty, 4)], af + 4);
                load4<T>(&S.B[buf][kk][micro_index<TN, BN>(tx, 0)], bf);
                if constexpr (TN == 8) load4<T>(&S.B[buf][kk][micro_index<TN, BN>(tx, 4)], bf + 4);
#pragma unroll
                for (int m = 0; m < TM; ++m)
#pragma unroll
                    for (int j = 0; j < TN; ++j) acc[m][j] = fma(af[m], bf[j], acc[m][j]);
            }
            if (more) stash(buf ^ 1);
            __syncthreads();
            buf ^= 1;
        }
    }

    // ---- split-K: combine the partial tiles of this (tile, column block) ----
    const int nsplit = a.tile_nsplit[tile];
    bool owner = true;
    if (nsplit > 1) {
        __shared__ int last;
        T *part = reinterpret_cast<T *>(a.part);
        const int64_t tile_elems = int64_t(TILE_R) * BN;
        const int ncb = gridDim.y;
        const int64_t slot = int64_t(a.tile_first[tile] + wu.chunk) * ncb + blockIdx.y;
        T *mine = part + slot * tile_elems;
#pragma unroll
        for (int m = 0; m < TM; ++m)
#pragma unroll
            for (int j = 0; j < TN; ++j)
                mine[micro_index<TM, TILE_R>(ty, m) * BN + micro_index<TN, BN>(tx, j)] = acc[m][j];
        __threadfence();
        __syncthreads();
        if (tid == 0) {
            unsigned *ctr = &a.counters[int64_t(tile) * ncb + blockIdx.y];
            last = atomicAdd(ctr, 1u) == unsigned(nsplit - 1);
            if (last) *ctr = 0u;
        }
        __syncthreads();
        owner = last != 0;
        if (owner) {
            __threadfence();
#pragma unroll
            for (int m = 0; m < TM; ++m)
#pragma unroll
                for (int j = 0; j < TN; ++j) acc[m][j] = T(0);
            for (int s = 0; s < nsplit; ++s) {
                const T *src = part + (int64_t(a.tile_first[tile] + s) * ncb + blockIdx.y) * tile_elems;
#pragma unroll
                for (int m = 0; m < TM; ++m)
#pragma unroll
                    for (int j = 0; j < TN; ++j)
                        acc[m][j] += __ldcg(&src[micro_index<TM, TILE_R>(ty, m) * BN + micro_index<TN, BN>(tx, j)]);
            }
        }
    }

    // ---- epilogue ----
    double pacc = 0.0;
    if (owner) {
        const double g2 = 2.0 * a.gamma;
#pragma unroll
        for (int m = 0; m < TM; ++m) {
            const int64_t row = r0 + micro_index<TM, TILE_R>(ty, m);
            if (row >= rows) continue;
#pragma unroll
            for (int j = 0; j < TN; ++j) {
                const int64_t n = n0 + micro_index<TN, BN>(tx, j);
                if (n >= N) continue;
                const double v = double(acc[m][j]);
                const int64_t k = row * N + n;
                if (FWD) {
                    if (MODE == FWD_STORE) {
                        out[k] = v;
                    } else if (MODE == FWD_RESID) {
                        const double r = v - aux[k];
                        out[k] = r;
                        pacc += r * r;
                    } else {
                        const double r = aux[k];
                        out[k] = r + v;
                        pacc += 2.0 * r * v + v * v;
                    }
                } else {
                    if (MODE == ADJ_STORE) {
                        out[k] = v;
                    } else {
                        double lx = 0.0;
                        if (g2 != 0.0) {
                            const double xi = aux[k];
                            if (row < M - 1) lx += xi - aux[k + N];
                            if (row > 0) lx += xi - aux[k - N];
                        }
                        out[k] = 2.0 * v + g2 * lx;
                    }
                }
            }
        }
    }
    if (FWD && MODE != FWD_STORE) {
        double vv[1] = {pacc};
        DevScalars *sc = a.sc;
        grid_reduce<1>(vv, a.partials, a.pstride, &sc->ticket[0], [sc](const double *t) {
            if (MODE == FWD_RESID) sc->res2 = t[0];
            else sc->dres = t[0];
        });
    }
}

// ----------------------------------------------------------------------------
// launchers
// ----------------------------------------------------------------------------
int band_bn(int64_t N)
{
    if (N <= 32) return 32;
    if (N <= 64) return 64;
    return 128;
}

template <typename T>
size_t band_smem_bytes(int bn)
{
    if (bn == 128) return sizeof(SmemTile<T, 128>);
    if (bn == 64) return sizeof(SmemTile<T, 64>);
    return sizeof(SmemTile<T, 32>);
}
template size_t band_smem_bytes<float>(int);
template size_t band_smem_bytes<double>(int);

static BandArgs band_args(Plan &p, int prec, bool fwd)
{
    BandArgs a;
    a.M = p.M; a.N = p.N; a.D = p.D;
    a.lam = p.lam; a.lo = p.lo; a.hi = p.hi; a.aoff = p.aoff;
    const bool dbl = prec == TOMO_PREC_FP64;
    a.anchor = dbl ? (const void *)p.anchor : (const void *)p.anchor_f;
    a.rinv = p.ratio_inv;
    a.rinv2 = p.ratio_inv_f2;
    a.lam2 = p.lam_f2;
    const Schedule &s = p.sched[fwd ? 0 : 1][dbl ? 1 : 0];
    a.units = s.units;
    a.tile_first = s.tile_first;
    a.tile_nsplit = s.tile_nsplit;
    a.counters = s.counters;
    a.part = s.part;
    a.gate = nullptr;
    a.partials = p.partials;
    a.pstride = p.max_partials;
    a.sc = p.sc;
    a.gamma = p.gamma;
    return a;
}

template <typename T, int BN, bool FWD, int MODE>
static cudaError_t launch_band_t(Plan &p, const BandArgs &a, int n_units, const double *In,
                                 double *out, const double *aux)
{
    auto kern = k_band<T, BN, FWD, MODE>;
    const size_t smem = sizeof(SmemTile<T, BN>);
    // one attribute call per instantiation (thread-safe static initialisation)
    static const cudaError_t cfg =
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (cfg != cudaSuccess) return cfg;
    dim3 grid(unsigned(n_units), unsigned((p.N + BN - 1) / BN));
    kern<<<grid, GEMM_THREADS, smem, p.stream>>>(a, In, out, aux);
    count_launch();
    return cudaGetLastError();
}

template <typename T, bool FWD, int MODE>
static cudaError_t launch_band_bn(Plan &p, const BandArgs &a, int n_units, const double *In,
                                  double *out, const double *aux)
{
    switch (band_bn(p.N)) {
    case 128: return launch_band_t<T, 128, FWD, MODE>(p, a, n_units, In, out, aux);
    case 64: return launch_band_t<T, 64, FWD, MODE>(p, a, n_units, In, out, aux);
    default: return launch_band_t<T, 32, FWD, MODE>(p, a, n_units, In, out, aux);
    }
}

template <bool FWD, int MODE>
static cudaError_t launch_band(Plan &p, int prec, const int32_t *gate, const double *In,
                               double *out, const double *aux)
{
    BandArgs a = band_args(p, prec, FWD);
    a.gate = gate;
    const bool dbl = prec == TOMO_PREC_FP64;
    const int n_units = p.sched[FWD ? 0 : 1][dbl ? 1 : 0].n_units;
    if (dbl) return launch_band_bn<double, FWD, MODE>(p, a, n_units, In, out, aux);
    return launch_band_bn<float, FWD, MODE>(p, a, n_units, In, out, aux);
}

cudaError_t launch_forward(Plan &p, int prec, FwdMode mode, const double *X, double *out,
                           const double *P_or_R, bool gated)
{
    const int32_t *gate = gated ? &p.sc->cg_active : nullptr;
    switch (mode) {
    case FWD_STORE: return launch_band<true, FWD_STORE>(p, prec, gate, X, out, P_or_R);
    case FWD_RESID: return launch_band<true, FWD_RESID>(p, prec, gate, X, out, P_or_R);
    default: return launch_band<true, FWD_DELTA>(p, prec, gate, X, out, P_or_R);
    }
}

// Line-search product: runs only if the trial kernel cleared it (no negative
// implicit entry), so a rejected stage-2 trial costs no contraction.
cudaError_t launch_forward_gated_ls(Plan &p, int prec, FwdMode mode, const double *X, double *out,
                                   const double *P_or_R)
{
    const int32_t *gate = &p.sc->ls_go;
    if (mode == FWD_RESID) return launch_band<true, FWD_RESID>(p, prec, gate, X, out, P_or_R);
    return launch_band<true, FWD_DELTA>(p, prec, gate, X, out, P_or_R);
}

cudaError_t launch_adjoint(Plan &p, int prec, AdjMode mode, const double *Y, double *out,
                           const double *Xreg, bool gated)
{
    const int32_t *gate = gated ? &p.sc->cg_active : nullptr;
    if (mode == ADJ_STORE) return launch_band<false, ADJ_STORE>(p, prec, gate, Y, out, Xreg);
    return launch_band<false, ADJ_GRAD>(p, prec, gate, Y, out, Xreg);
}

}  // namespace tomo
