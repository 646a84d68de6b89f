// smooth.cu -- long-range smoothing of a POVM estimate (Sec. "Regularisation
// and smoothing", Eq. smoothing):
//   Y_{i,n} = mean of X_{j,n} over j in [i - w_i, i + w_i],  w_i = floor(i / div),
// the window clipped to [0, M-1] (the mean then runs over the rows present),
// rows i < exclude copied unchanged.
//
// The windows grow with i (w ~ i/50), so a direct sum costs O(M^2 N / div)
// and is out of reach at M ~ 1e6.  The kernels instead form column prefix sums
// S_k = sum_{j <= k} X_j and take Y_i = (S_b - S_{a-1}) / (b - a + 1).  The
// difference of two large prefixes would cancel catastrophically in double (a
// window of values ~1e-10 far down a column whose early entries are ~1), so
// the prefixes are carried as unevaluated double-double sums (Knuth's
// TwoSum): the difference is then exact to ~1e-32 of the prefix and the only
// rounding left is that of the final division, as in the direct definition.
//
// Three launches on the plan stream:
//   1. per block of SMOOTH_ROWS rows and 128 columns: in-block inclusive
//      prefix (hi, lo) of every column, and the block's column totals;
//   2. per 128 columns: exclusive scan of the block totals, serially over the
//      blocks of each column (one thread per column);
//   3. per element: the window difference, the division, and the copy of the
//      excluded rows.
// Workspaces: two M x N double arrays for the prefix (hi, lo) and 2 x blocks x N
// doubles for the block offsets; the input is read only by launches 1 and 3
// (row i < exclude only), so X and Y may be the same array.
#include <cuda_runtime.h>

#include <cmath>

#include "tomo_internal.cuh"

namespace tomo {

constexpr int SMOOTH_ROWS = 128;
constexpr int SMOOTH_COLS = 128;

struct DD {
    double hi, lo;
};

// Knuth's TwoSum: s + e == a + b exactly.
__device__ __forceinline__ DD two_sum(double a, double b)
{
    const double s = __dadd_rn(a, b);
    const double bb = __dsub_rn(s, a);
    const double e = __dadd_rn(__dsub_rn(a, __dsub_rn(s, bb)), __dsub_rn(b, bb));
    return {s, e};
}

__device__ __forceinline__ DD dd_add(DD a, DD b)
{
    DD s = two_sum(a.hi, b.hi);
    const double t = __dadd_rn(s.lo, __dadd_rn(a.lo, b.lo));
    return two_sum(s.hi, t);
}

__device__ __forceinline__ DD dd_neg(DD a) { return {-a.hi, -a.lo}; }

__global__ void __launch_bounds__(SMOOTH_COLS)
k_smooth_block_prefix(int64_t M, int64_t N, const double *X, double *Shi, double *Slo,
                      double *Thi, double *Tlo)
{
    const int64_t n = int64_t(blockIdx.y) * SMOOTH_COLS + threadIdx.x;
    if (n >= N) return;
    const int64_t b = blockIdx.x;
    const int64_t r0 = b * SMOOTH_ROWS;
    const int64_t r1 = r0 + SMOOTH_ROWS < M ? r0 + SMOOTH_ROWS : M;
    DD acc{0.0, 0.0};
    for (int64_t i = r0; i < r1; ++i) {
        acc = dd_add(acc, DD{X[i * N + n], 0.0});
        Shi[i * N + n] = acc.hi;
        Slo[i * N + n] = acc.lo;
    }
    Thi[b * N + n] = acc.hi;
    Tlo[b * N + n] = acc.lo;
}

// In place: T_b <- sum of the totals of blocks 0..b-1.
__global__ void __launch_bounds__(SMOOTH_COLS)
k_smooth_block_offsets(int64_t nblk, int64_t N, double *Thi, double *Tlo)
{
    const int64_t n = int64_t(blockIdx.x) * SMOOTH_COLS + threadIdx.x;
    if (n >= N) return;
    DD acc{0.0, 0.0};
    for (int64_t b = 0; b < nblk; ++b) {
        const DD t{Thi[b * N + n], Tlo[b * N + n]};
        Thi[b * N + n] = acc.hi;
        Tlo[b * N + n] = acc.lo;
        acc = dd_add(acc, t);
    }
}

__device__ __forceinline__ DD prefix_at(int64_t k, int64_t N, int64_t n, const double *Shi,
                                        const double *Slo, const double *Thi, const double *Tlo)
{
    const int64_t b = k / SMOOTH_ROWS;
    return dd_add(DD{Thi[b * N + n], Tlo[b * N + n]}, DD{Shi[k * N + n], Slo[k * N + n]});
}

__global__ void __launch_bounds__(256)
k_smooth_apply(int64_t M, int64_t N, int64_t exclude, double div, const double *X, double *Y,
               const double *Shi, const double *Slo, const double *Thi, const double *Tlo)
{
    const int64_t total = M * N;
    for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < total;
         e += int64_t(gridDim.x) * blockDim.x) {
        const int64_t i = e / N, n = e - i * N;
        if (i < exclude) {
            Y[e] = X[e];
            continue;
        }
        const int64_t w = int64_t(floor(double(i) / div));
        const int64_t a = i - w < 0 ? 0 : i - w;
        const int64_t b = i + w > M - 1 ? M - 1 : i + w;
        DD s = prefix_at(b, N, n, Shi, Slo, Thi, Tlo);
        if (a > 0) s = dd_add(s, dd_neg(prefix_at(a - 1, N, n, Shi, Slo, Thi, Tlo)));
        const double v = __dadd_rn(s.hi, s.lo) / double(b - a + 1);
        // a mean of non-negative entries; the clamp only removes a -0 or a
        // rounding residue below zero
        Y[e] = v > 0.0 ? v : 0.0;
    }
}

cudaError_t launch_smooth(Plan &p, const double *X, double *Y, int64_t exclude, double div)
{
    const int64_t M = p.M, N = p.N;
    const int64_t nblk = (M + SMOOTH_ROWS - 1) / SMOOTH_ROWS;
    const unsigned cblk = unsigned((N + SMOOTH_COLS - 1) / SMOOTH_COLS);
    // prefix (hi, lo) in two M x N workspaces, block offsets (2 x nblk x N <= M x N
    // doubles since SMOOTH_ROWS >= 2) in a third
    double *Shi = p.s, *Slo = p.g, *Thi = p.x, *Tlo = p.x + nblk * N;
    k_smooth_block_prefix<<<dim3(unsigned(nblk), cblk), SMOOTH_COLS, 0, p.stream>>>(M, N, X, Shi, Slo,
                                                                                 Thi, Tlo);
    count_launch();
    k_smooth_block_offsets<<<cblk, SMOOTH_COLS, 0, p.stream>>>(nblk, N, Thi, Tlo);
    count_launch();
    int64_t grid = (M * N + 255) / 256;
    const int64_t cap = int64_t(p.num_sms) * 8;
    if (grid > cap) grid = cap;
    k_smooth_apply<<<unsigned(grid), 256, 0, p.stream>>>(M, N, exclude, div, X, Y, Shi, Slo, Thi, Tlo);
    count_launch();
    return cudaGetLastError();
}

}  // namespace tomo

// ---------------------------------------------------------------------------
// Infidelity of two phase-insensitive POVMs (Eq. fidelities), per outcome n:
// the operators are diagonal in the photon-number basis, so
//   F_n = (sum_i sqrt(A_in B_in))^2 / (sum_i A_in  sum_i B_in),
// and the result is 1 - F_n.  Two launches: per-CTA column sums of
// sqrt(A B), A and B over a block of rows (threads along the row, coalesced),
// then one thread per outcome adds the CTAs' sums in CTA order.
// ---------------------------------------------------------------------------
namespace tomo {

__global__ void __launch_bounds__(256)
k_fid_partials(int64_t M, int64_t N, int64_t rows_per_cta, const double *A, const double *B, double *part)
{
    const int64_t i0 = int64_t(blockIdx.x) * rows_per_cta;
    const int64_t i1 = i0 + rows_per_cta < M ? i0 + rows_per_cta : M;
    for (int64_t n = threadIdx.x; n < N; n += blockDim.x) {
        double sab = 0.0, sa = 0.0, sb = 0.0;
        for (int64_t i = i0; i < i1; ++i) {
            const double a = A[i * N + n], b = B[i * N + n];
            sab += sqrt(a * b);
            sa += a;
            sb += b;
        }
        double *o = part + int64_t(blockIdx.x) * 3 * N;
        o[n] = sab;
        o[N + n] = sa;
        o[2 * N + n] = sb;
    }
}

__global__ void k_fid_final(int64_t N, int64_t ctas, const double *part, double *out)
{
    const int64_t n = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    if (n >= N) return;
    double sab = 0.0, sa = 0.0, sb = 0.0;
    for (int64_t c = 0; c < ctas; ++c) {
        sab += part[c * 3 * N + n];
        sa += part[c * 3 * N + N + n];
        sb += part[c * 3 * N + 2 * N + n];
    }
    out[n] = 1.0 - (sab * sab) / (sa * sb);
}

cudaError_t launch_infidelity(Plan &p, const double *A, const double *B, double *out_dev)
{
    const int64_t M = p.M, N = p.N;
    // 3 N partial sums per CTA: in the M x N workspace s when 3 ctas <= M,
    // else (tiny M: one CTA) in the reduction partials (>= 4 x 1216 doubles)
    int64_t ctas = int64_t(p.num_sms) * 4;
    if (3 * ctas > M) ctas = M / 3 > 0 ? M / 3 : 1;
    const int64_t rows = (M + ctas - 1) / ctas;
    ctas = (M + rows - 1) / rows;
    double *part = (3 * ctas <= M) ? p.s : p.partials;
    k_fid_partials<<<unsigned(ctas), 256, 0, p.stream>>>(M, N, rows, A, B, part);
    k_fid_final<<<unsigned((N + 127) / 128), 128, 0, p.stream>>>(N, ctas, part, out_dev);
    count_launch(2);
    return cudaGetLastError();
}

}  // namespace tomo
