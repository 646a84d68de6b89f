// noalloc.cu -- tomo_objective_noalloc: the objective value
// f = ||P - F Theta||^2 + gamma sum (Theta_{i,n} - Theta_{i+1,n})^2 without a
// plan and without allocating anything.
//
// Some callers cannot allocate device memory at the point where they need the
// objective: code running inside a memory pool or arena that owns every
// allocation of the process (cudaMalloc/cudaFree would bypass it or fail),
// code called from inside a framework that forbids allocation in its hot loop
// (cudaMalloc/cudaFree synchronise the device), or a caller whose memory is
// already committed to its own buffers.  tomo_plan allocates its tables and
// workspaces, so such callers use this entry point instead.
//
// Its only scratch memory is the file-scope device array g_noalloc_scratch
// below: TOMO_NOALLOC_MAX_ROWS doubles (2 MiB), reserved in every device that
// loads the library for as long as the library stays loaded.  Host code may
// not use the array's name as a device address (on the host the symbol is a
// stand-in; a kernel given it would fault or, where the GPU can reach host
// memory, silently use the wrong memory).  The host therefore asks the
// runtime for the device address once per device, with that device current
// (cudaGetSymbolAddress), caches it, and passes it to the kernels.  The first
// call on each device performs that set-up; make that first call before any
// stream capture begins.
//
// Every call uses the same array and keeps the last call's contents: each call
// writes the D + M entries it reads before reading them, so nothing has to
// start at zero, but two calls whose kernels overlap on the GPU (different
// streams, or different host threads) race on the array and return garbage.
// Order such calls on one stream.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <mutex>

#include "poisson.cuh"
#include "tomo_device.cuh"
#include "tomo_internal.cuh"

namespace tomo {

constexpr int NOALLOC_THREADS = 128;

// Per-row partial sums: [0, D) the probes' sum_n r^2, [D, D + M) the
// regulariser's rows.
static __device__ __align__(256) double g_noalloc_scratch[TOMO_NOALLOC_MAX_ROWS];

// One CTA per probe (grid-stride): O_{d,n} = sum_i F_{d,i} Theta_{i,n} over the
// probe's band, weights evaluated in log space in double per photon number
// (no anchor table: the plan-free path has no tables), then
// scratch[d] = sum_n (O_{d,n} - P_{d,n})^2.  The same CTAs then write the
// regulariser rows scratch[D + i] = gamma sum_n (Theta_{i,n} - Theta_{i+1,n})^2.
__global__ void __launch_bounds__(NOALLOC_THREADS)
k_objective_rows(int64_t M, int64_t N, int64_t D, const double *lam, double band_k, double gamma,
                 const double *P, const double *Th, double *scratch)
{
    __shared__ double w[NOALLOC_THREADS];
    __shared__ double red[NOALLOC_THREADS / 32];
    const int tid = threadIdx.x;
    constexpr int NPT = MAX_N / NOALLOC_THREADS;  // outcomes per thread
    for (int64_t d = blockIdx.x; d < D; d += gridDim.x) {
        const double x = lam[d];
        if (!(x >= 0.0) || isinf(x)) {
            // an invalid mean photon number (negative, NaN or infinite; the
            // array lives in device memory, so the host cannot check it)
            // makes the objective NaN instead of indexing with a band
            // computed from it
            if (tid == 0) scratch[d] = __longlong_as_double(0x7ff8000000000000LL);
            continue;
        }
        int64_t lo, hi;
        if (band_k <= 0.0) {
            lo = 0;
            hi = M - 1;
        } else {
            const double s = sqrt(x);
            const double ks = __dmul_rn(band_k, s);
            const double a = floor(__dsub_rn(x, ks));
            double b = ceil(__dadd_rn(x, ks));
            if (b < 16.0) b = 16.0;
            lo = a < 0.0 ? 0 : int64_t(a);
            hi = b > double(M - 1) ? M - 1 : int64_t(b);
            if (lo > M - 1) lo = M;
        }
        double acc[NPT];
#pragma unroll
        for (int k = 0; k < NPT; ++k) acc[k] = 0.0;
        for (int64_t i0 = lo; i0 <= hi; i0 += NOALLOC_THREADS) {
            const int64_t i = i0 + tid;
            w[tid] = (i <= hi) ? poisson_weight(i, x) : 0.0;
            __syncthreads();
            const int cnt = int(hi - i0 + 1 < NOALLOC_THREADS ? hi - i0 + 1 : NOALLOC_THREADS);
            for (int j = 0; j < cnt; ++j) {
                const double wj = w[j];
                const double *row = Th + (i0 + j) * N;
#pragma unroll
                for (int k = 0; k < NPT; ++k) {
                    const int64_t n = tid + int64_t(k) * NOALLOC_THREADS;
                    if (n < N) acc[k] += wj * row[n];
                }
            }
            __syncthreads();
        }
        double s2 = 0.0;
#pragma unroll
        for (int k = 0; k < NPT; ++k) {
            const int64_t n = tid + int64_t(k) * NOALLOC_THREADS;
            if (n < N) {
                const double r = acc[k] - P[d * N + n];
                s2 += r * r;
            }
        }
        s2 = warp_sum(s2);
        if ((tid & 31) == 0) red[tid >> 5] = s2;
        __syncthreads();
        if (tid == 0) {
            double t = 0.0;
            for (int q = 0; q < NOALLOC_THREADS / 32; ++q) t += red[q];
            scratch[d] = t;
        }
        __syncthreads();
    }
    for (int64_t i = blockIdx.x; i < M; i += gridDim.x) {
        double s2 = 0.0;
        if (i < M - 1)
            for (int64_t n = tid; n < N; n += NOALLOC_THREADS) {
                const double t = Th[i * N + n] - Th[(i + 1) * N + n];
                s2 += t * t;
            }
        s2 = warp_sum(s2);
        if ((tid & 31) == 0) red[tid >> 5] = s2;
        __syncthreads();
        if (tid == 0) {
            double t = 0.0;
            for (int q = 0; q < NOALLOC_THREADS / 32; ++q) t += red[q];
            scratch[D + i] = gamma * t;
        }
        __syncthreads();
    }
}

// f = sum of the D + M partial sums, in index order within each thread and a
// fixed tree across threads (deterministic); one CTA.
__global__ void __launch_bounds__(256) k_objective_total(int64_t rows, const double *scratch, double *f)
{
    __shared__ double red[8];
    double s = 0.0;
    for (int64_t k = threadIdx.x; k < rows; k += 256) s += scratch[k];
    s = warp_sum(s);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int q = 0; q < 8; ++q) t += red[q];
        *f = t;
    }
}

// Device address of g_noalloc_scratch, looked up once per device.
static std::mutex g_scratch_mu;
static double *g_scratch_ptr[64];
static bool g_scratch_ready[64];

static cudaError_t scratch_address(double **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_ready[dev]) {
        void *ptr = nullptr;
        e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[dev] = static_cast<double *>(ptr);
        g_scratch_ready[dev] = true;
    }
    *out = g_scratch_ptr[dev];
    return cudaSuccess;
}

}  // namespace tomo

extern "C" tomo_status tomo_objective_noalloc(int64_t M, int64_t N, int64_t D, const double *lambda,
                                              double band_k, double gamma, const double *P,
                                              const double *Theta, double *f, void *stream)
{
    using namespace tomo;
    if (!lambda || !P || !Theta || !f) return tomo_set_error(TOMO_EINVAL, "NULL argument");
    if (M < 1 || N < 2 || N > MAX_N || D < 1)
        return tomo_set_error(TOMO_EINVAL, "sizes out of range (M >= 1, 2 <= N <= 1024, D >= 1)");
    if (D > TOMO_NOALLOC_MAX_ROWS || M > TOMO_NOALLOC_MAX_ROWS - D)
        return tomo_set_error(TOMO_EINVAL,
                              "D + M exceeds the scratch of tomo_objective_noalloc (TOMO_NOALLOC_MAX_ROWS = 262144)");
    if (!std::isfinite(gamma) || gamma < 0.0 || !std::isfinite(band_k))
        return tomo_set_error(TOMO_EINVAL, "gamma must be finite and >= 0, band_k finite");
    double *scratch = nullptr;
    cudaError_t e = scratch_address(&scratch);
    if (e != cudaSuccess) return tomo_set_error(TOMO_ECUDA, cudaGetErrorString(e));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int sms = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int64_t grid = int64_t(sms > 0 ? sms : 1) * 8;
    const int64_t rows = D > M ? D : M;
    if (grid > rows) grid = rows;
    k_objective_rows<<<unsigned(grid), NOALLOC_THREADS, 0, st>>>(M, N, D, lambda, band_k, gamma, P, Theta,
                                                                 scratch);
    count_launch();
    k_objective_total<<<1, 256, 0, st>>>(D + M, scratch, f);
    count_launch();
    e = cudaGetLastError();
    if (e != cudaSuccess) return tomo_set_error(TOMO_ECUDA, cudaGetErrorString(e));
    return TOMO_OK;
}
