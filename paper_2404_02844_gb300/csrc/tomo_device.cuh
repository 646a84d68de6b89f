// tomo_device.cuh -- device helpers shared by the kernels of libtomo:
// warp/block reductions and the deterministic "last CTA finalises" pattern.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "tomo_internal.cuh"

namespace tomo {

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ float warp_sum(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ int warp_sum_int(int v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ double warp_max(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

__device__ __forceinline__ double warp_min(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Reduces NV per-thread values over the whole grid.  Every CTA writes its NV
// partial sums to partials[k * stride + cta]; the CTA that takes the last
// ticket sums all partials in CTA order (fixed order: deterministic result)
// and calls fin(sums) from thread 0, then re-arms the ticket.  No CTA waits
// for another.  Must be called by every thread of every CTA.
template <int NV, typename Fin>
__device__ __forceinline__ void grid_reduce(double (&v)[NV], double *partials, int64_t stride,
                                            unsigned int *ticket, Fin fin)
{
    __shared__ double sh[NV][32];
    __shared__ int is_last;
    const int tid = threadIdx.x + threadIdx.y * blockDim.x;
    const int nthr = blockDim.x * blockDim.y;
    const int lane = tid & 31, warp = tid >> 5, nwarps = (nthr + 31) >> 5;
    const unsigned nblocks = gridDim.x * gridDim.y * gridDim.z;
    const unsigned bid = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        double t = warp_sum(v[k]);
        if (lane == 0) sh[k][warp] = t;
    }
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            double t = lane < nwarps ? sh[k][lane] : 0.0;
            t = warp_sum(t);
            if (lane == 0) partials[k * stride + bid] = t;
        }
        if (lane == 0) {
            __threadfence();
            unsigned got = atomicAdd(ticket, 1u);
            is_last = (got == nblocks - 1);
        }
    }
    __syncthreads();
    if (!is_last) return;
    __threadfence();
    double acc[NV];
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        double t = 0.0;
        for (unsigned b = tid; b < nblocks; b += nthr) t += __ldcg(&partials[k * stride + b]);
        acc[k] = t;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        double t = warp_sum(acc[k]);
        if (lane == 0) sh[k][warp] = t;
    }
    __syncthreads();
    if (tid == 0) {
        double tot[NV];
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            double t = 0.0;
            for (int w = 0; w < nwarps; ++w) t += sh[k][w];
            tot[k] = t;
        }
        fin(tot);
        *ticket = 0u;
        __threadfence();
    }
}

}  // namespace tomo
