// warmstart.cu -- learned warm start: a network that maps measured outcome
// frequencies P (D probes x C0 outcome columns) to a starting POVM Theta0
// (M x C0, every row on the simplex of its first ncols columns) for
// Algorithm 3, trained on (P, Theta) pairs.  The paper has no counterpart: it
// starts from Theta^(0) = 1/N.
//
// Network (one sample):
//   Y1 = conv1d(P, W1, b1, stride S1)             (D/S1) x C1
//   Y2 = conv1d(relu(Y1), W2, b2, stride S2)      (D/S1/S2) x C2
//   Y3 = W3 flat(relu(Y2)) + b3                   H
//   Z  = W4 relu(Y3) + b4                         M x C0 logits
//   Theta0[i, :] = softmax of Z[i, :] over the first ncols columns
// conv1d(X, W, b, S)[t, co] = b[co] + sum_{ci,k} W[co,ci,k] X[S t + k - K/2, ci]
// (zero padding).  Loss: row-wise cross-entropy against the target POVM,
// averaged over rows and samples; optimiser: Adam.
//
// Every kernel accumulates in float; training keeps float master weights,
// inference reads a bf16 copy of them (rounded to nearest even).  Reductions
// over the batch or over a layer's inputs run in a fixed order (one thread,
// or one CTA with a fixed tree): results do not depend on scheduling.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "tomo_internal.cuh"

namespace tomo {

namespace {

constexpr float ADAM_B1 = 0.9f, ADAM_B2 = 0.999f, ADAM_EPS = 1e-8f;
constexpr int RED_T = 256;

struct WsShape {
    int64_t D, C0, M;
    int64_t C1, C2, K, S1, S2, H;
    int64_t T1() const { return D / S1; }
    int64_t T2() const { return T1() / S2; }
    int64_t F() const { return T2() * C2; }
};

template <typename WT> __device__ __forceinline__ float ldw(const WT *p, int64_t i);
template <> __device__ __forceinline__ float ldw<float>(const float *p, int64_t i) { return p[i]; }
template <> __device__ __forceinline__ float ldw<__nv_bfloat16>(const __nv_bfloat16 *p, int64_t i)
{
    return __bfloat162float(p[i]);
}

__device__ __forceinline__ float block_sum(float v, float *sh)
{
    // fixed tree: warp shuffles, then warp 0 over the warp sums
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    float t = 0.f;
    if (warp == 0) {
        t = lane < int(blockDim.x >> 5) ? sh[lane] : 0.f;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    }
    __syncthreads();
    return t;  // valid in thread 0
}

// X0[b, s, c] = P[b, s, c] for c < ncols[b], else 0 (P rows of stride pstride)
__global__ void k_ws_load(int64_t B, int64_t rows, int64_t C0, const double *P, int64_t pstride,
                          const int32_t *ncols, float *X)
{
    const int64_t n = B * rows * C0;
    for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < n; e += int64_t(gridDim.x) * blockDim.x) {
        const int64_t c = e % C0, r = (e / C0) % rows, b = e / (C0 * rows);
        X[e] = c < ncols[b] ? float(P[(b * rows + r) * pstride + c]) : 0.f;
    }
}

template <typename WT, bool RELU_IN>
__global__ void k_conv_fwd(int64_t B, int64_t Tin, int64_t Cin, int64_t Tout, int64_t Cout, int64_t K,
                           int64_t S, const float *X, const WT *W, const WT *bias, float *Y)
{
    const int64_t n = B * Tout * Cout;
    for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < n; e += int64_t(gridDim.x) * blockDim.x) {
        const int64_t co = e % Cout, t = (e / Cout) % Tout, b = e / (Cout * Tout);
        float acc = ldw(bias, co);
        for (int64_t k = 0; k < K; ++k) {
            const int64_t s = S * t + k - K / 2;
            if (s < 0 || s >= Tin) continue;
            const float *x = X + (b * Tin + s) * Cin;
            for (int64_t ci = 0; ci < Cin; ++ci) {
                float xv = x[ci];
                if (RELU_IN) xv = fmaxf(xv, 0.f);
                acc = fmaf(ldw(W, (co * Cin + ci) * K + k), xv, acc);
            }
        }
        Y[e] = acc;
    }
}

// Y[b, o] = bias[o] + sum_j W[o, j] relu(X[b, j]); one CTA per (b, o)
template <typename WT>
__global__ void __launch_bounds__(RED_T) k_linear_fwd(int64_t Nout, int64_t Nin, const float *X, const WT *W,
                                                      const WT *bias, float *Y)
{
    __shared__ float sh[32];
    const int64_t b = blockIdx.y, o = blockIdx.x;
    float acc = 0.f;
    for (int64_t j = threadIdx.x; j < Nin; j += RED_T)
        acc = fmaf(ldw(W, o * Nin + j), fmaxf(X[b * Nin + j], 0.f), acc);
    acc = block_sum(acc, sh);
    if (threadIdx.x == 0) Y[b * Nout + o] = acc + ldw(bias, o);
}

// Z[b, j] = bias[j] + sum_h W[j, h] relu(Y3[b, h]) (short inner sum, thread per output)
template <typename WT>
__global__ void k_out_fwd(int64_t B, int64_t J, int64_t H, const float *Y3, const WT *W, const WT *bias, float *Z)
{
    const int64_t n = B * J;
    for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < n; e += int64_t(gridDim.x) * blockDim.x) {
        const int64_t j = e % J, b = e / J;
        float acc = ldw(bias, j);
        for (int64_t h = 0; h < H; ++h) acc = fmaf(ldw(W, j * H + h), fmaxf(Y3[b * H + h], 0.f), acc);
        Z[e] = acc;
    }
}

// Per row (b, i): Theta0 = masked softmax of Z (in place); with a target T:
// rowloss = -sum T log Theta0 and dZ = scale (Theta0 sum(T) - T).  One warp
// per row, C0 <= 32 * 8.
__global__ void k_softmax_ce(int64_t B, int64_t M, int64_t C0, const int32_t *ncols, float *Z, const float *T,
                             float *dZ, float scale, float *rowloss)
{
    constexpr int VPL = 8;
    const int lane = threadIdx.x & 31;
    const int64_t rows = B * M;
    const int64_t w0 = (blockIdx.x * int64_t(blockDim.x) + threadIdx.x) >> 5;
    const int64_t nw = (int64_t(gridDim.x) * blockDim.x) >> 5;
    for (int64_t r = w0; r < rows; r += nw) {
        const int64_t b = r / M;
        const int nc = ncols[b];
        float z[VPL];
        float mx = -INFINITY;
#pragma unroll
        for (int k = 0; k < VPL; ++k) {
            const int n = lane + 32 * k;
            z[k] = (n < nc && n < C0) ? Z[r * C0 + n] : -INFINITY;
            mx = fmaxf(mx, z[k]);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        float se = 0.f;
#pragma unroll
        for (int k = 0; k < VPL; ++k) {
            const int n = lane + 32 * k;
            if (n < nc && n < C0) se += expf(z[k] - mx);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) se += __shfl_xor_sync(0xffffffffu, se, o);
        const float lse = logf(se);
        float ts = 0.f, ls = 0.f;
        if (T) {
#pragma unroll
            for (int k = 0; k < VPL; ++k) {
                const int n = lane + 32 * k;
                if (n < nc && n < C0) {
                    const float t = T[r * C0 + n];
                    ts += t;
                    if (t > 0.f) ls -= t * (z[k] - mx - lse);
                }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                ts += __shfl_xor_sync(0xffffffffu, ts, o);
                ls += __shfl_xor_sync(0xffffffffu, ls, o);
            }
        }
#pragma unroll
        for (int k = 0; k < VPL; ++k) {
            const int n = lane + 32 * k;
            if (n >= C0) continue;
            const float th = (n < nc) ? expf(z[k] - mx - lse) : 0.f;
            Z[r * C0 + n] = th;
            if (dZ) dZ[r * C0 + n] = (n < nc) ? scale * (th * ts - T[r * C0 + n]) : 0.f;
        }
        if (rowloss && lane == 0) rowloss[r] = scale * ls;
    }
}

// gW4[j, h] = sum_b dZ[b, j] relu(Y3[b, h]), gb4[j] = sum_b dZ[b, j]
__global__ void k_out_bwd_w(int64_t B, int64_t J, int64_t H, const float *dZ, const float *Y3, float *gW, float *gb)
{
    for (int64_t j = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; j < J; j += int64_t(gridDim.x) * blockDim.x) {
        float sb = 0.f;
        for (int64_t b = 0; b < B; ++b) sb += dZ[b * J + j];
        gb[j] = sb;
        for (int64_t h = 0; h < H; ++h) {
            float s = 0.f;
            for (int64_t b = 0; b < B; ++b) s = fmaf(dZ[b * J + j], fmaxf(Y3[b * H + h], 0.f), s);
            gW[j * H + h] = s;
        }
    }
}

// dY3[b, h] = (sum_j dZ[b, j] W4[j, h]) [Y3 > 0]; one CTA per (b, h)
__global__ void __launch_bounds__(RED_T) k_out_bwd_x(int64_t J, int64_t H, const float *dZ, const float *W,
                                                     const float *Y3, float *dY3)
{
    __shared__ float sh[32];
    const int64_t b = blockIdx.y, h = blockIdx.x;
    float acc = 0.f;
    for (int64_t j = threadIdx.x; j < J; j += RED_T) acc = fmaf(dZ[b * J + j], W[j * H + h], acc);
    acc = block_sum(acc, sh);
    if (threadIdx.x == 0) dY3[b * H + h] = Y3[b * H + h] > 0.f ? acc : 0.f;
}

// gW3[o, f] = sum_b dY3[b, o] relu(X[b, f]); gb3[o] = sum_b dY3[b, o]
__global__ void k_lin_bwd_w(int64_t B, int64_t Nout, int64_t Nin, const float *dY, const float *X, float *gW,
                            float *gb)
{
    const int64_t n = Nout * Nin;
    for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < n; e += int64_t(gridDim.x) * blockDim.x) {
        const int64_t f = e % Nin, o = e / Nin;
        float s = 0.f;
        for (int64_t b = 0; b < B; ++b) s = fmaf(dY[b * Nout + o], fmaxf(X[b * Nin + f], 0.f), s);
        gW[e] = s;
        if (f == 0) {
            float t = 0.f;
            for (int64_t b = 0; b < B; ++b) t += dY[b * Nout + o];
            gb[o] = t;
        }
    }
}

// dX[b, f] = (sum_o dY[b, o] W[o, f]) [Xpre[b, f] > 0]
__global__ void k_lin_bwd_x(int64_t B, int64_t Nout, int64_t Nin, const float *dY, const float *W,
                            const float *Xpre, float *dX)
{
    const int64_t n = B * Nin;
    for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < n; e += int64_t(gridDim.x) * blockDim.x) {
        const int64_t f = e % Nin, b = e / Nin;
        float s = 0.f;
        for (int64_t o = 0; o < Nout; ++o) s = fmaf(dY[b * Nout + o], W[o * Nin + f], s);
        dX[e] = Xpre[e] > 0.f ? s : 0.f;
    }
}

// gW[co, ci, k] = sum_{b, t} dY[b, t, co] act(X[b, S t + k - K/2, ci]) (one CTA
// per weight); the CTAs with ci = k = 0 also write gb[co] = sum_{b, t} dY[b, t, co]
template <bool RELU_IN>
__global__ void __launch_bounds__(RED_T) k_conv_bwd_w(int64_t B, int64_t Tin, int64_t Cin, int64_t Tout,
                                                      int64_t Cout, int64_t K, int64_t S, const float *X,
                                                      const float *dY, float *gW, float *gb)
{
    __shared__ float sh[32];
    const int64_t w = blockIdx.x;
    const int64_t k = w % K, ci = (w / K) % Cin, co = w / (K * Cin);
    const int64_t n = B * Tout;
    float acc = 0.f, accb = 0.f;
    for (int64_t q = threadIdx.x; q < n; q += RED_T) {
        const int64_t t = q % Tout, b = q / Tout;
        const float d = dY[(b * Tout + t) * Cout + co];
        const int64_t s = S * t + k - K / 2;
        if (s >= 0 && s < Tin) {
            float xv = X[(b * Tin + s) * Cin + ci];
            if (RELU_IN) xv = fmaxf(xv, 0.f);
            acc = fmaf(d, xv, acc);
        }
        accb += d;
    }
    acc = block_sum(acc, sh);
    if (threadIdx.x == 0) gW[w] = acc;
    if (ci == 0 && k == 0) {
        accb = block_sum(accb, sh);
        if (threadIdx.x == 0) gb[co] = accb;
    }
}

// dX[b, s, ci] = (sum_{k, co: S t + k - K/2 = s} W[co, ci, k] dY[b, t, co]) [Xpre > 0]
__global__ void k_conv_bwd_x(int64_t B, int64_t Tin, int64_t Cin, int64_t Tout, int64_t Cout, int64_t K,
                             int64_t S, const float *W, const float *dY, const float *Xpre, float *dX)
{
    const int64_t n = B * Tin * Cin;
    for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < n; e += int64_t(gridDim.x) * blockDim.x) {
        const int64_t ci = e % Cin, s = (e / Cin) % Tin, b = e / (Cin * Tin);
        float acc = 0.f;
        for (int64_t k = 0; k < K; ++k) {
            const int64_t num = s + K / 2 - k;
            if (num < 0 || num % S != 0) continue;
            const int64_t t = num / S;
            if (t >= Tout) continue;
            for (int64_t co = 0; co < Cout; ++co)
                acc = fmaf(W[(co * Cin + ci) * K + k], dY[(b * Tout + t) * Cout + co], acc);
        }
        dX[e] = Xpre[e] > 0.f ? acc : 0.f;
    }
}

__global__ void k_adam(int64_t n, float *p, const float *g, float *m, float *v, float lr, float bc1, float bc2)
{
    for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < n; e += int64_t(gridDim.x) * blockDim.x) {
        const float gv = g[e];
        const float mv = ADAM_B1 * m[e] + (1.f - ADAM_B1) * gv;
        const float vv = ADAM_B2 * v[e] + (1.f - ADAM_B2) * gv * gv;
        m[e] = mv;
        v[e] = vv;
        p[e] -= lr * (mv / bc1) / (sqrtf(vv / bc2) + ADAM_EPS);
    }
}

__global__ void k_to_bf16(int64_t n, const float *p, __nv_bfloat16 *q)
{
    for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < n; e += int64_t(gridDim.x) * blockDim.x)
        q[e] = __float2bfloat16_rn(p[e]);
}

// out = sum of n values in index order per thread, fixed tree across threads
__global__ void __launch_bounds__(RED_T) k_sum(int64_t n, const float *x, float *out)
{
    __shared__ float sh[32];
    float s = 0.f;
    for (int64_t e = threadIdx.x; e < n; e += RED_T) s += x[e];
    s = block_sum(s, sh);
    if (threadIdx.x == 0) *out = s;
}

__global__ void k_ws_store(int64_t M, int64_t C0, int64_t N, const float *Th, double *out)
{
    const int64_t n = M * N;
    for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < n; e += int64_t(gridDim.x) * blockDim.x) {
        const int64_t c = e % N, i = e / N;
        out[e] = double(Th[i * C0 + c]);
    }
}

}  // namespace

struct WarmStart {
    WsShape s;
    int64_t max_batch;
    cudaStream_t stream;
    bool own_stream;
    int num_sms;
    int64_t nparam;
    int64_t oW1, ob1, oW2, ob2, oW3, ob3, oW4, ob4;
    float *param, *grad, *m, *v;
    __nv_bfloat16 *pbf;
    bool bf_dirty;
    int64_t step;
    float *X0, *Y1, *Y2, *Y3, *Z, *T, *dZ, *dY3, *dY2, *dA1, *rowloss, *loss;
    int32_t *ncols;
};

// Shape of a warm-start handle (probes, photon numbers, padded outcome
// columns) for the callers that pair it with a plan; false for NULL.
bool ws_shape(const void *handle, int64_t *D, int64_t *M, int64_t *C0)
{
    const WarmStart *w = static_cast<const WarmStart *>(handle);
    if (!w) return false;
    *D = w->s.D;
    *M = w->s.M;
    *C0 = w->s.C0;
    return true;
}

}  // namespace tomo

// ------------------------------------------------------------------ host side
namespace tomo {
namespace {

template <typename T>
cudaError_t ws_alloc(T **p, int64_t n)
{
    *p = nullptr;
    return cudaMalloc(reinterpret_cast<void **>(p), sizeof(T) * size_t(n > 0 ? n : 1));
}

unsigned grid_for(const WarmStart &w, int64_t n, int threads = 256)
{
    int64_t g = (n + threads - 1) / threads;
    const int64_t cap = int64_t(w.num_sms) * 16;
    if (g > cap) g = cap;
    if (g < 1) g = 1;
    return unsigned(g);
}

void free_ws(WarmStart *w)
{
    if (!w) return;
    void *ptrs[] = {w->param, w->grad, w->m, w->v, w->pbf, w->X0, w->Y1, w->Y2, w->Y3, w->Z,
                    w->T, w->dZ, w->dY3, w->dY2, w->dA1, w->rowloss, w->loss, w->ncols};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    if (w->own_stream && w->stream) cudaStreamDestroy(w->stream);
    delete w;
}

// SplitMix64 (Steele, Lea & Flood 2014): deterministic parameter initialisation
uint64_t splitmix64(uint64_t &x)
{
    uint64_t z = (x += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Forward pass of `B` samples whose padded inputs are in X0 and ncols;
// weights in float (training) or bf16 (inference).
template <typename WT>
cudaError_t ws_forward(WarmStart &w, const WT *P, int64_t B)
{
    const WsShape &s = w.s;
    const WT *W1 = P + w.oW1, *b1 = P + w.ob1, *W2 = P + w.oW2, *b2 = P + w.ob2;
    const WT *W3 = P + w.oW3, *b3 = P + w.ob3, *W4 = P + w.oW4, *b4 = P + w.ob4;
    k_conv_fwd<WT, false><<<grid_for(w, B * s.T1() * s.C1), 256, 0, w.stream>>>(
        B, s.D, s.C0, s.T1(), s.C1, s.K, s.S1, w.X0, W1, b1, w.Y1);
    k_conv_fwd<WT, true><<<grid_for(w, B * s.T2() * s.C2), 256, 0, w.stream>>>(
        B, s.T1(), s.C1, s.T2(), s.C2, s.K, s.S2, w.Y1, W2, b2, w.Y2);
    k_linear_fwd<WT><<<dim3(unsigned(s.H), unsigned(B)), RED_T, 0, w.stream>>>(s.H, s.F(), w.Y2, W3, b3, w.Y3);
    k_out_fwd<WT><<<grid_for(w, B * s.M * s.C0), 256, 0, w.stream>>>(B, s.M * s.C0, s.H, w.Y3, W4, b4, w.Z);
    count_launch(4);
    return cudaGetLastError();
}

// Loss (to w.loss) and gradient (to w.grad) of a batch already loaded into
// X0, T and ncols.
cudaError_t ws_loss_grad(WarmStart &w, int64_t B)
{
    const WsShape &s = w.s;
    cudaError_t e = ws_forward<float>(w, w.param, B);
    if (e != cudaSuccess) return e;
    const float scale = float(1.0 / (double(B) * double(s.M)));
    k_softmax_ce<<<grid_for(w, B * s.M * 32), 256, 0, w.stream>>>(B, s.M, s.C0, w.ncols, w.Z, w.T, w.dZ, scale,
                                                                  w.rowloss);
    k_sum<<<1, RED_T, 0, w.stream>>>(B * s.M, w.rowloss, w.loss);
    float *g = w.grad;
    const float *Wp = w.param;
    const int64_t J = s.M * s.C0;
    k_out_bwd_w<<<grid_for(w, J), 256, 0, w.stream>>>(B, J, s.H, w.dZ, w.Y3, g + w.oW4, g + w.ob4);
    k_out_bwd_x<<<dim3(unsigned(s.H), unsigned(B)), RED_T, 0, w.stream>>>(J, s.H, w.dZ, Wp + w.oW4, w.Y3, w.dY3);
    k_lin_bwd_w<<<grid_for(w, s.H * s.F()), 256, 0, w.stream>>>(B, s.H, s.F(), w.dY3, w.Y2, g + w.oW3, g + w.ob3);
    k_lin_bwd_x<<<grid_for(w, B * s.F()), 256, 0, w.stream>>>(B, s.H, s.F(), w.dY3, Wp + w.oW3, w.Y2, w.dY2);
    k_conv_bwd_w<true><<<unsigned(s.C2 * s.C1 * s.K), RED_T, 0, w.stream>>>(
        B, s.T1(), s.C1, s.T2(), s.C2, s.K, s.S2, w.Y1, w.dY2, g + w.oW2, g + w.ob2);
    k_conv_bwd_x<<<grid_for(w, B * s.T1() * s.C1), 256, 0, w.stream>>>(
        B, s.T1(), s.C1, s.T2(), s.C2, s.K, s.S2, Wp + w.oW2, w.dY2, w.Y1, w.dA1);
    k_conv_bwd_w<false><<<unsigned(s.C1 * s.C0 * s.K), RED_T, 0, w.stream>>>(
        B, s.D, s.C0, s.T1(), s.C1, s.K, s.S1, w.X0, w.dA1, g + w.oW1, g + w.ob1);
    count_launch(9);
    return cudaGetLastError();
}

}  // namespace
}  // namespace tomo

using tomo::WarmStart;

extern "C" {

tomo_status tomo_ws_create(tomo_ws_t *out, const tomo_ws_desc *d)
{
    using namespace tomo;
    if (!out) return tomo_set_error(TOMO_EINVAL, "NULL output handle");
    *out = nullptr;
    if (!d) return tomo_set_error(TOMO_EINVAL, "NULL descriptor");
    WsShape s{d->D, d->C0, d->M, d->C1, d->C2, d->K, d->S1, d->S2, d->H};
    if (s.D < 1 || s.C0 < 2 || s.C0 > 256 || s.M < 1 || s.C1 < 1 || s.C2 < 1 || s.K < 1 || s.S1 < 1 ||
        s.S2 < 1 || s.H < 1 || d->max_batch < 1 || s.D % s.S1 != 0 || s.T1() % s.S2 != 0 || s.T2() < 1)
        return tomo_set_error(TOMO_EINVAL,
                              "warm-start shape out of range (2 <= C0 <= 256, D divisible by S1, D/S1 by S2)");
    WarmStart *w = new (std::nothrow) WarmStart();
    if (!w) return tomo_set_error(TOMO_ENOMEM, "host allocation failed");
    w->s = s;
    w->max_batch = d->max_batch;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&w->num_sms, cudaDevAttrMultiProcessorCount, dev);
    if (d->stream) {
        w->stream = static_cast<cudaStream_t>(d->stream);
    } else {
        if (cudaStreamCreateWithFlags(&w->stream, cudaStreamNonBlocking) != cudaSuccess) {
            free_ws(w);
            return tomo_set_error(TOMO_ECUDA, "stream creation failed");
        }
        w->own_stream = true;
    }
    int64_t o = 0;
    w->oW1 = o; o += s.C1 * s.C0 * s.K;
    w->ob1 = o; o += s.C1;
    w->oW2 = o; o += s.C2 * s.C1 * s.K;
    w->ob2 = o; o += s.C2;
    w->oW3 = o; o += s.H * s.F();
    w->ob3 = o; o += s.H;
    w->oW4 = o; o += s.M * s.C0 * s.H;
    w->ob4 = o; o += s.M * s.C0;
    w->nparam = o;
    const int64_t B = w->max_batch;
    cudaError_t e = cudaSuccess;
    auto A = [&](auto **p, int64_t n) { if (e == cudaSuccess) e = ws_alloc(p, n); };
    A(&w->param, o); A(&w->grad, o); A(&w->m, o); A(&w->v, o); A(&w->pbf, o);
    A(&w->X0, B * s.D * s.C0); A(&w->Y1, B * s.T1() * s.C1); A(&w->Y2, B * s.F()); A(&w->Y3, B * s.H);
    A(&w->Z, B * s.M * s.C0); A(&w->T, B * s.M * s.C0); A(&w->dZ, B * s.M * s.C0); A(&w->dY3, B * s.H);
    A(&w->dY2, B * s.F()); A(&w->dA1, B * s.T1() * s.C1); A(&w->rowloss, B * s.M); A(&w->loss, 1);
    A(&w->ncols, B);
    if (e != cudaSuccess) {
        free_ws(w);
        return tomo_set_error(TOMO_ENOMEM, cudaGetErrorString(e));
    }
    // He-uniform weights (scaled down for the output layer so that Theta0
    // starts near uniform rows), zero biases
    std::vector<float> h(size_t(o), 0.f);
    uint64_t st = d->seed;
    auto fill = [&](int64_t off, int64_t n, double fan_in, double gain) {
        const double a = gain * std::sqrt(6.0 / fan_in);
        for (int64_t k = 0; k < n; ++k) {
            const double u = double(splitmix64(st) >> 11) * (1.0 / 9007199254740992.0);
            h[size_t(off + k)] = float((2.0 * u - 1.0) * a);
        }
    };
    fill(w->oW1, s.C1 * s.C0 * s.K, double(s.C0 * s.K), 1.0);
    fill(w->oW2, s.C2 * s.C1 * s.K, double(s.C1 * s.K), 1.0);
    fill(w->oW3, s.H * s.F(), double(s.F()), 1.0);
    fill(w->oW4, s.M * s.C0 * s.H, double(s.H), 0.1);
    // on the handle's stream (possibly non-blocking), finished before return
    if ((e = cudaMemcpyAsync(w->param, h.data(), sizeof(float) * size_t(o), cudaMemcpyHostToDevice,
                             w->stream)) != cudaSuccess ||
        (e = cudaMemsetAsync(w->m, 0, sizeof(float) * size_t(o), w->stream)) != cudaSuccess ||
        (e = cudaMemsetAsync(w->v, 0, sizeof(float) * size_t(o), w->stream)) != cudaSuccess ||
        (e = cudaStreamSynchronize(w->stream)) != cudaSuccess) {
        free_ws(w);
        return tomo_set_error(TOMO_ECUDA, cudaGetErrorString(e));
    }
    w->bf_dirty = true;
    *out = reinterpret_cast<tomo_ws_t>(w);
    return TOMO_OK;
}

void tomo_ws_destroy(tomo_ws_t ws) { tomo::free_ws(reinterpret_cast<WarmStart *>(ws)); }

int64_t tomo_ws_param_count(tomo_ws_t ws)
{
    const WarmStart *w = reinterpret_cast<const WarmStart *>(ws);
    return w ? w->nparam : -1;
}

tomo_status tomo_ws_get_params(tomo_ws_t ws, float *host)
{
    WarmStart *w = reinterpret_cast<WarmStart *>(ws);
    if (!w || !host) return tomo::tomo_set_error(TOMO_EINVAL, "NULL argument");
    cudaError_t e = cudaMemcpyAsync(host, w->param, sizeof(float) * size_t(w->nparam), cudaMemcpyDeviceToHost, w->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(w->stream);
    return e == cudaSuccess ? TOMO_OK : tomo::tomo_set_error(TOMO_ECUDA, cudaGetErrorString(e));
}

tomo_status tomo_ws_set_params(tomo_ws_t ws, const float *host)
{
    WarmStart *w = reinterpret_cast<WarmStart *>(ws);
    if (!w || !host) return tomo::tomo_set_error(TOMO_EINVAL, "NULL argument");
    cudaError_t e = cudaMemcpyAsync(w->param, host, sizeof(float) * size_t(w->nparam), cudaMemcpyHostToDevice, w->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(w->m, 0, sizeof(float) * size_t(w->nparam), w->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(w->v, 0, sizeof(float) * size_t(w->nparam), w->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(w->stream);
    w->step = 0;
    w->bf_dirty = true;
    return e == cudaSuccess ? TOMO_OK : tomo::tomo_set_error(TOMO_ECUDA, cudaGetErrorString(e));
}

static tomo_status ws_load_batch(WarmStart *w, const double *P, const double *T, const int32_t *ncols, int32_t B)
{
    using namespace tomo;
    if (!w || !P || !T || !ncols) return tomo_set_error(TOMO_EINVAL, "NULL argument");
    if (B < 1 || B > w->max_batch) return tomo_set_error(TOMO_EINVAL, "batch size out of range (1..max_batch)");
    for (int32_t b = 0; b < B; ++b)
        if (ncols[b] < 1 || ncols[b] > w->s.C0) return tomo_set_error(TOMO_EINVAL, "ncols out of range (1..C0)");
    const WsShape &s = w->s;
    cudaError_t e = cudaMemcpyAsync(w->ncols, ncols, sizeof(int32_t) * size_t(B), cudaMemcpyHostToDevice, w->stream);
    if (e != cudaSuccess) return tomo_set_error(TOMO_ECUDA, cudaGetErrorString(e));
    k_ws_load<<<grid_for(*w, B * s.D * s.C0), 256, 0, w->stream>>>(B, s.D, s.C0, P, s.C0, w->ncols, w->X0);
    k_ws_load<<<grid_for(*w, B * s.M * s.C0), 256, 0, w->stream>>>(B, s.M, s.C0, T, s.C0, w->ncols, w->T);
    count_launch(2);
    e = cudaGetLastError();
    return e == cudaSuccess ? TOMO_OK : tomo_set_error(TOMO_ECUDA, cudaGetErrorString(e));
}

tomo_status tomo_ws_loss_grad(tomo_ws_t ws, const double *P, const double *T, const int32_t *ncols, int32_t B,
                              float *loss_host, float *grad_host)
{
    using namespace tomo;
    WarmStart *w = reinterpret_cast<WarmStart *>(ws);
    tomo_status st = ws_load_batch(w, P, T, ncols, B);
    if (st != TOMO_OK) return st;
    cudaError_t e = ws_loss_grad(*w, B);
    if (e == cudaSuccess && loss_host)
        e = cudaMemcpyAsync(loss_host, w->loss, sizeof(float), cudaMemcpyDeviceToHost, w->stream);
    if (e == cudaSuccess && grad_host)
        e = cudaMemcpyAsync(grad_host, w->grad, sizeof(float) * size_t(w->nparam), cudaMemcpyDeviceToHost, w->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(w->stream);
    return e == cudaSuccess ? TOMO_OK : tomo_set_error(TOMO_ECUDA, cudaGetErrorString(e));
}

tomo_status tomo_ws_train_step(tomo_ws_t ws, const double *P, const double *T, const int32_t *ncols, int32_t B,
                               float lr, float *loss_host)
{
    using namespace tomo;
    WarmStart *w = reinterpret_cast<WarmStart *>(ws);
    if (!(lr > 0.f) || !std::isfinite(lr)) return tomo_set_error(TOMO_EINVAL, "learning rate must be finite and > 0");
    tomo_status st = ws_load_batch(w, P, T, ncols, B);
    if (st != TOMO_OK) return st;
    cudaError_t e = ws_loss_grad(*w, B);
    if (e != cudaSuccess) return tomo_set_error(TOMO_ECUDA, cudaGetErrorString(e));
    ++w->step;
    const float bc1 = 1.f - std::pow(ADAM_B1, float(w->step));
    const float bc2 = 1.f - std::pow(ADAM_B2, float(w->step));
    k_adam<<<grid_for(*w, w->nparam), 256, 0, w->stream>>>(w->nparam, w->param, w->grad, w->m, w->v, lr, bc1, bc2);
    count_launch();
    w->bf_dirty = true;
    if (loss_host) e = cudaMemcpyAsync(loss_host, w->loss, sizeof(float), cudaMemcpyDeviceToHost, w->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(w->stream);
    return e == cudaSuccess ? TOMO_OK : tomo_set_error(TOMO_ECUDA, cudaGetErrorString(e));
}

tomo_status tomo_ws_infer(tomo_ws_t ws, const double *P, int64_t N, double *Theta0)
{
    using namespace tomo;
    WarmStart *w = reinterpret_cast<WarmStart *>(ws);
    if (!w || !P || !Theta0) return tomo_set_error(TOMO_EINVAL, "NULL argument");
    if (N < 1 || N > w->s.C0) return tomo_set_error(TOMO_EINVAL, "N out of range (1..C0)");
    const WsShape &s = w->s;
    const int32_t nc = int32_t(N);
    cudaError_t e = cudaMemcpyAsync(w->ncols, &nc, sizeof(int32_t), cudaMemcpyHostToDevice, w->stream);
    if (e != cudaSuccess) return tomo_set_error(TOMO_ECUDA, cudaGetErrorString(e));
    if (w->bf_dirty) {
        k_to_bf16<<<grid_for(*w, w->nparam), 256, 0, w->stream>>>(w->nparam, w->param, w->pbf);
        count_launch();
        w->bf_dirty = false;
    }
    k_ws_load<<<grid_for(*w, s.D * s.C0), 256, 0, w->stream>>>(1, s.D, s.C0, P, N, w->ncols, w->X0);
    count_launch();
    e = ws_forward<__nv_bfloat16>(*w, w->pbf, 1);
    if (e != cudaSuccess) return tomo_set_error(TOMO_ECUDA, cudaGetErrorString(e));
    k_softmax_ce<<<grid_for(*w, s.M * 32), 256, 0, w->stream>>>(1, s.M, s.C0, w->ncols, w->Z, nullptr, nullptr,
                                                                0.f, nullptr);
    k_ws_store<<<grid_for(*w, s.M * N), 256, 0, w->stream>>>(s.M, s.C0, N, w->Z, Theta0);
    count_launch(2);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(w->stream);
    return e == cudaSuccess ? TOMO_OK : tomo_set_error(TOMO_ECUDA, cudaGetErrorString(e));
}

}  // extern "C"

// ---- parameter files: "TOMOWS01", the nine shape fields (int64), then the
// parameters (float32, little-endian as in memory)
extern "C" tomo_status tomo_ws_save(tomo_ws_t ws, const char *path)
{
    using namespace tomo;
    WarmStart *w = reinterpret_cast<WarmStart *>(ws);
    if (!w || !path) return tomo_set_error(TOMO_EINVAL, "NULL argument");
    std::vector<float> h(size_t(w->nparam));
    tomo_status st = tomo_ws_get_params(ws, h.data());
    if (st != TOMO_OK) return st;
    FILE *f = std::fopen(path, "wb");
    if (!f) return tomo_set_error(TOMO_EINVAL, "cannot open the parameter file for writing");
    const int64_t hdr[9] = {w->s.D, w->s.C0, w->s.M, w->s.C1, w->s.C2, w->s.K, w->s.S1, w->s.S2, w->s.H};
    bool ok = std::fwrite("TOMOWS01", 1, 8, f) == 8 && std::fwrite(hdr, sizeof(hdr), 1, f) == 1 &&
              std::fwrite(h.data(), sizeof(float), h.size(), f) == h.size();
    ok = (std::fclose(f) == 0) && ok;
    return ok ? TOMO_OK : tomo_set_error(TOMO_EINVAL, "writing the parameter file failed");
}

extern "C" tomo_status tomo_ws_load(tomo_ws_t ws, const char *path)
{
    using namespace tomo;
    WarmStart *w = reinterpret_cast<WarmStart *>(ws);
    if (!w || !path) return tomo_set_error(TOMO_EINVAL, "NULL argument");
    FILE *f = std::fopen(path, "rb");
    if (!f) return tomo_set_error(TOMO_EINVAL, "cannot open the parameter file");
    char magic[8];
    int64_t hdr[9];
    std::vector<float> h(size_t(w->nparam));
    bool ok = std::fread(magic, 1, 8, f) == 8 && std::memcmp(magic, "TOMOWS01", 8) == 0 &&
              std::fread(hdr, sizeof(hdr), 1, f) == 1;
    const int64_t want[9] = {w->s.D, w->s.C0, w->s.M, w->s.C1, w->s.C2, w->s.K, w->s.S1, w->s.S2, w->s.H};
    ok = ok && std::memcmp(hdr, want, sizeof(want)) == 0 &&
         std::fread(h.data(), sizeof(float), h.size(), f) == h.size();
    std::fclose(f);
    if (!ok) return tomo_set_error(TOMO_EINVAL, "parameter file missing, truncated or of another shape");
    return tomo_ws_set_params(ws, h.data());
}
