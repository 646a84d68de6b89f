// tc_band.cu -- the band contractions of the CG Hessian products on the
// 5th-generation tensor cores (tcgen05.mma, kind::f16).
//
//   forward  O = F U   : tile of 128 probes x BN outcomes, reduced over the
//                        union band of the tile's probes (photon numbers);
//   adjoint  Z = F^T O : tile of 128 photon numbers x BN outcomes, reduced
//                        over the probes whose band meets the tile;
//   HVP = 2 F^T (F u) + 2 gamma L u (Table ops, Hessian products).
//
// Operands are bf16: the weights (A) in tensor memory, 128 lanes = tile rows;
// the vector operand (B) in shared memory, K-major, 128-byte swizzled; the
// accumulator is f32 in tensor memory.  Precision is recovered by splitting
// every operand into hi + lo bf16 parts and accumulating hi*hi + hi*lo +
// lo*hi (three MMAs per K step of 16 into one accumulator, ~17 significant
// bits: the dropped lo*lo term is of the order of what the two-part split
// itself leaves, 2^-18).
//
// The contraction kernel is warp-specialised and persistent (one CTA per SM,
// a list of work units each):
//   producer warps 0-15 generate the Poisson weights of every 64-wide slice
//                       straight into a ring of four A stages in tensor
//                       memory (runs of 8 photon numbers from the log-space
//                       anchors, exact ratio recurrence in float; each warp
//                       writes its own lane quarter) and signal them on an
//                       mbarrier;
//   warp 16             issues the slice's MMAs into one of two tensor-memory
//                       accumulators and commits them to the barriers that
//                       free the stages and publish a finished unit;
//   warp 17             loads the vector operand of each slice by TMA from a
//                       transposed bf16 hi/lo copy (rows = outcomes,
//                       contiguous along the reduction index), up to four
//                       slices ahead of the MMAs;
//   warps 18-21         move each finished accumulator to the unit's f32
//                       partial tile (column-major, coalesced stores) while
//                       the MMAs of the next unit run in the other one.
// The reduction range of every tile is cut into work units (split-K, planned
// on the host); a finish kernel sums each tile's partials in unit order and
// runs the epilogue.  Every mbarrier wait is bounded: a role that gives up
// raises a CTA-wide abort flag, the others leave their loops, copies and MMAs
// in flight are drained (bounded) and the host sees TOMO_ETIMEOUT.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "tc_ptx.cuh"
#include "tomo_device.cuh"
#include "tomo_internal.cuh"

namespace tomo {

constexpr int TC_BK = 64;            // reduction slice per stage (one 128-byte bf16 row)
constexpr int TC_SA = 4;             // A (weight) stages, in tensor memory
constexpr int TC_SB = 4;             // B (vector) stages, filled by TMA
constexpr int TC_PROD = 512;         // producer threads (warps 0-15)
constexpr int TC_PW = TC_PROD / 32;  // producer warps
constexpr int TC_MMA_WARP = 16;      // MMA issue
constexpr int TC_TMA_WARP = 17;      // TMA of the vector operand
constexpr int TC_THREADS = 22 * 32;  // + epilogue warps 18-21
constexpr uint32_t TC_WAIT_LIMIT = 1u << 24;
constexpr int TC_WIN = 4;            // windows of the per-slice tables (filled three slices ahead)
static_assert(TC_SA == TC_SB, "one commit frees a slice's A and B stage");

template <int BN>
struct TcLayout {
    // shared memory: the B stages (TMA, 128-byte swizzle), the 8 x 8
    // transposes of the adjoint's producers, the per-slice tables, barriers
    static constexpr int B_BYTES = BN * TC_BK * 2;
    static constexpr int B_STAGE = 2 * B_BYTES;                      // hi + lo
    static constexpr int B_OFF = 0;
    static constexpr int STG_OFF = B_OFF + TC_SB * B_STAGE;
    static constexpr int STAGING_BYTES = 2 * (TC_PROD / 8) * 8 * 9 * 4;  // 8x8 transposes of both runs (+pad)
    static constexpr int TAB_OFF = STG_OFF + STAGING_BYTES;          // per-slice tables
    // per producer warp: TC_WIN windows of 16 table entries (the forward's
    // ratio pairs, 8 bytes, and the adjoint's probe metadata, 24 bytes) and
    // the adjoint's 32 ratio pairs of its rows
    static constexpr int TAB_R_OFF = 0;
    static constexpr int TAB_M_OFF = TAB_R_OFF + TC_PW * TC_WIN * 16 * 8;
    static constexpr int TAB_T_OFF = TAB_M_OFF + TC_PW * TC_WIN * 16 * 24;
    static constexpr int TAB_BYTES = TAB_T_OFF + TC_PW * 32 * 8;
    // forward: per producer warp, three windows of its lanes' anchors (two
    // runs each), filled two slices ahead
    static constexpr int ANC_OFF = TAB_OFF + TAB_BYTES;
    static constexpr int ANC_BYTES = TC_PW * 3 * 2 * 32 * 4;
    static constexpr int BAR_OFF = ANC_OFF + ANC_BYTES;
    static constexpr int NBARS = 2 * TC_SA + TC_SB + 4;              // a_full, a_empty, b_full, acc_full[2], acc_empty[2]
    static constexpr int CTRL_BYTES = NBARS * 8 + 16;                // + tensor-memory holder, abort flag
    // at least 117 KB, so that two CTAs never share an SM (and its tensor
    // memory, of which one CTA takes up to all 512 columns)
    static constexpr int USED = 1024 + BAR_OFF + CTRL_BYTES;
    static constexpr int TOTAL = USED > 117 * 1024 ? USED : 117 * 1024;
    // tensor memory: two accumulators of BN columns, then the A stages (hi
    // and lo parts of 128 rows x 64 bf16, 32 columns each)
    static constexpr int ACC_COLS = BN;
    static constexpr int A_COL = 2 * ACC_COLS;
    static constexpr int A_PART_COLS = TC_BK / 2;
    static constexpr int A_STAGE_COLS = 2 * A_PART_COLS;
    static constexpr int TMEM_NEED = A_COL + TC_SA * A_STAGE_COLS;
    static constexpr int TMEM_COLS = TMEM_NEED <= 256 ? 256 : 512;   // a power of two
    static_assert(BN >= 32 && TMEM_NEED <= 512, "tensor memory");
    static_assert(TOTAL <= 227 * 1024, "shared memory per CTA");
    static_assert(B_OFF % 1024 == 0 && B_STAGE % 1024 == 0 && B_BYTES % 1024 == 0, "swizzle atoms");
};

struct TcArgs {
    // operand B: tensor maps of the transposed bf16 hi/lo copies (rows =
    // outcomes, pitch bpitch, box 64 x BN, 128-byte swizzle)
    CUtensorMap tm_b_hi, tm_b_lo;
    int64_t M, N, D;
    const float2 *lam2;
    const int32_t *lo, *hi;
    const int64_t *aoff;
    const float *anchor;
    const float2 *rinv2;
    const WorkUnit *units;
    const int32_t *cta_first;     // units of CTA c: cta_first[c] .. cta_first[c+1]-1
    const int32_t *tile_first;
    const int32_t *tile_nsplit;
    float *part;
    const int32_t *gate;
    int32_t *err;                 // set to 1 if a bounded wait gave up
    const __nv_bfloat16 *b_hi, *b_lo;
    int64_t bpitch;
    // forward output: transposed bf16 hi/lo copy of O (pitch opitch)
    __nv_bfloat16 *o_hi, *o_lo;
    int64_t opitch;
    // adjoint output: q = 2 Z + 2 gamma L u (M x N), in float when vec_f32
    // (the CG vectors of the tensor-core form), else in double
    void *q;
    const void *u;
    int vec_f32;
    double gamma;
    // CG restriction fused into the adjoint finish (float vectors, one
    // column block, N % 4 == 0): q <- q - q_{i,m(i)} (stage 2) on the free
    // variables, 0 elsewhere, and p^T q, reduced over the finish CTAs in a
    // fixed order; the last CTA sets alpha = rz / pq (or stops the CG on
    // non-positive curvature)
    int restrict_stage;           // 0: off, 1 or 2: the CG stage
    const uint8_t *freem;
    const int32_t *mrow;
    const float *pvec;
    double *red_part;             // grid-reduction partials (one per finish CTA)
    int64_t red_stride;
    DevScalars *sc;
    // bound of every mbarrier wait (polls); the wait self-test withholds the
    // MMAs (skip_mma) so that every wait runs to this bound and gives up
    uint32_t wait_limit;
    int skip_mma;
};

struct ProbeMeta {
    int32_t lo, hi;     // band (lo > hi: empty)
    int64_t aoff;       // first anchor of the probe
    float2 lam;         // lambda as float hi + lo
};

__device__ __forceinline__ ProbeMeta load_meta(const TcArgs &a, int64_t d)
{
    ProbeMeta m;
    if (d < a.D) {
        m.lo = __ldg(&a.lo[d]);
        m.hi = __ldg(&a.hi[d]);
        m.aoff = __ldg(&a.aoff[d]);
        m.lam = __ldg(&a.lam2[d]);
    } else {
        m.lo = 1;
        m.hi = 0;
        m.aoff = 0;
        m.lam = make_float2(0.f, 0.f);
    }
    return m;
}

// Anchor of the run i_r.. of a probe, or 0 when the run misses the band.
__device__ __forceinline__ float anchor_of(const float *anchor, const ProbeMeta &m, int64_t i_r)
{
    if (i_r + RUN - 1 < m.lo || i_r > m.hi) return 0.f;
    const int64_t a0 = int64_t(m.lo) & ~int64_t(RUN - 1);
    return __ldg(&anchor[m.aoff + (i_r - a0) / RUN]);
}

// The run of 8 photon numbers i_r.. of a probe expanded from its anchor v
// (F at photon number i_r) with the exact ratio F_{i+1}/F_i = lambda / (i+1):
// lambda and rs[t] = 1/(i_r + t + 1) are compensated float pairs (hi + lo;
// the table is 16-byte aligned shared memory), so every ratio is the float
// rounding of the exact one and a run carries at most 8 roundings -- the
// same weights, bit for bit, in the forward and the adjoint contraction, and
// within float rounding of the SIMT contractions that give the gradient.
// Weights outside the band [lo, hi] are zero (checked per element only for
// runs that cross a band edge).
__device__ __forceinline__ void tc_expand_run(float v, float2 lam, int32_t lo, int32_t hi, int32_t i_r,
                                              const float2 *rs, float (&v8)[RUN])
{
    float q[RUN - 1];
#pragma unroll
    for (int t = 0; t < RUN - 1; t += 2) {
        const float4 r = *reinterpret_cast<const float4 *>(rs + t);      // pairs t, t + 1
        q[t] = fmaf(lam.x, r.x, fmaf(lam.x, r.y, lam.y * r.x));
        if (t + 1 < RUN - 1) q[t + 1] = fmaf(lam.x, r.z, fmaf(lam.x, r.w, lam.y * r.z));
    }
    v8[0] = v;
#pragma unroll
    for (int t = 1; t < RUN; ++t) v8[t] = v8[t - 1] * q[t - 1];
    if (i_r < lo || i_r + RUN - 1 > hi) {
#pragma unroll
        for (int t = 0; t < RUN; ++t)
            if (i_r + t < lo || i_r + t > hi) v8[t] = 0.f;
    }
}

// Packs 8 floats into hi and lo bf16 chunks (hi = rn(v), lo = rn(v - hi)),
// two values per conversion instruction.
__device__ __forceinline__ void split_pack(const float (&v)[8], uint4 &hi, uint4 &lo)
{
    uint32_t h[4], l[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const __nv_bfloat162 h2 = __floats2bfloat162_rn(v[2 * k], v[2 * k + 1]);
        const float2 hf = __bfloat1622float2(h2);
        const __nv_bfloat162 l2 = __floats2bfloat162_rn(v[2 * k] - hf.x, v[2 * k + 1] - hf.y);
        h[k] = *reinterpret_cast<const uint32_t *>(&h2);
        l[k] = *reinterpret_cast<const uint32_t *>(&l2);
    }
    hi = make_uint4(h[0], h[1], h[2], h[3]);
    lo = make_uint4(l[0], l[1], l[2], l[3]);
}

// A bounded wait observed by a whole warp: every lane polls, the warp gives
// up if any lane did (so the warp's control flow stays uniform).
__device__ __forceinline__ bool warp_wait(uint64_t *bar, uint32_t parity, uint32_t limit, const volatile int *abort)
{
    const bool ok = tc::mbar_wait_or_abort(bar, parity, limit, abort);
    return __all_sync(0xffffffffu, ok);
}

template <int BN, bool FWD>
__global__ void __launch_bounds__(TC_THREADS, 1) k_band_tc(const __grid_constant__ TcArgs a)
{
    using L = TcLayout<BN>;
    if (a.gate && *a.gate == 0) return;

    extern __shared__ unsigned char tc_raw[];
    const uint32_t raw_u32 = tc::smem_u32(tc_raw);
    unsigned char *sm = tc_raw + (((raw_u32 + 1023u) & ~1023u) - raw_u32);
    float *staging = reinterpret_cast<float *>(sm + L::STG_OFF);
    uint64_t *bars = reinterpret_cast<uint64_t *>(sm + L::BAR_OFF);
    uint64_t *a_full = bars, *a_empty = bars + TC_SA, *b_full = bars + 2 * TC_SA;
    uint64_t *acc_full = bars + 2 * TC_SA + TC_SB, *acc_empty = acc_full + 2;
    uint32_t *tmem_holder = reinterpret_cast<uint32_t *>(bars + L::NBARS);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_holder + 1);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (warp == 0) {
        tc::tmem_alloc(tmem_holder, L::TMEM_COLS);
        tc::tmem_relinquish();
    }
    if (tid == TC_MMA_WARP * 32) {
        for (int s = 0; s < TC_SA; ++s) {
            tc::mbar_init(&a_full[s], TC_PROD / 32);   // one arrival per producer warp
            tc::mbar_init(&a_empty[s], 1);             // MMA commit
        }
        for (int s = 0; s < TC_SB; ++s) tc::mbar_init(&b_full[s], 1);   // expect_tx arrival
        for (int s = 0; s < 2; ++s) {
            tc::mbar_init(&acc_full[s], 1);            // MMA commit
            tc::mbar_init(&acc_empty[s], 4);           // one arrival per epilogue warp
        }
        *abort_flag = 0;
        tc::mbar_fence_init();
        tc::tma_prefetch_desc(&a.tm_b_hi);
        tc::tma_prefetch_desc(&a.tm_b_lo);
    }
    tc::tc_fence_before_sync();
    __syncthreads();
    tc::tc_fence_after_sync();
    const uint32_t tmem = *tmem_holder;
    const int64_t n0 = int64_t(blockIdx.y) * BN;
    const int u_begin = a.cta_first[blockIdx.x], u_end = a.cta_first[blockIdx.x + 1];
    const uint32_t limit = a.wait_limit;

    if (warp < TC_MMA_WARP) {
        // ------------------------------------------------------------ producers
        // Every producer warp keeps its own tables in shared memory, so the
        // warps never wait for one another: windows of the 16 entries its two
        // runs per thread need (the forward's ratio pairs 1/(i+1) of its two
        // chunks of photon numbers, the adjoint's metadata of its 16 probes),
        // filled three slices ahead by lanes 0-15 with asynchronous copies,
        // and for the adjoint the ratio pairs of its 32 rows, per unit.  A
        // copy group is committed every slice; waiting for all but the latest
        // (then __syncwarp) publishes the tables of the next slice.  A warp
        // that gives up raises the abort flag; the others meet it in their
        // own bounded waits.
        constexpr int QRUNS = (TILE_R * TC_BK / RUN) / TC_PROD;       // 2 runs of 8 per thread
        static_assert(QRUNS * TC_PROD == TILE_R * TC_BK / RUN, "runs per producer");
        static_assert(QRUNS * 8 == 16, "16 table entries per producer warp");
        float *stg = staging + ((tid >> 3) * 8) * 9;
        float2 (*win_r)[16] = reinterpret_cast<float2 (*)[16]>(sm + L::TAB_OFF + L::TAB_R_OFF) + warp * TC_WIN;
        ProbeMeta (*win_m)[16] = reinterpret_cast<ProbeMeta (*)[16]>(sm + L::TAB_OFF + L::TAB_M_OFF) + warp * TC_WIN;
        float2 *rtile = reinterpret_cast<float2 *>(sm + L::TAB_OFF + L::TAB_T_OFF) + warp * 32;
        const ProbeMeta none{1, 0, 0, make_float2(0.f, 0.f)};
        // this thread's runs: row 32 (warp mod 4) + lane of the tile, and
        // reduction chunks (8 photon numbers, forward; 8 probes, adjoint)
        // warp / 4 + 4 q; table entry q * 8 + (lane mod 8) of a window
        const int row = 32 * (warp & 3) + lane;
        const int t8 = lane & 7;
        float (*wanc)[QRUNS][32] = reinterpret_cast<float (*)[QRUNS][32]>(sm + L::ANC_OFF) + warp * 3;
        static_assert(QRUNS == 2, "anchor windows hold two runs per lane");
        uint32_t g = 0;
        bool ok = true;
        for (int ui = u_begin; ui < u_end && ok; ++ui) {
            const WorkUnit wu = a.units[ui];
            const int nsteps = (wu.k1 - wu.k0) / TC_BK;
            if (nsteps == 0) continue;
            const int64_t r0 = int64_t(wu.tile) * TILE_R;
            // forward: every thread expands runs of one probe (its row)
            const ProbeMeta my = FWD ? load_meta(a, r0 + row) : none;
            // entry `lane` (< 16) of this warp's table of slice j, synchronously
            // or by asynchronous copies (entries outside the range are written
            // directly; the slot belongs to this lane alone)
            auto put_tab = [&](int j, bool async) {
                const int64_t k0j = int64_t(wu.k0) + int64_t(j) * TC_BK;
                const int c = (warp >> 2) + 4 * (lane >> 3);
                if (FWD) {
                    float2 *dst = &win_r[j % TC_WIN][lane];
                    const int64_t idx = k0j + c * RUN + t8 + 1;
                    if (idx > a.M + RUN) *dst = make_float2(0.f, 0.f);
                    else if (async) tc::cp_async<8>(dst, &a.rinv2[idx]);
                    else *dst = __ldg(&a.rinv2[idx]);
                } else {
                    ProbeMeta *dst = &win_m[j % TC_WIN][lane];
                    const int64_t d = k0j + c * 8 + t8;
                    if (d >= wu.k1 || d >= a.D) {
                        *dst = none;
                    } else if (async) {
                        tc::cp_async<4>(&dst->lo, &a.lo[d]);
                        tc::cp_async<4>(&dst->hi, &a.hi[d]);
                        tc::cp_async<8>(&dst->aoff, &a.aoff[d]);
                        tc::cp_async<8>(&dst->lam, &a.lam2[d]);
                    } else {
                        *dst = load_meta(a, d);
                    }
                }
            };
            // forward: the anchors of this lane's runs of slice j into window
            // j % 3, by asynchronous copies or directly (a run that misses the
            // band has weight 0: its slot is written directly)
            auto put_anchors_fwd = [&](int j, bool async) {
                const int64_t k0j = int64_t(wu.k0) + int64_t(j) * TC_BK;
                const int64_t a0 = int64_t(my.lo) & ~int64_t(RUN - 1);
#pragma unroll
                for (int q = 0; q < QRUNS; ++q) {
                    const int64_t i_r = k0j + int64_t((warp >> 2) + 4 * q) * RUN;
                    float *dst = &wanc[j % 3][q][lane];
                    if (i_r + RUN - 1 < my.lo || i_r > my.hi) {
                        *dst = 0.f;
                    } else {
                        const float *src = &a.anchor[my.aoff + (i_r - a0) / RUN];
                        if (async) tc::cp_async<4>(dst, src);
                        else *dst = __ldg(src);
                    }
                }
            };
            // adjoint: the anchors of every run of slice j, one slice ahead in
            // registers (tables of slice j in place)
            float anc[QRUNS];
            auto fetch_anchors = [&](int j) {
                const int64_t k0j = int64_t(wu.k0) + int64_t(j) * TC_BK;
#pragma unroll
                for (int q = 0; q < QRUNS; ++q) {
                    const int c = (warp >> 2) + 4 * q;
                    if (FWD) anc[q] = anchor_of(a.anchor, my, k0j + int64_t(c) * RUN);
                    else anc[q] = anchor_of(a.anchor, win_m[j % TC_WIN][q * 8 + t8], r0 + (row & ~7));
                }
            };
            {   // prologue of the unit: this warp's tables of slices 0 to 2 and
                // the adjoint's ratios of its rows (the warp is done with the
                // previous unit's tables)
                __syncwarp();
                if (lane < 16)
                    for (int j = 0; j < 3 && j < nsteps; ++j) put_tab(j, false);
                if (!FWD) {
                    const int64_t idx = r0 + row + 1;
                    rtile[lane] = idx <= a.M + RUN ? __ldg(&a.rinv2[idx]) : make_float2(0.f, 0.f);
                }
                if (FWD) {
                    put_anchors_fwd(0, false);
                    if (nsteps > 1) put_anchors_fwd(1, false);
                }
                __syncwarp();
                if (!FWD) fetch_anchors(0);
            }
            for (int s = 0; s < nsteps; ++s, ++g) {
                const int st = int(g % TC_SA);
                bool wok = true;
                if (g >= TC_SA) wok = warp_wait(&a_empty[st], ((g / TC_SA) - 1) & 1u, limit, abort_flag);
                if (!wok) {
                    *abort_flag = 1;
                    ok = false;
                    break;
                }
                // the copies issued at slice s - 2 have landed: the warp's
                // tables of slice s + 1 and (forward) this lane's anchors of
                // slice s; the warp is past slice s - 1, so its windows may
                // take slice s + 3 (tables) and s + 2 (anchors).  One copy
                // group per slice and thread.
                tc::cp_async_wait<1>();
                __syncwarp();
                if (lane < 16 && s + 3 < nsteps) put_tab(s + 3, true);
                if (FWD && s + 2 < nsteps) put_anchors_fwd(s + 2, true);
                tc::cp_async_commit();
                // this warp's lane quarter of the stage's hi part (lo: + 32 columns)
                const uint32_t a_hi = tmem + (uint32_t(32 * (warp & 3)) << 16) +
                                      uint32_t(L::A_COL + st * L::A_STAGE_COLS);
                // the MMAs that read this stage before are complete (a_empty)
                tc::tc_fence_after_sync();
                const int64_t k0 = int64_t(wu.k0) + int64_t(s) * TC_BK;
                const int w = s % TC_WIN;
                float ac[QRUNS];
                if (FWD) {
#pragma unroll
                    for (int q = 0; q < QRUNS; ++q) ac[q] = wanc[s % 3][q][lane];
                } else {
#pragma unroll
                    for (int q = 0; q < QRUNS; ++q) ac[q] = anc[q];
                    if (s + 1 < nsteps) fetch_anchors(s + 1);
                }
                // both runs of the thread: weights, the adjoint's transposes,
                // the hi/lo split, then the tensor-memory stores (independent
                // work interleaved, one warp synchronisation per step)
                static_assert(QRUNS == 2, "two runs per producer thread");
                float v8[QRUNS][RUN];
                int chunk[QRUNS];
#pragma unroll
                for (int q = 0; q < QRUNS; ++q) {
                    const int run = tid + q * TC_PROD;
                    if (FWD) {
                        // row = probe r0 + run % 128 (= 32 (warp mod 4) + lane),
                        // chunk = photon numbers k0 + 8 chunk .. + 7
                        chunk[q] = run / TILE_R;
                        tc_expand_run(ac[q], my.lam, my.lo, my.hi, int32_t(k0) + chunk[q] * RUN,
                                      &win_r[w][q * 8], v8[q]);
                    } else {
                        // 8 x 8 block (8 probes x 8 photon numbers) per group of 8
                        // lanes: lane t expands probe kb 8 + t over the photon
                        // numbers pb 8 .. + 7
                        const int g8 = run >> 3, t = run & 7;
                        const int pb = g8 % (TILE_R / 8), kb = g8 / (TILE_R / 8);
                        chunk[q] = kb;
                        const ProbeMeta &m = win_m[w][q * 8 + t];
                        float w8[RUN];
                        tc_expand_run(ac[q], m.lam, m.lo, m.hi, int32_t(r0) + pb * 8,
                                      &rtile[(pb - 4 * (warp & 3)) * 8], w8);
#pragma unroll
                        for (int j = 0; j < RUN; ++j) stg[q * (TC_PROD * 9) + t * 9 + j] = w8[j];
                    }
                }
                if (!FWD) {
                    // transposed through shared memory: lane t then holds the 8
                    // probes kb 8 .. + 7 of photon number pb 8 + t (its row)
                    __syncwarp();
                    const int t = tid & 7;
#pragma unroll
                    for (int q = 0; q < QRUNS; ++q)
#pragma unroll
                        for (int j = 0; j < RUN; ++j) v8[q][j] = stg[q * (TC_PROD * 9) + j * 9 + t];
                    __syncwarp();
                }
                uint4 hi[QRUNS], lo[QRUNS];
#pragma unroll
                for (int q = 0; q < QRUNS; ++q) split_pack(v8[q], hi[q], lo[q]);
                // the warp's own lane quarter; 8 bf16 of a chunk = 4 columns
                __syncwarp();
#pragma unroll
                for (int q = 0; q < QRUNS; ++q) {
                    tc::tmem_st_32x32b_x4(a_hi + uint32_t(chunk[q] * 4), hi[q]);
                    tc::tmem_st_32x32b_x4(a_hi + uint32_t(L::A_PART_COLS + chunk[q] * 4), lo[q]);
                }
                // the stores are complete before the MMA thread learns of them
                tc::tmem_wait_st();
                tc::tc_fence_before_sync();
                __syncwarp();
                if (lane == 0) tc::mbar_arrive(&a_full[st]);
            }
            // no copy may still be in flight into a window the next unit's
            // prologue rewrites
            tc::cp_async_wait<0>();
        }
        tc::cp_async_wait<0>();
    } else if (warp == TC_MMA_WARP) {
        // --------------------------------------------------- MMA issue (lane 0)
        if (lane == 0) {
            // hi*hi + hi*lo + lo*hi for each of the slice's four K steps of
            // 16, A from tensor memory (8 columns per step), B from shared
            // memory.  The B stages sit at a fixed stride, so a stage's
            // descriptor is the first stage's plus a multiple of the stride
            // (start-address field in 16-byte units; every shared-memory
            // address is below 2^18 bytes, so the field never carries).
            constexpr uint32_t IDESC = tc::idesc_bf16_f32(TILE_R, BN);
            const uint64_t db0 = tc::desc_kmajor_sw128(tc::smem_u32(sm + L::B_OFF));
            uint32_t g = 0, au = 0;
            int64_t last_commit = -1;
            bool ok = true;
            for (int ui = u_begin; ui < u_end && ok; ++ui) {
                const WorkUnit wu = a.units[ui];
                const int nsteps = (wu.k1 - wu.k0) / TC_BK;
                if (nsteps == 0) continue;
                const int acc = int(au & 1u);
                if (au >= 2 && !tc::mbar_wait_or_abort(&acc_empty[acc], ((au >> 1) - 1) & 1u, limit, abort_flag)) {
                    ok = false;
                    break;
                }
                tc::tc_fence_after_sync();
                const uint32_t d_tmem = tmem + uint32_t(acc * L::ACC_COLS);
                for (int s = 0; s < nsteps; ++s, ++g) {
                    const int st = int(g % TC_SA);
                    if (!tc::mbar_wait_or_abort(&b_full[st], (g / TC_SB) & 1u, limit, abort_flag)) { ok = false; break; }
                    if (!tc::mbar_wait_or_abort(&a_full[st], (g / TC_SA) & 1u, limit, abort_flag)) { ok = false; break; }
                    tc::tc_fence_after_sync();
                    if (!a.skip_mma) {
                        const uint32_t ah = tmem + uint32_t(L::A_COL + st * L::A_STAGE_COLS);
                        const uint32_t al = ah + uint32_t(L::A_PART_COLS);
                        const uint64_t bh = db0 + uint64_t(st) * uint64_t(L::B_STAGE >> 4);
                        const uint64_t bl = bh + uint64_t(L::B_BYTES >> 4);
#pragma unroll
                        for (int kk = 0; kk < TC_BK / 16; ++kk) {
                            const uint32_t acc0 = (s > 0 || kk > 0) ? 1u : 0u;   // 16 bf16 = 32 B per step
                            tc::mma_bf16_ts(d_tmem, ah + 8 * kk, bh + 2 * kk, IDESC, acc0);
                            tc::mma_bf16_ts(d_tmem, ah + 8 * kk, bl + 2 * kk, IDESC, 1u);
                            tc::mma_bf16_ts(d_tmem, al + 8 * kk, bh + 2 * kk, IDESC, 1u);
                        }
                        // frees the A and the B stage of this slice
                        tc::mma_commit(&a_empty[st]);
                        last_commit = int64_t(g);
                    }
                }
                if (!ok) break;
                if (!a.skip_mma) tc::mma_commit(&acc_full[acc]);
                ++au;
            }
            if (!ok) {
                *abort_flag = 1;
                // the last group of committed MMAs (its completion covers all
                // earlier ones) must be done before tensor memory is freed
                if (last_commit >= 0)
                    tc::mbar_wait_bounded(&a_empty[uint32_t(last_commit) % TC_SA],
                                          (uint32_t(last_commit) / TC_SA) & 1u, limit);
            }
        }
    } else if (warp == TC_TMA_WARP) {
        // ------------------------------------- TMA of the vector operand (lane 0)
        if (lane == 0) {
            // slice j goes to stage j % TC_SB once the MMAs of slice j - TC_SB
            // (same stage) are complete: up to TC_SB slices ahead of the MMAs
            uint32_t j = 0;
            bool ok = true;
            for (int ui = u_begin; ui < u_end && ok; ++ui) {
                const WorkUnit wu = a.units[ui];
                const int nsteps = (wu.k1 - wu.k0) / TC_BK;
                for (int s = 0; s < nsteps; ++s, ++j) {
                    const int bs = int(j % TC_SB);
                    if (j >= uint32_t(TC_SB) &&
                        !tc::mbar_wait_or_abort(&a_empty[bs], ((j / TC_SB) - 1) & 1u, limit, abort_flag)) {
                        ok = false;
                        break;
                    }
                    unsigned char *B_hi = sm + L::B_OFF + bs * L::B_STAGE;
                    const int32_t x = int32_t(int64_t(wu.k0) + int64_t(s) * TC_BK);
                    tc::mbar_arrive_expect_tx(&b_full[bs], 2u * L::B_BYTES);
                    tc::tma_load_2d(B_hi, &a.tm_b_hi, x, int32_t(n0), &b_full[bs]);
                    tc::tma_load_2d(B_hi + L::B_BYTES, &a.tm_b_lo, x, int32_t(n0), &b_full[bs]);
                }
            }
            if (!ok) *abort_flag = 1;
            // nothing may still target this CTA's memory when it exits: wait
            // for the last copy of every stage (no later copy of the stage was
            // issued, so its phase cannot move on)
            for (uint32_t k = j > uint32_t(TC_SB) ? j - TC_SB : 0u; k < j; ++k)
                tc::mbar_wait_bounded(&b_full[k % TC_SB], (k / TC_SB) & 1u, limit);
        }
    } else {
        // ---------------------------------------------------------- epilogue
        const int q = warp & 3;                 // tensor-memory lanes 32 q .. 32 q + 31
        const int ncb = gridDim.y;
        constexpr int TE = TILE_R * BN;
        uint32_t au = 0;
        for (int ui = u_begin; ui < u_end; ++ui) {
            const WorkUnit wu = a.units[ui];
            const int nsteps = (wu.k1 - wu.k0) / TC_BK;
            // partial tile of the unit, column-major: column c at c * 128
            float *dst = a.part + (int64_t(a.tile_first[wu.tile] + wu.chunk) * ncb + blockIdx.y) * TE + 32 * q + lane;
            if (nsteps == 0) {
#pragma unroll 8
                for (int c = 0; c < BN; ++c) dst[c * TILE_R] = 0.f;
                continue;
            }
            const int acc = int(au & 1u);
            if (!warp_wait(&acc_full[acc], (au >> 1) & 1u, limit, abort_flag)) {
                *abort_flag = 1;
                break;
            }
            tc::tc_fence_after_sync();
#pragma unroll 1
            for (int c0 = 0; c0 < BN; c0 += 32) {
                uint32_t r[16], r2[16];
                const uint32_t t = tmem + (uint32_t(32 * q) << 16) + uint32_t(acc * L::ACC_COLS + c0);
                tc::tmem_ld_32x32b_x16(t, r);
                tc::tmem_ld_32x32b_x16(t + 16, r2);
                tc::tmem_wait_ld(r, r2);
#pragma unroll
                for (int k = 0; k < 16; ++k) {
                    dst[(c0 + k) * TILE_R] = __uint_as_float(r[k]);
                    dst[(c0 + 16 + k) * TILE_R] = __uint_as_float(r2[k]);
                }
            }
            tc::tc_fence_before_sync();
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(&acc_empty[acc]);
            ++au;
        }
    }
    tc::tc_fence_before_sync();
    __syncthreads();
    tc::tc_fence_after_sync();
    if (warp == 0) tc::tmem_dealloc(tmem, L::TMEM_COLS);
    if (*abort_flag && tid == 0) atomicExch(a.err, 1);
}


// ----------------------------------------------------------------------------
// Finish of a tensor-core contraction: one CTA per (32-row slice of a tile,
// column block) sums the tile's split-K partials in unit order (loads of the
// next split in flight while the current one is added) and runs the epilogue
// of its slice:
//   forward:  the transposed bf16 hi/lo copies of O = F u (the adjoint's B
//             operand), stored as pairs along the probes;
//   adjoint:  q = 2 Z + 2 gamma L u along rows, with the optional CG
//             restriction and the p^T q grid reduction.
// ----------------------------------------------------------------------------
constexpr int FIN_RB = 32;            // rows per finish CTA
constexpr int FIN_T = 256;

template <int BN, bool FWD>
__global__ void __launch_bounds__(FIN_T) k_tc_finish(TcArgs a)
{
    if (a.gate && *a.gate == 0) return;
    constexpr int LD = BN + 1;
    constexpr int TE = TILE_R * BN;
    constexpr int IE = FIN_RB * BN;
    constexpr int P4 = IE / 4 / FIN_T;
    static_assert(IE % (4 * FIN_T) == 0, "slice divides into float4 per thread");
    __shared__ float zs[FIN_RB * LD];
    __shared__ float qm_s[FIN_RB];
    const int tid = threadIdx.x, lane = tid & 31;
    constexpr int SLICES = TILE_R / FIN_RB;
    const int tile = blockIdx.x / SLICES, rq = blockIdx.x % SLICES;
    const int64_t r0 = int64_t(tile) * TILE_R + int64_t(rq) * FIN_RB;
    const int64_t n0 = int64_t(blockIdx.y) * BN;
    const int ncb = gridDim.y;
    const int nsplit = a.tile_nsplit[tile];
    const int64_t split_stride = int64_t(ncb) * TE;
    // partial tiles are column-major (column c at c * 128): float4 f of the
    // slice holds rows rq * 32 + 4 (f % 8) .. + 3 of column f / 8
    const float4 *base = reinterpret_cast<const float4 *>(
        a.part + (int64_t(a.tile_first[tile]) * ncb + blockIdx.y) * TE) + rq * (FIN_RB / 4);
    auto f4_at = [](int f) { return (f >> 3) * (TILE_R / 4) + (f & 7); };

    float4 acc[P4], cur[P4];
#pragma unroll
    for (int j = 0; j < P4; ++j) {
        acc[j] = make_float4(0.f, 0.f, 0.f, 0.f);
        cur[j] = __ldcg(base + f4_at(tid + j * FIN_T));
    }
    for (int sidx = 0; sidx < nsplit; ++sidx) {
        float4 nxt[P4];
        if (sidx + 1 < nsplit) {
            const float4 *src = base + (sidx + 1) * (split_stride / 4);
#pragma unroll
            for (int j = 0; j < P4; ++j) nxt[j] = __ldcg(src + f4_at(tid + j * FIN_T));
        }
#pragma unroll
        for (int j = 0; j < P4; ++j) {
            acc[j].x += cur[j].x; acc[j].y += cur[j].y; acc[j].z += cur[j].z; acc[j].w += cur[j].w;
        }
        if (sidx + 1 < nsplit) {
#pragma unroll
            for (int j = 0; j < P4; ++j) cur[j] = nxt[j];
        }
    }
#pragma unroll
    for (int j = 0; j < P4; ++j) {
        const int f = tid + j * FIN_T, cc = f >> 3, rr = 4 * (f & 7);
        zs[rr * LD + cc] = acc[j].x;
        zs[(rr + 1) * LD + cc] = acc[j].y;
        zs[(rr + 2) * LD + cc] = acc[j].z;
        zs[(rr + 3) * LD + cc] = acc[j].w;
    }
    __syncthreads();

    if (FWD) {
        for (int e = tid; e < IE / 2; e += FIN_T) {
            const int nl = e / (FIN_RB / 2), rr = (e % (FIN_RB / 2)) * 2;
            const int64_t grow = r0 + rr, n = n0 + nl;
            if (grow >= a.D || n >= a.N) continue;
            const float v0 = zs[rr * LD + nl];
            const float v1 = grow + 1 < a.D ? zs[(rr + 1) * LD + nl] : 0.f;
            const __nv_bfloat162 h = __floats2bfloat162_rn(v0, v1);
            const float2 hf = __bfloat1622float2(h);
            const __nv_bfloat162 l = __floats2bfloat162_rn(v0 - hf.x, v1 - hf.y);
            if (grow + 1 < a.D) {
                *reinterpret_cast<__nv_bfloat162 *>(a.o_hi + n * a.opitch + grow) = h;
                *reinterpret_cast<__nv_bfloat162 *>(a.o_lo + n * a.opitch + grow) = l;
            } else {
                a.o_hi[n * a.opitch + grow] = h.x;
                a.o_lo[n * a.opitch + grow] = l.x;
            }
        }
        return;
    }

    const double g2 = 2.0 * a.gamma;
    const float g2f = float(g2);
    if (a.vec_f32 && (a.N % 4) == 0) {
        const float *u = static_cast<const float *>(a.u);
        float *q = static_cast<float *>(a.q);
        const int rstage = a.restrict_stage;
        if (rstage == 2) {
            if (tid < FIN_RB) {
                const int64_t grow = r0 + tid;
                float qm = 0.f;
                if (grow < a.M) {
                    const int m = a.mrow[grow];
                    float lx = 0.f;
                    if (g2f != 0.f) {
                        const float xc = u[grow * a.N + m];
                        if (grow < a.M - 1) lx += xc - u[(grow + 1) * a.N + m];
                        if (grow > 0) lx += xc - u[(grow - 1) * a.N + m];
                    }
                    qm = fmaf(g2f, lx, 2.f * zs[tid * LD + (m - int(n0))]);
                }
                qm_s[tid] = qm;
            }
            __syncthreads();
        }
        // a thread takes 4 consecutive columns (float4) of FIN_RB / RPI rows;
        // all loads of a pass are issued before any is used
        constexpr int CG = BN / 4;
        constexpr int RPI = FIN_T / CG;
        constexpr int PASSES = FIN_RB / RPI;
        const int cc = (tid % CG) * 4;
        const int64_t n = n0 + cc;
        float pq_acc = 0.f;
        float4 uc[PASSES], ud[PASSES], uu[PASSES], pv[PASSES];
        uchar4 fm[PASSES];
#pragma unroll
        for (int j = 0; j < PASSES; ++j) {
            const int64_t grow = r0 + j * RPI + tid / CG;
            const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
            uc[j] = ud[j] = uu[j] = pv[j] = z4;
            fm[j] = make_uchar4(0, 0, 0, 0);
            if (grow < a.M && n < a.N) {
                if (rstage != 0) {
                    fm[j] = *reinterpret_cast<const uchar4 *>(a.freem + grow * a.N + n);
                    pv[j] = *reinterpret_cast<const float4 *>(a.pvec + grow * a.N + n);
                }
                if (g2f != 0.f) {
                    uc[j] = *reinterpret_cast<const float4 *>(u + grow * a.N + n);
                    if (grow < a.M - 1) ud[j] = *reinterpret_cast<const float4 *>(u + (grow + 1) * a.N + n);
                    if (grow > 0) uu[j] = *reinterpret_cast<const float4 *>(u + (grow - 1) * a.N + n);
                }
            }
        }
#pragma unroll
        for (int j = 0; j < PASSES; ++j) {
            const int rr = j * RPI + tid / CG;
            const int64_t grow = r0 + rr;
            if (grow >= a.M || n >= a.N) continue;
            const bool has_d = grow < a.M - 1, has_u = grow > 0;
            const float *zr = &zs[rr * LD + cc];
            float4 o;
            o.x = fmaf(g2f, (has_d ? uc[j].x - ud[j].x : 0.f) + (has_u ? uc[j].x - uu[j].x : 0.f), 2.f * zr[0]);
            o.y = fmaf(g2f, (has_d ? uc[j].y - ud[j].y : 0.f) + (has_u ? uc[j].y - uu[j].y : 0.f), 2.f * zr[1]);
            o.z = fmaf(g2f, (has_d ? uc[j].z - ud[j].z : 0.f) + (has_u ? uc[j].z - uu[j].z : 0.f), 2.f * zr[2]);
            o.w = fmaf(g2f, (has_d ? uc[j].w - ud[j].w : 0.f) + (has_u ? uc[j].w - uu[j].w : 0.f), 2.f * zr[3]);
            if (rstage != 0) {
                const float qm = rstage == 2 ? qm_s[rr] : 0.f;
                o.x = fm[j].x ? o.x - qm : 0.f;
                o.y = fm[j].y ? o.y - qm : 0.f;
                o.z = fm[j].z ? o.z - qm : 0.f;
                o.w = fm[j].w ? o.w - qm : 0.f;
                pq_acc = fmaf(pv[j].x, o.x, pq_acc);
                pq_acc = fmaf(pv[j].y, o.y, pq_acc);
                pq_acc = fmaf(pv[j].z, o.z, pq_acc);
                pq_acc = fmaf(pv[j].w, o.w, pq_acc);
            }
            *reinterpret_cast<float4 *>(q + grow * a.N + n) = o;
        }
        if (rstage != 0) {
            double v[1] = {double(pq_acc)};
            DevScalars *sc = a.sc;
            grid_reduce<1>(v, a.red_part, a.red_stride, &sc->ticket[0], [sc](const double *t) {
                sc->pq = t[0];
                if (!(t[0] > 0.0)) sc->cg_active = 0;
                else sc->alpha = sc->rz / t[0];
            });
        }
        (void)lane;
        return;
    }
    // double vectors (or N not a multiple of 4): q = 2 Z + 2 gamma L u
    for (int e = tid; e < IE; e += FIN_T) {
        const int rr = e / BN, cc = e % BN;
        const int64_t grow = r0 + rr, n = n0 + cc;
        if (grow >= a.M || n >= a.N) continue;
        const int64_t k = grow * a.N + n;
        const float z = zs[rr * LD + cc];
        if (a.vec_f32) {
            const float *u = static_cast<const float *>(a.u);
            float lx = 0.f;
            if (g2f != 0.f) {
                const float xi = u[k];
                if (grow < a.M - 1) lx += xi - u[k + a.N];
                if (grow > 0) lx += xi - u[k - a.N];
            }
            static_cast<float *>(a.q)[k] = fmaf(g2f, lx, 2.f * z);
        } else {
            const double *u = static_cast<const double *>(a.u);
            double lx = 0.0;
            if (g2 != 0.0) {
                const double xi = u[k];
                if (grow < a.M - 1) lx += xi - u[k + a.N];
                if (grow > 0) lx += xi - u[k - a.N];
            }
            static_cast<double *>(a.q)[k] = 2.0 * double(z) + g2 * lx;
        }
    }
}

// ----------------------------------------------------------------------------
// u (double, M x N row-major) -> transposed bf16 hi/lo copies (rows = outcomes,
// pitch = padded M), through a 32 x 32 shared-memory tile so that both the
// reads and the writes are coalesced.  Gated like the CG kernels.
// ----------------------------------------------------------------------------
template <typename VT>
__global__ void k_transpose_split(const int32_t *gate, int64_t M, int64_t N, const VT *u,
                                  __nv_bfloat16 *t_hi, __nv_bfloat16 *t_lo, int64_t pitch)
{
    if (gate && *gate == 0) return;
    __shared__ VT tile[32][33];
    const int64_t i0 = int64_t(blockIdx.x) * 32, nb = int64_t(blockIdx.y) * 32;
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int64_t i = i0 + r, n = nb + threadIdx.x;
        tile[r][threadIdx.x] = (i < M && n < N) ? u[i * N + n] : VT(0);
    }
    __syncthreads();
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int64_t n = nb + r, i = i0 + threadIdx.x;
        if (n < N && i < M) {
            // hi = bf16(u), lo = bf16(u - hi)
            const VT v = tile[threadIdx.x][r];
            const __nv_bfloat16 h = __float2bfloat16_rn(float(v));
            t_hi[n * pitch + i] = h;
            t_lo[n * pitch + i] = __float2bfloat16_rn(float(v - VT(__bfloat162float(h))));
        }
    }
}

// ----------------------------------------------------------------------------
// CG direction update of the tensor-core form fused with the transposed split
// of the next Hessian product's input: p = z + beta p (float vectors, N <= 128,
// N % 4 == 0); stage 2 also lifts u = E p (column m(i) := -sum of the
// others).  The product input (p in stage 1, u in stage 2) is written as the
// transposed bf16 hi/lo mirror the forward contraction reads.  One CTA per 32
// rows (a warp per row, a float4 per lane), the transposition through a
// padded shared-memory tile.  Gated on the CG flag like the other CG kernels.
// ----------------------------------------------------------------------------
constexpr int UPS_ROWS = 32;

__global__ void __launch_bounds__(256)
k_cg_update_p_split(const int32_t *gate, const double *beta_p, int64_t M, int64_t N, int stage,
                    const int32_t *mrow, const float *z, float *p, float *u,
                    __nv_bfloat16 *t_hi, __nv_bfloat16 *t_lo, int64_t pitch)
{
    if (gate && *gate == 0) return;
    __shared__ float tile[UPS_ROWS][128 + 1];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t i0 = int64_t(blockIdx.x) * UPS_ROWS;
    const float be = float(*beta_p);
    const int nc = int(N / 4);
    for (int rr = warp; rr < UPS_ROWS; rr += 8) {
        const int64_t i = i0 + rr;
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (i < M) {
            if (lane < nc) {
                const float4 zv = reinterpret_cast<const float4 *>(z)[i * nc + lane];
                const float4 pv = reinterpret_cast<const float4 *>(p)[i * nc + lane];
                v.x = fmaf(be, pv.x, zv.x);
                v.y = fmaf(be, pv.y, zv.y);
                v.z = fmaf(be, pv.z, zv.z);
                v.w = fmaf(be, pv.w, zv.w);
                reinterpret_cast<float4 *>(p)[i * nc + lane] = v;
            }
            if (stage == 2) {
                const int m = mrow[i];
                float s = (v.x + v.y) + (v.z + v.w);
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
                const float4 vm = make_float4(__shfl_sync(0xffffffffu, v.x, m >> 2),
                                              __shfl_sync(0xffffffffu, v.y, m >> 2),
                                              __shfl_sync(0xffffffffu, v.z, m >> 2),
                                              __shfl_sync(0xffffffffu, v.w, m >> 2));
                const float pm = (m & 3) == 0 ? vm.x : (m & 3) == 1 ? vm.y : (m & 3) == 2 ? vm.z : vm.w;
                const float lift = -(s - pm);
                if (lane == (m >> 2)) {
                    if ((m & 3) == 0) v.x = lift;
                    else if ((m & 3) == 1) v.y = lift;
                    else if ((m & 3) == 2) v.z = lift;
                    else v.w = lift;
                }
                if (lane < nc) reinterpret_cast<float4 *>(u)[i * nc + lane] = v;
            }
        }
        if (lane < 32) {
            float *t = &tile[rr][4 * lane];
            t[0] = v.x; t[1] = v.y; t[2] = v.z; t[3] = v.w;
        }
    }
    __syncthreads();
    // chunk (n, j): photon numbers i0 + 8 j .. + 7 of outcome n, one 16-byte
    // copy of each part; rows beyond M hold zeros (the mirror's padding)
    for (int c = tid; c < int(N) * (UPS_ROWS / 8); c += 256) {
        const int n = c / (UPS_ROWS / 8), j = c % (UPS_ROWS / 8);
        const int64_t row0 = i0 + 8 * j;
        if (row0 >= M) continue;
        float v8[8];
#pragma unroll
        for (int t = 0; t < 8; ++t) v8[t] = tile[8 * j + t][n];
        uint4 hi, lo;
        split_pack(v8, hi, lo);
        *reinterpret_cast<uint4 *>(t_hi + n * pitch + row0) = hi;
        *reinterpret_cast<uint4 *>(t_lo + n * pitch + row0) = lo;
    }
}

// ----------------------------------------------------------------------------
// launchers
// ----------------------------------------------------------------------------
template <int BN, bool FWD>
static cudaError_t launch_tc_t(Plan &p, const TcArgs &a)
{
    auto kern = k_band_tc<BN, FWD>;
    const int smem = TcLayout<BN>::TOTAL;
    static const cudaError_t cfg =
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (cfg != cudaSuccess) return cfg;
    const Schedule &S = p.sched_tc[FWD ? 0 : 1];
    dim3 grid(unsigned(S.n_ctas), unsigned((p.N + BN - 1) / BN));
    kern<<<grid, TC_THREADS, smem, p.stream>>>(a);
    count_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    // the split-K combination and the epilogue, a 32-row slice per CTA
    dim3 fgrid(unsigned((FWD ? p.fwd_tiles : p.adj_tiles) * (TILE_R / FIN_RB)), unsigned((p.N + BN - 1) / BN));
    k_tc_finish<BN, FWD><<<fgrid, FIN_T, 0, p.stream>>>(a);
    count_launch();
    return cudaGetLastError();
}

template <bool FWD>
static cudaError_t launch_tc(Plan &p, const TcArgs &a)
{
    switch (band_bn(p.N)) {
    case 128: return launch_tc_t<128, FWD>(p, a);
    case 64: return launch_tc_t<64, FWD>(p, a);
    default: return launch_tc_t<32, FWD>(p, a);
    }
}

static TcArgs tc_args(Plan &p, bool fwd, const int32_t *gate)
{
    TcArgs a;
    a.tm_b_hi = fwd ? p.tm_ut_hi : p.tm_ot_hi;
    a.tm_b_lo = fwd ? p.tm_ut_lo : p.tm_ot_lo;
    a.M = p.M; a.N = p.N; a.D = p.D;
    a.lam2 = p.lam_f2; a.lo = p.lo; a.hi = p.hi; a.aoff = p.aoff;
    a.anchor = p.anchor_f; a.rinv2 = p.ratio_inv_f2;
    const Schedule &S = p.sched_tc[fwd ? 0 : 1];
    a.units = S.units; a.cta_first = S.cta_first;
    a.tile_first = S.tile_first; a.tile_nsplit = S.tile_nsplit;
    a.part = reinterpret_cast<float *>(S.part);
    a.gate = gate;
    a.err = &p.sc->tc_err;
    a.b_hi = fwd ? p.ut_hi : p.ot_hi;
    a.b_lo = fwd ? p.ut_lo : p.ot_lo;
    a.bpitch = fwd ? p.ut_pitch : p.ot_pitch;
    a.o_hi = p.ot_hi; a.o_lo = p.ot_lo; a.opitch = p.ot_pitch;
    a.q = nullptr; a.u = nullptr; a.vec_f32 = 0;
    a.gamma = p.gamma;
    a.restrict_stage = 0;
    a.freem = p.freem; a.mrow = p.mrow; a.pvec = reinterpret_cast<const float *>(p.p);
    a.red_part = p.partials;
    a.red_stride = p.max_partials;
    a.sc = p.sc;
    a.wait_limit = TC_WAIT_LIMIT;
    a.skip_mma = 0;
    return a;
}

// HV = 2 F^T (F V) + 2 gamma L V on the tensor cores (five launches: the
// transposed split copy of V, the forward tile product and its finish, the
// adjoint tile product and its finish with the smoothness term).
bool tc_restrict_fusable(const Plan &p)
{
    return p.cg_f32 && band_bn(p.N) >= p.N && (p.N % 4) == 0;
}

cudaError_t launch_tc_split_input(Plan &p, const void *V, bool vec_f32, bool gated)
{
    const int32_t *gate = gated ? &p.sc->cg_active : nullptr;
    dim3 tb(32, 8), tg(unsigned((p.M + 31) / 32), unsigned((p.N + 31) / 32));
    if (vec_f32)
        k_transpose_split<float><<<tg, tb, 0, p.stream>>>(gate, p.M, p.N, static_cast<const float *>(V),
                                                           p.ut_hi, p.ut_lo, p.ut_pitch);
    else
        k_transpose_split<double><<<tg, tb, 0, p.stream>>>(gate, p.M, p.N, static_cast<const double *>(V),
                                                            p.ut_hi, p.ut_lo, p.ut_pitch);
    count_launch();
    return cudaGetLastError();
}

bool tc_update_p_fusable(const Plan &p)
{
    return tc_restrict_fusable(p) && p.N <= 128;
}

cudaError_t launch_cg_update_p_split(Plan &p, int stage)
{
    float *pf = reinterpret_cast<float *>(p.p), *uf = reinterpret_cast<float *>(p.u);
    k_cg_update_p_split<<<unsigned((p.M + UPS_ROWS - 1) / UPS_ROWS), 256, 0, p.stream>>>(
        &p.sc->cg_active, &p.sc->beta, p.M, p.N, stage, p.mrow, reinterpret_cast<const float *>(p.z), pf, uf,
        p.ut_hi, p.ut_lo, p.ut_pitch);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_hvp_tc(Plan &p, const void *V, void *HV, bool vec_f32, bool gated, int restrict_stage,
                          bool split_input)
{
    const int32_t *gate = gated ? &p.sc->cg_active : nullptr;
    cudaError_t e;
    if (split_input && (e = launch_tc_split_input(p, V, vec_f32, gated)) != cudaSuccess) return e;
    TcArgs f = tc_args(p, true, gate);
    if ((e = launch_tc<true>(p, f)) != cudaSuccess) return e;
    TcArgs b = tc_args(p, false, gate);
    b.q = HV;
    b.u = V;
    b.vec_f32 = vec_f32 ? 1 : 0;
    b.restrict_stage = (vec_f32 && tc_restrict_fusable(p)) ? restrict_stage : 0;
    return launch_tc<false>(p, b);
}

// Self-test of the bounded waits: one Hessian product (double vectors) whose
// MMAs are withheld, so the stage and accumulator barriers never complete;
// with waits bounded at 4096 polls every CTA gives up, raises its abort flag,
// sets the error flag and returns.  Nothing is left in flight (no MMA was
// issued, every TMA copy is waited for), so the context stays usable.
cudaError_t launch_hvp_tc_wait_selftest(Plan &p, const double *V, double *HV)
{
    dim3 tb(32, 8), tg(unsigned((p.M + 31) / 32), unsigned((p.N + 31) / 32));
    k_transpose_split<double><<<tg, tb, 0, p.stream>>>(nullptr, p.M, p.N, V, p.ut_hi, p.ut_lo, p.ut_pitch);
    count_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    TcArgs f = tc_args(p, true, nullptr);
    f.wait_limit = 4096;
    f.skip_mma = 1;
    if ((e = launch_tc<true>(p, f)) != cudaSuccess) return e;
    TcArgs b = tc_args(p, false, nullptr);
    b.q = HV;
    b.u = V;
    b.wait_limit = 4096;
    b.skip_mma = 1;
    return launch_tc<false>(p, b);
}

size_t tc_smem_bytes(int bn)
{
    if (bn == 128) return TcLayout<128>::TOTAL;
    if (bn == 64) return TcLayout<64>::TOTAL;
    return TcLayout<32>::TOTAL;
}

// Tensor map of a transposed bf16 operand copy (rows x pitch elements, pitch
// a multiple of 64): boxes of 64 elements x bn rows with the 128-byte swizzle
// of the MMA operand layout.  The CUDA driver API's encoder is looked up once.
cudaError_t encode_operand_map(CUtensorMap *map, const void *base, int64_t pitch, int64_t rows, int bn)
{
    static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
    if (!encode) {
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
        if (e != cudaSuccess) return e;
        if (q != cudaDriverEntryPointSuccess || !fn) return cudaErrorNotSupported;
        encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    }
    const cuuint64_t dims[2] = {cuuint64_t(pitch), cuuint64_t(rows)};
    const cuuint64_t strides[1] = {cuuint64_t(pitch) * sizeof(__nv_bfloat16)};
    const cuuint32_t box[2] = {cuuint32_t(TC_BK), cuuint32_t(bn)};
    const cuuint32_t estr[2] = {1, 1};
    const CUresult r = encode(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(base), dims, strides, box,
                              estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                              CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

}  // namespace tomo
