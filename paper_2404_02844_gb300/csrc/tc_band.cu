// tc_band.cu -- the band contractions of the CG Hessian products on the
// 5th-generation tensor cores (tcgen05.mma, kind::f16).
//
//   forward  O = F U   : tile of 128 probes x BN outcomes, reduced over the
//                        union band of the tile's probes (photon numbers);
//   adjoint  Z = F^T O : tile of 128 photon numbers x BN outcomes, reduced
//                        over the probes whose band meets the tile;
//   HVP = 2 F^T (F u) + 2 gamma L u (Table ops, Hessian products).
//
// Operands are bf16 in shared memory, K-major, 128-byte swizzled; the
// accumulator is f32 in tensor memory.  Precision is recovered by splitting
// every operand into hi + lo bf16 parts and accumulating hi*hi + hi*lo +
// lo*hi (three MMAs per K slice, ~17 significant bits: the dropped lo*lo
// term is of the order of what the two-part split itself leaves, 2^-18).  The weights F are generated
// by all 256 threads straight into the swizzled A tile (runs of 8 photon
// numbers from the log-space anchors, exact ratio recurrence in float); the
// vector operand comes from a transposed bf16 hi/lo copy (rows = outcomes,
// contiguous along the reduction index) so that one 16-byte load is one
// swizzle chunk.  A single thread issues the MMAs of a stage and commits them
// to the stage's mbarrier while the other threads already produce the next
// stage (two stages).  The reduction range of every tile is cut into work
// units (split-K, planned on the host); every unit writes its f32 partial
// tile and a finish kernel sums each tile's partials in unit order.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "tc_ptx.cuh"
#include "tomo_device.cuh"
#include "tomo_internal.cuh"

namespace tomo {

constexpr int TC_BK = 64;       // reduction slice per stage (one 128-byte bf16 row)
constexpr int TC_STAGES = 2;      // A (weight) stages; the MMA barriers follow them
constexpr int TC_BSTAGES = 3;     // B (vector) stages: B is copied one step ahead
constexpr int TC_THREADS = 256;
constexpr uint32_t TC_WAIT_LIMIT = 1u << 24;

template <int BN, int SPLIT>
struct TcLayout {
    static constexpr int NPART = SPLIT == 3 ? 2 : 1;                 // hi (+ lo)
    static constexpr int A_BYTES = TILE_R * TC_BK * 2;               // 16 KB
    static constexpr int B_BYTES = BN * TC_BK * 2;
    static constexpr int A_STAGE = NPART * A_BYTES;
    static constexpr int B_STAGE = NPART * B_BYTES;
    static constexpr int STAGE_BYTES = TC_STAGES * A_STAGE + TC_BSTAGES * B_STAGE;  // all stages
    static constexpr int STAGING_BYTES = (TC_THREADS / 8) * 8 * 9 * 4;  // 8x8 transposes (+pad)
    static constexpr int CTRL_BYTES = 64;
    // per-unit tables: probe metadata (adjoint) and the 1/(i+1) pairs
    static constexpr int META_BYTES = TC_MAX_UNIT * 24;
    static constexpr int RINV_BYTES = (TC_MAX_UNIT + 2 * RUN + TILE_R) * 8;
    static constexpr int TOTAL = 1024 + STAGE_BYTES + STAGING_BYTES + CTRL_BYTES +
                                 META_BYTES + RINV_BYTES;
    static constexpr int TMEM_COLS = BN < 32 ? 32 : BN;
    static_assert(TOTAL <= 227 * 1024, "shared memory per CTA");
    static_assert(TILE_R * (BN + 1) * 4 + TILE_R * 4 <= STAGE_BYTES, "epilogue tile and row values fit the stage buffers");
};

struct TcArgs {
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
    unsigned int *counters;
    float *part;
    const int32_t *gate;
    int32_t *err;                 // set to 1 if a bounded wait gave up
    // operand B: transposed bf16 hi/lo copy, rows = outcomes, pitch bpitch
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

// Float weights of the run of 8 photon numbers i_r.. of probe d (zero outside
// the band); same recurrence as the float SIMT contraction.
__device__ __forceinline__ void tc_gen_run(const TcArgs &a, int64_t d, int64_t i_r, float (&v8)[RUN])
{
#pragma unroll
    for (int t = 0; t < RUN; ++t) v8[t] = 0.f;
    if (d >= a.D) return;
    const int64_t lo = a.lo[d], hi = a.hi[d];
    if (i_r + RUN - 1 < lo || i_r > hi) return;
    const int64_t a0 = lo & ~int64_t(RUN - 1);
    float v = a.anchor[a.aoff[d] + (i_r - a0) / RUN];
    const float2 lam = a.lam2[d];
#pragma unroll
    for (int t = 0; t < RUN; ++t) {
        const int64_t i = i_r + t;
        v8[t] = (i >= lo && i <= hi) ? v : 0.f;
        const float2 r = a.rinv2[i + 1];
        v = v * fmaf(lam.x, r.x, fmaf(lam.x, r.y, lam.y * r.x));
    }
}

struct ProbeMeta {
    int32_t lo, hi;     // band (lo > hi: empty)
    int64_t aoff;       // first anchor of the probe
    float2 lam;         // lambda as float hi + lo
};

__device__ __forceinline__ ProbeMeta load_meta(const TcArgs &a, int64_t d)
{
    ProbeMeta m;
    if (d < a.D) {
        m.lo = a.lo[d];
        m.hi = a.hi[d];
        m.aoff = a.aoff[d];
        m.lam = a.lam2[d];
    } else {
        m.lo = 1;
        m.hi = 0;
        m.aoff = 0;
        m.lam = make_float2(0.f, 0.f);
    }
    return m;
}

// Same run as tc_gen_run, from the probe's metadata and a shared-memory slice
// of the 1/(i+1) pairs (rs[i - rbase] = 1/(i+1)).
__device__ __forceinline__ void tc_gen_run_tbl(const float *anchor, const ProbeMeta &m, int64_t i_r,
                                               const float2 *rs, int64_t rbase, float (&v8)[RUN])
{
#pragma unroll
    for (int t = 0; t < RUN; ++t) v8[t] = 0.f;
    if (i_r + RUN - 1 < m.lo || i_r > m.hi) return;
    const int64_t a0 = int64_t(m.lo) & ~int64_t(RUN - 1);
    float v = anchor[m.aoff + (i_r - a0) / RUN];
#pragma unroll
    for (int t = 0; t < RUN; ++t) {
        const int64_t i = i_r + t;
        v8[t] = (i >= m.lo && i <= m.hi) ? v : 0.f;
        const float2 r = rs[i - rbase];
        v = v * fmaf(m.lam.x, r.x, fmaf(m.lam.x, r.y, m.lam.y * r.x));
    }
}

// Anchor of the run i_r.. of a probe, or 0 when the run misses the band.
__device__ __forceinline__ float anchor_of(const float *anchor, const ProbeMeta &m, int64_t i_r)
{
    if (i_r + RUN - 1 < m.lo || i_r > m.hi) return 0.f;
    const int64_t a0 = int64_t(m.lo) & ~int64_t(RUN - 1);
    return __ldg(&anchor[m.aoff + (i_r - a0) / RUN]);
}

// The run expanded from an anchor value already in a register.
__device__ __forceinline__ void tc_expand_run(float v, const ProbeMeta &m, int64_t i_r, const float2 *rs,
                                              int64_t rbase, float (&v8)[RUN])
{
#pragma unroll
    for (int t = 0; t < RUN; ++t) {
        const int64_t i = i_r + t;
        v8[t] = (i >= m.lo && i <= m.hi) ? v : 0.f;
        const float2 r = rs[i - rbase];
        v = v * fmaf(m.lam.x, r.x, fmaf(m.lam.x, r.y, m.lam.y * r.x));
    }
}

// 16-byte asynchronous global -> shared copy
__device__ __forceinline__ void cp_async16(void *smem_dst, const void *gsrc)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" :: "r"(tc::smem_u32(smem_dst)), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_commit()
{
    asm volatile("cp.async.commit_group;" ::: "memory");
}
__device__ __forceinline__ void cp_async_wait_group1()
{
    asm volatile("cp.async.wait_group 1;" ::: "memory");
}
__device__ __forceinline__ void cp_async_wait_all()
{
    asm volatile("cp.async.wait_all;" ::: "memory");
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

template <int BN, int SPLIT, bool FWD>
__global__ void __launch_bounds__(TC_THREADS, 1) k_band_tc(TcArgs a)
{
    using L = TcLayout<BN, SPLIT>;
    if (a.gate && *a.gate == 0) return;

    extern __shared__ unsigned char tc_raw[];
    const uint32_t raw_u32 = tc::smem_u32(tc_raw);
    unsigned char *sm = tc_raw + (((raw_u32 + 1023u) & ~1023u) - raw_u32);
    float *staging = reinterpret_cast<float *>(sm + L::STAGE_BYTES);
    uint64_t *bars = reinterpret_cast<uint64_t *>(sm + L::STAGE_BYTES + L::STAGING_BYTES);
    uint32_t *tmem_holder = reinterpret_cast<uint32_t *>(bars + TC_STAGES);
    ProbeMeta *meta_s = reinterpret_cast<ProbeMeta *>(sm + L::STAGE_BYTES + L::STAGING_BYTES +
                                                      L::CTRL_BYTES);
    float2 *rinv_s = reinterpret_cast<float2 *>(reinterpret_cast<unsigned char *>(meta_s) + L::META_BYTES);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (warp == 0) {
        tc::tmem_alloc(tmem_holder, L::TMEM_COLS);
        tc::tmem_relinquish();
    }
    if (tid == 0) {
        for (int s = 0; s < TC_STAGES; ++s) tc::mbar_init(&bars[s], 1);
        tc::mbar_fence_init();
    }
    tc::tc_fence_before_sync();
    __syncthreads();
    tc::tc_fence_after_sync();
    const uint32_t tmem = *tmem_holder;
    const int64_t n0 = int64_t(blockIdx.y) * BN;
    bool ok = true;
    // pipeline steps issued by this CTA so far (stage and mbarrier phase of
    // every step follow from it across units), and the last step whose MMAs
    // were committed (-1: none), known to every thread
    uint32_t gstep = 0;
    int64_t committed = -1;

    // the CTA's units, in order (one wave of persistent CTAs)
    const int u_end = a.cta_first[blockIdx.x + 1];
    for (int ui = a.cta_first[blockIdx.x]; ui < u_end; ++ui) {
    const WorkUnit wu = a.units[ui];
    const int tile = wu.tile;
    const int64_t r0 = int64_t(tile) * TILE_R;

    // unit tables: the 1/(i+1) pairs of every photon number the unit touches
    // (forward: the unit's photon range; adjoint: the tile's photon range)
    // and, for the adjoint, the metadata of the unit's probes
    const int64_t rbase = FWD ? int64_t(wu.k0) : r0;
    const int64_t rcount = FWD ? int64_t(wu.k1 - wu.k0) + 2 * RUN : int64_t(TILE_R) + 2 * RUN;
    for (int64_t k = tid; k < rcount; k += TC_THREADS) {
        const int64_t idx = rbase + k + 1;
        rinv_s[k] = idx < a.M + RUN + 1 ? a.rinv2[idx] : make_float2(0.f, 0.f);
    }
    if (!FWD)
        for (int64_t k = tid; k < int64_t(wu.k1 - wu.k0); k += TC_THREADS) meta_s[k] = load_meta(a, wu.k0 + k);
    // forward: every thread generates the runs of one probe (row tid % 128)
    const ProbeMeta my_meta = FWD ? load_meta(a, r0 + (tid % TILE_R)) : ProbeMeta{1, 0, 0, make_float2(0.f, 0.f)};
    __syncthreads();

    constexpr uint32_t IDESC = tc::idesc_bf16_f32(TILE_R, BN);
    const int nsteps = (wu.k1 - wu.k0) / TC_BK;

    // anchors of a slice: loaded one slice ahead so their latency overlaps the
    // current slice's arithmetic
    constexpr int QRUNS = (TILE_R * TC_BK / RUN) / TC_THREADS;
    auto run_probe = [&](int64_t k0, int q, ProbeMeta &m, int64_t &i_r, int &row, int &chunk) {
        const int run = tid + q * TC_THREADS;
        if (FWD) {
            row = run % TILE_R;
            chunk = run / TILE_R;
            m = my_meta;
            i_r = k0 + int64_t(chunk) * RUN;
        } else {
            const int g = run >> 3, t = run & 7;
            const int pb = g % (TILE_R / 8), kb = g / (TILE_R / 8);
            const int64_t dk = k0 + kb * 8 + t;
            m = (dk < wu.k1) ? meta_s[dk - wu.k0] : ProbeMeta{1, 0, 0, make_float2(0.f, 0.f)};
            i_r = r0 + pb * 8;
            row = pb * 8 + t;
            chunk = kb;
        }
    };
    float anc_next[QRUNS];
    if (nsteps > 0) {
#pragma unroll
        for (int q = 0; q < QRUNS; ++q) {
            ProbeMeta m; int64_t i_r; int row, chunk;
            run_probe(int64_t(wu.k0), q, m, i_r, row, chunk);
            anc_next[q] = anchor_of(a.anchor, m, i_r);
        }
    }

    // operand B of one step: the transposed bf16 copy of the vector, 16-byte
    // asynchronous copies into B stage `bs`, as one copy group
    constexpr int BCH = BN * (TC_BK / 8);          // 16-byte chunks per part
    auto issue_b = [&](int64_t kb0, int bs) {
        unsigned char *B_hi = sm + TC_STAGES * L::A_STAGE + bs * L::B_STAGE;
        unsigned char *B_lo = B_hi + L::B_BYTES;
#pragma unroll
        for (int q = 0; q < (L::NPART * BCH + TC_THREADS - 1) / TC_THREADS; ++q) {
            const int c = tid + q * TC_THREADS;
            if (c < L::NPART * BCH) {
                const int part = c / BCH, cc = c % BCH;
                const int n = cc / (TC_BK / 8), j = cc % (TC_BK / 8);
                const __nv_bfloat16 *src = (part == 0 ? a.b_hi : a.b_lo) + (n0 + n) * a.bpitch + kb0 + j * 8;
                cp_async16((part == 0 ? B_hi : B_lo) + tc::sw128_chunk(n, j), src);
            }
        }
        cp_async_commit();
    };

    for (int s = 0; s < nsteps; ++s) {
        const uint32_t g = gstep + uint32_t(s);
        const int st = int(g % TC_STAGES);            // A stage and MMA barrier
        const int bst = int(g % TC_BSTAGES);          // B stage
        unsigned char *A_hi = sm + st * L::A_STAGE;
        unsigned char *A_lo = A_hi + L::A_BYTES;                        // SPLIT == 3 only
        unsigned char *B_hi = sm + TC_STAGES * L::A_STAGE + bst * L::B_STAGE;
        unsigned char *B_lo = B_hi + L::B_BYTES;                        // SPLIT == 3 only
        if (g >= TC_STAGES) {
            // the MMAs of step g - 2 (maybe of the previous unit) read this A
            // stage and the B stage of step g + 1; their completion also
            // covers every earlier step
            if (!tc::mbar_wait_bounded(&bars[st], ((g / TC_STAGES) - 1) & 1u, a.wait_limit))
                ok = false;
        }
        const int64_t k0 = int64_t(wu.k0) + int64_t(s) * TC_BK;

        // ---- operand B: this step's copy (first step of a unit) and the
        // next step's, so that a copy's latency overlaps a whole step ----
        if (s == 0) issue_b(k0, bst);
        if (s + 1 < nsteps) issue_b(k0 + TC_BK, int((g + 1) % TC_BSTAGES));
        // ---- operand A: Poisson weights ----
        float anc_cur[QRUNS];
#pragma unroll
        for (int q = 0; q < QRUNS; ++q) anc_cur[q] = anc_next[q];
        if (s + 1 < nsteps) {
#pragma unroll
            for (int q = 0; q < QRUNS; ++q) {
                ProbeMeta m; int64_t i_r; int row, chunk;
                run_probe(k0 + TC_BK, q, m, i_r, row, chunk);
                anc_next[q] = anchor_of(a.anchor, m, i_r);
            }
        }
#pragma unroll
        for (int q = 0; q < QRUNS; ++q) {
            ProbeMeta m; int64_t i_r; int row, chunk;
            run_probe(k0, q, m, i_r, row, chunk);
            float v8[RUN];
            if (FWD) {
                // row = probe r0 + r, chunk = photon numbers k0 + 8 j .. + 7
                tc_expand_run(anc_cur[q], m, i_r, rinv_s, rbase, v8);
            } else {
                // 8 x 8 block (8 probes x 8 photon numbers) per group of 8
                // lanes, transposed through shared memory so that one lane
                // holds 8 consecutive probes of one photon number
                const int t = (tid + q * TC_THREADS) & 7;
                float w8[RUN];
                tc_expand_run(anc_cur[q], m, i_r, rinv_s, rbase, w8);
                float *stg = staging + ((tid >> 3) * 8) * 9;
#pragma unroll
                for (int j = 0; j < RUN; ++j) stg[t * 9 + j] = w8[j];
                __syncwarp();
#pragma unroll
                for (int j = 0; j < RUN; ++j) v8[j] = stg[j * 9 + t];
                __syncwarp();
            }
            uint4 hi, lo;
            split_pack(v8, hi, lo);
            *reinterpret_cast<uint4 *>(A_hi + tc::sw128_chunk(row, chunk)) = hi;
            if (SPLIT == 3) *reinterpret_cast<uint4 *>(A_lo + tc::sw128_chunk(row, chunk)) = lo;
        }
        // this step's B copy is complete when at most the next step's group
        // is still in flight
        if (s + 1 < nsteps) cp_async_wait_group1();
        else cp_async_wait_all();
        tc::fence_proxy_async_smem();
        tc::tc_fence_before_sync();
        // a wait that gave up in any thread stops the CTA here, uniformly and
        // before any further MMA is issued (the stages it would overwrite may
        // still be read by MMAs in flight)
        if (__syncthreads_or(ok ? 0 : 1)) {
            ok = false;
            break;
        }
        if (!a.skip_mma) committed = int64_t(g);
        if (tid == 0 && !a.skip_mma) {
            tc::tc_fence_after_sync();
            const uint32_t a_hi = tc::smem_u32(A_hi), a_lo = tc::smem_u32(A_lo);
            const uint32_t b_hi = tc::smem_u32(B_hi), b_lo = tc::smem_u32(B_lo);
#pragma unroll
            for (int kk = 0; kk < TC_BK / 16; ++kk) {
                const uint32_t off = kk * 32;   // 16 bf16 per MMA
                const uint32_t acc0 = (s > 0 || kk > 0) ? 1u : 0u;
                tc::mma_bf16(tmem, tc::desc_kmajor_sw128(a_hi + off), tc::desc_kmajor_sw128(b_hi + off), IDESC, acc0);
                if (SPLIT == 3) {
                    tc::mma_bf16(tmem, tc::desc_kmajor_sw128(a_hi + off), tc::desc_kmajor_sw128(b_lo + off), IDESC, 1u);
                    tc::mma_bf16(tmem, tc::desc_kmajor_sw128(a_lo + off), tc::desc_kmajor_sw128(b_hi + off), IDESC, 1u);
                }
            }
            tc::mma_commit(&bars[st]);
        }
    }
    if (ok && nsteps > 0) {
        const uint32_t g = gstep + uint32_t(nsteps - 1);
        if (!tc::mbar_wait_bounded(&bars[g % TC_STAGES], (g / TC_STAGES) & 1u, a.wait_limit))
            ok = false;
    }
    gstep += uint32_t(nsteps);
    tc::tc_fence_after_sync();
    if (__syncthreads_or(ok ? 0 : 1)) {
        ok = false;
        break;
    }

    // ---- this unit's f32 partial tile (split-K) ----
    // through a shared-memory copy (the stage buffers: every MMA and copy of
    // this unit is complete) so that the global writes run along rows.  The
    // finish kernel sums the partials of every tile in unit order and runs
    // the epilogue, spread over many CTAs.  Warp w reads TMEM lanes
    // 32 (w % 4) .. + 31 (tile rows) and the column half w / 4 (BN >= 64) or
    // all columns (BN == 32, warps 0-3 only).
    const int lg = warp & 3;
    const int row = lg * 32 + lane;
    constexpr int COLS_PER_WARP = BN >= 64 ? BN / 2 : BN;
    const int col0 = BN >= 64 ? (warp >> 2) * COLS_PER_WARP : 0;
    const bool active = BN >= 64 || warp < 4;
    const int ncb = gridDim.y;
    constexpr int LD = BN + 1;                 // padded row: conflict-free both ways
    constexpr int TE = TILE_R * BN;
    float *tile_s = reinterpret_cast<float *>(sm);
    if (active) {
#pragma unroll
        for (int c = 0; c < COLS_PER_WARP; c += 32) {
            uint32_t r[32];
            if (nsteps > 0) {
                tc::tmem_ld_32x32b_x32(tmem + (uint32_t(lg * 32) << 16) + uint32_t(col0 + c), r);
            } else {
#pragma unroll
                for (int k = 0; k < 32; ++k) r[k] = 0u;
            }
#pragma unroll
            for (int k = 0; k < 32; ++k) tile_s[row * LD + col0 + c + k] = __uint_as_float(r[k]);
        }
    }
    __syncthreads();
    {
        float *mine = a.part + (int64_t(a.tile_first[tile] + wu.chunk) * ncb + blockIdx.y) * TE;
        for (int e = tid; e < TE; e += TC_THREADS) mine[e] = tile_s[(e / BN) * LD + (e % BN)];
    }
    // the next unit's first MMA overwrites the accumulator and its tables
    // replace these: every thread is past its tensor-memory loads
    tc::tc_fence_before_sync();
    __syncthreads();
    }  // units
    if (!ok) {
        // the CTA gave up: no copy may still target its shared memory and no
        // committed MMA may still write its tensor memory when it is freed,
        // so wait for the copies and, once more with a bound, for the last
        // committed group of MMAs (their completion covers all earlier ones)
        cp_async_wait_all();
        if (committed >= 0) {
            const uint32_t g = uint32_t(committed);
            tc::mbar_wait_bounded(&bars[g % TC_STAGES], (g / TC_STAGES) & 1u, a.wait_limit);
        }
        tc::tc_fence_after_sync();
        __syncthreads();
    }
    if (warp == 0) tc::tmem_dealloc(tmem, L::TMEM_COLS);
    if (!ok && tid == 0) atomicExch(a.err, 1);
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
    const float4 *base = reinterpret_cast<const float4 *>(
        a.part + (int64_t(a.tile_first[tile]) * ncb + blockIdx.y) * TE + int64_t(rq) * IE);

    float4 acc[P4], cur[P4];
#pragma unroll
    for (int j = 0; j < P4; ++j) {
        acc[j] = make_float4(0.f, 0.f, 0.f, 0.f);
        cur[j] = __ldcg(base + tid + j * FIN_T);
    }
    for (int sidx = 0; sidx < nsplit; ++sidx) {
        float4 nxt[P4];
        if (sidx + 1 < nsplit) {
            const float4 *src = base + (sidx + 1) * (split_stride / 4);
#pragma unroll
            for (int j = 0; j < P4; ++j) nxt[j] = __ldcg(src + tid + j * FIN_T);
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
        const int e = (tid + j * FIN_T) * 4, rr = e / BN, cc = e % BN;
        float *d = &zs[rr * LD + cc];
        d[0] = acc[j].x; d[1] = acc[j].y; d[2] = acc[j].z; d[3] = acc[j].w;
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
template <int BN, int SPLIT, bool FWD>
static cudaError_t launch_tc_t(Plan &p, const TcArgs &a)
{
    auto kern = k_band_tc<BN, SPLIT, FWD>;
    const int smem = TcLayout<BN, SPLIT>::TOTAL;
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
    case 128: return launch_tc_t<128, 3, FWD>(p, a);
    case 64: return launch_tc_t<64, 3, FWD>(p, a);
    default: return launch_tc_t<32, 3, FWD>(p, a);
    }
}

static TcArgs tc_args(Plan &p, bool fwd, const int32_t *gate)
{
    TcArgs a;
    a.M = p.M; a.N = p.N; a.D = p.D;
    a.lam2 = p.lam_f2; a.lo = p.lo; a.hi = p.hi; a.aoff = p.aoff;
    a.anchor = p.anchor_f; a.rinv2 = p.ratio_inv_f2;
    const Schedule &S = p.sched_tc[fwd ? 0 : 1];
    a.units = S.units; a.cta_first = S.cta_first;
    a.tile_first = S.tile_first; a.tile_nsplit = S.tile_nsplit;
    a.counters = S.counters; a.part = reinterpret_cast<float *>(S.part);
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
// MMAs are withheld, so no mbarrier ever completes; with waits bounded at 4096
// polls every CTA gives up after its first unit, sets the error flag and
// returns.  Nothing is left in flight (no MMA was issued, every copy is waited
// for), so the context stays usable; the host re-arms the counters.
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
    if (bn == 128) return TcLayout<128, 3>::TOTAL;
    if (bn == 64) return TcLayout<64, 3>::TOTAL;
    return TcLayout<32, 3>::TOTAL;
}

}  // namespace tomo
