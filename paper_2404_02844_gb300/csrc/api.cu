// api.cu -- host side of libtomo: the C ABI declared in include/tomo.h.
// Plans own every device table and workspace; tomo_fit drives the two-stage
// two-metric projected truncated Newton method of App. B (Algorithm 3:
// Algorithm 2 then Algorithm 1) with all vector work in the kernels of
// band_gemm.cu / rowops.cu and only scalar decisions on the host.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstdarg>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <thread>
#include <utility>
#include <vector>
#include <tuple>
#include <mutex>
#include <map>

#include "tomo_internal.cuh"

namespace tomo {

static std::atomic<int64_t> g_launches{0};
void count_launch(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

static thread_local std::string g_err;

static tomo_status fail(tomo_status s, const char *fmt, ...) __attribute__((format(printf, 2, 3)));
static tomo_status fail(tomo_status s, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_err = buf;
    return s;
}

tomo_status tomo_set_error(tomo_status s, const char *msg)
{
    g_err = msg;
    return s;
}

#define CUDA_TRY(expr)                                                                     \
    do {                                                                                   \
        cudaError_t _e = (expr);                                                           \
        if (_e != cudaSuccess)                                                             \
            return fail(_e == cudaErrorMemoryAllocation ? TOMO_ENOMEM : TOMO_ECUDA,        \
                        "%s failed: %s (%s:%d)", #expr, cudaGetErrorString(_e), __FILE__,  \
                        __LINE__);                                                         \
    } while (0)

#define TOMO_TRY(expr)                      \
    do {                                    \
        tomo_status _s = (expr);            \
        if (_s != TOMO_OK) return _s;       \
    } while (0)

static bool is_device_pointer(const void *ptr)
{
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, ptr) != cudaSuccess) {
        cudaGetLastError();  // clear the sticky-free error of an unknown pointer
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

template <typename T>
static cudaError_t dalloc(T **p, int64_t count)
{
    if (count < 1) count = 1;
    return cudaMalloc(reinterpret_cast<void **>(p), sizeof(T) * size_t(count));
}

static void free_schedule(Schedule &s)
{
    void *sd[] = {s.units, s.tile_first, s.tile_nsplit, s.counters, s.part, s.cta_first};
    for (void *d : sd)
        if (d) cudaFree(d);
    s = Schedule{};
}

static void free_plan(Plan *p)
{
    if (!p) return;
    void *dev[] = {p->lam, p->lo, p->hi, p->aoff, p->anchor, p->anchor_f, p->ratio_inv,
                   p->ratio_inv_f2, p->lam_f2, p->fwd_klo, p->fwd_khi, p->adj_dlo, p->adj_dhi, p->h, p->hinv_f,
                   p->Th, p->trial, p->s, p->G, p->g, p->x, p->r, p->z, p->p, p->u, p->q,
                   p->dir, p->R, p->Rt, p->O, p->Pbuf, p->Xbuf, p->freem, p->var, p->mrow,
                   p->partials, p->sc, p->idx_buf, p->val_buf};
    for (void *d : dev)
        if (d) cudaFree(d);
    auto free_sched = [](Schedule &s) { free_schedule(s); };
    for (auto &row : p->sched)
        for (Schedule &s : row) free_sched(s);
    for (Schedule &s : p->sched_tc) free_sched(s);
    void *mir[] = {p->ut_hi, p->ut_lo, p->ot_hi, p->ot_lo};
    for (void *d : mir)
        if (d) cudaFree(d);
    for (auto &row : p->cg_exec)
        for (cudaGraphExec_t &g : row)
            if (g) cudaGraphExecDestroy(g);
    if (p->prof_ev_ready)
        for (auto &row : p->prof_ev)
            for (cudaEvent_t &e : row) cudaEventDestroy(e);
    if (p->ev_in) cudaEventDestroy(p->ev_in);
    if (p->ev_out) cudaEventDestroy(p->ev_out);
    if (p->work) cudaStreamDestroy(p->work);
    if (p->sc_host) cudaFreeHost(p->sc_host);
    if (p->scratch_host) cudaFreeHost(p->scratch_host);
    if (p->own_stream && p->stream) cudaStreamDestroy(p->stream);
    delete p;
}

static tomo_status read_scalars(Plan &p)
{
    CUDA_TRY(cudaMemcpyAsync(p.sc_host, p.sc, sizeof(DevScalars), cudaMemcpyDeviceToHost, p.stream));
    CUDA_TRY(cudaStreamSynchronize(p.stream));
    return TOMO_OK;
}

// Stages a caller buffer of `count` doubles: device pointers are used as they
// are, host buffers are copied into (lazily allocated) plan memory.
static tomo_status stage_in(Plan &p, const double *src, int64_t count, double **buf,
                            const double **out)
{
    if (is_device_pointer(src)) {
        *out = src;
        return TOMO_OK;
    }
    if (!*buf) CUDA_TRY(dalloc(buf, count));
    CUDA_TRY(cudaMemcpyAsync(*buf, src, sizeof(double) * size_t(count), cudaMemcpyHostToDevice,
                             p.stream));
    *out = *buf;
    return TOMO_OK;
}

// A bounded mbarrier wait of a tensor-core contraction gave up (the kernel
// set tc_err and skipped its remaining units; the finish kernels, which need
// no counters, still ran to their end): report it once and clear the flag.
static tomo_status check_tc_err(Plan &p)
{
    if (!hvp_on_tensor_cores(p.precision)) return TOMO_OK;
    int32_t err = 0;
    CUDA_TRY(cudaMemcpyAsync(&err, &p.sc->tc_err, sizeof(err), cudaMemcpyDeviceToHost, p.stream));
    CUDA_TRY(cudaStreamSynchronize(p.stream));
    if (!err) return TOMO_OK;
    CUDA_TRY(cudaMemsetAsync(&p.sc->tc_err, 0, sizeof(int32_t), p.stream));
    CUDA_TRY(cudaStreamSynchronize(p.stream));
    return fail(TOMO_ETIMEOUT, "a bounded tensor-core pipeline wait gave up");
}

static tomo_status check_finite(Plan &p, const double *x, int64_t n, const char *what)
{
    CUDA_TRY(launch_nonfinite_check(p, x, n, 0));
    TOMO_TRY(read_scalars(p));
    if (p.sc_host->nonfinite > 0.0)
        return fail(TOMO_ENONFINITE, "%s holds %.0f non-finite values", what, p.sc_host->nonfinite);
    return TOMO_OK;
}

// Host planning of a tensor-core schedule, a pure function of the tiles'
// reduction ranges [st, en): units in CTA order, the CTA boundaries and the
// number of units per tile (see make_schedule_tc).
static void plan_tc_units(const int64_t *st, const int64_t *en, int tiles, int align, int64_t max_unit,
                          int64_t ctas, std::vector<WorkUnit> &units, std::vector<int32_t> &cta_first,
                          std::vector<int32_t> &nsplit)
{
    int64_t W = 0;
    for (int t = 0; t < tiles; ++t) W += std::max<int64_t>(0, en[t] - st[t]);
    if (ctas < 1) ctas = 1;
    int64_t share = (W + ctas - 1) / ctas;
    share = std::max<int64_t>(align, ((share + align - 1) / align) * align);
    std::vector<std::vector<WorkUnit>> per_cta(1);
    std::vector<int32_t> empty;
    nsplit.assign(tiles, 0);
    int64_t room = share;
    for (int t = 0; t < tiles; ++t) {
        const int64_t len = en[t] - st[t];
        if (len <= 0) {
            empty.push_back(t);
            continue;
        }
        for (int64_t pos = st[t]; pos < en[t];) {
            if (room == 0) {
                per_cta.emplace_back();
                room = share;
            }
            const int64_t l = std::min({en[t] - pos, room, max_unit});
            per_cta.back().push_back(WorkUnit{t, nsplit[t]++, int32_t(pos), int32_t(pos + l)});
            pos += l;
            room -= l;
        }
    }
    // an empty reduction still writes its (zero) tile: spread those units
    // evenly over the CTAs
    const int64_t nc = int64_t(per_cta.size());
    for (size_t j = 0; j < empty.size(); ++j) {
        per_cta[size_t((int64_t(j) * nc) / int64_t(empty.size()))].push_back(WorkUnit{empty[j], 0, 0, 0});
        nsplit[empty[j]] = 1;
    }
    units.clear();
    cta_first.assign(1, 0);
    for (const auto &v : per_cta) {
        units.insert(units.end(), v.begin(), v.end());
        cta_first.push_back(int32_t(units.size()));
    }
}

// Host planning for many tiles (at least 8 per CTA): whole tiles dealt to the
// CTAs round-robin, tile t to CTA t mod ctas, in tile order.  Every tile is
// one unit (no split-K partial), neighbouring tiles (whose reduction ranges
// overlap) run at the same time on different SMs and share their vector
// operand in L2, and the CTAs' sums of tile lengths are close because the
// lengths change slowly from tile to tile.
static void plan_tc_tiles_rr(const int64_t *st, const int64_t *en, int tiles, int64_t ctas,
                             std::vector<WorkUnit> &units, std::vector<int32_t> &cta_first,
                             std::vector<int32_t> &nsplit)
{
    if (ctas < 1) ctas = 1;
    units.clear();
    cta_first.assign(1, 0);
    nsplit.assign(tiles, 1);
    for (int64_t c = 0; c < ctas && c < tiles; ++c) {
        for (int64_t t = c; t < tiles; t += ctas) {
            const bool empty = en[t] <= st[t];
            units.push_back(WorkUnit{int32_t(t), 0, empty ? 0 : int32_t(st[t]), empty ? 0 : int32_t(en[t])});
        }
        cta_first.push_back(int32_t(units.size()));
    }
}

// Tensor-core schedule, one wave of persistent CTAs: the reduction ranges of
// all tiles, laid end to end, are cut into `ctas` shares of equal length
// (multiples of `align`); a share that crosses a tile boundary becomes one
// unit per tile it touches, and no unit is longer than max_unit (the size of
// the per-unit tables in shared memory).  CTA c runs its units in order; every
// unit writes its partial tile and the finish kernel combines each tile's
// partials in unit order, so the result does not depend on the CTA timing.
static cudaError_t make_schedule_tc(Plan &p, Schedule &S, const std::vector<int64_t> &st,
                                    const std::vector<int64_t> &en, int align, int64_t max_unit,
                                    int64_t ctas, int64_t *max_ctas)
{
    const int tiles = int(st.size());
    const int bn = band_bn(p.N);
    const int64_t ncol = (p.N + bn - 1) / bn;
    std::vector<WorkUnit> units;
    std::vector<int32_t> cta_first, nsplit, first(tiles, 0);
    if (int64_t(tiles) >= 8 * ctas)
        plan_tc_tiles_rr(st.data(), en.data(), tiles, ctas, units, cta_first, nsplit);
    else
        plan_tc_units(st.data(), en.data(), tiles, align, max_unit, ctas, units, cta_first, nsplit);
    // every unit writes a partial tile (the finish kernel combines them)
    int64_t slots = 0;
    for (int t = 0; t < tiles; ++t) { first[t] = int32_t(slots); slots += nsplit[t]; }
    cudaError_t e;
    S.n_units = int(units.size());
    S.n_ctas = int(cta_first.size()) - 1;
    if ((e = dalloc(&S.units, int64_t(units.size())))) return e;
    if ((e = dalloc(&S.tile_first, tiles))) return e;
    if ((e = dalloc(&S.tile_nsplit, tiles))) return e;
    if ((e = dalloc(&S.cta_first, int64_t(cta_first.size())))) return e;
    if ((e = cudaMalloc(&S.part, std::max<int64_t>(1, slots * ncol) * TILE_R * bn * sizeof(float)))) return e;
    if ((e = cudaMemcpyAsync(S.units, units.data(), sizeof(WorkUnit) * units.size(), cudaMemcpyHostToDevice, p.stream)) ||
        (e = cudaMemcpyAsync(S.tile_first, first.data(), sizeof(int32_t) * tiles, cudaMemcpyHostToDevice, p.stream)) ||
        (e = cudaMemcpyAsync(S.tile_nsplit, nsplit.data(), sizeof(int32_t) * tiles, cudaMemcpyHostToDevice, p.stream)) ||
        (e = cudaMemcpyAsync(S.cta_first, cta_first.data(), sizeof(int32_t) * cta_first.size(),
                             cudaMemcpyHostToDevice, p.stream)))
        return e;
    // the finish kernel's grid reduction: one partial per (32-row slice, column block)
    *max_ctas = std::max<int64_t>(*max_ctas, std::max<int64_t>(S.n_ctas, tiles * (TILE_R / 32)) * ncol);
    return cudaSuccess;
}

// SIMT schedule (split-K): the reduction range of every tile is cut into
// work units of equal length KC, chosen so that the whole contraction has
// about `units_per_sm` units per SM and column block; one CTA per unit.
//   st/en: per-tile [start, end) of the reduction range (empty if equal)
//   align: unit boundaries are multiples of `align` relative to 0 when
//          `aligned_start` (start rounded down, end rounded up), else relative
//          to the tile's start
static cudaError_t make_schedule(Plan &p, Schedule &S, const std::vector<int64_t> &st,
                                 const std::vector<int64_t> &en, int align, size_t part_elem_bytes,
                                 int64_t *max_ctas, int64_t max_kc = INT64_MAX,
                                 int64_t units_per_sm = 4)
{
    const int tiles = int(st.size());
    const int bn = band_bn(p.N);
    const int64_t ncol = (p.N + bn - 1) / bn;
    int64_t W = 0;
    for (int t = 0; t < tiles; ++t) W += en[t] - st[t];
    const int64_t target = std::max<int64_t>(1, units_per_sm * int64_t(p.num_sms) / ncol);
    int64_t kc = std::max<int64_t>(4 * int64_t(align), (W + target - 1) / target);
    kc = ((kc + align - 1) / align) * align;
    if (kc > max_kc) kc = max_kc;
    std::vector<WorkUnit> units;
    std::vector<int32_t> first(tiles, 0), nsplit(tiles, 1);
    int64_t slots = 0;
    for (int t = 0; t < tiles; ++t) {
        const int64_t len = en[t] - st[t];
        const int64_t n = len > 0 ? (len + kc - 1) / kc : 1;
        nsplit[t] = int32_t(n);
        if (n > 1) { first[t] = int32_t(slots); slots += n; }
        for (int64_t c = 0; c < n; ++c) {
            WorkUnit u;
            u.tile = t;
            u.chunk = int32_t(c);
            u.k0 = int32_t(st[t] + c * kc);
            u.k1 = int32_t(std::min<int64_t>(st[t] + (c + 1) * kc, en[t]));
            if (len <= 0) u.k0 = u.k1 = 0;
            units.push_back(u);
        }
    }
    cudaError_t e;
    S.n_units = int(units.size());
    if ((e = dalloc(&S.units, int64_t(units.size())))) return e;
    if ((e = dalloc(&S.tile_first, tiles))) return e;
    if ((e = dalloc(&S.tile_nsplit, tiles))) return e;
    if ((e = dalloc(&S.counters, tiles * ncol))) return e;
    if ((e = cudaMalloc(&S.part, std::max<int64_t>(1, slots * ncol) * TILE_R * bn * part_elem_bytes))) return e;
    if ((e = cudaMemcpyAsync(S.units, units.data(), sizeof(WorkUnit) * units.size(), cudaMemcpyHostToDevice, p.stream)) ||
        (e = cudaMemcpyAsync(S.tile_first, first.data(), sizeof(int32_t) * tiles, cudaMemcpyHostToDevice, p.stream)) ||
        (e = cudaMemcpyAsync(S.tile_nsplit, nsplit.data(), sizeof(int32_t) * tiles, cudaMemcpyHostToDevice, p.stream)) ||
        (e = cudaMemsetAsync(S.counters, 0, sizeof(unsigned) * tiles * ncol, p.stream)))
        return e;
    *max_ctas = std::max<int64_t>(*max_ctas, int64_t(units.size()) * ncol);
    return cudaSuccess;
}

// Work-unit schedules of the band contractions: the reduction range of every
// tile (union band of a probe tile, or probe range of a photon-number tile)
// is cut into split-K units, per unit for the SIMT kernels and per persistent
// CTA share for the tensor-core kernels.
static cudaError_t build_schedules(Plan &p, bool tensor_cores)
{
    std::vector<int32_t> klo(p.fwd_tiles), khi(p.fwd_tiles), dlo(p.adj_tiles), dhi(p.adj_tiles);
    cudaError_t e;
    // tile ranges produced by the plan kernels on the plan stream
    if ((e = cudaMemcpyAsync(klo.data(), p.fwd_klo, sizeof(int32_t) * klo.size(), cudaMemcpyDeviceToHost, p.stream)) ||
        (e = cudaMemcpyAsync(khi.data(), p.fwd_khi, sizeof(int32_t) * khi.size(), cudaMemcpyDeviceToHost, p.stream)) ||
        (e = cudaMemcpyAsync(dlo.data(), p.adj_dlo, sizeof(int32_t) * dlo.size(), cudaMemcpyDeviceToHost, p.stream)) ||
        (e = cudaMemcpyAsync(dhi.data(), p.adj_dhi, sizeof(int32_t) * dhi.size(), cudaMemcpyDeviceToHost, p.stream)) ||
        (e = cudaStreamSynchronize(p.stream)))
        return e;
    int64_t max_ctas = 0;
    auto ranges = [&](bool fwd, int align_start, int align_end, std::vector<int64_t> &st,
                      std::vector<int64_t> &en) {
        const int tiles = fwd ? p.fwd_tiles : p.adj_tiles;
        st.assign(tiles, 0);
        en.assign(tiles, 0);
        for (int t = 0; t < tiles; ++t) {
            const int64_t a = fwd ? klo[t] : dlo[t], b = fwd ? khi[t] : dhi[t];
            if (a > b) continue;
            st[t] = (a / align_start) * align_start;
            en[t] = ((b + 1 + align_end - 1) / align_end) * align_end;
        }
    };
    for (int dir = 0; dir < 2; ++dir) {
        for (int dbl = 0; dbl < 2; ++dbl) {
            const int BK = dbl ? 16 : 32;
            const bool fwd = dir == 0;
            std::vector<int64_t> st, en;
            // forward: K steps aligned to BK from 0; adjoint: probe ranges as they are
            ranges(fwd, fwd ? BK : 1, fwd ? BK : 1, st, en);
            if ((e = make_schedule(p, p.sched[dir][dbl], st, en, BK,
                                   dbl ? sizeof(double) : sizeof(float), &max_ctas, INT64_MAX,
                                   p.ups_simt > 0 ? p.ups_simt : 4)))
                return e;
        }
    }
    if (tensor_cores) {
        // tensor-core tiles reduce in slices of 64 aligned to 64 (16-byte,
        // 128-byte-row loads from the zero-padded transposed copies)
        for (int dir = 0; dir < 2; ++dir) {
            std::vector<int64_t> st, en;
            ranges(dir == 0, 64, 64, st, en);
            // one CTA per SM (shared memory): one wave of persistent CTAs
            // with equal shares of the reduction work
            const int64_t ncol = (p.N + band_bn(p.N) - 1) / band_bn(p.N);
            const int64_t ctas = p.tc_ctas > 0 ? std::min<int64_t>(p.tc_ctas, p.num_sms / ncol)
                                               : p.num_sms / ncol;
            if ((e = make_schedule_tc(p, p.sched_tc[dir], st, en, 64, TC_MAX_UNIT,
                                      std::max<int64_t>(1, ctas), &max_ctas)))
                return e;
        }
        if (!p.ut_hi) {  // transposed operand mirrors (kept across schedule rebuilds)
            const int64_t npad = ((p.N + 127) / 128) * 128;
            p.ut_pitch = ((p.M + 63) / 64) * 64;
            p.ot_pitch = ((p.D + 63) / 64) * 64;
            const size_t ub = sizeof(__nv_bfloat16) * size_t(npad * p.ut_pitch);
            const size_t ob = sizeof(__nv_bfloat16) * size_t(npad * p.ot_pitch);
            if ((e = cudaMalloc(&p.ut_hi, ub)) || (e = cudaMalloc(&p.ut_lo, ub)) ||
                (e = cudaMalloc(&p.ot_hi, ob)) || (e = cudaMalloc(&p.ot_lo, ob)))
                return e;
            if ((e = cudaMemsetAsync(p.ut_hi, 0, ub, p.stream)) || (e = cudaMemsetAsync(p.ut_lo, 0, ub, p.stream)) ||
                (e = cudaMemsetAsync(p.ot_hi, 0, ob, p.stream)) || (e = cudaMemsetAsync(p.ot_lo, 0, ob, p.stream)))
                return e;
            const int bn = band_bn(p.N);
            if ((e = encode_operand_map(&p.tm_ut_hi, p.ut_hi, p.ut_pitch, npad, bn)) ||
                (e = encode_operand_map(&p.tm_ut_lo, p.ut_lo, p.ut_pitch, npad, bn)) ||
                (e = encode_operand_map(&p.tm_ot_hi, p.ot_hi, p.ot_pitch, npad, bn)) ||
                (e = encode_operand_map(&p.tm_ot_lo, p.ot_lo, p.ot_pitch, npad, bn)))
                return e;
        }
    }
    p.max_partials = std::max<int64_t>(p.max_partials, max_ctas);
    return cudaSuccess;
}

// ---------------------------------------------------------------------------
// Plan-time autotuner of the schedule density.  Candidates: SIMT units per SM
// and column block {1, 2, 4, 8}, or tensor-core persistent CTAs per column
// block {all SMs, 3/4, 1/2}.  Each candidate's schedules are built and the
// Hessian product is timed (CUDA events on the plan stream, best of 3 after
// one warm-up); the fastest is kept.  Choices are cached per process by
// (form, N, power-of-two class of M, of D), so instances of one class in a
// batch tune once.
// ---------------------------------------------------------------------------
struct TuneKey {
    int prec;
    int64_t N;
    int lm, ld;
    bool operator<(const TuneKey &o) const
    {
        return std::tie(prec, N, lm, ld) < std::tie(o.prec, o.N, o.lm, o.ld);
    }
};
static std::mutex g_tune_mu;
static std::map<TuneKey, std::pair<int, double>> g_tune_cache;

static int ilog2(int64_t x)
{
    int r = 0;
    while (x > 1) { x >>= 1; ++r; }
    return r;
}

static cudaError_t rebuild_schedules(Plan &p)
{
    for (auto &row : p.sched)
        for (Schedule &s : row) free_schedule(s);
    for (Schedule &s : p.sched_tc) free_schedule(s);
    const int64_t before = p.max_partials;
    cudaError_t e = build_schedules(p, hvp_on_tensor_cores(p.precision));
    if (e != cudaSuccess) return e;
    if (p.partials && p.max_partials > before) {
        cudaFree(p.partials);
        p.partials = nullptr;
        e = dalloc(&p.partials, RED_SLOTS * p.max_partials);
    }
    return e;
}

static cudaError_t time_hvp(Plan &p, double *ms)
{
    cudaError_t e = launch_fill(p, p.p, 1.0 / double(p.N), p.M * p.N);
    // float input of the tensor-core form: 1/N in every float, written as
    // doubles whose two halves are that float
    const float f = 1.0f / float(p.N);
    uint32_t fb;
    std::memcpy(&fb, &f, sizeof(fb));
    const uint64_t pair = (uint64_t(fb) << 32) | uint64_t(fb);
    double dpair;
    std::memcpy(&dpair, &pair, sizeof(dpair));
    if (e == cudaSuccess) e = launch_fill(p, p.u, dpair, (p.M * p.N + 1) / 2);
    if (e != cudaSuccess) return e;
    cudaEvent_t a, b;
    if ((e = cudaEventCreate(&a)) != cudaSuccess) return e;
    if ((e = cudaEventCreate(&b)) != cudaSuccess) { cudaEventDestroy(a); return e; }
    double best = 1e30;
    for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {
        e = cudaEventRecord(a, p.stream);
        if (e == cudaSuccess) {
            if (hvp_on_tensor_cores(p.precision)) {
                // the CG's float vectors (the first half of the double buffers)
                e = launch_hvp_tc(p, p.u, p.q, true, false);
            } else {
                e = launch_forward(p, prec_products(p.precision), FWD_STORE, p.p, p.O, nullptr, false);
                if (e == cudaSuccess)
                    e = launch_adjoint(p, prec_products(p.precision), ADJ_HESS, p.O, p.q, p.p, false);
            }
        }
        if (e == cudaSuccess) e = cudaEventRecord(b, p.stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(b);
        float t = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&t, a, b);
        if (rep > 0 && t < best) best = t;
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    *ms = best;
    return e;
}

static cudaError_t autotune(Plan &p)
{
    const bool tc = hvp_on_tensor_cores(p.precision);
    const int64_t ncol = (p.N + band_bn(p.N) - 1) / band_bn(p.N);
    const int full = int(std::max<int64_t>(1, p.num_sms / ncol));
    std::vector<int> cand = tc ? std::vector<int>{full, std::max(1, 3 * full / 4), std::max(1, full / 2)}
                               : std::vector<int>{1, 2, 4, 8};
    const TuneKey key{p.precision, p.N, ilog2(p.M), ilog2(p.D)};
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            (tc ? p.tc_ctas : p.ups_simt) = it->second.first;
            p.tuned = 1;
            p.tuned_cached = 1;
            p.tuned_ms = it->second.second;
            return rebuild_schedules(p);
        }
    }
    int best = cand[0];
    double best_ms = 1e30;
    for (int c : cand) {
        (tc ? p.tc_ctas : p.ups_simt) = c;
        cudaError_t e = rebuild_schedules(p);
        double ms = 0.0;
        if (e == cudaSuccess) e = time_hvp(p, &ms);
        if (e != cudaSuccess) return e;
        if (ms < best_ms) { best_ms = ms; best = c; }
    }
    (tc ? p.tc_ctas : p.ups_simt) = best;
    p.tuned = 1;
    p.tuned_ms = best_ms;
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        g_tune_cache[key] = {best, best_ms};
    }
    return rebuild_schedules(p);
}

// R = F Theta - P in double, f = ||R||^2 + g(Theta) (Eq. min + Eq. regul).
static tomo_status residual_objective(Plan &p, const double *P, const double *Th, double *R,
                                      double *f)
{
    CUDA_TRY(launch_forward(p, TOMO_PREC_FP64, FWD_RESID, Th, R, P, false));
    CUDA_TRY(launch_regulariser(p, Th));
    TOMO_TRY(read_scalars(p));
    *f = p.sc_host->res2 + p.sc_host->regval;
    return TOMO_OK;
}

}  // namespace tomo

using namespace tomo;

extern "C" {

const char *tomo_last_error(void) { return g_err.c_str(); }

int64_t tomo_kernel_launches(void) { return g_launches.load(); }

void tomo_fit_opts_default(tomo_fit_opts *o)
{
    if (!o) return;
    o->eps_kkt = 1e-10;
    o->eps_bar = 1e-6;
    o->beta = 0.75;
    o->c = 0.1;
    o->switch_tol = 1e-4;
    o->f_target = 0.0;
    o->max_newton = 1000;
    o->max_stage1 = 200;
    o->max_cg = 10000;
    o->ls_max = 50;
    o->start_stage = 1;
    o->warm_start = 0;
    o->stall_iters = 5;
    o->refresh_every = 8;
    o->profile = 0;
    o->trace_len = 0;
    o->cg_eta_max = 0.5;
    o->cg_eta_pow = 0.5;
    o->max_seconds = 0.0;
    o->trace = nullptr;
}

tomo_status tomo_plan(tomo_plan_t *out, const tomo_desc *d)
{
    if (!out) return fail(TOMO_EINVAL, "out is NULL");
    *out = nullptr;
    if (!d) return fail(TOMO_EINVAL, "desc is NULL");
    if (d->M < 1 || d->M > (int64_t(1) << 30)) return fail(TOMO_EINVAL, "M=%lld out of range", (long long)d->M);
    if (d->N < 2 || d->N > MAX_N) return fail(TOMO_EINVAL, "N=%lld out of range [2, %d]", (long long)d->N, MAX_N);
    if (d->D < 1 || d->D > (int64_t(1) << 30)) return fail(TOMO_EINVAL, "D=%lld out of range", (long long)d->D);
    if (!d->lambda) return fail(TOMO_EINVAL, "lambda is NULL");
    if (!std::isfinite(d->gamma) || d->gamma < 0.0) return fail(TOMO_EINVAL, "gamma must be finite and >= 0");
    if (!std::isfinite(d->band_k)) return fail(TOMO_EINVAL, "band_k must be finite");
    if (d->precision != TOMO_PREC_FP64 && d->precision != TOMO_PREC_FP32 &&
        d->precision != TOMO_PREC_MIXED && d->precision != TOMO_PREC_TC)
        return fail(TOMO_EINVAL, "unknown precision %d", d->precision);
    if (d->flags & ~uint32_t(TOMO_PLAN_AUTOTUNE)) return fail(TOMO_EINVAL, "unknown flag bits");
    for (int64_t k = 0; k < d->D; ++k) {
        const double l = d->lambda[k];
        if (!std::isfinite(l) || l < 0.0) return fail(TOMO_EINVAL, "lambda[%lld] is not finite and >= 0", (long long)k);
        if (k > 0 && l < d->lambda[k - 1])
            return fail(TOMO_EINVAL, "lambda must be non-decreasing (lambda[%lld] < lambda[%lld])",
                        (long long)k, (long long)(k - 1));
    }
    if ((d->M * d->N) > (int64_t(1) << 40) || (d->D * d->N) > (int64_t(1) << 40))
        return fail(TOMO_EINVAL, "problem too large");

    Plan *p = new (std::nothrow) Plan();
    if (!p) return fail(TOMO_ENOMEM, "host allocation failed");
    std::memset(p, 0, sizeof(Plan));
    p->M = d->M; p->N = d->N; p->D = d->D;
    p->gamma = d->gamma; p->band_k = d->band_k; p->precision = d->precision;
    p->cg_f32 = hvp_on_tensor_cores(d->precision);

    auto bail = [&](tomo_status s) { free_plan(p); return s; };
#define PLAN_TRY(expr)                                                                     \
    do {                                                                                   \
        cudaError_t _e = (expr);                                                           \
        if (_e != cudaSuccess)                                                             \
            return bail(fail(_e == cudaErrorMemoryAllocation ? TOMO_ENOMEM : TOMO_ECUDA,    \
                             "%s failed: %s", #expr, cudaGetErrorString(_e)));             \
    } while (0)

    PLAN_TRY(cudaGetDevice(&p->device));
    PLAN_TRY(cudaDeviceGetAttribute(&p->num_sms, cudaDevAttrMultiProcessorCount, p->device));
    if (d->stream) {
        p->stream = static_cast<cudaStream_t>(d->stream);
    } else {
        PLAN_TRY(cudaStreamCreateWithFlags(&p->stream, cudaStreamNonBlocking));
        p->own_stream = true;
    }
    PLAN_TRY(cudaStreamCreateWithFlags(&p->work, cudaStreamNonBlocking));
    PLAN_TRY(cudaEventCreateWithFlags(&p->ev_in, cudaEventDisableTiming));
    PLAN_TRY(cudaEventCreateWithFlags(&p->ev_out, cudaEventDisableTiming));
    const int64_t M = p->M, N = p->N, D = p->D, MN = M * N, DN = D * N;
    p->fwd_tiles = int((D + TILE_R - 1) / TILE_R);
    p->adj_tiles = int((M + TILE_R - 1) / TILE_R);
    // row kernels and the per-tile partials of the fused CG restriction;
    // raised by the schedules
    p->max_partials = std::max<int64_t>(int64_t(p->num_sms) * 8, p->adj_tiles);

    PLAN_TRY(dalloc(&p->lam, D));
    PLAN_TRY(dalloc(&p->lo, D));
    PLAN_TRY(dalloc(&p->hi, D));
    PLAN_TRY(dalloc(&p->aoff, D + 1));
    PLAN_TRY(dalloc(&p->ratio_inv, M + RUN + 1));
    PLAN_TRY(dalloc(&p->ratio_inv_f2, M + RUN + 1));
    PLAN_TRY(dalloc(&p->lam_f2, D));
    PLAN_TRY(dalloc(&p->fwd_klo, p->fwd_tiles));
    PLAN_TRY(dalloc(&p->fwd_khi, p->fwd_tiles));
    PLAN_TRY(dalloc(&p->adj_dlo, p->adj_tiles));
    PLAN_TRY(dalloc(&p->adj_dhi, p->adj_tiles));
    PLAN_TRY(dalloc(&p->h, M));
    PLAN_TRY(dalloc(&p->hinv_f, 2 * M));
    double **mn_bufs[] = {&p->Th, &p->trial, &p->s, &p->G, &p->g, &p->x, &p->r,
                          &p->z, &p->p, &p->u, &p->q, &p->dir};
    for (double **b : mn_bufs) PLAN_TRY(dalloc(b, MN));
    PLAN_TRY(dalloc(&p->R, DN));
    PLAN_TRY(dalloc(&p->Rt, DN));
    PLAN_TRY(dalloc(&p->O, DN));
    PLAN_TRY(dalloc(&p->freem, MN));
    PLAN_TRY(dalloc(&p->var, MN));
    PLAN_TRY(dalloc(&p->mrow, M));
    PLAN_TRY(dalloc(&p->sc, 1));
    PLAN_TRY(cudaMallocHost(reinterpret_cast<void **>(&p->sc_host), sizeof(DevScalars)));
    PLAN_TRY(cudaMallocHost(reinterpret_cast<void **>(&p->scratch_host), 64 * sizeof(double)));
    PLAN_TRY(cudaMemsetAsync(p->sc, 0, sizeof(DevScalars), p->stream));
    PLAN_TRY(cudaMemcpyAsync(p->lam, d->lambda, sizeof(double) * size_t(D), cudaMemcpyHostToDevice,
                             p->stream));
    PLAN_TRY(launch_plan_tables(*p));
    PLAN_TRY(launch_hess_diag(*p));
    PLAN_TRY(cudaStreamSynchronize(p->stream));
    PLAN_TRY(build_schedules(*p, hvp_on_tensor_cores(p->precision)));
    PLAN_TRY(dalloc(&p->partials, RED_SLOTS * p->max_partials));
    if (d->flags & TOMO_PLAN_AUTOTUNE) PLAN_TRY(autotune(*p));
    // every initialisation (zeroed counters and operand mirrors) is issued on
    // the plan stream, which may be non-blocking: finish it before any call
    // can launch work on another stream
    PLAN_TRY(cudaStreamSynchronize(p->stream));
#undef PLAN_TRY
    *out = reinterpret_cast<tomo_plan_t>(p);
    return TOMO_OK;
}

void tomo_plan_destroy(tomo_plan_t plan)
{
    Plan *p = reinterpret_cast<Plan *>(plan);
    if (!p) return;
    cudaStreamSynchronize(p->stream);
    free_plan(p);
}

tomo_status tomo_objective(tomo_plan_t plan, const double *P, const double *Theta, double *f_host,
                           double *grad)
{
    Plan *pp = reinterpret_cast<Plan *>(plan);
    if (!pp || !P || !Theta || !f_host) return fail(TOMO_EINVAL, "NULL argument");
    Plan &p = *pp;
    const int64_t MN = p.M * p.N, DN = p.D * p.N;
    const double *Pd, *Td;
    TOMO_TRY(stage_in(p, P, DN, &p.Pbuf, &Pd));
    TOMO_TRY(stage_in(p, Theta, MN, &p.Xbuf, &Td));
    TOMO_TRY(check_finite(p, Pd, DN, "P"));
    TOMO_TRY(check_finite(p, Td, MN, "Theta"));
    double f = 0.0;
    TOMO_TRY(residual_objective(p, Pd, Td, p.R, &f));
    *f_host = f;
    if (grad) {
        const bool gdev = is_device_pointer(grad);
        double *gd = gdev ? grad : p.G;
        CUDA_TRY(launch_adjoint(p, prec_gradient(p.precision), ADJ_GRAD, p.R, gd, Td, false));
        if (!gdev)
            CUDA_TRY(cudaMemcpyAsync(grad, gd, sizeof(double) * size_t(MN), cudaMemcpyDeviceToHost,
                                     p.stream));
    }
    CUDA_TRY(cudaStreamSynchronize(p.stream));
    if (!std::isfinite(f)) return fail(TOMO_ENONFINITE, "objective is not finite");
    return TOMO_OK;
}

}  // extern "C"

namespace tomo {

// Hessian products of the CG loop, launched `count` times; every kernel is
// gated on the device flag cg_active, so launches after convergence are
// empty.  Stage 1 multiplies p itself, stage 2 the lifted u = E p.
constexpr int CG_CHUNK = 4;

// Events bracketing the band contractions of one CG chunk (profiling); they
// live in the plan because captured graphs record them.
struct ChunkEvents {
    cudaEvent_t (*ev)[3];
};

static tomo_status prof_events(Plan &p, ChunkEvents *out)
{
    if (!p.prof_ev_ready) {
        for (auto &row : p.prof_ev)
            for (cudaEvent_t &e : row) CUDA_TRY(cudaEventCreate(&e));
        p.prof_ev_ready = true;
    }
    out->ev = p.prof_ev;
    return TOMO_OK;
}

static tomo_status cg_chunk(Plan &p, int stage, int count, const ChunkEvents *evs)
{
    const double *in = stage == 1 ? p.p : p.u;   // float data when p.cg_f32
    const bool tc = hvp_on_tensor_cores(p.precision);
    // while capturing, profiling events must become event-record nodes
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (evs) CUDA_TRY(cudaStreamIsCapturing(p.stream, &cap));
    const unsigned evflag = cap == cudaStreamCaptureStatusActive ? cudaEventRecordExternal : 0u;
    // tensor-core form with N <= 128: the mirror of the product input is
    // written by the previous direction update (or once after the set-up)
    const bool fused_p = tc && tc_update_p_fusable(p);
    for (int c = 0; c < count; ++c) {
        if (evs) CUDA_TRY(cudaEventRecordWithFlags(evs->ev[c][0], p.stream, evflag));
        if (tc) {
            // tensor cores: the whole Hessian product (forward + adjoint) is
            // timed as the "forward" interval, the adjoint interval is empty
            CUDA_TRY(launch_hvp_tc(p, in, p.q, p.cg_f32, true, stage, !fused_p));
            if (evs) CUDA_TRY(cudaEventRecordWithFlags(evs->ev[c][1], p.stream, evflag));
        } else {
            CUDA_TRY(launch_forward(p, prec_products(p.precision), FWD_STORE, in, p.O, nullptr, true));
            if (evs) CUDA_TRY(cudaEventRecordWithFlags(evs->ev[c][1], p.stream, evflag));
            CUDA_TRY(launch_adjoint(p, prec_products(p.precision), ADJ_HESS, p.O, p.q, in, true));
        }
        if (evs) CUDA_TRY(cudaEventRecordWithFlags(evs->ev[c][2], p.stream, evflag));
        // the tensor-core adjoint applies the restriction itself when it can
        if (!(tc && tc_restrict_fusable(p))) CUDA_TRY(launch_cg_restrict(p, stage));
        CUDA_TRY(launch_cg_update_xr(p, stage));
        if (fused_p) CUDA_TRY(launch_cg_update_p_split(p, stage));
        else CUDA_TRY(launch_cg_update_p(p, stage));
    }
    return TOMO_OK;
}

// One chunk of CG iterations: launched directly the first time (which also
// configures every kernel), then captured once into a CUDA graph per (stage,
// profile) and replayed.
static tomo_status run_cg_chunk(Plan &p, int stage, const ChunkEvents *evs)
{
    const int ks = stage - 1, kp = evs ? 1 : 0;
    if (p.cg_exec[ks][kp]) {
        CUDA_TRY(cudaGraphLaunch(p.cg_exec[ks][kp], p.stream));
        count_launch(p.cg_exec_kernels[ks][kp]);
        return TOMO_OK;
    }
    if (p.cg_direct_runs[ks][kp]++ < 1) return cg_chunk(p, stage, CG_CHUNK, evs);
    const int64_t l0 = tomo_kernel_launches();
    CUDA_TRY(cudaStreamBeginCapture(p.stream, cudaStreamCaptureModeThreadLocal));
    tomo_status st = cg_chunk(p, stage, CG_CHUNK, evs);
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(p.stream, &graph);
    const int nk = int(tomo_kernel_launches() - l0);
    count_launch(-nk);  // capture launched nothing
    if (st != TOMO_OK) {
        if (graph) cudaGraphDestroy(graph);
        return st;
    }
    CUDA_TRY(e);
    e = cudaGraphInstantiate(&p.cg_exec[ks][kp], graph, 0);
    cudaGraphDestroy(graph);
    CUDA_TRY(e);
    p.cg_exec_kernels[ks][kp] = nk;
    CUDA_TRY(cudaGraphLaunch(p.cg_exec[ks][kp], p.stream));
    count_launch(nk);
    return TOMO_OK;
}

struct LsResult {
    bool ok;
    double f_new, gts, alpha;
    int neg;      // trials rejected because an implicit entry went negative
};

// Backtracking line search of App. B along dir (or -g/diag when the device
// flag use_grad_dir is set): alpha = beta^m, m = 0, 1, ...; accept the first
// trial with f(trial) <= f + c g^T (trial - Theta) (stage 2 also needs every
// implicit entry Theta_{i,m(i)} >= 0).  Direct mode evaluates f(trial) from a
// fresh residual F trial - P; delta mode from R + F s with s = trial - Theta.
static tomo_status line_search(Plan &p, int stage, const double *P, double f,
                               const tomo_fit_opts &o, bool delta, int32_t *ls_count, LsResult *res)
{
    res->ok = false;
    res->neg = 0;
    double alpha = 1.0;
    for (int m = 0; m < o.ls_max; ++m, alpha *= o.beta) {
        ++*ls_count;
        CUDA_TRY(launch_trial(p, stage, alpha, delta));
        if (delta)
            CUDA_TRY(launch_forward_gated_ls(p, prec_products(p.precision), FWD_DELTA, p.s, p.Rt, p.R));
        else
            CUDA_TRY(launch_forward_gated_ls(p, TOMO_PREC_FP64, FWD_RESID, p.trial, p.Rt, P));
        TOMO_TRY(read_scalars(p));
        const DevScalars &s = *p.sc_host;
        if (s.neg) {
            ++res->neg;
            continue;
        }
        bool accept;
        double fn;
        if (delta) {
            const double df = s.dres + s.reg;
            accept = df <= o.c * s.gts;
            fn = f + df;
        } else {
            fn = s.res2 + s.reg;
            accept = fn <= f + o.c * s.gts;
        }
        if (accept) {
            res->ok = true;
            res->f_new = fn;
            res->gts = s.gts;
            res->alpha = alpha;
            return TOMO_OK;
        }
    }
    return TOMO_OK;
}

static tomo_status fit_impl(Plan &p, const double *P, const tomo_fit_opts &o, tomo_fit_report &rep)
{
    const int64_t M = p.M, N = p.N;
    const double MN = double(M) * double(N);
    const bool fp64 = p.precision == TOMO_PREC_FP64;
    const bool delta = !fp64;
    ChunkEvents evs;
    if (o.profile) TOMO_TRY(prof_events(p, &evs));
    double f = 0.0;
    TOMO_TRY(residual_objective(p, P, p.Th, p.R, &f));
    rep.refreshes = 1;
    int stage = o.start_stage == 2 ? 2 : 1;
    int stall = 0, since_refresh = 0;
    rep.stop = 2;
    const auto t_start = std::chrono::steady_clock::now();
    auto elapsed_ms = [&]() {
        return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_start).count();
    };
    for (int k = 0; k < o.max_newton; ++k) {
        if (o.max_seconds > 0.0 && elapsed_ms() >= 1e3 * o.max_seconds) break;
        double *trow = k < o.trace_len ? o.trace + size_t(k) * TOMO_TRACE_COLS : nullptr;
        // gradient G = 2 F^T R + 2 gamma L Theta
        CUDA_TRY(launch_adjoint(p, prec_gradient(p.precision), ADJ_GRAD, p.R, p.G, p.Th, false));
        if (stage == 1 && rep.iters_s1 >= o.max_stage1) stage = 2;
        CUDA_TRY(launch_setup1(p, stage, o.eps_bar));
        CUDA_TRY(launch_setup2(p, stage, o.max_cg, o.cg_eta_max, o.cg_eta_pow));
        // the first Hessian product's input mirror (later ones come from the
        // fused direction update)
        if (hvp_on_tensor_cores(p.precision) && tc_update_p_fusable(p))
            CUDA_TRY(launch_tc_split_input(p, stage == 1 ? p.p : p.u, p.cg_f32, true));
        TOMO_TRY(read_scalars(p));
        const double kkt = std::sqrt(p.sc_host->kkt2 / MN);
        if (!std::isfinite(kkt) || !std::isfinite(f))
            return fail(TOMO_ENONFINITE, "non-finite objective or gradient at iteration %d", k);
        if (kkt <= o.eps_kkt) { rep.stop = 0; break; }
        if (o.f_target > 0.0 && f <= o.f_target) {
            if (!fp64 && since_refresh > 0) {
                TOMO_TRY(residual_objective(p, P, p.Th, p.R, &f));
                ++rep.refreshes;
                since_refresh = 0;
            }
            if (f <= o.f_target) { rep.stop = 1; break; }
        }
        // truncated Newton direction: PCG on the free variables
        const double t_cg0 = trow ? elapsed_ms() : 0.0;
        int active = p.sc_host->cg_active;
        int done = 0;
        while (active) {
            TOMO_TRY(run_cg_chunk(p, stage, o.profile ? &evs : nullptr));
            TOMO_TRY(read_scalars(p));
            // a tensor-core wait that gave up leaves the product incomplete:
            // stop at once (tomo_fit reports it and clears the flag)
            if (p.sc_host->tc_err)
                return fail(TOMO_ETIMEOUT, "a bounded tensor-core pipeline wait gave up (Newton iteration %d)", k);
            active = p.sc_host->cg_active;
            if (o.profile) {
                // only the iterations that ran (the rest of the chunk exited
                // at the gate) are counted
                const int ran = p.sc_host->cg_iters - done;
                for (int c = 0; c < ran && c < CG_CHUNK; ++c) {
                    float a = 0.f, b = 0.f;
                    CUDA_TRY(cudaEventElapsedTime(&a, evs.ev[c][0], evs.ev[c][1]));
                    CUDA_TRY(cudaEventElapsedTime(&b, evs.ev[c][1], evs.ev[c][2]));
                    rep.fwd_ms += a;
                    rep.adj_ms += b;
                    ++rep.fwd_count;
                    ++rep.adj_count;
                }
            }
            done = p.sc_host->cg_iters;
        }
        rep.cg_total += p.sc_host->cg_iters;
        if (trow) {
            const DevScalars &c = *p.sc_host;
            trow[0] = stage;
            trow[1] = f;
            trow[2] = kkt;
            trow[3] = c.cg_iters;
            trow[4] = c.bn > 0.0 ? std::sqrt(c.rr) / c.bn : 0.0;
            trow[5] = 0.0;
            trow[6] = rep.ls_total;
            trow[9] = !(c.pq > 0.0) && c.cg_iters > 0 ? 2.0 : (c.cg_iters >= c.max_cg && !(std::sqrt(c.rr) <= c.tol)) ? 1.0 : 0.0;
            trow[10] = elapsed_ms() - t_cg0;
        }
        CUDA_TRY(launch_direction(p, stage));
        if (stage == 1) ++rep.iters_s1; else ++rep.iters_s2;

        LsResult ls;
        TOMO_TRY(line_search(p, stage, P, f, o, delta, &rep.ls_total, &ls));
        if (!ls.ok) {
            CUDA_TRY(launch_set_grad_dir(p));
            TOMO_TRY(line_search(p, stage, P, f, o, delta, &rep.ls_total, &ls));
        }
        if (trow) {
            trow[5] = ls.ok ? ls.alpha : 0.0;
            trow[6] = rep.ls_total - trow[6];
            trow[7] = elapsed_ms();
            trow[8] = ls.neg;
        }
        if (!ls.ok) {
            if (stage == 1) { stage = 2; continue; }
            rep.stop = 3;
            break;
        }
        std::swap(p.Th, p.trial);
        std::swap(p.R, p.Rt);
        if (stage == 1 && std::fabs(ls.gts / ls.alpha) <= o.switch_tol) stage = 2;
        const double f_new = ls.f_new;
        if (!(f_new < f * (1.0 - 1e-15))) {
            if (++stall >= o.stall_iters) { f = f_new; rep.stop = 3; break; }
        } else {
            stall = 0;
        }
        f = f_new;
        if (!fp64 && ++since_refresh >= o.refresh_every) {
            TOMO_TRY(residual_objective(p, P, p.Th, p.R, &f));
            ++rep.refreshes;
            since_refresh = 0;
        }
    }
    // final state, always in double
    TOMO_TRY(residual_objective(p, P, p.Th, p.R, &f));
    CUDA_TRY(launch_adjoint(p, TOMO_PREC_FP64, ADJ_GRAD, p.R, p.G, p.Th, false));
    CUDA_TRY(launch_kkt(p, p.Th, p.G));
    TOMO_TRY(read_scalars(p));
    rep.f = f;
    rep.kkt = std::sqrt(p.sc_host->kkt2 / MN);
    rep.stage_end = stage;
    if (!std::isfinite(f)) return fail(TOMO_ENONFINITE, "objective is not finite");
    return TOMO_OK;
}

}  // namespace tomo

extern "C" {

tomo_status tomo_fit(tomo_plan_t plan, const double *P, double *Theta, const tomo_fit_opts *opts,
                     tomo_fit_report *report)
{
    Plan *pp = reinterpret_cast<Plan *>(plan);
    if (!pp || !P || !Theta) return fail(TOMO_EINVAL, "NULL argument");
    Plan &p = *pp;
    tomo_fit_opts o;
    if (opts) o = *opts; else tomo_fit_opts_default(&o);
    if (!(o.beta > 0.0 && o.beta < 1.0) || !(o.c > 0.0 && o.c < 1.0) || o.max_newton < 0 ||
        o.max_cg < 0 || o.ls_max < 1 || !(o.eps_bar >= 0.0) || !(o.eps_kkt >= 0.0) ||
        o.refresh_every < 1 || o.stall_iters < 1 || !(o.cg_eta_max > 0.0 && o.cg_eta_max < 1.0) ||
        !(o.cg_eta_pow >= 0.0 && o.cg_eta_pow <= 2.0) || !(o.max_seconds >= 0.0) || o.trace_len < 0 ||
        (o.trace_len > 0 && !o.trace))
        return fail(TOMO_EINVAL, "invalid options");
    tomo_fit_report rep;
    std::memset(&rep, 0, sizeof(rep));
    const int64_t l0 = tomo_kernel_launches();
    const auto t0 = std::chrono::steady_clock::now();
    // the solve runs on the plan's work stream (capturable), fenced against
    // the caller's stream on entry and exit
    CUDA_TRY(cudaEventRecord(p.ev_in, p.stream));
    CUDA_TRY(cudaStreamWaitEvent(p.work, p.ev_in, 0));
    struct StreamSwap {
        Plan &p;
        cudaStream_t user;
        explicit StreamSwap(Plan &pl) : p(pl), user(pl.stream) { p.stream = p.work; }
        ~StreamSwap()
        {
            p.stream = user;
            if (cudaEventRecord(p.ev_out, p.work) == cudaSuccess) cudaStreamWaitEvent(user, p.ev_out, 0);
        }
    } swap_guard(p);
    const int64_t MN = p.M * p.N, DN = p.D * p.N;
    const double *Pd;
    TOMO_TRY(stage_in(p, P, DN, &p.Pbuf, &Pd));
    TOMO_TRY(check_finite(p, Pd, DN, "P"));
    const bool tdev = is_device_pointer(Theta);
    if (o.warm_start) {
        CUDA_TRY(cudaMemcpyAsync(p.Th, Theta, sizeof(double) * size_t(MN),
                                 tdev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, p.stream));
        TOMO_TRY(check_finite(p, p.Th, MN, "Theta"));
    } else {
        CUDA_TRY(launch_fill(p, p.Th, 1.0 / double(p.N), MN));
    }
    tomo_status st = fit_impl(p, Pd, o, rep);
    // the tensor-core flag is read and cleared on every exit path, so that a
    // timeout is never reported by a later call; it is the root cause of any
    // other failure of the same solve
    const tomo_status te = check_tc_err(p);
    if (te == TOMO_ETIMEOUT) return te;
    if (st != TOMO_OK) return st;
    TOMO_TRY(te);
    CUDA_TRY(cudaMemcpyAsync(Theta, p.Th, sizeof(double) * size_t(MN),
                             tdev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, p.stream));
    CUDA_TRY(cudaStreamSynchronize(p.stream));
    rep.time_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    rep.kernels = int32_t(tomo_kernel_launches() - l0);
    if (report) *report = rep;
    return rep.stop == 2 ? TOMO_ENOTCONV : TOMO_OK;
}

tomo_status tomo_fit_warm(tomo_plan_t plan, tomo_ws_t ws, const double *P, double *Theta,
                          double zero_below, const tomo_fit_opts *opts, tomo_fit_report *report,
                          int32_t *used_warm)
{
    Plan *pp = reinterpret_cast<Plan *>(plan);
    if (used_warm) *used_warm = 0;
    if (!pp || !ws || !P || !Theta) return fail(TOMO_EINVAL, "NULL argument");
    Plan &p = *pp;
    int64_t wD = 0, wM = 0, wC0 = 0;
    if (!(zero_below >= 0.0 && zero_below < 1.0)) return fail(TOMO_EINVAL, "zero_below must lie in [0, 1)");
    if (!ws_shape(ws, &wD, &wM, &wC0) || wD != p.D || wM != p.M || p.N > wC0)
        return fail(TOMO_EINVAL, "the warm-start handle does not match the plan (D, M, N <= C0)");
    if (!is_device_pointer(P) || !is_device_pointer(Theta))
        return fail(TOMO_EINVAL, "P and Theta must be device pointers");
    tomo_fit_opts o;
    if (opts) o = *opts; else tomo_fit_opts_default(&o);
    const int64_t MN = p.M * p.N;
    // Theta0 from the network, then f(Theta0) and f(1/N) in double
    TOMO_TRY(tomo_ws_infer(ws, P, p.N, Theta));
    if (zero_below > 0.0) CUDA_TRY(launch_zero_small_rows(p, Theta, zero_below));
    double f0 = 0.0, fu = 0.0;
    TOMO_TRY(residual_objective(p, P, Theta, p.R, &f0));
    CUDA_TRY(launch_fill(p, p.Th, 1.0 / double(p.N), MN));
    TOMO_TRY(residual_objective(p, P, p.Th, p.R, &fu));
    if (std::isfinite(f0) && f0 < fu) {
        o.warm_start = 1;
        tomo_fit_report rep;
        std::memset(&rep, 0, sizeof(rep));
        const tomo_status st = tomo_fit(plan, P, Theta, &o, &rep);
        if ((st == TOMO_OK || st == TOMO_ENOTCONV) && std::isfinite(rep.f)) {
            if (report) *report = rep;
            if (used_warm) *used_warm = 1;
            return st;
        }
    }
    // Theta0 no better than the uniform start, or the warm fit failed
    o.warm_start = 0;
    return tomo_fit(plan, P, Theta, &o, report);
}

tomo_status tomo_fit_batched(const tomo_desc *descs, const double *const *P, double *const *Theta,
                             int32_t count, const tomo_fit_opts *opts, tomo_fit_report *reports,
                             tomo_status *statuses, int32_t concurrency)
{
    if (count < 0 || (count > 0 && (!descs || !P || !Theta || !statuses)))
        return fail(TOMO_EINVAL, "invalid batch arguments");
    if (count == 0) return TOMO_OK;
    if (concurrency <= 0) concurrency = 8;
    if (concurrency > count) concurrency = count;
    int dev = 0;
    CUDA_TRY(cudaGetDevice(&dev));
    std::atomic<int> next{0};
    auto worker = [&]() {
        cudaSetDevice(dev);
        for (;;) {
            const int k = next.fetch_add(1);
            if (k >= count) break;
            tomo_fit_report rep;
            std::memset(&rep, 0, sizeof(rep));
            tomo_plan_t pl = nullptr;
            tomo_status st = tomo_plan(&pl, &descs[k]);
            if (st == TOMO_OK) {
                st = tomo_fit(pl, P[k], Theta[k], opts, &rep);
                tomo_plan_destroy(pl);
            }
            statuses[k] = st;
            if (reports) reports[k] = rep;
        }
    };
    std::vector<std::thread> pool;
    for (int t = 1; t < concurrency; ++t) pool.emplace_back(worker);
    worker();
    for (auto &th : pool) th.join();
    for (int k = 0; k < count; ++k)
        if (statuses[k] != TOMO_OK && statuses[k] != TOMO_ENOTCONV)
            return fail(statuses[k], "instance %d failed", k);
    return TOMO_OK;
}

tomo_status tomo_apply_F(tomo_plan_t plan, const double *X, double *O)
{
    Plan *p = reinterpret_cast<Plan *>(plan);
    if (!p || !X || !O) return fail(TOMO_EINVAL, "NULL argument");
    CUDA_TRY(launch_forward(*p, prec_products(p->precision), FWD_STORE, X, O, nullptr, false));
    CUDA_TRY(cudaStreamSynchronize(p->stream));
    return TOMO_OK;
}

tomo_status tomo_apply_Ft(tomo_plan_t plan, const double *Y, double *Z)
{
    Plan *p = reinterpret_cast<Plan *>(plan);
    if (!p || !Y || !Z) return fail(TOMO_EINVAL, "NULL argument");
    CUDA_TRY(launch_adjoint(*p, prec_products(p->precision), ADJ_STORE, Y, Z, nullptr, false));
    CUDA_TRY(cudaStreamSynchronize(p->stream));
    return TOMO_OK;
}

tomo_status tomo_hvp(tomo_plan_t plan, const double *V, double *HV)
{
    Plan *p = reinterpret_cast<Plan *>(plan);
    if (!p || !V || !HV) return fail(TOMO_EINVAL, "NULL argument");
    if (hvp_on_tensor_cores(p->precision)) {
        CUDA_TRY(launch_hvp_tc(*p, V, HV, false, false));
        CUDA_TRY(cudaStreamSynchronize(p->stream));
        TOMO_TRY(check_tc_err(*p));
    } else {
        CUDA_TRY(launch_forward(*p, prec_products(p->precision), FWD_STORE, V, p->O, nullptr, false));
        CUDA_TRY(launch_adjoint(*p, prec_products(p->precision), ADJ_GRAD, p->O, HV, V, false));
    }
    CUDA_TRY(cudaStreamSynchronize(p->stream));
    return TOMO_OK;
}

int64_t tomo_plan_tc_units(const int64_t *st, const int64_t *en, int32_t tiles, int32_t align,
                           int64_t max_unit, int64_t ctas, int32_t *units_out, int64_t capacity,
                           int32_t *cta_first_out, int32_t *nsplit_out, int32_t *n_ctas_out)
{
    if (!st || !en || tiles < 1 || align < 1 || max_unit < align || (max_unit % align) != 0 ||
        !units_out || !cta_first_out || !nsplit_out || !n_ctas_out) {
        tomo_set_error(TOMO_EINVAL, "invalid argument");
        return -1;
    }
    for (int32_t t = 0; t < tiles; ++t)
        if (en[t] > st[t] && ((st[t] % align) != 0 || (en[t] % align) != 0)) {
            tomo_set_error(TOMO_EINVAL, "tile ranges must be multiples of align");
            return -1;
        }
    std::vector<WorkUnit> units;
    std::vector<int32_t> cta_first, nsplit;
    plan_tc_units(st, en, tiles, align, max_unit, ctas, units, cta_first, nsplit);
    if (int64_t(units.size()) > capacity || int64_t(cta_first.size()) > ctas + 1) {
        tomo_set_error(TOMO_EINVAL, "output capacity too small");
        return -1;
    }
    for (size_t k = 0; k < units.size(); ++k) {
        units_out[4 * k] = units[k].tile;
        units_out[4 * k + 1] = units[k].chunk;
        units_out[4 * k + 2] = units[k].k0;
        units_out[4 * k + 3] = units[k].k1;
    }
    for (size_t k = 0; k < cta_first.size(); ++k) cta_first_out[k] = cta_first[k];
    for (int32_t t = 0; t < tiles; ++t) nsplit_out[t] = nsplit[size_t(t)];
    *n_ctas_out = int32_t(cta_first.size()) - 1;
    return int64_t(units.size());
}

tomo_status tomo_plan_info(tomo_plan_t plan, tomo_plan_info_t *info)
{
    Plan *p = reinterpret_cast<Plan *>(plan);
    if (!p || !info) return fail(TOMO_EINVAL, "NULL argument");
    const bool tc = hvp_on_tensor_cores(p->precision);
    info->autotuned = p->tuned;
    info->from_cache = p->tuned_cached;
    info->density = tc ? (p->tc_ctas > 0 ? p->tc_ctas : p->num_sms) : (p->ups_simt > 0 ? p->ups_simt : 4);
    info->tensor_cores = tc ? 1 : 0;
    info->hvp_ms = p->tuned_ms;
    const int dbl = prec_products(p->precision) == TOMO_PREC_FP64 ? 1 : 0;
    info->units_fwd = tc ? p->sched_tc[0].n_units : p->sched[0][dbl].n_units;
    info->units_adj = tc ? p->sched_tc[1].n_units : p->sched[1][dbl].n_units;
    info->ctas_fwd = tc ? p->sched_tc[0].n_ctas : p->sched[0][dbl].n_units;
    info->ctas_adj = tc ? p->sched_tc[1].n_ctas : p->sched[1][dbl].n_units;
    return TOMO_OK;
}

tomo_status tomo_selftest_tc_timeout(tomo_plan_t plan)
{
    Plan *p = reinterpret_cast<Plan *>(plan);
    if (!p) return fail(TOMO_EINVAL, "NULL argument");
    if (!hvp_on_tensor_cores(p->precision)) return fail(TOMO_EINVAL, "the plan is not in the tensor-core form");
    CUDA_TRY(launch_fill(*p, p->p, 1.0 / double(p->N), p->M * p->N));
    CUDA_TRY(launch_hvp_tc_wait_selftest(*p, p->p, p->q));
    CUDA_TRY(cudaStreamSynchronize(p->stream));
    return check_tc_err(*p);
}

tomo_status tomo_hess_diag(tomo_plan_t plan, double *h)
{
    Plan *p = reinterpret_cast<Plan *>(plan);
    if (!p || !h) return fail(TOMO_EINVAL, "NULL argument");
    CUDA_TRY(cudaMemcpyAsync(h, p->h, sizeof(double) * size_t(p->M), cudaMemcpyDefault, p->stream));
    CUDA_TRY(cudaStreamSynchronize(p->stream));
    return TOMO_OK;
}

tomo_status tomo_project_simplex(tomo_plan_t plan, const double *X, double *Y)
{
    Plan *p = reinterpret_cast<Plan *>(plan);
    if (!p || !X || !Y) return fail(TOMO_EINVAL, "NULL argument");
    CUDA_TRY(launch_project_rows(*p, X, Y));
    CUDA_TRY(cudaStreamSynchronize(p->stream));
    return TOMO_OK;
}

tomo_status tomo_smooth(tomo_plan_t plan, const double *X, double *Y, int64_t exclude, double div)
{
    Plan *p = reinterpret_cast<Plan *>(plan);
    if (!p || !X || !Y) return fail(TOMO_EINVAL, "NULL argument");
    if (exclude < 0 || !(div > 0.0)) return fail(TOMO_EINVAL, "exclude must be >= 0 and div > 0");
    CUDA_TRY(launch_smooth(*p, X, Y, exclude, div));
    CUDA_TRY(cudaStreamSynchronize(p->stream));
    return TOMO_OK;
}

tomo_status tomo_infidelity(tomo_plan_t plan, const double *Theta, const double *Theta_ref, double *infid_host)
{
    Plan *p = reinterpret_cast<Plan *>(plan);
    if (!p || !Theta || !Theta_ref || !infid_host) return fail(TOMO_EINVAL, "NULL argument");
    CUDA_TRY(launch_infidelity(*p, Theta, Theta_ref, p->O));
    CUDA_TRY(cudaMemcpyAsync(infid_host, p->O, sizeof(double) * size_t(p->N), cudaMemcpyDeviceToHost, p->stream));
    CUDA_TRY(cudaStreamSynchronize(p->stream));
    return TOMO_OK;
}

tomo_status tomo_kkt(tomo_plan_t plan, const double *Theta, const double *G, double *kkt_host)
{
    Plan *p = reinterpret_cast<Plan *>(plan);
    if (!p || !Theta || !G || !kkt_host) return fail(TOMO_EINVAL, "NULL argument");
    CUDA_TRY(launch_kkt(*p, Theta, G));
    TOMO_TRY(read_scalars(*p));
    *kkt_host = std::sqrt(p->sc_host->kkt2 / (double(p->M) * double(p->N)));
    return TOMO_OK;
}

tomo_status tomo_poisson_weights(tomo_plan_t plan, const int64_t *d, const int64_t *i,
                                 int64_t count, double *out_host)
{
    Plan *p = reinterpret_cast<Plan *>(plan);
    if (!p || (count > 0 && (!d || !i || !out_host)) || count < 0)
        return fail(TOMO_EINVAL, "invalid argument");
    if (count == 0) return TOMO_OK;
    if (count > p->idx_cap) {
        if (p->idx_buf) cudaFree(p->idx_buf);
        if (p->val_buf) cudaFree(p->val_buf);
        p->idx_buf = nullptr;
        p->val_buf = nullptr;
        p->idx_cap = 0;
        CUDA_TRY(dalloc(&p->idx_buf, 2 * count));
        CUDA_TRY(dalloc(&p->val_buf, count));
        p->idx_cap = count;
    }
    CUDA_TRY(cudaMemcpyAsync(p->idx_buf, d, sizeof(int64_t) * size_t(count), cudaMemcpyHostToDevice, p->stream));
    CUDA_TRY(cudaMemcpyAsync(p->idx_buf + count, i, sizeof(int64_t) * size_t(count), cudaMemcpyHostToDevice, p->stream));
    CUDA_TRY(launch_poisson_weights(*p, p->idx_buf, p->idx_buf + count, count, p->val_buf));
    CUDA_TRY(cudaMemcpyAsync(out_host, p->val_buf, sizeof(double) * size_t(count), cudaMemcpyDeviceToHost, p->stream));
    CUDA_TRY(cudaStreamSynchronize(p->stream));
    return TOMO_OK;
}

tomo_status tomo_bands(tomo_plan_t plan, int64_t *lo_host, int64_t *hi_host)
{
    Plan *p = reinterpret_cast<Plan *>(plan);
    if (!p || !lo_host || !hi_host) return fail(TOMO_EINVAL, "NULL argument");
    int32_t *tmp = new (std::nothrow) int32_t[size_t(2 * p->D)];
    if (!tmp) return fail(TOMO_ENOMEM, "host allocation failed");
    cudaError_t e1 = cudaMemcpyAsync(tmp, p->lo, sizeof(int32_t) * size_t(p->D), cudaMemcpyDeviceToHost, p->stream);
    cudaError_t e2 = cudaMemcpyAsync(tmp + p->D, p->hi, sizeof(int32_t) * size_t(p->D), cudaMemcpyDeviceToHost, p->stream);
    cudaError_t e3 = cudaStreamSynchronize(p->stream);
    if (e1 != cudaSuccess || e2 != cudaSuccess || e3 != cudaSuccess) {
        delete[] tmp;
        return fail(TOMO_ECUDA, "copy of the bands failed");
    }
    for (int64_t k = 0; k < p->D; ++k) {
        lo_host[k] = tmp[k];
        hi_host[k] = tmp[p->D + k];
    }
    delete[] tmp;
    return TOMO_OK;
}

}  // extern "C"
