// tomo_internal.cuh -- internal declarations shared by the CUDA translation
// units of libtomo (plan kernels, band contractions, row kernels, host API).
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/tomo.h"

namespace tomo {

// ---------------------------------------------------------------------------
// Geometry of the band contraction tiles.
//   Forward  O = F X   : tiles of TILE_R probes x BN columns, reduced over the
//                        union band of the tile's probes (photon numbers).
//   Adjoint  Z = F^T Y : tiles of TILE_R photon numbers x BN columns, reduced
//                        over the probes whose band meets the tile.
// The reduction range of every tile is cut into work units (split-K) planned
// on the host.  Poisson weights are generated in runs of RUN consecutive
// photon numbers from an anchor stored every RUN photon numbers (plan.cu).
// ---------------------------------------------------------------------------
constexpr int RUN = 8;
constexpr int TILE_R = 128;
constexpr int GEMM_THREADS = 256;
constexpr int TC_MAX_UNIT = 4096;         // longest reduction range of a tensor-core work unit (split schedules)
constexpr int ROW_WARPS = 8;              // warps per CTA in row kernels
constexpr int MAX_N = 1024;               // outcomes supported by row kernels
constexpr int RED_SLOTS = 4;              // partial-sum slots per reduction

// Device-resident scalars of the solver.  Written by the last CTA of the
// kernel that produces them (no host round trip between kernels).
struct DevScalars {
    // CG
    double rz, rr, pq, alpha, beta, bn, tol;
    int32_t cg_active, cg_iters, max_cg, pad0;
    // Newton iteration set-up
    double kkt2, w2, eps, gdir;
    int32_t use_grad_dir, pad1;
    // line search
    double alpha_ls, gts, reg, dres, f_trial;
    int32_t neg, accept, ls_go, tc_err;
    // objective pieces
    double res2, regval, nonfinite;
    // counters for the last-block reductions (one per concurrent site)
    unsigned int ticket[4];
};

// One CTA of a band contraction: reduction range [k0, k1) of tile `tile`,
// chunk index `chunk` among the tile's units.
struct WorkUnit {
    int32_t tile, chunk, k0, k1;
};

// Work-unit schedule of one contraction (direction x arithmetic type).
struct Schedule {
    WorkUnit *units;        // device, n_units
    int32_t *tile_first;    // device, per tile: first partial slot
    int32_t *tile_nsplit;   // device, per tile: number of units
    unsigned int *counters; // device, per (tile, column block)
    void *part;             // device partial tiles
    int n_units;
    // tensor-core schedules: CTA c runs units cta_first[c] .. cta_first[c+1]-1
    int32_t *cta_first;     // device, n_ctas + 1 (null for the SIMT schedules)
    int n_ctas;
};

struct Plan {
    int64_t M, N, D;
    double gamma, band_k;
    int precision;
    bool cg_f32;       // CG vectors x, r, z, p, u, q held as float (tensor-core form)
    cudaStream_t stream;
    bool own_stream;
    int device;
    int num_sms;
    // schedule density of the band contractions: SIMT units per SM and
    // column block, tensor-core persistent CTAs per column block (0: one per
    // SM); chosen by the plan-time autotuner when asked
    int ups_simt;
    int tc_ctas;
    int tuned;            // 1: the autotuner chose the density (timed or cached)
    int tuned_cached;     // 1: taken from the per-process cache
    double tuned_ms;      // Hessian-product time of the chosen density

    // problem tables (device)
    double *lam;       // D
    int32_t *lo, *hi;  // D, inclusive band; empty band: lo = M, hi = M - 1
    int64_t *aoff;     // D + 1 offsets into the anchor table
    double *anchor;    // F_{d, a0_d + RUN j}, a0_d = lo_d rounded down to RUN
    float *anchor_f;   // same, rounded to float
    double *ratio_inv; // M + RUN + 1: 1/i for i >= 1 (ratio_inv[0] unused)
    float2 *ratio_inv_f2;  // 1/i as an unevaluated float sum hi + lo
    float2 *lam_f2;        // lambda_d as hi + lo floats
    int32_t *fwd_klo, *fwd_khi;  // per forward tile (probes)
    int32_t *adj_dlo, *adj_dhi;  // per adjoint tile (photon numbers)
    double *h;         // M: Hessian diagonal
    float *hinv_f;     // 2 M: float 1/h and 1/(2h) (stage-1 and stage-2 preconditioners)
    int64_t n_anchor;
    int fwd_tiles, adj_tiles;
    Schedule sched[2][2];      // [forward, adjoint][float, double]
    Schedule sched_tc[2];      // tensor-core contractions [forward, adjoint]
    // transposed bf16 hi/lo copies of the tensor-core operands and their
    // tensor maps (TMA boxes of 64 x BN, 128-byte swizzle)
    __nv_bfloat16 *ut_hi, *ut_lo, *ot_hi, *ot_lo;
    int64_t ut_pitch, ot_pitch;
    CUtensorMap tm_ut_hi, tm_ut_lo, tm_ot_hi, tm_ot_lo;

    // solver execution: a plan-owned non-blocking work stream fenced against
    // the caller's stream, and CUDA graphs of the CG chunk per (stage, profile)
    cudaStream_t work;
    cudaEvent_t ev_in, ev_out;
    cudaGraphExec_t cg_exec[2][2];
    int cg_exec_kernels[2][2];
    int cg_direct_runs[2][2];
    cudaEvent_t prof_ev[4][3];
    bool prof_ev_ready;

    // workspaces (device), M x N unless noted
    double *Th, *trial, *s, *G, *g, *x, *r, *z, *p, *u, *q, *dir;
    double *R, *Rt, *O;      // D x N
    double *Pbuf;            // D x N staging of a host P
    double *Xbuf;            // M x N staging of host Theta / grad
    uint8_t *freem, *var;    // M x N masks
    int32_t *mrow;           // M
    double *partials;        // RED_SLOTS x max_partials
    int64_t max_partials;
    DevScalars *sc;          // device scalars
    DevScalars *sc_host;     // pinned mirror
    double *scratch_host;    // pinned host scratch (small)
    int64_t *idx_buf;        // scratch for tomo_poisson_weights
    double *val_buf;
    int64_t idx_cap;
};

// ------------------------------- launchers ---------------------------------
// plan.cu
cudaError_t launch_plan_tables(Plan &p);
cudaError_t launch_hess_diag(Plan &p);
cudaError_t launch_poisson_weights(Plan &p, const int64_t *d, const int64_t *i,
                                   int64_t count, double *out);

// band_gemm.cu
enum FwdMode { FWD_STORE = 0, FWD_RESID = 1, FWD_DELTA = 2 };
enum AdjMode { ADJ_STORE = 0, ADJ_GRAD = 1, ADJ_HESS = 2 };
// O = F X (mode STORE); R = F X - P with sum R^2 (RESID); Rt = R + F X with
// sum (2 R . FX + FX^2) (DELTA).  `prec` selects double or float arithmetic.
cudaError_t launch_forward(Plan &p, int prec, FwdMode mode, const double *X, double *out,
                           const double *P_or_R, bool gated);
cudaError_t launch_forward_gated_ls(Plan &p, int prec, FwdMode mode, const double *X, double *out,
                                   const double *P_or_R);
// Z = F^T Y (STORE); G = 2 F^T Y + 2 gamma L Xreg (GRAD / HESS: same formula,
// HESS is gated by the CG-active flag).
cudaError_t launch_adjoint(Plan &p, int prec, AdjMode mode, const double *Y, double *out,
                           const double *Xreg, bool gated);

// rowops.cu
cudaError_t launch_fill(Plan &p, double *x, double v, int64_t n);
cudaError_t launch_regulariser(Plan &p, const double *X);   // -> sc->regval
cudaError_t launch_project_rows(Plan &p, const double *X, double *Y);
// X_{i,n} < rel * max_n X_{i,n} -> 0, then each row rescaled to sum 1 (in place)
cudaError_t launch_zero_small_rows(Plan &p, double *X, double rel);
cudaError_t launch_kkt(Plan &p, const double *Th, const double *G);  // -> sc->kkt2
cudaError_t launch_setup1(Plan &p, int stage, double eps_bar);  // kkt2, w2, eps, g, var, mrow
cudaError_t launch_setup2(Plan &p, int stage, int max_cg, double eta_max, double eta_pow);  // I mask, CG start
cudaError_t launch_cg_restrict(Plan &p, int stage);
cudaError_t launch_cg_update_xr(Plan &p, int stage);
cudaError_t launch_cg_update_p(Plan &p, int stage);
cudaError_t launch_direction(Plan &p, int stage);
cudaError_t launch_trial(Plan &p, int stage, double alpha, bool delta_mode);
cudaError_t launch_set_grad_dir(Plan &p);
// smooth.cu
cudaError_t launch_smooth(Plan &p, const double *X, double *Y, int64_t exclude, double div);
cudaError_t launch_infidelity(Plan &p, const double *A, const double *B, double *out_dev);
cudaError_t launch_nonfinite_check(Plan &p, const double *x, int64_t n, int slot);

int band_bn(int64_t N);
template <typename T> size_t band_smem_bytes(int bn);

// arithmetic of the CG Hessian products / line-search products, and of the
// gradient, for a plan precision
inline int prec_products(int precision) { return precision == TOMO_PREC_FP64 ? TOMO_PREC_FP64 : TOMO_PREC_FP32; }
inline int prec_gradient(int precision)
{
    return (precision == TOMO_PREC_FP32 || precision == TOMO_PREC_TC) ? TOMO_PREC_FP32 : TOMO_PREC_FP64;
}
inline bool hvp_on_tensor_cores(int precision) { return precision == TOMO_PREC_TC; }

// tc_band.cu
// V, HV: float when vec_f32 (the CG vectors of the tensor-core form), else double
// restrict_stage 1 or 2 also applies the CG restriction of that stage to HV
// and finishes p^T q and alpha (float vectors, when tc_restrict_fusable)
// split_input = false: the transposed bf16 mirror of V is already current
// (written by launch_cg_update_p_split or launch_tc_split_input)
cudaError_t launch_hvp_tc(Plan &p, const void *V, void *HV, bool vec_f32, bool gated, int restrict_stage = 0,
                          bool split_input = true);
bool tc_restrict_fusable(const Plan &p);
// the transposed bf16 hi/lo mirror of a product input V (M x N, float or double)
cudaError_t launch_tc_split_input(Plan &p, const void *V, bool vec_f32, bool gated);
// CG direction update p = z + beta p (and u = E p in stage 2) fused with the
// mirror of the next product's input; float CG vectors, N <= 128, N % 4 == 0
bool tc_update_p_fusable(const Plan &p);
cudaError_t launch_cg_update_p_split(Plan &p, int stage);
cudaError_t launch_hvp_tc_wait_selftest(Plan &p, const double *V, double *HV);
size_t tc_smem_bytes(int bn);
// tensor map of a transposed bf16 operand copy (rows x pitch, box 64 x bn)
cudaError_t encode_operand_map(CUtensorMap *map, const void *base, int64_t pitch, int64_t rows, int bn);

// warmstart.cu: shape of a warm-start handle (false for NULL)
bool ws_shape(const void *handle, int64_t *D, int64_t *M, int64_t *C0);

// records a failure message for tomo_last_error (api.cu)
tomo_status tomo_set_error(tomo_status s, const char *msg);

// kernel launch accounting (all threads)
void count_launch(int n = 1);


}  // namespace tomo
