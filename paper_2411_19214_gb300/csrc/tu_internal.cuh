// tu_internal.cuh -- internal declarations shared by the translation units of
// libtu_ipfp.so: the market object, the per-row scaling update, and the inline
// PTX wrappers (mbarrier, TMA, tcgen05) used by the sm_103a kernels.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>
#include <string>
#include <utility>
#include <vector>

#include "../../include/tu_ipfp.h"

// ---------------------------------------------------------------------------
// Sizes shared by host and device code
// ---------------------------------------------------------------------------
namespace tu {

constexpr int kFusedOwnRows = 256;      // own-side rows per CTA tile (two 128-row MMAs)
constexpr int kFusedPartnerRows = 128;  // partner rows per pipeline stage (MMA N)
constexpr int kKBlock = 64;             // bf16 elements per 128-byte swizzle row
constexpr int kRowPad = 256;            // every per-side vector is padded to this multiple
constexpr int kMaxPartials = 4096;      // per-CTA FP64 partials per half-sweep

// results[] slots (FP64, device), written by the finalize kernels
enum : int {
  kResXInf = 0,   // max_x |r_x| / n_x of the state entering the X half-sweep
  kResXL1 = 1,    // sum_x |r_x|
  kResXSq = 2,    // sum_x u_x^2 after the X half-sweep
  kResYSq = 3,    // sum_y v_y^2 after the Y half-sweep
  kResNonfin = 4, // count of non-finite potentials written
  kResSlots = 8
};

// Per-market FP64 scalars on the device (tu_market::st), kept up to date by
// the preparation and finalize kernels of every half-sweep, so that no O(N)
// pass is needed to prepare a half-sweep or to take the translation step.
// Side s: 0 = X, 1 = Y.
enum : int {
  kStLmax = 0,     // [2] max over the side of its stored ell
  kStLogS = 2,     // [2] log sum e^{2 log u} over the side's true potentials
  kStOff = 4,      // [2] true log u = stored log u + offset (a translation not yet written to the arrays)
  kStTauNext = 6,  // the translation step for the next half-sweep of a sweep
  kStTauUsed = 7,  // the translation step the current half-sweep's preparation applied
  kStShift = 8,    // the current half-sweep's partner shift: lmax + offset + tau (natural log)
  kStOwnOff = 9,   // the current half-sweep's own-side offset: offset - tau
  kStSlots = 16
};

// Per-32-row group of a side (Side::grp, a float4): max 2 log u, sum of
// e^{2 log u - max}, max ell; written by the side's own half-sweep.
constexpr int kGroupRows = 32;
constexpr int kMaxSplit = 8;  // partner ranges per own tile (tu_market_set_split)

// Residual of the state entering an X half-sweep (the pass's `residual`):
// none, an estimate with FP32 terms (inside sweeps) or exact FP64 terms
// (certifying passes).
enum : int { kResidualNone = 0, kResidualEstimate = 1, kResidualExact = 2 };

// device error word codes (first error wins)
enum : int { kErrNone = 0, kErrTimeout = 1, kErrNonfinite = 2 };

struct Side {
  int64_t rows = 0;      // users on this side
  int64_t rows_pad = 0;  // rows rounded up to kRowPad
  double* log_u = nullptr;  // log u (side X) or log v (side Y), rows_pad (FP64 state)
  double* ell = nullptr;    // log u + b / (2 sigma), rows_pad (FP64 state)
  float* b2s = nullptr;     // b / (2 sigma), rows_pad, or nullptr without bias
  double* mass = nullptr;   // capacities, rows_pad (padding 1)
  float* pvec = nullptr;    // this side's potentials prepared for the other side's half-sweep, rows_pad
  float4* grp = nullptr;    // per-32-row groups {max 2 log u, scaled sum, max ell, 0}, rows_pad / 32 + 2 kMaxPartials
  double sum_mass = 0.0;    // host copy of sum of capacities
  __nv_bfloat16* fac16 = nullptr;  // packed [F | K] (or [G | L]) rows x kp, bf16, zero padded
  uint8_t* fac8 = nullptr;         // FP8 markets: packed rows x kp e4m3 of [F | K] / fs (zero padded)
  float* fs = nullptr;             // FP8 markets: per-row scales, rows_pad (padding 1)
  uint8_t* fold = nullptr;         // BF16 fused markets, kp = 64: this side's g / c as the K = 16 operand of
                                   // the partner tiles' extra MMA (rows_pad x 32 bytes, tcgen05 layout)
  int fp8_exp = 0;                 // FP8 markets with one scale per side: its exponent (fs = 2^fp8_exp)
  float* fac32 = nullptr;          // packed rows x kp, fp32 (dense path), zero padded
  CUtensorMap tm_own;       // TMA map, box kKBlock x kFusedOwnRows
  CUtensorMap tm_partner;   // TMA map, box kKBlock x kFusedPartnerRows
};

// Over-relaxation controller of the solve loops (host side, one per market).
// Plain sweeps until the residual is below 0.1 and (in automatic mode) the
// per-sweep decay q of the plain iteration has settled, then the fixed factor,
// or in automatic mode omega = 2 / (1 + sqrt(1 - q)) (successive
// over-relaxation) tapered towards 1 over the last decade above tol (the
// relaxed sweep amplifies the FP32 rounding of the row sums by about
// omega / (2 - omega)). In both modes the excess over 1 is halved whenever the
// residual grows tenfold over the best seen.
struct RelaxControl {
  static constexpr int kProbe = 10;  // sweeps between convergence-rate estimates
  double cfg = 1.0;                  // 1: plain; (1, 2): fixed; 0: automatic
  double omega = 1.0, target = 1.0, best = 1.0 / 0.0, q_prev = -1.0;
  int last_est = 0;
  std::vector<std::pair<int, double>> hist;

  explicit RelaxControl(double c = 1.0) : cfg(c) {}
  bool enabled() const { return cfg != 1.0; }

  // r: residual of the state entering the last sweep of a block that ended
  // after `done` sweeps (r > tol). Returns the omega of the next block.
  double observe(int done, double r, double tol);
};

// e4m3 markets (per-row or per-side scales)
inline bool is_fp8(int dtype) { return dtype == TU_DTYPE_FP8E4M3 || dtype == TU_DTYPE_FP8E4M3_SIDE; }

// The library's kernels are built for sm_103a only (compute capability 10.3):
// any other device would fail at the first launch ("no kernel image").
inline bool device_supported(int dev) {
  int major = 0, minor = 0;
  if (cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return major == 10 && minor == 3;
}

// Sweeps in the next block of a solve loop (the residual is read back between
// blocks). The first block is one sweep; each later one is at most twice the
// previous block, cut to the sweeps the per-sweep decay measured over the last
// block needs to take the residual to tol, and at most `cap`. r_prev and r are
// the residuals read after the last two blocks (r_prev < 0: none yet), last_k
// the sweeps of the last block (0: none yet).
inline int plan_block(int last_k, double r_prev, double r, double tol, int cap) {
  int k = last_k <= 0 ? 1 : 2 * last_k;
  if (last_k > 0 && r_prev > 0.0 && r > tol && r < r_prev && tol > 0.0) {
    const double log_q = std::log(r / r_prev) / (double)last_k;
    const double need = std::ceil(std::log(tol / r) / log_q);
    if (need >= 1.0 && need < (double)k) k = (int)need;
  }
  if (k > cap) k = cap;
  return k < 1 ? 1 : k;
}

}  // namespace tu

struct tu_market {
  int64_t N = 0, M = 0, d = 0;
  int64_t kp = 0;           // packed row length in elements: fused BF16 64, 128 or 256, FP8 128, 256
                            // or 512 bytes (fused_row_length); dense FP32 2d rounded up to 64
  bool fp8_caller_scales = false;  // FP8 created from caller e4m3 bytes and per-row scales
  float cmul = 0.0f;        // fused path: log2(e) / (2 sigma), times 2^(k_X + k_Y) for FP8 markets
  int dtype = 0, path = 0;
  double sigma = 1.0;
  int64_t partition = 0;
  cudaStream_t stream = nullptr;
  int device = 0;
  int num_sms = 0;
  tu::Side X, Y;
  float* Ahat = nullptr;     // dense path: N x ldA fp32
  int64_t ldA = 0;
  double* partials = nullptr;   // kMaxPartials x 4 doubles
  double* st = nullptr;          // device scalars (kSt*): shifts, sums, offsets and steps of both sides
  float* AhatT = nullptr;       // dense path: transpose of A-hat, M x ldN fp32
  int64_t ldN = 0;
  double* results = nullptr;       // device, kResSlots
  double* results_host = nullptr;  // pinned, kResSlots
  int* err_dev = nullptr;          // device error word
  int* err_host = nullptr;         // pinned
  void* staging = nullptr;         // device staging buffer for host-memory arguments
  size_t staging_bytes = 0;
  void* aux = nullptr;             // ranked-list hand-over scratch (grow-only)
  size_t aux_bytes = 0;
  cudaGraphExec_t graph = nullptr; // captured block of sweeps
  int graph_sweeps = 0;
  bool use_graphs = true;          // tu_market_use_graphs
  int small_mode = 1;              // tu_market_set_small_tiles: 0 256-row own tiles, 1 128-row when they
                                   // fit one wave, 2 always 128-row
  int split = 1;                   // tu_market_set_split: partner ranges per own tile (fused sweeps)
  bool split_blocks = false;       // tu_market_set_partner_blocks: the ranges run one after another
  int64_t l2_bytes = 0;            // the device's L2 size (partner tiles: evict-last / evict-first policy)
  float4* split_part = nullptr;    // split > 1: partial row sums, split x max(N, M)
  int* split_cnt = nullptr;        // split > 1: arrivals per (own tile, 32-row block), zeroed
  int split_cap = 0;               // the split the buffers were sized for
  bool translate = true;           // tu_market_set_translation: translation step before every half-sweep
  bool wide = false;               // factor range beyond one shift per half-sweep: per-row running maxima
  bool poisoned = false;
  std::string last_error;
  // benchmark timing (tu_profile_enable / tu_profile_read)
  // over-relaxation: device scalar read by every pass (graphs stay valid when it changes)
  double* omega_dev = nullptr;
  double* omega_host = nullptr;  // pinned staging for updates of omega_dev
  double omega_cfg = 1.0;        // 1: plain IPFP; (1, 2): fixed; 0: automatic in tu_ipfp_solve
  // serving: completion of the last asynchronous tu_ipfp_sweep (tu_market_query)
  cudaEvent_t done_ev = nullptr;
  double* query_host = nullptr;  // pinned: kResSlots doubles + the error word
  int64_t sweeps_enqueued = 0;
  int64_t query_sweeps = 0;
  // automatic relaxation of asynchronous sweeps (tu_market_relax_update)
  tu::RelaxControl relax;
  int64_t relax_base = 0;   // sweeps_enqueued when the controller was last reset
  int64_t relax_seen = -1;  // query_sweeps last fed to the controller
  bool profiling = false;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev_pool;
  size_t ev_used = 0;
};

// ---------------------------------------------------------------------------
// Launchers (one translation unit each); all return cudaGetLastError().
// ---------------------------------------------------------------------------
namespace tu {

// reduce.cu
// Prepare the partner's FP32 vector for a half-sweep of the other side and the
// pass's scalars (with translate, the translation step taken before it).
cudaError_t launch_prep(tu_market* m, Side& partner, int fused_mode, int translate);
// Reduce a pass's partials; after an update, also the own side's groups into
// the market scalars (ngroups: groups the pass wrote).
cudaError_t launch_finalize(tu_market* m, int nparts, int is_x, int residual, int update, int64_t ngroups);
// Groups and scalars of both sides from their stored potentials (after the
// potentials were set from outside a sweep).
cudaError_t launch_rescan(tu_market* m);
// Write the sides' pending offsets into their arrays (end of a block of sweeps).
cudaError_t launch_flush(tu_market* m);
cudaError_t launch_pack_factors(tu_market* m, Side& s, const void* A, const void* B, int src_dtype);
cudaError_t launch_init_side(tu_market* m, Side& s, const float* bias_dev, int has_bias);
cudaError_t launch_reset_potentials(tu_market* m, Side& s);
cudaError_t launch_set_potentials(tu_market* m, Side& s, const float* log_u_dev);
cudaError_t launch_set_potentials64(tu_market* m, Side& s, const double* log_u_dev);
cudaError_t launch_get_potentials(tu_market* m, Side& s, float* out_dev);  // FP64 state -> FP32
cudaError_t launch_row_norms(tu_market* m, Side& s, float* out_max);
// FP8 markets: max |entry| of the FP32 factor pair (A, B: rows x d each) into *out_max
cudaError_t launch_max_abs(tu_market* m, const float* A, const float* B, int64_t count, float* out_max);
// FP8 markets: pack [A | B | 0] * 2^-k into s.fac8 (rows x 128 e4m3, round to nearest even, saturating)
constexpr int kPerRowScale = -1000000;  // launch_pack_fp8_rows: each row its own scale
cudaError_t launch_pack_fp8_rows(tu_market* m, Side& s, const float* A, const float* B, int side_k,
                                 unsigned int* bad);
cudaError_t launch_pack_fp8_bytes(tu_market* m, Side& s, const uint8_t* A, const uint8_t* B, const float* sc,
                                  unsigned int* bad);
cudaError_t launch_sum_sq(tu_market* m, Side& s, int is_x);  // results[kResXSq or kResYSq] = sum exp(2 log u)

// dense.cu
cudaError_t launch_dense_build(tu_market* m);
cudaError_t launch_dense_rowpass(tu_market* m, int residual, int update, int* nparts_out, int64_t* ngroups_out);
cudaError_t launch_dense_colpass(tu_market* m, int update, int* nparts_out, int64_t* ngroups_out);

// fused.cu
cudaError_t fused_prepare(tu_market* m);  // tensor maps + kernel attributes
// The whole own side (nrows < 0), or own users [row0, row0 + nrows) only (no groups written).
cudaError_t launch_fused_halfsweep(tu_market* m, int side, int residual, int update, int* nparts_out,
                                   int64_t row0 = 0, int64_t nrows = -1);

// The fused half-sweep on caller-described device buffers (no market object).
struct FusedRaw {
  const __nv_bfloat16* own16;  // rows x kp packed own factors
  int64_t rows;
  const __nv_bfloat16* par16;  // cols x kp packed partner factors
  int64_t cols;
  int64_t kp;                  // 64 or 128
  double sigma;
  const float* g;              // prepared partner vector, >= ceil(cols / 128) * 128, -inf padded
  const double* lmax;          // partner shift
  const float* b2s;            // own bias / (2 sigma) or nullptr
  const double* mass;          // own capacities
  double* log_u;               // own log u (in: old, out: new)
  double* ell;                 // own ell (out)
  double* partials;            // >= min(ceil(rows / 256), num_sms) x 4
  int* err;
  int residual;
};
cudaError_t launch_fused_halfsweep_raw(const FusedRaw& r, cudaStream_t stream, int num_sms, int* nparts_out);

// One market of a batched launch, for the half-sweep that updates its "own"
// side against its "partner" side (device copy; the tensor maps keep their
// 128-byte alignment, so an array of these is a valid TMA operand array).
// Two per market: X against Y and Y against X.
struct BatchDesc {
  CUtensorMap tm_own;          // own packed factors, box kKBlock x kFusedOwnRows
  CUtensorMap tm_partner;      // partner packed factors, box kKBlock x kFusedPartnerRows
  const float* b2s;            // own bias / (2 sigma) or nullptr
  const double* mass;          // own capacities
  double* log_u;               // own potentials (in: old, out: new)
  double* ell;                 // own ell (out)
  const double* partner_ell;   // partner ell (read by the preparation kernel)
  float* g;                    // partner prepared vector (written by the preparation kernel)
  uint8_t* gfold;              // BF16, kp = 64: the partner's g / c operand of the extra MMA (written by the
                               // preparation kernel), else nullptr
  double* st;                  // the market's scalars (kSt*; shift and own offset of the pass)
  const float* fs_own;         // e4m3 markets: own per-row scales, else nullptr
  const float* fs_par;         // e4m3 markets: partner per-row scales, else nullptr
  float4* grp;                 // own-side groups (written by the pass, reduced by the finalize)
  const double* omega;         // over-relaxation factor of this market (device scalar)
  double dm_next;              // sum of own capacities - sum of partner capacities (the next step's tau)
  int own_side;                // 0: X is own, 1: Y is own
  int translate;               // the market's translation-step setting at batch creation
  int64_t rows;                // own users
  int64_t partner_rows;        // partner users
  int64_t partner_rows_pad;    // partner vector length (multiple of kRowPad)
  int num_own_tiles;           // ceil(rows / kFusedOwnRows)
  int num_partner_tiles;       // ceil(partner_rows / kFusedPartnerRows)
  int slot0;                   // first own-tile slot of this market in the partials array
  float c;                     // log2(e) / (2 sigma)
};

// Epilogue warps that write per-tile partials in a batched launch (the warps
// that own the row updates); each own tile has kBatchSlotWarps x 4 doubles.
constexpr int kBatchSlotWarps = 8;

// A batched half-sweep: the CTA b processes items[cta_start[b] .. cta_start[b + 1])
// in order, an item being (market, own tile).
struct BatchLaunch {
  const BatchDesc* desc;   // device, indexed by market
  const int2* items;       // device
  const int* cta_start;    // device, grid + 1 entries
  double* partials;        // device, [slot][kBatchSlotWarps][4]
  int* err;
  int grid;
  int64_t kp;              // 64 or 128 (BF16), the same for every market
  int dtype;               // the members' dtype (e4m3 markets: kp = 128 bytes per row, the same format)
  int residual;
  int update;
};
cudaError_t launch_fused_batch(const BatchLaunch& b, cudaStream_t stream);
// ranked lists / mu block through the tensor-core pipeline (partner vector prepared in log2 mode)
cudaError_t launch_fused_topk(tu_market* m, int side, int k, int64_t row0, int64_t nrows, int32_t* idx, float* logmu,
                              float* hand_v, int32_t* hand_i);
cudaError_t launch_fused_mu(tu_market* m, int64_t x0, int64_t nx, int64_t y0, int64_t ny, float* out, int64_t ld);

// topk.cu (dense-path outputs, read from A-hat)
cudaError_t launch_mu_block(tu_market* m, int64_t x0, int64_t nx, int64_t y0, int64_t ny, float* out,
                            int64_t ld);
cudaError_t launch_topk(tu_market* m, int side, int k, int64_t row0, int64_t nrows, int32_t* idx,
                        float* logmu);



}  // namespace tu

// ---------------------------------------------------------------------------
// Device helpers
// ---------------------------------------------------------------------------
#ifdef __CUDACC__
namespace tu {

constexpr double kLnHalf = -0.69314718055994530942;
constexpr float kLog2e = 1.4426950408889634f;

struct RowResult {
  double log_u, ell;
  double r_rel, r_abs, u2;
};

// ln (a + b + c) of a positive row sum given as three FP32 parts, to an
// absolute error of about 6e-8 whatever the size of the sum. The parts are
// added in FP32 with the rounding error of each addition kept (Knuth's
// two-sum), x = hi + lo; hi = m 2^e with m in [0.5, 1), so
// ln x = e ln 2 + ln m + lo / hi, and |ln m| < 0.7 keeps logf's rounding small.
// (logf(x) itself rounds to half an FP32 ulp of ln x: 4.8e-7 for the sums of
// ~1e6 terms of a large market, ln x ~ 14, which would put a floor of ~1e-6
// under the residual.)
__device__ __forceinline__ float two_sum(float a, float b, float& err) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  err = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return s;
}
__device__ __forceinline__ double log_row_sum(float a, float b, float c) {
  float e1, e2;
  const float s1 = two_sum(a, b, e1);
  const float hi = two_sum(s1, c, e2);
  const float lo = __fadd_rn(e1, e2);
  int ex;
  const float m = frexpf(hi, &ex);
  return __dadd_rn((double)ex * 0.69314718055994530942, (double)__fadd_rn(logf(m), __fdividef(lo, hi)));
}

// The closed-form update of Eq. iteration for one user, in logs.
//   ln_sum   : log of sum_y exp(phi_hat_xy / (2 sigma) + ell_y - shift)
//   shift    : the partner-side shift (max_y ell_y) taken out of the sum
//   b2s      : this user's bias / (2 sigma)
//   log_s    = log(1/2) + b2s + shift + ln_sum          (s = 1/2 sum_y A_xy v_y)
//   log u    = 1/2 log n - asinh(exp(log s - 1/2 log n)) (= sqrt(n + s^2) - s)
// With residual, r = u_old^2 + 2 u_old s - n is the row equation of Eq. IPFP
// evaluated at the state entering the half-sweep.
//
// Precision: the sums are FP32, so the transcendentals of the update are
// evaluated in FP32 (FP64 transcendentals are slow on this part) while the
// additions whose operands may be large and cancel (log s, log u, ell: |.| up
// to ~100 with popularity biases) stay in FP64. For z = log s - 1/2 log n > 0,
// asinh(e^z) = z + c(z) with c(z) = log1p(sqrt(1 + e^{-2z})) in (ln 2, 0.89],
// so only the bounded correction c is rounded to FP32 (absolute error ~1e-7).
// The residual r = u^2 + 2 u s - n (residual = kResidualExact) is formed from
// FP64 exponentials of the FP64 state, so a certified residual carries no FP32
// rounding; inside sweeps (kResidualEstimate), where it only decides when to
// certify, its terms are FP32 exponentials (absolute error ~2e-7 of n), which
// keeps two FP64 exponentials per row out of the half-sweep (FP64 throughput
// is a small fraction of FP32 on this part). The u^2 summed for the match
// count (sum n - sum u^2, where sum u^2 is a small part) is FP32.
//
// omega != 1 over-relaxes the update in the log domain:
// log u <- log u_old + omega * (update - log u_old) (same fixed point).
__device__ __forceinline__ RowResult row_update(double ln_sum, double shift, float b2s, double mass,
                                                double log_u_old, int residual, double omega = 1.0) {
  RowResult o;
  const double log_s = kLnHalf + (double)b2s + shift + ln_sum;
  o.r_rel = 0.0;
  o.r_abs = 0.0;
  if (residual == kResidualExact) {
    // r = u^2 + 2 u s - n with u^2 = e^{2 log u}, 2 u s = e^{log u + log s + ln 2}
    const double r = exp(2.0 * log_u_old) + exp(log_u_old + log_s + 0.69314718055994530942) - mass;
    o.r_abs = fabs(r);
    o.r_rel = fabs(r) / mass;
  } else if (residual == kResidualEstimate) {
    const double r = (double)expf((float)(2.0 * log_u_old)) +
                     (double)expf((float)(log_u_old + log_s + 0.69314718055994530942)) - mass;
    o.r_abs = fabs(r);
    o.r_rel = fabs(r) / mass;
  }
  const double hl = 0.5 * (double)logf((float)mass);
  const double z = log_s - hl;
  double a;
  if (z > 0.0) {
    const float c = log1pf(sqrtf(1.0f + expf((float)(-2.0 * z))));
    a = z + (double)c;
  } else {
    a = (double)asinhf(expf((float)z));
  }
  const double lu_upd = hl - a;
  const double lu = omega == 1.0 ? lu_upd : log_u_old + omega * (lu_upd - log_u_old);
  o.log_u = lu;
  o.ell = lu + (double)b2s;
  o.u2 = (double)expf((float)(2.0 * lu));
  return o;
}

// ---- translation step and the per-side scalars -------------------------------
// The translation step moves the log potentials of the side updated last by
// +tau and those of the side about to be updated by -tau. Everything it needs
// is kept in the per-market scalars (kSt*): the sums sum e^{2 log u} of both
// sides and the sides' shifts. The half-sweep that updates a side writes one
// (max 2 log u, scaled sum, max ell) group per 32 rows; a single-block
// finalize reduces the groups in a fixed order (the single-market and the
// batched finalize run the same routine with the same block size, so the
// batch's potentials stay bit-identical to the market's own sweeps) and
// computes tau for the next half-sweep; the move itself is recorded as a
// per-side offset and written to the arrays only when a side is next updated
// (for the updated side) or at the end of a block of sweeps.

// Block-wide reductions (every thread returns the result; `red` holds
// blockDim.x / 32 doubles). Sums in a fixed order: a butterfly within each warp
// (every lane ends with the same value), then the warps in order.
__device__ __forceinline__ double block_reduce_max(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  if (threadIdx.x % 32 == 0) red[threadIdx.x / 32] = v;
  __syncthreads();
  double b = -INFINITY;
  for (int w = 0; w < (int)blockDim.x / 32; ++w) b = fmax(b, red[w]);
  __syncthreads();
  return b;
}
__device__ __forceinline__ float block_reduce_maxf(float v, float* red) {
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  if (threadIdx.x % 32 == 0) red[threadIdx.x / 32] = v;
  __syncthreads();
  float b = -INFINITY;
  for (int w = 0; w < (int)blockDim.x / 32; ++w) b = fmaxf(b, red[w]);
  __syncthreads();
  return b;
}
__device__ __forceinline__ double block_reduce_sum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v = __dadd_rn(v, __shfl_xor_sync(0xffffffffu, v, o));
  if (threadIdx.x % 32 == 0) red[threadIdx.x / 32] = v;
  __syncthreads();
  double b = 0.0;
  for (int w = 0; w < (int)blockDim.x / 32; ++w) b = __dadd_rn(b, red[w]);
  __syncthreads();
  return b;
}

// The group of one warp's 32 rows (lanes with valid = false contribute
// nothing), as {m, s, e, 0}: a reference m near the max of 2 log u (the max of
// the FP32-rounded values), the sum s of e^{2 log u - m} (the argument formed
// in FP64, the terms in FP32, summed by an FP32 butterfly whose result every
// lane shares), and e, a max of ell (of the FP32-rounded values; it serves as
// a shift, and e^{ell - shift} may exceed 1 by a rounding). Warp-collective;
// every lane returns the same group. A NaN potential makes s NaN (the
// translation step then falls back to tau = 0). One FP64 operation per row:
// FP64 throughput is a small fraction of FP32 on this part.
__device__ __forceinline__ float4 warp_group(double lu, double ell, bool valid) {
  float m = valid ? (float)(2.0 * lu) : -INFINITY;
  float e = valid ? (float)ell : -INFINITY;
  for (int o = 16; o > 0; o >>= 1) {
    m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    e = fmaxf(e, __shfl_xor_sync(0xffffffffu, e, o));
  }
  float t = (valid && m > -INFINITY) ? expf((float)__dadd_rn(2.0 * lu, -(double)m)) : 0.0f;
  if (valid && isnan(lu)) t = NAN;
  for (int o = 16; o > 0; o >>= 1) t = __fadd_rn(t, __shfl_xor_sync(0xffffffffu, t, o));
  return make_float4(m, t, e, 0.0f);
}

// The empty group (no rows).
__device__ __forceinline__ float4 empty_group() { return make_float4(-INFINITY, 0.0f, -INFINITY, 0.0f); }

// (hi, lo) += (h2, l2): an FP32 sum carried with its rounding error. The
// two-sum is error-free and symmetric in its operands, so butterfly partners
// end with the same pair.
__device__ __forceinline__ void pair_add(float& hi, float& lo, float h2, float l2) {
  float e;
  hi = two_sum(hi, h2, e);
  lo = __fadd_rn(__fadd_rn(lo, l2), e);
}

// Reduce `ng` groups in a fixed order (every thread returns the results):
// lmax = max e (the side's shift), and log sum e^{2 log u} = top + ln(hi + lo),
// where top = max m and hi + lo = sum s e^{m - top} (FP32 terms summed with
// their rounding errors kept; the logarithm is taken by the caller, once).
struct GroupTotal {
  float lmax, top, hi, lo;
};
__device__ __forceinline__ GroupTotal block_reduce_groups(const float4* __restrict__ grp, int64_t ng, float* red) {
  float mm = -INFINITY, me = -INFINITY;
  for (int64_t i = threadIdx.x; i < ng; i += blockDim.x) {
    const float4 q = grp[i];
    mm = fmaxf(mm, q.x);
    me = fmaxf(me, q.z);
  }
  GroupTotal r;
  r.top = block_reduce_maxf(mm, red);
  r.lmax = block_reduce_maxf(me, red);
  float hi = 0.0f, lo = 0.0f;
  for (int64_t i = threadIdx.x; i < ng; i += blockDim.x) {
    const float4 q = grp[i];
    if (q.x > -INFINITY || isnan(q.y)) pair_add(hi, lo, q.y * expf(q.x - r.top), 0.0f);
  }
  for (int o = 16; o > 0; o >>= 1)
    pair_add(hi, lo, __shfl_xor_sync(0xffffffffu, hi, o), __shfl_xor_sync(0xffffffffu, lo, o));
  if (threadIdx.x % 32 == 0) {
    red[2 * (threadIdx.x / 32)] = hi;
    red[2 * (threadIdx.x / 32) + 1] = lo;
  }
  __syncthreads();
  hi = 0.0f;
  lo = 0.0f;
  for (int w = 0; w < (int)blockDim.x / 32; ++w) pair_add(hi, lo, red[2 * w], red[2 * w + 1]);
  __syncthreads();
  r.hi = hi;
  r.lo = lo;
  return r;
}

// log sum e^{2 log u} of a reduced side (one thread).
__device__ __forceinline__ double group_log_sum(const GroupTotal& t) {
  return (double)t.top + log_row_sum(t.hi, t.lo, 0.0f);
}

// The translation step (an extension; Sec. 5 names acceleration from optimal
// transport as future work). IPFP is block coordinate ascent on the concave
// dual whose stationarity conditions are Eq. IPFP. Moving the partner side's
// log potentials up by tau and the own side's down by tau leaves every pair
// term A_xy u_x v_y unchanged, so along that line the dual reads
//   const + tau (sum mass_P - sum mass_O) - 1/2 e^{2 tau} P - 1/2 e^{-2 tau} O,
// P = sum_P e^{2 log p}, O = sum_O e^{2 log o}, and its maximiser is
// tau = 1/2 log z with z the positive root of P z^2 - dm z - O = 0,
// dm = sum mass_P - sum mass_O, given log_p = log P and log_o = log O.
// dm = 0: z = sqrt(O / P). Otherwise, with L = log |dm|,
// w = log(4 P O / dm^2) and q = log(1 + sqrt(1 + e^w)), the root
// z = (dm + R) / (2 P) for dm > 0 and 2 O / (R - dm) for dm < 0,
// R = sqrt(dm^2 + 4 P O) = |dm| sqrt(1 + e^w), is
// log z = L + q - log 2 - log P (dm > 0) or log 2 + log O - L - q (dm < 0),
// with no cancellation; for |w| > 60, q = w / 2 or log 2 to double precision.
// Non-finite inputs (non-finite potentials, which the half-sweep reports)
// give tau = 0.
__device__ __forceinline__ double translation_tau(double log_p, double log_o, double dm) {
  const double ln2 = 0.69314718055994530942;
  double log_z;
  if (dm == 0.0) {
    log_z = 0.5 * __dadd_rn(log_o, -log_p);
  } else {
    const double L = log(fabs(dm));
    const double w = __dadd_rn(__dadd_rn(__dadd_rn(2.0 * ln2, log_p), log_o), -2.0 * L);
    const double q = w > 60.0 ? 0.5 * w : (w < -60.0 ? ln2 : log1p(sqrt(1.0 + exp(w))));
    log_z = dm > 0.0 ? __dadd_rn(__dadd_rn(__dadd_rn(L, q), -ln2), -log_p)
                     : __dadd_rn(__dadd_rn(__dadd_rn(ln2, log_o), -L), -q);
  }
  const double tau = 0.5 * log_z;
  return isfinite(tau) ? tau : 0.0;
}

// Scalars of a half-sweep that updates side `own` (one thread, before the
// pass): the translation step it takes (tau = 0 unless `translate`), the
// partner shift the pass adds back (natural log) and the own offset under
// which it reads the entering potentials.
__device__ __forceinline__ void prep_scalars(double* st, int own, int translate) {
  const int par = 1 - own;
  const double tau = translate ? st[kStTauNext] : 0.0;
  st[kStTauUsed] = tau;
  st[kStShift] = st[kStLmax + par] + st[kStOff + par] + tau;
  st[kStOwnOff] = st[kStOff + own] - tau;
}

// Scalars after a half-sweep that updated side `own` (one thread): the own
// side's shift and sum from its groups (its arrays now hold true values), the
// step taken before the pass recorded on the partner, and tau for the next
// half-sweep, which updates the partner against this side
// (dm_next = sum mass_own - sum mass_partner).
__device__ __forceinline__ double finite_or_zero(double v) { return (v > -INFINITY && v < INFINITY) ? v : 0.0; }
__device__ __forceinline__ void finish_scalars(double* st, int own, const GroupTotal& g, double dm_next) {
  const int par = 1 - own;
  const double tau = st[kStTauUsed];
  const double log_s_own = group_log_sum(g);
  // non-finite potentials are reported by the pass (its non-finite count)
  st[kStLmax + own] = finite_or_zero((double)g.lmax);
  st[kStLogS + own] = log_s_own;
  st[kStOff + own] = 0.0;
  st[kStOff + par] += tau;
  st[kStLogS + par] += 2.0 * tau;
  st[kStTauUsed] = 0.0;
  st[kStTauNext] = translation_tau(log_s_own, st[kStLogS + par], dm_next);
}

// Scalars of both sides from their reduced groups (one thread; potentials set
// from outside a sweep): shifts, sums, no offsets, and tau for the next
// half-sweep, which updates X against Y (dm = sum m - sum n).
__device__ __forceinline__ void rescan_scalars(double* st, const GroupTotal& x, const GroupTotal& y,
                                               double dm_y_minus_x) {
  const double sx = group_log_sum(x), sy = group_log_sum(y);
  st[kStLmax + 0] = finite_or_zero((double)x.lmax);
  st[kStLmax + 1] = finite_or_zero((double)y.lmax);
  st[kStLogS + 0] = sx;
  st[kStLogS + 1] = sy;
  st[kStOff + 0] = 0.0;
  st[kStOff + 1] = 0.0;
  st[kStTauUsed] = 0.0;
  st[kStTauNext] = translation_tau(sy, sx, dm_y_minus_x);
}

__device__ __forceinline__ uint64_t global_timer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Time limit of every device-side wait. No legitimate wait in these kernels
// lasts more than microseconds; a wait that runs out sets an error word.
constexpr uint64_t kWaitLimitNs = 2000000000ull;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// ---- mbarrier --------------------------------------------------------------
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait for the phase with the given parity. Returns false when the
// time limit runs out or another role of the CTA has raised the abort flag.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, volatile int* abort_flag,
                                          uint64_t limit_ns = kWaitLimitNs) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = global_timer_ns();
  while (true) {
    if (mbar_try_wait(bar, parity)) return true;
    if (*abort_flag) return false;
    if (global_timer_ns() - t0 > limit_ns) return false;
  }
}

// Bounded wait that ignores the abort flag: used while draining after an abort,
// so that copies and MMAs already issued complete before shared memory or TMEM
// is released.
__device__ __forceinline__ bool mbar_wait_drain(uint64_t* bar, uint32_t parity, uint64_t limit_ns) {
  const uint64_t t0 = global_timer_ns();
  while (!mbar_try_wait(bar, parity)) {
    if (global_timer_ns() - t0 > limit_ns) return false;
  }
  return true;
}

// ---- TMA -------------------------------------------------------------------
__device__ __forceinline__ void tma_load_2d(void* smem_dst, const CUtensorMap* map, uint64_t* bar, int x,
                                            int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], "
      "[%2];" ::"r"(smem_u32(smem_dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(x), "r"(y)
      : "memory");
}
// The same with an L2 cache policy (createpolicy) for the loaded lines.
__device__ __forceinline__ void tma_load_2d_hint(void* smem_dst, const CUtensorMap* map, uint64_t* bar, int x, int y,
                                                 uint64_t policy) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1, {%3, "
      "%4}], [%2], %5;" ::"r"(smem_u32(smem_dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(x), "r"(y), "l"(policy)
      : "memory");
}
// L2 policy: the given fraction of the accessed lines evict last, the rest
// with their priority unchanged (evict-first would drop a line before the
// other CTAs of the same wave read it).
__device__ __forceinline__ uint64_t l2_policy_keep_fraction(float fraction) {
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_last.L2::evict_unchanged.b64 %0, %1;" : "=l"(pol) : "f"(fraction));
  return pol;
}
__device__ __forceinline__ void tma_prefetch_map(const CUtensorMap* map) {
  asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(map)) : "memory");
}
// Order earlier writes of a tensor map held in global memory before its use by TMA.
__device__ __forceinline__ void tensormap_acquire(const CUtensorMap* map) {
  asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(reinterpret_cast<uint64_t>(map))
               : "memory");
}

// ---- tcgen05 ---------------------------------------------------------------
__device__ __forceinline__ void tmem_alloc(uint32_t* smem_dst, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(smem_dst)),
               "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
// D[tmem] (+)= A[smem] * B[smem]^T, both K-major, BF16 in, FP32 accumulate.
__device__ __forceinline__ void umma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                          uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}
// D[tmem] (+)= A[smem] * B[smem]^T, both K-major, e4m3 in (32 per 32-byte K step), FP32 accumulate.
__device__ __forceinline__ void umma_e4m3(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                          uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}
// Arrive on an mbarrier once every tcgen05 operation issued so far by this thread completes.
__device__ __forceinline__ void umma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   smem_u32(bar))
               : "memory");
}

// Shared-memory matrix descriptor for a K-major tile written by TMA with
// 128-byte swizzle: rows of 128 bytes, 8-row atoms 1024 bytes apart.
//   bits  0-13 start address >> 4     bits 16-29 leading byte offset >> 4 (unused here: 1)
//   bits 32-45 stride byte offset >> 4 (1024 B)   bits 46-47 descriptor version (1)
//   bits 61-63 layout: 2 = 128-byte swizzle
// With fold (BF16 fused markets, packed rows of one k block, d <= 32): for
// every partner row i, g_i / c split into three BF16 values hi + mid + lo
// (24 significant bits; -inf padding gives hi = -inf, mid = lo = 0), written
// as the row's K = 16 operand of the fused kernel's extra MMA (columns 0-2,
// the rest zero) in the unswizzled K-major tcgen05 layout of 128-row tiles:
// byte (i / 128) * 4096 + ((i % 128) / 8) * 256 + (k / 8) * 128 + (i % 8) * 16 + (k % 8) * 2.
__device__ __forceinline__ void write_fold_row(uint4* fold, int64_t i, float g, float inv_c) {
  unsigned short b[3] = {0, 0, 0};
  if (isinf(g)) {
    b[0] = __bfloat16_as_ushort(__float2bfloat16_rn(g));
  } else {
    const float v = g * inv_c;
    const __nv_bfloat16 hi = __float2bfloat16_rn(v);
    const float r1 = v - __bfloat162float(hi);
    const __nv_bfloat16 mid = __float2bfloat16_rn(r1);
    const __nv_bfloat16 lo = __float2bfloat16_rn(r1 - __bfloat162float(mid));
    b[0] = __bfloat16_as_ushort(hi);
    b[1] = __bfloat16_as_ushort(mid);
    b[2] = __bfloat16_as_ushort(lo);
  }
  const int64_t t = i / 128, r = i % 128;
  const int64_t q = t * 256 + (r / 8) * 16 + (r % 8);  // 16-byte chunk of columns 0-7
  fold[q] = make_uint4((uint32_t)b[0] | ((uint32_t)b[1] << 16), (uint32_t)b[2], 0u, 0u);
  fold[q + 8] = make_uint4(0u, 0u, 0u, 0u);  // columns 8-15
}

// Shared-memory descriptor of an unswizzled K-major operand: core matrices of
// 8 rows x 16 bytes, `lbo` bytes apart along K and `sbo` bytes apart along
// M / N (version 1, layout type 0).
__device__ __forceinline__ uint64_t sdesc_none(uint32_t smem_addr, uint32_t lbo, uint32_t sbo) {
  uint64_t desc = 0;
  desc |= (uint64_t)((smem_addr & 0x3FFFFu) >> 4);
  desc |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  desc |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  desc |= (uint64_t)1u << 46;
  return desc;
}

__device__ __forceinline__ uint64_t sdesc_sw128(uint32_t smem_addr) {
  uint64_t desc = 0;
  desc |= (uint64_t)((smem_addr & 0x3FFFFu) >> 4);
  desc |= (uint64_t)1u << 16;
  desc |= (uint64_t)(1024u >> 4) << 32;
  desc |= (uint64_t)1u << 46;
  desc |= (uint64_t)2u << 61;
  return desc;
}

// Instruction descriptor of tcgen05.mma kind::f16: D FP32 (bits 4-5 = 1),
// A and B BF16 (bits 7-9 = 1, 10-12 = 1), both K-major (bits 15, 16 = 0),
// N >> 3 in bits 17-22, M >> 4 in bits 24-28.
__host__ __device__ constexpr uint32_t idesc_bf16_f32(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
// Instruction descriptor of tcgen05.mma kind::f8f6f4: D FP32 (bits 4-5 = 1),
// A and B e4m3 (format 0 in bits 7-9 and 10-12), both K-major, N >> 3, M >> 4.
__host__ __device__ constexpr uint32_t idesc_e4m3_f32(int M, int N) {
  return (1u << 4) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// 32 lanes x 32 columns of FP32 from TMEM (lane quadrant fixed by the warp), then wait.
__device__ __forceinline__ void tmem_ld32x32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];\n\t"
      "tcgen05.wait::ld.sync.aligned;"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
        "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
        "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
        "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr)
      : "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

__device__ __forceinline__ void named_bar_sync(int id, int nthreads) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

// Order-preserving float <-> uint mapping for atomic max on floats of any sign.
__device__ __forceinline__ unsigned int float_to_ordered(float f) {
  unsigned int u = __float_as_uint(f);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

}  // namespace tu
#endif  // __CUDACC__
