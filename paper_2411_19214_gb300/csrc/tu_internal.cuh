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
  double* lmax = nullptr;   // device scalar: max_i ell_i
  double sum_mass = 0.0;    // host copy of sum of capacities
  __nv_bfloat16* fac16 = nullptr;  // packed [F | K] (or [G | L]) rows x kp, bf16, zero padded
  uint8_t* fac8 = nullptr;         // FP8 markets: packed rows x 128 e4m3 of [F | K] * 2^-fp8_exp
  int fp8_exp = 0;                 // FP8 markets: this side's power-of-two scale k
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
  int64_t kp = 0;           // packed inner dimension: 2d rounded up to a multiple of 64 (FP8: 128)
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
  double* mpartials = nullptr;  // kMaxPartials doubles (max reduction)
  double* tau_dev = nullptr;    // device scalar: the translation step of the current half-sweep
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
  bool small_tiles = true;         // tu_market_set_small_tiles: 128-row own tiles when they fit one wave
  bool translate = true;           // tu_market_set_translation: translation step before every half-sweep
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
// Prepare the partner's FP32 vector and shift for a half-sweep of the other
// side; with translate, first apply the translation step between the two sides.
cudaError_t launch_prep(tu_market* m, Side& partner, int fused_mode, int translate);
cudaError_t launch_finalize(tu_market* m, int nparts, int is_x, int residual);
cudaError_t launch_pack_factors(tu_market* m, Side& s, const void* A, const void* B, int src_dtype);
cudaError_t launch_init_side(tu_market* m, Side& s, const float* bias_dev, int has_bias);
cudaError_t launch_reset_potentials(tu_market* m, Side& s);
cudaError_t launch_set_potentials(tu_market* m, Side& s, const float* log_u_dev);
cudaError_t launch_get_potentials(tu_market* m, Side& s, float* out_dev);  // FP64 state -> FP32
cudaError_t launch_row_norms(tu_market* m, Side& s, float* out_max);
// FP8 markets: max |entry| of the FP32 factor pair (A, B: rows x d each) into *out_max
cudaError_t launch_max_abs(tu_market* m, const float* A, const float* B, int64_t count, float* out_max);
// FP8 markets: pack [A | B | 0] * 2^-k into s.fac8 (rows x 128 e4m3, round to nearest even, saturating)
cudaError_t launch_pack_fp8(tu_market* m, Side& s, const float* A, const float* B, int k);
cudaError_t launch_sum_sq(tu_market* m, Side& s, int is_x);  // results[kResXSq or kResYSq] = sum exp(2 log u)

// dense.cu
cudaError_t launch_dense_build(tu_market* m);
cudaError_t launch_dense_rowpass(tu_market* m, int residual, int update, int* nparts_out);
cudaError_t launch_dense_colpass(tu_market* m, int update, int* nparts_out);

// fused.cu
cudaError_t fused_prepare(tu_market* m);  // tensor maps + kernel attributes
cudaError_t launch_fused_halfsweep(tu_market* m, int side, int residual, int update, int* nparts_out);

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
  double* partner_ell;         // partner ell (read, and moved by the translation step, in the preparation kernel)
  double* partner_log_u;       // partner log potentials (moved by the translation step)
  float* g;                    // partner prepared vector (written by the preparation kernel)
  double* lmax;                // partner shift (written by the preparation kernel)
  const double* omega;         // over-relaxation factor of this market (device scalar)
  double dm;                   // sum of partner capacities - sum of own capacities (translation step)
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
  int64_t kp;              // 64 or 128, the same for every market
  int fp8;                 // e4m3 factors (kp = 128 bytes per row), the same for every market
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

// ln x of a positive row sum x (FP64, formed from FP32 partial sums), to an
// absolute error of about 6e-8 whatever the size of x. x = m 2^e with m in
// [0.5, 1), so ln x = e ln 2 + ln m, and ln m is logf of m rounded to FP32 plus
// the first-order term of that rounding; |ln m| < 0.7 keeps logf's rounding
// small. (logf(x) itself rounds to half an FP32 ulp of ln x: 4.8e-7 for the
// sums of ~1e6 terms of a large market, ln x ~ 14, which would put a floor of
// ~1e-6 under the residual.)
__device__ __forceinline__ double log_row_sum(double x) {
  int e;
  const double m = frexp(x, &e);
  const float mf = (float)m;
  return (double)e * 0.69314718055994530942 + (double)logf(mf) + (double)((float)(m - (double)mf) / mf);
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
// The residual's terms (u^2 and 2 u s) are FP64 exponentials of the FP64
// state, so the reported residual carries no FP32 rounding. The u^2 summed for
// the match count (sum n - sum u^2, where sum u^2 is a small part) stays FP32.
//
// omega != 1 over-relaxes the update in the log domain:
// log u <- log u_old + omega * (update - log u_old) (same fixed point).
__device__ __forceinline__ RowResult row_update(double ln_sum, double shift, float b2s, double mass,
                                                double log_u_old, bool residual, double omega = 1.0) {
  RowResult o;
  const double log_s = kLnHalf + (double)b2s + shift + ln_sum;
  o.r_rel = 0.0;
  o.r_abs = 0.0;
  if (residual) {
    // r = u^2 + 2 u s - n with u^2 = e^{2 log u}, 2 u s = e^{log u + log s + ln 2}
    const double r = exp(2.0 * log_u_old) + exp(log_u_old + log_s + 0.69314718055994530942) - mass;
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

// ---- translation step --------------------------------------------------------
// Block size of every kernel that computes the translation step. The single-
// market preparation and the batched one run the same routine with the same
// block size, so both give the same tau bit for bit (the batch's potentials
// stay bit-identical to the market's own sweeps).
constexpr int kTauThreads = 512;

// Block-wide reductions (every thread returns the result; `red` holds
// blockDim.x / 32 doubles). Sums in a fixed order: a butterfly within each warp
// (lane 0's value is kept), then the warps in order.
__device__ __forceinline__ double block_reduce_max(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  if (threadIdx.x % 32 == 0) red[threadIdx.x / 32] = v;
  __syncthreads();
  double b = -INFINITY;
  for (int w = 0; w < (int)blockDim.x / 32; ++w) b = fmax(b, red[w]);
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

// log sum_i exp(2 x_i) over one block, with the maximum factored out. Each
// scaled term e^d (d <= 0) is e^{fl(d)} in FP32 times (1 + (d - fl(d))), which
// keeps the rounding of d to FP32 out of the term; the terms are summed in
// FP64. A NaN x gives NaN.
__device__ __forceinline__ double block_log_sum_exp2(const double* __restrict__ x, int64_t n, double* red) {
  double mx = -INFINITY;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) mx = fmax(mx, 2.0 * x[i]);
  const double top = block_reduce_max(mx, red);
  double s = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
    const double d = __dadd_rn(2.0 * x[i], -top);
    const float dh = (float)d;
    s = __fma_rn((double)expf(dh), __dadd_rn(1.0, __dadd_rn(d, -(double)dh)), s);
  }
  return top + log(block_reduce_sum(s, red));
}

__device__ __forceinline__ double log_add_exp(double a, double b) {
  const double hi = fmax(a, b), lo = fmin(a, b);
  return __dadd_rn(hi, log1p(exp(__dadd_rn(lo, -hi))));
}

// The translation step (an extension; Sec. 5 names acceleration from optimal
// transport as future work). IPFP is block coordinate ascent on the concave
// dual whose stationarity conditions are Eq. IPFP. Moving the partner side's
// log potentials up by tau and the own side's down by tau leaves every pair
// term A_xy u_x v_y unchanged, so along that line the dual reads
//   const + tau (sum mass_P - sum mass_O) - 1/2 e^{2 tau} P - 1/2 e^{-2 tau} O,
// P = sum_P e^{2 log p}, O = sum_O e^{2 log o}, and its maximiser is
// tau = 1/2 log z with z the positive root of P z^2 - dm z - O = 0,
// dm = sum mass_P - sum mass_O: z = (dm + R) / (2 P) for dm >= 0 and
// 2 O / (R - dm) for dm < 0 (no cancellation), R = sqrt(dm^2 + 4 P O), all in
// logarithms. Non-finite inputs (non-finite potentials, which the half-sweep
// reports) give tau = 0.
__device__ __forceinline__ double translation_tau(double log_p, double log_o, double dm) {
  const double ln2 = 0.69314718055994530942;
  const double log_4po = __dadd_rn(__dadd_rn(2.0 * ln2, log_p), log_o);
  const double log_r = dm != 0.0 ? 0.5 * log_add_exp(2.0 * log(fabs(dm)), log_4po) : 0.5 * log_4po;
  double log_z;
  if (dm >= 0.0) {
    const double log_num = dm > 0.0 ? log_add_exp(log(dm), log_r) : log_r;
    log_z = __dadd_rn(__dadd_rn(log_num, -ln2), -log_p);
  } else {
    log_z = __dadd_rn(__dadd_rn(ln2, log_o), -log_add_exp(log_r, log(-dm)));
  }
  const double tau = 0.5 * log_z;
  return isfinite(tau) ? tau : 0.0;
}

// tau for the partner side P (potentials log_p, rows_p) and own side O over
// one block of kTauThreads threads (every thread returns it); `red` holds
// kTauThreads / 32 doubles.
__device__ __forceinline__ double block_translation_tau(const double* __restrict__ log_p, int64_t rows_p,
                                                        const double* __restrict__ log_o, int64_t rows_o, double dm,
                                                        double* red) {
  const double lp = block_log_sum_exp2(log_p, rows_p, red);
  const double lo = block_log_sum_exp2(log_o, rows_o, red);
  return translation_tau(lp, lo, dm);
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
