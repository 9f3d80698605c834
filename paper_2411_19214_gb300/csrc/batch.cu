// batch.cu -- many independent markets in one persistent launch per
// half-sweep (tu_batch_*): per-market descriptors, the longest-first item
// schedule over the SMs, the batched preparation and reduction kernels, and
// the solve loop in which converged markets leave the launch.
//
// Every market's arithmetic is that of its own sweep (Eq. iteration_minibatch):
// the preparation kernel computes the same shift and the same FP32 partner
// vector as the single-market path, and each own tile is reduced by the same
// epilogue code, so the potentials after k batched sweeps are bit-identical
// to k sweeps of the market alone. Only the order of the FP64 residual sums
// differs (per own tile and warp instead of per CTA).
#include <algorithm>
#include <cmath>
#include <cstddef>
#include <cstring>
#include <map>
#include <new>
#include <queue>
#include <string>
#include <vector>

#include "trace.h"
#include "tu_internal.cuh"

using namespace tu;

namespace {

constexpr int kPrepThreads = 512;
constexpr int kFinThreads = 256;
constexpr int kMaxBatch = 65536;
// Fixed cost of an item (own-tile load, pipeline fill, row updates), in units
// of one partner tile of MMA + epilogue work; used by the schedule only.
constexpr double kItemOverhead = 2.0;

// One schedule in device memory (and its pinned mirror), in ints:
//   [0]        number of listed markets n
//   [4 ..]     the n listed market indices
//   cta[s]     grid + 1 offsets into items[s], for side s = 0 (X own), 1 (Y own)
//   items[s]   (market, own tile) pairs, CTA by CTA
struct Schedule {
  int* dev = nullptr;
  int* host = nullptr;
  size_t ints = 0;
  size_t off_list = 4, off_cta[2] = {0, 0}, off_items[2] = {0, 0};
  std::vector<int> members;
  bool valid = false;
};

size_t round4(size_t v) { return (v + 3) & ~(size_t)3; }

static_assert(alignof(BatchDesc) >= 128 && sizeof(BatchDesc) % 128 == 0,
              "descriptor arrays keep every tensor map 128-byte aligned");

}  // namespace

struct tu_batch {
  int count = 0;
  int device = 0;
  int num_sms = 0;
  int grid = 0;  // CTAs of the batched half-sweep: one per SM
  int64_t kp = 0;
  int dtype = 0;  // the members' dtype (e4m3 markets: every member alike)
  cudaStream_t stream = nullptr;
  std::vector<tu_market*> markets;
  std::vector<double> relax_cfg;    // each market's relaxation setting at creation
  std::vector<float> c_host;        // each market's exponent multiplier as its descriptors hold it
  BatchDesc* desc_dev[2] = {nullptr, nullptr};  // [side][market]
  std::vector<int> own_tiles[2];    // per market
  std::vector<int> partner_tiles[2];
  int64_t tiles[2] = {0, 0};        // own tiles of all markets, per side
  double* partials = nullptr;       // [slot][kBatchSlotWarps][4]
  double* results = nullptr;        // [market][kResSlots]
  double* results_host = nullptr;   // pinned
  int* err_dev = nullptr;
  int* err_host = nullptr;          // pinned
  double* omega_dev = nullptr;      // [market]
  double* omega_host = nullptr;     // pinned
  Schedule sched[2];                // 0: sweeps, 1: certification passes
  std::map<int, cudaGraphExec_t> graphs;  // captured blocks of k sweeps over schedule 0
  bool profiling = false;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev_pool;
  size_t ev_used = 0;
  bool poisoned = false;
  std::string last_error;
};

namespace {

// ---------------------------------------------------------------------------
// Kernels: one CTA per listed market
// ---------------------------------------------------------------------------

// Partner preparation of a listed market: the FP32 vector
// g = (ell - max ell) log2(e), -inf padded, from the partner's shift kept in
// the market's scalars, and the pass's scalars (prep_scalars: the translation
// step in sweeps, sweep = 1, of a market that takes it; the partner shift; the
// own offset) -- the single-market preparation computes the same values.
__global__ void __launch_bounds__(kPrepThreads) k_batch_prep(const BatchDesc* __restrict__ desc,
                                                            const int* __restrict__ list,
                                                            const int* __restrict__ n_list, int sweep) {
  if ((int)blockIdx.x >= *n_list) return;
  const BatchDesc& d = desc[list[blockIdx.x]];
  const double top = d.st[kStLmax + (1 - d.own_side)];  // not written by prep_scalars
  if (threadIdx.x == 0) prep_scalars(d.st, d.own_side, sweep && d.translate);
  const float inv_c = 1.0f / d.c;  // (the single-market preparation's 1 / c, rounded alike)
  for (int64_t i = threadIdx.x; i < d.partner_rows_pad; i += blockDim.x) {
    const float v = i < d.partner_rows ? (float)((d.partner_ell[i] - top) * 1.4426950408889634) : -INFINITY;
    d.g[i] = v;
    if (d.gfold != nullptr) write_fold_row(reinterpret_cast<uint4*>(d.gfold), i, v, inv_c);
  }
}

// FP64 reduction of a listed market's per-tile partials into its result slots;
// after an updating pass, also the own side's groups into the market's scalars
// (the single-market finalize's routine with the same block size).
__global__ void __launch_bounds__(kFinThreads) k_batch_finalize(const BatchDesc* __restrict__ desc,
                                                               const int* __restrict__ list,
                                                               const int* __restrict__ n_list,
                                                               const double* __restrict__ partials, int is_x,
                                                               int residual, int update,
                                                               double* __restrict__ results) {
  if ((int)blockIdx.x >= *n_list) return;
  const int mk = list[blockIdx.x];
  const BatchDesc& d = desc[mk];
  __shared__ double s_max[kFinThreads], s_l1[kFinThreads], s_sq[kFinThreads], s_nf[kFinThreads];
  __shared__ float redf[2 * kFinThreads / 32];
  const int64_t s0 = (int64_t)d.slot0 * kBatchSlotWarps;
  const int64_t s1 = s0 + (int64_t)d.num_own_tiles * kBatchSlotWarps;
  double mx = 0.0, l1 = 0.0, sq = 0.0, nf = 0.0;
  for (int64_t i = s0 + threadIdx.x; i < s1; i += blockDim.x) {
    mx = fmax(mx, partials[4 * i + 0]);
    l1 += partials[4 * i + 1];
    sq += partials[4 * i + 2];
    nf += partials[4 * i + 3];
  }
  s_max[threadIdx.x] = mx;
  s_l1[threadIdx.x] = l1;
  s_sq[threadIdx.x] = sq;
  s_nf[threadIdx.x] = nf;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) {
      s_max[threadIdx.x] = fmax(s_max[threadIdx.x], s_max[threadIdx.x + w]);
      s_l1[threadIdx.x] += s_l1[threadIdx.x + w];
      s_sq[threadIdx.x] += s_sq[threadIdx.x + w];
      s_nf[threadIdx.x] += s_nf[threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    double* r = results + (int64_t)mk * kResSlots;
    if (is_x) {
      if (residual) {
        r[kResXInf] = s_max[0];
        r[kResXL1] = s_l1[0];
      }
      r[kResXSq] = s_sq[0];
    } else {
      r[kResYSq] = s_sq[0];
    }
    r[kResNonfin] += s_nf[0];
  }
  if (update) {
    const GroupTotal g = block_reduce_groups(d.grp, (d.rows + kGroupRows - 1) / kGroupRows, redf);
    if (threadIdx.x == 0) finish_scalars(d.st, d.own_side, g, d.dm_next);
  }
}

// u = v = 1 (Alg. 1 / Alg. 2 initialisation) for the listed markets, then
// their groups and scalars as the single-market rescan computes them.
__global__ void __launch_bounds__(kFinThreads) k_batch_reset(const BatchDesc* __restrict__ desc_x,
                                                            const BatchDesc* __restrict__ desc_y,
                                                            const int* __restrict__ list,
                                                            const int* __restrict__ n_list) {
  if ((int)blockIdx.x >= *n_list) return;
  const int mk = list[blockIdx.x];
  __shared__ float redf[2 * kFinThreads / 32];
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  GroupTotal tot[2];
  for (int s = 0; s < 2; ++s) {
    const BatchDesc& d = (s == 0 ? desc_x : desc_y)[mk];
    // each warp resets the rows of the groups it then forms
    const int64_t ng = (d.rows + kGroupRows - 1) / kGroupRows;
    for (int64_t g = warp; g < ng; g += kFinThreads / 32) {
      const int64_t i = g * kGroupRows + lane;
      const bool valid = i < d.rows;
      const double e = (valid && d.b2s != nullptr) ? (double)d.b2s[i] : 0.0;
      if (valid) {
        d.log_u[i] = 0.0;
        d.ell[i] = e;
      }
      const float4 gv = warp_group(0.0, e, valid);
      if (lane == 0) d.grp[g] = gv;
    }
    __syncthreads();
    tot[s] = block_reduce_groups(d.grp, ng, redf);
  }
  // the next half-sweep updates X against Y: dm = sum m - sum n
  if (threadIdx.x == 0) rescan_scalars(desc_x[mk].st, tot[0], tot[1], -desc_x[mk].dm_next);
}

// End of a block of batched sweeps: the listed markets' pending offsets
// written into their arrays and folded into their scalars.
__global__ void __launch_bounds__(kFinThreads) k_batch_flush(const BatchDesc* __restrict__ desc_x,
                                                            const BatchDesc* __restrict__ desc_y,
                                                            const int* __restrict__ list,
                                                            const int* __restrict__ n_list) {
  if ((int)blockIdx.x >= *n_list) return;
  const int mk = list[blockIdx.x];
  double* st = desc_x[mk].st;
  const double off[2] = {st[kStOff + 0], st[kStOff + 1]};
  for (int s = 0; s < 2; ++s) {
    if (off[s] == 0.0) continue;
    const BatchDesc& d = (s == 0 ? desc_x : desc_y)[mk];
    for (int64_t i = threadIdx.x; i < d.rows; i += blockDim.x) {
      d.log_u[i] += off[s];
      d.ell[i] += off[s];
    }
  }
  __syncthreads();  // every thread has read the offsets
  if (threadIdx.x == 0) {
    for (int s = 0; s < 2; ++s) {
      st[kStLmax + s] += off[s];
      st[kStOff + s] = 0.0;
    }
  }
}

// results[kResYSq] = sum_y v_y^2 in FP64 for the listed markets.
__global__ void __launch_bounds__(kFinThreads) k_batch_sum_sq(const BatchDesc* __restrict__ desc_y,
                                                             const int* __restrict__ list,
                                                             const int* __restrict__ n_list,
                                                             double* __restrict__ results) {
  if ((int)blockIdx.x >= *n_list) return;
  const int mk = list[blockIdx.x];
  const BatchDesc& d = desc_y[mk];
  __shared__ double red[kFinThreads / 32];
  double s = 0.0;
  for (int64_t i = threadIdx.x; i < d.rows; i += blockDim.x) s += exp(2.0 * d.log_u[i]);
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (threadIdx.x % 32 == 0) red[threadIdx.x / 32] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double b = 0.0;
    for (int w = 0; w < kFinThreads / 32; ++w) b += red[w];
    results[(int64_t)mk * kResSlots + kResYSq] = b;
  }
}

// ---------------------------------------------------------------------------
// Host helpers
// ---------------------------------------------------------------------------

tu_status bfail(tu_batch* b, tu_status s, const std::string& msg) {
  if (b != nullptr) b->last_error = msg;
  return s;
}

tu_status bfail_cuda(tu_batch* b, cudaError_t e, const char* what) {
  cudaGetLastError();
  if (b != nullptr) {
    b->last_error = std::string(what) + ": " + cudaGetErrorString(e);
    if (e != cudaErrorMemoryAllocation) b->poisoned = true;
  }
  return e == cudaErrorMemoryAllocation ? TU_ERR_OOM : TU_ERR_CUDA;
}

#define TB_CK(b, call)                                        \
  do {                                                        \
    cudaError_t _e = (call);                                  \
    if (_e != cudaSuccess) return bfail_cuda((b), _e, #call); \
  } while (0)

#define TB_TRY(expr)            \
  do {                          \
    tu_status _s = (expr);      \
    if (_s != TU_OK) return _s; \
  } while (0)

tu_status check_live(tu_batch* b) {
  if (b == nullptr) return TU_ERR_INVALID_ARG;
  if (b->poisoned) return TU_ERR_CUDA;
  b->last_error.clear();
  TB_CK(b, cudaSetDevice(b->device));
  return TU_OK;
}

// Work already enqueued on the members' streams completes before batch work
// (factors replaced since land in place: the descriptors hold the members'
// buffers; refresh_members follows what else the new factors change).
tu_status wait_members(tu_batch* b) {
  std::vector<cudaStream_t> seen;
  for (tu_market* m : b->markets) {
    if (m->stream == b->stream || std::find(seen.begin(), seen.end(), m->stream) != seen.end()) continue;
    seen.push_back(m->stream);
    TB_CK(b, cudaStreamSynchronize(m->stream));
  }
  return TU_OK;
}

// Members whose factors were replaced since the batch was made: the exponent
// multiplier of e4m3 markets with one scale per side moves with the sides'
// scales, so it is rewritten into both sides' descriptors (in stream order,
// before the launches that read it); a member whose new factors need the
// wide half-sweep (tu_market_create) is refused, as at creation.
tu_status refresh_members(tu_batch* b) {
  for (int i = 0; i < b->count; ++i) {
    const tu_market* m = b->markets[i];
    if (m->wide) return bfail(b, TU_ERR_UNSUPPORTED, "a member's replaced factors need the wide half-sweep");
    if (m->cmul == b->c_host[i]) continue;
    b->c_host[i] = m->cmul;
    for (int side = 0; side < 2; ++side)
      TB_CK(b, cudaMemcpyAsync(reinterpret_cast<char*>(b->desc_dev[side] + i) + offsetof(BatchDesc, c),
                               &b->c_host[i], sizeof(float), cudaMemcpyHostToDevice, b->stream));
  }
  return TU_OK;
}

tu_status sched_alloc(tu_batch* b, Schedule& S) {
  S.off_list = 4;
  S.off_cta[0] = round4(S.off_list + (size_t)b->count);
  S.off_cta[1] = round4(S.off_cta[0] + (size_t)b->grid + 1);
  S.off_items[0] = round4(S.off_cta[1] + (size_t)b->grid + 1);  // 16-byte aligned int2 arrays
  S.off_items[1] = round4(S.off_items[0] + 2 * (size_t)b->tiles[0]);
  S.ints = S.off_items[1] + 2 * (size_t)b->tiles[1];
  TB_CK(b, cudaMalloc(&S.dev, S.ints * sizeof(int)));
  TB_CK(b, cudaMallocHost(&S.host, S.ints * sizeof(int)));
  return TU_OK;
}

// List `members` in schedule S: every own tile of every member is an item;
// items are taken longest first (partner tiles + a fixed overhead) and each
// goes to the CTA with the least work so far (LPT), so one persistent launch
// of grid CTAs is balanced across markets of very different sizes.
tu_status sched_set(tu_batch* b, Schedule& S, const std::vector<int>& members) {
  if (S.valid && S.members == members) return TU_OK;
  TB_CK(b, cudaStreamSynchronize(b->stream));  // the pinned mirror may still be in a copy
  int* h = S.host;
  h[0] = (int)members.size();
  for (size_t i = 0; i < members.size(); ++i) h[S.off_list + i] = members[i];
  struct Item {
    int cost, mk, t;
  };
  std::vector<Item> items;
  std::vector<int> owner, fill(b->grid + 1);
  for (int side = 0; side < 2; ++side) {
    items.clear();
    for (int mk : members)
      for (int t = 0; t < b->own_tiles[side][mk]; ++t) items.push_back({b->partner_tiles[side][mk], mk, t});
    std::stable_sort(items.begin(), items.end(), [](const Item& a, const Item& c) { return a.cost > c.cost; });
    typedef std::pair<double, int> Load;  // (work so far, CTA); ties go to the lower CTA
    std::priority_queue<Load, std::vector<Load>, std::greater<Load>> heap;
    for (int c = 0; c < b->grid; ++c) heap.push({0.0, c});
    owner.assign(items.size(), 0);
    std::fill(fill.begin(), fill.end(), 0);
    for (size_t i = 0; i < items.size(); ++i) {
      Load l = heap.top();
      heap.pop();
      owner[i] = l.second;
      ++fill[l.second + 1];
      l.first += (double)items[i].cost + kItemOverhead;
      heap.push(l);
    }
    int* cta = h + S.off_cta[side];
    for (int c = 0; c < b->grid; ++c) fill[c + 1] += fill[c];
    for (int c = 0; c <= b->grid; ++c) cta[c] = fill[c];
    int* it = h + S.off_items[side];
    for (size_t i = 0; i < items.size(); ++i) {
      const int pos = fill[owner[i]]++;
      it[2 * pos + 0] = items[i].mk;
      it[2 * pos + 1] = items[i].t;
    }
  }
  TB_CK(b, cudaMemcpyAsync(S.dev, S.host, S.ints * sizeof(int), cudaMemcpyHostToDevice, b->stream));
  S.members = members;
  S.valid = true;
  return TU_OK;
}

cudaError_t profile_mark(tu_batch* b, bool start) {
  if (!b->profiling) return cudaSuccess;
  if (start) {
    if (b->ev_used == b->ev_pool.size()) {
      cudaEvent_t e0, e1;
      cudaError_t e = cudaEventCreate(&e0);
      if (e != cudaSuccess) return e;
      e = cudaEventCreate(&e1);
      if (e != cudaSuccess) {
        cudaEventDestroy(e0);
        return e;
      }
      b->ev_pool.push_back({e0, e1});
    }
    return cudaEventRecord(b->ev_pool[b->ev_used].first, b->stream);
  }
  const cudaError_t e = cudaEventRecord(b->ev_pool[b->ev_used].second, b->stream);
  ++b->ev_used;
  return e;
}

// One half-sweep over the markets listed in schedule si: prepare their partner
// vectors, run the batched tensor-core pass, reduce the partials per market.
cudaError_t enqueue_half(tu_batch* b, int si, int side, int residual, int update) {
  const Schedule& S = b->sched[si];
  const int* n = S.dev;
  const int* list = S.dev + S.off_list;
  k_batch_prep<<<b->count, kPrepThreads, 0, b->stream>>>(b->desc_dev[side], list, n, update);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if ((e = profile_mark(b, true)) != cudaSuccess) return e;
  BatchLaunch L;
  L.desc = b->desc_dev[side];
  L.items = reinterpret_cast<const int2*>(S.dev + S.off_items[side]);
  L.cta_start = S.dev + S.off_cta[side];
  L.partials = b->partials;
  L.err = b->err_dev;
  L.grid = b->grid;
  L.kp = b->kp;
  L.dtype = b->dtype;
  L.residual = residual;
  L.update = update;
  if ((e = launch_fused_batch(L, b->stream)) != cudaSuccess) return e;
  if ((e = profile_mark(b, false)) != cudaSuccess) return e;
  k_batch_finalize<<<b->count, kFinThreads, 0, b->stream>>>(b->desc_dev[side], list, n, b->partials,
                                                           side == 0 ? 1 : 0, residual, update, b->results);
  return cudaGetLastError();
}

cudaError_t enqueue_sweep(tu_batch* b) {
  cudaError_t e = enqueue_half(b, 0, 0, kResidualEstimate, 1);
  if (e != cudaSuccess) return e;
  return enqueue_half(b, 0, 1, 0, 1);
}

// After a block of sweeps over schedule 0: pending offsets into the arrays.
cudaError_t enqueue_flush(tu_batch* b) {
  const Schedule& S = b->sched[0];
  k_batch_flush<<<b->count, kFinThreads, 0, b->stream>>>(b->desc_dev[0], b->desc_dev[1], S.dev + S.off_list, S.dev);
  return cudaGetLastError();
}

bool stream_capturable(cudaStream_t s) { return s != nullptr && s != cudaStreamLegacy && s != cudaStreamPerThread; }

// k sweeps over schedule 0; a captured graph per k is replayed (the schedule
// lives in device memory, so the graphs stay valid when markets leave).
tu_status enqueue_sweeps(tu_batch* b, int k) {
  if (k <= 0) return TU_OK;
  if (!stream_capturable(b->stream) || k == 1 || b->profiling) {
    for (int i = 0; i < k; ++i) TB_CK(b, enqueue_sweep(b));
    TB_CK(b, enqueue_flush(b));
    return TU_OK;
  }
  auto found = b->graphs.find(k);
  if (found == b->graphs.end()) {
    cudaGraph_t g = nullptr;
    TB_CK(b, cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < k && e == cudaSuccess; ++i) e = enqueue_sweep(b);
    if (e == cudaSuccess) e = enqueue_flush(b);
    const cudaError_t e2 = cudaStreamEndCapture(b->stream, &g);
    if (e != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      return bfail_cuda(b, e, "capture of the batched sweep graph");
    }
    if (e2 != cudaSuccess) return bfail_cuda(b, e2, "cudaStreamEndCapture");
    cudaGraphExec_t ge = nullptr;
    const cudaError_t e3 = cudaGraphInstantiate(&ge, g, 0);
    cudaGraphDestroy(g);
    if (e3 != cudaSuccess) return bfail_cuda(b, e3, "cudaGraphInstantiate");
    found = b->graphs.emplace(k, ge).first;
  }
  TB_CK(b, cudaGraphLaunch(found->second, b->stream));
  return TU_OK;
}

tu_status clear_results(tu_batch* b) {
  TB_CK(b, cudaMemsetAsync(b->results, 0, (size_t)b->count * kResSlots * sizeof(double), b->stream));
  TB_CK(b, cudaMemsetAsync(b->err_dev, 0, sizeof(int), b->stream));
  return TU_OK;
}

tu_status read_results(tu_batch* b) {
  TB_CK(b, cudaMemcpyAsync(b->results_host, b->results, (size_t)b->count * kResSlots * sizeof(double),
                           cudaMemcpyDeviceToHost, b->stream));
  TB_CK(b, cudaMemcpyAsync(b->err_host, b->err_dev, sizeof(int), cudaMemcpyDeviceToHost, b->stream));
  TB_CK(b, cudaStreamSynchronize(b->stream));
  if (*b->err_host == kErrTimeout) return bfail(b, TU_ERR_TIMEOUT, "a device-side wait ran out of its time limit");
  if (*b->err_host != kErrNone) return bfail(b, TU_ERR_CUDA, "device error word set");
  return TU_OK;
}

// Residual of the current potentials of `members` (one X pass without update).
tu_status certify(tu_batch* b, const std::vector<int>& members) {
  TB_TRY(sched_set(b, b->sched[1], members));
  TB_CK(b, enqueue_half(b, 1, 0, kResidualExact, 0));
  return read_results(b);
}

tu_status upload_omega(tu_batch* b) {
  TB_CK(b, cudaMemcpyAsync(b->omega_dev, b->omega_host, (size_t)b->count * sizeof(double), cudaMemcpyHostToDevice,
                           b->stream));
  return TU_OK;
}

// Each market's relaxation factor outside a solve (its fixed factor, else 1),
// or at the start of a solve (1 for every market: relaxed markets begin with
// plain sweeps while their controller estimates the convergence rate).
tu_status reset_omega(tu_batch* b, bool solve_start = false) {
  TB_CK(b, cudaStreamSynchronize(b->stream));  // the pinned mirror may still be in a copy
  for (int i = 0; i < b->count; ++i)
    b->omega_host[i] = (!solve_start && b->relax_cfg[i] > 1.0) ? b->relax_cfg[i] : 1.0;
  return upload_omega(b);
}

double res(const tu_batch* b, int mk, int slot) { return b->results_host[(size_t)mk * kResSlots + slot]; }

}  // namespace

extern "C" {

void tu_batch_destroy(tu_batch_t b) {
  TU_TRACE("tu_batch_destroy");
  if (b == nullptr) return;
  cudaSetDevice(b->device);
  if (b->stream) cudaStreamSynchronize(b->stream);
  for (auto& g : b->graphs) cudaGraphExecDestroy(g.second);
  for (auto& pr : b->ev_pool) {
    cudaEventDestroy(pr.first);
    cudaEventDestroy(pr.second);
  }
  for (int s = 0; s < 2; ++s) {
    cudaFree(b->desc_dev[s]);
    cudaFree(b->sched[s].dev);
    cudaFreeHost(b->sched[s].host);
  }
  cudaFree(b->partials);
  cudaFree(b->results);
  cudaFree(b->err_dev);
  cudaFree(b->omega_dev);
  cudaFreeHost(b->results_host);
  cudaFreeHost(b->err_host);
  cudaFreeHost(b->omega_host);
  delete b;
}

const char* tu_batch_last_error(tu_batch_t b) { return b ? b->last_error.c_str() : ""; }

tu_status tu_batch_create(const tu_market_t* markets, int count, void* stream, tu_batch_t* out) {
  TU_TRACE("tu_batch_create");
  if (out == nullptr) return TU_ERR_INVALID_ARG;
  *out = nullptr;
  if (markets == nullptr || count < 1 || count > kMaxBatch) return TU_ERR_INVALID_ARG;
  std::vector<tu_market*> ms(markets, markets + count);
  for (int i = 0; i < count; ++i) {
    tu_market* m = ms[i];
    if (m == nullptr || m->poisoned || m->path != TU_PATH_FUSED) return TU_ERR_INVALID_ARG;
    if (m->kp != ms[0]->kp || m->device != ms[0]->device) return TU_ERR_INVALID_ARG;
    // one operand format (BF16 and FP32 inputs are both computed in BF16)
    if ((is_fp8(m->dtype) || is_fp8(ms[0]->dtype)) && m->dtype != ms[0]->dtype) return TU_ERR_INVALID_ARG;
    // the batched kernel keeps one shift per market and half-sweep, and is
    // built for packed rows of one or two 128-byte k blocks (e4m3: one)
    if (m->wide || m->kp > 128) return TU_ERR_UNSUPPORTED;
  }
  {
    std::vector<tu_market*> sorted(ms);
    std::sort(sorted.begin(), sorted.end());
    if (std::adjacent_find(sorted.begin(), sorted.end()) != sorted.end()) return TU_ERR_INVALID_ARG;
  }
  tu_batch* b = new (std::nothrow) tu_batch();
  if (b == nullptr) return TU_ERR_OOM;
  auto bail = [&](tu_status s) {
    tu_batch_destroy(b);
    return s;
  };
  b->count = count;
  b->device = ms[0]->device;
  b->num_sms = ms[0]->num_sms;
  b->grid = b->num_sms;
  b->kp = ms[0]->kp;
  b->dtype = ms[0]->dtype;
  b->stream = static_cast<cudaStream_t>(stream);
  b->markets = ms;
  b->c_host.assign(count, 0.0f);
  if (cudaSetDevice(b->device) != cudaSuccess) return bail(TU_ERR_CUDA);
  // descriptors: side 0 updates X against Y, side 1 updates Y against X
  std::vector<BatchDesc> desc(count);
  tu_status st;
  if ((st = [&]() -> tu_status {
        TB_CK(b, cudaMalloc(&b->omega_dev, (size_t)count * sizeof(double)));
        return TU_OK;
      }()) != TU_OK)
    return bail(st);
  for (int side = 0; side < 2; ++side) {
    b->own_tiles[side].resize(count);
    b->partner_tiles[side].resize(count);
    int64_t slot = 0;
    for (int i = 0; i < count; ++i) {
      tu_market* m = ms[i];
      const Side& own = side == 0 ? m->X : m->Y;
      const Side& par = side == 0 ? m->Y : m->X;
      BatchDesc& d = desc[i];
      memset(&d, 0, sizeof(d));
      d.tm_own = own.tm_own;
      d.tm_partner = par.tm_partner;
      d.b2s = own.b2s;
      d.mass = own.mass;
      d.log_u = own.log_u;
      d.ell = own.ell;
      d.partner_ell = par.ell;
      d.dm_next = own.sum_mass - par.sum_mass;
      d.own_side = side;
      d.st = m->st;
      d.grp = own.grp;
      d.translate = m->translate ? 1 : 0;
      d.g = par.pvec;
      d.omega = b->omega_dev + i;
      d.rows = own.rows;
      d.partner_rows = par.rows;
      d.partner_rows_pad = par.rows_pad;
      d.num_own_tiles = (int)((own.rows + kFusedOwnRows - 1) / kFusedOwnRows);
      d.num_partner_tiles = (int)((par.rows + kFusedPartnerRows - 1) / kFusedPartnerRows);
      d.slot0 = (int)slot;
      d.c = m->cmul;
      if (side == 0) b->c_host[i] = m->cmul;
      d.fs_own = own.fs;
      d.fs_par = par.fs;
      d.gfold = par.fold;
      b->own_tiles[side][i] = d.num_own_tiles;
      b->partner_tiles[side][i] = d.num_partner_tiles;
      slot += d.num_own_tiles;
      if (slot > ((int64_t)1 << 28)) return bail(bfail(b, TU_ERR_UNSUPPORTED, "too many own tiles in one batch"));
    }
    b->tiles[side] = slot;
    if ((st = [&]() -> tu_status {
          TB_CK(b, cudaMalloc(&b->desc_dev[side], (size_t)count * sizeof(BatchDesc)));
          TB_CK(b, cudaMemcpy(b->desc_dev[side], desc.data(), (size_t)count * sizeof(BatchDesc),
                              cudaMemcpyHostToDevice));
          return TU_OK;
        }()) != TU_OK)
      return bail(st);
  }
  if ((st = [&]() -> tu_status {
        const int64_t slots = std::max(b->tiles[0], b->tiles[1]) * kBatchSlotWarps;
        TB_CK(b, cudaMalloc(&b->partials, (size_t)slots * 4 * sizeof(double)));
        TB_CK(b, cudaMalloc(&b->results, (size_t)count * kResSlots * sizeof(double)));
        TB_CK(b, cudaMalloc(&b->err_dev, sizeof(int)));
        TB_CK(b, cudaMallocHost(&b->results_host, (size_t)count * kResSlots * sizeof(double)));
        TB_CK(b, cudaMallocHost(&b->err_host, sizeof(int)));
        TB_CK(b, cudaMallocHost(&b->omega_host, (size_t)count * sizeof(double)));
        TB_TRY(sched_alloc(b, b->sched[0]));
        TB_TRY(sched_alloc(b, b->sched[1]));
        return TU_OK;
      }()) != TU_OK)
    return bail(st);
  b->relax_cfg.resize(count);
  for (int i = 0; i < count; ++i) b->relax_cfg[i] = ms[i]->omega_cfg;
  if (reset_omega(b) != TU_OK || clear_results(b) != TU_OK || cudaStreamSynchronize(b->stream) != cudaSuccess)
    return bail(TU_ERR_CUDA);
  *out = b;
  return TU_OK;
}

tu_status tu_batch_profile_enable(tu_batch_t b, int enable) {
  TB_TRY(check_live(b));
  b->profiling = enable != 0;
  return TU_OK;
}

tu_status tu_batch_profile_read(tu_batch_t b, double* pass_ms, int64_t* passes) {
  TB_TRY(check_live(b));
  TB_CK(b, cudaStreamSynchronize(b->stream));
  double total = 0.0;
  for (size_t i = 0; i < b->ev_used; ++i) {
    float ms = 0.0f;
    TB_CK(b, cudaEventElapsedTime(&ms, b->ev_pool[i].first, b->ev_pool[i].second));
    total += ms;
  }
  if (pass_ms) *pass_ms = total;
  if (passes) *passes = (int64_t)b->ev_used;
  b->ev_used = 0;
  return TU_OK;
}

tu_status tu_batch_sweep(tu_batch_t b, int nsweeps, double* residual_out) {
  TU_TRACE("tu_batch_sweep");
  TB_TRY(check_live(b));
  if (nsweeps < 0) return bfail(b, TU_ERR_INVALID_ARG, "nsweeps < 0");
  TB_TRY(wait_members(b));
  TB_TRY(refresh_members(b));
  std::vector<int> all(b->count);
  for (int i = 0; i < b->count; ++i) all[i] = i;
  TB_TRY(sched_set(b, b->sched[0], all));
  TB_TRY(clear_results(b));
  TB_TRY(enqueue_sweeps(b, nsweeps));
  if (residual_out == nullptr) return TU_OK;
  TB_TRY(certify(b, all));
  bool nonfinite = false;
  for (int i = 0; i < b->count; ++i) {
    residual_out[i] = res(b, i, kResXInf);
    nonfinite = nonfinite || res(b, i, kResNonfin) > 0.0;
  }
  if (nonfinite) return bfail(b, TU_ERR_NONFINITE, "a computed potential is not finite");
  return TU_OK;
}

tu_status tu_batch_solve(tu_batch_t b, double tol, int max_iter, int warm_start, tu_solve_info* infos) {
  TU_TRACE("tu_batch_solve");
  TB_TRY(check_live(b));
  if (!(tol >= 0.0) || max_iter < 0) return bfail(b, TU_ERR_INVALID_ARG, "tol < 0 or max_iter < 0");
  TB_TRY(wait_members(b));
  TB_TRY(refresh_members(b));
  const int count = b->count;
  std::vector<int> all(count);
  for (int i = 0; i < count; ++i) all[i] = i;
  if (!warm_start) {
    TB_TRY(sched_set(b, b->sched[0], all));
    k_batch_reset<<<count, kFinThreads, 0, b->stream>>>(b->desc_dev[0], b->desc_dev[1], b->sched[0].dev + 4,
                                                          b->sched[0].dev);
    TB_CK(b, cudaGetLastError());
  }
  TB_TRY(reset_omega(b, true));
  TB_TRY(clear_results(b));
  std::vector<RelaxControl> ctl;
  ctl.reserve(count);
  for (int i = 0; i < count; ++i) ctl.emplace_back(b->relax_cfg[i]);
  std::vector<int> status(count, TU_ERR_NOT_CONVERGED), sweeps(count, 0);
  std::vector<double> r_inf(count, INFINITY), r_l1(count, INFINITY);
  auto record = [&](int mk) {
    r_inf[mk] = res(b, mk, kResXInf);
    r_l1[mk] = res(b, mk, kResXL1) / b->markets[mk]->X.sum_mass;
  };
  std::vector<int> active;
  TB_TRY(certify(b, all));
  for (int mk = 0; mk < count; ++mk) {
    record(mk);
    if (res(b, mk, kResNonfin) > 0.0) {
      status[mk] = TU_ERR_NONFINITE;
    } else if (r_inf[mk] <= tol) {
      status[mk] = TU_OK;
    } else {
      active.push_back(mk);
    }
  }
  int done = 0, last_k = 0;
  std::vector<double> r_prev(count, -1.0), r_last(count, -1.0);
  while (!active.empty() && done < max_iter) {
    // sweeps between host checks: about 2e9 pair evaluations per check, 1..64
    // (at most 16 while a market adapts its relaxation factor), and no more than
    // the active market closest to tol needs at its measured decay (plan_block)
    double pairs = 0.0;
    bool relaxing = false;
    for (int mk : active) {
      pairs += (double)b->markets[mk]->N * (double)b->markets[mk]->M;
      relaxing = relaxing || ctl[mk].enabled();
    }
    int block = (int)std::ceil(2e9 / pairs);
    block = block < 1 ? 1 : (block > 64 ? 64 : block);
    if (relaxing && block > 16) block = 16;
    int k = block;
    for (int mk : active) {
      const int want = plan_block(last_k, r_prev[mk], r_last[mk], tol, block);
      if (want < k) k = want;
    }
    if (k > max_iter - done) k = max_iter - done;
    last_k = k;
    TB_TRY(sched_set(b, b->sched[0], active));
    TB_TRY(enqueue_sweeps(b, k));
    TB_TRY(read_results(b));
    done += k;
    std::vector<int> keep, cand;
    bool omega_dirty = false;
    for (int mk : active) {
      sweeps[mk] = done;
      if (res(b, mk, kResNonfin) > 0.0) {
        status[mk] = TU_ERR_NONFINITE;
        record(mk);
        continue;
      }
      const double r = res(b, mk, kResXInf);
      r_prev[mk] = r_last[mk];
      r_last[mk] = r;
      if (r <= tol) {
        cand.push_back(mk);
        continue;
      }
      keep.push_back(mk);
      if (ctl[mk].enabled()) {
        const double next = ctl[mk].observe(done, r, tol);
        if (next != b->omega_host[mk]) {
          b->omega_host[mk] = next;
          omega_dirty = true;
        }
      }
    }
    if (omega_dirty) TB_TRY(upload_omega(b));
    if (!cand.empty()) {
      // the residual folded into the last sweep met tol: certify the returned state
      TB_TRY(certify(b, cand));
      for (int mk : cand) {
        record(mk);
        if (res(b, mk, kResNonfin) > 0.0) {
          status[mk] = TU_ERR_NONFINITE;
        } else if (r_inf[mk] <= tol) {
          status[mk] = TU_OK;
        } else {
          keep.push_back(mk);
        }
      }
      std::sort(keep.begin(), keep.end());
    }
    active.swap(keep);
  }
  if (!active.empty()) {
    TB_TRY(certify(b, active));
    for (int mk : active) record(mk);
  }
  TB_TRY(reset_omega(b));
  // match counts from the column equations: sum_xy mu_xy = sum m - sum v^2
  TB_TRY(sched_set(b, b->sched[1], all));
  k_batch_sum_sq<<<count, kFinThreads, 0, b->stream>>>(b->desc_dev[1], b->sched[1].dev + 4, b->sched[1].dev,
                                                         b->results);
  TB_CK(b, cudaGetLastError());
  TB_TRY(read_results(b));
  tu_status overall = TU_OK;
  for (int mk = 0; mk < count; ++mk) {
    if (status[mk] == TU_ERR_NONFINITE) overall = TU_ERR_NONFINITE;
    if (status[mk] == TU_ERR_NOT_CONVERGED && overall == TU_OK) overall = TU_ERR_NOT_CONVERGED;
    if (infos != nullptr) {
      infos[mk].sweeps = sweeps[mk];
      infos[mk].status = status[mk];
      infos[mk].residual_inf = r_inf[mk];
      infos[mk].residual_l1 = r_l1[mk];
      infos[mk].match_count = b->markets[mk]->Y.sum_mass - res(b, mk, kResYSq);
    }
  }
  if (overall == TU_ERR_NOT_CONVERGED) b->last_error = "max_iter reached before every market met tol";
  if (overall == TU_ERR_NONFINITE) b->last_error = "a computed potential is not finite";
  return overall;
}

}  // extern "C"
