// market.cu -- the C ABI (include/tu_ipfp.h): market lifetime, argument
// checking, host/device staging, the sweep loop with CUDA-graph replay, and the
// convergence test of tu_ipfp_solve.
#include <atomic>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <tuple>
#include <unordered_map>
#include <vector>

#include "trace.h"
#include "tu_internal.cuh"

using namespace tu;

namespace {

const char* kStatusNames[] = {"TU_OK",          "TU_ERR_INVALID_ARG", "TU_ERR_OOM",     "TU_ERR_CUDA",
                              "TU_ERR_NOT_CONVERGED", "TU_ERR_NONFINITE", "TU_ERR_TIMEOUT", "TU_ERR_UNSUPPORTED"};

int64_t round_up(int64_t a, int64_t b) { return (a + b - 1) / b * b; }

// Packed row length of the fused path: 2d elements rounded up to one, two or
// four 128-byte k blocks (BF16: 64, 128 or 256 elements; e4m3: 128, 256 or 512).
int64_t fused_row_length(int64_t d, bool fp8) {
  int64_t kp = fp8 ? 128 : kKBlock;
  while (kp < 2 * d) kp *= 2;
  return kp;
}

tu_status fail(tu_market* m, tu_status s, const std::string& msg) {
  if (m != nullptr) m->last_error = msg;
  return s;
}

tu_status fail_cuda(tu_market* m, cudaError_t e, const char* what) {
  cudaGetLastError();  // clear a sticky-free error so later calls can report their own
  if (m != nullptr) {
    m->last_error = std::string(what) + ": " + cudaGetErrorString(e);
    if (e != cudaErrorMemoryAllocation) m->poisoned = true;
  }
  return e == cudaErrorMemoryAllocation ? TU_ERR_OOM : TU_ERR_CUDA;
}

#define TU_CK(m, call)                                      \
  do {                                                      \
    cudaError_t _e = (call);                                \
    if (_e != cudaSuccess) return fail_cuda((m), _e, #call); \
  } while (0)

#define TU_TRY(expr)                 \
  do {                               \
    tu_status _s = (expr);           \
    if (_s != TU_OK) return _s;      \
  } while (0)

bool is_device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// ------------------------------------------------------------------ memory
// A market's device memory comes from a stream-ordered pool per device and
// is allocated and freed in the order of the market's own stream. cudaMalloc
// and cudaFree synchronise the device: in a loop that creates, updates and
// destroys markets while others sweep (serving), each of them would drain
// every other market's queued work. Freed blocks stay in the pool for the next
// market; the pool is trimmed when the last market of the process goes away.
// (The dense path's two resident kernel matrices keep cudaMalloc: they are
// created once per market and their placement was measured.)
constexpr int kMaxDevices = 64;
std::mutex g_pool_mu;
cudaMemPool_t g_pools[kMaxDevices] = {};
int g_live_markets = 0;

cudaMemPool_t market_pool(int device) {
  if (device < 0 || device >= kMaxDevices) return nullptr;
  std::lock_guard<std::mutex> lk(g_pool_mu);
  if (g_pools[device] == nullptr) {
    cudaMemPoolProps props{};
    props.allocType = cudaMemAllocationTypePinned;
    props.handleTypes = cudaMemHandleTypeNone;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = device;
    cudaMemPool_t pool = nullptr;
    if (cudaMemPoolCreate(&pool, &props) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    uint64_t keep = UINT64_MAX;  // no release at synchronisation points
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    g_pools[device] = pool;
  }
  return g_pools[device];
}

// Checked mode: guard bands of kGuardByte around every market buffer,
// verified when the buffer is freed (see tu_set_checked_mode). The band width
// keeps each buffer 256-byte aligned inside its block.
constexpr size_t kGuard = 256;
constexpr unsigned char kGuardByte = 0xA5;

bool checked_from_env() {
  const char* v = std::getenv("TU_CHECKED");
  return v != nullptr && std::strcmp(v, "1") == 0;
}

struct GuardedBlock {
  void* base;
  size_t bytes;  // the buffer's own size (between the bands)
};
std::atomic<bool> g_checked{checked_from_env()};
std::mutex g_guard_mu;
std::unordered_map<void*, GuardedBlock> g_guarded;  // buffer -> its block
int64_t g_violations = 0;
std::string g_last_violation;

// Compare the two bands of a guarded buffer with the pattern (after the work
// queued on `stream`); counts a violation when either changed.
void verify_guards(void* p, const GuardedBlock& g, cudaStream_t stream) {
  unsigned char band[2][kGuard];
  cudaError_t e = cudaMemcpyAsync(band[0], g.base, kGuard, cudaMemcpyDeviceToHost, stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(band[1], static_cast<char*>(g.base) + kGuard + g.bytes, kGuard, cudaMemcpyDeviceToHost,
                        stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return;  // the market's own error path reports CUDA failures
  }
  for (int side = 0; side < 2; ++side) {
    for (size_t i = 0; i < kGuard; ++i) {
      if (band[side][i] != kGuardByte) {
        char msg[200];
        snprintf(msg, sizeof(msg), "buffer %p of %zu bytes: %s guard band changed at byte %zu", p, g.bytes,
                 side == 0 ? "leading" : "trailing", i);
        std::lock_guard<std::mutex> lk(g_guard_mu);
        ++g_violations;
        g_last_violation = msg;
        return;
      }
    }
  }
}

tu_status dev_alloc_bytes(tu_market* m, void** p, size_t bytes) {
  *p = nullptr;
  if (bytes == 0) return TU_OK;
  cudaMemPool_t pool = market_pool(m->device);
  if (pool == nullptr) return fail(m, TU_ERR_CUDA, "device memory pool unavailable");
  const bool guarded = g_checked.load();
  void* base = nullptr;
  cudaError_t e = cudaMallocFromPoolAsync(&base, guarded ? bytes + 2 * kGuard : bytes, pool, m->stream);
  if (e != cudaSuccess) return fail_cuda(m, e, "cudaMallocFromPoolAsync");
  if (!guarded) {
    *p = base;
    return TU_OK;
  }
  e = cudaMemsetAsync(base, kGuardByte, kGuard, m->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(static_cast<char*>(base) + kGuard + bytes, kGuardByte, kGuard, m->stream);
  if (e != cudaSuccess) {
    cudaFreeAsync(base, m->stream);
    return fail_cuda(m, e, "guard bands");
  }
  *p = static_cast<char*>(base) + kGuard;
  std::lock_guard<std::mutex> lk(g_guard_mu);
  g_guarded[*p] = GuardedBlock{base, bytes};
  return TU_OK;
}

// Free a dev_alloc buffer in the order of the market's stream (guarded
// buffers: after their bands were checked).
void dev_free_bytes(tu_market* m, void* p) {
  if (p == nullptr) return;
  GuardedBlock g{nullptr, 0};
  {
    std::lock_guard<std::mutex> lk(g_guard_mu);
    auto it = g_guarded.find(p);
    if (it != g_guarded.end()) {
      g = it->second;
      g_guarded.erase(it);
    }
  }
  if (g.base == nullptr) {
    cudaFreeAsync(p, m->stream);
    return;
  }
  verify_guards(p, g, m->stream);
  cudaFreeAsync(g.base, m->stream);
}

template <typename T>
tu_status dev_alloc(tu_market* m, T** p, size_t count) {
  void* v = nullptr;
  const tu_status st = dev_alloc_bytes(m, &v, count * sizeof(T));
  *p = static_cast<T*>(v);
  return st;
}

// Stream-ordered release of a dev_alloc block (after the market's queued work).
template <typename T>
void dev_free(tu_market* m, T*& p) {
  dev_free_bytes(m, const_cast<void*>(static_cast<const void*>(p)));
  p = nullptr;
}

// A market's page-locked host mirrors (results, query snapshot, omega, error
// word) share one block from slabs of kSlabBlocks: page-locked allocations
// serialise the device like cudaMalloc. Slabs live for the process.
struct HostMirror {
  double results[kResSlots];
  double query[kResSlots + 1];
  double omega;
  int err;
};
constexpr size_t kMirrorBytes = (sizeof(HostMirror) + 63) / 64 * 64;
constexpr int kSlabBlocks = 64;
std::mutex g_mirror_mu;
std::vector<void*> g_mirror_free;

HostMirror* mirror_alloc() {
  std::lock_guard<std::mutex> lk(g_mirror_mu);
  if (g_mirror_free.empty()) {
    void* slab = nullptr;
    if (cudaMallocHost(&slab, kMirrorBytes * kSlabBlocks) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    for (int i = kSlabBlocks - 1; i >= 0; --i) g_mirror_free.push_back(static_cast<char*>(slab) + i * kMirrorBytes);
  }
  void* b = g_mirror_free.back();
  g_mirror_free.pop_back();
  return new (b) HostMirror();
}

void mirror_free(void* b) {
  if (b == nullptr) return;
  std::lock_guard<std::mutex> lk(g_mirror_mu);
  g_mirror_free.push_back(b);
}

tu_status ensure_staging(tu_market* m, size_t bytes) {
  if (m->staging_bytes >= bytes) return TU_OK;
  dev_free(m, m->staging);  // stream-ordered: after the copies that used it
  m->staging_bytes = 0;
  TU_TRY(dev_alloc_bytes(m, &m->staging, bytes));
  m->staging_bytes = bytes;
  return TU_OK;
}

// Device view of a caller pointer: the pointer itself if it is device memory,
// else a copy in the staging buffer at byte offset `off`.
tu_status device_view(tu_market* m, const void* src, size_t bytes, size_t off, const void** out) {
  if (is_device_ptr(src)) {
    *out = src;
    return TU_OK;
  }
  void* dst = static_cast<char*>(m->staging) + off;
  TU_CK(m, cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, m->stream));
  *out = dst;
  return TU_OK;
}

tu_status side_alloc(tu_market* m, Side& s, int64_t rows, bool has_bias) {
  s.rows = rows;
  s.rows_pad = round_up(rows, kRowPad);
  TU_TRY(dev_alloc(m, &s.log_u, s.rows_pad));
  TU_TRY(dev_alloc(m, &s.ell, s.rows_pad));
  TU_TRY(dev_alloc(m, &s.pvec, s.rows_pad));
  TU_TRY(dev_alloc(m, &s.mass, s.rows_pad));
  // groups of 32 rows; the dense pass's layout (rows dealt round-robin over up
  // to kMaxPartials CTAs) needs at most rows / 32 + 2 * kMaxPartials of them
  TU_TRY(dev_alloc(m, &s.grp, (size_t)(s.rows_pad / kGroupRows + 2 * kMaxPartials)));
  if (has_bias) TU_TRY(dev_alloc(m, &s.b2s, s.rows_pad));
  if (m->path == TU_PATH_FUSED && is_fp8(m->dtype)) {
    TU_TRY(dev_alloc(m, &s.fac8, (size_t)rows * m->kp));
    TU_TRY(dev_alloc(m, &s.fs, s.rows_pad));
    // one scale per side and 128-byte rows: the extra MMA's g / c operand
    if (m->dtype == TU_DTYPE_FP8E4M3_SIDE && m->kp == 128) TU_TRY(dev_alloc(m, &s.fold, (size_t)s.rows_pad * 32));
  } else if (m->path == TU_PATH_FUSED) {
    TU_TRY(dev_alloc(m, &s.fac16, (size_t)rows * m->kp));
    // the partner tiles' g / c operand of the fused kernel's extra MMA
    if (m->kp == kKBlock) TU_TRY(dev_alloc(m, &s.fold, (size_t)s.rows_pad * 32));
  } else {
    TU_TRY(dev_alloc(m, &s.fac32, (size_t)rows * m->kp));
  }
  return TU_OK;
}

void side_free(tu_market* m, Side& s) {
  dev_free(m, s.log_u);
  dev_free(m, s.ell);
  dev_free(m, s.pvec);
  dev_free(m, s.mass);
  dev_free(m, s.grp);
  dev_free(m, s.b2s);
  dev_free(m, s.fac16);
  dev_free(m, s.fac8);
  dev_free(m, s.fs);
  dev_free(m, s.fold);
  dev_free(m, s.fac32);
  s = Side();
}

tu_status upload_masses(tu_market* m, Side& s, const double* host) {
  double sum = 0.0;
  for (int64_t i = 0; i < s.rows; ++i) {
    const double v = host[i];
    if (!(v > 0.0) || !std::isfinite(v)) return fail(m, TU_ERR_INVALID_ARG, "capacities must be finite and > 0");
    sum += v;
  }
  s.sum_mass = sum;
  TU_CK(m, cudaMemcpyAsync(s.mass, host, (size_t)s.rows * sizeof(double), cudaMemcpyHostToDevice, m->stream));
  // padding capacities are 1 so that padded rows never produce log(0)
  if (s.rows_pad > s.rows) {
    const size_t npad = (size_t)(s.rows_pad - s.rows);
    double* ones = new (std::nothrow) double[npad];
    if (ones == nullptr) return fail(m, TU_ERR_OOM, "host allocation");
    for (size_t i = 0; i < npad; ++i) ones[i] = 1.0;
    cudaError_t e = cudaMemcpyAsync(s.mass + s.rows, ones, npad * sizeof(double), cudaMemcpyHostToDevice, m->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);  // `ones` is pageable and freed below
    delete[] ones;
    if (e != cudaSuccess) return fail_cuda(m, e, "mass padding");
  }
  return TU_OK;
}

// FP8 with one scale per side: smallest integer k with maxabs <= 448 * 2^k
// (exact comparisons with powers of two; 0 for an all-zero side).
int fp8_side_exponent(float maxabs) {
  if (!(maxabs > 0.0f)) return 0;
  int e = 0;
  std::frexp((double)maxabs / 448.0, &e);
  int k = e;
  while (std::ldexp(448.0, k - 1) >= (double)maxabs) --k;
  while (std::ldexp(448.0, k) < (double)maxabs) ++k;
  return k;
}

// FP8: quantize one side's factor pair (device pointers) into s.fac8 and its
// row scales s.fs: from FP32 rows (each row scaled by its own power of two,
// or TU_DTYPE_FP8E4M3_SIDE: all by the side's), or, with caller scales sc,
// from e4m3 bytes the caller quantized.
tu_status pack_side_fp8(tu_market* m, Side& s, const void* a, const void* b, const float* sc, unsigned int* bad) {
  unsigned int hbad = 0;
  TU_CK(m, cudaMemsetAsync(bad, 0, sizeof(unsigned int), m->stream));
  if (sc != nullptr) {
    TU_CK(m, launch_pack_fp8_bytes(m, s, static_cast<const uint8_t*>(a), static_cast<const uint8_t*>(b), sc, bad));
  } else {
    int side_k = kPerRowScale;
    if (m->dtype == TU_DTYPE_FP8E4M3_SIDE) {
      float mx = 0.0f;
      float* scratch = reinterpret_cast<float*>(bad + 1);
      TU_CK(m, launch_max_abs(m, static_cast<const float*>(a), static_cast<const float*>(b), s.rows * m->d, scratch));
      TU_CK(m, cudaMemcpyAsync(&mx, scratch, sizeof(float), cudaMemcpyDeviceToHost, m->stream));
      TU_CK(m, cudaStreamSynchronize(m->stream));
      if (!std::isfinite(mx)) return fail(m, TU_ERR_NONFINITE, "factor matrices contain NaN or Inf");
      side_k = s.fp8_exp = fp8_side_exponent(mx);
    }
    TU_CK(m, launch_pack_fp8_rows(m, s, static_cast<const float*>(a), static_cast<const float*>(b), side_k, bad));
  }
  TU_CK(m, cudaMemcpyAsync(&hbad, bad, sizeof(hbad), cudaMemcpyDeviceToHost, m->stream));
  TU_CK(m, cudaStreamSynchronize(m->stream));
  if (hbad != 0)
    return fail(m, TU_ERR_NONFINITE, sc ? "FP8 row scales contain NaN or Inf" : "factor matrices contain NaN or Inf");
  return TU_OK;
}

// Pack both factor pairs (and rebuild the dense kernel) from caller pointers.
// fsx, fsy: FP8 markets created with caller scales: the per-row scales of the
// e4m3 bytes F, K (resp. G, L), host or device; otherwise nullptr.
tu_status load_factors(tu_market* m, const void* F, const void* K, const void* G, const void* L,
                       const float* fsx = nullptr, const float* fsy = nullptr) {
  const bool fp8 = is_fp8(m->dtype);
  const bool prescaled = fp8 && m->fp8_caller_scales;
  const size_t esz = prescaled ? 1 : (m->dtype == TU_DTYPE_BF16 ? 2 : 4);
  const size_t bx = (size_t)m->N * m->d * esz, by = (size_t)m->M * m->d * esz;
  // (caller scales follow the two factor matrices in the staging buffer)
  const size_t sx = prescaled ? round_up((int64_t)(2 * bx), 256) : 0, sy = prescaled ? round_up((int64_t)(2 * by), 256) : 0;
  const size_t stage = 2 * (bx > by ? bx : by) + (prescaled ? 256 + 4 * (size_t)(m->N > m->M ? m->N : m->M) : 0);
  TU_TRY(ensure_staging(m, stage));
  unsigned int* bad = nullptr;  // [0]: the pack kernels' flag, [1]: a float scratch
  if (fp8) TU_TRY(dev_alloc(m, &bad, 2));
  auto pack = [&](Side& s, const void* a, const void* b, const float* sc) -> tu_status {
    if (fp8) return pack_side_fp8(m, s, a, b, sc, bad);
    TU_CK(m, launch_pack_factors(m, s, a, b, m->dtype));
    return TU_OK;
  };
  const void *a = nullptr, *b = nullptr, *sc = nullptr;
  tu_status st = device_view(m, F, bx, 0, &a);
  if (st == TU_OK) st = device_view(m, K, bx, bx, &b);
  if (st == TU_OK && prescaled) st = device_view(m, fsx, (size_t)m->N * 4, sx, &sc);
  if (st == TU_OK) st = pack(m->X, a, b, static_cast<const float*>(sc));
  if (st == TU_OK && cudaStreamSynchronize(m->stream) != cudaSuccess)  // the staging buffer is reused
    st = fail_cuda(m, cudaGetLastError(), "cudaStreamSynchronize");
  if (st == TU_OK) st = device_view(m, G, by, 0, &a);
  if (st == TU_OK) st = device_view(m, L, by, by, &b);
  if (st == TU_OK && prescaled) st = device_view(m, fsy, (size_t)m->M * 4, sy, &sc);
  if (st == TU_OK) st = pack(m->Y, a, b, static_cast<const float*>(sc));
  dev_free(m, bad);
  if (st != TU_OK) return st;
  // the multiplier of <a_x, b_y> in the exponent (log2 units; FP8 with per-row
  // scales: those are applied in the kernels; with one scale per side: folded in)
  m->cmul = (float)std::ldexp(1.4426950408889634 / (2.0 * m->sigma),
                              m->dtype == TU_DTYPE_FP8E4M3_SIDE ? m->X.fp8_exp + m->Y.fp8_exp : 0);
  // exponent-range check (Cauchy-Schwarz bound of |phi_hat| / (2 sigma))
  float* norms = nullptr;
  TU_TRY(dev_alloc(m, &norms, 2));
  float hn[2] = {0.f, 0.f};
  cudaError_t e = launch_row_norms(m, m->X, norms);
  if (e == cudaSuccess) e = launch_row_norms(m, m->Y, norms + 1);
  if (e == cudaSuccess) e = cudaMemcpyAsync(hn, norms, sizeof(hn), cudaMemcpyDeviceToHost, m->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
  dev_free(m, norms);
  if (e != cudaSuccess) return fail_cuda(m, e, "factor norms");
  if (!std::isfinite(hn[0]) || !std::isfinite(hn[1]))
    return fail(m, TU_ERR_NONFINITE, "factor matrices contain NaN or Inf");
  const double bound = (double)hn[0] * (double)hn[1] / (2.0 * m->sigma);  // FP8: norms of the quantized rows
  // One shift per half-sweep (the partner side's max ell) keeps every exponent
  // within +-bound log2(e) of the row's largest: up to 40, FP32 holds the
  // terms and their sums. Beyond, the fused path keeps a running maximum per
  // row and rescales the row's sum when it grows (one pass); the dense path's
  // materialised A-hat itself would leave the FP32 range.
  const bool wide = bound > 40.0;
  if (wide && m->path == TU_PATH_DENSE) {
    char buf[160];
    snprintf(buf, sizeof(buf), "max|a_x| * max|b_y| / (2 sigma) = %.3g exceeds 40 (FP32 range of A-hat)", bound);
    return fail(m, TU_ERR_UNSUPPORTED, buf);
  }
  m->wide = wide;
  if (m->path == TU_PATH_DENSE) TU_CK(m, launch_dense_build(m));
  TU_CK(m, cudaStreamSynchronize(m->stream));
  if (m->graph != nullptr) {
    cudaGraphExecDestroy(m->graph);
    m->graph = nullptr;
    m->graph_sweeps = 0;
  }
  return TU_OK;
}

tu_status check_device_error(tu_market* m) {
  if (*m->err_host == kErrTimeout) return fail(m, TU_ERR_TIMEOUT, "a device-side wait ran out of its time limit");
  if (*m->err_host != kErrNone) return fail(m, TU_ERR_CUDA, "device error word set");
  return TU_OK;
}

// Event pair around the main pass of a half-sweep (profiling only).
cudaError_t profile_mark(tu_market* m, bool start) {
  if (!m->profiling) return cudaSuccess;
  if (start) {
    if (m->ev_used == m->ev_pool.size()) {
      cudaEvent_t a, b;
      cudaError_t e = cudaEventCreate(&a);
      if (e != cudaSuccess) return e;
      e = cudaEventCreate(&b);
      if (e != cudaSuccess) {
        cudaEventDestroy(a);
        return e;
      }
      m->ev_pool.push_back({a, b});
    }
    return cudaEventRecord(m->ev_pool[m->ev_used].first, m->stream);
  }
  cudaError_t e = cudaEventRecord(m->ev_pool[m->ev_used].second, m->stream);
  ++m->ev_used;
  return e;
}

// One half-sweep: prepare the partner potentials and the pass's scalars, run
// the pass, reduce its partials (and, after an update, the own side's groups).
cudaError_t enqueue_half(tu_market* m, int side, int residual, int update) {
  Side& partner = side == 0 ? m->Y : m->X;
  // sweeps (update = 1) take the translation step; a certifying pass leaves the state as it is
  cudaError_t e = launch_prep(m, partner, m->path == TU_PATH_FUSED ? 1 : 0, update && m->translate ? 1 : 0);
  if (e != cudaSuccess) return e;
  if ((e = profile_mark(m, true)) != cudaSuccess) return e;
  int nparts = 0;
  int64_t ngroups = ((side == 0 ? m->N : m->M) + kGroupRows - 1) / kGroupRows;
  if (m->path == TU_PATH_FUSED) {
    e = launch_fused_halfsweep(m, side, residual, update, &nparts);
  } else if (side == 0) {
    e = launch_dense_rowpass(m, residual, update, &nparts, &ngroups);
  } else {
    e = launch_dense_colpass(m, update, &nparts, &ngroups);
  }
  if (e != cudaSuccess) return e;
  if ((e = profile_mark(m, false)) != cudaSuccess) return e;
  return launch_finalize(m, nparts, side == 0 ? 1 : 0, residual, update, ngroups);
}

// One sweep of Eq. iteration: u from v (with the residual of the entering
// state), then v from the new u.
cudaError_t enqueue_sweep(tu_market* m) {
  cudaError_t e = enqueue_half(m, 0, kResidualEstimate, 1);
  if (e != cudaSuccess) return e;
  return enqueue_half(m, 1, 0, 1);
}

bool stream_capturable(cudaStream_t s) { return s != nullptr && s != cudaStreamLegacy && s != cudaStreamPerThread; }

// k sweeps, then the translation steps still pending as offsets written into
// the potentials (so every other call sees plain arrays).
cudaError_t enqueue_block(tu_market* m, int k) {
  cudaError_t e = cudaSuccess;
  for (int i = 0; i < k && e == cudaSuccess; ++i) e = enqueue_sweep(m);
  if (e == cudaSuccess && k > 0) e = launch_flush(m);
  return e;
}

// Enqueue k sweeps, replaying a captured graph of k sweeps when possible.
tu_status enqueue_sweeps(tu_market* m, int k) {
  if (k <= 0) return TU_OK;
  if (m->use_graphs && stream_capturable(m->stream) && k > 1 && !m->profiling) {
    if (m->graph == nullptr || m->graph_sweeps != k) {
      if (m->graph != nullptr) {
        cudaGraphExecDestroy(m->graph);
        m->graph = nullptr;
      }
      cudaGraph_t g = nullptr;
      TU_CK(m, cudaStreamBeginCapture(m->stream, cudaStreamCaptureModeThreadLocal));
      cudaError_t e = enqueue_block(m, k);
      cudaError_t e2 = cudaStreamEndCapture(m->stream, &g);
      if (e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return fail_cuda(m, e, "capture of the sweep graph");
      }
      if (e2 != cudaSuccess) return fail_cuda(m, e2, "cudaStreamEndCapture");
      cudaError_t e3 = cudaGraphInstantiate(&m->graph, g, 0);
      cudaGraphDestroy(g);
      if (e3 != cudaSuccess) return fail_cuda(m, e3, "cudaGraphInstantiate");
      m->graph_sweeps = k;
    }
    TU_CK(m, cudaGraphLaunch(m->graph, m->stream));
    return TU_OK;
  }
  TU_CK(m, enqueue_block(m, k));
  return TU_OK;
}

tu_status read_results(tu_market* m) {
  TU_CK(m, cudaMemcpyAsync(m->results_host, m->results, kResSlots * sizeof(double), cudaMemcpyDeviceToHost,
                           m->stream));
  TU_CK(m, cudaMemcpyAsync(m->err_host, m->err_dev, sizeof(int), cudaMemcpyDeviceToHost, m->stream));
  TU_CK(m, cudaStreamSynchronize(m->stream));
  TU_TRY(check_device_error(m));
  if (m->results_host[kResNonfin] > 0.0) return fail(m, TU_ERR_NONFINITE, "a computed potential is not finite");
  return TU_OK;
}

// The partner split's arrival counters: 8 per own tile of 128 rows or more,
// for the larger side.
int64_t split_counter_count(const tu_market* m) {
  const int64_t rows = m->X.rows_pad > m->Y.rows_pad ? m->X.rows_pad : m->Y.rows_pad;
  return (rows / (kFusedOwnRows / 2) + 1) * (kFusedOwnRows / 32);
}

tu_status clear_results(tu_market* m) {
  TU_CK(m, cudaMemsetAsync(m->results, 0, kResSlots * sizeof(double), m->stream));
  TU_CK(m, cudaMemsetAsync(m->err_dev, 0, sizeof(int), m->stream));
  // every completed split launch leaves its counters at zero, but one that a
  // timed-out wait cut short may not: zeroed again before the next work
  if (m->split_cnt != nullptr)
    TU_CK(m, cudaMemsetAsync(m->split_cnt, 0, (size_t)split_counter_count(m) * sizeof(int), m->stream));
  return TU_OK;
}

// Residual of the current potentials (one X pass without update).
tu_status certify(tu_market* m, double* res_inf, double* res_l1) {
  TU_CK(m, enqueue_half(m, 0, kResidualExact, 0));
  TU_TRY(read_results(m));
  if (res_inf) *res_inf = m->results_host[kResXInf];
  if (res_l1) *res_l1 = m->results_host[kResXL1] / m->X.sum_mass;
  // tu_market_query then describes this synchronous call: every sweep done,
  // the certified residual and the match count of the returned state
  std::memcpy(m->query_host, m->results_host, kResSlots * sizeof(double));
  const int no_error = kErrNone;
  std::memcpy(m->query_host + kResSlots, &no_error, sizeof(int));
  if (m->done_ev == nullptr) TU_CK(m, cudaEventCreateWithFlags(&m->done_ev, cudaEventDisableTiming));
  TU_CK(m, cudaEventRecord(m->done_ev, m->stream));
  m->query_sweeps = m->sweeps_enqueued;
  return TU_OK;
}

// The over-relaxation factor every later pass reads (device scalar, so
// captured graphs stay valid).
tu_status set_omega(tu_market* m, double omega) {
  TU_CK(m, cudaStreamSynchronize(m->stream));  // the pinned staging word may still be in use
  *m->omega_host = omega;
  TU_CK(m, cudaMemcpyAsync(m->omega_dev, m->omega_host, sizeof(double), cudaMemcpyHostToDevice, m->stream));
  return TU_OK;
}

// Restart the controller of asynchronous sweeps (new factors, potentials or
// setting): plain sweeps again until the decay rate has been re-estimated.
tu_status relax_reset(tu_market* m) {
  m->relax = RelaxControl(m->omega_cfg);
  m->relax_base = m->sweeps_enqueued;
  m->relax_seen = -1;
  if (m->omega_cfg == 0.0 && *m->omega_host != 1.0) TU_TRY(set_omega(m, 1.0));
  return TU_OK;
}

tu_status check_live(tu_market* m) {
  if (m == nullptr) return TU_ERR_INVALID_ARG;
  if (m->poisoned) return TU_ERR_CUDA;
  m->last_error.clear();
  cudaError_t e = cudaSetDevice(m->device);
  if (e != cudaSuccess) return fail_cuda(m, e, "cudaSetDevice");
  return TU_OK;
}

// Device destination for an output of `bytes`; host destinations go through staging.
tu_status output_view(tu_market* m, void* dst, size_t bytes, size_t off, void** out, bool* is_host) {
  if (is_device_ptr(dst)) {
    *out = dst;
    *is_host = false;
    return TU_OK;
  }
  TU_TRY(ensure_staging(m, off + bytes));
  *out = static_cast<char*>(m->staging) + off;
  *is_host = true;
  return TU_OK;
}

}  // namespace

double tu::RelaxControl::observe(int done, double r, double tol) {
  best = r < best ? r : best;
  if (target > 1.0) {
    if (r > 10.0 * best) {
      target = 1.0 + 0.5 * (target - 1.0);
      if (target < 1.01) target = 1.0;
      best = r;
    }
    if (cfg > 1.0) {  // a fixed factor is applied as set (only the safeguard above lowers it)
      omega = target;
      return omega;
    }
    double w = std::log10(r / tol);
    w = w < 0.0 ? 0.0 : (w > 1.0 ? 1.0 : w);
    const double next = 1.0 + (target - 1.0) * w;
    if (std::fabs(next - omega) > 1e-3) omega = next;
    return omega;
  }
  if (omega == 1.0) {
    hist.push_back({done, r});
    if (r < 0.1 && done - last_est >= kProbe) {
      const std::pair<int, double>* base = nullptr;
      for (const auto& h : hist)
        if (h.first <= done - kProbe) base = &h;
      if (base != nullptr && base->second > 0.0 && r > 0.0) {
        const double q = std::pow(r / base->second, 1.0 / (double)(done - base->first));
        last_est = done;
        if (q > 0.0 && q < 1.0) {
          const bool settled = q_prev > 0.0 && std::fabs(q - q_prev) < 0.05 * (1.0 - q);
          if (cfg > 1.0 || settled) target = cfg > 1.0 ? cfg : std::fmin(1.98, 2.0 / (1.0 + std::sqrt(1.0 - q)));
          q_prev = q;
        }
      }
    }
  }
  return omega;
}

extern "C" {

const char* tu_status_string(tu_status s) {
  if ((int)s < 0 || (int)s > 7) return "TU_ERR_UNKNOWN";
  return kStatusNames[(int)s];
}

const char* tu_market_last_error(tu_market_t m) { return m ? m->last_error.c_str() : ""; }

tu_status tu_set_checked_mode(int enable) {
  g_checked.store(enable != 0);
  return TU_OK;
}

int64_t tu_guard_violations(char* last, int64_t last_size) {
  std::lock_guard<std::mutex> lk(g_guard_mu);
  if (last != nullptr && last_size > 0) {
    const size_t n = g_last_violation.size() < (size_t)(last_size - 1) ? g_last_violation.size() : (size_t)(last_size - 1);
    std::memcpy(last, g_last_violation.data(), n);
    last[n] = '\0';
  }
  return g_violations;
}

tu_status tu_profile_enable(tu_market_t m, int enable) {
  TU_TRY(check_live(m));
  m->profiling = enable != 0;
  return TU_OK;
}

tu_status tu_profile_read(tu_market_t m, double* pass_ms, int64_t* passes) {
  TU_TRY(check_live(m));
  TU_CK(m, cudaStreamSynchronize(m->stream));
  double total = 0.0;
  for (size_t i = 0; i < m->ev_used; ++i) {
    float ms = 0.0f;
    TU_CK(m, cudaEventElapsedTime(&ms, m->ev_pool[i].first, m->ev_pool[i].second));
    total += ms;
  }
  if (pass_ms) *pass_ms = total;
  if (passes) *passes = (int64_t)m->ev_used;
  m->ev_used = 0;
  return TU_OK;
}

void tu_market_destroy(tu_market_t m) {
  TU_TRACE("tu_market_destroy");
  if (m == nullptr) return;
  cudaSetDevice(m->device);
  if (m->stream) cudaStreamSynchronize(m->stream);
  for (auto& pr : m->ev_pool) {
    cudaEventDestroy(pr.first);
    cudaEventDestroy(pr.second);
  }
  if (m->graph) cudaGraphExecDestroy(m->graph);
  side_free(m, m->X);
  side_free(m, m->Y);
  for (float** a : {&m->Ahat, &m->AhatT}) {
    bool guarded;
    {
      std::lock_guard<std::mutex> lk(g_guard_mu);
      guarded = g_guarded.count(*a) != 0;
    }
    if (guarded) {
      dev_free(m, *a);
    } else if (*a != nullptr) {
      cudaFree(*a);
      *a = nullptr;
    }
  }
  dev_free(m, m->partials);
  dev_free(m, m->st);
  dev_free(m, m->split_part);
  dev_free(m, m->split_cnt);
  dev_free(m, m->results);
  dev_free(m, m->err_dev);
  dev_free(m, m->staging);
  dev_free(m, m->aux);
  dev_free(m, m->omega_dev);
  if (m->done_ev) cudaEventDestroy(m->done_ev);
  mirror_free(m->results_host);  // the block that holds all four host mirrors
  {
    // every market that reaches this point was counted by tu_market_create
    std::lock_guard<std::mutex> lk(g_pool_mu);
    if (--g_live_markets == 0 && m->device >= 0 && m->device < kMaxDevices && g_pools[m->device] != nullptr) {
      // the last market: return the pool's memory once its frees have run
      if (m->stream) cudaStreamSynchronize(m->stream);
      cudaMemPoolTrimTo(g_pools[m->device], 0);
    }
  }
  delete m;
}

namespace {
void apply_tuned(tu_market* m);  // (the autotuner, below)
}  // namespace

tu_status tu_market_create(const tu_market_desc* desc, tu_market_t* out) {
  TU_TRACE("tu_market_create");
  if (out == nullptr || desc == nullptr) return TU_ERR_INVALID_ARG;
  *out = nullptr;
  const tu_market_desc& D = *desc;
  if (D.N < 1 || D.M < 1 || D.d < 1 || D.N > (int64_t)1 << 31 || D.M > (int64_t)1 << 31 || D.d > 4096)
    return TU_ERR_INVALID_ARG;
  if (D.dtype != TU_DTYPE_BF16 && D.dtype != TU_DTYPE_FP32 && !is_fp8(D.dtype)) return TU_ERR_INVALID_ARG;
  if (D.path != TU_PATH_FUSED && D.path != TU_PATH_DENSE) return TU_ERR_INVALID_ARG;
  if (!D.F || !D.K || !D.G || !D.L || !D.n || !D.m) return TU_ERR_INVALID_ARG;
  if (!(D.sigma > 0.0) || !std::isfinite(D.sigma)) return TU_ERR_INVALID_ARG;
  if (D.partition < 0) return TU_ERR_INVALID_ARG;
  // caller-quantized FP8: both sides' scales, e4m3 factors only
  if ((D.fscale_x != nullptr) != (D.fscale_y != nullptr)) return TU_ERR_INVALID_ARG;
  if (D.fscale_x != nullptr && D.dtype != TU_DTYPE_FP8E4M3) return TU_ERR_INVALID_ARG;
  // fused path: packed rows of 1, 2 or 4 128-byte k blocks
  if (D.path == TU_PATH_FUSED && !is_fp8(D.dtype) && D.d > 128) return TU_ERR_UNSUPPORTED;
  if (is_fp8(D.dtype) && D.d > 256) return TU_ERR_UNSUPPORTED;
  if (is_fp8(D.dtype) && D.path != TU_PATH_FUSED) return TU_ERR_UNSUPPORTED;
  // the dense path keeps A-hat and its transpose resident
  if (D.path == TU_PATH_DENSE &&
      (double)D.N * (double)round_up(D.M, 4) * 4.0 + (double)D.M * (double)round_up(D.N, 4) * 4.0 > 200e9)
    return TU_ERR_UNSUPPORTED;

  tu_market* m = new (std::nothrow) tu_market();
  if (m == nullptr) return TU_ERR_OOM;
  m->N = D.N;
  m->M = D.M;
  m->d = D.d;
  m->kp = D.path == TU_PATH_FUSED ? fused_row_length(D.d, is_fp8(D.dtype)) : round_up(2 * D.d, kKBlock);
  m->fp8_caller_scales = D.fscale_x != nullptr;
  m->dtype = D.dtype;
  m->path = D.path;
  m->sigma = D.sigma;
  m->partition = D.partition;
  m->stream = static_cast<cudaStream_t>(D.stream);
  tu_status st = TU_OK;
  auto bail = [&](tu_status s) {
    tu_market_destroy(m);
    return s;
  };
  if (cudaGetDevice(&m->device) != cudaSuccess ||
      cudaDeviceGetAttribute(&m->num_sms, cudaDevAttrMultiProcessorCount, m->device) != cudaSuccess) {
    cudaGetLastError();
    delete m;
    return TU_ERR_CUDA;
  }
  if (!device_supported(m->device)) {
    delete m;
    return TU_ERR_UNSUPPORTED;
  }
  {
    int l2 = 0;
    if (cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, m->device) != cudaSuccess) {
      cudaGetLastError();
      l2 = 0;
    }
    m->l2_bytes = l2;
  }
  {
    std::lock_guard<std::mutex> lk(g_pool_mu);
    ++g_live_markets;  // from here on every exit goes through tu_market_destroy
  }
  if ((st = side_alloc(m, m->X, D.N, D.bias_x != nullptr)) != TU_OK) return bail(st);
  if ((st = side_alloc(m, m->Y, D.M, D.bias_y != nullptr)) != TU_OK) return bail(st);
  if ((st = dev_alloc(m, &m->partials, (size_t)kMaxPartials * 4)) != TU_OK) return bail(st);
  if ((st = dev_alloc(m, &m->st, (size_t)kStSlots)) != TU_OK) return bail(st);
  if ((st = dev_alloc(m, &m->results, (size_t)kResSlots)) != TU_OK) return bail(st);
  if ((st = dev_alloc(m, &m->err_dev, 1)) != TU_OK) return bail(st);
  {
    HostMirror* hm = mirror_alloc();
    if (hm == nullptr) return bail(TU_ERR_OOM);
    m->results_host = hm->results;
    m->query_host = hm->query;
    m->omega_host = &hm->omega;
    m->err_host = &hm->err;
  }
  *m->err_host = 0;
  if (D.path == TU_PATH_DENSE) {
    m->ldA = round_up(D.M, 4);
    m->ldN = round_up(D.N, 4);
    if (g_checked.load()) {  // checked mode: guarded like the other buffers
      if ((st = dev_alloc(m, &m->Ahat, (size_t)m->N * m->ldA)) != TU_OK) return bail(st);
      if ((st = dev_alloc(m, &m->AhatT, (size_t)m->M * m->ldN)) != TU_OK) return bail(st);
    } else {
      cudaError_t e = cudaMalloc(&m->Ahat, (size_t)m->N * m->ldA * sizeof(float));
      if (e == cudaSuccess) e = cudaMalloc(&m->AhatT, (size_t)m->M * m->ldN * sizeof(float));
      if (e != cudaSuccess) return bail(fail_cuda(m, e, "cudaMalloc(A-hat)"));
    }
  }
  // (allocated after the dense matrices: placing this small allocation before
  // them measurably slowed the dense row stream)
  if ((st = dev_alloc(m, &m->omega_dev, 1)) != TU_OK) return bail(st);
  *m->omega_host = 1.0;
  if (cudaMemcpyAsync(m->omega_dev, m->omega_host, sizeof(double), cudaMemcpyHostToDevice, m->stream) !=
      cudaSuccess)
    return bail(fail_cuda(m, cudaGetLastError(), "omega"));
  if ((st = upload_masses(m, m->X, D.n)) != TU_OK) return bail(st);
  if ((st = upload_masses(m, m->Y, D.m)) != TU_OK) return bail(st);
  // biases -> b / (2 sigma); potentials start at u = v = 1. A non-finite
  // bias is refused (TU_ERR_NONFINITE) like a non-finite factor.
  {
    const size_t bbytes = (size_t)(D.N > D.M ? D.N : D.M) * sizeof(float);
    if ((st = ensure_staging(m, bbytes)) != TU_OK) return bail(st);
    float* bmax = nullptr;
    if ((D.bias_x || D.bias_y) && (st = dev_alloc(m, &bmax, 1)) != TU_OK) return bail(st);
    auto init = [&](Side& s, const float* bias, int64_t rows, const char* what) -> tu_status {
      const void* bdev = nullptr;
      if (bias) {
        TU_TRY(device_view(m, bias, (size_t)rows * 4, 0, &bdev));
        float hm = 0.0f;
        const float* b = static_cast<const float*>(bdev);
        TU_CK(m, launch_max_abs(m, b, b, rows, bmax));
        TU_CK(m, cudaMemcpyAsync(&hm, bmax, sizeof(float), cudaMemcpyDeviceToHost, m->stream));
        TU_CK(m, cudaStreamSynchronize(m->stream));
        if (!std::isfinite(hm)) return fail(m, TU_ERR_NONFINITE, std::string(what) + " contains NaN or Inf");
      }
      TU_CK(m, launch_init_side(m, s, static_cast<const float*>(bdev), bias != nullptr));
      TU_CK(m, cudaStreamSynchronize(m->stream));  // the staging buffer is reused
      return TU_OK;
    };
    st = init(m->X, D.bias_x, D.N, "bias_x");
    if (st == TU_OK) st = init(m->Y, D.bias_y, D.M, "bias_y");
    dev_free(m, bmax);
    if (st != TU_OK) return bail(st);
  }
  if ((st = load_factors(m, D.F, D.K, D.G, D.L, D.fscale_x, D.fscale_y)) != TU_OK) {
    // keep the message for the caller by returning it through a status only
    return bail(st);
  }
  if (D.path == TU_PATH_FUSED) {
    cudaError_t e = fused_prepare(m);
    if (e != cudaSuccess) return bail(fail_cuda(m, e, "fused_prepare"));
    apply_tuned(m);
  }
  if (cudaMemsetAsync(m->st, 0, kStSlots * sizeof(double), m->stream) != cudaSuccess ||
      launch_rescan(m) != cudaSuccess)
    return bail(fail_cuda(m, cudaGetLastError(), "scalars of the initial potentials"));
  if (clear_results(m) != TU_OK || cudaStreamSynchronize(m->stream) != cudaSuccess) return bail(TU_ERR_CUDA);
  *out = m;
  return TU_OK;
}

tu_status tu_market_update_factors(tu_market_t m, const void* F, const void* K, const void* G, const void* L) {
  TU_TRACE("tu_market_update_factors");
  TU_TRY(check_live(m));
  if (!F || !K || !G || !L) return fail(m, TU_ERR_INVALID_ARG, "null factor pointer");
  if (m->fp8_caller_scales) return fail(m, TU_ERR_INVALID_ARG, "caller-scaled FP8 market: use the scaled update");
  TU_TRY(load_factors(m, F, K, G, L));
  return relax_reset(m);
}

tu_status tu_market_update_factors_fp8(tu_market_t m, const void* F, const void* K, const void* G, const void* L,
                                       const float* fscale_x, const float* fscale_y) {
  TU_TRACE("tu_market_update_factors_fp8");
  TU_TRY(check_live(m));
  if (!F || !K || !G || !L || !fscale_x || !fscale_y) return fail(m, TU_ERR_INVALID_ARG, "null pointer");
  if (!m->fp8_caller_scales) return fail(m, TU_ERR_INVALID_ARG, "not a caller-scaled FP8 market");
  TU_TRY(load_factors(m, F, K, G, L, fscale_x, fscale_y));
  return relax_reset(m);
}

tu_status tu_ipfp_sweep(tu_market_t m, int nsweeps, double* residual_out) {
  TU_TRACE("tu_ipfp_sweep");
  TU_TRY(check_live(m));
  if (nsweeps < 0) return fail(m, TU_ERR_INVALID_ARG, "nsweeps < 0");
  TU_TRY(clear_results(m));
  TU_TRY(enqueue_sweeps(m, nsweeps));
  m->sweeps_enqueued += nsweeps;
  if (residual_out != nullptr) {
    TU_TRY(certify(m, residual_out, nullptr));
  } else if (nsweeps > 0) {
    // snapshot of the FP64 results for tu_market_query, then the completion event
    TU_CK(m, cudaMemcpyAsync(m->query_host, m->results, kResSlots * sizeof(double), cudaMemcpyDeviceToHost,
                             m->stream));
    TU_CK(m, cudaMemcpyAsync(m->query_host + kResSlots, m->err_dev, sizeof(int), cudaMemcpyDeviceToHost,
                             m->stream));
    if (m->done_ev == nullptr) TU_CK(m, cudaEventCreateWithFlags(&m->done_ev, cudaEventDisableTiming));
    TU_CK(m, cudaEventRecord(m->done_ev, m->stream));
    m->query_sweeps = m->sweeps_enqueued;
  }
  return TU_OK;
}

tu_status tu_market_set_relaxation(tu_market_t m, double omega) {
  TU_TRY(check_live(m));
  if (!(omega == 0.0 || (omega >= 1.0 && omega < 2.0)))
    return fail(m, TU_ERR_INVALID_ARG, "omega must be 0 (automatic) or in [1, 2)");
  if (m->path == TU_PATH_DENSE && (omega != 1.0) != (m->omega_cfg != 1.0) && m->graph != nullptr) {
    // the captured dense sweeps use the row-pass variant of the previous setting
    TU_CK(m, cudaStreamSynchronize(m->stream));
    cudaGraphExecDestroy(m->graph);
    m->graph = nullptr;
    m->graph_sweeps = 0;
  }
  m->omega_cfg = omega;
  TU_TRY(set_omega(m, omega > 1.0 ? omega : 1.0));
  return relax_reset(m);
}

tu_status tu_market_use_graphs(tu_market_t m, int enable) {
  TU_TRY(check_live(m));
  m->use_graphs = enable != 0;
  if (!m->use_graphs && m->graph != nullptr) {
    TU_CK(m, cudaStreamSynchronize(m->stream));
    cudaGraphExecDestroy(m->graph);
    m->graph = nullptr;
    m->graph_sweeps = 0;
  }
  return TU_OK;
}

// ---------------------------------------------------------------------------
// Launch shape of the fused half-sweep (own-tile height, partner split) and
// its autotuner
// ---------------------------------------------------------------------------

namespace {

// captured sweeps hold the launch shape they were captured with
tu_status drop_graph(tu_market* m) {
  if (m->graph == nullptr) return TU_OK;
  TU_CK(m, cudaStreamSynchronize(m->stream));
  cudaGraphExecDestroy(m->graph);
  m->graph = nullptr;
  m->graph_sweeps = 0;
  return TU_OK;
}

// partial row sums (split x the larger side) and the arrival counters (8 per
// own tile of 128 rows or more), zeroed
tu_status ensure_split_buffers(tu_market* m, int split) {
  if (split <= m->split_cap) return TU_OK;
  TU_CK(m, cudaStreamSynchronize(m->stream));  // no pass still uses the old buffers
  dev_free(m, m->split_part);
  dev_free(m, m->split_cnt);
  m->split_cap = 0;
  const int64_t rows = m->X.rows_pad > m->Y.rows_pad ? m->X.rows_pad : m->Y.rows_pad;
  const int64_t blocks = split_counter_count(m);
  TU_TRY(dev_alloc(m, &m->split_part, (size_t)split * rows));
  TU_TRY(dev_alloc(m, &m->split_cnt, (size_t)blocks));
  TU_CK(m, cudaMemsetAsync(m->split_cnt, 0, (size_t)blocks * sizeof(int), m->stream));
  m->split_cap = split;
  return TU_OK;
}

tu_status set_shape(tu_market* m, int small_mode, int split, bool blocks) {
  if (small_mode == m->small_mode && split == m->split && blocks == m->split_blocks) return TU_OK;
  TU_TRY(drop_graph(m));
  if (split > 1) TU_TRY(ensure_split_buffers(m, split));
  m->small_mode = small_mode;
  m->split = split;
  m->split_blocks = split > 1 && blocks;
  return TU_OK;
}

// A shape code: split s > 0 (ranges of one own tile side by side) or -b
// (b partner blocks one after another), as tu_market_get_shape reports it.
tu_status set_shape_code(tu_market* m, int small_mode, int code) {
  return set_shape(m, small_mode, code < 0 ? -code : code, code < 0);
}

// The tuned shapes, by market shape: quarter-octave buckets of N and M, the
// packed row length, the operand format and the SM count.
struct TuneKey {
  int nb, mb;
  int64_t kp;
  int fmt;
  int sms;
  bool operator<(const TuneKey& o) const {
    return std::tie(nb, mb, kp, fmt, sms) < std::tie(o.nb, o.mb, o.kp, o.fmt, o.sms);
  }
};
struct TuneVal {
  int small_mode, split;
  double ms, ms_default;
};
std::mutex g_tune_mu;
std::map<TuneKey, TuneVal> g_tune;

int octave_bucket(int64_t n) { return (int)std::floor(4.0 * std::log2((double)n)); }
TuneKey tune_key(const tu_market* m) {
  return {octave_bucket(m->N), octave_bucket(m->M), m->kp, is_fp8(m->dtype) ? m->dtype : 0, m->num_sms};
}

// A new fused market takes the shape tuned for its bucket, if any (a failed
// allocation of the split buffers leaves the default shape).
void apply_tuned(tu_market* m) {
  TuneVal v{};
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune.find(tune_key(m));
    if (it == g_tune.end()) return;
    v = it->second;
  }
  if (set_shape_code(m, v.small_mode, v.split) != TU_OK) {
    m->last_error.clear();
    m->small_mode = 1;
    m->split = 1;
  }
}

// ms per sweep (both half-sweeps, no update, as a certifying pass runs them)
// of the current shape, over reps after one untimed sweep
tu_status time_shape(tu_market* m, int reps, double* ms) {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  TU_CK(m, cudaEventCreate(&e0));
  cudaError_t e = cudaEventCreate(&e1);
  for (int r = -1; r < reps && e == cudaSuccess; ++r) {
    if (r == 0) e = cudaEventRecord(e0, m->stream);
    if (e == cudaSuccess) e = enqueue_half(m, 0, kResidualEstimate, 0);
    if (e == cudaSuccess) e = enqueue_half(m, 1, kResidualNone, 0);
  }
  if (e == cudaSuccess) e = cudaEventRecord(e1, m->stream);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  float t = 0.0f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
  cudaEventDestroy(e0);
  if (e1 != nullptr) cudaEventDestroy(e1);
  if (e != cudaSuccess) return fail_cuda(m, e, "autotune timing");
  *ms = (double)t / reps;
  return TU_OK;
}

}  // namespace

tu_status tu_market_set_small_tiles(tu_market_t m, int mode) {
  TU_TRY(check_live(m));
  if (mode < 0 || mode > 2) return fail(m, TU_ERR_INVALID_ARG, "small-tile mode must be 0, 1 or 2");
  return set_shape(m, mode, m->split, m->split_blocks);
}

tu_status tu_market_set_split(tu_market_t m, int split) {
  TU_TRY(check_live(m));
  if (m->path != TU_PATH_FUSED) return fail(m, TU_ERR_UNSUPPORTED, "the partner split is a fused-path shape");
  if (split < 1 || split > kMaxSplit) return fail(m, TU_ERR_INVALID_ARG, "split must be in [1, 8]");
  return set_shape(m, m->small_mode, split, false);
}

tu_status tu_market_set_partner_blocks(tu_market_t m, int blocks) {
  TU_TRY(check_live(m));
  if (m->path != TU_PATH_FUSED) return fail(m, TU_ERR_UNSUPPORTED, "partner blocks are a fused-path shape");
  if (blocks < 1 || blocks > kMaxSplit) return fail(m, TU_ERR_INVALID_ARG, "blocks must be in [1, 8]");
  return set_shape(m, m->small_mode, blocks, true);
}

tu_status tu_market_get_shape(tu_market_t m, int* small_mode, int* split) {
  TU_TRY(check_live(m));
  if (small_mode != nullptr) *small_mode = m->small_mode;
  // (partner blocks are reported as a negative split)
  if (split != nullptr) *split = m->split_blocks ? -m->split : m->split;
  return TU_OK;
}

tu_status tu_market_autotune(tu_market_t m, int reps, tu_tune_info* info) {
  TU_TRACE("tu_market_autotune");
  TU_TRY(check_live(m));
  if (m->path != TU_PATH_FUSED) return fail(m, TU_ERR_UNSUPPORTED, "the autotuner chooses fused-path shapes");
  if (reps < 1 || reps > 1000) return fail(m, TU_ERR_INVALID_ARG, "reps must be in [1, 1000]");
  TU_CK(m, cudaStreamSynchronize(m->stream));
  TU_TRY(drop_graph(m));
  const int64_t rows = m->N > m->M ? m->N : m->M;
  const int64_t tiles = (rows + kFusedOwnRows - 1) / kFusedOwnRows;
  const int64_t ptiles = ((m->N < m->M ? m->N : m->M) + kFusedPartnerRows - 1) / kFusedPartnerRows;
  // candidates (own-tile mode, shape code): the default shape first;
  // 128-row tiles and partner splits only where waves are few enough for
  // their granularity to matter; partner blocks where the partner matrix is
  // several times the L2 a block should fit
  std::vector<std::pair<int, int>> cand = {{1, 1}, {0, 1}};
  if (tiles < 4 * (int64_t)m->num_sms) cand.push_back({2, 1});
  if (tiles < 8 * (int64_t)m->num_sms && !m->wide)
    for (int s : {2, 3, 4, 6, 8})
      if (s <= ptiles) {
        cand.push_back({0, s});
        if (tiles < 2 * (int64_t)m->num_sms) cand.push_back({2, s});
      }
  const double partner_bytes = (double)(m->N > m->M ? m->N : m->M) * (double)m->kp * (is_fp8(m->dtype) ? 1.0 : 2.0);
  if (partner_bytes > 96e6 && tiles >= 2 * (int64_t)m->num_sms && !m->wide)
    for (int b : {2, 3, 4, 6})
      if (b <= ptiles) cand.push_back({0, -b});
  const int small0 = m->small_mode, split0 = m->split_blocks ? -m->split : m->split;
  double best = 0.0, ms_default = 0.0;
  int bi = -1;
  tu_status st = TU_OK;
  for (size_t i = 0; i < cand.size() && st == TU_OK; ++i) {
    double ms = 0.0;
    st = set_shape_code(m, cand[i].first, cand[i].second);
    if (st == TU_OK) st = time_shape(m, reps, &ms);
    if (st != TU_OK) break;
    if (i == 0) ms_default = ms;
    if (bi < 0 || ms < best) {
      best = ms;
      bi = (int)i;
    }
  }
  if (st != TU_OK) {
    set_shape_code(m, small0, split0);
    return st;
  }
  TU_TRY(set_shape_code(m, cand[bi].first, cand[bi].second));
  TU_TRY(clear_results(m));
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune[tune_key(m)] = TuneVal{cand[bi].first, cand[bi].second, best, ms_default};
  }
  if (info != nullptr) {
    info->small_tiles = cand[bi].first;
    info->split = cand[bi].second;
    info->ms = best;
    info->ms_default = ms_default;
    info->candidates = (int)cand.size();
  }
  return TU_OK;
}

tu_status tu_autotune_cache_save(const char* path) {
  if (path == nullptr) return TU_ERR_INVALID_ARG;
  std::ofstream f(path);
  if (!f) return TU_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  f << "{\"tu_autotune\": 1, \"entries\": [\n";
  size_t i = 0;
  for (const auto& kv : g_tune) {
    char line[320];
    snprintf(line, sizeof(line),
             "{\"n_bucket\": %d, \"m_bucket\": %d, \"kp\": %lld, \"dtype\": %d, \"sms\": %d, "
             "\"small_tiles\": %d, \"split\": %d, \"ms\": %.6g, \"ms_default\": %.6g}%s\n",
             kv.first.nb, kv.first.mb, (long long)kv.first.kp, kv.first.fmt, kv.first.sms, kv.second.small_mode,
             kv.second.split, kv.second.ms, kv.second.ms_default, ++i < g_tune.size() ? "," : "");
    f << line;
  }
  f << "]}\n";
  return f.good() ? TU_OK : TU_ERR_INVALID_ARG;
}

tu_status tu_autotune_cache_load(const char* path) {
  if (path == nullptr) return TU_ERR_INVALID_ARG;
  std::ifstream f(path);
  if (!f) return TU_ERR_INVALID_ARG;
  std::map<TuneKey, TuneVal> read;
  std::string line;
  while (std::getline(f, line)) {
    TuneKey k{};
    TuneVal v{};
    long long kp = 0;
    if (line.find("\"n_bucket\"") == std::string::npos) continue;
    if (sscanf(line.c_str(),
               " {\"n_bucket\": %d, \"m_bucket\": %d, \"kp\": %lld, \"dtype\": %d, \"sms\": %d, "
               "\"small_tiles\": %d, \"split\": %d, \"ms\": %lf, \"ms_default\": %lf",
               &k.nb, &k.mb, &kp, &k.fmt, &k.sms, &v.small_mode, &v.split, &v.ms, &v.ms_default) != 9)
      return TU_ERR_INVALID_ARG;
    if (v.small_mode < 0 || v.small_mode > 2 || v.split == 0 || v.split < -kMaxSplit || v.split > kMaxSplit)
      return TU_ERR_INVALID_ARG;
    k.kp = kp;
    read[k] = v;
  }
  std::lock_guard<std::mutex> lk(g_tune_mu);
  for (const auto& kv : read) g_tune[kv.first] = kv.second;
  return TU_OK;
}

void tu_autotune_cache_clear(void) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune.clear();
}

tu_status tu_relax_schedule(double omega, double tol, const int* done, const double* residual, int count,
                            double* omega_out) {
  if (!(omega == 0.0 || (omega >= 1.0 && omega < 2.0)) || !(tol >= 0.0) || count < 0) return TU_ERR_INVALID_ARG;
  if (count > 0 && (done == nullptr || residual == nullptr || omega_out == nullptr)) return TU_ERR_INVALID_ARG;
  RelaxControl ctl(omega);
  for (int i = 0; i < count; ++i) {
    if (done[i] < 1 || (i > 0 && done[i] <= done[i - 1])) return TU_ERR_INVALID_ARG;
    omega_out[i] = ctl.observe(done[i], residual[i], tol);
  }
  return TU_OK;
}

tu_status tu_market_set_translation(tu_market_t m, int enable) {
  TU_TRY(check_live(m));
  if (enable != 0 && enable != 1) return fail(m, TU_ERR_INVALID_ARG, "enable must be 0 or 1");
  if ((enable != 0) != m->translate && m->graph != nullptr) {
    // captured sweeps use the preparation of the previous setting
    TU_CK(m, cudaStreamSynchronize(m->stream));
    cudaGraphExecDestroy(m->graph);
    m->graph = nullptr;
    m->graph_sweeps = 0;
  }
  m->translate = enable != 0;
  return relax_reset(m);
}

tu_status tu_market_relax_update(tu_market_t m, double tol) {
  TU_TRY(check_live(m));
  if (!(tol >= 0.0)) return fail(m, TU_ERR_INVALID_ARG, "tol < 0");
  if (m->omega_cfg != 0.0 || m->done_ev == nullptr || m->query_sweeps == m->relax_seen) return TU_OK;
  const cudaError_t e = cudaEventQuery(m->done_ev);
  if (e == cudaErrorNotReady) return TU_OK;  // the last block is still running
  if (e != cudaSuccess) return fail_cuda(m, e, "cudaEventQuery");
  m->relax_seen = m->query_sweeps;
  const double r = m->query_host[kResXInf];
  if (!(r > tol) || !std::isfinite(r)) return TU_OK;
  const double next = m->relax.observe((int)(m->query_sweeps - m->relax_base), r, tol);
  if (next != *m->omega_host) TU_TRY(set_omega(m, next));
  return TU_OK;
}

tu_status tu_market_query(tu_market_t m, int* idle, double* residual, double* match_count, int64_t* sweeps) {
  TU_TRY(check_live(m));
  if (m->done_ev != nullptr) {
    const cudaError_t e = cudaEventQuery(m->done_ev);
    if (e == cudaErrorNotReady) {
      if (idle) *idle = 0;
      return TU_OK;
    }
    if (e != cudaSuccess) return fail_cuda(m, e, "cudaEventQuery");
    int err_word = 0;
    memcpy(&err_word, m->query_host + kResSlots, sizeof(int));
    if (err_word == kErrTimeout) return fail(m, TU_ERR_TIMEOUT, "a device-side wait ran out of its time limit");
    if (m->query_host[kResNonfin] > 0.0) return fail(m, TU_ERR_NONFINITE, "a computed potential is not finite");
  }
  if (idle) *idle = 1;
  if (residual) *residual = m->done_ev ? m->query_host[kResXInf] : INFINITY;
  if (match_count) *match_count = m->done_ev ? m->Y.sum_mass - m->query_host[kResYSq] : 0.0;
  if (sweeps) *sweeps = m->query_sweeps;
  return TU_OK;
}

int64_t tu_market_footprint(int64_t N, int64_t M, int64_t d, int path) {
  if (N < 1 || M < 1 || d < 1) return 0;
  const int64_t kp = path == TU_PATH_FUSED ? fused_row_length(d, false) : round_up(2 * d, kKBlock);
  const int64_t np = round_up(N, kRowPad), mp = round_up(M, kRowPad);
  int64_t bytes = (np + mp) * (8 + 8 + 4 + 8 + 4) + (int64_t)kMaxPartials * 5 * 8 + 4096;
  // staging for host factor uploads (two matrices of the larger side)
  bytes += 2 * (N > M ? N : M) * d * 4;
  if (path == TU_PATH_FUSED) {
    bytes += (N + M) * kp * 2 + (np > mp ? np : mp) * 4;  // factors, per-row shifts
    if (kp == kKBlock) bytes += (np + mp) * 32;              // the extra MMA's g / c operand
  } else {
    bytes += (N + M) * kp * 4 + N * round_up(M, 4) * 4 + M * round_up(N, 4) * 4;
  }
  return bytes;
}

tu_status tu_ipfp_solve(tu_market_t m, double tol, int max_iter, int warm_start, tu_solve_info* info) {
  TU_TRACE("tu_ipfp_solve");
  TU_TRY(check_live(m));
  if (!(tol >= 0.0) || max_iter < 0) return fail(m, TU_ERR_INVALID_ARG, "tol < 0 or max_iter < 0");
  if (!warm_start) {
    TU_CK(m, launch_reset_potentials(m, m->X));
    TU_CK(m, launch_reset_potentials(m, m->Y));
    TU_CK(m, launch_rescan(m));
  }
  TU_TRY(clear_results(m));
  // sweeps between host checks: planned from the measured decay (plan_block),
  // at most about 2e9 pair evaluations per check and 64 sweeps
  const double pairs = (double)m->N * (double)m->M;
  int block = (int)std::ceil(2e9 / pairs);
  if (block < 1) block = 1;
  if (block > 64) block = 64;
  int done = 0, last_k = 0;
  double r_prev = -1.0, r_last = -1.0;
  double res_inf = INFINITY, res_l1 = INFINITY;
  tu_status status = TU_ERR_NOT_CONVERGED;
  // over-relaxation (RelaxControl): omega is re-chosen after every block
  RelaxControl ctl(m->omega_cfg);
  const bool relax = ctl.enabled();
  if (relax && block > 16) block = 16;  // finer control of omega
  double omega = 1.0;
  if (relax) TU_TRY(set_omega(m, 1.0));
  while (true) {
    TU_TRY(certify(m, &res_inf, &res_l1));
    if (res_inf <= tol) {
      status = TU_OK;
      break;
    }
    if (done >= max_iter) break;
    // sweep until the residual folded into the X half-sweeps (state entering
    // the last sweep of a block) reaches tol, then certify the returned state
    while (done < max_iter) {
      int k = plan_block(last_k, r_prev, r_last, tol, block);
      if (k > max_iter - done) k = max_iter - done;
      TU_TRY(enqueue_sweeps(m, k));
      m->sweeps_enqueued += k;
      TU_TRY(read_results(m));
      done += k;
      const double r = m->results_host[kResXInf];
      r_prev = r_last;
      r_last = r;
      last_k = k;
      if (r <= tol) break;
      if (!relax) continue;
      const double next = ctl.observe(done, r, tol);
      if (next != omega) {
        omega = next;
        TU_TRY(set_omega(m, omega));
      }
    }
  }
  if (relax) TU_TRY(set_omega(m, m->omega_cfg > 1.0 ? m->omega_cfg : 1.0));
  // match count from the column equations (they hold after every v update):
  // sum_xy mu_xy = sum m - sum v^2
  TU_TRY(clear_results(m));
  TU_CK(m, launch_sum_sq(m, m->Y, 0));
  TU_TRY(read_results(m));
  const double match = m->Y.sum_mass - m->results_host[kResYSq];
  if (info != nullptr) {
    info->sweeps = done;
    info->status = status;
    info->residual_inf = res_inf;
    info->residual_l1 = res_l1;
    info->match_count = match;
  }
  TU_TRY(relax_reset(m));  // the asynchronous controller restarts after a solve
  if (status != TU_OK) m->last_error = "max_iter reached before the residual met tol";
  return status;
}

tu_status tu_ipfp_solve_ranking(tu_market_t m, int k, int64_t sample, int check_every, int patience,
                                double score_eps, int max_iter, int warm_start, tu_solve_info* info) {
  TU_TRACE("tu_ipfp_solve_ranking");
  TU_TRY(check_live(m));
  if (k < 1 || k > 63 || k > m->N || k > m->M || sample < 1 || check_every < 1 || patience < 1 ||
      !(score_eps >= 0.0) || max_iter < 0)
    return fail(m, TU_ERR_INVALID_ARG, "ranking-stability arguments out of range");
  if (!warm_start) {
    TU_CK(m, launch_reset_potentials(m, m->X));
    TU_CK(m, launch_reset_potentials(m, m->Y));
    TU_CK(m, launch_rescan(m));
  }
  TU_TRY(clear_results(m));
  // per side: the users checked and the list length (k + 1 when there is a next partner)
  const int64_t rows[2] = {sample < m->N ? sample : m->N, sample < m->M ? sample : m->M};
  const int kq[2] = {k + 1 <= m->M ? k + 1 : k, k + 1 <= m->N ? k + 1 : k};
  const size_t n0 = (size_t)rows[0] * kq[0], n1 = (size_t)rows[1] * kq[1], nidx = n0 + n1;
  const size_t hand = (size_t)(rows[0] > rows[1] ? rows[0] : rows[1]) * 64;
  // device: indices of both sides, their log mu, then (fused) the hand-over scratch
  int32_t* buf = nullptr;
  TU_TRY(dev_alloc(m, &buf, 2 * nidx + 2 * hand));
  int32_t* d_idx = buf;
  float* d_lmu = reinterpret_cast<float*>(buf + nidx);
  std::vector<int32_t> cur(nidx), prev(nidx);
  std::vector<float> score(nidx);
  auto rank_lists = [&]() -> tu_status {
    for (int side = 0; side < 2; ++side) {
      const size_t off = side == 0 ? 0 : n0;
      cudaError_t e = launch_prep(m, side == 0 ? m->Y : m->X, m->path == TU_PATH_FUSED ? 1 : 0, 0);
      if (e == cudaSuccess) {
        if (m->path == TU_PATH_FUSED) {
          float* hv = reinterpret_cast<float*>(buf + 2 * nidx);
          e = launch_fused_topk(m, side, kq[side], 0, rows[side], d_idx + off, d_lmu + off, hv,
                                buf + 2 * nidx + hand);
        } else {
          e = launch_topk(m, side, kq[side], 0, rows[side], d_idx + off, d_lmu + off);
        }
      }
      if (e != cudaSuccess) return fail_cuda(m, e, "ranked lists");
    }
    TU_CK(m, cudaMemcpyAsync(cur.data(), d_idx, nidx * sizeof(int32_t), cudaMemcpyDeviceToHost, m->stream));
    TU_CK(m, cudaMemcpyAsync(score.data(), d_lmu, nidx * sizeof(float), cudaMemcpyDeviceToHost, m->stream));
    TU_CK(m, cudaStreamSynchronize(m->stream));
    return TU_OK;
  };
  // positions separated from both neighbours by more than score_eps must hold the same partner
  auto same_rankings = [&]() -> bool {
    for (int side = 0; side < 2; ++side) {
      const size_t off = side == 0 ? 0 : n0;
      for (int64_t r = 0; r < rows[side]; ++r) {
        const size_t b = off + (size_t)r * kq[side];
        for (int j = 0; j < k; ++j) {
          const double above = j == 0 ? INFINITY : (double)score[b + j - 1] - score[b + j];
          const double below = j + 1 < kq[side] ? (double)score[b + j] - score[b + j + 1] : INFINITY;
          if (above > score_eps && below > score_eps && cur[b + j] != prev[b + j]) return false;
        }
      }
    }
    return true;
  };
  RelaxControl ctl(m->omega_cfg);
  double omega = 1.0;
  tu_status st = TU_OK;
  if (ctl.enabled()) st = set_omega(m, 1.0);
  int done = 0, stable = 0;
  bool have_prev = false;
  tu_status status = TU_ERR_NOT_CONVERGED;
  while (st == TU_OK && done < max_iter) {
    const int ks = (max_iter - done) < check_every ? (max_iter - done) : check_every;
    st = enqueue_sweeps(m, ks);
    if (st == TU_OK) st = read_results(m);
    if (st != TU_OK) break;
    m->sweeps_enqueued += ks;
    done += ks;
    if (ctl.enabled()) {
      const double next = ctl.observe(done, m->results_host[kResXInf], 0.0);
      if (next != omega && (st = set_omega(m, next)) != TU_OK) break;
      omega = next;
    }
    if ((st = rank_lists()) != TU_OK) break;
    stable = (have_prev && same_rankings()) ? stable + 1 : 0;
    prev.swap(cur);
    have_prev = true;
    if (stable >= patience) {
      status = TU_OK;
      break;
    }
  }
  dev_free(m, buf);
  if (st != TU_OK) return st;
  if (ctl.enabled()) TU_TRY(set_omega(m, m->omega_cfg > 1.0 ? m->omega_cfg : 1.0));
  double res_inf = INFINITY, res_l1 = INFINITY;
  TU_TRY(certify(m, &res_inf, &res_l1));
  TU_TRY(clear_results(m));
  TU_CK(m, launch_sum_sq(m, m->Y, 0));
  TU_TRY(read_results(m));
  if (info != nullptr) {
    info->sweeps = done;
    info->status = status;
    info->residual_inf = res_inf;
    info->residual_l1 = res_l1;
    info->match_count = m->Y.sum_mass - m->results_host[kResYSq];
  }
  if (status != TU_OK) m->last_error = "max_iter reached before the rankings were stable";
  return status;
}

tu_status tu_mu_block(tu_market_t m, int64_t x0, int64_t nx, int64_t y0, int64_t ny, float* out, int64_t ld) {
  TU_TRACE("tu_mu_block");
  TU_TRY(check_live(m));
  if (out == nullptr || x0 < 0 || y0 < 0 || nx < 0 || ny < 0 || x0 + nx > m->N || y0 + ny > m->M || ld < ny)
    return fail(m, TU_ERR_INVALID_ARG, "mu block out of range");
  if (nx == 0 || ny == 0) return TU_OK;
  const size_t bytes = (size_t)((nx - 1) * ld + ny) * sizeof(float);
  void* dst;
  bool host;
  TU_TRY(output_view(m, out, bytes, 0, &dst, &host));
  if (m->path == TU_PATH_FUSED) {
    // Y potentials prepared in log2 mode, then the tensor-core mu epilogue
    TU_CK(m, launch_prep(m, m->Y, 1, 0));
    TU_CK(m, launch_fused_mu(m, x0, nx, y0, ny, static_cast<float*>(dst), ld));
  } else {
    TU_CK(m, launch_mu_block(m, x0, nx, y0, ny, static_cast<float*>(dst), ld));
  }
  if (host) {
    // pitched copy: the caller's columns [ny, ld) of each row are left untouched
    TU_CK(m, cudaMemcpy2DAsync(out, (size_t)ld * sizeof(float), dst, (size_t)ld * sizeof(float),
                               (size_t)ny * sizeof(float), (size_t)nx, cudaMemcpyDeviceToHost, m->stream));
    TU_CK(m, cudaStreamSynchronize(m->stream));
  }
  return TU_OK;
}

tu_status tu_topk_partners(tu_market_t m, int side, int k, int64_t row0, int64_t nrows, int32_t* idx,
                           float* log_mu) {
  TU_TRACE("tu_topk_partners");
  TU_TRY(check_live(m));
  const int64_t rows = side == 0 ? m->N : m->M;
  const int64_t partners = side == 0 ? m->M : m->N;
  if ((side != 0 && side != 1) || idx == nullptr || k < 1 || k > 64 || k > partners || row0 < 0 || nrows < 0 ||
      row0 + nrows > rows)
    return fail(m, TU_ERR_INVALID_ARG, "topk arguments out of range");
  if (nrows == 0) return TU_OK;
  const size_t ib = (size_t)nrows * k * sizeof(int32_t), vb = (size_t)nrows * k * sizeof(float);
  void *di, *dv = nullptr;
  bool hi, hv = false;
  // host outputs share the staging buffer: size it for both before either
  // view points into it (growing it later would free the first view's block)
  if (!is_device_ptr(idx) || (log_mu != nullptr && !is_device_ptr(log_mu)))
    TU_TRY(ensure_staging(m, (size_t)round_up((int64_t)ib, 256) + vb));
  TU_TRY(output_view(m, idx, ib, 0, &di, &hi));
  if (log_mu != nullptr) TU_TRY(output_view(m, log_mu, vb, round_up((int64_t)ib, 256), &dv, &hv));
  if (m->path == TU_PATH_FUSED) {
    // partner potentials in log2 mode; per-row candidate lists of the second
    // column half go through a nrows x k scratch buffer
    const size_t hb = (size_t)nrows * k * (sizeof(float) + sizeof(int32_t));
    if (m->aux_bytes < hb) {
      dev_free(m, m->aux);  // stream-ordered: after the passes that used it
      m->aux_bytes = 0;
      TU_TRY(dev_alloc_bytes(m, &m->aux, hb));
      m->aux_bytes = hb;
    }
    float* hv = static_cast<float*>(m->aux);
    int32_t* hi_ = reinterpret_cast<int32_t*>(hv + (size_t)nrows * k);
    TU_CK(m, launch_prep(m, side == 0 ? m->Y : m->X, 1, 0));
    TU_CK(m, launch_fused_topk(m, side, k, row0, nrows, static_cast<int32_t*>(di), static_cast<float*>(dv), hv, hi_));
  } else {
    TU_CK(m, launch_topk(m, side, k, row0, nrows, static_cast<int32_t*>(di), static_cast<float*>(dv)));
  }
  if (hi) TU_CK(m, cudaMemcpyAsync(idx, di, ib, cudaMemcpyDeviceToHost, m->stream));
  if (hv) TU_CK(m, cudaMemcpyAsync(log_mu, dv, vb, cudaMemcpyDeviceToHost, m->stream));
  if (hi || hv) TU_CK(m, cudaStreamSynchronize(m->stream));
  return TU_OK;
}

tu_status tu_get_potentials(tu_market_t m, float* log_u, float* log_v) {
  TU_TRACE("tu_get_potentials");
  TU_TRY(check_live(m));
  Side* sides[2] = {&m->X, &m->Y};
  float* outs[2] = {log_u, log_v};
  for (int i = 0; i < 2; ++i) {
    if (outs[i] == nullptr) continue;
    const size_t bytes = (size_t)sides[i]->rows * sizeof(float);
    void* dst;
    bool host;
    TU_TRY(output_view(m, outs[i], bytes, 0, &dst, &host));
    TU_CK(m, launch_get_potentials(m, *sides[i], static_cast<float*>(dst)));
    if (host) {
      TU_CK(m, cudaMemcpyAsync(outs[i], dst, bytes, cudaMemcpyDeviceToHost, m->stream));
      TU_CK(m, cudaStreamSynchronize(m->stream));
    }
  }
  return TU_OK;
}

tu_status tu_get_potentials_f64(tu_market_t m, double* log_u, double* log_v) {
  TU_TRACE("tu_get_potentials_f64");
  TU_TRY(check_live(m));
  Side* sides[2] = {&m->X, &m->Y};
  double* outs[2] = {log_u, log_v};
  for (int i = 0; i < 2; ++i) {
    if (outs[i] == nullptr) continue;
    // the state is written back after every block of sweeps, so it is the array itself
    TU_CK(m, cudaMemcpyAsync(outs[i], sides[i]->log_u, (size_t)sides[i]->rows * sizeof(double), cudaMemcpyDefault,
                             m->stream));
  }
  TU_CK(m, cudaStreamSynchronize(m->stream));
  return TU_OK;
}

tu_status tu_get_potentials_range_f64(tu_market_t m, int side, int64_t lo, int64_t hi, double* out) {
  TU_TRACE("tu_get_potentials_range_f64");
  TU_TRY(check_live(m));
  if (side != 0 && side != 1) return fail(m, TU_ERR_INVALID_ARG, "side must be 0 or 1");
  const Side& s = side == 0 ? m->X : m->Y;
  if (lo < 0 || hi < lo || hi > s.rows) return fail(m, TU_ERR_INVALID_ARG, "range outside the side's users");
  if (out == nullptr && hi > lo) return fail(m, TU_ERR_INVALID_ARG, "null output");
  if (hi > lo)
    TU_CK(m, cudaMemcpyAsync(out, s.log_u + lo, (size_t)(hi - lo) * sizeof(double), cudaMemcpyDefault, m->stream));
  TU_CK(m, cudaStreamSynchronize(m->stream));
  return TU_OK;
}

tu_status tu_ipfp_half_sweep_range(tu_market_t m, int side, int64_t lo, int64_t hi, double* residual_out) {
  TU_TRACE("tu_ipfp_half_sweep_range");
  TU_TRY(check_live(m));
  if (side != 0 && side != 1) return fail(m, TU_ERR_INVALID_ARG, "side must be 0 or 1");
  if (m->path != TU_PATH_FUSED) return fail(m, TU_ERR_UNSUPPORTED, "row ranges need the fused path");
  Side& own = side == 0 ? m->X : m->Y;
  Side& partner = side == 0 ? m->Y : m->X;
  if (lo < 0 || hi < lo || hi > own.rows) return fail(m, TU_ERR_INVALID_ARG, "range outside the side's users");
  TU_TRY(clear_results(m));
  if (hi > lo) {
    // no translation step: a shard's caller owns the step (it needs both sides' global sums)
    TU_CK(m, launch_prep(m, partner, 1, 0));
    int nparts = 0;
    TU_CK(m, launch_fused_halfsweep(m, side, residual_out ? kResidualExact : kResidualNone, 1, &nparts, lo, hi - lo));
    // the partials only; then the side's groups and the market's scalars from
    // the stored potentials (the next preparation reads the side's shift)
    TU_CK(m, launch_finalize(m, nparts, 1, residual_out ? 1 : 0, 0, 0));
    TU_CK(m, launch_rescan(m));
  }
  TU_TRY(read_results(m));
  if (residual_out != nullptr) {
    residual_out[0] = m->results_host[kResXInf];
    residual_out[1] = m->results_host[kResXL1];
  }
  return TU_OK;
}

tu_status tu_set_potentials_f64(tu_market_t m, const double* log_u, const double* log_v) {
  TU_TRACE("tu_set_potentials_f64");
  TU_TRY(check_live(m));
  Side* sides[2] = {&m->X, &m->Y};
  const double* ins[2] = {log_u, log_v};
  TU_TRY(ensure_staging(m, (size_t)(m->N > m->M ? m->N : m->M) * sizeof(double)));
  for (int i = 0; i < 2; ++i) {
    if (ins[i] == nullptr) continue;
    const void* src = nullptr;
    TU_TRY(device_view(m, ins[i], (size_t)sides[i]->rows * sizeof(double), 0, &src));
    TU_CK(m, launch_set_potentials64(m, *sides[i], static_cast<const double*>(src)));
    TU_CK(m, cudaStreamSynchronize(m->stream));
  }
  TU_CK(m, launch_rescan(m));
  return relax_reset(m);
}

tu_status tu_set_potentials(tu_market_t m, const float* log_u, const float* log_v) {
  TU_TRACE("tu_set_potentials");
  TU_TRY(check_live(m));
  Side* sides[2] = {&m->X, &m->Y};
  const float* ins[2] = {log_u, log_v};
  TU_TRY(ensure_staging(m, (size_t)(m->N > m->M ? m->N : m->M) * sizeof(float)));
  for (int i = 0; i < 2; ++i) {
    if (ins[i] == nullptr) continue;
    const void* src = nullptr;
    TU_TRY(device_view(m, ins[i], (size_t)sides[i]->rows * sizeof(float), 0, &src));
    TU_CK(m, launch_set_potentials(m, *sides[i], static_cast<const float*>(src)));
    TU_CK(m, cudaStreamSynchronize(m->stream));
  }
  TU_CK(m, launch_rescan(m));
  return relax_reset(m);
}

}  // extern "C"
