// topk.cu -- outputs of a solved dense-path market: blocks of mu (Eq.
// stable_condition, Alg. 1 final line) and ranked partner lists (top-k of log
// mu per user), read from the materialised kernel (the fused path forms them
// in the tensor-core pipeline, fused.cu).
//
// log mu_xy = phi_xy / (2 sigma) + log u_x + log v_y
//           = phi_hat_xy / (2 sigma) + ell_x + ell_y,   ell = log u + b / (2 sigma),
// where phi_hat is the bias-free surplus and log A-hat = phi_hat / (2 sigma).
#include "tu_internal.cuh"

namespace tu {

namespace {

constexpr int kMaxK = 64;

// log A-hat of (own r, partner c) at Ahat[r * rs + c * cs] (A-hat read row- or column-wise)
struct ScoreSrc {
  const float* Ahat;
  int64_t rs, cs;
  __device__ __forceinline__ float phi2s(int64_t r, int64_t c) const { return logf(Ahat[r * rs + c * cs]); }
};

__global__ void k_mu_block(ScoreSrc src, const double* __restrict__ ell_x, const double* __restrict__ ell_y, int64_t x0,
                           int64_t nx, int64_t y0, int64_t ny, float* __restrict__ out, int64_t ld) {
  const int64_t y = y0 + (int64_t)blockIdx.x * 32 + threadIdx.x;
  if (y >= y0 + ny) return;
  // rows in steps of the grid's height (at most 65,535 blocks of 8 rows)
  for (int64_t x = x0 + (int64_t)blockIdx.y * 8 + threadIdx.y; x < x0 + nx; x += (int64_t)gridDim.y * 8) {
    const double lm = (double)src.phi2s(x, y) + ell_x[x] + ell_y[y];
    out[(x - x0) * ld + (y - y0)] = (float)exp(lm);
  }
}

// One warp per own row of a row-major matrix A (A-hat for side 0, its
// resident transpose for side 1, so every row is read coalesced, float4 per
// lane). The order of log mu within a row is the order of the FP32 score
// log2(A[r][c]) + g_c, with g = (ell - shift) log2(e) of the partner side
// (the partner vector in log2 mode, -inf padded); each lane keeps a sorted
// top-k of the partners it visits (increasing index, so equal scores keep
// the lower index first) behind a threshold test, in shared memory for
// k <= kSharedK (local memory otherwise); then the 32 lists are merged by k
// rounds of a warp-wide argmax, and log mu of the k winners is evaluated in
// FP64 from A-hat and the potentials.
constexpr int kSharedK = 16;

template <bool SHARED>
__global__ void __launch_bounds__(256) k_topk(const float* __restrict__ A, int64_t ld, const float* __restrict__ g,
                                              const double* __restrict__ ell_own, const double* __restrict__ ell_par,
                                              int k, int64_t row0, int64_t nrows, int32_t* __restrict__ idx,
                                              float* __restrict__ logmu) {
  __shared__ float s_v[SHARED ? kSharedK : 1][256];
  __shared__ int32_t s_i[SHARED ? kSharedK : 1][256];
  float l_v[SHARED ? 1 : kMaxK];
  int32_t l_i[SHARED ? 1 : kMaxK];
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int64_t r = (int64_t)blockIdx.x * 8 + warp;
  if (r >= nrows) return;  // the whole warp leaves: no block-wide synchronisation follows
  const int64_t row = row0 + r;
  auto V = [&](int i) -> float& {
    if constexpr (SHARED) return s_v[i][threadIdx.x];
    else return l_v[i];
  };
  auto I = [&](int i) -> int32_t& {
    if constexpr (SHARED) return s_i[i][threadIdx.x];
    else return l_i[i];
  };
  int cnt = 0;
  float thr = -INFINITY;  // the k-th best of this lane once it holds k entries
  auto insert = [&](float sc, int32_t c) {
    int pos = cnt < k ? cnt : k - 1;
    while (pos > 0 && sc > V(pos - 1)) {
      V(pos) = V(pos - 1);
      I(pos) = I(pos - 1);
      --pos;
    }
    V(pos) = sc;
    I(pos) = c;
    if (cnt < k) ++cnt;
    if (cnt == k) thr = V(k - 1);
  };
  const float4* a4 = reinterpret_cast<const float4*>(A + row * ld);
  const float4* g4 = reinterpret_cast<const float4*>(g);
  const int64_t n4 = ld / 4;
  // Row bound: the k-th largest of the 32 lanes' best scores is at most the
  // row's k-th best (those k scores are distinct entries of the lists), so a
  // score below it cannot be listed; refreshed every 8 steps (k <= 32).
  float row_lb = -INFINITY;
  int step = 0;
  // warp-uniform trip count (the bound's shuffles need every lane); lanes past
  // the row's end see -inf scores
  for (int64_t q0 = 0; q0 < n4; q0 += 32, ++step) {
    const int64_t q = q0 + lane;
    float sc[4] = {-INFINITY, -INFINITY, -INFINITY, -INFINITY};
    if (q < n4) {
      const float4 av = a4[q];
      const float4 gv = __ldg(g4 + q);
      sc[0] = log2f(av.x) + gv.x;
      sc[1] = log2f(av.y) + gv.y;
      sc[2] = log2f(av.z) + gv.z;
      sc[3] = log2f(av.w) + gv.w;
    }
    const int32_t c = (int32_t)(4 * q);
#pragma unroll
    for (int e = 0; e < 4; ++e)
      if (sc[e] > thr && sc[e] >= row_lb) insert(sc[e], c + e);
    if (k <= 32 && (step & 7) == 7) {
      float m = cnt > 0 ? V(0) : -INFINITY;
      float kth = -INFINITY;
      for (int j = 0; j < k; ++j) {
        float best = m;
        for (int o = 16; o > 0; o >>= 1) best = fmaxf(best, __shfl_xor_sync(0xffffffffu, best, o));
        kth = best;
        // remove one occurrence of the maximum (the lowest lane holding it)
        const unsigned holders = __ballot_sync(0xffffffffu, m == best);
        if (lane == __ffs(holders) - 1) m = -INFINITY;
      }
      row_lb = kth;
    }
  }
  const double base = ell_own[row];
  int head = 0;
  for (int out_i = 0; out_i < k; ++out_i) {
    float bs = (head < cnt) ? V(head) : -INFINITY;
    int bi = (head < cnt) ? I(head) : 0x7fffffff;
    int bl = lane;
    for (int o = 16; o > 0; o >>= 1) {
      const float os = __shfl_xor_sync(0xffffffffu, bs, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      const int ol = __shfl_xor_sync(0xffffffffu, bl, o);
      if (os > bs || (os == bs && oi < bi)) {
        bs = os;
        bi = oi;
        bl = ol;
      }
    }
    if (lane == bl) ++head;
    if (lane == 0) {
      idx[r * k + out_i] = bi;
      if (logmu != nullptr) logmu[r * k + out_i] = (float)(log((double)A[row * ld + bi]) + ell_par[bi] + base);
    }
  }
}

}  // namespace

static ScoreSrc make_src(tu_market* m, int side) {
  ScoreSrc s{};
  s.Ahat = m->Ahat;
  s.rs = side == 0 ? m->ldA : 1;
  s.cs = side == 0 ? 1 : m->ldA;
  return s;
}

cudaError_t launch_mu_block(tu_market* m, int64_t x0, int64_t nx, int64_t y0, int64_t ny, float* out, int64_t ld) {
  dim3 block(32, 8);
  const int64_t row_blocks = (nx + 7) / 8;
  dim3 grid((unsigned)((ny + 31) / 32), (unsigned)(row_blocks < 65535 ? row_blocks : 65535));
  k_mu_block<<<grid, block, 0, m->stream>>>(make_src(m, 0), m->X.ell, m->Y.ell, x0, nx, y0, ny, out, ld);
  return cudaGetLastError();
}

cudaError_t launch_topk(tu_market* m, int side, int k, int64_t row0, int64_t nrows, int32_t* idx, float* logmu) {
  Side& own = side == 0 ? m->X : m->Y;
  Side& par = side == 0 ? m->Y : m->X;
  // the partner vector in log2 mode: g = (ell - shift) log2(e), -inf padded
  cudaError_t e = launch_prep(m, par, 1, 0);
  if (e != cudaSuccess) return e;
  const float* A = side == 0 ? m->Ahat : m->AhatT;
  const int64_t ld = side == 0 ? m->ldA : m->ldN;
  const unsigned grid = (unsigned)((nrows + 7) / 8);
  if (k <= kSharedK)
    k_topk<true><<<grid, 256, 0, m->stream>>>(A, ld, par.pvec, own.ell, par.ell, k, row0, nrows, idx, logmu);
  else
    k_topk<false><<<grid, 256, 0, m->stream>>>(A, ld, par.pvec, own.ell, par.ell, k, row0, nrows, idx, logmu);
  return cudaGetLastError();
}

}  // namespace tu
