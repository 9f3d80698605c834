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
  const int64_t x = x0 + (int64_t)blockIdx.y * 8 + threadIdx.y;
  if (x >= x0 + nx || y >= y0 + ny) return;
  const double lm = (double)src.phi2s(x, y) + ell_x[x] + ell_y[y];
  out[(x - x0) * ld + (y - y0)] = (float)exp(lm);
}

// One warp per own row: each lane keeps a sorted top-k of the partners it
// visits (increasing index, so equal scores keep the lower index first), then
// the 32 lists are merged by k rounds of a warp-wide argmax.
__global__ void __launch_bounds__(256) k_topk(ScoreSrc src, const double* __restrict__ ell_own,
                                              const double* __restrict__ ell_par, int64_t partners, int k,
                                              int64_t row0, int64_t nrows, int32_t* __restrict__ idx,
                                              float* __restrict__ logmu) {
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int64_t r = (int64_t)blockIdx.x * 8 + warp;
  if (r >= nrows) return;
  const int64_t row = row0 + r;
  float sv[kMaxK];
  int si[kMaxK];
  int cnt = 0;
  for (int64_t c = lane; c < partners; c += 32) {
    const float s = (float)((double)src.phi2s(row, c) + ell_par[c]);
    if (cnt == k && !(s > sv[k - 1])) continue;
    int pos = (cnt < k) ? cnt : k - 1;
    while (pos > 0 && s > sv[pos - 1]) {
      sv[pos] = sv[pos - 1];
      si[pos] = si[pos - 1];
      --pos;
    }
    sv[pos] = s;
    si[pos] = (int)c;
    if (cnt < k) ++cnt;
  }
  const double base = ell_own[row];
  int head = 0;
  for (int out_i = 0; out_i < k; ++out_i) {
    float bs = (head < cnt) ? sv[head] : -INFINITY;
    int bi = (head < cnt) ? si[head] : 0x7fffffff;
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
      if (logmu != nullptr) logmu[r * k + out_i] = (float)((double)bs + base);
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
  dim3 grid((unsigned)((ny + 31) / 32), (unsigned)((nx + 7) / 8));
  k_mu_block<<<grid, block, 0, m->stream>>>(make_src(m, 0), m->X.ell, m->Y.ell, x0, nx, y0, ny, out, ld);
  return cudaGetLastError();
}

cudaError_t launch_topk(tu_market* m, int side, int k, int64_t row0, int64_t nrows, int32_t* idx, float* logmu) {
  const Side& own = side == 0 ? m->X : m->Y;
  const Side& par = side == 0 ? m->Y : m->X;
  const unsigned grid = (unsigned)((nrows + 7) / 8);
  k_topk<<<grid, 256, 0, m->stream>>>(make_src(m, side), own.ell, par.ell, par.rows, k, row0, nrows, idx, logmu);
  return cudaGetLastError();
}

}  // namespace tu
