// reduce.cu -- O(N + M) kernels around the half-sweeps: factor packing, side
// initialisation, the partner-potential preparation that precedes every
// half-sweep, and the FP64 reductions that close it.
#include "tu_internal.cuh"

#include <cuda_fp8.h>

namespace tu {

namespace {

constexpr int kThreads = 256;

__global__ void k_pack_factors(const void* __restrict__ A, const void* __restrict__ B, int src_dtype,
                               int64_t rows, int64_t d, int64_t kp, __nv_bfloat16* __restrict__ out16,
                               float* __restrict__ out32) {
  // [A | B | 0] packed row-major rows x kp: the inner product of two packed rows
  // is <f_x, g_y> + <k_x, l_y> (Sec. 3.3), i.e. Phi = [F | K] [G | L]^T.
  const int64_t total = rows * kp;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = i / kp;
    const int64_t k = i - r * kp;
    float v = 0.0f;
    const void* src = nullptr;
    int64_t off = 0;
    if (k < d) {
      src = A;
      off = r * d + k;
    } else if (k < 2 * d) {
      src = B;
      off = r * d + (k - d);
    }
    if (src != nullptr) {
      if (src_dtype == TU_DTYPE_BF16) {
        v = __bfloat162float(reinterpret_cast<const __nv_bfloat16*>(src)[off]);
      } else {
        v = reinterpret_cast<const float*>(src)[off];
      }
    }
    if (out16 != nullptr) out16[i] = __float2bfloat16_rn(v);
    if (out32 != nullptr) out32[i] = v;
  }
}

// Largest |entry| of two FP32 arrays of `count` entries each (non-negative
// floats order like their bit patterns, so an unsigned atomicMax is exact).
__global__ void k_max_abs(const float* __restrict__ A, const float* __restrict__ B, int64_t count,
                          unsigned int* __restrict__ out) {
  __shared__ float red[kThreads / 32];
  float best = 0.0f;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
    const float a = fmaxf(fabsf(A[i]), fabsf(B[i]));
    // fmaxf drops a NaN operand: a NaN entry counts as +inf, so the host's finiteness check sees it
    best = (isnan(A[i]) || isnan(B[i])) ? INFINITY : fmaxf(best, a);
  }
  for (int o = 16; o > 0; o >>= 1) best = fmaxf(best, __shfl_xor_sync(0xffffffffu, best, o));
  if (threadIdx.x % 32 == 0) red[threadIdx.x / 32] = best;
  __syncthreads();
  if (threadIdx.x == 0) {
    float b = 0.0f;
    for (int w = 0; w < kThreads / 32; ++w) b = fmaxf(b, red[w]);
    atomicMax(out, __float_as_uint(b));
  }
}

// FP8 packing with per-row scales (one warp per row): row r of the output is
// [A_r | B_r | 0] * 2^-k_r rounded to the nearest e4m3 value (ties to even,
// saturating at +-448), kp bytes, with k_r the smallest integer such that
// max_i |entry| <= 448 * 2^k_r (exact: 448 = 0.875 * 2^9 and frexpf is exact),
// and fs[r] = 2^k_r the scale that multiplies the row back; an all-zero row
// has k_r = 0. With side_k != kPerRowScale every row takes k_r = side_k (one
// scale per side). Rows [rows, rows_pad) get fs = 1. A NaN or infinite entry
// sets *bad.
__global__ void k_pack_fp8_rows(const float* __restrict__ A, const float* __restrict__ B, int64_t rows,
                                int64_t rows_pad, int64_t d, int64_t kp, int side_k, uint8_t* __restrict__ out,
                                float* __restrict__ fs, unsigned int* __restrict__ bad) {
  const int lane = threadIdx.x % 32;
  const int64_t wpb = blockDim.x / 32;
  for (int64_t r = blockIdx.x * wpb + threadIdx.x / 32; r < rows_pad; r += (int64_t)gridDim.x * wpb) {
    if (r >= rows) {
      if (lane == 0) fs[r] = 1.0f;
      continue;
    }
    float mx = 0.0f;
    bool nonfinite = false;
    for (int64_t i = lane; i < 2 * d; i += 32) {
      const float v = i < d ? A[r * d + i] : B[r * d + (i - d)];
      nonfinite |= !isfinite(v);
      mx = fmaxf(mx, fabsf(v));
    }
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (__any_sync(0xffffffffu, nonfinite)) {
      if (lane == 0) atomicOr(bad, 1u);
      continue;
    }
    int k = side_k;
    if (side_k == kPerRowScale && mx > 0.0f) {
      int e = 0;
      frexpf(mx, &e);
      k = mx <= ldexpf(448.0f, e - 9) ? e - 9 : e - 8;
      if (k < -100) k = -100;  // (rows of subnormal size: 2^100 keeps the scaled entries finite)
    } else if (side_k == kPerRowScale) {
      k = 0;
    }
    const float inv = ldexpf(1.0f, -k);
    if (lane == 0) fs[r] = ldexpf(1.0f, k);
    for (int64_t i = lane; i < kp; i += 32) {
      float v = 0.0f;
      if (i < d) {
        v = A[r * d + i];
      } else if (i < 2 * d) {
        v = B[r * d + (i - d)];
      }
      out[r * kp + i] = (uint8_t)__nv_cvt_float_to_fp8(v * inv, __NV_SATFINITE, __NV_E4M3);
    }
  }
}

// FP8 packing of caller-quantized rows: [A_r | B_r | 0] copied as bytes (kp
// per row), fs[r] = sc[r]; rows [rows, rows_pad) get fs = 1. A non-finite
// scale sets *bad.
__global__ void k_pack_fp8_bytes(const uint8_t* __restrict__ A, const uint8_t* __restrict__ B,
                                 const float* __restrict__ sc, int64_t rows, int64_t rows_pad, int64_t d, int64_t kp,
                                 uint8_t* __restrict__ out, float* __restrict__ fs, unsigned int* __restrict__ bad) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < rows * kp;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = i / kp;
    const int64_t k = i - r * kp;
    uint8_t v = 0;
    if (k < d) {
      v = A[r * d + k];
    } else if (k < 2 * d) {
      v = B[r * d + (k - d)];
    }
    out[i] = v;
  }
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < rows_pad;
       r += (int64_t)gridDim.x * blockDim.x) {
    const float v = r < rows ? sc[r] : 1.0f;
    if (!isfinite(v)) atomicOr(bad, 1u);
    fs[r] = v;
  }
}

__global__ void k_init_side(const float* __restrict__ bias, int has_bias, float inv2s, int64_t rows,
                            int64_t rows_pad, float* __restrict__ b2s, double* __restrict__ log_u,
                            double* __restrict__ ell) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < rows_pad;
       i += (int64_t)gridDim.x * blockDim.x) {
    float b = 0.0f;
    if (has_bias && i < rows) b = (float)((double)bias[i] * (double)inv2s);
    if (b2s != nullptr) b2s[i] = b;
    log_u[i] = 0.0;  // u = 1 (Alg. 1 / Alg. 2 initialisation)
    ell[i] = (i < rows) ? (double)b : 0.0;
  }
}

__global__ void k_set_potentials(const float* __restrict__ src, const float* __restrict__ b2s, int64_t rows,
                                 double* __restrict__ log_u, double* __restrict__ ell) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < rows;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double lu = (src != nullptr) ? (double)src[i] : 0.0;
    log_u[i] = lu;
    ell[i] = (b2s != nullptr) ? lu + (double)b2s[i] : lu;
  }
}

__global__ void k_set_potentials64(const double* __restrict__ src, const float* __restrict__ b2s, int64_t rows,
                                   double* __restrict__ log_u, double* __restrict__ ell) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < rows;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double lu = src[i];
    log_u[i] = lu;
    ell[i] = (b2s != nullptr) ? lu + (double)b2s[i] : lu;
  }
}

__global__ void k_get_potentials(const double* __restrict__ log_u, int64_t rows, float* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < rows;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (float)log_u[i];
}

__global__ void k_row_norm_max(const float* __restrict__ f32, const __nv_bfloat16* __restrict__ f16,
                               const uint8_t* __restrict__ f8, const float* __restrict__ fs, int64_t rows,
                               int64_t kp, unsigned int* __restrict__ out) {
  __shared__ float red[kThreads / 32];
  float best = 0.0f;
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  for (int64_t r = blockIdx.x * (int64_t)(kThreads / 32) + warp; r < rows;
       r += (int64_t)gridDim.x * (kThreads / 32)) {
    float s = 0.0f;
    for (int64_t k = lane; k < kp; k += 32) {
      float v;
      if (f8 != nullptr) {
        const __half_raw h = __nv_cvt_fp8_to_halfraw((__nv_fp8_storage_t)f8[r * kp + k], __NV_E4M3);
        v = __half2float(__half(h)) * fs[r];
      } else {
        v = f32 ? f32[r * kp + k] : __bfloat162float(f16[r * kp + k]);
      }
      s = fmaf(v, v, s);
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    const float nrm = sqrtf(s);
    // fmaxf drops a NaN operand: a row with a NaN entry counts as an infinite norm
    best = isnan(nrm) ? INFINITY : fmaxf(best, nrm);
  }
  if (lane == 0) red[warp] = best;
  __syncthreads();
  if (threadIdx.x == 0) {
    float b = 0.0f;
    for (int w = 0; w < kThreads / 32; ++w) b = fmaxf(b, red[w]);
    atomicMax(out, __float_as_uint(b));  // non-negative floats order like their bit patterns
  }
}

// Partner preparation: the vector the half-sweep consumes, from the partner's
// stored ell and its maximum (a per-market scalar kept by the finalize
// kernels): fused_mode 1: (ell - max) * log2(e), padding -inf (exp2 of it is
// 0); fused_mode 0: exp(ell - max), padding 0. The vector depends on
// ell - max ell only, so no translation step or offset changes it; thread 0
// of block 0 records the pass's scalars (prep_scalars: its translation step,
// the partner shift it adds back and the own offset). No other thread reads
// the scalars it writes.
__global__ void k_prep(const double* __restrict__ ell, int64_t rows, int64_t rows_pad, double* __restrict__ st,
                       int own, int translate, int fused_mode, float* __restrict__ out, uint4* __restrict__ fold,
                       float inv_c) {
  const double top = st[kStLmax + (1 - own)];
  if (blockIdx.x == 0 && threadIdx.x == 0) prep_scalars(st, own, translate);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < rows_pad;
       i += (int64_t)gridDim.x * blockDim.x) {
    float v;
    if (i < rows) {
      // the FP64 state is rounded once, to the FP32 vector the half-sweep streams
      const double z = ell[i] - top;
      v = fused_mode ? (float)(z * 1.4426950408889634) : (float)exp(z);
    } else {
      v = fused_mode ? -INFINITY : 0.0f;
    }
    out[i] = v;
    if (fold != nullptr) write_fold_row(fold, i, v, inv_c);
  }
}

// Groups of a side's stored potentials (one warp per 32 rows), as a half-sweep
// writes them for the rows it updates.
__global__ void k_scan_groups(const double* __restrict__ log_u, const double* __restrict__ ell, int64_t rows,
                              float4* __restrict__ grp) {
  const int64_t ng = (rows + kGroupRows - 1) / kGroupRows;
  const int lane = threadIdx.x % 32;
  for (int64_t g = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / 32; g < ng;
       g += (int64_t)gridDim.x * blockDim.x / 32) {
    const int64_t r = g * kGroupRows + lane;
    const bool valid = r < rows;
    const float4 gv = warp_group(valid ? log_u[r] : 0.0, valid ? ell[r] : 0.0, valid);
    if (lane == 0) grp[g] = gv;
  }
}

// Scalars of both sides from their groups (one block): shifts and sums,
// offsets cleared, and tau for the next half-sweep, which updates X against Y.
__global__ void k_rescan_scalars(const float4* __restrict__ grp_x, int64_t ng_x, const float4* __restrict__ grp_y,
                                 int64_t ng_y, double dm_next, double* __restrict__ st) {
  __shared__ float red[2 * kThreads / 32];
  const GroupTotal x = block_reduce_groups(grp_x, ng_x, red);
  const GroupTotal y = block_reduce_groups(grp_y, ng_y, red);
  if (threadIdx.x == 0) rescan_scalars(st, x, y, dm_next);
}

// End of a block of sweeps: write the sides' offsets into their arrays (the
// scalars are folded by k_flush_scalars afterwards, so every block reads the
// offsets before any is cleared).
__global__ void k_flush(double* __restrict__ lu_x, double* __restrict__ ell_x, int64_t nx, double* __restrict__ lu_y,
                        double* __restrict__ ell_y, int64_t ny, const double* __restrict__ st) {
  const double ox = st[kStOff + 0], oy = st[kStOff + 1];
  const int64_t n = nx > ny ? nx : ny;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    if (ox != 0.0 && i < nx) {
      lu_x[i] += ox;
      ell_x[i] += ox;
    }
    if (oy != 0.0 && i < ny) {
      lu_y[i] += oy;
      ell_y[i] += oy;
    }
  }
}

__global__ void k_flush_scalars(double* __restrict__ st) {
  for (int s = 0; s < 2; ++s) {
    st[kStLmax + s] += st[kStOff + s];
    st[kStOff + s] = 0.0;
  }
}

// FP64 reduction of the per-CTA partials (max r/n, sum |r|, sum u^2, non-finite
// count). After a pass that updated its side (update), also that side's groups
// into the market scalars (finish_scalars), with the same routine and block
// size as the batched finalize.
__global__ void k_finalize(const double* __restrict__ partials, int nparts, int is_x, int residual, int update,
                           const float4* __restrict__ grp, int64_t ngroups, double dm_next, double* __restrict__ st,
                           double* __restrict__ results) {
  __shared__ double red[4][kThreads / 32];
  __shared__ float redf[2 * kThreads / 32];
  double mx = 0.0, l1 = 0.0, sq = 0.0, nf = 0.0;
  for (int i = threadIdx.x; i < nparts; i += blockDim.x) {
    mx = fmax(mx, partials[4 * i + 0]);
    l1 += partials[4 * i + 1];
    sq += partials[4 * i + 2];
    nf += partials[4 * i + 3];
  }
  for (int o = 16; o > 0; o >>= 1) {
    mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    l1 += __shfl_xor_sync(0xffffffffu, l1, o);
    sq += __shfl_xor_sync(0xffffffffu, sq, o);
    nf += __shfl_xor_sync(0xffffffffu, nf, o);
  }
  const int w = threadIdx.x / 32;
  if (threadIdx.x % 32 == 0) {
    red[0][w] = mx;
    red[1][w] = l1;
    red[2][w] = sq;
    red[3][w] = nf;
  }
  GroupTotal g{};
  if (update) g = block_reduce_groups(grp, ngroups, redf);  // synchronises the block
  else __syncthreads();
  if (threadIdx.x == 0) {
    for (int k = 1; k < kThreads / 32; ++k) {
      mx = fmax(mx, red[0][k]);
      l1 += red[1][k];
      sq += red[2][k];
      nf += red[3][k];
    }
    if (is_x) {
      if (residual) {
        results[kResXInf] = mx;
        results[kResXL1] = l1;
      }
      results[kResXSq] = sq;
    } else {
      results[kResYSq] = sq;
    }
    results[kResNonfin] += nf;
    if (update) finish_scalars(st, is_x ? 0 : 1, g, dm_next);
  }
}

// sum_i exp(2 log u_i) in FP64 as per-block partials in the common format.
__global__ void k_sum_sq(const double* __restrict__ log_u, int64_t rows, double* __restrict__ partials) {
  __shared__ double red[kThreads / 32];
  double s = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < rows;
       i += (int64_t)gridDim.x * blockDim.x)
    s += exp(2.0 * log_u[i]);
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (threadIdx.x % 32 == 0) red[threadIdx.x / 32] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double b = 0.0;
    for (int w = 0; w < kThreads / 32; ++w) b += red[w];
    partials[4 * blockIdx.x + 0] = 0.0;
    partials[4 * blockIdx.x + 1] = 0.0;
    partials[4 * blockIdx.x + 2] = b;
    partials[4 * blockIdx.x + 3] = 0.0;
  }
}

inline int grid_for(int64_t n, int num_sms, int per_sm = 8) {
  int64_t g = (n + kThreads - 1) / kThreads;
  const int64_t cap = (int64_t)num_sms * per_sm;
  if (g > cap) g = cap;
  if (g < 1) g = 1;
  return (int)g;
}

}  // namespace

cudaError_t launch_pack_factors(tu_market* m, Side& s, const void* A, const void* B, int src_dtype) {
  const int g = grid_for(s.rows * m->kp, m->num_sms, 16);
  k_pack_factors<<<g, kThreads, 0, m->stream>>>(A, B, src_dtype, s.rows, m->d, m->kp, s.fac16, s.fac32);
  return cudaGetLastError();
}

cudaError_t launch_init_side(tu_market* m, Side& s, const float* bias_dev, int has_bias) {
  const int g = grid_for(s.rows_pad, m->num_sms);
  k_init_side<<<g, kThreads, 0, m->stream>>>(bias_dev, has_bias, (float)(0.5 / m->sigma), s.rows,
                                               s.rows_pad, s.b2s, s.log_u, s.ell);
  return cudaGetLastError();
}

cudaError_t launch_reset_potentials(tu_market* m, Side& s) {
  const int g = grid_for(s.rows, m->num_sms);
  k_set_potentials<<<g, kThreads, 0, m->stream>>>(nullptr, s.b2s, s.rows, s.log_u, s.ell);
  return cudaGetLastError();
}

cudaError_t launch_get_potentials(tu_market* m, Side& s, float* out_dev) {
  const int g = grid_for(s.rows, m->num_sms);
  k_get_potentials<<<g, kThreads, 0, m->stream>>>(s.log_u, s.rows, out_dev);
  return cudaGetLastError();
}

cudaError_t launch_set_potentials64(tu_market* m, Side& s, const double* log_u_dev) {
  const int g = grid_for(s.rows, m->num_sms);
  k_set_potentials64<<<g, kThreads, 0, m->stream>>>(log_u_dev, s.b2s, s.rows, s.log_u, s.ell);
  return cudaGetLastError();
}

cudaError_t launch_set_potentials(tu_market* m, Side& s, const float* log_u_dev) {
  const int g = grid_for(s.rows, m->num_sms);
  k_set_potentials<<<g, kThreads, 0, m->stream>>>(log_u_dev, s.b2s, s.rows, s.log_u, s.ell);
  return cudaGetLastError();
}

cudaError_t launch_row_norms(tu_market* m, Side& s, float* out_max) {
  cudaError_t e = cudaMemsetAsync(out_max, 0, sizeof(float), m->stream);
  if (e != cudaSuccess) return e;
  int64_t blocks = (s.rows + (kThreads / 32) - 1) / (kThreads / 32);
  if (blocks > (int64_t)m->num_sms * 8) blocks = (int64_t)m->num_sms * 8;
  k_row_norm_max<<<(int)blocks, kThreads, 0, m->stream>>>(s.fac32, s.fac16, s.fac8, s.fs, s.rows, m->kp,
                                                          reinterpret_cast<unsigned int*>(out_max));
  return cudaGetLastError();
}

cudaError_t launch_max_abs(tu_market* m, const float* A, const float* B, int64_t count, float* out_max) {
  cudaError_t e = cudaMemsetAsync(out_max, 0, sizeof(float), m->stream);
  if (e != cudaSuccess) return e;
  k_max_abs<<<grid_for(count, m->num_sms, 8), kThreads, 0, m->stream>>>(A, B, count,
                                                                       reinterpret_cast<unsigned int*>(out_max));
  return cudaGetLastError();
}

cudaError_t launch_pack_fp8_rows(tu_market* m, Side& s, const float* A, const float* B, int side_k,
                                 unsigned int* bad) {
  const int g = grid_for(s.rows_pad * 32, m->num_sms, 8);  // one warp per row
  k_pack_fp8_rows<<<g, kThreads, 0, m->stream>>>(A, B, s.rows, s.rows_pad, m->d, m->kp, side_k, s.fac8, s.fs, bad);
  return cudaGetLastError();
}

cudaError_t launch_pack_fp8_bytes(tu_market* m, Side& s, const uint8_t* A, const uint8_t* B, const float* sc,
                                  unsigned int* bad) {
  const int g = grid_for(s.rows * m->kp, m->num_sms, 16);
  k_pack_fp8_bytes<<<g, kThreads, 0, m->stream>>>(A, B, sc, s.rows, s.rows_pad, m->d, m->kp, s.fac8, s.fs, bad);
  return cudaGetLastError();
}

cudaError_t launch_prep(tu_market* m, Side& partner, int fused_mode, int translate) {
  const int own = &partner == &m->Y ? 0 : 1;
  const int g = grid_for(partner.rows_pad, m->num_sms, 4);
  k_prep<<<g, kThreads, 0, m->stream>>>(partner.ell, partner.rows, partner.rows_pad, m->st, own, translate, fused_mode,
                                        partner.pvec, fused_mode ? reinterpret_cast<uint4*>(partner.fold) : nullptr,
                                        1.0f / m->cmul);  // (the batched preparation rounds 1 / c alike)
  return cudaGetLastError();
}

cudaError_t launch_rescan(tu_market* m) {
  for (Side* s : {&m->X, &m->Y}) {
    const int64_t ng = (s->rows + kGroupRows - 1) / kGroupRows;
    int g = (int)((ng * 32 + kThreads - 1) / kThreads);
    if (g > m->num_sms * 8) g = m->num_sms * 8;
    k_scan_groups<<<g < 1 ? 1 : g, kThreads, 0, m->stream>>>(s->log_u, s->ell, s->rows, s->grp);
  }
  k_rescan_scalars<<<1, kThreads, 0, m->stream>>>(m->X.grp, (m->X.rows + kGroupRows - 1) / kGroupRows, m->Y.grp,
                                                  (m->Y.rows + kGroupRows - 1) / kGroupRows,
                                                  m->Y.sum_mass - m->X.sum_mass, m->st);
  return cudaGetLastError();
}

cudaError_t launch_flush(tu_market* m) {
  const int64_t n = m->X.rows > m->Y.rows ? m->X.rows : m->Y.rows;
  k_flush<<<grid_for(n, m->num_sms, 4), kThreads, 0, m->stream>>>(m->X.log_u, m->X.ell, m->X.rows, m->Y.log_u,
                                                                   m->Y.ell, m->Y.rows, m->st);
  k_flush_scalars<<<1, 1, 0, m->stream>>>(m->st);
  return cudaGetLastError();
}

cudaError_t launch_sum_sq(tu_market* m, Side& s, int is_x) {
  int g = grid_for(s.rows, m->num_sms, 4);
  if (g > kMaxPartials) g = kMaxPartials;
  k_sum_sq<<<g, kThreads, 0, m->stream>>>(s.log_u, s.rows, m->partials);
  k_finalize<<<1, kThreads, 0, m->stream>>>(m->partials, g, is_x, 0, 0, nullptr, 0, 0.0, m->st, m->results);
  return cudaGetLastError();
}

cudaError_t launch_finalize(tu_market* m, int nparts, int is_x, int residual, int update, int64_t ngroups) {
  Side& own = is_x ? m->X : m->Y;
  Side& par = is_x ? m->Y : m->X;
  k_finalize<<<1, kThreads, 0, m->stream>>>(m->partials, nparts, is_x, residual, update, own.grp, ngroups,
                                            own.sum_mass - par.sum_mass, m->st, m->results);
  return cudaGetLastError();
}

}  // namespace tu
