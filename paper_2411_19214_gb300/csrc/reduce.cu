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

// FP8 packing: row r of the output is [A_r | B_r | 0] * 2^-k rounded to the
// nearest e4m3 value (ties to even), saturating at +-448; 128 bytes per row.
__global__ void k_pack_fp8(const float* __restrict__ A, const float* __restrict__ B, int64_t rows, int64_t d,
                           float scale, uint8_t* __restrict__ out) {
  const int64_t total = rows * 128;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = i / 128;
    const int64_t k = i - r * 128;
    float v = 0.0f;
    if (k < d) {
      v = A[r * d + k];
    } else if (k < 2 * d) {
      v = B[r * d + (k - d)];
    }
    out[i] = (uint8_t)__nv_cvt_float_to_fp8(v * scale, __NV_SATFINITE, __NV_E4M3);
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

__global__ void k_get_potentials(const double* __restrict__ log_u, int64_t rows, float* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < rows;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (float)log_u[i];
}

__global__ void k_row_norm_max(const float* __restrict__ f32, const __nv_bfloat16* __restrict__ f16,
                               const uint8_t* __restrict__ f8, float f8scale, int64_t rows, int64_t kp,
                               unsigned int* __restrict__ out) {
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
        v = __half2float(__half(h)) * f8scale;
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

// Partner preparation, phase 1: per-block maximum of ell.
__global__ void k_prep_max(const double* __restrict__ ell, int64_t rows, double* __restrict__ mpartials) {
  __shared__ double red[kThreads / 32];
  double mx = -INFINITY;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < rows;
       i += (int64_t)gridDim.x * blockDim.x)
    mx = fmax(mx, ell[i]);
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if (threadIdx.x % 32 == 0) red[threadIdx.x / 32] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    double b = -INFINITY;
    for (int w = 0; w < kThreads / 32; ++w) b = fmax(b, red[w]);
    mpartials[blockIdx.x] = b;
  }
}

// Translation step of a sweep's half-sweep (one CTA of kTauThreads): tau from
// the two sides' potentials, into *tau_out. The batched preparation computes
// the same value with the same routine and block size.
__global__ void __launch_bounds__(kTauThreads) k_prep_tau(const double* __restrict__ log_p, int64_t rows_p,
                                                          const double* __restrict__ log_o, int64_t rows_o, double dm,
                                                          double* __restrict__ tau_out) {
  __shared__ double red[kTauThreads / 32];
  const double tau = block_translation_tau(log_p, rows_p, log_o, rows_o, dm, red);
  if (threadIdx.x == 0) *tau_out = tau;
}

// Partner preparation, phase 2: shift = max ell; write the vector the
// half-sweep consumes. fused_mode 1: (ell - shift) * log2(e), padding -inf
// (exp2 of it is 0); fused_mode 0: exp(ell - shift), padding 0.
// With tau (the translation step, computed by k_prep_tau), the FP64 state
// moves: log p, ell_p += tau (partner side), log o, ell_o -= tau (own side).
// The prepared vector depends only on ell_p - max ell_p, which the move leaves
// unchanged, so it is written from the values before the move and the shift
// becomes max ell_p + tau.
__global__ void k_prep_write(double* __restrict__ ell, double* __restrict__ log_p, int64_t rows, int64_t rows_pad,
                             double* __restrict__ log_o, double* __restrict__ ell_o, int64_t rows_o,
                             const double* __restrict__ tau_in, const double* __restrict__ mpartials, int nparts,
                             int fused_mode, float* __restrict__ out, double* __restrict__ lmax) {
  __shared__ double red[kThreads / 32];
  __shared__ double shift_s;
  double mx = -INFINITY;
  for (int i = threadIdx.x; i < nparts; i += blockDim.x) mx = fmax(mx, mpartials[i]);
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if (threadIdx.x % 32 == 0) red[threadIdx.x / 32] = mx;
  __syncthreads();
  const double tau = tau_in != nullptr ? *tau_in : 0.0;
  if (threadIdx.x == 0) {
    double b = -INFINITY;
    for (int w = 0; w < kThreads / 32; ++w) b = fmax(b, red[w]);
    if (!(b > -INFINITY && b < INFINITY)) b = 0.0;  // non-finite potentials are reported elsewhere
    shift_s = b;
    if (blockIdx.x == 0) *lmax = b + tau;
  }
  __syncthreads();
  const double shift = shift_s;
  const int64_t n = tau_in != nullptr && rows_o > rows_pad ? rows_o : rows_pad;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    if (i < rows_pad) {
      float v;
      if (i < rows) {
        // the FP64 state is rounded once, to the FP32 vector the half-sweep streams
        const double e = ell[i];
        const double z = e - shift;
        v = fused_mode ? (float)(z * 1.4426950408889634) : (float)exp(z);
        if (tau_in != nullptr) {
          ell[i] = e + tau;
          log_p[i] += tau;
        }
      } else {
        v = fused_mode ? -INFINITY : 0.0f;
      }
      out[i] = v;
    }
    if (tau_in != nullptr && i < rows_o) {
      log_o[i] -= tau;
      ell_o[i] -= tau;
    }
  }
}

// FP64 reduction of the per-CTA partials (max r/n, sum |r|, sum u^2, non-finite count).
__global__ void k_finalize(const double* __restrict__ partials, int nparts, int is_x, int residual,
                           double* __restrict__ results) {
  __shared__ double s_max[kThreads], s_l1[kThreads], s_sq[kThreads], s_nf[kThreads];
  double mx = 0.0, l1 = 0.0, sq = 0.0, nf = 0.0;
  for (int i = threadIdx.x; i < nparts; i += blockDim.x) {
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
    if (is_x) {
      if (residual) {
        results[kResXInf] = s_max[0];
        results[kResXL1] = s_l1[0];
      }
      results[kResXSq] = s_sq[0];
    } else {
      results[kResYSq] = s_sq[0];
    }
    results[kResNonfin] += s_nf[0];
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
  k_row_norm_max<<<(int)blocks, kThreads, 0, m->stream>>>(s.fac32, s.fac16, s.fac8, ldexpf(1.0f, s.fp8_exp), s.rows,
                                                          m->kp, reinterpret_cast<unsigned int*>(out_max));
  return cudaGetLastError();
}

cudaError_t launch_max_abs(tu_market* m, const float* A, const float* B, int64_t count, float* out_max) {
  cudaError_t e = cudaMemsetAsync(out_max, 0, sizeof(float), m->stream);
  if (e != cudaSuccess) return e;
  k_max_abs<<<grid_for(count, m->num_sms, 8), kThreads, 0, m->stream>>>(A, B, count,
                                                                       reinterpret_cast<unsigned int*>(out_max));
  return cudaGetLastError();
}

cudaError_t launch_pack_fp8(tu_market* m, Side& s, const float* A, const float* B, int k) {
  const int g = grid_for(s.rows * 128, m->num_sms, 16);
  k_pack_fp8<<<g, kThreads, 0, m->stream>>>(A, B, s.rows, m->d, ldexpf(1.0f, -k), s.fac8);
  return cudaGetLastError();
}

cudaError_t launch_prep(tu_market* m, Side& partner, int fused_mode, int translate) {
  Side& own = &partner == &m->Y ? m->X : m->Y;
  int g1 = grid_for(partner.rows, m->num_sms, 4);
  if (g1 > kMaxPartials) g1 = kMaxPartials;
  k_prep_max<<<g1, kThreads, 0, m->stream>>>(partner.ell, partner.rows, m->mpartials);
  if (translate)
    k_prep_tau<<<1, kTauThreads, 0, m->stream>>>(partner.log_u, partner.rows, own.log_u, own.rows,
                                                 partner.sum_mass - own.sum_mass, m->tau_dev);
  const int64_t n2 = translate && own.rows > partner.rows_pad ? own.rows : partner.rows_pad;
  const int g2 = grid_for(n2, m->num_sms, 4);
  k_prep_write<<<g2, kThreads, 0, m->stream>>>(partner.ell, partner.log_u, partner.rows, partner.rows_pad, own.log_u,
                                                own.ell, own.rows, translate ? m->tau_dev : nullptr, m->mpartials, g1,
                                                fused_mode, partner.pvec, partner.lmax);
  return cudaGetLastError();
}

cudaError_t launch_sum_sq(tu_market* m, Side& s, int is_x) {
  int g = grid_for(s.rows, m->num_sms, 4);
  if (g > kMaxPartials) g = kMaxPartials;
  k_sum_sq<<<g, kThreads, 0, m->stream>>>(s.log_u, s.rows, m->partials);
  k_finalize<<<1, kThreads, 0, m->stream>>>(m->partials, g, is_x, 0, m->results);
  return cudaGetLastError();
}

cudaError_t launch_finalize(tu_market* m, int nparts, int is_x, int residual) {
  k_finalize<<<1, kThreads, 0, m->stream>>>(m->partials, nparts, is_x, residual, m->results);
  return cudaGetLastError();
}

}  // namespace tu
