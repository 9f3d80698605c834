// dense.cu -- batch IPFP (Alg. 1, Eq. iteration_matrix) over a materialised
// FP32 kernel. A-hat_xy = exp((Phi_xy - b^X_x - b^Y_y) / (2 sigma)) is built
// once; the biases live in the potentials (ell = log u + b / (2 sigma)), so
//     s_x = 1/2 exp(b^X_x / 2s) sum_y A-hat_xy exp(ell_y)
// and every half-sweep is one HBM stream over A-hat (N * M * 4 bytes).
//
// Row half-sweep (u step, s = A v / 2): one warp per row, 128-bit coalesced
// loads, warp-shuffle reduction, closed-form update in the epilogue.
// Column half-sweep (v step, s = A^T u / 2): column stripes of 1024 columns x
// a chunk of rows per CTA write FP32 partial sums; a second kernel adds the
// chunks per column and applies the update.
#include "tu_internal.cuh"

namespace tu {

namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;

// Streaming 128-bit load that does not allocate in L1 (A-hat is read once per pass).
__device__ __forceinline__ float4 ld_stream(const float4* p) {
  float4 v;
  asm volatile("ld.global.nc.L1::no_allocate.v4.f32 {%0, %1, %2, %3}, [%4];"
               : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
               : "l"(p));
  return v;
}

__global__ void __launch_bounds__(256) k_dense_build(const float* __restrict__ AX, const float* __restrict__ AY,
                                                     int64_t N, int64_t M, int64_t kp, float inv2s,
                                                     float* __restrict__ Ahat, int64_t ldA) {
  __shared__ float As[16][64 + 4];
  __shared__ float Bs[16][64 + 4];
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  const int64_t row0 = (int64_t)blockIdx.y * 64, col0 = (int64_t)blockIdx.x * 64;
  float acc[4][4] = {};
  for (int64_t k0 = 0; k0 < kp; k0 += 16) {
    for (int e = threadIdx.x; e < 16 * 64; e += kThreads) {
      const int r = e / 16, kk = e % 16;
      const int64_t gr = row0 + r, gc = col0 + r;
      As[kk][r] = (gr < N) ? AX[gr * kp + k0 + kk] : 0.0f;
      Bs[kk][r] = (gc < M) ? AY[gc * kp + k0 + kk] : 0.0f;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
      float a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty * 4 + i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx * 4 + j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int64_t r = row0 + ty * 4 + i;
    if (r >= N) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int64_t c = col0 + tx * 4 + j;
      if (c < ldA) Ahat[r * ldA + c] = (c < M) ? expf(acc[i][j] * inv2s) : 0.0f;
    }
  }
}

struct PartialAcc {
  double rmax = 0.0, rsum = 0.0, sq = 0.0, nf = 0.0;
  __device__ void add(const RowResult& rr) {
    rmax = fmax(rmax, rr.r_rel);
    rsum += rr.r_abs;
    sq += rr.u2;
    if (!isfinite(rr.log_u) || !isfinite(rr.ell)) nf += 1.0;
  }
};

// Block-level reduction of PartialAcc; thread 0 writes partials[4 * blockIdx.x ..].
__device__ void block_write_partials(PartialAcc a, double* __restrict__ partials) {
  __shared__ double s[4][kWarps];
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  for (int o = 16; o > 0; o >>= 1) {
    a.rmax = fmax(a.rmax, __shfl_xor_sync(0xffffffffu, a.rmax, o));
    a.rsum += __shfl_xor_sync(0xffffffffu, a.rsum, o);
    a.sq += __shfl_xor_sync(0xffffffffu, a.sq, o);
    a.nf += __shfl_xor_sync(0xffffffffu, a.nf, o);
  }
  if (lane == 0) {
    s[0][warp] = a.rmax;
    s[1][warp] = a.rsum;
    s[2][warp] = a.sq;
    s[3][warp] = a.nf;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double r0 = 0.0, r1 = 0.0, r2 = 0.0, r3 = 0.0;
    for (int w = 0; w < kWarps; ++w) {
      r0 = fmax(r0, s[0][w]);
      r1 += s[1][w];
      r2 += s[2][w];
      r3 += s[3][w];
    }
    partials[4 * blockIdx.x + 0] = r0;
    partials[4 * blockIdx.x + 1] = r1;
    partials[4 * blockIdx.x + 2] = r2;
    partials[4 * blockIdx.x + 3] = r3;
  }
}

__global__ void __launch_bounds__(kThreads) k_dense_rowpass(
    const float* __restrict__ Ahat, int64_t ldA, int64_t N, const float* __restrict__ w,
    const double* __restrict__ lmax_partner, const float* __restrict__ b2s, const double* __restrict__ mass,
    double* __restrict__ log_u, double* __restrict__ ell, double* __restrict__ partials, int residual,
    int update) {
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const double shift = *lmax_partner;
  const int64_t n4 = ldA / 4;
  const float4* w4 = reinterpret_cast<const float4*>(w);
  PartialAcc acc;
  for (int64_t row = (int64_t)blockIdx.x * kWarps + warp; row < N; row += (int64_t)gridDim.x * kWarps) {
    const float4* a4 = reinterpret_cast<const float4*>(Ahat + row * ldA);
    float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
    int64_t j = lane;
    for (; j + 96 < n4; j += 128) {
      const float4 a0 = ld_stream(a4 + j), a1 = ld_stream(a4 + j + 32);
      const float4 a2 = ld_stream(a4 + j + 64), a3 = ld_stream(a4 + j + 96);
      const float4 w0 = __ldg(w4 + j), w1 = __ldg(w4 + j + 32);
      const float4 w2 = __ldg(w4 + j + 64), w3 = __ldg(w4 + j + 96);
      s0 = fmaf(a0.x, w0.x, fmaf(a0.y, w0.y, fmaf(a0.z, w0.z, fmaf(a0.w, w0.w, s0))));
      s1 = fmaf(a1.x, w1.x, fmaf(a1.y, w1.y, fmaf(a1.z, w1.z, fmaf(a1.w, w1.w, s1))));
      s2 = fmaf(a2.x, w2.x, fmaf(a2.y, w2.y, fmaf(a2.z, w2.z, fmaf(a2.w, w2.w, s2))));
      s3 = fmaf(a3.x, w3.x, fmaf(a3.y, w3.y, fmaf(a3.z, w3.z, fmaf(a3.w, w3.w, s3))));
    }
    for (; j < n4; j += 32) {
      const float4 a0 = ld_stream(a4 + j);
      const float4 w0 = __ldg(w4 + j);
      s0 = fmaf(a0.x, w0.x, fmaf(a0.y, w0.y, fmaf(a0.z, w0.z, fmaf(a0.w, w0.w, s0))));
    }
    float s = (s0 + s1) + (s2 + s3);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) {
      const RowResult rr = row_update(log((double)s), shift, b2s ? b2s[row] : 0.0f, mass[row], log_u[row],
                                      residual != 0);
      if (update) {
        log_u[row] = rr.log_u;
        ell[row] = rr.ell;
      }
      acc.add(rr);
    }
  }
  block_write_partials(acc, partials);
}

__global__ void __launch_bounds__(kThreads) k_dense_colpart(const float* __restrict__ Ahat, int64_t ldA,
                                                            int64_t N, const float* __restrict__ z,
                                                            int64_t chunk_rows, float* __restrict__ colpart) {
  const int64_t c4 = (int64_t)blockIdx.x * kThreads + threadIdx.x;
  if (c4 * 4 >= ldA) return;
  const int64_t x0 = (int64_t)blockIdx.y * chunk_rows;
  int64_t x1 = x0 + chunk_rows;
  if (x1 > N) x1 = N;
  const float4* base = reinterpret_cast<const float4*>(Ahat) + c4;
  const int64_t stride4 = ldA / 4;
  float4 acc0 = make_float4(0.f, 0.f, 0.f, 0.f), acc1 = acc0;
  int64_t x = x0;
  for (; x + 3 < x1; x += 4) {
    const float4 a0 = ld_stream(base + x * stride4), a1 = ld_stream(base + (x + 1) * stride4);
    const float4 a2 = ld_stream(base + (x + 2) * stride4), a3 = ld_stream(base + (x + 3) * stride4);
    const float z0 = __ldg(z + x), z1 = __ldg(z + x + 1), z2 = __ldg(z + x + 2), z3 = __ldg(z + x + 3);
    acc0.x = fmaf(a0.x, z0, fmaf(a2.x, z2, acc0.x));
    acc0.y = fmaf(a0.y, z0, fmaf(a2.y, z2, acc0.y));
    acc0.z = fmaf(a0.z, z0, fmaf(a2.z, z2, acc0.z));
    acc0.w = fmaf(a0.w, z0, fmaf(a2.w, z2, acc0.w));
    acc1.x = fmaf(a1.x, z1, fmaf(a3.x, z3, acc1.x));
    acc1.y = fmaf(a1.y, z1, fmaf(a3.y, z3, acc1.y));
    acc1.z = fmaf(a1.z, z1, fmaf(a3.z, z3, acc1.z));
    acc1.w = fmaf(a1.w, z1, fmaf(a3.w, z3, acc1.w));
  }
  for (; x < x1; ++x) {
    const float4 a0 = ld_stream(base + x * stride4);
    const float z0 = __ldg(z + x);
    acc0.x = fmaf(a0.x, z0, acc0.x);
    acc0.y = fmaf(a0.y, z0, acc0.y);
    acc0.z = fmaf(a0.z, z0, acc0.z);
    acc0.w = fmaf(a0.w, z0, acc0.w);
  }
  float4 r;
  r.x = acc0.x + acc1.x;
  r.y = acc0.y + acc1.y;
  r.z = acc0.z + acc1.z;
  r.w = acc0.w + acc1.w;
  reinterpret_cast<float4*>(colpart + (int64_t)blockIdx.y * ldA)[c4] = r;
}

__global__ void __launch_bounds__(kThreads) k_dense_colfinal(
    const float* __restrict__ colpart, int chunks, int64_t ldA, int64_t M, const double* __restrict__ lmax_partner,
    const float* __restrict__ b2s, const double* __restrict__ mass, double* __restrict__ log_v,
    double* __restrict__ ell, double* __restrict__ partials, int update) {
  const double shift = *lmax_partner;
  PartialAcc acc;
  for (int64_t y = (int64_t)blockIdx.x * kThreads + threadIdx.x; y < M; y += (int64_t)gridDim.x * kThreads) {
    double s = 0.0;
    for (int c = 0; c < chunks; ++c) s += (double)colpart[(int64_t)c * ldA + y];
    const RowResult rr = row_update(log(s), shift, b2s ? b2s[y] : 0.0f, mass[y], log_v[y], false);
    if (update) {
      log_v[y] = rr.log_u;
      ell[y] = rr.ell;
    }
    acc.add(rr);
  }
  block_write_partials(acc, partials);
}

}  // namespace

cudaError_t launch_dense_build(tu_market* m) {
  dim3 grid((unsigned)((m->ldA + 63) / 64), (unsigned)((m->N + 63) / 64));
  k_dense_build<<<grid, kThreads, 0, m->stream>>>(m->X.fac32, m->Y.fac32, m->N, m->M, m->kp,
                                                  (float)(0.5 / m->sigma), m->Ahat, m->ldA);
  return cudaGetLastError();
}

cudaError_t launch_dense_rowpass(tu_market* m, int residual, int update, int* nparts_out) {
  int64_t g = (m->N + kWarps - 1) / kWarps;
  const int64_t cap = (int64_t)m->num_sms * 8;
  if (g > cap) g = cap;
  if (g > kMaxPartials) g = kMaxPartials;
  k_dense_rowpass<<<(int)g, kThreads, 0, m->stream>>>(m->Ahat, m->ldA, m->N, m->Y.pvec, m->Y.lmax, m->X.b2s,
                                                      m->X.mass, m->X.log_u, m->X.ell, m->partials, residual,
                                                      update);
  *nparts_out = (int)g;
  return cudaGetLastError();
}

cudaError_t launch_dense_colpass(tu_market* m, int update, int* nparts_out) {
  const int64_t n4 = m->ldA / 4;
  dim3 grid((unsigned)((n4 + kThreads - 1) / kThreads), (unsigned)m->col_chunks);
  const int64_t chunk_rows = (m->N + m->col_chunks - 1) / m->col_chunks;
  k_dense_colpart<<<grid, kThreads, 0, m->stream>>>(m->Ahat, m->ldA, m->N, m->X.pvec, chunk_rows, m->colpart);
  int64_t g = (m->M + kThreads - 1) / kThreads;
  if (g > kMaxPartials) g = kMaxPartials;
  k_dense_colfinal<<<(int)g, kThreads, 0, m->stream>>>(m->colpart, m->col_chunks, m->ldA, m->M, m->X.lmax,
                                                       m->Y.b2s, m->Y.mass, m->Y.log_u, m->Y.ell, m->partials, update);
  *nparts_out = (int)g;
  return cudaGetLastError();
}

}  // namespace tu
