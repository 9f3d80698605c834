// dense.cu -- batch IPFP (Alg. 1, Eq. iteration_matrix) over a materialised
// FP32 kernel. A-hat_xy = exp((Phi_xy - b^X_x - b^Y_y) / (2 sigma)) is built
// once; the biases live in the potentials (ell = log u + b / (2 sigma)), so
//     s_x = 1/2 exp(b^X_x / 2 sigma) sum_y A-hat_xy exp(ell_y)
// and every half-sweep is one HBM stream over a row-major matrix.
//
// HBM layout: A-hat (N x ldA, ldA = M rounded up to 4) and its transpose
// (M x ldN). With both resident, the v step (s = A^T u / 2) is the same row
// stream as the u step (s = A v / 2): one warp per row, 128-bit coalesced
// loads with kRowDepth loads in flight per lane, a warp-shuffle reduction and
// the closed-form update in the epilogue. Deterministic, no partial sums; the
// price is 2 * N * M * 4 bytes of HBM instead of N * M * 4.
#include "tu_internal.cuh"

namespace tu {

namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kRowDepth = 8;  // 16-byte loads in flight per lane in the row pass

// Streaming 128-bit load that does not allocate in L1 (A-hat is read once per pass).
__device__ __forceinline__ float4 ld_stream(const float4* p) {
  float4 v;
  asm volatile("ld.global.nc.L1::no_allocate.v4.f32 {%0, %1, %2, %3}, [%4];"
               : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
               : "l"(p));
  return v;
}

// A-hat and its transpose from the packed FP32 factors (setup, once per factor
// update). 64 x 64 output tile per CTA; the transposed tile is staged in
// shared memory so both stores are coalesced.
__global__ void __launch_bounds__(256) k_dense_build(const float* __restrict__ AX, const float* __restrict__ AY,
                                                     int64_t N, int64_t M, int64_t kp, float inv2s,
                                                     float* __restrict__ Ahat, int64_t ldA, float* __restrict__ AhatT,
                                                     int64_t ldN) {
  __shared__ float As[16][64 + 4];
  __shared__ float Bs[16][64 + 4];
  __shared__ float Ts[64][64 + 1];
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
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int64_t c = col0 + tx * 4 + j;
      const float v = (r < N && c < M) ? expf(acc[i][j] * inv2s) : 0.0f;
      Ts[tx * 4 + j][ty * 4 + i] = v;
      if (r < N && c < ldA) Ahat[r * ldA + c] = v;
    }
  }
  __syncthreads();
  // transposed tile: row c of A-hat^T holds column c of A-hat
  for (int e = threadIdx.x; e < 64 * 64; e += kThreads) {
    const int cl = e / 64, rl = e % 64;
    const int64_t c = col0 + cl, r = row0 + rl;
    if (c < M && r < ldN) AhatT[c * ldN + r] = (r < N) ? Ts[cl][rl] : 0.0f;
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

// One half-sweep over a row-major matrix A (rows x ld): for every row r,
// s_r = 1/2 exp(b_r / 2 sigma) exp(shift) sum_c A[r][c] w_c with
// w_c = exp(ell_c - shift) of the partner side (zero-padded to ld), then the
// closed-form update of the row's potential. RELAX: the update is
// over-relaxed by the device scalar *omega_p (markets with relaxation
// enabled); the plain instantiation is Eq. iteration exactly.
//
// Work split: the CTA's warps form groups of `wpr` warps; a group streams one
// row, each warp a contiguous 1/wpr of its columns, and rows go to CTAs and
// groups round-robin. With wpr = 8 a CTA streams one row at a time, so the
// kernel is balanced to one row per CTA (about 1 % here) rather than to one
// row per warp (a warp owning 4 or 5 of 20,000 rows left a 20 % tail). Warp
// partial sums are parked in shared memory; every kSlots rows the 32 lanes of
// warp 0 combine them in a fixed order and run the closed-form updates in
// parallel. Four CTAs per SM (64 registers, a few bytes of spill outside the
// streaming loop) measured 12 % faster than three without spill: occupancy
// sets the bytes in flight.
constexpr int kSlots = 32;

template <bool RELAX>
__global__ void __launch_bounds__(kThreads, 4) k_dense_rowpass(
    const float* __restrict__ A, int64_t ld, int64_t rows, int wpr, const float* __restrict__ w,
    const double* __restrict__ lmax_partner, const float* __restrict__ b2s, const double* __restrict__ mass,
    double* __restrict__ log_u, double* __restrict__ ell, double* __restrict__ partials, int residual,
    int update, const double* __restrict__ omega_p) {
  __shared__ float part[kSlots][kWarps];
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  // plain: the shift is loaded up front, overlapped with the stream (a load at
  // update time would lengthen every CTA's tail); relaxed: loaded at update
  // time with omega, so that neither is live across the streaming loop
  double shift = 0.0;
  if constexpr (!RELAX) shift = *lmax_partner;
  const int groups = kWarps / wpr;          // rows in flight per CTA
  const int grp = warp / wpr, wi = warp % wpr;
  // column indices in float4 units fit in 32 bits (ld <= 2^31 floats)
  const int n4 = (int)(ld / 4);
  const int seg = (n4 + wpr - 1) / wpr;
  const int c0 = wi * seg;
  const int c1 = c0 + seg < n4 ? c0 + seg : n4;
  const float4* w4 = reinterpret_cast<const float4*>(w);
  PartialAcc acc;
  int nslot = 0;
  int64_t first = (int64_t)blockIdx.x * groups;  // first row of the parked block
  auto flush = [&]() {
    __syncthreads();
    if (warp == 0 && lane < nslot) {
      // slot i holds row first + (i / groups) * gridDim.x * groups + i % groups
      const int64_t row = first + (int64_t)(lane / groups) * gridDim.x * groups + lane % groups;
      if (row < rows) {
        float sum = 0.0f;
        for (int k = 0; k < wpr; ++k) sum += part[lane][(lane % groups) * wpr + k];
        double omega = 1.0;
        if constexpr (RELAX) {
          shift = __ldg(lmax_partner);
          omega = (update && omega_p != nullptr) ? __ldg(omega_p) : 1.0;
        }
        const RowResult rr = row_update((double)logf(sum), shift, b2s ? b2s[row] : 0.0f, mass[row], log_u[row],
                                        residual != 0, omega);
        if (update) {
          log_u[row] = rr.log_u;
          ell[row] = rr.ell;
        }
        acc.add(rr);
      }
    }
    __syncthreads();
    nslot = 0;
  };
  for (int64_t rbase = (int64_t)blockIdx.x * groups; rbase < rows; rbase += (int64_t)gridDim.x * groups) {
    if (nslot == 0) first = rbase;
    const int64_t row = rbase + grp;
    if (row < rows) {
      const float4* a4 = reinterpret_cast<const float4*>(A + row * ld);
      float s4[4] = {0.f, 0.f, 0.f, 0.f};
      // every iteration keeps kRowDepth loads in flight, the last one predicated
      for (int base = c0; base < c1; base += 32 * kRowDepth) {
        float4 a[kRowDepth], ww[kRowDepth];
#pragma unroll
        for (int u = 0; u < kRowDepth; ++u) {
          const int j = base + lane + 32 * u;
          a[u] = j < c1 ? ld_stream(a4 + j) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int u = 0; u < kRowDepth; ++u) {
          const int j = base + lane + 32 * u;
          ww[u] = j < c1 ? __ldg(w4 + j) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int u = 0; u < kRowDepth; ++u)
          s4[u & 3] =
              fmaf(a[u].x, ww[u].x, fmaf(a[u].y, ww[u].y, fmaf(a[u].z, ww[u].z, fmaf(a[u].w, ww[u].w, s4[u & 3]))));
      }
      float s = (s4[0] + s4[1]) + (s4[2] + s4[3]);
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (lane == 0) part[nslot + grp][warp % kWarps] = s;
    }
    nslot += groups;
    if (nslot == kSlots) flush();
  }
  if (nslot > 0) flush();
  block_write_partials(acc, partials);
}

// Warps per row: as many as keep every lane of a warp busy for at least one
// full kRowDepth iteration (8, 4, 2 or 1).
int warps_per_row(int64_t ld) {
  const int64_t n4 = ld / 4;
  int wpr = kWarps;
  while (wpr > 1 && n4 / wpr < 32 * kRowDepth) wpr /= 2;
  return wpr;
}

int rowpass_grid(tu_market* m, int64_t rows, int64_t ld) {
  static int per_sm = 0;
  if (per_sm == 0) {
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_dense_rowpass<false>, kThreads, 0) != cudaSuccess ||
        b < 1)
      b = 2;
    per_sm = b;
  }
  int64_t g = (int64_t)m->num_sms * per_sm;  // exactly one resident wave, grid-stride over rows
  const int64_t groups = kWarps / warps_per_row(ld);
  const int64_t need = (rows + groups - 1) / groups;
  if (g > need) g = need;
  if (g > kMaxPartials) g = kMaxPartials;
  return (int)(g < 1 ? 1 : g);
}

}  // namespace

cudaError_t launch_dense_build(tu_market* m) {
  dim3 grid((unsigned)((m->M + 63) / 64), (unsigned)((m->N + 63) / 64));
  k_dense_build<<<grid, kThreads, 0, m->stream>>>(m->X.fac32, m->Y.fac32, m->N, m->M, m->kp,
                                                  (float)(0.5 / m->sigma), m->Ahat, m->ldA, m->AhatT, m->ldN);
  return cudaGetLastError();
}

cudaError_t launch_dense_rowpass(tu_market* m, int residual, int update, int* nparts_out) {
  const int g = rowpass_grid(m, m->N, m->ldA);
  auto kern = m->omega_cfg != 1.0 ? k_dense_rowpass<true> : k_dense_rowpass<false>;
  kern<<<g, kThreads, 0, m->stream>>>(m->Ahat, m->ldA, m->N, warps_per_row(m->ldA), m->Y.pvec, m->Y.lmax, m->X.b2s,
                                      m->X.mass, m->X.log_u, m->X.ell, m->partials, residual, update, m->omega_dev);
  *nparts_out = g;
  return cudaGetLastError();
}

cudaError_t launch_dense_colpass(tu_market* m, int update, int* nparts_out) {
  const int g = rowpass_grid(m, m->M, m->ldN);
  auto kern = m->omega_cfg != 1.0 ? k_dense_rowpass<true> : k_dense_rowpass<false>;
  kern<<<g, kThreads, 0, m->stream>>>(m->AhatT, m->ldN, m->M, warps_per_row(m->ldN), m->X.pvec, m->X.lmax, m->Y.b2s,
                                      m->Y.mass, m->Y.log_u, m->Y.ell, m->partials, 0, update, m->omega_dev);
  *nparts_out = g;
  return cudaGetLastError();
}

}  // namespace tu
