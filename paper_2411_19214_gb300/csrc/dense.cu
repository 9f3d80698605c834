// dense.cu -- batch IPFP (Alg. 1, Eq. iteration_matrix) over a materialised
// FP32 kernel. A-hat_xy = exp((Phi_xy - b^X_x - b^Y_y) / (2 sigma)) is built
// once; the biases live in the potentials (ell = log u + b / (2 sigma)), so
//     s_x = 1/2 exp(b^X_x / 2 sigma) sum_y A-hat_xy exp(ell_y)
// and every half-sweep is one HBM stream over a row-major matrix.
//
// HBM layout: A-hat (N x ldA, ldA = M rounded up to 4) and its transpose
// (M x ldN). With both resident, the v step (s = A^T u / 2) is the same row
// stream as the u step (s = A v / 2): each row is streamed once through a
// shared-memory ring by bulk copies, reduced in a fixed order and updated in
// closed form (k_dense_rowpass). Deterministic; the price is 2 * N * M * 4
// bytes of HBM instead of N * M * 4.
#include "tu_internal.cuh"

namespace tu {

namespace {

// s += x * w with Kahan compensation c (the running error of s, subtracted
// from the next term); the product enters the compensated add unrounded.
__device__ __forceinline__ void kahan_fma(float& s, float& c, float x, float w) {
  const float y = fmaf(x, w, -c);
  const float t = s + y;
  c = (t - s) - y;
  s = t;
}

constexpr int kThreads = 256;  // the A-hat build

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
  const int64_t col0 = (int64_t)blockIdx.x * 64;
  // row tiles in steps of the grid's height (at most 65,535), so that any N
  // fits one launch; the trip count is the same for every thread of a block
  for (int64_t row0 = (int64_t)blockIdx.y * 64; row0 < N; row0 += (int64_t)gridDim.y * 64) {
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
    __syncthreads();  // Ts is rewritten by the next row tile
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

// One half-sweep over a row-major matrix A (rows x ld): for every row r,
// s_r = 1/2 exp(b_r / 2 sigma) exp(shift) sum_c A[r][c] w_c with
// w_c = exp(ell_c - shift) of the partner side (zero-padded to ld), then the
// closed-form update of the row's potential. RELAX: the update is
// over-relaxed by the device scalar *omega_p (markets with relaxation
// enabled); the plain instantiation is Eq. iteration exactly.
//
// Roles of a CTA (rows blockIdx.x, blockIdx.x + gridDim.x, ... in turn):
//   producer warp   one thread streams each row in kChunk-float pieces into a
//                   kStages ring in shared memory with 1D bulk copies
//                   (completion counted on the stage's mbarrier), so the
//                   bytes in flight do not depend on registers or on what
//                   the other warps are doing;
//   consumer warps  every warp takes strided float4s of each piece against
//                   the partner vector, releases the stage, and parks its
//                   share of the row sum; a block of kSlots rows is handed
//                   over once complete (double-buffered);
//   update warp     sums a block's parked shares in a fixed order and runs
//                   the kSlots closed-form updates in parallel (one per lane),
//                   off the stream's critical path, then frees the buffer.
// Every wait is bounded and sets the market's error word when it runs out;
// the producer then waits for its copies in flight before the CTA exits.
constexpr int kStages = 4;
constexpr int kChunk = 4096;  // floats per stage (16 KB)
constexpr int kConsumerWarps = 8;
constexpr int kUpdateWarp = kConsumerWarps;
constexpr int kProducerWarp = kConsumerWarps + 1;
constexpr int kPassThreads = (kConsumerWarps + 2) * 32;
constexpr int kSlots = 32;  // rows per block of updates: one per lane of the update warp

struct PassSmem {
  float ring[kStages][kChunk];
  float part[2][kSlots][kConsumerWarps];
  uint64_t full[kStages];   // a piece has landed (transaction count)
  uint64_t empty[kStages];  // every consumer warp is done with the stage
  uint64_t done[2];         // a block's row shares are parked
  uint64_t freed[2];        // the update warp has read the block
  int abort;
};

__device__ __forceinline__ void bulk_copy(void* smem_dst, const void* gsrc, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(smem_dst)),
      "l"(reinterpret_cast<uint64_t>(gsrc)), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void pass_abort(int* err, volatile int* flag) {
  atomicCAS(err, kErrNone, kErrTimeout);
  *flag = 1;
}

template <bool RELAX>
__global__ void __launch_bounds__(kPassThreads) k_dense_rowpass(
    const float* __restrict__ A, int64_t ld, int64_t rows, const float* __restrict__ w,
    const double* __restrict__ st, const float* __restrict__ b2s, const double* __restrict__ mass,
    double* __restrict__ log_u, double* __restrict__ ell, float4* __restrict__ grp, int64_t grp_blocks,
    double* __restrict__ partials, int residual, int update, const double* __restrict__ omega_p,
    int* __restrict__ err) {
  extern __shared__ __align__(128) uint8_t pass_smem_raw[];
  PassSmem& S = *reinterpret_cast<PassSmem*>(pass_smem_raw);
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  volatile int* abort_flag = &S.abort;
  if (threadIdx.x == 0) {
    for (int t = 0; t < kStages; ++t) {
      mbar_init(&S.full[t], 1);
      mbar_init(&S.empty[t], kConsumerWarps);
    }
    for (int t = 0; t < 2; ++t) {
      mbar_init(&S.done[t], kConsumerWarps);
      mbar_init(&S.freed[t], 1);
    }
    S.abort = 0;
    fence_mbar_init();
  }
  __syncthreads();
  const int64_t G = gridDim.x;
  const int64_t nchunks = (ld + kChunk - 1) / kChunk;
  // rows of this CTA (the grid never exceeds rows)
  const int64_t nrows = (rows - blockIdx.x + G - 1) / G;

  if (warp == kProducerWarp) {
    if (lane == 0) {
      int t = 0;
      uint32_t ph = 0, issued = 0, issued_ph = 0;
      bool ok = true;
      for (int64_t k = 0; k < nrows && ok; ++k) {
        const float* arow = A + (blockIdx.x + k * G) * ld;
        for (int64_t c = 0; c < nchunks; ++c) {
          if (!mbar_wait(&S.empty[t], ph ^ 1u, abort_flag)) {
            ok = false;
            break;
          }
          const int64_t c0 = c * kChunk;
          const uint32_t n = (uint32_t)(ld - c0 < kChunk ? ld - c0 : kChunk);
          mbar_arrive_expect_tx(&S.full[t], n * 4u);
          bulk_copy(S.ring[t], arow + c0, n * 4u, &S.full[t]);
          issued |= 1u << t;
          issued_ph = (issued_ph & ~(1u << t)) | (ph << t);
          if (++t == kStages) {
            t = 0;
            ph ^= 1u;
          }
        }
      }
      if (!ok && !*abort_flag) pass_abort(err, abort_flag);
      // copies in flight complete before the CTA's shared memory is released
      for (int u = 0; u < kStages; ++u)
        if (issued & (1u << u)) mbar_wait_drain(&S.full[u], (issued_ph >> u) & 1u, 100000000ull);
    }
    return;
  }

  if (warp < kConsumerWarps) {
    const float4* w4 = reinterpret_cast<const float4*>(w);
    int t = 0;
    uint32_t ph = 0;
    bool ok = true;
    for (int64_t k = 0; k < nrows && ok; ++k) {
      // four compensated (Kahan) sums per lane: a row of a few million terms
      // gives each accumulator thousands of them, where a plain FP32 sum
      // would drift by that many units of 2^-24; the pass is memory-bound,
      // so the three extra operations per term are free
      float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
      float e0 = 0.f, e1 = 0.f, e2 = 0.f, e3 = 0.f;  // their compensations
      for (int64_t c = 0; c < nchunks; ++c) {
        const bool got = mbar_wait(&S.full[t], ph, abort_flag);
        if (!__all_sync(0xffffffffu, got)) {
          ok = false;
          break;
        }
        const int64_t c0 = c * kChunk;
        const int nq = (int)((ld - c0 < kChunk ? ld - c0 : kChunk) / 4);
        const float4* r4 = reinterpret_cast<const float4*>(S.ring[t]);
        const float4* g4 = w4 + c0 / 4;
        for (int q = warp * 32 + lane; q < nq; q += kConsumerWarps * 32) {
          const float4 x = r4[q];
          const float4 y = __ldg(g4 + q);
          kahan_fma(a0, e0, x.x, y.x);
          kahan_fma(a1, e1, x.y, y.y);
          kahan_fma(a2, e2, x.z, y.z);
          kahan_fma(a3, e3, x.w, y.w);
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&S.empty[t]);
        if (++t == kStages) {
          t = 0;
          ph ^= 1u;
        }
      }
      if (!ok) break;
      float sum = ((a0 - e0) + (a1 - e1)) + ((a2 - e2) + (a3 - e3));
      for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
      const int slot = (int)(k % kSlots);
      const int64_t blk = k / kSlots;
      const int pb = (int)(blk & 1);
      if (slot == 0 && blk >= 2) {
        // the update warp has read this buffer's previous block
        const bool fr = mbar_wait(&S.freed[pb], (uint32_t)(((blk >> 1) - 1) & 1), abort_flag);
        if (!__all_sync(0xffffffffu, fr)) {
          ok = false;
          break;
        }
      }
      if (lane == 0) {
        S.part[pb][slot][warp] = sum;
        if (slot == kSlots - 1 || k == nrows - 1) mbar_arrive(&S.done[pb]);
      }
    }
    if (!ok && !*abort_flag) pass_abort(err, abort_flag);
    return;
  }

  if (warp != kUpdateWarp) return;
  PartialAcc acc;
  // the pass's partner shift and own offset (market scalars set by the preparation)
  double shift = 0.0, own_off = 0.0;
  if constexpr (!RELAX) {
    shift = st[kStShift];
    own_off = st[kStOwnOff];
  }
  // a block's shares arrive after kSlots rows are streamed: allow for 1 GB/s per CTA
  const uint64_t block_limit = kWaitLimitNs + (uint64_t)kSlots * (uint64_t)ld * 4ull;
  bool ok = true;
  for (int64_t blk = 0; blk * kSlots < nrows; ++blk) {
    const int pb = (int)(blk & 1);
    const bool got = mbar_wait(&S.done[pb], (uint32_t)((blk >> 1) & 1), abort_flag, block_limit);
    if (!__all_sync(0xffffffffu, got)) {
      ok = false;
      break;
    }
    const int64_t k = blk * kSlots + lane;
    double lu_new = 0.0, ell_new = 0.0;
    if (k < nrows) {
      const int64_t row = blockIdx.x + k * G;
      // the eight warps' shares, added with their roundings kept (two-sum)
      float sum = 0.0f, err = 0.0f;
      for (int cw = 0; cw < kConsumerWarps; ++cw) {
        float e;
        sum = two_sum(sum, S.part[pb][lane][cw], e);
        err = __fadd_rn(err, e);
      }
      double omega = 1.0;
      if constexpr (RELAX) {
        shift = __ldg(st + kStShift);
        own_off = __ldg(st + kStOwnOff);
        omega = (update && omega_p != nullptr) ? __ldg(omega_p) : 1.0;
      }
      const RowResult rr = row_update(log_row_sum(sum, err, 0.0f), shift, b2s ? b2s[row] : 0.0f, mass[row],
                                      log_u[row] + own_off, residual, omega);
      if (update) {
        log_u[row] = rr.log_u;
        ell[row] = rr.ell;
      }
      lu_new = rr.log_u;
      ell_new = rr.ell;
      acc.add(rr);
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(&S.freed[pb]);
    if (update) {
      // the block's rows (this CTA's rows blk * 32 .. blk * 32 + 31) form group blk * G + blockIdx.x
      const float4 gv = warp_group(lu_new, ell_new, k < nrows);
      if (lane == 0) grp[blk * G + blockIdx.x] = gv;
    }
  }
  if (update && ok && lane == 0) {
    // groups of the blocks this CTA does not have (the grid's rows are
    // dealt round-robin, so some CTAs have one block fewer) contribute nothing
    for (int64_t blk = (nrows + kSlots - 1) / kSlots; blk < grp_blocks; ++blk) grp[blk * G + blockIdx.x] = empty_group();
  }
  if (!ok && !*abort_flag) pass_abort(err, abort_flag);
  // this warp holds every partial of the CTA
  for (int o = 16; o > 0; o >>= 1) {
    acc.rmax = fmax(acc.rmax, __shfl_xor_sync(0xffffffffu, acc.rmax, o));
    acc.rsum += __shfl_xor_sync(0xffffffffu, acc.rsum, o);
    acc.sq += __shfl_xor_sync(0xffffffffu, acc.sq, o);
    acc.nf += __shfl_xor_sync(0xffffffffu, acc.nf, o);
  }
  if (lane == 0) {
    partials[4 * blockIdx.x + 0] = acc.rmax;
    partials[4 * blockIdx.x + 1] = acc.rsum;
    partials[4 * blockIdx.x + 2] = acc.sq;
    partials[4 * blockIdx.x + 3] = acc.nf;
  }
}

// CTAs of a pass: as many as fit on the device at once (the ring's shared
// memory allows a few per SM), at most one per row.
int rowpass_grid(tu_market* m, int64_t rows) {
  static int per_sm = 0;
  if (per_sm == 0) {
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_dense_rowpass<false>, kPassThreads,
                                                      sizeof(PassSmem)) != cudaSuccess ||
        b < 1) {
      cudaGetLastError();
      b = 1;
    }
    per_sm = b;
  }
  int64_t g = (int64_t)m->num_sms * per_sm;
  if (g > rows) g = rows;
  if (g > kMaxPartials) g = kMaxPartials;
  return (int)(g < 1 ? 1 : g);
}

}  // namespace

cudaError_t launch_dense_build(tu_market* m) {
  // the row pass's ring exceeds the default 48 KB of dynamic shared memory
  // (set here, at creation and factor updates, never inside a graph capture)
  cudaError_t e = cudaFuncSetAttribute(k_dense_rowpass<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)sizeof(PassSmem));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_dense_rowpass<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)sizeof(PassSmem));
  if (e != cudaSuccess) return e;
  const int64_t row_tiles = (m->N + 63) / 64;
  dim3 grid((unsigned)((m->M + 63) / 64), (unsigned)(row_tiles < 65535 ? row_tiles : 65535));
  k_dense_build<<<grid, kThreads, 0, m->stream>>>(m->X.fac32, m->Y.fac32, m->N, m->M, m->kp,
                                                  (float)(0.5 / m->sigma), m->Ahat, m->ldA, m->AhatT, m->ldN);
  return cudaGetLastError();
}

cudaError_t launch_dense_rowpass(tu_market* m, int residual, int update, int* nparts_out, int64_t* ngroups_out) {
  const int g = rowpass_grid(m, m->N);
  const int64_t blocks = ((m->N + g - 1) / g + kSlots - 1) / kSlots;  // update blocks of the fullest CTA
  auto kern = m->omega_cfg != 1.0 ? k_dense_rowpass<true> : k_dense_rowpass<false>;
  kern<<<g, kPassThreads, sizeof(PassSmem), m->stream>>>(m->Ahat, m->ldA, m->N, m->Y.pvec, m->st, m->X.b2s,
                                                         m->X.mass, m->X.log_u, m->X.ell, m->X.grp, blocks,
                                                         m->partials, residual, update, m->omega_dev, m->err_dev);
  *nparts_out = g;
  *ngroups_out = blocks * g;
  return cudaGetLastError();
}

cudaError_t launch_dense_colpass(tu_market* m, int update, int* nparts_out, int64_t* ngroups_out) {
  const int g = rowpass_grid(m, m->M);
  const int64_t blocks = ((m->M + g - 1) / g + kSlots - 1) / kSlots;
  auto kern = m->omega_cfg != 1.0 ? k_dense_rowpass<true> : k_dense_rowpass<false>;
  kern<<<g, kPassThreads, sizeof(PassSmem), m->stream>>>(m->AhatT, m->ldN, m->M, m->X.pvec, m->st, m->Y.b2s,
                                                         m->Y.mass, m->Y.log_u, m->Y.ell, m->Y.grp, blocks,
                                                         m->partials, 0, update, m->omega_dev, m->err_dev);
  *nparts_out = g;
  *ngroups_out = blocks * g;
  return cudaGetLastError();
}

}  // namespace tu
