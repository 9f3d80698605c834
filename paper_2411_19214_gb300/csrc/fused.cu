// fused.cu -- mini-batch IPFP half-sweep (Alg. 2, Eq. iteration_minibatch) on
// sm_103a tensor cores. Phi is formed tile by tile and never written to HBM.
//
// For the half-sweep that updates side "own" against side "partner":
//   S_r = sum_c exp2( c * <a_r, b_c> + g_c ),   c = log2(e) / (2 sigma),
//   g_c = (ell_c - max ell) * log2(e)  (partner potential incl. bias, shifted <= 0),
// then log s_r = log(1/2) + bias_r/(2 sigma) + max ell + log S_r and the
// closed-form update of Eq. iteration gives the new log u_r.
//
// Because the partner biases are folded into g and the shift is the maximum of
// g, every exponent is bounded by c * |a_r| * |b_c| (checked on the host), so
// no per-pair running maximum is needed: the running-max rescale of
// flash-attention collapses to one shift per half-sweep.
//
// CTA layout (320 threads, one CTA per SM, persistent over own tiles):
//   warp 0     : TMA producer (one elected thread): the own tile [F|K]_j
//                (256 rows x kp) once per own tile, then partner tiles
//                (128 rows x kp) through a STAGES-deep shared-memory ring.
//   warp 1     : MMA issuer (one thread): two tcgen05.mma M=128 N=128 chains
//                (own rows 0-127 and 128-255) per partner tile into one of two
//                TMEM accumulator buffers (2 x 256 columns = all 512).
//   warps 2-9  : epilogue: warp w reads TMEM lanes 32*(w%4).. of own sub-tile
//                (w-2)/4, i.e. one own row per thread, so the row reduction
//                stays inside the thread (no shuffles): FFMA + ex2 + FADD per
//                pair, per-tile partials added into a compensated sum.
// Every wait is bounded (kWaitLimitNs); a wait that runs out raises the
// abort flag and the error word, the roles drain, TMEM is freed, and the
// kernel returns.
#include "tu_internal.cuh"

#include <mutex>

namespace tu {

namespace {

constexpr int kThreads = 320;
constexpr int kEpiWarps = 8;
constexpr int kOwnBytesPerKB = kFusedOwnRows * 128;          // 32 KB per 64-wide k block
constexpr int kPartnerBytesPerKB = kFusedPartnerRows * 128;  // 16 KB per 64-wide k block
constexpr uint32_t kTmemCols = 512;

struct FusedParams {
  int64_t rows;            // own-side users
  int num_own_tiles;       // ceil(rows / 256)
  int num_partner_tiles;   // ceil(partner rows / 128)
  float c;                 // log2(e) / (2 sigma)
  const float* g;          // partner prepared potentials, >= num_partner_tiles * 128, -inf padded
  const double* lmax;      // partner shift (natural log)
  const float* b2s;        // own bias / (2 sigma), or nullptr
  const double* mass;      // own capacities
  double* log_u;           // own potentials (in: old, out: new), FP64 state
  double* ell;             // own ell (out), FP64 state
  double* partials;        // [gridDim.x][4]
  int* err;                // device error word
  int residual;
  int update;
};

template <int KB>
constexpr int smem_bytes(int stages) {
  return 1024 /*alignment slack*/ + KB * kOwnBytesPerKB + stages * KB * kPartnerBytesPerKB + 512;
}

__device__ __forceinline__ void raise_error(int* err, volatile int* abort_flag, int code) {
  atomicCAS(err, kErrNone, code);
  *abort_flag = 1;
}

template <int KB, int STAGES>
__global__ void __launch_bounds__(kThreads, 1)
    k_fused_halfsweep(const __grid_constant__ CUtensorMap tm_own, const __grid_constant__ CUtensorMap tm_partner,
                      const FusedParams p) {
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw_u32 = smem_u32(smem_raw);
  uint8_t* smem = smem_raw + (((raw_u32 + 1023u) & ~1023u) - raw_u32);
  uint8_t* sA = smem;
  uint8_t* sB = smem + KB * kOwnBytesPerKB;
  uint64_t* bars = reinterpret_cast<uint64_t*>(sB + STAGES * KB * kPartnerBytesPerKB);
  uint64_t* full = bars;
  uint64_t* empty = bars + STAGES;
  uint64_t* a_full = bars + 2 * STAGES;
  uint64_t* a_empty = a_full + 1;
  uint64_t* tfull = a_full + 2;   // [2]
  uint64_t* tempty = a_full + 4;  // [2]
  uint64_t* mma_done = a_full + 6;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(mma_done + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  double* red = reinterpret_cast<double*>(mma_done + 2);  // 4 x kEpiWarps doubles

  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(a_full, 1);
    mbar_init(a_empty, 1);
    for (int b = 0; b < 2; ++b) {
      mbar_init(&tfull[b], 1);
      mbar_init(&tempty[b], kEpiWarps);
    }
    mbar_init(mma_done, 1);
    *abort_flag = 0;
    fence_mbar_init();
    tma_prefetch_map(&tm_own);
    tma_prefetch_map(&tm_partner);
  }
  if (warp == 0) {
    tmem_alloc(tmem_slot, kTmemCols);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;

  if (warp == 0) {
    // ------------------------------------------------------------ producer
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0, a_phase = 0;
      uint32_t armed[STAGES];
      for (int s = 0; s < STAGES; ++s) armed[s] = 0;
      uint32_t a_armed = 0;
      bool ok = true;
      for (int t = blockIdx.x; t < p.num_own_tiles && ok; t += gridDim.x) {
        if (!mbar_wait(a_empty, a_phase ^ 1u, abort_flag)) {
          ok = false;
          break;
        }
        a_phase ^= 1u;
        mbar_arrive_expect_tx(a_full, KB * kOwnBytesPerKB);
        for (int kb = 0; kb < KB; ++kb)
          tma_load_2d(sA + kb * kOwnBytesPerKB, &tm_own, a_full, kb * kKBlock, t * kFusedOwnRows);
        ++a_armed;
        for (int j = 0; j < p.num_partner_tiles; ++j) {
          if (!mbar_wait(&empty[stage], phase ^ 1u, abort_flag)) {
            ok = false;
            break;
          }
          mbar_arrive_expect_tx(&full[stage], KB * kPartnerBytesPerKB);
          for (int kb = 0; kb < KB; ++kb)
            tma_load_2d(sB + (stage * KB + kb) * kPartnerBytesPerKB, &tm_partner, &full[stage], kb * kKBlock,
                        j * kFusedPartnerRows);
          ++armed[stage];
          if (++stage == STAGES) {
            stage = 0;
            phase ^= 1u;
          }
        }
      }
      if (!ok) {
        if (!*abort_flag) raise_error(p.err, abort_flag, kErrTimeout);
        // let the copies already issued land before the CTA's shared memory goes away
        for (int s = 0; s < STAGES; ++s)
          if (armed[s]) mbar_wait_drain(&full[s], (armed[s] - 1u) & 1u, 10000000ull);
        if (a_armed) mbar_wait_drain(a_full, (a_armed - 1u) & 1u, 10000000ull);
      }
    }
    __syncwarp();
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      constexpr uint32_t idesc = idesc_bf16_f32(128, kFusedPartnerRows);
      int stage = 0, buf = 0;
      uint32_t phase = 0, tphase = 0, a_phase = 0;
      bool ok = true;
      const uint32_t a0 = smem_u32(sA);
      for (int t = blockIdx.x; t < p.num_own_tiles && ok; t += gridDim.x) {
        if (!mbar_wait(a_full, a_phase, abort_flag)) {
          ok = false;
          break;
        }
        a_phase ^= 1u;
        tc_fence_after();
        for (int j = 0; j < p.num_partner_tiles; ++j) {
          if (!mbar_wait(&full[stage], phase, abort_flag) || !mbar_wait(&tempty[buf], tphase ^ 1u, abort_flag)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t b0 = smem_u32(sB + stage * KB * kPartnerBytesPerKB);
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const uint32_t d_tmem = tmem_base + (uint32_t)(buf * 256 + h * 128);
#pragma unroll
            for (int k = 0; k < KB * 4; ++k) {
              const int kb = k >> 2, kk = k & 3;
              const uint64_t adesc = sdesc_sw128(a0 + kb * kOwnBytesPerKB + h * 128 * 128 + kk * 32);
              const uint64_t bdesc = sdesc_sw128(b0 + kb * kPartnerBytesPerKB + kk * 32);
              umma_bf16(d_tmem, adesc, bdesc, idesc, k > 0 ? 1u : 0u);
            }
          }
          umma_commit(&empty[stage]);
          umma_commit(&tfull[buf]);
          if (j == p.num_partner_tiles - 1) umma_commit(a_empty);
          if (++stage == STAGES) {
            stage = 0;
            phase ^= 1u;
          }
          buf ^= 1;
          if (buf == 0) tphase ^= 1u;
        }
      }
      if (!ok && !*abort_flag) raise_error(p.err, abort_flag, kErrTimeout);
      // all MMAs issued by this thread complete before TMEM is released
      umma_commit(mma_done);
      mbar_wait_drain(mma_done, 0, 100000000ull);
    }
    __syncwarp();
  } else {
    // ------------------------------------------------------------ epilogue
    const int ew = warp - 2;
    const int q = warp & 3;   // TMEM lane quadrant this warp may access
    const int h = ew >> 2;    // own sub-tile: rows [h*128, h*128+128)
    const float c = p.c;
    const double shift = __ldg(p.lmax);
    int buf = 0;
    uint32_t tphase = 0;
    bool ok = true;
    double r_max = 0.0, r_sum = 0.0, sq = 0.0, nf = 0.0;
    for (int t = blockIdx.x; t < p.num_own_tiles && ok; t += gridDim.x) {
      float sum = 0.0f, comp = 0.0f;
      for (int j = 0; j < p.num_partner_tiles; ++j) {
        const float* gt = p.g + (int64_t)j * kFusedPartnerRows;
        // every lane waits; the outcome is made warp-uniform so that the
        // .sync.aligned TMEM loads below never run with a partial warp
        if (!__all_sync(0xffffffffu, mbar_wait(&tfull[buf], tphase, abort_flag))) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t taddr = tmem_base + ((uint32_t)(q * 32) << 16) + (uint32_t)(buf * 256 + h * 128);
        float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
#pragma unroll
        for (int chunk = 0; chunk < 4; ++chunk) {
          float v[32];
          tmem_ld32x32(taddr + chunk * 32, v);
          if (chunk == 3) {
            // this warp's part of the accumulator buffer has been read: hand it back to the MMA warp
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&tempty[buf]);
          }
          const float4* g4 = reinterpret_cast<const float4*>(gt + chunk * 32);
#pragma unroll
          for (int i = 0; i < 8; ++i) {
            const float4 gg = __ldg(g4 + i);
            a0 += ex2_approx(fmaf(v[4 * i + 0], c, gg.x));
            a1 += ex2_approx(fmaf(v[4 * i + 1], c, gg.y));
            a2 += ex2_approx(fmaf(v[4 * i + 2], c, gg.z));
            a3 += ex2_approx(fmaf(v[4 * i + 3], c, gg.w));
          }
        }
        // compensated (Kahan) accumulation of the per-tile partial sums
        const float tile = (a0 + a1) + (a2 + a3);
        const float y = tile - comp;
        const float tsum = sum + y;
        comp = (tsum - sum) - y;
        sum = tsum;
        buf ^= 1;
        if (buf == 0) tphase ^= 1u;
      }
      if (!ok) break;
      const int64_t row = (int64_t)t * kFusedOwnRows + h * 128 + q * 32 + lane;
      if (row < p.rows) {
        const RowResult rr = row_update(log((double)sum), shift, p.b2s ? p.b2s[row] : 0.0f, p.mass[row],
                                        p.log_u[row], p.residual != 0);
        if (p.update) {
          p.log_u[row] = rr.log_u;
          p.ell[row] = rr.ell;
        }
        r_max = fmax(r_max, rr.r_rel);
        r_sum += rr.r_abs;
        sq += rr.u2;
        if (!isfinite(rr.log_u) || !isfinite(rr.ell)) nf += 1.0;
      }
    }
    if (!ok && !*abort_flag) raise_error(p.err, abort_flag, kErrTimeout);
    // reduce the CTA's partials over the 256 epilogue threads
    for (int o = 16; o > 0; o >>= 1) {
      r_max = fmax(r_max, __shfl_xor_sync(0xffffffffu, r_max, o));
      r_sum += __shfl_xor_sync(0xffffffffu, r_sum, o);
      sq += __shfl_xor_sync(0xffffffffu, sq, o);
      nf += __shfl_xor_sync(0xffffffffu, nf, o);
    }
    if (lane == 0) {
      red[0 * kEpiWarps + ew] = r_max;
      red[1 * kEpiWarps + ew] = r_sum;
      red[2 * kEpiWarps + ew] = sq;
      red[3 * kEpiWarps + ew] = nf;
    }
    named_bar_sync(1, kEpiWarps * 32);
    if (ew == 0 && lane == 0) {
      double m0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
      for (int w = 0; w < kEpiWarps; ++w) {
        m0 = fmax(m0, red[w]);
        s1 += red[kEpiWarps + w];
        s2 += red[2 * kEpiWarps + w];
        s3 += red[3 * kEpiWarps + w];
      }
      p.partials[4 * blockIdx.x + 0] = m0;
      p.partials[4 * blockIdx.x + 1] = s1;
      p.partials[4 * blockIdx.x + 2] = s2;
      p.partials[4 * blockIdx.x + 3] = s3;
    }
  }

  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(tmem_base, kTmemCols);
  }
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn get_encode_fn() {
  static EncodeTiledFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, []() {
    void* ptr = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(ptr);
  });
  return fn;
}

cudaError_t make_map(CUtensorMap* map, const __nv_bfloat16* base, int64_t rows, int64_t kp, int box_rows) {
  EncodeTiledFn enc = get_encode_fn();
  if (enc == nullptr) return cudaErrorNotSupported;
  const cuuint64_t dims[2] = {(cuuint64_t)kp, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)kp * sizeof(__nv_bfloat16)};
  const cuuint32_t box[2] = {(cuuint32_t)kKBlock, (cuuint32_t)box_rows};
  const cuuint32_t estr[2] = {1, 1};
  const CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<__nv_bfloat16*>(base), dims, strides,
                         box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                         CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

constexpr int kStagesKB1 = 6;
constexpr int kStagesKB2 = 4;

}  // namespace

cudaError_t fused_prepare(tu_market* m) {
  cudaError_t e;
  if ((e = make_map(&m->X.tm_own, m->X.fac16, m->X.rows, m->kp, kFusedOwnRows)) != cudaSuccess) return e;
  if ((e = make_map(&m->X.tm_partner, m->X.fac16, m->X.rows, m->kp, kFusedPartnerRows)) != cudaSuccess) return e;
  if ((e = make_map(&m->Y.tm_own, m->Y.fac16, m->Y.rows, m->kp, kFusedOwnRows)) != cudaSuccess) return e;
  if ((e = make_map(&m->Y.tm_partner, m->Y.fac16, m->Y.rows, m->kp, kFusedPartnerRows)) != cudaSuccess) return e;
  if ((e = cudaFuncSetAttribute(k_fused_halfsweep<1, kStagesKB1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                smem_bytes<1>(kStagesKB1))) != cudaSuccess)
    return e;
  if ((e = cudaFuncSetAttribute(k_fused_halfsweep<2, kStagesKB2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                smem_bytes<2>(kStagesKB2))) != cudaSuccess)
    return e;
  return cudaSuccess;
}

cudaError_t launch_fused_halfsweep(tu_market* m, int side, int residual, int update, int* nparts_out) {
  Side& own = side == 0 ? m->X : m->Y;
  Side& partner = side == 0 ? m->Y : m->X;
  FusedParams p;
  p.rows = own.rows;
  p.num_own_tiles = (int)((own.rows + kFusedOwnRows - 1) / kFusedOwnRows);
  p.num_partner_tiles = (int)((partner.rows + kFusedPartnerRows - 1) / kFusedPartnerRows);
  p.c = (float)(1.4426950408889634 / (2.0 * m->sigma));
  p.g = partner.pvec;
  p.lmax = partner.lmax;
  p.b2s = own.b2s;
  p.mass = own.mass;
  p.log_u = own.log_u;
  p.ell = own.ell;
  p.partials = m->partials;
  p.err = m->err_dev;
  p.residual = residual;
  p.update = update;
  int grid = p.num_own_tiles < m->num_sms ? p.num_own_tiles : m->num_sms;
  if (grid > kMaxPartials) grid = kMaxPartials;
  const int kb = (int)(m->kp / kKBlock);
  if (kb == 1) {
    k_fused_halfsweep<1, kStagesKB1><<<grid, kThreads, smem_bytes<1>(kStagesKB1), m->stream>>>(
        own.tm_own, partner.tm_partner, p);
  } else if (kb == 2) {
    k_fused_halfsweep<2, kStagesKB2><<<grid, kThreads, smem_bytes<2>(kStagesKB2), m->stream>>>(
        own.tm_own, partner.tm_partner, p);
  } else {
    return cudaErrorNotSupported;
  }
  *nparts_out = grid;
  return cudaGetLastError();
}

// Same kernel on caller-described buffers (no market object): used by the
// allocation-free entry point. Tensor maps are built on the host stack.
cudaError_t launch_fused_halfsweep_raw(const FusedRaw& r, cudaStream_t stream, int num_sms, int* nparts_out) {
  CUtensorMap own_map, partner_map;
  cudaError_t e;
  if ((e = make_map(&own_map, r.own16, r.rows, r.kp, kFusedOwnRows)) != cudaSuccess) return e;
  if ((e = make_map(&partner_map, r.par16, r.cols, r.kp, kFusedPartnerRows)) != cudaSuccess) return e;
  FusedParams p;
  p.rows = r.rows;
  p.num_own_tiles = (int)((r.rows + kFusedOwnRows - 1) / kFusedOwnRows);
  p.num_partner_tiles = (int)((r.cols + kFusedPartnerRows - 1) / kFusedPartnerRows);
  p.c = (float)(1.4426950408889634 / (2.0 * r.sigma));
  p.g = r.g;
  p.lmax = r.lmax;
  p.b2s = r.b2s;
  p.mass = r.mass;
  p.log_u = r.log_u;
  p.ell = r.ell;
  p.partials = r.partials;
  p.err = r.err;
  p.residual = r.residual;
  p.update = 1;
  int grid = p.num_own_tiles < num_sms ? p.num_own_tiles : num_sms;
  if (grid > kMaxPartials) grid = kMaxPartials;
  const int kb = (int)(r.kp / kKBlock);
  if (kb == 1) {
    if ((e = cudaFuncSetAttribute(k_fused_halfsweep<1, kStagesKB1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  smem_bytes<1>(kStagesKB1))) != cudaSuccess)
      return e;
    k_fused_halfsweep<1, kStagesKB1><<<grid, kThreads, smem_bytes<1>(kStagesKB1), stream>>>(own_map, partner_map, p);
  } else if (kb == 2) {
    if ((e = cudaFuncSetAttribute(k_fused_halfsweep<2, kStagesKB2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  smem_bytes<2>(kStagesKB2))) != cudaSuccess)
      return e;
    k_fused_halfsweep<2, kStagesKB2><<<grid, kThreads, smem_bytes<2>(kStagesKB2), stream>>>(own_map, partner_map, p);
  } else {
    return cudaErrorNotSupported;
  }
  *nparts_out = grid;
  return cudaGetLastError();
}

}  // namespace tu
