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
// CTA layout (576 threads, one CTA per SM, persistent over own tiles):
//   warp 0     : producer (one elected thread): TMA loads of the own tile
//                [F|K]_j (256 rows x kp) once per own tile (double-buffered
//                when kp = 64) and of partner tiles (128 rows x kp) through a
//                STAGES-deep shared-memory ring (a stage is a whole partner
//                tile, or with four 128-byte k blocks per row one k block of
//                it), plus a bulk copy of each partner tile's 128 g values
//                (e4m3 factors: and of its 128 row scales) into an 8-slot ring
//                that the epilogue reads with broadcast loads.
//   warp 1     : MMA issuer (one thread): two tcgen05.mma M=128 N=128 chains
//                (own rows 0-127 and 128-255) per partner tile into one of two
//                TMEM accumulator buffers (2 x 256 columns = all 512).
//   warps 2-17 : epilogue: epilogue warp e reads TMEM lane quadrant (e+2)%4
//                of own sub-tile (e/4)%2 and column half e/8 of every partner
//                tile, i.e. one own row and 64 columns per thread, so the row
//                reduction stays inside the thread; the two column halves of
//                a row meet through shared memory at the end of the own tile.
//                TMEM loads run one 32-column chunk ahead of the arithmetic;
//                per pair of columns one packed FMA (f32x2), two ex2.approx
//                and one packed add; per-tile partials go into a compensated
//                (Kahan) sum.
// In a batched launch the own tiles of a CTA come from a list of
// (market, own tile) items of many independent markets.
// Every wait is bounded (kWaitLimitNs); a wait that runs out raises the
// abort flag and the error word, the roles drain, TMEM is freed, and the
// kernel returns.
#include "tu_internal.cuh"

#include <cstring>
#include <mutex>

namespace tu {

namespace {

constexpr int kEpiWarps = 16;
constexpr int kThreads = 64 + kEpiWarps * 32;  // producer warp, MMA warp, epilogue warps
constexpr int kOwnBytesPerKB = kFusedOwnRows * 128;          // 32 KB per 64-wide k block
constexpr int kPartnerBytesPerKB = kFusedPartnerRows * 128;  // 16 KB per 64-wide k block
constexpr int kGSlots = 8;                                   // g ring depth
constexpr int kGBytes = kFusedPartnerRows * 4;               // one partner tile of g (512 B)
constexpr uint32_t kTmemCols = 512;

// Epilogue modes of the one fused kernel: the same TMA / MMA pipeline forms
// the tiles of c * phi_hat + g; the epilogue either reduces them (a half-sweep),
// keeps the k best columns of every row (ranked lists) or writes mu.
// Markets whose factor range is too wide for one shift per half-sweep (see
// market.cu) take kModeSweepWide: a half-sweep that keeps a running maximum
// per row and rescales the row's sum whenever it grows (the log-domain
// rescale of an online softmax), so that no term's exponent exceeds 0.
enum : int { kModeSweep = 0, kModeTopK = 1, kModeMu = 2, kModeTopKShared = 3, kModeSweepWide = 4 };

struct FusedParams {
  int64_t rows;            // own users of this launch: [row0, row0 + rows)
  int64_t row0;            // first own user
  int64_t col0;            // first partner column streamed (multiple of 4)
  int64_t ncols;           // partner columns streamed: [col0, col0 + ncols)
  int num_own_tiles;       // ceil(rows / 256)
  int num_partner_tiles;   // ceil(ncols / 128)
  float c;                 // log2(e) / (2 sigma)
  const float* g;          // partner prepared potentials (index = partner user), -inf padded
  const double* lmax;      // partner shift (natural log)
  const double* own_off;   // offset added to the stored own potentials, or nullptr for 0   (sweep)
  float4* grp;             // own-side groups written by an updating pass, or nullptr        (sweep)
  const float* b2s;        // own bias / (2 sigma), or nullptr          (sweep)
  const double* mass;      // own capacities                             (sweep)
  double* log_u;           // own potentials (in: old, out: new)          (sweep)
  double* ell;             // own ell: out (sweep), in (ranked lists, mu)
  double* partials;        // [gridDim.x][4]                              (sweep)
  int* err;                // device error word
  int residual;
  int update;
  const double* omega;     // over-relaxation factor (device scalar) or nullptr for 1  (sweep)
  // batched launches: per-market descriptors and this launch's item lists
  const BatchDesc* bdesc;
  const int2* items;
  const int* cta_start;
  // ranked lists: for own user row0 + r, idx[r * k + i], logmu[r * k + i], best first
  int k;
  int32_t* idx;
  float* logmu;
  float* hand_v;           // rows x k scratch: second column half's list
  int32_t* hand_i;
  // mu block: out[(r) * ld + (col - y0)] for partner col in [y0, y0 + ny)
  float* out;
  int64_t ld;
  int64_t y0;
  int64_t ny;
  // e4m3 factors: per-row scales of the own side (index row0 + r) and of the
  // partner side (index = partner user); the product of row r and partner
  // column j is fs_own[r] * fs_par[j] * <e4m3 row r, e4m3 row j>
  const float* fs_own;
  const float* fs_par;
  // partner split (single-market half-sweeps, 1 = off): an item is an own
  // tile and one of `split` contiguous ranges of its partner tiles; each
  // epilogue warp writes its rows' partial sums to part[s * rows + r], and the
  // warp that completes a (tile, 32-row block), counted in split_cnt, sums
  // the partials in range order and updates the rows
  int split;
  int range_major;         // items ordered range by range (every own tile against range 0 first)
  // L2 residency of the partner matrix (single-market launches): this
  // fraction of its lines is loaded evict-last, so that a partner matrix
  // larger than L2 keeps a fixed part resident across the waves of own tiles
  // (0: no hint)
  float l2_keep;
  float4* part;
  int* split_cnt;
  // folded g (BF16 half-sweeps, kp = 64): the partner side's g / c as the
  // K = 16 operand of one extra MMA per chain and partner tile, 4 KB per
  // partner tile of 128 rows in the unswizzled K-major layout (written by the
  // preparation kernel)
  const uint8_t* gfold;
};

// Own-tile buffers: with one 128-byte k block per row the next own tile is
// loaded while the current one is still in use (short items of batched
// launches); with two or four there is room for one only.
template <int KB>
constexpr int kABufs = KB == 1 ? 2 : 1;

// k blocks per partner stage: with four k blocks per row (d up to 128 in
// BF16, 256 in e4m3) a whole 64 KB partner tile would leave room for one
// stage beside the 128 KB own tile, so a stage then carries one k block and a
// partner tile takes four stages.
constexpr int kbs_for(int KB) { return KB == 4 ? 1 : KB; }

// Operand formats: BF16, e4m3 with one scale per side, e4m3 with one per row.
enum : int { kFmtBF16 = 0, kFmtE4M3Side = 1, kFmtE4M3Rows = 2 };

// shared memory: [A: ABUFS x KB x 32 KB][B: STAGES x KBS x 16 KB][g ring: 8 x 512 B]
//                [per-row scales: scale ring 8 x 512 B][barriers and flags: 512 B]
//                [reduction: 512 B][row hand-over: 2 x 256 floats]
constexpr int kTailBytes = 512 + 512 + 2 * kFusedOwnRows * 4;
// folded g: the partner tile's K = 16 operand rides in its (last) stage, the
// own side's constant operand (ones in columns 0-2) is one tile of its own.
// Taken for rows of one k block (d <= 32 in BF16, d <= 64 in e4m3 with one
// scale per side), where the tensor pipe has room for a fifth MMA per chain
// and the epilogue sheds its g loads: batched d = 32 half-sweep 5.44 -> 5.12
// ms, a 1e5 d = 32 sweep 3.54 -> 3.37 ms; with two BF16 k blocks (d =
// 33..64) the ninth MMA costs more than it saves (1e6 d = 64 half-sweep
// 184.5 -> 187.1 ms), so those keep g in the shared ring. e4m3 rows with one
// scale per side: 1e6 d = 64 half-sweep 149.4 -> 142.5 ms; there the fold MMA
// is a separate kind::f16 MMA (BF16 ones x BF16 g / c) into the same FP32
// accumulator. e4m3 rows with per-row scales cannot fold: the own row's scale
// multiplies phi, so no per-column constant added to it gives g in every row.
constexpr int kFoldBytes = kFusedPartnerRows * 32;
constexpr bool fold_for(int KB, int MODE, bool BATCH, int fmt, bool nofold) {
  return MODE == kModeSweep && (fmt == kFmtBF16 || fmt == kFmtE4M3Side) && KB == 1 && !nofold;
}
constexpr int stage_bytes(int KB, bool fold) { return kbs_for(KB) * kPartnerBytesPerKB + (fold ? kFoldBytes : 0); }
constexpr int smem_bytes(int KB, int fmt, int stages, bool fold = false) {
  return 1024 /*alignment slack*/ + (KB == 1 ? 2 : 1) * KB * kOwnBytesPerKB + stages * stage_bytes(KB, fold) +
         (fold ? kFoldBytes : 0) + kGSlots * kGBytes * (fmt == kFmtE4M3Rows ? 2 : 1) + kTailBytes;
}

__device__ __forceinline__ void raise_error(int* err, volatile int* abort_flag, int code) {
  atomicCAS(err, kErrNone, code);
  *abort_flag = 1;
}

// 1D bulk copy global -> shared, completion counted on an mbarrier (16-byte aligned, size % 16 == 0).
__device__ __forceinline__ void bulk_load(void* smem_dst, const void* gsrc, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(smem_dst)),
      "l"(reinterpret_cast<uint64_t>(gsrc)), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// Issue a 32-lane x 32-column FP32 TMEM load without waiting for it.
__device__ __forceinline__ void tmem_ld_issue(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr)
      : "memory");
}

// Wait for the outstanding TMEM loads; the registers are passed through so
// that no use of them can be scheduled before the wait.
__device__ __forceinline__ void tmem_ld_wait(uint32_t (&r)[32]) {
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                 "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]),
                 "+r"(r[15]), "+r"(r[16]), "+r"(r[17]), "+r"(r[18]), "+r"(r[19]), "+r"(r[20]), "+r"(r[21]),
                 "+r"(r[22]), "+r"(r[23]), "+r"(r[24]), "+r"(r[25]), "+r"(r[26]), "+r"(r[27]), "+r"(r[28]),
                 "+r"(r[29]), "+r"(r[30]), "+r"(r[31])
               :
               : "memory");
}

// acc(2 lanes) += (ex2(phi0 * c + g0), ex2(phi1 * c + g1)) with packed FP32x2 FMA and add.
__device__ __forceinline__ void pair_step(uint64_t& acc, uint32_t phi0, uint32_t phi1, float g0, float g1,
                                          uint64_t cc) {
  asm("{\n\t.reg .b64 a, gg, t, e;\n\t.reg .f32 t0, t1, e0, e1;\n\t"
      "mov.b64 a, {%1, %2};\n\t"
      "mov.b64 gg, {%3, %4};\n\t"
      "fma.rn.f32x2 t, a, %5, gg;\n\t"
      "mov.b64 {t0, t1}, t;\n\t"
      "ex2.approx.ftz.f32 e0, t0;\n\t"
      "ex2.approx.ftz.f32 e1, t1;\n\t"
      "mov.b64 e, {e0, e1};\n\t"
      "add.rn.f32x2 %0, %0, e;\n\t}"
      : "+l"(acc)
      : "r"(phi0), "r"(phi1), "f"(g0), "f"(g1), "l"(cc));
}

// e4m3 factors: acc += (ex2(phi0 f0 c + g0), ex2(phi1 f1 c + g1)), f the
// partner rows' scales (the own row's scale is folded into c).
__device__ __forceinline__ void pair_step_scaled(uint64_t& acc, uint32_t phi0, uint32_t phi1, float g0, float g1,
                                                 float f0, float f1, uint64_t cc) {
  asm("{\n\t.reg .b64 a, gg, ff, t, e;\n\t.reg .f32 t0, t1, e0, e1;\n\t"
      "mov.b64 a, {%1, %2};\n\t"
      "mov.b64 gg, {%3, %4};\n\t"
      "mov.b64 ff, {%5, %6};\n\t"
      "mul.rn.f32x2 t, a, ff;\n\t"
      "fma.rn.f32x2 t, t, %7, gg;\n\t"
      "mov.b64 {t0, t1}, t;\n\t"
      "ex2.approx.ftz.f32 e0, t0;\n\t"
      "ex2.approx.ftz.f32 e1, t1;\n\t"
      "mov.b64 e, {e0, e1};\n\t"
      "add.rn.f32x2 %0, %0, e;\n\t}"
      : "+l"(acc)
      : "r"(phi0), "r"(phi1), "f"(g0), "f"(g1), "f"(f0), "f"(f1), "l"(cc));
}

// Folded g: acc += (ex2(D0 * c), ex2(D1 * c)), D = phi + g / c from the MMA.
__device__ __forceinline__ void pair_step_fold(uint64_t& acc, uint32_t d0, uint32_t d1, uint64_t cc) {
  asm("{\n\t.reg .b64 a, t, e;\n\t.reg .f32 t0, t1, e0, e1;\n\t"
      "mov.b64 a, {%1, %2};\n\t"
      "mul.rn.f32x2 t, a, %3;\n\t"
      "mov.b64 {t0, t1}, t;\n\t"
      "ex2.approx.ftz.f32 e0, t0;\n\t"
      "ex2.approx.ftz.f32 e1, t1;\n\t"
      "mov.b64 e, {e0, e1};\n\t"
      "add.rn.f32x2 %0, %0, e;\n\t}"
      : "+l"(acc)
      : "r"(d0), "r"(d1), "l"(cc));
}

__device__ __forceinline__ void chunk_sum_fold(const uint32_t (&v)[32], uint64_t cc, uint64_t (&acc)[4]) {
#pragma unroll
  for (int i = 0; i < 16; ++i) pair_step_fold(acc[i & 3], v[2 * i], v[2 * i + 1], cc);
}

// phi of column i of a chunk, times the partner row's scale (e4m3 factors
// with per-row scales)
template <bool RS>
__device__ __forceinline__ float scaled_phi(uint32_t v, const float* fs, int i) {
  if constexpr (RS) return __uint_as_float(v) * fs[i];
  return __uint_as_float(v);
}

__device__ __forceinline__ float unpack_sum(uint64_t a) {
  return __uint_as_float((uint32_t)a) + __uint_as_float((uint32_t)(a >> 32));
}

// Sum over one 32-column chunk: 16 packed pairs into four packed accumulators.
template <bool RS>
__device__ __forceinline__ void chunk_sum(const uint32_t (&v)[32], const float4* gs4, const float4* fs4, uint64_t cc,
                                          uint64_t (&acc)[4]) {
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const float4 gg = gs4[i];
    if constexpr (RS) {
      const float4 ff = fs4[i];
      pair_step_scaled(acc[(2 * i) & 3], v[4 * i + 0], v[4 * i + 1], gg.x, gg.y, ff.x, ff.y, cc);
      pair_step_scaled(acc[(2 * i + 1) & 3], v[4 * i + 2], v[4 * i + 3], gg.z, gg.w, ff.z, ff.w, cc);
    } else {
      pair_step(acc[(2 * i) & 3], v[4 * i + 0], v[4 * i + 1], gg.x, gg.y, cc);
      pair_step(acc[(2 * i + 1) & 3], v[4 * i + 2], v[4 * i + 3], gg.z, gg.w, cc);
    }
  }
}

// ---- wide markets: one pass with a running maximum per row -----------------

// t = (phi0, phi1) * c + (g0, g1); e4m3 per-row scales: (phi0 f0, phi1 f1) * c + (g0, g1)
template <bool RS>
__device__ __forceinline__ uint64_t pair_exponents(uint32_t phi0, uint32_t phi1, float g0, float g1, float f0,
                                                   float f1, uint64_t cc) {
  uint64_t t;
  if constexpr (RS) {
    asm("{\n\t.reg .b64 a, gg, ff, x;\n\t"
        "mov.b64 a, {%1, %2};\n\t"
        "mov.b64 gg, {%3, %4};\n\t"
        "mov.b64 ff, {%5, %6};\n\t"
        "mul.rn.f32x2 x, a, ff;\n\t"
        "fma.rn.f32x2 %0, x, %7, gg;\n\t}"
        : "=l"(t)
        : "r"(phi0), "r"(phi1), "f"(g0), "f"(g1), "f"(f0), "f"(f1), "l"(cc));
  } else {
    asm("{\n\t.reg .b64 a, gg;\n\t"
        "mov.b64 a, {%1, %2};\n\t"
        "mov.b64 gg, {%3, %4};\n\t"
        "fma.rn.f32x2 %0, a, %5, gg;\n\t}"
        : "=l"(t)
        : "r"(phi0), "r"(phi1), "f"(g0), "f"(g1), "l"(cc));
  }
  return t;
}

// acc(2 lanes) += (ex2(t0 + m), ex2(t1 + m)), mm = (m, m)
__device__ __forceinline__ void ex2_add_shifted(uint64_t& acc, uint64_t t, uint64_t mm) {
  asm("{\n\t.reg .b64 x, e;\n\t.reg .f32 x0, x1, e0, e1;\n\t"
      "add.rn.f32x2 x, %1, %2;\n\t"
      "mov.b64 {x0, x1}, x;\n\t"
      "ex2.approx.ftz.f32 e0, x0;\n\t"
      "ex2.approx.ftz.f32 e1, x1;\n\t"
      "mov.b64 e, {e0, e1};\n\t"
      "add.rn.f32x2 %0, %0, e;\n\t}"
      : "+l"(acc)
      : "l"(t), "l"(mm));
}

// acc(2 lanes) *= (s, s)
__device__ __forceinline__ void scale2(uint64_t& acc, float s) {
  const uint64_t ss = ((uint64_t)__float_as_uint(s) << 32) | __float_as_uint(s);
  asm("mul.rn.f32x2 %0, %0, %1;" : "+l"(acc) : "l"(ss));
}

// The larger of a, b and c; NaN if any of them is NaN.
__device__ __forceinline__ float max3_nan(float a, float b, float c) {
  float r;
  asm("max.NaN.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
  return r;
}

// 2^d for an integer-valued d <= 0, as an exact power of two; 0 for d below
// -126 (FP32's normal range), for -inf and for NaN.
__device__ __forceinline__ float exp2_int(float d) {
  return d >= -126.0f ? __int_as_float((127 + (int)d) << 23) : 0.0f;
}

// One 32-column chunk of a wide market's row: the exponents t = c * phi + g,
// their largest; when that exceeds the row's running shift M (an integer,
// -inf before the first term) the shift becomes M' = ceil(max) and all the
// row has summed so far (this tile's packed partials acc, the compensated
// sum over the earlier tiles) is multiplied by 2^(M - M'), a power of two,
// so exactly; then acc += 2^(t - M). Every term is at most 1, and the row's
// log-sum is log(sum) + M ln 2.
template <bool RS>
__device__ __forceinline__ void chunk_sum_wide(uint32_t (&v)[32], const float4* gs4, const float4* fs4, uint64_t cc,
                                               uint64_t (&acc)[4], float& M, float& sum, float& comp) {
  // the exponents replace the loaded values in place
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const float4 gg = gs4[i];
    float4 ff = make_float4(1.f, 1.f, 1.f, 1.f);
    if constexpr (RS) ff = fs4[i];
    const uint64_t t0 = pair_exponents<RS>(v[4 * i + 0], v[4 * i + 1], gg.x, gg.y, ff.x, ff.y, cc);
    const uint64_t t1 = pair_exponents<RS>(v[4 * i + 2], v[4 * i + 3], gg.z, gg.w, ff.z, ff.w, cc);
    v[4 * i + 0] = (uint32_t)t0;
    v[4 * i + 1] = (uint32_t)(t0 >> 32);
    v[4 * i + 2] = (uint32_t)t1;
    v[4 * i + 3] = (uint32_t)(t1 >> 32);
  }
  float mx = -INFINITY;
#pragma unroll
  for (int k = 0; k < 16; ++k) mx = max3_nan(mx, __uint_as_float(v[2 * k]), __uint_as_float(v[2 * k + 1]));
  if (!(mx <= M)) {  // a larger maximum (or NaN, which then reaches the sum)
    const float Mn = ceilf(mx);
    const float sc = exp2_int(M - Mn);
    sum *= sc;
    comp *= sc;
#pragma unroll
    for (int k = 0; k < 4; ++k) scale2(acc[k], sc);
    M = Mn;
  }
  if (M == -INFINITY) return;  // every exponent so far is -inf: no terms
  const uint64_t mm = ((uint64_t)__float_as_uint(-M) << 32) | __float_as_uint(-M);
#pragma unroll
  for (int k = 0; k < 16; ++k)
    ex2_add_shifted(acc[k & 3], ((uint64_t)v[2 * k + 1] << 32) | v[2 * k], mm);
}

constexpr int kMaxTopK = 64;

// Insert score s of partner col into a thread's list, sorted by decreasing
// score; equal scores keep the earlier (lower) column first. Returns the new
// threshold (the k-th best score, -inf while the list is not full). Kept out
// of line: it runs rarely, and one copy keeps the hot loop small.
__device__ __noinline__ float top_insert(float* tv, int32_t* ti, int* cnt, int k, float s, int32_t col) {
  int c = *cnt;
  int pos = c < k ? c : k - 1;
  while (pos > 0 && s > tv[pos - 1]) {
    tv[pos] = tv[pos - 1];
    ti[pos] = ti[pos - 1];
    --pos;
  }
  tv[pos] = s;
  ti[pos] = col;
  if (c < k) *cnt = ++c;
  return c == k ? tv[k - 1] : -INFINITY;
}

// Ranked lists: score = c * phi_hat + g (log2 units, shifted; same order as
// log mu within a row). The chunk's maximum is compared with the running k-th
// best first, so most chunks cost one FFMA and one max per column.
template <bool RS>
__device__ __forceinline__ void chunk_topk(const uint32_t (&v)[32], const float* g, const float* fs, float c,
                                           int64_t colbase, int k, float* tv, int32_t* ti, int* cnt, float& thr) {
  const float4* g4 = reinterpret_cast<const float4*>(g);
  float s[32];
  float mx = -INFINITY;
#pragma unroll
  for (int i4 = 0; i4 < 8; ++i4) {
    const float4 gg = g4[i4];
    s[4 * i4 + 0] = fmaf(scaled_phi<RS>(v[4 * i4 + 0], fs, 4 * i4 + 0), c, gg.x);
    s[4 * i4 + 1] = fmaf(scaled_phi<RS>(v[4 * i4 + 1], fs, 4 * i4 + 1), c, gg.y);
    s[4 * i4 + 2] = fmaf(scaled_phi<RS>(v[4 * i4 + 2], fs, 4 * i4 + 2), c, gg.z);
    s[4 * i4 + 3] = fmaf(scaled_phi<RS>(v[4 * i4 + 3], fs, 4 * i4 + 3), c, gg.w);
    mx = fmaxf(mx, fmaxf(fmaxf(s[4 * i4 + 0], s[4 * i4 + 1]), fmaxf(s[4 * i4 + 2], s[4 * i4 + 3])));
  }
  if (mx > thr) {
#pragma unroll
    for (int e = 0; e < 32; ++e)
      if (s[e] > thr) thr = top_insert(tv, ti, cnt, k, s[e], (int32_t)(colbase + e));
  }
}

// Ranked lists with k <= kSharedTopK (kModeTopKShared): every epilogue
// thread keeps the k best (score, column) pairs of its row and column half in
// shared memory, entry i of thread t at [i * kEpiThreads + t] (a warp's
// accesses to one entry are conflict-free), sorted by decreasing score, equal
// scores in increasing column order (the order in which a column half's
// columns arrive). The list starts as k (-inf, INT32_MAX) pairs, so the k-th
// score is the threshold from the first column on. An insertion shifts at
// most k - 1 entries in shared memory. Rows whose rankings differ (a
// converged market, where the potentials cancel the popularity terms) insert
// at different columns, and a warp runs every lane's insertion in turn; with
// the list in shared memory each of those costs a few shared-memory round
// trips instead of a chain through local memory.
constexpr int kSharedTopK = 14;
constexpr int kEpiThreads = kEpiWarps * 32;
constexpr int kTopKListBytes = kSharedTopK * kEpiThreads * 8;
constexpr int kWideShiftBytes = 2 * kFusedOwnRows * 4;  // kModeSweepWide: the row hand-over's shifts
// shared memory a mode needs after the tail area
constexpr int mode_extra_bytes(int mode) {
  return mode == kModeTopKShared ? kTopKListBytes : (mode == kModeSweepWide ? kWideShiftBytes : 0);
}

__device__ __forceinline__ float lds_f32(uint32_t a) {
  float v;
  asm volatile("ld.shared.f32 %0, [%1];" : "=f"(v) : "r"(a));
  return v;
}
__device__ __forceinline__ int32_t lds_s32(uint32_t a) {
  int32_t v;
  asm volatile("ld.shared.s32 %0, [%1];" : "=r"(v) : "r"(a));
  return v;
}
__device__ __forceinline__ void sts_f32(uint32_t a, float v) { asm volatile("st.shared.f32 [%0], %1;" ::"r"(a), "f"(v)); }
__device__ __forceinline__ void sts_s32(uint32_t a, int32_t v) { asm volatile("st.shared.s32 [%0], %1;" ::"r"(a), "r"(v)); }

// Insert (s, col) into the list at shared addresses lv (scores) and li
// (columns) of one thread; s beats the current k-th score. Returns the new
// k-th score. Kept out of line: one copy serves every call site.
__device__ __noinline__ float list_insert(uint32_t lv, uint32_t li, int k, float s, int32_t col) {
  constexpr uint32_t kStride = kEpiThreads * 4;
  uint32_t pos = (uint32_t)(k - 1);
  while (pos > 0) {
    const float above = lds_f32(lv + (pos - 1) * kStride);
    if (!(s > above)) break;
    sts_f32(lv + pos * kStride, above);
    sts_s32(li + pos * kStride, lds_s32(li + (pos - 1) * kStride));
    --pos;
  }
  sts_f32(lv + pos * kStride, s);
  sts_s32(li + pos * kStride, col);
  return lds_f32(lv + (uint32_t)(k - 1) * kStride);
}

template <bool RS>
__device__ __forceinline__ void chunk_topk_shared(const uint32_t (&v)[32], const float* g, const float* fs, float c,
                                                  int64_t colbase, int k, uint32_t lv, uint32_t li, float& thr) {
  const float4* g4 = reinterpret_cast<const float4*>(g);
  float s[32];
  float mx = -INFINITY;
#pragma unroll
  for (int i4 = 0; i4 < 8; ++i4) {
    const float4 gg = g4[i4];
    s[4 * i4 + 0] = fmaf(scaled_phi<RS>(v[4 * i4 + 0], fs, 4 * i4 + 0), c, gg.x);
    s[4 * i4 + 1] = fmaf(scaled_phi<RS>(v[4 * i4 + 1], fs, 4 * i4 + 1), c, gg.y);
    s[4 * i4 + 2] = fmaf(scaled_phi<RS>(v[4 * i4 + 2], fs, 4 * i4 + 2), c, gg.z);
    s[4 * i4 + 3] = fmaf(scaled_phi<RS>(v[4 * i4 + 3], fs, 4 * i4 + 3), c, gg.w);
    mx = fmaxf(mx, fmaxf(fmaxf(s[4 * i4 + 0], s[4 * i4 + 1]), fmaxf(s[4 * i4 + 2], s[4 * i4 + 3])));
  }
  if (mx > thr) {
#pragma unroll
    for (int e = 0; e < 32; ++e)
      if (s[e] > thr) thr = list_insert(lv, li, k, s[e], (int32_t)(colbase + e));
  }
}

// mu block: mu = 2^(c * phi_hat + g + lo) * 2^hi, where hi + lo = (shift + ell_row) log2 e.
template <bool RS>
__device__ __forceinline__ void chunk_mu(const uint32_t (&v)[32], const float* g, const float* fs, float c,
                                         int64_t colbase, float lo, int hi, bool row_ok, int64_t r,
                                         const FusedParams& p) {
  if (!row_ok) return;
  float* orow = p.out + r * p.ld;
#pragma unroll
  for (int i = 0; i < 32; ++i) {
    const int64_t col = colbase + i;
    if (col >= p.y0 && col < p.y0 + p.ny) {
      const float t = fmaf(scaled_phi<RS>(v[i], fs, i), c, g[i]) + lo;
      // (wide markets: an exponent beyond the FP32 range is brought back by hi first)
      orow[col - p.y0] = fabsf(t) <= 100.0f ? ldexpf(ex2_approx(t), hi) : ex2_approx(t + (float)hi);
    }
  }
}

// The items of a batched launch are (market, own tile) pairs.
struct ItemRef {
  const BatchDesc* d;
  int t;
};
__device__ __forceinline__ ItemRef batch_item(const FusedParams& p, int it) {
  const int2 v = p.items[it];
  return {p.bdesc + v.x, v.y};
}

// This CTA's items: own tiles blockIdx.x, blockIdx.x + gridDim.x, ... of one
// market, or a contiguous range of the batched item list (all roles walk the
// same sequence).
template <bool BATCH>
__device__ __forceinline__ int item_begin(const FusedParams& p) {
  if constexpr (BATCH) return p.cta_start[blockIdx.x];
  return blockIdx.x;
}
template <bool BATCH, bool SPLIT>
__device__ __forceinline__ int item_end(const FusedParams& p) {
  if constexpr (BATCH) return p.cta_start[blockIdx.x + 1];
  if constexpr (SPLIT) return p.num_own_tiles * p.split;
  return p.num_own_tiles;
}

// An item of a single-market launch: own tile t and its partner tiles
// [jb, je) (range s of p.split equal parts). Items are ordered tile by tile
// (the ranges of one own tile on neighbouring CTAs), or with range_major
// range by range, so that all CTAs stream one range of the partner matrix
// (small enough to stay in L2) against every own tile before the next.
struct Span {
  int t, s, jb, je;
};
template <bool SPLIT>
__device__ __forceinline__ Span single_span(const FusedParams& p, int it) {
  if constexpr (!SPLIT) return {it, 0, 0, p.num_partner_tiles};
  const int S = p.split;
  int t, s;
  if (p.range_major) {
    s = it / p.num_own_tiles;
    t = it - s * p.num_own_tiles;
  } else {
    t = it / S;
    s = it - t * S;
  }
  const int npt = p.num_partner_tiles;
  return {t, s, (int)((int64_t)s * npt / S), (int)((int64_t)(s + 1) * npt / S)};
}
template <bool BATCH>
__device__ __forceinline__ int item_step() {
  if constexpr (BATCH) return 1;
  return gridDim.x;
}

// BATCH: the CTA's own tiles come from the launch's item list and may belong
// to different markets (tensor maps, vectors and sizes from BatchDesc); the
// residual partials are then written per own tile and epilogue warp instead
// of per CTA.
// KB: 128-byte k blocks per packed row (1, 2 or 4: BF16 kp = 64, 128, 256;
// e4m3 kp = 128, 256, 512).
// FMT: kFmtBF16, or e4m3 factors on tcgen05.mma kind::f8f6f4 with one scale
// per side (kFmtE4M3Side: both folded into p.c) or per row (kFmtE4M3Rows: the
// own row's scale is folded into the row's exponent multiplier, the partner
// rows' scales multiply the accumulator entries in the epilogue).
// SMALL: own tiles of 128 rows (one MMA chain; the epilogue warps of the
// second sub-tile take part in every barrier but load and compute nothing),
// for markets whose 256-row tiles would leave SMs idle: twice the CTAs, each
// finishing its rows in about half the time. Every row's arithmetic is the
// same as with 256-row tiles.
template <int KB, int STAGES, int MODE, bool BATCH, int FMT, bool SMALL = false, bool SPLIT = false,
          bool NOFOLD = false>
__global__ void __launch_bounds__(kThreads, 1)
    k_fused_halfsweep(const __grid_constant__ CUtensorMap tm_own, const __grid_constant__ CUtensorMap tm_partner,
                      const FusedParams p) {
  static_assert(!BATCH || MODE == kModeSweep, "batched launches run half-sweeps only");
  static_assert(!SPLIT || (MODE == kModeSweep && !BATCH), "partner splits are single-market half-sweeps");
  constexpr bool kSweepLike = MODE == kModeSweep || MODE == kModeSweepWide;
  static_assert(!(BATCH && SMALL), "batched launches use 256-row own tiles");
  constexpr int kOwn = SMALL ? kFusedOwnRows / 2 : kFusedOwnRows;  // rows of an own tile
  static_assert(KB == 1 || KB == 2 || KB == 4, "128-byte k blocks per row");
  constexpr bool F8 = FMT != kFmtBF16;      // e4m3 operands
  constexpr bool RS = FMT == kFmtE4M3Rows;  // per-row scales
  constexpr int ABUF = kABufs<KB>;
  constexpr int KBS = kbs_for(KB);   // k blocks per partner stage
  constexpr int SPT = KB / KBS;      // stages per partner tile
  constexpr int XB = F8 ? 128 : kKBlock;  // elements per 128-byte k block (TMA x coordinate step)
  constexpr bool FOLD = fold_for(KB, MODE, BATCH, FMT, NOFOLD);  // g added by an extra MMA
  constexpr int SB = stage_bytes(KB, FOLD);                        // bytes per partner stage
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw_u32 = smem_u32(smem_raw);
  uint8_t* smem = smem_raw + (((raw_u32 + 1023u) & ~1023u) - raw_u32);
  uint8_t* sA = smem;
  uint8_t* sB = smem + ABUF * KB * kOwnBytesPerKB;
  uint8_t* sOnes = sB + STAGES * SB;  // folded g: the own side's constant operand
  float* sG = reinterpret_cast<float*>(sOnes + (FOLD ? kFoldBytes : 0));
  float* sF = sG + kGSlots * kFusedPartnerRows;  // per-row scales: partner scale ring
  uint64_t* bars =
      reinterpret_cast<uint64_t*>(reinterpret_cast<uint8_t*>(sG) + kGSlots * kGBytes * (RS ? 2 : 1));
  uint64_t* full = bars;
  uint64_t* empty = bars + STAGES;
  uint64_t* gfull = bars + 2 * STAGES;
  uint64_t* gempty = gfull + kGSlots;
  uint64_t* a_full = gempty + kGSlots;  // [2]
  uint64_t* a_empty = a_full + 2;       // [2]
  uint64_t* tfull = a_full + 4;         // [2]
  uint64_t* tempty = a_full + 6;        // [2]
  uint64_t* mma_done = a_full + 8;
  uint64_t* rowfull = a_full + 9;   // [2] second column half of the rows written
  uint64_t* rowfree = a_full + 11;  // [2] row hand-over buffer read
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(a_full + 13);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  double* red = reinterpret_cast<double*>(reinterpret_cast<uint8_t*>(bars) + 512);      // 4 x kEpiWarps doubles
  float* rowbuf = reinterpret_cast<float*>(reinterpret_cast<uint8_t*>(bars) + 1024);   // 2 x 256 floats
  // ranked lists in shared memory (kModeTopKShared only): after the tail area
  float* topk_list = reinterpret_cast<float*>(reinterpret_cast<uint8_t*>(bars) + kTailBytes);
  // the running shifts of the second column half's rows (kModeSweepWide only): the same place
  float* wide_shift = topk_list;  // 2 x 256 floats
  static_assert(4 * kEpiWarps * 8 <= 512, "reduction area");
  static_assert((2 * STAGES + 2 * kGSlots + 13) * 8 + 8 <= 512, "barrier area");

  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int s = 0; s < kGSlots; ++s) {
      mbar_init(&gfull[s], 1);
      mbar_init(&gempty[s], kEpiWarps);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&a_full[b], 1);
      mbar_init(&a_empty[b], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&tfull[b], 1);
      mbar_init(&tempty[b], kEpiWarps);
    }
    mbar_init(mma_done, 1);
    for (int b = 0; b < 2; ++b) {
      mbar_init(&rowfull[b], kEpiWarps / 2);
      mbar_init(&rowfree[b], kEpiWarps / 2);
    }
    *abort_flag = 0;
    fence_mbar_init();
    if constexpr (!BATCH) {
      tma_prefetch_map(&tm_own);
      tma_prefetch_map(&tm_partner);
    }
  }
  if (warp == 0) {
    tmem_alloc(tmem_slot, kTmemCols);
    tmem_relinquish();
  }
  if constexpr (FOLD) {
    // the own side's operand of the extra MMA: BF16 ones in columns 0-2 of
    // every row (16-byte chunk q holds columns 0-7 when (q / 8) is even),
    // made visible to the tensor core's (async) proxy
    if (threadIdx.x < kFoldBytes / 16) {
      const bool cols0_7 = ((threadIdx.x / 8) % 2) == 0;
      reinterpret_cast<uint4*>(sOnes)[threadIdx.x] =
          cols0_7 ? make_uint4(0x3F803F80u, 0x00003F80u, 0u, 0u) : make_uint4(0u, 0u, 0u, 0u);
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;

  if (warp == 0) {
    // ------------------------------------------------------------ producer
    if (lane == 0) {
      int stage = 0, gs = 0, ab = 0;
      uint32_t phase = 0, gphase = 0, a_phase = 0;
      const bool hint = !BATCH && p.l2_keep > 0.0f;
      const uint64_t keep_policy = hint ? l2_policy_keep_fraction(p.l2_keep) : 0ull;
      uint32_t armed[STAGES], garmed[kGSlots], a_armed[2] = {0u, 0u};
      for (int s = 0; s < STAGES; ++s) armed[s] = 0;
      for (int s = 0; s < kGSlots; ++s) garmed[s] = 0;
      const BatchDesc* prev = nullptr;
      bool ok = true;
      for (int it = item_begin<BATCH>(p); it < item_end<BATCH, SPLIT>(p) && ok; it += item_step<BATCH>()) {
        const BatchDesc* bd = nullptr;
        int t, jb = 0, je;
        if constexpr (BATCH) {
          const ItemRef w = batch_item(p, it);
          bd = w.d;
          t = w.t;
          je = bd->num_partner_tiles;
          if (bd != prev) {
            tensormap_acquire(&bd->tm_own);
            tensormap_acquire(&bd->tm_partner);
            prev = bd;
          }
        } else {
          const Span sp = single_span<SPLIT>(p, it);
          t = sp.t;
          jb = sp.jb;
          je = sp.je;
        }
        const CUtensorMap* map_own = BATCH ? &bd->tm_own : &tm_own;
        const CUtensorMap* map_partner = BATCH ? &bd->tm_partner : &tm_partner;
        const float* gsrc = BATCH ? bd->g : p.g + p.col0;
        const float* fsrc = BATCH ? bd->fs_par : p.fs_par + p.col0;
        // (SMALL: the 256-row box also brings the next tile's rows, unused)
        const int64_t arow = BATCH ? (int64_t)t * kFusedOwnRows : p.row0 + (int64_t)t * kOwn;
        if (!mbar_wait(&a_empty[ab], a_phase ^ 1u, abort_flag)) {
          ok = false;
          break;
        }
        mbar_arrive_expect_tx(&a_full[ab], KB * kOwnBytesPerKB);
        for (int kb = 0; kb < KB; ++kb)
          tma_load_2d(sA + (ab * KB + kb) * kOwnBytesPerKB, map_own, &a_full[ab], kb * XB, (int)arow);
        ++a_armed[ab];
        if (++ab == ABUF) {
          ab = 0;
          a_phase ^= 1u;
        }
        for (int j = jb; j < je && ok; ++j) {
          for (int sp = 0; sp < SPT; ++sp) {
            if (!mbar_wait(&empty[stage], phase ^ 1u, abort_flag)) {
              ok = false;
              break;
            }
            const bool fold_here = FOLD && sp == SPT - 1;  // the tile's g operand rides in its last stage
            mbar_arrive_expect_tx(&full[stage], KBS * kPartnerBytesPerKB + (fold_here ? kFoldBytes : 0));
            for (int kb = 0; kb < KBS; ++kb) {
              const int px = (sp * KBS + kb) * XB, py = (int)(p.col0 + (int64_t)j * kFusedPartnerRows);
              if (hint) {
                tma_load_2d_hint(sB + stage * SB + kb * kPartnerBytesPerKB, map_partner, &full[stage], px, py,
                                 keep_policy);
              } else {
                tma_load_2d(sB + stage * SB + kb * kPartnerBytesPerKB, map_partner, &full[stage], px, py);
              }
            }
            if (fold_here)
              bulk_load(sB + stage * SB + KBS * kPartnerBytesPerKB,
                        (BATCH ? bd->gfold : p.gfold) + (int64_t)j * kFoldBytes, kFoldBytes, &full[stage]);
            ++armed[stage];
            if (++stage == STAGES) {
              stage = 0;
              phase ^= 1u;
            }
          }
          if (!ok) break;
          if (!mbar_wait(&gempty[gs], gphase ^ 1u, abort_flag)) {
            ok = false;
            break;
          }
          mbar_arrive_expect_tx(&gfull[gs], RS ? 2 * kGBytes : kGBytes);
          bulk_load(sG + gs * kFusedPartnerRows, gsrc + (int64_t)j * kFusedPartnerRows, kGBytes, &gfull[gs]);
          if constexpr (RS)
            bulk_load(sF + gs * kFusedPartnerRows, fsrc + (int64_t)j * kFusedPartnerRows, kGBytes, &gfull[gs]);
          ++garmed[gs];
          if (++gs == kGSlots) {
            gs = 0;
            gphase ^= 1u;
          }
        }
      }
      if (!ok) {
        if (!*abort_flag) raise_error(p.err, abort_flag, kErrTimeout);
        // let the copies already issued land before the CTA's shared memory goes away
        for (int s = 0; s < STAGES; ++s)
          if (armed[s]) mbar_wait_drain(&full[s], (armed[s] - 1u) & 1u, 10000000ull);
        for (int s = 0; s < kGSlots; ++s)
          if (garmed[s]) mbar_wait_drain(&gfull[s], (garmed[s] - 1u) & 1u, 10000000ull);
        for (int b = 0; b < ABUF; ++b)
          if (a_armed[b]) mbar_wait_drain(&a_full[b], (a_armed[b] - 1u) & 1u, 10000000ull);
      }
    }
    __syncwarp();
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      constexpr uint32_t idesc = F8 ? idesc_e4m3_f32(128, kFusedPartnerRows) : idesc_bf16_f32(128, kFusedPartnerRows);
      constexpr uint32_t idesc_fold = idesc_bf16_f32(128, kFusedPartnerRows);  // (BF16 in every format)
      int stage = 0, buf = 0, ab = 0;
      uint32_t phase = 0, tphase = 0, a_phase = 0;
      bool ok = true;
      for (int it = item_begin<BATCH>(p); it < item_end<BATCH, SPLIT>(p) && ok; it += item_step<BATCH>()) {
        int jb = 0, je;
        if constexpr (BATCH) {
          je = batch_item(p, it).d->num_partner_tiles;
        } else {
          const Span sp = single_span<SPLIT>(p, it);
          jb = sp.jb;
          je = sp.je;
        }
        if (!mbar_wait(&a_full[ab], a_phase, abort_flag)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t a0 = smem_u32(sA + ab * KB * kOwnBytesPerKB);
        uint64_t* a_release = &a_empty[ab];
        if (++ab == ABUF) {
          ab = 0;
          a_phase ^= 1u;
        }
        for (int j = jb; j < je && ok; ++j) {
          if (!mbar_wait(&tempty[buf], tphase ^ 1u, abort_flag)) {
            ok = false;
            break;
          }
          for (int sp = 0; sp < SPT; ++sp) {
            if (!mbar_wait(&full[stage], phase, abort_flag)) {
              ok = false;
              break;
            }
            tc_fence_after();
            const uint32_t b0 = smem_u32(sB + stage * SB);
#pragma unroll
            for (int h = 0; h < (SMALL ? 1 : 2); ++h) {
              const uint32_t d_tmem = tmem_base + (uint32_t)(buf * 256 + h * 128);
#pragma unroll
              for (int k = 0; k < KBS * 4; ++k) {
                const int kbl = k >> 2, kk = k & 3;
                const int kb = sp * KBS + kbl;  // k block within the packed row
                const uint64_t adesc = sdesc_sw128(a0 + kb * kOwnBytesPerKB + h * 128 * 128 + kk * 32);
                const uint64_t bdesc = sdesc_sw128(b0 + kbl * kPartnerBytesPerKB + kk * 32);
                const uint32_t accum = (sp > 0 || k > 0) ? 1u : 0u;
                if constexpr (F8) {
                  umma_e4m3(d_tmem, adesc, bdesc, idesc, accum);
                } else {
                  umma_bf16(d_tmem, adesc, bdesc, idesc, accum);
                }
              }
              if constexpr (FOLD) {
                // D += ones x (g / c): every row gets the partner column's g / c
                if (sp == SPT - 1)
                  umma_bf16(d_tmem, sdesc_none(smem_u32(sOnes), 128, 256),
                            sdesc_none(b0 + KBS * kPartnerBytesPerKB, 128, 256), idesc_fold, 1u);
              }
            }
            umma_commit(&empty[stage]);
            if (++stage == STAGES) {
              stage = 0;
              phase ^= 1u;
            }
          }
          if (!ok) break;
          umma_commit(&tfull[buf]);
          if (j == je - 1) umma_commit(a_release);
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
    const int ew = warp - 2;          // 0..15
    const int q = warp & 3;           // TMEM lane quadrant this warp may access
    const int h = (ew >> 2) & 1;      // own sub-tile: rows [h*128, h*128+128)
    const int half = ew >> 3;         // columns [half*64, half*64+64) of every partner tile
    uint64_t cc = 0ull;
    float crow = p.c;  // this thread's row's exponent multiplier (e4m3: times the row's scale)
    // single market: the shift, own offset and omega of the launch (batched: per item)
    const double shift0 = BATCH ? 0.0 : __ldg(p.lmax);
    // (ranked lists and mu blocks run on potentials without pending offsets:
    // every block of sweeps ends by writing them into the arrays)
    const double own_off0 = (kSweepLike && !BATCH && p.own_off != nullptr) ? *p.own_off : 0.0;
    const double omega0 = (!BATCH && p.omega != nullptr && p.update) ? *p.omega : 1.0;
    int buf = 0, gs = 0;
    uint32_t tphase = 0, gphase = 0;
    bool ok = true;
    double r_max = 0.0, r_sum = 0.0, sq = 0.0, nf = 0.0;
    uint32_t va[32], vb[32];
    // ranked lists: this thread's sorted candidates for its row and column half
    float tv[MODE == kModeTopK ? kMaxTopK : 1];
    int32_t ti[MODE == kModeTopK ? kMaxTopK : 1];
    // shared-memory lists (k <= kSharedTopK): this thread's entry 0
    const uint32_t lv = smem_u32(topk_list) + (uint32_t)(ew * 32 + lane) * 4u;
    const uint32_t li = lv + (uint32_t)(kSharedTopK * kEpiThreads) * 4u;
    int tcnt = 0;
    float thr = -INFINITY;
    int tile_iter = 0;
    for (int it = item_begin<BATCH>(p); it < item_end<BATCH, SPLIT>(p) && ok; it += item_step<BATCH>(), ++tile_iter) {
      const BatchDesc* bd = nullptr;
      int t, split_s = 0, jb = 0, je;
      if constexpr (BATCH) {
        const ItemRef w = batch_item(p, it);
        bd = w.d;
        t = w.t;
        je = bd->num_partner_tiles;
      } else {
        const Span sp = single_span<SPLIT>(p, it);
        t = sp.t;
        split_s = sp.s;
        jb = sp.jb;
        je = sp.je;
      }
      const double shift = BATCH ? bd->st[kStShift] : shift0;
      const int rloc = h * 128 + q * 32 + lane;          // row within the own tile
      const int64_t r = (int64_t)t * kOwn + rloc;         // row within the launch
      const bool row_ok = rloc < kOwn && r < (BATCH ? bd->rows : p.rows);
      crow = BATCH ? bd->c : p.c;
      if constexpr (RS) {
        const float* fso = BATCH ? bd->fs_own : p.fs_own;
        if (row_ok) crow *= fso[(BATCH ? 0 : p.row0) + r];
      }
      {
        const uint32_t cb = __float_as_uint(crow);
        cc = ((uint64_t)cb << 32) | cb;
      }
      float sum = 0.0f, comp = 0.0f;
      float mu_lo = 0.0f;
      int mu_hi = 0;
      float wide_m = -INFINITY;  // wide markets: the row's running shift (an integer, log2 units)
      if constexpr (MODE == kModeMu) {
        if (row_ok) {
          const double off = (shift + p.ell[p.row0 + r]) * 1.4426950408889634;
          const double fl = floor(off);
          mu_hi = (int)fl;
          mu_lo = (float)(off - fl);
        }
      }
      if constexpr (MODE == kModeTopK) {
        tcnt = 0;
        thr = -INFINITY;
      }
      if constexpr (MODE == kModeTopKShared) {
        for (int i = 0; i < p.k; ++i) {
          sts_f32(lv + (uint32_t)(i * kEpiThreads) * 4u, -INFINITY);
          sts_s32(li + (uint32_t)(i * kEpiThreads) * 4u, 0x7fffffff);
        }
        thr = -INFINITY;
      }
      for (int j = jb; j < je; ++j) {
        // every lane waits; the outcome is made warp-uniform so that the
        // .sync.aligned TMEM loads below never run with a partial warp
        const bool got = mbar_wait(&tfull[buf], tphase, abort_flag) && mbar_wait(&gfull[gs], gphase, abort_flag);
        if (!__all_sync(0xffffffffu, got)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t taddr =
            tmem_base + ((uint32_t)(q * 32) << 16) + (uint32_t)(buf * 256 + h * 128 + half * 64);
        const float* gsf = sG + gs * kFusedPartnerRows + half * 64;
        const float4* gs4 = reinterpret_cast<const float4*>(gsf);
        const float* fsf = sF + gs * kFusedPartnerRows + half * 64;  // (per-row scales only)
        const float4* fs4 = reinterpret_cast<const float4*>(fsf);
        const int64_t colbase = p.col0 + (int64_t)j * kFusedPartnerRows + half * 64;
        uint64_t acc[4] = {0ull, 0ull, 0ull, 0ull};
        // SMALL: the second sub-tile's warps keep step with the barriers only
        const bool idle = SMALL && h == 1;
        if (!idle) {
          // the second 32-column chunk is loaded while the first is processed
          tmem_ld_issue(taddr, va);
          tmem_ld_wait(va);
          tmem_ld_issue(taddr + 32, vb);
          if constexpr (FOLD) chunk_sum_fold(va, cc, acc);
          if constexpr (MODE == kModeSweep && !FOLD) chunk_sum<RS>(va, gs4, fs4, cc, acc);
          if constexpr (MODE == kModeSweepWide) chunk_sum_wide<RS>(va, gs4, fs4, cc, acc, wide_m, sum, comp);
          if constexpr (MODE == kModeTopK) chunk_topk<RS>(va, gsf, fsf, crow, colbase, p.k, tv, ti, &tcnt, thr);
          if constexpr (MODE == kModeTopKShared)
            chunk_topk_shared<RS>(va, gsf, fsf, crow, colbase, p.k, lv, li, thr);
          if constexpr (MODE == kModeMu) chunk_mu<RS>(va, gsf, fsf, crow, colbase, mu_lo, mu_hi, row_ok, r, p);
          tmem_ld_wait(vb);
        }
        // this warp's part of the accumulator buffer has been read: hand it back to the MMA warp
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&tempty[buf]);
        if (!idle) {
          if constexpr (FOLD) chunk_sum_fold(vb, cc, acc);
          if constexpr (MODE == kModeSweep && !FOLD) chunk_sum<RS>(vb, gs4 + 8, fs4 + 8, cc, acc);
          if constexpr (MODE == kModeSweepWide) chunk_sum_wide<RS>(vb, gs4 + 8, fs4 + 8, cc, acc, wide_m, sum, comp);
          if constexpr (MODE == kModeTopK)
            chunk_topk<RS>(vb, gsf + 32, fsf + 32, crow, colbase + 32, p.k, tv, ti, &tcnt, thr);
          if constexpr (MODE == kModeTopKShared)
            chunk_topk_shared<RS>(vb, gsf + 32, fsf + 32, crow, colbase + 32, p.k, lv, li, thr);
          if constexpr (MODE == kModeMu)
            chunk_mu<RS>(vb, gsf + 32, fsf + 32, crow, colbase + 32, mu_lo, mu_hi, row_ok, r, p);
        }
        // the g slot has been read by this warp
        __syncwarp();
        if (lane == 0) mbar_arrive(&gempty[gs]);
        if constexpr (kSweepLike) {
          // compensated (Kahan) accumulation of the per-tile partial sums
          const float tile =
              (unpack_sum(acc[0]) + unpack_sum(acc[1])) + (unpack_sum(acc[2]) + unpack_sum(acc[3]));
          const float y = tile - comp;
          const float tsum = sum + y;
          comp = (tsum - sum) - y;
          sum = tsum;
        }
        buf ^= 1;
        if (buf == 0) tphase ^= 1u;
        if (++gs == kGSlots) {
          gs = 0;
          gphase ^= 1u;
        }
      }
      if (!ok) break;
      if constexpr (MODE == kModeMu) continue;
      // the two column halves of a row meet (double-buffered by own-tile
      // parity, handed over through bounded mbarrier waits)
      const int pb = tile_iter & 1;
      const uint32_t rphase = (uint32_t)(tile_iter >> 1) & 1u;
      float* rb = rowbuf + pb * kFusedOwnRows;
      if (half == 1) {
        if (!__all_sync(0xffffffffu, mbar_wait(&rowfree[pb], rphase ^ 1u, abort_flag))) {
          ok = false;
          break;
        }
        if constexpr (kSweepLike) rb[rloc] = sum - comp;
        if constexpr (MODE == kModeSweepWide) wide_shift[pb * kFusedOwnRows + rloc] = wide_m;
        if constexpr (MODE == kModeTopK) {
          if (row_ok)
            for (int i = 0; i < p.k; ++i) {
              p.hand_v[r * p.k + i] = i < tcnt ? tv[i] : -INFINITY;
              p.hand_i[r * p.k + i] = i < tcnt ? ti[i] : 0x7fffffff;
            }
        }
        if constexpr (MODE == kModeTopKShared) {
          if (row_ok)
            for (int i = 0; i < p.k; ++i) {
              p.hand_v[r * p.k + i] = lds_f32(lv + (uint32_t)(i * kEpiThreads) * 4u);
              p.hand_i[r * p.k + i] = lds_s32(li + (uint32_t)(i * kEpiThreads) * 4u);
            }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&rowfull[pb]);
        continue;
      }
      if (!__all_sync(0xffffffffu, mbar_wait(&rowfull[pb], rphase, abort_flag))) {
        ok = false;
        break;
      }
      if constexpr (MODE == kModeTopK) {
        if (row_ok) {
          // merge the two sorted halves: higher score first, lower index on ties
          const double base = shift + p.ell[p.row0 + r];
          int a = 0, b = 0;
          for (int i = 0; i < p.k; ++i) {
            const float bv = p.hand_v[r * p.k + b];
            const int32_t bi = p.hand_i[r * p.k + b];
            const bool take_a = a < tcnt && (b >= p.k || tv[a] > bv || (tv[a] == bv && ti[a] < bi));
            const float sv = take_a ? tv[a] : bv;
            p.idx[r * p.k + i] = take_a ? ti[a] : bi;
            if (p.logmu != nullptr) p.logmu[r * p.k + i] = (float)((double)sv * 0.69314718055994530942 + base);
            if (take_a) ++a; else ++b;
          }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&rowfree[pb]);
      }
      if constexpr (MODE == kModeTopKShared) {
        if (row_ok) {
          // merge the two sorted halves (both exactly k entries, padded with
          // (-inf, INT32_MAX)): higher score first, lower index on ties
          const double base = shift + p.ell[p.row0 + r];
          int a = 0, b = 0;
          for (int i = 0; i < p.k; ++i) {
            const float av = lds_f32(lv + (uint32_t)(a * kEpiThreads) * 4u);
            const int32_t ai = lds_s32(li + (uint32_t)(a * kEpiThreads) * 4u);
            const float bv = p.hand_v[r * p.k + b];
            const int32_t bi = p.hand_i[r * p.k + b];
            const bool take_a = av > bv || (av == bv && ai < bi);
            const float sv = take_a ? av : bv;
            p.idx[r * p.k + i] = take_a ? ai : bi;
            if (p.logmu != nullptr) p.logmu[r * p.k + i] = (float)((double)sv * 0.69314718055994530942 + base);
            if (take_a) ++a; else ++b;
          }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&rowfree[pb]);
      }
      if constexpr (kSweepLike) {
        float other = rb[rloc];
        float row_m = 0.0f;  // wide markets: the shift of the row's sum (log2 units)
        if constexpr (MODE == kModeSweepWide) {
          // the two halves' sums onto the larger of their shifts (exact powers of two)
          const float other_m = wide_shift[pb * kFusedOwnRows + rloc];
          row_m = fmaxf(wide_m, other_m);
          const float own_scale = exp2_int(wide_m - row_m);
          sum *= own_scale;
          comp *= own_scale;
          other *= exp2_int(other_m - row_m);
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&rowfree[pb]);
        const int64_t row = p.row0 + r;
        // the row's sum as three FP32 parts (a split: summed over its ranges)
        float s_hi = sum, s_lo = -comp, s_o = other;
        if constexpr (SPLIT) {
          {
            // this range's partial; the warp that completes the (tile, 32-row
            // block) sums all ranges in order and updates the rows (no wait:
            // the other warps of this block move on)
            const int64_t blk = (int64_t)t * (kFusedOwnRows / 32) + (h * 128 + q * 32) / 32;
            if (row_ok) p.part[(int64_t)split_s * p.rows + r] = make_float4(sum, -comp, other, 0.0f);
            __threadfence();
            __syncwarp();
            int prev = 0;
            if (lane == 0) prev = atomicAdd(p.split_cnt + blk, 1);
            prev = __shfl_sync(0xffffffffu, prev, 0);
            if (prev != p.split - 1) continue;
            if (lane == 0) p.split_cnt[blk] = 0;  // ready for the next launch
            __threadfence();
            s_hi = s_lo = s_o = 0.0f;
            if (row_ok)
              for (int qs = 0; qs < p.split; ++qs) {
                const float4 v = __ldcg(p.part + (int64_t)qs * p.rows + r);
                float e1, e2, e3;
                s_hi = two_sum(s_hi, v.x, e1);
                s_hi = two_sum(s_hi, v.y, e2);
                s_hi = two_sum(s_hi, v.z, e3);
                s_lo = __fadd_rn(s_lo, __fadd_rn(e1, __fadd_rn(e2, e3)));
              }
          }
        }
        double lu_new = 0.0, ell_new = 0.0;
        if (row_ok) {
          const float* b2s = BATCH ? bd->b2s : p.b2s;
          double* log_u = BATCH ? bd->log_u : p.log_u;
          double* ell = BATCH ? bd->ell : p.ell;
          const double omega = BATCH ? ((bd->omega != nullptr && p.update) ? *bd->omega : 1.0) : omega0;
          const double own_off = BATCH ? bd->st[kStOwnOff] : own_off0;
          double ln_sum = log_row_sum(s_hi, s_lo, s_o);
          // wide markets: the row's shift comes back into the sum's logarithm
          if constexpr (MODE == kModeSweepWide) ln_sum = __fma_rn((double)row_m, 0.69314718055994530942, ln_sum);
          const RowResult rr = row_update(ln_sum, shift, b2s ? b2s[row] : 0.0f,
                                          (BATCH ? bd->mass : p.mass)[row], log_u[row] + own_off,
                                          p.residual, omega);
          if (p.update) {
            log_u[row] = rr.log_u;
            ell[row] = rr.ell;
          }
          lu_new = rr.log_u;
          ell_new = rr.ell;
          r_max = fmax(r_max, rr.r_rel);
          r_sum += rr.r_abs;
          sq += rr.u2;
          if (!isfinite(rr.log_u) || !isfinite(rr.ell)) nf += 1.0;
        }
        // this warp's 32 rows form one group of the own side (the finalize
        // reduces the groups into the side's shift and sum of u^2)
        float4* grp = BATCH ? bd->grp : p.grp;
        const int64_t g = (int64_t)t * (kOwn / kGroupRows) + (h * 128 + q * 32) / kGroupRows;
        if (p.update && grp != nullptr && !(SMALL && h == 1) &&
            g * kGroupRows < (BATCH ? bd->rows : p.rows)) {
          const float4 gv = warp_group(lu_new, ell_new, row_ok);
          if (lane == 0) grp[g] = gv;
        }
        if constexpr (BATCH) {
          // partials of this own tile and warp (warps ew = 0..7 own the row
          // updates); the batched finalize sums them per market in a fixed order
          for (int o = 16; o > 0; o >>= 1) {
            r_max = fmax(r_max, __shfl_xor_sync(0xffffffffu, r_max, o));
            r_sum += __shfl_xor_sync(0xffffffffu, r_sum, o);
            sq += __shfl_xor_sync(0xffffffffu, sq, o);
            nf += __shfl_xor_sync(0xffffffffu, nf, o);
          }
          if (lane == 0) {
            double* dst = p.partials + ((int64_t)(bd->slot0 + t) * kBatchSlotWarps + ew) * 4;
            dst[0] = r_max;
            dst[1] = r_sum;
            dst[2] = sq;
            dst[3] = nf;
          }
          r_max = r_sum = sq = nf = 0.0;
        }
      }
    }
    if (!ok && !*abort_flag) raise_error(p.err, abort_flag, kErrTimeout);
    if constexpr (kSweepLike && !BATCH) {
      // reduce the CTA's partials over the epilogue threads
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

// Tensor map over packed rows x kp factors (bf16, or e4m3 bytes when fp8);
// the box is one 128-byte swizzle row wide.
cudaError_t make_map(CUtensorMap* map, const void* base, int64_t rows, int64_t kp, int box_rows, bool fp8 = false) {
  EncodeTiledFn enc = get_encode_fn();
  if (enc == nullptr) return cudaErrorNotSupported;
  const size_t esz = fp8 ? 1 : sizeof(__nv_bfloat16);
  const cuuint64_t dims[2] = {(cuuint64_t)kp, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)kp * esz};
  const cuuint32_t box[2] = {(cuuint32_t)(128 / esz), (cuuint32_t)box_rows};
  const cuuint32_t estr[2] = {1, 1};
  const CUresult r = enc(map, fp8 ? CU_TENSOR_MAP_DATA_TYPE_UINT8 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2,
                         const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                         CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

constexpr int kSmemLimit = 232448;  // dynamic shared memory per CTA (227 KB)

// Partner stages per instantiation: as many as fit beside the own tile(s), the
// g (and scale) rings, the tail and (kModeTopKShared) the ranked lists, at
// most 6 whole tiles (one k block per row), 4 (two) or 5 single k blocks
// (four: 1.25 partner tiles in flight).
constexpr int stages_for(int KB, int MODE, int fmt, bool fold) {
  const int fixed = smem_bytes(KB, fmt, 0, fold) + mode_extra_bytes(MODE);
  const int fit = (kSmemLimit - fixed) / stage_bytes(KB, fold);
  const int cap = KB == 1 ? 6 : (KB == 2 ? 4 : 5);
  return fit < cap ? fit : cap;
}

template <int KB, int MODE, int FMT, bool FOLD>
constexpr int kStages = stages_for(KB, MODE, FMT, FOLD);

template <int KB, int MODE, int FMT, bool FOLD>
constexpr int kSmemTotal =
    smem_bytes(KB, FMT, kStages<KB, MODE, FMT, FOLD>, FOLD) + mode_extra_bytes(MODE);

// Instantiations that exist: batched launches take one or two k blocks
// (e4m3: one); the shared-memory ranked lists leave too little room for
// partner stages beside a four-block own tile (those lists use kModeTopK).
// SPLIT: the partner-split instantiation (single-market half-sweeps with
// tu_market_set_split > 1); the default kernel carries none of its code.
// NOFOLD: the BF16 half-sweep with g from the shared ring instead of the
// extra MMA, for callers without the folded operand (the allocation-free
// entry point).
template <int KB, int MODE, bool BATCH, int FMT, bool SPLIT = false, bool SMALL = false, bool NOFOLD = false>
constexpr bool kBuilt = !(BATCH && (KB == 4 || (FMT != kFmtBF16 && KB != 1))) &&
                        !(MODE == kModeTopKShared && KB == 4) && !(SPLIT && (MODE != kModeSweep || BATCH)) &&
                        !(NOFOLD && (!fold_for(KB, MODE, BATCH, FMT, false) || SPLIT || SMALL));

template <int KB, int MODE, bool BATCH, int FMT = kFmtBF16, bool SMALL = false, bool SPLIT = false,
          bool NOFOLD = false>
cudaError_t launch_kernel(const CUtensorMap& own, const CUtensorMap& partner, const FusedParams& p, int grid,
                          cudaStream_t stream) {
  if constexpr (!kBuilt<KB, MODE, BATCH, FMT, SPLIT, SMALL, NOFOLD>) {
    return cudaErrorNotSupported;
  } else {
    constexpr bool FD = fold_for(KB, MODE, BATCH, FMT, NOFOLD);
    static_assert(kStages<KB, MODE, FMT, FD> >= 2, "at least two partner stages");
    static_assert(kSmemTotal<KB, MODE, FMT, FD> <= kSmemLimit, "shared memory budget");
    if (FD && !BATCH && p.gfold == nullptr) return cudaErrorInvalidValue;  // the folded operand must be prepared
    k_fused_halfsweep<KB, kStages<KB, MODE, FMT, FD>, MODE, BATCH, FMT, SMALL, SPLIT, NOFOLD>
        <<<grid, kThreads, kSmemTotal<KB, MODE, FMT, FD>, stream>>>(own, partner, p);
    return cudaGetLastError();
  }
}

template <int KB, int MODE, bool BATCH, int FMT, bool SMALL, bool SPLIT = false, bool NOFOLD = false>
cudaError_t set_attribute_one() {
  if constexpr (!kBuilt<KB, MODE, BATCH, FMT, SPLIT, SMALL, NOFOLD>) {
    return cudaSuccess;
  } else {
    constexpr bool FD = fold_for(KB, MODE, BATCH, FMT, NOFOLD);
    return cudaFuncSetAttribute(
        k_fused_halfsweep<KB, kStages<KB, MODE, FMT, FD>, MODE, BATCH, FMT, SMALL, SPLIT, NOFOLD>,
        cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemTotal<KB, MODE, FMT, FD>);
  }
}

template <int MODE, bool BATCH, bool SMALL, int FMT, bool SPLIT = false>
cudaError_t set_attributes_fmt() {
  cudaError_t e = set_attribute_one<1, MODE, BATCH, FMT, SMALL, SPLIT>();
  if (e == cudaSuccess) e = set_attribute_one<2, MODE, BATCH, FMT, SMALL, SPLIT>();
  if (e == cudaSuccess) e = set_attribute_one<4, MODE, BATCH, FMT, SMALL, SPLIT>();
  return e;
}

template <int MODE, bool BATCH, bool SMALL, bool SPLIT = false>
cudaError_t set_attributes_variant() {
  cudaError_t e = set_attributes_fmt<MODE, BATCH, SMALL, kFmtBF16, SPLIT>();
  if (e == cudaSuccess) e = set_attributes_fmt<MODE, BATCH, SMALL, kFmtE4M3Side, SPLIT>();
  if (e == cudaSuccess) e = set_attributes_fmt<MODE, BATCH, SMALL, kFmtE4M3Rows, SPLIT>();
  return e;
}

template <int MODE, bool BATCH>
cudaError_t set_attributes_mode() {
  cudaError_t e = set_attributes_variant<MODE, BATCH, false>();
  if (e == cudaSuccess && !BATCH) e = set_attributes_variant<MODE, false, true>();
  if (MODE == kModeSweep && !BATCH) {
    if (e == cudaSuccess) e = set_attributes_variant<MODE, false, false, true>();
    if (e == cudaSuccess) e = set_attributes_variant<MODE, false, true, true>();
  }
  return e;
}

// Dynamic shared memory opt-in of every instantiation, on the current device.
cudaError_t set_kernel_attributes_now() {
  cudaError_t e = set_attributes_mode<kModeSweep, false>();
  if (e == cudaSuccess) e = set_attributes_mode<kModeTopK, false>();
  if (e == cudaSuccess) e = set_attributes_mode<kModeMu, false>();
  if (e == cudaSuccess) e = set_attributes_mode<kModeTopKShared, false>();
  if (e == cudaSuccess) e = set_attributes_mode<kModeSweep, true>();
  if (e == cudaSuccess) e = set_attributes_mode<kModeSweepWide, false>();
  // the allocation-free entry point's unfolded half-sweep (rows of one k block)
  if (e == cudaSuccess) e = set_attribute_one<1, kModeSweep, false, kFmtBF16, false, false, true>();
  return e;
}

// The opt-in is a property of each function in the device's context: made
// once per device (about 130 instantiations, a driver call each), not per
// market, so that creating markets stays cheap for a loop that creates many.
cudaError_t set_kernel_attributes() {
  static std::mutex mu;
  static bool done[64] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return set_kernel_attributes_now();
  std::lock_guard<std::mutex> lk(mu);
  if (done[dev]) return cudaSuccess;
  e = set_kernel_attributes_now();
  if (e == cudaSuccess) done[dev] = true;
  return e;
}

// 128-byte k blocks of a packed row: kp elements of 2 bytes (BF16) or 1 (e4m3).
int k_blocks(int64_t kp, int fmt) { return (int)(fmt != kFmtBF16 ? kp / 128 : kp / kKBlock); }

// The operand format of a market's dtype.
int fmt_of(int dtype) {
  return dtype == TU_DTYPE_FP8E4M3 ? kFmtE4M3Rows : (dtype == TU_DTYPE_FP8E4M3_SIDE ? kFmtE4M3Side : kFmtBF16);
}

template <int MODE, bool BATCH, bool SMALL, int FMT, bool SPLIT>
cudaError_t launch_fmt(int kb, const CUtensorMap& own, const CUtensorMap& partner, const FusedParams& p, int grid,
                       cudaStream_t stream) {
  if (kb == 1) return launch_kernel<1, MODE, BATCH, FMT, SMALL, SPLIT>(own, partner, p, grid, stream);
  if (kb == 2) return launch_kernel<2, MODE, BATCH, FMT, SMALL, SPLIT>(own, partner, p, grid, stream);
  if (kb == 4) return launch_kernel<4, MODE, BATCH, FMT, SMALL, SPLIT>(own, partner, p, grid, stream);
  return cudaErrorNotSupported;
}

template <int MODE, bool BATCH = false, bool SMALL = false, bool SPLIT = false>
cudaError_t launch_variant(int64_t kp, int fmt, const CUtensorMap& own, const CUtensorMap& partner,
                           const FusedParams& p, int grid, cudaStream_t stream) {
  const int kb = k_blocks(kp, fmt);
  if (fmt == kFmtE4M3Rows)
    return launch_fmt<MODE, BATCH, SMALL, kFmtE4M3Rows, SPLIT>(kb, own, partner, p, grid, stream);
  if (fmt == kFmtE4M3Side)
    return launch_fmt<MODE, BATCH, SMALL, kFmtE4M3Side, SPLIT>(kb, own, partner, p, grid, stream);
  return launch_fmt<MODE, BATCH, SMALL, kFmtBF16, SPLIT>(kb, own, partner, p, grid, stream);
}

// small: 128-row own tiles (single-market launches only; see use_small_tiles)
template <int MODE, bool BATCH = false>
cudaError_t launch_any(int64_t kp, int fmt, const CUtensorMap& own, const CUtensorMap& partner,
                       const FusedParams& p, int grid, cudaStream_t stream, bool small = false) {
  if constexpr (!BATCH && MODE == kModeSweep) {
    if (p.split > 1) {
      if (small) return launch_variant<MODE, false, true, true>(kp, fmt, own, partner, p, grid, stream);
      return launch_variant<MODE, false, false, true>(kp, fmt, own, partner, p, grid, stream);
    }
  }
  if constexpr (!BATCH) {
    if (small) return launch_variant<MODE, false, true>(kp, fmt, own, partner, p, grid, stream);
  }
  return launch_variant<MODE, BATCH, false>(kp, fmt, own, partner, p, grid, stream);
}

// 128-row own tiles when they all fit one wave (and the market allows them):
// a CTA with one MMA chain ends its tile in about 0.73 of the time of a
// 256-row tile (measured at 1e4 x 1e4), so the small tiles win only while
// SMs would otherwise stay idle; on a GPU already full (other markets' work
// on other streams) they lose a third of the per-SM throughput.
bool use_small_tiles(const tu_market* m, int64_t rows) {
  if (m->small_mode == 0) return false;
  if (m->small_mode == 2) return true;
  const int64_t t256 = (rows + kFusedOwnRows - 1) / kFusedOwnRows;
  const int64_t t128 = (rows + kFusedOwnRows / 2 - 1) / (kFusedOwnRows / 2);
  return t256 < m->num_sms && t128 <= m->num_sms;
}

FusedParams base_params(int64_t rows, int64_t row0, int64_t col0, int64_t ncols, float c, bool small = false) {
  FusedParams p{};
  const int own_rows = small ? kFusedOwnRows / 2 : kFusedOwnRows;
  p.rows = rows;
  p.row0 = row0;
  p.col0 = col0;
  p.ncols = ncols;
  p.num_own_tiles = (int)((rows + own_rows - 1) / own_rows);
  p.num_partner_tiles = (int)((ncols + kFusedPartnerRows - 1) / kFusedPartnerRows);
  p.c = c;
  p.split = 1;
  return p;
}

int grid_for_tiles(int tiles, int num_sms) {
  int grid = tiles < num_sms ? tiles : num_sms;
  if (grid > kMaxPartials) grid = kMaxPartials;
  return grid < 1 ? 1 : grid;
}

}  // namespace

cudaError_t fused_prepare(tu_market* m) {
  const bool f8 = is_fp8(m->dtype);
  const void* x = f8 ? (const void*)m->X.fac8 : (const void*)m->X.fac16;
  const void* y = f8 ? (const void*)m->Y.fac8 : (const void*)m->Y.fac16;
  cudaError_t e;
  if ((e = make_map(&m->X.tm_own, x, m->X.rows, m->kp, kFusedOwnRows, f8)) != cudaSuccess) return e;
  if ((e = make_map(&m->X.tm_partner, x, m->X.rows, m->kp, kFusedPartnerRows, f8)) != cudaSuccess) return e;
  if ((e = make_map(&m->Y.tm_own, y, m->Y.rows, m->kp, kFusedOwnRows, f8)) != cudaSuccess) return e;
  if ((e = make_map(&m->Y.tm_partner, y, m->Y.rows, m->kp, kFusedPartnerRows, f8)) != cudaSuccess) return e;
  return set_kernel_attributes();
}

cudaError_t launch_fused_halfsweep(tu_market* m, int side, int residual, int update, int* nparts_out,
                                   int64_t row0, int64_t nrows) {
  Side& own = side == 0 ? m->X : m->Y;
  Side& partner = side == 0 ? m->Y : m->X;
  const bool whole = nrows < 0;
  if (whole) {
    row0 = 0;
    nrows = own.rows;
  }
  const bool small = use_small_tiles(m, nrows);
  FusedParams p = base_params(nrows, row0, 0, partner.rows, m->cmul, small);
  p.g = partner.pvec;
  p.lmax = m->st + kStShift;
  p.own_off = m->st + kStOwnOff;
  p.grp = whole ? own.grp : nullptr;  // a range of rows does not write the side's groups
  p.b2s = own.b2s;
  p.mass = own.mass;
  p.log_u = own.log_u;
  p.ell = own.ell;
  p.partials = m->partials;
  p.err = m->err_dev;
  p.residual = residual;
  p.update = update;
  p.omega = m->omega_dev;
  p.fs_own = own.fs;
  p.fs_par = partner.fs;
  p.gfold = partner.fold;
  {
    // partner matrices larger than L2: keep a fixed 70 % of L2's worth resident
    const double pbytes = (double)partner.rows * (double)m->kp * (is_fp8(m->dtype) ? 1.0 : 2.0);
    const double keep = 0.7 * (double)m->l2_bytes;
    p.l2_keep = (m->l2_bytes > 0 && pbytes > keep) ? (float)(keep / pbytes) : 0.0f;
  }
  if (whole && !m->wide && m->split > 1 && m->split_part != nullptr) {
    // partner split: at most one range per partner tile
    p.split = m->split < p.num_partner_tiles ? m->split : p.num_partner_tiles;
    p.range_major = m->split_blocks ? 1 : 0;
    p.part = m->split_part;
    p.split_cnt = m->split_cnt;
  }
  const int grid = grid_for_tiles(p.num_own_tiles * p.split, m->num_sms);
  *nparts_out = grid;
  const int fmt = fmt_of(m->dtype);
  if (m->wide) return launch_any<kModeSweepWide>(m->kp, fmt, own.tm_own, partner.tm_partner, p, grid, m->stream, small);
  return launch_any<kModeSweep>(m->kp, fmt, own.tm_own, partner.tm_partner, p, grid, m->stream, small);
}

// Ranked lists of own users [row0, row0 + nrows) over all partners (the
// partner vector must have been prepared in log2 mode). hand_v / hand_i:
// nrows x k scratch.
cudaError_t launch_fused_topk(tu_market* m, int side, int k, int64_t row0, int64_t nrows, int32_t* idx,
                              float* logmu, float* hand_v, int32_t* hand_i) {
  Side& own = side == 0 ? m->X : m->Y;
  Side& partner = side == 0 ? m->Y : m->X;
  const bool small = use_small_tiles(m, nrows);
  FusedParams p = base_params(nrows, row0, 0, partner.rows, m->cmul, small);
  p.g = partner.pvec;
  p.lmax = m->st + kStShift;
  p.ell = own.ell;
  p.partials = m->partials;
  p.err = m->err_dev;
  p.k = k;
  p.idx = idx;
  p.logmu = logmu;
  p.hand_v = hand_v;
  p.hand_i = hand_i;
  p.fs_own = own.fs;
  p.fs_par = partner.fs;
  const int grid = grid_for_tiles(p.num_own_tiles, m->num_sms);
  const int fmt = fmt_of(m->dtype);
  if (k <= kSharedTopK && k_blocks(m->kp, fmt) < 4)
    return launch_any<kModeTopKShared>(m->kp, fmt, own.tm_own, partner.tm_partner, p, grid, m->stream, small);
  return launch_any<kModeTopK>(m->kp, fmt, own.tm_own, partner.tm_partner, p, grid, m->stream, small);
}

// mu for own X users [x0, x0 + nx) and partners [y0, y0 + ny) (the Y partner
// vector must have been prepared in log2 mode).
cudaError_t launch_fused_mu(tu_market* m, int64_t x0, int64_t nx, int64_t y0, int64_t ny, float* out, int64_t ld) {
  const int64_t c0 = y0 & ~(int64_t)3;  // the g bulk copies start 16-byte aligned
  const bool small = use_small_tiles(m, nx);
  FusedParams p = base_params(nx, x0, c0, y0 + ny - c0, m->cmul, small);
  p.g = m->Y.pvec;
  p.lmax = m->st + kStShift;
  p.ell = m->X.ell;
  p.partials = m->partials;
  p.err = m->err_dev;
  p.out = out;
  p.ld = ld;
  p.y0 = y0;
  p.ny = ny;
  p.fs_own = m->X.fs;
  p.fs_par = m->Y.fs;
  return launch_any<kModeMu>(m->kp, fmt_of(m->dtype), m->X.tm_own, m->Y.tm_partner, p,
                             grid_for_tiles(p.num_own_tiles, m->num_sms), m->stream, small);
}

// Same kernel on caller-described buffers (no market object): used by the
// allocation-free entry point. Tensor maps are built on the host stack.
cudaError_t launch_fused_halfsweep_raw(const FusedRaw& r, cudaStream_t stream, int num_sms, int* nparts_out) {
  CUtensorMap own_map, partner_map;
  cudaError_t e;
  if ((e = make_map(&own_map, r.own16, r.rows, r.kp, kFusedOwnRows)) != cudaSuccess) return e;
  if ((e = make_map(&partner_map, r.par16, r.cols, r.kp, kFusedPartnerRows)) != cudaSuccess) return e;
  if ((e = set_kernel_attributes()) != cudaSuccess) return e;
  FusedParams p = base_params(r.rows, 0, 0, r.cols, (float)(1.4426950408889634 / (2.0 * r.sigma)));
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
  const int grid = grid_for_tiles(p.num_own_tiles, num_sms);
  *nparts_out = grid;
  // (no folded operand here: the instantiation with g from the shared ring)
  if (r.kp == kKBlock) return launch_kernel<1, kModeSweep, false, kFmtBF16, false, false, true>(own_map, partner_map, p,
                                                                                              grid, stream);
  return launch_any<kModeSweep>(r.kp, kFmtBF16, own_map, partner_map, p, grid, stream);
}

// One half-sweep over the items of many markets (batched launch). The
// per-market tensor maps live in the descriptors, so the kernel's map
// parameters are unused.
cudaError_t launch_fused_batch(const BatchLaunch& b, cudaStream_t stream) {
  static_assert(kEpiWarps / 2 == kBatchSlotWarps, "per-tile partial slots");
  // (the shared-memory opt-in was made when the member markets were prepared)
  FusedParams p{};
  p.bdesc = b.desc;
  p.items = b.items;
  p.cta_start = b.cta_start;
  p.partials = b.partials;
  p.err = b.err;
  p.residual = b.residual;
  p.update = b.update;
  CUtensorMap unused;
  memset(&unused, 0, sizeof(unused));
  return launch_any<kModeSweep, true>(b.kp, fmt_of(b.dtype), unused, unused, p, b.grid, stream);
}

}  // namespace tu
