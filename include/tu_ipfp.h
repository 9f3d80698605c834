/*
 * tu_ipfp.h -- C ABI of the GB300 IPFP library (libtu_ipfp.so).
 *
 * Solves the Choo-Siow transferable-utility matching model of
 * "Parallel and Mini-Batch Stable Matching for Large-Scale Reciprocal
 * Recommender Systems" (arXiv 2411.19214) with the IPFP / Sinkhorn sweep.
 *
 * Model (Sec. 3.1-3.3). Side X has N users (candidates, index x, capacity n_x),
 * side Y has M users (employers, index y, capacity m_y). Each user carries two
 * d-dimensional factor vectors: f_x, k_x (rows of F, K) and g_y, l_y (rows of
 * G, L). The joint surplus is phi_xy = <f_x, g_y> + <k_x, l_y> + b^X_x + b^Y_y,
 * where the optional popularity biases b are an extension the paper does not
 * have (unit coefficient, kept in FP32 outside the tensor-core product).
 * With A = exp(Phi / (2 sigma)) (sigma is the paper's beta) and the scaling
 * vectors u_x = sqrt(mu_x0), v_y = sqrt(mu_0y), one sweep is (Eq. iteration):
 *     u_x <- sqrt(n_x + s_x^2) - s_x,  s_x = 1/2 sum_y A_xy v_y
 *     v_y <- sqrt(m_y + s_y^2) - s_y,  s_y = 1/2 sum_x A_xy u_x   (new u)
 * and the equilibrium is mu_xy = A_xy u_x v_y (Eq. stable_condition).
 * The library keeps log u and log v (FP64) and evaluates the update in the
 * algebraically identical form log u = 1/2 log n - asinh(s / sqrt(n)).
 *
 * Two paths compute the same iteration:
 *   TU_PATH_FUSED  mini-batch IPFP (Alg. 2 / Eq. iteration_minibatch): Phi is
 *                  formed tile by tile from BF16 (or e4m3) factors on the
 *                  tensor cores and never stored; requires d <= 128 (e4m3:
 *                  256).
 *   TU_PATH_DENSE  batch IPFP (Alg. 1 / Eq. iteration_matrix): the FP32 kernel
 *                  A-hat = exp((Phi - b^X - b^Y) / (2 sigma)) is materialised
 *                  once, with its transpose (2*N*M*4 bytes), and one of the
 *                  two is streamed every half-sweep.
 *
 * Conventions shared by every entry point:
 *   - Return codes only; nothing is thrown across the ABI.
 *   - Pointers marked "host or device" may point to host memory (pageable or
 *     pinned) or to device memory of the market's device; the library detects
 *     which and copies as needed. All device work is ordered on the market's
 *     stream. Calls that return host values synchronise that stream.
 *   - After TU_ERR_CUDA the market is poisoned: every later call returns
 *     TU_ERR_CUDA and only tu_market_destroy is valid.
 *   - A market is not thread-safe: one host thread at a time per market.
 */
#ifndef TU_IPFP_H
#define TU_IPFP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct tu_market* tu_market_t;

typedef enum {
  TU_OK = 0,
  TU_ERR_INVALID_ARG = 1,   /* a size, pointer or value is out of range */
  TU_ERR_OOM = 2,           /* device memory allocation failed */
  TU_ERR_CUDA = 3,          /* a CUDA call failed; the market is poisoned */
  TU_ERR_NOT_CONVERGED = 4, /* tu_ipfp_solve hit max_iter; potentials are still valid */
  TU_ERR_NONFINITE = 5,     /* an input or a computed potential is NaN or infinite */
  TU_ERR_TIMEOUT = 6,       /* a device-side wait ran out of its time limit */
  TU_ERR_UNSUPPORTED = 7    /* valid request outside what the library supports (e.g. d > 128 on the fused path) */
} tu_status;

enum { TU_DTYPE_BF16 = 0, TU_DTYPE_FP32 = 1, TU_DTYPE_FP8E4M3 = 2, TU_DTYPE_FP8E4M3_SIDE = 3 };
enum { TU_PATH_FUSED = 0, TU_PATH_DENSE = 1 };

typedef struct {
  int64_t N;             /* users on side X, >= 1 */
  int64_t M;             /* users on side Y, >= 1 */
  int64_t d;             /* factor dimension D of Sec. 3.3, >= 1 (fused path: <= 128, FP8 <= 256) */
  int32_t dtype;         /* element type of F, K, G, L: TU_DTYPE_BF16 (uint16 bit patterns) or TU_DTYPE_FP32.
                            The fused path computes with BF16 (FP32 inputs are rounded to nearest even);
                            the dense path computes with FP32 (BF16 inputs are widened exactly).
                            TU_DTYPE_FP8E4M3 (fused path only, d <= 256): the market computes with
                            e4m3 factors (OCP FP8: 4 exponent bits, bias 7, 3 mantissa bits, largest
                            finite 448) and one FP32 scale per row on the FP8 tensor cores. Without
                            fscale_x / fscale_y, F, K, G, L are FP32 and the library quantizes: row
                            x of [F | K] (resp. y of [G | L]) is scaled by 2^-k_x, k_x the smallest
                            integer with max |entry| <= 448 * 2^k_x, and rounded to nearest even
                            (saturating), with scale 2^k_x. The MMA multiplies e4m3 values exactly
                            (FP32 accumulation) and the product of rows x and y is scaled by
                            scale_x * scale_y in FP32. This is a lower-precision model of phi (about
                            3 % per entry), not the BF16 one.
                            TU_DTYPE_FP8E4M3_SIDE: the same from FP32 factors with one power-of-two
                            scale per side (k the smallest integer with max |entry| of the side <=
                            448 * 2^k), folded into the exponent multiplier: the faster FP8 mode
                            (the per-row scales cost one multiply and one shared load per pair;
                            with one scale per side and d <= 64 the partner potentials also ride
                            in the MMA), for sides whose rows have similar norms (small rows lose
                            precision to e4m3 subnormals). */
  int32_t path;          /* TU_PATH_FUSED or TU_PATH_DENSE */
  const void* F;         /* N x d row-major, host or device; copied (the market owns its copy) */
  const void* K;         /* N x d row-major, host or device; copied */
  const void* G;         /* M x d row-major, host or device; copied */
  const void* L;         /* M x d row-major, host or device; copied */
  const float* bias_x;   /* N FP32 popularity biases b^X (host or device), or NULL for none */
  const float* bias_y;   /* M FP32 popularity biases b^Y (host or device), or NULL for none */
  const double* n;       /* N capacities n_x > 0, HOST memory */
  const double* m;       /* M capacities m_y > 0, HOST memory */
  double sigma;          /* entropy scale beta of Eq. primary optimization, > 0 */
  int64_t partition;     /* rows per mini-batch of Alg. 2 (0: whole side). Results do not depend on it:
                            within a half-sweep every u_x depends only on the fixed v. */
  void* stream;          /* cudaStream_t for all work of this market (NULL: the legacy default stream) */
  const float* fscale_x; /* FP8 only, or NULL: per-row scales of X (N FP32, host or device). With them
                            F and K are the caller's e4m3 bytes (N x d each), row x of [F | K] standing
                            for fscale_x[x] times its e4m3 values. Both scales or neither. */
  const float* fscale_y; /* likewise for G and L (M scales) */
} tu_market_desc;

/* Create a market from factor matrices and capacities (Sec. 3.3, Alg. 2 inputs).
 * Potentials start at u = v = 1 (Alg. 1 / Alg. 2 initialisation).
 * Validates sizes, pointers, sigma > 0, capacities > 0 and finite. The
 * exponent range, bound = max_x |a_x| * max_y |b_y| / (2 sigma) with
 * a_x = (f_x, k_x), b_y = (g_y, l_y) (a Cauchy-Schwarz bound on the bias-free
 * part of phi / (2 sigma)), decides the arithmetic: up to 40, one shift per
 * half-sweep keeps every FP32 term in range; beyond ("wide" markets, strong
 * preferences or small sigma), the fused path keeps a running maximum of
 * every row's exponents and rescales the row's sum by an exact power of two
 * whenever it grows (one pass over the pairs, 1.2 to 1.3 times the time of
 * a narrow half-sweep), and the dense path refuses the market
 * (TU_ERR_UNSUPPORTED: its materialised FP32 A-hat would overflow). In wide
 * markets the FP32 accumulation of phi carries an absolute error of about
 * bound x 2^-24 x sqrt(2d) per exponent, above the 1e-7 of narrow ones, and
 * the attainable residual is about bound x 2^-24 (the FP32 spacing of the
 * large exponents and partner potentials that dominate a row). Biases
 * have no limit: they are folded into the potentials in log space. Sizes: 1 <= N, M <= 2^31
 * and 1 <= d <= 4096 (TU_ERR_INVALID_ARG otherwise); the fused path takes
 * d <= 128 (BF16; the MMA inner dimension 2d is padded to 64, 128 or 256, so
 * 64 < d <= 128 costs as much as d = 128) and FP8 d <= 256 (2d padded to 128,
 * 256 or 512), FP8 factors only on the fused path, a dense market at most 200 GB of A-hat and its transpose, and a
 * device of compute capability 10.3 (the library is built for sm_103a only)
 * (TU_ERR_UNSUPPORTED otherwise). On success *out owns device memory of about
 * (N + M) * 2 * d * 2 bytes (fused) or 2 * N * M * 4 bytes (dense), a staging
 * buffer for factor uploads of 2 * max(N, M) * d * (2 for BF16, else 4) bytes,
 * and O(N + M); tu_market_footprint gives the total. */
tu_status tu_market_create(const tu_market_desc* desc, tu_market_t* out);

/* Replace F, K, G, L (same shapes and dtype as at creation; host or device).
 * Potentials are kept, so the next solve can be warm-started. Dense markets
 * rebuild A-hat. The same checks as tu_market_create apply (TU_ERR_NONFINITE,
 * TU_ERR_UNSUPPORTED); after such a refusal the market's factors are
 * undefined until the next successful update (its potentials are kept). A
 * market created with FP8 caller scales takes tu_market_update_factors_fp8
 * instead (TU_ERR_INVALID_ARG here). */
tu_status tu_market_update_factors(tu_market_t mkt, const void* F, const void* K, const void* G,
                                   const void* L);

/* The same for a market created with fscale_x / fscale_y: new e4m3 bytes
 * F, K (N x d), G, L (M x d) and their per-row scales (host or device).
 * TU_ERR_INVALID_ARG for any other market; TU_ERR_NONFINITE for a non-finite
 * scale. */
tu_status tu_market_update_factors_fp8(tu_market_t mkt, const void* F, const void* K, const void* G,
                                       const void* L, const float* fscale_x, const float* fscale_y);

/* Run nsweeps >= 0 full sweeps of Eq. iteration (u from v, then v from the new u;
 * Alg. 1 loop body / Alg. 2 loop body), each half-sweep preceded by the
 * translation step unless tu_market_set_translation(mkt, 0) turned it off
 * (that step leaves the fixed point unchanged). If residual_out != NULL, synchronise and
 * store the row residual of the resulting potentials:
 *     max_x |u_x^2 + u_x sum_y A_xy v_y - n_x| / n_x     (row equations of Eq. IPFP,
 * terms and reduction in FP64), which costs one extra half-sweep of work. */
tu_status tu_ipfp_sweep(tu_market_t mkt, int nsweeps, double* residual_out);

typedef struct {
  int32_t sweeps;        /* sweeps run by this call */
  int32_t status;        /* the tu_status returned */
  double residual_inf;   /* max_x |r_x| / n_x of the returned potentials (Eq. IPFP rows) */
  double residual_l1;    /* sum_x |r_x| / sum_x n_x of the returned potentials */
  double match_count;    /* sum_xy mu_xy = sum_y m_y - sum_y v_y^2 (FP64 reduction) */
} tu_solve_info;

/* Sweep until residual_inf <= tol or max_iter sweeps (Alg. 1 with a stopping
 * rule; the paper runs a fixed count). warm_start = 0 resets to u = v = 1 first;
 * 1 continues from the current potentials. An estimate of the residual of each
 * sweep's input state (FP32 terms, FP64 reduction) is reduced inside the X
 * half-sweep and decides when to stop; the returned state is certified by one
 * final residual pass with FP64 terms. Returns TU_OK, TU_ERR_NOT_CONVERGED
 * (potentials valid), or an error. info may be NULL. */
tu_status tu_ipfp_solve(tu_market_t mkt, double tol, int max_iter, int warm_start, tu_solve_info* info);

/* mu_xy = exp(phi_xy / (2 sigma) + log u_x + log v_y) (Eq. stable_condition,
 * Alg. 1 final line) for x in [x0, x0 + nx), y in [y0, y0 + ny), written FP32
 * row-major to out (host or device) with leading dimension ld >= ny. */
tu_status tu_mu_block(tu_market_t mkt, int64_t x0, int64_t nx, int64_t y0, int64_t ny, float* out,
                      int64_t ld);

/* Ranked recommendation lists (Sec. 4.1 ranks a list per user; Sec. 3.3 scores
 * by log mu). side 0: for each x in [row0, row0 + nrows), the k partners y with
 * the largest mu_xy; side 1: for each y, the k partners x. Ties are broken by
 * the lower partner index. idx (int32) and log_mu (FP32, may be NULL) are
 * nrows x k row-major, host or device, best first. 1 <= k <= 64 and
 * k <= partner count. */
tu_status tu_topk_partners(tu_market_t mkt, int side, int k, int64_t row0, int64_t nrows, int32_t* idx,
                           float* log_mu);

/* Sweep until the recommendation lists stop changing (the early-stopping
 * criterion the paper proposes for practical use, Sec. 4.2 discussion: stop
 * when the rankings of candidates and employers stay stable for a number of
 * epochs). Every `check_every` sweeps the k best partners by log mu (the
 * ranked lists of tu_topk_partners) of the first min(sample, N) X users and
 * the first min(sample, M) Y users are recomputed, with the next partner's
 * score. A check passes when every list position whose log mu is more than
 * score_eps above the next entry's and below the previous entry's holds the
 * same partner as at the previous check (near-ties are not compared: at the
 * fixed point their order flips with the last bits of the potentials). The
 * call returns TU_OK after `patience` consecutive passing checks and
 * TU_ERR_NOT_CONVERGED after max_iter sweeps. warm_start and the relaxation
 * setting apply as in tu_ipfp_solve. info (may be NULL): sweeps run, status,
 * the certified residual of the returned state (rankings settle long before
 * the marginals) and the match count. Requires 1 <= k <= 63, k <= min(N, M),
 * sample >= 1, check_every >= 1, patience >= 1, score_eps >= 0, max_iter >= 0
 * (else TU_ERR_INVALID_ARG). */
tu_status tu_ipfp_solve_ranking(tu_market_t mkt, int k, int64_t sample, int check_every, int patience,
                                double score_eps, int max_iter, int warm_start, tu_solve_info* info);

/* Checkpoint / restore the solver state (the scaling vectors of Alg. 2's
 * output, Psi and Xi's last columns): log u (N floats) and log v (M floats),
 * host or device. Either pointer may be NULL to skip that side. */
tu_status tu_get_potentials(tu_market_t mkt, float* log_u, float* log_v);
tu_status tu_set_potentials(tu_market_t mkt, const float* log_u, const float* log_v);

/* The same state in full precision: log u (N doubles) and log v (M doubles),
 * host or device, either pointer NULL to skip that side. The FP32 copies above
 * round log u to about 6e-8 |log u|, which moves u by up to a few 1e-6 for the
 * potentials of popular users (|log u| ~ 40): enough to lift a converged
 * state's residual above a 1e-6 tolerance. A checkpoint taken and restored
 * with these calls resumes a solve exactly. The get call synchronises the
 * market's stream. */
tu_status tu_get_potentials_f64(tu_market_t mkt, double* log_u, double* log_v);
tu_status tu_set_potentials_f64(tu_market_t mkt, const double* log_u, const double* log_v);

/* One shard of a market split across GPUs (Sec. 3.3: within a half-sweep each
 * user's update depends only on the other side's fixed potentials, so the
 * users of a side can be split into contiguous shards, one per GPU, each
 * GPU holding every factor). side 0 updates X users [lo, hi) from the
 * market's current log v (the u step of Eq. iteration), side 1 updates Y users
 * [lo, hi) from the current log u (the v step); the other users of that side
 * keep their potentials. No translation step is taken (it needs both sides'
 * sums over all shards: the caller computes it from the gathered potentials
 * and writes them back with tu_set_potentials_f64); after the pass the
 * market's kept shifts and sums are recomputed from the stored potentials
 * (an O(N + M) pass), so any call may follow. residual_out (host, 2
 * doubles, may be NULL): max |r| / mass and sum |r| over the shard's users of
 * the equations of Eq. IPFP for that side (rows for side 0, columns for side
 * 1) at the entering state, FP64 terms; the MAX and SUM over shards give the
 * market's. Requires the fused path (TU_ERR_UNSUPPORTED otherwise) and
 * 0 <= lo <= hi <= users of the side (TU_ERR_INVALID_ARG otherwise).
 * Synchronises the market's stream. */
tu_status tu_ipfp_half_sweep_range(tu_market_t mkt, int side, int64_t lo, int64_t hi, double* residual_out);

/* FP64 log potentials of users [lo, hi) of one side (side 0: log u, 1: log v)
 * into out (hi - lo doubles, host or device), e.g. a shard's share of an
 * all-gather. Synchronises the market's stream. */
tu_status tu_get_potentials_range_f64(tu_market_t mkt, int side, int64_t lo, int64_t hi, double* out);

/* Over-relaxation of the log-domain update, an acceleration the paper does not
 * have (its Sec. 5 names acceleration as future work): log u <- log u +
 * omega * (update - log u), and the same for v. A fixed point of the relaxed
 * sweep is a fixed point of Eq. iteration, so the solution is unchanged.
 *   omega = 1 (default)  Alg. 1 exactly;
 *   1 < omega < 2        tu_ipfp_sweep applies it from the next sweep on;
 *                        tu_ipfp_solve applies it once the residual is below 0.1;
 *   omega = 0            automatic: tu_ipfp_solve runs plain sweeps until the
 *                        per-sweep decay q of the residual has settled, then uses
 *                        omega = 2 / (1 + sqrt(1 - q)) (successive over-relaxation),
 *                        lowered linearly towards 1 over the last decade of the
 *                        residual above tol (a relaxed sweep amplifies the FP32
 *                        rounding of the row sums by about omega / (2 - omega));
 * a fixed omega is applied as set, down to tol;
 * in both relaxed modes tu_ipfp_solve halves omega - 1 whenever the residual
 * grows tenfold over the best seen. Other values: TU_ERR_INVALID_ARG. */
tu_status tu_market_set_relaxation(tu_market_t mkt, double omega);

/* The relaxation controller of tu_ipfp_solve on a given residual trace, for
 * tests and tuning (no counterpart in the paper; no CUDA call, no market).
 * A fresh controller with setting `omega` (0 or [1, 2), as
 * tu_market_set_relaxation) observes, in order, the residual residual[i] read
 * after done[i] sweeps (done strictly increasing, >= 1) against `tol`, and
 * omega_out[i] receives the factor it sets for the sweeps that follow.
 * Invalid settings, tol < 0, count < 0, NULL arrays with count > 0 or a
 * non-increasing done: TU_ERR_INVALID_ARG. */
tu_status tu_relax_schedule(double omega, double tol, const int* done, const double* residual, int count,
                            double* omega_out);

/* Translation step, an acceleration the paper does not have (its Sec. 5 names
 * acceleration techniques from optimal transport as future work). IPFP solves
 * the row equations of Eq. IPFP exactly, then the column equations: block
 * coordinate ascent on the concave dual
 *     D(a, b) = sum n a + sum m b - 1/2 sum e^{2a} - 1/2 sum e^{2b} - sum_xy A_xy e^{a_x + b_y}
 * (a = log u, b = log v), whose gradient is Eq. IPFP. With enable = 1 (the
 * default) every half-sweep of a sweep is preceded by the exact maximisation
 * of D along one more direction: the side updated last moves by +tau in log
 * space and the side about to be updated by -tau. That move leaves every
 * mu_xy = A_xy u_x v_y unchanged, so tau has a closed form from sum u^2,
 * sum v^2, sum n and sum m (O(N + M) work, no pair work): tau = 1/2 log z, z the
 * positive root of P z^2 - (sum mass_P - sum mass_O) z - O = 0 with P, O the
 * sums of squared potentials of the two sides. Every step raises D, so the
 * iteration reaches the fixed point of Eq. iteration; on balanced markets,
 * whose slow mode is exactly this move (plain IPFP needs O(N) sweeps there),
 * it needs a handful of sweeps instead. enable = 0: Eq. iteration exactly.
 * The certifying pass of tu_ipfp_sweep's residual_out and of the solves
 * never moves the state. Other values: TU_ERR_INVALID_ARG. */
tu_status tu_market_set_translation(tu_market_t mkt, int enable);

/* Blocks of k > 1 sweeps replay a captured CUDA graph on the market's stream
 * (enable = 1, the default), or are launched kernel by kernel (0). Capturing
 * is not safe while another host thread uses the library: a capture in
 * progress makes some of that thread's calls (host copies, allocation) fail
 * and invalidates the capture, so callers that drive markets from several
 * threads turn graphs off. No counterpart in the paper. */
tu_status tu_market_use_graphs(tu_market_t mkt, int enable);

/* Launch shape of the fused half-sweep (no counterpart in the paper; results
 * are the same fixed point whatever the shape).
 * Own-tile height, mode = 0: 256-row own tiles; 1 (the default): 128-row
 * tiles when a market's 256-row tiles would leave SMs idle while its 128-row
 * tiles all fit one wave (twice the CTAs, each ending its tile sooner: an
 * isolated 1e4 x 1e4 sweep 0.171 -> 0.132 ms); 2: always 128-row tiles. A
 * 128-row tile delivers about two thirds of a 256-row tile's per-SM
 * throughput, so callers that keep the GPU full with many markets at once (a
 * serving loop) set 0. Results are bit-identical across modes (every row's
 * arithmetic is the same). Dense markets ignore it. TU_ERR_INVALID_ARG for
 * another mode. */
tu_status tu_market_set_small_tiles(tu_market_t mkt, int mode);

/* Partner split, 1 <= split <= 8 (fused markets; TU_ERR_UNSUPPORTED on the
 * dense path): each own tile's partner tiles are cut into `split` contiguous
 * ranges handled by different CTAs, and the CTA that completes a tile's
 * block of rows sums the ranges' partial row sums in range order and updates
 * the rows, so a market with few waves of own tiles fills the GPU in finer
 * steps (1e5 users: 391 tiles of 256 rows are 2.6 waves on 148 SMs, in
 * thirds 7.9). The sums are the same terms in another order (results agree
 * to rounding, not bit for bit with split = 1). Allocates split x max(N, M)
 * x 16 bytes of partial sums on first use. Applies to whole-side sweeps of
 * markets within the single-shift range (see tu_market_create). */
tu_status tu_market_set_split(tu_market_t mkt, int split);

/* Partner blocks, 1 <= blocks <= 8 (fused markets; TU_ERR_UNSUPPORTED on the
 * dense path): the same partial sums as a split into `blocks` ranges, but
 * with the items ordered range by range, so that all CTAs stream one block of
 * the partner matrix against every own tile before the next block, aiming to
 * read a block small enough for L2 from memory about once per half-sweep
 * instead of once per wave of own tiles (the partner matrix of a 1e6 x 1e6,
 * d = 64 market is 256 MB, L2 129 MB). Measured there with 3 blocks: DRAM
 * reads fell only to 7.8 GB per half-sweep and the half-sweep took 7 % longer
 * (each block restarts every own tile's pipeline), so the autotuner times
 * blocks as one candidate among others. Replaces any split. */
tu_status tu_market_set_partner_blocks(tu_market_t mkt, int blocks);

/* The market's launch shape: own-tile mode and partner split, a negative
 * split -b for b partner blocks (either pointer may be NULL). */
tu_status tu_market_get_shape(tu_market_t mkt, int* small_mode, int* split);

/* Autotuner of the launch shape: times the candidate (own-tile height,
 * partner split) pairs on this market, reps non-updating sweeps each after
 * one untimed sweep (the potentials are not changed), keeps the fastest for
 * the market and records it in a process-wide cache keyed by the market's
 * shape (quarter-octave buckets of N and M, the packed row length, the FP8
 * dtype or BF16, the SM count); fused markets created later with a cached
 * shape take the tuned launch shape. Candidates: the default shape, 256-row
 * tiles, 128-row tiles (fewer than 4 waves of 256-row tiles), splits 2, 3,
 * 4, 6, 8 (fewer than 8 waves) and partner blocks 2, 3, 4, 6 (partner
 * matrices above 96 MB, at least 2 waves); splits and blocks not for wide
 * markets. Synchronises.
 * TU_ERR_UNSUPPORTED on the dense path, TU_ERR_INVALID_ARG unless
 * 1 <= reps <= 1000. */
typedef struct {
  int small_tiles;    /* chosen own-tile mode (as tu_market_set_small_tiles) */
  int split;          /* chosen partner split (negative: -b partner blocks) */
  double ms;          /* ms per sweep of the chosen shape */
  double ms_default;  /* ms per sweep of the default shape (mode 1, split 1) */
  int candidates;     /* shapes timed */
} tu_tune_info;
tu_status tu_market_autotune(tu_market_t mkt, int reps, tu_tune_info* info);

/* The autotuner's cache as a JSON file (one entry per line; load merges the
 * file's entries, which replace cached ones with the same key). Save or load
 * of a path that cannot be opened, or load of a malformed file:
 * TU_ERR_INVALID_ARG (nothing is merged). */
tu_status tu_autotune_cache_save(const char* path);
tu_status tu_autotune_cache_load(const char* path);
void tu_autotune_cache_clear(void);

/* Automatic over-relaxation for asynchronous sweeps (no counterpart in the
 * paper). For a market whose relaxation setting is 0 (automatic), feed the
 * residual of the last completed tu_ipfp_sweep block (the value
 * tu_market_query reports) into the controller tu_ipfp_solve uses, and set the
 * factor the next sweeps apply: plain sweeps until the decay rate has settled,
 * then successive over-relaxation tapered towards 1 in the last decade above
 * tol. Non-blocking: does nothing while the last block is still running, for
 * other settings, or when the block was already fed. The controller restarts
 * when the factors, potentials or setting change and after tu_ipfp_solve.
 * tol < 0: TU_ERR_INVALID_ARG. */
tu_status tu_market_relax_update(tu_market_t mkt, double tol);

/* Non-blocking progress query for serving loops that keep many markets busy
 * from one host thread (no counterpart in the paper). tu_ipfp_sweep without
 * residual_out only enqueues work; this call checks, without waiting, whether
 * that work has finished. *idle = 1 when every sweep enqueued so far is done;
 * then *residual = max_x |r_x| / n_x of the state that entered the last sweep
 * (row equations of Eq. IPFP, reduced in FP64 inside that sweep's X
 * half-sweep from terms formed in FP32: an estimate within about 2e-7),
 * *match_count = sum m - sum v^2 after it, and *sweeps = sweeps
 * completed since creation. After a call that certifies its result
 * (tu_ipfp_sweep with residual_out, tu_ipfp_solve, tu_ipfp_solve_ranking),
 * *residual is that certified residual of the returned state. While busy
 * (*idle = 0) the other outputs are not written. Any output pointer may be
 * NULL. */
tu_status tu_market_query(tu_market_t mkt, int* idle, double* residual, double* match_count, int64_t* sweeps);

/* Device memory a market of this shape holds (bytes), for admission control:
 * the packed factors, the per-user state and the dense matrices if any, for
 * BF16 or FP32 factors in the default launch shape. A partner split
 * (tu_market_set_split, or a tuned shape a new market takes from the
 * autotuner's cache) adds split x max(N, M) x 16 bytes; e4m3 markets hold
 * 1-byte factors and 4 to 36 more bytes per user (scales, folded g). */
int64_t tu_market_footprint(int64_t N, int64_t M, int64_t d, int path);

/* Kernel timing for benchmarks (no counterpart in the paper). While enabled,
 * every half-sweep pass records a CUDA event pair on the market's stream
 * around its main kernel (fused: the tcgen05 half-sweep; dense: the row pass,
 * or the two column-pass kernels), and sweeps are launched directly instead of
 * through a captured graph. tu_profile_read synchronises the stream, returns
 * the summed elapsed milliseconds and the number of timed passes since the
 * last read (either pointer may be NULL), and starts a new count. */
tu_status tu_profile_enable(tu_market_t mkt, int enable);
tu_status tu_profile_read(tu_market_t mkt, double* pass_ms, int64_t* passes);

/* One fused X half-sweep on caller buffers that allocates no device memory.
 * The paper has no counterpart: this entry point exists for callers that cannot
 * call cudaMalloc, such as a serving process whose device memory is fully
 * budgeted by an admission controller or held by another allocator (a
 * framework's caching allocator), or a latency-critical loop where cudaMalloc /
 * cudaFree would synchronise the device. It computes what the u step of a
 * market sweep computes (Eq. iteration_minibatch, first line): for every own
 * user r,
 *     log u_r <- 1/2 log n_r - asinh(s_r / sqrt(n_r)),
 *     s_r = 1/2 sum_c exp((<a_r, b_c> + b^own_r + b^par_c) / (2 sigma)) v_c.
 * All pointers are DEVICE memory of the current device:
 *   own_packed      rows x kp BF16 row-major: [f_r | k_r | zeros], kp = 64 or 128 (>= 2d), 16-byte aligned
 *   partner_packed  cols x kp BF16 row-major: [g_c | l_c | zeros], 16-byte aligned
 *   own_bias        rows FP32 biases b^own, or NULL
 *   own_mass        rows FP64 capacities n_r > 0
 *   own_log_u_in    rows FP32: the log u entering the half-sweep (used only for the residual)
 *   partner_bias    cols FP32 biases b^par, or NULL
 *   partner_log_v   cols FP32 log v of the partners
 *   own_log_u_out   rows FP32: the new log u (may not alias own_log_u_in)
 * residual_out (host, may be NULL): if given, the call synchronises the stream
 * and stores max_r |u_r^2 + 2 u_r s_r - n_r| / n_r of the entering state (row
 * equations of Eq. IPFP), and reports device-side failures: TU_ERR_TIMEOUT (a
 * bounded wait ran out) and TU_ERR_NONFINITE (a computed potential is NaN or
 * infinite). Otherwise the call only enqueues work on `stream` and reports no
 * device-side failure; pass residual_out to have them checked.
 * A pointer of another device, or host memory, gives TU_ERR_INVALID_ARG; a
 * device other than compute capability 10.3 (the library is built for sm_103a
 * only) gives TU_ERR_UNSUPPORTED.
 * Limits: 1 <= rows <= 65536 and 1 <= cols <= 1048576 (TU_ERR_UNSUPPORTED
 * beyond them, and for kp other than 64 or 128); the factors must lie in the
 * single-shift range of tu_market_create (bound <= 40), which is not checked
 * here (there is no running-maximum variant for wide markets).
 * Scratch: one file-scope __device__ array of 5,644,576 bytes that every GPU
 * loading the library holds until the process exits; its device address is
 * resolved on the first call on each device (with that device current), so
 * make that first call before any stream capture. Every call shares the array
 * and it keeps the last call's contents: calls that overlap on the GPU (two
 * streams, two host threads) race and must be serialised by the caller. */
tu_status tu_fused_halfsweep_noalloc(int64_t rows, int64_t cols, int64_t kp, const void* own_packed,
                                     const void* partner_packed, const float* own_bias, const double* own_mass,
                                     const float* own_log_u_in, const float* partner_bias,
                                     const float* partner_log_v, double sigma, float* own_log_u_out,
                                     double* residual_out, void* stream);

/* ---- Many independent markets in one launch per half-sweep ----------------
 * The paper solves one market at a time; a batch sweeps many independent
 * markets together. Each market's arithmetic is exactly that of its own
 * tu_ipfp_sweep (Eq. iteration_minibatch, fused path): after k batched sweeps
 * its potentials are bit-identical to k sweeps of the market alone. Per
 * half-sweep the batch runs one preparation kernel, one persistent tensor-core
 * kernel over the (market, 256-user own tile) items of every active market,
 * scheduled longest-first over the SMs, and one reduction kernel. */
typedef struct tu_batch* tu_batch_t;

/* Group `count` markets (1 <= count <= 65536), all created with TU_PATH_FUSED
 * on the current device with the same packed width (BF16: 2d rounded up to 64
 * or 128; FP8: d <= 64) and the same dtype. The batch references the markets
 * (their buffers, tensor maps, sigma, relaxation and translation settings at
 * creation); destroy the batch before any of them. Wide markets (see
 * tu_market_create) and markets with d > 64 (BF16 with 2d > 128) cannot join
 * a batch (TU_ERR_UNSUPPORTED). A member's factors may be replaced
 * (tu_market_update_factors) between batch calls: the batch follows its new
 * scales (e4m3 with one scale per side), and tu_batch_sweep / tu_batch_solve
 * return TU_ERR_UNSUPPORTED while a member's factors are wide.
 * Batch work is ordered on `stream` (a cudaStream_t, or NULL for the legacy
 * default stream); every batch call first waits for work already enqueued on
 * the members' own streams, and the caller orders later member calls after
 * the batch's (every call below except tu_batch_sweep without residuals
 * returns with `stream` synchronised). Errors: TU_ERR_INVALID_ARG (count,
 * NULL, a dense-path, poisoned or repeated market, mixed widths or devices),
 * TU_ERR_OOM, TU_ERR_CUDA. */
tu_status tu_batch_create(const tu_market_t* markets, int count, void* stream, tu_batch_t* out);

/* nsweeps >= 0 sweeps of Eq. iteration on every market of the batch (each
 * with its fixed relaxation factor if one was set, else plain). residual_out:
 * NULL (enqueue only), or host memory for `count` doubles that receives each
 * market's max_x |r_x| / n_x of the returned state (one extra X pass without
 * update, as tu_ipfp_sweep's residual_out). TU_ERR_NONFINITE if a computed
 * potential of any market is not finite. */
tu_status tu_batch_sweep(tu_batch_t b, int nsweeps, double* residual_out);

/* Solve every market to max_x |r_x| / n_x <= tol, as tu_ipfp_solve does for
 * one (warm_start = 0 resets u = v = 1 first). Markets leave the launch as
 * soon as their residual is certified at or below tol, so the remaining ones
 * share the GPU; automatic relaxation (tu_market_set_relaxation(m, 0)) runs
 * per market. infos: host memory for `count` entries (may be NULL), filled
 * per market (sweeps it received, its status, residuals, match count).
 * Returns TU_OK if every market converged, TU_ERR_NONFINITE if any market
 * produced a non-finite potential, else TU_ERR_NOT_CONVERGED when some market
 * reached max_iter sweeps; potentials of every market stay valid. */
tu_status tu_batch_solve(tu_batch_t b, double tol, int max_iter, int warm_start, tu_solve_info* infos);

/* Kernel timing of the batched half-sweep kernel, as tu_profile_enable /
 * tu_profile_read for a market (events around each batched tensor-core
 * launch; no graph replay while enabled). */
tu_status tu_batch_profile_enable(tu_batch_t b, int enable);
tu_status tu_batch_profile_read(tu_batch_t b, double* pass_ms, int64_t* passes);

/* Free the batch (not its markets; safe on NULL). */
void tu_batch_destroy(tu_batch_t b);

/* Detail of the batch's last error ("" if none). */
const char* tu_batch_last_error(tu_batch_t b);

/* Failure-path diagnostic (no counterpart in the paper). Every wait of the
 * library's kernels is bounded: a wait that runs out sets a device error word,
 * the kernel drains and returns, and the call that launched it reports
 * TU_ERR_TIMEOUT. This entry point runs that bounded wait in a one-CTA kernel
 * on an mbarrier that nothing signals, with a limit of limit_seconds (0 < limit
 * <= 5, else TU_ERR_INVALID_ARG), on the legacy default stream of the current
 * device. Expected result: TU_ERR_TIMEOUT, with the measured wait in
 * *waited_seconds (may be NULL); TU_OK would mean the wait ended without a
 * signal; TU_ERR_CUDA / TU_ERR_OOM report a CUDA failure. The device stays
 * usable. */
tu_status tu_selftest_wait_timeout(double limit_seconds, double* waited_seconds);

/* Checked mode, a substitute for a memory sanitizer (no counterpart in the
 * paper). With enable != 0, markets created afterwards surround every device
 * buffer they own (factors, potentials, vectors, partials, staging and
 * scratch, the dense kernel matrices) with 256-byte guard bands of the byte
 * 0xA5, leaving the buffers themselves and every result unchanged. When such a
 * buffer is freed (tu_market_destroy, or a scratch buffer that grows) the
 * bands are read back: a band that changed means a kernel wrote outside the
 * buffer, and the buffer is counted in tu_guard_violations. Checked mode is
 * also on when the environment variable TU_CHECKED is "1" when the library is
 * loaded. It costs one synchronisation of the market's stream per freed
 * buffer. Batches' own small buffers are not guarded. Always TU_OK. */
tu_status tu_set_checked_mode(int enable);

/* Guard-band violations found since the library was loaded (0 in a correct
 * build). If last != NULL and last_size > 0, a description of the latest
 * violation (NUL-terminated, truncated to last_size) is written there. */
int64_t tu_guard_violations(char* last, int64_t last_size);

/* Free every resource of the market (safe on NULL). */
void tu_market_destroy(tu_market_t mkt);

/* Static description of a status code. */
const char* tu_status_string(tu_status s);

/* Detail of the market's last error ("" if none). Valid until the next call on mkt. */
const char* tu_market_last_error(tu_market_t mkt);

#ifdef __cplusplus
}
#endif

#endif /* TU_IPFP_H */
