/*
 * sfft.h -- C ABI of the B300 TT-SFFT Carr-Madan pricer.
 *
 * Prices European calls on a log-strike grid of M = 2^n points with the
 * Carr-Madan discrete Fourier transform (Sec. 2.1 of Hauck & Turkalj,
 * "Classical Tensor Train and Quantum Fourier Transform Approaches for
 * Large-Scale Carr-Madan Option Pricing"), evaluated as the tensor-train
 * Superfast Fourier Transform of Sec. 3: the integrand x_j (Eq. x, or its
 * Simpson-weighted variant) is held as a quantics tensor train of n binary
 * cores, the bit-reversed Fourier operator Q_n (Sec. 3.2) is applied as a
 * matrix-product operator, the result is rounded by QR/SVD sweeps, and prices
 * are read out in bit-reversed site order (Sec. 3.3, Eq. discretization_dft).
 * No length-M vector is formed on that path. A dense-FFT Carr-Madan baseline
 * (Sec. 4.1's FFT route) is exposed with the same calling convention.
 *
 * Conventions shared by every entry point:
 *   - Every function returns sfft_status; nothing throws across the ABI.
 *   - Pointers marked "device" are CUDA device pointers of the context's
 *     device (for example torch.cuda tensors' data_ptr()); pointers marked
 *     "host" are ordinary host memory. The caller owns every buffer it passes.
 *   - Device work is stream-ordered on the stream set with sfft_set_stream
 *     (default: the legacy default stream). Inside sfft_price_batch the
 *     TT-SVD builder runs on a stream of the context's own, forked from and
 *     joined back to that stream by events, so the call's work as a whole
 *     stays ordered on it. Calls that return per-instance status
 *     synchronise that stream before returning.
 *   - Invalid arguments are rejected on the host before any launch
 *     (SFFT_EINVAL); the text of the last error is sfft_last_error(ctx).
 *   - A context is used by one host thread at a time.
 *   - Complex numbers are stored as interleaved double pairs (re, im).
 *   - A tensor train (TT) crossing the ABI is "packed": core l (1-based) of
 *     shape (r_{l-1}, d, r_l) is stored row-major (last index fastest) at
 *     complex offset sum_{i<l} r_{i-1} d r_i; ranks[0] = ranks[n] = 1.
 *     Site 1 carries the most significant bit of the grid index, as in
 *     Eq. discretized_x: j = sum_l lambda_l 2^(n-l).
 *   - An MPO crossing the ABI is a packed TT with d = 4 whose physical index
 *     is 2*mu + lambda (mu = output bit, lambda = input bit of Eq. tto_format).
 */
#ifndef SFFT_H
#define SFFT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  SFFT_OK = 0,
  SFFT_EINVAL = 1,   /* invalid argument (shape, range, NaN, unsupported mode) */
  SFFT_EMOMENT = 2,  /* E[S_T^(alpha+1)] is infinite: Eq. damping_moment_condition fails */
  SFFT_ENOMEM = 3,   /* device or host allocation failed */
  SFFT_ECUDA = 4,    /* a CUDA runtime call failed (text in sfft_last_error) */
  SFFT_ERANK = 5,    /* a TT or MPO rank would exceed the cap */
  SFFT_ENOCONV = 6,  /* integrand builder did not reach the tolerance */
  SFFT_ETIMEOUT = 7, /* a bounded device-side wait expired */
  SFFT_EBOUNDS = 8   /* a price left the no-arbitrage bounds by more than
                        1e-6 S0 max(1, e^{-alpha k}) (k the log-moneyness):
                        the discrete sum does not resolve the damped integrand
                        (near a moment explosion at this alpha); prices are
                        still written, for inspection */
} sfft_status;

/* Characteristic-function models of log(S_T/S0). Sec. 2 gives Black-Scholes
 * and names Heston, Merton and Variance-Gamma; parameter slots p[]:
 *   SFFT_GBM    p = {sigma}
 *   SFFT_HESTON p = {kappa, theta, sigma_v, rho, v0}  (Heston 1993, "little
 *                   trap" form of Albrecher et al. 2007)
 *   SFFT_MERTON p = {sigma, lambda, mu_J, delta_J}     (Merton 1976)
 *   SFFT_VG     p = {sigma, nu, theta}                 (Madan-Carr-Chang 1998) */
typedef enum { SFFT_GBM = 0, SFFT_HESTON = 1, SFFT_MERTON = 2, SFFT_VG = 3 } sfft_model;

/* Quadrature of the Fourier integral (Eq. C_k_integral):
 *   SFFT_QUAD_SIMPSON_CM99: v_j = eta j, Simpson weights (1/3, 4/3, 2/3, ...),
 *     strikes k'_u = -pi/eta + 2 pi u/(M eta) -- the "higher-order quadrature
 *     weights incorporated into x_j" that the paper allows after
 *     Eq. discretization_dft.
 *   SFFT_QUAD_RECT_SYM: the paper's symmetric rectangle rule, Eqs.
 *     Ck_from_psi, x, discretization_dft; Delta_v = eta, or pi/sqrt(N) when
 *     eta <= 0 (the grid of Sec. 4), Delta_k = pi/(N Delta_v),
 *     k'_0 = -N Delta_k/2. */
typedef enum { SFFT_QUAD_SIMPSON_CM99 = 0, SFFT_QUAD_RECT_SYM = 1 } sfft_quad;

typedef struct {
  int32_t model;    /* sfft_model */
  int32_t quad;     /* sfft_quad */
  int32_t n;        /* grid exponent, M = 2^n, 1 <= n <= SFFT_MAX_N */
  int32_t max_rank; /* cap on the ranks of the integrand TT and of the rounded
                       output TT (a builder or rounding step that needs more
                       sets SFFT_ERANK); 0 -> SFFT_DEFAULT_MAX_RANK. The
                       intermediate ranks of the zip-up contraction, which the
                       rounding then lowers, are bounded only by the core-slot
                       capacity SFFT_MAX_RANK */
  double p[8];      /* model parameters, see sfft_model */
  double S0;        /* spot, > 0 */
  double r;         /* risk-free rate */
  double T;         /* maturity, > 0 */
  double alpha;     /* damping of Eq. damping_moment_condition; alpha < -1 prices puts */
  double eta;       /* frequency step (see sfft_quad) */
  double tol;       /* relative Frobenius truncation tolerance of the TT steps */
  double k0;        /* must be NaN (default grid start); reserved */
} sfft_problem;

/* Per-instance diagnostics. Build and core times are not kept per instance:
 * a batch's instances run concurrently, so the per-phase device times of a
 * whole call (integrand build, zip-up, rounding, readout, ...) come from the
 * profiling API (sfft_profile_enable / sfft_profile_read) instead. */
typedef struct {
  int32_t status;    /* sfft_status of this instance */
  int32_t int_rank;  /* max rank of the integrand TT */
  int32_t mpo_rank;  /* max rank of the Q_n MPO */
  int32_t out_rank;  /* max rank of the rounded output TT */
  int64_t tt_bytes;  /* bytes of the output TT cores (complex128) */
} sfft_info;

#define SFFT_MAX_N 48
#define SFFT_DEFAULT_MAX_RANK 32
#define SFFT_MAX_RANK 32
#define SFFT_MAX_MPO_RANK 32
#define SFFT_MAX_STRIKES 65536

typedef struct sfft_ctx sfft_ctx;

/* Create a context on CUDA device `device` (owns the MPO cache and device
 * workspaces). Returns SFFT_ECUDA if the device cannot be used. */
sfft_status sfft_create(sfft_ctx **ctx, int device);

/* Release the context and all device memory it owns (host call; synchronises
 * the context's stream first). NULL is accepted. */
sfft_status sfft_destroy(sfft_ctx *ctx);

/* Make all later device work of this context run on `cuda_stream`
 * (a cudaStream_t; NULL = legacy default stream). */
sfft_status sfft_set_stream(sfft_ctx *ctx, void *cuda_stream);

/* Arithmetic of the MPO x TT contraction of this context's pricing calls
 * (sfft_price_batch, captured batches):
 *   SFFT_PRECISION_FP64  (default) every step in FP64 on the CUDA cores;
 *   SFFT_PRECISION_MIXED the zip-up's MPO contraction of each site (Sec. 3.2,
 *     Eq. complexity_TTO), the complex product of the carried partial result
 *     with the operator core, runs on the fifth-generation tensor cores in
 *     complex FP32: one real GEMM in the 4M form [Re X | Im X] against
 *     [[Re W, Im W], [-Im W, Re W]], each FP32 operand split into three
 *     bfloat16 pieces (the six products of combined order <= 2, FP32
 *     accumulation), so its inputs keep FP32 precision.
 *     The QR and SVD steps, the carry contraction and the readout stay FP64.
 *     Sites whose panel exceeds one 128-row tile, and the instances the
 *     first-tier zip-up hands to its second tier, run in FP64. The prices
 *     then differ from the FP64 path by roughly the FP32 rounding of the
 *     contraction (checked to 1e-6 S0 at tolerance 1e-7). */
#define SFFT_PRECISION_FP64 0
#define SFFT_PRECISION_MIXED 1
sfft_status sfft_set_precision(sfft_ctx *ctx, int32_t precision);

/* ---- tuning of the first-tier launches ----
 * The first tier of the two-tier kernels runs several CTAs per SM on a small
 * shared-memory carve; how small pays depends on the batch. A tuning is the
 * carve of three of them: the TT-SVD builder's panel width (build_p <= 32
 * columns), the output rounding's rank (round_r <= 24) and the zip-up's CTAs
 * per SM (zip_ctas, 0 = as many as fit). The defaults are 32, 24 and 0.
 * sfft_autotune times the batch under the defaults and, by coordinate
 * descent, under zip_ctas 2, build_p 24 and 16, round_r 20 and 16 (each
 * configuration the best of `reps` calls, CUDA events on the context's
 * stream, the outputs written like sfft_price_batch), and caches the fastest
 * under the batch's signature; later pricing calls of this context (and
 * graphs created from it) with the same signature use it. The signature is
 * the device (compute capability, SM count) and the batch's size and its
 * distribution over grid exponents, models, tolerance decade and grid rule,
 * each count quantised to its binary order of magnitude (sfft_tune_key gives
 * the batch part). The cache is exported as text lines "<signature> build_p
 * round_r zip_ctas" and imported back, so that a given cache fixes the choice
 * without re-timing. Under the SFFT_TIER1 test hook tuning is refused
 * (SFFT_EINVAL) and the hook's limits apply. */
typedef struct {
  int32_t build_p;  /* TT-SVD builder, first tier: panel columns (2..32) */
  int32_t round_r;  /* output rounding, first tier: rank (1..24) */
  int32_t zip_ctas; /* zip-up, first tier: CTAs per SM (0 = as many as fit) */
} sfft_tune;
sfft_status sfft_autotune(sfft_ctx *ctx, const sfft_problem *probs, int32_t count, const int64_t *l_begin,
                          const int64_t *stride, const int32_t *q, double *prices, double *log_strikes,
                          int32_t reps, sfft_tune *chosen, double *ms_chosen, double *ms_default);
/* The configuration a batch would use on this context; *found (may be NULL)
 * says whether it came from the cache (else the defaults). Host only. */
sfft_status sfft_tune_lookup(sfft_ctx *ctx, const sfft_problem *probs, int32_t count, sfft_tune *cfg,
                             int32_t *found);
/* The configurations the last sfft_autotune timed, in order, with their
 * times (ms, best of its reps): cfgs and ms hold cap entries, *n receives
 * how many there were. */
sfft_status sfft_tune_trials(const sfft_ctx *ctx, sfft_tune *cfgs, double *ms, int32_t cap, int32_t *n);
/* The batch part of the signature as text (host only, no context). */
sfft_status sfft_tune_key(const sfft_problem *probs, int32_t count, char *buf, int32_t cap);
/* The cache as text into buf (capacity cap, NUL-terminated); *len receives
 * the length (buf may be NULL to ask for it). */
sfft_status sfft_tune_export(const sfft_ctx *ctx, char *buf, int64_t cap, int64_t *len);
/* Adds the lines of `text` to the cache (SFFT_EINVAL on a malformed line,
 * nothing added then). */
sfft_status sfft_tune_import(sfft_ctx *ctx, const char *text);

/* Hand-off counts of the last sfft_price_batch call on this context (host
 * array of 4): how many instances the first-tier launches of the TT-SVD
 * builder, the cross builder, the zip-up and the output rounding passed on to
 * their full-size second tier. A first-tier launch runs several CTAs per SM on
 * a small shared-memory carve; an instance whose panels or ranks outgrow that
 * carve is handed on, before any of its outputs is written, and the second
 * tier prices it from its unmodified inputs. Synchronises the context's
 * stream. Zeros before the first call.
 *
 * Test hooks (environment variables read by sfft_create; host side only,
 * nothing faults or stalls the device):
 *   SFFT_TIER1="build=8,round=6,cross=4,zipq=40,zipw=900" narrows the
 *     first-tier limits (builder panel columns, rounding rank, cross rank,
 *     zip-up panel columns, zip-up panel elements factored in shared memory)
 *     so that hand-offs and the global-memory factorisation paths run;
 *   SFFT_FAULT="enomem:<workspace>[:<times>]" fails that workspace's
 *     allocations with SFFT_ENOMEM; "jacobi:<sweeps>" caps the Jacobi sweeps
 *     of every SVD of a pricing call (non-convergence reports SFFT_ENOCONV);
 *     "enoconv:<position>" makes the builder result of that position among the
 *     call's valid instances SFFT_ENOCONV. Items are separated by ';'. */
sfft_status sfft_tier2_counts(sfft_ctx *ctx, int32_t *counts);

/* Strike selection helper (host only, no device work). For grid indices
 * u in [0, M) with log-moneyness k'_u in [lo_logm, hi_logm], returns the
 * first index l_begin, a power-of-two stride and the count q <= qmax of the
 * set {l_begin + i*stride}; l_begin is a multiple of stride. */
sfft_status sfft_strike_window(const sfft_problem *prob, double lo_logm,
                               double hi_logm, int32_t qmax, int64_t *l_begin,
                               int64_t *stride, int32_t *q);

/* Price `count` instances with the TT-SFFT path (Sec. 3.3).
 *   probs[count]              host  problem statements
 *   l_begin, stride, q        host  per-instance strike sets on the 2^n grid:
 *                                   u = l_begin + i*stride, i < q; stride a
 *                                   power of two, l_begin a multiple of it,
 *                                   u < 2^n, q <= SFFT_MAX_STRIKES
 *   prices, log_strikes       device, sum(q) doubles each, instance i's
 *                                   outputs start at sum_{k<i} q[k]; prices in
 *                                   currency units, log_strikes = log K
 *   inst_status[count]        host  per-instance sfft_status (may be NULL)
 *   info[count]               host  per-instance diagnostics (may be NULL)
 * A failing instance does not stop the batch: its prices are NaN and its
 * status says why; the call then returns the first such status. The MPO of
 * each distinct (n, tol) is built once and cached in the context. */
sfft_status sfft_price_batch(sfft_ctx *ctx, const sfft_problem *probs, int32_t count,
                             const int64_t *l_begin, const int64_t *stride,
                             const int32_t *q, double *prices, double *log_strikes,
                             int32_t *inst_status, sfft_info *info);

/* Same contract, dense-FFT Carr-Madan baseline: samples all M = 2^n integrand
 * values, runs an M-point FFT in device memory and gathers the requested
 * strikes. n <= SFFT_DENSE_MAX_N; needs 32*M bytes of device workspace. */
#define SFFT_DENSE_MAX_N 32
sfft_status sfft_dense_price_batch(sfft_ctx *ctx, const sfft_problem *probs, int32_t count,
                                   const int64_t *l_begin, const int64_t *stride,
                                   const int32_t *q, double *prices, double *log_strikes,
                                   int32_t *inst_status, sfft_info *info);

/* Same contract, the QFT route of Sec. 3 (QFT-based option pricing) by exact
 * statevector emulation: x is normalised to the amplitudes x/||x|| of
 * Eq. qft_input_state, the inverse QFT is applied (the unitary DFT of
 * Eq. dft, as M-point FFT passes in device memory), the measurement
 * probabilities p_l = |y~_l|^2 of Eq. qft_probabilities are formed, and each
 * price is read from sqrt(p_l) under the positive-phase assumption
 * (Eqs. qft_phase_assumption, qft_observable_price) with exact probabilities
 * (no shot noise). Prices therefore equal |.| of the dense route's
 * discretised sum. The phase assumption holds on the symmetric grid only
 * (quad = SFFT_QUAD_RECT_SYM, Eq. x): the one-sided Simpson sum has a genuine
 * imaginary part, so other grids are rejected with SFFT_EINVAL.
 * n <= SFFT_DENSE_MAX_N; 32*M bytes of device workspace. */
sfft_status sfft_qft_price_batch(sfft_ctx *ctx, const sfft_problem *probs, int32_t count,
                                 const int64_t *l_begin, const int64_t *stride,
                                 const int32_t *q, double *prices, double *log_strikes,
                                 int32_t *inst_status, sfft_info *info);

/* ---- captured batches (CUDA graphs) ----
 * The device work of one sfft_price_batch call, recorded as a CUDA graph and
 * replayed: repeated pricing of a batch of fixed shape without host planning
 * or per-kernel launch cost. The shape is every instance's n, tol, quad,
 * max_rank, k0 and strike set; model parameters, S0, r, T, alpha and eta may
 * change between replays through sfft_graph_update. (Sec. 3.2 builds the
 * transform once for reuse across evaluations; this carries the reuse to the
 * whole pricing step.)
 * sfft_graph_create runs the batch once in a private context, whose
 * workspaces, MPO cache and stream belong to the graph alone and never move,
 * then captures the same call; every instance must price, with status
 * SFFT_OK or SFFT_EBOUNDS (else the status of the first failure is returned
 * and *out stays NULL). prices and log_strikes
 * (device, sum(q) doubles each) stay bound to the graph. */
typedef struct sfft_graph sfft_graph;
sfft_status sfft_graph_create(sfft_ctx *ctx, const sfft_problem *probs, int32_t count,
                              const int64_t *l_begin, const int64_t *stride,
                              const int32_t *q, double *prices, double *log_strikes,
                              sfft_graph **out);
/* Enqueue one replay on `stream` (a cudaStream_t; NULL = legacy stream).
 * A replay on a different stream than the previous one first waits for it. */
sfft_status sfft_graph_launch(sfft_graph *g, void *stream);
/* New problem statements (count as at creation; the shape fields must match)
 * for the following replays. Waits for the previous replay to finish. */
sfft_status sfft_graph_update(sfft_graph *g, const sfft_problem *probs);
/* Per-instance status and diagnostics of the last replay (host arrays, may be
 * NULL); waits for it. Returns the first failing status, as sfft_price_batch. */
sfft_status sfft_graph_status(sfft_graph *g, int32_t *inst_status, sfft_info *info);
const char *sfft_graph_last_error(const sfft_graph *g);
sfft_status sfft_graph_destroy(sfft_graph *g);

/* ---- lower-level entry points (one pipeline step each; used by tests) ---- */

/* Integrand samples x_j (Eq. x or the Simpson variant) at `count` grid
 * indices j (device int64) into x (device, count complex). */
sfft_status sfft_sample_integrand(sfft_ctx *ctx, const sfft_problem *prob,
                                  const int64_t *j, int64_t count, double *x);

/* Integrand TT of one problem (Sec. 3.1/4.3: TT-SVD of the sampled support
 * block). ranks (host, n+1) receives the ranks, cores (device) the packed
 * cores; cap = capacity of `cores` in complex elements. */
sfft_status sfft_integrand_tt(sfft_ctx *ctx, const sfft_problem *prob, int32_t *ranks,
                              double *cores, int64_t cap);

/* The MPO of Q_n (Sec. 3.2) compressed to relative Frobenius tolerance tol,
 * copied packed (d = 4) into cores (device, capacity cap complex); ranks
 * (host, n+1). */
sfft_status sfft_mpo(sfft_ctx *ctx, int32_t n, double tol, int32_t *ranks, double *cores,
                     int64_t cap);

/* TT rounding (Oseledets' QR + truncated-SVD sweeps) of a packed TT with
 * physical dimension d in {2, 4}: in_ranks/in_cores in, out_ranks (host)
 * and out_cores (device, capacity cap) out. */
sfft_status sfft_tt_round(sfft_ctx *ctx, int32_t n, int32_t d, const int32_t *in_ranks,
                          const double *in_cores, double tol, int32_t max_rank,
                          int32_t *out_ranks, double *out_cores, int64_t cap);

/* y = Q_n x for a packed TT x (d = 2): zip-up MPO x TT contraction followed
 * by the rounding sweep at tolerance tol. Output TT in bit-reversed site
 * order: site l carries bit l-1 of the output index u. */
sfft_status sfft_tt_apply_qft(sfft_ctx *ctx, int32_t n, const int32_t *in_ranks,
                              const double *in_cores, double tol, int32_t max_rank,
                              int32_t *out_ranks, double *out_cores, int64_t cap);

/* ---- rounding without allocation ----
 * The paper has no counterpart to this entry point; it exists for callers that
 * cannot allocate device memory when they round (a host application whose
 * memory manager owns the device, a latency-critical loop that cannot afford
 * the device-wide synchronisation of cudaMalloc/cudaFree, a plugin that may
 * not create a library context). It runs the same rounding as sfft_tt_round
 * (Oseledets' QR orthogonalisation and truncated-SVD sweep) but keeps all of
 * its scratch in one statically sized device array of
 * SFFT_NOALLOC_SCRATCH_BYTES bytes inside the library, which every GPU that
 * loads the library holds until the process exits. It calls no cudaMalloc,
 * cudaFree or other allocating routine.
 *   n, d                 n <= SFFT_NOALLOC_MAX_N sites, d in {2, 4}
 *   in_ranks, out_ranks  host, n+1 entries each; every rank <= SFFT_MAX_RANK
 *   in_cores, out_cores  device, packed cores (out capacity `cap` complex)
 *   stream               cudaStream_t of the current device (NULL = default)
 *   errbuf, errlen       optional host buffer for a readable error message
 * Sizes beyond the limits are rejected with SFFT_EINVAL and a message in
 * errbuf. The first call on a device (the current one) looks up the array's
 * device address and sets the kernel's shared-memory limit. Every call shares
 * the one array and leaves its contents behind (the status word is cleared at
 * the start of each call), so calls that overlap on the GPU, on any streams or
 * threads, race. The call blocks: it copies ranks and status between host and
 * device and synchronises `stream` twice, so it returns only after the stream
 * has completed its work, and it must not be called while `stream` (or the
 * legacy stream) is being captured into a CUDA graph. When the output capacity
 * is too small, SFFT_EINVAL is returned and out_ranks is left untouched. */
#define SFFT_NOALLOC_MAX_N 48
#define SFFT_NOALLOC_SCRATCH_BYTES 3473920
sfft_status sfft_tt_round_noalloc(int32_t n, int32_t d, const int32_t *in_ranks,
                                  const double *in_cores, double tol, int32_t max_rank,
                                  int32_t *out_ranks, double *out_cores, int64_t cap,
                                  void *stream, char *errbuf, int32_t errlen);

/* ---- tracing ---- */

/* Phases timed by the profiler (index into the arrays of sfft_profile_read):
 * 0 support probe and work lists, 1 integrand TT build, 2 zip-up MPO x TT, 3 rounding,
 * 4 readout, 5 MPO build, 6 dense sampling (the dense route samples inside
 * its first FFT pass, so this phase is that pass), 7 the other dense FFT
 * passes, 8 dense gather, 9 integrand TT by cross interpolation (and its rounding);
 * phase 1 then counts the TT-SVD builder alone. */
#define SFFT_NPHASES 10

/* Turn per-launch CUDA-event timing and in-kernel algorithmic flop counting
 * on (on != 0) or off. Off by default; costs one event pair per launch. */
sfft_status sfft_profile_enable(sfft_ctx *ctx, int32_t on);

/* Read the accumulated per-phase totals since the last reset (host arrays of
 * SFFT_NPHASES entries each, any may be NULL): device milliseconds, launches,
 * algorithmic FP64 flops (complex multiply-add = 8), integrand evaluations
 * (for the zip-up phase: the number of sites whose MPO contraction ran on
 * the tensor cores, see sfft_set_precision).
 * Synchronises the context's stream. reset != 0 clears the totals. */
sfft_status sfft_profile_read(sfft_ctx *ctx, double *ms, double *flops, double *evals,
                              int64_t *launches, int32_t reset);

/* Measured FP64 fused multiply-add throughput of the context's device in
 * GFLOP/s (independent FMA chains over 8 blocks per SM, CUDA-event timed);
 * the denominator of the FP64 roofline of the TT kernels. */
sfft_status sfft_calibrate_fp64(sfft_ctx *ctx, double *gflops);

/* Static strings; never NULL. */
const char *sfft_status_string(sfft_status s);
const char *sfft_last_error(const sfft_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* SFFT_H */
