// Host runtime and C ABI of the TT-SFFT pricer (include/sfft.h): context,
// validation, grid planning (the scalars of Sec. 2.1), the damping-moment
// check (Eq. damping_moment_condition), the Q_n MPO cache and the stream-
// ordered launch sequence of the pricing path.
#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <deque>
#include <map>
#include <string>
#include <utility>
#include <vector>

#include "../../include/sfft.h"
#include "kernels.cuh"

static_assert(SFFT_MAX_N == SFFT_MAXN_DEV, "rank array stride");
static_assert(SFFT_MAX_RANK == SFFT_SLOT_RANK_DEV, "slot rank");

namespace {

const int kThreads = 256;
// First-tier launches of the two-tier kernels: 128-thread CTAs with carves
// for panels of up to kSmallP columns (builder) or ranks up to kSmallRoundR
// (rounding); the batch's integrand ranks stay below 10 and its output ranks
// below 25, so the full-size second tier rarely has work.
const int kThreadsSmall = 128;
const int kSmallP = 32;
const int kSmallRoundR = 24;
// Cross tier 1: ranks up to 16, so supercores of 32 x 32 and the assembly's
// maxvol work (2 N r + 2 r^2 + N = 1568 for N = 32, r = 16) fit W = (32 + 17) x 32.
const int kCrossSmallR = 16;
const int kCrossSmallHb = 17;
const int CROSS_RANK_CAP = SFFT_SLOT_RANK_DEV;
const int kHb = 36;  // row-block height reserved next to the 64-column panel
const int kSvdMaxBits = 14;  // support blocks up to 2^14 points: TT-SVD; wider: cross
const int kCrossSweeps = 6;

struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    bytes = 0;
  }
};

struct MpoEntry {
  int idx;        // slot index in the pool
  int n;
  double tol;
  long long off;  // complex offset in the MPO pool
  std::vector<int> ranks;
  // zip-up of the delta prefix (k_zipup on an all-delta TT): block offset in
  // the prefix pool (-1: not available) and its output ranks
  long long zoff = -1;
  std::vector<int> zranks;
};

}  // namespace

struct sfft_ctx {
  int device = 0;
  int num_sms = 0;
  cudaStream_t stream = nullptr;
  // the TT-SVD builder runs here, forked from and joined back to `stream`
  cudaStream_t side = nullptr;
  cudaEvent_t fork = nullptr, join = nullptr;
  std::string err;
  // MPO cache (pool of fixed-size slots)
  DevBuf mpo_pool;
  DevBuf mpo_ranks_dev;  // (SFFT_MAX_N+1) per cached MPO
  int mpo_slots = 0;
  DevBuf zpre_pool;       // SFFT_ZPRE_BLOCK complex per MPO slot
  DevBuf zpre_ranks_dev;  // (SFFT_MAX_N+1) per MPO slot
  std::deque<MpoEntry> mpos;  // stable addresses across push_back
  // batch workspaces (grow only)
  std::map<std::string, DevBuf> bufs;
  // profiling: CUDA events around every launch, per phase
  bool prof = false;
  double* prof_acc = nullptr;  // device: flops[NPHASE], evals[NPHASE]
  std::vector<cudaEvent_t> ev_pool;
  std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> ev_open;
  double prof_ms[SFFT_NPHASE_DEV] = {0};
  long long prof_launches[SFFT_NPHASE_DEV] = {0};
  // tier-1 limits of the two-tier launches (defaults: the carves' own
  // limits; the SFFT_TIER1 test hook narrows them to force hand-offs)
  struct Tier1 {
    int build_p = 32;    // TT-SVD builder: panel columns (2 r)
    int round_r = 24;    // output rounding: rank
    int cross_r = 16;    // cross builder: rank
    int zip_q = LA_MAXQ; // zip-up: panel columns (s' r')
    int zip_w = 1 << 30; // zip-up: panel elements factored in shared memory
    int zip_ctas = 0;    // zip-up: CTAs per SM (0: as many as fit)
  } t1;
  bool t1_hooked = false;  // SFFT_TIER1 set: its limits win over any tuning
  bool zpre_on = true;     // zip-up of the delta prefix taken from the MPO cache
  // tuned first-tier configurations by batch signature (sfft_autotune), the
  // one in force for the current call, and a forced one while tuning
  std::map<std::string, Tier1> tune;
  Tier1 cur;
  bool forcing = false;
  Tier1 force;
  std::vector<std::pair<Tier1, double>> trials;  // the last tuning's configurations and times
  // arithmetic of the zip-up's MPO contraction (SFFT_PRECISION_*)
  int precision = SFFT_PRECISION_FP64;
  // fault-injection test hooks (SFFT_FAULT), all on the host side
  std::string fault_enomem;    // workspace whose allocations fail
  int fault_enomem_left = 0;   // how many more times (< 0: always)
  int fault_jacobi = 0;        // > 0: Jacobi sweep limit during pricing calls
  int fault_enoconv = -1;      // >= 0: that batch position reports SFFT_ENOCONV
  // hand-off counts of the last TT pricing call's two-tier launches (device)
  int* defer_heads[4] = {nullptr, nullptr, nullptr, nullptr};
  // while a graph is being captured: host data of every upload is first
  // copied into this pinned arena (a captured copy must read pinned memory
  // that outlives the capture)
  struct Stage {
    char* base = nullptr;
    size_t cap = 0, used = 0;
    size_t p_off = 0, p_bytes = 0;  // where the instance parameters went
    bool overflow = false;
  }* stage = nullptr;
};

namespace {

sfft_status set_err(sfft_ctx* ctx, sfft_status s, const char* fmt, ...) {
  if (ctx) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    ctx->err = buf;
  }
  return s;
}

#define CK(call)                                                                          \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess)                                                                \
      return set_err(ctx, e_ == cudaErrorMemoryAllocation ? SFFT_ENOMEM : SFFT_ECUDA,     \
                     "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__,    \
                     __LINE__);                                                           \
  } while (0)

sfft_status ensure(sfft_ctx* ctx, const char* name, size_t bytes, void** out) {
  DevBuf& b = ctx->bufs[name];
  if (ctx->fault_enomem_left != 0 && ctx->fault_enomem == name) {
    if (ctx->fault_enomem_left > 0) --ctx->fault_enomem_left;
    return set_err(ctx, SFFT_ENOMEM, "allocation of %s (%zu bytes) failed: injected by SFFT_FAULT", name, bytes);
  }
  if (b.bytes < bytes) {
    if (b.p) {
      cudaError_t e = cudaStreamSynchronize(ctx->stream);
      if (e != cudaSuccess) return set_err(ctx, SFFT_ECUDA, "sync: %s", cudaGetErrorString(e));
    }
    b.release();
    size_t nb = std::max(bytes, (size_t)256);
    cudaError_t e = cudaMalloc(&b.p, nb);
    if (e != cudaSuccess) {
      b.p = nullptr;
      return set_err(ctx, SFFT_ENOMEM, "cudaMalloc(%zu) for %s: %s", nb, name,
                     cudaGetErrorString(e));
    }
    b.bytes = nb;
  }
  *out = b.p;
  return SFFT_OK;
}

bool finite(double x) { return isfinite(x) != 0; }

cudaEvent_t take_event(sfft_ctx* ctx) {
  if (!ctx->ev_pool.empty()) {
    cudaEvent_t e = ctx->ev_pool.back();
    ctx->ev_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

// Records a CUDA event pair around one launch when profiling is on.
struct PhaseScope {
  sfft_ctx* ctx;
  int phase;
  cudaEvent_t a = nullptr;
  PhaseScope(sfft_ctx* c, int ph) : ctx(c), phase(ph) {
    if (ctx->prof) {
      a = take_event(ctx);
      cudaEventRecord(a, ctx->stream);
    }
  }
  ~PhaseScope() {
    if (ctx->prof && a) {
      cudaEvent_t b = take_event(ctx);
      cudaEventRecord(b, ctx->stream);
      ctx->ev_open.push_back({phase, {a, b}});
    }
  }
};

double* acc_ptr(sfft_ctx* ctx) { return ctx->prof ? ctx->prof_acc : nullptr; }

// Moment-explosion time of E[S_T^p] under Heston (Andersen & Piterbarg 2007):
// the Riccati coefficient of v0 in log E[exp(p X_T)] solves
// B' = a B^2 - b B + c, B(0) = 0, with a = sv^2/2, b = kappa - rho sv p,
// c = p(p-1)/2, D = b^2 - 4ac; T* is the time B takes to reach infinity.
double heston_explosion_time(double kappa, double sv, double rho, double p) {
  const double b = kappa - rho * sv * p;
  const double D2 = b * b - sv * sv * p * (p - 1.0);
  if (D2 >= 0.0) {
    const double d = sqrt(D2);
    // real roots: B settles at the smaller one unless both are negative
    if (p * (p - 1.0) <= 0.0 || b >= 0.0) return INFINITY;
    if (d == 0.0) return -2.0 / b;
    return log((b - d) / (b + d)) / d;
  }
  // no real roots: T* = integral_0^inf dB / (a B^2 - b B + c)
  const double dl = sqrt(-D2);
  return 2.0 / dl * (0.5 * M_PI + atan(b / dl));
}

// Validation and planning of one problem (host side, before any launch).
sfft_status plan(sfft_ctx* ctx, const sfft_problem& pr, InstParams* out) {
  if (pr.model < 0 || pr.model > 3) return set_err(ctx, SFFT_EINVAL, "model %d", pr.model);
  if (pr.quad < 0 || pr.quad > 1) return set_err(ctx, SFFT_EINVAL, "quad %d", pr.quad);
  if (pr.n < 1 || pr.n > SFFT_MAX_N) return set_err(ctx, SFFT_EINVAL, "n=%d out of [1,%d]", pr.n, SFFT_MAX_N);
  if (!(pr.S0 > 0.0) || !finite(pr.S0)) return set_err(ctx, SFFT_EINVAL, "S0 must be finite and > 0");
  if (!(pr.T > 0.0) || !finite(pr.T)) return set_err(ctx, SFFT_EINVAL, "T must be finite and > 0");
  if (!finite(pr.r)) return set_err(ctx, SFFT_EINVAL, "r must be finite");
  if (!finite(pr.alpha) || pr.alpha == 0.0 || pr.alpha == -1.0)
    return set_err(ctx, SFFT_EINVAL, "alpha must be finite, not 0 or -1");
  if (!(pr.tol > 0.0 && pr.tol < 1.0)) return set_err(ctx, SFFT_EINVAL, "tol must be in (0,1)");
  if (!isnan(pr.k0)) return set_err(ctx, SFFT_EINVAL, "k0 must be NaN (default grid start)");
  if (pr.max_rank < 0 || pr.max_rank > SFFT_MAX_RANK)
    return set_err(ctx, SFFT_EINVAL, "max_rank %d out of [0,%d]", pr.max_rank, SFFT_MAX_RANK);
  if (pr.quad == SFFT_QUAD_SIMPSON_CM99 && !(pr.eta > 0.0 && finite(pr.eta)))
    return set_err(ctx, SFFT_EINVAL, "eta must be > 0 for Simpson");
  if (pr.quad == SFFT_QUAD_RECT_SYM && !finite(pr.eta)) return set_err(ctx, SFFT_EINVAL, "eta not finite");
  for (int i = 0; i < 8; ++i)
    if (!finite(pr.p[i])) return set_err(ctx, SFFT_EINVAL, "parameter p[%d] not finite", i);
  const double* p = pr.p;
  const double a1 = pr.alpha + 1.0;
  memset(out, 0, sizeof *out);
  switch (pr.model) {
    case SFFT_GBM:
      if (!(p[0] > 0.0)) return set_err(ctx, SFFT_EINVAL, "GBM sigma must be > 0");
      break;
    case SFFT_HESTON:
      if (!(p[0] > 0.0 && p[1] > 0.0 && p[2] > 0.0 && p[3] >= -1.0 && p[3] <= 1.0 && p[4] >= 0.0))
        return set_err(ctx, SFFT_EINVAL, "Heston needs kappa,theta,sigma_v > 0, |rho|<=1, v0>=0");
      if (!(heston_explosion_time(p[0], p[2], p[3], a1) > pr.T))
        return set_err(ctx, SFFT_EMOMENT, "Heston moment of order alpha+1 explodes before T");
      break;
    case SFFT_MERTON:
      if (!(p[0] > 0.0 && p[1] >= 0.0 && p[3] >= 0.0))
        return set_err(ctx, SFFT_EINVAL, "Merton needs sigma > 0, lambda >= 0, delta_J >= 0");
      out->kbar = exp(p[2] + 0.5 * p[3] * p[3]) - 1.0;
      break;
    case SFFT_VG: {
      if (!(p[0] > 0.0 && p[1] > 0.0)) return set_err(ctx, SFFT_EINVAL, "VG needs sigma, nu > 0");
      const double c1 = 1.0 - p[2] * p[1] - 0.5 * p[0] * p[0] * p[1];
      if (!(c1 > 0.0)) return set_err(ctx, SFFT_EINVAL, "VG: 1 - theta nu - sigma^2 nu/2 must be > 0");
      const double cp = 1.0 - p[2] * p[1] * a1 - 0.5 * p[0] * p[0] * p[1] * a1 * a1;
      if (!(cp > 0.0)) return set_err(ctx, SFFT_EMOMENT, "VG moment of order alpha+1 is infinite");
      out->omega = log(c1) / p[1];
      break;
    }
  }
  out->model = pr.model;
  out->quad = pr.quad;
  out->n = pr.n;
  out->max_rank = pr.max_rank ? pr.max_rank : SFFT_DEFAULT_MAX_RANK;
  for (int i = 0; i < 8; ++i) out->p[i] = pr.p[i];
  out->S0 = pr.S0;
  out->r = pr.r;
  out->T = pr.T;
  out->alpha = pr.alpha;
  out->tol = pr.tol;
  out->disc = exp(-pr.r * pr.T);
  const double M = ldexp(1.0, pr.n);
  if (pr.quad == SFFT_QUAD_SIMPSON_CM99) {
    out->dv = pr.eta;
    out->dk = 2.0 * M_PI / (M * pr.eta);
    out->k0 = -M_PI / pr.eta;
    out->N = 0;
  } else {
    const long long N = 1LL << (pr.n - 1);
    out->N = N;
    out->dv = pr.eta > 0.0 ? pr.eta : M_PI / sqrt((double)N);
    out->dk = M_PI / ((double)N * out->dv);
    out->k0 = -(double)N * out->dk / 2.0;
  }
  return SFFT_OK;
}

sfft_status check_strikes(sfft_ctx* ctx, int n, long long lb, long long stride, int q, int* tbits) {
  if (q < 0 || q > SFFT_MAX_STRIKES) return set_err(ctx, SFFT_EINVAL, "q=%d out of range", q);
  if (stride < 1 || (stride & (stride - 1))) return set_err(ctx, SFFT_EINVAL, "stride must be a power of two");
  if (lb < 0 || (lb & (stride - 1))) return set_err(ctx, SFFT_EINVAL, "l_begin must be a non-negative multiple of stride");
  int t = 0;
  while ((1LL << t) < stride) ++t;
  const long long M = 1LL << n;
  if (q > 0) {
    if (lb >= M) return set_err(ctx, SFFT_EINVAL, "l_begin beyond the grid");
    if (q > 1 && (t > n || lb + (long long)(q - 1) * stride >= M))
      return set_err(ctx, SFFT_EINVAL, "strike set runs beyond the grid");
  }
  *tbits = t;
  return SFFT_OK;
}

int blocks_per_sm(const void* fn, size_t smem, int threads = kThreads) {
  int b = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, fn, threads, smem) != cudaSuccess) b = 1;
  return std::max(b, 1);
}

size_t svd_smem() { return la::ts_svd_smem_bytes(LA_MAXP, kHb) + 256; }

sfft_status set_smem_attrs(sfft_ctx* ctx) {
  const int sm = (int)svd_smem();
  CK(cudaFuncSetAttribute(k_integrand_ttsvd, cudaFuncAttributeMaxDynamicSharedMemorySize, sm));
  CK(cudaFuncSetAttribute(k_integrand_cross, cudaFuncAttributeMaxDynamicSharedMemorySize, sm));
  CK(cudaFuncSetAttribute(k_tt_round, cudaFuncAttributeMaxDynamicSharedMemorySize,
                          (int)round_smem(4).bytes));
  CK(cudaFuncSetAttribute(k_zipup, cudaFuncAttributeMaxDynamicSharedMemorySize, sm));
  CK(cudaFuncSetAttribute(k_zipup_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, sm));
  CK(cudaFuncSetAttribute(k_fft_pass, cudaFuncAttributeMaxDynamicSharedMemorySize, 100 * 1024));
  return SFFT_OK;
}

// MPO of Q_n at tolerance tol: cached; built by k_mpo_interp + k_tt_round.
sfft_status build_mpos(sfft_ctx* ctx, const std::vector<std::pair<int, double>>& want);

const MpoEntry* find_mpo(const sfft_ctx* ctx, int n, double tol) {
  for (const auto& e : ctx->mpos)
    if (e.n == n && e.tol == tol) return &e;
  return nullptr;
}

sfft_status get_mpo(sfft_ctx* ctx, int n, double tol, const MpoEntry** out) {
  if (!(*out = find_mpo(ctx, n, tol))) {
    sfft_status s = build_mpos(ctx, {{n, tol}});
    if (s) return s;
    *out = find_mpo(ctx, n, tol);
  }
  return SFFT_OK;
}

// Host-to-device copy on the context's stream; during graph capture the
// source is first staged in the pinned arena.
sfft_status h2d(sfft_ctx* ctx, void* dst, const void* src, size_t bytes, bool is_params = false) {
  if (ctx->stage) {
    auto* st = ctx->stage;
    const size_t off = (st->used + 255) & ~(size_t)255;
    if (off + bytes > st->cap) {
      st->overflow = true;
      return set_err(ctx, SFFT_ENOMEM, "graph staging arena too small");
    }
    memcpy(st->base + off, src, bytes);
    if (is_params) {
      st->p_off = off;
      st->p_bytes = bytes;
    }
    st->used = off + bytes;
    src = st->base + off;
  }
  CK(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, ctx->stream));
  return SFFT_OK;
}

template <class T>
sfft_status upload(sfft_ctx* ctx, const char* name, const std::vector<T>& v, T** out) {
  void* p;
  sfft_status s = ensure(ctx, name, sizeof(T) * std::max<size_t>(v.size(), 1), &p);
  if (s) return s;
  if (!v.empty() && (s = h2d(ctx, p, v.data(), sizeof(T) * v.size(), strcmp(name, "P") == 0))) return s;
  *out = reinterpret_cast<T*>(p);
  return SFFT_OK;
}

// Build every (n, tol) MPO of `want` that is not cached yet. Each new MPO
// gets its interpolation launch; then one k_tt_round launch rounds all of
// them side by side (one CTA per MPO, d = 4, with left orthogonalisation),
// and one read-back fetches their ranks.
sfft_status build_mpos(sfft_ctx* ctx, const std::vector<std::pair<int, double>>& want) {
  std::vector<std::pair<int, double>> miss;
  for (const auto& w : want)
    if (!find_mpo(ctx, w.first, w.second) && std::find(miss.begin(), miss.end(), w) == miss.end())
      miss.push_back(w);
  if (miss.empty()) return SFFT_OK;
  const long long slot = (long long)SFFT_MAX_N * SFFT_CORE_STRIDE_D4;
  const int first = (int)ctx->mpos.size();
  const int nm = (int)miss.size();
  const int tot = first + nm;
  if (tot > ctx->mpo_slots) {
    // grow the pool (copy existing entries)
    const int nslots = std::max(tot, std::max(16, ctx->mpo_slots * 2));
    void* np = nullptr;
    void* nr = nullptr;
    CK(cudaMalloc(&np, sizeof(cd) * slot * nslots));
    CK(cudaMalloc(&nr, sizeof(int) * (SFFT_MAX_N + 1) * nslots));
    if (ctx->mpo_slots) {
      CK(cudaMemcpyAsync(np, ctx->mpo_pool.p, sizeof(cd) * slot * ctx->mpo_slots,
                         cudaMemcpyDeviceToDevice, ctx->stream));
      CK(cudaMemcpyAsync(nr, ctx->mpo_ranks_dev.p, sizeof(int) * (SFFT_MAX_N + 1) * ctx->mpo_slots,
                         cudaMemcpyDeviceToDevice, ctx->stream));
      CK(cudaStreamSynchronize(ctx->stream));
    }
    void* zp = nullptr;
    void* zr = nullptr;
    CK(cudaMalloc(&zp, sizeof(cd) * SFFT_ZPRE_BLOCK * nslots));
    CK(cudaMalloc(&zr, sizeof(int) * (SFFT_MAX_N + 1) * nslots));
    if (ctx->mpo_slots) {
      CK(cudaMemcpyAsync(zp, ctx->zpre_pool.p, sizeof(cd) * SFFT_ZPRE_BLOCK * ctx->mpo_slots,
                         cudaMemcpyDeviceToDevice, ctx->stream));
      CK(cudaMemcpyAsync(zr, ctx->zpre_ranks_dev.p, sizeof(int) * (SFFT_MAX_N + 1) * ctx->mpo_slots,
                         cudaMemcpyDeviceToDevice, ctx->stream));
      CK(cudaStreamSynchronize(ctx->stream));
    }
    ctx->mpo_pool.release();
    ctx->mpo_ranks_dev.release();
    ctx->zpre_pool.release();
    ctx->zpre_ranks_dev.release();
    ctx->mpo_pool.p = np;
    ctx->mpo_pool.bytes = sizeof(cd) * slot * nslots;
    ctx->mpo_ranks_dev.p = nr;
    ctx->mpo_ranks_dev.bytes = sizeof(int) * (SFFT_MAX_N + 1) * nslots;
    ctx->zpre_pool.p = zp;
    ctx->zpre_pool.bytes = sizeof(cd) * SFFT_ZPRE_BLOCK * nslots;
    ctx->zpre_ranks_dev.p = zr;
    ctx->zpre_ranks_dev.bytes = sizeof(int) * (SFFT_MAX_N + 1) * nslots;
    ctx->mpo_slots = nslots;
  }
  cd* pool = reinterpret_cast<cd*>(ctx->mpo_pool.p);
  int* rk = reinterpret_cast<int*>(ctx->mpo_ranks_dev.p);
  // rounding arguments indexed by pool slot; the list names the new slots
  std::vector<int> n_v(tot, 0), maxr_v(tot, SFFT_SLOT_RANK_DEV), list(nm);
  std::vector<double> tol_v(tot, 0.0);
  std::vector<long long> off_v(tot);
  for (int i = 0; i < tot; ++i) off_v[i] = slot * i;
  for (int k = 0; k < nm; ++k) {
    const int idx = first + k;
    n_v[idx] = miss[k].first;
    tol_v[idx] = miss[k].second;
    list[k] = idx;
  }
  int *n_d, *maxr_d, *list_d;
  double* tol_d;
  long long* off_d;
  sfft_status s;
  if ((s = upload(ctx, "mpo_n", n_v, &n_d)) || (s = upload(ctx, "mpo_maxr", maxr_v, &maxr_d)) ||
      (s = upload(ctx, "mpo_list", list, &list_d)) || (s = upload(ctx, "mpo_tol", tol_v, &tol_d)) ||
      (s = upload(ctx, "mpo_off", off_v, &off_d)))
    return s;
  void* p;
  if ((s = ensure(ctx, "mpo_counter", sizeof(int), &p))) return s;
  int* ctr = reinterpret_cast<int*>(p);
  CK(cudaMemsetAsync(ctr, 0, sizeof(int), ctx->stream));
  for (int k = 0; k < nm; ++k) {
    const int idx = first + k;
    PhaseScope ps(ctx, PH_MPO);
    k_mpo_interp<<<n_v[idx], kThreads, 0, ctx->stream>>>(n_v[idx], SFFT_MPO_NODES, pool + off_v[idx],
                                                         SFFT_CORE_STRIDE_D4, rk + (SFFT_MAX_N + 1) * idx);
  }
  CK(cudaGetLastError());
  const RoundSmem rs = round_smem(4);
  const int grid = std::min(nm, ctx->num_sms * blocks_per_sm((const void*)k_tt_round, rs.bytes));
  if ((s = ensure(ctx, "mpo_scratch", sizeof(cd) * (size_t)SFFT_ROUND_SCRATCH * grid, &p))) return s;
  {
    PhaseScope ps(ctx, PH_MPO);
    k_tt_round<<<grid, kThreads, rs.bytes, ctx->stream>>>(
        list_d, nm, ctr, n_d, 4, 1, tol_d, maxr_d, pool, off_d, SFFT_CORE_STRIDE_D4, rk,
        reinterpret_cast<cd*>(p), SFFT_ROUND_SCRATCH, nullptr, rs.hb, acc_ptr(ctx), PH_MPO, rs.pmax,
        rs.vcap, nullptr, nullptr);
  }
  CK(cudaGetLastError());
  // the zip-up of each new MPO with the all-delta TT (ranks 1, cores (1, 0)):
  // the prefix of every TT-SVD instance's zip-up, with the carry after each
  // site; full carve, one CTA per MPO, no profiling counters
  cd* zpool = reinterpret_cast<cd*>(ctx->zpre_pool.p);
  int* zrk = reinterpret_cast<int*>(ctx->zpre_ranks_dev.p);
  {
    std::vector<cd> delta((size_t)2 * SFFT_MAX_N);
    for (int i = 0; i < SFFT_MAX_N; ++i) {
      delta[2 * i] = make_double2(1.0, 0.0);
      delta[2 * i + 1] = make_double2(0.0, 0.0);
    }
    std::vector<long long> zero_off(tot, 0), zoff_v(tot);
    for (int i = 0; i < tot; ++i) zoff_v[i] = SFFT_ZPRE_BLOCK * i;
    std::vector<int> ones((size_t)(SFFT_MAX_N + 1) * tot, 1), zst(tot, 0);
    cd* delta_d;
    long long *zero_d, *zoff_d;
    int *ones_d, *zst_d;
    if ((s = upload(ctx, "zpre_delta", delta, &delta_d)) || (s = upload(ctx, "zpre_zero", zero_off, &zero_d)) ||
        (s = upload(ctx, "zpre_off", zoff_v, &zoff_d)) || (s = upload(ctx, "zpre_ones", ones, &ones_d)) ||
        (s = upload(ctx, "zpre_status", zst, &zst_d)))
      return s;
    const RoundSmem zs = zip_smem();
    const int zg = std::min(nm, ctx->num_sms * blocks_per_sm((const void*)k_zipup, zs.bytes));
    if ((s = ensure(ctx, "zpre_scratch", sizeof(cd) * (size_t)SFFT_ZIP_SCRATCH * zg, &p))) return s;
    cd* zscr = reinterpret_cast<cd*>(p);
    if ((s = ensure(ctx, "zpre_counter", sizeof(int), &p))) return s;
    int* zctr = reinterpret_cast<int*>(p);
    CK(cudaMemsetAsync(zctr, 0, sizeof(int), ctx->stream));
    ZipPrefix zp{nullptr, zoff_d, nullptr, nullptr, zpool};
    {
      PhaseScope ps(ctx, PH_MPO);
      k_zipup<<<zg, kThreads, zs.bytes, ctx->stream>>>(
          list_d, nm, zctr, n_d, tol_d, maxr_d, delta_d, zero_d, ones_d, pool, off_d, rk, zpool, zoff_d, zrk,
          2, SFFT_CORE_STRIDE_D4, SFFT_CORE_STRIDE_D2, zscr, SFFT_ZIP_SCRATCH, zst_d, zs.hb, nullptr, zs.vcap,
          nullptr, nullptr, LA_MAXQ, 1 << 30, zp);
    }
    CK(cudaGetLastError());
    std::vector<int> zr_h((size_t)(SFFT_MAX_N + 1) * nm), zst_h(nm);
    CK(cudaMemcpyAsync(zr_h.data(), zrk + (size_t)(SFFT_MAX_N + 1) * first, sizeof(int) * zr_h.size(),
                       cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaMemcpyAsync(zst_h.data(), zst_d + first, sizeof(int) * nm, cudaMemcpyDeviceToHost, ctx->stream));
    std::vector<int> rr((size_t)(SFFT_MAX_N + 1) * nm);
    CK(cudaMemcpyAsync(rr.data(), rk + (size_t)(SFFT_MAX_N + 1) * first, sizeof(int) * rr.size(),
                       cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    for (int k = 0; k < nm; ++k) {
      MpoEntry e;
      e.idx = first + k;
      e.n = miss[k].first;
      e.tol = miss[k].second;
      e.off = off_v[e.idx];
      e.ranks.assign(rr.begin() + (size_t)(SFFT_MAX_N + 1) * k, rr.begin() + (size_t)(SFFT_MAX_N + 1) * (k + 1));
      for (int i = 0; i <= e.n; ++i)
        if (e.ranks[i] < 1 || e.ranks[i] > SFFT_SLOT_RANK_DEV)
          return set_err(ctx, SFFT_ERANK, "MPO rank %d at bond %d", e.ranks[i], i);
      if (zst_h[k] == 0) {
        e.zoff = zoff_v[e.idx];
        e.zranks.assign(zr_h.begin() + (size_t)(SFFT_MAX_N + 1) * k,
                        zr_h.begin() + (size_t)(SFFT_MAX_N + 1) * (k + 1));
      }
      ctx->mpos.push_back(e);
    }
  }
  return SFFT_OK;
}

// Device-side state of one batch of valid instances through the TT path.
struct Batch {
  int count = 0;
  std::vector<int> n_host;  // grid exponent of each valid instance
  InstParams* P = nullptr;
  int* n_arr = nullptr;
  double* tol_arr = nullptr;
  int* maxr_arr = nullptr;
  int* status = nullptr;
  cd* A = nullptr;
  long long* a_off = nullptr;
  int* a_ranks = nullptr;
  cd* B = nullptr;
  int* b_ranks = nullptr;
  long long* w_off = nullptr;
  int* w_ranks = nullptr;
  int* zpre_t = nullptr;          // delta sites above each instance's TT-SVD block
  long long* zpre_off = nullptr;  // its MPO's prefix block (-1: none)
  int* zpre_ranks = nullptr;      // that prefix's ranks, per instance
  std::vector<int> mpo_max;
  int* all_list = nullptr;  // instances, largest n first
  int* counters = nullptr;  // work-queue counters of the launches
};

// Integrand TT -> zip-up -> rounding, for `valid` problems (host vectors of
// planned parameters). Leaves the output TTs in b.B.
sfft_status run_tt_path(sfft_ctx* ctx, const std::vector<InstParams>& prm, Batch& b,
                        const std::vector<const MpoEntry*>* mpos_in, bool apply) {
  const int cnt = (int)prm.size();
  b.count = cnt;
  sfft_status s;
  std::vector<int> n_arr(cnt), maxr(cnt);
  b.n_host.resize(cnt);
  for (int i = 0; i < cnt; ++i) b.n_host[i] = prm[i].n;
  std::vector<double> tol(cnt);
  std::vector<long long> off(cnt);
  long long tot = 0;
  for (int i = 0; i < cnt; ++i) {
    n_arr[i] = prm[i].n;
    maxr[i] = prm[i].max_rank;
    tol[i] = prm[i].tol;
    off[i] = tot;
    tot += (long long)prm[i].n * SFFT_CORE_STRIDE_D2;
  }
  if ((s = upload(ctx, "P", prm, &b.P))) return s;
  if ((s = upload(ctx, "n_arr", n_arr, &b.n_arr))) return s;
  if ((s = upload(ctx, "tol_arr", tol, &b.tol_arr))) return s;
  if ((s = upload(ctx, "maxr_arr", maxr, &b.maxr_arr))) return s;
  if ((s = upload(ctx, "a_off", off, &b.a_off))) return s;
  void* p;
  if ((s = ensure(ctx, "A", sizeof(cd) * std::max(tot, 1LL), &p))) return s;
  b.A = reinterpret_cast<cd*>(p);
  if ((s = ensure(ctx, "B", sizeof(cd) * std::max(tot, 1LL), &p))) return s;
  b.B = reinterpret_cast<cd*>(p);
  const size_t rk = sizeof(int) * (SFFT_MAX_N + 1) * std::max(cnt, 1);
  if ((s = ensure(ctx, "a_ranks", rk, &p))) return s;
  b.a_ranks = reinterpret_cast<int*>(p);
  if ((s = ensure(ctx, "b_ranks", rk, &p))) return s;
  b.b_ranks = reinterpret_cast<int*>(p);
  if ((s = ensure(ctx, "w_ranks", rk, &p))) return s;
  b.w_ranks = reinterpret_cast<int*>(p);
  if ((s = ensure(ctx, "status", sizeof(int) * std::max(cnt, 1), &p))) return s;
  b.status = reinterpret_cast<int*>(p);
  CK(cudaMemsetAsync(b.status, 0, sizeof(int) * std::max(cnt, 1), ctx->stream));
  if (cnt == 0) return SFFT_OK;

  // support probe -> block exponent m; small blocks by TT-SVD, wide ones by cross
  int* m_dev;
  if ((s = ensure(ctx, "m_arr", sizeof(int) * cnt, &p))) return s;
  m_dev = reinterpret_cast<int*>(p);
  {
    PhaseScope ps(ctx, PH_PROBE);
    k_support_probe<<<cnt, 64, 0, ctx->stream>>>(b.P, cnt, 1e-2, 4, m_dev);
  }
  CK(cudaGetLastError());
  // work lists of the builders, split and ordered on the device
  int *svd_dev, *cross_dev, *list_counts, *all_dev, *ctr;
  if ((s = ensure(ctx, "svd_list", sizeof(int) * cnt, &p))) return s;
  svd_dev = reinterpret_cast<int*>(p);
  if ((s = ensure(ctx, "cross_list", sizeof(int) * cnt, &p))) return s;
  cross_dev = reinterpret_cast<int*>(p);
  if ((s = ensure(ctx, "list_counts", sizeof(int) * 2, &p))) return s;
  list_counts = reinterpret_cast<int*>(p);
  {
    PhaseScope ps(ctx, PH_PROBE);
    k_build_lists<<<1, 1024, 0, ctx->stream>>>(m_dev, b.n_arr, cnt, kSvdMaxBits, svd_dev, cross_dev, list_counts);
  }
  CK(cudaGetLastError());
  // the zip-up, rounding and readout take every instance, largest n first
  std::vector<int> all_list(cnt);
  for (int i = 0; i < cnt; ++i) all_list[i] = i;
  std::stable_sort(all_list.begin(), all_list.end(), [&](int a, int c) { return prm[a].n > prm[c].n; });
  if ((s = upload(ctx, "all_list", all_list, &all_dev))) return s;
  if ((s = ensure(ctx, "counters", sizeof(int) * 16, &p))) return s;
  ctr = reinterpret_cast<int*>(p);
  CK(cudaMemsetAsync(ctr, 0, sizeof(int) * 16, ctx->stream));
  b.all_list = all_dev;
  // work-queue counters, one per launch of a step: 0 TT-SVD builder (tier 1),
  // 1 cross builder, 2 rounding of the cross output, 3 zip-up, 4 output
  // rounding (tier 1), 5 readout, 7 builder tier 2, 8 rounding tier 2,
  // 9 zip-up tier 2, 10 cross tier 2
  b.counters = ctr;
  const size_t smem = svd_smem();
  // hand-off lists of the two-tier launches: [count, instances...]
  int *defer_build, *defer_round, *defer_cross;
  if ((s = ensure(ctx, "defer_build", sizeof(int) * (cnt + 1), &p))) return s;
  defer_build = reinterpret_cast<int*>(p);
  if ((s = ensure(ctx, "defer_round", sizeof(int) * (cnt + 1), &p))) return s;
  defer_round = reinterpret_cast<int*>(p);
  if ((s = ensure(ctx, "defer_cross", sizeof(int) * (cnt + 1), &p))) return s;
  defer_cross = reinterpret_cast<int*>(p);
  CK(cudaMemsetAsync(defer_build, 0, sizeof(int), ctx->stream));
  CK(cudaMemsetAsync(defer_round, 0, sizeof(int), ctx->stream));
  // delta sites above each TT-SVD block (0 for the cross builder's instances)
  int* zpre_t;
  if ((s = ensure(ctx, "zpre_t", sizeof(int) * cnt, &p))) return s;
  zpre_t = reinterpret_cast<int*>(p);
  CK(cudaMemsetAsync(zpre_t, 0, sizeof(int) * cnt, ctx->stream));
  b.zpre_t = zpre_t;
  CK(cudaMemsetAsync(defer_cross, 0, sizeof(int), ctx->stream));
  // TT-SVD builder: tier 1 panels up to kSmallP columns in 128-thread CTAs,
  // several per SM; tier 2 the full carve for the instances tier 1 handed on
  const int build_p1 = std::min(ctx->cur.build_p, kSmallP);
  const size_t bsmem1 = la::ts_svd_smem_bytes(build_p1, build_p1) + 256;
  const int bgrid1 = std::min(cnt, ctx->num_sms * blocks_per_sm((const void*)k_integrand_ttsvd, bsmem1,
                                                                kThreadsSmall));
  const int bgrid2 = std::min(cnt, ctx->num_sms * blocks_per_sm((const void*)k_integrand_ttsvd, smem));
  const long long sstride = 2LL << kSvdMaxBits;
  if ((s = ensure(ctx, "build_scratch", sizeof(cd) * sstride * std::max(bgrid1, bgrid2), &p))) return s;
  cd* build_scratch = reinterpret_cast<cd*>(p);
  // cross builder: tier 1 ranks up to kCrossSmallR in 128-thread CTAs, every
  // instance in flight at once; tier 2 the rest; then the rounding of the
  // interpolatory cores
  const int xp = 2 * kCrossSmallR;
  const int xhb = kCrossSmallHb;
  const size_t xsmem1 = la::ts_svd_smem_bytes(xp, xhb) + 256;
  const int xgrid1 = std::min(cnt, ctx->num_sms * blocks_per_sm((const void*)k_integrand_cross, xsmem1,
                                                                kThreadsSmall));
  const int xgrid = std::min(cnt, ctx->num_sms * blocks_per_sm((const void*)k_integrand_cross, smem));
  if ((s = ensure(ctx, "cross_scratch", sizeof(cd) * (size_t)4096 * std::max(xgrid1, xgrid), &p))) return s;
  cd* cross_scratch = reinterpret_cast<cd*>(p);
  const RoundSmem xrs = round_smem(2);
  const int xgrid_r = std::min(cnt, ctx->num_sms * blocks_per_sm((const void*)k_tt_round, xrs.bytes));
  if ((s = ensure(ctx, "xround_scratch", sizeof(cd) * (size_t)SFFT_ROUND_SCRATCH * xgrid_r, &p))) return s;
  cd* xround_scratch = reinterpret_cast<cd*>(p);

  // The two builders take disjoint instances. The cross builder (a few long
  // instances, one per CTA) goes first on the caller's stream, where nothing
  // delays its dispatch; the TT-SVD builder follows on the side stream behind
  // the fork event, and its persistent CTAs fill every slot the cross CTAs
  // leave or free. (The other order lets the TT-SVD CTAs take every SM first
  // and pushes the cross builder behind them.)
  CK(cudaEventRecord(ctx->fork, ctx->stream));
  CK(cudaStreamWaitEvent(ctx->side, ctx->fork, 0));
  {
    PhaseScope ps(ctx, PH_CROSS);
    k_integrand_cross<<<xgrid1, kThreadsSmall, xsmem1, ctx->stream>>>(
        b.P, cross_dev, cnt, ctr + 1, cross_scratch, 4096, b.A, b.a_off, SFFT_CORE_STRIDE_D2, b.a_ranks,
        b.status, xhb, acc_ptr(ctx), kCrossSweeps, xp, std::min(ctx->cur.cross_r, kCrossSmallR), defer_cross,
        list_counts + 1, m_dev, zpre_t);
  }
  {
    PhaseScope ps(ctx, PH_CROSS);
    k_integrand_cross<<<xgrid, kThreads, smem, ctx->stream>>>(
        b.P, defer_cross + 1, 0, ctr + 10, cross_scratch, 4096, b.A, b.a_off, SFFT_CORE_STRIDE_D2, b.a_ranks,
        b.status, kHb, acc_ptr(ctx), kCrossSweeps, LA_MAXP, CROSS_RANK_CAP, nullptr, defer_cross, m_dev,
        zpre_t);
  }
  {
    // interpolatory cores -> right-orthonormal, truncated to tol
    PhaseScope ps(ctx, PH_CROSS);
    k_tt_round<<<xgrid_r, kThreads, xrs.bytes, ctx->stream>>>(
        cross_dev, cnt, ctr + 2, b.n_arr, 2, 1, b.tol_arr, b.maxr_arr, b.A, b.a_off, SFFT_CORE_STRIDE_D2,
        b.a_ranks, xround_scratch, SFFT_ROUND_SCRATCH, b.status, xrs.hb, acc_ptr(ctx), PH_CROSS, xrs.pmax,
        xrs.vcap, nullptr, list_counts + 1, zpre_t);
  }
  const cudaError_t main_err = cudaGetLastError();
  cudaStream_t main_stream = ctx->stream;
  ctx->stream = ctx->side;
  {
    PhaseScope ps(ctx, PH_BUILD);
    k_integrand_ttsvd<<<bgrid1, kThreadsSmall, bsmem1, ctx->stream>>>(
        b.P, m_dev, svd_dev, cnt, ctr + 0, build_scratch, sstride, b.A, b.a_off, SFFT_CORE_STRIDE_D2,
        b.a_ranks, b.status, build_p1, acc_ptr(ctx), build_p1, defer_build, list_counts, zpre_t);
  }
  {
    PhaseScope ps(ctx, PH_BUILD);
    k_integrand_ttsvd<<<bgrid2, kThreads, smem, ctx->stream>>>(
        b.P, m_dev, defer_build + 1, 0, ctr + 7, build_scratch, sstride, b.A, b.a_off, SFFT_CORE_STRIDE_D2,
        b.a_ranks, b.status, kHb, acc_ptr(ctx), LA_MAXP, nullptr, defer_build, zpre_t);
  }
  const cudaError_t side_err = cudaGetLastError();
  ctx->stream = main_stream;
  // join before anything else can fail, so no side-stream work is left
  // outside the caller's stream order (or open in a capture)
  CK(cudaEventRecord(ctx->join, ctx->side));
  CK(cudaStreamWaitEvent(ctx->stream, ctx->join, 0));
  CK(side_err);
  CK(main_err);
  if (ctx->fault_enoconv >= 0 && ctx->fault_enoconv < cnt) {
    // test hook: the builder of this batch position reports non-convergence
    static const int kEnoconv = SFFT_ENOCONV;
    CK(cudaMemcpyAsync(b.status + ctx->fault_enoconv, &kEnoconv, sizeof(int), cudaMemcpyHostToDevice,
                       ctx->stream));
  }
  if (!apply) return SFFT_OK;

  // MPO per instance
  std::vector<long long> w_off(cnt);
  std::vector<int> w_ranks((size_t)cnt * (SFFT_MAX_N + 1));
  for (int i = 0; i < cnt; ++i) {
    const MpoEntry* e = (*mpos_in)[i];
    w_off[i] = e->off;
    std::copy(e->ranks.begin(), e->ranks.end(), w_ranks.begin() + (size_t)i * (SFFT_MAX_N + 1));
  }
  if ((s = upload(ctx, "w_off", w_off, &b.w_off))) return s;
  if ((s = h2d(ctx, b.w_ranks, w_ranks.data(), sizeof(int) * w_ranks.size()))) return s;
  // the zip-up of each MPO's delta prefix, taken by the TT-SVD instances
  std::vector<long long> z_off(cnt);
  std::vector<int> z_ranks((size_t)cnt * (SFFT_MAX_N + 1), 1);
  for (int i = 0; i < cnt; ++i) {
    const MpoEntry* e = (*mpos_in)[i];
    z_off[i] = e->zoff;
    if (e->zoff >= 0) std::copy(e->zranks.begin(), e->zranks.end(), z_ranks.begin() + (size_t)i * (SFFT_MAX_N + 1));
  }
  if ((s = upload(ctx, "zpre_off_b", z_off, &b.zpre_off))) return s;
  if ((s = upload(ctx, "zpre_ranks_b", z_ranks, &b.zpre_ranks))) return s;
  const ZipPrefix zpre = ctx->zpre_on ? ZipPrefix{b.zpre_t, b.zpre_off, b.zpre_ranks,
                                                  reinterpret_cast<const cd*>(ctx->zpre_pool.p), nullptr}
                                      : ZipPrefix{};
  // tier 1: W-only carve, three CTAs per SM; tier 2: the full carve for the
  // instances whose panels (with their explicit Q) outgrow it
  int* defer_zip;
  if ((s = ensure(ctx, "defer_zip", sizeof(int) * (cnt + 1), &p))) return s;
  defer_zip = reinterpret_cast<int*>(p);
  CK(cudaMemsetAsync(defer_zip, 0, sizeof(int), ctx->stream));
  ctx->defer_heads[0] = defer_build;
  ctx->defer_heads[1] = defer_cross;
  ctx->defer_heads[2] = defer_zip;
  // work orders by decreasing sum_s r_s^2 (k_cost_order): the zip-up's from
  // the integrand ranks, the rounding's from the zip-up output ranks
  int *zip_order, *round_order;
  if ((s = ensure(ctx, "zip_order", sizeof(int) * cnt, &p))) return s;
  zip_order = reinterpret_cast<int*>(p);
  if ((s = ensure(ctx, "round_order", sizeof(int) * cnt, &p))) return s;
  round_order = reinterpret_cast<int*>(p);
  {
    PhaseScope ps(ctx, PH_ZIPUP);
    k_cost_order<<<1, 1024, 0, ctx->stream>>>(b.a_ranks, b.n_arr, cnt, zip_order);
  }
  CK(cudaGetLastError());
  const bool mixed = ctx->precision == SFFT_PRECISION_MIXED;
  // tier 1 of the FP64 path: 128-thread CTAs with a 32 x 64 panel block, six
  // per SM; the tensor-core variant keeps 256 threads and a 70 x 64 block
  const int zthreads1 = mixed ? kThreads : kThreadsSmall;
  const RoundSmem zs1 = zip_smem(true, mixed ? 70 : 32);
  const RoundSmem zs = zip_smem();
  // mixed precision: tier 1 runs each site's MPO contraction on the tensor
  // cores; tier 2 (rare, the full carve) stays FP64
  // The occupancy calculator reports one CTA per SM for any kernel that
  // allocates tensor memory; the hardware co-schedules as many as their
  // allocations fit (128 of the SM's 512 columns each here), so the tensor-
  // core zip-up takes the FP64 kernel's occupancy, capped at four per SM.
  int zbps = blocks_per_sm((const void*)k_zipup, zs1.bytes, zthreads1);
  if (mixed) zbps = std::min(zbps, 4);
  if (ctx->cur.zip_ctas > 0) zbps = std::min(zbps, ctx->cur.zip_ctas);
  const int zg1 = std::min(cnt, ctx->num_sms * zbps);
  const int zg2 = std::min(cnt, ctx->num_sms * blocks_per_sm((const void*)k_zipup, zs.bytes));
  if ((s = ensure(ctx, "zip_scratch", sizeof(cd) * (size_t)SFFT_ZIP_SCRATCH * std::max(zg1, zg2), &p)))
    return s;
  {
    PhaseScope ps(ctx, PH_ZIPUP);
    (mixed ? k_zipup_tc : k_zipup)<<<zg1, zthreads1, zs1.bytes, ctx->stream>>>(
        zip_order, cnt, ctr + 3, b.n_arr, b.tol_arr, b.maxr_arr, b.A, b.a_off, b.a_ranks,
        reinterpret_cast<const cd*>(ctx->mpo_pool.p), b.w_off, b.w_ranks, b.B, b.a_off, b.b_ranks,
        SFFT_CORE_STRIDE_D2, SFFT_CORE_STRIDE_D4, SFFT_CORE_STRIDE_D2, reinterpret_cast<cd*>(p),
        SFFT_ZIP_SCRATCH, b.status, zs1.hb, acc_ptr(ctx), zs1.vcap, defer_zip, nullptr, ctx->cur.zip_q,
        ctx->cur.zip_w, zpre);
  }
  CK(cudaGetLastError());
  {
    PhaseScope ps(ctx, PH_ZIPUP);
    k_zipup<<<zg2, kThreads, zs.bytes, ctx->stream>>>(
        defer_zip + 1, 0, ctr + 9, b.n_arr, b.tol_arr, b.maxr_arr, b.A, b.a_off, b.a_ranks,
        reinterpret_cast<const cd*>(ctx->mpo_pool.p), b.w_off, b.w_ranks, b.B, b.a_off, b.b_ranks,
        SFFT_CORE_STRIDE_D2, SFFT_CORE_STRIDE_D4, SFFT_CORE_STRIDE_D2, reinterpret_cast<cd*>(p),
        SFFT_ZIP_SCRATCH, b.status, zs.hb, acc_ptr(ctx), zs.vcap, nullptr, defer_zip, LA_MAXQ, ctx->cur.zip_w,
        zpre);
  }
  CK(cudaGetLastError());
  {
    PhaseScope ps(ctx, PH_ROUND);
    k_cost_order<<<1, 1024, 0, ctx->stream>>>(b.b_ranks, b.n_arr, cnt, round_order);
  }
  CK(cudaGetLastError());
  // tier 1: ranks up to kSmallRoundR in 128-thread CTAs; tier 2: the rest
  const RoundSmem rs1 = round_smem(2, false, std::min(ctx->cur.round_r, kSmallRoundR));
  const RoundSmem rs2 = round_smem(2, false);
  ctx->defer_heads[3] = defer_round;
  const int grid1 = std::min(cnt, ctx->num_sms * blocks_per_sm((const void*)k_tt_round, rs1.bytes, kThreadsSmall));
  const int grid2 = std::min(cnt, ctx->num_sms * blocks_per_sm((const void*)k_tt_round, rs2.bytes));
  if ((s = ensure(ctx, "round_scratch", sizeof(cd) * (size_t)SFFT_ROUND_SCRATCH * std::max(grid1, grid2), &p)))
    return s;
  {
    PhaseScope ps(ctx, PH_ROUND);
    k_tt_round<<<grid1, kThreadsSmall, rs1.bytes, ctx->stream>>>(
        round_order, cnt, ctr + 4, b.n_arr, 2, 0, b.tol_arr, b.maxr_arr, b.B, b.a_off, SFFT_CORE_STRIDE_D2,
        b.b_ranks, reinterpret_cast<cd*>(p), SFFT_ROUND_SCRATCH, b.status, rs1.hb, acc_ptr(ctx), PH_ROUND,
        rs1.pmax, rs1.vcap, defer_round, nullptr);
  }
  CK(cudaGetLastError());
  {
    PhaseScope ps(ctx, PH_ROUND);
    k_tt_round<<<grid2, kThreads, rs2.bytes, ctx->stream>>>(
        defer_round + 1, 0, ctr + 8, b.n_arr, 2, 0, b.tol_arr, b.maxr_arr, b.B, b.a_off, SFFT_CORE_STRIDE_D2,
        b.b_ranks, reinterpret_cast<cd*>(p), SFFT_ROUND_SCRATCH, b.status, rs2.hb, acc_ptr(ctx), PH_ROUND,
        rs2.pmax, rs2.vcap, nullptr, defer_round);
  }
  CK(cudaGetLastError());
  return SFFT_OK;
}

sfft_status copy_tt_out(sfft_ctx* ctx, const cd* base, const int* ranks_dev, int n, int d,
                        int core_stride, int* ranks_host, double* out, long long cap) {
  std::vector<int> r(SFFT_MAX_N + 1);
  CK(cudaMemcpyAsync(r.data(), ranks_dev, sizeof(int) * (SFFT_MAX_N + 1), cudaMemcpyDeviceToHost,
                     ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  long long need = 0;
  for (int s = 0; s < n; ++s) need += (long long)r[s] * d * r[s + 1];
  for (int s = 0; s <= n; ++s) ranks_host[s] = r[s];
  if (need > cap) return set_err(ctx, SFFT_EINVAL, "output capacity %lld < %lld", cap, need);
  long long o = 0;
  for (int s = 0; s < n; ++s) {
    const long long sz = (long long)r[s] * d * r[s + 1];
    CK(cudaMemcpyAsync(reinterpret_cast<cd*>(out) + o, base + (size_t)s * core_stride, sizeof(cd) * sz,
                       cudaMemcpyDeviceToDevice, ctx->stream));
    o += sz;
  }
  CK(cudaStreamSynchronize(ctx->stream));
  return SFFT_OK;
}

sfft_status copy_tt_in(sfft_ctx* ctx, const double* in, const int* ranks, int n, int d,
                       int core_stride, cd* base, int* ranks_dev) {
  for (int s = 0; s <= n; ++s)
    if (ranks[s] < 1 || ranks[s] > SFFT_SLOT_RANK_DEV || (d == 4 && ranks[s] > SFFT_SLOT_RANK_DEV))
      return set_err(ctx, SFFT_EINVAL, "rank %d at bond %d out of [1,%d]", ranks[s], s, SFFT_SLOT_RANK_DEV);
  if (ranks[0] != 1 || ranks[n] != 1) return set_err(ctx, SFFT_EINVAL, "boundary ranks must be 1");
  long long o = 0;
  for (int s = 0; s < n; ++s) {
    const long long sz = (long long)ranks[s] * d * ranks[s + 1];
    CK(cudaMemcpyAsync(base + (size_t)s * core_stride, reinterpret_cast<const cd*>(in) + o,
                       sizeof(cd) * sz, cudaMemcpyDeviceToDevice, ctx->stream));
    o += sz;
  }
  std::vector<int> r(SFFT_MAX_N + 1, 1);
  for (int s = 0; s <= n; ++s) r[s] = ranks[s];
  CK(cudaMemcpyAsync(ranks_dev, r.data(), sizeof(int) * (SFFT_MAX_N + 1), cudaMemcpyHostToDevice,
                     ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return SFFT_OK;
}

sfft_status finish_status(sfft_ctx* ctx, int count, const std::vector<int>& valid_idx,
                          const std::vector<int>& host_status, const int* dev_status,
                          int32_t* inst_status, sfft_info* info, const Batch* b,
                          const std::vector<const MpoEntry*>* mpos) {
  std::vector<int> st(count, 0);
  for (int i = 0; i < count; ++i) st[i] = host_status[i];
  std::vector<int> ds(valid_idx.size());
  std::vector<int> ar, br;
  if (!valid_idx.empty()) {
    CK(cudaMemcpyAsync(ds.data(), dev_status, sizeof(int) * ds.size(), cudaMemcpyDeviceToHost, ctx->stream));
    if (info && b) {
      ar.resize(valid_idx.size() * (SFFT_MAX_N + 1));
      br.resize(ar.size());
      CK(cudaMemcpyAsync(ar.data(), b->a_ranks, sizeof(int) * ar.size(), cudaMemcpyDeviceToHost, ctx->stream));
      CK(cudaMemcpyAsync(br.data(), b->b_ranks, sizeof(int) * br.size(), cudaMemcpyDeviceToHost, ctx->stream));
    }
  }
  CK(cudaStreamSynchronize(ctx->stream));
  for (size_t k = 0; k < valid_idx.size(); ++k) st[valid_idx[k]] = ds[k];
  sfft_status first = SFFT_OK;
  for (int i = 0; i < count; ++i) {
    if (inst_status) inst_status[i] = st[i];
    if (info) {
      info[i].status = st[i];
      info[i].int_rank = info[i].mpo_rank = info[i].out_rank = 0;
      info[i].tt_bytes = 0;
    }
    if (st[i] != SFFT_OK && first == SFFT_OK) first = (sfft_status)st[i];
  }
  if (info && b) {
    for (size_t k = 0; k < valid_idx.size(); ++k) {
      const int i = valid_idx[k];
      // the kernels write bonds 0..n of each instance's rank row; the rest of
      // the row is not theirs
      const int* a = ar.data() + k * (SFFT_MAX_N + 1);
      const int* c = br.data() + k * (SFFT_MAX_N + 1);
      const int nb = (k < b->n_host.size() ? b->n_host[k] : SFFT_MAX_N) + 1;
      info[i].int_rank = *std::max_element(a, a + nb);
      info[i].out_rank = *std::max_element(c, c + nb);
      if (mpos && (*mpos)[k]) {
        const auto& rr = (*mpos)[k]->ranks;
        info[i].mpo_rank = *std::max_element(rr.begin(), rr.end());
      }
    }
  }
  if (first != SFFT_OK && ctx->err.empty()) set_err(ctx, first, "instance failed: %s", sfft_status_string(first));
  return first;
}

// Signature of a batch for the tuning cache: its size and the distribution of
// what sets the kernels' work (grid exponents, models, tolerance, grid rule),
// each count quantised to its binary order of magnitude, so that batches
// drawn from the same workload share a signature. Host-side only.
std::string batch_signature(const sfft_problem* probs, int count) {
  int nb[6] = {0, 0, 0, 0, 0, 0}, mb[4] = {0, 0, 0, 0}, quads = 0;
  std::vector<double> tols;
  for (int i = 0; i < count; ++i) {
    const int n = probs[i].n;
    const int b = n <= 15 ? 0 : n <= 20 ? 1 : n <= 25 ? 2 : n <= 30 ? 3 : n <= 35 ? 4 : 5;
    nb[b]++;
    if (probs[i].model >= 0 && probs[i].model < 4) mb[probs[i].model]++;
    quads |= 1 << (probs[i].quad & 1);
    tols.push_back(probs[i].tol);
  }
  auto lg = [](int c) { int k = 0; while ((1 << k) <= c) ++k; return k; };  // 0 for 0, else floor(log2 c) + 1
  double tol_med = 1e-12;
  if (!tols.empty()) {
    std::nth_element(tols.begin(), tols.begin() + tols.size() / 2, tols.end());
    tol_med = tols[tols.size() / 2];
  }
  char buf[160];
  snprintf(buf, sizeof buf, "count=%d;n=%d,%d,%d,%d,%d,%d;model=%d,%d,%d,%d;tol=%d;quad=%d", lg(count), lg(nb[0]),
           lg(nb[1]), lg(nb[2]), lg(nb[3]), lg(nb[4]), lg(nb[5]), lg(mb[0]), lg(mb[1]), lg(mb[2]), lg(mb[3]),
           (int)lround(log10(tol_med > 0 ? tol_med : 1e-12)), quads);
  return buf;
}

std::string device_signature(const sfft_ctx* ctx) {
  cudaDeviceProp prop;
  char buf[96];
  if (cudaGetDeviceProperties(&prop, ctx->device) == cudaSuccess)
    snprintf(buf, sizeof buf, "sm%d%d x%d", prop.major, prop.minor, prop.multiProcessorCount);
  else
    snprintf(buf, sizeof buf, "sm? x%d", ctx->num_sms);
  return buf;
}

// The first-tier configuration of a call: the test hook's limits when set,
// else the forced one (while tuning), else the tuned one for the batch's
// signature, else the defaults.
void choose_tier1(sfft_ctx* ctx, const sfft_problem* probs, int count) {
  if (ctx->t1_hooked) {
    ctx->cur = ctx->t1;
  } else if (ctx->forcing) {
    ctx->cur = ctx->force;
  } else {
    auto it = ctx->tune.find(device_signature(ctx) + "|" + batch_signature(probs, count));
    ctx->cur = (it != ctx->tune.end()) ? it->second : sfft_ctx::Tier1();
  }
}

// Test hooks, read from the environment when a context is created. They only
// narrow limits or fail host calls; nothing faults or stalls the device.
//   SFFT_TIER1="build=8,round=6,cross=4,zipq=40,zipw=900"  tier-1 limits of the
//     two-tier launches (any subset), so that tests can force hand-offs
//   SFFT_FAULT="enomem:<workspace>[:<times>]"  that workspace's allocations
//     fail with SFFT_ENOMEM (every time, or the next <times> times)
//   SFFT_FAULT="jacobi:<sweeps>"  the SVDs of pricing calls stop after that
//     many Jacobi sweeps and report SFFT_ENOCONV when not converged
//   SFFT_FAULT="enoconv:<position>"  the builder result of that position among
//     a call's valid instances is replaced by SFFT_ENOCONV
// Several SFFT_FAULT items are separated by ';'.
//   SFFT_ZPRE=0  every instance's zip-up runs from site 0 instead of taking its
//     delta prefix from the MPO cache (tests compare the two)
void read_test_hooks(sfft_ctx* ctx) {
  if (const char* z = getenv("SFFT_ZPRE")) ctx->zpre_on = atoi(z) != 0;
  if (const char* t = getenv("SFFT_TIER1")) {
    ctx->t1_hooked = true;
    std::string str(t);
    size_t pos = 0;
    while (pos < str.size()) {
      size_t end = str.find(',', pos);
      if (end == std::string::npos) end = str.size();
      const std::string item = str.substr(pos, end - pos);
      const size_t eq = item.find('=');
      if (eq != std::string::npos) {
        const std::string key = item.substr(0, eq);
        const int v = atoi(item.c_str() + eq + 1);
        if (v > 0) {
          if (key == "build") ctx->t1.build_p = std::max(2, v);
          else if (key == "round") ctx->t1.round_r = v;
          else if (key == "cross") ctx->t1.cross_r = v;
          else if (key == "zipq") ctx->t1.zip_q = v;
          else if (key == "zipw") ctx->t1.zip_w = v;
        }
      }
      pos = end + 1;
    }
  }
  if (const char* f = getenv("SFFT_FAULT")) {
    std::string str(f);
    size_t pos = 0;
    while (pos < str.size()) {
      size_t end = str.find(';', pos);
      if (end == std::string::npos) end = str.size();
      const std::string item = str.substr(pos, end - pos);
      const size_t c1 = item.find(':');
      if (c1 != std::string::npos) {
        const std::string kind = item.substr(0, c1);
        const std::string rest = item.substr(c1 + 1);
        if (kind == "enomem") {
          const size_t c2 = rest.find(':');
          ctx->fault_enomem = rest.substr(0, c2);
          ctx->fault_enomem_left = (c2 == std::string::npos) ? -1 : std::max(0, atoi(rest.c_str() + c2 + 1));
        } else if (kind == "jacobi") {
          ctx->fault_jacobi = std::max(1, atoi(rest.c_str()));
        } else if (kind == "enoconv") {
          ctx->fault_enoconv = atoi(rest.c_str());
        }
      }
      pos = end + 1;
    }
  }
}

}  // namespace

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

const char* sfft_status_string(sfft_status s) {
  switch (s) {
    case SFFT_OK: return "ok";
    case SFFT_EINVAL: return "invalid argument";
    case SFFT_EMOMENT: return "damping moment E[S^(alpha+1)] is infinite";
    case SFFT_ENOMEM: return "out of memory";
    case SFFT_ECUDA: return "CUDA error";
    case SFFT_ERANK: return "rank cap reached";
    case SFFT_ENOCONV: return "integrand builder did not converge";
    case SFFT_ETIMEOUT: return "device wait timed out";
    case SFFT_EBOUNDS: return "prices outside the no-arbitrage bounds (grid too coarse for the damped integrand)";
  }
  return "unknown status";
}

const char* sfft_last_error(const sfft_ctx* ctx) { return ctx ? ctx->err.c_str() : "no context"; }

sfft_status sfft_create(sfft_ctx** out, int device) {
  if (!out) return SFFT_EINVAL;
  *out = nullptr;
  sfft_ctx* ctx = new sfft_ctx();
  ctx->device = device;
  cudaError_t e = cudaSetDevice(device);
  if (e != cudaSuccess) {
    delete ctx;
    return SFFT_ECUDA;
  }
  cudaDeviceProp prop;
  e = cudaGetDeviceProperties(&prop, device);
  if (e != cudaSuccess) {
    delete ctx;
    return SFFT_ECUDA;
  }
  ctx->num_sms = prop.multiProcessorCount;
  read_test_hooks(ctx);
  sfft_status s = set_smem_attrs(ctx);
  if (!s && (cudaStreamCreateWithFlags(&ctx->side, cudaStreamNonBlocking) != cudaSuccess ||
             cudaEventCreateWithFlags(&ctx->fork, cudaEventDisableTiming) != cudaSuccess ||
             cudaEventCreateWithFlags(&ctx->join, cudaEventDisableTiming) != cudaSuccess))
    s = SFFT_ECUDA;
  if (s) {
    sfft_destroy(ctx);
    return s;
  }
  *out = ctx;
  return SFFT_OK;
}

sfft_status sfft_destroy(sfft_ctx* ctx) {
  if (!ctx) return SFFT_OK;
  cudaSetDevice(ctx->device);
  cudaStreamSynchronize(ctx->stream);
  if (ctx->side) cudaStreamSynchronize(ctx->side);
  for (auto& kv : ctx->bufs) kv.second.release();
  for (auto& e : ctx->ev_open) {
    cudaEventDestroy(e.second.first);
    cudaEventDestroy(e.second.second);
  }
  for (auto e : ctx->ev_pool) cudaEventDestroy(e);
  if (ctx->fork) cudaEventDestroy(ctx->fork);
  if (ctx->join) cudaEventDestroy(ctx->join);
  if (ctx->side) cudaStreamDestroy(ctx->side);
  if (ctx->prof_acc) cudaFree(ctx->prof_acc);
  ctx->mpo_pool.release();
  ctx->mpo_ranks_dev.release();
  delete ctx;
  return SFFT_OK;
}

sfft_status sfft_set_stream(sfft_ctx* ctx, void* stream) {
  if (!ctx) return SFFT_EINVAL;
  ctx->stream = reinterpret_cast<cudaStream_t>(stream);
  return SFFT_OK;
}

struct GraphCapture;
static sfft_status price_common(sfft_ctx* ctx, const sfft_problem* probs, int32_t count,
                                const int64_t* l_begin, const int64_t* stride, const int32_t* q,
                                double* prices, double* log_strikes, int32_t* inst_status,
                                sfft_info* info, int mode, GraphCapture* gc = nullptr);


sfft_status sfft_tune_key(const sfft_problem* probs, int32_t count, char* buf, int32_t cap) {
  if (!probs || count < 1 || !buf || cap < 1) return SFFT_EINVAL;
  const std::string k = batch_signature(probs, count);
  if ((int)k.size() + 1 > cap) return SFFT_EINVAL;
  memcpy(buf, k.c_str(), k.size() + 1);
  return SFFT_OK;
}

static void to_tune(const sfft_ctx::Tier1& t, sfft_tune* out) {
  out->build_p = t.build_p;
  out->round_r = t.round_r;
  out->zip_ctas = t.zip_ctas;
}

sfft_status sfft_tune_lookup(sfft_ctx* ctx, const sfft_problem* probs, int32_t count, sfft_tune* cfg,
                             int32_t* found) {
  if (!ctx || !probs || count < 1 || !cfg) return SFFT_EINVAL;
  auto it = ctx->tune.find(device_signature(ctx) + "|" + batch_signature(probs, count));
  if (found) *found = it != ctx->tune.end();
  to_tune(it != ctx->tune.end() ? it->second : sfft_ctx::Tier1(), cfg);
  return SFFT_OK;
}

sfft_status sfft_tune_trials(const sfft_ctx* ctx, sfft_tune* cfgs, double* ms, int32_t cap, int32_t* n) {
  if (!ctx || cap < 0 || (cap > 0 && (!cfgs || !ms))) return SFFT_EINVAL;
  const int m = std::min<int>(cap, (int)ctx->trials.size());
  for (int i = 0; i < m; ++i) {
    to_tune(ctx->trials[i].first, cfgs + i);
    ms[i] = ctx->trials[i].second;
  }
  if (n) *n = (int32_t)ctx->trials.size();
  return SFFT_OK;
}

sfft_status sfft_tune_export(const sfft_ctx* ctx, char* buf, int64_t cap, int64_t* len) {
  if (!ctx) return SFFT_EINVAL;
  std::string out;
  for (const auto& kv : ctx->tune) {
    char line[64];
    snprintf(line, sizeof line, " %d %d %d\n", kv.second.build_p, kv.second.round_r, kv.second.zip_ctas);
    out += kv.first + line;
  }
  if (len) *len = (int64_t)out.size();
  if (!buf) return SFFT_OK;
  if ((int64_t)out.size() + 1 > cap) return SFFT_EINVAL;
  memcpy(buf, out.c_str(), out.size() + 1);
  return SFFT_OK;
}

sfft_status sfft_tune_import(sfft_ctx* ctx, const char* text) {
  if (!ctx || !text) return SFFT_EINVAL;
  const std::string all(text);
  size_t pos = 0;
  std::map<std::string, sfft_ctx::Tier1> add;
  while (pos < all.size()) {
    size_t end = all.find('\n', pos);
    if (end == std::string::npos) end = all.size();
    const std::string line = all.substr(pos, end - pos);
    pos = end + 1;
    if (line.empty()) continue;
    // "<device>|<batch> build_p round_r zip_ctas": the key holds spaces, the
    // three numbers are the last three fields
    size_t c3 = line.rfind(' ');
    size_t c2 = c3 == std::string::npos ? c3 : line.rfind(' ', c3 - 1);
    size_t c1 = c2 == std::string::npos ? c2 : line.rfind(' ', c2 - 1);
    if (c1 == std::string::npos || c1 == 0) return set_err(ctx, SFFT_EINVAL, "tune line: %s", line.c_str());
    sfft_ctx::Tier1 t;
    t.build_p = atoi(line.c_str() + c1 + 1);
    t.round_r = atoi(line.c_str() + c2 + 1);
    t.zip_ctas = atoi(line.c_str() + c3 + 1);
    if (t.build_p < 2 || t.build_p > 32 || t.round_r < 1 || t.round_r > 32 || t.zip_ctas < 0 || t.zip_ctas > 8)
      return set_err(ctx, SFFT_EINVAL, "tune values out of range: %s", line.c_str());
    add[line.substr(0, c1)] = t;
  }
  for (auto& kv : add) ctx->tune[kv.first] = kv.second;
  return SFFT_OK;
}

sfft_status sfft_autotune(sfft_ctx* ctx, const sfft_problem* probs, int32_t count, const int64_t* l_begin,
                          const int64_t* stride, const int32_t* q, double* prices, double* log_strikes,
                          int32_t reps, sfft_tune* chosen, double* ms_chosen, double* ms_default) {
  if (!ctx || !probs || count < 1 || reps < 1) return set_err(ctx, SFFT_EINVAL, "bad arguments");
  if (ctx->t1_hooked) return set_err(ctx, SFFT_EINVAL, "first-tier limits are fixed by SFFT_TIER1");
  if (ctx->prof) return set_err(ctx, SFFT_EINVAL, "turn profiling off before tuning");
  CK(cudaSetDevice(ctx->device));
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  std::vector<int32_t> st(count);
  auto run = [&](const sfft_ctx::Tier1& t, double* ms) -> sfft_status {
    ctx->forcing = true;
    ctx->force = t;
    double best = 1e300;
    sfft_status r = SFFT_OK;
    for (int k = 0; k < reps && r == SFFT_OK; ++k) {
      cudaEventRecord(e0, ctx->stream);
      r = price_common(ctx, probs, count, l_begin, stride, q, prices, log_strikes, st.data(), nullptr, 0);
      cudaEventRecord(e1, ctx->stream);
      cudaEventSynchronize(e1);
      float f = 0.f;
      cudaEventElapsedTime(&f, e0, e1);
      best = std::min(best, (double)f);
    }
    ctx->forcing = false;
    // a failing instance (EBOUNDS, EMOMENT, ...) does not stop the tuning
    if (r != SFFT_OK && r != SFFT_ECUDA && r != SFFT_ENOMEM && r != SFFT_EINVAL) r = SFFT_OK;
    *ms = best;
    if (r == SFFT_OK) ctx->trials.push_back({t, best});
    return r;
  };
  ctx->trials.clear();
  sfft_ctx::Tier1 def, best = def;
  double t_def = 0.0, t_best = 0.0, t = 0.0;
  sfft_status s = run(def, &t_def);  // the first run also builds the batch's operators
  ctx->trials.clear();
  if (s == SFFT_OK) s = run(def, &t_def);
  t_best = t_def;
  // coordinate descent over the first-tier carves: zip-up CTAs per SM, the
  // builder's panel width, the output rounding's rank
  const int zips[] = {2};
  const int builds[] = {24, 16};
  const int rounds[] = {20, 16};
  for (int z : zips) {
    sfft_ctx::Tier1 c = best;
    c.zip_ctas = z;
    if (s == SFFT_OK && (s = run(c, &t)) == SFFT_OK && t < t_best) { best = c; t_best = t; }
  }
  for (int bp : builds) {
    sfft_ctx::Tier1 c = best;
    c.build_p = bp;
    if (s == SFFT_OK && (s = run(c, &t)) == SFFT_OK && t < t_best) { best = c; t_best = t; }
  }
  for (int rr : rounds) {
    sfft_ctx::Tier1 c = best;
    c.round_r = rr;
    if (s == SFFT_OK && (s = run(c, &t)) == SFFT_OK && t < t_best) { best = c; t_best = t; }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (s != SFFT_OK) return s;
  ctx->tune[device_signature(ctx) + "|" + batch_signature(probs, count)] = best;
  if (chosen) to_tune(best, chosen);
  if (ms_chosen) *ms_chosen = t_best;
  if (ms_default) *ms_default = t_def;
  return SFFT_OK;
}

sfft_status sfft_set_precision(sfft_ctx* ctx, int32_t precision) {
  if (!ctx || (precision != SFFT_PRECISION_FP64 && precision != SFFT_PRECISION_MIXED)) return SFFT_EINVAL;
  ctx->precision = precision;
  return SFFT_OK;
}

sfft_status sfft_tier2_counts(sfft_ctx* ctx, int32_t* counts) {
  if (!ctx || !counts) return SFFT_EINVAL;
  CK(cudaSetDevice(ctx->device));
  for (int k = 0; k < 4; ++k) {
    counts[k] = 0;
    if (ctx->defer_heads[k])
      CK(cudaMemcpyAsync(counts + k, ctx->defer_heads[k], sizeof(int32_t), cudaMemcpyDeviceToHost, ctx->stream));
  }
  CK(cudaStreamSynchronize(ctx->stream));
  return SFFT_OK;
}

sfft_status sfft_strike_window(const sfft_problem* prob, double lo, double hi, int32_t qmax,
                               int64_t* l_begin, int64_t* stride, int32_t* q) {
  if (!prob || !l_begin || !stride || !q || qmax < 1 || !(lo <= hi)) return SFFT_EINVAL;
  InstParams P;
  sfft_status s = plan(nullptr, *prob, &P);
  if (s != SFFT_OK && s != SFFT_EMOMENT) return s;
  const long long M = 1LL << P.n;
  long long u_lo = (long long)ceil((lo - P.k0) / P.dk - 1e-9);
  long long u_hi = (long long)floor((hi - P.k0) / P.dk + 1e-9);
  u_lo = std::max(u_lo, 0LL);
  u_hi = std::min(u_hi, M - 1);
  long long st = 1;
  for (;;) {
    const long long first = ((u_lo + st - 1) / st) * st;
    const long long cnt = (u_hi >= first) ? (u_hi - first) / st + 1 : 0;
    if (cnt <= qmax) {
      *l_begin = first;
      *stride = st;
      *q = (int32_t)cnt;
      return SFFT_OK;
    }
    st *= 2;
  }
}

sfft_status sfft_sample_integrand(sfft_ctx* ctx, const sfft_problem* prob, const int64_t* j,
                                  int64_t count, double* x) {
  if (!ctx || !prob || count < 0 || (count > 0 && (!j || !x))) return set_err(ctx, SFFT_EINVAL, "bad arguments");
  ctx->err.clear();
  CK(cudaSetDevice(ctx->device));
  InstParams P;
  sfft_status s = plan(ctx, *prob, &P);
  if (s) return s;
  if (count == 0) return SFFT_OK;
  void* pd;
  if ((s = ensure(ctx, "sample_P", sizeof(InstParams), &pd))) return s;
  CK(cudaMemcpyAsync(pd, &P, sizeof P, cudaMemcpyHostToDevice, ctx->stream));
  const int grid = (int)std::min<long long>((count + kThreads - 1) / kThreads, 148LL * 16);
  k_sample<<<grid, kThreads, 0, ctx->stream>>>(reinterpret_cast<InstParams*>(pd),
                                               reinterpret_cast<const long long*>(j), count,
                                               reinterpret_cast<cd*>(x));
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(ctx->stream));
  return SFFT_OK;
}

sfft_status sfft_mpo(sfft_ctx* ctx, int32_t n, double tol, int32_t* ranks, double* cores, int64_t cap) {
  if (!ctx || n < 1 || n > SFFT_MAX_N || !(tol > 0.0 && tol < 1.0) || !ranks || !cores)
    return set_err(ctx, SFFT_EINVAL, "bad arguments");
  ctx->err.clear();
  CK(cudaSetDevice(ctx->device));
  const MpoEntry* e;
  sfft_status s = get_mpo(ctx, n, tol, &e);
  if (s) return s;
  const int idx = e->idx;
  return copy_tt_out(ctx, reinterpret_cast<const cd*>(ctx->mpo_pool.p) + e->off,
                     reinterpret_cast<const int*>(ctx->mpo_ranks_dev.p) + (SFFT_MAX_N + 1) * idx, n, 4,
                     SFFT_CORE_STRIDE_D4, ranks, cores, cap);
}

sfft_status sfft_integrand_tt(sfft_ctx* ctx, const sfft_problem* prob, int32_t* ranks, double* cores,
                              int64_t cap) {
  if (!ctx || !prob || !ranks || !cores) return set_err(ctx, SFFT_EINVAL, "bad arguments");
  ctx->err.clear();
  CK(cudaSetDevice(ctx->device));
  std::vector<InstParams> prm(1);
  sfft_status s = plan(ctx, *prob, &prm[0]);
  if (s) return s;
  Batch b;
  ctx->cur = ctx->t1_hooked ? ctx->t1 : sfft_ctx::Tier1();
  if ((s = run_tt_path(ctx, prm, b, nullptr, false))) return s;
  int st = 0;
  CK(cudaMemcpyAsync(&st, b.status, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  if (st) return set_err(ctx, (sfft_status)st, "integrand TT: %s", sfft_status_string((sfft_status)st));
  return copy_tt_out(ctx, b.A, b.a_ranks, prm[0].n, 2, SFFT_CORE_STRIDE_D2, ranks, cores, cap);
}

sfft_status sfft_tt_round(sfft_ctx* ctx, int32_t n, int32_t d, const int32_t* in_ranks,
                          const double* in_cores, double tol, int32_t max_rank, int32_t* out_ranks,
                          double* out_cores, int64_t cap) {
  if (!ctx || n < 1 || n > SFFT_MAX_N || (d != 2 && d != 4) || !in_ranks || !in_cores || !out_ranks ||
      !out_cores || !(tol > 0.0 && tol < 1.0) || max_rank < 0 || max_rank > SFFT_MAX_RANK)
    return set_err(ctx, SFFT_EINVAL, "bad arguments");
  ctx->err.clear();
  CK(cudaSetDevice(ctx->device));
  void* p;
  sfft_status s;
  const int stride = (d == 2) ? SFFT_CORE_STRIDE_D2 : SFFT_CORE_STRIDE_D4;
  if ((s = ensure(ctx, "rt_tt", sizeof(cd) * (size_t)n * stride, &p))) return s;
  cd* T = reinterpret_cast<cd*>(p);
  void* rd;
  if ((s = ensure(ctx, "rt_ranks", sizeof(int) * (SFFT_MAX_N + 1), &rd))) return s;
  if ((s = copy_tt_in(ctx, in_cores, in_ranks, n, d, stride, T, reinterpret_cast<int*>(rd)))) return s;
  std::vector<int> nv(1, n), mr(1, max_rank ? max_rank : SFFT_DEFAULT_MAX_RANK), st0(1, 0);
  std::vector<double> tv(1, tol);
  std::vector<long long> off(1, 0);
  int *nd, *md, *sd;
  double* td;
  long long* od;
  if ((s = upload(ctx, "rt_n", nv, &nd)) || (s = upload(ctx, "rt_m", mr, &md)) ||
      (s = upload(ctx, "rt_tol", tv, &td)) || (s = upload(ctx, "rt_off", off, &od)) ||
      (s = upload(ctx, "rt_st", st0, &sd)))
    return s;
  void* scr;
  if ((s = ensure(ctx, "rt_scratch", sizeof(cd) * SFFT_ROUND_SCRATCH, &scr))) return s;
  const RoundSmem rs = round_smem(d);
  k_tt_round<<<1, kThreads, rs.bytes, ctx->stream>>>(nullptr, 1, nullptr, nd, d, 1, td, md, T, od, stride,
                                                    reinterpret_cast<int*>(rd), reinterpret_cast<cd*>(scr),
                                                    SFFT_ROUND_SCRATCH, sd, rs.hb, nullptr, PH_ROUND, rs.pmax,
                                                    rs.vcap, nullptr, nullptr);
  CK(cudaGetLastError());
  int st = 0;
  CK(cudaMemcpyAsync(&st, sd, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  if (st) return set_err(ctx, (sfft_status)st, "rounding: %s", sfft_status_string((sfft_status)st));
  return copy_tt_out(ctx, T, reinterpret_cast<int*>(rd), n, d, stride, out_ranks, out_cores, cap);
}

sfft_status sfft_tt_apply_qft(sfft_ctx* ctx, int32_t n, const int32_t* in_ranks, const double* in_cores,
                              double tol, int32_t max_rank, int32_t* out_ranks, double* out_cores,
                              int64_t cap) {
  if (!ctx || n < 1 || n > SFFT_MAX_N || !in_ranks || !in_cores || !out_ranks || !out_cores ||
      !(tol > 0.0 && tol < 1.0) || max_rank < 0 || max_rank > SFFT_MAX_RANK)
    return set_err(ctx, SFFT_EINVAL, "bad arguments");
  ctx->err.clear();
  CK(cudaSetDevice(ctx->device));
  const MpoEntry* e;
  sfft_status s = get_mpo(ctx, n, tol, &e);
  if (s) return s;
  void* p;
  if ((s = ensure(ctx, "ap_A", sizeof(cd) * (size_t)n * SFFT_CORE_STRIDE_D2, &p))) return s;
  cd* A = reinterpret_cast<cd*>(p);
  if ((s = ensure(ctx, "ap_B", sizeof(cd) * (size_t)n * SFFT_CORE_STRIDE_D2, &p))) return s;
  cd* B = reinterpret_cast<cd*>(p);
  void *ra, *rb, *rw;
  if ((s = ensure(ctx, "ap_ra", sizeof(int) * (SFFT_MAX_N + 1), &ra)) ||
      (s = ensure(ctx, "ap_rb", sizeof(int) * (SFFT_MAX_N + 1), &rb)) ||
      (s = ensure(ctx, "ap_rw", sizeof(int) * (SFFT_MAX_N + 1), &rw)))
    return s;
  if ((s = copy_tt_in(ctx, in_cores, in_ranks, n, 2, SFFT_CORE_STRIDE_D2, A, reinterpret_cast<int*>(ra))))
    return s;
  CK(cudaMemcpyAsync(rw, e->ranks.data(), sizeof(int) * (SFFT_MAX_N + 1), cudaMemcpyHostToDevice, ctx->stream));
  std::vector<int> nv(1, n), mr(1, max_rank ? max_rank : SFFT_DEFAULT_MAX_RANK), st0(1, 0);
  std::vector<double> tv(1, tol);
  std::vector<long long> off(1, 0), woff(1, e->off);
  int *nd, *md, *sd;
  double* td;
  long long *od, *wd;
  if ((s = upload(ctx, "ap_n", nv, &nd)) || (s = upload(ctx, "ap_m", mr, &md)) ||
      (s = upload(ctx, "ap_tol", tv, &td)) || (s = upload(ctx, "ap_off", off, &od)) ||
      (s = upload(ctx, "ap_woff", woff, &wd)) || (s = upload(ctx, "ap_st", st0, &sd)))
    return s;
  void* scr;
  if ((s = ensure(ctx, "ap_scratch", sizeof(cd) * (size_t)(SFFT_ZIP_SCRATCH + SFFT_ROUND_SCRATCH), &scr)))
    return s;
  const RoundSmem zs = zip_smem();
  k_zipup<<<1, kThreads, zs.bytes, ctx->stream>>>(
      nullptr, 1, nullptr, nd, td, md, A, od, reinterpret_cast<int*>(ra), reinterpret_cast<const cd*>(ctx->mpo_pool.p), wd,
      reinterpret_cast<int*>(rw), B, od, reinterpret_cast<int*>(rb), SFFT_CORE_STRIDE_D2,
      SFFT_CORE_STRIDE_D4, SFFT_CORE_STRIDE_D2, reinterpret_cast<cd*>(scr), SFFT_ZIP_SCRATCH, sd, zs.hb,
      nullptr, zs.vcap, nullptr, nullptr, LA_MAXQ, 1 << 30, ZipPrefix{});
  CK(cudaGetLastError());
  const RoundSmem rs = round_smem(2, false);
  k_tt_round<<<1, kThreads, rs.bytes, ctx->stream>>>(nullptr, 1, nullptr, nd, 2, 0, td, md, B, od,
                                                    SFFT_CORE_STRIDE_D2, reinterpret_cast<int*>(rb),
                                                    reinterpret_cast<cd*>(scr), SFFT_ROUND_SCRATCH, sd, rs.hb,
                                                    nullptr, PH_ROUND, rs.pmax, rs.vcap, nullptr, nullptr);
  CK(cudaGetLastError());
  int st = 0;
  CK(cudaMemcpyAsync(&st, sd, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  if (st) return set_err(ctx, (sfft_status)st, "apply: %s", sfft_status_string((sfft_status)st));
  return copy_tt_out(ctx, B, reinterpret_cast<int*>(rb), n, 2, SFFT_CORE_STRIDE_D2, out_ranks, out_cores, cap);
}

// What a captured pricing call leaves for reading its statuses later.
struct GraphCapture {
  Batch b;
  std::vector<int> valid, host_status;
  std::vector<const MpoEntry*> mp;
};

static sfft_status price_common(sfft_ctx* ctx, const sfft_problem* probs, int32_t count,
                                const int64_t* l_begin, const int64_t* stride, const int32_t* q,
                                double* prices, double* log_strikes, int32_t* inst_status,
                                sfft_info* info, int mode, GraphCapture* gc) {
  // mode 0: TT-SFFT; 1: dense-FFT baseline; 2: QFT route by statevector emulation
  const bool dense = mode != 0;
  if (!ctx || count < 0 || (count > 0 && (!probs || !l_begin || !stride || !q)))
    return set_err(ctx, SFFT_EINVAL, "bad arguments");
  ctx->err.clear();
  CK(cudaSetDevice(ctx->device));
  std::vector<int> host_status(count, 0), tbits(count, 0);
  std::vector<long long> out_off(count, 0);
  long long tot_q = 0;
  for (int i = 0; i < count; ++i) {
    out_off[i] = tot_q;
    tot_q += std::max(q[i], 0);
  }
  if (tot_q > 0 && (!prices || !log_strikes)) return set_err(ctx, SFFT_EINVAL, "output buffers are NULL");
  std::vector<InstParams> prm;
  std::vector<int> valid;
  std::vector<long long> lb_v, off_v;
  std::vector<int> tb_v, q_v;
  for (int i = 0; i < count; ++i) {
    InstParams P;
    sfft_status s = plan(ctx, probs[i], &P);
    if (s == SFFT_OK) s = check_strikes(ctx, probs[i].n, l_begin[i], stride[i], q[i], &tbits[i]);
    if (s == SFFT_OK && dense && probs[i].n > SFFT_DENSE_MAX_N)
      s = set_err(ctx, SFFT_EINVAL, "dense and statevector routes limited to n <= %d", SFFT_DENSE_MAX_N);
    // the positive-phase readout needs the symmetric grid: on the one-sided
    // Simpson grid the discretised sum has a genuine imaginary part
    if (s == SFFT_OK && mode == 2 && probs[i].quad != SFFT_QUAD_RECT_SYM)
      s = set_err(ctx, SFFT_EINVAL, "the QFT route needs the symmetric grid (SFFT_QUAD_RECT_SYM)");
    host_status[i] = s;
    if (s != SFFT_OK) continue;
    valid.push_back(i);
    prm.push_back(P);
    lb_v.push_back(l_begin[i]);
    off_v.push_back(out_off[i]);
    tb_v.push_back(tbits[i]);
    q_v.push_back(q[i]);
  }
  // prices of rejected instances are NaN: every byte 0xFF makes the double
  // 0xFFFFFFFFFFFFFFFF, a quiet NaN, for any q (a rejected q may exceed
  // SFFT_MAX_STRIKES)
  for (int i = 0; i < count; ++i)
    if (host_status[i] != SFFT_OK && q[i] > 0)
      CK(cudaMemsetAsync(prices + out_off[i], 0xFF, sizeof(double) * (size_t)q[i], ctx->stream));
  const int cnt = (int)prm.size();
  if (cnt == 0) return finish_status(ctx, count, valid, host_status, nullptr, inst_status, info, nullptr, nullptr);
  sfft_status s;
  if (dense) {
    // one instance at a time, whole GPU per instance
    int maxn = 1;
    for (auto& P : prm) maxn = std::max(maxn, P.n);
    void* xb;
    if ((s = ensure(ctx, "dense_x", sizeof(cd) * (1ULL << maxn), &xb))) return s;
    int* st_dev;
    void* p;
    if ((s = ensure(ctx, "status", sizeof(int) * cnt, &p))) return s;
    st_dev = reinterpret_cast<int*>(p);
    CK(cudaMemsetAsync(st_dev, 0, sizeof(int) * cnt, ctx->stream));
    void* dg;
    if ((s = ensure(ctx, "dense_digits", sizeof(int) * 16, &dg))) return s;
    const int nparts = ctx->num_sms * 8;
    double* nrm_part = nullptr;
    if (mode == 2) {
      void* np;
      if ((s = ensure(ctx, "qft_norm", sizeof(double) * (nparts + 1), &np))) return s;
      nrm_part = reinterpret_cast<double*>(np);
    }
    for (int k = 0; k < cnt; ++k) {
      const InstParams& P = prm[k];
      const long long M = 1LL << P.n;
      cd* x = reinterpret_cast<cd*>(xb);
      // all samples first, in index order, so that every FFT pass is the
      // transform alone (fused into the first pass they cost the same); the
      // statevector route then normalises them
      {
        PhaseScope ps(ctx, PH_DENSE_SAMPLE);
        k_dense_sample<<<ctx->num_sms * 8, kThreads, 0, ctx->stream>>>(P, x, M);
      }
      CK(cudaGetLastError());
      if (mode == 2) {
        // amplitude encoding: x <- x / ||x|| (Eq. qft_input_state)
        PhaseScope ps(ctx, PH_DENSE_SAMPLE);
        k_norm2_partial<<<nparts, kThreads, 0, ctx->stream>>>(x, M, nrm_part);
        k_norm2_final<<<1, 32, 0, ctx->stream>>>(nrm_part, nparts, nrm_part + nparts);
        k_scale_unit<<<ctx->num_sms * 8, kThreads, 0, ctx->stream>>>(x, M, nrm_part + nparts);
        CK(cudaGetLastError());
      }
      // passes of at most 2^10-point sub-transforms, digits as even as possible
      const int npass = (P.n + 9) / 10;
      std::vector<int> dig(npass);
      int left = P.n;
      for (int pp = 0; pp < npass; ++pp) {
        dig[pp] = (left + (npass - pp) - 1) / (npass - pp);
        left -= dig[pp];
      }
      long long L = M;
      for (int pp = 0; pp < npass; ++pp) {
        const int R = dig[pp];
        const long long Lp = L >> R;
        // columns per block: adjacent offsets s, or in the last pass (Lp = 1)
        // adjacent sub-transforms
        const int cols = (int)std::min<long long>(Lp == 1 ? (M >> R) : Lp, std::max(1, 2048 >> R));
        const size_t smem = sizeof(cd) * ((size_t)(1 << R) * cols + (1 << R) + 64 * (size_t)cols);
        const long long nblk = Lp == 1 ? (M / L) / cols : (M / L) * (Lp / cols);
        const int grid =
            (int)std::min<long long>(nblk, (long long)ctx->num_sms * blocks_per_sm((const void*)k_fft_pass, smem));
        {
          PhaseScope ps(ctx, PH_DENSE_FFT);
          k_fft_pass<<<grid, kThreads, smem, ctx->stream>>>(x, M, Lp, R, cols);
        }
        CK(cudaGetLastError());
        L = Lp;
      }
      CK(cudaMemcpyAsync(dg, dig.data(), sizeof(int) * npass, cudaMemcpyHostToDevice, ctx->stream));
      if (q_v[k] > 0) {
        PhaseScope ps(ctx, PH_DENSE_GATHER);
        if (mode == 2)
          k_qft_gather<<<(q_v[k] + kThreads - 1) / kThreads, kThreads, 0, ctx->stream>>>(
              P, x, P.n, reinterpret_cast<int*>(dg), npass, lb_v[k], tb_v[k], q_v[k], nrm_part + nparts,
              prices + off_v[k], log_strikes + off_v[k]);
        else
          k_dense_gather<<<(q_v[k] + kThreads - 1) / kThreads, kThreads, 0, ctx->stream>>>(
              P, x, P.n, reinterpret_cast<int*>(dg), npass, lb_v[k], tb_v[k], q_v[k], prices + off_v[k],
              log_strikes + off_v[k]);
        CK(cudaGetLastError());
      }
    }
    return finish_status(ctx, count, valid, host_status, st_dev, inst_status, info, nullptr, nullptr);
  }
  {
    std::vector<std::pair<int, double>> want;
    for (const auto& P : prm) want.push_back({P.n, P.tol});
    if ((s = build_mpos(ctx, want))) return s;
  }
  std::vector<const MpoEntry*> mp(cnt);
  for (int k = 0; k < cnt; ++k) {
    if ((s = get_mpo(ctx, prm[k].n, prm[k].tol, &mp[k]))) return s;
  }
  Batch b;
  choose_tier1(ctx, probs, count);
  if (ctx->fault_jacobi > 0) CK(sfft_set_jacobi_cap(ctx->fault_jacobi, ctx->stream));
  s = run_tt_path(ctx, prm, b, &mp, true);
  if (ctx->fault_jacobi > 0) CK(sfft_set_jacobi_cap(60, ctx->stream));
  if (s) return s;
  long long* lb_d;
  long long* off_d;
  int *tb_d, *q_d;
  if ((s = upload(ctx, "lb", lb_v, &lb_d)) || (s = upload(ctx, "outoff", off_v, &off_d)) ||
      (s = upload(ctx, "tb", tb_v, &tb_d)) || (s = upload(ctx, "qv", q_v, &q_d)))
    return s;
  void* p;
  const int grid = std::min(cnt, ctx->num_sms * 4);
  if ((s = ensure(ctx, "readout_scratch", sizeof(cd) * (size_t)SFFT_READOUT_SCRATCH * grid, &p))) return s;
  {
    PhaseScope ps(ctx, PH_READOUT);
    k_readout<<<grid, kThreads, 0, ctx->stream>>>(b.all_list, cnt, b.counters + 5, b.P, b.B, b.a_off, b.b_ranks, SFFT_CORE_STRIDE_D2,
                                                  lb_d, tb_d, q_d, off_d, prices, log_strikes, b.status,
                                                  reinterpret_cast<cd*>(p), SFFT_READOUT_SCRATCH);
  }
  CK(cudaGetLastError());
  if (gc) {  // being captured: the statuses are read after each replay
    gc->b = b;
    gc->valid = valid;
    gc->host_status = host_status;
    gc->mp = mp;
    return SFFT_OK;
  }
  return finish_status(ctx, count, valid, host_status, b.status, inst_status, info, &b, &mp);
}

sfft_status sfft_calibrate_fp64(sfft_ctx* ctx, double* gflops) {
  if (!ctx || !gflops) return SFFT_EINVAL;
  CK(cudaSetDevice(ctx->device));
  void* p;
  sfft_status s = ensure(ctx, "calib", 64, &p);
  if (s) return s;
  const int grid = ctx->num_sms * 8, iters = 1 << 14;
  cudaEvent_t a = take_event(ctx), b = take_event(ctx);
  k_dfma_peak<<<grid, kThreads, 0, ctx->stream>>>(reinterpret_cast<double*>(p), 256);  // warm-up
  CK(cudaEventRecord(a, ctx->stream));
  k_dfma_peak<<<grid, kThreads, 0, ctx->stream>>>(reinterpret_cast<double*>(p), iters);
  CK(cudaEventRecord(b, ctx->stream));
  CK(cudaGetLastError());
  CK(cudaEventSynchronize(b));
  float ms = 0.f;
  CK(cudaEventElapsedTime(&ms, a, b));
  ctx->ev_pool.push_back(a);
  ctx->ev_pool.push_back(b);
  *gflops = 16.0 * iters * (double)grid * kThreads / (ms * 1e-3) / 1e9;
  return SFFT_OK;
}

sfft_status sfft_profile_enable(sfft_ctx* ctx, int32_t on) {
  if (!ctx) return SFFT_EINVAL;
  CK(cudaSetDevice(ctx->device));
  if (on && !ctx->prof_acc) {
    CK(cudaMalloc(reinterpret_cast<void**>(&ctx->prof_acc), sizeof(double) * 2 * SFFT_NPHASE_DEV));
    CK(cudaMemset(ctx->prof_acc, 0, sizeof(double) * 2 * SFFT_NPHASE_DEV));
  }
  ctx->prof = on != 0;
  return SFFT_OK;
}

sfft_status sfft_profile_read(sfft_ctx* ctx, double* ms, double* flops, double* evals,
                              int64_t* launches, int32_t reset) {
  if (!ctx) return SFFT_EINVAL;
  CK(cudaSetDevice(ctx->device));
  CK(cudaStreamSynchronize(ctx->stream));
  for (auto& e : ctx->ev_open) {
    float t = 0.f;
    CK(cudaEventElapsedTime(&t, e.second.first, e.second.second));
    ctx->prof_ms[e.first] += t;
    ctx->prof_launches[e.first] += 1;
    ctx->ev_pool.push_back(e.second.first);
    ctx->ev_pool.push_back(e.second.second);
  }
  ctx->ev_open.clear();
  double host[2 * SFFT_NPHASE_DEV] = {0};
  if (ctx->prof_acc)
    CK(cudaMemcpy(host, ctx->prof_acc, sizeof host, cudaMemcpyDeviceToHost));
  for (int i = 0; i < SFFT_NPHASE_DEV; ++i) {
    if (ms) ms[i] = ctx->prof_ms[i];
    if (launches) launches[i] = ctx->prof_launches[i];
    if (flops) flops[i] = host[i];
    if (evals) evals[i] = host[SFFT_NPHASE_DEV + i];
  }
  if (reset) {
    for (int i = 0; i < SFFT_NPHASE_DEV; ++i) {
      ctx->prof_ms[i] = 0.0;
      ctx->prof_launches[i] = 0;
    }
    if (ctx->prof_acc) CK(cudaMemset(ctx->prof_acc, 0, sizeof(double) * 2 * SFFT_NPHASE_DEV));
  }
  return SFFT_OK;
}

sfft_status sfft_price_batch(sfft_ctx* ctx, const sfft_problem* probs, int32_t count, const int64_t* l_begin,
                             const int64_t* stride, const int32_t* q, double* prices, double* log_strikes,
                             int32_t* inst_status, sfft_info* info) {
  return price_common(ctx, probs, count, l_begin, stride, q, prices, log_strikes, inst_status, info, 0);
}

sfft_status sfft_dense_price_batch(sfft_ctx* ctx, const sfft_problem* probs, int32_t count,
                                   const int64_t* l_begin, const int64_t* stride, const int32_t* q,
                                   double* prices, double* log_strikes, int32_t* inst_status,
                                   sfft_info* info) {
  return price_common(ctx, probs, count, l_begin, stride, q, prices, log_strikes, inst_status, info, 1);
}

sfft_status sfft_qft_price_batch(sfft_ctx* ctx, const sfft_problem* probs, int32_t count,
                                 const int64_t* l_begin, const int64_t* stride, const int32_t* q,
                                 double* prices, double* log_strikes, int32_t* inst_status,
                                 sfft_info* info) {
  return price_common(ctx, probs, count, l_begin, stride, q, prices, log_strikes, inst_status, info, 2);
}


// ---------------------------------------------------------------------------
// Captured batches (CUDA graphs)
// ---------------------------------------------------------------------------
struct sfft_graph {
  sfft_ctx* own = nullptr;  // private context: its buffers never move while the graph lives
  cudaGraph_t g = nullptr;
  cudaGraphExec_t ge = nullptr;
  sfft_ctx::Stage stage;
  int count = 0;
  std::vector<sfft_problem> probs;
  GraphCapture gc;
  cudaStream_t last = nullptr;
  bool launched = false;
};

sfft_status sfft_graph_destroy(sfft_graph* g) {
  if (!g) return SFFT_OK;
  if (g->own) cudaSetDevice(g->own->device);
  if (g->launched) cudaStreamSynchronize(g->last);
  if (g->ge) cudaGraphExecDestroy(g->ge);
  if (g->g) cudaGraphDestroy(g->g);
  if (g->stage.base) cudaFreeHost(g->stage.base);
  if (g->own) sfft_destroy(g->own);
  delete g;
  return SFFT_OK;
}

sfft_status sfft_graph_create(sfft_ctx* ctx, const sfft_problem* probs, int32_t count,
                              const int64_t* l_begin, const int64_t* stride, const int32_t* q,
                              double* prices, double* log_strikes, sfft_graph** out) {
  if (!ctx || !out || count < 1 || !probs || !l_begin || !stride || !q || !prices || !log_strikes)
    return set_err(ctx, SFFT_EINVAL, "bad arguments");
  *out = nullptr;
  if (ctx->prof) return set_err(ctx, SFFT_EINVAL, "turn profiling off before capturing a graph");
  sfft_graph* g = new sfft_graph;
  g->count = count;
  g->probs.assign(probs, probs + count);
  sfft_status s = sfft_create(&g->own, ctx->device);
  if (s) {
    delete g;
    return set_err(ctx, s, "graph: context creation failed");
  }
  // the private context prices as the caller's does
  g->own->precision = ctx->precision;
  g->own->t1 = ctx->t1;
  g->own->t1_hooked = ctx->t1_hooked;
  g->own->tune = ctx->tune;
  // 1. a plain run sizes every workspace and builds the MPOs
  std::vector<int32_t> st(count);
  s = price_common(g->own, probs, count, l_begin, stride, q, prices, log_strikes, st.data(), nullptr, 0);
  // SFFT_EBOUNDS means computed, outside the bounds: its prices are written
  // on every replay and sfft_graph_status reports it
  if (s == SFFT_EBOUNDS) s = SFFT_OK;
  for (int i = 0; s == SFFT_OK && i < count; ++i)
    if (st[i] != SFFT_OK && st[i] != SFFT_EBOUNDS) s = (sfft_status)st[i];
  if (s) {
    set_err(ctx, s, "graph: every instance must price (%s)", g->own->err.c_str());
    sfft_graph_destroy(g);
    return s;
  }
  // 2. capture the same call on a private stream, uploads staged in pinned memory
  g->stage.cap = (size_t)count * 2048 + (1 << 20);
  if (cudaMallocHost(reinterpret_cast<void**>(&g->stage.base), g->stage.cap) != cudaSuccess) {
    sfft_graph_destroy(g);
    return set_err(ctx, SFFT_ENOMEM, "graph: pinned staging arena");
  }
  cudaStream_t cs;
  if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) {
    sfft_graph_destroy(g);
    return set_err(ctx, SFFT_ECUDA, "graph: stream creation");
  }
  cudaStream_t keep = g->own->stream;
  g->own->stream = cs;
  g->own->stage = &g->stage;
  cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    s = price_common(g->own, probs, count, l_begin, stride, q, prices, log_strikes, nullptr, nullptr, 0,
                     &g->gc);
    const cudaError_t e2 = cudaStreamEndCapture(cs, &g->g);
    if (s == SFFT_OK && e2 != cudaSuccess) s = SFFT_ECUDA;
  } else {
    s = SFFT_ECUDA;
  }
  g->own->stage = nullptr;
  g->own->stream = keep;
  cudaStreamDestroy(cs);
  if (s == SFFT_OK && cudaGraphInstantiate(&g->ge, g->g, 0) != cudaSuccess) s = SFFT_ECUDA;
  if (s) {
    set_err(ctx, s, "graph: capture failed (%s)", g->own->err.c_str());
    cudaGetLastError();
    sfft_graph_destroy(g);
    return s;
  }
  *out = g;
  return SFFT_OK;
}

sfft_status sfft_graph_launch(sfft_graph* g, void* stream) {
  if (!g) return SFFT_EINVAL;
  sfft_ctx* ctx = g->own;
  CK(cudaSetDevice(ctx->device));
  cudaStream_t sm = reinterpret_cast<cudaStream_t>(stream);
  if (g->launched && g->last != sm) CK(cudaStreamSynchronize(g->last));
  CK(cudaGraphLaunch(g->ge, sm));
  g->last = sm;
  g->launched = true;
  return SFFT_OK;
}

sfft_status sfft_graph_update(sfft_graph* g, const sfft_problem* probs) {
  if (!g || !probs) return SFFT_EINVAL;
  sfft_ctx* ctx = g->own;
  CK(cudaSetDevice(ctx->device));
  std::vector<InstParams> prm(g->count);
  for (int i = 0; i < g->count; ++i) {
    const sfft_problem& a = g->probs[i];
    const sfft_problem& b = probs[i];
    if (a.n != b.n || a.tol != b.tol || a.quad != b.quad || a.max_rank != b.max_rank ||
        (isnan(a.k0) != isnan(b.k0)) || (!isnan(a.k0) && a.k0 != b.k0))
      return set_err(ctx, SFFT_EINVAL, "instance %d: n, tol, quad, max_rank and k0 are fixed by the graph", i);
    sfft_status s = plan(ctx, b, &prm[i]);
    if (s) return s;
  }
  if (sizeof(InstParams) * prm.size() != g->stage.p_bytes)
    return set_err(ctx, SFFT_EINVAL, "graph: parameter block size changed");
  // the previous replay may still be reading the arena
  if (g->launched) CK(cudaStreamSynchronize(g->last));
  memcpy(g->stage.base + g->stage.p_off, prm.data(), g->stage.p_bytes);
  for (int i = 0; i < g->count; ++i) g->probs[i] = probs[i];
  return SFFT_OK;
}

sfft_status sfft_graph_status(sfft_graph* g, int32_t* inst_status, sfft_info* info) {
  if (!g) return SFFT_EINVAL;
  sfft_ctx* ctx = g->own;
  if (!g->launched) return set_err(ctx, SFFT_EINVAL, "graph not launched yet");
  CK(cudaSetDevice(ctx->device));
  cudaStream_t keep = g->own->stream;
  g->own->stream = g->last;
  const sfft_status s = finish_status(g->own, g->count, g->gc.valid, g->gc.host_status, g->gc.b.status,
                                      inst_status, info, &g->gc.b, &g->gc.mp);
  g->own->stream = keep;
  return s;
}

const char* sfft_graph_last_error(const sfft_graph* g) { return (g && g->own) ? g->own->err.c_str() : ""; }

}  // extern "C"
