// TT-SFFT kernels for sm_103a: integrand TT (TT-SVD of the sampled support
// block), Q_n MPO generator, zip-up MPO x TT contraction, TT rounding and the
// bit-reversed readout of prices (Sec. 3 of the paper).
//
// Storage: each TT (or MPO, d = 4) of an instance occupies n "core slots" of
// core_stride complex elements; core s (0-based site, site s+1 of the paper)
// of shape (r_s, d, r_{s+1}) is stored compactly, index [a][sigma][b] at
// a*d*r_{s+1} + sigma*r_{s+1} + b. Ranks live in an int array of n+1 entries.
// Site s carries bit (n-1-s) of the input index j (most significant first,
// Eq. discretized_x) and bit s of the output index u after Q_n (Sec. 3.2).
//
// One CTA works on one instance at a time (grid-stride over the batch); the
// site sweeps are sequential, the dense algebra inside a site is spread over
// the CTA. Large per-site panels live in a per-CTA global scratch slice, which
// stays resident in L2.
#include <cuda_bf16.h>

#include "kernels.cuh"
#include "tc.cuh"

using namespace la;

namespace {

__device__ __forceinline__ cd* core_ptr(cd* base, int core_stride, int s) {
  return base + (size_t)s * core_stride;
}


struct SvdSmem {
  cd* W;
  cd* V;
  double* sig;
  cd* tau;
  int* flag;
  int* misc;
};

__device__ SvdSmem carve_svd_smem(void* raw, int p, int hb, int vcap = 0) {
  SvdSmem s;
  char* c = reinterpret_cast<char*>(raw);
  s.W = reinterpret_cast<cd*>(c);
  c += sizeof(cd) * (size_t)(p + hb) * p;
  s.V = reinterpret_cast<cd*>(c);
  c += sizeof(cd) * (size_t)(vcap > 0 ? vcap : p * p);
  s.sig = reinterpret_cast<double*>(c);
  c += sizeof(double) * p;
  s.tau = reinterpret_cast<cd*>(c);
  c += sizeof(cd) * p;
  s.flag = reinterpret_cast<int*>(c);
  s.misc = s.flag + 1;
  return s;
}

// out (q x k, row-major) = Z (q x p, row-major) * V[:, :k] (V column-major p x *)
__device__ void gemm_zv(const cd* Z, long long q, int p, const cd* V, int k, cd* out) {
  const long long tot = q * (long long)k;
  for (long long idx = threadIdx.x; idx < tot; idx += blockDim.x) {
    const long long i = idx / k;
    const int c = (int)(idx - i * k);
    const cd* zr = Z + (size_t)i * p;
    const cd* vc = V + (size_t)c * p;
    cd acc = mkc(0.0, 0.0);
    for (int j = 0; j < p; ++j) acc = cfma(zr[j], vc[j], acc);
    out[idx] = acc;
  }
}

__device__ double cta_norm2(const cd* x, long long len, double* red) {
  double s = 0.0;
  for (long long i = threadIdx.x; i < len; i += blockDim.x) s += cabs2(x[i]);
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  double tot = 0.0;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += red[w];
  __syncthreads();
  return tot;
}

}  // namespace

// Work distribution shared by the per-instance kernels: slot k of `count`
// processes instance list[k] (or k). With a counter the CTAs take slots from it
// in order (the host sorts the list largest-first); without, slots are striped
// by blockIdx.
#define WORK_LOOP_BEGIN(list, count, counter)                               \
  __shared__ int sh_slot_;                                                  \
  int k_static_ = blockIdx.x;                                               \
  for (;;) {                                                                \
    if (threadIdx.x == 0) sh_slot_ = (counter) ? atomicAdd((counter), 1) : k_static_; \
    __syncthreads();                                                        \
    const int slot_ = sh_slot_;                                             \
    __syncthreads();                                                        \
    k_static_ += gridDim.x;                                                 \
    if (slot_ >= (count)) break;                                            \
    const int inst = (list) ? (list)[slot_] : slot_;
#define WORK_LOOP_END }

// Two-tier launches: a first launch with a small shared-memory carve (more
// CTAs per SM) hands every instance that does not fit it to a second launch
// with the full carve. The hand-off appends the instance to defer[1..]
// (defer[0] counts them) before anything of it has been written that the
// second launch would not rewrite; the second launch reads its count from
// defer[0] (dcount), so the host never waits for the first.
__device__ __forceinline__ void defer_instance(int* defer, int inst) {
  if (threadIdx.x == 0) {
    const int i = atomicAdd(defer, 1);
    defer[1 + i] = inst;
  }
}

// ---------------------------------------------------------------------------
// K1: integrand samples at listed indices
// ---------------------------------------------------------------------------
__global__ void k_sample(const InstParams* __restrict__ P, const long long* j,
                         long long count, cd* x) {
  const InstParams prm = *P;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count;
       i += (long long)gridDim.x * blockDim.x)
    x[i] = integrand(prm, j[i]);
}

// ---------------------------------------------------------------------------
// Support probe: smallest m such that the integrand beyond 2^m is negligible.
// Probes j = 2^i (1 + k/4), k < 4; m is the smallest exponent for which every
// probe at or beyond 2^m has |x_j| * j <= probe_tol * max |x|.
// ---------------------------------------------------------------------------
__global__ void k_support_probe(const InstParams* __restrict__ P, int count, double probe_factor,
                                int m_min, int* m_out) {
  const int inst = blockIdx.x;
  if (inst >= count) return;
  const InstParams prm = P[inst];
  const double probe_tol = probe_factor * prm.tol;
  __shared__ double mag[4 * 64];
  __shared__ double jv[4 * 64];
  const int n = prm.n;
  const int nprobe = 4 * n;
  for (int t = threadIdx.x; t < nprobe; t += blockDim.x) {
    const int i = t >> 2, k = t & 3;
    long long j = (1LL << i) + ((1LL << i) >> 2) * k;
    if (j >= (1LL << n)) j = (1LL << n) - 1;
    const cd x = integrand(prm, j);
    mag[t] = cabsd(x);
    jv[t] = (double)j;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double mx = 0.0;
    for (int t = 0; t < nprobe; ++t) mx = fmax(mx, mag[t]);
    {
      const cd x0 = integrand(prm, 0);
      mx = fmax(mx, cabsd(x0));
    }
    int m = n;
    if (prm.quad == Q_SIMPSON) {
      // scan from the top: find the lowest exponent whose probes beyond are small
      int mm = n;
      for (int e = n - 1; e >= 0; --e) {
        bool ok = true;
        for (int k = 0; k < 4; ++k) {
          const int t = 4 * e + k;
          if (mag[t] * jv[t] > probe_tol * mx) ok = false;
        }
        if (!ok) break;
        mm = e;
      }
      m = max(mm + 1, min(m_min, n));
      m = min(m, n);
    }
    m_out[inst] = m;
  }
}

// ---------------------------------------------------------------------------
// Work lists of the two builders, on the device (no host round trip): support
// exponents m <= svd_max_bits go to the TT-SVD builder, largest m first, the
// rest to the cross builder, largest n first; counts[0] and counts[1] receive
// the list lengths. One block, bucketed by key with shared-memory counters;
// the order among equal keys is arbitrary, which changes no result (every
// instance is built by one CTA alone).
// ---------------------------------------------------------------------------
__global__ void k_build_lists(const int* m_arr, const int* n_arr, int count, int svd_max_bits,
                              int* svd_list, int* cross_list, int* counts) {
  __shared__ int hs[64], hc[64];
  for (int i = threadIdx.x; i < 64; i += blockDim.x) {
    hs[i] = 0;
    hc[i] = 0;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < count; i += blockDim.x) {
    const int m = m_arr[i];
    if (m <= svd_max_bits)
      atomicAdd(&hs[max(m, 0)], 1);
    else
      atomicAdd(&hc[min(n_arr[i], 63)], 1);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    // bucket offsets, largest key first
    int os = 0, oc = 0;
    for (int k = 63; k >= 0; --k) {
      const int ts = hs[k], tc = hc[k];
      hs[k] = os;
      hc[k] = oc;
      os += ts;
      oc += tc;
    }
    counts[0] = os;
    counts[1] = oc;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < count; i += blockDim.x) {
    const int m = m_arr[i];
    if (m <= svd_max_bits)
      svd_list[atomicAdd(&hs[max(m, 0)], 1)] = i;
    else
      cross_list[atomicAdd(&hc[min(n_arr[i], 63)], 1)] = i;
  }
}

// ---------------------------------------------------------------------------
// Work order of the zip-up and the rounding: instances by decreasing cost, the
// longest first so that the persistent CTAs end together. The cost key is
// sum_s r_s^2 over the instance's TT ranks (the integrand's for the zip-up,
// the zip-up output's for the rounding): it tracks an instance's zip-up time
// with correlation 0.89 on the mixed batch, against 0.45 for n. One block,
// buckets of 16 key units; equal buckets in arbitrary order, which changes no
// result (every instance is processed by one CTA alone).
// ---------------------------------------------------------------------------
#define ORDER_BUCKETS 4096
__global__ void k_cost_order(const int* ranks_all, const int* n_arr, int count, int* order) {
  __shared__ int hist[ORDER_BUCKETS];
  for (int i = threadIdx.x; i < ORDER_BUCKETS; i += blockDim.x) hist[i] = 0;
  __syncthreads();
  auto bucket = [&](int inst) {
    const int* r = ranks_all + (size_t)inst * (SFFT_MAXN_DEV + 1);
    const int n = min(max(n_arr[inst], 0), SFFT_MAXN_DEV);
    int key = 0;  // ranks clamped: an instance that failed earlier may hold any
    for (int j = 0; j <= n; ++j) {
      const int rj = min(max(r[j], 0), SFFT_SLOT_RANK_DEV);
      key += rj * rj;
    }
    return min(key >> 4, ORDER_BUCKETS - 1);
  };
  for (int i = threadIdx.x; i < count; i += blockDim.x) atomicAdd(&hist[bucket(i)], 1);
  __syncthreads();
  if (threadIdx.x == 0) {
    // bucket offsets, largest key first
    int o = 0;
    for (int k = ORDER_BUCKETS - 1; k >= 0; --k) {
      const int c = hist[k];
      hist[k] = o;
      o += c;
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < count; i += blockDim.x) order[atomicAdd(&hist[bucket(i)], 1)] = i;
}

// ---------------------------------------------------------------------------
// K2: integrand TT by TT-SVD of the support block (Sec. 3.1; Oseledets 2011)
// ---------------------------------------------------------------------------
// The block x_j, j < 2^m, is swept from its least significant bit: at step t
// the carried matrix Z (2^(m-t-1) rows = remaining high bits, 2 r columns =
// (lambda, rank)) is factorised Z = U S V^H; V^H becomes core n-1-t and Z V
// the next carry. Sites above the block (Simpson grid, m < n) hold the
// rank-one core delta_{lambda,0}.
__global__ void k_integrand_ttsvd(const InstParams* __restrict__ P, const int* m_arr,
                                  const int* list, int count, int* counter, cd* scratch,
                                  long long scratch_stride,
                                  cd* tt, const long long* tt_off,
                                  int core_stride, int* ranks_all,
                                  int* status, int hb, double* acc, int pmax, int* defer,
                                  const int* dcount, int* zpre_t) {
  // panels of at most pmax columns (carve sized by the launch); with defer
  // set, instances that need wider panels go to the full-size launch.
  // zpre_t (may be null) receives the number of delta sites above the block.
  extern __shared__ double4 smem_raw[];
  SvdSmem sm = carve_svd_smem(smem_raw, pmax, hb);
  const int wcap = (pmax + hb) * pmax;
  __shared__ int perm_b[LA_MAXP];
  __shared__ double red_b[32];
  const int count_ = dcount ? *dcount : count;
  double fl = 0.0, evals = 0.0;
  WORK_LOOP_BEGIN(list, count_, counter)
    const InstParams prm = P[inst];
    const int n = prm.n;
    const int m = m_arr[inst];
    if (m < 0) continue;  // not built (status already set)
    const int rmax = prm.max_rank;
    int* ranks = ranks_all + (size_t)inst * (SFFT_MAXN_DEV + 1);
    cd* base = tt + tt_off[inst];
    cd* bufA = scratch + (size_t)blockIdx.x * scratch_stride;
    cd* bufB = bufA + (1LL << m);
    const long long Mb = 1LL << m;
    for (long long j = threadIdx.x; j < Mb; j += blockDim.x) bufA[j] = integrand(prm, j);
    __syncthreads();
    evals += (double)Mb;
    int st = 0;
    cd* Z = bufA;
    cd* O = bufB;
    long long q = Mb >> 1;
    int rprev = 1;
    // truncation budget per bond from the block's norm; each SVD may first
    // drop a part of squared norm <= delta^2 / 64 by pivoted QR (ts_svd's
    // prefilter), counted against the budget
    const double delta = prm.tol * sqrt(cta_norm2(bufA, Mb, red_b)) / sqrt((double)max(n - 1, 1));
    int site = n - 1;
    bool deferred = false;
    for (int t = 0; t < m; ++t, --site) {
      const int p = 2 * rprev;
      if (defer && p > pmax) {
        defer_instance(defer, inst);
        deferred = true;
        break;
      }
      cd* G = core_ptr(base, core_stride, site);
      if (q == 1) {
        // top of the block: the carry itself is the core (1, 2, rprev)
        for (int idx = threadIdx.x; idx < p; idx += blockDim.x) G[idx] = Z[idx];
        if (threadIdx.x == 0) {
          ranks[site] = 1;
          ranks[site + 1] = rprev;
        }
        __syncthreads();
        break;
      }
      TsSvd sv = ts_svd(Z, q, p, p, sm.W, wcap, sm.V, sm.sig, sm.tau, sm.flag, delta * delta * (1.0 / 64.0), perm_b);
      if (sv.sweeps < 0) st = SFFT_ENOCONV_DEV;
      int k = trunc_rank_tail(sm.sig, sv.m, delta, sv.tail2);
      if (k > rmax) {
        st = SFFT_ERANK_DEV;
        k = rmax;
      }
      // core (k, 2, rprev): G[c][lam][b] = conj(V[(lam, b), c])
      for (int idx = threadIdx.x; idx < k * p; idx += blockDim.x) {
        const int c = idx / p, rem = idx - c * p;
        G[idx] = cconj(sm.V[(size_t)c * p + rem]);
      }
      if (threadIdx.x == 0) {
        ranks[site] = k;
        ranks[site + 1] = rprev;
      }
      gemm_zv(Z, q, p, sm.V, k, O);
      __syncthreads();
      fl += sv.flops + flops_gemm(q, p, k);
      cd* tmp = Z;
      Z = O;
      O = tmp;
      q >>= 1;
      rprev = k;
    }
    if (deferred) continue;
    // sites above the block
    for (int s = 0; s < n - m; ++s) {
      cd* G = core_ptr(base, core_stride, s);
      if (threadIdx.x == 0) {
        G[0] = mkc(1.0, 0.0);
        G[1] = mkc(0.0, 0.0);
        ranks[s] = 1;
      }
    }
    if (threadIdx.x == 0) {
      ranks[0] = 1;
      ranks[n] = 1;
      status[inst] = st;
      if (zpre_t) zpre_t[inst] = n - m;
    }
    __syncthreads();
  WORK_LOOP_END
  if (acc && threadIdx.x == 0) {
    atomicAdd(acc + PH_BUILD, fl);
    atomicAdd(acc + SFFT_NPHASE_DEV + PH_BUILD, evals);
  }
}

// ---------------------------------------------------------------------------
// K2b: integrand TT by two-site cross interpolation (Sec. 3.1's TT-cross)
// ---------------------------------------------------------------------------
// For integrands whose numerical support is too wide to sample densely. Index
// sets: I[b] holds r_b prefixes (the b most significant bits of j), J[b] holds
// r_b suffixes (the n - b least significant bits), for bonds b = 0..n. The
// two-site supercore at bond b (sites b-1, b) is
//   Phi[(i, l1), (l2, t)] = x( ((I[b-1][i] 2 + l1) 2 + l2) 2^(n-b-1) + J[b+1][t] ).
// Left-to-right sweeps pick I[b] from the columns (i, l1) of Phi^T,
// right-to-left sweeps pick J[b] from the columns (l2, t) of Phi: in both a
// column-pivoted QR, stopped once the trailing norm is below 0.01 tol of the
// supercore's norm (rank cap max_rank), keeps the pivot columns, i.e. the
// greedy maximum-volume subset that maxvol would refine. Sweeps stop
// when the ranks repeat, after at least two. Assembly then runs one left-to-right pass: the fibre
// matrix F_s[(i, l), t] = x((I[s][i] 2 + l) 2^(n-s-1) + J[s+1][t]) is factored
// F = Q R, maxvol on Q gives I[s+1], and the core is Q Q[piv]^{-1}, which
// interpolates x on the cross (Oseledets & Tyrtyshnikov 2010; Savostyanov &
// Oseledets 2011). Rounding afterwards makes the cores right-orthonormal.
// Index choice of a cross step: the k columns of Z (q x p) picked by a
// column-pivoted QR truncated at ctol (the greedy maximum-volume column
// subset, as in Q-DEIM), k capped at rmax; returns k, the columns in piv, and
// sets *over when the rank wanted more than rmax columns.
// Pivoting Z and pivoting R of Z = Q R choose the same columns, so the rank
// is the one a rank-revealing QR of the supercore gives.
__device__ int cross_pick_columns(const cd* Z, int q, int p, SvdSmem& sm, int hb, double ctol, int rmax,
                              int* piv, int* iw, double* red_d, int* red_i, bool* over, double* fl) {
  __shared__ int perm_[LA_MAXP];
  (void)hb;
  (void)iw;
  (void)red_d;
  (void)red_i;
  // Z (row-major) -> W (column-major, leading dim q)
  for (int idx = threadIdx.x; idx < q * p; idx += blockDim.x) {
    const int row = idx / p, col = idx - row * p;
    sm.W[(size_t)col * q + row] = Z[idx];
  }
  __syncthreads();
  const RowBasis rb = pivqr_trunc(sm.W, q, q, p, ctol, rmax + 1, sm.tau, sm.sig, perm_);
  int k = rb.k;
  *over = k > rmax;
  if (k > rmax) k = rmax;
  for (int c = threadIdx.x; c < k; c += blockDim.x) piv[c] = perm_[c];
  __syncthreads();
  *fl += rb.flops;
  return k;
}

#define CROSS_R SFFT_SLOT_RANK_DEV
#define CROSS_R0 8

__device__ __forceinline__ long long cross_seed(int t, int L) {
  // candidate suffixes: 0, 1, all-ones, 2, 3, 5, 8, 13, 21, 34, ...
  if (L < 4) return t;  // few suffixes: take them all (t < 2^L)
  const long long top = (L >= 62) ? 0x3fffffffffffffffLL : ((1LL << L) - 1);
  if (t == 0) return 0;
  if (t == 1) return 1;
  if (t == 2) return top;
  long long a = 2, b = 3;
  for (int k = 3; k < t; ++k) {
    const long long c = a + b;
    a = b;
    b = c;
  }
  return a;
}

__global__ void k_integrand_cross(const InstParams* __restrict__ P, const int* list, int count,
                                  int* counter, cd* scratch, long long scratch_stride, cd* tt,
                                  const long long* tt_off, int core_stride, int* ranks_all,
                                  int* status, int hb, double* acc, int max_sweeps, int pmax,
                                  int rcap, int* defer, const int* dcount, const int* m_arr,
                                  int* zpre_t) {
  // panels of at most pmax columns (carve sized by the launch); with defer
  // set, ranks are capped at rcap and an instance that needs more goes to the
  // full-size launch before anything of it is written. m_arr (may be null):
  // the support probe's block exponents; zpre_t (may be null) receives the
  // number of delta sites above the block.
  extern __shared__ double4 smem_raw[];
  SvdSmem sm = carve_svd_smem(smem_raw, pmax, hb);
  __shared__ long long Iset[(SFFT_MAXN_DEV + 1) * CROSS_R];
  __shared__ long long Jset[(SFFT_MAXN_DEV + 1) * CROSS_R];
  __shared__ int rk[SFFT_MAXN_DEV + 1];
  __shared__ int rprev[SFFT_MAXN_DEV + 1];
  __shared__ int piv[2 * CROSS_R];
  __shared__ int iw[2 * CROSS_R];
  __shared__ double red_d[32];
  __shared__ int red_i[32];
  double fl = 0.0, evals = 0.0;
  cd* Z = scratch + (size_t)blockIdx.x * scratch_stride;
  const int count_ = dcount ? *dcount : count;
  WORK_LOOP_BEGIN(list, count_, counter)
    const InstParams prm = P[inst];
    // the cross runs on the block of the m least significant bits (the
    // support probe's); the n - m sites above it hold the rank-one
    // delta_{lam,0}, as the TT-SVD builder leaves them. Below, n is the
    // block's number of sites and j < 2^n the grid index.
    const int n_full = prm.n;
    const int n = m_arr ? min(max(m_arr[inst], 1), n_full) : n_full;
    const int site0 = n_full - n;
    const int rmax_i = min(prm.max_rank, CROSS_R);
    const int rmax = defer ? min(rmax_i, rcap) : rmax_i;
    bool hand_off = false;
    const double ctol = 0.01 * prm.tol;
    int st = 0;
    cd* base = tt + tt_off[inst] + (size_t)site0 * core_stride;
    int* rg = ranks_all + (size_t)inst * (SFFT_MAXN_DEV + 1) + site0;
    // initial right sets (seeds) and ranks
    for (int b = threadIdx.x; b <= n; b += blockDim.x) {
      const int L = n - b;
      int r0 = (b == 0 || b == n) ? 1 : CROSS_R0;
      if (L < 30) r0 = min(r0, 1 << L);
      if (b < 30) r0 = min(r0, 1 << b);
      r0 = max(r0, 1);
      rk[b] = r0;
      rprev[b] = 0;
      for (int t = 0; t < r0; ++t) Jset[b * CROSS_R + t] = (b == n) ? 0 : cross_seed(t, L);
      if (b == 0) Iset[0] = 0;
    }
    __syncthreads();
    for (int sw = 0; sw < max_sweeps; ++sw) {
      // ---- left to right: choose I[b]
      for (int b = 1; b < n; ++b) {
        const int rl = rk[b - 1], rr = rk[b + 1];
        const int p = 2 * rl, q = 2 * rr;
        const int sh = n - b - 1;
        for (int e = threadIdx.x; e < p * q; e += blockDim.x) {
          const int row = e / p, col = e - row * p;  // row (l2, t), col (i, l1)
          const int l2 = row / rr, t = row - l2 * rr, i = col >> 1, l1 = col & 1;
          const long long j = ((((Iset[(b - 1) * CROSS_R + i] << 1) | l1) << 1 | l2) << sh) | Jset[(b + 1) * CROSS_R + t];
          Z[e] = cconj(integrand(prm, j));
        }
        __syncthreads();
        evals += (double)p * q;
        bool over;
        int k = cross_pick_columns(Z, q, p, sm, hb, ctol, rmax, piv, iw, red_d, red_i, &over, &fl);
        if (over) {
          if (rmax < rmax_i) {
            hand_off = true;
            break;
          }
          st = SFFT_ERANK_DEV;
        }
        for (int c = threadIdx.x; c < k; c += blockDim.x)
          Iset[b * CROSS_R + c] = (Iset[(b - 1) * CROSS_R + (piv[c] >> 1)] << 1) | (piv[c] & 1);
        if (threadIdx.x == 0) rk[b] = k;
        __syncthreads();
      }
      if (hand_off) break;
      // ---- right to left: choose J[b]
      for (int b = n - 1; b >= 1; --b) {
        const int rl = rk[b - 1], rr = rk[b + 1];
        const int q = 2 * rl, p = 2 * rr;
        const int sh = n - b - 1;
        for (int e = threadIdx.x; e < p * q; e += blockDim.x) {
          const int row = e / p, col = e - row * p;  // row (i, l1), col (l2, t)
          const int i = row >> 1, l1 = row & 1, l2 = col / rr, t = col - l2 * rr;
          const long long j = ((((Iset[(b - 1) * CROSS_R + i] << 1) | l1) << 1 | l2) << sh) | Jset[(b + 1) * CROSS_R + t];
          Z[e] = integrand(prm, j);
        }
        __syncthreads();
        evals += (double)p * q;
        bool over;
        int k = cross_pick_columns(Z, q, p, sm, hb, ctol, rmax, piv, iw, red_d, red_i, &over, &fl);
        if (over) {
          if (rmax < rmax_i) {
            hand_off = true;
            break;
          }
          st = SFFT_ERANK_DEV;
        }
        for (int c = threadIdx.x; c < k; c += blockDim.x) {
          const int l2 = piv[c] / rr, t = piv[c] - l2 * rr;
          Jset[b * CROSS_R + c] = ((long long)l2 << sh) | Jset[(b + 1) * CROSS_R + t];
        }
        if (threadIdx.x == 0) rk[b] = k;
        __syncthreads();
      }
      if (hand_off) break;
      // converged when the ranks repeat
      int same = 1;
      for (int b = 0; b <= n; ++b) same &= (rk[b] == rprev[b]);
      __syncthreads();
      for (int b = threadIdx.x; b <= n; b += blockDim.x) rprev[b] = rk[b];
      __syncthreads();
      if (same && sw >= 1) break;
    }
    if (hand_off) {
      defer_instance(defer, inst);
      continue;
    }
    // ---- assembly: interpolatory cores, left to right
    if (threadIdx.x == 0) Iset[0] = 0;
    __syncthreads();
    for (int s = 0; s < n; ++s) {
      const int rl = rk[s];
      cd* G = core_ptr(base, core_stride, s);
      if (s == n - 1) {
        for (int e = threadIdx.x; e < 2 * rl; e += blockDim.x) {
          const int i = e >> 1, l = e & 1;
          G[e] = integrand(prm, (Iset[s * CROSS_R + i] << 1) | l);
        }
        evals += 2.0 * rl;
        __syncthreads();
        break;
      }
      const int rr = rk[s + 1];
      const int N = 2 * rl;
      const int sh = n - s - 1;
      for (int e = threadIdx.x; e < N * rr; e += blockDim.x) {
        const int c = e / N, row = e - c * N;  // column-major F
        const int i = row >> 1, l = row & 1;
        const long long j = ((((Iset[s * CROSS_R + i] << 1) | l)) << sh) | Jset[(s + 1) * CROSS_R + c];
        sm.W[e] = integrand(prm, j);
      }
      __syncthreads();
      evals += (double)N * rr;
      qr_inplace(sm.W, N, N, rr, sm.tau);
      const int kq = min(N, rr);
      form_q(sm.W, N, N, kq, sm.tau, sm.V, N);
      maxvol(sm.V, N, N, kq, piv, sm.W, iw, red_d, red_i);
      // core (rl, 2, kq): G[i][l][c] = B[c * N + (i, l)] with B = Q Q[piv]^{-1} in W
      for (int e = threadIdx.x; e < N * kq; e += blockDim.x) {
        const int row = e / kq, c = e - row * kq;
        G[e] = sm.W[(size_t)c * N + row];
      }
      for (int c = threadIdx.x; c < kq; c += blockDim.x)
        Iset[(s + 1) * CROSS_R + c] = (Iset[s * CROSS_R + (piv[c] >> 1)] << 1) | (piv[c] & 1);
      if (threadIdx.x == 0) rk[s + 1] = kq;
      __syncthreads();
      fl += flops_qr(N, rr) + flops_formq(N, kq);
    }
    for (int b = threadIdx.x; b <= n; b += blockDim.x) rg[b] = rk[b];
    for (int s = threadIdx.x; s < site0; s += blockDim.x) {
      cd* G = core_ptr(tt + tt_off[inst], core_stride, s);
      G[0] = mkc(1.0, 0.0);
      G[1] = mkc(0.0, 0.0);
      rg[s - site0] = 1;
    }
    if (threadIdx.x == 0) {
      rg[0] = 1;
      rg[n] = 1;
      status[inst] = max(status[inst], st);
      if (zpre_t) zpre_t[inst] = site0;
    }
    __syncthreads();
  WORK_LOOP_END
  if (acc && threadIdx.x == 0) {
    atomicAdd(acc + PH_CROSS, fl);
    atomicAdd(acc + SFFT_NPHASE_DEV + PH_CROSS, evals);
  }
}

// ---------------------------------------------------------------------------
// K3: Q_n MPO by barycentric Chebyshev interpolation of the bond variable
// ---------------------------------------------------------------------------
// Q_n = M^{-1/2} prod_l exp(-i pi mu_l (lambda_l + B_l)) with
// B_l = sum_{l' > l} lambda_l' 2^(l - l') in [0, 1) (the product form of the
// bit-reversed DFT, Sec. 3.2). The dependence of sites 1..l on B_l is an
// entire function exp(-2 pi i A B_l), A in [0,1), so it is carried across
// bond l by its values at P Chebyshev nodes b_q of [0,1]; B_{l-1} =
// (lambda_l + B_l)/2 gives the transfer core
//   W_l[p, mu, lambda, q] = 2^{-1/2} L_p((lambda + b_q)/2) exp(-i pi mu (lambda + b_q)),
// with the first core at p = 0 alone and the last at B_n = 0. Rounding then
// compresses the bonds to the requested tolerance.
__device__ __forceinline__ double cheb_node(int q, int P) {
  return 0.5 * (1.0 - cospi((2.0 * q + 1.0) / (2.0 * P)));
}
__device__ __forceinline__ double cheb_bw(int q, int P) {
  return ((q & 1) ? -1.0 : 1.0) * sinpi((2.0 * q + 1.0) / (2.0 * P));
}
// Lagrange basis L_p(x) at nodes b_q, barycentric form of the second kind
__device__ double lagrange(int p, double x, int P) {
  double den = 0.0, num = 0.0;
  for (int q = 0; q < P; ++q) {
    const double d = x - cheb_node(q, P);
    if (d == 0.0) return q == p ? 1.0 : 0.0;
    const double t = cheb_bw(q, P) / d;
    den += t;
    if (q == p) num = t;
  }
  return num / den;
}

__global__ void k_mpo_interp(int n, int P, cd* W, int core_stride,
                             int* ranks) {
  const double s2 = 0.70710678118654752;
  for (int s = blockIdx.x; s < n; s += gridDim.x) {
    const int r0 = (s == 0) ? 1 : P;
    const int r1 = (s == n - 1) ? 1 : P;
    cd* G = W + (size_t)s * core_stride;
    const int tot = r0 * 4 * r1;
    for (int idx = threadIdx.x; idx < tot; idx += blockDim.x) {
      const int a = idx / (4 * r1);
      const int rem = idx - a * 4 * r1;
      const int sg = rem / r1, b = rem - sg * r1;
      const int mu = sg >> 1, lam = sg & 1;
      const double bq = (s == n - 1) ? 0.0 : cheb_node(b, P);
      const double x = 0.5 * (lam + bq);
      const double lp = (s == 0) ? 1.0 : lagrange(a, x, P);
      double ph_re = 1.0, ph_im = 0.0;
      if (mu) {
        // exp(-i pi (lam + bq))
        double sn, cs;
        sincospi(lam + bq, &sn, &cs);
        ph_re = cs;
        ph_im = -sn;
      }
      G[idx] = mkc(s2 * lp * ph_re, s2 * lp * ph_im);
    }
    if (threadIdx.x == 0) {
      ranks[s] = r0;
      if (s == n - 1) ranks[n] = 1;
    }
  }
}

// ---------------------------------------------------------------------------
// K5: TT rounding (Oseledets 2011): optional left-to-right orthogonalisation
// by Householder QR, then a right-to-left sweep of truncated SVDs with
// delta = tol ||A|| / sqrt(n-1). Works in place on a slot TT with d in {2,4}.
// ---------------------------------------------------------------------------
// Right-to-left step at site s, X = G_s as r_s x (d r_{s+1}) = U S V^H:
// the SVD of Z = X^H gives U and S; with k kept, Y = Z U_k = V_k S_k is
// orthonormalised by QR, Y = Q_V R_V, and X ~= (X Q_V) Q_V^H: G_s becomes
// Q_V^H, right-orthonormal to machine precision, and X Q_V moves into
// G_{s-1} (no division by small singular values). The projection onto
// span(Q_V) is exact whatever the orthogonality of U_k, so the error is the
// truncated tail plus the coupling of kept to dropped directions times the
// dropped singular values; the Jacobi iteration may therefore stop once its
// rotations fall below 1e-2 relative.
// The SVD of Z is taken after a column-pivoted QR that drops trailing rows of
// squared norm at most delta^2 / 64 (pq_svd): Hestenes' method then runs on
// the k' kept rows only, and the dropped norm counts against the truncation
// budget, so the error bound is that of the plain truncated SVD and the rank
// exceeds the plain SVD's only where its tail lies within delta^2 / 64 of
// delta^2.
__global__ void __maxnreg__(72) k_tt_round(const int* list, int count, int* counter, const int* n_arr, int d,
                           int left_orth,
                           const double* tol_arr, const int* maxrank_arr,
                           cd* tt, const long long* tt_off, int core_stride,
                           int* ranks_all, cd* scratch,
                           long long scratch_stride, int* status, int hb,
                           double* acc, int phase, int pmax, int vcap, int* defer,
                           const int* dcount, const int* site0_arr) {
  // site0_arr (may be null): per instance, the first site rounded; the sites
  // above it (rank-one delta cores) are left as they are
  // shared memory sized by the launch: panels of at most pmax columns, Q
  // blocks of vcap elements (see round_smem_bytes on the host)
  extern __shared__ double4 smem_raw[];
  SvdSmem sm = carve_svd_smem(smem_raw, pmax, hb, vcap);
  __shared__ double red[32];
  // ranks of the instance in flight: thread 0 updates them between barriers,
  // every thread reads them, so they live in shared memory
  __shared__ int r[SFFT_MAXN_DEV + 1];
  __shared__ int perm_s[SFFT_SLOT_RANK_DEV];  // column order of the pivoted QR
  const int count_ = dcount ? *dcount : count;
  double fl = 0.0;
  WORK_LOOP_BEGIN(list, count_, counter)
    // n: the sites rounded; the bond budget below counts every bond of the TT
    const int n_full = n_arr[inst];
    const int site0 = site0_arr ? min(max(site0_arr[inst], 0), n_full - 1) : 0;
    const int n = n_full - site0;
    const double tol = tol_arr[inst];
    const int rmax = maxrank_arr[inst];
    int* rg = ranks_all + (size_t)inst * (SFFT_MAXN_DEV + 1) + site0;
    __syncthreads();
    for (int i = threadIdx.x; i <= n; i += blockDim.x) r[i] = rg[i];
    __syncthreads();
    cd* base = tt + tt_off[inst] + (size_t)site0 * core_stride;
    cd* tmp = scratch + (size_t)blockIdx.x * scratch_stride;
    int st = 0;
    if (status && status[inst] != 0) continue;
    if (defer) {
      // ranks never grow here, so the input ranks decide whether the carve fits
      int mr = 0;
      for (int i = 0; i <= n; ++i) mr = max(mr, r[i]);
      if (mr > pmax) {
        defer_instance(defer, inst);
        continue;
      }
    }
    if (left_orth) {
      for (int s = 0; s + 1 < n; ++s) {
        const int r0 = r[s], r1 = r[s + 1], r2 = r[s + 2];
        cd* G = core_ptr(base, core_stride, s);
        cd* H = core_ptr(base, core_stride, s + 1);
        const int q = r0 * d;
        const int kq = min(q, r1);
        // G (q x r1, row-major) -> W column-major
        for (int idx = threadIdx.x; idx < q * r1; idx += blockDim.x) {
          const int i = idx / r1, j = idx - i * r1;
          sm.W[(size_t)j * q + i] = G[idx];
        }
        __syncthreads();
        qr_inplace(sm.W, q, q, r1, sm.tau);
        form_q(sm.W, q, q, kq, sm.tau, sm.V, q);
        // G <- Q (q x kq); H <- R H with R = upper kq x r1 of W
        for (int idx = threadIdx.x; idx < q * kq; idx += blockDim.x) {
          const int i = idx / kq, c = idx - i * kq;
          G[idx] = sm.V[(size_t)c * q + i];
        }
        const int cols = d * r2;
        for (int idx = threadIdx.x; idx < kq * cols; idx += blockDim.x) {
          const int c = idx / cols, col = idx - c * cols;
          cd acc = mkc(0.0, 0.0);
          for (int a = c; a < r1; ++a) acc = cfma(sm.W[(size_t)a * q + c], H[(size_t)a * cols + col], acc);
          tmp[idx] = acc;
        }
        __syncthreads();
        for (int idx = threadIdx.x; idx < kq * cols; idx += blockDim.x) H[idx] = tmp[idx];
        if (threadIdx.x == 0) r[s + 1] = kq;
        __syncthreads();
        fl += flops_qr(q, r1) + flops_formq(q, kq) + flops_gemm(kq, cols, r1);
      }
    }
    // norm of the tensor = norm of the last core (cores before it are left-orthonormal)
    {
      cd* G = core_ptr(base, core_stride, n - 1);
      const double nn = cta_norm2(G, (long long)r[n - 1] * d * r[n], red);
      const double delta = tol * sqrt(nn) / sqrt((double)max(n_full - 1, 1));
      for (int s = n - 1; s >= 1; --s) {
        const int r0 = r[s], r1 = r[s + 1], rm = r[s - 1];
        cd* Gs = core_ptr(base, core_stride, s);
        cd* Gp = core_ptr(base, core_stride, s - 1);
        const int q = d * r1;
        // Z = X^H with X = Gs as r0 x (d r1): Z[(sig,b), a] = conj(Gs[a][sig][b])
        cd* Zt = tmp;
        cd* Y = tmp + (size_t)q * r0;
        cd* QV = Y + (size_t)q * r0;
        // Z row-major into the scratch (for Y below) and column-major into W
        // (leading dim pmax + hb >= d r1 = q), where the SVD factors it
        const int ldw = pmax + hb;
        for (int idx = threadIdx.x; idx < q * r0; idx += blockDim.x) {
          const int a = idx / q, row = idx - a * q;
          const cd z = cconj(Gs[idx]);
          Zt[(size_t)row * r0 + a] = z;
          sm.W[(size_t)a * ldw + row] = z;
        }
        __syncthreads();
        // the pivoted-QR prefilter may drop a norm of up to delta^2 / 64 before
        // the SVD; the truncation counts it against the budget
        TsSvd sv = pq_svd(sm.W, ldw, q, r0, delta * delta * (1.0 / 64.0), sm.V, sm.sig, sm.tau, perm_s,
                          sm.flag, 1e-4);
        if (sv.sweeps < 0) st = SFFT_ENOCONV_DEV;
        int k = trunc_rank_tail(sm.sig, sv.m, delta, sv.tail2);
        if (k > rmax) {
          st = SFFT_ERANK_DEV;
          k = rmax;
        }
        // Y = Z U_k (q x k), then QR: Y = Q_V R_V
        gemm_zv(Zt, q, r0, sm.V, k, Y);
        __syncthreads();
        for (int idx = threadIdx.x; idx < q * k; idx += blockDim.x) {
          const int i = idx / k, j = idx - i * k;
          sm.W[(size_t)j * q + i] = Y[idx];
        }
        __syncthreads();
        qr_inplace(sm.W, q, q, k, sm.tau);
        const int kk = min(q, k);
        form_q(sm.W, q, q, kk, sm.tau, QV, q);
        // Gs <- Q_V^H (kk x q)
        for (int idx = threadIdx.x; idx < kk * q; idx += blockDim.x) {
          const int c = idx / q, row = idx - c * q;
          Gs[idx] = cconj(QV[(size_t)c * q + row]);
        }
        // T1 = X Q_V (r0 x kk) into Y (free now), then Gp <- Gp T1: the rows
        // of X are projected onto span(Q_V) exactly, so the result does not
        // depend on how orthogonal the Jacobi vectors U_k are
        for (int idx = threadIdx.x; idx < r0 * kk; idx += blockDim.x) {
          const int a = idx / kk, c = idx - a * kk;
          const cd* qc = QV + (size_t)c * q;
          cd acc = mkc(0.0, 0.0);
          for (int row = 0; row < q; ++row) acc = cfma(cconj(Zt[(size_t)row * r0 + a]), qc[row], acc);
          Y[idx] = acc;
        }
        __syncthreads();
        const int rows = rm * d;
        cd* out = QV + (size_t)q * kk;
        for (int idx = threadIdx.x; idx < rows * kk; idx += blockDim.x) {
          const int row = idx / kk, c = idx - row * kk;
          cd acc = mkc(0.0, 0.0);
          for (int a = 0; a < r0; ++a) acc = cfma(Gp[(size_t)row * r0 + a], Y[(size_t)a * kk + c], acc);
          out[idx] = acc;
        }
        __syncthreads();
        for (int idx = threadIdx.x; idx < rows * kk; idx += blockDim.x) Gp[idx] = out[idx];
        if (threadIdx.x == 0) r[s] = kk;
        __syncthreads();
        fl += sv.flops + flops_gemm(q, r0, k) + flops_qr(q, k) + flops_formq(q, kk) +
              flops_gemm(r0, kk, q) + flops_gemm(rows, kk, r0);
      }
    }
    for (int i = threadIdx.x; i <= n; i += blockDim.x) rg[i] = r[i];
    if (threadIdx.x == 0 && status) status[inst] = max(status[inst], st);
    __syncthreads();
  WORK_LOOP_END
  if (acc && threadIdx.x == 0) atomicAdd(acc + phase, fl);
}

// ---------------------------------------------------------------------------
// Mixed precision: the zip-up's MPO contraction on the tensor cores
// ---------------------------------------------------------------------------
// The panel Z[(a', b'), (c, mu)] = sum_{a, lam} Dt[c][a][lam][b'] conj(W[a][2 mu + lam][a'])
// is the complex product X Y^T with X[(c, b'), (a, lam)] = Dt[c][a][lam][b']
// (M = r_c r' rows, K = 2 s columns) and Y[(mu, a'), (a, lam)] =
// conj(W[a][2 mu + lam][a']) (N = 2 s' rows). In real arithmetic it is the
// single GEMM D' = A' B'^T with
//   A' = [Re X | Im X]                        (M x 2K)
//   B' = [[Re W, Im W], [-Im W, Re W]]        (2N x 2K: rows (mu, a'), then again)
// so that D'[m, n] = Re Z' and D'[m, N + n] = Im Z' (the 4M form), run as
// tcgen05.mma kind::f16 on one 128-row tile with FP32 accumulation in tensor
// memory. Every operand value v is split into three bfloat16 pieces
// v0 = bf16(v), v1 = bf16(v - v0), v2 = bf16(v - v0 - v1), which hold v to
// about 2^-25 (FP32 precision), and the six products v_i w_j with i + j <= 2
// are formed. For each K step of 16 the leading product v0 w0 and the five
// smaller ones go to two separate accumulators; the step's two partial
// panels are then added in FP64 into a panel in the CTA's global scratch
// (L2-resident), so no FP32 sum runs over more than one K step. Long FP32
// accumulations, compounded over the n sites of the zip-up chain, would
// otherwise set the price error. The operand tiles live in the shared-memory
// block W, which the panel may overwrite once the last MMAs have completed.
struct ZipTc {
  uint32_t tmem;
  uint64_t* mbar;
  uint32_t phase;
};

// the three bfloat16 pieces of v (split from the FP64 value), as bit patterns
__device__ __forceinline__ void bf16_split3(double v, uint16_t* b) {
  const __nv_bfloat16 h0 = __double2bfloat16(v);
  const double r1 = v - (double)__bfloat162float(h0);
  const __nv_bfloat16 h1 = __double2bfloat16(r1);
  const double r2 = r1 - (double)__bfloat162float(h1);
  const __nv_bfloat16 h2 = __double2bfloat16(r2);
  b[0] = __bfloat16_as_ushort(h0);
  b[1] = __bfloat16_as_ushort(h1);
  b[2] = __bfloat16_as_ushort(h2);
}

// Operand bytes the contraction needs for M rows, K = 2 s complex columns and
// N1 = 2 s' complex outputs (0 when one tile cannot hold it: 128 rows, two
// accumulators of at most 64 columns in the CTA's 128 tensor-memory columns).
__device__ __forceinline__ int zip_tc_bytes(int M, int K, int N1) {
  const int kp = (2 * K + 15) & ~15, np = (2 * N1 + 15) & ~15;
  if (M > 128 || np > 64 || np < 16) return 0;
  return 3 * (128 + np) * kp * 2;
}

// Forms the panel in Zg (global scratch, FP64: Zg[idx] = Z, idx = (a' r' +
// b') p + (c 2 + mu)) and then stores it where the FP64 loop would: the
// conjugate into sm_panel when given, else into Zg itself (conjugated when
// conj_out). Returns false when a bounded wait for the MMAs expired.
__device__ bool zip_panel_tc(const cd* Dt, const cd* Ws, int rc, int s0, int s1, int rA1, unsigned char* opnd,
                             ZipTc& tz, cd* Zg, cd* sm_panel, int q, int p, bool conj_out) {
  const int M = rc * rA1, K = 2 * s0, N1 = 2 * s1;
  const int kp = (2 * K + 15) & ~15, np = (2 * N1 + 15) & ~15;
  const int kb = 2 * kp;  // bytes of an operand row
  unsigned char* A[3] = {opnd, opnd + 128 * kb, opnd + 2 * 128 * kb};
  unsigned char* Bp[3] = {opnd + 3 * 128 * kb, opnd + 3 * 128 * kb + np * kb, opnd + 3 * 128 * kb + 2 * np * kb};
  // A' rows m = (c, b'), columns (re | im) of (a, lam). Rows from M on feed
  // only output rows that are never read, so they are not staged (whatever
  // they hold); the K padding of the staged rows is zero.
  for (int e = threadIdx.x; e < M * kp; e += blockDim.x) {
    const int m = e / kp, k = e - m * kp;
    double v = 0.0;
    if (k < 2 * K) {
      const int c = m / rA1, bp = m - c * rA1;
      const int kk = k < K ? k : k - K;
      const int a = kk >> 1, lam = kk & 1;
      const cd d = Dt[(((size_t)c * s0 + a) * 2 + lam) * rA1 + bp];
      v = k < K ? d.x : d.y;
    }
    uint16_t b[3];
    bf16_split3(v, b);
    const uint32_t off = tc::kmajor_off(m, 2 * k, kb);
#pragma unroll
    for (int i = 0; i < 3; ++i) *reinterpret_cast<uint16_t*>(A[i] + off) = b[i];
  }
  // B' rows n = (mu, a') for the real part, N1 + n for the imaginary part;
  // the padding rows from 2 N1 on feed only columns that are never read, and
  // the K padding is zero on both operands
  for (int e = threadIdx.x; e < 2 * N1 * kp; e += blockDim.x) {
    const int n = e / kp, k = e - n * kp;
    double v = 0.0;
    if (k < 2 * K) {
      const bool imag_row = n >= N1;
      const int nn = imag_row ? n - N1 : n;
      const int mu = nn / s1, ap = nn - mu * s1;
      const bool second = k >= K;
      const int kk = second ? k - K : k;
      const int a = kk >> 1, lam = kk & 1;
      const cd w = Ws[(size_t)a * 4 * s1 + (2 * mu + lam) * s1 + ap];
      v = imag_row ? (second ? w.x : -w.y) : (second ? w.y : w.x);
    }
    uint16_t b[3];
    bf16_split3(v, b);
    const uint32_t off = tc::kmajor_off(n, 2 * k, kb);
#pragma unroll
    for (int i = 0; i < 3; ++i) *reinterpret_cast<uint16_t*>(Bp[i] + off) = b[i];
  }
  tc::fence_proxy_async();
  const uint32_t idesc = tc::idesc_bf16(128, np);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ngrp = (int)(blockDim.x >> 5) / 4;
  const int m = 32 * (w & 3) + lane;
  const int c = m / rA1, bp = m - c * rA1;
  for (int ks = 0; ks < kp / 16; ++ks) {
    tc::fence_before_sync();
    __syncthreads();
    if (threadIdx.x == 0) {
      tc::fence_after_sync();
      const uint32_t o = (uint32_t)ks * 256u;  // 16 bf16 = 32 bytes = two core columns
      // accumulator 0: v0 w0; accumulator 1 (columns np..): the five smaller products
      tc::mma_bf16(tz.tmem, tc::kmajor_desc(tc::smem_u32(A[0]) + o, kb), tc::kmajor_desc(tc::smem_u32(Bp[0]) + o, kb),
                   idesc, 0u);
      const int pi[5] = {1, 0, 2, 1, 0}, pj[5] = {1, 2, 0, 0, 1};
      for (int t = 0; t < 5; ++t)
        tc::mma_bf16(tz.tmem + (uint32_t)np, tc::kmajor_desc(tc::smem_u32(A[pi[t]]) + o, kb),
                     tc::kmajor_desc(tc::smem_u32(Bp[pj[t]]) + o, kb), idesc, t ? 1u : 0u);
      tc::commit(tz.mbar);
    }
    const bool ok = __syncthreads_and(tc::mbar_wait(tz.mbar, tz.phase, 1LL << 22));
    tz.phase ^= 1u;
    if (!ok) return false;
    tc::fence_after_sync();
    // this K step's partial panel, added in FP64: warp w reads lanes
    // 32 (w % 4) .. + 31 (rows m); the warps past the first four take the
    // other 16-column blocks
    if (w < 4 * ngrp) {
      for (int cb = 16 * (w >> 2); cb < np; cb += 16 * ngrp) {
        float v0[16], v1[16];
        const uint32_t ta = tz.tmem + ((uint32_t)(32 * (w & 3)) << 16) + (uint32_t)cb;
        tc::tmem_ld16(ta, v0);
        tc::tmem_ld16(ta + (uint32_t)np, v1);
        if (m < M) {
#pragma unroll
          for (int i = 0; i < 16; ++i) {
            const int n = cb + i;
            if (n < 2 * N1) {
              const bool imag = n >= N1;
              const int nn = imag ? n - N1 : n;
              const int mu = nn / s1, ap = nn - mu * s1;
              const size_t idx = (size_t)(ap * rA1 + bp) * p + (c * 2 + mu);
              double* t = reinterpret_cast<double*>(Zg + idx) + (imag ? 1 : 0);
              const double part = (double)v0[i] + (double)v1[i];
              *t = ks ? *t + part : part;
            }
          }
        }
      }
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  // where the FP64 loop leaves the panel
  for (int idx = threadIdx.x; idx < q * p; idx += blockDim.x) {
    if (sm_panel)
      sm_panel[idx] = cconj(Zg[idx]);
    else if (conj_out)
      Zg[idx] = cconj(Zg[idx]);
  }
  __syncthreads();
  return true;
}

// ---------------------------------------------------------------------------
// K4: zip-up MPO x TT contraction (Stoudenmire & White 2010), left to right.
// ---------------------------------------------------------------------------
// Carry C (r' x s r) from the previous site is stored as CH = C^H. At site s:
//   Dt[c][a][lam][b'] = sum_b CH[(a,b), c] conj(A[b][lam][b'])         (= conj D)
//   Z[(a',b'), (c,mu)] = sum_{a,lam} Dt[c][a][lam][b'] conj(W[a][2mu+lam][a'])
// so Z = T^H with T = C (W . A) the (r' 2) x (s' r') panel. The right singular
// vectors V of Z are the left singular vectors of T: V becomes the output core
// B_s[c][mu][c''] and Z V = T^H V the next carry CH. Singular values below
// ztol * ||T|| are dropped; the final rounding sweep sets the ranks.
template <bool TC>
__device__ __forceinline__ void zipup_body(const int* list, int count, int* counter, const int* n_arr, const double* tol_arr,
                        const int* maxrank_arr, const cd* A,
                        const long long* a_off, const int* a_ranks_all,
                        const cd* Wmpo, const long long* w_off,
                        const int* w_ranks_all, cd* B,
                        const long long* b_off, int* b_ranks_all,
                        int core_stride_a, int core_stride_w, int core_stride_b,
                        cd* scratch, long long scratch_stride,
                        int* status, int hb, double* acc, int vcap, int* defer, const int* dcount,
                        int qmax1, int wlim, ZipPrefix zp) {
  // shared memory: W ((LA_MAXP + hb) x LA_MAXP) for the panel T and, in its
  // spent columns, the explicit Q; V (vcap elements) for the streaming
  // fallback of panels larger than W. A launch without V (vcap <= 1) hands
  // the instances that need it to the full-size launch (defer).
  // qmax1: most panel columns a launch with defer set keeps (<= LA_MAXQ);
  // wlim: most panel elements factored directly in shared memory (<= the
  // carve's W); both are the carve's own limits unless a test narrows them.
  // TC: the MPO contraction of each site on the tensor cores (zip_panel_tc)
  // wherever one tile holds it, in FP64 on the CUDA cores elsewhere.
  extern __shared__ double4 smem_raw[];
  SvdSmem sm = carve_svd_smem(smem_raw, LA_MAXP, hb, vcap);
  const int wcap = (LA_MAXP + hb) * LA_MAXP;
  const int wdir = min(wlim, wcap);
  const int qfit = min(qmax1, LA_MAXQ);
  const bool has_v = vcap > 1;
  __shared__ int zperm[LA_MAXQ];
  __shared__ double zcn[LA_MAXQ];
  const int count_ = dcount ? *dcount : count;
  double fl = 0.0;
  double tc_sites = 0.0;  // sites whose MPO contraction ran on the tensor cores
  ZipTc tz;
  __shared__ uint64_t tc_mbar;
  __shared__ uint32_t tc_slot;
  bool tc_fail = false;
  if constexpr (TC) {
    if (threadIdx.x == 0) {
      tc::mbar_init(&tc_mbar, 1);
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if ((threadIdx.x >> 5) == 0) tc::tmem_alloc(&tc_slot, 128);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    tz.tmem = tc_slot;
    tz.mbar = &tc_mbar;
    tz.phase = 0u;
  }
  WORK_LOOP_BEGIN(list, count_, counter)
    const int n = n_arr[inst];
    const double ztol = tol_arr[inst] / sqrt((double)max(n - 1, 1));
    const int rmax = maxrank_arr[inst];
    const int* ra = a_ranks_all + (size_t)inst * (SFFT_MAXN_DEV + 1);
    const int* rw = w_ranks_all + (size_t)inst * (SFFT_MAXN_DEV + 1);
    int* rb = b_ranks_all + (size_t)inst * (SFFT_MAXN_DEV + 1);
    const cd* Ab = A + a_off[inst];
    const cd* Wb = Wmpo + w_off[inst];
    cd* Bb = B + b_off[inst];
    cd* CH = scratch + (size_t)blockIdx.x * scratch_stride;
    cd* Dt = CH + SFFT_ZIP_CH_DEV;
    cd* Z = Dt + SFFT_ZIP_D_DEV;
    // 3-multiplication products x conj(y): T1 = sum xr yr, T2 = sum xi yi,
    // T3 = sum (xr + xi)(yr - yi); re = T1 + T2, im = T3 - T1 + T2. The
    // planes below hold xr + xi of the carry and of D, yr - yi of the cores.
    double* CHs = reinterpret_cast<double*>(Z + SFFT_ZIP_Z_DEV);
    double* Dts = CHs + SFFT_ZIP_CH_DEV;
    double* Ass = Dts + SFFT_ZIP_D_DEV;
    double* Wss = Ass + 2 * SFFT_SLOT_RANK_DEV * SFFT_SLOT_RANK_DEV;
    int st = 0;
    if (status[inst] != 0) continue;
    if (threadIdx.x == 0) {
      CH[0] = mkc(1.0, 0.0);
      rb[0] = 1;
      rb[n] = 1;
    }
    __syncthreads();
    int rc = 1;
    int s_begin = 0;
    if (zp.t && zp.t[inst] > 0 && zp.off[inst] >= 0) {
      // sites 0..t-1 carry the integrand's delta cores: their output cores
      // and the carry after site t-1 come from the MPO's prefix block
      const int t = zp.t[inst];
      const cd* blk = zp.pool + zp.off[inst];
      const int* pr = zp.ranks + (size_t)inst * (SFFT_MAXN_DEV + 1);
      for (int s = 0; s < t; ++s) {
        const int len = pr[s] * 2 * pr[s + 1];
        const cd* src = blk + (size_t)s * SFFT_CORE_STRIDE_D2;
        cd* dst = Bb + (size_t)s * core_stride_b;
        for (int idx = threadIdx.x; idx < len; idx += blockDim.x) __stcs(dst + idx, src[idx]);
      }
      rc = pr[t];
      const cd* csrc = blk + SFFT_ZPRE_CARRY_BASE + (size_t)(t - 1) * SFFT_ZIP_CARRY_STRIDE;
      for (int idx = threadIdx.x; idx < rw[t] * rc; idx += blockDim.x) CH[idx] = csrc[idx];
      if (threadIdx.x == 0)
        for (int s = 1; s <= t; ++s) rb[s] = pr[s];
      s_begin = t;
      __syncthreads();
    }
    bool deferred = false;
    for (int s = s_begin; s < n; ++s) {
      const int rA0 = ra[s], rA1 = ra[s + 1], s0 = rw[s], s1 = rw[s + 1];
      {
        // a launch without V handles panels of up to LA_MAXQ columns (in W,
        // or in global scratch when larger); the rest go on (uniform over the CTA)
        const bool fits = s1 * rA1 <= qfit;
        if (defer && !fits && s < n - 1) {
          defer_instance(defer, inst);
          deferred = true;
          break;
        }
      }
      const cd* As = Ab + (size_t)s * core_stride_a;
      const cd* Ws = Wb + (size_t)s * core_stride_w;
      // sum planes of this site's factors
      for (int idx = threadIdx.x; idx < s0 * rA0 * rc; idx += blockDim.x) CHs[idx] = CH[idx].x + CH[idx].y;
      for (int idx = threadIdx.x; idx < rA0 * 2 * rA1; idx += blockDim.x) Ass[idx] = As[idx].x - As[idx].y;
      for (int idx = threadIdx.x; idx < s0 * 4 * s1; idx += blockDim.x) Wss[idx] = Ws[idx].x - Ws[idx].y;
      __syncthreads();
      // Dt[c][a][lam][b'] = sum_b CH[(a, b), c] conj(A[b][lam][b'])
      const int nd = rc * s0 * 2 * rA1;
      for (int idx = threadIdx.x; idx < nd; idx += blockDim.x) {
        int rem = idx;
        const int bp = rem % rA1; rem /= rA1;
        const int lam = rem & 1; rem >>= 1;
        const int a = rem % s0; const int c = rem / s0;
        double t1 = 0.0, t2 = 0.0, t3 = 0.0;
        for (int b = 0; b < rA0; ++b) {
          const size_t ci = (size_t)(a * rA0 + b) * rc + c;
          const size_t ai = (size_t)b * 2 * rA1 + lam * rA1 + bp;
          const cd x = CH[ci], y = As[ai];
          t1 = fma(x.x, y.x, t1);
          t2 = fma(x.y, y.y, t2);
          t3 = fma(CHs[ci], Ass[ai], t3);
        }
        const double re = t1 + t2, im = t3 - t1 + t2;
        Dt[idx] = mkc(re, im);
        Dts[idx] = re + im;
      }
      __syncthreads();
      const int q = s1 * rA1, p = 2 * rc;
      // T = Z^H (p x q, column-major) goes straight to shared memory when it
      // fits: Z's row-major buffer and T's column-major one share the index
      const bool direct = q <= LA_MAXQ && p * q <= wdir;
      // without V, a panel larger than W is factored in place in the CTA's
      // global scratch instead (same steps, L2-resident)
      const bool gdirect = !direct && !has_v && q <= LA_MAXQ;
      cd* Tp = direct ? sm.W : Z;
      bool on_tc = false;
      if constexpr (TC) {
        const int need = zip_tc_bytes(rc * rA1, 2 * s0, 2 * s1);
        if (!tc_fail && need > 0 && need <= (int)(sizeof(cd) * wcap)) {
          on_tc = true;
          tc_sites += 1.0;
          if (!zip_panel_tc(Dt, Ws, rc, s0, s1, rA1, reinterpret_cast<unsigned char*>(sm.W), tz, Z,
                            direct ? sm.W : nullptr, q, p, gdirect)) {
            tc_fail = true;
            st = SFFT_ETIMEOUT_DEV;
          }
        }
      }
      for (int idx = threadIdx.x; idx < (on_tc ? 0 : q * p); idx += blockDim.x) {
        const int row = idx / p, col = idx - row * p;
        const int ap = row / rA1, bp = row - ap * rA1;
        const int c = col >> 1, mu = col & 1;
        double t1 = 0.0, t2 = 0.0, t3 = 0.0;
        for (int a = 0; a < s0; ++a) {
#pragma unroll
          for (int lam = 0; lam < 2; ++lam) {
            const size_t di = (((size_t)c * s0 + a) * 2 + lam) * rA1 + bp;
            const size_t wi = (size_t)a * 4 * s1 + (2 * mu + lam) * s1 + ap;
            const cd d = Dt[di], w = Ws[wi];
            t1 = fma(d.x, w.x, t1);
            t2 = fma(d.y, w.y, t2);
            t3 = fma(Dts[di], Wss[wi], t3);
          }
        }
        const cd acc = mkc(t1 + t2, t3 - t1 + t2);
        if (direct)
          sm.W[idx] = cconj(acc);
        else
          Z[idx] = gdirect ? cconj(acc) : acc;
      }
      __syncthreads();
      fl += flops_gemm(nd, rA0, 1) + flops_gemm((long long)q * p, 2 * s0, 1);
      // output cores are written once here and read back only by the
      // rounding launch: streaming stores (evict first) keep the CTA's
      // scratch resident in L2 while 0.4 GB of cores stream out
      cd* Bs = Bb + (size_t)s * core_stride_b;
      if (s == n - 1) {
        // q == 1: B[c][mu][0] = conj(Z[0, (c, mu)])
        for (int idx = threadIdx.x; idx < p; idx += blockDim.x)
          __stcs(Bs + idx, direct ? sm.W[idx] : (gdirect ? Z[idx] : cconj(Z[idx])));
        __syncthreads();
        break;
      }
      if (direct || gdirect) {
        // column-pivoted QR of T stopped at the truncation rank k: the next
        // carry is CH = Z B = (R[:k] P^T)^H, read from R first; then T's
        // columns k.. are free and the explicit Q = B (the output core) is
        // formed there, behind the reflectors (else in V)
        const RowBasis rbz = pivqr_trunc<true>(Tp, p, p, q, ztol, SFFT_SLOT_RANK_DEV + 1, sm.tau, zcn, zperm);
        int k = rbz.k;
        if (k > SFFT_SLOT_RANK_DEV) {
          st = SFFT_ERANK_DEV;
          k = SFFT_SLOT_RANK_DEV;
        }
        for (int idx = threadIdx.x; idx < q * k; idx += blockDim.x) {
          const int i = idx / k, c = idx - i * k;
          CH[(size_t)zperm[i] * k + c] = (c <= i) ? cconj(Tp[(size_t)i * p + c]) : mkc(0.0, 0.0);
        }
        __syncthreads();
        // Q goes behind T's kept columns when W holds both, else in V, else
        // in the CTA's global scratch Z (unused when T sits in W); a panel in
        // global memory leaves all of W to Q
        cd* Qd = gdirect ? sm.W : (2 * k * p <= wcap) ? sm.W + (size_t)p * k : (has_v ? sm.V : Z);
        form_q(Tp, p, p, k, sm.tau, Qd, p);
        for (int idx = threadIdx.x; idx < p * k; idx += blockDim.x) {
          const int row = idx / k, cc = idx - row * k;
          __stcs(Bs + idx, Qd[(size_t)cc * p + row]);
        }
        if (threadIdx.x == 0) rb[s + 1] = k;
        __syncthreads();
        if (zp.carry_out)
          for (int idx = threadIdx.x; idx < q * k; idx += blockDim.x)
            zp.carry_out[zp.off[inst] + SFFT_ZPRE_CARRY_BASE + (size_t)s * SFFT_ZIP_CARRY_STRIDE + idx] = CH[idx];
        fl += rbz.flops + flops_formq(p, k);
        rc = k;
        continue;
      }
      // otherwise: rank-revealing QR of the panel in global memory gives the
      // kept left subspace of T, and the carry is the product Z B
      const RowBasis rbz = rrqr_basis(Z, q, p, p, sm.W, wcap, sm.V, ztol, SFFT_SLOT_RANK_DEV + 1,
                                      sm.tau, zcn, zperm);
      int k = rbz.k;
      if (k > SFFT_SLOT_RANK_DEV) {
        st = SFFT_ERANK_DEV;
        k = SFFT_SLOT_RANK_DEV;
      }
      (void)rmax;
      // B_s[c][mu][c''] = B[(c, mu), c''] (B in W, column-major, leading dim p)
      for (int idx = threadIdx.x; idx < p * k; idx += blockDim.x) {
        const int row = idx / k, cc = idx - row * k;
        __stcs(Bs + idx, sm.W[(size_t)cc * p + row]);
      }
      gemm_zv(Z, q, p, sm.W, k, CH);
      if (threadIdx.x == 0) rb[s + 1] = k;
      __syncthreads();
      if (zp.carry_out)
        for (int idx = threadIdx.x; idx < q * k; idx += blockDim.x)
          zp.carry_out[zp.off[inst] + SFFT_ZPRE_CARRY_BASE + (size_t)s * SFFT_ZIP_CARRY_STRIDE + idx] = CH[idx];
      fl += rbz.flops + flops_gemm(q, p, k);
      rc = k;
    }
    if (deferred) continue;
    if (threadIdx.x == 0) status[inst] = max(status[inst], st);
    __syncthreads();
  WORK_LOOP_END
  if (acc && threadIdx.x == 0) {
    atomicAdd(acc + PH_ZIPUP, fl);
    if (tc_sites > 0.0) atomicAdd(acc + SFFT_NPHASE_DEV + PH_ZIPUP, tc_sites);
  }
  if constexpr (TC) {
    tc::fence_before_sync();
    __syncthreads();
    if ((threadIdx.x >> 5) == 0) {
      tc::fence_after_sync();
      tc::tmem_free(tz.tmem, 128);
    }
  }
}

#define ZIPUP_PARAMS                                                                                  \
  const int *list, int count, int *counter, const int *n_arr, const double *tol_arr,                 \
      const int *maxrank_arr, const cd *A, const long long *a_off, const int *a_ranks_all,           \
      const cd *Wmpo, const long long *w_off, const int *w_ranks_all, cd *B, const long long *b_off, \
      int *b_ranks_all, int core_stride_a, int core_stride_w, int core_stride_b, cd *scratch,        \
      long long scratch_stride, int *status, int hb, double *acc, int vcap, int *defer,              \
      const int *dcount, int qmax1, int wlim, ZipPrefix zp
#define ZIPUP_ARGS                                                                                  \
  list, count, counter, n_arr, tol_arr, maxrank_arr, A, a_off, a_ranks_all, Wmpo, w_off, w_ranks_all, \
      B, b_off, b_ranks_all, core_stride_a, core_stride_w, core_stride_b, scratch, scratch_stride,    \
      status, hb, acc, vcap, defer, dcount, qmax1, wlim, zp

__global__ void __launch_bounds__(256, 3) k_zipup(ZIPUP_PARAMS) { zipup_body<false>(ZIPUP_ARGS); }
__global__ void __launch_bounds__(256, 3) k_zipup_tc(ZIPUP_PARAMS) { zipup_body<true>(ZIPUP_ARGS); }


// ---------------------------------------------------------------------------
// K6: readout in bit-reversed site order (Sec. 3.3, Eq. discretization_dft)
// ---------------------------------------------------------------------------
// Requested outputs u = l_begin + i*2^t, i < q. Sites 0..t-1 carry the fixed
// low bits: a row vector v. Sites t..t+h-1 carry the next h bits: a tree of
// 2^h row vectors v B[...]. Sites t+h..n-1: column vectors R_s[prefix] for the
// contiguous range of prefixes u >> s, built from the top. Then
// y_u = Lv[(u >> t) mod 2^h] . R_{t+h}[u >> (t+h)].
__global__ void k_readout(const int* list, int count, int* counter, const InstParams* __restrict__ P, const cd* B,
                          const long long* b_off, const int* b_ranks_all,
                          int core_stride, const long long* l_begin,
                          const int* tbits, const int* qarr,
                          const long long* out_off, double* prices,
                          double* logk, int* status,
                          cd* scratch, long long scratch_stride) {
  __shared__ cd Lv[(1 << READOUT_TREE_BITS) * SFFT_SLOT_RANK_DEV];
  __shared__ cd Lv2[(1 << READOUT_TREE_BITS) * SFFT_SLOT_RANK_DEV];
  WORK_LOOP_BEGIN(list, count, counter)
    const InstParams prm = P[inst];
    const int n = prm.n;
    const int* rb = b_ranks_all + (size_t)inst * (SFFT_MAXN_DEV + 1);
    const cd* Bb = B + b_off[inst];
    const long long lb = l_begin[inst];
    const int q = qarr[inst];
    const int t = min(tbits[inst], n);
    const long long u_last = lb + ((long long)(q - 1) << tbits[inst]);
    double* pr = prices + out_off[inst];
    double* lk = logk + out_off[inst];
    const double ls0 = log(prm.S0);
    if (status[inst] != 0 || q <= 0) {
      for (int i = threadIdx.x; i < q; i += blockDim.x) {
        pr[i] = __longlong_as_double(0x7ff8000000000000ULL);
        const long long u = lb + ((long long)i << tbits[inst]);
        lk[i] = ls0 + prm.k0 + prm.dk * (double)u;
      }
      continue;
    }
    const int h = min(READOUT_TREE_BITS, n - t);
    // 1. fixed low bits
    if (threadIdx.x == 0) Lv[0] = mkc(1.0, 0.0);
    __syncthreads();
    for (int s = 0; s < t; ++s) {
      const int r0 = rb[s], r1 = rb[s + 1];
      const int bit = (int)((lb >> s) & 1);
      const cd* G = Bb + (size_t)s * core_stride;
      for (int b = threadIdx.x; b < r1; b += blockDim.x) {
        cd acc = mkc(0.0, 0.0);
        for (int a = 0; a < r0; ++a) acc = cfma(Lv[a], G[(size_t)a * 2 * r1 + bit * r1 + b], acc);
        Lv2[b] = acc;
      }
      __syncthreads();
      for (int b = threadIdx.x; b < r1; b += blockDim.x) Lv[b] = Lv2[b];
      __syncthreads();
    }
    // 2. tree over h bits: after level k there are 2^k vectors (index = low k bits)
    for (int k = 0; k < h; ++k) {
      const int s = t + k;
      const int r0 = rb[s], r1 = rb[s + 1];
      const cd* G = Bb + (size_t)s * core_stride;
      const int nv = 1 << k;
      for (int idx = threadIdx.x; idx < 2 * nv * r1; idx += blockDim.x) {
        const int b = idx % r1;
        const int cidx = idx / r1;  // new index: old c plus bit k
        const int c = cidx & (nv - 1), bit = cidx >> k;
        cd acc = mkc(0.0, 0.0);
        for (int a = 0; a < r0; ++a) acc = cfma(Lv[c * SFFT_SLOT_RANK_DEV + a], G[(size_t)a * 2 * r1 + bit * r1 + b], acc);
        Lv2[cidx * SFFT_SLOT_RANK_DEV + b] = acc;
      }
      __syncthreads();
      for (int idx = threadIdx.x; idx < 2 * nv * SFFT_SLOT_RANK_DEV; idx += blockDim.x) Lv[idx] = Lv2[idx];
      __syncthreads();
    }
    // 3. right vectors for prefixes at sites n-1 .. t+h
    const int sh = t + h;
    cd* R0 = scratch + (size_t)blockIdx.x * scratch_stride;
    const long long rcap = scratch_stride / 2;
    cd* R1 = R0 + rcap;
    if (threadIdx.x == 0) R0[0] = mkc(1.0, 0.0);  // R_n[0] = [1]
    __syncthreads();
    long long pmin_prev = 0;
    for (int s = n - 1; s >= sh; --s) {
      const int r0 = rb[s], r1 = rb[s + 1];
      const cd* G = Bb + (size_t)s * core_stride;
      const long long pmin = lb >> s, pmax = u_last >> s;
      const long long cnt = pmax - pmin + 1;
      for (long long idx = threadIdx.x; idx < cnt * r0; idx += blockDim.x) {
        const long long pi = idx / r0;
        const int a = (int)(idx - pi * r0);
        const long long pre = pmin + pi;
        const int bit = (int)(pre & 1);
        const long long par = (pre >> 1) - pmin_prev;
        const cd* Rp = R0 + par * r1;
        cd acc = mkc(0.0, 0.0);
        for (int b = 0; b < r1; ++b) acc = cfma(G[(size_t)a * 2 * r1 + bit * r1 + b], Rp[b], acc);
        R1[pi * r0 + a] = acc;
      }
      __syncthreads();
      cd* tmp = R0;
      R0 = R1;
      R1 = tmp;
      pmin_prev = pmin;
    }
    // 4. combine and price
    const int rmid = rb[sh];
    const long long pbase = (sh < n) ? (lb >> sh) : 0;
    // a call price lies in [max(S0 - K e^{-rT}, 0), S0]. Outside it by more
    // than 1e-6 S0 max(1, e^{-alpha k}) the discrete sum has not resolved the
    // integrand: the factor e^{-alpha k} of the price amplifies the sum's own
    // rounding at far strikes (Sec. 4), so the band widens with it there.
    // The test runs in FP32 (a float price is good to ~6e-8 relative, far
    // inside the band); the wide band is formed only for a price outside the
    // narrow one.
    bool out_of_bounds = false;
    const float s0f = (float)prm.S0, discf = (float)prm.disc, band0 = 1e-6f * s0f;
    // price = S0 f sgn Re(y_u) with f = e^{-alpha k'} sqrt(M) c (price_factor;
    // c = 1/pi on the Simpson grid, dv/(2 pi) on the symmetric one). A thread's
    // strikes are spaced by blockDim 2^t grid points, so after one exponential
    // each next e^{-alpha k'} is the previous one times a fixed ratio (at most
    // 16 products: a few ulps)
    const double sqM = ldexp(1.0, n / 2) * ((n & 1) ? 1.4142135623730951 : 1.0);
    const double fscale =
        prm.S0 * sqM * (prm.quad == Q_SIMPSON ? 0.3183098861837907 : prm.dv * 0.15915494309189535);
    const double ratio = exp(-prm.alpha * prm.dk * (double)((long long)blockDim.x << tbits[inst]));
    double ea = 0.0;
    for (int i = threadIdx.x; i < q; i += blockDim.x) {
      const long long u = lb + ((long long)i << tbits[inst]);
      const int c = (int)((u >> t) & ((1 << h) - 1));
      const long long pi = (sh < n) ? ((u >> sh) - pbase) : 0;
      cd acc = mkc(0.0, 0.0);
      for (int a = 0; a < rmid; ++a) acc = cfma(Lv[c * SFFT_SLOT_RANK_DEV + a], R0[pi * rmid + a], acc);
      const double km = prm.k0 + prm.dk * (double)u;
      ea = (i == (int)threadIdx.x) ? exp(-prm.alpha * km) : ea * ratio;
      const double sgn = (prm.quad == Q_SIMPSON || !(u & 1)) ? 1.0 : -1.0;
      const double price = fscale * ea * sgn * acc.x;
      pr[i] = price;
      lk[i] = ls0 + km;
      const float pf = (float)price, kf = (float)km;
      const float lower = fmaxf(s0f * (1.0f - expf(kf) * discf), 0.0f);
      if (!(pf >= lower - band0 && pf <= s0f + band0)) {
        const float band = band0 * fmaxf(1.0f, expf(-(float)prm.alpha * kf));
        out_of_bounds |= !(pf >= lower - band && pf <= s0f + band);
      }
    }
    if (__syncthreads_or(out_of_bounds) && threadIdx.x == 0) status[inst] = SFFT_EBOUNDS_DEV;
  WORK_LOOP_END
}

// Jacobi sweep limit of every SVD the kernels of this file run (a test hook of
// the host runtime; 60 by default). Stream-ordered, so a call can set it for
// its own launches and restore it after them.
cudaError_t sfft_set_jacobi_cap(int sweeps, cudaStream_t stream) {
  return cudaMemcpyToSymbolAsync(la_jacobi_cap, &sweeps, sizeof(int), 0, cudaMemcpyHostToDevice, stream);
}
