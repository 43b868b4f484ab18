// CTA-cooperative dense linear algebra on small complex FP64 matrices, the
// building blocks of every TT step (TT-SVD, zip-up MPO x TT contraction,
// rounding): Householder QR (LAPACK zlarfg convention), one-sided Jacobi SVD
// (Hestenes' method), and the "tall-skinny SVD" that combines them.
//
// Every function here must be called by all threads of the block; matrices
// passed as "smem" live in shared memory, column-major with a leading
// dimension; "Z" inputs are row-major with leading dimension p and may live in
// global memory (they are read only).
#pragma once
#include "cplx.cuh"

#define LA_MAXP 64  // most columns a tall-skinny factorisation handles

namespace la {

__device__ __forceinline__ int lane_id() { return threadIdx.x & 31; }
__device__ __forceinline__ int warp_id() { return threadIdx.x >> 5; }
__device__ __forceinline__ int n_warps() { return blockDim.x >> 5; }

// x 2^(1023 - eb) as a float (eb: a biased FP64 exponent >= that of |x|),
// built from the bit fields with integer operations, truncated toward zero;
// values below the float range (and zero) give 0.
__device__ __forceinline__ float scaled_f32(double x, int eb) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int ex = (int)((b >> 52) & 0x7ff);
  const int ef = ex - eb + 127;
  if (ex == 0 || ef <= 0) return 0.0f;
  return __uint_as_float((unsigned int)(b >> 32 & 0x80000000ull) | ((unsigned int)ef << 23) |
                         (unsigned int)((b >> 29) & 0x7fffffull));
}
// f 2^(eb - 1023) as a double, exactly, by integer operations (f normal, the
// result in range; zero and subnormal f give 0).
__device__ __forceinline__ double f32_unscaled(float f, int eb) {
  const unsigned int fb = __float_as_uint(f);
  const int ef = (int)((fb >> 23) & 0xff);
  if (ef == 0) return 0.0;
  return __longlong_as_double((long long)(((unsigned long long)(fb & 0x80000000u) << 32) |
                                          ((unsigned long long)(ef - 127 + eb) << 52) |
                                          ((unsigned long long)(fb & 0x7fffffu) << 29)));
}

// The biased exponent eb of a power of two 2^(eb - 1023) >= sqrt(x), x >= 0
// (from the bit fields; 1023 for x = 0).
__device__ __forceinline__ int sqrt_exp_bound(double x) {
  const int e2 = (int)((__double_as_longlong(x) >> 52) & 0x7ff);
  return e2 == 0 ? 1023 : 1023 + ((e2 - 1022 + 1) >> 1);
}

__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Cost model behind the Householder and Jacobi routines below. FP64
// throughput on this part is set by warp instructions, not lanes: an SM
// retires about one FP64 warp instruction per 19 cycles (one per ~64 cycles
// on each of its four sub-partitions) whether 1 or 32 lanes are active, and a
// warp shuffle-add reduction costs one FP64 instruction per step. So every
// FP64 instruction should carry as many useful lanes as possible, with as few
// reduction steps as possible. A reflector is applied to a set of columns by
// groups of S lanes per column (S a power of two dividing 32); the rows below
// the pivot are strided over the S lanes and each column's dot product needs
// only log2(S) shuffle steps. S minimises the FP64 instruction count
//   ceil(ncols S / 32) * (8 ceil(rows / S) + 2 log2 S + 6).
__device__ __forceinline__ int hh_group_log2(int ncols, int rows) {
  int best = 0;
  long long best_cost = 0x7fffffffffffffffLL;
  for (int lg = 0; lg <= 5; ++lg) {
    const int S = 1 << lg;
    const long long w = ((long long)ncols * S + 31) >> 5;
    const long long cost = w * (8 * ((rows + S - 1) / S) + 2 * lg + 6);
    if (cost < best_cost) {
      best_cost = cost;
      best = lg;
    }
  }
  return best;
}

// c_j <- c_j - t v (v^H c_j) for the columns j in [j0, j1) of A (leading dim
// lda), with v_k = 1 implicit and v_i = v[i] for k < i < h. t = conj(tau)
// applies H^H (QR), t = tau applies H (building Q). post(j, c_j[k]) is called
// by one lane per column with the updated row-k entry. Every thread of the
// block must call this; each lane touches only its own rows, so the caller
// needs a barrier before and after.
struct HhNoPost {
  __device__ void operator()(int, cd) const {}
};
template <class Post>
static __device__ void hh_apply(const cd* v, int k, int h, cd t, cd* A, int lda, int j0, int j1,
                                Post post) {
  const int ncols = j1 - j0;
  if (ncols <= 0) return;
  const int lg = hh_group_log2(ncols, h - k - 1);
  const int S = 1 << lg;
  const int lane = lane_id();
  const int sl = lane & (S - 1);
  const int gpw = 32 >> lg;            // groups per warp
  const int gpb = n_warps() * gpw;     // groups per block
  // the bound is uniform over a warp, so every lane reaches the shuffles
  for (int g0 = warp_id() * gpw; g0 < ncols; g0 += gpb) {
    const int g = g0 + (lane >> lg);
    const bool act = g < ncols;
    cd* c = A + (size_t)(j0 + (act ? g : 0)) * lda;
    cd dot = (act && sl == 0) ? c[k] : mkc(0.0, 0.0);
    if (act)
      for (int i = k + 1 + sl; i < h; i += S) dot = cfmac(v[i], c[i], dot);
    for (int o = S >> 1; o > 0; o >>= 1) {
      dot.x += __shfl_xor_sync(0xffffffffu, dot.x, o);
      dot.y += __shfl_xor_sync(0xffffffffu, dot.y, o);
    }
    if (act) {
      const cd f = cmul(t, dot);
      if (sl == 0) {
        const cd ck = csub(c[k], f);
        c[k] = ck;
        post(j0 + g, ck);
      }
      const cd nf = cneg(f);
      for (int i = k + 1 + sl; i < h; i += S) c[i] = cfma(v[i], nf, c[i]);
    }
  }
}

// As hh_apply with t = conj(tau), and also returns through post(j, c_j[k],
// ||c_j[k+1..h)||^2) the squared norm of the updated rows below the pivot,
// summed over the group's lanes (the column norms a pivoted QR needs). It is
// recomputed from the updated entries, not downdated, and formed in FP32:
// cn[j] = ||c_j[k..h)||^2 before the update bounds every entry after it (the
// reflector preserves that norm), so the entries scaled by the power of two
// 2^(1023 - eb) >= 1 / sqrt(cn[j]) convert to floats of modulus <= 1 by
// integer bit operations, and their squares add in FP32 (relative error
// ~1e-6, entries below 2^-126 of the bound dropped); one FP64 scaling per
// column restores the units. No FP64 instruction per entry. With F32NORM
// false the squares add in FP64 (two FMAs per entry) and the norms are exact.
template <bool F32NORM, class Post>
static __device__ void hh_apply_norms(const cd* v, int k, int h, cd t, cd* A, int lda, int j0, int j1,
                                      Post post, const double* cn) {
  const int ncols = j1 - j0;
  if (ncols <= 0) return;
  const int lg = hh_group_log2(ncols, h - k - 1);
  const int S = 1 << lg;
  const int lane = lane_id();
  const int sl = lane & (S - 1);
  const int gpw = 32 >> lg;
  const int gpb = n_warps() * gpw;
  for (int g0 = warp_id() * gpw; g0 < ncols; g0 += gpb) {
    const int g = g0 + (lane >> lg);
    const bool act = g < ncols;
    cd* c = A + (size_t)(j0 + (act ? g : 0)) * lda;
    const int eb = act ? sqrt_exp_bound(cn[j0 + g]) : 1023;
    cd dot = (act && sl == 0) ? c[k] : mkc(0.0, 0.0);
    if (act)
      for (int i = k + 1 + sl; i < h; i += S) dot = cfmac(v[i], c[i], dot);
    for (int o = S >> 1; o > 0; o >>= 1) {
      dot.x += __shfl_xor_sync(0xffffffffu, dot.x, o);
      dot.y += __shfl_xor_sync(0xffffffffu, dot.y, o);
    }
    float nf32 = 0.f;
    double nf64 = 0.0;
    cd ck = mkc(0.0, 0.0);
    if (act) {
      const cd f = cmul(t, dot);
      if (sl == 0) {
        ck = csub(c[k], f);
        c[k] = ck;
      }
      const cd nf = cneg(f);
      for (int i = k + 1 + sl; i < h; i += S) {
        const cd u = cfma(v[i], nf, c[i]);
        c[i] = u;
        if (F32NORM) {
          const float ux = scaled_f32(u.x, eb), uy = scaled_f32(u.y, eb);
          nf32 = fmaf(ux, ux, fmaf(uy, uy, nf32));
        } else {
          nf64 = fma(u.x, u.x, fma(u.y, u.y, nf64));
        }
      }
    }
    for (int o = S >> 1; o > 0; o >>= 1) {
      if (F32NORM)
        nf32 += __shfl_xor_sync(0xffffffffu, nf32, o);
      else
        nf64 += __shfl_xor_sync(0xffffffffu, nf64, o);
    }
    if (act && sl == 0) post(j0 + g, ck, F32NORM ? scalbn((double)nf32, 2 * (eb - 1023)) : nf64);
  }
}

// Householder reflector of col[k..h) (LAPACK zlarfg convention), computed by
// one warp: H^H (a0; x) = (beta; 0) with beta real, H = I - tau v v^H,
// v = (1; x / (a0 - beta)). On return col[k] = beta, col[k+1..h) = v, and the
// returned tau is valid in every lane. The sum of squares is taken unscaled;
// only when it would leave the safe range (entries below ~1e-140 or above
// ~1e140) is the column rescaled by its largest modulus first.
// tot_known >= 0 is the caller's exact squared norm of col[k..h) (a pivoted
// QR carries it for every column), which replaces the warp's own sum; a
// column with x = 0 then gets the reflector beta = -a0 instead of H = I,
// which is as exact. In the safe range beta and 1/beta come from one
// reciprocal square root.
static __device__ cd hh_reflector_warp(cd* col, int k, int h, double tot_known = -1.0) {
  const int lane = lane_id();
  // the pivot is read by lane 0 only and broadcast, so lane 0 may overwrite
  // it below without racing the other lanes
  cd a0 = (lane == 0) ? col[k] : mkc(0.0, 0.0);
  a0.x = __shfl_sync(0xffffffffu, a0.x, 0);
  a0.y = __shfl_sync(0xffffffffu, a0.y, 0);
  double tot;
  if (tot_known >= 0.0) {
    tot = tot_known;
    if (tot == 0.0) return mkc(0.0, 0.0);  // a zero column: H = I
  } else {
    double ss = 0.0;
    for (int i = k + 1 + lane; i < h; i += 32) ss = fma(col[i].x, col[i].x, fma(col[i].y, col[i].y, ss));
    ss = warp_sum(ss);
    if (ss == 0.0 && a0.y == 0.0) return mkc(0.0, 0.0);  // H = I
    tot = cabs2(a0) + ss;
  }
  double beta, rb;
  cd scal;
  if (tot > 1e-280 && tot < 1e280) {
    const double rs = rsqrt(tot);
    beta = -copysign(tot * rs, a0.x);
    rb = -copysign(rs, a0.x);  // 1 / beta
    const cd d = mkc(a0.x - beta, a0.y);  // |d| >= |beta|: no cancellation
    const double rd = 1.0 / cabs2(d);
    scal = mkc(d.x * rd, -d.y * rd);
  } else {
    double amax = fmax(fabs(a0.x), fabs(a0.y));
    for (int i = k + 1 + lane; i < h; i += 32) amax = fmax(amax, fmax(fabs(col[i].x), fabs(col[i].y)));
    amax = warp_max(amax);
    const double inv = (amax > 1e-290) ? 1.0 / amax : 0.0;
    double s = 0.0;
    for (int i = k + 1 + lane; i < h; i += 32) s += cabs2(cscale(col[i], inv));
    s = warp_sum(s);
    if (inv == 0.0 || (s == 0.0 && a0.y == 0.0)) return mkc(0.0, 0.0);
    const cd a0s = cscale(a0, inv);
    beta = -copysign(amax * sqrt(cabs2(a0s) + s), a0.x);
    scal = cdiv(mkc(1.0, 0.0), mkc(a0.x - beta, a0.y));
    rb = 1.0 / beta;
  }
  const cd tau = mkc((beta - a0.x) * rb, -a0.y * rb);
  for (int i = k + 1 + lane; i < h; i += 32) col[i] = cmul(col[i], scal);
  if (lane == 0) col[k] = mkc(beta, 0.0);
  return tau;
}

// Householder QR in place. W: h x p, column-major (leading dim ld). On return
// the upper triangle of the leading min(h,p) rows holds R (W = Q R); the
// strictly lower part holds the reflectors v (v_0 = 1 implicit) and must not
// be read as R. Reflector k: H_k = I - tau_k v v^H with
// H_k^H (a0; x) = (beta; 0), beta real (LAPACK zlarfg); Q = H_0 H_1 ... .
// taus[k] (smem, min(h,p) entries) receives tau_k.
static __device__ void qr_inplace(cd* W, int ld, int h, int p, cd* taus) {
  const int kmax = min(h, p);
  for (int k = 0; k < kmax; ++k) {
    cd* col = W + (size_t)k * ld;
    if (warp_id() == 0) {
      const cd tau = hh_reflector_warp(col, k, h);
      if (lane_id() == 0) taus[k] = tau;
    }
    __syncthreads();
    const cd tau = taus[k];
    if (tau.x != 0.0 || tau.y != 0.0) hh_apply(col, k, h, cconj(tau), W, ld, k + 1, p, HhNoPost());
    __syncthreads();
  }
}

// Explicit Q (h x kq, column-major, leading dim ldq; any address space) of a
// factorisation left by qr_inplace: Q = H_0 ... H_{kq-1} [I; 0], built by
// applying the reflectors in reverse order to the identity columns (columns
// j < k are untouched by H_k).
static __device__ void form_q(const cd* W, int ld, int h, int kq, const cd* taus, cd* Q, int ldq) {
  for (int idx = threadIdx.x; idx < h * kq; idx += blockDim.x) {
    const int j = idx / h, i = idx - j * h;
    Q[(size_t)j * ldq + i] = mkc(i == j ? 1.0 : 0.0, 0.0);
  }
  __syncthreads();
  for (int k = kq - 1; k >= 0; --k) {
    const cd tau = taus[k];
    if (tau.x != 0.0 || tau.y != 0.0) hh_apply(W + (size_t)k * ld, k, h, tau, Q, ldq, k, kq, HhNoPost());
    __syncthreads();
  }
}

// One-sided Jacobi (Hestenes): rotates the m columns of L (p rows, column
// major, leading dim ld) until every pair is orthogonal to working precision,
// |l_a^H l_b| <= tol * ||l_a|| ||l_b||. Columns are visited in round-robin
// tournament order, the m/2 pairs of a round in parallel. A pair is handled
// by a group of G lanes (G a power of two): rows are strided over the group
// and a^H b reduced in log2(G) shuffle steps. G minimises the FP64
// instruction count of a round (the cost model above hh_group_log2): the
// rotation parameters cost about as much as 2 rows of dot products and
// updates, and are shared by all pairs of a warp.
// Rotation of a pair (a, b) with alpha = |a|^2, beta = |b|^2, g = a^H b,
// D = beta - alpha: t = sign(D) 2|g| / (|D| + sqrt(D^2 + 4|g|^2)) is the
// tangent of the annihilating angle, c = 1/sqrt(1 + t^2), and with
// sp = c t conj(g)/|g| the update is a <- c a - sp b, b <- conj(sp) a + c b.
// (Rutishauser's rotation with the phase of g moved onto the new b; b is
// then a singular direction up to a unit factor, which no caller depends on.)
// A sweep in which no rotated pair had |g|^2 > big2 alpha beta (big2 = 1e-8,
// couplings below 1e-4, unless the caller passes another) ends the
// iteration: cyclic Jacobi converges quadratically, so it leaves the pairs
// near big2.
// Returns the number of sweeps used, or -1 if max_sweeps did not reach
// convergence.
__device__ __forceinline__ int jacobi_group_log2(int npair, int p) {
  int best = 0;
  long long best_cost = 0x7fffffffffffffffLL;
  for (int lg = 0; lg <= 5; ++lg) {
    const int G = 1 << lg;
    const long long w = ((long long)npair * G + 31) >> 5;
    const long long cost = w * (16 * ((p + G - 1) / G) + 2 * lg + 40);
    if (cost < best_cost) {
      best_cost = cost;
      best = lg;
    }
  }
  return best;
}

// F32ROT: the column norms, the pair's dot product a^H b, the rotation tests
// and the rotation parameters in FP32, on data scaled by powers of two
// (integer bit operations: no FP64 instruction); only the rotation itself
// is applied in FP64. g then carries ~1e-7 of |a| |b| and c
// and s FP32 rounding, so each rotation is unitary to ~1e-7 and leaves
// ~1e-7 of the coupling: the column norms (the singular values) are
// accurate to ~1e-6 relative, and the columns span the dominant subspaces
// to within ~1e-6 of the dropped singular values. Only a caller that
// projects onto the subspace exactly (pq_svd in the rounding) uses it; the
// FP64 form keeps the exact-unitarity guarantee for the rest.
template <bool F32ROT>
static __device__ int hestenes_t(cd* L, int ld, int p, int m, int max_sweeps, int* sh_flag, double big2) {
  const int lane = lane_id(), warp = warp_id();
  if (m < 2) return 0;
  const int mp = m + (m & 1);
  const int npair = mp / 2;
  const int lg = jacobi_group_log2(npair, p);
  const int G = 1 << lg;
  const int sub = lane & (G - 1);
  const int ppw = 32 >> lg;           // pairs per warp
  const int ppb = n_warps() * ppw;    // pairs per block pass
  // a pair counts as orthogonal once |a^H b| <= tol |a| |b|, the rounding
  // level of a p-term complex dot product; after max_sweeps the result is
  // accepted if no pair is worse than 1e-10 (reported as not converged otherwise)
  const double tol = 1.0e-15 * (double)max(p, 8);
  const double tol2 = tol * tol;
  // squared column norms: exact at the start of every sweep, then carried
  // through the sweep's rotations by alpha' = alpha - w|g|^2, beta' =
  // beta + w|g|^2 (so the rounds only need a^H b); the singular values the
  // callers use come from the columns themselves after the last sweep
  __shared__ double cn2[LA_MAXP];
  // F32ROT: column c is kept as dsc[c] times the stored column, so that a
  // rotation's factor c folds into dsc and the stored update takes two
  // complex FMAs per entry; dsc is folded back before returning
  __shared__ float dsc[LA_MAXP];
  if constexpr (F32ROT) {
    for (int c = threadIdx.x; c < m; c += blockDim.x) dsc[c] = 1.0f;
    __syncthreads();
  }
  int ret = -1;
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    if (threadIdx.x == 0) *sh_flag = 0;
    for (int c = threadIdx.x; c < m; c += blockDim.x) {
      cd* col = L + (size_t)c * ld;
      if constexpr (F32ROT) {
        // a scale below 2^-20 is folded into the column (rare: many large
        // rotations of one column)
        float dc = dsc[c];
        if (dc < 0x1p-20f) {
          const double d = f32_unscaled(dc, 1023);
          for (int i = 0; i < p; ++i) col[i] = cscale(col[i], d);
          dc = 1.0f;
          dsc[c] = dc;
        }
        // to FP32 accuracy, which is all the FP32 rotation parameters use:
        // the entries scaled by 2^(1023 - ec), ec the largest exponent among
        // them, summed in FP32 (no FP64 instruction)
        int ec = 0;
        for (int i = 0; i < p; ++i) {
          ec = max(ec, (int)((__double_as_longlong(col[i].x) >> 52) & 0x7ff));
          ec = max(ec, (int)((__double_as_longlong(col[i].y) >> 52) & 0x7ff));
        }
        ec = min(max(ec + 1, 600), 1440);
        float sf = 0.0f;
        for (int i = 0; i < p; ++i) {
          const float xr = scaled_f32(col[i].x, ec), xi = scaled_f32(col[i].y, ec);
          sf = fmaf(xr, xr, fmaf(xi, xi, sf));
        }
        cn2[c] = f32_unscaled(sf * dc * dc, 2 * ec - 1023);
      } else {
        double s = 0.0;
        for (int i = 0; i < p; ++i) s = fma(col[i].x, col[i].x, fma(col[i].y, col[i].y, s));
        cn2[c] = s;
      }
    }
    __syncthreads();
    for (int t = 0; t < mp - 1; ++t) {
      // the bound is uniform over a warp, so every lane reaches the shuffles
      for (int e0 = warp * ppw; e0 < npair; e0 += ppb) {
        const int e = e0 + (lane >> lg);
        int a = 0, b = 0;
        bool live = e < npair;
        if (live) {
          if (e == 0) {
            a = t;
            b = mp - 1;
          } else {
            a = (t + e) % (mp - 1);
            b = (t - e + mp - 1) % (mp - 1);
          }
          live = a < m && b < m;
        }
        cd* ca = L + (size_t)a * ld;
        cd* cb = L + (size_t)b * ld;
        if constexpr (F32ROT) {
          // a^H b in FP32 on the pair's data scaled by 2^(1023 - es) >= 1 /
          // (larger column norm), entries converted by integer operations:
          // its error, ~1e-7 of |a| |b|, is the level the FP32 rotation
          // parameters leave anyway, and the stop rule asks only for 1e-2.
          // The tests below compare the squares on the scale 2^(2 (1023 - es)).
          const double al = live ? cn2[a] : 0.0, be = live ? cn2[b] : 0.0;
          const float da = live ? dsc[a] : 1.0f, db = live ? dsc[b] : 1.0f;
          // the stored entries are bounded by 2^(es - 1023): the true norms'
          // bounds over the scales (whose exponents are <= 0). Norms outside
          // about 1e+-130 would leave the float range: such a pair is not
          // rotated (its scaled entries read as zero)
          const int eda = ((__float_as_int(da) >> 23) & 0xff) - 127;
          const int edb = ((__float_as_int(db) >> 23) & 0xff) - 127;
          const int es = min(max(max(sqrt_exp_bound(al) - eda, sqrt_exp_bound(be) - edb), 600), 1440);
          float gxf = 0.0f, gyf = 0.0f;
          if (live)
            for (int i = sub; i < p; i += G) {
              const cd x = ca[i], y = cb[i];
              const float xr = scaled_f32(x.x, es), xi = scaled_f32(x.y, es);
              const float yr = scaled_f32(y.x, es), yi = scaled_f32(y.y, es);
              gxf = fmaf(xr, yr, fmaf(xi, yi, gxf));
              gyf = fmaf(xr, yi, fmaf(-xi, yr, gyf));
            }
          for (int o = G >> 1; o > 0; o >>= 1) {
            gxf += __shfl_xor_sync(0xffffffffu, gxf, o);
            gyf += __shfl_xor_sync(0xffffffffu, gyf, o);
          }
          if (!live) continue;
          // g of the true columns, on the scale 2^(2 (1023 - es))
          gxf *= da * db;
          gyf *= da * db;
          const int e2 = 2 * es - 1023;
          const float alf = scaled_f32(al, e2), bef = scaled_f32(be, e2);
          const float G2f = fmaf(gxf, gxf, gyf * gyf);
          const float abf = alf * bef;
          if (G2f > (float)tol2 * abf && G2f > 0.0f) {
            // the rotation of the FP64 branch below, in FP32
            const float Df = bef - alf;
            const float uf = fmaf(Df, Df, 4.0f * G2f);
            const float rf = uf * rsqrtf(uf);
            const float hf = fabsf(Df) + rf;
            const float qf = rsqrtf(2.0f * rf * hf);
            // a' = c (a - t b), b' = c (b + conj(t) a) with t = w conj(g),
            // w = 2 sign(D) / h = 4 sign(D) r q^2; on the stored columns
            // a~' = a~ - t1 b~, b~' = b~ + t2 a~ with t1 = t db / da,
            // t2 = conj(t) da / db, and the factor c moves into the scales
            const float cf = hf * qf;
            const float wf = copysignf(4.0f * rf * qf * qf, Df);
            const float txf = wf * gxf, tyf = -wf * gyf;
            const float r1 = db / da, r2 = da / db;
            const double t1x = f32_unscaled(txf * r1, 1023), t1y = f32_unscaled(tyf * r1, 1023);
            const double t2x = f32_unscaled(txf * r2, 1023), t2y = f32_unscaled(-tyf * r2, 1023);
            // the carried norms, alpha - w|g|^2 and beta + w|g|^2, on the same scale
            const float dnf = copysignf(4.0f * G2f * rf * qf * qf, Df);
            for (int i = sub; i < p; i += G) {
              const cd x = ca[i], y = cb[i];
              ca[i] = mkc(fma(-t1x, y.x, fma(t1y, y.y, x.x)), fma(-t1x, y.y, fma(-t1y, y.x, x.y)));
              cb[i] = mkc(fma(t2x, x.x, fma(-t2y, x.y, y.x)), fma(t2x, x.y, fma(t2y, x.x, y.y)));
            }
            if (sub == 0) {
              cn2[a] = f32_unscaled(fmaxf(alf - dnf, 0.0f), e2);
              cn2[b] = f32_unscaled(bef + dnf, e2);
              dsc[a] = da * cf;
              dsc[b] = db * cf;
              atomicOr(sh_flag, (G2f > (float)big2 * abf) ? 7 : (G2f > 1e-20f * abf) ? 3 : 1);
            }
          }
        } else {
          double gx = 0.0, gy = 0.0;
          if (live)
            for (int i = sub; i < p; i += G) {
              const cd x = ca[i], y = cb[i];
              gx = fma(x.x, y.x, fma(x.y, y.y, gx));
              gy = fma(x.x, y.y, fma(-x.y, y.x, gy));
            }
          for (int o = G >> 1; o > 0; o >>= 1) {
            gx += __shfl_xor_sync(0xffffffffu, gx, o);
            gy += __shfl_xor_sync(0xffffffffu, gy, o);
          }
          if (!live) continue;
          const double al = cn2[a], be = cn2[b];
          const double g2 = fma(gx, gx, gy * gy);
          const double ab = al * be;
          if (g2 > tol2 * ab && g2 > 1e-290) {
            // t, c and sp are invariant under a common scaling of al, be, g;
            // rescale only when the squares below could overflow
            double D = be - al, G2 = g2, sx = gx, sy = gy;
            const double big = fmax(al, be);
            if (big > 1e140) {
              const double inv = 1.0 / big;
              D *= inv;
              sx *= inv;
              sy *= inv;
              G2 = fma(sx, sx, sy * sy);
            }
            // Rotation with tangent t = w |g|, w = 2 sign(D) / h, where
            // u = D^2 + 4 |g|^2, r = sqrt(u), h = |D| + r. Since
            // 1 + w^2 |g|^2 = 2 r / h, with q = 1 / sqrt(2 r h):
            //   c = 1 / sqrt(1 + t^2) = h q,   c w = 2 sign(D) q,
            //   w |g|^2 = 2 sign(D) |g|^2 / h = 4 sign(D) |g|^2 r q^2,
            // two reciprocal square roots and no division
            const double u = fma(D, D, 4.0 * G2);
            const double r = u * rsqrt(u);
            const double h = fabs(D) + r;
            const double qq = rsqrt(2.0 * r * h);
            const double c = h * qq;
            const double cw = copysign(2.0 * qq, D);
            const double spx = cw * sx, spy = -cw * sy;           // sp = c w conj(g)
            // w|g|^2 in true units (w G2 carries one factor of the scaling)
            const double wg2 = copysign(4.0 * G2 * r * qq * qq, D);
            const double dn = (big > 1e140) ? wg2 * big : wg2;
            for (int i = sub; i < p; i += G) {
              const cd x = ca[i], y = cb[i];
              ca[i] = mkc(fma(c, x.x, -fma(spx, y.x, -spy * y.y)), fma(c, x.y, -fma(spx, y.y, spy * y.x)));
              cb[i] = mkc(fma(c, y.x, fma(spx, x.x, spy * x.y)), fma(c, y.y, fma(spx, x.y, -spy * x.x)));
            }
            if (sub == 0) {
              cn2[a] = fmax(al - dn, 0.0);
              cn2[b] = be + dn;
              atomicOr(sh_flag, (g2 > big2 * ab) ? 7 : (g2 > 1e-20 * ab) ? 3 : 1);
            }
          }
        }
      }
      __syncthreads();
    }
    const int any = *sh_flag;
    __syncthreads();
    // every rotation of this sweep was below sqrt(big2) relative (1e-4 by
    // default): Jacobi's quadratic convergence leaves every pair near big2 /
    // (relative gap) after it. The
    // rotations are unitary, so A V = [columns] stays exact whatever is left;
    // the residual only makes the kept columns orthogonal to ~1e-8, and their
    // norms (the singular values used for truncation) accurate to ~1e-16
    if (!(any & 4)) {
      ret = sweep + 1;
      break;
    }
    if (sweep == max_sweeps - 1) {
      ret = (any & 2) ? -1 : max_sweeps;
      break;
    }
  }
  if constexpr (F32ROT) {
    // the true columns: each stored column times its scale
    for (int idx = threadIdx.x; idx < m * p; idx += blockDim.x) {
      const int c = idx / p, i = idx - c * p;
      L[(size_t)c * ld + i] = cscale(L[(size_t)c * ld + i], f32_unscaled(dsc[c], 1023));
    }
    __syncthreads();
  }
  return ret;
}

static __device__ int hestenes(cd* L, int ld, int p, int m, int max_sweeps, int* sh_flag, double big2 = 1e-8) {
  return hestenes_t<false>(L, ld, p, m, max_sweeps, sh_flag, big2);
}

// Shared-memory layout needed by ts_svd for p columns and row blocks of hb.
__host__ __device__ inline size_t ts_svd_smem_bytes(int p, int hb) {
  return sizeof(cd) * ((size_t)(p + hb) * p + (size_t)p * p + p) + sizeof(double) * p + 64;
}

struct TsSvd {
  int m;          // number of singular triplets = min(q, p) (pq_svd: the QR rank kept)
  int sweeps;     // Jacobi sweeps (-1: not converged)
  double flops;   // algorithmic FP64 flops of this factorisation
  double tail2;   // squared norm dropped before the SVD (pq_svd; 0 for ts_svd)
};

// Algorithmic FP64 flop counts (complex multiply-add = 8 real flops), in
// closed form and integer arithmetic: every thread evaluates them, and on
// this part FP64 instructions are the scarce resource, so the bookkeeping
// must not spend any.
// Householder QR of h x p: sum_{i<k} 16 (h-i)(p-1-i) + 10 (h-i), k = min(h, p).
__host__ __device__ inline double flops_qr(long long h, long long p) {
  const long long k = h < p ? h : p;
  if (k <= 0) return 0.0;
  const long long s1 = k * h * (p - 1) - (h + p - 1) * (k * (k - 1) / 2) + (k - 1) * k * (2 * k - 1) / 6;
  const long long s2 = k * h - k * (k - 1) / 2;
  return (double)(16 * s1 + 10 * s2);
}
// One Householder step (column i of an h x p factorisation): the i-th term above.
__host__ __device__ inline double flops_qr_step(long long h, long long p, long long i) {
  return (double)(16 * (h - i) * (p - 1 - i) + 10 * (h - i));
}
// Explicit Q: sum_{i<kq} 16 (h-i)(kq-i).
__host__ __device__ inline double flops_formq(long long h, long long kq) {
  if (kq <= 0) return 0.0;
  const long long s = kq * h * kq - (h + kq) * (kq * (kq - 1) / 2) + (kq - 1) * kq * (2 * kq - 1) / 6;
  return (double)(16 * s);
}
__host__ __device__ inline double flops_hestenes(long long p, long long m, long long sweeps) {
  return (double)(sweeps * m * (m - 1) / 2 * 26 * p);
}
__host__ __device__ inline double flops_gemm(long long m, long long n, long long k) { return (double)(8 * m * n * k); }

// Truncated Householder QR with column pivoting of A (m x ncol, column-major,
// leading dim lda, smem): A P = Q R with the column of largest remaining norm
// first, stopped at the smallest k >= 1 with ||R[k:, k:]||_F <= delta_rel
// ||A||_F (or at k = min(m, ncol, kmax); delta_rel < 0 never stops early). On
// return rows 0..k-1 of R are final in the upper part of A (pivoted column
// order), the reflectors of steps 0..k-1 lie below the diagonal with
// taus[0..k), and perm[i] is the original index of pivoted column i.
// ||R[k:, k:]||_F is the error of keeping k rows. The remaining column norms
// are summed exactly from the updated rows at every step (by the lanes that
// update them), so no downdating error builds up near the truncation level.
// Smem: taus (min(m, ncol) entries), cn and perm (ncol entries).
#define LA_MAXQ 128
struct RowBasis {
  int k;
  double flops;
  double tail2;  // ||R[k:, k:]||_F^2 at the stop: the squared norm of the dropped rows
};

// F32NORM: the trailing column norms in FP32 (hh_apply_norms), for panels
// tall enough that their per-entry FP64 cost matters; the reflector then sums
// its own column, the carried norms serving only the pivot choice and the
// stop (decisions within ~1e-6 of the threshold may move). Otherwise the norms
// are exact and the reflector takes its column's norm from them.
template <bool F32NORM = false>
static __device__ RowBasis pivqr_trunc(cd* A, int lda, int m, int ncol, double delta_rel, int kmax, cd* taus,
                                       double* cn, int* perm, double delta_abs2 = -1.0) {
  // delta_abs2 >= 0 replaces the relative threshold by an absolute one:
  // stop once ||R[k:, k:]||_F^2 <= delta_abs2
  __shared__ int ctl;  // 1 once the rank is found
  __shared__ double tail_sh;
  const int lane = lane_id(), warp = warp_id();
  RowBasis out;
  out.k = 1;
  out.flops = 0.0;
  out.tail2 = 0.0;
  // exact column norms
  for (int j = warp; j < ncol; j += n_warps()) {
    const cd* cj = A + (size_t)j * lda;
    double ss = 0.0;
    for (int i = lane; i < m; i += 32) ss = fma(cj[i].x, cj[i].x, fma(cj[i].y, cj[i].y, ss));
    ss = warp_sum(ss);
    if (lane == 0) {
      cn[j] = ss;
      perm[j] = j;
    }
  }
  __syncthreads();
  double total = 0.0;
  for (int j = lane; j < ncol; j += 32) total += cn[j];
  total = warp_sum(total);
  const double delta2 = delta_abs2 >= 0.0 ? delta_abs2 : delta_rel < 0.0 ? -1.0 : delta_rel * delta_rel * total;
  const int kstop = min(min(m, ncol), kmax);
  for (int k = 0;; ++k) {
    if (warp == 0) {
      // trailing norm ||R[k:, k:]||^2 and the pivot column. The norms are
      // >= 0, so their bit patterns order like the values: the argmax runs
      // on integers (ties to the lowest index), off the FP64 pipe
      double tr = 0.0;
      long long best = -1;
      int bi = 0x7fffffff;
      for (int j = k + lane; j < ncol; j += 32) {
        const double v = cn[j];
        tr += v;
        const long long key = __double_as_longlong(v);
        if (key > best) {
          best = key;
          bi = j;
        }
      }
      tr = warp_sum(tr);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const long long ov = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ov > best || (ov == best && oi < bi)) {
          best = ov;
          bi = oi;
        }
      }
      const bool stop = (k >= 1 && tr <= delta2) || k >= kstop;
      if (!stop) {
        if (bi != k) {
          cd* ck = A + (size_t)k * lda;
          cd* cb = A + (size_t)bi * lda;
          for (int i = lane; i < m; i += 32) {
            const cd tmp = ck[i];
            ck[i] = cb[i];
            cb[i] = tmp;
          }
          if (lane == 0) {
            const double t1 = cn[k];
            cn[k] = cn[bi];
            cn[bi] = t1;
            const int t3 = perm[k];
            perm[k] = perm[bi];
            perm[bi] = t3;
          }
        }
        __syncwarp();
        const cd tau = F32NORM ? hh_reflector_warp(A + (size_t)k * lda, k, m)
                               : hh_reflector_warp(A + (size_t)k * lda, k, m, cn[k]);
        if (lane == 0) taus[k] = tau;
      }
      if (lane == 0) {
        ctl = stop ? 1 : 0;
        tail_sh = tr;
      }
    }
    __syncthreads();
    if (ctl) {
      out.k = max(k, 1);
      out.tail2 = tail_sh;
      break;
    }
    const cd tau = taus[k];
    if (tau.x != 0.0 || tau.y != 0.0) {
      hh_apply_norms<F32NORM>(A + (size_t)k * lda, k, m, cconj(tau), A, lda, k + 1, ncol,
                              [&](int j, cd, double nn) { cn[j] = nn; }, cn);
    } else {
      // H = I: rows below k are unchanged; drop row k from the norms
      for (int j = k + 1 + threadIdx.x; j < ncol; j += blockDim.x) {
        const cd* cj = A + (size_t)j * lda;
        double ss = 0.0;
        for (int i = k + 1; i < m; ++i) ss = fma(cj[i].x, cj[i].x, fma(cj[i].y, cj[i].y, ss));
        cn[j] = ss;
      }
    }
    __syncthreads();
    out.flops += flops_qr_step(m, ncol, k);
  }
  return out;
}

// Right singular vectors of a tall-skinny Z (q x p, row-major, leading dim
// ldz, read only; any address space). Streaming Householder QR over row blocks
// of hb rows gives R (Z = Q R); the columns of L = R^H are then orthogonalised
// by Hestenes' method, so L W = Y with Y/||Y|| the left singular vectors of
// R^H, i.e. the right singular vectors of Z.
// Output: V (p x m, column-major, leading dim p) in smem, sig[m] in
// descending order, with V[:, i] the vector of sig[i].
// W: smem work of wcap >= (p + 1) * p + p elements; row blocks are as tall
// as W allows (hb = wcap / p - p rows below the running R).
// Streaming Householder QR of a tall Z (q x p, row-major, leading dim ldz,
// read only): row blocks of hb = wcap/p - p rows are stacked under the running
// R and factored again. On return R (nR x p, upper triangular, nR = min(q, p))
// is in the top rows of W, column-major with leading dim p + hb.
static __device__ int stream_qr(const cd* Z, long long q, int p, int ldz, cd* W, int wcap, cd* taus,
                                int* ldw_out) {
  const int hb = wcap / p - p;
  const int ldw = p + hb;
  int nR = 0;  // rows of R currently held at the top of W
  for (long long r0 = 0; r0 < q || (r0 == 0 && q == 0); r0 += hb) {
    const int b = (int)min((long long)hb, q - r0);
    // load block rows r0..r0+b below R
    for (int idx = threadIdx.x; idx < b * p; idx += blockDim.x) {
      const int i = idx / p, j = idx - i * p;
      W[(size_t)j * ldw + nR + i] = Z[(size_t)(r0 + i) * ldz + j];
    }
    __syncthreads();
    const int h = nR + b;
    qr_inplace(W, ldw, h, p, taus);
    nR = min(h, p);
    // clear below the diagonal of R (reflector storage)
    for (int idx = threadIdx.x; idx < nR * p; idx += blockDim.x) {
      const int j = idx / nR, i = idx - j * nR;
      if (i > j) W[(size_t)j * ldw + i] = mkc(0.0, 0.0);
    }
    __syncthreads();
    if (q == 0) break;
  }
  *ldw_out = ldw;
  return nR;
}

// Jacobi sweep limit of ts_svd (60). A context's fault-injection hook lowers
// it to make the SVDs report non-convergence (SFFT_ENOCONV) without any
// device fault; every kernel reads it at each factorisation.
static __device__ int la_jacobi_cap = 60;

// After Hestenes' method on the m columns of V (p rows, leading dim p): the
// column norms are the singular values; sort them descending (stable by
// index) into sig[0..m) and normalise the columns in the same order. W:
// smem scratch of p * (m + 1) elements.
static __device__ void svd_finish(cd* V, int p, int m, cd* W, double* sig) {
  double* nrm = reinterpret_cast<double*>(W);
  for (int c = warp_id(); c < m; c += n_warps()) {
    double s = 0.0;
    for (int i = lane_id(); i < p; i += 32) s += cabs2(V[(size_t)c * p + i]);
    s = warp_sum(s);
    if (lane_id() == 0) nrm[c] = sqrt(s);
  }
  __syncthreads();
  cd* Vs = W + p;  // after the norms
  for (int c = threadIdx.x; c < m; c += blockDim.x) {
    int rank = 0;
    const double sc = nrm[c];
    for (int o = 0; o < m; ++o) {
      const double so = nrm[o];
      rank += (so > sc) || (so == sc && o < c);
    }
    sig[rank] = sc;
    const double inv = sc > 1e-290 ? 1.0 / sc : 0.0;
    for (int i = 0; i < p; ++i) Vs[(size_t)rank * p + i] = cscale(V[(size_t)c * p + i], inv);
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < p * m; idx += blockDim.x) V[idx] = Vs[idx];
  __syncthreads();
}

// pre2 >= 0 (with perm, p ints of smem) adds pq_svd's prefilter on R: a
// column-pivoted QR of R drops trailing rows of squared norm <= pre2
// (returned in tail2, for the caller's truncation to count) and Hestenes'
// method runs on the k' kept rows only (m = k').
static __device__ TsSvd ts_svd(const cd* Z, long long q, int p, int ldz, cd* W, int wcap, cd* V,
                        double* sig, cd* taus, int* sh_flag, double pre2 = -1.0, int* perm = nullptr) {
  const int hb = wcap / p - p;
  int ldw;
  const int nR = stream_qr(Z, q, p, ldz, W, wcap, taus, &ldw);
  int m = nR;
  double tail2 = 0.0, fpre = 0.0;
  if (pre2 >= 0.0 && perm) {
    const RowBasis rb = pivqr_trunc(W, ldw, nR, p, -1.0, nR, taus, sig, perm, pre2);
    m = rb.k;
    tail2 = rb.tail2;
    fpre = rb.flops;
    // L[perm[j], i] = conj(R2[i, j]) for j >= i (R2 the pivoted QR's rows)
    for (int idx = threadIdx.x; idx < p * m; idx += blockDim.x) {
      const int i = idx / p, j = idx - i * p;
      V[(size_t)i * p + perm[j]] = (j >= i) ? cconj(W[(size_t)j * ldw + i]) : mkc(0.0, 0.0);
    }
  } else {
    // L = R^H (p x m) into V
    for (int idx = threadIdx.x; idx < p * m; idx += blockDim.x) {
      const int c = idx / p, i = idx - c * p;
      V[(size_t)c * p + i] = (i >= c) ? cconj(W[(size_t)i * ldw + c]) : mkc(0.0, 0.0);
    }
  }
  __syncthreads();
  TsSvd out;
  out.m = m;
  const int cap = la_jacobi_cap;
  out.sweeps = hestenes(V, p, p, m, cap, sh_flag);
  {
    // QR of the stacked row blocks, Jacobi sweeps, norms and sort
    double f = 0.0;
    long long rows = q, carried = 0;
    while (rows > 0) {
      const long long b = rows < hb ? rows : hb;
      f += flops_qr(carried + b, p);
      carried = carried + b < p ? carried + b : p;
      rows -= b;
    }
    out.flops = f + fpre + flops_hestenes(p, m, out.sweeps < 0 ? cap : out.sweeps) + (double)(4 * p * m);
  }
  out.tail2 = tail2;
  svd_finish(V, p, m, W, sig);
  return out;
}

// Smallest k >= 1 with sqrt(sum_{i >= k} sig_i^2) <= delta (sig descending);
// evaluated redundantly by every thread.
__device__ __forceinline__ int trunc_rank(const double* sig, int m, double delta) {
  double tail = 0.0;
  const double d2 = delta * delta;
  int k = m;
  for (int i = m - 1; i >= 0; --i) {
    tail = fma(sig[i], sig[i], tail);
    if (tail <= d2) k = i; else break;
  }
  return max(k, 1);
}

// As trunc_rank with tail2 already dropped: the smallest k >= 1 with
// tail2 + sum_{i >= k} sig_i^2 <= delta^2.
__device__ __forceinline__ int trunc_rank_tail(const double* sig, int m, double delta, double tail2) {
  double tail = tail2;
  const double d2 = delta * delta;
  int k = m;
  for (int i = m - 1; i >= 0; --i) {
    tail = fma(sig[i], sig[i], tail);
    if (tail <= d2) k = i; else break;
  }
  return max(k, 1);
}

// Dominant right singular vectors of A (q x p, column-major in smem, leading
// dim lda; overwritten). A Householder QR with column pivoting, A P = Q R,
// stops at the first k' whose dropped rows have ||R[k':, k':]||_F^2 <= pre2;
// Hestenes' method then takes the SVD of the kept rows, B = R[:k', :] P^T
// (k' x p): the columns of L = B^H (p x k') are orthogonalised, and their
// norms and directions are the singular values and right singular vectors of
// B. Since A^H A = B^H B + (dropped)^H (dropped), the singular values satisfy
// sig_i(B) <= sig_i(A), and for every k
//   sum_{i>=k} sig_i(A)^2 <= sum_{i>=k} sig_i(B)^2 + tail2 <= that + pre2,
// so truncating B's SVD with the dropped norm tail2 counted against the
// budget keeps the error bound of a truncated SVD of A, at a rank at most one
// interval of pre2 above the optimal one. Output as ts_svd (m = k'), with
// tail2 returned. big2: the squared relative rotation size below which a
// sweep ends the Jacobi iteration (see hestenes). Smem: V (p x k'), sig and
// perm (p entries), taus (min(q, p)).
static __device__ TsSvd pq_svd(cd* A, int lda, int q, int p, double pre2, cd* V, double* sig, cd* taus,
                               int* perm, int* sh_flag, double big2 = 1e-8) {
  const RowBasis rb = pivqr_trunc(A, lda, q, p, -1.0, min(q, p), taus, sig, perm, pre2);
  const int m = rb.k;
  // L[perm[j], i] = conj(R[i, j]) for j >= i (R upper trapezoidal in pivoted order)
  for (int idx = threadIdx.x; idx < p * m; idx += blockDim.x) {
    const int i = idx / p, j = idx - i * p;
    V[(size_t)i * p + perm[j]] = (j >= i) ? cconj(A[(size_t)j * lda + i]) : mkc(0.0, 0.0);
  }
  __syncthreads();
  TsSvd out;
  out.m = m;
  const int cap = la_jacobi_cap;
  out.sweeps = hestenes_t<true>(V, p, p, m, cap, sh_flag, big2);
  out.flops = rb.flops + flops_hestenes(p, m, out.sweeps < 0 ? cap : out.sweeps) + (double)(4 * p * m);
  out.tail2 = rb.tail2;
  svd_finish(V, p, m, A, sig);
  return out;
}

// CTA-wide argmax of |x_i|^2 over i < len with x given by a functor; ties go
// to the lowest index. red_d / red_i: smem scratch of blockDim/32 entries.
template <class F>
__device__ int cta_argmax(int len, F val, double* red_d, int* red_i) {
  double best = -1.0;
  int bi = 0x7fffffff;
  for (int i = threadIdx.x; i < len; i += blockDim.x) {
    const double v = val(i);
    if (v > best || (v == best && i < bi)) {
      best = v;
      bi = i;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const double ov = __shfl_xor_sync(0xffffffffu, best, o);
    const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
    if (ov > best || (ov == best && oi < bi)) {
      best = ov;
      bi = oi;
    }
  }
  if (lane_id() == 0) {
    red_d[warp_id()] = best;
    red_i[warp_id()] = bi;
  }
  __syncthreads();
  double b2 = -1.0;
  int i2 = 0x7fffffff;
  for (int w = 0; w < n_warps(); ++w)
    if (red_d[w] > b2 || (red_d[w] == b2 && red_i[w] < i2)) {
      b2 = red_d[w];
      i2 = red_i[w];
    }
  __syncthreads();
  return i2;
}

// Maxvol (Goreinov, Oseledets, Savostyanov, Tyrtyshnikov, Zamarashkin, 2010):
// r rows of A (N x r, column-major, leading dim lda, N >= r, smem) whose
// r x r submatrix has locally maximal volume, i.e. every entry of
// B = A A[piv]^{-1} has modulus <= 1 + 1e-2. Start: rows chosen by Gaussian
// elimination with partial pivoting. piv[r] (smem) receives the rows.
// work: smem of 2 N r + 2 r r + N complex; iw: N ints; red_*: reduction scratch.
static __device__ void maxvol(const cd* A, int lda, int N, int r, int* piv, cd* work, int* iw,
                              double* red_d, int* red_i) {
  cd* C = work;                 // N x r elimination copy, then B
  cd* S = C + (size_t)N * r;    // r x 2r Gauss-Jordan block [A[piv] | I]
  cd* fac = S + (size_t)2 * r * r;  // N factors
  for (int idx = threadIdx.x; idx < N * r; idx += blockDim.x) C[idx] = A[(idx / N) * lda + idx % N];
  for (int i = threadIdx.x; i < N; i += blockDim.x) iw[i] = 0;
  __syncthreads();
  // 1. partial-pivoting elimination picks the starting rows
  for (int c = 0; c < r; ++c) {
    const int pr = cta_argmax(N, [&](int i) { return iw[i] ? -1.0 : cabs2(C[c * N + i]); }, red_d, red_i);
    if (threadIdx.x == 0) {
      piv[c] = pr;
      iw[pr] = 1;
    }
    __syncthreads();
    const cd pv = C[c * N + pr];
    const bool nz = cabs2(pv) > 0.0;
    for (int i = threadIdx.x; i < N; i += blockDim.x)
      fac[i] = (!iw[i] && nz) ? cdiv(C[c * N + i], pv) : mkc(0.0, 0.0);
    __syncthreads();
    for (int idx = threadIdx.x; idx < N * (r - c - 1); idx += blockDim.x) {
      const int cc = c + 1 + idx / N, i = idx % N;
      C[cc * N + i] = csub(C[cc * N + i], cmul(fac[i], C[cc * N + pr]));
    }
    __syncthreads();
  }
  // 2. S = [A[piv] | I]; Gauss-Jordan with partial pivoting -> A[piv]^{-1}
  for (int idx = threadIdx.x; idx < r * 2 * r; idx += blockDim.x) {
    const int i = idx / (2 * r), j = idx % (2 * r);
    S[idx] = (j < r) ? A[j * lda + piv[i]] : mkc((j - r) == i ? 1.0 : 0.0, 0.0);
  }
  __syncthreads();
  for (int c = 0; c < r; ++c) {
    const int pr = c + cta_argmax(r - c, [&](int i) { return cabs2(S[(c + i) * 2 * r + c]); }, red_d, red_i);
    if (pr != c)
      for (int j = threadIdx.x; j < 2 * r; j += blockDim.x) {
        const cd t = S[c * 2 * r + j];
        S[c * 2 * r + j] = S[pr * 2 * r + j];
        S[pr * 2 * r + j] = t;
      }
    __syncthreads();
    const cd pv = S[c * 2 * r + c];
    const cd inv = cabs2(pv) > 0.0 ? cdiv(mkc(1.0, 0.0), pv) : mkc(0.0, 0.0);
    __syncthreads();
    for (int j = threadIdx.x; j < 2 * r; j += blockDim.x) S[c * 2 * r + j] = cmul(S[c * 2 * r + j], inv);
    __syncthreads();
    for (int i = threadIdx.x; i < r; i += blockDim.x) fac[i] = (i == c) ? mkc(0.0, 0.0) : S[i * 2 * r + c];
    __syncthreads();
    for (int idx = threadIdx.x; idx < r * 2 * r; idx += blockDim.x) {
      const int i = idx / (2 * r), j = idx % (2 * r);
      if (i != c) S[idx] = csub(S[idx], cmul(fac[i], S[c * 2 * r + j]));
    }
    __syncthreads();
  }
  // 3. B = A A[piv]^{-1} (N x r, column-major) into C
  for (int idx = threadIdx.x; idx < N * r; idx += blockDim.x) {
    const int j = idx / N, i = idx % N;
    cd acc = mkc(0.0, 0.0);
    for (int a = 0; a < r; ++a) acc = cfma(A[a * lda + i], S[a * 2 * r + r + j], acc);
    C[idx] = acc;
  }
  __syncthreads();
  // 4. swap in the largest entry until all are <= 1 + 1e-2 (bounded)
  for (int it = 0; it < 8 * r + 8; ++it) {
    const int e = cta_argmax(N * r, [&](int idx) { return cabs2(C[idx]); }, red_d, red_i);
    const int j = e / N, i = e % N;
    const cd bij = C[e];
    if (cabs2(bij) <= (1.0 + 1e-2) * (1.0 + 1e-2)) break;
    // B <- B - B[:, j] (B[i, :] - e_j) / B[i, j]
    for (int a = threadIdx.x; a < N; a += blockDim.x) fac[a] = cdiv(C[j * N + a], bij);
    cd* rowi = S;  // reuse: r entries
    for (int c = threadIdx.x; c < r; c += blockDim.x)
      rowi[c] = (c == j) ? csub(C[c * N + i], mkc(1.0, 0.0)) : C[c * N + i];
    __syncthreads();
    for (int idx = threadIdx.x; idx < N * r; idx += blockDim.x) {
      const int c = idx / N, a = idx % N;
      C[idx] = csub(C[idx], cmul(fac[a], rowi[c]));
    }
    if (threadIdx.x == 0) piv[j] = i;
    __syncthreads();
  }
}

// Truncated row-space basis of a tall Z (q x p) by rank-revealing QR.
// Z = Q R by the streaming QR; then R P = Q2 R2 by pivqr_trunc, so that the
// trailing block R2[k:, k:] has Frobenius norm equal to the error of keeping
// k rows; k is the smallest rank with that norm <= delta_rel * ||Z||_F
// (k >= 1, k <= kmax). The kept rows span (R2[:k] P^T); B (p x k,
// column-major, leading dim p, in W on return) is an orthonormal basis of
// their conjugate span, so Z ~= Z B B^H with error at most the trailing norm.
// Smem: W (wcap >= (p + 1) p), V (p x p), taus and cn (p entries each), perm (p ints).
static __device__ RowBasis rrqr_basis(const cd* Z, long long q, int p, int ldz, cd* W, int wcap, cd* V,
                                      double delta_rel, int kmax, cd* taus, double* cn, int* perm) {
  int ldw;
  const int m = stream_qr(Z, q, p, ldz, W, wcap, taus, &ldw);
  double fl = 0.0;
  {
    long long rows = q, carried = 0;
    const int hb = wcap / p - p;
    while (rows > 0) {
      const long long b = rows < hb ? rows : hb;
      fl += flops_qr(carried + b, p);
      carried = carried + b < p ? carried + b : p;
      rows -= b;
    }
  }
  RowBasis out = pivqr_trunc(W, ldw, m, p, delta_rel, kmax, taus, cn, perm);
  out.flops += fl;
  const int k = out.k;
  // M = (R2[:k] P^T)^H (p x k) into V: M[perm[j], c] = conj(R2[c, j])
  for (int idx = threadIdx.x; idx < p * k; idx += blockDim.x) {
    const int c = idx / p, j = idx - c * p;
    V[(size_t)c * p + perm[j]] = (j >= c) ? cconj(W[(size_t)j * ldw + c]) : mkc(0.0, 0.0);
  }
  __syncthreads();
  // B = orthonormal basis of span(M), written to W (leading dim p)
  qr_inplace(V, p, p, k, taus);
  form_q(V, p, p, min(p, k), taus, W, p);
  out.flops += flops_qr(p, k) + flops_formq(p, min(p, k));
  return out;
}

}  // namespace la
