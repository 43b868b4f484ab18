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

__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Householder QR in place. W: h x p, column-major (leading dim ld). On return
// the upper triangle of the leading min(h,p) rows holds R (W = Q R); the
// strictly lower part holds the reflectors v (v_0 = 1 implicit) and must not
// be read as R. Reflector k: H_k = I - tau_k v v^H with
// H_k^H (a0; x) = (beta; 0), beta real (LAPACK zlarfg); Q = H_0 H_1 ... .
// taus[k] (smem, min(h,p) entries) receives tau_k.
static __device__ void qr_inplace(cd* W, int ld, int h, int p, cd* taus) {
  const int lane = lane_id(), warp = warp_id(), nw = n_warps();
  const int kmax = min(h, p);
  for (int k = 0; k < kmax; ++k) {
    cd* col = W + (size_t)k * ld;
    if (warp == 0) {
      // the pivot is read by lane 0 only and broadcast, so lane 0 may
      // overwrite it below without racing the other lanes
      cd a0 = (lane == 0) ? col[k] : mkc(0.0, 0.0);
      a0.x = __shfl_sync(0xffffffffu, a0.x, 0);
      a0.y = __shfl_sync(0xffffffffu, a0.y, 0);
      // norms are taken on the column scaled by its largest modulus, so that
      // squares of tiny entries neither underflow nor turn beta into zero
      double amax = fmax(fabs(a0.x), fabs(a0.y));
      for (int i = k + 1 + lane; i < h; i += 32) amax = fmax(amax, fmax(fabs(col[i].x), fabs(col[i].y)));
      amax = warp_max(amax);
      const double inv = (amax > 1e-290) ? 1.0 / amax : 0.0;
      double s = 0.0;
      for (int i = k + 1 + lane; i < h; i += 32) s += cabs2(cscale(col[i], inv));
      s = warp_sum(s);
      cd tau = mkc(0.0, 0.0);
      if (inv != 0.0 && !(s == 0.0 && a0.y == 0.0)) {
        const cd a0s = cscale(a0, inv);
        const double beta = -copysign(amax * sqrt(cabs2(a0s) + s), a0.x);
        tau = mkc((beta - a0.x) / beta, -a0.y / beta);
        const cd scal = cdiv(mkc(1.0, 0.0), mkc(a0.x - beta, a0.y));
        for (int i = k + 1 + lane; i < h; i += 32) col[i] = cmul(col[i], scal);
        if (lane == 0) col[k] = mkc(beta, 0.0);
      }
      if (lane == 0) taus[k] = tau;
    }
    __syncthreads();
    const cd tau = taus[k];
    if (tau.x != 0.0 || tau.y != 0.0) {
      const cd ctau = cconj(tau);
      for (int j = k + 1 + warp; j < p; j += nw) {
        cd* cj = W + (size_t)j * ld;
        cd dot = (lane == 0) ? cj[k] : mkc(0.0, 0.0);
        for (int i = k + 1 + lane; i < h; i += 32) dot = cfmac(col[i], cj[i], dot);
        dot = warp_csum(dot);
        const cd f = cmul(ctau, dot);
        if (lane == 0) cj[k] = csub(cj[k], f);
        const cd nf = cneg(f);
        for (int i = k + 1 + lane; i < h; i += 32) cj[i] = cfma(col[i], nf, cj[i]);
      }
    }
    __syncthreads();
  }
}

// Explicit Q (h x kq, column-major, leading dim ldq; any address space) of a
// factorisation left by qr_inplace: Q = H_0 ... H_{kq-1} [I; 0], built by
// applying the reflectors in reverse order to the identity columns.
static __device__ void form_q(const cd* W, int ld, int h, int kq, const cd* taus, cd* Q, int ldq) {
  const int lane = lane_id(), warp = warp_id(), nw = n_warps();
  for (int idx = threadIdx.x; idx < h * kq; idx += blockDim.x) {
    const int j = idx / h, i = idx - j * h;
    Q[(size_t)j * ldq + i] = mkc(i == j ? 1.0 : 0.0, 0.0);
  }
  __syncthreads();
  for (int k = kq - 1; k >= 0; --k) {
    const cd tau = taus[k];
    if (tau.x != 0.0 || tau.y != 0.0) {
      const cd* v = W + (size_t)k * ld;
      for (int j = k + warp; j < kq; j += nw) {
        cd* qj = Q + (size_t)j * ldq;
        cd dot = (lane == 0) ? qj[k] : mkc(0.0, 0.0);
        for (int i = k + 1 + lane; i < h; i += 32) dot = cfmac(v[i], qj[i], dot);
        dot = warp_csum(dot);
        const cd f = cmul(tau, dot);
        if (lane == 0) qj[k] = csub(qj[k], f);
        const cd nf = cneg(f);
        for (int i = k + 1 + lane; i < h; i += 32) qj[i] = cfma(v[i], nf, qj[i]);
      }
    }
    __syncthreads();
  }
}

// One-sided Jacobi (Hestenes): rotates the m columns of L (p rows, column
// major, leading dim ld) until every pair is orthogonal to working precision,
// |l_a^H l_b| <= tol * ||l_a|| ||l_b||. Columns are visited in round-robin
// tournament order. A pair is handled by a group of 8 lanes (four pairs per
// warp): the columns are short (p <= 64), so narrower groups spend fewer lanes
// on the per-pair rotation arithmetic, which every lane of a group repeats.
// Each warp runs the same number of group iterations, so the group reductions
// can use full-warp shuffles. Returns the number of sweeps used, or -1 if
// max_sweeps did not reach convergence.
static __device__ int hestenes(cd* L, int ld, int p, int m, int max_sweeps, int* sh_flag) {
  const int lane = lane_id(), warp = warp_id(), nw = n_warps();
  const int sub = lane & 7, grp = lane >> 3;  // 4 groups of 8 lanes per warp
  if (m < 2) return 0;
  const int mp = m + (m & 1);
  const int npair = mp / 2;
  // a pair counts as orthogonal once |a^H b| <= tol |a| |b|, the rounding
  // level of a p-term complex dot product; after max_sweeps the result is
  // accepted if no pair is worse than 1e-10 (reported as not converged otherwise)
  const double tol = 1.0e-15 * (double)max(p, 8);
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    if (threadIdx.x == 0) *sh_flag = 0;
    __syncthreads();
    for (int t = 0; t < mp - 1; ++t) {
      for (int e0 = 4 * warp; e0 < npair; e0 += 4 * nw) {
        const int e = e0 + grp;
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
        double al = 0.0, be = 0.0, gx = 0.0, gy = 0.0;
        if (live)
          for (int i = sub; i < p; i += 8) {
            const cd x = ca[i], y = cb[i];
            al = fma(x.x, x.x, fma(x.y, x.y, al));
            be = fma(y.x, y.x, fma(y.y, y.y, be));
            gx = fma(x.x, y.x, fma(x.y, y.y, gx));
            gy = fma(x.x, y.y, fma(-x.y, y.x, gy));
          }
#pragma unroll
        for (int o = 4; o > 0; o >>= 1) {
          al += __shfl_xor_sync(0xffffffffu, al, o);
          be += __shfl_xor_sync(0xffffffffu, be, o);
          gx += __shfl_xor_sync(0xffffffffu, gx, o);
          gy += __shfl_xor_sync(0xffffffffu, gy, o);
        }
        if (!live) continue;
        const double ga = sqrt(fma(gx, gx, gy * gy));
        const double nab = sqrt(al) * sqrt(be);
        if (ga > tol * nab && ga > 1e-300) {
          const double zeta = (be - al) / (2.0 * ga);
          // hypot keeps zeta^2 from overflowing when one column is tiny: then
          // t ~ 1/(2 zeta), the small-angle rotation
          const double tt = copysign(1.0, zeta) / (fabs(zeta) + hypot(1.0, zeta));
          const double c = rsqrt(fma(tt, tt, 1.0));
          const double s = c * tt;
          const double ig = 1.0 / ga;
          const cd ph = mkc(gx * ig, -gy * ig);  // exp(-i arg g)
          for (int i = sub; i < p; i += 8) {
            const cd x = ca[i];
            const cd y = cmul(cb[i], ph);
            ca[i] = mkc(fma(c, x.x, -s * y.x), fma(c, x.y, -s * y.y));
            cb[i] = mkc(fma(s, x.x, c * y.x), fma(s, x.y, c * y.y));
          }
          if (sub == 0) atomicOr(sh_flag, (ga > 1e-10 * nab) ? 3 : 1);
        }
      }
      __syncthreads();
    }
    const int any = *sh_flag;
    __syncthreads();
    if (!any) return sweep + 1;
    if (sweep == max_sweeps - 1) return (any & 2) ? -1 : max_sweeps;
  }
  return -1;
}

// Shared-memory layout needed by ts_svd for p columns and row blocks of hb.
__host__ __device__ inline size_t ts_svd_smem_bytes(int p, int hb) {
  return sizeof(cd) * ((size_t)(p + hb) * p + (size_t)p * p + p) + sizeof(double) * p + 64;
}

struct TsSvd {
  int m;          // number of singular triplets = min(q, p)
  int sweeps;     // Jacobi sweeps (-1: not converged)
  double flops;   // algorithmic FP64 flops of this factorisation
};

// Algorithmic FP64 flop counts (complex multiply-add = 8 real flops).
__host__ __device__ inline double flops_qr(double h, double p) {
  double f = 0.0;
  const double k = h < p ? h : p;
  for (double i = 0; i < k; i += 1.0) f += 16.0 * (h - i) * (p - i - 1.0) + 10.0 * (h - i);
  return f;
}
__host__ __device__ inline double flops_formq(double h, double kq) {
  double f = 0.0;
  for (double i = 0; i < kq; i += 1.0) f += 16.0 * (h - i) * (kq - i);
  return f;
}
__host__ __device__ inline double flops_hestenes(double p, double m, double sweeps) {
  return sweeps * 0.5 * m * (m - 1.0) * 26.0 * p;
}
__host__ __device__ inline double flops_gemm(double m, double n, double k) { return 8.0 * m * n * k; }

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

static __device__ TsSvd ts_svd(const cd* Z, long long q, int p, int ldz, cd* W, int wcap, cd* V,
                        double* sig, cd* taus, int* sh_flag) {
  const int hb = wcap / p - p;
  int ldw;
  const int nR = stream_qr(Z, q, p, ldz, W, wcap, taus, &ldw);
  const int m = nR;
  // L = R^H (p x m) into V
  for (int idx = threadIdx.x; idx < p * m; idx += blockDim.x) {
    const int c = idx / p, i = idx - c * p;
    V[(size_t)c * p + i] = (i >= c) ? cconj(W[(size_t)i * ldw + c]) : mkc(0.0, 0.0);
  }
  __syncthreads();
  TsSvd out;
  out.m = m;
  out.sweeps = hestenes(V, p, p, m, 60, sh_flag);
  {
    // QR of the stacked row blocks, Jacobi sweeps, norms and sort
    double f = 0.0;
    long long rows = q, carried = 0;
    while (rows > 0) {
      const long long b = rows < hb ? rows : hb;
      f += flops_qr((double)(carried + b), (double)p);
      carried = carried + b < p ? carried + b : p;
      rows -= b;
    }
    out.flops = f + flops_hestenes(p, m, out.sweeps < 0 ? 60 : out.sweeps) + 4.0 * p * m;
  }
  // column norms
  double* nrm = reinterpret_cast<double*>(W);  // W is free now
  for (int c = warp_id(); c < m; c += n_warps()) {
    double s = 0.0;
    for (int i = lane_id(); i < p; i += 32) s += cabs2(V[(size_t)c * p + i]);
    s = warp_sum(s);
    if (lane_id() == 0) nrm[c] = sqrt(s);
  }
  __syncthreads();
  // sort descending (stable by index), normalise into W after the norms
  cd* Vs = W + p;  // p*m elements, fits in (p+hb)*p - p
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
  return out;
}

// Smallest k >= 1 with sqrt(sum_{i >= k} sig_i^2) <= delta (sig descending);
// evaluated redundantly by every thread.
__device__ __forceinline__ int trunc_rank(const double* sig, int m, double delta) {
  double tail = 0.0;
  int k = m;
  for (int i = m - 1; i >= 0; --i) {
    tail += sig[i] * sig[i];
    if (sqrt(tail) <= delta) k = i; else break;
  }
  return max(k, 1);
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
// Z = Q R by the streaming QR; then R P = Q2 R2 by Householder QR with column
// pivoting (the column of largest remaining norm first), so that the trailing
// block R2[k:, k:] has Frobenius norm equal to the error of keeping k rows.
// k is the smallest rank with that norm <= delta_rel * ||Z||_F (k >= 1,
// k <= kmax). The kept rows span (R2[:k] P^T); B (p x k, column-major, leading
// dim p, in W on return) is an orthonormal basis of their conjugate span, so
// Z ~= Z B B^H with error at most the trailing norm.
// Smem: W (wcap >= (p + 1) p), V (p x p), taus and cn (p entries each), perm (p ints).
struct RowBasis {
  int k;
  double flops;
};

static __device__ RowBasis rrqr_basis(const cd* Z, long long q, int p, int ldz, cd* W, int wcap, cd* V,
                                      double delta_rel, int kmax, cd* taus, double* cn, int* perm,
                                      double* red_d, int* red_i) {
  const int lane = lane_id(), warp = warp_id(), nw = n_warps();
  int ldw;
  const int m = stream_qr(Z, q, p, ldz, W, wcap, taus, &ldw);
  RowBasis out;
  out.flops = 0.0;
  for (int j = threadIdx.x; j < p; j += blockDim.x) perm[j] = j;
  __syncthreads();
  const int kmax_q = min(m, p);
  double total = 0.0;
  // pivoted Householder QR of R (m x p) in place
  for (int k = 0; k < kmax_q; ++k) {
    for (int j = k + warp; j < p; j += nw) {
      const cd* cj = W + (size_t)j * ldw;
      double amax = 0.0;
      for (int i = k + lane; i < m; i += 32) amax = fmax(amax, fmax(fabs(cj[i].x), fabs(cj[i].y)));
      amax = warp_max(amax);
      const double inv = amax > 1e-290 ? 1.0 / amax : 0.0;
      double ss = 0.0;
      for (int i = k + lane; i < m; i += 32) ss += cabs2(cscale(cj[i], inv));
      ss = warp_sum(ss);
      if (lane == 0) cn[j] = ss * amax * amax;
    }
    __syncthreads();
    if (k == 0) {
      for (int j = 0; j < p; ++j) total += cn[j];
    }
    const int jm = k + cta_argmax(p - k, [&](int t) { return cn[k + t]; }, red_d, red_i);
    if (jm != k) {
      for (int i = threadIdx.x; i < m; i += blockDim.x) {
        const cd t = W[(size_t)k * ldw + i];
        W[(size_t)k * ldw + i] = W[(size_t)jm * ldw + i];
        W[(size_t)jm * ldw + i] = t;
      }
      if (threadIdx.x == 0) {
        const int t = perm[k];
        perm[k] = perm[jm];
        perm[jm] = t;
      }
    }
    __syncthreads();
    // one Householder step on column k (rows k..m-1), applied to columns > k
    cd* col = W + (size_t)k * ldw;
    if (warp == 0) {
      cd a0 = (lane == 0) ? col[k] : mkc(0.0, 0.0);
      a0.x = __shfl_sync(0xffffffffu, a0.x, 0);
      a0.y = __shfl_sync(0xffffffffu, a0.y, 0);
      double amax = fmax(fabs(a0.x), fabs(a0.y));
      for (int i = k + 1 + lane; i < m; i += 32) amax = fmax(amax, fmax(fabs(col[i].x), fabs(col[i].y)));
      amax = warp_max(amax);
      const double inv = (amax > 1e-290) ? 1.0 / amax : 0.0;
      double ss = 0.0;
      for (int i = k + 1 + lane; i < m; i += 32) ss += cabs2(cscale(col[i], inv));
      ss = warp_sum(ss);
      cd tau = mkc(0.0, 0.0);
      if (inv != 0.0 && !(ss == 0.0 && a0.y == 0.0)) {
        const cd a0s = cscale(a0, inv);
        const double beta = -copysign(amax * sqrt(cabs2(a0s) + ss), a0.x);
        tau = mkc((beta - a0.x) / beta, -a0.y / beta);
        const cd scal = cdiv(mkc(1.0, 0.0), mkc(a0.x - beta, a0.y));
        for (int i = k + 1 + lane; i < m; i += 32) col[i] = cmul(col[i], scal);
        if (lane == 0) col[k] = mkc(beta, 0.0);
      }
      if (lane == 0) taus[k] = tau;
    }
    __syncthreads();
    const cd tau = taus[k];
    if (tau.x != 0.0 || tau.y != 0.0) {
      const cd ctau = cconj(tau);
      for (int j = k + 1 + warp; j < p; j += nw) {
        cd* cj = W + (size_t)j * ldw;
        cd dot = (lane == 0) ? cj[k] : mkc(0.0, 0.0);
        for (int i = k + 1 + lane; i < m; i += 32) dot = cfmac(col[i], cj[i], dot);
        dot = warp_csum(dot);
        const cd f = cmul(ctau, dot);
        const cd nf = cneg(f);
        if (lane == 0) cj[k] = csub(cj[k], f);
        for (int i = k + 1 + lane; i < m; i += 32) cj[i] = cfma(col[i], nf, cj[i]);
      }
    }
    __syncthreads();
    out.flops += 20.0 * (m - k) * (p - k);
  }
  // rank from the trailing row norms of R2 (upper trapezoidal, row i from column i)
  for (int i = warp; i < kmax_q; i += nw) {
    double ss = 0.0;
    for (int j = i + lane; j < p; j += 32) {
      const cd v = W[(size_t)j * ldw + i];
      ss += cabs2(v);
    }
    ss = warp_sum(ss);
    if (lane == 0) cn[i] = ss;
  }
  __syncthreads();
  const double delta = delta_rel * sqrt(total);
  int k = kmax_q;
  {
    double tail = 0.0;
    for (int i = kmax_q - 1; i >= 0; --i) {
      tail += cn[i];
      if (sqrt(tail) <= delta) k = i; else break;
    }
  }
  k = max(k, 1);
  k = min(k, kmax);
  out.k = k;
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
