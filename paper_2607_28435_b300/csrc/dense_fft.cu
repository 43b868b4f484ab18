// Dense-FFT Carr-Madan baseline (the FFT route of Sec. 4.1): every integrand
// value x_j, j < M = 2^n, is evaluated in index order, the in-place M-point
// FFT runs as a sequence of ceil(n / 10) passes of 2^R-point transforms
// (R <= 10) through shared memory, and the requested strikes are gathered and
// priced (Eq. discretization_dft).
//
// Pass with sub-transform length L = 2^R * Lp: for every sub-transform b and
// offset s < Lp the 2^R elements x[bL + s + r Lp] are transformed,
// X_k = sum_r x_r exp(-2 pi i r k / 2^R), twiddled by exp(-2 pi i s k / L) and
// stored back at bL + s + k Lp. After all passes the output of frequency u sits
// at the digit-reversed position sum_p k_p Lp_p, k_p the p-th digit of u
// (least significant first).
#include "kernels.cuh"

__global__ void k_dense_sample(InstParams prm, cd* x, long long M) {
  for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < M;
       j += (long long)gridDim.x * blockDim.x)
    x[j] = integrand(prm, j);
}

__device__ __forceinline__ cd unit_root(long long t, long long L) {
  // exp(-2 pi i t / L) with the argument formed exactly (L a power of two)
  double sn, cs;
  sincospi(2.0 * (double)t / (double)L, &sn, &cs);
  return mkc(cs, -sn);
}

// One pass of the transform. Each block takes `cols` adjacent offsets s of
// one sub-transform b: the 2^R elements x[bL + s + r Lp] of every column go
// to shared memory. The 2^R-point DFT of every
// column then runs as decimation-in-frequency levels of radix 8 (three bits
// each, in registers: one butterfly per thread, an exchange through shared
// memory between levels) and a last level of radix 4 or 2. Level l with span
// N splits its groups of N rows into the N/r butterflies n1: inputs at rows
// n1 + (N/r) n2, outputs y_k2 = sum_n2 x_n2 w_r^(n2 k2) times w_N^(n1 k2)
// back at rows n1 + (N/r) k2. Frequency k = k_0 + r_0 k_1 + r_0 r_1 k_2 + ...
// then sits at row sum_l k_l (2^R / (r_0 ... r_l)) (digits reversed). Each
// output is twiddled by exp(-2 pi i s k / L) and stored at bL + s + k Lp.
// The last pass (Lp = 1) has no inter-pass twiddle and contiguous
// sub-transforms: there a block's columns are `cols` consecutive
// sub-transforms b, loaded and stored in index order.
// Twiddles: w_(2^R)^j for j < 2^R in a table built once per block of the
// persistent grid; exp(-2 pi i s k / L) as the product of two 32-entry
// tables per column, w^(32 k_hi) and w^(k_lo) with k = 32 k_hi + k_lo and
// w = exp(-2 pi i s / L); every entry is formed exactly from its reduced
// integer argument. Radix-8 butterfly: the three radix-2 steps of the
// 8-point DFT, with w_8 = (1 - i)/sqrt 2 and w_8^3 as one sum and one scaling
// per component and w_8^2 = -i as a swap.
__device__ __forceinline__ cd mul_mi(cd a) { return mkc(a.y, -a.x); }  // a (-i)

__device__ __forceinline__ void dft4(cd z0, cd z1, cd z2, cd z3, cd& o0, cd& o1, cd& o2, cd& o3) {
  const cd s0 = cadd(z0, z2), d0 = csub(z0, z2), s1 = cadd(z1, z3), d1 = mul_mi(csub(z1, z3));
  o0 = cadd(s0, s1);
  o2 = csub(s0, s1);
  o1 = cadd(d0, d1);
  o3 = csub(d0, d1);
}

// 8-point DFT, natural order in and out; h = 1/sqrt(2)
__device__ __forceinline__ void dft8(cd* a, double h) {
  cd u[4], v[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    u[j] = cadd(a[j], a[j + 4]);
    v[j] = csub(a[j], a[j + 4]);
  }
  v[1] = mkc((v[1].x + v[1].y) * h, (v[1].y - v[1].x) * h);    // w_8
  v[2] = mul_mi(v[2]);                                        // w_8^2
  v[3] = mkc((v[3].y - v[3].x) * h, -(v[3].x + v[3].y) * h);  // w_8^3
  dft4(u[0], u[1], u[2], u[3], a[0], a[2], a[4], a[6]);
  dft4(v[0], v[1], v[2], v[3], a[1], a[3], a[5], a[7]);
}

__global__ void __launch_bounds__(256) k_fft_pass(cd* x, long long M, long long Lp, int R, int cols) {
  extern __shared__ double4 smem_raw[];
  cd* sm = reinterpret_cast<cd*>(smem_raw);
  const int Rn = 1 << R;
  cd* tw = sm + (size_t)Rn * cols;  // w_(2^R)^j
  cd* t_lo = tw + Rn;               // [c][32]
  cd* t_hi = t_lo + 32 * cols;      // [c][32]
  for (int i = threadIdx.x; i < Rn; i += blockDim.x) tw[i] = unit_root(i, Rn);
  const double h = 0.70710678118654752440;  // 1/sqrt(2)
  const long long L = Lp * Rn;
  const bool last = Lp == 1;
  const long long per_sub = last ? 1 : Lp / cols;
  const int lc = __ffs(cols) - 1;  // cols is a power of two
  const long long nblk = last ? (M / L) / cols : (M / L) * per_sub;
  for (long long blk = blockIdx.x; blk < nblk; blk += gridDim.x) {
    const long long b = last ? blk * cols : blk / per_sub;
    const long long s0 = last ? 0 : (blk - b * per_sub) * cols;
    const long long base = b * L + s0;
    __syncthreads();
    for (int e = threadIdx.x; e < (last ? 0 : 64 * cols); e += blockDim.x) {
      const int c = e >> 6, j = e & 31;
      const long long s = s0 + c;
      if ((e & 63) < 32)
        t_lo[c * 32 + j] = unit_root((s * j) & (L - 1), L);
      else
        t_hi[c * 32 + j] = unit_root((s * 32 * j) & (L - 1), L);
    }
    for (int e = threadIdx.x; e < Rn * cols; e += blockDim.x) {
      if (last) {
        const int c = e >> R, r = e & (Rn - 1);  // x[base + c Rn + r] = x[base + e]
        sm[(size_t)r * cols + c] = x[base + e];
      } else {
        const int r = e >> lc, c = e & (cols - 1);
        sm[e] = x[base + (long long)r * Lp + c];
      }
    }
    __syncthreads();
    int span = Rn, bits = R;
    while (bits > 0) {
      const int rb = bits >= 3 ? 3 : bits;
      const int q = span >> rb;            // stride between a butterfly's inputs
      const int lq = __ffs(q) - 1;
      const int tstep = Rn / span;         // w_span^m = tw[m tstep]
      const int nbf = (Rn >> rb) * cols;
      for (int t = threadIdx.x; t < nbf; t += blockDim.x) {
        const int c = t & (cols - 1), u = t >> lc;
        const int n1 = u & (q - 1);
        const int row0 = ((u >> lq) * span) + n1;
        cd a[8];
        if (rb == 3) {
#pragma unroll
          for (int n2 = 0; n2 < 8; ++n2) a[n2] = sm[(size_t)(row0 + n2 * q) * cols + c];
          dft8(a, h);
          if (q > 1) {
#pragma unroll
            for (int k2 = 1; k2 < 8; ++k2) a[k2] = cmul(a[k2], tw[(n1 * k2 * tstep) & (Rn - 1)]);
          }
#pragma unroll
          for (int k2 = 0; k2 < 8; ++k2) sm[(size_t)(row0 + k2 * q) * cols + c] = a[k2];
        } else if (rb == 2) {
#pragma unroll
          for (int n2 = 0; n2 < 4; ++n2) a[n2] = sm[(size_t)(row0 + n2 * q) * cols + c];
          dft4(a[0], a[1], a[2], a[3], a[4], a[5], a[6], a[7]);
          if (q > 1) {
#pragma unroll
            for (int k2 = 1; k2 < 4; ++k2) a[4 + k2] = cmul(a[4 + k2], tw[(n1 * k2 * tstep) & (Rn - 1)]);
          }
#pragma unroll
          for (int k2 = 0; k2 < 4; ++k2) sm[(size_t)(row0 + k2 * q) * cols + c] = a[4 + k2];
        } else {
          const cd a0 = sm[(size_t)row0 * cols + c], a1 = sm[(size_t)(row0 + q) * cols + c];
          sm[(size_t)row0 * cols + c] = cadd(a0, a1);
          const cd d = csub(a0, a1);
          sm[(size_t)(row0 + q) * cols + c] = (q > 1) ? cmul(d, tw[(n1 * tstep) & (Rn - 1)]) : d;
        }
      }
      __syncthreads();
      span = q;
      bits -= rb;
    }
    for (int e = threadIdx.x; e < Rn * cols; e += blockDim.x) {
      const int k = last ? (e & (Rn - 1)) : (e >> lc), c = last ? (e >> R) : (e & (cols - 1));
      // row of frequency k: its digits (radix 8, then 4 or 2) reversed
      int p = 0, rem = k, sp = Rn, bl = R;
      while (bl > 0) {
        const int rb = bl >= 3 ? 3 : bl;
        sp >>= rb;
        p += (rem & ((1 << rb) - 1)) * sp;
        rem >>= rb;
        bl -= rb;
      }
      const cd v = sm[(size_t)p * cols + c];
      if (last)
        x[base + e] = v;
      else
        x[base + (long long)k * Lp + c] = cmul(v, cmul(t_hi[c * 32 + (k >> 5)], t_lo[c * 32 + (k & 31)]));
    }
  }
}

__global__ void k_dense_gather(InstParams prm, const cd* y, int n,
                               const int* digits, int ndig, long long l_begin,
                               int tbits, int q, double* prices,
                               double* logk) {
  const double inv_sqM = 1.0 / (ldexp(1.0, n / 2) * ((n & 1) ? 1.4142135623730951 : 1.0));
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < q; i += gridDim.x * blockDim.x) {
    const long long u = l_begin + ((long long)i << tbits);
    long long pos = 0, rem = u;
    int used = 0;
    for (int p = 0; p < ndig; ++p) {
      const int R = digits[p];
      used += R;
      const long long k = rem & ((1LL << R) - 1);
      rem >>= R;
      pos += k << (n - used);
    }
    const cd v = y[pos];
    double sgn;
    const double f = price_factor(prm, u, &sgn);
    prices[i] = prm.S0 * f * sgn * v.x * inv_sqM;
    logk[i] = log(prm.S0) + prm.k0 + prm.dk * (double)u;
  }
}

// ---------------------------------------------------------------------------
// Statevector emulation of the QFT route (Sec. 3, QFT-based option pricing):
// the sampled x is normalised to the amplitudes x / ||x|| of
// Eq. qft_input_state, the passes above apply the inverse QFT (unitary up to
// the 1/sqrt(M) taken in the gather), the measurement probabilities are
// p_l = |y~_l|^2 (Eq. qft_probabilities), and the price is read from sqrt(p_l)
// under the positive-phase assumption (Eqs. qft_phase_assumption,
// qft_observable_price) with exact probabilities.
// ---------------------------------------------------------------------------

// ||x||^2 in two deterministic stages: per-block partial sums, then one
// thread adds the partials in order.
__global__ void k_norm2_partial(const cd* x, long long M, double* part) {
  __shared__ double red[32];
  double s = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < M;
       i += (long long)gridDim.x * blockDim.x)
    s = fma(x[i].x, x[i].x, fma(x[i].y, x[i].y, s));
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    part[blockIdx.x] = t;
  }
}

__global__ void k_norm2_final(const double* part, int nparts, double* nrm2) {
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    double t = 0.0;
    for (int b = 0; b < nparts; ++b) t += part[b];
    *nrm2 = t;
  }
}

// x <- x / ||x||: the amplitude-encoded state
__global__ void k_scale_unit(cd* x, long long M, const double* nrm2) {
  const double n2 = *nrm2;
  const double inv = n2 > 0.0 ? 1.0 / sqrt(n2) : 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < M;
       i += (long long)gridDim.x * blockDim.x)
    x[i] = cscale(x[i], inv);
}

// Requested strikes of the QFT route: p_l = |y~_l|^2 with y~ the unitary
// transform of the normalised state (the passes leave it scaled by sqrt(M)),
// price = S0 f_l ||x|| sqrt(p_l), f_l the same factor as the dense route
// (e^{-alpha k_l} Delta_v sqrt(M) / (2 pi) on the paper's grid).
__global__ void k_qft_gather(InstParams prm, const cd* y, int n, const int* digits, int ndig,
                             long long l_begin, int tbits, int q, const double* nrm2,
                             double* prices, double* logk) {
  const double inv_M = ldexp(1.0, -n);
  const double xnorm = sqrt(*nrm2);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < q; i += gridDim.x * blockDim.x) {
    const long long u = l_begin + ((long long)i << tbits);
    long long pos = 0, rem = u;
    int used = 0;
    for (int p = 0; p < ndig; ++p) {
      const int R = digits[p];
      used += R;
      const long long k = rem & ((1LL << R) - 1);
      rem >>= R;
      pos += k << (n - used);
    }
    const double pl = cabs2(y[pos]) * inv_M;
    double sgn;
    const double f = price_factor(prm, u, &sgn);
    prices[i] = prm.S0 * f * xnorm * sqrt(pl);
    logk[i] = log(prm.S0) + prm.k0 + prm.dk * (double)u;
  }
}
