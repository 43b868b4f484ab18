// Dense-FFT Carr-Madan baseline (the FFT route of Sec. 4.1): every integrand
// value x_j, j < M = 2^n, is evaluated inside the first pass of an in-place
// M-point FFT that runs as a sequence of radix-2^R decimation-in-frequency
// passes through shared memory, and the requested strikes are gathered and
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

// With `sample` set (the first pass), the pass evaluates the integrand at its
// indices instead of reading x: sampling is fused into the first pass, and
// the array is written once, transformed. The twiddles exp(-2 pi i s k / L)
// of a block come from two small tables per column, w^(16 kh) and w^kl with
// k = 16 kh + kl and w = exp(-2 pi i s / L), each entry formed exactly from
// its reduced integer argument, so a twiddle costs one complex product.
__global__ void k_fft_pass(cd* x, long long M, long long Lp, int R, int cols, InstParams P, int sample) {
  extern __shared__ double4 smem_raw[];
  cd* sm = reinterpret_cast<cd*>(smem_raw);
  const int Rn = 1 << R;
  cd* tw = sm + (size_t)Rn * cols;
  cd* t_lo = tw + Rn;            // [c][kl], 16 per column
  cd* t_hi = t_lo + 16 * cols;   // [c][kh], 16 per column
  for (int i = threadIdx.x; i < Rn; i += blockDim.x) tw[i] = unit_root(i, Rn);
  const long long L = Lp * Rn;
  const long long per_sub = Lp / cols;
  const int lc = __ffs(cols) - 1;  // cols is a power of two
  const long long nblk = (M / L) * per_sub;
  for (long long blk = blockIdx.x; blk < nblk; blk += gridDim.x) {
    const long long b = blk / per_sub;
    const long long s0 = (blk - b * per_sub) * cols;
    const long long base = b * L + s0;
    __syncthreads();
    for (int e = threadIdx.x; e < 32 * cols; e += blockDim.x) {
      const int c = e >> 5, j = e & 15;
      const long long s = s0 + c;
      if ((e & 31) < 16)
        t_lo[c * 16 + j] = unit_root((s * j) & (L - 1), L);
      else
        t_hi[c * 16 + j] = unit_root((s * 16 * j) & (L - 1), L);
    }
    for (int e = threadIdx.x; e < Rn * cols; e += blockDim.x) {
      const int r = e >> lc, c = e & (cols - 1);
      const long long j = base + (long long)r * Lp + c;
      sm[e] = sample ? integrand(P, j) : x[j];
    }
    __syncthreads();
    // radix-2 stages; the last two have trivial twiddles (1, and -i)
    for (int lh = R - 1; lh >= 2; --lh) {
      const int half = 1 << lh;
      const int stride_tw = Rn >> (lh + 1);
      for (int bf = threadIdx.x; bf < (Rn >> 1) * cols; bf += blockDim.x) {
        const int c = bf & (cols - 1), j = bf >> lc;
        const int g = j >> lh, i = j & (half - 1);
        const int r0 = (g << (lh + 1)) + i, r1 = r0 + half;
        const cd a = sm[r0 * cols + c], bb = sm[r1 * cols + c];
        sm[r0 * cols + c] = cadd(a, bb);
        sm[r1 * cols + c] = cmul(csub(a, bb), tw[i * stride_tw]);
      }
      __syncthreads();
    }
    if (R >= 2) {
      // span 4: twiddles 1 and exp(-i pi / 2) = -i
      for (int bf = threadIdx.x; bf < (Rn >> 1) * cols; bf += blockDim.x) {
        const int c = bf & (cols - 1), j = bf >> lc;
        const int g = j >> 1, i = j & 1;
        const int r0 = (g << 2) + i, r1 = r0 + 2;
        const cd a = sm[r0 * cols + c], bb = sm[r1 * cols + c];
        sm[r0 * cols + c] = cadd(a, bb);
        const cd d = csub(a, bb);
        sm[r1 * cols + c] = i ? mkc(d.y, -d.x) : d;
      }
      __syncthreads();
    }
    if (R >= 1) {
      // span 2: twiddle 1
      for (int bf = threadIdx.x; bf < (Rn >> 1) * cols; bf += blockDim.x) {
        const int c = bf & (cols - 1), j = bf >> lc;
        const int r0 = j << 1, r1 = r0 + 1;
        const cd a = sm[r0 * cols + c], bb = sm[r1 * cols + c];
        sm[r0 * cols + c] = cadd(a, bb);
        sm[r1 * cols + c] = csub(a, bb);
      }
      __syncthreads();
    }
    for (int e = threadIdx.x; e < Rn * cols; e += blockDim.x) {
      const int k = e >> lc, c = e & (cols - 1);
      const int kr = (int)(__brev((unsigned)k) >> (32 - R));
      const cd v = sm[kr * cols + c];
      x[base + (long long)k * Lp + c] = cmul(v, cmul(t_hi[c * 16 + (k >> 4)], t_lo[c * 16 + (k & 15)]));
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
