// Characteristic functions, psi and the integrand x_j on the device.
//
// Log-moneyness throughout: X = log(S_T/S0), phi1(u) = E[exp(iuX)], call
// price C(K) = S0 * C1(log(K/S0)). This equals the paper's absolute-log-strike
// form of Eqs. psi, x and discretization_dft exactly (the S0 phases cancel)
// and makes the grid phases exact fractions of a turn.
#pragma once
#include "cplx.cuh"
#include <stdint.h>

enum { M_GBM = 0, M_HESTON = 1, M_MERTON = 2, M_VG = 3 };
enum { Q_SIMPSON = 0, Q_RECT = 1 };

// Per-instance constants planned on the host (grid scalars of Sec. 2.1 and
// model constants that depend only on the parameters).
struct InstParams {
  int32_t model, quad, n, max_rank;
  double p[8];
  double S0, r, T, alpha, tol;
  double dv;      // frequency step (eta or Delta_v)
  double dk;      // log-strike step
  double k0;      // log-moneyness of grid index 0
  double disc;    // exp(-rT)
  double omega;   // VG martingale correction
  double kbar;    // Merton mean jump size exp(muJ + dJ^2/2) - 1
  long long N;    // RECT_SYM half size M/2
};

// phi1(u) for complex u.
__device__ __forceinline__ cd phi1(const InstParams& P, cd u) {
  const cd iu = mkc(-u.y, u.x);
  const cd u2 = cmul(u, u);
  const double r = P.r, T = P.T;
  switch (P.model) {
    case M_GBM: {
      const double s2 = P.p[0] * P.p[0];
      const cd e = cadd(cscale(iu, (r - 0.5 * s2) * T), cscale(u2, -0.5 * s2 * T));
      return cexpd(e);
    }
    case M_HESTON: {
      const double kappa = P.p[0], theta = P.p[1], sv = P.p[2], rho = P.p[3], v0 = P.p[4];
      const double sv2 = sv * sv;
      const cd b = csub(mkc(kappa, 0.0), cscale(iu, rho * sv));
      const cd d = csqrtd(cadd(cmul(b, b), cscale(cadd(iu, u2), sv2)));
      const cd bmd = csub(b, d);
      const cd g = cdiv(bmd, cadd(b, d));
      const cd e = cexpd(cscale(d, -T));
      const cd one = mkc(1.0, 0.0);
      const cd ge1 = csub(one, cmul(g, e));
      const cd lg = clogd(cdiv(ge1, csub(one, g)));
      const cd C = cscale(csub(cscale(bmd, T), cscale(lg, 2.0)), kappa * theta / sv2);
      const cd D = cdiv(cmul(cscale(bmd, 1.0 / sv2), csub(one, e)), ge1);
      return cexpd(cadd(cadd(cscale(iu, r * T), C), cscale(D, v0)));
    }
    case M_MERTON: {
      const double s2 = P.p[0] * P.p[0], lam = P.p[1], mu = P.p[2], dj = P.p[3];
      const cd drift = cscale(iu, (r - 0.5 * s2 - lam * P.kbar) * T);
      const cd diff = cscale(u2, -0.5 * s2 * T);
      const cd jexp = cexpd(csub(cscale(iu, mu), cscale(u2, 0.5 * dj * dj)));
      const cd jump = cscale(csub(jexp, mkc(1.0, 0.0)), lam * T);
      return cexpd(cadd(cadd(drift, diff), jump));
    }
    default: {  // M_VG
      const double s2 = P.p[0] * P.p[0], nu = P.p[1], th = P.p[2];
      const cd base = cadd(csub(mkc(1.0, 0.0), cscale(iu, th * nu)), cscale(u2, 0.5 * s2 * nu));
      const cd e = csub(cscale(iu, (r + P.omega) * T), cscale(clogd(base), T / nu));
      return cexpd(e);
    }
  }
}

// Eq. psi: psi1(v) = exp(-rT) phi1(v - i(alpha+1)) / ((alpha + iv)(alpha + 1 + iv)).
__device__ __forceinline__ cd psi1(const InstParams& P, double v) {
  const cd num = phi1(P, mkc(v, -(P.alpha + 1.0)));
  const cd den = cmul(mkc(P.alpha, v), mkc(P.alpha + 1.0, v));
  return cscale(cdiv(num, den), P.disc);
}

// Values below 1e-150 in modulus are returned as zero: they cannot move a
// price, and their squares would underflow inside the factorisations.
__device__ __forceinline__ cd flush_tiny(cd x) {
  return (fmax(fabs(x.x), fabs(x.y)) < 1e-150) ? mkc(0.0, 0.0) : x;
}

// Integrand x_j at grid index j in [0, 2^n).
//  SIMPSON_CM99: x_j = (-1)^j w_j eta psi1(eta j), w = 1/3, 4/3, 2/3, ...
//  RECT_SYM (Eq. x with Delta_v k'_0 = -pi/2): x_j = i^j (-i)^N psi1(Delta_v (j - N)).
__device__ __forceinline__ cd integrand_raw(const InstParams& P, long long j);
__device__ __forceinline__ cd integrand(const InstParams& P, long long j) {
  return flush_tiny(integrand_raw(P, j));
}
__device__ __forceinline__ cd integrand_raw(const InstParams& P, long long j) {
  if (P.quad == Q_SIMPSON) {
    const double w = (j == 0) ? (1.0 / 3.0) : ((j & 1) ? (4.0 / 3.0) : (2.0 / 3.0));
    const double sgn = (j & 1) ? -1.0 : 1.0;
    return cscale(psi1(P, P.dv * (double)j), sgn * w * P.dv);
  }
  const cd ps = psi1(P, P.dv * (double)(j - P.N));
  // i^j (-i)^N = i^(j - N) = i^((j + 3N) mod 4)
  const int e = (int)((j + 3 * (P.N & 3)) & 3);
  switch (e) {
    case 0: return ps;
    case 1: return mkc(-ps.y, ps.x);
    case 2: return cneg(ps);
    default: return mkc(ps.y, -ps.x);
  }
}

// Real price factor and sign for output index u: price = S0 * f * Re(sgn * y_u)
// (Eq. discretization_dft and its Simpson analogue).
__device__ __forceinline__ double price_factor(const InstParams& P, long long u, double* sgn) {
  const double kp = P.k0 + P.dk * (double)u;
  const double sqM = ldexp(1.0, P.n / 2) * ((P.n & 1) ? 1.4142135623730951 : 1.0);
  if (P.quad == Q_SIMPSON) {
    *sgn = 1.0;
    return exp(-P.alpha * kp) * sqM * 0.3183098861837907;  // 1/pi
  }
  *sgn = (u & 1) ? -1.0 : 1.0;
  return exp(-P.alpha * kp) * P.dv * sqM * 0.15915494309189535;  // 1/(2 pi)
}
