// Complex FP64 helpers for the SFFT kernels (interleaved double2 = re, im).
#pragma once
#include <cuda_runtime.h>
#include <math.h>

typedef double2 cd;

__host__ __device__ __forceinline__ cd mkc(double re, double im) { return make_double2(re, im); }
__device__ __forceinline__ cd cadd(cd a, cd b) { return mkc(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ cd csub(cd a, cd b) { return mkc(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ cd cneg(cd a) { return mkc(-a.x, -a.y); }
__device__ __forceinline__ cd cconj(cd a) { return mkc(a.x, -a.y); }
__device__ __forceinline__ cd cscale(cd a, double s) { return mkc(a.x * s, a.y * s); }
__device__ __forceinline__ cd cmul(cd a, cd b) {
  return mkc(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
// conj(a) * b
__device__ __forceinline__ cd cmulc(cd a, cd b) {
  return mkc(fma(a.x, b.x, a.y * b.y), fma(a.x, b.y, -a.y * b.x));
}
// a * b + c
__device__ __forceinline__ cd cfma(cd a, cd b, cd c) {
  return mkc(fma(a.x, b.x, fma(-a.y, b.y, c.x)), fma(a.x, b.y, fma(a.y, b.x, c.y)));
}
// conj(a) * b + c
__device__ __forceinline__ cd cfmac(cd a, cd b, cd c) {
  return mkc(fma(a.x, b.x, fma(a.y, b.y, c.x)), fma(a.x, b.y, fma(-a.y, b.x, c.y)));
}
__device__ __forceinline__ double cabs2(cd a) { return fma(a.x, a.x, a.y * a.y); }
__device__ __forceinline__ double cabsd(cd a) { return hypot(a.x, a.y); }
__device__ __forceinline__ cd cdiv(cd a, cd b) {
  // Smith's algorithm
  if (fabs(b.x) >= fabs(b.y)) {
    double r = b.y / b.x, d = b.x + b.y * r;
    return mkc((a.x + a.y * r) / d, (a.y - a.x * r) / d);
  } else {
    double r = b.x / b.y, d = b.x * r + b.y;
    return mkc((a.x * r + a.y) / d, (a.y * r - a.x) / d);
  }
}
__device__ __forceinline__ cd cexpd(cd z) {
  double s, c;
  sincos(z.y, &s, &c);
  double e = exp(z.x);
  return mkc(e * c, e * s);
}
__device__ __forceinline__ cd clogd(cd z) { return mkc(log(hypot(z.x, z.y)), atan2(z.y, z.x)); }
// principal square root
__device__ __forceinline__ cd csqrtd(cd z) {
  double r = hypot(z.x, z.y);
  if (r == 0.0) return mkc(0.0, 0.0);
  double t = sqrt(0.5 * (r + fabs(z.x)));
  if (z.x >= 0.0) return mkc(t, z.y / (2.0 * t));
  return mkc(fabs(z.y) / (2.0 * t), copysign(t, z.y));
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ cd warp_csum(cd v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
    v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
  }
  return v;
}
