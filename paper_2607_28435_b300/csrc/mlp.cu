// Price surrogate: forward, backward and Adam kernels of a GELU multilayer
// perceptron with bfloat16 weights and float32 accumulation (C ABI in
// include/sfft_mlp.h). The network is not part of the paper's method; it is
// a learned stand-in for repeated queries in a parameter box, with the SFFT
// pricer as its fallback.
//
// Every product is one tiled GEMM, C[m, n] = sum_k A(m, k) B(n, k), with the
// operands addressed through strides so that the same kernel serves
// x W^T (forward), dz W (backward, data) and dz^T h (backward, weights). The
// tiles are 64 x 64 outputs per 256-thread CTA, 4 x 4 per thread, k in
// steps of 16 through shared memory; the weight reductions over the batch
// split k across CTAs and add their partial tiles atomically.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>

#include "../../include/sfft_mlp.h"

namespace {

constexpr int kTile = 64;
constexpr int kStepK = 16;
constexpr int kThreads = 256;

enum { EPI_PLAIN = 0, EPI_FWD = 1, EPI_BWD = 2 };

__device__ __forceinline__ float bf16_to_float(uint16_t b) { return __uint_as_float((uint32_t)b << 16); }
__device__ __forceinline__ float load_operand(const float* p) { return *p; }
__device__ __forceinline__ float load_operand(const uint16_t* p) { return bf16_to_float(*p); }

// round to the nearest bfloat16, ties to even (finite inputs)
__device__ __forceinline__ uint16_t float_to_bf16(float f) {
  uint32_t u = __float_as_uint(f);
  u += 0x7FFFu + ((u >> 16) & 1u);
  return (uint16_t)(u >> 16);
}

// GELU(z) = z Phi(z) and its derivative Phi(z) + z phi(z)
__device__ __forceinline__ float gelu(float z) { return z * normcdff(z); }
__device__ __forceinline__ float gelu_grad(float z) {
  return normcdff(z) + z * 0.3989422804014327f * expf(-0.5f * z * z);
}

// C[m, n] (row stride ldc) from A(m, k) = A[m sam + k sak] and
// B(n, k) = B[n sbn + k sbk], k in [z kchunk, min(K, (z + 1) kchunk)).
//   EPI_PLAIN: C = acc, or C += acc atomically when k is split (gridDim.z > 1)
//   EPI_FWD:   z = acc + bias[n]; C = z (if C), H = GELU(z) (if H)
//   EPI_BWD:   C = acc * GELU'(Zp[m, n])
template <typename TB, int EPI>
__global__ void __launch_bounds__(kThreads) k_mlp_gemm(int M, int N, int K, const float* __restrict__ A,
                                                      long long sam, long long sak,
                                                      const TB* __restrict__ B, long long sbn,
                                                      long long sbk, float* C, long long ldc,
                                                      const float* __restrict__ bias, float* H,
                                                      const float* __restrict__ Zp, int kchunk) {
  __shared__ __align__(16) float As[kStepK][kTile + 4];
  __shared__ __align__(16) float Bs[kStepK][kTile + 4];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int m0 = blockIdx.y * kTile, n0 = blockIdx.x * kTile;
  const int kbeg = blockIdx.z * kchunk;
  const int kend = min(K, kbeg + kchunk);
  float acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
  for (int k0 = kbeg; k0 < kend; k0 += kStepK) {
    // stage a 64 x 16 tile of each operand, walking the unit-stride index
    // fastest so that neighbouring threads read neighbouring addresses
    for (int e = threadIdx.x; e < kTile * kStepK; e += kThreads) {
      int mm, kk;
      if (sak == 1) {
        kk = e % kStepK;
        mm = e / kStepK;
      } else {
        mm = e % kTile;
        kk = e / kTile;
      }
      const int m = m0 + mm, k = k0 + kk;
      As[kk][mm] = (m < M && k < kend) ? A[(long long)m * sam + (long long)k * sak] : 0.f;
      int nn, kb;
      if (sbk == 1) {
        kb = e % kStepK;
        nn = e / kStepK;
      } else {
        nn = e % kTile;
        kb = e / kTile;
      }
      const int n = n0 + nn, kq = k0 + kb;
      Bs[kb][nn] = (n < N && kq < kend) ? load_operand(B + (long long)n * sbn + (long long)kq * sbk) : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < kStepK; ++kk) {
      const float4 av = *reinterpret_cast<const float4*>(&As[kk][ty * 4]);
      const float4 bv = *reinterpret_cast<const float4*>(&Bs[kk][tx * 4]);
      const float a[4] = {av.x, av.y, av.z, av.w};
      const float b[4] = {bv.x, bv.y, bv.z, bv.w};
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int m = m0 + ty * 4 + i;
    if (m >= M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int n = n0 + tx * 4 + j;
      if (n >= N) continue;
      const long long o = (long long)m * ldc + n;
      if (EPI == EPI_PLAIN) {
        if (gridDim.z > 1)
          atomicAdd(C + o, acc[i][j]);
        else
          C[o] = acc[i][j];
      } else if (EPI == EPI_FWD) {
        const float z = acc[i][j] + bias[n];
        if (C) C[o] = z;
        if (H) H[o] = gelu(z);
      } else {
        C[o] = acc[i][j] * gelu_grad(Zp[o]);
      }
    }
  }
}

// out[c] += sum of dz[r, c] over this CTA's rows (out zeroed by the caller)
__global__ void k_mlp_colsum(const float* __restrict__ dz, long long rows, int w, long long chunk,
                             float* out) {
  const long long r0 = (long long)blockIdx.x * chunk;
  const long long r1 = min(rows, r0 + chunk);
  for (int c = threadIdx.x; c < w; c += blockDim.x) {
    float s = 0.f;
    for (long long r = r0; r < r1; ++r) s += dz[r * w + c];
    atomicAdd(out + c, s);
  }
}

// dy = 2 (y - t) / batch; loss += sum (y - t)^2 / batch (loss zeroed by the caller)
__global__ void k_mlp_mse(const float* __restrict__ y, const float* __restrict__ t, long long batch,
                          float* dy, float* loss) {
  __shared__ float red[kThreads / 32];
  const float inv = 1.0f / (float)batch;
  float s = 0.f;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < batch;
       i += (long long)gridDim.x * blockDim.x) {
    const float d = y[i] - t[i];
    dy[i] = 2.0f * d * inv;
    s = fmaf(d, d, s);
  }
  if (!loss) return;
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    float b = 0.f;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) b += red[w];
    atomicAdd(loss, b * inv);
  }
}

__global__ void k_mlp_normalize(const double* __restrict__ raw, long long batch, int n_in,
                                const double* __restrict__ lo, const double* __restrict__ hi, float* x,
                                int* in_box) {
  for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < batch;
       r += (long long)gridDim.x * blockDim.x) {
    int ok = 1;
    for (int c = 0; c < n_in; ++c) {
      const double v = raw[r * n_in + c];
      ok &= (v >= lo[c] && v <= hi[c]) ? 1 : 0;
      x[r * n_in + c] = (float)(2.0 * (v - lo[c]) / (hi[c] - lo[c]) - 1.0);
    }
    if (in_box) in_box[r] = ok;
  }
}

__global__ void k_mlp_adam(long long count, float* p, uint16_t* pb, const float* __restrict__ g, float* m,
                           float* v, float lr, float b1, float b2, float eps, float c1, float c2) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < count;
       i += (long long)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = fmaf(b1, m[i], (1.0f - b1) * gi);
    const float vi = fmaf(b2, v[i], (1.0f - b2) * gi * gi);
    m[i] = mi;
    v[i] = vi;
    const float pi = p[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    p[i] = pi;
    if (pb) pb[i] = float_to_bf16(pi);
  }
}

bool net_ok(const sfft_mlp* net) {
  if (!net || net->n_layers < 1 || net->n_layers > SFFT_MLP_MAX_LAYERS) return false;
  if (net->mode != SFFT_MLP_TENSOR_CORES && net->mode != SFFT_MLP_CUDA_CORES) return false;
  for (int l = 0; l <= net->n_layers; ++l)
    if (net->width[l] < 1 || net->width[l] > 1024) return false;
  if (net->width[net->n_layers] != 1) return false;
  for (int l = 0; l < net->n_layers; ++l)
    if (!net->w[l] || !net->b[l]) return false;
  return true;
}

int max_hidden(const sfft_mlp* net) {
  int w = 1;
  for (int l = 1; l < net->n_layers; ++l) w = std::max(w, (int)net->width[l]);
  return w;
}

// offsets (floats) of z_l and h_l, l = 1 .. L-1, in the forward workspace
long long ws_z(const sfft_mlp* net, long long batch, int l) {
  long long o = 0;
  for (int k = 1; k < l; ++k) o += 2 * batch * net->width[k];
  return o;
}
long long ws_h(const sfft_mlp* net, long long batch, int l) { return ws_z(net, batch, l) + batch * net->width[l]; }

// grid.y of the batch-row tiles is limited to 65535
bool batch_ok(long long batch) { return batch >= 0 && (batch + kTile - 1) / kTile <= 65535; }

int grid_1d(long long n) { return (int)std::max(1LL, std::min((n + kThreads - 1) / kThreads, 148LL * 8)); }

sfft_status launch_status() { return cudaGetLastError() == cudaSuccess ? SFFT_OK : SFFT_ECUDA; }

}  // namespace

// tensor-core forward pass (mlp_tc.cu)
bool sfft_mlp_tc_shape_ok(const sfft_mlp* net);
sfft_status sfft_mlp_forward_tc(const sfft_mlp* net, const float* x, int64_t batch, float* y, float* ws,
                                cudaStream_t s);
int sfft_mlp_tc_timeouts_read();
long long sfft_mlp_tc_packed_bytes(const sfft_mlp* net);
sfft_status sfft_mlp_tc_pack(const sfft_mlp* net, void* out, cudaStream_t s);

extern "C" {

int64_t sfft_mlp_pack_bytes(const sfft_mlp* net) {
  if (!net_ok(net) || !sfft_mlp_tc_shape_ok(net)) return -1;
  return sfft_mlp_tc_packed_bytes(net);
}

sfft_status sfft_mlp_pack(const sfft_mlp* net, void* packed, void* stream) {
  if (!net_ok(net) || !sfft_mlp_tc_shape_ok(net) || !packed) return SFFT_EINVAL;
  return sfft_mlp_tc_pack(net, packed, reinterpret_cast<cudaStream_t>(stream));
}

int32_t sfft_mlp_tc_timeouts(void) { return sfft_mlp_tc_timeouts_read(); }

int64_t sfft_mlp_workspace_floats(const sfft_mlp* net, int64_t batch) {
  if (!net_ok(net) || batch < 0) return -1;
  return ws_z(net, batch, net->n_layers);
}

sfft_status sfft_mlp_normalize(const double* raw, int64_t batch, int32_t n_in, const double* lo,
                               const double* hi, float* x, int32_t* in_box, void* stream) {
  if (batch < 0 || n_in < 1 || (batch > 0 && (!raw || !lo || !hi || !x))) return SFFT_EINVAL;
  if (batch == 0) return SFFT_OK;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  k_mlp_normalize<<<grid_1d(batch), kThreads, 0, s>>>(raw, batch, n_in, lo, hi, x, in_box);
  return launch_status();
}

sfft_status sfft_mlp_forward(const sfft_mlp* net, const float* x, int64_t batch, float* y, float* ws,
                             float* ws_scratch, void* stream) {
  if (!net_ok(net) || !batch_ok(batch) || (batch > 0 && (!x || !y || (!ws && !ws_scratch && net->n_layers > 1))))
    return SFFT_EINVAL;
  if (batch == 0) return SFFT_OK;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (net->mode == SFFT_MLP_TENSOR_CORES) {
    if (!sfft_mlp_tc_shape_ok(net)) return SFFT_EINVAL;
    return sfft_mlp_forward_tc(net, x, batch, y, ws, s);
  }
  const int L = net->n_layers;
  const long long maxw = max_hidden(net);
  const float* h = x;
  for (int l = 1; l <= L; ++l) {
    const int win = net->width[l - 1], wl = net->width[l];
    float* Z = nullptr;
    float* H = nullptr;
    if (l < L) {
      if (ws) {
        Z = ws + ws_z(net, batch, l);
        H = ws + ws_h(net, batch, l);
      } else {
        H = ws_scratch + (long long)((l - 1) & 1) * batch * maxw;
      }
    } else {
      Z = y;  // the output layer is linear: y = z_L
    }
    const dim3 grid((wl + kTile - 1) / kTile, (unsigned)((batch + kTile - 1) / kTile), 1);
    k_mlp_gemm<uint16_t, EPI_FWD><<<grid, kThreads, 0, s>>>((int)batch, wl, win, h, win, 1, net->w[l - 1],
                                                            win, 1, Z, wl, net->b[l - 1], H, nullptr,
                                                            win);
    if (launch_status()) return SFFT_ECUDA;
    h = H;
  }
  return SFFT_OK;
}

sfft_status sfft_mlp_mse_grad(const float* y, const float* t, int64_t batch, float* dy, float* loss,
                              void* stream) {
  if (batch < 0 || (batch > 0 && (!y || !t || !dy))) return SFFT_EINVAL;
  if (batch == 0) return SFFT_OK;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (loss && cudaMemsetAsync(loss, 0, sizeof(float), s) != cudaSuccess) return SFFT_ECUDA;
  k_mlp_mse<<<grid_1d(batch), kThreads, 0, s>>>(y, t, batch, dy, loss);
  return launch_status();
}

sfft_status sfft_mlp_backward(const sfft_mlp* net, const float* x, int64_t batch, const float* ws,
                              const float* dy, float* const* gw, float* const* gb, float* scratch,
                              void* stream) {
  if (!net_ok(net) || batch < 1 || !batch_ok(batch) || !x || !dy || !gw || !gb ||
      (net->n_layers > 1 && (!ws || !scratch)))
    return SFFT_EINVAL;
  for (int l = 0; l < net->n_layers; ++l)
    if (!gw[l] || !gb[l]) return SFFT_EINVAL;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const int L = net->n_layers;
  const long long maxw = max_hidden(net);
  const float* dz = dy;
  for (int l = L; l >= 1; --l) {
    const int wl = net->width[l], wprev = net->width[l - 1];
    const float* hprev = (l > 1) ? ws + ws_h(net, batch, l - 1) : x;
    // gw_l = dz_l^T h_{l-1}: a reduction over the batch, split across CTAs
    if (cudaMemsetAsync(gw[l - 1], 0, sizeof(float) * (size_t)wl * wprev, s) != cudaSuccess ||
        cudaMemsetAsync(gb[l - 1], 0, sizeof(float) * (size_t)wl, s) != cudaSuccess)
      return SFFT_ECUDA;
    const int tiles = ((wprev + kTile - 1) / kTile) * ((wl + kTile - 1) / kTile);
    const long long max_split = std::max(1LL, ((long long)batch + 255) / 256);
    const int split = (int)std::min<long long>(max_split, std::max(1, (2 * 148 + tiles - 1) / tiles));
    const long long kc = (((long long)batch + split - 1) / split + kStepK - 1) / kStepK * kStepK;
    const dim3 g1((wprev + kTile - 1) / kTile, (wl + kTile - 1) / kTile, split);
    k_mlp_gemm<float, EPI_PLAIN><<<g1, kThreads, 0, s>>>(wl, wprev, (int)batch, dz, 1, wl, hprev, 1, wprev,
                                                         gw[l - 1], wprev, nullptr, nullptr, nullptr,
                                                         (int)kc);
    if (launch_status()) return SFFT_ECUDA;
    const long long chunk = std::max(1LL, ((long long)batch + 148 * 4 - 1) / (148 * 4));
    k_mlp_colsum<<<(unsigned)((batch + chunk - 1) / chunk), kThreads, 0, s>>>(dz, batch, wl, chunk, gb[l - 1]);
    if (launch_status()) return SFFT_ECUDA;
    if (l > 1) {
      // dz_{l-1} = (dz_l W_l) * GELU'(z_{l-1})
      float* dn = scratch + (long long)(l & 1) * batch * maxw;
      const dim3 g2((wprev + kTile - 1) / kTile, (unsigned)((batch + kTile - 1) / kTile), 1);
      k_mlp_gemm<uint16_t, EPI_BWD><<<g2, kThreads, 0, s>>>((int)batch, wprev, wl, dz, wl, 1, net->w[l - 1], 1,
                                                            wprev, dn, wprev, nullptr, nullptr,
                                                            ws + ws_z(net, batch, l - 1), wl);
      if (launch_status()) return SFFT_ECUDA;
      dz = dn;
    }
  }
  return SFFT_OK;
}

sfft_status sfft_mlp_adam(int64_t count, float* p, uint16_t* p_bf16, const float* g, float* m, float* v,
                          float lr, float beta1, float beta2, float eps, int64_t step, void* stream) {
  if (count < 0 || step < 1 || (count > 0 && (!p || !g || !m || !v))) return SFFT_EINVAL;
  if (count == 0) return SFFT_OK;
  const float c1 = (float)(1.0 - pow((double)beta1, (double)step));
  const float c2 = (float)(1.0 - pow((double)beta2, (double)step));
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  k_mlp_adam<<<grid_1d(count), kThreads, 0, s>>>(count, p, p_bf16, g, m, v, lr, beta1, beta2, eps, c1, c2);
  return launch_status();
}

}  // extern "C"
