// Price surrogate forward pass on the fifth-generation tensor cores: every
// layer's product runs as tcgen05.mma kind::f16 (bfloat16 operands, float32
// accumulation in tensor memory), the bias, GELU and bfloat16 rounding of the
// activations are fused into the epilogue, and the activations of a 128-row
// tile never leave shared memory between layers.
//
// One CTA (128 threads, two per SM) takes 128-row tiles of the batch in turn:
//   layer 1   A = the inputs split into bfloat16 pairs hi + lo (hi the nearest
//             bfloat16 of x, lo that of x - hi), B = [W_1 | W_1] along K, so a
//             single K = 16 MMA forms sum_k (hi_k + lo_k) W_1[n, k]: the inputs
//             keep about 16 significant bits instead of bfloat16's 8;
//   layers 2.. A = the previous layer's bfloat16 activations (128 x K in
//             shared memory), B = W_l streamed from global memory (L2) in
//             K-chunks of 32 through two shared-memory buffers, MMAs of
//             chunk c overlapping the copy of chunk c + 1;
//   epilogue  each warp reads its 32 rows of the accumulator from tensor
//             memory, adds the bias, applies GELU and writes the rounded
//             activations back as the next layer's A operand (and, when a
//             workspace is given, z and h to global memory for the backward
//             pass); the last hidden layer instead folds the linear output
//             layer y = h W_L^T + b_L into its epilogue.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "../../include/sfft_mlp.h"
#include "tc.cuh"

namespace {

constexpr int kRows = 128;      // rows per tile = tensor-memory lanes
constexpr int kMaxW = 256;      // widest layer (accumulator columns)
constexpr int kChunk = 32;      // K elements per streamed weight chunk
constexpr int kThreadsTc = 128;
constexpr uint32_t kTmemCols = 256;
constexpr long long kWaitPolls = 1LL << 22;

// shared memory: A tile (128 x 256 bf16), two weight-chunk buffers
// (256 x 32 bf16 each), bias and output weights (fp32), barriers
constexpr int kABytes = kRows * kMaxW * 2;
constexpr int kBBytes = kMaxW * kChunk * 2;
constexpr int kSmemBytes = kABytes + 2 * kBBytes + 2 * kMaxW * 4 + 64 + 1024;

struct TcNet {
  int L;
  int w[SFFT_MLP_MAX_LAYERS + 1];
  const uint16_t* W[SFFT_MLP_MAX_LAYERS];
  const float* b[SFFT_MLP_MAX_LAYERS];
};

__device__ int g_mlp_tc_timeouts = 0;

__device__ __forceinline__ float gelu_f(float z) { return z * normcdff(z); }

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<const uint32_t*>(&v);
}
__device__ __forceinline__ float bf16_round(float a) { return __bfloat162float(__float2bfloat16_rn(a)); }

__global__ void __launch_bounds__(kThreadsTc, 2)
    k_mlp_fwd_tc(TcNet net, const float* __restrict__ x, long long batch, float* y, float* ws) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  // 1024-byte aligned base for the operand tiles
  unsigned char* base = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  unsigned char* As = base;
  unsigned char* Bs0 = As + kABytes;
  float* bias_s = reinterpret_cast<float*>(Bs0 + 2 * kBBytes);
  float* wout_s = bias_s + kMaxW;
  uint64_t* mbar = reinterpret_cast<uint64_t*>(wout_s + kMaxW);  // 3 barriers
  uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar + 3);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int L = net.L;
  if (tid == 0) {
    for (int i = 0; i < 3; ++i) tc::mbar_init(mbar + i, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) tc::tmem_alloc(tslot, kTmemCols);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *tslot;
  uint32_t phase[3] = {0u, 0u, 0u};
  bool ok = true;
  const uint32_t As_a = tc::smem_u32(As);
  const uint32_t Bs_a[2] = {tc::smem_u32(Bs0), tc::smem_u32(Bs0 + kBBytes)};
  const float bL = (L >= 1) ? net.b[L - 1][0] : 0.f;
  // output-layer weights (1 x w_{L-1}) as floats, once
  for (int k = tid; k < net.w[L - 1]; k += kThreadsTc)
    wout_s[k] = __uint_as_float((uint32_t)net.W[L - 1][k] << 16);

  const long long ntiles = (batch + kRows - 1) / kRows;
  for (long long tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
    const long long row0 = tile * kRows;
    const long long row = row0 + tid;  // this thread's row in staging and epilogue
    const bool live = row < batch;
    // ---- layer 1 operands: A = [hi(x) | lo(x)], B = [W_1 | W_1], K = 16
    {
      const int w0 = net.w[0];
      float xv[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) xv[k] = (live && k < w0) ? x[row * w0 + k] : 0.f;
      uint32_t hi[4], lo[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const float h0 = bf16_round(xv[2 * k]), h1 = bf16_round(xv[2 * k + 1]);
        hi[k] = pack_bf16(h0, h1);
        lo[k] = pack_bf16(xv[2 * k] - h0, xv[2 * k + 1] - h1);
      }
      *reinterpret_cast<uint4*>(As + tc::kmajor_off(tid, 0, 32)) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
      *reinterpret_cast<uint4*>(As + tc::kmajor_off(tid, 16, 32)) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
      const int w1 = net.w[1];
      for (int n = tid; n < w1; n += kThreadsTc) {
        uint32_t wv[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const uint32_t a = (2 * k < w0) ? net.W[0][n * w0 + 2 * k] : 0u;
          const uint32_t b = (2 * k + 1 < w0) ? net.W[0][n * w0 + 2 * k + 1] : 0u;
          wv[k] = a | (b << 16);
        }
        const uint4 v = make_uint4(wv[0], wv[1], wv[2], wv[3]);
        *reinterpret_cast<uint4*>(Bs0 + tc::kmajor_off(n, 0, 32)) = v;
        *reinterpret_cast<uint4*>(Bs0 + tc::kmajor_off(n, 16, 32)) = v;
      }
    }
    for (int l = 1; l < L && ok; ++l) {
      const int K = net.w[l - 1], N = net.w[l];
      for (int c = tid; c < N; c += kThreadsTc) bias_s[c] = net.b[l - 1][c];
      const uint32_t idesc = tc::idesc_bf16(kRows, N);
      if (l == 1) {
        tc::fence_proxy_async();
        tc::fence_before_sync();
        __syncthreads();
        if (tid == 0) {
          tc::fence_after_sync();
          tc::mma_bf16(tmem, tc::kmajor_desc(As_a, 32), tc::kmajor_desc(Bs_a[0], 32), idesc, 0u);
          tc::commit(mbar + 2);
        }
        ok = __syncthreads_and(tc::mbar_wait(mbar + 2, phase[2], kWaitPolls));
        phase[2] ^= 1u;
      } else {
        // stream W_l (N x K, row-major = K-major) in chunks of kChunk along K
        const int nch = (K + kChunk - 1) / kChunk;
        const uint16_t* Wl = net.W[l - 1];
        auto load_chunk = [&](int c) {
          const int k0 = c * kChunk, kc = min(kChunk, K - k0), kb = 2 * kc;
          const int pieces = N * (kc >> 3);
          unsigned char* dst = Bs0 + (c & 1) * kBBytes;
          for (int pc = tid; pc < pieces; pc += kThreadsTc) {
            const int n = pc / (kc >> 3), j = pc - n * (kc >> 3);
            tc::cp_async16(tc::smem_u32(dst + tc::kmajor_off(n, 16 * j, kb)), Wl + (size_t)n * K + k0 + 8 * j);
          }
          tc::cp_async_commit();
        };
        load_chunk(0);
        if (nch > 1) load_chunk(1);
        for (int c = 0; c < nch && ok; ++c) {
          if (c + 1 < nch)
            tc::cp_async_wait<1>();
          else
            tc::cp_async_wait<0>();
          tc::fence_proxy_async();
          tc::fence_before_sync();
          __syncthreads();
          const int k0 = c * kChunk, kc = min(kChunk, K - k0);
          if (tid == 0) {
            tc::fence_after_sync();
            for (int kk = 0; kk < kc / 16; ++kk) {
              const uint64_t ad = tc::kmajor_desc(As_a + (uint32_t)(k0 + 16 * kk) * 16u, 2 * K);
              const uint64_t bd = tc::kmajor_desc(Bs_a[c & 1] + (uint32_t)kk * 256u, 2 * kc);
              tc::mma_bf16(tmem, ad, bd, idesc, (c | kk) ? 1u : 0u);
            }
            tc::commit(mbar + (c & 1));
          }
          if (c + 2 < nch) {
            // buffer c & 1 is free once chunk c's MMAs completed
            ok = __syncthreads_and(tc::mbar_wait(mbar + (c & 1), phase[c & 1], kWaitPolls));
            phase[c & 1] ^= 1u;
            if (ok) load_chunk(c + 2);
          }
        }
        // the last one or two commits: every MMA of the layer has completed
        for (int c = max(0, nch - 2); c < nch && ok; ++c) {
          ok = __syncthreads_and(tc::mbar_wait(mbar + (c & 1), phase[c & 1], kWaitPolls));
          phase[c & 1] ^= 1u;
        }
      }
      if (!ok) break;
      tc::fence_after_sync();
      // ---- epilogue: rows 32 warp + lane, columns in blocks of 16
      const bool last = (l == L - 1);
      const int rloc = 32 * warp + lane;
      const long long grow = row0 + rloc;
      const bool glive = grow < batch;
      float* zg = nullptr;
      float* hg = nullptr;
      if (ws && glive) {
        long long o = 0;
        for (int k = 1; k < l; ++k) o += 2 * batch * net.w[k];
        zg = ws + o + grow * N;
        hg = ws + o + batch * N + grow * N;
      }
      float yacc = 0.f;
      for (int cb = 0; cb < N; cb += 16) {
        float v[16];
        tc::tmem_ld16(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)cb, v);
        float h[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          v[i] += bias_s[cb + i];
          h[i] = bf16_round(gelu_f(v[i]));
        }
        if (last) {
#pragma unroll
          for (int i = 0; i < 16; ++i) yacc = fmaf(h[i], wout_s[cb + i], yacc);
        } else {
          uint32_t pk[8];
#pragma unroll
          for (int i = 0; i < 8; ++i) pk[i] = pack_bf16(h[2 * i], h[2 * i + 1]);
          *reinterpret_cast<uint4*>(As + tc::kmajor_off(rloc, 2 * cb, 2 * N)) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
          *reinterpret_cast<uint4*>(As + tc::kmajor_off(rloc, 2 * cb + 16, 2 * N)) =
              make_uint4(pk[4], pk[5], pk[6], pk[7]);
        }
        if (zg) {
#pragma unroll
          for (int i = 0; i < 16; i += 4) {
            *reinterpret_cast<float4*>(zg + cb + i) = make_float4(v[i], v[i + 1], v[i + 2], v[i + 3]);
            *reinterpret_cast<float4*>(hg + cb + i) = make_float4(h[i], h[i + 1], h[i + 2], h[i + 3]);
          }
        }
      }
      if (last && glive) y[grow] = yacc + bL;
      // the accumulator is read and A rewritten before the next MMAs
      tc::fence_before_sync();
      __syncthreads();
    }
  }
  if (!ok) {
    if (tid == 0) atomicAdd(&g_mlp_tc_timeouts, 1);
  }
  tc::cp_async_wait<0>();  // no copy of this thread is left in flight
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_free(tmem, kTmemCols);
}

}  // namespace

// Shape the tensor-core forward pass handles: at least one hidden layer,
// inputs w_0 <= 8, hidden widths multiples of 16 in [16, 256], one output.
bool sfft_mlp_tc_shape_ok(const sfft_mlp* net) {
  if (net->n_layers < 2 || net->width[0] < 1 || net->width[0] > 8 || net->width[net->n_layers] != 1) return false;
  for (int l = 1; l < net->n_layers; ++l)
    if (net->width[l] < 16 || net->width[l] > kMaxW || (net->width[l] & 15)) return false;
  return true;
}

sfft_status sfft_mlp_forward_tc(const sfft_mlp* net, const float* x, int64_t batch, float* y, float* ws,
                                cudaStream_t s) {
  // the hidden layers' weights are copied to shared memory in 16-byte pieces
  // and the workspace is written in 16-byte vectors
  for (int l = 1; l + 1 < net->n_layers; ++l)
    if (reinterpret_cast<uintptr_t>(net->w[l]) & 15) return SFFT_EINVAL;
  if (reinterpret_cast<uintptr_t>(ws) & 15) return SFFT_EINVAL;
  static int attr_dev = -1;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return SFFT_ECUDA;
  if (attr_dev != dev) {
    if (cudaFuncSetAttribute(k_mlp_fwd_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes) != cudaSuccess)
      return SFFT_ECUDA;
    attr_dev = dev;
  }
  int sms = 148;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  TcNet tn;
  tn.L = net->n_layers;
  for (int l = 0; l <= net->n_layers; ++l) tn.w[l] = net->width[l];
  for (int l = 0; l < net->n_layers; ++l) {
    tn.W[l] = net->w[l];
    tn.b[l] = net->b[l];
  }
  const long long ntiles = (batch + kRows - 1) / kRows;
  const int grid = (int)std::max(1LL, std::min(ntiles, 2LL * sms));
  k_mlp_fwd_tc<<<grid, kThreadsTc, kSmemBytes, s>>>(tn, x, batch, y, ws);
  return cudaGetLastError() == cudaSuccess ? SFFT_OK : SFFT_ECUDA;
}

int sfft_mlp_tc_timeouts_read() {
  int v = 0;
  if (cudaMemcpyFromSymbol(&v, g_mlp_tc_timeouts, sizeof(int)) != cudaSuccess) return -1;
  return v;
}
