// Price surrogate forward pass on the fifth-generation tensor cores: every
// layer's product runs as tcgen05.mma kind::f16 (bfloat16 operands, float32
// accumulation in tensor memory), the bias, GELU and bfloat16 rounding of the
// activations are fused into the epilogue, and the activations of a tile
// never leave shared memory between layers.
//
// One persistent CTA per SM, warp-specialised, works on pairs of 128-row
// tiles (slots 0 and 1) with one tensor-memory accumulator each:
//   warp 0      producer: bulk asynchronous copies (cp.async.bulk, completing
//               on mbarriers) of the weights, pre-packed in the operand layout
//               (sfft_mlp_pack), through a ring of shared-memory stages;
//   warp 1      one thread issues the MMAs of a layer for slot 0, then slot 1,
//               and commits each accumulator to the epilogue;
//   warps 2..17 epilogue, eight warps per slot (a thread owns one row and
//               half of the columns): stage the inputs, then for each hidden
//               layer drain the slot's accumulator (tcgen05.ld), add the bias,
//               apply GELU, round to bfloat16 and write the next layer's A
//               operand into shared memory. The linear output layer
//               y = h W_L^T + b_L is one more MMA with W_L padded to 16 zero
//               rows, whose column 0 the epilogue reads last.
// While the epilogue drains one slot, the tensor cores run the other slot's
// layer, so the two overlap.
//
// Layer 1 takes the inputs as the bfloat16 pair hi + lo (hi = bf16(x), lo =
// bf16(x - hi)) against B = [W_1 | W_1] along K: one K = 16 MMA forms
// sum_k (hi_k + lo_k) W_1[n, k], so the inputs keep about 16 significant bits
// instead of bfloat16's 8.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "../../include/sfft_mlp.h"
#include "tc.cuh"

namespace {

constexpr int kRows = 128;         // rows per tile = tensor-memory lanes
constexpr int kMaxW = 256;         // widest hidden layer (accumulator columns)
constexpr int kMaxHidden = SFFT_MLP_MAX_LAYERS - 1;
constexpr int kChunk = 64;         // K elements per weight stage
// The MMA thread waits on one stage barrier per chunk, and every such wait
// between MMAs leaves the tensor pipe idle for ~180 cycles (measured on
// B300): 64-wide chunks (four MMAs per wait) in two 32 KB stages beat 32-wide
// ones in three 16 KB stages (0.866 against 0.940 ms for 2^20 queries); the
// bulk copy of the next chunk still lands while the current one runs.
constexpr int kStages = 2;
constexpr int kEpiWarps = 16;   // eight per slot: two per lane quadrant, one per column half
constexpr int kThreadsTc = 32 * (2 + kEpiWarps);
constexpr int kOutRows = 16;    // the output layer's single row, padded to the smallest MMA width
constexpr uint32_t kTmemCols = 512;  // two accumulators of 256 columns
constexpr long long kWaitPolls = 1LL << 22;

constexpr int kABytes = kRows * kMaxW * 2;  // one slot's activations
constexpr int kBBytes = kMaxW * kChunk * 2;  // one weight stage
constexpr int kB1Bytes = kMaxW * 32;         // [W_1 | W_1], K = 16
constexpr int kSmemBytes = 2 * kABytes + kStages * kBBytes + kB1Bytes + 4 * kMaxHidden * kMaxW + 128 + 1024;

struct TcNet {
  int L;
  int w[SFFT_MLP_MAX_LAYERS + 1];
  const uint16_t* W[SFFT_MLP_MAX_LAYERS];
  const float* b[SFFT_MLP_MAX_LAYERS];
  long long pk_off[SFFT_MLP_MAX_LAYERS];  // byte offset of W[l]'s chunks in the packed image (l >= 1)
};

__device__ int g_mlp_tc_timeouts = 0;

// GELU(z) = z Phi(z), Phi(z) = (1 + erf(z / sqrt 2)) / 2, with erf from
// Hastings' rational approximation (Abramowitz & Stegun 7.1.26; absolute
// error at most 1.5e-7 on x >= 0):
//   erf(x) = 1 - t (a1 + t (a2 + t (a3 + t (a4 + t a5)))) exp(-x^2),
//   t = 1 / (1 + p x),
// so the tail Q(|z|) = (1 - erf(|z| / sqrt 2)) / 2 costs one reciprocal and
// one exponential, and Phi(z) = 1 - Q for z >= 0, Q for z < 0. The error in
// GELU, at most 8e-8 |z|, lies far below the bfloat16 rounding that follows.
__device__ __forceinline__ float rcp_approx(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
// The scalar form, which gelu2 below evaluates on pairs (kept as its
// specification; the kernels call gelu2).
[[maybe_unused]] __device__ __forceinline__ float gelu_f(float z) {
  // with a = |z|: 1 + p x = 1 + (p / sqrt 2) a and exp(-x^2) = 2^(-a^2 log2(e) / 2);
  // the coefficients carry the factor 1/2 of Q
  const float a = fabsf(z);
  const float t = rcp_approx(fmaf(0.23164188827f, a, 1.0f));
  float pl = fmaf(t, 0.5307027145f, -0.7265760135f);
  pl = fmaf(t, pl, 0.7107068705f);
  pl = fmaf(t, pl, -0.142248368f);
  pl = fmaf(t, pl, 0.127414796f);
  float e;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(e) : "f"(-0.72134752044448170f * a * a));
  // z Phi(z) = max(z, 0) - |z| Q(|z|) for either sign of z
  return fmaf(-(a * t) * pl, e, fmaxf(z, 0.f));
}

// The same GELU on two activations held as a pair in one 64-bit register:
// the products and the polynomial run as packed FP32 instructions
// (fma/mul.rn.f32x2, one instruction for both lanes of the pair), the two
// reciprocals, exponentials and maxima per element. The arithmetic and its
// rounding are those of gelu_f (the sign of Q folded into the coefficients).
__device__ __forceinline__ uint64_t f2_fma(uint64_t a, uint64_t b, uint64_t c) {
  uint64_t d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
__device__ __forceinline__ uint64_t f2_mul(uint64_t a, uint64_t b) {
  uint64_t d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ uint64_t f2_add(uint64_t a, uint64_t b) {
  uint64_t d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ uint64_t f2_pack(float lo, float hi) {
  uint64_t d;
  asm("mov.b64 %0, {%1, %2};" : "=l"(d) : "f"(lo), "f"(hi));
  return d;
}
__device__ __forceinline__ void f2_unpack(uint64_t p, float& lo, float& hi) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(p));
}
// a float constant in both halves (folded by the compiler)
__device__ __forceinline__ uint64_t f2c(float f) {
  const uint64_t b = __float_as_uint(f);
  return (b << 32) | b;
}
__device__ __forceinline__ float ex2_approx(float x) {
  float r;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ uint64_t gelu2(uint64_t z) {
  const uint64_t a = z & 0x7FFFFFFF7FFFFFFFull;  // |z| in both halves
  float d0, d1;
  f2_unpack(f2_fma(f2c(0.23164188827f), a, f2c(1.0f)), d0, d1);
  const uint64_t t = f2_pack(rcp_approx(d0), rcp_approx(d1));
  // -P(t): the coefficients of gelu_f, negated
  uint64_t pl = f2_fma(t, f2c(-0.5307027145f), f2c(0.7265760135f));
  pl = f2_fma(t, pl, f2c(-0.7107068705f));
  pl = f2_fma(t, pl, f2c(0.142248368f));
  pl = f2_fma(t, pl, f2c(-0.127414796f));
  float s0, s1;
  f2_unpack(f2_mul(f2_mul(a, f2c(-0.72134752044448170f)), a), s0, s1);
  const uint64_t e = f2_pack(ex2_approx(s0), ex2_approx(s1));
  float z0, z1;
  f2_unpack(z, z0, z1);
  const uint64_t m = f2_pack(fmaxf(z0, 0.f), fmaxf(z1, 0.f));
  // z Phi(z) = max(z, 0) - |z| t P(t) e
  return f2_fma(f2_mul(f2_mul(a, t), pl), e, m);
}

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<const uint32_t*>(&v);
}
__device__ __forceinline__ float bf16_lo(uint32_t p) { return __uint_as_float(p << 16); }
__device__ __forceinline__ float bf16_hi(uint32_t p) { return __uint_as_float(p & 0xFFFF0000u); }
__device__ __forceinline__ float bf16_round(float a) { return __bfloat162float(__float2bfloat16_rn(a)); }

// Byte offset, in a layer's part of the packed weight image, of element
// (n, k) of its W (N x K): chunk c = k / 64 holds N x min(64, K - 64 c)
// elements in the K-major operand layout.
__device__ __forceinline__ long long packed_off(int n, int k, int N, int K) {
  const int c = k / kChunk, kc = min(kChunk, K - c * kChunk);
  return (long long)c * N * kChunk * 2 + tc::kmajor_off(n, 2 * (k - c * kChunk), 2 * kc);
}

__global__ void k_mlp_pack(TcNet net, unsigned char* out) {
  // [W_1 | W_1] (w_1 x 16, rows of 32 bytes) first, then every later hidden layer
  const int w0 = net.w[0], w1 = net.w[1];
  const long long stride = (long long)gridDim.x * blockDim.x;
  const long long tot1 = (long long)w1 * 16;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < tot1; i += stride) {
    const int n = (int)(i / 16), k = (int)(i % 16);
    const int kk = k & 7;
    const uint16_t v = kk < w0 ? net.W[0][n * w0 + kk] : (uint16_t)0;
    *reinterpret_cast<uint16_t*>(out + tc::kmajor_off(n, 2 * k, 32)) = v;
  }
  for (int l = 1; l < net.L; ++l) {
    // hidden layers N x K; the output layer (l = L - 1, one row) as 16 rows
    const int K = net.w[l], N = (l + 1 < net.L) ? net.w[l + 1] : kOutRows;
    const long long tot = (long long)N * K;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < tot; i += stride) {
      const int n = (int)(i / K), k = (int)(i % K);
      const uint16_t v = (l + 1 < net.L || n == 0) ? net.W[l][(long long)n * K + k] : (uint16_t)0;
      *reinterpret_cast<uint16_t*>(out + net.pk_off[l] + packed_off(n, k, N, K)) = v;
    }
  }
}

__global__ void __launch_bounds__(kThreadsTc, 1)
    k_mlp_fwd_tc(TcNet net, const unsigned char* __restrict__ packed, const float* __restrict__ x, long long batch,
                 float* y, float* ws) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* base = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  unsigned char* Aslot[2] = {base, base + kABytes};
  unsigned char* ring = base + 2 * kABytes;
  unsigned char* B1 = ring + kStages * kBBytes;
  float* bias_s = reinterpret_cast<float*>(B1 + kB1Bytes);  // [hidden layer][kMaxW]
  uint64_t* bars = reinterpret_cast<uint64_t*>(bias_s + kMaxHidden * kMaxW);
  uint64_t* w_full = bars;
  uint64_t* w_empty = bars + kStages;
  uint64_t* acc_full = bars + 2 * kStages;
  uint64_t* a_ready = acc_full + 2;
  uint64_t* b1_full = a_ready + 2;
  uint32_t* tslot = reinterpret_cast<uint32_t*>(b1_full + 1);
  volatile int* abort = reinterpret_cast<volatile int*>(tslot + 1);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int L = net.L, H = L - 1;
  if (tid == 0) {
    for (int i = 0; i < kStages; ++i) {
      tc::mbar_init(w_full + i, 1);
      tc::mbar_init(w_empty + i, 1);
    }
    for (int i = 0; i < 2; ++i) {
      tc::mbar_init(acc_full + i, 1);
      tc::mbar_init(a_ready + i, kEpiWarps * 16);  // the eight warps of slot i
    }
    tc::mbar_init(b1_full, 1);
    *abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  for (int i = tid; i < H * kMaxW; i += kThreadsTc) {
    const int l = i / kMaxW, c = i - l * kMaxW;
    bias_s[i] = c < net.w[l + 1] ? net.b[l][c] : 0.f;
  }
  if (warp == 1) tc::tmem_alloc(tslot, kTmemCols);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *tslot;
  const long long ntiles = (batch + kRows - 1) / kRows;
  const long long npairs = (ntiles + 1) / 2;

  if (warp == 0) {
    // ---------------------------------------------------------------- producer
    if (lane == 0) {
      const uint32_t b1_bytes = (uint32_t)net.w[1] * 32u;
      tc::mbar_expect_tx(b1_full, b1_bytes);
      tc::bulk_g2s(tc::smem_u32(B1), packed, b1_bytes, b1_full);
      uint32_t g = 0;
      bool go = true;
      for (long long pair = blockIdx.x; pair < npairs && go; pair += gridDim.x)
        for (int l = 1; l <= H && go; ++l) {
          const int K = net.w[l], N = (l < H) ? net.w[l + 1] : kOutRows;
          const int nch = (K + kChunk - 1) / kChunk;
          for (int s = 0; s < 2 && go; ++s)
            for (int c = 0; c < nch; ++c, ++g) {
              const int st = (int)(g % kStages);
              const uint32_t round = g / kStages;
              if (!tc::mbar_wait_or_abort(w_empty + st, (round & 1u) ^ 1u, kWaitPolls, abort)) {
                go = false;
                break;
              }
              const uint32_t bytes = (uint32_t)N * 2u * (uint32_t)min(kChunk, K - c * kChunk);
              tc::mbar_expect_tx(w_full + st, bytes);
              tc::bulk_g2s(tc::smem_u32(ring + st * kBBytes),
                           packed + net.pk_off[l] + (long long)c * N * kChunk * 2, bytes, w_full + st);
            }
        }
      if (!go) {
        // let the copies already issued land before the CTA exits: the last
        // copy into each stage completes the phase (g_last / kStages) & 1
        for (int st = 0; st < kStages; ++st) {
          if (g < (uint32_t)(st + 1)) continue;
          const uint32_t last = g - 1 - (uint32_t)((g - 1 - st) % kStages);
          tc::mbar_wait(w_full + st, (last / kStages) & 1u, 1 << 16);
        }
      }
    }
  } else if (warp == 1) {
    // ---------------------------------------------------------------- MMA issue
    if (lane == 0) {
      bool go = tc::mbar_wait_or_abort(b1_full, 0u, kWaitPolls, abort);
      uint32_t g = 0, ar_ph[2] = {0u, 0u};
      for (long long pair = blockIdx.x; pair < npairs && go; pair += gridDim.x)
        for (int l = 0; l <= H && go; ++l) {
          const int K = net.w[l], N = (l < H) ? net.w[l + 1] : kOutRows;
          const uint32_t idesc = tc::idesc_bf16(kRows, N);
          for (int s = 0; s < 2 && go; ++s) {
            if (!tc::mbar_wait_or_abort(a_ready + s, ar_ph[s], kWaitPolls, abort)) {
              go = false;
              break;
            }
            ar_ph[s] ^= 1u;
            tc::fence_after_sync();
            const uint32_t d = tmem + 256u * (uint32_t)s;
            const uint32_t a_addr = tc::smem_u32(Aslot[s]);
            if (l == 0) {
              tc::mma_bf16(d, tc::kmajor_desc(a_addr, 32), tc::kmajor_desc(tc::smem_u32(B1), 32), idesc, 0u);
            } else {
              const int nch = (K + kChunk - 1) / kChunk;
              for (int c = 0; c < nch; ++c, ++g) {
                const int st = (int)(g % kStages);
                if (!tc::mbar_wait_or_abort(w_full + st, (g / kStages) & 1u, kWaitPolls, abort)) {
                  go = false;
                  break;
                }
                tc::fence_after_sync();
                const int kc = min(kChunk, K - c * kChunk);
                const uint32_t b_addr = tc::smem_u32(ring + st * kBBytes);
                for (int kk = 0; kk < kc / 16; ++kk) {
                  const uint64_t ad = tc::kmajor_desc(a_addr + (uint32_t)(c * kChunk + 16 * kk) * 16u, 2 * K);
                  const uint64_t bd = tc::kmajor_desc(b_addr + (uint32_t)kk * 256u, 2 * kc);
                  tc::mma_bf16(d, ad, bd, idesc, (c | kk) ? 1u : 0u);
                }
                tc::commit(w_empty + st);  // the stage is free once these MMAs complete
              }
            }
            if (go) tc::commit(acc_full + s);
          }
        }
    }
  } else {
    // ---------------------------------------------------------------- epilogue
    // warps 2..9 serve slot 0, warps 10..17 slot 1; within a slot, the two
    // warps of a lane quadrant take alternate 16-column blocks
    const int e = warp - 2;
    const int s = e >> 3;
    const int q = warp & 3;  // tensor-memory lane quadrant this warp may read
    const int half = (e >> 2) & 1;
    const int rloc = 32 * q + lane;
    const uint32_t tbase = tmem + 256u * (uint32_t)s + ((uint32_t)(32 * q) << 16);
    unsigned char* As = Aslot[s];
    uint32_t af_ph = 0u;
    bool go = true;
    const float bL = net.b[H][0];
    const int w0 = net.w[0];
    for (long long pair = blockIdx.x; pair < npairs && go; pair += gridDim.x) {
      const long long grow = (2 * pair + s) * kRows + rloc;
      const bool glive = grow < batch;
      if (half == 0) {
        // this slot's inputs: A = [hi(x) | lo(x)], K = 16
        float xv[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) xv[k] = (glive && k < w0) ? x[grow * w0 + k] : 0.f;
        uint32_t hi[4], lo[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const float h0 = bf16_round(xv[2 * k]), h1 = bf16_round(xv[2 * k + 1]);
          hi[k] = pack_bf16(h0, h1);
          lo[k] = pack_bf16(xv[2 * k] - h0, xv[2 * k + 1] - h1);
        }
        *reinterpret_cast<uint4*>(As + tc::kmajor_off(rloc, 0, 32)) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
        *reinterpret_cast<uint4*>(As + tc::kmajor_off(rloc, 16, 32)) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
        tc::fence_proxy_async();
      }
      tc::fence_before_sync();
      tc::mbar_arrive(a_ready + s);
      for (int l = 1; l <= H + 1; ++l) {
        if (!tc::mbar_wait_or_abort(acc_full + s, af_ph, kWaitPolls, abort)) {
          go = false;
          break;
        }
        af_ph ^= 1u;
        tc::fence_after_sync();
        if (l == H + 1) {
          // output layer: column 0 of the accumulator
          if (half == 0) {
            float v[16];
            tc::tmem_ld16(tbase, v);
            if (glive) y[grow] = v[0] + bL;
          }
          break;  // the next pair's staging arrives for this slot
        }
        const int N = net.w[l];
        const float* bias = bias_s + (l - 1) * kMaxW;
        float* zg = nullptr;
        float* hg = nullptr;
        if (ws && glive) {
          long long o = 0;
          for (int k = 1; k < l; ++k) o += 2 * batch * net.w[k];
          zg = ws + o + grow * N;
          hg = ws + o + batch * N + grow * N;
        }
        // software-pipelined: the load of the next block is in flight while
        // this one is computed
        uint32_t rn[16];
        tc::tmem_ld16_start(tbase + (uint32_t)(16 * half), rn);
        tc::tmem_ld_wait16(rn);
        for (int cb = 16 * half; cb < N; cb += 32) {
          float v[16];
#pragma unroll
          for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(rn[i]);
          if (cb + 32 < N) tc::tmem_ld16_start(tbase + (uint32_t)(cb + 32), rn);
          uint32_t pk[8];
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            const float4 bb = *reinterpret_cast<const float4*>(bias + cb + 4 * i);
#pragma unroll
            for (int h = 0; h < 2; ++h) {
              const int j = 2 * i + h;
              const uint64_t zz = f2_add(f2_pack(v[2 * j], v[2 * j + 1]), h ? f2_pack(bb.z, bb.w) : f2_pack(bb.x, bb.y));
              f2_unpack(zz, v[2 * j], v[2 * j + 1]);
              float g0, g1;
              f2_unpack(gelu2(zz), g0, g1);
              pk[j] = pack_bf16(g0, g1);
            }
          }
          *reinterpret_cast<uint4*>(As + tc::kmajor_off(rloc, 2 * cb, 2 * N)) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
          *reinterpret_cast<uint4*>(As + tc::kmajor_off(rloc, 2 * cb + 16, 2 * N)) =
              make_uint4(pk[4], pk[5], pk[6], pk[7]);
          if (zg) {
#pragma unroll
            for (int i = 0; i < 16; i += 4) {
              *reinterpret_cast<float4*>(zg + cb + i) = make_float4(v[i], v[i + 1], v[i + 2], v[i + 3]);
              *reinterpret_cast<float4*>(hg + cb + i) = make_float4(
                  bf16_lo(pk[i / 2]), bf16_hi(pk[i / 2]), bf16_lo(pk[i / 2 + 1]), bf16_hi(pk[i / 2 + 1]));
            }
          }
          if (cb + 32 < N) tc::tmem_ld_wait16(rn);
        }
        tc::fence_proxy_async();
        tc::fence_before_sync();
        tc::mbar_arrive(a_ready + s);  // A holds the next layer's input; the accumulator is drained
      }
    }
  }
  if (*abort && tid == 0) atomicAdd(&g_mlp_tc_timeouts, 1);
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 1) {
    tc::fence_after_sync();
    tc::tmem_free(tmem, kTmemCols);
  }
}

void fill_net(const sfft_mlp* net, TcNet* tn) {
  tn->L = net->n_layers;
  for (int l = 0; l <= net->n_layers; ++l) tn->w[l] = net->width[l];
  long long off = (long long)net->width[1] * 32;
  for (int l = 0; l < net->n_layers; ++l) {
    tn->W[l] = net->w[l];
    tn->b[l] = net->b[l];
    tn->pk_off[l] = 0;
    if (l >= 1) {
      tn->pk_off[l] = off;
      off += 2LL * net->width[l] * (l + 1 < net->n_layers ? net->width[l + 1] : kOutRows);
    }
  }
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

long long sfft_mlp_tc_packed_bytes(const sfft_mlp* net) {
  long long off = (long long)net->width[1] * 32;
  for (int l = 1; l < net->n_layers; ++l)
    off += 2LL * net->width[l] * (l + 1 < net->n_layers ? net->width[l + 1] : kOutRows);
  return off;
}

sfft_status sfft_mlp_tc_pack(const sfft_mlp* net, void* out, cudaStream_t s) {
  if (reinterpret_cast<uintptr_t>(out) & 15) return SFFT_EINVAL;
  TcNet tn;
  fill_net(net, &tn);
  k_mlp_pack<<<148, 256, 0, s>>>(tn, reinterpret_cast<unsigned char*>(out));
  return cudaGetLastError() == cudaSuccess ? SFFT_OK : SFFT_ECUDA;
}

sfft_status sfft_mlp_forward_tc(const sfft_mlp* net, const float* x, int64_t batch, float* y, float* ws,
                                cudaStream_t s) {
  // the packed weights are copied in 16-byte aligned bulk pieces and the
  // workspace is written in 16-byte vectors
  if (!net->tc_weights || (reinterpret_cast<uintptr_t>(net->tc_weights) & 15)) return SFFT_EINVAL;
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
  fill_net(net, &tn);
  const long long npairs = ((batch + kRows - 1) / kRows + 1) / 2;
  const int grid = (int)std::max(1LL, std::min(npairs, (long long)sms));
  k_mlp_fwd_tc<<<grid, kThreadsTc, kSmemBytes, s>>>(tn, reinterpret_cast<const unsigned char*>(net->tc_weights),
                                                   x, batch, y, ws);
  return cudaGetLastError() == cudaSuccess ? SFFT_OK : SFFT_ECUDA;
}

int sfft_mlp_tc_timeouts_read() {
  int v = 0;
  if (cudaMemcpyFromSymbol(&v, g_mlp_tc_timeouts, sizeof(int)) != cudaSuccess) return -1;
  return v;
}
