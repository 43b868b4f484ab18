// TT rounding without any device allocation.
//
// Some callers cannot allocate device memory at the moment they need to round a
// tensor train: an application whose memory manager owns the whole device and
// hands out nothing at run time, a latency-critical loop in which the implicit
// device synchronisation of cudaMalloc/cudaFree is not acceptable, or a plugin
// that must not create or hold a library context. For them this file provides
// sfft_tt_round_noalloc: the same rounding kernel as sfft_tt_round, with all of
// its scratch (working copy of the cores, per-site panels, ranks, parameters
// and status) in one statically sized __device__ array below. The array is part
// of the library image, so every GPU that loads the library holds it until the
// process exits.
//
// Host code cannot use the array's name as a device address (it names a host
// stand-in), so the device address is looked up once per device with
// cudaGetSymbolAddress, with that device current, on the first call made on it.
#include <mutex>

#include <stdio.h>

#include "../../include/sfft.h"
#include "kernels.cuh"

namespace {

const int kThreadsNa = 256;

// layout of the static scratch (byte offsets, each 256-byte aligned)
constexpr size_t kSlotElems = SFFT_CORE_STRIDE_D4;  // one core slot, any d <= 4
constexpr size_t kTTBytes = sizeof(cd) * kSlotElems * SFFT_NOALLOC_MAX_N;
constexpr size_t kTmpBytes = sizeof(cd) * SFFT_ROUND_SCRATCH;
constexpr size_t kRankOff = kTTBytes + kTmpBytes;
constexpr size_t kParamOff = kRankOff + 256;
constexpr size_t kScratchBytes = kParamOff + 256;
static_assert(sizeof(int) * (SFFT_MAXN_DEV + 1) <= 256, "rank block");

struct NaParams {
  int n;
  int maxrank;
  double tol;
  long long off;
  int status;
  int pad;
};
static_assert(sizeof(NaParams) <= 256, "param block");

}  // namespace

// The scratch itself: SFFT_NOALLOC_SCRATCH_BYTES bytes per device.
static __device__ __align__(256) unsigned char g_round_scratch[kScratchBytes];
static_assert(kScratchBytes == SFFT_NOALLOC_SCRATCH_BYTES, "header limit");

namespace {

std::mutex g_mu;
void* g_dev_ptr[256];  // device address of g_round_scratch, per device id
bool g_attr_set[256];

void say(char* errbuf, int32_t errlen, const char* msg) {
  if (errbuf && errlen > 0) snprintf(errbuf, (size_t)errlen, "%s", msg);
}

// Once per device, with that device current: resolve the array's device
// address and allow the kernel its dynamic shared memory.
sfft_status scratch_on_current_device(unsigned char** out, char* errbuf, int32_t errlen) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) {
    say(errbuf, errlen, "no current CUDA device");
    return SFFT_ECUDA;
  }
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_dev_ptr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_round_scratch);
    if (e != cudaSuccess || !p) {
      say(errbuf, errlen, "cudaGetSymbolAddress of the static scratch failed");
      return SFFT_ECUDA;
    }
    g_dev_ptr[dev] = p;
  }
  if (!g_attr_set[dev]) {
    const int smem = (int)round_smem(4).bytes;
    if (cudaFuncSetAttribute(k_tt_round, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) !=
        cudaSuccess) {
      say(errbuf, errlen, "cudaFuncSetAttribute failed");
      return SFFT_ECUDA;
    }
    g_attr_set[dev] = true;
  }
  *out = reinterpret_cast<unsigned char*>(g_dev_ptr[dev]);
  return SFFT_OK;
}

}  // namespace

#define NA_CK(call, what)                                  \
  do {                                                     \
    if ((call) != cudaSuccess) {                           \
      say(errbuf, errlen, what);                           \
      return SFFT_ECUDA;                                   \
    }                                                      \
  } while (0)

extern "C" sfft_status sfft_tt_round_noalloc(int32_t n, int32_t d, const int32_t* in_ranks,
                                             const double* in_cores, double tol,
                                             int32_t max_rank, int32_t* out_ranks,
                                             double* out_cores, int64_t cap, void* stream,
                                             char* errbuf, int32_t errlen) {
  if (n < 1 || n > SFFT_NOALLOC_MAX_N) {
    char m[160];
    snprintf(m, sizeof m, "n = %d is outside [1, %d], the size the static scratch holds", n,
             SFFT_NOALLOC_MAX_N);
    say(errbuf, errlen, m);
    return SFFT_EINVAL;
  }
  if ((d != 2 && d != 4) || !in_ranks || !in_cores || !out_ranks || !out_cores ||
      !(tol > 0.0 && tol < 1.0) || max_rank < 0 || max_rank > SFFT_MAX_RANK) {
    say(errbuf, errlen, "invalid argument (d must be 2 or 4, pointers non-NULL, 0 < tol < 1)");
    return SFFT_EINVAL;
  }
  if (in_ranks[0] != 1 || in_ranks[n] != 1) {
    say(errbuf, errlen, "boundary ranks must be 1");
    return SFFT_EINVAL;
  }
  for (int s = 0; s <= n; ++s)
    if (in_ranks[s] < 1 || in_ranks[s] > SFFT_MAX_RANK) {
      char m[160];
      snprintf(m, sizeof m, "rank %d at bond %d is outside [1, %d], the size the static scratch holds",
               in_ranks[s], s, SFFT_MAX_RANK);
      say(errbuf, errlen, m);
      return SFFT_EINVAL;
    }
  unsigned char* base = nullptr;
  sfft_status st = scratch_on_current_device(&base, errbuf, errlen);
  if (st != SFFT_OK) return st;
  cudaStream_t sm = reinterpret_cast<cudaStream_t>(stream);
  cd* tt = reinterpret_cast<cd*>(base);
  cd* tmp = reinterpret_cast<cd*>(base + kTTBytes);
  int* ranks = reinterpret_cast<int*>(base + kRankOff);
  NaParams* prm = reinterpret_cast<NaParams*>(base + kParamOff);
  const int stride = (int)kSlotElems;
  // packed input cores -> core slots
  long long o = 0;
  for (int s = 0; s < n; ++s) {
    const long long sz = (long long)in_ranks[s] * d * in_ranks[s + 1];
    NA_CK(cudaMemcpyAsync(tt + (size_t)s * stride, reinterpret_cast<const cd*>(in_cores) + o,
                          sizeof(cd) * sz, cudaMemcpyDeviceToDevice, sm),
          "copy of the input cores failed");
    o += sz;
  }
  // parameters; the status word must start at zero
  int rk[SFFT_MAXN_DEV + 1];
  for (int s = 0; s <= SFFT_MAXN_DEV; ++s) rk[s] = (s <= n) ? in_ranks[s] : 1;
  NaParams hp = {n, max_rank ? max_rank : SFFT_DEFAULT_MAX_RANK, tol, 0, 0, 0};
  NA_CK(cudaMemcpyAsync(ranks, rk, sizeof rk, cudaMemcpyHostToDevice, sm), "rank upload failed");
  NA_CK(cudaMemcpyAsync(prm, &hp, sizeof hp, cudaMemcpyHostToDevice, sm), "parameter upload failed");
  const RoundSmem rsm = round_smem(d);
  k_tt_round<<<1, kThreadsNa, rsm.bytes, sm>>>(nullptr, 1, nullptr, &prm->n, d, 1, &prm->tol,
                                              &prm->maxrank, tt, &prm->off, stride, ranks, tmp,
                                              SFFT_ROUND_SCRATCH, &prm->status, rsm.hb, nullptr, PH_ROUND,
                                              rsm.pmax, rsm.vcap, nullptr, nullptr);
  NA_CK(cudaGetLastError(), "launch of the rounding kernel failed");
  NaParams back;
  NA_CK(cudaMemcpyAsync(rk, ranks, sizeof rk, cudaMemcpyDeviceToHost, sm), "rank download failed");
  NA_CK(cudaMemcpyAsync(&back, prm, sizeof back, cudaMemcpyDeviceToHost, sm), "status download failed");
  NA_CK(cudaStreamSynchronize(sm), "rounding kernel failed");
  if (back.status != 0) {
    say(errbuf, errlen, sfft_status_string((sfft_status)back.status));
    return (sfft_status)back.status;
  }
  long long need = 0;
  for (int s = 0; s < n; ++s) need += (long long)rk[s] * d * rk[s + 1];
  if (need > cap) {
    // out_ranks is left as the caller passed it
    char m[160];
    snprintf(m, sizeof m, "output capacity %lld complex is below the %lld the rounded cores need",
             (long long)cap, need);
    say(errbuf, errlen, m);
    return SFFT_EINVAL;
  }
  for (int s = 0; s <= n; ++s) out_ranks[s] = rk[s];
  o = 0;
  for (int s = 0; s < n; ++s) {
    const long long sz = (long long)rk[s] * d * rk[s + 1];
    NA_CK(cudaMemcpyAsync(reinterpret_cast<cd*>(out_cores) + o, tt + (size_t)s * stride,
                          sizeof(cd) * sz, cudaMemcpyDeviceToDevice, sm),
          "copy of the output cores failed");
    o += sz;
  }
  NA_CK(cudaStreamSynchronize(sm), "output copy failed");
  say(errbuf, errlen, "ok");
  return SFFT_OK;
}
