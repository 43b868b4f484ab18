// Kernel declarations and device-side limits shared by the SFFT kernels and
// the host runtime.
#pragma once
#include "cplx.cuh"
#include "la.cuh"
#include "model.cuh"

#define SFFT_MAXN_DEV 48
#define SFFT_SLOT_RANK_DEV 32                 // rank capacity of a core slot
#define SFFT_CORE_STRIDE_D2 (SFFT_SLOT_RANK_DEV * 2 * SFFT_SLOT_RANK_DEV)
#define SFFT_CORE_STRIDE_D4 (SFFT_SLOT_RANK_DEV * 4 * SFFT_SLOT_RANK_DEV)
// zip-up scratch: carry (q x k), D (r' s 2 r) and the panel Z (s r x 2 r')
#define SFFT_ZIP_CH_DEV (SFFT_SLOT_RANK_DEV * SFFT_SLOT_RANK_DEV * SFFT_SLOT_RANK_DEV)
#define SFFT_ZIP_D_DEV (2 * SFFT_SLOT_RANK_DEV * SFFT_SLOT_RANK_DEV * SFFT_SLOT_RANK_DEV)
#define SFFT_ZIP_Z_DEV (2 * SFFT_SLOT_RANK_DEV * SFFT_SLOT_RANK_DEV * SFFT_SLOT_RANK_DEV)
// real planes of the 3-multiplication products (doubles): carry re+im, D
// re+im, integrand core re-im, MPO core re-im; counted here in complex units
#define SFFT_ZIP_SUM_AW (6 * SFFT_SLOT_RANK_DEV * SFFT_SLOT_RANK_DEV)
#define SFFT_ZIP_SUMS_DEV ((SFFT_ZIP_CH_DEV + SFFT_ZIP_D_DEV + SFFT_ZIP_SUM_AW) / 2)
#define SFFT_ZIP_SCRATCH (SFFT_ZIP_CH_DEV + SFFT_ZIP_D_DEV + SFFT_ZIP_Z_DEV + SFFT_ZIP_SUMS_DEV)
#define SFFT_ROUND_SCRATCH (5 * SFFT_CORE_STRIDE_D4)
// zip-up of the delta prefix, one block per cached MPO: the output cores of
// sites 0..n-1 (stride SFFT_CORE_STRIDE_D2), then the carry after each site
// (stride SFFT_ZIP_CARRY_STRIDE: MPO rank x carried rank, both <= the slot rank)
#define SFFT_ZIP_CARRY_STRIDE (SFFT_SLOT_RANK_DEV * SFFT_SLOT_RANK_DEV)
#define SFFT_ZPRE_CARRY_BASE ((long long)SFFT_MAXN_DEV * SFFT_CORE_STRIDE_D2)
#define SFFT_ZPRE_BLOCK (SFFT_ZPRE_CARRY_BASE + (long long)SFFT_MAXN_DEV * SFFT_ZIP_CARRY_STRIDE)
#define READOUT_TREE_BITS 5                   // low bits expanded as a tree in the readout
#define SFFT_READOUT_SCRATCH (2 * 2112 * SFFT_SLOT_RANK_DEV)
#define SFFT_MPO_NODES 24                     // Chebyshev nodes of the MPO construction

// profiling phases (index into the flop / evaluation accumulators)
enum { PH_PROBE = 0, PH_BUILD = 1, PH_ZIPUP = 2, PH_ROUND = 3, PH_READOUT = 4, PH_MPO = 5,
       PH_DENSE_SAMPLE = 6, PH_DENSE_FFT = 7, PH_DENSE_GATHER = 8, PH_CROSS = 9 };
#define SFFT_NPHASE_DEV 10

// status codes (same values as sfft_status)
#define SFFT_EINVAL_DEV 1
#define SFFT_ERANK_DEV 5
#define SFFT_ENOCONV_DEV 6
#define SFFT_ETIMEOUT_DEV 7
#define SFFT_EBOUNDS_DEV 8

__global__ void k_sample(const InstParams* P, const long long* j, long long count, cd* x);
__global__ void k_support_probe(const InstParams* P, int count, double probe_tol, int m_min,
                                int* m_out);
// instances by decreasing sum_s r_s^2 of their TT ranks (work order)
__global__ void k_cost_order(const int* ranks_all, const int* n_arr, int count, int* order);
__global__ void k_build_lists(const int* m_arr, const int* n_arr, int count, int svd_max_bits,
                              int* svd_list, int* cross_list, int* counts);
__global__ void k_integrand_ttsvd(const InstParams* P, const int* m_arr, const int* list, int count,
                                  int* counter, cd* scratch,
                                  long long scratch_stride, cd* tt, const long long* tt_off,
                                  int core_stride, int* ranks_all, int* status, int hb, double* acc,
                                  int pmax, int* defer, const int* dcount, int* zpre_t);
__global__ void k_integrand_cross(const InstParams* P, const int* list, int count, int* counter,
                                  cd* scratch, long long scratch_stride, cd* tt,
                                  const long long* tt_off, int core_stride, int* ranks_all,
                                  int* status, int hb, double* acc, int max_sweeps, int pmax,
                                  int rcap, int* defer, const int* dcount, const int* m_arr,
                                  int* zpre_t);
__global__ void k_mpo_interp(int n, int P, cd* W, int core_stride, int* ranks);
__global__ void k_tt_round(const int* list, int count, int* counter, const int* n_arr, int d,
                           int left_orth, const double* tol_arr,
                           const int* maxrank_arr, cd* tt, const long long* tt_off,
                           int core_stride, int* ranks_all, cd* scratch,
                           long long scratch_stride, int* status, int hb, double* acc, int phase,
                           int pmax, int vcap, int* defer, const int* dcount,
                           const int* site0_arr = nullptr);

// Shared memory of k_tt_round for physical dimension d: panels of at most
// SFFT_SLOT_RANK_DEV columns; W holds a (d r) x r block, V the explicit Q.
struct RoundSmem {
  int pmax, hb, vcap;
  size_t bytes;
};
// Shared memory of k_zipup: 8-row panel blocks at 64 columns and a
// 64 x (rank cap + 1) basis block, small enough for two CTAs per SM.
// small: W only, wrows x 64 elements (hb = wrows - 64 may be negative; the
// explicit Q is formed in T's spent columns, else in global scratch). At
// wrows = 32 (32 KB) six 128-thread CTAs share an SM (with the kernel's
// 85-register bound); the tensor-core variant stages its operand tiles in W
// and takes wrows = 70 at 256 threads, three per SM.
inline RoundSmem zip_smem(bool small = false, int wrows = 70) {
  RoundSmem r;
  r.pmax = LA_MAXP;
  r.hb = small ? wrows - LA_MAXP : 8;
  r.vcap = small ? 1 : LA_MAXP * (SFFT_SLOT_RANK_DEV + 1);
  r.bytes = sizeof(cd) * ((size_t)(r.pmax + r.hb) * r.pmax + r.vcap + r.pmax) + sizeof(double) * r.pmax + 320;
  return r;
}
// Shared memory of k_tt_round. The left-orthogonalisation pass writes an
// explicit Q of d r x r into V; without it (left_orth = 0) V holds only the
// r x r right singular vectors, and the smaller carve lets 4 CTAs share an SM
// for d = 2. A launch with left_orth = 1 must use the full carve.
inline RoundSmem round_smem(int d, bool left_orth = true, int pmax = SFFT_SLOT_RANK_DEV) {
  RoundSmem r;
  r.pmax = pmax;
  r.hb = (d - 1) * pmax;  // W = (pmax + hb) pmax >= d r x r
  r.vcap = (left_orth ? d : 1) * pmax * pmax;
  r.bytes = sizeof(cd) * ((size_t)(r.pmax + r.hb) * r.pmax + r.vcap + r.pmax) + sizeof(double) * r.pmax + 320;
  return r;
}
// The zip-up over sites whose integrand cores are the rank-one delta_{lam,0}
// (the sites above a TT-SVD block) depends on the MPO alone. It is run once
// per cached MPO on an all-delta TT (carry_out set: the carry after every
// site is kept) and then copied into each instance's zip-up, which starts at
// the first site of its block. All pointers may be null (no prefix).
struct ZipPrefix {
  const int* t;           // per instance: sites taken from the prefix (0: none)
  const long long* off;   // per instance: offset of its MPO's prefix block (< 0: none)
  const int* ranks;       // per instance, SFFT_MAXN_DEV + 1 each: the prefix's output ranks
  const cd* pool;         // prefix blocks (SFFT_ZPRE_BLOCK complex each)
  cd* carry_out;          // precompute: the pool, whose carries the launch writes
};
__global__ void k_zipup(const int* list, int count, int* counter, const int* n_arr,
                        const double* tol_arr, const int* maxrank_arr,
                        const cd* A, const long long* a_off, const int* a_ranks_all,
                        const cd* Wmpo, const long long* w_off, const int* w_ranks_all, cd* B,
                        const long long* b_off, int* b_ranks_all, int core_stride_a,
                        int core_stride_w, int core_stride_b, cd* scratch,
                        long long scratch_stride, int* status, int hb, double* acc, int vcap, int* defer,
                        const int* dcount, int qmax1, int wlim, ZipPrefix zp);
// The same with the MPO contraction of each site on the tensor cores (tcgen05,
// FP32 operands as three bfloat16 pieces, FP32 accumulation) wherever one
// 128-row tile holds it; the QR steps stay FP64.
__global__ void k_zipup_tc(const int* list, int count, int* counter, const int* n_arr,
                           const double* tol_arr, const int* maxrank_arr,
                           const cd* A, const long long* a_off, const int* a_ranks_all,
                           const cd* Wmpo, const long long* w_off, const int* w_ranks_all, cd* B,
                           const long long* b_off, int* b_ranks_all, int core_stride_a,
                           int core_stride_w, int core_stride_b, cd* scratch,
                           long long scratch_stride, int* status, int hb, double* acc, int vcap, int* defer,
                           const int* dcount, int qmax1, int wlim, ZipPrefix zp);
// Jacobi sweep limit of the SVDs in the TT kernels (test hook; default 60),
// enqueued on `stream`. The value is taken from pageable host memory before
// the call returns; not for use while the stream is being captured.
cudaError_t sfft_set_jacobi_cap(int sweeps, cudaStream_t stream);
__global__ void k_readout(const int* list, int count, int* counter, const InstParams* P,
                          const cd* B, const long long* b_off,
                          const int* b_ranks_all, int core_stride, const long long* l_begin,
                          const int* tbits, const int* qarr, const long long* out_off,
                          double* prices, double* logk, int* status, cd* scratch,
                          long long scratch_stride);

__global__ void k_dfma_peak(double* out, int iters);

// dense-FFT baseline
__global__ void k_dense_sample(InstParams prm, cd* x, long long M);
__global__ void k_fft_pass(cd* x, long long M, long long Lp, int R, int cols_per_block);
__global__ void k_dense_gather(InstParams prm, const cd* y, int n, const int* digits, int ndig,
                               long long l_begin, int tbits, int q, double* prices, double* logk);
// statevector emulation of the QFT route
__global__ void k_norm2_partial(const cd* x, long long M, double* part);
__global__ void k_norm2_final(const double* part, int nparts, double* nrm2);
__global__ void k_scale_unit(cd* x, long long M, const double* nrm2);
__global__ void k_qft_gather(InstParams prm, const cd* y, int n, const int* digits, int ndig,
                             long long l_begin, int tbits, int q, const double* nrm2,
                             double* prices, double* logk);
