// sk_exact_launch.cuh -- the single-job Gray-code kernels and their launchers.
//
// One persistent grid (a multiple of the SM count) pulls work items from a
// device counter, one warp-sized chunk (32 items, one per lane) at a time, so
// the 32 lanes of a warp always walk the same Gray schedule on different
// prefixes.  Each thread keeps its residues, the warp combines them with
// shuffles, and one lane per warp adds them into the job's slots with a
// compare-and-swap modular add (order independent, so the result is
// bit-exact whatever the schedule).
//
// Two arithmetic forms of the term product (same residues):
//   limb_kernel<delta, n>       -- exact signed-digit products and sums,
//                                  reduced modulo the primes once per item;
//   mont_kernel<delta, n, NPR>  -- per-term signed Montgomery products modulo
//                                  each 62-bit prime.
#pragma once
#include <cuda_runtime.h>

#include <atomic>

#include "sk_exact.cuh"

namespace sk {

// Host-side caches of launch shapes are kept per device (a process may drive
// several GPUs, each current in its own host threads) and read and written
// atomically; concurrent first calls compute and store the same value.
constexpr int kMaxDevices = 64;

// Resident CTAs per SM of one kernel, per device and block size (multiples of
// 32 up to 256).
struct OccupancyCache {
  std::atomic<int> per_sm[kMaxDevices][9];
};

// SM count of device `dev` (looked up once per device).
inline int device_sm_count(int dev) {
  static std::atomic<int> cache[kMaxDevices];
  const bool keyed = dev >= 0 && dev < kMaxDevices;
  int v = keyed ? cache[dev].load(std::memory_order_relaxed) : 0;
  if (v <= 0) {
    v = 0;
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    if (v <= 0) return 1;
    if (keyed) cache[dev].store(v, std::memory_order_relaxed);
  }
  return v;
}

// Scratch words of one launch (device memory, zeroed before the launch).
struct ExactScratch {
  unsigned long long counter;            // next chunk of items
  unsigned long long res[kMaxPrimes];    // residues of the sum, raw
  unsigned int err;                      // nonzero: a bounded loop gave up
  unsigned int pad;
};

struct ExactLaunch {
  ExactJob job;
  Primes P;
  int nprimes;
  unsigned long long item_lo;            // first item of this launch
  unsigned long long item_hi;            // one past the last item
  ExactScratch* scratch;                 // device
  unsigned long long* item_res;          // optional: [item_hi-item_lo][nprimes]
  int block_threads;
  int grid;                              // 0: SMs x resident blocks
  cudaStream_t stream;
};

constexpr int kCasLimit = 1 << 22;

// Two resident 256-thread CTAs per SM: 128 registers per thread, which holds
// the n correlations, the window of outer values and the accumulators
// without spills.
#ifndef SK_EXACT_MIN_BLOCKS
#define SK_EXACT_MIN_BLOCKS 2
#endif

__device__ __forceinline__ void atomic_addmod(unsigned long long* addr, unsigned long long v,
                                              unsigned long long p, unsigned int* err) {
  if (v == 0) return;
  unsigned long long old = *((volatile unsigned long long*)addr);
  for (int it = 0; it < kCasLimit; ++it) {
    unsigned long long nv = addmod(old, v, p);
    unsigned long long seen = atomicCAS(addr, old, nv);
    if (seen == old) return;
    old = seen;
  }
  atomicOr(err, 1u);
}

__device__ __forceinline__ void warp_flush(unsigned long long (&tot)[kMaxPrimes], int nprimes,
                                           const Primes& P, unsigned long long* slots,
                                           unsigned int* err) {
#pragma unroll
  for (int i = 0; i < kMaxPrimes; ++i) {
    if (i >= nprimes) break;
    unsigned long long v = tot[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
      v = addmod(v, __shfl_xor_sync(0xffffffffu, v, o), (unsigned long long)P.pr[i].p);
    if ((threadIdx.x & 31) == 0) atomic_addmod(&slots[i], v, (unsigned long long)P.pr[i].p, err);
    tot[i] = 0;
  }
}

// One exact-form work item, compiled once per (delta, n) and called by both
// the single-job kernel and the batch kernel.
template <int DELTA, int N>
__device__ __noinline__ Res4 limb_item(unsigned long long pres, int m, unsigned long long item,
                                       const Primes* P, int nprimes, signed char* ws_col) {
  LimbAcc<DELTA, N> A(*P);
  unsigned long long r[kMaxPrimes];
  run_item<DELTA, N>(pres, m, item, ws_col, A, nprimes, r);
  Res4 out;
#pragma unroll
  for (int i = 0; i < kMaxPrimes; ++i) out.r[i] = r[i];
  return out;
}

template <int DELTA, int N>
struct LimbItem {
  __device__ __forceinline__ static Res4 eval(const ExactJob& job, const Primes& P, int nprimes,
                                              unsigned long long item, signed char* ws_col) {
    return limb_item<DELTA, N>(job.pres, job.m, item, &P, nprimes, ws_col);
  }
};

template <int DELTA, int N, int NPR>
struct MontItem {
  __device__ __forceinline__ static Res4 eval(const ExactJob& job, const Primes& P, int nprimes,
                                              unsigned long long item, signed char* ws_col) {
    MontAcc<DELTA, N, NPR> A(P);
    unsigned long long r[kMaxPrimes];
    run_item<DELTA, N>(job.pres, job.m, item, ws_col, A, nprimes, r);
    Res4 out;
#pragma unroll
    for (int i = 0; i < kMaxPrimes; ++i) out.r[i] = r[i];
    return out;
  }
};

// The persistent work loop shared by both arithmetic forms.
template <class Item>
__device__ __forceinline__ void work_loop(const ExactJob& job, const Primes& P, int nprimes,
                                          unsigned long long item_lo, unsigned long long item_hi,
                                          ExactScratch* scr, unsigned long long* item_res) {
  extern __shared__ signed char sk_ws[];
  const unsigned long long count = item_hi - item_lo;
  const int lane = threadIdx.x & 31;
  signed char* ws_col = sk_ws + threadIdx.x;
  unsigned long long tot[kMaxPrimes] = {0, 0, 0, 0};
  for (;;) {
    unsigned long long base = 0;
    if (lane == 0) base = atomicAdd(&scr->counter, 32ULL);
    base = __shfl_sync(0xffffffffu, base, 0);
    if (base >= count) break;
    const unsigned long long it = base + lane;
    if (it < count) {
      const unsigned long long q =
          job.fixed_bit ? insert_zero_bit(item_lo + it, job.fixed_bit - job.m) : item_lo + it;
      const Res4 r = Item::eval(job, P, nprimes, q, ws_col);
#pragma unroll
      for (int i = 0; i < kMaxPrimes; ++i) {
        if (i >= nprimes) break;
        tot[i] = addmod(tot[i], r.r[i], (unsigned long long)P.pr[i].p);
        if (item_res) item_res[it * nprimes + i] = r.r[i];
      }
    }
  }
  warp_flush(tot, nprimes, P, scr->res, &scr->err);
}

template <int DELTA, int N>
__global__ void __launch_bounds__(256, SK_EXACT_MIN_BLOCKS)
    limb_kernel(ExactJob job, Primes P, int nprimes, unsigned long long item_lo,
                unsigned long long item_hi, ExactScratch* scr, unsigned long long* item_res) {
  work_loop<LimbItem<DELTA, N>>(job, P, nprimes, item_lo, item_hi, scr, item_res);
}

template <int DELTA, int N, int NPR>
__global__ void __launch_bounds__(256, SK_EXACT_MIN_BLOCKS)
    mont_kernel(ExactJob job, Primes P, unsigned long long item_lo, unsigned long long item_hi,
                ExactScratch* scr, unsigned long long* item_res) {
  work_loop<MontItem<DELTA, N, NPR>>(job, P, NPR, item_lo, item_hi, scr, item_res);
}

// Grid: SMs x resident CTAs per SM of the current device, never more warps
// than 32-item chunks.
template <class K>
cudaError_t exact_grid(K kernel, const ExactLaunch& L, size_t smem, OccupancyCache& occ,
                       int* grid_out) {
  const int bt = L.block_threads;
  if (bt < 32 || bt > 256 || (bt & 31)) return cudaErrorInvalidValue;
  int grid = L.grid;
  if (grid <= 0) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const bool keyed = dev >= 0 && dev < kMaxDevices;
    int nb = keyed ? occ.per_sm[dev][bt / 32].load(std::memory_order_relaxed) : 0;
    if (nb <= 0) {
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kernel, bt, smem);
      if (e != cudaSuccess) return e;
      if (nb <= 0) nb = 1;
      if (keyed) occ.per_sm[dev][bt / 32].store(nb, std::memory_order_relaxed);
    }
    grid = device_sm_count(dev) * nb;
    unsigned long long chunks = (L.item_hi - L.item_lo + 31) / 32;
    unsigned long long warps_per_block = (unsigned long long)bt / 32;
    unsigned long long need = (chunks + warps_per_block - 1) / warps_per_block;
    if ((unsigned long long)grid > need) grid = (int)(need ? need : 1);
  }
  *grid_out = grid;
  return cudaSuccess;
}

template <int DELTA, int N, int NPR>
cudaError_t launch_exact(const ExactLaunch& L) {
  static OccupancyCache bps;
  if (L.nprimes != NPR) return cudaErrorInvalidValue;
  const size_t smem = (size_t)ws_len(DELTA, N) * kWsStride;
  int grid = 0;
  cudaError_t e = exact_grid(mont_kernel<DELTA, N, NPR>, L, smem, bps, &grid);
  if (e != cudaSuccess) return e;
  mont_kernel<DELTA, N, NPR><<<grid, L.block_threads, smem, L.stream>>>(
      L.job, L.P, L.item_lo, L.item_hi, L.scratch, L.item_res);
  return cudaGetLastError();
}

template <int DELTA, int N>
cudaError_t launch_limb(const ExactLaunch& L) {
  static OccupancyCache bps;
  if (L.nprimes < 1 || L.nprimes > kMaxPrimes) return cudaErrorInvalidValue;
  const size_t smem = (size_t)ws_len(DELTA, N) * kWsStride;
  int grid = 0;
  cudaError_t e = exact_grid(limb_kernel<DELTA, N>, L, smem, bps, &grid);
  if (e != cudaSuccess) return e;
  limb_kernel<DELTA, N><<<grid, L.block_threads, smem, L.stream>>>(
      L.job, L.P, L.nprimes, L.item_lo, L.item_hi, L.scratch, L.item_res);
  return cudaGetLastError();
}

typedef cudaError_t (*ExactLaunchFn)(const ExactLaunch&);

// Montgomery-form launchers for delta in {0, 1}, n in [1, kMaxN], three
// primes (null for combinations that were not compiled; four moduli go
// through the exact form).
ExactLaunchFn exact_launcher(int delta, int n, int nprimes);
// Exact-limb launchers for delta in {0, 1}, n in [1, kMaxN].
ExactLaunchFn limb_launcher(int delta, int n);

}  // namespace sk

#define SK_INSTANTIATE_EXACT(N)                                                \
  template cudaError_t sk::launch_exact<0, N, 3>(const sk::ExactLaunch&);      \
  template cudaError_t sk::launch_exact<1, N, 3>(const sk::ExactLaunch&);      \
  template cudaError_t sk::launch_limb<0, N>(const sk::ExactLaunch&);          \
  template cudaError_t sk::launch_limb<1, N>(const sk::ExactLaunch&);
