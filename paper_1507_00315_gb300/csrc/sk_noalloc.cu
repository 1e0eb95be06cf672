// sk_noalloc.cu -- an allocation-free variant of skolem_item_residues.
//
// Some callers cannot let a library call cudaMalloc or cudaFree: a
// framework whose caching allocator owns the device memory budget (a stray
// cudaMalloc can fail or fragment it under memory pressure), and
// latency-sensitive host loops that cannot absorb the device-wide
// synchronisation cudaFree implies.  This entry point runs the same
// Gray-code kernel as skolem_item_residues (exact form), but its device
// scratch -- the
// launch record (work counter, residue slots, error word) and the per-item
// staging of the residues before they are copied to the caller's host
// buffer -- lives in one file-scope __device__ array of fixed size, which
// every GPU that loads the library holds until the process exits.  It creates
// no stream and no event and calls no allocating CUDA or library routine.
//
// In host code the array's name is only a host-side stand-in for the device
// symbol, so the device address is fetched once per device with
// cudaGetSymbolAddress (with that device current) and cached.  The first call
// on a device performs this set-up; make that first call before any stream
// capture.  All calls share the array and it keeps the last call's contents:
// the launch record is cleared at the start of every call, and calls whose
// work overlaps on the GPU (different streams, or different host threads)
// race on it.
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>

#include "sk_exact_launch.cuh"
#include "sk_host_common.h"

namespace sk {

unsigned long long position_mask(int variant, int n);   // sk_host_exact.cu
int limb_max_m(int delta, int n);                       // sk_host_exact.cu

namespace {

constexpr int kHeaderWords = 32;   // 256 bytes: one ExactScratch, padded
constexpr unsigned long long kNoAllocWords =
    kHeaderWords + (unsigned long long)SK_NOALLOC_MAX_ITEMS * SK_MAX_PRIMES;
static_assert(sizeof(ExactScratch) <= kHeaderWords * 8, "launch record must fit the header");

static __device__ __align__(256) unsigned long long sk_noalloc_scratch[kNoAllocWords];

std::mutex g_setup_mu;
unsigned long long* g_scratch_ptr[kMaxDevices] = {nullptr};

// Device address of the scratch array on the current device (set-up once per
// device).  Returns an SK status.
int scratch_address(unsigned long long** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return SK_ECUDA;
  std::lock_guard<std::mutex> lock(g_setup_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, sk_noalloc_scratch);
    if (e != cudaSuccess || !p) return SK_ECUDA;
    g_scratch_ptr[dev] = (unsigned long long*)p;
  }
  *out = g_scratch_ptr[dev];
  return SK_OK;
}

}  // namespace
}  // namespace sk

extern "C" int skolem_item_residues_noalloc(int variant, int n, int m, uint64_t q_lo,
                                            uint64_t count, int nprimes, const uint64_t* primes,
                                            void* stream, uint64_t* out) {
  using namespace sk;
  if (!out || !primes || count == 0) return SK_EINVAL;
  if (count > (uint64_t)SK_NOALLOC_MAX_ITEMS) return SK_EINVAL;   // beyond the static scratch
  if (variant < SK_SKOLEM || variant > SK_HOOKED || n < 1 || n > kMaxN) return SK_EINVAL;
  sk_count_opts o;
  std::memset(&o, 0, sizeof(o));
  o.nprimes = nprimes;
  for (int i = 0; i < nprimes && i < SK_MAX_PRIMES; ++i) o.primes[i] = primes[i];
  int k = 0;
  uint64_t pv[kMaxPrimes];
  Primes P;
  int st = prepare_primes(&o, &k, pv, &P);
  if (st) return st;
  const int F = 2 * n - 1, U = inner_bits(n), delta = variant == SK_LANGFORD ? 1 : 0;
  if (m < U || m > F || m > limb_max_m(delta, n) || F - m > 40) return SK_EINVAL;
  const unsigned long long items = 1ULL << (F - m);
  if (q_lo >= items || count > items - q_lo) return SK_EINVAL;
  ExactLaunchFn fn = limb_launcher(delta, n);
  if (!fn) return SK_EINVAL;
  st = check_device();
  if (st) return st;
  unsigned long long* base = nullptr;
  st = scratch_address(&base);
  if (st) return st;

  cudaStream_t s = (cudaStream_t)stream;
  ExactScratch* rec = (ExactScratch*)base;
  unsigned long long* item_res = base + kHeaderWords;
  cudaError_t e = cudaMemsetAsync(rec, 0, sizeof(ExactScratch), s);
  if (e != cudaSuccess) return cuda_status(e);
  ExactLaunch L;
  L.job.pres = position_mask(variant, n);
  L.job.items = items;
  L.job.m = m;
  L.job.job = 0;
  L.job.fixed_bit = 0;
  L.P = P;
  L.nprimes = k;
  L.item_lo = q_lo;
  L.item_hi = q_lo + count;
  L.scratch = rec;
  L.item_res = item_res;
  L.block_threads = 256;
  L.grid = 0;
  L.stream = s;
  e = fn(L);
  if (e != cudaSuccess) return cuda_status(e);
  ExactScratch h;
  e = cudaMemcpyAsync(&h, rec, sizeof(h), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(out, item_res, count * k * sizeof(uint64_t), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_status(e);
  if (h.err) return SK_ETIMEOUT;
  return SK_OK;
}
