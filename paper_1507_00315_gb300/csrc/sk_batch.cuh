// sk_batch.cuh -- work-item function of the persistent batched sweep.
//
// The batch kernel (sk_batch.cu) serves many exact-count jobs of different
// (variant, n) in one launch.  Jobs are laid end to end in a space of
// 32-item chunks, largest job first; every warp takes the next chunk from a
// device counter, finds its job, and calls the compiled walk of that job's
// (delta, n) -- one non-inlined device function per instance, defined in the
// per-n translation units and linked at device-link time.
#pragma once
#include "sk_exact_launch.cuh"

namespace sk {

// One job of a batch as the device sees it.
struct BatchJobDev {
  unsigned long long pres;       // position mask
  unsigned long long items;      // work items of the job
  unsigned long long chunk_lo;   // first global chunk of the job
  unsigned long long chunks;     // chunks of the job (ceil(items / 32))
  int m;                         // walk bits per item
  int code;                      // delta * 32 + n
  int pad[2];
};

// Residues of one item of a job (zero for an item past the job's end); the
// walk itself is the exact-form item function of the single-job kernel.
template <int DELTA, int N>
__device__ __forceinline__ Res4 batch_item_impl(const BatchJobDev* job, const Primes* P,
                                                int nprimes, unsigned long long item,
                                                signed char* ws_col) {
  if (item < job->items) return limb_item<DELTA, N>(job->pres, job->m, item, P, nprimes, ws_col);
  Res4 out = {{0, 0, 0, 0}};
  return out;
}

}  // namespace sk

#define SK_BATCH_FN(D, N) sk_batch_item_d##D##_n##N
#define SK_DECLARE_BATCH(N)                                                                  \
  extern __device__ sk::Res4 SK_BATCH_FN(0, N)(const sk::BatchJobDev*, const sk::Primes*, int, \
                                               unsigned long long, signed char*);             \
  extern __device__ sk::Res4 SK_BATCH_FN(1, N)(const sk::BatchJobDev*, const sk::Primes*, int, \
                                               unsigned long long, signed char*);
#define SK_DEFINE_BATCH(N)                                                                   \
  __device__ __noinline__ sk::Res4 SK_BATCH_FN(0, N)(const sk::BatchJobDev* j,               \
                                                     const sk::Primes* P, int np,            \
                                                     unsigned long long it, signed char* ws) { \
    return sk::batch_item_impl<0, N>(j, P, np, it, ws);                                      \
  }                                                                                          \
  __device__ __noinline__ sk::Res4 SK_BATCH_FN(1, N)(const sk::BatchJobDev* j,               \
                                                     const sk::Primes* P, int np,            \
                                                     unsigned long long it, signed char* ws) { \
    return sk::batch_item_impl<1, N>(j, P, np, it, ws);                                      \
  }
