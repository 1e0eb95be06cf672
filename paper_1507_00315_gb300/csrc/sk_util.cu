// sk_util.cu -- INT32 throughput microbenchmark, the denominator of the exact
// kernel's roofline (an integer-ALU-bound path: no tensor cores, ~no DRAM).
//
// Each thread runs 8 independent dependency chains for `iters` rounds.
// mode 0: every op is a 32-bit multiply-add (mad.lo.u32).
// mode 1: alternating multiply-adds and three-input adds / logic ops, the mix
//         the Gray-code kernel issues (multiplier pipe plus integer ALU).
#include <cuda_runtime.h>

#include <cstdint>

#include "sk_host_common.h"

namespace sk {

template <int MODE>
__global__ void __launch_bounds__(256) int_peak_kernel(unsigned iters, unsigned seed,
                                                       unsigned* sink) {
  unsigned a0 = seed ^ threadIdx.x, a1 = a0 + 1, a2 = a0 + 2, a3 = a0 + 3;
  unsigned a4 = a0 + 4, a5 = a0 + 5, a6 = a0 + 6, a7 = a0 + 7;
  const unsigned m = seed | 1u, c = seed >> 3;
  for (unsigned i = 0; i < iters; ++i) {
#pragma unroll
    for (int r = 0; r < 16; ++r) {
      if (MODE == 0) {
        asm volatile("mad.lo.u32 %0, %0, %8, %9;\n\tmad.lo.u32 %1, %1, %8, %9;\n\t"
                     "mad.lo.u32 %2, %2, %8, %9;\n\tmad.lo.u32 %3, %3, %8, %9;\n\t"
                     "mad.lo.u32 %4, %4, %8, %9;\n\tmad.lo.u32 %5, %5, %8, %9;\n\t"
                     "mad.lo.u32 %6, %6, %8, %9;\n\tmad.lo.u32 %7, %7, %8, %9;"
                     : "+r"(a0), "+r"(a1), "+r"(a2), "+r"(a3), "+r"(a4), "+r"(a5), "+r"(a6), "+r"(a7)
                     : "r"(m), "r"(c));
      } else {
        asm volatile("mad.lo.u32 %0, %0, %8, %9;\n\tlop3.b32 %1, %1, %8, %9, 0x96;\n\t"
                     "mad.lo.u32 %2, %2, %8, %9;\n\tlop3.b32 %3, %3, %8, %9, 0x96;\n\t"
                     "mad.lo.u32 %4, %4, %8, %9;\n\tlop3.b32 %5, %5, %8, %9, 0x96;\n\t"
                     "mad.lo.u32 %6, %6, %8, %9;\n\tlop3.b32 %7, %7, %8, %9, 0x96;"
                     : "+r"(a0), "+r"(a1), "+r"(a2), "+r"(a3), "+r"(a4), "+r"(a5), "+r"(a6), "+r"(a7)
                     : "r"(m), "r"(c));
      }
    }
  }
  unsigned v = a0 ^ a1 ^ a2 ^ a3 ^ a4 ^ a5 ^ a6 ^ a7;
  if (v == 0x12345678u) sink[0] = v;     // keeps the chains live
}

}  // namespace sk

// Measures INT32 operations per second on the current device.  mode 0:
// multiply-adds only; mode 1: multiply-add / logic mix.  ops_per_s (host):
// thread-level 32-bit operations per second; ms (host, may be NULL): the
// timed launch's duration.  Returns an SK status.
extern "C" int sk_int32_peak(int mode, double* ops_per_s, double* ms) {
  if (!ops_per_s || mode < 0 || mode > 1) return SK_EINVAL;
  int st = sk::check_device();
  if (st) return st;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  unsigned* sink = nullptr;
  if (cudaMalloc(&sink, 16) != cudaSuccess) return SK_ENOMEM;
  const int threads = 256, blocks = sms * 8;
  const unsigned iters = 4096;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  auto launch = [&](unsigned it) {
    if (mode == 0) sk::int_peak_kernel<0><<<blocks, threads>>>(it, 12345u, sink);
    else sk::int_peak_kernel<1><<<blocks, threads>>>(it, 12345u, sink);
  };
  launch(64);                                  // warm-up
  cudaEventRecord(e0);
  launch(iters);
  cudaEventRecord(e1);
  cudaError_t e = cudaEventSynchronize(e1);
  float t = 0.f;
  cudaEventElapsedTime(&t, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(sink);
  if (e != cudaSuccess) return sk::cuda_status(e);
  const double ops = (double)blocks * threads * iters * 16.0 * 8.0;
  *ops_per_s = ops / (t * 1e-3);
  if (ms) *ms = t;
  return SK_OK;
}
