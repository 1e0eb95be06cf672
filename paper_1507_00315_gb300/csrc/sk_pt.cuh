// sk_pt.cuh -- device side of the parallel-tempering approximate count
// (Sec. 3, Algorithm 2).
//
// State space: the simplified problem of Sec. 3 -- pair k sits at any start
// bin s in [0, 2n - d_k) of 2n bins, overlaps allowed; the energy is the
// number of empty bins.  One warp runs one ladder of M <= 32 temperatures;
// lane l keeps the configuration that started at rung l (its start slots and
// bin occupancies in shared memory, its energy in a register) and carries a
// temperature label r that exchanges swap: configurations never move between
// lanes, labels do (a lane-of-rung table, one entry per lane, follows them).
//
// Random numbers: Philox-4x32-10 (Salmon et al., SC'11), one call per
// (counter, key): counter (k, rung, ladder, 1) for the start slot of pair k,
// (t, rung, ladder, 2) for iteration t at that rung -- word 0: pair, word 1:
// slot, word 2: acceptance of the move of the configuration at the rung,
// word 3: acceptance of the exchange of rungs (rung, rung+1); key = the
// 64-bit seed.  (One block per rung and iteration: the exchange needs no
// call of its own.)
// Acceptance compares a 32-bit word w with a threshold T = ceil(p 2^32)
// (T = 2^32: always), i.e. accept iff w / 2^32 < p.
#pragma once
#include <cstdint>

namespace sk {

constexpr int kPtMaxRungs = 32;
constexpr int kPtMaxN = 40;

struct PtParams {
  int n, delta, M, bins;          // bins = 2n
  int ladders;                    // L
  int warps_per_block;
  unsigned long long iters, burnin;
  unsigned key0, key1;
};

__device__ __forceinline__ uint4 philox4x32_10(uint4 c, unsigned k0, unsigned k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const unsigned hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
    const unsigned hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
    c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return c;
}

// Shared-memory layout of one warp: the energy histogram (M x (bins+1)
// 16-bit counters, flushed to global memory every kPtFlush iterations),
// accepted moves and exchanges (M u32 each), start slots ([k][lane] bytes)
// and bin occupancies ([b][lane] bytes).  The acceptance thresholds stay in
// global memory (L1-cached), so about 28 warps fit on an SM.
constexpr unsigned kPtFlush = 32768;
__host__ __device__ inline size_t pt_warp_bytes(int M, int n) {
  const size_t hist = ((size_t)M * (2 * n + 1) * 2 + 15) / 16 * 16 + 2 * (size_t)M * 4;
  const size_t st = (size_t)(n + 1) * 32 + (size_t)(2 * n) * 32;
  return (hist + st + 15) / 16 * 16;
}
__host__ __device__ inline size_t pt_smem_bytes(int M, int n, int wpb) {
  return (size_t)wpb * pt_warp_bytes(M, n);
}

// Host helpers shared by the plain and the learned chains (sk_pt.cu).
unsigned long long accept_threshold(double x);
int pt_learned_run(int variant, int n, int M, const double* beta, int L, uint64_t iters,
                   uint64_t burnin, uint64_t seed, const void* model, uint64_t* hist,
                   uint64_t* accm, uint64_t* accs, void* stream, double* kernel_ms);
double pt_estimate_from_hist(int variant, int n, int M, const double* beta, const uint64_t* hist,
                             double* ratios);

}  // namespace sk
