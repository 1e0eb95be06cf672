// sk_pt.cuh -- device side of the parallel-tempering approximate count
// (Sec. 3, Algorithm 2).
//
// State space: the simplified problem of Sec. 3 -- pair k sits at any start
// bin s in [0, 2n - d_k) of 2n bins, overlaps allowed; the energy is the
// number of empty bins.  W warps run one ladder of M <= 32 W temperatures
// (W = 1 up to 32 rungs, W = 2 up to 64).  Lane j of the ladder's warp h
// always serves rung 32 h + j; the configurations stay where they started
// (column l of the ladder's start-slot and bin-occupancy tables in shared
// memory belongs to the configuration that started at rung l) and an
// exchange of rungs j, j+1 swaps the column indices and energies that their
// lanes hold (a warp shuffle; between rungs 31 and 32, a shared-memory slot
// and a barrier of the two warps).  Per-rung quantities (thresholds,
// acceptance counters, the energy histogram column) therefore stay with one
// lane.
//
// Random numbers: Philox-4x32-10 (Salmon et al., SC'11), one call per
// (counter, key): counter (k, rung, ladder, 1) for the start slot of pair k,
// (t, rung, ladder, 2) for iteration t at that rung -- word 0: pair, word 1:
// slot, word 2: acceptance of the move of the configuration at the rung,
// word 3: acceptance of the exchange of rungs (rung, rung+1); key = the
// 64-bit seed.  (One block per rung and iteration: the exchange needs no
// call of its own.)
// Acceptance compares a 32-bit word w with a threshold T = ceil(p 2^32)
// (T = 2^32: always; T = 0 where e^-x underflows: never), i.e. accept iff
// w / 2^32 < p.
#pragma once
#include <cstdint>

namespace sk {

constexpr int kPtMaxRungs = 64;        // plain chains: two warps a ladder above 32
constexpr int kPtMaxRungsLearned = 32; // the learned chains' exchange kernel: one warp a ladder
constexpr int kPtMaxN = 64;      // plain chains (the paper's closing estimate is S(64))
constexpr int kMlpMaxN = 40;     // the learned proposal (its move table, input width 128)
constexpr int kPtErrorGroups = 16;   // ladder groups behind pt_estimate's standard error

struct PtParams {
  int n, delta, M, bins;          // bins = 2n
  int ladders;                    // L
  int warps_per_block;            // a multiple of the warps per ladder
  unsigned iters, burnin;
  unsigned key0, key1;
  unsigned rk[20];                // Philox round keys: (key0 + r W0, key1 + r W1), r = 0..9
  int groups;                     // energy histograms kept per group of ladders (>= 1)
};

// Ladder group of a ladder: `groups` equal runs of consecutive ladders.
__host__ __device__ inline int pt_group(int ladder, int ladders, int groups) {
  return (int)((long long)ladder * groups / ladders);
}

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

// Philox-4x32-10 with the ten round keys given (rk[2r], rk[2r+1] = the key
// after r bumps): the same function as philox4x32_10, the key schedule
// computed once on the host.
__device__ __forceinline__ uint4 philox4x32_10_rk(uint4 c, const unsigned* rk) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const unsigned hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
    const unsigned hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
    c = make_uint4(hi1 ^ c.y ^ rk[2 * r], lo1, hi0 ^ c.w ^ rk[2 * r + 1], lo0);
  }
  return c;
}

// Shared-memory layout of one ladder of W warps (32 W columns): the energy
// histogram ([E][rung] 16-bit counters, flushed to global memory every
// kPtFlush iterations), then the start slots ([k][column]), bin occupancies
// ([b][column]) and the round-trip marks ([column]), one byte an entry.  Thresholds stay in
// registers (moves) and global memory, L1-cached (exchanges).
constexpr unsigned kPtFlush = 32768;
__host__ __device__ inline size_t pt_hist_bytes(int n, int W) {
  return ((size_t)(2 * n + 1) * 32 * W * 2 + 15) / 16 * 16;
}
__host__ __device__ inline size_t pt_ladder_bytes(int n, int W) {
  const size_t st = (size_t)(n + 1) * 32 * W + (size_t)(2 * n) * 32 * W + (size_t)32 * W;
  return (pt_hist_bytes(n, W) + st + 15) / 16 * 16;
}
__host__ __device__ inline size_t pt_smem_bytes(int n, int W, int wpb) {
  return (size_t)(wpb / W) * pt_ladder_bytes(n, W);
}

// Host helpers shared by the plain and the learned chains (sk_pt.cu).
unsigned long long accept_threshold(double x);
int pt_learned_run(int variant, int n, int M, const double* beta, int L, uint64_t iters,
                   uint64_t burnin, uint64_t seed, const void* model, uint64_t* hist,
                   uint64_t* accm, uint64_t* accs, void* stream, double* kernel_ms);
double pt_estimate_from_hist(int variant, int n, int M, const double* beta, const uint64_t* hist,
                             double* ratios);

}  // namespace sk
