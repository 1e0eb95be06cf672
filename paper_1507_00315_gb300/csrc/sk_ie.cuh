// sk_ie.cuh -- device side of the inclusion-exclusion count (Sec. 2: the
// third counting approach the paper lists, after Larsen).
//
// Universe: every way of placing each pair k at two positions a, a+d_k of P,
// overlaps allowed.  A placement that leaves no position of P empty is a
// sequence; one that avoids every position of a set S lies inside T = P \ S,
// and there are prod_k N_k(T) of those, N_k(T) = #{a : a, a+d_k in T}.  By
// inclusion-exclusion over S the sequences (reflections distinct) number
//   sum_{T subset of P} (-1)^{|P| - |T|} prod_k N_k(T).
// This shares no arithmetic with Lemma 2.1 (no +-1 variables, no division by
// 2^{2n-1}, no symmetry): it is an independent route to the same counts.
//
// Variables.  y_i = 1 iff the i-th position of P (increasing order) is in T,
// i = 0..2n-1.  Positions 1..2n-1 belong to P in every variant, so variable i
// is bit i of the position mask for i <= 2n-2; variable 2n-1 is max P (bit
// 2n-1, or bit 2n for hooked Skolem).  A work item of walk width m fixes
// variables m..2n-1 from its index q (bit b of q -> variable m+b) and runs the
// low m through all 2^m values in reflected Gray order: the low U of them
// unrolled with compile-time states, the others flipped from a shared-memory
// copy of y, the layout of the signed-sum walk (sk_exact.cuh).
//
// A flip of y_j by dy = +-1 changes each N_k by dy (y_{j-d_k} + y_{j+d_k}).
// Every flip changes |T| by one, so the term signs alternate along the walk
// exactly as the signs of prod x do in Lemma 2.1's walk, and the signed-digit
// accumulator of the exact form (LimbAcc) sums the terms unchanged.  Each N_k
// lies in [0, L_k], L_k the number of pairs at distance d_k -- the bound the
// digit plan of that form is built on -- so the digits, the walk-width limit
// and the per-item reduction modulo the primes carry over.
#pragma once
#include "sk_exact_launch.cuh"

namespace sk {

constexpr int kMaxIeN = 24;      // largest n with a compiled inclusion-exclusion kernel

// Inner flip for step S (1 <= S < 2^U), or the reset flip (S = 0: bit U-1
// returns from 1 to 0 at the end of a block).  near[i] = y at position U+i.
template <int DELTA, int N, int U, int S>
__device__ __forceinline__ void ie_inner_update(int (&c)[N], const int (&near)[near_count(DELTA, N)]) {
  constexpr int Gpre = (S == 0) ? (1 << (U - 1)) : gray(S - 1);
  constexpr int j = (S == 0) ? (U - 1) : ctz_c(S);
  constexpr int dy = ((Gpre >> j) & 1) ? -1 : 1;
#pragma unroll
  for (int k = 1; k <= N; ++k) {
    const int d = k + DELTA;
    const int il = j - d, ir = j + d;
    int K = 0;
    if (il >= 0) K += dy * ((Gpre >> il) & 1);
    if (ir < U) {
      K += dy * ((Gpre >> ir) & 1);
      c[k - 1] += K;
    } else {
      if (dy > 0) c[k - 1] = c[k - 1] + K + near[ir - U];
      else        c[k - 1] = c[k - 1] + K - near[ir - U];
    }
  }
}

// Outer flip of bit J (the inner bits are all 0 at this point, and 0 in ws).
template <int DELTA, int N, int U>
__device__ __forceinline__ void ie_outer_flip(int J, int (&c)[N], int (&near)[near_count(DELTA, N)],
                                              unsigned wsa) {
  const unsigned wj = wsa + (unsigned)J * kWsStride;
  const int yJ = lds_s8(wj);
  const int dy = 1 - 2 * yJ;
#pragma unroll
  for (int k = 1; k <= N; ++k) {
    const int d = k + DELTA;
    const int t = lds_s8(wj - d * kWsStride) + lds_s8(wj + d * kWsStride);
    c[k - 1] += dy * t;
  }
  sts_s8(wj, 1 - yJ);
#define SK_IE_NCASE(I)                                                           \
  case I:                                                                        \
    if constexpr ((I) < near_count(DELTA, N)) near[(I)] = 1 - near[(I)];         \
    break;
  switch (J - U) {
    SK_IE_NCASE(0) SK_IE_NCASE(1) SK_IE_NCASE(2) SK_IE_NCASE(3) SK_IE_NCASE(4)
    SK_IE_NCASE(5) SK_IE_NCASE(6) SK_IE_NCASE(7) SK_IE_NCASE(8) SK_IE_NCASE(9)
    SK_IE_NCASE(10) SK_IE_NCASE(11) SK_IE_NCASE(12) SK_IE_NCASE(13) SK_IE_NCASE(14)
    SK_IE_NCASE(15) SK_IE_NCASE(16) SK_IE_NCASE(17) SK_IE_NCASE(18) SK_IE_NCASE(19)
    SK_IE_NCASE(20) SK_IE_NCASE(21) SK_IE_NCASE(22) SK_IE_NCASE(23) SK_IE_NCASE(24)
    SK_IE_NCASE(25)
    default: break;
  }
#undef SK_IE_NCASE
}

template <int DELTA, int N, int U, int S, class Acc>
__device__ __forceinline__ void ie_inner_walk(int (&c)[N], const int (&near)[near_count(DELTA, N)],
                                              Acc& A) {
  if constexpr (S < (1 << U)) {
    if constexpr (S > 0) ie_inner_update<DELTA, N, U, S>(c, near);
#pragma unroll
    for (int k = 0; k < N; ++k) asm volatile("" : "+r"(c[k]));
    A.template term<S>(c);
    ie_inner_walk<DELTA, N, U, S + 1>(c, near, A);
  }
}

// Sum over one item into A, then A.finish: residues in [0, p).
template <int DELTA, int N, class Acc>
__device__ __forceinline__ void run_item_ie(unsigned long long pres, int m, unsigned long long q,
                                            signed char* ws_col, Acc& A, int nprimes,
                                            unsigned long long (&res)[kMaxPrimes]) {
  constexpr int U = inner_bits(N);
  constexpr int NEAR = near_count(DELTA, N);
  constexpr int PAD = ws_pad(DELTA, N);
  static_assert(NEAR <= 26, "near window of the outer flip");
  const int F = 2 * N - 1;                      // variables 0..2N-2 are bits 0..2N-2
  const int top = 63 - __clzll((long long)pres);
  const unsigned long long low = (q & ((1ULL << (F - m)) - 1ULL)) << m;
  const unsigned long long T = (low | (((q >> (F - m)) & 1ULL) << top)) & pres;
  int c[N];
#pragma unroll
  for (int k = 1; k <= N; ++k) c[k - 1] = __popcll(T & (T >> (k + DELTA)));
  // ws = y (0 / 1; 0 off P and for the walk bits, which start outside T)
  const unsigned wsa = (unsigned)__cvta_generic_to_shared(ws_col) + PAD * kWsStride;
  for (int i = -PAD; i < 2 * N + 1 + PAD; ++i) {
    const int v = (i >= 0 && i < 64) ? (int)((T >> i) & 1ULL) : 0;
    sts_s8(wsa + (unsigned)(i * kWsStride), v);
  }
  int near[NEAR];
#pragma unroll
  for (int i = 0; i < NEAR; ++i) near[i] = lds_s8(wsa + (unsigned)((U + i) * kWsStride));
  // sign (-1)^{|P| - |T|} of the first term (|P| = 2N is even); every outer
  // flip negates it, applied by negating the accumulator as in run_item
  const int sb0 = (__popcll(T) & 1) ? -1 : 1;
  const unsigned long long nblocks = 1ULL << (m - U);
  for (unsigned long long b = 0;; ++b) {
    ie_inner_walk<DELTA, N, U, 0>(c, near, A);
    if (b + 1 == nblocks) break;
    ie_inner_update<DELTA, N, U, 0>(c, near);          // inner bits back to 0
    const int J = U + __ffsll((long long)(b + 1)) - 1;
    ie_outer_flip<DELTA, N, U>(J, c, near, wsa);
    A.negate();
  }
  const bool flip = (sb0 < 0) != ((nblocks - 1) & 1ULL);
  A.finish(flip, nprimes, res);
}

template <int DELTA, int N>
__device__ __noinline__ Res4 ie_item(unsigned long long pres, int m, unsigned long long item,
                                     const Primes* P, int nprimes, signed char* ws_col) {
  LimbAcc<DELTA, N> A(*P);
  unsigned long long r[kMaxPrimes];
  run_item_ie<DELTA, N>(pres, m, item, ws_col, A, nprimes, r);
  Res4 out;
#pragma unroll
  for (int i = 0; i < kMaxPrimes; ++i) out.r[i] = r[i];
  return out;
}

template <int DELTA, int N>
struct IeItem {
  __device__ __forceinline__ static Res4 eval(const ExactJob& job, const Primes& P, int nprimes,
                                              unsigned long long item, signed char* ws_col) {
    return ie_item<DELTA, N>(job.pres, job.m, item, &P, nprimes, ws_col);
  }
};

template <int DELTA, int N>
__global__ void __launch_bounds__(256, SK_EXACT_MIN_BLOCKS)
    ie_kernel(ExactJob job, Primes P, int nprimes, unsigned long long item_lo,
              unsigned long long item_hi, ExactScratch* scr, unsigned long long* item_res) {
  work_loop<IeItem<DELTA, N>>(job, P, nprimes, item_lo, item_hi, scr, item_res);
}

template <int DELTA, int N>
cudaError_t launch_ie(const ExactLaunch& L) {
  static OccupancyCache bps;
  if (L.nprimes < 1 || L.nprimes > kMaxPrimes || L.job.fixed_bit) return cudaErrorInvalidValue;
  const size_t smem = (size_t)ws_len(DELTA, N) * kWsStride;
  int grid = 0;
  cudaError_t e = exact_grid(ie_kernel<DELTA, N>, L, smem, bps, &grid);
  if (e != cudaSuccess) return e;
  ie_kernel<DELTA, N><<<grid, L.block_threads, smem, L.stream>>>(
      L.job, L.P, L.nprimes, L.item_lo, L.item_hi, L.scratch, L.item_res);
  return cudaGetLastError();
}

// Inclusion-exclusion launchers for delta in {0, 1}, n in [1, kMaxIeN].
ExactLaunchFn ie_launcher(int delta, int n);

}  // namespace sk

#define SK_INSTANTIATE_IE(N)                                                  \
  template cudaError_t sk::launch_ie<0, N>(const sk::ExactLaunch&);           \
  template cudaError_t sk::launch_ie<1, N>(const sk::ExactLaunch&);
