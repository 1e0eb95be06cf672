// sk_mirror.cuh -- the exact count with Lemma 2.3 (reversal) on top of
// Lemma 2.2, Skolem and Langford (P = {1..2n} maps onto itself under
// i -> 2n+1-i; hooked Skolem's P does not).
//
// Lemma 2.3: F(n, X) = F(n, reverse(X)); prod x is unchanged too.  With x_2n
// held at +1 (Lemma 2.2) the map that keeps that variable fixed is
//   sigma(X) = reverse(X)          if x_1 = +1,
//   sigma(X) = -reverse(X)         if x_1 = -1   (Lemma 2.2 on top),
// an involution of the half-space under which the summand is invariant.
//
// Work items.  Bits as in sk_exact.cuh (bit i = position i+1; bit 2n-1 held
// at +1).  An item fixes bit 0 (x_1, its "side" s) and the middle bits
// h+1 .. 2n-2-h; it walks bits 1..h and their mirror images 2n-2..2n-1-h
// (m = 2h walk bits: walk index t < h is bit t+1, walk index h+i is bit
// 2n-1-h+i), the low U of them (bits 1..U) unrolled with compile-time
// states.  sigma maps the terms of an item one-to-one onto the terms of the
// item whose middle is the reversed (s = +1) or reversed-and-negated
// (s = -1) pattern, so the two items have equal sums.
//
// The middle bits form mirror pairs (bit h+1+i, bit 2n-2-h-i), i = 0, 1, ...
// from the outside in; sigma acts on each pair alone: s = +1 swaps its two
// values, s = -1 swaps and negates them.  The first pair sigma does not fix
// decides which of two partner items is enumerated: for s = +1 the first
// unequal pair, enumerated as (x = +1, x = -1) with weight 2 (the partner
// (-1, +1) skipped); for s = -1 the first equal pair, enumerated as (+1, +1)
// with weight 2 (partner (-1, -1) skipped).  Items whose first `depth` pairs
// are all fixed by sigma are enumerated as they are, weight 1.  Per side:
//   block d = 0 .. depth-1:  pairs 0..d-1 sigma-fixed (one free bit each),
//                            pair d canonical, pairs d+1.. free (2 bits each),
//                            weight 2;
//   block depth:             pairs 0..depth-1 sigma-fixed, the rest free,
//                            weight 1;
// a fraction 1/2 + 2^{-depth-1} of the items, whose weighted sums add up to
// the sum over the whole half-space.
#pragma once
#include "sk_exact_launch.cuh"

namespace sk {

constexpr int kMirrorDepth = 8;        // mirror pairs examined for the canonical choice
constexpr int kMirrorMinN = 6;         // smallest order with a compiled mirrored kernel

// Shape of the item space of one (n, h).
struct MirrorShape {
  int n, h, pairs, depth;              // pairs = (2n-2-2h)/2 middle mirror pairs
  unsigned long long block_lo[kMirrorDepth + 2];   // first item of each block, per side
  unsigned long long per_side;         // items per side
};

__host__ __device__ inline MirrorShape mirror_shape(int n, int h) {
  MirrorShape sh{};
  sh.n = n;
  sh.h = h;
  sh.pairs = n - 1 - h;
  sh.depth = sh.pairs < kMirrorDepth ? sh.pairs : kMirrorDepth;
  unsigned long long lo = 0;
  for (int d = 0; d < sh.depth; ++d) {
    sh.block_lo[d] = lo;
    lo += 1ULL << (d + 2 * (sh.pairs - 1 - d));
  }
  sh.block_lo[sh.depth] = lo;
  lo += 1ULL << (sh.depth + 2 * (sh.pairs - sh.depth));
  sh.block_lo[sh.depth + 1] = lo;
  sh.per_side = lo;
  return sh;
}

// Item q (0 <= q < 2 per_side) -> the fixed bits (bit set = x of -1): bit 0
// and the middle; *weight = 1 or 2.
__host__ __device__ inline unsigned long long mirror_item_bits(const MirrorShape& sh,
                                                               unsigned long long q, int* weight) {
  const int side = q >= sh.per_side ? 1 : 0;      // 1: x_1 = -1
  unsigned long long r = side ? q - sh.per_side : q;
  int d = 0;
  while (d < sh.depth && r >= sh.block_lo[d + 1]) ++d;
  r -= sh.block_lo[d];
  const int n = sh.n, h = sh.h;
  unsigned long long bits = (unsigned long long)side;
  // pairs 0..d-1: fixed by sigma; one free bit e each
  for (int i = 0; i < d; ++i) {
    const unsigned long long e = (r >> i) & 1ULL;
    const unsigned long long f = side ? (e ^ 1ULL) : e;    // s = -1: unequal pair
    bits |= (e << (h + 1 + i)) | (f << (2 * n - 2 - h - i));
  }
  r >>= d;
  int first_free = d;
  if (d < sh.depth) {
    // pair d canonical: s = +1 -> (x = +1, x = -1); s = -1 -> (+1, +1)
    if (!side) bits |= 1ULL << (2 * n - 2 - h - d);
    first_free = d + 1;
    *weight = 2;
  } else {
    *weight = 1;
  }
  for (int i = first_free; i < sh.pairs; ++i) {
    bits |= ((r & 1ULL) << (h + 1 + i)) | (((r >> 1) & 1ULL) << (2 * n - 2 - h - i));
    r >>= 2;
  }
  return bits;
}

// Walk index t (0 <= t < 2h) -> bit.
__host__ __device__ __forceinline__ int mirror_walk_bit(int n, int h, int t) {
  return t < h ? t + 1 : 2 * n - 1 - h + (t - h);
}

// Inner flip for step S (or the reset flip, S = 0) of the mirrored walk: the
// inner bits are bits 1..U (relative index j = bit - 1), so a left neighbour
// at relative -1 is bit 0 (w0 = 2 x_1, fixed per item) and one further left
// is off the span; right neighbours beyond the block are near[i] = w at bit
// U+1+i.
template <int DELTA, int N, int U, int S>
__device__ __forceinline__ void mirror_inner_update(int (&c)[N],
                                                    const int (&near)[near_count(DELTA, N)],
                                                    int w0) {
  constexpr int Gpre = (S == 0) ? (1 << (U - 1)) : gray(S - 1);
  constexpr int j = (S == 0) ? (U - 1) : ctz_c(S);
  constexpr int xj = xin(Gpre, j);
#pragma unroll
  for (int k = 1; k <= N; ++k) {
    const int d = k + DELTA;
    const int il = j - d, ir = j + d;
    int K = 0;
    if (il >= 0) K += -2 * xj * xin(Gpre, il);
    int v = c[k - 1] + K;
    if (il == -1) v = xj > 0 ? v - w0 : v + w0;
    if (ir < U) {
      v += -2 * xj * xin(Gpre, ir);
    } else {
      v = xj > 0 ? v - near[ir - U] : v + near[ir - U];
    }
    c[k - 1] = v;
  }
}

// Outer flip of bit P (the inner bits are all +1 at this point, +2 in ws).
template <int DELTA, int N, int U>
__device__ __forceinline__ void mirror_outer_flip(int P, int (&c)[N],
                                                  int (&near)[near_count(DELTA, N)], unsigned wsa) {
  const unsigned wj = wsa + (unsigned)P * kWsStride;
  const int sJ = lds_s8(wj) >> 1;
#pragma unroll
  for (int k = 1; k <= N; ++k) {
    const int d = k + DELTA;
    const int t = lds_s8(wj - d * kWsStride) + lds_s8(wj + d * kWsStride);
    c[k - 1] -= sJ * t;
  }
  sts_s8(wj, -2 * sJ);
#define SK_MIRROR_NCASE(I)                                                        \
  case I:                                                                         \
    if constexpr ((I) < near_count(DELTA, N)) near[(I)] = -near[(I)];             \
    break;
  switch (P - U - 1) {
    SK_MIRROR_NCASE(0) SK_MIRROR_NCASE(1) SK_MIRROR_NCASE(2) SK_MIRROR_NCASE(3)
    SK_MIRROR_NCASE(4) SK_MIRROR_NCASE(5) SK_MIRROR_NCASE(6) SK_MIRROR_NCASE(7)
    SK_MIRROR_NCASE(8) SK_MIRROR_NCASE(9) SK_MIRROR_NCASE(10) SK_MIRROR_NCASE(11)
    SK_MIRROR_NCASE(12) SK_MIRROR_NCASE(13) SK_MIRROR_NCASE(14) SK_MIRROR_NCASE(15)
    SK_MIRROR_NCASE(16) SK_MIRROR_NCASE(17) SK_MIRROR_NCASE(18) SK_MIRROR_NCASE(19)
    SK_MIRROR_NCASE(20) SK_MIRROR_NCASE(21) SK_MIRROR_NCASE(22) SK_MIRROR_NCASE(23)
    SK_MIRROR_NCASE(24) SK_MIRROR_NCASE(25) SK_MIRROR_NCASE(26) SK_MIRROR_NCASE(27)
    SK_MIRROR_NCASE(28) SK_MIRROR_NCASE(29) SK_MIRROR_NCASE(30) SK_MIRROR_NCASE(31)
    SK_MIRROR_NCASE(32)
    default: break;
  }
#undef SK_MIRROR_NCASE
}

template <int DELTA, int N, int U, int S, class Acc>
__device__ __forceinline__ void mirror_inner_walk(int (&c)[N],
                                                  const int (&near)[near_count(DELTA, N)], int w0,
                                                  Acc& A) {
  if constexpr (S < (1 << U)) {
    if constexpr (S > 0) mirror_inner_update<DELTA, N, U, S>(c, near, w0);
#pragma unroll
    for (int k = 0; k < N; ++k) asm volatile("" : "+r"(c[k]));
    A.template term<S>(c);
    mirror_inner_walk<DELTA, N, U, S + 1>(c, near, w0, A);
  }
}

// Sum over one mirrored item (m = 2h walk bits) into A, then A.finish, then
// times the item's weight: residues in [0, p).
template <int DELTA, int N, class Acc>
__device__ __forceinline__ void run_item_mirror(int h, unsigned long long q, signed char* ws_col,
                                                Acc& A, int nprimes, const Primes& P,
                                                unsigned long long (&res)[kMaxPrimes]) {
  constexpr int U = inner_bits(N);
  constexpr int NEAR = near_count(DELTA, N);
  constexpr int PAD = ws_pad(DELTA, N);
  static_assert(NEAR <= 33, "near window of the outer flip");
  const MirrorShape sh = mirror_shape(N, h);
  int weight = 1;
  const unsigned long long neg = mirror_item_bits(sh, q, &weight);
  const unsigned long long pres = (2 * N >= 64) ? ~0ULL : ((1ULL << (2 * N)) - 1ULL);
  int c[N];
#pragma unroll
  for (int k = 1; k <= N; ++k) {
    const int d = k + DELTA;
    const unsigned long long pm = pres & (pres >> d);
    c[k - 1] = __popcll(pm) - 2 * __popcll(pm & (neg ^ (neg >> d)));
  }
  const unsigned wsa = (unsigned)__cvta_generic_to_shared(ws_col) + PAD * kWsStride;
  for (int i = -PAD; i < 2 * N + 1 + PAD; ++i) {
    int v = 0;
    if (i >= 0 && i < 2 * N) v = ((neg >> i) & 1ULL) ? -2 : 2;
    sts_s8(wsa + (unsigned)(i * kWsStride), v);
  }
  int near[NEAR];
#pragma unroll
  for (int i = 0; i < NEAR; ++i) near[i] = lds_s8(wsa + (unsigned)((U + 1 + i) * kWsStride));
  const int w0 = (neg & 1ULL) ? -2 : 2;
  const int sb0 = (__popcll(neg) & 1) ? -1 : 1;
  const unsigned long long nblocks = 1ULL << (2 * h - U);
  for (unsigned long long b = 0;; ++b) {
    mirror_inner_walk<DELTA, N, U, 0>(c, near, w0, A);
    if (b + 1 == nblocks) break;
    mirror_inner_update<DELTA, N, U, 0>(c, near, w0);
    const int J = U + __ffsll((long long)(b + 1)) - 1;
    mirror_outer_flip<DELTA, N, U>(mirror_walk_bit(N, h, J), c, near, wsa);
    A.negate();
  }
  const bool flip = (sb0 < 0) != ((nblocks - 1) & 1ULL);
  A.finish(flip, nprimes, res);
  if (weight == 2) {
#pragma unroll
    for (int i = 0; i < kMaxPrimes; ++i)
      if (i < nprimes) res[i] = addmod(res[i], res[i], (unsigned long long)P.pr[i].p);
  }
}

template <int DELTA, int N>
__device__ __noinline__ Res4 mirror_item(int h, unsigned long long item, const Primes* P,
                                         int nprimes, signed char* ws_col) {
  LimbAcc<DELTA, N> A(*P);
  unsigned long long r[kMaxPrimes];
  run_item_mirror<DELTA, N>(h, item, ws_col, A, nprimes, *P, r);
  Res4 out;
#pragma unroll
  for (int i = 0; i < kMaxPrimes; ++i) out.r[i] = r[i];
  return out;
}

// The job's walk width m = 2h travels in ExactJob::m.
template <int DELTA, int N>
struct MirrorItem {
  __device__ __forceinline__ static Res4 eval(const ExactJob& job, const Primes& P, int nprimes,
                                              unsigned long long item, signed char* ws_col) {
    return mirror_item<DELTA, N>(job.m >> 1, item, &P, nprimes, ws_col);
  }
};

template <int DELTA, int N>
__global__ void __launch_bounds__(256, SK_EXACT_MIN_BLOCKS)
    mirror_kernel(ExactJob job, Primes P, int nprimes, unsigned long long item_lo,
                  unsigned long long item_hi, ExactScratch* scr, unsigned long long* item_res) {
  work_loop<MirrorItem<DELTA, N>>(job, P, nprimes, item_lo, item_hi, scr, item_res);
}

template <int DELTA, int N>
cudaError_t launch_mirror(const ExactLaunch& L) {
  static OccupancyCache bps;
  if (L.nprimes < 1 || L.nprimes > kMaxPrimes || L.job.fixed_bit || (L.job.m & 1))
    return cudaErrorInvalidValue;
  const size_t smem = (size_t)ws_len(DELTA, N) * kWsStride;
  int grid = 0;
  cudaError_t e = exact_grid(mirror_kernel<DELTA, N>, L, smem, bps, &grid);
  if (e != cudaSuccess) return e;
  mirror_kernel<DELTA, N><<<grid, L.block_threads, smem, L.stream>>>(
      L.job, L.P, L.nprimes, L.item_lo, L.item_hi, L.scratch, L.item_res);
  return cudaGetLastError();
}

// Mirrored-walk launchers for delta in {0, 1}, n in [kMirrorMinN, kMaxN].
ExactLaunchFn mirror_launcher(int delta, int n);

}  // namespace sk

#define SK_INSTANTIATE_MIRROR(N)                                                  \
  template cudaError_t sk::launch_mirror<0, N>(const sk::ExactLaunch&);           \
  template cudaError_t sk::launch_mirror<1, N>(const sk::ExactLaunch&);
