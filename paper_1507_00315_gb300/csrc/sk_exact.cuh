// sk_exact.cuh -- device side of the exact count (sm_103a).
//
// The count is Lemma 2.1 of the paper: the number of pairings (reflections
// distinct) equals 2^{-2n} sum_{x in {+1,-1}^P} (prod x) prod_k c_k(x) with
// c_k(x) = sum_a x_a x_{a+d_k}.  Lemma 2.2 fixes the variable at max P to +1,
// so the sum H runs over the 2n-1 free variables and equals C * 2^{2n-1}.
//
// Bits.  Position i+1 of the paper is bit i.  Skolem (d_k = k) and Langford
// (d_k = k+1) use bits 0..2n-1, with bit 2n-1 fixed to +1.  Hooked Skolem uses
// bits 0..2n with bit 2n-1 absent (x = 0) and bit 2n fixed to +1.  In every
// problem the free variables are bits 0..2n-2.
//
// Work item.  An item fixes the free bits m..2n-2 from its index q (bit set
// means x = -1) and runs the low m bits through all 2^m values.  The low U bits
// (the "inner" bits) are walked by a fully unrolled reflected Gray code whose
// every state is known at compile time; bits U..m-1 (the "outer" walk bits)
// flip once per 2^U terms (Sec. 2.1: Gray-code order, one variable per step,
// O(n) update of the correlations).
//
// Per flip of bit j every c_k changes by -2 x_j (x_{j-d_k} + x_{j+d_k}).  For an
// inner flip, x_j and every inner neighbour are compile-time constants, and
// the only run-time operand is the outer neighbour, held as w_i = 2 x_i
// (0 for an absent position), so each c_k update is one three-input add.
//
// Product.  |c_k| <= L_k = number of pairs (a, a+d_k) in the span, so the c_k
// are multiplied in int32 groups whose bound stays below 2^31.  Two forms of
// the rest give the same residues (Sec. 2.2: residues modulo co-primes,
// rebuilt by the Chinese remainder theorem on the host):
//   exact digit form (default): the groups are combined exactly in signed
//     radix-2^31 digits and summed in 64-bit words per digit; the item sum is
//     reduced modulo each 62-bit prime once per item.
//   Montgomery form: the first two groups form an exact int64 head (< 2^62);
//     each further group enters through one signed Montgomery step modulo
//     each prime.  A step with R = 2^32 on a in (-2^62, 2^62) and b in
//     (-2^31, 2^31) returns (a b + m p) / 2^32 with m chosen so the division
//     is exact; the result is congruent to a b R^{-1} and stays inside
//     (-2^62, 2^62).  Every term takes the same number of steps, so the sum
//     carries one known factor R^{-(g-2)} that the host removes.
#pragma once
#include <cstdint>

namespace sk {

constexpr int kMaxN = 31;        // largest n with a compiled kernel (2n+1 <= 63 bits)
constexpr int kMaxPrimes = 4;

struct Prime {          // one modulus, split for the signed Montgomery step
  long long p;          // odd, 2^62 - 2^31 < p < 2^62
  int lo;               // signed low limb:  p = hi * 2^32 + lo, lo < 0
  int hi;               // always 2^30 in that window
  unsigned npinv;       // -p^{-1} mod 2^32
};

struct Primes {
  Prime pr[kMaxPrimes];
};

struct Res4 {                    // residues of one work item
  unsigned long long r[kMaxPrimes];
};

// Parameters of one exact-count problem as the kernels see it.
struct ExactJob {
  unsigned long long pres;   // bit i set iff position i+1 belongs to P
  unsigned long long items;  // number of work items (2^{F-m}, F free bits)
  int m;                     // walk bits per item
  int job;                   // slot index of this job's residues
  int fixed_bit;             // 0: none; else a free bit >= m held at +1 (Lemma
                             // 2.4): item indices skip it
};

// Item index -> the free-bit pattern above the walk: a zero is inserted at
// bit `hole` (the fixed variable), the bits at and above it move up by one.
__host__ __device__ __forceinline__ unsigned long long insert_zero_bit(unsigned long long q,
                                                                      int hole) {
  const unsigned long long low = q & ((1ULL << hole) - 1);
  return low | ((q >> hole) << (hole + 1));
}

// ------------------------------------------------------------ compile time

__host__ __device__ constexpr int gray(int s) { return s ^ (s >> 1); }
__host__ __device__ constexpr int ctz_c(int s) {
  int j = 0;
  while (!((s >> j) & 1)) ++j;
  return j;
}
// +1 / -1 value of inner bit i in Gray state G
__host__ __device__ constexpr int xin(int G, int i) { return ((G >> i) & 1) ? -1 : 1; }

// Unrolled Gray bits per block (2^U terms of straight-line code).
#ifndef SK_INNER_BITS
#define SK_INNER_BITS 5
#endif
__host__ __device__ constexpr int inner_bits(int N) {
  return (2 * N - 1) < SK_INNER_BITS ? (2 * N - 1) : SK_INNER_BITS;
}

struct GroupInfo {
  int g;               // number of groups
  int start[kMaxN + 1];
};

// Greedy grouping of c_1..c_N (bounds L_k = 2N - k - DELTA, at least 1) so
// that every group's bound is below 2^31.
__host__ __device__ constexpr GroupInfo make_groups(int DELTA, int N) {
  GroupInfo gi{};
  gi.g = 0;
  long long prod = 1;
  for (int k = 1; k <= N; ++k) {
    long long L = 2LL * N - k - DELTA;
    if (L < 1) L = 1;
    if (k == 1 || prod * L > 2147483647LL) {
      gi.start[gi.g++] = k - 1;
      prod = 1;
    }
    prod *= L;
  }
  gi.start[gi.g] = N;
  return gi;
}

// ------------------------------------------------------------ device math

// Signed Montgomery step: returns r == a * b * 2^{-32} (mod p),
// |r| < (|a| + p) / 2.  (al, ah) is a with a signed low limb:
// a = ah * 2^32 + al.  P1 = al * b and AH = ah * b are shared across primes.
// Every modulus lies in (2^62 - 2^31, 2^62), so its high limb is exactly 2^30
// and m * p = m * lo + (m << 62): the high product is a shift.
__device__ __forceinline__ long long mont_finish(long long P1, long long AH, const Prime& P) {
  int m = (int)((unsigned)P1 * P.npinv);
  long long X = (long long)m * P.lo + P1;     // divisible by 2^32
  return AH + (X >> 32) + ((long long)m << 30);
}

__device__ __forceinline__ void split_signed(long long a, int& al, int& ah) {
  al = (int)(unsigned)a;
  ah = (int)((a - al) >> 32);
}

// 96-bit signed accumulator (a0, a1 unsigned limbs, a2 signed top limb).
__device__ __forceinline__ void acc_add(unsigned& a0, unsigned& a1, unsigned& a2, long long r) {
  unsigned lo = (unsigned)r, hi = (unsigned)((unsigned long long)r >> 32);
  unsigned sx = (unsigned)((int)hi >> 31);
  asm("add.cc.u32 %0, %0, %3;\n\taddc.cc.u32 %1, %1, %4;\n\taddc.u32 %2, %2, %5;"
      : "+r"(a0), "+r"(a1), "+r"(a2)
      : "r"(lo), "r"(hi), "r"(sx));
}
__device__ __forceinline__ void acc_sub(unsigned& a0, unsigned& a1, unsigned& a2, long long r) {
  unsigned lo = (unsigned)r, hi = (unsigned)((unsigned long long)r >> 32);
  unsigned sx = (unsigned)((int)hi >> 31);
  asm("sub.cc.u32 %0, %0, %3;\n\tsubc.cc.u32 %1, %1, %4;\n\tsubc.u32 %2, %2, %5;"
      : "+r"(a0), "+r"(a1), "+r"(a2)
      : "r"(lo), "r"(hi), "r"(sx));
}

// (a2 * 2^64 + a1 * 2^32 + a0) mod p, in [0, p).
__device__ __forceinline__ void acc_neg(unsigned& a0, unsigned& a1, unsigned& a2) {
  const unsigned z = 0u;
  asm("sub.cc.u32 %0, %3, %0;\n\tsubc.cc.u32 %1, %3, %1;\n\tsubc.u32 %2, %3, %2;"
      : "+r"(a0), "+r"(a1), "+r"(a2)
      : "r"(z));
}

__device__ __forceinline__ unsigned long long acc_reduce(unsigned a0, unsigned a1, unsigned a2,
                                                         long long p) {
  unsigned long long L = ((unsigned long long)a1 << 32) | a0;
  long long t64 = (long long)(((unsigned __int128)1 << 64) % (unsigned __int128)p);  // 2^64 mod p
  __int128 v = (__int128)(int)a2 * t64 + (__int128)(L % (unsigned long long)p);
  long long r = (long long)(v % p);
  if (r < 0) r += p;
  return (unsigned long long)r;
}

__device__ __forceinline__ unsigned long long addmod(unsigned long long a, unsigned long long b,
                                                     unsigned long long p) {
  unsigned long long s = a + b;
  return s >= p ? s - p : s;
}

// ------------------------------------------------------------ Gray updates

__host__ __device__ constexpr int near_count(int DELTA, int N) { return N + DELTA; }
// Shared-memory copy of w: positions -PAD .. 2N+PAD, PAD = N+1+DELTA, zero
// outside the span, so an outer flip reads both neighbours without checks.
__host__ __device__ constexpr int ws_pad(int DELTA, int N) { return N + 1 + DELTA; }
__host__ __device__ constexpr int ws_len(int DELTA, int N) { return 2 * ws_pad(DELTA, N) + 2 * N + 1; }
constexpr int kWsStride = 256;   // threads per block, at most

// Inner flip for step S (1 <= S < 2^U), or the reset flip (S = 0: bit U-1
// returns from -1 to +1 at the end of a block).  near[i] = w at position U+i.
template <int DELTA, int N, int U, int S>
__device__ __forceinline__ void inner_update(int (&c)[N], const int (&near)[near_count(DELTA, N)]) {
  constexpr int Gpre = (S == 0) ? (1 << (U - 1)) : gray(S - 1);
  constexpr int j = (S == 0) ? (U - 1) : ctz_c(S);
  constexpr int xj = xin(Gpre, j);
#pragma unroll
  for (int k = 1; k <= N; ++k) {
    const int d = k + DELTA;
    const int il = j - d, ir = j + d;
    int K = 0;
    if (il >= 0) K += -2 * xj * xin(Gpre, il);
    if (ir < U) {
      K += -2 * xj * xin(Gpre, ir);
      c[k - 1] += K;
    } else {
      if (xj > 0) c[k - 1] = c[k - 1] + K - near[ir - U];
      else        c[k - 1] = c[k - 1] + K + near[ir - U];
    }
  }
}

// Byte loads and stores of the shared copy of w (32-bit shared addresses, so
// they stay shared-memory accesses inside the non-inlined item function).
__device__ __forceinline__ int lds_s8(unsigned a) {
  int v;
  asm volatile("ld.shared.s8 %0, [%1];" : "=r"(v) : "r"(a));
  return v;
}
__device__ __forceinline__ void sts_s8(unsigned a, int v) {
  asm volatile("st.shared.s8 [%0], %1;" ::"r"(a), "r"(v));
}

// Outer flip of bit J (inner bits all +1 at this point, and +2 in ws).
// wsa: shared-memory address of this thread's entry for position 0.
template <int DELTA, int N, int U>
__device__ __forceinline__ void outer_flip(int J, int (&c)[N], int (&near)[near_count(DELTA, N)],
                                           unsigned wsa) {
  const unsigned wj = wsa + (unsigned)J * kWsStride;
  const int sJ = lds_s8(wj) >> 1;
#pragma unroll
  for (int k = 1; k <= N; ++k) {
    const int d = k + DELTA;
    const int t = lds_s8(wj - d * kWsStride) + lds_s8(wj + d * kWsStride);
    c[k - 1] -= sJ * t;
  }
  sts_s8(wj, -2 * sJ);
  // keep the register window in step with ws
#define SK_NCASE(I)                                                              \
  case I:                                                                        \
    if constexpr ((I) < near_count(DELTA, N)) near[(I)] = -near[(I)];            \
    break;
  switch (J - U) {
    SK_NCASE(0) SK_NCASE(1) SK_NCASE(2) SK_NCASE(3) SK_NCASE(4) SK_NCASE(5) SK_NCASE(6)
    SK_NCASE(7) SK_NCASE(8) SK_NCASE(9) SK_NCASE(10) SK_NCASE(11) SK_NCASE(12) SK_NCASE(13)
    SK_NCASE(14) SK_NCASE(15) SK_NCASE(16) SK_NCASE(17) SK_NCASE(18) SK_NCASE(19) SK_NCASE(20)
    SK_NCASE(21) SK_NCASE(22) SK_NCASE(23) SK_NCASE(24) SK_NCASE(25) SK_NCASE(26) SK_NCASE(27)
    SK_NCASE(28) SK_NCASE(29) SK_NCASE(30) SK_NCASE(31)
    default: break;
  }
#undef SK_NCASE
}

// ------------------------------------------------------------ group products

template <int DELTA, int N>
__device__ __forceinline__ void group_products(const int (&c)[N],
                                               int (&G)[make_groups(DELTA, N).g]) {
  constexpr GroupInfo gi = make_groups(DELTA, N);
#pragma unroll
  for (int g = 0; g < gi.g; ++g) {
    int v = c[gi.start[g]];
#pragma unroll
    for (int k = gi.start[g] + 1; k < gi.start[g + 1]; ++k) v *= c[k];
    G[g] = v;
  }
}

// ------------------------------------------------------------ Montgomery form

// r[i] == prod_k c_k * R^{-(g-2)} (mod p_i), |r[i]| < 2^62 (exact for g <= 2).
template <int DELTA, int N, int NPR>
__device__ __forceinline__ void term_residues(const int (&c)[N], const Primes& P,
                                              long long (&r)[NPR]) {
  constexpr GroupInfo gi = make_groups(DELTA, N);
  int G[gi.g];
  group_products<DELTA, N>(c, G);
  if constexpr (gi.g == 1) {
#pragma unroll
    for (int i = 0; i < NPR; ++i) r[i] = (long long)G[0];
  } else {
    const long long head = (long long)G[0] * G[1];
    if constexpr (gi.g == 2) {
#pragma unroll
      for (int i = 0; i < NPR; ++i) r[i] = head;
    } else {
      int al, ah;
      split_signed(head, al, ah);
      const long long P1 = (long long)al * G[2];
      const long long AH = (long long)ah * G[2];
#pragma unroll
      for (int i = 0; i < NPR; ++i) {
        long long x = mont_finish(P1, AH, P.pr[i]);
#pragma unroll
        for (int g = 3; g < gi.g; ++g) {
          int bl, bh;
          split_signed(x, bl, bh);
          x = mont_finish((long long)bl * G[g], (long long)bh * G[g], P.pr[i]);
        }
        r[i] = x;
      }
    }
  }
}

// Accumulator of the Montgomery form: per term, the product modulo each
// prime by signed Montgomery steps; terms S and S+1 (S even) have opposite
// signs of prod x, so their difference (|.| < 2^63) enters a 96-bit
// accumulator per prime once.
template <int DELTA, int N, int NPR>
struct MontAcc {
  const Primes& P;
  unsigned acc[NPR][3];
  long long r0[NPR];
  __device__ __forceinline__ explicit MontAcc(const Primes& P_) : P(P_) {
#pragma unroll
    for (int i = 0; i < NPR; ++i) acc[i][0] = acc[i][1] = acc[i][2] = 0u;
  }
  template <int S>
  __device__ __forceinline__ void term(const int (&c)[N]) {
    if constexpr ((S & 1) == 0) {
      term_residues<DELTA, N, NPR>(c, P, r0);
    } else {
      long long r1[NPR];
      term_residues<DELTA, N, NPR>(c, P, r1);
#pragma unroll
      for (int i = 0; i < NPR; ++i) acc_add(acc[i][0], acc[i][1], acc[i][2], r0[i] - r1[i]);
    }
  }
  __device__ __forceinline__ void negate() {
#pragma unroll
    for (int i = 0; i < NPR; ++i) acc_neg(acc[i][0], acc[i][1], acc[i][2]);
  }
  // raw residues (times R^{-(g-2)}) in [0, p), sign applied when flip
  __device__ __forceinline__ void finish(bool flip, int, unsigned long long (&res)[kMaxPrimes]) {
    if (flip) negate();
#pragma unroll
    for (int i = 0; i < NPR; ++i) res[i] = acc_reduce(acc[i][0], acc[i][1], acc[i][2], P.pr[i].p);
  }
};

// ------------------------------------------------------------ exact digit form

// Signed-digit form of the exact product.  The c_k are multiplied in int32
// groups (bound below 2^31 each); the running product of the groups is kept
// as signed radix-2^31 digits r_0..r_{K-1} (r_i in [0, 2^31) below the top,
// the top digit signed), so every digit is an int32 and digit * group is one
// signed 32x32->64 multiply(-add).  A term enters 64-bit accumulators, one
// per digit, in one of two ways:
//   tail form:  the last group T (bound below 2^tb) is not folded into the
//               digits; acc_i += r_i * T is one multiply-add per digit.  An
//               item of 2^m terms fits when m <= 32 - tb.
//   digit form: every group is folded in; acc_i +/-= r_i is a 64-bit add per
//               digit.  An item fits when m <= 31.
// No absolute values, sign masks or carry chains per term.  The item sum
// sum_i acc_i 2^{31 i} is reduced modulo the primes once, at the end of the
// item (Sec. 2.2: residues modulo co-primes).
constexpr int kMaxGroups = 12;

struct DigitPlan {
  int tail_form;              // 1: tail form, 0: digit form
  int tree;                   // group products as balanced trees (else chains)
  int ng;                     // groups folded into the digits
  int fac[kMaxN];             // factor indices (0-based k-1), group by group
  int start[kMaxGroups + 1];  // group g: fac[start[g] .. start[g+1])
  int ntail;                  // tail: fac[start[ng] .. start[ng] + ntail)
  int tail_bits;              // tail bound < 2^tail_bits
  int digits[kMaxGroups];     // digits of the product of groups 0..g
  int kd;                     // digits of the folded product
  int cost;                   // estimated multiply-pipe cycles per term
  int max_m;                  // largest walk width of an item
};

__host__ __device__ constexpr long long factor_bound(int DELTA, int N, int k) {
  const long long L = 2LL * N - k - DELTA;
  return L < 1 ? 1 : L;
}

// Groups of the factors idx[0..n) with bound < 2^31 each: contiguous greedy
// in index order, or first-fit decreasing by bound into as few groups as it
// finds.  Writes fac / start / ng.
__host__ __device__ constexpr bool pack_groups(int DELTA, int N, const int* idx, int n,
                                               bool greedy, DigitPlan& dp) {
  if (greedy) {
    int ng = 0, pos = 0;
    long long pr = 1;
    for (int i = 0; i < n; ++i) {
      const long long L = factor_bound(DELTA, N, idx[i] + 1);
      if (i == 0 || pr * L >= 2147483648LL) {
        if (ng >= kMaxGroups) return false;
        dp.start[ng++] = pos;
        pr = 1;
      }
      pr *= L;
      dp.fac[pos++] = idx[i];
    }
    dp.ng = ng;
    dp.start[ng] = pos;
    return true;
  }
  int ord[kMaxN] = {};
  for (int i = 0; i < n; ++i) ord[i] = idx[i];
  for (int i = 1; i < n; ++i) {          // largest bound first
    const int v = ord[i];
    int j = i - 1;
    while (j >= 0 && factor_bound(DELTA, N, ord[j] + 1) < factor_bound(DELTA, N, v + 1)) {
      ord[j + 1] = ord[j];
      --j;
    }
    ord[j + 1] = v;
  }
  for (int nb = 1; nb <= kMaxGroups && nb <= n; ++nb) {
    long long prod[kMaxGroups] = {};
    int cnt[kMaxGroups] = {};
    int member[kMaxGroups][kMaxN] = {};
    for (int g = 0; g < nb; ++g) prod[g] = 1;
    bool ok = true;
    for (int i = 0; i < n && ok; ++i) {
      const long long L = factor_bound(DELTA, N, ord[i] + 1);
      int best = -1;                      // the fullest group that still fits
      for (int g = 0; g < nb; ++g)
        if (prod[g] * L < 2147483648LL && (best < 0 || prod[g] > prod[best])) best = g;
      if (best < 0) {
        ok = false;
      } else {
        prod[best] *= L;
        member[best][cnt[best]++] = ord[i];
      }
    }
    if (!ok) continue;
    int pos = 0, ng = 0;
    for (int g = 0; g < nb; ++g) {
      if (!cnt[g]) continue;
      dp.start[ng++] = pos;
      for (int i = 0; i < cnt[g]; ++i) dp.fac[pos++] = member[g][i];
    }
    dp.ng = ng;
    dp.start[ng] = pos;
    return true;
  }
  return false;
}

// Digits after each folded group (from the exact bound, 8 x 32-bit limbs)
// and the estimated cost: 2 multiply-pipe cycles per int32 product, 4 per
// 32x32->64 product.
__host__ __device__ constexpr void digit_counts(int DELTA, int N, DigitPlan& dp) {
  unsigned w[8] = {1, 0, 0, 0, 0, 0, 0, 0};
  int wide = 0;
  dp.kd = 1;
  for (int g = 0; g < dp.ng; ++g) {
    for (int i = dp.start[g]; i < dp.start[g + 1]; ++i) {
      const unsigned long long L = (unsigned long long)factor_bound(DELTA, N, dp.fac[i] + 1);
      unsigned long long carry = 0;
      for (int j = 0; j < 8; ++j) {
        const unsigned long long x = (unsigned long long)w[j] * L + carry;
        w[j] = (unsigned)x;
        carry = x >> 32;
      }
    }
    int top = 7;
    while (top > 0 && w[top] == 0) --top;
    int bits = 0;
    while (bits < 32 && (w[top] >> bits)) ++bits;
    bits += top * 32;
    const int k = (bits + 30) / 31;
    if (g > 0) wide += dp.digits[g - 1];
    dp.digits[g] = k < 1 ? 1 : k;
    dp.kd = dp.digits[g];
  }
  if (dp.tail_form) wide += dp.kd;
  const int nf = dp.start[dp.ng] + dp.ntail;
  const int imul = nf - dp.ng - (dp.tail_form ? 1 : 0);
  dp.cost = 2 * imul + 4 * wide + (dp.tail_form ? 0 : 1);
}

// Reorders the groups and the factors inside each group (a seeded shuffle;
// the grouping itself is unchanged).  Different orders give the compiler
// different instruction schedules of the same work.
__host__ __device__ constexpr DigitPlan permute_plan(int DELTA, int N, DigitPlan dp,
                                                     unsigned seed) {
  if (!seed) return dp;
  unsigned x = seed * 2654435761u + 12345u;
  int order[kMaxGroups] = {};
  for (int g = 0; g < dp.ng; ++g) order[g] = g;
  for (int g = dp.ng - 1; g > 0; --g) {
    x = x * 1664525u + 1013904223u;
    const int j = (int)((x >> 8) % (unsigned)(g + 1));
    const int t = order[g];
    order[g] = order[j];
    order[j] = t;
  }
  DigitPlan q = dp;
  int pos = 0;
  for (int g = 0; g < dp.ng; ++g) {
    const int og = order[g], n = dp.start[og + 1] - dp.start[og];
    int f[kMaxN] = {};
    for (int i = 0; i < n; ++i) f[i] = dp.fac[dp.start[og] + i];
    for (int i = n - 1; i > 0; --i) {
      x = x * 1664525u + 1013904223u;
      const int j = (int)((x >> 8) % (unsigned)(i + 1));
      const int t = f[i];
      f[i] = f[j];
      f[j] = t;
    }
    q.start[g] = pos;
    for (int i = 0; i < n; ++i) q.fac[pos++] = f[i];
  }
  q.start[dp.ng] = pos;
  for (int i = 0; i < dp.ntail; ++i) q.fac[pos + i] = dp.fac[dp.start[dp.ng] + i];
  digit_counts(DELTA, N, q);
  if (q.ng == 0) q.kd = 1;
  return q;
}

// How a (delta, n) kernel is planned: rule 0 picks the form, the tail and the
// grouping of least estimated cost; rule 1 takes the tail form with the last
// factors below 2^14 as tail and contiguous greedy groups.  The entries were
// chosen by timing every variant on the GB300 (2^34-term slices of S(n),
// L(n), compiled as the library is); plans of equal cost can differ by up to
// 30 % in speed because the compiler schedules them differently.
struct PlanVariant {
  int rule, greedy, tree;
  unsigned seed;
};
__host__ __device__ constexpr PlanVariant plan_variant(int DELTA, int N) {
  if (N < 14) return {0, 1, 0, 0};
  if (N > 24) return {0, 0, 0, 0};
  constexpr PlanVariant skolem[11] = {
      {0, 1, 0, 0}, {0, 0, 0, 0}, {0, 1, 0, 1}, {1, 0, 1, 1}, {1, 0, 0, 2}, {1, 0, 1, 2},
      {0, 0, 1, 1}, {0, 1, 0, 0}, {1, 0, 1, 1}, {0, 1, 1, 0}, {1, 0, 0, 0}};
  constexpr PlanVariant langford[11] = {
      {1, 0, 0, 0}, {0, 1, 1, 0}, {0, 1, 0, 2}, {1, 0, 0, 1}, {1, 0, 0, 0}, {1, 0, 0, 3},
      {1, 0, 0, 2}, {0, 0, 1, 1}, {1, 0, 0, 0}, {0, 1, 0, 2}, {1, 0, 1, 1}};
  return DELTA ? langford[N - 14] : skolem[N - 14];
}

// Smallest walk width the planner gives an item: long enough that its setup
// and final reduction stay a small part of it.
__host__ __device__ constexpr int digit_min_walk_bits(int N) {
  return (2 * N - 1) < 12 ? (2 * N - 1) : 12;
}

__host__ __device__ constexpr DigitPlan make_digit_plan(int DELTA, int N) {
  const PlanVariant pv = plan_variant(DELTA, N);
  const int min_m = digit_min_walk_bits(N);
  int all[kMaxN] = {};
  for (int i = 0; i < N; ++i) all[i] = i;
  DigitPlan best{};
  best.cost = 1 << 30;
  if (pv.rule == 1) {
    long long tp = factor_bound(DELTA, N, N);
    int t = N - 1;
    while (t > 0 && tp * factor_bound(DELTA, N, t) < (1LL << 14)) {
      tp *= factor_bound(DELTA, N, t);
      --t;
    }
    int b = 0;
    while ((1LL << b) <= tp) ++b;
    DigitPlan dp{};
    dp.tail_form = 1;
    dp.ntail = N - t;
    dp.tail_bits = b;
    if (32 - b >= min_m && pack_groups(DELTA, N, all, t, true, dp)) {
      for (int i = 0; i < dp.ntail; ++i) dp.fac[dp.start[dp.ng] + i] = t + i;
      digit_counts(DELTA, N, dp);
      dp.max_m = 32 - b;
      best = dp;
    }
  }
  if (best.cost == (1 << 30)) {
    {
      DigitPlan dp{};
      if (pack_groups(DELTA, N, all, N, pv.greedy != 0, dp)) {
        digit_counts(DELTA, N, dp);
        dp.max_m = 31;
        best = dp;
      }
    }
    for (int tb = 4; tb <= 28; ++tb) {
      // tail: the last factors (smallest bounds) while the bound stays < 2^tb
      long long tp = factor_bound(DELTA, N, N);
      if (tp >= (1LL << tb)) continue;
      int t = N - 1;
      while (t > 0 && tp * factor_bound(DELTA, N, t) < (1LL << tb)) {
        tp *= factor_bound(DELTA, N, t);
        --t;
      }
      int b = 0;
      while ((1LL << b) <= tp) ++b;
      if (32 - b < min_m) continue;
      DigitPlan dp{};
      dp.tail_form = 1;
      dp.ntail = N - t;
      dp.tail_bits = b;
      if (t == 0) {
        dp.ng = 0;
        dp.start[0] = 0;
      } else if (!pack_groups(DELTA, N, all, t, pv.greedy != 0, dp)) {
        continue;
      }
      for (int i = 0; i < dp.ntail; ++i) dp.fac[dp.start[dp.ng] + i] = t + i;
      digit_counts(DELTA, N, dp);
      if (dp.ng == 0) dp.kd = 1;
      dp.max_m = 32 - b;
      if (dp.cost < best.cost || (dp.cost == best.cost && dp.max_m > best.max_m)) best = dp;
    }
  }
  const int mm = best.max_m;
  best = permute_plan(DELTA, N, best, pv.seed);
  best.max_m = mm;
  best.tree = pv.tree;
  return best;
}

// Largest walk width of an item whose sum fits the 64-bit digit accumulators.
__host__ __device__ constexpr int limb_max_walk_bits(int DELTA, int N) {
  return make_digit_plan(DELTA, N).max_m;
}

// Signed 32 x 32 -> 64 multiply(-add): one instruction on the device.
__host__ __device__ __forceinline__ long long wide_mul_s32(int a, int b) {
#ifdef __CUDA_ARCH__
  long long d;
  asm("mul.wide.s32 %0, %1, %2;" : "=l"(d) : "r"(a), "r"(b));
  return d;
#else
  return (long long)a * b;
#endif
}
__host__ __device__ __forceinline__ long long wide_mad_s32(int a, int b, long long c) {
#ifdef __CUDA_ARCH__
  long long d;
  asm("mad.wide.s32 %0, %1, %2, %3;" : "=l"(d) : "r"(a), "r"(b), "l"(c));
  return d;
#else
  return (long long)a * b + c;
#endif
}

// Product of the n factors c[f[0..n)]: a balanced tree or a chain of int32
// products (n and f are compile-time constants once the callers unroll).
template <int NN>
__host__ __device__ __forceinline__ int group_product(const int (&c)[NN], const int* f, int n,
                                                      bool tree) {
  if (tree) {
    int v[NN];
#pragma unroll
    for (int i = 0; i < NN; ++i)
      if (i < n) v[i] = c[f[i]];
#pragma unroll
    for (int w = 1; w < NN; w *= 2)
#pragma unroll
      for (int i = 0; i + w < NN; i += 2 * w)
        if (i + w < n) v[i] *= v[i + w];
    return v[0];
  }
  int v = c[f[0]];
#pragma unroll
  for (int i = 1; i < NN; ++i)
    if (i < n) v *= c[f[i]];
  return v;
}

// Digits r of one term's folded groups and its tail product T (tail form;
// T = 1 in the digit form), negated when NEG:
//   tail form:  (-1)^NEG prod_k c_k = T * sum_i r_i 2^{31 i}
//   digit form: (-1)^NEG prod_k c_k = sum_i r_i 2^{31 i}
template <int DELTA, int N, int NEG>
__host__ __device__ __forceinline__ void digit_product(const int (&c)[N],
                                                      int (&r)[make_digit_plan(DELTA, N).kd],
                                                      int& T) {
  constexpr DigitPlan dp = make_digit_plan(DELTA, N);
  constexpr int K = dp.kd;
  T = 1;
  if constexpr (dp.tail_form) {
    T = group_product(c, dp.fac + dp.start[dp.ng], dp.ntail, dp.tree != 0);
    if constexpr (NEG) T = -T;
  }
  if constexpr (dp.ng == 0) {
    r[0] = 1;
  } else {
    int G[dp.ng];
#pragma unroll
    for (int g = 0; g < dp.ng; ++g)
      G[g] = group_product(c, dp.fac + dp.start[g], dp.start[g + 1] - dp.start[g], dp.tree != 0);
    if constexpr (!dp.tail_form && NEG) G[0] = -G[0];
    r[0] = G[0];
#pragma unroll
    for (int g = 1; g < dp.ng; ++g) {
      const int kc = dp.digits[g - 1], kn = dp.digits[g];
      long long carry = 0;
#pragma unroll
      for (int i = 0; i < K; ++i) {
        if (i < kn) {
          const long long v = (i < kc) ? (i == 0 ? wide_mul_s32(r[i], G[g])
                                                 : wide_mad_s32(r[i], G[g], carry))
                                       : carry;
          if (i < kn - 1) {
            r[i] = (int)((unsigned)v & 0x7FFFFFFFu);
            carry = v >> 31;
          } else {
            r[i] = (int)v;
          }
        }
      }
    }
  }
}

// Reductions for a modulus p in (2^62 - 2^31, 2^62), the window every prime
// of the exact count lies in.
// a mod p in [0, p) for any signed 64-bit a: a quotient estimate in double
// precision is off by at most one, which one correction on each side fixes.
__host__ __device__ __forceinline__ unsigned long long signed_mod(long long a,
                                                                 unsigned long long p) {
  const long long q = (long long)((double)a / (double)p);
  long long r = a - q * (long long)p;        // |r| < 2p: no overflow
  if (r < 0) r += (long long)p;
  if (r >= (long long)p) r -= (long long)p;
  if (r < 0) r += (long long)p;
  return (unsigned long long)r;
}
// (u 2^31 + a) mod p for u, a in [0, p): with u = uh 2^31 + ul and
// 2^62 = p + delta (0 < delta < 2^31), u 2^31 == uh delta + ul 2^31.
__host__ __device__ __forceinline__ unsigned long long horner31_mod(unsigned long long u,
                                                                   unsigned long long a,
                                                                   unsigned long long p) {
  const unsigned long long delta = (1ULL << 62) - p;
  unsigned long long v = (u >> 31) * delta + ((u & 0x7FFFFFFFULL) << 31) + a;   // < 3 * 2^62
  v = (v >> 62) * delta + (v & ((1ULL << 62) - 1));                            // < 2^62 + 2^33
  if (v >= p) v -= p;
  if (v >= p) v -= p;
  return v;
}

// Residues of (flip ? -1 : 1) * sum_{i<K} a_i 2^{31 i} modulo the primes.
// Kept out of line: code around the walk changes how the compiler allocates
// and schedules the walk itself (by up to 10 % in speed), so the item
// function holds the walk and little else.
constexpr int kMaxDigits = 6;
static __device__ __noinline__ void reduce_digits(const long long (&a)[kMaxDigits], int K, bool flip,
                                           int nprimes, const Primes* P,
                                           unsigned long long (&res)[kMaxPrimes]) {
  for (int j = 0; j < kMaxPrimes; ++j) {
    if (j >= nprimes) {
      res[j] = 0;
      continue;
    }
    const unsigned long long p = (unsigned long long)P->pr[j].p;
    unsigned long long u = 0;
    for (int i = K - 1; i >= 0; --i) u = horner31_mod(u, signed_mod(a[i], p), p);
    res[j] = (flip && u) ? p - u : u;
  }
}

// Accumulator of the exact form: one 64-bit signed word per digit.
template <int DELTA, int N>
struct LimbAcc {
  static constexpr int K = make_digit_plan(DELTA, N).kd;
  static constexpr int TAIL = make_digit_plan(DELTA, N).tail_form;
  static_assert(K <= kMaxDigits, "digits of the exact product");
  const Primes& P;
  long long acc[K];
  __device__ __forceinline__ explicit LimbAcc(const Primes& P_) : P(P_) {
#pragma unroll
    for (int i = 0; i < K; ++i) acc[i] = 0;
  }
  template <int S>
  __device__ __forceinline__ void term(const int (&c)[N]) {
    int r[K];
    int T;
    digit_product<DELTA, N, (S & 1)>(c, r, T);
    if constexpr (TAIL) {
#pragma unroll
      for (int i = 0; i < K; ++i) acc[i] = wide_mad_s32(r[i], T, acc[i]);
    } else {
#pragma unroll
      for (int i = 0; i < K; ++i) acc[i] += (long long)r[i];
    }
  }
  __device__ __forceinline__ void negate() {
#pragma unroll
    for (int i = 0; i < K; ++i) acc[i] = -acc[i];
  }
  // residues of (flip ? -1 : 1) * sum_i acc_i 2^{31 i}, in [0, p)
  __device__ __forceinline__ void finish(bool flip, int nprimes,
                                         unsigned long long (&res)[kMaxPrimes]) {
    long long a[kMaxDigits] = {};
#pragma unroll
    for (int i = 0; i < K; ++i) a[i] = acc[i];
    reduce_digits(a, K, flip, nprimes, &P, res);
  }
};

// ------------------------------------------------------------ the walk

template <int DELTA, int N, int U, int S, class Acc>
__device__ __forceinline__ void inner_walk(int (&c)[N], const int (&near)[near_count(DELTA, N)],
                                           Acc& A) {
  if constexpr (S < (1 << U)) {
    if constexpr (S > 0) inner_update<DELTA, N, U, S>(c, near);
#pragma unroll
    for (int k = 0; k < N; ++k) asm volatile("" : "+r"(c[k]));
    A.template term<S>(c);
    inner_walk<DELTA, N, U, S + 1>(c, near, A);
  }
}

// Sum over one item into A, then A.finish: residues in [0, p).
// ws_col: this thread's column of the shared w array (stride kWsStride).
template <int DELTA, int N, class Acc>
__device__ __forceinline__ void run_item(unsigned long long pres, int m, unsigned long long q,
                                         signed char* ws_col, Acc& A, int nprimes,
                                         unsigned long long (&res)[kMaxPrimes]) {
  constexpr int U = inner_bits(N);
  constexpr int NEAR = near_count(DELTA, N);
  constexpr int PAD = ws_pad(DELTA, N);
  const unsigned long long neg = (q << m) & pres;
  int c[N];
#pragma unroll
  for (int k = 1; k <= N; ++k) {
    const int d = k + DELTA;
    const unsigned long long pm = pres & (pres >> d);
    c[k - 1] = __popcll(pm) - 2 * __popcll(pm & (neg ^ (neg >> d)));
  }
  // w = 2x (0 off the span); inner positions start at +1
  const unsigned wsa = (unsigned)__cvta_generic_to_shared(ws_col) + PAD * kWsStride;
  for (int i = -PAD; i < 2 * N + 1 + PAD; ++i) {
    int v = 0;
    if (i >= 0 && i < 64) {
      const int present = (int)((pres >> i) & 1ULL);
      const int negative = (int)((neg >> i) & 1ULL);
      v = present ? (negative ? -2 : 2) : 0;
    }
    sts_s8(wsa + (unsigned)(i * kWsStride), v);
  }
  int near[NEAR];
#pragma unroll
  for (int i = 0; i < NEAR; ++i) near[i] = lds_s8(wsa + (unsigned)((U + i) * kWsStride));
  // sign of prod x at the first block; every outer flip negates it, which the
  // loop applies by negating the accumulator (see below)
  const int sb0 = (__popcll(neg) & 1) ? -1 : 1;
  const unsigned long long nblocks = 1ULL << (m - U);
  for (unsigned long long b = 0;; ++b) {
    inner_walk<DELTA, N, U, 0>(c, near, A);
    if (b + 1 == nblocks) break;
    inner_update<DELTA, N, U, 0>(c, near);             // inner bits back to +1
    const int J = U + __ffsll((long long)(b + 1)) - 1;
    outer_flip<DELTA, N, U>(J, c, near, wsa);
    // block b+1 has the opposite sign of prod x: negate what was summed so far
    // and keep adding with the same signs; the total is fixed once below
    A.negate();
  }
  // A = (-1)^{nblocks-1} * sum_b (-1)^b block_b; wanted: sb0 * sum_b (-1)^b block_b
  const bool flip = (sb0 < 0) != ((nblocks - 1) & 1ULL);
  A.finish(flip, nprimes, res);
}

}  // namespace sk
