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
// Product.  |c_k| <= L_k = number of pairs (a, a+d_k) in the span.  The c_k
// are multiplied in int32 in groups whose bound stays below 2^31; the first two
// groups form an exact int64 head (< 2^62); each further group enters through
// one signed Montgomery step modulo each 62-bit prime (Sec. 2.2: residues
// modulo co-primes, rebuilt by the Chinese remainder theorem on the host).  A
// Montgomery step with R = 2^32 on a in (-2^62, 2^62) and b in (-2^31, 2^31)
// returns (a b + m p) / 2^32 with m chosen so the division is exact; the result
// is congruent to a b R^{-1} and stays inside (-2^62, 2^62).  Every term of a
// problem takes the same number of steps, so the sum carries one known factor
// R^{-(g-2)} that the host removes.
#pragma once
#include <cstdint>

namespace sk {

constexpr int kMaxN = 28;        // largest n with a compiled kernel
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
  unsigned long long items;  // number of work items (2^{2n-1-m})
  int m;                     // walk bits per item
  int job;                   // slot index of this job's residues
};

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

// Outer flip of bit J (inner bits all +1 at this point, and +2 in ws).
// ws points at this thread's entry for position 0.
template <int DELTA, int N, int U>
__device__ __forceinline__ void outer_flip(int J, int (&c)[N], int (&near)[near_count(DELTA, N)],
                                           signed char* ws) {
  signed char* wj = ws + J * kWsStride;
  const int sJ = (int)(*wj) >> 1;
#pragma unroll
  for (int k = 1; k <= N; ++k) {
    const int d = k + DELTA;
    const int t = (int)wj[-d * kWsStride] + (int)wj[d * kWsStride];
    c[k - 1] -= sJ * t;
  }
  *wj = (signed char)(-2 * sJ);
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

// ------------------------------------------------------------ exact limb form

// Compile-time bit lengths of the products of the c_k bounds L_k, group by
// group, computed in 32-bit limbs.
struct BoundInfo {
  int bits[kMaxN + 1];   // bit length of prod of bounds of groups 0..j
};
__host__ __device__ constexpr BoundInfo make_bounds(int DELTA, int N) {
  BoundInfo bi{};
  GroupInfo gi = make_groups(DELTA, N);
  unsigned w[8] = {1, 0, 0, 0, 0, 0, 0, 0};
  for (int g = 0; g < gi.g; ++g) {
    for (int k = gi.start[g] + 1; k <= gi.start[g + 1]; ++k) {
      long long L = 2LL * N - k - DELTA;
      if (L < 1) L = 1;
      unsigned long long carry = 0;
      for (int i = 0; i < 8; ++i) {
        unsigned long long t = (unsigned long long)w[i] * (unsigned long long)L + carry;
        w[i] = (unsigned)t;
        carry = t >> 32;
      }
    }
    int top = 7;
    while (top > 0 && w[top] == 0) --top;
    int b = 0;
    while (b < 32 && (w[top] >> b)) ++b;
    bi.bits[g] = top * 32 + b;
  }
  return bi;
}
__host__ __device__ constexpr int limbs_of(int bits) { return bits < 1 ? 1 : (bits + 31) / 32; }
// Headroom of the accumulator for the sum of 2^m terms of one item.
constexpr int kLimbHeadroom = 26;
__host__ __device__ constexpr int acc_limbs(int DELTA, int N) {
  return limbs_of(make_bounds(DELTA, N).bits[make_groups(DELTA, N).g - 1] + 1 + kLimbHeadroom);
}
// Largest walk width m whose item sum fits the accumulator.
__host__ __device__ constexpr int limb_max_walk_bits(int DELTA, int N) {
  return 32 * acc_limbs(DELTA, N) - make_bounds(DELTA, N).bits[make_groups(DELTA, N).g - 1] - 1;
}

// acc += x (AL limbs, x already sign-extended), one carry chain.
template <int AL>
__device__ __forceinline__ void limbs_add(unsigned (&a)[AL], const unsigned (&x)[AL]) {
  if constexpr (AL == 1) {
    a[0] += x[0];
  } else if constexpr (AL == 2) {
    asm("add.cc.u32 %0, %0, %2;\n\taddc.u32 %1, %1, %3;"
        : "+r"(a[0]), "+r"(a[1]) : "r"(x[0]), "r"(x[1]));
  } else if constexpr (AL == 3) {
    asm("add.cc.u32 %0, %0, %3;\n\taddc.cc.u32 %1, %1, %4;\n\taddc.u32 %2, %2, %5;"
        : "+r"(a[0]), "+r"(a[1]), "+r"(a[2]) : "r"(x[0]), "r"(x[1]), "r"(x[2]));
  } else if constexpr (AL == 4) {
    asm("add.cc.u32 %0, %0, %4;\n\taddc.cc.u32 %1, %1, %5;\n\taddc.cc.u32 %2, %2, %6;\n\t"
        "addc.u32 %3, %3, %7;"
        : "+r"(a[0]), "+r"(a[1]), "+r"(a[2]), "+r"(a[3])
        : "r"(x[0]), "r"(x[1]), "r"(x[2]), "r"(x[3]));
  } else if constexpr (AL == 5) {
    asm("add.cc.u32 %0, %0, %5;\n\taddc.cc.u32 %1, %1, %6;\n\taddc.cc.u32 %2, %2, %7;\n\t"
        "addc.cc.u32 %3, %3, %8;\n\taddc.u32 %4, %4, %9;"
        : "+r"(a[0]), "+r"(a[1]), "+r"(a[2]), "+r"(a[3]), "+r"(a[4])
        : "r"(x[0]), "r"(x[1]), "r"(x[2]), "r"(x[3]), "r"(x[4]));
  } else if constexpr (AL == 6) {
    asm("add.cc.u32 %0, %0, %6;\n\taddc.cc.u32 %1, %1, %7;\n\taddc.cc.u32 %2, %2, %8;\n\t"
        "addc.cc.u32 %3, %3, %9;\n\taddc.cc.u32 %4, %4, %10;\n\taddc.u32 %5, %5, %11;"
        : "+r"(a[0]), "+r"(a[1]), "+r"(a[2]), "+r"(a[3]), "+r"(a[4]), "+r"(a[5])
        : "r"(x[0]), "r"(x[1]), "r"(x[2]), "r"(x[3]), "r"(x[4]), "r"(x[5]));
  } else {
    static_assert(AL >= 1 && AL <= 6, "accumulator width");
  }
}

// Accumulator of the exact form: the product of the |group products| as an
// exact unsigned multi-limb integer (only as many limbs as the bounds need),
// added with its sign into an exact two's-complement accumulator: a negative
// term adds ~|t| and counts one in `ones` (-|t| = ~|t| + 1).  The item sum is
// reduced modulo each prime once, at the end of the item.
template <int DELTA, int N>
struct LimbAcc {
  static constexpr int NG = make_groups(DELTA, N).g;
  static constexpr int PL = limbs_of(make_bounds(DELTA, N).bits[NG - 1]);
  static constexpr int AL = acc_limbs(DELTA, N);
  const Primes& P;
  unsigned acc[AL];
  int ones;
  __device__ __forceinline__ explicit LimbAcc(const Primes& P_) : P(P_), ones(0) {
#pragma unroll
    for (int i = 0; i < AL; ++i) acc[i] = 0u;
  }
  template <int S>
  __device__ __forceinline__ void term(const int (&c)[N]) {
    constexpr GroupInfo gi = make_groups(DELTA, N);
    constexpr BoundInfo bi = make_bounds(DELTA, N);
    int G[gi.g];
    group_products<DELTA, N>(c, G);
    // sign of the term: parity of the negative groups, flipped on odd steps
    unsigned sg = (S & 1) ? 0x80000000u : 0u;
#pragma unroll
    for (int g = 0; g < gi.g; ++g) sg ^= (unsigned)G[g];
    const unsigned m = (unsigned)((int)sg >> 31);
    unsigned a[gi.g];
#pragma unroll
    for (int g = 0; g < gi.g; ++g) a[g] = (unsigned)abs(G[g]);
    unsigned p[PL];
    if constexpr (gi.g == 1) {
      p[0] = a[0];
    } else {
      constexpr int L1 = limbs_of(bi.bits[1]);
      const unsigned long long t = (unsigned long long)a[0] * a[1];
      p[0] = (unsigned)t;
      if constexpr (L1 > 1) p[1] = (unsigned)(t >> 32);
#pragma unroll
      for (int g = 2; g < gi.g; ++g) {
        const int lp = limbs_of(bi.bits[g - 1]);      // limbs so far
        const int ln = limbs_of(bi.bits[g]);          // limbs after this factor
        unsigned carry = 0;
#pragma unroll
        for (int i = 0; i < ln; ++i) {
          if (i < lp) {
            if (i == ln - 1) {
              p[i] = p[i] * a[g] + carry;               // top limb: no carry out
            } else {
              const unsigned long long t2 = (unsigned long long)p[i] * a[g] + carry;
              p[i] = (unsigned)t2;
              carry = (unsigned)(t2 >> 32);
            }
          } else {
            p[i] = carry;                                // the new top limb
          }
        }
      }
    }
    unsigned x[AL];
#pragma unroll
    for (int i = 0; i < AL; ++i) x[i] = (i < PL) ? (p[i] ^ m) : m;
    limbs_add<AL>(acc, x);
    ones -= (int)m;
  }
  __device__ __forceinline__ void negate() {
#pragma unroll
    for (int i = 0; i < AL; ++i) acc[i] = ~acc[i];   // -(acc + ones) = ~acc + (1 - ones)
    ones = 1 - ones;
  }
  __device__ __forceinline__ void finish(bool flip, int nprimes,
                                         unsigned long long (&res)[kMaxPrimes]) {
    if (flip) negate();
    unsigned x[AL];
    const unsigned sx = (unsigned)(ones >> 31);
#pragma unroll
    for (int i = 0; i < AL; ++i) x[i] = (i == 0) ? (unsigned)ones : sx;
    limbs_add<AL>(acc, x);
#pragma unroll
    for (int i = 0; i < kMaxPrimes; ++i) {
      if (i >= nprimes) { res[i] = 0; continue; }
      const long long p = P.pr[i].p;
      long long r = (long long)(int)acc[AL - 1] % p;
      if (r < 0) r += p;
      unsigned long long u = (unsigned long long)r;
#pragma unroll
      for (int j = AL - 2; j >= 0; --j)
        u = (unsigned long long)((((unsigned __int128)u << 32) | acc[j]) % (unsigned long long)p);
      res[i] = u;
    }
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
  signed char* ws = ws_col + PAD * kWsStride;
  for (int i = -PAD; i < 2 * N + 1 + PAD; ++i) {
    int v = 0;
    if (i >= 0 && i < 64) {
      const int present = (int)((pres >> i) & 1ULL);
      const int negative = (int)((neg >> i) & 1ULL);
      v = present ? (negative ? -2 : 2) : 0;
    }
    ws[i * kWsStride] = (signed char)v;
  }
  int near[NEAR];
#pragma unroll
  for (int i = 0; i < NEAR; ++i) near[i] = (int)ws[(U + i) * kWsStride];
  // sign of prod x at the first block; every outer flip negates it, which the
  // loop applies by negating the accumulator (see below)
  const int sb0 = (__popcll(neg) & 1) ? -1 : 1;
  const unsigned long long nblocks = 1ULL << (m - U);
  for (unsigned long long b = 0;; ++b) {
    inner_walk<DELTA, N, U, 0>(c, near, A);
    if (b + 1 == nblocks) break;
    inner_update<DELTA, N, U, 0>(c, near);             // inner bits back to +1
    const int J = U + __ffsll((long long)(b + 1)) - 1;
    outer_flip<DELTA, N, U>(J, c, near, ws);
    // block b+1 has the opposite sign of prod x: negate what was summed so far
    // and keep adding with the same signs; the total is fixed once below
    A.negate();
  }
  // A = (-1)^{nblocks-1} * sum_b (-1)^b block_b; wanted: sb0 * sum_b (-1)^b block_b
  const bool flip = (sb0 < 0) != ((nblocks - 1) & 1ULL);
  A.finish(flip, nprimes, res);
}

}  // namespace sk
