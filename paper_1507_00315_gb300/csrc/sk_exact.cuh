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
  long long p;          // odd, 2^61 < p < 2^62
  int lo;               // signed low limb:  p = hi * 2^32 + lo
  int hi;
  unsigned npinv;       // -p^{-1} mod 2^32
};

struct Primes {
  Prime pr[kMaxPrimes];
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

__host__ __device__ constexpr int inner_bits(int N) { return (2 * N - 1) < 5 ? (2 * N - 1) : 5; }

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
__device__ __forceinline__ long long mont_finish(long long P1, long long AH, const Prime& P) {
  int m = (int)((unsigned)P1 * P.npinv);
  long long X = (long long)m * P.lo + P1;     // divisible by 2^32
  long long r = AH + (X >> 32);
  return r + (long long)m * P.hi;
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

// ------------------------------------------------------------ one term

// Adds (-1)^s * sb * prod_k c_k (mod each prime, times R^{-(g-2)}) into the
// accumulators; ODD selects the subtraction.
template <int DELTA, int N, int NPR, bool ODD>
__device__ __forceinline__ void eval_term(const int (&c)[N], int sb, const Primes& P,
                                          unsigned (&acc)[NPR][3]) {
  constexpr GroupInfo gi = make_groups(DELTA, N);
  int G[gi.g];
#pragma unroll
  for (int g = 0; g < gi.g; ++g) {
    int v = c[gi.start[g]];
#pragma unroll
    for (int k = gi.start[g] + 1; k < gi.start[g + 1]; ++k) v *= c[k];
    G[g] = v;
  }
  G[gi.g - 1] *= sb;                      // the block's sign of prod x
  if constexpr (gi.g == 1) {
#pragma unroll
    for (int i = 0; i < NPR; ++i) {
      if (ODD) acc_sub(acc[i][0], acc[i][1], acc[i][2], (long long)G[0]);
      else     acc_add(acc[i][0], acc[i][1], acc[i][2], (long long)G[0]);
    }
  } else {
    const long long head = (long long)G[0] * G[1];
    if constexpr (gi.g == 2) {
#pragma unroll
      for (int i = 0; i < NPR; ++i) {
        if (ODD) acc_sub(acc[i][0], acc[i][1], acc[i][2], head);
        else     acc_add(acc[i][0], acc[i][1], acc[i][2], head);
      }
    } else {
      int al, ah;
      split_signed(head, al, ah);
      const long long P1 = (long long)al * G[2];
      const long long AH = (long long)ah * G[2];
#pragma unroll
      for (int i = 0; i < NPR; ++i) {
        long long r = mont_finish(P1, AH, P.pr[i]);
#pragma unroll
        for (int g = 3; g < gi.g; ++g) {
          int bl, bh;
          split_signed(r, bl, bh);
          r = mont_finish((long long)bl * G[g], (long long)bh * G[g], P.pr[i]);
        }
        if (ODD) acc_sub(acc[i][0], acc[i][1], acc[i][2], r);
        else     acc_add(acc[i][0], acc[i][1], acc[i][2], r);
      }
    }
  }
}

template <int DELTA, int N, int NPR, int U, int S>
__device__ __forceinline__ void inner_walk(int (&c)[N], const int (&near)[near_count(DELTA, N)],
                                           int sb, const Primes& P, unsigned (&acc)[NPR][3]) {
  if constexpr (S < (1 << U)) {
    if constexpr (S > 0) inner_update<DELTA, N, U, S>(c, near);
#pragma unroll
    for (int k = 0; k < N; ++k) asm volatile("" : "+r"(c[k]));
    eval_term<DELTA, N, NPR, (S & 1) != 0>(c, sb, P, acc);
    inner_walk<DELTA, N, NPR, U, S + 1>(c, near, sb, P, acc);
  }
}

// ------------------------------------------------------------ work item

// Sum over one item: returns the raw residues (times R^{-(g-2)}) in [0, p).
// ws: this thread's column of the shared w array (stride kWsStride).
template <int DELTA, int N, int NPR>
__device__ __forceinline__ void run_item(unsigned long long pres, int m, unsigned long long q,
                                         const Primes& P, signed char* ws_col,
                                         unsigned long long (&res)[NPR]) {
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
  int sb = (__popcll(neg) & 1) ? -1 : 1;
  unsigned acc[NPR][3];
#pragma unroll
  for (int i = 0; i < NPR; ++i) acc[i][0] = acc[i][1] = acc[i][2] = 0u;

  const unsigned long long nblocks = 1ULL << (m - U);
  for (unsigned long long b = 0;; ++b) {
    inner_walk<DELTA, N, NPR, U, 0>(c, near, sb, P, acc);
    if (b + 1 == nblocks) break;
    inner_update<DELTA, N, U, 0>(c, near);             // inner bits back to +1
    const int J = U + __ffsll((long long)(b + 1)) - 1;
    outer_flip<DELTA, N, U>(J, c, near, ws);
    sb = -sb;
  }
#pragma unroll
  for (int i = 0; i < NPR; ++i) res[i] = acc_reduce(acc[i][0], acc[i][1], acc[i][2], P.pr[i].p);
}

}  // namespace sk
