// Host check of the exact kernel's per-term digit product for every
// (delta, n) plan the library compiles (n = 1..31, Skolem / hooked and
// Langford distances):
//   * (-1)^NEG prod_k c_k == T * sum_i r_i 2^{31 i}, compared modulo two primes;
//   * every digit below the top lies in [0, 2^31);
//   * the item-sum bound of the plan's accumulators: tail form |T| < 2^tb and
//     31 + tb + max_m <= 63 (64-bit signed words hold 2^max_m terms of
//     |r_i T| < 2^{31 + tb}); digit form max_m <= 31.
// Inputs: every factor at its bound L_k with random signs, and uniform
// random values in [-L_k, L_k].  Prints one line per plan; exit status 1 if
// any check fails.
#include <cstdio>
#include <random>
#include <utility>

#include "sk_exact.cuh"

using namespace sk;

static unsigned long long mod_p(long long x, unsigned long long p) {
  long long y = x % (long long)p;
  return (unsigned long long)(y < 0 ? y + (long long)p : y);
}

template <int D, int N>
int check_plan(std::mt19937_64& rng, int trials) {
  constexpr DigitPlan dp = make_digit_plan(D, N);
  int bad = 0;
  if (dp.tail_form) {
    if (31 + dp.tail_bits + dp.max_m > 63) ++bad;
  } else if (dp.max_m > 31) {
    ++bad;
  }
  const unsigned long long ps[2] = {(1ULL << 61) - 1, 1000000007ULL};
  for (int t = 0; t < trials; ++t) {
    int c[N];
    for (int k = 1; k <= N; ++k) {
      const long long L = factor_bound(D, N, k);
      long long v = (t & 1) ? L : (long long)(rng() % (unsigned long long)(2 * L + 1)) - L;
      if ((t & 1) && (rng() & 1)) v = -v;
      c[k - 1] = (int)v;
    }
    int r[dp.kd];
    int T;
    const bool neg = (t >> 1) & 1;
    if (neg) digit_product<D, N, 1>(c, r, T);
    else     digit_product<D, N, 0>(c, r, T);
    if (dp.tail_form && (T >= (1 << dp.tail_bits) || -T >= (1 << dp.tail_bits))) ++bad;
    for (int i = 0; i + 1 < dp.kd; ++i)
      if (r[i] < 0) ++bad;
    for (unsigned long long p : ps) {
      unsigned long long want = neg ? p - 1 : 1;      // (-1)^NEG
      for (int k = 0; k < N; ++k) want = (unsigned long long)((unsigned __int128)want * mod_p(c[k], p) % p);
      unsigned long long h = 0;
      for (int i = dp.kd - 1; i >= 0; --i)
        h = (unsigned long long)((((unsigned __int128)h << 31) + mod_p(r[i], p)) % p);
      const unsigned long long got = (unsigned long long)((unsigned __int128)h * mod_p(T, p) % p);
      if (got != want) ++bad;
    }
  }
  std::printf("delta=%d n=%2d form=%s groups=%d tail=%d tail_bits=%2d digits=%d max_m=%2d bad=%d\n",
              D, N, dp.tail_form ? "tail " : "digit", dp.ng, dp.ntail, dp.tail_bits, dp.kd,
              dp.max_m, bad);
  return bad;
}

template <int D, int... Ns>
int check_all(std::mt19937_64& rng, std::integer_sequence<int, Ns...>) {
  return (check_plan<D, Ns + 1>(rng, 4000) + ...);
}

int main() {
  std::mt19937_64 rng(1);
  int bad = check_all<0>(rng, std::make_integer_sequence<int, kMaxN>{});
  bad += check_all<1>(rng, std::make_integer_sequence<int, kMaxN>{});
  std::printf("total bad=%d\n", bad);
  return bad ? 1 : 0;
}
