// Host check of the item enumeration of the mirrored walk (Lemma 2.3 on top
// of Lemma 2.2, csrc/sk_mirror.cuh) for every (n, h) with n <= 12:
//   * the decoded items are distinct, and each fixes only bit 0 and the
//     middle bits h+1 .. 2n-2-h;
//   * for every prefix pattern o (x_1 and the middle), with sigma(o) its
//     mirror image -- the middle reversed (x_1 = +1) or reversed and negated
//     (x_1 = -1), computed here bit by bit from the definition -- the
//     weights of the enumerated items in the orbit {o, sigma(o)} add up to the
//     orbit's size, so the weighted item sums equal the sum over all items;
//   * the walk bits are bits 1..h and their mirror images 2n-1-i, disjoint
//     from the fixed bits and from bit 2n-1.
// Prints one line per (n, h); exit status 1 if any check fails.
#include <cstdio>
#include <map>
#include <set>

#include "sk_mirror.cuh"

using namespace sk;

static unsigned long long sigma(int n, int h, unsigned long long o) {
  const bool neg = o & 1ULL;
  unsigned long long r = o & 1ULL;
  for (int b = h + 1; b <= 2 * n - 2 - h; ++b) {
    unsigned long long v = (o >> (2 * n - 1 - b)) & 1ULL;      // the mirror bit's value
    if (neg) v ^= 1ULL;
    r |= v << b;
  }
  return r;
}

int main() {
  int bad_total = 0;
  for (int n = 2; n <= 12; ++n) {
    for (int h = 1; h <= n - 1; ++h) {
      int bad = 0;
      const MirrorShape sh = mirror_shape(n, h);
      unsigned long long fixed_mask = 1ULL;
      for (int b = h + 1; b <= 2 * n - 2 - h; ++b) fixed_mask |= 1ULL << b;
      std::set<unsigned long long> seen;
      std::map<unsigned long long, int> wsum;
      for (unsigned long long q = 0; q < 2 * sh.per_side; ++q) {
        int w = 0;
        const unsigned long long o = mirror_item_bits(sh, q, &w);
        if (o & ~fixed_mask) ++bad;
        if (!seen.insert(o).second) ++bad;
        if (w != 1 && w != 2) ++bad;
        const unsigned long long s = sigma(n, h, o);
        wsum[o < s ? o : s] += w;
      }
      // every orbit of the 2^{1 + middle} patterns
      const int L = 2 * n - 2 - 2 * h;
      for (unsigned long long x = 0; x < (1ULL << (1 + L)); ++x) {
        const unsigned long long o = (x & 1ULL) | ((x >> 1) << (h + 1));
        const unsigned long long s = sigma(n, h, o);
        if (sigma(n, h, s) != o) ++bad;                          // an involution
        const int size = (s == o) ? 1 : 2;
        const auto it = wsum.find(o < s ? o : s);
        if (it == wsum.end() || it->second != size) ++bad;
      }
      std::set<int> walk;
      for (int t = 0; t < 2 * h; ++t) {
        const int b = mirror_walk_bit(n, h, t);
        if (b < 1 || b > 2 * n - 2 || ((fixed_mask >> b) & 1ULL)) ++bad;
        walk.insert(b);
      }
      for (int b : walk)
        if (!walk.count(2 * n - 1 - b)) ++bad;                    // closed under the mirror
      if ((int)walk.size() != 2 * h) ++bad;
      std::printf("n=%d h=%d items=%llu of %llu bad=%d\n", n, h, 2 * sh.per_side,
                  1ULL << (1 + L), bad);
      bad_total += bad;
    }
  }
  std::printf("total bad=%d\n", bad_total);
  return bad_total ? 1 : 0;
}
