// sk_host_exact.cu -- host runtime of the exact count: work planning (Sec.
// 2.2: power-of-two splits of the assignments), launches, checkpointed
// chunks, and the C ABI entry points skolem_count / skolem_count_ex /
// skolem_item_residues, and the same runtime for the inclusion-exclusion
// count (Sec. 2, third approach): sk_count_inclusion_exclusion /
// sk_ie_item_residues.
#include <algorithm>
#include <chrono>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <unistd.h>
#include <vector>

#include "sk_exact_launch.cuh"
#include "sk_host_common.h"
#include "sk_ie.cuh"
#include "sk_mirror.cuh"

namespace sk {

// ------------------------------------------------------------ launcher table

#define SK_EXTERN_EXACT(N)                                                         \
  extern template cudaError_t launch_exact<0, N, 3>(const ExactLaunch&);          \
  extern template cudaError_t launch_exact<1, N, 3>(const ExactLaunch&);
SK_EXTERN_EXACT(1) SK_EXTERN_EXACT(2) SK_EXTERN_EXACT(3) SK_EXTERN_EXACT(4) SK_EXTERN_EXACT(5)
SK_EXTERN_EXACT(6) SK_EXTERN_EXACT(7) SK_EXTERN_EXACT(8) SK_EXTERN_EXACT(9) SK_EXTERN_EXACT(10)
SK_EXTERN_EXACT(11) SK_EXTERN_EXACT(12) SK_EXTERN_EXACT(13) SK_EXTERN_EXACT(14)
SK_EXTERN_EXACT(15) SK_EXTERN_EXACT(16) SK_EXTERN_EXACT(17) SK_EXTERN_EXACT(18)
SK_EXTERN_EXACT(19) SK_EXTERN_EXACT(20) SK_EXTERN_EXACT(21) SK_EXTERN_EXACT(22)
SK_EXTERN_EXACT(23) SK_EXTERN_EXACT(24) SK_EXTERN_EXACT(25) SK_EXTERN_EXACT(26)
SK_EXTERN_EXACT(27) SK_EXTERN_EXACT(28)
SK_EXTERN_EXACT(29) SK_EXTERN_EXACT(30) SK_EXTERN_EXACT(31)
#undef SK_EXTERN_EXACT

#define SK_EXTERN_LIMB(N)                                                          \
  extern template cudaError_t launch_limb<0, N>(const ExactLaunch&);                \
  extern template cudaError_t launch_limb<1, N>(const ExactLaunch&);
SK_EXTERN_LIMB(1) SK_EXTERN_LIMB(2) SK_EXTERN_LIMB(3) SK_EXTERN_LIMB(4) SK_EXTERN_LIMB(5)
SK_EXTERN_LIMB(6) SK_EXTERN_LIMB(7) SK_EXTERN_LIMB(8) SK_EXTERN_LIMB(9) SK_EXTERN_LIMB(10)
SK_EXTERN_LIMB(11) SK_EXTERN_LIMB(12) SK_EXTERN_LIMB(13) SK_EXTERN_LIMB(14)
SK_EXTERN_LIMB(15) SK_EXTERN_LIMB(16) SK_EXTERN_LIMB(17) SK_EXTERN_LIMB(18)
SK_EXTERN_LIMB(19) SK_EXTERN_LIMB(20) SK_EXTERN_LIMB(21) SK_EXTERN_LIMB(22)
SK_EXTERN_LIMB(23) SK_EXTERN_LIMB(24) SK_EXTERN_LIMB(25) SK_EXTERN_LIMB(26)
SK_EXTERN_LIMB(27) SK_EXTERN_LIMB(28)
SK_EXTERN_LIMB(29) SK_EXTERN_LIMB(30) SK_EXTERN_LIMB(31)
#undef SK_EXTERN_LIMB

#define SK_ROW(N) {launch_exact<0, N, 3>, launch_exact<1, N, 3>}
static const ExactLaunchFn kTable[kMaxN + 1][2] = {
    {nullptr, nullptr},
    SK_ROW(1), SK_ROW(2), SK_ROW(3), SK_ROW(4), SK_ROW(5), SK_ROW(6), SK_ROW(7),
    SK_ROW(8), SK_ROW(9), SK_ROW(10), SK_ROW(11), SK_ROW(12), SK_ROW(13), SK_ROW(14),
    SK_ROW(15), SK_ROW(16), SK_ROW(17), SK_ROW(18), SK_ROW(19), SK_ROW(20), SK_ROW(21),
    SK_ROW(22), SK_ROW(23), SK_ROW(24), SK_ROW(25), SK_ROW(26), SK_ROW(27), SK_ROW(28),
    SK_ROW(29), SK_ROW(30), SK_ROW(31)};
#undef SK_ROW

ExactLaunchFn exact_launcher(int delta, int n, int nprimes) {
  if (delta < 0 || delta > 1 || n < 1 || n > kMaxN || nprimes != 3) return nullptr;
  return kTable[n][delta];
}

#define SK_LROW(N) {launch_limb<0, N>, launch_limb<1, N>}
static const ExactLaunchFn kLimbTable[kMaxN + 1][2] = {
    {nullptr, nullptr},
    SK_LROW(1), SK_LROW(2), SK_LROW(3), SK_LROW(4), SK_LROW(5), SK_LROW(6), SK_LROW(7),
    SK_LROW(8), SK_LROW(9), SK_LROW(10), SK_LROW(11), SK_LROW(12), SK_LROW(13), SK_LROW(14),
    SK_LROW(15), SK_LROW(16), SK_LROW(17), SK_LROW(18), SK_LROW(19), SK_LROW(20), SK_LROW(21),
    SK_LROW(22), SK_LROW(23), SK_LROW(24), SK_LROW(25), SK_LROW(26), SK_LROW(27), SK_LROW(28),
    SK_LROW(29), SK_LROW(30), SK_LROW(31)};
#undef SK_LROW

ExactLaunchFn limb_launcher(int delta, int n) {
  if (delta < 0 || delta > 1 || n < 1 || n > kMaxN) return nullptr;
  return kLimbTable[n][delta];
}

#define SK_EXTERN_IE(N)                                                            \
  extern template cudaError_t launch_ie<0, N>(const ExactLaunch&);                  \
  extern template cudaError_t launch_ie<1, N>(const ExactLaunch&);
SK_EXTERN_IE(1) SK_EXTERN_IE(2) SK_EXTERN_IE(3) SK_EXTERN_IE(4) SK_EXTERN_IE(5) SK_EXTERN_IE(6)
SK_EXTERN_IE(7) SK_EXTERN_IE(8) SK_EXTERN_IE(9) SK_EXTERN_IE(10) SK_EXTERN_IE(11) SK_EXTERN_IE(12)
SK_EXTERN_IE(13) SK_EXTERN_IE(14) SK_EXTERN_IE(15) SK_EXTERN_IE(16) SK_EXTERN_IE(17)
SK_EXTERN_IE(18) SK_EXTERN_IE(19) SK_EXTERN_IE(20) SK_EXTERN_IE(21) SK_EXTERN_IE(22)
SK_EXTERN_IE(23) SK_EXTERN_IE(24)
#undef SK_EXTERN_IE

#define SK_IROW(N) {launch_ie<0, N>, launch_ie<1, N>}
static const ExactLaunchFn kIeTable[kMaxIeN + 1][2] = {
    {nullptr, nullptr},
    SK_IROW(1), SK_IROW(2), SK_IROW(3), SK_IROW(4), SK_IROW(5), SK_IROW(6), SK_IROW(7),
    SK_IROW(8), SK_IROW(9), SK_IROW(10), SK_IROW(11), SK_IROW(12), SK_IROW(13), SK_IROW(14),
    SK_IROW(15), SK_IROW(16), SK_IROW(17), SK_IROW(18), SK_IROW(19), SK_IROW(20), SK_IROW(21),
    SK_IROW(22), SK_IROW(23), SK_IROW(24)};
#undef SK_IROW
static_assert(kMaxIeN == 24, "the table above lists n = 1..kMaxIeN");

ExactLaunchFn ie_launcher(int delta, int n) {
  if (delta < 0 || delta > 1 || n < 1 || n > kMaxIeN) return nullptr;
  return kIeTable[n][delta];
}

#define SK_EXTERN_MIRROR(N)                                                        \
  extern template cudaError_t launch_mirror<0, N>(const ExactLaunch&);              \
  extern template cudaError_t launch_mirror<1, N>(const ExactLaunch&);
SK_EXTERN_MIRROR(6) SK_EXTERN_MIRROR(7) SK_EXTERN_MIRROR(8) SK_EXTERN_MIRROR(9)
SK_EXTERN_MIRROR(10) SK_EXTERN_MIRROR(11) SK_EXTERN_MIRROR(12) SK_EXTERN_MIRROR(13)
SK_EXTERN_MIRROR(14) SK_EXTERN_MIRROR(15) SK_EXTERN_MIRROR(16) SK_EXTERN_MIRROR(17)
SK_EXTERN_MIRROR(18) SK_EXTERN_MIRROR(19) SK_EXTERN_MIRROR(20) SK_EXTERN_MIRROR(21)
SK_EXTERN_MIRROR(22) SK_EXTERN_MIRROR(23) SK_EXTERN_MIRROR(24) SK_EXTERN_MIRROR(25)
SK_EXTERN_MIRROR(26) SK_EXTERN_MIRROR(27) SK_EXTERN_MIRROR(28) SK_EXTERN_MIRROR(29)
SK_EXTERN_MIRROR(30) SK_EXTERN_MIRROR(31)
#undef SK_EXTERN_MIRROR

#define SK_MROW(N) {launch_mirror<0, N>, launch_mirror<1, N>}
static const ExactLaunchFn kMirrorTable[kMaxN + 1][2] = {
    {nullptr, nullptr}, {nullptr, nullptr}, {nullptr, nullptr}, {nullptr, nullptr},
    {nullptr, nullptr}, {nullptr, nullptr},
    SK_MROW(6), SK_MROW(7), SK_MROW(8), SK_MROW(9), SK_MROW(10), SK_MROW(11), SK_MROW(12),
    SK_MROW(13), SK_MROW(14), SK_MROW(15), SK_MROW(16), SK_MROW(17), SK_MROW(18), SK_MROW(19),
    SK_MROW(20), SK_MROW(21), SK_MROW(22), SK_MROW(23), SK_MROW(24), SK_MROW(25), SK_MROW(26),
    SK_MROW(27), SK_MROW(28), SK_MROW(29), SK_MROW(30), SK_MROW(31)};
#undef SK_MROW
static_assert(kMirrorMinN == 6 && kMaxN == 31, "the table above lists n = 6..31");

ExactLaunchFn mirror_launcher(int delta, int n) {
  if (delta < 0 || delta > 1 || n < kMirrorMinN || n > kMaxN) return nullptr;
  return kMirrorTable[n][delta];
}

// Largest walk width of the exact form (compile-time table per (delta, n)).
template <int D, int N>
struct LimbMaxM { static constexpr int v = limb_max_walk_bits(D, N); };
#define SK_LM(N) {LimbMaxM<0, N>::v, LimbMaxM<1, N>::v}
static const int kLimbMaxM[kMaxN + 1][2] = {
    {0, 0}, SK_LM(1), SK_LM(2), SK_LM(3), SK_LM(4), SK_LM(5), SK_LM(6), SK_LM(7), SK_LM(8),
    SK_LM(9), SK_LM(10), SK_LM(11), SK_LM(12), SK_LM(13), SK_LM(14), SK_LM(15), SK_LM(16),
    SK_LM(17), SK_LM(18), SK_LM(19), SK_LM(20), SK_LM(21), SK_LM(22), SK_LM(23), SK_LM(24),
    SK_LM(25), SK_LM(26), SK_LM(27), SK_LM(28), SK_LM(29), SK_LM(30), SK_LM(31)};
#undef SK_LM

// ------------------------------------------------------------ planning

// Position set of Sec. 1.1 / 1.2 as a bit mask (bit i = position i+1).
unsigned long long position_mask(int variant, int n) {
  if (variant == SK_HOOKED) {
    unsigned long long all = (n >= 32) ? ~0ULL : ((1ULL << (2 * n + 1)) - 1);
    return all & ~(1ULL << (2 * n - 1));
  }
  return (1ULL << (2 * n)) - 1;
}

int default_walk_bits(int n) {
  const int F = 2 * n - 1;
  const int U = inner_bits(n);
  // aim at 2^22 items (2^24 for the largest orders) so a persistent grid of
  // ~80k threads gets dozens of items each and the tail stays short
  int m = F - (n >= 22 ? 24 : 22);
  if (m < U + 4) m = U + 4;
  if (m > F) m = F;
  if (m < U) m = U;
  return m;
}

// What an exact count sums: Lemma 2.1's signed sum over the +-1 assignments
// (after Lemma 2.2), or the inclusion-exclusion sum over the sets of
// positions (Sec. 2, third approach; every one of the 2n variables free).
enum { kMethodAlgebraic = 0, kMethodInclusionExclusion = 1 };

struct Plan {
  int method;
  int variant, n, delta, m, U, nprimes, block_threads, grid, arith;
  int symmetry;     // SK_SYMMETRY_* used
  int sign;         // Lemma 2.4 sign s (+1 / -1) when symmetry uses it
  int fixed_bit;    // free bit held at +1 by Lemma 2.4, or an extended
                    // sequence's hole (0: none); item indices skip it
  int hole;         // extended Skolem sequences: the hole position (0: none)
  unsigned long long pres, items;
  uint64_t primes[kMaxPrimes];
  Primes P;
  ExactLaunchFn fn;
};

static int make_plan(int variant, int n, const sk_count_opts* o, Plan* pl,
                     int method = kMethodAlgebraic, int hole = 0) {
  if (variant < SK_SKOLEM || variant > SK_HOOKED || n < 1 || n > kMaxN) return SK_EINVAL;
  // Extended Skolem sequences (Sec. 1.2; one hole in 1..2n+1, d_k = k):
  // holes 1 and 2n+1 leave the Skolem problem, 2 and 2n the hooked one.  Any
  // other hole is mirrored into the upper half (reversal maps the sequences
  // of hole h onto those of hole 2n+2-h), left out of the position mask, and
  // skipped by the item index like Lemma 2.4's fixed variable -- so it must
  // lie above the walk (bit >= walk width >= the unrolled inner width).
  int hole_bit = -1;
  if (hole) {
    if (method != kMethodAlgebraic || variant != SK_SKOLEM || hole < 1 || hole > 2 * n + 1)
      return SK_EINVAL;
    if (o && o->symmetry != SK_SYMMETRY_NEGATION) return SK_EINVAL;
    if (hole == 2 || hole == 2 * n) {
      variant = SK_HOOKED;
    } else if (hole != 1 && hole != 2 * n + 1) {
      variant = SK_HOOKED;                     // d_k = k over the span 1..2n+1
      hole_bit = std::max(hole, 2 * n + 2 - hole) - 1;
    }
  }
  std::memset(pl, 0, sizeof(*pl));
  pl->method = method;
  pl->hole = hole;
  if (method == kMethodInclusionExclusion) {
    // the same walk over all 2n variables of P: no symmetry, exact-digit form
    if (n > kMaxIeN) return SK_EINVAL;
    if (o && (o->arith != SK_ARITH_LIMBS || o->symmetry != SK_SYMMETRY_NEGATION)) return SK_EINVAL;
  } else if (method != kMethodAlgebraic) {
    return SK_EINVAL;
  }
  pl->variant = variant;
  pl->n = n;
  pl->delta = (variant == SK_LANGFORD) ? 1 : 0;
  int st = prepare_primes(o, &pl->nprimes, pl->primes, &pl->P);
  if (st) return st;
  const int F = 2 * n - 1;
  pl->arith = o ? o->arith : SK_ARITH_LIMBS;
  if (pl->arith != SK_ARITH_LIMBS && pl->arith != SK_ARITH_MONTGOMERY) return SK_EINVAL;
  pl->U = inner_bits(n);
  const int mmax = pl->arith == SK_ARITH_LIMBS ? kLimbMaxM[n][pl->delta] : F;
  if (o && o->walk_bits) {
    pl->m = o->walk_bits;
  } else {
    pl->m = default_walk_bits(n);
    if (pl->m > mmax) pl->m = mmax;
  }
  pl->pres = position_mask(variant, n);
  if (hole_bit >= 0) pl->pres = ((1ULL << (2 * n + 1)) - 1ULL) & ~(1ULL << hole_bit);
  // Lemma 2.4: negating the even positions multiplies the summand by
  // s = (-1)^{#even positions in P + #odd d_k}.  With s = +1 the summand is
  // constant on {X, X with the odd (Skolem, Langford) or even (hooked; its
  // fixed position 2n+1 is odd) positions negated}, so one more free
  // variable -- the highest of that parity -- is held at +1 and the sum
  // doubled; with s = -1 the sum is 0.
  const int sym = o ? o->symmetry : SK_SYMMETRY_NEGATION;
  if (sym != SK_SYMMETRY_NEGATION && sym != SK_SYMMETRY_NEGATION_EVEN &&
      sym != SK_SYMMETRY_REVERSAL && sym != SK_SYMMETRY_REVERSAL_EVEN)
    return SK_EINVAL;
  const bool reversal = sym == SK_SYMMETRY_REVERSAL || sym == SK_SYMMETRY_REVERSAL_EVEN;
  if (reversal && (variant == SK_HOOKED || pl->arith != SK_ARITH_LIMBS))
    return SK_EINVAL;                     // hooked Skolem's P is not reversal-symmetric
  pl->symmetry = SK_SYMMETRY_NEGATION;
  pl->sign = 1;
  pl->fixed_bit = 0;
  int Feff = F;
  // Lemmas 2.3 and 2.4 together need the mirrored walk (n >= kMirrorMinN);
  // below it, Lemma 2.4 alone
  const bool even_only = sym == SK_SYMMETRY_NEGATION_EVEN ||
                         (sym == SK_SYMMETRY_REVERSAL_EVEN && n < kMirrorMinN);
  if (sym == SK_SYMMETRY_REVERSAL_EVEN && n >= kMirrorMinN) {
    // the sign of Lemma 2.4 decides the zero classes; the mirrored items
    // below carry the rest
    int e = 0, odd_d = 0;
    for (int i = 0; i < 64; ++i)
      if (((pl->pres >> i) & 1ULL) && (i & 1)) ++e;
    for (int k = 1; k <= n; ++k) odd_d += (k + pl->delta) & 1;
    pl->sign = ((e + odd_d) & 1) ? -1 : 1;
  }
  if (even_only && n >= 4) {
    int e = 0, odd_d = 0;
    for (int i = 0; i < 64; ++i)
      if (((pl->pres >> i) & 1ULL) && (i & 1)) ++e;     // bit i = position i+1
    for (int k = 1; k <= n; ++k) odd_d += (k + pl->delta) & 1;
    pl->symmetry = SK_SYMMETRY_NEGATION_EVEN;
    pl->sign = ((e + odd_d) & 1) ? -1 : 1;
    pl->fixed_bit = (variant == SK_HOOKED) ? 2 * n - 3 : 2 * n - 2;
    Feff = F - 1;
    if (!(o && o->walk_bits) && pl->m > pl->fixed_bit) pl->m = pl->fixed_bit;
    if (pl->m > pl->fixed_bit) return SK_EINVAL;        // the fixed bit must lie above the walk
  }
  if (hole_bit >= 0) {
    pl->fixed_bit = hole_bit;
    if (!(o && o->walk_bits) && pl->m > hole_bit) pl->m = hole_bit;
    if (pl->m > hole_bit) return SK_EINVAL;             // the hole must lie above the walk
  }
  if (pl->m < pl->U || pl->m > F || pl->m > mmax || F - pl->m > 56) return SK_EINVAL;
  if (method == kMethodInclusionExclusion) Feff = F + 1;   // max P is a variable too
  pl->items = 1ULL << (Feff - pl->m);
  // Lemma 2.3 (reversal): the mirrored walk over bits 1..h and their mirror
  // images, items = x_1 and the middle bits, one of each pair of mirror-image
  // items enumerated with weight 2 (sk_mirror.cuh)
  if (reversal && n >= kMirrorMinN) {
    int m = pl->m;
    if (!(o && o->walk_bits)) {
      const int cap = std::min(mmax, 2 * n - 2) & ~1;
      m = (m + 1) & ~1;
      if (m > cap) m = cap;
      if (m < 2 * pl->U) m = 2 * pl->U;
    }
    if ((m & 1) || m / 2 < pl->U || m > 2 * n - 2 || m > mmax) return SK_EINVAL;
    pl->m = m;
    pl->symmetry = sym;
    // Lemma 2.4 in the existence classes: negating the odd positions keeps
    // the summand, flips x_1 and keeps x_2n, and maps the mirrored walk's
    // positions onto themselves, so it carries every item with x_1 = +1
    // onto one with x_1 = -1 of equal sum: the x_1 = +1 side alone (items
    // 0 .. per_side-1), doubled on the host
    const unsigned long long per_side = mirror_shape(n, m / 2).per_side;
    pl->items = sym == SK_SYMMETRY_REVERSAL_EVEN ? per_side : 2 * per_side;
  }
  pl->block_threads = (o && o->block_threads) ? o->block_threads : 256;
  if (pl->block_threads < 32 || pl->block_threads > 256 || (pl->block_threads & 31)) return SK_EINVAL;
  pl->grid = (o && o->grid > 0) ? o->grid : 0;
  const bool mirrored =
      pl->symmetry == SK_SYMMETRY_REVERSAL || pl->symmetry == SK_SYMMETRY_REVERSAL_EVEN;
  pl->fn = method == kMethodInclusionExclusion     ? ie_launcher(pl->delta, n)
           : mirrored                              ? mirror_launcher(pl->delta, n)
           : pl->arith == SK_ARITH_LIMBS          ? limb_launcher(pl->delta, n)
                                                  : exact_launcher(pl->delta, n, pl->nprimes);
  if (!pl->fn) return SK_EINVAL;
  return SK_OK;
}

// Multiplies raw residues of the Montgomery form by R^{e}, e = groups - 2,
// removing the factor every term carries (the exact form has none).
static void unmont(const Plan& pl, uint64_t* res) {
  if (pl.arith != SK_ARITH_MONTGOMERY) return;
  GroupInfo gi = make_groups(pl.delta, pl.n);
  int e = gi.g > 2 ? gi.g - 2 : 0;
  for (int i = 0; i < pl.nprimes; ++i) {
    uint64_t R = ((u128)1 << 32) % pl.primes[i];
    res[i] = mulmod(res[i] % pl.primes[i], powmod(R, (uint64_t)e, pl.primes[i]), pl.primes[i]);
  }
}

// One launch over items [lo, hi): raw residues into res (host).
static int run_chunk(const Plan& pl, unsigned long long lo, unsigned long long hi,
                     ExactScratch* dscr, cudaStream_t st, cudaEvent_t e0, cudaEvent_t e1,
                     uint64_t* res, double* kernel_ms, unsigned long long* item_res,
                     int* grid_used) {
  cudaError_t e = cudaMemsetAsync(dscr, 0, sizeof(ExactScratch), st);
  if (e != cudaSuccess) return cuda_status(e);
  ExactLaunch L;
  L.job.pres = pl.pres;
  L.job.items = pl.items;
  L.job.m = pl.m;
  L.job.job = 0;
  L.job.fixed_bit = pl.fixed_bit;
  L.P = pl.P;
  L.nprimes = pl.nprimes;
  L.item_lo = lo;
  L.item_hi = hi;
  L.scratch = dscr;
  L.item_res = item_res;
  L.block_threads = pl.block_threads;
  L.grid = pl.grid;
  L.stream = st;
  cudaEventRecord(e0, st);
  e = pl.fn(L);
  if (e != cudaSuccess) return cuda_status(e);
  cudaEventRecord(e1, st);
  ExactScratch h;
  e = cudaMemcpyAsync(&h, dscr, sizeof(h), cudaMemcpyDeviceToHost, st);
  if (e != cudaSuccess) return cuda_status(e);
  e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_status(e);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  *kernel_ms += ms;
  if (h.err) return SK_ETIMEOUT;
  for (int i = 0; i < pl.nprimes; ++i) res[i] = h.res[i];
  if (grid_used) *grid_used = pl.grid;
  return SK_OK;
}

// ------------------------------------------------------------ checkpoint

struct Ckpt {
  std::string path;
  std::string header;
  std::vector<int> have;                 // per chunk: 1 if done
  std::vector<uint64_t> res;             // per chunk: nprimes residues
};

static std::string ckpt_header(const Plan& pl, unsigned long long chunk_items,
                               unsigned long long nchunks) {
  char buf[512];
  // the arithmetic form is not part of the job: both give the same residues
  std::snprintf(buf, sizeof(buf), "SKCKPT1 v=%d n=%d m=%d k=%d p=%llu,%llu,%llu,%llu items=%llu chunk=%llu chunks=%llu",
                pl.variant, pl.n, pl.m, pl.nprimes, (unsigned long long)pl.primes[0],
                (unsigned long long)pl.primes[1], (unsigned long long)pl.primes[2],
                (unsigned long long)(pl.nprimes > 3 ? pl.primes[3] : 0), pl.items, chunk_items,
                nchunks);
  std::string h(buf);
  if (pl.symmetry == SK_SYMMETRY_NEGATION_EVEN) h += " s=lemma2.4";
  if (pl.symmetry == SK_SYMMETRY_REVERSAL) h += " s=lemma2.3";
  if (pl.symmetry == SK_SYMMETRY_REVERSAL_EVEN) h += " s=lemma2.3+2.4";
  if (pl.method == kMethodInclusionExclusion) h += " method=inclusion-exclusion";
  if (pl.hole) h += " hole=" + std::to_string(pl.hole);
  return h;
}

// Reads an existing checkpoint; a missing file is an empty checkpoint.  A
// final line without its newline is a torn write and is ignored.
static int ckpt_load(Ckpt* ck, const Plan& pl) {
  FILE* f = std::fopen(ck->path.c_str(), "rb");
  if (!f) return SK_OK;
  std::string all;
  char buf[4096];
  size_t r;
  while ((r = std::fread(buf, 1, sizeof(buf), f)) > 0) all.append(buf, r);
  std::fclose(f);
  size_t pos = 0;
  bool first = true;
  while (pos < all.size()) {
    size_t nl = all.find('\n', pos);
    if (nl == std::string::npos) {        // torn tail: cut it off so the next
      if (truncate(ck->path.c_str(), (off_t)pos) != 0) return SK_ECKPT;  // append starts clean
      break;
    }
    std::string line = all.substr(pos, nl - pos);
    pos = nl + 1;
    if (first) {
      if (line != ck->header) return SK_ECKPT;
      first = false;
      continue;
    }
    unsigned long long idx = 0, v[4] = {0, 0, 0, 0};
    unsigned crc = 0;
    int got = std::sscanf(line.c_str(), "chunk %llu %llu %llu %llu %llu crc=%x", &idx, &v[0], &v[1],
                          &v[2], &v[3], &crc);
    if (got != 6) return SK_ECKPT;
    size_t cpos = line.find(" crc=");
    if (cpos == std::string::npos || crc32(line.data(), cpos) != crc) return SK_ECKPT;
    if (idx >= ck->have.size()) return SK_ECKPT;
    for (int i = 0; i < pl.nprimes; ++i)
      if (v[i] >= pl.primes[i]) return SK_ECKPT;
    if (ck->have[idx]) {
      for (int i = 0; i < pl.nprimes; ++i)
        if (ck->res[idx * pl.nprimes + i] != v[i]) return SK_ECKPT;
    }
    ck->have[idx] = 1;
    for (int i = 0; i < pl.nprimes; ++i) ck->res[idx * pl.nprimes + i] = v[i];
  }
  return SK_OK;
}

static int ckpt_append(const Ckpt& ck, bool write_header, unsigned long long idx,
                       const uint64_t* v, int k) {
  FILE* f = std::fopen(ck.path.c_str(), "ab");
  if (!f) return SK_ECKPT;
  char line[512];
  int len = std::snprintf(line, sizeof(line), "chunk %llu %llu %llu %llu %llu", idx,
                          (unsigned long long)v[0], (unsigned long long)v[1],
                          (unsigned long long)v[2], (unsigned long long)(k > 3 ? v[3] : 0));
  uint32_t crc = crc32(line, (size_t)len);
  int ok = 1;
  if (write_header) ok &= std::fprintf(f, "%s\n", ck.header.c_str()) > 0;
  ok &= std::fprintf(f, "%s crc=%08x\n", line, crc) > 0;
  ok &= std::fflush(f) == 0;
  ok &= fsync(fileno(f)) == 0;
  std::fclose(f);
  return ok ? SK_OK : SK_ECKPT;
}

// ------------------------------------------------------------ count

static void u128_half(sk_u128* v) {
  v->lo = (v->lo >> 1) | (v->hi << 63);
  v->hi >>= 1;
}

int limb_max_m(int delta, int n) {
  if (delta < 0 || delta > 1 || n < 1 || n > kMaxN) return 0;
  return kLimbMaxM[n][delta];
}

// Work items per launch: all of them without a checkpoint; with one, about
// 2^37 terms per launch but at least 2^22 items, so that each of the ~80k
// resident threads gets dozens of items and the last wave of a launch stays
// short; opts->chunk_items overrides.  At most the job's items.
static unsigned long long plan_chunk_items(const Plan& pl, const sk_count_opts* o, bool ckpt_on) {
  unsigned long long chunk = (o && o->chunk_items) ? o->chunk_items : 0;
  if (!chunk) {
    if (ckpt_on) {
      int lg = 37 - pl.m;
      if (lg < 22) lg = 22;
      chunk = lg >= 40 ? pl.items : (1ULL << lg);
    } else {
      chunk = pl.items;
    }
  }
  if (chunk > pl.items) chunk = pl.items;
  return chunk;
}

// The plan of skolem_count_ex without running it (host only): the fields of
// the report that do not depend on the sums.
static int plan_report(int variant, int n, const sk_count_opts* o, sk_count_report* rep) {
  if (!rep) return SK_EINVAL;
  Plan pl;
  int st = make_plan(variant, n, o, &pl);
  if (st) return st;
  if (o && o->convention != SK_COUNT_REFLECTIONS_IDENTIFIED && o->convention != SK_COUNT_ALL)
    return SK_EINVAL;
  std::memset(rep, 0, sizeof(*rep));
  rep->nprimes = pl.nprimes;
  for (int i = 0; i < pl.nprimes; ++i) rep->primes[i] = pl.primes[i];
  rep->walk_bits = pl.m;
  rep->inner_bits = pl.U;
  rep->arith = pl.arith;
  rep->block_threads = pl.block_threads;
  rep->grid = pl.grid;
  rep->symmetry = pl.symmetry;
  if (pl.sign < 0) {                      // a zero class of Lemma 2.4: nothing to evaluate
    rep->complete = 1;
    return SK_OK;
  }
  const bool ckpt_on = o && o->checkpoint_path && o->checkpoint_path[0];
  const unsigned long long chunk = plan_chunk_items(pl, o, ckpt_on);
  rep->items = pl.items;
  rep->terms = pl.items << pl.m;
  rep->chunks_total = (pl.items + chunk - 1) / chunk;
  return SK_OK;
}

// Output convention of a coefficient C (pairings, reflections distinct).
// Sec. 1.3: no sequence of order n > 1 is its own reflection; the single
// Skolem sequence of order 1 (1,1) is.
int apply_convention(int variant, int n, int convention, sk_u128 coeff, sk_u128* out) {
  sk_u128 v = coeff;
  if (convention == SK_COUNT_REFLECTIONS_IDENTIFIED && variant != SK_HOOKED) {
    if (variant == SK_SKOLEM && n == 1) {
      v.lo += 1;
    } else if (v.lo & 1) {
      return SK_EMISMATCH;
    }
    u128_half(&v);
  }
  *out = v;
  return SK_OK;
}

// CRT, checks and output convention of one job from its residues H mod p_i.
int finalize_count(int variant, int n, int convention, int nprimes, const uint64_t* primes,
                   const uint64_t* H, sk_u128* out) {
  sk_u128 coeff = {0, 0};
  int st = crt_coefficient(n, nprimes, primes, H, &coeff);
  if (st) return st;
  return apply_convention(variant, n, convention, coeff, out);
}

// Output convention of an extended sequence count: reversal maps hole h to
// hole 2n+2-h, so reflections are identified only where it maps the position
// set onto itself -- holes 1 and 2n+1 (the Skolem problem) and n+1 (Rosa's:
// no sequence is its own reflection, the pair of 1s cannot be symmetric about
// n+1) -- and the count of any other hole is returned as it is.
static int apply_convention_hole(int n, int hole, int convention, sk_u128 coeff, sk_u128* out) {
  if (hole == 1 || hole == 2 * n + 1) return apply_convention(SK_SKOLEM, n, convention, coeff, out);
  if (hole == n + 1 && convention == SK_COUNT_REFLECTIONS_IDENTIFIED) {
    if (coeff.lo & 1) return SK_EMISMATCH;
    u128_half(&coeff);
  }
  *out = coeff;
  return SK_OK;
}

int count_impl(int variant, int n, const sk_count_opts* o, sk_u128* out, sk_count_report* rep,
               int method = kMethodAlgebraic, int hole = 0) {
  auto t0 = std::chrono::steady_clock::now();
  Plan pl;
  int st = make_plan(variant, n, o, &pl, method, hole);
  if (st) return st;
  if (o && o->convention != SK_COUNT_REFLECTIONS_IDENTIFIED && o->convention != SK_COUNT_ALL)
    return SK_EINVAL;
  st = check_device();
  if (st) return st;
  if (pl.sign < 0) {
    // Lemma 2.4 with s = -1: the sum is 0 (a zero class); nothing to evaluate
    if (rep) {
      std::memset(rep, 0, sizeof(*rep));
      rep->nprimes = pl.nprimes;
      for (int i = 0; i < pl.nprimes; ++i) rep->primes[i] = pl.primes[i];
      rep->walk_bits = pl.m;
      rep->inner_bits = pl.U;
      rep->arith = pl.arith;
      rep->block_threads = pl.block_threads;
      rep->grid = pl.grid;
      rep->complete = 1;
      rep->symmetry = pl.symmetry;
      rep->wall_ms =
          std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    }
    if (out) *out = sk_u128{0, 0};
    return SK_OK;
  }
  cudaStream_t stream = (o && o->stream) ? (cudaStream_t)o->stream : nullptr;
  bool own_stream = false;
  if (!stream) {
    if (cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking) != cudaSuccess) return SK_ECUDA;
    own_stream = true;
  }
  const bool ckpt_on = o && o->checkpoint_path && o->checkpoint_path[0];
  const unsigned long long chunk = plan_chunk_items(pl, o, ckpt_on);
  const unsigned long long nchunks = (pl.items + chunk - 1) / chunk;
  Ckpt ck;
  ck.have.assign(ckpt_on ? nchunks : 0, 0);
  ck.res.assign(ckpt_on ? nchunks * pl.nprimes : 0, 0);
  uint64_t resumed = 0;
  bool file_exists = false;
  if (ckpt_on) {
    ck.path = o->checkpoint_path;
    ck.header = ckpt_header(pl, chunk, nchunks);
    st = ckpt_load(&ck, pl);
    if (st) { if (own_stream) cudaStreamDestroy(stream); return st; }
    FILE* f = std::fopen(ck.path.c_str(), "rb");
    if (f) {
      std::fseek(f, 0, SEEK_END);
      file_exists = std::ftell(f) > 0;
      std::fclose(f);
    }
    for (auto h : ck.have) resumed += h;
  }

  ExactScratch* dscr = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t ce = cudaMalloc(&dscr, sizeof(ExactScratch));
  if (ce != cudaSuccess) { if (own_stream) cudaStreamDestroy(stream); return cuda_status(ce); }
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  uint64_t H[kMaxPrimes] = {0, 0, 0, 0};
  double kms = 0.0;
  uint64_t done_new = 0, done_total = resumed;
  const uint64_t max_new = (o && o->max_chunks) ? o->max_chunks : 0;
  for (unsigned long long c = 0; c < nchunks && st == SK_OK; ++c) {
    uint64_t r[kMaxPrimes] = {0, 0, 0, 0};
    if (ckpt_on && ck.have[c]) {
      for (int i = 0; i < pl.nprimes; ++i) r[i] = ck.res[c * pl.nprimes + i];
    } else {
      if (max_new && done_new >= max_new) continue;
      unsigned long long lo = c * chunk, hi = lo + chunk < pl.items ? lo + chunk : pl.items;
      st = run_chunk(pl, lo, hi, dscr, stream, e0, e1, r, &kms, nullptr, nullptr);
      if (st) break;
      if (ckpt_on) {
        st = ckpt_append(ck, !file_exists, c, r, pl.nprimes);
        file_exists = true;
        if (st) break;
        ck.have[c] = 1;
      }
      ++done_new;
      ++done_total;
    }
    for (int i = 0; i < pl.nprimes; ++i) H[i] = (H[i] + r[i]) % pl.primes[i];
  }
  cudaFree(dscr);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (own_stream) cudaStreamDestroy(stream);
  if (st) return st;
  const bool complete = done_total == nchunks;
  unmont(pl, H);
  if (pl.symmetry == SK_SYMMETRY_NEGATION_EVEN ||     // Lemma 2.4, s = +1: H = 2 H'
      pl.symmetry == SK_SYMMETRY_REVERSAL_EVEN)
    for (int i = 0; i < pl.nprimes; ++i) H[i] = (H[i] * 2) % pl.primes[i];
  sk_u128 coeff = {0, 0};
  if (complete) {
    // Lemma 2.1: H = C 2^{2n-1}; inclusion-exclusion: H = C
    st = crt_shifted(method == kMethodInclusionExclusion ? 0 : 2 * n - 1, pl.nprimes, pl.primes, H,
                     &coeff);
    if (st) return st;
  }
  if (rep) {
    std::memset(rep, 0, sizeof(*rep));
    rep->nprimes = pl.nprimes;
    for (int i = 0; i < pl.nprimes; ++i) {
      rep->primes[i] = pl.primes[i];
      rep->residues[i] = complete ? H[i] : 0;
    }
    rep->coefficient = coeff;
    rep->terms = pl.items << pl.m;
    rep->items = pl.items;
    rep->symmetry = pl.symmetry;
    rep->walk_bits = pl.m;
    rep->inner_bits = pl.U;
    rep->arith = pl.arith;
    rep->block_threads = pl.block_threads;
    rep->grid = pl.grid;
    rep->chunks_total = nchunks;
    rep->chunks_done = done_total;
    rep->chunks_resumed = resumed;
    rep->complete = complete ? 1 : 0;
    rep->kernel_ms = kms;
    rep->wall_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  }
  if (!complete) return SK_OK;
  sk_u128 v;
  const int conv = o ? o->convention : SK_COUNT_REFLECTIONS_IDENTIFIED;
  st = pl.hole ? apply_convention_hole(n, pl.hole, conv, coeff, &v)
               : apply_convention(variant, n, conv, coeff, &v);
  if (st) return st;
  if (out) *out = v;
  return SK_OK;
}

int item_residues_impl(int variant, int n, int m, uint64_t q_lo, uint64_t count, int nprimes,
                       const uint64_t* primes, int arith, uint64_t* out,
                       int method = kMethodAlgebraic, int hole = 0) {
  // items of an extended sequence's own position set: holes n+1..2n+1 (a
  // lower hole would be counted on its mirror image)
  if (hole && hole < n + 1) return SK_EINVAL;
  if (!out || !primes || count == 0 || count > (1ULL << 20)) return SK_EINVAL;
  sk_count_opts o;
  std::memset(&o, 0, sizeof(o));
  o.nprimes = nprimes;
  o.arith = arith;
  for (int i = 0; i < nprimes && i < SK_MAX_PRIMES; ++i) o.primes[i] = primes[i];
  o.walk_bits = m;
  Plan pl;
  int st = make_plan(variant, n, &o, &pl, method, hole);
  if (st) return st;
  if (q_lo >= pl.items || count > pl.items - q_lo) return SK_EINVAL;
  st = check_device();
  if (st) return st;
  cudaStream_t stream;
  if (cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking) != cudaSuccess) return SK_ECUDA;
  ExactScratch* dscr = nullptr;
  unsigned long long* dres = nullptr;
  cudaError_t ce = cudaMalloc(&dscr, sizeof(ExactScratch));
  if (ce == cudaSuccess) ce = cudaMalloc(&dres, count * pl.nprimes * sizeof(unsigned long long));
  if (ce != cudaSuccess) {
    cudaFree(dscr);
    cudaStreamDestroy(stream);
    return cuda_status(ce);
  }
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  uint64_t r[kMaxPrimes];
  double kms = 0;
  st = run_chunk(pl, q_lo, q_lo + count, dscr, stream, e0, e1, r, &kms, dres, nullptr);
  std::vector<uint64_t> h(count * pl.nprimes);
  if (!st) {
    ce = cudaMemcpy(h.data(), dres, h.size() * sizeof(uint64_t), cudaMemcpyDeviceToHost);
    if (ce != cudaSuccess) st = cuda_status(ce);
  }
  cudaFree(dscr);
  cudaFree(dres);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaStreamDestroy(stream);
  if (st) return st;
  for (uint64_t q = 0; q < count; ++q) {
    unmont(pl, &h[q * pl.nprimes]);
    for (int i = 0; i < pl.nprimes; ++i) out[q * pl.nprimes + i] = h[q * pl.nprimes + i];
  }
  return SK_OK;
}

}  // namespace sk

extern "C" int skolem_count(int variant, int n, sk_u128* out) {
  if (!out) return SK_EINVAL;
  return sk::count_impl(variant, n, nullptr, out, nullptr);
}

extern "C" int skolem_count_ex(int variant, int n, const sk_count_opts* opts, sk_u128* out,
                               sk_count_report* rep) {
  return sk::count_impl(variant, n, opts, out, rep);
}

extern "C" int sk_count_plan(int variant, int n, const sk_count_opts* opts, sk_count_report* rep) {
  return sk::plan_report(variant, n, opts, rep);
}

// The host step after the sums, for sums computed in parts (work-item ranges
// on different GPUs): the parts' residues added modulo each prime, then the
// CRT, checks and output convention of skolem_count_ex.  Host code only.
extern "C" int sk_count_from_residues(int variant, int n, int convention, int nprimes,
                                      const uint64_t* primes, uint64_t parts,
                                      const uint64_t* residues, sk_u128* out) {
  if (variant < SK_SKOLEM || variant > SK_HOOKED || n < 1 || n > sk::kMaxN) return SK_EINVAL;
  if (convention != SK_COUNT_REFLECTIONS_IDENTIFIED && convention != SK_COUNT_ALL)
    return SK_EINVAL;
  if (!residues || !out || parts == 0) return SK_EINVAL;
  sk_count_opts o;
  std::memset(&o, 0, sizeof(o));
  o.nprimes = nprimes;
  if (primes)
    for (int i = 0; i < nprimes && i < SK_MAX_PRIMES; ++i) o.primes[i] = primes[i];
  int k = 0;
  uint64_t pv[SK_MAX_PRIMES] = {};
  sk::Primes P;
  int st = sk::prepare_primes(&o, &k, pv, &P);
  if (st) return st;
  uint64_t H[SK_MAX_PRIMES] = {};
  for (uint64_t q = 0; q < parts; ++q)
    for (int i = 0; i < k; ++i) {
      const uint64_t r = residues[q * (uint64_t)k + i];
      if (r >= pv[i]) return SK_EINVAL;
      H[i] = (uint64_t)(((unsigned __int128)H[i] + r) % pv[i]);
    }
  return sk::finalize_count(variant, n, convention, k, pv, H, out);
}

extern "C" int skolem_item_residues(int variant, int n, int m, uint64_t q_lo, uint64_t count,
                                    int nprimes, const uint64_t* primes, uint64_t* out) {
  return sk::item_residues_impl(variant, n, m, q_lo, count, nprimes, primes, SK_ARITH_LIMBS, out);
}

extern "C" int skolem_item_residues_ex(int variant, int n, int m, uint64_t q_lo, uint64_t count,
                                       int nprimes, const uint64_t* primes, int arith,
                                       uint64_t* out) {
  return sk::item_residues_impl(variant, n, m, q_lo, count, nprimes, primes, arith, out);
}

extern "C" int sk_count_inclusion_exclusion(int variant, int n, const sk_count_opts* opts,
                                            sk_u128* out, sk_count_report* rep) {
  return sk::count_impl(variant, n, opts, out, rep, sk::kMethodInclusionExclusion);
}

extern "C" int sk_ie_item_residues(int variant, int n, int m, uint64_t q_lo, uint64_t count,
                                   int nprimes, const uint64_t* primes, uint64_t* out) {
  return sk::item_residues_impl(variant, n, m, q_lo, count, nprimes, primes, SK_ARITH_LIMBS, out,
                                sk::kMethodInclusionExclusion);
}

extern "C" int sk_count_extended(int n, int hole, const sk_count_opts* opts, sk_u128* out,
                                 sk_count_report* rep) {
  if (hole < 1 || hole > 2 * n + 1) return SK_EINVAL;    // (hole 0 would mean "no hole")
  return sk::count_impl(SK_SKOLEM, n, opts, out, rep, sk::kMethodAlgebraic, hole);
}

extern "C" int sk_extended_item_residues(int n, int hole, int m, uint64_t q_lo, uint64_t count,
                                         int nprimes, const uint64_t* primes, uint64_t* out) {
  if (hole < 1 || hole > 2 * n + 1) return SK_EINVAL;
  return sk::item_residues_impl(SK_SKOLEM, n, m, q_lo, count, nprimes, primes, SK_ARITH_LIMBS, out,
                                sk::kMethodAlgebraic, hole);
}
