// sk_host_common.cu -- moduli, CRT (Sec. 2.2), CRC-32, device checks.
#include "sk_host_common.h"

#include <cstring>

namespace sk {

static const uint64_t kDefaultPrimes[4] = {
    4611686018427387847ULL,  // 2^62 - 57
    4611686018427387817ULL,  // 2^62 - 87
    4611686018427387787ULL,  // 2^62 - 117
    4611686018427387761ULL,  // 2^62 - 143
};

int prepare_primes(const sk_count_opts* o, int* nprimes, uint64_t* primes, Primes* P) {
  int k = (o && o->nprimes) ? o->nprimes : 3;
  if (k < 3 || k > SK_MAX_PRIMES) return SK_EINVAL;
  for (int i = 0; i < k; ++i) {
    uint64_t p = (o && o->primes[i]) ? o->primes[i] : kDefaultPrimes[i];
    // the device's Montgomery step relies on a high limb of exactly 2^30
    if (!(p & 1) || p <= (1ULL << 62) - (1ULL << 31) || p >= (1ULL << 62)) return SK_EINVAL;
    for (int j = 0; j < i; ++j)
      if (gcd_u64(p, primes[j]) != 1) return SK_EINVAL;
    primes[i] = p;
  }
  std::memset(P, 0, sizeof(*P));
  for (int i = 0; i < k; ++i) P->pr[i] = make_prime(primes[i]);
  for (int i = k; i < kMaxPrimes; ++i) P->pr[i] = make_prime(kDefaultPrimes[i]);
  *nprimes = k;
  return SK_OK;
}

// ---------------------------------------------------------------- CRT

namespace {
struct Big {                // little-endian 64-bit limbs
  uint64_t w[4];
};
Big big_from_u128(u128 v) {
  Big b{};
  b.w[0] = (uint64_t)v;
  b.w[1] = (uint64_t)(v >> 64);
  return b;
}
Big big_mul_u64(const Big& a, uint64_t m) {
  Big r{};
  u128 carry = 0;
  for (int i = 0; i < 4; ++i) {
    u128 t = (u128)a.w[i] * m + carry;
    r.w[i] = (uint64_t)t;
    carry = t >> 64;
  }
  return r;
}
Big big_add(const Big& a, const Big& b) {
  Big r{};
  u128 c = 0;
  for (int i = 0; i < 4; ++i) {
    u128 t = (u128)a.w[i] + b.w[i] + c;
    r.w[i] = (uint64_t)t;
    c = t >> 64;
  }
  return r;
}
int big_cmp(const Big& a, const Big& b) {
  for (int i = 3; i >= 0; --i) {
    if (a.w[i] != b.w[i]) return a.w[i] < b.w[i] ? -1 : 1;
  }
  return 0;
}
uint64_t big_mod(const Big& a, uint64_t p) {
  uint64_t r = 0;
  for (int i = 3; i >= 0; --i) r = (uint64_t)((((u128)r << 64) | a.w[i]) % p);
  return r;
}
}  // namespace

int crt_coefficient(int n, int nprimes, const uint64_t* p, const uint64_t* H, sk_u128* coeff) {
  return crt_shifted(2 * n - 1, nprimes, p, H, coeff);   // Lemma 2.1 divisor after Lemma 2.2
}

int crt_shifted(int s, int nprimes, const uint64_t* p, const uint64_t* H, sk_u128* coeff) {
  if (s < 0 || s > 127) return SK_EINVAL;
  // Garner: x = r1 + p1 (t2 + p2 t3), 0 <= x < M = p1 p2 p3.
  const uint64_t r1 = H[0] % p[0], r2 = H[1] % p[1], r3 = H[2] % p[2];
  uint64_t t2 = mulmod((r2 + p[1] - r1 % p[1]) % p[1], invmod(p[0] % p[1], p[1]), p[1]);
  uint64_t u = mulmod((r3 + p[2] - r1 % p[2]) % p[2], invmod(p[0] % p[2], p[2]), p[2]);
  uint64_t t3 = mulmod((u + p[2] - t2 % p[2]) % p[2], invmod(p[1] % p[2], p[2]), p[2]);
  u128 y = (u128)t2 + (u128)p[1] * t3;
  Big x = big_add(big_mul_u64(big_from_u128(y), p[0]), big_from_u128(r1));
  Big M = big_mul_u64(big_from_u128((u128)p[0] * p[1]), p[2]);
  // H = C 2^s >= 0, so x must lie in the lower half of [0, M).
  Big x2 = big_add(x, x);
  if (big_cmp(x2, M) >= 0) return SK_EMISMATCH;
  if (nprimes >= 4 && big_mod(x, p[3]) != H[3] % p[3]) return SK_EMISMATCH;
  // low s bits must vanish
  for (int b = 0; b < s; ++b)
    if ((x.w[b / 64] >> (b % 64)) & 1ULL) return SK_EMISMATCH;
  Big c{};
  for (int i = 0; i < 4; ++i) {
    int src = i + s / 64, sh = s % 64;
    uint64_t lo = src < 4 ? x.w[src] : 0, hi = (src + 1) < 4 ? x.w[src + 1] : 0;
    c.w[i] = sh ? ((lo >> sh) | (hi << (64 - sh))) : lo;
  }
  if (c.w[2] || c.w[3]) return SK_ERANGE;
  coeff->lo = c.w[0];
  coeff->hi = c.w[1];
  return SK_OK;
}

// ---------------------------------------------------------------- CRC-32

namespace {
struct Crc32Table {
  uint32_t t[256];
  Crc32Table() {
    for (uint32_t i = 0; i < 256; ++i) {
      uint32_t c = i;
      for (int k = 0; k < 8; ++k) c = (c & 1) ? 0xEDB88320u ^ (c >> 1) : c >> 1;
      t[i] = c;
    }
  }
};
}  // namespace

uint32_t crc32(const void* data, size_t len) {
  static const Crc32Table tab;          // built once, thread-safe (function-local static)
  const uint32_t* table = tab.t;
  const unsigned char* b = (const unsigned char*)data;
  uint32_t c = 0xFFFFFFFFu;
  for (size_t i = 0; i < len; ++i) c = table[(c ^ b[i]) & 0xFF] ^ (c >> 8);
  return c ^ 0xFFFFFFFFu;
}

int check_device() {
  int dev = 0, count = 0;
  if (cudaGetDeviceCount(&count) != cudaSuccess || count < 1) {
    cudaGetLastError();
    return SK_ECUDA;
  }
  if (cudaGetDevice(&dev) != cudaSuccess) return SK_ECUDA;
  int major = 0;
  cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
  if (major != 10) return SK_ECUDA;
  return SK_OK;
}

}  // namespace sk

extern "C" void sk_default_primes(uint64_t* out4) {
  if (!out4) return;
  for (int i = 0; i < 4; ++i) out4[i] = sk::kDefaultPrimes[i];
}

extern "C" const char* sk_strerror(int status) {
  switch (status) {
    case SK_OK: return "ok";
    case SK_EINVAL: return "invalid argument";
    case SK_ERANGE: return "moduli cannot represent the value";
    case SK_ECUDA: return "CUDA error or no usable device";
    case SK_ENOMEM: return "out of memory";
    case SK_ETIMEOUT: return "a bounded device loop gave up";
    case SK_EMISMATCH: return "consistency check failed";
    case SK_ECKPT: return "checkpoint unreadable, corrupt or for another job";
    default: return "unknown status";
  }
}

extern "C" int sk_version(void) { return 100; }
