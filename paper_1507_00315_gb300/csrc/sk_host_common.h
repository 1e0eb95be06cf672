// sk_host_common.h -- host helpers shared by the library's translation units:
// modular arithmetic on 62-bit moduli, the CRT of Sec. 2.2, CRC-32 for the
// checkpoint file, CUDA error mapping.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <string>

#include "../../include/skolem.h"
#include "sk_exact.cuh"

namespace sk {

typedef unsigned __int128 u128;

inline uint64_t mulmod(uint64_t a, uint64_t b, uint64_t p) { return (uint64_t)((u128)a * b % p); }
inline uint64_t powmod(uint64_t a, uint64_t e, uint64_t p) {
  uint64_t r = 1 % p;
  a %= p;
  while (e) {
    if (e & 1) r = mulmod(r, a, p);
    a = mulmod(a, a, p);
    e >>= 1;
  }
  return r;
}
inline uint64_t gcd_u64(uint64_t a, uint64_t b) {
  while (b) { uint64_t t = a % b; a = b; b = t; }
  return a;
}
// inverse of a modulo odd p (a coprime to p), by the extended Euclid algorithm
inline uint64_t invmod(uint64_t a, uint64_t p) {
  __int128 t = 0, nt = 1, r = p, nr = a % p;
  while (nr) {
    __int128 q = r / nr, tmp;
    tmp = t - q * nt; t = nt; nt = tmp;
    tmp = r - q * nr; r = nr; nr = tmp;
  }
  if (t < 0) t += p;
  return (uint64_t)t;
}

// Split a modulus for the device's signed Montgomery step (R = 2^32).
inline Prime make_prime(uint64_t p) {
  Prime P;
  P.p = (long long)p;
  P.lo = (int)(uint32_t)p;
  P.hi = (int)(((long long)p - (long long)P.lo) >> 32);
  uint32_t inv = 1;                       // Newton: inv = p^{-1} mod 2^32
  for (int i = 0; i < 6; ++i) inv *= 2u - (uint32_t)p * inv;
  P.npinv = 0u - inv;
  return P;
}

// Validates and fills the moduli of an exact count.  Returns SK_OK/SK_EINVAL.
int prepare_primes(const sk_count_opts* o, int* nprimes, uint64_t* primes, Primes* P);

// Chinese remainder theorem over the first three moduli (Garner), the
// symmetric-range, 2^{2n-1}-divisibility and check-prime tests, and the
// division that yields the coefficient (pairings, reflections distinct).
int crt_coefficient(int n, int nprimes, const uint64_t* primes, const uint64_t* H,
                    sk_u128* coeff);
// The same with a divisor 2^shift (2n-1 for Lemma 2.1 after Lemma 2.2; 0 for
// the inclusion-exclusion sum, which is the count itself).
int crt_shifted(int shift, int nprimes, const uint64_t* primes, const uint64_t* H, sk_u128* out);

uint32_t crc32(const void* data, size_t len);

inline int cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return SK_OK;
  if (e == cudaErrorMemoryAllocation) return SK_ENOMEM;
  return SK_ECUDA;
}

// Checks that a usable device (compute capability 10.x) is current.
int check_device();

}  // namespace sk
