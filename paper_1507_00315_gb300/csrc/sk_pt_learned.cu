// sk_pt_learned.cu -- tempering chains whose move proposal is the trained
// network (an addition to Sec. 3; the ladder, statistics, exchanges and the
// estimator are those of Algorithm 2).  A move (k, s) is drawn from the
// softmax of the current state's logits over its valid moves; it is accepted
// with min(1, e^{-beta dE} q(C | C') / q(C' | C)) (Metropolis-Hastings), where
// q(C | C') is the probability of the reverse move (k, old slot) under the
// proposed state's logits, so the chains keep the Boltzmann weights of the
// plain ones.  Configurations live in global memory; per iteration the
// network runs once, on every proposed state, and an accepted state keeps its
// logits for the next draw.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "sk_host_common.h"
#include "sk_mlp.cuh"
#include "sk_pt.cuh"

namespace sk {

struct LearnedDev {
  int n, delta, M, L, B, nb, NMp;
  unsigned key0, key1;
  unsigned char* slots;      // [B][n] current configurations, c = ladder * M + l
  int* E;                    // [B]
  int* rung;                 // [B]
  int* lor;                  // [L][M]: configuration holding rung j
  __nv_bfloat16* Zcur;       // [B][NMp] logits of the current states (bf16)
  float* lse;                // [B] log-normaliser over their valid moves
  int4* prop;                // [B] (k, old slot, new slot, dE)
  float* lq_fwd;             // [B] log q(C' | C)
  unsigned* hist;            // [L][M][nb]
  unsigned* accm;            // [L][M]
  unsigned* accs;            // [L][M]
  const double* beta;        // [M]
  const unsigned long long* tswap;   // [M][nb]
};

// Per-block tables of the move layout: the pair k and the start slot of
// every move m (moves of pair k are off[k] .. off[k+1]-1), so a lane tests
// "m is a valid move" (its slot is not the pair's current one) from the
// tables and the state's slots in shared memory.
constexpr int kMaxMoves = 2560;        // sum_k (2n - d_k) for n <= kMlpMaxN, padded to 256
struct MoveMaps {
  __align__(16) unsigned char k[kMaxMoves];
  __align__(16) unsigned char s[kMaxMoves];
};

__device__ __forceinline__ void build_move_maps(const MoveTable& mt, MoveMaps& mm) {
  for (int m = threadIdx.x; m < kMaxMoves; m += blockDim.x) {
    if (m >= mt.NM) {                      // padding: pair 0, never valid (slot 0 of pair 0 = 0)
      mm.k[m] = 0;
      mm.s[m] = 0;
      continue;
    }
    int lo = 1, hi = mt.n;                 // the pair with off[k] <= m < off[k+1]
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (mt.off[mid] <= m) lo = mid;
      else hi = mid - 1;
    }
    mm.k[m] = (unsigned char)lo;
    mm.s[m] = (unsigned char)(m - mt.off[lo]);
  }
}

// One warp loads a configuration: lane k-1 takes pair k (slot, and its two
// bins into the occupancy counts when occ is given).  s_slot[0] = 0 makes
// the padding moves (pair 0, slot 0) invalid.
__device__ __forceinline__ void load_state(const unsigned char* sl, int n, int delta,
                                           unsigned char* s_slot, int* occ, int lane) {
  if (occ)
    for (int i = lane; i < 2 * n; i += 32) occ[i] = 0;
  if (lane == 0) s_slot[0] = 0;
  __syncwarp();
  for (int k = 1 + lane; k <= n; k += 32) {
    const int s = sl[k - 1];
    s_slot[k] = (unsigned char)s;
    if (occ) {
      atomicAdd(&occ[s], 1);
      atomicAdd(&occ[s + k + delta], 1);
    }
  }
  __syncwarp();
}

// Pull `bytes` bytes at p into L2 (one 128-byte line a lane at a time): a
// warp asks for the next chain's rows before it works on the current one,
// so the per-chain loads wait on L2 rather than on HBM.
__device__ __forceinline__ void prefetch_l2(const void* p, size_t bytes, int lane) {
  const char* c = (const char*)p;
  for (size_t o = (size_t)lane * 128; o < bytes; o += 32 * 128)
    asm volatile("prefetch.global.L2 [%0];" ::"l"(c + o));
}

// A chain's logit row (bf16) held in registers: chunk c of 256 moves, lane l
// holds moves 256 c + 8 l .. + 7 in one 16-byte word.  Lanes whose 8 moves
// all lie beyond NM load nothing (their words are never used).  CH = the
// chunks of the move table, ceil(NM / 256): the kernels are compiled for
// each CH up to kLtChunks, so no lane walks chunks the problem does not have.
constexpr int kLtChunks = kMaxMoves / 256;
template <int CH>
struct LogitRow {
  uint4 w[CH];
  unsigned valid[CH];          // bit i: move 256 c + 8 l + i is a valid move of the state
};

__device__ __forceinline__ float bf16_lo(unsigned x) { return __uint_as_float(x << 16); }
__device__ __forceinline__ float bf16_hi(unsigned x) { return __uint_as_float(x & 0xFFFF0000u); }
__device__ __forceinline__ float row_elem(const uint4& w, int i) {
  const unsigned x = i < 4 ? (i < 2 ? w.x : w.y) : (i < 6 ? w.z : w.w);
  return (i & 1) ? bf16_hi(x) : bf16_lo(x);
}

template <int CH>
__device__ __forceinline__ void load_row(const __nv_bfloat16* z, int NM, int lane, LogitRow<CH>& r) {
#pragma unroll
  for (int c = 0; c < CH; ++c) {
    const int m0 = c * 256 + lane * 8;
    r.w[c] = m0 < NM ? __ldg((const uint4*)(z + m0)) : make_uint4(0, 0, 0, 0);
  }
}

// Valid-move bits of the state in s_slot for the row's layout.
template <int CH>
__device__ __forceinline__ void row_valid(const MoveMaps& mm, const unsigned char* s_slot, int NM,
                                          int lane, LogitRow<CH>& r) {
#pragma unroll
  for (int c = 0; c < CH; ++c) {
    const int m0 = c * 256 + lane * 8;
    unsigned bits = 0;
    if (m0 < NM) {
      const uint2 kk = *(const uint2*)&mm.k[m0];
      const uint2 ss = *(const uint2*)&mm.s[m0];
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const unsigned k = ((i < 4 ? kk.x : kk.y) >> (8 * (i & 3))) & 0xFFu;
        const unsigned sl = ((i < 4 ? ss.x : ss.y) >> (8 * (i & 3))) & 0xFFu;
        bits |= (unsigned)(sl != s_slot[k]) << i;
      }
    }
    r.valid[c] = bits;
  }
}

// log sum exp of the row over its valid moves, in one pass over the
// registers: each lane keeps a running maximum and the sum scaled to it
// (rescaled when the maximum grows), then the lanes' pairs are combined.
template <int CH>
__device__ __forceinline__ float row_lse(const LogitRow<CH>& r) {
  float mx = -INFINITY, sum = 0.f;
#pragma unroll
  for (int c = 0; c < CH; ++c)
#pragma unroll
    for (int i = 0; i < 8; ++i)
      if ((r.valid[c] >> i) & 1u) {
        const float z = row_elem(r.w[c], i);
        if (z > mx) {
          sum = sum * __expf(mx - z) + 1.f;
          mx = z;
        } else {
          sum += __expf(z - mx);
        }
      }
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    const float m2 = __shfl_xor_sync(0xffffffffu, mx, o);
    const float s2 = __shfl_xor_sync(0xffffffffu, sum, o);
    const float mn = fmaxf(mx, m2);
    sum = mn == -INFINITY ? 0.f : sum * __expf(mx - mn) + s2 * __expf(m2 - mn);
    mx = mn;
  }
  return mx + __logf(sum);
}

__global__ void lt_init_kernel(LearnedDev d) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= d.B) return;
  const int ladder = c / d.M, l = c % d.M, bins = 2 * d.n;
  unsigned char occ[2 * kPtMaxN];
  for (int b = 0; b < bins; ++b) occ[b] = 0;
  for (int k = 1; k <= d.n; ++k) {
    const unsigned L = (unsigned)(bins - (k + d.delta));
    const uint4 w = philox4x32_10(make_uint4((unsigned)k, (unsigned)l, (unsigned)ladder, 1u),
                                  d.key0, d.key1);
    const int s = (int)__umulhi(w.x, L);
    d.slots[(size_t)c * d.n + k - 1] = (unsigned char)s;
    occ[s] += 1;
    occ[s + k + d.delta] += 1;
  }
  int E = 0;
  for (int b = 0; b < bins; ++b) E += occ[b] == 0;
  d.E[c] = E;
  d.rung[c] = l;
  d.lor[c] = l;
}

// After a forward pass of the current states: keep their logits and lse.
template <int CH>
__global__ void __launch_bounds__(256, CH <= 4 ? 4 : 2) lt_keep_kernel(LearnedDev d, MoveTable mt,
                                                      const __nv_bfloat16* Z) {
  __shared__ MoveMaps mm;
  __shared__ unsigned char s_slot[8][kPtMaxN + 8];
  build_move_maps(mt, mm);
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int c = blockIdx.x * 8 + w; c < d.B; c += gridDim.x * 8) {
    load_state(d.slots + (size_t)c * d.n, d.n, d.delta, s_slot[w], nullptr, lane);
    LogitRow<CH> r;
    load_row(Z + (size_t)c * d.NMp, mt.NM, lane, r);
    row_valid(mm, s_slot[w], mt.NM, lane, r);
    const float l = row_lse(r);
    __nv_bfloat16* zc = d.Zcur + (size_t)c * d.NMp;
#pragma unroll
    for (int k = 0; k < CH; ++k)
      if (k * 256 + lane * 8 < mt.NM) *(uint4*)(zc + k * 256 + lane * 8) = r.w[k];
    if (lane == 0) d.lse[c] = l;
    __syncwarp();
  }
}

// Statistics of iteration t, then a move drawn from the current softmax; the
// proposed configuration goes to `prop_slots` (the network's input).  The
// draw is an inverse CDF over the valid moves in move order, from the row in
// registers: the chunk sums (warp reductions), the chunk that holds u *
// total, a scan of its lanes' sums, then the lane that holds it walks its 8
// moves.
template <int CH>
__global__ void __launch_bounds__(256, CH <= 4 ? 4 : 2) lt_propose_kernel(LearnedDev d, MoveTable mt, unsigned t,
                                                         int count_stats,
                                                         unsigned char* prop_slots) {
  __shared__ MoveMaps mm;
  __shared__ int s_occ[8][2 * kPtMaxN];
  __shared__ unsigned char s_slot[8][kPtMaxN + 8];
  build_move_maps(mt, mm);
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int NM = mt.NM;
  for (int c = blockIdx.x * 8 + w; c < d.B; c += gridDim.x * 8) {
    const int cn = c + gridDim.x * 8;
    if (cn < d.B) {
      prefetch_l2(d.Zcur + (size_t)cn * d.NMp, (size_t)NM * 2, lane);
      prefetch_l2(d.slots + (size_t)cn * d.n, (size_t)d.n, lane);
    }
    LogitRow<CH> r;
    load_row(d.Zcur + (size_t)c * d.NMp, NM, lane, r);
    const int ladder = c / d.M, rg = d.rung[c], E = d.E[c];
    if (lane == 0 && count_stats) d.hist[((size_t)ladder * d.M + rg) * d.nb + E] += 1;
    load_state(d.slots + (size_t)c * d.n, d.n, d.delta, s_slot[w], s_occ[w], lane);
    row_valid(mm, s_slot[w], NM, lane, r);
    const float lse = d.lse[c];
    const uint4 rw = philox4x32_10(make_uint4(t, (unsigned)rg, (unsigned)ladder, 5u), d.key0, d.key1);
    // per lane and chunk: the sum of exp(z - lse) over its valid moves
    float part[CH], csum[CH];
    float total = 0.f;
#pragma unroll
    for (int k = 0; k < CH; ++k) {
      float a = 0.f;
#pragma unroll
      for (int i = 0; i < 8; ++i)
        if ((r.valid[k] >> i) & 1u) a += __expf(row_elem(r.w[k], i) - lse);
      part[k] = a;
      csum[k] = warp_sum(a);
      total += csum[k];
    }
    const float target = ((float)rw.x + 0.5f) * 2.3283064365386963e-10f * total;
    // the chunk: the first whose running sum reaches the target (the last
    // one with valid moves if rounding leaves the target above the total)
    float run = 0.f, pk = 0.f;
    uint4 wk = make_uint4(0, 0, 0, 0);
    unsigned vk = 0;
    int kc = -1, klast = 0;
#pragma unroll
    for (int k = 0; k < CH; ++k) {
      const bool any = __any_sync(0xffffffffu, r.valid[k] != 0u);
      if (any) klast = k;
      if (kc < 0 && any && run + csum[k] >= target) {
        kc = k;
      } else if (kc < 0) {
        run += csum[k];
      }
    }
    if (kc < 0) {                          // rounding: take the last chunk with valid moves
      kc = klast;
      run = total;                         // every lane of that chunk then falls through to its last move
#pragma unroll
      for (int k = 0; k < CH; ++k)
        if (k == klast) run -= csum[k];
    }
#pragma unroll
    for (int k = 0; k < CH; ++k)
      if (k == kc) { pk = part[k]; wk = r.w[k]; vk = r.valid[k]; }
    // lanes of the chunk: inclusive scan of their sums
    float incl = pk;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const float u = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += u;
    }
    const unsigned hit = __ballot_sync(0xffffffffu, vk != 0u && run + incl >= target);
    const unsigned withv = __ballot_sync(0xffffffffu, vk != 0u);
    const int ln = hit ? __ffs(hit) - 1 : 31 - __clz(withv);   // withv != 0: the chunk has valid moves
    int pick_i = -1;
    if (lane == ln) {
      float a = run + incl - pk;           // exclusive: the running sum before this lane's moves
      int last = -1;
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        if ((vk >> i) & 1u) {
          last = i;
          a += __expf(row_elem(wk, i) - lse);
          if (pick_i < 0 && a >= target) pick_i = i;
        }
      }
      if (pick_i < 0) pick_i = last;
    }
    pick_i = __shfl_sync(0xffffffffu, pick_i, ln);
    const uint4 wp = make_uint4(__shfl_sync(0xffffffffu, wk.x, ln), __shfl_sync(0xffffffffu, wk.y, ln),
                                __shfl_sync(0xffffffffu, wk.z, ln), __shfl_sync(0xffffffffu, wk.w, ln));
    const int pick = kc * 256 + ln * 8 + pick_i;
    const int kp = mm.k[pick];
    const int s_new = mm.s[pick], s_old = s_slot[w][kp];
    const int dE = move_delta_e(s_occ[w], s_old, kp + d.delta, s_new);
    unsigned char* ps = prop_slots + (size_t)c * d.n;
    for (int i = lane; i < d.n; i += 32)
      ps[i] = (i + 1 == kp) ? (unsigned char)s_new : s_slot[w][i + 1];
    if (lane == 0) {
      d.prop[c] = make_int4(kp, s_old, s_new, dE);
      d.lq_fwd[c] = row_elem(wp, pick_i) - lse;
    }
    __syncwarp();
  }
}

// Metropolis-Hastings acceptance with the proposed states' logits Zp (bf16).
template <int CH>
__global__ void __launch_bounds__(256, CH <= 4 ? 4 : 2) lt_accept_kernel(LearnedDev d, MoveTable mt, unsigned t,
                                                        const unsigned char* prop_slots,
                                                        const __nv_bfloat16* Zp) {
  __shared__ MoveMaps mm;
  __shared__ unsigned char s_slot[8][kPtMaxN + 8];
  build_move_maps(mt, mm);
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int NM = mt.NM;
  for (int c = blockIdx.x * 8 + w; c < d.B; c += gridDim.x * 8) {
    const int cn = c + gridDim.x * 8;
    if (cn < d.B) {
      prefetch_l2(Zp + (size_t)cn * d.NMp, (size_t)NM * 2, lane);
      prefetch_l2(prop_slots + (size_t)cn * d.n, (size_t)d.n, lane);
    }
    const __nv_bfloat16* zp = Zp + (size_t)c * d.NMp;
    LogitRow<CH> r;
    load_row(zp, NM, lane, r);
    const int ladder = c / d.M, rg = d.rung[c];
    load_state(prop_slots + (size_t)c * d.n, d.n, d.delta, s_slot[w], nullptr, lane);
    row_valid(mm, s_slot[w], NM, lane, r);
    const float lse_p = row_lse(r);
    const int4 pr = d.prop[c];
    const float lq_rev = __bfloat162float(zp[mt.off[pr.x] + pr.y]) - lse_p;
    const float log_a = (float)(-d.beta[rg] * (double)pr.w) + lq_rev - d.lq_fwd[c];
    const uint4 rw = philox4x32_10(make_uint4(t, (unsigned)rg, (unsigned)ladder, 5u), d.key0, d.key1);
    const float u = ((float)rw.y + 0.5f) * 2.3283064365386963e-10f;
    const bool acc = log_a >= 0.f || logf(u) < log_a;
    if (acc) {
      for (int i = lane; i < d.n; i += 32) d.slots[(size_t)c * d.n + i] = s_slot[w][i + 1];
      __nv_bfloat16* zc = d.Zcur + (size_t)c * d.NMp;
#pragma unroll
      for (int k = 0; k < CH; ++k)
        if (k * 256 + lane * 8 < NM) *(uint4*)(zc + k * 256 + lane * 8) = r.w[k];
      if (lane == 0) {
        d.lse[c] = lse_p;
        d.E[c] += pr.w;
        d.accm[(size_t)ladder * d.M + rg] += 1;
      }
    }
    __syncwarp();
  }
}

// Exchanges of iteration t, one warp per ladder, lane j for rung j.
__global__ void lt_exchange_kernel(LearnedDev d, unsigned t) {
  const int lane = threadIdx.x & 31;
  const int ladder = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (ladder >= d.L) return;
  const int M = d.M;
  int* lor = d.lor + (size_t)ladder * M;
  const int my = lane < M ? lor[lane] : 0;
  const int Er = lane < M ? d.E[(size_t)ladder * M + my] : 0;
  const int En = __shfl_down_sync(0xffffffffu, Er, 1);
  int dec = 0;
  if (lane + 1 < M && (lane & 1) == (int)(t & 1u)) {
    const uint4 w = philox4x32_10(make_uint4(t, (unsigned)lane, (unsigned)ladder, 3u), d.key0,
                                  d.key1);
    const int de = Er - En;
    dec = (de <= 0 || (unsigned long long)w.x < d.tswap[lane * d.nb + de]) ? 1 : 0;
    if (dec) d.accs[(size_t)ladder * M + lane] += 1;
  }
  const int down = __shfl_down_sync(0xffffffffu, my, 1), up = __shfl_up_sync(0xffffffffu, my, 1);
  const int dec_up = __shfl_up_sync(0xffffffffu, dec, 1);
  const int nl = dec ? down : ((lane > 0 && dec_up) ? up : my);
  if (lane < M) {
    lor[lane] = nl;
    d.rung[(size_t)ladder * M + nl] = lane;
  }
}

// out[i] = sum over ladders of in[l][i].
__global__ void lt_reduce_kernel(const unsigned* in, int L, int per, unsigned long long* out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= per) return;
  unsigned long long s = 0;
  for (int l = 0; l < L; ++l) s += in[(size_t)l * per + i];
  out[i] = s;
}

}  // namespace sk

namespace sk {

// The per-chain kernels for the chunk count of the move table.
#define SK_LT_CHUNKS(X) X(1) X(2) X(3) X(4) X(5) X(6) X(7) X(8) X(9) X(10)
static_assert(kLtChunks == 10, "one case per chunk count");
struct LtKernels {
  void (*keep)(LearnedDev, MoveTable, const __nv_bfloat16*);
  void (*propose)(LearnedDev, MoveTable, unsigned, int, unsigned char*);
  void (*accept)(LearnedDev, MoveTable, unsigned, const unsigned char*, const __nv_bfloat16*);
};
static bool lt_kernels(int ch, LtKernels* k) {
  switch (ch) {
#define SK_LT_CASE(c) \
  case c: *k = {lt_keep_kernel<c>, lt_propose_kernel<c>, lt_accept_kernel<c>}; return true;
    SK_LT_CHUNKS(SK_LT_CASE)
#undef SK_LT_CASE
    default: return false;
  }
}

int pt_learned_run(int variant, int n, int M, const double* beta, int L, uint64_t iters,
                   uint64_t burnin, uint64_t seed, const void* model, uint64_t* hist,
                   uint64_t* accm, uint64_t* accs, void* stream, double* kernel_ms) {
  Mlp* m = (Mlp*)model;
  if (!m || !beta || !hist || iters > 0xffffffffULL) return SK_EINVAL;
  if (m->variant != variant || m->n != n || M < 2 || M > kPtMaxRungsLearned || L < 1) return SK_EINVAL;
  const int B = L * M, Bp = (B + 127) / 128 * 128, nb = 2 * n + 1;
  if (Bp > m->max_batch) return SK_EINVAL;
  int st = check_device();
  if (st) return st;
  std::vector<unsigned long long> ts((size_t)M * nb, 0);
  for (int j = 0; j + 1 < M; ++j)
    for (int de = 1; de <= 2 * n; ++de)
      ts[j * nb + de] = accept_threshold((beta[j + 1] - beta[j]) * (double)de);
  cudaStream_t s = (cudaStream_t)stream;
  bool own = false;
  if (!s) {
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) return SK_ECUDA;
    own = true;
  }
  // the per-chain kernels loop over chains, 8 per block, 8 blocks per SM (two
  // waves of the 4 resident ones)
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int chain_grid = std::min((B + 7) / 8, 8 * (sms > 0 ? sms : 1));
  LearnedDev d;
  std::memset(&d, 0, sizeof(d));
  d.n = n; d.delta = m->delta; d.M = M; d.L = L; d.B = B; d.nb = nb; d.NMp = m->NMp;
  d.key0 = (unsigned)seed; d.key1 = (unsigned)(seed >> 32);
  auto al = [](size_t x) { return (x + 255) / 256 * 256; };
  size_t off = 0;
  const size_t o_sl = off; off = al(off + (size_t)B * n);
  const size_t o_E = off; off = al(off + (size_t)B * 4);
  const size_t o_r = off; off = al(off + (size_t)B * 4);
  const size_t o_lor = off; off = al(off + (size_t)B * 4);
  const size_t o_z = off; off = al(off + (size_t)B * m->NMp * 2);
  const size_t o_lse = off; off = al(off + (size_t)B * 4);
  const size_t o_pr = off; off = al(off + (size_t)B * 16);
  const size_t o_lq = off; off = al(off + (size_t)B * 4);
  const size_t o_h = off; off = al(off + (size_t)L * M * nb * 4);
  const size_t o_am = off; off = al(off + (size_t)L * M * 4);
  const size_t o_as = off; off = al(off + (size_t)L * M * 4);
  const size_t o_b = off; off = al(off + (size_t)M * 8);
  const size_t o_ts = off; off = al(off + ts.size() * 8);
  const size_t o_out = off; off = al(off + ((size_t)M * nb + 2 * M) * 8);
  char* p = nullptr;
  cudaError_t e = cudaMalloc(&p, off);
  if (e != cudaSuccess) {
    if (own) cudaStreamDestroy(s);
    return SK_ENOMEM;
  }
  d.slots = (unsigned char*)(p + o_sl);
  d.E = (int*)(p + o_E);
  d.rung = (int*)(p + o_r);
  d.lor = (int*)(p + o_lor);
  d.Zcur = (__nv_bfloat16*)(p + o_z);
  d.lse = (float*)(p + o_lse);
  d.prop = (int4*)(p + o_pr);
  d.lq_fwd = (float*)(p + o_lq);
  d.hist = (unsigned*)(p + o_h);
  d.accm = (unsigned*)(p + o_am);
  d.accs = (unsigned*)(p + o_as);
  d.beta = (const double*)(p + o_b);
  d.tswap = (const unsigned long long*)(p + o_ts);
  unsigned long long* out = (unsigned long long*)(p + o_out);
  const MoveTable mt = move_table(*m);
  LtKernels lk;
  if (!lt_kernels((mt.NM + 255) / 256, &lk)) {
    cudaFree(p);
    if (own) cudaStreamDestroy(s);
    return SK_EINVAL;
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  e = cudaMemsetAsync(p + o_h, 0, o_b - o_h, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(p + o_b, beta, (size_t)M * 8, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(p + o_ts, ts.data(), ts.size() * 8, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(m->slots, 0, (size_t)Bp * n, s);   // padding rows
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e == cudaSuccess) e = cudaEventRecord(e0, s);
  if (e == cudaSuccess) {
    lt_init_kernel<<<(B + 255) / 256, 256, 0, s>>>(d);
    e = cudaMemcpyAsync(m->slots, d.slots, (size_t)B * n, cudaMemcpyDeviceToDevice, s);
  }
  const __nv_bfloat16* Zb = (const __nv_bfloat16*)m->Z;      // the forward's bf16 logits
  if (e == cudaSuccess) e = mlp_forward_dev(*m, Bp, s, true);
  if (e == cudaSuccess) {
    lk.keep<<<chain_grid, 256, 0, s>>>(d, mt, Zb);
    e = cudaGetLastError();
  }
  for (uint64_t t = 0; t < iters && e == cudaSuccess; ++t) {
    lk.propose<<<chain_grid, 256, 0, s>>>(d, mt, (unsigned)t, t >= burnin ? 1 : 0, m->slots);
    e = mlp_forward_dev(*m, Bp, s, true);
    if (e != cudaSuccess) break;
    lk.accept<<<chain_grid, 256, 0, s>>>(d, mt, (unsigned)t, m->slots, Zb);
    lt_exchange_kernel<<<(L + 3) / 4, 128, 0, s>>>(d, (unsigned)t);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) {
    const int per = M * nb;
    lt_reduce_kernel<<<(per + 255) / 256, 256, 0, s>>>(d.hist, L, per, out);
    lt_reduce_kernel<<<1, 64, 0, s>>>(d.accm, L, M, out + per);
    lt_reduce_kernel<<<1, 64, 0, s>>>(d.accs, L, M, out + per + M);
    e = cudaEventRecord(e1, s);
  }
  std::vector<unsigned long long> h((size_t)M * nb + 2 * M);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h.data(), out, h.size() * 8, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  float ms = 0.f;
  if (e == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(p);
  if (own) cudaStreamDestroy(s);
  if (e != cudaSuccess) return cuda_status(e);
  for (size_t i = 0; i < (size_t)M * nb; ++i) hist[i] = h[i];
  for (int j = 0; j < M; ++j) {
    if (accm) accm[j] = h[(size_t)M * nb + j];
    if (accs) accs[j] = h[(size_t)M * nb + M + j];
  }
  if (kernel_ms) *kernel_ms = ms;
  return SK_OK;
}

}  // namespace sk

extern "C" int sk_pt_run_learned(int variant, int n, int M, const double* beta, int L,
                                 uint64_t iters, uint64_t burnin, uint64_t seed, const void* model,
                                 uint64_t* hist, uint64_t* acc_move, uint64_t* acc_swap) {
  return sk::pt_learned_run(variant, n, M, beta, L, iters, burnin, seed, model, hist, acc_move,
                            acc_swap, nullptr, nullptr);
}
