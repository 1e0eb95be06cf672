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
  unsigned rk[20];           // Philox round keys of (key0, key1), computed on the host
  unsigned char* slots;      // [B][n] current configurations, c = ladder * M + l
  int* E;                    // [B]
  int* rung;                 // [B]
  int* lor;                  // [L][M]: configuration holding rung j
  __nv_bfloat16* Zcur;       // [B][NMp] logits of the current states (bf16)
  float* lse;                // [B] log-normaliser over their valid moves
  int4* prop;                // [B] (k | old slot << 8 | new slot << 16, dE, log q(C' | C)
                             //      as float bits, the acceptance test's uniform word)
  unsigned* hist;            // [L][M][nb]
  unsigned* accm;            // [L][M]
  unsigned* accs;            // [L][M]
  const double* beta;        // [M]
  const unsigned long long* tswap;   // [M][nb]
};

// Per-block tables of the move layout: the pair k and the start slot of
// every move m (moves of pair k are off[k] .. off[k+1]-1), read for the one
// move a chain draws; and the offsets off[k] themselves.
constexpr int kMaxMoves = 2560;        // sum_k (2n - d_k) for n <= kMlpMaxN, padded to 256
struct MoveMaps {
  __align__(16) unsigned char k[kMaxMoves];
  __align__(16) unsigned char s[kMaxMoves];
  int off[kPtMaxN + 2];
};

// The first `moves` entries of the tables (the chunks a kernel covers).
__device__ __forceinline__ void build_move_maps(const MoveTable& mt, MoveMaps& mm, int moves) {
  for (int k = threadIdx.x; k <= mt.n + 1; k += blockDim.x) mm.off[k] = k ? mt.off[k] : 0;
  for (int m = threadIdx.x; m < moves; m += blockDim.x) {
    if (m >= mt.NM) {                      // padding
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

// A configuration in registers: lane k-1 holds the start slot of pair k,
// lane k-33 that of pair k > 32 (-1: no such pair).
__device__ __forceinline__ void load_slots(const unsigned char* sl, int n, int lane, int& sa,
                                           int& sb) {
  sa = lane < n ? (int)sl[lane] : -1;
  sb = lane + 32 < n ? (int)sl[lane + 32] : -1;
}

// The start slot of pair k (1..n) from the lanes that hold the configuration.
__device__ __forceinline__ int slot_of(int sa, int sb, int k) {
  const int a = __shfl_sync(0xffffffffu, sa, (k - 1) & 31);
  const int b = __shfl_sync(0xffffffffu, sb, (k - 33) & 31);
  return k <= 32 ? a : b;
}

// Bin occupancies of the configuration into the warp's counts occ[2n].
__device__ __forceinline__ void place_occupancy(int sa, int sb, int n, int delta, int* occ,
                                                int lane) {
  for (int i = lane; i < 2 * n; i += 32) occ[i] = 0;
  __syncwarp();
  if (sa >= 0) {
    atomicAdd(&occ[sa], 1);
    atomicAdd(&occ[sa + lane + 1 + delta], 1);
  }
  if (sb >= 0) {
    atomicAdd(&occ[sb], 1);
    atomicAdd(&occ[sb + lane + 33 + delta], 1);
  }
  __syncwarp();
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

// e^(z - lse) as 2^(z log2(e) - lse log2(e)): one fused multiply-add and the
// hardware base-2 exponential (lse2 = lse log2(e)).
__device__ __forceinline__ float exp_shifted(float z, float lse2) {
  const float x = fmaf(z, 1.4426950408889634f, -lse2);
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

template <int CH>
__device__ __forceinline__ void load_row(const __nv_bfloat16* z, int NM, int lane, LogitRow<CH>& r) {
#pragma unroll
  for (int c = 0; c < CH; ++c) {
    const int m0 = c * 256 + lane * 8;
    r.w[c] = m0 < NM ? __ldg((const uint4*)(z + m0)) : make_uint4(0, 0, 0, 0);
  }
}

// Valid-move bits of the configuration (sa, sb) for the row's layout.  A
// state has exactly one invalid move per pair (its current slot), so the
// lanes set those n bits in the warp's bitmask bits[CH * 8] (one atomicOr a
// pair) and each lane reads back the byte of its 8 moves per chunk; moves
// from NM on are invalid too.
template <int CH>
__device__ __forceinline__ void row_valid(const MoveMaps& mm, int sa, int sb, int NM, int lane,
                                          unsigned* bits, LogitRow<CH>& r) {
  for (int i = lane; i < CH * 8; i += 32) bits[i] = 0;
  __syncwarp();
  if (sa >= 0) {
    const int m = mm.off[lane + 1] + sa;
    atomicOr(&bits[m >> 5], 1u << (m & 31));
  }
  if (sb >= 0) {
    const int m = mm.off[lane + 33] + sb;
    atomicOr(&bits[m >> 5], 1u << (m & 31));
  }
  __syncwarp();
  const unsigned char* by = (const unsigned char*)bits;   // byte 32 c + l: moves 256 c + 8 l ..
#pragma unroll
  for (int c = 0; c < CH; ++c) {
    const int m0 = c * 256 + lane * 8;
    const int left = NM - m0;
    const unsigned in = left <= 0 ? 0u : (left >= 8 ? 0xFFu : (1u << left) - 1u);
    r.valid[c] = ~(unsigned)by[c * 32 + lane] & in;
  }
}

// log sum exp of the row over its valid moves, from the registers: the
// maximum on the packed bf16 pairs (invalid moves replaced by -inf; a bf16
// maximum is exact), then the sum of e^(z - max) over the valid moves, each
// reduced over the warp.
template <int CH>
__device__ __forceinline__ float row_lse(const LogitRow<CH>& r) {
  __nv_bfloat162 acc = __halves2bfloat162(__ushort_as_bfloat16((unsigned short)0xFF80u),
                                          __ushort_as_bfloat16((unsigned short)0xFF80u));
#pragma unroll
  for (int c = 0; c < CH; ++c)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const unsigned x = j == 0 ? r.w[c].x : (j == 1 ? r.w[c].y : (j == 2 ? r.w[c].z : r.w[c].w));
      const unsigned b = (r.valid[c] >> (2 * j)) & 3u;
      const unsigned m = ((b & 1u) * 0xFFFFu) | ((b >> 1) * 0xFFFF0000u);
      const unsigned v = (x & m) | (0xFF80FF80u & ~m);
      acc = __hmax2(acc, *(const __nv_bfloat162*)&v);
    }
  const float mx = warp_max(fmaxf(__bfloat162float(acc.x), __bfloat162float(acc.y)));
  const float mx2 = mx * 1.4426950408889634f;
  float sum = 0.f;
#pragma unroll
  for (int c = 0; c < CH; ++c)
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const float e = exp_shifted(row_elem(r.w[c], i), mx2);
      sum += ((r.valid[c] >> i) & 1u) ? e : 0.f;
    }
  return mx + __logf(warp_sum(sum));
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
  __shared__ unsigned s_bits[8][kLtChunks * 8];
  build_move_maps(mt, mm, 0);
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int c = blockIdx.x * 8 + w; c < d.B; c += gridDim.x * 8) {
    int sa, sb;
    load_slots(d.slots + (size_t)c * d.n, d.n, lane, sa, sb);
    LogitRow<CH> r;
    load_row(Z + (size_t)c * d.NMp, mt.NM, lane, r);
    row_valid(mm, sa, sb, mt.NM, lane, s_bits[w], r);
    const float l = row_lse(r);
    __nv_bfloat16* zc = d.Zcur + (size_t)c * d.NMp;
#pragma unroll
    for (int k = 0; k < CH; ++k)
      if (k * 256 + lane * 8 < mt.NM) *(uint4*)(zc + k * 256 + lane * 8) = r.w[k];
    if (lane == 0) d.lse[c] = l;
    __syncwarp();
  }
}

// A chain's inputs to the propose kernel, loaded one chain ahead: its logit
// row, its configuration (lanes), rung, energy and log-normaliser.
template <int CH>
struct ProposeIn {
  LogitRow<CH> r;
  int sa, sb, rung, E;
  float lse;
};

template <int CH>
__device__ __forceinline__ void load_propose_in(const LearnedDev& d, int NM, int c, int lane,
                                                ProposeIn<CH>& in) {
  load_row(d.Zcur + (size_t)c * d.NMp, NM, lane, in.r);
  load_slots(d.slots + (size_t)c * d.n, d.n, lane, in.sa, in.sb);
  in.rung = d.rung[c];
  in.E = d.E[c];
  in.lse = d.lse[c];
}

// Statistics of iteration t, then a move drawn from the current softmax; the
// proposed configuration goes to `prop_slots`, and its bin occupancies
// straight into the network's input rows X ([B][K1] bf16), so the forward
// that follows needs no input kernel.  The draw is an inverse CDF over the
// valid moves in move order, from the row in registers: the chunk sums
// (warp reductions), the chunk that holds u * total, a scan of its lanes'
// sums, then the lane that holds it walks its 8 moves.  The proposal record
// carries the move, dE, log q(C' | C) and the uniform word of the
// acceptance test (the same Philox block, word 1), so the accept kernel
// computes no Philox block of its own.  Each warp loads the next chain's row
// and state while it works on the current one.
template <int CH>
__global__ void __launch_bounds__(256, CH <= 4 ? 3 : 2)
    lt_propose_kernel(LearnedDev d, MoveTable mt, unsigned t, int count_stats,
                      unsigned char* prop_slots, __nv_bfloat16* X, int K1) {
  __shared__ MoveMaps mm;
  __shared__ int s_occ[8][2 * kPtMaxN];
  __shared__ unsigned s_bits[8][kLtChunks * 8];
  build_move_maps(mt, mm, CH * 256);
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int NM = mt.NM, stride = gridDim.x * 8;
  int c = blockIdx.x * 8 + w;
  ProposeIn<CH> cur;
  if (c < d.B) load_propose_in(d, NM, c, lane, cur);
  for (; c < d.B; c += stride) {
    ProposeIn<CH> nxt;
    if (c + stride < d.B) load_propose_in(d, NM, c + stride, lane, nxt);
    const int ladder = c / d.M, rg = cur.rung;
    if (lane == 0 && count_stats)
      atomicAdd(&d.hist[((size_t)ladder * d.M + rg) * d.nb + cur.E], 1u);
    place_occupancy(cur.sa, cur.sb, d.n, d.delta, s_occ[w], lane);
    LogitRow<CH>& r = cur.r;
    row_valid(mm, cur.sa, cur.sb, NM, lane, s_bits[w], r);
    const float lse = cur.lse;
    const uint4 rw = philox4x32_10_rk(make_uint4(t, (unsigned)rg, (unsigned)ladder, 5u), d.rk);
    // per lane and chunk: the sum of exp(z - lse) over its valid moves
    const float lse2 = lse * 1.4426950408889634f;
    float part[CH], csum[CH];
    float total = 0.f;
#pragma unroll
    for (int k = 0; k < CH; ++k) {
      float a = 0.f;
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const float e = exp_shifted(row_elem(r.w[k], i), lse2);
        a += ((r.valid[k] >> i) & 1u) ? e : 0.f;
      }
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
    // that lane's 8 moves, one a lane on lanes 0..7: the running sum before
    // them, a scan of their terms, the first that reaches the target (else
    // its last valid move)
    const float excl = __shfl_sync(0xffffffffu, run + incl - pk, ln);
    const unsigned vl = __shfl_sync(0xffffffffu, vk, ln);
    const uint4 wp = make_uint4(__shfl_sync(0xffffffffu, wk.x, ln), __shfl_sync(0xffffffffu, wk.y, ln),
                                __shfl_sync(0xffffffffu, wk.z, ln), __shfl_sync(0xffffffffu, wk.w, ln));
    const int li = lane & 7;
    const bool vi = lane < 8 && ((vl >> li) & 1u);
    float sc = vi ? exp_shifted(row_elem(wp, li), lse2) : 0.f;
#pragma unroll
    for (int o = 1; o < 8; o <<= 1) {
      const float u = __shfl_up_sync(0xffffffffu, sc, o, 8);
      if (li >= o) sc += u;
    }
    const unsigned hit8 = __ballot_sync(0xffffffffu, vi && excl + sc >= target);
    const unsigned val8 = __ballot_sync(0xffffffffu, vi);
    const int pick_i = hit8 ? __ffs(hit8) - 1 : 31 - __clz(val8);
    const int pick = kc * 256 + ln * 8 + pick_i;
    const int kp = mm.k[pick];
    const int s_new = mm.s[pick], s_old = slot_of(cur.sa, cur.sb, kp);
    const int dk = kp + d.delta;
    const int dE = move_delta_e(s_occ[w], s_old, dk, s_new);
    unsigned char* ps = prop_slots + (size_t)c * d.n;
    if (cur.sa >= 0) ps[lane] = (unsigned char)(lane + 1 == kp ? s_new : cur.sa);
    if (cur.sb >= 0) ps[lane + 32] = (unsigned char)(lane + 33 == kp ? s_new : cur.sb);
    if (lane == 0) {
      d.prop[c] = make_int4(kp | (s_old << 8) | (s_new << 16), dE,
                            __float_as_int(row_elem(wp, pick_i) - lse), (int)rw.y);
      // the proposed configuration's occupancies
      s_occ[w][s_old] -= 1;
      s_occ[w][s_old + dk] -= 1;
      s_occ[w][s_new] += 1;
      s_occ[w][s_new + dk] += 1;
    }
    __syncwarp();
    // its network input row: four adjacent bf16 occupancies a lane (one
    // 8-byte store; bins beyond 2n are 0)
    for (int col = lane * 4; col < K1; col += 128) {
      unsigned short h[4];
#pragma unroll
      for (int i = 0; i < 4; ++i)
        h[i] = __bfloat16_as_ushort(
            __float2bfloat16(col + i < 2 * d.n ? (float)s_occ[w][col + i] : 0.f));
      *(uint2*)(X + (size_t)c * K1 + col) =
          make_uint2((unsigned)h[0] | ((unsigned)h[1] << 16), (unsigned)h[2] | ((unsigned)h[3] << 16));
    }
    __syncwarp();
    cur = nxt;
  }
}

// A chain's inputs to the accept kernel, loaded one chain ahead: the
// proposed state's logit row and configuration, the rung and the proposal
// record.
template <int CH>
struct AcceptIn {
  LogitRow<CH> r;
  int sa, sb, rung;
  int4 pr;
};

template <int CH>
__device__ __forceinline__ void load_accept_in(const LearnedDev& d, const __nv_bfloat16* Zp,
                                               const unsigned char* prop_slots, int NM, int c,
                                               int lane, AcceptIn<CH>& in) {
  load_row(Zp + (size_t)c * d.NMp, NM, lane, in.r);
  load_slots(prop_slots + (size_t)c * d.n, d.n, lane, in.sa, in.sb);
  in.rung = d.rung[c];
  in.pr = d.prop[c];
}

// Metropolis-Hastings acceptance with the proposed states' logits Zp (bf16):
// the log-normaliser of the proposed row and its logit of the reverse move
// (taken from the lane that holds it), then the decision with the uniform
// word the propose kernel drew; an accepted state keeps its row as the
// chain's current logits.  Each warp loads the next chain's inputs while it
// works on the current one.
template <int CH>
__global__ void __launch_bounds__(256, CH <= 4 ? 3 : 2)
    lt_accept_kernel(LearnedDev d, MoveTable mt, unsigned t, const unsigned char* prop_slots,
                     const __nv_bfloat16* Zp) {
  __shared__ MoveMaps mm;
  __shared__ unsigned s_bits[8][kLtChunks * 8];
  __shared__ double s_beta[kPtMaxRungsLearned];
  build_move_maps(mt, mm, 0);
  for (int i = threadIdx.x; i < d.M; i += blockDim.x) s_beta[i] = d.beta[i];
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int NM = mt.NM, stride = gridDim.x * 8;
  int c = blockIdx.x * 8 + w;
  AcceptIn<CH> cur;
  if (c < d.B) load_accept_in(d, Zp, prop_slots, NM, c, lane, cur);
  for (; c < d.B; c += stride) {
    AcceptIn<CH> nxt;
    if (c + stride < d.B) load_accept_in(d, Zp, prop_slots, NM, c + stride, lane, nxt);
    const int ladder = c / d.M, rg = cur.rung;
    LogitRow<CH>& r = cur.r;
    row_valid(mm, cur.sa, cur.sb, NM, lane, s_bits[w], r);
    const float lse_p = row_lse(r);
    // the reverse move (k, old slot): chunk, lane and element that hold it
    const int kp = cur.pr.x & 0xFF, s_old = (cur.pr.x >> 8) & 0xFF, dE = cur.pr.y;
    const int idx = mm.off[kp] + s_old;
    const int kc = idx >> 8, ln = (idx & 255) >> 3, ei = idx & 7;
    uint4 wk = make_uint4(0, 0, 0, 0);
#pragma unroll
    for (int k = 0; k < CH; ++k)
      if (k == kc) wk = r.w[k];
    const uint4 wr = make_uint4(__shfl_sync(0xffffffffu, wk.x, ln), __shfl_sync(0xffffffffu, wk.y, ln),
                                __shfl_sync(0xffffffffu, wk.z, ln), __shfl_sync(0xffffffffu, wk.w, ln));
    const float lq_rev = row_elem(wr, ei) - lse_p;
    const float log_a = (float)(-s_beta[rg] * (double)dE) + lq_rev - __int_as_float(cur.pr.z);
    const float u = ((float)(unsigned)cur.pr.w + 0.5f) * 2.3283064365386963e-10f;
    const bool acc = log_a >= 0.f || logf(u) < log_a;
    if (acc) {
      unsigned char* sl = d.slots + (size_t)c * d.n;
      if (cur.sa >= 0) sl[lane] = (unsigned char)cur.sa;
      if (cur.sb >= 0) sl[lane + 32] = (unsigned char)cur.sb;
      __nv_bfloat16* zc = d.Zcur + (size_t)c * d.NMp;
#pragma unroll
      for (int k = 0; k < CH; ++k)
        if (k * 256 + lane * 8 < NM) *(uint4*)(zc + k * 256 + lane * 8) = r.w[k];
      if (lane == 0) {
        d.lse[c] = lse_p;
        atomicAdd(&d.E[c], dE);
        atomicAdd(&d.accm[(size_t)ladder * d.M + rg], 1u);
      }
    }
    __syncwarp();
    cur = nxt;
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
  void (*propose)(LearnedDev, MoveTable, unsigned, int, unsigned char*, __nv_bfloat16*, int);
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
  for (int r = 0; r < 10; ++r) {
    d.rk[2 * r] = d.key0 + 0x9E3779B9u * (unsigned)r;
    d.rk[2 * r + 1] = d.key1 + 0xBB67AE85u * (unsigned)r;
  }
  auto al = [](size_t x) { return (x + 255) / 256 * 256; };
  size_t off = 0;
  const size_t o_sl = off; off = al(off + (size_t)B * n);
  const size_t o_E = off; off = al(off + (size_t)B * 4);
  const size_t o_r = off; off = al(off + (size_t)B * 4);
  const size_t o_lor = off; off = al(off + (size_t)B * 4);
  const size_t o_z = off; off = al(off + (size_t)B * m->NMp * 2);
  const size_t o_lse = off; off = al(off + (size_t)B * 4);
  const size_t o_pr = off; off = al(off + (size_t)B * 16);
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
    lk.propose<<<chain_grid, 256, 0, s>>>(d, mt, (unsigned)t, t >= burnin ? 1 : 0, m->slots, m->X,
                                          m->K1);
    e = mlp_forward_dev(*m, Bp, s, true, true);     // propose wrote the input rows
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
