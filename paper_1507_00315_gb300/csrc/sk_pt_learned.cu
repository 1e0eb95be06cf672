// sk_pt_learned.cu -- tempering chains whose move proposal is the trained
// network (an addition to Sec. 3; the ladder, statistics, exchanges and the
// estimator are those of Algorithm 2).  A move (k, s) is drawn from the
// softmax of the current state's logits over its valid moves; it is accepted
// with min(1, e^{-beta dE} q(C | C') / q(C' | C)) (Metropolis-Hastings), where
// q(C | C') is the probability of the reverse move (k, old slot) under the
// proposed state's logits, so the chains keep the Boltzmann weights of the
// plain ones.  Configurations live in global memory; per iteration the
// network runs once, on every proposed state, then one kernel tests every
// chain's move and draws its next one; an accepted state keeps its logits and
// per-lane weight sums, so a rejected move costs no second pass over a row.
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
  float* mx;                 // [B] the shift of their stored weight sums (the row's largest
                             //   element; its valid moves' maximum where that underflows)
  float* parts;              // [B][CH][32] per lane and chunk: sum of e^(z - mx) over the
                             //   lane's valid moves of the chunk (the current state's)
  int4* prop;                // [B] (k | old slot << 8 | new slot << 16, dE, log q(C' | C)
                             //      as float bits, the acceptance test's uniform word)
  unsigned* hist;            // [L][M][nb]
  unsigned* accm;            // [L][M]
  unsigned* accs;            // [L][M]
  const double* beta;        // [M]
  const struct MoveMaps* maps;   // the move layout tables (host_move_maps)
  const unsigned long long* tswap;   // [M][nb]
};

// Per-block tables of the move layout: the pair k and the start slot of
// every move m (moves of pair k are off[k] .. off[k+1]-1), read for the one
// move a chain draws; and the offsets off[k] themselves.  Built once per run
// on the host (host_move_maps; padding moves are pair 0, slot 0), kept in
// global memory and copied into each block's shared memory.
constexpr int kMaxMoves = 2560;        // sum_k (2n - d_k) for n <= kMlpMaxN, padded to 256
struct MoveMaps {
  __align__(16) unsigned char k[kMaxMoves];
  __align__(16) unsigned char s[kMaxMoves];
  __align__(16) int off[kPtMaxN + 4];
};
static_assert(sizeof(MoveMaps) % 16 == 0, "copied in 16-byte words");

static void host_move_maps(const MoveTable& mt, MoveMaps* mm) {
  std::memset(mm, 0, sizeof(*mm));
  for (int k = 1; k <= mt.n + 1; ++k) mm->off[k] = mt.off[k];
  for (int k = 1; k <= mt.n; ++k)
    for (int m = mt.off[k]; m < mt.off[k + 1]; ++m) {
      mm->k[m] = (unsigned char)k;
      mm->s[m] = (unsigned char)(m - mt.off[k]);
    }
}

__device__ __forceinline__ void copy_move_maps(const MoveMaps* g, MoveMaps& mm) {
  const uint4* src = (const uint4*)g;
  uint4* dst = (uint4*)&mm;
  for (int i = threadIdx.x; i < (int)(sizeof(MoveMaps) / 16); i += blockDim.x) dst[i] = __ldg(src + i);
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

// The start slot of pair k (1..n, a different pair on each lane) from the
// lanes that hold the configuration.
__device__ __forceinline__ int slot_of_lanes(int sa, int sb, int k) {
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

// The largest element of the row (valid moves or not; the words beyond the
// table hold -inf, the padding columns inside the last word 0): a shift for
// the weights that needs no masks.
template <int CH>
__device__ __forceinline__ float row_max_all(const LogitRow<CH>& r) {
  __nv_bfloat162 acc = *(const __nv_bfloat162*)&r.w[0].x;
#pragma unroll
  for (int c = 0; c < CH; ++c) {
    if (c) acc = __hmax2(acc, *(const __nv_bfloat162*)&r.w[c].x);
    acc = __hmax2(acc, *(const __nv_bfloat162*)&r.w[c].y);
    acc = __hmax2(acc, *(const __nv_bfloat162*)&r.w[c].z);
    acc = __hmax2(acc, *(const __nv_bfloat162*)&r.w[c].w);
  }
  return warp_max(fmaxf(__bfloat162float(acc.x), __bfloat162float(acc.y)));
}

// This lane's sums, per chunk, of e^(z - shift) over its valid moves (shift2
// = shift log2(e)); returns their total.
template <int CH>
__device__ __forceinline__ float row_parts(const LogitRow<CH>& r, float shift2, float* part) {
  float tot = 0.f;
#pragma unroll
  for (int c = 0; c < CH; ++c) {
    float a = 0.f;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const float e = exp_shifted(row_elem(r.w[c], i), shift2);
      a += ((r.valid[c] >> i) & 1u) ? e : 0.f;
    }
    part[c] = a;
    tot += a;
  }
  return tot;
}

// The inverse-CDF draw at u * total over the weights e^(z - shift) of the
// valid moves, taken in (lane, chunk, element) order (any fixed order gives
// the same distribution), in two parts.  draw_select: from this lane's
// per-chunk sums, an inclusive scan of the lanes' totals finds the lane whose
// running sum reaches the target and that lane's chunk sums find its chunk
// (where rounding leaves the target above every running sum: the last lane,
// and chunk, with weight).  draw_finish: lanes 0..7 hold the chunk's 8
// logits and whether each is valid; a scan of their weights picks the move
// (else the last valid one).
struct DrawSel {
  int ln, kb;          // lane and chunk holding the move
  float excl, target;  // running sum before that lane's chunk; u * total
};

template <int CH>
__device__ __forceinline__ DrawSel draw_select(const float* part, float u, int lane) {
  float lane_tot = 0.f;
#pragma unroll
  for (int k = 0; k < CH; ++k) lane_tot += part[k];
  float incl = lane_tot;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const float v = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += v;
  }
  DrawSel d;
  d.target = u * __shfl_sync(0xffffffffu, incl, 31);
  const unsigned hit = __ballot_sync(0xffffffffu, lane_tot > 0.f && incl >= d.target);
  const unsigned withw = __ballot_sync(0xffffffffu, lane_tot > 0.f);
  d.ln = hit ? __ffs(hit) - 1 : 31 - __clz(withw);
  // every lane finds the chunk it would take; lane ln's answer is used
  float run = incl - lane_tot, before = 0.f, last_before = 0.f;
  int kc = -1, klast = 0;
#pragma unroll
  for (int k = 0; k < CH; ++k) {
    if (part[k] > 0.f) {
      klast = k;
      last_before = run;
      if (kc < 0 && run + part[k] >= d.target) {
        kc = k;
        before = run;
      }
    }
    if (kc < 0) run += part[k];
  }
  if (kc < 0) {
    kc = klast;
    before = last_before;
  }
  d.kb = __shfl_sync(0xffffffffu, kc, d.ln);
  d.excl = __shfl_sync(0xffffffffu, before, d.ln);
  return d;
}

__device__ __forceinline__ int draw_finish(const DrawSel& d, float zi, bool vi, float shift2,
                                           int lane) {
  const int li = lane & 7;
  float sc = vi ? exp_shifted(zi, shift2) : 0.f;
#pragma unroll
  for (int o = 1; o < 8; o <<= 1) {
    const float v = __shfl_up_sync(0xffffffffu, sc, o, 8);
    if (li >= o) sc += v;
  }
  const unsigned hit8 = __ballot_sync(0xffffffffu, vi && d.excl + sc >= d.target);
  const unsigned val8 = __ballot_sync(0xffffffffu, vi);
  return hit8 ? __ffs(hit8) - 1 : 31 - __clz(val8);
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

constexpr float kLog2e = 1.4426950408889634f;

// Asynchronous 16-byte copy global -> shared (cp.async, L2 only) and the
// waits on this thread's own copies.
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(
                   (unsigned)__cvta_generic_to_shared(dst)),
               "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;" ::: "memory");
}
__device__ __forceinline__ void cp_async_wait_prev() {   // all groups but the newest
  asm volatile("cp.async.wait_group 1;" ::: "memory");
}

// A chain's inputs to the step kernel, loaded one chain ahead: the proposed
// configuration, the chain's rung, energy and proposal record, and its
// current state's shift and log-normaliser (registers); the proposed
// state's logit row, the current state's row and this current state's
// stored weight sums (the warp's shared-memory staging, copied
// asynchronously; nothing here waits for a load).  first: only the proposed
// (initial) rows exist.
template <int CH>
struct StepIn {
  int sa, sb, rung, E;
  float lse, mx;
  int4 pr;
};

template <int CH>
struct StepBuf {
  uint4 row[CH * 32];      // proposed state's logits, lane l's words at l, l + 32, ...
  uint4 crow[CH * 32];     // current state's logits
  float part[CH * 32];     // current state's weight sums
};

__device__ __forceinline__ void cp_async4(float* dst, const float* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(
                   (unsigned)__cvta_generic_to_shared(dst)),
               "l"(src)
               : "memory");
}

template <int CH>
__device__ __forceinline__ void load_step_in(const LearnedDev& d, const __nv_bfloat16* Zp,
                                             const unsigned char* prop_slots, int NM, int c,
                                             int lane, bool first, StepBuf<CH>& buf,
                                             StepIn<CH>& in) {
  load_slots(prop_slots + (size_t)c * d.n, d.n, lane, in.sa, in.sb);
  in.rung = d.rung[c];
  in.E = d.E[c];
  const __nv_bfloat16* z = Zp + (size_t)c * d.NMp;
#pragma unroll
  for (int k = 0; k < CH; ++k)
    if (k * 256 + lane * 8 < NM) cp_async16(&buf.row[k * 32 + lane], z + k * 256 + lane * 8);
  if (!first) {
    const __nv_bfloat16* zc = d.Zcur + (size_t)c * d.NMp;
    const float* pp = d.parts + (size_t)c * CH * 32 + lane;
#pragma unroll
    for (int k = 0; k < CH; ++k) {
      if (k * 256 + lane * 8 < NM) cp_async16(&buf.crow[k * 32 + lane], zc + k * 256 + lane * 8);
      cp_async4(&buf.part[k * 32 + lane], pp + k * 32);
    }
    in.lse = d.lse[c];
    in.mx = d.mx[c];
    in.pr = d.prop[c];
  }
  cp_async_commit();
}

// One chain step after the network's forward over the proposed states (one
// warp a chain; the next chain's inputs are fetched while the warp works).
//   * Iteration t + 1's draw is keyed by the configuration (its index l in
//     the ladder), not by its rung, so it may precede iteration t's
//     exchanges: Philox (t + 1, l, ladder, 5), word 0 the draw, word 1 the
//     next test's uniform; lane j computes the block of the warp's j-th
//     chain.
//   * The Metropolis-Hastings test, unless the bound rejects the move
//     outright (see the loop):
//     the proposed row's shift (its largest element; the maximum over the
//     valid moves if that leaves every weight below 1e-30), this lane's sums
//     of e^(z - shift) over its valid moves, the log-normaliser, the reverse
//     move's logit from the lane that holds it, and min(1, e^(-beta dE)
//     q(C | C') / q(C' | C)) against the uniform drawn with the proposal.
//     An accepted state becomes the chain's current state (configuration,
//     row, sums, shift, log-normaliser stored) and the draw runs on its sums
//     and row in registers; after a rejection it runs on the current
//     state's stored weight sums (lane and chunk), then lanes 0..7 take that
//     chunk's 8 logits from the staged current row.
//   * The drawn move's dE, its record (move, dE, log q, the next test's
//     uniform word), the proposed configuration and its network input row
//     are written for the next forward.
// first: the states in Zp are the chains' initial ones, taken unconditionally
// (nothing to test; nothing is stored yet), and the draw is iteration 0's;
// count0 counts their energies as iteration 0's statistics.  propose = 0: no
// draw (the last iteration).  Dynamic shared memory: two stagings per warp
// (StepBuf: proposed row, current row, current sums; lt_step_smem).
template <int CH>
__host__ __device__ constexpr int lt_step_smem() {
  return 8 * 2 * (int)sizeof(StepBuf<CH>);
}

template <int CH>
__global__ void __launch_bounds__(256, CH <= 3 ? 3 : 2)
    lt_step_kernel(LearnedDev d, MoveTable mt, unsigned t, int first, int propose, int count0,
                   unsigned char* prop_slots, const __nv_bfloat16* Zp, __nv_bfloat16* X, int K1) {
  __shared__ MoveMaps mm;
  __shared__ int s_occ[8][2 * kPtMaxN];
  __shared__ unsigned s_bits[8][kLtChunks * 8];
  __shared__ float s_beta[kPtMaxRungsLearned];
  extern __shared__ __align__(16) unsigned char s_dyn[];   // [warp][2] StepBuf
  // launched as a programmatic dependent of the forward's last layer: the
  // next kernel may set up now; the tables above are not written by the
  // forward, its logits are read only after it has completed
  asm volatile("griddepcontrol.launch_dependents;");
  copy_move_maps(d.maps, mm);
  for (int i = threadIdx.x; i < d.M; i += blockDim.x) s_beta[i] = (float)d.beta[i];
  __syncthreads();
  asm volatile("griddepcontrol.wait;" ::: "memory");
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, li = lane & 7;
  const int NM = mt.NM, stride = gridDim.x * 8;
  const bool fst = first != 0;
  const unsigned tn = fst ? 0u : t + 1u;             // the iteration whose move is drawn
  StepBuf<CH>* wbuf = (StepBuf<CH>*)s_dyn + 2 * w;
  int c = blockIdx.x * 8 + w;
  StepIn<CH> cur;
  if (c < d.B) load_step_in(d, Zp, prop_slots, NM, c, lane, fst, wbuf[0], cur);
  unsigned rwx = 0, rwy = 0;                         // Philox words of the warp's chain j0 + lane
  for (int j = 0; c < d.B; c += stride, ++j) {
    if ((j & 31) == 0 && propose) {
      const int cc = c + lane * stride;
      if (cc < d.B) {
        const int lc = cc / d.M;
        const uint4 rw = philox4x32_10_rk(make_uint4(tn, (unsigned)(cc - lc * d.M), (unsigned)lc, 5u), d.rk);
        rwx = rw.x;
        rwy = rw.y;
      }
    }
    const unsigned rx = __shfl_sync(0xffffffffu, rwx, j & 31);
    const unsigned ry = __shfl_sync(0xffffffffu, rwy, j & 31);
    StepIn<CH> nxt;
    if (c + stride < d.B)
      load_step_in(d, Zp, prop_slots, NM, c + stride, lane, fst, wbuf[(j + 1) & 1], nxt);
    else
      cp_async_commit();                             // keep one group per chain
    const int ladder = c / d.M, rg = cur.rung;
    int sa = cur.sa, sb = cur.sb;
    const float u = ((float)rx + 0.5f) * 2.3283064365386963e-10f;
    // the draw in case of rejection: lane, chunk, and that chunk's logits
    StepBuf<CH>& sbuf = wbuf[j & 1];
    cp_async_wait_prev();                            // this chain's staged rows and sums
    // whether the test needs the proposed row: the reverse move is valid in
    // the proposed state, so log q(C | C') <= 0 and log a <= -beta dE -
    // log q(C' | C); a uniform with log u at or above that bound (plus 1e-3
    // of rounding slack) rejects without it
    bool full = true;
    if (!fst) {
      const float ua = ((float)(unsigned)cur.pr.w + 0.5f) * 2.3283064365386963e-10f;
      const float bound = -s_beta[cur.rung] * (float)cur.pr.y - __int_as_float(cur.pr.z);
      full = __logf(ua) < bound + 1e-3f;
    }
    const int kp = cur.pr.x & 0xFF, s_old = (cur.pr.x >> 8) & 0xFF;
    bool acc = fst;
    int E = cur.E;
    LogitRow<CH> r;
    float part[CH], mx = 0.f, lse_p = 0.f;
    if (full) {
#pragma unroll
      for (int k = 0; k < CH; ++k)
        r.w[k] = k * 256 + lane * 8 < NM ? sbuf.row[k * 32 + lane]
                                         : make_uint4(0xFF80FF80u, 0xFF80FF80u, 0xFF80FF80u, 0xFF80FF80u);
      row_valid(mm, sa, sb, NM, lane, s_bits[w], r);
      mx = row_max_all(r);
      float total = warp_sum(row_parts(r, mx * kLog2e, part));
      if (!(total > 1e-30f)) {
        // rare: the valid moves' maximum instead, in rolled loops over the
        // staged row (few live registers)
        float m2 = -INFINITY;
#pragma unroll
        for (int k = 0; k < CH; ++k) {
          const unsigned short* h = (const unsigned short*)&sbuf.row[k * 32 + lane];
#pragma unroll 1
          for (int i = 0; i < 8; ++i)
            if ((r.valid[k] >> i) & 1u) m2 = fmaxf(m2, __uint_as_float((unsigned)h[i] << 16));
        }
        mx = warp_max(m2);
        total = 0.f;
#pragma unroll
        for (int k = 0; k < CH; ++k) {
          const unsigned short* h = (const unsigned short*)&sbuf.row[k * 32 + lane];
          float a = 0.f;
#pragma unroll 1
          for (int i = 0; i < 8; ++i)
            if ((r.valid[k] >> i) & 1u)
              a += exp_shifted(__uint_as_float((unsigned)h[i] << 16), mx * kLog2e);
          part[k] = a;
          total += a;
        }
        total = warp_sum(total);
      }
      lse_p = mx + __logf(total);
      if (!fst) {
        const int dE = cur.pr.y;
        const int idx = mm.off[kp] + s_old;          // the reverse move
        const int kc = idx >> 8, ln = (idx & 255) >> 3, ei = idx & 7;
        uint4 wk = r.w[0];
#pragma unroll
        for (int k = 1; k < CH; ++k)
          if (k == kc) wk = r.w[k];
        const uint4 wr = make_uint4(__shfl_sync(0xffffffffu, wk.x, ln), __shfl_sync(0xffffffffu, wk.y, ln),
                                    __shfl_sync(0xffffffffu, wk.z, ln), __shfl_sync(0xffffffffu, wk.w, ln));
        const float lq_rev = row_elem(wr, ei) - lse_p;
        const float log_a = -s_beta[rg] * (float)dE + lq_rev - __int_as_float(cur.pr.z);
        const float ua = ((float)(unsigned)cur.pr.w + 0.5f) * 2.3283064365386963e-10f;
        acc = log_a >= 0.f || __logf(ua) < log_a;
        if (acc) {
          E += dE;
          unsigned char* sl = d.slots + (size_t)c * d.n;
          if (sa >= 0) sl[lane] = (unsigned char)sa;
          if (sb >= 0) sl[lane + 32] = (unsigned char)sb;
          if (lane == 0) {
            d.E[c] = E;
            d.accm[(size_t)ladder * d.M + rg] += 1u;   // one configuration a rung and ladder
          }
        }
      } else if (count0 && lane == 0) {
        d.hist[((size_t)ladder * d.M + rg) * d.nb + E] += 1u;
      }
      if (acc) {                                     // store the new current state
        __nv_bfloat16* zc = d.Zcur + (size_t)c * d.NMp;
        float* pp = d.parts + (size_t)c * CH * 32 + lane;
#pragma unroll
        for (int k = 0; k < CH; ++k) {
          if (k * 256 + lane * 8 < NM) *(uint4*)(zc + k * 256 + lane * 8) = r.w[k];
          pp[k * 32] = part[k];
        }
        if (lane == 0) {
          d.lse[c] = lse_p;
          d.mx[c] = mx;
        }
      }
    }
    if (propose) {
      int pick;
      float zq, lse_c;
      if (acc) {
        const DrawSel sel = draw_select<CH>(part, u, lane);
        uint4 wk = r.w[0];
        unsigned vk = r.valid[0];
#pragma unroll
        for (int k = 1; k < CH; ++k)
          if (k == sel.kb) {
            wk = r.w[k];
            vk = r.valid[k];
          }
        const unsigned vl = __shfl_sync(0xffffffffu, vk, sel.ln);
        const uint4 wp = make_uint4(__shfl_sync(0xffffffffu, wk.x, sel.ln), __shfl_sync(0xffffffffu, wk.y, sel.ln),
                                    __shfl_sync(0xffffffffu, wk.z, sel.ln), __shfl_sync(0xffffffffu, wk.w, sel.ln));
        const float zi = row_elem(wp, li);
        const int pi = draw_finish(sel, zi, lane < 8 && ((vl >> li) & 1u), mx * kLog2e, lane);
        zq = __shfl_sync(0xffffffffu, zi, pi);
        pick = sel.kb * 256 + sel.ln * 8 + pi;
        lse_c = lse_p;
      } else {
        // back to the current state (pair kp at its old slot); lanes 0..7
        // test whether their move of the drawn chunk is valid there (inside
        // the table, and not the pair's current slot)
        if (lane + 1 == kp) sa = s_old;
        if (lane + 33 == kp) sb = s_old;
        float cpart[CH];
#pragma unroll
        for (int k = 0; k < CH; ++k) cpart[k] = sbuf.part[k * 32 + lane];
        const DrawSel rej = draw_select<CH>(cpart, u, lane);
        const float zrej = __uint_as_float(
            (unsigned)((const unsigned short*)&sbuf.crow[rej.kb * 32 + rej.ln])[li] << 16);
        const int m = rej.kb * 256 + rej.ln * 8 + li;
        const int km = m < NM ? mm.k[m] : 1;
        const int cs = slot_of_lanes(sa, sb, km);
        const bool vi = lane < 8 && m < NM && cs != (int)mm.s[m];
        const int pi = draw_finish(rej, zrej, vi, cur.mx * kLog2e, lane);
        zq = __shfl_sync(0xffffffffu, zrej, pi);
        pick = rej.kb * 256 + rej.ln * 8 + pi;
        lse_c = cur.lse;
      }
      place_occupancy(sa, sb, d.n, d.delta, s_occ[w], lane);
      const int kq = mm.k[pick], q_new = mm.s[pick], q_old = slot_of(sa, sb, kq);
      const int dk = kq + d.delta;
      const int dEq = move_delta_e(s_occ[w], q_old, dk, q_new);
      unsigned char* ps = prop_slots + (size_t)c * d.n;
      if (sa >= 0) ps[lane] = (unsigned char)(lane + 1 == kq ? q_new : sa);
      if (sb >= 0) ps[lane + 32] = (unsigned char)(lane + 33 == kq ? q_new : sb);
      if (lane == 0) {
        d.prop[c] = make_int4(kq | (q_old << 8) | (q_new << 16), dEq, __float_as_int(zq - lse_c),
                              (int)ry);
        // the proposed configuration's occupancies
        s_occ[w][q_old] -= 1;
        s_occ[w][q_old + dk] -= 1;
        s_occ[w][q_new] += 1;
        s_occ[w][q_new + dk] += 1;
      }
      __syncwarp();
      // its network input row: four adjacent bf16 occupancies a lane (one
      // 8-byte store; a count below 256 is exact in bf16, its float's upper
      // half), the columns of the 2n bins only -- the rest of the row stays
      // 0 from the initial states' input rows
      for (int col = lane * 4; col < 2 * d.n; col += 128) {
        unsigned h[4];
#pragma unroll
        for (int i = 0; i < 4; ++i)
          h[i] = col + i < 2 * d.n ? __float_as_uint((float)s_occ[w][col + i]) >> 16 : 0u;
        *(uint2*)(X + (size_t)c * K1 + col) = make_uint2(h[0] | (h[1] << 16), h[2] | (h[3] << 16));
      }
    }
    __syncwarp();
    cur = nxt;
  }
  asm volatile("cp.async.wait_all;" ::: "memory");
}

// Exchanges of iteration t, one warp per ladder, lane j for rung j; count:
// the energies the rungs hold afterwards are iteration t + 1's statistics.
__global__ void lt_exchange_kernel(LearnedDev d, unsigned t, int count) {
  const int lane = threadIdx.x & 31;
  const int ladder = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (ladder >= d.L) return;
  const int M = d.M;
  int* lor = d.lor + (size_t)ladder * M;
  const int my = lane < M ? lor[lane] : 0;
  const int Er = lane < M ? d.E[(size_t)ladder * M + my] : 0;
  const int En = __shfl_down_sync(0xffffffffu, Er, 1), Eu = __shfl_up_sync(0xffffffffu, Er, 1);
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
  const bool from_up = lane > 0 && dec_up;
  const int nl = dec ? down : (from_up ? up : my);
  const int nE = dec ? En : (from_up ? Eu : Er);
  if (lane < M) {
    lor[lane] = nl;
    d.rung[(size_t)ladder * M + nl] = lane;
    if (count) d.hist[((size_t)ladder * M + lane) * d.nb + nE] += 1u;
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
  void (*step)(LearnedDev, MoveTable, unsigned, int, int, int, unsigned char*,
               const __nv_bfloat16*, __nv_bfloat16*, int);
  int smem;                      // the step kernel's dynamic shared memory
};
static bool lt_kernels(int ch, LtKernels* k) {
  switch (ch) {
#define SK_LT_CASE(c) \
  case c: *k = {lt_step_kernel<c>, lt_step_smem<c>()}; return true;
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
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
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
  const size_t o_mx = off; off = al(off + (size_t)B * 4);
  const int CHn = (m->NMp + 255) / 256;   // >= the move table's chunks
  const size_t o_pa = off; off = al(off + (size_t)B * CHn * 32 * 4);
  const size_t o_pr = off; off = al(off + (size_t)B * 16);
  const size_t o_h = off; off = al(off + (size_t)L * M * nb * 4);
  const size_t o_am = off; off = al(off + (size_t)L * M * 4);
  const size_t o_as = off; off = al(off + (size_t)L * M * 4);
  const size_t o_b = off; off = al(off + (size_t)M * 8);
  const size_t o_mm = off; off = al(off + sizeof(MoveMaps));
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
  d.mx = (float*)(p + o_mx);
  d.parts = (float*)(p + o_pa);
  d.prop = (int4*)(p + o_pr);
  d.hist = (unsigned*)(p + o_h);
  d.accm = (unsigned*)(p + o_am);
  d.accs = (unsigned*)(p + o_as);
  d.beta = (const double*)(p + o_b);
  d.maps = (const MoveMaps*)(p + o_mm);
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
  e = cudaFuncSetAttribute((const void*)lk.step, cudaFuncAttributeMaxDynamicSharedMemorySize, lk.smem);
  // the step kernel loops over chains, 8 per block: one wave of the blocks
  // that fit on the device at once (no part-empty last wave)
  int resident = 0;
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&resident, (const void*)lk.step, 256, lk.smem);
  const int chain_grid =
      std::max(1, std::min((B + 7) / 8, std::max(resident, 1) * (sms > 0 ? sms : 1)));
  if (e == cudaSuccess) e = cudaMemsetAsync(p + o_h, 0, o_b - o_h, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(p + o_b, beta, (size_t)M * 8, cudaMemcpyHostToDevice, s);
  MoveMaps hmm;
  host_move_maps(mt, &hmm);
  if (e == cudaSuccess) e = cudaMemcpyAsync(p + o_mm, &hmm, sizeof(hmm), cudaMemcpyHostToDevice, s);
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
  // the initial states' forward, then their rows kept and iteration 0's draw
  if (e == cudaSuccess) e = mlp_forward_dev(*m, Bp, s, true);
  if (e == cudaSuccess) {
    lk.step<<<chain_grid, 256, lk.smem, s>>>(d, mt, 0u, 1, iters > 0 ? 1 : 0,
                                       iters > 0 && burnin == 0 ? 1 : 0, m->slots, Zb, m->X, m->K1);
    e = cudaGetLastError();
  }
  // The exchanges of iteration t run on a side stream beside the first layer
  // of iteration t + 1 (which reads only the input rows and the weights); the
  // stream joins them before the second layer, ahead of the step kernel of
  // t + 1 (it reads the rungs and writes the energies they read).
  cudaStream_t xs = nullptr;
  cudaEvent_t ev_step = nullptr, ev_exch = nullptr;
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&xs, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev_step, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev_exch, cudaEventDisableTiming);
  // Per iteration: layer 1, the join with the previous exchanges, layers 2
  // and 3 and the step kernel each launched as a programmatic dependent of
  // the kernel before it (it sets up while that one finishes).
  for (uint64_t t = 0; t < iters && e == cudaSuccess; ++t) {
    // the step kernel wrote the input rows
    e = mlp_forward_dev(*m, Bp, s, true, true, t > 0 ? ev_exch : nullptr, true);
    if (e != cudaSuccess) break;
    const bool more = t + 1 < iters;
    e = launch_dependent(lk.step, chain_grid, 256, (size_t)lk.smem, s, d, mt, (unsigned)t, 0,
                         more ? 1 : 0, 0, m->slots, Zb, m->X, m->K1);
    if (e == cudaSuccess) e = cudaEventRecord(ev_step, s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(xs, ev_step, 0);
    if (e != cudaSuccess) break;
    lt_exchange_kernel<<<(L + 3) / 4, 128, 0, xs>>>(d, (unsigned)t,
                                                    more && t + 1 >= burnin ? 1 : 0);
    e = cudaEventRecord(ev_exch, xs);
    if (e == cudaSuccess) e = cudaGetLastError();
  }
  if (e == cudaSuccess && iters > 0) e = cudaStreamWaitEvent(s, ev_exch, 0);
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
  if (e != cudaSuccess && xs) cudaStreamSynchronize(xs);   // nothing of it left in flight
  if (ev_step) cudaEventDestroy(ev_step);
  if (ev_exch) cudaEventDestroy(ev_exch);
  if (xs) cudaStreamDestroy(xs);
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
