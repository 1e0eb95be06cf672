// sk_pt.cu -- the parallel-tempering kernel (Sec. 3, Algorithm 2) and its
// host runtime: thresholds, ladder tuning, the estimator, the C ABI.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <limits>
#include <vector>

#include "sk_host_common.h"
#include "sk_pt.cuh"

namespace sk {

// Barrier of the two warps of ladder `lw` (0 or 1) of a block of 4 warps:
// named barriers 1 and 2, 64 threads (constant ids, so the kernel reserves
// three barriers, not sixteen).
__device__ __forceinline__ void ladder_pair_sync(int lw) {
  if (lw == 0)
    asm volatile("bar.sync 1, 64;" ::: "memory");
  else
    asm volatile("bar.sync 2, 64;" ::: "memory");
}

// Per-warp view of one ladder's tables and this lane's per-rung constants.
// A ladder has W warps (W = 1: up to 32 rungs; W = 2: up to 64): lane j of
// warp h serves rung 32 h + j, and the tables have C = 32 W columns.
struct PtLane {
  unsigned short* hist;                 // [E][C]
  unsigned char* slot;                  // [k][C], k = 1..n
  unsigned char* occ;                   // [b][C]
  unsigned char* dir;                   // [C]: the last end of the ladder each column's
                                        // configuration sat at (0 none, 1 rung 0, 2 rung M-1)
  unsigned long long tm1, tm2;          // move thresholds at this lane's rung, dE = 1, 2
  const unsigned long long* tswap;      // [M][bins+1]
  int rung, M, n, delta, bins, nb;
  unsigned burnin;
  bool active;                          // rung < M
  // W = 2: the rung pair (31, 32) across the two warps meets in `xs`
  // (double-buffered by iteration parity) at named barrier `bar`
  unsigned* xs;                         // [2][3]: pk of rung 31, its word 3, pk of rung 32
  int lw;                               // ladder of the block
};

// Iteration t at rung S.rung, Philox block wc: the energy statistic, one
// Metropolis move of the configuration in column c (energy E), then the
// exchange of this rung's pair (j, j+1), j = t mod 2.  Branch-free: every
// store and the threshold load happen, with unchanged values where a move
// or exchange is rejected.  With two warps a ladder, the pair (31, 32) is
// exchanged through shared memory on odd iterations, after a barrier of the
// two warps (also the point where the columns that change warp become the
// other warp's).  TRIPS: first the lanes at the two ends of the ladder look
// at their configurations -- at rung 0 a configuration that has reached rung
// M-1 since it was last there completes a round trip (counted from `burnin`
// on), at rung M-1 one that came from rung 0 is marked.
template <int W, bool TRIPS>
__device__ __forceinline__ void pt_step(const PtLane& S, const uint4 wc, const unsigned t, int& c,
                                        int& E, unsigned& accm, unsigned& accs, unsigned& trips) {
  constexpr int C = 32 * W;
  if constexpr (TRIPS) {
    if (S.rung == 0 || S.rung == S.M - 1) {
      const int dv = S.dir[c];
      if (S.rung == 0) {
        trips += (unsigned)(dv == 2 && t >= S.burnin);
        S.dir[c] = 1;
      } else if (dv == 1) {
        S.dir[c] = 2;
      }
    }
  }
  unsigned xw_lo = __shfl_up_sync(0xffffffffu, wc.w, 1);          // word 3 of rung - 1
  S.hist[E * C + S.rung] += (unsigned short)(S.active && t >= S.burnin);
  // Metropolis move: pair k to another start slot
  const int k = 1 + (int)__umulhi(wc.x, (unsigned)S.n);
  const int d = k + S.delta;
  const int L = S.bins - d;
  unsigned char* sk = &S.slot[k * C + c];
  const int s_old = *sk;
  // L = 1 (Langford n = 2, k = 2): no other slot; s_new = s_old keeps the
  // reads inside the table and the move is never taken
  int s_new = s_old;
  if (L >= 2) {
    s_new = (int)__umulhi(wc.y, (unsigned)(L - 1));
    s_new += s_new >= s_old;
  }
  unsigned char* o1 = &S.occ[s_old * C + c];
  unsigned char* o2 = &S.occ[(s_old + d) * C + c];
  unsigned char* o3 = &S.occ[s_new * C + c];
  unsigned char* o4 = &S.occ[(s_new + d) * C + c];
  const int a1 = *o1, a2 = *o2, a3 = *o3, a4 = *o4;
  // dE: taking the pair out empties the bins it was alone in; putting it
  // back fills the empty bins it lands on (a new bin may be the old pair's
  // other bin: s_new = s_old + d or s_new + d = s_old)
  const int b3 = a3 - (s_new == s_old + d);
  const int b4 = a4 - (s_new + d == s_old);
  const int dE = (a1 == 1) + (a2 == 1) - (b3 == 0) - (b4 == 0);
  const unsigned long long thr = dE <= 0 ? (1ull << 32) : (dE == 1 ? S.tm1 : S.tm2);
  const bool acc = S.active && L >= 2 && (unsigned long long)wc.z < thr;
  // counts written in this order are right when bins coincide: o3 == o2
  // ends at b3 + 1 = a2, o4 == o1 at b4 + 1 = a1
  const int ai = acc;
  *o1 = (unsigned char)(a1 - ai);
  *o2 = (unsigned char)(a2 - ai);
  *o3 = (unsigned char)(acc ? b3 + 1 : a3);
  *o4 = (unsigned char)(acc ? b4 + 1 : a4);
  *sk = (unsigned char)(acc ? s_new : s_old);
  E += acc ? dE : 0;
  accm += ai;
  __syncwarp();
  // exchange: both lanes of a pair take the same decision from the lower
  // rung's word 3
  const int pk = (E << 8) | c;
  int dn = __shfl_down_sync(0xffffffffu, pk, 1);
  int up = __shfl_up_sync(0xffffffffu, pk, 1);
  if constexpr (W == 2) {
    if (t & 1u) {                                     // the pair (31, 32) is active
      unsigned* x = S.xs + 3 * (int)((t >> 1) & 1u);
      if (S.rung == 31) { x[0] = (unsigned)pk; x[1] = wc.w; }
      if (S.rung == 32) x[2] = (unsigned)pk;
      ladder_pair_sync(S.lw);
      if (S.rung == 31) dn = (int)x[2];
      if (S.rung == 32) { up = (int)x[0]; xw_lo = x[1]; }
    }
  }
  const int par = (S.rung ^ (int)t) & 1;              // 0: lower rung of its pair, 1: upper
  const int row = S.rung - par;                       // the pair (row, row + 1)
  const bool valid = row >= 0 && row + 1 < S.M;
  const int o = par ? up : dn;
  const int de = par ? (o >> 8) - E : E - (o >> 8);
  const unsigned xw = par ? xw_lo : wc.w;
  const unsigned long long T = __ldg(S.tswap + (valid ? row : 0) * S.nb + (de > 0 ? de : 0));
  const bool dec = valid && (de <= 0 || (unsigned long long)xw < T);
  c = dec ? (o & 0xff) : c;
  E = dec ? (o >> 8) : E;
  accs += dec && !par;
}

// W warps = one ladder (W = 1: up to 32 rungs, W = 2: up to 64); persistent
// over ladders.  Per iteration t, in the order of Algorithm 2: the energy
// statistics of every rung (after burn-in), one Metropolis move per
// configuration, then the exchanges of the pairs (j, j+1) with j = t mod 2.
// Lane j of warp h serves rung 32 h + j (see sk_pt.cuh): it holds the column
// c of the configuration now at that rung and its energy E.  TRIPS: the
// round trips of the configurations between the ends of the ladder are
// counted into *trips_g.
template <int W, bool TRIPS>
__global__ void __launch_bounds__(128, 7)
    pt_kernel(PtParams p, const unsigned long long* __restrict__ tmove_g,
              const unsigned long long* __restrict__ tswap_g, unsigned long long* hist_g,
              unsigned long long* accm_g, unsigned long long* accs_g, unsigned char* final_slots,
              unsigned long long* trips_g) {
  constexpr int C = 32 * W;
  extern __shared__ __align__(16) unsigned char pt_smem[];
  __shared__ unsigned xslot[2][6];                    // W = 2: per ladder of the block
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int lw = warp / W, h = warp % W;              // ladder of the block, warp in the ladder
  const int rung = 32 * h + lane;
  const int M = p.M, n = p.n, bins = p.bins, nb = bins + 1;
  unsigned char* wbase = pt_smem + (size_t)lw * pt_ladder_bytes(n, W);
  PtLane S;
  S.hist = (unsigned short*)wbase;
  S.slot = wbase + pt_hist_bytes(n, W);
  S.occ = S.slot + (n + 1) * C;
  S.dir = S.occ + bins * C;
  S.rung = rung;
  S.M = M;
  S.n = n;
  S.delta = p.delta;
  S.bins = bins;
  S.nb = nb;
  S.burnin = p.burnin;
  S.active = rung < M;
  S.tm1 = S.active ? __ldg(&tmove_g[rung * 2]) : 0ull;
  S.tm2 = S.active ? __ldg(&tmove_g[rung * 2 + 1]) : 0ull;
  S.tswap = tswap_g;
  S.xs = xslot[lw & 1];
  S.lw = lw;
  unsigned short* hist = S.hist;
  unsigned char* slot = S.slot;
  unsigned char* occ = S.occ;
  const bool active = S.active;
  const int lpb = p.warps_per_block / W;              // ladders per block
  for (int ladder = blockIdx.x * lpb + lw; ladder < p.ladders; ladder += gridDim.x * lpb) {
    for (int e = 0; e < nb; ++e) hist[e * C + rung] = 0;
    for (int b = 0; b < bins; ++b) occ[b * C + rung] = 0;
    for (int k = 0; k <= n; ++k) slot[k * C + rung] = 0;
    S.dir[rung] = 0;
    // column `rung` <- the configuration that starts at that rung
    int c = rung, E = 0;
    unsigned accm = 0, accs = 0, trips = 0;
    if (active) {
      for (int k = 1; k <= n; ++k) {
        const unsigned L = (unsigned)(bins - (k + p.delta));
        const uint4 w = philox4x32_10_rk(
            make_uint4((unsigned)k, (unsigned)rung, (unsigned)ladder, 1u), p.rk);
        const int s = (int)__umulhi(w.x, L);
        slot[k * C + rung] = (unsigned char)s;
        occ[s * C + rung] += 1;
        occ[(s + k + p.delta) * C + rung] += 1;
      }
      for (int b = 0; b < bins; ++b) E += occ[b * C + rung] == 0;
    }
    __syncwarp();
    for (unsigned long long t0 = 0; t0 < p.iters; t0 += kPtFlush) {
      const unsigned t1 = (unsigned)(t0 + kPtFlush < p.iters ? t0 + kPtFlush : p.iters);
      // two iterations a trip, each one's Philox block computed while the
      // other waits on shared memory (the blocks do not depend on the state)
      uint4 wa = philox4x32_10_rk(make_uint4((unsigned)t0, (unsigned)rung, (unsigned)ladder, 2u), p.rk);
      unsigned t = (unsigned)t0;
      for (; t + 1 < t1; t += 2) {
        const uint4 wb = philox4x32_10_rk(make_uint4(t + 1u, (unsigned)rung, (unsigned)ladder, 2u), p.rk);
        pt_step<W, TRIPS>(S, wa, t, c, E, accm, accs, trips);
        wa = philox4x32_10_rk(make_uint4(t + 2u, (unsigned)rung, (unsigned)ladder, 2u), p.rk);
        pt_step<W, TRIPS>(S, wb, t + 1, c, E, accm, accs, trips);
      }
      if (t < t1) pt_step<W, TRIPS>(S, wa, t, c, E, accm, accs, trips);
      if (t1 < p.iters && active) {                // 16-bit counters: flush this rung's column
        unsigned long long* hist_l =
            hist_g + (size_t)pt_group(ladder, p.ladders, p.groups) * M * nb;
        for (int e = 0; e < nb; ++e) {
          const unsigned v = hist[e * C + rung];
          if (v) { atomicAdd(&hist_l[(size_t)rung * nb + e], (unsigned long long)v); hist[e * C + rung] = 0; }
        }
      }
    }
    if constexpr (W == 2) ladder_pair_sync(lw);
    // flush this ladder
    if (active) {
      unsigned long long* hist_l = hist_g + (size_t)pt_group(ladder, p.ladders, p.groups) * M * nb;
      for (int e = 0; e < nb; ++e) {
        const unsigned v = hist[e * C + rung];
        if (v) atomicAdd(&hist_l[(size_t)rung * nb + e], (unsigned long long)v);
      }
      if (accm) atomicAdd(&accm_g[rung], (unsigned long long)accm);
      if (accs) atomicAdd(&accs_g[rung], (unsigned long long)accs);
      if (TRIPS && trips) atomicAdd(trips_g, (unsigned long long)trips);
      if (final_slots)
        for (int k = 1; k <= n; ++k)
          final_slots[((size_t)ladder * M + rung) * n + (k - 1)] = slot[k * C + c];
    }
    if constexpr (W == 2) ladder_pair_sync(lw);
    __syncwarp();
  }
}

}  // namespace sk

// ===================================================================== host

namespace sk {

// ceil(p 2^32) with p = e^{-x}, x > 0; 2^32 means "always".
unsigned long long accept_threshold(double x) {
  const double p = std::exp(-x);
  const double t = std::ceil(std::ldexp(p, 32));
  if (t >= 4294967296.0) return 1ULL << 32;
  return (unsigned long long)t;
}

namespace {

int pt_check(int variant, int n, int M, const double* beta, int L) {
  if (variant != SK_SKOLEM && variant != SK_LANGFORD) return SK_EINVAL;
  if (n < 2 || n > kPtMaxN || M < 1 || M > kPtMaxRungs || L < 1 || !beta) return SK_EINVAL;
  const int delta = variant == SK_LANGFORD ? 1 : 0;
  for (int k = 1; k <= n; ++k)
    if (2 * n - (k + delta) < 1) return SK_EINVAL;
  for (int j = 0; j < M; ++j) {
    if (!(beta[j] >= 0.0) || !std::isfinite(beta[j])) return SK_EINVAL;
    if (j && beta[j] < beta[j - 1]) return SK_EINVAL;
  }
  return SK_OK;
}

}  // namespace

// Runs L ladders for `iters` iterations; host outputs as in the header.
// With groups > 1 the histograms are also kept per group of ladders
// (group_hist: groups x M x (2n+1), host), hist being their sum.  With
// round_trips (host, one value) the kernel also counts the round trips of
// the configurations between the ends of the ladder.
int pt_run_impl(int variant, int n, int M, const double* beta, int L, uint64_t iters,
                uint64_t burnin, uint64_t seed, uint64_t* hist, uint64_t* accm, uint64_t* accs,
                uint8_t* final_slots, void* stream, double* kernel_ms, int groups = 1,
                uint64_t* group_hist = nullptr, uint64_t* round_trips = nullptr) {
  int st = pt_check(variant, n, M, beta, L);
  if (st) return st;
  if (!hist || iters > 0xffffffffULL || groups < 1 || groups > L || (groups > 1 && !group_hist))
    return SK_EINVAL;
  st = check_device();
  if (st) return st;
  const int bins = 2 * n, nb = bins + 1;
  // thresholds: moves [M][dE = 1, 2], exchanges [M][de]
  std::vector<unsigned long long> tm((size_t)M * 2, 0), ts((size_t)M * nb, 0);
  for (int j = 0; j < M; ++j) {
    for (int de = 1; de <= 2; ++de) tm[j * 2 + de - 1] = accept_threshold(beta[j] * (double)de);
    if (j + 1 < M)
      for (int de = 1; de <= bins; ++de)
        ts[j * nb + de] = accept_threshold((beta[j + 1] - beta[j]) * (double)de);
  }
  PtParams p;
  p.n = n;
  p.delta = variant == SK_LANGFORD ? 1 : 0;
  p.M = M;
  p.bins = bins;
  p.ladders = L;
  const int W = M > 32 ? 2 : 1;                  // warps a ladder
  p.warps_per_block = 4;
  p.iters = (unsigned)iters;
  p.burnin = (unsigned)std::min<uint64_t>(burnin, iters);
  p.key0 = (unsigned)seed;
  p.key1 = (unsigned)(seed >> 32);
  for (int r = 0; r < 10; ++r) {
    p.rk[2 * r] = p.key0 + 0x9E3779B9u * (unsigned)r;
    p.rk[2 * r + 1] = p.key1 + 0xBB67AE85u * (unsigned)r;
  }
  p.groups = groups;
  const size_t n_hist = (size_t)groups * M * nb, n_fin = final_slots ? (size_t)L * M * n : 0;
  const size_t bytes = (tm.size() + ts.size() + n_hist + 2 * (size_t)M + 1) * 8 + n_fin;
  cudaStream_t s = (cudaStream_t)stream;
  bool own = false;
  if (!s) {
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) return SK_ECUDA;
    own = true;
  }
  unsigned long long* d = nullptr;
  cudaError_t e = cudaMalloc(&d, bytes);
  if (e != cudaSuccess) {
    if (own) cudaStreamDestroy(s);
    return cuda_status(e);
  }
  unsigned long long* dtm = d;
  unsigned long long* dts = dtm + tm.size();
  unsigned long long* dh = dts + ts.size();
  unsigned long long* dam = dh + n_hist;
  unsigned long long* das = dam + M;
  unsigned long long* dtrips = das + M;
  unsigned char* dfin = final_slots ? (unsigned char*)(dtrips + 1) : nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  e = cudaMemcpyAsync(dtm, tm.data(), tm.size() * 8, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dts, ts.data(), ts.size() * 8, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(dh, 0, (n_hist + 2 * (size_t)M + 1) * 8, s);
  const size_t smem = pt_smem_bytes(n, W, p.warps_per_block);
  const bool trips = round_trips != nullptr;
  const auto kernel = W == 2 ? (trips ? pt_kernel<2, true> : pt_kernel<2, false>)
                             : (trips ? pt_kernel<1, true> : pt_kernel<1, false>);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, 32 * p.warps_per_block, smem);
  int grid = sms * (per_sm > 0 ? per_sm : 1);
  const int lpb = p.warps_per_block / W;
  const int need = (L + lpb - 1) / lpb;
  if (grid > need) grid = need;
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e == cudaSuccess) e = cudaEventRecord(e0, s);
  if (e == cudaSuccess) {
    kernel<<<grid, 32 * p.warps_per_block, smem, s>>>(p, dtm, dts, dh, dam, das, dfin, dtrips);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaEventRecord(e1, s);
  std::vector<unsigned long long> hh(n_hist + 2 * (size_t)M + 1);
  if (e == cudaSuccess) e = cudaMemcpyAsync(hh.data(), dh, hh.size() * 8, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess && final_slots)
    e = cudaMemcpyAsync(final_slots, dfin, n_fin, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  float ms = 0.f;
  if (e == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(d);
  if (own) cudaStreamDestroy(s);
  if (e != cudaSuccess) return cuda_status(e);
  const size_t per = (size_t)M * nb;
  for (size_t i = 0; i < per; ++i) {
    unsigned long long v = 0;
    for (int g = 0; g < groups; ++g) v += hh[(size_t)g * per + i];
    hist[i] = v;
  }
  if (groups > 1)
    for (size_t i = 0; i < n_hist; ++i) group_hist[i] = hh[i];
  for (int j = 0; j < M; ++j) {
    if (accm) accm[j] = hh[n_hist + j];
    if (accs) accs[j] = hh[n_hist + M + j];
  }
  if (round_trips) *round_trips = hh[n_hist + 2 * (size_t)M];
  if (kernel_ms) *kernel_ms = ms;
  return SK_OK;
}

// Sec. 3: S ~ 1/2 Z(0) prod_j Ratio(j); Ratio(j) = mean of
// e^{-(beta_{j+1} - beta_j) E} at rung j, and for the last rung
// (beta_{M+1} = infinity) the fraction of samples with E = 0.
double pt_estimate_from_hist(int variant, int n, int M, const double* beta, const uint64_t* hist,
                             double* ratios) {
  const int nb = 2 * n + 1, delta = variant == SK_LANGFORD ? 1 : 0;
  long double logs = std::log(0.5L);
  for (int k = 1; k <= n; ++k) logs += std::log((long double)(2 * n - (k + delta)));
  for (int j = 0; j < M; ++j) {
    long double tot = 0, acc = 0;
    for (int E = 0; E < nb; ++E) {
      const long double h = (long double)hist[j * nb + E];
      tot += h;
      if (j + 1 < M) acc += h * std::exp(-(long double)(beta[j + 1] - beta[j]) * E);
      else if (E == 0) acc += h;
    }
    const long double rr = tot > 0 ? acc / tot : 0;
    if (ratios) ratios[j] = (double)rr;
    logs += std::log(rr);
  }
  return (double)std::exp(logs);
}

// Pooled estimate of `groups` histograms (groups x M x (2n+1)) and, with
// groups >= 2, the relative standard error of it: the sample standard
// deviation of the group estimates over their mean and sqrt(groups) (NaN
// when the mean is 0).
double pt_pooled_estimate(int variant, int n, int M, const double* beta, int groups,
                          const uint64_t* ghist, double* ratios, double* rel_stderr) {
  const size_t per = (size_t)M * (2 * n + 1);
  std::vector<uint64_t> pooled(per, 0);
  for (int g = 0; g < groups; ++g)
    for (size_t i = 0; i < per; ++i) pooled[i] += ghist[(size_t)g * per + i];
  const double est = pt_estimate_from_hist(variant, n, M, beta, pooled.data(), ratios);
  if (rel_stderr) {
    *rel_stderr = 0.0;
    if (groups > 1) {
      std::vector<double> eg(groups);
      double mean = 0.0;
      for (int g = 0; g < groups; ++g) {
        eg[g] = pt_estimate_from_hist(variant, n, M, beta, ghist + (size_t)g * per, nullptr);
        mean += eg[g] / groups;
      }
      double var = 0.0;
      for (int g = 0; g < groups; ++g) var += (eg[g] - mean) * (eg[g] - mean) / (groups - 1);
      *rel_stderr = mean > 0.0 ? std::sqrt(var / groups) / mean
                               : std::numeric_limits<double>::quiet_NaN();
    }
  }
  return est;
}

}  // namespace sk

extern "C" int sk_pt_estimate_hist(int variant, int n, int M, const double* beta, int groups,
                                   const uint64_t* hist, double* out, double* ratios,
                                   double* rel_stderr) {
  if (variant != SK_SKOLEM && variant != SK_LANGFORD) return SK_EINVAL;
  if (n < 2 || n > sk::kPtMaxN || M < 1 || M > sk::kPtMaxRungs || groups < 1) return SK_EINVAL;
  if (!beta || !hist || !out) return SK_EINVAL;
  for (int j = 0; j < M; ++j) {
    if (!(beta[j] >= 0.0) || !std::isfinite(beta[j])) return SK_EINVAL;
    if (j && beta[j] < beta[j - 1]) return SK_EINVAL;
  }
  *out = sk::pt_pooled_estimate(variant, n, M, beta, groups, hist, ratios, rel_stderr);
  return SK_OK;
}

extern "C" int sk_pt_run(int variant, int n, int M, const double* beta, int L, uint64_t iters,
                         uint64_t burnin, uint64_t seed, uint64_t* hist, uint64_t* acc_move,
                         uint64_t* acc_swap, uint8_t* final_slots) {
  return sk::pt_run_impl(variant, n, M, beta, L, iters, burnin, seed, hist, acc_move, acc_swap,
                         final_slots, nullptr, nullptr);
}

extern "C" int sk_pt_run_trips(int variant, int n, int M, const double* beta, int L,
                               uint64_t iters, uint64_t burnin, uint64_t seed, uint64_t* hist,
                               uint64_t* acc_move, uint64_t* acc_swap, uint8_t* final_slots,
                               uint64_t* round_trips) {
  if (!round_trips) return SK_EINVAL;
  return sk::pt_run_impl(variant, n, M, beta, L, iters, burnin, seed, hist, acc_move, acc_swap,
                         final_slots, nullptr, nullptr, 1, nullptr, round_trips);
}

namespace sk {

// Pilot-tuned ladder: beta_0 = 0 and beta_{M-1} = beta_max fixed; the inner
// temperatures are moved so that every neighbour pair has the same
// -log(exchange acceptance) (Sec. 3 asks for acceptance >= 1/2 with few
// temperatures); a few short pilot runs, each re-spacing the ladder along
// the cumulative -log acceptance.
int tune_ladder(int variant, int n, int M, double beta_max, uint64_t seed, void* stream,
                double* beta) {
  if (M < 2) {
    beta[0] = 0.0;
    return SK_OK;
  }
  for (int j = 0; j < M; ++j) {            // start: dense at small beta
    const double x = (double)j / (M - 1);
    beta[j] = beta_max * (std::exp(3.0 * x) - 1.0) / (std::exp(3.0) - 1.0);
  }
  const int nb = 2 * n + 1, L = 256;
  const uint64_t iters = 4096, burn = 512;
  std::vector<uint64_t> hist((size_t)M * nb), am(M), as(M);
  for (int round = 0; round < 5; ++round) {
    int st = pt_run_impl(variant, n, M, beta, L, iters, burn, seed + 7919 * (round + 1),
                         hist.data(), am.data(), as.data(), nullptr, stream, nullptr);
    if (st) return st;
    std::vector<double> C(M, 0.0);
    for (int j = 0; j + 1 < M; ++j) {
      const double tries = (double)L * (double)((iters + ((j & 1) ? 0 : 1)) / 2);
      double a = as[j] / tries;
      a = std::min(std::max(a, 0.02), 0.999);
      C[j + 1] = C[j] - std::log(a);
    }
    std::vector<double> nbeta(M);
    nbeta[0] = 0.0;
    nbeta[M - 1] = beta_max;
    for (int k = 1; k + 1 < M; ++k) {
      const double target = C[M - 1] * k / (M - 1);
      int j = 0;
      while (j + 2 < M && C[j + 1] < target) ++j;
      const double span = C[j + 1] - C[j];
      const double f = span > 0 ? (target - C[j]) / span : 0.0;
      nbeta[k] = beta[j] + f * (beta[j + 1] - beta[j]);
    }
    for (int k = 1; k < M; ++k) nbeta[k] = std::max(nbeta[k], nbeta[k - 1]);
    for (int k = 0; k < M; ++k) beta[k] = nbeta[k];
  }
  return SK_OK;
}

int pt_estimate_impl(int variant, int n, uint64_t budget, const sk_pt_opts* o, double* out,
                     sk_pt_report* rep) {
  auto t0 = std::chrono::steady_clock::now();
  if (!out || budget == 0 || budget > 0xffffffffULL) return SK_EINVAL;
  const int M = (o && o->rungs) ? o->rungs : 32;
  const int L = (o && o->ladders) ? o->ladders : 4096;
  const uint64_t seed = o ? o->seed : 0;
  const double bf = (o && o->burnin_frac != 0.0) ? o->burnin_frac : 0.1;
  const uint64_t burnin = bf < 0 ? 0 : (uint64_t)(bf * (double)budget);
  const int proposal = o ? o->proposal : SK_PT_PLAIN;
  if (M < 1 || M > kPtMaxRungs || L < 1 || burnin >= budget) return SK_EINVAL;
  if (proposal != SK_PT_PLAIN && proposal != SK_PT_LEARNED) return SK_EINVAL;
  if (proposal == SK_PT_LEARNED && M > kPtMaxRungsLearned) return SK_EINVAL;
  if (variant != SK_SKOLEM && variant != SK_LANGFORD) return SK_EINVAL;
  if (n < 2 || n > kPtMaxN) return SK_EINVAL;
  std::vector<double> beta(M);
  if (o && o->beta) {
    for (int j = 0; j < M; ++j) beta[j] = o->beta[j];
  } else {
    const double bmax = (o && o->beta_max > 0) ? o->beta_max : 32.0;
    int st = tune_ladder(variant, n, M, bmax, seed ^ 0x5DEECE66DULL, o ? o->stream : nullptr,
                         beta.data());
    if (st) return st;
  }
  auto t1 = std::chrono::steady_clock::now();
  const int nb = 2 * n + 1;
  std::vector<uint64_t> hist((size_t)M * nb), am(M), as(M);
  // plain chains: histograms per group of ladders for the standard error
  const int groups = proposal == SK_PT_LEARNED ? 1 : std::min(kPtErrorGroups, L);
  std::vector<uint64_t> ghist(groups > 1 ? (size_t)groups * M * nb : 0);
  double kms = 0.0;
  int st;
  if (proposal == SK_PT_LEARNED)
    st = pt_learned_run(variant, n, M, beta.data(), L, budget, burnin, seed, o->model, hist.data(),
                        am.data(), as.data(), o ? o->stream : nullptr, &kms);
  uint64_t trips = 0;
  const bool want_trips = o && o->round_trips && proposal == SK_PT_PLAIN;
  if (proposal == SK_PT_PLAIN)
    st = pt_run_impl(variant, n, M, beta.data(), L, budget, burnin, seed, hist.data(), am.data(),
                     as.data(), nullptr, o ? o->stream : nullptr, &kms, groups, ghist.data(),
                     want_trips ? &trips : nullptr);
  if (st) return st;
  double ratios[kPtMaxRungs];
  double rel_se = 0.0;
  const double est = groups > 1
      ? pt_pooled_estimate(variant, n, M, beta.data(), groups, ghist.data(), ratios, &rel_se)
      : pt_estimate_from_hist(variant, n, M, beta.data(), hist.data(), ratios);
  *out = est;
  if (rep) {
    std::memset(rep, 0, sizeof(*rep));
    rep->rungs = M;
    rep->ladders = L;
    rep->iterations = budget;
    rep->burnin = burnin;
    for (int j = 0; j < M; ++j) {
      rep->beta[j] = beta[j];
      rep->ratio[j] = ratios[j];
      rep->acc_move[j] = (double)am[j] / ((double)L * (double)budget);
      const double tries = (double)L * (double)((budget + ((j & 1) ? 0 : 1)) / 2);
      rep->acc_swap[j] = j + 1 < M ? (double)as[j] / tries : 0.0;
    }
    rep->estimate = est;
    rep->rel_stderr = rel_se;
    rep->round_trips = trips;
    rep->kernel_ms = kms;
    rep->tune_ms = std::chrono::duration<double, std::milli>(t1 - t0).count();
    rep->wall_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  }
  return SK_OK;
}

}  // namespace sk

extern "C" int pt_estimate(int variant, int n, uint64_t budget, double* out) {
  return sk::pt_estimate_impl(variant, n, budget, nullptr, out, nullptr);
}

extern "C" int pt_estimate_ex(int variant, int n, uint64_t budget, const sk_pt_opts* opts,
                              double* out, sk_pt_report* rep) {
  return sk::pt_estimate_impl(variant, n, budget, opts, out, rep);
}

extern "C" int sk_pt_tune_ladder(int variant, int n, int rungs, double beta_max, uint64_t seed,
                                 double* beta) {
  if (!beta || rungs < 1 || rungs > sk::kPtMaxRungs || !(beta_max > 0)) return SK_EINVAL;
  if (variant != SK_SKOLEM && variant != SK_LANGFORD) return SK_EINVAL;
  if (n < 2 || n > sk::kPtMaxN) return SK_EINVAL;
  int st = sk::check_device();
  if (st) return st;
  return sk::tune_ladder(variant, n, rungs, beta_max, seed, nullptr, beta);
}
