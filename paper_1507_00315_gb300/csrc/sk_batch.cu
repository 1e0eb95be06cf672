// sk_batch.cu -- the persistent batched sweep and the autotuner.
//
// skolem_count_batch runs many exact-count jobs (variant x n) in one
// persistent launch captured in a CUDA graph: jobs are laid end to end in a
// space of 32-item chunks, largest job first (longest-processing-time order),
// every warp pulls the next chunk from a device counter, finds its job by
// binary search over the chunk offsets, and runs that job's compiled walk.  A
// warp keeps its residues while it stays on one job and flushes them into the
// job's slots (modular CAS add) when it moves on.  The same jobs can instead
// run as one launch per job (SK_BATCH_PER_JOB), the baseline it is measured
// against.  skolem_autotune times candidate walk widths and block sizes for
// one (variant, n) on a fixed number of terms and keeps the fastest.
#include <algorithm>
#include <chrono>
#include <cstring>
#include <mutex>
#include <vector>

#include "sk_batch.cuh"
#include "sk_exact_launch.cuh"
#include "sk_host_common.h"

SK_DECLARE_BATCH(1) SK_DECLARE_BATCH(2) SK_DECLARE_BATCH(3) SK_DECLARE_BATCH(4)
SK_DECLARE_BATCH(5) SK_DECLARE_BATCH(6) SK_DECLARE_BATCH(7) SK_DECLARE_BATCH(8)
SK_DECLARE_BATCH(9) SK_DECLARE_BATCH(10) SK_DECLARE_BATCH(11) SK_DECLARE_BATCH(12)
SK_DECLARE_BATCH(13) SK_DECLARE_BATCH(14) SK_DECLARE_BATCH(15) SK_DECLARE_BATCH(16)
SK_DECLARE_BATCH(17) SK_DECLARE_BATCH(18) SK_DECLARE_BATCH(19) SK_DECLARE_BATCH(20)
SK_DECLARE_BATCH(21) SK_DECLARE_BATCH(22) SK_DECLARE_BATCH(23) SK_DECLARE_BATCH(24)
SK_DECLARE_BATCH(25) SK_DECLARE_BATCH(26) SK_DECLARE_BATCH(27) SK_DECLARE_BATCH(28)
SK_DECLARE_BATCH(29) SK_DECLARE_BATCH(30) SK_DECLARE_BATCH(31)

namespace sk {

unsigned long long position_mask(int variant, int n);                     // sk_host_exact.cu
int default_walk_bits(int n);                                             // sk_host_exact.cu
int limb_max_m(int delta, int n);                                         // sk_host_exact.cu
int finalize_count(int variant, int n, int convention, int nprimes, const uint64_t* primes,
                   const uint64_t* H, sk_u128* out);                      // sk_host_exact.cu

struct BatchScratch {
  unsigned long long counter;   // next chunk
  unsigned int err;
  unsigned int pad;
};

__device__ __forceinline__ Res4 batch_dispatch(int code, const BatchJobDev* j, const Primes* P,
                                               int np, unsigned long long it, signed char* ws) {
#define SK_BCASE(N)                                     \
  case N: return SK_BATCH_FN(0, N)(j, P, np, it, ws);   \
  case 32 + N: return SK_BATCH_FN(1, N)(j, P, np, it, ws);
  switch (code) {
    SK_BCASE(1) SK_BCASE(2) SK_BCASE(3) SK_BCASE(4) SK_BCASE(5) SK_BCASE(6) SK_BCASE(7)
    SK_BCASE(8) SK_BCASE(9) SK_BCASE(10) SK_BCASE(11) SK_BCASE(12) SK_BCASE(13) SK_BCASE(14)
    SK_BCASE(15) SK_BCASE(16) SK_BCASE(17) SK_BCASE(18) SK_BCASE(19) SK_BCASE(20)
    SK_BCASE(21) SK_BCASE(22) SK_BCASE(23) SK_BCASE(24) SK_BCASE(25) SK_BCASE(26)
    SK_BCASE(27) SK_BCASE(28) SK_BCASE(29) SK_BCASE(30) SK_BCASE(31)
    default: break;
  }
#undef SK_BCASE
  Res4 z = {{0, 0, 0, 0}};
  return z;
}

__global__ void __launch_bounds__(256, SK_EXACT_MIN_BLOCKS)
    batch_kernel(const BatchJobDev* __restrict__ jobs, int njobs, unsigned long long total_chunks,
                 const Primes* P, int nprimes, BatchScratch* scr, unsigned long long* res) {
  extern __shared__ signed char sk_ws[];
  const int lane = threadIdx.x & 31;
  signed char* ws_col = sk_ws + threadIdx.x;
  unsigned long long tot[kMaxPrimes] = {0, 0, 0, 0};
  int cur = -1;
  for (;;) {
    unsigned long long c = 0;
    if (lane == 0) c = atomicAdd(&scr->counter, 1ULL);
    c = __shfl_sync(0xffffffffu, c, 0);
    if (c >= total_chunks) break;
    int lo = 0, hi = njobs - 1;                  // last job with chunk_lo <= c
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (jobs[mid].chunk_lo <= c) lo = mid;
      else hi = mid - 1;
    }
    if (lo != cur) {
      if (cur >= 0) warp_flush(tot, nprimes, *P, res + (size_t)cur * kMaxPrimes, &scr->err);
      cur = lo;
    }
    const BatchJobDev* j = &jobs[lo];
    const unsigned long long item = (c - j->chunk_lo) * 32ULL + (unsigned long long)lane;
    const Res4 r = batch_dispatch(j->code, j, P, nprimes, item, ws_col);
#pragma unroll
    for (int i = 0; i < kMaxPrimes; ++i)
      if (i < nprimes) tot[i] = addmod(tot[i], r.r[i], (unsigned long long)P->pr[i].p);
  }
  if (cur >= 0) warp_flush(tot, nprimes, *P, res + (size_t)cur * kMaxPrimes, &scr->err);
}

}  // namespace sk

// ===================================================================== host

namespace sk {
namespace {

struct Tuned {
  int m = 0, bt = 0;
  double rate = 0.0;
};
std::mutex g_tune_mu;
Tuned g_tuned[2][kMaxN + 1];

int batch_primes(const sk_batch_opts* o, int* k, uint64_t* pv, Primes* P) {
  sk_count_opts co;
  std::memset(&co, 0, sizeof(co));
  if (o) {
    co.nprimes = o->nprimes;
    for (int i = 0; i < SK_MAX_PRIMES; ++i) co.primes[i] = o->primes[i];
  }
  return prepare_primes(&co, k, pv, P);
}

int delta_of(int variant) { return variant == SK_LANGFORD ? 1 : 0; }

// Times the exact-form kernel of one (variant, n) on its first items -- one
// full wave, SMs x 512 resident threads with one item each, so every
// candidate is timed in the steady state of a long launch -- and keeps the
// fastest configuration; the default one unless another is at least 3 %
// faster (single timings of this length vary by about 1 %).
int tune_impl(int variant, int n, const sk_batch_opts* o, sk_tune_result* out) {
  if (variant < SK_SKOLEM || variant > SK_HOOKED || n < 1 || n > kMaxN || !out) return SK_EINVAL;
  int k = 0;
  uint64_t pv[kMaxPrimes];
  Primes P;
  int st = batch_primes(o, &k, pv, &P);
  if (st) return st;
  st = check_device();
  if (st) return st;
  const int delta = delta_of(variant), F = 2 * n - 1, U = inner_bits(n);
  const int mmax = limb_max_m(delta, n) < F ? limb_max_m(delta, n) : F;
  int m0 = default_walk_bits(n);
  if (m0 > mmax) m0 = mmax;
  std::vector<int> ms;
  for (int dm = -4; dm <= 4; dm += 2) {
    const int m = m0 + dm;
    if (m >= U && m <= mmax && F - m <= 56) ms.push_back(m);
  }
  ExactLaunchFn fn = limb_launcher(delta, n);
  cudaStream_t s = (o && o->stream) ? (cudaStream_t)o->stream : nullptr;
  bool own = false;
  if (!s) {
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) return SK_ECUDA;
    own = true;
  }
  ExactScratch* d = nullptr;
  if (cudaMalloc(&d, sizeof(ExactScratch)) != cudaSuccess) {
    if (own) cudaStreamDestroy(s);
    return SK_ENOMEM;
  }
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const unsigned long long wave = (unsigned long long)(sms > 0 ? sms : 1) * 512ULL;
  Tuned best, dflt;
  int cand = 0;
  const int bts[2] = {128, 256};
  for (int m : ms) {
    const unsigned long long items = 1ULL << (F - m);
    const unsigned long long sample = wave < items ? wave : items;
    for (int bt : bts) {
      ExactLaunch L;
      std::memset(&L, 0, sizeof(L));
      L.job.pres = position_mask(variant, n);
      L.job.items = items;
      L.job.m = m;
      L.P = P;
      L.nprimes = k;
      L.item_lo = 0;
      L.item_hi = sample;
      L.scratch = d;
      L.block_threads = bt;
      L.stream = s;
      float ms_t = 0.f;
      cudaError_t e = cudaSuccess;
      for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {    // warm, then timed
        e = cudaMemsetAsync(d, 0, sizeof(ExactScratch), s);
        if (e == cudaSuccess) e = cudaEventRecord(e0, s);
        if (e == cudaSuccess) e = fn(L);
        if (e == cudaSuccess) e = cudaEventRecord(e1, s);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms_t, e0, e1);
      }
      if (e != cudaSuccess) { st = cuda_status(e); break; }
      ++cand;
      const double rate = (double)sample * (double)(1ULL << m) / (ms_t * 1e-3);
      if (rate > best.rate) { best.rate = rate; best.m = m; best.bt = bt; }
      if (m == m0 && bt == 256) { dflt.rate = rate; dflt.m = m; dflt.bt = bt; }
    }
    if (st) break;
  }
  if (dflt.rate > 0 && best.rate < 1.03 * dflt.rate) best = dflt;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(d);
  if (own) cudaStreamDestroy(s);
  if (st) return st;
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tuned[delta][n] = best;
  }
  out->walk_bits = best.m;
  out->block_threads = best.bt;
  out->terms_per_s = best.rate;
  out->candidates = cand;
  return SK_OK;
}

}  // namespace
}  // namespace sk

extern "C" int skolem_autotune(int variant, int n, const sk_batch_opts* opts, sk_tune_result* out) {
  return sk::tune_impl(variant, n, opts, out);
}

namespace sk {
namespace {

struct JobPlan {
  int variant, n, delta, m;
  unsigned long long items, terms;
};

int batch_impl(const sk_job* jobs, int njobs, const sk_batch_opts* o, sk_u128* outs, int* status,
               sk_batch_report* rep) {
  auto t0 = std::chrono::steady_clock::now();
  if (!jobs || !outs || njobs < 1 || njobs > 4096) return SK_EINVAL;
  const int mode = o ? o->mode : SK_BATCH_PERSISTENT;
  if (mode != SK_BATCH_PERSISTENT && mode != SK_BATCH_PER_JOB) return SK_EINVAL;
  const int conv = o ? o->convention : SK_COUNT_REFLECTIONS_IDENTIFIED;
  if (conv != SK_COUNT_REFLECTIONS_IDENTIFIED && conv != SK_COUNT_ALL) return SK_EINVAL;
  int k = 0;
  uint64_t pv[kMaxPrimes];
  Primes P;
  int st = batch_primes(o, &k, pv, &P);
  if (st) return st;
  int bt = (o && o->block_threads) ? o->block_threads : 0;
  if (bt && (bt < 32 || bt > 256 || (bt & 31))) return SK_EINVAL;
  std::vector<JobPlan> plan(njobs);
  for (int j = 0; j < njobs; ++j) {
    const int v = jobs[j].variant, n = jobs[j].n;
    if (v < SK_SKOLEM || v > SK_HOOKED || n < 1 || n > kMaxN) return SK_EINVAL;
    plan[j].variant = v;
    plan[j].n = n;
    plan[j].delta = delta_of(v);
    plan[j].terms = 1ULL << (2 * n - 1);
  }
  st = check_device();
  if (st) return st;
  const int repeats = (o && o->repeats > 0) ? o->repeats : 1;
  // walk widths: explicit, else tuned, else the planner's
  int bt_tuned = 0;
  unsigned long long tuned_terms = 0;
  for (int j = 0; j < njobs; ++j) {
    JobPlan& J = plan[j];
    const int F = 2 * J.n - 1, U = inner_bits(J.n);
    const int mmax = limb_max_m(J.delta, J.n) < F ? limb_max_m(J.delta, J.n) : F;
    int m = (o && o->walk_bits[J.n]) ? o->walk_bits[J.n] : 0;
    if (!m && o && o->autotune) {
      Tuned t;
      {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        t = g_tuned[J.delta][J.n];
      }
      if (!t.m) {
        sk_tune_result r;
        st = tune_impl(J.variant, J.n, o, &r);
        if (st) return st;
        t.m = r.walk_bits;
        t.bt = r.block_threads;
      }
      m = t.m;
      if (J.terms > tuned_terms) { tuned_terms = J.terms; bt_tuned = t.bt; }
    }
    if (!m) m = default_walk_bits(J.n) < mmax ? default_walk_bits(J.n) : mmax;
    if (m < U || m > mmax || F - m > 56) return SK_EINVAL;
    J.m = m;
    J.items = 1ULL << (F - m);
  }
  if (!bt) bt = bt_tuned ? bt_tuned : 256;
  // largest job first
  std::vector<int> order(njobs);
  for (int j = 0; j < njobs; ++j) order[j] = j;
  std::stable_sort(order.begin(), order.end(),
                   [&](int a, int b) { return plan[a].terms > plan[b].terms; });
  std::vector<BatchJobDev> hj(njobs);
  unsigned long long chunk = 0, terms = 0;
  int max_ws = 0;
  for (int r = 0; r < njobs; ++r) {
    const JobPlan& J = plan[order[r]];
    BatchJobDev& d = hj[r];
    std::memset(&d, 0, sizeof(d));
    d.pres = position_mask(J.variant, J.n);
    d.items = J.items;
    d.chunk_lo = chunk;
    d.chunks = (J.items + 31) / 32;
    d.m = J.m;
    d.code = J.delta * 32 + J.n;
    chunk += d.chunks;
    terms += J.terms;
    const int w = ws_len(J.delta, J.n);
    if (w > max_ws) max_ws = w;
  }
  const unsigned long long total_chunks = chunk;
  // device layout: jobs | primes | batch scratch | residues | per-job scratch
  const size_t off_p = (sizeof(BatchJobDev) * njobs + 255) / 256 * 256;
  const size_t off_s = off_p + (sizeof(Primes) + 255) / 256 * 256;
  const size_t off_r = off_s + 256;
  const size_t off_j = off_r + ((size_t)njobs * kMaxPrimes * 8 + 255) / 256 * 256;
  const size_t bytes = off_j + sizeof(ExactScratch) * (size_t)njobs;
  const size_t out_bytes = bytes - off_s;           // what comes back to the host
  cudaStream_t s = (o && o->stream) ? (cudaStream_t)o->stream : nullptr;
  bool own = false;
  if (!s) {
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) return SK_ECUDA;
    own = true;
  }
  char* dbuf = nullptr;
  char* hbuf = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  double kms_last = 0.0, kms_min = 1e300;
  int grid = 0, launches = 0;
  cudaError_t e = cudaMalloc(&dbuf, bytes);
  if (e == cudaSuccess) e = cudaHostAlloc(&hbuf, out_bytes, cudaHostAllocDefault);
  if (e == cudaSuccess) e = cudaMemcpy(dbuf, hj.data(), sizeof(BatchJobDev) * njobs, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(dbuf + off_p, &P, sizeof(Primes), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  const size_t smem = (size_t)max_ws * kWsStride;
  if (e == cudaSuccess && mode == SK_BATCH_PERSISTENT) {
    int dev = 0, sms = 0, nb = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, batch_kernel, bt, smem);
    grid = sms * (nb > 0 ? nb : 1);
    const unsigned long long need = (total_chunks + bt / 32 - 1) / (bt / 32);
    if ((unsigned long long)grid > need) grid = (int)need;
    launches = 1;
  }
  auto enqueue = [&]() -> cudaError_t {
    cudaError_t r = cudaMemsetAsync(dbuf + off_s, 0, bytes - off_s, s);
    if (r != cudaSuccess) return r;
    if (mode == SK_BATCH_PERSISTENT) {
      batch_kernel<<<grid, bt, smem, s>>>((const BatchJobDev*)dbuf, njobs, total_chunks,
                                          (const Primes*)(dbuf + off_p), k,
                                          (BatchScratch*)(dbuf + off_s),
                                          (unsigned long long*)(dbuf + off_r));
      r = cudaGetLastError();
    } else {
      launches = 0;
      for (int q = 0; q < njobs && r == cudaSuccess; ++q) {
        const JobPlan& J = plan[order[q]];
        ExactLaunch L;
        std::memset(&L, 0, sizeof(L));
        L.job.pres = hj[q].pres;
        L.job.items = J.items;
        L.job.m = J.m;
        L.P = P;
        L.nprimes = k;
        L.item_lo = 0;
        L.item_hi = J.items;
        L.scratch = (ExactScratch*)(dbuf + off_j) + q;
        L.block_threads = bt;
        L.stream = s;
        r = limb_launcher(J.delta, J.n)(L);
        ++launches;
      }
    }
    if (r != cudaSuccess) return r;
    return cudaMemcpyAsync(hbuf, dbuf + off_s, out_bytes, cudaMemcpyDeviceToHost, s);
  };
  const bool use_graph = mode == SK_BATCH_PERSISTENT && !(o && o->no_graph);
  if (e == cudaSuccess && use_graph) {
    e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      cudaError_t r = enqueue();
      e = cudaStreamEndCapture(s, &graph);
      if (r != cudaSuccess) e = r;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
  }
  auto t1 = std::chrono::steady_clock::now();
  for (int it = 0; it < repeats && e == cudaSuccess; ++it) {
    e = cudaEventRecord(e0, s);
    if (e == cudaSuccess) e = use_graph ? cudaGraphLaunch(exec, s) : enqueue();
    if (e == cudaSuccess) e = cudaEventRecord(e1, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    kms_last = ms;
    if (ms < kms_min) kms_min = ms;
  }
  if (e == cudaSuccess) {
    const BatchScratch* hs = (const BatchScratch*)hbuf;
    const unsigned long long* hr = (const unsigned long long*)(hbuf + (off_r - off_s));
    const ExactScratch* hjs = (const ExactScratch*)(hbuf + (off_j - off_s));
    bool err = mode == SK_BATCH_PERSISTENT ? hs->err != 0 : false;
    for (int q = 0; q < njobs; ++q)
      if (mode == SK_BATCH_PER_JOB && hjs[q].err) err = true;
    if (err) st = SK_ETIMEOUT;
    for (int q = 0; q < njobs && !st; ++q) {
      const int j = order[q];
      uint64_t H[kMaxPrimes] = {0, 0, 0, 0};
      for (int i = 0; i < k; ++i)
        H[i] = mode == SK_BATCH_PERSISTENT ? hr[(size_t)q * kMaxPrimes + i] : hjs[q].res[i];
      const int sj = finalize_count(plan[j].variant, plan[j].n, conv, k, pv, H, &outs[j]);
      if (status) status[j] = sj;
      if (sj) st = SK_EMISMATCH;
    }
  } else {
    st = cuda_status(e);
  }
  if (exec) cudaGraphExecDestroy(exec);
  if (graph) cudaGraphDestroy(graph);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(dbuf);
  if (hbuf) cudaFreeHost(hbuf);
  if (own) cudaStreamDestroy(s);
  if (rep && (st == SK_OK || st == SK_EMISMATCH)) {
    std::memset(rep, 0, sizeof(*rep));
    rep->kernel_ms = kms_last;
    rep->kernel_ms_min = kms_min;
    rep->prepare_ms = std::chrono::duration<double, std::milli>(t1 - t0).count();
    rep->wall_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    rep->terms = terms;
    rep->chunks = total_chunks;
    rep->launches = launches;
    rep->grid = grid;
    rep->block_threads = bt;
  }
  return st;
}

}  // namespace
}  // namespace sk

extern "C" int skolem_count_batch(const sk_job* jobs, int njobs, const sk_batch_opts* opts,
                                  sk_u128* outs, int* status, sk_batch_report* rep) {
  return sk::batch_impl(jobs, njobs, opts, outs, status, rep);
}
