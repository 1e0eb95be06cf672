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
  float* Zcur;               // [B][NMp] logits of the current states
  float* lse;                // [B] log-normaliser over their valid moves
  int4* prop;                // [B] (k, old slot, new slot, dE)
  float* lq_fwd;             // [B] log q(C' | C)
  unsigned* hist;            // [L][M][nb]
  unsigned* accm;            // [L][M]
  unsigned* accs;            // [L][M]
  const double* beta;        // [M]
  const unsigned long long* tswap;   // [M][nb]
};

__device__ __forceinline__ void load_state(const unsigned char* sl, int n, int delta,
                                           unsigned char* s_slot, unsigned char* s_occ, int lane) {
  for (int i = lane; i < 2 * n; i += 32) s_occ[i] = 0;
  __syncwarp();
  if (lane == 0)
    for (int k = 1; k <= n; ++k) {
      const int s = sl[k - 1];
      s_slot[k] = (unsigned char)s;
      s_occ[s] += 1;
      s_occ[s + k + delta] += 1;
    }
  __syncwarp();
}

// log sum exp of the logits z over the valid moves of the state in smem.
__device__ float valid_lse(const float* z, const MoveTable& mt, const unsigned char* s_slot,
                           int lane) {
  float mx = -INFINITY;
  for (int m = lane, k = 1; m < mt.NM; m += 32) {
    while (m >= mt.off[k + 1]) ++k;
    if (m - mt.off[k] != s_slot[k]) mx = fmaxf(mx, z[m]);
  }
  mx = warp_max(mx);
  float sum = 0.f;
  for (int m = lane, k = 1; m < mt.NM; m += 32) {
    while (m >= mt.off[k + 1]) ++k;
    if (m - mt.off[k] != s_slot[k]) sum += expf(z[m] - mx);
  }
  return mx + logf(warp_sum(sum));
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
__global__ void __launch_bounds__(256) lt_keep_kernel(LearnedDev d, MoveTable mt, const float* Z) {
  __shared__ unsigned char s_occ[8][2 * kPtMaxN];
  __shared__ unsigned char s_slot[8][kPtMaxN + 1];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, c = blockIdx.x * 8 + w;
  if (c >= d.B) return;
  load_state(d.slots + (size_t)c * d.n, d.n, d.delta, s_slot[w], s_occ[w], lane);
  const float* z = Z + (size_t)c * d.NMp;
  float* zc = d.Zcur + (size_t)c * d.NMp;
  for (int m = lane; m < d.NMp; m += 32) zc[m] = z[m];
  const float l = valid_lse(z, mt, s_slot[w], lane);
  if (lane == 0) d.lse[c] = l;
}

// Statistics of iteration t, then a move drawn from the current softmax; the
// proposed configuration goes to `prop_slots` (the network's input).
__global__ void __launch_bounds__(256) lt_propose_kernel(LearnedDev d, MoveTable mt, unsigned t,
                                                         int count_stats,
                                                         unsigned char* prop_slots) {
  __shared__ unsigned char s_occ[8][2 * kPtMaxN];
  __shared__ unsigned char s_slot[8][kPtMaxN + 1];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, c = blockIdx.x * 8 + w;
  if (c >= d.B) return;
  const int ladder = c / d.M, r = d.rung[c], E = d.E[c];
  if (lane == 0 && count_stats) d.hist[((size_t)ladder * d.M + r) * d.nb + E] += 1;
  load_state(d.slots + (size_t)c * d.n, d.n, d.delta, s_slot[w], s_occ[w], lane);
  const float* z = d.Zcur + (size_t)c * d.NMp;
  const float lse = d.lse[c];
  const uint4 rw = philox4x32_10(make_uint4(t, (unsigned)r, (unsigned)ladder, 5u), d.key0, d.key1);
  // inverse CDF over the valid moves: lane-contiguous chunks, warp scan
  const int CH = (mt.NM + 31) / 32, m0 = lane * CH, m1 = min(mt.NM, m0 + CH);
  float part = 0.f;
  int k = 1;
  while (m0 < mt.NM && m0 >= mt.off[k + 1]) ++k;
  const int k0 = k;
  for (int m = m0; m < m1; ++m) {
    while (m >= mt.off[k + 1]) ++k;
    if (m - mt.off[k] != s_slot[w][k]) part += expf(z[m] - lse);
  }
  float incl = part;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const float v = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += v;
  }
  const float total = __shfl_sync(0xffffffffu, incl, 31);
  const float target = ((float)rw.x + 0.5f) * 2.3283064365386963e-10f * total;
  const unsigned hit = __ballot_sync(0xffffffffu, incl >= target && part > 0.f);
  const int owner = hit ? __ffs(hit) - 1 : 31;
  int pick = -1;
  if (lane == owner) {
    float cum = incl - part;
    k = k0;
    for (int m = m0; m < m1; ++m) {
      while (m >= mt.off[k + 1]) ++k;
      if (m - mt.off[k] == s_slot[w][k]) continue;
      cum += expf(z[m] - lse);
      pick = m;
      if (cum >= target) break;
    }
  }
  pick = __shfl_sync(0xffffffffu, pick, owner);
  if (pick < 0) {                     // rounding left nothing: last valid move
    int last = -1;
    for (int m = lane, kk = 1; m < mt.NM; m += 32) {
      while (m >= mt.off[kk + 1]) ++kk;
      if (m - mt.off[kk] != s_slot[w][kk]) last = m;
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) last = max(last, __shfl_xor_sync(0xffffffffu, last, o));
    pick = last;
  }
  int kp = 1;
  while (pick >= mt.off[kp + 1]) ++kp;
  const int s_new = pick - mt.off[kp], s_old = s_slot[w][kp];
  const int dE = move_delta_e(s_occ[w], s_old, kp + d.delta, s_new);
  unsigned char* ps = prop_slots + (size_t)c * d.n;
  for (int i = lane; i < d.n; i += 32)
    ps[i] = (i + 1 == kp) ? (unsigned char)s_new : s_slot[w][i + 1];
  if (lane == 0) {
    d.prop[c] = make_int4(kp, s_old, s_new, dE);
    d.lq_fwd[c] = z[pick] - lse;
  }
}

// Metropolis-Hastings acceptance with the proposed states' logits Zp.
__global__ void __launch_bounds__(256) lt_accept_kernel(LearnedDev d, MoveTable mt, unsigned t,
                                                        const unsigned char* prop_slots,
                                                        const float* Zp) {
  __shared__ unsigned char s_occ[8][2 * kPtMaxN];
  __shared__ unsigned char s_slot[8][kPtMaxN + 1];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, c = blockIdx.x * 8 + w;
  if (c >= d.B) return;
  const int ladder = c / d.M, r = d.rung[c];
  load_state(prop_slots + (size_t)c * d.n, d.n, d.delta, s_slot[w], s_occ[w], lane);
  const float* zp = Zp + (size_t)c * d.NMp;
  const float lse_p = valid_lse(zp, mt, s_slot[w], lane);
  const int4 pr = d.prop[c];
  const float lq_rev = zp[mt.off[pr.x] + pr.y] - lse_p;
  const float log_a = (float)(-d.beta[r] * (double)pr.w) + lq_rev - d.lq_fwd[c];
  const uint4 rw = philox4x32_10(make_uint4(t, (unsigned)r, (unsigned)ladder, 5u), d.key0, d.key1);
  const float u = ((float)rw.y + 0.5f) * 2.3283064365386963e-10f;
  const bool acc = log_a >= 0.f || logf(u) < log_a;
  if (!acc) return;
  for (int i = lane; i < d.n; i += 32) d.slots[(size_t)c * d.n + i] = s_slot[w][i + 1];
  float* zc = d.Zcur + (size_t)c * d.NMp;
  for (int m = lane; m < d.NMp; m += 32) zc[m] = zp[m];
  if (lane == 0) {
    d.lse[c] = lse_p;
    d.E[c] += pr.w;
    d.accm[(size_t)ladder * d.M + r] += 1;
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

int pt_learned_run(int variant, int n, int M, const double* beta, int L, uint64_t iters,
                   uint64_t burnin, uint64_t seed, const void* model, uint64_t* hist,
                   uint64_t* accm, uint64_t* accs, void* stream, double* kernel_ms) {
  Mlp* m = (Mlp*)model;
  if (!m || !beta || !hist || iters > 0xffffffffULL) return SK_EINVAL;
  if (m->variant != variant || m->n != n || M < 2 || M > kPtMaxRungs || L < 1) return SK_EINVAL;
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
  const size_t o_z = off; off = al(off + (size_t)B * m->NMp * 4);
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
  d.Zcur = (float*)(p + o_z);
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
  if (e == cudaSuccess) e = mlp_forward_dev(*m, Bp, s);
  if (e == cudaSuccess) {
    lt_keep_kernel<<<(B + 7) / 8, 256, 0, s>>>(d, mt, m->Z);
    e = cudaGetLastError();
  }
  for (uint64_t t = 0; t < iters && e == cudaSuccess; ++t) {
    lt_propose_kernel<<<(B + 7) / 8, 256, 0, s>>>(d, mt, (unsigned)t, t >= burnin ? 1 : 0,
                                                  m->slots);
    e = mlp_forward_dev(*m, Bp, s);
    if (e != cudaSuccess) break;
    lt_accept_kernel<<<(B + 7) / 8, 256, 0, s>>>(d, mt, (unsigned)t, m->slots, m->Z);
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
