// sk_gemm_tc.cuh -- BF16 GEMM on the 5th-generation tensor cores (tcgen05)
// for the proposal network: C[M x N] = A[M x K] * B^T (+ bias), A row-major
// [M][K], B stored [N][K] (both K-major), FP32 accumulation in tensor
// memory.  M % 128 == 0, N % 256 == 0, K % 64 == 0.  Epilogues: FP32 (+ bias)
// -- the logits, and the partial products of a K split; BF16 ReLU(+ bias) --
// the hidden layers; BF16 masked by an auxiliary matrix (C = acc where
// aux > 0) -- the backward's activation gradients.  The B operand is either
// resident (the forward: K <= 256, loaded once per CTA) or streamed slice by
// slice beside A through the stage ring (the backward: any K).  A K split
// (ksplit > 1) gives each CTA a range of K slices and writes its partial
// product to rows ks * M .. ks * M + M - 1 of C (FP32), summed afterwards in
// a fixed order.
//
// Persistent and warp-specialised, one CTA (6 warps) per SM:
//   * every CTA owns one 256-wide column tile of B for the whole launch: its
//     K/64 slices ([256][64] bf16, 128-byte swizzle) are loaded once by TMA
//     and stay in shared memory;
//   * warp 0 (one lane) streams the CTA's 128-row tiles of A by TMA, one
//     [128][64] slice per stage of a 4-deep ring (mbarriers full / empty);
//   * warp 1 (one lane) issues tcgen05.mma (128 x 256 x 16) for each slice
//     into one of two 256-column accumulators in tensor memory and commits
//     them to the ring's "empty" barrier and, per tile, to "acc full";
//   * warps 2-5 (the epilogue) read the finished accumulator with
//     tcgen05.ld (each warp its 32 lanes = rows), add the bias, apply ReLU
//     and round to bf16 (or keep fp32), write each 128-byte column slab of
//     their 32 rows into a 128-byte-swizzled staging buffer in shared memory
//     (two per warp) and store it to global memory with one TMA bulk-tensor
//     store, then release the accumulator ("acc empty") so the MMA warp can
//     start the tile after next while the epilogue of this one runs.
// Every wait is bounded (poll count and 2 s of %globaltimer): on expiry the
// role records an error word and stops; before the CTA frees its tensor
// memory each role waits (bounded) for its own copies and MMAs in flight.
#pragma once
#include <cuda.h>
#include <cuda_bf16.h>

#include <cstdint>

namespace sk {

constexpr int kTcBM = 128, kTcBN = 256, kTcBK = 64, kTcStages = 4, kTcMaxK = 256;
constexpr int kTcSliceA = kTcBM * kTcBK * 2;                  // 16 KB
constexpr int kTcSliceB = kTcBN * kTcBK * 2;                  // 32 KB
constexpr int kTcStage = 32 * 128;                            // staging: 32 rows x 128 B
constexpr int kTcThreads = 192;                               // 6 warps
constexpr int kTcSmem =
    (kTcMaxK / kTcBK) * kTcSliceB + kTcStages * kTcSliceA + 4 * 2 * kTcStage + 1024;
// streamed B: each stage of the ring holds an A slice and a B slice
constexpr int kTcSmemStream = kTcStages * (kTcSliceA + kTcSliceB) + 4 * 2 * kTcStage + 1024;
// both stay within the 227 KB a block may hold, with the kernel's ~1.2 KB of
// static shared memory (barriers, bias)
static_assert(kTcSmem + 1280 <= 232448 && kTcSmemStream + 1280 <= 232448, "shared memory");

enum { kTcEpiF32 = 0, kTcEpiReluBf16 = 1, kTcEpiMaskBf16 = 2, kTcEpiBf16 = 3 };
constexpr unsigned kTcWaitLimit = 1u << 24;                   // polls
constexpr unsigned long long kTcWaitNs = 2000000000ULL;       // and at most 2 s

struct TcGemmArgs {
  int M, N, K;
  const float* bias;              // [N] or null
  unsigned* err;                  // set nonzero if a wait gave up
  int ksplit;                     // K ranges (0 or 1: none); needs K / 64 % ksplit == 0
  const __nv_bfloat16* aux;       // kTcEpiMaskBf16: [M][ldaux], C = acc where aux > 0
  int ldaux;
  int nvalid;                     // > 0: only columns < nvalid are wanted (the last column
                                  // tile multiplies and stores that many, rounded up to 16)
  int pdl;                        // launch as a programmatic dependent of the previous kernel
                                  // of the stream; only where B is not written by it or by any
                                  // kernel since the last ordinary launch
};

__device__ __forceinline__ unsigned tc_smem_u32(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ unsigned long long tc_now() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Bounded wait for the completion of the phase with the given parity.
__device__ __forceinline__ bool tc_wait(unsigned mbar, unsigned parity) {
  const unsigned long long t0 = tc_now();
  for (unsigned it = 0; it < kTcWaitLimit; ++it) {
    unsigned ok;
    asm volatile(
        "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
        : "=r"(ok)
        : "r"(mbar), "r"(parity)
        : "memory");
    if (ok) return true;
    if ((it & 255) == 255 && tc_now() - t0 > kTcWaitNs) return false;
  }
  return false;
}

__device__ __forceinline__ void tc_expect_tx(unsigned mbar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mbar), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void tc_arrive(unsigned mbar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(mbar) : "memory");
}

// 2D TMA load of the box at (x = column, y = row) into shared memory.
__device__ __forceinline__ void tc_tma_load(unsigned dst, const CUtensorMap* map, int x, int y,
                                            unsigned mbar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
      ::"r"(dst), "l"(map), "r"(x), "r"(y), "r"(mbar)
      : "memory");
}

// 2D TMA store of the staged box at (x = column, y = row); one bulk group.
__device__ __forceinline__ void tc_tma_store(const CUtensorMap* map, unsigned src, int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%1, %2}], [%3];" ::"l"(map),
      "r"(x), "r"(y), "r"(src)
      : "memory");
  asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}

// Shared-memory matrix descriptor, K-major, 128-byte swizzle: 8-row groups
// of 128-byte rows 1024 bytes apart (stride byte offset), version 1.
__device__ __forceinline__ unsigned long long tc_desc_sw128(unsigned saddr) {
  unsigned long long d = 0;
  d |= (unsigned long long)((saddr >> 4) & 0x3FFF);
  d |= 1ULL << 16;                                   // leading byte offset (unused)
  d |= (unsigned long long)(1024 >> 4) << 32;        // stride byte offset
  d |= 1ULL << 46;                                   // descriptor version
  d |= 2ULL << 61;                                   // layout: 128-byte swizzle
  return d;
}

// Instruction descriptor of kind::f16: D fp32, A and B bf16, both K-major.
__host__ __device__ constexpr unsigned tc_idesc(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((unsigned)(N >> 3) << 17) |
         ((unsigned)(M >> 4) << 24);
}

// The 32 x kCols accumulator block of a warp's lane quarter at TMEM address
// taddr (columns taddr .. taddr + kCols - 1) into v, 16 columns a load; no
// wait (tcgen05.wait::ld before v is read).
template <int kCols>
__device__ __forceinline__ void tc_ld_slab(unsigned (&v)[kCols], unsigned taddr) {
#pragma unroll
  for (int h = 0; h < kCols / 16; ++h)
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,"
        "%12,%13,%14,%15}, [%16];"
        : "=r"(v[h * 16 + 0]), "=r"(v[h * 16 + 1]), "=r"(v[h * 16 + 2]), "=r"(v[h * 16 + 3]),
          "=r"(v[h * 16 + 4]), "=r"(v[h * 16 + 5]), "=r"(v[h * 16 + 6]), "=r"(v[h * 16 + 7]),
          "=r"(v[h * 16 + 8]), "=r"(v[h * 16 + 9]), "=r"(v[h * 16 + 10]), "=r"(v[h * 16 + 11]),
          "=r"(v[h * 16 + 12]), "=r"(v[h * 16 + 13]), "=r"(v[h * 16 + 14]), "=r"(v[h * 16 + 15])
        : "r"(taddr + (unsigned)(h * 16)));
}

// One 128-byte-wide slab of a warp's 32 rows (accumulators v, waited; bias
// b of its columns): converted (bf16 pairs rounded to nearest-even, element i
// in the low half; or fp32), written into staging buffer (slab & 1) of the
// warp in the layout a 128-byte-swizzled TMA store reads (row `lane`, 16-byte
// chunk c at position c ^ (row & 7)) and stored at (x, y); the buffer's
// previous store must have read it out first.
template <int EPI, int kCols>
__device__ __forceinline__ void tc_store_slab(const unsigned (&v)[kCols], const float* b,
                                              unsigned char* stage0, unsigned slab, int lane,
                                              const CUtensorMap* cmap, int x, int y) {
  if (lane == 0) asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory");
  __syncwarp();
  unsigned char* st = stage0 + (slab & 1) * kTcStage;
  unsigned w[32];
#pragma unroll
  for (int i = 0; i < kCols; i += 2) {
    const float2 bb = *(const float2*)&b[i];
    float f0 = __uint_as_float(v[i]) + bb.x, f1 = __uint_as_float(v[i + 1]) + bb.y;
    if constexpr (EPI == kTcEpiF32) {
      w[i] = __float_as_uint(f0);
      w[i + 1] = __float_as_uint(f1);
    } else {
      if constexpr (EPI == kTcEpiReluBf16) {
        f0 = fmaxf(f0, 0.f);
        f1 = fmaxf(f1, 0.f);
      }
      const __nv_bfloat162 p = __floats2bfloat162_rn(f0, f1);
      w[i / 2] = *(const unsigned*)&p;
    }
  }
  const unsigned rbase = tc_smem_u32(st) + (unsigned)lane * 128u;
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const unsigned addr = rbase + (unsigned)((c ^ (lane & 7)) * 16);
    asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(w[4 * c]),
                 "r"(w[4 * c + 1]), "r"(w[4 * c + 2]), "r"(w[4 * c + 3])
                 : "memory");
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  __syncwarp();
  if (lane == 0) tc_tma_store(cmap, tc_smem_u32(st), x, y);
}

// EPI: kTcEpiF32 C = fp32 (acc + bias); kTcEpiReluBf16 C = bf16(relu(acc +
// bias)); kTcEpiMaskBf16 C = bf16(acc) where aux > 0, else 0; kTcEpiBf16 C =
// bf16(acc + bias).  STREAMB: the B
// slices travel with the A slices through the ring instead of staying
// resident (any K).
template <int EPI, bool STREAMB>
__global__ void __launch_bounds__(kTcThreads, 1)
    gemm_tc_kernel(const __grid_constant__ CUtensorMap amap,
                   const __grid_constant__ CUtensorMap bmap,
                   const __grid_constant__ CUtensorMap cmap, TcGemmArgs g) {
  constexpr int BF16 = EPI != kTcEpiF32;
  constexpr int kStageBytes = STREAMB ? kTcSliceA + kTcSliceB : kTcSliceA;
  extern __shared__ __align__(1024) unsigned char tc_smem[];
  __shared__ __align__(8) unsigned long long full_bar[kTcStages], empty_bar[kTcStages];
  __shared__ __align__(8) unsigned long long b_bar, accf_bar[2], acce_bar[2];
  __shared__ unsigned tmem_base_s;
  __shared__ __align__(8) float sbias[kTcBN];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  unsigned char* base = (unsigned char*)(((size_t)tc_smem + 1023) & ~(size_t)1023);
  const int KS = g.ksplit > 1 ? g.ksplit : 1;
  const int nkb = g.K / kTcBK / KS;                  // K slices per tile of this CTA
  // resident B: nkb x [256][64], then the ring of [128][64] A slices;
  // streamed B: the ring of ([128][64] A, [256][64] B) stages
  unsigned char* sB = base;
  unsigned char* sA = STREAMB ? base : base + nkb * kTcSliceB;
  unsigned char* sC = sA + kTcStages * kStageBytes;  // 4 warps x 2 staging buffers
  const int NT = g.N / kTcBN, MT = g.M / kTcBM;
  const int groups = gridDim.x / (NT * KS);          // CTAs per (column tile, K range)
  const int nt = blockIdx.x % NT, ks = (blockIdx.x / NT) % KS, m_first = blockIdx.x / (NT * KS);
  const int kb0 = ks * nkb;                          // first K slice of this CTA
  // columns of this CTA's tile that are multiplied (a multiple of 16)
  const int ncols = g.nvalid > 0 ? min(kTcBN, (g.nvalid - nt * kTcBN + 15) / 16 * 16) : kTcBN;
  const int my_tiles = (m_first < MT) ? (MT - m_first + groups - 1) / groups : 0;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kTcStages; ++s) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tc_smem_u32(&full_bar[s])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tc_smem_u32(&empty_bar[s])));
    }
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tc_smem_u32(&b_bar)));
    for (int a = 0; a < 2; ++a) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tc_smem_u32(&accf_bar[a])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 128;" ::"r"(tc_smem_u32(&acce_bar[a])));
    }
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     tc_smem_u32(&tmem_base_s)),
                 "r"(512));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const unsigned tmem = tmem_base_s;
  // the next kernel of the stream may start its own set-up now (it waits
  // for this grid's completion before it reads what this grid writes)
  asm volatile("griddepcontrol.launch_dependents;");

  if (warp == 0) {
    // ---------------------------------------------------------------- TMA producer
    if (lane == 0) {
      bool ok = true;
      const unsigned bb = tc_smem_u32(&b_bar);
      if (STREAMB) {
        tc_arrive(bb);                               // nothing resident to wait for
      } else {
        tc_expect_tx(bb, (unsigned)(nkb * kTcSliceB));
        for (int kb = 0; kb < nkb; ++kb)
          tc_tma_load(tc_smem_u32(sB + kb * kTcSliceB), &bmap, (kb0 + kb) * kTcBK, nt * kTcBN, bb);
      }
      // launched as a programmatic dependent (g.pdl): the previous kernel's
      // results (A) only after it has completed; resident weights (B) may
      // come earlier, as they do not change between such launches (a no-op
      // for an ordinary launch)
      asm volatile("griddepcontrol.wait;" ::: "memory");
      unsigned u = 0;                                // slices issued
      for (int t = 0; t < my_tiles && ok; ++t) {
        const int mt = m_first + t * groups;
        for (int kb = 0; kb < nkb && ok; ++kb, ++u) {
          const int s = (int)(u % kTcStages);
          const unsigned ph = (u / kTcStages) & 1u;
          if (!tc_wait(tc_smem_u32(&empty_bar[s]), ph ^ 1u)) {
            ok = false;
            break;
          }
          const unsigned fb = tc_smem_u32(&full_bar[s]);
          unsigned char* stg = sA + s * kStageBytes;
          tc_expect_tx(fb, (unsigned)kStageBytes);
          tc_tma_load(tc_smem_u32(stg), &amap, (kb0 + kb) * kTcBK, mt * kTcBM, fb);
          if (STREAMB)
            tc_tma_load(tc_smem_u32(stg + kTcSliceA), &bmap, (kb0 + kb) * kTcBK, nt * kTcBN, fb);
        }
      }
      if (!ok) atomicOr(g.err, 1u);
      // wait for this thread's copies in flight: the last use of every stage
      // and the resident slices of B
      for (int s = 0; s < kTcStages; ++s) {
        if ((unsigned)s >= u) break;
        const unsigned last = u - 1 - ((u - 1 - (unsigned)s) % kTcStages);
        if (!tc_wait(tc_smem_u32(&full_bar[s]), (last / kTcStages) & 1u)) atomicOr(g.err, 8u);
      }
      if (!tc_wait(bb, 0)) atomicOr(g.err, 8u);
    }
  } else if (warp == 1) {
    // ---------------------------------------------------------------- MMA issuer
    if (lane == 0) {
      bool ok = tc_wait(tc_smem_u32(&b_bar), 0);
      const unsigned idesc = tc_idesc(kTcBM, ncols);
      unsigned u = 0;
      int committed = -1;                            // last tile committed to acc full
      for (int t = 0; t < my_tiles && ok; ++t) {
        const int acc = t & 1;
        if (!tc_wait(tc_smem_u32(&acce_bar[acc]), ((t >> 1) & 1) ^ 1)) {
          ok = false;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;");
        const unsigned d = tmem + (unsigned)(acc * kTcBN);
        for (int kb = 0; kb < nkb && ok; ++kb, ++u) {
          const int s = (int)(u % kTcStages);
          if (!tc_wait(tc_smem_u32(&full_bar[s]), (u / kTcStages) & 1u)) {
            ok = false;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;");
          const unsigned a0 = tc_smem_u32(sA + s * kStageBytes);
          const unsigned b0 =
              STREAMB ? a0 + (unsigned)kTcSliceA : tc_smem_u32(sB + kb * kTcSliceB);
#pragma unroll
          for (int kk = 0; kk < kTcBK / 16; ++kk) {
            // K = 16 bf16 = 32 bytes further along the swizzled 128-byte rows
            const unsigned long long ad = tc_desc_sw128(a0 + kk * 32);
            const unsigned long long bd = tc_desc_sw128(b0 + kk * 32);
            const unsigned accum = (kb > 0 || kk > 0) ? 1u : 0u;
            asm volatile(
                "{ .reg .pred p; setp.ne.b32 p, %4, 0;\n\t"
                "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p; }" ::"r"(d),
                "l"(ad), "l"(bd), "r"(idesc), "r"(accum));
          }
          asm volatile(
              "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                  tc_smem_u32(&empty_bar[s])));
        }
        if (!ok) break;
        asm volatile(
            "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                tc_smem_u32(&accf_bar[acc])));
        committed = t;
      }
      if (!ok) atomicOr(g.err, 2u);
      // wait for this thread's MMAs in flight (the last commit of each
      // accumulator completes after every MMA issued before it)
      for (int t = committed; t >= 0 && t > committed - 2; --t)
        if (!tc_wait(tc_smem_u32(&accf_bar[t & 1]), (t >> 1) & 1)) atomicOr(g.err, 8u);
    }
  } else {
    // ---------------------------------------------------------------- epilogue
    const int q = warp & 3;                          // TMEM lane quarter of this warp
    constexpr int kCols = BF16 ? 64 : 32;            // columns per 128-byte slab
    unsigned char* stage0 = sC + q * 2 * kTcStage;
    // the bias of this CTA's column tile, staged once (named barrier of the
    // 128 epilogue threads)
    for (int i = threadIdx.x - 64; i < kTcBN; i += 128)
      sbias[i] = g.bias ? __ldg(g.bias + nt * kTcBN + i) : 0.f;
    asm volatile("bar.sync 1, 128;" ::: "memory");
    bool ok = true;
    unsigned slab = 0;                               // slabs stored by this warp
    for (int t = 0; t < my_tiles; ++t) {
      const int acc = t & 1;
      const int mt = m_first + t * groups;
      if (!tc_wait(tc_smem_u32(&accf_bar[acc]), (t >> 1) & 1)) {
        ok = false;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;");
      const int n0 = nt * kTcBN, row0 = mt * kTcBM + q * 32;
      const int crow0 = ks * g.M + row0;             // a K split's partial goes to its own rows
      if constexpr (EPI != kTcEpiMaskBf16) {
        // software-pipelined: the next slab's accumulator loads are in flight
        // while this slab is converted, staged and stored
        const int nsl = (ncols + kCols - 1) / kCols;
        unsigned va[kCols], vb[kCols];
        tc_ld_slab<kCols>(va, tmem + ((unsigned)(q * 32) << 16) + (unsigned)(acc * kTcBN));
#pragma unroll 1
        for (int i = 0; i < nsl; i += 2) {
          asm volatile("tcgen05.wait::ld.sync.aligned;");
          if (i + 1 < nsl)
            tc_ld_slab<kCols>(vb, tmem + ((unsigned)(q * 32) << 16) +
                                      (unsigned)(acc * kTcBN + (i + 1) * kCols));
          tc_store_slab<EPI, kCols>(va, sbias + i * kCols, stage0, slab++, lane, &cmap,
                                    n0 + i * kCols, crow0);
          if (i + 1 < nsl) {
            asm volatile("tcgen05.wait::ld.sync.aligned;");
            if (i + 2 < nsl)
              tc_ld_slab<kCols>(va, tmem + ((unsigned)(q * 32) << 16) +
                                        (unsigned)(acc * kTcBN + (i + 2) * kCols));
            tc_store_slab<EPI, kCols>(vb, sbias + (i + 1) * kCols, stage0, slab++, lane, &cmap,
                                      n0 + (i + 1) * kCols, crow0);
          }
        }
      } else {
        // the masked epilogue also reads this row's 64 auxiliary bf16 values
        // of each slab (C = acc where aux > 0): one slab at a time
#pragma unroll 1
        for (int c0 = 0; c0 < ncols; c0 += kCols, ++slab) {
          // the staging buffer of two slabs ago must have been read out
          if (lane == 0) asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory");
          __syncwarp();
          unsigned char* st = stage0 + (slab & 1) * kTcStage;
          unsigned v[kCols];
          tc_ld_slab<kCols>(v, tmem + ((unsigned)(q * 32) << 16) + (unsigned)(acc * kTcBN + c0));
          uint4 ax[8];
          const uint4* ap = (const uint4*)(g.aux + (size_t)(row0 + lane) * g.ldaux + n0 + c0);
#pragma unroll
          for (int c = 0; c < 8; ++c) ax[c] = __ldg(ap + c);
          asm volatile("tcgen05.wait::ld.sync.aligned;");
          unsigned w[32];                              // this row's 128 bytes of the slab
          // two results at a time, one packed round-to-nearest-even
          // conversion per pair (element i in the low half)
#pragma unroll
          for (int i = 0; i < kCols; i += 2) {
            const unsigned word = (&ax[i / 8].x)[(i / 2) & 3];
            const short h0 = (short)(word & 0xFFFFu), h1 = (short)(word >> 16);
            const float f0 = h0 > 0 ? __uint_as_float(v[i]) : 0.f;      // aux > 0 (bf16 bits)
            const float f1 = h1 > 0 ? __uint_as_float(v[i + 1]) : 0.f;
            const __nv_bfloat162 p = __floats2bfloat162_rn(f0, f1);
            w[i / 2] = *(const unsigned*)&p;
          }
          // row `lane` of the slab, 16-byte chunk c at chunk position c ^ (row & 7)
          // (the layout a 128-byte-swizzled TMA store reads)
          const unsigned rbase = tc_smem_u32(st) + (unsigned)lane * 128u;
#pragma unroll
          for (int c = 0; c < 8; ++c) {
            const unsigned addr = rbase + (unsigned)((c ^ (lane & 7)) * 16);
            asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(w[4 * c]),
                         "r"(w[4 * c + 1]), "r"(w[4 * c + 2]), "r"(w[4 * c + 3])
                         : "memory");
          }
          asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
          __syncwarp();
          if (lane == 0) tc_tma_store(&cmap, tc_smem_u32(st), n0 + c0, crow0);
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;");
      tc_arrive(tc_smem_u32(&acce_bar[acc]));
    }
    if (lane == 0) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
    if (!ok && lane == 0) atomicOr(g.err, 4u);
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
  }
}

}  // namespace sk
