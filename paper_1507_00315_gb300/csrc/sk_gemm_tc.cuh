// sk_gemm_tc.cuh -- BF16 GEMM on the 5th-generation tensor cores (tcgen05)
// for the proposal network's forward pass: C[M x N] = A[M x K] * B^T, A stored
// row-major [M][K] (activations), B stored [N][K] (the weights kept K-major),
// FP32 accumulation in tensor memory, fused bias + ReLU -> bf16 or fp32 out.
//
// One CTA (4 warps) per 128 x 256 output tile.  Each 64-wide K slice of A
// (128 x 64) and B (256 x 64) is copied by cp.async into shared memory in the
// canonical no-swizzle K-major layout -- 8-row x 16-byte core matrices, the 8
// core matrices of one 8-row group along K contiguous (128 B apart), groups
// 1024 B apart -- two stages deep.  One thread issues four tcgen05.mma
// (K = 16 each) per slice into a 128-lane x 256-column fp32 accumulator in
// tensor memory and commits them to an mbarrier; the slice's buffer is
// refilled only after that mbarrier flips.  Every wait is bounded: on expiry
// the kernel records an error word, waits (bounded) for its own MMAs,
// releases its tensor memory and returns.  The epilogue reads the accumulator
// with tcgen05.ld (each warp its 32 lanes = rows).
#pragma once
#include <cuda_bf16.h>
#include <cstdint>

namespace sk {

constexpr int kTcBM = 128, kTcBN = 256, kTcBK = 64, kTcStages = 2;
constexpr int kTcTileA = kTcBM * kTcBK * 2;          // 16 KB
constexpr int kTcTileB = kTcBN * kTcBK * 2;          // 32 KB
constexpr int kTcSmem = kTcStages * (kTcTileA + kTcTileB) + 1024;
constexpr unsigned kTcWaitLimit = 1u << 22;          // polls
constexpr unsigned long long kTcWaitNs = 2000000000ULL;    // and at most 2 s

struct TcGemmArgs {
  int M, N, K;                    // M % 128 == 0, N % 256 == 0, K % 64 == 0
  const __nv_bfloat16* A;         // [M][lda]
  int lda;
  const __nv_bfloat16* Bt;        // [N][ldb]
  int ldb;
  void* C;                        // [M][ldc] bf16 (relu) or fp32
  int ldc;
  const float* bias;              // [N] or null
  int relu_bf16;                  // 1: bf16(relu(acc + bias)); 0: fp32 acc + bias
  unsigned* err;                  // set nonzero if a wait gave up
};

__device__ __forceinline__ unsigned tc_smem_u32(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}

// Shared-memory matrix descriptor, no swizzle: start address, leading
// (K-direction) and stride (M/N-direction) byte offsets, version 1.
__device__ __forceinline__ unsigned long long tc_desc(unsigned saddr, unsigned lbo, unsigned sbo) {
  unsigned long long d = 0;
  d |= (unsigned long long)((saddr >> 4) & 0x3FFF);
  d |= (unsigned long long)((lbo >> 4) & 0x3FFF) << 16;
  d |= (unsigned long long)((sbo >> 4) & 0x3FFF) << 32;
  d |= 1ULL << 46;                                 // descriptor version
  return d;                                        // layout type 0: no swizzle
}

// Instruction descriptor of kind::f16: D fp32, A and B bf16, both K-major.
__host__ __device__ constexpr unsigned tc_idesc(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((unsigned)(N >> 3) << 17) |
         ((unsigned)(M >> 4) << 24);
}

__device__ __forceinline__ unsigned long long tc_now() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ bool tc_wait(unsigned mbar, unsigned parity) {
  const unsigned long long t0 = tc_now();
  for (unsigned it = 0; it < kTcWaitLimit; ++it) {
    if ((it & 255) == 255 && tc_now() - t0 > kTcWaitNs) return false;
    unsigned ok;
    asm volatile(
        "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
        : "=r"(ok)
        : "r"(mbar), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}

// Copies rows [r0, r0 + rows) x k-slice [k0, k0 + 64) of a row-major bf16
// matrix into the canonical core-matrix layout at smem `dst`.
__device__ __forceinline__ void tc_load_tile(unsigned char* dst, const __nv_bfloat16* src, int ld,
                                             int r0, int k0, int rows) {
  const int chunks = rows * (kTcBK / 8);          // 16-byte chunks
  for (int c = threadIdx.x; c < chunks; c += blockDim.x) {
    const int r = c >> 3, kc = c & 7;
    const unsigned off = (unsigned)(((r >> 3) * 8 + kc) * 128 + (r & 7) * 16);
    const void* g = src + (size_t)(r0 + r) * ld + k0 + kc * 8;
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(tc_smem_u32(dst + off)),
                 "l"(g));
  }
}

__global__ void __launch_bounds__(128, 1) gemm_tc_kernel(TcGemmArgs g) {
  extern __shared__ __align__(1024) unsigned char tc_smem[];
  __shared__ __align__(8) unsigned long long mbar[kTcStages];
  __shared__ unsigned tmem_base_s;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.y * kTcBM, n0 = blockIdx.x * kTcBN;
  unsigned char* base = (unsigned char*)(((size_t)tc_smem + 1023) & ~(size_t)1023);
  unsigned char* sA[kTcStages];
  unsigned char* sB[kTcStages];
  for (int s = 0; s < kTcStages; ++s) {
    sA[s] = base + s * (kTcTileA + kTcTileB);
    sB[s] = sA[s] + kTcTileA;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     tc_smem_u32(&tmem_base_s)),
                 "r"(256));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (threadIdx.x == 0) {
    for (int s = 0; s < kTcStages; ++s)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tc_smem_u32(&mbar[s])));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const unsigned tmem = tmem_base_s;
  const unsigned idesc = tc_idesc(kTcBM, kTcBN);
  const int nk = g.K / kTcBK;
  unsigned phase[kTcStages] = {0, 0};
  bool pending[kTcStages] = {false, false};
  bool ok = true;

  // prologue: slice 0 into stage 0
  tc_load_tile(sA[0], g.A, g.lda, m0, 0, kTcBM);
  tc_load_tile(sB[0], g.Bt, g.ldb, n0, 0, kTcBN);
  asm volatile("cp.async.commit_group;");
  for (int kb = 0; kb < nk; ++kb) {
    const int s = kb & 1;
    // next slice into the other stage once its previous MMAs are done
    if (kb + 1 < nk) {
      const int s2 = s ^ 1;
      if (pending[s2]) {
        if (!tc_wait(tc_smem_u32(&mbar[s2]), phase[s2])) ok = false;
        phase[s2] ^= 1;
        pending[s2] = false;
      }
      tc_load_tile(sA[s2], g.A, g.lda, m0, (kb + 1) * kTcBK, kTcBM);
      tc_load_tile(sB[s2], g.Bt, g.ldb, n0, (kb + 1) * kTcBK, kTcBN);
      asm volatile("cp.async.commit_group;");
      asm volatile("cp.async.wait_group 1;");
    } else {
      asm volatile("cp.async.wait_group 0;");
    }
    asm volatile("fence.proxy.async.shared::cta;");
    __syncthreads();
    if (threadIdx.x == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;");
      const unsigned a0 = tc_smem_u32(sA[s]), b0 = tc_smem_u32(sB[s]);
#pragma unroll
      for (int kk = 0; kk < kTcBK / 16; ++kk) {
        // a K = 16 step covers two core matrices along K (2 x 128 B)
        const unsigned long long ad = tc_desc(a0 + kk * 256, 128, 1024);
        const unsigned long long bd = tc_desc(b0 + kk * 256, 128, 1024);
        const unsigned acc = (kb > 0 || kk > 0) ? 1u : 0u;
        asm volatile(
            "{ .reg .pred p; setp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p; }" ::"r"(tmem),
            "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
      }
      asm volatile(
          "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
              tc_smem_u32(&mbar[s])));
    }
    pending[s] = true;
    __syncthreads();
  }
  // wait for the last MMAs of both stages
  for (int s = 0; s < kTcStages; ++s)
    if (pending[s]) {
      if (!tc_wait(tc_smem_u32(&mbar[s]), phase[s])) ok = false;
      phase[s] ^= 1;
    }
  asm volatile("tcgen05.fence::after_thread_sync;");
  if (!ok) {
    if (lane == 0) atomicOr(g.err, 1u);
  } else {
    // epilogue: warp w reads lanes 32w..32w+31 (rows), 8 columns at a time
    const int row = m0 + warp * 32 + lane;
    for (int c0 = 0; c0 < kTcBN; c0 += 8) {
      unsigned v[8];
      const unsigned taddr = tmem + ((unsigned)(warp * 32) << 16) + (unsigned)c0;
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
          : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
            "=r"(v[7])
          : "r"(taddr));
      asm volatile("tcgen05.wait::ld.sync.aligned;");
      float f[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        f[i] = __uint_as_float(v[i]);
        if (g.bias) f[i] += g.bias[n0 + c0 + i];
      }
      if (g.relu_bf16) {
        __nv_bfloat162* dst =
            (__nv_bfloat162*)((__nv_bfloat16*)g.C + (size_t)row * g.ldc + n0 + c0);
#pragma unroll
        for (int i = 0; i < 4; ++i)
          dst[i] = __floats2bfloat162_rn(fmaxf(f[2 * i], 0.f), fmaxf(f[2 * i + 1], 0.f));
      } else {
        float4* dst = (float4*)((float*)g.C + (size_t)row * g.ldc + n0 + c0);
        dst[0] = make_float4(f[0], f[1], f[2], f[3]);
        dst[1] = make_float4(f[4], f[5], f[6], f[7]);
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(256));
}

}  // namespace sk
