// sk_gemm.cuh -- BF16 GEMM with FP32 accumulation for the move-proposal
// network: C[M x N] = A[M x K] * B[K x N], with fused epilogues.
//
// Layouts: A is stored row-major [M][K] (AT = false) or as its transpose
// [K][M] (AT = true); B is stored [K][N] (BT = false) or [N][K] (BT = true).
// CTA tile 128 x 128 x 32, 8 warps of 64 x 32, two shared-memory stages
// filled by cp.async, fragments by ldmatrix (.trans for the transposed
// storages), warp-level mma.sync m16n8k16.  Every dimension must be a
// multiple of the tile (the host pads); split-K (gridDim.z) adds partial
// tiles with FP32 atomics.
#pragma once
#include <cuda_bf16.h>
#include <cstdint>

namespace sk {

enum GemmEpi {
  EPI_F32 = 0,          // C (float) = acc + bias
  EPI_BF16_RELU = 1,    // C (bf16)  = relu(acc + bias)
  EPI_BF16_MASK = 2,    // C (bf16)  = acc where aux > 0, else 0
  EPI_ATOMIC = 3,       // C (float) += acc
  EPI_BF16 = 4          // C (bf16)  = acc + bias
};

struct GemmArgs {
  int M, N, K;
  const __nv_bfloat16* A;
  int lda;
  const __nv_bfloat16* B;
  int ldb;
  void* C;
  int ldc;
  const float* bias;            // [N] or null
  const __nv_bfloat16* aux;     // EPI_BF16_MASK: [M][ldc]
};

constexpr int kGBM = 128, kGBN = 128, kGBK = 32, kGPad = 8;

__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void cp_async16(void* s, const void* g) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_u32(s)), "l"(g));
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cp_wait0() { asm volatile("cp.async.wait_group 0;\n" ::); }

__device__ __forceinline__ void ldm_x4(unsigned (&r)[4], const void* p) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(smem_u32(p)));
}
__device__ __forceinline__ void ldm_x4_t(unsigned (&r)[4], const void* p) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(smem_u32(p)));
}
__device__ __forceinline__ void mma_bf16(float (&c)[4], const unsigned (&a)[4], unsigned b0,
                                         unsigned b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// Shared-memory tile geometry: the stored orientation is kept.
template <bool T, int ROWS_NT, int ROWS_T>
struct TileShape {
  // not transposed: [ROWS_NT][kGBK + pad]; transposed: [kGBK][ROWS_T + pad]
  static constexpr int rows = T ? kGBK : ROWS_NT;
  static constexpr int cols = T ? ROWS_T + kGPad : kGBK + kGPad;
  static constexpr int elems = rows * cols;
};

template <bool AT, bool BT, int EPI>
__global__ void __launch_bounds__(256) gemm_bf16_kernel(GemmArgs g) {
  using TA = TileShape<AT, kGBM, kGBM>;
  using TB = TileShape<!BT, kGBN, kGBN>;   // B stored [K][N] is the "transposed" case
  __shared__ __align__(16) __nv_bfloat16 sA[2][TA::elems];
  __shared__ __align__(16) __nv_bfloat16 sB[2][TB::elems];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int wm = warp & 1, wn = warp >> 1;            // 2 x 4 warps
  const int m0 = blockIdx.y * kGBM, n0 = blockIdx.x * kGBN;
  const int ksplit = gridDim.z;
  const int kchunk = g.K / ksplit;
  const int kbeg = blockIdx.z * kchunk, kend = kbeg + kchunk;

  auto load_tile = [&](int st, int k0) {
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      const int idx = tid + c * 256;                   // 512 chunks of 8 elements
      if (!AT) {                                       // A [M][K]: 128 rows x 4 chunks
        const int r = idx >> 2, q = idx & 3;
        cp_async16(&sA[st][r * TA::cols + q * 8], g.A + (size_t)(m0 + r) * g.lda + k0 + q * 8);
      } else {                                         // A^T [K][M]: 32 rows x 16 chunks
        const int r = idx >> 4, q = idx & 15;
        cp_async16(&sA[st][r * TA::cols + q * 8], g.A + (size_t)(k0 + r) * g.lda + m0 + q * 8);
      }
      if (BT) {                                        // B [N][K]: 128 rows x 4 chunks
        const int r = idx >> 2, q = idx & 3;
        cp_async16(&sB[st][r * TB::cols + q * 8], g.B + (size_t)(n0 + r) * g.ldb + k0 + q * 8);
      } else {                                         // B [K][N]: 32 rows x 16 chunks
        const int r = idx >> 4, q = idx & 15;
        cp_async16(&sB[st][r * TB::cols + q * 8], g.B + (size_t)(k0 + r) * g.ldb + n0 + q * 8);
      }
    }
    cp_commit();
  };

  float acc[4][4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int e = 0; e < 4; ++e) acc[i][j][e] = 0.f;

  int st = 0;
  load_tile(0, kbeg);
  for (int k0 = kbeg; k0 < kend; k0 += kGBK) {
    cp_wait0();
    __syncthreads();
    if (k0 + kGBK < kend) load_tile(st ^ 1, k0 + kGBK);
    const __nv_bfloat16* a_s = sA[st];
    const __nv_bfloat16* b_s = sB[st];
#pragma unroll
    for (int kk = 0; kk < kGBK; kk += 16) {
      unsigned af[4][4];
      const int i8 = lane >> 3, r8 = lane & 7;
#pragma unroll
      for (int mi = 0; mi < 4; ++mi) {
        const int mb = wm * 64 + mi * 16;
        if (!AT) {
          const int m = mb + r8 + (i8 & 1) * 8, k = kk + (i8 >> 1) * 8;
          ldm_x4(af[mi], &a_s[m * TA::cols + k]);
        } else {
          const int k = kk + r8 + (i8 >> 1) * 8, m = mb + (i8 & 1) * 8;
          ldm_x4_t(af[mi], &a_s[k * TA::cols + m]);
        }
      }
#pragma unroll
      for (int nj = 0; nj < 2; ++nj) {
        const int nb = wn * 32 + nj * 16;
        unsigned bf[4];
        if (BT) {
          const int n = nb + r8 + (i8 >> 1) * 8, k = kk + (i8 & 1) * 8;
          ldm_x4(bf, &b_s[n * TB::cols + k]);
        } else {
          const int k = kk + r8 + (i8 & 1) * 8, n = nb + (i8 >> 1) * 8;
          ldm_x4_t(bf, &b_s[k * TB::cols + n]);
        }
#pragma unroll
        for (int mi = 0; mi < 4; ++mi) {
          mma_bf16(acc[mi][nj * 2 + 0], af[mi], bf[0], bf[1]);
          mma_bf16(acc[mi][nj * 2 + 1], af[mi], bf[2], bf[3]);
        }
      }
    }
    st ^= 1;
  }

  // epilogue
#pragma unroll
  for (int mi = 0; mi < 4; ++mi) {
#pragma unroll
    for (int ni = 0; ni < 4; ++ni) {
      const int col = n0 + wn * 32 + ni * 8 + (lane & 3) * 2;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int row = m0 + wm * 64 + mi * 16 + (lane >> 2) + h * 8;
        float v0 = acc[mi][ni][h * 2 + 0], v1 = acc[mi][ni][h * 2 + 1];
        if (EPI == EPI_ATOMIC) {
          float* C = (float*)g.C + (size_t)row * g.ldc + col;
          atomicAdd(C, v0);
          atomicAdd(C + 1, v1);
          continue;
        }
        if (g.bias && (EPI == EPI_F32 || EPI == EPI_BF16_RELU || EPI == EPI_BF16)) {
          v0 += g.bias[col];
          v1 += g.bias[col + 1];
        }
        if (EPI == EPI_F32) {
          float2* C = (float2*)((float*)g.C + (size_t)row * g.ldc + col);
          *C = make_float2(v0, v1);
        } else {
          if (EPI == EPI_BF16_RELU) {
            v0 = fmaxf(v0, 0.f);
            v1 = fmaxf(v1, 0.f);
          } else if (EPI == EPI_BF16_MASK) {
            const __nv_bfloat162 a2 =
                *(const __nv_bfloat162*)(g.aux + (size_t)row * g.ldc + col);
            if (!(__bfloat162float(a2.x) > 0.f)) v0 = 0.f;
            if (!(__bfloat162float(a2.y) > 0.f)) v1 = 0.f;
          }
          *(__nv_bfloat162*)((__nv_bfloat16*)g.C + (size_t)row * g.ldc + col) =
              __floats2bfloat162_rn(v0, v1);
        }
      }
    }
  }
}

}  // namespace sk
