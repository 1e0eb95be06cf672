// sk_mlp.cu -- the move-proposal network of the learned tempering chains
// (an addition to Sec. 3): occupancy of the 2n bins -> 256 ReLU -> 256 ReLU
// -> one logit per move (k, s), BF16 weights with FP32 accumulation and FP32
// master weights, trained on the GPU with hand-written forward/backward and
// Adam.  Target of a state C: t(m) ~ exp(-beta* dE(m)) over its valid moves;
// loss: cross entropy of the masked softmax.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <random>
#include <vector>

#include "sk_exact_launch.cuh"
#include "sk_gemm.cuh"
#include "sk_gemm_tc.cuh"
#include "sk_host_common.h"
#include "sk_mlp.cuh"

namespace sk {

template <bool AT, bool BT, int EPI>
cudaError_t gemm(const GemmArgs& g, int splits, cudaStream_t s) {
  if (g.M % kGBM || g.N % kGBN || g.K % (kGBK * splits)) return cudaErrorInvalidValue;
  dim3 grid(g.N / kGBN, g.M / kGBM, splits);
  gemm_bf16_kernel<AT, BT, EPI><<<grid, 256, 0, s>>>(g);
  return cudaGetLastError();
}

// X[b][i] = occupancy of bin i of state b (0 beyond 2n; n <= 40, so the
// bins fit a 128-entry histogram).  One warp per
// state: the pairs are counted into a shared histogram, then each lane
// writes four adjacent bf16 inputs (one 8-byte store; a row is 256 bytes).
__global__ void __launch_bounds__(256) mlp_inputs_kernel(const unsigned char* __restrict__ slots,
                                                         int B, int n, int delta, int K1,
                                                         __nv_bfloat16* X) {
  __shared__ unsigned occ[8][128];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int b = blockIdx.x * 8 + w;
  if (b >= B) return;
  for (int i = lane; i < 128; i += 32) occ[w][i] = 0;
  __syncwarp();
  for (int k = 1 + lane; k <= n; k += 32) {
    const int s = slots[(size_t)b * n + (k - 1)];
    if (s < 2 * n - (k + delta)) {      // a start outside the pair's range counts nothing
      atomicAdd(&occ[w][s], 1u);
      atomicAdd(&occ[w][s + k + delta], 1u);
    }
  }
  __syncwarp();
  for (int c = lane * 4; c < K1; c += 128) {
    unsigned short h[4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
      h[i] = __bfloat16_as_ushort(__float2bfloat16((c + i < 2 * n) ? (float)occ[w][c + i] : 0.f));
    *(uint2*)(X + (size_t)b * K1 + c) =
        make_uint2((unsigned)h[0] | ((unsigned)h[1] << 16), (unsigned)h[2] | ((unsigned)h[3] << 16));
  }
}

// Bias gradients: column sums of a [rows][cols] bf16 matrix in two passes of
// fixed order (the same bits every call).  Pass 1: block (x, y) sums rows
// y*kColRows .. of 32 columns, 8 row phases per column (a warp reads 32
// adjacent columns of one row), then the phases in order in shared memory,
// into part[y][c].  Pass 2 (splitk_sum_kernel) adds the parts in order y.
constexpr int kColRows = 128;
__global__ void colsum_part_kernel(const __nv_bfloat16* __restrict__ in, int rows, int cols,
                                   float* __restrict__ part) {
  __shared__ float s[8][33];
  const int c = blockIdx.x * 32 + threadIdx.x;
  const int r0 = blockIdx.y * kColRows, r1 = min(rows, r0 + kColRows);
  float a = 0.f;
  if (c < cols)
    for (int r = r0 + threadIdx.y; r < r1; r += 8) a += __bfloat162float(in[(size_t)r * cols + c]);
  s[threadIdx.y][threadIdx.x] = a;
  __syncthreads();
  if (threadIdx.y == 0 && c < cols) {
    float t = 0.f;
    for (int i = 0; i < 8; ++i) t += s[i][threadIdx.x];
    part[(size_t)blockIdx.y * cols + c] = t;
  }
}

// Adam (Kingma & Ba 2015) over the flat parameter vector; refreshes the bf16
// copies of the weight matrices.
__global__ void adam_kernel(float* w, const float* g, float* m, float* v, size_t count, float lr,
                            float b1, float b2, float eps, float c1, float c2,
                            __nv_bfloat16* wb, size_t nweights_b) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count;
       i += (size_t)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float wi = w[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    w[i] = wi;
    if (i < nweights_b) wb[i] = __float2bfloat16(wi);
  }
}

__global__ void f32_to_bf16_kernel(const float* in, __nv_bfloat16* out, size_t count) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count;
       i += (size_t)gridDim.x * blockDim.x)
    out[i] = __float2bfloat16(in[i]);
}

}  // namespace sk

namespace sk {

// One warp per state: target t(m) ~ exp(-beta* dE(m)) over the valid moves,
// q = masked softmax of the logits, dZ = (q - t) / B, loss += -sum t log q / B.
// The state's logit row is loaded at once into registers (CH chunks of 256
// moves, lane l holding moves 256 c + 8 l .. + 7, two 16-byte loads a chunk);
// the pair and slot of each move come from a per-block table, dE from the
// state's bin counts in shared memory.  One instantiation per CH = NMp / 256.
template <int CH>
__global__ void __launch_bounds__(256)
    mlp_loss_kernel(const float* __restrict__ Z, int ldz, const unsigned char* __restrict__ slots,
                    int B, MoveTable mt, float beta_star, float inv_B, __nv_bfloat16* dZ,
                    float* loss) {
  __shared__ unsigned char mk[CH * 256], msl[CH * 256];
  __shared__ int s_occ[8][2 * kPtMaxN];
  __shared__ unsigned char s_slot[8][kPtMaxN + 1];
  for (int m = threadIdx.x; m < CH * 256; m += blockDim.x) {
    int k = 0, sl = 0;
    if (m < mt.NM) {                       // the pair with off[k] <= m < off[k+1]
      int lo = 1, hi = mt.n;
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (mt.off[mid] <= m) lo = mid;
        else hi = mid - 1;
      }
      k = lo;
      sl = m - mt.off[lo];
    }
    mk[m] = (unsigned char)k;
    msl[m] = (unsigned char)sl;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int b = blockIdx.x * 8 + w;
  if (b >= B) return;
  const int n = mt.n, NM = mt.NM;
  float z[CH][8];
  const float* zr = Z + (size_t)b * ldz;
#pragma unroll
  for (int c = 0; c < CH; ++c) {
    const int m0 = c * 256 + lane * 8;
    float4 a = make_float4(0.f, 0.f, 0.f, 0.f), e = a;
    if (m0 < NM) {
      a = __ldg((const float4*)(zr + m0));
      e = __ldg((const float4*)(zr + m0 + 4));
    }
    z[c][0] = a.x; z[c][1] = a.y; z[c][2] = a.z; z[c][3] = a.w;
    z[c][4] = e.x; z[c][5] = e.y; z[c][6] = e.z; z[c][7] = e.w;
  }
  for (int i = lane; i < 2 * n; i += 32) s_occ[w][i] = 0;
  if (lane == 0) s_slot[w][0] = 0;
  __syncwarp();
  for (int k = 1 + lane; k <= n; k += 32) {           // lane k-1 places pair k
    const int s = slots[(size_t)b * n + (k - 1)];
    s_slot[w][k] = (unsigned char)s;
    atomicAdd(&s_occ[w][s], 1);
    atomicAdd(&s_occ[w][s + k + mt.delta], 1);
  }
  __syncwarp();
  // valid moves and their dE
  int de[CH][8];
  unsigned vb[CH];
  float zmax = -INFINITY;
  int demin = 1 << 20;
#pragma unroll
  for (int c = 0; c < CH; ++c) {
    vb[c] = 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int m = c * 256 + lane * 8 + i;
      const int k = mk[m], sl = msl[m];
      const int sk = s_slot[w][k];
      const bool v = m < NM && sl != sk;     // padding: pair 0, slot 0 = s_slot[0]
      de[c][i] = v ? move_delta_e(s_occ[w], sk, k + mt.delta, sl) : 0;
      vb[c] |= (unsigned)v << i;
      if (v) {
        zmax = fmaxf(zmax, z[c][i]);
        demin = min(demin, de[c][i]);
      }
    }
  }
  zmax = warp_max(zmax);
#pragma unroll
  for (int o = 16; o; o >>= 1) demin = min(demin, __shfl_xor_sync(0xffffffffu, demin, o));
  const float wmax = -beta_star * (float)demin;
  float sq = 0.f, stt = 0.f;
#pragma unroll
  for (int c = 0; c < CH; ++c)
#pragma unroll
    for (int i = 0; i < 8; ++i)
      if ((vb[c] >> i) & 1u) {
        sq += __expf(z[c][i] - zmax);
        stt += __expf(-beta_star * (float)de[c][i] - wmax);
      }
  sq = warp_sum(sq);
  stt = warp_sum(stt);
  const float lse = zmax + __logf(sq);
  float l = 0.f;
  __nv_bfloat16* dz = dZ + (size_t)b * ldz;
#pragma unroll
  for (int c = 0; c < CH; ++c) {
    unsigned wd[4];
#pragma unroll
    for (int i = 0; i < 8; i += 2) {
      float g[2];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        g[h] = 0.f;
        if ((vb[c] >> (i + h)) & 1u) {
          const float q = __expf(z[c][i + h] - lse);
          const float t = __expf(-beta_star * (float)de[c][i + h] - wmax) / stt;
          g[h] = (q - t) * inv_B;
          l -= t * (z[c][i + h] - lse);
        }
      }
      const __nv_bfloat162 p2 = __floats2bfloat162_rn(g[0], g[1]);
      wd[i / 2] = *(const unsigned*)&p2;
    }
    *(uint4*)(dz + c * 256 + lane * 8) = make_uint4(wd[0], wd[1], wd[2], wd[3]);
  }
  l = warp_sum(l);
  if (lane == 0) atomicAdd(loss, l * inv_B);
}

// The loss kernel for the model's move-table size (NMp / 256 chunks).
static cudaError_t launch_loss(const Mlp& m, int B, float beta_star, float* loss, cudaStream_t s) {
  const MoveTable mt = move_table(m);
  const dim3 grid((B + 7) / 8), block(256);
  switch (m.NMp / 256) {
#define SK_LOSS_CASE(c)                                                                     \
  case c:                                                                                   \
    mlp_loss_kernel<c><<<grid, block, 0, s>>>(m.Z, m.NMp, m.slots, B, mt, beta_star,       \
                                              1.0f / (float)B, m.dZ, loss);                 \
    break;
    SK_LOSS_CASE(1) SK_LOSS_CASE(2) SK_LOSS_CASE(3) SK_LOSS_CASE(4) SK_LOSS_CASE(5)
    SK_LOSS_CASE(6) SK_LOSS_CASE(7) SK_LOSS_CASE(8) SK_LOSS_CASE(9) SK_LOSS_CASE(10)
#undef SK_LOSS_CASE
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

MoveTable move_table(const Mlp& m) {
  MoveTable t;
  std::memset(&t, 0, sizeof(t));
  t.n = m.n;
  t.delta = m.delta;
  t.NM = m.NM;
  for (int k = 1; k <= m.n + 1; ++k) t.off[k] = m.off[k];
  return t;
}

// Up to three transposes in one launch: out[c][r] = in[r][c] for a
// [rows][cols] bf16 matrix (rows, cols multiples of 64; blockIdx.z picks the
// matrix).  64 x 64 tiles move in 16-byte pieces through shared memory (row
// pitch 66 elements: the 4-byte stores of a warp hit distinct banks).  With
// part, the tile's column sums over its 64 rows are also written, in a fixed
// order, to part[r0 / 64][c] (the first pass of a bias gradient).
struct TransposeJob {
  const __nv_bfloat16* in;
  __nv_bfloat16* out;
  float* part;
  int rows, cols;
};
struct TransposeJobs {
  TransposeJob j[3];
};

__global__ void __launch_bounds__(256) transpose_set_kernel(TransposeJobs jobs) {
  __shared__ __align__(16) __nv_bfloat16 t[64][66];
  // this block's matrix, chosen field by field (a dynamic index into the
  // parameter array would copy it to local memory)
  const int z = blockIdx.z;
  TransposeJob J;
  J.in = z == 0 ? jobs.j[0].in : (z == 1 ? jobs.j[1].in : jobs.j[2].in);
  J.out = z == 0 ? jobs.j[0].out : (z == 1 ? jobs.j[1].out : jobs.j[2].out);
  J.part = z == 0 ? jobs.j[0].part : (z == 1 ? jobs.j[1].part : jobs.j[2].part);
  J.rows = z == 0 ? jobs.j[0].rows : (z == 1 ? jobs.j[1].rows : jobs.j[2].rows);
  J.cols = z == 0 ? jobs.j[0].cols : (z == 1 ? jobs.j[1].cols : jobs.j[2].cols);
  const int c0 = blockIdx.x * 64, r0 = blockIdx.y * 64;
  if (c0 >= J.cols || r0 >= J.rows) return;          // a smaller matrix's spare blocks
  for (int q = threadIdx.x; q < 512; q += 256) {
    const int i = q >> 3, c8 = (q & 7) * 8;
    const uint4 v = *(const uint4*)(J.in + (size_t)(r0 + i) * J.cols + c0 + c8);
    unsigned* dst = (unsigned*)&t[i][c8];
    dst[0] = v.x;
    dst[1] = v.y;
    dst[2] = v.z;
    dst[3] = v.w;
  }
  __syncthreads();
  for (int q = threadIdx.x; q < 512; q += 256) {
    const int o = q >> 3, r8 = (q & 7) * 8;          // output row c0 + o, columns r0 + r8 ..
    unsigned w[4];
#pragma unroll
    for (int k = 0; k < 4; ++k)
      w[k] = (unsigned)__bfloat16_as_ushort(t[r8 + 2 * k][o]) |
             ((unsigned)__bfloat16_as_ushort(t[r8 + 2 * k + 1][o]) << 16);
    *(uint4*)(J.out + (size_t)(c0 + o) * J.rows + r0 + r8) = make_uint4(w[0], w[1], w[2], w[3]);
  }
  if (J.part && threadIdx.x < 64) {
    float a = 0.f;
    for (int i = 0; i < 64; ++i) a += __bfloat162float(t[i][threadIdx.x]);
    J.part[(size_t)blockIdx.y * J.cols + c0 + threadIdx.x] = a;
  }
}

static cudaError_t transpose_set(const TransposeJob* jobs, int count, cudaStream_t s) {
  TransposeJobs J;
  std::memset(&J, 0, sizeof(J));
  int gx = 1, gy = 1;
  for (int i = 0; i < count; ++i) {
    if (jobs[i].rows % 64 || jobs[i].cols % 64) return cudaErrorInvalidValue;
    J.j[i] = jobs[i];
    gx = std::max(gx, jobs[i].cols / 64);
    gy = std::max(gy, jobs[i].rows / 64);
  }
  transpose_set_kernel<<<dim3(gx, gy, count), 256, 0, s>>>(J);
  return cudaGetLastError();
}

// The K-major (transposed) bf16 weights of the tcgen05 forward, one launch.
cudaError_t refresh_transposed(Mlp& m, cudaStream_t s) {
  const TransposeJob jobs[3] = {{m.W1, m.W1t, nullptr, m.K1, kHidden},
                                {m.W2, m.W2t, nullptr, kHidden, kHidden},
                                {m.W3, m.W3t, nullptr, kHidden, m.NMp}};
  cudaError_t e = transpose_set(jobs, 3, s);
  if (e == cudaSuccess) m.wt_dirty = 0;
  return e;
}

// The driver's tensor-map encoder, found through the runtime (no link
// against the driver library).
static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)f;
  }
  return fn;
}

// 2D tensor map of a row-major [rows][cols] matrix of bf16 (esize 2) or
// fp32 (esize 4), box [box_rows][128 bytes], 128-byte swizzle.
// A 2-D map of rows x cols elements, ld elements between rows (ld >= cols;
// 0: ld = cols); boxes of 128 bytes x box_rows, 128-byte swizzle.  A TMA
// store writes only the part of a box inside the map.
static bool encode_map(CUtensorMap* map, const void* ptr, int esize, int rows, int cols,
                       int box_rows, int ld = 0, bool promote256 = true) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (!enc) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)(ld > 0 ? ld : cols) * esize};
  const cuuint32_t box[2] = {(cuuint32_t)(128 / esize), (cuuint32_t)box_rows};
  const cuuint32_t estr[2] = {1, 1};
  return enc(map, esize == 2 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32,
             2, const_cast<void*>(ptr), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
             CU_TENSOR_MAP_SWIZZLE_128B,
             promote256 ? CU_TENSOR_MAP_L2_PROMOTION_L2_256B : CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

static bool make_tc_maps(Mlp& m) {
  // X: the first layer reads the first K1f (64 for n <= 32) of each row's
  // K1 = 128 columns, so its loads are promoted in L2 by 128 bytes only
  return encode_map(&m.tmA[0], m.X, 2, m.max_batch, m.K1, kTcBM, 0, m.K1f >= m.K1) &&
         encode_map(&m.tmA[1], m.H1, 2, m.max_batch, kHidden, kTcBM) &&
         encode_map(&m.tmA[2], m.H2, 2, m.max_batch, kHidden, kTcBM) &&
         encode_map(&m.tmB[0], m.W1t, 2, kHidden, m.K1, kTcBN) &&
         encode_map(&m.tmB[1], m.W2t, 2, kHidden, kHidden, kTcBN) &&
         encode_map(&m.tmB[2], m.W3t, 2, m.NMp, kHidden, kTcBN) &&
         encode_map(&m.tmC[0], m.H1, 2, m.max_batch, kHidden, 32) &&
         encode_map(&m.tmC[1], m.H2, 2, m.max_batch, kHidden, 32) &&
         encode_map(&m.tmC[2], m.Z, 4, m.max_batch, m.NMp, 32) &&
         // the chains' bf16 logits: only the move table's columns (rounded
         // up to 8, whole 16-byte words; those columns' weights are 0) are
         // stored, the row stride stays NMp
         encode_map(&m.tmZb, m.Z, 2, m.max_batch, (m.NM + 7) / 8 * 8, 32, m.NMp) &&
         encode_map(&m.tmBA[0], m.dZ, 2, m.max_batch, m.NMp, kTcBM) &&
         encode_map(&m.tmBA[1], m.dH2, 2, m.max_batch, kHidden, kTcBM) &&
         encode_map(&m.tmBB[0], m.W3, 2, kHidden, m.NMp, kTcBN) &&
         encode_map(&m.tmBB[1], m.W2, 2, kHidden, kHidden, kTcBN) &&
         encode_map(&m.tmBC[0], m.dH2, 2, m.max_batch, kHidden, 32) &&
         encode_map(&m.tmBC[1], m.dH1, 2, m.max_batch, kHidden, 32);
}

// The shared-memory opt-in is a per-device function attribute: set it once
// per device, with that device current, for every instantiation used.
static cudaError_t tc_attributes(int* dev_out) {
  int dev = 0;
  cudaError_t e0 = cudaGetDevice(&dev);
  if (e0 != cudaSuccess) return e0;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  static std::once_flag once[kMaxDevices];
  static cudaError_t attr_err[kMaxDevices];
  std::call_once(once[dev], [dev]() {
    const cudaFuncAttribute at = cudaFuncAttributeMaxDynamicSharedMemorySize;
    cudaError_t e = cudaFuncSetAttribute(gemm_tc_kernel<kTcEpiReluBf16, false>, at, kTcSmem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(gemm_tc_kernel<kTcEpiF32, false>, at, kTcSmem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(gemm_tc_kernel<kTcEpiBf16, false>, at, kTcSmem);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(gemm_tc_kernel<kTcEpiMaskBf16, true>, at, kTcSmemStream);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(gemm_tc_kernel<kTcEpiF32, true>, at, kTcSmemStream);
    attr_err[dev] = e;
  });
  *dev_out = dev;
  return attr_err[dev];
}

// C = A B^T on tcgen05 (epilogue EPI; STREAMB: B streamed through the ring,
// any K; a K split of g.ksplit ranges writes its partials to rows ks * M..).
// Grid: one CTA per SM, a whole number of CTAs per (column tile, K range).
template <int EPI, bool STREAMB>
cudaError_t gemm_tc_launch(const TcGemmArgs& g, const CUtensorMap& amap, const CUtensorMap& bmap,
                           const CUtensorMap& cmap, cudaStream_t s) {
  const int KS = g.ksplit > 1 ? g.ksplit : 1;
  if (g.M <= 0 || g.K <= 0 || g.M % kTcBM || g.N % kTcBN || g.K % (kTcBK * KS))
    return cudaErrorInvalidValue;
  if (!STREAMB && (g.K > kTcMaxK || KS > 1)) return cudaErrorInvalidValue;
  if (EPI == kTcEpiMaskBf16 && (!g.aux || g.ldaux % 8)) return cudaErrorInvalidValue;
  // a narrowed last column tile keeps at least one column
  if (g.nvalid < 0 || g.nvalid > g.N || (g.nvalid > 0 && g.nvalid <= g.N - kTcBN))
    return cudaErrorInvalidValue;
  int dev = 0;
  cudaError_t e = tc_attributes(&dev);
  if (e != cudaSuccess) return e;
  const int sms = device_sm_count(dev);
  const int NT = g.N / kTcBN, MT = g.M / kTcBM;
  int per = sms / (NT * KS);
  if (per < 1) per = 1;
  if (per > MT) per = MT;
  const int grid = per * NT * KS;
  if (g.pdl) return launch_dependent(gemm_tc_kernel<EPI, STREAMB>, grid, kTcThreads,
                                     STREAMB ? kTcSmemStream : kTcSmem, s, amap, bmap, cmap, g);
  gemm_tc_kernel<EPI, STREAMB><<<grid, kTcThreads, STREAMB ? kTcSmemStream : kTcSmem, s>>>(
      amap, bmap, cmap, g);
  return cudaGetLastError();
}

// The forward's layers: epi = kTcEpiReluBf16 (hidden layers), kTcEpiF32 or
// kTcEpiBf16 (logits).
cudaError_t gemm_tc(const TcGemmArgs& g, const CUtensorMap& amap, const CUtensorMap& bmap,
                    const CUtensorMap& cmap, int epi, cudaStream_t s) {
  if (epi == kTcEpiReluBf16) return gemm_tc_launch<kTcEpiReluBf16, false>(g, amap, bmap, cmap, s);
  if (epi == kTcEpiBf16) return gemm_tc_launch<kTcEpiBf16, false>(g, amap, bmap, cmap, s);
  return gemm_tc_launch<kTcEpiF32, false>(g, amap, bmap, cmap, s);
}

// Forward pass for B (multiple of 128) states whose slots are already in
// m.slots: X, H1, H2 (bf16) and Z (fp32 logits, or bf16 with logits_bf16).
cudaError_t mlp_forward_dev(Mlp& m, int B, cudaStream_t s, bool logits_bf16, bool inputs_ready,
                            cudaEvent_t before_l2, bool dependent) {
  if (!inputs_ready)
    mlp_inputs_kernel<<<(B + 7) / 8, 256, 0, s>>>(m.slots, B, m.n, m.delta, m.K1, m.X);
  if (m.use_tc) {
    cudaError_t e = cudaSuccess;
    if (m.wt_dirty) e = refresh_transposed(m, s);
    if (e != cudaSuccess) return e;
    TcGemmArgs t;
    std::memset(&t, 0, sizeof(t));
    t.M = B; t.N = kHidden; t.K = m.K1f; t.bias = m.b1; t.err = m.tc_err;
    e = gemm_tc(t, m.tmA[0], m.tmB[0], m.tmC[0], kTcEpiReluBf16, s);
    if (e == cudaSuccess && before_l2) e = cudaStreamWaitEvent(s, before_l2, 0);
    if (e != cudaSuccess) return e;
    t.K = kHidden; t.bias = m.b2; t.pdl = dependent ? 1 : 0;
    e = gemm_tc(t, m.tmA[1], m.tmB[1], m.tmC[1], kTcEpiReluBf16, s);
    if (e != cudaSuccess) return e;
    t.N = m.NMp; t.bias = m.b3;
    if (logits_bf16) t.nvalid = (m.NM + 7) / 8 * 8;   // the columns tmZb stores
    return logits_bf16 ? gemm_tc(t, m.tmA[2], m.tmB[2], m.tmZb, kTcEpiBf16, s)
                       : gemm_tc(t, m.tmA[2], m.tmB[2], m.tmC[2], kTcEpiF32, s);
  }
  GemmArgs g;
  std::memset(&g, 0, sizeof(g));
  g.M = B; g.N = kHidden; g.K = m.K1f; g.A = m.X; g.lda = m.K1; g.B = m.W1; g.ldb = kHidden;
  g.C = m.H1; g.ldc = kHidden; g.bias = m.b1;
  cudaError_t e = gemm<false, false, EPI_BF16_RELU>(g, 1, s);
  if (e == cudaSuccess && before_l2) e = cudaStreamWaitEvent(s, before_l2, 0);
  if (e != cudaSuccess) return e;
  g.K = kHidden; g.A = m.H1; g.lda = kHidden; g.B = m.W2; g.C = m.H2; g.bias = m.b2;
  e = gemm<false, false, EPI_BF16_RELU>(g, 1, s);
  if (e != cudaSuccess) return e;
  g.N = m.NMp; g.A = m.H2; g.B = m.W3; g.ldb = m.NMp; g.C = m.Z; g.ldc = m.NMp; g.bias = m.b3;
  return logits_bf16 ? gemm<false, false, EPI_BF16>(g, 1, s) : gemm<false, false, EPI_F32>(g, 1, s);
}

// out[i] = sum over ks of ws[ks][i], in the order ks = 0, 1, ... (the K
// split's partial products, summed the same way every call).
__global__ void splitk_sum_kernel(const float* __restrict__ ws, int KS, size_t count,
                                  float* __restrict__ out) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count;
       i += (size_t)gridDim.x * blockDim.x) {
    float a = 0.f;
    for (int k = 0; k < KS; ++k) a += ws[(size_t)k * count + i];
    out[i] = a;
  }
}

// K ranges of a weight-gradient product: a power of two that divides the K
// slices, at most 16, aiming at one CTA per SM.
static int ksplit_for(int tiles, int kslices, int sms) {
  int ks = 1;
  while (ks < 16 && tiles * ks * 2 <= sms && kslices % (ks * 2) == 0) ks *= 2;
  return ks;
}

// gW[i] = sum over ks of ws[ks][i] (i < MN, the K split's partial products)
// and gb[c] = sum over p of part[p][c] (c < N, the column sums of the
// transpose's 64-row tiles), each in a fixed order: the last pass of a weight
// gradient and of its bias gradient in one launch.
__global__ void grad_finish_kernel(const float* __restrict__ ws, int KS, size_t MN, float* gW,
                                   const float* __restrict__ part, int parts, int N, float* gb) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < MN + N;
       i += (size_t)gridDim.x * blockDim.x) {
    float a = 0.f;
    if (i < MN) {
      for (int k = 0; k < KS; ++k) a += ws[(size_t)k * MN + i];
      gW[i] = a;
    } else {
      const size_t c = i - MN;
      for (int p = 0; p < parts; ++p) a += part[(size_t)p * N + c];
      gb[c] = a;
    }
  }
}

// The workspace of the tcgen05 backward for batches up to B: K-major copies
// TA [256][B] and TB [NMp][B] of the weight-gradient operands, 16 K-split
// partials of the largest weight gradient, and the bias gradients' column
// sums of 64-row tiles [B / 64][NMp].  Grown on demand.
struct BwdSpace {
  __nv_bfloat16 *TA, *TB;
  float *WS, *part;
};
static cudaError_t bwd_workspace(Mlp& m, int B, BwdSpace* w) {
  auto a256 = [](size_t x) { return (x + 255) / 256 * 256; };
  const size_t wide = m.NMp > kHidden ? m.NMp : kHidden;
  const size_t ta = a256((size_t)kHidden * B * 2), tb = a256((size_t)m.NMp * B * 2),
               ws = a256((size_t)16 * kHidden * wide * 4), pt = (size_t)(B / 64) * wide * 4;
  if (ta + tb + ws + pt > m.bwd_bytes) {
    if (m.bwd_ws) cudaFree(m.bwd_ws);
    m.bwd_ws = nullptr;
    m.bwd_bytes = 0;
    cudaError_t e = cudaMalloc(&m.bwd_ws, ta + tb + ws + pt);
    if (e != cudaSuccess) return e;
    m.bwd_bytes = ta + tb + ws + pt;
  }
  char* p = (char*)m.bwd_ws;
  w->TA = (__nv_bfloat16*)p;
  w->TB = (__nv_bfloat16*)(p + ta);
  w->WS = (float*)(p + ta + tb);
  w->part = (float*)(p + ta + tb + ws);
  return cudaSuccess;
}

// One weight gradient gW [M][N] (fp32) = A^T D and its bias gradient gb [N]
// = the column sums of D, on tcgen05; A [B][M] and D [B][N] bf16 row-major:
// both transposed to K-major copies in one launch (which also sums D's
// 64-row tiles), the K = B reduction split over CTAs, then the partials of
// both summed in a fixed order.
static cudaError_t weight_grad_tc(Mlp& m, int B, const __nv_bfloat16* A, int M,
                                  const __nv_bfloat16* D, int N, float* gW, float* gb,
                                  const BwdSpace& w, int sms, cudaStream_t s) {
  const TransposeJob jobs[2] = {{A, w.TA, nullptr, B, M}, {D, w.TB, w.part, B, N}};
  cudaError_t e = transpose_set(jobs, 2, s);
  if (e != cudaSuccess) return e;
  const int KS = ksplit_for((M / kTcBM) * (N / kTcBN), B / kTcBK, sms);
  CUtensorMap am, bm, cm;
  if (!encode_map(&am, w.TA, 2, M, B, kTcBM) || !encode_map(&bm, w.TB, 2, N, B, kTcBN) ||
      !encode_map(&cm, w.WS, 4, KS * M, N, 32))
    return cudaErrorInvalidValue;
  TcGemmArgs g;
  std::memset(&g, 0, sizeof(g));
  g.M = M; g.N = N; g.K = B; g.ksplit = KS; g.err = m.tc_err;
  e = gemm_tc_launch<kTcEpiF32, true>(g, am, bm, cm, s);
  if (e != cudaSuccess) return e;
  const size_t MN = (size_t)M * N;
  grad_finish_kernel<<<(unsigned)std::min<size_t>((MN + N + 255) / 256, 1024), 256, 0, s>>>(
      w.WS, KS, MN, gW, w.part, B / 64, N, gb);
  return cudaGetLastError();
}

// out[c] = sum over the B rows of in[r][c] (B a multiple of 128), in a fixed order.
static void colsum(const Mlp& m, const __nv_bfloat16* in, int B, int cols, float* out,
                   cudaStream_t s) {
  const int parts = (B + kColRows - 1) / kColRows;
  colsum_part_kernel<<<dim3((cols + 31) / 32, parts), dim3(32, 8), 0, s>>>(in, B, cols, m.colpart);
  splitk_sum_kernel<<<(cols + 255) / 256, 256, 0, s>>>(m.colpart, parts, (size_t)cols, out);
}

int splits_for(int K) {
  int sp = 1;
  while (sp < 16 && K % (kGBK * sp * 2) == 0 && K / (sp * 2) >= 256) sp *= 2;
  return sp;
}

// The side stream of the tcgen05 backward and its four events, made on first use.
static cudaError_t side_stream(Mlp& m) {
  if (m.side) return cudaSuccess;
  cudaError_t e = cudaStreamCreateWithFlags(&m.side, cudaStreamNonBlocking);
  for (int i = 0; i < 4 && e == cudaSuccess; ++i)
    e = cudaEventCreateWithFlags(&m.ev[i], cudaEventDisableTiming);
  return e;
}

// Loss and gradients of a batch (after mlp_forward_dev): gW*, gb* (fp32).
// The loss goes to *loss when given (accumulated: the caller zeroes it),
// else to m.loss (zeroed here).
cudaError_t mlp_backward_dev(Mlp& m, int B, float beta_star, cudaStream_t s,
                             float* loss = nullptr) {
  cudaError_t e = cudaSuccess;
  if (!m.use_tc) e = cudaMemsetAsync(m.gW1, 0, m.nparams * sizeof(float), s);  // atomics add up
  if (e == cudaSuccess && !loss) e = cudaMemsetAsync(m.loss, 0, sizeof(float), s);
  if (e != cudaSuccess) return e;
  e = launch_loss(m, B, beta_star, loss ? loss : m.loss, s);
  if (e != cudaSuccess) return e;
  if (m.use_tc) {
    // tcgen05: dH = (dZ W^T) * [H > 0] with W streamed as B, on s; the
    // weight and bias gradients (K-major copies, a fixed-order K split) on a
    // side stream, each as soon as its activation gradient exists; s waits
    // for the side stream at the end
    BwdSpace w;
    e = bwd_workspace(m, B, &w);
    if (e == cudaSuccess) e = side_stream(m);
    if (e != cudaSuccess) return e;
    int dev = 0;
    cudaGetDevice(&dev);
    const int sms = device_sm_count(dev);
    e = cudaEventRecord(m.ev[0], s);                               // dZ
    if (e == cudaSuccess) e = cudaStreamWaitEvent(m.side, m.ev[0], 0);
    if (e == cudaSuccess)
      e = weight_grad_tc(m, B, m.H2, kHidden, m.dZ, m.NMp, m.gW3, m.gb3, w, sms, m.side);
    if (e != cudaSuccess) return e;
    TcGemmArgs t;
    std::memset(&t, 0, sizeof(t));
    t.M = B; t.N = kHidden; t.K = m.NMp; t.err = m.tc_err; t.aux = m.H2; t.ldaux = kHidden;
    e = gemm_tc_launch<kTcEpiMaskBf16, true>(t, m.tmBA[0], m.tmBB[0], m.tmBC[0], s);
    if (e == cudaSuccess) e = cudaEventRecord(m.ev[1], s);        // dH2
    if (e == cudaSuccess) e = cudaStreamWaitEvent(m.side, m.ev[1], 0);
    if (e == cudaSuccess)
      e = weight_grad_tc(m, B, m.H1, kHidden, m.dH2, kHidden, m.gW2, m.gb2, w, sms, m.side);
    if (e != cudaSuccess) return e;
    t.K = kHidden; t.aux = m.H1;
    e = gemm_tc_launch<kTcEpiMaskBf16, true>(t, m.tmBA[1], m.tmBB[1], m.tmBC[1], s);
    if (e == cudaSuccess) e = cudaEventRecord(m.ev[2], s);        // dH1
    if (e == cudaSuccess) e = cudaStreamWaitEvent(m.side, m.ev[2], 0);
    if (e == cudaSuccess)
      e = weight_grad_tc(m, B, m.X, m.K1, m.dH1, kHidden, m.gW1, m.gb1, w, sms, m.side);
    if (e == cudaSuccess) e = cudaEventRecord(m.ev[3], m.side);   // every gradient
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, m.ev[3], 0);
    return e;
  }
  GemmArgs g;
  std::memset(&g, 0, sizeof(g));
  const int sp = splits_for(B);
  // dW3 = H2^T dZ
  g.M = kHidden; g.N = m.NMp; g.K = B; g.A = m.H2; g.lda = kHidden; g.B = m.dZ; g.ldb = m.NMp;
  g.C = m.gW3; g.ldc = m.NMp;
  e = gemm<true, false, EPI_ATOMIC>(g, sp, s);
  if (e != cudaSuccess) return e;
  // dH2 = (dZ W3^T) * [H2 > 0]
  std::memset(&g, 0, sizeof(g));
  g.M = B; g.N = kHidden; g.K = m.NMp; g.A = m.dZ; g.lda = m.NMp; g.B = m.W3; g.ldb = m.NMp;
  g.C = m.dH2; g.ldc = kHidden; g.aux = m.H2;
  e = gemm<false, true, EPI_BF16_MASK>(g, 1, s);
  if (e != cudaSuccess) return e;
  // dW2 = H1^T dH2
  std::memset(&g, 0, sizeof(g));
  g.M = kHidden; g.N = kHidden; g.K = B; g.A = m.H1; g.lda = kHidden; g.B = m.dH2;
  g.ldb = kHidden; g.C = m.gW2; g.ldc = kHidden;
  e = gemm<true, false, EPI_ATOMIC>(g, sp, s);
  if (e != cudaSuccess) return e;
  // dH1 = (dH2 W2^T) * [H1 > 0]
  std::memset(&g, 0, sizeof(g));
  g.M = B; g.N = kHidden; g.K = kHidden; g.A = m.dH2; g.lda = kHidden; g.B = m.W2;
  g.ldb = kHidden; g.C = m.dH1; g.ldc = kHidden; g.aux = m.H1;
  e = gemm<false, true, EPI_BF16_MASK>(g, 1, s);
  if (e != cudaSuccess) return e;
  // dW1 = X^T dH1
  std::memset(&g, 0, sizeof(g));
  g.M = m.K1; g.N = kHidden; g.K = B; g.A = m.X; g.lda = m.K1; g.B = m.dH1; g.ldb = kHidden;
  g.C = m.gW1; g.ldc = kHidden;
  e = gemm<true, false, EPI_ATOMIC>(g, sp, s);
  if (e != cudaSuccess) return e;
  // bias gradients: column sums
  colsum(m, m.dZ, B, m.NMp, m.gb3, s);
  colsum(m, m.dH2, B, kHidden, m.gb2, s);
  colsum(m, m.dH1, B, kHidden, m.gb1, s);
  return cudaGetLastError();
}

}  // namespace sk

namespace sk {

__global__ void gather_slots_kernel(const unsigned char* __restrict__ all, const unsigned* __restrict__ idx,
                                    int B, int n, unsigned char* out) {
  const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i >= (size_t)B * n) return;
  const size_t b = i / n, k = i % n;
  out[i] = all[(size_t)idx[b] * n + k];
}

static size_t al256(size_t x) { return (x + 255) / 256 * 256; }

int mlp_create(int variant, int n, int max_batch, uint64_t seed, Mlp** out) {
  if (variant != SK_SKOLEM && variant != SK_LANGFORD) return SK_EINVAL;
  if (n < 2 || n > kMlpMaxN || max_batch < 128 || max_batch % 128) return SK_EINVAL;
  int st = check_device();
  if (st) return st;
  Mlp* m = new Mlp;
  std::memset(m, 0, sizeof(*m));
  m->variant = variant;
  m->n = n;
  m->delta = variant == SK_LANGFORD ? 1 : 0;
  m->bins = 2 * n;
  m->K1 = 128;
  m->K1f = (2 * n + 63) / 64 * 64;
  m->max_batch = max_batch;
  m->off[1] = 0;
  for (int k = 1; k <= n; ++k) m->off[k + 1] = m->off[k] + (2 * n - (k + m->delta));
  m->NM = m->off[n + 1];
  m->NMp = (m->NM + 255) / 256 * 256;
  const size_t w1 = (size_t)m->K1 * kHidden, w2 = (size_t)kHidden * kHidden,
               w3 = (size_t)kHidden * m->NMp;
  m->nparams = w1 + w2 + w3 + 2 * kHidden + m->NMp;
  const size_t B = (size_t)max_batch;
  size_t off = 0;
  const size_t o_par = off; off = al256(off + m->nparams * 4);
  const size_t o_grad = off; off = al256(off + m->nparams * 4);
  const size_t o_am = off; off = al256(off + m->nparams * 4);
  const size_t o_av = off; off = al256(off + m->nparams * 4);
  const size_t o_wb = off; off = al256(off + (w1 + w2 + w3) * 2);
  const size_t o_sl = off; off = al256(off + B * n);
  const size_t o_x = off; off = al256(off + B * m->K1 * 2);
  const size_t o_h1 = off; off = al256(off + B * kHidden * 2);
  const size_t o_h2 = off; off = al256(off + B * kHidden * 2);
  const size_t o_dh1 = off; off = al256(off + B * kHidden * 2);
  const size_t o_dh2 = off; off = al256(off + B * kHidden * 2);
  const size_t o_dz = off; off = al256(off + B * m->NMp * 2);
  const size_t o_z = off; off = al256(off + B * m->NMp * 4);
  const size_t o_loss = off; off = al256(off + 4);
  const size_t o_cp = off; off = al256(off + (B / 128) * (size_t)m->NMp * 4);
  const size_t o_wt = off; off = al256(off + (w1 + w2 + w3) * 2);
  const size_t o_err = off; off = al256(off + 4);
  char* p = nullptr;
  if (cudaMalloc(&p, off) != cudaSuccess) {
    delete m;
    return SK_ENOMEM;
  }
  m->block = p;
  float* par = (float*)(p + o_par);
  m->mW1 = par; m->mW2 = par + w1; m->mW3 = par + w1 + w2;
  m->b1 = par + w1 + w2 + w3; m->b2 = m->b1 + kHidden; m->b3 = m->b2 + kHidden;
  float* gr = (float*)(p + o_grad);
  m->gW1 = gr; m->gW2 = gr + w1; m->gW3 = gr + w1 + w2;
  m->gb1 = gr + w1 + w2 + w3; m->gb2 = m->gb1 + kHidden; m->gb3 = m->gb2 + kHidden;
  m->am = (float*)(p + o_am);
  m->av = (float*)(p + o_av);
  __nv_bfloat16* wb = (__nv_bfloat16*)(p + o_wb);
  m->W1 = wb; m->W2 = wb + w1; m->W3 = wb + w1 + w2;
  m->slots = (unsigned char*)(p + o_sl);
  m->X = (__nv_bfloat16*)(p + o_x);
  m->H1 = (__nv_bfloat16*)(p + o_h1);
  m->H2 = (__nv_bfloat16*)(p + o_h2);
  m->dH1 = (__nv_bfloat16*)(p + o_dh1);
  m->dH2 = (__nv_bfloat16*)(p + o_dh2);
  m->dZ = (__nv_bfloat16*)(p + o_dz);
  m->Z = (float*)(p + o_z);
  m->loss = (float*)(p + o_loss);
  m->colpart = (float*)(p + o_cp);
  __nv_bfloat16* wt = (__nv_bfloat16*)(p + o_wt);
  m->W1t = wt; m->W2t = wt + w1; m->W3t = wt + w1 + w2;
  m->tc_err = (unsigned*)(p + o_err);
  m->use_tc = 1;
  m->wt_dirty = 1;
  if (!make_tc_maps(*m)) {          // the driver could not describe the buffers
    cudaFree(p);
    delete m;
    return SK_ECUDA;
  }
  // He-normal initial weights (input rows beyond 2n and move columns beyond
  // NM stay zero), zero biases
  std::vector<float> h(m->nparams, 0.f);
  std::mt19937_64 rng(seed);
  std::normal_distribution<float> nd(0.f, 1.f);
  const float s1 = std::sqrt(2.f / (float)m->bins), s2 = std::sqrt(2.f / kHidden),
              s3 = std::sqrt(1.f / kHidden);
  for (int i = 0; i < m->bins; ++i)
    for (int j = 0; j < kHidden; ++j) h[(size_t)i * kHidden + j] = s1 * nd(rng);
  for (size_t i = 0; i < w2; ++i) h[w1 + i] = s2 * nd(rng);
  for (int i = 0; i < kHidden; ++i)
    for (int j = 0; j < m->NM; ++j) h[w1 + w2 + (size_t)i * m->NMp + j] = s3 * nd(rng);
  cudaError_t e = cudaMemcpy(par, h.data(), m->nparams * 4, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(m->am, 0, m->nparams * 4);
  if (e == cudaSuccess) e = cudaMemset(m->av, 0, m->nparams * 4);
  if (e == cudaSuccess) e = cudaMemset(m->tc_err, 0, 4);
  if (e == cudaSuccess) {
    f32_to_bf16_kernel<<<256, 256>>>(par, wb, w1 + w2 + w3);
    e = cudaDeviceSynchronize();
  }
  if (e != cudaSuccess) {
    cudaFree(p);
    delete m;
    return cuda_status(e);
  }
  *out = m;
  return SK_OK;
}

// Host parameter layout (unpadded, as in the reference): W1 [2n][256], b1
// [256], W2 [256][256], b2 [256], W3 [256][NM], b3 [NM].
size_t host_param_count(const Mlp& m) {
  return (size_t)m.bins * kHidden + kHidden + (size_t)kHidden * kHidden + kHidden +
         (size_t)kHidden * m.NM + m.NM;
}

// dev (padded layout W1|W2|W3|b1|b2|b3) <-> host (unpadded W1|b1|W2|b2|W3|b3)
void pack_host(const Mlp& m, const float* dev_flat, float* host) {
  const size_t w1 = (size_t)m.K1 * kHidden, w2 = (size_t)kHidden * kHidden,
               w3 = (size_t)kHidden * m.NMp;
  size_t o = 0;
  for (int i = 0; i < m.bins; ++i)
    for (int j = 0; j < kHidden; ++j) host[o++] = dev_flat[(size_t)i * kHidden + j];
  for (int j = 0; j < kHidden; ++j) host[o++] = dev_flat[w1 + w2 + w3 + j];
  for (size_t i = 0; i < w2; ++i) host[o++] = dev_flat[w1 + i];
  for (int j = 0; j < kHidden; ++j) host[o++] = dev_flat[w1 + w2 + w3 + kHidden + j];
  for (int i = 0; i < kHidden; ++i)
    for (int j = 0; j < m.NM; ++j) host[o++] = dev_flat[w1 + w2 + (size_t)i * m.NMp + j];
  for (int j = 0; j < m.NM; ++j) host[o++] = dev_flat[w1 + w2 + w3 + 2 * kHidden + j];
}

void unpack_host(const Mlp& m, const float* host, float* dev_flat) {
  const size_t w1 = (size_t)m.K1 * kHidden, w2 = (size_t)kHidden * kHidden,
               w3 = (size_t)kHidden * m.NMp;
  std::memset(dev_flat, 0, m.nparams * 4);
  size_t o = 0;
  for (int i = 0; i < m.bins; ++i)
    for (int j = 0; j < kHidden; ++j) dev_flat[(size_t)i * kHidden + j] = host[o++];
  for (int j = 0; j < kHidden; ++j) dev_flat[w1 + w2 + w3 + j] = host[o++];
  for (size_t i = 0; i < w2; ++i) dev_flat[w1 + i] = host[o++];
  for (int j = 0; j < kHidden; ++j) dev_flat[w1 + w2 + w3 + kHidden + j] = host[o++];
  for (int i = 0; i < kHidden; ++i)
    for (int j = 0; j < m.NM; ++j) dev_flat[w1 + w2 + (size_t)i * m.NMp + j] = host[o++];
  for (int j = 0; j < m.NM; ++j) dev_flat[w1 + w2 + w3 + 2 * kHidden + j] = host[o++];
}

// Copies B host states into m.slots (zero states pad up to a multiple of
// 128) and returns the padded count.
int upload_states(Mlp& m, const uint8_t* slots, int B, cudaStream_t s, cudaError_t* e) {
  const int Bp = (B + 127) / 128 * 128;
  *e = cudaMemsetAsync(m.slots, 0, (size_t)Bp * m.n, s);
  if (*e == cudaSuccess) *e = cudaMemcpyAsync(m.slots, slots, (size_t)B * m.n, cudaMemcpyHostToDevice, s);
  return Bp;
}

}  // namespace sk

using sk::Mlp;

extern "C" int sk_mlp_create(int variant, int n, int max_batch, uint64_t seed, void** model) {
  if (!model) return SK_EINVAL;
  Mlp* m = nullptr;
  int st = sk::mlp_create(variant, n, max_batch, seed, &m);
  if (st == SK_OK) *model = m;
  return st;
}

extern "C" void sk_mlp_destroy(void* model) {
  Mlp* m = (Mlp*)model;
  if (!m) return;
  if (m->side) {
    cudaStreamSynchronize(m->side);
    for (int i = 0; i < 4; ++i)
      if (m->ev[i]) cudaEventDestroy(m->ev[i]);
    cudaStreamDestroy(m->side);
  }
  if (m->bwd_ws) cudaFree(m->bwd_ws);
  cudaFree(m->block);
  delete m;
}

extern "C" int sk_mlp_dims(const void* model, int* n_moves, int* n_params) {
  const Mlp* m = (const Mlp*)model;
  if (!m) return SK_EINVAL;
  if (n_moves) *n_moves = m->NM;
  if (n_params) *n_params = (int)sk::host_param_count(*m);
  return SK_OK;
}

extern "C" int sk_mlp_set_params(void* model, const float* params) {
  Mlp* m = (Mlp*)model;
  if (!m || !params) return SK_EINVAL;
  std::vector<float> d(m->nparams);
  sk::unpack_host(*m, params, d.data());
  cudaError_t e = cudaMemcpy(m->mW1, d.data(), m->nparams * 4, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(m->am, 0, m->nparams * 4);
  if (e == cudaSuccess) e = cudaMemset(m->av, 0, m->nparams * 4);
  if (e == cudaSuccess) {
    sk::f32_to_bf16_kernel<<<256, 256>>>(m->mW1, m->W1, m->nparams - 2 * sk::kHidden - m->NMp);
    e = cudaDeviceSynchronize();
  }
  m->adam_t = 0;
  m->wt_dirty = 1;
  return sk::cuda_status(e);
}

extern "C" int sk_mlp_get_params(const void* model, float* params) {
  const Mlp* m = (const Mlp*)model;
  if (!m || !params) return SK_EINVAL;
  std::vector<float> d(m->nparams);
  cudaError_t e = cudaMemcpy(d.data(), m->mW1, m->nparams * 4, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return sk::cuda_status(e);
  sk::pack_host(*m, d.data(), params);
  return SK_OK;
}

extern "C" int sk_mlp_get_train_state(const void* model, float* adam_m, float* adam_v,
                                      float* used, int64_t* t) {
  const Mlp* m = (const Mlp*)model;
  if (!m) return SK_EINVAL;
  std::vector<float> d(m->nparams);
  cudaError_t e = cudaSuccess;
  if (adam_m) {
    e = cudaMemcpy(d.data(), m->am, m->nparams * 4, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return sk::cuda_status(e);
    sk::pack_host(*m, d.data(), adam_m);
  }
  if (adam_v) {
    e = cudaMemcpy(d.data(), m->av, m->nparams * 4, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return sk::cuda_status(e);
    sk::pack_host(*m, d.data(), adam_v);
  }
  if (used) {
    // the biases enter the forward as FP32 masters, the weight matrices as
    // their BF16 copies (widened exactly: a bf16 is the top half of a float)
    e = cudaMemcpy(d.data(), m->mW1, m->nparams * 4, cudaMemcpyDeviceToHost);
    const size_t nwb = (size_t)m->K1 * sk::kHidden + (size_t)sk::kHidden * sk::kHidden +
                       (size_t)sk::kHidden * m->NMp;
    std::vector<uint16_t> wb(nwb);
    if (e == cudaSuccess) e = cudaMemcpy(wb.data(), m->W1, nwb * 2, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return sk::cuda_status(e);
    for (size_t i = 0; i < nwb; ++i) {
      const uint32_t u = (uint32_t)wb[i] << 16;
      std::memcpy(&d[i], &u, 4);
    }
    sk::pack_host(*m, d.data(), used);
  }
  if (t) *t = m->adam_t;
  return SK_OK;
}

extern "C" int sk_mlp_forward(void* model, const uint8_t* slots, int B, float* logits) {
  Mlp* m = (Mlp*)model;
  if (!m || !slots || !logits || B < 1 || B > m->max_batch) return SK_EINVAL;
  cudaError_t e;
  const int Bp = sk::upload_states(*m, slots, B, nullptr, &e);
  if (e == cudaSuccess) e = sk::mlp_forward_dev(*m, Bp, nullptr);
  if (e == cudaSuccess)
    e = cudaMemcpy2D(logits, (size_t)m->NM * 4, m->Z, (size_t)m->NMp * 4, (size_t)m->NM * 4, B,
                     cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return sk::cuda_status(e);
  unsigned err = 0;
  e = cudaMemcpy(&err, m->tc_err, 4, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return sk::cuda_status(e);
  return err ? SK_ETIMEOUT : SK_OK;
}

extern "C" int sk_mlp_forward_bf16(void* model, const uint8_t* slots, int B, uint16_t* logits) {
  Mlp* m = (Mlp*)model;
  if (!m || !slots || !logits || B < 1 || B > m->max_batch) return SK_EINVAL;
  cudaError_t e;
  const int Bp = sk::upload_states(*m, slots, B, nullptr, &e);
  if (e == cudaSuccess) e = sk::mlp_forward_dev(*m, Bp, nullptr, true);
  if (e == cudaSuccess)
    e = cudaMemcpy2D(logits, (size_t)m->NM * 2, m->Z, (size_t)m->NMp * 2, (size_t)m->NM * 2, B,
                     cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return sk::cuda_status(e);
  unsigned err = 0;
  e = cudaMemcpy(&err, m->tc_err, 4, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return sk::cuda_status(e);
  return err ? SK_ETIMEOUT : SK_OK;
}

extern "C" int sk_mlp_loss_grad(void* model, const uint8_t* slots, int B, float beta_star,
                                float* loss, float* grads) {
  Mlp* m = (Mlp*)model;
  if (!m || !slots || B < 128 || B % 128 || B > m->max_batch) return SK_EINVAL;
  cudaError_t e;
  sk::upload_states(*m, slots, B, nullptr, &e);
  if (e == cudaSuccess) e = sk::mlp_forward_dev(*m, B, nullptr);
  if (e == cudaSuccess) e = sk::mlp_backward_dev(*m, B, beta_star, nullptr);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return sk::cuda_status(e);
  if (loss) cudaMemcpy(loss, m->loss, 4, cudaMemcpyDeviceToHost);
  if (grads) {
    std::vector<float> d(m->nparams);
    e = cudaMemcpy(d.data(), m->gW1, m->nparams * 4, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return sk::cuda_status(e);
    sk::pack_host(*m, d.data(), grads);
  }
  return SK_OK;
}

namespace sk {

int mlp_train_impl(Mlp& m, const uint8_t* states, uint64_t count, int epochs, int batch, float lr,
                   float beta_star, uint64_t seed, float* final_loss, double* ms_out) {
  if (!states || count < (uint64_t)batch || epochs < 1 || batch < 128 || batch % 128 ||
      batch > m.max_batch || !(lr > 0))
    return SK_EINVAL;
  const uint64_t steps = count / (uint64_t)batch;
  unsigned char* dstates = nullptr;
  unsigned* didx = nullptr;
  float* hloss = nullptr;
  float* dloss = nullptr;                 // per-step losses of an epoch, read back once
  cudaStream_t s = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaMalloc(&dstates, count * m.n);
  if (e == cudaSuccess) e = cudaMalloc(&didx, count * sizeof(unsigned));
  if (e == cudaSuccess) e = cudaHostAlloc(&hloss, steps * sizeof(float), cudaHostAllocDefault);
  if (e == cudaSuccess) e = cudaMalloc(&dloss, steps * sizeof(float));
  if (e == cudaSuccess) e = cudaMemcpy(dstates, states, count * m.n, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  std::vector<unsigned> perm(count);
  for (uint64_t i = 0; i < count; ++i) perm[i] = (unsigned)i;
  std::mt19937_64 rng(seed);
  const size_t nwb = (size_t)m.K1 * kHidden + (size_t)kHidden * kHidden + (size_t)kHidden * m.NMp;
  if (e == cudaSuccess) e = cudaEventRecord(e0, s);
  double last = 0.0;
  for (int ep = 0; ep < epochs && e == cudaSuccess; ++ep) {
    if (seed != SK_MLP_KEEP_ORDER) std::shuffle(perm.begin(), perm.end(), rng);
    e = cudaMemcpyAsync(didx, perm.data(), count * sizeof(unsigned), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);   // perm is reused next epoch
    if (e == cudaSuccess) e = cudaMemsetAsync(dloss, 0, steps * sizeof(float), s);
    for (uint64_t st = 0; st < steps && e == cudaSuccess; ++st) {
      const size_t tot = (size_t)batch * m.n;
      gather_slots_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(dstates, didx + st * batch,
                                                                       batch, m.n, m.slots);
      e = mlp_forward_dev(m, batch, s);
      if (e == cudaSuccess) e = mlp_backward_dev(m, batch, beta_star, s, dloss + st);
      if (e != cudaSuccess) break;
      m.adam_t += 1;
      const float c1 = 1.f - std::pow(0.9f, (float)m.adam_t);
      const float c2 = 1.f - std::pow(0.999f, (float)m.adam_t);
      adam_kernel<<<1024, 256, 0, s>>>(m.mW1, m.gW1, m.am, m.av, m.nparams, lr, 0.9f, 0.999f,
                                       1e-8f, c1, c2, m.W1, nwb);
      m.wt_dirty = 1;
      e = cudaGetLastError();
    }
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(hloss, dloss, steps * sizeof(float), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) {
      double acc = 0;
      for (uint64_t st = 0; st < steps; ++st) acc += hloss[st];
      last = acc / (double)steps;
    }
  }
  if (e == cudaSuccess) e = cudaEventRecord(e1, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  float ms = 0.f;
  if (e == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(dstates);
  cudaFree(didx);
  cudaFree(dloss);
  if (hloss) cudaFreeHost(hloss);
  if (s) cudaStreamDestroy(s);
  if (e != cudaSuccess) return cuda_status(e);
  if (final_loss) *final_loss = (float)last;
  if (ms_out) *ms_out = ms;
  return SK_OK;
}

}  // namespace sk

extern "C" int sk_mlp_train(void* model, const uint8_t* states, uint64_t count, int epochs,
                            int batch, float lr, float beta_star, uint64_t seed, float* final_loss,
                            double* ms) {
  Mlp* m = (Mlp*)model;
  if (!m) return SK_EINVAL;
  return sk::mlp_train_impl(*m, states, count, epochs, batch, lr, beta_star, seed, final_loss, ms);
}

// The tcgen05 forward records an error word when a bounded wait gives up.
extern "C" int sk_mlp_set_gemm(void* model, int use_tensor_memory_path) {
  Mlp* m = (Mlp*)model;
  if (!m) return SK_EINVAL;
  m->use_tc = use_tensor_memory_path ? 1 : 0;
  return SK_OK;
}

extern "C" int sk_mlp_check(void* model) {
  Mlp* m = (Mlp*)model;
  if (!m) return SK_EINVAL;
  unsigned err = 0;
  cudaError_t e = cudaMemcpy(&err, m->tc_err, 4, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return sk::cuda_status(e);
  return err ? SK_ETIMEOUT : SK_OK;
}
