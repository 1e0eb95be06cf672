// sk_mlp.cuh -- the move-proposal network's state and the helpers shared by
// its training code (sk_mlp.cu) and the learned tempering chains
// (sk_pt_learned.cu).
#pragma once
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <utility>

#include "sk_pt.cuh"

namespace sk {

constexpr int kHidden = 256;

struct Mlp {
  int variant, n, delta, bins;
  int K1;                 // input width, padded to 128 (the row stride of X, the rows of W1)
  int K1f;                // the forward's input width: 2n rounded up to 64 (the columns
                          // of X beyond 2n are 0, so the first layer's sum stops there)
  int NM, NMp;            // moves, padded to 256
  int max_batch;
  int off[kPtMaxN + 2];   // move offsets per pair k (1-based), off[n+1] = NM
  // parameters: bf16 copies used by the GEMMs, fp32 masters, Adam moments
  __nv_bfloat16 *W1, *W2, *W3;
  float *b1, *b2, *b3;
  float *mW1, *mW2, *mW3;                    // fp32 master weights
  float *gW1, *gW2, *gW3, *gb1, *gb2, *gb3;  // gradients
  float *am, *av;                            // Adam moments over all parameters
  int adam_t;
  size_t nparams;                            // W1 | W2 | W3 | b1 | b2 | b3 (fp32 view)
  // activations for max_batch states
  unsigned char* slots;
  __nv_bfloat16 *X, *H1, *H2, *dZ, *dH1, *dH2;
  // K-major (transposed) bf16 weights for the tcgen05 forward: [out][in]
  __nv_bfloat16 *W1t, *W2t, *W3t;
  int use_tc;                                // 1: forward on tcgen05 (default)
  int wt_dirty;                              // transposed copies need a refresh
  unsigned* tc_err;                          // error word of the tcgen05 GEMM
  // TMA descriptors of the tcgen05 forward (128-byte swizzle): operands A =
  // X, H1, H2 ([max_batch][K], boxes [128][64]) and B = W1t, W2t, W3t ([N][K],
  // boxes [256][64]); results C = H1, H2 (bf16, boxes [32][64]) and Z (fp32,
  // boxes [32][32])
  CUtensorMap tmA[3], tmB[3], tmC[3];
  CUtensorMap tmZb;                          // Z's memory as bf16 [max_batch][NMp] (learned chains)
  // tcgen05 backward: A = dZ, dH2; B = W3, W2 (stored [in][out] = [N][K]);
  // C = dH2, dH1 (bf16, masked by H2 > 0, H1 > 0)
  CUtensorMap tmBA[2], tmBB[2], tmBC[2];
  void* bwd_ws;                              // K-major operand copies + K-split partials
  size_t bwd_bytes;
  cudaStream_t side;                         // the backward's weight-gradient stream
  cudaEvent_t ev[4];                         // its fork and join points
  float* Z;
  float* loss;                               // [1]
  float* colpart;                            // [max_batch / 128][NMp]: bias-gradient partials
  void* block;                               // one allocation holding all of the above
};

struct MoveTable {
  int n, delta, NM;
  int off[kPtMaxN + 2];   // off[k], k = 1..n+1: first move of pair k
};

// dE of moving pair k (start s_k) to start s (d = k + delta), from the bin
// occupancies occ of the configuration: taking the pair out empties the bins
// it was alone in; putting it back fills the empty bins it lands on.
template <class Occ>
__device__ __forceinline__ int move_delta_e(const Occ* occ, int sk, int d, int s) {
  const int out = (occ[sk] == 1) + (occ[sk + d] == 1);
  const int o1 = occ[s] - (s == sk) - (s == sk + d);
  const int o2 = occ[s + d] - (s + d == sk) - (s + d == sk + d);
  return out - (o1 == 0) - (o2 == 0);
}

__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Forward pass for B (multiple of 128) states whose start slots are in
// m.slots: X, H1, H2 (bf16) and the logits Z (fp32, [B][NMp]; with
// logits_bf16, bf16 [B][NMp] in the first half of Z's memory).  With
// inputs_ready the caller has already written the input rows X.  before_l2:
// an event the stream waits for between the first and the second layer.
// dependent: the second and third layers are launched as programmatic
// dependents of the layer before (they may set up while it finishes; only
// while the weights stay unchanged, as in a tempering run).
cudaError_t mlp_forward_dev(Mlp& m, int B, cudaStream_t s, bool logits_bf16 = false,
                            bool inputs_ready = false, cudaEvent_t before_l2 = nullptr,
                            bool dependent = false);

// Launch of kernel k as a programmatic dependent of the previous kernel of
// stream s (it must execute griddepcontrol.wait before it reads what that
// kernel writes).
template <class... KArgs, class... Args>
cudaError_t launch_dependent(void (*k)(KArgs...), int grid, int block, size_t smem,
                             cudaStream_t s, Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3((unsigned)block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k, std::forward<Args>(args)...);
}
MoveTable move_table(const Mlp& m);

}  // namespace sk
