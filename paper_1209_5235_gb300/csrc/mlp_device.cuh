// mlp_device.cuh -- the candidate-proposal MLP on the tensor cores (sm_103a).
//
// Network: 9 -> 64 -> 64 -> 32, GELU (erf form) after the two hidden layers,
// softmax over the first n_cand of the 32 outputs.  Inputs: the point in the
// voxel node's own coordinates (3, each in [-1, 1]), the direction (3), log E
// scaled to ~[0, 1], n_cand / 32 and 1.  Output: the list slot of the daughter
// the ray most likely enters first.  The proposal only orders the exact
// candidate tests; it never changes a result.
//
// Inference is warp-level: the 32 lanes' feature rows form a 32 x 16 BF16 tile
// (K padded from 9), and each layer is a few mma.sync m16n8k16 (BF16 inputs,
// FP32 accumulation) against BF16 weights held in shared memory.  A warp-level
// MMA is the right tensor-core instruction here: the persistent transport
// kernel runs its warps independently, so CTA-wide tcgen05 tiles (128 rows,
// TMEM, one issuing thread per CTA) cannot be formed inside it.
#pragma once

#include <cuda_bf16.h>

#include <cstdint>

namespace g4n {
namespace mlp {

constexpr int kIn = 9, kInPad = 16, kHid = 64, kOut = 32;
// padded row strides (bf16 elements) to keep shared-memory fragment loads conflict free
constexpr int kSIn = 24, kSHid = 72, kSOut = 33;
constexpr int kNParams = kIn * kHid + kHid + kHid * kHid + kHid + kHid * kOut + kOut;  // 6880

// Shared-memory image of the weights: transposed (n-major) BF16 with padded rows, FP32 biases.
struct SmemWeights {
  __nv_bfloat16 w1t[kHid * kSIn];   // [n][k], k < 16 (rows 9..15 zero)
  __nv_bfloat16 w2t[kHid * kSHid];  // [n][k], k < 64
  __nv_bfloat16 w3t[kOut * kSHid];  // [n][k], k < 64
  float b1[kHid], b2[kHid], b3[kOut];
};

// Per-warp scratch: input tile, two hidden tiles; the FP32 logits reuse the first
// hidden tile, which layer 3 no longer reads.
struct SmemWarp {
  __nv_bfloat16 x[32 * kSIn];
  union {
    __nv_bfloat16 h1[32 * kSHid];
    float logits[32 * kSOut];
  };
  __nv_bfloat16 h2[32 * kSHid];
};
static_assert(sizeof(float) * 32 * kSOut <= sizeof(__nv_bfloat16) * 32 * kSHid, "logits must fit in h1");

__device__ __forceinline__ uint32_t ld_pair(const __nv_bfloat16 *p) { return *reinterpret_cast<const uint32_t *>(p); }

__device__ __forceinline__ void mma_bf16(float &d0, float &d1, float &d2, float &d3, uint32_t a0, uint32_t a1,
                                         uint32_t a2, uint32_t a3, uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d0), "+f"(d1), "+f"(d2), "+f"(d3)
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

__device__ __forceinline__ float gelu(float x) { return 0.5f * x * (1.0f + erff(x * 0.70710678118654752f)); }

// One layer for the warp's 32 rows: out[32][N] = act(in[32][K] W + b).  `in` has row stride
// SA, wt is [N][K] with row stride SB.  act: GELU then BF16 into `hout` (stride kSHid), or
// (logits) FP32 into `fout` (stride kSOut).
template <int K, int N, int SA, int SB, bool LOGITS>
__device__ __forceinline__ void layer(const __nv_bfloat16 *in, const __nv_bfloat16 *wt, const float *bias,
                                      __nv_bfloat16 *hout, float *fout) {
  const int lane = threadIdx.x & 31, g = lane >> 2, q = lane & 3;
#pragma unroll
  for (int mt = 0; mt < 2; ++mt) {
    const __nv_bfloat16 *a_lo = in + (mt * 16 + g) * SA + 2 * q;
    const __nv_bfloat16 *a_hi = a_lo + 8 * SA;
#pragma unroll
    for (int nt = 0; nt < N / 8; ++nt) {
      const int col = nt * 8 + 2 * q;
      float d0 = bias[col], d1 = bias[col + 1], d2 = d0, d3 = d1;
      const __nv_bfloat16 *bp = wt + (nt * 8 + g) * SB + 2 * q;
#pragma unroll
      for (int kt = 0; kt < K / 16; ++kt) {
        mma_bf16(d0, d1, d2, d3, ld_pair(a_lo + kt * 16), ld_pair(a_hi + kt * 16), ld_pair(a_lo + kt * 16 + 8),
                 ld_pair(a_hi + kt * 16 + 8), ld_pair(bp + kt * 16), ld_pair(bp + kt * 16 + 8));
      }
      const int r0 = mt * 16 + g, r1 = r0 + 8;
      if (LOGITS) {
        fout[r0 * kSOut + col] = d0;
        fout[r0 * kSOut + col + 1] = d1;
        fout[r1 * kSOut + col] = d2;
        fout[r1 * kSOut + col + 1] = d3;
      } else {
        *reinterpret_cast<__nv_bfloat162 *>(hout + r0 * kSHid + col) = __floats2bfloat162_rn(gelu(d0), gelu(d1));
        *reinterpret_cast<__nv_bfloat162 *>(hout + r1 * kSHid + col) = __floats2bfloat162_rn(gelu(d2), gelu(d3));
      }
    }
  }
}

// Warp-collective forward pass.  Every lane writes its feature row (zeros if it has none)
// before the call; afterwards lane i's logits are in W.logits[i * kSOut ...].
__device__ __forceinline__ void forward_warp(const SmemWeights &Wt, SmemWarp &W) {
  __syncwarp();
  layer<kInPad, kHid, kSIn, kSIn, false>(W.x, Wt.w1t, Wt.b1, W.h1, nullptr);
  __syncwarp();
  layer<kHid, kHid, kSHid, kSHid, false>(W.h1, Wt.w2t, Wt.b2, W.h2, nullptr);
  __syncwarp();
  layer<kHid, kOut, kSHid, kSHid, true>(W.h2, Wt.w3t, Wt.b3, nullptr, W.logits);
  __syncwarp();
}

// Lane's feature row into the warp's input tile.
__device__ __forceinline__ void put_features(SmemWarp &W, const float *f) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int k = 0; k < kInPad; k += 2)
    *reinterpret_cast<__nv_bfloat162 *>(W.x + lane * kSIn + k) =
        __floats2bfloat162_rn(k < kIn ? f[k] : 0.f, k + 1 < kIn ? f[k + 1] : 0.f);
}

// Masked argmax of the lane's logits over slots [0, n) (first slot wins ties).
__device__ __forceinline__ int argmax_row(const SmemWarp &W, int n) {
  const int lane = threadIdx.x & 31;
  int best = 0;
  float bv = W.logits[lane * kSOut];
  for (int s = 1; s < n; ++s) {
    const float x = W.logits[lane * kSOut + s];
    if (x > bv) {
      bv = x;
      best = s;
    }
  }
  return best;
}

// Fill the shared-memory weight image from the device copy (block-collective).
__device__ __forceinline__ void load_weights(SmemWeights &S, const SmemWeights *g) {
  const int n = sizeof(SmemWeights) / 16;
  const uint4 *src = reinterpret_cast<const uint4 *>(g);
  uint4 *dst = reinterpret_cast<uint4 *>(&S);
  for (int i = threadIdx.x; i < n; i += blockDim.x) dst[i] = src[i];
}

}  // namespace mlp
}  // namespace g4n
