// mlp.cu -- training and inference entry points of the candidate-proposal MLP.
//
// Training is done on the GPU by this file's own kernels: a small GEMM (BF16
// inputs on the tensor cores with mma.sync and FP32 accumulation, or plain
// FP32 FMA for reference gradients), bias+GELU, masked softmax cross-entropy,
// the GELU backward, bias-gradient reductions and an Adam update of FP32
// master weights.  The packed FP32 parameter layout used by the API is
//   W1[9][64], b1[64], W2[64][64], b2[64], W3[64][32], b3[32]   (6880 floats),
// W[k][n] mapping input k to output n.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <string>
#include <vector>

#include "g4n_internal.h"
#include "mlp_device.cuh"

using namespace g4n;
using namespace g4n::mlp;

namespace {

constexpr int kOffW1 = 0, kOffB1 = kOffW1 + kIn * kHid, kOffW2 = kOffB1 + kHid, kOffB2 = kOffW2 + kHid * kHid,
              kOffW3 = kOffB2 + kHid, kOffB3 = kOffW3 + kHid * kOut;

// ---------------------------------------------------------------- GEMM
// C[M x N] (+)= op(A)[M x K] op(B)[K x N], FP32 storage; A(m, k) = transA ? A[k * lda + m] : A[m * lda + k],
// B(k, n) = transB ? B[n * ldb + k] : B[k * ldb + n].  M, K multiples of 16, N a multiple of 8.
// One warp per 16 x 8 output tile and K chunk (blockIdx.z); chunks add into C atomically.

__device__ __forceinline__ float ldA(const float *A, int lda, bool tA, int m, int k) {
  return tA ? A[(int64_t)k * lda + m] : A[(int64_t)m * lda + k];
}
__device__ __forceinline__ float ldB(const float *B, int ldb, bool tB, int k, int n) {
  return tB ? B[(int64_t)n * ldb + k] : B[(int64_t)k * ldb + n];
}
__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<const uint32_t *>(&v);
}

__global__ void k_gemm_bf16(int M, int N, int K, int kchunk, const float *__restrict__ A, int lda, bool tA,
                            const float *__restrict__ B, int ldb, bool tB, float *__restrict__ C, int ldc) {
  const int lane = threadIdx.x & 31, g = lane >> 2, q = lane & 3;
  const int warp = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int tiles_n = N / 8;
  const int tm = warp / tiles_n, tn = warp % tiles_n;
  if (tm * 16 >= M) return;
  const int k0 = blockIdx.z * kchunk, k1 = min(K, k0 + kchunk);
  const int m0 = tm * 16, n0 = tn * 8;
  float d0 = 0.f, d1 = 0.f, d2 = 0.f, d3 = 0.f;
  for (int k = k0; k < k1; k += 16) {
    const int kc = k + 2 * q;
    const uint32_t a0 = pack_bf16(ldA(A, lda, tA, m0 + g, kc), ldA(A, lda, tA, m0 + g, kc + 1));
    const uint32_t a1 = pack_bf16(ldA(A, lda, tA, m0 + g + 8, kc), ldA(A, lda, tA, m0 + g + 8, kc + 1));
    const uint32_t a2 = pack_bf16(ldA(A, lda, tA, m0 + g, kc + 8), ldA(A, lda, tA, m0 + g, kc + 9));
    const uint32_t a3 = pack_bf16(ldA(A, lda, tA, m0 + g + 8, kc + 8), ldA(A, lda, tA, m0 + g + 8, kc + 9));
    const uint32_t b0 = pack_bf16(ldB(B, ldb, tB, kc, n0 + g), ldB(B, ldb, tB, kc + 1, n0 + g));
    const uint32_t b1 = pack_bf16(ldB(B, ldb, tB, kc + 8, n0 + g), ldB(B, ldb, tB, kc + 9, n0 + g));
    mma_bf16(d0, d1, d2, d3, a0, a1, a2, a3, b0, b1);
  }
  float *c0 = C + (int64_t)(m0 + g) * ldc + n0 + 2 * q;
  float *c1 = c0 + (int64_t)8 * ldc;
  atomicAdd(c0, d0);
  atomicAdd(c0 + 1, d1);
  atomicAdd(c1, d2);
  atomicAdd(c1 + 1, d3);
}

// FP32 reference GEMM: one thread per output element and K chunk.
__global__ void k_gemm_fp32(int M, int N, int K, int kchunk, const float *__restrict__ A, int lda, bool tA,
                            const float *__restrict__ B, int ldb, bool tB, float *__restrict__ C, int ldc) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= (int64_t)M * N) return;
  const int m = (int)(e / N), n = (int)(e % N);
  const int k0 = blockIdx.z * kchunk, k1 = min(K, k0 + kchunk);
  float acc = 0.f;
  for (int k = k0; k < k1; ++k) acc = fmaf(ldA(A, lda, tA, m, k), ldB(B, ldb, tB, k, n), acc);
  atomicAdd(&C[(int64_t)m * ldc + n], acc);
}

// ---------------------------------------------------------------- elementwise

__device__ __forceinline__ float gelu_grad(float x) {
  const float cdf = 0.5f * (1.0f + erff(x * 0.70710678118654752f));
  return cdf + x * 0.39894228040143268f * expf(-0.5f * x * x);
}

// Z += b (per column); H = GELU(Z).
__global__ void k_bias_gelu(int64_t rows, int cols, float *__restrict__ Z, const float *__restrict__ b,
                            float *__restrict__ H) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= rows * cols) return;
  const float z = Z[e] + b[e % cols];
  Z[e] = z;
  H[e] = gelu(z);
}

// Logits += b3; masked softmax over the first ncand[r] columns; loss (sum) and dZ3 = (p - onehot) / scale.
__global__ void k_softmax_ce(int64_t rows, float *__restrict__ Z3, const float *__restrict__ b3,
                             const int32_t *__restrict__ label, const int32_t *__restrict__ ncand,
                             const int64_t *__restrict__ idx, float inv_scale, float *__restrict__ dZ3,
                             double *__restrict__ loss) {
  const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (r >= rows) return;
  const int64_t src = idx ? idx[r] : r;
  const int n = max(1, min(kOut, ncand[src]));
  const int y = label[src];
  float *z = Z3 + r * kOut;
  float mx = -INFINITY;
  for (int c = 0; c < kOut; ++c) {
    z[c] += b3[c];
    if (c < n) mx = fmaxf(mx, z[c]);
  }
  float s = 0.f;
  for (int c = 0; c < n; ++c) s += expf(z[c] - mx);
  const float lse = mx + logf(s);
  atomicAdd(loss, (double)(lse - z[y]));
  for (int c = 0; c < kOut; ++c) {
    const float p = c < n ? expf(z[c] - lse) : 0.f;
    dZ3[r * kOut + c] = (p - (c == y ? 1.f : 0.f)) * inv_scale;
  }
}

__global__ void k_gelu_bwd(int64_t n, float *__restrict__ dH, const float *__restrict__ Z) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e < n) dH[e] *= gelu_grad(Z[e]);
}

__global__ void k_colsum(int64_t rows, int cols, const float *__restrict__ X, float *__restrict__ out) {
  const int c = blockIdx.x;
  float acc = 0.f;
  for (int64_t r = threadIdx.x; r < rows; r += blockDim.x) acc += X[r * cols + c];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  __shared__ float red[32];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0.f;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    out[c] = t;
  }
}

// Gather a minibatch of padded feature rows (16 columns, zeros beyond 9).
__global__ void k_gather(int64_t rows, const float *__restrict__ feat, const int64_t *__restrict__ idx,
                         float *__restrict__ X) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= rows * kInPad) return;
  const int64_t r = e / kInPad;
  const int k = (int)(e % kInPad);
  const int64_t src = idx ? idx[r] : r;
  X[e] = k < kIn ? feat[src * kIn + k] : 0.f;
}

// Minibatch index: a fixed-stride walk through a random rotation, a permutation of [0, n).
__global__ void k_batch_index(int64_t rows, int64_t n, int64_t start, int64_t stride, int64_t offset,
                              int64_t *__restrict__ idx) {
  const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (r < rows) idx[r] = (int64_t)((((uint64_t)(start + r) % (uint64_t)n) * (uint64_t)stride + (uint64_t)offset) % (uint64_t)n);
}

__global__ void k_add_double(double *dst, const double *src) { *dst += *src; }

__global__ void k_adam(int n, float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m,
                       float *__restrict__ v, float lr, float b1, float b2, float c1, float c2, float eps) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  m[i] = b1 * m[i] + (1.f - b1) * g[i];
  v[i] = b2 * v[i] + (1.f - b2) * g[i] * g[i];
  p[i] -= lr * (m[i] * c1) / (sqrtf(v[i] * c2) + eps);
}

// Shared-memory image (transposed BF16, padded) from the packed FP32 parameters.
__global__ void k_pack_image(const float *__restrict__ P, SmemWeights *__restrict__ S) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  for (int e = t; e < kHid * kSIn; e += gridDim.x * blockDim.x) {
    const int n = e / kSIn, k = e % kSIn;
    S->w1t[e] = __float2bfloat16_rn(k < kIn ? P[kOffW1 + k * kHid + n] : 0.f);
  }
  for (int e = t; e < kHid * kSHid; e += gridDim.x * blockDim.x) {
    const int n = e / kSHid, k = e % kSHid;
    S->w2t[e] = __float2bfloat16_rn(k < kHid ? P[kOffW2 + k * kHid + n] : 0.f);
  }
  for (int e = t; e < kOut * kSHid; e += gridDim.x * blockDim.x) {
    const int n = e / kSHid, k = e % kSHid;
    S->w3t[e] = __float2bfloat16_rn(k < kHid ? P[kOffW3 + k * kOut + n] : 0.f);
  }
  for (int e = t; e < kHid; e += gridDim.x * blockDim.x) {
    S->b1[e] = P[kOffB1 + e];
    S->b2[e] = P[kOffB2 + e];
  }
  for (int e = t; e < kOut; e += gridDim.x * blockDim.x) S->b3[e] = P[kOffB3 + e];
}

// Padded copy of W1 (16 x 64; rows 9..15 zero) for the training GEMMs.
__global__ void k_pad_w1(const float *__restrict__ P, float *__restrict__ W1p) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e < kInPad * kHid) W1p[e] = (e / kHid) < kIn ? P[kOffW1 + e] : 0.f;
}

// Inference through the fused device code path: one warp per 32 feature rows.
__global__ void __launch_bounds__(128) k_predict(int64_t n, const float *__restrict__ feat,
                                                 const SmemWeights *__restrict__ gw, float *__restrict__ logits) {
  extern __shared__ __align__(16) unsigned char smem[];
  SmemWeights &sw = *reinterpret_cast<SmemWeights *>(smem);
  load_weights(sw, gw);
  __syncthreads();
  SmemWarp &W = reinterpret_cast<SmemWarp *>(smem + sizeof(SmemWeights))[threadIdx.x >> 5];
  const int lane = threadIdx.x & 31;
  for (int64_t base = (blockIdx.x * (int64_t)blockDim.x) + (threadIdx.x & ~31); base < n;
       base += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = base + lane;
    float f[kIn];
    for (int k = 0; k < kIn; ++k) f[k] = r < n ? feat[r * kIn + k] : 0.f;
    put_features(W, f);
    forward_warp(sw, W);
    if (r < n)
      for (int c = 0; c < kOut; ++c) logits[r * kOut + c] = W.logits[lane * kSOut + c];
    __syncwarp();
  }
}

struct MlpState {
  float *P = nullptr, *G = nullptr, *M = nullptr, *V = nullptr;  // kNParams each
  SmemWeights *img = nullptr;
  float *W1p = nullptr;
  int64_t step = 0;
  // training scratch for `cap` rows
  int64_t cap = 0;
  float *X = nullptr, *Z1 = nullptr, *H1 = nullptr, *Z2 = nullptr, *H2 = nullptr, *Z3 = nullptr, *dZ3 = nullptr,
        *dH2 = nullptr, *dH1 = nullptr, *dW1p = nullptr;
  int64_t *idx = nullptr;
  double *loss = nullptr;
};

MlpState *state(g4n_ctx *ctx) { return reinterpret_cast<MlpState *>(ctx->mlp); }

void free_scratch(MlpState *s) {
  cudaFree(s->X); cudaFree(s->Z1); cudaFree(s->H1); cudaFree(s->Z2); cudaFree(s->H2); cudaFree(s->Z3);
  cudaFree(s->dZ3); cudaFree(s->dH2); cudaFree(s->dH1); cudaFree(s->dW1p); cudaFree(s->idx); cudaFree(s->loss);
  s->X = s->Z1 = s->H1 = s->Z2 = s->H2 = s->Z3 = s->dZ3 = s->dH2 = s->dH1 = s->dW1p = nullptr;
  s->idx = nullptr;
  s->loss = nullptr;
  s->cap = 0;
}

int ensure_scratch(g4n_ctx *ctx, MlpState *s, int64_t rows) {
  if (s->cap >= rows) return G4N_OK;
  cudaDeviceSynchronize();
  free_scratch(s);
  bool ok = cudaMalloc(&s->X, rows * kInPad * 4) == cudaSuccess && cudaMalloc(&s->Z1, rows * kHid * 4) == cudaSuccess &&
            cudaMalloc(&s->H1, rows * kHid * 4) == cudaSuccess && cudaMalloc(&s->Z2, rows * kHid * 4) == cudaSuccess &&
            cudaMalloc(&s->H2, rows * kHid * 4) == cudaSuccess && cudaMalloc(&s->Z3, rows * kOut * 4) == cudaSuccess &&
            cudaMalloc(&s->dZ3, rows * kOut * 4) == cudaSuccess && cudaMalloc(&s->dH2, rows * kHid * 4) == cudaSuccess &&
            cudaMalloc(&s->dH1, rows * kHid * 4) == cudaSuccess && cudaMalloc(&s->dW1p, kInPad * kHid * 4) == cudaSuccess &&
            cudaMalloc(&s->idx, rows * 8) == cudaSuccess && cudaMalloc(&s->loss, 8) == cudaSuccess;
  if (!ok) {
    free_scratch(s);
    return g4n_fail(ctx, G4N_ERR_OOM, "mlp: scratch allocation failed");
  }
  s->cap = rows;
  return G4N_OK;
}

void gemm(bool bf16, int M, int N, int K, const float *A, int lda, bool tA, const float *B, int ldb, bool tB, float *C,
          int ldc, cudaStream_t st) {
  const int ksplit = std::max(1, std::min(256, K / 256));
  const int kchunk = ((K + ksplit - 1) / ksplit + 15) / 16 * 16;
  const int nz = (K + kchunk - 1) / kchunk;
  if (bf16) {
    const int warps = (M / 16) * (N / 8);
    dim3 grid((warps + 3) / 4, 1, nz);
    k_gemm_bf16<<<grid, 128, 0, st>>>(M, N, K, kchunk, A, lda, tA, B, ldb, tB, C, ldc);
  } else {
    dim3 grid((int)(((int64_t)M * N + 127) / 128), 1, nz);
    k_gemm_fp32<<<grid, 128, 0, st>>>(M, N, K, kchunk, A, lda, tA, B, ldb, tB, C, ldc);
  }
}

inline int blocks(int64_t n, int b = 256) { return (int)std::max<int64_t>(1, (n + b - 1) / b); }

// Forward + backward over `rows` samples (rows a multiple of 16; the caller pads with
// ncand = 1, label = 0 rows of zero weight via inv_scale).  Gradients into s->G.
void forward_backward(MlpState *s, bool bf16, int64_t rows, const float *feat, const int32_t *label,
                      const int32_t *ncand, const int64_t *idx, float inv_scale, cudaStream_t st) {
  const int R = (int)rows;
  float *P = s->P, *G = s->G;
  cudaMemsetAsync(s->loss, 0, 8, st);
  k_gather<<<blocks(rows * kInPad), 256, 0, st>>>(rows, feat, idx, s->X);
  k_pad_w1<<<blocks(kInPad * kHid), 256, 0, st>>>(P, s->W1p);
  cudaMemsetAsync(s->Z1, 0, rows * kHid * 4, st);
  gemm(bf16, R, kHid, kInPad, s->X, kInPad, false, s->W1p, kHid, false, s->Z1, kHid, st);
  k_bias_gelu<<<blocks(rows * kHid), 256, 0, st>>>(rows, kHid, s->Z1, P + kOffB1, s->H1);
  cudaMemsetAsync(s->Z2, 0, rows * kHid * 4, st);
  gemm(bf16, R, kHid, kHid, s->H1, kHid, false, P + kOffW2, kHid, false, s->Z2, kHid, st);
  k_bias_gelu<<<blocks(rows * kHid), 256, 0, st>>>(rows, kHid, s->Z2, P + kOffB2, s->H2);
  cudaMemsetAsync(s->Z3, 0, rows * kOut * 4, st);
  gemm(bf16, R, kOut, kHid, s->H2, kHid, false, P + kOffW3, kOut, false, s->Z3, kOut, st);
  k_softmax_ce<<<blocks(rows), 256, 0, st>>>(rows, s->Z3, P + kOffB3, label, ncand, idx, inv_scale, s->dZ3, s->loss);
  // backward
  cudaMemsetAsync(G, 0, kNParams * 4, st);
  gemm(bf16, kHid, kOut, R, s->H2, kHid, true, s->dZ3, kOut, false, G + kOffW3, kOut, st);    // dW3 = H2^T dZ3
  k_colsum<<<kOut, 256, 0, st>>>(rows, kOut, s->dZ3, G + kOffB3);
  cudaMemsetAsync(s->dH2, 0, rows * kHid * 4, st);
  gemm(bf16, R, kHid, kOut, s->dZ3, kOut, false, P + kOffW3, kOut, true, s->dH2, kHid, st);   // dH2 = dZ3 W3^T
  k_gelu_bwd<<<blocks(rows * kHid), 256, 0, st>>>(rows * kHid, s->dH2, s->Z2);
  gemm(bf16, kHid, kHid, R, s->H1, kHid, true, s->dH2, kHid, false, G + kOffW2, kHid, st);    // dW2 = H1^T dZ2
  k_colsum<<<kHid, 256, 0, st>>>(rows, kHid, s->dH2, G + kOffB2);
  cudaMemsetAsync(s->dH1, 0, rows * kHid * 4, st);
  gemm(bf16, R, kHid, kHid, s->dH2, kHid, false, P + kOffW2, kHid, true, s->dH1, kHid, st);   // dH1 = dZ2 W2^T
  k_gelu_bwd<<<blocks(rows * kHid), 256, 0, st>>>(rows * kHid, s->dH1, s->Z1);
  cudaMemsetAsync(s->dW1p, 0, kInPad * kHid * 4, st);
  gemm(bf16, kInPad, kHid, R, s->X, kInPad, true, s->dH1, kHid, false, s->dW1p, kHid, st);   // dW1 = X^T dZ1
  cudaMemcpyAsync(G + kOffW1, s->dW1p, kIn * kHid * 4, cudaMemcpyDeviceToDevice, st);
  k_colsum<<<kHid, 256, 0, st>>>(rows, kHid, s->dH1, G + kOffB1);
}

int check_data(g4n_ctx *ctx, int64_t n, const void *feat, const void *label, const void *ncand) {
  if (!ctx) return G4N_ERR_ARG;
  if (ctx->device < 0) return g4n_fail(ctx, G4N_ERR_STATE, "host-only context: no device work");
  if (!state(ctx)) return g4n_fail(ctx, G4N_ERR_STATE, "mlp: no parameters loaded (g4n_mlp_load)");
  if (n < 1 || !feat || !label || !ncand) return g4n_fail(ctx, G4N_ERR_ARG, "mlp: empty or null training data");
  return G4N_OK;
}

}  // namespace

// Device image of the loaded weights (for the fused inference in the transport kernel); null if none.
const SmemWeights *g4n_mlp_image(g4n_ctx *ctx) {
  MlpState *s = state(ctx);
  return s ? s->img : nullptr;
}

void g4n_mlp_free(g4n_ctx *ctx) {
  MlpState *s = state(ctx);
  if (!s) return;
  free_scratch(s);
  cudaFree(s->P); cudaFree(s->G); cudaFree(s->M); cudaFree(s->V); cudaFree(s->img); cudaFree(s->W1p);
  delete s;
  ctx->mlp = nullptr;
}

extern "C" {

int g4n_mlp_load(g4n_ctx *ctx, const float *params) {
  if (!ctx || !params) return g4n_fail(ctx, G4N_ERR_ARG, "mlp_load: null argument");
  if (ctx->device < 0) return g4n_fail(ctx, G4N_ERR_STATE, "host-only context: no device work");
  for (int i = 0; i < kNParams; ++i)
    if (!std::isfinite(params[i])) return g4n_fail(ctx, G4N_ERR_ARG, "mlp_load: non-finite parameter");
  cudaSetDevice(ctx->device);
  MlpState *s = state(ctx);
  if (!s) {
    s = new MlpState();
    bool ok = cudaMalloc(&s->P, kNParams * 4) == cudaSuccess && cudaMalloc(&s->G, kNParams * 4) == cudaSuccess &&
              cudaMalloc(&s->M, kNParams * 4) == cudaSuccess && cudaMalloc(&s->V, kNParams * 4) == cudaSuccess &&
              cudaMalloc(&s->img, sizeof(SmemWeights)) == cudaSuccess &&
              cudaMalloc(&s->W1p, kInPad * kHid * 4) == cudaSuccess;
    ctx->mlp = s;
    if (!ok) {
      g4n_mlp_free(ctx);
      return g4n_fail(ctx, G4N_ERR_OOM, "mlp_load: allocation failed");
    }
  }
  if (cudaMemcpy(s->P, params, kNParams * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemset(s->M, 0, kNParams * 4) != cudaSuccess || cudaMemset(s->V, 0, kNParams * 4) != cudaSuccess)
    return g4n_fail(ctx, G4N_ERR_CUDA, "mlp_load: upload failed");
  s->step = 0;
  k_pack_image<<<8, 256>>>(s->P, s->img);
  if (cudaDeviceSynchronize() != cudaSuccess) return g4n_fail(ctx, G4N_ERR_CUDA, "mlp_load: packing failed");
  return G4N_OK;
}

int g4n_mlp_get(g4n_ctx *ctx, float *params) {
  if (!ctx || !params) return g4n_fail(ctx, G4N_ERR_ARG, "mlp_get: null argument");
  MlpState *s = state(ctx);
  if (!s) return g4n_fail(ctx, G4N_ERR_STATE, "mlp_get: no parameters loaded");
  cudaSetDevice(ctx->device);
  if (cudaMemcpy(params, s->P, kNParams * 4, cudaMemcpyDeviceToHost) != cudaSuccess)
    return g4n_fail(ctx, G4N_ERR_CUDA, "mlp_get: copy failed");
  return G4N_OK;
}

int g4n_mlp_predict(g4n_ctx *ctx, int64_t n, const float *feat, float *out_logits, g4n_stream stream) {
  if (!ctx) return G4N_ERR_ARG;
  if (!state(ctx)) return g4n_fail(ctx, G4N_ERR_STATE, "mlp_predict: no parameters loaded");
  if (n < 0) return g4n_fail(ctx, G4N_ERR_ARG, "mlp_predict: n < 0");
  if (n == 0) return G4N_OK;
  if (!feat || !out_logits) return g4n_fail(ctx, G4N_ERR_ARG, "mlp_predict: null array");
  cudaSetDevice(ctx->device);
  const int grid = (int)std::min<int64_t>((n + 127) / 128, (int64_t)ctx->sm_count * 8);
  const size_t smem = sizeof(SmemWeights) + 4 * sizeof(SmemWarp);
  cudaFuncSetAttribute(k_predict, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  k_predict<<<grid, 128, smem, (cudaStream_t)stream>>>(n, feat, state(ctx)->img, out_logits);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return g4n_fail(ctx, G4N_ERR_CUDA, std::string("mlp_predict launch: ") + cudaGetErrorString(e));
  return G4N_OK;
}

int g4n_mlp_grad(g4n_ctx *ctx, int64_t n, const float *feat, const int32_t *label, const int32_t *ncand,
                 int32_t precision, float *out_grads, double *out_loss) {
  int rc = check_data(ctx, n, feat, label, ncand);
  if (rc) return rc;
  if (!out_grads || !out_loss) return g4n_fail(ctx, G4N_ERR_ARG, "mlp_grad: null output");
  if (n % 16) return g4n_fail(ctx, G4N_ERR_ARG, "mlp_grad: n must be a multiple of 16");
  cudaSetDevice(ctx->device);
  MlpState *s = state(ctx);
  if ((rc = ensure_scratch(ctx, s, n))) return rc;
  forward_backward(s, precision == 0, n, feat, label, ncand, nullptr, 1.0f / (float)n, 0);
  double loss = 0.0;
  if (cudaMemcpy(out_grads, s->G, kNParams * 4, cudaMemcpyDeviceToHost) != cudaSuccess ||
      cudaMemcpy(&loss, s->loss, 8, cudaMemcpyDeviceToHost) != cudaSuccess)
    return g4n_fail(ctx, G4N_ERR_CUDA, "mlp_grad: failed");
  *out_loss = loss / (double)n;
  return G4N_OK;
}

int g4n_mlp_train(g4n_ctx *ctx, int64_t n, const float *feat, const int32_t *label, const int32_t *ncand,
                  int32_t epochs, int32_t batch, float lr, uint64_t seed, float *out_loss, g4n_stream stream) {
  int rc = check_data(ctx, n, feat, label, ncand);
  if (rc) return rc;
  if (epochs < 1 || batch < 16 || batch % 16 || !(lr > 0.f)) return g4n_fail(ctx, G4N_ERR_ARG, "mlp_train: bad settings");
  if (n < batch) return g4n_fail(ctx, G4N_ERR_ARG, "mlp_train: fewer samples than one batch");
  cudaSetDevice(ctx->device);
  cudaStream_t st = (cudaStream_t)stream;
  MlpState *s = state(ctx);
  if ((rc = ensure_scratch(ctx, s, batch))) return rc;
  const int64_t nb = n / batch;
  double *d_epoch = nullptr;
  if (cudaMalloc(&d_epoch, 8) != cudaSuccess) return g4n_fail(ctx, G4N_ERR_OOM, "mlp_train: allocation failed");
  for (int ep = 0; ep < epochs; ++ep) {
    // a random stride coprime with n and a random offset: a permutation of the samples per epoch
    uint64_t h = seed * 0x9E3779B97F4A7C15ull + (uint64_t)ep * 0xD1B54A32D192ED03ull + 1;
    h ^= h >> 31;
    h *= 0xBF58476D1CE4E5B9ull;
    h ^= h >> 27;
    uint64_t stride = (h % (uint64_t)n) | 1;
    while (std::gcd(stride, (uint64_t)n) != 1) stride += 2;
    const uint64_t offset = (h >> 17) % (uint64_t)n;
    cudaMemsetAsync(d_epoch, 0, 8, st);
    for (int64_t b = 0; b < nb; ++b) {
      k_batch_index<<<blocks(batch), 256, 0, st>>>(batch, n, b * batch, (int64_t)stride, (int64_t)offset, s->idx);
      forward_backward(s, true, batch, feat, label, ncand, s->idx, 1.0f / (float)batch, st);
      ++s->step;
      const float c1 = 1.0f / (1.0f - std::pow(0.9f, (float)s->step));
      const float c2 = 1.0f / (1.0f - std::pow(0.999f, (float)s->step));
      k_adam<<<blocks(kNParams), 256, 0, st>>>(kNParams, s->P, s->G, s->M, s->V, lr, 0.9f, 0.999f, c1, c2, 1e-8f);
      k_add_double<<<1, 1, 0, st>>>(d_epoch, s->loss);  // epoch loss accumulates on the device
    }
    k_pack_image<<<8, 256, 0, st>>>(s->P, s->img);
    double tot = 0.0;
    cudaMemcpyAsync(&tot, d_epoch, 8, cudaMemcpyDeviceToHost, st);
    cudaStreamSynchronize(st);
    if (out_loss) out_loss[ep] = (float)(tot / ((double)nb * batch));
  }
  cudaFree(d_epoch);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return g4n_fail(ctx, G4N_ERR_CUDA, std::string("mlp_train: ") + cudaGetErrorString(e));
  return G4N_OK;
}

}  // extern "C"
