// Cut-scoring MLP (64 -> 256 -> 256 -> 1): forward, backward and Adam.
//
// Not part of the paper: a small network that predicts the log2
// reconstruction cost of a candidate wire cut from structural features.
// Weights are kept as FP32 masters (updated by Adam) and BF16 copies (read
// by the forward and backward passes); activations and every accumulation
// are FP32.  Layers: z1 = x W1 + b1, h1 = relu(z1), z2 = h1 W2 + b2,
// h2 = relu(z2), y = h2 W3 + b3; loss = mean (y - t)^2.  W_l is [in][out].
#include "internal.cuh"
#include "../../include/cutqc_mlp.h"

#include <cuda_bf16.h>

namespace cutqc {
namespace {

constexpr int D0 = 64, D1 = 256, D2 = 256, D3 = 1;
constexpr int64_t OFF_W1 = 0, OFF_B1 = OFF_W1 + D0 * D1, OFF_W2 = OFF_B1 + D1, OFF_B2 = OFF_W2 + D1 * D2,
                  OFF_W3 = OFF_B2 + D2, OFF_B3 = OFF_W3 + D2 * D3, NPARAM = OFF_B3 + D3;

// C[M][N] = op(A)[M][K] * op(B)[K][N] (+ bias[N]) (relu optional), FP32
// accumulate.  A is FP32 [M][K] (trans_a: stored [K][M]); B is BF16 [K][N]
// (trans_b: stored [N][K]) or FP32 when b32 != null.  64 x 64 tiles, 256
// threads, 4 x 4 outputs each.
template <bool TA, bool TB>
__global__ void __launch_bounds__(256)
dense_kernel(const float* __restrict__ A, const __nv_bfloat16* __restrict__ Bh, const float* __restrict__ B32,
             const float* __restrict__ bias, float* __restrict__ C, float* __restrict__ Cpre, int M, int N, int K,
             int relu, int accumulate) {
  __shared__ float As[16][64 + 1];
  __shared__ float Bs[16][64 + 1];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int m0 = blockIdx.y * 64, n0 = blockIdx.x * 64;
  float acc[4][4] = {};
  for (int k0 = 0; k0 < K; k0 += 16) {
    for (int i = threadIdx.x; i < 16 * 64; i += 256) {
      const int kk = i / 64, mm = i % 64;
      const int m = m0 + mm, k = k0 + kk;
      float a = 0.f;
      if (m < M && k < K) a = TA ? A[(int64_t)k * M + m] : A[(int64_t)m * K + k];
      As[kk][mm] = a;
      const int n = n0 + mm;
      float b = 0.f;
      if (n < N && k < K) {
        const int64_t idx = TB ? (int64_t)n * K + k : (int64_t)k * N + n;
        b = B32 ? B32[idx] : __bfloat162float(Bh[idx]);
      }
      Bs[kk][mm] = b;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
      float av[4], bv[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) av[i] = As[kk][ty * 4 + i];
#pragma unroll
      for (int j = 0; j < 4; ++j) bv[j] = Bs[kk][tx * 4 + j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int m = m0 + ty * 4 + i;
    if (m >= M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int n = n0 + tx * 4 + j;
      if (n >= N) continue;
      float v = acc[i][j] + (bias ? bias[n] : 0.f);
      if (accumulate) v += C[(int64_t)m * N + n];
      if (Cpre) Cpre[(int64_t)m * N + n] = v;
      C[(int64_t)m * N + n] = relu ? fmaxf(v, 0.f) : v;
    }
  }
}

// column sums: out[n] = sum_m X[m][n]
__global__ void colsum_kernel(const float* __restrict__ X, int M, int N, float* __restrict__ out) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  float s = 0.f;
  for (int m = 0; m < M; ++m) s += X[(int64_t)m * N + n];
  out[n] = s;
}

// dy = 2/B (y - t); loss = mean (y - t)^2 (FP64 accumulation, one block)
__global__ void loss_kernel(const float* __restrict__ y, const float* __restrict__ t, int B, float* __restrict__ dy,
                            double* __restrict__ loss) {
  __shared__ double red[256];
  double s = 0.0;
  for (int i = threadIdx.x; i < B; i += blockDim.x) {
    const float d = y[i] - t[i];
    dy[i] = 2.f * d / (float)B;
    s += (double)d * d;
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = blockDim.x / 2; w; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0 && loss) *loss = red[0] / B;
}

// relu' mask: g *= (z > 0)
__global__ void relu_grad_kernel(float* __restrict__ g, const float* __restrict__ z, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    if (z[i] <= 0.f) g[i] = 0.f;
}

// Adam (bias-corrected) on the FP32 masters; refresh the BF16 copies
__global__ void adam_kernel(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, __nv_bfloat16* __restrict__ pb, int64_t n, float lr, float b1,
                            float b2, float eps, float c1, float c2) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float pi = p[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    p[i] = pi;
    pb[i] = __float2bfloat16_rn(pi);
  }
}

__global__ void to_bf16_kernel(const float* __restrict__ p, __nv_bfloat16* __restrict__ pb, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    pb[i] = __float2bfloat16_rn(p[i]);
}

template <bool TA, bool TB>
int dense(const float* A, const __nv_bfloat16* Bh, const float* B32, const float* bias, float* C, float* Cpre, int M,
          int N, int K, int relu, int accumulate, cudaStream_t st) {
  dim3 grid((N + 63) / 64, (M + 63) / 64);
  dense_kernel<TA, TB><<<grid, 256, 0, st>>>(A, Bh, B32, bias, C, Cpre, M, N, K, relu, accumulate);
  CUTQC_LAUNCH_CHECK("dense_kernel");
  return CUTQC_OK;
}

struct Work {
  float *z1, *h1, *z2, *h2, *y, *dy, *g1, *g2;
};

size_t work_floats(int B) { return (size_t)B * (2 * D1 + 2 * D2 + 2 + D1 + D2); }

Work carve(float* w, int B) {
  Work k;
  k.z1 = w;
  k.h1 = k.z1 + (size_t)B * D1;
  k.z2 = k.h1 + (size_t)B * D1;
  k.h2 = k.z2 + (size_t)B * D2;
  k.y = k.h2 + (size_t)B * D2;
  k.dy = k.y + B;
  k.g1 = k.dy + B;
  k.g2 = k.g1 + (size_t)B * D1;
  return k;
}

int forward(const float* p32, const __nv_bfloat16* pb, const float* x, int B, const Work& k, cudaStream_t st) {
  int rc;
  if ((rc = dense<false, false>(x, pb + OFF_W1, nullptr, p32 + OFF_B1, k.h1, k.z1, B, D1, D0, 1, 0, st))) return rc;
  if ((rc = dense<false, false>(k.h1, pb + OFF_W2, nullptr, p32 + OFF_B2, k.h2, k.z2, B, D2, D1, 1, 0, st))) return rc;
  return dense<false, false>(k.h2, pb + OFF_W3, nullptr, p32 + OFF_B3, k.y, nullptr, B, D3, D2, 0, 0, st);
}

// gradients of mean (y - t)^2 into grad (flat, same layout as the params)
int backward(const __nv_bfloat16* pb, const float* x, const float* t, int B, const Work& k, float* grad,
             double* loss, cudaStream_t st) {
  int rc;
  loss_kernel<<<1, 256, 0, st>>>(k.y, t, B, k.dy, loss);
  CUTQC_LAUNCH_CHECK("loss_kernel");
  // dW3 = h2^T dy, db3 = sum dy
  if ((rc = dense<true, false>(k.h2, nullptr, k.dy, nullptr, grad + OFF_W3, nullptr, D2, D3, B, 0, 0, st))) return rc;
  colsum_kernel<<<1, 32, 0, st>>>(k.dy, B, D3, grad + OFF_B3);
  // dh2 = dy W3^T, masked by relu'(z2)
  if ((rc = dense<false, true>(k.dy, pb + OFF_W3, nullptr, nullptr, k.g2, nullptr, B, D2, D3, 0, 0, st))) return rc;
  relu_grad_kernel<<<256, 256, 0, st>>>(k.g2, k.z2, (int64_t)B * D2);
  // dW2 = h1^T dz2, db2
  if ((rc = dense<true, false>(k.h1, nullptr, k.g2, nullptr, grad + OFF_W2, nullptr, D1, D2, B, 0, 0, st))) return rc;
  colsum_kernel<<<(D2 + 255) / 256, 256, 0, st>>>(k.g2, B, D2, grad + OFF_B2);
  // dh1 = dz2 W2^T, masked
  if ((rc = dense<false, true>(k.g2, pb + OFF_W2, nullptr, nullptr, k.g1, nullptr, B, D1, D2, 0, 0, st))) return rc;
  relu_grad_kernel<<<256, 256, 0, st>>>(k.g1, k.z1, (int64_t)B * D1);
  // dW1 = x^T dz1, db1
  if ((rc = dense<true, false>(x, nullptr, k.g1, nullptr, grad + OFF_W1, nullptr, D0, D1, B, 0, 0, st))) return rc;
  colsum_kernel<<<(D1 + 255) / 256, 256, 0, st>>>(k.g1, B, D1, grad + OFF_B1);
  count_launches(4);          // the check below covers the five launches above
  CUTQC_LAUNCH_CHECK("mlp backward");
  return CUTQC_OK;
}

int check(const float* p, const void* pb, int B, size_t ws_bytes, const void* ws) {
  if (!p || !pb) return set_error(CUTQC_EINVAL, "null parameters");
  if (B < 1 || B > (1 << 20)) return set_error(CUTQC_EINVAL, "batch out of range");
  if (ws_bytes < work_floats(B) * sizeof(float) || !ws) return set_error(CUTQC_ENOMEM, "MLP workspace too small");
  return CUTQC_OK;
}

}  // namespace
}  // namespace cutqc

using namespace cutqc;

extern "C" int cutqc_mlp_param_count(int64_t* n) {
  if (!n) return set_error(CUTQC_EINVAL, "null");
  *n = NPARAM;
  return CUTQC_OK;
}

extern "C" int cutqc_mlp_workspace_size(int batch, size_t* bytes) {
  if (!bytes || batch < 1) return set_error(CUTQC_EINVAL, "bad arguments");
  *bytes = work_floats(batch) * sizeof(float);
  return CUTQC_OK;
}

extern "C" int cutqc_mlp_sync_bf16(const float* params, void* params_bf16, void* stream) {
  if (!params || !params_bf16) return set_error(CUTQC_EINVAL, "null parameters");
  to_bf16_kernel<<<64, 256, 0, (cudaStream_t)stream>>>(params, (__nv_bfloat16*)params_bf16, NPARAM);
  CUTQC_LAUNCH_CHECK("to_bf16_kernel");
  return CUTQC_OK;
}

extern "C" int cutqc_mlp_forward(const float* params, const void* params_bf16, const float* x, int batch, float* y,
                                 void* ws, size_t ws_bytes, void* stream) {
  int rc = check(params, params_bf16, batch, ws_bytes, ws);
  if (rc) return rc;
  if (!x || !y) return set_error(CUTQC_EINVAL, "null x or y");
  Work k = carve((float*)ws, batch);
  cudaStream_t st = (cudaStream_t)stream;
  if ((rc = forward(params, (const __nv_bfloat16*)params_bf16, x, batch, k, st))) return rc;
  CUTQC_CUDA_TRY(cudaMemcpyAsync(y, k.y, sizeof(float) * batch, cudaMemcpyDeviceToDevice, st));
  return CUTQC_OK;
}

extern "C" int cutqc_mlp_gradients(const float* params, const void* params_bf16, const float* x, const float* t,
                                   int batch, float* grad, double* loss, void* ws, size_t ws_bytes, void* stream) {
  int rc = check(params, params_bf16, batch, ws_bytes, ws);
  if (rc) return rc;
  if (!x || !t || !grad) return set_error(CUTQC_EINVAL, "null x, t or grad");
  Work k = carve((float*)ws, batch);
  cudaStream_t st = (cudaStream_t)stream;
  if ((rc = forward(params, (const __nv_bfloat16*)params_bf16, x, batch, k, st))) return rc;
  return backward((const __nv_bfloat16*)params_bf16, x, t, batch, k, grad, loss, st);
}

extern "C" int cutqc_mlp_adam(float* params, void* params_bf16, const float* grad, float* m, float* v, int step,
                              float lr, float beta1, float beta2, float eps, void* stream) {
  if (!params || !params_bf16 || !grad || !m || !v || step < 1) return set_error(CUTQC_EINVAL, "bad arguments");
  const float c1 = 1.f - powf(beta1, (float)step), c2 = 1.f - powf(beta2, (float)step);
  adam_kernel<<<64, 256, 0, (cudaStream_t)stream>>>(params, grad, m, v, (__nv_bfloat16*)params_bf16, NPARAM, lr,
                                                    beta1, beta2, eps, c1, c2);
  CUTQC_LAUNCH_CHECK("adam_kernel");
  return CUTQC_OK;
}

extern "C" int cutqc_mlp_train_step(float* params, void* params_bf16, float* grad, float* m, float* v, int step,
                                    float lr, const float* x, const float* t, int batch, double* loss, void* ws,
                                    size_t ws_bytes, void* stream) {
  int rc = cutqc_mlp_gradients(params, params_bf16, x, t, batch, grad, loss, ws, ws_bytes, stream);
  if (rc) return rc;
  return cutqc_mlp_adam(params, params_bf16, grad, m, v, step, lr, 0.9f, 0.999f, 1e-8f, stream);
}
