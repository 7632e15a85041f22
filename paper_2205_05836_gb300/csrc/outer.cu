// Last contraction step over few cut terms (K <= 16), Eq. 1 written out:
//   P[m][n] = alpha * sum_k A[m][k] * B[n][k]
// with FP32 fused multiply-adds on CUDA cores.  At K = 4 a probability costs
// 4 multiply-adds and 4 bytes of output, so the step is bound by its stores
// alone; the tensor-core GEMM would pad K to 64 and drain every tile through
// its epilogue warps, which cannot keep up with HBM there.  Output row-major
// in the column index (n_contig): P[m][n] at rowoff(m) + n, rowoff a shift or
// a bit deposit of m.  With the same epilogue statistics as the GEMMs: the
// float64 total (sum) and the largest value of each 32 x 64 block (cmax,
// for the top-T selection of DD).
#include "internal.cuh"
#include "contract.cuh"

#include <algorithm>

namespace cutqc {

namespace {

constexpr int kOuterRows = 32, kOuterCols = 128, kOuterThreads = 256;
// smaller steps (DD's 2^16-bin jobs) stay with the batched FP32 GEMM: one
// launch for all jobs of a level, and enough CTAs for a small output
constexpr double kOuterMinOutputs = (double)(1 << 22);

// CTA: one column tile of 128 columns (lane -> 4 consecutive columns, one
// float4 store per row) and a stride of 32-row groups (warp w -> rows
// 4w .. 4w + 3 of a group).  The tile's B values stay in registers for all
// of the CTA's rows; only A rows are loaded per group (the same address
// across the warp).  a4: A rows are 16-byte aligned runs of K floats.
template <int K>
__global__ void __launch_bounds__(kOuterThreads)
outer_small_k_kernel(const float* __restrict__ A, int64_t lda, const float* __restrict__ B, int64_t ldb, int64_t M,
                     int64_t N, float alpha, uint64_t mask_m, int m_shift, float* __restrict__ out,
                     double* __restrict__ sum, float* __restrict__ cmax, int a4) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t tiles_n = N / kOuterCols, groups = M / kOuterRows;
  const int64_t c = blockIdx.x % tiles_n;
  const int64_t g_step = gridDim.x / tiles_n;     // the grid is a multiple of tiles_n
  const int64_t n = c * kOuterCols + 4 * lane;
  __shared__ float smax[8][2];
  float b[4][K];
#pragma unroll
  for (int j = 0; j < 4; ++j)
#pragma unroll
    for (int k = 0; k < K; ++k) b[j][k] = __ldg(B + (n + j) * ldb + k);
  double local = 0.0;
  for (int64_t g = blockIdx.x / tiles_n; g < groups; g += g_step) {
    const int64_t m0 = g * kOuterRows;
    float part = 0.f, mx = -INFINITY;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int64_t m = m0 + 4 * warp + i;
      float a[K];
      if (K % 4 == 0 && a4) {
#pragma unroll
        for (int k = 0; k < K; k += 4) {
          const float4 q = __ldg(reinterpret_cast<const float4*>(A + m * lda + k));
          a[k] = q.x; a[k + 1] = q.y; a[k + 2] = q.z; a[k + 3] = q.w;
        }
      } else {
#pragma unroll
        for (int k = 0; k < K; ++k) a[k] = __ldg(A + m * lda + k);
      }
      float v[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        float acc = 0.f;
#pragma unroll
        for (int k = 0; k < K; ++k) acc = fmaf(a[k], b[j][k], acc);
        v[j] = acc * alpha;
      }
      const int64_t roff = m_shift >= 0 ? (m << m_shift) : (int64_t)pdep64((uint64_t)m, mask_m);
      __stcs(reinterpret_cast<float4*>(out + roff + n), make_float4(v[0], v[1], v[2], v[3]));
      part += (v[0] + v[1]) + (v[2] + v[3]);
      mx = fmaxf(mx, fmaxf(fmaxf(v[0], v[1]), fmaxf(v[2], v[3])));
    }
    if (sum) local += (double)part;
    if (cmax) {
      // lanes 0..15 hold columns n0 .. n0 + 63, lanes 16..31 the next 64
      for (int off = 8; off; off >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, off));
      if ((lane & 15) == 0) smax[warp][lane >> 4] = mx;
      __syncthreads();
      if (threadIdx.x < 2) {
        float bm = smax[0][threadIdx.x];
        for (int w = 1; w < 8; ++w) bm = fmaxf(bm, smax[w][threadIdx.x]);
        cmax[g * (N / 64) + c * 2 + threadIdx.x] = bm;
      }
      __syncthreads();
    }
  }
  if (sum) {
    for (int off = 16; off; off >>= 1) local += __shfl_xor_sync(0xffffffffu, local, off);
    if (lane == 0) atomicAdd(sum, local);
  }
}

}  // namespace

bool outer_small_k_supported(int64_t K, int64_t M, int64_t N, uint64_t mask_m, uint64_t mask_n) {
  return (K == 1 || K == 4 || K == 16) && M > 0 && N > 0 && M % kOuterRows == 0 && N % kOuterCols == 0 &&
         (double)M * (double)N >= kOuterMinOutputs && mask_is_low(mask_n) && (mask_m & mask_n) == 0;
}

int launch_outer_small_k(const float* A, int64_t lda, const float* B, int64_t ldb, int64_t M, int64_t N, int64_t K,
                         float alpha, uint64_t mask_m, uint64_t mask_n, float* out, double* sum, float* cmax,
                         cudaStream_t st) {
  if (!outer_small_k_supported(K, M, N, mask_m, mask_n))
    return set_error(CUTQC_EINVAL, "internal: outer-product step needs K in {1,4,16}, 32 | M, 128 | N, row-major n");
  if (((uintptr_t)out & 15) != 0) return set_error(CUTQC_EINVAL, "internal: output not 16-byte aligned");
  // every column tile gets the same number of CTAs, each walking a stride
  // of the 32-row groups; the grid fits on the GPU at once (a second,
  // partial wave of these long-running CTAs would leave SMs idle)
  const void* fn = K == 1 ? (const void*)outer_small_k_kernel<1>
                 : K == 4 ? (const void*)outer_small_k_kernel<4> : (const void*)outer_small_k_kernel<16>;
  int resident = 0;
  CUTQC_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&resident, fn, kOuterThreads, 0));
  const int64_t tiles_n = N / kOuterCols, groups = M / kOuterRows;
  const int64_t slots = (int64_t)sm_count() * std::max(1, resident);
  const int64_t per_tile = std::max<int64_t>(1, std::min<int64_t>(groups, slots / tiles_n));
  if (tiles_n * per_tile > 0x7fffffffLL) return set_error(CUTQC_EUNSUPPORTED, "outer-product step too wide");
  const int grid = (int)(tiles_n * per_tile);
  const int m_shift = mask_contig_shift(mask_m);
  const int a4 = (lda % 4 == 0 && ((uintptr_t)A & 15) == 0) ? 1 : 0;
  switch (K) {
    case 1:
      outer_small_k_kernel<1><<<grid, kOuterThreads, 0, st>>>(A, lda, B, ldb, M, N, alpha, mask_m, m_shift, out, sum,
                                                              cmax, a4);
      break;
    case 4:
      outer_small_k_kernel<4><<<grid, kOuterThreads, 0, st>>>(A, lda, B, ldb, M, N, alpha, mask_m, m_shift, out, sum,
                                                              cmax, a4);
      break;
    default:
      outer_small_k_kernel<16><<<grid, kOuterThreads, 0, st>>>(A, lda, B, ldb, M, N, alpha, mask_m, m_shift, out,
                                                               sum, cmax, a4);
      break;
  }
  CUTQC_LAUNCH_CHECK("outer_small_k_kernel");
  return CUTQC_OK;
}

}  // namespace cutqc
