// Pairwise contraction building blocks for Eq. 1 (Full Definition).
//
// A contraction step joins two tensors Ta [2^oa][4^ka], Tb [2^ob][4^kb]
// (columns = cut digits in ascending edge id) over their shared cut edges S:
//   T[(xa, xb)][(ea', eb')] = sum_{s in 4^|S|} Ta[xa][(ea', s)] Tb[xb][(eb', s)]
// which is a GEMM C[m][n] = sum_s A'[m][s] B'[n][s] with m = (xa, ea'),
// n = (xb, eb').  The result index is a bit deposit of m and n:
//   out = pdep(m, mask_m) | pdep(n, mask_n)
// which covers the Kronecker order of Eq. 1, the uncut circuit's qubit order,
// and the digit interleaving of intermediate tensors alike.
//
// This file holds the operand gather ("prep": builds A' or B' K-major, either
// float32 or as a float16 hi/lo pair with a power-of-two scale per row) and
// the float32 CUDA-core GEMM.  The tensor-core GEMM is in gemm_tc.cu.
#include "internal.cuh"
#include "contract.cuh"
#include "sgemm_tile.cuh"

#include <algorithm>
#include <mutex>
#include <set>

namespace cutqc {

// ----------------------------------------------------------------- prep

// One warp per output row.  Local row r -> operand row m = r + row0;
// m = (xp, open): xp = the high bits, open = the low 2*n_open bits.  The
// source row x is xp with its bits moved by the row map (bit j of xp goes to
// bit rm.bit[j] of x; identity unless rm.permute).  K index s = shared digits;
// source column = pdep(open, open_dmask) | pdep(s, shared_dmask).
// Half mode: a power-of-two scale puts the max |x| of the row (mode 0) or of
// the whole operand (mode 1, max read from *gmax) in [2^14, 2^15) (clamped to
// [2^-60, 2^60] so that the scale, its inverse and the epilogue's product of
// two scales and 2^-K stay normal floats; values that small contribute below
// float32 resolution of any output); y = x / scale is split as hi = fp16(y),
// lo = fp16(y - hi).  Mode 2 only accumulates max|x| into *gmax (float bits:
// the values are non-negative, so integer max orders them).  When the source
// columns are the row itself (no gather) and K is a multiple of 4, lanes move
// float4 / 4 x half vectors, each lane holding its part of the row.
__device__ __forceinline__ float pow2_scale(float mx) {
  if (!(mx > 0.f)) return 1.f;
  int e = 0;
  frexpf(mx, &e);          // mx = f * 2^e, f in [0.5, 1)
  return ldexpf(1.f, max(-60, min(60, e - 15)));
}
__device__ __forceinline__ uint2 pack4(__half a, __half b, __half c, __half d) {
  __half2 p = __halves2half2(a, b), q = __halves2half2(c, d);
  return make_uint2(*reinterpret_cast<uint32_t*>(&p), *reinterpret_cast<uint32_t*>(&q));
}
constexpr int PREP_VEC_MAX = 8;   // float4 per lane kept in registers (K <= 1024)

__global__ void prep_kernel(OperandView v, RowMap rm, int64_t row0, int64_t rows, int64_t K, int64_t Kp,
                            float* __restrict__ out32, __half* __restrict__ hi,
                            __half* __restrict__ lo, float* __restrict__ scale, int64_t src_bstride,
                            int64_t dst_bstride, int mode, unsigned int* __restrict__ gmax,
                            const int* __restrict__ cols, const int* __restrict__ meta) {
  // batch item blockIdx.y: source and destinations offset by their strides
  v.src += (int64_t)blockIdx.y * src_bstride;
  if (out32) out32 += (int64_t)blockIdx.y * dst_bstride * Kp;
  if (hi) {
    hi += (int64_t)blockIdx.y * dst_bstride * Kp;
    lo += (int64_t)blockIdx.y * dst_bstride * Kp;
    scale += (int64_t)blockIdx.y * dst_bstride;
  }
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  const int64_t C = (int64_t)1 << (2 * v.k);
  const bool contig = v.n_open == 0 && v.shared_dmask == (uint64_t)(C - 1);
  // the shared digits are the lowest digit positions: row r's K values are
  // consecutive from obase (the open digits sit above them)
  const bool low_shared = cols == nullptr && v.shared_dmask == (((uint64_t)1 << (2 * v.n_shared)) - 1);
  // column list (cut-term pruning): operand column s < meta[0] is source
  // column cols[s]; columns [meta[0], meta[2]) are zero; the rest of the row
  // is not written (the GEMM reads meta[2] / 64 k-blocks)
  int64_t Kw = Kp;      // columns written per row (the row stride stays Kp)
  __shared__ int scols[kPruneMaxK];
  if (cols) {
    K = __ldg(meta);
    Kw = __ldg(meta + 2);
    for (int64_t s = threadIdx.x; s < K; s += blockDim.x) scols[s] = __ldg(cols + s);
    __syncthreads();
  }
  float wmax = 0.f;    // mode 2: this warp's running max
  for (int64_t r = warp; r < rows; r += nwarps) {
    const int64_t m = r + row0;
    const uint64_t xp = (uint64_t)m >> (2 * v.n_open);
    uint64_t x = xp;
    if (rm.permute) {
      x = 0;
      for (int j = 0; j < rm.n; ++j) x |= ((xp >> j) & 1) << rm.bit[j];
    }
    const uint64_t open = (uint64_t)m & (((uint64_t)1 << (2 * v.n_open)) - 1);
    const uint64_t obase = pdep64(open, v.open_dmask);
    const float* row = v.src + (int64_t)x * C;
    auto col = [&](int64_t s) -> int64_t {
      if (cols) s = scols[s];
      return contig ? s : (int64_t)(obase | pdep64((uint64_t)s, v.shared_dmask));
    };
    if (out32) {
      for (int64_t s = lane; s < Kw; s += 32) {
        float val = 0.f;
        if (s < K) val = __ldg(row + col(s));
        out32[r * Kp + s] = val;
      }
      continue;
    }
    if (low_shared && hi && (K & 3) == 0 && K <= 128 * PREP_VEC_MAX &&
        ((reinterpret_cast<uintptr_t>(row + obase) & 15) == 0)) {
      const float4* row4 = reinterpret_cast<const float4*>(row + obase);
      const int64_t K4 = K >> 2, Kp4 = Kw >> 2;
      float4 val[PREP_VEC_MAX];
      float mx = 0.f;
#pragma unroll
      for (int i = 0; i < PREP_VEC_MAX; ++i) {
        const int64_t j = lane + 32 * i;
        val[i] = j < K4 ? __ldg(row4 + j) : make_float4(0.f, 0.f, 0.f, 0.f);
        mx = fmaxf(mx, fmaxf(fmaxf(fabsf(val[i].x), fabsf(val[i].y)), fmaxf(fabsf(val[i].z), fabsf(val[i].w))));
      }
      for (int off = 16; off; off >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, off));
      if (mode == 2) {
        wmax = fmaxf(wmax, mx);
        continue;
      }
      const float sc = pow2_scale(mode == 1 ? __uint_as_float(*gmax) : mx);
      const float inv = 1.f / sc;   // exact: power of two
      if (lane == 0 && (mode == 0 || r == 0)) scale[mode == 0 ? r : 0] = sc;
      uint2* h4 = reinterpret_cast<uint2*>(hi + r * Kp);
      uint2* l4 = reinterpret_cast<uint2*>(lo + r * Kp);
#pragma unroll
      for (int i = 0; i < PREP_VEC_MAX; ++i) {
        const int64_t j = lane + 32 * i;
        if (j < K4) {
          const float y0 = val[i].x * inv, y1 = val[i].y * inv, y2 = val[i].z * inv, y3 = val[i].w * inv;
          const __half a0 = __float2half_rn(y0), a1 = __float2half_rn(y1), a2 = __float2half_rn(y2),
                       a3 = __float2half_rn(y3);
          h4[j] = pack4(a0, a1, a2, a3);
          l4[j] = pack4(__float2half_rn(y0 - __half2float(a0)), __float2half_rn(y1 - __half2float(a1)),
                        __float2half_rn(y2 - __half2float(a2)), __float2half_rn(y3 - __half2float(a3)));
        }
      }
      for (int64_t j = K4 + lane; j < Kp4; j += 32) {
        h4[j] = make_uint2(0, 0);
        l4[j] = make_uint2(0, 0);
      }
      continue;
    }
    float mx = 0.f;
    if (mode == 1) {
      mx = __uint_as_float(*gmax);
    } else {
#pragma unroll 4
      for (int64_t s = lane; s < K; s += 32) mx = fmaxf(mx, fabsf(__ldg(row + col(s))));
      for (int off = 16; off; off >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, off));
      if (mode == 2) {
        wmax = fmaxf(wmax, mx);
        continue;
      }
    }
    const float sc = pow2_scale(mx);
    const float inv = 1.f / sc;   // exact: power of two
    if (lane == 0 && (mode == 0 || r == 0)) scale[mode == 0 ? r : 0] = sc;
    // four gathered loads in flight per lane, then the splits and stores
    for (int64_t s0 = lane; s0 < Kw; s0 += 128) {
      float y[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int64_t s = s0 + 32 * u;
        y[u] = s < K ? __ldg(row + col(s)) * inv : 0.f;
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int64_t s = s0 + 32 * u;
        if (s < Kw) {
          const __half h = __float2half_rn(y[u]);
          hi[r * Kp + s] = h;
          lo[r * Kp + s] = __float2half_rn(y[u] - __half2float(h));
        }
      }
    }
  }
  if (mode == 2) {
    // one atomic per block
    __shared__ float bmax[32];
    if (lane == 0) bmax[threadIdx.x >> 5] = wmax;
    __syncthreads();
    if (threadIdx.x == 0) {
      float m = 0.f;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = fmaxf(m, bmax[w]);
      atomicMax(gmax, __float_as_uint(m));
    }
  }
}

// max |x| over n contiguous floats into *gmax (float bits; the values are
// non-negative, so the integer max orders them): float4 loads, four in
// flight per thread, one atomic per block.  Stands in for the max pass of an
// operand-wide scale when the operand covers its whole source tensor (every
// row, every column: the same set of values).
__global__ void __launch_bounds__(256) absmax_kernel(const float* __restrict__ x, int64_t n,
                                                     unsigned int* __restrict__ gmax) {
  const float4* x4 = reinterpret_cast<const float4*>(x);
  const int64_t n4 = n >> 2;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  float mx = 0.f;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += 4 * stride) {
    float4 v[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) v[u] = i + u * stride < n4 ? __ldg(x4 + i + u * stride) : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int u = 0; u < 4; ++u)
      mx = fmaxf(mx, fmaxf(fmaxf(fabsf(v[u].x), fabsf(v[u].y)), fmaxf(fabsf(v[u].z), fabsf(v[u].w))));
  }
  for (int64_t i = 4 * n4 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
    mx = fmaxf(mx, fabsf(__ldg(x + i)));
  for (int off = 16; off; off >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, off));
  __shared__ float bmax[8];
  if ((threadIdx.x & 31) == 0) bmax[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    float m = 0.f;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = fmaxf(m, bmax[w]);
    atomicMax(gmax, __float_as_uint(m));
  }
}

// Rows of K = Kp = 256 values, the shared digits the lowest of the source
// columns (the usual operand of a 4-cut contraction): one warp per row as in
// prep_kernel's vector path (two float4 per lane), but kPrepRows rows per
// step with all their loads issued before the splits, so that a warp keeps
// 4 KiB in flight instead of 1.  Modes 0 and 1 of prep_kernel, same results.
constexpr int kPrepRows = 4;

__global__ void __launch_bounds__(256)
prep_rows256_kernel(OperandView v, RowMap rm, int64_t row0, int64_t rows, __half* __restrict__ hi,
                    __half* __restrict__ lo, float* __restrict__ scale, int64_t src_bstride, int64_t dst_bstride,
                    int mode, const unsigned int* __restrict__ gmax) {
  constexpr int K4 = 64;
  v.src += (int64_t)blockIdx.y * src_bstride;
  hi += (int64_t)blockIdx.y * dst_bstride * 256;
  lo += (int64_t)blockIdx.y * dst_bstride * 256;
  scale += (int64_t)blockIdx.y * dst_bstride;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  const int64_t C = (int64_t)1 << (2 * v.k);
  const float gsc = mode == 1 ? pow2_scale(__uint_as_float(*gmax)) : 1.f;
  for (int64_t base = (int64_t)warp * kPrepRows; base < rows; base += (int64_t)nwarps * kPrepRows) {
    float4 val[kPrepRows][2];
#pragma unroll
    for (int g = 0; g < kPrepRows; ++g) {
      const int64_t r = base + g;
      val[g][0] = val[g][1] = make_float4(0.f, 0.f, 0.f, 0.f);
      if (r < rows) {
        const int64_t m = r + row0;
        const uint64_t xp = (uint64_t)m >> (2 * v.n_open);
        uint64_t x = xp;
        if (rm.permute) {
          x = 0;
          for (int j = 0; j < rm.n; ++j) x |= ((xp >> j) & 1) << rm.bit[j];
        }
        const uint64_t open = (uint64_t)m & (((uint64_t)1 << (2 * v.n_open)) - 1);
        const float4* row4 = reinterpret_cast<const float4*>(v.src + (int64_t)x * C + pdep64(open, v.open_dmask));
        val[g][0] = __ldg(row4 + lane);
        val[g][1] = __ldg(row4 + lane + 32);
      }
    }
#pragma unroll
    for (int g = 0; g < kPrepRows; ++g) {
      const int64_t r = base + g;
      if (r >= rows) break;
      float sc = gsc;
      if (mode == 0) {
        float mx = 0.f;
#pragma unroll
        for (int i = 0; i < 2; ++i)
          mx = fmaxf(mx, fmaxf(fmaxf(fabsf(val[g][i].x), fabsf(val[g][i].y)),
                               fmaxf(fabsf(val[g][i].z), fabsf(val[g][i].w))));
        for (int off = 16; off; off >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, off));
        sc = pow2_scale(mx);
      }
      const float inv = 1.f / sc;   // exact: power of two
      if (lane == 0 && (mode == 0 || r == 0)) scale[mode == 0 ? r : 0] = sc;
      uint2* h4 = reinterpret_cast<uint2*>(hi + r * 256);
      uint2* l4 = reinterpret_cast<uint2*>(lo + r * 256);
#pragma unroll
      for (int i = 0; i < 2; ++i) {
        const float y0 = val[g][i].x * inv, y1 = val[g][i].y * inv, y2 = val[g][i].z * inv, y3 = val[g][i].w * inv;
        const __half a0 = __float2half_rn(y0), a1 = __float2half_rn(y1), a2 = __float2half_rn(y2),
                     a3 = __float2half_rn(y3);
        h4[lane + 32 * i] = pack4(a0, a1, a2, a3);
        l4[lane + 32 * i] = pack4(__float2half_rn(y0 - __half2float(a0)), __float2half_rn(y1 - __half2float(a1)),
                                  __float2half_rn(y2 - __half2float(a2)), __float2half_rn(y3 - __half2float(a3)));
      }
    }
  }
  static_assert(K4 == 2 * 32, "two float4 per lane per row");
}

// Rows of 256 source values with a column list (cut-term pruning): each
// row read whole as in prep_rows256_kernel (two float4 per lane, kPrepRows
// rows per warp in flight) into the warp's part of shared memory, then the
// kept columns gathered from there.  A few dozen scattered columns of a 1 KB
// row touch nearly all of its sectors anyway, and whole-row vector loads
// take far fewer instructions than one load per kept column.  Output column
// s < meta[0] is source column cols[s], columns [meta[0], meta[2]) are zero,
// the rest of the row (stride 256) is not written.  Modes 0 and 1 of
// prep_kernel, same results.
__global__ void __launch_bounds__(256)
prep_rows256_cols_kernel(OperandView v, RowMap rm, int64_t row0, int64_t rows, __half* __restrict__ hi,
                         __half* __restrict__ lo, float* __restrict__ scale, int mode,
                         const unsigned int* __restrict__ gmax, const int* __restrict__ cols,
                         const int* __restrict__ meta) {
  __shared__ __align__(16) float srow[8][kPrepRows][256];
  __shared__ int scols[256];
  const int K = __ldg(meta), Kw = __ldg(meta + 2);
  for (int c = threadIdx.x; c < K; c += blockDim.x) scols[c] = __ldg(cols + c);
  __syncthreads();
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  const int64_t C = (int64_t)1 << (2 * v.k);
  const float gsc = mode == 1 ? pow2_scale(__uint_as_float(*gmax)) : 1.f;
  float (*sw)[256] = srow[threadIdx.x >> 5];
  for (int64_t base = (int64_t)warp * kPrepRows; base < rows; base += (int64_t)nwarps * kPrepRows) {
    float4 val[kPrepRows][2];
#pragma unroll
    for (int g = 0; g < kPrepRows; ++g) {
      const int64_t r = base + g;
      val[g][0] = val[g][1] = make_float4(0.f, 0.f, 0.f, 0.f);
      if (r < rows) {
        const int64_t m = r + row0;
        const uint64_t xp = (uint64_t)m >> (2 * v.n_open);
        uint64_t x = xp;
        if (rm.permute) {
          x = 0;
          for (int j = 0; j < rm.n; ++j) x |= ((xp >> j) & 1) << rm.bit[j];
        }
        const uint64_t open = (uint64_t)m & (((uint64_t)1 << (2 * v.n_open)) - 1);
        const float4* row4 = reinterpret_cast<const float4*>(v.src + (int64_t)x * C + pdep64(open, v.open_dmask));
        val[g][0] = __ldg(row4 + lane);
        val[g][1] = __ldg(row4 + lane + 32);
      }
    }
    __syncwarp();        // the previous step's gathers from sw are done
#pragma unroll
    for (int g = 0; g < kPrepRows; ++g) {
      reinterpret_cast<float4*>(sw[g])[lane] = val[g][0];
      reinterpret_cast<float4*>(sw[g])[lane + 32] = val[g][1];
    }
    __syncwarp();
#pragma unroll
    for (int g = 0; g < kPrepRows; ++g) {
      const int64_t r = base + g;
      if (r >= rows) break;
      float y[2][4];
      float mx = 0.f;
#pragma unroll
      for (int j = 0; j < 2; ++j)
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int c = 4 * (lane + 32 * j) + e;
          y[j][e] = c < K ? sw[g][scols[c]] : 0.f;
          mx = fmaxf(mx, fabsf(y[j][e]));
        }
      float sc = gsc;
      if (mode == 0) {
        for (int off = 16; off; off >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, off));
        sc = pow2_scale(mx);
      }
      const float inv = 1.f / sc;   // exact: power of two
      if (lane == 0 && (mode == 0 || r == 0)) scale[mode == 0 ? r : 0] = sc;
      uint2* h4 = reinterpret_cast<uint2*>(hi + r * 256);
      uint2* l4 = reinterpret_cast<uint2*>(lo + r * 256);
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        const int q = lane + 32 * j;
        if (4 * q >= Kw) continue;
        const float y0 = y[j][0] * inv, y1 = y[j][1] * inv, y2 = y[j][2] * inv, y3 = y[j][3] * inv;
        const __half a0 = __float2half_rn(y0), a1 = __float2half_rn(y1), a2 = __float2half_rn(y2),
                     a3 = __float2half_rn(y3);
        h4[q] = pack4(a0, a1, a2, a3);
        l4[q] = pack4(__float2half_rn(y0 - __half2float(a0)), __float2half_rn(y1 - __half2float(a1)),
                      __float2half_rn(y2 - __half2float(a2)), __float2half_rn(y3 - __half2float(a3)));
      }
    }
  }
}

// Short rows (Kp = 8 G half columns, K <= Kp values, K % 4 == 0, the
// shared digits the lowest of the source columns): G lanes per row, each
// lane loading its 8 columns (two float4, zeros past K) and writing them as
// one 16-byte vector of hi and one of lo; a warp takes 32 / G rows at once
// (one warp per row left most lanes idle: 2^18 rows of K = 4 took 97 us).
// Same modes and results as prep_kernel.
template <int G>
__global__ void __launch_bounds__(256)
prep_small_kernel(OperandView v, RowMap rm, int64_t row0, int64_t rows, int64_t K, __half* __restrict__ hi,
                  __half* __restrict__ lo, float* __restrict__ scale, int64_t src_bstride, int64_t dst_bstride,
                  int mode, unsigned int* __restrict__ gmax) {
  constexpr int Kp = 8 * G, RPW = 32 / G;
  v.src += (int64_t)blockIdx.y * src_bstride;
  hi += (int64_t)blockIdx.y * dst_bstride * Kp;
  lo += (int64_t)blockIdx.y * dst_bstride * Kp;
  scale += (int64_t)blockIdx.y * dst_bstride;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31, gl = lane % G, sub = lane / G;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  const int64_t C = (int64_t)1 << (2 * v.k);
  const float gsc = mode == 1 ? pow2_scale(__uint_as_float(*gmax)) : 1.f;
  float wmax = 0.f;
  for (int64_t base = (int64_t)warp * RPW; base < rows; base += (int64_t)nwarps * RPW) {
    const int64_t r = base + sub;
    const bool valid = r < rows;
    float4 a = make_float4(0.f, 0.f, 0.f, 0.f), b = a;
    if (valid) {
      const int64_t m = r + row0;
      const uint64_t xp = (uint64_t)m >> (2 * v.n_open);
      uint64_t x = xp;
      if (rm.permute) {
        x = 0;
        for (int j = 0; j < rm.n; ++j) x |= ((xp >> j) & 1) << rm.bit[j];
      }
      const uint64_t open = (uint64_t)m & (((uint64_t)1 << (2 * v.n_open)) - 1);
      const float4* row4 = reinterpret_cast<const float4*>(v.src + (int64_t)x * C + pdep64(open, v.open_dmask));
      if (8 * gl < K) a = __ldg(row4 + 2 * gl);
      if (8 * gl + 4 < K) b = __ldg(row4 + 2 * gl + 1);
    }
    float mx = fmaxf(fmaxf(fmaxf(fabsf(a.x), fabsf(a.y)), fmaxf(fabsf(a.z), fabsf(a.w))),
                     fmaxf(fmaxf(fabsf(b.x), fabsf(b.y)), fmaxf(fabsf(b.z), fabsf(b.w))));
#pragma unroll
    for (int off = 1; off < G; off <<= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, off));
    if (mode == 2) {
      wmax = fmaxf(wmax, mx);
      continue;
    }
    if (!valid) continue;
    const float sc = mode == 1 ? gsc : pow2_scale(mx);
    const float inv = 1.f / sc;   // exact: power of two
    if (gl == 0 && (mode == 0 || r == 0)) scale[mode == 0 ? r : 0] = sc;
    const float y[8] = {a.x * inv, a.y * inv, a.z * inv, a.w * inv, b.x * inv, b.y * inv, b.z * inv, b.w * inv};
    __half h[8], l[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      h[i] = __float2half_rn(y[i]);
      l[i] = __float2half_rn(y[i] - __half2float(h[i]));
    }
    const uint2 h0 = pack4(h[0], h[1], h[2], h[3]), h1 = pack4(h[4], h[5], h[6], h[7]);
    const uint2 l0 = pack4(l[0], l[1], l[2], l[3]), l1 = pack4(l[4], l[5], l[6], l[7]);
    reinterpret_cast<uint4*>(hi + r * Kp)[gl] = make_uint4(h0.x, h0.y, h1.x, h1.y);
    reinterpret_cast<uint4*>(lo + r * Kp)[gl] = make_uint4(l0.x, l0.y, l1.x, l1.y);
  }
  if (mode == 2) {
    // each row group of the warp kept its own rows' max: combine the groups
#pragma unroll
    for (int off = G; off < 32; off <<= 1) wmax = fmaxf(wmax, __shfl_xor_sync(0xffffffffu, wmax, off));
    __shared__ float bmax[32];
    if (lane == 0) bmax[threadIdx.x >> 5] = wmax;
    __syncthreads();
    if (threadIdx.x == 0) {
      float m = 0.f;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = fmaxf(m, bmax[w]);
      atomicMax(gmax, __float_as_uint(m));
    }
  }
}

// Transposing variant for operands whose open digits are the lowest digits
// of the source columns (n_open >= 3): for a fixed source row x and shared
// index s, the operand rows (x, open) and (x, open + 1) are adjacent in
// memory, while one operand row's K values are 4^n_open floats apart.  A
// block takes 32 consecutive operand rows (one source row x, 32 consecutive
// open values): its warps read the tile [K][32] with one coalesced 128-byte
// load per s (each warp a contiguous run of s, the source column advanced by
// a submask increment), stage it in shared memory ([K][33], conflict-free
// both ways), then write the rows K-major exactly as prep_kernel does.
// Requires row0 % 32 == 0 so that a tile never straddles two source rows.
constexpr int kTrBatch = 8;

__global__ void prep_tr_kernel(OperandView v, RowMap rm, int64_t row0, int64_t rows, int64_t K, int64_t Kp,
                               float* __restrict__ out32, __half* __restrict__ hi, __half* __restrict__ lo,
                               float* __restrict__ scale, int64_t src_bstride, int64_t dst_bstride, int mode,
                               unsigned int* __restrict__ gmax) {
  extern __shared__ float tile[];   // [K][33]
  v.src += (int64_t)blockIdx.y * src_bstride;
  if (out32) out32 += (int64_t)blockIdx.y * dst_bstride * Kp;
  if (hi) {
    hi += (int64_t)blockIdx.y * dst_bstride * Kp;
    lo += (int64_t)blockIdx.y * dst_bstride * Kp;
    scale += (int64_t)blockIdx.y * dst_bstride;
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  const int64_t C = (int64_t)1 << (2 * v.k);
  const int ob = 2 * v.n_open;
  const int64_t per = (K + nw - 1) / nw;
  const int64_t s_lo = warp * per < K ? warp * per : K;
  const int64_t s_hi = s_lo + per < K ? s_lo + per : K;
  const uint64_t smask = v.shared_dmask;
  const uint64_t col_lo = pdep64((uint64_t)s_lo, smask);
  const int64_t ntiles = (rows + 31) >> 5;
  float wmax = 0.f;
  for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int64_t r0 = t << 5;
    const int64_t m0 = r0 + row0;
    const uint64_t xp = (uint64_t)m0 >> ob;
    uint64_t x = xp;
    if (rm.permute) {
      x = 0;
      for (int j = 0; j < rm.n; ++j) x |= ((xp >> j) & 1) << rm.bit[j];
    }
    const uint64_t open0 = (uint64_t)m0 & (((uint64_t)1 << ob) - 1);
    const bool rvalid = r0 + lane < rows;
    const float* base = v.src + (int64_t)x * C + (int64_t)open0 + lane;
    uint64_t col = col_lo;
    for (int64_t s0 = s_lo; s0 < s_hi; s0 += kTrBatch) {
      // kTrBatch loads in flight per lane before any store to shared memory
      float val[kTrBatch];
#pragma unroll
      for (int u = 0; u < kTrBatch; ++u) {
        val[u] = (rvalid && s0 + u < s_hi) ? __ldg(base + col) : 0.f;
        col = ((col | ~smask) + 1) & smask;     // next submask of smask in increasing order
      }
#pragma unroll
      for (int u = 0; u < kTrBatch; ++u) {
        if (s0 + u >= s_hi) break;
        if (mode == 2) wmax = fmaxf(wmax, fabsf(val[u]));
        else tile[(s0 + u) * 33 + lane] = val[u];
      }
    }
    if (mode == 2) continue;
    __syncthreads();
    for (int rr = warp; rr < 32; rr += nw) {
      const int64_t r = r0 + rr;
      if (r >= rows) break;
      if (out32) {
        for (int64_t s = lane; s < Kp; s += 32) out32[r * Kp + s] = s < K ? tile[s * 33 + rr] : 0.f;
        continue;
      }
      float mx = 0.f;
      if (mode == 1) {
        mx = __uint_as_float(*gmax);
      } else {
        for (int64_t s = lane; s < K; s += 32) mx = fmaxf(mx, fabsf(tile[s * 33 + rr]));
        for (int off = 16; off; off >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, off));
      }
      const float sc = pow2_scale(mx);
      const float inv = 1.f / sc;   // exact: power of two
      if (lane == 0 && (mode == 0 || r == 0)) scale[mode == 0 ? r : 0] = sc;
      for (int64_t s = lane; s < Kp; s += 32) {
        const float y = s < K ? tile[s * 33 + rr] * inv : 0.f;
        const __half h = __float2half_rn(y);
        hi[r * Kp + s] = h;
        lo[r * Kp + s] = __float2half_rn(y - __half2float(h));
      }
    }
    __syncthreads();
  }
  if (mode == 2) {
    for (int off = 16; off; off >>= 1) wmax = fmaxf(wmax, __shfl_xor_sync(0xffffffffu, wmax, off));
    __shared__ float bmax[32];
    if (lane == 0) bmax[warp] = wmax;
    __syncthreads();
    if (threadIdx.x == 0) {
      float m = 0.f;
      for (int w = 0; w < nw; ++w) m = fmaxf(m, bmax[w]);
      atomicMax(gmax, __float_as_uint(m));
    }
  }
}

// ------------------------------------------------ cut-term pruning
// Term k of a contraction (one assignment of the shared cut digits)
// contributes alpha * A[m][k] * B[n][k] to output (m, n); summed over the
// outputs, its absolute contribution is at most
//   w_k = alpha * sum_m |A[m][k]| * sum_n |B[n][k]|.
// colw_kernel accumulates sum_rows |operand[row][k]| and max_rows
// |operand[row][k]| (warp per row, the columns a lane owns in registers --
// float4 loads when a row's K values are contiguous -- then a block
// reduction and one atomic per column and block); prune_select_kernel drops
// the terms of smallest w_k while their total stays <= tol and writes the
// kept columns in ascending order.  Dropping them changes the output by at
// most tol in L1 (TV by tol / 2).
template <int NPL>
__global__ void __launch_bounds__(256)
colw_kernel(OperandView v, RowMap rm, int64_t row0, int64_t rows, int64_t K, float* __restrict__ colw,
            unsigned int* __restrict__ colmax) {
  extern __shared__ float part[];   // [K] sums, then [K] maxima (float bits)
  unsigned int* pmax = reinterpret_cast<unsigned int*>(part + K);
  for (int64_t s = threadIdx.x; s < K; s += blockDim.x) {
    part[s] = 0.f;
    pmax[s] = 0u;
  }
  __syncthreads();
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  const int64_t C = (int64_t)1 << (2 * v.k);
  const bool contig = v.n_open == 0 && v.shared_dmask == (uint64_t)(C - 1);
  const bool low_shared = v.shared_dmask == (((uint64_t)1 << (2 * v.n_shared)) - 1);
  const bool vec = low_shared && (K & 127) == 0 && ((reinterpret_cast<uintptr_t>(v.src) & 15) == 0);
  float acc[NPL], mx[NPL];
#pragma unroll
  for (int i = 0; i < NPL; ++i) acc[i] = mx[i] = 0.f;
  // rows of exactly 256 contiguous values: kPrepRows rows per warp step, all
  // their loads issued first (one row at a time kept 1 KB in flight per warp)
  const bool vec4 = vec && NPL == 8 && K == 256;
  for (int64_t base = (int64_t)warp * kPrepRows; vec4 && base < rows; base += (int64_t)nwarps * kPrepRows) {
    float4 q[kPrepRows][2];
#pragma unroll
    for (int g = 0; g < kPrepRows; ++g) {
      const int64_t r = base + g;
      q[g][0] = q[g][1] = make_float4(0.f, 0.f, 0.f, 0.f);
      if (r < rows) {
        const int64_t m = r + row0;
        const uint64_t xp = (uint64_t)m >> (2 * v.n_open);
        uint64_t x = xp;
        if (rm.permute) {
          x = 0;
          for (int j = 0; j < rm.n; ++j) x |= ((xp >> j) & 1) << rm.bit[j];
        }
        const uint64_t open = (uint64_t)m & (((uint64_t)1 << (2 * v.n_open)) - 1);
        const float4* row4 = reinterpret_cast<const float4*>(v.src + (int64_t)x * C + pdep64(open, v.open_dmask));
        q[g][0] = __ldg(row4 + lane);
        q[g][1] = __ldg(row4 + lane + 32);
      }
    }
#pragma unroll
    for (int g = 0; g < kPrepRows; ++g)
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        const float e[4] = {fabsf(q[g][j].x), fabsf(q[g][j].y), fabsf(q[g][j].z), fabsf(q[g][j].w)};
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          acc[4 * j + t] += e[t];
          mx[4 * j + t] = fmaxf(mx[4 * j + t], e[t]);
        }
      }
  }
  for (int64_t r = warp; !vec4 && r < rows; r += nwarps) {
    const int64_t m = r + row0;
    const uint64_t xp = (uint64_t)m >> (2 * v.n_open);
    uint64_t x = xp;
    if (rm.permute) {
      x = 0;
      for (int j = 0; j < rm.n; ++j) x |= ((xp >> j) & 1) << rm.bit[j];
    }
    const uint64_t open = (uint64_t)m & (((uint64_t)1 << (2 * v.n_open)) - 1);
    const uint64_t obase = pdep64(open, v.open_dmask);
    const float* row = v.src + (int64_t)x * C;
    if (vec) {
      // lane owns columns 4 (lane + 32 j) .. +3, j < K / 128
      const float4* row4 = reinterpret_cast<const float4*>(row + obase);
#pragma unroll
      for (int j = 0; j < NPL / 4; ++j) {
        if (128 * j < K) {
          const float4 q = __ldg(row4 + lane + 32 * j);
          const float e[4] = {fabsf(q.x), fabsf(q.y), fabsf(q.z), fabsf(q.w)};
#pragma unroll
          for (int t = 0; t < 4; ++t) {
            acc[4 * j + t] += e[t];
            mx[4 * j + t] = fmaxf(mx[4 * j + t], e[t]);
          }
        }
      }
    } else {
#pragma unroll
      for (int i = 0; i < NPL; ++i) {
        const int64_t s = lane + 32 * i;
        if (s < K) {
          const float e = fabsf(__ldg(row + (contig ? s : (int64_t)(obase | pdep64((uint64_t)s, v.shared_dmask)))));
          acc[i] += e;
          mx[i] = fmaxf(mx[i], e);
        }
      }
    }
  }
#pragma unroll
  for (int i = 0; i < NPL; ++i) {
    const int64_t s = vec ? 4 * (lane + 32 * (i / 4)) + (i % 4) : lane + 32 * i;
    if (s < K) {
      atomicAdd(&part[s], acc[i]);
      atomicMax(&pmax[s], __float_as_uint(mx[i]));   // non-negative floats order as integers
    }
  }
  __syncthreads();
  for (int64_t s = threadIdx.x; s < K; s += blockDim.x) {
    atomicAdd(colw + s, part[s]);
    if (colmax) atomicMax(colmax + s, pmax[s]);
  }
}

constexpr int PRUNE_MAX_K = (int)kPruneMaxK;

// One CTA of 1024 threads (K <= 1024): rank the terms by (w_k, k), prefix
// sums of the sorted weights, the cut, and the compaction of the kept
// columns, all by parallel scans in shared memory.  Also the largest |B|
// over the kept columns (the column operand's scale), into *gmax_b.
__global__ void __launch_bounds__(1024)
prune_select_kernel(const float* __restrict__ wa, const float* __restrict__ wb,
                    const unsigned int* __restrict__ bmax, int K, float alpha, float tol, int* __restrict__ cols,
                    int* __restrict__ meta, unsigned int* __restrict__ gmax_b) {
  __shared__ float w[PRUNE_MAX_K];
  __shared__ float scan[PRUNE_MAX_K];
  __shared__ int iscan[PRUNE_MAX_K];
  __shared__ int cut;
  __shared__ unsigned int kmax;
  const int k = threadIdx.x;
  if (k == 0) { cut = 0; kmax = 0u; }
  if (k < K) w[k] = alpha * wa[k] * wb[k];
  __syncthreads();
  int rank = 0;
  if (k < K) {
    const float wk = w[k];
    for (int j = 0; j < K; ++j) {
      const float wj = w[j];
      rank += (wj < wk || (wj == wk && j < k)) ? 1 : 0;
    }
    scan[rank] = wk;
  }
  __syncthreads();
  // inclusive prefix sums of the ascending weights
  for (int off = 1; off < K; off <<= 1) {
    const float add = (k < K && k >= off) ? scan[k - off] : 0.f;
    __syncthreads();
    if (k < K) scan[k] += add;
    __syncthreads();
  }
  // the prefix sums are non-decreasing: cut = how many of them are <= tol
  if (k < K && scan[k] <= tol && (k + 1 == K || scan[k + 1] > tol)) cut = k + 1;
  __syncthreads();
  const int keep = (k < K && rank >= cut) ? 1 : 0;
  if (keep && bmax) atomicMax(&kmax, bmax[k]);
  if (k < PRUNE_MAX_K) iscan[k] = keep;
  __syncthreads();
  for (int off = 1; off < K; off <<= 1) {
    const int add = (k < K && k >= off) ? iscan[k - off] : 0;
    __syncthreads();
    if (k < K) iscan[k] += add;
    __syncthreads();
  }
  if (keep) cols[iscan[k] - 1] = k;
  if (k == 0) {
    const int n = K > 0 ? iscan[K - 1] : 0;
    const int nkb = n > 0 ? (n + 63) / 64 : 1;
    meta[0] = n;
    meta[1] = nkb;
    meta[2] = nkb * 64;
    meta[3] = cut;
    if (gmax_b) *gmax_b = kmax;
  }
}

int launch_prune_select(const OperandView& va, const int* a_bits, int a_nbits, int64_t a_row0, int64_t a_rows,
                        const OperandView& vb, const int* b_bits, int b_nbits, int64_t b_rows, float alpha,
                        double tol, float* colw, int* cols, int* meta, unsigned int* gmax_b, cudaStream_t st) {
  const int64_t K = va.kdim();
  if (K > PRUNE_MAX_K) return set_error(CUTQC_EUNSUPPORTED, "cut-term pruning needs K <= %d", PRUNE_MAX_K);
  // colw: [K] sums of A, [K] sums of B, [K] maxima of B
  unsigned int* bmax = reinterpret_cast<unsigned int*>(colw + 2 * K);
  CUTQC_CUDA_TRY(cudaMemsetAsync(colw, 0, 3 * K * sizeof(float), st));
  auto one = [&](const OperandView& v, const int* bits, int nbits, int64_t row0, int64_t rows, float* out,
                 unsigned int* omax) -> int {
    if (rows <= 0) return CUTQC_OK;
    RowMap rm{};
    rm.n = nbits;
    for (int j = 0; j < nbits; ++j) {
      rm.bit[j] = (int8_t)bits[j];
      if (bits[j] != j) rm.permute = 1;
    }
    int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((rows * 32 + 255) / 256, (int64_t)sm_count() * 8));
    const size_t smem = 2 * (size_t)K * sizeof(float);
    if (K <= 256) {
      // one wave of grid-stride CTAs (a partial second wave would idle SMs)
      int resident = 0;
      CUTQC_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&resident, colw_kernel<8>, 256, smem));
      blocks = std::min(blocks, sm_count() * std::max(1, resident));
    }
    if (K <= 256) colw_kernel<8><<<blocks, 256, smem, st>>>(v, rm, row0, rows, K, out, omax);
    else colw_kernel<32><<<blocks, 256, smem, st>>>(v, rm, row0, rows, K, out, omax);
    CUTQC_LAUNCH_CHECK("colw_kernel");
    return CUTQC_OK;
  };
  int rc = one(va, a_bits, a_nbits, a_row0, a_rows, colw, nullptr);
  if (!rc) rc = one(vb, b_bits, b_nbits, 0, b_rows, colw + K, bmax);
  if (rc) return rc;
  // float prefix sums: a margin keeps the exact total of the dropped bounds <= tol
  prune_select_kernel<<<1, 1024, 0, st>>>(colw, colw + K, bmax, (int)K, alpha, (float)(tol * (1.0 - 1e-5)), cols, meta,
                                          gmax_b);
  CUTQC_LAUNCH_CHECK("prune_select_kernel");
  return CUTQC_OK;
}

constexpr int64_t PREP_TR_MAX_K = 1024;   // staged tile [K][33] floats: 132 KiB at most

bool prep_covers_source(const OperandView& v, int64_t row0, int64_t rows) {
  return row0 == 0 && rows == v.rows() && v.n_open + v.n_shared == v.k && ((uintptr_t)v.src & 15) == 0;
}

int launch_prep_rows(const OperandView& v, const int* row_bits, int n_bits, int64_t row0, int64_t rows,
                     int64_t Kp, float* out32, __half* hi, __half* lo, float* scale, cudaStream_t st,
                     int batch, int64_t src_bstride, unsigned int* gmax, const int* cols, const int* meta,
                     bool gmax_ready) {
  if (rows <= 0) return CUTQC_OK;
  RowMap rm{};
  rm.n = n_bits;
  rm.permute = 0;
  if (n_bits > (int)sizeof(rm.bit)) return set_error(CUTQC_EUNSUPPORTED, "too many row bits");
  for (int j = 0; j < n_bits; ++j) {
    rm.bit[j] = (int8_t)row_bits[j];
    if (row_bits[j] != j) rm.permute = 1;
  }
  const int64_t K = v.kdim();
  int blocks = (int)std::min<int64_t>((rows * 32 + 255) / 256, (int64_t)sm_count() * 16);
  // the max pass of an operand-wide scale: when the operand is its whole
  // source tensor (all rows, no column list) a plain reduction over the
  // tensor's floats gives the same max
  const bool whole = !cols && prep_covers_source(v, row0, rows);
  if (gmax_ready && (!gmax || !whole)) return set_error(CUTQC_EINVAL, "internal: a ready max needs the whole tensor");
  // *gmax = max |x| of the operand: nothing when the producer already wrote
  // it, else zeroed and reduced over the whole source tensor when the operand
  // covers it, else by the view's own max pass (view_max)
  auto max_pass = [&](auto&& view_max) -> int {
    if (gmax_ready) return CUTQC_OK;
    CUTQC_CUDA_TRY(cudaMemsetAsync(gmax, 0, sizeof(unsigned int), st));
    if (whole) {
      const int64_t n = ((int64_t)1 << v.o) << (2 * v.k);
      const int ab = (int)std::max<int64_t>(1, std::min<int64_t>((n / 4 + 1023) / 1024, (int64_t)sm_count() * 8));
      absmax_kernel<<<ab, 256, 0, st>>>(v.src, n, gmax);
      CUTQC_LAUNCH_CHECK("absmax_kernel");
      return CUTQC_OK;
    }
    return view_max();
  };
  if (blocks < 1) blocks = 1;
  if (batch < 1 || batch > 65535) return set_error(CUTQC_EUNSUPPORTED, "batch %d out of range", batch);
  const bool low_open = v.open_dmask == (((uint64_t)1 << (2 * v.n_open)) - 1);
  if (!cols && v.n_open >= 3 && low_open && v.n_shared > 0 && K <= PREP_TR_MAX_K && row0 % 32 == 0) {
    // strided rows: transpose through shared memory (prep_tr_kernel)
    static std::mutex mu;
    static std::set<int> done;
    int dev = 0;
    cudaGetDevice(&dev);
    {
      std::lock_guard<std::mutex> lk(mu);
      if (!done.count(dev)) {
        CUTQC_CUDA_TRY(cudaFuncSetAttribute(prep_tr_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            (int)(PREP_TR_MAX_K * 33 * sizeof(float))));
        done.insert(dev);
      }
    }
    const size_t smem = (size_t)K * 33 * sizeof(float);
    const int per_sm = std::max(1, std::min(8, (int)((200 * 1024) / smem)));
    const int tblocks = (int)std::max<int64_t>(1, std::min<int64_t>((rows + 31) / 32, (int64_t)sm_count() * per_sm));
    if (gmax) {
      if (batch != 1) return set_error(CUTQC_EINVAL, "internal: operand-wide scale needs batch 1");
      int rc = max_pass([&]() -> int {
        prep_tr_kernel<<<dim3(tblocks, 1), 256, 0, st>>>(v, rm, row0, rows, K, Kp, out32, hi, lo, scale, src_bstride,
                                                         rows, 2, gmax);
        CUTQC_LAUNCH_CHECK("prep_tr_kernel (max)");
        return CUTQC_OK;
      });
      if (rc) return rc;
      prep_tr_kernel<<<dim3(tblocks, 1), 256, smem, st>>>(v, rm, row0, rows, K, Kp, out32, hi, lo, scale,
                                                          src_bstride, rows, 1, gmax);
    } else {
      prep_tr_kernel<<<dim3(tblocks, batch), 256, smem, st>>>(v, rm, row0, rows, K, Kp, out32, hi, lo, scale,
                                                              src_bstride, rows, 0, nullptr);
    }
    CUTQC_LAUNCH_CHECK("prep_tr_kernel");
    return CUTQC_OK;
  }
  const bool low_shared = v.shared_dmask == (((uint64_t)1 << (2 * v.n_shared)) - 1);
  if (!cols && !out32 && hi && low_shared && K % 4 == 0 && K <= Kp && Kp == 64 &&
      ((uintptr_t)v.src & 15) == 0 && src_bstride % 4 == 0) {
    // (Kp is 64 here: K is a power of four, padded to a multiple of 64)
    constexpr int G = 8, rpb = 256 / G;
    const int sblocks = (int)std::max<int64_t>(1, std::min<int64_t>((rows + rpb - 1) / rpb, (int64_t)sm_count() * 8));
    auto launch = [&](int mode) {
      prep_small_kernel<G><<<dim3(sblocks, mode == 0 ? batch : 1), 256, 0, st>>>(v, rm, row0, rows, K, hi, lo, scale,
                                                                                src_bstride, rows, mode, gmax);
    };
    if (gmax) {
      if (batch != 1) return set_error(CUTQC_EINVAL, "internal: operand-wide scale needs batch 1");
      int rc = max_pass([&]() -> int {
        launch(2);
        CUTQC_LAUNCH_CHECK("prep_small_kernel (max)");
        return CUTQC_OK;
      });
      if (rc) return rc;
      launch(1);
    } else {
      launch(0);
    }
    CUTQC_LAUNCH_CHECK("prep_small_kernel");
    return CUTQC_OK;
  }
  if (!cols && !out32 && hi && low_shared && K == 256 && Kp == 256 && ((uintptr_t)v.src & 15) == 0 &&
      src_bstride % 4 == 0) {
    const int rblocks = (int)std::max<int64_t>(
        1, std::min<int64_t>((rows + 8 * kPrepRows - 1) / (8 * kPrepRows), (int64_t)sm_count() * 8));
    if (gmax) {
      if (batch != 1) return set_error(CUTQC_EINVAL, "internal: operand-wide scale needs batch 1");
      int rc = max_pass([&]() -> int {
        prep_kernel<<<dim3(blocks, 1), 256, 0, st>>>(v, rm, row0, rows, K, Kp, out32, hi, lo, scale, src_bstride,
                                                     rows, 2, gmax, cols, meta);
        CUTQC_LAUNCH_CHECK("prep_kernel (max)");
        return CUTQC_OK;
      });
      if (rc) return rc;
    }
    prep_rows256_kernel<<<dim3(rblocks, gmax ? 1 : batch), 256, 0, st>>>(v, rm, row0, rows, hi, lo, scale,
                                                                         src_bstride, rows, gmax ? 1 : 0, gmax);
    CUTQC_LAUNCH_CHECK("prep_rows256_kernel");
    return CUTQC_OK;
  }
  if (cols && !out32 && hi && low_shared && K == 256 && Kp == 256 && batch == 1 && ((uintptr_t)v.src & 15) == 0) {
    // (with a column list the max over the kept columns is already in *gmax)
    const int rblocks = (int)std::max<int64_t>(
        1, std::min<int64_t>((rows + 8 * kPrepRows - 1) / (8 * kPrepRows), (int64_t)sm_count() * 4));
    prep_rows256_cols_kernel<<<rblocks, 256, 0, st>>>(v, rm, row0, rows, hi, lo, scale, gmax ? 1 : 0, gmax, cols,
                                                      meta);
    CUTQC_LAUNCH_CHECK("prep_rows256_cols_kernel");
    return CUTQC_OK;
  }
  if (gmax) {
    // one scale for the whole operand: max pass, then the split (with a
    // column list the max over the kept columns is already in *gmax)
    if (batch != 1) return set_error(CUTQC_EINVAL, "internal: operand-wide scale needs batch 1");
    if (!cols) {
      int rc = max_pass([&]() -> int {
        prep_kernel<<<dim3(blocks, 1), 256, 0, st>>>(v, rm, row0, rows, K, Kp, out32, hi, lo, scale, src_bstride,
                                                     rows, 2, gmax, cols, meta);
        CUTQC_LAUNCH_CHECK("prep_kernel (max)");
        return CUTQC_OK;
      });
      if (rc) return rc;
    }
    prep_kernel<<<dim3(blocks, 1), 256, 0, st>>>(v, rm, row0, rows, K, Kp, out32, hi, lo, scale, src_bstride, rows, 1,
                                                 gmax, cols, meta);
  } else {
    prep_kernel<<<dim3(blocks, batch), 256, 0, st>>>(v, rm, row0, rows, K, Kp, out32, hi, lo, scale, src_bstride,
                                                     rows, 0, nullptr, cols, meta);
  }
  CUTQC_LAUNCH_CHECK("prep_kernel");
  return CUTQC_OK;
}

// ------------------------------------------------------------ SIMT GEMM
// (tile body in sgemm_tile.cuh)

__global__ void __launch_bounds__(256)
sgemm_kernel(const float* __restrict__ A, int64_t lda, const float* __restrict__ B, int64_t ldb,
             int64_t M, int64_t N, int64_t K, float alpha, uint64_t mask_m, uint64_t mask_n,
             int m_contig_shift, int n_contig, float* __restrict__ out, double* __restrict__ sum,
             int streaming, int64_t a_bstride, int64_t b_bstride, int64_t out_bstride) {
  // batch item blockIdx.z
  const DenseRows la{A + (int64_t)blockIdx.z * a_bstride, lda};
  const DenseRows lb{B + (int64_t)blockIdx.z * b_bstride, ldb};
  sgemm_tile(la, lb, M, N, K, alpha, mask_m, mask_n, m_contig_shift, n_contig,
             out + (int64_t)blockIdx.z * out_bstride, sum ? sum + blockIdx.z : nullptr, streaming, blockIdx.y,
             blockIdx.x);
}

int launch_sgemm(const float* A, int64_t lda, const float* B, int64_t ldb, int64_t M, int64_t N,
                 int64_t K, float alpha, uint64_t mask_m, uint64_t mask_n, float* out, double* sum,
                 int streaming, cudaStream_t st, int batch, int64_t a_bstride, int64_t b_bstride,
                 int64_t out_bstride) {
  if (M <= 0 || N <= 0) return CUTQC_OK;
  int64_t gm = (M + SG_BM - 1) / SG_BM, gn = (N + SG_BN - 1) / SG_BN;
  if (gm > 65535) return set_error(CUTQC_EUNSUPPORTED, "too many row tiles (%lld)", (long long)gm);
  if (gn > 0x7fffffff) return set_error(CUTQC_EUNSUPPORTED, "too many column tiles");
  int n_contig = mask_is_low(mask_n);
  int m_shift = mask_contig_shift(mask_m);
  if (batch < 1 || batch > 65535) return set_error(CUTQC_EUNSUPPORTED, "batch %d out of range", batch);
  sgemm_kernel<<<dim3((unsigned)gn, (unsigned)gm, (unsigned)batch), 256, 0, st>>>(
      A, lda, B, ldb, M, N, K, alpha, mask_m, mask_n, m_shift, n_contig, out, sum, streaming, a_bstride, b_bstride,
      out_bstride);
  CUTQC_LAUNCH_CHECK("sgemm_kernel");
  return CUTQC_OK;
}

}  // namespace cutqc
