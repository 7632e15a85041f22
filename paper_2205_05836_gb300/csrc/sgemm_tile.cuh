// The float32 CUDA-core GEMM tile with the bit-deposit epilogue, shared by
// the stand-alone GEMM launch (contract.cu) and the persistent DD kernel
// (dd_persist.cu).
//   C[m][n] = alpha * sum_s A[m][s] B[n][s]
// CTA tile 128 x 128, BK = 16, 256 threads, 8 x 8 outputs per thread split
// in two 4-wide column groups (tx*4 and 64 + tx*4) and two 4-high row groups.
// Operands come through loaders: `row(m)` resolves row m once per tile and
// `at(row, s)` reads element s of it, so that a gathered operand (bit-moved
// rows, digit-scattered columns) costs no staging copy.
#pragma once

#include "internal.cuh"

namespace cutqc {

constexpr int SG_BM = 128, SG_BN = 128, SG_BK = 16;

__device__ __forceinline__ void store_out(float* out, uint64_t idx, float v, int streaming) {
  if (streaming) __stcs(out + idx, v);
  else out[idx] = v;
}

// Row-major, K-contiguous operand: element (m, s) at p[m * ld + s], read
// through the read-only path (for data no launch writes while it runs).
struct DenseRows {
  const float* p;
  int64_t ld;
  typedef const float* Row;
  __device__ __forceinline__ Row row(int64_t m) const { return p + m * ld; }
  __device__ __forceinline__ float at(Row r, int64_t s) const { return __ldg(r + s); }
};

// One output tile (tile_m, tile_n) of one GEMM; out, sum and the loaders
// already point at the batch item.  Every thread of the CTA calls it.
template <class LA, class LB>
__device__ __forceinline__ void sgemm_tile(const LA& la, const LB& lb, int64_t M, int64_t N, int64_t K,
                                           float alpha, uint64_t mask_m, uint64_t mask_n, int m_contig_shift,
                                           int n_contig, float* __restrict__ out, double* __restrict__ sum,
                                           int streaming, int64_t tile_m, int64_t tile_n) {
  __shared__ __align__(16) float As[2][SG_BK][SG_BM + 4];
  __shared__ __align__(16) float Bs[2][SG_BK][SG_BN + 4];
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const int64_t m0 = tile_m * SG_BM;
  const int64_t n0 = tile_n * SG_BN;
  // global load mapping: each thread loads 8 values of A and 8 of B per k-tile
  // (rows lr and lr + 64, k columns lk*4 .. +3)
  const int lr = tid >> 2, lk = (tid & 3) * 4;
  float acc[8][8];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;

  // the two rows of A and of B this thread loads, resolved once per tile
  typename LA::Row arow[2];
  typename LB::Row brow[2];
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int64_t mr = m0 + lr + 64 * h, nr = n0 + lr + 64 * h;
    arow[h] = la.row(mr < M ? mr : 0);
    brow[h] = lb.row(nr < N ? nr : 0);
  }
  float ra[8], rb[8];
  auto gload = [&](int64_t k0) {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      int64_t mr = m0 + lr + 64 * h, nr = n0 + lr + 64 * h;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        int64_t kk = k0 + lk + q;
        ra[h * 4 + q] = (mr < M && kk < K) ? la.at(arow[h], kk) : 0.f;
        rb[h * 4 + q] = (nr < N && kk < K) ? lb.at(brow[h], kk) : 0.f;
      }
    }
  };
  auto sstore = [&](int buf) {
#pragma unroll
    for (int h = 0; h < 2; ++h)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        As[buf][lk + q][lr + 64 * h] = ra[h * 4 + q];
        Bs[buf][lk + q][lr + 64 * h] = rb[h * 4 + q];
      }
  };
  const int64_t nk = (K + SG_BK - 1) / SG_BK;
  gload(0);
  sstore(0);
  __syncthreads();
  for (int64_t kt = 0; kt < nk; ++kt) {
    const int buf = kt & 1;
    if (kt + 1 < nk) gload((kt + 1) * SG_BK);
#pragma unroll
    for (int k = 0; k < SG_BK; ++k) {
      float4 a0 = *reinterpret_cast<const float4*>(&As[buf][k][ty * 4]);
      float4 a1 = *reinterpret_cast<const float4*>(&As[buf][k][64 + ty * 4]);
      float4 b0 = *reinterpret_cast<const float4*>(&Bs[buf][k][tx * 4]);
      float4 b1 = *reinterpret_cast<const float4*>(&Bs[buf][k][64 + tx * 4]);
      float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
      float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
    }
    if (kt + 1 < nk) sstore(buf ^ 1);
    __syncthreads();
  }
  // epilogue
  double local = 0.0;
  uint64_t coff[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    int64_t n = n0 + (j < 4 ? tx * 4 + j : 64 + tx * 4 + (j - 4));
    coff[j] = n_contig ? (uint64_t)n : pdep64((uint64_t)n, mask_n);
  }
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    int64_t m = m0 + (i < 4 ? ty * 4 + i : 64 + ty * 4 + (i - 4));
    if (m >= M) continue;
    uint64_t roff = m_contig_shift >= 0 ? ((uint64_t)m << m_contig_shift) : pdep64((uint64_t)m, mask_m);
    float part[8];      // pairwise float partial per row of 8, float64 across rows
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      int64_t n = n0 + (j < 4 ? tx * 4 + j : 64 + tx * 4 + (j - 4));
      part[j] = 0.f;
      if (n >= N) continue;
      float v = acc[i][j] * alpha;
      store_out(out, roff | coff[j], v, streaming);
      part[j] = v;
    }
    local += (double)(((part[0] + part[1]) + (part[2] + part[3])) + ((part[4] + part[5]) + (part[6] + part[7])));
  }
  if (sum) {
    for (int off = 16; off; off >>= 1) local += __shfl_xor_sync(0xffffffffu, local, off);
    if ((tid & 31) == 0) atomicAdd(sum, local);
  }
}

// A 64 x 64 output tile for small GEMMs (many short contractions, where one
// 128 x 128 tile's serial k loop is the critical path): 256 threads, 4 x 4
// outputs per thread, k in chunks of 32 (eight values of A and of B per
// thread and chunk, issued together; thread (r, l) loads row r, columns
// l, l + 4, ...).  Every output is the same fmaf chain over k ascending as in
// sgemm_tile (zero padding past K leaves it unchanged: it never holds -0), so
// the two tiles give identical outputs; only the float64 sum is grouped
// differently.
constexpr int SG64_BM = 64, SG64_BN = 64, SG64_BK = 32;

// A 256 x 16 tile for contractions with few columns (N <= 16, where a 64 x 64
// tile would leave most of its outputs out of range): k in chunks of 16,
// thread t stages row t of A and element t of B's 16 x 16 chunk, and
// computes rows 4 (t >> 2) .. + 3, columns 4 (t & 3) .. + 3.  Same fmaf
// chains, so the same outputs as the other tiles.
constexpr int SGN_BM = 256, SGN_BN = 16, SGN_BK = 16;

// The tiles' staging arrays (one per block, shared by every instantiation).
// Row pitch 72 in the 64 x 64 tile: the stores of a warp (8 rows x 4 k
// columns) hit 32 banks.
struct TileSmem {
  union {
    struct {
      __align__(16) float A[SG64_BK][SG64_BM + 8];
      __align__(16) float B[SG64_BK][SG64_BN + 8];
    } sq;
    struct {
      __align__(16) float A[SGN_BK][SGN_BM + 4];
      __align__(16) float B[SGN_BK][SGN_BN + 4];
    } narrow;
  };
};

template <class LA, class LB>
__device__ __forceinline__ void sgemm_tile64(const LA& la, const LB& lb, int64_t M, int64_t N, int64_t K,
                                             float alpha, uint64_t mask_m, uint64_t mask_n, int m_contig_shift,
                                             int n_contig, float* __restrict__ out, double* __restrict__ sum,
                                             int streaming, int64_t tile_m, int64_t tile_n, TileSmem& sm) {
  auto& As = sm.sq.A;
  auto& Bs = sm.sq.B;
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const int64_t m0 = tile_m * SG64_BM;
  const int64_t n0 = tile_n * SG64_BN;
  const int lr = tid >> 2, lk = tid & 3;
  float acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
  const int64_t mr = m0 + lr, nr = n0 + lr;
  const typename LA::Row arow = la.row(mr < M ? mr : 0);
  const typename LB::Row brow = lb.row(nr < N ? nr : 0);
  float ra[8], rb[8];
  auto gload = [&](int64_t k0) {
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int64_t kk = k0 + lk + 4 * q;
      ra[q] = (mr < M && kk < K) ? la.at(arow, kk) : 0.f;
      rb[q] = (nr < N && kk < K) ? lb.at(brow, kk) : 0.f;
    }
  };
  auto sstore = [&]() {
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      As[lk + 4 * q][lr] = ra[q];
      Bs[lk + 4 * q][lr] = rb[q];
    }
  };
  const int64_t nk = (K + SG64_BK - 1) / SG64_BK;
  gload(0);
  sstore();
  __syncthreads();
  for (int64_t kt = 0; kt < nk; ++kt) {
    if (kt + 1 < nk) gload((kt + 1) * SG64_BK);
#pragma unroll
    for (int k = 0; k < SG64_BK; ++k) {
      const float4 a = *reinterpret_cast<const float4*>(&As[k][ty * 4]);
      const float4 b = *reinterpret_cast<const float4*>(&Bs[k][tx * 4]);
      const float av[4] = {a.x, a.y, a.z, a.w};
      const float bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
    }
    __syncthreads();
    if (kt + 1 < nk) {
      sstore();
      __syncthreads();
    }
  }
  double local = 0.0;
  uint64_t coff[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int64_t n = n0 + tx * 4 + j;
    coff[j] = n_contig ? (uint64_t)n : pdep64((uint64_t)n, mask_n);
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int64_t m = m0 + ty * 4 + i;
    if (m >= M) continue;
    const uint64_t roff = m_contig_shift >= 0 ? ((uint64_t)m << m_contig_shift) : pdep64((uint64_t)m, mask_m);
    float part[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int64_t n = n0 + tx * 4 + j;
      part[j] = 0.f;
      if (n >= N) continue;
      const float v = acc[i][j] * alpha;
      store_out(out, roff | coff[j], v, streaming);
      part[j] = v;
    }
    local += (double)((part[0] + part[1]) + (part[2] + part[3]));
  }
  if (sum) {
    for (int off = 16; off; off >>= 1) local += __shfl_xor_sync(0xffffffffu, local, off);
    if ((tid & 31) == 0) atomicAdd(sum, local);
  }
}

template <class LA, class LB>
__device__ __forceinline__ void sgemm_tile_narrow(const LA& la, const LB& lb, int64_t M, int64_t N, int64_t K,
                                                  float alpha, uint64_t mask_m, uint64_t mask_n, int m_contig_shift,
                                                  int n_contig, float* __restrict__ out, double* __restrict__ sum,
                                                  int streaming, int64_t tile_m, int64_t tile_n, TileSmem& sm) {
  auto& As = sm.narrow.A;
  auto& Bs = sm.narrow.B;
  const int tid = threadIdx.x;
  const int tx = tid & 3, ty = tid >> 2;
  const int64_t m0 = tile_m * SGN_BM;
  const int64_t n0 = tile_n * SGN_BN;
  float acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
  const int64_t mr = m0 + tid;                       // the A row this thread stages
  const int64_t nr = n0 + (tid >> 4), kb = tid & 15;   // the B element this thread stages
  const typename LA::Row arow = la.row(mr < M ? mr : 0);
  const typename LB::Row brow = lb.row(nr < N ? nr : 0);
  float ra[SGN_BK], rb;
  auto gload = [&](int64_t k0) {
#pragma unroll
    for (int q = 0; q < SGN_BK; ++q) ra[q] = (mr < M && k0 + q < K) ? la.at(arow, k0 + q) : 0.f;
    rb = (nr < N && k0 + kb < K) ? lb.at(brow, k0 + kb) : 0.f;
  };
  auto sstore = [&]() {
#pragma unroll
    for (int q = 0; q < SGN_BK; ++q) As[q][tid] = ra[q];
    Bs[kb][tid >> 4] = rb;
  };
  const int64_t nk = (K + SGN_BK - 1) / SGN_BK;
  gload(0);
  sstore();
  __syncthreads();
  for (int64_t kt = 0; kt < nk; ++kt) {
    if (kt + 1 < nk) gload((kt + 1) * SGN_BK);
#pragma unroll
    for (int k = 0; k < SGN_BK; ++k) {
      const float4 a = *reinterpret_cast<const float4*>(&As[k][ty * 4]);
      const float4 b = *reinterpret_cast<const float4*>(&Bs[k][tx * 4]);
      const float av[4] = {a.x, a.y, a.z, a.w};
      const float bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
    }
    __syncthreads();
    if (kt + 1 < nk) {
      sstore();
      __syncthreads();
    }
  }
  double local = 0.0;
  uint64_t coff[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int64_t n = n0 + tx * 4 + j;
    coff[j] = n_contig ? (uint64_t)n : pdep64((uint64_t)n, mask_n);
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int64_t m = m0 + ty * 4 + i;
    if (m >= M) continue;
    const uint64_t roff = m_contig_shift >= 0 ? ((uint64_t)m << m_contig_shift) : pdep64((uint64_t)m, mask_m);
    float part[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int64_t n = n0 + tx * 4 + j;
      part[j] = 0.f;
      if (n >= N) continue;
      const float v = acc[i][j] * alpha;
      store_out(out, roff | coff[j], v, streaming);
      part[j] = v;
    }
    local += (double)((part[0] + part[1]) + (part[2] + part[3]));
  }
  if (sum) {
    for (int off = 16; off; off >>= 1) local += __shfl_xor_sync(0xffffffffu, local, off);
    if ((tid & 31) == 0) atomicAdd(sum, local);
  }
}

}  // namespace cutqc
