// K1: attribution.  Subcircuit variant outputs -> edge-basis tensors.
//
// Circuit Cutting section (Eq. 1): every cut runs over the Pauli bases
// {I,X,Y,Z}; the subcircuit is initialised / measured differently per basis.
// From rho = 1/2 sum_M Tr(rho M) M:
//   initialised cut (state runs |0>,|1>,|+>,|+i>):
//     I = p0 + p1, X = 2p+ - p0 - p1, Y = 2p+i - p0 - p1, Z = p0 - p1
//   measured cut (basis runs computational, X, Y; outcome m):
//     I = sum_m pZ(m), X = sum_m (-1)^m pX(m), Y = sum_m (-1)^m pY(m),
//     Z = sum_m (-1)^m pZ(m)
//
// The map is a tensor product of one small map per cut.  Initialised side
// (attr_init_pass): a CTA owns R consecutive outcome rows and one measurement
// run, stages the fiber of the init digits for its rows in shared memory
// (loads coalesced along the outcome index) and applies the per-cut maps
// axis by axis.  Measured side (attr_meas_run): a CTA owns one measurement
// run and 128 output rows, each thread takes the Walsh-Hadamard transform of
// its row's 2^k_out outcomes in registers and writes the basis strings that
// run serves; with measured cuts only (attr_meas_grp) a CTA takes the 9 runs
// that fill whole blocks of 16 columns and stores them as 16-byte vectors.
// Subcircuits with both kinds of cut take two passes through a
// float32 workspace: the measured side first, on the variants as given
// (3^k_out runs x 2^k_out outcomes -> 4^k_out bases per output row), then the
// initialised side along the columns of the smaller result
// (attr_init_cols).  Arithmetic is float32 after the (float64 or float32)
// loads; HBM-bound.
#include "internal.cuh"

#include <algorithm>
#include <mutex>
#include <set>
#include <utility>
#include <vector>

namespace cutqc {

namespace {

constexpr int kMaxKin = 6;
constexpr int kMaxKout = 5;
constexpr int kThreads = 512;
constexpr int kBatch = 16;           // loads in flight per thread

struct AttrParams {
  int w, k_in, k_out;
  int64_t n_rows;           // rows handled by the grid (2^w or 2^o)
  int R;                    // rows per CTA
  uint64_t out_mask;        // local-qubit mask of the output qubits
  uint64_t meas_mask[kMaxKout];  // local-qubit bit of each measured cut
  int col_shift_in[kMaxKin];     // 2 * rank of each init cut's edge
  int col_shift_out[kMaxKout];   // 2 * rank of each measured cut's edge
  int k;                    // k_in + k_out
};

__device__ __forceinline__ float load_val(const double* p) { return f64_to_f32_rn(__ldg(p)); }
__device__ __forceinline__ float load_val(const float* p) { return __ldg(p); }
// The conversion alone, for loops that issue all their loads first (a
// conversion between two loads would hold the second back).  Value i of
// such a loop (i known at compile time) converts on the FP64 pipe when even
// and on the integer pipes (f64_to_f32_rn) when odd: on GB300 either alone,
// given every value, bounds these kernels (FP64 pipe 90% busy, or ALU 74%);
// both round to nearest even, so the results are the same.
__device__ __forceinline__ float to_f32(double x, int i) { return (i & 1) ? f64_to_f32_rn(x) : __double2float_rn(x); }
__device__ __forceinline__ float to_f32(float x, int) { return x; }

// 4x4 map of the initialised side: bases I, X, Y, Z from the runs
// |0>, |1>, |+>, |+i> (in registers).
__device__ __forceinline__ void init_map4(const float (&p)[4], float (&o)[4]) {
  const float s01 = p[0] + p[1];
  o[0] = s01;
  o[1] = 2.f * p[2] - s01;
  o[2] = 2.f * p[3] - s01;
  o[3] = p[0] - p[1];
}

// Rows per CTA of the initialised-side pass: as many as fit a 72 KiB padded
// [F][R + 1] block (three CTAs per SM), at most 64 (512-byte runs of float64).
__host__ __device__ constexpr int rows_for(int F) {
  return F * 65 * 4 <= 72 * 1024 ? 64 : F * 33 * 4 <= 72 * 1024 ? 32 : F * 17 * 4 <= 72 * 1024 ? 16
       : F * 9 * 4 <= 72 * 1024 ? 8 : F * 5 * 4 <= 72 * 1024 ? 4 : F * 3 * 4 <= 72 * 1024 ? 2 : 1;
}
__host__ __device__ constexpr int pow3(int k) { return k == 0 ? 1 : 3 * pow3(k - 1); }

// Initialised-side pass (KIN init cuts, compile time).  Fiber over the 4^KIN
// init digits, R consecutive outcome rows x (full w-bit index), fixed
// measurement run index `mrun` (blockIdx.y).  Shared memory holds the fiber
// as [f][R + 1] (padded: row-major and column-major walks are conflict
// free).  Each step takes two digits: a thread loads the 16 values of one
// (digit j, digit j+1) block of one row, applies the 4x4 map along both in
// registers and writes them back.  final_layout: write attributed[x][col]
// (only when k_out == 0); otherwise the [4^k_in][3^k_out][2^w] layout with
// states replaced by bases.
template <typename T, int KIN>
__global__ void __launch_bounds__(kThreads)
attr_init_pass(const T* __restrict__ src, float* __restrict__ dst, AttrParams p, int final_layout) {
  constexpr int F = 1 << (2 * KIN);
  constexpr int R = rows_for(F);
  constexpr int RS = R + 1;
  extern __shared__ float sm[];
  float* buf = sm;                                             // [F][RS]
  unsigned short* cperm = reinterpret_cast<unsigned short*>(buf + F * RS);   // column -> fiber index
  const int64_t x0 = (int64_t)blockIdx.x * R;
  const int mrun = blockIdx.y;
  int nm = 1;
  for (int j = 0; j < p.k_out; ++j) nm *= 3;
  const int64_t W = (int64_t)1 << p.w;
  const int rows = (int)(p.n_rows - x0 < R ? p.n_rows - x0 : R);
  if (final_layout) {
    for (int c = threadIdx.x; c < F; c += kThreads) {
      int f = 0;
#pragma unroll
      for (int j = 0; j < KIN; ++j) f |= ((c >> p.col_shift_in[j]) & 3) << (2 * j);
      cperm[c] = (unsigned short)f;
    }
  }
  const T* base = src + (int64_t)mrun * W + x0;
  const int64_t fstride = (int64_t)nm * W;
  // loads in batches of kBatch per thread (all issued before any store)
  for (int i0 = 0; i0 < F * R; i0 += kThreads * kBatch) {
    T raw[kBatch];
#pragma unroll
    for (int u = 0; u < kBatch; ++u) {
      const int i = i0 + u * kThreads + threadIdx.x;
      const int f = i / R, r = i % R;
      raw[u] = (i < F * R && r < rows) ? __ldg(base + f * fstride + r) : T(0);
    }
#pragma unroll
    for (int u = 0; u < kBatch; ++u) {
      const int i = i0 + u * kThreads + threadIdx.x;
      if (i < F * R) buf[(i / R) * RS + i % R] = to_f32(raw[u], u);
    }
  }
  __syncthreads();
#pragma unroll
  for (int j = 0; j < KIN; j += 2) {
    if (j + 1 < KIN) {
      const int groups = F >> 4;
      for (int it = threadIdx.x; it < groups * R; it += kThreads) {
        const int r = it % R, grp = it / R;
        const int lowmask = (1 << (2 * j)) - 1;
        const int base_f = (grp & lowmask) | ((grp >> (2 * j)) << (2 * j + 4));
        float v[4][4];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int b = 0; b < 4; ++b) v[a][b] = buf[(base_f | (a << (2 * j)) | (b << (2 * j + 2))) * RS + r];
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          float col[4] = {v[0][b], v[1][b], v[2][b], v[3][b]}, o[4];
          init_map4(col, o);
#pragma unroll
          for (int a = 0; a < 4; ++a) v[a][b] = o[a];
        }
#pragma unroll
        for (int a = 0; a < 4; ++a) {
          float o[4];
          init_map4(v[a], o);
#pragma unroll
          for (int b = 0; b < 4; ++b) buf[(base_f | (a << (2 * j)) | (b << (2 * j + 2))) * RS + r] = o[b];
        }
      }
    } else {
      const int groups = F >> 2;
      for (int it = threadIdx.x; it < groups * R; it += kThreads) {
        const int r = it % R, grp = it / R;
        const int lowmask = (1 << (2 * j)) - 1;
        const int base_f = (grp & lowmask) | ((grp >> (2 * j)) << (2 * j + 2));
        float v[4], o[4];
#pragma unroll
        for (int a = 0; a < 4; ++a) v[a] = buf[(base_f | (a << (2 * j))) * RS + r];
        init_map4(v, o);
#pragma unroll
        for (int a = 0; a < 4; ++a) buf[(base_f | (a << (2 * j))) * RS + r] = o[a];
      }
    }
    __syncthreads();
  }
  if (final_layout) {
    // attributed[x][col], c fastest: coalesced along the row
    float* out = dst + x0 * F;
#pragma unroll 4
    for (int i = threadIdx.x; i < rows * F; i += kThreads) {
      const int r = i / F, c = i % F;
      out[i] = buf[cperm[c] * RS + r];
    }
  } else {
    float* out = dst + (int64_t)mrun * W + x0;
#pragma unroll 4
    for (int i = threadIdx.x; i < F * R; i += kThreads) {
      const int f = i / R, r = i % R;
      if (r < rows) out[f * fstride + r] = buf[f * RS + r];
    }
  }
}

// Initialised-side map for subcircuits with both kinds of cut.  The
// measured-side pass left W[s][mu][x] in the workspace (s: the init cuts'
// states |0>, |1>, |+>, |+i> as digits, mu: the measured cuts' bases as
// digits, x: output row, dense).  Every fiber W[.][mu][x] over the 4^KIN states is
// mapped to bases by the per-cut 4x4 map (init_map4), digit pair by digit
// pair, and written to the attributed layout A[x][col], col holding each
// cut's digit at its edge's rank.  A CTA takes P consecutive (x, mu) and all
// states: loads are runs of P floats, fibers sit in shared memory as
// [P][F + 1] (conflict-free both ways), and stores walk the fiber fastest
// when an init digit holds column bit 0 (ifast), else the (x, mu) index.
constexpr int kColThreads = 256;
// Fibers per CTA: 8192 values (32 KiB) per CTA, runs of 128 bytes per state
// at F = 256.  (16 KiB blocks, twice the CTAs, measured the same.)
__host__ __device__ constexpr int cols_fibers(int F) { return F >= 4096 ? 1 : (8192 / F > 64 ? 64 : 8192 / F); }

template <int KIN>
__global__ void __launch_bounds__(kColThreads)
attr_init_cols(const float* __restrict__ src, float* __restrict__ dst, AttrParams p, int64_t n_fibers, int ifast) {
  constexpr int F = 1 << (2 * KIN);
  constexpr int P = cols_fibers(F);
  constexpr int FS = F + 1;
  constexpr int LB = 16;                                                // loads in flight per thread
  __shared__ float buf[P * FS];
  __shared__ int64_t fbase[P];
  __shared__ int ioff[F];
  const int64_t C = (int64_t)1 << (2 * p.k);
  for (int i = threadIdx.x; i < F; i += kColThreads) {
    int off = 0;
#pragma unroll
    for (int j = 0; j < KIN; ++j) off |= ((i >> (2 * j)) & 3) << p.col_shift_in[j];
    ioff[i] = off;
  }
  const int64_t nblk = (n_fibers + P - 1) / P;
  for (int64_t blk = blockIdx.x; blk < nblk; blk += gridDim.x) {
    const int64_t f0 = blk * P;
    __syncthreads();          // the previous block's stores have read buf and fbase
    for (int i = threadIdx.x; i < P; i += kColThreads) {
      const int64_t f = f0 + i;           // fiber = g * 2^o + x
      const int64_t x = f % p.n_rows;
      const int mu = (int)(f / p.n_rows);
      int moff = 0;
      for (int j = 0; j < p.k_out; ++j) moff |= ((mu >> (2 * j)) & 3) << p.col_shift_out[j];
      fbase[i] = x * C + moff;
    }
    // loads: state s, fiber pl (pl fastest: runs of P consecutive floats)
    for (int i0 = 0; i0 < P * F; i0 += kColThreads * LB) {
      float v[LB];
#pragma unroll
      for (int u = 0; u < LB; ++u) {
        const int i = i0 + u * kColThreads + threadIdx.x;
        const int sidx = i / P, pl = i % P;
        v[u] = (i < P * F && f0 + pl < n_fibers) ? __ldg(src + (int64_t)sidx * n_fibers + f0 + pl) : 0.f;
      }
#pragma unroll
      for (int u = 0; u < LB; ++u) {
        const int i = i0 + u * kColThreads + threadIdx.x;
        if (i < P * F) buf[(i % P) * FS + i / P] = v[u];
      }
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < KIN; j += 2) {
      if (j + 1 < KIN) {
        constexpr int groups = F >= 16 ? F >> 4 : 1;      // (this branch needs KIN >= 2)
        for (int it = threadIdx.x; it < groups * P; it += kColThreads) {
          const int fl = it % P, grp = it / P;   // lanes over fibers: rows FS apart, distinct banks
          const int lowmask = (1 << (2 * j)) - 1;
          const int base_f = (grp & lowmask) | ((grp >> (2 * j)) << (2 * j + 4));
          float* fb = buf + fl * FS;
          float v[4][4];
#pragma unroll
          for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) v[a][b] = fb[base_f | (a << (2 * j)) | (b << (2 * j + 2))];
#pragma unroll
          for (int b = 0; b < 4; ++b) {
            float col[4] = {v[0][b], v[1][b], v[2][b], v[3][b]}, o[4];
            init_map4(col, o);
#pragma unroll
            for (int a = 0; a < 4; ++a) v[a][b] = o[a];
          }
#pragma unroll
          for (int a = 0; a < 4; ++a) {
            float o[4];
            init_map4(v[a], o);
#pragma unroll
            for (int b = 0; b < 4; ++b) fb[base_f | (a << (2 * j)) | (b << (2 * j + 2))] = o[b];
          }
        }
      } else {
        constexpr int groups = F >> 2;
        for (int it = threadIdx.x; it < groups * P; it += kColThreads) {
          const int fl = it % P, grp = it / P;   // lanes over fibers: rows FS apart, distinct banks
          const int lowmask = (1 << (2 * j)) - 1;
          const int base_f = (grp & lowmask) | ((grp >> (2 * j)) << (2 * j + 2));
          float* fb = buf + fl * FS;
          float v[4], o[4];
#pragma unroll
          for (int a = 0; a < 4; ++a) v[a] = fb[base_f | (a << (2 * j))];
          init_map4(v, o);
#pragma unroll
          for (int a = 0; a < 4; ++a) fb[base_f | (a << (2 * j))] = o[a];
        }
      }
      __syncthreads();
    }
    for (int i = threadIdx.x; i < P * F; i += kColThreads) {
      int fl, io;
      if (ifast) { fl = i / F; io = i % F; } else { io = i / P; fl = i % P; }
      if (f0 + fl < n_fibers) dst[fbase[fl] + ioff[io]] = buf[fl * FS + io];
    }
  }
}

template <typename T, int KIN>
size_t init_smem() { return (size_t)(1 << (2 * KIN)) * (rows_for(1 << (2 * KIN)) + 1) * 4 + (2u << (2 * KIN)); }

// k == 0: plain conversion to float32.
template <typename T>
__global__ void attr_copy(const T* __restrict__ src, float* __restrict__ dst, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = load_val(src + i);
}

int validate_sub(const cutqc_subcircuit* s) {
  if (!s) return set_error(CUTQC_EINVAL, "null subcircuit");
  if (s->w < 1 || s->w > CUTQC_MAX_WIDTH) return set_error(CUTQC_EINVAL, "width %d out of range", s->w);
  if (s->k_in < 0 || s->k_out < 0 || s->k_in > s->w || s->k_out > s->w)
    return set_error(CUTQC_EINVAL, "bad cut counts k_in=%d k_out=%d", s->k_in, s->k_out);
  if ((s->k_in && (!s->in_local || !s->in_edge)) || (s->k_out && (!s->out_local || !s->out_edge)))
    return set_error(CUTQC_EINVAL, "missing cut arrays");
  for (int j = 0; j < s->k_in; ++j) {
    if (s->in_local[j] < 0 || s->in_local[j] >= s->w || (j && s->in_local[j] <= s->in_local[j - 1]))
      return set_error(CUTQC_EINVAL, "in_local must be strictly ascending in [0,w)");
    if (s->in_edge[j] < 0) return set_error(CUTQC_EINVAL, "negative edge id");
  }
  for (int j = 0; j < s->k_out; ++j) {
    if (s->out_local[j] < 0 || s->out_local[j] >= s->w || (j && s->out_local[j] <= s->out_local[j - 1]))
      return set_error(CUTQC_EINVAL, "out_local must be strictly ascending in [0,w)");
    if (s->out_edge[j] < 0) return set_error(CUTQC_EINVAL, "negative edge id");
  }
  std::vector<int> e;
  for (int j = 0; j < s->k_in; ++j) e.push_back(s->in_edge[j]);
  for (int j = 0; j < s->k_out; ++j) e.push_back(s->out_edge[j]);
  std::sort(e.begin(), e.end());
  for (size_t i = 1; i < e.size(); ++i)
    if (e[i] == e[i - 1]) return set_error(CUTQC_EINVAL, "edge %d appears twice in one subcircuit", e[i]);
  return CUTQC_OK;
}

void fill_params(const cutqc_subcircuit* s, AttrParams* p) {
  p->w = s->w;
  p->k_in = s->k_in;
  p->k_out = s->k_out;
  p->k = s->k_in + s->k_out;
  uint64_t meas = 0;
  for (int j = 0; j < s->k_out; ++j) {
    p->meas_mask[j] = (uint64_t)1 << s->out_local[j];
    meas |= p->meas_mask[j];
  }
  p->out_mask = (((uint64_t)1 << s->w) - 1) & ~meas;
  std::vector<int> e;
  for (int j = 0; j < s->k_in; ++j) e.push_back(s->in_edge[j]);
  for (int j = 0; j < s->k_out; ++j) e.push_back(s->out_edge[j]);
  std::sort(e.begin(), e.end());
  auto rank = [&](int id) { return (int)(std::lower_bound(e.begin(), e.end(), id) - e.begin()); };
  for (int j = 0; j < s->k_in; ++j) p->col_shift_in[j] = 2 * rank(s->in_edge[j]);
  for (int j = 0; j < s->k_out; ++j) p->col_shift_out[j] = 2 * rank(s->out_edge[j]);
}

// Opt a kernel in to the largest dynamic shared memory the passes use, once
// per kernel and device.
constexpr int kAttrMaxSmem = 110 * 1024;
cudaError_t set_max_smem(const void* fn) {
  static std::mutex mu;
  static std::set<std::pair<const void*, int>> done;
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lk(mu);
  if (done.count({fn, dev})) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, kAttrMaxSmem);
  if (e == cudaSuccess) done.insert({fn, dev});
  return e;
}


template <typename T, int KIN>
int run_init(const T* src, float* out, const AttrParams& p, int final_layout, cudaStream_t st) {
  constexpr int F = 1 << (2 * KIN);
  constexpr int R = rows_for(F);
  const size_t smem = init_smem<T, KIN>();
  int nm = 1;
  for (int j = 0; j < p.k_out; ++j) nm *= 3;
  dim3 grid((unsigned)((p.n_rows + R - 1) / R), nm);
  CUTQC_CUDA_TRY(set_max_smem((const void*)attr_init_pass<T, KIN>));
  attr_init_pass<T, KIN><<<grid, kThreads, smem, st>>>(src, out, p, final_layout);
  CUTQC_LAUNCH_CHECK("attr_init_pass");
  return CUTQC_OK;
}


template <typename T>
int dispatch_init(const T* src, float* out, const AttrParams& p, int final_layout, cudaStream_t st) {
  switch (p.k_in) {
    case 1: return run_init<T, 1>(src, out, p, final_layout, st);
    case 2: return run_init<T, 2>(src, out, p, final_layout, st);
    case 3: return run_init<T, 3>(src, out, p, final_layout, st);
    case 4: return run_init<T, 4>(src, out, p, final_layout, st);
    case 5: return run_init<T, 5>(src, out, p, final_layout, st);
    case 6: return run_init<T, 6>(src, out, p, final_layout, st);
  }
  return set_error(CUTQC_EUNSUPPORTED, "k_in = %d", p.k_in);
}

template <int KIN>
int run_init_cols(const float* src, float* out, const AttrParams& p, cudaStream_t st) {
  constexpr int F = 1 << (2 * KIN);
  constexpr int P = cols_fibers(F);
  const int64_t n_fibers = p.n_rows << (2 * p.k_out);
  int ifast = 0;
  for (int j = 0; j < p.k_in; ++j) ifast |= p.col_shift_in[j] == 0;
  const int64_t blocks = (n_fibers + P - 1) / P;
  if (blocks > 0x7fffffffLL) return set_error(CUTQC_EUNSUPPORTED, "attribution tensor too large");
  const int64_t grid = blocks;
  attr_init_cols<KIN><<<(unsigned)grid, kColThreads, 0, st>>>(src, out, p, n_fibers, ifast);
  CUTQC_LAUNCH_CHECK("attr_init_cols");
  return CUTQC_OK;
}

int dispatch_init_cols(const float* src, float* out, const AttrParams& p, cudaStream_t st) {
  switch (p.k_in) {
    case 1: return run_init_cols<1>(src, out, p, st);
    case 2: return run_init_cols<2>(src, out, p, st);
    case 3: return run_init_cols<3>(src, out, p, st);
    case 4: return run_init_cols<4>(src, out, p, st);
    case 5: return run_init_cols<5>(src, out, p, st);
    case 6: return run_init_cols<6>(src, out, p, st);
  }
  return set_error(CUTQC_EUNSUPPORTED, "k_in = %d", p.k_in);
}


// Shared by the two measured-side kernels: the outcome values of output row
// x of one run and their Walsh-Hadamard transform over the outcome bits
// (entry `mask` = sum_b (-1)^popcount(b & mask) V[b]).  The row's offset
// within the run is x with a zero bit inserted at each measured qubit (the
// cut qubits are in ascending order); outcome b adds the bits of its
// measured qubits.  Offsets fit 32 bits (w <= 30).
template <typename T, int KOUT>
__device__ __forceinline__ void load_run_row(const T* run, const AttrParams& p, int x, bool ok,
                                             float (&v)[1 << KOUT]) {
  constexpr int NB = 1 << KOUT;
  int rb = x;
#pragma unroll
  for (int j = 0; j < KOUT; ++j) {
    const int lowm = (int)p.meas_mask[j] - 1;
    rb = ((rb & ~lowm) << 1) | (rb & lowm);
  }
  const T* row = run + rb;
  T raw[NB];
  int bp[NB];
  bp[0] = 0;
#pragma unroll
  for (int j = 0; j < KOUT; ++j) {
    const int mj = (int)p.meas_mask[j];
#pragma unroll
    for (int b = 0; b < (1 << j); ++b) bp[b | (1 << j)] = bp[b] | mj;
  }
#pragma unroll
  for (int b = 0; b < NB; ++b) raw[b] = ok ? __ldg(row + bp[b]) : T(0);
#pragma unroll
  for (int b = 0; b < NB; ++b) v[b] = to_f32(raw[b], b);
#pragma unroll
  for (int h = 1; h < NB; h <<= 1)
#pragma unroll
    for (int i = 0; i < NB; ++i)
      if ((i & h) == 0) {
        const float a = v[i], c = v[i | h];
        v[i] = a + c;
        v[i | h] = a - c;
      }
}

// Measured side of a subcircuit with both kinds of cut, one measurement run
// at a time.  CTA (x block, run m, init state s): each thread loads the
// 2^KOUT outcome values of one output row x of run m (a warp's loads are
// runs of consecutive values when the output qubits are the low local bits),
// takes their Walsh-Hadamard transform in registers, and writes the basis
// strings g whose run is m -- a measured cut's digit is X or Y where the run
// measured in that basis, I or Z where it measured in the computational
// basis -- to W[s][g][x], x fastest (coalesced).  The transform entry of
// each basis string is fixed | z, z the subset of the computational digits
// read as Z; lane i works out where entry i goes (the same for the whole
// CTA) and the warp reads it by shuffle.
constexpr int kRunRows = 128;     // threads per CTA

template <typename T, int KOUT>
__global__ void __launch_bounds__(kRunRows)
attr_meas_run(const T* __restrict__ src, float* __restrict__ dst, AttrParams p, int staged, int64_t n_xb) {
  constexpr int NB = 1 << KOUT;
  constexpr int NM = pow3(KOUT);
  constexpr int G = 1 << (2 * KOUT);
  const int64_t W = (int64_t)1 << p.w;
  // task: x block fastest, then the run, then the init state (consecutive
  // CTAs read neighbouring blocks of the variants)
  const int64_t task = blockIdx.x;
  const int64_t xb = task % n_xb;
  const int m = (int)((task / n_xb) % NM);
  const int s = (int)(task / n_xb / NM);
  const int lane = threadIdx.x & 31;
  const int x = (int)(xb * kRunRows) + threadIdx.x;
  const bool ok = x < p.n_rows;
  float v[NB];
  load_run_row<T, KOUT>(src + ((int64_t)s * NM + m) * W, p, x, ok, v);
  // run m's digits (base 3): 0 computational, 1 X, 2 Y
  int fixed = 0, comp = 0, gx = 0;
#pragma unroll
  for (int j = 0, mm = m; j < KOUT; ++j, mm /= 3) {
    const int md = mm % 3;
    if (md) { fixed |= 1 << j; gx |= md << (2 * j); } else comp |= 1 << j;
  }
  // lane i: the column of entry i in the output (basis string g when staged,
  // the attributed layout's column otherwise), -1 if the run has no entry i
  int my_col = -1;
  if (lane < NB && (lane & fixed) == fixed) {
    const int z = lane & comp;
    int g = gx;
#pragma unroll
    for (int j = 0; j < KOUT; ++j)
      if ((z >> j) & 1) g |= 3 << (2 * j);
    if (staged) {
      my_col = g;
    } else {
      int col = 0;
#pragma unroll
      for (int j = 0; j < KOUT; ++j) col |= ((g >> (2 * j)) & 3) << p.col_shift_out[j];
      my_col = col;
    }
  }
#pragma unroll
  for (int i = 0; i < NB; ++i) {
    const int col = __shfl_sync(0xffffffffu, my_col, i);
    if (col < 0 || !ok) continue;
    if (staged) dst[((int64_t)s * G + col) * p.n_rows + x] = v[i];
    else dst[(int64_t)x * G + col] = v[i];      // no init cut: row x of the attributed layout
  }
}

// Measured side of a subcircuit with measured cuts only, written straight
// into the attributed layout [x][col].  There one run's basis strings are
// scattered over the row (a digit's four bases come from three runs), so a
// CTA takes a group of runs instead: the 3^NG runs over the bases of the NG
// cuts whose digits are the lowest of the column index (NG = 2, or 1 for a
// single cut), with the other cuts' measurement bases fixed.  Those runs
// cover, for each choice of I or Z at the other computational cuts, a block
// of 4^NG consecutive columns.  Warp r of the CTA takes run r of the group
// for kGrpRows consecutive rows (lane = row: the loads and transform of
// attr_meas_run), parks its values in shared memory, and the CTA then
// stores each row's blocks as whole 16-byte vectors.  dst 16-byte aligned.
constexpr int kGrpRows = 32;

template <typename T, int KOUT>
__global__ void __launch_bounds__(32 * (KOUT >= 2 ? 9 : 3))
attr_meas_grp(const T* __restrict__ src, float* __restrict__ dst, AttrParams p, int ja, int jb, int64_t n_xb) {
  constexpr int NB = 1 << KOUT;
  constexpr int NG = KOUT >= 2 ? 2 : 1;
  constexpr int GC = 1 << (2 * NG);           // columns of a block
  constexpr int RS = GC + 1;                  // padded tile row
  constexpr int G = 1 << (2 * KOUT);
  constexpr int SO = 1 << (KOUT - NG);        // most blocks a group writes
  __shared__ float tile[SO * kGrpRows * RS];  // [block][row][column]
  const int64_t W = (int64_t)1 << p.w;
  const int64_t xb = blockIdx.x % n_xb;
  const int key = (int)(blockIdx.x / n_xb);   // base-3 digits of the other cuts, in cut order
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // measurement basis per cut (0 computational, 1 X, 2 Y; two bits per cut
  // in dig): the grouped cuts' from the warp index, the others' from the key
  int dig = 0, m = 0, fixed = 0, comp = 0;
  {
    int kk = key, p3 = 1;
#pragma unroll
    for (int j = 0; j < KOUT; ++j) {
      int d;
      if (j == ja) d = warp % 3;
      else if (NG == 2 && j == jb) d = warp / 3;
      else { d = kk % 3; kk /= 3; }
      dig |= d << (2 * j);
      m += d * p3;
      p3 *= 3;
      if (d) fixed |= 1 << j; else comp |= 1 << j;
    }
  }
  const int x = (int)(xb * kGrpRows) + lane;
  const bool ok = x < p.n_rows;
  float v[NB];
  load_run_row<T, KOUT>(src + (int64_t)m * W, p, x, ok, v);
  // lane i: where entry i = fixed | z goes in the tile (z: Z at those
  // computational cuts, I at the others), -1 if the run has no entry i.  The
  // column within the block comes from the grouped cuts' digits, the block
  // from z's bits at the other computational cuts (in cut order).
  int my_off = -1;
  if (lane < NB && (lane & fixed) == fixed) {
    const int z = lane & comp;
    int cl = 0, sb = 0, nb = 0;
#pragma unroll
    for (int j = 0; j < KOUT; ++j) {
      const int dj = (dig >> (2 * j)) & 3;
      const int d = ((z >> j) & 1) ? 3 : dj;
      if (j == ja) cl |= d;
      else if (NG == 2 && j == jb) cl |= d << 2;
      else if (dj == 0) { sb |= ((z >> j) & 1) << nb; ++nb; }
    }
    my_off = sb * (kGrpRows * RS) + cl;
  }
  float* trow = tile + lane * RS;
#pragma unroll
  for (int i = 0; i < NB; ++i) {
    const int off = __shfl_sync(0xffffffffu, my_off, i);
    if (off >= 0) trow[off] = v[i];
  }
  __syncthreads();
  // blocks of this group: 2^(computational cuts among the others)
  int n_oc = 0;
#pragma unroll
  for (int j = 0; j < KOUT; ++j)
    if (j != ja && !(NG == 2 && j == jb) && ((dig >> (2 * j)) & 3) == 0) ++n_oc;
  constexpr int Q = GC / 4;                   // 16-byte vectors per block row
  const int items = (1 << n_oc) * kGrpRows * Q;
  for (int it = threadIdx.x; it < items; it += blockDim.x) {
    const int q = it % Q, row = (it / Q) % kGrpRows, sb = it / Q / kGrpRows;
    const int64_t xr = xb * kGrpRows + row;
    if (xr >= p.n_rows) continue;
    int col = 0, nb = 0;
#pragma unroll
    for (int j = 0; j < KOUT; ++j) {
      if (j == ja || (NG == 2 && j == jb)) continue;
      int d = (dig >> (2 * j)) & 3;
      if (d == 0) { d = ((sb >> nb) & 1) ? 3 : 0; ++nb; }
      col |= d << p.col_shift_out[j];
    }
    const float* t = tile + (sb * kGrpRows + row) * RS + 4 * q;
    *reinterpret_cast<float4*>(dst + xr * (int64_t)G + col + 4 * q) = make_float4(t[0], t[1], t[2], t[3]);
  }
}

template <typename T, int KOUT>
int run_meas_grp(const T* src, float* out, const AttrParams& p, cudaStream_t st) {
  int ja = -1, jb = -1;
  for (int j = 0; j < KOUT; ++j) {
    if (p.col_shift_out[j] == 0) ja = j;
    if (p.col_shift_out[j] == 2) jb = j;
  }
  if (ja < 0 || (KOUT >= 2 && jb < 0)) return set_error(CUTQC_EINVAL, "internal: measured cuts' columns");
  constexpr int NG = KOUT >= 2 ? 2 : 1;
  const int64_t xb = (p.n_rows + kGrpRows - 1) / kGrpRows;
  const int64_t ntask = xb * pow3(KOUT - NG);
  if (ntask > 0x7fffffffLL) return set_error(CUTQC_EUNSUPPORTED, "attribution tensor too large");
  attr_meas_grp<T, KOUT><<<(unsigned)ntask, 32 * pow3(NG), 0, st>>>(src, out, p, ja, jb, xb);
  CUTQC_LAUNCH_CHECK("attr_meas_grp");
  return CUTQC_OK;
}

template <typename T>
int dispatch_meas_grp(const T* src, float* out, const AttrParams& p, cudaStream_t st) {
  switch (p.k_out) {
    case 1: return run_meas_grp<T, 1>(src, out, p, st);
    case 2: return run_meas_grp<T, 2>(src, out, p, st);
    case 3: return run_meas_grp<T, 3>(src, out, p, st);
    case 4: return run_meas_grp<T, 4>(src, out, p, st);
    case 5: return run_meas_grp<T, 5>(src, out, p, st);
  }
  return set_error(CUTQC_EUNSUPPORTED, "k_out = %d", p.k_out);
}

template <typename T, int KOUT>
int run_meas_run(const T* src, float* out, const AttrParams& p, int staged, cudaStream_t st) {
  const int64_t xb = (p.n_rows + kRunRows - 1) / kRunRows;
  const int64_t ntask = xb * pow3(KOUT) << (2 * p.k_in);
  // one task per CTA (a grid of resident CTAs walking the tasks measured
  // slower: 86 against 76 us on the 32-qubit chain's middle subcircuits)
  if (ntask > 0x7fffffffLL) return set_error(CUTQC_EUNSUPPORTED, "attribution tensor too large");
  const int64_t grid = ntask;
  attr_meas_run<T, KOUT><<<(unsigned)grid, kRunRows, 0, st>>>(src, out, p, staged, xb);
  CUTQC_LAUNCH_CHECK("attr_meas_run");
  return CUTQC_OK;
}

template <typename T>
int dispatch_meas_run(const T* src, float* out, const AttrParams& p, int staged, cudaStream_t st) {
  switch (p.k_out) {
    case 1: return run_meas_run<T, 1>(src, out, p, staged, st);
    case 2: return run_meas_run<T, 2>(src, out, p, staged, st);
    case 3: return run_meas_run<T, 3>(src, out, p, staged, st);
    case 4: return run_meas_run<T, 4>(src, out, p, staged, st);
    case 5: return run_meas_run<T, 5>(src, out, p, staged, st);
  }
  return set_error(CUTQC_EUNSUPPORTED, "k_out = %d", p.k_out);
}

template <typename T>
int launch_attr(const cutqc_subcircuit* s, const T* src, float* dst, float* tmp, cudaStream_t st) {
  AttrParams p{};
  fill_params(s, &p);
  const int o = s->w - s->k_out;
  if (p.k == 0) {
    int64_t n = (int64_t)1 << s->w;
    int blocks = (int)std::min<int64_t>((n + 255) / 256, 4096);
    attr_copy<T><<<blocks, 256, 0, st>>>(src, dst, n);
    CUTQC_LAUNCH_CHECK("attr_copy");
    return CUTQC_OK;
  }
  if (s->k_in > 0 && s->k_out > 0) {
    // both kinds of cut: the measured side first, on the variants as given
    // (the init states stand where the bases will be), which shrinks the
    // data from 3^k_out * 2^w to 4^k_out * 2^o values per init state; then
    // the initialised side along the columns, from the workspace into dst
    p.n_rows = (int64_t)1 << o;
    int rc = dispatch_meas_run<T>(src, tmp, p, 1, st);
    if (rc) return rc;
    return dispatch_init_cols(tmp, dst, p, st);
  }
  if (s->k_in > 0) {
    p.n_rows = (int64_t)1 << s->w;
    return dispatch_init<T>(src, dst, p, 1, st);
  }
  p.n_rows = (int64_t)1 << o;
  if (((uintptr_t)dst & 15) == 0) return dispatch_meas_grp<T>(src, dst, p, st);
  return dispatch_meas_run<T>(src, dst, p, 0, st);
}

}  // namespace

int validate_subcircuit(const cutqc_subcircuit* s) { return validate_sub(s); }

}  // namespace cutqc

using namespace cutqc;

extern "C" int cutqc_attribute_workspace_size(const cutqc_subcircuit* s, size_t* bytes) {
  int rc = validate_sub(s);
  if (rc) return rc;
  if (!bytes) return set_error(CUTQC_EINVAL, "null bytes");
  if (s->k_in > kMaxKin || s->k_out > kMaxKout)
    return set_error(CUTQC_EUNSUPPORTED, "attribution supports k_in <= %d, k_out <= %d", kMaxKin, kMaxKout);
  size_t n = 0;
  if (s->k_in > 0 && s->k_out > 0)       // the measured side's output, [2^o][4^k] float32
    n = ((size_t)1 << (s->w - s->k_out)) * ((size_t)1 << (2 * (s->k_in + s->k_out))) * sizeof(float);
  *bytes = n;
  return CUTQC_OK;
}

extern "C" int cutqc_attribute(const cutqc_subcircuit* s, const void* variants_dev, int dtype,
                               float* attributed_dev, void* ws_dev, size_t ws_bytes, void* stream) {
  size_t need = 0;
  int rc = cutqc_attribute_workspace_size(s, &need);
  if (rc) return rc;
  if (!variants_dev || !attributed_dev) return set_error(CUTQC_EINVAL, "null tensor pointer");
  if (dtype != CUTQC_F64 && dtype != CUTQC_F32) return set_error(CUTQC_EINVAL, "dtype must be CUTQC_F64 or CUTQC_F32");
  if (ws_bytes < need || (need && !ws_dev)) return set_error(CUTQC_ENOMEM, "attribution workspace needs %zu bytes", need);
  cudaStream_t st = (cudaStream_t)stream;
  if (dtype == CUTQC_F64)
    return launch_attr<double>(s, (const double*)variants_dev, attributed_dev, (float*)ws_dev, st);
  return launch_attr<float>(s, (const float*)variants_dev, attributed_dev, (float*)ws_dev, st);
}

// ------------------------------------------------- attribution, no allocation
//
// Some callers cannot allocate device memory at all: code that runs while a
// memory pool owns the whole device, plugins whose host forbids cudaMalloc
// between set-up and tear-down, or callers that must not synchronise (a
// cudaMalloc or cudaFree can synchronise the device).  For them this variant
// takes its scratch from a fixed array that the library declares at file
// scope, so the call itself allocates nothing; the caller still owns the
// variant and attributed tensors.
//
// The array is kNoAllocScratchBytes (32 MiB) of device memory on every GPU
// that loads this library, held until the process exits.  Its device
// address is looked up once per device (cudaGetSymbolAddress) on the first
// call that needs scratch (a subcircuit with both kinds of cut) made with
// that device current, so that first call should come before any stream
// capture.  All calls share the one array and it keeps whatever
// the last call left there: calls that may overlap on the GPU (different
// streams, no ordering between them) race on it and must not be issued that
// way.  Nothing in it needs to start at zero: the pass that writes it covers
// every element the next pass reads.

namespace cutqc {
namespace {

constexpr size_t kNoAllocScratchBytes = (size_t)32 << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

int noalloc_scratch(void** ptr) {
  static std::mutex mu;
  static std::vector<void*> addr;       // per device id
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_error(e, "cudaGetDevice");
  std::lock_guard<std::mutex> lk(mu);
  if ((int)addr.size() <= dev) addr.resize(dev + 1, nullptr);
  if (!addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_error(e, "cudaGetSymbolAddress(no-allocation scratch)");
    addr[dev] = p;
  }
  *ptr = addr[dev];
  return CUTQC_OK;
}

}  // namespace
}  // namespace cutqc

extern "C" int cutqc_attribute_noalloc(const cutqc_subcircuit* s, const void* variants_dev, int dtype,
                                       float* attributed_dev, void* stream) {
  size_t need = 0;
  int rc = cutqc_attribute_workspace_size(s, &need);
  if (rc) return rc;
  if (!variants_dev || !attributed_dev) return set_error(CUTQC_EINVAL, "null tensor pointer");
  if (dtype != CUTQC_F64 && dtype != CUTQC_F32) return set_error(CUTQC_EINVAL, "dtype must be CUTQC_F64 or CUTQC_F32");
  if (need > kNoAllocScratchBytes)
    return set_error(CUTQC_EUNSUPPORTED,
                     "this subcircuit needs %zu bytes of scratch; the no-allocation variant has %zu "
                     "(use cutqc_attribute with a workspace)",
                     need, kNoAllocScratchBytes);
  // subcircuits with one kind of cut need no scratch: no symbol lookup then
  void* scratch = nullptr;
  if (need > 0 && (rc = noalloc_scratch(&scratch))) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  if (dtype == CUTQC_F64)
    return launch_attr<double>(s, (const double*)variants_dev, attributed_dev, (float*)scratch, st);
  return launch_attr<float>(s, (const float*)variants_dev, attributed_dev, (float*)scratch, st);
}
