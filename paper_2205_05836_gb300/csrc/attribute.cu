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
// The map is a tensor product of one small map per cut.  A CTA owns R
// consecutive outcome rows and one value of the "other" index, stages the
// fiber of all cut digits for its rows in shared memory (loads coalesced
// along the outcome index), applies the per-cut maps axis by axis, and
// writes the result.  Subcircuits with both kinds of cut take two passes
// (initialised axes first, through a float32 workspace).  Arithmetic is
// float32 after the (float64 or float32) loads; HBM-bound.
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
constexpr int kThreads = 256;

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

__device__ __forceinline__ float load_val(const double* p) { return (float)__ldg(p); }
__device__ __forceinline__ float load_val(const float* p) { return __ldg(p); }

// 4x4 map of the initialised side: rows I, X, Y, Z; columns |0>,|1>,|+>,|+i>.
__device__ __forceinline__ float init_map(int d, const float* in, int stride) {
  float p0 = in[0], p1 = in[stride], pp = in[2 * stride], ppi = in[3 * stride];
  switch (d) {
    case 0: return p0 + p1;
    case 1: return 2.f * pp - p0 - p1;
    case 2: return 2.f * ppi - p0 - p1;
    default: return p0 - p1;
  }
}

// Initialised-side pass.  Fiber over the 4^k_in init digits, R consecutive
// outcome rows x (full w-bit index), fixed measurement run index `mrun`
// (blockIdx.y).  final_layout: write attributed[x][col] (only valid when
// k_out == 0); else write the [4^k_in][3^k_out][2^w] layout with states
// replaced by bases.
template <typename T>
__global__ void __launch_bounds__(kThreads)
attr_init_pass(const T* __restrict__ src, float* __restrict__ dst, AttrParams p, int final_layout) {
  extern __shared__ float sm[];
  const int F = 1 << (2 * p.k_in);
  const int R = p.R;
  float* buf0 = sm;
  float* buf1 = sm + F * R;
  const int64_t x0 = (int64_t)blockIdx.x * R;
  const int mrun = blockIdx.y;
  const int nm = [&] { int v = 1; for (int j = 0; j < p.k_out; ++j) v *= 3; return v; }();
  const int64_t W = (int64_t)1 << p.w;
  const int rows = (int)(p.n_rows - x0 < R ? p.n_rows - x0 : R);
  // load: element (f, r) at src[(f * nm + mrun) * W + x0 + r]
  for (int i = threadIdx.x; i < F * R; i += blockDim.x) {
    int f = i / R, r = i - f * R;
    float v = 0.f;
    if (r < rows) v = load_val(src + ((int64_t)f * nm + mrun) * W + x0 + r);
    buf0[i] = v;
  }
  __syncthreads();
  float* in = buf0;
  float* out = buf1;
  for (int j = 0; j < p.k_in; ++j) {
    const int stride = (1 << (2 * j)) * R;   // digit j of f has weight 4^j
    for (int i = threadIdx.x; i < F * R; i += blockDim.x) {
      int f = i / R, r = i - f * R;
      int d = (f >> (2 * j)) & 3;
      int base = ((f & ~(3 << (2 * j))) * R) + r;
      out[i] = init_map(d, in + base, stride);
    }
    __syncthreads();
    float* t = in; in = out; out = t;
  }
  if (final_layout) {
    // attributed[x][col]: col = sum_j d_j << col_shift_in[j]
    const int C = F;   // k_out == 0 so 4^k == F
    for (int i = threadIdx.x; i < rows * C; i += blockDim.x) {
      int r = i / C, c = i - r * C;
      int f = 0;
      for (int j = 0; j < p.k_in; ++j) f |= ((c >> p.col_shift_in[j]) & 3) << (2 * j);
      dst[(x0 + r) * C + c] = in[f * R + r];
    }
  } else {
    for (int i = threadIdx.x; i < F * R; i += blockDim.x) {
      int f = i / R, r = i - f * R;
      if (r < rows) dst[((int64_t)f * nm + mrun) * W + x0 + r] = in[i];
    }
  }
}

// Measured-side pass.  Fiber over (run digit m_j in {0,1,2}, outcome bit b_j)
// per measured cut, combined as u_j = 2 m_j + b_j (radix 6); R consecutive
// output rows x_out; fixed init digits `dinit` (blockIdx.y).  Writes
// attributed[x_out][col(dinit, dmeas)].
template <typename T>
__global__ void __launch_bounds__(kThreads)
attr_meas_pass(const T* __restrict__ src, float* __restrict__ dst, AttrParams p) {
  extern __shared__ float sm[];
  int F = 1;
  for (int j = 0; j < p.k_out; ++j) F *= 6;
  const int R = p.R;
  float* buf0 = sm;
  float* buf1 = sm + F * R;
  int64_t* rowbase = reinterpret_cast<int64_t*>(buf1 + F * R);   // [R]
  int64_t* bpart = rowbase + R;                                  // [2^k_out]
  const int64_t x0 = (int64_t)blockIdx.x * R;
  const int dinit = blockIdx.y;
  int nm = 1;
  for (int j = 0; j < p.k_out; ++j) nm *= 3;
  const int64_t W = (int64_t)1 << p.w;
  const int rows = (int)(p.n_rows - x0 < R ? p.n_rows - x0 : R);
  for (int r = threadIdx.x; r < R; r += blockDim.x) rowbase[r] = (int64_t)pdep64((uint64_t)(x0 + r), p.out_mask);
  for (int b = threadIdx.x; b < (1 << p.k_out); b += blockDim.x) {
    uint64_t v = 0;
    for (int j = 0; j < p.k_out; ++j)
      if ((b >> j) & 1) v |= p.meas_mask[j];
    bpart[b] = (int64_t)v;
  }
  __syncthreads();
  // load: fiber index f = sum_j u_j 6^j, u_j = 2 m_j + b_j
  for (int i = threadIdx.x; i < F * R; i += blockDim.x) {
    int f = i / R, r = i - f * R;
    int t = f, m = 0, b = 0, w3 = 1;
    for (int j = 0; j < p.k_out; ++j) {
      int u = t % 6; t /= 6;
      m += (u >> 1) * w3; w3 *= 3;
      b |= (u & 1) << j;
    }
    float v = 0.f;
    if (r < rows) v = load_val(src + ((int64_t)dinit * nm + m) * W + (rowbase[r] | bpart[b]));
    buf0[i] = v;
  }
  __syncthreads();
  // axis j: radix 6 -> radix 4; digits < j already radix 4
  float* in = buf0;
  float* out = buf1;
  int Fin = F;
  for (int j = 0; j < p.k_out; ++j) {
    int low = 1 << (2 * j);          // size of processed (radix-4) digits below j
    int hi_in = Fin / (low * 6);     // size of the digits above j
    int Fout = low * 4 * hi_in;
    for (int i = threadIdx.x; i < Fout * R; i += blockDim.x) {
      int g = i / R, r = i - g * R;
      int lo_part = g % low;
      int d = (g / low) & 3;
      int hi_part = g / (low * 4);
      // (run, w0, w1): I (0,+,+) X (1,+,-) Y (2,+,-) Z (0,+,-)
      int run = (d == 3) ? 0 : d;
      float w1 = (d == 0) ? 1.f : -1.f;
      int f0 = lo_part + low * (2 * run + 0) + low * 6 * hi_part;
      int f1 = lo_part + low * (2 * run + 1) + low * 6 * hi_part;
      out[i] = in[f0 * R + r] + w1 * in[f1 * R + r];
    }
    Fin = Fout;
    __syncthreads();
    float* t = in; in = out; out = t;
  }
  // write: dmeas index g = sum_j d_j 4^j
  const int G = Fin;                         // 4^k_out
  const int64_t C = (int64_t)1 << (2 * p.k);
  int cin = 0;
  for (int j = 0; j < p.k_in; ++j) cin |= ((dinit >> (2 * j)) & 3) << p.col_shift_in[j];
  for (int i = threadIdx.x; i < rows * G; i += blockDim.x) {
    int r = i / G, g = i - r * G;
    int c = cin;
    for (int j = 0; j < p.k_out; ++j) c |= ((g >> (2 * j)) & 3) << p.col_shift_out[j];
    dst[(x0 + r) * C + c] = in[g * R + r];
  }
}

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
constexpr int kAttrMaxSmem = 100 * 1024;
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

int pick_rows(int fiber, int64_t max_rows) {
  int R = 32;
  while (R > 1 && (size_t)fiber * R * 2 * sizeof(float) > 96 * 1024) R >>= 1;
  while (R > 1 && R > max_rows) R >>= 1;
  return R;
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
  const T* meas_src = src;
  bool meas_from_tmp = false;
  if (s->k_in > 0) {
    const int F = 1 << (2 * s->k_in);
    p.n_rows = (int64_t)1 << s->w;
    p.R = pick_rows(F, p.n_rows);
    size_t smem = (size_t)F * p.R * 2 * sizeof(float);
    if (smem > (size_t)kAttrMaxSmem) return set_error(CUTQC_EUNSUPPORTED, "attribution fiber too large");
    int nm = 1;
    for (int j = 0; j < s->k_out; ++j) nm *= 3;
    dim3 grid((unsigned)((p.n_rows + p.R - 1) / p.R), nm);
    int final_layout = s->k_out == 0;
    float* out = final_layout ? dst : tmp;
    CUTQC_CUDA_TRY(set_max_smem((const void*)attr_init_pass<T>));
    attr_init_pass<T><<<grid, kThreads, smem, st>>>(src, out, p, final_layout);
    CUTQC_LAUNCH_CHECK("attr_init_pass");
    if (final_layout) return CUTQC_OK;
    meas_from_tmp = true;
  }
  {
    int F = 1;
    for (int j = 0; j < s->k_out; ++j) F *= 6;
    p.n_rows = (int64_t)1 << o;
    p.R = pick_rows(F, p.n_rows);
    size_t smem = (size_t)F * p.R * 2 * sizeof(float) + (size_t)(p.R + (1 << s->k_out)) * sizeof(int64_t);
    if (smem > (size_t)kAttrMaxSmem) return set_error(CUTQC_EUNSUPPORTED, "attribution fiber too large");
    dim3 grid((unsigned)((p.n_rows + p.R - 1) / p.R), 1u << (2 * s->k_in));
    if (meas_from_tmp) {
      CUTQC_CUDA_TRY(set_max_smem((const void*)attr_meas_pass<float>));
      attr_meas_pass<float><<<grid, kThreads, smem, st>>>(tmp, dst, p);
    } else {
      CUTQC_CUDA_TRY(set_max_smem((const void*)attr_meas_pass<T>));
      attr_meas_pass<T><<<grid, kThreads, smem, st>>>(meas_src, dst, p);
    }
    CUTQC_LAUNCH_CHECK("attr_meas_pass");
  }
  return CUTQC_OK;
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
  if (s->k_in > 0 && s->k_out > 0) {
    size_t nm = 1;
    for (int j = 0; j < s->k_out; ++j) nm *= 3;
    n = ((size_t)1 << (2 * s->k_in)) * nm * ((size_t)1 << s->w) * sizeof(float);
  }
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
