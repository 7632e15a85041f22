// Dynamic definition (Algorithm 1): merge, bin reconstruction, selection.
//
// Each recursion labels up to M qubits active, fixes the zoomed ones and
// merges the rest.  Attribution is linear and acts only on cut qubits, so the
// merge applies to every attributed tensor before reconstruction:
//   merged[a][c] = sum_m attributed[x(a, z, m)][c]
// with x built from the active bits a, the zoom bits z and the merged bits m
// of the subcircuit's outputs (the GPU analogue of grouping the QPU shots by
// active-qubit state).  The 2^#active bins are then Eq. 1 on the merged
// tensors (the shared contraction planner, all jobs of a level batched in one
// launch per step), and the T largest bins are selected per job.
#include "internal.cuh"
#include "contract.cuh"

#include <algorithm>
#include <cmath>
#include <map>
#include <vector>

namespace cutqc {

namespace {

// Compensated float32 accumulation (Kahan) of one column over the merged rows.
struct Kahan {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add(float v) {
    float y = v - c;
    float t = s + y;
    c = (t - s) - y;
    s = t;
  }
};

// grid: x = merged row a, y = job.  zoom value of job j: zoom_dev ? zoom_dev[j]
// : zoom_val.  Threads split columns and, when there are few columns, the
// merged index range; slices are combined through shared memory.
__global__ void __launch_bounds__(256)
dd_merge_kernel(const float* __restrict__ att, int k, uint64_t act_mask, uint64_t merged_mask, uint64_t zoom_mask,
                uint64_t zoom_val, const uint64_t* __restrict__ zoom_dev, int n_merged, float* __restrict__ out) {
  __shared__ float red[256];
  const int64_t C = (int64_t)1 << (2 * k);
  const int a = blockIdx.x;
  const int job = blockIdx.y;
  const int64_t rows_a = (int64_t)gridDim.x;
  const uint64_t z = (zoom_dev ? __ldg(zoom_dev + job) : zoom_val) & zoom_mask;
  const uint64_t base = pdep64((uint64_t)a, act_mask) | z;
  const int64_t M = (int64_t)1 << n_merged;
  float* dst = out + ((int64_t)job * rows_a + a) * C;
  const int cw = (int)(C < 256 ? C : 256);
  const int slices = 256 / cw;
  const int c_local = threadIdx.x % cw;
  const int slice = threadIdx.x / cw;
  for (int64_t c0 = 0; c0 < C; c0 += cw) {
    Kahan acc;
    if (slice < slices)
      for (int64_t m = slice; m < M; m += slices) {
        const uint64_t x = base | pdep64((uint64_t)m, merged_mask);
        acc.add(__ldg(att + (int64_t)x * C + c0 + c_local));
      }
    red[threadIdx.x] = acc.s;
    __syncthreads();
    if (slice == 0) {
      float s = red[c_local];
      for (int q = 1; q < slices; ++q) s += red[q * cw + c_local];
      dst[c0 + c_local] = s;
    }
    __syncthreads();
  }
}

// One CTA per job: top-T bins by (value desc, index asc), and the float64
// bin total is left in bin_sum by the reconstruction's epilogue.
__global__ void __launch_bounds__(1024)
dd_topk_kernel(const float* __restrict__ bins, int64_t nb, int T, int32_t* __restrict__ top_idx,
               float* __restrict__ top_val) {
  __shared__ float sv[32];
  __shared__ int64_t si[32];
  __shared__ float pick_v;
  __shared__ int64_t pick_i;
  const float* b = bins + (int64_t)blockIdx.x * nb;
  float pv = INFINITY;
  int64_t pi = -1;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int t = 0; t < T; ++t) {
    float bv = -INFINITY;
    int64_t bi = -1;
    for (int64_t i = threadIdx.x; i < nb; i += blockDim.x) {
      float v = b[i];
      bool after = (v < pv) || (v == pv && i > pi);   // strictly after the previous pick
      if (!after) continue;
      if (bi < 0 || v > bv || (v == bv && i < bi)) { bv = v; bi = i; }
    }
    for (int off = 16; off; off >>= 1) {
      float ov = __shfl_xor_sync(0xffffffffu, bv, off);
      int64_t oi = __shfl_xor_sync(0xffffffffu, bi, off);
      if (oi >= 0 && (bi < 0 || ov > bv || (ov == bv && oi < bi))) { bv = ov; bi = oi; }
    }
    if (lane == 0) { sv[warp] = bv; si[warp] = bi; }
    __syncthreads();
    if (warp == 0) {
      const int nw = blockDim.x >> 5;
      bv = lane < nw ? sv[lane] : -INFINITY;
      bi = lane < nw ? si[lane] : -1;
      for (int off = 16; off; off >>= 1) {
        float ov = __shfl_xor_sync(0xffffffffu, bv, off);
        int64_t oi = __shfl_xor_sync(0xffffffffu, bi, off);
        if (oi >= 0 && (bi < 0 || ov > bv || (ov == bv && oi < bi))) { bv = ov; bi = oi; }
      }
      if (lane == 0) {
        pick_v = bv;
        pick_i = bi;
        top_idx[(int64_t)blockIdx.x * T + t] = (int32_t)bi;
        top_val[(int64_t)blockIdx.x * T + t] = bi >= 0 ? bv : 0.f;
      }
    }
    __syncthreads();
    pv = pick_v;
    pi = pick_i;
    __syncthreads();
  }
}

__global__ void sum_f64_kernel(const float* __restrict__ x, int64_t n, double* __restrict__ sum) {
  double local = 0.0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x * 16;
  for (int64_t i0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * 16; i0 < n; i0 += stride) {
    float part = 0.f;
    if (i0 + 16 <= n && ((((uintptr_t)(x + i0)) & 15) == 0)) {
      const float4* p = reinterpret_cast<const float4*>(x + i0);
      float4 a = __ldg(p), b = __ldg(p + 1), c = __ldg(p + 2), d = __ldg(p + 3);
      part = ((a.x + a.y) + (a.z + a.w)) + ((b.x + b.y) + (b.z + b.w)) + ((c.x + c.y) + (c.z + c.w)) +
             ((d.x + d.y) + (d.z + d.w));
    } else {
      for (int64_t i = i0; i < n && i < i0 + 16; ++i) part += x[i];
    }
    local += (double)part;
  }
  for (int off = 16; off; off >>= 1) local += __shfl_xor_sync(0xffffffffu, local, off);
  if ((threadIdx.x & 31) == 0) atomicAdd(sum, local);
}

int merge_masks(const cutqc_subcircuit* s, const int8_t* role, uint64_t* act, uint64_t* mrg, uint64_t* zm,
                uint64_t* zv) {
  const int o = s->w - s->k_out;
  *act = *mrg = *zm = *zv = 0;
  for (int t = 0; t < o; ++t) {
    const uint64_t b = (uint64_t)1 << t;
    switch (role[t]) {
      case 0: *act |= b; break;
      case 1: *mrg |= b; break;
      case 2: *zm |= b; break;
      case 3: *zm |= b; *zv |= b; break;
      default: return set_error(CUTQC_EINVAL, "role[%d] = %d not in 0..3", t, (int)role[t]);
    }
  }
  return CUTQC_OK;
}

int launch_merge(const cutqc_subcircuit* s, const float* att, uint64_t act, uint64_t mrg, uint64_t zm, uint64_t zv,
                 const uint64_t* zoom_dev, int n_jobs, float* out, cudaStream_t st) {
  const int k = s->k_in + s->k_out;
  const int a = __builtin_popcountll(act);
  if (a > 30) return set_error(CUTQC_EUNSUPPORTED, "too many active bits");
  if ((int64_t)1 << a > 0x7fffffffLL) return set_error(CUTQC_EUNSUPPORTED, "too many rows");
  if (n_jobs < 1 || n_jobs > 65535) return set_error(CUTQC_EINVAL, "n_jobs out of range");
  dd_merge_kernel<<<dim3(1u << a, n_jobs), 256, 0, st>>>(att, k, act, mrg, zm, zv, zoom_dev, __builtin_popcountll(mrg),
                                                          out);
  CUTQC_LAUNCH_CHECK("dd_merge_kernel");
  return CUTQC_OK;
}

int dd_inputs(int n_sub, const cutqc_subcircuit* s, const int32_t* active_bits, const int32_t* bin_bit,
              std::vector<TensorDesc>* in, int* total_bits) {
  if (n_sub < 1 || !s || !active_bits) return set_error(CUTQC_EINVAL, "bad DD job description");
  int tot = 0;
  std::map<int, int> uses;
  in->clear();
  for (int i = 0; i < n_sub; ++i) {
    int rc = validate_subcircuit(&s[i]);
    if (rc) return rc;
    const int o = s[i].w - s[i].k_out;
    if (active_bits[i] < 0 || active_bits[i] > o) return set_error(CUTQC_EINVAL, "active_bits[%d] out of range", i);
    TensorDesc t;
    t.o = active_bits[i];
    for (int j = 0; j < s[i].k_in; ++j) t.edges.push_back(s[i].in_edge[j]);
    for (int j = 0; j < s[i].k_out; ++j) t.edges.push_back(s[i].out_edge[j]);
    std::sort(t.edges.begin(), t.edges.end());
    tot += t.o;
    in->push_back(t);
  }
  if (tot > 30) return set_error(CUTQC_EUNSUPPORTED, "%d bin bits > 30", tot);
  if (tot > 0 && !bin_bit) return set_error(CUTQC_EINVAL, "null bin_bit");
  std::vector<int> seen(tot, 0);
  int q = 0;
  for (int i = 0; i < n_sub; ++i)
    for (int b = 0; b < (*in)[i].o; ++b) {
      int p = bin_bit[q++];
      if (p < 0 || p >= tot || seen[p]) return set_error(CUTQC_EINVAL, "bin_bit must be a permutation of 0..%d", tot - 1);
      seen[p] = 1;
      (*in)[i].pos.push_back(p);
    }
  *total_bits = tot;
  return CUTQC_OK;
}

}  // namespace

}  // namespace cutqc

using namespace cutqc;

extern "C" int cutqc_dd_merge(const cutqc_subcircuit* s, const float* attributed, const int8_t* role, float* merged,
                              void* stream) {
  int rc = validate_subcircuit(s);
  if (rc) return rc;
  if (!attributed || !merged || !role) return set_error(CUTQC_EINVAL, "null pointer");
  uint64_t act, mrg, zm, zv;
  if ((rc = merge_masks(s, role, &act, &mrg, &zm, &zv))) return rc;
  return launch_merge(s, attributed, act, mrg, zm, zv, nullptr, 1, merged, (cudaStream_t)stream);
}

extern "C" int cutqc_dd_merge_batch(const cutqc_subcircuit* s, const float* attributed, uint64_t active_mask,
                                    uint64_t zoom_mask, int n_jobs, const uint64_t* zoom_dev, float* merged,
                                    void* stream) {
  int rc = validate_subcircuit(s);
  if (rc) return rc;
  if (!attributed || !merged || !zoom_dev) return set_error(CUTQC_EINVAL, "null pointer");
  const int o = s->w - s->k_out;
  const uint64_t all = o >= 64 ? ~0ull : (((uint64_t)1 << o) - 1);
  if ((active_mask | zoom_mask) & ~all) return set_error(CUTQC_EINVAL, "mask bits beyond the %d outputs", o);
  if (active_mask & zoom_mask) return set_error(CUTQC_EINVAL, "a bit cannot be active and zoomed");
  const uint64_t mrg = all & ~active_mask & ~zoom_mask;
  return launch_merge(s, attributed, active_mask, mrg, zoom_mask, 0, zoom_dev, n_jobs, merged, (cudaStream_t)stream);
}

extern "C" int cutqc_dd_step_workspace_size(int n_sub, const cutqc_subcircuit* s, const int32_t* active_bits,
                                            int n_jobs, size_t* bytes) {
  if (!bytes) return set_error(CUTQC_EINVAL, "null bytes");
  std::vector<TensorDesc> in;
  int tot = 0;
  // bin_bit does not change the workspace: use the identity order
  std::vector<int32_t> ident;
  for (int i = 0; i < n_sub && active_bits; ++i)
    for (int b = 0; b < active_bits[i]; ++b) ident.push_back((int32_t)ident.size());
  int rc = dd_inputs(n_sub, s, active_bits, ident.data(), &in, &tot);
  if (rc) return rc;
  if (n_jobs < 1) return set_error(CUTQC_EINVAL, "n_jobs must be >= 1");
  ContractionPlan plan;
  if ((rc = plan_contraction_batched(in, CUTQC_PREC_FP32_SIMT, n_jobs, &plan))) return rc;
  *bytes = plan.ws_bytes;
  return CUTQC_OK;
}

extern "C" int cutqc_dd_step(int n_sub, const cutqc_subcircuit* s, const int32_t* active_bits, const int32_t* bin_bit,
                             int n_jobs, const float* const* merged, float* bins, double* bin_sum, int topk,
                             int32_t* top_idx, float* top_val, void* ws_dev, size_t ws_bytes, void* stream) {
  std::vector<TensorDesc> in;
  int tot = 0;
  int rc = dd_inputs(n_sub, s, active_bits, bin_bit, &in, &tot);
  if (rc) return rc;
  if (n_jobs < 1 || n_jobs > 65535) return set_error(CUTQC_EINVAL, "n_jobs out of range");
  if (!merged || !bins) return set_error(CUTQC_EINVAL, "null pointer");
  for (int i = 0; i < n_sub; ++i)
    if (!merged[i]) return set_error(CUTQC_EINVAL, "null merged tensor");
  if (topk < 0 || topk > 32) return set_error(CUTQC_EUNSUPPORTED, "topk must be in 0..32");
  if (topk > 0 && (!top_idx || !top_val)) return set_error(CUTQC_EINVAL, "null top-k outputs");
  ContractionPlan plan;
  if ((rc = plan_contraction_batched(in, CUTQC_PREC_FP32_SIMT, n_jobs, &plan))) return rc;
  if (ws_bytes < plan.ws_bytes || (plan.ws_bytes && !ws_dev))
    return set_error(CUTQC_ENOMEM, "DD workspace needs %zu bytes", plan.ws_bytes);
  cudaStream_t st = (cudaStream_t)stream;
  std::vector<int64_t> bstride(n_sub);
  for (int i = 0; i < n_sub; ++i) bstride[i] = ((int64_t)1 << in[i].o) << (2 * in[i].edges.size());
  const int64_t nb = (int64_t)1 << tot;
  if (bin_sum) CUTQC_CUDA_TRY(cudaMemsetAsync(bin_sum, 0, sizeof(double) * n_jobs, st));
  rc = run_plan(plan, merged, bstride.data(), n_jobs, bins, nb, bin_sum, std::ldexp(1.0f, -plan.K),
                CUTQC_PREC_FP32_SIMT, 0, -1, (uint8_t*)ws_dev, st);
  if (rc) return rc;
  if (topk > 0) {
    int threads = (int)std::min<int64_t>(1024, std::max<int64_t>(32, (nb + 31) / 32 * 32));
    dd_topk_kernel<<<n_jobs, threads, 0, st>>>(bins, nb, topk, top_idx, top_val);
    CUTQC_LAUNCH_CHECK("dd_topk_kernel");
  }
  return CUTQC_OK;
}

extern "C" int cutqc_sum_f64(const float* x, int64_t n, double* sum, void* stream) {
  if (!x || !sum || n < 0) return set_error(CUTQC_EINVAL, "bad arguments");
  if (n == 0) return CUTQC_OK;
  int blocks = (int)std::min<int64_t>((n / 16 + 255) / 256 + 1, (int64_t)sm_count() * 8);
  sum_f64_kernel<<<blocks, 256, 0, (cudaStream_t)stream>>>(x, n, sum);
  CUTQC_LAUNCH_CHECK("sum_f64_kernel");
  return CUTQC_OK;
}
