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
#include "dd_kernels.cuh"
#include "dd_host.cuh"

#include <algorithm>
#include <cstring>
#include <cmath>
#include <map>
#include <mutex>
#include <vector>

namespace cutqc {

namespace {

// grid: x = CTAs walking the (merged row a, job) pairs, z = slice of the
// merged index range (body in dd_kernels.cuh).
__global__ void __launch_bounds__(256)
dd_merge_kernel(const float* __restrict__ att, int k, uint64_t act_mask, uint64_t merged_mask, uint64_t zoom_mask,
                uint64_t zoom_val, const uint64_t* __restrict__ zoom_dev, const ZoomFromJobs zj, int n_jobs,
                int64_t rows_a, int n_merged, int log_slices, float* __restrict__ out) {
  dd_merge_body<false>(att, k, act_mask, merged_mask, zoom_mask, zoom_val, zoom_dev, zj, n_jobs, rows_a, n_merged,
                       log_slices, out, blockIdx.x, gridDim.x, blockIdx.z);
}

__global__ void dd_merge_reduce(const float* __restrict__ part, int S, int64_t E, float* __restrict__ out) {
  dd_merge_reduce_body<false>(part, S, E, out, blockIdx.x, gridDim.x);
}

// CTA (job blockIdx.x, chunk blockIdx.y) of the top-T selection.  gate
// (nullable): the job is skipped unless gate[job] > gate_cap.
template <int TCAP, bool kCand>
__global__ void __launch_bounds__(1024)
dd_topk_kernel(const float* __restrict__ vals, const int32_t* __restrict__ cidx, int64_t n, int64_t chunk_len, int T,
               int32_t* __restrict__ top_idx, float* __restrict__ top_val, const int* __restrict__ gate = nullptr,
               int gate_cap = 0) {
  if (gate && __ldg(gate + blockIdx.x) <= gate_cap) return;
  dd_topk_body<TCAP, kCand, false>(vals, cidx, n, chunk_len, T, top_idx, top_val, blockIdx.x, blockIdx.y,
                                   gridDim.y);
}

// Top-T from block maxima.  The output of the last contraction step is cut
// into blocks (32 rows x 64 columns), and that step (the paired GEMM or the
// outer-product kernel) wrote each block's largest value.  Let
// v* be the T-th largest of the block maxima: T distinct bins are >= v*, so
// every bin among the T largest is >= v*, and so is the maximum of its block.
// The blocks whose maximum is >= v* therefore hold all of the T largest bins
// (exactly T blocks unless maxima tie at v*); only they are read again.
constexpr int kBlockRows = 32, kBlockCols = 64, kBlockBins = kBlockRows * kBlockCols;
constexpr int kBlockCap = 32;                         // blocks read again per job, at most
constexpr int64_t kBlockMaxMinBins = (int64_t)1 << 22;   // smaller jobs scan their bins
constexpr int64_t kBlockMaxChunk = (int64_t)1 << 12;      // block maxima per chunk of their scan

// Blocks of job blockIdx.y whose maximum is >= v* (the T-th entry of the
// job's top-T over its block maxima; -inf when it has fewer than T blocks).
// count[job] may exceed cap: only the first cap are listed.
__global__ void dd_block_collect(const float* __restrict__ cmax, int64_t C, const int32_t* __restrict__ kidx,
                                 const float* __restrict__ kval, int T, int cap, int* __restrict__ count,
                                 int32_t* __restrict__ list) {
  const int job = blockIdx.y;
  const float thr = kidx[(int64_t)job * T + T - 1] >= 0 ? kval[(int64_t)job * T + T - 1] : -INFINITY;
  const float* c = cmax + (int64_t)job * C;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < C; i += (int64_t)gridDim.x * blockDim.x) {
    if (__ldg(c + i) >= thr) {
      const int p = atomicAdd(count + job, 1);
      if (p < cap) list[(int64_t)job * cap + p] = (int32_t)i;
    }
  }
}

// CTA (slot blockIdx.x, job blockIdx.y): copies listed block `slot` of the
// job as (value, bin index) pairs; unused slots get index -1.  The bin index
// of output (m, n) is pdep(m, mask_m) | pdep(n, mask_n).
__global__ void dd_block_gather(const float* __restrict__ bins, int64_t nb, const int* __restrict__ count,
                                const int32_t* __restrict__ list, int cap, int64_t cols, int64_t M, int64_t N,
                                uint64_t mask_m, uint64_t mask_n, float* __restrict__ gv, int32_t* __restrict__ gi) {
  const int job = blockIdx.y, slot = blockIdx.x;
  const int used = min(__ldg(count + job), cap);
  float* ov = gv + ((int64_t)job * cap + slot) * kBlockBins;
  int32_t* oi = gi + ((int64_t)job * cap + slot) * kBlockBins;
  if (slot >= used) {
    for (int e = threadIdx.x; e < kBlockBins; e += blockDim.x) oi[e] = -1;
    return;
  }
  const int64_t blk = __ldg(list + (int64_t)job * cap + slot);
  const int64_t r0 = (blk / cols) * kBlockRows, c0 = (blk % cols) * kBlockCols;
  // the block's row and column offsets, deposited once; -1: beyond M or N
  __shared__ int64_t roff[kBlockRows], coff[kBlockCols];
  for (int t = threadIdx.x; t < kBlockRows + kBlockCols; t += blockDim.x) {
    if (t < kBlockRows) {
      const int64_t m = r0 + t;
      roff[t] = m < M ? (int64_t)pdep64((uint64_t)m, mask_m) : -1;
    } else {
      const int64_t n = c0 + (t - kBlockRows);
      coff[t - kBlockRows] = n < N ? (int64_t)pdep64((uint64_t)n, mask_n) : -1;
    }
  }
  __syncthreads();
  const float* b = bins + (int64_t)job * nb;
  for (int e = threadIdx.x; e < kBlockBins; e += blockDim.x) {
    const int64_t ro = roff[e / kBlockCols], co = coff[e % kBlockCols];
    if (ro >= 0 && co >= 0) {
      const int64_t off = ro | co;
      ov[e] = __ldg(b + off);
      oi[e] = (int32_t)off;
    } else {
      oi[e] = -1;
    }
  }
}


// Large jobs: chunks of the chunked first pass of the top-T selection.
// Under a tensor-core precision, a level's contraction steps with fewer
// outputs (all jobs together) run in FP32 on CUDA cores: at DD's usual
// 2^16-bin jobs the split's per-job operand preps and launches cost more
// than its GEMMs save (three 16-active-qubit circuits: 1.5 ms against
// 0.39 ms; the dense recursion's 2^20-output middle step also ran faster
// in FP32), and FP32 is at least as accurate.
constexpr int64_t kDdMinTcOutputs = (int64_t)1 << 22;
constexpr int64_t kTopkChunkMin = (int64_t)1 << 16;   // bins per chunk at least
constexpr int64_t kTopkChunksMax = 2048;
inline int64_t topk_chunks(int64_t nb, int64_t min_chunk = kTopkChunkMin) {
  if (nb <= min_chunk) return 1;
  return std::min<int64_t>(kTopkChunksMax, (nb + min_chunk - 1) / min_chunk);
}
// candidate scratch of the chunked pass for n_jobs jobs of nb bins (bytes)
inline size_t topk_scratch(int64_t nb, int n_jobs, int64_t min_chunk = kTopkChunkMin) {
  const int64_t c = topk_chunks(nb, min_chunk);
  return c > 1 ? align_up((size_t)n_jobs * c * 32 * (sizeof(int32_t) + sizeof(float)), 256) : 0;
}

// scratch of the block-maximum selection for n_jobs jobs of nb bins (bytes)
inline size_t block_max_scratch(int64_t nb, int n_jobs) {
  if (nb < kBlockMaxMinBins) return 0;
  const int64_t C = nb / kBlockBins;
  const size_t per = sizeof(int32_t) + sizeof(float);
  return align_up((size_t)n_jobs * C * sizeof(float), 256) + topk_scratch(C, n_jobs, kBlockMaxChunk) +
         align_up((size_t)n_jobs * 32 * per, 256) + align_up((size_t)n_jobs * sizeof(int), 256) +
         align_up((size_t)n_jobs * kBlockCap * sizeof(int32_t), 256) +
         align_up((size_t)n_jobs * kBlockCap * kBlockBins * per, 256) +
         align_up((size_t)n_jobs * kBlockCap * 32 * per, 256);
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
  const int64_t rows_a = (int64_t)1 << a;
  const int groups = merge_groups(k, __builtin_popcountll(mrg), 0);
  dd_merge_kernel<<<dim3(merge_grid(rows_a * n_jobs, 1, groups), 1, 1), 256, 0, st>>>(
      att, k, act, mrg, zm, zv, zoom_dev, ZoomFromJobs{}, n_jobs, rows_a, __builtin_popcountll(mrg), 0, out);
  CUTQC_LAUNCH_CHECK("dd_merge_kernel");
  return CUTQC_OK;
}

}  // namespace

}  // namespace cutqc

// ------------------------------------------------- shapes of a DD level
// (declared in dd_host.cuh; also used by the persistent kernel's builder)
namespace cutqc {

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

// Workspace of one step: the contraction plan's (for the given precision;
// for FP32 sized for any bin order) and the chunked top-T candidates.
int dd_step_ws(int n_sub, const cutqc_subcircuit* s, const int32_t* active_bits, int n_jobs, int precision,
                      size_t* bytes, int64_t min_tc_outputs) {
  if (min_tc_outputs < 0) min_tc_outputs = kDdMinTcOutputs;
  if (!bytes) return set_error(CUTQC_EINVAL, "null bytes");
  std::vector<TensorDesc> in;
  int tot = 0;
  // the bin order decides which operands need a gather copy: plan with the
  // identity order and size for the worst case
  std::vector<int32_t> ident;
  for (int i = 0; i < n_sub && active_bits; ++i)
    for (int b = 0; b < active_bits[i]; ++b) ident.push_back((int32_t)ident.size());
  int rc = dd_inputs(n_sub, s, active_bits, ident.data(), &in, &tot);
  if (rc) return rc;
  if (n_jobs < 1) return set_error(CUTQC_EINVAL, "n_jobs must be >= 1");
  ContractionPlan plan;
  if ((rc = plan_contraction_batched(in, precision, n_jobs, &plan, true, min_tc_outputs))) return rc;
  *bytes = align_up(plan.ws_bytes, 256) + topk_scratch((int64_t)1 << tot, n_jobs) +
           block_max_scratch((int64_t)1 << tot, n_jobs);
  return CUTQC_OK;
}

int level_shape(int n_sub, const cutqc_subcircuit* s, int n, int M, int depth, LevelShape* L) {
  L->depth = depth;
  L->active.clear();
  for (int q = depth * M; q < std::min(n, depth * M + M); ++q) L->active.push_back(q);
  const int lo = depth * M, hi = depth * M + (int)L->active.size();
  L->active_bits.assign(n_sub, 0);
  L->bin_bit.clear();
  L->act_mask.assign(n_sub, 0);
  L->zoom_mask.assign(n_sub, 0);
  for (int i = 0; i < n_sub; ++i) {
    const int o = s[i].w - s[i].k_out;
    for (int t = 0; t < o; ++t) {
      const int q = s[i].out_qubit[t];
      if (q < 0 || q >= n) return set_error(CUTQC_EINVAL, "out_qubit %d outside 0..%d", q, n - 1);
      if (q >= lo && q < hi) {
        L->act_mask[i] |= (uint64_t)1 << t;
        L->active_bits[i]++;
        L->bin_bit.push_back(q - lo);
      } else if (q < lo) {
        L->zoom_mask[i] |= (uint64_t)1 << t;
      }
    }
  }
  return CUTQC_OK;
}

// Workspace for one level of n_jobs jobs.
// merge_ctas: about how many CTAs share one subcircuit's merge (slices of the
// merged index range, each at least 64 long)
int level_layout(int n_sub, const cutqc_subcircuit* s, const LevelShape& L, int n_jobs, RunLayout* R,
                 int merge_ctas) {
  size_t ws = 0;
  auto take = [&](size_t b) { size_t o = ws; ws = align_up(ws + b, 256); return o; };
  for (int i = 0; i < n_sub; ++i) {
    const int k = s[i].k_in + s[i].k_out;
    const size_t elems = (size_t)n_jobs * ((size_t)1 << L.active_bits[i]) * ((size_t)1 << (2 * k));
    R->merged_off[i] = take(elems * sizeof(float));
    R->zoom_off[i] = take((size_t)n_jobs * sizeof(uint64_t));
    const int o = s[i].w - s[i].k_out;
    const int n_merged = o - L.active_bits[i] - __builtin_popcountll(L.zoom_mask[i]);
    int ls = 0;
    while (ls < n_merged - 6 && ((int64_t)n_jobs << (L.active_bits[i] + ls + 1)) <= merge_ctas) ++ls;
    R->log_slices[i] = ls;
    R->part_off[i] = ls ? take(elems * ((size_t)1 << ls) * sizeof(float)) : 0;
  }
  // enough for either precision and any tensor-core size floor (the
  // default one, or every step on the split path)
  size_t step = 0, step_tc = 0, step_all_tc = 0;
  int rc = dd_step_ws(n_sub, s, L.active_bits.data(), n_jobs, CUTQC_PREC_FP32_SIMT, &step);
  if (rc) return rc;
  if ((rc = dd_step_ws(n_sub, s, L.active_bits.data(), n_jobs, CUTQC_PREC_FP16X3_TC_PRUNE, &step_tc))) return rc;
  if ((rc = dd_step_ws(n_sub, s, L.active_bits.data(), n_jobs, CUTQC_PREC_FP16X3_TC_PRUNE, &step_all_tc, 0)))
    return rc;
  step = std::max(step, std::max(step_tc, step_all_tc));
  R->step_off = take(step);
  R->top_idx_off = take((size_t)n_jobs * 32 * sizeof(int32_t));
  R->top_val_off = take((size_t)n_jobs * 32 * sizeof(float));
  R->sum_off = take((size_t)n_jobs * sizeof(double));
  R->total = ws;
  return CUTQC_OK;
}

int validate_run(int n_sub, const cutqc_subcircuit* s, int n, int M, int T) {
  if (n_sub < 1 || n_sub > 64) return set_error(CUTQC_EINVAL, "n_sub must be in 1..64");
  if (n < 1 || n > 128) return set_error(CUTQC_EUNSUPPORTED, "n_qubits must be in 1..128");
  if (M < 1 || M > 30) return set_error(CUTQC_EUNSUPPORTED, "M must be in 1..30");
  if (T < 0 || T > 32) return set_error(CUTQC_EUNSUPPORTED, "T must be in 0..32");
  int tot = 0;
  for (int i = 0; i < n_sub; ++i) {
    int rc = validate_subcircuit(&s[i]);
    if (rc) return rc;
    tot += s[i].w - s[i].k_out;
  }
  if (tot != n) return set_error(CUTQC_EINVAL, "outputs (%d) != n_qubits (%d)", tot, n);
  return CUTQC_OK;
}

// Level workspace (reused by every level) and, after it, room for the job
// records of a level-synchronous run (used by cutqc_dd_run).
int run_ws(int n_sub, const cutqc_subcircuit* s, int n, int M, int T, size_t* level_bytes, size_t* total) {
  size_t best = 0;
  const int depths = (n + M - 1) / M;
  for (int d = 0; d < depths; ++d) {
    LevelShape L;
    int rc = level_shape(n_sub, s, n, M, d, &L);
    if (rc) return rc;
    RunLayout R;
    if ((rc = level_layout(n_sub, s, L, std::max(1, T), &R, kMergeCtasMax))) return rc;
    best = std::max(best, R.total);
  }
  const size_t records = 1 + (size_t)(depths - 1) * std::max(1, T);
  *level_bytes = align_up(best, 256);
  *total = *level_bytes + align_up(records * sizeof(cutqc_dd_job_result), 256) + 256;
  return CUTQC_OK;
}

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
  return dd_step_ws(n_sub, s, active_bits, n_jobs, CUTQC_PREC_FP32_SIMT, bytes);
}

// The T largest of each job's nb entries (vals + job * nb) into top_idx /
// top_val [n_jobs][T]: one CTA per job, or for large jobs a chunked pass
// into the candidate scratch cand (topk_scratch(nb, n_jobs) bytes) and one
// CTA per job over the chunks' candidates.  gate: as for dd_topk_kernel.
static int launch_topk_scan(const float* vals, int64_t nb, int n_jobs, int topk, int cap, int32_t* cand,
                            int32_t* top_idx, float* top_val, const int* gate, int gate_cap, cudaStream_t st,
                            int64_t min_chunk = kTopkChunkMin) {
  const int64_t chunks = topk_chunks(nb, min_chunk);
  if (chunks == 1) {
    const int threads = (int)std::min<int64_t>(cap, std::max<int64_t>(32, (nb + 31) / 32 * 32));
    if (topk <= 4)
      dd_topk_kernel<4, false><<<dim3(n_jobs, 1), threads, 0, st>>>(vals, nullptr, nb, nb, topk, top_idx, top_val,
                                                                    gate, gate_cap);
    else
      dd_topk_kernel<32, false><<<dim3(n_jobs, 1), threads, 0, st>>>(vals, nullptr, nb, nb, topk, top_idx, top_val,
                                                                     gate, gate_cap);
  } else {
    int32_t* cidx = cand;
    float* cval = (float*)(cidx + (size_t)n_jobs * chunks * 32);
    const int64_t clen = (nb + chunks - 1) / chunks;
    const int64_t ncand = chunks * topk;
    const int64_t cthreads = std::min<int64_t>(cap, 512);   // several CTAs per SM: more loads in flight
    if (topk <= 4) {
      dd_topk_kernel<4, false><<<dim3(n_jobs, (unsigned)chunks), (int)cthreads, 0, st>>>(vals, nullptr, nb, clen,
                                                                                        topk, cidx, cval, gate,
                                                                                        gate_cap);
      CUTQC_LAUNCH_CHECK("dd_topk_kernel (chunks)");
      dd_topk_kernel<4, true><<<dim3(n_jobs, 1), 1024, 0, st>>>(cval, cidx, ncand, ncand, topk, top_idx, top_val,
                                                                gate, gate_cap);
    } else {
      dd_topk_kernel<32, false><<<dim3(n_jobs, (unsigned)chunks), (int)cthreads, 0, st>>>(vals, nullptr, nb, clen,
                                                                                         topk, cidx, cval, gate,
                                                                                         gate_cap);
      CUTQC_LAUNCH_CHECK("dd_topk_kernel (chunks)");
      dd_topk_kernel<32, true><<<dim3(n_jobs, 1), 1024, 0, st>>>(cval, cidx, ncand, ncand, topk, top_idx, top_val,
                                                                 gate, gate_cap);
    }
  }
  CUTQC_LAUNCH_CHECK("dd_topk_kernel");
  return CUTQC_OK;
}

// topk_threads: threads per job of the top-T pass (0: up to 1024).
// precision: CUTQC_PREC_FP32_SIMT, or CUTQC_PREC_FP16X3_TC(_PRUNE) for jobs
// of at least 4 bins whose bins start 16-byte aligned (smaller ones take
// FP32).
static int dd_step_impl(int n_sub, const cutqc_subcircuit* s, const int32_t* active_bits, const int32_t* bin_bit,
                        int n_jobs, const float* const* merged, float* bins, double* bin_sum, int topk,
                        int32_t* top_idx, float* top_val, void* ws_dev, size_t ws_bytes, void* stream,
                        int topk_threads, int precision = CUTQC_PREC_FP32_SIMT,
                        int64_t min_tc_outputs = kDdMinTcOutputs) {
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
  if (precision != CUTQC_PREC_FP32_SIMT && precision != CUTQC_PREC_FP16X3_TC && precision != CUTQC_PREC_FP16X3_TC_PRUNE)
    return set_error(CUTQC_EINVAL, "unknown precision %d", precision);
  const int64_t nb = (int64_t)1 << tot;
  if (precision != CUTQC_PREC_FP32_SIMT && (nb < 4 || ((uintptr_t)bins & 15) != 0)) precision = CUTQC_PREC_FP32_SIMT;
  ContractionPlan plan;
  if ((rc = plan_contraction_batched(in, precision, n_jobs, &plan, false, min_tc_outputs))) return rc;
  const size_t plan_ws = align_up(plan.ws_bytes, 256);
  const size_t topk_ws = topk_scratch(nb, n_jobs);
  const size_t bmax_ws = topk > 0 ? block_max_scratch(nb, n_jobs) : 0;
  const size_t need = plan_ws + topk_ws + bmax_ws;
  if (ws_bytes < need || (need && !ws_dev)) return set_error(CUTQC_ENOMEM, "DD workspace needs %zu bytes", need);
  cudaStream_t st = (cudaStream_t)stream;
  std::vector<int64_t> bstride(n_sub);
  for (int i = 0; i < n_sub; ++i) bstride[i] = ((int64_t)1 << in[i].o) << (2 * in[i].edges.size());
  if (bin_sum) CUTQC_CUDA_TRY(cudaMemsetAsync(bin_sum, 0, sizeof(double) * n_jobs, st));
  uint8_t* bm = (uint8_t*)ws_dev + plan_ws + topk_ws;
  BlockMaxSink sink;
  if (bmax_ws) {
    sink.cmax = (float*)bm;
    sink.per_item = nb / kBlockBins;
    set_block_max_sink(&sink);
  }
  rc = run_plan(plan, merged, bstride.data(), n_jobs, bins, nb, bin_sum, std::ldexp(1.0f, -plan.K), precision, 0, -1,
                (uint8_t*)ws_dev, st);
  set_block_max_sink(nullptr);
  if (rc) return rc;
  if (topk > 0) {
    const int threads = topk_threads > 0 ? std::min(1024, std::max(32, topk_threads / 32 * 32)) : 1024;
    int32_t* cidx = (int32_t*)((uint8_t*)ws_dev + plan_ws);
    if (!sink.written) {
      if ((rc = launch_topk_scan(bins, nb, n_jobs, topk, threads, cidx, top_idx, top_val, nullptr, 0, st))) return rc;
      return CUTQC_OK;
    }
    // block maxima: the T largest of them, the blocks at or above the T-th,
    // their bins; the full scan runs only for jobs with more than
    // kBlockCap such blocks (maxima tied at the threshold)
    const int64_t C = sink.per_item;
    const size_t per = sizeof(int32_t) + sizeof(float);
    uint8_t* p = bm + align_up((size_t)n_jobs * C * sizeof(float), 256);
    int32_t* k1 = (int32_t*)p;
    p += topk_scratch(C, n_jobs, kBlockMaxChunk);
    int32_t* kidx = (int32_t*)p;
    float* kval = (float*)(kidx + (size_t)n_jobs * 32);
    p += align_up((size_t)n_jobs * 32 * per, 256);
    int* count = (int*)p;
    p += align_up((size_t)n_jobs * sizeof(int), 256);
    int32_t* list = (int32_t*)p;
    p += align_up((size_t)n_jobs * kBlockCap * sizeof(int32_t), 256);
    float* gv = (float*)p;
    int32_t* gi = (int32_t*)(gv + (size_t)n_jobs * kBlockCap * kBlockBins);
    p += align_up((size_t)n_jobs * kBlockCap * kBlockBins * per, 256);
    int32_t* bidx = (int32_t*)p;
    float* bval = (float*)(bidx + (size_t)n_jobs * kBlockCap * 32);
    if ((rc = launch_topk_scan(sink.cmax, C, n_jobs, topk, threads, k1, kidx, kval, nullptr, 0, st, kBlockMaxChunk)))
      return rc;
    CUTQC_CUDA_TRY(cudaMemsetAsync(count, 0, sizeof(int) * n_jobs, st));
    const int64_t cblocks = std::min<int64_t>((C + 255) / 256, (int64_t)sm_count() * 4);
    dd_block_collect<<<dim3((unsigned)cblocks, n_jobs), 256, 0, st>>>(sink.cmax, C, kidx, kval, topk, kBlockCap, count,
                                                                     list);
    CUTQC_LAUNCH_CHECK("dd_block_collect");
    dd_block_gather<<<dim3(kBlockCap, n_jobs), 256, 0, st>>>(bins, nb, count, list, kBlockCap,
                                                            (sink.N + kBlockCols - 1) / kBlockCols, sink.M, sink.N,
                                                            sink.mask_m, sink.mask_n, gv, gi);
    CUTQC_LAUNCH_CHECK("dd_block_gather");
    const int64_t gn = (int64_t)kBlockCap * kBlockBins, bn = (int64_t)kBlockCap * topk;
    if (topk <= 4) {
      dd_topk_kernel<4, true><<<dim3(n_jobs, kBlockCap), 256, 0, st>>>(gv, gi, gn, kBlockBins, topk, bidx, bval);
      CUTQC_LAUNCH_CHECK("dd_topk_kernel (blocks)");
      dd_topk_kernel<4, true><<<dim3(n_jobs, 1), 256, 0, st>>>(bval, bidx, bn, bn, topk, top_idx, top_val);
    } else {
      dd_topk_kernel<32, true><<<dim3(n_jobs, kBlockCap), 256, 0, st>>>(gv, gi, gn, kBlockBins, topk, bidx, bval);
      CUTQC_LAUNCH_CHECK("dd_topk_kernel (blocks)");
      dd_topk_kernel<32, true><<<dim3(n_jobs, 1), 256, 0, st>>>(bval, bidx, bn, bn, topk, top_idx, top_val);
    }
    CUTQC_LAUNCH_CHECK("dd_topk_kernel");
    // jobs whose maxima tied beyond the cap: the full scan, gated on the device
    if ((rc = launch_topk_scan(bins, nb, n_jobs, topk, threads, cidx, top_idx, top_val, count, kBlockCap, st)))
      return rc;
  }
  return CUTQC_OK;
}

extern "C" int cutqc_dd_step(int n_sub, const cutqc_subcircuit* s, const int32_t* active_bits, const int32_t* bin_bit,
                             int n_jobs, const float* const* merged, float* bins, double* bin_sum, int topk,
                             int32_t* top_idx, float* top_val, void* ws_dev, size_t ws_bytes, void* stream) {
  return dd_step_impl(n_sub, s, active_bits, bin_bit, n_jobs, merged, bins, bin_sum, topk, top_idx, top_val, ws_dev,
                      ws_bytes, stream, 0);
}

extern "C" int cutqc_sum_f64(const float* x, int64_t n, double* sum, void* stream) {
  if (!x || !sum || n < 0) return set_error(CUTQC_EINVAL, "bad arguments");
  if (n == 0) return CUTQC_OK;
  int blocks = (int)std::min<int64_t>((n / 16 + 255) / 256 + 1, (int64_t)sm_count() * 8);
  sum_f64_kernel<<<blocks, 256, 0, (cudaStream_t)stream>>>(x, n, sum);
  CUTQC_LAUNCH_CHECK("sum_f64_kernel");
  return CUTQC_OK;
}

// ---------------------------------------------------------------- Algorithm 1

namespace cutqc {
namespace {

__global__ void dd_select_kernel(cutqc_dd_job_result* __restrict__ jobs, int job0, int nj, LevelInfo L,
                                 int64_t bins_off0, int64_t nb, const double* __restrict__ bsum,
                                 const int32_t* __restrict__ tidx, const float* __restrict__ tval, int T,
                                 int has_children, int n_next, int32_t* __restrict__ n_jobs_dev) {
  if (blockIdx.x != 0) return;
  dd_select_body<false>(jobs, job0, nj, L, bins_off0, nb, bsum, tidx, tval, T, has_children, n_next, n_jobs_dev);
}

// The first job: nothing zoomed.
__global__ void dd_first_job_kernel(cutqc_dd_job_result* __restrict__ jobs) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  dd_first_job_body(jobs);
}

}  // namespace
}  // namespace cutqc

namespace cutqc {
namespace {

// Enqueue a level-synchronous run: no host synchronisation, no host copies.
int enqueue_levels(int n_sub, const cutqc_subcircuit* s, const float* const* att, int n, int M, int Rmax, int T,
                   int max_jobs, cutqc_dd_job_result* jobs_dev, int32_t* n_jobs_dev, float* bins, int64_t bins_cap,
                   uint8_t* ws, size_t ws_bytes, cudaStream_t st, const cutqc_dd_options* opt) {
  int merge_ctas = kMergeCtasDefault, topk_threads = 0, precision = CUTQC_PREC_FP32_SIMT;
  int64_t min_tc_outputs = kDdMinTcOutputs;
  if (opt) {
    if (opt->merge_ctas < 0 || opt->merge_ctas > kMergeCtasMax || opt->topk_threads < 0 || opt->topk_threads > 1024)
      return set_error(CUTQC_EINVAL, "options out of range (merge_ctas <= %d, topk_threads <= 1024)", kMergeCtasMax);
    if (opt->precision != CUTQC_PREC_FP32_SIMT && opt->precision != CUTQC_PREC_FP16X3_TC &&
        opt->precision != CUTQC_PREC_FP16X3_TC_PRUNE)
      return set_error(CUTQC_EINVAL, "options: unknown precision %d", opt->precision);
    if (opt->merge_ctas) merge_ctas = opt->merge_ctas;
    topk_threads = opt->topk_threads;
    precision = opt->precision;
    if (opt->tc_min_outputs < 0 || opt->tc_min_outputs > 62)
      return set_error(CUTQC_EINVAL, "options: tc_min_outputs must be in 0..62");
    if (opt->tc_min_outputs) min_tc_outputs = (int64_t)1 << (opt->tc_min_outputs - 1);
  }
  for (int i = 0; i < n_sub; ++i)
    if (s[i].w - s[i].k_out > 32) return set_error(CUTQC_EUNSUPPORTED, "more than 32 outputs in a subcircuit");
  const int depths = (n + M - 1) / M;
  const int levels = T > 0 ? std::min(Rmax, depths) : 1;   // T = 0 expands nothing
  const int Tn = std::max(1, T);
  // sizes first: every level's jobs and bins must fit
  {
    int64_t jobs_total = 0, bins_total = 0;
    for (int level = 0; level < levels; ++level) {
      const int nj = level == 0 ? 1 : Tn;
      const int na = std::min(n, level * M + M) - level * M;
      jobs_total += nj;
      bins_total += (int64_t)nj << na;
    }
    if (jobs_total > max_jobs) return set_error(CUTQC_ENOMEM, "a run of %d levels needs %lld job records", levels,
                                                (long long)jobs_total);
    if (bins_total > bins_cap) return set_error(CUTQC_ENOMEM, "bins_capacity too small (%lld needed)",
                                                (long long)bins_total);
  }
  dd_first_job_kernel<<<1, 32, 0, st>>>(jobs_dev);
  CUTQC_LAUNCH_CHECK("dd_first_job_kernel");
  int job0 = 0;
  int64_t bins_off = 0;
  for (int level = 0; level < levels; ++level) {
    const int nj = level == 0 ? 1 : Tn;
    LevelShape L;
    int rc = level_shape(n_sub, s, n, M, level, &L);
    if (rc) return rc;
    RunLayout lay;
    if ((rc = level_layout(n_sub, s, L, nj, &lay, merge_ctas))) return rc;
    if (lay.total > ws_bytes) return set_error(CUTQC_ENOMEM, "DD workspace too small for a level");
    std::vector<const float*> merged(n_sub);
    // the subcircuits' merges are independent: fork them over the side
    // streams, join before the reconstruction
    SideStreams* ss = nullptr;
    if ((rc = side_streams(st, &ss))) return rc;
    {
      std::lock_guard<std::mutex> side_lock(ss->mu);
      const int nside = std::min(n_sub, kSideStreams);
      CUTQC_CUDA_TRY(cudaEventRecord(ss->fork, st));
      for (int j = 0; j < nside; ++j) CUTQC_CUDA_TRY(cudaStreamWaitEvent(ss->s[j], ss->fork, 0));
      for (int i = 0; i < n_sub; ++i) {
        cudaStream_t ms = ss->s[i % nside];
        float* mdev = (float*)(ws + lay.merged_off[i]);
        const int o = s[i].w - s[i].k_out;
        const uint64_t all = o >= 64 ? ~0ull : (((uint64_t)1 << o) - 1);
        const uint64_t mrg = all & ~L.act_mask[i] & ~L.zoom_mask[i];
        const int k = s[i].k_in + s[i].k_out;
        const int a = __builtin_popcountll(L.act_mask[i]);
        const int ls = lay.log_slices[i];
        float* part = ls ? (float*)(ws + lay.part_off[i]) : mdev;
        // each job's zoom value comes from its record (written by the previous
        // level's selection on the device)
        ZoomFromJobs zj{};
        zj.jobs = jobs_dev + job0;
        zj.o = o;
        zj.lo = level * M;
        for (int t = 0; t < o; ++t) zj.outq[t] = (int8_t)s[i].out_qubit[t];
        const int64_t rows_a = (int64_t)1 << a;
        const int groups = merge_groups(k, __builtin_popcountll(mrg), ls);
        dd_merge_kernel<<<dim3(merge_grid(rows_a * nj, 1 << ls, groups), 1, 1u << ls), 256, 0, ms>>>(
            att[i], k, L.act_mask[i], mrg, L.zoom_mask[i], 0, nullptr, zj, nj, rows_a, __builtin_popcountll(mrg), ls,
            part);
        CUTQC_LAUNCH_CHECK("dd_merge_kernel");
        if (ls) {
          const int64_t E = ((int64_t)nj << a) << (2 * k);
          const int blocks = (int)std::min<int64_t>((E + 255) / 256, (int64_t)sm_count() * 8);
          dd_merge_reduce<<<blocks, 256, 0, ms>>>(part, 1 << ls, E, mdev);
          CUTQC_LAUNCH_CHECK("dd_merge_reduce");
        }
        merged[i] = mdev;
      }
      for (int j = 0; j < nside; ++j) {
        CUTQC_CUDA_TRY(cudaEventRecord(ss->join[j], ss->s[j]));
        CUTQC_CUDA_TRY(cudaStreamWaitEvent(st, ss->join[j], 0));
      }
    }
    const int64_t nb = (int64_t)1 << L.active.size();
    int32_t* tidx = (int32_t*)(ws + lay.top_idx_off);
    float* tval = (float*)(ws + lay.top_val_off);
    double* bsum = (double*)(ws + lay.sum_off);
    if ((rc = dd_step_impl(n_sub, s, L.active_bits.data(), L.bin_bit.data(), nj, merged.data(), bins + bins_off, bsum,
                           T, tidx, tval, ws + lay.step_off, lay.total - lay.step_off, st, topk_threads,
                           precision, min_tc_outputs)))
      return rc;
    LevelInfo li{};
    li.level = level;
    li.depth = level;
    li.n_active = (int)L.active.size();
    for (int a = 0; a < li.n_active; ++a) li.active[a] = (int8_t)L.active[a];
    const int has_children = level + 1 < levels && T > 0;
    dd_select_kernel<<<1, 32, 0, st>>>(jobs_dev, job0, nj, li, bins_off, nb, bsum, tidx, tval, T, has_children,
                                       has_children ? Tn : 0, n_jobs_dev);
    CUTQC_LAUNCH_CHECK("dd_select_kernel");
    job0 += nj;
    bins_off += nj * nb;
  }
  return CUTQC_OK;
}

}  // namespace
}  // namespace cutqc

extern "C" int cutqc_dd_run_workspace_size(int n_sub, const cutqc_subcircuit* s, int n, int M, int T,
                                           size_t* bytes) {
  int rc = validate_run(n_sub, s, n, M, T);
  if (rc) return rc;
  if (!bytes) return set_error(CUTQC_EINVAL, "null bytes");
  size_t level = 0;
  return run_ws(n_sub, s, n, M, T, &level, bytes);
}

extern "C" int cutqc_dd_run_async(int n_sub, const cutqc_subcircuit* s, const float* const* att, int n, int M, int Rmax,
                                  int T, int max_jobs, cutqc_dd_job_result* jobs_dev, int32_t* n_jobs_dev, float* bins,
                                  int64_t bins_cap, const cutqc_dd_options* opt, void* ws_dev, size_t ws_bytes,
                                  void* stream) {
  int rc = validate_run(n_sub, s, n, M, T);
  if (rc) return rc;
  if (!att || !jobs_dev || !n_jobs_dev || !bins || !ws_dev || max_jobs < 1 || Rmax < 1)
    return set_error(CUTQC_EINVAL, "bad arguments");
  for (int i = 0; i < n_sub; ++i)
    if (!att[i]) return set_error(CUTQC_EINVAL, "null attributed tensor");
  size_t level = 0, total = 0;
  if ((rc = run_ws(n_sub, s, n, M, T, &level, &total))) return rc;
  if (ws_bytes < level) return set_error(CUTQC_ENOMEM, "DD workspace needs %zu bytes", level);
  return enqueue_levels(n_sub, s, att, n, M, Rmax, T, max_jobs, jobs_dev, n_jobs_dev, bins, bins_cap,
                        (uint8_t*)ws_dev, ws_bytes, (cudaStream_t)stream, opt);
}

extern "C" int cutqc_dd_run(int n_sub, const cutqc_subcircuit* s, const float* const* att, int n, int M, int Rmax,
                            int T, int strategy, int max_jobs, cutqc_dd_job_result* jobs, int* n_jobs_out,
                            float* bins, int64_t bins_cap, void* ws_dev, size_t ws_bytes, void* stream) {
  int rc = validate_run(n_sub, s, n, M, T);
  if (rc) return rc;
  if (!att || !jobs || !n_jobs_out || !bins || max_jobs < 1 || Rmax < 1)
    return set_error(CUTQC_EINVAL, "bad arguments");
  if (strategy != 0 && strategy != 1) return set_error(CUTQC_EINVAL, "strategy must be 0 (DFS) or 1 (BFS)");
  size_t level_bytes = 0, need = 0;
  if ((rc = run_ws(n_sub, s, n, M, T, &level_bytes, &need))) return rc;
  if (ws_bytes < need || !ws_dev) return set_error(CUTQC_ENOMEM, "DD workspace needs %zu bytes", need);
  cudaStream_t st = (cudaStream_t)stream;
  uint8_t* ws = (uint8_t*)ws_dev;
  if (strategy == 1 || T <= 1) {
    // level-synchronous (depth first with T <= 1 is the same schedule): the
    // selection runs on the device, the records come back once at the end
    const int depths = (n + M - 1) / M;
    const size_t records = 1 + (size_t)(depths - 1) * std::max(1, T);
    cutqc_dd_job_result* jdev = (cutqc_dd_job_result*)(ws + level_bytes);
    int32_t* ndev = (int32_t*)(ws + level_bytes + align_up(records * sizeof(cutqc_dd_job_result), 256));
    if ((rc = enqueue_levels(n_sub, s, att, n, M, Rmax, T, (int)records, jdev, ndev, bins, bins_cap, ws, level_bytes,
                             st, nullptr)))
      return rc;
    int32_t nrec = 0;
    std::vector<cutqc_dd_job_result> host(records);
    CUTQC_CUDA_TRY(cudaMemcpyAsync(&nrec, ndev, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    CUTQC_CUDA_TRY(cudaMemcpyAsync(host.data(), jdev, records * sizeof(cutqc_dd_job_result), cudaMemcpyDeviceToHost, st));
    CUTQC_CUDA_TRY(cudaStreamSynchronize(st));
    int out = 0;
    for (int r = 0; r < nrec && r < (int)records; ++r) {
      if (host[r].level < 0) continue;
      if (out >= max_jobs) return set_error(CUTQC_ENOMEM, "more than max_jobs jobs");
      cutqc_dd_job_result J = host[r];
      jobs[out++] = J;
    }
    // parents index the compacted list
    std::vector<int> remap(records, -1);
    for (int r = 0, k = 0; r < nrec && r < (int)records; ++r)
      if (host[r].level >= 0) remap[r] = k++;
    for (int j = 0; j < out; ++j)
      if (jobs[j].parent >= 0) jobs[j].parent = remap[jobs[j].parent];
    *n_jobs_out = out;
    return CUTQC_OK;
  }
  int n_jobs = 0;
  int64_t bins_used = 0;
  struct Pending { double value; int parent; int bin; int depth; uint64_t zm[2], zv[2]; };
  auto qbit = [](const uint64_t* m, int q) { return (m[q >> 6] >> (q & 63)) & 1; };
  // run one level: all `todo` entries share `depth`
  auto run_level = [&](int level, std::vector<Pending>& todo, std::vector<int>* new_jobs) -> int {
    const int depth = todo[0].depth;
    const int nj = (int)todo.size();
    LevelShape L;
    int r = level_shape(n_sub, s, n, M, depth, &L);
    if (r) return r;
    RunLayout lay;
    if ((r = level_layout(n_sub, s, L, nj, &lay))) return r;
    if (lay.total > ws_bytes) return set_error(CUTQC_ENOMEM, "DD workspace too small for a level");
    if (n_jobs + nj > max_jobs) return set_error(CUTQC_ENOMEM, "more than max_jobs jobs");
    const int64_t nb = (int64_t)1 << L.active.size();
    if (bins_used + nb * nj > bins_cap) return set_error(CUTQC_ENOMEM, "bins_capacity too small");
    // per subcircuit zoom values of each job (over its output bits)
    std::vector<const float*> merged(n_sub);
    for (int i = 0; i < n_sub; ++i) {
      const int o = s[i].w - s[i].k_out;
      std::vector<uint64_t> zv(nj, 0);
      for (int j = 0; j < nj; ++j)
        for (int t = 0; t < o; ++t) {
          const int q = s[i].out_qubit[t];
          if (((L.zoom_mask[i] >> t) & 1) && qbit(todo[j].zv, q)) zv[j] |= (uint64_t)1 << t;
        }
      uint64_t* zdev = (uint64_t*)(ws + lay.zoom_off[i]);
      CUTQC_CUDA_TRY(cudaMemcpyAsync(zdev, zv.data(), nj * sizeof(uint64_t), cudaMemcpyHostToDevice, st));
      float* mdev = (float*)(ws + lay.merged_off[i]);
      r = cutqc_dd_merge_batch(&s[i], att[i], L.act_mask[i], L.zoom_mask[i], nj, zdev, mdev, st);
      if (r) return r;
      merged[i] = mdev;
      // the pageable source of the copy above must outlive it
      CUTQC_CUDA_TRY(cudaStreamSynchronize(st));
    }
    float* bdev = bins + bins_used;
    int32_t* tidx = (int32_t*)(ws + lay.top_idx_off);
    float* tval = (float*)(ws + lay.top_val_off);
    double* bsum = (double*)(ws + lay.sum_off);
    r = cutqc_dd_step(n_sub, s, L.active_bits.data(), L.bin_bit.data(), nj, merged.data(), bdev, bsum, T, tidx, tval,
                      ws + lay.step_off, lay.total - lay.step_off, st);
    if (r) return r;
    std::vector<int32_t> hidx((size_t)nj * std::max(1, T));
    std::vector<float> hval((size_t)nj * std::max(1, T));
    std::vector<double> hsum(nj);
    if (T > 0) {
      CUTQC_CUDA_TRY(cudaMemcpyAsync(hidx.data(), tidx, (size_t)nj * T * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
      CUTQC_CUDA_TRY(cudaMemcpyAsync(hval.data(), tval, (size_t)nj * T * sizeof(float), cudaMemcpyDeviceToHost, st));
    }
    CUTQC_CUDA_TRY(cudaMemcpyAsync(hsum.data(), bsum, nj * sizeof(double), cudaMemcpyDeviceToHost, st));
    CUTQC_CUDA_TRY(cudaStreamSynchronize(st));
    for (int j = 0; j < nj; ++j) {
      cutqc_dd_job_result& J = jobs[n_jobs];
      memset(&J, 0, sizeof(J));
      J.level = level;
      J.depth = depth;
      J.parent = todo[j].parent;
      J.parent_bin = todo[j].bin;
      J.n_active = (int)L.active.size();
      for (int a = 0; a < J.n_active; ++a) J.active[a] = L.active[a];
      for (int w = 0; w < 2; ++w) { J.zoom_mask[w] = todo[j].zm[w]; J.zoom_val[w] = todo[j].zv[w]; }
      J.bin_sum = hsum[j];
      for (int t = 0; t < 32; ++t) { J.top_idx[t] = -1; J.top_val[t] = 0.f; }
      for (int t = 0; t < T; ++t) { J.top_idx[t] = hidx[(size_t)j * T + t]; J.top_val[t] = hval[(size_t)j * T + t]; }
      J.bins_offset = bins_used + (int64_t)j * nb;
      new_jobs->push_back(n_jobs);
      ++n_jobs;
    }
    bins_used += nb * nj;
    return CUTQC_OK;
  };
  // children of a job: its top bins, if merged qubits remain
  auto children = [&](int jid, std::vector<Pending>* out) {
    const cutqc_dd_job_result& J = jobs[jid];
    if ((J.depth + 1) * M >= n) return;          // nothing left to merge
    for (int t = 0; t < T; ++t) {
      const int b = J.top_idx[t];
      if (b < 0) continue;
      Pending p{};
      p.value = J.top_val[t];
      p.parent = jid;
      p.bin = b;
      p.depth = J.depth + 1;
      for (int w = 0; w < 2; ++w) { p.zm[w] = J.zoom_mask[w]; p.zv[w] = J.zoom_val[w]; }
      for (int a = 0; a < J.n_active; ++a) {
        const int q = J.active[a];
        p.zm[q >> 6] |= (uint64_t)1 << (q & 63);
        if ((b >> a) & 1) p.zv[q >> 6] |= (uint64_t)1 << (q & 63);
      }
      out->push_back(p);
    }
  };
  auto by_value = [](const Pending& a, const Pending& b) { return a.value > b.value; };
  std::vector<Pending> first(1);
  first[0].parent = -1;
  first[0].bin = -1;
  first[0].depth = 0;
  if (strategy == 1) {
    std::vector<Pending> todo = first;
    for (int level = 0; level < Rmax && !todo.empty(); ++level) {
      std::vector<int> made;
      if ((rc = run_level(level, todo, &made))) return rc;
      std::vector<Pending> cand;
      for (int jid : made) children(jid, &cand);
      std::stable_sort(cand.begin(), cand.end(), by_value);
      if ((int)cand.size() > T) cand.resize(T);
      todo = cand;
    }
  } else {
    std::vector<Pending> Lst;
    Pending cur = first[0];
    for (int r = 0; r < Rmax; ++r) {
      std::vector<Pending> one{cur};
      std::vector<int> made;
      if ((rc = run_level(r, one, &made))) return rc;
      children(made[0], &Lst);
      std::stable_sort(Lst.begin(), Lst.end(), by_value);
      if ((int)Lst.size() > T) Lst.resize(T);
      if (Lst.empty()) break;
      cur = Lst.front();
      Lst.erase(Lst.begin());
    }
  }
  *n_jobs_out = n_jobs;
  return CUTQC_OK;
}
