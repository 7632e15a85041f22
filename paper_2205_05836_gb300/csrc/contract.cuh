// Declarations shared by the contraction translation units.
#pragma once

#include "internal.cuh"

#include <mutex>
#include <vector>

namespace cutqc {

// True if mask == 2^b - 1 for some b (the low bits, in order).
inline bool mask_is_low(uint64_t mask) { return (mask & (mask + 1)) == 0; }

// If mask is one contiguous run of bits starting at bit s, return s, else -1.
inline int mask_contig_shift(uint64_t mask) {
  if (mask == 0) return 0;
  int s = __builtin_ctzll(mask);
  uint64_t run = mask >> s;
  return ((run & (run + 1)) == 0) ? s : -1;
}

int validate_subcircuit(const cutqc_subcircuit* s);

// Row-bit map of an operand gather: operand row bit j comes from source row
// bit bit[j] (only when permute != 0).
struct RowMap {
  int8_t bit[40];
  int n;
  int permute;
};

// Operand gather of rows [row0, row0 + rows): float32 (out32 != null) or
// float16 hi/lo with a power-of-two scale per row; K padded with zeros to Kp.
// batch > 1: item b reads v.src + b * src_bstride and writes rows * Kp
// elements (rows scales) further per item.  gmax != null (half mode, batch
// 1): one scale for the whole operand, written to scale[0]; gmax is a device
// word of scratch.
// cols/meta (device, nullable): gather only operand columns cols[0..meta[0])
// (cut-term pruning), zero-fill to meta[2], leave the rest of each row.
// gmax_ready: *gmax already holds the operand's max |x| (written by the
// GEMM that produced the source tensor), so the max pass is skipped; only
// for an operand that covers its source tensor (prep_covers_source).
int launch_prep_rows(const OperandView& v, const int* row_bits, int n_bits, int64_t row0, int64_t rows,
                     int64_t Kp, float* out32, __half* hi, __half* lo, float* scale, cudaStream_t st,
                     int batch = 1, int64_t src_bstride = 0, unsigned int* gmax = nullptr,
                     const int* cols = nullptr, const int* meta = nullptr, bool gmax_ready = false);
// True when operand rows [row0, row0 + rows) of the view are every element of
// its source tensor, each once (all rows; the open and shared digits are all
// of the source's digits; a 16-byte aligned source).
bool prep_covers_source(const OperandView& v, int64_t row0, int64_t rows);

// Cut-term pruning of one contraction (row operand rows [a_row0, +a_rows),
// column operand all b_rows rows): per term k the bound w_k = alpha *
// sum|A[.][k]| * sum|B[.][k]|; the terms of smallest bound whose total is
// <= tol are dropped.  colw: 3K floats of scratch; cols: K ints (kept terms,
// ascending); meta: 4 ints {kept, k-blocks, kept rounded up to 64, dropped};
// gmax_b: the largest |B| over the kept columns (float bits), the column
// operand's scale for launch_prep_rows with that column list.
constexpr int64_t kPruneMaxK = 1024;   // larger contractions are not pruned
inline size_t prune_scratch_bytes(int64_t K) {
  return align_up((size_t)K * (3 * sizeof(float) + sizeof(int)) + 4 * sizeof(int), 256);
}
int launch_prune_select(const OperandView& va, const int* a_bits, int a_nbits, int64_t a_row0, int64_t a_rows,
                        const OperandView& vb, const int* b_bits, int b_nbits, int64_t b_rows, float alpha,
                        double tol, float* colw, int* cols, int* meta, unsigned int* gmax_b, cudaStream_t st);

// float32 CUDA-core GEMM with bit-deposit epilogue.
// batch > 1: item b uses A + b*a_bstride, B + b*b_bstride, out + b*out_bstride,
// sum + b.
int launch_sgemm(const float* A, int64_t lda, const float* B, int64_t ldb, int64_t M, int64_t N,
                 int64_t K, float alpha, uint64_t mask_m, uint64_t mask_n, float* out, double* sum,
                 int streaming, cudaStream_t st, int batch = 1, int64_t a_bstride = 0, int64_t b_bstride = 0,
                 int64_t out_bstride = 0);

// Side streams per (device, caller stream) for independent work inside one
// call (a level's merges, independent contraction steps), forked from and
// joined back into the caller's stream with events (a CUDA graph capture
// records them as edges).  Hold `mu` from the fork to the join.
constexpr int kSideStreams = 8;
constexpr int kSideEvents = 64;
struct SideStreams {
  std::mutex mu;
  cudaStream_t s[kSideStreams];
  cudaEvent_t fork, join[kSideStreams];
  cudaEvent_t done[kSideEvents];   // per contraction step
};
int side_streams(cudaStream_t caller, SideStreams** out);

// ------------------------------------------------------- contraction plans
// A tensor [2^o][4^|edges|] whose row bit b lands at output position pos[b].
struct TensorDesc {
  int o = 0;
  std::vector<int> edges;   // ascending
  std::vector<int> pos;
};

struct PlanOperand {
  int tensor = -1;
  OperandView view{};
  bool trivial = false;
  std::vector<int> row_bits;
  size_t off32 = 0, off_hi = 0, off_lo = 0, off_scale = 0;
};

struct PlanStage {
  int a = -1, b = -1, result = -1;
  bool final_stage = false;
  bool tc = false;          // tensor-core split path (else FP32 on CUDA cores)
  bool outer = false;       // last step over K <= 16 terms: the FP32 outer-product kernel (outer.cu)
  PlanOperand opa, opb;
  int64_t M = 0, N = 0, K = 0, Kp = 0;
  uint64_t mask_m = 0, mask_n = 0;
  size_t off_result = 0;
  size_t result_elems = 0;
  size_t off_prune = 0;     // cut-term pruning scratch of the last step (per batch item)
};

struct ContractionPlan {
  std::vector<TensorDesc> tensors;
  std::vector<int> stage_of;          // per tensor: producing stage or -1
  std::vector<PlanStage> stages;
  int K = 0;                          // number of distinct cut edges
  int n = 0;                          // output bits
  size_t ws_bytes = 0;                // per batch item
  int64_t final_rows = 1, final_cols = 1;
};

// Greedy pairwise plan over the input tensors; every edge must appear in
// exactly two inputs.
int plan_contraction(const std::vector<TensorDesc>& inputs, int precision, ContractionPlan* plan);
// ws_upper_bound: size the workspace as if every operand needed its gather
// copy, so that the size holds for any output-bit order of the inputs.
// min_tc_outputs: under a tensor-core precision, steps with fewer outputs
// over all batch items (M * N * batch) run in FP32 on CUDA cores (at least
// as accurate; for small steps the split's operand preps cost more than the
// GEMM saves).
int plan_contraction_batched(const std::vector<TensorDesc>& inputs, int precision, int batch,
                             ContractionPlan* plan, bool ws_upper_bound = false, int64_t min_tc_outputs = 0);

// Runs the plan for `batch` independent items: input i of item b at
// inputs[i] + b * in_bstride[i]; output of item b at out + b * out_bstride;
// sum + b (if sum).  Workspace: plan.ws_bytes * batch.  in_ready (nullable):
// one event per input (null entries allowed) that the steps reading that
// input wait for on their stream.
int run_plan(const ContractionPlan& plan, const float* const* inputs, const int64_t* in_bstride, int batch,
             float* out, int64_t out_bstride, double* sum, float alpha, int precision, int64_t row_begin,
             int64_t row_end, uint8_t* ws, cudaStream_t st, const cudaEvent_t* in_ready = nullptr);

// Last step over few cut terms: P[m][n] = alpha * sum_k A[m][k] B[n][k] in
// FP32 on CUDA cores, row-major in n (mask_n the low bits), K in {1, 4, 16},
// M a multiple of 32, N of 128, at least 2^22 outputs; sum (nullable) gets the float64 total and
// cmax (nullable) the 32 x 64 block maxima laid out as for the paired GEMM.
bool outer_small_k_supported(int64_t K, int64_t M, int64_t N, uint64_t mask_m, uint64_t mask_n);
int launch_outer_small_k(const float* A, int64_t lda, const float* B, int64_t ldb, int64_t M, int64_t N, int64_t K,
                         float alpha, uint64_t mask_m, uint64_t mask_n, float* out, double* sum, float* cmax,
                         cudaStream_t st);

// Tensor-core GEMM (tcgen05, FP16 hi/lo split, three products) with the same
// epilogue; operands from launch_prep_rows in half mode with Kp % 64 == 0:
// the row operand with per-row scales, the column operand with one scale
// (scale[0]).
struct TcOperand {
  const __half* hi;
  const __half* lo;
  const float* scale;
  int64_t rows;
};
// Pairs of SMs (tcgen05 cta_group::2) with A resident, for Kp <= 256.
bool tc_pair_supported(int64_t Kp);
// num_kb_dev (nullable, device): the number of 64-wide k-blocks to use,
// read by the kernel (at most Kp / 64); the operands' row stride stays Kp.
// cmax (nullable, device, paired kernel only): for each 32-row x 64-column
// block of the M x N result (stripe r = m / 32, block c = n / 64) its largest
// value at cmax[r * ceil(N / 64) + c].  amax (nullable, device, paired kernel
// only, not with cmax): atomicMax of the float bits of every |output| (the
// caller zeroes it first).
int launch_tc_pair_gemm(const TcOperand& a, const TcOperand& b, int64_t Kp, float alpha, uint64_t mask_m,
                        uint64_t mask_n, float* out, double* sum, int streaming, cudaStream_t st,
                        const int* num_kb_dev = nullptr, float* cmax = nullptr, unsigned int* amax = nullptr);
int launch_tc_gemm(const TcOperand& a, const TcOperand& b, int64_t Kp, float alpha, uint64_t mask_m,
                   uint64_t mask_n, float* out, double* sum, int streaming, cudaStream_t st,
                   const int* num_kb_dev = nullptr, float* cmax = nullptr, unsigned int* amax = nullptr);

// Block maxima of the final step's output (DD's top-T selection).  Set on
// the calling thread around run_plan: when the final step runs on the paired
// tensor-core GEMM (M >= 32, N >= 64) or as outer products
// (launch_outer_small_k), over the full row range, with ceil(M/32) *
// ceil(N/64) == per_item, it writes item b's block maxima at cmax + b *
// per_item (layout as for launch_tc_pair_gemm) and records the output
// geometry; otherwise `written` stays false.
struct BlockMaxSink {
  float* cmax = nullptr;
  int64_t per_item = 0;
  bool written = false;
  int64_t M = 0, N = 0;
  uint64_t mask_m = 0, mask_n = 0;
};
void set_block_max_sink(BlockMaxSink* sink);   // nullptr: none

}  // namespace cutqc
