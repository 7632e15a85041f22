// Full-definition reconstruction (Eq. 1) over any number of subcircuits.
//
// Host planner: greedy pairwise contraction order (cheapest contraction
// first, pairs that share a cut edge before pairs that do not).  Each tensor
// carries, for each of its row bits, the position that bit takes in the final
// output (Kronecker order: subcircuit 0's bits most significant; original
// order: the uncut qubit index), and its open cut edges (ascending id).  A
// step gathers its two operands K-major over the shared edges (prep) and runs
// one GEMM whose epilogue deposits m and n bits into the result index: the
// intermediate layout [rows][open-edge digits] for inner steps, the requested
// output order for the last step.  The 2^-K normalisation of Eq. 1 is applied
// exactly (power of two) by the last step.
#include "internal.cuh"
#include "contract.cuh"

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

namespace cutqc {

// ---------------------------------------------------------------- errors

static thread_local std::string g_last_error;

// Events that the next reconstruction on this thread records around its last
// contraction's GEMM launch (then clears): see cutqc_fd_timing_events.
static thread_local cudaEvent_t g_gemm_start = nullptr, g_gemm_stop = nullptr;

// Readiness events of the next reconstruction's inputs on this thread (one
// per subcircuit, null = ready at the call): see cutqc_fd_input_events.
static thread_local std::vector<cudaEvent_t> g_input_events;

// Block maxima requested for the next final step on this thread.
static thread_local BlockMaxSink* g_bmax = nullptr;
void set_block_max_sink(BlockMaxSink* sink) { g_bmax = sink; }

int set_error(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return code;
}

static std::atomic<long long> g_launches{0};

void count_launches(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

int cuda_error(cudaError_t e, const char* where) {
  return set_error(CUTQC_ECUDA, "%s: %s", where, cudaGetErrorString(e));
}

static std::mutex g_dev_mu;
static std::map<int, int*> g_status;
static std::map<int, int> g_sms;

int* device_status_ptr() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
  std::lock_guard<std::mutex> lk(g_dev_mu);
  auto it = g_status.find(dev);
  if (it != g_status.end()) return it->second;
  int* p = nullptr;
  if (cudaMalloc(&p, sizeof(int)) != cudaSuccess) return nullptr;
  if (cudaMemset(p, 0, sizeof(int)) != cudaSuccess) return nullptr;
  g_status[dev] = p;
  return p;
}

int sm_count() {
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lk(g_dev_mu);
  auto it = g_sms.find(dev);
  if (it != g_sms.end()) return it->second;
  int n = 0;
  cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
  if (n <= 0) n = 1;
  g_sms[dev] = n;
  return n;
}

// Side streams per (device, caller stream), created once and kept for the
// process: a level's merges are independent and run on them, forked from
// and joined back into the caller's stream with events, which a CUDA graph
// capture records as edges.  Separate sets per caller stream keep runs on
// different streams independent; the set's mutex is held from the fork to
// the join so that two host threads never interleave on its events.
int side_streams(cudaStream_t caller, SideStreams** out) {
  static std::mutex mu;
  static std::map<std::pair<int, cudaStream_t>, SideStreams*> pool;
  int dev = 0;
  CUTQC_CUDA_TRY(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(mu);
  auto key = std::make_pair(dev, caller);
  if (pool.size() >= 64 && !pool.count(key)) key.second = nullptr;   // many streams: share one set
  auto it = pool.find(key);
  if (it == pool.end()) {
    SideStreams* p = new SideStreams();
    for (int i = 0; i < kSideStreams; ++i) {
      CUTQC_CUDA_TRY(cudaStreamCreateWithFlags(&p->s[i], cudaStreamNonBlocking));
      CUTQC_CUDA_TRY(cudaEventCreateWithFlags(&p->join[i], cudaEventDisableTiming));
    }
    for (int i = 0; i < kSideEvents; ++i)
      CUTQC_CUDA_TRY(cudaEventCreateWithFlags(&p->done[i], cudaEventDisableTiming));
    CUTQC_CUDA_TRY(cudaEventCreateWithFlags(&p->fork, cudaEventDisableTiming));
    it = pool.emplace(key, p).first;
  }
  *out = it->second;
  return CUTQC_OK;
}

// ---------------------------------------------------------------- planning

namespace {

uint64_t digit_mask(const std::vector<int>& all_edges, const std::vector<int>& subset) {
  uint64_t m = 0;
  for (int e : subset) {
    auto it = std::lower_bound(all_edges.begin(), all_edges.end(), e);
    int r = (int)(it - all_edges.begin());
    m |= (uint64_t)3 << (2 * r);
  }
  return m;
}

}  // namespace

int plan_contraction_batched(const std::vector<TensorDesc>& inputs, int precision, int batch,
                             ContractionPlan* plan, bool ws_upper_bound, int64_t min_tc_outputs) {
  if (inputs.empty()) return set_error(CUTQC_EINVAL, "no tensors");
  if (precision != CUTQC_PREC_FP32_SIMT && precision != CUTQC_PREC_FP16X3_TC && precision != CUTQC_PREC_FP16X3_TC_PRUNE)
    return set_error(CUTQC_EINVAL, "unknown precision %d", precision);
  std::map<int, int> uses;
  int n = 0;
  for (auto& t : inputs) {
    n += t.o;
    for (int e : t.edges) uses[e]++;
    if ((int)t.pos.size() != t.o) return set_error(CUTQC_EINVAL, "internal: positions");
  }
  for (auto& kv : uses)
    if (kv.second != 2) return set_error(CUTQC_EINVAL, "cut edge %d must join exactly two subcircuits", kv.first);
  plan->K = (int)uses.size();
  plan->n = n;
  plan->tensors = inputs;
  plan->stage_of.assign(inputs.size(), -1);
  plan->stages.clear();
  size_t ws = 0;
  auto take = [&](size_t bytes) {
    size_t o = ws;
    ws = align_up(ws + bytes * (size_t)batch, 256);
    return o;
  };
  std::vector<int> alive;
  for (size_t i = 0; i < inputs.size(); ++i) alive.push_back((int)i);
  while (alive.size() > 1) {
    int best_a = -1, best_b = -1;
    bool best_share = false;
    double best_cost = 0;
    for (size_t x = 0; x < alive.size(); ++x)
      for (size_t y = x + 1; y < alive.size(); ++y) {
        const TensorDesc& A = plan->tensors[alive[x]];
        const TensorDesc& B = plan->tensors[alive[y]];
        std::vector<int> uni, inter;
        std::set_union(A.edges.begin(), A.edges.end(), B.edges.begin(), B.edges.end(), std::back_inserter(uni));
        std::set_intersection(A.edges.begin(), A.edges.end(), B.edges.begin(), B.edges.end(), std::back_inserter(inter));
        bool share = !inter.empty();
        double cost = 2.0 * std::pow(4.0, (double)uni.size()) * std::pow(2.0, (double)(A.o + B.o));
        bool better = best_a < 0 || (share && !best_share) || (share == best_share && cost < best_cost);
        if (better) { best_a = alive[x]; best_b = alive[y]; best_share = share; best_cost = cost; }
      }
    const bool final_stage = alive.size() == 2;
    if (!final_stage) {
      // the operand holding the lowest open edge goes to the columns: the
      // result's lowest index bits are then its digits, and the tensor-core
      // GEMM stores runs of consecutive floats straight from registers
      const TensorDesc& A = plan->tensors[best_a];
      const TensorDesc& B = plan->tensors[best_b];
      std::vector<int> shared2, open2;
      std::set_intersection(A.edges.begin(), A.edges.end(), B.edges.begin(), B.edges.end(), std::back_inserter(shared2));
      std::set_symmetric_difference(A.edges.begin(), A.edges.end(), B.edges.begin(), B.edges.end(),
                                    std::back_inserter(open2));
      if (!open2.empty() && std::binary_search(A.edges.begin(), A.edges.end(), open2.front()))
        std::swap(best_a, best_b);
    }
    if (final_stage) {
      // the operand holding the most significant output bit goes to the rows
      const TensorDesc& A = plan->tensors[best_a];
      const TensorDesc& B = plan->tensors[best_b];
      int ma = A.o ? *std::max_element(A.pos.begin(), A.pos.end()) : -1;
      int mb = B.o ? *std::max_element(B.pos.begin(), B.pos.end()) : -1;
      if (mb > ma) std::swap(best_a, best_b);
    }
    const TensorDesc A = plan->tensors[best_a];
    const TensorDesc B = plan->tensors[best_b];
    std::vector<int> shared, open_a, open_b, uni_open;
    std::set_intersection(A.edges.begin(), A.edges.end(), B.edges.begin(), B.edges.end(), std::back_inserter(shared));
    std::set_difference(A.edges.begin(), A.edges.end(), shared.begin(), shared.end(), std::back_inserter(open_a));
    std::set_difference(B.edges.begin(), B.edges.end(), shared.begin(), shared.end(), std::back_inserter(open_b));
    std::set_union(open_a.begin(), open_a.end(), open_b.begin(), open_b.end(), std::back_inserter(uni_open));
    if (A.o + B.o + 2 * (int)uni_open.size() > 40) return set_error(CUTQC_EUNSUPPORTED, "intermediate tensor too large");
    PlanStage st;
    st.a = best_a;
    st.b = best_b;
    st.final_stage = final_stage;
    auto make_operand = [&](const TensorDesc& T, int tidx, const std::vector<int>& open, PlanOperand* op) {
      op->tensor = tidx;
      OperandView& v = op->view;
      v.src = nullptr;
      v.o = T.o;
      v.k = (int)T.edges.size();
      v.open_dmask = digit_mask(T.edges, open);
      v.shared_dmask = digit_mask(T.edges, shared);
      v.n_open = (int)open.size();
      v.n_shared = (int)shared.size();
      // last step: operand row bit j = the source bit with the j-th smallest
      // output position, so that a plain bit deposit places every bit
      op->row_bits.resize(T.o);
      for (int b = 0; b < T.o; ++b) op->row_bits[b] = b;
      if (final_stage)
        std::sort(op->row_bits.begin(), op->row_bits.end(), [&](int x, int y) { return T.pos[x] < T.pos[y]; });
      bool ident_rows = true;
      for (int b = 0; b < T.o; ++b) ident_rows &= op->row_bits[b] == b;
      op->trivial = v.n_open == 0 && v.n_shared == v.k && ident_rows;
    };
    make_operand(A, best_a, open_a, &st.opa);
    make_operand(B, best_b, open_b, &st.opb);
    st.M = st.opa.view.rows();
    st.N = st.opb.view.rows();
    st.K = st.opa.view.kdim();
    TensorDesc R;
    R.o = A.o + B.o;
    R.edges = uni_open;
    if (final_stage) {
      uint64_t mm = 0, mn = 0;
      for (int b = 0; b < A.o; ++b) mm |= (uint64_t)1 << A.pos[b];
      for (int b = 0; b < B.o; ++b) mn |= (uint64_t)1 << B.pos[b];
      st.mask_m = mm;
      st.mask_n = mn;
      plan->final_rows = st.M;
      plan->final_cols = st.N;
      R.pos = B.pos;
      R.pos.insert(R.pos.end(), A.pos.begin(), A.pos.end());
    } else {
      // result rows above the open digits: the operand whose rows hold the
      // lower output positions takes the lower row bits (whichever operand
      // is in the GEMM's rows), so that a later step gathers whole rows in
      // order
      const int E2 = 2 * (int)uni_open.size();
      const int min_a = A.o ? *std::min_element(A.pos.begin(), A.pos.end()) : 1 << 30;
      const int min_b = B.o ? *std::min_element(B.pos.begin(), B.pos.end()) : 1 << 30;
      const bool a_low = min_a < min_b;
      const int base_a = E2 + (a_low ? 0 : B.o), base_b = E2 + (a_low ? A.o : 0);
      uint64_t mm = 0, mn = 0;
      for (int b = 0; b < A.o; ++b) mm |= (uint64_t)1 << (base_a + b);
      for (int b = 0; b < B.o; ++b) mn |= (uint64_t)1 << (base_b + b);
      mm |= digit_mask(uni_open, open_a);
      mn |= digit_mask(uni_open, open_b);
      st.mask_m = mm;
      st.mask_n = mn;
      const TensorDesc& lo_t = a_low ? A : B;
      const TensorDesc& hi_t = a_low ? B : A;
      R.pos = lo_t.pos;
      R.pos.insert(R.pos.end(), hi_t.pos.begin(), hi_t.pos.end());
    }
    // the last step over a handful of cut terms is store-bound: FP32 outer
    // products at HBM speed (FMAs, no split) beat the tensor-core GEMM,
    // which pads the terms to 64 and drains every tile through its epilogue
    st.outer = final_stage && outer_small_k_supported(st.K, st.M, st.N, st.mask_m, st.mask_n);
    st.tc = !st.outer && precision != CUTQC_PREC_FP32_SIMT &&
            (double)st.M * (double)st.N * batch >= (double)min_tc_outputs;
    if (st.tc) {
      st.Kp = (int64_t)align_up((size_t)st.K, 64);
      for (PlanOperand* op : {&st.opa, &st.opb}) {
        int64_t rows = op->view.rows();
        op->off_hi = take((size_t)rows * st.Kp * sizeof(__half));
        op->off_lo = take((size_t)rows * st.Kp * sizeof(__half));
        op->off_scale = take((size_t)rows * sizeof(float) + 16);
      }
      if (precision == CUTQC_PREC_FP16X3_TC_PRUNE && final_stage && st.K <= kPruneMaxK)
        st.off_prune = take(prune_scratch_bytes(st.K));
    } else {
      st.Kp = st.K;
      for (PlanOperand* op : {&st.opa, &st.opb})
        if (!op->trivial || ws_upper_bound) op->off32 = take((size_t)op->view.rows() * st.Kp * sizeof(float));
    }
    if (!final_stage) {
      st.result_elems = ((size_t)1 << R.o) * ((size_t)1 << (2 * uni_open.size()));
      st.off_result = take(st.result_elems * sizeof(float));
    }
    st.result = (int)plan->tensors.size();
    plan->tensors.push_back(R);
    plan->stage_of.push_back((int)plan->stages.size());
    plan->stages.push_back(st);
    alive.erase(std::remove(alive.begin(), alive.end(), best_a), alive.end());
    alive.erase(std::remove(alive.begin(), alive.end(), best_b), alive.end());
    alive.push_back(st.result);
  }
  if (inputs.size() == 1) {
    plan->final_rows = (int64_t)1 << inputs[0].o;
    plan->final_cols = 1;
  }
  plan->ws_bytes = ws;
  return CUTQC_OK;
}

int plan_contraction(const std::vector<TensorDesc>& inputs, int precision, ContractionPlan* plan) {
  return plan_contraction_batched(inputs, precision, 1, plan);
}

namespace {

// Single-tensor case: out[pdep(x, mask)] = alpha * T[x][0].
__global__ void single_copy(const float* __restrict__ T, int64_t rows, uint64_t mask, float alpha,
                            float* __restrict__ out, double* __restrict__ sum, int64_t in_bstride,
                            int64_t out_bstride) {
  T += (int64_t)blockIdx.y * in_bstride;
  out += (int64_t)blockIdx.y * out_bstride;
  if (sum) sum += blockIdx.y;
  double local = 0;
  for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < rows; x += (int64_t)gridDim.x * blockDim.x) {
    float v = alpha * T[x];
    out[pdep64((uint64_t)x, mask)] = v;
    local += v;
  }
  if (sum) {
    for (int off = 16; off; off >>= 1) local += __shfl_xor_sync(0xffffffffu, local, off);
    if ((threadIdx.x & 31) == 0) atomicAdd(sum, local);
  }
}

}  // namespace

int run_plan(const ContractionPlan& plan, const float* const* inputs, const int64_t* in_bstride, int batch,
             float* out, int64_t out_bstride, double* sum, float alpha_final, int precision, int64_t row_begin,
             int64_t row_end, uint8_t* ws, cudaStream_t caller, const cudaEvent_t* in_ready) {
  const size_t n_in = plan.stage_of.size() - plan.stages.size();
  if (plan.stages.empty()) {
    if (in_ready && in_ready[0]) CUTQC_CUDA_TRY(cudaStreamWaitEvent(caller, in_ready[0], 0));
    const TensorDesc& T = plan.tensors[0];
    uint64_t mask = 0;
    for (int b = 0; b < T.o; ++b) mask |= (uint64_t)1 << T.pos[b];
    int64_t rows = (int64_t)1 << T.o;
    int blocks = (int)std::min<int64_t>((rows + 255) / 256, 8192);
    single_copy<<<dim3(blocks, batch), 256, 0, caller>>>(inputs[0], rows, mask, alpha_final, out, sum, in_bstride[0],
                                                         out_bstride);
    CUTQC_LAUNCH_CHECK("single_copy");
    return CUTQC_OK;
  }
  if (row_end < 0) row_end = plan.final_rows;
  const bool partial = row_begin != 0 || row_end != plan.final_rows;
  auto src_of = [&](int t, int64_t* bstride) -> const float* {
    if (t < (int)n_in) {
      *bstride = in_bstride[t];
      return inputs[t];
    }
    const PlanStage& s = plan.stages[plan.stage_of[t]];
    *bstride = (int64_t)s.result_elems;
    return (const float*)(ws + s.off_result);
  };
  int rc;
  const size_t ns_all = plan.stages.size();
  // Column operands with an operand-wide scale need the max |x| of their
  // source.  When that source is an earlier step's result, covered whole by
  // the operand, the paired GEMM that writes it also reduces its max into the
  // operand's max word (the consumer's scale slot 1), and the consumer's prep
  // skips its max pass.  max_into[s] = the consuming step, or -1.
  std::vector<int> max_into(ns_all, -1);
  if (precision != CUTQC_PREC_FP32_SIMT) {
    for (size_t c = 0; c < ns_all; ++c) {
      const PlanStage& cs = plan.stages[c];
      const int dep = plan.stage_of[cs.b];
      if (dep < 0 || !cs.tc || !plan.stages[dep].tc) continue;
      const bool pruned = precision == CUTQC_PREC_FP16X3_TC_PRUNE && cs.final_stage && cs.K <= kPruneMaxK;
      OperandView vb = cs.opb.view;
      vb.src = (const float*)(ws + plan.stages[dep].off_result);
      if (!pruned && tc_pair_supported(plan.stages[dep].Kp) && prep_covers_source(vb, 0, cs.N))
        max_into[dep] = (int)c;
    }
  }
  // wait_b: an event the column operand's producer records on another
  // stream; the tensor-core path waits for it after preparing the row
  // operand (which then runs beside that producer), the other paths first
  auto run_stage = [&](const PlanStage& stg0, cudaStream_t st, size_t si, cudaEvent_t wait_b) -> int {
    PlanStage stg = stg0;
    int64_t sa_b = 0, sb_b = 0;
    stg.opa.view.src = src_of(stg.a, &sa_b);
    stg.opb.view.src = src_of(stg.b, &sb_b);
    int64_t r0 = 0, M = stg.M;
    if (stg.final_stage && partial) {
      r0 = row_begin;
      M = row_end - row_begin;
    }
    float* dst = stg.final_stage ? out : (float*)(ws + stg.off_result);
    const int64_t dst_b = stg.final_stage ? out_bstride : (int64_t)stg.result_elems;
    const float alpha = stg.final_stage ? alpha_final : 1.0f;
    double* sum_ptr = stg.final_stage ? sum : nullptr;
    const int streaming = stg.final_stage ? 1 : 0;
    if (!stg.tc && wait_b) CUTQC_CUDA_TRY(cudaStreamWaitEvent(st, wait_b, 0));
    if (stg.tc) {
      const bool prune = precision == CUTQC_PREC_FP16X3_TC_PRUNE && stg.final_stage && stg.K <= kPruneMaxK;
      // the term selection reads both operands
      if (prune && wait_b) CUTQC_CUDA_TRY(cudaStreamWaitEvent(st, wait_b, 0));
      const size_t prune_bytes = prune_scratch_bytes(stg.K);
      for (int b = 0; b < batch; ++b) {
        OperandView va = stg.opa.view, vb = stg.opb.view;
        va.src += b * sa_b;
        vb.src += b * sb_b;
        __half* ah = (__half*)(ws + stg.opa.off_hi) + (size_t)b * M * stg.Kp;
        __half* al = (__half*)(ws + stg.opa.off_lo) + (size_t)b * M * stg.Kp;
        float* as = (float*)(ws + stg.opa.off_scale) + (size_t)b * M;
        __half* bh = (__half*)(ws + stg.opb.off_hi) + (size_t)b * stg.N * stg.Kp;
        __half* bl = (__half*)(ws + stg.opb.off_lo) + (size_t)b * stg.N * stg.Kp;
        float* bs = (float*)(ws + stg.opb.off_scale) + (size_t)b * stg.N;
        int* cols = nullptr;
        int* meta = nullptr;
        if (prune) {
          // the kept terms of this item, chosen on the device
          uint8_t* pb = ws + stg.off_prune + (size_t)b * prune_bytes;
          float* colw = (float*)pb;
          cols = (int*)(colw + 3 * stg.K);
          meta = cols + stg.K;
          rc = launch_prune_select(va, stg.opa.row_bits.data(), (int)stg.opa.row_bits.size(), r0, M, vb,
                                   stg.opb.row_bits.data(), (int)stg.opb.row_bits.size(), stg.N, alpha,
                                   CUTQC_PRUNE_TOL, colw, cols, meta, reinterpret_cast<unsigned int*>(bs + 1), st);
          if (rc) return rc;
        }
        rc = launch_prep_rows(va, stg.opa.row_bits.data(), (int)stg.opa.row_bits.size(), r0, M, stg.Kp, nullptr, ah,
                              al, as, st, 1, 0, nullptr, cols, meta);
        if (rc) return rc;
        if (!prune && wait_b && b == 0) CUTQC_CUDA_TRY(cudaStreamWaitEvent(st, wait_b, 0));
        const int bdep = plan.stage_of[stg.b];
        const bool max_ready = bdep >= 0 && max_into[bdep] == (int)si;
        rc = launch_prep_rows(vb, stg.opb.row_bits.data(), (int)stg.opb.row_bits.size(), 0, stg.N, stg.Kp, nullptr,
                              bh, bl, bs, st, 1, 0, reinterpret_cast<unsigned int*>(bs + 1), cols, meta, max_ready);
        if (rc) return rc;
        TcOperand ta{ah, al, as, M}, tb{bh, bl, bs, stg.N};
        const bool timed = stg.final_stage && g_gemm_start && b == 0;
        if (timed) CUTQC_CUDA_TRY(cudaEventRecord(g_gemm_start, st));
        float* cmax = nullptr;
        if (stg.final_stage && g_bmax && g_bmax->cmax && !partial && tc_pair_supported(stg.Kp) && M >= 32 &&
            stg.N >= 64 && ((M + 31) / 32) * ((stg.N + 63) / 64) == g_bmax->per_item) {
          cmax = g_bmax->cmax + (size_t)b * g_bmax->per_item;
          if (b == batch - 1) {
            g_bmax->written = true;
            g_bmax->M = M;
            g_bmax->N = stg.N;
            g_bmax->mask_m = stg.mask_m;
            g_bmax->mask_n = stg.mask_n;
          }
        }
        unsigned int* amax = nullptr;
        if (max_into[si] >= 0) {
          // the consuming step's column-operand max word for this item
          const PlanStage& cs = plan.stages[max_into[si]];
          amax = reinterpret_cast<unsigned int*>((float*)(ws + cs.opb.off_scale) + (size_t)b * cs.N + 1);
          CUTQC_CUDA_TRY(cudaMemsetAsync(amax, 0, sizeof(unsigned int), st));
        }
        rc = launch_tc_gemm(ta, tb, stg.Kp, alpha, stg.mask_m, stg.mask_n, dst + b * dst_b,
                            sum_ptr ? sum_ptr + b : nullptr, streaming, st, prune ? meta + 1 : nullptr, cmax, amax);
        if (rc) return rc;
        if (stg.final_stage && g_gemm_start && b == batch - 1) {
          CUTQC_CUDA_TRY(cudaEventRecord(g_gemm_stop, st));
          g_gemm_start = g_gemm_stop = nullptr;
        }
      }
      return CUTQC_OK;
    }
    if (stg.outer && !partial) {
      // FP32 outer products per item; operands gathered as for the FP32
      // GEMM (Kp = K)
      for (int b = 0; b < batch; ++b) {
        OperandView va = stg.opa.view, vb = stg.opb.view;
        va.src += b * sa_b;
        vb.src += b * sb_b;
        const float* A = va.src;
        const float* B = vb.src;
        int64_t lda = stg.K, ldb = stg.K;
        if (!stg.opa.trivial) {
          float* a32 = (float*)(ws + stg.opa.off32) + (size_t)b * M * stg.Kp;
          rc = launch_prep_rows(va, stg.opa.row_bits.data(), (int)stg.opa.row_bits.size(), 0, M, stg.Kp, a32, nullptr,
                                nullptr, nullptr, st);
          if (rc) return rc;
          A = a32;
          lda = stg.Kp;
        }
        if (!stg.opb.trivial) {
          float* b32 = (float*)(ws + stg.opb.off32) + (size_t)b * stg.N * stg.Kp;
          rc = launch_prep_rows(vb, stg.opb.row_bits.data(), (int)stg.opb.row_bits.size(), 0, stg.N, stg.Kp, b32,
                                nullptr, nullptr, nullptr, st);
          if (rc) return rc;
          B = b32;
          ldb = stg.Kp;
        }
        float* cmax = nullptr;
        if (g_bmax && g_bmax->cmax && ((M + 31) / 32) * ((stg.N + 63) / 64) == g_bmax->per_item) {
          cmax = g_bmax->cmax + (size_t)b * g_bmax->per_item;
          if (b == batch - 1) {
            g_bmax->written = true;
            g_bmax->M = M;
            g_bmax->N = stg.N;
            g_bmax->mask_m = stg.mask_m;
            g_bmax->mask_n = stg.mask_n;
          }
        }
        const bool timed = g_gemm_start && b == 0;
        if (timed) CUTQC_CUDA_TRY(cudaEventRecord(g_gemm_start, st));
        rc = launch_outer_small_k(A, lda, B, ldb, M, stg.N, stg.K, alpha, stg.mask_m, stg.mask_n, dst + b * dst_b,
                                  sum_ptr ? sum_ptr + b : nullptr, cmax, st);
        if (rc) return rc;
        if (g_gemm_start && b == batch - 1) {
          CUTQC_CUDA_TRY(cudaEventRecord(g_gemm_stop, st));
          g_gemm_start = g_gemm_stop = nullptr;
        }
      }
      return CUTQC_OK;
    }
    const float* A;
    const float* B;
    int64_t lda, ldb, a_b, b_b;
    if (stg.opa.trivial) {
      A = stg.opa.view.src + r0 * stg.K;
      lda = stg.K;
      a_b = sa_b;
    } else {
      float* a32 = (float*)(ws + stg.opa.off32);
      rc = launch_prep_rows(stg.opa.view, stg.opa.row_bits.data(), (int)stg.opa.row_bits.size(), r0, M, stg.Kp, a32,
                            nullptr, nullptr, nullptr, st, batch, sa_b);
      if (rc) return rc;
      A = a32;
      lda = stg.Kp;
      a_b = M * stg.Kp;
    }
    if (stg.opb.trivial) {
      B = stg.opb.view.src;
      ldb = stg.K;
      b_b = sb_b;
    } else {
      float* b32 = (float*)(ws + stg.opb.off32);
      rc = launch_prep_rows(stg.opb.view, stg.opb.row_bits.data(), (int)stg.opb.row_bits.size(), 0, stg.N, stg.Kp,
                            b32, nullptr, nullptr, nullptr, st, batch, sb_b);
      if (rc) return rc;
      B = b32;
      ldb = stg.Kp;
      b_b = stg.N * stg.Kp;
    }
    const bool timed = stg.final_stage && g_gemm_start;
    if (timed) CUTQC_CUDA_TRY(cudaEventRecord(g_gemm_start, st));
    rc = launch_sgemm(A, lda, B, ldb, M, stg.N, stg.K, alpha, stg.mask_m, stg.mask_n, dst, sum_ptr, streaming, st,
                      batch, a_b, b_b, dst_b);
    if (rc) return rc;
    if (timed) {
      CUTQC_CUDA_TRY(cudaEventRecord(g_gemm_stop, st));
      g_gemm_start = g_gemm_stop = nullptr;
    }
    return CUTQC_OK;
  };
  // A step that does not read the previous step's result can run beside it:
  // such steps (when large enough to pay for the stream hop: 2^22 outputs
  // or more; small steps, as in DD levels, gained nothing measurable and
  // lost to the extra dependencies) go to side streams, after the caller's
  // earlier work (fork)
  // and the steps they read; the others stay on the caller's stream in plan
  // order (waiting for any side step they read), and the side streams join
  // it at the end.  A plan that is one chain of dependent steps therefore
  // adds no stream hops.
  const size_t ns = plan.stages.size();
  std::vector<char> side(ns, 0);
  for (size_t si = 1; si < ns && ns <= (size_t)kSideEvents; ++si) {
    const PlanStage& x = plan.stages[si];
    const int prev_result = plan.stages[si - 1].result;
    const bool big = (double)x.M * (double)x.N * batch >= (double)(1 << 22);
    side[si] = big && !x.final_stage && x.a != prev_result && x.b != prev_result;
  }
  const bool par = std::any_of(side.begin(), side.end(), [](char c) { return c != 0; });
  SideStreams* ss = nullptr;
  std::unique_lock<std::mutex> side_lock;
  if (par) {
    if ((rc = side_streams(caller, &ss))) return rc;
    side_lock = std::unique_lock<std::mutex>(ss->mu);
    CUTQC_CUDA_TRY(cudaEventRecord(ss->fork, caller));
  }
  int nside = 0;
  std::vector<char> on_side(ns, 0);
  for (size_t si = 0; si < ns; ++si) {
    const PlanStage& stg = plan.stages[si];
    cudaStream_t st = caller;
    cudaEvent_t wait_b = nullptr;
    if (par) {
      if (side[si]) {
        st = ss->s[nside % kSideStreams];
        ++nside;
        on_side[si] = 1;
        CUTQC_CUDA_TRY(cudaStreamWaitEvent(st, ss->fork, 0));
      }
      const int da = plan.stage_of[stg.a], db = plan.stage_of[stg.b];
      if (da >= 0 && (on_side[da] || side[si])) CUTQC_CUDA_TRY(cudaStreamWaitEvent(st, ss->done[da], 0));
      if (db >= 0 && db != da && (on_side[db] || side[si])) wait_b = ss->done[db];
    }
    // inputs written by work the caller issued elsewhere
    for (int t : {stg.a, stg.b})
      if (in_ready && t < (int)n_in && in_ready[t]) CUTQC_CUDA_TRY(cudaStreamWaitEvent(st, in_ready[t], 0));
    if ((rc = run_stage(stg, st, si, wait_b))) return rc;
    if (par) CUTQC_CUDA_TRY(cudaEventRecord(ss->done[si], st));
  }
  nside = std::min(nside, kSideStreams);
  for (int j = 0; j < nside; ++j) {
    CUTQC_CUDA_TRY(cudaEventRecord(ss->join[j], ss->s[j]));
    CUTQC_CUDA_TRY(cudaStreamWaitEvent(caller, ss->join[j], 0));
  }
  return CUTQC_OK;
}

namespace {

int fd_inputs(int n_sub, const cutqc_subcircuit* s, int out_order, std::vector<TensorDesc>* out) {
  if (n_sub < 1 || !s) return set_error(CUTQC_EINVAL, "n_sub must be >= 1");
  if (out_order != CUTQC_ORDER_KRON && out_order != CUTQC_ORDER_ORIGINAL)
    return set_error(CUTQC_EINVAL, "out_order must be KRON or ORIGINAL");
  int n = 0;
  std::map<int, std::pair<int, int>> edge_use;   // edge -> (#init sides, #meas sides)
  for (int i = 0; i < n_sub; ++i) {
    int rc = validate_subcircuit(&s[i]);
    if (rc) return rc;
    const int o = s[i].w - s[i].k_out;
    if (o > 0 && !s[i].out_qubit) return set_error(CUTQC_EINVAL, "missing out_qubit");
    n += o;
    for (int j = 0; j < s[i].k_in; ++j) edge_use[s[i].in_edge[j]].first++;
    for (int j = 0; j < s[i].k_out; ++j) edge_use[s[i].out_edge[j]].second++;
  }
  if (n > CUTQC_MAX_QUBITS) return set_error(CUTQC_EUNSUPPORTED, "%d output qubits > %d", n, CUTQC_MAX_QUBITS);
  for (auto& kv : edge_use)
    if (kv.second.first != 1 || kv.second.second != 1)
      return set_error(CUTQC_EINVAL, "cut edge %d must be measured once and initialised once", kv.first);
  if ((int)edge_use.size() > CUTQC_MAX_CUTS)
    return set_error(CUTQC_EUNSUPPORTED, "%d cuts > %d", (int)edge_use.size(), CUTQC_MAX_CUTS);
  if (out_order == CUTQC_ORDER_ORIGINAL) {
    std::vector<int> seen(n, 0);
    for (int i = 0; i < n_sub; ++i)
      for (int t = 0; t < s[i].w - s[i].k_out; ++t) {
        int x = s[i].out_qubit[t];
        if (x < 0 || x >= n || seen[x]) return set_error(CUTQC_EINVAL, "out_qubit must be a permutation of 0..n-1");
        seen[x] = 1;
      }
  }
  out->clear();
  int offset = n;
  for (int i = 0; i < n_sub; ++i) {
    TensorDesc t;
    t.o = s[i].w - s[i].k_out;
    for (int j = 0; j < s[i].k_in; ++j) t.edges.push_back(s[i].in_edge[j]);
    for (int j = 0; j < s[i].k_out; ++j) t.edges.push_back(s[i].out_edge[j]);
    std::sort(t.edges.begin(), t.edges.end());
    offset -= t.o;
    for (int b = 0; b < t.o; ++b) t.pos.push_back(out_order == CUTQC_ORDER_KRON ? offset + b : s[i].out_qubit[b]);
    out->push_back(t);
  }
  return CUTQC_OK;
}

}  // namespace

}  // namespace cutqc

using namespace cutqc;

extern "C" const char* cutqc_last_error(void) { return g_last_error.c_str(); }

extern "C" const char* cutqc_version(void) { return "cutqc-gb300 0.1 (sm_103a)"; }

extern "C" int cutqc_device_status(int32_t* status_out) {
  if (!status_out) return set_error(CUTQC_EINVAL, "null status_out");
  int* p = device_status_ptr();
  if (!p) return set_error(CUTQC_ECUDA, "no device status word");
  CUTQC_CUDA_TRY(cudaDeviceSynchronize());
  int v = 0;
  CUTQC_CUDA_TRY(cudaMemcpy(&v, p, sizeof(int), cudaMemcpyDeviceToHost));
  CUTQC_CUDA_TRY(cudaMemset(p, 0, sizeof(int)));
  *status_out = v;
  return CUTQC_OK;
}

extern "C" int cutqc_kernel_launches(int64_t* count) {
  if (!count) return set_error(CUTQC_EINVAL, "null count");
  *count = (int64_t)g_launches.load(std::memory_order_relaxed);
  return CUTQC_OK;
}

extern "C" int cutqc_fd_input_events(int n, const void* const* events) {
  if (n < 0 || n > 4096) return set_error(CUTQC_EINVAL, "n = %d outside 0..4096", n);
  if (n > 0 && !events) return set_error(CUTQC_EINVAL, "null event array");
  g_input_events.assign(n, nullptr);
  for (int i = 0; i < n; ++i) g_input_events[i] = (cudaEvent_t)events[i];
  return CUTQC_OK;
}

extern "C" int cutqc_fd_timing_events(void* start_event, void* stop_event) {
  if ((start_event == nullptr) != (stop_event == nullptr))
    return set_error(CUTQC_EINVAL, "give both events or neither");
  g_gemm_start = (cudaEvent_t)start_event;
  g_gemm_stop = (cudaEvent_t)stop_event;
  return CUTQC_OK;
}

extern "C" int cutqc_fd_shape(int n_sub, const cutqc_subcircuit* s, int64_t* rows, int64_t* cols) {
  std::vector<TensorDesc> in;
  int rc = fd_inputs(n_sub, s, CUTQC_ORDER_KRON, &in);
  if (rc) return rc;
  ContractionPlan plan;
  if ((rc = plan_contraction(in, CUTQC_PREC_FP32_SIMT, &plan))) return rc;
  if (rows) *rows = plan.final_rows;
  if (cols) *cols = plan.final_cols;
  return CUTQC_OK;
}

extern "C" int cutqc_reconstruct_fd_workspace_size(int n_sub, const cutqc_subcircuit* s, int precision,
                                                   size_t* bytes) {
  if (!bytes) return set_error(CUTQC_EINVAL, "null bytes");
  size_t best = 0;
  bool any = false;
  for (int order : {CUTQC_ORDER_KRON, CUTQC_ORDER_ORIGINAL}) {
    std::vector<TensorDesc> in;
    ContractionPlan plan;
    int rc = fd_inputs(n_sub, s, order, &in);
    if (!rc) rc = plan_contraction(in, precision, &plan);
    if (rc) {
      if (order == CUTQC_ORDER_KRON) return rc;
      continue;
    }
    best = std::max(best, plan.ws_bytes);
    any = true;
  }
  if (!any) return set_error(CUTQC_EINVAL, "no valid plan");
  *bytes = best;
  return CUTQC_OK;
}

extern "C" int cutqc_reconstruct_fd(int n_sub, const cutqc_subcircuit* s, const float* const* attributed,
                                    int out_order, int precision, int64_t row_begin, int64_t row_end,
                                    float* out, double* sum, void* ws_dev, size_t ws_bytes, void* stream) {
  // this call's input events (if any were set), cleared whatever happens
  std::vector<cudaEvent_t> ready;
  ready.swap(g_input_events);
  if (!ready.empty() && (int)ready.size() != n_sub)
    return set_error(CUTQC_EINVAL, "%d input events set for %d subcircuits", (int)ready.size(), n_sub);
  std::vector<TensorDesc> in;
  int rc = fd_inputs(n_sub, s, out_order, &in);
  if (rc) return rc;
  ContractionPlan plan;
  if ((rc = plan_contraction(in, precision, &plan))) return rc;
  if (!attributed || !out) return set_error(CUTQC_EINVAL, "null pointer");
  for (int i = 0; i < n_sub; ++i)
    if (!attributed[i]) return set_error(CUTQC_EINVAL, "null attributed tensor %d", i);
  if (ws_bytes < plan.ws_bytes || (plan.ws_bytes && !ws_dev))
    return set_error(CUTQC_ENOMEM, "FD workspace needs %zu bytes", plan.ws_bytes);
  if (row_end < 0) row_end = plan.final_rows;
  if (row_begin < 0 || row_begin > row_end || row_end > plan.final_rows)
    return set_error(CUTQC_EINVAL, "row range [%lld, %lld) outside [0, %lld)", (long long)row_begin,
                     (long long)row_end, (long long)plan.final_rows);
  const bool partial = row_begin != 0 || row_end != plan.final_rows;
  if (partial) {
    if (out_order != CUTQC_ORDER_KRON) return set_error(CUTQC_EINVAL, "a partial row range needs CUTQC_ORDER_KRON");
    if (plan.stages.empty()) return set_error(CUTQC_EINVAL, "no row split for a single subcircuit");
    const PlanStage& f = plan.stages.back();
    const int shift = mask_contig_shift(f.mask_m);
    if (shift < 0 || shift + __builtin_popcountll(f.mask_m) != plan.n)
      return set_error(CUTQC_EUNSUPPORTED, "row split needs the row operand to hold the top output bits");
  }
  std::vector<int64_t> bstride(n_sub, 0);
  return run_plan(plan, attributed, bstride.data(), 1, out, 0, sum, std::ldexp(1.0f, -plan.K), precision, row_begin,
                  row_end, (uint8_t*)ws_dev, (cudaStream_t)stream, ready.empty() ? nullptr : ready.data());
}
