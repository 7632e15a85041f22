// Host-side shapes of one recursion level of Algorithm 1, shared by the
// level-by-level launches (dd.cu) and the persistent kernel's builder
// (dd_persist.cu).  Definitions in dd.cu.
#pragma once

#include "contract.cuh"

#include <algorithm>
#include <vector>

namespace cutqc {

struct LevelShape {
  int depth = 0;
  std::vector<int> active;                 // qubits, ascending
  std::vector<int32_t> active_bits;        // per subcircuit
  std::vector<int32_t> bin_bit;            // subcircuit-major
  std::vector<uint64_t> act_mask, zoom_mask;   // per subcircuit, over output bits
};

struct RunLayout {
  size_t merged_off[64];
  size_t zoom_off[64];
  size_t part_off[64];      // partial sums of the slices (when log_slices > 0)
  int log_slices[64];
  size_t step_off = 0, top_idx_off = 0, top_val_off = 0, sum_off = 0;
  size_t total = 0;
};

constexpr int kMergeCtasDefault = 1024, kMergeCtasMax = 4096;

// CTAs of a merge launch: enough to fill the GPU once (`ctas` of them, by
// default 8 per SM), each walking rows (`groups` rows at a time:
// merge_groups in dd_kernels.cuh)
inline unsigned merge_grid(int64_t rows, int slices, int groups = 1, int64_t ctas = 0) {
  if (ctas <= 0) ctas = (int64_t)sm_count() * 8;
  const int64_t cap = std::max<int64_t>(1, ctas / std::max(1, slices));
  const int64_t walk = (rows + groups - 1) / std::max(1, groups);
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>(walk, cap));
}

// The contraction inputs of one bin job: one tensor per subcircuit with its
// active rows (active_bits[i]) and cut edges; bin_bit places the rows.
int dd_inputs(int n_sub, const cutqc_subcircuit* s, const int32_t* active_bits, const int32_t* bin_bit,
              std::vector<TensorDesc>* in, int* total_bits);
// Workspace of one step of n_jobs jobs (contraction plan and top-T scratch).
// min_tc_outputs: as plan_contraction_batched (-1: the library's default).
int dd_step_ws(int n_sub, const cutqc_subcircuit* s, const int32_t* active_bits, int n_jobs, int precision,
               size_t* bytes, int64_t min_tc_outputs = -1);
// Active qubits, per-subcircuit active/zoom masks and bin bits at a depth.
int level_shape(int n_sub, const cutqc_subcircuit* s, int n, int M, int depth, LevelShape* L);
// Workspace layout of one level of n_jobs jobs (merge_ctas: about how many
// CTAs share one subcircuit's merge).
int level_layout(int n_sub, const cutqc_subcircuit* s, const LevelShape& L, int n_jobs, RunLayout* R,
                 int merge_ctas = kMergeCtasDefault);
int validate_run(int n_sub, const cutqc_subcircuit* s, int n, int M, int T);
// Level workspace (reused by every level) and the total with the job records
// of a level-synchronous run.
int run_ws(int n_sub, const cutqc_subcircuit* s, int n, int M, int T, size_t* level_bytes, size_t* total);

}  // namespace cutqc
