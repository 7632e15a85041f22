// Algorithm 1 (breadth first) for several circuits in one persistent launch.
//
// The level-by-level path (dd.cu) enqueues a chain of small launches per
// level: merges, slice reductions, one GEMM per contraction step, top-T, the
// level selection.  Those jobs are small (2^16 bins at M = 16), so the chain
// is bound by launch latency and by each launch's ramp and tail, not by the
// GPU.  Here the whole run of every circuit is one program of phases; one
// cooperative launch of a grid that fits on the GPU at once walks it, with a
// grid-wide barrier between phases.  Phase p holds the p-th step of every
// circuit, so the circuits fill the GPU together:
//   merge (+ zero the bin totals)  ->  slice reduction (when sliced)  ->
//   one phase per depth of the contraction plan (independent steps share a
//   phase; 64 x 64 GEMM tiles, 256 x 16 for steps of at most 16 columns,
//   whose operands are gathered on the fly, no staging copy)  ->  chunked
//   top-T of each job's bins  ->  the level selection
//   (each job's top T from its chunks' candidates, then Algorithm 1's list L
//   truncated to T, written as the next level's job records).
// Within a phase a CTA takes tasks (merge walkers, GEMM tiles, top-T chunks)
// in a fixed stride; the results are those of the level-by-level path: the
// same merge slicing and partial-sum order, the same fmaf chain over k per
// bin, the same selection order (bin totals are float64 atomics in both).
//
// Memory ordering: data written in one phase is read in a later one by other
// CTAs, after a barrier that each CTA enters with a device-scope release (its
// arrival, after a block barrier) and leaves with a device-scope acquire;
// those reads use ld.global.cg (through L2), never the non-coherent
// read-only path.  Every barrier wait is bounded: a CTA that
// waits too long records CUTQC_ETIMEOUT in the device status word and raises
// an abort flag, and every CTA then returns.
#include "internal.cuh"
#include "contract.cuh"
#include "dd_kernels.cuh"
#include "dd_host.cuh"
#include "sgemm_tile.cuh"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

namespace cutqc {
namespace {

constexpr long long kBarrierTimeoutCycles = 4000000000LL;   // ~2 s at 2 GHz
constexpr int kThreads = 256;
constexpr int kTopkChunkDefault = 2048;

// A contraction operand read in place: operand row m = (xp, open) with xp
// the high bits (moved to source row bits bit[j] when permute) and open the
// low 2 * n_open bits; element s = source column pdep(open, open_dmask) |
// pdep(s, shared_dmask) (s itself when contig).  The same map as the staged
// gather of the level-by-level path.
struct GView {
  const float* src;
  int64_t bstride;       // floats between batch items (jobs)
  int64_t C;             // source columns, 4^k
  uint64_t open_dmask, shared_dmask;
  int n_open, contig, permute, nbits;
  int8_t bit[40];
};

template <bool kCoherent>
struct GatherRows {
  const float* src;      // this batch item's source
  int64_t C;
  uint64_t open_dmask, shared_dmask;
  int n_open, contig;
  const GView* v;        // row bit map (read twice per tile)
  __device__ __forceinline__ GatherRows(const GView& g, int64_t b)
      : src(g.src + b * g.bstride), C(g.C), open_dmask(g.open_dmask), shared_dmask(g.shared_dmask),
        n_open(g.n_open), contig(g.contig), v(&g) {}
  struct Row {
    const float* p;
    uint64_t obase;
  };
  __device__ __forceinline__ Row row(int64_t m) const {
    const uint64_t xp = (uint64_t)m >> (2 * n_open);
    uint64_t x = xp;
    if (v->permute) {
      x = 0;
      const int nb = v->nbits;
      for (int j = 0; j < nb; ++j) x |= ((xp >> j) & 1) << v->bit[j];
    }
    const uint64_t open = (uint64_t)m & (((uint64_t)1 << (2 * n_open)) - 1);
    return Row{src + (int64_t)x * C, pdep64(open, open_dmask)};
  }
  __device__ __forceinline__ float at(const Row& r, int64_t s) const {
    const int64_t c = contig ? s : (int64_t)(r.obase | pdep64((uint64_t)s, shared_dmask));
    return ldx<kCoherent>(r.p + c);
  }
};

enum OpType : int { OP_ZERO = 0, OP_MERGE, OP_REDUCE, OP_GEMM, OP_TOPK, OP_SELECT };

struct ZeroOp {          // bin totals of a level (and the first job record)
  double* p;
  int n;
  cutqc_dd_job_result* first_job;
};
struct MergeOp {
  const float* att;
  float* out;
  ZoomFromJobs zj;
  uint64_t act, mrg, zm;
  int64_t rows_a;
  int k, n_jobs, n_merged, log_slices, nx;
};
struct ReduceOp {
  const float* part;
  float* out;
  int64_t E;
  int S, nblocks;
};
struct GemmOp {
  GView a, b;
  int64_t M, N, K;
  float alpha;
  uint64_t mask_m, mask_n;
  int m_shift, n_contig, streaming, gm, gn;
  int narrow;            // 256 x 16 tiles (N <= 16), else 64 x 64
  float* out;
  int64_t out_bstride;
  double* sum;
};
struct TopkOp {
  const float* vals;
  int32_t* cidx;
  float* cval;
  int64_t n, clen;
  int T, chunks;
};
struct SelectOp {
  cutqc_dd_job_result* jobs;
  LevelInfo L;
  int64_t bins_off0, nb;
  const double* bsum;
  const int32_t* cidx;
  const float* cval;
  int32_t* tidx;
  float* tval;
  int32_t* n_jobs_dev;
  int job0, nj, ncand, T, has_children, n_next;
};
struct alignas(16) Op {
  int type, task0, ntasks;
  union {
    ZeroOp zero;
    MergeOp merge;
    ReduceOp reduce;
    GemmOp gemm;
    TopkOp topk;
    SelectOp select;
  } u;
};

// The arrival counter and the release word on separate 128-byte lines: the
// waiters' polls do not contend with the arrivals.
struct alignas(128) GridBar {
  unsigned int arrived;
  unsigned int pad0[31];
  unsigned int gen;
  int abort;
  unsigned int pad1[30];
};

struct Program {
  const Op* ops;
  const int* phase_op;       // [n_phases + 1]: ops of phase p
  const int* phase_tasks;    // [n_phases]
  int n_phases;
  GridBar* bar;
  int* status;
  long long* trace;          // [n_phases + 1]: CTA 0's clock at the start and after each phase
};

__device__ __forceinline__ unsigned int ld_acquire(const unsigned int* p) {
  unsigned int v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ unsigned int atom_add_acq_rel(unsigned int* p, unsigned int v) {
  unsigned int old;
  asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
  return old;
}
__device__ __forceinline__ void red_add_release(unsigned int* p, unsigned int v) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Grid-wide barrier of a cooperative launch (every CTA resident).  Thread 0
// of each CTA arrives with an acquire-release add (after the block barrier,
// so the CTA's writes are ordered before it); the last arriver resets the
// count and releases the generation word, which the others poll with acquire
// loads.  Returns false when the run is aborted (a wait ran out, here or in
// another CTA).
__device__ bool grid_barrier(GridBar* g, int* status) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int res = 1;
    volatile int* vabort = &g->abort;
    const unsigned int my_gen = ld_acquire(&g->gen);
    if (atom_add_acq_rel(&g->arrived, 1u) == gridDim.x - 1) {
      atomicExch(&g->arrived, 0u);
      red_add_release(&g->gen, 1u);
    } else {
      const long long t0 = clock64();
      while (ld_acquire(&g->gen) == my_gen) {
        if (*vabort) { res = 0; break; }
        if (clock64() - t0 > kBarrierTimeoutCycles) {
          atomicExch(&g->abort, 1);
          record_status(status, CUTQC_ETIMEOUT);
          res = 0;
          break;
        }
        __nanosleep(8);
      }
    }
    ok = res && !*vabort;
  }
  __syncthreads();
  return ok != 0;
}

// The T best of n (value, index) candidates by (value desc, index asc), one
// warp: each lane keeps its best TCAP, then T rounds of a warp arg-max.
template <int TCAP>
__device__ __forceinline__ void warp_topk_candidates(const float* __restrict__ cval, const int32_t* __restrict__ cidx,
                                                     int n, int T, int32_t* __restrict__ out_idx,
                                                     float* __restrict__ out_val) {
  const int lane = threadIdx.x & 31;
  float lv[TCAP];
  int li[TCAP];
#pragma unroll
  for (int u = 0; u < TCAP; ++u) { lv[u] = -INFINITY; li[u] = -1; }
  int cnt = 0;
  for (int q = lane; q < n; q += 32) {
    const int idx = ldx<true>(cidx + q);
    if (idx < 0) continue;
    const float v = ldx<true>(cval + q);
    if (cnt == T && !dd_better(v, idx, lv[T - 1], li[T - 1])) continue;
    int pos = cnt < T ? cnt : T - 1;
#pragma unroll
    for (int u = TCAP - 1; u > 0; --u)
      if (u <= pos && dd_better(v, idx, lv[u - 1], li[u - 1])) { lv[u] = lv[u - 1]; li[u] = li[u - 1]; pos = u - 1; }
    lv[pos] = v;
    li[pos] = idx;
    if (cnt < T) ++cnt;
  }
  int head = 0;
  for (int t = 0; t < T; ++t) {
    float bv = -INFINITY;
    int bi = -1;
#pragma unroll
    for (int u = 0; u < TCAP; ++u)
      if (u == head && head < cnt) { bv = lv[u]; bi = li[u]; }
    const int mine = bi;
    for (int off = 16; off; off >>= 1) {
      const float ov = __shfl_xor_sync(0xffffffffu, bv, off);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, off);
      if (oi >= 0 && (bi < 0 || ov > bv || (ov == bv && oi < bi))) { bv = ov; bi = oi; }
    }
    if (lane == 0) {
      out_idx[t] = bi;
      out_val[t] = bi >= 0 ? bv : 0.f;
    }
    if (bi >= 0 && mine == bi) ++head;   // the owner of the winner advances (indices are distinct)
  }
}

template <int TCAP>
__device__ __forceinline__ void select_task(const SelectOp& s) {
  // each job's T best from its chunks' candidates (one warp per job), then
  // the level selection
  if (s.T > 0) {
    const int warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int j = warp; j < s.nj; j += nw)
      warp_topk_candidates<TCAP>(s.cval + (int64_t)j * s.ncand, s.cidx + (int64_t)j * s.ncand, s.ncand, s.T,
                                 s.tidx + (int64_t)j * s.T, s.tval + (int64_t)j * s.T);
    __syncthreads();
  }
  dd_select_body<true>(s.jobs, s.job0, s.nj, s.L, s.bins_off0, s.nb, s.bsum, s.tidx, s.tval, s.T, s.has_children,
                       s.n_next, s.n_jobs_dev);
}

__device__ __forceinline__ void run_task(const Op& op, int t, TileSmem& tsm) {
  switch (op.type) {
    case OP_ZERO: {
      const ZeroOp& z = op.u.zero;
      for (int i = threadIdx.x; i < z.n; i += blockDim.x) z.p[i] = 0.0;
      if (z.first_job && threadIdx.x == 0) dd_first_job_body(z.first_job);
      break;
    }
    case OP_MERGE: {
      const MergeOp& m = op.u.merge;
      dd_merge_body<true>(m.att, m.k, m.act, m.mrg, m.zm, 0, nullptr, m.zj, m.n_jobs, m.rows_a, m.n_merged,
                          m.log_slices, m.out, t % m.nx, m.nx, t / m.nx);
      break;
    }
    case OP_REDUCE: {
      const ReduceOp& r = op.u.reduce;
      dd_merge_reduce_body<true>(r.part, r.S, r.E, r.out, t, r.nblocks);
      break;
    }
    case OP_GEMM: {
      const GemmOp& g = op.u.gemm;
      const int per = g.gm * g.gn;
      const int b = t / per, rem = t - b * per;
      const GatherRows<true> la(g.a, b), lb(g.b, b);
      float* out = g.out + (int64_t)b * g.out_bstride;
      double* sum = g.sum ? g.sum + b : nullptr;
      if (g.narrow)
        sgemm_tile_narrow(la, lb, g.M, g.N, g.K, g.alpha, g.mask_m, g.mask_n, g.m_shift, g.n_contig, out, sum,
                          g.streaming, rem / g.gn, rem % g.gn, tsm);
      else
        sgemm_tile64(la, lb, g.M, g.N, g.K, g.alpha, g.mask_m, g.mask_n, g.m_shift, g.n_contig, out, sum,
                     g.streaming, rem / g.gn, rem % g.gn, tsm);
      break;
    }
    case OP_TOPK: {
      const TopkOp& k = op.u.topk;
      if (k.T <= 4)
        dd_topk_body<4, false, true>(k.vals, nullptr, k.n, k.clen, k.T, k.cidx, k.cval, t / k.chunks, t % k.chunks,
                                     k.chunks);
      else
        dd_topk_body<32, false, true>(k.vals, nullptr, k.n, k.clen, k.T, k.cidx, k.cval, t / k.chunks,
                                      t % k.chunks, k.chunks);
      break;
    }
    case OP_SELECT: {
      const SelectOp& s = op.u.select;
      if (s.T <= 4) select_task<4>(s);
      else select_task<32>(s);
      break;
    }
    default:
      break;
  }
}

constexpr int kPhaseOpsCached = 256;
// kMinBlocks: CTAs per SM the registers are budgeted for (2, 3 or 4; the
// grid is that many per SM when they fit).
template <int kMinBlocks>
__global__ void __launch_bounds__(kThreads, kMinBlocks) dd_persistent_kernel(const Program pg) {
  // the current op's parameters and the phase's op boundaries, in shared
  // memory (the program is read-only for the launch)
  __shared__ Op sop;
  __shared__ int s_task0[kPhaseOpsCached];
  __shared__ TileSmem tsm;
  const bool tracer = blockIdx.x == 0 && threadIdx.x == 0;
  if (tracer) pg.trace[0] = clock64();
  for (int p = 0; p < pg.n_phases; ++p) {
    const int o0 = __ldg(pg.phase_op + p), o1 = __ldg(pg.phase_op + p + 1);
    const int nt = __ldg(pg.phase_tasks + p);
    for (int i = threadIdx.x; i < o1 - o0 && i < kPhaseOpsCached; i += blockDim.x)
      s_task0[i] = __ldg(&pg.ops[o0 + i].task0);
    __syncthreads();
    auto task0 = [&](int i) { return i - o0 < kPhaseOpsCached ? s_task0[i - o0] : __ldg(&pg.ops[i].task0); };
    int oi = o0, cur = -1;
    for (int t = blockIdx.x; t < nt; t += gridDim.x) {
      while (oi + 1 < o1 && t >= task0(oi + 1)) ++oi;   // tasks ascend with the op index
      if (oi != cur) {
        const int4* src = reinterpret_cast<const int4*>(pg.ops + oi);
        int4* dst = reinterpret_cast<int4*>(&sop);
        for (int i = threadIdx.x; i < (int)(sizeof(Op) / sizeof(int4)); i += blockDim.x) dst[i] = __ldg(src + i);
        __syncthreads();
        cur = oi;
      }
      run_task(sop, t - sop.task0, tsm);
      __syncthreads();
    }
    if (p + 1 < pg.n_phases && !grid_barrier(pg.bar, pg.status)) return;
    if (tracer) pg.trace[p + 1] = clock64();
  }
}

// ------------------------------------------------------------------ host

constexpr int kCtasPerSmDefault = 3;

struct BatchOpts {
  int merge_ctas = kMergeCtasDefault;
  int topk_chunk = kTopkChunkDefault;
  int ctas = 0;   // 0: every CTA that fits at once
  int ctas_per_sm = kCtasPerSmDefault;
  int narrow_max_n = SGN_BN;   // contraction steps of at most this many columns take 256 x 16 tiles
};

int read_opts(const cutqc_dd_batch_options* o, BatchOpts* b) {
  *b = BatchOpts{};
  if (!o) return CUTQC_OK;
  if (o->merge_ctas < 0 || o->merge_ctas > kMergeCtasMax)
    return set_error(CUTQC_EINVAL, "merge_ctas must be in 0..%d", kMergeCtasMax);
  if (o->topk_chunk < 0 || (o->topk_chunk && (o->topk_chunk < 256 || (o->topk_chunk & (o->topk_chunk - 1)))))
    return set_error(CUTQC_EINVAL, "topk_chunk must be 0 or a power of two >= 256");
  if (o->ctas < 0) return set_error(CUTQC_EINVAL, "ctas must be >= 0");
  if (o->ctas_per_sm != 0 && (o->ctas_per_sm < 2 || o->ctas_per_sm > 4))
    return set_error(CUTQC_EINVAL, "ctas_per_sm must be 0 or 2..4");
  if (o->narrow_max_n != 0 && o->narrow_max_n != -1 && o->narrow_max_n != 16 && o->narrow_max_n != 32 &&
      o->narrow_max_n != 64)
    return set_error(CUTQC_EINVAL, "narrow_max_n must be 0 (default), -1 (never), 16, 32 or 64");
  if (o->narrow_max_n) b->narrow_max_n = o->narrow_max_n < 0 ? 0 : o->narrow_max_n;
  if (o->ctas_per_sm) b->ctas_per_sm = o->ctas_per_sm;
  if (o->merge_ctas) b->merge_ctas = o->merge_ctas;
  if (o->topk_chunk) b->topk_chunk = o->topk_chunk;
  b->ctas = o->ctas;
  return CUTQC_OK;
}

struct Built {
  std::vector<Op> ops;
  std::vector<int> phase_op, phase_tasks;
  std::vector<int> phase_kinds;   // per phase: bit t set if an op of type t runs in it
  std::vector<int64_t> phase_fma; // per phase: multiply-adds of its contraction steps (M N K per job)
  size_t ops_off = 0, phase_off = 0, tasks_off = 0, trace_off = 0, total = 0;
};

// Builds the program of all runs for a workspace at `base` (nullptr: sizes
// only; the layout does not depend on the address).
int build_program(int n_runs, const cutqc_dd_run_desc* runs, const BatchOpts& opt, uint8_t* base, Built* out) {
  if (n_runs < 1 || !runs) return set_error(CUTQC_EINVAL, "no runs");
  std::vector<std::vector<std::vector<Op>>> phases(n_runs);   // [run][phase] ops
  std::vector<size_t> run_bytes(n_runs), run_topk_off(n_runs);
  // pass 1: per-run workspace sizes (level workspace + top-T candidates)
  for (int r = 0; r < n_runs; ++r) {
    const cutqc_dd_run_desc& R = runs[r];
    int rc = validate_run(R.n_sub, R.subcircuits, R.n_qubits, R.M, R.T);
    if (rc) return rc;
    if (R.n_sub < 2) return set_error(CUTQC_EUNSUPPORTED, "run %d: one subcircuit (no contraction)", r);
    if (!R.attributed_dev || !R.jobs_dev || !R.n_jobs_dev || !R.bins_dev || R.max_jobs < 1 || R.R < 1)
      return set_error(CUTQC_EINVAL, "run %d: bad arguments", r);
    for (int i = 0; i < R.n_sub; ++i) {
      if (!R.attributed_dev[i]) return set_error(CUTQC_EINVAL, "run %d: null attributed tensor", r);
      if (R.subcircuits[i].w - R.subcircuits[i].k_out > 32)
        return set_error(CUTQC_EUNSUPPORTED, "run %d: more than 32 outputs in a subcircuit", r);
    }
    const int depths = (R.n_qubits + R.M - 1) / R.M;
    const int levels = R.T > 0 ? std::min(R.R, depths) : 1;   // T = 0 expands nothing
    const int Tn = std::max(1, R.T);
    size_t lvl = 0, topk = 0;
    int64_t jobs_total = 0, bins_total = 0;
    for (int level = 0; level < levels; ++level) {
      const int nj = level == 0 ? 1 : Tn;
      LevelShape L;
      if ((rc = level_shape(R.n_sub, R.subcircuits, R.n_qubits, R.M, level, &L))) return rc;
      RunLayout lay;
      if ((rc = level_layout(R.n_sub, R.subcircuits, L, nj, &lay, opt.merge_ctas))) return rc;
      lvl = std::max(lvl, lay.total);
      const int64_t nb = (int64_t)1 << L.active.size();
      const int64_t chunks = (nb + opt.topk_chunk - 1) / opt.topk_chunk;
      topk = std::max(topk, (size_t)nj * chunks * Tn * (sizeof(int32_t) + sizeof(float)));
      jobs_total += nj;
      bins_total += (int64_t)nj * nb;
    }
    if (jobs_total > R.max_jobs)
      return set_error(CUTQC_ENOMEM, "run %d: %d levels need %lld job records", r, levels, (long long)jobs_total);
    if (bins_total > R.bins_capacity)
      return set_error(CUTQC_ENOMEM, "run %d: bins_capacity too small (%lld needed)", r, (long long)bins_total);
    run_topk_off[r] = align_up(lvl, 256);
    run_bytes[r] = run_topk_off[r] + align_up(topk, 256);
  }
  size_t off = align_up(sizeof(GridBar), 256);
  std::vector<size_t> run_off(n_runs);
  for (int r = 0; r < n_runs; ++r) {
    run_off[r] = off;
    off += run_bytes[r];
  }
  const size_t data_end = off;
  // pass 2: the phases of each run
  for (int r = 0; r < n_runs; ++r) {
    const cutqc_dd_run_desc& R = runs[r];
    const cutqc_subcircuit* s = R.subcircuits;
    uint8_t* ws = base ? base + run_off[r] : nullptr;
    int32_t* cidx = ws ? (int32_t*)(ws + run_topk_off[r]) : nullptr;
    const int depths = (R.n_qubits + R.M - 1) / R.M;
    const int levels = R.T > 0 ? std::min(R.R, depths) : 1;
    const int Tn = std::max(1, R.T);
    auto& ph = phases[r];
    auto phase = [&](size_t p) -> std::vector<Op>& {
      if (ph.size() <= p) ph.resize(p + 1);
      return ph[p];
    };
    int job0 = 0;
    int64_t bins_off = 0;
    for (int level = 0; level < levels; ++level) {
      const int nj = level == 0 ? 1 : Tn;
      LevelShape L;
      int rc = level_shape(R.n_sub, s, R.n_qubits, R.M, level, &L);
      if (rc) return rc;
      RunLayout lay;
      if ((rc = level_layout(R.n_sub, s, L, nj, &lay, opt.merge_ctas))) return rc;
      const int64_t nb = (int64_t)1 << L.active.size();
      double* bsum = ws ? (double*)(ws + lay.sum_off) : nullptr;
      // phase: zero the bin totals (and write the first record), merges
      const size_t p_merge = ph.size();
      {
        Op z{};
        z.type = OP_ZERO;
        z.ntasks = 1;
        z.u.zero.p = bsum;
        z.u.zero.n = nj;
        z.u.zero.first_job = level == 0 ? R.jobs_dev : nullptr;
        phase(p_merge).push_back(z);
      }
      std::vector<const float*> merged(R.n_sub);
      bool any_slices = false;
      for (int i = 0; i < R.n_sub; ++i) {
        const int o = s[i].w - s[i].k_out;
        const uint64_t all = o >= 64 ? ~0ull : (((uint64_t)1 << o) - 1);
        const uint64_t mrg = all & ~L.act_mask[i] & ~L.zoom_mask[i];
        const int k = s[i].k_in + s[i].k_out;
        const int a = __builtin_popcountll(L.act_mask[i]);
        const int ls = lay.log_slices[i];
        float* mdev = ws ? (float*)(ws + lay.merged_off[i]) : nullptr;
        float* part = ls ? (ws ? (float*)(ws + lay.part_off[i]) : nullptr) : mdev;
        const int64_t rows_a = (int64_t)1 << a;
        Op m{};
        m.type = OP_MERGE;
        MergeOp& mo = m.u.merge;
        mo.att = R.attributed_dev[i];
        mo.out = part;
        // level 0 zooms nothing: its merges read no job record (the record
        // they would read is written by this phase's zero op), zoom value 0
        mo.zj.jobs = level == 0 ? nullptr : R.jobs_dev + job0;
        mo.zj.o = o;
        mo.zj.lo = level * R.M;
        for (int t = 0; t < o; ++t) mo.zj.outq[t] = (int8_t)s[i].out_qubit[t];
        mo.act = L.act_mask[i];
        mo.mrg = mrg;
        mo.zm = L.zoom_mask[i];
        mo.rows_a = rows_a;
        mo.k = k;
        mo.n_jobs = nj;
        mo.n_merged = __builtin_popcountll(mrg);
        mo.log_slices = ls;
        // walkers: at most one per CTA of the grid (fewer, longer tasks)
        mo.nx = (int)merge_grid(rows_a * nj, 1 << ls, merge_groups(k, mo.n_merged, ls),
                                (int64_t)sm_count() * opt.ctas_per_sm);
        m.ntasks = mo.nx << ls;
        phase(p_merge).push_back(m);
        if (ls) {
          any_slices = true;
          const int64_t E = ((int64_t)nj << a) << (2 * k);
          Op q{};
          q.type = OP_REDUCE;
          q.u.reduce.part = part;
          q.u.reduce.out = mdev;
          q.u.reduce.E = E;
          q.u.reduce.S = 1 << ls;
          q.u.reduce.nblocks = (int)std::min<int64_t>((E + kThreads - 1) / kThreads, (int64_t)sm_count() * 8);
          q.ntasks = q.u.reduce.nblocks;
          phase(p_merge + 1).push_back(q);
        }
        merged[i] = mdev;
      }
      const size_t p_contract = p_merge + (any_slices ? 2 : 1);
      // the bin reconstruction: the planner's steps, one phase per depth
      std::vector<TensorDesc> in;
      int tot = 0;
      if ((rc = dd_inputs(R.n_sub, s, L.active_bits.data(), L.bin_bit.data(), &in, &tot))) return rc;
      ContractionPlan plan;
      if ((rc = plan_contraction_batched(in, CUTQC_PREC_FP32_SIMT, nj, &plan))) return rc;
      if (plan.stages.empty()) return set_error(CUTQC_EUNSUPPORTED, "run %d: nothing to contract", r);
      uint8_t* step = ws ? ws + lay.step_off : nullptr;
      const size_t n_in = in.size();
      std::vector<int> depth(plan.tensors.size(), 0);
      int max_depth = 0;
      // the level selection (its candidates are filled in below)
      Op q{};
      q.type = OP_SELECT;
      q.ntasks = 1;
      {
        SelectOp& so = q.u.select;
        so.jobs = R.jobs_dev;
        so.L.level = level;
        so.L.depth = level;
        so.L.n_active = (int)L.active.size();
        for (int a = 0; a < so.L.n_active; ++a) so.L.active[a] = (int8_t)L.active[a];
        so.bins_off0 = bins_off;
        so.nb = nb;
        so.bsum = bsum;
        so.tidx = ws ? (int32_t*)(ws + lay.top_idx_off) : nullptr;
        so.tval = ws ? (float*)(ws + lay.top_val_off) : nullptr;
        so.n_jobs_dev = R.n_jobs_dev;
        so.job0 = job0;
        so.nj = nj;
        so.T = R.T;
        so.has_children = level + 1 < levels && R.T > 0;
        so.n_next = so.has_children ? Tn : 0;
      }
      for (const PlanStage& stg : plan.stages) {
        const int d = 1 + std::max(depth[stg.a], depth[stg.b]);
        depth[stg.result] = d;
        max_depth = std::max(max_depth, d);
        auto view_of = [&](const PlanOperand& op, int t, GView* g) -> int {
          const OperandView& v = op.view;
          if (t < (int)n_in) {
            g->src = merged[t];
            g->bstride = ((int64_t)1 << in[t].o) << (2 * in[t].edges.size());
          } else {
            const PlanStage& prod = plan.stages[plan.stage_of[t]];
            g->src = step ? (const float*)(step + prod.off_result) : nullptr;
            g->bstride = (int64_t)prod.result_elems;
          }
          g->C = (int64_t)1 << (2 * v.k);
          g->open_dmask = v.open_dmask;
          g->shared_dmask = v.shared_dmask;
          g->n_open = v.n_open;
          g->contig = v.n_open == 0 && v.shared_dmask == (uint64_t)(g->C - 1);
          g->nbits = (int)op.row_bits.size();
          if (g->nbits > (int)sizeof(g->bit)) return set_error(CUTQC_EUNSUPPORTED, "too many row bits");
          g->permute = 0;
          for (int j = 0; j < g->nbits; ++j) {
            g->bit[j] = (int8_t)op.row_bits[j];
            if (op.row_bits[j] != j) g->permute = 1;
          }
          return CUTQC_OK;
        };
        Op g{};
        g.type = OP_GEMM;
        GemmOp& go = g.u.gemm;
        if ((rc = view_of(stg.opa, stg.a, &go.a)) || (rc = view_of(stg.opb, stg.b, &go.b))) return rc;
        go.M = stg.M;
        go.N = stg.N;
        go.K = stg.K;
        go.mask_m = stg.mask_m;
        go.mask_n = stg.mask_n;
        go.m_shift = mask_contig_shift(stg.mask_m);
        go.n_contig = mask_is_low(stg.mask_n);
        go.narrow = stg.N <= opt.narrow_max_n;
        const int64_t tm = go.narrow ? SGN_BM : SG64_BM, tn = go.narrow ? SGN_BN : SG64_BN;
        const int64_t gm = (stg.M + tm - 1) / tm, gn = (stg.N + tn - 1) / tn;
        if (gm * gn * nj > 0x3fffffff) return set_error(CUTQC_EUNSUPPORTED, "run %d: too many GEMM tiles", r);
        go.gm = (int)gm;
        go.gn = (int)gn;
        if (stg.final_stage) {
          go.alpha = std::ldexp(1.0f, -plan.K);
          go.out = R.bins_dev + bins_off;
          go.out_bstride = nb;
          go.sum = bsum;
          go.streaming = 1;
        } else {
          go.alpha = 1.0f;
          go.out = step ? (float*)(step + stg.off_result) : nullptr;
          go.out_bstride = (int64_t)stg.result_elems;
          go.sum = nullptr;
          go.streaming = 0;
        }
        g.ntasks = (int)(gm * gn * nj);
        phase(p_contract + d - 1).push_back(g);
      }
      size_t p_next = p_contract + max_depth;
      // chunked top-T, then the selection
      const int64_t chunks = (nb + opt.topk_chunk - 1) / opt.topk_chunk;
      float* cval = cidx ? (float*)(cidx + (size_t)nj * chunks * Tn) : nullptr;
      if (R.T > 0) {
        Op k{};
        k.type = OP_TOPK;
        k.u.topk.vals = R.bins_dev + bins_off;
        k.u.topk.cidx = cidx;
        k.u.topk.cval = cval;
        k.u.topk.n = nb;
        k.u.topk.clen = std::min<int64_t>(nb, opt.topk_chunk);
        k.u.topk.T = R.T;
        k.u.topk.chunks = (int)chunks;
        k.ntasks = (int)(nj * chunks);
        phase(p_next++).push_back(k);
      }
      q.u.select.cidx = cidx;
      q.u.select.cval = cval;
      q.u.select.ncand = (int)(chunks * R.T);
      phase(p_next).push_back(q);
      job0 += nj;
      bins_off += (int64_t)nj * nb;
    }
  }
  // merge the runs phase by phase
  size_t n_phases = 0;
  for (auto& ph : phases) n_phases = std::max(n_phases, ph.size());
  out->ops.clear();
  out->phase_op.assign(1, 0);
  out->phase_tasks.clear();
  out->phase_kinds.clear();
  out->phase_fma.clear();
  for (size_t p = 0; p < n_phases; ++p) {
    // ops with few tasks first (a level selection, a few long tiles): CTA i
    // takes task i first, so they start at once and the many short tasks of
    // the other ops fill in around them
    std::vector<Op> ops_p;
    for (auto& ph : phases)
      if (p < ph.size()) ops_p.insert(ops_p.end(), ph[p].begin(), ph[p].end());
    std::stable_sort(ops_p.begin(), ops_p.end(), [](const Op& x, const Op& y) { return x.ntasks < y.ntasks; });
    int64_t tasks = 0;
    for (Op op : ops_p) {
      op.task0 = (int)tasks;
      tasks += op.ntasks;
      out->ops.push_back(op);
    }
    if (tasks > 0x7fffffff) return set_error(CUTQC_EUNSUPPORTED, "too many tasks in one phase");
    int kinds = 0;
    int64_t fma = 0;
    for (int i = out->phase_op.back(); i < (int)out->ops.size(); ++i) {
      const Op& op = out->ops[i];
      kinds |= 1 << op.type;
      if (op.type == OP_GEMM)
        fma += op.u.gemm.M * op.u.gemm.N * op.u.gemm.K * (op.ntasks / (op.u.gemm.gm * op.u.gemm.gn));
    }
    out->phase_kinds.push_back(kinds);
    out->phase_fma.push_back(fma);
    out->phase_op.push_back((int)out->ops.size());
    out->phase_tasks.push_back((int)tasks);
  }
  size_t o = align_up(data_end, 256);
  out->ops_off = o;
  o = align_up(o + out->ops.size() * sizeof(Op), 256);
  out->phase_off = o;
  o = align_up(o + out->phase_op.size() * sizeof(int), 256);
  out->tasks_off = o;
  o = align_up(o + out->phase_tasks.size() * sizeof(int), 256);
  out->trace_off = o;
  o = align_up(o + (out->phase_tasks.size() + 1) * sizeof(long long), 256);
  out->total = o;
  return CUTQC_OK;
}

typedef void (*PersistentKernel)(const Program);
PersistentKernel persistent_kernel(int per_sm) {
  switch (per_sm) {
    case 3: return dd_persistent_kernel<3>;
    case 4: return dd_persistent_kernel<4>;
    default: return dd_persistent_kernel<2>;
  }
}

int max_resident_ctas(int per_sm_wanted, int* out) {
  int per_sm = 0;
  CUTQC_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, persistent_kernel(per_sm_wanted), kThreads,
                                                               0));
  if (per_sm < 1) return set_error(CUTQC_EUNSUPPORTED, "the persistent DD kernel does not fit on an SM");
  *out = std::min(per_sm, per_sm_wanted) * sm_count();
  return CUTQC_OK;
}

}  // namespace
}  // namespace cutqc

struct cutqc_dd_batch {
  cutqc::Program pg;
  cutqc::PersistentKernel kernel;
  int grid;
  int n_ops;
  int device;
  std::vector<int> kinds, tasks;   // per phase
  std::vector<int64_t> fma;
};

using namespace cutqc;

extern "C" int cutqc_dd_batch_workspace_size(int n_runs, const cutqc_dd_run_desc* runs,
                                             const cutqc_dd_batch_options* opt, size_t* bytes) {
  if (!bytes) return set_error(CUTQC_EINVAL, "null bytes");
  BatchOpts o;
  int rc = read_opts(opt, &o);
  if (rc) return rc;
  Built b;
  if ((rc = build_program(n_runs, runs, o, nullptr, &b))) return rc;
  *bytes = b.total;
  return CUTQC_OK;
}

extern "C" int cutqc_dd_batch_shape(int n_runs, const cutqc_dd_run_desc* runs, const cutqc_dd_batch_options* opt,
                                    int32_t* n_phases, int32_t* n_ops, int64_t* tasks) {
  BatchOpts o;
  int rc = read_opts(opt, &o);
  if (rc) return rc;
  Built b;
  if ((rc = build_program(n_runs, runs, o, nullptr, &b))) return rc;
  if (n_phases) *n_phases = (int32_t)b.phase_tasks.size();
  if (n_ops) *n_ops = (int32_t)b.ops.size();
  if (tasks) {
    int64_t t = 0;
    for (int x : b.phase_tasks) t += x;
    *tasks = t;
  }
  return CUTQC_OK;
}

extern "C" int cutqc_dd_batch_create(int n_runs, const cutqc_dd_run_desc* runs, const cutqc_dd_batch_options* opt,
                                     void* ws_dev, size_t ws_bytes, cutqc_dd_batch** out) {
  if (!out) return set_error(CUTQC_EINVAL, "null handle");
  *out = nullptr;
  if (!ws_dev) return set_error(CUTQC_EINVAL, "null workspace");
  if (((uintptr_t)ws_dev & 255) != 0) return set_error(CUTQC_EINVAL, "workspace must be 256-byte aligned");
  BatchOpts o;
  int rc = read_opts(opt, &o);
  if (rc) return rc;
  Built b;
  if ((rc = build_program(n_runs, runs, o, (uint8_t*)ws_dev, &b))) return rc;
  if (ws_bytes < b.total) return set_error(CUTQC_ENOMEM, "DD batch workspace needs %zu bytes", b.total);
  int grid = 0;
  if ((rc = max_resident_ctas(o.ctas_per_sm, &grid))) return rc;
  if (o.ctas > 0) grid = std::min(grid, o.ctas);
  uint8_t* ws = (uint8_t*)ws_dev;
  CUTQC_CUDA_TRY(cudaMemcpy(ws + b.ops_off, b.ops.data(), b.ops.size() * sizeof(Op), cudaMemcpyHostToDevice));
  CUTQC_CUDA_TRY(cudaMemcpy(ws + b.phase_off, b.phase_op.data(), b.phase_op.size() * sizeof(int),
                            cudaMemcpyHostToDevice));
  CUTQC_CUDA_TRY(cudaMemcpy(ws + b.tasks_off, b.phase_tasks.data(), b.phase_tasks.size() * sizeof(int),
                            cudaMemcpyHostToDevice));
  int* status = device_status_ptr();
  if (!status) return set_error(CUTQC_ECUDA, "no device status word");
  cutqc_dd_batch* h = new (std::nothrow) cutqc_dd_batch;
  if (!h) return set_error(CUTQC_ENOMEM, "host allocation");
  h->pg.ops = (const Op*)(ws + b.ops_off);
  h->pg.phase_op = (const int*)(ws + b.phase_off);
  h->pg.phase_tasks = (const int*)(ws + b.tasks_off);
  h->pg.n_phases = (int)b.phase_tasks.size();
  h->pg.bar = (GridBar*)ws;
  h->pg.status = status;
  h->pg.trace = (long long*)(ws + b.trace_off);
  h->kinds = b.phase_kinds;
  h->tasks = b.phase_tasks;
  h->fma = b.phase_fma;
  h->grid = grid;
  h->kernel = persistent_kernel(o.ctas_per_sm);
  h->n_ops = (int)b.ops.size();
  cudaGetDevice(&h->device);
  *out = h;
  return CUTQC_OK;
}

extern "C" int cutqc_dd_batch_launch(const cutqc_dd_batch* b, void* stream) {
  if (!b) return set_error(CUTQC_EINVAL, "null handle");
  cudaStream_t st = (cudaStream_t)stream;
  CUTQC_CUDA_TRY(cudaMemsetAsync(b->pg.bar, 0, sizeof(GridBar), st));
  if (b->pg.n_phases == 0) return CUTQC_OK;
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3((unsigned)b->grid);
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  CUTQC_CUDA_TRY(cudaLaunchKernelEx(&cfg, b->kernel, b->pg));
  count_launches(1);
  return CUTQC_OK;
}

extern "C" int cutqc_dd_batch_info(const cutqc_dd_batch* b, int32_t* n_phases, int32_t* n_ops, int32_t* grid_ctas) {
  if (!b) return set_error(CUTQC_EINVAL, "null handle");
  if (n_phases) *n_phases = b->pg.n_phases;
  if (n_ops) *n_ops = b->n_ops;
  if (grid_ctas) *grid_ctas = b->grid;
  return CUTQC_OK;
}

extern "C" int cutqc_dd_batch_phases(const cutqc_dd_batch* b, int32_t* kinds, int32_t* tasks, int64_t* fma,
                                     int64_t* cycles, int n) {
  if (!b) return set_error(CUTQC_EINVAL, "null handle");
  if (n != b->pg.n_phases) return set_error(CUTQC_EINVAL, "n must be the number of phases (%d)", b->pg.n_phases);
  for (int p = 0; p < n; ++p) {
    if (kinds) kinds[p] = b->kinds[p];
    if (tasks) tasks[p] = b->tasks[p];
    if (fma) fma[p] = b->fma[p];
  }
  if (cycles && n > 0) {
    std::vector<long long> t(n + 1);
    CUTQC_CUDA_TRY(cudaMemcpy(t.data(), b->pg.trace, (n + 1) * sizeof(long long), cudaMemcpyDeviceToHost));
    for (int p = 0; p < n; ++p) cycles[p] = t[p + 1] - t[p];
  }
  return CUTQC_OK;
}

extern "C" int cutqc_dd_batch_destroy(cutqc_dd_batch* b) {
  delete b;
  return CUTQC_OK;
}
