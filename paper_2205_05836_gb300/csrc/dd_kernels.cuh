// Device bodies of the dynamic-definition steps (Algorithm 1): merge, the
// slice reduction of the merge, top-T selection and the level selection.
// The stand-alone launches (dd.cu) and the persistent kernel (dd_persist.cu)
// run the same bodies; each takes its block coordinates as arguments.
//
// kCoherent: the body reads data that other CTAs of the same launch wrote
// earlier (the persistent kernel, after a grid barrier).  Such reads go
// through L2 (ld.global.cg), never through the non-coherent read-only path,
// which is only valid for data no CTA writes while the launch runs.
#pragma once

#include "internal.cuh"

#include <math.h>

namespace cutqc {

template <bool kCoherent, class T>
__device__ __forceinline__ T ldx(const T* p) {
  if constexpr (kCoherent) return __ldcg(p);
  else return __ldg(p);
}

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

// Zoom source of a merge: either a per-job array of zoom values over the
// subcircuit's output bits (zoom_dev), or the level's job records, from which
// each job's value is derived (bit t = the fixed value of output qubit
// outq[t], for the qubits below lo), or one constant (zoom_val).
struct ZoomFromJobs {
  const cutqc_dd_job_result* jobs;   // null: not used
  int o, lo;
  int8_t outq[32];
};

template <bool kCoherent>
__device__ __forceinline__ uint64_t job_zoom(const ZoomFromJobs& zj, int job) {
  const cutqc_dd_job_result& J = zj.jobs[job];
  const unsigned long long zv0 = ldx<kCoherent>((const unsigned long long*)&J.zoom_val[0]);
  const unsigned long long zv1 = ldx<kCoherent>((const unsigned long long*)&J.zoom_val[1]);
  uint64_t z = 0;
  for (int t = 0; t < zj.o; ++t) {
    const int q = zj.outq[t];
    if (q < zj.lo && ((((q >> 6) ? zv1 : zv0) >> (q & 63)) & 1)) z |= (uint64_t)1 << t;
  }
  return z;
}

// Merge: merged[job][a][c] = sum_m attributed[x(a, z_job, m)][c] over the
// merged index range of slice bz (2^log_slices slices; slice bz writes its
// partial sums to out + bz * n_jobs * rows_a * C).  Block bx of nbx walks
// the (merged row a, job) pairs.  Threads split columns and, when there are
// few columns, the slice's merged indices; sub-slices are combined through
// shared memory.  The attributed tensor is read-only for the launch.
template <bool kCoherent>
__device__ __forceinline__ void dd_merge_body(const float* __restrict__ att, int k, uint64_t act_mask,
                                              uint64_t merged_mask, uint64_t zoom_mask, uint64_t zoom_val,
                                              const uint64_t* __restrict__ zoom_dev, const ZoomFromJobs& zj,
                                              int n_jobs, int64_t rows_a, int n_merged, int log_slices,
                                              float* __restrict__ out, int64_t bx, int64_t nbx, int bz) {
  __shared__ float red[256];
  const int64_t C = (int64_t)1 << (2 * k);
  const int64_t Mper = (int64_t)1 << (n_merged - log_slices);
  const int64_t m0 = (int64_t)bz * Mper;
  const int cw = (int)(C < 256 ? C : 256);
  const int slices = 256 / cw;
  const int c_local = threadIdx.x % cw;
  const int slice = threadIdx.x / cw;
  for (int64_t ra = bx; ra < rows_a * n_jobs; ra += nbx) {
    const int job = (int)(ra / rows_a);
    const int64_t a = ra - (int64_t)job * rows_a;
    const uint64_t z = (zj.jobs ? job_zoom<kCoherent>(zj, job) : zoom_dev ? __ldg(zoom_dev + job) : zoom_val) &
                       zoom_mask;
    const uint64_t base = pdep64((uint64_t)a, act_mask) | z;
    float* dst = out + (((int64_t)bz * n_jobs + job) * rows_a + a) * C;
    for (int64_t c0 = 0; c0 < C; c0 += cw) {
      Kahan acc;
      if (slice < slices)
        for (int64_t m = m0 + slice; m < m0 + Mper; m += slices) {
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
}

// out[e] = sum over the S slices of part[s * E + e], in slice order; block bx
// of nbx.
template <bool kCoherent>
__device__ __forceinline__ void dd_merge_reduce_body(const float* __restrict__ part, int S, int64_t E,
                                                     float* __restrict__ out, int64_t bx, int64_t nbx) {
  for (int64_t e = bx * blockDim.x + threadIdx.x; e < E; e += nbx * blockDim.x) {
    Kahan acc;
    for (int q = 0; q < S; ++q) acc.add(ldx<kCoherent>(part + (int64_t)q * E + e));
    out[e] = acc.s;
  }
}

// The T largest entries of one job by (value desc, index asc).  Block (job,
// chunk) of (., nchunks) scans entries [chunk * chunk_len, (chunk + 1) *
// chunk_len) of job `job`'s n entries and writes its T best to slot (job *
// nchunks + chunk).  kCand = false: the entries are bins and an entry's index
// is its position; kCand = true: the entries are (value, index) candidates of
// an earlier pass (index -1 = none), which is how large jobs are finished
// (chunked pass, then one block per job over the chunks' candidates).  One
// pass: each thread keeps its own best TCAP (sorted), then T rounds pick the
// block's best head and advance its owner.
__device__ __forceinline__ bool dd_better(float v, int i, float w, int j) {
  return v > w || (v == w && i < j);
}

template <int TCAP, bool kCand, bool kCoherent>
__device__ __forceinline__ void dd_topk_body(const float* __restrict__ vals, const int32_t* __restrict__ cidx,
                                             int64_t n, int64_t chunk_len, int T, int32_t* __restrict__ top_idx,
                                             float* __restrict__ top_val, int job, int chunk, int nchunks) {
  __shared__ float sv[32];
  __shared__ int si[32];
  __shared__ int win_i;
  const float* b = vals + (int64_t)job * n;
  const int32_t* ci = kCand ? cidx + (int64_t)job * n : nullptr;
  const int64_t lo = (int64_t)chunk * chunk_len;
  const int64_t hi = lo + chunk_len < n ? lo + chunk_len : n;
  const int64_t slot = ((int64_t)job * nchunks + chunk) * T;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float lv[TCAP];
  int li[TCAP];
#pragma unroll
  for (int u = 0; u < TCAP; ++u) { lv[u] = -INFINITY; li[u] = -1; }   // read only once filled
  int cnt = 0;
  auto offer = [&](float v, int idx) {
    if (cnt == T && !dd_better(v, idx, lv[T - 1], li[T - 1])) return;
    int pos = cnt < T ? cnt : T - 1;
#pragma unroll
    for (int u = TCAP - 1; u > 0; --u)
      if (u <= pos && dd_better(v, idx, lv[u - 1], li[u - 1])) { lv[u] = lv[u - 1]; li[u] = li[u - 1]; pos = u - 1; }
    // pos is now the first slot whose left neighbour ranks before (v, idx)
    lv[pos] = v;
    li[pos] = idx;
    if (cnt < T) ++cnt;
  };
  int64_t tail0 = lo;
  if (!kCand && (((uintptr_t)(b + lo)) & 15) == 0) {
    // bins: float4 loads, four in flight per thread (the order in which a
    // thread offers entries does not matter: ties compare indices)
    constexpr int U = 4;
    const float4* p4 = reinterpret_cast<const float4*>(b + lo);
    const int64_t n4 = (hi - lo) >> 2;
    for (int64_t q = threadIdx.x; q < n4; q += U * (int64_t)blockDim.x) {
      float4 v[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int64_t qu = q + u * (int64_t)blockDim.x;
        v[u] = qu < n4 ? ldx<kCoherent>(p4 + qu) : make_float4(0.f, 0.f, 0.f, 0.f);
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int64_t qu = q + u * (int64_t)blockDim.x;
        if (qu < n4) {
          const int i0 = (int)(lo + 4 * qu);
          offer(v[u].x, i0); offer(v[u].y, i0 + 1); offer(v[u].z, i0 + 2); offer(v[u].w, i0 + 3);
        }
      }
    }
    tail0 = lo + 4 * n4;
  }
  for (int64_t i = tail0 + threadIdx.x; i < hi; i += blockDim.x) {
    const float v = ldx<kCoherent>(b + i);
    const int idx = kCand ? ldx<kCoherent>(ci + i) : (int)i;
    if (kCand && idx < 0) continue;
    offer(v, idx);
  }
  int head = 0;
  for (int t = 0; t < T; ++t) {
    float bv = -INFINITY;
    int bi = -1;
#pragma unroll
    for (int u = 0; u < TCAP; ++u)
      if (u == head && head < cnt) { bv = lv[u]; bi = li[u]; }
    for (int off = 16; off; off >>= 1) {
      const float ov = __shfl_xor_sync(0xffffffffu, bv, off);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, off);
      if (oi >= 0 && (bi < 0 || ov > bv || (ov == bv && oi < bi))) { bv = ov; bi = oi; }
    }
    if (lane == 0) { sv[warp] = bv; si[warp] = bi; }
    __syncthreads();
    if (warp == 0) {
      const int nw = blockDim.x >> 5;
      bv = lane < nw ? sv[lane] : -INFINITY;
      bi = lane < nw ? si[lane] : -1;
      for (int off = 16; off; off >>= 1) {
        const float ov = __shfl_xor_sync(0xffffffffu, bv, off);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, off);
        if (oi >= 0 && (bi < 0 || ov > bv || (ov == bv && oi < bi))) { bv = ov; bi = oi; }
      }
      if (lane == 0) {
        win_i = bi;
        top_idx[slot + t] = bi;
        top_val[slot + t] = bi >= 0 ? bv : 0.f;
      }
    }
    __syncthreads();
    // the owner of the winning index advances (indices are distinct)
    if (head < cnt && win_i >= 0) {
      int cur = -1;
#pragma unroll
      for (int u = 0; u < TCAP; ++u)
        if (u == head) cur = li[u];
      if (cur == win_i) ++head;
    }
    __syncthreads();
  }
}

struct LevelInfo {
  int level, depth, n_active;
  int8_t active[32];
};

// Run by the first warp of a block (the other threads return at once; no
// block-wide barrier inside).  Completes the records of this level's jobs
// (bin totals, the T largest bins, bin offsets) and, when merged qubits
// remain, writes the records of the next level: the T largest bins over all
// valid jobs of this level, ordered by value (stable: job order, then each
// job's own order, for equal values) -- Algorithm 1's list L truncated to T.
// Records past the candidates are placeholders (level -1).  Lane 0 ranks the
// candidates; the 32-entry arrays of a record are written one entry per lane.
template <bool kCoherent>
__device__ __forceinline__ void dd_select_body(cutqc_dd_job_result* __restrict__ jobs, int job0, int nj,
                                               const LevelInfo& L, int64_t bins_off0, int64_t nb,
                                               const double* __restrict__ bsum, const int32_t* __restrict__ tidx,
                                               const float* __restrict__ tval, int T, int has_children, int n_next,
                                               int32_t* __restrict__ n_jobs_dev) {
  __shared__ int cj[32], cb[32], cnt_s;
  // the level's candidates (nj * T of them, job order) loaded in parallel
  __shared__ int kb[1024];
  __shared__ float kv[1024];
  if (threadIdx.x >= 32) return;
  const int lane = threadIdx.x;
  for (int j = 0; j < nj; ++j) {
    cutqc_dd_job_result& J = jobs[job0 + j];
    const bool valid = ldx<kCoherent>(&J.level) >= 0;
    const int32_t ti = (valid && lane < T) ? ldx<kCoherent>(tidx + (int64_t)j * T + lane) : -1;
    J.top_idx[lane] = ti;
    J.top_val[lane] = ti >= 0 ? ldx<kCoherent>(tval + (int64_t)j * T + lane) : 0.f;
    J.active[lane] = lane < L.n_active ? L.active[lane] : 0;
    if (lane == 0) {
      J.n_active = L.n_active;
      J.bin_sum = valid ? ldx<kCoherent>(bsum + j) : 0.0;
      J.bins_offset = bins_off0 + (int64_t)j * nb;
    }
  }
  if (!has_children) {
    if (lane == 0) *n_jobs_dev = job0 + nj;
    return;
  }
  const int ncand = nj * T <= 1024 ? nj * T : 1024;
  for (int q = lane; q < ncand; q += 32) {
    const int j = q / T;
    const int b = ldx<kCoherent>(&jobs[job0 + j].level) >= 0 ? ldx<kCoherent>(tidx + q) : -1;
    kb[q] = b;
    kv[q] = b >= 0 ? ldx<kCoherent>(tval + q) : 0.f;
  }
  __syncwarp();
  if (lane == 0) {
    float cv[32];
    int cnt = 0;
    for (int j = 0; j < nj; ++j) {
      for (int t = 0; t < T; ++t) {
        const int q = j * T + t;
        if (q >= ncand) break;
        const int b = kb[q];
        if (b < 0) continue;
        const float v = kv[q];
        int pos = cnt;
        while (pos > 0 && cv[pos - 1] < v) --pos;     // after every entry of equal value
        if (pos >= T) continue;
        const int last = cnt < T ? cnt : T - 1;
        for (int u = last; u > pos; --u) { cv[u] = cv[u - 1]; cj[u] = cj[u - 1]; cb[u] = cb[u - 1]; }
        cv[pos] = v;
        cj[pos] = j;
        cb[pos] = b;
        if (cnt < T) ++cnt;
      }
    }
    cnt_s = cnt;
  }
  __syncwarp();
  const int cnt = cnt_s;
  const int next0 = job0 + nj;
  for (int c = 0; c < n_next; ++c) {
    cutqc_dd_job_result& R = jobs[next0 + c];
    R.top_idx[lane] = -1;
    R.top_val[lane] = 0.f;
    R.active[lane] = 0;
    if (lane == 0) {
      R.n_active = 0;
      R.bin_sum = 0.0;
      R.bins_offset = 0;
      R.depth = L.depth + 1;
      if (c < cnt) {
        const cutqc_dd_job_result& P = jobs[job0 + cj[c]];
        R.level = L.level + 1;
        R.parent = job0 + cj[c];
        R.parent_bin = cb[c];
        for (int w = 0; w < 2; ++w) {
          R.zoom_mask[w] = ldx<kCoherent>((const unsigned long long*)&P.zoom_mask[w]);
          R.zoom_val[w] = ldx<kCoherent>((const unsigned long long*)&P.zoom_val[w]);
        }
        for (int a = 0; a < L.n_active; ++a) {
          const int q = L.active[a];
          R.zoom_mask[q >> 6] |= (uint64_t)1 << (q & 63);
          if ((cb[c] >> a) & 1) R.zoom_val[q >> 6] |= (uint64_t)1 << (q & 63);
        }
      } else {
        R.level = -1;
        R.parent = -1;
        R.parent_bin = -1;
        for (int w = 0; w < 2; ++w) { R.zoom_mask[w] = 0; R.zoom_val[w] = 0; }
      }
    }
  }
  if (lane == 0) *n_jobs_dev = next0 + n_next;
}

// The first job of a run: nothing zoomed.  One thread.
__device__ __forceinline__ void dd_first_job_body(cutqc_dd_job_result* __restrict__ jobs) {
  cutqc_dd_job_result& J = jobs[0];
  J.level = 0;
  J.depth = 0;
  J.parent = -1;
  J.parent_bin = -1;
  for (int w = 0; w < 2; ++w) { J.zoom_mask[w] = 0; J.zoom_val[w] = 0; }
}

}  // namespace cutqc
