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
// partial sums to out + bz * n_jobs * rows_a * C).  The CTA's threads form
// G = 256 / cw groups of cw = min(C, 256) column threads.  When the slice
// holds at least G merged indices, block bx of nbx walks the (merged row a,
// job) pairs one at a time, group g sums the indices m0 + g, m0 + g + G, ...
// (compensated), and the groups' sums are added in group order; otherwise
// (merge_groups() > 1) each group takes its own row, rows bx * G + g, then
// nbx * G further, and sums the slice's indices in order.  The attributed
// tensor is read-only for the launch.  Loads of consecutive merged indices
// are issued four at a time; the source row of index m + d is the bit
// deposit of m + d, carried in the deposited domain.
__host__ __device__ __forceinline__ int merge_groups(int k, int n_merged, int log_slices) {
  const int cw = 2 * k >= 8 ? 256 : (1 << (2 * k));
  const int G = 256 / cw;
  return ((int64_t)1 << (n_merged - log_slices)) < G ? G : 1;
}

// sum over count indices first, first + step, ... of att[(base | pdep(m)) * C + col]
__device__ __forceinline__ float merge_run(const float* __restrict__ att, int64_t C, uint64_t base,
                                           uint64_t merged_mask, int64_t first, int64_t step, int64_t count,
                                           int64_t col) {
  Kahan acc;
  const uint64_t keep = ~merged_mask;
  const uint64_t dx = pdep64((uint64_t)step, merged_mask);
  uint64_t x = pdep64((uint64_t)first, merged_mask);
  auto next = [&](uint64_t v) { return ((v | keep) + dx) & merged_mask; };
  int64_t i = 0;
  for (; i + 4 <= count; i += 4) {
    const uint64_t x1 = next(x), x2 = next(x1), x3 = next(x2);
    const float v0 = __ldg(att + (int64_t)(base | x) * C + col);
    const float v1 = __ldg(att + (int64_t)(base | x1) * C + col);
    const float v2 = __ldg(att + (int64_t)(base | x2) * C + col);
    const float v3 = __ldg(att + (int64_t)(base | x3) * C + col);
    acc.add(v0);
    acc.add(v1);
    acc.add(v2);
    acc.add(v3);
    x = next(x3);
  }
  for (; i < count; ++i) {
    acc.add(__ldg(att + (int64_t)(base | x) * C + col));
    x = next(x);
  }
  return acc.s;
}

template <bool kCoherent>
__device__ __forceinline__ void dd_merge_body(const float* __restrict__ att, int k, uint64_t act_mask,
                                              uint64_t merged_mask, uint64_t zoom_mask, uint64_t zoom_val,
                                              const uint64_t* __restrict__ zoom_dev, const ZoomFromJobs& zj,
                                              int n_jobs, int64_t rows_a, int n_merged, int log_slices,
                                              float* __restrict__ out, int64_t bx, int64_t nbx, int bz) {
  __shared__ float red[256];
  __shared__ uint64_t zs[32];
  const int64_t C = (int64_t)1 << (2 * k);
  const int64_t Mper = (int64_t)1 << (n_merged - log_slices);
  const int64_t m0 = (int64_t)bz * Mper;
  const int cw = (int)(C < 256 ? C : 256);
  const int G = 256 / cw;
  const int c_local = threadIdx.x % cw;
  const int grp = threadIdx.x / cw;
  // the jobs' zoom values, once per block when they come from the records
  const bool zsm = zj.jobs && n_jobs <= 32;
  if (zsm) {
    if (threadIdx.x < n_jobs) zs[threadIdx.x] = job_zoom<kCoherent>(zj, threadIdx.x);
    __syncthreads();
  }
  auto zoom_of = [&](int job) -> uint64_t {
    return (zsm ? zs[job] : zj.jobs ? job_zoom<kCoherent>(zj, job) : zoom_dev ? __ldg(zoom_dev + job) : zoom_val) &
           zoom_mask;
  };
  const int64_t total = rows_a * n_jobs;
  if (merge_groups(k, n_merged, log_slices) > 1) {
    const int64_t stride = nbx * G;
    if (Mper == 1) {
      // one merged index per row: a gather; four rows in flight per thread
      const uint64_t xm = pdep64((uint64_t)m0, merged_mask);
      for (int64_t ra0 = bx * G + grp; ra0 < total; ra0 += 4 * stride) {
        int64_t src[4], dst[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int64_t ra = ra0 + u * stride;
          src[u] = dst[u] = -1;
          if (ra < total) {
            const int job = (int)(ra / rows_a);
            const int64_t a = ra - (int64_t)job * rows_a;
            src[u] = (int64_t)(pdep64((uint64_t)a, act_mask) | zoom_of(job) | xm) * C;
            dst[u] = (((int64_t)bz * n_jobs + job) * rows_a + a) * C;
          }
        }
        for (int64_t c0 = 0; c0 < C; c0 += cw) {
          float v[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) v[u] = src[u] >= 0 ? __ldg(att + src[u] + c0 + c_local) : 0.f;
#pragma unroll
          for (int u = 0; u < 4; ++u)
            if (dst[u] >= 0) out[dst[u] + c0 + c_local] = v[u];
        }
      }
      return;
    }
    for (int64_t ra = bx * G + grp; ra < total; ra += stride) {
      const int job = (int)(ra / rows_a);
      const int64_t a = ra - (int64_t)job * rows_a;
      const uint64_t base = pdep64((uint64_t)a, act_mask) | zoom_of(job);
      float* dst = out + (((int64_t)bz * n_jobs + job) * rows_a + a) * C;
      for (int64_t c0 = 0; c0 < C; c0 += cw)
        dst[c0 + c_local] = merge_run(att, C, base, merged_mask, m0, 1, Mper, c0 + c_local);
    }
    return;
  }
  for (int64_t ra = bx; ra < total; ra += nbx) {
    const int job = (int)(ra / rows_a);
    const int64_t a = ra - (int64_t)job * rows_a;
    const uint64_t base = pdep64((uint64_t)a, act_mask) | zoom_of(job);
    float* dst = out + (((int64_t)bz * n_jobs + job) * rows_a + a) * C;
    const int64_t cnt = (Mper - grp + G - 1) / G;
    for (int64_t c0 = 0; c0 < C; c0 += cw) {
      red[threadIdx.x] = merge_run(att, C, base, merged_mask, m0 + grp, G, cnt, c0 + c_local);
      __syncthreads();
      if (grp == 0) {
        float s = red[c_local];
        for (int q = 1; q < G; ++q) s += red[q * cw + c_local];
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

// One thread's best T <= TCAP entries, sorted.  Short lists insert by a
// compare-and-swap chain over the kept slots: every index is a compile-time
// constant, so the list lives in registers.  Once the list is full, thr/thri
// hold its T-th entry and an entry enters only if it ranks before that one.
template <int TCAP>
struct TopList {
  float lv[TCAP];
  int li[TCAP];
  int cnt;
  float thr;
  int thri;
  __device__ __forceinline__ void init() {
#pragma unroll
    for (int u = 0; u < TCAP; ++u) { lv[u] = -INFINITY; li[u] = -1; }   // read only once filled
    cnt = 0;
    thr = -INFINITY;
    thri = -1;
  }
  // long lists: shift the worse entries right and write the new one at a
  // computed slot (the list sits in local memory; insertions are rare, so
  // one out-of-line copy serves every call site)
  __device__ __noinline__ void insert_long(float v, int idx, int T) {
    int pos = cnt < T ? cnt : T - 1;
#pragma unroll
    for (int u = TCAP - 1; u > 0; --u)
      if (u <= pos && dd_better(v, idx, lv[u - 1], li[u - 1])) { lv[u] = lv[u - 1]; li[u] = li[u - 1]; pos = u - 1; }
    lv[pos] = v;
    li[pos] = idx;
  }
  __device__ __forceinline__ void offer(float v, int idx, int T) {
    if (cnt == T && !dd_better(v, idx, thr, thri)) return;
    if constexpr (TCAP <= 8) {
      float cv = v;
      int cix = idx;
#pragma unroll
      for (int u = 0; u < TCAP; ++u) {
        if (u < cnt) {
          if (dd_better(cv, cix, lv[u], li[u])) {
            const float tv = lv[u];
            const int ti = li[u];
            lv[u] = cv; li[u] = cix; cv = tv; cix = ti;
          }
        } else if (u == cnt && u < T) {
          lv[u] = cv; li[u] = cix;
        }
      }
    } else {
      insert_long(v, idx, T);
    }
    if (cnt < T) ++cnt;
    if (cnt == T) {
#pragma unroll
      for (int u = 0; u < TCAP; ++u)
        if (u == T - 1) { thr = lv[u]; thri = li[u]; }
    }
  }
};

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
  TopList<TCAP> L;
  L.init();
  auto offer = [&](float v, int idx) { L.offer(v, idx, T); };
  int64_t tail0 = lo;
  if (!kCand && (((uintptr_t)(b + lo)) & 15) == 0) {
    // bins: float4 loads, four in flight per thread.  A thread offers its
    // entries in increasing index order, so once its list is full an entry
    // equal to the T-th kept value never enters and a float4 whose largest
    // lane is <= thr is skipped whole.
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
        const float m = fmaxf(fmaxf(v[u].x, v[u].y), fmaxf(v[u].z, v[u].w));
        if (qu < n4 && (L.cnt < T || m > L.thr)) {
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
      if (u == head && head < L.cnt) { bv = L.lv[u]; bi = L.li[u]; }
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
    if (head < L.cnt && win_i >= 0) {
      int cur = -1;
#pragma unroll
      for (int u = 0; u < TCAP; ++u)
        if (u == head) cur = L.li[u];
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
// block-wide barrier inside).  Completes the records of this level's nj <= 32
// jobs (bin totals, the T largest bins, bin offsets) and, when merged qubits
// remain, writes the records of the next level: the T largest bins over all
// valid jobs of this level, ordered by value (stable: job order, then each
// job's own order, for equal values) -- Algorithm 1's list L truncated to T.
// Records past the candidates are placeholders (level -1).  The loads are
// issued across lanes (lane j: job j; the nj * T candidates by all lanes),
// lane 0 ranks the candidates, lane c writes next-level record c, and the
// 32-entry arrays of a record are written one entry per lane.
template <bool kCoherent>
__device__ __forceinline__ void dd_select_body(cutqc_dd_job_result* __restrict__ jobs, int job0, int nj,
                                               const LevelInfo& L, int64_t bins_off0, int64_t nb,
                                               const double* __restrict__ bsum, const int32_t* __restrict__ tidx,
                                               const float* __restrict__ tval, int T, int has_children, int n_next,
                                               int32_t* __restrict__ n_jobs_dev) {
  __shared__ int cj[32], cb[32], cnt_s;
  // the level's candidates (nj * T <= 1024 of them, job order)
  __shared__ int kb[1024];
  __shared__ float kv[1024];
  if (threadIdx.x >= 32) return;
  const int lane = threadIdx.x;
  int lvl = -1;
  double bs = 0.0;
  if (lane < nj) {
    lvl = ldx<kCoherent>(&jobs[job0 + lane].level);
    if (lvl >= 0) bs = ldx<kCoherent>(bsum + lane);
  }
  const unsigned valid = __ballot_sync(0xffffffffu, lane < nj && lvl >= 0);
  const int ncand = nj * T;
  for (int q = lane; q < ncand; q += 32) {
    const int b = ((valid >> (q / T)) & 1) ? ldx<kCoherent>(tidx + q) : -1;
    kb[q] = b;
    kv[q] = b >= 0 ? ldx<kCoherent>(tval + q) : 0.f;
  }
  __syncwarp();
  for (int j = 0; j < nj; ++j) {
    cutqc_dd_job_result& J = jobs[job0 + j];
    const int32_t ti = lane < T ? kb[j * T + lane] : -1;
    J.top_idx[lane] = ti;
    J.top_val[lane] = ti >= 0 ? kv[j * T + lane] : 0.f;
    J.active[lane] = lane < L.n_active ? L.active[lane] : 0;
  }
  if (lane < nj) {
    cutqc_dd_job_result& J = jobs[job0 + lane];
    J.n_active = L.n_active;
    J.bin_sum = lvl >= 0 ? bs : 0.0;
    J.bins_offset = bins_off0 + (int64_t)lane * nb;
  }
  if (!has_children) {
    if (lane == 0) *n_jobs_dev = job0 + nj;
    return;
  }
  if (lane == 0) {
    float cv[32];
    int cnt = 0;
    for (int q = 0; q < ncand; ++q) {
      const int b = kb[q];
      if (b < 0) continue;
      const float v = kv[q];
      int pos = cnt;
      while (pos > 0 && cv[pos - 1] < v) --pos;     // after every entry of equal value
      if (pos >= T) continue;
      const int last = cnt < T ? cnt : T - 1;
      for (int u = last; u > pos; --u) { cv[u] = cv[u - 1]; cj[u] = cj[u - 1]; cb[u] = cb[u - 1]; }
      cv[pos] = v;
      cj[pos] = q / T;
      cb[pos] = b;
      if (cnt < T) ++cnt;
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
  }
  if (lane < n_next) {
    cutqc_dd_job_result& R = jobs[next0 + lane];
    R.n_active = 0;
    R.bin_sum = 0.0;
    R.bins_offset = 0;
    R.depth = L.depth + 1;
    if (lane < cnt) {
      const cutqc_dd_job_result& P = jobs[job0 + cj[lane]];
      unsigned long long zm[2], zv[2];
      for (int w = 0; w < 2; ++w) {
        zm[w] = ldx<kCoherent>((const unsigned long long*)&P.zoom_mask[w]);
        zv[w] = ldx<kCoherent>((const unsigned long long*)&P.zoom_val[w]);
      }
      for (int a = 0; a < L.n_active; ++a) {
        const int q = L.active[a];
        const unsigned long long bit = 1ull << (q & 63);
        if (q >> 6) {
          zm[1] |= bit;
          if ((cb[lane] >> a) & 1) zv[1] |= bit;
        } else {
          zm[0] |= bit;
          if ((cb[lane] >> a) & 1) zv[0] |= bit;
        }
      }
      R.level = L.level + 1;
      R.parent = job0 + cj[lane];
      R.parent_bin = cb[lane];
      R.zoom_mask[0] = zm[0];
      R.zoom_mask[1] = zm[1];
      R.zoom_val[0] = zv[0];
      R.zoom_val[1] = zv[1];
    } else {
      R.level = -1;
      R.parent = -1;
      R.parent_bin = -1;
      for (int w = 0; w < 2; ++w) { R.zoom_mask[w] = 0; R.zoom_val[w] = 0; }
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
