/* cutqc.h -- C ABI of the GB300 reconstruction library for cut quantum
 * circuits (Tang & Martonosi, "Cutting Quantum Circuits to Run on Quantum and
 * Classical Platforms", arXiv 2205.05836).
 *
 * The library rebuilds the output distribution of a circuit that was cut into
 * subcircuits by K wire cuts, from the subcircuits' measured outputs:
 *
 *   attribution    variant outputs -> edge-basis tensors   (Circuit Cutting
 *                  section: per cut the Pauli bases {I,X,Y,Z}, subcircuits
 *                  "initialized and measured slightly differently")
 *   FD             P = 2^-K sum_{e in {I,X,Y,Z}^K} kron_i p_{i,e}   (Eq. 1,
 *                  Full Definition Post-Processing)
 *   DD             bins over active qubits, merged qubits summed, zoomed
 *                  qubits fixed (Algorithm 1, Dynamic Definition)
 *
 * Conventions (all calls):
 *  - Pointers named *_dev or documented as device pointers are CUDA device
 *    memory owned by the caller; the library never frees caller memory and
 *    never allocates device memory except where a call says so.
 *  - `stream` is a cudaStream_t passed as void*; work is enqueued
 *    asynchronously on it (0 = legacy default stream).  Host arrays are read
 *    during the call only.
 *  - Every call returns CUTQC_OK or a negative error code; the text of the
 *    last error of the calling thread is returned by cutqc_last_error().
 *    Arguments are validated on the host before any launch; on an error
 *    nothing is enqueued.
 *  - Bit order: qubit q of the uncut circuit is bit q of an output index;
 *    local qubit q of a subcircuit is bit q of its outcome index.
 *  - Edge bases are numbered I=0, X=1, Y=2, Z=3.
 */
#ifndef CUTQC_H
#define CUTQC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define CUTQC_OK 0
#define CUTQC_EINVAL (-1)      /* bad shape, descriptor or argument */
#define CUTQC_ENOMEM (-2)      /* workspace smaller than the size query */
#define CUTQC_ECUDA (-3)       /* CUDA error (launch or runtime) */
#define CUTQC_ETIMEOUT (-4)    /* a bounded device-side wait expired */
#define CUTQC_EUNSUPPORTED (-5)/* valid but outside the library's limits */

#define CUTQC_F64 0
#define CUTQC_F32 1

#define CUTQC_ORDER_KRON 0     /* numpy kron order: subcircuit 0's bits most significant */
#define CUTQC_ORDER_ORIGINAL 1 /* index = sum_q b_q 2^q over the uncut circuit's qubits */

#define CUTQC_PREC_FP32_SIMT 0  /* FP32 CUDA-core contraction */
#define CUTQC_PREC_FP16X3_TC 1  /* tcgen05 tensor cores: FP16 hi/lo split operands with
                                   per-row power-of-two scales, hi*hi + hi*lo + lo*hi,
                                   FP32 accumulation in tensor memory */
#define CUTQC_PREC_FP16X3_TC_PRUNE 2
                                /* as CUTQC_PREC_FP16X3_TC, and the last contraction
                                   skips cut terms of negligible weight: term k (an
                                   assignment of the digits it sums over) is bounded by
                                   w_k = 2^-K sum_m |A[m][k]| sum_n |B[n][k]| in L1 over
                                   the outputs; the terms of smallest w_k are skipped
                                   while their total stays <= CUTQC_PRUNE_TOL, so the
                                   output moves by at most that in L1 (TV by half).
                                   The kept terms are chosen on the device. */
#define CUTQC_PRUNE_TOL 9.313225746154785e-10  /* 2^-30 */

/* Limits of the library. */
#define CUTQC_MAX_QUBITS 34     /* n of an FD reconstruction (2^34 outputs) */
#define CUTQC_MAX_CUTS 16       /* K per reconstruction */
#define CUTQC_MAX_WIDTH 30      /* w of one subcircuit */

/* One subcircuit (host memory).  Its local qubits 0..w-1 are its wire
 * segments.  k_in of them start at a cut (initialised in |0>,|1>,|+>,|+i>),
 * k_out end at a cut (measured in the computational, X or Y basis); the
 * other w - k_out local qubits are outputs of the uncut circuit.
 *   in_local[j], out_local[j]  local qubit of the j-th init / meas cut,
 *                              strictly ascending
 *   in_edge[j], out_edge[j]    global cut-edge id (0..K-1) of that cut
 *   out_qubit[t]               uncut-circuit qubit of the t-th output qubit
 *                              (outputs in ascending local order)        */
typedef struct cutqc_subcircuit {
  int32_t w;
  int32_t k_in;
  int32_t k_out;
  const int32_t* in_local;
  const int32_t* out_local;
  const int32_t* in_edge;
  const int32_t* out_edge;
  const int32_t* out_qubit;
} cutqc_subcircuit;

/* Text of the calling thread's last error ("" if none). */
const char* cutqc_last_error(void);

/* Library version string. */
const char* cutqc_version(void);

/* Reads and clears the device status word written by bounded device-side
 * waits (0 = none expired).  Synchronises the device. */
int cutqc_device_status(int32_t* status_out);

/* Number of kernels the library has enqueued in this process so far (a
 * launch captured into a CUDA graph counts once, at capture; graph replays
 * do not count).  No paper counterpart: for launch accounting.             */
int cutqc_kernel_launches(int64_t* count);

/* Failure-path self test (no paper counterpart): launches one CTA that waits
 * on an mbarrier nothing arrives on, with the same bounded wait (about 2 s of
 * clock cycles) as every mbarrier wait in the library's kernels.  When the
 * bound expires the CTA records CUTQC_ETIMEOUT in the device status word and
 * returns; the context stays usable.  waited_dev (device int32, nullable)
 * receives the cycles waited / 2^20.  Asynchronous on `stream`; read the
 * code with cutqc_device_status().  Nothing faults, traps or hangs.        */
int cutqc_selftest_wait_timeout(int32_t* waited_dev, void* stream);

/* ------------------------------------------------------------ attribution
 * Circuit Cutting section (Eq. 1 and the worked example: three measurement
 * and four initialisation variants per cut).  With the one-qubit identity
 * rho = 1/2 sum_M Tr(rho M) M:
 *   measured cut, outcome m:  I = sum_m pZ(m), Z = sum_m (-1)^m pZ(m),
 *                             X = sum_m (-1)^m pX(m), Y = sum_m (-1)^m pY(m)
 *   initialised cut:          I = p0 + p1, Z = p0 - p1,
 *                             X = 2 p+ - p0 - p1, Y = 2 p+i - p0 - p1
 * (the 1/2 per cut is applied by the reconstruction).
 *
 * variants_dev: [4^k_in][3^k_out][2^w] (F64 or F32), init digit j (state of
 *   the j-th init cut: 0 |0>, 1 |1>, 2 |+>, 3 |+i>) has weight 4^j, meas digit
 *   j (0 computational, 1 X basis, 2 Y basis) weight 3^j.
 * attributed_dev: [2^o][4^k] float32, o = w - k_out, k = k_in + k_out; row =
 *   output bits (t-th output qubit = bit t), column = sum_j d_j 4^j over the
 *   subcircuit's cut edges sorted by ascending edge id.
 * Workspace: cutqc_attribute_workspace_size bytes of device memory: 2^o *
 * 4^k * 4 bytes for a subcircuit with both initialised and measured cuts
 * (the measured side's float32 result), 0 bytes otherwise.
 * Errors: CUTQC_EINVAL on a bad descriptor, CUTQC_ENOMEM if ws_bytes is too
 * small, CUTQC_EUNSUPPORTED if k_in > 6 or k_out > 5.                      */
int cutqc_attribute_workspace_size(const cutqc_subcircuit* s, size_t* bytes);
int cutqc_attribute(const cutqc_subcircuit* s, const void* variants_dev, int variants_dtype,
                    float* attributed_dev, void* ws_dev, size_t ws_bytes, void* stream);

/* Attribution that allocates nothing (the paper has no counterpart).  For
 * callers that cannot allocate device memory during the call (a memory pool
 * owns the device, the host forbids cudaMalloc after set-up, or an
 * allocation's implicit synchronisation is not allowed): same inputs, outputs
 * and results as cutqc_attribute, but the scratch of the two-pass case comes
 * from a static 32 MiB device array of the library (held on every GPU that
 * loads it until the process exits).  The first call on a device that needs
 * scratch (a subcircuit with both initialised and measured cuts) looks up
 * that array's address with that device current; make it before any stream
 * capture.  Calls share the array and it keeps the last call's contents:
 * calls that can overlap on the GPU race and must be ordered by the caller.
 * Errors as cutqc_attribute, plus CUTQC_EUNSUPPORTED when the subcircuit
 * needs more than 32 MiB of scratch (cutqc_attribute_workspace_size).       */
int cutqc_attribute_noalloc(const cutqc_subcircuit* s, const void* variants_dev, int variants_dtype,
                            float* attributed_dev, void* stream);

/* --------------------------------------------------------- FD reconstruction
 * Eq. 1 with the 1/2-per-cut normalisation: P = 2^-K sum_e kron_i A_i[:, c_i(e)].
 * The subcircuits (n_sub >= 1, their attributed tensors as produced by
 * cutqc_attribute) are contracted pairwise in a greedy order (cheapest
 * contraction first); every cut edge must appear in exactly two of them.
 *
 * out_dev: float32 output in out_order (KRON or ORIGINAL).  Rows
 * [row_begin, row_end) of the final contraction are written, where a row is
 * one value of the high output bits (the operand that the final step puts in
 * the rows); row_end = -1 means all rows.  With a partial range the output
 * must be in KRON order and out_dev receives indices
 * [row_begin * cols, row_end * cols) (cols from cutqc_fd_shape) starting at
 * out_dev[0].  This is the offset/stride split used to shard one
 * reconstruction over several GPUs.
 * sum_dev: optional (nullable) float64 scalar += sum of the written outputs.
 * Workspace: cutqc_reconstruct_fd_workspace_size bytes.
 * Errors: CUTQC_EINVAL (descriptor, edge matching, sum of outputs > 34 bits,
 * order), CUTQC_ENOMEM (workspace), CUTQC_EUNSUPPORTED (limits),
 * CUTQC_ETIMEOUT is reported later through cutqc_device_status().         */
int cutqc_fd_shape(int n_sub, const cutqc_subcircuit* s, int64_t* rows, int64_t* cols);
/* Kernel timing (no paper counterpart): the next cutqc_reconstruct_fd made
 * by the calling thread records start_event just before its last
 * contraction's GEMM launch and stop_event just after it, on the stream that
 * launch uses (the caller's), then forgets both; cudaEventElapsedTime gives
 * that kernel's duration.  Events are cudaEvent_t (created with timing) owned
 * by the caller; null, null cancels.  Errors: CUTQC_EINVAL if only one event
 * is given.                                                                 */
int cutqc_fd_timing_events(void* start_event, void* stop_event);
/* Input readiness (no paper counterpart): the next cutqc_reconstruct_fd made
 * by the calling thread does not need its attributed tensors written when it
 * is issued.  Instead, every contraction step that reads subcircuit i's
 * tensor first makes its stream wait for events[i] (a cudaEvent_t the caller
 * records after the work that writes that tensor, on any stream of the same
 * device), so that steps over early inputs run while later ones are still
 * being attributed.  A null entry means that input is ready when the call is
 * issued.  n must equal that call's n_sub (else that call fails with
 * CUTQC_EINVAL).  The events are the caller's; the setting applies to one
 * call and is then cleared, and n = 0 clears it.  Errors: CUTQC_EINVAL for
 * n outside 0..4096 or a null array with n > 0.                            */
int cutqc_fd_input_events(int n, const void* const* events);
/* Launch shape of the tensor-core contraction on SM pairs (process-wide; no
 * paper counterpart): each pair takes work items of one 256-row block of the
 * row operand and up to this many consecutive 128-column tiles (0, the
 * default: chosen per launch to balance the pairs).  Results do not depend
 * on it, only the time and the order of the float64 total's additions.  For
 * autotuning.  Errors: CUTQC_EINVAL outside 0..4096.                       */
int cutqc_fd_set_tiles_per_item(int tiles_per_item);
int cutqc_reconstruct_fd_workspace_size(int n_sub, const cutqc_subcircuit* s, int precision,
                                        size_t* bytes);
int cutqc_reconstruct_fd(int n_sub, const cutqc_subcircuit* s, const float* const* attributed_dev,
                         int out_order, int precision, int64_t row_begin, int64_t row_end,
                         float* out_dev, double* sum_dev, void* ws_dev, size_t ws_bytes,
                         void* stream);

/* ------------------------------------------------------------------- DD
 * Algorithm 1 (Dynamic Definition).  A bin job fixes ("zooms") some qubits,
 * keeps up to M qubits active and merges the rest.  Because attribution is
 * linear and touches only cut qubits, merging is applied to each attributed
 * tensor: merged[a][c] = sum over the subcircuit's merged output bits of
 * attributed[x][c], over rows x whose zoomed bits equal the job's zoom bits;
 * a = the active output bits (in ascending output order).
 *
 * cutqc_dd_merge: one subcircuit, one job.  role (host, [o]): per output
 *   qubit 0 = active, 1 = merged, 2 = zoomed to 0, 3 = zoomed to 1.
 *   merged_dev: [2^a][4^k] float32.
 * cutqc_dd_merge_batch: one subcircuit, n_jobs jobs that share the
 *   active/merged split; zoom_dev (device, [n_jobs] uint64) holds per job the
 *   values of the zoomed output bits (bit t = value of output qubit t; other
 *   bits ignored), zoom_mask (host) marks which output bits are zoomed.  Job j
 *   writes merged_dev + j * 2^a * 4^k.  Reads only device data decided at run
 *   time, so it can sit in a captured CUDA graph.
 *
 * cutqc_dd_step: reconstructs the 2^(sum a_i) bins of each of n_jobs jobs
 * from their merged tensors (Eq. 1 at bin level: the FD contraction in FP32
 * arithmetic, the bin total accumulated in FP64), then selects the T largest
 * bins per job (ties to the lower bin index; T = 0 skips the selection).  Bin
 * bit order is given by bin_bit (host, [sum a_i], subcircuit-major): the bin
 * bit that each active row bit of each subcircuit takes; use bit j = j-th
 * active qubit in ascending uncut-circuit order for Algorithm 1's bins.
 *   merged_dev[i]   device, subcircuit i: n_jobs consecutive [2^a_i][4^k_i]
 *                   tensors (the layout cutqc_dd_merge_batch writes)
 *   bins_dev        device, n_jobs consecutive [2^(sum a_i)] float32 vectors
 *   bin_sum_dev     device [n_jobs] float64, set to each job's bin total
 *                   (nullable)
 *   top_idx_dev / top_val_dev   device [n_jobs][T] int32 / float32 (-1 / 0
 *                   where a job has fewer than T bins)
 * All jobs share the subcircuit descriptors, active counts and bin_bit (one
 * recursion level of one circuit).  The call enqueues a fixed sequence of
 * launches that reads only device data, so it can be captured in a CUDA graph.
 * Workspace: cutqc_dd_step_workspace_size bytes.  T <= 32, sum a_i <= 30.      */
int cutqc_dd_merge(const cutqc_subcircuit* s, const float* attributed_dev, const int8_t* role,
                   float* merged_dev, void* stream);
int cutqc_dd_merge_batch(const cutqc_subcircuit* s, const float* attributed_dev,
                         uint64_t active_mask, uint64_t zoom_mask, int n_jobs,
                         const uint64_t* zoom_dev, float* merged_dev, void* stream);
int cutqc_dd_step_workspace_size(int n_sub, const cutqc_subcircuit* s, const int32_t* active_bits,
                                 int n_jobs, size_t* bytes);
int cutqc_dd_step(int n_sub, const cutqc_subcircuit* s, const int32_t* active_bits,
                  const int32_t* bin_bit, int n_jobs, const float* const* merged_dev,
                  float* bins_dev, double* bin_sum_dev, int topk, int32_t* top_idx_dev,
                  float* top_val_dev, void* ws_dev, size_t ws_bytes, void* stream);

/* Algorithm 1 end to end.  Active qubits at depth d are the M lowest
 * unresolved ones, i.e. qubits [d*M, min(n, d*M + M)); the qubits below d*M
 * are zoomed to the bin being expanded; the rest are merged.
 *   strategy 0 (DFS, Algorithm 1 as written): each recursion reconstructs one
 *     bin job, appends its T largest bins that still have merged qubits to L,
 *     keeps the T largest of L (stable: earlier entries first among equal
 *     values) and pops the largest as the next job; stops after R recursions
 *     or when L is empty.
 *   strategy 1 (BFS): level by level; the next level expands the T largest
 *     bins (with merged qubits) over all jobs of the current level; at most R
 *     levels.  The jobs of one level run as one batch.
 * jobs (host, [max_jobs]) receives one record per job in execution order;
 * bins_dev receives each job's 2^n_active bins at jobs[j].bins_offset
 * (floats), bins_capacity floats in all.  BFS, and DFS with T <= 1 (the same
 * schedule), select on the device and synchronise `stream` once at the end;
 * DFS with T > 1 reads each recursion's selection on the host.  Limits:
 * n <= 128, M <= 30, T <= 32.  Workspace: cutqc_dd_run_workspace_size bytes. */
typedef struct cutqc_dd_job_result {
  int32_t level;            /* recursion (DFS) or level (BFS) index */
  int32_t depth;            /* qubits below depth * M are zoomed */
  int32_t parent;           /* job this one zooms into, -1 for the first */
  int32_t parent_bin;       /* bin of the parent it expands */
  int32_t n_active;
  int32_t active[32];       /* active qubits, ascending: bin bit j = active[j] */
  uint64_t zoom_mask[2];    /* qubit q fixed <=> bit q (q < 128) */
  uint64_t zoom_val[2];     /* its value */
  double bin_sum;           /* float64 total of the job's bins */
  int32_t top_idx[32];      /* T largest bins, -1 past the end */
  float top_val[32];
  int64_t bins_offset;      /* offset of the bins in bins_dev (floats) */
} cutqc_dd_job_result;

int cutqc_dd_run_workspace_size(int n_sub, const cutqc_subcircuit* s, int n_qubits, int M, int T,
                                size_t* bytes);
int cutqc_dd_run(int n_sub, const cutqc_subcircuit* s, const float* const* attributed_dev,
                 int n_qubits, int M, int R, int T, int strategy, int max_jobs,
                 cutqc_dd_job_result* jobs, int* n_jobs_out, float* bins_dev, int64_t bins_capacity,
                 void* ws_dev, size_t ws_bytes, void* stream);
/* Options of cutqc_dd_run_async (zero fields take defaults).  Launch shapes
 * (results agree within float32 rounding of the merge sums across settings):
 *   merge_ctas    about how many CTAs share one subcircuit's merge: the
 *                 merged index range is cut into slices of >= 64 indices
 *                 whose partial sums a second pass adds in a fixed order
 *                 (default 1024, at most 4096)
 *   topk_threads  threads per job of the top-T pass (default up to 1024)
 * Arithmetic of the bin reconstruction (Eq. 1 on the merged tensors):
 *   precision     CUTQC_PREC_FP32_SIMT (default) or CUTQC_PREC_FP16X3_TC,
 *                 the FD tensor-core path; levels whose jobs have fewer than
 *                 4 bins, or whose bins do not start 16-byte aligned, run
 *                 in FP32, and so does every contraction step with fewer
 *                 than 2^22 outputs over the level's jobs (FP32 on CUDA
 *                 cores is the faster and no less accurate choice there;
 *                 tc_min_outputs moves that floor).
 *                 Bin totals are float64 either way.
 * Jobs of more than 2^16 bins select their top T in two passes (chunks of
 * the bins, then the chunks' candidates), with the same order.  Jobs of at
 * least 2^22 bins whose last contraction step runs on SM pairs (tensor-core
 * path) or as FP32 outer products (a last step over at most 16 cut terms,
 * any precision) take it from block maxima instead: that step also writes
 * the largest value of each 32 x 64 block of its output, and only the
 * blocks whose maximum reaches the T-th largest block maximum are read
 * again (every bin among the T largest lies in one of them); a job where
 * more than 32 blocks reach it takes the two-pass scan.  The result is the
 * same.                                                                     */
typedef struct cutqc_dd_options {
  int32_t merge_ctas;
  int32_t topk_threads;
  int32_t precision;
  int32_t tc_min_outputs;   /* 0: steps below 2^22 outputs run in FP32; b > 0: the
                               floor is 2^(b-1) outputs (1: every step on the
                               split path) */
} cutqc_dd_options;

/* Algorithm 1, level by level (strategy 1 above; with T = 1 also the depth
 * first order), enqueued without any host synchronisation or host copy, so
 * that it can be captured in a CUDA graph and replayed: level 0 has one job,
 * every later level T jobs (the T largest bins of the previous level, chosen
 * on the device); at most min(R, ceil(n / M)) levels (one when T = 0).
 *   jobs_dev    device [max_jobs] records, written in level order; a record
 *               with level < 0 is a placeholder (fewer than T bins to expand)
 *   n_jobs_dev  device int32, set to the number of records written
 * The bins of record r are at bins_dev + jobs_dev[r].bins_offset.  opt
 * (host, nullable) chooses launch shapes.  Host arguments are read during the
 * call only.  Errors as cutqc_dd_run; workspace: cutqc_dd_run_workspace_size
 * bytes (enough for any options).                                            */
int cutqc_dd_run_async(int n_sub, const cutqc_subcircuit* s, const float* const* attributed_dev,
                       int n_qubits, int M, int R, int T, int max_jobs, cutqc_dd_job_result* jobs_dev,
                       int32_t* n_jobs_dev, float* bins_dev, int64_t bins_capacity,
                       const cutqc_dd_options* opt, void* ws_dev, size_t ws_bytes, void* stream);

/* Algorithm 1 (breadth first, as cutqc_dd_run_async) for several circuits in
 * ONE persistent launch.  The recursion levels of Algorithm 1 (its merge
 * steps, the bin reconstruction of Eq. 1 on the merged tensors, and the
 * choice of the bins to expand) are small for each circuit (2^M bins per
 * job); here every step of every circuit is one phase of a program that a
 * single cooperative launch walks, with a grid-wide barrier between phases
 * and the circuits sharing each phase.  Results per run are those of
 * cutqc_dd_run_async with FP32 reconstruction and the same merge_ctas: the
 * same job records (bin totals within float64 rounding of their atomic sum),
 * bins and top-T selections.
 * One run description per circuit:
 *   n_sub, subcircuits (host [n_sub]), attributed_dev (host array of n_sub
 *   device pointers), n_qubits, M, R, T: as cutqc_dd_run_async (n_sub >= 2)
 *   jobs_dev, n_jobs_dev, bins_dev, bins_capacity, max_jobs: that run's
 *   outputs, as cutqc_dd_run_async.
 * Options (zero fields take defaults): merge_ctas as cutqc_dd_options;
 * topk_chunk bins per task of the chunked top-T phase (a power of two >=
 * 256, default 2048); ctas caps the grid (default: every CTA that fits at
 * once);
 * ctas_per_sm (2..4, default 3) the CTAs per SM that the kernel's registers
 * are budgeted for (more resident warps, fewer registers each); narrow_max_n
 * the tile shape of the contraction steps (below).
 * cutqc_dd_batch_create validates the runs, lays out `ws_dev` (at least
 * cutqc_dd_batch_workspace_size bytes, 256-byte aligned, owned by the caller
 * and kept alive and untouched while the handle is used) and writes the
 * program into it with a synchronous copy: call it outside stream capture.
 * The run descriptions are read during the call only; the device pointers in
 * them are baked into the program.  cutqc_dd_batch_launch enqueues one
 * memset and one cooperative launch on `stream` (capturable in a CUDA graph);
 * launches on one handle must not overlap.  A barrier wait that runs out
 * (about 2 s) records CUTQC_ETIMEOUT in the device status word
 * (cutqc_device_status) and ends the launch.  Errors: CUTQC_EINVAL (bad
 * descriptions or options), CUTQC_EUNSUPPORTED (one subcircuit, more than 32
 * outputs in a subcircuit, limits of cutqc_dd_run), CUTQC_ENOMEM (records,
 * bins or workspace too small).                                             */
typedef struct cutqc_dd_run_desc {
  int32_t n_sub;
  const cutqc_subcircuit* subcircuits;
  const float* const* attributed_dev;
  int32_t n_qubits, M, R, T;
  int32_t max_jobs;
  cutqc_dd_job_result* jobs_dev;
  int32_t* n_jobs_dev;
  float* bins_dev;
  int64_t bins_capacity;
} cutqc_dd_run_desc;

typedef struct cutqc_dd_batch_options {
  int32_t merge_ctas;
  int32_t topk_chunk;
  int32_t ctas;
  int32_t ctas_per_sm;
  int32_t narrow_max_n;   /* GEMM tiles of the bin reconstruction: contraction
                             steps of at most this many columns take 256 x 16
                             tiles, the others 64 x 64 (16, 32 or 64; 0:
                             default 16; -1: never 256 x 16).  Results are the
                             same for every setting (each bin is the same
                             fmaf chain over k).                          */
} cutqc_dd_batch_options;

typedef struct cutqc_dd_batch cutqc_dd_batch;

int cutqc_dd_batch_workspace_size(int n_runs, const cutqc_dd_run_desc* runs,
                                  const cutqc_dd_batch_options* opt, size_t* bytes);
/* The program's shape without building it on a device (host only: no device
 * pointer is read): phases, ops and tasks summed over the phases (the merge
 * tasks depend on the current device's SM count).                           */
int cutqc_dd_batch_shape(int n_runs, const cutqc_dd_run_desc* runs, const cutqc_dd_batch_options* opt,
                         int32_t* n_phases, int32_t* n_ops, int64_t* tasks);
int cutqc_dd_batch_create(int n_runs, const cutqc_dd_run_desc* runs, const cutqc_dd_batch_options* opt,
                          void* ws_dev, size_t ws_bytes, cutqc_dd_batch** out);
int cutqc_dd_batch_launch(const cutqc_dd_batch* batch, void* stream);
/* Shape of the program: phases (grid barriers + 1), ops, CTAs launched.     */
int cutqc_dd_batch_info(const cutqc_dd_batch* batch, int32_t* n_phases, int32_t* n_ops, int32_t* grid_ctas);
/* Per phase p < n (n = the number of phases): kinds[p] has bit t set when an
 * op of kind t runs in it (0 zero bin totals, 1 merge, 2 slice reduction,
 * 3 contraction step, 4 chunked top-T, 5 level selection), tasks[p] its
 * tasks, fma[p] the multiply-adds of its contraction steps (M * N * K per
 * job), cycles[p] the SM clock cycles CTA 0 saw it take in the last
 * completed launch (a synchronous copy).  Any output may be null.           */
int cutqc_dd_batch_phases(const cutqc_dd_batch* batch, int32_t* kinds, int32_t* tasks, int64_t* fma,
                          int64_t* cycles, int n);
int cutqc_dd_batch_destroy(cutqc_dd_batch* batch);

/* ------------------------------------------------------------- reductions
 * sum_dev (device float64 scalar) += sum of x_dev[0..n) in float64.          */
int cutqc_sum_f64(const float* x_dev, int64_t n, double* sum_dev, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* CUTQC_H */
