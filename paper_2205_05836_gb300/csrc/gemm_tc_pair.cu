// Tensor-core contraction for Eq. 1 on pairs of SMs (tcgen05 cta_group::2).
//
// Same products as tc_gemm_kernel (FP16 hi/lo split operands, three
// products, power-of-two row / operand scales), for K <= 256 (four 64-wide
// k-blocks).  Each 128 values of k accumulate in a fresh TMEM accumulator
// ("chunk", 24 MMAs), cross products (hi x lo, lo x hi) first and hi x hi
// last: the tensor core rounds its FP32 accumulator toward zero, and only
// the last MMAs of a chunk do so at the chunk's full magnitude.  Chunks are
// added in registers with round-to-nearest.  (Modelled on the 30-qubit
// workload, this order with 128-wide chunks leaves a third of the bias of
// 64-wide chunks in product order: sum p error -3.6e-7 against -5.4e-7.)
// The kernel is organised to move fewer operand bytes per output:
//
// * a cluster of two CTAs on two SMs computes 256 x 128 output tiles with
//   one MMA stream (M = 256, N = 128, K = 16 per instruction): CTA r holds
//   A rows r*128 .. +127 and B rows r*64 .. +63 of the tile, the tensor core
//   reads both halves of B from both shared memories, and each CTA's tensor
//   memory receives its own 128 rows x 128 columns;
// * A stays resident: a pair takes a work item (one 256-row block of A and a
//   run of consecutive 128-column tiles) and keeps the CTA's A rows for all
//   k: A hi in tensor memory (written by the epilogue warps, read by two of
//   the three products), A lo in shared memory (one TMA load per item).
//   Only B streams (16 KiB per CTA per k-block, 5 stages), so a CTA moves 1
//   byte of operands per byte of output (4 for a 128 x 128 tile that streams
//   both operands).
// * one thread cannot issue N = 128 pair MMAs as fast as the tensor core
//   runs them, so two threads issue alternate chunks;
// * three 128-column accumulator buffers let the MMAs run two chunks (256
//   values of k) ahead of the epilogue.
//
// Tensor memory per CTA (512 columns): A hi [0, 128) (two fp16 values of k
// per 32-bit column), chunk accumulators at 128, 256, 384.
//
// Roles (both CTAs): warp 8 lane 0 loads B per k-block; lane 0 of warps 9
// and 10 of CTA 0 issue the MMAs (alternate chunks); warps 0-7 write A hi to
// tensor memory and load A lo at the start of an item, then drain the
// chunks, scale and store their CTA's rows.  Row-major outputs (out[m * N +
// n]) go straight from registers (16 x 256-bit tensor-memory loads give each
// quad of lanes 8 consecutive columns of a row: whole 32-byte sectors per
// store) -- staging them through shared memory would add 128 KiB of shared
// memory traffic per tile on top of the MMAs' operand reads and the B
// stream, more than the SM's shared memory bandwidth allows at the tensor
// rate.  Other bit-deposit layouts go through a staged transpose.  The loads of both CTAs complete on CTA 0's
// barriers (it waits for both halves); MMA completion is multicast to the
// barriers of both CTAs; epilogue warps of both CTAs report A written and
// chunk buffers read on CTA 0's barriers.  Every wait is bounded; on expiry
// a CTA records CUTQC_ETIMEOUT, raises its abort flag and falls through to
// the common exit (a cluster barrier, then tensor memory is freed).
#include "internal.cuh"
#include "contract.cuh"
#include "tc_ptx.cuh"

#include <algorithm>
#include <atomic>
#include <mutex>
#include <set>

namespace cutqc {

namespace {

using namespace tc;

constexpr int BM = 128;                                  // A rows per CTA (256 per pair)
constexpr int BN = 128;                                  // output columns per tile
constexpr int BNH = BN / 2;                              // B rows per CTA
constexpr int BK = 64;                                   // k per block (128-byte rows)
constexpr int MAX_KB = 4;                                // resident A: k <= 256
constexpr int STAGES_MAX = 10;
constexpr int NBUF = 3;                                  // chunk buffers in TMEM
constexpr int KB_PER_CHUNK = 2;                          // 128 values of k per accumulator
constexpr int A_COLS = MAX_KB * BK / 2;                  // 128 TMEM columns of A hi
constexpr int ACC_COL0 = A_COLS;                         // first accumulator column
constexpr int A_KB_BYTES = BM * BK * 2;                  // 16 KiB: A lo, one k-block
constexpr int ALO_BYTES = MAX_KB * A_KB_BYTES;           // 64 KiB
constexpr int B_HALF = BNH * BK * 2;                     // 8 KiB
constexpr int STAGE_BYTES = 2 * B_HALF;                  // 16 KiB: B hi + lo, one k-block
constexpr int TMEM_COLS = 512;
static_assert(ACC_COL0 + NBUF * BN <= TMEM_COLS, "tensor memory budget");
constexpr int NUM_THREADS = 352;
constexpr int EPI_WARPS = 8;
constexpr int EPI_COLS = 64;                             // columns per epilogue warp
constexpr int kStatBlockMax = 1, kStatAbsMax = 2;        // epilogue statistics (tc_pair_gemm_kernel)
constexpr int BLK_FLOATS = 32 * 32;                      // one 32 x 32 staging block
constexpr int EPI_STG_BYTES = EPI_WARPS * (EPI_COLS / 32) * BLK_FLOATS * 4;   // 64 KiB
// Direct stores need no staging block: its 64 KiB go to five more B stages,
// which keeps the B stream ahead of the MMAs while the output stream loads
// the memory system (4.27 -> 4.05 ms on the 32-qubit chain's last step).
template <bool kDirect> struct Cfg {
  static constexpr int STAGES = kDirect ? 10 : 5;
  static constexpr int STG = kDirect ? 0 : EPI_STG_BYTES;
};

struct PairMaps {
  CUtensorMap a_lo;         // [rows][Kp] fp16, box 64 x 128
  CUtensorMap b_hi, b_lo;   // [rows][Kp] fp16, box 64 x 64
};

struct PairArgs {
  const __half* a_hi;   // [M][Kp]
  int64_t Kp;
  const float* sa;
  const float* sb;
  int64_t M, N;
  int num_kb;
  const int* num_kb_dev;  // nullable: k-blocks in use, read on the device (<= num_kb)
  int num_mp;           // 256-row blocks of A
  int64_t num_nt;       // 128-column tiles
  int64_t tiles_per_item;
  int64_t num_items;
  float alpha;
  uint64_t mask_m, mask_n;
  int n_contig;
  int m_shift;
  int m_low5;           // mask_m holds address bits 0..4 (rows 32-aligned are consecutive)
  uint64_t coff_lo[64]; // pdep(c, mask_n) for c < 64: column offsets inside a 64-aligned group
  float* out;
  double* sum;
  float* cmax;          // nullable: largest value of each 32-row x 64-column block of the output
  unsigned int* amax;   // nullable: largest |output| of the launch (float bits, atomicMax)
  int64_t cmax_cols;    // blocks per 32-row stripe: ceil(N / 64)
  int streaming;
  int* status;
};

struct Tail {
  uint64_t full[STAGES_MAX];     // CTA 0: both CTAs' B halves of a stage landed
  uint64_t empty[STAGES_MAX];    // each CTA: its stage may be refilled
  uint64_t cfull[NBUF];      // each CTA: chunk buffer holds a finished chunk
  uint64_t cempty[NBUF];     // CTA 0: both CTAs' epilogues read the buffer
  uint64_t afull;            // CTA 0: both CTAs wrote A hi to TMEM and their A lo landed
  uint64_t aempty;           // each CTA: both issuers are done with A
  uint64_t fin[2];           // CTA 0: every MMA of issuer j finished
  uint32_t tmem_slot;
  int abort_flag;
};

template <bool kDirect>
constexpr size_t smem_bytes() {
  return 1024 + ALO_BYTES + Cfg<kDirect>::STAGES * STAGE_BYTES + Cfg<kDirect>::STG + sizeof(Tail);
}
static_assert(smem_bytes<true>() <= 232448 && smem_bytes<false>() <= 232448, "shared memory budget");

// kind::f16, A = B = F16, D = F32, both K-major, N = 128, M = 256.
constexpr uint32_t kIdescPair = (1u << 4) | ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(256 >> 4) << 24);

__device__ __forceinline__ uint32_t cta_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
// address of the same shared variable in CTA `rank` of the cluster
__device__ __forceinline__ uint32_t map_to_rank(uint32_t saddr, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(saddr), "r"(rank));
  return r;
}
__device__ __forceinline__ void cluster_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
  asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// Arrive on a barrier of another CTA of the cluster.  Default (CTA-scope
// release) semantics: the only thing published is that this warp's tensor
// memory reads finished, which tcgen05.wait::ld and the tcgen05 fence before
// it already order; a cluster-scope release would add a full memory fence
// per chunk.
__device__ __forceinline__ void remote_arrive(uint32_t cluster_bar) {
  asm volatile("mbarrier.arrive.shared::cluster.b64 _, [%0];" ::"r"(cluster_bar) : "memory");
}
// TMA load into this CTA's shared memory, completing on an mbarrier that may
// sit in the peer CTA (a shared::cluster address)
__device__ __forceinline__ void tma_load_pair(uint32_t dst, const CUtensorMap* map, int c0, int c1,
                                              uint32_t cluster_bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.cta_group::2.shared::cluster.global.mbarrier::complete_tx::bytes "
      "[%0], [%1, {%2, %3}], [%4];"
      ::"r"(dst), "l"((uint64_t)map), "r"(c0), "r"(c1), "r"(cluster_bar)
      : "memory");
}
// D (TMEM) (+)= A (shared memory, both CTAs' rows) x B (shared memory, both CTAs' halves)
__device__ __forceinline__ void umma_pair_ss(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t accum) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n\t}\n"
      ::"r"(d_tmem), "l"(adesc), "l"(bdesc), "r"(kIdescPair), "r"(accum)
      : "memory");
}
// D (TMEM) (+)= A (TMEM, both CTAs' rows) x B (shared memory, both CTAs' halves)
__device__ __forceinline__ void umma_pair_ts(uint32_t d_tmem, uint32_t a_tmem, uint64_t bdesc, uint32_t accum) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::2.kind::f16 [%0], [%1], %2, %3, p;\n\t}\n"
      ::"r"(d_tmem), "r"(a_tmem), "l"(bdesc), "r"(kIdescPair), "r"(accum)
      : "memory");
}
// 32 lanes x 32 columns of 32 bits from registers (lane = thread)
__device__ __forceinline__ void tmem_st32(uint32_t taddr, const uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], "
      "{%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,"
      "%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32};"
      ::"r"(taddr), "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]),
        "r"(r[8]), "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15]),
        "r"(r[16]), "r"(r[17]), "r"(r[18]), "r"(r[19]), "r"(r[20]), "r"(r[21]), "r"(r[22]), "r"(r[23]),
        "r"(r[24]), "r"(r[25]), "r"(r[26]), "r"(r[27]), "r"(r[28]), "r"(r[29]), "r"(r[30]), "r"(r[31])
      : "memory");
}
// 16 lanes x 256 bits, repeated 8 times along the columns: thread t gets
// r[4 q + e] = (lane t / 4 + 8 (e / 2), column 8 q + 2 (t % 4) + e % 2)
__device__ __forceinline__ void tmem_ld16x256_x8(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.16x256b.x8.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
        "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
        "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
        "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
}
// Arrive on CTA 0's barrier after writing tensor memory that CTA 0's MMAs
// read: cluster-scope release (once per work item).
__device__ __forceinline__ void remote_arrive_release_cluster(uint32_t cluster_bar) {
  asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(cluster_bar) : "memory");
}
// arrive (once) on the barrier at this offset in every CTA of `mask` when
// all tcgen05 operations issued so far by this thread have completed
__device__ __forceinline__ void umma_commit_mc(uint32_t bar, uint16_t mask) {
  asm volatile(
      "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;"
      ::"r"(bar), "h"(mask)
      : "memory");
}

// kStat: 0 nothing more; kStatBlockMax: each epilogue warp's 32 x 64 block
// maximum per tile into args.cmax; kStatAbsMax: the largest |output| of the
// launch into *args.amax (float bits; the values are non-negative, so the
// integer max orders them).
template <bool kRowMajor, int kStat>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(NUM_THREADS, 1)
tc_pair_gemm_kernel(const __grid_constant__ PairMaps maps, const PairArgs args) {
  constexpr int STAGES = Cfg<kRowMajor>::STAGES;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  uint8_t* alo_smem = smem;
  uint8_t* b_smem = smem + ALO_BYTES;
  float* stg_all = reinterpret_cast<float*>(smem + ALO_BYTES + STAGES * STAGE_BYTES);
  Tail* tail = reinterpret_cast<Tail*>(smem + ALO_BYTES + STAGES * STAGE_BYTES + Cfg<kRowMajor>::STG);
  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  // k-blocks in use: a count chosen on the device (cut-term pruning) when
  // given, never more than the operands hold
  const int num_kb = args.num_kb_dev ? max(1, min(args.num_kb, __ldg(args.num_kb_dev))) : args.num_kb;
  const uint32_t rank = cta_rank();
  const int64_t pair = blockIdx.x >> 1;
  const int64_t num_pairs = gridDim.x >> 1;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(smem_u32(&tail->full[s]), 1);
      mbar_init(smem_u32(&tail->empty[s]), 1);
    }
    for (int b = 0; b < NBUF; ++b) {
      mbar_init(smem_u32(&tail->cfull[b]), 1);
      mbar_init(smem_u32(&tail->cempty[b]), 2 * EPI_WARPS);
    }
    mbar_init(smem_u32(&tail->afull), 2 * EPI_WARPS);
    mbar_init(smem_u32(&tail->aempty), 2);
    mbar_init(smem_u32(&tail->fin[0]), 1);
    mbar_init(smem_u32(&tail->fin[1]), 1);
    tail->abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    // one warp of each CTA of the pair allocates, collectively
    asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tail->tmem_slot)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  cluster_sync();           // both CTAs' barriers are initialised before any remote use
  tc_fence_after();
  const uint32_t tmem_base = tail->tmem_slot;
  volatile int* abort_flag = &tail->abort_flag;
  auto fail = [&]() {
    *abort_flag = 1;
    record_status(args.status, CUTQC_ETIMEOUT);
  };

  if (warp == 8) {
    // ------------------------------------------------------------ producer
    if (lane == 0) {
      bool issued[STAGES] = {};
      uint32_t issued_par[STAGES] = {};
      int stage = 0;
      uint32_t phase = 0;
      bool ok = true;
      for (int64_t item = pair; item < args.num_items && ok && !*abort_flag; item += num_pairs) {
        const int64_t t0 = (item / args.num_mp) * args.tiles_per_item;
        const int64_t t1 = t0 + args.tiles_per_item < args.num_nt ? t0 + args.tiles_per_item : args.num_nt;
        for (int64_t nt = t0; nt < t1 && ok; ++nt) {
          int brow = (int)(nt * BN) + (int)rank * BNH;
          if (brow >= args.N) brow = 0;     // columns beyond N are never stored
          for (int kb = 0; kb < num_kb; ++kb) {
            if (!mbar_wait(smem_u32(&tail->empty[stage]), phase ^ 1u, abort_flag)) { fail(); ok = false; break; }
            uint8_t* st = b_smem + stage * STAGE_BYTES;
            const uint32_t lead_full = map_to_rank(smem_u32(&tail->full[stage]), 0);
            if (rank == 0) mbar_expect_tx(smem_u32(&tail->full[stage]), 2 * STAGE_BYTES);
            tma_load_pair(smem_u32(st), &maps.b_hi, kb * BK, brow, lead_full);
            tma_load_pair(smem_u32(st + B_HALF), &maps.b_lo, kb * BK, brow, lead_full);
            issued[stage] = true;
            issued_par[stage] = phase;
            if (++stage == STAGES) { stage = 0; phase ^= 1u; }
          }
        }
      }
      // Every copy this CTA started completes on CTA 0's barriers, which
      // this thread cannot wait on; wait instead until the MMAs that read
      // them have finished (each stage's last use) before exiting.
      for (int s = 0; s < STAGES; ++s)
        if (issued[s] && !mbar_wait(smem_u32(&tail->empty[s]), issued_par[s], nullptr))
          record_status(args.status, CUTQC_ETIMEOUT);
    }
  } else if (warp == 9 || warp == 10) {
    // ----------------------------------------------------------- MMA issue
    // Two issuing threads: chunk c (KB_PER_CHUNK k-blocks of one tile,
    // counted over the whole kernel) is issued by thread c % 2 into
    // accumulator buffer c % NBUF; k-block g (counted over the whole kernel)
    // sits in stage g % STAGES.  Within a chunk the hi x lo and lo x hi
    // products go first and the hi x hi products last, so that only the
    // last MMAs truncate (round toward zero) at the chunk's full magnitude.
    const int j = warp - 9;
    if (lane == 0 && rank == 0) {
      uint32_t aphase = 0;
      int64_t c = 0, g = 0;
      bool ok = true;
      for (int64_t item = pair; item < args.num_items && ok && !*abort_flag; item += num_pairs) {
        const int64_t t0 = (item / args.num_mp) * args.tiles_per_item;
        const int64_t t1 = t0 + args.tiles_per_item < args.num_nt ? t0 + args.tiles_per_item : args.num_nt;
        if (!mbar_wait(smem_u32(&tail->afull), aphase, abort_flag)) { fail(); ok = false; break; }
        aphase ^= 1u;
        tc_fence_after();
        for (int64_t nt = t0; nt < t1 && ok; ++nt) {
          for (int kb0 = 0; kb0 < num_kb; kb0 += KB_PER_CHUNK, ++c) {
            const int nkb = num_kb - kb0 < KB_PER_CHUNK ? num_kb - kb0 : KB_PER_CHUNK;
            if ((int)(c & 1) != j) { g += nkb; continue; }
            const int buf = (int)(c % NBUF);
            const uint32_t buf_phase = (uint32_t)((c / NBUF) & 1);
            if (!mbar_wait(smem_u32(&tail->cempty[buf]), buf_phase ^ 1u, abort_flag)) { fail(); ok = false; break; }
            tc_fence_after();
            int stage[KB_PER_CHUNK];
            for (int q = 0; q < nkb && ok; ++q) {
              stage[q] = (int)((g + q) % STAGES);
              const uint32_t phase = (uint32_t)(((g + q) / STAGES) & 1);
              if (!mbar_wait(smem_u32(&tail->full[stage[q]]), phase, abort_flag)) { fail(); ok = false; }
            }
            if (!ok) break;
            tc_fence_after();
            const uint32_t d = tmem_base + (uint32_t)(ACC_COL0 + buf * BN);
            uint32_t accum = 0;
            for (int pass = 0; pass < 2; ++pass) {        // 0: cross products, 1: hi x hi
              for (int q = 0; q < nkb; ++q) {
                const int kb = kb0 + q;
                const uint32_t ah = tmem_base + (uint32_t)(kb * (BK / 2));
                const uint32_t al = smem_u32(alo_smem + kb * A_KB_BYTES);
                const uint32_t bh = smem_u32(b_smem + stage[q] * STAGE_BYTES), bl = bh + B_HALF;
#pragma unroll
                for (int kk = 0; kk < BK / 16; ++kk) {
                  // 16 values of k: 8 TMEM columns of A hi, 32 bytes inside the
                  // swizzle rows of A lo and B
                  const uint32_t ta = kk * 8, off = kk * 32;
                  const uint64_t dbh = sw128_desc(bh + off);
                  if (pass == 0) {
                    umma_pair_ts(d, ah + ta, sw128_desc(bl + off), accum);
                    umma_pair_ss(d, sw128_desc(al + off), dbh, 1u);
                    accum = 1u;
                  } else {
                    umma_pair_ts(d, ah + ta, dbh, 1u);
                  }
                }
              }
            }
            for (int q = 0; q < nkb; ++q) umma_commit_mc(smem_u32(&tail->empty[stage[q]]), 0x3);
            umma_commit_mc(smem_u32(&tail->cfull[buf]), 0x3);
            g += nkb;
          }
        }
        if (ok) umma_commit_mc(smem_u32(&tail->aempty), 0x3);   // this issuer is done with A
      }
      // all MMAs this thread issued complete before tensor memory is freed
      umma_commit_mc(smem_u32(&tail->fin[j]), 0x1);
      if (!mbar_wait(smem_u32(&tail->fin[j]), 0, nullptr)) record_status(args.status, CUTQC_ETIMEOUT);
    }
  } else {
    // ------------------------------------------------------------ epilogue
    // warp w: TMEM lanes 32*(w%4).. = tile rows, columns 64*(w/4) .. +63
    // At the start of an item, warp w also writes A hi rows 32*(w%4) .. +31
    // of the CTA's block, k-blocks kb with kb % 2 == w / 4, to tensor memory;
    // warp 0 lane 0 loads the CTA's A lo rows by TMA.
    const int g = warp & 3, h = warp >> 2;
    int buf = 0;
    uint32_t buf_phase = 0;
    uint32_t aphase = 0;
    double local = 0.0;
    [[maybe_unused]] float amx = 0.f;    // kStatAbsMax: this thread's largest |output|
    const float sbg = __ldg(args.sb);
    float* stg0 = stg_all + warp * (EPI_COLS / 32) * BLK_FLOATS;
    const uint32_t lead_afull = map_to_rank(smem_u32(&tail->afull), 0);
    float tot[EPI_COLS];
    bool ok = true;
    static_assert(EPI_COLS == 64, "block maxima cover one warp's 32 rows x 64 columns");
    // the warp's block of a tile (rows row0 .. +31, columns col0 .. +63):
    // its largest value, for the top-T selection of the caller
    auto put_cmax = [&](float mx, int64_t row0, int64_t col0) {
      for (int off = 16; off; off >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, off));
      if (lane == 0 && row0 < args.M && col0 < args.N) args.cmax[(row0 >> 5) * args.cmax_cols + (col0 >> 6)] = mx;
    };
    for (int64_t item = pair; item < args.num_items && ok && !*abort_flag; item += num_pairs) {
      const int mp = (int)(item % args.num_mp);
      const int64_t t0 = (item / args.num_mp) * args.tiles_per_item;
      const int64_t t1 = t0 + args.tiles_per_item < args.num_nt ? t0 + args.tiles_per_item : args.num_nt;
      const int64_t mrow0 = (int64_t)mp * 2 * BM + (int64_t)rank * BM + g * 32;
      const int64_t m = mrow0 + lane;
      const bool mvalid = m < args.M;
      // direct-store layout: this thread's rows mrow0 + lane/4 + 16 h2 + 8 rsel,
      // each with its scale and its output offset (the row bits deposited)
      const int64_t rtile0 = mrow0 + (lane >> 2);
      float rsv[4];
      int64_t rowoff[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int64_t mm = rtile0 + 16 * (i >> 1) + 8 * (i & 1);
        const bool v = kRowMajor && mm < args.M;
        rsv[i] = v ? args.alpha * __ldg(args.sa + mm) * sbg : 0.f;
        rowoff[i] = !v ? 0 : args.m_shift >= 0 ? (mm << args.m_shift) : (int64_t)pdep64((uint64_t)mm, args.mask_m);
      }
      // ---- A rows of this item into tensor memory, once the previous
      // item's MMAs are done with the old ones
      if (!mbar_wait(smem_u32(&tail->aempty), aphase ^ 1u, abort_flag)) { fail(); ok = false; break; }
      aphase ^= 1u;
      tc_fence_after();
      if (warp == 0 && lane == 0) {
        // A lo rows of this CTA (CTA 1's rows may lie wholly beyond M: it then
        // loads rows from 0, which are never stored)
        int arow = mp * 2 * BM + (int)rank * BM;
        if (arow >= args.M) arow = 0;
        for (int kb = 0; kb < num_kb; ++kb)
          tma_load_pair(smem_u32(alo_smem + kb * A_KB_BYTES), &maps.a_lo, kb * BK, arow, lead_afull);
      }
      {
        const uint4* row = reinterpret_cast<const uint4*>(args.a_hi + (mvalid ? m : 0) * args.Kp);
        const uint32_t tbase = tmem_base + ((uint32_t)(g * 32) << 16);
        for (int kb = h; kb < num_kb; kb += 2) {
          uint32_t r[32];
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            uint4 v = mvalid ? __ldg(row + kb * 8 + q) : make_uint4(0, 0, 0, 0);
            r[4 * q] = v.x;
            r[4 * q + 1] = v.y;
            r[4 * q + 2] = v.z;
            r[4 * q + 3] = v.w;
          }
          tmem_st32(tbase + (uint32_t)(kb * (BK / 2)), r);
        }
        asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) {
        // CTA 0's warp 0 arrives with the byte count of both CTAs' A lo loads
        if (rank == 0 && warp == 0)
          mbar_expect_tx(smem_u32(&tail->afull), (uint32_t)(2 * num_kb * A_KB_BYTES));
        else
          remote_arrive_release_cluster(lead_afull);
      }
      for (int64_t nt = t0; nt < t1 && ok; ++nt) {
#pragma unroll
        for (int i = 0; i < EPI_COLS; ++i) tot[i] = 0.f;
        for (int ch = 0; ch < (num_kb + KB_PER_CHUNK - 1) / KB_PER_CHUNK; ++ch) {
          if (!mbar_wait(smem_u32(&tail->cfull[buf]), buf_phase, abort_flag)) { fail(); ok = false; break; }
          tc_fence_after();
          __syncwarp();
          uint32_t r0[32], r1[32];
          const uint32_t taddr =
              tmem_base + ((uint32_t)(g * 32) << 16) + (uint32_t)(ACC_COL0 + buf * BN + h * EPI_COLS);
          if constexpr (kRowMajor) {
            // two 16-lane halves, 64 columns each: tot[32 h2 + 4 q + e] is
            // row g*32 + 16 h2 + lane/4 + 8 (e/2), column 8 q + 2 (lane%4) + e%2
            tmem_ld16x256_x8(taddr, r0);
            tmem_ld16x256_x8(taddr + (16u << 16), r1);
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
          } else {
            // thread = row: tot[i] is row g*32 + lane, column i
            tmem_ld32(taddr, r0);
            tmem_ld32(taddr + 32, r1);
          }
#pragma unroll
          for (int i = 0; i < 32; ++i) {
            tot[i] += __uint_as_float(r0[i]);
            tot[32 + i] += __uint_as_float(r1[i]);
          }
          tc_fence_before();
          __syncwarp();
          if (lane == 0) remote_arrive(map_to_rank(smem_u32(&tail->cempty[buf]), 0));
          if (++buf == NBUF) { buf = 0; buf_phase ^= 1u; }
        }
        if (!ok) break;
        const float rs = mvalid ? args.alpha * __ldg(args.sa + m) * sbg : 0.f;
        const int64_t nbase = nt * BN + h * EPI_COLS;
        if (kRowMajor) {
          // straight from registers: the column bits 0..5 are address bits
          // 0..5, so the warp's 64 columns of a row are 64 consecutive floats
          // at pdep(row) + pdep(nbase); per instruction the warp writes 8 rows
          // x 32 bytes (4 lanes per row), whole sectors; no staging through
          // shared memory, whose bandwidth the MMAs' operand reads and the B
          // stream already use
          const int64_t nb0 = nbase + 2 * (lane & 3);
          const int64_t cb = (args.n_contig ? nbase : (int64_t)pdep64((uint64_t)nbase, args.mask_n)) + 2 * (lane & 3);
          float part = 0.f;     // this thread's 64 outputs of the tile; float64 across tiles
          [[maybe_unused]] float mx = -INFINITY;
#pragma unroll
          for (int h2 = 0; h2 < 2; ++h2)
#pragma unroll
            for (int rsel = 0; rsel < 2; ++rsel) {
              const int64_t mm = rtile0 + 16 * h2 + 8 * rsel;
              const float rsm = rsv[2 * h2 + rsel];
              float* orow = args.out + rowoff[2 * h2 + rsel] + cb;
#pragma unroll
              for (int q = 0; q < EPI_COLS / 8; ++q) {
                const float a = tot[32 * h2 + 4 * q + 2 * rsel] * rsm, b = tot[32 * h2 + 4 * q + 2 * rsel + 1] * rsm;
                if (mm < args.M && nb0 + 8 * q < args.N) {
                  __stcs(reinterpret_cast<float2*>(orow + 8 * q), make_float2(a, b));
                  part += a + b;
                  if constexpr (kStat == kStatBlockMax) mx = fmaxf(mx, fmaxf(a, b));
                  if constexpr (kStat == kStatAbsMax) amx = fmaxf(amx, fmaxf(fabsf(a), fabsf(b)));
                }
              }
            }
          if (args.sum) local += (double)part;
          if constexpr (kStat == kStatBlockMax) put_cmax(mx, mrow0, nbase);
        } else {
          const uint64_t roff =
              mvalid ? (args.m_shift >= 0 ? ((uint64_t)m << args.m_shift) : pdep64((uint64_t)m, args.mask_m)) : 0;
          if (args.m_low5) {
            // the low 5 bits of the row index are the low 5 address bits:
            // for each column the warp's 32 rows are 32 consecutive floats
            // (thread = row), stored column by column without staging.
            // nbase is a multiple of 64, so pdep(nbase + c) = pdep(nbase) |
            // pdep(c), the second term a constant of the launch.
            const uint64_t cbase = args.n_contig ? (uint64_t)nbase : pdep64((uint64_t)nbase, args.mask_n);
            float* const obase = args.out + (mvalid ? roff : 0);
            float part = 0.f;
            [[maybe_unused]] float mx = -INFINITY;
#pragma unroll
            for (int c = 0; c < EPI_COLS; ++c) {
              if (nbase + c >= args.N) break;
              const float val = tot[c] * rs;
              if (mvalid) {
                float* ptr = obase + (cbase | args.coff_lo[c]);
                if (args.streaming) __stcs(ptr, val); else *ptr = val;
                part += val;
                if constexpr (kStat == kStatBlockMax) mx = fmaxf(mx, val);
                if constexpr (kStat == kStatAbsMax) amx = fmaxf(amx, fabsf(val));
              }
            }
            if (args.sum) local += (double)part;
            if constexpr (kStat == kStatBlockMax) put_cmax(mx, mrow0, nbase);
            continue;
          }
          // general bit deposit through the staging block (XOR-swizzled by
          // row) so that lanes walk the columns of one row at a time
          [[maybe_unused]] float mx = -INFINITY;
#pragma unroll
          for (int q = 0; q < EPI_COLS / 32; ++q) {
            const int64_t n0 = nbase + q * 32;
            if (n0 >= args.N) break;
            float* stg = stg0 + q * BLK_FLOATS;
            __syncwarp();
#pragma unroll
            for (int c = 0; c < 32; ++c) stg[lane * 32 + (c ^ lane)] = tot[q * 32 + c] * rs;
            __syncwarp();
            const int64_t n = n0 + lane;
            const bool nvalid = n < args.N;
            const uint64_t coff = args.n_contig ? (uint64_t)n : pdep64((uint64_t)n, args.mask_n);
            float part = 0.f;
#pragma unroll 4
            for (int r = 0; r < 32; ++r) {
              const uint64_t roff_r = __shfl_sync(0xffffffffu, roff, r);
              const bool mv_r = __shfl_sync(0xffffffffu, mvalid ? 1 : 0, r) != 0;
              const float val = stg[r * 32 + (lane ^ r)];
              if (mv_r && nvalid) {
                float* ptr = args.out + (roff_r | coff);
                if (args.streaming) __stcs(ptr, val); else *ptr = val;
                part += val;
                if constexpr (kStat == kStatBlockMax) mx = fmaxf(mx, val);
                if constexpr (kStat == kStatAbsMax) amx = fmaxf(amx, fabsf(val));
              }
            }
            if (args.sum) local += (double)part;
          }
          if constexpr (kStat == kStatBlockMax) put_cmax(mx, mrow0, nbase);
        }
      }
    }
    __syncwarp();
    if (args.sum) {
      for (int off = 16; off; off >>= 1) local += __shfl_xor_sync(0xffffffffu, local, off);
      if (lane == 0) atomicAdd(args.sum, local);
    }
    if constexpr (kStat == kStatAbsMax) {
      for (int off = 16; off; off >>= 1) amx = fmaxf(amx, __shfl_xor_sync(0xffffffffu, amx, off));
      if (lane == 0) atomicMax(args.amax, __float_as_uint(amx));
    }
  }

  // Both CTAs reach this point only after their roles ended: CTA 0's MMAs
  // have completed, every chunk was read, every copy landed.
  tc_fence_before();
  __syncthreads();
  cluster_sync();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(TMEM_COLS) : "memory");
  }
}

int make_map(CUtensorMap* map, const __half* base, int64_t rows, int64_t Kp, int box_rows) {
  auto enc = get_encode();
  if (!enc) return set_error(CUTQC_ECUDA, "cuTensorMapEncodeTiled unavailable");
  if (((uintptr_t)base & 15) != 0) return set_error(CUTQC_EINVAL, "operand not 16-byte aligned");
  cuuint64_t dims[2] = {(cuuint64_t)Kp, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)Kp * sizeof(__half)};
  cuuint32_t box[2] = {(cuuint32_t)BK, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, const_cast<__half*>(base), dims, strides, box, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return set_error(CUTQC_ECUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
  return CUTQC_OK;
}

// Tiles per work item set by cutqc_fd_set_tiles_per_item (0: chosen below).
std::atomic<int> g_tiles_per_item{0};

// Tiles per work item: the fewest tile slots on the busiest pair, counting
// an A load (the pipe drains, the new A block lands) as about two tiles of
// time.  (One tile undercounted it where tiles are short: the dense DD
// recursion's one-k-block GEMM, 1024 row blocks x 32 column tiles, ran 3%
// faster with whole-row-block items than with the 16-tile items that
// weight picked; the FD picks are the same under both.)
int64_t pick_tiles_per_item(int64_t num_mp, int64_t num_nt, int64_t pairs) {
  int64_t best_t = 1;
  double best = 1e300;
  for (int64_t t = 4; t <= 64; ++t) {
    const int64_t items = num_mp * ((num_nt + t - 1) / t);
    const int64_t per_pair = (items + pairs - 1) / pairs;
    const double cost = (double)per_pair * ((double)std::min(t, num_nt) + 2.0);
    if (cost < best) { best = cost; best_t = t; }
  }
  return std::min(best_t, num_nt);
}

}  // namespace

bool tc_pair_supported(int64_t Kp) { return Kp > 0 && Kp % BK == 0 && Kp / BK <= MAX_KB; }

int set_pair_tiles_per_item(int t) {
  if (t < 0 || t > 4096) return set_error(CUTQC_EINVAL, "tiles per item must be in 0..4096");
  g_tiles_per_item.store(t, std::memory_order_relaxed);
  return CUTQC_OK;
}

int launch_tc_pair_gemm(const TcOperand& a, const TcOperand& b, int64_t Kp, float alpha, uint64_t mask_m,
                        uint64_t mask_n, float* out, double* sum, int streaming, cudaStream_t st,
                        const int* num_kb_dev, float* cmax, unsigned int* amax) {
  if (a.rows <= 0 || b.rows <= 0) return CUTQC_OK;
  if (!tc_pair_supported(Kp)) return set_error(CUTQC_EINVAL, "paired tensor-core K must be 64..256, a multiple of 64");
  if (a.rows >= ((int64_t)1 << 30) || b.rows >= ((int64_t)1 << 30)) return set_error(CUTQC_EUNSUPPORTED, "too many rows");
  PairMaps maps;
  int rc;
  if (((uintptr_t)a.hi & 15) != 0) return set_error(CUTQC_EINVAL, "operand not 16-byte aligned");
  if ((rc = make_map(&maps.a_lo, a.lo, a.rows, Kp, BM))) return rc;
  if ((rc = make_map(&maps.b_hi, b.hi, b.rows, Kp, BNH))) return rc;
  if ((rc = make_map(&maps.b_lo, b.lo, b.rows, Kp, BNH))) return rc;
  PairArgs args{};
  args.a_hi = a.hi;
  args.Kp = Kp;
  args.sa = a.scale;
  args.sb = b.scale;
  args.M = a.rows;
  args.N = b.rows;
  args.num_kb = (int)(Kp / BK);
  args.num_kb_dev = num_kb_dev;
  const int64_t num_mp = (a.rows + 2 * BM - 1) / (2 * BM);
  args.num_mp = (int)num_mp;
  args.num_nt = (b.rows + BN - 1) / BN;
  const int64_t pairs_avail = std::max(1, sm_count() / 2);
  const int forced = g_tiles_per_item.load(std::memory_order_relaxed);
  args.tiles_per_item = forced > 0 ? std::min<int64_t>(forced, args.num_nt)
                                   : pick_tiles_per_item(num_mp, args.num_nt, pairs_avail);
  args.num_items = num_mp * ((args.num_nt + args.tiles_per_item - 1) / args.tiles_per_item);
  args.alpha = alpha;
  args.mask_m = mask_m;
  args.mask_n = mask_n;
  args.n_contig = mask_is_low(mask_n) ? 1 : 0;
  args.m_shift = mask_contig_shift(mask_m);
  args.m_low5 = (mask_m & 31) == 31 ? 1 : 0;
  for (int c = 0; c < 64; ++c) args.coff_lo[c] = pdep64((uint64_t)c, mask_n);
  args.out = out;
  args.sum = sum;
  if (cmax && amax) return set_error(CUTQC_EINVAL, "internal: one epilogue statistic per launch");
  args.cmax = cmax;
  args.amax = amax;
  args.cmax_cols = (b.rows + 63) / 64;
  args.streaming = streaming;
  args.status = device_status_ptr();
  // direct 8-byte stores from registers when column bits 0..5 are output
  // address bits 0..5 (e.g. out[m * N + n] with N a multiple of 64, or an
  // intermediate whose lowest open digits come from the column operand) and
  // the base is 8-byte aligned
  const bool row_major = (mask_n & 63) == 63 && (mask_m & mask_n) == 0 && ((uintptr_t)out & 7) == 0;
  if (args.n_contig && ((uintptr_t)out & 15) != 0) return set_error(CUTQC_EINVAL, "output not 16-byte aligned");
  {
    static std::mutex mu;
    static std::set<int> done;
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(mu);
    if (!done.count(dev)) {
      const void* fns[6] = {(const void*)tc_pair_gemm_kernel<true, 0>, (const void*)tc_pair_gemm_kernel<true, 1>,
                            (const void*)tc_pair_gemm_kernel<true, 2>, (const void*)tc_pair_gemm_kernel<false, 0>,
                            (const void*)tc_pair_gemm_kernel<false, 1>, (const void*)tc_pair_gemm_kernel<false, 2>};
      for (int i = 0; i < 6; ++i)
        CUTQC_CUDA_TRY(cudaFuncSetAttribute(fns[i], cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            (int)(i < 3 ? smem_bytes<true>() : smem_bytes<false>())));
      done.insert(dev);
    }
  }
  const int64_t pairs = std::min<int64_t>(args.num_items, pairs_avail);
  const int grid = (int)(2 * pairs);
  const int stat = cmax ? kStatBlockMax : amax ? kStatAbsMax : 0;
  if (row_major) {
    const size_t sm = smem_bytes<true>();
    if (stat == kStatBlockMax) tc_pair_gemm_kernel<true, kStatBlockMax><<<grid, NUM_THREADS, sm, st>>>(maps, args);
    else if (stat == kStatAbsMax) tc_pair_gemm_kernel<true, kStatAbsMax><<<grid, NUM_THREADS, sm, st>>>(maps, args);
    else tc_pair_gemm_kernel<true, 0><<<grid, NUM_THREADS, sm, st>>>(maps, args);
  } else {
    const size_t sm = smem_bytes<false>();
    if (stat == kStatBlockMax) tc_pair_gemm_kernel<false, kStatBlockMax><<<grid, NUM_THREADS, sm, st>>>(maps, args);
    else if (stat == kStatAbsMax) tc_pair_gemm_kernel<false, kStatAbsMax><<<grid, NUM_THREADS, sm, st>>>(maps, args);
    else tc_pair_gemm_kernel<false, 0><<<grid, NUM_THREADS, sm, st>>>(maps, args);
  }
  CUTQC_LAUNCH_CHECK("tc_pair_gemm_kernel");
  return CUTQC_OK;
}

}  // namespace cutqc

extern "C" int cutqc_fd_set_tiles_per_item(int tiles_per_item) {
  return cutqc::set_pair_tiles_per_item(tiles_per_item);
}
