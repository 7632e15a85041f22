// Tensor-core contraction for Eq. 1 on sm_103a (tcgen05 + TMA + TMEM).
//
// C[m][n] = alpha * sa[m] * sb * sum_s (Ah Bh + Ah Bl + Al Bh)[m][n][s]
// where A = sa * (Ah + Al), B = sb * (Bh + Bl) are the float16 hi/lo splits of
// the float32 operands (power-of-two scales: one per row of A, one for all of
// B, see prep_kernel): about 22 significant bits per operand, products exact
// in the FP32 accumulator.  The signed I/X/Y/Z terms of Eq. 1 cancel (sum
// |terms| is ~10x |P| on the 30-qubit supremacy workload), which is why a
// single FP16/BF16/TF32 pass is not accurate enough and the split is used.
//
// The tensor core rounds its FP32 accumulator toward zero after each MMA,
// which over a long chain of signed terms leaves a negative bias (about
// -1.5e-6 in sum p on the 30-qubit workload).  Every 64 values of k are
// therefore accumulated in a fresh TMEM accumulator (a "chunk", 12 MMAs),
// and the chunks are added in registers with round-to-nearest; from 4^6
// values of k on (64 chunks and more) that sum is compensated (Kahan), so
// that the rounding of a long chain of chunk totals does not grow with K.
//
// Kernel organisation (one CTA per SM, persistent over 128 x 128 tiles):
//   warp 8       TMA producer: per 64-wide k-block loads A_hi, A_lo, B_hi,
//                B_lo (128 x 64 each) into a 2-stage 128B-swizzled ring
//   warp 9       MMA issuer: 4 x 3 tcgen05.mma (M=128, N=128, K=16) per
//                k-block (one chunk) into one of four 128 x 128 FP32 chunk
//                buffers in TMEM (so the MMAs run up to three chunks ahead
//                of the epilogue)
//   warps 0-7    epilogue: warp w owns TMEM lanes 32*(w%4).. (tile rows) and
//                columns 64*(w/4)..+63; adds every chunk into 64 register
//                totals, then scales and stores the tile.  Row-major outputs
//                (out[m * N + n]) go out as 32 x 32 TMA bulk-tensor stores
//                from a 128B-swizzled staging block per 32 x 32 block (one
//                block per store, so a warp never waits for its own stores
//                within a tile); other bit-deposit layouts
//                (out[pdep(m, mask_m) | pdep(n, mask_n)]) through a staged
//                transpose and per-element stores.  Optional FP64 sum.
// Tiles are walked with m fastest so the few B tiles in flight stay in L2.
// Every barrier wait is bounded in time; on expiry the CTA records
// CUTQC_ETIMEOUT in the device status word, drains its own copies and MMAs,
// frees its tensor memory and returns.
#include "internal.cuh"
#include "contract.cuh"

#include "tc_ptx.cuh"

#include <mutex>
#include <set>

namespace cutqc {

namespace {

using namespace tc;

constexpr int BM = 128, BN = 128, BK = 64;               // BK in fp16 elements (128-byte rows)
constexpr int STAGES = 2;
constexpr int KB_PER_CHUNK = 1;                          // chunk = 64 values of k = 12 MMAs
constexpr int NBUF = 4;                                  // chunk buffers in TMEM
constexpr int A_TILE = BM * BK * 2;                      // 16 KiB
constexpr int B_TILE = BN * BK * 2;                      // 16 KiB
constexpr int STAGE_BYTES = 2 * A_TILE + 2 * B_TILE;     // 64 KiB
constexpr int TMEM_COLS = NBUF * BN;                     // 512
constexpr int NUM_THREADS = 320;
constexpr int kCompensatedMinKb = 64;   // k-blocks (4^6 = 4096 values of k) from which chunk sums are compensated
constexpr int EPI_THREADS = 256;
constexpr int EPI_COLS = 64;                             // columns per epilogue warp
constexpr int BLK_FLOATS = 32 * 32;                      // one 32 x 32 staging block
constexpr int STG_BYTES = 8 * (EPI_COLS / 32) * BLK_FLOATS * 4;   // 64 KiB

struct TcMaps {
  CUtensorMap a_hi, a_lo, b_hi, b_lo;
  CUtensorMap out;   // row-major output [M][N] float32, 32 x 32 box, 128B swizzle
};

struct TcArgs {
  const float* sa;
  const float* sb;
  int64_t M, N;
  int num_kb;
  const int* num_kb_dev;  // nullable: k-blocks in use, read on the device (<= num_kb)
  int num_m_blk;
  int64_t num_tiles;
  float alpha;
  uint64_t mask_m, mask_n;
  int n_contig;
  int m_shift;
  float* out;
  double* sum;
  int streaming;
  int row_major;      // out[m * N + n]: bulk-tensor stores through maps.out
  int* status;
};

struct SmemTail {
  uint64_t full[STAGES];
  uint64_t empty[STAGES];
  uint64_t cfull[NBUF];
  uint64_t cempty[NBUF];
  uint64_t fin;
  uint32_t tmem_slot;
  int abort_flag;
};

constexpr size_t SMEM_BYTES = 1024 + STAGES * STAGE_BYTES + STG_BYTES + sizeof(SmemTail);
static_assert(SMEM_BYTES <= 232448, "shared memory budget");

// Instruction descriptor: kind::f16, A = B = F16, D = F32, both K-major,
// N = 128, M = 128.
constexpr uint32_t kIdesc = (1u << 4) | (0u << 7) | (0u << 10) | ((uint32_t)(BN >> 3) << 17) |
                            ((uint32_t)(BM >> 4) << 24);

__device__ __forceinline__ void umma_f16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t accum) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n"
      ::"r"(d_tmem), "l"(adesc), "l"(bdesc), "r"(kIdesc), "r"(accum)
      : "memory");
}
__device__ __forceinline__ void umma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
               : "memory");
}
template <bool kRowMajor, bool kCompensated>
__global__ void __launch_bounds__(NUM_THREADS, 1)
tc_gemm_kernel(const __grid_constant__ TcMaps maps, const TcArgs args) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  float* stg_all = reinterpret_cast<float*>(smem + STAGES * STAGE_BYTES);
  SmemTail* tail = reinterpret_cast<SmemTail*>(smem + STAGES * STAGE_BYTES + STG_BYTES);
  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  // k-blocks in use: a count chosen on the device (cut-term pruning) when
  // given, never more than the operands hold
  const int num_kb = args.num_kb_dev ? max(1, min(args.num_kb, __ldg(args.num_kb_dev))) : args.num_kb;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(smem_u32(&tail->full[s]), 1);
      mbar_init(smem_u32(&tail->empty[s]), 1);
    }
    for (int a = 0; a < NBUF; ++a) {
      mbar_init(smem_u32(&tail->cfull[a]), 1);
      mbar_init(smem_u32(&tail->cempty[a]), EPI_THREADS);
    }
    mbar_init(smem_u32(&tail->fin), 1);
    tail->abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tail->tmem_slot)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
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
      for (int64_t tile = blockIdx.x; tile < args.num_tiles && !*abort_flag; tile += gridDim.x) {
        const int mb = (int)(tile % args.num_m_blk);
        const int nb = (int)(tile / args.num_m_blk);
        bool ok = true;
        for (int kb = 0; kb < num_kb; ++kb) {
          if (!mbar_wait(smem_u32(&tail->empty[stage]), phase ^ 1u, abort_flag)) { fail(); ok = false; break; }
          uint8_t* st = smem + stage * STAGE_BYTES;
          const uint32_t bar = smem_u32(&tail->full[stage]);
          mbar_expect_tx(bar, STAGE_BYTES);
          tma_load_2d(smem_u32(st), &maps.a_hi, kb * BK, mb * BM, bar);
          tma_load_2d(smem_u32(st + A_TILE), &maps.a_lo, kb * BK, mb * BM, bar);
          tma_load_2d(smem_u32(st + 2 * A_TILE), &maps.b_hi, kb * BK, nb * BN, bar);
          tma_load_2d(smem_u32(st + 2 * A_TILE + B_TILE), &maps.b_lo, kb * BK, nb * BN, bar);
          issued[stage] = true;
          issued_par[stage] = phase;
          if (++stage == STAGES) { stage = 0; phase ^= 1u; }
        }
        if (!ok) break;
      }
      // every copy this thread started has landed before the CTA may exit
      for (int s = 0; s < STAGES; ++s)
        if (issued[s] && !mbar_wait(smem_u32(&tail->full[s]), issued_par[s], nullptr))
          record_status(args.status, CUTQC_ETIMEOUT);
    }
  } else if (warp == 9) {
    // ----------------------------------------------------------- MMA issue
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0;
      int buf = 0;
      uint32_t buf_phase = 0;
      bool any = false;
      for (int64_t tile = blockIdx.x; tile < args.num_tiles && !*abort_flag; tile += gridDim.x) {
        bool ok = true;
        for (int kb = 0; kb < num_kb; ++kb) {
          const int ks = kb % KB_PER_CHUNK;
          if (ks == 0) {
            if (!mbar_wait(smem_u32(&tail->cempty[buf]), buf_phase ^ 1u, abort_flag)) { fail(); ok = false; break; }
            tc_fence_after();
          }
          if (!mbar_wait(smem_u32(&tail->full[stage]), phase, abort_flag)) { fail(); ok = false; break; }
          tc_fence_after();
          const uint32_t d = tmem_base + (uint32_t)(buf * BN);
          const uint32_t st = smem_u32(smem + stage * STAGE_BYTES);
          const uint32_t ah = st, al = st + A_TILE, bh = st + 2 * A_TILE, bl = st + 2 * A_TILE + B_TILE;
#pragma unroll
          for (int kk = 0; kk < BK / 16; ++kk) {
            const uint32_t off = kk * 32;   // 16 fp16 = 32 bytes along k inside the swizzle row
            const uint64_t dah = sw128_desc(ah + off), dal = sw128_desc(al + off);
            const uint64_t dbh = sw128_desc(bh + off), dbl = sw128_desc(bl + off);
            umma_f16(d, dah, dbh, (ks | kk) != 0 ? 1u : 0u);
            umma_f16(d, dah, dbl, 1u);
            umma_f16(d, dal, dbh, 1u);
          }
          any = true;
          umma_commit(smem_u32(&tail->empty[stage]));
          if (ks == KB_PER_CHUNK - 1 || kb == num_kb - 1) {
            umma_commit(smem_u32(&tail->cfull[buf]));
            if (++buf == NBUF) { buf = 0; buf_phase ^= 1u; }
          }
          if (++stage == STAGES) { stage = 0; phase ^= 1u; }
        }
        if (!ok) break;
      }
      // all MMAs issued by this thread complete before tensor memory is freed
      if (any) {
        umma_commit(smem_u32(&tail->fin));
        if (!mbar_wait(smem_u32(&tail->fin), 0, nullptr)) record_status(args.status, CUTQC_ETIMEOUT);
      }
    }
  } else {
    // ------------------------------------------------------------ epilogue
    // warp w: TMEM lanes 32*(w%4).. = tile rows, columns 64*(w/4) .. +63
    const int g = warp & 3, h = warp >> 2;
    int buf = 0;
    uint32_t buf_phase = 0;
    double local = 0.0;
    const int row = g * 32 + lane;
    const int num_chunks = (num_kb + KB_PER_CHUNK - 1) / KB_PER_CHUNK;
    const float sbg = __ldg(args.sb);
    float* stg0 = stg_all + warp * (EPI_COLS / 32) * BLK_FLOATS;
    float tot[EPI_COLS];
    // long chunk chains (kCompensated): compensated (Kahan) float32 sums of
    // the chunks, the rounding error of each add carried in comp
    float comp[kCompensated ? EPI_COLS : 1];
    for (int64_t tile = blockIdx.x; tile < args.num_tiles && !*abort_flag; tile += gridDim.x) {
      const int mb = (int)(tile % args.num_m_blk);
      const int nb = (int)(tile / args.num_m_blk);
#pragma unroll
      for (int i = 0; i < EPI_COLS; ++i) tot[i] = 0.f;
      if constexpr (kCompensated) {
#pragma unroll
        for (int i = 0; i < EPI_COLS; ++i) comp[i] = 0.f;
      }
      bool ok = true;
      for (int ch = 0; ch < num_chunks; ++ch) {
        if (!mbar_wait(smem_u32(&tail->cfull[buf]), buf_phase, abort_flag)) { fail(); ok = false; break; }
        tc_fence_after();
        __syncwarp();
        const uint32_t taddr = tmem_base + ((uint32_t)(g * 32) << 16) + (uint32_t)(buf * BN + h * EPI_COLS);
        if constexpr (kCompensated) {
#pragma unroll
          for (int half = 0; half < 2; ++half) {
            uint32_t r0[32];
            tmem_ld32(taddr + 32 * half, r0);
#pragma unroll
            for (int i = 0; i < 32; ++i) {
              const int j = 32 * half + i;
              const float y = __uint_as_float(r0[i]) - comp[j];
              const float t = tot[j] + y;
              comp[j] = (t - tot[j]) - y;
              tot[j] = t;
            }
          }
        } else {
          uint32_t r0[32], r1[32];
          tmem_ld32(taddr, r0);
          tmem_ld32(taddr + 32, r1);
#pragma unroll
          for (int i = 0; i < 32; ++i) {
            tot[i] += __uint_as_float(r0[i]);
            tot[32 + i] += __uint_as_float(r1[i]);
          }
        }
        tc_fence_before();
        mbar_arrive(smem_u32(&tail->cempty[buf]));
        if (++buf == NBUF) { buf = 0; buf_phase ^= 1u; }
      }
      if (!ok) break;
      const int64_t m = (int64_t)mb * BM + row;
      const bool mvalid = m < args.M;
      const float rs = mvalid ? args.alpha * __ldg(args.sa + m) * sbg : 0.f;
      const int64_t nbase = (int64_t)nb * BN + h * EPI_COLS;
      if (kRowMajor) {
        // one 32 x 32 TMA box per block, from its own 128B-swizzled staging
        // block (16-byte chunk j of row r sits at chunk j ^ (r & 7)); rows or
        // columns beyond the output are clipped by the tensor map
        const int64_t mrow0 = (int64_t)mb * BM + g * 32;
#pragma unroll
        for (int q = 0; q < EPI_COLS / 32; ++q) {
          const int64_t n0 = nbase + q * 32;
          if (n0 >= args.N) break;
          float* v = tot + q * 32;
#pragma unroll
          for (int c = 0; c < 32; ++c) v[c] *= rs;
          float* stg = stg0 + q * BLK_FLOATS;
          // this block's previous store (one tile ago) has read the staging
          if (lane == 0) bulk_wait_read_le1();
          __syncwarp();
          float4* row4 = reinterpret_cast<float4*>(stg + lane * 32);
#pragma unroll
          for (int c = 0; c < 8; ++c)
            row4[c ^ (lane & 7)] = make_float4(v[4 * c], v[4 * c + 1], v[4 * c + 2], v[4 * c + 3]);
          fence_proxy_async();
          __syncwarp();
          if (lane == 0) {
            tma_store_2d(&maps.out, smem_u32(stg), (int)n0, (int)mrow0);
            bulk_commit();
          }
          if (args.sum && mvalid) {
            float t[16];
#pragma unroll
            for (int i = 0; i < 16; ++i) t[i] = v[i] + v[i + 16];
#pragma unroll
            for (int w2 = 8; w2; w2 >>= 1)
#pragma unroll
              for (int i = 0; i < w2; ++i) t[i] += t[i + w2];
            local += (double)t[0];
          }
        }
      } else {
        // general bit deposit: each 32 x 32 block goes through the staging
        // block (XOR-swizzled by row) so that lanes walk the columns of one
        // row at a time
        const uint64_t roff = mvalid ? (args.m_shift >= 0 ? ((uint64_t)m << args.m_shift) : pdep64((uint64_t)m, args.mask_m)) : 0;
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
          float part = 0.f;     // float over 32 rows, float64 across blocks
#pragma unroll 4
          for (int r = 0; r < 32; ++r) {
            const uint64_t roff_r = __shfl_sync(0xffffffffu, roff, r);
            const bool mv_r = __shfl_sync(0xffffffffu, mvalid ? 1 : 0, r) != 0;
            const float val = stg[r * 32 + (lane ^ r)];
            if (mv_r && nvalid) {
              float* ptr = args.out + (roff_r | coff);
              if (args.streaming) __stcs(ptr, val); else *ptr = val;
              part += val;
            }
          }
          if (args.sum) local += (double)part;
        }
      }
    }
    if (kRowMajor && lane == 0) bulk_wait0();   // every bulk store has completed
    __syncwarp();
    if (args.sum) {
      for (int off = 16; off; off >>= 1) local += __shfl_xor_sync(0xffffffffu, local, off);
      if (lane == 0) atomicAdd(args.sum, local);
    }
  }

  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(TMEM_COLS) : "memory");
  }
}

int make_out_map(CUtensorMap* map, float* base, int64_t rows, int64_t cols) {
  auto enc = get_encode();
  if (!enc) return set_error(CUTQC_ECUDA, "cuTensorMapEncodeTiled unavailable");
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)cols * sizeof(float)};
  cuuint32_t box[2] = {32, 32};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return set_error(CUTQC_ECUDA, "cuTensorMapEncodeTiled (output) failed (%d)", (int)r);
  return CUTQC_OK;
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

}  // namespace

int launch_tc_gemm(const TcOperand& a, const TcOperand& b, int64_t Kp, float alpha, uint64_t mask_m,
                   uint64_t mask_n, float* out, double* sum, int streaming, cudaStream_t st, const int* num_kb_dev,
                   float* cmax, unsigned int* amax) {
  if (a.rows <= 0 || b.rows <= 0) return CUTQC_OK;
  if (tc_pair_supported(Kp))
    return launch_tc_pair_gemm(a, b, Kp, alpha, mask_m, mask_n, out, sum, streaming, st, num_kb_dev, cmax, amax);
  if (amax) return set_error(CUTQC_EINVAL, "internal: output max needs the paired kernel");
  if (Kp % BK != 0 || Kp <= 0) return set_error(CUTQC_EINVAL, "tensor-core K must be a multiple of %d", BK);
  if (Kp / BK > (1 << 20)) return set_error(CUTQC_EUNSUPPORTED, "K too large");
  TcMaps maps;
  int rc;
  if ((rc = make_map(&maps.a_hi, a.hi, a.rows, Kp, BM))) return rc;
  if ((rc = make_map(&maps.a_lo, a.lo, a.rows, Kp, BM))) return rc;
  if ((rc = make_map(&maps.b_hi, b.hi, b.rows, Kp, BN))) return rc;
  if ((rc = make_map(&maps.b_lo, b.lo, b.rows, Kp, BN))) return rc;
  TcArgs args{};
  args.sa = a.scale;
  args.sb = b.scale;
  args.M = a.rows;
  args.N = b.rows;
  args.num_kb = (int)(Kp / BK);
  args.num_kb_dev = num_kb_dev;
  const int64_t mblk = (a.rows + BM - 1) / BM, nblk = (b.rows + BN - 1) / BN;
  if (mblk > 0x7fffffff || nblk > 0x7fffffff) return set_error(CUTQC_EUNSUPPORTED, "too many tiles");
  args.num_m_blk = (int)mblk;
  args.num_tiles = mblk * nblk;
  args.alpha = alpha;
  args.mask_m = mask_m;
  args.mask_n = mask_n;
  args.n_contig = mask_is_low(mask_n) ? 1 : 0;
  args.m_shift = mask_contig_shift(mask_m);
  args.out = out;
  args.sum = sum;
  args.streaming = streaming;
  args.status = device_status_ptr();
  // bulk-tensor stores when the output is out[m * N + n] with a 16-byte
  // aligned base and row pitch
  args.row_major = 0;
  if (args.n_contig && args.m_shift >= 0 && mask_n == (((uint64_t)1 << args.m_shift) - 1) &&
      ((uint64_t)1 << args.m_shift) == (uint64_t)b.rows && (b.rows * 4) % 16 == 0 && ((uintptr_t)out & 15) == 0 &&
      b.rows <= ((int64_t)1 << 31) && a.rows <= ((int64_t)1 << 31)) {
    if ((rc = make_out_map(&maps.out, out, a.rows, b.rows))) return rc;
    args.row_major = 1;
  }
  if (args.n_contig && ((uintptr_t)out & 15) != 0) return set_error(CUTQC_EINVAL, "output not 16-byte aligned");
  {
    static std::mutex mu;
    static std::set<int> done;
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(mu);
    if (!done.count(dev)) {
      CUTQC_CUDA_TRY(cudaFuncSetAttribute(tc_gemm_kernel<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)SMEM_BYTES));
      CUTQC_CUDA_TRY(cudaFuncSetAttribute(tc_gemm_kernel<false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)SMEM_BYTES));
      CUTQC_CUDA_TRY(cudaFuncSetAttribute(tc_gemm_kernel<true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)SMEM_BYTES));
      CUTQC_CUDA_TRY(cudaFuncSetAttribute(tc_gemm_kernel<false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)SMEM_BYTES));
      done.insert(dev);
    }
  }
  const int grid = (int)std::min<int64_t>(args.num_tiles, (int64_t)sm_count());
  // 4^6 terms or more (64+ chunks, e.g. the 4^K sum of K >= 8 cuts): the
  // chunk totals are added with compensation
  const bool comp = args.num_kb >= kCompensatedMinKb;
  if (args.row_major) {
    if (comp) tc_gemm_kernel<true, true><<<grid, NUM_THREADS, SMEM_BYTES, st>>>(maps, args);
    else tc_gemm_kernel<true, false><<<grid, NUM_THREADS, SMEM_BYTES, st>>>(maps, args);
  } else {
    if (comp) tc_gemm_kernel<false, true><<<grid, NUM_THREADS, SMEM_BYTES, st>>>(maps, args);
    else tc_gemm_kernel<false, false><<<grid, NUM_THREADS, SMEM_BYTES, st>>>(maps, args);
  }
  CUTQC_LAUNCH_CHECK("tc_gemm_kernel");
  return CUTQC_OK;
}

}  // namespace cutqc
