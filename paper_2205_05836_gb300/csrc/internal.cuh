// Internal helpers shared by the CUDA translation units of libcutqc.
// Nothing here is part of the public C ABI (see include/cutqc.h).
#pragma once

#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <stdint.h>
#include <stddef.h>

#include "../../include/cutqc.h"

namespace cutqc {

// ---------------------------------------------------------------- host side

// Records a message for cutqc_last_error() (thread-local) and returns code.
int set_error(int code, const char* fmt, ...);
// Maps a CUDA runtime error to CUTQC_ECUDA with its text.
int cuda_error(cudaError_t e, const char* where);

#define CUTQC_CUDA_TRY(expr)                                          \
  do {                                                                \
    cudaError_t _e = (expr);                                          \
    if (_e != cudaSuccess) return ::cutqc::cuda_error(_e, #expr);     \
  } while (0)

// Kernels enqueued (or captured into a graph) by the library, process-wide:
// every launch site is followed by one CUTQC_LAUNCH_CHECK, which counts it;
// a check that covers several launches adds the others with count_launches.
void count_launches(int n);

#define CUTQC_LAUNCH_CHECK(where)                                     \
  do {                                                                \
    ::cutqc::count_launches(1);                                       \
    cudaError_t _e = cudaGetLastError();                              \
    if (_e != cudaSuccess) return ::cutqc::cuda_error(_e, where);     \
  } while (0)

// Device-side status word: kernels that wait on a barrier give up after a
// bounded time and record why here; the host reads it with
// cutqc_device_status().
int* device_status_ptr();

// Number of SMs of the current device (cached per device).
int sm_count();

inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// ---------------------------------------------------------------- device side

__device__ __forceinline__ void record_status(int* status, int code) {
  if (status) atomicCAS(status, 0, code);
}

// IEEE 754 binary64 -> binary32, round to nearest, ties to even, on the
// integer pipes.  GB300's FP64 pipe converts only a few values per SM per
// clock, which is what bounded the FP64 attribution loads; this follows the
// two formats' definitions instead.  Binary64 fields: sign, 11-bit exponent
// e (bias 1023), 52-bit fraction; binary32: 8-bit exponent (bias 127), 23-bit
// fraction, subnormals in units of 2^-149.  NaN stays a (quiet) NaN.
// The rare cases: binary32 subnormals and underflow, overflow, infinities,
// NaN (e in 1..896 or 1151..2047).
__device__ __forceinline__ float f64_to_f32_rare(unsigned hi, unsigned lo) {
  const unsigned sign = hi & 0x80000000u;
  const int e = (int)((hi >> 20) & 0x7ffu);
  const unsigned fh = hi & 0xfffffu;                        // fraction bits 51..32
  if (e == 0x7ff) return __uint_as_float(sign | ((fh | lo) ? 0x7fc00000u : 0x7f800000u));
  if (e >= 1151) return __uint_as_float(sign | 0x7f800000u);  // |d| >= 2^128
  // binary32 subnormal or zero: d = sig * 2^(e - 1075) with sig = 2^52 +
  // fraction, i.e. sig * 2^(e - 926) units of 2^-149
  const int s = 926 - e;                                     // >= 30 here
  if (e == 0 || s >= 54) return __uint_as_float(sign);
  const unsigned long long sig = (1ull << 52) | ((unsigned long long)fh << 32) | lo;
  unsigned long long q = sig >> s;
  const unsigned long long rem = sig & ((1ull << s) - 1), half = 1ull << (s - 1);
  q += (rem > half || (rem == half && (q & 1ull))) ? 1ull : 0ull;
  return __uint_as_float(sign | (unsigned)q);
}

// The common case in a handful of instructions: a binary32 normal result
// (biased exponent e - 896 in 1..254: rebias the exponent, keep fraction bits
// 51..29, round on bits 28..0, the low bit of r deciding a tie; a carry out
// of the fraction bumps the exponent, to infinity above the largest float),
// or zero for e = 0 (zero or a binary64 subnormal).  The rare cases run only
// in warps that hold one, behind a vote, so that the common path keeps its
// registers and needs no branch per value.
__device__ __forceinline__ float f64_to_f32_rn(double d) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(d);
  const unsigned hi = (unsigned)(u >> 32), lo = (unsigned)u;
  const unsigned mag = hi & 0x7fffffffu;
  const unsigned e = mag >> 20;
  unsigned r = ((mag - (896u << 20)) << 3) | (lo >> 29);
  r += ((lo & 0x1fffffffu) + (r & 1u)) > 0x10000000u ? 1u : 0u;
  r = e == 0 ? 0u : r;
  float f = __uint_as_float((hi & 0x80000000u) | r);
  const bool rare = e != 0 && e - 897u >= 254u;
  if (__any_sync(__activemask(), rare)) {
    if (rare) f = f64_to_f32_rare(hi, lo);
  }
  return f;
}

// Software bit deposit: scatter the low bits of v to the set bits of mask.
__host__ __device__ __forceinline__ uint64_t pdep64(uint64_t v, uint64_t mask) {
  uint64_t r = 0;
  while (mask) {
    uint64_t low = mask & (~mask + 1);
    if (v & 1) r |= low;
    v >>= 1;
    mask &= mask - 1;
  }
  return r;
}

// Software bit extract: gather the bits of v at the set bits of mask.
__host__ __device__ __forceinline__ uint64_t pext64(uint64_t v, uint64_t mask) {
  uint64_t r = 0;
  int k = 0;
  while (mask) {
    uint64_t low = mask & (~mask + 1);
    if (v & low) r |= (uint64_t)1 << k;
    ++k;
    mask &= mask - 1;
  }
  return r;
}

// A contraction step's operand view and result layout (see contract.cu).
struct OperandView {
  const float* src;      // [2^o][4^k] fp32 tensor (rows x, columns c)
  int o;                 // output bits of the source tensor
  int k;                 // cut digits of the source tensor (columns 4^k)
  uint64_t open_dmask;   // bit mask (2 bits per digit) of the open digits in c
  uint64_t shared_dmask; // bit mask of the shared (contracted) digits in c
  int n_open;            // number of open digits
  int n_shared;          // number of shared digits
  int64_t rows() const { return ((int64_t)1 << o) << (2 * n_open); }
  int64_t kdim() const { return (int64_t)1 << (2 * n_shared); }
};

}  // namespace cutqc
