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
