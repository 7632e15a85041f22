// Failure-path self test: a wait that can never be satisfied, bounded the
// way every wait of the library's kernels is bounded.  One CTA initialises
// an mbarrier that nothing arrives on and waits on it with mbar_wait (the
// helper the tensor-core kernels use); when the bound expires the CTA
// records CUTQC_ETIMEOUT in the device status word and returns, so the
// context stays usable and the host reads the code with
// cutqc_device_status().  Nothing faults, traps or hangs.
#include "internal.cuh"
#include "tc_ptx.cuh"

namespace cutqc {
namespace {

__global__ void selftest_wait_kernel(int* status, int* waited) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x != 0) return;
  const uint32_t b = tc::smem_u32(&bar);
  tc::mbar_init(b, 1);
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  const long long t0 = clock64();
  const bool ok = tc::mbar_wait(b, 0, nullptr);   // phase 0 never completes: no arrival
  if (waited) *waited = (int)((clock64() - t0) >> 20);   // cycles / 2^20
  if (!ok) record_status(status, CUTQC_ETIMEOUT);
}

}  // namespace
}  // namespace cutqc

extern "C" int cutqc_selftest_wait_timeout(int32_t* waited_dev, void* stream) {
  using namespace cutqc;
  int* status = device_status_ptr();
  if (!status) return set_error(CUTQC_ECUDA, "no device status word");
  selftest_wait_kernel<<<1, 32, 0, (cudaStream_t)stream>>>(status, waited_dev);
  CUTQC_LAUNCH_CHECK("selftest_wait_kernel");
  return CUTQC_OK;
}
