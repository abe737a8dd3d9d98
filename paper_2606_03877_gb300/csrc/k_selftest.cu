// k_selftest.cu -- self-test of the bounded waits of the persistent tensor-core kernels.
//
// Every wait of those kernels (an mbarrier phase that an MMA commit or a TMA copy completes) is
// a try-wait loop that gives up after a wall-time limit, raises the block's abort flag and makes
// the kernel finish without further MMAs and with MLPS_ERR_TIMEOUT in its status word, so that
// no call can hang the device. This entry point runs the same wait, `mbar_wait`, on a barrier
// that nothing ever arrives at, and reports through the same status word: a test can make a wait
// run out on the GPU without any fault, and check that the context stays usable afterwards.
#include <cuda_runtime.h>

#include "mlps_common.cuh"
#include "tc_ptx.cuh"

namespace mlps {
namespace {

__global__ void k_selftest_wait(int* status, uint64_t limit_ns) {
  __shared__ __align__(8) uint64_t bar;
  __shared__ int abort_flag;
  const uint32_t b = tc::smem_u32(&bar);
  if (threadIdx.x == 0) {
    tc::mbar_init(b, 1);
    abort_flag = 0;
    tc::fence_mbar_init();
  }
  __syncthreads();
  // no thread arrives: phase 0 never completes and every thread's wait gives up (the first at
  // limit_ns, the others on the abort flag it raises)
  const bool ok = tc::mbar_wait(b, 0u, &abort_flag, limit_ns);
  __syncthreads();
  if (threadIdx.x == 0 && (!ok || abort_flag)) set_status(status, MLPS_ERR_TIMEOUT);
}

}  // namespace
}  // namespace mlps

extern "C" mlps_status mlps_selftest_bounded_wait(int32_t limit_us, void* scratch, size_t scratch_bytes,
                                                  void* stream) {
  if (!scratch || scratch_bytes < 256 || (reinterpret_cast<uintptr_t>(scratch) & 255) != 0)
    return MLPS_ERR_INVALID_ARGUMENT;
  if (limit_us < 1 || limit_us > 1000000) return MLPS_ERR_INVALID_ARGUMENT;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int* status = static_cast<int*>(scratch);
  if (cudaMemsetAsync(status, 0, 256, st) != cudaSuccess) return MLPS_ERR_CUDA;
  mlps::k_selftest_wait<<<1, 64, 0, st>>>(status, (uint64_t)limit_us * 1000ull);
  return cudaGetLastError() == cudaSuccess ? MLPS_OK : MLPS_ERR_CUDA;
}
