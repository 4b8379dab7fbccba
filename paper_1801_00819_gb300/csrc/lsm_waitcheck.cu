// Check of the bounded waits the tcgen05 kernels use: one block waits on an mbarrier that nothing
// will ever arrive at.  The wait must give up after its time limit and the kernel must return
// normally, reporting the timeout, so that the context stays usable.  No tensor-core work runs.
#include <cuda_runtime.h>

#include "../../include/lsm.h"
#include "lsm_internal.h"
#include "lsm_umma.cuh"

namespace lsm {

static __device__ int g_wait_outcome;  // 1: the wait completed, 2: it gave up

__global__ void bounded_wait_check_kernel() {
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) umma::mbar_init(&bar, 1);  // expects one arrival that never comes
    __syncthreads();
    const bool done = umma::mbar_wait(&bar, 0);
    __syncthreads();
    if (threadIdx.x == 0) g_wait_outcome = done ? 1 : 2;
}

}  // namespace lsm

extern "C" int lsm_check_bounded_wait(void* stream) {
    using namespace lsm;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const int zero = 0;
    if (cudaMemcpyToSymbolAsync(g_wait_outcome, &zero, sizeof(int), 0, cudaMemcpyHostToDevice, st) != cudaSuccess) {
        cudaGetLastError();
        return LSM_ERR_CUDA;
    }
    bounded_wait_check_kernel<<<1, 32, 0, st>>>();
    count_launch();
    int outcome = 0;
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpyFromSymbolAsync(&outcome, g_wait_outcome, sizeof(int), 0, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
        cudaGetLastError();
        return LSM_ERR_CUDA;
    }
    return outcome == 2 ? LSM_ERR_TIMEOUT : outcome == 1 ? LSM_OK : LSM_ERR_CUDA;
}
