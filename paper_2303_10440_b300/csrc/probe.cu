// Failure-detection check: a bounded mbarrier wait that nothing completes, reported through the device
// error flag (the same bounded wait guards every pipeline stage of the mesh-transform kernels).
#include <cuda_runtime.h>

#include "../../include/deltamic.h"
#include "dm_common.cuh"

namespace {

// A bounded wait that nothing completes: one mbarrier in shared memory that no thread arrives at.
// Every thread gives up after limit_ns, records ERR_TIMEOUT and returns; thread 0 invalidates the
// barrier. The same bounded wait guards every pipeline stage of the mesh-transform kernels.
__global__ void k_probe_wait(uint64_t limit_ns, int* err) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        dm::mbar_init(&bar, 1);
        dm::mbar_fence_init();
    }
    __syncthreads();
    if (!dm::mbar_wait_bounded(&bar, 0, limit_ns)) atomicOr(err, dm::ERR_TIMEOUT);
    __syncthreads();
    if (threadIdx.x == 0) asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(dm::smem_u32(&bar)) : "memory");
}

}  // namespace

extern "C" dm_status dm_probe_wait_timeout(int32_t device, uint64_t limit_ns, int32_t* status) {
    if (!status || limit_ns == 0 || limit_ns > 2000000000ull) return DM_ERR_ARG;
    int prev = 0;
    if (cudaGetDevice(&prev) != cudaSuccess || cudaSetDevice(device) != cudaSuccess) return DM_ERR_CUDA;
    int* d_err = nullptr;
    int h_err = 0;
    dm_status st = DM_OK;
    if (cudaMalloc(&d_err, sizeof(int)) != cudaSuccess || cudaMemset(d_err, 0, sizeof(int)) != cudaSuccess) {
        st = DM_ERR_CUDA;
    } else {
        k_probe_wait<<<1, 64>>>(limit_ns, d_err);
        if (cudaMemcpy(&h_err, d_err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) st = DM_ERR_CUDA;
        // the context stays usable after the expired wait
        if (st == DM_OK && cudaMemset(d_err, 0, sizeof(int)) != cudaSuccess) st = DM_ERR_CUDA;
    }
    if (d_err) cudaFree(d_err);
    cudaGetLastError();
    cudaSetDevice(prev);
    if (st == DM_OK) *status = (h_err & dm::ERR_TIMEOUT) ? DM_ERR_TIMEOUT : DM_OK;
    return st;
}
