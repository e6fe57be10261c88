// Throughput probe of the MUFU (XU) operations the mesh-transform sums spend per term: sin/cos pairs
// and approximate reciprocals, issued as independent dependency chains by enough warps to fill every
// SM, timed with CUDA events. The result is the denominator of the forward sum's XU roofline.
#include <cuda_runtime.h>

#include "../../include/deltamic.h"
#include "dm_common.cuh"

namespace {

constexpr int PT = 256;      // threads per block
constexpr int CHAINS = 8;    // independent chains per thread
constexpr int ITERS = 4096;  // steps per chain

__global__ void __launch_bounds__(PT) k_probe_sincos(float* out, float seed) {
    float x[CHAINS];
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) x[c] = seed + 1e-3f * threadIdx.x + 0.1f * c;
    for (int i = 0; i < ITERS; ++i) {
#pragma unroll
        for (int c = 0; c < CHAINS; ++c) {
            float s, co;
            __sincosf(x[c], &s, &co);
            x[c] = s + co;
        }
    }
    float acc = 0.f;
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) acc += x[c];
    if (acc == 12345.0f) out[0] = acc;  // keeps the chains live; never true for these inputs
}

__global__ void __launch_bounds__(PT) k_probe_rcp(float* out, float seed) {
    float x[CHAINS];
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) x[c] = seed + 1e-3f * threadIdx.x + 0.1f * c;
    for (int i = 0; i < ITERS; ++i) {
#pragma unroll
        for (int c = 0; c < CHAINS; ++c) {
            float r;
            asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x[c]));
            x[c] = r + 1.0f;
        }
    }
    float acc = 0.f;
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) acc += x[c];
    if (acc == 12345.0f) out[0] = acc;
}

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

extern "C" dm_status dm_probe_mufu(int32_t kind, int32_t device, double* ops_per_s) {
    if (!ops_per_s || (kind != 0 && kind != 1)) return DM_ERR_ARG;
    int prev = 0;
    if (cudaGetDevice(&prev) != cudaSuccess || cudaSetDevice(device) != cudaSuccess) return DM_ERR_CUDA;
    int sms = 0;
    float* out = nullptr;
    cudaEvent_t a = nullptr, b = nullptr;
    dm_status st = DM_OK;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess ||
        cudaMalloc(&out, sizeof(float)) != cudaSuccess || cudaEventCreate(&a) != cudaSuccess ||
        cudaEventCreate(&b) != cudaSuccess) {
        st = DM_ERR_CUDA;
    } else {
        const unsigned blocks = (unsigned)sms * 8;
        float ms = 0.f;
        for (int rep = 0; rep < 2 && st == DM_OK; ++rep) {  // the first launch warms up
            cudaEventRecord(a);
            if (kind == 0)
                k_probe_sincos<<<blocks, PT>>>(out, 0.3f);
            else
                k_probe_rcp<<<blocks, PT>>>(out, 0.3f);
            cudaEventRecord(b);
            if (cudaEventSynchronize(b) != cudaSuccess || cudaEventElapsedTime(&ms, a, b) != cudaSuccess)
                st = DM_ERR_CUDA;
        }
        const double per_step = kind == 0 ? 2.0 : 1.0;  // a sin/cos pair is two MUFU operations
        if (st == DM_OK) *ops_per_s = (double)blocks * PT * CHAINS * ITERS * per_step / (ms * 1e-3);
    }
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    if (out) cudaFree(out);
    cudaGetLastError();
    cudaSetDevice(prev);
    return st;
}
