// Benchmark-only probe (built as its own library, libdm_mufu_probe.so, not part of libdeltamic.so):
// throughput of the MUFU (XU) operations the mesh-transform sums spend per term, sin/cos pairs and
// approximate reciprocals, issued as independent dependency chains by enough warps to fill every SM and
// timed with CUDA events. The result is the denominator of the forward sum's XU roofline.
//
//   int dm_probe_mufu(int kind, int device, double* ops_per_s)
//     kind 0 = sin/cos pairs (__sincosf; a pair counts 2), kind 1 = rcp.approx; operations per second on
//     `device`. Runs two launches on the default stream and synchronises. Returns 0, -1 for a bad argument,
//     -6 for a CUDA error.
#include <cuda_runtime.h>
#include <stdint.h>

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

}  // namespace

extern "C" int dm_probe_mufu(int32_t kind, int32_t device, double* ops_per_s) {
    if (!ops_per_s || (kind != 0 && kind != 1)) return -1;
    int prev = 0;
    if (cudaGetDevice(&prev) != cudaSuccess || cudaSetDevice(device) != cudaSuccess) return -6;
    int sms = 0;
    float* out = nullptr;
    cudaEvent_t a = nullptr, b = nullptr;
    int st = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess ||
        cudaMalloc(&out, sizeof(float)) != cudaSuccess || cudaEventCreate(&a) != cudaSuccess ||
        cudaEventCreate(&b) != cudaSuccess) {
        st = -6;
    } else {
        const unsigned blocks = (unsigned)sms * 8;
        float ms = 0.f;
        for (int rep = 0; rep < 2 && st == 0; ++rep) {  // the first launch warms up
            cudaEventRecord(a);
            if (kind == 0)
                k_probe_sincos<<<blocks, PT>>>(out, 0.3f);
            else
                k_probe_rcp<<<blocks, PT>>>(out, 0.3f);
            cudaEventRecord(b);
            if (cudaEventSynchronize(b) != cudaSuccess || cudaEventElapsedTime(&ms, a, b) != cudaSuccess)
                st = -6;
        }
        const double per_step = kind == 0 ? 2.0 : 1.0;  // a sin/cos pair is two MUFU operations
        if (st == 0) *ops_per_s = (double)blocks * PT * CHAINS * ITERS * per_step / (ms * 1e-3);
    }
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    if (out) cudaFree(out);
    cudaGetLastError();
    cudaSetDevice(prev);
    return st;
}
