// Common device helpers: complex arithmetic, bulk (TMA) copies into shared memory,
// mbarriers with bounded waits, block reductions.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace dm {

// Device-side fault flags (bit set in ctx->d_err).
enum : int {
    ERR_TIMEOUT = 1,     // a bounded wait on an mbarrier expired
    ERR_BAD_INDEX = 2,   // a face index outside [0, n_v)
    ERR_NONFINITE = 4,   // NaN/Inf in vertex positions
    ERR_DEGENERATE = 8,  // normaliser (total weighted area, or enclosed volume) not > 0
};

template <class R>
struct Cx {
    R x, y;
};

template <class R>
__device__ __forceinline__ Cx<R> cmul(Cx<R> a, Cx<R> b) {
    return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
template <class R>
__device__ __forceinline__ Cx<R> cconjmul(Cx<R> a, Cx<R> b) {  // conj(a) * b
    return {a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x};
}
template <class R>
__device__ __forceinline__ R re_mul(Cx<R> a, Cx<R> b) {  // Re(a * b)
    return a.x * b.x - a.y * b.y;
}

// ---------------------------------------------------------------- shared-memory bulk copies
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

// Make the barrier initialisation visible to the async (bulk-copy) proxy.
__device__ __forceinline__ void mbar_fence_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Order this thread's earlier generic-proxy shared-memory accesses before later async-proxy writes.
__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

// 1D bulk copy global -> shared, completion signalled on `bar` (complete_tx).
// dst and src must be 16-byte aligned and bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

// Wait for phase `parity` of `bar`, giving up after `limit_ns` nanoseconds.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, uint64_t limit_ns) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    while (true) {
        if (mbar_try_wait(bar, parity)) return true;
        if (global_ns() - t0 > limit_ns) return false;
    }
}

constexpr uint64_t kWaitLimitNs = 1000000000ull;  // 1 s

// ---------------------------------------------------------------- tile pipeline
// Streams n_tiles tiles of TILE records from `src` through STAGES shared-memory stages.
// full[s] completes when the bulk copy of a tile into stage s has landed; empty[s] collects
// one arrival per warp when that warp is done with the stage; warp 0 then refills it. No
// block-wide barrier per tile, so warps may run up to STAGES - 1 tiles apart. Every wait is
// bounded; on expiry the thread sets ERR_TIMEOUT, stops, and thread 0 waits (bounded) for
// the copies it issued. body(const Rec* tile) consumes one tile. Call with all threads of the
// block after a __syncthreads; n_warps = blockDim.x / 32.
template <int STAGES, int TILE, class Rec, class Body>
__device__ __forceinline__ void run_tile_pipeline(const Rec* __restrict__ src, int n_tiles, Rec (*stage)[TILE],
                                                  uint64_t* full, uint64_t* empty, int* err, Body&& body) {
    constexpr uint32_t kBytes = TILE * sizeof(Rec);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], blockDim.x >> 5);
        }
        mbar_fence_init();
    }
    __syncthreads();
    int issued = n_tiles < STAGES ? n_tiles : STAGES;
    if (tid == 0)
        for (int t = 0; t < issued; ++t) {
            mbar_arrive_expect_tx(&full[t], kBytes);
            bulk_g2s(stage[t], src + (int64_t)t * TILE, kBytes, &full[t]);
        }
    int t = 0;
    bool ok = true;
    for (; t < n_tiles; ++t) {
        const int s = t % STAGES;
        const uint32_t par = (uint32_t)(t / STAGES) & 1u;
        if (!mbar_wait_bounded(&full[s], par, kWaitLimitNs)) {
            ok = false;
            break;
        }
        body(stage[s]);
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[s]);
        if (warp == 0 && t + STAGES < n_tiles) {
            if (!mbar_wait_bounded(&empty[s], par, kWaitLimitNs)) {
                ok = false;
                break;
            }
            if (lane == 0) {
                fence_proxy_async_smem();
                mbar_arrive_expect_tx(&full[s], kBytes);
                bulk_g2s(stage[s], src + (int64_t)(t + STAGES) * TILE, kBytes, &full[s]);
            }
            issued = t + STAGES + 1;
            __syncwarp();
        }
    }
    if (!ok) {
        atomicOr(err, ERR_TIMEOUT);
        if (tid == 0)
            for (int u = t; u < issued; ++u) mbar_wait_bounded(&full[u % STAGES], (uint32_t)(u / STAGES) & 1u, kWaitLimitNs);
    }
}

// ---------------------------------------------------------------- reductions
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Deterministic block sum (fixed tree order). `scratch` holds >= 32 doubles. Result valid in thread 0.
template <int NT>
__device__ __forceinline__ double block_sum(double v, double* scratch) {
    v = warp_sum(v);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) scratch[wid] = v;
    __syncthreads();
    double r = 0.0;
    if (wid == 0) {
        r = lane < NT / 32 ? scratch[lane] : 0.0;
        r = warp_sum(r);
    }
    return r;
}

// Error-free sum of two floats (Knuth's two-sum): t + e == a + b exactly.
__device__ __forceinline__ void two_sum(float a, float b, float& t, float& e) {
    t = a + b;
    const float bp = t - a;
    e = (a - (t - bp)) + (b - bp);
}

// Deterministic block sum of per-thread compensated FP32 sums (thread value s - c, the convention of
// a Kahan sum): within a warp the pairs are combined in FP32 by error-free additions in a fixed
// butterfly order, the warps' values in FP64. No per-thread FP64 work. `scratch` holds >= 32 doubles;
// result valid in thread 0.
template <int NT>
__device__ __forceinline__ double block_sum_comp(float s, float c, double* scratch) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float s2 = __shfl_xor_sync(0xffffffffu, s, o), c2 = __shfl_xor_sync(0xffffffffu, c, o);
        float t, e;
        two_sum(s, s2, t, e);
        s = t;
        c = (c + c2) - e;  // (s1 - c1) + (s2 - c2) = t - ((c1 + c2) - e)
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) scratch[wid] = (double)s - (double)c;
    __syncthreads();
    double r = 0.0;
    if (wid == 0) {
        r = lane < NT / 32 ? scratch[lane] : 0.0;
        r = warp_sum(r);
    }
    return r;
}

// K such block sums at once, with two barriers in all: thread k < K returns sum k (the warps' values
// added in warp order); other threads return 0. `scratch` holds >= K * NT / 32 doubles.
template <int NT, int K>
__device__ __forceinline__ double block_sums_comp(float (&s)[K], float (&c)[K], double* scratch) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const float s2 = __shfl_xor_sync(0xffffffffu, s[k], o), c2 = __shfl_xor_sync(0xffffffffu, c[k], o);
            float t, e;
            two_sum(s[k], s2, t, e);
            s[k] = t;
            c[k] = (c[k] + c2) - e;
        }
    }
    constexpr int W = NT / 32;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) {
#pragma unroll
        for (int k = 0; k < K; ++k) scratch[k * W + wid] = (double)s[k] - (double)c[k];
    }
    __syncthreads();
    double r = 0.0;
    if (threadIdx.x < K)
        for (int w = 0; w < W; ++w) r += scratch[threadIdx.x * W + w];
    return r;
}

// Division by a grid dimension without a run-time divide: for n < 2^32, n / d is the high word of
// n * m with m = ceil(2^64 / d) (exact, since n (m - 2^64 / d) / 2^64 < 2^-32 < 1 / d).
struct FastDiv {
    unsigned long long m;
    uint32_t d;
};
inline FastDiv make_fastdiv(uint32_t d) {
    FastDiv f;
    f.d = d;
    f.m = d > 1 ? ~0ull / d + 1 : 0;
    return f;
}
__device__ __forceinline__ uint32_t fdiv(uint32_t n, const FastDiv& f) {
    return f.d > 1 ? (uint32_t)__umul64hi((unsigned long long)n, f.m) : n;
}

// Half-spectrum index (< 2^32) -> integer frequency, with the divisions by Nzh and Ny precomputed.
__device__ __forceinline__ void decode_h_fast(uint32_t idx, const FastDiv& dzh, const FastDiv& dy, int Nx, int Ny,
                                              int& nx, int& ny, int& nz) {
    const uint32_t t = fdiv(idx, dzh);
    const int iz = (int)(idx - t * dzh.d);
    const uint32_t ix = fdiv(t, dy);
    const int iy = (int)(t - ix * dy.d);
    nx = (int)ix < (Nx + 1) / 2 ? (int)ix : (int)ix - Nx;
    ny = iy < (Ny + 1) / 2 ? iy : iy - Ny;
    nz = iz;
}

// Half-spectrum index -> integer frequency (fftfreq convention on x, y; n_z = iz).
__device__ __forceinline__ void decode_h(int64_t idx, int Nx, int Ny, int Nzh, int& nx, int& ny, int& nz) {
    const int iz = (int)(idx % Nzh);
    const int64_t t = idx / Nzh;
    const int iy = (int)(t % Ny);
    const int ix = (int)(t / Ny);
    nx = ix < (Nx + 1) / 2 ? ix : ix - Nx;
    ny = iy < (Ny + 1) / 2 ? iy : iy - Ny;
    nz = iz;
}

}  // namespace dm
