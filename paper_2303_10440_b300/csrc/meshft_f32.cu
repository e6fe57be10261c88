// FP32 mixed-precision mesh Fourier transform (Eq. 5, 7-8) and its adjoint (Eq. 6, 9-10).
//
// Forward: one thread per band frequency, holding its integer frequency n and
// wavevector xi in registers; the block walks the triangle list in tiles of
// FWD_TILE records that a bulk (TMA) copy stages into shared memory, double
// buffered on two mbarriers. Every thread reads the same record (broadcast).
// Per term: exact phase of vertex 1 by integer arithmetic, two FP32 dot
// products for the phase differences, the local divided difference
// (meshft_math.cuh), three sincos and one reciprocal. Sums are FP32 within a
// tile and compensated (Kahan) across tiles.
//
// Adjoint: one thread per triangle (record in registers); the block walks a
// chunk of the band in tiles of ADJ_FTILE frequency records staged the same
// way. Each thread accumulates its triangle's 10 (surface) or 12 (volume) sums
// over the chunk's frequencies in registers, so the reduction over frequencies
// needs no inter-thread communication; chunks are summed afterwards in FP64 in
// a fixed order (deterministic).
#include "dm_kernels.cuh"
#include "meshft_math.cuh"

namespace dm {

namespace {

constexpr float kTwoPiOver2p32 = 1.4629180792671596e-09f;  // 2 pi / 2^32

__device__ __forceinline__ void kahan_add(float& s, float& c, float v) {
    const float y = v - c;
    const float t = s + y;
    c = (t - s) - y;
    s = t;
}

template <int MODE, bool EXPLICIT>
__global__ void __launch_bounds__(FWD_THREADS) k_fwd_f32(const TriF32* __restrict__ tris, int n_tiles, FreqSrc fs,
                                                         float tpx, float tpy, float tpz,
                                                         const double* __restrict__ d_vol, float2* __restrict__ S,
                                                         int* __restrict__ err) {
    __shared__ __align__(128) TriF32 tile[2][FWD_TILE];
    __shared__ __align__(8) uint64_t bar[2];
    const int tid = threadIdx.x;
    const int64_t M = fs.dM ? *fs.dM : fs.M;
    if ((int64_t)blockIdx.x * FWD_THREADS >= M) return;  // whole block beyond the band (uniform)
    const int64_t m = (int64_t)blockIdx.x * FWD_THREADS + tid;
    const bool active = m < M;

    int nx = 0, ny = 0, nz = 0;
    if (active) {
        if (EXPLICIT) {
            nx = fs.nlist[3 * m];
            ny = fs.nlist[3 * m + 1];
            nz = fs.nlist[3 * m + 2];
        } else {
            const int64_t idx = fs.idx ? (int64_t)fs.idx[m] : m;
            decode_h(idx, fs.Nx, fs.Ny, fs.Nzh, nx, ny, nz);
        }
    }
    const float xx = (float)nx * tpx, xy = (float)ny * tpy, xz = (float)nz * tpz;
    const uint32_t unx = (uint32_t)nx, uny = (uint32_t)ny, unz = (uint32_t)nz;

    constexpr uint32_t kTileBytes = FWD_TILE * sizeof(TriF32);
    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        mbar_fence_init();
    }
    __syncthreads();
    if (tid == 0) {
        mbar_arrive_expect_tx(&bar[0], kTileBytes);
        bulk_g2s(&tile[0][0], tris, kTileBytes, &bar[0]);
    }

    float accx = 0.f, accy = 0.f, cx = 0.f, cy = 0.f;
    for (int t = 0; t < n_tiles; ++t) {
        const int st = t & 1;
        if (tid == 0 && t + 1 < n_tiles) {
            fence_proxy_async_smem();
            mbar_arrive_expect_tx(&bar[st ^ 1], kTileBytes);
            bulk_g2s(&tile[st ^ 1][0], tris + (int64_t)(t + 1) * FWD_TILE, kTileBytes, &bar[st ^ 1]);
        }
        const bool ok = mbar_wait_bounded(&bar[st], (t >> 1) & 1, kWaitLimitNs);
        if (__syncthreads_or(!ok)) {
            if (tid == 0) {
                atomicOr(err, ERR_TIMEOUT);
                mbar_wait_bounded(&bar[st], (t >> 1) & 1, kWaitLimitNs);
                if (t + 1 < n_tiles) mbar_wait_bounded(&bar[st ^ 1], ((t + 1) >> 1) & 1, kWaitLimitNs);
            }
            return;
        }
        float px = 0.f, py = 0.f;
#pragma unroll 2
        for (int j = 0; j < FWD_TILE; ++j) {
            const TriF32& T = tile[st][j];
            const uint32_t P = unx * T.U[0] + uny * T.U[1] + unz * T.U[2];
            const float ph = (float)(int32_t)P * kTwoPiOver2p32;
            const float a = xx * T.e21x + xy * T.e21y + xz * T.e21z;
            const float b = xx * T.e31x + xy * T.e31y + xz * T.e31z;
            TriLocal<float, false> o;
            tri_local<float, false>(a, b, o);
            float sp, cp;
            __sincosf(ph, &sp, &cp);
            const Cx<float> r = cmul(Cx<float>{cp, -sp}, o.rho);
            const Cx<float> f = cmul(r, o.f);
            const float w = MODE == 0 ? T.w0 : xx * T.w0 + xy * T.w1 + xz * T.w2;
            px += w * f.x;
            py += w * f.y;
        }
        kahan_add(accx, cx, px);
        kahan_add(accy, cy, py);
        __syncthreads();
    }
    if (!active) return;
    if (MODE == 1) {
        // volume: S = (i / |xi|^2) sum_T (xi . n_T) f_T, and the enclosed volume at xi = 0
        const float k2 = xx * xx + xy * xy + xz * xz;
        if (nx == 0 && ny == 0 && nz == 0) {
            accx = (float)*d_vol;
            accy = 0.f;
        } else {
            const float ik2 = 1.0f / k2;
            const float tx = -accy * ik2, ty = accx * ik2;
            accx = tx;
            accy = ty;
        }
    }
    S[m] = make_float2(accx, accy);
}

template <int MODE>
__global__ void __launch_bounds__(ADJ_THREADS) k_adj_f32(const TriF32* __restrict__ tris, int64_t n_t,
                                                         int64_t n_t_pad, const FreqF32* __restrict__ fr,
                                                         const int64_t* __restrict__ dM, int64_t M_max,
                                                         int tiles_per_chunk, float* __restrict__ partial,
                                                         int* __restrict__ err) {
    constexpr int NACC = MODE == 0 ? NACC_SURF : NACC_VOL;
    __shared__ __align__(128) FreqF32 tile[2][ADJ_FTILE];
    __shared__ __align__(8) uint64_t bar[2];
    const int tid = threadIdx.x;
    const int64_t t = (int64_t)blockIdx.x * ADJ_THREADS + tid;
    const int64_t M = dM ? *dM : M_max;
    const int n_ftiles = (int)((M + ADJ_FTILE - 1) / ADJ_FTILE);
    const int f0 = blockIdx.y * tiles_per_chunk;
    const int f1 = min(f0 + tiles_per_chunk, n_ftiles);

    const TriF32 T = tris[t < n_t_pad ? t : 0];
    float tot[NACC], comp[NACC];
#pragma unroll
    for (int k = 0; k < NACC; ++k) tot[k] = comp[k] = 0.f;

    if (f1 > f0) {
        constexpr uint32_t kTileBytes = ADJ_FTILE * sizeof(FreqF32);
        if (tid == 0) {
            mbar_init(&bar[0], 1);
            mbar_init(&bar[1], 1);
            mbar_fence_init();
        }
        __syncthreads();
        if (tid == 0) {
            mbar_arrive_expect_tx(&bar[0], kTileBytes);
            bulk_g2s(&tile[0][0], fr + (int64_t)f0 * ADJ_FTILE, kTileBytes, &bar[0]);
        }
        for (int ft = f0; ft < f1; ++ft) {
            const int i = ft - f0;
            const int st = i & 1;
            if (tid == 0 && ft + 1 < f1) {
                fence_proxy_async_smem();
                mbar_arrive_expect_tx(&bar[st ^ 1], kTileBytes);
                bulk_g2s(&tile[st ^ 1][0], fr + (int64_t)(ft + 1) * ADJ_FTILE, kTileBytes, &bar[st ^ 1]);
            }
            const bool ok = mbar_wait_bounded(&bar[st], (i >> 1) & 1, kWaitLimitNs);
            if (__syncthreads_or(!ok)) {
                if (tid == 0) {
                    atomicOr(err, ERR_TIMEOUT);
                    mbar_wait_bounded(&bar[st], (i >> 1) & 1, kWaitLimitNs);
                    if (ft + 1 < f1) mbar_wait_bounded(&bar[st ^ 1], ((i + 1) >> 1) & 1, kWaitLimitNs);
                }
                return;
            }
            float part[NACC];
#pragma unroll
            for (int k = 0; k < NACC; ++k) part[k] = 0.f;
#pragma unroll 1
            for (int j = 0; j < ADJ_FTILE; ++j) {
                const FreqF32& Fq = tile[st][j];
                const uint32_t P = (uint32_t)Fq.n[0] * T.U[0] + (uint32_t)Fq.n[1] * T.U[1] + (uint32_t)Fq.n[2] * T.U[2];
                const float ph = (float)(int32_t)P * kTwoPiOver2p32;
                const float xx = Fq.xi[0], xy = Fq.xi[1], xz = Fq.xi[2];
                const float a = xx * T.e21x + xy * T.e21y + xz * T.e21z;
                const float b = xx * T.e31x + xy * T.e31y + xz * T.e31z;
                TriLocal<float, true> o;
                tri_local<float, true>(a, b, o);
                float sp, cp;
                __sincosf(ph, &sp, &cp);
                const Cx<float> r = cmul(Cx<float>{cp, -sp}, o.rho);
                const Cx<float> H = cmul(Cx<float>{Fq.Gr, -Fq.Gi}, r);  // conj(Gw) exp(-i phi1) rho
                const float rf = re_mul(H, o.f);
                const float t0 = re_mul(H, o.D[0]), t1 = re_mul(H, o.D[1]), t2 = re_mul(H, o.D[2]);
                const float tv1 = sel3(o.p1, t0, t1, t2);
                const float tlo = sel3(o.plo, t0, t1, t2);
                const float thi = sel3(o.phi, t0, t1, t2);
                float tv2 = o.ab ? tlo : thi;
                float tv3 = o.ab ? thi : tlo;
                float tw1 = tv1;
                if (MODE == 0) {
                    part[0] += rf;
                } else {
                    const float wn = xx * T.w0 + xy * T.w1 + xz * T.w2;  // xi . n_T
                    part[0] += rf * xx;
                    part[1] += rf * xy;
                    part[2] += rf * xz;
                    tw1 *= wn;
                    tv2 *= wn;
                    tv3 *= wn;
                }
                constexpr int B = MODE == 0 ? 1 : 3;
                part[B + 0] += tw1 * xx;
                part[B + 1] += tw1 * xy;
                part[B + 2] += tw1 * xz;
                part[B + 3] += tv2 * xx;
                part[B + 4] += tv2 * xy;
                part[B + 5] += tv2 * xz;
                part[B + 6] += tv3 * xx;
                part[B + 7] += tv3 * xy;
                part[B + 8] += tv3 * xz;
            }
#pragma unroll
            for (int k = 0; k < NACC; ++k) kahan_add(tot[k], comp[k], part[k]);
            __syncthreads();
        }
    }
    if (t < n_t_pad) {
        float* out = partial + (int64_t)blockIdx.y * NACC * n_t_pad + t;
#pragma unroll
        for (int k = 0; k < NACC; ++k) out[(int64_t)k * n_t_pad] = t < n_t ? tot[k] : 0.f;
    }
}

}  // namespace

cudaError_t launch_fwd_f32(int mode, const TriF32* tris, int64_t n_t_pad, const FreqSrc& fs, const Geom& g,
                           const double* d_vol, float2* S, int* d_err, cudaStream_t st) {
    const int n_tiles = (int)(n_t_pad / FWD_TILE);
    const float tpx = (float)(2.0 * M_PI / g.L[0]), tpy = (float)(2.0 * M_PI / g.L[1]),
                tpz = (float)(2.0 * M_PI / g.L[2]);
    const int64_t blocks = (fs.M + FWD_THREADS - 1) / FWD_THREADS;
    if (blocks <= 0 || n_tiles <= 0) return cudaSuccess;
    const dim3 grid((unsigned)blocks);
    const bool ex = fs.nlist != nullptr;
    if (mode == 0 && !ex) k_fwd_f32<0, false><<<grid, FWD_THREADS, 0, st>>>(tris, n_tiles, fs, tpx, tpy, tpz, d_vol, S, d_err);
    if (mode == 0 && ex) k_fwd_f32<0, true><<<grid, FWD_THREADS, 0, st>>>(tris, n_tiles, fs, tpx, tpy, tpz, d_vol, S, d_err);
    if (mode == 1 && !ex) k_fwd_f32<1, false><<<grid, FWD_THREADS, 0, st>>>(tris, n_tiles, fs, tpx, tpy, tpz, d_vol, S, d_err);
    if (mode == 1 && ex) k_fwd_f32<1, true><<<grid, FWD_THREADS, 0, st>>>(tris, n_tiles, fs, tpx, tpy, tpz, d_vol, S, d_err);
    return cudaGetLastError();
}

int adj_chunks_f32(int64_t n_t, int64_t M_max, int sm_count) {
    const int64_t tblocks = (n_t + ADJ_THREADS - 1) / ADJ_THREADS;
    const int64_t ftiles = (M_max + ADJ_FTILE - 1) / ADJ_FTILE;
    const int64_t target = (int64_t)sm_count * 8;  // enough resident blocks to fill every SM
    int64_t c = (target + tblocks - 1) / tblocks;
    if (c < 1) c = 1;
    if (c > ftiles) c = ftiles;
    if (c > 65535) c = 65535;
    return (int)(c < 1 ? 1 : c);
}

cudaError_t launch_adj_f32(int mode, const TriF32* tris, int64_t n_t, int64_t n_t_pad, const FreqF32* fr,
                           const int64_t* dM, int64_t M_max, float* partial, int n_chunks, int* d_err, cudaStream_t st) {
    const int64_t ftiles = (M_max + ADJ_FTILE - 1) / ADJ_FTILE;
    const int tpc = (int)((ftiles + n_chunks - 1) / n_chunks);
    const dim3 grid((unsigned)(n_t_pad / ADJ_THREADS), (unsigned)n_chunks);
    if (mode == 0)
        k_adj_f32<0><<<grid, ADJ_THREADS, 0, st>>>(tris, n_t, n_t_pad, fr, dM, M_max, tpc, partial, d_err);
    else
        k_adj_f32<1><<<grid, ADJ_THREADS, 0, st>>>(tris, n_t, n_t_pad, fr, dM, M_max, tpc, partial, d_err);
    return cudaGetLastError();
}

}  // namespace dm
