// Plain FP64 mesh Fourier transform and adjoint: the reference GPU path.
//
// Same mathematics as the FP32 kernels (meshft_math.cuh instantiated for double,
// with longer Taylor and series expansions and 64-bit fixed-point phases), but
// no shared-memory staging: each thread walks the triangle (or frequency) list
// straight from global memory. It is the "one fit at a time, FP64" comparator.
#include "dm_kernels.cuh"
#include "meshft_math.cuh"

namespace dm {

namespace {

constexpr double kTwoPiOver2p64 = 3.4061215800865545e-19;  // 2 pi / 2^64

template <int MODE, bool EXPLICIT>
__global__ void __launch_bounds__(F64_THREADS) k_fwd_f64(const TriF64* __restrict__ tris, int64_t n_t, FreqSrc fs,
                                                         double tpx, double tpy, double tpz,
                                                         const double* __restrict__ d_vol, double2* __restrict__ S) {
    const int64_t M = fs.dM ? *fs.dM : fs.M;
    const int64_t m = (int64_t)blockIdx.x * F64_THREADS + threadIdx.x;
    if (m >= M) return;
    int nx, ny, nz;
    if (EXPLICIT) {
        nx = fs.nlist[3 * m];
        ny = fs.nlist[3 * m + 1];
        nz = fs.nlist[3 * m + 2];
    } else {
        const int64_t idx = fs.idx ? (int64_t)fs.idx[m] : m;
        decode_h(idx, fs, nx, ny, nz);
    }
    const double xx = nx * tpx, xy = ny * tpy, xz = nz * tpz;
    const uint64_t unx = (uint64_t)(int64_t)nx, uny = (uint64_t)(int64_t)ny, unz = (uint64_t)(int64_t)nz;
    double accx = 0.0, accy = 0.0;
    for (int64_t t = 0; t < n_t; ++t) {
        const TriF64& T = tris[t];
        const uint64_t P = unx * T.U[0] + uny * T.U[1] + unz * T.U[2];
        const double ph = (double)(int64_t)P * kTwoPiOver2p64;
        const double a = xx * T.e21[0] + xy * T.e21[1] + xz * T.e21[2];
        const double b = xx * T.e31[0] + xy * T.e31[1] + xz * T.e31[2];
        TriLocal<double, false> o;
        tri_local<double, false>(a, b, o);
        double sp, cp;
        sincos(ph, &sp, &cp);
        const Cx<double> f = cmul(cmul(Cx<double>{cp, -sp}, o.rho), o.f);
        const double w = MODE == 0 ? T.w[0] : xx * T.w[0] + xy * T.w[1] + xz * T.w[2];
        accx += w * f.x;
        accy += w * f.y;
    }
    if (MODE == 1) {
        if (nx == 0 && ny == 0 && nz == 0) {
            accx = *d_vol;
            accy = 0.0;
        } else {
            const double ik2 = 1.0 / (xx * xx + xy * xy + xz * xz);
            const double tx = -accy * ik2, ty = accx * ik2;
            accx = tx;
            accy = ty;
        }
    }
    S[m] = make_double2(accx, accy);
}

template <int MODE>
__global__ void __launch_bounds__(F64_THREADS) k_adj_f64(const TriF64* __restrict__ tris, int64_t n_t,
                                                         const FreqF64* __restrict__ fr, const int64_t* __restrict__ dM,
                                                         int64_t M_max, int64_t per_chunk,
                                                         double* __restrict__ partial) {
    constexpr int NACC = MODE == 0 ? NACC_SURF : NACC_VOL;
    const int64_t t = (int64_t)blockIdx.x * F64_THREADS + threadIdx.x;
    if (t >= n_t) return;
    const int64_t M = dM ? *dM : M_max;
    const int64_t m0 = (int64_t)blockIdx.y * per_chunk;
    const int64_t m1 = min(m0 + per_chunk, M);
    const TriF64 T = tris[t];
    double acc[NACC];
#pragma unroll
    for (int k = 0; k < NACC; ++k) acc[k] = 0.0;
    for (int64_t m = m0; m < m1; ++m) {
        const FreqF64& Fq = fr[m];
        const uint64_t P = (uint64_t)(int64_t)Fq.n[0] * T.U[0] + (uint64_t)(int64_t)Fq.n[1] * T.U[1] +
                           (uint64_t)(int64_t)Fq.n[2] * T.U[2];
        const double ph = (double)(int64_t)P * kTwoPiOver2p64;
        const double xx = Fq.xi[0], xy = Fq.xi[1], xz = Fq.xi[2];
        const double a = xx * T.e21[0] + xy * T.e21[1] + xz * T.e21[2];
        const double b = xx * T.e31[0] + xy * T.e31[1] + xz * T.e31[2];
        TriLocal<double, true> o;
        tri_local<double, true>(a, b, o);
        double sp, cp;
        sincos(ph, &sp, &cp);
        const Cx<double> H = cmul(Cx<double>{Fq.Gr, -Fq.Gi}, cmul(Cx<double>{cp, -sp}, o.rho));
        const double rf = re_mul(H, o.f);
        const double t0 = re_mul(H, o.D[0]), t1 = re_mul(H, o.D[1]), t2 = re_mul(H, o.D[2]);
        double tv1 = sel3(o.p1, t0, t1, t2);
        const double tlo = sel3(o.plo, t0, t1, t2), thi = sel3(o.phi, t0, t1, t2);
        double tv2 = o.ab ? tlo : thi, tv3 = o.ab ? thi : tlo;
        if (MODE == 0) {
            acc[0] += rf;
        } else {
            const double wn = xx * T.w[0] + xy * T.w[1] + xz * T.w[2];
            acc[0] += rf * xx;
            acc[1] += rf * xy;
            acc[2] += rf * xz;
            tv1 *= wn;
            tv2 *= wn;
            tv3 *= wn;
        }
        constexpr int B = MODE == 0 ? 1 : 3;
        acc[B + 0] += tv1 * xx;
        acc[B + 1] += tv1 * xy;
        acc[B + 2] += tv1 * xz;
        acc[B + 3] += tv2 * xx;
        acc[B + 4] += tv2 * xy;
        acc[B + 5] += tv2 * xz;
        acc[B + 6] += tv3 * xx;
        acc[B + 7] += tv3 * xy;
        acc[B + 8] += tv3 * xz;
    }
    double* out = partial + (int64_t)blockIdx.y * NACC * n_t + t;
#pragma unroll
    for (int k = 0; k < NACC; ++k) out[(int64_t)k * n_t] = acc[k];
}

}  // namespace

cudaError_t launch_fwd_f64(int mode, const TriF64* tris, int64_t n_t, const FreqSrc& fs, const Geom& g,
                           const double* d_vol, double2* S, cudaStream_t st) {
    const double tpx = 2.0 * M_PI / g.L[0], tpy = 2.0 * M_PI / g.L[1], tpz = 2.0 * M_PI / g.L[2];
    const int64_t blocks = (fs.M + F64_THREADS - 1) / F64_THREADS;
    if (blocks <= 0) return cudaSuccess;
    const bool ex = fs.nlist != nullptr;
    const dim3 grid((unsigned)blocks);
    if (mode == 0 && !ex) k_fwd_f64<0, false><<<grid, F64_THREADS, 0, st>>>(tris, n_t, fs, tpx, tpy, tpz, d_vol, S);
    if (mode == 0 && ex) k_fwd_f64<0, true><<<grid, F64_THREADS, 0, st>>>(tris, n_t, fs, tpx, tpy, tpz, d_vol, S);
    if (mode == 1 && !ex) k_fwd_f64<1, false><<<grid, F64_THREADS, 0, st>>>(tris, n_t, fs, tpx, tpy, tpz, d_vol, S);
    if (mode == 1 && ex) k_fwd_f64<1, true><<<grid, F64_THREADS, 0, st>>>(tris, n_t, fs, tpx, tpy, tpz, d_vol, S);
    return cudaGetLastError();
}

int adj_chunks_f64(int64_t n_t, int64_t M_max, int sm_count) {
    const int64_t tblocks = (n_t + F64_THREADS - 1) / F64_THREADS;
    // ~64 (triangle block, chunk) units per SM so that the SMs finish together (the FP32 adjoint
    // lost 10% to the last, partly filled round of blocks at 8 units per SM)
    const int64_t target = (int64_t)sm_count * 64;
    int64_t c = (target + tblocks - 1) / tblocks;
    if (c < 1) c = 1;
    if (c > M_max) c = M_max > 0 ? M_max : 1;
    if (c > 65535) c = 65535;
    return (int)c;
}

cudaError_t launch_adj_f64(int mode, const TriF64* tris, int64_t n_t, const FreqF64* fr, const int64_t* dM,
                           int64_t M_max, double* partial, int n_chunks, cudaStream_t st) {
    const int64_t per = (M_max + n_chunks - 1) / n_chunks;
    const dim3 grid((unsigned)((n_t + F64_THREADS - 1) / F64_THREADS), (unsigned)n_chunks);
    if (mode == 0)
        k_adj_f64<0><<<grid, F64_THREADS, 0, st>>>(tris, n_t, fr, dM, M_max, per, partial);
    else
        k_adj_f64<1><<<grid, F64_THREADS, 0, st>>>(tris, n_t, fr, dM, M_max, per, partial);
    return cudaGetLastError();
}

}  // namespace dm
