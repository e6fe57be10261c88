// Stage kernels around the two mesh-transform sums: triangle records, narrow band,
// transfer-function multiply, loss and residual, adjoint records, deterministic
// reductions, per-vertex assembly (Eq. 6 quotient rule) and Adam.
//
// Every reduction here is a fixed-order tree in FP64 (no floating-point atomics),
// so repeated runs are bitwise identical.
#include <cmath>

#include <algorithm>
#include <atomic>
#include <type_traits>

#include "dm_kernels.cuh"

namespace dm {

namespace {

constexpr int NT = 256;

// ---------------------------------------------------------------- triangle records
__device__ __forceinline__ void fixed32(double u, uint32_t& U) {
    u -= floor(u);
    U = (uint32_t)(uint64_t)llrint(u * 4294967296.0);  // 2^32 wraps to 0
}
__device__ __forceinline__ void fixed64(double u, uint64_t& U) {
    u -= floor(u);
    const double s = u * 4294967296.0;
    const double hi = floor(s);
    const double lo = (s - hi) * 4294967296.0;
    U = ((uint64_t)hi << 32) + (uint64_t)llrint(lo);
}

__device__ __forceinline__ void store_rec(TriF32& r, const double* v1, const double* e21, const double* e31,
                                          const double* w, const Geom& g) {
    for (int a = 0; a < 3; ++a) fixed32(v1[a] / g.L[a], r.U[a]);
    r.pad = 0;
    const auto dup = [](double v) { return make_float2((float)v, (float)v); };
    r.e21x = dup(e21[0]);
    r.e21y = dup(e21[1]);
    r.e21z = dup(e21[2]);
    r.e31x = dup(e31[0]);
    r.e31y = dup(e31[1]);
    r.e31z = dup(e31[2]);
    r.w0 = dup(w[0]);
    r.w1 = dup(w[1]);
    r.w2 = dup(w[2]);
    r.pad2 = make_float2(0.f, 0.f);
}
__device__ __forceinline__ void store_rec(TriF64& r, const double* v1, const double* e21, const double* e31,
                                          const double* w, const Geom& g) {
    for (int a = 0; a < 3; ++a) {
        fixed64(v1[a] / g.L[a], r.U[a]);
        r.e21[a] = e21[a];
        r.e31[a] = e31[a];
        r.w[a] = w[a];
    }
}

template <class Rec>
__device__ __forceinline__ void k_tri_prep_body(int mode, const double* __restrict__ V, int64_t n_v,
                                                 const int32_t* __restrict__ F, int64_t n_t,
                                                 const float* __restrict__ wts, Geom g, Rec* __restrict__ rec,
                                                 int64_t n_t_pad, double* __restrict__ partial, int* err, int64_t blk, int64_t nblk) {
    __shared__ double scratch[32];
    const int64_t t = blk * NT + threadIdx.x;
    double contrib = 0.0;
    if (t < n_t_pad) {
        Rec r;
        memset(&r, 0, sizeof(Rec));
        if (t < n_t) {
            const int32_t i0 = F[3 * t], i1 = F[3 * t + 1], i2 = F[3 * t + 2];
            const bool ok = i0 >= 0 && i0 < n_v && i1 >= 0 && i1 < n_v && i2 >= 0 && i2 < n_v;
            if (!ok) {
                atomicOr(err, ERR_BAD_INDEX);
            } else {
                double v[3][3];
                bool fin = true;
                for (int a = 0; a < 3; ++a) {
                    v[0][a] = V[3 * (int64_t)i0 + a] - g.origin[a];
                    v[1][a] = V[3 * (int64_t)i1 + a] - g.origin[a];
                    v[2][a] = V[3 * (int64_t)i2 + a] - g.origin[a];
                    fin = fin && isfinite(v[0][a]) && isfinite(v[1][a]) && isfinite(v[2][a]);
                }
                if (!fin) {
                    atomicOr(err, ERR_NONFINITE);
                } else {
                    double e21[3], e31[3], n[3], w[3];
                    for (int a = 0; a < 3; ++a) {
                        e21[a] = v[1][a] - v[0][a];
                        e31[a] = v[2][a] - v[0][a];
                    }
                    n[0] = e21[1] * e31[2] - e21[2] * e31[1];
                    n[1] = e21[2] * e31[0] - e21[0] * e31[2];
                    n[2] = e21[0] * e31[1] - e21[1] * e31[0];
                    if (mode == 0) {
                        const double A = 0.5 * sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
                        const double rho = wts ? (double)wts[t] : 1.0;
                        w[0] = 2.0 * A * rho;
                        w[1] = w[2] = 0.0;
                        contrib = rho * A;
                    } else {
                        w[0] = n[0];
                        w[1] = n[1];
                        w[2] = n[2];
                        // signed volume of the cone from the origin: v1 . (v2 x v3) / 6
                        contrib = (v[0][0] * (v[1][1] * v[2][2] - v[1][2] * v[2][1]) +
                                   v[0][1] * (v[1][2] * v[2][0] - v[1][0] * v[2][2]) +
                                   v[0][2] * (v[1][0] * v[2][1] - v[1][1] * v[2][0])) /
                                  6.0;
                    }
                    store_rec(r, v[0], e21, e31, w, g);
                }
            }
        }
        rec[t] = r;
    }
    const double s = block_sum<NT>(contrib, scratch);
    if (threadIdx.x == 0) partial[blk] = s;
}
template <class Rec>
__global__ void __launch_bounds__(NT) k_tri_prep(int mode, const double* __restrict__ V, int64_t n_v,
                                                 const int32_t* __restrict__ F, int64_t n_t,
                                                 const float* __restrict__ wts, Geom g, Rec* __restrict__ rec,
                                                 int64_t n_t_pad, double* __restrict__ partial, int* err) {
    k_tri_prep_body<Rec>(mode, V, n_v, F, n_t, wts, g, rec, n_t_pad, partial, err, (int64_t)blockIdx.x, (int64_t)gridDim.x);
}

// out[k] = sum_{b < n} x[b * count + k]  (one block per k, fixed order)
// err_nonpos (nullable): ERR_DEGENERATE is raised there when a sum is not > 0 (zero, negative, NaN).
__device__ __forceinline__ void k_sum_body(const double* __restrict__ x, int64_t n, int count, int k,
                                           double* __restrict__ out, int* __restrict__ err_nonpos) {
    __shared__ double scratch[32];
    double s = 0.0;
    for (int64_t b = threadIdx.x; b < n; b += 1024) s += x[b * count + k];
    s = block_sum<1024>(s, scratch);
    if (threadIdx.x == 0) {
        out[k] = s;
        if (err_nonpos && !(s > 0.0)) atomicOr(err_nonpos, ERR_DEGENERATE);
    }
}
__global__ void __launch_bounds__(1024) k_sum(const double* __restrict__ x, int64_t n, int count,
                                              double* __restrict__ out, int* __restrict__ err_nonpos) {
    k_sum_body(x, n, count, (int)blockIdx.x, out, err_nonpos);
}

// ---------------------------------------------------------------- narrow band
__device__ __forceinline__ double otf_expo(const double* psf, int kind, double x, double y, double z) {
    if (kind == 0) return psf[0] * psf[0] * x * x + psf[1] * psf[1] * y * y + psf[2] * psf[2] * z * z;
    const double* c = psf + 3;  // xx, yy, zz, xy, xz, yz
    return c[0] * x * x + c[1] * y * y + c[2] * z * z + 2.0 * (c[3] * x * y + c[4] * x * z + c[5] * y * z);
}

// h_hat(xi) in FP64 (the FP64 path).
template <class R>
__device__ __forceinline__ R otf_r(const double* psf, int kind, double x, double y, double z);
template <>
__device__ __forceinline__ double otf_r<double>(const double* psf, int kind, double x, double y, double z) {
    return exp(-0.5 * otf_expo(psf, kind, x, y, z));
}
// h_hat(xi) in FP32 (the FP32 images' own precision) from the PSF numbers rounded to FP32 (c[0..2]
// sigma, c[3..8] covariance, staged once per block): no per-frequency FP64 load or conversion.
__device__ __forceinline__ float otf_f(const float* c, int kind, float xf, float yf, float zf) {
    float e;
    if (kind == 0) {
        e = c[0] * c[0] * xf * xf + c[1] * c[1] * yf * yf + c[2] * c[2] * zf * zf;
    } else {
        e = c[3] * xf * xf + c[4] * yf * yf + c[5] * zf * zf +
            2.0f * (c[6] * xf * yf + c[7] * xf * zf + c[8] * yf * zf);
    }
    return expf(-0.5f * e);
}
// The 9 PSF numbers in the path's precision, in shared memory (threads 0..8; a barrier follows).
template <class R>
__device__ __forceinline__ void stage_psf(const double* __restrict__ psf, R* c) {
    if (threadIdx.x < 9) c[threadIdx.x] = (R)psf[threadIdx.x];
}

struct BandArgs {
    const double* psf;
    int kind;
    double tau;
    double e_max;  // -2 ln tau: h_hat > tau  <=>  xi^T Sigma xi < e_max
    float e_max_f;  // e_max in FP32
    float tpf[3];   // tp in FP32
    int Nx, Ny, Nz, Nzh;
    FastDiv div_zh, div_y;
    double tp[3];
    int64_t nH;
};

// h_hat(xi) > tau, decided on the exponent e = xi^T Sigma xi (no exp). The exponent is first formed in
// FP32 with a bound on its rounding error (at most a few units in the last place of each of its
// non-negative magnitude terms, counted with a wide factor); only a frequency whose FP32 exponent
// lies within that bound of the threshold is decided in FP64, as the FP64 oracle decides it (and,
// within rounding of the threshold, by the exp form as written). So the band is the oracle's,
// bit for bit, with FP64 arithmetic on a thin shell of frequencies only.
__device__ __forceinline__ bool in_band(const BandArgs& b, int64_t idx) {
    int nx, ny, nz;
    decode_h_fast((uint32_t)idx, b.div_zh, b.div_y, b.Nx, b.Ny, nx, ny, nz);
    const float x = (float)nx * b.tpf[0], y = (float)ny * b.tpf[1], z = (float)nz * b.tpf[2];
    float e32, mag;
    if (b.kind == 0) {
        const float s0 = (float)b.psf[0], s1 = (float)b.psf[1], s2 = (float)b.psf[2];
        e32 = s0 * s0 * x * x + s1 * s1 * y * y + s2 * s2 * z * z;
        mag = e32;
    } else {
        const double* c = b.psf + 3;
        const float c0 = (float)c[0], c1 = (float)c[1], c2 = (float)c[2], c3 = (float)c[3], c4 = (float)c[4],
                    c5 = (float)c[5];
        e32 = c0 * x * x + c1 * y * y + c2 * z * z + 2.0f * (c3 * x * y + c4 * x * z + c5 * y * z);
        mag = fabsf(c0) * x * x + fabsf(c1) * y * y + fabsf(c2) * z * z +
              2.0f * (fabsf(c3 * x * y) + fabsf(c4 * x * z) + fabsf(c5 * y * z));
    }
    const float bound = 32.0f * 5.96e-8f * (mag + b.e_max_f);  // 32 units of 2^-24, relative to the magnitudes
    if (fabsf(e32 - b.e_max_f) > bound) return e32 < b.e_max_f;
    const double e = otf_expo(b.psf, b.kind, nx * b.tp[0], ny * b.tp[1], nz * b.tp[2]);
    if (fabs(e - b.e_max) > 1e-9 * b.e_max) return e < b.e_max;
    return exp(-0.5 * e) > b.tau;
}

__global__ void __launch_bounds__(NT) k_band_count(BandArgs b, int64_t* __restrict__ counts) {
    const int64_t idx = (int64_t)blockIdx.x * NT + threadIdx.x;
    const int flag = idx < b.nH ? (int)in_band(b, idx) : 0;
    const int c = __syncthreads_count(flag);
    if (threadIdx.x == 0) counts[blockIdx.x] = c;
}

// In-place exclusive scan of n int64 values (one block); total into *total.
__global__ void __launch_bounds__(1024) k_scan_i64(int64_t* __restrict__ x, int64_t n, int64_t* __restrict__ total) {
    __shared__ int64_t part[1024];
    const int64_t per = (n + 1023) / 1024;
    const int64_t b0 = threadIdx.x * per, b1 = min(b0 + per, n);
    int64_t s = 0;
    for (int64_t i = b0; i < b1; ++i) s += x[i];
    part[threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        int64_t run = 0;
        for (int i = 0; i < 1024; ++i) {
            const int64_t v = part[i];
            part[i] = run;
            run += v;
        }
        if (total) *total = run;
    }
    __syncthreads();
    int64_t run = part[threadIdx.x];
    for (int64_t i = b0; i < b1; ++i) {
        const int64_t v = x[i];
        x[i] = run;
        run += v;
    }
}

__global__ void __launch_bounds__(NT) k_band_write(BandArgs b, const int64_t* __restrict__ offsets,
                                                   int32_t* __restrict__ idx_out) {
    __shared__ int warp_tot[NT / 32];
    const int64_t idx = (int64_t)blockIdx.x * NT + threadIdx.x;
    const bool flag = idx < b.nH && in_band(b, idx);
    const unsigned bal = __ballot_sync(0xffffffffu, flag);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) warp_tot[wid] = __popc(bal);
    __syncthreads();
    int before = 0;
    for (int w = 0; w < wid; ++w) before += warp_tot[w];
    before += __popc(bal & ((1u << lane) - 1u));
    if (flag) idx_out[offsets[blockIdx.x] + before] = (int32_t)idx;
}

// ---------------------------------------------------------------- transfer function and image
// Per-thread running sum in the path's precision: FP32 with a Kahan compensation in the FP32 path
// (B300's FP64 adds run at a small fraction of its FP32 rate, and these kernels add one term per
// element), plain FP64 in the FP64 path; blocks then combine the per-thread sums in FP64.
template <class R>
struct TSum;
template <>
struct TSum<float> {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float v) {
        const float y = v - c;
        const float t = s + y;
        c = (t - s) - y;
        s = t;
    }
    __device__ __forceinline__ double get() const { return (double)s - (double)c; }
};
template <>
struct TSum<double> {
    double s = 0.0;
    __device__ __forceinline__ void add(double v) { s += v; }
    __device__ __forceinline__ double get() const { return s; }
};
// Block sum of the threads' TSum values (result valid in thread 0; scratch >= 32 doubles).
template <int NT>
__device__ __forceinline__ double block_sum_t(const TSum<float>& p, double* scratch) {
    return block_sum_comp<NT>(p.s, p.c, scratch);
}
template <int NT>
__device__ __forceinline__ double block_sum_t(const TSum<double>& p, double* scratch) {
    return block_sum<NT>(p.s, scratch);
}

// Wavevector component of integer frequency n in the path's precision.
template <class R>
__device__ __forceinline__ R wave(int n, R tp) {
    return (R)n * tp;
}

template <class R>
__device__ __forceinline__ void k_scatter_body(const Cx<R>* __restrict__ S, FreqSrc fs, const double* __restrict__ psf,
                                                int kind, const double* __restrict__ d_norm, double tpx, double tpy,
                                                double tpz, double inv_VL, Cx<R>* __restrict__ spec, int64_t blk, int64_t nblk) {
    __shared__ R s_scale;  // one FP64 division per block, not per frequency
    __shared__ R s_c[9];
    if (threadIdx.x == 0) s_scale = (R)(inv_VL / *d_norm);
    stage_psf(psf, s_c);
    __syncthreads();
    const int64_t M = fs.dM ? *fs.dM : fs.M;
    // grid-stride, so that the per-block set-up above is paid by few blocks
    for (int64_t m = blk * NT + threadIdx.x; m < M; m += nblk * NT) {
        const int64_t idx = fs.idx ? (int64_t)fs.idx[m] : m;
        int nx, ny, nz;
        decode_h(idx, fs, nx, ny, nz);
        R hh;
        if constexpr (std::is_same<R, float>::value)
            hh = otf_f(s_c, kind, wave<R>(nx, (R)tpx), wave<R>(ny, (R)tpy), wave<R>(nz, (R)tpz));
        else
            hh = otf_r<R>(psf, kind, wave<R>(nx, (R)tpx), wave<R>(ny, (R)tpy), wave<R>(nz, (R)tpz));
        const R sc = hh * s_scale;
        const Cx<R> s = S[m];
        spec[idx] = Cx<R>{s.x * sc, s.y * sc};
    }
}
template <class R>
__global__ void __launch_bounds__(NT) k_scatter(const Cx<R>* __restrict__ S, FreqSrc fs, const double* __restrict__ psf,
                                                int kind, const double* __restrict__ d_norm, double tpx, double tpy,
                                                double tpz, double inv_VL, Cx<R>* __restrict__ spec) {
    k_scatter_body<R>(S, fs, psf, kind, d_norm, tpx, tpy, tpz, inv_VL, spec, (int64_t)blockIdx.x, (int64_t)gridDim.x);
}

template <class R>
__device__ __forceinline__ void k_loss_body(const R* __restrict__ I, const R* __restrict__ T, int64_t n, int kind,
                                             R* __restrict__ resid, double* __restrict__ partial, double inv_n, int64_t blk, int64_t nblk) {
    __shared__ double scratch[32];
    // per voxel in the path's precision R, per-thread sums as TSum, the block sum in FP64
    TSum<R> lsum;
    const R s = kind == 1 ? (R)(2.0 * inv_n) : (R)2;
    for (int64_t j = blk * NT + threadIdx.x; j < n; j += nblk * NT) {
        const R t = T[j];
        const R d = I[j] - t;
        const R w = kind == 2 ? t : (R)1;
        const R wd = w * d;
        lsum.add(wd * d);
        resid[j] = s * wd;
    }
    double l = block_sum_t<NT>(lsum, scratch);
    if (kind == 1) l *= inv_n;
    if (threadIdx.x == 0) partial[blk] = l;
}
template <class R>
__global__ void __launch_bounds__(NT) k_loss(const R* __restrict__ I, const R* __restrict__ T, int64_t n, int kind,
                                             R* __restrict__ resid, double* __restrict__ partial, double inv_n) {
    k_loss_body<R>(I, T, n, kind, resid, partial, inv_n, (int64_t)blockIdx.x, (int64_t)gridDim.x);
}

// Adjoint record of frequency m: lane m % 2 of pair record m / 2 (FP32), or record m (FP64).
__device__ __forceinline__ void set_rec(FreqPairF32* fr, int64_t m, int nx, int ny, int nz, double x, double y,
                                        double z, double gr, double gi) {
    FreqPairF32& r = fr[m >> 1];
    int32_t* n = (m & 1) ? r.nB : r.nA;
    n[0] = nx;
    n[1] = ny;
    n[2] = nz;
    float* lane = reinterpret_cast<float*>(&r.x) + (m & 1);  // x, y, z, Gr, Gi are consecutive float2
    lane[0] = (float)x;
    lane[2] = (float)y;
    lane[4] = (float)z;
    lane[6] = (float)gr;
    lane[8] = (float)gi;
}
__device__ __forceinline__ void set_rec(FreqPairF32* fr, int64_t m, int nx, int ny, int nz, float x, float y, float z,
                                        float gr, float gi) {
    FreqPairF32& r = fr[m >> 1];
    int32_t* n = (m & 1) ? r.nB : r.nA;
    n[0] = nx;
    n[1] = ny;
    n[2] = nz;
    float* lane = reinterpret_cast<float*>(&r.x) + (m & 1);
    lane[0] = x;
    lane[2] = y;
    lane[4] = z;
    lane[6] = gr;
    lane[8] = gi;
}
__device__ __forceinline__ void set_rec(FreqF64* fr, int64_t m, int nx, int ny, int nz, double x, double y, double z,
                                        double gr, double gi) {
    FreqF64& r = fr[m];
    r.n[0] = nx;
    r.n[1] = ny;
    r.n[2] = nz;
    r.pad = 0;
    r.xi[0] = x;
    r.xi[1] = y;
    r.xi[2] = z;
    r.Gr = gr;
    r.Gi = gi;
    r.pad2 = 0.0;
}
// The gather's record writes. FP32: lanes 2k and 2k + 1 of a warp hold frequencies A and B of one
// pair record and exchange halves, so that each writes 32 contiguous bytes with two 16-byte stores
// (all 32 lanes must call it). FP64: one record per lane.
__device__ __forceinline__ void put_rec(FreqPairF32* fr, int64_t m, int nx, int ny, int nz, float x, float y, float z,
                                        float gr, float gi) {
    const unsigned full = 0xffffffffu;
    const int ox = __shfl_xor_sync(full, nx, 1), oy = __shfl_xor_sync(full, ny, 1), oz = __shfl_xor_sync(full, nz, 1);
    const float px = __shfl_xor_sync(full, x, 1), py = __shfl_xor_sync(full, y, 1), pz = __shfl_xor_sync(full, z, 1);
    const float pgr = __shfl_xor_sync(full, gr, 1), pgi = __shfl_xor_sync(full, gi, 1);
    int4* r = reinterpret_cast<int4*>(fr + (m >> 1));
    if ((m & 1) == 0) {  // A: nA[3], nB[0] | nB[1], nB[2], x.A, x.B
        r[0] = make_int4(nx, ny, nz, ox);
        r[1] = make_int4(oy, oz, __float_as_int(x), __float_as_int(px));
    } else {  // B: y.A, y.B, z.A, z.B | Gr.A, Gr.B, Gi.A, Gi.B
        r[2] = make_int4(__float_as_int(py), __float_as_int(y), __float_as_int(pz), __float_as_int(z));
        r[3] = make_int4(__float_as_int(pgr), __float_as_int(gr), __float_as_int(pgi), __float_as_int(gi));
    }
}
__device__ __forceinline__ void put_rec(FreqF64* fr, int64_t m, int nx, int ny, int nz, double x, double y, double z,
                                        double gr, double gi) {
    set_rec(fr, m, nx, ny, nz, x, y, z, gr, gi);
}

// Partials per block: [0..5] dL/dpsf (3 used for kind DIAG), [6] coefficient of d(norm)/dv.
constexpr int NPART = 8;

template <class R, class FR>
__device__ __forceinline__ void k_gather_body(int mode, const Cx<R>* __restrict__ spec, const Cx<R>* __restrict__ S,
                                               FreqSrc fs, const double* __restrict__ psf, int kind,
                                               const double* __restrict__ d_norm, double tpx, double tpy, double tpz,
                                               double inv_VL, FR* __restrict__ fr, int64_t M_pad,
                                               double* __restrict__ partial, int64_t blk, int64_t nblk) {
    // Per frequency in the path's precision R; the sums over frequencies in FP64. Grid-stride over
    // the padded band, so each block reduces its partial sums once.
    __shared__ double scratch[7 * NT / 32];  // >= 32 doubles for the FP64 block sums
    static_assert(7 * NT / 32 >= 32 && NT >= 7, "k_gather's scratch serves block_sum_t (32) and 7 sums");
    __shared__ R s_rin;  // one FP64 division per block
    __shared__ R s_c[9];
    if (threadIdx.x == 0) s_rin = (R)(1.0 / *d_norm);
    stage_psf(psf, s_c);
    __syncthreads();
    const int64_t M = fs.dM ? *fs.dM : fs.M;
    const R rin = s_rin;
    const R cvl = (R)inv_VL;
    const R s0 = s_c[0], s1 = s_c[1], s2 = s_c[2];
    const R tx = (R)tpx, ty = (R)tpy, tz = (R)tpz;
    TSum<R> part[7];
    for (int64_t m = blk * NT + threadIdx.x; m < M_pad; m += nblk * NT) {
        // padding records (m >= M) are zeros; every lane of a warp runs the same iterations (M_pad
        // is a multiple of 256), as the paired record write below needs
        int nx = 0, ny = 0, nz = 0;
        R x = 0, y = 0, z = 0, wr = 0, wi = 0;
        if (m < M) {
            const int64_t idx = fs.idx ? (int64_t)fs.idx[m] : m;
            decode_h(idx, fs, nx, ny, nz);
            x = wave<R>(nx, tx);
            y = wave<R>(ny, ty);
            z = wave<R>(nz, tz);
            const R c = (nz == 0 || 2 * nz == fs.Nz) ? (R)1 : (R)2;
            const Cx<R> F = spec[idx];
            const R Gx = c * cvl * F.x, Gy = c * cvl * F.y;  // dL/dX
            R hh;
            if constexpr (std::is_same<R, float>::value)
                hh = otf_f(s_c, kind, x, y, z);
            else
                hh = otf_r<R>(psf, kind, x, y, z);
            const Cx<R> Sm = S[m];
            const R ux = Sm.x * rin, uy = Sm.y * rin;  // u_hat
            const R g = (Gx * ux + Gy * uy) * hh;      // Re(conj(G) X)
            if (kind == 0) {
                part[0].add(-g * s0 * x * x);
                part[1].add(-g * s1 * y * y);
                part[2].add(-g * s2 * z * z);
            } else {
                const R hg = (R)-0.5 * g;
                part[0].add(hg * x * x);
                part[1].add(hg * y * y);
                part[2].add(hg * z * z);
                part[3].add(-g * x * y);
                part[4].add(-g * x * z);
                part[5].add(-g * y * z);
            }
            R Gur = Gx * hh * rin, Gui = Gy * hh * rin;  // dL/du_hat / norm
            const bool zero = nx == 0 && ny == 0 && nz == 0;
            if (zero) {
                Gur = Gui = (R)0;  // u_hat(0) = 1 for every mesh: no gradient through xi = 0
            } else {
                part[6].add(-(Gur * ux + Gui * uy));  // -cq
            }
            wr = Gur;
            wi = Gui;
            if (mode == 1 && !zero) {  // volume: Gw = -i Gu / |xi|^2
                const R ik2 = (R)1 / (x * x + y * y + z * z);
                wr = Gui * ik2;
                wi = -Gur * ik2;
            }
        }
        put_rec(fr, m, nx, ny, nz, x, y, z, wr, wi);
    }
    if constexpr (std::is_same<R, float>::value) {
        float ps[7], pc[7];
#pragma unroll
        for (int k = 0; k < 7; ++k) {
            ps[k] = part[k].s;
            pc[k] = part[k].c;
        }
        const double v = block_sums_comp<NT, 7>(ps, pc, scratch);
        if (threadIdx.x < 7) partial[blk * NPART + threadIdx.x] = v;
    } else {
        for (int k = 0; k < 7; ++k) {
            const double v = block_sum_t<NT>(part[k], scratch);
            if (threadIdx.x == 0) partial[blk * NPART + k] = v;
        }
    }
    if (threadIdx.x == 0) partial[blk * NPART + 7] = 0.0;
}
template <class R, class FR>
__global__ void __launch_bounds__(NT) k_gather(int mode, const Cx<R>* __restrict__ spec, const Cx<R>* __restrict__ S,
                                               FreqSrc fs, const double* __restrict__ psf, int kind,
                                               const double* __restrict__ d_norm, double tpx, double tpy, double tpz,
                                               double inv_VL, FR* __restrict__ fr, int64_t M_pad,
                                               double* __restrict__ partial) {
    k_gather_body<R, FR>(mode, spec, S, fs, psf, kind, d_norm, tpx, tpy, tpz, inv_VL, fr, M_pad, partial, (int64_t)blockIdx.x, (int64_t)gridDim.x);
}

template <class R, class FR>
__global__ void __launch_bounds__(NT) k_prep_raw(int mode, const Cx<R>* __restrict__ G, const int32_t* __restrict__ nl,
                                                 int64_t M, double tpx, double tpy, double tpz, FR* __restrict__ fr,
                                                 int64_t M_pad, double* __restrict__ partial) {
    __shared__ double scratch[32];
    const int64_t m = (int64_t)blockIdx.x * NT + threadIdx.x;
    double k0 = 0.0;
    if (m < M) {
        const int nx = nl[3 * m], ny = nl[3 * m + 1], nz = nl[3 * m + 2];
        const double x = nx * tpx, y = ny * tpy, z = nz * tpz;
        double wr = (double)G[m].x, wi = (double)G[m].y;
        if (mode == 1) {
            if (nx == 0 && ny == 0 && nz == 0) {
                k0 = wr;  // S(0) = enclosed volume: its derivative goes through d(Vol)/dv
                wr = wi = 0.0;
            } else {
                const double ik2 = 1.0 / (x * x + y * y + z * z);
                const double tr = wi * ik2, ti = -wr * ik2;
                wr = tr;
                wi = ti;
            }
        }
        set_rec(fr, m, nx, ny, nz, x, y, z, wr, wi);
    } else if (m < M_pad) {
        set_rec(fr, m, 0, 0, 0, 0.0, 0.0, 0.0, 0.0, 0.0);
    }
    const double s = block_sum<NT>(k0, scratch);
    if (threadIdx.x == 0) {
        for (int k = 0; k < NPART; ++k) partial[blockIdx.x * NPART + k] = 0.0;
        partial[blockIdx.x * NPART + 6] = s;
    }
}

// acc[t][k] = sum over chunks c of partial[c][k][t]. A block covers 32 triangles (lanes) of one
// accumulator k (blockIdx.y) and one slice of the chunks (blockIdx.z of gridDim.z) with RC_WARPS
// warps: warp w adds the slice's chunks c = c0 + w, c0 + w + RC_WARPS, ... in that order into four
// interleaved sums, and warp 0 adds the warps' sums in warp order. With one slice the result goes to
// acc; with several (few triangles: too few blocks otherwise) each slice's sum goes to
// out_slices[slice][k][t] and k_reduce_slices adds the slices in order. The order is fixed by the
// chunk and slice counts alone, so the result is reproducible.
// M_max >= 0: the chunks cut the band's ADJ_FTILE tiles (the device count *dM when given, else
// M_max) into n_chunks runs of ceil(tiles / n_chunks); chunks past the last tile hold zeros and are
// left out.
constexpr int RC_WARPS = 16;
template <class R>
__device__ __forceinline__ void k_reduce_chunks_body(const R* __restrict__ partial, int n_chunks, int nacc,
                                                                 int64_t n_t, int64_t n_t_pad,
                                                                 double* __restrict__ acc,
                                                                 const int64_t* __restrict__ dM, int64_t M_max,
                                                                 double* __restrict__ out_slices, int bx, int by, int bz, int gz) {
    __shared__ double sh[RC_WARPS][32];
    const int slice_len = (n_chunks + gz - 1) / gz;
    if (M_max >= 0) {
        const int64_t M = dM ? *dM : M_max;
        const int64_t tiles = (M + ADJ_FTILE - 1) / ADJ_FTILE;
        const int64_t tpc = (tiles + n_chunks - 1) / n_chunks;
        n_chunks = tpc > 0 ? (int)min((int64_t)n_chunks, (tiles + tpc - 1) / tpc) : 0;
    }
    const int c0 = bz * slice_len;
    const int c1 = min(n_chunks, c0 + slice_len);
    const int lane = threadIdx.x, w = threadIdx.y;
    const int64_t t = (int64_t)bx * 32 + lane;
    const int k = by;
    const int64_t cs = (int64_t)nacc * n_t_pad;  // stride between chunks
    TSum<R> s0, s1, s2, s3;  // per-thread sums in the path's precision (compensated in FP32)
    if (t < n_t) {
        const R* p = partial + (int64_t)k * n_t_pad + t;
        int c = c0 + w;
        for (; c + 3 * RC_WARPS < c1; c += 4 * RC_WARPS) {
            s0.add(p[c * cs]);
            s1.add(p[(c + RC_WARPS) * cs]);
            s2.add(p[(c + 2 * RC_WARPS) * cs]);
            s3.add(p[(c + 3 * RC_WARPS) * cs]);
        }
        for (; c < c1; c += RC_WARPS) s0.add(p[c * cs]);
    }
    sh[w][lane] = (s0.get() + s1.get()) + (s2.get() + s3.get());
    __syncthreads();
    if (w == 0 && t < n_t) {
        double r = 0.0;
#pragma unroll
        for (int i = 0; i < RC_WARPS; ++i) r += sh[i][lane];
        if (gz == 1)
            acc[t * nacc + k] = r;
        else
            out_slices[((int64_t)bz * nacc + k) * n_t + t] = r;
    }
}
template <class R>
__global__ void __launch_bounds__(32 * RC_WARPS) k_reduce_chunks(const R* __restrict__ partial, int n_chunks, int nacc,
                                                                 int64_t n_t, int64_t n_t_pad,
                                                                 double* __restrict__ acc,
                                                                 const int64_t* __restrict__ dM, int64_t M_max,
                                                                 double* __restrict__ out_slices) {
    k_reduce_chunks_body<R>(partial, n_chunks, nacc, n_t, n_t_pad, acc, dM, M_max, out_slices, (int)blockIdx.x, (int)blockIdx.y, (int)blockIdx.z, (int)gridDim.z);
}

// acc[t][k] = sum over slices s (in order) of slices[s][k][t].
__device__ __forceinline__ void k_reduce_slices_body(const double* __restrict__ slices, int n_slices, int nacc,
                                                      int64_t n_t, double* __restrict__ acc, int64_t blk, int64_t nblk) {
    const int64_t i = blk * NT + threadIdx.x;
    if (i >= n_t * nacc) return;
    const int64_t k = i / n_t, t = i - k * n_t;
    double r = 0.0;
    for (int s = 0; s < n_slices; ++s) r += slices[((int64_t)s * nacc + k) * n_t + t];
    acc[t * nacc + k] = r;
}
__global__ void __launch_bounds__(NT) k_reduce_slices(const double* __restrict__ slices, int n_slices, int nacc,
                                                      int64_t n_t, double* __restrict__ acc) {
    k_reduce_slices_body(slices, n_slices, nacc, n_t, acc, (int64_t)blockIdx.x, (int64_t)gridDim.x);
}

// ---------------------------------------------------------------- gradient assembly
__device__ __forceinline__ void cross(const double* a, const double* b, double* o) {
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}

// contrib[t][p][3]: the corner (t, p) share of dL/dv_p (Eq. 6, 9).
__device__ __forceinline__ void k_assemble_body(int mode, const double* __restrict__ V, const int32_t* __restrict__ F,
                                                 int64_t n_t, int64_t n_v, const float* __restrict__ wts, Geom g,
                                                 const double* __restrict__ acc, const double* __restrict__ d_coef,
                                                 double* __restrict__ contrib, int64_t blk, int64_t nblk) {
    const int64_t t = blk * NT + threadIdx.x;
    if (t >= n_t) return;
    double out[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
    int32_t id[3] = {F[3 * t], F[3 * t + 1], F[3 * t + 2]};
    const bool ok = id[0] >= 0 && id[0] < n_v && id[1] >= 0 && id[1] < n_v && id[2] >= 0 && id[2] < n_v;
    if (ok) {
        double v[3][3];
        for (int p = 0; p < 3; ++p)
            for (int a = 0; a < 3; ++a) v[p][a] = V[3 * (int64_t)id[p] + a] - g.origin[a];
        double e[3][3];  // e1 = v3 - v2, e2 = v1 - v3, e3 = v2 - v1
        for (int a = 0; a < 3; ++a) {
            e[0][a] = v[2][a] - v[1][a];
            e[1][a] = v[0][a] - v[2][a];
            e[2][a] = v[1][a] - v[0][a];
        }
        const double coef = *d_coef;
        if (mode == 0) {
            const int NA = NACC_SURF;
            const double* ac = acc + t * NA;
            double n[3];
            cross(e[2], e[0], n);
            const double nn = sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
            const double A = 0.5 * nn;
            const double rho = wts ? (double)wts[t] : 1.0;
            double N[3] = {0, 0, 0};
            if (nn > 0)
                for (int a = 0; a < 3; ++a) N[a] = n[a] / nn;
            for (int p = 0; p < 3; ++p) {
                double w[3] = {0, 0, 0};
                if (nn > 0) cross(e[p], N, w);  // w_p = e_p x N
                for (int a = 0; a < 3; ++a)
                    out[p][a] = rho * (-w[a] * ac[0] + 2.0 * A * ac[1 + 3 * p + a]) + coef * (-0.5 * rho * w[a]);
            }
        } else {
            const int NA = NACC_VOL;
            const double* ac = acc + t * NA;
            const double alpha[3] = {ac[0], ac[1], ac[2]};
            for (int p = 0; p < 3; ++p) {
                double ax[3], dvol[3];
                cross(alpha, e[p], ax);
                cross(v[(p + 1) % 3], v[(p + 2) % 3], dvol);
                for (int a = 0; a < 3; ++a) out[p][a] = ax[a] + ac[3 + 3 * p + a] + coef * dvol[a] / 6.0;
            }
        }
    }
    for (int p = 0; p < 3; ++p)
        for (int a = 0; a < 3; ++a) contrib[(3 * t + p) * 3 + a] = out[p][a];
}
__global__ void __launch_bounds__(NT) k_assemble(int mode, const double* __restrict__ V, const int32_t* __restrict__ F,
                                                 int64_t n_t, int64_t n_v, const float* __restrict__ wts, Geom g,
                                                 const double* __restrict__ acc, const double* __restrict__ d_coef,
                                                 double* __restrict__ contrib) {
    k_assemble_body(mode, V, F, n_t, n_v, wts, g, acc, d_coef, contrib, (int64_t)blockIdx.x, (int64_t)gridDim.x);
}

__global__ void __launch_bounds__(NT) k_csr_count(const int32_t* __restrict__ F, int64_t n3, int64_t n_v,
                                                  int32_t* __restrict__ cnt, int* err) {
    const int64_t e = (int64_t)blockIdx.x * NT + threadIdx.x;
    if (e >= n3) return;
    const int32_t v = F[e];
    if (v >= 0 && v < n_v)
        atomicAdd(&cnt[v], 1);
    else
        atomicOr(err, ERR_BAD_INDEX);
}

__global__ void __launch_bounds__(1024) k_scan_i32(const int32_t* __restrict__ cnt, int64_t n,
                                                   int32_t* __restrict__ ptr) {
    __shared__ int32_t part[1024];
    const int64_t per = (n + 1023) / 1024;
    const int64_t b0 = threadIdx.x * per, b1 = min(b0 + per, n);
    int32_t s = 0;
    for (int64_t i = b0; i < b1; ++i) s += cnt[i];
    part[threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        int32_t run = 0;
        for (int i = 0; i < 1024; ++i) {
            const int32_t v = part[i];
            part[i] = run;
            run += v;
        }
        ptr[n] = run;
    }
    __syncthreads();
    int32_t run = part[threadIdx.x];
    for (int64_t i = b0; i < b1; ++i) {
        ptr[i] = run;
        run += cnt[i];
    }
}

__global__ void __launch_bounds__(NT) k_csr_fill(const int32_t* __restrict__ F, int64_t n3, int64_t n_v,
                                                 const int32_t* __restrict__ ptr, int32_t* __restrict__ cursor,
                                                 int32_t* __restrict__ ent) {
    const int64_t e = (int64_t)blockIdx.x * NT + threadIdx.x;
    if (e >= n3) return;
    const int32_t v = F[e];
    if (v < 0 || v >= n_v) return;
    const int32_t pos = atomicAdd(&cursor[v], 1);
    ent[ptr[v] + pos] = (int32_t)e;
}

// Sort each vertex's corner list so the per-vertex sum has a fixed order.
__global__ void __launch_bounds__(NT) k_csr_sort(const int32_t* __restrict__ ptr, int64_t n_v, int32_t* __restrict__ ent) {
    const int64_t v = (int64_t)blockIdx.x * NT + threadIdx.x;
    if (v >= n_v) return;
    const int32_t b = ptr[v], e = ptr[v + 1];
    for (int32_t i = b + 1; i < e; ++i) {
        const int32_t x = ent[i];
        int32_t j = i - 1;
        while (j >= b && ent[j] > x) {
            ent[j + 1] = ent[j];
            --j;
        }
        ent[j + 1] = x;
    }
}

__device__ __forceinline__ void k_vertex_gather_body(const int32_t* __restrict__ ptr, const int32_t* __restrict__ ent,
                                                      const double* __restrict__ contrib, int64_t n_v,
                                                      double* __restrict__ dV, int64_t blk, int64_t nblk) {
    const int64_t v = blk * NT + threadIdx.x;
    if (v >= n_v) return;
    double s0 = 0, s1 = 0, s2 = 0;
    for (int32_t i = ptr[v]; i < ptr[v + 1]; ++i) {
        const int64_t c = (int64_t)ent[i] * 3;
        s0 += contrib[c];
        s1 += contrib[c + 1];
        s2 += contrib[c + 2];
    }
    dV[3 * v] = s0;
    dV[3 * v + 1] = s1;
    dV[3 * v + 2] = s2;
}
__global__ void __launch_bounds__(NT) k_vertex_gather(const int32_t* __restrict__ ptr, const int32_t* __restrict__ ent,
                                                      const double* __restrict__ contrib, int64_t n_v,
                                                      double* __restrict__ dV) {
    k_vertex_gather_body(ptr, ent, contrib, n_v, dV, (int64_t)blockIdx.x, (int64_t)gridDim.x);
}

// ---------------------------------------------------------------- Adam
// One Adam update of element i; bc1 = 1 - b1^t and bc2 = 1 - b2^t are the bias corrections of step t.
__device__ __forceinline__ void adam_elem(double* __restrict__ p, const double* __restrict__ g, double* __restrict__ m,
                                          double* __restrict__ v, int64_t i, double lr, double b1, double b2,
                                          double eps, double bc1, double bc2) {
    const double gi = g[i];
    const double mi = b1 * m[i] + (1.0 - b1) * gi;
    const double vi = b2 * v[i] + (1.0 - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const double mh = mi / bc1;
    const double vh = vi / bc2;
    p[i] -= lr * mh / (sqrt(vh) + eps);
}

__global__ void __launch_bounds__(NT) k_adam(double* __restrict__ p, const double* __restrict__ g, double* __restrict__ m,
                                             double* __restrict__ v, int64_t n, double lr, double b1, double b2,
                                             double eps, int64_t step, const int64_t* __restrict__ d_step,
                                             double decay) {
    const int64_t i = (int64_t)blockIdx.x * NT + threadIdx.x;
    if (i >= n) return;
    const double t = (double)(d_step ? *d_step : step);
    if (decay != 1.0) lr *= pow(decay, t - 1.0);  // step t takes the rate lr decay^(t-1)
    adam_elem(p, g, m, v, i, lr, b1, b2, eps, 1.0 - pow(b1, t), 1.0 - pow(b2, t));
}

// End of one fit step: hist[t - step0 - 1] = loss of the step, then t += 1 (t: the Adam step on the
// device, so that one captured step replays unchanged).
__global__ void k_fit_tick(double* __restrict__ hist, const double* __restrict__ d_loss, int64_t* __restrict__ d_step,
                           int64_t step0) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        const int64_t t = *d_step;
        hist[t - step0 - 1] = *d_loss;
        *d_step = t + 1;
    }
}

__global__ void k_set_params(double* dst, Params16 p, int n) {
    if (threadIdx.x < n) dst[threadIdx.x] = p.v[threadIdx.x];
}

inline unsigned nblk(int64_t n) { return (unsigned)((n + NT - 1) / NT); }

// Blocks of NT threads of kernel FN that the current device holds at once (occupancy x SM count),
// looked up once per device and kernel.
template <auto FN>
cudaError_t one_wave(int* out) {
    static std::atomic<int> cache[64];
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    int w = dev < 64 ? cache[dev].load() : 0;
    if (w == 0) {
        int per_sm = 0, sms = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, FN, NT, 0);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
        w = std::max(1, per_sm) * std::max(1, sms);
        if (dev < 64) cache[dev].store(w);
    }
    *out = w;
    return cudaSuccess;
}

// ---------------------------------------------------------------- batched stages (fit server)
// Block b of a batched launch belongs to the largest job j with offs[j] <= b (offs[0] = 0 and offs[nj]
// = the launch's blocks; a job without blocks in the stage has offs[j] = offs[j + 1] and is never
// found), as its block b - offs[j] of offs[j + 1] - offs[j].
struct BatchBlock {
    int j;
    int64_t b, nb;
};
__device__ __forceinline__ BatchBlock batch_block(const int* __restrict__ offs, int nj) {
    const int b = (int)blockIdx.x;
    int lo = 0, hi = nj;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (offs[mid] <= b)
            lo = mid;
        else
            hi = mid;
    }
    return {lo, (int64_t)(b - offs[lo]), (int64_t)(offs[lo + 1] - offs[lo])};
}

__device__ __forceinline__ double two_pi_over(double L) { return 2.0 * M_PI / L; }

__global__ void __launch_bounds__(NT) kb_tri_prep(const StageJob* __restrict__ jobs, const int* __restrict__ offs,
                                                  int nj, int* err) {
    const BatchBlock q = batch_block(offs, nj);
    const StageJob& J = jobs[q.j];
    k_tri_prep_body<TriF32>(J.mode, J.V, J.n_v, J.F, J.n_t, J.wts, J.g, J.tris, J.n_t_pad, J.partial, err, q.b, q.nb);
}

// Zero the half spectrum of a narrow-band job (the scatter writes the band entries only).
__global__ void __launch_bounds__(NT) kb_zero(const StageJob* __restrict__ jobs, const int* __restrict__ offs, int nj) {
    const BatchBlock q = batch_block(offs, nj);
    const StageJob& J = jobs[q.j];
    float4* p = reinterpret_cast<float4*>(J.spec);
    const int64_t n4 = J.nH / 2;  // two complex values per float4
    for (int64_t i = q.b * NT + threadIdx.x; i < n4; i += q.nb * NT) p[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    if ((J.nH & 1) && q.b == 0 && threadIdx.x == 0) J.spec[J.nH - 1] = Cx<float>{0.f, 0.f};
}

__global__ void __launch_bounds__(NT) kb_scatter(const StageJob* __restrict__ jobs, const int* __restrict__ offs,
                                                 int nj) {
    const BatchBlock q = batch_block(offs, nj);
    const StageJob& J = jobs[q.j];
    const Geom g = J.g;
    k_scatter_body<float>((const Cx<float>*)J.S, J.fs, J.params, J.psf_kind, J.params + 16, two_pi_over(g.L[0]),
                          two_pi_over(g.L[1]), two_pi_over(g.L[2]), 1.0 / (g.L[0] * g.L[1] * g.L[2]), J.spec, q.b,
                          q.nb);
}

__global__ void __launch_bounds__(NT) kb_loss(const StageJob* __restrict__ jobs, const int* __restrict__ offs, int nj) {
    const BatchBlock q = batch_block(offs, nj);
    const StageJob& J = jobs[q.j];
    k_loss_body<float>(J.image, J.target, J.N, J.loss_kind, J.resid, J.partial, 1.0 / (double)J.N, q.b, q.nb);
}

__global__ void __launch_bounds__(NT) kb_gather(const StageJob* __restrict__ jobs, const int* __restrict__ offs,
                                                int nj) {
    const BatchBlock q = batch_block(offs, nj);
    const StageJob& J = jobs[q.j];
    const Geom g = J.g;
    k_gather_body<float, FreqPairF32>(J.mode, J.spec, (const Cx<float>*)J.S, J.fs, J.params, J.psf_kind,
                                      J.params + 16, two_pi_over(g.L[0]), two_pi_over(g.L[1]), two_pi_over(g.L[2]),
                                      1.0 / (g.L[0] * g.L[1] * g.L[2]), J.fr, J.M_pad, J.partial, q.b, q.nb);
}

// params[dst + k] = sum over the job's blocks b of the producing stage of partial[b * count + k]
// (block = (job, k), the single-job k_sum's order).
__global__ void __launch_bounds__(1024) kb_sum(const StageJob* __restrict__ jobs, const int* __restrict__ offs,
                                               int count, int dst, int* __restrict__ err_nonpos) {
    const int j = (int)blockIdx.x / count, k = (int)blockIdx.x - j * count;
    const StageJob& J = jobs[j];
    k_sum_body(J.partial, offs[j + 1] - offs[j], count, k, J.params + dst, err_nonpos);
}

// Chunk reduction: the job's blocks are its single-job grid (tb, nacc, slices) in x-fastest order.
__global__ void __launch_bounds__(32 * RC_WARPS) kb_reduce_chunks(const StageJob* __restrict__ jobs,
                                                                  const int* __restrict__ offs, int nj) {
    const BatchBlock q = batch_block(offs, nj);
    const StageJob& J = jobs[q.j];
    const int tb = (int)((J.n_t + 31) / 32);
    const int bx = (int)(q.b % tb), rest = (int)(q.b / tb);
    const int by = rest % J.nacc, bz = rest / J.nacc;
    k_reduce_chunks_body<float>(J.adjp, J.n_chunks, J.nacc, J.n_t, J.n_t_pad, J.acc, nullptr, -1, J.red, bx, by, bz,
                                J.rc_slices);
}

__global__ void __launch_bounds__(NT) kb_reduce_slices(const StageJob* __restrict__ jobs, const int* __restrict__ offs,
                                                       int nj) {
    const BatchBlock q = batch_block(offs, nj);
    const StageJob& J = jobs[q.j];
    k_reduce_slices_body(J.red, J.rc_slices, J.nacc, J.n_t, J.acc, q.b, q.nb);
}

__global__ void __launch_bounds__(NT) kb_assemble(const StageJob* __restrict__ jobs, const int* __restrict__ offs,
                                                  int nj) {
    const BatchBlock q = batch_block(offs, nj);
    const StageJob& J = jobs[q.j];
    k_assemble_body(J.mode, J.V, J.F, J.n_t, J.n_v, J.wts, J.g, J.acc, J.params + 30, J.contrib, q.b, q.nb);
}

__global__ void __launch_bounds__(NT) kb_vertex_gather(const StageJob* __restrict__ jobs, const int* __restrict__ offs,
                                                       int nj) {
    const BatchBlock q = batch_block(offs, nj);
    const StageJob& J = jobs[q.j];
    k_vertex_gather_body(J.ptr, J.ent, J.contrib, J.n_v, J.dV, q.b, q.nb);
}

// Split sums of the forward for the jobs with triangle splits: per element the order of the single-job
// k_fwd_reduce (compensated FP32 over the splits in order).
__global__ void __launch_bounds__(256) kb_fwd_reduce(const StageJob* __restrict__ jobs, const int* __restrict__ offs,
                                                     int nj) {
    const BatchBlock q = batch_block(offs, nj);
    const StageJob& J = jobs[q.j];
    const int64_t M = J.fs.dM ? *J.fs.dM : J.fs.M;
    for (int64_t m = q.b * 256 + threadIdx.x; m < M; m += q.nb * 256) {
        TSum<float> sx, sy;
        for (int ts = 0; ts < J.fsplits; ++ts) {
            const float2 v = J.S_part[(int64_t)ts * M + m];
            sx.add(v.x);
            sy.add(v.y);
        }
        J.S[m] = make_float2(sx.s, sy.s);
    }
}

// Adam on the vertices with the job's step t (on the device) and rate lr decay^(t-1).
__global__ void __launch_bounds__(NT) kb_adam(const StageJob* __restrict__ jobs, const int* __restrict__ offs, int nj) {
    const BatchBlock q = batch_block(offs, nj);
    const StageJob& J = jobs[q.j];
    const int64_t i = q.b * NT + threadIdx.x;
    if (i >= 3 * J.n_v) return;
    const double t = (double)*J.d_step;
    const double lr = J.decay != 1.0 ? J.lr_v * pow(J.decay, t - 1.0) : J.lr_v;
    adam_elem(J.V, J.dV, J.mV, J.vV, i, lr, J.b1, J.b2, J.eps, 1.0 - pow(J.b1, t), 1.0 - pow(J.b2, t));
}

// End of a step, one thread per job: Adam on sigma (lr_psf > 0) with the gradient params[24..26],
// the loss into the history and the engine's array, and the step counter advanced.
__global__ void kb_tick(const StageJob* __restrict__ jobs, int nj, double* __restrict__ losses) {
    const int j = (int)(blockIdx.x * blockDim.x + threadIdx.x);
    if (j >= nj) return;
    const StageJob& J = jobs[j];
    const int64_t step = *J.d_step;
    const double t = (double)step;
    if (J.lr_psf > 0) {
        const double lr = J.decay != 1.0 ? J.lr_psf * pow(J.decay, t - 1.0) : J.lr_psf;
        const double bc1 = 1.0 - pow(J.b1, t), bc2 = 1.0 - pow(J.b2, t);
        for (int a = 0; a < 3; ++a) adam_elem(J.params, J.params + 24, J.ms, J.vs, a, lr, J.b1, J.b2, J.eps, bc1, bc2);
    }
    const double L = J.params[17];
    J.hist[step - J.step0 - 1] = L;
    losses[j] = L;
    *J.d_step = step + 1;
}

}  // namespace

template <class Rec>
cudaError_t launch_tri_prep(int mode, const double* V, int64_t n_v, const int32_t* F, int64_t n_t, const float* wts,
                            const Geom& g, Rec* rec, int64_t n_t_pad, double* norm_partial, int* n_blocks_out,
                            int* d_err, cudaStream_t st) {
    const unsigned b = nblk(n_t_pad);
    *n_blocks_out = (int)b;
    k_tri_prep<Rec><<<b, NT, 0, st>>>(mode, V, n_v, F, n_t, wts, g, rec, n_t_pad, norm_partial, d_err);
    return cudaGetLastError();
}
template cudaError_t launch_tri_prep<TriF32>(int, const double*, int64_t, const int32_t*, int64_t, const float*,
                                             const Geom&, TriF32*, int64_t, double*, int*, int*, cudaStream_t);
template cudaError_t launch_tri_prep<TriF64>(int, const double*, int64_t, const int32_t*, int64_t, const float*,
                                             const Geom&, TriF64*, int64_t, double*, int*, int*, cudaStream_t);

cudaError_t launch_sum(const double* x, int64_t n, int stride, int count, double* out, cudaStream_t st) {
    (void)stride;
    k_sum<<<count, 1024, 0, st>>>(x, n, count, out, nullptr);
    return cudaGetLastError();
}

cudaError_t launch_norm_sum(const double* x, int64_t n, double* out, int* d_err, cudaStream_t st) {
    k_sum<<<1, 1024, 0, st>>>(x, n, 1, out, d_err);
    return cudaGetLastError();
}

cudaError_t launch_band(const double* d_psf, int psf_kind, double tau, int Nx, int Ny, int Nz, const Geom& g,
                        int32_t* idx, int64_t* dM, int64_t* block_counts, cudaStream_t st) {
    BandArgs b;
    b.psf = d_psf;
    b.kind = psf_kind;
    b.tau = tau;
    b.e_max = -2.0 * log(tau);
    b.e_max_f = (float)b.e_max;
    b.Nx = Nx;
    b.Ny = Ny;
    b.Nz = Nz;
    b.Nzh = Nz / 2 + 1;
    b.div_zh = make_fastdiv((uint32_t)b.Nzh);
    b.div_y = make_fastdiv((uint32_t)Ny);
    for (int a = 0; a < 3; ++a) {
        b.tp[a] = 2.0 * M_PI / g.L[a];
        b.tpf[a] = (float)b.tp[a];
    }
    b.nH = (int64_t)Nx * Ny * b.Nzh;
    const unsigned nb = nblk(b.nH);
    k_band_count<<<nb, NT, 0, st>>>(b, block_counts);
    k_scan_i64<<<1, 1024, 0, st>>>(block_counts, nb, dM);
    k_band_write<<<nb, NT, 0, st>>>(b, block_counts, idx);
    return cudaGetLastError();
}

template <class R>
cudaError_t launch_scatter(const Cx<R>* S, const FreqSrc& fs, const double* d_psf, int psf_kind, const double* d_norm,
                           const Geom& g, Cx<R>* spec, bool zero_first, cudaStream_t st) {
    const int64_t nH = (int64_t)fs.Nx * fs.Ny * fs.Nzh;
    if (zero_first) {
        cudaError_t e = cudaMemsetAsync(spec, 0, nH * sizeof(Cx<R>), st);
        if (e != cudaSuccess) return e;
    }
    const double VL = g.L[0] * g.L[1] * g.L[2];
    int wave = 0;
    const cudaError_t e = one_wave<k_scatter<R>>(&wave);  // grid-stride over one wave of resident blocks
    if (e != cudaSuccess) return e;
    const unsigned nb = (unsigned)std::min<int64_t>(nblk(fs.M), wave);
    k_scatter<R><<<nb, NT, 0, st>>>(S, fs, d_psf, psf_kind, d_norm, 2.0 * M_PI / g.L[0], 2.0 * M_PI / g.L[1],
                                            2.0 * M_PI / g.L[2], 1.0 / VL, spec);
    return cudaGetLastError();
}
template cudaError_t launch_scatter<float>(const Cx<float>*, const FreqSrc&, const double*, int, const double*,
                                           const Geom&, Cx<float>*, bool, cudaStream_t);
template cudaError_t launch_scatter<double>(const Cx<double>*, const FreqSrc&, const double*, int, const double*,
                                            const Geom&, Cx<double>*, bool, cudaStream_t);

template <class R>
cudaError_t launch_loss(const R* I, const R* T, int64_t n, int kind, R* resid, double* partial, int* n_blocks_out,
                        cudaStream_t st) {
    int wave = 0;
    const cudaError_t e = one_wave<k_loss<R>>(&wave);  // grid-stride over one wave of resident blocks
    if (e != cudaSuccess) return e;
    const int64_t b = std::min<int64_t>(nblk(n), std::min(wave, 4096));
    *n_blocks_out = (int)b;
    k_loss<R><<<(unsigned)b, NT, 0, st>>>(I, T, n, kind, resid, partial, 1.0 / (double)n);
    return cudaGetLastError();
}
template cudaError_t launch_loss<float>(const float*, const float*, int64_t, int, float*, double*, int*, cudaStream_t);
template cudaError_t launch_loss<double>(const double*, const double*, int64_t, int, double*, double*, int*,
                                         cudaStream_t);

template <class R, class FR>
cudaError_t launch_gather(int mode, const Cx<R>* spec, const Cx<R>* S, const FreqSrc& fs, const double* d_psf,
                          int psf_kind, const double* d_norm, const Geom& g, FR* fr, int64_t M_pad, double* partial,
                          int* n_blocks_out, cudaStream_t st) {
    if (M_pad % NT != 0) return cudaErrorInvalidValue;  // whole warps per iteration (paired record writes)
    // grid-stride over one wave of resident blocks: each block's seven reductions are paid once per
    // block slot (at 128^3 with 80 triangles 2048 blocks took 45 us, one wave of 592 27 us)
    int wave = 0;
    cudaError_t e = one_wave<k_gather<R, FR>>(&wave);
    if (e != cudaSuccess) return e;
    const unsigned b = (unsigned)std::min<int64_t>(nblk(M_pad), wave);
    *n_blocks_out = (int)b;
    const double VL = g.L[0] * g.L[1] * g.L[2];
    k_gather<R, FR><<<b, NT, 0, st>>>(mode, spec, S, fs, d_psf, psf_kind, d_norm, 2.0 * M_PI / g.L[0],
                                      2.0 * M_PI / g.L[1], 2.0 * M_PI / g.L[2], 1.0 / VL, fr, M_pad, partial);
    return cudaGetLastError();
}
template cudaError_t launch_gather<float, FreqF32>(int, const Cx<float>*, const Cx<float>*, const FreqSrc&,
                                                   const double*, int, const double*, const Geom&, FreqF32*, int64_t,
                                                   double*, int*, cudaStream_t);
template cudaError_t launch_gather<double, FreqF64>(int, const Cx<double>*, const Cx<double>*, const FreqSrc&,
                                                    const double*, int, const double*, const Geom&, FreqF64*, int64_t,
                                                    double*, int*, cudaStream_t);

template <class R, class FR>
cudaError_t launch_prep_raw(int mode, const Cx<R>* G, const int32_t* nlist, int64_t M, const Geom& g, FR* fr,
                            int64_t M_pad, double* partial, int* n_blocks_out, cudaStream_t st) {
    const unsigned b = nblk(M_pad);
    *n_blocks_out = (int)b;
    k_prep_raw<R, FR><<<b, NT, 0, st>>>(mode, G, nlist, M, 2.0 * M_PI / g.L[0], 2.0 * M_PI / g.L[1],
                                        2.0 * M_PI / g.L[2], fr, M_pad, partial);
    return cudaGetLastError();
}
template cudaError_t launch_prep_raw<float, FreqF32>(int, const Cx<float>*, const int32_t*, int64_t, const Geom&,
                                                     FreqF32*, int64_t, double*, int*, cudaStream_t);
template cudaError_t launch_prep_raw<double, FreqF64>(int, const Cx<double>*, const int32_t*, int64_t, const Geom&,
                                                      FreqF64*, int64_t, double*, int*, cudaStream_t);

template <class R>
cudaError_t launch_reduce_chunks(const R* partial, int n_chunks, int nacc, int64_t n_t, int64_t n_t_pad, double* acc,
                                 cudaStream_t st, const int64_t* dM, int64_t M_max, double* scratch, int sm_count) {
    if (n_t <= 0 || nacc <= 0) return cudaSuccess;
    const int64_t tb = (n_t + 31) / 32;
    // few triangles: split the chunks into slices so that about 4 blocks per SM run (the scratch
    // holds reduce_scratch_elems(sm_count) doubles, enough for slices * nacc * n_t at that count)
    const int64_t slices = scratch ? reduce_slices_for(n_t, nacc, n_chunks, sm_count) : 1;
    const dim3 grid((unsigned)tb, (unsigned)nacc, (unsigned)slices), block(32, RC_WARPS);
    k_reduce_chunks<R><<<grid, block, 0, st>>>(partial, n_chunks, nacc, n_t, n_t_pad, acc, dM, M_max, scratch);
    if (slices > 1) k_reduce_slices<<<nblk(n_t * nacc), NT, 0, st>>>(scratch, (int)slices, nacc, n_t, acc);
    return cudaGetLastError();
}
template cudaError_t launch_reduce_chunks<float>(const float*, int, int, int64_t, int64_t, double*, cudaStream_t,
                                                 const int64_t*, int64_t, double*, int);
template cudaError_t launch_reduce_chunks<double>(const double*, int, int, int64_t, int64_t, double*, cudaStream_t,
                                                  const int64_t*, int64_t, double*, int);

size_t reduce_scratch_elems(int sm_count) { return (size_t)256 * (sm_count > 0 ? sm_count : 1); }

cudaError_t launch_assemble(int mode, const double* V, const int32_t* F, int64_t n_t, int64_t n_v, const float* wts,
                            const Geom& g, const double* acc, const double* d_coef, double* contrib, cudaStream_t st) {
    k_assemble<<<nblk(n_t), NT, 0, st>>>(mode, V, F, n_t, n_v, wts, g, acc, d_coef, contrib);
    return cudaGetLastError();
}

cudaError_t launch_csr(const int32_t* F, int64_t n_t, int64_t n_v, int32_t* cnt, int32_t* ptr, int32_t* ent,
                       int* d_err, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(cnt, 0, n_v * sizeof(int32_t), st);
    if (e != cudaSuccess) return e;
    k_csr_count<<<nblk(3 * n_t), NT, 0, st>>>(F, 3 * n_t, n_v, cnt, d_err);
    k_scan_i32<<<1, 1024, 0, st>>>(cnt, n_v, ptr);
    e = cudaMemsetAsync(cnt, 0, n_v * sizeof(int32_t), st);
    if (e != cudaSuccess) return e;
    k_csr_fill<<<nblk(3 * n_t), NT, 0, st>>>(F, 3 * n_t, n_v, ptr, cnt, ent);
    k_csr_sort<<<nblk(n_v), NT, 0, st>>>(ptr, n_v, ent);
    return cudaGetLastError();
}

cudaError_t launch_scan_i32(const int32_t* cnt, int64_t n, int32_t* ptr, cudaStream_t st) {
    k_scan_i32<<<1, 1024, 0, st>>>(cnt, n, ptr);
    return cudaGetLastError();
}

cudaError_t launch_vertex_gather(const int32_t* ptr, const int32_t* ent, const double* contrib, int64_t n_v,
                                 double* dV, cudaStream_t st) {
    k_vertex_gather<<<nblk(n_v), NT, 0, st>>>(ptr, ent, contrib, n_v, dV);
    return cudaGetLastError();
}

cudaError_t launch_adam(double* p, const double* g, double* m, double* v, int64_t n, double lr, double b1, double b2,
                        double eps, int64_t step, cudaStream_t st) {
    k_adam<<<nblk(n), NT, 0, st>>>(p, g, m, v, n, lr, b1, b2, eps, step, nullptr, 1.0);
    return cudaGetLastError();
}
cudaError_t launch_adam_dev_step(double* p, const double* g, double* m, double* v, int64_t n, double lr, double b1,
                                 double b2, double eps, const int64_t* d_step, double decay, cudaStream_t st) {
    k_adam<<<nblk(n), NT, 0, st>>>(p, g, m, v, n, lr, b1, b2, eps, 0, d_step, decay);
    return cudaGetLastError();
}

cudaError_t launch_fit_tick(double* hist, const double* d_loss, int64_t* d_step, int64_t step0, cudaStream_t st) {
    k_fit_tick<<<1, 32, 0, st>>>(hist, d_loss, d_step, step0);
    return cudaGetLastError();
}

void batch_stage_blocks(const StageJob& J, int sm_count, int counts[BS_COUNT]) {
    int w_scatter = 0, w_loss = 0, w_gather = 0;
    one_wave<k_scatter<float>>(&w_scatter);
    one_wave<k_loss<float>>(&w_loss);
    one_wave<k_gather<float, FreqPairF32>>(&w_gather);
    for (int s = 0; s < BS_COUNT; ++s) counts[s] = 0;
    counts[BS_PREP] = (int)nblk(J.n_t_pad);
    counts[BS_FWDRED] = J.fsplits > 1 ? (int)std::min<int64_t>(nblk(J.nH), 4LL * sm_count) : 0;
    counts[BS_ZERO] = J.band ? (int)std::min<int64_t>(nblk((J.nH + 1) / 2), 8LL * sm_count) : 0;
    // the single-job launches' grids: one wave of resident blocks at most
    counts[BS_SCATTER] = (int)std::min<int64_t>(nblk(J.nH), std::max(1, w_scatter));
    counts[BS_LOSS] = (int)std::min<int64_t>(nblk(J.N), std::min(std::max(1, w_loss), 4096));
    counts[BS_GATHER] = (int)std::min<int64_t>(nblk(J.M_pad), std::max(1, w_gather));
    counts[BS_REDUCE] = (int)((J.n_t + 31) / 32) * J.nacc * J.rc_slices;
    counts[BS_SLICES] = J.rc_slices > 1 ? (int)nblk(J.n_t * J.nacc) : 0;
    counts[BS_ASSEMBLE] = (int)nblk(J.n_t);
    counts[BS_VGATHER] = (int)nblk(J.n_v);
    counts[BS_ADAM] = J.vertex_adam ? (int)nblk(3 * J.n_v) : 0;
}

int reduce_slices_for(int64_t n_t, int nacc, int n_chunks, int sm_count) {
    const int64_t tb = (n_t + 31) / 32;
    int64_t slices = 1;
    if (sm_count > 0 && tb * nacc < 4LL * sm_count) {
        slices = (4LL * sm_count + tb * nacc - 1) / (tb * nacc);
        slices = std::min<int64_t>(slices, std::max(1, n_chunks / (4 * RC_WARPS)));
        if (slices * nacc * n_t > (int64_t)reduce_scratch_elems(sm_count)) slices = 1;
    }
    return (int)slices;
}

cudaError_t launch_batch_stage(int stage, const StageJob* jobs, const int* offsets, int nj, int total, int* d_err,
                               cudaStream_t st) {
    if (total <= 0 || nj <= 0) return cudaSuccess;
    const int* o = offsets + (size_t)stage * (nj + 1);
    switch (stage) {
        case BS_PREP: kb_tri_prep<<<total, NT, 0, st>>>(jobs, o, nj, d_err); break;
        case BS_FWDRED: kb_fwd_reduce<<<total, 256, 0, st>>>(jobs, o, nj); break;
        case BS_ZERO: kb_zero<<<total, NT, 0, st>>>(jobs, o, nj); break;
        case BS_SCATTER: kb_scatter<<<total, NT, 0, st>>>(jobs, o, nj); break;
        case BS_LOSS: kb_loss<<<total, NT, 0, st>>>(jobs, o, nj); break;
        case BS_GATHER: kb_gather<<<total, NT, 0, st>>>(jobs, o, nj); break;
        case BS_REDUCE: kb_reduce_chunks<<<total, dim3(32, RC_WARPS), 0, st>>>(jobs, o, nj); break;
        case BS_SLICES: kb_reduce_slices<<<total, NT, 0, st>>>(jobs, o, nj); break;
        case BS_ASSEMBLE: kb_assemble<<<total, NT, 0, st>>>(jobs, o, nj); break;
        case BS_VGATHER: kb_vertex_gather<<<total, NT, 0, st>>>(jobs, o, nj); break;
        case BS_ADAM: kb_adam<<<total, NT, 0, st>>>(jobs, o, nj); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_batch_sum(const StageJob* jobs, const int* stage_offsets, int nj, int count, int dst, int* flag_err,
                             cudaStream_t st) {
    if (nj <= 0) return cudaSuccess;
    kb_sum<<<nj * count, 1024, 0, st>>>(jobs, stage_offsets, count, dst, flag_err);
    return cudaGetLastError();
}

cudaError_t launch_batch_tick(const StageJob* jobs, int nj, double* losses, cudaStream_t st) {
    if (nj <= 0) return cudaSuccess;
    kb_tick<<<(nj + 63) / 64, 64, 0, st>>>(jobs, nj, losses);
    return cudaGetLastError();
}

cudaError_t launch_set_params(double* dst, Params16 p, int n, cudaStream_t st) {
    k_set_params<<<1, 32, 0, st>>>(dst, p, n);
    return cudaGetLastError();
}

}  // namespace dm
