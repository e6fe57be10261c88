// Optimiser layer of the staggered fit (Section 5.1-5.2): the combinatorial mesh
// Laplacian, the smoothing solve (1 + lambda L) X = B of the large-steps update,
// the uniform-Adam step, and the Cholesky parameterisation Sigma = C C^T of the
// PSF covariance.
//
// The smoothing solve is Jacobi-preconditioned conjugate gradients with one CTA
// per coordinate: the system is small (n_v ~ 1e3-1e4) and fixed for a whole fit,
// each iteration is one sparse product and two block reductions, and one CTA
// keeps the iterate, residual, search direction, product and inverse diagonal in
// shared memory whenever 5 n_v values fit (10,000+ vertices in FP32). There is no
// inter-CTA waiting anywhere.
#include <atomic>
#include <cmath>
#include <cstdint>

#include "dm_kernels.cuh"

namespace dm {
namespace {

constexpr int OT = 256;         // threads of the element-wise kernels
constexpr int PCG_T = 1024;     // threads of a PCG CTA
constexpr int PCG_RED = 128;    // reduction scratch (values of type R) at the start of shared memory

inline unsigned oblk(int64_t n) { return (unsigned)((n + OT - 1) / OT); }

// ----------------------------------------------------------------- Laplacian
// Row v lists the unique neighbours of v: the other two corners of every triangle in v's
// star (corner entries e = 3 t + p, sorted), first occurrences only, then sorted.
__device__ __forceinline__ int32_t star_candidate(const int32_t* __restrict__ F, const int32_t* __restrict__ ent,
                                                  int32_t k) {
    const int32_t e = ent[k >> 1];
    const int32_t t = e / 3, p = e - 3 * t;
    const int32_t q = (k & 1) ? (p == 0 ? 2 : p - 1) : (p == 2 ? 0 : p + 1);
    return F[3 * t + q];
}

__global__ void __launch_bounds__(OT) k_lap_rows(const int32_t* __restrict__ F, const int32_t* __restrict__ sptr,
                                                 const int32_t* __restrict__ ent, int64_t n_v,
                                                 const int32_t* __restrict__ lptr, int32_t* __restrict__ cnt,
                                                 int32_t* __restrict__ col, int* err) {
    const int64_t v = (int64_t)blockIdx.x * OT + threadIdx.x;
    if (v >= n_v) return;
    const int32_t k0 = 2 * sptr[v], k1 = 2 * sptr[v + 1];
    int32_t n = 0;
    int32_t w = lptr ? lptr[v] : 0;
    for (int32_t k = k0; k < k1; ++k) {
        const int32_t u = star_candidate(F, ent, k);
        if (u < 0 || u >= n_v) {
            atomicOr(err, ERR_BAD_INDEX);
            continue;
        }
        if (u == v) continue;
        bool seen = false;
        for (int32_t j = k0; j < k && !seen; ++j) seen = star_candidate(F, ent, j) == u;
        if (seen) continue;
        if (lptr) col[w++] = u;
        ++n;
    }
    if (!lptr) {
        cnt[v] = n;
        return;
    }
    // sort the row so that every sum over it has a fixed order
    const int32_t b = lptr[v];
    for (int32_t i = b + 1; i < b + n; ++i) {
        const int32_t x = col[i];
        int32_t j = i - 1;
        while (j >= b && col[j] > x) {
            col[j + 1] = col[j];
            --j;
        }
        col[j + 1] = x;
    }
}

// ----------------------------------------------------------------- PCG
template <class R>
struct PcgArgs {
    const int32_t* lp;
    const int32_t* lc;
    int64_t n_v;
    double lam;
    const double* b;   // [n_v][3]
    double* x;         // [n_v][3] start in, solution out
    double* sub_into;  // nullable: sub_into -= x on exit
    R* work;           // [3][5][n_v] when the vectors do not fit in shared memory
    int use_smem;
    double tol;
    int max_iter;
    unsigned long long* stats;  // [0] total iterations, [1] most in one solve, [2] unconverged solves
};

template <class R>
__device__ __forceinline__ R warp_sum_r(R v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Sum of NV values over the CTA; every thread returns the totals.
template <class R, int NV>
__device__ __forceinline__ void cta_sum(R (&a)[NV], R* red) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k) a[k] = warp_sum_r(a[k]);
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < NV; ++k) red[32 * k + wid] = a[k];
    __syncthreads();
    if (wid == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            R s = red[32 * k + lane];
            s = warp_sum_r(s);
            if (lane == 0) red[96 + k] = s;
        }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < NV; ++k) a[k] = red[96 + k];
    __syncthreads();
}

// (1 + lam L) p at row i; the row's degree comes with its bounds.
template <class R>
__device__ __forceinline__ R apply_row(const int32_t* __restrict__ lp, const int32_t* __restrict__ lc, const R* p,
                                       int64_t i, R lam) {
    const int32_t b = lp[i], e = lp[i + 1];
    R s = 0;
    for (int32_t k = b; k < e; ++k) s += p[lc[k]];
    return (R(1) + lam * (R)(e - b)) * p[i] - lam * s;
}

template <class R>
__global__ void __launch_bounds__(PCG_T) k_pcg(PcgArgs<R> a) {
    extern __shared__ __align__(16) unsigned char pcg_smem[];
    R* red = reinterpret_cast<R*>(pcg_smem);
    const int c = blockIdx.x;
    const int64_t n = a.n_v;
    R* base = a.use_smem ? red + PCG_RED : a.work + (int64_t)c * 5 * n;
    R* xs = base;
    R* r = base + n;
    R* p = base + 2 * n;
    R* q = base + 3 * n;
    R* dinv = base + 4 * n;
    const R lam = (R)a.lam;

    for (int64_t i = threadIdx.x; i < n; i += PCG_T) {
        xs[i] = (R)a.x[3 * i + c];
        dinv[i] = R(1) / (R(1) + lam * (R)(a.lp[i + 1] - a.lp[i]));
    }
    __syncthreads();
    R s3[3] = {0, 0, 0};  // ||b||^2, <r, z>, ||r||^2
    for (int64_t i = threadIdx.x; i < n; i += PCG_T) {
        const R bi = (R)a.b[3 * i + c];
        const R ri = bi - apply_row(a.lp, a.lc, xs, i, lam);
        const R zi = ri * dinv[i];
        r[i] = ri;
        p[i] = zi;
        s3[0] += bi * bi;
        s3[1] += ri * zi;
        s3[2] += ri * ri;
    }
    cta_sum<R, 3>(s3, red);  // also orders the writes of p before the first product
    const R bb = s3[0];
    R rz = s3[1], rr = s3[2];
    const R stop = (R)(a.tol * a.tol) * bb;
    int it = 0;
    if (bb == R(0)) {
        for (int64_t i = threadIdx.x; i < n; i += PCG_T) xs[i] = 0;
        rr = 0;
    }
    while (rr > stop && it < a.max_iter) {
        R pq[1] = {0};
        for (int64_t i = threadIdx.x; i < n; i += PCG_T) {
            const R qi = apply_row(a.lp, a.lc, p, i, lam);
            q[i] = qi;
            pq[0] += p[i] * qi;
        }
        cta_sum<R, 1>(pq, red);
        const R alpha = rz / pq[0];
        R s2[2] = {0, 0};
        for (int64_t i = threadIdx.x; i < n; i += PCG_T) {
            xs[i] += alpha * p[i];
            const R ri = r[i] - alpha * q[i];
            r[i] = ri;
            s2[0] += ri * ri * dinv[i];
            s2[1] += ri * ri;
        }
        cta_sum<R, 2>(s2, red);
        const R beta = s2[0] / rz;
        rz = s2[0];
        rr = s2[1];
        for (int64_t i = threadIdx.x; i < n; i += PCG_T) p[i] = r[i] * dinv[i] + beta * p[i];
        __syncthreads();
        ++it;
    }
    for (int64_t i = threadIdx.x; i < n; i += PCG_T) {
        const double xi = (double)xs[i];
        a.x[3 * i + c] = xi;
        if (a.sub_into) a.sub_into[3 * i + c] -= xi;
    }
    if (threadIdx.x == 0 && a.stats) {
        atomicAdd(&a.stats[0], (unsigned long long)it);
        atomicMax(&a.stats[1], (unsigned long long)it);
        if (rr > stop) atomicAdd(&a.stats[2], 1ull);
    }
}

// ----------------------------------------------------------------- uniform Adam
__global__ void __launch_bounds__(OT) k_au_moments(const double* __restrict__ g, double* __restrict__ m,
                                                   double* __restrict__ v, int64_t n, double b1, double b2,
                                                   double* __restrict__ part_max) {
    __shared__ double red[OT / 32];
    const int64_t i = (int64_t)blockIdx.x * OT + threadIdx.x;
    double vi = 0.0;
    if (i < n) {
        const double gi = g[i];
        m[i] = b1 * m[i] + (1.0 - b1) * gi;
        vi = b2 * v[i] + (1.0 - b2) * gi * gi;
        v[i] = vi;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) vi = fmax(vi, __shfl_xor_sync(0xffffffffu, vi, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = vi;
    __syncthreads();
    if (threadIdx.x == 0) {
        double mx = red[0];
        for (int w = 1; w < OT / 32; ++w) mx = fmax(mx, red[w]);
        part_max[blockIdx.x] = mx;
    }
}

__global__ void __launch_bounds__(OT) k_au_step(const double* __restrict__ m, const double* __restrict__ part_max,
                                                int nb, int64_t n, double lr, double b1, double b2, double eps,
                                                int64_t step, const int64_t* __restrict__ d_step, double decay,
                                                double* __restrict__ delta) {
    __shared__ double vmax_s;
    if (threadIdx.x < 32) {
        double mx = 0.0;
        for (int k = threadIdx.x; k < nb; k += 32) mx = fmax(mx, part_max[k]);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        if (threadIdx.x == 0) vmax_s = mx;
    }
    __syncthreads();
    const int64_t i = (int64_t)blockIdx.x * OT + threadIdx.x;
    if (i >= n) return;
    const double t = (double)(d_step ? *d_step : step);
    if (decay != 1.0) lr *= pow(decay, t - 1.0);  // step t takes the rate lr decay^(t-1)
    const double mh = m[i] / (1.0 - pow(b1, t));
    const double vh = vmax_s / (1.0 - pow(b2, t));
    delta[i] = lr * mh / (sqrt(vh) + eps);
}

// ----------------------------------------------------------------- Cholesky PSF
// C = (C00, C11, C22, C10, C20, C21); covariance numbers (xx, yy, zz, xy, xz, yz) at psf + 3.
__global__ void k_chol_to_cov(const double* __restrict__ C, double* __restrict__ psf) {
    if (threadIdx.x != 0) return;
    const double a = C[0], b = C[1], c = C[2], d = C[3], e = C[4], f = C[5];
    psf[3] = a * a;
    psf[4] = d * d + b * b;
    psf[5] = e * e + f * f + c * c;
    psf[6] = a * d;
    psf[7] = a * e;
    psf[8] = d * e + b * f;
}

// dL/dC = 2 G C on the lower triangle, G the symmetric gradient (half of each
// off-diagonal number in both of its places).
__global__ void k_chol_grad(const double* __restrict__ C, const double* __restrict__ gcov, double* __restrict__ gC) {
    if (threadIdx.x != 0) return;
    const double a = C[0], b = C[1], c = C[2], d = C[3], e = C[4], f = C[5];
    const double gxx = gcov[0], gyy = gcov[1], gzz = gcov[2], gxy = gcov[3], gxz = gcov[4], gyz = gcov[5];
    gC[0] = 2.0 * gxx * a + gxy * d + gxz * e;
    gC[1] = 2.0 * gyy * b + gyz * f;
    gC[2] = 2.0 * gzz * c;
    gC[3] = gxy * a + 2.0 * gyy * d + gyz * e;
    gC[4] = gxz * a + gyz * d + 2.0 * gzz * e;
    gC[5] = gyz * b + 2.0 * gzz * f;
}

}  // namespace

cudaError_t launch_laplacian(const int32_t* F, const int32_t* sptr, const int32_t* ent, int64_t n_v, int32_t* cnt,
                             int32_t* lptr, int32_t* lcol, int* d_err, cudaStream_t st) {
    k_lap_rows<<<oblk(n_v), OT, 0, st>>>(F, sptr, ent, n_v, nullptr, cnt, nullptr, d_err);
    cudaError_t e = launch_scan_i32(cnt, n_v, lptr, st);
    if (e != cudaSuccess) return e;
    k_lap_rows<<<oblk(n_v), OT, 0, st>>>(F, sptr, ent, n_v, lptr, cnt, lcol, d_err);
    return cudaGetLastError();
}

size_t pcg_work_elems(int64_t n_v) { return (size_t)15 * n_v; }

template <class R>
cudaError_t launch_pcg(const int32_t* lptr, const int32_t* lcol, int64_t n_v, double lam, const double* B, double* X,
                       double* sub_into, R* work, double tol, int max_iter, unsigned long long* stats,
                       cudaStream_t st) {
    int dev = 0, max_smem = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return e;
    const size_t want = (PCG_RED + 5 * (size_t)n_v) * sizeof(R);
    const bool smem = want <= (size_t)max_smem;
    const size_t bytes = smem ? want : PCG_RED * sizeof(R);
    // raise the kernel's dynamic shared-memory limit to the opt-in maximum once per device
    static std::atomic<int> raised[64];
    if (bytes > 48 * 1024 && (dev >= 64 || raised[dev].load() == 0)) {
        e = cudaFuncSetAttribute(k_pcg<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem);
        if (e != cudaSuccess) return e;
        if (dev < 64) raised[dev].store(1);
    }
    PcgArgs<R> a;
    a.lp = lptr;
    a.lc = lcol;
    a.n_v = n_v;
    a.lam = lam;
    a.b = B;
    a.x = X;
    a.sub_into = sub_into;
    a.work = work;
    a.use_smem = smem ? 1 : 0;
    a.tol = tol;
    a.max_iter = max_iter;
    a.stats = stats;
    k_pcg<R><<<3, PCG_T, bytes, st>>>(a);
    return cudaGetLastError();
}

template cudaError_t launch_pcg<float>(const int32_t*, const int32_t*, int64_t, double, const double*, double*, double*,
                                       float*, double, int, unsigned long long*, cudaStream_t);
template cudaError_t launch_pcg<double>(const int32_t*, const int32_t*, int64_t, double, const double*, double*,
                                        double*, double*, double, int, unsigned long long*, cudaStream_t);

int adam_uniform_partials(int64_t n) { return (int)oblk(n); }

cudaError_t launch_adam_uniform(const double* g, double* m, double* v, double* delta, int64_t n, double lr, double b1,
                                double b2, double eps, int64_t step, double* part_max, cudaStream_t st,
                                const int64_t* d_step, double decay) {
    const unsigned nb = oblk(n);
    k_au_moments<<<nb, OT, 0, st>>>(g, m, v, n, b1, b2, part_max);
    k_au_step<<<nb, OT, 0, st>>>(m, part_max, (int)nb, n, lr, b1, b2, eps, step, d_step, decay, delta);
    return cudaGetLastError();
}

cudaError_t launch_chol_to_cov(const double* C, double* d_psf, cudaStream_t st) {
    k_chol_to_cov<<<1, 32, 0, st>>>(C, d_psf);
    return cudaGetLastError();
}

cudaError_t launch_chol_grad(const double* C, const double* gcov, double* gC, cudaStream_t st) {
    k_chol_grad<<<1, 32, 0, st>>>(C, gcov, gC);
    return cudaGetLastError();
}

}  // namespace dm
