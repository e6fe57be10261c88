// 3D real <-> half-spectrum DFTs for the image stage (the inverse transform that
// turns I_hat = u_hat h_hat into voxels, Eq. 1, and its adjoint).
//
// Each pass transforms every line along one axis. A block stages a batch of lines
// into shared memory (coalesced along the contiguous axis), runs a mixed-radix
// (2, 3, 4, 5) Stockham autosort FFT there (ping-pong buffers, one __syncthreads
// per radix stage), and writes the batch back. The z pass of the inverse builds
// the Hermitian-completed line (real parts of the self-conjugate n_z = 0 and
// Nyquist coefficients) before a complex inverse transform; the z pass of the
// forward keeps the first Nz/2+1 outputs. All transforms are unnormalised.
#include <cmath>

#include "dm_kernels.cuh"

namespace dm {

namespace {

constexpr int FFT_THREADS = 256;

template <class R>
__device__ __forceinline__ Cx<R> twiddle(const Cx<R>* tw, int idx, int dir) {
    const Cx<R> w = tw[idx];
    return dir < 0 ? w : Cx<R>{w.x, -w.y};
}

// y[m] = sum_q v[q] exp(dir 2 pi i q m / r), in place.
template <class R>
__device__ __forceinline__ void small_dft(Cx<R>* v, int r, int dir) {
    if (r == 2) {
        const Cx<R> a = v[0], b = v[1];
        v[0] = {a.x + b.x, a.y + b.y};
        v[1] = {a.x - b.x, a.y - b.y};
    } else if (r == 4) {
        const Cx<R> s02 = {v[0].x + v[2].x, v[0].y + v[2].y}, d02 = {v[0].x - v[2].x, v[0].y - v[2].y};
        const Cx<R> s13 = {v[1].x + v[3].x, v[1].y + v[3].y}, d13 = {v[1].x - v[3].x, v[1].y - v[3].y};
        // w = exp(dir i pi/2) = dir * i ;  w * d13 = dir * (-d13.y, d13.x)
        const Cx<R> wd = {-(R)dir * d13.y, (R)dir * d13.x};
        v[0] = {s02.x + s13.x, s02.y + s13.y};
        v[1] = {d02.x + wd.x, d02.y + wd.y};
        v[2] = {s02.x - s13.x, s02.y - s13.y};
        v[3] = {d02.x - wd.x, d02.y - wd.y};
    } else if (r == 3) {
        const R h = (R)0.86602540378443864676 * (R)dir;  // dir * sqrt(3)/2
        const Cx<R> t = {v[1].x + v[2].x, v[1].y + v[2].y}, d = {v[1].x - v[2].x, v[1].y - v[2].y};
        const Cx<R> m = {v[0].x - (R)0.5 * t.x, v[0].y - (R)0.5 * t.y};
        const Cx<R> id = {-h * d.y, h * d.x};  // i * h * d
        v[0] = {v[0].x + t.x, v[0].y + t.y};
        v[1] = {m.x + id.x, m.y + id.y};
        v[2] = {m.x - id.x, m.y - id.y};
    } else {  // r == 5: direct 5-point DFT
        const R c1 = (R)0.30901699437494742410, c2 = (R)-0.80901699437494742410;
        const R s1 = (R)0.95105651629515357212 * (R)dir, s2 = (R)0.58778525229247312917 * (R)dir;
        const R cs[5] = {1, c1, c2, c2, c1};
        const R sn[5] = {0, s1, s2, -s2, -s1};
        Cx<R> y[5];
#pragma unroll
        for (int mm = 0; mm < 5; ++mm) {
            R ax = 0, ay = 0;
#pragma unroll
            for (int q = 0; q < 5; ++q) {
                const int k = (q * mm) % 5;
                ax += v[q].x * cs[k] - v[q].y * sn[k];
                ay += v[q].x * sn[k] + v[q].y * cs[k];
            }
            y[mm] = {ax, ay};
        }
#pragma unroll
        for (int mm = 0; mm < 5; ++mm) v[mm] = y[mm];
    }
}

// Stockham FFT of `nl` lines of length N stored as a[k * LS + line]; returns the buffer holding the result.
template <class R>
__device__ Cx<R>* fft_lines(Cx<R>* a, Cx<R>* b, const FFTAxis ax, int LS, int nl, int dir) {
    const Cx<R>* tw = (const Cx<R>*)ax.tw;
    const int N = ax.N;
    int Ns = 1;
    for (int f = 0; f < ax.nf; ++f) {
        const int r = ax.radix[f];
        const int nb = N / r;
        const int tstride = N / (Ns * r);
        for (int w = threadIdx.x; w < nb * nl; w += blockDim.x) {
            const int line = w % nl, j = w / nl;
            const int k = j % Ns;
            Cx<R> v[5];
#pragma unroll
            for (int q = 0; q < 5; ++q)
                if (q < r) v[q] = a[(j + q * nb) * LS + line];
            if (Ns > 1) {
#pragma unroll
                for (int q = 1; q < 5; ++q)
                    if (q < r) v[q] = cmul(v[q], twiddle(tw, q * k * tstride, dir));
            }
            small_dft(v, r, dir);
            const int base = (j / Ns) * Ns * r + k;
#pragma unroll
            for (int q = 0; q < 5; ++q)
                if (q < r) b[(base + q * Ns) * LS + line] = v[q];
        }
        __syncthreads();
        Cx<R>* t = a;
        a = b;
        b = t;
        Ns *= r;
    }
    return a;
}

__host__ __device__ inline int lines_per_block(int N) {
    int nl = 4096 / N;
    if (nl > 16) nl = 16;
    if (nl < 1) nl = 1;
    return nl;
}

// Complex transform of all lines along an axis with element stride `inner`:
// element (o, k, c) at o*N*inner + k*inner + c, lines indexed by (o, c).
template <class R>
__global__ void __launch_bounds__(FFT_THREADS) k_fft_strided(Cx<R>* data, const FFTAxis ax, int64_t inner,
                                                             int dir) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int N = ax.N;
    const int nl = lines_per_block(N);
    const int LS = nl + 1;
    Cx<R>* a = (Cx<R>*)smem_raw;
    Cx<R>* b = a + N * LS;
    const int64_t col_blocks = (inner + nl - 1) / nl;
    const int64_t o = blockIdx.x / col_blocks;
    const int64_t c0 = (blockIdx.x % col_blocks) * nl;
    const int ncols = (int)min((int64_t)nl, inner - c0);
    Cx<R>* base = data + o * N * inner + c0;
    for (int i = threadIdx.x; i < N * nl; i += blockDim.x) {
        const int c = i % nl, k = i / nl;
        a[k * LS + c] = c < ncols ? base[(int64_t)k * inner + c] : Cx<R>{0, 0};
    }
    __syncthreads();
    Cx<R>* res = fft_lines<R>(a, b, ax, LS, nl, dir);
    for (int i = threadIdx.x; i < N * nl; i += blockDim.x) {
        const int c = i % nl, k = i / nl;
        if (c < ncols) base[(int64_t)k * inner + c] = res[k * LS + c];
    }
}

// Inverse z pass: lines of Nzh complex (contiguous) -> Nz reals (contiguous).
template <class R>
__global__ void __launch_bounds__(FFT_THREADS) k_fft_z_c2r(const Cx<R>* spec, R* out, const FFTAxis ax, int Nzh,
                                                           int64_t nlines) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int N = ax.N;
    const int nl = lines_per_block(N);
    const int LS = nl + 1;
    Cx<R>* a = (Cx<R>*)smem_raw;
    Cx<R>* b = a + N * LS;
    const int64_t l0 = (int64_t)blockIdx.x * nl;
    const int nv = (int)min((int64_t)nl, nlines - l0);
    for (int i = threadIdx.x; i < Nzh * nl; i += blockDim.x) {
        const int k = i % Nzh, c = i / Nzh;
        Cx<R> v = c < nv ? spec[(l0 + c) * Nzh + k] : Cx<R>{0, 0};
        const bool self_conj = (k == 0) || (2 * k == N);
        if (self_conj) v.y = 0;
        a[k * LS + c] = v;
        if (k > 0 && 2 * k < N) a[(N - k) * LS + c] = Cx<R>{v.x, -v.y};
    }
    __syncthreads();
    Cx<R>* res = fft_lines<R>(a, b, ax, LS, nl, +1);
    for (int i = threadIdx.x; i < N * nl; i += blockDim.x) {
        const int k = i % N, c = i / N;
        if (c < nv) out[(l0 + c) * N + k] = res[k * LS + c].x;
    }
}

// Forward z pass: lines of Nz reals -> first Nzh complex outputs.
template <class R>
__global__ void __launch_bounds__(FFT_THREADS) k_fft_z_r2c(const R* in, Cx<R>* spec, const FFTAxis ax, int Nzh,
                                                           int64_t nlines) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int N = ax.N;
    const int nl = lines_per_block(N);
    const int LS = nl + 1;
    Cx<R>* a = (Cx<R>*)smem_raw;
    Cx<R>* b = a + N * LS;
    const int64_t l0 = (int64_t)blockIdx.x * nl;
    const int nv = (int)min((int64_t)nl, nlines - l0);
    for (int i = threadIdx.x; i < N * nl; i += blockDim.x) {
        const int k = i % N, c = i / N;
        a[k * LS + c] = Cx<R>{c < nv ? in[(l0 + c) * N + k] : (R)0, (R)0};
    }
    __syncthreads();
    Cx<R>* res = fft_lines<R>(a, b, ax, LS, nl, -1);
    for (int i = threadIdx.x; i < Nzh * nl; i += blockDim.x) {
        const int k = i % Nzh, c = i / Nzh;
        if (c < nv) spec[(l0 + c) * Nzh + k] = res[k * LS + c];
    }
}

template <class R>
cudaError_t set_smem(const void* fn, size_t bytes) {
    if (bytes <= 48 * 1024) return cudaSuccess;
    return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

}  // namespace

bool fft_factor(int N, FFTAxis& a) {
    a.N = N;
    a.nf = 0;
    int n = N;
    if (N < 1 || N > 1024) return false;
    while (n % 4 == 0 && a.nf < 16) { a.radix[a.nf++] = 4; n /= 4; }
    while (n % 2 == 0 && a.nf < 16) { a.radix[a.nf++] = 2; n /= 2; }
    while (n % 3 == 0 && a.nf < 16) { a.radix[a.nf++] = 3; n /= 3; }
    while (n % 5 == 0 && a.nf < 16) { a.radix[a.nf++] = 5; n /= 5; }
    return n == 1;
}

size_t fft_smem_bytes(int N, int elem_bytes) {
    const int nl = lines_per_block(N);
    return (size_t)2 * N * (nl + 1) * elem_bytes;
}

template <class R>
cudaError_t launch_c2r(const Cx<R>* spec_in, Cx<R>* work, R* out, int Nx, int Ny, int Nz, const FFTAxis* ax,
                       cudaStream_t st) {
    const int Nzh = Nz / 2 + 1;
    const int64_t nH = (int64_t)Nx * Ny * Nzh;
    cudaError_t e;
    if (work != spec_in) {
        e = cudaMemcpyAsync(work, spec_in, nH * sizeof(Cx<R>), cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) return e;
    }
    // x pass (stride Ny*Nzh), y pass (stride Nzh), then the real z pass.
    {
        const size_t sm = fft_smem_bytes(Nx, sizeof(Cx<R>));
        if ((e = set_smem<R>((const void*)k_fft_strided<R>, sm)) != cudaSuccess) return e;
        const int64_t inner = (int64_t)Ny * Nzh;
        const int64_t blocks = (inner + lines_per_block(Nx) - 1) / lines_per_block(Nx);
        if (Nx > 1) k_fft_strided<R><<<(unsigned)blocks, FFT_THREADS, sm, st>>>(work, ax[0], inner, +1);
    }
    {
        const size_t sm = fft_smem_bytes(Ny, sizeof(Cx<R>));
        if ((e = set_smem<R>((const void*)k_fft_strided<R>, sm)) != cudaSuccess) return e;
        const int64_t blocks = (int64_t)Nx * ((Nzh + lines_per_block(Ny) - 1) / lines_per_block(Ny));
        if (Ny > 1) k_fft_strided<R><<<(unsigned)blocks, FFT_THREADS, sm, st>>>(work, ax[1], Nzh, +1);
    }
    {
        const size_t sm = fft_smem_bytes(Nz, sizeof(Cx<R>));
        if ((e = set_smem<R>((const void*)k_fft_z_c2r<R>, sm)) != cudaSuccess) return e;
        const int64_t nlines = (int64_t)Nx * Ny;
        const int64_t blocks = (nlines + lines_per_block(Nz) - 1) / lines_per_block(Nz);
        k_fft_z_c2r<R><<<(unsigned)blocks, FFT_THREADS, sm, st>>>(work, out, ax[2], Nzh, nlines);
    }
    return cudaGetLastError();
}

template <class R>
cudaError_t launch_r2c(const R* in, Cx<R>* spec_out, int Nx, int Ny, int Nz, const FFTAxis* ax, cudaStream_t st) {
    const int Nzh = Nz / 2 + 1;
    cudaError_t e;
    {
        const size_t sm = fft_smem_bytes(Nz, sizeof(Cx<R>));
        if ((e = set_smem<R>((const void*)k_fft_z_r2c<R>, sm)) != cudaSuccess) return e;
        const int64_t nlines = (int64_t)Nx * Ny;
        const int64_t blocks = (nlines + lines_per_block(Nz) - 1) / lines_per_block(Nz);
        k_fft_z_r2c<R><<<(unsigned)blocks, FFT_THREADS, sm, st>>>(in, spec_out, ax[2], Nzh, nlines);
    }
    {
        const size_t sm = fft_smem_bytes(Ny, sizeof(Cx<R>));
        if ((e = set_smem<R>((const void*)k_fft_strided<R>, sm)) != cudaSuccess) return e;
        const int64_t blocks = (int64_t)Nx * ((Nzh + lines_per_block(Ny) - 1) / lines_per_block(Ny));
        if (Ny > 1) k_fft_strided<R><<<(unsigned)blocks, FFT_THREADS, sm, st>>>(spec_out, ax[1], Nzh, -1);
    }
    {
        const size_t sm = fft_smem_bytes(Nx, sizeof(Cx<R>));
        if ((e = set_smem<R>((const void*)k_fft_strided<R>, sm)) != cudaSuccess) return e;
        const int64_t inner = (int64_t)Ny * Nzh;
        const int64_t blocks = (inner + lines_per_block(Nx) - 1) / lines_per_block(Nx);
        if (Nx > 1) k_fft_strided<R><<<(unsigned)blocks, FFT_THREADS, sm, st>>>(spec_out, ax[0], inner, -1);
    }
    return cudaGetLastError();
}

template cudaError_t launch_c2r<float>(const Cx<float>*, Cx<float>*, float*, int, int, int, const FFTAxis*,
                                       cudaStream_t);
template cudaError_t launch_c2r<double>(const Cx<double>*, Cx<double>*, double*, int, int, int, const FFTAxis*,
                                        cudaStream_t);
template cudaError_t launch_r2c<float>(const float*, Cx<float>*, int, int, int, const FFTAxis*, cudaStream_t);
template cudaError_t launch_r2c<double>(const double*, Cx<double>*, int, int, int, const FFTAxis*, cudaStream_t);

}  // namespace dm
