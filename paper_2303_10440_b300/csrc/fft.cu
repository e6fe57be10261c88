// 3D real <-> half-spectrum DFTs for the image stage (the inverse transform that
// turns I_hat = u_hat h_hat into voxels, Eq. 1, and its adjoint).
//
// Each pass transforms every line along one axis. FP32 lines of a power-of-two
// length 16 .. 1024 are held in registers (a four-step split N = N1 N2 with one
// exchange through shared memory; see "FP32 power-of-two lines in registers").
// Other lengths, and FP64, stage a batch of lines in shared memory (coalesced
// along the contiguous axis), run a Stockham autosort FFT there (radices 2, 3, 4,
// 5, 7, 11, 13, or 8 for compile-time powers of two; ping-pong buffers, one
// __syncthreads per radix stage), and write the batch back. The z pass of the
// inverse reads the Hermitian-completed line (real parts of the self-conjugate
// n_z = 0 and Nyquist coefficients) for a complex inverse transform; the z pass
// of the forward keeps the first Nz/2+1 outputs. All transforms are unnormalised.
#include <atomic>
#include <cmath>
#include <type_traits>

#include "dm_kernels.cuh"

namespace dm {

namespace {

constexpr int FFT_THREADS = 256;

template <class R>
__device__ __forceinline__ Cx<R> twiddle(const Cx<R>* tw, int idx, int dir) {
    const Cx<R> w = tw[idx];
    return dir < 0 ? w : Cx<R>{w.x, -w.y};
}

// 4-point DFT in place: y[m] = sum_q v[q] exp(dir 2 pi i q m / 4).
template <class R>
__device__ __forceinline__ void dft4(Cx<R>* v, int dir) {
    const Cx<R> s02 = {v[0].x + v[2].x, v[0].y + v[2].y}, d02 = {v[0].x - v[2].x, v[0].y - v[2].y};
    const Cx<R> s13 = {v[1].x + v[3].x, v[1].y + v[3].y}, d13 = {v[1].x - v[3].x, v[1].y - v[3].y};
    // w = exp(dir i pi/2) = dir * i ;  w * d13 = dir * (-d13.y, d13.x)
    const Cx<R> wd = {-(R)dir * d13.y, (R)dir * d13.x};
    v[0] = {s02.x + s13.x, s02.y + s13.y};
    v[1] = {d02.x + wd.x, d02.y + wd.y};
    v[2] = {s02.x - s13.x, s02.y - s13.y};
    v[3] = {d02.x - wd.x, d02.y - wd.y};
}

// cos(2 pi k / P) (sine = false) or sin(2 pi k / P) (sine = true) for the odd primes P = 7, 11, 13 and
// k = 1 .. (P - 1) / 2 (the rest follow by symmetry); the arguments are compile-time constants where
// dft_prime uses it, so each call folds to a literal.
__host__ __device__ constexpr double prime_root(int P, int k, bool sine) {
    if (P == 7) {
        switch (k) {
            case 1: return sine ? 0.78183148246802980363 : 0.62348980185873359439;
            case 2: return sine ? 0.97492791218182361934 : -0.22252093395631433737;
            case 3: return sine ? 0.43388373911755823142 : -0.90096886790241903498;
        }
    }
    if (P == 11) {
        switch (k) {
            case 1: return sine ? 0.54064081745559755543 : 0.84125353283118120551;
            case 2: return sine ? 0.90963199535451833011 : 0.41541501300188643508;
            case 3: return sine ? 0.98982144188093279524 : -0.14231483827328500480;
            case 4: return sine ? 0.75574957435425826890 : -0.65486073394528498959;
            case 5: return sine ? 0.28173255684142967104 : -0.95949297361449736865;
        }
    }
    if (P == 13) {
        switch (k) {
            case 1: return sine ? 0.46472317204376850652 : 0.88545602565320991051;
            case 2: return sine ? 0.82298386589365635224 : 0.56806474673115592289;
            case 3: return sine ? 0.99270887409805397272 : 0.12053668025532300601;
            case 4: return sine ? 0.93501624268541483342 : -0.35460488704253545489;
            case 5: return sine ? 0.66312265824079519305 : -0.74851074817110119231;
            case 6: return sine ? 0.23931566428755768339 : -0.97094181742605201180;
        }
    }
    return sine ? 0.0 : 1.0;
}

// Direct P-point DFT for an odd prime P, y[m] = sum_q v[q] w^(q m) with w = exp(dir 2 pi i / P): the
// inputs are paired as s_q = v[q] + v[P-q], d_q = v[q] - v[P-q] (q = 1 .. (P-1)/2), so that
// y[m] = v[0] + sum_q (s_q cos(2 pi q m / P) + dir i d_q sin(2 pi q m / P)).
template <class R, int P>
__device__ __forceinline__ void dft_prime(Cx<R>* v, int dir) {
    constexpr int H = (P - 1) / 2;
    Cx<R> sq[H + 1], dq[H + 1];
    Cx<R> y0 = v[0];
#pragma unroll
    for (int q = 1; q <= H; ++q) {
        sq[q] = {v[q].x + v[P - q].x, v[q].y + v[P - q].y};
        dq[q] = {v[q].x - v[P - q].x, v[q].y - v[P - q].y};
        y0.x += sq[q].x;
        y0.y += sq[q].y;
    }
    Cx<R> y[P];
    y[0] = y0;
#pragma unroll
    for (int m = 1; m < P; ++m) {
        R ax = v[0].x, ay = v[0].y;
#pragma unroll
        for (int q = 1; q <= H; ++q) {
            const int k = (q * m) % P;
            const R c = (R)(k <= H ? prime_root(P, k, false) : prime_root(P, P - k, false));
            const R sn = (R)(k <= H ? prime_root(P, k, true) : -prime_root(P, P - k, true)) * (R)dir;
            ax += sq[q].x * c - dq[q].y * sn;
            ay += sq[q].y * c + dq[q].x * sn;
        }
        y[m] = {ax, ay};
    }
#pragma unroll
    for (int m = 0; m < P; ++m) v[m] = y[m];
}

// Largest radix a stage may take: fft_factor's radices are 2, 3, 4, 5 and, for lengths with such a
// factor, 7, 11, 13 (BIG); the power-of-two path also takes 8. A mixed-radix kernel that may meet 7-13
// holds 13 values per butterfly and every prime DFT, which takes its registers from 46 to 119: lengths
// without those factors run a kernel compiled without them.
template <bool BIG>
__host__ __device__ constexpr int max_radix() { return BIG ? 13 : 5; }

// y[m] = sum_q v[q] exp(dir 2 pi i q m / r), in place (r = 7, 11, 13 only when BIG).
template <class R, bool BIG>
__device__ __forceinline__ void small_dft(Cx<R>* v, int r, int dir) {
    if (r == 2) {
        const Cx<R> a = v[0], b = v[1];
        v[0] = {a.x + b.x, a.y + b.y};
        v[1] = {a.x - b.x, a.y - b.y};
    } else if (r == 4) {
        dft4(v, dir);
    } else if (r == 3) {
        const R h = (R)0.86602540378443864676 * (R)dir;  // dir * sqrt(3)/2
        const Cx<R> t = {v[1].x + v[2].x, v[1].y + v[2].y}, d = {v[1].x - v[2].x, v[1].y - v[2].y};
        const Cx<R> m = {v[0].x - (R)0.5 * t.x, v[0].y - (R)0.5 * t.y};
        const Cx<R> id = {-h * d.y, h * d.x};  // i * h * d
        v[0] = {v[0].x + t.x, v[0].y + t.y};
        v[1] = {m.x + id.x, m.y + id.y};
        v[2] = {m.x - id.x, m.y - id.y};
    } else if (r == 8) {
        // two 4-point DFTs on the even and odd inputs, combined with the powers of exp(dir 2 pi i / 8)
        Cx<R> e[4] = {v[0], v[2], v[4], v[6]}, o[4] = {v[1], v[3], v[5], v[7]};
        dft4(e, dir);
        dft4(o, dir);
        const R c = (R)0.70710678118654752440;
        const R d = (R)dir;
        const Cx<R> t1 = {c * (o[1].x - d * o[1].y), c * (o[1].y + d * o[1].x)};   // (1 + dir i)/sqrt2 o1
        const Cx<R> t2 = {-d * o[2].y, d * o[2].x};                                  // dir i o2
        const Cx<R> t3 = {c * (-o[3].x - d * o[3].y), c * (-o[3].y + d * o[3].x)};  // (-1 + dir i)/sqrt2 o3
        v[0] = {e[0].x + o[0].x, e[0].y + o[0].y};
        v[4] = {e[0].x - o[0].x, e[0].y - o[0].y};
        v[1] = {e[1].x + t1.x, e[1].y + t1.y};
        v[5] = {e[1].x - t1.x, e[1].y - t1.y};
        v[2] = {e[2].x + t2.x, e[2].y + t2.y};
        v[6] = {e[2].x - t2.x, e[2].y - t2.y};
        v[3] = {e[3].x + t3.x, e[3].y + t3.y};
        v[7] = {e[3].x - t3.x, e[3].y - t3.y};
    } else if (BIG && r == 7) {
        if constexpr (BIG) dft_prime<R, 7>(v, dir);
    } else if (BIG && r == 11) {
        if constexpr (BIG) dft_prime<R, 11>(v, dir);
    } else if (BIG && r == 13) {
        if constexpr (BIG) dft_prime<R, 13>(v, dir);
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

// Lines per block: a batch of about 2048 elements, at most 16 lines (a power of two for power-of-two N).
__host__ __device__ constexpr int lines_per_block(int N) { return 2048 / N > 16 ? 16 : (2048 / N < 1 ? 1 : 2048 / N); }
// Shared-memory row stride (elements) of a batch of nl lines: element k of line c sits at k * stride + c.
// Every kernel, the Stockham stages and the shared-memory size use this one definition.
__host__ __device__ constexpr int line_stride(int nl) { return nl + 1; }

// Stockham FFT of `nl` lines of length N stored as a[k * LS + line]; returns the buffer holding the result.
template <class R, bool BIG>
__device__ Cx<R>* fft_lines(Cx<R>* a, Cx<R>* b, const FFTAxis ax, int LS, int nl, int dir) {
    constexpr int MAX_RADIX = max_radix<BIG>();
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
            Cx<R> v[MAX_RADIX];
#pragma unroll
            for (int q = 0; q < MAX_RADIX; ++q)
                if (q < r) v[q] = a[(j + q * nb) * LS + line];
            if (Ns > 1) {
#pragma unroll
                for (int q = 1; q < MAX_RADIX; ++q)
                    if (q < r) v[q] = cmul(v[q], twiddle(tw, q * k * tstride, dir));
            }
            small_dft<R, BIG>(v, r, dir);
            const int base = (j / Ns) * Ns * r + k;
#pragma unroll
            for (int q = 0; q < MAX_RADIX; ++q)
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


// The same Stockham FFT for a power-of-two length known at compile time: radix-8 stages, then one
// radix-4 or radix-2 stage for the rest, every index computation on constants (no run-time division).
template <class R, int N, int NL, int NS>
__device__ __forceinline__ Cx<R>* stockham_p2(Cx<R>* a, Cx<R>* b, const Cx<R>* tw, int dir) {
    if constexpr (NS >= N) {
        return a;
    } else {
        constexpr int r = ((N / NS) % 8 == 0) ? 8 : (((N / NS) % 4 == 0) ? 4 : 2);
        constexpr int nb = N / r;
        constexpr int tstride = N / (NS * r);
        constexpr int LS = line_stride(NL);
        for (int w = threadIdx.x; w < nb * NL; w += FFT_THREADS) {
            const int line = w % NL, j = w / NL;
            const int k = j % NS;
            Cx<R> v[8];
#pragma unroll
            for (int q = 0; q < r; ++q) v[q] = a[(j + q * nb) * LS + line];
            if constexpr (NS > 1) {
#pragma unroll
                for (int q = 1; q < r; ++q) v[q] = cmul(v[q], twiddle(tw, q * k * tstride, dir));
            }
            small_dft<R, false>(v, r, dir);
            const int base = (j / NS) * NS * r + k;
#pragma unroll
            for (int q = 0; q < r; ++q) b[(base + q * NS) * LS + line] = v[q];
        }
        __syncthreads();
        return stockham_p2<R, N, NL, NS * r>(b, a, tw, dir);
    }
}

// Line transform: the compile-time power-of-two path when NC > 0, else the mixed-radix one (NC = 0:
// radices up to 5; NC = NC_BIG: also 7, 11, 13).
constexpr int NC_BIG = -1;
template <class R, int NC>
__device__ __forceinline__ Cx<R>* transform_lines(Cx<R>* a, Cx<R>* b, const FFTAxis& ax, int LS, int nl, int dir) {
    if constexpr (NC > 0)
        return stockham_p2<R, NC, lines_per_block(NC), 1>(a, b, (const Cx<R>*)ax.tw, dir);
    else
        return fft_lines<R, NC == NC_BIG>(a, b, ax, LS, nl, dir);
}

// Complex transform of all lines along an axis with element stride `inner`:
// element (o, k, c) at o*N*inner + k*inner + c, lines indexed by (o, c).
template <class R, int NC>
__device__ __forceinline__ void k_fft_strided_body(const Cx<R>* src, Cx<R>* dst, const FFTAxis ax, int64_t inner,
                                                   int dir, int64_t blk, int64_t nblk) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int N = NC > 0 ? NC : ax.N;
    const int nl = lines_per_block(N);
    const int LS = line_stride(nl);
    Cx<R>* a = (Cx<R>*)smem_raw;
    Cx<R>* b = a + N * LS;
    const int64_t col_blocks = (inner + nl - 1) / nl;
    const int64_t o = blk / col_blocks;
    const int64_t c0 = (blk % col_blocks) * nl;
    const int ncols = (int)min((int64_t)nl, inner - c0);
    // every read of the block's lines precedes the barrier and every write follows it, so src == dst is fine
    const Cx<R>* sbase = src + o * N * inner + c0;
    Cx<R>* dbase = dst + o * N * inner + c0;
    for (int i = threadIdx.x; i < N * nl; i += blockDim.x) {
        const int c = i % nl, k = i / nl;
        a[k * LS + c] = c < ncols ? sbase[(int64_t)k * inner + c] : Cx<R>{0, 0};
    }
    __syncthreads();
    Cx<R>* res = transform_lines<R, NC>(a, b, ax, LS, nl, dir);
    for (int i = threadIdx.x; i < N * nl; i += blockDim.x) {
        const int c = i % nl, k = i / nl;
        if (c < ncols) dbase[(int64_t)k * inner + c] = res[k * LS + c];
    }
}
template <class R, int NC>
__global__ void __launch_bounds__(FFT_THREADS) k_fft_strided(const Cx<R>* src, Cx<R>* dst, const FFTAxis ax,
                                                             int64_t inner, int dir) {
    k_fft_strided_body<R, NC>(src, dst, ax, inner, dir, (int64_t)blockIdx.x, (int64_t)gridDim.x);
}

// Inverse z pass: lines of Nzh complex (contiguous) -> Nz reals (contiguous).
template <class R, int NC>
__device__ __forceinline__ void k_fft_z_c2r_body(const Cx<R>* spec, R* out, const FFTAxis ax, int Nzh_,
                                                           int64_t nlines, int64_t blk, int64_t nblk) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int N = NC > 0 ? NC : ax.N;
    const int Nzh = NC > 0 ? NC / 2 + 1 : Nzh_;
    const int nl = lines_per_block(N);
    const int LS = line_stride(nl);
    Cx<R>* a = (Cx<R>*)smem_raw;
    Cx<R>* b = a + N * LS;
    const int64_t l0 = blk * nl;
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
    Cx<R>* res = transform_lines<R, NC>(a, b, ax, LS, nl, +1);
    for (int i = threadIdx.x; i < N * nl; i += blockDim.x) {
        const int k = i % N, c = i / N;
        if (c < nv) out[(l0 + c) * N + k] = res[k * LS + c].x;
    }
}
template <class R, int NC>
__global__ void __launch_bounds__(FFT_THREADS) k_fft_z_c2r(const Cx<R>* spec, R* out, const FFTAxis ax, int Nzh_,
                                                           int64_t nlines) {
    k_fft_z_c2r_body<R, NC>(spec, out, ax, Nzh_, nlines, (int64_t)blockIdx.x, (int64_t)gridDim.x);
}

// Forward z pass: lines of Nz reals -> first Nzh complex outputs.
template <class R, int NC>
__device__ __forceinline__ void k_fft_z_r2c_body(const R* in, Cx<R>* spec, const FFTAxis ax, int Nzh_,
                                                           int64_t nlines, int64_t blk, int64_t nblk) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int N = NC > 0 ? NC : ax.N;
    const int Nzh = NC > 0 ? NC / 2 + 1 : Nzh_;
    const int nl = lines_per_block(N);
    const int LS = line_stride(nl);
    Cx<R>* a = (Cx<R>*)smem_raw;
    Cx<R>* b = a + N * LS;
    const int64_t l0 = blk * nl;
    const int nv = (int)min((int64_t)nl, nlines - l0);
    for (int i = threadIdx.x; i < N * nl; i += blockDim.x) {
        const int k = i % N, c = i / N;
        a[k * LS + c] = Cx<R>{c < nv ? in[(l0 + c) * N + k] : (R)0, (R)0};
    }
    __syncthreads();
    Cx<R>* res = transform_lines<R, NC>(a, b, ax, LS, nl, -1);
    for (int i = threadIdx.x; i < Nzh * nl; i += blockDim.x) {
        const int k = i % Nzh, c = i / Nzh;
        if (c < nv) spec[(l0 + c) * Nzh + k] = res[k * LS + c];
    }
}
template <class R, int NC>
__global__ void __launch_bounds__(FFT_THREADS) k_fft_z_r2c(const R* in, Cx<R>* spec, const FFTAxis ax, int Nzh_,
                                                           int64_t nlines) {
    k_fft_z_r2c_body<R, NC>(in, spec, ax, Nzh_, nlines, (int64_t)blockIdx.x, (int64_t)gridDim.x);
}

// ---------------------------------------------------------------- FP32 power-of-two lines in registers
// For N = 16 .. 1024 the FP32 passes split N = N1 N2 (N2 = 2^floor(log2(N) / 2), N1 = N / N2, so N1 is N2
// or 2 N2) and keep each line in the registers of T = N2 threads. With k = k2 + N2 k1 and m = m1 + N1 m2,
//   X[m1 + N1 m2] = sum_k2 w_N2^(k2 m2) [ w_N^(k2 m1) sum_k1 x[k2 + N2 k1] w_N1^(k1 m1) ]
// (w_M = exp(dir 2 pi i / M); the four-step factorisation of the DFT): thread k2 loads x[k2 + N2 k1]
// (k1 < N1) from global memory, runs the N1-point DFT in registers and applies the twiddles w_N^(k2 m1);
// one exchange through shared memory gives thread t the values of m1 = t, t + T, .. for its N2-point
// DFTs, whose outputs go straight to global memory. One shared-memory round trip per pass instead of
// one per radix stage, and no staging copy of the lines.

__host__ __device__ constexpr int ilog2c(int n) { return n <= 1 ? 0 : 1 + ilog2c(n / 2); }
__host__ __device__ constexpr bool p2_reg(int N) { return N >= 16 && N <= 1024 && (N & (N - 1)) == 0; }

template <int N>
struct P2 {
    static constexpr int N2 = 1 << (ilog2c(N) / 2);
    static constexpr int N1 = N / N2;
    static constexpr int T = N2;                // threads per line
    static constexpr int NL = FFT_THREADS / T;  // lines per block
    // Strided passes (consecutive lanes take consecutive lines, so that the global accesses coalesce):
    // value (k2, m1) of line c at k2 * ROW + m1 * NL + c. z passes (consecutive lanes run along a line):
    // at c * LINE + k2 * RS + m1. The paddings make both sides of the exchange free of bank conflicts
    // (each half-warp's 8-byte accesses fall on 16 distinct bank pairs).
    static constexpr int ROW = N1 * NL + (NL < 16 ? 8 : 0);
    static constexpr int RS = N1 + 1;
    static constexpr int LINE = N2 * RS;
    static constexpr size_t SMEM_STRIDED = (size_t)N2 * ROW * sizeof(Cx<float>);
    static constexpr size_t SMEM_Z = (size_t)NL * LINE * sizeof(Cx<float>);
};
int p2_lines_per_block(int N) { return FFT_THREADS / (1 << (ilog2c(N) / 2)); }

// cos(j pi / 16) for j = 0 .. 8: the first octant of the 32nd roots of unity.
__host__ __device__ constexpr float cos_pi16(int j) {
    switch (j) {
        case 0: return 1.0f;
        case 1: return 0.98078528040323044913f;
        case 2: return 0.92387953251128675613f;
        case 3: return 0.83146961230254523708f;
        case 4: return 0.70710678118654752440f;
        case 5: return 0.55557023301960222474f;
        case 6: return 0.38268343236508977173f;
        case 7: return 0.19509032201612826785f;
        default: return 0.0f;
    }
}
// cos(k pi / 16) for any k in 0 .. 31, by the symmetries of the cosine.
__host__ __device__ constexpr float cos_k32(int k) {
    return k <= 8 ? cos_pi16(k) : k <= 16 ? -cos_pi16(16 - k) : k <= 24 ? -cos_pi16(k - 16) : cos_pi16(32 - k);
}
// a exp(DIR 2 pi i k / 32) for 0 <= k < 32 (k is a constant once the caller's loops are unrolled; the
// multiples of a quarter turn are exact).
template <int DIR>
__device__ __forceinline__ Cx<float> rot32(Cx<float> a, int k) {
    if (k == 0) return a;
    if (k == 8) return DIR > 0 ? Cx<float>{-a.y, a.x} : Cx<float>{a.y, -a.x};
    if (k == 16) return {-a.x, -a.y};
    if (k == 24) return DIR > 0 ? Cx<float>{a.y, -a.x} : Cx<float>{-a.y, a.x};
    const Cx<float> w = {cos_k32(k), (float)DIR * cos_k32((40 - k) % 32)};  // sin(x) = cos(pi/2 - x)
    return cmul(a, w);
}

__host__ __device__ constexpr int bit_reverse(int i, int bits) {
    int r = 0;
    for (int b = 0; b < bits; ++b) r |= ((i >> b) & 1) << (bits - 1 - b);
    return r;
}

// y[m] = sum_q v[q] exp(DIR 2 pi i q m / M) in place, M a power of two up to 32: radix-2 decimation in
// time on the bit-reversed inputs, every index and twiddle a constant after unrolling.
template <int M, int DIR>
__device__ __forceinline__ void dft_reg(Cx<float>* v) {
    constexpr int B = ilog2c(M);
    static_assert((1 << B) == M && M <= 32, "dft_reg takes powers of two up to 32");
    Cx<float> u[M];
#pragma unroll
    for (int i = 0; i < M; ++i) u[bit_reverse(i, B)] = v[i];
#pragma unroll
    for (int h = 1; h < M; h *= 2) {  // DFTs of length h combined into length 2h
#pragma unroll
        for (int s0 = 0; s0 < M; s0 += 2 * h) {
#pragma unroll
            for (int j = 0; j < h; ++j) {
                const Cx<float> a = u[s0 + j], b = rot32<DIR>(u[s0 + j + h], j * (16 / h));
                u[s0 + j] = {a.x + b.x, a.y + b.y};
                u[s0 + j + h] = {a.x - b.x, a.y - b.y};
            }
        }
    }
#pragma unroll
    for (int i = 0; i < M; ++i) v[i] = u[i];
}

// v[m] *= exp(DIR 2 pi i t m / N) for m < E (t E <= N), from the table tw[j] = exp(-2 pi i j / N): the
// factors for m = 2^b are table values, the others products of those of m's binary digits.
template <int E, int DIR>
__device__ __forceinline__ void twiddle_pow(Cx<float>* v, int t, const Cx<float>* __restrict__ tw) {
    constexpr int B = ilog2c(E);
    Cx<float> p[B > 0 ? B : 1];
#pragma unroll
    for (int b = 0; b < B; ++b) {
        const Cx<float> w = tw[t << b];
        p[b] = DIR > 0 ? Cx<float>{w.x, -w.y} : w;
    }
#pragma unroll
    for (int m = 1; m < E; ++m) {
        Cx<float> f = {1.f, 0.f};
        bool first = true;
#pragma unroll
        for (int b = 0; b < B; ++b) {
            if ((m >> b) & 1) {
                f = first ? p[b] : cmul(f, p[b]);
                first = false;
            }
        }
        v[m] = cmul(v[m], f);
    }
}

// Complex pass over nlines lines of N elements with element stride `inner`: line L = o * inner + c
// (o = L / inner) starts at o * N * inner + c. src == dst is allowed (all reads of a block's lines
// precede its barrier, all writes follow it, and no two blocks share a line).
template <int N, int DIR>
__device__ __forceinline__ void p2_strided_body(const Cx<float>* src, Cx<float>* dst, int64_t inner, int64_t nlines,
                                                const Cx<float>* __restrict__ tw, int64_t blk) {
    using P = P2<N>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Cx<float>* Y = (Cx<float>*)smem_raw;
    const int c = threadIdx.x % P::NL, t = threadIdx.x / P::NL;
    const int64_t L = blk * P::NL + c;
    const bool act = L < nlines;
    const int64_t o = act ? L / inner : 0;
    const int64_t off = act ? o * N * inner + (L - o * inner) : 0;
    Cx<float> v[P::N1];
#pragma unroll
    for (int k1 = 0; k1 < P::N1; ++k1)
        v[k1] = act ? src[off + (int64_t)(t + P::N2 * k1) * inner] : Cx<float>{0.f, 0.f};
    dft_reg<P::N1, DIR>(v);
    twiddle_pow<P::N1, DIR>(v, t, tw);
#pragma unroll
    for (int m1 = 0; m1 < P::N1; ++m1) Y[t * P::ROW + m1 * P::NL + c] = v[m1];
    __syncthreads();
#pragma unroll
    for (int r = 0; r < P::N1 / P::N2; ++r) {
        const int m1 = t + P::T * r;
        Cx<float> u[P::N2];
#pragma unroll
        for (int k2 = 0; k2 < P::N2; ++k2) u[k2] = Y[k2 * P::ROW + m1 * P::NL + c];
        dft_reg<P::N2, DIR>(u);
        if (act) {
#pragma unroll
            for (int m2 = 0; m2 < P::N2; ++m2) dst[off + (int64_t)(m1 + P::N1 * m2) * inner] = u[m2];
        }
    }
}

// Inverse z pass: nlines lines of N/2 + 1 coefficients (contiguous) -> N reals; the Hermitian half
// (k > N/2) is read as conj(X[N - k]), and the n_z = 0 and Nyquist coefficients count by their real parts.
template <int N>
__device__ __forceinline__ void p2_z_c2r_body(const Cx<float>* spec, float* out, int64_t nlines,
                                              const Cx<float>* __restrict__ tw, int64_t blk) {
    using P = P2<N>;
    constexpr int H = N / 2;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Cx<float>* Y = (Cx<float>*)smem_raw;
    const int t = threadIdx.x % P::T, c = threadIdx.x / P::T;
    const int64_t L = blk * P::NL + c;
    const bool act = L < nlines;
    const Cx<float>* s = spec + (act ? L : 0) * (H + 1);
    Cx<float> v[P::N1];
#pragma unroll
    for (int k1 = 0; k1 < P::N1; ++k1) {
        const int k = t + P::N2 * k1;
        Cx<float> x = {0.f, 0.f};
        if (act) {
            if (k <= H) {
                x = s[k];
                if (k == 0 || k == H) x.y = 0.f;
            } else {
                x = s[N - k];
                x.y = -x.y;
            }
        }
        v[k1] = x;
    }
    dft_reg<P::N1, 1>(v);
    twiddle_pow<P::N1, 1>(v, t, tw);
    Cx<float>* Yc = Y + c * P::LINE;
#pragma unroll
    for (int m1 = 0; m1 < P::N1; ++m1) Yc[t * P::RS + m1] = v[m1];
    __syncthreads();
#pragma unroll
    for (int r = 0; r < P::N1 / P::N2; ++r) {
        const int m1 = t + P::T * r;
        Cx<float> u[P::N2];
#pragma unroll
        for (int k2 = 0; k2 < P::N2; ++k2) u[k2] = Yc[k2 * P::RS + m1];
        dft_reg<P::N2, 1>(u);
        if (act) {
#pragma unroll
            for (int m2 = 0; m2 < P::N2; ++m2) out[L * N + m1 + P::N1 * m2] = u[m2].x;
        }
    }
}

// Forward z pass: nlines lines of N reals (contiguous) -> the first N/2 + 1 coefficients.
template <int N>
__device__ __forceinline__ void p2_z_r2c_body(const float* in, Cx<float>* spec, int64_t nlines,
                                              const Cx<float>* __restrict__ tw, int64_t blk) {
    using P = P2<N>;
    constexpr int H = N / 2;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Cx<float>* Y = (Cx<float>*)smem_raw;
    const int t = threadIdx.x % P::T, c = threadIdx.x / P::T;
    const int64_t L = blk * P::NL + c;
    const bool act = L < nlines;
    const float* s = in + (act ? L : 0) * N;
    Cx<float> v[P::N1];
#pragma unroll
    for (int k1 = 0; k1 < P::N1; ++k1) v[k1] = {act ? s[t + P::N2 * k1] : 0.f, 0.f};
    dft_reg<P::N1, -1>(v);
    twiddle_pow<P::N1, -1>(v, t, tw);
    Cx<float>* Yc = Y + c * P::LINE;
#pragma unroll
    for (int m1 = 0; m1 < P::N1; ++m1) Yc[t * P::RS + m1] = v[m1];
    __syncthreads();
#pragma unroll
    for (int r = 0; r < P::N1 / P::N2; ++r) {
        const int m1 = t + P::T * r;
        Cx<float> u[P::N2];
#pragma unroll
        for (int k2 = 0; k2 < P::N2; ++k2) u[k2] = Yc[k2 * P::RS + m1];
        dft_reg<P::N2, -1>(u);
        if (act) {
#pragma unroll
            for (int m2 = 0; m2 < P::N2; ++m2) {
                const int m = m1 + P::N1 * m2;
                if (m <= H) spec[L * (H + 1) + m] = u[m2];
            }
        }
    }
}

template <int N, int DIR>
__global__ void __launch_bounds__(FFT_THREADS) k_p2_strided(const Cx<float>* src, Cx<float>* dst, int64_t inner,
                                                            int64_t nlines, const Cx<float>* __restrict__ tw) {
    p2_strided_body<N, DIR>(src, dst, inner, nlines, tw, (int64_t)blockIdx.x);
}
template <int N>
__global__ void __launch_bounds__(FFT_THREADS) k_p2_z_c2r(const Cx<float>* __restrict__ spec, float* __restrict__ out,
                                                          int64_t nlines, const Cx<float>* __restrict__ tw) {
    p2_z_c2r_body<N>(spec, out, nlines, tw, (int64_t)blockIdx.x);
}
template <int N>
__global__ void __launch_bounds__(FFT_THREADS) k_p2_z_r2c(const float* __restrict__ in, Cx<float>* __restrict__ spec,
                                                          int64_t nlines, const Cx<float>* __restrict__ tw) {
    p2_z_r2c_body<N>(in, spec, nlines, tw, (int64_t)blockIdx.x);
}

// Batched passes (fit server): the jobs of one line length in one launch; block b belongs to the
// largest job j with offs[j] <= b, as its block b - offs[j] of its single-job grid.
struct FFTBlock {
    int j;
    int64_t b, nb;
};
__device__ __forceinline__ FFTBlock fft_block(const int* __restrict__ offs, int nj) {
    const int bi = (int)blockIdx.x;
    int lo = 0, hi = nj;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (offs[mid] <= bi)
            lo = mid;
        else
            hi = mid;
    }
    return {lo, (int64_t)(bi - offs[lo]), (int64_t)(offs[lo + 1] - offs[lo])};
}
template <class R, int NC>
__global__ void __launch_bounds__(FFT_THREADS) kb_fft_strided(const FFTJob* __restrict__ jobs,
                                                              const int* __restrict__ offs, int nj, int dir) {
    const FFTBlock q = fft_block(offs, nj);
    const FFTJob& J = jobs[q.j];
    k_fft_strided_body<R, NC>((const Cx<R>*)J.src, (Cx<R>*)J.dst, J.ax, J.inner, dir, q.b, q.nb);
}
template <class R, int NC>
__global__ void __launch_bounds__(FFT_THREADS) kb_fft_z_c2r(const FFTJob* __restrict__ jobs,
                                                            const int* __restrict__ offs, int nj) {
    const FFTBlock q = fft_block(offs, nj);
    const FFTJob& J = jobs[q.j];
    k_fft_z_c2r_body<R, NC>((const Cx<R>*)J.src, (R*)J.dst, J.ax, J.Nzh, J.lines, q.b, q.nb);
}
template <class R, int NC>
__global__ void __launch_bounds__(FFT_THREADS) kb_fft_z_r2c(const FFTJob* __restrict__ jobs,
                                                            const int* __restrict__ offs, int nj) {
    const FFTBlock q = fft_block(offs, nj);
    const FFTJob& J = jobs[q.j];
    k_fft_z_r2c_body<R, NC>((const R*)J.src, (Cx<R>*)J.dst, J.ax, J.Nzh, J.lines, q.b, q.nb);
}

template <int N, int DIR>
__global__ void __launch_bounds__(FFT_THREADS) kb_p2_strided(const FFTJob* __restrict__ jobs,
                                                             const int* __restrict__ offs, int nj) {
    const FFTBlock q = fft_block(offs, nj);
    const FFTJob& J = jobs[q.j];
    p2_strided_body<N, DIR>((const Cx<float>*)J.src, (Cx<float>*)J.dst, J.inner, J.lines * J.inner,
                            (const Cx<float>*)J.ax.tw, q.b);
}
template <int N>
__global__ void __launch_bounds__(FFT_THREADS) kb_p2_z_c2r(const FFTJob* __restrict__ jobs,
                                                           const int* __restrict__ offs, int nj) {
    const FFTBlock q = fft_block(offs, nj);
    const FFTJob& J = jobs[q.j];
    p2_z_c2r_body<N>((const Cx<float>*)J.src, (float*)J.dst, J.lines, (const Cx<float>*)J.ax.tw, q.b);
}
template <int N>
__global__ void __launch_bounds__(FFT_THREADS) kb_p2_z_r2c(const FFTJob* __restrict__ jobs,
                                                           const int* __restrict__ offs, int nj) {
    const FFTBlock q = fft_block(offs, nj);
    const FFTJob& J = jobs[q.j];
    p2_z_r2c_body<N>((const float*)J.src, (Cx<float>*)J.dst, J.lines, (const Cx<float>*)J.ax.tw, q.b);
}

// Raises kernel FN's dynamic shared-memory limit to the device's opt-in maximum, once per device,
// so that later launches (also those captured into a CUDA graph) need no attribute call.
template <auto FN>
cudaError_t set_smem(size_t bytes) {
    if (bytes <= 48 * 1024) return cudaSuccess;
    static std::atomic<int> raised[64];
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 64 && raised[dev].load() != 0) return cudaSuccess;
    int max_smem = 0;
    if ((e = cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev)) != cudaSuccess) return e;
    if (bytes > (size_t)max_smem) return cudaErrorInvalidValue;
    if ((e = cudaFuncSetAttribute((const void*)FN, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem)) != cudaSuccess)
        return e;
    if (dev < 64) raised[dev].store(1);
    return cudaSuccess;
}

}  // namespace

bool fft_factor(int N, FFTAxis& a) {
    a.N = N;
    a.nf = 0;
    int n = N;
    if (N < 1 || N > FFT_MAX_N) return false;
    while (n % 4 == 0 && a.nf < 16) { a.radix[a.nf++] = 4; n /= 4; }
    while (n % 2 == 0 && a.nf < 16) { a.radix[a.nf++] = 2; n /= 2; }
    for (const int p : {3, 5, 7, 11, 13})
        while (n % p == 0 && a.nf < 16) { a.radix[a.nf++] = p; n /= p; }
    return n == 1;
}

// Whether an axis's factorisation uses a radix above 5 (the NC_BIG kernels).
static bool has_big_radix(const FFTAxis& a) {
    for (int f = 0; f < a.nf; ++f)
        if (a.radix[f] > 5) return true;
    return false;
}

size_t fft_smem_bytes(int N, int elem_bytes) {
    const int nl = lines_per_block(N);
    return (size_t)2 * N * line_stride(nl) * elem_bytes;
}

// One pass over every line of an axis: for FP32 power-of-two lengths 16 .. 1024 the register-resident
// kernels, for other powers of two up to 4096 the Stockham kernel instantiated for the length (NC = N),
// otherwise the mixed-radix kernel (NC = 0, or NC_BIG when the length has a factor 7, 11 or 13).
enum PassKind { PASS_STRIDED, PASS_Z_C2R, PASS_Z_R2C };

// FP32 power-of-two lengths 16 .. 1024: the register-resident passes.
template <int N>
cudaError_t run_p2_pass(PassKind kind, const void* src, void* dst, const FFTAxis& ax, int64_t inner, int64_t outer,
                        int dir, cudaStream_t st) {
    using P = P2<N>;
    const Cx<float>* tw = (const Cx<float>*)ax.tw;
    cudaError_t e;
    if (kind == PASS_STRIDED) {
        const int64_t nlines = inner * outer;
        const unsigned blocks = (unsigned)((nlines + P::NL - 1) / P::NL);
        if (dir > 0) {
            if ((e = set_smem<k_p2_strided<N, 1>>(P::SMEM_STRIDED)) != cudaSuccess) return e;
            k_p2_strided<N, 1><<<blocks, FFT_THREADS, P::SMEM_STRIDED, st>>>((const Cx<float>*)src, (Cx<float>*)dst,
                                                                              inner, nlines, tw);
        } else {
            if ((e = set_smem<k_p2_strided<N, -1>>(P::SMEM_STRIDED)) != cudaSuccess) return e;
            k_p2_strided<N, -1><<<blocks, FFT_THREADS, P::SMEM_STRIDED, st>>>((const Cx<float>*)src, (Cx<float>*)dst,
                                                                               inner, nlines, tw);
        }
    } else {
        const unsigned blocks = (unsigned)((outer + P::NL - 1) / P::NL);
        if (kind == PASS_Z_C2R) {
            if ((e = set_smem<k_p2_z_c2r<N>>(P::SMEM_Z)) != cudaSuccess) return e;
            k_p2_z_c2r<N><<<blocks, FFT_THREADS, P::SMEM_Z, st>>>((const Cx<float>*)src, (float*)dst, outer, tw);
        } else {
            if ((e = set_smem<k_p2_z_r2c<N>>(P::SMEM_Z)) != cudaSuccess) return e;
            k_p2_z_r2c<N><<<blocks, FFT_THREADS, P::SMEM_Z, st>>>((const float*)src, (Cx<float>*)dst, outer, tw);
        }
    }
    return cudaGetLastError();
}

template <class R, int NC>
cudaError_t run_pass(PassKind kind, const void* src, void* dst, const FFTAxis& ax, int64_t inner, int64_t outer,
                     int Nzh, int dir, cudaStream_t st) {
    if constexpr (std::is_same<R, float>::value && p2_reg(NC)) {
        return run_p2_pass<NC>(kind, src, dst, ax, inner, outer, dir, st);
    } else {
        const int N = ax.N;
        const int nl = lines_per_block(N);
        const size_t sm = fft_smem_bytes(N, sizeof(Cx<R>));
        cudaError_t e;
        if (kind == PASS_STRIDED) {
            if ((e = set_smem<k_fft_strided<R, NC>>(sm)) != cudaSuccess) return e;
            const int64_t blocks = outer * ((inner + nl - 1) / nl);
            k_fft_strided<R, NC><<<(unsigned)blocks, FFT_THREADS, sm, st>>>((const Cx<R>*)src, (Cx<R>*)dst, ax, inner,
                                                                              dir);
        } else if (kind == PASS_Z_C2R) {
            if ((e = set_smem<k_fft_z_c2r<R, NC>>(sm)) != cudaSuccess) return e;
            const int64_t blocks = (outer + nl - 1) / nl;
            k_fft_z_c2r<R, NC><<<(unsigned)blocks, FFT_THREADS, sm, st>>>((const Cx<R>*)src, (R*)dst, ax, Nzh, outer);
        } else {
            if ((e = set_smem<k_fft_z_r2c<R, NC>>(sm)) != cudaSuccess) return e;
            const int64_t blocks = (outer + nl - 1) / nl;
            k_fft_z_r2c<R, NC><<<(unsigned)blocks, FFT_THREADS, sm, st>>>((const R*)src, (Cx<R>*)dst, ax, Nzh, outer);
        }
        return cudaGetLastError();
    }
}

template <class R>
cudaError_t pass(PassKind kind, const void* src, void* dst, const FFTAxis& ax, int64_t inner, int64_t outer, int Nzh,
                 int dir, cudaStream_t st) {
    switch (ax.N) {
        case 16: return run_pass<R, 16>(kind, src, dst, ax, inner, outer, Nzh, dir, st);
        case 32: return run_pass<R, 32>(kind, src, dst, ax, inner, outer, Nzh, dir, st);
        case 64: return run_pass<R, 64>(kind, src, dst, ax, inner, outer, Nzh, dir, st);
        case 128: return run_pass<R, 128>(kind, src, dst, ax, inner, outer, Nzh, dir, st);
        case 256: return run_pass<R, 256>(kind, src, dst, ax, inner, outer, Nzh, dir, st);
        case 512: return run_pass<R, 512>(kind, src, dst, ax, inner, outer, Nzh, dir, st);
        case 1024: return run_pass<R, 1024>(kind, src, dst, ax, inner, outer, Nzh, dir, st);
        case 2048: return run_pass<R, 2048>(kind, src, dst, ax, inner, outer, Nzh, dir, st);
        case 4096: return run_pass<R, 4096>(kind, src, dst, ax, inner, outer, Nzh, dir, st);
        default:
            return has_big_radix(ax) ? run_pass<R, NC_BIG>(kind, src, dst, ax, inner, outer, Nzh, dir, st)
                                     : run_pass<R, 0>(kind, src, dst, ax, inner, outer, Nzh, dir, st);
    }
}

template <int NC>
cudaError_t run_batch_pass(int kind, const FFTJob* jobs, const int* offs, int nj, int total, int N, int dir,
                           cudaStream_t st) {
    cudaError_t e;
    if constexpr (p2_reg(NC)) {
        using P = P2<NC>;
        if (kind == FFT_STRIDED) {
            if (dir > 0) {
                if ((e = set_smem<kb_p2_strided<NC, 1>>(P::SMEM_STRIDED)) != cudaSuccess) return e;
                kb_p2_strided<NC, 1><<<total, FFT_THREADS, P::SMEM_STRIDED, st>>>(jobs, offs, nj);
            } else {
                if ((e = set_smem<kb_p2_strided<NC, -1>>(P::SMEM_STRIDED)) != cudaSuccess) return e;
                kb_p2_strided<NC, -1><<<total, FFT_THREADS, P::SMEM_STRIDED, st>>>(jobs, offs, nj);
            }
        } else if (kind == FFT_Z_C2R) {
            if ((e = set_smem<kb_p2_z_c2r<NC>>(P::SMEM_Z)) != cudaSuccess) return e;
            kb_p2_z_c2r<NC><<<total, FFT_THREADS, P::SMEM_Z, st>>>(jobs, offs, nj);
        } else {
            if ((e = set_smem<kb_p2_z_r2c<NC>>(P::SMEM_Z)) != cudaSuccess) return e;
            kb_p2_z_r2c<NC><<<total, FFT_THREADS, P::SMEM_Z, st>>>(jobs, offs, nj);
        }
        return cudaGetLastError();
    } else {
        const size_t sm = fft_smem_bytes(N, sizeof(Cx<float>));
        if (kind == FFT_STRIDED) {
            if ((e = set_smem<kb_fft_strided<float, NC>>(sm)) != cudaSuccess) return e;
            kb_fft_strided<float, NC><<<total, FFT_THREADS, sm, st>>>(jobs, offs, nj, dir);
        } else if (kind == FFT_Z_C2R) {
            if ((e = set_smem<kb_fft_z_c2r<float, NC>>(sm)) != cudaSuccess) return e;
            kb_fft_z_c2r<float, NC><<<total, FFT_THREADS, sm, st>>>(jobs, offs, nj);
        } else {
            if ((e = set_smem<kb_fft_z_r2c<float, NC>>(sm)) != cudaSuccess) return e;
            kb_fft_z_r2c<float, NC><<<total, FFT_THREADS, sm, st>>>(jobs, offs, nj);
        }
        return cudaGetLastError();
    }
}

int64_t fft_pass_blocks(int kind, const FFTJob& j) {
    if (p2_reg(j.ax.N)) {
        const int nl = p2_lines_per_block(j.ax.N);
        const int64_t lines = kind == FFT_STRIDED ? j.lines * j.inner : j.lines;
        return (lines + nl - 1) / nl;
    }
    const int nl = lines_per_block(j.ax.N);
    if (kind == FFT_STRIDED) return j.lines * ((j.inner + nl - 1) / nl);  // lines: the outer count
    return (j.lines + nl - 1) / nl;
}

cudaError_t launch_fft_batch(int kind, int N, const FFTJob* jobs, const int* offsets, int nj, int total, int dir,
                             cudaStream_t st) {
    if (total <= 0 || nj <= 0) return cudaSuccess;
    switch (N) {
        case 16: return run_batch_pass<16>(kind, jobs, offsets, nj, total, N, dir, st);
        case 32: return run_batch_pass<32>(kind, jobs, offsets, nj, total, N, dir, st);
        case 64: return run_batch_pass<64>(kind, jobs, offsets, nj, total, N, dir, st);
        case 128: return run_batch_pass<128>(kind, jobs, offsets, nj, total, N, dir, st);
        case 256: return run_batch_pass<256>(kind, jobs, offsets, nj, total, N, dir, st);
        case 512: return run_batch_pass<512>(kind, jobs, offsets, nj, total, N, dir, st);
        case 1024: return run_batch_pass<1024>(kind, jobs, offsets, nj, total, N, dir, st);
        case 2048: return run_batch_pass<2048>(kind, jobs, offsets, nj, total, N, dir, st);
        case 4096: return run_batch_pass<4096>(kind, jobs, offsets, nj, total, N, dir, st);
        default: {
            FFTAxis f;
            if (!fft_factor(N, f)) return cudaErrorInvalidValue;
            return has_big_radix(f) ? run_batch_pass<NC_BIG>(kind, jobs, offsets, nj, total, N, dir, st)
                                    : run_batch_pass<0>(kind, jobs, offsets, nj, total, N, dir, st);
        }
    }
}

template <class R>
cudaError_t launch_c2r(const Cx<R>* spec_in, Cx<R>* work, R* out, int Nx, int Ny, int Nz, const FFTAxis* ax,
                       cudaStream_t st) {
    const int Nzh = Nz / 2 + 1;
    cudaError_t e;
    // x pass (stride Ny*Nzh), y pass (stride Nzh), then the real z pass; the first pass that runs reads
    // spec_in and writes work, so spec_in is left unchanged when it differs from work.
    const Cx<R>* cur = spec_in;
    if (Nx > 1) {
        if ((e = pass<R>(PASS_STRIDED, cur, work, ax[0], (int64_t)Ny * Nzh, 1, Nzh, +1, st)) != cudaSuccess) return e;
        cur = work;
    }
    if (Ny > 1) {
        if ((e = pass<R>(PASS_STRIDED, cur, work, ax[1], Nzh, Nx, Nzh, +1, st)) != cudaSuccess) return e;
        cur = work;
    }
    return pass<R>(PASS_Z_C2R, cur, out, ax[2], 0, (int64_t)Nx * Ny, Nzh, +1, st);
}

template <class R>
cudaError_t launch_r2c(const R* in, Cx<R>* spec_out, int Nx, int Ny, int Nz, const FFTAxis* ax, cudaStream_t st) {
    const int Nzh = Nz / 2 + 1;
    cudaError_t e;
    if ((e = pass<R>(PASS_Z_R2C, in, spec_out, ax[2], 0, (int64_t)Nx * Ny, Nzh, -1, st)) != cudaSuccess) return e;
    if (Ny > 1 && (e = pass<R>(PASS_STRIDED, spec_out, spec_out, ax[1], Nzh, Nx, Nzh, -1, st)) != cudaSuccess)
        return e;
    if (Nx > 1 && (e = pass<R>(PASS_STRIDED, spec_out, spec_out, ax[0], (int64_t)Ny * Nzh, 1, Nzh, -1, st)) !=
                      cudaSuccess)
        return e;
    return cudaSuccess;
}

template cudaError_t launch_c2r<float>(const Cx<float>*, Cx<float>*, float*, int, int, int, const FFTAxis*,
                                       cudaStream_t);
template cudaError_t launch_c2r<double>(const Cx<double>*, Cx<double>*, double*, int, int, int, const FFTAxis*,
                                        cudaStream_t);
template cudaError_t launch_r2c<float>(const float*, Cx<float>*, int, int, int, const FFTAxis*, cudaStream_t);
template cudaError_t launch_r2c<double>(const double*, Cx<double>*, int, int, int, const FFTAxis*, cudaStream_t);

}  // namespace dm
