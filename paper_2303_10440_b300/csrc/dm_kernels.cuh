// Internal interface between the C ABI (api.cu) and the kernel translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "dm_common.cuh"

namespace dm {

// ---------------------------------------------------------------- records
// Per-triangle record of the FP32 path (96 B; staged into shared memory in tiles).
//   U   : fixed-point fraction of (v1 - origin)/L per axis (2^32 = one period), so the
//         phase of vertex 1 at integer frequency n is 2 pi (n . U mod 2^32) / 2^32, exactly.
//   e21 : v2 - v1,  e31 : v3 - v1   (physical units)
//   w   : surface: (density * 2A, 0, 0);  volume: n_T = (v2 - v1) x (v3 - v1)
// Every float field is stored twice (x, x) so that two terms evaluated together with
// paired FP32 instructions can use it as one 8-byte operand.
struct __align__(16) TriF32 {
    uint32_t U[3];
    uint32_t pad;
    float2 e21x, e21y, e21z;
    float2 e31x, e31y, e31z;
    float2 w0, w1, w2;
    float2 pad2;
};
static_assert(sizeof(TriF32) == 96, "TriF32 layout");

// FP64 path: same fields, 64-bit fixed point and doubles (96 B).
struct __align__(16) TriF64 {
    uint64_t U[3];
    double e21[3];
    double e31[3];
    double w[3];
};
static_assert(sizeof(TriF64) == 96, "TriF64 layout");

// Adjoint records. FP32: two frequencies (lanes A, B) per 64 B record, so a thread evaluates
// both against its triangle with paired FP32 instructions: integer frequencies, wavevectors and
// the complex weight Gw the per-triangle sums contract with. FP64: one frequency per record.
struct __align__(16) FreqPairF32 {
    int32_t nA[3];
    int32_t nB[3];
    float2 x, y, z;   // (A, B)
    float2 Gr, Gi;    // (A, B)
};
static_assert(sizeof(FreqPairF32) == 64, "FreqPairF32 layout");
typedef FreqPairF32 FreqF32;  // the FP32 adjoint record type

struct __align__(16) FreqF64 {
    int32_t n[3];
    int32_t pad;
    double xi[3];
    double Gr, Gi;
    double pad2;
};
static_assert(sizeof(FreqF64) == 64, "FreqF64 layout");

constexpr int FWD_TILE = 128;   // triangles per shared-memory tile (FP32 forward)
constexpr int FWD_THREADS = 256;
constexpr int ADJ_FTILE = 256;  // frequencies per shared-memory tile (FP32 adjoint; 128 pair records)
constexpr int ADJ_THREADS = 128;
constexpr int F64_THREADS = 128;

// Accumulators per triangle in the adjoint: surface {a, b1[3], b2[3], b3[3]};
// volume {alpha[3], b1[3], b2[3], b3[3]}.
constexpr int NACC_SURF = 10;
constexpr int NACC_VOL = 12;

// Frequency source for the forward transform: explicit triples, or band indices into H
// (idx == nullptr means the identity band, m = index in H).
struct FreqSrc {
    const int32_t* nlist;  // [M][3] or nullptr
    const int32_t* idx;    // [M] band indices or nullptr
    const int64_t* dM;     // device band size (nullptr: use M)
    int64_t M;             // host-side upper bound / exact size
    int Nx, Ny, Nzh, Nz;
    FastDiv div_zh, div_y;  // divisions by Nzh and Ny for index decoding
    // grid dimensions and their divisors
    void set_dims(int nx, int ny, int nz) {
        Nx = nx;
        Ny = ny;
        Nz = nz;
        Nzh = nz / 2 + 1;
        div_zh = make_fastdiv((uint32_t)Nzh);
        div_y = make_fastdiv((uint32_t)ny);
    }
};
__device__ __forceinline__ void decode_h(int64_t idx, const FreqSrc& fs, int& nx, int& ny, int& nz) {
    decode_h_fast((uint32_t)idx, fs.div_zh, fs.div_y, fs.Nx, fs.Ny, nx, ny, nz);
}

struct Geom {
    double L[3];       // periods
    double origin[3];  // grid origin
};

// ---------------------------------------------------------------- launchers (return cudaGetLastError())
// Mesh transform (FP32 mixed path).
// S_part (nullable): room for fwd_partial_elems(fs.M, sm_count) partial spectra; when given, the
// triangle list of each frequency block is split so that the launch has about fwd_target_units
// units (at least ~4 triangle tiles per split) and the partial spectra are summed in a fixed order;
// when NULL every block takes the whole triangle list.
// n_t: real triangles; the records are padded with zeros to whole 64-record tiles.
cudaError_t launch_fwd_f32(int mode, const TriF32* tris, int64_t n_t, const FreqSrc& fs, const Geom& g,
                           const double* d_vol, float2* S, float2* S_part, int sm_count, int* d_err, cudaStream_t st);
size_t fwd_partial_elems(int64_t M_max, int sm_count);
// Work units the forward aims for on sm_count SMs (frequency blocks x triangle splits).
int fwd_target_units(int sm_count);
cudaError_t launch_adj_f32(int mode, const TriF32* tris, int64_t n_t, int64_t n_t_pad, const FreqF32* fr,
                           const int64_t* dM, int64_t M_max, float* partial, int n_chunks, int* d_err, cudaStream_t st);
int adj_chunks_f32(int64_t n_t, int64_t M_max, int sm_count);

// Batched (multi-job) persistent launches of the FP32 sums.
struct BatchFwdJob {
    const TriF32* tris;
    int n_tiles;  // 64-record tiles
    int last;     // real triangles in the last tile
    int mode;
    FreqSrc fs;
    float tp[3];
    const double* d_vol;
    float2* S;
    int splits;      // triangle splits per frequency block (fixed per job); > 1: partial spectra in S_part
    float2* S_part;  // [splits][M] with M the job's band size on the device
};
struct BatchAdjJob {
    const TriF32* tris;
    int64_t n_t, n_t_pad;
    const FreqPairF32* fr;
    const int64_t* dM;
    int64_t M_max;
    int mode;
    int chunk_tiles;  // frequency tiles per unit (fixed per job: results do not depend on the batch)
    float* partial;   // [chunks][10|12][n_t_pad]
};
struct BatchUnit {
    int job;
    int a;  // forward: frequency block; adjoint: triangle block
    int b;  // adjoint: frequency chunk
    int pad;
};
// One launch per label (mode: DM_SURFACE / DM_VOLUME); every unit's job must have that label.
// Forward units are (job, frequency block, triangle split); a job with splits > 1 needs
// launch_fwd_reduce_splits afterwards.
cudaError_t launch_fwd_batch_f32(int mode, const BatchFwdJob* jobs, const BatchUnit* units, int n_units, int* counter,
                                 int grid, int* d_err, cudaStream_t st);
cudaError_t launch_adj_batch_f32(int mode, const BatchAdjJob* jobs, const BatchUnit* units, int n_units, int* counter,
                                 int grid, int* d_err, cudaStream_t st);
// S[m] = sum over the `splits` partial spectra in S_part (fixed order, FP64), m < the band size.
cudaError_t launch_fwd_reduce_splits(const FreqSrc& fs, int splits, const float2* S_part, float2* S, int sm_count,
                                     cudaStream_t st);
int batch_blocks_per_sm_fwd(int mode);
int batch_blocks_per_sm_adj(int mode);
constexpr int FWD_BLOCK_FREQS = 2 * FWD_THREADS;  // band frequencies per forward block

// Triangle splits per forward frequency block: about `target` work units over the band's fb blocks,
// at most one per triangle tile and 64 in all (1 when target <= 0).
__host__ __device__ inline int fwd_splits(int64_t fb, int n_tiles, int target) {
    if (target <= 0 || fb <= 0) return 1;
    int64_t sp = (target + fb - 1) / fb;
    if (sp > n_tiles) sp = n_tiles;
    if (sp > 64) sp = 64;
    return sp < 1 ? 1 : (int)sp;
}
constexpr int FWD_REC_TILE = 64;                  // triangle records per forward pipeline stage

// ---------------------------------------------------------------- batched stages (fit server)
// One served job's arguments for the stage kernels that the server runs for every job of an
// iteration in one launch each (FP32 path). Each stage gives every job a block count fixed by the
// job's own sizes (and the device), so a job's results do not depend on the other jobs of a launch.
struct StageJob {
    int mode, psf_kind, loss_kind;
    int band;            // narrow band: the half spectrum is zeroed before the scatter
    int64_t n_v, n_t, n_t_pad, N, nH, M_pad;
    Geom g;
    double* V;
    const int32_t* F;
    const float* wts;
    TriF32* tris;
    double* params;      // [0..8] psf, [16] normaliser, [17] loss, [24..31] gather sums
    double* partial;     // per-block partial sums of the stage reductions
    FreqSrc fs;
    float2* S;
    const float2* S_part;  // [fsplits][M] partial spectra when fsplits > 1
    int fsplits;
    int rc_slices;       // slices of the chunk reduction (> 1: second pass over red)
    Cx<float>* spec;
    float* image;
    const float* target;
    float* resid;
    FreqPairF32* fr;
    const float* adjp;
    int n_chunks, nacc;
    double* acc;
    double* red;
    double* contrib;
    const int32_t* ptr;
    const int32_t* ent;
    double* dV;
    int vertex_adam;     // Adam on the vertices in the batched update (large-steps jobs run their own)
    double *mV, *vV, *ms, *vs, *hist;
    int64_t* d_step;     // Adam step t of the job's next step
    int64_t step0;
    double lr_v, lr_psf, b1, b2, eps, decay;
};

// Batched stage ids: offsets[s * (nj + 1) + j] is the first block of job j in stage s's launch
// (offsets[s * (nj + 1) + nj] = the launch's blocks).
enum BatchStage {
    BS_PREP, BS_FWDRED, BS_ZERO, BS_SCATTER, BS_LOSS, BS_GATHER, BS_REDUCE, BS_SLICES, BS_ASSEMBLE,
    BS_VGATHER, BS_ADAM, BS_COUNT
};
// Per-job block counts of every batched stage (the single-job launches' counts for the same sizes).
void batch_stage_blocks(const StageJob& J, int sm_count, int counts[BS_COUNT]);
// Slices of the chunk reduction of a job (launch_reduce_chunks' choice with the scratch given).
int reduce_slices_for(int64_t n_t, int nacc, int n_chunks, int sm_count);
// One launch per stage over the nj jobs of `jobs` (device table); total = offsets[s*(nj+1) + nj].
cudaError_t launch_batch_stage(int stage, const StageJob* jobs, const int* offsets, int nj, int total, int* d_err,
                               cudaStream_t st);
// Sums of the per-block partials of a stage into params: params[dst + k] = sum over the job's blocks b
// of partial[b * count + k], k < count (one block per (job, k)); flag_err: ERR_DEGENERATE when not > 0.
cudaError_t launch_batch_sum(const StageJob* jobs, const int* stage_offsets, int nj, int count, int dst, int* flag_err,
                             cudaStream_t st);
// End of a step for every job: Adam on sigma (lr_psf > 0) with the step t, hist[t - step0 - 1] = loss,
// losses[j] = loss, t += 1.
cudaError_t launch_batch_tick(const StageJob* jobs, int nj, double* losses, cudaStream_t st);

// Mesh transform (FP64 plain path).
cudaError_t launch_fwd_f64(int mode, const TriF64* tris, int64_t n_t, const FreqSrc& fs, const Geom& g,
                           const double* d_vol, double2* S, cudaStream_t st);
cudaError_t launch_adj_f64(int mode, const TriF64* tris, int64_t n_t, const FreqF64* fr, const int64_t* dM,
                           int64_t M_max, double* partial, int n_chunks, cudaStream_t st);
int adj_chunks_f64(int64_t n_t, int64_t M_max, int sm_count);

// Triangle records and per-triangle normaliser (area*density or signed volume).
template <class Rec>
cudaError_t launch_tri_prep(int mode, const double* V, int64_t n_v, const int32_t* F, int64_t n_t, const float* wts,
                            const Geom& g, Rec* rec, int64_t n_t_pad, double* norm_partial, int* n_blocks_out,
                            int* d_err, cudaStream_t st);

// Deterministic sum of `n` doubles into out[0] (one block).
cudaError_t launch_sum(const double* x, int64_t n, int stride, int count, double* out, cudaStream_t st);
// The mesh normaliser (sum of the triangle-record partials): as launch_sum, and ERR_DEGENERATE in
// d_err when it is not > 0 (zero total weighted area, non-positive enclosed volume).
cudaError_t launch_norm_sum(const double* x, int64_t n, double* out, int* d_err, cudaStream_t st);

// Narrow band: writes indices of H with h_hat > tau into idx (ordered), size into dM.
cudaError_t launch_band(const double* d_psf, int psf_kind, double tau, int Nx, int Ny, int Nz, const Geom& g,
                        int32_t* idx, int64_t* dM, int64_t* block_counts, cudaStream_t st);

// spec[H] = 0 outside the band, S_m / norm * h_hat / (Lx Ly Lz) on it.
template <class R>
cudaError_t launch_scatter(const Cx<R>* S, const FreqSrc& fs, const double* d_psf, int psf_kind,
                           const double* d_norm, const Geom& g, Cx<R>* spec, bool zero_first, cudaStream_t st);

// Loss and residual; per-block FP64 partials of the loss.
template <class R>
cudaError_t launch_loss(const R* I, const R* T, int64_t n, int kind, R* resid, double* partial, int* n_blocks_out,
                        cudaStream_t st);

// After the forward real DFT of the residual: build adjoint frequency records (Gw), and
// per-block partials of dL/dpsf (3 or 6) and of cq = sum Re(conj(Gu) u_hat).
template <class R, class FR>
cudaError_t launch_gather(int mode, const Cx<R>* spec, const Cx<R>* S, const FreqSrc& fs, const double* d_psf,
                          int psf_kind, const double* d_norm, const Geom& g, FR* fr, int64_t M_pad, double* partial,
                          int* n_blocks_out, cudaStream_t st);

// Raw adjoint records from a caller's G on explicit frequencies (dm_meshft_adjoint).
template <class R, class FR>
cudaError_t launch_prep_raw(int mode, const Cx<R>* G, const int32_t* nlist, int64_t M, const Geom& g, FR* fr,
                            int64_t M_pad, double* partial, int* n_blocks_out, cudaStream_t st);

// Sum per-chunk partial accumulators: acc[t][k] = sum_c partial[c][k][t]. M_max >= 0 (FP32 single-job
// adjoint): only the chunks that hold band tiles are read (the band size *dM, or M_max when dM is
// NULL; the others hold zeros); M_max < 0: every chunk.
// scratch (nullable): reduce_scratch_elems(sm_count) doubles; with it a mesh of few triangles splits the
// chunks into slices summed in a second, fixed-order pass (enough blocks for every SM).
template <class R>
cudaError_t launch_reduce_chunks(const R* partial, int n_chunks, int nacc, int64_t n_t, int64_t n_t_pad, double* acc,
                                 cudaStream_t st, const int64_t* dM = nullptr, int64_t M_max = -1,
                                 double* scratch = nullptr, int sm_count = 0);
size_t reduce_scratch_elems(int sm_count);

// Per-corner gradient contributions, then the per-vertex gather through the vertex star.
cudaError_t launch_assemble(int mode, const double* V, const int32_t* F, int64_t n_t, int64_t n_v, const float* wts,
                            const Geom& g, const double* acc, const double* d_coef, double* contrib, cudaStream_t st);
cudaError_t launch_csr(const int32_t* F, int64_t n_t, int64_t n_v, int32_t* cnt, int32_t* ptr, int32_t* ent,
                       int* d_err, cudaStream_t st);
cudaError_t launch_vertex_gather(const int32_t* ptr, const int32_t* ent, const double* contrib, int64_t n_v,
                                 double* dV, cudaStream_t st);

// Exclusive prefix sum of n counts into ptr[0..n] (ptr[n] = total); one CTA.
cudaError_t launch_scan_i32(const int32_t* cnt, int64_t n, int32_t* ptr, cudaStream_t st);

// Optimiser layer (optim.cu). Combinatorial Laplacian rows (unique neighbours, sorted) from
// the vertex star (sptr, ent of launch_csr); lcol needs room for 2 * (3 n_t) entries.
cudaError_t launch_laplacian(const int32_t* F, const int32_t* sptr, const int32_t* ent, int64_t n_v, int32_t* cnt,
                             int32_t* lptr, int32_t* lcol, int* d_err, cudaStream_t st);
// (1 + lam L) X = B for the 3 columns of [n_v][3] doubles; X is the start and the result;
// sub_into (nullable) -= X. work: pcg_work_elems(n_v) values of R (used when the vectors do
// not fit in shared memory). stats (nullable, device): total / most iterations, unconverged.
size_t pcg_work_elems(int64_t n_v);
template <class R>
cudaError_t launch_pcg(const int32_t* lptr, const int32_t* lcol, int64_t n_v, double lam, const double* B, double* X,
                       double* sub_into, R* work, double tol, int max_iter, unsigned long long* stats,
                       cudaStream_t st);
// Uniform Adam: m, v updated; delta = lr m_hat / (sqrt(max v_hat) + eps). part_max holds
// adam_uniform_partials(n) doubles. With d_step the step t is read from the device (step ignored), and
// decay != 1 makes the rate lr decay^(t-1).
int adam_uniform_partials(int64_t n);
cudaError_t launch_adam_uniform(const double* g, double* m, double* v, double* delta, int64_t n, double lr, double b1,
                                double b2, double eps, int64_t step, double* part_max, cudaStream_t st,
                                const int64_t* d_step = nullptr, double decay = 1.0);
// Sigma = C C^T into the covariance numbers of the device PSF parameters, and dL/dC from dL/dcov.
cudaError_t launch_chol_to_cov(const double* C, double* d_psf, cudaStream_t st);
cudaError_t launch_chol_grad(const double* C, const double* gcov, double* gC, cudaStream_t st);

// Adam update on n doubles; the _dev_step form reads the step t from the device and takes the rate
// lr decay^(t-1) (decay 1: constant), so that a captured step replays unchanged.
cudaError_t launch_adam(double* p, const double* g, double* m, double* v, int64_t n, double lr, double b1, double b2,
                        double eps, int64_t step, cudaStream_t st);
cudaError_t launch_adam_dev_step(double* p, const double* g, double* m, double* v, int64_t n, double lr, double b1,
                                 double b2, double eps, const int64_t* d_step, double decay, cudaStream_t st);
// hist[*d_step - step0 - 1] = *d_loss; ++*d_step (one thread)
cudaError_t launch_fit_tick(double* hist, const double* d_loss, int64_t* d_step, int64_t step0, cudaStream_t st);

// FFT (own: FP32 power-of-two lines in registers, otherwise a mixed-radix Stockham in shared memory).
struct FFTAxis {
    int N;
    int nf;
    int radix[16];
    const void* tw;  // N twiddles exp(-2 pi i k / N), double2 or float2
};
template <class R>
cudaError_t launch_c2r(const Cx<R>* spec_in, Cx<R>* work, R* out, int Nx, int Ny, int Nz, const FFTAxis* ax,
                       cudaStream_t st);
template <class R>
cudaError_t launch_r2c(const R* in, Cx<R>* spec_out, int Nx, int Ny, int Nz, const FFTAxis* ax, cudaStream_t st);
// Axis lengths the FFT takes: 1..FFT_MAX_N with prime factors 2, 3, 5, 7, 11, 13 (the shared memory of a
// pass, fft_smem_bytes, also has to fit the device: FP64 lines up to 2048).
constexpr int FFT_MAX_N = 4096;
bool fft_factor(int N, FFTAxis& a);
size_t fft_smem_bytes(int N, int elem_bytes);

// Batched FFT passes over the jobs of one line length: complex strided passes, or the real z passes.
struct FFTJob {
    const void* src;
    void* dst;
    FFTAxis ax;
    int64_t inner;  // strided: element stride of the lines; z passes: 0
    int64_t lines;  // strided: number of outer blocks of lines (the single-job pass's `outer`); z: lines
    int Nzh;
};
enum FFTPassKind { FFT_STRIDED = 0, FFT_Z_C2R = 1, FFT_Z_R2C = 2 };
// Blocks one job takes in a batched pass (the single-job pass's grid).
int64_t fft_pass_blocks(int kind, const FFTJob& j);
cudaError_t launch_fft_batch(int kind, int N, const FFTJob* jobs, const int* offsets, int nj, int total, int dir,
                             cudaStream_t st);


// Small helpers.
struct Params16 {
    double v[16];
};
// Write up to 16 doubles passed by value into device memory (stream ordered, no host staging).
cudaError_t launch_set_params(double* dst, Params16 p, int n, cudaStream_t st);

}  // namespace dm
