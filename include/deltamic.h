/*
 * deltamic.h — C ABI of the B300 (sm_103a) mesh-Fourier fluorescence renderer.
 *
 * The library renders a 3D fluorescence image from a triangle mesh and a
 * Gaussian PSF entirely in Fourier space and differentiates it:
 *
 *   u_hat(xi)  = S(xi) / |Lambda|,   S(xi) = sum_T int_T exp(-i x.xi) dS        (Eq. 5, 7-8)
 *   h_hat(xi)  = exp(-1/2 xi^T Sigma xi)                                        (Eq. 2)
 *   I_j        = (1/(Lx Ly Lz)) sum_{n in band} c_n Re(u_hat h_hat exp(i xi_n.x_j)) (Eq. 1)
 *   loss       = ||I - T||^2, its mean, or <(I - T)^2, T>                        (Sec. 5.1-5.2)
 *   dL/dV, dL/dSigma                                                            (Eq. 6, 9-10)
 *
 * Paper: S. Ichbiah, A. Sinha, F. Delbary, H. Turlier, "Inverse 3D Microscopy
 * Rendering for Cell Shape Inference with Active Mesh" (arXiv 2303.10440).
 *
 * Conventions shared by every call
 * --------------------------------
 * Grid: N = (Nx, Ny, Nz) voxels of size h; voxel j sits at origin + j*h; the
 *   image is periodic with period L = N*h. Real images are C-ordered [x][y][z].
 * Frequencies: xi_n = 2*pi*n/L (elementwise). The half spectrum H holds
 *   n_x in fftfreq(Nx), n_y in fftfreq(Ny), n_z in 0..Nz/2, stored C-ordered as
 *   [Nx][Ny][Nz/2+1] complex (index ix -> n_x = ix < (Nx+1)/2 ? ix : ix - Nx).
 *   c_n = 1 on the planes n_z = 0 and (even Nz) n_z = Nz/2, else 2.
 * Band: {n in H : h_hat(xi_n) > band_tau} (Sec. 5.1 narrow band); band_tau <= 0
 *   selects all of H. Band entries are ordered by their index in H.
 * Mesh: V[n_v][3] double, F[n_t][3] int32 (0-based), faces counter-clockwise
 *   seen from outside. label 0 = surface-labelled (density on the triangles,
 *   normalised by total area); label 1 = volume-labelled (uniform density inside
 *   a closed mesh, normalised by enclosed volume).
 * Precision (dm_options.precision): DM_FP64 computes everything in double and
 *   uses double image buffers; DM_FP32_MIXED runs the (frequency, triangle) sums
 *   in FP32 with exact integer phase reduction and compensated accumulation,
 *   keeps reductions in FP64, and uses float image buffers.
 * Memory: every pointer argument may be device memory or host memory; the
 *   library tells them apart with cudaPointerGetAttributes. Host inputs are
 *   copied to the context's workspace on the call's stream; host outputs are
 *   written back and the stream is synchronised before the call returns.
 *   The caller owns every buffer it passes; the library never frees them.
 * Streams: `stream` is a cudaStream_t (NULL = legacy default stream). All device
 *   work of a call is enqueued on it; device outputs are valid in stream order.
 * Errors: calls return DM_OK (0) or a negative dm_status; dm_last_error() gives
 *   a message. Faults detected on the device (a bad face index, a wait that
 *   timed out) are reported by the next call that synchronises, or by dm_sync().
 * Threads: a context is used by one host thread at a time.
 */
#ifndef DELTAMIC_H
#define DELTAMIC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t dm_status;
#define DM_OK 0
#define DM_ERR_ARG (-1)         /* null pointer, size <= 0, NaN/Inf, sigma <= 0, index out of range */
#define DM_ERR_OOM (-2)         /* device memory could not be reserved */
#define DM_ERR_DEGENERATE (-3)  /* zero total area (surface) or non-positive volume (volume mode) */
#define DM_ERR_OPEN_MESH (-4)   /* volume mode on a mesh that is not edge-manifold closed */
#define DM_ERR_TIMEOUT (-5)     /* a bounded device-side wait expired */
#define DM_ERR_CUDA (-6)        /* a CUDA runtime call failed */
#define DM_ERR_UNSUPPORTED (-7) /* grid axis longer than 4096 (FP64: 2048) or with a prime factor > 13,
                                   or a half spectrum of 2^31 entries or more */

#define DM_FP64 0
#define DM_FP32_MIXED 1

#define DM_SURFACE 0
#define DM_VOLUME 1

#define DM_LOSS_L2 0       /* sum_j (I_j - T_j)^2                   (Sec. 5.2) */
#define DM_LOSS_MSE 1      /* (1/N) sum_j (I_j - T_j)^2                        */
#define DM_LOSS_WEIGHTED 2 /* sum_j T_j (I_j - T_j)^2               (Sec. 5.1) */

#define DM_PSF_DIAG 0 /* Sigma = diag(sigma^2); gradient w.r.t. sigma[3]      */
#define DM_PSF_FULL 1 /* Sigma from cov = (xx, yy, zz, xy, xz, yz); gradient w.r.t. cov[6] */

typedef struct dm_ctx dm_ctx;

typedef struct {
    int32_t precision;     /* DM_FP64 or DM_FP32_MIXED */
    int32_t device;        /* CUDA device ordinal */
    int32_t no_graphs;     /* 0: dm_fit / dm_fit_resume capture one optimisation step as a CUDA graph
                            * and replay it; 1: enqueue every step's kernels one by one. Results are
                            * bitwise identical either way. */
} dm_options;

typedef struct {
    int32_t n[3];      /* voxels per axis; each axis 1..4096 (FP64 path: 1..2048) with prime factors
                          2, 3, 5, 7, 11, 13; Nx * Ny * (Nz/2 + 1) < 2^31 */
    double h[3];       /* voxel size per axis (> 0) */
    double origin[3];  /* position of voxel (0,0,0) */
} dm_grid;

typedef struct {
    int32_t kind;      /* DM_PSF_DIAG or DM_PSF_FULL */
    double sigma[3];   /* spatial standard deviations (kind DIAG), > 0 */
    double cov[6];     /* spatial covariance (kind FULL), positive definite */
    double band_tau;   /* narrow-band threshold on h_hat; <= 0 keeps the whole half spectrum */
} dm_psf;

typedef struct {
    const double* V;          /* [n_v][3] vertex positions */
    int64_t n_v;
    const int32_t* F;         /* [n_t][3] 0-based vertex indices, CCW from outside */
    int64_t n_t;
    const float* tri_weight;  /* optional [n_t] fluorophore density per triangle (NULL = 1);
                                 surface mode only (Sec. 3.3: interfaces carry density 2) */
    int32_t label;            /* DM_SURFACE or DM_VOLUME */
    int32_t reserved;
} dm_mesh;

/* ---------------------------------------------------------------- context */

/* Create a context bound to opt->device. *ctx receives the handle. */
dm_status dm_create(dm_ctx** ctx, const dm_options* opt);
/* Release the context and its workspace. Safe on NULL. */
dm_status dm_destroy(dm_ctx* ctx);
/* Message describing the last failure of a call on ctx ("" if none). Owned by ctx. */
const char* dm_last_error(const dm_ctx* ctx);
/* Bytes of device workspace a loss_and_grad call needs for this grid and mesh size. */
dm_status dm_workspace_size(const dm_ctx* ctx, const dm_grid* grid, int64_t n_v, int64_t n_t, size_t* bytes);
/* Grow the workspace to at least `bytes` now (so later calls do not allocate). */
dm_status dm_reserve(dm_ctx* ctx, size_t bytes);
/* Synchronise `stream` and report any device-side fault recorded since the last check. */
dm_status dm_sync(dm_ctx* ctx, void* stream);
/* Debug check of a mesh (host or device arrays; synchronises; ctx may be NULL for host arrays, and
 * then no GPU is needed): DM_ERR_ARG for a face index outside
 * [0, n_v), a non-finite vertex or density, or tri_weight with the volume label; DM_ERR_DEGENERATE
 * for a zero total (weighted) area or a non-positive enclosed volume; DM_ERR_OPEN_MESH when the
 * volume label's mesh is not closed and consistently oriented (every directed edge p -> q used
 * once, and q -> p once). The path itself raises DM_ERR_DEGENERATE from the device normaliser:
 * calls that synchronise (loss and gradients, fits) return it, asynchronous ones (render, stage
 * calls) at the next dm_sync. The fit server runs this check at submit. */
dm_status dm_check_mesh(dm_ctx* ctx, const dm_mesh* mesh);
/* Number of this library's kernels launched since the library was loaded (instrumentation). */
int64_t dm_kernel_launches(const dm_ctx* ctx);

/* Stage timing (instrumentation). While enabled, every call records a CUDA event pair on its
 * stream around each stage; dm_profile_read synchronises on them and returns, per stage,
 * the accumulated milliseconds and the number of timed executions since the previous read. */
#define DM_STAGE_PARAMS 0   /* PSF parameters to the device                 */
#define DM_STAGE_PREP 1     /* triangle records and normaliser (Sec. 4.1.2) */
#define DM_STAGE_BAND 2     /* narrow band (Sec. 5.1)                       */
#define DM_STAGE_FWD 3      /* mesh transform sum (Eq. 5, 7-8)              */
#define DM_STAGE_SCATTER 4  /* transfer-function multiply (Eq. 1-2)         */
#define DM_STAGE_C2R 5      /* inverse real 3D DFT                          */
#define DM_STAGE_LOSS 6     /* loss and residual (Sec. 5.1-5.2)             */
#define DM_STAGE_R2C 7      /* forward real 3D DFT of the residual          */
#define DM_STAGE_GATHER 8   /* adjoint records, dL/dpsf                     */
#define DM_STAGE_ADJ 9      /* mesh transform adjoint sum (Eq. 9-10)        */
#define DM_STAGE_REDUCE 10  /* per-chunk sums                               */
#define DM_STAGE_ASSEMBLE 11 /* per-vertex gradient (Eq. 6)                 */
#define DM_STAGE_ADAM 12    /* optimiser update                             */
#define DM_STAGE_SMOOTH 13  /* large-steps smoothing solves (Sec. 5.1)      */
#define DM_NUM_STAGES 14
dm_status dm_profile_enable(dm_ctx* ctx, int32_t enable);
/* ms, calls: arrays of DM_NUM_STAGES (either may be NULL). */
dm_status dm_profile_read(dm_ctx* ctx, double* ms, int64_t* calls);

/* Failure-detection check with no counterpart in the paper: runs one block whose threads wait on an
 * mbarrier that nothing completes, with the bounded wait the mesh-transform pipelines use, limited to
 * limit_ns (<= 2 s). *status = DM_ERR_TIMEOUT when the wait expired and was reported through the
 * device error flag (the expected outcome), DM_OK otherwise; the context stays usable. Synchronises. */
dm_status dm_probe_wait_timeout(int32_t device, uint64_t limit_ns, int32_t* status);

/* ---------------------------------------------------------------- stages */

/* Narrow band (Sec. 5.1). Writes the band's indices into H (ordered) to idx_out
 * (nullable; capacity Nx*Ny*(Nz/2+1)) and its size to *M_out (host). Synchronises. */
dm_status dm_band(dm_ctx* ctx, const dm_psf* psf, const dm_grid* grid, int32_t* idx_out, int64_t* M_out, void* stream);

/* Raw mesh spectrum at M integer frequencies (Eq. 5 numerator, Eq. 7-8):
 *   S_m = sum_T w_T int_T exp(-i x'.xi_m) dS   (surface; w_T = tri_weight or 1)
 *   S_m = int_V exp(-i x'.xi_m) dV            (volume)
 * with x' = x - grid.origin and xi_m = 2 pi n_m / L. freq_n: [M][3] int32.
 * S_out: [M] complex (interleaved re, im) in double (DM_FP64) or float. */
dm_status dm_meshft(dm_ctx* ctx, const dm_mesh* mesh, const dm_grid* grid, const int32_t* freq_n, int64_t M,
                    void* S_out, void* stream);

/* Vertex adjoint of dm_meshft: dV[v] = sum_m Re(conj(G_m) dS_m/dv) (Eq. 9-10 summed per
 * vertex, without the area quotient of Eq. 6). G: [M] complex (double or float, as S_out).
 * dV_out: [n_v][3] double, overwritten. */
dm_status dm_meshft_adjoint(dm_ctx* ctx, const dm_mesh* mesh, const dm_grid* grid, const int32_t* freq_n,
                            int64_t M, const void* G, double* dV_out, void* stream);

/* Unnormalised inverse real 3D DFT: out_j = sum_{n in H} c_n Re(spec_n exp(2 pi i n.j/N)).
 * spec: [Nx][Ny][Nz/2+1] complex, image: [Nx][Ny][Nz] real (double or float). spec is only read; a
 * device spectrum that does not overlap the image is read in place, any other is copied first. */
dm_status dm_c2r(dm_ctx* ctx, const dm_grid* grid, const void* spec, void* image, void* stream);
/* Unnormalised forward real 3D DFT onto H: spec_n = sum_j image_j exp(-2 pi i n.j/N). */
dm_status dm_r2c(dm_ctx* ctx, const dm_grid* grid, const void* image, void* spec, void* stream);

/* Allocation-free variant of dm_meshft (FP32 mixed path). The paper has no counterpart: this
 * entry point exists for callers that may not allocate device memory after start-up (a server
 * that reserves all of its memory up front, or a framework that owns every allocation through
 * its own pool), since dm_meshft grows a context workspace with cudaMalloc. It takes no context
 * and calls no allocating routine: its scratch (triangle records, partial sums, fault flags) is a
 * file-scope device array of DM_NOALLOC_SCRATCH_BYTES per device, held until the process exits.
 * Arguments as dm_meshft; S_out is [M] complex float. Every pointer must be device memory of
 * the calling thread's current device. fault_flags (nullable, device int) receives 0, or bit 2
 * for a face index outside [0, n_v), bit 4 for a non-finite vertex, bit 8 for a zero total area
 * or non-positive enclosed volume (stream ordered).
 * Returns DM_ERR_ARG for NULL or host pointers, n_t > DM_NOALLOC_MAX_TRIANGLES or bad sizes;
 * DM_ERR_CUDA if a launch fails. The first call on a device is a start-up warm-up: it looks up the
 * scratch address (once per device) and, with CUDA's lazy module loading, is when the kernels'
 * modules and the scratch array are placed on the device, so it can still take device memory or
 * fail under memory pressure; make it at start-up, before any stream capture. Later calls take no
 * device memory. All calls on a device share the scratch: calls that overlap on the GPU race and
 * must be serialised by the caller. */
#define DM_NOALLOC_MAX_TRIANGLES 65536
#define DM_NOALLOC_SCRATCH_BYTES (8u << 20)
dm_status dm_meshft_noalloc(const dm_mesh* mesh, const dm_grid* grid, const int32_t* freq_n, int64_t M, void* S_out,
                            int32_t* fault_flags, void* stream);

/* ---------------------------------------------------------------- renderer */

/* Render the image (Eq. 1 via I_hat = u_hat h_hat) into image[Nx][Ny][Nz]. */
dm_status dm_render(dm_ctx* ctx, const dm_mesh* mesh, const dm_psf* psf, const dm_grid* grid, void* image,
                    void* stream);

/* Render, compare with target[Nx][Ny][Nz] under `loss`, and differentiate.
 * L (nullable): 1 double. dV (nullable): [n_v][3] double dL/dV.
 * dpsf (nullable): 3 doubles dL/dsigma (DIAG) or 6 doubles dL/dcov (FULL).
 * image_out (nullable): the rendered image. */
dm_status dm_loss_and_grad(dm_ctx* ctx, const dm_mesh* mesh, const dm_psf* psf, const dm_grid* grid,
                           const void* target, int32_t loss, double* L, double* dV, double* dpsf, void* image_out,
                           void* stream);

/* Adjoint of dm_render for a given dL/dI[Nx][Ny][Nz] (autograd backward): the spectrum
 * is recomputed, not stored. dV, dpsf as in dm_loss_and_grad (nullable). */
dm_status dm_render_adjoint(dm_ctx* ctx, const dm_mesh* mesh, const dm_psf* psf, const dm_grid* grid,
                            const void* dL_dI, double* dV, double* dpsf, void* stream);

/* ---------------------------------------------------------------- optimisation */

/* One Adam step (Kingma & Ba) on n doubles, in place: m, v are the moment buffers
 * (device, caller-owned, zero before step 1); step >= 1. */
dm_status dm_adam(dm_ctx* ctx, double* param, const double* grad, double* m, double* v, int64_t n, double lr,
                  double beta1, double beta2, double eps, int64_t step, void* stream);

typedef struct {
    int32_t steps;        /* Adam iterations */
    int32_t loss;         /* DM_LOSS_* */
    double lr_vertex;     /* Adam learning rate for vertex positions */
    double lr_psf;        /* Adam learning rate for sigma (0 = keep the PSF fixed) */
    double beta1, beta2, eps;
} dm_fit_options;

/* Optimiser state of a fit, for checkpoint and resume. The arrays are HOST memory owned by the
 * caller ([n_v][3] doubles each); warm may be NULL (Adam fits have no smoothing solves). */
typedef struct {
    int64_t step;        /* optimiser steps taken so far (Adam's bias correction continues from here) */
    double sigma[3];     /* current PSF sigma */
    double m_sigma[3];   /* Adam moments of sigma */
    double v_sigma[3];
    double* m_V;         /* [n_v][3] first moments of the vertex optimiser */
    double* v_V;         /* [n_v][3] second moments */
    double* warm;        /* [2][n_v][3] starting guesses of the two large-steps smoothing solves, or NULL */
} dm_fit_state;

/* Fit vertices (and sigma when lr_psf > 0) to target by Adam, entirely on the device.
 * V_io: [n_v][3] initial positions in, fitted positions out. psf_io->sigma updated in place
 * (host struct). loss_history (nullable): [steps] doubles, the loss before each step. */
dm_status dm_fit(dm_ctx* ctx, const dm_mesh* mesh, double* V_io, dm_psf* psf_io, const dm_grid* grid,
                 const void* target, const dm_fit_options* opt, double* loss_history, void* stream);

/* dm_fit continued from a checkpoint: state (host, in/out) holds the optimiser state after
 * state->step steps (zeros and step 0 for a fresh start) and V_io the vertices at that point; the
 * call takes opt->steps more steps, sigma starts from state->sigma, and the state after the last
 * step is written back (moments, sigma, step). A fit of a + b steps equals a fit of a steps
 * followed by a resumed fit of b steps, bit for bit. Synchronises the stream. */
dm_status dm_fit_resume(dm_ctx* ctx, const dm_mesh* mesh, double* V_io, dm_psf* psf_io, const dm_grid* grid,
                        const void* target, const dm_fit_options* opt, dm_fit_state* state, double* loss_history,
                        void* stream);

/* ---------------------------------------------------------------- staggered fit
 * Section 5.1 ("A staggered optimization scheme") and Section 5.2 ("PSF optimization step"):
 * rounds of (a) shape steps on the narrow band of the current PSF, PSF held, then (b) PSF
 * steps on every frequency of the half spectrum, shape held. The shape optimiser of the paper
 * is the large-steps update v <- v - eta (1 + lambda L)^-2 dL/dv with uniform Adam (lambda = 50,
 * after Nicolet et al. 2021); the PSF optimiser is Adam on the covariance. */
#define DM_OPT_ADAM 0        /* plain Adam on the vertex positions */
#define DM_OPT_LARGE_STEPS 1 /* uniform Adam on u = (1 + lambda L) v */

/* Smoothing solve of the large-steps update: X = (1 + lambda L)^-1 B, L the combinatorial
 * Laplacian of the mesh edges (degree minus adjacency over the unique undirected edges of F).
 * F: [n_t][3] int32 (host or device). B, X: DEVICE [n_v][3] doubles; X holds the starting
 * guess on entry (zeros are fine) and the solution on return. Jacobi-preconditioned conjugate
 * gradients in the context's precision, one CTA per coordinate, until ||r|| <= tol ||b||
 * (tol <= 0: 1e-6 for DM_FP32_MIXED, 1e-12 for DM_FP64) or max_iter iterations (<= 0: 2000).
 * iters (nullable, host int64[3]): total iterations of the 3 columns, the most in one column,
 * and the number of columns that stopped at max_iter. Synchronises the stream when iters is
 * given. DM_ERR_ARG: NULL or host B / X, lambda < 0, indices out of range. */
dm_status dm_smooth_solve(dm_ctx* ctx, const int32_t* F, int64_t n_t, int64_t n_v, double lambda, const double* B,
                          double* X, double tol, int32_t max_iter, int64_t* iters, void* stream);

/* One uniform-Adam step (Nicolet et al. 2021) on n DEVICE doubles: m, v (zero before step 1)
 * are updated in place and delta[i] = lr m_hat[i] / (sqrt(max_j v_hat[j]) + eps); the caller
 * moves the parameter by -delta. */
dm_status dm_adam_uniform(dm_ctx* ctx, const double* grad, double* m, double* v, double* delta, int64_t n, double lr,
                          double beta1, double beta2, double eps, int64_t step, void* stream);

typedef struct {
    int32_t rounds;       /* staggered rounds */
    int32_t shape_steps;  /* (a) steps per round: narrow band (psf band_tau), PSF held */
    int32_t psf_steps;    /* (b) steps per round: whole half spectrum, shape held */
    int32_t shape_loss;   /* DM_LOSS_*; the paper's shape loss is DM_LOSS_WEIGHTED */
    int32_t psf_loss;     /* DM_LOSS_*; the paper's PSF loss is DM_LOSS_L2 */
    int32_t optimizer;    /* DM_OPT_LARGE_STEPS (the paper's) or DM_OPT_ADAM */
    double lr_vertex;     /* step size of the vertex optimiser */
    double lr_psf;        /* Adam step size on the Cholesky factor of Sigma */
    double lambda;        /* smoothing weight of the large-steps update (the paper: 50) */
    double beta1, beta2, eps;
    double cg_tol;        /* smoothing-solve tolerance (<= 0: the dm_smooth_solve default) */
    int32_t cg_max_iter;  /* smoothing-solve iteration limit (<= 0: 2000) */
    int32_t reserved;
} dm_stagger_options;

typedef struct {
    int64_t cg_iterations;   /* over all smoothing solves and columns */
    int64_t cg_max;          /* most iterations of one column */
    int64_t cg_unconverged;  /* columns that stopped at cg_max_iter */
} dm_stagger_stats;

/* The staggered fit, entirely on the device. The covariance is parameterised as
 * Sigma = C C^T, C lower triangular (6 numbers), and Adam acts on C; a DIAG psf_io starts from
 * C = diag(sigma). On return psf_io is DM_PSF_FULL with the fitted cov (and sigma = the square
 * roots of its diagonal); band_tau is kept. V_io: [n_v][3] host or device, fitted positions
 * out. shape_loss (nullable): [rounds * shape_steps] doubles, psf_loss (nullable):
 * [rounds * psf_steps] doubles, each the loss before its step. stats nullable.
 * DM_ERR_ARG: a covariance that is not positive definite, bad options. */
dm_status dm_fit_staggered(dm_ctx* ctx, const dm_mesh* mesh, double* V_io, dm_psf* psf_io, const dm_grid* grid,
                           const void* target, const dm_stagger_options* opt, double* shape_loss, double* psf_loss,
                           dm_stagger_stats* stats, void* stream);

/* ---------------------------------------------------------------- fit server
 * Continuous batching of many shape fits on one GPU (FP32 mixed path). Jobs are copied at
 * submit into a queue; an engine thread admits them first-in first-out whenever a slot
 * (max_jobs) and room in the server's device arena (memory_bytes) are free, keeps each
 * admitted job's mesh, Adam state, band and target on the device, and runs iterations in
 * which every active job advances by one Adam step: the forward and adjoint mesh-transform
 * sums of all active jobs run as one persistent launch each, over a work list of
 * (job, frequency block) and (job, triangle block, frequency chunk) units. A job's results do
 * not depend on which other jobs share its iterations. Finished jobs leave at the end of an
 * iteration and queued jobs join at the start of the next. */
typedef struct dm_server dm_server;

#define DM_SCHED_FIFO 0     /* admit in arrival order; every admitted job advances every iteration */
#define DM_SCHED_SHORTEST 1 /* admit and advance the jobs with the least remaining work first */

typedef struct {
    int32_t device;        /* CUDA device ordinal */
    int32_t max_jobs;      /* jobs resident on the device at once (batch slots), >= 1 */
    size_t memory_bytes;   /* device arena for job state (0: half of the free device memory) */
    int32_t chunk_tiles;   /* most adjoint frequency tiles (256 frequencies) per work unit (0: 1024); each
                              job uses fewer so that it alone yields ~64 units per SM */
    int32_t policy;        /* DM_SCHED_FIFO or DM_SCHED_SHORTEST */
    double batch_terms;    /* DM_SCHED_SHORTEST: most triangle-frequency terms per step that one iteration
                              takes on (jobs in policy order; the first always runs); <= 0: no limit */
    double max_wait_s;     /* a resident job that has not advanced for this long goes first (<= 0: never) */
    int32_t no_graphs;     /* nonzero: enqueue every iteration directly. Otherwise (the default) the second
                              iteration over an unchanged set of advanced jobs is captured as a CUDA graph and
                              replayed until the set changes; results are the same either way */
} dm_server_options;

typedef struct {
    const double* V;       /* host [n_v][3] initial vertices (copied at submit) */
    int64_t n_v;
    const int32_t* F;      /* host [n_t][3] (copied at submit) */
    int64_t n_t;
    const float* target;   /* host [Nx][Ny][Nz] target image (copied at submit) */
    dm_grid grid;
    dm_psf psf;            /* DM_PSF_DIAG; sigma is the initial value when fit.lr_psf > 0 */
    dm_fit_options fit;    /* steps, loss, learning rates, Adam constants */
    int32_t label;         /* DM_SURFACE or DM_VOLUME */
    int32_t optimizer;     /* vertex optimiser: DM_OPT_ADAM or DM_OPT_LARGE_STEPS (uniform Adam on
                              u = (1 + lambda L) v, FP32 smoothing solves, tolerance 1e-6) */
    double lambda;         /* large-steps smoothing weight (<= 0: 50) */
    double lr_decay;       /* step t (from 1, continuing across resume) uses fit.lr_vertex * lr_decay^(t-1)
                              and likewise lr_psf; 0 or 1: constant rates; otherwise in (0, 1) */
    const float* tri_weight; /* host [n_t] per-triangle densities (copied at submit; surface label only,
                              finite, >= 0, not all 0), or NULL for density 1 (Sec. 3.3, 4.1) */
    const dm_fit_state* resume; /* NULL, or the state of a preempted job (copied at submit): V is then
                              that job's vertices and fit.steps the steps still to take */
} dm_job;

#define DM_JOB_QUEUED 0
#define DM_JOB_RUNNING 1
#define DM_JOB_DONE 2
#define DM_JOB_FAILED 3
#define DM_JOB_PREEMPTED 4

typedef struct {
    int32_t state;         /* DM_JOB_* */
    int32_t steps_done;
    double t_submit;       /* seconds on the server clock */
    double t_start;        /* admission */
    double t_end;          /* completion */
    double last_loss;      /* loss before the last completed step */
} dm_job_status;

typedef struct {
    int64_t iterations;    /* engine iterations run */
    int64_t jobs_done;
    int64_t job_steps;     /* Adam steps summed over jobs */
    int64_t peak_active;   /* largest batch */
    double busy_s;         /* engine time spent in iterations */
    size_t bytes_in_use;   /* arena bytes held by admitted jobs */
    size_t bytes_peak;
    size_t bytes_total;
    int64_t graph_replays; /* iterations run as one launch of a captured CUDA graph */
} dm_server_stats;

/* Create a server and start its engine thread. */
dm_status dm_server_create(dm_server** srv, const dm_server_options* opt);
/* Validate and enqueue a job (all inputs copied). DM_ERR_OOM if it can never fit the arena. */
dm_status dm_server_submit(dm_server* srv, const dm_job* job, int64_t* job_id);
dm_status dm_server_status(dm_server* srv, int64_t job_id, dm_job_status* out);
/* Block until the job is done (or failed); DM_ERR_TIMEOUT after timeout_s seconds (< 0: forever). */
dm_status dm_server_wait(dm_server* srv, int64_t job_id, double timeout_s);
/* Copy a finished job's results (host buffers, each nullable): V_out [n_v][3], sigma_out [3],
 * loss_history [steps]; then forget the job. */
dm_status dm_server_result(dm_server* srv, int64_t job_id, double* V_out, double* sigma_out, double* loss_history);
/* Checkpoint: stop a queued or running job at the next iteration boundary and copy its vertices
 * (V_out, host [n_v][3]) and optimiser state (state: host arrays of the caller, each nullable) out;
 * the job ends in DM_JOB_PREEMPTED and is forgotten. Submitting it again with dm_job.resume = state,
 * V = V_out and fit.steps = the steps still to take continues it bit for bit. Waits up to timeout_s
 * (< 0: no limit; DM_ERR_TIMEOUT). DM_ERR_ARG: unknown job, or it finished first (take its result). */
dm_status dm_server_preempt(dm_server* srv, int64_t job_id, double timeout_s, double* V_out, dm_fit_state* state);
dm_status dm_server_get_stats(dm_server* srv, dm_server_stats* out);
/* Seconds since the server was created (the clock of dm_job_status). */
double dm_server_clock(const dm_server* srv);
/* Stop the engine after its current iteration and release every resource. */
dm_status dm_server_shutdown(dm_server* srv);

#ifdef __cplusplus
}
#endif

#endif /* DELTAMIC_H */
