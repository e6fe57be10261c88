// Internal helpers shared by the C ABI (api.cu) and the fit server (serve.cu): the
// context, workspace arena, FFT plans, stage timing and the single-job pipeline.
#pragma once

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "../../include/deltamic.h"
#include "dm_kernels.cuh"

namespace dm {
extern std::atomic<int64_t> g_launches;  // kernels launched by this library (instrumentation)
// Host-side mesh validation (mesh_check.cu): DM_OK, DM_ERR_ARG, DM_ERR_DEGENERATE or, for the volume
// label, DM_ERR_OPEN_MESH; *why receives the reason.
dm_status check_mesh_host(const double* V, int64_t n_v, const int32_t* F, int64_t n_t, const float* W, int label,
                          std::string* why);
}
using namespace dm;


struct dm_ctx {
    int precision = DM_FP32_MIXED;
    int device = 0;
    int sm_count = 148;
    std::string err;
    int* d_err = nullptr;
    char* ws = nullptr;
    size_t ws_cap = 0;
    std::map<int, void*> tw32, tw64;  // FFT twiddle tables per length
    bool graphs = true;               // replay captured fit steps (dm_options.no_graphs == 0)
    cudaStream_t cap = nullptr;       // stream used only to capture graphs (nothing runs on it)
    // stage timing
    bool prof = false;
    std::vector<cudaEvent_t> ev_pool;
    struct Pending {
        int stage;
        cudaEvent_t a, b;
    };
    std::vector<Pending> pending;
    double prof_ms[DM_NUM_STAGES] = {0};
    int64_t prof_calls[DM_NUM_STAGES] = {0};
    cudaEvent_t take_event() {
        if (ev_pool.empty()) {
            cudaEvent_t e;
            cudaEventCreate(&e);
            return e;
        }
        cudaEvent_t e = ev_pool.back();
        ev_pool.pop_back();
        return e;
    }
};

namespace {

inline dm_status fail(dm_ctx* c, dm_status code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    if (c) c->err = buf;
    return code;
}

#define CK(expr)                                                                                       \
    do {                                                                                               \
        cudaError_t e_ = (expr);                                                                       \
        if (e_ != cudaSuccess) return fail(ctx, DM_ERR_CUDA, "%s: %s", #expr, cudaGetErrorString(e_)); \
    } while (0)

#define LAUNCH(n, ...)             \
    do {                           \
        CK((__VA_ARGS__));         \
        g_launches += (n);         \
    } while (0)

// Records a CUDA event pair around a stage when profiling is enabled.
struct Stage {
    dm_ctx* c;
    int id;
    cudaStream_t st;
    cudaEvent_t a = nullptr;
    Stage(dm_ctx* ctx, int stage, cudaStream_t s) : c(ctx), id(stage), st(s) {
        if (c->prof) {
            a = c->take_event();
            cudaEventRecord(a, st);
        }
    }
    ~Stage() {
        if (a) {
            cudaEvent_t b = c->take_event();
            cudaEventRecord(b, st);
            c->pending.push_back({id, a, b});
        }
    }
};

// Captures body(stream) into an executable CUDA graph on the context's capture stream, in thread-
// local capture mode (other threads' CUDA calls are unaffected); nothing runs during the capture.
// Returns false, leaving no error state behind, when the capture or the instantiation fails; the
// caller then runs the body directly.
template <class Body>
bool capture_graph(dm_ctx* ctx, const Body& body, cudaGraphExec_t* exec) {
    *exec = nullptr;
    if (!ctx->cap && cudaStreamCreateWithFlags(&ctx->cap, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        ctx->cap = nullptr;
        return false;
    }
    if (cudaStreamBeginCapture(ctx->cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    const std::string err0 = ctx->err;
    const dm_status bs = body(ctx->cap);
    cudaGraph_t g = nullptr;
    const cudaError_t ce = cudaStreamEndCapture(ctx->cap, &g);
    bool ok = bs == DM_OK && ce == cudaSuccess && g != nullptr;
    if (ok && cudaGraphInstantiate(exec, g, 0) != cudaSuccess) {
        ok = false;
        *exec = nullptr;
    }
    if (g) cudaGraphDestroy(g);
    if (!ok) {
        cudaGetLastError();
        ctx->err = err0;
    }
    return ok;
}

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        cudaGetDevice(&prev);
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur = -1;
        cudaGetDevice(&cur);
        if (prev >= 0 && cur != prev) cudaSetDevice(prev);
    }
};

bool is_device_ptr(const void* p) {
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

struct Arena {
    char* base = nullptr;
    size_t off = 0;
    template <class T>
    T* take(size_t n) {
        off = (off + 255) & ~(size_t)255;
        T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
        off += n * sizeof(T);
        return p;
    }
};

dm_status ensure_ws(dm_ctx* ctx, size_t bytes) {
    if (bytes <= ctx->ws_cap) return DM_OK;
    if (ctx->ws) {
        cudaDeviceSynchronize();
        cudaFree(ctx->ws);
        ctx->ws = nullptr;
        ctx->ws_cap = 0;
    }
    size_t want = bytes + bytes / 8 + (1 << 20);
    cudaError_t e = cudaMalloc(&ctx->ws, want);
    if (e != cudaSuccess) {
        cudaGetLastError();
        ctx->ws = nullptr;
        return fail(ctx, DM_ERR_OOM, "workspace of %zu bytes: %s", want, cudaGetErrorString(e));
    }
    ctx->ws_cap = want;
    return DM_OK;
}

dm_status check_dev_err(dm_ctx* ctx, cudaStream_t st) {
    CK(cudaStreamSynchronize(st));
    int h = 0;
    CK(cudaMemcpy(&h, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (h) {
        CK(cudaMemset(ctx->d_err, 0, sizeof(int)));
        if (h & ERR_BAD_INDEX) return fail(ctx, DM_ERR_ARG, "face index outside [0, n_v)");
        if (h & ERR_NONFINITE) return fail(ctx, DM_ERR_ARG, "non-finite vertex position");
        if (h & ERR_TIMEOUT) return fail(ctx, DM_ERR_TIMEOUT, "a bounded device wait expired");
        if (h & ERR_DEGENERATE)
            return fail(ctx, DM_ERR_DEGENERATE, "zero total (weighted) area, or non-positive enclosed volume");
    }
    return DM_OK;
}

int64_t round_up(int64_t x, int64_t m) { return (x + m - 1) / m * m; }

// FFT plans: twiddle tables are computed on the host in double and cached per length.
dm_status fft_axes(dm_ctx* ctx, const int n[3], FFTAxis ax[3]) {
    const bool f64 = ctx->precision == DM_FP64;
    int max_smem = 0;
    CK(cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, ctx->device));
    for (int a = 0; a < 3; ++a) {
        if (!fft_factor(n[a], ax[a]))
            return fail(ctx, DM_ERR_UNSUPPORTED,
                        "grid axis %d has length %d (need 1..%d with prime factors 2, 3, 5, 7, 11, 13)", a, n[a],
                        FFT_MAX_N);
        if (fft_smem_bytes(n[a], f64 ? 16 : 8) > (size_t)max_smem)
            return fail(ctx, DM_ERR_UNSUPPORTED, "grid axis %d of length %d is too long for the %s FFT", a, n[a],
                        f64 ? "FP64" : "FP32");
        auto& cache = f64 ? ctx->tw64 : ctx->tw32;
        auto it = cache.find(n[a]);
        if (it == cache.end()) {
            const int N = n[a];
            std::vector<double> w(2 * (size_t)N);
            for (int k = 0; k < N; ++k) {
                // exp(-2 pi i k / N)
                const double ang = -2.0 * M_PI * (double)k / (double)N;
                w[2 * k] = cos(ang);
                w[2 * k + 1] = sin(ang);
            }
            void* d = nullptr;
            const size_t bytes = (size_t)N * (f64 ? 16 : 8);
            CK(cudaMalloc(&d, bytes));
            if (f64) {
                CK(cudaMemcpy(d, w.data(), bytes, cudaMemcpyHostToDevice));
            } else {
                std::vector<float> wf(w.begin(), w.end());
                CK(cudaMemcpy(d, wf.data(), bytes, cudaMemcpyHostToDevice));
            }
            it = cache.emplace(N, d).first;
        }
        ax[a].tw = it->second;
    }
    return DM_OK;
}

dm_status check_grid(dm_ctx* ctx, const dm_grid* g) {
    if (!g) return fail(ctx, DM_ERR_ARG, "grid is NULL");
    for (int a = 0; a < 3; ++a) {
        if (g->n[a] < 1) return fail(ctx, DM_ERR_ARG, "grid.n[%d] = %d", a, g->n[a]);
        if (!(g->h[a] > 0) || !std::isfinite(g->h[a])) return fail(ctx, DM_ERR_ARG, "grid.h[%d] must be > 0", a);
        if (!std::isfinite(g->origin[a])) return fail(ctx, DM_ERR_ARG, "grid.origin is not finite");
    }
    // half-spectrum indices are 32-bit
    if ((int64_t)g->n[0] * g->n[1] * (g->n[2] / 2 + 1) >= ((int64_t)1 << 31))
        return fail(ctx, DM_ERR_UNSUPPORTED, "grid of %d x %d x %d: half spectrum too large", g->n[0], g->n[1], g->n[2]);
    return DM_OK;
}

dm_status check_psf(dm_ctx* ctx, const dm_psf* p) {
    if (!p) return fail(ctx, DM_ERR_ARG, "psf is NULL");
    if (p->kind == DM_PSF_DIAG) {
        for (int a = 0; a < 3; ++a)
            if (!(p->sigma[a] > 0) || !std::isfinite(p->sigma[a])) return fail(ctx, DM_ERR_ARG, "sigma must be > 0");
    } else if (p->kind == DM_PSF_FULL) {
        const double* c = p->cov;
        for (int k = 0; k < 6; ++k)
            if (!std::isfinite(c[k])) return fail(ctx, DM_ERR_ARG, "cov is not finite");
        // positive definite by leading principal minors (Sylvester)
        const double m1 = c[0], m2 = c[0] * c[1] - c[3] * c[3];
        const double m3 = c[0] * (c[1] * c[2] - c[5] * c[5]) - c[3] * (c[3] * c[2] - c[5] * c[4]) +
                          c[4] * (c[3] * c[5] - c[1] * c[4]);
        if (!(m1 > 0 && m2 > 0 && m3 > 0)) return fail(ctx, DM_ERR_ARG, "cov must be positive definite");
    } else {
        return fail(ctx, DM_ERR_ARG, "psf.kind = %d", p->kind);
    }
    if (!std::isfinite(p->band_tau)) return fail(ctx, DM_ERR_ARG, "band_tau is not finite");
    return DM_OK;
}

dm_status check_mesh(dm_ctx* ctx, const dm_mesh* m, bool F_on_host) {
    if (!m || !m->V || !m->F) return fail(ctx, DM_ERR_ARG, "mesh, V or F is NULL");
    if (m->n_v < 3 || m->n_t < 1) return fail(ctx, DM_ERR_ARG, "mesh needs n_v >= 3 and n_t >= 1");
    if (m->n_t > (int64_t)1 << 28 || m->n_v > (int64_t)1 << 29) return fail(ctx, DM_ERR_ARG, "mesh too large");
    if (m->label != DM_SURFACE && m->label != DM_VOLUME) return fail(ctx, DM_ERR_ARG, "label = %d", m->label);
    if (m->label == DM_VOLUME && m->tri_weight) return fail(ctx, DM_ERR_ARG, "tri_weight is for surface mode only");
    if (F_on_host) {
        for (int64_t i = 0; i < 3 * m->n_t; ++i)
            if (m->F[i] < 0 || m->F[i] >= m->n_v) return fail(ctx, DM_ERR_ARG, "F[%lld] = %d out of range", (long long)i, m->F[i]);
    }
    return DM_OK;
}

// ------------------------------------------------------------------ pipeline
enum Job { JOB_RENDER = 1, JOB_LOSS = 2, JOB_ADJOINT = 4 };

struct Sizes {
    bool f64;
    int sm_count;
    int64_t nH, N, n_v, n_t, n_t_pad, M_max, M_pad;
    int n_chunks, nacc;
    bool band;  // narrow band active (tau > 0)
    bool fwd_split = true;  // room for the forward's triangle-split partial spectra (not in served jobs)
};

struct Bufs {
    double* d_params;  // [0..8] psf, [16] norm, [17] loss, [18] coef, [24..31] psf grad
    double* partial;   // block partials (norm / loss / gather)
    void* tris;
    void* S;
    void* S_part;  // FP32 forward: partial spectra of its triangle splits
    void* spec;
    void* image;
    void* resid;
    void* fr;
    void* adjp;
    double* acc;
    double* red;  // chunk-reduction slices (reduce_scratch_elems)
    double* contrib;
    int32_t* cnt;
    int32_t* ptr;
    int32_t* ent;
    int32_t* band_idx;
    int64_t* band_counts;
    int64_t* dM;
    // staging of host inputs
    double* V;
    int32_t* F;
    float* wts;
    void* target;
    double* dV;
};

size_t layout(const Sizes& z, Arena& A, Bufs& b, bool stageV, bool stageF, bool stageW, bool stageT, bool stageDV) {
    const size_t R = z.f64 ? 8 : 4;
    b.d_params = A.take<double>(32);
    const int64_t nparts = std::max<int64_t>({(z.n_t_pad + 255) / 256, 4096, (z.M_pad + 255) / 256 * 8});
    b.partial = A.take<double>(nparts);
    b.tris = A.take<char>(z.n_t_pad * (z.f64 ? sizeof(TriF64) : sizeof(TriF32)));
    b.S = A.take<char>(z.M_max * 2 * R);
    b.S_part = z.f64 || !z.fwd_split ? nullptr
                                     : A.take<char>(fwd_partial_elems(z.M_max, z.sm_count) * sizeof(float2));
    b.spec = A.take<char>(z.nH * 2 * R);
    b.image = A.take<char>(z.N * R);
    b.resid = A.take<char>(z.N * R);
    b.fr = A.take<char>(z.M_pad * (z.f64 ? sizeof(FreqF64) : sizeof(FreqPairF32) / 2));
    b.adjp = A.take<char>((size_t)z.n_chunks * z.nacc * z.n_t_pad * R);
    b.acc = A.take<double>(z.n_t * z.nacc);
    b.red = A.take<double>(reduce_scratch_elems(z.sm_count));
    b.contrib = A.take<double>(z.n_t * 9);
    b.cnt = A.take<int32_t>(z.n_v);
    b.ptr = A.take<int32_t>(z.n_v + 1);
    b.ent = A.take<int32_t>(3 * z.n_t);
    b.band_idx = z.band ? A.take<int32_t>(z.nH) : nullptr;
    b.band_counts = z.band ? A.take<int64_t>((z.nH + 255) / 256 + 1) : nullptr;
    b.dM = A.take<int64_t>(1);
    b.V = stageV ? A.take<double>(3 * z.n_v) : nullptr;
    b.F = stageF ? A.take<int32_t>(3 * z.n_t) : nullptr;
    b.wts = stageW ? A.take<float>(z.n_t) : nullptr;
    b.target = stageT ? A.take<char>(z.N * R) : nullptr;
    b.dV = A.take<double>(3 * z.n_v);  // gradient sink when dV is host memory or not requested
    (void)stageDV;
    return A.off + 256;
}

Sizes make_sizes(const dm_ctx* ctx, const dm_grid* g, int64_t n_v, int64_t n_t, bool band, int label) {
    Sizes z;
    z.f64 = ctx->precision == DM_FP64;
    z.sm_count = ctx->sm_count;
    const int Nzh = g->n[2] / 2 + 1;
    z.nH = (int64_t)g->n[0] * g->n[1] * Nzh;
    z.N = (int64_t)g->n[0] * g->n[1] * g->n[2];
    z.n_v = n_v;
    z.n_t = n_t;
    z.n_t_pad = round_up(n_t, FWD_TILE);
    z.M_max = z.nH;
    z.M_pad = round_up(z.nH, ADJ_FTILE);
    z.nacc = label == DM_VOLUME ? NACC_VOL : NACC_SURF;
    z.n_chunks = z.f64 ? adj_chunks_f64(n_t, z.M_max, ctx->sm_count) : adj_chunks_f32(n_t, z.M_max, ctx->sm_count);
    z.band = band;
    return z;
}

Geom make_geom(const dm_grid* g) {
    Geom G;
    for (int a = 0; a < 3; ++a) {
        G.L[a] = g->n[a] * g->h[a];
        G.origin[a] = g->origin[a];
    }
    return G;
}

Params16 psf_params(const dm_psf* p) {
    Params16 q;
    memset(&q, 0, sizeof(q));
    for (int a = 0; a < 3; ++a) q.v[a] = p->sigma[a];
    for (int k = 0; k < 6; ++k) q.v[3 + k] = p->cov[k];
    return q;
}

// Device inputs of one pipeline run (all device pointers).
struct Inputs {
    const double* V;
    const int32_t* F;
    const float* wts;
    int64_t n_v, n_t;
    int label;
    const void* target;  // JOB_LOSS
    int loss;
    const void* dLdI;    // JOB_ADJOINT without loss
};

struct Outputs {
    void* image;     // device, nullable (else internal)
    double* dV;      // device, nullable
    bool want_grad;  // run the adjoint
    bool psf_only = false;  // stop after dL/dpsf (no vertex adjoint)
};

// Runs the full chain on device buffers; results: b.d_params[17] = L, [24..29] = dpsf, out.dV.
template <class R>
dm_status pipeline(dm_ctx* ctx, const Sizes& z, Bufs& b, const Inputs& in, const dm_psf* psf, const dm_grid* grid,
                   int jobs, const Outputs& out, cudaStream_t st, bool psf_on_device) {
    using TriRec = typename std::conditional<sizeof(R) == 4, TriF32, TriF64>::type;
    using FreqRec = typename std::conditional<sizeof(R) == 4, FreqF32, FreqF64>::type;
    const Geom G = make_geom(grid);
    const int mode = in.label;
    double* d_psf = b.d_params;
    double* d_norm = b.d_params + 16;
    double* d_loss = b.d_params + 17;
    double* d_coef = b.d_params + 18;
    double* d_dpsf = b.d_params + 24;
    if (!psf_on_device) {
        Stage sg(ctx, DM_STAGE_PARAMS, st);
        LAUNCH(1, launch_set_params(d_psf, psf_params(psf), 9, st));
    }

    // triangle records and normaliser
    {
        Stage sg(ctx, DM_STAGE_PREP, st);
        int nb = 0;
        LAUNCH(1, launch_tri_prep<TriRec>(mode, in.V, in.n_v, in.F, in.n_t, in.wts, G, (TriRec*)b.tris, z.n_t_pad,
                                          b.partial, &nb, ctx->d_err, st));
        LAUNCH(1, launch_norm_sum(b.partial, nb, d_norm, ctx->d_err, st));
    }

    // narrow band
    FreqSrc fs;
    fs.nlist = nullptr;
    fs.set_dims(grid->n[0], grid->n[1], grid->n[2]);
    fs.M = z.nH;
    if (z.band) {
        Stage sg(ctx, DM_STAGE_BAND, st);
        LAUNCH(3, launch_band(d_psf, psf->kind, psf->band_tau, grid->n[0], grid->n[1], grid->n[2], G, b.band_idx,
                              b.dM, b.band_counts, st));
        fs.idx = b.band_idx;
        fs.dM = b.dM;
    } else {
        fs.idx = nullptr;
        fs.dM = nullptr;
    }

    // forward mesh transform
    {
        Stage sg(ctx, DM_STAGE_FWD, st);
        if (sizeof(R) == 4)
            LAUNCH(2, launch_fwd_f32(mode, (const TriF32*)b.tris, z.n_t, fs, G, d_norm, (float2*)b.S,
                                     (float2*)b.S_part, z.sm_count, ctx->d_err, st));
        else
            LAUNCH(1, launch_fwd_f64(mode, (const TriF64*)b.tris, z.n_t, fs, G, d_norm, (double2*)b.S, st));
    }

    FFTAxis ax[3];
    dm_status s = fft_axes(ctx, grid->n, ax);
    if (s != DM_OK) return s;
    R* image = (R*)(out.image ? out.image : b.image);
    if ((jobs & JOB_RENDER) || (jobs & JOB_LOSS)) {
        {
            Stage sg(ctx, DM_STAGE_SCATTER, st);
            LAUNCH(1, launch_scatter<R>((const Cx<R>*)b.S, fs, d_psf, psf->kind, d_norm, G, (Cx<R>*)b.spec, z.band,
                                        st));
        }
        Stage sg(ctx, DM_STAGE_C2R, st);
        LAUNCH(3, launch_c2r<R>((const Cx<R>*)b.spec, (Cx<R>*)b.spec, image, grid->n[0], grid->n[1], grid->n[2], ax,
                                st));
    }
    const R* resid = nullptr;
    if (jobs & JOB_LOSS) {
        Stage sg(ctx, DM_STAGE_LOSS, st);
        int nl = 0;
        LAUNCH(1, launch_loss<R>(image, (const R*)in.target, z.N, in.loss, (R*)b.resid, b.partial, &nl, st));
        LAUNCH(1, launch_sum(b.partial, nl, 1, 1, d_loss, st));
        resid = (const R*)b.resid;
    } else if (jobs & JOB_ADJOINT) {
        resid = (const R*)in.dLdI;
    }
    if (!out.want_grad || !resid) return DM_OK;

    // adjoint: forward DFT of the residual, adjoint records, per-triangle sums
    {
        Stage sg(ctx, DM_STAGE_R2C, st);
        LAUNCH(3, launch_r2c<R>(resid, (Cx<R>*)b.spec, grid->n[0], grid->n[1], grid->n[2], ax, st));
    }
    {
        Stage sg(ctx, DM_STAGE_GATHER, st);
        int ng = 0;
        LAUNCH(1, launch_gather<R, FreqRec>(mode, (const Cx<R>*)b.spec, (const Cx<R>*)b.S, fs, d_psf, psf->kind, d_norm,
                                            G, (FreqRec*)b.fr, z.M_pad, b.partial, &ng, st));
        LAUNCH(1, launch_sum(b.partial, ng, 8, 8, d_dpsf, st));  // [24..29] dpsf, [30] coef
    }
    if (out.psf_only) return DM_OK;
    {
        Stage sg(ctx, DM_STAGE_ADJ, st);
        if (sizeof(R) == 4)
            LAUNCH(1, launch_adj_f32(mode, (const TriF32*)b.tris, z.n_t, z.n_t_pad, (const FreqF32*)b.fr, fs.dM,
                                     z.M_max, (float*)b.adjp, z.n_chunks, ctx->d_err, st));
        else
            LAUNCH(1, launch_adj_f64(mode, (const TriF64*)b.tris, z.n_t, (const FreqF64*)b.fr, fs.dM, z.M_max,
                                     (double*)b.adjp, z.n_chunks, st));
    }
    const int64_t tpad = sizeof(R) == 4 ? z.n_t_pad : z.n_t;
    {
        Stage sg(ctx, DM_STAGE_REDUCE, st);
        LAUNCH(1, launch_reduce_chunks<R>((const R*)b.adjp, z.n_chunks, z.nacc, z.n_t, tpad, b.acc, st,
                                          sizeof(R) == 4 ? fs.dM : nullptr, sizeof(R) == 4 ? z.M_max : -1, b.red,
                                          z.sm_count));
    }
    (void)d_coef;
    Stage sg(ctx, DM_STAGE_ASSEMBLE, st);
    LAUNCH(1, launch_assemble(mode, in.V, in.F, z.n_t, z.n_v, in.wts, G, b.acc, d_dpsf + 6, b.contrib, st));
    LAUNCH(4, launch_csr(in.F, z.n_t, z.n_v, b.cnt, b.ptr, b.ent, ctx->d_err, st));
    LAUNCH(1, launch_vertex_gather(b.ptr, b.ent, b.contrib, z.n_v, out.dV, st));
    return DM_OK;
}

}  // namespace
