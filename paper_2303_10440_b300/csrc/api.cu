// C ABI of the renderer (include/deltamic.h): contexts, workspace, host/device
// staging, and the orchestration of the stage kernels into render, loss_and_grad,
// render_adjoint and the on-device fit loop.
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

using namespace dm;

namespace {
std::atomic<int64_t> g_launches{0};
}

struct dm_ctx {
    int precision = DM_FP32_MIXED;
    int device = 0;
    int sm_count = 148;
    std::string err;
    int* d_err = nullptr;
    char* ws = nullptr;
    size_t ws_cap = 0;
    std::map<int, void*> tw32, tw64;  // FFT twiddle tables per length
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

dm_status fail(dm_ctx* c, dm_status code, const char* fmt, ...) {
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
    }
    return DM_OK;
}

int64_t round_up(int64_t x, int64_t m) { return (x + m - 1) / m * m; }

// FFT plans: twiddle tables are computed on the host in double and cached per length.
dm_status fft_axes(dm_ctx* ctx, const int n[3], FFTAxis ax[3]) {
    const bool f64 = ctx->precision == DM_FP64;
    for (int a = 0; a < 3; ++a) {
        if (!fft_factor(n[a], ax[a]))
            return fail(ctx, DM_ERR_UNSUPPORTED, "grid axis %d has length %d (need 1..1024 with factors 2,3,5)", a,
                        n[a]);
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
    int64_t nH, N, n_v, n_t, n_t_pad, M_max, M_pad;
    int n_chunks, nacc;
    bool band;  // narrow band active (tau > 0)
};

struct Bufs {
    double* d_params;  // [0..8] psf, [16] norm, [17] loss, [18] coef, [24..31] psf grad
    double* partial;   // block partials (norm / loss / gather)
    void* tris;
    void* S;
    void* spec;
    void* image;
    void* resid;
    void* fr;
    void* adjp;
    double* acc;
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
    b.spec = A.take<char>(z.nH * 2 * R);
    b.image = A.take<char>(z.N * R);
    b.resid = A.take<char>(z.N * R);
    b.fr = A.take<char>(z.M_pad * (z.f64 ? sizeof(FreqF64) : sizeof(FreqPairF32) / 2));
    b.adjp = A.take<char>((size_t)z.n_chunks * z.nacc * z.n_t_pad * R);
    b.acc = A.take<double>(z.n_t * z.nacc);
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
        LAUNCH(1, launch_sum(b.partial, nb, 1, 1, d_norm, st));
    }

    // narrow band
    FreqSrc fs;
    fs.nlist = nullptr;
    fs.Nx = grid->n[0];
    fs.Ny = grid->n[1];
    fs.Nz = grid->n[2];
    fs.Nzh = grid->n[2] / 2 + 1;
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
            LAUNCH(1, launch_fwd_f32(mode, (const TriF32*)b.tris, z.n_t_pad, fs, G, d_norm, (float2*)b.S, ctx->d_err,
                                     st));
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
        LAUNCH(1, launch_reduce_chunks<R>((const R*)b.adjp, z.n_chunks, z.nacc, z.n_t, tpad, b.acc, st));
    }
    (void)d_coef;
    Stage sg(ctx, DM_STAGE_ASSEMBLE, st);
    LAUNCH(1, launch_assemble(mode, in.V, in.F, z.n_t, z.n_v, in.wts, G, b.acc, d_dpsf + 6, b.contrib, st));
    LAUNCH(4, launch_csr(in.F, z.n_t, z.n_v, b.cnt, b.ptr, b.ent, ctx->d_err, st));
    LAUNCH(1, launch_vertex_gather(b.ptr, b.ent, b.contrib, z.n_v, out.dV, st));
    return DM_OK;
}

// Shared front end of render / loss_and_grad / render_adjoint.
dm_status run(dm_ctx* ctx, const dm_mesh* mesh, const dm_psf* psf, const dm_grid* grid, int jobs, const void* target,
              int loss, const void* dLdI, double* L, double* dV, double* dpsf, void* image, void* stream_v) {
    if (!ctx) return DM_ERR_ARG;
    ctx->err.clear();
    DeviceGuard dg(ctx->device);
    cudaStream_t st = (cudaStream_t)stream_v;
    dm_status s;
    if ((s = check_grid(ctx, grid)) != DM_OK) return s;
    if ((s = check_psf(ctx, psf)) != DM_OK) return s;
    const bool V_dev = is_device_ptr(mesh ? mesh->V : nullptr);
    const bool F_dev = is_device_ptr(mesh ? mesh->F : nullptr);
    if ((s = check_mesh(ctx, mesh, !F_dev)) != DM_OK) return s;
    const bool W_dev = mesh->tri_weight ? is_device_ptr(mesh->tri_weight) : true;
    if ((jobs & JOB_LOSS) && !target) return fail(ctx, DM_ERR_ARG, "target is NULL");
    if ((jobs & JOB_LOSS) && (loss < 0 || loss > 2)) return fail(ctx, DM_ERR_ARG, "loss = %d", loss);
    if ((jobs & JOB_ADJOINT) && !dLdI) return fail(ctx, DM_ERR_ARG, "dL_dI is NULL");
    const bool T_dev = target ? is_device_ptr(target) : true;
    const bool D_dev = dLdI ? is_device_ptr(dLdI) : true;
    const bool I_dev = image ? is_device_ptr(image) : true;
    const bool dV_dev = dV ? is_device_ptr(dV) : true;
    const bool f64 = ctx->precision == DM_FP64;
    const bool band = psf->band_tau > 0;

    Sizes z = make_sizes(ctx, grid, mesh->n_v, mesh->n_t, band, mesh->label);
    Arena A;
    Bufs b;
    const bool stageT = (target && !T_dev) || (dLdI && !D_dev);
    const size_t need = layout(z, A, b, !V_dev, !F_dev, !W_dev, stageT, dV && !dV_dev);
    if ((s = ensure_ws(ctx, need)) != DM_OK) return s;
    A.base = ctx->ws;
    A.off = 0;
    layout(z, A, b, !V_dev, !F_dev, !W_dev, stageT, dV && !dV_dev);

    const size_t R = f64 ? 8 : 4;
    Inputs in;
    in.V = mesh->V;
    in.F = mesh->F;
    in.wts = mesh->tri_weight;
    in.n_v = mesh->n_v;
    in.n_t = mesh->n_t;
    in.label = mesh->label;
    in.target = target;
    in.loss = loss;
    in.dLdI = dLdI;
    if (!V_dev) {
        CK(cudaMemcpyAsync(b.V, mesh->V, 3 * mesh->n_v * sizeof(double), cudaMemcpyHostToDevice, st));
        in.V = b.V;
    }
    if (!F_dev) {
        CK(cudaMemcpyAsync(b.F, mesh->F, 3 * mesh->n_t * sizeof(int32_t), cudaMemcpyHostToDevice, st));
        in.F = b.F;
    }
    if (!W_dev) {
        CK(cudaMemcpyAsync(b.wts, mesh->tri_weight, mesh->n_t * sizeof(float), cudaMemcpyHostToDevice, st));
        in.wts = b.wts;
    }
    if (target && !T_dev) {
        CK(cudaMemcpyAsync(b.target, target, z.N * R, cudaMemcpyHostToDevice, st));
        in.target = b.target;
    }
    if (dLdI && !D_dev) {
        CK(cudaMemcpyAsync(b.target, dLdI, z.N * R, cudaMemcpyHostToDevice, st));
        in.dLdI = b.target;
    }
    Outputs out;
    out.image = (image && I_dev) ? image : nullptr;
    out.want_grad = (dV != nullptr || dpsf != nullptr) && (jobs & (JOB_LOSS | JOB_ADJOINT));
    out.dV = (dV && dV_dev) ? dV : b.dV;

    if (f64)
        s = pipeline<double>(ctx, z, b, in, psf, grid, jobs, out, st, false);
    else
        s = pipeline<float>(ctx, z, b, in, psf, grid, jobs, out, st, false);
    if (s != DM_OK) return s;

    bool sync = false;
    if (image && !I_dev) {
        CK(cudaMemcpyAsync(image, b.image, z.N * R, cudaMemcpyDeviceToHost, st));
        sync = true;
    }
    if (dV && !dV_dev) {
        CK(cudaMemcpyAsync(dV, b.dV, 3 * mesh->n_v * sizeof(double), cudaMemcpyDeviceToHost, st));
        sync = true;
    }
    const int npsf = psf->kind == DM_PSF_FULL ? 6 : 3;
    if (L) {
        if (is_device_ptr(L)) {
            CK(cudaMemcpyAsync(L, b.d_params + 17, sizeof(double), cudaMemcpyDeviceToDevice, st));
        } else {
            CK(cudaMemcpyAsync(L, b.d_params + 17, sizeof(double), cudaMemcpyDeviceToHost, st));
            sync = true;
        }
    }
    if (dpsf && out.want_grad) {
        if (is_device_ptr(dpsf)) {
            CK(cudaMemcpyAsync(dpsf, b.d_params + 24, npsf * sizeof(double), cudaMemcpyDeviceToDevice, st));
        } else {
            CK(cudaMemcpyAsync(dpsf, b.d_params + 24, npsf * sizeof(double), cudaMemcpyDeviceToHost, st));
            sync = true;
        }
    }
    if (sync) return check_dev_err(ctx, st);
    return DM_OK;
}

}  // namespace

// ======================================================================= C ABI
extern "C" {

dm_status dm_create(dm_ctx** out, const dm_options* opt) {
    if (!out) return DM_ERR_ARG;
    *out = nullptr;
    dm_ctx* ctx = new dm_ctx();
    if (opt) {
        if (opt->precision != DM_FP64 && opt->precision != DM_FP32_MIXED) {
            delete ctx;
            return DM_ERR_ARG;
        }
        ctx->precision = opt->precision;
        ctx->device = opt->device;
    }
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ctx->device < 0 || ctx->device >= ndev) {
        cudaGetLastError();
        delete ctx;
        return DM_ERR_CUDA;
    }
    DeviceGuard dg(ctx->device);
    cudaDeviceProp p;
    if (cudaGetDeviceProperties(&p, ctx->device) == cudaSuccess) ctx->sm_count = p.multiProcessorCount;
    if (cudaMalloc(&ctx->d_err, sizeof(int)) != cudaSuccess || cudaMemset(ctx->d_err, 0, sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        delete ctx;
        return DM_ERR_CUDA;
    }
    *out = ctx;
    return DM_OK;
}

dm_status dm_destroy(dm_ctx* ctx) {
    if (!ctx) return DM_OK;
    DeviceGuard dg(ctx->device);
    cudaDeviceSynchronize();
    if (ctx->ws) cudaFree(ctx->ws);
    if (ctx->d_err) cudaFree(ctx->d_err);
    for (auto& kv : ctx->tw32) cudaFree(kv.second);
    for (auto& kv : ctx->tw64) cudaFree(kv.second);
    for (auto& p : ctx->pending) {
        cudaEventDestroy(p.a);
        cudaEventDestroy(p.b);
    }
    for (auto e : ctx->ev_pool) cudaEventDestroy(e);
    delete ctx;
    return DM_OK;
}

const char* dm_last_error(const dm_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

int64_t dm_kernel_launches(const dm_ctx* ctx) {
    (void)ctx;
    return g_launches.load();
}

dm_status dm_workspace_size(const dm_ctx* ctx, const dm_grid* grid, int64_t n_v, int64_t n_t, size_t* bytes) {
    if (!ctx || !grid || !bytes || n_v < 1 || n_t < 1) return DM_ERR_ARG;
    Sizes z = make_sizes(ctx, grid, n_v, n_t, true, DM_VOLUME);
    Arena A;
    Bufs b;
    *bytes = layout(z, A, b, true, true, true, true, true);
    return DM_OK;
}

dm_status dm_profile_enable(dm_ctx* ctx, int32_t enable) {
    if (!ctx) return DM_ERR_ARG;
    ctx->prof = enable != 0;
    return DM_OK;
}

dm_status dm_profile_read(dm_ctx* ctx, double* ms, int64_t* calls) {
    if (!ctx) return DM_ERR_ARG;
    DeviceGuard dg(ctx->device);
    for (auto& p : ctx->pending) {
        float t = 0.f;
        cudaEventSynchronize(p.b);
        if (cudaEventElapsedTime(&t, p.a, p.b) == cudaSuccess) {
            ctx->prof_ms[p.stage] += t;
            ctx->prof_calls[p.stage] += 1;
        }
        cudaGetLastError();
        ctx->ev_pool.push_back(p.a);
        ctx->ev_pool.push_back(p.b);
    }
    ctx->pending.clear();
    for (int k = 0; k < DM_NUM_STAGES; ++k) {
        if (ms) ms[k] = ctx->prof_ms[k];
        if (calls) calls[k] = ctx->prof_calls[k];
        ctx->prof_ms[k] = 0.0;
        ctx->prof_calls[k] = 0;
    }
    return DM_OK;
}

dm_status dm_reserve(dm_ctx* ctx, size_t bytes) {
    if (!ctx) return DM_ERR_ARG;
    DeviceGuard dg(ctx->device);
    return ensure_ws(ctx, bytes);
}

dm_status dm_sync(dm_ctx* ctx, void* stream) {
    if (!ctx) return DM_ERR_ARG;
    DeviceGuard dg(ctx->device);
    return check_dev_err(ctx, (cudaStream_t)stream);
}

dm_status dm_render(dm_ctx* ctx, const dm_mesh* mesh, const dm_psf* psf, const dm_grid* grid, void* image,
                    void* stream) {
    if (!image) return fail(ctx, DM_ERR_ARG, "image is NULL");
    return run(ctx, mesh, psf, grid, JOB_RENDER, nullptr, 0, nullptr, nullptr, nullptr, nullptr, image, stream);
}

dm_status dm_loss_and_grad(dm_ctx* ctx, const dm_mesh* mesh, const dm_psf* psf, const dm_grid* grid,
                           const void* target, int32_t loss, double* L, double* dV, double* dpsf, void* image_out,
                           void* stream) {
    return run(ctx, mesh, psf, grid, JOB_LOSS, target, loss, nullptr, L, dV, dpsf, image_out, stream);
}

dm_status dm_render_adjoint(dm_ctx* ctx, const dm_mesh* mesh, const dm_psf* psf, const dm_grid* grid,
                            const void* dL_dI, double* dV, double* dpsf, void* stream) {
    return run(ctx, mesh, psf, grid, JOB_ADJOINT, nullptr, 0, dL_dI, nullptr, dV, dpsf, nullptr, stream);
}

dm_status dm_band(dm_ctx* ctx, const dm_psf* psf, const dm_grid* grid, int32_t* idx_out, int64_t* M_out,
                  void* stream) {
    if (!ctx) return DM_ERR_ARG;
    ctx->err.clear();
    DeviceGuard dg(ctx->device);
    dm_status s;
    if ((s = check_grid(ctx, grid)) != DM_OK) return s;
    if ((s = check_psf(ctx, psf)) != DM_OK) return s;
    if (!M_out) return fail(ctx, DM_ERR_ARG, "M_out is NULL");
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t nH = (int64_t)grid->n[0] * grid->n[1] * (grid->n[2] / 2 + 1);
    Arena A;
    double* d_psf = A.take<double>(16);
    int32_t* idx = A.take<int32_t>(nH);
    int64_t* counts = A.take<int64_t>((nH + 255) / 256 + 1);
    int64_t* dM = A.take<int64_t>(1);
    if ((s = ensure_ws(ctx, A.off + 256)) != DM_OK) return s;
    A.base = ctx->ws;
    A.off = 0;
    d_psf = A.take<double>(16);
    idx = A.take<int32_t>(nH);
    counts = A.take<int64_t>((nH + 255) / 256 + 1);
    dM = A.take<int64_t>(1);
    const Geom G = make_geom(grid);
    LAUNCH(1, launch_set_params(d_psf, psf_params(psf), 9, st));
    const double tau = psf->band_tau > 0 ? psf->band_tau : -1.0;  // tau <= 0: every h_hat > -1
    LAUNCH(3, launch_band(d_psf, psf->kind, tau, grid->n[0], grid->n[1], grid->n[2], G, idx, dM, counts, st));
    int64_t M = 0;
    CK(cudaMemcpyAsync(&M, dM, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    *M_out = M;
    if (idx_out) {
        CK(cudaMemcpyAsync(idx_out, idx, M * sizeof(int32_t), cudaMemcpyDefault, st));
        CK(cudaStreamSynchronize(st));
    }
    return DM_OK;
}

namespace {

// Buffers of the raw mesh-transform calls (explicit frequency lists).
struct RawBufs {
    double* d_params;
    double* partial;
    void* tris;
    int32_t* nlist;
    void* S;
    void* G;
    void* fr;
    void* adjp;
    double* acc;
    double* contrib;
    int32_t* cnt;
    int32_t* ptr;
    int32_t* ent;
    double* V;
    int32_t* F;
    float* wts;
    double* dV;
};

size_t raw_layout(const dm_ctx* ctx, int64_t n_v, int64_t n_t, int64_t M, int label, Arena& A, RawBufs& b,
                  int* n_chunks_out) {
    const bool f64 = ctx->precision == DM_FP64;
    const size_t R = f64 ? 8 : 4;
    const int64_t n_t_pad = round_up(n_t, FWD_TILE);
    const int64_t M_pad = round_up(M, ADJ_FTILE);
    const int nacc = label == DM_VOLUME ? NACC_VOL : NACC_SURF;
    const int nc = f64 ? adj_chunks_f64(n_t, M, ctx->sm_count) : adj_chunks_f32(n_t, M, ctx->sm_count);
    *n_chunks_out = nc;
    b.d_params = A.take<double>(32);
    b.partial = A.take<double>(std::max<int64_t>({(n_t_pad + 255) / 256, (M_pad + 255) / 256 * 8, 64}));
    b.tris = A.take<char>(n_t_pad * (f64 ? sizeof(TriF64) : sizeof(TriF32)));
    b.nlist = A.take<int32_t>(3 * M);
    b.S = A.take<char>(M * 2 * R);
    b.G = A.take<char>(M * 2 * R);
    b.fr = A.take<char>(M_pad * (f64 ? sizeof(FreqF64) : sizeof(FreqPairF32) / 2));
    b.adjp = A.take<char>((size_t)nc * nacc * n_t_pad * R);
    b.acc = A.take<double>(n_t * nacc);
    b.contrib = A.take<double>(9 * n_t);
    b.cnt = A.take<int32_t>(n_v);
    b.ptr = A.take<int32_t>(n_v + 1);
    b.ent = A.take<int32_t>(3 * n_t);
    b.V = A.take<double>(3 * n_v);
    b.F = A.take<int32_t>(3 * n_t);
    b.wts = A.take<float>(n_t);
    b.dV = A.take<double>(3 * n_v);
    return A.off + 256;
}

dm_status raw_common(dm_ctx* ctx, const dm_mesh* mesh, const dm_grid* grid, const int32_t* freq_n, int64_t M,
                     RawBufs& b, int* n_chunks, const double** V, const int32_t** F, const float** W,
                     const int32_t** nl, cudaStream_t st) {
    dm_status s;
    if ((s = check_grid(ctx, grid)) != DM_OK) return s;
    const bool F_dev = is_device_ptr(mesh ? mesh->F : nullptr);
    if ((s = check_mesh(ctx, mesh, !F_dev)) != DM_OK) return s;
    if (!freq_n || M < 1) return fail(ctx, DM_ERR_ARG, "frequency list is empty");
    Arena A;
    const size_t need = raw_layout(ctx, mesh->n_v, mesh->n_t, M, mesh->label, A, b, n_chunks);
    if ((s = ensure_ws(ctx, need)) != DM_OK) return s;
    A.base = ctx->ws;
    A.off = 0;
    raw_layout(ctx, mesh->n_v, mesh->n_t, M, mesh->label, A, b, n_chunks);
    *V = mesh->V;
    *F = mesh->F;
    *W = mesh->tri_weight;
    *nl = freq_n;
    if (!is_device_ptr(mesh->V)) {
        CK(cudaMemcpyAsync(b.V, mesh->V, 3 * mesh->n_v * sizeof(double), cudaMemcpyHostToDevice, st));
        *V = b.V;
    }
    if (!F_dev) {
        CK(cudaMemcpyAsync(b.F, mesh->F, 3 * mesh->n_t * sizeof(int32_t), cudaMemcpyHostToDevice, st));
        *F = b.F;
    }
    if (mesh->tri_weight && !is_device_ptr(mesh->tri_weight)) {
        CK(cudaMemcpyAsync(b.wts, mesh->tri_weight, mesh->n_t * sizeof(float), cudaMemcpyHostToDevice, st));
        *W = b.wts;
    }
    if (!is_device_ptr(freq_n)) {
        CK(cudaMemcpyAsync(b.nlist, freq_n, 3 * M * sizeof(int32_t), cudaMemcpyHostToDevice, st));
        *nl = b.nlist;
    }
    const Geom G = make_geom(grid);
    const int64_t n_t_pad = round_up(mesh->n_t, FWD_TILE);
    int nb = 0;
    if (ctx->precision == DM_FP64)
        LAUNCH(1, launch_tri_prep<TriF64>(mesh->label, *V, mesh->n_v, *F, mesh->n_t, *W, G, (TriF64*)b.tris, n_t_pad,
                                          b.partial, &nb, ctx->d_err, st));
    else
        LAUNCH(1, launch_tri_prep<TriF32>(mesh->label, *V, mesh->n_v, *F, mesh->n_t, *W, G, (TriF32*)b.tris, n_t_pad,
                                          b.partial, &nb, ctx->d_err, st));
    LAUNCH(1, launch_sum(b.partial, nb, 1, 1, b.d_params + 16, st));
    return DM_OK;
}

}  // namespace

dm_status dm_meshft(dm_ctx* ctx, const dm_mesh* mesh, const dm_grid* grid, const int32_t* freq_n, int64_t M,
                    void* S_out, void* stream) {
    if (!ctx) return DM_ERR_ARG;
    ctx->err.clear();
    DeviceGuard dg(ctx->device);
    if (!S_out) return fail(ctx, DM_ERR_ARG, "S_out is NULL");
    cudaStream_t st = (cudaStream_t)stream;
    RawBufs b;
    int nc;
    const double* V;
    const int32_t* F;
    const float* W;
    const int32_t* nl;
    dm_status s = raw_common(ctx, mesh, grid, freq_n, M, b, &nc, &V, &F, &W, &nl, st);
    if (s != DM_OK) return s;
    const bool f64 = ctx->precision == DM_FP64;
    const size_t R = f64 ? 8 : 4;
    const bool S_dev = is_device_ptr(S_out);
    void* S = S_dev ? S_out : b.S;
    FreqSrc fs;
    fs.nlist = nl;
    fs.idx = nullptr;
    fs.dM = nullptr;
    fs.M = M;
    fs.Nx = grid->n[0];
    fs.Ny = grid->n[1];
    fs.Nz = grid->n[2];
    fs.Nzh = grid->n[2] / 2 + 1;
    const Geom G = make_geom(grid);
    if (f64)
        LAUNCH(1, launch_fwd_f64(mesh->label, (const TriF64*)b.tris, mesh->n_t, fs, G, b.d_params + 16, (double2*)S, st));
    else
        LAUNCH(1, launch_fwd_f32(mesh->label, (const TriF32*)b.tris, round_up(mesh->n_t, FWD_TILE), fs, G,
                                 b.d_params + 16, (float2*)S, ctx->d_err, st));
    if (!S_dev) {
        CK(cudaMemcpyAsync(S_out, b.S, M * 2 * R, cudaMemcpyDeviceToHost, st));
        return check_dev_err(ctx, st);
    }
    return DM_OK;
}

dm_status dm_meshft_adjoint(dm_ctx* ctx, const dm_mesh* mesh, const dm_grid* grid, const int32_t* freq_n, int64_t M,
                            const void* Gin, double* dV_out, void* stream) {
    if (!ctx) return DM_ERR_ARG;
    ctx->err.clear();
    DeviceGuard dg(ctx->device);
    if (!Gin || !dV_out) return fail(ctx, DM_ERR_ARG, "G or dV_out is NULL");
    cudaStream_t st = (cudaStream_t)stream;
    RawBufs b;
    int nc;
    const double* V;
    const int32_t* F;
    const float* W;
    const int32_t* nl;
    dm_status s = raw_common(ctx, mesh, grid, freq_n, M, b, &nc, &V, &F, &W, &nl, st);
    if (s != DM_OK) return s;
    const bool f64 = ctx->precision == DM_FP64;
    const size_t R = f64 ? 8 : 4;
    const void* Gd = Gin;
    if (!is_device_ptr(Gin)) {
        CK(cudaMemcpyAsync(b.G, Gin, M * 2 * R, cudaMemcpyHostToDevice, st));
        Gd = b.G;
    }
    const bool dV_dev = is_device_ptr(dV_out);
    double* dV = dV_dev ? dV_out : b.dV;
    const Geom G = make_geom(grid);
    const int64_t M_pad = round_up(M, ADJ_FTILE);
    const int64_t n_t_pad = round_up(mesh->n_t, FWD_TILE);
    const int nacc = mesh->label == DM_VOLUME ? NACC_VOL : NACC_SURF;
    int ng = 0;
    if (f64) {
        LAUNCH(1, launch_prep_raw<double, FreqF64>(mesh->label, (const Cx<double>*)Gd, nl, M, G, (FreqF64*)b.fr, M_pad,
                                                   b.partial, &ng, st));
    } else {
        LAUNCH(1, launch_prep_raw<float, FreqF32>(mesh->label, (const Cx<float>*)Gd, nl, M, G, (FreqF32*)b.fr, M_pad,
                                                  b.partial, &ng, st));
    }
    LAUNCH(1, launch_sum(b.partial, ng, 8, 8, b.d_params + 24, st));
    if (f64) {
        LAUNCH(1, launch_adj_f64(mesh->label, (const TriF64*)b.tris, mesh->n_t, (const FreqF64*)b.fr, nullptr, M,
                                 (double*)b.adjp, nc, st));
        LAUNCH(1, launch_reduce_chunks<double>((const double*)b.adjp, nc, nacc, mesh->n_t, mesh->n_t, b.acc, st));
    } else {
        LAUNCH(1, launch_adj_f32(mesh->label, (const TriF32*)b.tris, mesh->n_t, n_t_pad, (const FreqF32*)b.fr, nullptr,
                                 M, (float*)b.adjp, nc, ctx->d_err, st));
        LAUNCH(1, launch_reduce_chunks<float>((const float*)b.adjp, nc, nacc, mesh->n_t, n_t_pad, b.acc, st));
    }
    LAUNCH(1, launch_assemble(mesh->label, V, F, mesh->n_t, mesh->n_v, W, G, b.acc, b.d_params + 30, b.contrib, st));
    LAUNCH(4, launch_csr(F, mesh->n_t, mesh->n_v, b.cnt, b.ptr, b.ent, ctx->d_err, st));
    LAUNCH(1, launch_vertex_gather(b.ptr, b.ent, b.contrib, mesh->n_v, dV, st));
    (void)R;
    if (!dV_dev) {
        CK(cudaMemcpyAsync(dV_out, b.dV, 3 * mesh->n_v * sizeof(double), cudaMemcpyDeviceToHost, st));
        return check_dev_err(ctx, st);
    }
    return DM_OK;
}

static dm_status fft_call(dm_ctx* ctx, const dm_grid* grid, const void* in, void* out, bool inverse, void* stream) {
    if (!ctx) return DM_ERR_ARG;
    ctx->err.clear();
    DeviceGuard dg(ctx->device);
    dm_status s;
    if ((s = check_grid(ctx, grid)) != DM_OK) return s;
    if (!in || !out) return fail(ctx, DM_ERR_ARG, "NULL buffer");
    cudaStream_t st = (cudaStream_t)stream;
    const bool f64 = ctx->precision == DM_FP64;
    const size_t R = f64 ? 8 : 4;
    const int64_t nH = (int64_t)grid->n[0] * grid->n[1] * (grid->n[2] / 2 + 1);
    const int64_t N = (int64_t)grid->n[0] * grid->n[1] * grid->n[2];
    FFTAxis ax[3];
    if ((s = fft_axes(ctx, grid->n, ax)) != DM_OK) return s;
    Arena A;
    A.take<char>(nH * 2 * R);
    A.take<char>(N * R);
    if ((s = ensure_ws(ctx, A.off + 256)) != DM_OK) return s;
    A.base = ctx->ws;
    A.off = 0;
    char* spec = A.take<char>(nH * 2 * R);
    char* img = A.take<char>(N * R);
    const bool in_dev = is_device_ptr(in), out_dev = is_device_ptr(out);
    if (inverse) {
        CK(cudaMemcpyAsync(spec, in, nH * 2 * R, in_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
        void* dst = out_dev ? out : img;
        if (f64)
            LAUNCH(3, launch_c2r<double>((Cx<double>*)spec, (Cx<double>*)spec, (double*)dst, grid->n[0], grid->n[1],
                                         grid->n[2], ax, st));
        else
            LAUNCH(3, launch_c2r<float>((Cx<float>*)spec, (Cx<float>*)spec, (float*)dst, grid->n[0], grid->n[1],
                                        grid->n[2], ax, st));
        if (!out_dev) {
            CK(cudaMemcpyAsync(out, img, N * R, cudaMemcpyDeviceToHost, st));
            CK(cudaStreamSynchronize(st));
        }
    } else {
        const void* src = in;
        if (!in_dev) {
            CK(cudaMemcpyAsync(img, in, N * R, cudaMemcpyHostToDevice, st));
            src = img;
        }
        void* dst = out_dev ? out : spec;
        if (f64)
            LAUNCH(3, launch_r2c<double>((const double*)src, (Cx<double>*)dst, grid->n[0], grid->n[1], grid->n[2], ax, st));
        else
            LAUNCH(3, launch_r2c<float>((const float*)src, (Cx<float>*)dst, grid->n[0], grid->n[1], grid->n[2], ax, st));
        if (!out_dev) {
            CK(cudaMemcpyAsync(out, spec, nH * 2 * R, cudaMemcpyDeviceToHost, st));
            CK(cudaStreamSynchronize(st));
        }
    }
    return DM_OK;
}

dm_status dm_c2r(dm_ctx* ctx, const dm_grid* grid, const void* spec, void* image, void* stream) {
    return fft_call(ctx, grid, spec, image, true, stream);
}

dm_status dm_r2c(dm_ctx* ctx, const dm_grid* grid, const void* image, void* spec, void* stream) {
    return fft_call(ctx, grid, image, spec, false, stream);
}

dm_status dm_adam(dm_ctx* ctx, double* param, const double* grad, double* m, double* v, int64_t n, double lr,
                  double beta1, double beta2, double eps, int64_t step, void* stream) {
    if (!ctx) return DM_ERR_ARG;
    ctx->err.clear();
    DeviceGuard dg(ctx->device);
    if (!param || !grad || !m || !v || n < 1 || step < 1) return fail(ctx, DM_ERR_ARG, "bad Adam arguments");
    if (!is_device_ptr(param) || !is_device_ptr(grad) || !is_device_ptr(m) || !is_device_ptr(v))
        return fail(ctx, DM_ERR_ARG, "dm_adam needs device buffers");
    Stage sg(ctx, DM_STAGE_ADAM, (cudaStream_t)stream);
    LAUNCH(1, launch_adam(param, grad, m, v, n, lr, beta1, beta2, eps, step, (cudaStream_t)stream));
    return DM_OK;
}

dm_status dm_fit(dm_ctx* ctx, const dm_mesh* mesh, double* V_io, dm_psf* psf_io, const dm_grid* grid,
                 const void* target, const dm_fit_options* opt, double* loss_history, void* stream) {
    if (!ctx) return DM_ERR_ARG;
    ctx->err.clear();
    DeviceGuard dg(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    dm_status s;
    if (!opt || opt->steps < 1) return fail(ctx, DM_ERR_ARG, "fit options: steps >= 1");
    if (!V_io || !target) return fail(ctx, DM_ERR_ARG, "V_io or target is NULL");
    if ((s = check_grid(ctx, grid)) != DM_OK) return s;
    if ((s = check_psf(ctx, psf_io)) != DM_OK) return s;
    if (opt->lr_psf > 0 && psf_io->kind != DM_PSF_DIAG)
        return fail(ctx, DM_ERR_UNSUPPORTED, "dm_fit adapts sigma of a diagonal PSF only");
    if (opt->loss < 0 || opt->loss > 2) return fail(ctx, DM_ERR_ARG, "loss = %d", opt->loss);
    const bool F_dev = is_device_ptr(mesh ? mesh->F : nullptr);
    if ((s = check_mesh(ctx, mesh, !F_dev)) != DM_OK) return s;
    const bool f64 = ctx->precision == DM_FP64;
    const size_t R = f64 ? 8 : 4;
    const bool band = psf_io->band_tau > 0;
    Sizes z = make_sizes(ctx, grid, mesh->n_v, mesh->n_t, band, mesh->label);
    const bool W_host = mesh->tri_weight && !is_device_ptr(mesh->tri_weight);
    const bool T_dev = is_device_ptr(target);
    Arena A;
    Bufs b;
    layout(z, A, b, true, !F_dev, W_host, !T_dev, false);
    const int64_t nV = 3 * mesh->n_v;
    A.take<double>(2 * nV + 8);  // Adam moments of V and sigma
    A.take<double>(opt->steps);
    if ((s = ensure_ws(ctx, A.off + 256)) != DM_OK) return s;
    A.base = ctx->ws;
    A.off = 0;
    layout(z, A, b, true, !F_dev, W_host, !T_dev, false);
    double* mom = A.take<double>(2 * nV + 8);
    double* hist = A.take<double>(opt->steps);
    double *mV = mom, *vV = mom + nV, *ms = mom + 2 * nV, *vs = ms + 4;

    // the fit owns a device copy of V
    CK(cudaMemcpyAsync(b.V, V_io, nV * sizeof(double), cudaMemcpyDefault, st));
    CK(cudaMemsetAsync(mom, 0, (2 * nV + 8) * sizeof(double), st));
    Inputs in;
    in.V = b.V;
    in.F = mesh->F;
    in.wts = mesh->tri_weight;
    in.n_v = mesh->n_v;
    in.n_t = mesh->n_t;
    in.label = mesh->label;
    in.target = target;
    in.loss = opt->loss;
    in.dLdI = nullptr;
    if (!F_dev) {
        CK(cudaMemcpyAsync(b.F, mesh->F, 3 * mesh->n_t * sizeof(int32_t), cudaMemcpyHostToDevice, st));
        in.F = b.F;
    }
    if (W_host) {
        CK(cudaMemcpyAsync(b.wts, mesh->tri_weight, mesh->n_t * sizeof(float), cudaMemcpyHostToDevice, st));
        in.wts = b.wts;
    }
    if (!T_dev) {
        CK(cudaMemcpyAsync(b.target, target, z.N * R, cudaMemcpyHostToDevice, st));
        in.target = b.target;
    }
    LAUNCH(1, launch_set_params(b.d_params, psf_params(psf_io), 9, st));
    Outputs out;
    out.image = nullptr;
    out.dV = b.dV;
    out.want_grad = true;
    for (int it = 0; it < opt->steps; ++it) {
        if (f64)
            s = pipeline<double>(ctx, z, b, in, psf_io, grid, JOB_LOSS, out, st, true);
        else
            s = pipeline<float>(ctx, z, b, in, psf_io, grid, JOB_LOSS, out, st, true);
        if (s != DM_OK) return s;
        CK(cudaMemcpyAsync(hist + it, b.d_params + 17, sizeof(double), cudaMemcpyDeviceToDevice, st));
        Stage sg(ctx, DM_STAGE_ADAM, st);
        LAUNCH(1, launch_adam(b.V, b.dV, mV, vV, nV, opt->lr_vertex, opt->beta1, opt->beta2, opt->eps, it + 1, st));
        if (opt->lr_psf > 0)
            LAUNCH(1, launch_adam(b.d_params, b.d_params + 24, ms, vs, 3, opt->lr_psf, opt->beta1, opt->beta2,
                                  opt->eps, it + 1, st));
    }
    CK(cudaMemcpyAsync(V_io, b.V, nV * sizeof(double), cudaMemcpyDefault, st));
    double sig[3];
    CK(cudaMemcpyAsync(sig, b.d_params, 3 * sizeof(double), cudaMemcpyDeviceToHost, st));
    if (loss_history) CK(cudaMemcpyAsync(loss_history, hist, opt->steps * sizeof(double), cudaMemcpyDefault, st));
    s = check_dev_err(ctx, st);
    if (s != DM_OK) return s;
    if (opt->lr_psf > 0)
        for (int a = 0; a < 3; ++a) psf_io->sigma[a] = sig[a];
    return DM_OK;
}

}  // extern "C"
