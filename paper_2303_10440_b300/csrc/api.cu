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

namespace dm {
std::atomic<int64_t> g_launches{0};
}

#include "api_internal.cuh"

namespace {

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
        ctx->graphs = opt->no_graphs == 0;
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
    if (ctx->cap) cudaStreamDestroy(ctx->cap);
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
    double* red;
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
    b.red = A.take<double>(reduce_scratch_elems(ctx->sm_count));
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
    LAUNCH(1, launch_norm_sum(b.partial, nb, b.d_params + 16, ctx->d_err, st));
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
    fs.set_dims(grid->n[0], grid->n[1], grid->n[2]);
    const Geom G = make_geom(grid);
    if (f64)
        LAUNCH(1, launch_fwd_f64(mesh->label, (const TriF64*)b.tris, mesh->n_t, fs, G, b.d_params + 16, (double2*)S, st));
    else
        LAUNCH(1, launch_fwd_f32(mesh->label, (const TriF32*)b.tris, mesh->n_t, fs, G,
                                 b.d_params + 16, (float2*)S, nullptr, ctx->sm_count, ctx->d_err, st));
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
        LAUNCH(1, launch_reduce_chunks<double>((const double*)b.adjp, nc, nacc, mesh->n_t, mesh->n_t, b.acc, st, nullptr,
                                               -1, b.red, ctx->sm_count));
    } else {
        LAUNCH(1, launch_adj_f32(mesh->label, (const TriF32*)b.tris, mesh->n_t, n_t_pad, (const FreqF32*)b.fr, nullptr,
                                 M, (float*)b.adjp, nc, ctx->d_err, st));
        LAUNCH(1, launch_reduce_chunks<float>((const float*)b.adjp, nc, nacc, mesh->n_t, n_t_pad, b.acc, st, nullptr, M,
                                              b.red, ctx->sm_count));
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
        // a device spectrum is read in place by the first pass (and left unchanged) unless it overlaps the
        // image; a host one, or an overlapping one, is copied into the workspace first
        const char* ib = (const char*)in;
        const char* ob = (const char*)out;
        const bool overlap = out_dev && ib < ob + N * R && ob < ib + nH * 2 * R;
        const bool direct = in_dev && !overlap;
        if (!direct)
            CK(cudaMemcpyAsync(spec, in, nH * 2 * R, in_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
        const void* sin = direct ? in : spec;
        void* dst = out_dev ? out : img;
        if (f64)
            LAUNCH(3, launch_c2r<double>((const Cx<double>*)sin, (Cx<double>*)spec, (double*)dst, grid->n[0],
                                         grid->n[1], grid->n[2], ax, st));
        else
            LAUNCH(3, launch_c2r<float>((const Cx<float>*)sin, (Cx<float>*)spec, (float*)dst, grid->n[0], grid->n[1],
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

dm_status dm_fit_resume(dm_ctx* ctx, const dm_mesh* mesh, double* V_io, dm_psf* psf_io, const dm_grid* grid,
                        const void* target, const dm_fit_options* opt, dm_fit_state* state, double* loss_history,
                        void* stream) {
    if (!ctx) return DM_ERR_ARG;
    ctx->err.clear();
    DeviceGuard dg(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    dm_status s;
    if (!opt || opt->steps < 1) return fail(ctx, DM_ERR_ARG, "fit options: steps >= 1");
    if (!V_io || !target) return fail(ctx, DM_ERR_ARG, "V_io or target is NULL");
    if (state && (state->step < 0 || !state->m_V || !state->v_V))
        return fail(ctx, DM_ERR_ARG, "fit state: step >= 0 and both vertex moment arrays");
    dm_psf* const psf_user = psf_io;
    dm_psf psf_start;
    if (state && psf_io) {  // sigma continues from the checkpoint
        psf_start = *psf_io;
        for (int a = 0; a < 3; ++a) psf_start.sigma[a] = state->sigma[a];
        psf_io = &psf_start;
    }
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
    A.take<int64_t>(1);
    if ((s = ensure_ws(ctx, A.off + 256)) != DM_OK) return s;
    A.base = ctx->ws;
    A.off = 0;
    layout(z, A, b, true, !F_dev, W_host, !T_dev, false);
    double* mom = A.take<double>(2 * nV + 8);
    double* hist = A.take<double>(opt->steps);
    int64_t* d_step = A.take<int64_t>(1);  // Adam step t of the running iteration
    double *mV = mom, *vV = mom + nV, *ms = mom + 2 * nV, *vs = ms + 4;

    // the fit owns a device copy of V
    CK(cudaMemcpyAsync(b.V, V_io, nV * sizeof(double), cudaMemcpyDefault, st));
    CK(cudaMemsetAsync(mom, 0, (2 * nV + 8) * sizeof(double), st));
    const int64_t step0 = state ? state->step : 0;
    if (state) {
        CK(cudaMemcpyAsync(mV, state->m_V, nV * sizeof(double), cudaMemcpyHostToDevice, st));
        CK(cudaMemcpyAsync(vV, state->v_V, nV * sizeof(double), cudaMemcpyHostToDevice, st));
        CK(cudaMemcpyAsync(ms, state->m_sigma, 3 * sizeof(double), cudaMemcpyHostToDevice, st));
        CK(cudaMemcpyAsync(vs, state->v_sigma, 3 * sizeof(double), cudaMemcpyHostToDevice, st));
    }
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
    const int64_t t_first = step0 + 1;
    CK(cudaMemcpyAsync(d_step, &t_first, sizeof(int64_t), cudaMemcpyHostToDevice, st));
    // One optimisation step, identical on every iteration: the Adam step t lives on the device and
    // the closing tick stores the loss at hist[t - step0 - 1] and advances t.
    const auto fit_step = [&](cudaStream_t q) -> dm_status {
        const dm_status r = f64 ? pipeline<double>(ctx, z, b, in, psf_io, grid, JOB_LOSS, out, q, true)
                                : pipeline<float>(ctx, z, b, in, psf_io, grid, JOB_LOSS, out, q, true);
        if (r != DM_OK) return r;
        Stage sg(ctx, DM_STAGE_ADAM, q);
        LAUNCH(1, launch_adam_dev_step(b.V, b.dV, mV, vV, nV, opt->lr_vertex, opt->beta1, opt->beta2, opt->eps,
                                       d_step, 1.0, q));
        if (opt->lr_psf > 0)
            LAUNCH(1, launch_adam_dev_step(b.d_params, b.d_params + 24, ms, vs, 3, opt->lr_psf, opt->beta1,
                                           opt->beta2, opt->eps, d_step, 1.0, q));
        LAUNCH(1, launch_fit_tick(hist, b.d_params + 17, d_step, step0, q));
        return DM_OK;
    };
    // The first step runs directly: it also creates the FFT tables and raises kernel attributes,
    // which a capture must not do.
    if ((s = fit_step(st)) != DM_OK) return s;
    int it = 1;
    if (ctx->graphs && !ctx->prof && opt->steps >= 3) {
        cudaGraphExec_t ge = nullptr;
        const int64_t l0 = g_launches;
        if (capture_graph(ctx, fit_step, &ge)) {
            const int64_t per = g_launches - l0;
            g_launches = l0;
            for (; it < opt->steps; ++it) {
                const cudaError_t le = cudaGraphLaunch(ge, st);
                if (le != cudaSuccess) {
                    cudaGraphExecDestroy(ge);
                    return fail(ctx, DM_ERR_CUDA, "cudaGraphLaunch: %s", cudaGetErrorString(le));
                }
                g_launches += per;
            }
            cudaGraphExecDestroy(ge);  // freed once the launches in flight complete
        } else {
            g_launches = l0;  // the capture failed; the remaining steps run directly
        }
    }
    for (; it < opt->steps; ++it)
        if ((s = fit_step(st)) != DM_OK) return s;
    CK(cudaMemcpyAsync(V_io, b.V, nV * sizeof(double), cudaMemcpyDefault, st));
    double sig[3];
    CK(cudaMemcpyAsync(sig, b.d_params, 3 * sizeof(double), cudaMemcpyDeviceToHost, st));
    if (loss_history) CK(cudaMemcpyAsync(loss_history, hist, opt->steps * sizeof(double), cudaMemcpyDefault, st));
    if (state) {
        CK(cudaMemcpyAsync(state->m_V, mV, nV * sizeof(double), cudaMemcpyDeviceToHost, st));
        CK(cudaMemcpyAsync(state->v_V, vV, nV * sizeof(double), cudaMemcpyDeviceToHost, st));
        CK(cudaMemcpyAsync(state->m_sigma, ms, 3 * sizeof(double), cudaMemcpyDeviceToHost, st));
        CK(cudaMemcpyAsync(state->v_sigma, vs, 3 * sizeof(double), cudaMemcpyDeviceToHost, st));
    }
    s = check_dev_err(ctx, st);
    if (s != DM_OK) return s;
    if (state) {
        state->step = step0 + opt->steps;
        for (int a = 0; a < 3; ++a) state->sigma[a] = sig[a];
    }
    if (opt->lr_psf > 0)
        for (int a = 0; a < 3; ++a) psf_user->sigma[a] = sig[a];
    return DM_OK;
}

dm_status dm_fit(dm_ctx* ctx, const dm_mesh* mesh, double* V_io, dm_psf* psf_io, const dm_grid* grid,
                 const void* target, const dm_fit_options* opt, double* loss_history, void* stream) {
    return dm_fit_resume(ctx, mesh, V_io, psf_io, grid, target, opt, nullptr, loss_history, stream);
}

}  // extern "C"
