// C ABI of the staggered fit (Section 5.1-5.2): the smoothing solve and uniform-Adam
// step of the large-steps vertex update, and the on-device staggered shape/PSF loop.
#include "api_internal.cuh"

namespace {

// Laplacian and solver buffers of one mesh.
struct LapBufs {
    int32_t* cnt;
    int32_t* sptr;
    int32_t* ent;
    int32_t* lptr;
    int32_t* lcol;
    void* work;
    unsigned long long* stats;  // [0] total, [1] max, [2] unconverged
};

void lap_layout(Arena& A, LapBufs& L, int64_t n_v, int64_t n_t, size_t R) {
    L.cnt = A.take<int32_t>(n_v);
    L.sptr = A.take<int32_t>(n_v + 1);
    L.ent = A.take<int32_t>(3 * n_t);
    L.lptr = A.take<int32_t>(n_v + 1);
    L.lcol = A.take<int32_t>(6 * n_t);
    L.work = A.take<char>(pcg_work_elems(n_v) * R);
    L.stats = A.take<unsigned long long>(4);
}

dm_status build_laplacian(dm_ctx* ctx, const int32_t* F, int64_t n_t, int64_t n_v, const LapBufs& L,
                          cudaStream_t st) {
    LAUNCH(4, launch_csr(F, n_t, n_v, L.cnt, L.sptr, L.ent, ctx->d_err, st));
    LAUNCH(3, launch_laplacian(F, L.sptr, L.ent, n_v, L.cnt, L.lptr, L.lcol, ctx->d_err, st));
    CK(cudaMemsetAsync(L.stats, 0, 4 * sizeof(unsigned long long), st));
    return DM_OK;
}

dm_status smooth(dm_ctx* ctx, const LapBufs& L, int64_t n_v, double lam, const double* B, double* X, double* sub_into,
                 double tol, int max_iter, cudaStream_t st) {
    Stage sg(ctx, DM_STAGE_SMOOTH, st);
    if (ctx->precision == DM_FP64)
        LAUNCH(1, launch_pcg<double>(L.lptr, L.lcol, n_v, lam, B, X, sub_into, (double*)L.work, tol, max_iter, L.stats,
                                     st));
    else
        LAUNCH(1, launch_pcg<float>(L.lptr, L.lcol, n_v, lam, B, X, sub_into, (float*)L.work, tol, max_iter, L.stats,
                                    st));
    return DM_OK;
}

double default_tol(const dm_ctx* ctx, double tol) {
    if (tol > 0) return tol;
    return ctx->precision == DM_FP64 ? 1e-12 : 1e-6;
}

// 3x3 Cholesky of a covariance (xx, yy, zz, xy, xz, yz) into (C00, C11, C22, C10, C20, C21).
bool host_cholesky(const double cov[6], double C[6]) {
    const double xx = cov[0], yy = cov[1], zz = cov[2], xy = cov[3], xz = cov[4], yz = cov[5];
    if (!(xx > 0)) return false;
    const double a = std::sqrt(xx);
    const double d = xy / a, e = xz / a;
    const double bb = yy - d * d;
    if (!(bb > 0)) return false;
    const double b = std::sqrt(bb);
    const double f = (yz - d * e) / b;
    const double cc = zz - e * e - f * f;
    if (!(cc > 0)) return false;
    C[0] = a;
    C[1] = b;
    C[2] = std::sqrt(cc);
    C[3] = d;
    C[4] = e;
    C[5] = f;
    return true;
}

}  // namespace

extern "C" {

dm_status dm_smooth_solve(dm_ctx* ctx, const int32_t* F, int64_t n_t, int64_t n_v, double lambda, const double* B,
                          double* X, double tol, int32_t max_iter, int64_t* iters, void* stream) {
    if (!ctx) return DM_ERR_ARG;
    ctx->err.clear();
    DeviceGuard dg(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    if (!F || !B || !X) return fail(ctx, DM_ERR_ARG, "F, B or X is NULL");
    if (n_v < 1 || n_t < 1 || n_t > (int64_t)1 << 28 || n_v > (int64_t)1 << 29)
        return fail(ctx, DM_ERR_ARG, "bad mesh sizes");
    if (!(lambda >= 0)) return fail(ctx, DM_ERR_ARG, "lambda must be >= 0");
    if (!is_device_ptr(B) || !is_device_ptr(X)) return fail(ctx, DM_ERR_ARG, "B and X must be device buffers");
    const bool F_dev = is_device_ptr(F);
    if (!F_dev)
        for (int64_t i = 0; i < 3 * n_t; ++i)
            if (F[i] < 0 || F[i] >= n_v) return fail(ctx, DM_ERR_ARG, "F[%lld] out of range", (long long)i);
    const size_t R = ctx->precision == DM_FP64 ? 8 : 4;
    Arena A;
    LapBufs L;
    lap_layout(A, L, n_v, n_t, R);
    int32_t* Fd = A.take<int32_t>(F_dev ? 0 : 3 * n_t);
    dm_status s;
    if ((s = ensure_ws(ctx, A.off + 256)) != DM_OK) return s;
    A.base = ctx->ws;
    A.off = 0;
    lap_layout(A, L, n_v, n_t, R);
    Fd = A.take<int32_t>(F_dev ? 0 : 3 * n_t);
    const int32_t* Fu = F;
    if (!F_dev) {
        CK(cudaMemcpyAsync(Fd, F, 3 * n_t * sizeof(int32_t), cudaMemcpyHostToDevice, st));
        Fu = Fd;
    }
    if ((s = build_laplacian(ctx, Fu, n_t, n_v, L, st)) != DM_OK) return s;
    if ((s = smooth(ctx, L, n_v, lambda, B, X, nullptr, default_tol(ctx, tol), max_iter > 0 ? max_iter : 2000, st)) !=
        DM_OK)
        return s;
    if (iters) {
        unsigned long long h[4];
        CK(cudaMemcpyAsync(h, L.stats, sizeof(h), cudaMemcpyDeviceToHost, st));
        if ((s = check_dev_err(ctx, st)) != DM_OK) return s;
        for (int k = 0; k < 3; ++k) iters[k] = (int64_t)h[k];
    }
    return DM_OK;
}

dm_status dm_adam_uniform(dm_ctx* ctx, const double* grad, double* m, double* v, double* delta, int64_t n, double lr,
                          double beta1, double beta2, double eps, int64_t step, void* stream) {
    if (!ctx) return DM_ERR_ARG;
    ctx->err.clear();
    DeviceGuard dg(ctx->device);
    if (!grad || !m || !v || !delta || n < 1 || step < 1) return fail(ctx, DM_ERR_ARG, "bad uniform-Adam arguments");
    if (!is_device_ptr(grad) || !is_device_ptr(m) || !is_device_ptr(v) || !is_device_ptr(delta))
        return fail(ctx, DM_ERR_ARG, "dm_adam_uniform needs device buffers");
    Arena A;
    A.take<double>(adam_uniform_partials(n));
    dm_status s;
    if ((s = ensure_ws(ctx, A.off + 256)) != DM_OK) return s;
    Stage sg(ctx, DM_STAGE_ADAM, (cudaStream_t)stream);
    LAUNCH(2, launch_adam_uniform(grad, m, v, delta, n, lr, beta1, beta2, eps, step, (double*)ctx->ws,
                                  (cudaStream_t)stream));
    return DM_OK;
}

dm_status dm_fit_staggered(dm_ctx* ctx, const dm_mesh* mesh, double* V_io, dm_psf* psf_io, const dm_grid* grid,
                           const void* target, const dm_stagger_options* opt, double* shape_loss, double* psf_loss,
                           dm_stagger_stats* stats, void* stream) {
    if (!ctx) return DM_ERR_ARG;
    ctx->err.clear();
    DeviceGuard dg(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    dm_status s;
    if (!opt || opt->rounds < 1 || opt->shape_steps < 0 || opt->psf_steps < 0)
        return fail(ctx, DM_ERR_ARG, "stagger options: rounds >= 1, steps >= 0");
    if (opt->shape_loss < 0 || opt->shape_loss > 2 || opt->psf_loss < 0 || opt->psf_loss > 2)
        return fail(ctx, DM_ERR_ARG, "bad loss kind");
    if (opt->optimizer != DM_OPT_ADAM && opt->optimizer != DM_OPT_LARGE_STEPS)
        return fail(ctx, DM_ERR_ARG, "optimizer = %d", opt->optimizer);
    if (!(opt->lambda >= 0)) return fail(ctx, DM_ERR_ARG, "lambda must be >= 0");
    if (!V_io || !target) return fail(ctx, DM_ERR_ARG, "V_io or target is NULL");
    if ((s = check_grid(ctx, grid)) != DM_OK) return s;
    if ((s = check_psf(ctx, psf_io)) != DM_OK) return s;
    const bool F_dev = is_device_ptr(mesh ? mesh->F : nullptr);
    if ((s = check_mesh(ctx, mesh, !F_dev)) != DM_OK) return s;

    // initial Cholesky factor of Sigma
    double cov0[6], C0[6];
    if (psf_io->kind == DM_PSF_FULL) {
        for (int k = 0; k < 6; ++k) cov0[k] = psf_io->cov[k];
    } else {
        for (int a = 0; a < 3; ++a) cov0[a] = psf_io->sigma[a] * psf_io->sigma[a];
        cov0[3] = cov0[4] = cov0[5] = 0.0;
    }
    if (!host_cholesky(cov0, C0)) return fail(ctx, DM_ERR_ARG, "the covariance is not positive definite");
    dm_psf pw = *psf_io;  // the working PSF: full covariance on the device
    pw.kind = DM_PSF_FULL;
    for (int k = 0; k < 6; ++k) pw.cov[k] = cov0[k];
    dm_psf pf = pw;  // PSF steps: every frequency
    pf.band_tau = 0.0;

    const bool f64 = ctx->precision == DM_FP64;
    const size_t R = f64 ? 8 : 4;
    const bool band = pw.band_tau > 0;
    const Sizes z = make_sizes(ctx, grid, mesh->n_v, mesh->n_t, band, mesh->label);
    Sizes zf = z;
    zf.band = false;
    const bool W_host = mesh->tri_weight && !is_device_ptr(mesh->tri_weight);
    const bool T_dev = is_device_ptr(target);
    const int64_t nV = 3 * mesh->n_v;
    const int64_t n_hs = (int64_t)opt->rounds * opt->shape_steps, n_hp = (int64_t)opt->rounds * opt->psf_steps;
    const bool ls = opt->optimizer == DM_OPT_LARGE_STEPS;

    auto carve = [&](Arena& A, Bufs& b, LapBufs& L, double*& st_v, double*& st_c, double*& hs, double*& hp,
                     double*& aup) {
        layout(z, A, b, true, !F_dev, W_host, !T_dev, false);
        st_v = A.take<double>(5 * nV);   // m, v, gu (warm start), w (warm start), delta
        st_c = A.take<double>(32);       // C, gC, mC, vC
        hs = A.take<double>(n_hs + 1);
        hp = A.take<double>(n_hp + 1);
        aup = A.take<double>(adam_uniform_partials(nV));
        lap_layout(A, L, mesh->n_v, mesh->n_t, R);
    };
    Arena A;
    Bufs b;
    LapBufs L;
    double *sv, *sc, *hs, *hp, *aup;
    carve(A, b, L, sv, sc, hs, hp, aup);
    if ((s = ensure_ws(ctx, A.off + 256)) != DM_OK) return s;
    A.base = ctx->ws;
    A.off = 0;
    carve(A, b, L, sv, sc, hs, hp, aup);
    double *mV = sv, *vV = sv + nV, *gu = sv + 2 * nV, *wv = sv + 3 * nV, *dl = sv + 4 * nV;
    double *C = sc, *gC = sc + 8, *mC = sc + 16, *vC = sc + 24;

    CK(cudaMemcpyAsync(b.V, V_io, nV * sizeof(double), cudaMemcpyDefault, st));
    CK(cudaMemsetAsync(sv, 0, 5 * nV * sizeof(double), st));
    CK(cudaMemsetAsync(sc, 0, 32 * sizeof(double), st));
    CK(cudaMemcpyAsync(C, C0, 6 * sizeof(double), cudaMemcpyHostToDevice, st));
    Inputs in;
    in.V = b.V;
    in.F = mesh->F;
    in.wts = mesh->tri_weight;
    in.n_v = mesh->n_v;
    in.n_t = mesh->n_t;
    in.label = mesh->label;
    in.target = target;
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
    LAUNCH(1, launch_set_params(b.d_params, psf_params(&pw), 9, st));
    if (ls && opt->shape_steps > 0 && (s = build_laplacian(ctx, in.F, mesh->n_t, mesh->n_v, L, st)) != DM_OK) return s;
    const double tol = default_tol(ctx, opt->cg_tol);
    const int max_it = opt->cg_max_iter > 0 ? opt->cg_max_iter : 2000;

    Outputs shape_out;
    shape_out.image = nullptr;
    shape_out.dV = b.dV;
    shape_out.want_grad = true;
    Outputs psf_out = shape_out;
    psf_out.psf_only = true;
    int64_t ts = 0, tp = 0;
    for (int r = 0; r < opt->rounds; ++r) {
        in.loss = opt->shape_loss;
        for (int k = 0; k < opt->shape_steps; ++k) {  // (a) narrow band, PSF held
            s = f64 ? pipeline<double>(ctx, z, b, in, &pw, grid, JOB_LOSS, shape_out, st, true)
                    : pipeline<float>(ctx, z, b, in, &pw, grid, JOB_LOSS, shape_out, st, true);
            if (s != DM_OK) return s;
            CK(cudaMemcpyAsync(hs + ts, b.d_params + 17, sizeof(double), cudaMemcpyDeviceToDevice, st));
            ++ts;
            if (ls) {
                if ((s = smooth(ctx, L, mesh->n_v, opt->lambda, b.dV, gu, nullptr, tol, max_it, st)) != DM_OK) return s;
                {
                    Stage sg(ctx, DM_STAGE_ADAM, st);
                    LAUNCH(2, launch_adam_uniform(gu, mV, vV, dl, nV, opt->lr_vertex, opt->beta1, opt->beta2, opt->eps,
                                                  ts, aup, st));
                }
                if ((s = smooth(ctx, L, mesh->n_v, opt->lambda, dl, wv, b.V, tol, max_it, st)) != DM_OK) return s;
            } else {
                Stage sg(ctx, DM_STAGE_ADAM, st);
                LAUNCH(1, launch_adam(b.V, b.dV, mV, vV, nV, opt->lr_vertex, opt->beta1, opt->beta2, opt->eps, ts, st));
            }
        }
        in.loss = opt->psf_loss;
        for (int k = 0; k < opt->psf_steps; ++k) {  // (b) every frequency, shape held
            s = f64 ? pipeline<double>(ctx, zf, b, in, &pf, grid, JOB_LOSS, psf_out, st, true)
                    : pipeline<float>(ctx, zf, b, in, &pf, grid, JOB_LOSS, psf_out, st, true);
            if (s != DM_OK) return s;
            CK(cudaMemcpyAsync(hp + tp, b.d_params + 17, sizeof(double), cudaMemcpyDeviceToDevice, st));
            ++tp;
            Stage sg(ctx, DM_STAGE_ADAM, st);
            LAUNCH(1, launch_chol_grad(C, b.d_params + 24, gC, st));
            LAUNCH(1, launch_adam(C, gC, mC, vC, 6, opt->lr_psf, opt->beta1, opt->beta2, opt->eps, tp, st));
            LAUNCH(1, launch_chol_to_cov(C, b.d_params, st));
        }
    }
    CK(cudaMemcpyAsync(V_io, b.V, nV * sizeof(double), cudaMemcpyDefault, st));
    double cov[6];
    unsigned long long hst[4];
    CK(cudaMemcpyAsync(cov, b.d_params + 3, 6 * sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(hst, L.stats, sizeof(hst), cudaMemcpyDeviceToHost, st));
    if (shape_loss && n_hs) CK(cudaMemcpyAsync(shape_loss, hs, n_hs * sizeof(double), cudaMemcpyDefault, st));
    if (psf_loss && n_hp) CK(cudaMemcpyAsync(psf_loss, hp, n_hp * sizeof(double), cudaMemcpyDefault, st));
    if ((s = check_dev_err(ctx, st)) != DM_OK) return s;
    psf_io->kind = DM_PSF_FULL;
    for (int k = 0; k < 6; ++k) psf_io->cov[k] = cov[k];
    for (int a = 0; a < 3; ++a) psf_io->sigma[a] = std::sqrt(std::max(cov[a], 0.0));
    if (stats) {
        const bool ran = ls && opt->shape_steps > 0;
        stats->cg_iterations = ran ? (int64_t)hst[0] : 0;
        stats->cg_max = ran ? (int64_t)hst[1] : 0;
        stats->cg_unconverged = ran ? (int64_t)hst[2] : 0;
    }
    return DM_OK;
}

}  // extern "C"
