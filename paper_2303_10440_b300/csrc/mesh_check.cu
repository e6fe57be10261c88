// Host-side mesh validation: face indices, finite vertices and densities, a positive normaliser
// (total weighted area for the surface label, enclosed volume for the volume label; Sec. 4.1) and,
// for the volume label, a closed and consistently oriented mesh (the divergence form of the volume
// transform needs one). Used by dm_check_mesh (a debug call) and by the fit server at submit.
#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "api_internal.cuh"

namespace dm {

dm_status check_mesh_host(const double* V, int64_t n_v, const int32_t* F, int64_t n_t, const float* W, int label,
                          std::string* why) {
    if (!V || !F || n_v < 3 || n_t < 1) {
        *why = "mesh: V and F required, n_v >= 3, n_t >= 1";
        return DM_ERR_ARG;
    }
    if (label != DM_SURFACE && label != DM_VOLUME) {
        *why = "mesh: label must be DM_SURFACE or DM_VOLUME";
        return DM_ERR_ARG;
    }
    if (W && label != DM_SURFACE) {
        *why = "tri_weight is for the surface label only";
        return DM_ERR_ARG;
    }
    for (int64_t i = 0; i < 3 * n_v; ++i)
        if (!std::isfinite(V[i])) {
            *why = "non-finite vertex position";
            return DM_ERR_ARG;
        }
    for (int64_t i = 0; i < 3 * n_t; ++i)
        if (F[i] < 0 || F[i] >= n_v) {
            *why = "face index outside [0, n_v)";
            return DM_ERR_ARG;
        }
    double measure = 0.0;
    for (int64_t t = 0; t < n_t; ++t) {
        const double* a = V + 3 * (int64_t)F[3 * t];
        const double* b = V + 3 * (int64_t)F[3 * t + 1];
        const double* c = V + 3 * (int64_t)F[3 * t + 2];
        if (label == DM_SURFACE) {
            const double e1[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]};
            const double e2[3] = {c[0] - a[0], c[1] - a[1], c[2] - a[2]};
            const double n[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2],
                                 e1[0] * e2[1] - e1[1] * e2[0]};
            double w = 1.0;
            if (W) {
                w = W[t];
                if (!(w >= 0.0) || !std::isfinite(w)) {
                    *why = "tri_weight: densities must be finite and >= 0";
                    return DM_ERR_ARG;
                }
            }
            measure += w * 0.5 * std::sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
        } else {
            // signed volume of the cone from the origin: a . (b x c) / 6
            measure += (a[0] * (b[1] * c[2] - b[2] * c[1]) + a[1] * (b[2] * c[0] - b[0] * c[2]) +
                        a[2] * (b[0] * c[1] - b[1] * c[0])) / 6.0;
        }
    }
    if (!(measure > 0.0)) {
        *why = label == DM_SURFACE ? "zero total (weighted) area" : "non-positive enclosed volume";
        return DM_ERR_DEGENERATE;
    }
    if (label == DM_VOLUME) {
        // closed and consistently oriented: every directed edge (p -> q) occurs once, and so does (q -> p)
        std::vector<uint64_t> e(3 * (size_t)n_t);
        for (int64_t t = 0; t < n_t; ++t)
            for (int k = 0; k < 3; ++k) {
                const uint64_t p = (uint64_t)F[3 * t + k], q = (uint64_t)F[3 * t + (k + 1) % 3];
                e[3 * t + k] = p * (uint64_t)n_v + q;
            }
        std::sort(e.begin(), e.end());
        for (size_t i = 0; i < e.size(); ++i) {
            const uint64_t p = e[i] / (uint64_t)n_v, q = e[i] % (uint64_t)n_v;
            if ((i + 1 < e.size() && e[i + 1] == e[i]) || p == q ||
                !std::binary_search(e.begin(), e.end(), q * (uint64_t)n_v + p)) {
                *why = "volume label: the mesh is not closed and consistently oriented (edge " + std::to_string(p) +
                       " -> " + std::to_string(q) + ")";
                return DM_ERR_OPEN_MESH;
            }
        }
    }
    return DM_OK;
}

}  // namespace dm

extern "C" {

dm_status dm_check_mesh(dm_ctx* ctx, const dm_mesh* mesh) {
    using namespace dm;
    if (!mesh) return DM_ERR_ARG;
    if (ctx) ctx->err.clear();
    if (!mesh->V || !mesh->F || mesh->n_v < 3 || mesh->n_t < 1)
        return fail(ctx, DM_ERR_ARG, "mesh: V and F required, n_v >= 3, n_t >= 1");
    if (!ctx) {
        // no context: host arrays only, and no CUDA call beyond the pointer checks
        std::string why;
        if (is_device_ptr(mesh->V) || is_device_ptr(mesh->F) || is_device_ptr(mesh->tri_weight)) return DM_ERR_ARG;
        return check_mesh_host(mesh->V, mesh->n_v, mesh->F, mesh->n_t, mesh->tri_weight, mesh->label, &why);
    }
    DeviceGuard dg(ctx->device);
    // device arrays are copied to the host (a debug call: it synchronises)
    std::vector<double> hV;
    std::vector<int32_t> hF;
    std::vector<float> hW;
    const double* V = mesh->V;
    const int32_t* F = mesh->F;
    const float* W = mesh->tri_weight;
    if (is_device_ptr(V)) {
        hV.resize(3 * (size_t)mesh->n_v);
        CK(cudaMemcpy(hV.data(), V, hV.size() * sizeof(double), cudaMemcpyDeviceToHost));
        V = hV.data();
    }
    if (is_device_ptr(F)) {
        hF.resize(3 * (size_t)mesh->n_t);
        CK(cudaMemcpy(hF.data(), F, hF.size() * sizeof(int32_t), cudaMemcpyDeviceToHost));
        F = hF.data();
    }
    if (W && is_device_ptr(W)) {
        hW.resize((size_t)mesh->n_t);
        CK(cudaMemcpy(hW.data(), W, hW.size() * sizeof(float), cudaMemcpyDeviceToHost));
        W = hW.data();
    }
    std::string why;
    const dm_status s = check_mesh_host(V, mesh->n_v, F, mesh->n_t, W, mesh->label, &why);
    if (s != DM_OK) return fail(ctx, s, "%s", why.c_str());
    return DM_OK;
}

}  // extern "C"
