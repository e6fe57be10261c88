// Allocation-free variant of dm_meshft (FP32 mixed path).
//
// Who needs it: callers that must never trigger a device allocation inside the
// library — for example a serving process that reserves all of its device memory
// at start-up and treats any later cudaMalloc as an error (cudaMalloc can
// synchronise the device and can fail under memory pressure), or a host framework
// that routes every device allocation through its own pool and cannot let a
// library allocate behind its back. dm_meshft stages its triangle records in a
// context workspace that is grown with cudaMalloc on demand; this entry point
// needs no context at all and keeps that scratch in a fixed, file-scope device
// array instead.
//
// Limits and behaviour:
// * at most DM_NOALLOC_MAX_TRIANGLES triangles (the scratch holds their records);
// * every pointer must be device memory of the calling thread's current device;
// * the scratch is one array per device, shared by every call: calls that overlap
//   on the GPU (different streams, or host threads using the same device) race on
//   it and must be serialised by the caller;
// * the first call on a device looks up the array's device address with
//   cudaGetSymbolAddress (once per device); under CUDA's lazy module loading it is
//   also when the kernels' modules and the array are placed on the device, so it
//   can still take device memory: make that first call at start-up, as a warm-up,
//   before any stream capture. Later calls take no device memory.
#include <mutex>

#include "../../include/deltamic.h"
#include "dm_kernels.cuh"

using namespace dm;

namespace {

// Scratch layout: [0, 64) fault flags (int), [64, 72) normaliser (double),
// [256, 8192) per-block partial sums of the normaliser, [8192, ...) triangle records.
constexpr size_t kFlagsOff = 0;
constexpr size_t kNormOff = 64;
constexpr size_t kPartialOff = 256;
constexpr size_t kRecOff = 8192;
static_assert(kRecOff + (size_t)DM_NOALLOC_MAX_TRIANGLES * sizeof(TriF32) <= DM_NOALLOC_SCRATCH_BYTES,
              "scratch too small for the stated triangle limit");
static_assert((DM_NOALLOC_MAX_TRIANGLES / 256) * sizeof(double) <= kRecOff - kPartialOff, "partial area");

static __device__ __align__(256) unsigned char g_noalloc_scratch[DM_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned char* g_dev_scratch[kMaxDevices] = {nullptr};

// Device address of the scratch array on the current device (looked up once per device).
dm_status scratch_on_current_device(unsigned char** out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return DM_ERR_CUDA;
    }
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_dev_scratch[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return DM_ERR_CUDA;
        }
        g_dev_scratch[dev] = static_cast<unsigned char*>(p);
    }
    *out = g_dev_scratch[dev];
    return DM_OK;
}

bool on_device(const void* p, int dev) {
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) && a.device == dev;
}

}  // namespace

extern "C" dm_status dm_meshft_noalloc(const dm_mesh* mesh, const dm_grid* grid, const int32_t* freq_n, int64_t M,
                                       void* S_out, int32_t* fault_flags, void* stream) {
    if (!mesh || !grid || !freq_n || !S_out || M < 1) return DM_ERR_ARG;
    if (mesh->n_t < 1 || mesh->n_t > DM_NOALLOC_MAX_TRIANGLES || mesh->n_v < 3) return DM_ERR_ARG;
    if (mesh->label != DM_SURFACE && mesh->label != DM_VOLUME) return DM_ERR_ARG;
    if (mesh->label == DM_VOLUME && mesh->tri_weight) return DM_ERR_ARG;
    if (M > ((int64_t)1 << 31) - 1) return DM_ERR_ARG;
    for (int a = 0; a < 3; ++a)
        if (grid->n[a] < 1 || !(grid->h[a] > 0)) return DM_ERR_ARG;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return DM_ERR_CUDA;
    }
    if (!on_device(mesh->V, dev) || !on_device(mesh->F, dev) || !on_device(freq_n, dev) || !on_device(S_out, dev) ||
        (mesh->tri_weight && !on_device(mesh->tri_weight, dev)) || (fault_flags && !on_device(fault_flags, dev)))
        return DM_ERR_ARG;
    unsigned char* base = nullptr;
    dm_status s = scratch_on_current_device(&base);
    if (s != DM_OK) return s;

    cudaStream_t st = (cudaStream_t)stream;
    int* d_err = reinterpret_cast<int*>(base + kFlagsOff);
    double* d_norm = reinterpret_cast<double*>(base + kNormOff);
    double* partial = reinterpret_cast<double*>(base + kPartialOff);
    TriF32* rec = reinterpret_cast<TriF32*>(base + kRecOff);
    const int64_t n_t_pad = (mesh->n_t + FWD_TILE - 1) / FWD_TILE * FWD_TILE;

    Geom g;
    for (int a = 0; a < 3; ++a) {
        g.L[a] = grid->n[a] * grid->h[a];
        g.origin[a] = grid->origin[a];
    }
    FreqSrc fs;
    fs.nlist = freq_n;
    fs.idx = nullptr;
    fs.dM = nullptr;
    fs.M = M;
    fs.set_dims(grid->n[0], grid->n[1], grid->n[2]);

    // The fault flags must start at zero for this call; records, partials and the
    // normaliser are fully rewritten before they are read.
    if (cudaMemsetAsync(d_err, 0, sizeof(int), st) != cudaSuccess) {
        cudaGetLastError();
        return DM_ERR_CUDA;
    }
    int nb = 0;
    cudaError_t e = launch_tri_prep<TriF32>(mesh->label, mesh->V, mesh->n_v, mesh->F, mesh->n_t, mesh->tri_weight, g,
                                            rec, n_t_pad, partial, &nb, d_err, st);
    if (e == cudaSuccess) e = launch_norm_sum(partial, nb, d_norm, d_err, st);
    if (e == cudaSuccess) e = launch_fwd_f32(mesh->label, rec, mesh->n_t, fs, g, d_norm, (float2*)S_out, nullptr, 0, d_err, st);
    if (e == cudaSuccess && fault_flags) e = cudaMemcpyAsync(fault_flags, d_err, sizeof(int), cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return DM_ERR_CUDA;
    }
    return DM_OK;
}
