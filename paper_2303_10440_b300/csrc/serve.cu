// Continuous-batching fit server (include/deltamic.h, "fit server").
//
// Engine thread, per iteration:
//   admit   queued jobs move in (in arrival order, or least work first) while a batch slot and
//           arena room are free; their mesh, target, PSF parameters, optimiser state, vertex star
//           and band live on the device;
//   step    the selected resident jobs advance by one optimiser step: per-job stage kernels on
//           each job's stream, and the two mesh-transform sums of all of them as one persistent
//           batched launch each per label (work lists of equal-cost units pulled from an atomic
//           counter); while the selection is unchanged the step replays as a captured CUDA graph;
//   retire  jobs that reached their step count copy their results to the host and release
//           their arena block.
// Arrivals therefore join at the next iteration while earlier jobs are still running, and
// their work overlaps on the device inside the same launches.
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>

#include "api_internal.cuh"

namespace {

// First-fit allocator over one device allocation (256-byte granules).
class DeviceArena {
  public:
    char* base = nullptr;
    size_t total = 0, in_use = 0, peak = 0;

    bool init(size_t bytes) {
        bytes &= ~(size_t)255;
        if (cudaMalloc(&base, bytes) != cudaSuccess) {
            cudaGetLastError();
            base = nullptr;
            return false;
        }
        total = bytes;
        free_[0] = bytes;
        return true;
    }
    void release() {
        if (base) cudaFree(base);
        base = nullptr;
        free_.clear();
    }
    bool alloc(size_t bytes, size_t* off) {
        bytes = (bytes + 255) & ~(size_t)255;
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= bytes) {
                *off = it->first;
                const size_t rest = it->second - bytes, at = it->first + bytes;
                free_.erase(it);
                if (rest) free_[at] = rest;
                in_use += bytes;
                peak = std::max(peak, in_use);
                return true;
            }
        }
        return false;
    }
    void release_block(size_t off, size_t bytes) {
        bytes = (bytes + 255) & ~(size_t)255;
        in_use -= bytes;
        auto it = free_.emplace(off, bytes).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }

  private:
    std::map<size_t, size_t> free_;
};

struct SJob {
    int64_t id = 0;
    std::vector<double> V;
    std::vector<int32_t> F;
    std::vector<float> T;
    std::vector<float> W;  // per-triangle densities (empty: 1)
    dm_grid grid;
    dm_psf psf;
    dm_fit_options fit;
    int label = DM_SURFACE;
    int optimizer = DM_OPT_ADAM;
    double lambda = 50.0;
    double lr_decay = 1.0;  // per-step factor on the learning rates
    int fsplits = 1;                 // triangle splits of the batched forward (fixed by the job's sizes)
    float2* S_part = nullptr;        // [fsplits][M] partial spectra when fsplits > 1
    int state = DM_JOB_QUEUED;
    int steps_done = 0;
    double terms_step = 0;  // triangle-frequency terms of one step (triangles x half-spectrum size)
    double t_last = 0;      // when the job last advanced (or was admitted)
    // checkpoint / resume: the optimiser state the job starts from, and the one it stopped at
    int64_t step0 = 0;
    bool has_resume = false, preempt_req = false;
    std::vector<double> r_mV, r_vV, r_warm;
    double r_ms[3] = {0, 0, 0}, r_vs[3] = {0, 0, 0};
    std::vector<double> ck_V, ck_mV, ck_vV, ck_warm;
    double ck_sigma[3] = {0, 0, 0}, ck_ms[3] = {0, 0, 0}, ck_vs[3] = {0, 0, 0};
    int64_t ck_step = 0;
    double t_submit = 0, t_start = 0, t_end = 0, last_loss = NAN;
    // device state
    size_t off = 0, bytes = 0;
    Sizes z;
    Bufs b;
    double *mV = nullptr, *vV = nullptr, *ms = nullptr, *vs = nullptr, *hist = nullptr;
    int64_t* d_step = nullptr;  // Adam step t of the job's next step (device: a captured iteration replays unchanged)
    int64_t t_first = 1;        // its value at admission (host source of the upload)
    // large-steps state: Laplacian rows, solver work, warm starts, uniform-Adam step and maxima
    int32_t *lptr = nullptr, *lcol = nullptr;
    float* pcg_work = nullptr;
    double *gu = nullptr, *wv = nullptr, *dl = nullptr, *aup = nullptr;
    unsigned long long* cg_stats = nullptr;
    FFTAxis ax[3];
    int chunk_tiles = 1;
    cudaStream_t stream = nullptr;  // the job's stream for its own stage kernels (held while admitted)
    cudaEvent_t ev = nullptr;       // marks the end of the job's stage work within an iteration
    // results
    std::vector<double> V_out, hist_out;
    double sigma_out[3] = {0, 0, 0};
};

// Adjoint frequency tiles per work unit for a job: small enough that the job alone yields about
// 64 units per SM (so that a job running alone keeps every SM busy to the end of the launch: a
// 128^3 cell alone took 34.3 ms per served step at 8 units per SM, 31.7 ms at 64), at most
// max_tiles. It depends only on the job's own sizes, so a job's results do not depend on the other
// jobs in its iterations.
int job_chunk_tiles(const Sizes& z, int max_tiles, int sm_count) {
    const int64_t ftiles = (z.M_max + ADJ_FTILE - 1) / ADJ_FTILE;
    const int64_t tblocks = z.n_t_pad / ADJ_THREADS;
    const int64_t target = 64 * (int64_t)sm_count;
    int64_t c = (ftiles * tblocks + target - 1) / target;
    if (c < 1) c = 1;
    if (c > max_tiles) c = max_tiles;
    return (int)c;
}

size_t job_layout(const Sizes& z, int steps, int64_t n_v, Arena& A, Bufs& b, double** mom, double** hist,
                  SJob* J) {
    layout(z, A, b, true, true, !J->W.empty(), true, false);
    // forward units: (frequency block, triangle split), the split count chosen as for a single fit
    // (about 112 units per SM for the job alone, about four tiles per split) from the job's own sizes
    const int64_t fb = (z.M_max + FWD_BLOCK_FREQS - 1) / FWD_BLOCK_FREQS;
    const int n_tiles = (int)((z.n_t + FWD_REC_TILE - 1) / FWD_REC_TILE);
    J->fsplits = fwd_splits(fb, (n_tiles + 3) / 4, fwd_target_units(z.sm_count));
    J->S_part = J->fsplits > 1 ? A.take<float2>((size_t)J->fsplits * z.M_max) : nullptr;
    *mom = A.take<double>(6 * n_v + 8);
    *hist = A.take<double>(steps);
    J->d_step = A.take<int64_t>(1);
    if (J->optimizer == DM_OPT_LARGE_STEPS) {
        J->lptr = A.take<int32_t>(n_v + 1);
        J->lcol = A.take<int32_t>(6 * z.n_t);
        J->pcg_work = A.take<float>(pcg_work_elems(n_v));
        J->gu = A.take<double>(3 * n_v);
        J->wv = A.take<double>(3 * n_v);
        J->dl = A.take<double>(3 * n_v);
        J->aup = A.take<double>(adam_uniform_partials(3 * n_v));
        J->cg_stats = A.take<unsigned long long>(4);
    }
    return A.off + 256;
}

}  // namespace

struct dm_server {
    dm_ctx* ctx = nullptr;
    cudaStream_t st = nullptr;
    DeviceArena arena;
    int device = 0, max_jobs = 1, chunk_tiles = 32;
    int policy = DM_SCHED_FIFO;
    double batch_terms = 0, max_wait_s = 0;
    std::vector<SJob*> run;  // the resident jobs advanced by the current iteration
    std::mutex mu;
    std::condition_variable cv;
    std::deque<SJob*> pending;
    std::vector<SJob*> active;
    std::unordered_map<int64_t, SJob*> jobs;
    int64_t next_id = 1;
    bool stop = false;
    std::thread engine;
    std::chrono::steady_clock::time_point t0;
    dm_server_stats stats;
    // unit lists (rebuilt when the active set changes) and their staging
    bool dirty = true;
    std::vector<BatchFwdJob> fj;
    std::vector<BatchAdjJob> aj;
    std::vector<BatchUnit> uf, ua;   // surface jobs' units first, then volume jobs'
    size_t nf_surf = 0, na_surf = 0; // how many units of uf / ua belong to surface jobs
    BatchFwdJob* d_fj = nullptr;
    BatchAdjJob* d_aj = nullptr;
    BatchUnit *d_uf = nullptr, *d_ua = nullptr;
    size_t cap_fj = 0, cap_aj = 0, cap_uf = 0, cap_ua = 0;
    int* d_counter = nullptr;
    double* h_loss = nullptr;  // pinned, one per batch slot
    double* d_losses = nullptr;  // device, one per batch slot (written by the batched tick)
    // batched stage launches: the job table, per-stage block offsets, FFT pass groups
    std::vector<StageJob> sj;
    std::vector<int> offs;  // [BS_COUNT][nj + 1]
    int totals[BS_COUNT] = {0};
    struct FFTGroup {
        int kind, N, dir, nj, total;
        size_t jobs_at, offs_at;  // into fftj / fft_offs
    };
    std::vector<FFTGroup> c2r_groups, r2c_groups;  // in launch order (x, y, z passes; z, y, x passes)
    std::vector<FFTJob> fftj;
    std::vector<int> fft_offs;
    StageJob* d_sj = nullptr;
    int *d_offs = nullptr, *d_fft_offs = nullptr;
    FFTJob* d_fftj = nullptr;
    size_t cap_sj = 0, cap_offs = 0, cap_fftj = 0, cap_fft_offs = 0;
    int grid_fwd[2] = {0, 0}, grid_adj[2] = {0, 0};  // persistent grid per label
    std::vector<std::pair<cudaStream_t, cudaEvent_t>> free_streams;  // job streams not in use
    cudaEvent_t ev_fwd = nullptr, ev_adj = nullptr;                  // after each batched launch
    int64_t since_sync = 0;
    bool use_graphs = true;              // capture an iteration and replay it while the job set is unchanged
    cudaGraphExec_t gexec = nullptr;     // the captured iteration of the current job set
    int64_t graph_launches = 0;          // kernels one replay launches
    int64_t same_run = 0;                // iterations run over the current job set

    double now() const { return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count(); }
};

namespace {

bool grow(void** p, size_t* cap, size_t need, size_t elem) {
    if (need <= *cap) return true;
    if (*p) cudaFree(*p);
    *p = nullptr;
    size_t n = std::max(need, *cap * 2 + 16);
    if (cudaMalloc(p, n * elem) != cudaSuccess) {
        cudaGetLastError();
        *cap = 0;
        return false;
    }
    *cap = n;
    return true;
}

// Device state of an admitted job; returns false (nothing held) if the arena has no room.
bool setup_job(dm_server* S, SJob* J) {
    dm_ctx* ctx = S->ctx;
    Sizes z = make_sizes(ctx, &J->grid, (int64_t)J->V.size() / 3, (int64_t)J->F.size() / 3, J->psf.band_tau > 0,
                         J->label);
    z.fwd_split = false;  // the batched forward takes whole triangle lists
    const int64_t ftiles = (z.M_max + ADJ_FTILE - 1) / ADJ_FTILE;
    J->chunk_tiles = job_chunk_tiles(z, S->chunk_tiles, ctx->sm_count);
    z.n_chunks = (int)((ftiles + J->chunk_tiles - 1) / J->chunk_tiles);  // fixed per job
    Arena A;
    Bufs b;
    double *mom, *hist;
    const size_t bytes = job_layout(z, J->fit.steps, z.n_v, A, b, &mom, &hist, J);
    size_t off;
    if (!S->arena.alloc(bytes, &off)) return false;
    A.base = S->arena.base + off;
    A.off = 0;
    job_layout(z, J->fit.steps, z.n_v, A, b, &mom, &hist, J);
    J->off = off;
    J->bytes = bytes;
    J->z = z;
    J->b = b;
    J->mV = mom;
    J->vV = mom + 3 * z.n_v;
    J->ms = mom + 6 * z.n_v;
    J->vs = J->ms + 4;
    J->hist = hist;
    J->t_first = J->step0 + 1;
    if (S->free_streams.empty()) {
        cudaStream_t js;
        cudaEvent_t je;
        if (cudaStreamCreateWithFlags(&js, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&je, cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            S->arena.release_block(off, bytes);
            return false;
        }
        S->free_streams.push_back({js, je});
    }
    J->stream = S->free_streams.back().first;
    J->ev = S->free_streams.back().second;
    S->free_streams.pop_back();
    cudaStream_t st = J->stream;
    bool ok = cudaMemcpyAsync(b.V, J->V.data(), J->V.size() * sizeof(double), cudaMemcpyHostToDevice, st) ==
                  cudaSuccess &&
              cudaMemcpyAsync(b.F, J->F.data(), J->F.size() * sizeof(int32_t), cudaMemcpyHostToDevice, st) ==
                  cudaSuccess &&
              cudaMemcpyAsync(b.target, J->T.data(), J->T.size() * sizeof(float), cudaMemcpyHostToDevice, st) ==
                  cudaSuccess &&
              (J->W.empty() ||
               cudaMemcpyAsync(b.wts, J->W.data(), J->W.size() * sizeof(float), cudaMemcpyHostToDevice, st) ==
                   cudaSuccess) &&
              cudaMemsetAsync(mom, 0, (6 * z.n_v + 8) * sizeof(double), st) == cudaSuccess &&
              launch_set_params(b.d_params, psf_params(&J->psf), 9, st) == cudaSuccess &&
              cudaMemcpyAsync(J->d_step, &J->t_first, sizeof(int64_t), cudaMemcpyHostToDevice, st) == cudaSuccess &&
              launch_csr(b.F, z.n_t, z.n_v, b.cnt, b.ptr, b.ent, ctx->d_err, st) == cudaSuccess &&
              fft_axes(ctx, J->grid.n, J->ax) == DM_OK;
    g_launches += 5;
    if (ok && J->optimizer == DM_OPT_LARGE_STEPS) {
        ok = launch_laplacian(b.F, b.ptr, b.ent, z.n_v, b.cnt, J->lptr, J->lcol, ctx->d_err, st) == cudaSuccess &&
             cudaMemsetAsync(J->gu, 0, 3 * z.n_v * sizeof(double), st) == cudaSuccess &&
             cudaMemsetAsync(J->wv, 0, 3 * z.n_v * sizeof(double), st) == cudaSuccess &&
             cudaMemsetAsync(J->cg_stats, 0, 4 * sizeof(unsigned long long), st) == cudaSuccess;
        g_launches += 3;
        if (ok && J->has_resume && J->r_warm.size() == (size_t)6 * z.n_v)
            ok = cudaMemcpyAsync(J->gu, J->r_warm.data(), 3 * z.n_v * sizeof(double), cudaMemcpyHostToDevice, st) ==
                     cudaSuccess &&
                 cudaMemcpyAsync(J->wv, J->r_warm.data() + 3 * z.n_v, 3 * z.n_v * sizeof(double),
                                 cudaMemcpyHostToDevice, st) == cudaSuccess;
    }
    // the band of a job that keeps its PSF is the same at every step: computed once here (a job that
    // learns sigma recomputes it every step)
    if (ok && z.band && J->fit.lr_psf <= 0) {
        ok = launch_band(b.d_params, J->psf.kind, J->psf.band_tau, J->grid.n[0], J->grid.n[1], J->grid.n[2],
                         make_geom(&J->grid), b.band_idx, b.dM, b.band_counts, st) == cudaSuccess;
        g_launches += 3;
    }
    if (ok && J->has_resume) {
        const int64_t nV = 3 * z.n_v;
        ok = cudaMemcpyAsync(J->mV, J->r_mV.data(), nV * sizeof(double), cudaMemcpyHostToDevice, st) == cudaSuccess &&
             cudaMemcpyAsync(J->vV, J->r_vV.data(), nV * sizeof(double), cudaMemcpyHostToDevice, st) == cudaSuccess &&
             cudaMemcpyAsync(J->ms, J->r_ms, 3 * sizeof(double), cudaMemcpyHostToDevice, st) == cudaSuccess &&
             cudaMemcpyAsync(J->vs, J->r_vs, 3 * sizeof(double), cudaMemcpyHostToDevice, st) == cudaSuccess;
    }
    // iterations with a single job run its stage kernels on the server stream: order them after the uploads
    if (ok) ok = cudaEventRecord(J->ev, st) == cudaSuccess && cudaStreamWaitEvent(S->st, J->ev, 0) == cudaSuccess;
    // host vectors stay until the uploads have run (synchronised at the end of the iteration)
    if (!ok) {
        cudaGetLastError();
        S->arena.release_block(off, bytes);
        S->free_streams.push_back({J->stream, J->ev});
        return false;
    }
    return true;
}

// The batched stage launches of the jobs in S->run: one StageJob per job (index as in S->run), the
// per-stage block offsets, and the FFT passes grouped by line length.
void build_stage_tables(dm_server* S) {
    const int nj = (int)S->run.size();
    const int sms = S->ctx->sm_count;
    S->sj.resize(nj);
    for (int j = 0; j < nj; ++j) {
        const SJob* J = S->run[j];
        const Sizes& z = J->z;
        const Bufs& b = J->b;
        StageJob& q = S->sj[j];
        memset(&q, 0, sizeof(q));
        q.mode = J->label;
        q.psf_kind = J->psf.kind;
        q.loss_kind = J->fit.loss;
        q.band = z.band ? 1 : 0;
        q.n_v = z.n_v;
        q.n_t = z.n_t;
        q.n_t_pad = z.n_t_pad;
        q.N = z.N;
        q.nH = z.nH;
        q.M_pad = z.M_pad;
        q.g = make_geom(&J->grid);
        q.V = b.V;
        q.F = b.F;
        q.wts = b.wts;
        q.tris = (TriF32*)b.tris;
        q.params = b.d_params;
        q.partial = b.partial;
        q.fs = S->fj[j].fs;
        q.S = (float2*)b.S;
        q.S_part = J->S_part;
        q.fsplits = J->fsplits;
        q.rc_slices = reduce_slices_for(z.n_t, z.nacc, z.n_chunks, sms);
        q.spec = (Cx<float>*)b.spec;
        q.image = (float*)b.image;
        q.target = (const float*)b.target;
        q.resid = (float*)b.resid;
        q.fr = (FreqPairF32*)b.fr;
        q.adjp = (const float*)b.adjp;
        q.n_chunks = z.n_chunks;
        q.nacc = z.nacc;
        q.acc = b.acc;
        q.red = b.red;
        q.contrib = b.contrib;
        q.ptr = b.ptr;
        q.ent = b.ent;
        q.dV = b.dV;
        q.vertex_adam = J->optimizer == DM_OPT_ADAM ? 1 : 0;
        q.mV = J->mV;
        q.vV = J->vV;
        q.ms = J->ms;
        q.vs = J->vs;
        q.hist = J->hist;
        q.d_step = J->d_step;
        q.step0 = J->step0;
        q.lr_v = J->fit.lr_vertex;
        q.lr_psf = J->fit.lr_psf;
        q.b1 = J->fit.beta1;
        q.b2 = J->fit.beta2;
        q.eps = J->fit.eps;
        q.decay = J->lr_decay;
    }
    S->offs.assign((size_t)BS_COUNT * (nj + 1), 0);
    for (int j = 0; j < nj; ++j) {
        int c[BS_COUNT];
        batch_stage_blocks(S->sj[j], sms, c);
        for (int st = 0; st < BS_COUNT; ++st) {
            int* o = S->offs.data() + (size_t)st * (nj + 1);
            o[j + 1] = o[j] + c[st];
        }
    }
    for (int st = 0; st < BS_COUNT; ++st) S->totals[st] = S->offs[(size_t)st * (nj + 1) + nj];
    // FFT passes: inverse x, y, z (complex, complex, complex-to-real), forward z, y, x; each pass grouped
    // by line length (one launch per length)
    S->fftj.clear();
    S->fft_offs.clear();
    S->c2r_groups.clear();
    S->r2c_groups.clear();
    const auto add_pass = [&](std::vector<dm_server::FFTGroup>& out, int kind, int dir, int axis) {
        std::map<int, std::vector<FFTJob>> by_n;
        for (int j = 0; j < nj; ++j) {
            const SJob* J = S->run[j];
            const int* n = J->grid.n;
            if (kind == FFT_STRIDED && n[axis] <= 1) continue;  // a length-1 axis needs no pass
            const int Nzh = n[2] / 2 + 1;
            FFTJob f;
            f.ax = J->ax[axis];
            f.Nzh = Nzh;
            if (kind == FFT_STRIDED) {
                f.src = f.dst = J->b.spec;
                f.inner = axis == 0 ? (int64_t)n[1] * Nzh : Nzh;
                f.lines = axis == 0 ? 1 : n[0];
            } else {
                f.src = kind == FFT_Z_C2R ? J->b.spec : J->b.resid;
                f.dst = kind == FFT_Z_C2R ? J->b.image : J->b.spec;
                f.inner = 0;
                f.lines = (int64_t)n[0] * n[1];
            }
            by_n[f.ax.N].push_back(f);
        }
        for (auto& kv : by_n) {
            dm_server::FFTGroup g;
            g.kind = kind;
            g.N = kv.first;
            g.dir = dir;
            g.nj = (int)kv.second.size();
            g.jobs_at = S->fftj.size();
            g.offs_at = S->fft_offs.size();
            int total = 0;
            S->fft_offs.push_back(0);
            for (const FFTJob& f : kv.second) {
                S->fftj.push_back(f);
                total += (int)fft_pass_blocks(kind, f);
                S->fft_offs.push_back(total);
            }
            g.total = total;
            out.push_back(g);
        }
    };
    add_pass(S->c2r_groups, FFT_STRIDED, +1, 0);
    add_pass(S->c2r_groups, FFT_STRIDED, +1, 1);
    add_pass(S->c2r_groups, FFT_Z_C2R, +1, 2);
    add_pass(S->r2c_groups, FFT_Z_R2C, -1, 2);
    add_pass(S->r2c_groups, FFT_STRIDED, -1, 1);
    add_pass(S->r2c_groups, FFT_STRIDED, -1, 0);
}

bool rebuild_units(dm_server* S) {
    const size_t nj = S->run.size();
    S->fj.resize(nj);
    S->aj.resize(nj);
    S->uf.clear();
    S->ua.clear();
    std::vector<int> order(nj);
    for (size_t j = 0; j < nj; ++j) {
        SJob* J = S->run[j];
        const Sizes& z = J->z;
        const Bufs& b = J->b;
        const Geom G = make_geom(&J->grid);
        BatchFwdJob& f = S->fj[j];
        f.tris = (const TriF32*)b.tris;
        f.n_tiles = (int)((z.n_t + FWD_REC_TILE - 1) / FWD_REC_TILE);
        f.last = (int)(z.n_t - (int64_t)(f.n_tiles - 1) * FWD_REC_TILE);
        f.mode = J->label;
        f.fs.nlist = nullptr;
        f.fs.idx = z.band ? b.band_idx : nullptr;
        f.fs.dM = z.band ? b.dM : nullptr;
        f.fs.M = z.nH;
        f.fs.set_dims(J->grid.n[0], J->grid.n[1], J->grid.n[2]);
        for (int a = 0; a < 3; ++a) f.tp[a] = (float)(2.0 * M_PI / G.L[a]);
        f.d_vol = b.d_params + 16;
        f.S = (float2*)b.S;
        f.splits = J->fsplits;
        f.S_part = J->S_part;
        BatchAdjJob& a = S->aj[j];
        a.tris = (const TriF32*)b.tris;
        a.n_t = z.n_t;
        a.n_t_pad = z.n_t_pad;
        a.fr = (const FreqPairF32*)b.fr;
        a.dM = z.band ? b.dM : nullptr;
        a.M_max = z.M_max;
        a.mode = J->label;
        a.chunk_tiles = J->chunk_tiles;
        a.partial = (float*)b.adjp;
        order[j] = (int)j;
    }
    // surface jobs before volume jobs (one launch per label), largest triangle counts first within
    // each: their forward units cost the most
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
        const SJob *a = S->run[x], *b = S->run[y];
        return a->label != b->label ? a->label < b->label : a->z.n_t > b->z.n_t;
    });
    S->nf_surf = S->na_surf = 0;
    for (int j : order) {
        const int64_t nb = (S->run[j]->z.nH + FWD_BLOCK_FREQS - 1) / FWD_BLOCK_FREQS;
        for (int64_t k = 0; k < nb; ++k)
            for (int sp = 0; sp < S->run[j]->fsplits; ++sp) S->uf.push_back({j, (int)k, sp, 0});
        if (S->run[j]->label == DM_SURFACE) S->nf_surf = S->uf.size();
    }
    for (int j : order) {
        const Sizes& z = S->run[j]->z;
        const int64_t tb = z.n_t_pad / ADJ_THREADS;
        for (int c = 0; c < z.n_chunks; ++c)
            for (int64_t t = 0; t < tb; ++t) S->ua.push_back({j, (int)t, c, 0});
        if (S->run[j]->label == DM_SURFACE) S->na_surf = S->ua.size();
    }
    build_stage_tables(S);
    bool ok = grow((void**)&S->d_fj, &S->cap_fj, nj, sizeof(BatchFwdJob)) &&
              grow((void**)&S->d_aj, &S->cap_aj, nj, sizeof(BatchAdjJob)) &&
              grow((void**)&S->d_uf, &S->cap_uf, S->uf.size(), sizeof(BatchUnit)) &&
              grow((void**)&S->d_ua, &S->cap_ua, S->ua.size(), sizeof(BatchUnit)) &&
              grow((void**)&S->d_sj, &S->cap_sj, nj, sizeof(StageJob)) &&
              grow((void**)&S->d_offs, &S->cap_offs, S->offs.size(), sizeof(int)) &&
              grow((void**)&S->d_fftj, &S->cap_fftj, std::max<size_t>(1, S->fftj.size()), sizeof(FFTJob)) &&
              grow((void**)&S->d_fft_offs, &S->cap_fft_offs, std::max<size_t>(1, S->fft_offs.size()), sizeof(int));
    // the tables change only with the set of jobs advanced, so they are uploaded here (stream-ordered
    // after the previous iteration's batched launches) and not every iteration
    cudaStream_t st = S->st;
    ok = ok && cudaMemcpyAsync(S->d_fj, S->fj.data(), nj * sizeof(BatchFwdJob), cudaMemcpyHostToDevice, st) == cudaSuccess;
    ok = ok && cudaMemcpyAsync(S->d_aj, S->aj.data(), nj * sizeof(BatchAdjJob), cudaMemcpyHostToDevice, st) == cudaSuccess;
    ok = ok && cudaMemcpyAsync(S->d_uf, S->uf.data(), S->uf.size() * sizeof(BatchUnit), cudaMemcpyHostToDevice, st) ==
                   cudaSuccess;
    ok = ok && cudaMemcpyAsync(S->d_ua, S->ua.data(), S->ua.size() * sizeof(BatchUnit), cudaMemcpyHostToDevice, st) ==
                   cudaSuccess;
    ok = ok && cudaMemcpyAsync(S->d_sj, S->sj.data(), nj * sizeof(StageJob), cudaMemcpyHostToDevice, st) == cudaSuccess;
    ok = ok && cudaMemcpyAsync(S->d_offs, S->offs.data(), S->offs.size() * sizeof(int), cudaMemcpyHostToDevice, st) ==
                   cudaSuccess;
    ok = ok && (S->fftj.empty() || cudaMemcpyAsync(S->d_fftj, S->fftj.data(), S->fftj.size() * sizeof(FFTJob),
                                                   cudaMemcpyHostToDevice, st) == cudaSuccess);
    ok = ok && (S->fft_offs.empty() || cudaMemcpyAsync(S->d_fft_offs, S->fft_offs.data(),
                                                       S->fft_offs.size() * sizeof(int), cudaMemcpyHostToDevice,
                                                       st) == cudaSuccess);
    S->dirty = !ok;
    return ok;
}

// Enqueue one optimiser step of every job in S->run on the server stream: each stage of the step is one
// launch over all jobs (job table, per-job block counts fixed by each job's own sizes), the two
// mesh-transform sums are the persistent batched launches, and only a large-steps job's smoothing
// solves and uniform-Adam step run as launches of their own. Every value that changes from step to
// step lives on the device (the Adam step counters), so the same sequence can be captured once and
// replayed. Adds the kernels it launches to *nl_out; false if an enqueue failed.
bool enqueue_step(dm_server* S, int64_t* nl_out) {
    dm_ctx* ctx = S->ctx;
    cudaStream_t st = S->st;
    const int nj = (int)S->run.size();
    bool ok = true;
    int64_t nlk = 0;
    const auto stage = [&](int s) {
        if (S->totals[s] <= 0) return;
        ok &= launch_batch_stage(s, S->d_sj, S->d_offs, nj, S->totals[s], ctx->d_err, st) == cudaSuccess;
        nlk += 1;
    };
    const auto stage_sum = [&](int s, int count, int dst) {
        ok &= launch_batch_sum(S->d_sj, S->d_offs + (size_t)s * (nj + 1), nj, count, dst, nullptr, st) == cudaSuccess;
        nlk += 1;
    };
    const auto fft = [&](const std::vector<dm_server::FFTGroup>& groups) {
        for (const auto& g : groups) {
            ok &= launch_fft_batch(g.kind, g.N, S->d_fftj + g.jobs_at, S->d_fft_offs + g.offs_at, g.nj, g.total, g.dir,
                                   st) == cudaSuccess;
            nlk += 1;
        }
    };
    // triangle records and normalisers; the bands of jobs that learn sigma
    stage(BS_PREP);
    stage_sum(BS_PREP, 1, 16);
    for (SJob* J : S->run) {
        if (!J->z.band || J->fit.lr_psf <= 0) continue;
        ok &= launch_band(J->b.d_params, J->psf.kind, J->psf.band_tau, J->grid.n[0], J->grid.n[1], J->grid.n[2],
                          make_geom(&J->grid), J->b.band_idx, J->b.dM, J->b.band_counts, st) == cudaSuccess;
        nlk += 3;
    }
    // mesh-transform sums: one persistent launch per label present, surface units first (grids no
    // larger than the unit lists, so a small batch launches no idle blocks)
    const size_t nfl[2] = {S->nf_surf, S->uf.size() - S->nf_surf};
    const size_t nal[2] = {S->na_surf, S->ua.size() - S->na_surf};
    for (int m = 0; m < 2; ++m) {
        if (nfl[m] == 0) continue;
        const int gf = (int)std::min<size_t>((size_t)S->grid_fwd[m], nfl[m]);
        ok &= launch_fwd_batch_f32(m, S->d_fj, S->d_uf + (m ? S->nf_surf : 0), (int)nfl[m], S->d_counter, gf,
                                   ctx->d_err, st) == cudaSuccess;
        nlk += 1;
    }
    stage(BS_FWDRED);
    // image, loss, adjoint records
    stage(BS_ZERO);
    stage(BS_SCATTER);
    fft(S->c2r_groups);
    stage(BS_LOSS);
    stage_sum(BS_LOSS, 1, 17);
    fft(S->r2c_groups);
    stage(BS_GATHER);
    stage_sum(BS_GATHER, 8, 24);
    for (int m = 0; m < 2; ++m) {
        if (nal[m] == 0) continue;
        const int ga = (int)std::min<size_t>((size_t)S->grid_adj[m], nal[m]);
        ok &= launch_adj_batch_f32(m, S->d_aj, S->d_ua + (m ? S->na_surf : 0), (int)nal[m], S->d_counter, ga,
                                   ctx->d_err, st) == cudaSuccess;
        nlk += 1;
    }
    // per-vertex gradients and the update
    stage(BS_REDUCE);
    stage(BS_SLICES);
    stage(BS_ASSEMBLE);
    stage(BS_VGATHER);
    stage(BS_ADAM);
    for (SJob* J : S->run) {
        if (J->optimizer != DM_OPT_LARGE_STEPS) continue;
        // v -= (1 + lambda L)^-1 AdamUniform((1 + lambda L)^-1 dL/dv), step t = *J->d_step
        const dm_fit_options& o = J->fit;
        const int64_t n_v = J->z.n_v;
        ok &= launch_pcg<float>(J->lptr, J->lcol, n_v, J->lambda, J->b.dV, J->gu, nullptr, J->pcg_work, 1e-6, 2000,
                                J->cg_stats, st) == cudaSuccess;
        ok &= launch_adam_uniform(J->gu, J->mV, J->vV, J->dl, 3 * n_v, o.lr_vertex, o.beta1, o.beta2, o.eps, 0, J->aup,
                                  st, J->d_step, J->lr_decay) == cudaSuccess;
        ok &= launch_pcg<float>(J->lptr, J->lcol, n_v, J->lambda, J->dl, J->wv, J->b.V, J->pcg_work, 1e-6, 2000,
                                J->cg_stats, st) == cudaSuccess;
        nlk += 4;
    }
    // sigma (lr_psf > 0), the loss history and the step counters; the losses to the host
    ok &= launch_batch_tick(S->d_sj, nj, S->d_losses, st) == cudaSuccess;
    ok &= cudaMemcpyAsync(S->h_loss, S->d_losses, nj * sizeof(double), cudaMemcpyDeviceToHost, st) == cudaSuccess;
    nlk += 1;
    *nl_out += nlk;
    return ok;
}

// Drop the captured iteration (the set of jobs it advances changed).
void drop_graph(dm_server* S) {
    if (S->gexec) cudaGraphExecDestroy(S->gexec);  // freed once its launches in flight complete
    S->gexec = nullptr;
    S->same_run = 0;
}

// One Adam step of every job in S->run. The first iteration after the set of jobs changes runs
// directly (it uploads the unit tables and raises kernel attributes); the second is captured as a
// CUDA graph, which later iterations over the same set replay with one launch. Synchronises only
// when `sync` is set; returns false on a device fault seen at a sync.
bool iterate(dm_server* S, bool sync) {
    dm_ctx* ctx = S->ctx;
    cudaStream_t st = S->st;
    if (S->dirty) {
        drop_graph(S);
        if (!rebuild_units(S)) return false;
    }
    const size_t nj = S->run.size();
    bool ok = true;
    int64_t nl = 0;
    if (S->gexec) {
        ok = cudaGraphLaunch(S->gexec, st) == cudaSuccess;
        nl = S->graph_launches;
        std::lock_guard<std::mutex> lk(S->mu);
        S->stats.graph_replays += 1;
    } else if (S->use_graphs && S->same_run >= 1) {
        cudaGraph_t g = nullptr;
        bool cap = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
        if (cap) {
            cap = enqueue_step(S, &nl);
            cap = cudaStreamEndCapture(st, &g) == cudaSuccess && cap && g != nullptr;
            cap = cap && cudaGraphInstantiate(&S->gexec, g, 0) == cudaSuccess;
            if (g) cudaGraphDestroy(g);
        }
        if (cap) {
            S->graph_launches = nl;
            ok = cudaGraphLaunch(S->gexec, st) == cudaSuccess;
            std::lock_guard<std::mutex> lk(S->mu);
            S->stats.graph_replays += 1;
        } else {
            // the capture failed (nothing of it ran): run this and later iterations directly
            cudaGetLastError();
            S->gexec = nullptr;
            S->use_graphs = false;
            nl = 0;
            ok = enqueue_step(S, &nl);
        }
    } else {
        ok = enqueue_step(S, &nl);
    }
    g_launches += nl;
    S->same_run += 1;
    for (size_t j = 0; j < nj; ++j) S->run[j]->steps_done += 1;
    if (sync) {
        ok &= cudaStreamSynchronize(st) == cudaSuccess;
        for (SJob* J : S->run) ok &= cudaStreamSynchronize(J->stream) == cudaSuccess;
        int h = 0;
        ok &= cudaMemcpy(&h, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost) == cudaSuccess;
        if (h) {
            cudaMemset(ctx->d_err, 0, sizeof(int));
            ok = false;
        }
        for (size_t j = 0; j < nj; ++j) S->run[j]->last_loss = S->h_loss[j];
    }
    if (!ok) cudaGetLastError();
    return ok;
}

void finish_job(dm_server* S, SJob* J, int state) {
    if (state == DM_JOB_PREEMPTED) {
        // the job's stage work and the batched launches that read its buffers are complete
        cudaStreamSynchronize(J->stream);
        cudaStreamSynchronize(S->st);
        const int64_t nV = 3 * J->z.n_v;
        J->ck_V.resize(nV);
        J->ck_mV.resize(nV);
        J->ck_vV.resize(nV);
        cudaMemcpy(J->ck_V.data(), J->b.V, nV * sizeof(double), cudaMemcpyDeviceToHost);
        cudaMemcpy(J->ck_mV.data(), J->mV, nV * sizeof(double), cudaMemcpyDeviceToHost);
        cudaMemcpy(J->ck_vV.data(), J->vV, nV * sizeof(double), cudaMemcpyDeviceToHost);
        cudaMemcpy(J->ck_ms, J->ms, 3 * sizeof(double), cudaMemcpyDeviceToHost);
        cudaMemcpy(J->ck_vs, J->vs, 3 * sizeof(double), cudaMemcpyDeviceToHost);
        cudaMemcpy(J->ck_sigma, J->b.d_params, 3 * sizeof(double), cudaMemcpyDeviceToHost);
        if (J->optimizer == DM_OPT_LARGE_STEPS) {
            J->ck_warm.resize(2 * nV);
            cudaMemcpy(J->ck_warm.data(), J->gu, nV * sizeof(double), cudaMemcpyDeviceToHost);
            cudaMemcpy(J->ck_warm.data() + nV, J->wv, nV * sizeof(double), cudaMemcpyDeviceToHost);
        }
        J->ck_step = J->step0 + J->steps_done;
    }
    if (state == DM_JOB_DONE) {
        const int64_t nV = 3 * J->z.n_v;
        J->V_out.resize(nV);
        J->hist_out.resize(J->fit.steps);
        cudaMemcpy(J->V_out.data(), J->b.V, nV * sizeof(double), cudaMemcpyDeviceToHost);
        cudaMemcpy(J->sigma_out, J->b.d_params, 3 * sizeof(double), cudaMemcpyDeviceToHost);
        cudaMemcpy(J->hist_out.data(), J->hist, J->fit.steps * sizeof(double), cudaMemcpyDeviceToHost);
    }
    S->arena.release_block(J->off, J->bytes);
    if (J->stream) S->free_streams.push_back({J->stream, J->ev});
    J->stream = nullptr;
    std::vector<double>().swap(J->V);
    std::vector<int32_t>().swap(J->F);
    std::vector<float>().swap(J->T);
    std::vector<float>().swap(J->W);
    std::lock_guard<std::mutex> lk(S->mu);
    J->state = state;
    J->t_end = S->now();
    if (state == DM_JOB_DONE) S->stats.jobs_done += 1;
}

// Jobs whose checkpoint was requested leave at this iteration boundary with their state on the host;
// queued ones leave with the state they were submitted with.
void handle_preempts(dm_server* S) {
    std::vector<SJob*> keep;
    bool any = false;
    for (SJob* J : S->active) {
        bool req;
        {
            std::lock_guard<std::mutex> lk(S->mu);
            req = J->preempt_req;
        }
        if (req) {
            finish_job(S, J, DM_JOB_PREEMPTED);
            any = true;
        } else {
            keep.push_back(J);
        }
    }
    if (any) {
        S->active.swap(keep);
        S->dirty = true;
        S->run.clear();
    }
    std::lock_guard<std::mutex> lk(S->mu);
    for (auto it = S->pending.begin(); it != S->pending.end();) {
        SJob* J = *it;
        if (!J->preempt_req) {
            ++it;
            continue;
        }
        const size_t nV = J->V.size();
        J->ck_V = J->V;
        J->ck_mV = J->has_resume ? J->r_mV : std::vector<double>(nV, 0.0);
        J->ck_vV = J->has_resume ? J->r_vV : std::vector<double>(nV, 0.0);
        if (J->optimizer == DM_OPT_LARGE_STEPS)
            J->ck_warm = J->r_warm.size() == 2 * nV ? J->r_warm : std::vector<double>(2 * nV, 0.0);
        for (int a = 0; a < 3; ++a) {
            J->ck_sigma[a] = J->psf.sigma[a];
            J->ck_ms[a] = J->r_ms[a];
            J->ck_vs[a] = J->r_vs[a];
        }
        J->ck_step = J->step0;
        J->state = DM_JOB_PREEMPTED;
        J->t_end = S->now();
        std::vector<double>().swap(J->V);
        std::vector<int32_t>().swap(J->F);
        std::vector<float>().swap(J->T);
        std::vector<float>().swap(J->W);
        it = S->pending.erase(it);
        any = true;
    }
    if (any) S->cv.notify_all();
}

// Remaining work of a job in triangle-frequency terms.
double remaining(const SJob* J) { return (double)(J->fit.steps - J->steps_done) * J->terms_step; }

// The resident jobs an iteration advances: all of them (FIFO), or (SHORTEST) jobs idle for longer
// than max_wait_s, then the least remaining work first, while the iteration's terms stay within
// batch_terms (the first job always runs).
std::vector<SJob*> select_run(dm_server* S) {
    if (S->policy != DM_SCHED_SHORTEST) return S->active;
    std::vector<SJob*> c = S->active;
    const double now = S->now();
    const auto aged = [&](const SJob* J) { return S->max_wait_s > 0 && now - J->t_last > S->max_wait_s; };
    std::stable_sort(c.begin(), c.end(), [&](const SJob* x, const SJob* y) {
        const bool ax = aged(x), ay = aged(y);
        if (ax != ay) return ax;
        return remaining(x) < remaining(y);
    });
    std::vector<SJob*> run;
    double terms = 0;
    for (SJob* J : c) {
        if (!run.empty() && S->batch_terms > 0 && terms + J->terms_step > S->batch_terms) continue;
        run.push_back(J);
        terms += J->terms_step;
    }
    return run;
}

void engine_main(dm_server* S) {
    cudaSetDevice(S->device);
    while (true) {
        {
            std::unique_lock<std::mutex> lk(S->mu);
            S->cv.wait(lk, [&] { return S->stop || !S->pending.empty() || !S->active.empty(); });
            if (S->stop) break;
        }
        handle_preempts(S);
        // admission: FIFO takes the head of the queue (a job that does not fit yet blocks the ones
        // behind it); SHORTEST takes the queued job with the least work, a long-waiting one first
        while ((int)S->active.size() < S->max_jobs) {
            SJob* J = nullptr;
            size_t pos = 0;
            {
                std::lock_guard<std::mutex> lk(S->mu);
                if (S->pending.empty()) break;
                if (S->policy == DM_SCHED_SHORTEST) {
                    const double now = S->now();
                    bool best_aged = false;
                    for (size_t k = 0; k < S->pending.size(); ++k) {
                        SJob* C = S->pending[k];
                        const bool aged = S->max_wait_s > 0 && now - C->t_submit > S->max_wait_s;
                        if (!J || (aged && !best_aged) || (aged == best_aged && remaining(C) < remaining(J))) {
                            J = C;
                            pos = k;
                            best_aged = aged;
                        }
                    }
                } else {
                    J = S->pending.front();
                }
            }
            if (!setup_job(S, J)) break;
            {
                std::lock_guard<std::mutex> lk(S->mu);
                S->pending.erase(S->pending.begin() + (std::ptrdiff_t)pos);
                J->state = DM_JOB_RUNNING;
                J->t_start = S->now();
                J->t_last = J->t_start;
            }
            S->active.push_back(J);
        }
        if (S->active.empty()) continue;
        S->stats.peak_active = std::max<int64_t>(S->stats.peak_active, (int64_t)S->active.size());
        std::vector<SJob*> run = select_run(S);
        if (run != S->run) {
            S->run.swap(run);
            S->dirty = true;
        }
        const double t_it = S->now();
        bool sync = ++S->since_sync >= 16;
        for (SJob* J : S->run) sync = sync || J->steps_done + 1 >= J->fit.steps;
        if (sync) S->since_sync = 0;
        const bool ok = iterate(S, sync);
        const double t_done = S->now();
        for (SJob* J : S->run) J->t_last = t_done;
        {
            std::lock_guard<std::mutex> lk(S->mu);
            S->stats.iterations += 1;
            S->stats.job_steps += (int64_t)S->run.size();
            S->stats.busy_s += t_done - t_it;
        }
        // retire
        std::vector<SJob*> keep;
        for (SJob* J : S->active) {
            if (!ok)
                finish_job(S, J, DM_JOB_FAILED);
            else if (J->steps_done >= J->fit.steps)
                finish_job(S, J, DM_JOB_DONE);
            else
                keep.push_back(J);
        }
        if (keep.size() != S->active.size()) {
            S->dirty = true;
            S->run.clear();
        }
        S->active.swap(keep);
        {
            std::lock_guard<std::mutex> lk(S->mu);
            S->stats.bytes_in_use = S->arena.in_use;
            S->stats.bytes_peak = S->arena.peak;
        }
        S->cv.notify_all();
    }
    // shutdown: release whatever is still admitted
    for (SJob* J : S->active) finish_job(S, J, DM_JOB_FAILED);
    S->active.clear();
    S->run.clear();
    S->cv.notify_all();
}

dm_status validate_job(const dm_job* j) {
    if (!j || !j->V || !j->F || !j->target || j->n_v < 3 || j->n_t < 1) return DM_ERR_ARG;
    if (j->fit.steps < 1 || j->fit.loss < 0 || j->fit.loss > 2) return DM_ERR_ARG;
    if (j->psf.kind != DM_PSF_DIAG) return DM_ERR_UNSUPPORTED;
    if (j->label != DM_SURFACE && j->label != DM_VOLUME) return DM_ERR_ARG;
    if (j->optimizer != DM_OPT_ADAM && j->optimizer != DM_OPT_LARGE_STEPS) return DM_ERR_ARG;
    if (j->resume) {
        if (j->resume->step < 0 || !j->resume->m_V || !j->resume->v_V) return DM_ERR_ARG;
        for (int a = 0; a < 3; ++a)
            if (!(j->resume->sigma[a] > 0) || !std::isfinite(j->resume->sigma[a])) return DM_ERR_ARG;
    }
    if (std::isnan(j->lambda)) return DM_ERR_ARG;
    if (!(j->lr_decay >= 0.0 && j->lr_decay <= 1.0)) return DM_ERR_ARG;
    if (j->tri_weight) {
        if (j->label != DM_SURFACE) return DM_ERR_ARG;
        bool any = false;
        for (int64_t t = 0; t < j->n_t; ++t) {
            const float w = j->tri_weight[t];
            if (!(w >= 0.f) || !std::isfinite(w)) return DM_ERR_ARG;
            any |= w > 0.f;
        }
        if (!any) return DM_ERR_ARG;
    }
    for (int a = 0; a < 3; ++a) {
        if (!(j->psf.sigma[a] > 0) || !(j->grid.h[a] > 0) || j->grid.n[a] < 1) return DM_ERR_ARG;
        FFTAxis ax;
        if (!fft_factor(j->grid.n[a], ax)) return DM_ERR_UNSUPPORTED;
    }
    if ((int64_t)j->grid.n[0] * j->grid.n[1] * (j->grid.n[2] / 2 + 1) >= ((int64_t)1 << 31)) return DM_ERR_UNSUPPORTED;
    for (int64_t i = 0; i < 3 * j->n_t; ++i)
        if (j->F[i] < 0 || j->F[i] >= j->n_v) return DM_ERR_ARG;
    for (int64_t i = 0; i < 3 * j->n_v; ++i)
        if (!std::isfinite(j->V[i])) return DM_ERR_ARG;
    return DM_OK;
}

}  // namespace

extern "C" {

dm_status dm_server_create(dm_server** out, const dm_server_options* opt) {
    if (!out || !opt || opt->max_jobs < 1) return DM_ERR_ARG;
    if (opt->policy != DM_SCHED_FIFO && opt->policy != DM_SCHED_SHORTEST) return DM_ERR_ARG;
    *out = nullptr;
    dm_options o{DM_FP32_MIXED, opt->device, 0};
    dm_ctx* ctx = nullptr;
    dm_status s = dm_create(&ctx, &o);
    if (s != DM_OK) return s;
    dm_server* S = new dm_server();
    S->ctx = ctx;
    S->device = opt->device;
    S->max_jobs = opt->max_jobs;
    S->chunk_tiles = opt->chunk_tiles > 0 ? opt->chunk_tiles : 1024;
    S->policy = opt->policy;
    S->batch_terms = opt->batch_terms;
    S->max_wait_s = opt->max_wait_s;
    S->use_graphs = opt->no_graphs == 0;
    S->t0 = std::chrono::steady_clock::now();
    memset(&S->stats, 0, sizeof(S->stats));
    DeviceGuard dg(opt->device);
    size_t bytes = opt->memory_bytes;
    if (bytes == 0) {
        size_t fr = 0, tot = 0;
        cudaMemGetInfo(&fr, &tot);
        bytes = fr / 2;
    }
    bool ok = S->arena.init(bytes) && cudaStreamCreateWithFlags(&S->st, cudaStreamNonBlocking) == cudaSuccess &&
              cudaMalloc(&S->d_counter, sizeof(int)) == cudaSuccess &&
              cudaMallocHost(&S->h_loss, sizeof(double) * (size_t)S->max_jobs) == cudaSuccess &&
              cudaMalloc(&S->d_losses, sizeof(double) * (size_t)S->max_jobs) == cudaSuccess &&
              cudaEventCreateWithFlags(&S->ev_fwd, cudaEventDisableTiming) == cudaSuccess &&
              cudaEventCreateWithFlags(&S->ev_adj, cudaEventDisableTiming) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        S->arena.release();
        if (S->st) cudaStreamDestroy(S->st);
        if (S->d_counter) cudaFree(S->d_counter);
        if (S->d_losses) cudaFree(S->d_losses);
        dm_destroy(ctx);
        delete S;
        return DM_ERR_OOM;
    }
    S->stats.bytes_total = S->arena.total;
    const int sms = ctx->sm_count;
    for (int m = 0; m < 2; ++m) {
        S->grid_fwd[m] = sms * batch_blocks_per_sm_fwd(m);
        S->grid_adj[m] = sms * batch_blocks_per_sm_adj(m);
    }
    S->engine = std::thread(engine_main, S);
    *out = S;
    return DM_OK;
}

dm_status dm_server_submit(dm_server* S, const dm_job* job, int64_t* job_id) {
    if (!S || !job_id) return DM_ERR_ARG;
    dm_status s = validate_job(job);
    if (s != DM_OK) return s;
    std::string why;  // degenerate or (volume label) open meshes are refused here, not mid-batch
    if ((s = check_mesh_host(job->V, job->n_v, job->F, job->n_t, job->tri_weight, job->label, &why)) != DM_OK) return s;
    SJob* J = new SJob();
    J->V.assign(job->V, job->V + 3 * job->n_v);
    J->F.assign(job->F, job->F + 3 * job->n_t);
    const int64_t N = (int64_t)job->grid.n[0] * job->grid.n[1] * job->grid.n[2];
    J->T.assign(job->target, job->target + N);
    if (job->tri_weight) J->W.assign(job->tri_weight, job->tri_weight + job->n_t);
    J->grid = job->grid;
    J->psf = job->psf;
    J->fit = job->fit;
    J->label = job->label;
    J->optimizer = job->optimizer;
    if (job->resume) {
        const dm_fit_state* r = job->resume;
        J->has_resume = true;
        J->step0 = r->step;
        J->r_mV.assign(r->m_V, r->m_V + 3 * job->n_v);
        J->r_vV.assign(r->v_V, r->v_V + 3 * job->n_v);
        if (r->warm) J->r_warm.assign(r->warm, r->warm + 6 * job->n_v);
        for (int a = 0; a < 3; ++a) {
            J->r_ms[a] = r->m_sigma[a];
            J->r_vs[a] = r->v_sigma[a];
            J->psf.sigma[a] = r->sigma[a];
        }
    }
    J->terms_step = (double)job->n_t * (double)job->grid.n[0] * job->grid.n[1] * (job->grid.n[2] / 2 + 1);
    J->lambda = job->lambda > 0 ? job->lambda : 50.0;
    J->lr_decay = job->lr_decay > 0 ? job->lr_decay : 1.0;
    // a job whose state can never fit the arena is refused now rather than queued forever
    Sizes z = make_sizes(S->ctx, &job->grid, job->n_v, job->n_t, job->psf.band_tau > 0, job->label);
    z.fwd_split = false;
    const int64_t ftiles = (z.M_max + ADJ_FTILE - 1) / ADJ_FTILE;
    const int ct = job_chunk_tiles(z, S->chunk_tiles, S->ctx->sm_count);
    z.n_chunks = (int)((ftiles + ct - 1) / ct);
    Arena A;
    Bufs b;
    double *mom, *hist;
    if (job_layout(z, job->fit.steps, job->n_v, A, b, &mom, &hist, J) > S->arena.total) {
        delete J;
        return DM_ERR_OOM;
    }
    {
        std::lock_guard<std::mutex> lk(S->mu);
        J->id = S->next_id++;
        J->t_submit = S->now();
        S->jobs[J->id] = J;
        S->pending.push_back(J);
        *job_id = J->id;
    }
    S->cv.notify_all();
    return DM_OK;
}

dm_status dm_server_status(dm_server* S, int64_t id, dm_job_status* out) {
    if (!S || !out) return DM_ERR_ARG;
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->jobs.find(id);
    if (it == S->jobs.end()) return DM_ERR_ARG;
    const SJob* J = it->second;
    out->state = J->state;
    out->steps_done = J->steps_done;
    out->t_submit = J->t_submit;
    out->t_start = J->t_start;
    out->t_end = J->t_end;
    out->last_loss = J->last_loss;
    return DM_OK;
}

dm_status dm_server_wait(dm_server* S, int64_t id, double timeout_s) {
    if (!S) return DM_ERR_ARG;
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->jobs.find(id);
    if (it == S->jobs.end()) return DM_ERR_ARG;
    SJob* J = it->second;
    auto done = [&] {
        return J->state == DM_JOB_DONE || J->state == DM_JOB_FAILED || J->state == DM_JOB_PREEMPTED || S->stop;
    };
    if (timeout_s < 0)
        S->cv.wait(lk, done);
    else if (!S->cv.wait_for(lk, std::chrono::duration<double>(timeout_s), done))
        return DM_ERR_TIMEOUT;
    if (J->state == DM_JOB_PREEMPTED) return DM_ERR_ARG;
    return J->state == DM_JOB_DONE ? DM_OK : DM_ERR_CUDA;
}

dm_status dm_server_preempt(dm_server* S, int64_t id, double timeout_s, double* V_out, dm_fit_state* st) {
    if (!S) return DM_ERR_ARG;
    SJob* J = nullptr;
    {
        std::unique_lock<std::mutex> lk(S->mu);
        auto it = S->jobs.find(id);
        if (it == S->jobs.end()) return DM_ERR_ARG;
        J = it->second;
        if (J->state == DM_JOB_DONE || J->state == DM_JOB_FAILED || J->state == DM_JOB_PREEMPTED) return DM_ERR_ARG;
        J->preempt_req = true;
        S->cv.notify_all();
        auto done = [&] {
            return J->state == DM_JOB_PREEMPTED || J->state == DM_JOB_DONE || J->state == DM_JOB_FAILED || S->stop;
        };
        if (timeout_s < 0)
            S->cv.wait(lk, done);
        else if (!S->cv.wait_for(lk, std::chrono::duration<double>(timeout_s), done))
            return DM_ERR_TIMEOUT;
        if (J->state != DM_JOB_PREEMPTED) return J->state == DM_JOB_DONE ? DM_ERR_ARG : DM_ERR_CUDA;
        S->jobs.erase(it);
    }
    const size_t nV = J->ck_V.size();
    if (V_out) memcpy(V_out, J->ck_V.data(), nV * sizeof(double));
    if (st) {
        st->step = J->ck_step;
        for (int a = 0; a < 3; ++a) {
            st->sigma[a] = J->ck_sigma[a];
            st->m_sigma[a] = J->ck_ms[a];
            st->v_sigma[a] = J->ck_vs[a];
        }
        if (st->m_V) memcpy(st->m_V, J->ck_mV.data(), nV * sizeof(double));
        if (st->v_V) memcpy(st->v_V, J->ck_vV.data(), nV * sizeof(double));
        if (st->warm && J->ck_warm.size() == 2 * nV) memcpy(st->warm, J->ck_warm.data(), 2 * nV * sizeof(double));
    }
    delete J;
    return DM_OK;
}

dm_status dm_server_result(dm_server* S, int64_t id, double* V_out, double* sigma_out, double* loss_history) {
    if (!S) return DM_ERR_ARG;
    SJob* J = nullptr;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        auto it = S->jobs.find(id);
        if (it == S->jobs.end()) return DM_ERR_ARG;
        J = it->second;
        if (J->state != DM_JOB_DONE) return J->state == DM_JOB_FAILED ? DM_ERR_CUDA : DM_ERR_ARG;
        S->jobs.erase(it);
    }
    if (V_out) memcpy(V_out, J->V_out.data(), J->V_out.size() * sizeof(double));
    if (sigma_out) memcpy(sigma_out, J->sigma_out, 3 * sizeof(double));
    if (loss_history) memcpy(loss_history, J->hist_out.data(), J->hist_out.size() * sizeof(double));
    delete J;
    return DM_OK;
}

dm_status dm_server_get_stats(dm_server* S, dm_server_stats* out) {
    if (!S || !out) return DM_ERR_ARG;
    std::lock_guard<std::mutex> lk(S->mu);
    *out = S->stats;
    return DM_OK;
}

double dm_server_clock(const dm_server* S) { return S ? S->now() : 0.0; }

dm_status dm_server_shutdown(dm_server* S) {
    if (!S) return DM_OK;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
    }
    S->cv.notify_all();
    if (S->engine.joinable()) S->engine.join();
    DeviceGuard dg(S->device);
    cudaStreamSynchronize(S->st);
    if (S->gexec) cudaGraphExecDestroy(S->gexec);
    for (auto& kv : S->jobs) delete kv.second;  // queued, finished and unclaimed jobs
    S->arena.release();
    cudaFree(S->d_fj);
    cudaFree(S->d_aj);
    cudaFree(S->d_uf);
    cudaFree(S->d_ua);
    cudaFree(S->d_counter);
    cudaFree(S->d_losses);
    cudaFree(S->d_sj);
    cudaFree(S->d_offs);
    cudaFree(S->d_fftj);
    cudaFree(S->d_fft_offs);
    cudaFreeHost(S->h_loss);
    for (auto& p : S->free_streams) {
        cudaStreamDestroy(p.first);
        cudaEventDestroy(p.second);
    }
    if (S->ev_fwd) cudaEventDestroy(S->ev_fwd);
    if (S->ev_adj) cudaEventDestroy(S->ev_adj);
    cudaStreamDestroy(S->st);
    dm_destroy(S->ctx);
    delete S;
    return DM_OK;
}

}  // extern "C"
