#!/usr/bin/env python
"""Throughput of one shape-fit step of the mesh-Fourier renderer on one B300.

A step is one pass of the whole hot path on the largest single-fit workload
(icosphere level 5 = 20480 triangles, SH l <= 10 deformation, 256x256x128 grid of
(0.5, 0.5, 1) um voxels, Gaussian PSF sigma = (0.25, 0.25, 0.7) um, the whole
half spectrum of 4,259,840 frequencies): triangle records, mesh transform over
every (frequency, triangle) pair, transfer-function multiply, inverse 3D DFT, MSE
loss and residual, forward 3D DFT of the residual, dL/dsigma, the adjoint mesh
transform, per-vertex assembly, and the Adam update of the vertices.
`--workload c2` runs the 128^3 single cell (5120 triangles, narrow band h_hat > 1e-3).

Metric: forward + backward (triangle x frequency) terms per second,
2 * M * n_t / step time. Prints one JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""

from __future__ import annotations

import argparse
import ctypes
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "fwd+bwd tri*freq terms/s; served fits/s & p99 vs plain FP64 path at <=1e-4 err"
UNIT = "terms/s"
# Algorithmic work per (frequency, triangle) term on the FP32 pipe (lane operations) and on
# the MUFU (sin/cos/rcp) pipe: evaluating Eq. 8 once (forward) and Eq. 8 + Eq. 10 with the
# contraction into the per-triangle sums (adjoint). These are the method's counts (3 sincos and one
# common-denominator reciprocal per term), not the kernels' instruction counts: the forward kernel
# issues exactly these 7 MUFU operations per term, the adjoint 9 (it forms E and q of both gaps).
OPS_PER_TERM = {"fwd": 45, "adj": 110}
MUFU_PER_TERM = {"fwd": 7, "adj": 7}


# DRAM traffic per launch of the dominant kernels (dram__bytes_read.sum + dram__bytes_write.sum from one
# ncu capture of `python bench.py --workload W --steps 1 --warmup 3 --no-cpu-baseline --no-e2e --no-serve
# --no-fp64`, one kernel, one launch), keyed by workload and kernel, with the SHA-256 of the mesh-transform
# sources it was taken on (comments excluded, kernel_sources_digest): a capture of other code is not
# reported (the traffic is then null).
MEASURED_TRAFFIC = {
    ("c3", "k_adj_f32"): {"bytes": 146.96e6 + 72.33e6, "sources": "74bf4f20cf7c95ca"},
    ("c3", "k_fwd_f32"): {"bytes": 2.70e6 + 9.43e6, "sources": "74bf4f20cf7c95ca"},
}
TRAFFIC_SOURCES = ("meshft_f32.cu", "meshft_math.cuh", "dm_kernels.cuh", "dm_common.cuh")


def kernel_sources_digest() -> str:
    """SHA-256 (first 16 hex digits) of the mesh-transform sources with their comments and blank lines
    removed, so that an edit of a comment keeps a capture valid and any edit of the code does not."""
    import hashlib
    import re

    h = hashlib.sha256()
    for name in TRAFFIC_SOURCES:
        with open(os.path.join(ROOT, "paper_2303_10440_b300", "csrc", name), encoding="utf-8") as f:
            text = f.read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        code = "\n".join(line.rstrip() for line in text.splitlines() if line.strip())
        h.update(code.encode())
    return h.hexdigest()[:16]


def measured_traffic(workload: str, kernel: str) -> dict:
    m = MEASURED_TRAFFIC.get((workload, kernel))
    digest = kernel_sources_digest()
    if not m or m["sources"] != digest:
        return {"traffic": None, "traffic_note": f"no ncu capture of these kernel sources ({digest}) on this workload"}
    return {"traffic": m["bytes"], "traffic_unit": "DRAM bytes per launch (ncu dram__bytes_read.sum + "
            "dram__bytes_write.sum)", "traffic_sources": digest}


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--workload", choices=["c3", "c2", "c1", "c2s", "c3s"], default="c3",
                   help="c3: 256x256x128, 20480 triangles (default); c2: 128^3 single cell, 5120 triangles; "
                   "c1: 32^3 icosphere; c2s: the c2 cell on a 64^3 grid of doubled voxels and c3s: the c3 cell on "
                   "128x128x64 doubled voxels (small profiling cases)")
    p.add_argument("--precision", choices=["fp32", "fp64"], default="fp32",
                   help="fp32: the FP32 mixed path (headline); fp64: the plain FP64 path (comparator)")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-serve", action="store_true", help="skip the serving leg")
    p.add_argument("--no-fp64", action="store_true", help="skip the plain FP64 path's step beside the FP32 one")
    p.add_argument("--mode", choices=["step", "serve-c4", "serve-c5", "serve-batch", "serve-budget", "stagger", "robust",
                                      "fft", "scaling", "mufu"],
                   default="step",
                   help="step: the headline fit-step benchmark; serve-c4: 32-cell tissue through the fit server; "
                   "serve-c5: Poisson stream of serving requests; stagger: the staggered shape/PSF fit "
                   "(large-steps shape steps on the narrow band, PSF steps on the whole spectrum); robust: "
                   "sweeps of initial scale, initial shift and image noise through the fit server; fft: the inverse "
                   "and forward real 3D transforms alone, GB/s against the measured HBM copy bandwidth; scaling: "
                   "step time against grid size and triangle count (the paper's GPU timing figure) and a "
                   "narrow-band case")
    p.add_argument("--rounds", type=int, default=4, help="staggered rounds in the stagger mode")
    p.add_argument("--fit-steps", type=int, default=0, help="Adam steps per job in the serve modes (0: 20 / 100)")
    p.add_argument("--jobs", type=int, default=12, help="requests in serve-c5")
    p.add_argument("--graphs", type=int, default=1, help="serve-batch: replay iterations as CUDA graphs (0: direct)")
    p.add_argument("--capacity-fits-per-s", type=float, default=0.0,
                   help="serve-c5: the saturated throughput the capacity fractions refer to (0: the best served "
                   "throughput measured at --rates in the same run)")
    p.add_argument("--legs", default="fifo,shortest,sequential",
                   help="serve modes: which legs to run (fifo, shortest, sequential one-at-a-time FP32)")
    p.add_argument("--lr-decay", type=float, default=0.998, help="per-step learning-rate factor in the robust mode")
    p.add_argument("--clip-target", type=int, default=1, help="robust mode: clip noisy targets at zero")
    p.add_argument("--rates", default="10,20,50,100,200,500", help="Poisson arrival rates (1/s) in serve-c5")
    p.add_argument("--capacity-fracs", default="0.25,0.5,1",
                   help="serve-c5 arrival rates as fractions of the measured saturated throughput ('' for none)")
    return p.parse_args()


def make_case(name):
    import synth

    if name == "c2":
        return synth.config_c2()
    if name == "c3":
        return synth.config_c3()
    if name == "c2s":
        c = synth.config_c2()
        c.grid = synth.Grid(n=(64, 64, 64), h=(1.0, 1.0, 2.0))
        c.name = "c2s_cell_sh6_64cube_profile"
        return c
    if name == "c3s":
        c = synth.config_c3()
        c.grid = synth.Grid(n=(128, 128, 64), h=(1.0, 1.0, 2.0))
        c.name = "c3s_cell_sh10_128x128x64_profile"
        return c
    return synth.config_c1()


def whole_job_value(t_ms_local: float, terms_per_rank: float, world: int, device=None):
    """Max of the ranks' timed-region durations (ms) and the whole-job rate: every rank processes
    terms_per_rank terms in the timed region (weak scaling: independent fits, no data exchange)."""
    import torch

    t = torch.tensor([t_ms_local], dtype=torch.float64, device=device)
    if world > 1:
        import torch.distributed as dist

        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    t_max = float(t.item())
    return world * terms_per_rank / (t_max / 1e3), t_max


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = (
        "index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
        "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
        "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap"
    )

    def __init__(self, uuid: str | None):
        self.uuid = uuid
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200"]
        if self.uuid:
            cmd.insert(1, f"--id={self.uuid}")
        try:
            self.proc = subprocess.Popen(cmd, stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({n for r in rows for n, v in zip(names, r[5:9]) if v.lower().startswith("active")})
        return {
            "sm_mhz": float(np.median(sm)) if sm else None,
            "sm_max_mhz": max(mx) if mx else None,
            "reasons": reasons,
            "samples": len(rows),
        }


# ----------------------------------------------------------------------------- CPU oracle legs
def oracle_sample(case, n_freq: int, seed: int = 0):
    """A seeded random subset of the band (all triangles kept) for timing the CPU oracle."""
    import oracle

    nvec, _ = oracle.half_spectrum(case.grid.n)
    xi_all = oracle.wavevectors(nvec, case.grid)
    band = oracle.band_mask(oracle.otf(xi_all, case.psf), case.psf.band_tau)
    idx = np.nonzero(band)[0]
    rng = np.random.default_rng(seed)
    sel = np.sort(rng.choice(idx, size=min(n_freq, len(idx)), replace=False))
    G = (rng.normal(size=len(sel)) + 1j * rng.normal(size=len(sel))) / len(sel)
    return xi_all[sel], G, int(band.sum())


def time_oracle_step(case, xi, G):
    import oracle

    Vs = case.V_init - np.asarray(case.grid.origin)
    t0 = time.perf_counter()
    oracle.mesh_ft(Vs, case.F, xi)
    oracle.mesh_ft_adjoint(Vs, case.F, xi, G)
    return time.perf_counter() - t0


def cpu_sample_freqs(case, terms=1.6e8):
    """Band frequencies of the CPU oracle's sample: about `terms` forward terms (x all triangles), which
    the FP64 oracle evaluates forward and adjoint in roughly 10-20 s on 16 host cores."""
    return max(512, int(terms / case.F.shape[0]))


def cpu_baseline(case, n_freq=None):
    import oracle

    xi, G, _ = oracle_sample(case, n_freq or cpu_sample_freqs(case))
    dt = time_oracle_step(case, xi, G)
    terms = 2.0 * len(xi) * case.F.shape[0]
    return {
        "value": terms / dt,
        "unit": UNIT,
        "cores": oracle.num_threads(),
        "kind": "oracle",
        "sample": f"FP64 oracle forward + adjoint on {len(xi)} seeded random band frequencies x all "
        f"{case.F.shape[0]} triangles ({dt:.1f} s, OpenMP over frequencies/triangles)",
    }


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import oracle

    case = make_case(args.workload)
    n_freq = max(96, int(8e6 / case.F.shape[0]))  # ~0.7 s of oracle work per step
    xi, G, M = oracle_sample(case, n_freq)
    for _ in range(args.warmup):
        time_oracle_step(case, xi, G)
    total = 0.0
    for _ in range(args.steps):
        total += time_oracle_step(case, xi, G)
    terms = 2.0 * len(xi) * case.F.shape[0] * args.steps
    value = terms / total
    out = {
        "impl": "reference",
        "metric": METRIC,
        "value": value,
        "unit": UNIT,
        "n_gpus": args.gpus,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64",
        "data": "synthetic",
        "config": workload_config(case, M),
        "cpu_baseline": {
            "value": value,
            "unit": UNIT,
            "cores": oracle.num_threads(),
            "kind": "oracle",
            "sample": f"each step: FP64 oracle forward + adjoint on {len(xi)} seeded random band frequencies x "
            f"all {case.F.shape[0]} triangles",
        },
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out), flush=True)


L2_NOTE = "flushed (256 MB write) between timed steps, outside the events"


def workload_config(case, M, l2=L2_NOTE):
    """The workload's description; identical in both arms of the benchmark."""
    return {
        "workload": case.name,
        "grid": list(case.grid.n),
        "voxel_um": list(case.grid.h),
        "n_triangles": int(case.F.shape[0]),
        "n_vertices": int(case.V_init.shape[0]),
        "band_size": int(M),
        "band_tau": case.psf.band_tau,
        "psf_sigma_um": list(case.psf.sigma),
        "loss": "mse",
        "optimizer": "adam(vertices)",
        "l2": l2,
    }


# ----------------------------------------------------------------------------- serving
def serving_jobs(r32, n_jobs, seed, levels, sides, steps):
    """Fit requests drawn like the serving workload (random icosphere level, grid side and
    anisotropic sigma; target = render of an SH-deformed cell), restricted to `levels`/`sides`."""
    import torch

    import synth

    rng = np.random.default_rng(seed)
    jobs = []
    for k in range(n_jobs):
        lev = int(rng.choice(levels))
        side = int(rng.choice(sides))
        grid = synth.Grid(n=(side, side, side), h=(0.5, 0.5, 1.0))
        sxy, sz = float(rng.uniform(0.15, 0.3)), float(rng.uniform(0.4, 0.9))
        R = 0.3 * float(min(grid.L))
        V_t, F = synth.sh_deformed_sphere(lev, R, grid.center, lmax=6, coef_sigma=0.03 * R, seed=10_000 + k)
        V0, _ = synth.sphere_mesh(lev, R, grid.center)
        psf = synth.Psf(sigma=(sxy, sxy, sz), band_tau=1e-3)
        T = r32.render(torch.as_tensor(V_t).cuda(), torch.as_tensor(F).cuda(), grid, psf).cpu().numpy()
        jobs.append(dict(V=V0, F=F, target=T, grid=grid, psf=psf, steps=steps, lr_vertex=1e-2 * min(grid.h)))
    return jobs


def _queue_latencies(arrivals, durations):
    """One job at a time in arrival order, from measured durations: completion = max(arrival, previous
    completion) + duration (used only where running the leg would take too long, and labelled so)."""
    t, lat = 0.0, []
    for a, d in zip(arrivals, durations):
        t = max(t, a) + d
        lat.append(t - a)
    return np.array(lat), t - arrivals[0]


def _one_at_a_time_run(r, jobs, arrivals, dev):
    """The one-fit-at-a-time path, run open loop: requests arrive at `arrivals` (seconds) into a FIFO
    queue that one worker drains, each job through dm_fit alone (inputs copied from the host first, as
    the server copies them at admission). Returns (latencies, span) as observed on the wall clock."""
    import queue
    import threading

    import torch

    q = queue.Queue()
    done = [0.0] * len(jobs)

    def worker():
        while True:
            k = q.get()
            if k is None:
                return
            j = jobs[k]
            Vd, Fd = torch.as_tensor(j["V"]).to(dev), torch.as_tensor(j["F"]).to(dev)
            Td = torch.as_tensor(j["target"]).to(dev)
            r.fit(Vd, Fd, j["grid"], j["psf"], Td, steps=j["steps"], lr_vertex=j["lr_vertex"])
            torch.cuda.synchronize(dev)
            done[k] = time.perf_counter()

    torch.cuda.synchronize(dev)
    th = threading.Thread(target=worker)
    th.start()
    t0 = time.perf_counter()
    for k, a in enumerate(arrivals):
        delay = t0 + a - time.perf_counter()
        if delay > 0:
            time.sleep(delay)
        q.put(k)
    q.put(None)
    th.join()
    lat = np.array([done[k] - (t0 + arrivals[k]) for k in range(len(jobs))])
    return lat, max(done) - t0


def _stats(lat, span, n):
    return {"fits_per_s": n / span, "p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
            "span_s": span}


def _served_run(jobs, arrivals, dev, keep=False, **server_kw):
    import threading

    from paper_2303_10440_b300.serve import FitServer

    srv = FitServer(device=dev.index or 0, max_jobs=32, **server_kw)
    ids = [None] * len(jobs)
    t0 = srv.clock()

    def feeder():
        for k, j in enumerate(jobs):
            delay = t0 + arrivals[k] - srv.clock()
            if delay > 0:
                time.sleep(delay)
            ids[k] = srv.submit(**j)

    th = threading.Thread(target=feeder)
    th.start()
    th.join()
    res = []
    for i in ids:
        srv.wait(i, timeout=7200)
        res.append(srv.result(i))
    st = srv.stats()
    srv.shutdown()
    lat = np.array([r.latency for r in res])
    span = max(r.t_end for r in res) - min(r.t_submit for r in res)
    out = dict(_stats(lat, span, len(jobs)), peak_batch=int(st["peak_active"]), iterations=int(st["iterations"]))
    if keep:
        out["results"] = res
    return out


def serving_leg(args, dev, n_jobs=16, rates=(10.0, 50.0, 100.0, 500.0), steps=10, levels=(2, 3), sides=(32, 48, 64),
                with_fp64=True):
    """Served fits/s and p50/p99 latency vs one-job-at-a-time FP32 and plain FP64 at each arrival rate.

    Every leg runs open loop on the wall clock: the served legs through the fit server, the one-at-a-time
    FP32 leg through a worker that runs dm_fit on one job at a time. The plain FP64 leg (about 100x slower)
    runs once, at the highest rate, where every request is queued at once."""
    from paper_2303_10440_b300 import Renderer

    r32 = Renderer("fp32", device=dev.index or 0)
    jobs = serving_jobs(r32, n_jobs, 5, levels, sides, steps)
    _one_at_a_time_run(r32, jobs[:2], [0.0, 0.0], dev)  # warm-up (modules, FFT tables)
    out = {
        "workload": f"{n_jobs} fit requests, icosphere levels {list(levels)}, cubic grids {list(sides)} of "
        f"(0.5, 0.5, 1) um, sigma_xy~U(0.15,0.3) um, sigma_z~U(0.4,0.9) um, {steps} Adam steps each, "
        f"open-loop Poisson arrivals",
        "one_at_a_time_note": "sequential_fp32 / plain_fp64: each job alone through dm_fit (FP32 / FP64 context) "
        "by one worker draining an open-loop FIFO queue, latencies observed on the wall clock",
        "rates": {},
    }
    for rate in rates:
        rng = np.random.default_rng(6)
        arrivals = np.cumsum(rng.exponential(1.0 / rate, size=n_jobs))
        arrivals -= arrivals[0]
        # shortest-first within ~1 ms of mesh-transform work per iteration (3e8 terms): the small jobs finish
        # first under load (a budget of 3e9 takes every job of this mix each iteration, like FIFO)
        entry = {"served_fp32": _served_run(jobs, arrivals, dev),
                 "served_fp32_shortest_first": _served_run(jobs, arrivals, dev, policy="shortest", batch_terms=3e8)}
        lat, span = _one_at_a_time_run(r32, jobs, arrivals, dev)
        entry["sequential_fp32"] = _stats(lat, span, n_jobs)
        if with_fp64 and rate == max(rates):
            r64 = Renderer("fp64", device=dev.index or 0)
            lat, span = _one_at_a_time_run(r64, jobs, arrivals, dev)
            entry["plain_fp64"] = _stats(lat, span, n_jobs)
            r64.close()
        out["rates"][f"{rate:g}/s"] = entry
    if with_fp64:
        import torch

        r64 = Renderer("fp64", device=dev.index or 0)
        errs = []
        for j in jobs:
            Vd, Fd = torch.as_tensor(j["V"]).to(dev), torch.as_tensor(j["F"]).to(dev)
            a = r32.render(Vd, Fd, j["grid"], j["psf"]).double()
            b = r64.render(Vd, Fd, j["grid"], j["psf"])
            errs.append(float(torch.linalg.norm(a - b) / torch.linalg.norm(b)))
        out["max_render_rel_err_fp32_vs_fp64"] = max(errs)
        r64.close()
    r32.close()
    return out


# ----------------------------------------------------------------------------- our arm
def run_ours(args):
    import torch

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_2303_10440_b300 import Renderer

    case = make_case(args.workload)
    grid, psf = case.grid, case.psf
    r = Renderer(args.precision, device=local)
    M = len(r.band(grid, psf))
    n_t = case.F.shape[0]
    terms_step = 2.0 * M * n_t

    Fd = torch.as_tensor(case.F).to(dev)
    T = r.render(torch.as_tensor(case.V_true).to(dev), Fd, grid, psf)  # target: the deformed cell
    Vd = torch.as_tensor(case.V_init).to(dev).clone()
    dVd = torch.empty_like(Vd)
    Ld = torch.empty(1, dtype=torch.float64, device=dev)
    dpsfd = torch.empty(3, dtype=torch.float64, device=dev)
    mom = torch.zeros_like(Vd)
    vel = torch.zeros_like(Vd)
    lr = 1e-2 * min(grid.h)
    stream = torch.cuda.current_stream(dev)
    step_no = [0]

    def step():
        r.loss_and_grad(Vd, Fd, grid, psf, T, "mse", L_out=Ld, dV_out=dVd, dpsf_out=dpsfd, stream=stream)
        step_no[0] += 1
        r.adam(Vd, dVd, mom, vel, step_no[0], lr, stream=stream)

    for _ in range(max(args.warmup, 0)):
        step()
    torch.cuda.synchronize(dev)

    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # 256 MB > 126 MB L2
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    uuid = None
    try:
        uuid = "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        pass
    clocks = ClockSampler(uuid)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize(dev)
    clocks.start()
    time.sleep(0.3)
    r.profile(True)
    r.profile_read()
    launches0 = r.kernel_launches()
    for k in range(args.steps):
        flush.fill_(float(k))  # evict L2 between timed steps (outside the events)
        ev[k][0].record(stream)
        step()
        ev[k][1].record(stream)
    torch.cuda.synchronize(dev)
    launches = r.kernel_launches() - launches0
    stages = r.profile_read()
    r.profile(False)
    if world > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    t_ms = sum(a.elapsed_time(b) for a, b in ev)
    value, t_max = whole_job_value(t_ms, terms_step * args.steps, world, dev)


    # roofline of the dominant kernel (event-timed inside the library on this stream)
    dom = max(("fwd", "adj"), key=lambda s: stages[s][0])
    kern = {"fwd": "k_fwd_f32", "adj": "k_adj_f32"} if args.precision == "fp32" else {"fwd": "k_fwd_f64", "adj": "k_adj_f64"}
    dom_ms = stages[dom][0] / max(stages[dom][1], 1)
    terms_launch = M * n_t
    f_mhz = clk.get("sm_mhz") or 1920.0
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    peak = 128.0 * sms * f_mhz * 1e6 / 1e12  # FP32-pipe lane operations per second (Tops/s)
    achieved = terms_launch * OPS_PER_TERM[dom] / (dom_ms / 1e3) / 1e12
    roofline = {
        "bound": "alu",
        "kernel": kern[dom],
        "achieved": achieved,
        "peak": peak,
        "unit": "Tops/s",
        "frac": achieved / peak,
        **measured_traffic(args.workload, kern[dom]),
        "ops_per_term": OPS_PER_TERM[dom],
        "mufu_per_term": MUFU_PER_TERM[dom],
        "terms_per_launch": terms_launch,
        "launch_ms": dom_ms,
        "peak_basis": f"128 FP32 lanes x {sms} SMs x median SM clock {f_mhz:.0f} MHz under load",
        "fwd_terms_per_s": terms_launch / (stages["fwd"][0] / max(stages["fwd"][1], 1) / 1e3),
        "adj_terms_per_s": terms_launch / (stages["adj"][0] / max(stages["adj"][1], 1) / 1e3),
        "stage_ms_per_step": {k: v[0] / max(args.steps, 1) for k, v in stages.items() if v[1]},
    }

    out = {
        "metric": METRIC,
        "value": value,
        "unit": UNIT,
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": t_max / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32" if args.precision == "fp32" else "f64",
        "data": "synthetic",
        "config": workload_config(case, M),
        "roofline": roofline,
        "clocks": clk,
        "gpu_launches": int(launches),
    }

    if not args.no_e2e:
        out["e2e"] = e2e_through_host_buffers(r, case, grid, psf, T, terms_step, args, dev, world)
    if not args.no_serve:
        out["serving"] = serving_leg(args, dev)
    if rank == 0 and args.precision == "fp32" and not args.no_fp64:
        out["fp64_plain"] = fp64_plain_step(case, grid, psf, T, terms_step, dev)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(case)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def fp64_plain_step(case, grid, psf, T_dev, terms_step, dev, full_limit=2e10):
    """The plain FP64 path beside the FP32 one. Up to `full_limit` terms per step: the same fit step
    (dm_loss_and_grad on device buffers) in an FP64 context, one warm-up and one CUDA-event-timed step.
    Larger workloads (one FP64 step of the 256x256x128 cell takes over a minute): the two FP64 mesh-transform
    sums (dm_meshft, dm_meshft_adjoint) over a seeded random 1/16 of the band x all triangles, whose cost is
    linear in the terms; the stage kernels are < 2% of a step."""
    import torch

    from paper_2303_10440_b300 import Renderer

    r64 = Renderer("fp64", device=dev.index or 0)
    Vd = torch.as_tensor(case.V_init).to(dev)
    Fd = torch.as_tensor(case.F).to(dev)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if terms_step <= full_limit:
        T64 = T_dev.double()
        r64.loss_and_grad(Vd, Fd, grid, psf, T64, "mse")
        torch.cuda.synchronize(dev)
        a.record()
        r64.loss_and_grad(Vd, Fd, grid, psf, T64, "mse")
        b.record()
        torch.cuda.synchronize(dev)
        ms = a.elapsed_time(b)
        r64.close()
        return {"value": terms_step / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms, "steps": 1,
                "note": "same workload and step through the FP64 context (plain path); FP64 rate-bound on B300"}
    band = r64.band(grid, psf).cpu().numpy()
    rng = np.random.default_rng(11)
    sel = np.sort(rng.choice(len(band), size=len(band) // 16, replace=False))
    nzh = grid.n[2] // 2 + 1
    idx = band[sel].astype(np.int64)
    iz, t = idx % nzh, idx // nzh
    iy, ix = t % grid.n[1], t // grid.n[1]
    nx = np.where(ix < (grid.n[0] + 1) // 2, ix, ix - grid.n[0])
    ny = np.where(iy < (grid.n[1] + 1) // 2, iy, iy - grid.n[1])
    fn = torch.as_tensor(np.stack([nx, ny, iz], axis=1).astype(np.int32)).to(dev)
    G = torch.randn(len(sel), dtype=torch.complex128, device=dev) / len(sel)
    r64.meshft(Vd, Fd, grid, fn[:4096])
    r64.meshft_adjoint(Vd, Fd, grid, fn[:4096], G[:4096])
    torch.cuda.synchronize(dev)
    a.record()
    r64.meshft(Vd, Fd, grid, fn)
    r64.meshft_adjoint(Vd, Fd, grid, fn, G)
    b.record()
    torch.cuda.synchronize(dev)
    ms = a.elapsed_time(b)
    r64.close()
    terms = 2.0 * len(sel) * case.F.shape[0]
    return {"value": terms / (ms * 1e-3), "unit": UNIT, "ms_sample": ms, "ms_per_step_extrapolated":
            ms * terms_step / terms, "steps": 1,
            "note": f"FP64 context: dm_meshft + dm_meshft_adjoint on a seeded random 1/16 of the band "
            f"({len(sel)} frequencies) x all {case.F.shape[0]} triangles, CUDA-event timed; the per-step time is "
            f"extrapolated linearly in terms (FP64 rate-bound on B300)"}


def e2e_through_host_buffers(r, case, grid, psf, T_dev, terms_step, args, dev, world):
    """Same metric through dm_loss_and_grad with pinned HOST buffers: every step copies the mesh
    and the target image to the device and the loss, dL/dV and dL/dsigma back."""
    import torch

    Vh = torch.as_tensor(case.V_init).pin_memory()
    Fh = torch.as_tensor(case.F).pin_memory()
    Th = T_dev.cpu().pin_memory()
    Lh = torch.empty(1, dtype=torch.float64).pin_memory()
    dVh = torch.empty_like(Vh).pin_memory()
    dph = torch.empty(3, dtype=torch.float64).pin_memory()
    for _ in range(max(args.warmup, 1)):
        r.loss_and_grad(Vh, Fh, grid, psf, Th, "mse", L_out=Lh, dV_out=dVh, dpsf_out=dph)
    torch.cuda.synchronize(dev)
    if world > 1:
        torch.distributed.barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        r.loss_and_grad(Vh, Fh, grid, psf, Th, "mse", L_out=Lh, dV_out=dVh, dpsf_out=dph)
    torch.cuda.synchronize(dev)
    dt = time.perf_counter() - t0
    t = torch.tensor([dt], dtype=torch.float64, device=dev)
    if world > 1:
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    h2d = Vh.numel() * 8 + Fh.numel() * 4 + Th.numel() * 4
    d2h = 8 + dVh.numel() * 8 + 3 * 8
    return {
        "value": world * terms_step * args.steps / float(t.item()),
        "unit": UNIT,
        "h2d_bytes_per_step": int(h2d),
        "d2h_bytes_per_step": int(d2h),
        "call": "dm_loss_and_grad (host V, F, target; host L, dV, dpsf)",
    }


def _job_terms(j):
    n = j["grid"].n
    return 2.0 * n[0] * n[1] * (n[2] // 2 + 1) * j["F"].shape[0] * j["steps"]


def _poisson_arrivals(rate, n, seed=7):
    """Open-loop arrival times: exponential gaps at `rate` per second, the first request at t = 0."""
    a = np.cumsum(np.random.default_rng(seed).exponential(1.0 / rate, size=n))
    return a - a[0]


def _fp64_alone(jobs, dev, k_small=2):
    """The plain FP64 path on the k_small cheapest jobs, each run alone through dm_fit (FP64 context):
    measured durations, and the FP64 terms/s they imply (used for the other jobs, labelled)."""
    import torch

    from paper_2303_10440_b300 import Renderer

    r64 = Renderer("fp64", device=dev.index or 0)
    order = sorted(range(len(jobs)), key=lambda k: _job_terms(jobs[k]))[:k_small]
    durs = {}
    for k in order:
        j = jobs[k]
        torch.cuda.synchronize(dev)
        t = time.perf_counter()
        Vd, Fd = torch.as_tensor(j["V"]).to(dev), torch.as_tensor(j["F"]).to(dev)
        Td = torch.as_tensor(j["target"]).to(dev)
        r64.fit(Vd, Fd, j["grid"], j["psf"], Td, steps=j["steps"], lr_vertex=j["lr_vertex"])
        torch.cuda.synchronize(dev)
        durs[k] = time.perf_counter() - t
    r64.close()
    rate = sum(_job_terms(jobs[k]) for k in order) / sum(durs.values())
    return durs, rate


def _sampled_spectrum_errors(jobs, results, dev, n_freq=256):
    """Per job: the fitted mesh's spectrum on seeded random band frequencies, FP32 path against the FP64
    path (relative L2, and weighted by the transfer function, i.e. the image's Fourier coefficients)."""
    import torch

    from paper_2303_10440_b300 import Renderer

    r32, r64 = Renderer("fp32", device=dev.index or 0), Renderer("fp64", device=dev.index or 0)
    errs = []
    for k, (j, res) in enumerate(zip(jobs, results)):
        g = j["grid"]
        band = r32.band(g, j["psf"]).numpy().astype(np.int64)
        sel = band[np.sort(np.random.default_rng(100 + k).choice(len(band), size=min(n_freq, len(band)),
                                                                     replace=False))]
        nzh = g.n[2] // 2 + 1
        iz, t = sel % nzh, sel // nzh
        iy, ix = t % g.n[1], t // g.n[1]
        fn = np.stack([np.where(ix < (g.n[0] + 1) // 2, ix, ix - g.n[0]),
                       np.where(iy < (g.n[1] + 1) // 2, iy, iy - g.n[1]), iz], axis=1).astype(np.int32)
        Vd, Fd, fd = (torch.as_tensor(x).to(dev) for x in (res.V, j["F"], fn))
        a = r32.meshft(Vd, Fd, g, fd).cpu().numpy().astype(np.complex128)
        b = r64.meshft(Vd, Fd, g, fd).cpu().numpy()
        xi = 2 * np.pi * fn / np.asarray(g.L)
        hh = np.exp(-0.5 * (xi ** 2 * np.asarray(j["psf"].sigma) ** 2).sum(1))
        errs.append({"job": k, "spectrum": float(np.linalg.norm(a - b) / np.linalg.norm(b)),
                     "image_coefficients": float(np.linalg.norm((a - b) * hh) / np.linalg.norm(b * hh))})
    r32.close()
    r64.close()
    return errs


def run_serve_mode(args):
    import torch

    import synth
    from paper_2303_10440_b300 import Renderer

    dev = torch.device("cuda", 0)
    r32 = Renderer("fp32")
    if args.mode == "serve-c4":
        steps = args.fit_steps or 20
        _, cells = synth.config_c4_cells()
        jobs = []
        for k, c in enumerate(cells):
            T = r32.render(torch.as_tensor(c["V_true"]).to(dev), torch.as_tensor(c["F"]).to(dev), c["grid"],
                           c["psf"]).cpu().numpy()
            noisy, scale = synth.add_poisson_gaussian_noise(T, 200.0, 2.0, seed=500 + k)
            jobs.append(dict(V=c["V_init"], F=c["F"], target=noisy / scale, grid=c["grid"], psf=c["psf"], steps=steps,
                             lr_vertex=1e-2 * min(c["grid"].h)))
        workload = (f"32 SH-deformed cells packed in a 256^3 tissue (levels 3-5, radii 8-20 um), one fit per cell "
                    f"on its 64^3-128^3 crop, Poisson(peak 200) + N(0, 2^2) noise, {steps} Adam steps, all jobs "
                    f"submitted together (one persistent batched launch per iteration)")
        rates = {"batch": np.zeros(len(jobs))}
    else:
        steps = args.fit_steps or 100
        rng = np.random.default_rng(55)
        jobs = []
        for k in range(args.jobs):
            c = synth.config_c5_job(rng, k)
            T = r32.render(torch.as_tensor(c["V_true"]).to(dev), torch.as_tensor(c["F"]).to(dev), c["grid"],
                           c["psf"]).cpu().numpy()
            jobs.append(dict(V=c["V_init"], F=c["F"], target=T, grid=c["grid"], psf=c["psf"], steps=steps,
                             lr_vertex=1e-2 * min(c["grid"].h)))
        workload = (f"the first {len(jobs)} requests of the seeded serving stream (levels 2-6 = 320-81920 triangles, "
                    f"cubic grids 64-256 of (0.5, 0.5, 1) um, random anisotropic sigma), {steps} Adam steps each, "
                    f"open-loop Poisson arrivals")
        rates = {f"{rate:g}/s": _poisson_arrivals(rate, len(jobs)) for rate in
                 (float(x) for x in args.rates.split(",") if x)}
    legs_wanted = set(args.legs.split(","))
    total_terms = sum(_job_terms(j) for j in jobs)
    smallest = min(range(len(jobs)), key=lambda k: _job_terms(jobs[k]))
    _one_at_a_time_run(r32, [jobs[smallest]], [0.0], dev)  # warm-up (modules, FFT tables)
    fp64_durs, fp64_rate = _fp64_alone(jobs, dev)
    out = {"metric": "served fits/s and p50/p99 latency vs one-at-a-time FP32 and plain FP64", "mode": args.mode,
           "workload": workload, "n_jobs": len(jobs), "total_terms": total_terms,
           "job_terms": [_job_terms(j) for j in jobs], "results": {},
           "plain_fp64_measured": {"jobs": sorted(fp64_durs), "seconds": [fp64_durs[k] for k in sorted(fp64_durs)],
                                   "terms_per_s": fp64_rate},
           "one_at_a_time_note": "sequential_fp32: one worker drains an open-loop FIFO queue, each job alone "
                                 "through dm_fit, latencies observed; plain_fp64: the measured FP64 durations of the "
                                 "two cheapest jobs and, for the others, their terms at the FP64 terms/s those two "
                                 "measured, queued in arrival order (labelled: an FP64 run of the rest would take hours)"}
    fp64_durs_all = [fp64_durs.get(k, _job_terms(j) / fp64_rate) for k, j in enumerate(jobs)]
    first_served = None

    def legs(arr, rate=None):
        nonlocal first_served
        e = {}
        if "fifo" in legs_wanted:
            served = _served_run(jobs, arr, dev, keep=first_served is None)
            if first_served is None:
                first_served = served.pop("results")
            served["terms_per_s"] = total_terms / served["span_s"]
            e["served_fp32"] = served
        if "shortest" in legs_wanted:
            # least-remaining-work scheduling within a per-iteration term budget (about 10 ms of work)
            shortest = _served_run(jobs, arr, dev, policy="shortest", batch_terms=3e9)
            shortest["terms_per_s"] = total_terms / shortest["span_s"]
            e["served_fp32_shortest_first"] = shortest
        if "sequential" in legs_wanted:
            lat, span = _one_at_a_time_run(r32, jobs, arr, dev)
            e["sequential_fp32"] = dict(_stats(lat, span, len(jobs)), terms_per_s=total_terms / span)
        lat64, span64 = _queue_latencies(arr, fp64_durs_all)
        e["plain_fp64_from_measured"] = dict(_stats(lat64, span64, len(jobs)), terms_per_s=fp64_rate)
        if rate is not None:
            e["arrival_rate_per_s"] = rate
        return e

    def report(name, entry):
        # one line per finished arrival schedule, so that a run cut short keeps the legs it finished
        print(json.dumps({"partial": name, **entry}), flush=True)

    for name, arr in rates.items():
        out["results"][name] = legs(arr)
        report(name, out["results"][name])
    fracs = [float(x) for x in args.capacity_fracs.split(",") if x] if args.mode == "serve-c5" else []
    if fracs:
        # capacity = the best served throughput seen at the saturating rates above, or the one given
        cap = args.capacity_fits_per_s or max(
            max(e.get("served_fp32", {}).get("fits_per_s", 0.0),
                e.get("served_fp32_shortest_first", {}).get("fits_per_s", 0.0)) for e in out["results"].values())
        out["capacity_fits_per_s"] = cap
        for f in fracs:
            out["results"][f"{f:g}x capacity"] = legs(_poisson_arrivals(f * cap, len(jobs)), rate=f * cap)
            report(f"{f:g}x capacity", out["results"][f"{f:g}x capacity"])
    if first_served is not None:
        out["per_job_error_fp32_vs_fp64_sampled"] = _sampled_spectrum_errors(jobs, first_served, dev)
    print(json.dumps(out), flush=True)


def run_serve_batch_mode(args):
    """The serving leg's 16 small requests (levels 2-3, 32-64^3, 10 Adam steps) submitted together to the fit
    server; prints the server's statistics (engine time per iteration). With --graphs 0 every kernel launches
    directly, for a launch list."""
    import torch

    from paper_2303_10440_b300 import Renderer
    from paper_2303_10440_b300.serve import FitServer

    r32 = Renderer("fp32")
    jobs = serving_jobs(r32, 16, 5, (2, 3), (32, 48, 64), args.fit_steps or 10)
    torch.cuda.synchronize()
    srv = FitServer(device=0, max_jobs=32, graphs=bool(args.graphs))
    t0 = srv.clock()
    ids = [srv.submit(**j) for j in jobs]
    for i in ids:
        srv.wait(i, timeout=600)
    span = srv.clock() - t0
    st = srv.stats()
    srv.shutdown()
    print(json.dumps({"mode": "serve-batch", "jobs": len(jobs), "span_s": span,
                      **{k: st[k] for k in ("iterations", "busy_s", "job_steps", "peak_active", "graph_replays")}}),
          flush=True)


def run_serve_budget_mode(args):
    """The serving leg's 16 small requests at 500/s: served FIFO, served shortest-first at per-iteration term
    budgets of 1e8-3e9, and one at a time (every leg open loop, observed)."""
    import torch

    from paper_2303_10440_b300 import Renderer

    dev = torch.device("cuda", 0)
    r32 = Renderer("fp32")
    jobs = serving_jobs(r32, 16, 5, (2, 3), (32, 48, 64), args.fit_steps or 10)
    rng = np.random.default_rng(6)
    arr = np.cumsum(rng.exponential(1.0 / 500, size=16))
    arr -= arr[0]
    _served_run(jobs, arr, dev)  # warm-up
    out = {"mode": "serve-budget", "fifo": _served_run(jobs, arr, dev)}
    for bt in (1e8, 3e8, 1e9, 3e9):
        out[f"shortest_{bt:g}"] = _served_run(jobs, arr, dev, policy="shortest", batch_terms=bt)
    lat, span = _one_at_a_time_run(r32, jobs, arr, dev)
    out["sequential"] = _stats(lat, span, 16)
    print(json.dumps(out), flush=True)


def run_stagger_mode(args):
    """Times the staggered fit: per shape step (narrow band, large-steps update with its two smoothing
    solves) and per PSF step (whole half spectrum, no vertex adjoint), with the library's stage split."""
    import torch

    import synth
    from paper_2303_10440_b300 import PSF, Renderer

    dev = torch.device("cuda", 0)
    case = make_case(args.workload)
    r = Renderer("fp32" if args.precision == "fp32" else "fp64")
    Fd = torch.as_tensor(case.F).to(dev)
    sig = case.psf.sigma
    true_cov = (sig[0] ** 2, sig[1] ** 2, sig[2] ** 2, 0.15 * sig[0] * sig[1], 0.1 * sig[0] * sig[2],
                -0.1 * sig[1] * sig[2])
    T = r.render(torch.as_tensor(case.V_true).to(dev), Fd, case.grid, PSF(cov=true_cov))
    tau = case.psf.band_tau if case.psf.band_tau > 0 else 1e-2
    psf0 = PSF(sigma=tuple(1.15 * s for s in sig), band_tau=tau)
    S, P = 5, 5
    kw = dict(lr_vertex=0.5, lr_psf=0.01 * min(sig))
    r.fit_staggered(torch.as_tensor(case.V_init).to(dev), Fd, case.grid, psf0, T, rounds=1, shape_steps=1, psf_steps=1,
                    **kw)
    band = int(r.band(case.grid, psf0).numel())
    nH = case.grid.n[0] * case.grid.n[1] * (case.grid.n[2] // 2 + 1)

    def timed(shape_steps, psf_steps, prof=False):
        r.profile(prof)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        out = r.fit_staggered(torch.as_tensor(case.V_init).to(dev), Fd, case.grid, psf0, T, rounds=args.rounds,
                              shape_steps=shape_steps, psf_steps=psf_steps, **kw)
        b.record()
        torch.cuda.synchronize()
        st = r.profile_read() if prof else None
        r.profile(False)
        return a.elapsed_time(b), out, st

    t_shape, _, _ = timed(S, 0)
    t_psf, _, _ = timed(0, P)
    t_all, (V, psf, hs, hp, cg), stages = timed(S, P, prof=True)
    n_t = len(case.F)
    out = {
        "metric": "staggered fit: ms per shape step and per PSF step",
        "mode": "stagger",
        "precision": args.precision,
        "workload": f"{case.name}: {n_t} triangles, grid {tuple(case.grid.n)}; target rendered with an oblique "
                    f"covariance {tuple(round(c, 4) for c in true_cov)}; start: the initial mesh and a round PSF "
                    f"1.15x wider; {args.rounds} rounds of {S} shape + {P} PSF steps",
        "band_frequencies_shape_step": band,
        "half_spectrum_frequencies_psf_step": nH,
        "ms_per_shape_step": t_shape / (args.rounds * S),
        "ms_per_psf_step": t_psf / (args.rounds * P),
        "ms_per_round": t_all / args.rounds,
        # the headline's unit: forward and adjoint terms both counted
        "shape_terms_per_s": 2 * n_t * band / (t_shape / (args.rounds * S) * 1e-3),
        "cg_iterations_per_column_solve": cg["iterations"] / max(1, 2 * 3 * args.rounds * S),
        "cg_max": cg["max"],
        "stage_ms_per_round": {k: v[0] / args.rounds for k, v in stages.items() if v[1]},
        "shape_loss": [float(hs[0]), float(hs[-1])],
        "psf_loss": [float(hp[0]), float(hp[-1])],
        "cov_fitted": [round(c, 5) for c in psf.cov],
        "cov_true": [round(c, 5) for c in true_cov],
    }
    print(json.dumps(out), flush=True)


def run_robust_mode(args):
    """Robustness to initial conditions and noise (the paper's synthetic robustness study, with a seeded
    SH-deformed cell in place of its graphics mesh): every sweep point is one fit job of the served path
    (large-steps optimiser, target-weighted loss); reports the image MSE of the fitted mesh against the
    clean target and the symmetric mean nearest-vertex distance to the true mesh."""
    import torch
    from scipy.spatial import cKDTree

    import synth
    from paper_2303_10440_b300 import PSF, Renderer
    from paper_2303_10440_b300.serve import FitServer

    dev = torch.device("cuda", 0)
    steps = args.fit_steps or 300
    grid = synth.Grid(n=(64, 64, 64), h=(0.5, 0.5, 1.0))
    R = 8.0
    Vt, F = synth.sh_deformed_sphere(4, R, grid.center, lmax=6, coef_sigma=0.06 * R, seed=31)
    psf = PSF(sigma=(0.3, 0.3, 0.7), band_tau=1e-3)
    r32 = Renderer("fp32")
    clean = r32.render(torch.as_tensor(Vt).to(dev), torch.as_tensor(F).to(dev), grid, psf).cpu().numpy()
    ref_ms = float(np.mean(clean ** 2))
    points = []
    for s in (0.5, 0.75, 1.0, 1.25, 1.5):
        points.append(("scale", s, synth.sphere_mesh(4, s * R, grid.center)[0], clean))
    for d in (0.0, 1.0, 2.0, 4.0, 6.0):
        c = np.asarray(grid.center) + np.array([d, 0.5 * d, 0.0])
        points.append(("shift_um", d, synth.sphere_mesh(4, R, c)[0], clean))
    for k, peak in enumerate((1000.0, 200.0, 50.0, 10.0)):
        noisy, scale = synth.add_poisson_gaussian_noise(clean, peak, 2.0, seed=70 + k)
        if args.clip_target:
            # the read noise makes some background voxels negative; as weights of the target-weighted
            # loss they would reward intensity there
            noisy = np.maximum(noisy, 0.0)
        points.append(("noise_peak_counts", peak, synth.sphere_mesh(4, R, grid.center)[0], noisy / scale))
    decay = args.lr_decay
    jobs = [dict(V=V0, F=F, target=T, grid=grid, psf=psf, steps=steps, lr_vertex=1.0, loss="weighted",
                 optimizer="large_steps", lr_decay=decay) for _, _, V0, T in points]
    srv = FitServer(device=0, max_jobs=len(jobs))
    t0 = srv.clock()
    ids = [srv.submit(**j) for j in jobs]
    res = []
    for i in ids:
        assert srv.wait(i, timeout=1200)
        res.append(srv.result(i))
    span = srv.clock() - t0
    srv.shutdown()
    tree_t = cKDTree(Vt)
    cen = np.asarray(grid.center)

    def radial_error(V):
        """mean | |v - c| - r_true(direction of v) |: distance to the true (star-shaped) surface along rays."""
        d = V - cen
        n = np.linalg.norm(d, axis=1)
        return float(np.mean(np.abs(n - synth.sh_radius(d / n[:, None], R, 6, 0.06 * R, 31))))

    rows = []
    for (kind, val, V0, _), rr in zip(points, res):
        img = r32.render(torch.as_tensor(rr.V).to(dev), torch.as_tensor(F).to(dev), grid, psf).cpu().numpy()
        img0 = r32.render(torch.as_tensor(V0).to(dev), torch.as_tensor(F).to(dev), grid, psf).cpu().numpy()
        d_f = 0.5 * (tree_t.query(rr.V)[0].mean() + cKDTree(rr.V).query(Vt)[0].mean())
        d_0 = 0.5 * (tree_t.query(V0)[0].mean() + cKDTree(V0).query(Vt)[0].mean())
        h = np.asarray(rr.loss_history)
        rows.append(dict(sweep=kind, value=val, rel_image_mse_init=float(np.mean((img0 - clean) ** 2)) / ref_ms,
                         rel_image_mse_fit=float(np.mean((img - clean) ** 2)) / ref_ms,
                         radial_err_um_init=radial_error(V0), radial_err_um_fit=radial_error(rr.V),
                         vertex_set_dist_um_init=float(d_0), vertex_set_dist_um_fit=float(d_f),
                         loss_first=float(h[0]), loss_min=float(h.min()), loss_last=float(h[-1])))
    band = int(r32.band(grid, psf).numel())
    out = {"metric": "robustness to initial scale, shift and noise: image MSE and surface distance after the fit",
           "mode": "robust",
           "workload": f"SH-deformed cell (level 4, 5120 triangles, R = {R} um, l <= 6) in 64^3 of (0.5, 0.5, 1) um, "
                       f"sigma (0.3, 0.3, 0.7) um, band {band}; start: spheres of the sweep; {steps} large-steps "
                       f"iterations (lambda 50, lr 1.0 x {decay:g}^(t-1) at step t), target-weighted loss; "
                       f"Poisson(peak) + N(0, 2^2) noise",
           "jobs": len(jobs), "served_span_s": span, "fits_per_s": len(jobs) / span,
           "terms_per_s": 2.0 * band * len(F) * steps * len(jobs) / span, "rows": rows}
    print(json.dumps(out), flush=True)


def run_fft_mode(args):
    """The half-spectrum inverse (C2R) and forward (R2C) 3D transforms through dm_c2r / dm_r2c on device
    buffers, CUDA-event timed (L2 flushed before each call). Bytes per transform: each of the three axis
    passes reads and writes the array once (two complex passes over the half spectrum, one real/complex
    z pass), i.e. 2 * (2 |H| * 8 B) + (|H| * 8 B + N * 4 B); dm_c2r's first pass reads the (const) input
    spectrum where it lies and writes the workspace, so there is no staging copy."""
    import torch

    from paper_2303_10440_b300 import Grid, Renderer

    dev = torch.device("cuda", 0)
    r = Renderer("fp32")
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    hbm = float(peaks.get("hbm_gbs", 6400.0))
    flush = torch.empty(256 * 2**20 // 4, dtype=torch.float32, device=dev)
    rows = []
    for n in (128, 256, 512):
        grid = Grid(n=(n, n, n), h=(0.5, 0.5, 1.0))
        nH = n * n * (n // 2 + 1)
        spec = torch.randn(n, n, n // 2 + 1, dtype=torch.complex64, device=dev)
        img = torch.randn(n, n, n, dtype=torch.float32, device=dev)
        passes = 2 * (2 * nH * 8) + (nH * 8 + n**3 * 4)
        res = {}
        for name, fn, nbytes in (("c2r", lambda: r.c2r(grid, spec), passes),
                                 ("r2c", lambda: r.r2c(grid, img), passes)):
            for _ in range(3):
                fn()
            ts = []
            for _ in range(10):
                flush.fill_(1.0)
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record()
                fn()
                b.record()
                torch.cuda.synchronize()
                ts.append(a.elapsed_time(b))
            ms = float(np.median(ts))
            res[name] = {"ms": ms, "bytes": nbytes, "GB_per_s": nbytes / (ms * 1e-3) / 1e9,
                         "frac_of_hbm": nbytes / (ms * 1e-3) / 1e9 / hbm}
        rows.append({"grid": [n, n, n], **res})
        del spec, img
    print(json.dumps({"metric": "3D real FFT (C2R / R2C) throughput", "mode": "fft", "hbm_peak_gbs": hbm,
                      "hbm_peak_source": "MEASURED_PEAKS.json" if "hbm_gbs" in peaks else "fallback", "rows": rows}),
          flush=True)


def run_scaling_mode(args):
    """Fit-step time (forward + adjoint through dm_loss_and_grad, device buffers, CUDA events) against
    (i) the grid side for an 80-triangle icosphere on the whole spectrum, (ii) the triangle count on
    100^3, and (iii) a narrow-band case (128^3, h = 1, sigma = (2, 2, 5) voxels, tau = 1e-3); the FP64
    oracle is timed on the small cases for the GPU / CPU ratio."""
    import torch

    import synth
    from paper_2303_10440_b300 import Renderer

    dev = torch.device("cuda", 0)
    r = Renderer("fp32")
    flush = torch.empty(256 * 2**20 // 4, dtype=torch.float32, device=dev)

    def step_ms(V, F, grid, psf, reps=5):
        Vd, Fd = torch.as_tensor(V).to(dev), torch.as_tensor(F).to(dev)
        T = r.render(Vd * 1.01, Fd, grid, psf)
        # warm up for at least ~0.2 s of calls: a tiny case would otherwise be timed while the
        # clocks are still rising after the CPU oracle's run
        t_end = time.perf_counter() + 0.2
        n_warm = 0
        while n_warm < 2 or time.perf_counter() < t_end:
            r.loss_and_grad(Vd, Fd, grid, psf, T, "mse")
            n_warm += 1
        torch.cuda.synchronize()
        ts = []
        for _ in range(reps):
            flush.fill_(0.0)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            r.loss_and_grad(Vd, Fd, grid, psf, T, "mse")
            b.record()
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b))
        return float(np.median(ts)), int(r.band(grid, psf).numel())

    def oracle_ms(V, F, grid, psf):
        import oracle

        T = oracle.render(V * 1.01, F, grid, psf)["image"]
        t0 = time.perf_counter()
        oracle.loss_and_grad(V, F, grid, psf, T, "mse")
        return (time.perf_counter() - t0) * 1e3

    out = {"metric": "fit-step time against grid size and triangle count", "mode": "scaling", "grid_sweep": [],
           "triangle_sweep": [], "narrow_band": None}
    V1, F1 = synth.sphere_mesh(1, 1.0, (0, 0, 0))
    for n in (16, 32, 64, 128, 256):
        grid = synth.Grid(n=(n, n, n), h=(1.0, 1.0, 1.0))
        V = V1 * (0.3 * n) + np.asarray(grid.center)
        psf = synth.Psf(sigma=(0.8, 0.8, 0.8))
        ms, M = step_ms(V, F1, grid, psf)
        row = {"grid": n, "triangles": len(F1), "band": M, "ms": ms, "terms_per_s": 2 * M * len(F1) / (ms * 1e-3)}
        if n <= 32:
            row["oracle_ms"] = oracle_ms(V, F1, grid, psf)
            row["gpu_over_oracle"] = row["oracle_ms"] / ms
        out["grid_sweep"].append(row)
    grid = synth.Grid(n=(100, 100, 100), h=(1.0, 1.0, 1.0))
    for lev in (1, 2, 3, 4, 5, 6):
        V, F = synth.sphere_mesh(lev, 30.0, (50.0, 50.0, 50.0))
        ms, M = step_ms(V, F, grid, synth.Psf(sigma=(0.8, 0.8, 0.8)), reps=3 if lev >= 5 else 5)
        out["triangle_sweep"].append({"grid": 100, "triangles": len(F), "band": M, "ms": ms,
                                      "terms_per_s": 2 * M * len(F) / (ms * 1e-3)})
    grid = synth.Grid(n=(128, 128, 128), h=(1.0, 1.0, 1.0))
    V, F = synth.sh_deformed_sphere(4, 30.0, (64.0, 64.0, 64.0), lmax=6, coef_sigma=1.8, seed=2)
    psf = synth.Psf(sigma=(2.0, 2.0, 5.0), band_tau=1e-3)
    ms, M = step_ms(V, F, grid, psf)
    full_ms, Mf = step_ms(V, F, grid, synth.Psf(sigma=(2.0, 2.0, 5.0)))
    out["narrow_band"] = {"grid": 128, "triangles": len(F), "sigma_voxels": [2, 2, 5], "tau": 1e-3, "band": M,
                          "half_spectrum": Mf, "ms": ms, "ms_whole_spectrum": full_ms,
                          "terms_per_s": 2 * M * len(F) / (ms * 1e-3)}
    print(json.dumps(out), flush=True)


def run_mufu_probe(args):
    """Throughput of the MUFU sin/cos and reciprocal instructions the mesh-transform sums use, measured with
    a kernel of independent chains (the XU roofline of the forward sum)."""
    from paper_2303_10440_b300 import build

    lib = ctypes.CDLL(build.build_probe())
    lib.dm_probe_mufu.restype = ctypes.c_int
    lib.dm_probe_mufu.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.POINTER(ctypes.c_double)]
    res = {}
    for kind, name in ((0, "sincos"), (1, "rcp")):
        ops = ctypes.c_double()
        st = lib.dm_probe_mufu(kind, 0, ctypes.byref(ops))
        if st != 0:
            raise RuntimeError(f"dm_probe_mufu: {st}")
        res[name] = ops.value
    print(json.dumps({"metric": "MUFU throughput", "mode": "mufu", **res}), flush=True)


def main():
    args = parse()
    if args.mode == "mufu":
        run_mufu_probe(args)
        return
    if args.mode == "scaling":
        run_scaling_mode(args)
        return
    if args.mode == "fft":
        run_fft_mode(args)
        return
    if args.mode == "robust":
        run_robust_mode(args)
        return
    if args.mode == "stagger":
        run_stagger_mode(args)
        return
    if args.mode == "serve-batch":
        run_serve_batch_mode(args)
        return
    if args.mode == "serve-budget":
        run_serve_budget_mode(args)
        return
    if args.mode != "step":
        run_serve_mode(args)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
