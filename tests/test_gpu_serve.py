"""Continuous-batching fit server: a job's result is the same alone and in a mix, late
arrivals join running batches, admission waits for device memory, invalid jobs are refused."""

import time

import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu

STEPS = 6


def _jobs(r32):
    """Five uneven jobs: grids 32^3-64^3, icosphere levels 2-3, targets rendered from SH-deformed cells."""
    specs = [((64, 64, 64), 3, 7.0), ((32, 32, 32), 2, 4.0), ((48, 48, 48), 3, 5.0), ((64, 64, 32), 2, 6.0),
             ((40, 40, 40), 3, 4.5)]
    jobs = []
    for k, (n, lev, R) in enumerate(specs):
        grid = synth.Grid(n=n, h=(0.5, 0.5, 1.0) if n[2] == n[0] else (0.5, 0.5, 2.0))
        R = min(R, 0.3 * float(min(grid.L)))
        V_t, F = synth.sh_deformed_sphere(lev, R, grid.center, lmax=4, coef_sigma=0.04 * R, seed=40 + k)
        V0, _ = synth.sphere_mesh(lev, R, grid.center)
        psf = synth.Psf(sigma=(0.4, 0.4, 0.9), band_tau=1e-3)
        T = r32.render(torch.as_tensor(V_t).cuda(), torch.as_tensor(F).cuda(), grid, psf).cpu().numpy()
        jobs.append(dict(V=V0, F=F, target=T, grid=grid, psf=psf, steps=STEPS, lr_vertex=0.02))
    return jobs


@pytest.fixture(scope="module")
def setup():
    from paper_2303_10440_b300 import Renderer

    r32 = Renderer("fp32")
    jobs = _jobs(r32)
    yield r32, jobs
    r32.close()


def _run(server, jobs, order, late=()):
    ids = {}
    for k in order:
        ids[k] = server.submit(**jobs[k])
    if late:
        # wait until the batch is running, then add more jobs
        first = ids[order[0]]
        t_end = time.time() + 60
        while server.status(first)["steps_done"] < 1 and time.time() < t_end:
            time.sleep(0.001)
        for k in late:
            ids[k] = server.submit(**jobs[k])
    out = {}
    for k, i in ids.items():
        assert server.wait(i, timeout=300)
        out[k] = server.result(i)
    return out


def test_result_is_the_same_alone_and_in_the_mix(setup):
    from paper_2303_10440_b300.serve import FitServer

    r32, jobs = setup
    s1 = FitServer(max_jobs=8)
    alone = _run(s1, jobs, [0])[0]
    s1.shutdown()
    s2 = FitServer(max_jobs=8)
    mix = _run(s2, jobs, [1, 2, 0], late=[3, 4])
    st = s2.stats()
    s2.shutdown()
    assert st["peak_active"] >= 3
    assert np.array_equal(alone.V, mix[0].V)
    assert np.array_equal(alone.loss_history, mix[0].loss_history)
    print(f"\n[serve] alone == in mix (bitwise); peak batch {st['peak_active']}, iterations {st['iterations']}")


def test_served_fit_matches_the_standalone_fit(setup):
    from paper_2303_10440_b300.serve import FitServer

    r32, jobs = setup
    s = FitServer(max_jobs=4)
    res = _run(s, jobs, [0, 1])
    s.shutdown()
    for k in (0, 1):
        j = jobs[k]
        Vf, sig, hist = r32.fit(torch.as_tensor(j["V"]).cuda(), torch.as_tensor(j["F"]).cuda(), j["grid"], j["psf"],
                                torch.as_tensor(j["target"]).cuda(), steps=STEPS, lr_vertex=j["lr_vertex"])
        Vf = Vf.cpu().numpy()
        moved = np.linalg.norm(Vf - j["V"])
        assert moved > 0
        assert np.linalg.norm(res[k].V - Vf) < 1e-3 * moved
        assert np.allclose(res[k].loss_history, hist.numpy(), rtol=1e-4)


def test_served_fit_on_a_grid_with_factors_7_11_13(setup):
    """A job on a 28 x 26 x 22 grid (the batched FFT passes with radices 7, 13 and 11) served next to a
    power-of-two job: alone and in the mix bit for bit, and close to the standalone fit."""
    from paper_2303_10440_b300.serve import FitServer

    r32, jobs = setup
    grid = synth.Grid(n=(28, 26, 22), h=(0.5, 0.5, 1.0))
    R = 0.3 * float(min(grid.L))
    V_t, F = synth.sh_deformed_sphere(2, R, grid.center, lmax=4, coef_sigma=0.04 * R, seed=47)
    V0, _ = synth.sphere_mesh(2, R, grid.center)
    psf = synth.Psf(sigma=(0.4, 0.4, 0.9), band_tau=1e-3)
    T = r32.render(torch.as_tensor(V_t).cuda(), torch.as_tensor(F).cuda(), grid, psf).cpu().numpy()
    job = dict(V=V0, F=F, target=T, grid=grid, psf=psf, steps=STEPS, lr_vertex=0.02)
    s1 = FitServer(max_jobs=4)
    i = s1.submit(**job)
    assert s1.wait(i, timeout=300)
    alone = s1.result(i)
    s1.shutdown()
    s2 = FitServer(max_jobs=4)
    ids = [s2.submit(**jobs[1]), s2.submit(**job)]
    for k in ids:
        assert s2.wait(k, timeout=300)
    mix = s2.result(ids[1])
    s2.shutdown()
    assert np.array_equal(alone.V, mix.V)
    assert np.array_equal(alone.loss_history, mix.loss_history)
    Vf, _, hist = r32.fit(torch.as_tensor(V0).cuda(), torch.as_tensor(F).cuda(), grid, psf, torch.as_tensor(T).cuda(),
                          steps=STEPS, lr_vertex=job["lr_vertex"])
    Vf = Vf.cpu().numpy()
    moved = np.linalg.norm(Vf - V0)
    assert moved > 0
    assert np.linalg.norm(alone.V - Vf) < 1e-3 * moved
    assert np.allclose(alone.loss_history, hist.numpy(), rtol=1e-4)


def test_late_arrivals_join_running_batches(setup):
    from paper_2303_10440_b300.serve import FitServer

    _, jobs = setup
    long_job = dict(jobs[0], steps=60)
    s = FitServer(max_jobs=8)
    a = s.submit(**long_job)
    deadline = time.time() + 120
    while s.status(a)["steps_done"] < 2 and time.time() < deadline:
        time.sleep(0.001)
    b = s.submit(**jobs[1])
    c = s.submit(**jobs[2])
    for i in (a, b, c):
        assert s.wait(i, timeout=300)
    ra, rb, rc = s.result(a), s.result(b), s.result(c)
    s.shutdown()
    # b and c were admitted and finished while a was still running
    assert rb.t_start < ra.t_end and rc.t_start < ra.t_end
    assert rb.t_end < ra.t_end


def test_admission_waits_for_device_memory(setup):
    from paper_2303_10440_b300.serve import FitServer

    r32, jobs = setup
    j = jobs[1]  # 32^3 job
    probe = FitServer(max_jobs=1)
    i = probe.submit(**j)
    assert probe.wait(i, timeout=300)
    one_job = probe.stats()["bytes_peak"]  # arena bytes one such job holds
    probe.shutdown()
    s = FitServer(max_jobs=8, memory_bytes=int(one_job * 1.5))
    ids = [s.submit(**j) for _ in range(3)]
    res = [None] * 3
    for k, i in enumerate(ids):
        assert s.wait(i, timeout=300)
        res[k] = s.result(i)
    st = s.stats()
    with pytest.raises(RuntimeError, match="DM_ERR_OOM"):
        s.submit(**jobs[0])  # a 64^3 job can never fit this arena
    s.shutdown()
    assert st["peak_active"] == 1
    for k in (1, 2):
        assert res[k].t_start >= res[k - 1].t_end
    assert np.array_equal(res[0].V, res[1].V) and np.array_equal(res[1].V, res[2].V)


def test_invalid_jobs_are_refused(setup):
    from paper_2303_10440_b300.serve import FitServer

    _, jobs = setup
    s = FitServer(max_jobs=2)
    bad = dict(jobs[1])
    F = bad["F"].copy()
    F[0, 0] = 10**6
    bad["F"] = F
    with pytest.raises(RuntimeError, match="DM_ERR_ARG"):
        s.submit(**bad)
    bad = dict(jobs[1], grid=synth.Grid(n=(17, 17, 17), h=(1, 1, 1)))
    with pytest.raises(RuntimeError, match="DM_ERR_UNSUPPORTED"):
        s.submit(**bad)
    n_t = jobs[1]["F"].shape[0]
    for w, kw in ((np.full(n_t, -1.0), {}), (np.zeros(n_t), {}), (np.full(n_t, np.nan), {}),
                  (np.ones(n_t), {"label": "volume"})):
        with pytest.raises(RuntimeError, match="DM_ERR_ARG"):
            s.submit(**dict(jobs[1], weights=w, **kw))
    # degenerate and (volume label) open meshes are refused at submit, not in a running batch
    with pytest.raises(RuntimeError, match="DM_ERR_DEGENERATE"):
        s.submit(**dict(jobs[1], V=np.repeat(jobs[1]["V"][:1], len(jobs[1]["V"]), axis=0)))
    with pytest.raises(RuntimeError, match="DM_ERR_OPEN_MESH"):
        s.submit(**dict(jobs[1], F=jobs[1]["F"][:-1].copy(), label="volume"))
    s.shutdown()


def test_large_steps_job_matches_the_staggered_shape_fit(setup):
    """A served job with the large-steps optimiser (Section 5.1) follows dm_fit_staggered's shape steps."""
    from paper_2303_10440_b300.serve import FitServer

    r32, jobs = setup
    j = dict(jobs[1], optimizer="large_steps", lr_vertex=0.5)
    s = FitServer(max_jobs=2)
    i = s.submit(**j)
    assert s.wait(i, timeout=300)
    res = s.result(i)
    s.shutdown()
    V, _, hs, _, cg = r32.fit_staggered(torch.as_tensor(j["V"]).cuda(), torch.as_tensor(j["F"]).cuda(), j["grid"],
                                        j["psf"], torch.as_tensor(j["target"]).cuda(), rounds=1, shape_steps=STEPS,
                                        psf_steps=0, lr_vertex=0.5, lr_psf=0.0, shape_loss="mse")
    moved = np.linalg.norm(V.cpu().numpy() - j["V"])
    assert moved > 0 and cg["iterations"] > 0
    assert np.linalg.norm(res.V - V.cpu().numpy()) < 1e-3 * moved
    assert np.allclose(res.loss_history, hs.numpy(), rtol=1e-4)


def test_large_steps_job_is_the_same_alone_and_among_adam_jobs(setup):
    from paper_2303_10440_b300.serve import FitServer

    _, jobs = setup
    ls = dict(jobs[2], optimizer="large_steps", lr_vertex=0.5)
    s1 = FitServer(max_jobs=4)
    a = s1.submit(**ls)
    assert s1.wait(a, timeout=300)
    alone = s1.result(a)
    s1.shutdown()
    s2 = FitServer(max_jobs=4)
    ids = [s2.submit(**jobs[1]), s2.submit(**ls), s2.submit(**jobs[3])]
    for i in ids:
        assert s2.wait(i, timeout=300)
    mix = s2.result(ids[1])
    s2.shutdown()
    assert np.array_equal(alone.V, mix.V)
    assert np.array_equal(alone.loss_history, mix.loss_history)


def test_shortest_policy_runs_small_jobs_first_with_unchanged_results(setup):
    """DM_SCHED_SHORTEST: resident jobs with the least remaining work advance first, within a per-iteration
    term budget; a big job submitted first waits for the small ones, and every result is the same as alone."""
    from paper_2303_10440_b300.serve import FitServer

    _, jobs = setup
    big = dict(jobs[0], steps=30)          # 64^3, 1280 triangles: 1.7e8 terms per step
    small = dict(jobs[1], steps=STEPS)     # 32^3, 320 triangles: 5.6e6 terms per step
    s0 = FitServer(max_jobs=2)
    i0 = s0.submit(**small)
    assert s0.wait(i0, timeout=300)
    alone = s0.result(i0)
    s0.shutdown()
    s = FitServer(max_jobs=8, policy="shortest", batch_terms=1e8)
    a = s.submit(**big)
    ids = [s.submit(**small) for _ in range(3)]
    for i in [a] + ids:
        assert s.wait(i, timeout=300)
    rb = s.result(a)
    rs = [s.result(i) for i in ids]
    s.shutdown()
    assert all(r.t_end < rb.t_end for r in rs)
    for r in rs:
        assert np.array_equal(r.V, alone.V) and np.array_equal(r.loss_history, alone.loss_history)
    assert len(rb.loss_history) == 30 and rb.loss_history[-1] < rb.loss_history[0]


@pytest.mark.parametrize("optimizer,lr,decay", [("adam", 0.02, 1.0), ("large_steps", 0.5, 1.0),
                                               ("large_steps", 0.5, 0.9)])
def test_preempted_job_resumes_bit_for_bit(setup, optimizer, lr, decay):
    """Checkpoint / resume in the server: stop a running job, resubmit it with its state, and the result
    equals the uninterrupted run (vertices and the remaining losses); a decaying rate continues from
    the checkpoint's step."""
    from paper_2303_10440_b300.serve import FitServer

    _, jobs = setup
    steps = 60  # long enough that the preemption lands while the job still runs, on any host
    job = dict(jobs[2], steps=steps, optimizer=optimizer, lr_vertex=lr, lr_psf=0.002, lr_decay=decay)
    s0 = FitServer(max_jobs=2)
    i0 = s0.submit(**job)
    assert s0.wait(i0, timeout=300)
    full = s0.result(i0)
    s0.shutdown()
    s = FitServer(max_jobs=2)
    i = s.submit(**job)
    t_end = time.time() + 120
    while s.status(i)["steps_done"] < 4 and time.time() < t_end:
        time.sleep(0.001)
    out = s.preempt(i, timeout=120)
    assert out is not None
    V, state = out
    k = state["step"]
    assert 4 <= k < steps
    j = s.submit(**dict(job, V=V, steps=steps - k, resume=state))
    assert s.wait(j, timeout=300)
    rest = s.result(j)
    s.shutdown()
    assert np.array_equal(rest.V, full.V)
    assert np.array_equal(rest.loss_history, full.loss_history[k:])


def test_preempting_a_queued_job_returns_its_start_state(setup):
    from paper_2303_10440_b300.serve import FitServer

    _, jobs = setup
    s = FitServer(max_jobs=1)
    a = s.submit(**dict(jobs[0], steps=40))
    b = s.submit(**jobs[1])
    out = s.preempt(b, timeout=60)
    assert s.wait(a, timeout=300)
    s.result(a)
    s.shutdown()
    assert out is not None
    V, state = out
    assert state["step"] == 0 and np.array_equal(V, jobs[1]["V"])
    assert not np.any(state["m_V"]) and not np.any(state["v_V"])


@pytest.mark.parametrize("optimizer,lr", [("adam", 0.02), ("large_steps", 0.5)])
def test_rate_decay_scales_each_step(setup, optimizer, lr):
    """Step t of a job with lr_decay g takes the rate lr g^(t-1): the first step equals the constant-rate
    job's, and the second step's displacement is g times the constant-rate job's second displacement
    (same point, same moments; Adam's step is linear in the rate, and so is the large-steps smoothing
    solve up to its stopping rule: relative residual 1e-6 from the previous step's solution, times the
    smoothing matrix's condition number, ~600 here)."""
    from paper_2303_10440_b300.serve import FitServer

    _, jobs = setup
    g = 0.5
    base = dict(jobs[1], optimizer=optimizer, lr_vertex=lr)
    s = FitServer(max_jobs=1)

    def run(**kw):
        i = s.submit(**dict(base, **kw))
        assert s.wait(i, timeout=300)
        return s.result(i).V

    V1, V1d = run(steps=1), run(steps=1, lr_decay=g)
    V2, V2d = run(steps=2), run(steps=2, lr_decay=g)
    s.shutdown()
    assert np.array_equal(V1, V1d)
    d, dd = V2 - V1, V2d - V1
    assert np.linalg.norm(d) > 0
    tol = 1e-12 if optimizer == "adam" else 2e-3
    assert np.linalg.norm(dd - g * d) <= tol * np.linalg.norm(d)


def test_volume_job_in_a_mixed_batch(setup):
    """A volume-labelled job runs in the batched launches of its own label beside surface jobs: the same
    result alone and in the mix (bitwise), and the standalone dm_fit's within FP32 tolerance."""
    from paper_2303_10440_b300.serve import FitServer

    r32, jobs = setup
    j = jobs[2]
    # a target without the start's symmetries: Adam's first steps are +-lr on every coordinate, so a
    # gradient component that vanishes by symmetry would turn rounding differences into full steps
    R = 0.9 * float(np.linalg.norm(j["V"][0] - np.asarray(j["grid"].center)))
    Vt, _ = synth.sh_deformed_sphere(3, R, j["grid"].center, lmax=4, coef_sigma=0.05 * R, seed=77)
    T = r32.render(torch.as_tensor(Vt).cuda(), torch.as_tensor(j["F"]).cuda(), j["grid"], j["psf"],
                   label="volume").cpu().numpy()
    vj = dict(j, target=T, label="volume")
    s1 = FitServer(max_jobs=4)
    alone = _run(s1, [vj], [0])[0]
    s1.shutdown()
    s2 = FitServer(max_jobs=4)
    mix = _run(s2, [jobs[1], vj, jobs[3]], [0, 1, 2])
    st = s2.stats()
    s2.shutdown()
    assert st["peak_active"] >= 2
    assert np.array_equal(alone.V, mix[1].V)
    assert np.array_equal(alone.loss_history, mix[1].loss_history)
    Vf, sig, hist = r32.fit(torch.as_tensor(j["V"]).cuda(), torch.as_tensor(j["F"]).cuda(), j["grid"], j["psf"],
                            torch.as_tensor(T).cuda(), steps=STEPS, lr_vertex=j["lr_vertex"], label="volume")
    Vf = Vf.cpu().numpy()
    moved = np.linalg.norm(Vf - j["V"])
    assert moved > 0
    assert np.linalg.norm(mix[1].V - Vf) < 1e-3 * moved
    assert np.allclose(mix[1].loss_history, hist.numpy(), rtol=1e-4)


def test_weighted_multicell_job_matches_the_standalone_fit(setup):
    """A two-cell foam with a doubled shared wall (densities 1 and 2, Sections 3.3 and 4.1) as one served job:
    the same result alone and in a mix, and the standalone weighted fit's within FP32 tolerance."""
    from paper_2303_10440_b300.serve import FitServer

    r32, jobs = setup
    grid = synth.Grid(n=(32, 32, 24), h=(0.5, 0.5, 1.0))
    V0, F, rho = synth.box_foam((2, 1, 1), (5.0, 6.0, 6.0), subdiv=2, origin=(3.0, 5.0, 6.0), jitter=0.1, seed=2)
    Vt = V0 + 0.2 * np.cos(V0[:, [2, 0, 1]] / 2.5)
    psf = synth.Psf(sigma=(0.4, 0.4, 0.9), band_tau=1e-3)
    W = rho.astype(np.float32)
    T = r32.render(torch.as_tensor(Vt).cuda(), torch.as_tensor(F).cuda(), grid, psf,
                   weights=torch.as_tensor(W).cuda()).cpu().numpy()
    wj = dict(V=V0, F=F, target=T, grid=grid, psf=psf, steps=STEPS, lr_vertex=0.02, weights=W)
    s1 = FitServer(max_jobs=4)
    alone = _run(s1, [wj], [0])[0]
    s1.shutdown()
    s2 = FitServer(max_jobs=4)
    mix = _run(s2, [jobs[1], wj], [0, 1])
    s2.shutdown()
    assert np.array_equal(alone.V, mix[1].V)
    assert np.array_equal(alone.loss_history, mix[1].loss_history)
    Vf, sig, hist = r32.fit(torch.as_tensor(V0).cuda(), torch.as_tensor(F).cuda(), grid, psf, torch.as_tensor(T).cuda(),
                            steps=STEPS, lr_vertex=0.02, weights=torch.as_tensor(W).cuda())
    Vf = Vf.cpu().numpy()
    moved = np.linalg.norm(Vf - V0)
    assert moved > 0
    assert np.linalg.norm(mix[1].V - Vf) < 1e-3 * moved
    assert np.allclose(mix[1].loss_history, hist.numpy(), rtol=1e-4)
    # the densities matter: an unweighted job ends elsewhere
    s3 = FitServer(max_jobs=1)
    plain = _run(s3, [dict(wj, weights=None)], [0])[0]
    s3.shutdown()
    assert np.linalg.norm(plain.V - mix[1].V) > 1e-2 * moved


def test_graph_replayed_iterations_equal_direct_ones(setup):
    """While the set of advanced jobs is unchanged the server replays one captured iteration (a CUDA
    graph; the Adam step and its decayed rate are read on the device): the vertices, sigma and loss
    histories are bitwise those of a server that enqueues every iteration directly, for a batch (job
    streams forked and joined inside the graph: Adam, large steps, decay, PSF learning) and for a lone job
    (all on the server stream)."""
    from paper_2303_10440_b300.serve import FitServer

    _, jobs = setup
    mix = [dict(jobs[0]), dict(jobs[1], optimizer="large_steps", lr_vertex=0.5, lr_decay=0.9, lr_psf=0.002),
           dict(jobs[2], lr_decay=0.95, lr_psf=0.002), dict(jobs[3], steps=9)]
    lone = [dict(jobs[4], steps=12, lr_psf=0.002, lr_decay=0.97)]
    for batch in (mix, lone):
        res, stats = {}, {}
        for graphs in (True, False):
            s = FitServer(max_jobs=8, graphs=graphs)
            res[graphs] = _run(s, batch, list(range(len(batch))))
            stats[graphs] = s.stats()
            s.shutdown()
        assert stats[False]["graph_replays"] == 0
        # the first iteration over a job set runs directly, the second is captured, the rest replay it
        # (how often the batch's set changes depends on when the submissions reach the engine)
        assert stats[True]["graph_replays"] > 0
        if len(batch) == 1:
            assert stats[True]["graph_replays"] == stats[True]["iterations"] - 1
        for k in range(len(batch)):
            a, b = res[True][k], res[False][k]
            assert np.array_equal(a.V, b.V)
            assert np.array_equal(a.sigma, b.sigma)
            assert np.array_equal(a.loss_history, b.loss_history)
            assert np.all(np.isfinite(a.loss_history)) and np.all(a.loss_history > 0)  # every step's loss stored
        print(f"\n[serve] {len(batch)} job(s): graph replays {stats[True]['graph_replays']} of "
              f"{stats[True]['iterations']} iterations, results bitwise the direct ones")
