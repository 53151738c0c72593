"""Batched and served reconstructions (nlos_reconstruct_batch, nlos_server_*):
every scene's result is the same alone, in a batch and in the served mix (bit
for bit: a job's launch sequence and reduction order do not depend on its
neighbours), admission respects the HBM budget, and failures are reported."""

import numpy as np
import pytest

import synth
from oracle import lct
from tests.gpu_util import dev, host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nlos():
    from paper_2301_00406_gb300 import nlos as mod
    mod.load()
    return mod


def make_job(nlos, i):
    """Mixed sizes, masks and models, seeded by i."""
    shapes = [(16, 64), (32, 128), (16, 128), (32, 256)]
    n, nt = shapes[i % len(shapes)]
    model = 1 + (i % 2)
    bw = 32e-12 * 256 / nt
    mask = synth.stride_mask(n, n, 2) if i % 3 else synth.random_mask(n, n, 0.25, i)
    g = lct.Geometry(n, n, nt, bw)
    vol = synth.scene_patches(n, n, nt, i) if model == 2 else synth.scene_planes_glyph(n, n, nt, i)
    tau0 = synth.poisson_measurement(lct.Operator(g).forward(vol), mask, 50.0, 2.0, 100 + i)
    p = nlos.params_default(model)
    p.iters = 12 + (i % 3) * 4
    return dict(n=n, nt=nt, bw=bw, mask=mask, tau0=tau0.astype(np.float32), params=p)


def alone(nlos, job):
    plan = nlos.Plan(job["n"], job["n"], job["nt"], job["bw"], mask=job["mask"])
    u, _ = nlos.reconstruct_t(plan, job["params"], dev(job["tau0"]))
    out = host(u)
    plan.close()
    return out


def test_batch_equals_alone(nlos):
    import torch
    jobs = [make_job(nlos, i) for i in range(6)]
    plans = [nlos.Plan(j["n"], j["n"], j["nt"], j["bw"], mask=j["mask"]) for j in jobs]
    t0 = [dev(j["tau0"]) for j in jobs]
    us = [torch.empty_like(t) for t in t0]
    stream = torch.cuda.current_stream().cuda_stream
    stats = nlos.reconstruct_batch(plans, [j["params"] for j in jobs], [t.data_ptr() for t in t0],
                                   [u.data_ptr() for u in us], stream=stream)
    torch.cuda.synchronize()
    for j, u, st in zip(jobs, us, stats):
        assert st["status"] == 0 and st["iters_done"] == j["params"].iters
        assert np.array_equal(host(u), alone(nlos, j))
    for p in plans:
        p.close()


def test_batch_rejects_duplicate_plan(nlos):
    import torch
    j = make_job(nlos, 0)
    plan = nlos.Plan(j["n"], j["n"], j["nt"], j["bw"], mask=j["mask"])
    t = dev(j["tau0"])
    u = torch.empty_like(t)
    with pytest.raises(nlos.NlosError):
        nlos.reconstruct_batch([plan, plan], [j["params"]] * 2, [t.data_ptr()] * 2, [u.data_ptr()] * 2)


def test_served_equals_alone(nlos):
    """A long job first, then ten short ones of mixed size, sampling and
    model: with the contexts prepared before the submissions, the short jobs
    are admitted while the long one runs, so the mix really overlaps on the
    device (at least two jobs running at once), and every result is the one
    the job gives alone, bit for bit."""
    long_job = make_job(nlos, 3)                          # 32 x 32 x 256, Algorithm 2
    long_job["params"].iters = 600
    jobs = [long_job] + [make_job(nlos, i) for i in range(10)]
    srv = nlos.Server(hbm_budget_bytes=8 << 30, max_slots=4)
    for j in jobs:
        assert srv.prepare(j["n"], j["n"], j["nt"], j["bw"], j["params"], contexts=1, mask=j["mask"]) >= 1
    outs = [np.full(j["tau0"].shape, np.nan, np.float32) for j in jobs]
    ids = [srv.submit(j["n"], j["n"], j["nt"], j["bw"], j["params"], j["tau0"], o, mask=j["mask"])
           for j, o in zip(jobs, outs)]
    for jid in ids:
        st = srv.wait(jid, timeout_s=120.0)
        assert st is not None and st["status"] == 0
    info = srv.info()
    assert info["completed"] == len(jobs) and info["failed"] == 0
    assert 2 <= info["peak_running"] <= 4, info
    srv.close()
    for j, o in zip(jobs, outs):
        assert np.array_equal(o, alone(nlos, j).astype(np.float32))


def test_admission_respects_budget(nlos):
    from paper_2301_00406_gb300 import nlos as mod
    jobs = [make_job(nlos, 3)] * 3              # 32x32x256, model 2
    # budget sized from the first run: one job's context fits, two do not
    probe = mod.Server(hbm_budget_bytes=8 << 30, max_slots=1)
    o = np.zeros(jobs[0]["tau0"].shape, np.float32)
    jid = probe.submit(32, 32, 256, jobs[0]["bw"], jobs[0]["params"], jobs[0]["tau0"], o, mask=jobs[0]["mask"])
    probe.wait(jid, 120.0)
    one = probe.info()["bytes_peak"]
    probe.close()
    srv = mod.Server(hbm_budget_bytes=int(one * 1.3), max_slots=8)
    outs = [np.zeros(j["tau0"].shape, np.float32) for j in jobs]
    ids = [srv.submit(32, 32, 256, j["bw"], j["params"], j["tau0"], o, mask=j["mask"]) for j, o in zip(jobs, outs)]
    for jid in ids:
        assert srv.wait(jid, 120.0)["status"] == 0
    info = srv.info()
    assert info["peak_running"] == 1 and info["bytes_peak"] <= info["budget"]
    srv.close()
    ref = alone(nlos, jobs[0]).astype(np.float32)
    for o in outs:
        assert np.array_equal(o, ref)


def test_server_prepare_warms_contexts(nlos):
    """nlos_server_prepare builds the plan and idle contexts with captured graphs
    ahead of the jobs; jobs then reuse them (no new device memory) and give the
    same result as the plan alone; contexts beyond the budget are not made."""
    j = make_job(nlos, 1)                       # 32x32x128, model 2
    srv = nlos.Server(hbm_budget_bytes=8 << 30, max_slots=4)
    assert srv.prepare(j["n"], j["n"], j["nt"], j["bw"], j["params"], contexts=2, mask=j["mask"]) == 2
    warm = srv.info()
    assert warm["running"] == 0 and warm["completed"] == 0 and warm["bytes_in_use"] > 0
    # asking again creates nothing new
    assert srv.prepare(j["n"], j["n"], j["nt"], j["bw"], j["params"], contexts=2, mask=j["mask"]) == 2
    assert srv.info()["bytes_in_use"] == warm["bytes_in_use"]
    outs = [np.full(j["tau0"].shape, np.nan, np.float32) for _ in range(2)]
    ids = [srv.submit(j["n"], j["n"], j["nt"], j["bw"], j["params"], j["tau0"], o, mask=j["mask"]) for o in outs]
    for jid in ids:
        assert srv.wait(jid, timeout_s=120.0)["status"] == 0
    info = srv.info()
    assert info["completed"] == 2 and info["bytes_peak"] == warm["bytes_in_use"]
    srv.close()
    ref = alone(nlos, j).astype(np.float32)
    for o in outs:
        assert np.array_equal(o, ref)
    # a budget that holds the plan but no context: nothing is made, no error
    tiny = nlos.Server(hbm_budget_bytes=1 << 20, max_slots=2)
    assert tiny.prepare(j["n"], j["n"], j["nt"], j["bw"], j["params"], contexts=3, mask=j["mask"]) == 0
    tiny.close()


def test_job_larger_than_budget_fails(nlos):
    j = make_job(nlos, 0)
    srv = nlos.Server(hbm_budget_bytes=1 << 20, max_slots=2)
    o = np.zeros(j["tau0"].shape, np.float32)
    jid = srv.submit(j["n"], j["n"], j["nt"], j["bw"], j["params"], j["tau0"], o, mask=j["mask"])
    with pytest.raises(nlos.NlosError) as e:
        srv.wait(jid, 60.0)
    assert e.value.status == -2
    srv.close()


def test_destroy_cancels_queued_jobs(nlos):
    jobs = [make_job(nlos, 3) for _ in range(6)]
    for j in jobs:
        j["params"].iters = 60
    srv = nlos.Server(hbm_budget_bytes=8 << 30, max_slots=1)
    outs = [np.zeros(j["tau0"].shape, np.float32) for j in jobs]
    ids = [srv.submit(32, 32, 256, j["bw"], j["params"], j["tau0"], o, mask=j["mask"]) for j, o in zip(jobs, outs)]
    srv.close(cancel_pending=True, timeout_s=60.0)   # returns; no hang
    # ids are gone with the server; the point is that close() returned
    assert len(ids) == 6


def test_reconstruct_prepare_then_run_matches_plain_run(nlos):
    import torch
    job = make_job(nlos, 3)
    plan = nlos.Plan(job["n"], job["n"], job["nt"], job["bw"], mask=job["mask"])
    tau0 = dev(job["tau0"])
    u_plain = torch.empty_like(tau0)
    st_plain = plan.reconstruct(job["params"], tau0.data_ptr(), u_plain.data_ptr())
    u = torch.empty_like(tau0)
    assert plan.reconstruct_prepare(job["params"], tau0.data_ptr(), u.data_ptr()) is True
    st = plan.reconstruct(job["params"], tau0.data_ptr(), u.data_ptr())
    assert torch.equal(u, u_plain) and st["energy"] == st_plain["energy"]
    p = nlos.params_default(job["params"].model)
    p.iters, p.eps_stop = 3, 1e-9                       # stop decided on the device: a looped graph
    assert plan.reconstruct_prepare(p, tau0.data_ptr(), u.data_ptr()) is True
    p.iters = 0                                         # nothing to run: no graph
    assert plan.reconstruct_prepare(p, tau0.data_ptr(), u.data_ptr()) is False
