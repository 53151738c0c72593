"""Runs whose iteration count is decided on the device -- the relative-energy
stop of Algorithms 1-2 and a backtracking rule that can reject -- replayed as
one CUDA graph whose loops are conditional nodes.

Checks: the graph run equals the host-stepped run bit for bit (kernel timing
on makes nlos_reconstruct step from the host), the stop fires at the FP64
oracle's iteration, the backtracking counts match the oracle, and a
backtracking rule that gives up ends the run with NLOS_ERR_DIVERGED."""

import numpy as np
import pytest

import synth
from oracle import admm, lct
from tests.gpu_util import dev, host, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nlos():
    from paper_2301_00406_gb300 import nlos as mod
    mod.load()
    return mod


def scene(model, n, nt, seed):
    key = "c1_alg1_32x32x256" if model == 1 else "c2_alg2_64x64x512"
    cfg = dict(synth.CONFIGS[key])
    cfg.update(nx=n, ny=n, nt=nt, bin_width_s=cfg["bin_width_s"] * cfg["nt"] / nt)
    g = lct.Geometry(n, n, nt, cfg["bin_width_s"])
    mask = synth.make_mask(cfg)
    vol = synth.make_volume(cfg, seed)
    sig = lct.Operator(g).forward(vol)
    tau0 = synth.poisson_measurement(sig, mask, cfg["peak"], cfg["background"], seed + 1)
    return cfg, g, mask, tau0


def params(nlos, model, cfg, iters):
    p = nlos.params_default(model)
    if model == 1:
        p.a, p.b, p.mu = cfg["a"], cfg["b"], cfg["mu"]
    else:
        p.a_u, p.b_u, p.a_tau, p.b_tau = cfg["a_u"], cfg["b_u"], cfg["a_tau"], cfg["b_tau"]
        p.lambda_, p.mu1, p.mu2, p.mu3 = cfg["lam"], cfg["mu1"], cfg["mu2"], cfg["mu3"]
    p.iters = iters
    return p


def run_both(nlos, plan, p, tau0, want_tau):
    """(graph run, host-stepped run) of the same reconstruction."""
    import torch
    t0 = dev(tau0)
    outs = []
    for timing in (False, True):
        plan.timing_enable(timing)
        try:
            u = torch.empty_like(t0)
            tau = torch.empty_like(t0) if want_tau else None
            st = plan.reconstruct(p, t0.data_ptr(), u.data_ptr(), tau.data_ptr() if want_tau else 0,
                                  nlos._stream())
            torch.cuda.synchronize()
            outs.append((u, tau, st))
        finally:
            plan.timing_enable(False)
    return outs


def stop_threshold(e, first=6):
    """An eps_stop that the relative changes e cross with a margin of at least 2 %
    on both sides (the FP32 energies agree with the oracle's to about 1e-6):
    the geometric mean of e[k] and min(e[:k]) for the first k >= first where
    they differ by 5 %; returns (eps, k + 1 iterations)."""
    for k in range(first, len(e)):
        m = min(e[:k])
        if m >= 1.05 * e[k]:
            return float(np.sqrt(m * e[k])), k + 1
    return None, None


@pytest.mark.parametrize("model", [1, 2])
def test_energy_stop_graph_equals_host_and_oracle(nlos, model):
    n, nt, cap = 16, 64, 60
    cfg, g, mask, tau0 = scene(model, n, nt, seed=11)
    op = lct.Operator(g, mask)
    if model == 1:
        _, h = admm.alg1(tau0, mask, g, cfg["a"], cfg["b"], cfg["mu"], cap, op=op)
    else:
        _, _, h = admm.alg2(tau0, mask, g, cfg["a_u"], cfg["b_u"], cfg["a_tau"], cfg["b_tau"], cfg["lam"],
                            cfg["mu1"], cfg["mu2"], cfg["mu3"], cap, op=op)
    eps, n_stop = stop_threshold(h["e"])
    assert eps is not None, h["e"]
    plan = nlos.Plan(n, n, nt, cfg["bin_width_s"], mask=mask)
    p = params(nlos, model, cfg, cap)
    p.eps_stop = eps
    assert plan.reconstruct_prepare(p, dev(tau0).data_ptr(), dev(tau0).data_ptr()) is True
    (ug, tg, sg), (uh, th, sh) = run_both(nlos, plan, p, tau0, model == 2)
    assert sg["iters_done"] == sh["iters_done"] == n_stop, (sg["iters_done"], sh["iters_done"], n_stop)
    assert np.array_equal(host(ug), host(uh)) and sg["energy"] == sh["energy"]
    if model == 2:
        assert np.array_equal(host(tg), host(th))
    if model == 1:
        u_ref, h2 = admm.alg1(tau0, mask, g, cfg["a"], cfg["b"], cfg["mu"], cap, op=op, eps_stop=eps)
    else:
        u_ref, _, h2 = admm.alg2(tau0, mask, g, cfg["a_u"], cfg["b_u"], cfg["a_tau"], cfg["b_tau"], cfg["lam"],
                                 cfg["mu1"], cfg["mu2"], cfg["mu3"], cap, op=op, eps_stop=eps)
    assert len(h2["E"]) == n_stop
    assert rel_l2(host(ug), u_ref) < 1e-3


def test_warm_started_energy_stop_graph_equals_host(nlos):
    n, nt = 16, 64
    cfg, g, mask, tau0 = scene(2, n, nt, seed=12)
    c1 = synth.CONFIGS["c1_alg1_32x32x256"]
    plan = nlos.Plan(n, n, nt, cfg["bin_width_s"], mask=mask)
    p = params(nlos, 2, cfg, 40)
    p.a, p.b, p.mu = c1["a"], c1["b"], c1["mu"]
    p.warm_start_iters = 5
    p.eps_stop = 2e-3
    (ug, tg, sg), (uh, th, sh) = run_both(nlos, plan, p, tau0, True)
    assert 1 <= sg["iters_done"] == sh["iters_done"] <= 40
    assert np.array_equal(host(ug), host(uh)) and np.array_equal(host(tg), host(th))
    assert sg["energy"] == sh["energy"] and sg["restarts"] == sh["restarts"]


def test_backtracking_loop_graph_equals_host_and_oracle(nlos):
    n, nt, iters = 8, 64, 8
    cfg, g, mask, tau0 = scene(1, n, nt, seed=0)
    op = lct.Operator(g, mask)
    n2, _ = lct.power_norm2(op)
    plan = nlos.Plan(n, n, nt, cfg["bin_width_s"], mask=mask)
    p = params(nlos, 1, cfg, iters)
    p.L0 = 1e-3 * n2                                   # rejects about ten times in the first iteration
    assert plan.reconstruct_prepare(p, dev(tau0).data_ptr(), dev(tau0).data_ptr()) is True
    (ug, _, sg), (uh, _, sh) = run_both(nlos, plan, p, tau0, False)
    assert np.array_equal(host(ug), host(uh))
    assert sg["backtracks"] == sh["backtracks"] and sg["L"] == sh["L"] and sg["iters_done"] == iters
    u_ref, h = admm.alg1(tau0, mask, g, cfg["a"], cfg["b"], cfg["mu"], iters, L0=p.L0, op=op)
    assert sg["backtracks"] == sum(h["backtracks"]) and sg["backtracks"] >= 9
    assert rel_l2(host(ug), u_ref) < 1e-3


def test_backtracking_give_up_ends_graph_run(nlos):
    import torch
    n, nt = 8, 64
    cfg, g, mask, tau0 = scene(1, n, nt, seed=0)
    op = lct.Operator(g, mask)
    n2, _ = lct.power_norm2(op)
    plan = nlos.Plan(n, n, nt, cfg["bin_width_s"], mask=mask)
    p = params(nlos, 1, cfg, 8)
    p.L0, p.max_backtracks = 1e-3 * n2, 2             # needs about ten rejections: gives up at the third
    t0 = dev(tau0)
    u = torch.empty_like(t0)
    assert plan.reconstruct_prepare(p, t0.data_ptr(), u.data_ptr()) is True
    with pytest.raises(nlos.NlosError) as ei:
        plan.reconstruct(p, t0.data_ptr(), u.data_ptr())
    assert ei.value.status == nlos.NLOS_ERR_DIVERGED
    # the plan and its context stay usable
    p.L0, p.max_backtracks = 0.0, 30
    st = plan.reconstruct(p, t0.data_ptr(), u.data_ptr())
    assert st["status"] == 0 and st["iters_done"] == 8
