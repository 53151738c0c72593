"""GPU parity of the full ADMM reconstructions (nlos_reconstruct) against
the FP64 oracle: 1e-3 relative L2 on the volume after the fixed iteration
count, matching energies, backtracking counts and the zero fixed point."""

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


def scene(model, n, nt, seed=0, mask_kind="stride"):
    key = "c1_alg1_32x32x256" if model == 1 else "c2_alg2_64x64x512"
    cfg = dict(synth.CONFIGS[key])
    cfg.update(nx=n, ny=n, nt=nt, bin_width_s=cfg["bin_width_s"] * cfg["nt"] / nt)
    g = lct.Geometry(n, n, nt, cfg["bin_width_s"])
    mask = synth.make_mask(cfg) if mask_kind == "stride" else synth.random_mask(n, n, 0.25, seed + 9)
    vol = synth.make_volume(cfg, seed)
    sig = lct.Operator(g).forward(vol)
    tau0 = synth.poisson_measurement(sig, mask, cfg["peak"], cfg["background"], seed + 1)
    return cfg, g, mask, vol, tau0


def alg1_params(nlos, cfg, iters, L0):
    p = nlos.params_default(1)
    p.a, p.b, p.mu, p.iters, p.L0 = cfg["a"], cfg["b"], cfg["mu"], iters, L0
    return p


def alg2_params(nlos, cfg, iters, L0):
    p = nlos.params_default(2)
    p.a_u, p.b_u, p.a_tau, p.b_tau = cfg["a_u"], cfg["b_u"], cfg["a_tau"], cfg["b_tau"]
    p.lambda_, p.mu1, p.mu2, p.mu3 = cfg["lam"], cfg["mu1"], cfg["mu2"], cfg["mu3"]
    p.iters, p.L0 = iters, L0
    return p


@pytest.mark.parametrize("n,nt,iters", [(16, 64, 1), (16, 64, 10), (32, 256, 30)])
def test_alg1_parity(nlos, n, nt, iters):
    cfg, g, mask, vol, tau0 = scene(1, n, nt)
    op = lct.Operator(g, mask)
    n2, _ = lct.power_norm2(op)
    plan = nlos.Plan(n, n, nt, cfg["bin_width_s"], mask=mask)
    u_gpu, st = nlos.reconstruct_t(plan, alg1_params(nlos, cfg, iters, 2 * n2), dev(tau0))
    u_ref, h = admm.alg1(tau0, mask, g, cfg["a"], cfg["b"], cfg["mu"], iters, L0=2 * n2, op=op)
    err = rel_l2(host(u_gpu), u_ref)
    assert err < (1e-5 if iters == 1 else 1e-3), err
    assert st["iters_done"] == iters and st["backtracks"] == 0 and st["status"] == 0
    assert abs(st["energy"] - h["E"][-1]) <= 1e-3 * abs(h["E"][-1])
    assert abs(st["primal_res"] - h["primal_res"][-1]) <= 1e-3 * h["primal_res"][-1] + 1e-9


def test_alg1_default_L0_uses_plan_norm(nlos):
    cfg, g, mask, vol, tau0 = scene(1, 16, 64, seed=4, mask_kind="random")
    op = lct.Operator(g, mask)
    plan = nlos.Plan(16, 16, 64, cfg["bin_width_s"], mask=mask)
    u_gpu, st = nlos.reconstruct_t(plan, alg1_params(nlos, cfg, 8, 0.0), dev(tau0))
    u_ref, h = admm.alg1(tau0, mask, g, cfg["a"], cfg["b"], cfg["mu"], 8, op=op)
    assert rel_l2(host(u_gpu), u_ref) < 1e-3
    assert abs(st["L"] - h["L"][-1]) <= 1e-4 * h["L"][-1]


def test_alg1_backtracking_counts(nlos):
    cfg, g, mask, vol, tau0 = scene(1, 8, 64)
    op = lct.Operator(g, mask)
    n2, _ = lct.power_norm2(op)
    plan = nlos.Plan(8, 8, 64, cfg["bin_width_s"], mask=mask)
    L0 = 1e-3 * n2
    u_gpu, st = nlos.reconstruct_t(plan, alg1_params(nlos, cfg, 8, L0), dev(tau0))
    u_ref, h = admm.alg1(tau0, mask, g, cfg["a"], cfg["b"], cfg["mu"], 8, L0=L0, op=op)
    assert st["backtracks"] == sum(h["backtracks"])
    assert st["L"] == pytest.approx(h["L"][-1], rel=1e-12)
    assert rel_l2(host(u_gpu), u_ref) < 1e-3


def test_zero_data_fixed_point(nlos):
    n, nt = 16, 64
    plan = nlos.Plan(n, n, nt, 128e-12, mask=synth.stride_mask(n, n, 2))
    tau0 = np.zeros((n, n, nt))
    p = nlos.params_default(1)
    p.iters = 4
    u, st = nlos.reconstruct_t(plan, p, dev(tau0))
    assert np.all(host(u) == 0.0) and st["energy"] == 0.0
    p = nlos.params_default(2)
    p.iters = 4
    u, tau, st = nlos.reconstruct_t(plan, p, dev(tau0), want_tau=True)
    assert np.all(host(u) == 0.0) and np.all(host(tau) == 0.0)


@pytest.mark.parametrize("n,nt,iters", [(16, 64, 1), (16, 128, 20), (32, 256, 30)])
def test_alg2_parity(nlos, n, nt, iters):
    cfg, g, mask, vol, tau0 = scene(2, n, nt)
    op = lct.Operator(g, mask)
    n2, _ = lct.power_norm2(op, masked=False)
    plan = nlos.Plan(n, n, nt, cfg["bin_width_s"], mask=mask)
    u_gpu, tau_gpu, st = nlos.reconstruct_t(plan, alg2_params(nlos, cfg, iters, 2 * n2), dev(tau0), want_tau=True)
    u_ref, tau_ref, h = admm.alg2(tau0, mask, g, cfg["a_u"], cfg["b_u"], cfg["a_tau"], cfg["b_tau"], cfg["lam"],
                                  cfg["mu1"], cfg["mu2"], cfg["mu3"], iters, L0=2 * n2, op=op)
    eu, et = rel_l2(host(u_gpu), u_ref), rel_l2(host(tau_gpu), tau_ref)
    tol = 1e-5 if iters == 1 else 1e-3
    assert eu < tol and et < tol, (eu, et)
    assert st["restarts"] == sum(h["restart"])
    assert abs(st["energy"] - h["E"][-1]) <= 1e-3 * abs(h["E"][-1])


def test_alg2_warm_start_parity(nlos):
    # the remark after Algorithm 2: u starts from W Algorithm-1 iterations, tau from 0
    n, nt, W, iters = 16, 64, 6, 12
    cfg, g, mask, vol, tau0 = scene(2, n, nt, seed=2)
    c1 = synth.CONFIGS["c1_alg1_32x32x256"]
    op = lct.Operator(g, mask)
    n2, _ = lct.power_norm2(op, masked=False)
    plan = nlos.Plan(n, n, nt, cfg["bin_width_s"], mask=mask)
    p = alg2_params(nlos, cfg, iters, 2 * n2)
    p.a, p.b, p.mu = c1["a"], c1["b"], c1["mu"]
    p.warm_start_iters = W
    u_gpu, tau_gpu, st = nlos.reconstruct_t(plan, p, dev(tau0), want_tau=True)
    u_w, _ = admm.alg1(tau0, mask, g, c1["a"], c1["b"], c1["mu"], W, op=op)
    u_ref, tau_ref, h = admm.alg2(tau0, mask, g, cfg["a_u"], cfg["b_u"], cfg["a_tau"], cfg["b_tau"], cfg["lam"],
                                  cfg["mu1"], cfg["mu2"], cfg["mu3"], iters, L0=2 * n2, op=op, u_init=u_w)
    eu, et = rel_l2(host(u_gpu), u_ref), rel_l2(host(tau_gpu), tau_ref)
    assert eu < 1e-3 and et < 1e-3, (eu, et)
    assert st["iters_done"] == iters and st["status"] == 0
    assert st["restarts"] == sum(h["restart"])
    assert abs(st["energy"] - h["E"][-1]) <= 1e-3 * abs(h["E"][-1])
    # and it differs from the cold start
    p.warm_start_iters = 0
    u_cold, _ = nlos.reconstruct_t(plan, p, dev(tau0))
    assert rel_l2(host(u_cold), u_ref) > 1e-2


@pytest.mark.parametrize("kind", ["tac", "trv"])
def test_alg1_phi_variant_parity(nlos, kind):
    # phi = a + b |kappa| (TAC) and sqrt(a + b kappa^2) (TRV), Sec. 3
    n, nt, iters = 16, 64, 10
    cfg, g, mask, vol, tau0 = scene(1, n, nt, seed=5)
    op = lct.Operator(g, mask)
    n2, _ = lct.power_norm2(op)
    plan = nlos.Plan(n, n, nt, cfg["bin_width_s"], mask=mask)
    p = alg1_params(nlos, cfg, iters, 2 * n2)
    p.phi = {"tac": nlos.PHI_TAC, "trv": nlos.PHI_TRV}[kind]
    u_gpu, st = nlos.reconstruct_t(plan, p, dev(tau0))
    u_ref, h = admm.alg1(tau0, mask, g, cfg["a"], cfg["b"], cfg["mu"], iters, L0=2 * n2, op=op, phi_kind=kind)
    assert rel_l2(host(u_gpu), u_ref) < 1e-3
    assert abs(st["energy"] - h["E"][-1]) <= 1e-3 * abs(h["E"][-1])


def test_alg2_phi_variant_parity(nlos):
    n, nt, iters = 16, 64, 10
    cfg, g, mask, vol, tau0 = scene(2, n, nt, seed=6)
    op = lct.Operator(g, mask)
    n2, _ = lct.power_norm2(op, masked=False)
    plan = nlos.Plan(n, n, nt, cfg["bin_width_s"], mask=mask)
    p = alg2_params(nlos, cfg, iters, 2 * n2)
    p.phi = nlos.PHI_TAC
    u_gpu, tau_gpu, st = nlos.reconstruct_t(plan, p, dev(tau0), want_tau=True)
    u_ref, tau_ref, h = admm.alg2(tau0, mask, g, cfg["a_u"], cfg["b_u"], cfg["a_tau"], cfg["b_tau"], cfg["lam"],
                                  cfg["mu1"], cfg["mu2"], cfg["mu3"], iters, L0=2 * n2, op=op, phi_kind="tac")
    assert rel_l2(host(u_gpu), u_ref) < 1e-3 and rel_l2(host(tau_gpu), tau_ref) < 1e-3


@pytest.mark.parametrize("model", [1, 2])
def test_reconstruct_from_host_memory_equals_device_call(nlos, model):
    """nlos_reconstruct_host (tau0 from host memory, u and tau back to host
    memory, pageable and pinned buffers) gives the bits of nlos_reconstruct
    on device buffers, and the same statistics."""
    import torch
    n, nt = 32, 128
    cfg, g, mask, vol, tau0 = scene(model, n, nt, seed=4)
    plan = nlos.Plan(n, n, nt, cfg["bin_width_s"], mask=mask)
    p = alg1_params(nlos, cfg, 9, 0.0) if model == 1 else alg2_params(nlos, cfg, 9, 0.0)
    t = dev(tau0)
    u_dev, tau_dev = torch.empty_like(t), torch.empty_like(t)
    st_dev = plan.reconstruct(p, t.data_ptr(), u_dev.data_ptr(), tau_dev.data_ptr() if model == 2 else 0)
    t_host = np.ascontiguousarray(tau0, dtype=np.float32)
    for pinned in (False, True):
        if pinned:
            tin = torch.tensor(t_host).pin_memory()
            uo, to = torch.empty_like(tin).pin_memory(), torch.empty_like(tin).pin_memory()
            ptrs = (tin.data_ptr(), uo.data_ptr(), to.data_ptr())
            get = (lambda: (uo.numpy(), to.numpy()))
        else:
            uo_np, to_np = np.full_like(t_host, np.nan), np.full_like(t_host, np.nan)
            ptrs = (t_host.ctypes.data, uo_np.ctypes.data, to_np.ctypes.data)
            get = (lambda: (uo_np, to_np))
        st_host = plan.reconstruct_host(p, ptrs[0], ptrs[1], ptrs[2] if model == 2 else 0)
        u_h, tau_h = get()
        assert np.array_equal(u_h, host(u_dev).astype(np.float32))
        if model == 2:
            assert np.array_equal(tau_h, host(tau_dev).astype(np.float32))
        assert st_host["iters_done"] == st_dev["iters_done"] and st_host["energy"] == st_dev["energy"]
    plan.close()


@pytest.mark.parametrize("n,nt,mask_kind", [(16, 64, "stride"), (32, 256, "stride"), (32, 128, "random")])
def test_backprojection_start_against_oracle(nlos, n, nt, mask_kind):
    """NLOS_INIT_BACKPROJECT with no iterations returns u0 = s A_D^T tau0
    (the device-computed scale s = ||g||^2 / ||A_D g||^2), within the
    operator tolerance of the FP64 oracle."""
    cfg, g, mask, vol, tau0 = scene(1, n, nt, seed=3, mask_kind=mask_kind)
    op = lct.Operator(g, mask)
    plan = nlos.Plan(n, n, nt, cfg["bin_width_s"], mask=mask)
    p = alg1_params(nlos, cfg, 0, 1.0)
    p.init = nlos.INIT_BACKPROJECT
    u_gpu, st = nlos.reconstruct_t(plan, p, dev(tau0))
    u_ref, s_ref = admm.backprojection_init(op, tau0)
    assert s_ref > 0
    err = rel_l2(host(u_gpu), u_ref)
    assert err < 1e-5, err


@pytest.mark.parametrize("model,iters", [(1, 20), (2, 12)])
def test_reconstruction_from_backprojection_start(nlos, model, iters):
    """Algorithms 1 and 2 started from the back-projection against the
    oracle's runs from its own back-projection start."""
    n, nt = 16, 128
    cfg, g, mask, vol, tau0 = scene(model, n, nt, seed=6)
    op = lct.Operator(g, mask)
    n2, _ = lct.power_norm2(op, masked=model == 1)
    plan = nlos.Plan(n, n, nt, cfg["bin_width_s"], mask=mask)
    u0, _ = admm.backprojection_init(op, tau0)
    if model == 1:
        p = alg1_params(nlos, cfg, iters, 2 * n2)
        p.init = nlos.INIT_BACKPROJECT
        u_gpu, st = nlos.reconstruct_t(plan, p, dev(tau0))
        u_ref, h = admm.alg1(tau0, mask, g, cfg["a"], cfg["b"], cfg["mu"], iters, L0=2 * n2, op=op, u_init=u0)
    else:
        p = alg2_params(nlos, cfg, iters, 2 * n2)
        p.init = nlos.INIT_BACKPROJECT
        u_gpu, tau_gpu, st = nlos.reconstruct_t(plan, p, dev(tau0), want_tau=True)
        u_ref, tau_ref, h = admm.alg2(tau0, mask, g, cfg["a_u"], cfg["b_u"], cfg["a_tau"], cfg["b_tau"], cfg["lam"],
                                      cfg["mu1"], cfg["mu2"], cfg["mu3"], iters, L0=2 * n2, op=op, u_init=u0)
        assert rel_l2(host(tau_gpu), tau_ref) < 1e-3
        assert st["restarts"] == sum(h["restart"])
    assert st["status"] == 0 and st["iters_done"] == iters
    assert rel_l2(host(u_gpu), u_ref) < 1e-3
    assert abs(st["energy"] - h["E"][-1]) <= 1e-3 * abs(h["E"][-1])
    assert abs(st["rel_change"] - h["e"][-1]) <= 1e-2 * h["e"][-1] + 1e-9
