"""Full-size cases against stored FP64 oracle results (written by the
generators in tests/golden/ from oracle/ and synth/ only):

* precision case: Algorithm 1 on 128 x 128 x 1024 (8 ps bins, 32 x 32
  stride-4 sampling, 12 iterations);
* the benchmark's size: Algorithm 1 on 128 x 128 x 512 (16 ps bins, 32 x 32
  stride-4 sampling, 12 iterations), run as one graph launch like the bench;
* dual-domain case: Algorithm 2 on 64 x 64 x 512 (16 ps bins, 32 x 32
  stride-2 sampling, 100 iterations with adaptive restart);
* Algorithm 2 at the benchmark's size (128 x 128 x 512, 6 iterations), one
  graph launch.

Bar: 1e-3 relative L2 on the stored columns and on the global norms,
matching energy, and depth-map agreement (exact bin and within one bin).
Algorithm 2 also matches the restart pattern of the oracle."""
import os

import numpy as np
import pytest

import synth
from oracle import admm
from tests.gpu_util import dev, host, rel_l2

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "c4_alg1_128x128x1024.npz")


def test_c4_alg1_128x128x1024_against_oracle():
    from paper_2301_00406_gb300 import nlos
    z = np.load(GOLDEN)
    cfg = synth.CONFIGS["c4_alg1_128x128x1024"]
    nx, ny, nt = cfg["nx"], cfg["ny"], cfg["nt"]
    mask = synth.make_mask(cfg)
    tau0 = synth.pulse_transients(nx, ny, nt, mask, seed=0)
    plan = nlos.Plan(nx, ny, nt, cfg["bin_width_s"], mask=mask)
    p = nlos.params_default(1)
    p.a, p.b, p.mu, p.iters = cfg["a"], cfg["b"], cfg["mu"], int(z["iters"])
    u_dev, st = nlos.reconstruct_t(plan, p, dev(tau0))
    u = host(u_dev).astype(np.float64)
    cols_err = rel_l2(u.reshape(nx * ny, nt)[z["cols"]], z["u_cols"].astype(np.float64))
    norm_err = abs(np.linalg.norm(u) - float(z["norm"])) / float(z["norm"])
    e_err = abs(st["energy"] - float(z["energy"][-1])) / abs(float(z["energy"][-1]))
    d_gpu = admm.depth_map(u)
    d_ref = z["depth"].astype(np.int64)
    exact = float(np.mean(d_gpu == d_ref))
    near = float(np.mean(np.abs(d_gpu - d_ref) <= 1))
    print(f"c4: columns rel L2 {cols_err:.3e}, norm {norm_err:.3e}, energy {e_err:.3e}, "
          f"depth exact {exact:.4f}, within 1 bin {near:.4f}")
    assert st["iters_done"] == int(z["iters"]) and st["status"] == 0
    assert cols_err < 1e-3 and norm_err < 1e-3 and e_err < 1e-3
    assert exact >= 0.99 and near >= 0.999


GOLDEN_C2 = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "c2_alg2_64x64x512.npz")


def test_c2_alg2_64x64x512_against_oracle():
    from paper_2301_00406_gb300 import nlos
    z = np.load(GOLDEN_C2)
    cfg = synth.CONFIGS["c2_alg2_64x64x512"]
    nx, ny, nt = cfg["nx"], cfg["ny"], cfg["nt"]
    mask = synth.make_mask(cfg)
    tau0 = synth.pulse_transients(nx, ny, nt, mask, seed=1)
    plan = nlos.Plan(nx, ny, nt, cfg["bin_width_s"], mask=mask)
    p = nlos.params_default(2)
    p.a_u, p.b_u, p.a_tau, p.b_tau = cfg["a_u"], cfg["b_u"], cfg["a_tau"], cfg["b_tau"]
    p.lambda_, p.mu1, p.mu2, p.mu3 = cfg["lam"], cfg["mu1"], cfg["mu2"], cfg["mu3"]
    p.iters = int(z["iters"])
    u_dev, tau_dev, st = nlos.reconstruct_t(plan, p, dev(tau0), want_tau=True)
    u, tau = host(u_dev).astype(np.float64), host(tau_dev).astype(np.float64)
    cols = z["cols"]
    eu = rel_l2(u.reshape(nx * ny, nt)[cols], z["u_cols"].astype(np.float64))
    et = rel_l2(tau.reshape(nx * ny, nt)[cols], z["tau_cols"].astype(np.float64))
    nu = abs(np.linalg.norm(u) - float(z["norm_u"])) / float(z["norm_u"])
    ntau = abs(np.linalg.norm(tau) - float(z["norm_tau"])) / float(z["norm_tau"])
    e_err = abs(st["energy"] - float(z["energy"][-1])) / abs(float(z["energy"][-1]))
    l_err = abs(st["L"] - float(z["L"][-1])) / float(z["L"][-1])
    d_gpu, d_ref = admm.depth_map(u), z["depth"].astype(np.int64)
    exact = float(np.mean(d_gpu == d_ref))
    near = float(np.mean(np.abs(d_gpu - d_ref) <= 1))
    print(f"c2: u columns {eu:.3e}, tau columns {et:.3e}, norms {nu:.3e} {ntau:.3e}, energy {e_err:.3e}, "
          f"L {l_err:.3e}, restarts {st['restarts']} vs {int(z['restart'].sum())}, "
          f"depth exact {exact:.4f}, within 1 bin {near:.4f}")
    assert st["iters_done"] == int(z["iters"]) and st["status"] == 0
    assert eu < 1e-3 and et < 1e-3 and nu < 1e-3 and ntau < 1e-3
    assert e_err < 1e-3 and l_err < 1e-3
    assert st["restarts"] == int(z["restart"].sum())
    assert exact >= 0.99 and near >= 0.999


GOLDEN_HEAD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "headline_alg1_128x128x512.npz")


def test_headline_alg1_128x128x512_against_oracle():
    from paper_2301_00406_gb300 import nlos
    z = np.load(GOLDEN_HEAD)
    cfg = synth.CONFIGS["headline_128x128x512"]
    nx, ny, nt = cfg["nx"], cfg["ny"], cfg["nt"]
    mask = synth.make_mask(cfg)
    tau0 = synth.pulse_transients(nx, ny, nt, mask, seed=int(z["seed"]))
    plan = nlos.Plan(nx, ny, nt, cfg["bin_width_s"], mask=mask)
    p = nlos.params_default(1)
    p.a, p.b, p.mu, p.iters = cfg["a"], cfg["b"], cfg["mu"], int(z["iters"])
    t = dev(tau0)
    u_dev = t.new_empty(t.shape)
    assert plan.reconstruct_prepare(p, t.data_ptr(), u_dev.data_ptr()) is True   # one graph launch
    st = plan.reconstruct(p, t.data_ptr(), u_dev.data_ptr())
    u = host(u_dev).astype(np.float64)
    cols_err = rel_l2(u.reshape(nx * ny, nt)[z["cols"]], z["u_cols"].astype(np.float64))
    norm_err = abs(np.linalg.norm(u) - float(z["norm"])) / float(z["norm"])
    e_err = abs(st["energy"] - float(z["energy"][-1])) / abs(float(z["energy"][-1]))
    d_gpu, d_ref = admm.depth_map(u), z["depth"].astype(np.int64)
    exact = float(np.mean(d_gpu == d_ref))
    near = float(np.mean(np.abs(d_gpu - d_ref) <= 1))
    print(f"headline: columns rel L2 {cols_err:.3e}, norm {norm_err:.3e}, energy {e_err:.3e}, "
          f"depth exact {exact:.4f}, within 1 bin {near:.4f}")
    assert st["iters_done"] == int(z["iters"]) and st["status"] == 0
    assert cols_err < 1e-3 and norm_err < 1e-3 and e_err < 1e-3
    assert exact >= 0.99 and near >= 0.999


GOLDEN_HEAD2 = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "headline_alg2_128x128x512.npz")


def test_headline_alg2_128x128x512_against_oracle():
    """Algorithm 2 at the benchmark's size, as one graph launch, against the
    stored FP64 oracle run (u and tau on fixed columns, norms, energy, L,
    restarts, depth map)."""
    import torch
    from paper_2301_00406_gb300 import nlos
    z = np.load(GOLDEN_HEAD2)
    cfg = synth.CONFIGS["headline_128x128x512"]
    nx, ny, nt = cfg["nx"], cfg["ny"], cfg["nt"]
    mask = synth.make_mask(cfg)
    tau0 = synth.pulse_transients(nx, ny, nt, mask, seed=int(z["seed"]))
    plan = nlos.Plan(nx, ny, nt, cfg["bin_width_s"], mask=mask)
    p = nlos.params_default(2)
    p.a_u, p.b_u, p.a_tau, p.b_tau = cfg["a_u"], cfg["b_u"], cfg["a_tau"], cfg["b_tau"]
    p.lambda_, p.mu1, p.mu2, p.mu3 = cfg["lam"], cfg["mu1"], cfg["mu2"], cfg["mu3"]
    p.iters = int(z["iters"])
    t = dev(tau0)
    u_dev, tau_dev = torch.empty_like(t), torch.empty_like(t)
    assert plan.reconstruct_prepare(p, t.data_ptr(), u_dev.data_ptr(), tau_dev.data_ptr()) is True
    st = plan.reconstruct(p, t.data_ptr(), u_dev.data_ptr(), tau_dev.data_ptr())
    u, tau = host(u_dev).astype(np.float64), host(tau_dev).astype(np.float64)
    cols = z["cols"]
    eu = rel_l2(u.reshape(nx * ny, nt)[cols], z["u_cols"].astype(np.float64))
    et = rel_l2(tau.reshape(nx * ny, nt)[cols], z["tau_cols"].astype(np.float64))
    nu = abs(np.linalg.norm(u) - float(z["norm_u"])) / float(z["norm_u"])
    ntau = abs(np.linalg.norm(tau) - float(z["norm_tau"])) / float(z["norm_tau"])
    e_err = abs(st["energy"] - float(z["energy"][-1])) / abs(float(z["energy"][-1]))
    l_err = abs(st["L"] - float(z["L"][-1])) / float(z["L"][-1])
    d_gpu, d_ref = admm.depth_map(u), z["depth"].astype(np.int64)
    exact = float(np.mean(d_gpu == d_ref))
    near = float(np.mean(np.abs(d_gpu - d_ref) <= 1))
    print(f"headline alg2: u columns {eu:.3e}, tau columns {et:.3e}, norms {nu:.3e} {ntau:.3e}, "
          f"energy {e_err:.3e}, L {l_err:.3e}, restarts {st['restarts']} vs {int(z['restart'].sum())}, "
          f"depth exact {exact:.4f}, within 1 bin {near:.4f}")
    assert st["iters_done"] == int(z["iters"]) and st["status"] == 0
    assert eu < 1e-3 and et < 1e-3 and nu < 1e-3 and ntau < 1e-3
    assert e_err < 1e-3 and l_err < 1e-3
    assert st["restarts"] == int(z["restart"].sum())
    assert exact >= 0.99 and near >= 0.999
