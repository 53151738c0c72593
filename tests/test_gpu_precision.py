"""Precision case: Algorithm 1 on 128 x 128 x 1024 (8 ps bins, 32 x 32
stride-4 sampling), FP32 GPU against the FP64 oracle's stored result
(tests/golden/c4_alg1_128x128x1024.npz, written by make_c4_alg1.py from
oracle/ and synth/ only): 1e-3 relative L2 on the stored columns and on the
global norm, matching energy, and the depth-map agreement (exact bin and
within one bin)."""
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
