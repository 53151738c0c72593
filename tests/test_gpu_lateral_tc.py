"""The tensor-core lateral stage (nlos_plan_set_lateral): the H convolution
of every kt plane as DFT-matrix products with tcgen05.mma, split-BF16
(mode 1) or single-pass BF16 (mode 2), against the FP64 oracle.

* Operator parity: A, A_D, A^T, A_D^T on random inputs at 128 x 128 lateral
  size (the size the stage supports), nt = 64 and 512; mode 1 within the
  1e-5 bar of the FP32 kernels, mode 2 within 1e-2 (one BF16 rounding per
  operand and four chained products).
* Repeat launches give identical bits (fixed accumulation order), and no
  MMA completion wait gave up.
* Sizes other than 128 are refused.
* The precision case (128 x 128 x 1024, 12 Algorithm-1 iterations) against
  the stored FP64 oracle run, with the relative L2 and the depth-map
  agreement of each mode printed: the comparison between the FP32 lateral
  stage and the split-BF16 tensor-core one."""
import os

import numpy as np
import pytest

import synth
from oracle import admm, lct
from tests.gpu_util import dev, host, rel_l2

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "c4_alg1_128x128x1024.npz")
TOL = {1: 1e-5, 2: 1e-2}


@pytest.fixture(scope="module")
def nlos():
    from paper_2301_00406_gb300 import nlos as mod
    mod.load()
    return mod


@pytest.mark.parametrize("mode", [1, 2])
@pytest.mark.parametrize("nt,stride", [(64, 4), (512, 4), (64, 3)])
def test_tc_lateral_operator_parity(nlos, mode, nt, stride):
    n = 128
    bw = 32e-12 * 256 / nt
    g = lct.Geometry(n, n, nt, bw)
    mask = synth.stride_mask(n, n, stride)
    plan = nlos.Plan(n, n, nt, bw, mask=mask)
    plan.set_lateral(mode)
    op = lct.Operator(g, mask)
    rng = np.random.default_rng(n + nt + mode + stride)
    u, r = rng.random(g.shape), rng.standard_normal(g.shape)
    outs = [host(nlos.forward_t(plan, dev(u), apply_mask=False)), host(nlos.forward_t(plan, dev(u), apply_mask=True)),
            host(nlos.adjoint_t(plan, dev(r), apply_mask=False)), host(nlos.adjoint_t(plan, dev(r), apply_mask=True))]
    errs = [rel_l2(outs[0], op.forward(u)), rel_l2(outs[1], op.forward_d(u)),
            rel_l2(outs[2], op.adjoint(r)), rel_l2(outs[3], op.adjoint_d(r))]
    print(f"mode {mode} nt {nt} stride {stride}: A {errs[0]:.2e}, A_D {errs[1]:.2e}, A^T {errs[2]:.2e}, "
          f"A_D^T {errs[3]:.2e}")
    assert max(errs) < TOL[mode], errs
    # unsampled columns of A_D u are exactly zero
    m = np.asarray(mask, dtype=bool)
    assert np.all(outs[1][~m] == 0)
    # identical bits on a second launch
    again = host(nlos.adjoint_t(plan, dev(r), apply_mask=True))
    assert np.array_equal(again, outs[3])
    plan.set_lateral(mode)                                # raises if a wait gave up
    plan.set_lateral(0)                                   # back to the FFT kernels
    assert rel_l2(host(nlos.forward_t(plan, dev(u), apply_mask=False)), op.forward(u)) < 1e-5


def test_tc_lateral_refuses_other_sizes(nlos):
    plan = nlos.Plan(64, 64, 64, 64e-12)
    with pytest.raises(nlos.NlosError):
        plan.set_lateral(1)
    plan.set_lateral(0)


def test_tc_lateral_precision_case(nlos):
    z = np.load(GOLDEN)
    cfg = synth.CONFIGS["c4_alg1_128x128x1024"]
    nx, ny, nt = cfg["nx"], cfg["ny"], cfg["nt"]
    mask = synth.make_mask(cfg)
    tau0 = synth.pulse_transients(nx, ny, nt, mask, seed=0)
    plan = nlos.Plan(nx, ny, nt, cfg["bin_width_s"], mask=mask)
    p = nlos.params_default(1)
    p.a, p.b, p.mu, p.iters = cfg["a"], cfg["b"], cfg["mu"], int(z["iters"])
    d_ref = z["depth"].astype(np.int64)
    res = {}
    for mode in (0, 1, 2):
        plan.set_lateral(mode)
        u_dev, st = nlos.reconstruct_t(plan, p, dev(tau0))
        u = host(u_dev).astype(np.float64)
        cols = rel_l2(u.reshape(nx * ny, nt)[z["cols"]], z["u_cols"].astype(np.float64))
        d = admm.depth_map(u)
        res[mode] = (cols, float(np.mean(d == d_ref)), float(np.mean(np.abs(d - d_ref) <= 1)), st)
        print(f"precision case, lateral mode {mode}: columns rel L2 {cols:.3e}, depth exact {res[mode][1]:.4f}, "
              f"within 1 bin {res[mode][2]:.4f}")
    plan.set_lateral(0)
    assert all(r[3]["status"] == 0 for r in res.values())
    assert res[0][0] < 1e-3 and res[1][0] < 1e-3
    assert res[1][1] >= 0.99 and res[2][2] >= 0.99
    assert res[2][0] < 5e-2
