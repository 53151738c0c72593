"""GPU parity of the operator passes (through the C ABI) against the FP64
oracle: A, A_D, A^T, A_D^T, the FFT solve of Eq. 11 and phi(kappa(u)).
Tolerance: 1e-5 relative L2 per operator application (FP32 arithmetic)."""

import numpy as np
import pytest

import synth
from oracle import admm, lct
from tests.gpu_util import dev, host, rel_l2

pytestmark = pytest.mark.gpu
TOL = 1e-5


@pytest.fixture(scope="module")
def nlos():
    from paper_2301_00406_gb300 import nlos as mod
    mod.load()
    return mod


CASES = [
    (8, 16, "compensated", None),
    (16, 64, "compensated", "stride2"),
    (16, 64, "raw", "stride2"),
    (32, 256, "compensated", "stride2"),
    (16, 1024, "compensated", "random"),   # nt = 1024 path (8 columns per CTA)
    (32, 128, "compensated", "ragged"),    # sampled count not a multiple of 16
    (64, 512, "compensated", "stride2"),
    (64, 256, "compensated", "random"),    # four-CTA lateral pass, scattered sampled rows
    (128, 64, "compensated", "ragged"),    # four-CTA lateral pass at N = 128, ragged sample list
    # sampled rows on one residue class mod 4 (x passes folded to the lattice)
    (128, 64, "compensated", "lattice4_0"),
    (128, 32, "raw", "lattice4_3"),
    (128, 64, "compensated", "rows1mod4"),  # rows x = 1 mod 4, scattered y, some rows empty
]


def make_mask(n, kind, seed=3):
    if kind is None:
        return None
    if kind == "stride2":
        return synth.stride_mask(n, n, 2)
    if kind == "random":
        return synth.random_mask(n, n, 0.25, seed)
    if kind.startswith("lattice4_"):
        r = int(kind[-1])
        m = np.zeros((n, n), np.uint8)
        m[r::4, (r + 1) % 4::4] = 1
        return m
    if kind == "rows1mod4":
        m = np.zeros((n, n), np.uint8)
        rng = np.random.default_rng(seed)
        for x in range(1, n - 8, 4):
            m[x, rng.permutation(n)[:rng.integers(1, 9)]] = 1
        return m
    if kind == "ragged":
        m = np.zeros(n * n, np.uint8)
        m[np.random.default_rng(seed).permutation(n * n)[:37]] = 1
        return m.reshape(n, n)
    raise ValueError(kind)


def setup(nlos, n, nt, rad, mk):
    bw = 32e-12 * 256 / nt
    g = lct.Geometry(n, n, nt, bw, radiometry=rad)
    mask = make_mask(n, mk)
    plan = nlos.Plan(n, n, nt, bw, radiometry=rad, mask=mask)
    op = lct.Operator(g, mask)
    return g, mask, plan, op


@pytest.mark.parametrize("n,nt,rad,mk", CASES)
def test_forward_parity(nlos, n, nt, rad, mk):
    g, mask, plan, op = setup(nlos, n, nt, rad, mk)
    rng = np.random.default_rng(n + nt)
    u = rng.random(g.shape)
    got = host(nlos.forward_t(plan, dev(u), apply_mask=False))
    assert rel_l2(got, op.forward(u)) < TOL
    got = host(nlos.forward_t(plan, dev(u), apply_mask=True))
    want = op.forward_d(u)
    assert rel_l2(got, want) < TOL
    if mask is not None:
        assert np.all(got[mask == 0] == 0.0)


@pytest.mark.parametrize("n,nt,rad,mk", CASES)
def test_adjoint_parity(nlos, n, nt, rad, mk):
    g, mask, plan, op = setup(nlos, n, nt, rad, mk)
    rng = np.random.default_rng(n * nt)
    r = rng.standard_normal(g.shape)
    got = host(nlos.adjoint_t(plan, dev(r), apply_mask=False))
    assert rel_l2(got, op.adjoint(r)) < TOL
    got = host(nlos.adjoint_t(plan, dev(r), apply_mask=True))
    assert rel_l2(got, op.adjoint_d(r)) < TOL


@pytest.mark.parametrize("n,nt", [(16, 64), (32, 256)])
def test_gpu_adjoint_identity(nlos, n, nt):
    g, mask, plan, op = setup(nlos, n, nt, "compensated", "stride2")
    rng = np.random.default_rng(11)
    x, y = rng.standard_normal(g.shape), rng.standard_normal(g.shape)
    ax = host(nlos.forward_t(plan, dev(x), apply_mask=True))
    aty = host(nlos.adjoint_t(plan, dev(y), apply_mask=True))
    lhs, rhs = np.sum(ax * y), np.sum(x * aty)
    assert abs(lhs - rhs) <= 1e-5 * np.linalg.norm(ax) * np.linalg.norm(y)


@pytest.mark.parametrize("n,nt,c0,c1", [(8, 16, 1.0, 0.1), (32, 256, 93.4, 0.1), (64, 512, 3.0, 800.0),
                                        (16, 1024, 2.0, 1.0), (128, 64, 5.0, 3.0)])
def test_solve_parity(nlos, n, nt, c0, c1):
    plan = nlos.Plan(n, n, nt, 16e-12)
    rhs = np.random.default_rng(5).standard_normal((n, n, nt))
    got = host(nlos.solve_t(plan, dev(rhs), c0, c1))
    assert rel_l2(got, admm.fft_solve(rhs, c0, c1)) < TOL


@pytest.mark.parametrize("kind", ["tsc", "tac", "trv"])
def test_curvature_weight_parity(nlos, kind):
    n, nt = 32, 64
    plan = nlos.Plan(n, n, nt, 16e-12)
    vol = synth.scene_planes_glyph(n, n, nt, 2)
    u = vol + 0.05 * np.random.default_rng(2).standard_normal(vol.shape)
    a, b, eps = 1e-4, 3e-2, 1e-3
    got = host(nlos.curvature_weight_t(plan, dev(u), a, b, kind, eps))
    want = admm.phi(admm.curvature(u.astype(np.float32).astype(np.float64), eps), a, b, kind)
    assert rel_l2(got, want) < TOL


def test_norm2_matches_oracle(nlos):
    g, mask, plan, op = setup(nlos, 16, 64, "compensated", "stride2")
    want, _ = lct.power_norm2(op)
    got = plan.norm2(True)
    assert abs(got - want) <= 1e-4 * want
    want_full, _ = lct.power_norm2(lct.Operator(g), masked=False)
    assert abs(plan.norm2(False) - want_full) <= 1e-4 * want_full


def test_forward_full_size_sampled_columns(nlos):
    # 128 x 128 x 512 (the headline geometry): the whole volume against the oracle
    n, nt, bw = 128, 512, 16e-12
    g = lct.Geometry(n, n, nt, bw)
    mask = synth.stride_mask(n, n, 4)
    plan = nlos.Plan(n, n, nt, bw, mask=mask)
    vol = synth.scene_patches(n, n, nt, 0)
    got = host(nlos.forward_t(plan, dev(vol), apply_mask=True))
    want = lct.Operator(g, mask).forward_d(vol)
    assert rel_l2(got, want) < TOL


def test_adjoint_full_size_sampled_columns(nlos):
    # 128 x 128 x 512: A_D^T of a measurement on the 32 x 32 sampled grid
    n, nt, bw = 128, 512, 16e-12
    g = lct.Geometry(n, n, nt, bw)
    mask = synth.stride_mask(n, n, 4)
    plan = nlos.Plan(n, n, nt, bw, mask=mask)
    rng = np.random.default_rng(11)
    tau = (rng.random((n, n, nt)) * mask[:, :, None]).astype(np.float32)
    got = host(nlos.adjoint_t(plan, dev(tau), apply_mask=True))
    want = lct.Operator(g, mask).adjoint_d(tau.astype(np.float64))
    assert rel_l2(got, want) < TOL


def test_invalid_arguments(nlos):
    import torch
    plan = nlos.Plan(8, 8, 16, 16e-12)
    u = torch.zeros(8 * 8 * 16 + 1, device="cuda")
    with pytest.raises(nlos.NlosError):
        plan.forward(u.data_ptr() + 4, u.data_ptr(), 0)   # misaligned
    with pytest.raises(nlos.NlosError):
        plan.forward(0, u.data_ptr(), 0)
    with pytest.raises(nlos.NlosError):
        plan.solve(u.data_ptr(), u.data_ptr(), 0.0, 1.0)
