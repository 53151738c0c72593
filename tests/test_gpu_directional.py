"""The directional (normal-weighted) confocal model of Sec. 2
(nlos_forward_directional / nlos_adjoint_directional) against the FP64
oracle: operator parity at 1e-5 relative L2 with and without the sampling
mask, on random normal fields and on a planar scatterer with one tilted
normal; the transpose through the dot-product identity on the GPU path;
overlapping input and output refused."""

import numpy as np
import pytest

import synth
from oracle import lct
from tests.gpu_util import dev, host, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nlos():
    from paper_2301_00406_gb300 import nlos as mod
    mod.load()
    return mod


def normals_of(shape, seed):
    rng = np.random.default_rng(seed)
    v = rng.standard_normal((3,) + shape)
    v[2] = -np.abs(v[2]) - 0.5
    return v / np.sqrt(np.sum(v * v, axis=0))


@pytest.mark.parametrize("n,nt,stride", [(16, 64, 2), (32, 128, 4), (128, 256, 4)])
def test_directional_operator_parity(nlos, n, nt, stride):
    bw = 32e-12 * 256 / nt
    g = lct.Geometry(n, n, nt, bw)
    mask = synth.stride_mask(n, n, stride)
    op = lct.Operator(g, mask)
    plan = nlos.Plan(n, n, nt, bw, mask=mask)
    normals = normals_of(g.shape, n + nt)
    rng = np.random.default_rng(n)
    u, r = rng.random(g.shape), rng.standard_normal(g.shape)
    dn = dev(normals)
    for masked in (False, True):
        t_gpu = host(nlos.forward_directional_t(plan, dev(u), dn, apply_mask=masked))
        t_ref = lct.directional_forward(op, u, normals, masked=masked)
        u_gpu = host(nlos.adjoint_directional_t(plan, dev(r), dn, apply_mask=masked))
        u_ref = lct.directional_adjoint(op, r, normals, masked=masked)
        ef, ea = rel_l2(t_gpu, t_ref), rel_l2(u_gpu, u_ref)
        print(f"n {n} nt {nt} masked {masked}: forward {ef:.2e}, adjoint {ea:.2e}")
        assert ef < 1e-5 and ea < 1e-5
        if masked:
            assert np.all(t_gpu[~np.asarray(mask, dtype=bool)] == 0)
    # transpose on the GPU path itself
    x, y = dev(u), dev(r)
    fx = nlos.forward_directional_t(plan, x, dn, apply_mask=True)
    aty = nlos.adjoint_directional_t(plan, y, dn, apply_mask=True)
    lhs, rhs = float((fx.double() * y.double()).sum()), float((x.double() * aty.double()).sum())
    assert abs(lhs - rhs) <= 1e-5 * float(fx.double().norm() * y.double().norm())
    plan.close()


def test_directional_tilted_plane(nlos):
    n, nt = 32, 128
    g = lct.Geometry(n, n, nt, 64e-12)
    op = lct.Operator(g)
    plan = nlos.Plan(n, n, nt, 64e-12)
    u = np.zeros(g.shape)
    u[6:26, 4:24, 80] = 1.0
    nrm = np.stack([np.full(g.shape, 0.45), np.full(g.shape, 0.45), np.full(g.shape, -np.sqrt(1 - 2 * 0.45 ** 2))])
    t_gpu = host(nlos.forward_directional_t(plan, dev(u), dev(nrm)))
    assert rel_l2(t_gpu, lct.directional_forward(op, u, nrm, masked=False)) < 1e-5
    # the tilt moves the measured intensity across the wall relative to the albedo model
    t_alb = host(nlos.forward_t(plan, dev(u)))
    ratio = t_gpu.sum(2) / np.maximum(t_alb.sum(2), 1e-30)
    live = t_alb.sum(2) > 1e-6 * t_alb.sum()
    assert (ratio[live].max() - ratio[live].min()) / ratio[live].mean() > 0.05


def test_directional_rejects_overlap(nlos):
    import torch
    plan = nlos.Plan(16, 16, 64, 128e-12)
    u = torch.zeros((16, 16, 64), device="cuda")
    nrm = torch.zeros((3, 16, 16, 64), device="cuda")
    with pytest.raises(nlos.NlosError):
        nlos.check(nlos.load().nlos_forward_directional(plan.handle, u.data_ptr(), nrm.data_ptr(), u.data_ptr(), 0, 0))
