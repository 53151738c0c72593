"""nlos_midpoint_confocal (the midpoint conversion of non-confocal transients,
Sec. 4) against the FP64 oracle: random inputs on several grids and laser
points, the warp itself through a ramp input, the benchmark's size, and
argument checks."""

import numpy as np
import pytest

from oracle import nonconfocal as nc
from tests.gpu_util import dev, host, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nlos():
    from paper_2301_00406_gb300 import nlos as mod
    mod.load()
    return mod


CASES = [
    (8, 8, 64, 32e-12, 1.0, (0.0, 0.0)),
    (16, 32, 256, 32e-12, 1.0, (0.13, -0.41)),      # nx != ny, laser off the grid
    (32, 32, 1024, 8e-12, 0.512, (0.9, 0.7)),        # laser outside the patch: long offsets
    (64, 64, 512, 16e-12, 1.0, (-0.2, 0.35)),
]


@pytest.mark.parametrize("nx,ny,nt,bw,W,laser", CASES)
def test_midpoint_parity(nlos, nx, ny, nt, bw, W, laser):
    rng = np.random.default_rng(nx + nt)
    tau = rng.random((nx, ny, nt)).astype(np.float32)
    out = host(nlos.midpoint_confocal_t(dev(tau), bw, W, laser)).astype(np.float64)
    ref = nc.midpoint_confocal(tau.astype(np.float64), bw, W, laser)
    err = rel_l2(out, ref)
    print(f"midpoint {nx}x{ny}x{nt}: rel L2 {err:.2e}, max abs {np.abs(out - ref).max():.2e}")
    assert err < 1e-6 and np.abs(out - ref).max() < 1e-5


@pytest.mark.parametrize("nx,ny,nt,bw,W,laser", CASES[1:3])
def test_midpoint_warp_positions(nlos, nx, ny, nt, bw, W, laser):
    # a ramp tau_nc[..., k] = k converts to the source position p itself
    # where p <= nt - 1: the FP64 positions and their tap split, seen in FP32
    tau = np.broadcast_to(np.arange(nt, dtype=np.float32), (nx, ny, nt)).copy()
    out = host(nlos.midpoint_confocal_t(dev(tau), bw, W, laser)).astype(np.float64)
    p = nc.midpoint_positions(nx, ny, nt, bw, W, laser)
    inside = p <= nt - 1
    assert np.all(np.abs(out[inside] - p[inside]) <= 4e-7 * np.maximum(p[inside], 1.0))
    beyond = p >= nt
    assert np.all(out[beyond] == 0.0)


def test_midpoint_benchmark_size(nlos):
    import torch
    nx = ny = 128
    nt, bw, W, laser = 512, 16e-12, 1.0, (0.25, -0.15)
    rng = np.random.default_rng(5)
    tau = rng.random((nx, ny, nt)).astype(np.float32)
    t = dev(tau)
    out = torch.empty_like(t)
    st = torch.cuda.current_stream().cuda_stream
    for _ in range(3):
        nlos.midpoint_confocal(nx, ny, nt, bw, W, laser, t.data_ptr(), out.data_ptr(), st)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(10):
        nlos.midpoint_confocal(nx, ny, nt, bw, W, laser, t.data_ptr(), out.data_ptr(), st)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / 10
    ref = nc.midpoint_confocal(tau.astype(np.float64), bw, W, laser)
    err = rel_l2(host(out).astype(np.float64), ref)
    print(f"midpoint 128x128x512: {ms:.3f} ms per conversion ({2 * tau.nbytes / ms / 1e6:.0f} GB/s), rel L2 {err:.2e}")
    assert err < 1e-6


def test_midpoint_rejects_bad_arguments(nlos):
    import torch
    t = torch.zeros((8, 8, 64), device="cuda")
    o = torch.zeros_like(t)
    with pytest.raises(nlos.NlosError):
        nlos.midpoint_confocal(8, 8, 60, 32e-12, 1.0, (0, 0), t.data_ptr(), o.data_ptr())   # nt not a power of 2
    with pytest.raises(nlos.NlosError):
        nlos.midpoint_confocal(8, 8, 64, -1.0, 1.0, (0, 0), t.data_ptr(), o.data_ptr())    # bin width
    with pytest.raises(nlos.NlosError):
        nlos.midpoint_confocal(8, 8, 64, 32e-12, 1.0, (0, 0), t.data_ptr(), t.data_ptr())  # in place
    with pytest.raises(nlos.NlosError):
        nlos.midpoint_confocal(8, 8, 64, 32e-12, 1.0, (float("nan"), 0), t.data_ptr(), o.data_ptr())


def test_point_scatterer_through_conversion_and_reconstruction(nlos):
    """Non-confocal transients of a point scatterer below the midpoint of
    detector (i0, j0) and the laser (a one-bin pulse at the time of the path
    laser -> scatterer -> detector, for every detector), converted on the GPU
    and reconstructed with Algorithm 1 on the midpoint grid (wall width W/2):
    the reconstruction's maximum lies at column (i0, j0) and at the
    scatterer's depth bin."""
    from oracle.lct import C_LIGHT
    nx = ny = 32
    nt, bw, W = 256, 32e-12, 1.0
    laser = np.array([0.1, -0.05])
    i0, j0, kz = 19, 11, 140
    x = nc.detector_centres(nx, W)
    m = (laser + np.array([x[i0], x[j0]])) / 2
    R = C_LIGHT * nt * bw / 2
    z = (kz + 0.5) / nt * R                                # depth bin centre kz
    xp = np.array([m[0], m[1], z])
    tau = np.zeros((nx, ny, nt))
    k = np.arange(nt)
    for i in range(nx):
        for j in range(ny):
            s = np.array([x[i], x[j], 0.0])
            path = np.linalg.norm(xp - np.array([laser[0], laser[1], 0.0])) + np.linalg.norm(xp - s)
            c = path / (C_LIGHT * bw) - 0.5
            tau[i, j] = np.maximum(0.0, 1.0 - np.abs(k - c))
    conf = nlos.midpoint_confocal_t(dev(tau), bw, W, laser)
    conf_h = host(conf)
    assert int(np.argmax(conf_h[i0, j0])) == kz            # exact below the midpoint
    plan = nlos.Plan(nx, ny, nt, bw, wall_width_m=W / 2)
    p = nlos.params_default(1)
    p.iters = 30
    u_dev, st = nlos.reconstruct_t(plan, p, conf / float(conf_h.max()))
    u = host(u_dev)
    assert st["status"] == 0
    flat = int(np.argmax(u))
    ui, uj, uk = np.unravel_index(flat, u.shape)
    print(f"converted point scatterer: reconstruction peak at ({ui}, {uj}, {uk}), expected ({i0}, {j0}, {kz})")
    assert abs(ui - i0) <= 1 and abs(uj - j0) <= 1 and abs(uk - kz) <= 2
