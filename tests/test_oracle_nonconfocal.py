"""Pins of the FP64 midpoint conversion (oracle/nonconfocal.py) against the
path-length geometry of the non-confocal setting, special cases and
invariants -- no GPU, no CUDA library."""

import numpy as np
import pytest

from oracle import nonconfocal as nc
from oracle.lct import C_LIGHT


def test_zero_offset_column_is_identity():
    # laser on the centre of detector (3, 5): that column needs no warp
    nx, ny, nt, W, bw = 8, 8, 64, 1.0, 32e-12
    x = nc.detector_centres(nx, W)
    laser = (x[3], x[5])
    rng = np.random.default_rng(0)
    tau = rng.random((nx, ny, nt))
    out = nc.midpoint_confocal(tau, bw, W, laser)
    assert np.allclose(out[3, 5], tau[3, 5], rtol=0, atol=1e-12)
    # every other column is shifted to later non-confocal times
    p = nc.midpoint_positions(nx, ny, nt, bw, W, laser)
    k = np.arange(nt)
    assert np.allclose(p[3, 5], k, rtol=0, atol=1e-9)
    off = np.ones((nx, ny), bool)
    off[3, 5] = False
    assert np.all(p[off] > k[None, :] + 1e-6)


@pytest.mark.parametrize("i,j,laser,kc", [(0, 0, (0.0, 0.0), 100), (7, 2, (0.31, -0.2), 37),
                                          (4, 6, (-0.45, 0.45), 250)])
def test_scatterer_below_midpoint_reads_its_path_length(i, j, laser, kc):
    # A scatterer on the wall normal through the midpoint m of detector s and
    # laser l, at the depth whose confocal arrival time is bin centre kc:
    # confocal bin kc must read the non-confocal record at the time of the
    # path l -> scatterer -> s, from explicit 3-D distances.
    nx, ny, nt, W, bw = 8, 8, 512, 1.0, 16e-12
    x = nc.detector_centres(nx, W)
    s = np.array([x[i], x[j], 0.0])
    lpt = np.array([laser[0], laser[1], 0.0])
    m = (s + lpt) / 2
    z = C_LIGHT * (kc + 0.5) * bw / 2                  # 2 z / c = t_kc
    xp = m + np.array([0.0, 0.0, z])
    t_nc = (np.linalg.norm(xp - lpt) + np.linalg.norm(xp - s)) / C_LIGHT
    p = nc.midpoint_positions(nx, ny, nt, bw, W, laser)
    assert abs(p[i, j, kc] - (t_nc / bw - 0.5)) < 1e-9
    # a one-bin pulse at that time converts to a pulse peaking at bin kc
    tau = np.zeros((nx, ny, nt))
    c = t_nc / bw - 0.5
    tau[i, j] = np.maximum(0.0, 1.0 - np.abs(np.arange(nt) - c))
    out = nc.midpoint_confocal(tau, bw, W, laser)
    assert int(np.argmax(out[i, j])) == kc


def test_warp_is_causal_monotone_and_shrinks_with_depth():
    nx, ny, nt, W, bw = 16, 16, 256, 1.0, 32e-12
    p = nc.midpoint_positions(nx, ny, nt, bw, W, (0.2, -0.1))
    k = np.arange(nt)
    assert np.all(p >= k - 1e-12)                      # never reads earlier times
    assert np.all(np.diff(p, axis=2) > 0)              # order of arrivals kept
    d = p - k
    assert np.all(np.diff(d, axis=2) < 1e-12)          # the offset shrinks with depth
    # dp/dk = t_k / t_nc <= 1: the warp compresses, never stretches
    assert np.all(np.diff(p, axis=2) <= 1 + 1e-12)


def test_reads_past_the_record_are_zero_and_conversion_is_linear():
    nx, ny, nt, W, bw = 4, 4, 32, 2.0, 64e-12
    laser = (0.9, 0.9)
    rng = np.random.default_rng(1)
    a, b = rng.random((nx, ny, nt)), rng.standard_normal((nx, ny, nt))
    conv = lambda t: nc.midpoint_confocal(t, bw, W, laser)  # noqa: E731
    assert np.allclose(conv(2.0 * a - 3.0 * b), 2.0 * conv(a) - 3.0 * conv(b), rtol=0, atol=1e-12)
    p = nc.midpoint_positions(nx, ny, nt, bw, W, laser)
    out = conv(np.ones((nx, ny, nt)))
    assert np.all(out[p >= nt] == 0.0)                  # beyond the last bin: no data
    inside = p <= nt - 1
    assert np.allclose(out[inside], 1.0, rtol=0, atol=1e-12)


def test_midpoints_form_a_half_width_scan_grid():
    # m_ij = (l + s_ij) / 2 are the centres of an nx x ny grid of width W / 2
    # shifted by l / 2: the converted data is a confocal scan of wall W / 2.
    n, W = 16, 1.0
    laser = (0.3, -0.25)
    x = nc.detector_centres(n, W)
    mx = (laser[0] + x) / 2
    assert np.allclose(mx, nc.detector_centres(n, W / 2) + laser[0] / 2, rtol=0, atol=1e-15)
