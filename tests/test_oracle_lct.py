"""Pins of the FP64 oracle operator (oracle/lct.py) against closed forms,
brute force and the physics of Eq. 2 -- no GPU, no CUDA library."""

import numpy as np
import pytest

from oracle import lct


def geom(n=8, nt=32, rad="compensated", bw=None):
    if bw is None:
        bw = 32e-12 * 256 / nt
    return lct.Geometry(n, n, nt, bw, radiometry=rad)


# --- resampling tables (R_z, R_t^{-1}) against their closed forms -----------

@pytest.mark.parametrize("nt", [16, 64, 256, 512, 1024])
def test_rt_positions_exact(nt):
    # The v-grid position of rho_k^2 is (k + 1/2)^2 / nt - 1/2, clamped; the
    # taps must reproduce it exactly (dyadic rationals, exact in FP64).
    k0, w0, w1, wt = lct.rt_table(nt)
    for k in range(nt):
        q = min(max(((2 * k + 1) ** 2 / (4 * nt)) - 0.5, 0.0), nt - 1.0)
        assert k0[k] + w1[k] == q
        assert 0 <= k0[k] <= nt - 2
        assert w0[k] + w1[k] == 1.0
    # first bins with (k+1/2)^2 < nt/2 clamp onto v-bin 0
    nclamp = sum(1 for k in range(nt) if (k + 0.5) ** 2 < nt / 2)
    assert np.all(k0[:nclamp] == 0) and np.all(w1[:nclamp] == 0.0)
    rho = (np.arange(nt) + 0.5) / nt
    assert np.array_equal(wt, rho)
    _, _, _, wraw = lct.rt_table(nt, "raw")
    assert np.allclose(wraw * rho ** 3, 1.0, rtol=1e-15, atol=0)


@pytest.mark.parametrize("nt", [16, 64, 256, 512, 1024])
def test_rz_interpolates_linear_functions(nt):
    # R_z of a function linear in the rho-index is g_j * (a + b p_j) with
    # p_j = clamp(sqrt((j + 1/2) nt) - 1/2): an index, weight or clamp error fails.
    a, b = 0.25, 1.5
    u = a + b * np.arange(nt, dtype=np.float64)
    got = lct.apply_rz(u[None, None, :], nt)[0, 0]
    j = np.arange(nt)
    p = np.clip(np.sqrt((j + 0.5) * nt) - 0.5, 0, nt - 1)
    want = (a + b * p) / (2.0 * np.sqrt((j + 0.5) / nt))
    assert np.allclose(got, want, rtol=1e-14, atol=0)
    # the last v-bins lie beyond rho_{nt-1}: clamped to the end bin
    i0, w0, w1, _ = lct.rz_table(nt)
    assert i0[-1] == nt - 2 and w1[-1] == 1.0


def test_rt_interpolates_linear_functions():
    nt = 128
    c = 3.0 - 0.5 * np.arange(nt, dtype=np.float64)
    got = lct.apply_rt_inv(c[None, None, :], nt, "compensated")[0, 0]
    k = np.arange(nt)
    q = np.clip((k + 0.5) ** 2 / nt - 0.5, 0, nt - 1)
    want = ((k + 0.5) / nt) * (3.0 - 0.5 * q)
    assert np.allclose(got, want, rtol=1e-14, atol=1e-14)


# --- the cone kernel ----------------------------------------------------------

def test_kernel_partition_of_unity():
    g = geom(16, 64)
    h = lct.cone_kernel(g, normalise=False)
    w = lct.cone_weights(g)
    for a, i in enumerate(range(-15, 16)):
        for b, j in enumerate(range(-15, 16)):
            col = h[i % 32, j % 32]
            if w[a, b] <= g.nt - 1:
                assert abs(col.sum() - 1.0) < 1e-12
                # mass sits on floor(w) and floor(w)+1 only, centred on w
                assert abs(np.dot(col, np.arange(g.nt)) - w[a, b]) < 1e-12
            else:
                assert col.sum() <= 1.0
    # the kernel is even in the lateral offsets and zero at offset -n
    assert np.array_equal(h, h[(-np.arange(32)) % 32][:, (-np.arange(32)) % 32])
    assert np.all(h[16] == 0) and np.all(h[:, 16] == 0)
    hn = lct.cone_kernel(g)
    assert abs(np.sum(hn * hn) - 1.0) < 1e-12


def test_cone_offsets_match_geometry():
    # w_ij in v-bins equals nt * (lateral distance / R)^2
    g = lct.Geometry(8, 8, 64, 16e-12, wall_width_m=0.7)
    w = lct.cone_weights(g)
    R = lct.C_LIGHT * 64 * 16e-12 / 2
    d2 = ((3 * 0.7 / 8) ** 2 + (5 * 0.7 / 8) ** 2)
    assert abs(w[7 + 3, 7 - 5] - 64 * d2 / R ** 2) < 1e-12


# --- H by padded FFT against brute-force summation ------------------------------

@pytest.mark.parametrize("n,nt", [(8, 32), (16, 64)])
def test_h_fft_matches_brute_force(n, nt):
    g = geom(n, nt)
    x = np.random.default_rng(1).standard_normal(g.shape)
    a = lct.apply_h(x, g)
    b = lct.brute_force_h(x, g)
    assert np.linalg.norm(a - b) <= 1e-12 * np.linalg.norm(b)


def test_h_of_unit_impulse_is_the_kernel():
    g = geom(8, 32)
    x = np.zeros(g.shape)
    x[0, 0, 0] = 1.0
    h = lct.cone_kernel(g)
    assert np.allclose(lct.apply_h(x, g), h[:8, :8, :], atol=1e-15)


# --- A against the physical direct summation of Eq. 2 ----------------------------

def _fit(t1, t2):
    return float(np.sum(t1 * t2) / np.sum(t2 * t2))


@pytest.mark.parametrize("rad", ["compensated", "raw"])
@pytest.mark.parametrize("pos", [(5, 9, 30), (8, 8, 50), (3, 12, 22)])
def test_forward_matches_direct_summation_point(rad, pos):
    g = lct.Geometry(16, 16, 64, 128e-12, radiometry=rad)
    u = np.zeros(g.shape)
    u[pos] = 1.0
    t1 = lct.Operator(g).forward(u)
    t2 = lct.direct_summation(u, g)
    live = (t1.sum(2) > 1e-9 * t1.sum()) & (t2.sum(2) > 1e-9 * t2.sum())
    k = np.arange(g.nt)
    c1 = (t1 * k).sum(2)[live] / t1.sum(2)[live]
    c2 = (t2 * k).sum(2)[live] / t2.sum(2)[live]
    assert np.max(np.abs(c1 - c2)) < 0.5          # arrival-time centroid, bins
    p1 = np.argmax(t1, 2)[live]
    p2 = np.argmax(t2, 2)[live]
    assert np.max(np.abs(p1 - p2)) <= 1           # peak bin within +-1
    # A point-samples a one-voxel-thin shell on the t-grid (two-tap R_t^{-1}), so
    # a single scatterer's per-bin amplitudes depend on its sub-bin phase; only
    # arrival times are compared here, amplitudes on extended scatterers below.


@pytest.mark.parametrize("rad", ["compensated", "raw"])
def test_forward_matches_direct_summation_plane(rad):
    g = lct.Geometry(16, 16, 64, 128e-12, radiometry=rad)
    u = np.zeros(g.shape)
    u[3:13, 2:12, 40] = 1.0
    t1 = lct.Operator(g).forward(u)
    t2 = lct.direct_summation(u, g)
    s = _fit(t1, t2)
    tot1, tot2 = t1.sum(2), s * t2.sum(2)
    assert np.max(np.abs(tot1 / tot2 - 1.0)) < 0.05   # per-scan-point totals within 5 %
    assert np.linalg.norm(t1 - s * t2) < 0.1 * np.linalg.norm(t1)
    k = np.arange(g.nt)
    c1 = (t1 * k).sum(2) / tot1
    c2 = (t2 * k).sum(2) / t2.sum(2)
    assert np.max(np.abs(c1 - c2)) < 0.5


def test_raw_and_compensated_differ_by_t4():
    rng = np.random.default_rng(3)
    u = rng.random((8, 8, 32))
    gc, gr = geom(8, 32, "compensated"), geom(8, 32, "raw")
    tc = lct.Operator(gc).forward(u)
    tr = lct.Operator(gr).forward(u)
    rho = (np.arange(32) + 0.5) / 32
    assert np.allclose(tr * rho ** 4, tc, rtol=1e-12, atol=0)


# --- transpose, sampling and the operator norm --------------------------------------

@pytest.mark.parametrize("rad", ["compensated", "raw"])
def test_adjoint_dot_product_identity(rad):
    g = geom(16, 64, rad)
    mask = np.random.default_rng(5).integers(0, 2, (16, 16)).astype(np.uint8)
    op = lct.Operator(g, mask)
    rng = np.random.default_rng(6)
    x, y = rng.standard_normal(g.shape), rng.standard_normal(g.shape)
    lhs = np.sum(op.forward_d(x) * y)
    rhs = np.sum(x * op.adjoint_d(y))
    assert abs(lhs - rhs) <= 1e-12 * np.sqrt(np.sum(op.forward_d(x) ** 2) * np.sum(y * y))


def test_adjoint_is_explicit_transpose():
    g = geom(8, 16)
    mask = np.eye(8, dtype=np.uint8)
    op = lct.Operator(g, mask)
    Mx = lct.explicit_matrix(op)
    V = Mx.shape[0]
    At = np.stack([op.adjoint_d(e.reshape(g.shape)).ravel() for e in np.eye(V)], 1)
    assert np.max(np.abs(At - Mx.T)) <= 1e-13 * np.max(np.abs(Mx))


def test_sampling_operator():
    g = geom(8, 16)
    mask = np.zeros((8, 8), dtype=np.uint8)
    mask[1::2, 1::2] = 1
    op = lct.Operator(g, mask)
    rng = np.random.default_rng(7)
    t = op.forward_d(rng.standard_normal(g.shape))
    assert np.all(t[mask == 0] == 0.0)
    r = rng.standard_normal(g.shape)
    r2 = r.copy()
    r2[mask == 0] = 1e9  # values off the mask must be ignored by A_D^T
    assert np.array_equal(op.adjoint_d(r), op.adjoint_d(r2))
    cols = lct.sampled_columns(mask)
    assert np.array_equal(cols, np.array([i * 8 + j for i in range(8) for j in range(8)
                                          if mask[i, j]], dtype=np.int32))
    assert np.all(np.diff(cols) > 0)


@pytest.mark.parametrize("rad", ["compensated", "raw"])
def test_power_iteration_matches_svd(rad):
    g = geom(8, 16, rad)
    mask = np.zeros((8, 8), dtype=np.uint8)
    mask[::2, ::2] = 1
    op = lct.Operator(g, mask)
    n2, _ = lct.power_norm2(op, max_iter=5000)
    s = np.linalg.svd(lct.explicit_matrix(op), compute_uv=False)
    assert abs(n2 - s[0] ** 2) <= 1e-8 * s[0] ** 2


# --- the directional (normal-weighted) confocal model (Sec. 2) ---------------------

def _normals(shape, seed):
    rng = np.random.default_rng(seed)
    v = rng.standard_normal((3,) + shape)
    v[2] = -np.abs(v[2]) - 0.5                   # facing the wall (z decreases towards it)
    return list(v / np.sqrt(np.sum(v * v, axis=0)))


def test_directional_equals_entrywise_weighted_matrix():
    """The six-term expansion equals A's explicit matrix with every entry
    (scan point x', time bin k; voxel x) weighted by ((x' - x) . n(x))^2 /
    d_k^2, d_k the distance of bin k's cone: an independent computation of
    the same operator in which every term of the expansion takes part."""
    g = geom(8, 16)
    op = lct.Operator(g)
    normals = _normals(g.shape, 1)
    A = lct.explicit_matrix(op, masked=False)
    nx, ny, nt = g.shape
    W, R = g.wall_width_m, g.range_m
    X = (np.arange(nx) + 0.5 - nx / 2) * W / nx / R
    Y = (np.arange(ny) + 0.5 - ny / 2) * W / ny / R
    Z = (np.arange(nt) + 0.5) / nt
    ii, jj, kk = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nt), indexing="ij")
    ri, rj, rk = ii.ravel(), jj.ravel(), kk.ravel()          # row (scan point, time bin) = column index layout
    a, b, c = (n.ravel() for n in normals)
    dot = ((X[ri][:, None] - X[ri][None, :]) * a[None, :] + (Y[rj][:, None] - Y[rj][None, :]) * b[None, :]
           - Z[rk][None, :] * c[None, :])
    Ad = A * dot * dot / (Z[rk] ** 2)[:, None]
    u = np.random.default_rng(2).standard_normal(g.shape)
    want = (Ad @ u.ravel()).reshape(g.shape)
    got = lct.directional_forward(op, u, normals, masked=False)
    assert np.max(np.abs(got - want)) <= 1e-12 * np.max(np.abs(want))


@pytest.mark.parametrize("tilt", [(0.0, 0.0), (0.5, 0.0), (0.45, 0.45)])
def test_directional_matches_direct_summation_plane(tilt):
    """A fronto-parallel plane with one normal everywhere (tilted in x and y)
    against the directional model summed voxel by voxel, as for the albedo
    model: per-scan-point totals within 5 % after one scale fit."""
    g = lct.Geometry(16, 16, 64, 128e-12)
    u = np.zeros(g.shape)
    u[3:13, 2:12, 40] = 1.0
    nz = -np.sqrt(1.0 - tilt[0] ** 2 - tilt[1] ** 2)
    normals = [np.full(g.shape, tilt[0]), np.full(g.shape, tilt[1]), np.full(g.shape, nz)]
    t1 = lct.directional_forward(lct.Operator(g), u, normals, masked=False)
    t2 = lct.directional_direct_summation(u, normals, g)
    s = _fit(t1, t2)
    tot1, tot2 = t1.sum(2), s * t2.sum(2)
    assert np.max(np.abs(tot1 / tot2 - 1.0)) < 0.05
    assert np.linalg.norm(t1 - s * t2) < 0.1 * np.linalg.norm(t1)
    k = np.arange(g.nt)
    assert np.max(np.abs((t1 * k).sum(2) / tot1 - (t2 * k).sum(2) / t2.sum(2))) < 0.5
    # the tilt changes the measurement (the model is not the albedo model)
    ta = lct.Operator(g).forward(u)
    ratio = tot1 / ta.sum(2)
    assert (np.max(ratio) - np.min(ratio)) / np.mean(ratio) > 0.05


def test_directional_adjoint_dot_product_identity():
    g = geom(16, 64)
    mask = np.random.default_rng(5).integers(0, 2, (16, 16)).astype(np.uint8)
    op = lct.Operator(g, mask)
    normals = _normals(g.shape, 3)
    rng = np.random.default_rng(6)
    x, y = rng.standard_normal(g.shape), rng.standard_normal(g.shape)
    fx = lct.directional_forward(op, x, normals)
    lhs = np.sum(fx * y)
    rhs = np.sum(x * lct.directional_adjoint(op, y, normals))
    assert abs(lhs - rhs) <= 1e-12 * np.sqrt(np.sum(fx * fx) * np.sum(y * y))
