"""Pins of the FP64 oracle solvers (oracle/admm.py): closed forms, the
optimality conditions of each sub-problem written from the augmented
Lagrangians of Sec. 3.1 (Eq. 5-12) and Sec. 4.1, and the convergence
behaviour the paper reports (the remark after Algorithm 1)."""

import math
import os

import numpy as np
import pytest

import synth
from oracle import admm, lct

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# --- shrinkage (Eq. 7) -----------------------------------------------------------

def test_shrink_closed_forms():
    a = np.array([3.0, 4.0, 0.0]).reshape(3, 1)
    assert np.allclose(admm.shrink(a, np.array([2.0]))[:, 0], [1.8, 2.4, 0.0], rtol=0, atol=1e-15)
    assert np.all(admm.shrink(a, np.array([5.0])) == 0.0)           # |a| <= b -> 0
    assert np.all(admm.shrink(a, np.array([7.5])) == 0.0)
    assert np.array_equal(admm.shrink(a, np.array([0.0])), a)       # b = 0 -> a
    assert np.all(admm.shrink(np.zeros((3, 1)), np.array([1.0])) == 0.0)


def test_shrink_minimises_weighted_l1_l2():
    # v = shrink(a, b) minimises b|v| + 1/2 |v - a|^2 per voxel (Eq. 6 divided by mu)
    rng = np.random.default_rng(0)
    a = rng.standard_normal((3, 400))
    b = rng.uniform(0.0, 2.0, 400)
    v = admm.shrink(a, b)

    def obj(x):
        return b * np.sqrt(np.sum(x * x, 0)) + 0.5 * np.sum((x - a) ** 2, 0)

    f0 = obj(v)
    for _ in range(50):
        assert np.all(f0 <= obj(v + 1e-3 * rng.standard_normal(v.shape)) + 1e-15)
    nv = np.sqrt(np.sum(v * v, 0))
    nz = nv > 0
    # subgradient condition: b v/|v| + v - a = 0 where v != 0, |a| <= b where v = 0
    assert np.allclose((b * v / np.where(nz, nv, 1.0) + v - a)[:, nz], 0.0, atol=1e-12)
    assert np.all(np.sqrt(np.sum(a * a, 0))[~nz] <= b[~nz] + 1e-15)


# --- finite differences, Laplacian eigenvalues and the FFT solve (Eq. 11) ---------

def test_grad_adjoint():
    rng = np.random.default_rng(1)
    u = rng.standard_normal((8, 6, 10))
    p = rng.standard_normal((3, 8, 6, 10))
    assert abs(np.sum(admm.grad(u) * p) - np.sum(u * admm.grad_adj(p))) < 1e-12


def test_grad_is_forward_difference():
    u = np.arange(4 * 5 * 6, dtype=np.float64).reshape(4, 5, 6) ** 2
    g = admm.grad(u)
    assert g[0, 1, 2, 3] == u[2, 2, 3] - u[1, 2, 3]
    assert g[1, 1, 4, 3] == u[1, 0, 3] - u[1, 4, 3]        # periodic wrap in y
    assert g[2, 3, 2, 5] == u[3, 2, 0] - u[3, 2, 5]        # periodic wrap in t


def test_laplacian_eigs_are_fft_of_stencil():
    shape = (8, 4, 16)
    s = np.zeros(shape)
    s[0, 0, 0] = 6.0
    for d in range(3):
        for o in (1, -1):
            idx = [0, 0, 0]
            idx[d] = o % shape[d]
            s[tuple(idx)] -= 1.0
    assert np.allclose(np.fft.fftn(s).real, admm.laplacian_eigs(shape), atol=1e-13)
    assert np.allclose(np.fft.fftn(s).imag, 0.0, atol=1e-13)


@pytest.mark.parametrize("c0,c1", [(1.0, 0.1), (93.4, 0.1), (3.0, 800.0)])
def test_fft_solve_residual(c0, c1):
    rng = np.random.default_rng(2)
    rhs = rng.standard_normal((8, 8, 32))
    x = admm.fft_solve(rhs, c0, c1)
    back = c0 * x + c1 * admm.grad_adj(admm.grad(x))
    assert np.max(np.abs(back - rhs)) < 1e-12 * max(1.0, c1)


# --- curvature and phi (Sec. 3) ---------------------------------------------------------

def test_curvature_of_plane_is_zero_exactly():
    n = 12
    x, y, t = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    u = (2 * x - 3 * y + 5 * t).astype(np.float64)
    k = admm.curvature(u, 1e-6)
    assert np.all(k[1:n - 1, 1:n - 1, 1:n - 1] == 0.0)


def _ball_fields(n=48):
    x, y, t = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    c = (n / 2 + 0.3, n / 2 - 0.2, n / 2 + 0.1)
    r = np.sqrt((x - c[0]) ** 2 + (y - c[1]) ** 2 + (t - c[2]) ** 2)
    rc = np.sqrt((x - c[0]) ** 2 + (y - c[1]) ** 2)
    return r, rc


@pytest.mark.parametrize("r0", [6, 8, 10, 12])
def test_curvature_of_sphere_and_cylinder(r0):
    # distance functions: div(grad r / |grad r|) = 2/r (sphere), 1/r (cylinder)
    r, rc = _ball_fields()
    for field, dim in ((r, 2.0), (rc, 1.0)):
        k = admm.curvature(field, 1e-6)
        sh = np.abs(field - r0) < 0.5
        rel = (k[sh] - dim / field[sh]) / (dim / field[sh])
        assert np.max(np.abs(rel)) < 0.4 / r0      # first-order differences: O(1/r)
        assert abs(np.mean(rel)) < 5e-3


def test_phi_variants():
    k = np.array([-2.0, 0.0, 0.5])
    assert np.allclose(admm.phi(k, 0.1, 0.3, "tsc"), 0.1 + 0.3 * k * k)
    assert np.allclose(admm.phi(k, 0.1, 0.3, "tac"), [0.7, 0.1, 0.25])
    assert np.allclose(admm.phi(k, 0.1, 0.3, "trv"), np.sqrt([1.3, 0.1, 0.175]))
    # b = 0 gives plain TV weights
    assert np.all(admm.phi(k, 0.2, 0.0) == 0.2)


# --- FISTA scalars (Algorithm 1) ---------------------------------------------------------

def test_fista_scalars():
    t1 = admm.fista_next(1.0)
    assert abs(t1 - (1 + math.sqrt(5)) / 2) < 1e-15
    assert (1.0 - 1.0) / t1 == 0.0                     # beta_0 = 0
    t = 1.0
    for k in range(1, 200):
        t_prev, t = t, admm.fista_next(t)
        assert t >= (k + 2) / 2.0                      # Beck-Teboulle: t_k >= (k+1)/2
        assert abs((t * t - t) - t_prev * t_prev) <= 1e-12 * t * t   # t^2 - t = t_prev^2


# --- optimality of each sub-problem against the augmented Lagrangians ----------------------

def _central_dd(obj, x, d, h=1e-3):
    return (obj(x + h * d) - obj(x - h * d)) / (2 * h)


def test_u_step_minimises_linearised_lagrangian():
    # Eq. 9/10 with g(u) of Eq. 8: <grad f, u - u_bar> + L/2 |u - u_bar|^2 + mu/2 |nabla u - (v + Lambda/mu)|^2
    rng = np.random.default_rng(3)
    sh = (8, 8, 16)
    u_bar, gf = rng.standard_normal(sh), rng.standard_normal(sh)
    v, lam = rng.standard_normal((3,) + sh), rng.standard_normal((3,) + sh)
    L, mu = 7.0, 0.3
    u = admm.u_solve(u_bar, gf, admm.u_rhs_reg(v, lam, mu), L, mu)

    def model(x):
        return (np.sum(gf * (x - u_bar)) + 0.5 * L * np.sum((x - u_bar) ** 2)
                + 0.5 * mu * np.sum((admm.grad(x) - (v + lam / mu)) ** 2))

    scale = abs(model(u)) + 1.0
    for _ in range(5):
        d = rng.standard_normal(sh)
        assert abs(_central_dd(model, u, d)) < 1e-8 * scale


def test_f_step_minimises_lagrangian():
    rng = np.random.default_rng(4)
    sh = (8, 8, 16)
    M = (rng.random((8, 8, 1)) < 0.3).astype(np.float64)
    tau0 = M * rng.random(sh)
    tau_bar, lam3 = rng.standard_normal(sh), rng.standard_normal(sh)
    lam_w, mu3 = 235.0, 2.0
    f = admm.f_step(tau0, M, tau_bar, lam3, lam_w, mu3)

    def obj(x):
        return (0.5 * lam_w * np.sum((M * (x - tau0)) ** 2) + np.sum(lam3 * (x - tau_bar))
                + 0.5 * mu3 * np.sum((x - tau_bar) ** 2))

    for _ in range(5):
        d = rng.standard_normal(sh)
        assert abs(_central_dd(obj, f, d)) < 1e-7 * (abs(obj(f)) + 1)


def test_tau_step_minimises_lagrangian():
    rng = np.random.default_rng(5)
    sh = (8, 8, 16)
    au, f, lam3 = rng.standard_normal(sh), rng.standard_normal(sh), rng.standard_normal(sh)
    w, lam2 = rng.standard_normal((3,) + sh), rng.standard_normal((3,) + sh)
    mu2, mu3 = 800.0, 2.0
    tau = admm.tau_solve(au, w, lam2, f, lam3, mu2, mu3)

    def obj(x):
        gx = admm.grad(x)
        return (0.5 * np.sum((au - x) ** 2) + np.sum(lam2 * (w - gx)) + 0.5 * mu2 * np.sum((w - gx) ** 2)
                + np.sum(lam3 * (f - x)) + 0.5 * mu3 * np.sum((f - x) ** 2))

    for _ in range(5):
        d = rng.standard_normal(sh)
        assert abs(_central_dd(obj, tau, d)) < 1e-8 * (abs(obj(tau)) + 1)


def test_v_step_minimises_lagrangian():
    # Eq. 6: sum phi |v| + mu/2 |v - (nabla u - Lambda/mu)|^2
    rng = np.random.default_rng(6)
    sh = (6, 6, 8)
    u, lam = rng.standard_normal(sh), rng.standard_normal((3,) + sh)
    ph, mu = rng.uniform(0, 1, sh), 0.7
    v = admm.v_step(u, lam, ph, mu)

    def obj(x):
        return (np.sum(ph * np.sqrt(np.sum(x * x, 0)))
                + 0.5 * mu * np.sum((x - (admm.grad(u) - lam / mu)) ** 2))

    f0 = obj(v)
    for _ in range(30):
        assert f0 <= obj(v + 1e-4 * rng.standard_normal(v.shape)) + 1e-12


# --- solvers on small seeded scenes ---------------------------------------------------------

def _small_scene(model, n=16, nt=128, seed=0):
    key = "c1_alg1_32x32x256" if model == 1 else "c2_alg2_64x64x512"
    cfg = dict(synth.CONFIGS[key])
    cfg.update(nx=n, ny=n, nt=nt, bin_width_s=cfg["bin_width_s"] * cfg["nt"] / nt)
    g = lct.Geometry(n, n, nt, cfg["bin_width_s"])
    mask = synth.make_mask(cfg)
    vol = synth.make_volume(cfg, seed)
    sig = lct.Operator(g).forward(vol)
    tau0 = synth.poisson_measurement(sig, mask, cfg["peak"], cfg["background"], seed + 1)
    return cfg, g, mask, vol, tau0


def test_zero_data_is_a_fixed_point():
    cfg, g, mask, _, _ = _small_scene(1, 8, 32)
    tau0 = np.zeros(g.shape)
    u, h = admm.alg1(tau0, mask, g, 1e-4, 1e-5, 0.1, 5)
    assert np.all(u == 0.0) and h["E"] == [0.0] * 5
    u, tau, h = admm.alg2(tau0, mask, g, 1e-4, 1e-4, 1e-4, 3e-2, 235.0, 1.0, 800.0, 2.0, 5)
    assert np.all(u == 0.0) and np.all(tau == 0.0)


def test_alg1_energy_and_residual_decrease():
    cfg, g, mask, vol, tau0 = _small_scene(1)
    u, h = admm.alg1(tau0, mask, g, cfg["a"], cfg["b"], cfg["mu"], 40)
    E = np.array(h["E"])
    assert E[-1] < E[0]
    assert np.mean(np.diff(E) < 0) >= 0.8
    assert h["primal_res"][-1] < h["primal_res"][1]
    assert sum(h["backtracks"]) == 0                 # L0 = 2 ||A_D||^2 never rejects
    # the reconstruction puts the surfaces at the right depth
    d, dt = admm.depth_map(u), admm.depth_map(vol)
    ok = dt >= 0
    assert np.mean(np.abs(d[ok] - dt[ok]) <= 2) > 0.8


def test_alg2_energy_decreases_with_restart():
    cfg, g, mask, vol, tau0 = _small_scene(2)
    p = cfg
    u, tau, h = admm.alg2(tau0, mask, g, p["a_u"], p["b_u"], p["a_tau"], p["b_tau"], p["lam"],
                          p["mu1"], p["mu2"], p["mu3"], 60)
    E = np.array(h["E"])
    assert E[-1] < 0.5 * E[0]
    assert np.mean(np.diff(E) < 0) >= 0.7
    assert h["primal_res_f"][-1] < h["primal_res_f"][1]
    d, dt = admm.depth_map(u), admm.depth_map(vol)
    ok = dt >= 0
    assert np.mean(np.abs(d[ok] - dt[ok]) <= 2) > 0.8


def test_backtracking_counts():
    cfg, g, mask, _, tau0 = _small_scene(1, 8, 64)
    op = lct.Operator(g, mask)
    n2, _ = lct.power_norm2(op)
    _, h = admm.alg1(tau0, mask, g, cfg["a"], cfg["b"], cfg["mu"], 8, norm2=n2, op=op)
    assert h["backtracks"] == [0] * 8 and h["L"] == [2 * n2] * 8
    L0 = 1e-3 * n2
    _, h = admm.alg1(tau0, mask, g, cfg["a"], cfg["b"], cfg["mu"], 8, L0=L0, op=op)
    n1 = h["backtracks"][0]
    assert 1 <= n1 <= math.ceil(math.log2(1e3))      # L0 * 2^n1 reaches ||A_D||^2 at most
    assert h["L"][0] == L0 * 2 ** n1                 # L doubles exactly per rejection (eta = 2)
    assert h["L"][-1] == L0 * 2 ** sum(h["backtracks"])
    assert h["L"][-1] <= 2 * n2                      # never beyond twice the Lipschitz constant
    assert sum(h["backtracks"][1:]) <= 3             # then L is (nearly) stable


# --- the paper's parameter settings (golden) -----------------------------------------------

def _golden_params():
    vals = {}
    with open(os.path.join(GOLDEN, "paper_parameters.txt")) as fh:
        for line in fh:
            line = line.split("#", 1)[0].strip()
            if line:
                k, v = line.split("=")
                vals[k.strip()] = float(v)
    return vals


def test_configs_use_paper_parameters():
    gp = _golden_params()
    c1 = synth.CONFIGS["c1_alg1_32x32x256"]
    c2 = synth.CONFIGS["c2_alg2_64x64x512"]
    assert (c1["a"], c1["b"], c1["mu"]) == (gp["alg1_a_8x8"], gp["alg1_b_8x8"], gp["alg1_mu"])
    assert (c2["mu1"], c2["mu2"], c2["mu3"]) == (gp["alg2_mu1"], gp["alg2_mu2"], gp["alg2_mu3"])
    assert (c2["lam"], c2["a_tau"], c2["b_tau"], c2["a_u"], c2["b_u"]) == (
        gp["alg2_lambda_8x8"], gp["alg2_a_tau_8x8"], gp["alg2_b_tau_8x8"],
        gp["alg2_a_u_8x8"], gp["alg2_b_u_8x8"])
    assert c1["bin_width_s"] == gp["bowling_bin_width_s"] and c1["nt"] == gp["bowling_bins"]


def test_backprojection_init_against_explicit_matrix_least_squares():
    """u0 = s A_D^T tau0 with s the least-squares scale, recomputed from the
    explicit matrix of A_D and numpy's least-squares solver on a tiny grid."""
    g = lct.Geometry(8, 8, 16, 128e-12)
    mask = synth.stride_mask(8, 8, 2)
    op = lct.Operator(g, mask)
    tau0 = np.random.default_rng(5).random(g.shape) * op.M
    u0, sc = admm.backprojection_init(op, tau0)
    A = lct.explicit_matrix(op)                      # A_D: rows of unsampled columns are zero
    b = tau0.ravel()
    gv = A.T @ b
    s_ls = np.linalg.lstsq((A @ gv)[:, None], b, rcond=None)[0][0]
    assert abs(sc - s_ls) <= 1e-10 * abs(s_ls)
    assert np.allclose(u0.ravel(), s_ls * gv, rtol=1e-10, atol=1e-14 * np.abs(gv).max())


def test_backprojection_scale_minimises_the_data_term():
    cfg, g, mask, vol, tau0 = _small_scene(1, 16, 64)
    op = lct.Operator(g, mask)
    u0, sc = admm.backprojection_init(op, tau0)
    d = op.M * tau0

    def f(s):
        r = op.forward_d(u0 * (s / sc)) - d
        return 0.5 * float(np.sum(r * r))
    assert sc > 0
    for s in (0.5 * sc, 0.9 * sc, 0.99 * sc, 1.01 * sc, 1.1 * sc, 2.0 * sc, 0.0):
        assert f(sc) <= f(s)


def test_backprojection_of_point_scatterer_peaks_at_it():
    n, nt = 16, 64
    g = lct.Geometry(n, n, nt, 32e-12 * 256 / nt)
    mask = synth.stride_mask(n, n, 2)
    op = lct.Operator(g, mask)
    vol = np.zeros(g.shape)
    vol[8, 8, 30] = 1.0                              # a sampled column (stride 2, offset 1 would be odd)
    vol[9, 9, 30] = 1.0
    u0, _ = admm.backprojection_init(op, op.forward_d(vol))
    x, y, t = np.unravel_index(np.argmax(u0), u0.shape)
    assert abs(t - 30) <= 1 and abs(x - 8.5) <= 1.5 and abs(y - 8.5) <= 1.5


def test_backprojection_zero_data_and_default_start():
    cfg, g, mask, _, tau0 = _small_scene(1, 8, 32)
    op = lct.Operator(g, mask)
    u0, sc = admm.backprojection_init(op, np.zeros(g.shape))
    assert sc == 0.0 and np.all(u0 == 0.0)
    # an explicit zero start is the default start, bit for bit
    ua, ha = admm.alg1(tau0, mask, g, cfg["a"], cfg["b"], cfg["mu"], 4, op=op)
    ub, hb = admm.alg1(tau0, mask, g, cfg["a"], cfg["b"], cfg["mu"], 4, op=op, u_init=np.zeros(g.shape))
    assert np.array_equal(ua, ub) and ha["E"] == hb["E"]


def test_alg1_from_backprojection_decreases_energy():
    cfg, g, mask, vol, tau0 = _small_scene(1)
    op = lct.Operator(g, mask)
    u0, _ = admm.backprojection_init(op, tau0)
    u, h = admm.alg1(tau0, mask, g, cfg["a"], cfg["b"], cfg["mu"], 30, op=op, u_init=u0)
    E = np.array(h["E"])
    assert E[-1] < E[0] and np.mean(np.diff(E) < 0) >= 0.8
    assert sum(h["backtracks"]) == 0
