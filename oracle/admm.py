"""FP64 oracle of the curvature-regularised ADMM solvers (Algorithms 1 and 2).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Written from Sec. 3 (Eq. 4-12, Algorithm 1) and Sec. 4.1 (Eq. 13,
Algorithm 2).  Readings where the paper is silent:

* Finite differences (Sec. 3.1): unit grid spacing on x, y, t; the gradient
  is the forward difference with periodic wrap, nabla^* = -div with backward
  differences (periodic), so nabla^* nabla is diagonalised by the FFT as
  Eq. 11 requires, with eigenvalues sum_d 4 sin^2(pi k_d / N_d).
* |.| in the TV term and in the shrinkage of Eq. 7 is the Euclidean norm of
  the 3-vector at each voxel (isotropic); shrink(0, b) = 0.
* Curvature (Sec. 3): n = nabla u / sqrt(|nabla u|^2 + eps^2),
  kappa = backward-difference divergence of n.
* The v-step of Algorithm 1 (Eq. 7) is taken at the extrapolated point
  u-bar, the point at which the saddle-point step of Algorithm 1 evaluates L.
* The linearised u-step (Eq. 9-11) uses a backtracking rule on L (named in
  the abstract only): accept when
  f(u+) <= f(u-bar) + <grad f(u-bar), u+ - u-bar> + L/2 ||u+ - u-bar||^2,
  else L <- eta L and solve again; L is kept across iterations.
  L0 defaults to 2 ||A_D||_2^2 (below Eq. 10).
* Algorithm 2's sub-steps are not printed; they are the exact minimisers of
  its augmented Lagrangian in the Gauss-Seidel order v, w, f, u, tau, then the
  three multiplier ascents, with the u-step linearised as in Algorithm 1.
* Algorithm 2 extrapolates both u and tau with the FISTA weights; to keep
  that stable it resets the sequence (t <- 1) whenever E(u, tau) increases
  (adaptive restart).  Algorithm 1 runs without restart, as printed.

Parity status: pinned by tests/test_oracle_admm.py (closed-form shrinkage,
curvature of planes, spheres and cylinders, FFT-solve residual, eigenvalues
against the FFT of the Laplacian stencil, sub-problem optimality conditions,
FISTA scalars, backtracking counts, zero fixed point, energy decrease).
"""

import math

import numpy as np

from .lct import Operator, power_norm2

# ---------------------------------------------------------------------------
# Finite differences and the FFT-diagonal Laplacian (Sec. 3.1.2, Eq. 11)
# ---------------------------------------------------------------------------


def grad(u):
    """Forward differences with periodic wrap: (3,) + u.shape."""
    return np.stack([np.roll(u, -1, axis=d) - u for d in range(3)])


def div_b(p):
    """Backward-difference divergence with periodic wrap of a (3, ...) field."""
    return sum(p[d] - np.roll(p[d], 1, axis=d) for d in range(3))


def grad_adj(p):
    """nabla^*, the adjoint of ``grad``: -div_b."""
    return -div_b(p)


def laplacian_eigs(shape):
    """Eigenvalues of nabla^* nabla on the periodic grid, full FFT layout."""
    lam = np.zeros(shape)
    for d, n in enumerate(shape):
        k = np.arange(n)
        e = 4.0 * np.sin(np.pi * k / n) ** 2
        sh = [1, 1, 1]
        sh[d] = n
        lam = lam + e.reshape(sh)
    return lam


def fft_solve(rhs, c0, c1):
    """Solve (c0 I + c1 nabla^* nabla) x = rhs by FFT (Eq. 11)."""
    lam = laplacian_eigs(rhs.shape)
    return np.real(np.fft.ifftn(np.fft.fftn(rhs) / (c0 + c1 * lam)))


# ---------------------------------------------------------------------------
# Shrinkage (Eq. 7), curvature and the weight phi (Sec. 3)
# ---------------------------------------------------------------------------


def shrink(a, b):
    """shrinkage(a, b) = max(|a| - b, 0) a / |a| per voxel, |.| over axis 0."""
    na = np.sqrt(np.sum(a * a, axis=0))
    scale = np.where(na > 0.0, np.maximum(na - b, 0.0) / np.where(na > 0.0, na, 1.0), 0.0)
    return a * scale


def curvature(u, eps):
    """kappa = div(nabla u / |nabla u|) with |nabla u| regularised by eps."""
    g = grad(u)
    n = g / np.sqrt(np.sum(g * g, axis=0) + eps * eps)
    return div_b(n)


def phi(kappa, a, b, kind="tsc"):
    """phi(kappa) of Sec. 3: TSC a + b k^2 (default), TAC a + b|k|, TRV sqrt(a + b k^2)."""
    if kind == "tsc":
        return a + b * kappa * kappa
    if kind == "tac":
        return a + b * np.abs(kappa)
    if kind == "trv":
        return np.sqrt(a + b * kappa * kappa)
    raise ValueError(kind)


def tv_norm(u):
    """|nabla u| per voxel (isotropic)."""
    g = grad(u)
    return np.sqrt(np.sum(g * g, axis=0))


def fista_next(t):
    """t^{k+1} = (1 + sqrt(1 + 4 t^2)) / 2 (Algorithm 1)."""
    return (1.0 + math.sqrt(1.0 + 4.0 * t * t)) / 2.0


# ---------------------------------------------------------------------------
# Algorithm 1: object-domain model (Eq. 4)
# ---------------------------------------------------------------------------


# ---------------------------------------------------------------------------
# Sub-problem minimisers (Sec. 3.1.1-3.1.3 and the Lagrangian of Sec. 4.1)
# ---------------------------------------------------------------------------


def v_step(u_bar, lam, phi_w, mu):
    """Eq. 7: v = shrinkage(nabla u-bar - Lambda/mu, phi/mu)."""
    return shrink(grad(u_bar) - lam / mu, phi_w / mu)


def u_rhs_reg(v, lam, mu):
    """The regulariser part of the right-hand side of the PDE above Eq. 11:
    mu nabla^*(v + Lambda/mu)."""
    return mu * grad_adj(v + lam / mu)


def u_solve(u_bar, grad_f, rhs_reg, L, mu):
    """Eq. 11: u = F^{-1}[F(L u-bar - grad f(u-bar) + rhs_reg) / (L + mu F(nabla^* nabla))]."""
    return fft_solve(L * u_bar - grad_f + rhs_reg, L, mu)


def f_step(tau0_masked, M, tau_bar, lam3, lam_w, mu3):
    """Minimiser over f of lambda/2 ||f - tau0||^2_{Omega minus X} + <Lambda_3, f - tau-bar>
    + mu_3/2 ||f - tau-bar||^2 (Sec. 4.1), pointwise."""
    return (lam_w * M * tau0_masked + mu3 * tau_bar - lam3) / (lam_w * M + mu3)


def tau_solve(au, w, lam2, f, lam3, mu2, mu3):
    """Minimiser over tau of 1/2 ||A u - tau||^2 + <Lambda_2, w - nabla tau> + mu_2/2 ||w - nabla tau||^2
    + <Lambda_3, f - tau> + mu_3/2 ||f - tau||^2 (Sec. 4.1), by FFT as in Eq. 11."""
    rhs = au + mu2 * grad_adj(w + lam2 / mu2) + mu3 * (f + lam3 / mu3)
    return fft_solve(rhs, 1.0 + mu3, mu2)


class BacktrackingError(RuntimeError):
    pass


def linearised_step(fwd, adj, data, u_bar, rhs_reg, L, c1, eta, max_backtracks):
    """Eq. 9-11 with the backtracking rule on L.

    f(u) = 1/2 ||fwd(u) - data||^2, grad f = adj(fwd(u) - data).  Returns
    (u_plus, L, n_rejections, fwd(u_plus), f(u_bar), grad f(u_bar)).
    """
    r = fwd(u_bar) - data
    f_bar = 0.5 * float(np.sum(r * r))
    gf = adj(r)
    rejections = 0
    while True:
        u_plus = u_solve(u_bar, gf, rhs_reg, L, c1)
        d = u_plus - u_bar
        au = fwd(u_plus)
        rp = au - data
        f_plus = 0.5 * float(np.sum(rp * rp))
        model = f_bar + float(np.sum(gf * d)) + 0.5 * L * float(np.sum(d * d))
        if f_plus <= model:
            return u_plus, L, rejections, au, f_bar, gf
        rejections += 1
        if rejections > max_backtracks:
            raise BacktrackingError("backtracking did not terminate")
        L *= eta


def alg1(tau0, mask, geom, a, b, mu, iters, L0=None, eta=2.0, eps_normal=1e-6,
         phi_kind="tsc", eps_stop=0.0, max_backtracks=30, norm2=None, op=None,
         restart=False, u_init=None):
    """Algorithm 1: ADMM for min_u 1/2 ||A u - tau0||^2_{Omega minus X} + R(kappa(u)).

    Per iteration, in order: v (Eq. 7 at u-bar), the linearised u-step with
    backtracking (Eq. 9-11), the multiplier ascent (Eq. 12), t and u-bar
    (FISTA extrapolation of Algorithm 1), phi(kappa(u^{k+1})) and the
    relative energy change e^{k+1}.  With ``restart`` the FISTA sequence is
    reset (t <- 1, so the next extrapolation weight is 0) whenever the energy
    increases.  ``u_init`` replaces the zero start u^0 = u-bar^0 = 0 (phi and
    the initial energy are then those of u_init).  Returns (u, history).
    """
    if op is None:
        op = Operator(geom, mask)
    M = op.M
    data = M * tau0
    shape = geom.shape
    if L0 is None or L0 <= 0:
        if norm2 is None:
            norm2, _ = power_norm2(op)
        L0 = 2.0 * norm2
    L = float(L0)

    u = np.zeros(shape) if u_init is None else np.array(u_init, dtype=np.float64)
    u_bar = u.copy()
    lam = np.zeros((3,) + shape)
    ph = phi(curvature(u, eps_normal), a, b, phi_kind)
    t = 1.0
    r0 = op.forward_d(u) - data
    E_prev = 0.5 * float(np.sum(r0 * r0)) + float(np.sum(ph * tv_norm(u)))

    hist = {"E": [], "e": [], "L": [], "backtracks": [], "f": [], "primal_res": [], "du": []}
    for _ in range(iters):
        v = v_step(u_bar, lam, ph, mu)
        rhs_reg = u_rhs_reg(v, lam, mu)
        u_new, L, nrej, au, _, _ = linearised_step(
            op.forward_d, op.adjoint_d, data, u_bar, rhs_reg, L, mu, eta, max_backtracks)
        gu = grad(u_new)
        lam = lam + mu * (v - gu)
        t_new = fista_next(t)
        beta = (t - 1.0) / t_new
        du = u_new - u_bar
        u_bar = u_new + beta * (u_new - u)
        u = u_new
        t = t_new
        ph = phi(curvature(u, eps_normal), a, b, phi_kind)
        rp = au - data
        f = 0.5 * float(np.sum(rp * rp))
        E = f + float(np.sum(ph * np.sqrt(np.sum(gu * gu, axis=0))))
        e = abs(E_prev - E) / abs(E) if E != 0.0 else 0.0
        hist["E"].append(E)
        hist["e"].append(e)
        hist["L"].append(L)
        hist["backtracks"].append(nrej)
        hist["f"].append(f)
        hist["primal_res"].append(float(np.sqrt(np.sum((v - gu) ** 2))))
        hist["du"].append(float(np.sqrt(np.sum(du * du))))
        hist.setdefault("restart", []).append(bool(restart and E > E_prev))
        if restart and E > E_prev:
            t = 1.0
        E_prev = E
        if eps_stop > 0.0 and e <= eps_stop:
            break
    return u, hist


def backprojection_init(op, tau0):
    """Back-projection start u^0 = s A_D^T tau0 (the direct back-projection
    reconstruction the paper contrasts with the iterative methods, Sec. 1;
    used here, like the Algorithm-1 start of Algorithm 2 in the remark after
    Algorithm 2, to initialise the ADMM).  The paper fixes no scale; reading:
    s minimises the data term 1/2 ||A_D (s g) - tau0||^2 over s, with
    g = A_D^T tau0, which is s = <A_D g, tau0> / ||A_D g||^2 = ||g||^2 / ||A_D g||^2
    (the exact line-search step of steepest descent from u = 0); s = 0 when
    A_D g = 0.  Returns (u0, s)."""
    g = op.adjoint_d(tau0)
    ag = op.forward_d(g)
    den = float(np.sum(ag * ag))
    sc = float(np.sum(g * g)) / den if den > 0.0 else 0.0
    return sc * g, sc


# ---------------------------------------------------------------------------
# Algorithm 2: dual signal/object-domain model (Eq. 13)
# ---------------------------------------------------------------------------


def alg2(tau0, mask, geom, a_u, b_u, a_tau, b_tau, lam, mu1, mu2, mu3, iters,
         L0=None, eta=2.0, eps_normal=1e-6, phi_kind="tsc", eps_stop=0.0,
         max_backtracks=30, norm2=None, op=None, u_init=None, restart=True):
    """Algorithm 2: ADMM for the dual-domain energy E(u, tau) of Eq. 13.

    Splitting v = nabla u, w = nabla tau, f = tau with multipliers
    Lambda_1..3 and penalties mu_1..3 (augmented Lagrangian of Sec. 4.1).
    Sub-steps, each the exact minimiser of that Lagrangian given the others:

      v   = shrink(nabla u-bar - Lambda_1/mu_1, phi_u/mu_1)
      w   = shrink(nabla tau-bar - Lambda_2/mu_2, phi_tau/mu_2)
      f   = (lambda M tau0 + mu_3 tau-bar - Lambda_3) / (lambda M + mu_3)
      u+  = linearised step on 1/2 ||A u - tau-bar||^2 (Eq. 9-11 with the
            unmasked A), denominator L + mu_1 lambda(k), backtracking on L
      tau+ = F^{-1}[F(A u+ + mu_2 nabla^*(w + Lambda_2/mu_2)
                       + mu_3 (f + Lambda_3/mu_3)) / ((1 + mu_3) + mu_2 lambda(k))]
      Lambda_1 += mu_1 (v - nabla u+), Lambda_2 += mu_2 (w - nabla tau+),
      Lambda_3 += mu_3 (f - tau+)

    then the shared FISTA extrapolation of u and tau and the phi refresh of
    Algorithm 2.  ``u_init`` warm-starts u (the remark after Algorithm 2).

    ``restart`` (default on): whenever E(u, tau) increases the FISTA sequence
    is reset (t <- 1), so the next extrapolation weight is 0.  The paper does
    not say how Algorithm 2 keeps its extrapolated tau-bar stable; without a
    restart this reading diverges on seeded scenes (the energy grows by
    orders of magnitude within 100 iterations), with it E decreases.
    Returns (u, tau, history).
    """
    if op is None:
        op = Operator(geom, mask)
    M = op.M
    data0 = M * tau0
    shape = geom.shape
    if L0 is None or L0 <= 0:
        if norm2 is None:
            norm2, _ = power_norm2(op, masked=False)
        L0 = 2.0 * norm2
    L = float(L0)

    u = np.zeros(shape) if u_init is None else np.array(u_init, dtype=np.float64)
    u_bar = u.copy()
    tau = np.zeros(shape)
    tau_bar = np.zeros(shape)
    lam1 = np.zeros((3,) + shape)
    lam2 = np.zeros((3,) + shape)
    lam3 = np.zeros(shape)
    ph_u = phi(curvature(u, eps_normal), a_u, b_u, phi_kind)
    ph_t = phi(curvature(tau, eps_normal), a_tau, b_tau, phi_kind)
    t = 1.0

    def energy(au, tu, ph_uu, ph_tt, gu, gt):
        r = au - tu
        s = M * (tu - tau0)
        return (0.5 * float(np.sum(r * r)) + 0.5 * lam * float(np.sum(s * s))
                + float(np.sum(ph_uu * np.sqrt(np.sum(gu * gu, axis=0))))
                + float(np.sum(ph_tt * np.sqrt(np.sum(gt * gt, axis=0)))))

    E_prev = energy(op.forward(u), tau, ph_u, ph_t, grad(u), grad(tau))
    hist = {"E": [], "e": [], "L": [], "backtracks": [], "primal_res_u": [],
            "primal_res_tau": [], "primal_res_f": []}
    for _ in range(iters):
        v = v_step(u_bar, lam1, ph_u, mu1)
        w = v_step(tau_bar, lam2, ph_t, mu2)
        f = f_step(data0, M, tau_bar, lam3, lam, mu3)
        rhs_reg = u_rhs_reg(v, lam1, mu1)
        u_new, L, nrej, au, _, _ = linearised_step(
            op.forward, op.adjoint, tau_bar, u_bar, rhs_reg, L, mu1, eta, max_backtracks)
        tau_new = tau_solve(au, w, lam2, f, lam3, mu2, mu3)
        gu = grad(u_new)
        gt = grad(tau_new)
        lam1 = lam1 + mu1 * (v - gu)
        lam2 = lam2 + mu2 * (w - gt)
        lam3 = lam3 + mu3 * (f - tau_new)
        t_new = fista_next(t)
        beta = (t - 1.0) / t_new
        u_bar = u_new + beta * (u_new - u)
        tau_bar = tau_new + beta * (tau_new - tau)
        u, tau, t = u_new, tau_new, t_new
        ph_u = phi(curvature(u, eps_normal), a_u, b_u, phi_kind)
        ph_t = phi(curvature(tau, eps_normal), a_tau, b_tau, phi_kind)
        E = energy(au, tau, ph_u, ph_t, gu, gt)
        e = abs(E_prev - E) / abs(E) if E != 0.0 else 0.0
        hist["E"].append(E)
        hist["e"].append(e)
        hist["L"].append(L)
        hist["backtracks"].append(nrej)
        hist["primal_res_u"].append(float(np.sqrt(np.sum((v - gu) ** 2))))
        hist["primal_res_tau"].append(float(np.sqrt(np.sum((w - gt) ** 2))))
        hist["primal_res_f"].append(float(np.sqrt(np.sum((f - tau_new) ** 2))))
        hist.setdefault("restart", []).append(bool(restart and E > E_prev))
        if restart and E > E_prev:
            t = 1.0
        E_prev = E
        if eps_stop > 0.0 and e <= eps_stop:
            break
    return u, tau, hist


def depth_map(u, rel_threshold=0.1):
    """Per-column argmax depth of u (ties to the smallest index); -1 where the
    column maximum is below rel_threshold * max(u)."""
    d = np.argmax(u, axis=2)
    colmax = np.max(u, axis=2)
    thr = rel_threshold * float(np.max(u)) if np.max(u) > 0 else np.inf
    return np.where(colmax >= thr, d, -1)
