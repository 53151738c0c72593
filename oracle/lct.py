"""FP64 oracle of the discrete confocal light-cone-transform operator.

TEST INFRASTRUCTURE ONLY (see the package docstring): imported by tests/,
__graft_entry__.smoke() and bench.py's CPU-baseline legs, never by the
product path.

The paper states the confocal volumetric-albedo model (Sec. 2, Eq. 2)

    tau(x', t) = integral over the hidden half-space of u(x) / d(x', x)^4
                 * delta(2 d(x', x) - t c) dx

and its discrete form (Eq. 3) tau = A u = R_t^{-1} H R_z u, where H is a
shift-invariant 3-D convolution and R_t, R_z act on the time and depth axes.
It does not spell out the discretisation.  This module writes out the reading
used throughout the library (every choice below is one of the readings listed
in the design notes):

* Geometry.  Range R = c * nt * bin_width / 2.  Depth bin k and time bin k
  share the normalised coordinate rho_k = (k + 1/2) / nt (depth z = rho R,
  time t = 2 rho R / c).  The scan grid and the voxel grid share lateral
  centres x_i = (i + 1/2 - nx/2) * W / nx on a W x W wall patch.
* Change of variables (from Eq. 2, substituting v = (z/R)^2 and
  nu = (ct/(2R))^2):  nu^{3/2} tau(nu) = [h * u~](nu) with
  u~(v) = u(sqrt v) / (2 sqrt v) and h(x, y, w) = delta(x^2 + y^2 - w),
  lateral coordinates in units of R.
* R_z:  on the v-grid v_j = (j + 1/2)/nt, u~_j is the two-tap linear
  interpolation of u on the rho-grid at rho = sqrt(v_j), times 1/(2 sqrt v_j).
* H:  linear (non-circular) convolution with the cone kernel
  h[i, j, m] = max(0, 1 - |m - w_ij|), w_ij = nt ((i dx)^2 + (j dy)^2) / R^2,
  for |i| < nx, |j| < ny, 0 <= m < nt, scaled to unit L2 norm.
* R_t^{-1}:  tau_k = wt_k * [two-tap linear interpolation of the convolution
  output on the v-grid at v = rho_k^2].  wt_k = rho_k^{-3} is the raw
  radiometry of Eq. 2 (``radiometry='raw'``).  ``radiometry='compensated'``
  (the default) models the transient already multiplied by t^4, the usual
  compensation of the 1/d^4 fall-off, so wt_k = rho_k^{-3} * rho_k^4 = rho_k.
* Interpolation clamps at the grid ends: a sample position p is clipped to
  [0, n-1], i0 = min(floor(p), n-2), frac = p - i0.
* D (Sec. 3, below Eq. 8: A_D = D A) keeps the measured scan columns; the
  missing region X is the complement of the mask.

Pins: tests/test_oracle_lct.py (brute-force convolution, direct summation of
Eq. 2, partition of unity of the kernel, adjoint identity and explicit
matrix transpose, power iteration against an SVD).
"""

from dataclasses import dataclass

import numpy as np

C_LIGHT = 299_792_458.0  # m/s

RADIOMETRY = ("compensated", "raw")


@dataclass(frozen=True)
class Geometry:
    """Scan/volume geometry of one confocal scene (Sec. 2)."""

    nx: int
    ny: int
    nt: int
    bin_width_s: float
    wall_width_m: float = 1.0
    radiometry: str = "compensated"

    def __post_init__(self):
        for n in (self.nx, self.ny, self.nt):
            if n < 2 or (n & (n - 1)) != 0:
                raise ValueError("nx, ny, nt must be powers of two >= 2")
        if self.radiometry not in RADIOMETRY:
            raise ValueError(f"radiometry must be one of {RADIOMETRY}")

    @property
    def range_m(self) -> float:
        """R = c * nt * bin_width / 2: the depth covered by the time axis."""
        return C_LIGHT * self.nt * self.bin_width_s / 2.0

    @property
    def shape(self):
        return (self.nx, self.ny, self.nt)


def _two_tap(p, n):
    """Clamped linear-interpolation taps for sample positions p on an n-grid."""
    p = np.clip(p, 0.0, float(n - 1))
    i0 = np.minimum(np.floor(p), n - 2).astype(np.int64)
    frac = p - i0
    return i0, 1.0 - frac, frac


def rz_table(nt):
    """R_z taps: for v-bin j, (i0_j, w0_j, w1_j, g_j) with
    u~_j = g_j * (w0_j u[i0_j] + w1_j u[i0_j + 1]),  g_j = 1 / (2 sqrt v_j).

    The rho-grid position of rho = sqrt(v_j) is sqrt((j + 1/2) nt) - 1/2.
    """
    j = np.arange(nt, dtype=np.float64)
    p = np.sqrt((j + 0.5) * nt) - 0.5
    i0, w0, w1 = _two_tap(p, nt)
    g = 1.0 / (2.0 * np.sqrt((j + 0.5) / nt))
    return i0, w0, w1, g


def rt_table(nt, radiometry="compensated"):
    """R_t^{-1} taps: for time bin k, (k0_k, w0_k, w1_k, wt_k) with
    tau_k = wt_k * (w0_k c[k0_k] + w1_k c[k0_k + 1]).

    The v-grid position of v = rho_k^2 is (k + 1/2)^2 / nt - 1/2 (exact in
    FP64 for power-of-two nt).  wt_k = rho_k^{-3} (raw) or rho_k (compensated).
    """
    k = np.arange(nt, dtype=np.float64)
    q = (k + 0.5) ** 2 / nt - 0.5
    k0, w0, w1 = _two_tap(q, nt)
    rho = (k + 0.5) / nt
    if radiometry == "raw":
        wt = 1.0 / (rho * rho * rho)
    elif radiometry == "compensated":
        wt = rho.copy()
    else:
        raise ValueError(radiometry)
    return k0, w0, w1, wt


def cone_weights(geom: Geometry):
    """Lateral cone offsets: w_ij = nt ((i dx)^2 + (j dy)^2) / R^2 for
    i in (-nx, nx), j in (-ny, ny); returned as an array indexed [i + nx - 1, j + ny - 1]."""
    dx = geom.wall_width_m / geom.nx
    dy = geom.wall_width_m / geom.ny
    R = geom.range_m
    i = np.arange(-(geom.nx - 1), geom.nx, dtype=np.float64)
    j = np.arange(-(geom.ny - 1), geom.ny, dtype=np.float64)
    s = (i[:, None] * dx) * (i[:, None] * dx) + (j[None, :] * dy) * (j[None, :] * dy)
    return geom.nt * s / (R * R)


def cone_kernel(geom: Geometry, normalise=True):
    """Cone kernel h on the lateral-periodic grid (2nx, 2ny, nt).

    h[i mod 2nx, j mod 2ny, m] = max(0, 1 - |m - w_ij|) for 0 <= m < nt: the
    delta(x^2 + y^2 - w) of the transformed model splatted onto the v-axis
    with a linear hat.  With ``normalise`` the kernel is scaled to unit L2 norm.
    """
    nx, ny, nt = geom.shape
    w = cone_weights(geom)
    m = np.arange(nt, dtype=np.float64)
    cols = np.maximum(0.0, 1.0 - np.abs(m[None, None, :] - w[:, :, None]))
    h = np.zeros((2 * nx, 2 * ny, nt))
    ii = np.arange(-(nx - 1), nx) % (2 * nx)
    jj = np.arange(-(ny - 1), ny) % (2 * ny)
    h[np.ix_(ii, jj)] = cols
    if normalise:
        h /= np.sqrt(np.sum(h * h))
    return h


# ---------------------------------------------------------------------------
# The three factors of A = R_t^{-1} H R_z (Eq. 3) and their transposes.
# ---------------------------------------------------------------------------

def apply_rz(u, nt):
    i0, w0, w1, g = rz_table(nt)
    return g * (w0 * u[..., i0] + w1 * u[..., i0 + 1])


def apply_rz_t(ut, nt):
    i0, w0, w1, g = rz_table(nt)
    out = np.zeros_like(ut)
    np.add.at(out, (Ellipsis, i0), g * w0 * ut)
    np.add.at(out, (Ellipsis, i0 + 1), g * w1 * ut)
    return out


def apply_rt_inv(c, nt, radiometry):
    k0, w0, w1, wt = rt_table(nt, radiometry)
    return wt * (w0 * c[..., k0] + w1 * c[..., k0 + 1])


def apply_rt_inv_t(tau, nt, radiometry):
    k0, w0, w1, wt = rt_table(nt, radiometry)
    out = np.zeros_like(tau)
    np.add.at(out, (Ellipsis, k0), wt * w0 * tau)
    np.add.at(out, (Ellipsis, k0 + 1), wt * w1 * tau)
    return out


def kernel_spectrum(geom: Geometry):
    """3-D real FFT of h zero-padded to (2nx, 2ny, 2nt)."""
    nx, ny, nt = geom.shape
    hp = np.zeros((2 * nx, 2 * ny, 2 * nt))
    hp[:, :, :nt] = cone_kernel(geom)
    return np.fft.rfftn(hp)


def apply_h(x, geom: Geometry, hk=None):
    """Linear 3-D convolution with h, output cropped to the volume grid.

    out[x, y, n] = sum over (x', y', v <= n) of h[x - x', y - y', n - v] x[x', y', v].
    Computed as a circular convolution on the zero-padded (2nx, 2ny, 2nt) grid,
    which equals the linear one on the cropped range.
    """
    nx, ny, nt = geom.shape
    if hk is None:
        hk = kernel_spectrum(geom)
    xp = np.zeros((2 * nx, 2 * ny, 2 * nt))
    xp[:nx, :ny, :nt] = x
    y = np.fft.irfftn(np.fft.rfftn(xp) * hk, s=xp.shape, axes=(0, 1, 2))
    return y[:nx, :ny, :nt]


def apply_h_t(y, geom: Geometry, hk=None):
    """Transpose of apply_h: correlation with h, cropped."""
    nx, ny, nt = geom.shape
    if hk is None:
        hk = kernel_spectrum(geom)
    yp = np.zeros((2 * nx, 2 * ny, 2 * nt))
    yp[:nx, :ny, :nt] = y
    x = np.fft.irfftn(np.fft.rfftn(yp) * np.conj(hk), s=yp.shape, axes=(0, 1, 2))
    return x[:nx, :ny, :nt]


def brute_force_h(x, geom: Geometry):
    """apply_h by direct summation over the kernel's nonzero taps (tiny grids)."""
    nx, ny, nt = geom.shape
    h = cone_kernel(geom)
    out = np.zeros((nx, ny, nt))
    for di in range(-(nx - 1), nx):
        for dj in range(-(ny - 1), ny):
            col = h[di % (2 * nx), dj % (2 * ny)]
            for m in np.nonzero(col)[0]:
                # out[x + di, y + dj, v + m] += h * x[x, y, v]
                xs = slice(max(0, -di), min(nx, nx - di))
                ys = slice(max(0, -dj), min(ny, ny - dj))
                xd = slice(xs.start + di, xs.stop + di)
                yd = slice(ys.start + dj, ys.stop + dj)
                out[xd, yd, m:] += col[m] * x[xs, ys, : nt - m]
    return out


class Operator:
    """A = R_t^{-1} H R_z (Eq. 3) with its transpose and the sampling D.

    ``mask`` is an (nx, ny) array of {0, 1}; A_D = D A keeps the sampled
    columns (zero elsewhere) and A_D^T r = A^T (D r).
    """

    def __init__(self, geom: Geometry, mask=None):
        self.geom = geom
        self.hk = kernel_spectrum(geom)
        if mask is None:
            mask = np.ones((geom.nx, geom.ny), dtype=np.uint8)
        self.mask = np.asarray(mask, dtype=np.uint8)
        self.M = self.mask.astype(np.float64)[:, :, None]

    def forward(self, u):
        g = self.geom
        return apply_rt_inv(apply_h(apply_rz(u, g.nt), g, self.hk), g.nt, g.radiometry)

    def adjoint(self, tau):
        g = self.geom
        return apply_rz_t(apply_h_t(apply_rt_inv_t(tau, g.nt, g.radiometry), g, self.hk), g.nt)

    def forward_d(self, u):
        return self.M * self.forward(u)

    def adjoint_d(self, r):
        return self.adjoint(self.M * r)


def sampled_columns(mask):
    """Compact list of sampled scan columns, ascending in x * ny + y (D of Sec. 3)."""
    m = np.asarray(mask).reshape(-1)
    return np.nonzero(m)[0].astype(np.int32)


def explicit_matrix(op: Operator, masked=True):
    """Dense matrix of A (or A_D) from unit vectors; tiny grids only."""
    g = op.geom
    V = g.nx * g.ny * g.nt
    Mx = np.zeros((V, V))
    for c in range(V):
        e = np.zeros(V)
        e[c] = 1.0
        e = e.reshape(g.shape)
        Mx[:, c] = (op.forward_d(e) if masked else op.forward(e)).ravel()
    return Mx


def power_norm2(op: Operator, masked=True, max_iter=200, rtol=1e-12):
    """||A_D||_2^2 by power iteration on A_D^T A_D from the all-ones vector.

    The estimate at each step is the Rayleigh quotient ||A_D x||^2 of the
    unit vector x; the iteration stops when it changes by less than
    rtol (relative) or after max_iter steps.  Returns (estimate, steps).
    """
    g = op.geom
    fwd = op.forward_d if masked else op.forward
    adj = op.adjoint_d if masked else op.adjoint
    x = np.ones(g.shape)
    x /= np.sqrt(np.sum(x * x))
    lam = 0.0
    for it in range(1, max_iter + 1):
        y = fwd(x)
        lam_new = float(np.sum(y * y))
        z = adj(y)
        nz = np.sqrt(np.sum(z * z))
        if nz == 0.0:
            return 0.0, it
        x = z / nz
        if it > 1 and abs(lam_new - lam) <= rtol * lam_new:
            return lam_new, it
        lam = lam_new
    return lam, max_iter


def direct_summation(u, geom: Geometry):
    """Eq. 2 summed voxel by voxel: tau(x', k) = sum u / d^4 * hat_k(2 d / (c dt)).

    Voxel centres at lateral x_i and depth z = rho_k R; time bin k has centre
    (k + 1/2) dt and hat_k(s) = max(0, 1 - |s - 1/2 - k|) splats the arrival
    time s (in bins) linearly onto the two nearest bins.  With compensated
    radiometry the result is multiplied by rho_k^4 (the t^4 compensation).
    Physical constants are not absorbed: compare after a global scale fit.
    """
    nx, ny, nt = geom.shape
    W, R, dt = geom.wall_width_m, geom.range_m, geom.bin_width_s
    xs = (np.arange(nx) + 0.5 - nx / 2) * W / nx
    ys = (np.arange(ny) + 0.5 - ny / 2) * W / ny
    zs = (np.arange(nt) + 0.5) / nt * R
    tau = np.zeros((nx, ny, nt))
    vox = np.argwhere(u != 0)
    for (a, b, c) in vox:
        d = np.sqrt((xs[:, None] - xs[a]) ** 2 + (ys[None, :] - ys[b]) ** 2 + zs[c] ** 2)
        s = 2.0 * d / (C_LIGHT * dt) - 0.5  # arrival position in bin-centre units
        k0 = np.floor(s).astype(np.int64)
        f = s - k0
        amp = u[a, b, c] / d ** 4
        for kk, wgt in ((k0, 1.0 - f), (k0 + 1, f)):
            ok = (kk >= 0) & (kk < nt)
            ii, jj = np.nonzero(ok)
            np.add.at(tau, (ii, jj, kk[ok]), (amp * wgt)[ok])
    if geom.radiometry == "compensated":
        rho = (np.arange(nt) + 0.5) / nt
        tau *= rho ** 4
    return tau


# ---------------------------------------------------------------------------
# Directional (normal-weighted) confocal model (Sec. 2)
# ---------------------------------------------------------------------------

def directional_terms(geom: Geometry, normals):
    """The six (input field factor, output weight) pairs of the directional
    confocal operator, coordinates in units of the range R.

    The paper's non-confocal direction-albedo model (Sec. 2) weights u(x) by
    the two cosines ((x'_i - x) . n / d_i) ((x'_d - x) . n / d_d) on top of the
    albedo model's fall-off; with illumination and detection at the same wall
    point x' (the confocal case) the weight is ((x' - x) . n(x))^2 / d^2.
    Reading: this is the directional model "before the albedo reduction"
    (the printed confocal formula writes the two normal factors without the
    direction, n . n, which is 1 for unit normals).  With n = (a, b, c) and
    g = X a + Y b + Z c (X, Y the voxel's lateral coordinates, Z its depth),
    (x' - x) . n = X' a + Y' b - g, and its square expands into
        X'^2 a^2 + Y'^2 b^2 + g^2 + 2 X'Y' a b - 2 X' a g - 2 Y' b g,
    a sum of products of a field on the voxel grid and a weight on the scan
    point, so tau = sum_t w_t(x', t) A(f_t u) with the albedo operator A of
    Eq. 3 and w_t including 1 / d^2 = 1 / rho_t^2 (distance of the time bin's
    cone, rho_t = (k + 1/2) / nt).  Returns [(f_t, w_t)], f_t of the volume's
    shape, w_t of shape (nx, ny, nt)."""
    nx, ny, nt = geom.shape
    W, R = geom.wall_width_m, geom.range_m
    X = (np.arange(nx) + 0.5 - nx / 2) * W / nx / R
    Y = (np.arange(ny) + 0.5 - ny / 2) * W / ny / R
    Z = (np.arange(nt) + 0.5) / nt
    a, b, c = (np.asarray(n, dtype=np.float64) for n in normals)
    g = X[:, None, None] * a + Y[None, :, None] * b + Z[None, None, :] * c
    inv_d2 = 1.0 / (Z * Z)                       # time bin k: d / R = (k + 1/2) / nt
    Xp = np.broadcast_to(X[:, None, None], geom.shape)
    Yp = np.broadcast_to(Y[None, :, None], geom.shape)
    w = lambda s: s * inv_d2[None, None, :]      # noqa: E731
    return [(a * a, w(Xp * Xp)), (b * b, w(Yp * Yp)), (g * g, w(np.ones(geom.shape))),
            (a * b, w(2.0 * Xp * Yp)), (a * g, w(-2.0 * Xp)), (b * g, w(-2.0 * Yp))]


def directional_forward(op: Operator, u, normals, masked=True):
    """tau = D sum_t w_t A(f_t u): the directional confocal model (see
    directional_terms) on the plan's discretisation of A (Eq. 3)."""
    tau = np.zeros(op.geom.shape)
    for f, w in directional_terms(op.geom, normals):
        tau += w * op.forward(f * u)
    return op.M * tau if masked else tau


def directional_adjoint(op: Operator, tau, normals, masked=True):
    """Transpose of directional_forward: sum_t f_t A^T(w_t D^T tau)."""
    r = op.M * tau if masked else tau
    u = np.zeros(op.geom.shape)
    for f, w in directional_terms(op.geom, normals):
        u += f * op.adjoint(w * r)
    return u


def directional_direct_summation(u, normals, geom: Geometry):
    """The directional confocal model summed voxel by voxel: as
    direct_summation, with each voxel's contribution weighted by
    ((x' - x) . n(x) / d)^2."""
    nx, ny, nt = geom.shape
    W, R, dt = geom.wall_width_m, geom.range_m, geom.bin_width_s
    xs = (np.arange(nx) + 0.5 - nx / 2) * W / nx
    ys = (np.arange(ny) + 0.5 - ny / 2) * W / ny
    zs = (np.arange(nt) + 0.5) / nt * R
    a, b, c = (np.asarray(n, dtype=np.float64) for n in normals)
    tau = np.zeros((nx, ny, nt))
    for (p, q, s) in np.argwhere(u != 0):
        dxw = xs[:, None] - xs[p]
        dyw = ys[None, :] - ys[q]
        d = np.sqrt(dxw ** 2 + dyw ** 2 + zs[s] ** 2)
        cosv = (dxw * a[p, q, s] + dyw * b[p, q, s] - zs[s] * c[p, q, s]) / d
        pos = 2.0 * d / (C_LIGHT * dt) - 0.5
        k0 = np.floor(pos).astype(np.int64)
        fr = pos - k0
        amp = u[p, q, s] * cosv * cosv / d ** 4
        for kk, wgt in ((k0, 1.0 - fr), (k0 + 1, fr)):
            ok = (kk >= 0) & (kk < nt)
            ii, jj = np.nonzero(ok)
            np.add.at(tau, (ii, jj, kk[ok]), (amp * wgt)[ok])
    if geom.radiometry == "compensated":
        rho = (np.arange(nt) + 0.5) / nt
        tau *= rho ** 4
    return tau
