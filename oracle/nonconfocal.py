"""FP64 oracle of the midpoint conversion of non-confocal transients into
confocal ones.

TEST INFRASTRUCTURE ONLY (see the package docstring): imported by tests/,
never by the product path.

Sec. 4 (evaluation on non-confocal data) runs the confocal solvers on a
non-confocal measurement after converting it with the midpoint approximation
of f-k migration; the paper cites the method without stating it.  Reading
used here, derived from the path lengths:

* A measurement with the laser at the wall point l and the detector at s is
  treated as a confocal measurement at the midpoint m = (l + s) / 2.
* For a scatterer on the wall normal through m at depth z the non-confocal
  path is 2 sqrt(z^2 + h^2) with h = |s - l| / 2, and the confocal path at m
  is 2 z.  The arrival times therefore satisfy
      t_nc^2 = t_c^2 + (|s - l| / c)^2,
  exactly for such scatterers and approximately for the others.
* The confocal transient at m is the non-confocal one read on that warp,
      tau_c(m, t_k) = tau_nc(s, sqrt(t_k^2 + (|s - l| / c)^2)),
  t_k = (k + 1/2) dt the bin centres, by two-tap linear interpolation between
  bin centres, zero outside the recorded bins; the amplitude is not changed.
* The detector grid s_ij = (x_i, y_j), x_i = (i + 1/2 - nx/2) W / nx (the
  scan grid of the confocal geometry), maps to the midpoint grid of spacing
  W / (2 nx) on a W/2 x W/2 patch centred at l / 2: the result is a confocal
  scan with wall width W / 2.

The source bin positions are computed in FP64 by the sequence of correctly
rounded operations written out in `midpoint_positions`.

Pins: tests/test_oracle_nonconfocal.py (zero offset is the identity, the
exact arrival time of a scatterer below the midpoint, the warp's
monotonicity and causality, linearity).
"""

import numpy as np

from .lct import C_LIGHT


def detector_centres(n, wall_width_m):
    """x_i = (i + 1/2 - n/2) * (W / n), the scan grid's lateral centres."""
    return (np.arange(n) + 0.5 - n / 2) * (wall_width_m / n)


def midpoint_positions(nx, ny, nt, bin_width_s, wall_width_m, laser_xy):
    """p[i, j, k]: the fractional non-confocal bin read by confocal bin k of
    column (i, j), p = sqrt(t_k^2 + q2_ij) * (1 / dt) - 1/2 with
    t_k = (k + 1/2) dt and q2_ij = ((x_i - l_x)^2 + (y_j - l_y)^2) / c^2."""
    dt = float(bin_width_s)
    inv_dt = 1.0 / dt
    x = detector_centres(nx, wall_width_m)
    y = detector_centres(ny, wall_width_m)
    dx = x[:, None] - float(laser_xy[0])
    dy = y[None, :] - float(laser_xy[1])
    q2 = (dx * dx + dy * dy) / (C_LIGHT * C_LIGHT)
    tk = (np.arange(nt) + 0.5) * dt
    tp = np.sqrt(tk[None, None, :] * tk[None, None, :] + q2[:, :, None])
    return tp * inv_dt - 0.5


def midpoint_confocal(tau_nc, bin_width_s, wall_width_m, laser_xy):
    """Confocal transients [nx][ny][nt] at the midpoints of the detector grid
    and the laser point, from non-confocal ones tau_nc [nx][ny][nt]."""
    tau_nc = np.asarray(tau_nc, dtype=np.float64)
    nx, ny, nt = tau_nc.shape
    p = midpoint_positions(nx, ny, nt, bin_width_s, wall_width_m, laser_xy)
    i0 = np.floor(p).astype(np.int64)
    w = p - i0

    def sample(idx):
        inside = (idx >= 0) & (idx < nt)
        vals = np.take_along_axis(tau_nc, np.clip(idx, 0, nt - 1), axis=2)
        return np.where(inside, vals, 0.0)

    return (1.0 - w) * sample(i0) + w * sample(i0 + 1)
