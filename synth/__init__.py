"""Seeded synthetic inputs shared by the tests, the bench and the oracle checks.

This module holds NO arithmetic of the reconstruction method: it draws
hidden-scene albedo volumes, scan masks and Poisson photon counts.  The
measurement's noiseless signal (the forward model applied to the scene) is
passed in by the caller, who computes it with the operator under test or
with the oracle.

Scenes are self-generated stand-ins shaped like the paper's workloads
(64x64 / 32x32 scans over a 1 m wall, 256 bins of 32 ps or 512 of 16 ps,
planar and curved surfaces at 0.3-0.9 of the range); none of the paper's
datasets is reproduced.
"""

import numpy as np


def stride_mask(nx, ny, stride):
    """Regular under-sampling: keep (i, j) with i = j = floor(stride/2) mod stride."""
    m = np.zeros((nx, ny), dtype=np.uint8)
    o = stride // 2
    m[o::stride, o::stride] = 1
    return m


def random_mask(nx, ny, fraction, seed):
    """Exactly round(fraction * nx * ny) sampled points, chosen by a seeded permutation."""
    rng = np.random.default_rng(seed)
    k = int(round(fraction * nx * ny))
    idx = rng.permutation(nx * ny)[:k]
    m = np.zeros(nx * ny, dtype=np.uint8)
    m[idx] = 1
    return m.reshape(nx, ny)


def _glyph_L(vol, rng, nx, ny, nt, albedo):
    """A thin 'L': a 2-voxel-wide vertical stroke 12 tall and a 2-wide foot 8 long."""
    h, w = min(12, nx - 2), min(8, ny - 2)
    x0 = int(rng.integers(0, max(1, nx - h)))
    y0 = int(rng.integers(0, max(1, ny - w)))
    z = int(np.floor(nt * rng.uniform(0.3, 0.9)))
    vol[x0:x0 + h, y0:y0 + 2, z] = albedo
    vol[x0 + h - 2:x0 + h, y0:y0 + w, z] = albedo


def scene_planes_glyph(nx, ny, nt, seed):
    """Two fronto-parallel rectangular patches (sides U{6..14} voxels, one voxel
    thick, depth floor(nt U[0.3, 0.9])) plus an L-shaped glyph; albedo U[0.3, 1]."""
    rng = np.random.default_rng(seed)
    vol = np.zeros((nx, ny, nt), dtype=np.float64)
    for _ in range(2):
        sx = int(rng.integers(6, 15))
        sy = int(rng.integers(6, 15))
        sx, sy = min(sx, nx - 1), min(sy, ny - 1)
        x0 = int(rng.integers(0, nx - sx + 1))
        y0 = int(rng.integers(0, ny - sy + 1))
        z = int(np.floor(nt * rng.uniform(0.3, 0.9)))
        vol[x0:x0 + sx, y0:y0 + sy, z] = rng.uniform(0.3, 1.0)
    _glyph_L(vol, rng, nx, ny, nt, rng.uniform(0.3, 1.0))
    return vol


def scene_patches(nx, ny, nt, seed, n_min=3, n_max=5, albedo_lo=0.2):
    """3-5 random patches: tilted planes (depth linear across the patch) or
    spherical caps (depth z0 + r^2 / (2 Rc), Rc in [20, 60] voxels);
    albedo U[albedo_lo, 1]; one voxel per (x, y) column of the patch."""
    rng = np.random.default_rng(seed)
    vol = np.zeros((nx, ny, nt), dtype=np.float64)
    n = int(rng.integers(n_min, n_max + 1))
    for _ in range(n):
        sx = int(rng.integers(max(4, nx // 8), max(5, nx // 3)))
        sy = int(rng.integers(max(4, ny // 8), max(5, ny // 3)))
        x0 = int(rng.integers(0, nx - sx + 1))
        y0 = int(rng.integers(0, ny - sy + 1))
        z0 = nt * rng.uniform(0.3, 0.8)
        alb = rng.uniform(albedo_lo, 1.0)
        xs = np.arange(sx) - (sx - 1) / 2.0
        ys = np.arange(sy) - (sy - 1) / 2.0
        X, Y = np.meshgrid(xs, ys, indexing="ij")
        if rng.uniform() < 0.5:
            gx, gy = rng.uniform(-0.5, 0.5, size=2) * (nt / nx) * 0.25
            depth = z0 + gx * X + gy * Y
        else:
            rc = rng.uniform(20.0, 60.0)
            depth = z0 + (X * X + Y * Y) / (2.0 * rc) * (nt / nx) * 0.25
        zi = np.clip(np.floor(depth), 0, nt - 1).astype(np.int64)
        vol[x0 + np.arange(sx)[:, None], y0 + np.arange(sy)[None, :], zi] = alb
    return vol


def poisson_measurement(signal, mask, peak, background, seed):
    """Photon counts y ~ Poisson(peak * signal / max(signal) + background) on the
    sampled columns, normalised tau0 = y / max(y); zero off the mask."""
    rng = np.random.default_rng(seed)
    s = np.asarray(signal, dtype=np.float64)
    smax = float(np.max(s))
    lam = peak * (s / smax if smax > 0 else s) + background
    lam = np.maximum(lam, 0.0)
    y = rng.poisson(lam).astype(np.float64)
    y *= np.asarray(mask, dtype=np.float64)[:, :, None]
    ymax = float(np.max(y))
    return y / ymax if ymax > 0 else y


def _lcg_uniforms(seed, n):
    """n numbers in [0, 1) from a 64-bit linear congruential sequence (integer
    arithmetic only, so identical on every platform and numpy version)."""
    x = (int(seed) * 6364136223846793005 + 1442695040888963407) % (1 << 64)
    out = []
    for _ in range(n):
        x = (x * 6364136223846793005 + 1442695040888963407) % (1 << 64)
        out.append((x >> 11) / float(1 << 53))
    return out


def pulse_transients(nx, ny, nt, mask, seed, width_bins=1.5, floor=0.02):
    """Seeded synthetic transients without random sampling: every sampled
    column holds a main return at a depth that varies smoothly across the
    wall (0.35-0.75 of the range), a weaker second return behind it on part
    of the wall, and a constant floor; normalised to max 1, zero off the mask.
    Built from closed-form functions and integer-generated phases only, so
    both sides of a comparison can regenerate it on any machine."""
    u = _lcg_uniforms(seed, 6)
    x = (np.arange(nx) + 0.5)[:, None] / nx
    y = (np.arange(ny) + 0.5)[None, :] / ny
    d1 = nt * (0.55 + 0.15 * np.sin(2 * np.pi * (x + u[0])) * np.cos(2 * np.pi * (y + u[1])))
    d2 = d1 + nt * (0.08 + 0.04 * u[2])
    a1 = 0.6 + 0.4 * np.cos(np.pi * (x - u[3])) ** 2
    a2 = 0.35 * (np.sin(2 * np.pi * (x + y + u[4])) > 0.2 * (2 * u[5] - 1))
    t = np.arange(nt)[None, None, :]
    sig = (a1[:, :, None] * np.exp(-0.5 * ((t - d1[:, :, None]) / width_bins) ** 2)
           + a2[:, :, None] * np.exp(-0.5 * ((t - d2[:, :, None]) / width_bins) ** 2) + floor)
    sig *= np.asarray(mask, dtype=np.float64)[:, :, None]
    m = float(np.max(sig))
    return sig / m if m > 0 else sig


# Workloads used by the tests and the bench (sizes and parameters of the
# paper's experiments; see the design notes for the recipe).
CONFIGS = {
    "c1_alg1_32x32x256": dict(nx=32, ny=32, nt=256, bin_width_s=32e-12, stride=2,
                              scene="planes_glyph", peak=100.0, background=1.0,
                              model=1, iters=30, a=9e-5, b=2e-5, mu=0.1),
    "c2_alg2_64x64x512": dict(nx=64, ny=64, nt=512, bin_width_s=16e-12, stride=2,
                              scene="patches", peak=50.0, background=2.0,
                              model=2, iters=100, lam=235.0, a_u=2e-4, b_u=4.5e-4,
                              a_tau=4e-4, b_tau=3e-2, mu1=1.0, mu2=800.0, mu3=2.0),
    "headline_128x128x512": dict(nx=128, ny=128, nt=512, bin_width_s=16e-12, stride=4,
                                 scene="patches", peak=50.0, background=2.0,
                                 model=1, iters=50, a=9e-5, b=2e-5, mu=0.1,
                                 lam=235.0, a_u=2e-4, b_u=4.5e-4,
                                 a_tau=4e-4, b_tau=3e-2, mu1=1.0, mu2=800.0, mu3=2.0),
    # precision case: 8 ps bins over the same 1.2288 m range, 32x32 sampled
    "c4_alg1_128x128x1024": dict(nx=128, ny=128, nt=1024, bin_width_s=8e-12, stride=4,
                                 scene="pulses", model=1, iters=12, a=9e-5, b=2e-5, mu=0.1),
}


def make_volume(cfg, seed):
    if cfg["scene"] == "planes_glyph":
        return scene_planes_glyph(cfg["nx"], cfg["ny"], cfg["nt"], seed)
    return scene_patches(cfg["nx"], cfg["ny"], cfg["nt"], seed)


def make_mask(cfg, seed=0):
    if "stride" in cfg:
        return stride_mask(cfg["nx"], cfg["ny"], cfg["stride"])
    return random_mask(cfg["nx"], cfg["ny"], cfg.get("fraction", 0.25), seed)
