"""Writes tests/golden/c2_alg2_64x64x512.npz: the FP64 oracle's Algorithm-2
reconstruction of the dual-domain case (64 x 64 x 512, 16 ps bins, 32 x 32
stride-2 sampling, 100 iterations; lambda, a_u, b_u, a_tau, b_tau and
mu_1..3 of the Bowling settings), tau0 the seeded pulse transients.

Only oracle/ and synth/ are used.  Stored: the energy history and restart
flags, the Lipschitz estimates, the global 2-norms of u and tau, the depth
map of u, and u and tau on 96 fixed columns (every 64th column index plus
the 32 sampled columns of one row).

    PYTHONPATH=. python tests/golden/make_c2_alg2.py     (about 20 minutes)
"""
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import synth  # noqa: E402
from oracle import admm, lct  # noqa: E402

NAME = "c2_alg2_64x64x512"


def golden_columns(nx, ny):
    cols = list(range(0, nx * ny, 64))
    row = 1 * ny                                          # sampled row x = 1 (stride 2, offset 1)
    cols += [row + j for j in range(1, ny, 2)]
    return np.array(sorted(set(cols)), dtype=np.int32)


def main():
    cfg = synth.CONFIGS["c2_alg2_64x64x512"]
    nx, ny, nt = cfg["nx"], cfg["ny"], cfg["nt"]
    mask = synth.make_mask(cfg)
    tau0 = synth.pulse_transients(nx, ny, nt, mask, seed=1)
    g = lct.Geometry(nx, ny, nt, cfg["bin_width_s"])
    op = lct.Operator(g, mask)
    t0 = time.time()
    u, tau, hist = admm.alg2(tau0, mask, g, cfg["a_u"], cfg["b_u"], cfg["a_tau"], cfg["b_tau"], cfg["lam"],
                             cfg["mu1"], cfg["mu2"], cfg["mu3"], cfg["iters"], op=op)
    cols = golden_columns(nx, ny)
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), NAME + ".npz")
    np.savez_compressed(out, cols=cols, u_cols=u.reshape(nx * ny, nt)[cols].astype(np.float32),
                        tau_cols=tau.reshape(nx * ny, nt)[cols].astype(np.float32),
                        depth=admm.depth_map(u).astype(np.int16), energy=np.array(hist["E"]),
                        restart=np.array(hist["restart"], dtype=np.int8), L=np.array(hist["L"]),
                        norm_u=np.linalg.norm(u), norm_tau=np.linalg.norm(tau), iters=cfg["iters"])
    print(f"wrote {out} in {time.time() - t0:.0f} s; E = {hist['E'][-1]:.6g}, restarts {sum(hist['restart'])}")


if __name__ == "__main__":
    main()
