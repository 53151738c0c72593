"""Writes tests/golden/headline_alg2_128x128x512.npz: the FP64 oracle's
Algorithm-2 reconstruction at the benchmark's size (128 x 128 x 512, 16 ps
bins, 32 x 32 stride-4 sampling; lambda, a_u, b_u, a_tau, b_tau and mu_1..3
of the Bowling settings), 50 iterations, tau0 the seeded pulse transients.
The GPU test runs it as one graph launch, as the benchmark's Algorithm-2
line does.

Only oracle/ and synth/ are used.  Stored: the energy history and restart
flags, the Lipschitz estimates, the global 2-norms of u and tau, the depth
map of u, and u and tau on 96 fixed columns (every 256th column index plus
the 32 sampled columns of one row).

    PYTHONPATH=. python tests/golden/make_headline_alg2.py     (about 60 minutes)
"""
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import synth  # noqa: E402
from oracle import admm, lct  # noqa: E402

NAME = "headline_alg2_128x128x512"
ITERS = 50
SEED = 2


def golden_columns(nx, ny):
    cols = list(range(0, nx * ny, 256))                   # spread over the wall
    row = 2 * ny                                         # sampled row x = 2 (stride 4, offset 2)
    cols += [row + j for j in range(2, ny, 4)]           # its 32 sampled columns
    return np.array(sorted(set(cols)), dtype=np.int32)


def main():
    cfg = synth.CONFIGS["headline_128x128x512"]
    nx, ny, nt = cfg["nx"], cfg["ny"], cfg["nt"]
    mask = synth.make_mask(cfg)
    tau0 = synth.pulse_transients(nx, ny, nt, mask, seed=SEED)
    g = lct.Geometry(nx, ny, nt, cfg["bin_width_s"])
    op = lct.Operator(g, mask)
    t0 = time.time()
    u, tau, hist = admm.alg2(tau0, mask, g, cfg["a_u"], cfg["b_u"], cfg["a_tau"], cfg["b_tau"], cfg["lam"],
                             cfg["mu1"], cfg["mu2"], cfg["mu3"], ITERS, op=op)
    cols = golden_columns(nx, ny)
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), NAME + ".npz")
    np.savez_compressed(out, cols=cols, u_cols=u.reshape(nx * ny, nt)[cols].astype(np.float32),
                        tau_cols=tau.reshape(nx * ny, nt)[cols].astype(np.float32),
                        depth=admm.depth_map(u).astype(np.int16), energy=np.array(hist["E"]),
                        restart=np.array(hist["restart"], dtype=np.int8), L=np.array(hist["L"]),
                        norm_u=np.linalg.norm(u), norm_tau=np.linalg.norm(tau), iters=ITERS, seed=SEED)
    print(f"wrote {out} in {time.time() - t0:.0f} s; E = {hist['E'][-1]:.6g}, restarts {sum(hist['restart'])}")


if __name__ == "__main__":
    main()
