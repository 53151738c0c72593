"""Writes tests/golden/headline_alg1_128x128x512.npz: the FP64 oracle's
Algorithm-1 reconstruction at the benchmark's size (128 x 128 x 512, 16 ps
bins, 32 x 32 stride-4 sampling; a, b, mu of the Bowling settings), 50
iterations, tau0 the seeded pulse transients.

Only oracle/ and synth/ are used.  Stored: the energy history, the Lipschitz
estimates, the global 2-norm and sum of u, the depth map of u, and u on 64
fixed columns (every 256th column index plus the 32 sampled columns of one
row), so a GPU run at the benchmark's launch configuration can be compared
without the 34 MB volume.

    PYTHONPATH=. python tests/golden/make_headline_alg1.py     (about 25 minutes)
"""
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import synth  # noqa: E402
from oracle import admm, lct  # noqa: E402

NAME = "headline_alg1_128x128x512"
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
    u, hist = admm.alg1(tau0, mask, g, cfg["a"], cfg["b"], cfg["mu"], ITERS, op=op)
    cols = golden_columns(nx, ny)
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), NAME + ".npz")
    np.savez_compressed(out, cols=cols, u_cols=u.reshape(nx * ny, nt)[cols].astype(np.float32),
                        depth=admm.depth_map(u).astype(np.int16), energy=np.array(hist["E"]),
                        L=np.array(hist["L"]), norm=np.linalg.norm(u), total=float(np.sum(u)),
                        iters=ITERS, seed=SEED)
    print(f"wrote {out} in {time.time() - t0:.0f} s; E = {hist['E'][-1]:.6g}, backtracks {sum(hist['backtracks'])}")


if __name__ == "__main__":
    main()
