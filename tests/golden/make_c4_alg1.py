"""Writes tests/golden/c4_alg1_128x128x1024.npz: the FP64 oracle's Algorithm-1
reconstruction of the 128 x 128 x 1024 precision case (8 ps bins, 32 x 32
stride-4 sampling, seeded pulse transients as tau0).

Only oracle/ and synth/ are used.  Stored: the energy history, the global
2-norm and sum of u, the depth map (argmax over t, -1 where the column
maximum is below 0.1 max u), and u on 64 fixed columns (every 256th column
index plus the 32 columns of one sampled row), so a GPU run of the same
configuration can be compared without the 67 MB volume.

    PYTHONPATH=. python tests/golden/make_c4_alg1.py     (about 15 minutes)
"""
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import synth  # noqa: E402
from oracle import admm, lct  # noqa: E402

NAME = "c4_alg1_128x128x1024"


def golden_columns(nx, ny):
    cols = list(range(0, nx * ny, 256))                   # spread over the wall
    row = 2 * ny                                         # sampled row x = 2 (stride 4, offset 2)
    cols += [row + j for j in range(2, ny, 4)]           # its 32 sampled columns
    return np.array(sorted(set(cols)), dtype=np.int32)


def main():
    cfg = synth.CONFIGS[NAME]
    nx, ny, nt = cfg["nx"], cfg["ny"], cfg["nt"]
    mask = synth.make_mask(cfg)
    tau0 = synth.pulse_transients(nx, ny, nt, mask, seed=0)
    g = lct.Geometry(nx, ny, nt, cfg["bin_width_s"])
    op = lct.Operator(g, mask)
    t0 = time.time()
    u, hist = admm.alg1(tau0, mask, g, cfg["a"], cfg["b"], cfg["mu"], cfg["iters"], op=op)
    cols = golden_columns(nx, ny)
    flat = u.reshape(nx * ny, nt)
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), NAME + ".npz")
    np.savez_compressed(out, cols=cols, u_cols=flat[cols].astype(np.float32),
                        depth=admm.depth_map(u).astype(np.int16), energy=np.array(hist["E"]),
                        L=np.array(hist["L"]), norm=np.linalg.norm(u), total=float(np.sum(u)),
                        iters=cfg["iters"])
    print(f"wrote {out} in {time.time() - t0:.0f} s; E = {hist['E'][-1]:.6g}, backtracks {sum(hist['backtracks'])}")


if __name__ == "__main__":
    main()
