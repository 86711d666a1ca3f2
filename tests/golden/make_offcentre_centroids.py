"""Writes offcentre_3d_centroids.txt: the FP64 oracle's droplet centroids on the 3D off-centre
collision (128x64x64 D3Q19, R = 12, density ratio 10, seeded impact offset; the inputs come from
the seeded workload generator, rounded to the 2^-30 grid the GPU stores phi on) at several steps
up to 2000.

Only the oracle computes here: the stored values are the oracle's, never the CUDA path's. A
centroid is the phi-weighted mean (x, y, z) of the left or the right half of the box in x (one
droplet each before they meet); the GPU test takes the same centroids of the GPU's phi.

    python tests/golden/make_offcentre_centroids.py      # about 10-20 minutes on 8 cores
"""
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402
from paper_2603_17481_gb300 import workloads as W  # noqa: E402

CHECKPOINTS = (200, 500, 1000, 1500, 2000)
OUT = os.path.join(HERE, "offcentre_3d_centroids.txt")


def half_box_centroids(cfg, ph):
    nx, ny, nz = cfg["nx"], cfg["ny"], cfg["nz"]
    g = np.asarray(ph).reshape(nz, ny, nx)
    out = []
    for sl in (slice(0, nx // 2), slice(nx // 2, nx)):
        m = g[:, :, sl]
        zz, yy, xx = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx)[sl], indexing="ij")
        out.append([(m * xx).sum() / m.sum(), (m * yy).sum() / m.sum(), (m * zz).sum() / m.sum()])
    return np.array(out)


def main():
    O.build()
    cfg, phi, u = W.droplets_offcentre_3d()
    phi = W.to_q30_grid(phi)
    P = O.make_params(cfg)
    f = O.init(P, phi, u)
    ph, done, rows = phi, 0, []
    t0 = time.time()
    for c in CHECKPOINTS:
        f, ph, _ = O.step(P, f, ph, c - done)
        done = c
        cen = half_box_centroids(cfg, ph)
        rows.append((c, cen))
        print(f"step {c}: {cen.ravel()} ({time.time() - t0:.0f} s)", flush=True)
    with open(OUT, "w") as fh:
        fh.write("# FP64 oracle droplet centroids, 3D off-centre collision 128x64x64 D3Q19, R=12, ratio 10,\n")
        fh.write(f"# impact offset b = {cfg['impact_offset']:.17g} (seed 17481), phi on the 2^-30 grid at t = 0.\n")
        fh.write("# Written by tests/golden/make_offcentre_centroids.py (oracle only).\n")
        fh.write("# step  left_x left_y left_z  right_x right_y right_z\n")
        for c, cen in rows:
            fh.write(f"{c} " + " ".join(f"{v:.17g}" for v in cen.ravel()) + "\n")


if __name__ == "__main__":
    main()
