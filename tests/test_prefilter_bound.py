"""The lower bound behind the near-contact brick prefilter, checked against the oracle's pairing.

For a 4x4x4 brick B with component ranges [lo, hi] of its gated normals, and [L, H] the ranges over
the 27 bricks around it (which hold every cell y with |y_a - x_a| <= 3 on each axis, for every x in B), the product is
bilinear in each component, so n(x).n(y) >= sum_a min(lo_a L_a, lo_a H_a, hi_a L_a, hi_a H_a). A
brick whose bound exceeds cos_opp + 1e-5 can hold no cell that meets the facing gate of Eq. 62. This
test recomputes the bound in FP64 from the oracle's isotropic gradient (Eq. 22 normals, Eq. 57) on
seeded fields and checks that no cell the oracle pairs lies in a brick the bound clears, and that the
bound clears most bricks of an isolated droplet (so the check is not vacuous).
"""
import numpy as np
import pytest

from paper_2603_17481_gb300 import workloads as W


def _brick_bound(orc, cfg, phi):
    P = orc.make_params(cfg)
    nx, ny, nz = cfg["nx"], cfg["ny"], cfg["nz"]
    g = orc.grad_iso(P, phi)
    n = g / (np.sqrt((g ** 2).sum(axis=0)) + cfg["eps_n"])
    pc = np.clip(phi, 0.0, 1.0)
    gated = pc * (1.0 - pc) >= cfg["q_th"]
    shp = (nz // 4, 4, ny // 4, 4, nx // 4, 4)
    lo = [np.where(gated, n[a], np.inf).reshape(shp).min(axis=(1, 3, 5)) for a in range(3)]
    hi = [np.where(gated, n[a], -np.inf).reshape(shp).max(axis=(1, 3, 5)) for a in range(3)]
    L, H = [], []
    for a in range(3):
        la, ha = lo[a].copy(), hi[a].copy()
        for dz in (-1, 0, 1):
            for dy in (-1, 0, 1):
                for dx in (-1, 0, 1):
                    la = np.minimum(la, np.roll(lo[a], (dz, dy, dx), axis=(0, 1, 2)))
                    ha = np.maximum(ha, np.roll(hi[a], (dz, dy, dx), axis=(0, 1, 2)))
        L.append(la)
        H.append(ha)
    has = lo[0] <= hi[0]
    bound = np.zeros(has.shape)
    with np.errstate(invalid="ignore"):
        for a in range(3):
            c = np.stack([lo[a] * L[a], lo[a] * H[a], hi[a] * L[a], hi[a] * H[a]])
            bound += np.where(has, c.min(axis=0), 0.0)
    cleared = has & (bound > cfg["cos_opp"] + 1e-5)
    return P, gated, has, cleared


def _brick_of_cells(cfg):
    nx, ny, nz = cfg["nx"], cfg["ny"], cfg["nz"]
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    return (z // 4).ravel(), (y // 4).ravel(), (x // 4).ravel()


@pytest.mark.parametrize("shape,seed", [((24, 20, 16), 3), ((32, 16, 12), 8), ((28, 24, 20), 21)])
def test_no_paired_cell_in_a_cleared_brick(orc, shape, seed):
    cfg = W.base_config(3, *shape, 19, rho_g=0.1)
    phi, _ = W.smooth_random_fields(cfg, seed=seed)
    phi = W.to_q30_grid(phi)
    P, gated, has, cleared = _brick_bound(orc, cfg, phi)
    part, _, _ = orc.nci(P, phi)
    paired = part[:, 0] != orc.NO_PARTNER
    assert paired.sum() > 0
    bz, by, bx = _brick_of_cells(cfg)
    assert not np.any(cleared[bz, by, bx] & paired)


def test_planar_gap_is_never_cleared(orc):
    """Two parallel interfaces 3 cells apart face each other: the bricks along the gap hold paired
    cells and the bound must keep them."""
    cfg = W.base_config(3, 32, 8, 8, 19, rho_g=0.1)
    x = np.tile(np.arange(32, dtype=float), 64)
    phi = W.to_q30_grid(0.5 * (1 + np.tanh(2 * (1.5 - np.abs(x - 15.5)) / cfg["eps"])))
    P, gated, has, cleared = _brick_bound(orc, cfg, phi)
    part, _, _ = orc.nci(P, phi)
    paired = part[:, 0] != orc.NO_PARTNER
    assert paired.sum() > 0
    bz, by, bx = _brick_of_cells(cfg)
    assert not np.any(cleared[bz, by, bx] & paired)


def test_isolated_droplet_is_cleared(orc):
    cfg = W.base_config(3, 40, 40, 40, 19)
    phi, _ = W.droplet_fields(cfg, [(19.7, 20.2, 19.9)], [12.0], [(0, 0, 0)])
    P, gated, has, cleared = _brick_bound(orc, cfg, W.to_q30_grid(phi))
    assert has.sum() > 50
    assert cleared.sum() >= 0.9 * has.sum()
