"""Pins of the oracle's interfacial curvature (Sec. 3.4, Eq. 78): kappa = div n with the outward
normal n = grad(phi) / (|grad(phi)| + eps_n).

* A bubble of radius R (phi = 0 inside): n is radial and div n = 2 / r at distance r, so the band
  mean of kappa equals the band mean of 2 / r up to the stencil's truncation error.
* A cylindrical bubble (invariant along z): div n = 1 / r.
* A planar film: kappa vanishes up to the eps_n floor of the normal.
* A droplet (phi = 1 inside) gives the same |kappa| with the opposite sign.
"""
import numpy as np
import pytest

from paper_2603_17481_gb300 import workloads as W


def _band_mean_inv_r(cfg, phi, c, p, dims=3):
    nx, ny, nz = cfg["nx"], cfg["ny"], cfg["nz"]
    n = np.arange(phi.size)
    d = [n % nx - c[0], (n // nx) % ny - c[1], n // (nx * ny) - c[2]]
    r = np.sqrt(sum(x * x for x in d[:dims]))
    pc = np.clip(phi, 0, 1)
    band = pc * (1 - pc) >= cfg["q_th"]
    return np.mean(p / r[band]), band.sum()


@pytest.mark.parametrize("R", [10.0, 16.0])
def test_sphere_mean_curvature(orc, R):
    cfg = W.base_config(3, 48, 48, 48, 19)
    c = (23.7, 24.2, 23.9)
    phi, _ = W.droplet_fields(cfg, [c], [R], [(0, 0, 0)], bubbles=True)
    k = orc.curvature(orc.make_params(cfg), phi, 0.0, 0.5, 50)
    ref, nb = _band_mean_inv_r(cfg, phi, c, 2.0)
    assert k["band_cells"] == nb
    assert abs(k["mean"] - ref) < 0.03 * ref
    assert k["hist"].sum() == nb  # every band value lies in [0, 0.5)
    # the histogram peaks near 2 / R
    centres = (np.arange(50) + 0.5) * 0.01
    assert abs(centres[np.argmax(k["hist"])] - 2.0 / R) < 0.03


def test_cylinder_and_droplet_sign(orc):
    cfg = W.base_config(3, 48, 48, 8, 19)
    nx = ny = 48
    n = np.arange(48 * 48 * 8)
    x, y = n % nx - 23.6, (n // nx) % ny - 24.1
    r = np.sqrt(x * x + y * y)
    prof = 0.5 * (1 + np.tanh(2 * (14.0 - r) / cfg["eps"]))
    bubble, drop = 1 - prof, prof
    P = orc.make_params(cfg)
    kb = orc.curvature(P, bubble, -1.0, 1.0, 20)
    kd = orc.curvature(P, drop, -1.0, 1.0, 20)
    band = bubble * (1 - bubble) >= cfg["q_th"]
    ref = np.mean(1.0 / r[band])
    assert abs(kb["mean"] - ref) < 0.03 * ref
    assert abs(kd["mean"] + kb["mean"]) < 1e-12


def test_planar_interface_is_flat(orc):
    cfg = W.base_config(3, 32, 8, 8, 19)
    x = np.tile(np.arange(32, dtype=float), 64)
    phi = 0.5 * (1 + np.tanh(2 * (np.abs(x - 15.5) - 6.0) / cfg["eps"]))
    k = orc.curvature(orc.make_params(cfg), phi, -1.0, 1.0, 10)
    assert k["band_cells"] > 0 and abs(k["mean"]) < 1e-3
