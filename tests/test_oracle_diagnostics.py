"""Pins of the oracle's self-tuning diagnostics (Sec. 3.3, Eq. 74): the film volume, the normal
projections of the repulsive and capillary forces over the film, and the repulsion's peak and sum.

* Planar film: on a profile that varies along x only, the D3Q27 isotropic gradient and Laplacian
  reduce to the central differences (phi(x+1) - phi(x-1)) / 2 and phi(x+1) - 2 phi + phi(x-1), so
  every film sum has a closed form in the tanh profile (with F_rep from Eqs. 66-73 as pinned in
  test_oracle_nci).
* An isolated droplet has no film.
* F_rep is linear in A_rep and independent of sigma; F_cap = mu_phi grad(phi) is linear in sigma
  (beta and k both scale with sigma): R_n scales as A_rep / sigma on a fixed film.
"""
import numpy as np
import pytest

from paper_2603_17481_gb300 import workloads as W


def _planar(cfg, gap=1.0):
    nx, ny, nz = cfg["nx"], cfg["ny"], cfg["nz"]
    x = np.tile(np.arange(nx, dtype=float), ny * nz)
    s = np.abs(x - 11.5) - gap / 2
    return 0.5 * (1 + np.tanh(2 * s / cfg["eps"])), x, s


def test_planar_film_closed_form(orc):
    cfg = W.base_config(3, 24, 8, 8, 19, rho_g=0.1, decide_f32=0, eps_n=1e-12)
    P = orc.make_params(cfg)
    phi, x, s = _planar(cfg)
    d = orc.nci_diagnostics(P, phi)
    # closed forms along one x row: film cells are the gated ones (depth 0 and 1 on each side)
    prof = lambda xx: 0.5 * (1 + np.tanh(2 * (np.abs(xx - 11.5) - 0.5) / cfg["eps"]))
    xs = np.arange(24, dtype=float)
    p0, pp, pm = prof(xs), prof(xs + 1), prof(xs - 1)
    g = 0.5 * (pp - pm)
    lap = pp - 2 * p0 + pm
    beta, kap = 12 * cfg["sigma"] / cfg["eps"], 1.5 * cfg["sigma"] * cfg["eps"]
    mu = 4 * beta * p0 * (p0 - 1) * (p0 - 0.5) - kap * lap
    n = g / (np.abs(g) + cfg["eps_n"])
    q = p0 * (1 - p0)
    film = q >= 0.125
    assert film.sum() == 4
    sd = np.abs(np.abs(xs - 11.5) - 0.5)
    rho = cfg["rho_g"] + (cfg["rho_l"] - cfg["rho_g"]) * p0
    frep = rho * cfg["A_rep"] * np.clip(q, 1e-12, 0.25 - 1e-12) / (1 + (2 * sd) ** 4)
    rows = cfg["ny"] * cfg["nz"]
    assert d["V_film"] == 4 * rows
    assert abs(d["sum_rep_n"] - rows * np.sum((frep * np.abs(n))[film])) < 1e-9 * d["sum_rep_n"]
    assert abs(d["sum_cap_n"] - rows * np.sum(np.abs(mu * g * n)[film])) < 1e-9 * d["sum_cap_n"]
    assert abs(d["sum_rep"] - rows * np.sum(frep[film])) < 1e-9 * d["sum_rep"]
    assert abs(d["max_rep"] - np.max(frep[film])) < 1e-9 * d["max_rep"]  # f_face = 1 - O(eps_n / |g|)
    assert d["R_n"] > 0 and abs(d["mean_rep"] - d["sum_rep"] / d["V_film"]) < 1e-15


@pytest.mark.parametrize("dim,R,n", [(2, 16.0, 64), (3, 12.0, 40)])
def test_isolated_droplet_has_no_film(orc, dim, R, n):
    cfg = W.base_config(dim, n, n, n if dim == 3 else 1, 9 if dim == 2 else 19)
    P = orc.make_params(cfg)
    c = (n / 2 - 0.3, n / 2 + 0.2, n / 2 - 0.1 if dim == 3 else 0.0)
    phi, _ = W.droplet_fields(cfg, [c], [R], [(0, 0, 0)])
    d = orc.nci_diagnostics(P, phi)
    assert d["V_film"] == 0 and d["sum_rep_n"] == 0 and d["sum_cap_n"] == 0 and d["max_rep"] == 0
    assert d["R_n"] == 0 and d["mean_rep"] == 0


def _pair(**kw):
    cfg = W.base_config(3, 48, 32, 32, 19, rho_g=0.1, **kw)
    phi, _ = W.droplet_fields(cfg, [(14.3, 15.6, 15.4), (33.1, 16.2, 15.7)], [8.0, 8.0], [(0, 0, 0)] * 2)
    return cfg, phi


def test_scaling_in_A_rep_and_sigma(orc):
    cfg, phi = _pair(A_rep=0.02, sigma=0.02)
    d1 = orc.nci_diagnostics(orc.make_params(cfg), phi)
    assert d1["V_film"] > 20
    cfg2, _ = _pair(A_rep=0.04, sigma=0.02)
    d2 = orc.nci_diagnostics(orc.make_params(cfg2), phi)
    cfg3, _ = _pair(A_rep=0.02, sigma=0.04)
    d3 = orc.nci_diagnostics(orc.make_params(cfg3), phi)
    assert d2["V_film"] == d1["V_film"] == d3["V_film"]
    for k in ("sum_rep_n", "sum_rep", "max_rep"):
        assert abs(d2[k] - 2 * d1[k]) < 1e-12 * d2[k]
        assert abs(d3[k] - d1[k]) < 1e-12 * d1[k]
    assert abs(d2["sum_cap_n"] - d1["sum_cap_n"]) < 1e-12 * d1["sum_cap_n"]
    assert abs(d3["sum_cap_n"] - 2 * d1["sum_cap_n"]) < 1e-12 * d3["sum_cap_n"]
    assert abs(d2["R_n"] - 2 * d1["R_n"]) < 1e-12 * d2["R_n"]
    assert abs(d3["R_n"] - 0.5 * d1["R_n"]) < 1e-12 * d1["R_n"]
