"""Near-contact film statistics (Sec. 3.3, Eq. 74) through the C ABI against the FP64 oracle."""
import numpy as np
import pytest

import oracle as O
from paper_2603_17481_gb300 import binding as B
from paper_2603_17481_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def gpu():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2603_17481_gb300 import build
    build.build()
    O.build()
    torch.cuda.set_device(0)
    return True


def _pair(dim=3, **kw):
    if dim == 3:
        cfg = W.base_config(3, 48, 32, 32, 19, rho_g=0.1, **kw)
        c = [(14.3, 15.6, 15.4), (33.1, 16.2, 15.7)]
    else:
        cfg = W.base_config(2, 96, 48, 1, 9, rho_g=0.1, **kw)
        c = [(30.2, 23.6, 0.0), (65.9, 24.3, 0.0)]
    phi, _ = W.droplet_fields(cfg, c, [8.0 if dim == 3 else 16.0] * 2, [(0, 0, 0)] * 2)
    return cfg, W.to_q30_grid(phi)


def _gpu_diag(cfg, phi):
    sim = B.Lbm(cfg)
    sim.init_fields(phi, np.zeros((3, phi.size)))
    d = sim.nci_diagnostics()
    part, _ = sim.read_nci()
    sim.close()
    return d, part


@pytest.mark.parametrize("dim", [2, 3])
def test_film_statistics_match_oracle(dim):
    cfg, phi = _pair(dim)
    P = O.make_params(cfg)
    do = O.nci_diagnostics(P, phi)
    dg, part_g = _gpu_diag(cfg, phi)
    part_o, _, marg = O.nci(P, phi)
    mis = np.any(part_g != part_o, axis=1)
    assert np.all(marg[mis] < 1e-5)
    assert do["V_film"] > 10
    assert abs(dg["V_film"] - do["V_film"]) <= mis.sum()
    if mis.sum() == 0:
        for k in ("sum_rep_n", "sum_cap_n", "sum_rep", "R_n", "mean_rep"):
            assert abs(dg[k] - do[k]) <= 2e-5 * abs(do[k]), (k, dg[k], do[k])
        assert abs(dg["max_rep"] - do["max_rep"]) <= 2e-5 * do["max_rep"]


def test_film_statistics_scale_and_vanish():
    cfg, phi = _pair(3, A_rep=0.02, sigma=0.02)
    d1, _ = _gpu_diag(cfg, phi)
    d2, _ = _gpu_diag(_pair(3, A_rep=0.04, sigma=0.02)[0], phi)
    d3, _ = _gpu_diag(_pair(3, A_rep=0.02, sigma=0.04)[0], phi)
    assert d1["V_film"] == d2["V_film"] == d3["V_film"] > 0
    assert abs(d2["R_n"] / d1["R_n"] - 2.0) < 1e-5 and abs(d3["R_n"] / d1["R_n"] - 0.5) < 1e-5
    off, _ = _gpu_diag(dict(cfg, nci_on=0), phi)
    assert all(v == 0.0 for v in off.values())
    single = W.base_config(3, 40, 40, 40, 19)
    ph1, _ = W.droplet_fields(single, [(19.7, 20.2, 19.9)], [12.0], [(0, 0, 0)])
    iso, _ = _gpu_diag(single, W.to_q30_grid(ph1))
    assert all(v == 0.0 for v in iso.values())


@pytest.mark.parametrize("dim", [2, 3])
def test_curvature_matches_oracle(dim):
    """Interfacial mean curvature (Eq. 78) of a few bubbles: band cells identical, mean within 1e-4,
    and histogram counts differing only where a value sits within FP32 rounding of a bin edge."""
    if dim == 3:
        cfg = W.base_config(3, 64, 48, 40, 19)
        c, R = [(16.3, 20.1, 19.6), (44.7, 27.2, 21.3)], [9.0, 12.0]
        lo, hi, nb = 0.0, 0.5, 100
    else:
        cfg = W.base_config(2, 128, 96, 1, 9)
        c, R = [(40.2, 45.3, 0.0), (90.6, 50.1, 0.0)], [14.0, 20.0]
        lo, hi, nb = 0.0, 0.25, 100
    phi, _ = W.droplet_fields(cfg, c, R, [(0, 0, 0)] * 2, bubbles=True)
    phi = W.to_q30_grid(phi)
    ko = O.curvature(O.make_params(cfg), phi, lo, hi, nb)
    sim = B.Lbm(cfg)
    sim.init_fields(phi, np.zeros((3, phi.size)))
    kg = sim.curvature(lo, hi, nb)
    sim.close()
    assert kg["band_cells"] == ko["band_cells"] > 100
    assert abs(kg["mean"] - ko["mean"]) <= 1e-4 * abs(ko["mean"])
    assert abs(int(kg["hist"].sum()) - int(ko["hist"].sum())) <= 2
    assert np.abs(kg["hist"] - ko["hist"]).sum() <= max(4, 0.002 * ko["hist"].sum())


@pytest.mark.parametrize("dim", [2, 3])
def test_energy_spectrum_matches_oracle(dim):
    """Carrier-phase spectrum (Sec. 3.4) through cuFFT against the oracle's numpy FFT on the same
    state: every shell within 1e-5 of the total, the total within 1e-6."""
    if dim == 3:
        cfg = W.base_config(3, 40, 36, 32, 19, rho_g=0.1)
        c, R = [(12.3, 17.1, 15.6), (28.7, 19.2, 16.3)], [6.0, 7.0]
    else:
        cfg = W.base_config(2, 96, 64, 1, 9, rho_g=0.1)
        c, R = [(30.2, 31.3, 0.0), (66.6, 33.1, 0.0)], [10.0, 12.0]
    phi, _ = W.droplet_fields(cfg, c, R, [(0, 0, 0)] * 2, bubbles=True)
    phi = W.to_q30_grid(phi)
    P, _, u, f = _random_state_from(cfg, phi)
    _, uo = O.moments(P, f, phi)
    Eo = O.energy_spectrum(P, phi, uo, 48)
    sim = B.Lbm(cfg)
    sim.set_state(f, phi)
    Eg = sim.energy_spectrum(48)
    sim.close()
    assert Eo.sum() > 0
    assert np.max(np.abs(Eg - Eo)) <= 1e-5 * Eo.sum()
    assert abs(Eg.sum() - Eo.sum()) <= 1e-6 * Eo.sum()


def _random_state_from(cfg, phi, seed=21):
    """Equilibrium populations of a smooth random velocity field on the given phi."""
    _, u = W.smooth_random_fields(cfg, seed=seed, pairs=False)
    P = O.make_params(cfg)
    f = O.init(P, phi, u)
    return P, phi, u, f


_CLOSING = {
    # two pairs closing in (x and z), every side a multiple of 32 x 8 x 4 tiles
    (64, 48, 40): [((16.3, 20.1, 19.6), 8.0, (0.02, 0.0, 0.0)), ((34.9, 21.2, 20.3), 8.0, (-0.02, 0.0, 0.0)),
                   ((50.2, 36.4, 12.3), 6.0, (0.0, 0.0, 0.015)), ((50.9, 36.0, 27.6), 7.0, (0.0, 0.0, -0.015))],
    # partial tiles in x and y (sides multiples of 4 only), one pair across the periodic x boundary
    (68, 44, 28): [((14.2, 22.3, 13.6), 7.0, (0.02, 0.0, 0.0)), ((31.0, 23.1, 14.2), 8.0, (-0.02, 0.0, 0.0)),
                   ((63.5, 36.2, 14.1), 6.0, (0.02, 0.0, 0.0)), ((10.0, 36.8, 13.8), 6.0, (-0.02, 0.0, 0.0))],
}


@pytest.mark.parametrize("dims", list(_CLOSING))
def test_listed_pass_after_steps(dims):
    """Droplets closing in for 40 steps: the per-step near-contact pass over the listed tiles (with
    the brick prefilter, which applies where every side is a multiple of 4) then finds exactly the
    partners and forces of the pass over every tile, and those follow the oracle on the same phi."""
    cfg = W.base_config(3, *dims, 19, rho_g=0.1)
    c, R, U = zip(*_CLOSING[dims])
    phi, u = W.droplet_fields(cfg, c, R, U)
    sim = B.Lbm(cfg)
    sim.init_fields(W.to_q30_grid(phi), u)
    sim.step(40)
    dl = sim.nci_diagnostics()           # listed tiles, as every step runs it
    part_all, frep_all = sim.read_nci()  # every tile, no prefilter
    ph, _, _ = sim.read_fields()
    sim.close()
    film = part_all[:, 0] != np.iinfo(np.int32).min
    assert film.sum() > 20
    assert dl["V_film"] == film.sum()
    s = np.sqrt((frep_all[:, film] ** 2).sum(axis=0)).sum()
    assert abs(dl["sum_rep"] - s) <= 1e-6 * s
    part_o, _, marg = O.nci(O.make_params(cfg), ph)
    mis = np.any(part_all != part_o, axis=1)
    assert np.all(marg[mis] < 1e-5)


@pytest.mark.parametrize("dims,seed", [((8, 8, 8), 1), ((12, 8, 8), 2), ((16, 12, 8), 3), ((36, 20, 16), 4)])
def test_listed_pass_on_small_grids(dims, seed):
    """Random interfaces on small grids whose sides are multiples of 4 (fewer bricks than a tile holds,
    brick neighbourhoods that wrap onto themselves): the per-step near-contact pass over the listed
    tiles, with the brick prefilter, equals the pass over every tile at t = 0 and after 3 steps."""
    cfg = W.base_config(3, *dims, 19, rho_g=0.1)
    phi, u = W.smooth_random_fields(cfg, seed=seed)
    sim = B.Lbm(cfg)
    sim.init_fields(W.to_q30_grid(phi), u)
    films = []
    for steps in (0, 3):
        sim.step(steps)
        dl = sim.nci_diagnostics()
        part, frep = sim.read_nci()
        film = part[:, 0] != np.iinfo(np.int32).min
        assert dl["V_film"] == film.sum()
        s = np.sqrt((frep[:, film] ** 2).sum(axis=0)).sum()
        assert abs(dl["sum_rep"] - s) <= 1e-6 * s
        films.append(int(film.sum()))
    sim.close()
    assert max(films) > 0


def test_full_size_swarm_listed_pass_and_mass():
    """The 512^3 swarm grid and launch configuration of bench.py (D3Q19, FP32 store, 1500 bubbles),
    with surface gaps of eps so that films exist from the start: after 10 steps the sum of the
    fixed-point phi is unchanged, and the per-step near-contact pass over the listed tiles (with the
    brick prefilter) finds exactly the partners and forces of the pass over every tile."""
    cfg, cs, rs = W.bubble_swarm(gap_eps=1.0)
    phi, u = W.bubble_swarm_fields(cfg, cs, rs)
    sim = B.Lbm(cfg)
    sim.init_fields(phi, u)
    del phi, u
    m0, _ = sim.mass()
    sim.step(10)
    m1, _ = sim.mass()
    assert m1 == m0
    dl = sim.nci_diagnostics()
    part, frep = sim.read_nci()
    sim.close()
    film = part[:, 0] != np.iinfo(np.int32).min
    del part
    assert film.sum() > 1000
    assert dl["V_film"] == film.sum()
    s = np.sqrt((frep[:, film] ** 2).sum(axis=0)).sum()
    assert abs(dl["sum_rep"] - s) <= 1e-6 * s
