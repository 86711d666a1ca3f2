"""Host-side logic of the workloads and the benchmark: the sweep's parameter ranges, the box-local
swarm generator against the all-cells generator, and the periodic bubble counter."""
import math
import os
import sys

import numpy as np

from paper_2603_17481_gb300 import workloads as W

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


def test_sweep_parameters():
    cases = W.collision_sweep(512)
    assert len(cases) == 512
    assert {c["nx"] for c in cases} == set(W.SWEEP_GRIDS)
    for c in cases:
        L, R = c["nx"], c["R"]
        assert c["ny"] == c["nz"] == L and R == L / 6
        assert 1.0 <= c["weber"] <= 100.0 and 0.0 <= c["impact_offset"] <= 2 * R
        # We = rho_l U^2 (2R) / sigma is the drawn Weber number
        assert math.isclose(c["rho_l"] * c["speed"] ** 2 * 2 * R / c["sigma"], c["weber"], rel_tol=1e-12)
        assert c["sigma"] == 1e-3 and c["speed"] <= 0.08
        (x0, y0, _), (x1, y1, _) = c["centers"]
        assert math.isclose(x1 - x0, 2 * R + 8) and math.isclose(y1 - y0, c["impact_offset"])
    # reproducible from the seed
    assert W.collision_sweep(3, seed=5) == W.collision_sweep(3, seed=5)


def test_swarm_fields_match_all_cells_profile():
    cfg, cs, rs = W.bubble_swarm(L=80, nb=8, seed=4)
    assert len(cs) == 8
    for i in range(len(cs)):
        for j in range(i):
            d = cs[i] - cs[j]
            d -= 80 * np.round(d / 80)
            assert np.linalg.norm(d) >= rs[i] + rs[j] + 2 * cfg["eps"]
    phi, u = W.bubble_swarm_fields(cfg, cs, rs)
    ref, _ = W.droplet_fields(cfg, cs, rs, [(0, 0, 0)] * len(cs), bubbles=True)
    # each truncated profile tail is below 1.2e-7, so the fields differ by less than that per bubble
    assert np.max(np.abs(phi - ref)) < 1.2e-7 * len(cs)
    assert not np.any(u)


def test_count_bubbles_periodic():
    g = np.zeros((8, 8, 8), bool)
    g[0, 0, 0] = g[7, 0, 0] = True  # joined across z
    g[3, 3, 3] = True
    g[0, 5, 0] = g[0, 5, 7] = True  # joined across x
    g[2, 0, 4] = g[2, 7, 4] = True  # joined across y
    assert bench.count_bubbles(g) == 4
    g[3, 3, 4] = True  # touches (3,3,3)
    assert bench.count_bubbles(g) == 4
    g[5, 5, 5] = True
    assert bench.count_bubbles(g) == 5
    n, vols = bench.count_bubbles(g, volumes=True)
    assert n == 5 and sorted(vols) == [1, 2, 2, 2, 2]
    assert bench.count_bubbles(np.zeros((4, 4, 4), bool)) == 0


def test_count_bubbles_of_generated_swarm():
    cfg, cs, rs = W.bubble_swarm(L=96, nb=20, seed=9)
    phi, _ = W.bubble_swarm_fields(cfg, cs, rs)
    n, vols = bench.count_bubbles((phi < 0.5).reshape(96, 96, 96), volumes=True)
    assert n == len(cs) == len(vols)
    # each component's volume is its sphere's to within the lattice sampling of the surface
    exp = sorted(4.0 / 3.0 * np.pi * rs ** 3)
    assert np.all(np.abs(np.asarray(vols) - exp) < 0.05 * np.asarray(exp))


def test_centroids_of_two_droplets():
    # lattice-symmetric centres, 24 cells from the halves' borders (profile tails below 1e-8)
    cfg = W.base_config(3, 96, 16, 12, 19)
    phi, _ = W.droplet_fields(cfg, [(24.0, 7.5, 5.5), (71.5, 7.5, 5.5)], [5.0, 5.0], [(0, 0, 0)] * 2)
    c = bench.centroids(cfg, phi)
    assert abs(c[0] - 24.0) < 1e-6 and abs(c[1] - 71.5) < 1e-6


def test_workload_extras_do_not_shadow_parameters():
    """Workload dictionaries carry extra keys (diameter, speed, ...) next to the model parameters:
    none of them may overwrite a parameter such as the mobility D."""
    import oracle as O
    base = W.base_config(3, 8, 8, 8, 19)
    for cfg in W.selftune_cases()[:3] + W.collision_sweep(3):
        assert cfg["D"] == base["D"] and cfg["p"] == base["p"] and cfg["eps"] == base["eps"]
        extra = set(cfg) - set(base)
        assert not extra & set(O._FIELDS)


def test_kernels_per_step():
    """Kernel launches of one step as the bench claims them: the brick prefilter adds one kernel on 3D
    grids whose sides are multiples of 4, and the split step (3D, near-contact on, nx even) runs the
    hydrodynamic update as two launches."""
    assert bench.kernels_per_step(W.base_config(3, 64, 48, 40, 19)) == 5
    assert bench.kernels_per_step(W.base_config(3, 64, 48, 40, 19), overlap=True) == 6
    assert bench.kernels_per_step(W.base_config(3, 37, 21, 13, 19), overlap=True) == 4
    assert bench.kernels_per_step(W.base_config(3, 38, 21, 13, 19), overlap=True) == 5
    assert bench.kernels_per_step(W.base_config(3, 64, 48, 40, 19, nci_on=0)) == 2
    assert bench.kernels_per_step(W.base_config(2, 128, 64, 1, 9)) == 4
    assert all(bench.kernels_per_step(c) == 5 for c in W.collision_sweep(8))
    assert all(bench.nci_kernels(c) == 3 for c in W.collision_sweep(8))
    big = W.base_config(3, 1024, 1024, 256, 27)  # Q N > 2^32: 64-bit offsets, one launch
    assert not bench.split_applies(big) and bench.kernels_per_step(big, overlap=True) == 5
