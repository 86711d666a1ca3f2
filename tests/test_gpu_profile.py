"""The per-kernel profiler through the C ABI: kind masks and the kernel count of each pass."""
import numpy as np
import pytest

from paper_2603_17481_gb300 import binding as B
from paper_2603_17481_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def gpu():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2603_17481_gb300 import build
    build.build()
    torch.cuda.set_device(0)
    return True


@pytest.mark.parametrize("dims,nci_kernels,hydro_kernels,overlap",
                         [((32, 24, 16), 3, 1, 0), ((32, 24, 16), 3, 2, 8), ((33, 17, 12), 2, 1, 0)])
def test_profile_kinds_and_counts(dims, nci_kernels, hydro_kernels, overlap):
    """hydro_kernels: 2 in the split step (lbm_set_overlap > 0, nx even), 1 otherwise."""
    cfg = W.base_config(3, *dims, 19, rho_g=0.1)
    phi, u = W.smooth_random_fields(cfg, seed=5)
    sim = B.Lbm(cfg)
    assert sim.overlap() == 0
    sim.set_overlap(overlap)
    sim.init_fields(W.to_q30_grid(phi), u)
    sim.profile_kinds(["hydro"])
    sim.step(3)
    p = sim.profile_read()
    assert p["hydro"][1] == 3 * hydro_kernels and p["hydro"][0] > 0
    assert p["nci"] == (0.0, 0) and p["phase"] == (0.0, 0)
    sim.profile(True)  # a fresh tally of every kind
    sim.step(2)
    p = sim.profile_read()
    assert p["hydro"][1] == 2 * hydro_kernels and p["phase"][1] == 2 and p["nci"][1] == 2 * nci_kernels
    assert all(p[k][0] > 0 for k in ("nci", "hydro", "phase"))
    sim.profile_kinds([])
    sim.step(1)
    assert sim.profile_read()["hydro"] == (0.0, 0)
    # sampling: the first pass and every third after it (passes 0, 3, 6 of 7)
    sim.profile_kinds(["hydro", "phase"])
    sim.profile_sample(3)
    sim.step(7)
    p = sim.profile_read()
    assert p["hydro"][1] == 3 * hydro_kernels and p["phase"][1] == 3 and p["hydro"][0] > 0
    sim.profile_sample(1)
    sim.close()
