"""Host I/O of lbm_init_fields and lbm_read_fields: page-locked host arrays are read and written in
place by the conversion kernels, other host memory goes through the staging buffer. Both routes,
and any mix of them, must give bit-identical states and fields."""
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


def _pinned(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).reshape(-1).pin_memory()


@pytest.mark.parametrize("store", ["f32", "f16"])
def test_pinned_and_pageable_io_are_identical(store):
    import torch
    cfg = W.base_config(3, 37, 21, 13, 19, rho_g=0.1)
    phi, u = W.smooth_random_fields(cfg, seed=41)
    phi = W.to_q30_grid(phi)
    N = W.ncells(cfg)
    ps = W.noise(N, 42, 5e-3)
    routes = {
        "pageable": (phi, u, ps),
        "pinned": (_pinned(phi), _pinned(u), _pinned(ps)),
        "mixed": (_pinned(phi), u, _pinned(ps)),
    }
    out = {}
    for name, (a, b, c) in routes.items():
        sim = B.Lbm(cfg, store=store)
        sim.init_fields(a, b, c)
        f0, p0 = sim.get_state()
        sim.step(7)
        if name == "pageable":
            fields = sim.read_fields()
        else:
            o_phi = torch.empty(N, dtype=torch.float64).pin_memory()
            o_u = torch.empty(3 * N, dtype=torch.float64).pin_memory()
            o_ps = np.empty(N) if name == "mixed" else torch.empty(N, dtype=torch.float64).pin_memory()
            sim.read_fields(phi=o_phi, u=o_u, pstar=o_ps)
            fields = (o_phi.numpy(), o_u.numpy().reshape(3, N), np.asarray(o_ps))
        m = sim.mass()
        sim.close()
        out[name] = (f0, p0, fields, m)
    ref = out["pageable"]
    assert np.array_equal(ref[1], phi)
    for name in ("pinned", "mixed"):
        got = out[name]
        assert np.array_equal(got[0], ref[0]) and np.array_equal(got[1], ref[1]), name
        for x, y in zip(got[2], ref[2]):
            assert np.array_equal(np.asarray(x).reshape(-1), np.asarray(y).reshape(-1)), name
        assert got[3][0] == ref[3][0] and np.array_equal(got[3][1], ref[3][1]), name


def test_pinned_view_inside_a_larger_allocation():
    """Arrays that are views into one page-locked allocation (offsets, not its start) read and
    write in place as well, and only their own elements are touched."""
    import torch
    cfg = W.base_config(3, 24, 16, 12, 19, rho_g=0.1)
    phi, u = W.smooth_random_fields(cfg, seed=43)
    phi = W.to_q30_grid(phi)
    N = W.ncells(cfg)
    big = torch.zeros(7 * N, dtype=torch.float64).pin_memory()
    big[N:2 * N] = torch.from_numpy(phi)
    big[2 * N:5 * N] = torch.from_numpy(np.ascontiguousarray(u).reshape(-1))
    a = B.Lbm(cfg)
    a.init_fields(big[N:2 * N], big[2 * N:5 * N])
    b = B.Lbm(cfg)
    b.init_fields(phi, u)
    a.step(3)
    b.step(3)
    sentinel = torch.full((7 * N,), -7.0, dtype=torch.float64).pin_memory()
    a.read_fields(phi=sentinel[N:2 * N], u=sentinel[2 * N:5 * N], pstar=sentinel[5 * N:6 * N])
    ph, uu, pp = b.read_fields()
    a.close()
    b.close()
    s = sentinel.numpy()
    assert np.array_equal(s[N:2 * N], ph) and np.array_equal(s[2 * N:5 * N], uu.reshape(-1))
    assert np.array_equal(s[5 * N:6 * N], pp)
    assert np.all(s[:N] == -7.0) and np.all(s[6 * N:] == -7.0)

