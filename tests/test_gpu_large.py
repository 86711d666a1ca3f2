"""The largest grids: population offsets beyond 32 bits (Q N > 2^32, the hydrodynamic kernel's 64-bit
offset instance). A field that repeats a small period is a fixed point of periodic translation, so
after any number of steps the large grid must hold the small grid's state repeated: every cell of
the large run is checked against the small run (same one-cell kernel, 32-bit offsets there), which
itself follows the FP64 oracle in the parity tests."""
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


def _tile(a, small, reps):
    """Field of the small grid (x fastest) repeated reps = (rx, ry, rz) times."""
    nx, ny, nz = small
    return np.tile(a.reshape(nz, ny, nx), (reps[2], reps[1], reps[0])).reshape(-1)


def test_64bit_offsets_match_the_repeated_small_grid():
    # D3Q27 on 560 x 560 x 512: Q N = 4.34e9 > 2^32. The small period 35 x 35 x 32 has odd nx, so
    # it runs the same one-cell kernel with 32-bit offsets.
    small, reps = (35, 35, 32), (16, 16, 16)
    big = tuple(s * r for s, r in zip(small, reps))
    cs = W.base_config(3, *small, 27, rho_g=0.1)
    cb = W.base_config(3, *big, 27, rho_g=0.1)
    assert 27 * W.ncells(cb) > 2 ** 32
    phi, u = W.smooth_random_fields(cs, seed=61)
    phi = W.to_q30_grid(phi)
    steps = 12
    s = B.Lbm(cs)
    s.init_fields(phi, u)
    s.step(steps)
    ph_s, u_s, ps_s = s.read_fields()
    part_s, _ = s.read_nci()
    s.close()
    assert (part_s[:, 0] != np.iinfo(np.int32).min).sum() > 0  # near-contact pairs are active

    b = B.Lbm(cb)
    b.init_fields(_tile(phi, small, reps), np.stack([_tile(u[a], small, reps) for a in range(3)]))
    del phi, u
    b.step(steps)
    ph_b, u_b, ps_b = b.read_fields()
    m_b = b.mass()[0]
    b.close()
    assert np.max(np.abs(ph_b - _tile(ph_s, small, reps))) <= 1e-7
    assert np.max(np.abs(ps_b - _tile(ps_s, small, reps))) <= 1e-6
    for a in range(3):
        assert np.max(np.abs(u_b[a] - _tile(u_s[a], small, reps))) <= 1e-6
    # the fixed-point phi sum is exact: the large grid holds the small one's mass repeated
    assert m_b == pytest.approx(float(np.round(ph_s * 2 ** 30).sum()) * np.prod(reps) / 2 ** 30, rel=1e-15)
