"""The split step of lbm_step: the near-contact pass (Sec. 2.3) and the hydrodynamic update of the
cells of the listed near-contact tiles run on a second stream, concurrent with the hydrodynamic
update (Sec. 2.1) of every other cell. Each cell is written by one of the two launches with the
same arithmetic, so the state must be bit-identical to the one-stream step: through active contact,
on grids with partial tiles in every direction, for any number of scan blocks, and when the two
orders alternate from step to step."""
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


# droplet pairs closing in: (centre, radius, velocity)
_CLOSING = {
    # whole 32 x 8 x 4 near-contact tiles and 64-cell paired rows; the brick prefilter applies
    (64, 48, 40): [((16.3, 20.1, 19.6), 8.0, (0.02, 0.0, 0.0)), ((34.9, 21.2, 20.3), 8.0, (-0.02, 0.0, 0.0)),
                   ((50.2, 36.4, 12.3), 6.0, (0.0, 0.0, 0.015)), ((50.9, 36.0, 27.6), 7.0, (0.0, 0.0, -0.015))],
    # partial tiles in x and y (a paired row whose second near-contact tile lies beyond the grid),
    # one pair across the periodic x boundary; the prefilter applies
    (68, 44, 28): [((14.2, 22.3, 13.6), 7.0, (0.02, 0.0, 0.0)), ((31.0, 23.1, 14.2), 8.0, (-0.02, 0.0, 0.0)),
                   ((63.5, 36.2, 14.1), 6.0, (0.02, 0.0, 0.0)), ((10.0, 36.8, 13.8), 6.0, (-0.02, 0.0, 0.0))],
    # partial tiles in y and z, no side a multiple of 4 (no prefilter), a pair across the z boundary
    (70, 42, 30): [((18.4, 20.6, 14.2), 7.0, (0.02, 0.0, 0.0)), ((35.7, 21.1, 15.0), 7.0, (-0.02, 0.0, 0.0)),
                   ((52.3, 30.2, 26.1), 6.0, (0.0, 0.0, 0.015)), ((52.8, 29.7, 9.4), 6.0, (0.0, 0.0, -0.015))],
}


def _sim(dims, store="f32", Q=19):
    cfg = W.base_config(3, *dims, Q, rho_g=0.1)
    c, R, U = zip(*_CLOSING[dims])
    phi, u = W.droplet_fields(cfg, c, R, U)
    sim = B.Lbm(cfg, store=store)
    sim.init_fields(W.to_q30_grid(phi), u)
    return sim


def _run(dims, overlaps, steps, store="f32", Q=19):
    """State after `steps` steps, with lbm_set_overlap(overlaps[k % len]) before step k."""
    sim = _sim(dims, store, Q)
    for k in range(steps):
        sim.set_overlap(overlaps[k % len(overlaps)])
        sim.step(1)
    f, ph = sim.get_state()
    part, _ = sim.read_nci()
    m = sim.mass()[0]
    sim.close()
    return f, ph, part, m


@pytest.mark.parametrize("dims", list(_CLOSING))
def test_split_step_bit_identical_through_contact(dims):
    sim = _sim(dims)
    assert sim.overlap() == 0  # the default: one stream
    sim.close()
    f1, ph1, part1, m1 = _run(dims, [0], 60)        # one stream
    f2, ph2, part2, m2 = _run(dims, [38], 60)       # split, 38 scan blocks
    assert np.array_equal(f1, f2) and np.array_equal(ph1, ph2)
    assert np.array_equal(part1, part2)
    film = part1[:, 0] != np.iinfo(np.int32).min
    assert film.sum() > 20  # the films are active
    assert m1 == m2


@pytest.mark.parametrize("overlaps", [[1], [1000], [0, 5], [7, 0, 0]])
def test_split_step_any_blocks_and_alternating(overlaps):
    """One scan block, more than one per SM (capped), and the two orders alternating step by step
    (the near-contact lists and their marks stay consistent across them)."""
    dims = (68, 44, 28)
    f1, ph1, _, _ = _run(dims, [0], 45)
    f2, ph2, _, _ = _run(dims, overlaps, 45)
    assert np.array_equal(f1, f2) and np.array_equal(ph1, ph2)


@pytest.mark.parametrize("store,Q", [("f16", 19), ("bf16", 19), ("f32", 27)])
def test_split_step_stores_and_d3q27(store, Q):
    dims = (64, 48, 40)
    f1, ph1, _, _ = _run(dims, [0], 40, store, Q)
    f2, ph2, _, _ = _run(dims, [38], 40, store, Q)
    assert np.array_equal(f1, f2) and np.array_equal(ph1, ph2)


def test_split_step_after_set_state():
    """lbm_set_state lists the tiles of the new phi (and marks them) for the split step."""
    dims = (64, 48, 40)
    a, b = _sim(dims), _sim(dims)
    b.set_overlap(38)
    a.step(20)
    b.step(20)
    f, ph = a.get_state()
    a.set_state(f, ph)
    b.set_state(f, ph)
    a.step(25)
    b.step(25)
    fa, pa = a.get_state()
    fb, pb = b.get_state()
    a.close()
    b.close()
    assert np.array_equal(fa, fb) and np.array_equal(pa, pb)


def test_split_step_refused_where_it_does_not_apply():
    """Odd nx (the one-cell hydrodynamic kernel) and the near-contact pass off: one stream only."""
    for cfg in (W.base_config(3, 33, 17, 12, 19, rho_g=0.1), W.base_config(3, 32, 24, 16, 19, rho_g=0.1, nci_on=0)):
        sim = B.Lbm(cfg)
        assert sim.overlap() == 0
        sim.set_overlap(0)
        with pytest.raises(B.LbmError) as e:
            sim.set_overlap(4)
        assert e.value.code == B.LBM_ERR_STATE
        sim.close()
    sim = B.Lbm(W.base_config(3, 32, 24, 16, 19, rho_g=0.1))
    with pytest.raises(B.LbmError) as e:
        sim.set_overlap(-1)
    assert e.value.code == B.LBM_ERR_ARG
    sim.close()
