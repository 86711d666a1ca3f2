"""Moment-record storage (LBM_STORE_MOMENTS, the thread-safe moment representation of Sec. 2.1):
each cell stores the record of its post-collision state and pulls f_i by evaluating the
regularized post-collision population (Eqs. 3, 11, 15-17, Guo term) at the record of x - c_i.
Against the FP64 oracle from the state that the record initialisation represents (cell x pulls
f_eq_i of x - c_i, i.e. the oracle's equilibrium populations streamed one step): the populations
it reconstructs, one step, and 200-step collisions, at the population store's tolerances."""
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


def _streamed(cfg, f):
    """f_i(x) -> f_i(x - c_i): the populations one periodic streaming step moves into each cell."""
    c, _ = O.lattice(cfg["dim"], cfg["Q"])
    shape = (cfg["nz"], cfg["ny"], cfg["nx"])
    out = np.empty_like(f)
    for i in range(cfg["Q"]):
        out[i] = np.roll(f[i].reshape(shape), shift=(c[i, 2], c[i, 1], c[i, 0]), axis=(0, 1, 2)).reshape(-1)
    return out


def _record_start(cfg, phi, u, pstar=None):
    """The oracle's state that the record initialisation of (phi, u, p*) represents."""
    P = O.make_params(cfg)
    f = _streamed(cfg, O.init(P, phi, u, pstar=pstar))
    return P, f


def test_streamed_helper_is_a_pull():
    """The test's own shift, pinned on a marked cell: f_i lands at x + c_i."""
    cfg = W.base_config(3, 7, 5, 4, 19)
    c, _ = O.lattice(3, 19)
    f = np.zeros((19, 7 * 5 * 4))
    x, y, z = 6, 0, 3
    f[:, x + 7 * (y + 5 * z)] = 1.0
    g = _streamed(cfg, f)
    for i in range(19):
        xs, ys, zs = (x + c[i, 0]) % 7, (y + c[i, 1]) % 5, (z + c[i, 2]) % 4
        assert g[i, xs + 7 * (ys + 5 * zs)] == 1.0 and g[i].sum() == 1.0


@pytest.mark.parametrize("Q,shape,seed", [(19, (37, 21, 13), 31), (27, (35, 19, 11), 32), (19, (64, 12, 9), 33)])
def test_record_store_populations_and_one_step(Q, shape, seed):
    """Random smooth fields with nearly touching droplets, p* noise: the populations the records
    represent (within FP32 rounding of the record), the moments of the pulled populations, then one
    step (populations, phi, u, p*), on ragged tile counts."""
    cfg = W.base_config(3, *shape, Q, rho_g=0.1)
    phi, u = W.smooth_random_fields(cfg, seed=seed)
    phi = W.to_q30_grid(phi)
    ps = W.noise(W.ncells(cfg), seed + 1, 5e-3)
    P, f = _record_start(cfg, phi, u, ps)
    sim = B.Lbm(cfg, store="mom")
    sim.init_fields(phi, u, ps)
    fg, phg = sim.get_state()
    assert np.max(np.abs(fg - f)) < 1e-6 and np.array_equal(phg, phi)
    _, ug, psg = sim.read_fields()
    pso, uo = O.moments(P, f, phi)
    assert np.max(np.abs(ug - uo)) < 1e-6 and np.max(np.abs(psg - pso)) < 1e-6
    sim.step(1)
    fg, phg = sim.get_state()
    fo, pho, _ = O.step(P, f, phi, 1)
    _, ug, psg = sim.read_fields()
    pso, uo = O.moments(P, fo, pho)
    sim.close()
    df, dphi = float(np.max(np.abs(fg - fo))), float(np.max(np.abs(phg - pho)))
    du, dps = float(np.max(np.abs(ug - uo))), float(np.max(np.abs(psg - pso)))
    print(f"[moments] D3Q{Q} one step: |df| {df:.2e} |dphi| {dphi:.2e} |du| {du:.2e} |dp*| {dps:.2e}")
    assert df < 1e-6 and du < 1e-6 and dps < 1e-6
    # the pulled populations carry one more FP32 stage than stored ones (their evaluation from the
    # FP32 record), about 1e-7 in u; phi moves by the face fluxes of u, so 3e-7 instead of 1e-7
    assert dphi < 3e-7
    assert np.round(phg * 2 ** 30).sum() == np.round(phi * 2 ** 30).sum()


@pytest.mark.parametrize("Q", [19, 27])
def test_record_store_collision_200_steps(Q):
    """Off-centre collision (64x40x40, ratio 10, R = 8) with the near-contact pass on, 200 steps:
    max|dphi| <= 1e-5, max|du| <= 1e-6 against the FP64 oracle."""
    cfg = W.base_config(3, 64, 40, 40, Q, rho_g=0.1)
    cx, cy, cz = 31.5, 19.5, 19.5
    phi, u = W.droplet_fields(cfg, [(cx - 12.0, cy - 2.1, cz), (cx + 12.0, cy + 2.1, cz)], [8.0, 8.0],
                              [(0.02, 0, 0), (-0.02, 0, 0)])
    phi = W.to_q30_grid(phi)
    P, f = _record_start(cfg, phi, u)
    fo, pho, _ = O.step(P, f, phi, 200)
    _, uo = O.moments(P, fo, pho)
    sim = B.Lbm(cfg, store="mom")
    sim.init_fields(phi, u)
    sim.step(200)
    phg, ug, _ = sim.read_fields()
    m = sim.mass()[0]
    sim.close()
    dphi, du = float(np.max(np.abs(phg - pho))), float(np.max(np.abs(ug - uo)))
    print(f"[moments] D3Q{Q} max|dphi|={dphi:.3e} max|du|={du:.3e}")
    assert dphi <= 1e-5 and du <= 1e-6
    assert m == pytest.approx(float(np.round(phi * 2 ** 30).sum()) / 2 ** 30, abs=0, rel=1e-15)


def test_record_store_batch_and_refusals():
    """A batch of record-store contexts steps as the per-case graph (bit-equal to lbm_step); the
    record store refuses lbm_set_state, 2D lattices and the split step."""
    cfgs = [W.base_config(3, 40, 24, 16, 19, rho_g=0.1), W.base_config(3, 32, 32, 20, 19, rho_g=0.1)]
    sims, refs = [], []
    for k, cfg in enumerate(cfgs):
        phi, u = W.smooth_random_fields(cfg, seed=40 + k)
        phi = W.to_q30_grid(phi)
        a, b = B.Lbm(cfg, store="mom"), B.Lbm(cfg, store="mom")
        a.init_fields(phi, u)
        b.init_fields(phi, u)
        sims.append(a)
        refs.append(b)
    batch = B.LbmBatch(sims, nstreams=2)
    assert batch.config()["fused"] == 0
    batch.step(5)
    batch.synchronize()
    for a, b in zip(sims, refs):
        b.step(5)
        fa, pa = a.get_state()
        fb, pb = b.get_state()
        assert np.array_equal(fa, fb) and np.array_equal(pa, pb)
    batch.close()
    f, ph = refs[0].get_state()
    with pytest.raises(B.LbmError) as e:
        refs[0].set_state(f, ph)
    assert e.value.code == B.LBM_ERR_STATE
    with pytest.raises(B.LbmError) as e:
        refs[0].set_overlap(8)
    assert e.value.code == B.LBM_ERR_STATE
    for s in sims + refs:
        s.close()
    with pytest.raises(B.LbmError) as e:
        B.Lbm(W.base_config(2, 32, 16, 1, 9), store="mom")
    assert e.value.code == B.LBM_ERR_ARG
