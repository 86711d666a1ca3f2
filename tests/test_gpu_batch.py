"""Batched sweep: contexts advanced together through one CUDA graph give exactly the states that
per-case lbm_step calls give, and a sweep case follows the FP64 oracle."""
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


def _small_cases():
    """Uneven small cases, 2D and 3D, both stencil families, near-contact on and off."""
    cases = []
    for i, L in enumerate((24, 40, 32, 20, 36)):
        cfg = W.collision_sweep(1, seed=100 + i, grids=(L,))[0]
        if i == 3:
            cfg["nci_on"] = 0
        cases.append(cfg)
    c2 = W.base_config(2, 70, 38, 1, 9, rho_g=0.1)
    c2.update(centers=[(24.0, 19.3, 0.0), (45.5, 18.6, 0.0)], R=8.0,
              velocities=[(0.02, 0.0, 0.0), (-0.02, 0.0, 0.0)])
    cases.append(c2)
    c27 = W.collision_sweep(1, seed=7, grids=(28,))[0]
    c27["Q"] = 27
    cases.append(c27)
    return cases


def _states(sims):
    return [s.get_state() for s in sims]


@pytest.mark.parametrize("nstreams", [1, 3, 16])
def test_batch_matches_per_case_steps(nstreams):
    cases = _small_cases()
    single, batched = [], []
    for cfg in cases:
        phi, u = W.sweep_case_fields(cfg)
        for lst in (single, batched):
            s = B.Lbm(cfg)
            s.init_fields(phi, u)
            lst.append(s)
    batch = B.LbmBatch(batched, nstreams=nstreams)
    # even (graph only), odd (graph + one plain step), none, plain only, then an odd count followed
    # by an even one, so that the graph of the flipped buffer parity runs
    for n in (4, 3, 0, 1, 3, 2, 1, 4):
        batch.step(n)
        for s in single:
            s.step(n)
        for a, b in zip(_states(single), _states(batched)):
            assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    for a, b in zip(single, batched):
        ma, pa = a.mass()
        mb, pb = b.mass()
        assert ma == mb and np.array_equal(pa, pb)
    batch.close()
    for s in single + batched:
        s.close()


@pytest.mark.parametrize("flags", [1, 0])
def test_batch_of_split_step_contexts(flags):
    """Contexts running the split step (lbm_set_overlap) in a batch: the per-case graph (flags 1)
    captures their two-stream steps, the fused mode their odd plain steps; both bit-equal to
    one-stream per-case steps."""
    cases = _small_cases()
    single, batched = [], []
    for cfg in cases:
        phi, u = W.sweep_case_fields(cfg)
        for lst in (single, batched):
            s = B.Lbm(cfg)
            s.init_fields(phi, u)
            lst.append(s)
        split = cfg["dim"] == 3 and cfg["nci_on"] and cfg["nx"] % 2 == 0
        if split:
            batched[-1].set_overlap(8)
        assert batched[-1].overlap() == (8 if split else 0)
    assert sum(s.overlap() > 0 for s in batched) >= 3
    batch = B.LbmBatch(batched, nstreams=3, flags=flags)
    for n in (4, 3, 1, 2):
        batch.step(n)
        for s in single:
            s.step(n)
        for a, b in zip(_states(single), _states(batched)):
            assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    batch.close()
    for s in single + batched:
        s.close()


def _uniform_3d_cases(Q=19):
    """Uneven 3D cases of one lattice (x sides even), near-contact on and off: the fused batch."""
    cases = []
    for i, (L, nci) in enumerate(((24, 1), (40, 1), (32, 0), (20, 1), (36, 1), (28, 1))):
        cfg = W.collision_sweep(1, seed=200 + i, grids=(L,))[0]
        cfg["nci_on"] = nci
        cfg["Q"] = Q
        cases.append(cfg)
    c = W.base_config(3, 48, 22, 17, Q, rho_g=0.1)  # ragged y and z tiles
    phi, u = W.droplet_fields(c, [(14.5, 10.5, 8.0), (33.0, 11.5, 8.5)], [6.0, 6.0], [(0.02, 0, 0), (-0.02, 0, 0)])
    cases.append((c, phi, u))
    return cases


@pytest.mark.parametrize("Q,store,flags", [(19, "f32", 0), (19, "f16", 0), (27, "f32", 0), (19, "f32", 2), (19, "f32", 4),
                                           (19, "f32", 8), (19, "f32", 16), (19, "f16", 4 | 16)])
def test_fused_batch_matches_per_case_steps(Q, store, flags):
    """One launch per pass over all cases (fused mode, tuned or not): the same states, bit for bit,
    as per-case lbm_step calls, through even and odd step counts in both buffer parities."""
    single, batched = [], []
    for c in _uniform_3d_cases(Q):
        cfg, phi, u = c if isinstance(c, tuple) else (c, *W.sweep_case_fields(c))
        for lst in (single, batched):
            s = B.Lbm(cfg, store=store)
            s.init_fields(phi, u)
            lst.append(s)
    batch = B.LbmBatch(batched, nstreams=4, flags=flags)
    cfg = batch.config()
    assert cfg["hydro_ty"] in (2, 4, 8) and cfg["phase_rows"] in (2, 4)
    if flags:
        assert cfg["fused"] == 1
        assert cfg["hydro_ty"] == (2 if flags & 4 else (8 if flags & 8 else 4))
        assert cfg["phase_rows"] == (2 if flags & 16 else 4)
    else:
        t = cfg["tune_ms"]
        assert all(v > 0 for v in t.values())
        assert cfg["fused"] == (1 if t["step_fused"] < 0.97 * t["step_per_case"] else 0)
    for n in (4, 3, 0, 1, 3, 2, 1, 6):
        batch.step(n)
        for s in single:
            s.step(n)
        for a, b in zip(_states(single), _states(batched)):
            assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    for a, b in zip(single, batched):
        ma, pa = a.mass()
        mb, pb = b.mass()
        assert ma == mb and np.array_equal(pa, pb)
    batch.close()
    for s in single + batched:
        s.close()


def test_batch_modes():
    """Mixed 2D / 3D cases, or the per-case flag, give the per-case graph; uniform 3D cases fuse."""
    mixed = [B.Lbm(c) for c in _small_cases()[:2]] + [B.Lbm(W.base_config(2, 30, 20, 1, 9))]
    for s in mixed:
        N = W.ncells(s.cfg)
        s.init_fields(np.zeros(N), np.zeros((3, N)))
    b = B.LbmBatch(mixed, nstreams=2)
    assert b.config()["fused"] == 0
    b.close()
    b = B.LbmBatch(mixed[:2], nstreams=2, flags=B.LBM_BATCH_PER_CASE)
    assert b.config()["fused"] == 0
    b.close()
    b = B.LbmBatch(mixed[:2], nstreams=2, flags=B.LBM_BATCH_NO_TUNE)
    assert b.config()["fused"] == 1
    b.close()
    for bad in (32, 4 | 8):
        with pytest.raises(B.LbmError):
            B.LbmBatch(mixed[:2], nstreams=2, flags=bad)
    for s in mixed:
        s.close()


def test_batch_case_against_oracle():
    """A 40^3 sweep case advanced 20 steps inside a batch of three against the FP64 oracle."""
    cfgs = [W.collision_sweep(1, seed=s, grids=(L,))[0] for s, L in ((3, 40), (4, 24), (5, 32))]
    sims = []
    for cfg in cfgs:
        phi, u = W.sweep_case_fields(cfg)
        s = B.Lbm(cfg)
        s.init_fields(phi, u)
        sims.append(s)
    batch = B.LbmBatch(sims, nstreams=2)
    batch.step(20)
    cfg = cfgs[0]
    phi, u = W.sweep_case_fields(cfg)
    P = O.make_params(cfg)
    f = O.init(P, phi, u)
    fo, pho, _ = O.step(P, f, phi, 20)
    _, uo = O.moments(P, fo, pho)
    phg, ug, _ = sims[0].read_fields()
    assert np.max(np.abs(phg - pho)) <= 1e-5
    assert np.max(np.abs(ug - uo)) <= 1e-6
    batch.close()
    for s in sims:
        s.close()


def test_batch_refuses_contexts_reinitialised_out_of_step():
    """A context re-initialised outside the batch no longer holds either captured buffer parity
    together with the others: the batch refuses to launch rather than step stale buffers."""
    cfgs = [W.collision_sweep(1, seed=s, grids=(L,))[0] for s, L in ((11, 24), (12, 20))]
    sims = []
    for cfg in cfgs:
        phi, u = W.sweep_case_fields(cfg)
        s = B.Lbm(cfg)
        s.init_fields(phi, u)
        sims.append(s)
    batch = B.LbmBatch(sims, nstreams=2)
    batch.step(1)  # both contexts now hold the flipped parity
    phi, u = W.sweep_case_fields(cfgs[0])
    sims[0].init_fields(phi, u)  # back to the creation parity, the other context is not
    with pytest.raises(B.LbmError) as e:
        batch.step(2)
    assert e.value.code == B.LBM_ERR_STATE
    batch.close()
    for s in sims:
        s.close()


def test_batch_rejects_bad_contexts():
    cfg = W.collision_sweep(1, seed=1, grids=(20,))[0]
    phi, u = W.sweep_case_fields(cfg)
    checked = B.Lbm(cfg, mass_check_every=10)
    checked.init_fields(phi, u)
    fresh = B.Lbm(cfg)  # never initialised
    ok = B.Lbm(cfg)
    ok.init_fields(phi, u)
    with pytest.raises(B.LbmError) as e:
        B.LbmBatch([ok, checked])
    assert e.value.code == -1
    with pytest.raises(B.LbmError) as e:
        B.LbmBatch([ok, fresh])
    assert e.value.code == -5
    with pytest.raises(B.LbmError) as e:
        B.LbmBatch([ok, ok])
    assert e.value.code == -1
    for s in (checked, fresh, ok):
        s.close()
