"""GPU parity: the CUDA path (through the C ABI) against the FP64 CPU oracle on identical seeded
inputs. Tolerances: single step (identical input) 1e-6 on populations and velocities, 1e-7 on
phi; trajectories max|dphi| <= 1e-5 and max|du| <= 1e-6 after 200 steps; near-contact decisions
identical except at cells whose oracle decision margin is below 1e-5."""
import os

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


def _random_state(cfg, seed, f_noise=2e-3):
    phi, u = W.smooth_random_fields(cfg, seed=seed)
    phi = W.to_q30_grid(phi)
    P = O.make_params(cfg)
    N = W.ncells(cfg)
    ps = W.noise(N, seed + 1, 5e-3)
    f = O.init(P, phi, u, pstar=ps)
    _, w = O.lattice(cfg["dim"], cfg["Q"])
    f = f + f_noise * w[:, None] * W.noise((cfg["Q"], N), seed + 2)
    return P, phi, u, f


def _compare_nci(sim, P, phi, tol_margin=1e-5):
    part_g, frep_g = sim.read_nci()
    part_o, frep_o, marg = O.nci(P, phi)
    chi_o = part_o[:, 0] != O.NO_PARTNER
    diff = np.any(part_g != part_o, axis=1)
    assert np.all(marg[diff] < tol_margin), f"{diff.sum()} partner mismatches at robust cells"
    ok = ~diff
    scale = max(np.max(np.abs(frep_o)), 1e-30)
    assert np.max(np.abs(frep_g[:, ok] - frep_o[:, ok])) <= 2e-5 * scale
    return int(chi_o.sum()), int(diff.sum())


CASES_1STEP = [
    (3, 19, (37, 21, 13), 11, "f32"),
    (3, 27, (35, 19, 11), 12, "f32"),
    (2, 9, (45, 27, 1), 13, "f32"),
    (3, 19, (8, 8, 8), 14, "f32"),
    (3, 19, (64, 12, 9), 15, "f32"),
]


@pytest.mark.parametrize("dim,Q,shape", [(3, 19, (37, 21, 13)), (3, 27, (35, 19, 11)), (2, 9, (45, 27, 1))])
@pytest.mark.parametrize("store", ["f32", "f16", "bf16"])
def test_initial_populations_are_the_equilibrium(dim, Q, shape, store):
    """lbm_init_fields sets f_eq(p*, u) of Eq. 11 (evaluated in FP32): every population within a few
    FP32 units of the oracle's FP64 equilibrium (FP32 store), or within one unit of the storage
    precision of f / w (FP16, BF16). A dropped term (the cubic 4.5 (c.u)^3 is above 1e-5 here) or a
    swapped direction fails by orders of magnitude."""
    cfg = W.base_config(dim, *shape, Q, rho_g=0.1)
    phi, u = W.smooth_random_fields(cfg, seed=29)
    phi = W.to_q30_grid(phi)
    u = 3.0 * u  # |u| up to about 0.1, so every term of the polynomial is well above FP32 rounding
    N = W.ncells(cfg)
    ps = W.noise(N, 30, 5e-3)
    P = O.make_params(cfg)
    fo = O.init(P, phi, u, pstar=ps)
    c, w = O.lattice(dim, Q)
    sim = B.Lbm(cfg, store=store)
    sim.init_fields(phi, u, ps)
    fg, phg = sim.get_state()
    sim.close()
    assert np.array_equal(phg, phi)
    go, gg = fo / w[:, None], fg / w[:, None]
    c = np.asarray(c, dtype=np.float64)
    assert np.max(np.abs(c @ u)) > 0.05
    if store == "f32":
        # FP32 rounding scales with sum_a |c_a u_a| (the sum c.u may cancel), with |p*| and |u|^2
        cabs = np.abs(c) @ np.abs(u)
        scale = np.abs(ps)[None, :] + 3.0 * cabs + 4.5 * cabs ** 2 + 1.5 * np.sum(u * u, axis=0)[None, :] + 1e-3
        err = np.abs(gg - go) / scale
        assert np.max(err) <= 8 * 2.0 ** -24, f"max error {np.max(err):.3e} of the term scale"
    else:
        ulp = 2.0 ** -10 if store == "f16" else 2.0 ** -7
        assert np.all(np.abs(gg - go) <= ulp * np.abs(go) + 2.0 ** -24)


@pytest.mark.parametrize("dim,Q,shape,seed,store", CASES_1STEP)
def test_single_step_identical_input(dim, Q, shape, seed, store):
    """One step from a random non-equilibrium state with two nearly touching droplets: near-contact
    partners and force, velocity moments, post-step populations and phi, on ragged tile counts."""
    cfg = W.base_config(dim, *shape, Q, rho_g=0.1)
    P, phi, u, f = _random_state(cfg, seed)
    sim = B.Lbm(cfg, store=store)
    sim.set_state(f, phi)
    nchi, nmis = _compare_nci(sim, P, phi)
    assert nchi > 0
    _, ug, psg = sim.read_fields()
    pso, uo = O.moments(P, f, phi)
    assert np.max(np.abs(ug - uo)) < 1e-6
    assert np.max(np.abs(psg - pso)) < 1e-6
    sim.step(1)
    fg, phg = sim.get_state()
    fo, pho, _ = O.step(P, f, phi, 1)
    assert np.max(np.abs(fg - fo)) < 1e-6
    assert np.max(np.abs(phg - pho)) < 1e-7
    m0 = np.round(phi * 2 ** 30).sum()
    assert np.round(phg * 2 ** 30).sum() == m0  # exact fixed-point conservation


@pytest.mark.parametrize("dim,Q,shape,seed,store", CASES_1STEP[:3])
def test_single_step_fp64_decisions(dim, Q, shape, seed, store):
    """The oracle with every near-contact decision (gate, similarity, facing, tie-break) taken in
    FP64 on FP64 normals, against the kernels' binary32 decisions: partners identical except where
    the FP64 decision margin is below 1e-5; then one step of populations and phi."""
    cfg = W.base_config(dim, *shape, Q, rho_g=0.1, decide_f32=0)
    P, phi, u, f = _random_state(cfg, seed)
    assert P.decide_f32 == 0
    sim = B.Lbm(cfg, store=store)
    sim.set_state(f, phi)
    nchi, _ = _compare_nci(sim, P, phi)
    assert nchi > 0
    part_g, _ = sim.read_nci()
    part_o, _, _ = O.nci(P, phi)
    diff = np.any(part_g != part_o, axis=1)
    print(f"[parity] FP64 decisions: {int(diff.sum())} of {nchi} near-contact cells decided differently")
    # a decision taken differently (only where its margin is below 1e-5, checked above) changes the
    # force at its cell; one step carries that to the cell's lattice neighbours (streaming, and the
    # face velocities of the phase update), which are left out of the comparison
    reach = _dilate(diff, cfg)
    sim.step(1)
    fg, phg = sim.get_state()
    fo, pho, _ = O.step(P, f, phi, 1)
    assert np.max(np.abs(fg - fo)[:, ~reach]) < 1e-6
    assert np.max(np.abs(phg - pho)[~reach]) < 1e-7


def _dilate(mask, cfg):
    """mask grown by one cell in every direction (3x3x3, 3x3 in 2D), periodic."""
    g = mask.reshape(cfg["nz"], cfg["ny"], cfg["nx"])
    out = g.copy()
    zs = (-1, 0, 1) if cfg["dim"] == 3 else (0,)
    for dz in zs:
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                out |= np.roll(g, (dz, dy, dx), axis=(0, 1, 2))
    return out.ravel()


@pytest.mark.parametrize("which", ["C1", "C2"])
def test_trajectories_fp64_decisions_200_steps(which):
    """The 2D head-on (C1) and 3D off-centre (C2) collisions against the oracle with FP64 near-contact
    decisions: max|dphi| <= 1e-5 and max|du| <= 1e-6 after 200 steps."""
    cfg, phi, u = W.droplets_head_on_2d() if which == "C1" else W.droplets_offcentre_3d()
    cfg["decide_f32"] = 0
    phi = W.to_q30_grid(phi)
    P = O.make_params(cfg)
    f = O.init(P, phi, u)
    fo, pho, _ = O.step(P, f, phi, 200)
    _, uo = O.moments(P, fo, pho)
    sim = B.Lbm(cfg)
    sim.init_fields(phi, u)
    sim.step(200)
    phg, ug, _ = sim.read_fields()
    _check_traj(phg, pho, ug, uo)


def test_head_on_2d_128x64_200_steps():
    """2D head-on collision (128x64 D2Q9), 200 steps: max|dphi| <= 1e-5, max|du| <= 1e-6."""
    cfg, phi, u = W.droplets_head_on_2d()
    phi = W.to_q30_grid(phi)
    P = O.make_params(cfg)
    f = O.init(P, phi, u)
    fo, pho, _ = O.step(P, f, phi, 200)
    _, uo = O.moments(P, fo, pho)
    sim = B.Lbm(cfg)
    sim.init_fields(phi, u)
    sim.step(200)
    phg, ug, _ = sim.read_fields()
    _check_traj(phg, pho, ug, uo)


def _check_traj(phg, pho, ug, uo, tphi=1e-5, tu=1e-6):
    dphi, du = float(np.max(np.abs(phg - pho))), float(np.max(np.abs(ug - uo)))
    print(f"[parity] max|dphi|={dphi:.3e} max|du|={du:.3e}")
    assert dphi <= tphi and du <= tu, f"max|dphi|={dphi:.3e} (tol {tphi}), max|du|={du:.3e} (tol {tu})"


def test_head_on_2d_128x64_contact_400_steps():
    """The same collision through its near-contact phase (the repulsion switches on near step
    250): partners compared at step 400, and fields within 1e-5 (phi) / 1e-6 (u)."""
    cfg, phi, u = W.droplets_head_on_2d()
    phi = W.to_q30_grid(phi)
    P = O.make_params(cfg)
    f = O.init(P, phi, u)
    fo, pho, _ = O.step(P, f, phi, 400)
    _, uo = O.moments(P, fo, pho)
    sim = B.Lbm(cfg)
    sim.init_fields(phi, u)
    sim.step(400)
    phg, ug, _ = sim.read_fields()
    _check_traj(phg, pho, ug, uo)
    # near-contact decisions on the GPU's own phi^400, same input on both sides: identical partners
    # except where the oracle's decision margin is below 1e-5, forces within 2e-5 of their maximum
    nchi, _ = _compare_nci(sim, P, phg)
    assert nchi > 0
    # and along the two trajectories: the GPU's partners on its phi against the oracle's on its own
    # phi (they differ by <= 1e-5); a decision may differ only where the oracle's margin is below 1e-3
    part_g, _ = sim.read_nci()
    part_o, _, marg_o = O.nci(P, pho)
    chi_o = part_o[:, 0] != O.NO_PARTNER
    assert chi_o.sum() > 0
    diff = np.any(part_g != part_o, axis=1)
    assert np.all(marg_o[diff] < 1e-3), f"{diff.sum()} trajectory partner mismatches at robust cells"
    assert diff.sum() <= 0.02 * chi_o.sum()


def test_offcentre_3d_128x64x64_200_steps():
    """3D off-centre collision (128x64x64 D3Q19, ratio 10, seeded impact offset), 200 steps:
    max|dphi| <= 1e-5, max|du| <= 1e-6."""
    cfg, phi, u = W.droplets_offcentre_3d()
    phi = W.to_q30_grid(phi)
    P = O.make_params(cfg)
    f = O.init(P, phi, u)
    fo, pho, _ = O.step(P, f, phi, 200)
    _, uo = O.moments(P, fo, pho)
    sim = B.Lbm(cfg)
    sim.init_fields(phi, u)
    sim.step(200)
    phg, ug, _ = sim.read_fields()
    _check_traj(phg, pho, ug, uo)


def test_d3q27_collision_200_steps():
    """The paper's own hydrodynamic lattice, D3Q27, on an off-centre collision (64x40x40, ratio 10,
    R = 8), 200 steps: max|dphi| <= 1e-5, max|du| <= 1e-6 against the FP64 oracle."""
    cfg = W.base_config(3, 64, 40, 40, 27, rho_g=0.1)
    cx, cy, cz = 31.5, 19.5, 19.5
    phi, u = W.droplet_fields(cfg, [(cx - 12.0, cy - 2.1, cz), (cx + 12.0, cy + 2.1, cz)], [8.0, 8.0],
                              [(0.02, 0, 0), (-0.02, 0, 0)])
    phi = W.to_q30_grid(phi)
    P = O.make_params(cfg)
    f = O.init(P, phi, u)
    fo, pho, _ = O.step(P, f, phi, 200)
    _, uo = O.moments(P, fo, pho)
    sim = B.Lbm(cfg)
    sim.init_fields(phi, u)
    sim.step(200)
    phg, ug, _ = sim.read_fields()
    _check_traj(phg, pho, ug, uo)


@pytest.mark.parametrize("store,tol", [("f16", 1e-3), ("bf16", 1e-3)])
def test_half_precision_store_phi_error_and_mass(store, tol):
    """Populations stored as FP16/BF16 (f/w_i) with FP32 arithmetic, ratio-100 collision
    (128x64x64, R = 12), 200 steps: phi error against the FP64 oracle below tol, phi mass exact."""
    cfg, phi, u = W.droplets_head_on_3d(nx=128, ny=64, nz=64, R=12.0)
    phi = W.to_q30_grid(phi)
    P = O.make_params(cfg)
    f = O.init(P, phi, u)
    fo, pho, _ = O.step(P, f, phi, 200)
    sim = B.Lbm(cfg, store=store)
    sim.init_fields(phi, u)
    m0, _ = sim.mass()
    sim.step(200)
    m1, _ = sim.mass()
    phg, _, _ = sim.read_fields(want=("phi",))
    dphi = float(np.max(np.abs(phg - pho)))
    assert dphi <= tol, f"{store}: max|dphi|={dphi:.3e}"
    assert abs(m1 - m0) <= 1e-12 * abs(m0)


def test_mass_and_momentum_reductions():
    """lbm_mass: sum(phi) equals the FP64 sum of the read-back phi; sum(rho u) equals the FP64
    sum from the read-back fields."""
    cfg = W.base_config(3, 33, 17, 12, 19, rho_g=0.1)
    P, phi, u, f = _random_state(cfg, 5)
    sim = B.Lbm(cfg)
    sim.set_state(f, phi)
    sim.step(3)
    m, mom = sim.mass()
    phg, ug, _ = sim.read_fields()
    rho = cfg["rho_g"] + (cfg["rho_l"] - cfg["rho_g"]) * phg
    assert abs(m - phg.sum()) <= 1e-12 * abs(m)
    assert np.max(np.abs(mom - (rho * ug).sum(axis=1))) <= 1e-9


def test_zero_steps_and_state_roundtrip():
    cfg = W.base_config(3, 20, 12, 9, 27)
    P, phi, u, f = _random_state(cfg, 8)
    sim = B.Lbm(cfg)
    sim.set_state(f, phi)
    sim.step(0)
    fg, phg = sim.get_state()
    assert np.max(np.abs(fg - f)) < 1e-7 * np.max(np.abs(f)) + 1e-12
    assert np.array_equal(phg, phi)


def test_nci_off_and_single_phase():
    """Degenerate cases: repulsion off (chi read-back empty when nothing is near), uniform phi
    (no interface: forces vanish) keeps a uniform flow exactly uniform."""
    cfg = W.base_config(3, 16, 8, 8, 19, nci_on=0)
    N = W.ncells(cfg)
    phi = np.ones(N)
    u = np.zeros((3, N))
    u[0] = 0.03
    sim = B.Lbm(cfg)
    sim.init_fields(phi, u)
    sim.step(10)
    phg, ug, psg = sim.read_fields()
    assert np.max(np.abs(ug[0] - 0.03)) < 1e-7
    assert np.max(np.abs(ug[1:])) < 1e-7
    assert np.array_equal(phg, phi)


def test_step_before_init_and_nan_detection():
    cfg = W.base_config(3, 16, 8, 8, 19)
    sim = B.Lbm(cfg, mass_check_every=1)
    with pytest.raises(B.LbmError) as ei:
        sim.step(1)
    assert ei.value.code == B.LBM_ERR_STATE
    N = W.ncells(cfg)
    phi, u = W.droplet_fields(cfg, [(8, 4, 4)], [3.0], [(0, 0, 0)])
    u[0, 5] = np.nan  # injected on the host: the periodic check must report it
    sim.init_fields(phi, u)
    with pytest.raises(B.LbmError) as ei:
        sim.step(2)
    assert ei.value.code == B.LBM_ERR_UNSTABLE


def test_full_size_single_step_256x128x128():
    """The benchmark's launch configuration (256x128x128 D3Q19, ratio 100): one step from the
    initial state against the oracle on the whole grid."""
    cfg, phi, u = W.droplets_head_on_3d()
    phi = W.to_q30_grid(phi)
    P = O.make_params(cfg)
    f = O.init(P, phi, u)
    fo, pho, _ = O.step(P, f, phi, 1)
    sim = B.Lbm(cfg)
    sim.init_fields(phi, u)
    sim.step(1)
    fg, phg = sim.get_state()
    assert np.max(np.abs(fg - fo)) < 1e-6
    assert np.max(np.abs(phg - pho)) < 1e-7


def _half_box_centroids(cfg, ph):
    nx, ny, nz = cfg["nx"], cfg["ny"], cfg["nz"]
    g = np.asarray(ph).reshape(nz, ny, nx)
    out = []
    for sl in (slice(0, nx // 2), slice(nx // 2, nx)):
        m = g[:, :, sl]
        zz, yy, xx = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx)[sl], indexing="ij")
        out.append([(m * xx).sum() / m.sum(), (m * yy).sum() / m.sum(), (m * zz).sum() / m.sum()])
    return np.array(out)


def test_offcentre_3d_centroids_after_2000_steps():
    """Droplet centroids (phi-weighted, per half-box in x) within 0.05 cells of the FP64 oracle's at
    every stored checkpoint up to 2000 steps. The oracle's centroids are stored in
    tests/golden/offcentre_3d_centroids.txt, written by make_offcentre_centroids.py beside it."""
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "offcentre_3d_centroids.txt")
    rows = np.loadtxt(path, comments="#")
    cfg, phi, u = W.droplets_offcentre_3d()
    phi = W.to_q30_grid(phi)
    sim = B.Lbm(cfg)
    sim.init_fields(phi, u)
    done = 0
    for row in rows:
        step = int(row[0])
        sim.step(step - done)
        done = step
        phg, _, _ = sim.read_fields(want=("phi",))
        err = np.max(np.abs(_half_box_centroids(cfg, phg) - row[1:].reshape(2, 3)))
        assert err <= 0.05, f"step {step}: centroid error {err:.4f} cells"
    assert done == 2000


@pytest.mark.parametrize("case", ["E1", "E2"])
def test_paper_impacts_density_ratio_1000(case):
    """The paper's impact set-ups (Sec. 3.1) at density ratio 1000, reduced to 128x64x64 with D = 20:
    E1 head-on (We 4.6) and E2 off-axis (We 4.8, B = 0.32).
    (a) the approach, 50 steps from the initial fields: max|dphi| <= 1e-5, max|du| <= 1e-6;
    (b) at the oracle's own state after 100 steps (in contact, the repulsion active), identical input
        on both sides: near-contact partners identical except where the oracle's decision margin is
        below 1e-5, and one step of populations and phi within 1e-6 / 1e-7 outside the reach of a
        decision taken differently.
    Through contact the two trajectories are not compared point by point: the facing decisions of
    Eqs. 61-65 are discontinuous, and in the mirror-symmetric head-on film a decision flipped by
    binary32 rounding changes the force by O(A_rep) at that cell (measured: E1 departs to 1e-3 by
    step 125 with the repulsion on, and stays at 1e-6 with it off)."""
    cfg, phi, u = W.droplets_paper_impact(case, D=20.0, shape=(128, 64, 64))
    phi = W.to_q30_grid(phi)
    P = O.make_params(cfg)
    f = O.init(P, phi, u)
    f50, ph50, _ = O.step(P, f, phi, 50)
    _, u50 = O.moments(P, f50, ph50)
    sim = B.Lbm(cfg)
    sim.init_fields(phi, u)
    sim.step(50)
    phg, ug, _ = sim.read_fields()
    _check_traj(phg, ph50, ug, u50)
    f100, ph100, _ = O.step(P, f50, ph50, 50)
    assert np.all(np.isfinite(f100)) and np.all(np.isfinite(ph100))
    sim.set_state(f100, ph100)
    nchi, _ = _compare_nci(sim, P, ph100)
    assert nchi > 0, "the repulsion is not active at step 100"
    part_g, _ = sim.read_nci()
    part_o, _, _ = O.nci(P, ph100)
    reach = _dilate(np.any(part_g != part_o, axis=1), cfg)
    sim.step(1)
    fg, phg = sim.get_state()
    fo, pho, _ = O.step(P, f100, ph100, 1)
    assert np.max(np.abs(fg - fo)[:, ~reach]) < 1e-6
    assert np.max(np.abs(phg - pho)[~reach]) < 1e-7
    sim.close()


@pytest.mark.parametrize("case", ["E1", "E2"])
def test_paper_impacts_density_ratio_1000_stable(case):
    """The same reduced E1/E2 set-ups at density ratio 1000 on the GPU alone for 1500 steps, through
    approach, contact and rebound: the periodic FP64 check finds no NaN/Inf, phi mass is exact, and
    both droplets keep their liquid cores (phi > 1/2 somewhere in each half of the box)."""
    cfg, phi, u = W.droplets_paper_impact(case, D=20.0, shape=(128, 64, 64))
    phi = W.to_q30_grid(phi)
    sim = B.Lbm(cfg, mass_check_every=100, mass_tol=0.0)
    sim.init_fields(phi, u)
    m0, _ = sim.mass()
    sim.step(1500)
    m1, _ = sim.mass()
    phg, ug, _ = sim.read_fields()
    assert m1 == m0
    assert np.all(np.isfinite(phg)) and np.all(np.isfinite(ug))
    assert np.max(np.abs(ug)) < 0.2
    g = phg.reshape(cfg["nz"], cfg["ny"], cfg["nx"])
    assert g[:, :, :cfg["nx"] // 2].max() > 0.5 and g[:, :, cfg["nx"] // 2:].max() > 0.5
    sim.close()
@pytest.fixture(scope="module")
def c3_oracle():
    """The FP64 oracle's phi and velocity on the full 256x128x128 ratio-100 collision after 50, 100
    and 200 steps (about four minutes of host time, shared by the tests below)."""
    cfg, phi, u = W.droplets_head_on_3d()
    phi = W.to_q30_grid(phi)
    P = O.make_params(cfg)
    f = O.init(P, phi, u)
    out, ph, done = {}, phi, 0
    for k in (50, 100, 200):
        f, ph, _ = O.step(P, f, ph, k - done)
        done = k
        _, uo = O.moments(P, f, ph)
        out[k] = (ph.copy(), uo)
    return cfg, phi, u, out


def _c3_check(cfg, phi, u, ref, store, tmax, tq999, tu):
    sim = B.Lbm(cfg, store=store)
    sim.init_fields(phi, u)
    m0, _ = sim.mass()
    done, fails = 0, []
    for k in (50, 100, 200):
        sim.step(k - done)
        done = k
        phg, ug, _ = sim.read_fields(want=("phi", "u"))
        pho, uo = ref[k]
        d = np.abs(phg - pho)
        dmax, dq = float(d.max()), float(np.quantile(d, 0.999))
        du = float(np.max(np.abs(ug - uo)))
        dc = float(np.max(np.abs(_half_box_centroids(cfg, phg) - _half_box_centroids(cfg, pho))))
        print(f"[parity] C3 {store} step {k}: max|dphi|={dmax:.3e} q999={dq:.3e} max|du|={du:.3e} centroids {dc:.2e}")
        if k in tmax and dmax > tmax[k]:
            fails.append(f"step {k}: max|dphi| {dmax:.3e} > {tmax[k]}")
        if k in tq999 and dq > tq999[k]:
            fails.append(f"step {k}: 99.9th percentile of |dphi| {dq:.3e} > {tq999[k]}")
        if k in tu and du > tu[k]:
            fails.append(f"step {k}: max|du| {du:.3e} > {tu[k]}")
        if k == 200 and dc > 0.05:
            fails.append(f"step {k}: centroid error {dc:.3e} cells > 0.05")
    m1, _ = sim.mass()
    sim.close()
    assert m1 == m0, "phi mass changed"
    assert not fails, "; ".join(fails)


def test_full_size_fp32_against_fp64_oracle(c3_oracle):
    """The benchmark's collision at full size (256x128x128 D3Q19, ratio 100, the bench's launch
    configuration) in FP32 against the FP64 oracle: max|dphi| <= 1e-5 and max|du| <= 1e-6 at steps 50
    and 100; at step 200, after the films have formed and the facing decisions in the mirror-symmetric
    film make the two trajectories part pointwise, the 99.9th percentile of |dphi| <= 1e-5 and the
    droplet centroids within 0.05 cells; phi mass exact."""
    cfg, phi, u, ref = c3_oracle
    _c3_check(cfg, phi, u, ref, "f32", {50: 1e-5, 100: 1e-5}, {200: 1e-5}, {50: 1e-6, 100: 1e-6})


@pytest.mark.parametrize("store", ["f16", pytest.param("bf16", marks=pytest.mark.xfail(
    strict=True, reason="BF16 storage misses the 1e-3 phi target: 99.9th percentile 1.3e-3 at step 100"))])
def test_full_size_half_store_against_fp64_oracle(c3_oracle, store):
    """FP16 and BF16 population storage on the full-size collision against the FP64 oracle: max|dphi|
    <= 1e-3 at step 50; the 99.9th percentile of |dphi| <= 1e-3 at steps 100 and 200 (from about
    step 75 the droplet interiors, where phi departs from 1 by ~1 % and |grad phi| is comparable
    to eps_n, turn any perturbation of the size that half-precision storage makes into a local
    compressive flux of up to ~1e-3 per step); droplet centroids within 0.05 cells at step 200;
    phi mass exact."""
    cfg, phi, u, ref = c3_oracle
    _c3_check(cfg, phi, u, ref, store, {50: 1e-3}, {100: 1e-3, 200: 1e-3}, {})
