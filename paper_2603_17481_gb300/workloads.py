"""Seeded synthetic workloads: parameter sets and initial fields.

This module only places droplets/bubbles and draws random numbers. It holds none of the
method's arithmetic (no lattice, stencil, collision or near-contact code) so that the CUDA path
and the CPU reference can both take their inputs from it.

Initial fields follow the usual diffuse-interface set-up: every droplet (or bubble) is a
hyperbolic-tangent profile of width ``eps`` around its radius, phi = 1 in the liquid, and each
droplet carries its own uniform velocity weighted by its own profile.
"""
from __future__ import annotations

import math

import numpy as np

#: Near-contact detection and force parameters printed in Sec. 2.3.2 (w, q_th, eta, cos_opp) and
#: Sec. 2.2.6 / Eq. 71 (h0 = 1 lattice unit, p = 4). eps_q is a small floor. eps_n, the
#: regularisation of the normal grad(phi) / (|grad(phi)| + eps_n) (Eq. 57, also used for the
#: compressive normal of Eq. 25), is not given in the paper: 1e-4 keeps the normal well defined
#: where |grad(phi)| is round-off (bulk regions with phi slightly off 0 or 1), while changing it by
#: at most 0.1 % in the interfacial band where |grad(phi)| >= 0.1.
PAPER_NCI = dict(nci_on=1, w=3, q_th=0.125, eta=0.1, cos_opp=-0.8, h0=1.0, p=4.0,
                 eps_q=1e-12, eps_n=1e-4)

Q30 = float(1 << 30)


def base_config(dim, nx, ny, nz, Q, **kw):
    cfg = dict(dim=dim, nx=nx, ny=ny, nz=nz, Q=Q, rho_l=1.0, rho_g=1.0, nu_l=0.005, nu_g=0.05,
               sigma=0.02, eps=4.0, D=0.1, A_rep=0.02, g=(0.0, 0.0, 0.0))
    cfg.update(PAPER_NCI)
    cfg.update(kw)
    return cfg


def ncells(cfg):
    return cfg["nx"] * cfg["ny"] * cfg["nz"]


def to_q30_grid(phi):
    """Round phi to the nearest multiple of 2^-30 so that a fixed-point store holds it exactly."""
    return np.round(np.asarray(phi, dtype=np.float64) * Q30) / Q30


def _coords(cfg):
    nx, ny, nz = cfg["nx"], cfg["ny"], cfg["nz"]
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    return x.ravel().astype(np.float64), y.ravel().astype(np.float64), z.ravel().astype(np.float64)


def _min_image(d, L):
    return d - L * np.round(d / L)


def droplet_fields(cfg, centers, radii, velocities, bubbles=False):
    """phi and u (shape (3, N)) for a set of droplets (liquid inside) or bubbles (gas inside).

    Droplets: phi = min(1, sum_k prof_k); bubbles: phi = max(0, 1 - sum_k prof_k), with
    prof_k = (1 + tanh(2 (R_k - r_k) / eps)) / 2 and r_k the minimum-image distance to centre k.
    u = sum_k prof_k U_k.
    """
    eps = cfg["eps"]
    x, y, z = _coords(cfg)
    N = x.size
    prof_sum = np.zeros(N)
    u = np.zeros((3, N))
    for c, R, U in zip(centers, radii, velocities):
        dx = _min_image(x - c[0], cfg["nx"])
        dy = _min_image(y - c[1], cfg["ny"])
        dz = _min_image(z - c[2], cfg["nz"]) if cfg["dim"] == 3 else 0.0 * z
        r = np.sqrt(dx * dx + dy * dy + dz * dz)
        prof = 0.5 * (1.0 + np.tanh(2.0 * (R - r) / eps))
        prof_sum += prof
        for a in range(3):
            u[a] += prof * U[a]
    phi = np.maximum(0.0, 1.0 - prof_sum) if bubbles else np.minimum(1.0, prof_sum)
    return phi, u


# --------------------------------------------------------------------------------------------
# The five workloads (sizes, lattices, physical parameters) and their initial fields.
# --------------------------------------------------------------------------------------------

def droplets_head_on_2d():
    """2D head-on collision, 128x64 D2Q9, R = 16, centres 40 apart, +-0.02, density ratio 1."""
    cfg = base_config(2, 128, 64, 1, 9, steps=200)
    phi, u = droplet_fields(cfg, [(43.5, 31.5, 0.0), (83.5, 31.5, 0.0)], [16.0, 16.0],
                            [(0.02, 0, 0), (-0.02, 0, 0)])
    return cfg, phi, u


def droplets_offcentre_3d(seed=17481, nx=128, ny=64, nz=64, R=12.0):
    """3D collision, 128x64x64 D3Q19, R = 12, separation 2R + 8 along x, impact offset
    b ~ U(0, 1) * R along y, relative speed 0.04, density ratio 10."""
    cfg = base_config(3, nx, ny, nz, 19, rho_g=0.1, steps=2000)
    rng = np.random.default_rng(seed)
    b = float(rng.uniform(0.0, 1.0)) * R
    cx, cy, cz = (nx - 1) / 2.0, (ny - 1) / 2.0, (nz - 1) / 2.0
    sep = 2 * R + 8
    centers = [(cx - sep / 2, cy - b / 2, cz), (cx + sep / 2, cy + b / 2, cz)]
    phi, u = droplet_fields(cfg, centers, [R, R], [(0.02, 0, 0), (-0.02, 0, 0)])
    cfg["impact_offset"] = b
    return cfg, phi, u


def droplets_head_on_3d(nx=256, ny=128, nz=128, R=24.0, Q=19):
    """3D head-on collision, 256x128x128 D3Q19, R = 24, separation 2R + 8, speed 0.04, ratio 100."""
    cfg = base_config(3, nx, ny, nz, Q, rho_g=0.01, steps=5000)
    cx, cy, cz = (nx - 1) / 2.0, (ny - 1) / 2.0, (nz - 1) / 2.0
    sep = 2 * R + 8
    centers = [(cx - sep / 2, cy, cz), (cx + sep / 2, cy, cz)]
    phi, u = droplet_fields(cfg, centers, [R, R], [(0.02, 0, 0), (-0.02, 0, 0)])
    return cfg, phi, u


def droplets_paper_impact(case="E1", L=512, D=80.0, gap=8.0, Q=19, ratio=1000.0, shape=None):
    """The paper's droplet-impact set-ups of Sec. 3.1 as synthetic stress workloads: a periodic L^3
    box (paper: 512^3), two droplets of diameter D (paper: D_lu = 80), density ratio 1000,
    sigma = 0.02, moving along x with relative speed U from We = rho_l U^2 D / sigma.
    E1: head-on, We = 4.60, B = 0, nu_l = 0.005, nu_g = 0.05.
    E2: off-axis, We = 4.8, B = 0.32 (centre offset B D along y), nu_l = 0.0012, nu_g = 0.012.
    The paper does not state the initial separation; the surfaces start `gap` cells apart. `shape`
    (nx, ny, nz) replaces the cubic box for reduced cases."""
    if case == "E1":
        we, B, nu_l, nu_g = 4.60, 0.0, 0.005, 0.05
    elif case == "E2":
        we, B, nu_l, nu_g = 4.8, 0.32, 0.0012, 0.012
    else:
        raise ValueError(case)
    sigma, rho_l = 0.02, 1.0
    nx, ny, nz = shape if shape is not None else (L, L, L)
    cfg = base_config(3, nx, ny, nz, Q, rho_l=rho_l, rho_g=rho_l / ratio, nu_l=nu_l, nu_g=nu_g, sigma=sigma,
                      A_rep=sigma)
    U = math.sqrt(we * sigma / (rho_l * D))
    R = D / 2.0
    cx, cy, cz = (nx - 1) / 2.0, (ny - 1) / 2.0, (nz - 1) / 2.0
    sep = 2 * R + gap
    off = B * D
    centers = [(cx - sep / 2, cy - off / 2, cz), (cx + sep / 2, cy + off / 2, cz)]
    phi, u = droplet_fields(cfg, centers, [R, R], [(U / 2, 0, 0), (-U / 2, 0, 0)])
    cfg.update(case=case, We=we, B=B, U_rel=U, diameter=D)
    return cfg, phi, u


#: Grid edges of the batched collision sweep (cubic periodic boxes).
SWEEP_GRIDS = (48, 64, 80, 96)


def collision_sweep(n=512, seed=17481, sigma=1e-3, we_min=1.0, we_max=100.0, grids=SWEEP_GRIDS):
    """Parameter sets of the batched sweep: ``n`` independent 3D D3Q19 collisions, density ratio 10.

    Case i draws from ``default_rng(seed + i)``: its cubic grid edge L from ``grids``, R = L / 6, a
    Weber number We = rho_l U^2 (2R) / sigma log-uniform in [we_min, we_max], set through the
    relative speed U = sqrt(We sigma / (rho_l 2R)) (U <= 0.08 for sigma = 1e-3), and an impact
    offset b ~ U(0, 1) 2R along y. A_rep = sigma; viscosities as in the other collisions. The
    droplets start 2R + 8 apart along x, moving at -+U/2. Fields come from ``sweep_case_fields``.
    """
    out = []
    for i in range(n):
        rng = np.random.default_rng(seed + i)
        L = int(grids[int(rng.integers(0, len(grids)))])
        R = L / 6.0
        we = float(math.exp(rng.uniform(math.log(we_min), math.log(we_max))))
        b = float(rng.uniform(0.0, 1.0)) * 2.0 * R
        U = math.sqrt(we * sigma / (1.0 * 2.0 * R))
        cfg = base_config(3, L, L, L, 19, rho_g=0.1, sigma=sigma, A_rep=sigma, steps=1000)
        c = (L - 1) / 2.0
        sep = 2 * R + 8
        cfg.update(case=i, R=R, weber=we, impact_offset=b, speed=U,
                   centers=[(c - sep / 2, c - b / 2, c), (c + sep / 2, c + b / 2, c)],
                   velocities=[(U / 2, 0.0, 0.0), (-U / 2, 0.0, 0.0)])
        out.append(cfg)
    return out


def selftune_cases(diameters=(24, 32, 48), sigmas=(0.005, 0.01, 0.02), ratios=(0.5, 1.0, 2.0), we=4.6):
    """Head-on collisions over D x sigma x A_rep / sigma, for the film statistics of Sec. 3.3.

    Each case is a periodic box (2D + 24) x (D + 16)^2 with two droplets of diameter D, 2R + 8 apart
    along x, approaching at the relative speed U = sqrt(We sigma / (rho_l D)) with We = 4.6 (the
    head-on experiment of Sec. 3.1); density ratio 10 and the other parameters as in the
    collisions above. Fields come from ``sweep_case_fields``. (The diameter is stored as ``diameter``: ``D``
    is the phase-field mobility.)
    """
    out = []
    for D in diameters:
        for sg in sigmas:
            for r in ratios:
                R = D / 2.0
                L, T = int(2 * D + 24), int(D + 16)
                U = math.sqrt(we * sg / (1.0 * D))
                cfg = base_config(3, L, T, T, 19, rho_g=0.1, sigma=sg, A_rep=r * sg)
                c = (L - 1) / 2.0, (T - 1) / 2.0
                sep = 2 * R + 8
                cfg.update(R=R, diameter=float(D), weber=we, speed=U, A_over_sigma=r,
                           centers=[(c[0] - sep / 2, c[1], c[1]), (c[0] + sep / 2, c[1], c[1])],
                           velocities=[(U / 2, 0.0, 0.0), (-U / 2, 0.0, 0.0)])
                out.append(cfg)
    return out


def sweep_case_fields(cfg):
    """phi (rounded to the 2^-30 grid) and u of one sweep case."""
    phi, u = droplet_fields(cfg, cfg["centers"], [cfg["R"], cfg["R"]], cfg["velocities"])
    return to_q30_grid(phi), u


def swarm_centres(L, nb, rmin, rmax, gap, seed=17481, max_tries=2_000_000):
    """Rejection-sampled non-overlapping bubbles in a periodic cube: centre distance >= R_i + R_j + gap."""
    rng = np.random.default_rng(seed)
    cs, rs = [], []
    tries = 0
    while len(cs) < nb and tries < max_tries:
        tries += 1
        c = rng.uniform(0.0, L, size=3)
        r = rng.uniform(rmin, rmax)
        ok = True
        for c2, r2 in zip(cs, rs):
            d = _min_image(c - c2, L)
            if math.sqrt(float(d @ d)) < r + r2 + gap:
                ok = False
                break
        if ok:
            cs.append(c)
            rs.append(r)
    return np.array(cs), np.array(rs)


def bubble_swarm(L=512, nb=1500, seed=17481, rmin=8.0, rmax=12.0, gap_eps=2.0):
    """Buoyant bubble swarm, L^3 D3Q19, nb bubbles R ~ U[8, 12], ratio 100, g = 1e-6, sigma = 0.01.

    Bubble surfaces start at least gap_eps * eps apart, so that their diffuse interfaces do not
    overlap at t = 0: at a gap of 2 eps, phi midway between two bubbles is 0.96 (at a gap of eps it
    would be 0.76, inside the interfacial band, and such pairs merge before any film forms).
    """
    cfg = base_config(3, L, L, L, 19, rho_g=0.01, sigma=0.01, nu_l=1e-3, nu_g=1e-2, A_rep=0.01,
                      g=(0.0, 0.0, -1e-6), steps=10000)
    cs, rs = swarm_centres(L, nb, rmin, rmax, gap_eps * cfg["eps"], seed=seed)
    cfg["n_bubbles"] = len(cs)
    return cfg, cs, rs


def bubble_swarm_fields(cfg, cs, rs, cut=4.0):
    """phi of the bubble swarm (gas inside, phi = 0), u = 0, built box by box.

    Each bubble's profile (1 + tanh(2 (R - r) / eps)) / 2 is evaluated only within a cube of half
    width R + cut * eps around its centre (beyond it the profile is below 1.2e-7 for cut = 4 and is
    taken as 0); phi = max(0, 1 - sum of profiles), rounded to the 2^-30 grid. Returns phi (N,)
    and u (3, N) in x-fastest order.
    """
    nx, ny, nz = cfg["nx"], cfg["ny"], cfg["nz"]
    eps = cfg["eps"]
    acc = np.zeros((nz, ny, nx))
    for c, R in zip(cs, rs):
        h = int(math.ceil(R + cut * eps))
        lo = [int(math.floor(c[a])) - h for a in range(3)]
        ix = np.arange(lo[0], lo[0] + 2 * h + 2)
        iy = np.arange(lo[1], lo[1] + 2 * h + 2)
        iz = np.arange(lo[2], lo[2] + 2 * h + 2)
        dx, dy, dz = ix - c[0], iy - c[1], iz - c[2]
        r = np.sqrt(dz[:, None, None] ** 2 + dy[None, :, None] ** 2 + dx[None, None, :] ** 2)
        prof = 0.5 * (1.0 + np.tanh(2.0 * (R - r) / eps))
        prof[r > R + cut * eps] = 0.0
        acc[np.ix_(iz % nz, iy % ny, ix % nx)] += prof
    phi = np.maximum(0.0, 1.0 - acc).reshape(-1)
    return to_q30_grid(phi), np.zeros((3, phi.size))


def smooth_random_fields(cfg, seed, n_modes=4, amp_u=0.03, pairs=True):
    """Random smooth periodic phi in (0, 1) with sharp-ish interfaces plus a smooth random u.

    phi = (1 + tanh(s)) / 2 of a sum of random low Fourier modes; with ``pairs`` the box also
    holds two droplets close enough for their interfaces to face each other.
    """
    rng = np.random.default_rng(seed)
    x, y, z = _coords(cfg)
    nx, ny, nz = cfg["nx"], cfg["ny"], cfg["nz"]
    s = np.zeros(x.size)
    for _ in range(n_modes):
        kx, ky = rng.integers(-2, 3, size=2)
        kz = rng.integers(-2, 3) if cfg["dim"] == 3 else 0
        ph = rng.uniform(0, 2 * np.pi)
        s += rng.normal() * np.cos(2 * np.pi * (kx * x / nx + ky * y / ny + kz * z / nz) + ph)
    phi = 0.5 * (1.0 + np.tanh(1.5 * s))
    if pairs:
        R = max(2.0, min(nx, ny) / 5.0)
        cz = (nz - 1) / 2.0
        centers = [(nx / 2.0 - R - 1.3, ny / 2.0 + 0.3, cz), (nx / 2.0 + R + 1.1, ny / 2.0 - 0.4, cz)]
        pd, _ = droplet_fields(cfg, centers, [R, R], [(0, 0, 0), (0, 0, 0)])
        m = pd > 0.02
        phi = np.where(m, pd, phi)
    u = np.zeros((3, x.size))
    dims = 3 if cfg["dim"] == 3 else 2
    for a in range(dims):
        for _ in range(2):
            kx, ky = rng.integers(-2, 3, size=2)
            kz = rng.integers(-2, 3) if cfg["dim"] == 3 else 0
            ph = rng.uniform(0, 2 * np.pi)
            u[a] += amp_u / 2 * rng.normal() * np.cos(
                2 * np.pi * (kx * x / nx + ky * y / ny + kz * z / nz) + ph)
    return phi, u


def noise(shape, seed, scale=1.0):
    """Seeded standard-normal noise (used to push populations off equilibrium in tests)."""
    return scale * np.random.default_rng(seed).standard_normal(shape)
