"""Pins of the oracle's isotropic stencils (Eqs. 22-23) and phase-field update (Eq. 28 with
Eqs. 29-35) against closed forms, invariants and the tanh equilibrium of Eq. 43."""
import numpy as np
import pytest

from paper_2603_17481_gb300 import workloads as W


def _grid(cfg):
    nx, ny, nz = cfg["nx"], cfg["ny"], cfg["nz"]
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    return x.ravel().astype(float), y.ravel().astype(float), z.ravel().astype(float)


@pytest.mark.parametrize("dim", [2, 3])
def test_iso_gradient_laplacian_plane_wave(orc, dim):
    """Plane wave cos(k x): the isotropic gradient is exactly -sin(k) sin(kx) and the isotropic
    Laplacian exactly 2 (cos k - 1) cos(kx), because the weights with c_x = +-1 add up to
    cs^2 / 2 on each side (second-moment identity), in 2D (D2Q9) and 3D (D3Q27)."""
    for n in (8, 16):
        _plane_wave(orc, dim, n)


def _plane_wave(orc, dim, n):
    cfg = W.base_config(dim, n, 8, 8 if dim == 3 else 1, 9 if dim == 2 else 19)
    P = orc.make_params(cfg)
    for axis in range(dim):
        x, y, z = _grid(cfg)
        coord = (x, y, z)[axis]
        L = (cfg["nx"], cfg["ny"], cfg["nz"])[axis]
        k = 2 * np.pi * 2 / L
        psi = np.cos(k * coord)
        g = orc.grad_iso(P, psi)
        lap = orc.lap_iso(P, psi)
        ref = np.zeros_like(g)
        ref[axis] = -np.sin(k) * np.sin(k * coord)
        assert np.max(np.abs(g - ref)) < 1e-14
        assert np.max(np.abs(lap - 2 * (np.cos(k) - 1) * psi)) < 1e-14


@pytest.mark.parametrize("dim", [2, 3])
def test_iso_stencils_exact_on_polynomials(orc, dim):
    """Away from the periodic seam the gradient is exact on linear fields and the Laplacian is
    exact on quadratics (2 per unit squared coordinate, 0 for mixed terms)."""
    n = 12
    cfg = W.base_config(dim, n, n, n if dim == 3 else 1, 9 if dim == 2 else 19)
    P = orc.make_params(cfg)
    x, y, z = _grid(cfg)
    interior = (x > 0) & (x < n - 1) & (y > 0) & (y < n - 1)
    if dim == 3:
        interior &= (z > 0) & (z < n - 1)
    lin = 0.3 + 0.7 * x - 1.1 * y + (0.5 * z if dim == 3 else 0)
    g = orc.grad_iso(P, lin)
    assert np.max(np.abs(g[0][interior] - 0.7)) < 1e-13
    assert np.max(np.abs(g[1][interior] + 1.1)) < 1e-13
    if dim == 3:
        assert np.max(np.abs(g[2][interior] - 0.5)) < 1e-13
    quad = x * x + 0.5 * y * y - 0.3 * x * y + (2.0 * z * z + 0.2 * y * z if dim == 3 else 0)
    lap = orc.lap_iso(P, quad)
    ref = 2.0 + 1.0 + (4.0 if dim == 3 else 0.0)
    assert np.max(np.abs(lap[interior] - ref)) < 1e-11


def test_minmod_truth_table(orc):
    """Eq. 32."""
    cases = [((1.0, 2.0), 1.0), ((2.0, 1.0), 1.0), ((-1.0, -2.0), -1.0), ((-3.0, -0.5), -0.5),
             ((1.0, -1.0), 0.0), ((0.0, 5.0), 0.0), ((-2.0, 0.0), 0.0), ((0.25, 0.25), 0.25)]
    for (a, b), r in cases:
        assert orc.minmod(a, b) == r


def _line_cfg(n, **kw):
    base = dict(nci_on=0, D=0.0)
    base.update(kw)
    return W.base_config(2, n, 4, 1, 9, **base)


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_muscl_linear_ramp_is_translated_exactly(orc, axis):
    """MUSCL-minmod (Eqs. 29-34) reconstructs a linear profile exactly, so with a uniform
    velocity u and D = 0 (kappa = 0) the interior of a ramp of slope s moves by exactly -u s,
    along each axis of a 3D box (the other velocity components are set to distractor values
    that must not enter this axis's fluxes)."""
    shape = [8, 8, 8]
    shape[axis] = 40
    cfg = W.base_config(3, *shape, 19, nci_on=0, D=0.0)
    P = orc.make_params(cfg)
    coord = _grid(cfg)[axis]
    phi = 0.1 + 0.02 * coord
    for uval in (0.3, -0.45):
        u = np.full((3, phi.size), 0.2)
        u[axis] = uval
        out = orc.phi_update(P, phi, u)
        inner = (coord >= 3) & (coord <= 36)
        assert np.max(np.abs(out[inner] - (phi[inner] - uval * 0.02))) < 1e-15


def test_muscl_step_is_first_order_upwind(orc):
    """At a step the minmod slopes vanish, so the face value is the upwind cell value
    (Eq. 34: u >= 0 takes the left state): a unit step moving right with u = 0.5 fills the first
    downstream cell to 0.5 and empties the last upstream cell to 0.5 at the trailing edge."""
    n = 32
    cfg = _line_cfg(n)
    P = orc.make_params(cfg)
    x, _, _ = _grid(cfg)
    phi = ((x >= 8) & (x < 20)).astype(float)
    u = np.zeros((3, phi.size))
    u[0] = 0.5
    out = orc.phi_update(P, phi, u).reshape(4, n)[0]
    ref = ((np.arange(n) >= 8) & (np.arange(n) < 20)).astype(float)
    ref[8] = 0.5
    ref[20] = 0.5
    assert np.max(np.abs(out - ref)) < 1e-15
    u[0] = -0.5
    out = orc.phi_update(P, phi, u).reshape(4, n)[0]
    ref = ((np.arange(n) >= 8) & (np.arange(n) < 20)).astype(float)
    ref[7] = 0.5
    ref[19] = 0.5
    assert np.max(np.abs(out - ref)) < 1e-15


def test_face_velocity_is_arithmetic_mean(orc):
    """For phi = 1 the flux difference is u_{i+1/2} - u_{i-1/2} = (u_{i+1} - u_{i-1}) / 2."""
    n = 24
    cfg = _line_cfg(n)
    P = orc.make_params(cfg)
    x, _, _ = _grid(cfg)
    phi = np.ones_like(x)
    u = np.zeros((3, x.size))
    u[0] = 0.05 * np.sin(2 * np.pi * x / n)
    out = orc.phi_update(P, phi, u)
    ref = 1.0 - 0.5 * (0.05 * np.sin(2 * np.pi * (x + 1) / n) - 0.05 * np.sin(2 * np.pi * (x - 1) / n))
    assert np.max(np.abs(out - ref)) < 1e-15


def test_diffusion_of_cosine(orc):
    """With u = 0 and a negligible compression (eps huge, kappa = 4D/eps -> 0), one update
    multiplies cos(kx) by 1 + 2 D (cos k - 1) (isotropic Laplacian, tau_diff = D)."""
    n = 32
    D = 0.1
    cfg = _line_cfg(n, D=D, eps=1e30)
    P = orc.make_params(cfg)
    x, _, _ = _grid(cfg)
    k = 2 * np.pi * 3 / n
    phi = 0.5 + 0.3 * np.cos(k * x)
    out = orc.phi_update(P, phi, np.zeros((3, x.size)))
    ref = 0.5 + 0.3 * np.cos(k * x) * (1 + 2 * D * (np.cos(k) - 1))
    assert np.max(np.abs(out - ref)) < 1e-15


def _slab(cfg, eps_prof, x):
    n = cfg["nx"]
    sd = np.minimum(x - (n / 4 - 0.5), (3 * n / 4 - 0.5) - x)
    return 0.5 * (1 + np.tanh(2 * sd / eps_prof))


def test_compression_sharpens_a_wide_interface(orc):
    """The compressive term (Eq. 35, kappa = 4D/eps) steepens a profile wider than eps: after
    200 updates of a width-8 tanh slab with eps = 4 the maximum slope grows toward the
    equilibrium slope 1/eps, and the mass is unchanged."""
    n = 64
    cfg = _line_cfg(n, D=0.1, eps=4.0)
    P = orc.make_params(cfg)
    x, _, _ = _grid(cfg)
    phi = _slab(cfg, 8.0, x)
    u = np.zeros((3, x.size))
    ph = phi.copy()
    for _ in range(200):
        ph = orc.phi_update(P, ph, u)
    s0 = np.max(np.abs(np.diff(phi.reshape(4, n)[0])))
    s1 = np.max(np.abs(np.diff(ph.reshape(4, n)[0])))
    assert s0 < 0.13 and s1 > 0.2
    assert abs(ph.sum() - phi.sum()) < 1e-12 * phi.sum()


@pytest.mark.parametrize("eps", [4.0, 8.0])
def test_flat_interface_tanh_equilibrium(orc, eps):
    """The tanh profile of Eq. 43 is the continuum equilibrium of Eq. 24 with kappa = 4D/eps
    (D phi' = kappa phi (1 - phi)). On the lattice it stays close to it; the deviation after 1000
    updates is below 6e-3 at eps = 4 and shrinks about fourfold at eps = 8 (O(eps^-2) error)."""
    n = 32 * int(eps / 4)
    cfg = _line_cfg(n, D=0.1, eps=eps)
    P = orc.make_params(cfg)
    x, _, _ = _grid(cfg)
    phi = _slab(cfg, eps, x)
    u = np.zeros((3, x.size))
    ph = phi.copy()
    for _ in range(1000):
        ph = orc.phi_update(P, ph, u)
    dev = np.max(np.abs(ph - phi))
    assert dev < (6e-3 if eps == 4.0 else 2e-3)
    assert abs(ph.sum() - phi.sum()) < 1e-12 * phi.sum()


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_flat_interface_3d_each_axis(orc, axis):
    """The flat-interface equilibrium in 3D (D3Q27 compressive divergence and Laplacian) along
    each axis: deviation after 500 updates below 6e-3 and the same for every axis."""
    shape = [4, 4, 4]
    shape[axis] = 32
    cfg = W.base_config(3, *shape, 19, nci_on=0, D=0.1)
    P = orc.make_params(cfg)
    coord = _grid(cfg)[axis]
    sd = np.minimum(coord - 7.5, 23.5 - coord)
    phi = 0.5 * (1 + np.tanh(2 * sd / 4.0))
    ph = phi.copy()
    u = np.zeros((3, phi.size))
    for _ in range(500):
        ph = orc.phi_update(P, ph, u)
    dev = np.max(np.abs(ph - phi))
    assert 1e-4 < dev < 6e-3
    assert abs(ph.sum() - phi.sum()) < 1e-12 * phi.sum()


@pytest.mark.parametrize("dim", [2, 3])
def test_phase_update_conserves_mass(orc, dim):
    """Eq. 29 is a flux difference and the isotropic Laplacian and divergence sum to zero over a
    periodic box: sum(phi) is invariant for any phi and u (to FP64 round-off)."""
    cfg = W.base_config(dim, 20, 14, 10 if dim == 3 else 1, 9 if dim == 2 else 19)
    P = orc.make_params(cfg)
    phi, u = W.smooth_random_fields(cfg, seed=7, amp_u=0.1)
    ph = phi.copy()
    for _ in range(50):
        ph = orc.phi_update(P, ph, u)
    assert abs(ph.sum() - phi.sum()) < 1e-12 * phi.sum()
    assert np.max(np.abs(ph - phi)) > 1e-3  # something did move
