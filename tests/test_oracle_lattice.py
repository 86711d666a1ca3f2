"""Pins of the oracle's lattice tables, equilibrium, Guo source and regularization against
textbook lattice identities and the moment algebra of Sec. 2.1 (Eqs. 11-17)."""
import itertools

import numpy as np
import pytest

CS2 = 1.0 / 3.0
LATTICES = [(2, 9), (3, 19), (3, 27)]


def _moment(f, c, idx):
    m = np.ones(len(f))
    for a in idx:
        m = m * c[:, a]
    return float(np.sum(f * m))


@pytest.mark.parametrize("dim,Q", LATTICES)
def test_lattice_isotropy(orc, dim, Q):
    c, w = orc.lattice(dim, Q)
    assert abs(w.sum() - 1.0) < 1e-15
    # ordering rule: |c|^2 ascending, then (cz, cy, cx) lexicographic
    keys = [(int(v @ v), int(v[2]), int(v[1]), int(v[0])) for v in c]
    assert keys == sorted(keys)
    assert len(set(map(tuple, c.tolist()))) == Q
    # every velocity has its opposite
    s = set(map(tuple, c.tolist()))
    assert all(tuple((-v).tolist()) in s for v in c)
    d = range(dim)
    for a in d:
        assert abs(_moment(w, c, [a])) < 1e-15
        for b in d:
            assert abs(_moment(w, c, [a, b]) - CS2 * (a == b)) < 1e-15
            for e in d:
                assert abs(_moment(w, c, [a, b, e])) < 1e-15
                for g in d:
                    iso = CS2 ** 2 * ((a == b) * (e == g) + (a == e) * (b == g) + (a == g) * (b == e))
                    assert abs(_moment(w, c, [a, b, e, g]) - iso) < 1e-15


def _supported_third(dim, Q):
    """Third-order moments c_a c_b c_c that the lattice represents (no component cubed, and for
    D3Q19 no xyz product)."""
    out = []
    for idx in itertools.combinations_with_replacement(range(dim), 3):
        if any(idx.count(a) == 3 for a in range(dim)):
            continue
        if len(set(idx)) == 3 and Q == 19:
            continue
        out.append(idx)
    return out


def _d3q19_alias(Q, idx, T):
    """D3Q19 has no (+-1,+-1,+-1) velocities, so its Hermite polynomials H3_aae and H3_ekk
    (k the third axis) are not orthogonal: sum_i w_i H3_aae H3_ekk = -cs^6 while
    sum_i w_i H3_aae^2 = 2 cs^6. A third-order Hermite term sum T_def H3_def / (6 cs^6) therefore
    returns, for the moment c_a c_a c_e, T_aae - T_ekk / 2. On D2Q9 and D3Q27 the alias is 0."""
    if Q != 19:
        return 0.0
    a = next(i for i in idx if idx.count(i) == 2)  # the repeated index
    e = next(i for i in idx if idx.count(i) == 1)
    k = 3 - a - e
    return -0.5 * T(e, k, k)


@pytest.mark.parametrize("dim,Q", LATTICES)
def test_equilibrium_moments(orc, dim, Q):
    """Eq. 11: sum f = p*, sum f c = u, sum f cc = p* cs2 I + uu and the third moment
    cs2 (u d + u d + u d) + uuu (pins the three-permutation reading of Eq. 13)."""
    c, _ = orc.lattice(dim, Q)
    rng = np.random.default_rng(1)
    for _ in range(5):
        u = np.zeros(3)
        u[:dim] = rng.uniform(-0.1, 0.1, dim)
        ps = rng.uniform(-0.05, 0.05)
        f = orc.feq(dim, Q, ps, u)
        assert abs(f.sum() - ps) < 1e-15
        for a in range(dim):
            assert abs(_moment(f, c, [a]) - u[a]) < 1e-15
            for b in range(dim):
                assert abs(_moment(f, c, [a, b]) - (ps * CS2 * (a == b) + u[a] * u[b])) < 1e-15
        for (a, b, e) in _supported_third(dim, Q):
            ref = CS2 * (u[a] * (b == e) + u[b] * (a == e) + u[e] * (a == b)) + u[a] * u[b] * u[e]
            ref += _d3q19_alias(Q, (a, b, e), lambda i, j, k: u[i] * u[j] * u[k])
            assert abs(_moment(f, c, [a, b, e]) - ref) < 1e-15


@pytest.mark.parametrize("dim,Q", LATTICES)
def test_guo_source_moments(orc, dim, Q):
    """Eq. 17: sum S = 0, sum S c = F/rho, sum S cc = u F' + F' u."""
    c, _ = orc.lattice(dim, Q)
    rng = np.random.default_rng(2)
    u = np.zeros(3)
    Fr = np.zeros(3)
    u[:dim] = rng.uniform(-0.1, 0.1, dim)
    Fr[:dim] = rng.uniform(-1e-3, 1e-3, dim)
    S = orc.guo(dim, Q, u, Fr)
    assert abs(S.sum()) < 1e-17
    for a in range(dim):
        assert abs(_moment(S, c, [a]) - Fr[a]) < 1e-17
        for b in range(dim):
            assert abs(_moment(S, c, [a, b]) - (u[a] * Fr[b] + u[b] * Fr[a])) < 1e-17


@pytest.mark.parametrize("dim,Q", LATTICES)
def test_regularized_projection(orc, dim, Q):
    """Eq. 14 is a Hermite projection: zeroth and first moments vanish, the second moment returns
    A2 and the supported third moments return A3 = u A2 + u A2 + u A2 (Eq. 16)."""
    c, _ = orc.lattice(dim, Q)
    rng = np.random.default_rng(3)
    u = np.zeros(3)
    u[:dim] = rng.uniform(-0.1, 0.1, dim)
    A2 = np.zeros((3, 3))
    M = rng.uniform(-1e-3, 1e-3, (dim, dim))
    A2[:dim, :dim] = M + M.T
    R = orc.regularized(dim, Q, u, A2)
    assert abs(R.sum()) < 1e-17
    for a in range(dim):
        assert abs(_moment(R, c, [a])) < 1e-17
        for b in range(dim):
            assert abs(_moment(R, c, [a, b]) - A2[a, b]) < 1e-16
    A3 = lambda i, j, k: u[i] * A2[j, k] + u[j] * A2[i, k] + u[k] * A2[i, j]
    for (a, b, e) in _supported_third(dim, Q):
        ref = A3(a, b, e) + _d3q19_alias(Q, (a, b, e), A3)
        assert abs(_moment(R, c, [a, b, e]) - ref) < 1e-16


def test_ghost_mode_removed_by_regularization(orc):
    """A population perturbation orthogonal to all Hermite moments up to third order (the
    fourth-order xxyy mode) is removed by the regularized collision: f_post = f_eq exactly,
    whereas a plain BGK collision would keep (1 - omega) of it."""
    from paper_2603_17481_gb300 import workloads as W
    dim, Q = 2, 9
    c, w = orc.lattice(dim, Q)
    cfg = W.base_config(2, 8, 8, 1, 9, nci_on=0)
    P = orc.make_params(cfg)
    u = np.array([0.03, -0.02, 0.0])
    ps = 0.004
    feq = orc.feq(dim, Q, ps, u)
    ghost = w * (c[:, 0] ** 2 - CS2) * (c[:, 1] ** 2 - CS2)
    f = feq + 0.01 * ghost
    fpost, uo, pso = orc.hydro_cell(P, f, 1.0, np.zeros(3), 0.0)
    assert np.max(np.abs(fpost - feq)) < 1e-16
    assert np.max(np.abs(uo - u)) < 1e-16
    assert abs(pso - ps) < 1e-16
