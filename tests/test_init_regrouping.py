"""The initial equilibrium as the GPU evaluates it: Eq. 11's third-order polynomial regrouped over each
direction pair (c, -c) into an even and an odd part,
    f_eq(+-c) / w = E +- O,  E = p* - 1.5 |u|^2 + 4.5 (c.u)^2,  O = (c.u) (3 - 4.5 |u|^2 + 4.5 (c.u)^2),
evaluated in FP32. Checked on the host against the oracle's FP64 equilibrium (orc_feq): the regrouping
in FP64 agrees to rounding, and the FP32 sequence of operations (each FMA rounded once) stays within
the bound the GPU test asserts, 8 FP32 units of the scale of the polynomial's terms. Test
infrastructure: the kernel's sequence is restated here in numpy, not imported from the CUDA path."""
import numpy as np
import pytest

import oracle as O

F32 = np.float32


def _fma(a, b, c):
    """a b + c rounded once to FP32 (the product of two FP32 values is exact in FP64)."""
    return F32(np.float64(a) * np.float64(b) + np.float64(c))


def _pairs(c):
    """(i, opposite of i) for every direction pair, i the lower index."""
    out = []
    for i in range(1, len(c)):
        j = int(np.where((c == -c[i]).all(axis=1))[0][0])
        if i < j:
            out.append((i, j))
    return out


def _regrouped(c, ps, u, dtype):
    """f_eq / w per direction from the even / odd split, every operation in dtype."""
    if dtype == np.float64:
        uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2]
        A, B = ps - 1.5 * uu, 3.0 - 4.5 * uu
    else:
        u = u.astype(F32)
        uu = _fma(u[0], u[0], _fma(u[1], u[1], u[2] * u[2]))
        A, B = _fma(F32(-1.5), uu, ps.astype(F32)), _fma(F32(-4.5), uu, F32(3.0))
    g = np.zeros((len(c), u.shape[1]), dtype=dtype)
    g[0] = A
    for i, j in _pairs(c):
        cu = np.zeros(u.shape[1], dtype=dtype)
        for a in range(3):  # signed sums of the components, in the kernel's order
            if c[i, a] > 0:
                cu = cu + u[a]
            elif c[i, a] < 0:
                cu = cu - u[a]
        s = cu * cu
        if dtype == np.float64:
            E, Od = A + 4.5 * s, cu * (B + 4.5 * s)
        else:
            E, Od = _fma(F32(4.5), s, A), cu * _fma(F32(4.5), s, B)
        g[i], g[j] = E + Od, E - Od
    return g


@pytest.fixture(scope="module")
def orc():
    O.build()
    return O


@pytest.mark.parametrize("dim,Q", [(2, 9), (3, 19), (3, 27)])
def test_regrouped_equilibrium_matches_the_oracle(orc, dim, Q):
    rng = np.random.default_rng(17481 + Q)
    n = 400
    u = rng.uniform(-0.12, 0.12, size=(3, n))
    if dim == 2:
        u[2] = 0.0
    ps = rng.normal(0.0, 5e-3, size=n)
    c, w = orc.lattice(dim, Q)
    c = np.asarray(c, dtype=np.int64)
    ref = np.stack([orc.feq(dim, Q, ps[k], u[:, k]) for k in range(n)], axis=1) / w[:, None]
    g64 = _regrouped(c, ps, u, np.float64)
    assert np.max(np.abs(g64 - ref)) < 1e-15  # the regrouping is Eq. 11, term for term
    g32 = _regrouped(c, ps, u, F32).astype(np.float64)
    g32 = (w[:, None].astype(F32) * g32.astype(F32)).astype(np.float64) / w[:, None]  # FP32 store of f
    cabs = np.abs(c).astype(np.float64) @ np.abs(u)
    scale = np.abs(ps)[None, :] + 3.0 * cabs + 4.5 * cabs ** 2 + 1.5 * np.sum(u * u, axis=0)[None, :] + 1e-3
    err = np.max(np.abs(g32 - ref) / scale)
    assert err <= 8 * 2.0 ** -24, f"{err / 2.0 ** -24:.2f} FP32 units"
    # the bound is tight enough to catch a dropped cubic term or a swapped pair
    cu = c.astype(np.float64) @ u
    assert np.max(4.5 * np.abs(cu) ** 3 / scale) > 1e3 * 8 * 2.0 ** -24
    i, j = _pairs(c)[0]
    swapped = g32.copy()
    swapped[[i, j]] = swapped[[j, i]]
    assert np.max(np.abs(swapped - ref) / scale) > 1e3 * 8 * 2.0 ** -24
