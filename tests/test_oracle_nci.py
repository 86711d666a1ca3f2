"""Pins of the oracle's near-contact interaction (Sec. 2.2-2.3, Eqs. 36-73) against the
closed-form derivation of the proximity indicator (Eqs. 43-46), a planar thin film whose every
term is known in closed form, the isolated-droplet case and a brute-force partner search."""
import math
import os

import numpy as np
import pytest

from paper_2603_17481_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_paper_parameters_match_print():
    """The workload parameters equal the values printed in Sec. 2.3.2 and Eq. 71."""
    vals = {}
    with open(os.path.join(GOLDEN, "paper_nci_parameters.txt")) as fh:
        for line in fh:
            line = line.split("#")[0].strip()
            if line:
                k, v = line.split()
                vals[k] = float(v)
    for k, v in vals.items():
        assert W.PAPER_NCI[k] == v, k


@pytest.mark.parametrize("s", [0.05, 0.3, 0.9, 1.4, 1.76, 2.5])
@pytest.mark.parametrize("eps", [4.0, 6.0])
def test_h_of_q_recovers_twice_the_depth(orc, s, eps):
    """Eqs. 43-46: for a cell at depth s in the tanh profile, q = phi (1 - phi) maps back to
    h = 2 |s| exactly (derivation chain, independent of how arcosh is evaluated)."""
    phi = 0.5 * (1 + math.tanh(2 * s / eps))
    q = phi * (1 - phi)
    assert abs(orc.h_of_q(q, eps) - 2 * s) < 1e-9 * max(1.0, s)


def test_h_of_q_equals_artanh_form(orc):
    """arcosh(1/(2 sqrt q)) = artanh(sqrt(1 - 4q)) for 0 < q < 1/4 (exact identity)."""
    for q in np.linspace(0.01, 0.2499, 40):
        assert abs(orc.h_of_q(q, 4.0) - 4.0 * math.atanh(math.sqrt(1 - 4 * q))) < 1e-12


def test_w_h_values(orc):
    """Eq. 42 / Eq. 71 with h0 = 1, p = 4: w(0) = 1, w(1) = 1/2, w(2) = 1/17."""
    assert orc.w_h(0.0) == 1.0
    assert abs(orc.w_h(1.0) - 0.5) < 1e-16
    assert abs(orc.w_h(2.0) - 1.0 / 17.0) < 1e-16
    assert abs(orc.w_h(2.0, h0=2.0, p=2.0) - 0.5) < 1e-16


def _film_cfg(ratio=10.0, decide_f32=0):
    cfg = W.base_config(3, 24, 8, 8, 19, rho_g=1.0 / ratio, decide_f32=decide_f32, eps_n=1e-12)
    return cfg


def _film_phi(cfg, gap):
    """Gas film of gap `gap` (between the two phi = 1/2 levels) centred at x = 11.5, liquid on
    both sides; each side is an exact tanh profile of depth s = |x - 11.5| - gap/2."""
    nx, ny, nz = cfg["nx"], cfg["ny"], cfg["nz"]
    x = np.tile(np.arange(nx, dtype=float), ny * nz)
    d = np.abs(x - 11.5)
    s = d - gap / 2
    phi = 0.5 * (1 + np.tanh(2 * s / cfg["eps"]))
    return phi, x, s


@pytest.mark.parametrize("decide_f32", [0, 1])
def test_planar_film_closed_form(orc, decide_f32):
    """Planar gas film with gap 1: the gated cells (q >= 1/8) are the two cells on each side
    (depths s = 0 and 1); each pairs with its mirror cell straight across the film (offset 1 and
    3: the nearer opposite cells fail the 10 % similarity gate), the normals are exactly
    antiparallel (f_face = 1), q_pair = q(x), h = 2|s| (Eq. 46), and with the orientation toward
    the partner (Sec. 2.3.3) F_rep = +-rho A_rep q w_h(2|s|) along x, zero across. The normals'
    eps_n = 1e-12 floor makes f_face = 1 - O(eps_n / |grad phi|), hence the 1e-9 tolerance."""
    cfg = _film_cfg(decide_f32=decide_f32)
    P = orc.make_params(cfg)
    phi, x, s = _film_phi(cfg, 1.0)
    part, frep, marg = orc.nci(P, phi)
    q = phi * (1 - phi)
    gated = q >= 0.125
    assert set(np.round(np.abs(s[gated]), 12)) == {0.0, 1.0}
    chi = part[:, 0] != orc.NO_PARTNER
    assert np.array_equal(chi, gated)
    left = x < 11.5
    exp_off = np.where(left, 1, -1) * (2 * np.abs(s) + 1).astype(int)
    assert np.array_equal(part[gated, 0], exp_off[gated])
    assert np.all(part[gated, 1:] == 0)
    rho = cfg["rho_g"] + (cfg["rho_l"] - cfg["rho_g"]) * phi
    qcl = np.clip(q, 1e-12, 0.25 - 1e-12)
    wh = 1.0 / (1.0 + (2 * np.abs(s)) ** 4)
    ref = np.where(gated, np.where(left, 1.0, -1.0) * rho * cfg["A_rep"] * qcl * wh, 0.0)
    assert np.max(np.abs(frep[0] - ref)) < 1e-9 * np.max(np.abs(ref))
    assert np.max(np.abs(frep[1:])) == 0.0
    # exact antisymmetry across the film mid-plane
    fx = frep[0].reshape(8, 8, 24)[0]
    assert np.max(np.abs(fx + fx[:, ::-1])) < 1e-15


@pytest.mark.parametrize("dim,R,n", [(2, 16.0, 64), (3, 12.0, 40)])
def test_isolated_droplet_has_no_partner(orc, dim, R, n):
    """An isolated droplet: within the 7-cell window all gated normals lie within a few degrees
    of each other, far from the facing threshold n.n <= -0.8, so chi = 0 and F_rep = 0."""
    cfg = W.base_config(dim, n, n, n if dim == 3 else 1, 9 if dim == 2 else 19)
    P = orc.make_params(cfg)
    c = (n / 2 - 0.3, n / 2 + 0.2, n / 2 - 0.1 if dim == 3 else 0.0)
    phi, _ = W.droplet_fields(cfg, [c], [R], [(0, 0, 0)])
    part, frep, _ = orc.nci(P, phi)
    assert np.all(part[:, 0] == orc.NO_PARTNER)
    assert np.max(np.abs(frep)) == 0.0
    assert np.sum(phi * (1 - phi) >= 0.125) > 100  # the gate itself is active


def _brute_force_partners(orc, P, cfg, phi):
    """Every cell y of the periodic box within Chebyshev distance w (minimum image) is tested
    with the criteria of Eqs. 59-62 and ranked by (|r|^2, -f_face, canonical index)."""
    dim, w = cfg["dim"], cfg["w"]
    nx, ny, nz = cfg["nx"], cfg["ny"], cfg["nz"]
    N = nx * ny * nz
    g = orc.grad_iso(P, phi)
    nrm = g / (np.sqrt((g * g).sum(0)) + cfg["eps_n"])
    pc = np.clip(phi, 0, 1)
    q = pc * (1 - pc)
    idx = np.arange(N)
    X, Y, Z = idx % nx, (idx // nx) % ny, idx // (nx * ny)
    out = np.full((N, 3), orc.NO_PARTNER, dtype=np.int64)
    W_ = 2 * w + 1
    for n in np.nonzero(q >= cfg["q_th"])[0]:
        rx = (X - X[n] + nx // 2) % nx - nx // 2
        ry = (Y - Y[n] + ny // 2) % ny - ny // 2
        rz = (Z - Z[n] + nz // 2) % nz - nz // 2 if dim == 3 else np.zeros(N, int)
        inwin = (np.abs(rx) <= w) & (np.abs(ry) <= w) & (np.abs(rz) <= w) & (idx != n)
        dot = (nrm[:, n:n + 1] * nrm).sum(0)
        ok = inwin & (q >= cfg["q_th"]) & (np.abs(q - q[n]) <= cfg["eta"] * max(q[n], cfg["eps_q"])) \
            & (dot <= cfg["cos_opp"])
        cand = np.nonzero(ok)[0]
        if cand.size == 0:
            continue
        zr = w if dim == 3 else 0
        keys = [(rx[m] ** 2 + ry[m] ** 2 + rz[m] ** 2, -max(0.0, -dot[m]),
                 ((rz[m] + zr) * W_ + ry[m] + w) * W_ + rx[m] + w, m) for m in cand]
        best = min(keys)[3]
        out[n] = (rx[best], ry[best], rz[best])
    return out


@pytest.mark.parametrize("dim,shape,seed", [(2, (23, 17, 1), 5), (2, (8, 8, 1), 2), (3, (8, 8, 8), 4),
                                            (3, (13, 11, 9), 11), (3, (12, 10, 8), 3)])
def test_partner_selection_brute_force(orc, dim, shape, seed):
    """The oracle's window scan (Eq. 60) agrees with a brute-force search over the whole periodic
    box on random fields holding a pair of nearly touching droplets (FP64 decisions)."""
    cfg = W.base_config(dim, *shape, 9 if dim == 2 else 19, decide_f32=0)
    P = orc.make_params(cfg)
    phi, _ = W.smooth_random_fields(cfg, seed=seed)
    part, frep, marg = orc.nci(P, phi)
    ref = _brute_force_partners(orc, P, cfg, phi)
    chi = part[:, 0] != orc.NO_PARTNER
    assert chi.sum() > 5
    assert np.array_equal(part.astype(np.int64), ref)
    # partners beyond the inscribed sphere: the window is the full cube of (2w+1)^d - 1 positions
    # (342 in 3D for w = 3, Sec. 2.3.2), not the ball |r| <= w
    d2 = (part[chi].astype(np.int64) ** 2).sum(1)
    assert d2.max() > cfg["w"] ** 2
