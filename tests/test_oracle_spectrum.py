"""Pins of the oracle's carrier-phase energy spectrum (Sec. 3.4): Parseval's identity, a single
Fourier mode that puts all its energy in one shell, and the exclusion of the gas phase."""
import numpy as np

import oracle as O
from paper_2603_17481_gb300 import workloads as W


def test_single_mode_lands_in_its_shell(orc):
    cfg = W.base_config(3, 32, 32, 32, 19)
    P = O.make_params(cfg)
    n = np.arange(32 ** 3)
    x, y, z = n % 32, (n // 32) % 32, n // 1024
    A = 0.01
    u = np.zeros((3, n.size))
    u[0] = A * np.cos(2 * np.pi * (3 * y + 4 * z) / 32)  # |m| = 5
    E = O.energy_spectrum(P, np.ones(n.size), u, 20)
    assert abs(E[5] - A * A / 4) < 1e-15 and abs(E.sum() - A * A / 4) < 1e-15


def test_parseval_with_gas_excluded(orc):
    cfg = W.base_config(3, 24, 20, 16, 19)
    P = O.make_params(cfg)
    rng = np.random.default_rng(3)
    N = 24 * 20 * 16
    u = rng.standard_normal((3, N)) * 0.01
    phi, _ = W.droplet_fields(cfg, [(11.3, 9.8, 7.6)], [5.0], [(0, 0, 0)], bubbles=True)
    E = O.energy_spectrum(P, phi, u, 64)  # every shell of this box is below 64
    chi = phi >= 0.5
    assert 0 < (~chi).sum() < N
    up = np.where(chi, u - u[:, chi].mean(axis=1, keepdims=True), 0.0)
    assert abs(E.sum() - 0.5 * (up ** 2).sum() / N) < 1e-12 * E.sum()
    # the gas velocity does not enter
    u2 = u.copy()
    u2[:, ~chi] = 5.0
    assert np.allclose(O.energy_spectrum(P, phi, u2, 64), E, rtol=1e-12, atol=0)
