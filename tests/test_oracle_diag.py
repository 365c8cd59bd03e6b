"""Pins of the oracle's diagnostics definitions on fields with known answers."""
import numpy as np

from oracle import diag as D


def test_structure_factor_single_mode():
    ny, nx, m = 64, 64, 8
    x = np.arange(nx)
    phi = 0.3 * np.cos(2 * np.pi * m * x / nx)[None, :] * np.ones((ny, 1))
    kb, Sb, k_peak, S_peak = D.structure_factor(phi)
    dk = 2 * np.pi / 64
    assert abs(k_peak - m * dk) < 1e-12
    # two modes (+-k) of |FFT|^2 = (0.3 N / 2)^2 each, divided by N, averaged over the shell
    shell = np.floor(np.sqrt(np.add.outer(np.fft.fftfreq(ny) ** 2, np.fft.fftfreq(nx) ** 2)) * nx + 0.5)
    count = int((shell == m).sum())
    N = nx * ny
    assert abs(S_peak - 2 * (0.3 * N / 2) ** 2 / N / count) < 1e-9


def test_orientation_limits():
    ny, nx = 32, 48
    y, x = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    par = np.cos(2 * np.pi * 4 * (y + 0.5) / ny)     # layers parallel to the walls
    perp = np.cos(2 * np.pi * 6 * x / nx)            # layers perpendicular to the walls
    assert abs(D.orientation(par, True)[0] - 1.0) < 1e-12
    assert abs(D.orientation(perp, True)[0] + 1.0) < 1e-12
    s3 = D.orientation(np.cos(2 * np.pi * 2 * np.arange(16) / 16)[:, None, None] * np.ones((16, 8, 8)), False)[0]
    assert abs(s3 - 1.0) < 1e-12
    s_lay = D.orientation(perp, True)[1]
    assert np.allclose(s_lay, -1.0)
