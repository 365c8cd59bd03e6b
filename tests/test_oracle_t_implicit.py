"""Pins of the implicit temperature reference (oracle/t_implicit.py) against
closed forms and limits that fix it independently of its own matrix."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from oracle import t_implicit as TI


def _lam(k, n):
    return 2.0 * (1.0 - math.cos(2.0 * math.pi * k / n))


def test_periodic_fourier_mode_is_divided_by_one_plus_xi_lambda():
    # a lattice Fourier mode of the periodic 5-point Laplacian: eigenvalue -(lam_x + lam_y)
    ny, nx, xi = 6, 8, 0.7
    y, x = np.mgrid[0:ny, 0:nx]
    T = np.cos(2 * math.pi * 3 * x / nx) * np.cos(2 * math.pi * 1 * y / ny)
    out = TI.implicit_step(T, xi, 0.0, walls=0, t_mode=0)
    np.testing.assert_allclose(out, T / (1 + xi * (_lam(3, nx) + _lam(1, ny))), atol=1e-12)


def test_periodic_3d_mode():
    nz, ny, nx, xi = 5, 4, 6, 2.5
    z, y, x = np.mgrid[0:nz, 0:ny, 0:nx]
    T = np.sin(2 * math.pi * 2 * x / nx) * np.cos(2 * math.pi * 1 * z / nz) + 0.3
    out = TI.implicit_step(T, xi, 0.0, walls=0, t_mode=0)
    want = 0.3 + (T - 0.3) / (1 + xi * (_lam(2, nx) + _lam(1, nz)))
    np.testing.assert_allclose(out, want, atol=1e-12)


def test_layers_mode_sine_profile_along_the_wall_normal():
    # Dirichlet rows 0 and L-1 at T_w; the interior deviation sin(pi m j / (L-1))
    # is an eigenvector of the interior second difference with eigenvalue
    # 2 (1 - cos(pi m / (L-1))), uniform along x
    L, nx, xi, Tw = 9, 4, 1.3, 0.5
    j = np.arange(L)[:, None] * np.ones((1, nx))
    m = 2
    T = Tw + 0.2 * np.sin(math.pi * m * j / (L - 1))
    out = TI.implicit_step(T, xi, Tw, walls=1, t_mode=0)
    lam = 2 * (1 - math.cos(math.pi * m / (L - 1)))
    np.testing.assert_allclose(out, Tw + 0.2 * np.sin(math.pi * m * j / (L - 1)) / (1 + xi * lam), atol=1e-12)


def test_halfway_mode_cosine_profile_along_the_wall_normal():
    # ghost 2 T_w - T: the deviation from T_w is odd about the half-way planes,
    # so sin(pi m (j + 1/2) / L) is an eigenvector with 2 (1 - cos(pi m / L))
    L, nx, xi, Tw = 7, 4, 0.9, 0.45
    j = np.arange(L)[:, None] * np.ones((1, nx))
    m = 3
    T = Tw + 0.1 * np.sin(math.pi * m * (j + 0.5) / L)
    out = TI.implicit_step(T, xi, Tw, walls=1, t_mode=1)
    lam = 2 * (1 - math.cos(math.pi * m / L))
    np.testing.assert_allclose(out, Tw + 0.1 * np.sin(math.pi * m * (j + 0.5) / L) / (1 + xi * lam), atol=1e-12)


def test_large_xi_relaxes_to_the_wall_temperature():
    rng = np.random.default_rng(1)
    T = 1.1 + 0.05 * rng.standard_normal((10, 6))
    for mode in (0, 1):
        out = TI.implicit_step(T, 1e12, 0.5, walls=1, t_mode=mode)
        np.testing.assert_allclose(out, 0.5, atol=1e-9)


def test_small_xi_matches_one_explicit_step_to_second_order():
    rng = np.random.default_rng(2)
    T = 1.0 + 0.1 * rng.standard_normal((8, 7))
    Tw = 0.5
    T[0] = T[-1] = Tw
    xi = 1e-4
    out = TI.implicit_step(T, xi, Tw, walls=1, t_mode=0)
    lap = np.zeros_like(T)
    lap[1:-1] = (np.roll(T, 1, 1) + np.roll(T, -1, 1))[1:-1] + T[:-2] + T[2:] - 4 * T[1:-1]
    expl = T + xi * lap
    expl[0] = expl[-1] = Tw
    assert np.abs(out - expl).max() < 50 * xi ** 2


# ---- isotropic 9-/19-point stencil (stencil = 1) ----------------------------
def _iso_lap2(qx, qy):
    # Fourier symbol of [4 (nearest) + (diagonal) - 20 A] / 6
    return (8 * (math.cos(qx) + math.cos(qy)) + 4 * math.cos(qx) * math.cos(qy) - 20) / 6


def _iso_lap3(qx, qy, qz):
    cx, cy, cz = math.cos(qx), math.cos(qy), math.cos(qz)
    return (4 * (cx + cy + cz) + 4 * (cx * cy + cx * cz + cy * cz) - 24) / 6


def test_iso_periodic_modes_are_divided_by_one_minus_xi_symbol():
    ny, nx, xi = 6, 8, 0.7
    y, x = np.mgrid[0:ny, 0:nx]
    T = np.cos(2 * math.pi * 3 * x / nx + 2 * math.pi * 1 * y / ny)
    out = TI.implicit_step(T, xi, 0.0, walls=0, t_mode=0, stencil=1)
    np.testing.assert_allclose(out, T / (1 - xi * _iso_lap2(2 * math.pi * 3 / nx, 2 * math.pi / ny)), atol=1e-12)
    nz, ny, nx, xi = 5, 4, 6, 2.5
    z, y, x = np.mgrid[0:nz, 0:ny, 0:nx]
    T = np.sin(2 * math.pi * (2 * x / nx + y / ny - z / nz)) + 0.3
    out = TI.implicit_step(T, xi, 0.0, walls=0, t_mode=0, stencil=1)
    lam = _iso_lap3(2 * math.pi * 2 / nx, 2 * math.pi / ny, -2 * math.pi / nz)
    np.testing.assert_allclose(out, 0.3 + (T - 0.3) / (1 - xi * lam), atol=1e-12)


@pytest.mark.parametrize("t_mode", [0, 1])
def test_iso_wall_modes_with_diagonal_ghosts(t_mode):
    """T - T_w = eps cos(kx x) s(j), s the Dirichlet eigenvector of the wall rule:
    the x dependence makes the diagonal neighbours (and their ghosts) count, and
    the mode is divided by 1 - xi Lambda(kx, q) with Lambda the 9-point symbol."""
    L, nx, xi, Tw = 9, 6, 1.3, 0.5
    j = np.arange(L)[:, None]
    x = np.arange(nx)[None, :]
    kx, m = 2 * math.pi * 2 / nx, 3
    q = math.pi * m / (L - 1) if t_mode == 0 else math.pi * m / L
    s = np.sin(q * j) if t_mode == 0 else np.sin(q * (j + 0.5))
    dev = 0.2 * np.cos(kx * x) * s
    out = TI.implicit_step(Tw + dev, xi, Tw, walls=1, t_mode=t_mode, stencil=1)
    np.testing.assert_allclose(out, Tw + dev / (1 - xi * _iso_lap2(kx, q)), atol=1e-12)


@pytest.mark.parametrize("t_mode", [0, 1])
def test_iso_small_xi_matches_one_explicit_oracle_step(t_mode):
    """To first order in xi the implicit step is the oracle's explicit step with
    the same stencil and wall rule (the two differ at O(xi^2))."""
    ny, nx, Tw, xi = 8, 7, 0.5, 1e-4
    cfg = O.make_cfg(nx=nx, ny=ny, walls=1, t_wall_mode=t_mode, hydro=0, phi_amp=0.0, xi=xi, T0=1.0,
                     T_w=Tw, stencil=1)
    assert cfg.nsub == 1
    st = O.init(cfg)
    st.T = 1.0 + 0.1 * np.random.default_rng(3).standard_normal((ny, nx))
    if t_mode == 0:
        st.T[0] = st.T[-1] = Tw
    expl = O.step(st).T
    out = TI.implicit_step(st.T, xi, Tw, walls=1, t_mode=t_mode, stencil=1)
    assert np.abs(out - expl).max() < 50 * xi ** 2
    assert np.abs(out - st.T).max() > 1e3 * xi ** 2          # the step itself is O(xi)
