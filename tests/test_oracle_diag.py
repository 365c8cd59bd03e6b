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


# ---- free energy (Eq. fren, phi part, on the lattice) ---------------------
def _random_state(d, walls, seed):
    from oracle import oracle as O

    shp = dict(nx=9, ny=8, nz=7) if d == 3 else dict(nx=11, ny=8)
    cfg = O.make_cfg(d=d, walls=walls, b=0.7, kappa=-0.3, c=0.4, Tc=1.0, **shp)
    rng = np.random.default_rng(seed)
    st = O.init(cfg)
    st.phi = 0.3 * rng.standard_normal(st.phi.shape)
    st.T = 0.5 + rng.random(st.T.shape)
    return O, cfg, st


import pytest  # noqa: E402


@pytest.mark.parametrize("d,walls", [(2, 1), (2, 0), (3, 1)])
def test_free_energy_derivative_is_oracle_mu(d, walls):
    """Eq. chem is the variational derivative of Eq. fren: the central finite
    difference of free_energy in phi at single sites (wall layers, corners and
    the bulk) equals the oracle's mu there.  The energy is a quartic in phi(r),
    so the O(h^2) error of the difference is 2 b phi h^2 at most."""
    O, cfg, st = _random_state(d, walls, 4)
    mu = O.aux(st)["mu"]
    fe = lambda p: D.free_energy(p, st.T, bool(walls), cfg.b, cfg.kappa, cfg.c, cfg.Tc)
    h = 1e-4
    shape = st.phi.shape
    picks = [tuple(0 for _ in shape), tuple(n - 1 for n in shape), tuple(n // 2 for n in shape),
             (shape[0] - 1,) + tuple(0 for _ in shape[1:]), (0,) + tuple(n - 1 for n in shape[1:])]
    for idx in picks:
        p1, p2 = st.phi.copy(), st.phi.copy()
        p1[idx] += h
        p2[idx] -= h
        num = (fe(p1) - fe(p2)) / (2 * h)
        assert abs(num - mu[idx]) < 1e-7 * max(1.0, abs(mu[idx])), (idx, num, mu[idx])


def test_free_energy_single_mode_periodic():
    """phi = A cos(q x), q = 2 pi m / L, uniform a on a periodic box: with
    lambda = 4 sin^2(q/2) (the 5-point symbol), the lattice sums are
    N [a A^2/4 + 3 b A^4/32 + kappa lambda A^2/4 + c lambda^2 A^2/4]
    (mean cos^2 = 1/2, mean cos^4 = 3/8, a link difference is
    -2 A sin(q/2) sin(q x + q/2))."""
    ny, nx, m, A = 6, 40, 3, 0.37
    b, kappa, c, Tc, T = 0.9, -0.21, 0.33, 1.0, 0.55
    a = (T - Tc) / Tc
    q = 2 * np.pi * m / nx
    lam = 4 * np.sin(q / 2) ** 2
    phi = A * np.cos(q * np.arange(nx))[None, :] * np.ones((ny, 1))
    N = nx * ny
    want = N * (a * A ** 2 / 4 + 3 * b * A ** 4 / 32 + kappa * lam * A ** 2 / 4 + c * lam ** 2 * A ** 2 / 4)
    got = D.free_energy(phi, np.full_like(phi, T), False, b, kappa, c, Tc)
    assert abs(got - want) < 1e-12 * N


def test_free_energy_half_sample_cosine_between_walls():
    """phi = A cos(pi m (y + 1/2) / L) between walls (even about both halfway
    walls): the mirrored 5-point Laplacian has the eigenvalue
    lambda = 4 sin^2(pi m / 2L), and the L - 1 links along y carry
    sum (dphi)^2 = A^2 lambda L / 2 per column, so the energy is
    nx [a A^2 L/4 + 3 b A^4 L/32 + kappa lambda A^2 L/4 + c lambda^2 A^2 L/4]."""
    L, nx, m, A = 24, 5, 5, 0.41
    b, kappa, c, Tc, T = 1.3, -0.11, 0.27, 1.0, 0.8
    a = (T - Tc) / Tc
    lam = 4 * np.sin(np.pi * m / (2 * L)) ** 2
    phi = A * np.cos(np.pi * m * (np.arange(L) + 0.5) / L)[:, None] * np.ones((1, nx))
    want = nx * L * (a * A ** 2 / 4 + 3 * b * A ** 4 / 32 + kappa * lam * A ** 2 / 4 + c * lam ** 2 * A ** 2 / 4)
    got = D.free_energy(phi, np.full_like(phi, T), True, b, kappa, c, Tc)
    assert abs(got - want) < 1e-12 * nx * L
