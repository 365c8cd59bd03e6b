"""Pins of the oracle's isotropic stencils (stencil = 1).

With the weights of the velocity set, the first derivative is
d_a A = 3 sum_i w_i e_ia A(r + e_i) and the Laplacian 6 sum_i w_i [A(r + e_i) -
A(r)] (Thampi, Ansumali, Adhikari & Succi, J. Comput. Phys. 234 (2013) 1).
Their Fourier symbols are closed forms; in 2D
  lap:  [8 (cos qx + cos qy) + 4 cos qx cos qy - 20] / 6,
  d_x:  (i/3) sin qx (2 + cos qy),
and in 3D
  lap:  [4 (cx + cy + cz) + 4 (cx cy + cx cz + cy cz) - 24] / 6,
  d_x:  (i/3) sin qx (1 + cos qy + cos qz).
Each test below drives the whole oracle step (or its auxiliary fields) with a
single lattice mode and checks the result against these symbols, so that a
dropped diagonal, a wrong weight or a wrong wall image fails one of them.  The
last tests check isotropy itself: two modes of equal |q| along an axis and
off it decay at rates that differ by O(q^6), where the compact 5-point rates
differ at O(q^4).
"""
import numpy as np
import pytest

from oracle import oracle as O


def iso_lap2(qx, qy):
    return (8 * (np.cos(qx) + np.cos(qy)) + 4 * np.cos(qx) * np.cos(qy) - 20) / 6


def iso_lap3(qx, qy, qz):
    cx, cy, cz = np.cos(qx), np.cos(qy), np.cos(qz)
    return (4 * (cx + cy + cz) + 4 * (cx * cy + cx * cz + cy * cz) - 24) / 6


def iso_dx2(qx, qy):
    return np.sin(qx) * (2 + np.cos(qy)) / 3


def iso_dx3(qx, qy, qz):
    return np.sin(qx) * (1 + np.cos(qy) + np.cos(qz)) / 3


def _lin_factor(lam, cfg, a):
    # lam = -(eigenvalue of the Laplacian); mu = (a + kappa lam + c lam^2) phi
    return 1.0 - cfg.Gamma * lam * (a + cfg.kappa * lam + cfg.c * lam ** 2)


@pytest.mark.parametrize("walls,hydro", [(0, 0), (1, 0), (0, 1)])
def test_linear_stage_iso_fourier_factor_2d(walls, hydro):
    """b = 0, uniform a: every lattice eigenmode of Eq. massdiff is multiplied per
    step by 1 - Gamma lam (a + kappa lam + c lam^2) with lam from the 9-point
    symbol.  With walls the eigenmodes along y are half-sample cosines (even
    image about the planes half a spacing out), diagonal links included."""
    ny, nx = 12, 16
    cfg = O.make_cfg(nx=nx, ny=ny, walls=walls, hydro=hydro, b=0.0, kappa=-0.025, c=0.02,
                     Gamma=0.05, Tc=1.0, T0=0.7, T_w=0.7, xi=0.0, stencil=1)
    st = O.init(cfg)
    rng = np.random.default_rng(15)
    amp = 1e-7 if hydro else 1e-3
    st.phi = amp * rng.standard_normal((ny, nx))
    st.T[:] = 0.7
    out = O.step(st)
    qx = 2 * np.pi * np.fft.fftfreq(nx)[None, :]
    if walls:
        import scipy.fft as sfft
        qy = (np.pi * np.arange(ny) / ny)[:, None]
        t0 = np.fft.fft(sfft.dct(st.phi, type=2, axis=0), axis=1)
        t1 = np.fft.fft(sfft.dct(out.phi, type=2, axis=0), axis=1)
    else:
        qy = 2 * np.pi * np.fft.fftfreq(ny)[:, None]
        t0, t1 = np.fft.fft2(st.phi), np.fft.fft2(out.phi)
    lam = -iso_lap2(qx, qy)
    rtol = 1e-6 if hydro else 1e-11
    np.testing.assert_allclose(t1 / t0, _lin_factor(lam, cfg, -0.3), rtol=rtol, atol=rtol)


def test_linear_stage_iso_fourier_factor_3d():
    nz, ny, nx = 6, 5, 8
    cfg = O.make_cfg(d=3, nx=nx, ny=ny, nz=nz, walls=0, hydro=0, b=0.0, T0=0.7, T_w=0.7,
                     Tc=1.0, xi=0.0, stencil=1)
    st = O.init(cfg)
    st.phi = 1e-3 * np.random.default_rng(16).standard_normal((nz, ny, nx))
    st.T[:] = 0.7
    out = O.step(st)
    qz, qy, qx = np.meshgrid(*[2 * np.pi * np.fft.fftfreq(n) for n in (nz, ny, nx)], indexing="ij")
    lam = -iso_lap3(qx, qy, qz)
    np.testing.assert_allclose(np.fft.fftn(out.phi) / np.fft.fftn(st.phi),
                               _lin_factor(lam, cfg, -0.3), rtol=1e-11, atol=1e-11)


def test_advection_iso_fourier_factor():
    """mu = F = 0 and a uniform flow u0: the isotropic flux divergence multiplies
    mode q by exactly 1 - i (u0x Dx(q) + u0y Dy(q))."""
    ny, nx = 10, 16
    cfg = O.make_cfg(nx=nx, ny=ny, walls=0, hydro=1, b=0.0, kappa=0.0, c=0.0, Tc=1.0, T0=1.0,
                     T_w=1.0, xi=0.0, tau=0.8, stencil=1)
    u0 = np.array([0.03, -0.02, 0.0])
    st = O.init(cfg)
    fe = O.feq(2, 1.0, u0)
    st.f = np.ascontiguousarray(fe[:, None, None] * np.ones((1, ny, nx)))
    st.phi = 1e-2 * np.random.default_rng(17).standard_normal((ny, nx))
    st.T[:] = 1.0
    out = O.step(st)
    qy = 2 * np.pi * np.fft.fftfreq(ny)[:, None]
    qx = 2 * np.pi * np.fft.fftfreq(nx)[None, :]
    expect = 1 - 1j * (u0[0] * iso_dx2(qx, qy) + u0[1] * iso_dx2(qy, qx))
    np.testing.assert_allclose(np.fft.fft2(out.phi) / np.fft.fft2(st.phi), expect, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("d", [2, 3])
def test_force_of_a_single_mode_pressure(d):
    """Only the a term (b = kappa = c = 0, uniform a): P_ab = a phi^2/2 delta_ab,
    so with phi^2 = 1 + eps cos(k.r) the force is exactly
    F_b = (a eps / 2) D_b(k) sin(k.r), D_b the isotropic gradient symbol."""
    shp = (6, 5, 8) if d == 3 else (10, 12)
    m = (1, 2, 3) if d == 3 else (2, 3)            # mode numbers along (slowest .. x)
    cfg = O.make_cfg(d=d, nx=shp[-1], ny=shp[-2], nz=shp[0] if d == 3 else 1, walls=0,
                     b=0.0, kappa=0.0, c=0.0, Tc=1.0, T0=0.7, T_w=0.7, xi=0.0, stencil=1)
    st = O.init(cfg)
    grids = np.meshgrid(*[np.arange(n) for n in shp], indexing="ij")
    k = [2 * np.pi * mi / n for mi, n in zip(m, shp)]
    phase = sum(ki * g for ki, g in zip(k, grids))
    eps, a = 0.5, -0.3
    st.phi = np.sqrt(1 + eps * np.cos(phase))
    st.T[:] = 0.7
    F = O.aux(st)["F"]
    if d == 2:
        ky, kx = k
        D = [iso_dx2(kx, ky), iso_dx2(ky, kx)]
    else:
        kz, ky, kx = k
        D = [iso_dx3(kx, ky, kz), iso_dx3(ky, kx, kz), iso_dx3(kz, kx, ky)]
    for b in range(d):
        np.testing.assert_allclose(F[b], a * eps / 2 * D[b] * np.sin(phase), rtol=0, atol=1e-14)


@pytest.mark.parametrize("d", [2, 3])
def test_iso_wall_rule_equals_mirror_lattice(d):
    """Diagonal offsets across a wall read the mirror image with the field's
    parity: the walled lattice equals the first half of a periodic lattice of
    twice the length holding the state and its mirror image."""
    shp = (5, 6, 7) if d == 3 else (9, 10)
    L = shp[0]
    kw = dict(nx=shp[-1], ny=shp[-2], nz=shp[0] if d == 3 else 1)
    par = dict(d=d, xi=0.0, tau=0.9, b=0.8, kappa=-0.2, c=0.3, stencil=1)
    st = O.init(O.make_cfg(walls=1, **par, **kw))
    rng = np.random.default_rng(19)
    e, w = O.velocity_set(d)
    st.phi = 0.3 * rng.standard_normal(st.phi.shape)
    st.T = 0.5 + rng.random(st.T.shape)
    st.f = np.ascontiguousarray(w.reshape((-1,) + (1,) * d) * (1 + 0.05 * rng.standard_normal(st.f.shape)))
    refl = [int(np.where((e[:, :d - 1] == e[i, :d - 1]).all(1) & (e[:, d - 1] == -e[i, d - 1]))[0][0])
            for i in range(len(w))]
    dbl = lambda x: np.concatenate([x, x[::-1]], axis=0)
    kw2 = dict(kw)
    kw2["nz" if d == 3 else "ny"] = 2 * L
    stp = O.init(O.make_cfg(walls=0, **par, **kw2))
    stp.phi, stp.T = dbl(st.phi), dbl(st.T)
    stp.f = np.ascontiguousarray(np.stack([np.concatenate([st.f[i], st.f[refl[i]][::-1]], axis=0)
                                           for i in range(len(w))]))
    aw, ap = O.aux(st), O.aux(stp)
    np.testing.assert_allclose(aw["mu"], ap["mu"][:L], rtol=0, atol=1e-13)
    np.testing.assert_allclose(aw["F"][:, :L], ap["F"][:, :L], rtol=0, atol=1e-13)
    np.testing.assert_allclose(aw["u"][:, :L], ap["u"][:, :L], rtol=0, atol=1e-13)
    np.testing.assert_allclose(O.step(st).phi, O.step(stp).phi[:L], rtol=0, atol=1e-14)


@pytest.mark.parametrize("t_wall_mode", [0, 1])
def test_iso_heat_modes_with_wall_ghosts(t_wall_mode):
    """T - T_w = eps cos(kx x) s(y) with s the Dirichlet eigenvector of the wall
    rule (sin(pi m y/(ny-1)) with held wall layers, sin(pi m (y+1/2)/ny) with the
    halfway ghost 2 T_w - T) is multiplied per sub-step by 1 + (xi/nsub) Lambda,
    Lambda the 9-point symbol; the x dependence makes the diagonal ghosts count."""
    ny, nx, Tw, xi, steps = 14, 12, 0.5, 0.15, 3
    cfg = O.make_cfg(nx=nx, ny=ny, walls=1, t_wall_mode=t_wall_mode, hydro=0, phi_amp=0.0,
                     xi=xi, T0=1.0, T_w=Tw, stencil=1)
    assert cfg.nsub == 1
    st = O.init(cfg)
    y = np.arange(ny)[:, None]
    x = np.arange(nx)[None, :]
    kx, m = 2 * np.pi * 3 / nx, 2
    qy = np.pi * m / (ny - 1) if t_wall_mode == 0 else np.pi * m / ny
    s = np.sin(qy * y) if t_wall_mode == 0 else np.sin(qy * (y + 0.5))
    dev = 0.2 * np.cos(kx * x) * s
    st.T = Tw + dev
    out = O.run(st, steps)
    fac = (1 + xi * iso_lap2(kx, qy)) ** steps
    np.testing.assert_allclose(out.T - Tw, fac * dev, rtol=0, atol=1e-14)


def _decay_rate(d, shape, mode):
    """-(Laplacian eigenvalue) of one lattice mode, measured from one oracle step
    with mu = a phi (b = kappa = c = 0): phi' = phi + Gamma a lap phi."""
    res = []
    for stencil in (0, 1):
        kw = dict(nx=shape[-1], ny=shape[-2], nz=shape[0] if d == 3 else 1)
        cfg = O.make_cfg(d=d, walls=0, hydro=0, b=0.0, kappa=0.0, c=0.0, Gamma=0.05, Tc=1.0,
                         T0=0.7, T_w=0.7, xi=0.0, stencil=stencil, **kw)
        st = O.init(cfg)
        grids = np.meshgrid(*[np.arange(n) for n in shape], indexing="ij")
        phase = sum(2 * np.pi * mi / n * g for mi, n, g in zip(mode, shape, grids))
        st.phi = 1e-3 * np.cos(phase)
        st.T[:] = 0.7
        out = O.step(st)
        idx = tuple(mi % n for mi, n in zip(mode, shape))
        r = np.fft.fftn(out.phi)[idx] / np.fft.fftn(st.phi)[idx]
        res.append(((1 - r) / (cfg.Gamma * -0.3)).real)
    return res


@pytest.mark.parametrize("d", [2, 3])
def test_isotropy_equal_wavenumber_modes(d):
    """Modes of equal |q| along an axis and off it: (5,0) and (3,4) on 64^2;
    (3,0,0) and (2,2,1) on 24^3.  The isotropic rates agree to within 2 % of
    the compact stencil's spread, and along the axis both stencils agree."""
    if d == 2:
        shape, m_ax, m_off = (64, 64), (0, 5), (4, 3)
    else:
        shape, m_ax, m_off = (24, 24, 24), (0, 0, 3), (1, 2, 2)
    c_ax, i_ax = _decay_rate(d, shape, m_ax)
    c_off, i_off = _decay_rate(d, shape, m_off)
    q2 = (2 * np.pi * 5 / 64) ** 2 if d == 2 else (2 * np.pi * 3 / 24) ** 2
    assert abs(c_ax - i_ax) < 1e-10
    spread_c = abs(c_ax - c_off) / q2
    spread_i = abs(i_ax - i_off) / q2
    assert spread_c > 5e-3
    assert spread_i < 0.02 * spread_c, (spread_i, spread_c)


@pytest.mark.parametrize("d", [2, 3])
def test_largest_isotropic_eigenvalue(d):
    """The largest -(Laplacian eigenvalue) of the isotropic stencils is 16/3, at
    q = (pi, pi) in 2D and q = (pi, pi, 0) in 3D (the stability limit of the
    explicit phi update uses it); the compact stencils reach 4d there."""
    if d == 2:
        shape, mode = (8, 8), (4, 4)
        q = np.linspace(-np.pi, np.pi, 121)
        grid_max = (-iso_lap2(q[:, None], q[None, :])).max()
    else:
        shape, mode = (6, 8, 8), (0, 4, 4)
        q = np.linspace(-np.pi, np.pi, 49)
        grid_max = (-iso_lap3(q[:, None, None], q[None, :, None], q[None, None, :])).max()
    compact, iso = _decay_rate(d, shape, mode)
    assert abs(iso - 16 / 3) < 1e-9 and abs(compact - 8) < 1e-9
    assert abs(grid_max - 16 / 3) < 1e-12
