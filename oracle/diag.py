"""Plain numpy definitions of the run diagnostics (FP64).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The paper fixes the Mach check (Sec. 2: |u|_max / c_s < 0.1, n ~ 1) and talks
about lamellae parallel or perpendicular to the walls (Sec. 3) without
defining a number for it; it defines no structure factor.  The definitions
below are this project's readings, written out plainly:

* sums: total mass sum n, order parameter sum phi, momentum sum n u (with the
  half-force shift of Eq. moment), |u|_max and Ma = |u|_max / c_s;
* orientation: s = (d <(d_perp phi)^2> / <|grad phi|^2> - 1) / (d - 1), with
  central differences and the even wall reflection; s = +1 for lamellae
  parallel to the walls, -1 (d = 2) for lamellae perpendicular to them; also
  per layer along the wall normal;
* structure factor: S(k) = |sum_r (phi - mean) e^{-i k.r}|^2 / N over the whole
  box, averaged over shells of width dk = 2 pi / L_min (bin b = round(|k|/dk),
  b = 1 .. L_min // 2); S_peak = max_b S_b; k_peak = sum k_b S_b / sum S_b over
  the bins with S_b > S_peak / 2, k_b = b dk;
* free energy (phi part of Eq. fren) on the lattice: sum_r [a phi^2/2 +
  b phi^4/4 + c (nabla^2 phi)^2 / 2] + kappa/2 sum_links (phi(r + e) - phi(r))^2,
  the links joining nearest neighbours (periodic axes wrap; no link crosses a
  wall) and nabla^2 the 5-/7-point Laplacian with the even wall reflection.
  This is the lattice functional whose derivative with respect to phi(r) is
  the chemical potential of Eq. chem as the compact stencils discretise it
  (-kappa nabla^2 phi is minus the derivative of the link sum), so the pair
  (free energy, mu) is consistent site by site.
"""
from __future__ import annotations

import numpy as np

CS = 1.0 / np.sqrt(3.0)


def _pad(a: np.ndarray, axis: int, walls: bool, wall_axis: int) -> np.ndarray:
    widths = [(0, 0)] * a.ndim
    widths[axis] = (1, 1)
    mode = "symmetric" if (walls and axis == wall_axis) else "wrap"
    return np.pad(a, widths, mode=mode)


def _central(a: np.ndarray, axis: int, walls: bool, wall_axis: int) -> np.ndarray:
    p = _pad(a, axis, walls, wall_axis)
    sl_hi = [slice(None)] * a.ndim
    sl_lo = [slice(None)] * a.ndim
    sl_hi[axis] = slice(2, None)
    sl_lo[axis] = slice(0, -2)
    return 0.5 * (p[tuple(sl_hi)] - p[tuple(sl_lo)])


def _laplacian(a: np.ndarray, walls: bool, wall_axis: int) -> np.ndarray:
    out = np.zeros_like(a)
    for ax in range(a.ndim):
        p = _pad(a, ax, walls, wall_axis)
        sl_hi = [slice(None)] * a.ndim
        sl_lo = [slice(None)] * a.ndim
        sl_hi[ax] = slice(2, None)
        sl_lo[ax] = slice(0, -2)
        out += p[tuple(sl_hi)] + p[tuple(sl_lo)] - 2.0 * a
    return out


def gradients(phi: np.ndarray, walls: bool):
    """Central-difference gradient components, array axes order (z,) y, x."""
    wall_axis = 0  # the slowest array axis is the wall normal (y in 2D, z in 3D)
    return [_central(phi, ax, walls, wall_axis) for ax in range(phi.ndim)]


def orientation(phi: np.ndarray, walls: bool):
    """(s, s_per_layer) as defined in the module docstring."""
    d = phi.ndim
    g = gradients(phi, walls)
    gperp2 = g[0] ** 2
    gall2 = sum(x ** 2 for x in g)
    red = tuple(range(1, d))
    tot = gall2.mean()
    s = (d * gperp2.mean() / tot - 1.0) / (d - 1) if tot > 0 else 0.0
    lay_all = gall2.mean(axis=red)
    lay_perp = gperp2.mean(axis=red)
    with np.errstate(invalid="ignore", divide="ignore"):
        s_layer = np.where(lay_all > 0, (d * lay_perp / lay_all - 1.0) / (d - 1), 0.0)
    return float(s), s_layer


def structure_factor(phi: np.ndarray):
    """(k_b, S_b, k_peak, S_peak) as defined in the module docstring."""
    N = phi.size
    dphi = phi - phi.mean()
    Sk = np.abs(np.fft.fftn(dphi)) ** 2 / N
    ks = np.meshgrid(*[2 * np.pi * np.fft.fftfreq(n) for n in phi.shape], indexing="ij")
    kmag = np.sqrt(sum(k ** 2 for k in ks))
    Lmin = min(phi.shape)
    dk = 2 * np.pi / Lmin
    B = Lmin // 2
    b = np.floor(kmag / dk + 0.5).astype(np.int64)
    sums = np.bincount(b.reshape(-1), weights=Sk.reshape(-1), minlength=B + 1)[: B + 1]
    cnts = np.bincount(b.reshape(-1), minlength=B + 1)[: B + 1]
    Sb = np.where(cnts > 0, sums / np.maximum(cnts, 1), 0.0)
    Sb[0] = 0.0
    kb = np.arange(B + 1) * dk
    S_peak = Sb[1:].max() if B >= 1 else 0.0
    sel = Sb > 0.5 * S_peak
    sel[0] = False
    k_peak = float((kb[sel] * Sb[sel]).sum() / Sb[sel].sum()) if S_peak > 0 else 0.0
    return kb, Sb, k_peak, float(S_peak)


def link_squares(phi: np.ndarray, walls: bool) -> float:
    """sum over nearest-neighbour links of (phi(r + e) - phi(r))^2; along the
    wall normal (the slowest array axis) only links inside the lattice."""
    acc = 0.0
    for ax in range(phi.ndim):
        dl = np.diff(phi, axis=ax) if (walls and ax == 0) else np.roll(phi, -1, axis=ax) - phi
        acc += float((dl ** 2).sum())
    return acc


def free_energy(phi: np.ndarray, T: np.ndarray, walls: bool, b: float, kappa: float,
                c: float, Tc: float) -> float:
    a = (T - Tc) / Tc
    psi = _laplacian(phi, walls, 0)
    local = a * phi ** 2 / 2 + b * phi ** 4 / 4 + c * psi ** 2 / 2
    return float(local.sum()) + kappa / 2 * link_squares(phi, walls)


def sums(aux: dict, phi: np.ndarray):
    """Conservation sums and the Mach number from oracle aux fields."""
    n, u = aux["n"], aux["u"]
    d = phi.ndim
    umag = np.sqrt(sum(u[a] ** 2 for a in range(3)))
    umax = float(umag.max())
    return {
        "mass": float(n.sum()),
        "phi_sum": float(phi.sum()),
        "mom": [float((n * u[a]).sum()) for a in range(3)],
        "umax": umax,
        "mach": umax / CS,
        "d": d,
    }
