"""Seeded synthetic inputs and the named workloads.

This module holds no arithmetic of the method: it only draws random numbers
(numpy, seeded) and lists the parameter sets of the workloads.  Both the CUDA
path and the oracle receive what it produces.

Workloads (2D lamellar quench between two cold walls, the physics of the
64 x 64 reference case with kappa < 0 so that the lamellar wavelength
2 pi / sqrt(-kappa/2c) is about 8 sites):
  small64:   64 x 64, FP64, xi = 0.01, 2000 steps, diagnostics every 200
  prec1024:  1024 x 1024, FP32 deviations, xi in {1e-3, 1e-1}, 50k steps
  ens96:     96 runs, 24 each of 128^2, 256^2, 384^2, 512^2, xi log-uniform in
             [1e-4, 1], tau in {0.6, 1, 3}
  cube384:   384^3 D3Q19, FP32, walls normal to z, xi in {1e-3, 1e-2}, tau in {0.6, 3}
  sur256:    256 x 256 for the learned surrogate, xi log-uniform in [1e-4, 1]
"""
from __future__ import annotations

import numpy as np

BASE = dict(b=1.0, kappa=-0.025, c=0.02, Gamma=0.05, Tc=1.0, T0=1.1, T_w=0.5, tau=1.0, n0=1.0,
            phi_amp=0.05, walls=1, t_wall_mode=0, hydro=1)

WORKLOADS = {
    "small64": dict(BASE, d=2, nx=64, ny=64, xi=0.01, precision="fp64", steps=2000, diag_every=200),
    "prec1024": dict(BASE, d=2, nx=1024, ny=1024, xi=1e-3, precision="fp32", steps=50000),
    "cube384": dict(BASE, d=3, nx=384, ny=384, nz=384, xi=1e-3, tau=0.6, precision="fp32", steps=20000),
    "sur256": dict(BASE, d=2, nx=256, ny=256, precision="fp32"),
}


def ensemble_members(seed: int = 2011):
    """The 96-run ensemble: (nx, ny, xi, tau, seed) per run, sizes interleaved."""
    rng = np.random.default_rng(seed)
    sizes = [128, 256, 384, 512] * 24
    xis = 10.0 ** rng.uniform(-4.0, 0.0, size=96)
    taus = rng.choice([0.6, 1.0, 3.0], size=96)
    return [dict(nx=s, ny=s, xi=float(x), tau=float(t), seed=1000 + i)
            for i, (s, x, t) in enumerate(zip(sizes, xis, taus))]


def random_state(shape, Q, seed, phi_amp=0.3, f_rel=0.05, T_lo=0.5, T_hi=1.1, dtype=np.float64):
    """Random phi (uniform), T (uniform) and relative population perturbations
    r (normal); a caller builds f_i = w_i (1 + r_i) with its own weights."""
    rng = np.random.default_rng(seed)
    phi = rng.uniform(-phi_amp, phi_amp, size=shape).astype(dtype)
    T = rng.uniform(T_lo, T_hi, size=shape).astype(dtype)
    r = (f_rel * rng.standard_normal((Q,) + tuple(shape))).astype(dtype)
    return phi, T, r
