"""Implicit temperature step: the plain FP64 reference.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``): the tests compare the
library's implicit temperature update with this definition.

The paper advances the temperature with the explicit diffusion equation
d_t T = xi lap T (Sec. 2, after Eq. massdiff), which needs xi <= 1/(2d) per
step; the library otherwise splits a step into n_sub explicit sub-steps.  Its
implicit option takes one backward-Euler step per time step,

    (I - xi L) T(t+1) = T(t),

with L the same 5-point (2D) / 7-point (3D) Laplacian and the same wall rules
as the explicit update:
  * walls off: periodic in every direction;
  * LF_TWALL_LAYERS (0): the first and last layer along the wall normal are
    held at T_w; the rows next to them see T_w as their neighbour;
  * LF_TWALL_HALFWAY (1): every layer is unknown; the ghost beyond each wall
    is 2 T_w - T of the layer next to it.
The matrix is written out here from that definition, one stencil entry at a
time, and solved with a sparse direct solver.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla


def implicit_matrix(shape, xi, walls, t_mode):
    """Sparse (I - xi L) over the unknown sites and the right-hand-side offset
    that the wall values contribute; shape = (ny, nx) or (nz, ny, nx), the
    wall normal is axis 0 (y in 2D, z in 3D)."""
    shape = tuple(shape)
    dims = len(shape)
    nw = shape[0]
    n = int(np.prod(shape))
    idx = np.arange(n).reshape(shape)
    rows, cols, vals = [], [], []
    fixed = np.zeros(shape, dtype=bool)
    if walls and t_mode == 0:
        fixed[0] = True
        fixed[-1] = True
    extra_diag = np.zeros(shape)           # from the halfway ghosts
    wall_rhs = np.zeros(shape)              # coefficient of T_w in the right-hand side
    for pos in np.ndindex(*shape):
        i = idx[pos]
        if fixed[pos]:
            rows.append(i); cols.append(i); vals.append(1.0)
            continue
        diag = 1.0 + 2 * dims * xi
        for ax in range(dims):
            for step in (-1, 1):
                q = list(pos)
                q[ax] += step
                if ax == 0 and walls and (q[0] < 0 or q[0] >= nw):
                    # halfway ghost 2 T_w - T(pos)  (layers mode never reaches here)
                    diag += xi
                    wall_rhs[pos] += 2.0 * xi
                    continue
                q[ax] %= shape[ax]
                j = idx[tuple(q)]
                if walls and t_mode == 0 and fixed[tuple(q)]:
                    wall_rhs[pos] += xi            # neighbour held at T_w
                    continue
                rows.append(i); cols.append(j); vals.append(-xi)
        rows.append(i); cols.append(i); vals.append(diag)
    A = sp.csr_matrix((vals, (rows, cols)), shape=(n, n))
    return A, fixed, wall_rhs


def implicit_step(T, xi, T_w, walls, t_mode):
    """One backward-Euler step of the temperature (FP64); T has the wall
    normal on axis 0."""
    T = np.asarray(T, dtype=np.float64)
    A, fixed, wall_rhs = implicit_matrix(T.shape, xi, walls, t_mode)
    rhs = T.copy()
    rhs[fixed] = T_w
    rhs = rhs + wall_rhs * T_w
    out = spla.spsolve(A.tocsc(), rhs.ravel())
    return out.reshape(T.shape)
