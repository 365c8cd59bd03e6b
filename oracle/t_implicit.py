"""Implicit temperature step: the plain FP64 reference.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``): the tests compare the
library's implicit temperature update with this definition.

The paper advances the temperature with the explicit diffusion equation
d_t T = xi lap T (Sec. 2, after Eq. massdiff), which needs xi <= 1/(2d) per
step; the library otherwise splits a step into n_sub explicit sub-steps.  Its
implicit option takes one backward-Euler step per time step,

    (I - xi L) T(t+1) = T(t),

with L the same Laplacian and the same wall rules as the explicit update.
L A(r) = sum_e c_e [A(r + e) - A(r)] over the stencil's offsets e: the axis
neighbours with c_e = 1 (compact 5-/7-point stencil), or every velocity of
D2Q9 / D3Q19 with c_e = 6 w_e (isotropic 9-/19-point stencil: 2/3 and 1/6 in
2D, 1/3 and 1/6 in 3D).  Wall rules:
  * walls off: periodic in every direction;
  * LF_TWALL_LAYERS (0): the first and last layer along the wall normal are
    held at T_w; the rows next to them see T_w as their neighbour;
  * LF_TWALL_HALFWAY (1): every layer is unknown; the ghost beyond each wall
    is 2 T_w - T of its mirror image across the wall plane (the site with the
    wall layer's normal coordinate and the offset's other coordinates).
The matrix is written out here from that definition, one stencil entry at a
time, and solved with a sparse direct solver.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla


def stencil_offsets(dims, stencil):
    """[(offset, c_e)] of L A = sum_e c_e [A(r + e) - A(r)], offsets in array
    axis order (wall normal first)."""
    out = []
    for e in np.ndindex(*([3] * dims)):
        e = tuple(int(v) - 1 for v in e)
        m2 = sum(v * v for v in e)
        if m2 == 0:
            continue
        if stencil == 0:
            if m2 == 1:
                out.append((e, 1.0))
        elif m2 <= 2:
            w = (1 / 9 if m2 == 1 else 1 / 36) if dims == 2 else (1 / 18 if m2 == 1 else 1 / 36)
            out.append((e, 6.0 * w))
    return out


def implicit_matrix(shape, xi, walls, t_mode, stencil=0):
    """Sparse (I - xi L) over the unknown sites and the right-hand-side offset
    that the wall values contribute; shape = (ny, nx) or (nz, ny, nx), the
    wall normal is axis 0 (y in 2D, z in 3D)."""
    shape = tuple(shape)
    dims = len(shape)
    offsets = stencil_offsets(dims, stencil)
    nw = shape[0]
    n = int(np.prod(shape))
    idx = np.arange(n).reshape(shape)
    rows, cols, vals = [], [], []
    fixed = np.zeros(shape, dtype=bool)
    if walls and t_mode == 0:
        fixed[0] = True
        fixed[-1] = True
    wall_rhs = np.zeros(shape)              # coefficient of T_w in the right-hand side
    for pos in np.ndindex(*shape):
        i = idx[pos]
        if fixed[pos]:
            rows.append(i); cols.append(i); vals.append(1.0)
            continue
        diag = 1.0 + xi * sum(c for _, c in offsets)
        for e, c in offsets:
            q = [p + v for p, v in zip(pos, e)]
            if walls and (q[0] < 0 or q[0] >= nw):
                # halfway ghost 2 T_w - T(mirror), the mirror keeping the wall
                # layer of pos (layers mode never reaches here)
                q[0] = pos[0]
                q = [v % n_ for v, n_ in zip(q, shape)]
                rows.append(i); cols.append(idx[tuple(q)]); vals.append(xi * c)
                wall_rhs[pos] += 2.0 * xi * c
                continue
            q = [v % n_ for v, n_ in zip(q, shape)]
            j = idx[tuple(q)]
            if walls and t_mode == 0 and fixed[tuple(q)]:
                wall_rhs[pos] += xi * c            # neighbour held at T_w
                continue
            rows.append(i); cols.append(j); vals.append(-xi * c)
        rows.append(i); cols.append(i); vals.append(diag)
    A = sp.csr_matrix((vals, (rows, cols)), shape=(n, n))
    return A, fixed, wall_rhs


def implicit_step(T, xi, T_w, walls, t_mode, stencil=0):
    """One backward-Euler step of the temperature (FP64); T has the wall
    normal on axis 0."""
    T = np.asarray(T, dtype=np.float64)
    A, fixed, wall_rhs = implicit_matrix(T.shape, xi, walls, t_mode, stencil)
    rhs = T.copy()
    rhs[fixed] = T_w
    rhs = rhs + wall_rhs * T_w
    out = spla.spsolve(A.tocsc(), rhs.ravel())
    return out.reshape(T.shape)
