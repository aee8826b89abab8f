"""Explicit CSR assembly of the linear systems of one time step (oracle).

Sec. 3.1 of the paper: the pressure Poisson equation becomes a sparse linear
system stored in Compressed-Row Storage (CSR) and solved by PCG; the SpMV
follows that representation.  This module builds those matrices entry by
entry, as the paper's unoptimised code does every step.  A
``scipy.sparse.csr_matrix`` holds the result and performs y = A x (a library
SpMV used as one step).

Readings (the paper prints no stencil):

* Pressure: A = -h^2 * (7-point Laplacian) with homogeneous Neumann walls,
  which is what zero normal velocity on every wall implies for the
  projection.  Row c: A[c,c] = n_c (number of neighbours inside the box,
  3..6), A[c,n] = -1 for each such neighbour.  Symmetric, positive
  semi-definite, null space = constants.
* Diffusion (viscosity, added to the paper's inviscid Euler equations as a
  separate backward-Euler substep in Stam's order): for velocity component
  ``comp`` the unknowns are the faces that are not wall-normal; with
  c = nu*dt/h^2 the matrix is H = I + c*L where L is the 7-point negative
  Laplacian (scaled by h^2) with these wall rules:
  - along the component's own axis a neighbour on a wall-normal face is a
    known zero (diagonal +1, no off-diagonal);
  - along a tangential axis a neighbour outside the box is the ghost
    2W - u_c (diagonal +2, right-hand side +2 c W).
  H is symmetric positive definite.

Pins (tests/test_oracle_operators.py): exact symmetry and integer entries,
zero row sums of A, the full spectrum of A against the DCT-II closed form
sum_d 4 sin^2(pi k_d / (2 n_d)) for grids up to 6^3 (one zero eigenvalue),
and H applied to the closed-form sine modes of each component.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .mac import Cavity, interior_mask, wall_value


def _lin(shape):
    return np.arange(int(np.prod(shape))).reshape(shape)


def poisson_csr(nx: int, ny: int, nz: int) -> sp.csr_matrix:
    """Neumann 7-point matrix A (scaled by h^2) on an nx x ny x nz cell grid."""
    shape = (nz, ny, nx)
    idx = _lin(shape)
    n = idx.size
    rows, cols, vals = [], [], []
    diag = np.zeros(shape)
    for a in range(3):  # array axis: 0 z, 1 y, 2 x
        for s in (-1, 1):
            src = [slice(None)] * 3
            dst = [slice(None)] * 3
            if s < 0:
                src[a], dst[a] = slice(1, None), slice(None, -1)
            else:
                src[a], dst[a] = slice(None, -1), slice(1, None)
            r = idx[tuple(src)].ravel()
            c = idx[tuple(dst)].ravel()
            rows.append(r)
            cols.append(c)
            vals.append(-np.ones(r.size))
            diag[tuple(src)] += 1.0
    rows.append(idx.ravel())
    cols.append(idx.ravel())
    vals.append(diag.ravel())
    A = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(n, n))
    A.sum_duplicates()
    A.sort_indices()
    return A


def diffusion_csr(cav: Cavity, comp: int):
    """H = I + c*L for velocity component ``comp`` and its wall right-hand side.

    Returns (H, bnd, mask): H acts on the unknown faces (``mask`` True, in
    C order), bnd is the constant vector c * sum(2 W) from the ghost rule, so
    the backward-Euler system is H x = u_star[mask] + bnd.
    """
    shape = cav.face_shape(comp)
    mask = interior_mask(cav, comp)
    num = -np.ones(shape, dtype=np.int64)
    num[mask] = np.arange(int(mask.sum()))
    n = int(mask.sum())
    c = cav.nu * cav.dt / (cav.h * cav.h)
    rows, cols, vals = [], [], []
    diag = np.zeros(shape)
    bnd = np.zeros(shape)
    own = 2 - comp  # array axis of the component's own direction
    for a in range(3):
        phys = 2 - a
        for s in (-1, 1):
            # every face, the neighbour at offset s along array axis a
            nb_ok = np.ones(shape, dtype=bool)
            sl_lo = [slice(None)] * 3
            if s < 0:
                sl_lo[a] = 0
            else:
                sl_lo[a] = shape[a] - 1
            nb_ok[tuple(sl_lo)] = False  # neighbour outside the array
            if a == own:
                # neighbour exists in the array (may be a known wall face)
                diag += 1.0
                shifted = np.roll(num, -s, axis=a)
                link = mask & nb_ok & (shifted >= 0)
                rows.append(num[link])
                cols.append(shifted[link])
                vals.append(-np.ones(int(link.sum())))
            else:
                side = 0 if s < 0 else 1
                W = wall_value(cav, comp, phys, side)
                inside = mask & nb_ok
                ghost = mask & ~nb_ok
                diag[inside] += 1.0
                shifted = np.roll(num, -s, axis=a)
                rows.append(num[inside])
                cols.append(shifted[inside])
                vals.append(-np.ones(int(inside.sum())))
                diag[ghost] += 2.0
                bnd[ghost] += 2.0 * W
    L = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(n, n))
    L = L + sp.diags(diag[mask])
    H = (sp.identity(n, format="csr") + c * L).tocsr()
    H.sum_duplicates()
    H.sort_indices()
    return H, c * bnd[mask], mask


def diffusion_L_csr(cav: Cavity, comp: int):
    """The integer matrix L of ``diffusion_csr`` (H = I + c L), for pins."""
    H, _, mask = diffusion_csr(Cavity(cav.nx, cav.ny, cav.nz, cav.length, dt=1.0,
                                      nu=cav.h * cav.h, lid_u=cav.lid_u), comp)
    n = H.shape[0]
    return (H - sp.identity(n, format="csr")).tocsr(), mask
