"""Staggered (MAC) grid of the cavity and its wall rules (oracle, FP64).

Sec. 3 of the paper: the fluid fills a closed cube; one wall (the "lid")
moves tangentially; walls carry simple Dirichlet conditions.  Sec. 3.1: the
velocity components live on cell faces, the pressure at cell centres
(staggered grid, Harlow & Welch).

Readings fixed here (the paper gives no formulas):

* Cells are cubes of edge h = length / nx; the box is nx*h x ny*h x nz*h.
* u lives on x-faces, shape (nz, ny, nx+1); v on y-faces, (nz, ny+1, nx);
  w on z-faces, (nz+1, ny, nx); p at centres, (nz, ny, nx).  x is fastest.
* Normal velocity on every wall is zero: u[:, :, 0] = u[:, :, nx] = 0 and
  likewise for v (y walls) and w (z walls).  These faces never change.
* The lid is the y = ny*h wall, moving in +x with speed ``lid_u``; every
  other wall is at rest.  So the tangential wall value is ``lid_u`` for u on
  the top wall and 0 everywhere else.
* Tangential values outside the box are ghosts mirrored through the wall
  value W: ghost = 2 W - (value on the mirrored interior sample).  Where a
  sample lies outside along several axes, the ghost layers are filled axis by
  axis in the order x, y, z, each later axis covering the ghost layers of the
  earlier ones.

Parity: the ghost layer construction is pinned through the advection and
diffusion tests (walls at rest give odd extensions; exact wall values at the
wall position), see ``tests/test_oracle_step.py``.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass(frozen=True)
class Cavity:
    """Geometry and physical parameters of one cavity."""

    nx: int
    ny: int
    nz: int
    length: float = 1.0          # box edge along x; h = length / nx
    dt: float = 0.01
    rho: float = 1.0
    nu: float = 0.0
    lid_u: float = 1.0
    g: tuple = (0.0, 0.0, 0.0)   # lid forcing offset per unit time (Sec. 3)
    rtol: float = 1e-8
    max_iters: int = 0           # 0 -> 20 * max(nx, ny, nz)
    advect_order: int = 1        # backtrace: 1 explicit Euler, 2 explicit midpoint (RK2)
    warm_start: bool = False     # pressure solve starts from the previous step's p (else 0)

    @property
    def h(self) -> float:
        return self.length / self.nx

    @property
    def extent(self):
        h = self.h
        return (self.nx * h, self.ny * h, self.nz * h)

    @property
    def iter_cap(self) -> int:
        return self.max_iters if self.max_iters > 0 else 20 * max(self.nx, self.ny, self.nz)

    def face_shape(self, comp: int):
        nx, ny, nz = self.nx, self.ny, self.nz
        return [(nz, ny, nx + 1), (nz, ny + 1, nx), (nz + 1, ny, nx)][comp]

    @property
    def cell_shape(self):
        return (self.nz, self.ny, self.nx)


def wall_value(cav: Cavity, comp: int, axis: int, side: int) -> float:
    """Tangential wall velocity of component ``comp`` on wall (axis, side).

    axis: 0 x, 1 y, 2 z; side: 0 low, 1 high.  Only u on the top y wall moves.
    """
    if comp == 0 and axis == 1 and side == 1:
        return cav.lid_u
    return 0.0


def ghosted(cav: Cavity, f: np.ndarray, comp: int) -> np.ndarray:
    """Copy of face field ``f`` with one ghost layer on each tangential axis.

    Along the component's own (normal) axis the array already contains the
    wall faces and no ghost is added.  Returns (array, offsets) where offsets
    are the index shifts (z, y, x) of the interior inside the returned array.
    """
    pad = [0, 0, 0]  # in array axis order (z, y, x)
    for axis in range(3):          # physical axis 0 x, 1 y, 2 z
        if axis != comp:
            pad[2 - axis] = 1
    e = np.zeros(tuple(s + 2 * q for s, q in zip(f.shape, pad)))
    oz, oy, ox = pad
    e[oz:oz + f.shape[0], oy:oy + f.shape[1], ox:ox + f.shape[2]] = f
    # Fill ghost layers axis by axis: x, then y, then z.
    for axis in range(3):
        if axis == comp:
            continue
        a = 2 - axis  # array axis
        n = f.shape[a]
        lo_w = wall_value(cav, comp, axis, 0)
        hi_w = wall_value(cav, comp, axis, 1)
        e_sw = np.moveaxis(e, a, 0)  # view with the filled axis first
        e_sw[0] = 2.0 * lo_w - e_sw[1]
        e_sw[n + 1] = 2.0 * hi_w - e_sw[n]
    return e, (oz, oy, ox)


def interior_mask(cav: Cavity, comp: int) -> np.ndarray:
    """True on faces that are unknowns (every face except wall-normal ones)."""
    shape = cav.face_shape(comp)
    m = np.ones(shape, dtype=bool)
    a = 2 - comp
    idx = [slice(None)] * 3
    idx[a] = 0
    m[tuple(idx)] = False
    idx[a] = shape[a] - 1
    m[tuple(idx)] = False
    return m


def face_positions(cav: Cavity, comp: int):
    """Physical coordinates (X, Y, Z) of every face of component ``comp``.

    u face (i, j, k) sits at (i h, (j+1/2) h, (k+1/2) h); v and w likewise
    with the half shift removed on their own axis.
    """
    nzs, nys, nxs = cav.face_shape(comp)
    h = cav.h
    off = [0.5, 0.5, 0.5]
    off[comp] = 0.0
    k, j, i = np.meshgrid(np.arange(nzs), np.arange(nys), np.arange(nxs), indexing="ij")
    return ((i + off[0]) * h, (j + off[1]) * h, (k + off[2]) * h)


def cell_centres(cav: Cavity):
    h = cav.h
    k, j, i = np.meshgrid(np.arange(cav.nz), np.arange(cav.ny), np.arange(cav.nx), indexing="ij")
    return ((i + 0.5) * h, (j + 0.5) * h, (k + 0.5) * h)


def kinetic_energy(u, v, w) -> float:
    """Discrete kinetic energy sum of squares over all faces (times 1/2)."""
    return 0.5 * (np.sum(u * u) + np.sum(v * v) + np.sum(w * w))
