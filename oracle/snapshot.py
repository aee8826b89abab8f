"""Per-cell snapshot table of the cavity state (oracle).

Sec. 3.2 of the paper: the proxy app writes the state to a CSV file every
step for visualisation.  The columns are a reading (the paper names none):
cell centre x, y, z = (i + 1/2) h, (j + 1/2) h, (k + 1/2) h, the cell-centred
velocity (the mean of the two faces of the cell along each axis) and p, one
row per cell with x fastest.

Pinned by tests/test_oracle_csv.py: on fields linear in the face positions
the centred velocity equals the field at the centre exactly, and row order
and positions follow the MAC layout.  This module is test infrastructure.
"""
from __future__ import annotations

import numpy as np

from .mac import Cavity


def cell_table(cav: Cavity, u, v, w, p) -> np.ndarray:
    """(nx*ny*nz, 7) float64 table: x, y, z, u_c, v_c, w_c, p."""
    nx, ny, nz = cav.nx, cav.ny, cav.nz
    h = cav.length / nx
    # arrays are (z, y, x): u (nz, ny, nx+1), v (nz, ny+1, nx), w (nz+1, ny, nx)
    uc = 0.5 * (u[:, :, :-1] + u[:, :, 1:])
    vc = 0.5 * (v[:, :-1, :] + v[:, 1:, :])
    wc = 0.5 * (w[:-1, :, :] + w[1:, :, :])
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    cols = [(i + 0.5) * h, (j + 0.5) * h, (k + 0.5) * h, uc, vc, wc, np.asarray(p)]
    return np.stack([c.reshape(-1) for c in cols], axis=1)
