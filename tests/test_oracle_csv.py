"""Pins of the snapshot table (oracle/snapshot.py)."""
import numpy as np

from oracle.mac import Cavity
from oracle.snapshot import cell_table


def test_linear_fields_are_exact_at_centres():
    cav = Cavity(nx=6, ny=5, nz=4, length=1.5)
    h = cav.length / cav.nx
    # u = 2 x + 3 on the u faces (x = i h), v = -y, w = 0.5 z + 1
    k, j, i = np.meshgrid(np.arange(4), np.arange(5), np.arange(7), indexing="ij")
    u = 2.0 * (i * h) + 3.0
    k, j, i = np.meshgrid(np.arange(4), np.arange(6), np.arange(6), indexing="ij")
    v = -(j * h)
    k, j, i = np.meshgrid(np.arange(5), np.arange(5), np.arange(6), indexing="ij")
    w = 0.5 * (k * h) + 1.0
    p = np.arange(6 * 5 * 4, dtype=np.float64).reshape(4, 5, 6)
    t = cell_table(cav, u, v, w, p)
    x, y, z = t[:, 0], t[:, 1], t[:, 2]
    np.testing.assert_allclose(t[:, 3], 2.0 * x + 3.0, rtol=1e-15)
    np.testing.assert_allclose(t[:, 4], -y, rtol=1e-15)
    np.testing.assert_allclose(t[:, 5], 0.5 * z + 1.0, rtol=1e-15)
    # x fastest: row r is cell (r % nx, (r // nx) % ny, r // (nx ny)); p in the same order
    r = np.arange(t.shape[0])
    np.testing.assert_array_equal(t[:, 6], r.astype(np.float64))
    np.testing.assert_allclose(x, (r % 6 + 0.5) * h, rtol=1e-15)
    np.testing.assert_allclose(z, (r // 30 + 0.5) * h, rtol=1e-15)
