"""Pins of the oracle's assembled matrices against closed forms (no GPU).

Pressure matrix (Sec. 3.1, CSR Poisson system): symmetric, integer, zero row
sums, and its full spectrum equals the separable DCT-II closed form
lambda(k) = sum_d 4 sin^2(pi k_d / (2 n_d)), k_d = 0..n_d-1, with exactly
one zero eigenvalue.  Diffusion matrices: each component's L has the
sine-mode eigenvectors of its wall rules (DST-I along the component's own
axis, DST-II along the tangential axes).
"""
import itertools

import numpy as np
import pytest

from oracle.mac import Cavity
from oracle.operators import diffusion_csr, diffusion_L_csr, poisson_csr

SHAPES = [(1, 1, 6), (2, 3, 4), (3, 3, 3), (4, 5, 3), (6, 6, 6), (5, 2, 6)]


def dct_eigs(nx, ny, nz):
    lam = []
    for kx, ky, kz in itertools.product(range(nx), range(ny), range(nz)):
        lam.append(4 * np.sin(np.pi * kx / (2 * nx)) ** 2 + 4 * np.sin(np.pi * ky / (2 * ny)) ** 2
                   + 4 * np.sin(np.pi * kz / (2 * nz)) ** 2)
    return np.sort(np.array(lam))


@pytest.mark.parametrize("shape", SHAPES)
def test_poisson_symmetric_integer_rowsum(shape):
    A = poisson_csr(*shape).toarray()
    assert np.array_equal(A, A.T)
    assert np.array_equal(A, np.round(A))
    assert np.all(A.sum(axis=1) == 0)
    d = np.diag(A)
    assert d.min() >= 0 and d.max() <= 6
    # off-diagonals are 0 or -1 and the diagonal counts them
    off = A - np.diag(d)
    assert set(np.unique(off)) <= {0.0, -1.0}
    assert np.array_equal(-off.sum(axis=1), d)



@pytest.mark.parametrize("shape", [(1, 1, 5), (3, 4, 5), (8, 6, 7)])
def test_poisson_energy_is_sum_over_grid_edges(shape):
    """p.Ap equals the sum of (p_i - p_j)^2 over the pairs of face-adjacent
    cells (counted once): the form the GPU direction kernel reduces."""
    nx, ny, nz = shape
    A = poisson_csr(nx, ny, nz)
    p = np.random.default_rng(3).standard_normal((nz, ny, nx))
    edges = sum(float(np.sum(np.diff(p, axis=ax) ** 2)) for ax in range(3))
    assert float(p.ravel() @ (A @ p.ravel())) == pytest.approx(edges, rel=1e-13)

@pytest.mark.parametrize("shape", SHAPES)
def test_poisson_spectrum_closed_form(shape):
    A = poisson_csr(*shape).toarray()
    ev = np.linalg.eigvalsh(A)
    ref = dct_eigs(*shape)
    np.testing.assert_allclose(ev, ref, atol=1e-12)
    assert np.sum(np.abs(ev) < 1e-10) == 1  # PSD, null space = constants


@pytest.mark.parametrize("shape,k", [((8, 6, 4), (1, 2, 3)), ((16, 16, 16), (1, 1, 1)),
                                     ((7, 9, 5), (6, 0, 2))])
def test_poisson_dct_mode_is_eigenvector(shape, k):
    nx, ny, nz = shape
    A = poisson_csr(*shape)
    kk, jj, ii = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    mode = (np.cos(np.pi * k[0] * (ii + 0.5) / nx) * np.cos(np.pi * k[1] * (jj + 0.5) / ny)
            * np.cos(np.pi * k[2] * (kk + 0.5) / nz)).ravel()
    lam = sum(4 * np.sin(np.pi * kd / (2 * nd)) ** 2 for kd, nd in zip(k, shape))
    np.testing.assert_allclose(A @ mode, lam * mode, atol=1e-12)


def sine_mode(cav, comp, k):
    """Closed-form eigenvector of the diffusion L of component ``comp``."""
    n = (cav.nx, cav.ny, cav.nz)
    shape = cav.face_shape(comp)
    kk, jj, ii = np.meshgrid(*[np.arange(s) for s in shape], indexing="ij")
    idx = (ii, jj, kk)
    m = np.ones(shape)
    lam = 0.0
    for d in range(3):
        if d == comp:      # faces on the walls are known zeros: DST-I
            m = m * np.sin(np.pi * k[d] * idx[d] / n[d])
        else:              # ghost mirrored through a zero wall: DST-II
            m = m * np.sin(np.pi * k[d] * (idx[d] + 0.5) / n[d])
        lam += 4 * np.sin(np.pi * k[d] / (2 * n[d])) ** 2
    return m, lam


@pytest.mark.parametrize("comp", [0, 1, 2])
@pytest.mark.parametrize("k", [(1, 1, 1), (2, 3, 1), (3, 1, 4)])
def test_diffusion_sine_modes(comp, k):
    cav = Cavity(5, 6, 4, lid_u=0.7)
    kk = list(k)
    n = (cav.nx, cav.ny, cav.nz)
    kk[comp] = min(kk[comp], n[comp] - 1)
    for d in range(3):
        kk[d] = min(kk[d], n[d])
    L, mask = diffusion_L_csr(cav, comp)
    m, lam = sine_mode(cav, comp, kk)
    np.testing.assert_allclose(L @ m[mask], lam * m[mask], atol=1e-12)


@pytest.mark.parametrize("comp", [0, 1, 2])
def test_diffusion_matrix_spd_and_lid_term(comp):
    cav = Cavity(4, 5, 3, dt=0.1, nu=0.05, lid_u=2.0)
    H, bnd, mask = diffusion_csr(cav, comp)
    Hd = H.toarray()
    assert np.allclose(Hd, Hd.T, atol=0)
    assert np.linalg.eigvalsh(Hd).min() >= 1.0 - 1e-12  # I + c L, L PSD
    c = cav.nu * cav.dt / cav.h ** 2
    # only u faces touching the lid see the moving wall: c * 2 * lid_u
    shape = cav.face_shape(comp)
    expect = np.zeros(shape)
    if comp == 0:
        expect[:, cav.ny - 1, :] = c * 2.0 * cav.lid_u
    np.testing.assert_allclose(bnd, expect[mask], atol=1e-15)
