"""Seeded synthetic inputs shared by the CUDA path, the oracle and the tests.

This module holds no arithmetic of the solver itself: it only draws numbers.
Every value is a pure function of (seed, stream, linear index) through a
counter-based generator, so any subset of an input can be regenerated
without drawing the rest, on any machine, bit for bit.

Generator: the SplitMix64 output function (Steele, Lea, Flood, "Fast
splittable pseudorandom number generators", OOPSLA 2014) applied twice:

    key   = mix(seed + G * (stream + 1))
    bits  = mix(key + G * (index + 1))          G = 0x9E3779B97F4A7C15
    U     = (bits >> 11) * 2**-53               uniform on [0, 1)

Gaussian draws use the Box-Muller transform of two uniforms taken from
streams 2s and 2s+1.

Workloads (lid-driven cavity, Sec. 3 of the paper; sizes from the cavity and
Poisson configurations this library is measured on):

* ``cavity_perturbation``: uniform[-amp, amp] on every face that is not a
  wall-normal face, zero on wall-normal faces; stream = component (0 u, 1 v,
  2 w).  The paper's own start state is v0 = 0, p0 = 1 (Sec. 3, eq. 3); the
  perturbation breaks the mirror symmetry the exact start state has.
* ``gaussian_rhs``: N(0, 1) iid per cell with the mean removed, the
  right-hand side of a standalone Neumann-Poisson solve.
"""
from __future__ import annotations

import numpy as np

_G = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _mix(z: np.ndarray) -> np.ndarray:
    z = z.astype(np.uint64, copy=True)
    z ^= z >> np.uint64(30)
    z *= _M1
    z ^= z >> np.uint64(27)
    z *= _M2
    z ^= z >> np.uint64(31)
    return z


def uniform01(seed: int, stream: int, index: np.ndarray) -> np.ndarray:
    """Uniform doubles on [0, 1) for the given linear indices (53-bit)."""
    with np.errstate(over="ignore"):
        key = _mix(np.asarray([seed], dtype=np.uint64) + _G * np.uint64(stream + 1))
        idx = np.asarray(index, dtype=np.uint64)
        bits = _mix(key + _G * (idx + np.uint64(1)))
    return (bits >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def face_shapes(nx: int, ny: int, nz: int):
    """Array shapes (z, y, x order, x fastest) of the u, v, w face grids."""
    return [(nz, ny, nx + 1), (nz, ny + 1, nx), (nz + 1, ny, nx)]


def cavity_perturbation(nx: int, ny: int, nz: int, seed: int, amp: float = 1e-3):
    """Seeded uniform[-amp, amp] perturbation of u, v, w (wall-normal faces 0).

    Returns three C-contiguous float64 arrays shaped (z, y, x).
    """
    out = []
    for comp, shape in enumerate(face_shapes(nx, ny, nz)):
        n = int(np.prod(shape))
        vals = uniform01(seed, comp, np.arange(n, dtype=np.uint64))
        f = (amp * (2.0 * vals - 1.0)).reshape(shape)
        axis = 2 - comp  # x is the last array axis, z the first
        sl = [slice(None)] * 3
        sl[axis] = 0
        f[tuple(sl)] = 0.0
        sl[axis] = shape[axis] - 1
        f[tuple(sl)] = 0.0
        out.append(np.ascontiguousarray(f))
    return out


def gaussian_rhs(nx: int, ny: int, nz: int, seed: int) -> np.ndarray:
    """N(0,1) iid per cell, mean removed; shape (z, y, x), float64."""
    n = nx * ny * nz
    idx = np.arange(n, dtype=np.uint64)
    u1 = uniform01(seed, 0, idx)
    u2 = uniform01(seed, 1, idx)
    g = np.sqrt(-2.0 * np.log1p(-u1)) * np.cos(2.0 * np.pi * u2)
    g -= g.mean()
    return g.reshape(nz, ny, nx)


def batch_edges(n: int, seed: int = 5, choices=(32, 48, 64, 96)):
    """Edge lengths of n cubic cavities drawn uniformly from ``choices``
    (stream 7 of the counter-based generator)."""
    u = uniform01(seed, 7, np.arange(n, dtype=np.uint64))
    idx = np.minimum((u * len(choices)).astype(np.int64), len(choices) - 1)
    return [int(choices[i]) for i in idx]


def uniform_field(shape, seed: int, stream: int = 0, lo: float = -1.0, hi: float = 1.0):
    """Uniform[lo, hi) field of the given shape (for operator parity tests)."""
    n = int(np.prod(shape))
    vals = uniform01(seed, stream, np.arange(n, dtype=np.uint64))
    return (lo + (hi - lo) * vals).reshape(shape)
