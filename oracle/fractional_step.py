"""One fractional step of the lid-driven cavity (oracle, FP64).

Sec. 3 / 3.1 of the paper: the state (v, p) starts at v0 = 0, p0 = 1
(eq. 3); each fixed-length time step applies, in order,

1. ``apply_forces``     external forces g as a time-invariant offset
                        (Table 1: applyForces);
2. ``advect``           semi-Lagrangian advection of the velocity
                        (Table 1: solveAdvection);
3. ``diffuse``          backward-Euler viscosity, an addition to the
                        paper's inviscid equations, placed in Stam's order
                        (forces, advect, diffuse, project);
4. ``pressure_rhs``     divergence of the intermediate velocity;
5. ``solve_pressure``   CSR assembly + PCG on the Poisson system
                        (Table 1: solvePressureCorrection / pcg);
6. ``correct``          subtract the pressure gradient
                        (Table 1: applyPressureCorrection), then fix the
                        pressure gauge to mean 1 (p0 = 1).

Readings (the paper prints no formulas for any substep):

* forcing: the paper models the lid's push with g; here component c of
  every non-wall-normal face in the top cell layer (j = ny - 1) gains
  dt * g[c]; the lid itself enters as the tangential wall value of u
  (``mac``).  All configurations use g = 0.
* advection: each non-wall-normal face takes the velocity at its own
  position (its own component, the other two as the mean of the four
  nearest faces of that component), traces back one explicit Euler step
  x - dt * v, clamps the point into the box, and samples the old field there
  by trilinear interpolation with ``floor`` cell lookup and the ghost rule of
  ``mac``.  Only old values are read.
* diffusion: H x = u* + bnd with x0 = u* (``operators.diffusion_csr``),
  skipped when nu = 0.
* pressure: A p = -(rho h / dt) * (sum of outgoing face differences), with
  the mean of the right-hand side removed (exactly zero in exact arithmetic
  by the discrete divergence theorem), cold start p = 0.
* correction: u_f -= dt / (rho h) * (p_c - p_c') on faces between two
  cells; wall-normal faces stay zero.

Pins (tests/test_oracle_step.py): the face-difference sum after the step
equals -dt/(rho h) times the true solver residual; the projection never raises the
kinetic energy; mirror symmetry z -> L - z; zero state stays zero with
p = 1; zero-velocity advection is the identity; trilinear sampling and the
face-velocity averages are exact on linear fields; the diffusion solve of a
closed-form sine mode returns mode / (1 + c lambda); a stored snapshot of a
small run guards against regressions (tests/golden).
"""
from __future__ import annotations

import numpy as np

from .krylov import dic_precond, identity_precond, jacobi_precond, pcg
from .mac import Cavity, ghosted, interior_mask
from .operators import diffusion_csr, poisson_csr


# --------------------------------------------------------------------------
# 1. applyForces
# --------------------------------------------------------------------------
def apply_forces(cav: Cavity, u, v, w):
    out = [u.copy(), v.copy(), w.copy()]
    for comp in range(3):
        gc = cav.g[comp]
        if gc == 0.0:
            continue
        f = out[comp]
        m = interior_mask(cav, comp)
        top = np.zeros_like(m)
        top[:, cav.ny - 1, :] = True
        f[m & top] += cav.dt * gc
    return tuple(out)


# --------------------------------------------------------------------------
# 2. semi-Lagrangian advection
# --------------------------------------------------------------------------
def _interior_indices(cav: Cavity, comp: int):
    m = interior_mask(cav, comp)
    K, J, I = np.nonzero(m)
    return I, J, K


def face_velocity(cav: Cavity, fields, comp: int, I, J, K):
    """Velocity vector at faces (I, J, K) of component ``comp``.

    Own component: the face value.  Other component d: mean of the four
    d-faces at offsets o_c in {-1, 0} along comp's axis and o_d in {0, +1}
    along d's axis, summed in that loop order (o_c outer).
    """
    vel = []
    for d in range(3):
        f = fields[d]
        if d == comp:
            vel.append(f[K, J, I].astype(np.float64))
            continue
        s = np.zeros(I.shape)
        for oc in (-1, 0):
            for od in (0, 1):
                idx = [I.copy(), J.copy(), K.copy()]
                idx[comp] = idx[comp] + oc
                idx[d] = idx[d] + od
                s = s + f[idx[2], idx[1], idx[0]]
        vel.append(0.25 * s)
    return vel


def interpolate(cav: Cavity, f, comp: int, X, Y, Z):
    """Trilinear sample of face field ``f`` (component ``comp``) at points."""
    e, (oz, oy, ox) = ghosted(cav, f, comp)
    h = cav.h
    n = (cav.nx, cav.ny, cav.nz)
    g = [X / h, Y / h, Z / h]
    lo, t = [], []
    for d in range(3):
        if d != comp:
            g[d] = g[d] - 0.5
            lmin = -1
        else:
            lmin = 0
        l = np.clip(np.floor(g[d]).astype(np.int64), lmin, n[d] - 1)
        lo.append(l)
        t.append(g[d] - l)

    def at(di, dj, dk):
        return e[lo[2] + dk + oz, lo[1] + dj + oy, lo[0] + di + ox]

    def lerp(a, b, s):
        return a + s * (b - a)

    c00 = lerp(at(0, 0, 0), at(1, 0, 0), t[0])
    c10 = lerp(at(0, 1, 0), at(1, 1, 0), t[0])
    c01 = lerp(at(0, 0, 1), at(1, 0, 1), t[0])
    c11 = lerp(at(0, 1, 1), at(1, 1, 1), t[0])
    c0 = lerp(c00, c10, t[1])
    c1 = lerp(c01, c11, t[1])
    return lerp(c0, c1, t[2])


def advect(cav: Cavity, u, v, w):
    """Semi-Lagrangian advection (Sec. 3.1).  Backtrace: explicit Euler,
    x - dt v(x) (advect_order 1), or the explicit midpoint rule (advect_order
    2, a reading of the paper's "optimizing the advection kernel" future
    work): x_m = x - (dt/2) v(x), x - dt v(x_m), with v(x_m) sampled
    trilinearly from each component's own grid; every point is clamped into
    the box."""
    fields = (u, v, w)
    ext = cav.extent
    h = cav.h
    out = []
    for comp in range(3):
        I, J, K = _interior_indices(cav, comp)
        off = [0.5, 0.5, 0.5]
        off[comp] = 0.0
        pos = [(I + off[0]) * h, (J + off[1]) * h, (K + off[2]) * h]
        vel = face_velocity(cav, fields, comp, I, J, K)
        if cav.advect_order == 2:
            mid = [np.clip(pos[d] - 0.5 * cav.dt * vel[d], 0.0, ext[d]) for d in range(3)]
            vel = [interpolate(cav, fields[d], d, *mid) for d in range(3)]
        back = [np.clip(pos[d] - cav.dt * vel[d], 0.0, ext[d]) for d in range(3)]
        new = fields[comp].copy()
        new[K, J, I] = interpolate(cav, fields[comp], comp, *back)
        out.append(new)
    return tuple(out)


# --------------------------------------------------------------------------
# 3. implicit diffusion (viscosity)
# --------------------------------------------------------------------------
def diffuse(cav: Cavity, fields, fixed_iters=(None, None, None)):
    if cav.nu == 0.0:
        return tuple(f.copy() for f in fields), [None, None, None]
    out, stats = [], []
    for comp in range(3):
        H, bnd, mask = diffusion_csr(cav, comp)
        f = fields[comp]
        rhs = f[mask] + bnd
        x, st = pcg(H, rhs, x0=f[mask], rtol=cav.rtol, max_iters=cav.iter_cap,
                    fixed_iters=fixed_iters[comp])
        g = f.copy()
        g[mask] = x
        out.append(g)
        stats.append(st)
    return tuple(out), stats


# --------------------------------------------------------------------------
# 4.-6. projection
# --------------------------------------------------------------------------
def divergence_sum(u, v, w):
    """Sum of outgoing face differences per cell (h times the divergence)."""
    return (u[:, :, 1:] - u[:, :, :-1]) + (v[:, 1:, :] - v[:, :-1, :]) + (w[1:, :, :] - w[:-1, :, :])


def pressure_rhs(cav: Cavity, u, v, w):
    b = -(cav.rho * cav.h / cav.dt) * divergence_sum(u, v, w)
    return b - b.mean()


def solve_pressure(cav: Cavity, b, precond="none", fixed_iters=None, x0=None):
    A = poisson_csr(cav.nx, cav.ny, cav.nz)
    if precond == "dic":
        pc = dic_precond(A)[0]
    else:
        pc = identity_precond if precond == "none" else jacobi_precond(A)
    x, st = pcg(A, b.ravel(), x0=None if x0 is None else np.asarray(x0).ravel(), rtol=cav.rtol,
                max_iters=cav.iter_cap, precond=pc, fixed_iters=fixed_iters)
    return x.reshape(cav.cell_shape), st


def correct(cav: Cavity, u, v, w, p):
    s = cav.dt / (cav.rho * cav.h)
    u, v, w = u.copy(), v.copy(), w.copy()
    u[:, :, 1:-1] -= s * (p[:, :, 1:] - p[:, :, :-1])
    v[:, 1:-1, :] -= s * (p[:, 1:, :] - p[:, :-1, :])
    w[1:-1, :, :] -= s * (p[1:, :, :] - p[:-1, :, :])
    return u, v, w


def gauge(p):
    return p + (1.0 - p.mean())


# --------------------------------------------------------------------------
# the whole step
# --------------------------------------------------------------------------
def initial_state(cav: Cavity, perturbation=None):
    """v0 = 0 (+ optional perturbation of the non-wall-normal faces), p0 = 1."""
    if perturbation is None:
        u, v, w = (np.zeros(cav.face_shape(c)) for c in range(3))
    else:
        u, v, w = (np.array(a, dtype=np.float64, copy=True) for a in perturbation)
    return u, v, w, np.ones(cav.cell_shape)


def step(cav: Cavity, state, fixed_iters=None, precond="none"):
    """Advance (u, v, w, p) by one time step; returns (state, stats dict).

    fixed_iters: optional dict {"p": k, "u": k, "v": k, "w": k} replaying
    iteration counts of the solves instead of the stopping test.
    """
    fx = fixed_iters or {}
    u, v, w, p_prev = state
    u, v, w = apply_forces(cav, u, v, w)
    u, v, w = advect(cav, u, v, w)
    (u, v, w), dstats = diffuse(cav, (u, v, w), (fx.get("u"), fx.get("v"), fx.get("w")))
    b = pressure_rhs(cav, u, v, w)
    x, pst = solve_pressure(cav, b, precond=precond, fixed_iters=fx.get("p"),
                            x0=p_prev if cav.warm_start else None)
    u, v, w = correct(cav, u, v, w, x)
    p = gauge(x)
    stats = {"p": pst, "u": dstats[0], "v": dstats[1], "w": dstats[2], "b": b, "x": x}
    return (u, v, w, p), stats


def simulate(cav: Cavity, state, nsteps: int, fixed_iters_per_step=None, precond="none"):
    history = []
    for s in range(nsteps):
        fx = fixed_iters_per_step[s] if fixed_iters_per_step is not None else None
        state, st = step(cav, state, fixed_iters=fx, precond=precond)
        history.append(st)
    return state, history
