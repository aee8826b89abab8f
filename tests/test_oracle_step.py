"""Pins of the oracle's time step (Sec. 3 / 3.1): invariants and exact cases."""
import numpy as np
import pytest

from oracle import fractional_step as fs
from oracle.mac import Cavity, face_positions, kinetic_energy
from oracle.operators import poisson_csr
from paper_2504_03697_gb300.synthetic import cavity_perturbation, uniform_field


def _state(cav, seed=1, amp=1e-3):
    return fs.initial_state(cav, cavity_perturbation(cav.nx, cav.ny, cav.nz, seed, amp))


def test_projection_divergence_equals_scaled_residual():
    cav = Cavity(12, 10, 8, dt=0.02, nu=0.01, lid_u=1.0)
    st = _state(cav, amp=0.05)
    for _ in range(3):
        st, info = fs.step(cav, st)
    u, v, w, _ = st
    r = info["b"].ravel() - poisson_csr(cav.nx, cav.ny, cav.nz) @ info["x"].ravel()
    div = fs.divergence_sum(u, v, w).ravel()
    s = cav.dt / (cav.rho * cav.h)
    np.testing.assert_allclose(div, -s * r, rtol=0, atol=1e-13 * np.abs(div).max() + 1e-16)
    # and therefore divergence-free to the solve tolerance
    assert np.linalg.norm(div) <= s * 1.01e-8 * np.linalg.norm(info["b"])


def test_projection_never_raises_kinetic_energy():
    cav = Cavity(10, 10, 10, dt=0.05, nu=0.0, lid_u=1.0)
    u, v, w, _ = _state(cav, seed=4, amp=0.3)
    b = fs.pressure_rhs(cav, u, v, w)
    x, st = fs.solve_pressure(cav, b)
    u2, v2, w2 = fs.correct(cav, u, v, w, x)
    e0, e1 = kinetic_energy(u, v, w), kinetic_energy(u2, v2, w2)
    assert e1 < e0
    # Pythagoras: the removed part is orthogonal to the result
    removed = kinetic_energy(u - u2, v - v2, w - w2)
    assert abs(e0 - (e1 + removed)) <= 1e-8 * e0


def test_zero_state_stays_at_rest():
    cav = Cavity(6, 6, 6, dt=0.01, nu=0.01, lid_u=0.0)
    st = fs.initial_state(cav)
    st, info = fs.step(cav, st)
    for f in st[:3]:
        assert np.all(f == 0.0)
    assert np.all(st[3] == 1.0)
    assert info["p"].iters == 0


def test_mirror_symmetry_in_z():
    """z -> L - z mirror: u, v even and w odd stay so to round-off."""
    cav = Cavity(8, 8, 8, dt=0.02, nu=0.01, lid_u=1.0)
    u, v, w = cavity_perturbation(8, 8, 8, seed=9, amp=1e-2)
    u = 0.5 * (u + u[::-1])
    v = 0.5 * (v + v[::-1])
    w = 0.5 * (w - w[::-1])
    st = (u, v, w, np.ones(cav.cell_shape))
    for _ in range(4):
        st, _ = fs.step(cav, st)
    u, v, w, p = st
    scale = max(np.abs(u).max(), np.abs(v).max(), np.abs(w).max())
    assert np.abs(u - u[::-1]).max() <= 1e-10 * scale
    assert np.abs(v - v[::-1]).max() <= 1e-10 * scale
    assert np.abs(w + w[::-1]).max() <= 1e-10 * scale
    assert np.abs(p - p[::-1]).max() <= 1e-8 * np.abs(p).max()


@pytest.mark.parametrize("comp", [0, 1, 2])
def test_sampler_reproduces_samples(comp):
    cav = Cavity(5, 7, 6, lid_u=1.3)
    f = uniform_field(cav.face_shape(comp), seed=20 + comp)
    X, Y, Z = face_positions(cav, comp)
    g = fs.interpolate(cav, f, comp, X, Y, Z)
    np.testing.assert_allclose(g, f, rtol=0, atol=1e-14)


@pytest.mark.parametrize("comp", [0, 1, 2])
def test_sampler_exact_on_linear_fields(comp):
    cav = Cavity(9, 8, 10)
    X, Y, Z = face_positions(cav, comp)
    f = 0.3 + 1.7 * X - 0.9 * Y + 2.3 * Z
    rng = np.random.default_rng(7)
    ext = cav.extent
    h = cav.h
    # points inside the region spanned by real samples (no ghost involved)
    pts = [rng.uniform(h, e - h, 500) for e in ext]
    g = fs.interpolate(cav, f, comp, *pts)
    np.testing.assert_allclose(g, 0.3 + 1.7 * pts[0] - 0.9 * pts[1] + 2.3 * pts[2], rtol=1e-13)


def test_sampler_hits_wall_values_on_walls():
    """The ghost rule makes any field equal the wall velocity on the wall:
    u = lid_u on the lid, 0 on the resting walls; v, w = 0 on their
    tangential walls."""
    cav = Cavity(6, 5, 7, lid_u=1.7)
    rng = np.random.default_rng(1)
    ext = cav.extent
    for comp in range(3):
        f = uniform_field(cav.face_shape(comp), seed=comp)
        for axis in range(3):
            if axis == comp:
                continue
            for side in (0, 1):
                pts = [rng.uniform(0.2 * e, 0.8 * e, 200) for e in ext]
                pts[axis] = np.full(200, 0.0 if side == 0 else ext[axis])
                g = fs.interpolate(cav, f, comp, *pts)
                expect = cav.lid_u if (comp == 0 and axis == 1 and side == 1) else 0.0
                np.testing.assert_allclose(g, expect, rtol=0, atol=1e-14)


def test_face_velocity_exact_on_linear_fields():
    cav = Cavity(7, 6, 5)
    coef = [(0.1, 0.5, -0.2, 0.7), (-0.3, 0.2, 0.9, -0.4), (0.6, -0.8, 0.3, 0.25)]
    fields = []
    for d in range(3):
        X, Y, Z = face_positions(cav, d)
        a, bx, by, bz = coef[d]
        fields.append(a + bx * X + by * Y + bz * Z)
    for comp in range(3):
        X, Y, Z = face_positions(cav, comp)
        m = np.ones(cav.face_shape(comp), dtype=bool)
        sl = [slice(None)] * 3
        sl[2 - comp] = 0
        m[tuple(sl)] = False
        sl[2 - comp] = -1
        m[tuple(sl)] = False
        K, J, I = np.nonzero(m)
        vel = fs.face_velocity(cav, fields, comp, I, J, K)
        for d in range(3):
            a, bx, by, bz = coef[d]
            expect = a + bx * X[K, J, I] + by * Y[K, J, I] + bz * Z[K, J, I]
            np.testing.assert_allclose(vel[d], expect, rtol=1e-13, atol=1e-15)


def test_zero_velocity_advection_is_identity():
    cav = Cavity(6, 6, 6, dt=0.5, lid_u=1.0)
    z = [np.zeros(cav.face_shape(c)) for c in range(3)]
    out = fs.advect(cav, *z)
    for f in out:
        assert np.all(f == 0.0)


def test_uniform_flow_advects_linear_field_exactly():
    """Interior u = U0 (uniform flow) with v = w = 0: faces two cells away
    from the x walls backtrace to x - dt U0 inside the sampled region, where
    trilinear interpolation of the uniform field is exact."""
    cav = Cavity(10, 6, 6, dt=0.01, lid_u=0.0)
    u = np.zeros(cav.face_shape(0))
    u[:, :, 1:-1] = 0.8
    v = np.zeros(cav.face_shape(1))
    w = np.zeros(cav.face_shape(2))
    u2, v2, w2 = fs.advect(cav, u, v, w)
    np.testing.assert_allclose(u2[1:-1, 1:-1, 2:-2], 0.8, rtol=1e-14)
    assert np.all(v2 == 0) and np.all(w2 == 0)


@pytest.mark.parametrize("comp", [0, 1, 2])
def test_diffusion_of_sine_mode(comp):
    from tests.test_oracle_operators import sine_mode
    cav = Cavity(6, 5, 7, dt=0.05, nu=0.02, lid_u=0.0, rtol=1e-13)
    m, lam = sine_mode(cav, comp, (1, 2, 1))
    fields = [np.zeros(cav.face_shape(c)) for c in range(3)]
    fields[comp] = m
    out, stats = fs.diffuse(cav, fields)
    c = cav.nu * cav.dt / cav.h ** 2
    np.testing.assert_allclose(out[comp], m / (1 + c * lam), rtol=0, atol=1e-12)


def test_forces_touch_only_top_layer():
    cav = Cavity(4, 5, 3, dt=0.1, g=(2.0, -1.0, 0.5))
    z = [np.zeros(cav.face_shape(c)) for c in range(3)]
    u, v, w = fs.apply_forces(cav, *z)
    assert np.all(u[:, :4, 1:-1] == 0) and np.allclose(u[:, 4, 1:-1], 0.2)
    assert np.all(u[:, :, 0] == 0) and np.all(u[:, :, -1] == 0)
    assert np.allclose(v[:, 4, :], -0.1) and np.all(v[:, 5, :] == 0) and np.all(v[:, :4, :] == 0)
    assert np.allclose(w[1:-1, 4, :], 0.05) and np.all(w[0] == 0) and np.all(w[-1] == 0)


def test_backtrace_direction_and_distance():
    """Uniform u = U0 carries a field v = a X: the new v at X equals a (X -
    dt U0) (backtrace upstream by dt * velocity, the off-component velocity
    being the mean of the four u faces around each v face)."""
    cav = Cavity(12, 8, 6, dt=0.05, lid_u=0.0)
    U0, a = 0.7, 1.9
    u = np.zeros(cav.face_shape(0))
    u[:, :, 1:-1] = U0
    X, Y, Z = face_positions(cav, 1)
    v = a * X
    v[:, 0, :] = 0.0
    v[:, -1, :] = 0.0
    w = np.zeros(cav.face_shape(2))
    _, v2, _ = fs.advect(cav, u, v, w)
    # v faces whose u neighbours are interior and whose backtrace stays
    # within the sampled region (away from all walls)
    sl = (slice(1, -1), slice(2, -2), slice(2, -2))
    np.testing.assert_allclose(v2[sl], a * (X[sl] - cav.dt * U0), rtol=1e-13)


def test_midpoint_backtrace_on_a_linear_flow():
    """u = b X (v = w = 0): the explicit midpoint backtrace of a u face at X
    lands at X (1 - dt b + (dt b)^2 / 2) (trilinear sampling is exact on the
    linear field), so the advected u is b X (1 - dt b + (dt b)^2 / 2); the
    Euler backtrace gives b X (1 - dt b).  Faces away from the walls."""
    b = 1.3
    for order, factor in ((2, lambda q: 1 - q + q * q / 2), (1, lambda q: 1 - q)):
        cav = Cavity(16, 6, 6, dt=0.05, lid_u=0.0, advect_order=order)
        X, _, _ = face_positions(cav, 0)
        u = b * X
        u[:, :, 0] = 0.0
        u[:, :, -1] = 0.0
        v = np.zeros(cav.face_shape(1))
        w = np.zeros(cav.face_shape(2))
        u2, _, _ = fs.advect(cav, u, v, w)
        sl = (slice(1, -1), slice(1, -1), slice(2, -3))
        np.testing.assert_allclose(u2[sl], b * X[sl] * factor(cav.dt * b), rtol=1e-13)


def test_midpoint_equals_euler_for_uniform_flow():
    cav1 = Cavity(10, 6, 6, dt=0.02, lid_u=0.0)
    cav2 = Cavity(10, 6, 6, dt=0.02, lid_u=0.0, advect_order=2)
    u = np.zeros(cav1.face_shape(0))
    u[:, :, 1:-1] = 0.6
    X, Y, Z = face_positions(cav1, 1)
    v = 0.3 * X
    v[:, 0, :] = 0.0
    v[:, -1, :] = 0.0
    w = np.zeros(cav1.face_shape(2))
    a = fs.advect(cav1, u, v, w)
    b = fs.advect(cav2, u, v, w)
    sl = (slice(1, -1), slice(2, -2), slice(2, -2))
    np.testing.assert_allclose(b[1][sl], a[1][sl], rtol=1e-14)


def test_gauge_mean_is_one():
    cav = Cavity(8, 8, 8, dt=0.01, nu=0.01, lid_u=1.0)
    st = _state(cav)
    st, _ = fs.step(cav, st)
    assert abs(st[3].mean() - 1.0) < 1e-14


def test_warm_start_from_the_solution_takes_no_iteration():
    """A pressure solve started from its own converged solution stops at
    once; a warm-started run tracks the cold one within the solver tolerance."""
    cav = Cavity(10, 8, 6, dt=0.01, nu=0.01, lid_u=1.0, rtol=1e-10)
    st = _state(cav)
    st, stats = fs.step(cav, st)
    b = stats["b"]
    x, s1 = fs.solve_pressure(cav, b)
    x2, s2 = fs.solve_pressure(cav, b, x0=x)
    assert s1.iters > 10 and s2.iters == 0 and s2.converged
    cold = Cavity(10, 8, 6, dt=0.01, nu=0.01, lid_u=1.0, rtol=1e-10)
    warm = Cavity(10, 8, 6, dt=0.01, nu=0.01, lid_u=1.0, rtol=1e-10, warm_start=True)
    a, bst = _state(cold), _state(warm)
    it_c = it_w = 0
    for _ in range(4):
        a, sa = fs.step(cold, a)
        bst, sb = fs.step(warm, bst)
        it_c += sa["p"].iters
        it_w += sb["p"].iters
    assert it_w < it_c
    for fa, fb in zip(a, bst):
        assert np.abs(fa - fb).max() <= 1e-7 * max(1.0, np.abs(fa).max())
