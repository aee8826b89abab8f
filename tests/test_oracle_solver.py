"""Pins of the oracle's PCG (Sec. 3.1) against brute force and closed forms."""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle.krylov import cg_update, dic_precond, jacobi_precond, pcg
from oracle.operators import poisson_csr
from paper_2504_03697_gb300.synthetic import uniform_field


def _dense_zero_mean_solve(A, b):
    """Zero-mean solution of the singular Neumann system by a dense LU solve
    of the nonsingular A + 1 1^T / n (same solution when sum(b) = 0)."""
    Ad = A.toarray()
    n = Ad.shape[0]
    return np.linalg.solve(Ad + np.ones((n, n)) / n, b)


@pytest.mark.parametrize("shape", [(2, 2, 2), (1, 1, 6), (3, 4, 5), (6, 6, 6)])
def test_cg_matches_dense_pseudo_inverse(shape):
    A = poisson_csr(*shape)
    b = uniform_field(shape[::-1], seed=11).ravel()
    b -= b.mean()
    x, st = pcg(A, b, rtol=1e-14, max_iters=10000)
    assert st.converged and not st.breakdown
    ref = _dense_zero_mean_solve(A, b)
    assert np.linalg.norm(x - ref) <= 1e-12 * np.linalg.norm(ref)


def _mode(shape, k):
    nx, ny, nz = shape
    kk, jj, ii = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    m = (np.cos(np.pi * k[0] * (ii + 0.5) / nx) * np.cos(np.pi * k[1] * (jj + 0.5) / ny)
         * np.cos(np.pi * k[2] * (kk + 0.5) / nz)).ravel()
    lam = sum(4 * np.sin(np.pi * kd / (2 * nd)) ** 2 for kd, nd in zip(k, shape))
    return m, lam


def test_single_mode_one_iteration():
    shape = (12, 10, 8)
    A = poisson_csr(*shape)
    m, lam = _mode(shape, (2, 1, 3))
    x, st = pcg(A, m, rtol=1e-10)
    assert st.converged and st.iters == 1
    np.testing.assert_allclose(x, m / lam, rtol=1e-12, atol=1e-14)


def test_two_modes_two_iterations():
    shape = (12, 10, 8)
    A = poisson_csr(*shape)
    m1, l1 = _mode(shape, (2, 1, 3))
    m2, l2 = _mode(shape, (5, 0, 1))
    x, st = pcg(A, m1 + 0.5 * m2, rtol=1e-10)
    assert st.converged and st.iters == 2
    np.testing.assert_allclose(x, m1 / l1 + 0.5 * m2 / l2, rtol=1e-10, atol=1e-12)


def test_zero_rhs_zero_iterations():
    A = poisson_csr(4, 4, 4)
    x, st = pcg(A, np.zeros(64), rtol=1e-8)
    assert st.iters == 0 and st.converged and np.all(x == 0)


@pytest.mark.parametrize("n,err", [(16, 3.2e-3), (64, 2.0e-4)])
def test_manufactured_cosine(n, err):
    """p = cos(pi x) cos(pi y) cos(pi z): the sampled field is the (1,1,1)
    discrete mode, so A x = 3 pi^2 h^2 p_s has x = (3 pi^2 h^2 / lambda) p_s;
    the relative discretisation error |3 pi^2 h^2 / lambda - 1| is O(h^2)."""
    h = 1.0 / n
    c = (np.arange(n) + 0.5) * h
    Z, Y, X = np.meshgrid(c, c, c, indexing="ij")
    ps = (np.cos(np.pi * X) * np.cos(np.pi * Y) * np.cos(np.pi * Z)).ravel()
    lam = 3 * 4 * np.sin(np.pi / (2 * n)) ** 2
    A = poisson_csr(n, n, n)
    x, st = pcg(A, 3 * np.pi ** 2 * h * h * ps, rtol=1e-12)
    assert st.converged
    np.testing.assert_allclose(x, (3 * np.pi ** 2 * h * h / lam) * ps, rtol=0, atol=1e-10)
    rel = np.linalg.norm(x - ps) / np.linalg.norm(ps)
    assert abs(rel - err) < 0.05 * err


def test_polynomial_solution_second_order():
    """P = q(x) + q(y) + q(z), q = x^2 (1-x)^2 (zero normal derivative at
    both walls); -lap P = -(q''(x) + q''(y) + q''(z)).  Error ratio ~4 per
    halving of h confirms the O(h^2) discretisation."""
    errs = []
    for n in (8, 16, 32):
        h = 1.0 / n
        c = (np.arange(n) + 0.5) * h
        Z, Y, X = np.meshgrid(c, c, c, indexing="ij")
        q = lambda s: s ** 2 * (1 - s) ** 2
        qpp = lambda s: 12 * s ** 2 - 12 * s + 2
        P = (q(X) + q(Y) + q(Z)).ravel()
        f = (-(qpp(X) + qpp(Y) + qpp(Z))).ravel() * h * h
        f -= f.mean()
        x, st = pcg(poisson_csr(n, n, n), f, rtol=1e-12)
        assert st.converged
        d = (x - x.mean()) - (P - P.mean())
        errs.append(np.sqrt(np.mean(d * d)))  # RMS error (the max-norm ratio
        # reaches 4 more slowly because the wall rows are first order)
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 3.7 < r1 < 4.1 and 3.9 < r2 < 4.05


def test_dic_exact_on_tridiagonal():
    """With no fill-in to drop, DIC is the exact LDL^T factorisation, so PCG
    converges in one iteration and d equals the LDL^T pivots."""
    n = 9
    main = 2.0 + 0.3 * np.arange(n) / n
    T = sp.diags([-np.ones(n - 1), main, -np.ones(n - 1)], [-1, 0, 1], format="csr")
    apply, d = dic_precond(T)
    L = np.linalg.cholesky(T.toarray())
    np.testing.assert_allclose(d, np.diag(L) ** 2, rtol=1e-13)
    b = np.sin(np.arange(n) + 1.0)
    x, st = pcg(T, b, rtol=1e-12, precond=apply)
    assert st.converged and st.iters == 1
    np.testing.assert_allclose(x, np.linalg.solve(T.toarray(), b), rtol=1e-12)


def test_dic_pivots_on_the_neumann_pressure_matrix():
    """DIC of the 3D Neumann matrix: deep interior pivots reach the fixed
    point of d = 6 - 3/d, i.e. 3 + sqrt(6); every pivot of a small grid
    equals the textbook IC(0) computed densely (fill outside the pattern of
    A dropped); all pivots positive, so M is SPD although A is singular."""
    n = 24
    A = poisson_csr(n, n, n)
    _, d = dic_precond(A)
    assert abs(d.reshape(n, n, n)[12, 12, 12] - (3.0 + np.sqrt(6.0))) < 1e-12
    assert d.min() > 1.5
    A3 = poisson_csr(3, 4, 3)
    Ad = A3.toarray()
    m = Ad.shape[0]
    L = np.zeros((m, m))
    for i in range(m):  # IC(0): Cholesky restricted to the pattern of A
        for j in range(i + 1):
            if Ad[i, j] == 0.0:
                continue
            s = Ad[i, j] - L[i, :j] @ L[j, :j]
            L[i, j] = np.sqrt(s) if i == j else s / L[j, j]
    _, d3 = dic_precond(A3)
    # with the lower-triangle pattern of A, IC(0) = (D + L_A) D^-1/2: its diagonal squared is d
    np.testing.assert_allclose(d3, np.diag(L) ** 2, rtol=1e-13)


def test_dic_pcg_on_the_pressure_system_beats_cg():
    n = 16
    A = poisson_csr(n, n, n)
    b = np.random.default_rng(3).standard_normal(n ** 3)
    b -= b.mean()
    apply, _ = dic_precond(A)
    x, st = pcg(A, b, rtol=1e-8, precond=apply, max_iters=2000)
    _, st_cg = pcg(A, b, rtol=1e-8, max_iters=2000)
    assert st.converged and st.rel_resid <= 1e-8
    assert st.iters < 0.5 * st_cg.iters


def test_jacobi_on_diagonal_matrix_one_iteration():
    D = sp.diags(np.arange(1.0, 11.0), format="csr")
    b = np.cos(np.arange(10.0))
    x, st = pcg(D, b, rtol=1e-12, precond=jacobi_precond(D))
    assert st.iters == 1
    np.testing.assert_allclose(x, b / np.arange(1.0, 11.0), rtol=1e-14)


def test_jacobi_pcg_matches_dense():
    shape = (5, 4, 6)
    A = poisson_csr(*shape)
    b = uniform_field(shape[::-1], seed=3).ravel()
    b -= b.mean()
    x, st = pcg(A, b, rtol=1e-14, precond=jacobi_precond(A), max_iters=5000)
    assert st.converged
    ref = _dense_zero_mean_solve(A, b)
    xc = x - x.mean()
    assert np.linalg.norm(xc - ref) <= 1e-11 * np.linalg.norm(ref)


def test_fixed_iteration_replay():
    A = poisson_csr(6, 5, 4)
    b = uniform_field((4, 5, 6), seed=5).ravel()
    b -= b.mean()
    x1, s1 = pcg(A, b, rtol=1e-8)
    x2, s2 = pcg(A, b, rtol=1e-8, fixed_iters=s1.iters)
    assert s2.iters == s1.iters
    np.testing.assert_array_equal(x1, x2)


def test_cg_update_orthogonality_and_true_residual():
    """With alpha = r.r / p.Ap (p = r, first CG step) the updated residual is
    orthogonal to p and equals b - A x; the returned value is its norm^2."""
    A = poisson_csr(5, 4, 3)
    b = uniform_field((3, 4, 5), seed=21).ravel()
    b -= b.mean()
    x = np.zeros_like(b)
    r = b.copy()
    p = r.copy()
    q = A @ p
    alpha = float(r @ r) / float(p @ q)
    rr = cg_update(x, r, p, q, alpha)
    assert abs(float(p @ r)) <= 1e-13 * float(p @ p)
    assert np.allclose(r, b - A @ x, rtol=0, atol=1e-14)
    assert np.allclose(x, alpha * b, rtol=0, atol=1e-15)
    assert rr == pytest.approx(float(np.sum(r * r)), rel=1e-15)
    assert rr < float(b @ b)


# ----------------------------------------------------------------------------
# ir_cg: CG with a low-precision inner recurrence and FP64 reliable updates
# ----------------------------------------------------------------------------
def test_ir_cg_in_fp64_without_refinement_is_plain_cg():
    """With FP64 'inner' vectors, delta = 0 (refine only at convergence) and
    a nonsingular SPD matrix, the recurrence is CG's: same iteration count
    and the same iterate, bit for bit."""
    from oracle.krylov import ir_cg
    from oracle.mac import Cavity
    from oracle.operators import diffusion_csr
    cav = Cavity(6, 5, 4, dt=0.05, nu=0.3)
    H, _, mask = diffusion_csr(cav, 1)
    b = np.random.default_rng(8).standard_normal(H.shape[0])
    x_ref, st_ref = pcg(H, b, rtol=1e-10, max_iters=10000)
    x, st = ir_cg(H, b, rtol=1e-10, delta=0.0, inner=np.float64, singular=False)
    assert st.converged and st.iters == st_ref.iters and st.refinements == 1
    assert np.array_equal(x, x_ref)


@pytest.mark.parametrize("shape", [(8, 6, 5), (16, 12, 10)])
def test_ir_cg_fp32_reaches_the_fp64_tolerance(shape):
    """FP32 inner recurrence on the singular pressure system: the FP64 true
    residual meets rtol, and the zero-mean solution lies within
    2 rtol ||b|| / lambda_min of the dense solve (lambda_min from the DCT
    closed form)."""
    from oracle.krylov import ir_cg
    A = poisson_csr(*shape)
    b = uniform_field(shape[::-1], seed=12).ravel()
    b -= b.mean()
    x, st = ir_cg(A, b, rtol=1e-8, delta=0.1)
    assert st.converged and st.refinements >= 5
    assert np.linalg.norm(b - A @ x) <= 1.0001e-8 * np.linalg.norm(b)
    ref = _dense_zero_mean_solve(A, b)
    lam = min(4 * np.sin(np.pi / (2 * n)) ** 2 for n in shape)
    assert np.linalg.norm((x - x.mean()) - ref) <= 2e-8 * np.linalg.norm(b) / lam


def test_ir_cg_refinements_follow_delta():
    """Each refinement marks a fall of the residual by delta: a smaller delta
    needs fewer refinements for the same tolerance."""
    from oracle.krylov import ir_cg
    A = poisson_csr(12, 10, 8)
    b = uniform_field((8, 10, 12), seed=13).ravel()
    _, coarse = ir_cg(A, b, rtol=1e-8, delta=1e-3)
    _, fine = ir_cg(A, b, rtol=1e-8, delta=0.1)
    assert coarse.converged and fine.converged
    assert coarse.refinements < fine.refinements
    assert 6 <= fine.refinements <= 12 and coarse.refinements <= 5


def test_ir_cg_zero_rhs_and_nonsingular_fp32():
    from oracle.krylov import ir_cg
    from oracle.mac import Cavity
    from oracle.operators import diffusion_csr
    A = poisson_csr(4, 4, 4)
    x, st = ir_cg(A, np.zeros(64))
    assert st.converged and st.iters == 0 and not x.any()
    cav = Cavity(8, 7, 6, dt=0.05, nu=0.2)
    H, _, _ = diffusion_csr(cav, 0)
    b = np.random.default_rng(9).standard_normal(H.shape[0])
    x, st = ir_cg(H, b, rtol=1e-8, delta=1e-4, singular=False)
    assert st.converged
    assert np.linalg.norm(b - H @ x) <= 1.0001e-8 * np.linalg.norm(b)
    ref = np.linalg.solve(H.toarray(), b)
    assert np.linalg.norm(x - ref) <= 2e-8 * np.linalg.norm(b)  # ||H^-1|| <= 1


# ----------------------------------------------------------------------------
# ir_fpcg: flexible CG with a low-precision recurrence and FP64 reliable
# updates (the learned-preconditioner solve in mixed precision)
# ----------------------------------------------------------------------------
def _block_mean(x, shape, k):
    """Mean over k^3 blocks, repeated back onto the grid (x flat, shape x-fastest (nx, ny, nz))."""
    nx, ny, nz = shape
    g = x.reshape(nz, ny, nx)
    m = g.reshape(nz // k, k, ny // k, k, nx // k, k).mean(axis=(1, 3, 5))
    return np.repeat(np.repeat(np.repeat(m, k, 0), k, 1), k, 2).ravel()


def _smoother(shape, w=2.0):
    """M(r) = r + w B2 r: symmetric positive definite, maps zero-mean vectors
    to zero-mean vectors (block means preserve the total)."""
    return lambda r: r + w * _block_mean(r, shape, 2)


def _lam_min(shape):
    return min(4 * np.sin(np.pi / (2 * n)) ** 2 for n in shape if n > 1)


@pytest.mark.parametrize("precond", ["identity", "smoother"])
def test_ir_fpcg_in_fp64_is_flexible_cg(precond):
    """FP64 'inner' vectors and delta = 0 (refine only at convergence): the
    recurrence is fpcg's (the Polak-Ribiere beta written with the recurrence
    difference -alpha q): the same iteration count (+-1 at the threshold) and
    solutions within the rtol bound; with the identity also pcg's count."""
    from oracle.krylov import fpcg, ir_fpcg
    shape = (8, 8, 6)
    A = poisson_csr(*shape)
    b = uniform_field(shape[::-1], seed=21).ravel()
    M = (lambda r: r.copy()) if precond == "identity" else _smoother(shape)
    x, st = ir_fpcg(A, b, M, rtol=1e-10, delta=0.0, inner=np.float64)
    xf, sf = fpcg(A, b, M, rtol=1e-10)
    assert st.converged and sf.converged and st.refinements == 1 and st.plain_iters == 0
    assert abs(st.iters - sf.iters) <= 1
    bm = b - b.mean()
    bound = 2e-10 * np.linalg.norm(bm) / _lam_min(shape)
    assert np.linalg.norm((x - x.mean()) - (xf - xf.mean())) <= bound
    if precond == "identity":
        _, sp_ = pcg(A, bm, rtol=1e-10, max_iters=10000)
        assert abs(st.iters - sp_.iters) <= 1
    else:
        _, s0 = fpcg(A, b, lambda r: r.copy(), rtol=1e-10)
        assert st.iters < s0.iters  # the smoother helps


@pytest.mark.parametrize("precond", ["identity", "smoother"])
def test_ir_fpcg_fp32_reaches_the_fp64_tolerance(precond):
    from oracle.krylov import ir_fpcg
    shape = (16, 12, 8)
    A = poisson_csr(*shape)
    b = uniform_field(shape[::-1], seed=22).ravel()
    M = (lambda r: r.copy()) if precond == "identity" else _smoother(shape)
    x, st = ir_fpcg(A, b, M, rtol=1e-8, delta=0.1)
    bm = b - b.mean()
    assert st.converged and st.refinements >= 3 and st.plain_iters == 0
    assert np.linalg.norm(bm - A @ x) <= 1.0001e-8 * np.linalg.norm(bm)
    ref = _dense_zero_mean_solve(A, bm)
    assert np.linalg.norm((x - x.mean()) - ref) <= 2e-8 * np.linalg.norm(bm) / _lam_min(shape)


def test_ir_fpcg_scale_of_the_preconditioner_does_not_matter():
    from oracle.krylov import ir_fpcg
    shape = (8, 8, 6)
    A = poisson_csr(*shape)
    b = uniform_field(shape[::-1], seed=23).ravel()
    M = _smoother(shape)
    x1, s1 = ir_fpcg(A, b, M, rtol=1e-10, delta=0.0, inner=np.float64)
    x2, s2 = ir_fpcg(A, b, lambda r: -3.0 * M(r), rtol=1e-10, delta=0.0, inner=np.float64)
    assert s1.iters == s2.iters and s2.plain_iters == 0
    assert np.allclose(x1, x2, rtol=0, atol=1e-9 * np.abs(x1).max())


def test_ir_fpcg_falls_back_on_breakdown_and_stagnation():
    """A zero preconditioner gives z~.r = 0 at once (breakdown): plain CG
    from the first iteration.  A fixed vector gives beta = -1 on the second
    iteration, a zero direction (p.q = 0): plain CG from the true residual
    after one iteration.  A fresh random vector each call keeps p.q > 0 but
    does not reduce the residual: plain CG after the stagnation window.  All
    still meet the FP64 tolerance; zero b takes no iteration."""
    from oracle.krylov import ir_fpcg
    shape = (12, 10, 8)
    A = poisson_csr(*shape)
    b = uniform_field(shape[::-1], seed=24).ravel()
    bm = b - b.mean()
    x, st = ir_fpcg(A, b, lambda r: np.zeros_like(r), rtol=1e-8)
    assert st.converged and st.plain_iters == st.iters > 0
    fixed = uniform_field(shape[::-1], seed=25).ravel()
    x, st = ir_fpcg(A, b, lambda r: fixed.copy(), rtol=1e-8)
    assert st.converged and st.iters - st.plain_iters == 1
    assert np.linalg.norm(bm - A @ x) <= 1.0001e-8 * np.linalg.norm(bm)
    rng = np.random.default_rng(26)
    x, st = ir_fpcg(A, b, lambda r: rng.standard_normal(r.size), rtol=1e-8, stagnation=20)
    assert st.converged and 0 < st.plain_iters < st.iters and st.iters - st.plain_iters >= 20
    assert np.linalg.norm(bm - A @ x) <= 1.0001e-8 * np.linalg.norm(bm)
    x, st = ir_fpcg(A, np.zeros(A.shape[0]), lambda r: r.copy())
    assert st.converged and st.iters == 0 and not x.any()


def test_ir_cg_starting_iterate():
    """x0 = 0 is the cold start (bitwise); x0 = a solution within the
    tolerance takes no iteration; x0 = a partial CG iterate needs fewer
    iterations than the cold start."""
    from oracle.krylov import ir_cg
    shape = (12, 10, 8)
    A = poisson_csr(*shape)
    b = uniform_field(shape[::-1], seed=27).ravel()
    x1, s1 = ir_cg(A, b, rtol=1e-8)
    x2, s2 = ir_cg(A, b, rtol=1e-8, x0=np.zeros(b.size))
    assert np.array_equal(x1, x2) and s1.iters == s2.iters and s1.refinements == s2.refinements
    bm = b - b.mean()
    xs, _ = pcg(A, bm, rtol=1e-12, max_iters=10000)
    x3, s3 = ir_cg(A, b, rtol=1e-8, x0=xs)
    assert s3.converged and s3.iters == 0 and np.array_equal(x3, xs)
    xp, _ = pcg(A, bm, rtol=1e-15, max_iters=20)
    _, s4 = ir_cg(A, b, rtol=1e-8, x0=xp)
    assert s4.converged and s4.iters < s1.iters
