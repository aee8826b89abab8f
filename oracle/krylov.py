"""Preconditioned conjugate gradients, textbook form (oracle, FP64).

Sec. 3.1 of the paper: the pressure system is solved by a Preconditioned
Conjugate Gradient (PCG) solver with either a simplified Diagonal-based
Incomplete Cholesky (DIC) or a Jacobi preconditioner; Table 1 names the
pieces (spmv, precondition, dot, vector add/scale).  This module writes out
Hestenes-Stiefel PCG with ``numpy.dot`` for the inner products and the CSR
SpMV of ``operators``.

Stopping rule (the paper defines none; reading): stop when the recurrence
residual satisfies ||r|| <= rtol ||b||, then recompute the true residual
b - A x; if it also passes, the solve has converged, otherwise CG restarts
from the true residual (p = M^-1 r).  ||b|| = 0 returns x = 0 after zero
iterations.  The iteration cap counts CG iterations (SpMVs with p).

``fixed_iters`` replays a given number of iterations with no stopping test;
parity tests use it to follow the iteration counts of the CUDA path, because
two correct CGs whose sums run in different orders may stop one iteration
apart.

DIC reading: d_i = a_ii - sum_{j < i, a_ij != 0} a_ij^2 / d_j and
M = (D + L) D^-1 (D + L^T) with L the strict lower triangle of A (the
"simplified" form keeps the sparsity of A).  The incomplete factor drops
the fill that would make the last pivot of the singular Neumann pressure
matrix vanish, so every pivot stays positive (deep in the interior the
pivots approach 3 + sqrt(6), about 5.449, the fixed point of d = 6 - 3/d)
and M is SPD; DIC applies to the pressure system directly.

Pins (tests/test_oracle_solver.py): dense pseudo-inverse solves on grids up
to 6^3, exactly one iteration for a single DCT mode and two for two modes,
the manufactured cosine solution in closed form, the O(h^2) rate on a
polynomial solution, and DIC = exact factorisation on tridiagonal matrices
(one PCG iteration).  ``cg_update`` is the step every ``pcg`` iteration
takes, so those pins cover it; tests/test_oracle_solver.py also checks that
with alpha = r.r / p.Ap it leaves r orthogonal to p and equal to b - A x.

``ir_cg`` (the mixed-precision solve: the same CG with its recurrence in
FP32 and FP64 reliable updates) is pinned by tests/test_oracle_solver.py:
with FP64 inner vectors and no refinement before convergence it takes
``pcg``'s iterates bit for bit on an SPD matrix; in FP32 it meets the FP64
true-residual tolerance and lies within 2 rtol ||b|| / lambda_min of the
dense solve of the pressure system (within 2 rtol ||b|| for I + c L); a
smaller refinement factor needs fewer refinements; x0 = 0 reproduces the
cold start bit for bit and x0 = the solution takes no iteration.

``fpcg`` (flexible PCG for a preconditioner that may vary between
iterations) is pinned by tests/test_oracle_unet.py: with M = identity or a
fixed SPD M it takes the iterates of ``pcg`` (the Polak-Ribiere beta equals
the Fletcher-Reeves one when z_{k+1}.r_k = 0), M = -I gives the same iterates
as M = I (flexible CG is invariant to the preconditioner's scale), with M =
the exact inverse on the zero-mean subspace it converges in one iteration,
and a preconditioner returning zero (breakdown) or a fixed vector
(stagnation) makes it fall back to plain CG and still converge.

``ir_fpcg`` (flexible CG with its recurrence in FP32 and FP64 reliable
updates: the learned-preconditioner solve in mixed precision) is pinned by
tests/test_oracle_solver.py: with FP64 inner vectors and no refinement
before convergence it takes the iteration counts and the solution of
``pcg`` with the identity and with a fixed SPD diagonal preconditioner, and
of ``fpcg`` with the same preconditioner; in FP32 it meets the FP64
true-residual tolerance and lies within 2 rtol ||b|| / lambda_min of the
dense solve; M and -3 M give the same iterates in FP64; a zero
preconditioner (breakdown) or an input-independent one (stagnation) makes
it fall back to plain CG and still converge.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg  # noqa: F401  (spsolve_triangular)


@dataclass
class SolveStats:
    iters: int = 0
    restarts: int = 0
    converged: bool = False
    breakdown: bool = False
    rel_resid: float = 0.0   # true ||b - A x|| / ||b|| at exit


def identity_precond(r):
    return r.copy()


def jacobi_precond(A: sp.csr_matrix):
    inv_d = 1.0 / A.diagonal()
    return lambda r: inv_d * r


def dic_precond(A: sp.csr_matrix):
    """Simplified diagonal-based incomplete Cholesky (Sec. 3.1), sequential."""
    A = A.tocsr()
    n = A.shape[0]
    d = np.zeros(n)
    indptr, indices, data = A.indptr, A.indices, A.data
    for i in range(n):
        s = 0.0
        aii = 0.0
        for t in range(indptr[i], indptr[i + 1]):
            j = indices[t]
            if j < i:
                s += data[t] * data[t] / d[j]
            elif j == i:
                aii = data[t]
        d[i] = aii - s
    lower = sp.tril(A, k=-1).tocsr()
    DL = (sp.diags(d) + lower).tocsr()
    DU = (sp.diags(d) + lower.T).tocsr()

    def apply(r):
        y = sp.linalg.spsolve_triangular(DL, r, lower=True)
        return sp.linalg.spsolve_triangular(DU, d * y, lower=False)

    return apply, d


def cg_update(x, r, p, q, alpha):
    """The vector step of a CG iteration (Table 1: vector add / scale, dot):
    x <- x + alpha p and r <- r - alpha q in place; returns r.r of the new r."""
    x += alpha * p
    r -= alpha * q
    return float(np.dot(r, r))


def pcg(A, b, x0=None, rtol=1e-8, max_iters=1000, precond=identity_precond,
        fixed_iters=None, max_restarts=8):
    """Solve A x = b; returns (x, SolveStats)."""
    n = b.size
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=np.float64, copy=True)
    st = SolveStats()
    bb = float(np.dot(b, b))
    if bb == 0.0:
        st.converged = True
        return np.zeros(n), st
    tol2 = rtol * rtol * bb
    r = b - A @ x
    z = precond(r)
    p = z.copy()
    rz = float(np.dot(r, z))
    rr = float(np.dot(r, r))
    while True:
        if fixed_iters is not None:
            if st.iters == fixed_iters:
                break
        else:
            if rr <= tol2:
                rt = b - A @ x
                rrt = float(np.dot(rt, rt))
                if rrt <= tol2:
                    st.converged = True
                    break
                st.restarts += 1
                if st.restarts > max_restarts:
                    break
                r = rt
                z = precond(r)
                p = z.copy()
                rz = float(np.dot(r, z))
                rr = rrt
            if st.iters == max_iters:
                break
        q = A @ p
        pq = float(np.dot(p, q))
        if not pq > 0.0:
            st.breakdown = True
            break
        alpha = rz / pq
        rr = cg_update(x, r, p, q, alpha)
        z = precond(r)
        rz_new = float(np.dot(r, z))
        beta = rz_new / rz
        rz = rz_new
        p = z + beta * p
        st.iters += 1
    st.rel_resid = float(np.linalg.norm(b - A @ x) / np.sqrt(bb))
    return x, st


@dataclass
class FlexStats:
    iters: int = 0
    plain_iters: int = 0      # iterations after the switch to plain CG
    restarts: int = 0
    converged: bool = False
    fell_back: bool = False
    rel_resid: float = 0.0


def fpcg(A, b, precond, rtol=1e-8, max_iters=1000, stagnation=50, max_restarts=8):
    """Flexible PCG with the Polak-Ribiere beta (learned preconditioner, a
    reading of the paper's "other preconditioners", Sec. 5).

    b has its mean removed first (Neumann system, consistent right-hand side).
    One iteration: q = A p, alpha = (r.z)/(p.q), x += alpha p, r -= alpha q,
    z' = M(r), beta = z'.(r_new - r_old)/(r_old.z_old), p = z' + beta p.
    A preconditioner that is not positive definite may give z.r < 0; alpha
    then is negative and still the exact line search along p (r.p = r.z), so
    only z.r = 0, a non-positive p.q or a non-finite value is a breakdown.
    A breakdown, or `stagnation` iterations without the residual norm
    halving, switches to plain CG (M = identity) restarted from the true
    residual of the current x.  Convergence is judged by the
    true residual ||b - A x|| <= rtol ||b||; when the recurrence passes but
    the true residual does not, the iteration restarts from it.
    Returns (x, FlexStats)."""
    b = b - b.mean()
    n = b.size
    st = FlexStats()
    bb = float(np.dot(b, b))
    x = np.zeros(n)
    if bb == 0.0:
        st.converged = True
        return x, st
    tol2 = rtol * rtol * bb
    plain = False
    M = precond

    def start():
        r = b - A @ x
        z = r.copy() if plain else M(r)
        return r, z, z.copy(), float(np.dot(z, r))

    r, z, p, rz = start()
    best = bb
    since = 0
    while True:
        bad = not (rz != 0.0 and np.isfinite(rz))
        if not bad:
            if st.iters >= max_iters:
                break
            q = A @ p
            pq = float(np.dot(p, q))
            bad = not (pq > 0.0 and np.isfinite(pq))
        if bad:
            if plain:
                break
            plain = True
            st.fell_back = True
            st.restarts += 1
            r, z, p, rz = start()
            continue
        alpha = rz / pq
        x = x + alpha * p
        r_old = r
        r = r - alpha * q
        st.iters += 1
        if plain:
            st.plain_iters += 1
        rr = float(np.dot(r, r))
        if rr <= tol2:
            rt = b - A @ x
            if float(np.dot(rt, rt)) <= tol2:
                st.converged = True
                break
            st.restarts += 1
            if st.restarts > max_restarts:
                break
            r = rt
            z = r.copy() if plain else M(r)
            p = z.copy()
            rz = float(np.dot(z, r))
            continue
        if rr < 0.25 * best:
            best, since = rr, 0
        else:
            since += 1
            if not plain and since >= stagnation:
                plain = True
                st.fell_back = True
                st.restarts += 1
                r, z, p, rz = start()
                continue
        z_new = r.copy() if plain else M(r)
        rz_new = float(np.dot(z_new, r))
        beta = float(np.dot(z_new, r - r_old)) / rz
        rz = rz_new
        z = z_new
        p = z + beta * p
    st.rel_resid = float(np.linalg.norm(b - A @ x) / np.sqrt(bb))
    return x, st


@dataclass
class IrStats:
    iters: int = 0            # inner (low-precision) CG iterations
    refinements: int = 0      # FP64 true-residual replacements
    converged: bool = False
    breakdown: bool = False
    rel_resid: float = 0.0    # true ||b - A x|| / ||b|| at exit


def ir_cg(A, b, rtol=1e-8, delta=0.1, max_iters=10000, max_outer=1000, inner=np.float32, singular=True, x0=None):
    """CG with an inner recurrence in a lower precision and FP64 reliable
    updates (the mixed-precision solve of the pressure and diffusion systems:
    Sec. 3.1's CG with its vectors, operator and recurrence in `inner`).

    The FP64 state is x and the true residual r = b - A x.  A refinement
    loads the recurrence residual from it, r_in = r (minus its mean when the
    system is singular, the Neumann pressure matrix), and starts an inner
    correction x_in = 0.  Each inner iteration, all vectors and the operator
    in `inner` precision, the inner products summed in FP64:
        p = r_in + beta p,  q = A p,  alpha = rz / p.q,
        x_in += alpha p,  r_in -= alpha q,  rz' = r_in.r_in.
    When rz' has fallen by delta^2 below the true residual of the last
    refinement (or below rtol^2 ||b||^2) the correction is added to x in
    FP64, the true residual is recomputed, and the next direction keeps p
    with beta = (new r_in . r_in) / rz (the residual it replaces).
    Otherwise beta = rz' / rz.  Convergence is declared on the FP64 true
    residual only.  b has its mean removed first when `singular`.  x0
    (optional) is the starting iterate (the first true residual is
    b - A x0); by default 0.  Returns (x, IrStats)."""
    A64 = A.astype(np.float64)
    Ain = A.astype(inner)
    b = np.asarray(b, dtype=np.float64)
    if singular:
        b = b - b.mean()
    st = IrStats()
    n = b.size
    x = np.zeros(n)
    bb = float(np.dot(b, b))
    if bb == 0.0:
        st.converged = True
        return x, st
    tol2 = rtol * rtol * bb
    if x0 is not None:
        x = np.array(x0, dtype=np.float64, copy=True).ravel()
    r = b - A64 @ x if x0 is not None else b.copy()
    rr = float(np.dot(r, r))
    p = np.zeros(n, dtype=inner)
    rz = 0.0
    beta = 0.0
    first = True
    while True:
        # refinement point: judge, then restart the inner recurrence
        if rr <= tol2:
            st.converged = True
            break
        if st.refinements > max_outer or st.iters >= max_iters:
            break
        r_in = (r - r.mean() if singular else r).astype(inner)
        x_in = np.zeros(n, dtype=inner)
        rz_new = float(np.dot(r_in.astype(np.float64), r_in.astype(np.float64)))
        if not first:
            beta = rz_new / rz
        rz = rz_new
        rz_ref = rr
        refine = False
        while st.iters < max_iters:
            p = (r_in if first else r_in + inner(beta) * p).astype(inner)
            q = (Ain @ p).astype(inner)
            pq = float(np.dot(p.astype(np.float64), q.astype(np.float64)))
            if not (pq > 0.0) or not np.isfinite(pq):
                st.breakdown = True
                break
            alpha = inner(rz / pq)
            x_in = (x_in + alpha * p).astype(inner)
            r_in = (r_in - alpha * q).astype(inner)
            rz_new = float(np.dot(r_in.astype(np.float64), r_in.astype(np.float64)))
            first = False
            st.iters += 1
            if rz_new <= delta * delta * rz_ref or rz_new <= tol2:
                refine = True
                break
            beta = rz_new / rz
            rz = rz_new
        x = x + x_in.astype(np.float64)
        r = b - A64 @ x
        rr = float(np.dot(r, r))
        if not refine:
            break
        st.refinements += 1
    st.converged = st.converged or rr <= tol2
    st.rel_resid = float(np.sqrt(rr / bb))
    return x, st


@dataclass
class FlexIrStats:
    iters: int = 0            # inner (low-precision) flexible-CG iterations
    refinements: int = 0      # FP64 true-residual replacements
    plain_iters: int = 0      # iterations run as plain CG after a fall-back
    converged: bool = False
    breakdown: bool = False
    rel_resid: float = 0.0    # true ||b - A x|| / ||b|| at exit


def ir_fpcg(A, b, precond, rtol=1e-8, delta=0.1, max_iters=10000, max_outer=1000, stagnation=50,
            inner=np.float32):
    """Flexible CG (Polak-Ribiere) with its recurrence in a lower precision
    and FP64 reliable updates: the learned-preconditioner pressure solve in
    mixed precision (``fpcg`` in the precision split of ``ir_cg``).

    The FP64 state is x and the true residual r = b - A x (b has its mean
    removed; the Neumann pressure system).  A refinement loads r_in = r -
    mean(r) in `inner` precision and a zero correction x_in.  Each inner
    iteration, vectors and operator in `inner` precision, inner products
    summed in FP64:
        z = M(r_in) (r_in itself once running as plain CG), z~ = z - mean(z),
        beta = -alpha_old z~.q_old / (z~.r)_old   (0 for a new direction),
        p = z~ + beta p,  q = A p,  alpha = z~.r_in / p.q,
        x_in += alpha p,  r_in -= alpha q.
    -alpha_old q_old is r_new - r_old, so beta is the Polak-Ribiere one; after
    a refinement it is formed the same way (the direction is kept).  When
    r_in.r_in has fallen by delta^2 below the true residual of the last
    refinement (or below rtol^2 ||b||^2) the correction is added to x in
    FP64 and the true residual recomputed.  z~.r_in = 0 (or a non-finite
    value) switches to plain CG along r_in; a direction with p.q <= 0 (or
    `stagnation` iterations without the residual norm halving) switches to
    plain CG from the next true residual (a refinement, then a new
    direction).  Convergence only on the
    FP64 true residual.  Returns (x, FlexIrStats)."""
    A64 = A.astype(np.float64)
    Ain = A.astype(inner)
    b = np.asarray(b, dtype=np.float64)
    b = b - b.mean()
    n = b.size
    st = FlexIrStats()
    x = np.zeros(n)
    bb = float(np.dot(b, b))
    if bb == 0.0:
        st.converged = True
        return x, st

    def dot(u, v):
        return float(np.dot(u.astype(np.float64), v.astype(np.float64)))

    tol2 = rtol * rtol * bb
    r = b.copy()
    rr = bb
    p = np.zeros(n, dtype=inner)
    q_old = np.zeros(n, dtype=inner)
    alpha = zr = best = 0.0
    first, plain, since = True, False, 0
    while True:
        if rr <= tol2:
            st.converged = True
            break
        if st.refinements > max_outer or st.iters >= max_iters:
            break
        r_in = (r - r.mean()).astype(inner)
        x_in = np.zeros(n, dtype=inner)
        rz_ref = rr
        if st.iters == 0:
            best = dot(r_in, r_in)
        refine = False
        while st.iters < max_iters:
            z = r_in if plain else np.asarray(precond(r_in.astype(np.float64))).astype(inner)
            m = float(np.sum(z.astype(np.float64))) / n
            zr_new = dot(z, r_in) - m * float(np.sum(r_in.astype(np.float64)))
            zq = 0.0 if first else dot(z, q_old) - m * float(np.sum(q_old.astype(np.float64)))
            if not plain and not (zr_new != 0.0 and np.isfinite(zr_new) and np.isfinite(zq)):
                plain, first = True, True  # the preconditioner's step is unusable
                z = r_in
                m = float(np.sum(r_in.astype(np.float64))) / n
                zr_new = dot(r_in, r_in) - m * float(np.sum(r_in.astype(np.float64)))
                zq = 0.0
            if not (zr_new != 0.0 and np.isfinite(zr_new)):
                st.breakdown = True
                break
            beta = 0.0 if first else -alpha * zq / zr
            zr = zr_new
            zc = (z.astype(np.float64) - m).astype(inner)
            p = zc if first else (zc + inner(beta) * p).astype(inner)
            q = (Ain @ p).astype(inner)
            pq = dot(p, q)
            if not (pq > 0.0) or not np.isfinite(pq):
                if plain:
                    st.breakdown = True
                    break
                plain, first, refine = True, True, True  # no usable flexible step:
                break                                    # plain CG from the true residual
            alpha = zr / pq
            x_in = (x_in + inner(alpha) * p).astype(inner)
            r_in = (r_in - inner(alpha) * q).astype(inner)
            q_old = q
            rr_new = dot(r_in, r_in)
            first = False
            st.iters += 1
            if plain:
                st.plain_iters += 1
            restart = False
            if rr_new < 0.25 * best:
                best, since = rr_new, 0
            elif not plain:
                since += 1
                if since >= stagnation:
                    plain, first, restart = True, True, True
            if restart or rr_new <= delta * delta * rz_ref or rr_new <= tol2:
                refine = True
                break
        x = x + x_in.astype(np.float64)
        r = b - A64 @ x
        rr = float(np.dot(r, r))
        if not refine:
            break
        st.refinements += 1
    st.converged = st.converged or rr <= tol2
    st.rel_resid = float(np.sqrt(rr / bb))
    return x, st
