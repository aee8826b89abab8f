"""GPU checks of the FP32-inner / FP64-refined pressure solve (CFD_SOLVER_IR).

The refined path is judged like every solve here: by the true FP64
residual ||b - A x|| <= rtol ||b|| (recomputed on the host with the oracle's
CSR matrix), and its solution is compared with the oracle's FP64 CG within
the bound both rtol-solutions obey: ||x_ir - x_oracle||_2 <= 2 rtol ||b||_2
/ lambda_min, lambda_min = min_d 4 sin^2(pi / (2 n_d)) being the smallest
nonzero eigenvalue of A (the comparison removes the null-space mean).  The
velocity after a projection then differs by at most 2 dt/(rho h) times the
pressure difference.  Per-field max-abs errors are printed for the record.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import fractional_step as fs  # noqa: E402
from oracle.krylov import pcg  # noqa: E402
from oracle.mac import Cavity as OCav  # noqa: E402
from oracle.operators import poisson_csr  # noqa: E402
from paper_2504_03697_gb300.synthetic import gaussian_rhs, uniform_field  # noqa: E402

pytestmark = pytest.mark.gpu

ITERS_PER_PASS = 4  # FP32 iterations per pass of the graph form's inner loop body


def assert_graph_kernels(ran, base, st):
    """Kernels a graph-form solve ran: `base` (2 per FP32 iteration plus the
    fixed ones) and, per inner loop (at most one per refinement plus the
    first), the 2 (ITERS_PER_PASS - 1) or fewer kernels of its last pass
    that return at once because the loop was left."""
    extra = ran - base
    assert extra % 2 == 0 and 0 <= extra <= 2 * (ITERS_PER_PASS - 1) * (st["outer_iters"] + 1), (ran, base, st)


@pytest.fixture(scope="module")
def cfd():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2504_03697_gb300 import build as B
    B.build()
    from paper_2504_03697_gb300 import cfd as _cfd
    return _cfd


def lam_min(shape):
    return min(4 * np.sin(np.pi / (2 * n)) ** 2 for n in shape if n > 1)


@pytest.mark.parametrize("shape,delta", [((48, 40, 32), 0.0), ((17, 9, 13), 0.0), ((64, 64, 64), 0.01),
                                         ((33, 31, 30), 0.3), ((1, 1, 9), 0.0)])
def test_ir_solve_true_residual_and_bound(cfd, shape, delta):
    nx, ny, nz = shape
    cav = cfd.Cavity(cfd.make_params(nx, ny, nz, solver="ir", ir_delta=delta))
    b = gaussian_rhs(nx, ny, nz, seed=4)
    bg = torch.tensor(b, device="cuda")
    xg = torch.zeros_like(bg)
    rc, st = cav.solve_pressure(bg, xg)
    assert rc == cfd.CFD_OK, st
    assert st["outer_iters"] >= 1 and st["rel_resid"] <= 1e-8
    A = poisson_csr(nx, ny, nz)
    x = xg.cpu().numpy().ravel()
    bo = b.ravel() - b.mean()
    true_rel = np.linalg.norm(bo - A @ x) / np.linalg.norm(bo)
    assert true_rel <= 1.0001e-8, true_rel
    xo, so = pcg(A, bo, rtol=1e-8, max_iters=10 ** 6)
    d = (x - x.mean()) - (xo - xo.mean())
    bound = 2 * 1e-8 * np.linalg.norm(bo) / lam_min(shape)
    assert np.linalg.norm(d) <= bound, (np.linalg.norm(d), bound)
    print(f"IR {shape}: inner {st['iters']} outer {st['outer_iters']} (FP64 CG {so.iters}), "
          f"max|dx| {np.abs(d).max():.2e}, true rel resid {true_rel:.2e}")


def test_ir_projection_fields_within_bound(cfd):
    shape = (24, 20, 16)
    nx, ny, nz = shape
    cav = cfd.Cavity(cfd.make_params(nx, ny, nz, solver="ir", dt=0.02, lid_u=1.0))
    ocav = OCav(nx, ny, nz, dt=0.02, lid_u=1.0)
    f = []
    for c in range(3):
        a = uniform_field(ocav.face_shape(c), seed=6, stream=c)
        ax = 2 - c
        sl = [slice(None)] * 3
        sl[ax] = 0
        a[tuple(sl)] = 0.0
        sl[ax] = -1
        a[tuple(sl)] = 0.0
        f.append(a)
    for name, a in zip("uvw", f):
        cav.set_field(name, a)
    rc, st = cav.substep("project")
    assert rc == cfd.CFD_OK and st["rel_resid"] <= 1e-8
    b = fs.pressure_rhs(ocav, *f)
    x, _ = fs.solve_pressure(ocav, b)
    ref_u = fs.correct(ocav, *f, x)
    p_gpu = cav.read_field("p").numpy()
    p_ref = fs.gauge(x)
    pbound = 2 * 1e-8 * np.linalg.norm(b) / lam_min(shape)
    dp = np.linalg.norm((p_gpu - p_gpu.mean()) - (p_ref - p_ref.mean()))
    assert dp <= pbound
    s = ocav.dt / (ocav.rho * ocav.h)
    errs = {"p": float(np.abs(p_gpu - p_ref).max())}
    for c, name in enumerate("uvw"):
        g = cav.read_field(name).numpy()
        errs[name] = float(np.abs(g - ref_u[c]).max())
        assert errs[name] <= 2 * s * pbound
    u, v, w = (cav.read_field(n).numpy() for n in "uvw")
    assert np.linalg.norm(fs.divergence_sum(u, v, w)) <= s * 1.01e-8 * np.linalg.norm(b)
    print("IR projection max-abs errors vs FP64 oracle:", errs)


def test_ir_cavity_steps_converge(cfd):
    cav = cfd.Cavity(cfd.make_params(32, 32, 32, solver="ir", dt=0.01, nu=0.001, lid_u=1.0))
    rc, stats = cav.step(5)
    assert rc == cfd.CFD_OK
    assert all(s["rel_resid"] <= 1e-8 and s["outer_iters"] >= 1 for s in stats[1:])


# ----------------------------------------------------------------------------
# graph form (cfd_set_ir_form GRAPH): the same method as device-side loops
# over streaming kernels; judged by the same rules
# ----------------------------------------------------------------------------
def _graph_cavity(cfd, shape, form="graph", **kw):
    cav = cfd.Cavity(cfd.make_params(*shape, solver="ir", **kw))
    cav.set_ir_form(form)
    return cav


def _check_solution(shape, b, x, st, rtol=1e-8):
    nx, ny, nz = shape
    A = poisson_csr(nx, ny, nz)
    bo = b.ravel() - b.mean()
    true_rel = np.linalg.norm(bo - A @ x) / np.linalg.norm(bo)
    assert true_rel <= rtol * 1.0001, true_rel
    np.testing.assert_allclose(true_rel, st["rel_resid"], rtol=1e-6, atol=1e-14)
    xo, so = pcg(A, bo, rtol=rtol, max_iters=10 ** 6)
    d = (x - x.mean()) - (xo - xo.mean())
    bound = 2 * rtol * np.linalg.norm(bo) / lam_min(shape)
    assert np.linalg.norm(d) <= bound, (np.linalg.norm(d), bound)
    return so


@pytest.mark.parametrize("shape,delta", [((48, 40, 32), 0.0), ((64, 64, 64), 0.01), ((36, 20, 19), 0.3),
                                         ((128, 24, 16), 0.0), ((4, 9, 5), 0.0), ((4, 1, 1), 0.0)])
def test_ir_graph_true_residual_and_bound(cfd, shape, delta):
    nx, ny, nz = shape
    cav = _graph_cavity(cfd, shape, ir_delta=delta)
    b = gaussian_rhs(nx, ny, nz, seed=4)
    bg = torch.tensor(b, device="cuda")
    xg = torch.zeros_like(bg)
    l0 = cav.launch_count()
    rc, st = cav.solve_pressure(bg, xg)
    assert rc == cfd.CFD_OK, st
    assert st["outer_iters"] >= 1
    so = _check_solution(shape, b, xg.cpu().numpy().ravel(), st)
    # kernels the graph ran: prologue 2, each outer pass 2, each FP32
    # iteration 2, epilogue 3 (the loop structure as designed), plus the
    # kernels left over in the last pass of each inner loop (4 iterations
    # per pass of its body: at most 6 per inner loop)
    assert_graph_kernels(cav.launch_count() - l0, 2 + 2 * (st["outer_iters"] + 1) + 2 * st["iters"] + 3, st)
    print(f"IR graph {shape}: inner {st['iters']} outer {st['outer_iters']} (FP64 CG {so.iters})")


def test_ir_graph_matches_persistent_and_repeats_bitwise(cfd):
    shape = (64, 48, 40)
    nx, ny, nz = shape
    b = gaussian_rhs(nx, ny, nz, seed=9)
    bg = torch.tensor(b, device="cuda")
    out = {}
    for form in ("persistent", "graph", "graph"):
        cav = _graph_cavity(cfd, shape, form=form)
        xg = torch.zeros_like(bg)
        rc, st = cav.solve_pressure(bg, xg)
        assert rc == cfd.CFD_OK
        out.setdefault(form, []).append((xg.cpu().numpy().ravel(), st))
    xp, sp = out["persistent"][0]
    (xg1, sg1), (xg2, sg2) = out["graph"]
    assert np.array_equal(xg1, xg2) and sg1 == sg2
    bound = 4 * 1e-8 * np.linalg.norm(b.ravel() - b.mean()) / lam_min(shape)
    assert np.linalg.norm((xg1 - xg1.mean()) - (xp - xp.mean())) <= bound
    assert abs(sg1["iters"] - sp["iters"]) <= max(3, sp["iters"] // 20)


def test_ir_graph_warm_start_and_projection(cfd):
    """The projection substep (warm start from p, gauge to mean 1) in the
    graph form, against the FP64 oracle within the rtol bound."""
    shape = (24, 20, 16)
    nx, ny, nz = shape
    cav = _graph_cavity(cfd, shape, dt=0.02, lid_u=1.0, warm_start=True)
    ocav = OCav(nx, ny, nz, dt=0.02, lid_u=1.0)
    f = []
    for c in range(3):
        a = uniform_field(ocav.face_shape(c), seed=8, stream=c)
        ax = 2 - c
        sl = [slice(None)] * 3
        sl[ax] = 0
        a[tuple(sl)] = 0.0
        sl[ax] = -1
        a[tuple(sl)] = 0.0
        f.append(a)
    for name, a in zip("uvw", f):
        cav.set_field(name, a)
    cav.set_field("p", 1.0 + 0.1 * uniform_field((nz, ny, nx), seed=2))
    rc, st = cav.substep("project")
    assert rc == cfd.CFD_OK and st["rel_resid"] <= 1e-8
    b = fs.pressure_rhs(ocav, *f)
    x, _ = fs.solve_pressure(ocav, b)
    p_gpu = cav.read_field("p").numpy()
    assert abs(p_gpu.mean() - 1.0) <= 1e-12
    pbound = 2 * 1e-8 * np.linalg.norm(b) / lam_min(shape)
    assert np.linalg.norm((p_gpu - p_gpu.mean()) - (x - x.mean())) <= pbound
    u, v, w = (cav.read_field(n).numpy() for n in "uvw")
    s = ocav.dt / (ocav.rho * ocav.h)
    assert np.linalg.norm(fs.divergence_sum(u, v, w)) <= s * 1.01e-8 * np.linalg.norm(b)


def test_ir_graph_edge_cases(cfd):
    shape = (16, 12, 10)
    nx, ny, nz = shape
    # zero right-hand side: no iteration, x = 0
    cav = _graph_cavity(cfd, shape)
    bg = torch.zeros((nz, ny, nx), dtype=torch.float64, device="cuda")
    xg = torch.full_like(bg, 5.0)
    rc, st = cav.solve_pressure(bg, xg)
    assert rc == cfd.CFD_OK and st["iters"] == 0 and st["rel_resid"] == 0.0
    assert torch.count_nonzero(xg).item() == 0
    # iteration cap: not converged, x holds the folded last iterate whose
    # true residual is the one reported
    cav = _graph_cavity(cfd, shape, max_iters=7)
    b = gaussian_rhs(nx, ny, nz, seed=5)
    bg = torch.tensor(b, device="cuda")
    xg = torch.zeros_like(bg)
    rc, st = cav.solve_pressure(bg, xg)
    assert rc == cfd.CFD_ERR_NOT_CONVERGED and st["iters"] == 7
    A = poisson_csr(nx, ny, nz)
    bo = b.ravel() - b.mean()
    true_rel = np.linalg.norm(bo - A @ xg.cpu().numpy().ravel()) / np.linalg.norm(bo)
    np.testing.assert_allclose(true_rel, st["rel_resid"], rtol=1e-9)
    assert 1e-8 < true_rel < 1.0
    # the returned x is the 7th CG iterate itself: the update kernels defer
    # every other iteration's x32 term, and a cap after an odd number of
    # iterations leaves one pending, which the passes after the loop must add
    # (one missing term alpha p moves x by far more than the FP32 rounding)
    for cap in (7, 8):
        cav = _graph_cavity(cfd, shape, max_iters=cap)
        xg = torch.zeros_like(bg)
        rc, st = cav.solve_pressure(bg, xg)
        assert rc == cfd.CFD_ERR_NOT_CONVERGED and st["iters"] == cap
        x_cap, _ = pcg(A, bo, rtol=1e-8, max_iters=10 ** 6, fixed_iters=cap)
        err = np.abs(xg.cpu().numpy().ravel() - x_cap).max() / np.abs(x_cap).max()
        assert err < 1e-4, (cap, err)
    # a NaN in b: breakdown reported, no hang
    cav = _graph_cavity(cfd, shape)
    b[3, 4, 5] = np.nan
    bg = torch.tensor(b, device="cuda")
    rc, st = cav.solve_pressure(bg, torch.zeros_like(bg))
    assert rc == cfd.CFD_ERR_BREAKDOWN


def test_ir_graph_form_rejected_when_nx_not_multiple_of_four(cfd):
    cav = cfd.Cavity(cfd.make_params(17, 8, 8, solver="ir"))
    with pytest.raises(cfd.CfdError):
        cav.set_ir_form("graph")
    cav.set_ir_form("persistent")


def test_ir_graph_cavity_steps(cfd):
    cav = _graph_cavity(cfd, (32, 32, 32), dt=0.01, nu=0.001, lid_u=1.0)
    rc, stats = cav.step(5)
    assert rc == cfd.CFD_OK
    assert all(s["rel_resid"] <= 1e-8 and s["outer_iters"] >= 1 for s in stats[1:])


def test_ir_graph_full_size_256(cfd):
    """256^3 standalone solve (the benchmarked size, automatic form = graph):
    the true residual is recomputed from the oracle's matrix plane by plane
    (a row of plane k touches planes k-1..k+1 only)."""
    n = 256
    cav = cfd.Cavity(cfd.make_params(n, n, n, solver="ir"))
    b = gaussian_rhs(n, n, n, seed=0)
    bg = torch.tensor(b, device="cuda")
    xg = torch.zeros_like(bg)
    l0 = cav.launch_count()
    rc, st = cav.solve_pressure(bg, xg)
    assert rc == cfd.CFD_OK
    assert_graph_kernels(cav.launch_count() - l0, 2 + 2 * (st["outer_iters"] + 1) + 2 * st["iters"] + 3, st)
    x = xg.cpu().numpy()
    bo = b - b.mean()
    A3, A2 = poisson_csr(n, n, 3), poisson_csr(n, n, 2)
    rr = 0.0
    for k in range(n):
        if k == 0:
            y = (A2 @ x[0:2].ravel()).reshape(2, n, n)[0]
        elif k == n - 1:
            y = (A2 @ x[n - 2:n].ravel()).reshape(2, n, n)[1]
        else:
            y = (A3 @ x[k - 1:k + 2].ravel()).reshape(3, n, n)[1]
        rr += float(np.sum((bo[k] - y) ** 2))
    true_rel = np.sqrt(rr) / np.linalg.norm(bo)
    assert true_rel <= 1.0001e-8, true_rel
    np.testing.assert_allclose(true_rel, st["rel_resid"], rtol=1e-6)


# ----------------------------------------------------------------------------
# diffusion solves of the IR solver, both forms: FP32 CG with FP64
# refinement on the velocity matrices H = I + c L (face grids one wider
# along their own axis).  Judged by the FP64 true residual with the oracle's
# matrix, and against the oracle's FP64 CG within 2 rtol ||b|| (both
# solutions have residual <= rtol ||b|| and ||H^-1|| <= 1, H = I + c L with
# L positive semi-definite).
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("form", ["graph", "persistent"])
@pytest.mark.parametrize("shape,nu", [((16, 16, 16), 0.05), ((20, 12, 9), 0.2), ((4, 8, 5), 0.5)])
def test_ir_diffusion_within_bound(cfd, shape, nu, form):
    from oracle.operators import diffusion_csr
    nx, ny, nz = shape
    cav = _graph_cavity(cfd, shape, form=form, dt=0.02, nu=nu, lid_u=1.0)
    ocav = OCav(nx, ny, nz, dt=0.02, nu=nu, lid_u=1.0)
    f = []
    for c in range(3):
        a = uniform_field(ocav.face_shape(c), seed=9, stream=c, lo=-1.0, hi=1.0)
        ax = 2 - c
        sl = [slice(None)] * 3
        sl[ax] = 0
        a[tuple(sl)] = 0.0
        sl[ax] = -1
        a[tuple(sl)] = 0.0
        f.append(a)
    for name, a in zip("uvw", f):
        cav.set_field(name, a)
    l0 = cav.launch_count()
    rc, st = cav.substep("diffuse")
    assert rc == cfd.CFD_OK and st["diff_status"] == cfd.CFD_OK
    if form == "graph":
        assert cav.launch_count() - l0 >= 3 * (2 + 2 + 3)  # three graph solves ran
    ref, _ = fs.diffuse(ocav, f)
    for c, name in enumerate("uvw"):
        H, bnd, mask = diffusion_csr(ocav, c)
        g = cav.read_field(name).numpy()
        bvec = f[c][mask] + bnd
        true_rel = np.linalg.norm(bvec - H @ g[mask]) / np.linalg.norm(bvec)
        assert true_rel <= 1.0001e-8, (name, true_rel)
        assert np.linalg.norm(g[mask] - ref[c][mask]) <= 2e-8 * np.linalg.norm(bvec)
        assert np.array_equal(g[~mask], f[c][~mask])  # wall-normal faces untouched
        assert st["diff_iters"][c] >= 1


def test_ir_graph_cavity_with_diffusion_converges(cfd):
    cav = _graph_cavity(cfd, (32, 32, 32), dt=0.01, nu=0.01, lid_u=1.0)
    rc, stats = cav.step(4)
    assert rc == cfd.CFD_OK
    # from rest only u (the lid's ghost term) has a nonzero diffusion
    # right-hand side at first; zero right-hand sides take no iteration
    assert all(s["rel_resid"] <= 1e-8 and s["diff_status"] == cfd.CFD_OK and s["diff_iters"][0] >= 1
               for s in stats)
