"""GPU parity of the CUDA path against the FP64 oracle, through the C-ABI.

Tolerances (FP64 paths): 1e-10 relative per field, where relative means
max|gpu - oracle| / max|oracle| of that field, with the oracle replaying the
GPU's per-solve CG iteration counts (two correct CGs that sum in different
orders can stop one iteration apart).  Operator applications compare at
1e-14 relative (integer coefficients, only the summation order differs).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import fractional_step as fs  # noqa: E402
from oracle.krylov import dic_precond, jacobi_precond, pcg  # noqa: E402
from oracle.mac import Cavity as OCav  # noqa: E402
from oracle.operators import poisson_csr  # noqa: E402
from paper_2504_03697_gb300.synthetic import cavity_perturbation, gaussian_rhs, uniform_field  # noqa: E402

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-10


@pytest.fixture(scope="module")
def cfd():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2504_03697_gb300 import build as B
    B.build()
    from paper_2504_03697_gb300 import cfd as _cfd
    return _cfd


def rel_err(g, o):
    g = np.asarray(g)
    o = np.asarray(o)
    return float(np.abs(g - o).max() / max(np.abs(o).max(), 1e-300))


def make(cfd, n, **kw):
    nx, ny, nz = n if isinstance(n, tuple) else (n, n, n)
    keep = ("dt", "nu", "lid_u", "g", "rho", "length", "rtol", "max_iters", "advect_order", "warm_start")
    return cfd.Cavity(cfd.make_params(nx, ny, nz, **kw)), OCav(nx, ny, nz, **{k: v for k, v in kw.items() if k in keep})


# ----------------------------------------------------------------------------
# operator apply (the paper's SpMV, matrix-free)
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("shape", [(1, 1, 7), (5, 5, 5), (17, 9, 13), (33, 8, 3), (40, 20, 70), (64, 64, 64),
                                   (100, 37, 5)])
def test_apply_poisson_matches_csr(cfd, shape):
    cav, _ = make(cfd, shape)
    nx, ny, nz = shape
    x = uniform_field((nz, ny, nx), seed=7)
    xg = torch.tensor(x, device="cuda")
    yg = torch.empty_like(xg)
    cav.apply_poisson(xg, yg)
    y = poisson_csr(nx, ny, nz) @ x.ravel()
    np.testing.assert_allclose(yg.cpu().numpy().ravel(), y, rtol=0, atol=1e-14 * 6)


# ----------------------------------------------------------------------------
# standalone pressure solves
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("shape,solver", [((16, 16, 16), "cg"), ((17, 9, 13), "cg"), ((48, 40, 32), "cg"),
                                          ((16, 16, 16), "jacobi"), ((17, 9, 13), "jacobi"), ((2, 2, 2), "cg")])
def test_pressure_solve_parity(cfd, shape, solver):
    nx, ny, nz = shape
    cav, _ = make(cfd, shape, solver=solver)
    b = gaussian_rhs(nx, ny, nz, seed=3)
    bg = torch.tensor(b, device="cuda")
    xg = torch.zeros_like(bg)
    rc, st = cav.solve_pressure(bg, xg)
    assert rc == cfd.CFD_OK and st["rel_resid"] <= 1e-8
    A = poisson_csr(nx, ny, nz)
    pc = jacobi_precond(A) if solver == "jacobi" else (lambda r: r.copy())
    bo = b.ravel() - b.mean()
    x_rep, s_rep = pcg(A, bo, rtol=1e-8, max_iters=10 ** 6, precond=pc, fixed_iters=st["iters"])
    assert rel_err(xg.cpu().numpy().ravel(), x_rep) < FP64_TOL
    # the oracle's own stopping agrees to within a couple of iterations
    x_own, s_own = pcg(A, bo, rtol=1e-8, max_iters=10 ** 6, precond=pc)
    assert abs(s_own.iters - st["iters"]) <= 2
    np.testing.assert_allclose(np.linalg.norm(bo), st["b_norm"], rtol=1e-12)


@pytest.mark.parametrize("variant", ["single", "two"])
@pytest.mark.parametrize("shape,bps,tz", [((48, 40, 32), 0, 0), ((17, 9, 13), 0, 0), ((64, 64, 64), 1, 8),
                                          ((96, 96, 96), 1, 1), ((33, 8, 3), 2, 2)])
def test_cg_variants_parity(cfd, variant, shape, bps, tz):
    # the single-reduction (Chronopoulos-Gear) and textbook forms against the
    # oracle's textbook CG, on the register path (small grids / deep tiles)
    # and the memory path (96^3 with one block per SM and depth-1 tiles)
    nx, ny, nz = shape
    cav, _ = make(cfd, shape)
    cav.set_cg_variant(variant)
    cav.set_solver_shape(bps, tz)
    b = gaussian_rhs(nx, ny, nz, seed=4)
    bg = torch.tensor(b, device="cuda")
    xg = torch.zeros_like(bg)
    rc, st = cav.solve_pressure(bg, xg)
    assert rc == cfd.CFD_OK and st["rel_resid"] <= 1e-8, st
    A = poisson_csr(nx, ny, nz)
    bo = b.ravel() - b.mean()
    x_rep, _ = pcg(A, bo, rtol=1e-8, max_iters=10 ** 6, fixed_iters=st["iters"])
    assert rel_err(xg.cpu().numpy().ravel(), x_rep) < FP64_TOL
    x_own, s_own = pcg(A, bo, rtol=1e-8, max_iters=10 ** 6)
    assert abs(s_own.iters - st["iters"]) <= 2


def _sms():
    return torch.cuda.get_device_properties(0).multi_processor_count


def _tiles8(shape):
    nx, ny, nz = shape
    return -(-nx // 32) * -(-ny // 8) * -(-nz // 8)


@pytest.mark.parametrize("shape,warm", [((64, 64, 64), False), ((61, 62, 59), False), ((63, 50, 64), False),
                                        ((61, 62, 59), True)])
def test_tile_resident_cg_parity(cfd, shape, warm):
    # the tile-resident single-reduction kernel (the automatic shape when the
    # 32 x 8 x 8 tiles number more than half of the SMs and at most one per
    # SM): ragged tiles in x, y and z, cold and warm starts, against the
    # oracle's textbook CG with the GPU's iteration count replayed
    nx, ny, nz = shape
    if not (_sms() / 2 < _tiles8(shape) <= _sms()):
        pytest.skip("grid does not take the tile-resident kernel on this device")
    cav, _ = make(cfd, shape, warm_start=warm)
    assert cav.solver_shape(0)["tile_resident"]
    b = gaussian_rhs(nx, ny, nz, seed=5)
    x0 = uniform_field((nz, ny, nx), seed=6) if warm else np.zeros((nz, ny, nx))
    bg = torch.tensor(b, device="cuda")
    xg = torch.tensor(x0, device="cuda")
    rc, st = cav.solve_pressure(bg, xg)
    assert rc == cfd.CFD_OK and st["rel_resid"] <= 1e-8, st
    A = poisson_csr(nx, ny, nz)
    bo = b.ravel() - b.mean()
    x_rep, _ = pcg(A, bo, x0=x0.ravel(), rtol=1e-8, max_iters=10 ** 6, fixed_iters=st["iters"])
    assert rel_err(xg.cpu().numpy().ravel(), x_rep) < FP64_TOL
    x_own, s_own = pcg(A, bo, x0=x0.ravel(), rtol=1e-8, max_iters=10 ** 6)
    assert abs(s_own.iters - st["iters"]) <= 2
    np.testing.assert_allclose(np.linalg.norm(bo), st["b_norm"], rtol=1e-12)


def test_tile_resident_cg_zero_rhs_and_cap(cfd):
    shape = (64, 64, 64)
    if not (_sms() / 2 < _tiles8(shape) <= _sms()):
        pytest.skip("grid does not take the tile-resident kernel on this device")
    cav, _ = make(cfd, shape)
    assert cav.solver_shape(0)["tile_resident"]
    bg = torch.zeros(shape, dtype=torch.float64, device="cuda")
    xg = torch.full_like(bg, 3.0)
    rc, st = cav.solve_pressure(bg, xg)
    assert rc == cfd.CFD_OK and st["iters"] == 0 and st["rel_resid"] == 0.0
    assert torch.all(xg == 0)
    cav5, _ = make(cfd, shape, max_iters=5)
    b = gaussian_rhs(64, 64, 64, seed=2)
    bg = torch.tensor(b, device="cuda")
    xg = torch.zeros_like(bg)
    rc, st = cav5.solve_pressure(bg, xg)
    assert rc == cfd.CFD_ERR_NOT_CONVERGED and st["iters"] == 5 and st["rel_resid"] > 1e-8
    A = poisson_csr(64, 64, 64)
    bo = b.ravel() - b.mean()
    x_rep, _ = pcg(A, bo, rtol=1e-8, max_iters=10 ** 6, fixed_iters=5)
    assert rel_err(xg.cpu().numpy().ravel(), x_rep) < FP64_TOL
    r = bo - A @ xg.cpu().numpy().ravel()
    np.testing.assert_allclose(st["rel_resid"], np.linalg.norm(r) / np.linalg.norm(bo), rtol=1e-9)


def test_zero_rhs_solve(cfd):
    cav, _ = make(cfd, (8, 8, 8))
    bg = torch.zeros((8, 8, 8), dtype=torch.float64, device="cuda")
    xg = torch.full_like(bg, 3.0)
    rc, st = cav.solve_pressure(bg, xg)
    assert rc == cfd.CFD_OK and st["iters"] == 0
    assert torch.all(xg == 0)


def test_iteration_cap_reports_not_converged(cfd):
    cav, _ = make(cfd, (24, 24, 24), max_iters=3)
    bg = torch.tensor(gaussian_rhs(24, 24, 24, seed=1), device="cuda")
    xg = torch.zeros_like(bg)
    rc, st = cav.solve_pressure(bg, xg)
    assert rc == cfd.CFD_ERR_NOT_CONVERGED and st["iters"] == 3 and st["rel_resid"] > 1e-8


def test_nan_rhs_reports_breakdown(cfd):
    cav, _ = make(cfd, (8, 8, 8))
    b = gaussian_rhs(8, 8, 8, seed=1)
    b[3, 4, 5] = np.nan
    bg = torch.tensor(b, device="cuda")
    xg = torch.zeros_like(bg)
    rc, st = cav.solve_pressure(bg, xg)
    assert rc == cfd.CFD_ERR_BREAKDOWN


# ----------------------------------------------------------------------------
# substeps
# ----------------------------------------------------------------------------
def _random_velocity(ocav, seed, amp):
    return [uniform_field(ocav.face_shape(c), seed=seed, stream=c, lo=-amp, hi=amp) for c in range(3)]


def _load(cav, fields, p=None):
    for name, f in zip("uvw", fields):
        cav.set_field(name, f)
    if p is not None:
        cav.set_field("p", p)


def _zero_walls(ocav, fields):
    out = []
    for c, f in enumerate(fields):
        f = f.copy()
        a = 2 - c
        sl = [slice(None)] * 3
        sl[a] = 0
        f[tuple(sl)] = 0.0
        sl[a] = -1
        f[tuple(sl)] = 0.0
        out.append(f)
    return out


@pytest.mark.parametrize("order", [1, 2])
@pytest.mark.parametrize("shape", [(16, 16, 16), (17, 9, 13), (5, 31, 4)])
def test_advect_parity(cfd, shape, order):
    cav, ocav = make(cfd, shape, dt=0.05, lid_u=1.3, advect_order=order)
    f = _zero_walls(ocav, _random_velocity(ocav, 5, 2.0))  # backtraces cross cells and walls
    _load(cav, f)
    cav.substep("advect")
    ref = fs.advect(ocav, *f)
    for c, name in enumerate("uvw"):
        assert rel_err(cav.read_field(name).numpy(), ref[c]) < 1e-13


def test_forces_parity(cfd):
    cav, ocav = make(cfd, (9, 7, 6), dt=0.1, g=(0.5, -0.25, 2.0))
    f = _zero_walls(ocav, _random_velocity(ocav, 2, 1.0))
    _load(cav, f)
    cav.substep("forces")
    ref = fs.apply_forces(ocav, *f)
    for c, name in enumerate("uvw"):
        np.testing.assert_array_equal(cav.read_field(name).numpy(), ref[c])


@pytest.mark.parametrize("shape", [(16, 16, 16), (17, 9, 13)])
def test_diffuse_parity(cfd, shape):
    cav, ocav = make(cfd, shape, dt=0.02, nu=0.05, lid_u=1.0)
    f = _zero_walls(ocav, _random_velocity(ocav, 9, 1.0))
    _load(cav, f)
    rc, st = cav.substep("diffuse")
    assert rc == cfd.CFD_OK
    ref, rst = fs.diffuse(ocav, f, fixed_iters=tuple(st["diff_iters"]))
    for c, name in enumerate("uvw"):
        assert rel_err(cav.read_field(name).numpy(), ref[c]) < FP64_TOL
    own, ost = fs.diffuse(ocav, f)
    for c in range(3):
        assert abs(ost[c].iters - st["diff_iters"][c]) <= 1


@pytest.mark.parametrize("shape", [(16, 16, 16), (17, 9, 13)])
def test_project_parity(cfd, shape):
    cav, ocav = make(cfd, shape, dt=0.02, nu=0.0, lid_u=1.0)
    f = _zero_walls(ocav, _random_velocity(ocav, 4, 1.0))
    _load(cav, f)
    rc, st = cav.substep("project")
    assert rc == cfd.CFD_OK
    b = fs.pressure_rhs(ocav, *f)
    x, _ = fs.solve_pressure(ocav, b, fixed_iters=st["iters"])
    ref = fs.correct(ocav, *f, x)
    for c, name in enumerate("uvw"):
        assert rel_err(cav.read_field(name).numpy(), ref[c]) < FP64_TOL
    assert rel_err(cav.read_field("p").numpy(), fs.gauge(x)) < FP64_TOL
    # divergence-free to the solve tolerance
    u, v, w = (cav.read_field(n).numpy() for n in "uvw")
    div = fs.divergence_sum(u, v, w)
    s = ocav.dt / (ocav.rho * ocav.h)
    assert np.linalg.norm(div) <= s * 1.01e-8 * np.linalg.norm(b)


# ----------------------------------------------------------------------------
# whole steps
# ----------------------------------------------------------------------------
def _run_pair(cfd, shape, steps, seed, concurrent=None, **kw):
    cav, ocav = make(cfd, shape, **kw)
    if concurrent is not None:  # None: the handle's default
        cav.set_concurrent_diffusion(concurrent)
    nx, ny, nz = shape
    init = cavity_perturbation(nx, ny, nz, seed=seed, amp=1e-3)
    _load(cav, init)
    rc, stats = cav.step(steps)
    assert rc == cfd.CFD_OK, stats
    fixed = [{"p": s["iters"], "u": s["diff_iters"][0], "v": s["diff_iters"][1], "w": s["diff_iters"][2]}
             for s in stats]
    st, hist = fs.simulate(ocav, fs.initial_state(ocav, init), steps, fixed_iters_per_step=fixed)
    errs = {name: rel_err(cav.read_field(name).numpy(), st[i]) for i, name in enumerate("uvwp")}
    return cav, ocav, stats, st, errs


def test_cavity_16cube_20_steps(cfd):
    """Plain method, FP64: 16^3, lid 1.0, nu 0.01, dt 0.01, 20 steps, seed 1."""
    cav, ocav, stats, st, errs = _run_pair(cfd, (16, 16, 16), 20, 1, dt=0.01, nu=0.01, lid_u=1.0)
    for name, e in errs.items():
        assert e < FP64_TOL, (name, e)
    for s in stats:
        assert s["rel_resid"] <= 1e-8 and s["status"] == 0 and s["diff_status"] == 0
    u, v, w = (cav.read_field(n).numpy() for n in "uvw")
    assert np.abs(fs.divergence_sum(u, v, w)).max() < 1e-8


def test_cavity_64cube_steps(cfd):
    """Same cavity at 64^3 (nu 0.001), FP64, first 3 steps replayed."""
    cav, ocav, stats, st, errs = _run_pair(cfd, (64, 64, 64), 3, 2, dt=0.01, nu=0.001, lid_u=1.0)
    for name, e in errs.items():
        assert e < FP64_TOL, (name, e)


def test_cavity_63cube_steps_tile_resident(cfd):
    """63^3 cavity, FP64: the pressure grid and all three velocity grids take
    the tile-resident CG (128 tiles each); 3 steps against the oracle."""
    shape = (63, 63, 63)
    if not (_sms() / 2 < _tiles8(shape) <= _sms() and _tiles8((64, 63, 63)) <= _sms()):
        pytest.skip("grids do not take the tile-resident kernel on this device")
    # one diffusion solve at a time: concurrent solves share the device and
    # take the register path
    cav, ocav, stats, st, errs = _run_pair(cfd, shape, 3, 4, concurrent=False, dt=0.01, nu=0.002, lid_u=1.0)
    shapes = [cav.solver_shape(k) for k in range(4)]
    assert all(sh["tile_resident"] for sh in shapes), shapes
    for name, e in errs.items():
        assert e < FP64_TOL, (name, e)
    for s in stats:
        assert s["rel_resid"] <= 1e-8 and s["status"] == 0 and s["diff_status"] == 0


@pytest.mark.parametrize("shape,kw", [((17, 9, 13), dict(dt=0.02, nu=0.01, lid_u=1.0)),
                                      ((1, 1, 1), dict(dt=0.01, nu=0.01, lid_u=1.0)),
                                      ((2, 3, 2), dict(dt=0.01, nu=0.0, lid_u=2.0)),
                                      ((12, 12, 12), dict(dt=0.01, nu=0.0, lid_u=1.0, solver="jacobi")),
                                      ((10, 8, 6), dict(dt=0.01, nu=0.02, lid_u=1.0, g=(1.0, 0.0, -0.5)))])
def test_cavity_edge_cases(cfd, shape, kw):
    solver = kw.pop("solver", "cg")
    cav, ocav = make(cfd, shape, solver=solver, **kw)
    nx, ny, nz = shape
    init = cavity_perturbation(nx, ny, nz, seed=3, amp=1e-2)
    _load(cav, init)
    rc, stats = cav.step(5)
    assert rc == cfd.CFD_OK
    fixed = [{"p": s["iters"], "u": s["diff_iters"][0], "v": s["diff_iters"][1], "w": s["diff_iters"][2]}
             for s in stats]
    st, _ = fs.simulate(ocav, fs.initial_state(ocav, init), 5, fixed_iters_per_step=fixed,
                        precond="jacobi" if solver == "jacobi" else "none")
    for i, name in enumerate("uvwp"):
        assert rel_err(cav.read_field(name).numpy(), st[i]) < FP64_TOL, name


def test_zero_state_stays_at_rest(cfd):
    cav, ocav = make(cfd, (8, 8, 8), lid_u=0.0, nu=0.01)
    rc, stats = cav.step(3)
    assert rc == cfd.CFD_OK and all(s["iters"] == 0 for s in stats)
    for name in "uvw":
        assert torch.all(cav.read_field(name) == 0)
    assert torch.all(cav.read_field("p") == 1.0)


def test_bitwise_deterministic(cfd):
    outs = []
    for _ in range(2):
        cav, _ = make(cfd, (24, 20, 16), dt=0.01, nu=0.01, lid_u=1.0)
        _load(cav, cavity_perturbation(24, 20, 16, seed=8, amp=1e-3))
        cav.step(4)
        outs.append([cav.read_field(n).numpy() for n in "uvwp"])
    for a, b in zip(*outs):
        np.testing.assert_array_equal(a, b)


# ----------------------------------------------------------------------------
# CSV snapshot output (cfd_snapshot / cfd_snapshot_write_csv)
# ----------------------------------------------------------------------------
def test_csv_snapshot_matches_state(cfd, tmp_path):
    from oracle.snapshot import cell_table
    shape = (12, 10, 8)
    cav, ocav = make(cfd, shape, nu=0.01, lid_u=1.0)
    for name, f in zip("uvw", cavity_perturbation(*shape, seed=5)):
        cav.set_field(name, f)
    cav.step(3)
    fields = {f: cav.read_field(f).numpy() for f in "uvwp"}
    cav.snapshot()
    cav.step(1)  # overlaps the copy; the file must still hold the state before this step
    path = tmp_path / "snap.csv"
    cav.write_csv(str(path), threads=3)
    with open(path) as fh:
        assert fh.readline().strip() == "x,y,z,u,v,w,p"
    got = np.loadtxt(path, delimiter=",", skiprows=1)
    ref = cell_table(ocav, fields["u"], fields["v"], fields["w"], fields["p"])
    np.testing.assert_array_equal(got, ref)  # 17 significant digits round-trip exactly


# ----------------------------------------------------------------------------
# DIC-preconditioned CG (the paper's default preconditioner)
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("shape", [(16, 16, 16), (17, 9, 13), (24, 20, 28), (2, 3, 2)])
def test_dic_solve_parity(cfd, shape):
    nx, ny, nz = shape
    cav, _ = make(cfd, shape, solver="dic")
    b = gaussian_rhs(nx, ny, nz, seed=6)
    bg = torch.tensor(b, device="cuda")
    xg = torch.zeros_like(bg)
    rc, st = cav.solve_pressure(bg, xg)
    assert rc == cfd.CFD_OK and st["rel_resid"] <= 1e-8, st
    A = poisson_csr(nx, ny, nz)
    apply, _ = dic_precond(A)
    bo = b.ravel() - b.mean()
    x_rep, _ = pcg(A, bo, rtol=1e-8, max_iters=10 ** 6, precond=apply, fixed_iters=st["iters"])
    assert rel_err(xg.cpu().numpy().ravel(), x_rep) < FP64_TOL
    x_own, s_own = pcg(A, bo, rtol=1e-8, max_iters=10 ** 6, precond=apply)
    assert abs(s_own.iters - st["iters"]) <= 2
    _, s_cg = pcg(A, bo, rtol=1e-8, max_iters=10 ** 6)
    print(f"{shape}: DIC-PCG {st['iters']} iterations, CG {s_cg.iters}")


def test_dic_cavity_steps(cfd):
    shape, steps = (16, 16, 16), 5
    cav, ocav = make(cfd, shape, dt=0.01, nu=0.01, lid_u=1.0, solver="dic")
    init = cavity_perturbation(*shape, seed=1, amp=1e-3)
    _load(cav, init)
    rc, stats = cav.step(steps)
    assert rc == cfd.CFD_OK, stats
    fixed = [{"p": s["iters"], "u": s["diff_iters"][0], "v": s["diff_iters"][1], "w": s["diff_iters"][2]}
             for s in stats]
    st, _ = fs.simulate(ocav, fs.initial_state(ocav, init), steps, fixed_iters_per_step=fixed, precond="dic")
    for i, name in enumerate("uvwp"):
        assert rel_err(cav.read_field(name).numpy(), st[i]) < FP64_TOL, name


def test_dic_on_a_line_breaks_down_cleanly(cfd):
    # 1 x 1 x n: no fill to drop, the factor is exact and the last pivot of the
    # singular matrix is 0: a breakdown status, not a fault or a hang
    cav, _ = make(cfd, (1, 1, 9), solver="dic")
    b = np.sin(np.arange(9.0)).reshape(9, 1, 1)
    bg = torch.tensor(b, device="cuda")
    xg = torch.zeros_like(bg)
    rc, st = cav.solve_pressure(bg, xg)
    assert rc == cfd.CFD_ERR_BREAKDOWN and st["status"] == cfd.CFD_ERR_BREAKDOWN


def test_cavity_midpoint_backtrace_steps(cfd):
    """The cavity with the explicit-midpoint backtrace: 16^3, 8 steps."""
    cav, ocav, stats, st, errs = _run_pair(cfd, (16, 16, 16), 8, 2, dt=0.01, nu=0.01, lid_u=1.0, advect_order=2)
    for name, e in errs.items():
        assert e < FP64_TOL, (name, e)


# ----------------------------------------------------------------------------
# assembled CSR path (the paper's matrix format) vs the matrix-free operator
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("shape", [(1, 1, 7), (5, 4, 3), (17, 9, 13), (64, 64, 64)])
def test_csr_matrix_and_spmv(cfd, shape):
    nx, ny, nz = shape
    M = cfd.CsrMatrix(nx, ny, nz)
    ref = poisson_csr(nx, ny, nz)
    rp, col, val = M.arrays()
    assert M.nnz == ref.nnz
    np.testing.assert_array_equal(rp.numpy(), ref.indptr)      # integer structure: exact
    np.testing.assert_array_equal(col.numpy(), ref.indices)
    np.testing.assert_array_equal(val.numpy(), ref.data)
    cav, _ = make(cfd, shape)
    x = torch.tensor(uniform_field((nz, ny, nx), seed=9), device="cuda")
    y1 = torch.empty_like(x)
    y2 = torch.empty_like(x)
    M.spmv(x, y1)
    cav.apply_poisson(x, y2)
    torch.cuda.synchronize()
    np.testing.assert_allclose(y1.cpu().numpy().ravel(), ref @ x.cpu().numpy().ravel(), rtol=0, atol=1e-14 * 6)
    np.testing.assert_allclose(y1.cpu().numpy(), y2.cpu().numpy(), rtol=0, atol=1e-14 * 6)


def test_cavity_warm_started_pressure(cfd):
    """Pressure solves started from the previous step's p: 16^3, 6 steps."""
    cav, ocav, stats, st, errs = _run_pair(cfd, (16, 16, 16), 6, 3, dt=0.01, nu=0.01, lid_u=1.0, warm_start=True)
    for name, e in errs.items():
        assert e < FP64_TOL, (name, e)
    assert sum(s["iters"] for s in stats[1:]) < sum(s["iters"] for s in stats[:1]) * (len(stats) - 1)



# ----------------------------------------------------------------------------
# the three diffusion solves run at once (cfd_set_concurrent_diffusion)
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("shape", [(16, 16, 16), (17, 9, 13)])
def test_diffuse_parity_concurrent(cfd, shape):
    cav, ocav = make(cfd, shape, dt=0.02, nu=0.05, lid_u=1.0)
    cav.set_concurrent_diffusion(True)
    f = _zero_walls(ocav, _random_velocity(ocav, 9, 1.0))
    _load(cav, f)
    rc, st = cav.substep("diffuse")
    assert rc == cfd.CFD_OK and st["diff_status"] == cfd.CFD_OK
    ref, rst = fs.diffuse(ocav, f, fixed_iters=tuple(st["diff_iters"]))
    for c, name in enumerate("uvw"):
        assert rel_err(cav.read_field(name).numpy(), ref[c]) < FP64_TOL


@pytest.mark.parametrize("shape,steps", [((16, 16, 16), 6), ((64, 64, 64), 3)])
def test_cavity_steps_concurrent_diffusion(cfd, shape, steps):
    cav, ocav, stats, st, errs = _run_pair(cfd, shape, steps, 2, concurrent=True, dt=0.01, nu=0.001 if shape[0] == 64
                                           else 0.01, lid_u=1.0)
    for name, e in errs.items():
        assert e < FP64_TOL, (name, e)
    assert all(s["diff_status"] == 0 and s["status"] == 0 for s in stats)


def test_concurrent_diffusion_needs_its_workspace(cfd):
    cav, _ = make(cfd, (8, 8, 8), dt=0.01, nu=0.0, lid_u=1.0)
    with pytest.raises(cfd.CfdError):
        cav.set_concurrent_diffusion(True)
    cav.set_concurrent_diffusion(False)
