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
