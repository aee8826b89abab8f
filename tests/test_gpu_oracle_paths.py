"""Oracle parity of the mixed-precision, batched and flexible-CG paths.

Every check here compares a CUDA path with the FP64 oracle (``oracle/``)
on the same seeded inputs, step by step:

* whole cavity steps (``cfd_step``) with the FP32-inner / FP64-refined
  solver, in the graph and the persistent form, on a cube and on ragged
  grids: before each step the GPU's state is read back and the oracle's
  step (forces, advection, diffusion, projection, gauge; Sec. 3.1) is run
  from it;
* every cavity of a mixed-precision batch, the same way;
* the CUDA flexible PCG against ``oracle.krylov.fpcg`` driven by the float64
  network ``oracle.unet.precondition`` on the same parameters;
* the iteration and refinement counts of the mixed-precision solve against
  the oracle's model of it, ``oracle.krylov.ir_cg``.

Tolerances.  Two solves that both stop at ||b - A x|| <= rtol ||b|| differ
by at most 2 rtol ||b|| / lambda_min (pressure, after mean removal;
lambda_min = min_d 4 sin^2(pi / (2 n_d))) or 2 rtol ||b|| (velocity
diffusion, ||H^-1|| <= 1).  Over a whole step: with D the face-difference
(divergence) operator on the interior faces, A = D D^T and the projection
u -> u - D^T A^+ D u is orthogonal, so a difference d of the intermediate
velocity reaches the new velocity with norm at most ||d||; a pressure
residual r moves the velocity by s ||D^T A^+ r|| <= s ||r|| / sqrt(lambda_min)
(s = dt / (rho h)) and the pressure by ||r|| / lambda_min; the pressure
right-hand side -D d / s moves the pressure by at most ||d|| / (s
sqrt(lambda_min)).  These are the bounds asserted below; per-field max-abs
errors are printed for the record.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import fractional_step as fs  # noqa: E402
from oracle import unet as ou  # noqa: E402
from oracle.krylov import fpcg, ir_cg  # noqa: E402
from oracle.mac import Cavity as OCav  # noqa: E402
from oracle.operators import diffusion_csr, poisson_csr  # noqa: E402
from paper_2504_03697_gb300.synthetic import cavity_perturbation, gaussian_rhs  # noqa: E402

pytestmark = pytest.mark.gpu

RTOL = 1e-8


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


def read_state(cav):
    return tuple(cav.read_field(f).numpy().copy() for f in "uvwp")


def check_step_against_oracle(ocav, start, gpu_end, gpu_stats, label):
    """Run the oracle's step from the GPU's start state and assert the
    whole-step bounds of the module header; returns the max-abs errors."""
    shape = (ocav.nx, ocav.ny, ocav.nz)
    ref, st = fs.step(ocav, start)
    # diffusion right-hand sides of this step (forces and advection are the
    # oracle's, equal to the GPU's to 1e-13: both are plain FP64 sweeps)
    fu, fv, fw = fs.apply_forces(ocav, *start[:3])
    adv = fs.advect(ocav, fu, fv, fw)
    d2 = 0.0
    for c in range(3):
        if ocav.nu > 0.0:
            _, bnd, mask = diffusion_csr(ocav, c)
            d2 += (2.0 * RTOL * np.linalg.norm(adv[c][mask] + bnd)) ** 2
    vel_norm = np.sqrt(sum(float(np.sum(a * a)) for a in adv))
    d_star = np.sqrt(d2) + 1e-11 * vel_norm  # intermediate velocity
    s = ocav.dt / (ocav.rho * ocav.h)
    bnorm = float(np.linalg.norm(st["b"]))
    lm = lam_min(shape)
    vel_bound = d_star + 2.0001 * s * RTOL * bnorm / np.sqrt(lm)
    p_bound = d_star / (s * np.sqrt(lm)) + 2.0001 * RTOL * bnorm / lm
    dv = np.sqrt(sum(float(np.sum((g - o) ** 2)) for g, o in zip(gpu_end[:3], ref[:3])))
    pg, po = gpu_end[3], ref[3]
    dp = float(np.linalg.norm((pg - pg.mean()) - (po - po.mean())))
    errs = {n: float(np.abs(g - o).max()) for n, g, o in zip("uvwp", gpu_end, ref)}
    assert dv <= vel_bound, (label, dv, vel_bound)
    assert dp <= p_bound, (label, dp, p_bound)
    assert abs(pg.mean() - 1.0) <= 1e-12, label  # gauge
    assert gpu_stats["status"] == 0 and gpu_stats["rel_resid"] <= RTOL * 1.0001, (label, gpu_stats)
    assert gpu_stats["diff_status"] == 0, (label, gpu_stats)
    return errs, dv / vel_bound, dp / p_bound


@pytest.mark.parametrize("form,shape", [("graph", (16, 16, 16)), ("graph", (20, 12, 9)),
                                        ("persistent", (16, 16, 16)), ("persistent", (17, 9, 13))])
def test_ir_cavity_steps_match_oracle_per_step(cfd, form, shape):
    nx, ny, nz = shape
    nu, dt, steps = 0.01, 0.01, 4
    cav = cfd.Cavity(cfd.make_params(nx, ny, nz, dt=dt, nu=nu, lid_u=1.0, solver="ir"))
    cav.set_ir_form(form)
    ocav = OCav(nx, ny, nz, dt=dt, nu=nu, lid_u=1.0)
    for name, f in zip("uvw", cavity_perturbation(nx, ny, nz, seed=1, amp=1e-3)):
        cav.set_field(name, f)
    for k in range(steps):
        start = read_state(cav)
        rc, st = cav.step(1)
        assert rc == cfd.CFD_OK, st
        assert st[0]["outer_iters"] >= 1
        errs, fv, fp = check_step_against_oracle(ocav, start, read_state(cav), st[0], f"{form} {shape} step {k}")
        print(f"IR {form} {shape} step {k}: max-abs {errs}, velocity {fv:.2e} / pressure {fp:.2e} of the bound")


def test_ir_batch_matches_oracle_per_cavity(cfd):
    specs = [((24, 24, 24), 0.01), ((32, 28, 20), 0.005), ((16, 16, 16), 0.02), ((20, 12, 9), 0.0)]
    prms = [cfd.make_params(*shape, dt=0.01, nu=nu, lid_u=1.0, solver="ir") for shape, nu in specs]
    b = cfd.Batch(prms)
    for i, (shape, _) in enumerate(specs):
        for name, f in zip("uvw", cavity_perturbation(*shape, seed=30 + i, amp=1e-2)):
            b.cavity(i).set_field(name, f)
    for k in range(3):
        starts = [read_state(b.cavity(i)) for i in range(len(specs))]
        rc, st = b.step(1)
        assert rc == cfd.CFD_OK
        for i, (shape, nu) in enumerate(specs):
            ocav = OCav(*shape, dt=0.01, nu=nu, lid_u=1.0)
            errs, fv, fp = check_step_against_oracle(ocav, starts[i], read_state(b.cavity(i)), st[i],
                                                     f"batch cavity {i} step {k}")
            print(f"IR batch cavity {i} {shape} step {k}: max-abs {errs}, {fv:.2e} / {fp:.2e} of the bound")


def test_ir_batch_odd_widths_match_oracle(cfd):
    """Batched mixed-precision solves on widths that are not multiples of 4:
    pressure on scalar lanes (17, 18 wide), velocity matrices on padded
    float4 rows, one cavity with forces; every step within the whole-step
    bounds against the oracle."""
    specs = [((17, 9, 13), dict(nu=0.01, g=(0.0, 0.0, 0.0))), ((18, 10, 12), dict(nu=0.02, g=(0.5, 0.0, -0.25))),
             ((20, 12, 9), dict(nu=0.0, g=(0.0, 0.0, 0.0)))]
    prms = [cfd.make_params(*shape, dt=0.01, lid_u=1.0, solver="ir", **kw) for shape, kw in specs]
    b = cfd.Batch(prms)
    for i, (shape, _) in enumerate(specs):
        for name, f in zip("uvw", cavity_perturbation(*shape, seed=60 + i, amp=1e-2)):
            b.cavity(i).set_field(name, f)
    for k in range(3):
        starts = [read_state(b.cavity(i)) for i in range(len(specs))]
        rc, st = b.step(1)
        assert rc == cfd.CFD_OK
        for i, (shape, kw) in enumerate(specs):
            ocav = OCav(*shape, dt=0.01, lid_u=1.0, **kw)
            errs, fv, fp = check_step_against_oracle(ocav, starts[i], read_state(b.cavity(i)), st[i],
                                                     f"odd batch cavity {i} step {k}")
            print(f"IR batch (odd widths) cavity {i} {shape} step {k}: max-abs {errs}, {fv:.2e} / {fp:.2e} of the bound")


def passthrough_params(w0=1.0, w1=1.0):
    """Hand-set U-Net: every layer passes channel 0 through its centre tap;
    the skip halves carry weight 1 and the up-sampled coarse channels w0 (at
    level 0) and w1 (at level 1), so M(r) = r + w0 B2 r + w0 w1 B4 r (B the
    block means), an SPD preconditioner."""
    layers = []
    for name, _, c0, c1, cout, ks in ou.LAYERS:
        w = torch.zeros(cout, c0 + c1, ks, ks, ks, dtype=torch.float64)
        m = ks // 2
        w[0, 0, m, m, m] = 1.0
        if c1:
            w[0, c0, m, m, m] = w0 if name == "L0c" else w1
        layers.append((w, torch.zeros(cout, dtype=torch.float64)))
    return ou.flatten(layers).float()


@pytest.mark.parametrize("shape,w", [((16, 16, 16), (1.0, 1.0)), ((16, 12, 8), (4.0, 4.0)),
                                     ((24, 20, 16), (4.0, 4.0))])
def test_fpcg_matches_oracle_flexible_cg(cfd, shape, w):
    """The CUDA flexible PCG against oracle.krylov.fpcg with the oracle's
    network on the same parameters (the hand-set weights are BF16 values).
    The oracle's network stores its input and activations rounded to BF16,
    as the CUDA network does (``oracle.unet.bf16_store``), so both run
    flexible CG with the same preconditioner up to FP32-vs-FP64 accumulation
    order: the iteration counts must agree within 5 % (at least 3), neither
    may fall back to plain CG, and the solutions must lie within the rtol
    bound of each other.  The float64 network is run too and its count
    printed: BF16 storage costs flexible CG some iterations."""
    nx, ny, nz = shape
    params = passthrough_params(*w)
    net = cfd.UNet(nx, ny, nz, seed=0)
    net.set_params(params)
    b = gaussian_rhs(nx, ny, nz, seed=31)
    bg = torch.tensor(b.ravel(), device="cuda")
    xg = torch.zeros_like(bg)
    rc, st = net.fpcg_solve(bg, xg, rtol=RTOL)
    assert rc == cfd.CFD_OK and st["outer_iters"] == 0, st
    layers = ou.unflatten(params.double())
    A = poisson_csr(nx, ny, nz)
    cap = 20 * max(shape)
    xo, so = fpcg(A, b.ravel(), lambda r: ou.precondition(layers, r.reshape(nz, ny, nx), store=ou.bf16_store).ravel(),
                  rtol=RTOL, max_iters=cap)
    _, s64 = fpcg(A, b.ravel(), lambda r: ou.precondition(layers, r.reshape(nz, ny, nx)).ravel(), rtol=RTOL,
                  max_iters=cap)
    assert so.converged and not so.fell_back, so
    assert abs(st["iters"] - so.iters) <= max(3, so.iters // 20), (st["iters"], so.iters)
    bo = b.ravel() - b.mean()
    x = xg.cpu().numpy()
    true_rel = np.linalg.norm(bo - A @ x) / np.linalg.norm(bo)
    assert true_rel <= RTOL * 1.0001
    d = (x - x.mean()) - (xo - xo.mean())
    bound = 2 * RTOL * np.linalg.norm(bo) / lam_min(shape)
    assert np.linalg.norm(d) <= bound, (np.linalg.norm(d), bound)
    print(f"FPCG {shape} w={w}: GPU {st['iters']} iterations, oracle {so.iters} (BF16 storage), "
          f"{s64.iters} (float64 network); max|dx| {np.abs(d).max():.2e} (bound {bound:.2e})")


@pytest.mark.parametrize("form", ["graph", "persistent"])
@pytest.mark.parametrize("shape,delta", [((32, 32, 32), 0.1), ((48, 40, 32), 0.01), ((20, 12, 12), 0.3)])
def test_ir_counts_match_oracle_model(cfd, form, shape, delta):
    """Inner iterations and refinements of the mixed-precision pressure
    solve against oracle.krylov.ir_cg (the same method in numpy: FP32
    vectors and operator, FP64 dot products, FP64 reliable updates) at the
    same refinement factor.  FP32 rounding differs between the two (FMA
    contraction, summation order), so counts may drift by a few iterations:
    the inner count must agree within 5 % (at least 4) and the refinements
    within 2; the solutions within the rtol bound."""
    nx, ny, nz = shape
    cav = cfd.Cavity(cfd.make_params(nx, ny, nz, solver="ir", ir_delta=delta))
    cav.set_ir_form(form)
    b = gaussian_rhs(nx, ny, nz, seed=17)
    bg = torch.tensor(b, device="cuda")
    xg = torch.zeros_like(bg)
    rc, st = cav.solve_pressure(bg, xg)
    assert rc == cfd.CFD_OK, st
    A = poisson_csr(nx, ny, nz)
    xo, so = ir_cg(A, b.ravel(), rtol=RTOL, delta=delta, max_iters=20 * max(shape))
    assert so.converged, so
    assert abs(st["iters"] - so.iters) <= max(4, so.iters // 20), (st["iters"], so.iters)
    assert abs(st["outer_iters"] - so.refinements) <= 2, (st["outer_iters"], so.refinements)
    x = xg.cpu().numpy().ravel()
    bo = b.ravel() - b.mean()
    d = (x - x.mean()) - (xo - xo.mean())
    assert np.linalg.norm(d) <= 2 * RTOL * np.linalg.norm(bo) / lam_min(shape)
    print(f"IR {form} {shape} delta {delta}: GPU {st['iters']} it / {st['outer_iters']} ref, "
          f"oracle {so.iters} it / {so.refinements} ref")
