"""GPU checks of the learned preconditioner in mixed precision.

Two device-resident paths, both one CUDA graph per solve:

* flexible CG with the U-Net as preconditioner, FP32 vectors and FP64
  reliable-update refinement (solver FPCG, graph form), against the
  oracle's model of the same method, ``oracle.krylov.ir_fpcg``, driven by
  the oracle's network with BF16 storage (``oracle.unet.bf16_store``, the
  CUDA network's precision): iteration and refinement counts, the plain-CG
  fall-back, the kernels the graph runs, and whole cavity steps against the
  oracle's step;
* the learned initial guess x0 = alpha M(b) in front of the mixed-precision
  solve (solver IR, learned_guess = 1): x0 against the oracle's network and
  line search, the solve from it against ``oracle.krylov.ir_cg`` started
  from the oracle's x0, and whole cavity steps.

Every solve is judged by the FP64 true residual and compared with the
oracle within the rtol bound (2 rtol ||b|| / lambda_min, mean removed).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import unet as ou  # noqa: E402
from oracle.krylov import ir_cg, ir_fpcg, pcg  # noqa: E402
from oracle.mac import Cavity as OCav  # noqa: E402
from oracle.operators import poisson_csr  # noqa: E402
from paper_2504_03697_gb300.synthetic import cavity_perturbation, gaussian_rhs  # noqa: E402
from tests.test_gpu_oracle_paths import check_step_against_oracle, passthrough_params, read_state  # noqa: E402

pytestmark = pytest.mark.gpu

RTOL = 1e-8
NET_KERNELS = 13  # first layer, 7 tensor-core convolutions, 2 poolings, 2 up-samplings, head


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


def oracle_net(params, shape):
    nx, ny, nz = shape
    layers = ou.unflatten(params.double())
    return lambda r: ou.precondition(layers, r.reshape(nz, ny, nx), store=ou.bf16_store).ravel()


def check_solution(shape, b, x, st, xo):
    nx, ny, nz = shape
    A = poisson_csr(nx, ny, nz)
    bo = b.ravel() - b.mean()
    true_rel = np.linalg.norm(bo - A @ x) / np.linalg.norm(bo)
    assert true_rel <= RTOL * 1.0001, true_rel
    np.testing.assert_allclose(true_rel, st["rel_resid"], rtol=1e-6, atol=1e-14)
    d = (x - x.mean()) - (xo - xo.mean())
    bound = 2 * RTOL * np.linalg.norm(bo) / lam_min(shape)
    assert np.linalg.norm(d) <= bound, (np.linalg.norm(d), bound)
    return np.abs(d).max(), bound


def fpcg_cavity(cfd, shape, params, **kw):
    cav = cfd.Cavity(cfd.make_params(*shape, solver="fpcg", **kw))
    net = cfd.UNet(*shape, seed=0)
    net.set_params(params)
    cav.attach_preconditioner(net)
    cav._net = net
    return cav


@pytest.mark.parametrize("shape,w,delta", [((16, 16, 16), (1.0, 1.0), 0.1), ((24, 20, 16), (4.0, 4.0), 0.1),
                                           ((16, 12, 8), (4.0, 4.0), 0.01)])
def test_fpcg_graph_matches_oracle_mixed_precision_model(cfd, shape, w, delta):
    nx, ny, nz = shape
    params = passthrough_params(*w)
    cav = fpcg_cavity(cfd, shape, params, ir_delta=delta)
    b = gaussian_rhs(nx, ny, nz, seed=41)
    bg = torch.tensor(b, device="cuda")
    xg = torch.zeros_like(bg)
    l0 = cav.launch_count()
    rc, st = cav.solve_pressure(bg, xg)
    assert rc == cfd.CFD_OK, st
    assert st["restarts"] == 0, st  # no iteration ran as plain CG
    # kernels: prologue 2, each outer pass 2, each iteration 4 + the network, epilogue 3
    assert cav.launch_count() - l0 == 2 + 2 * (st["outer_iters"] + 1) + (4 + NET_KERNELS) * st["iters"] + 3
    A = poisson_csr(nx, ny, nz)
    xo, so = ir_fpcg(A, b.ravel(), oracle_net(params, shape), rtol=RTOL, delta=delta, max_iters=20 * max(shape))
    assert so.converged and so.plain_iters == 0, so
    assert abs(st["iters"] - so.iters) <= max(3, so.iters // 20), (st["iters"], so.iters)
    assert abs(st["outer_iters"] - so.refinements) <= 2, (st["outer_iters"], so.refinements)
    dmax, bound = check_solution(shape, b, xg.cpu().numpy().ravel(), st, xo)
    _, scg = pcg(A, b.ravel() - b.mean(), rtol=RTOL, max_iters=10 ** 5)
    print(f"FPCG graph {shape} w={w} delta={delta}: GPU {st['iters']} it / {st['outer_iters']} ref, "
          f"oracle {so.iters} / {so.refinements} (FP64 CG {scg.iters}); max|dx| {dmax:.2e} (bound {bound:.2e})")


def test_fpcg_graph_falls_back_to_plain_cg(cfd):
    """A zero network gives z = 0, so z~.r = 0: plain CG from the first
    iteration (every iteration counted as plain; the network node runs once
    and is skipped after), as in the oracle's model with the same network.
    A random (untrained) network is an indefinite, non-symmetric operator:
    the solve must still meet the FP64 tolerance, by its own steps or after
    falling back; its counts are printed, not compared (the switch point of
    a stagnating recurrence depends on rounding)."""
    shape = (16, 16, 16)
    nx, ny, nz = shape
    b = gaussian_rhs(nx, ny, nz, seed=42)
    A = poisson_csr(nx, ny, nz)
    bm = b.ravel() - b.mean()
    xcg, _ = pcg(A, bm, rtol=RTOL, max_iters=10 ** 5)
    zero = torch.zeros(ou.param_count())
    cav = fpcg_cavity(cfd, shape, zero)
    bg = torch.tensor(b, device="cuda")
    xg = torch.zeros_like(bg)
    l0 = cav.launch_count()
    rc, st = cav.solve_pressure(bg, xg)
    assert rc == cfd.CFD_OK, st
    assert st["restarts"] == st["iters"] > 0, st
    # the network ran once (the first f_norm); the plain iterations skip it
    assert cav.launch_count() - l0 == 2 + 2 * (st["outer_iters"] + 1) + 4 * st["iters"] + NET_KERNELS + 3
    xo, so = ir_fpcg(A, b.ravel(), oracle_net(zero, shape), rtol=RTOL, max_iters=20 * max(shape))
    assert so.converged and so.plain_iters == so.iters
    assert abs(st["iters"] - so.iters) <= max(3, so.iters // 20), (st["iters"], so.iters)
    check_solution(shape, b, xg.cpu().numpy().ravel(), st, xo)
    rand = torch.from_numpy(np.random.default_rng(3).standard_normal(ou.param_count()) * 0.1).float()
    cav = fpcg_cavity(cfd, shape, rand)
    xg.zero_()
    rc, st = cav.solve_pressure(bg, xg)
    assert rc == cfd.CFD_OK, st
    check_solution(shape, b, xg.cpu().numpy().ravel(), st, xcg)
    print(f"random network: {st['iters']} iterations, {st['restarts']} as plain CG, {st['outer_iters']} refinements")


@pytest.mark.parametrize("shape", [(16, 16, 16), (24, 20, 16)])
def test_fpcg_graph_cavity_steps_match_oracle_per_step(cfd, shape):
    nx, ny, nz = shape
    cav = fpcg_cavity(cfd, shape, passthrough_params(4.0, 4.0), dt=0.01, nu=0.01, lid_u=1.0)
    ocav = OCav(nx, ny, nz, dt=0.01, nu=0.01, lid_u=1.0)
    for name, f in zip("uvw", cavity_perturbation(nx, ny, nz, seed=5, amp=1e-3)):
        cav.set_field(name, f)
    for k in range(3):
        start = read_state(cav)
        rc, st = cav.step(1)
        assert rc == cfd.CFD_OK, st
        assert st[0]["restarts"] == 0 and st[0]["diff_iters"][0] >= 1
        errs, fv, fp = check_step_against_oracle(ocav, start, read_state(cav), st[0], f"fpcg {shape} step {k}")
        print(f"FPCG graph cavity {shape} step {k}: {st[0]['iters']} it; max-abs {errs}, {fv:.2e} / {fp:.2e} "
              f"of the bound")


def test_fpcg_host_form_still_selectable(cfd):
    shape = (16, 16, 16)
    cav = fpcg_cavity(cfd, shape, passthrough_params(1.0, 1.0))
    cav.set_fpcg_form("host")
    b = torch.tensor(gaussian_rhs(*shape, seed=43), device="cuda")
    x = torch.zeros_like(b)
    rc, st = cav.solve_pressure(b, x)
    assert rc == cfd.CFD_OK and st["rel_resid"] <= RTOL and st["outer_iters"] == 0
    with pytest.raises(cfd.CfdError):
        cfd.Cavity(cfd.make_params(16, 16, 16, solver="ir")).set_fpcg_form("graph")


def guess_cavity(cfd, shape, params, **kw):
    cav = cfd.Cavity(cfd.make_params(*shape, solver="ir", learned_guess=True, **kw))
    net = cfd.UNet(*shape, seed=0)
    net.set_params(params)
    cav.attach_preconditioner(net)
    cav._net = net
    return cav


def oracle_guess(params, shape, b):
    """x0 = alpha z~, z~ = M(b - mean b) (the network, BF16 storage, mean
    removed), alpha = z~.b / z~.A z~."""
    nx, ny, nz = shape
    bm = b.ravel() - b.mean()
    zt = oracle_net(params, shape)(bm)
    A = poisson_csr(nx, ny, nz)
    return (zt @ bm) / (zt @ (A @ zt)) * zt


@pytest.mark.parametrize("shape,w", [((16, 16, 16), (1.0, 1.0)), ((24, 20, 16), (4.0, 4.0))])
def test_learned_guess_matches_oracle_and_solve_from_it(cfd, shape, w):
    nx, ny, nz = shape
    params = passthrough_params(*w)
    cav = guess_cavity(cfd, shape, params)
    b = gaussian_rhs(nx, ny, nz, seed=44)
    bg = torch.tensor(b, device="cuda")
    x0 = torch.zeros_like(bg)
    cav.learned_guess(bg, x0)
    torch.cuda.synchronize()
    x0o = oracle_guess(params, shape, b)
    g = x0.cpu().numpy().ravel()
    rel = np.linalg.norm(g - x0o) / np.linalg.norm(x0o)
    assert rel <= 1e-3, rel
    # the solve starting from it
    xg = torch.full_like(bg, 3.0)  # the guess replaces whatever x holds
    l0 = cav.launch_count()
    rc, st = cav.solve_pressure(bg, xg)
    assert rc == cfd.CFD_OK, st
    ran, base = cav.launch_count() - l0, 4 + NET_KERNELS + 2 + 2 * (st["outer_iters"] + 1) + 2 * st["iters"] + 3
    # plus the kernels that return at once in the last pass of each inner
    # loop (4 FP32 iterations per pass of its body)
    assert (ran - base) % 2 == 0 and 0 <= ran - base <= 6 * (st["outer_iters"] + 1), (ran, base, st)
    A = poisson_csr(nx, ny, nz)
    xo, so = ir_cg(A, b.ravel(), rtol=RTOL, delta=0.01, x0=x0o, max_iters=20 * max(shape))
    _, cold = ir_cg(A, b.ravel(), rtol=RTOL, delta=0.01, max_iters=20 * max(shape))
    assert so.converged
    assert abs(st["iters"] - so.iters) <= max(4, so.iters // 20), (st["iters"], so.iters)
    dmax, bound = check_solution(shape, b, xg.cpu().numpy().ravel(), st, xo)
    print(f"learned guess {shape} w={w}: |x0 - oracle| / |x0| {rel:.1e}; IR from it GPU {st['iters']} it, "
          f"oracle {so.iters} (cold start {cold.iters}); max|dx| {dmax:.2e}")


def test_learned_guess_of_a_zero_network_is_the_cold_start(cfd):
    shape = (24, 20, 16)
    nx, ny, nz = shape
    b = torch.tensor(gaussian_rhs(nx, ny, nz, seed=45), device="cuda")
    cav = guess_cavity(cfd, shape, torch.zeros(ou.param_count()))
    x1 = torch.zeros_like(b)
    rc, s1 = cav.solve_pressure(b, x1)
    ref = cfd.Cavity(cfd.make_params(*shape, solver="ir"))
    ref.set_ir_form("graph")
    x2 = torch.zeros_like(b)
    rc2, s2 = ref.solve_pressure(b, x2)
    assert rc == rc2 == cfd.CFD_OK
    assert s1["iters"] == s2["iters"] and s1["outer_iters"] == s2["outer_iters"]
    assert torch.equal(x1, x2)


def test_learned_guess_cavity_steps_match_oracle_per_step(cfd):
    shape = (16, 16, 16)
    nx, ny, nz = shape
    cav = guess_cavity(cfd, shape, passthrough_params(4.0, 4.0), dt=0.01, nu=0.01, lid_u=1.0)
    ocav = OCav(nx, ny, nz, dt=0.01, nu=0.01, lid_u=1.0)
    for name, f in zip("uvw", cavity_perturbation(nx, ny, nz, seed=6, amp=1e-3)):
        cav.set_field(name, f)
    for k in range(3):
        start = read_state(cav)
        rc, st = cav.step(1)
        assert rc == cfd.CFD_OK, st
        errs, fv, fp = check_step_against_oracle(ocav, start, read_state(cav), st[0], f"guess step {k}")
        print(f"learned guess cavity step {k}: {st[0]['iters']} it; max-abs {errs}, {fv:.2e} / {fp:.2e} of the bound")


def test_learned_correction_of_the_warm_start(cfd):
    """learned_guess with warm_start: the network corrects the previous
    pressure (x0 = x + alpha M(b - A x)).  A zero network leaves the warm
    start as it is (the solve is bitwise the plain warm-started IR graph
    solve); cavity steps with the pass-through network against the oracle
    per step."""
    shape = (24, 20, 16)
    nx, ny, nz = shape
    b = torch.tensor(gaussian_rhs(nx, ny, nz, seed=46), device="cuda")
    x_start = torch.tensor(gaussian_rhs(nx, ny, nz, seed=47), device="cuda") * 0.01
    cav = guess_cavity(cfd, shape, torch.zeros(ou.param_count()), warm_start=True)
    x1 = x_start.clone()
    rc, s1 = cav.solve_pressure(b, x1)
    ref = cfd.Cavity(cfd.make_params(*shape, solver="ir", warm_start=True))
    ref.set_ir_form("graph")
    x2 = x_start.clone()
    rc2, s2 = ref.solve_pressure(b, x2)
    assert rc == rc2 == cfd.CFD_OK
    assert s1["iters"] == s2["iters"] and torch.equal(x1, x2)
    cav = guess_cavity(cfd, (16, 16, 16), passthrough_params(4.0, 4.0), dt=0.01, nu=0.01, lid_u=1.0, warm_start=True)
    ocav = OCav(16, 16, 16, dt=0.01, nu=0.01, lid_u=1.0)
    for name, f in zip("uvw", cavity_perturbation(16, 16, 16, seed=7, amp=1e-3)):
        cav.set_field(name, f)
    for k in range(3):
        start = read_state(cav)
        rc, st = cav.step(1)
        assert rc == cfd.CFD_OK, st
        errs, fv, fp = check_step_against_oracle(ocav, start, read_state(cav), st[0], f"warm guess step {k}")
        print(f"learned correction of the warm start, step {k}: {st[0]['iters']} it; {fv:.2e} / {fp:.2e} of the bound")


def test_learned_paths_argument_checks(cfd):
    with pytest.raises(cfd.CfdError):
        cfd.Cavity(cfd.make_params(16, 16, 16, solver="cg", learned_guess=True))
    with pytest.raises(cfd.CfdError):
        cfd.Cavity(cfd.make_params(18, 16, 16, solver="ir", learned_guess=True))
    cav = cfd.Cavity(cfd.make_params(16, 16, 16, solver="ir", learned_guess=True))
    b = torch.tensor(gaussian_rhs(16, 16, 16, seed=1), device="cuda")
    with pytest.raises(cfd.CfdError):
        cav.solve_pressure(b, torch.zeros_like(b))  # no network attached
    plain = cfd.Cavity(cfd.make_params(16, 16, 16, solver="ir"))
    with pytest.raises(cfd.CfdError):
        plain.attach_preconditioner(cfd.UNet(16, 16, 16))
    with pytest.raises(cfd.CfdError):
        cfd.Batch([cfd.make_params(16, 16, 16, solver="ir", learned_guess=True)])
