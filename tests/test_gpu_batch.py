"""GPU checks of batched cavities (one persistent launch per solve family).

Every cavity of a batch must match the FP64 oracle run on that cavity alone
(replaying the batch's per-step iteration counts), at the same 1e-10
tolerance as single cavities; a graph-captured batch must reproduce the
directly launched one bit for bit.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import fractional_step as fs  # noqa: E402
from oracle.mac import Cavity as OCav  # noqa: E402
from paper_2504_03697_gb300.synthetic import cavity_perturbation  # noqa: E402

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-10

SPECS = [((16, 16, 16), 0.01), ((24, 20, 16), 0.01), ((32, 32, 32), 0.005), ((12, 12, 12), 0.0), ((20, 20, 20), 0.02)]


@pytest.fixture(scope="module")
def cfd():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2504_03697_gb300 import build as B
    B.build()
    from paper_2504_03697_gb300 import cfd as _cfd
    return _cfd


def _batch(cfd, specs, solver="cg", seed0=30):
    prms = [cfd.make_params(*shape, dt=0.01, nu=nu, lid_u=1.0, solver=solver) for shape, nu in specs]
    b = cfd.Batch(prms)
    inits = []
    for i, (shape, nu) in enumerate(specs):
        init = cavity_perturbation(*shape, seed=seed0 + i, amp=1e-2)
        inits.append(init)
        for name, f in zip("uvw", init):
            b.cavity(i).set_field(name, f)
    return b, inits


def rel_err(g, o):
    return float(np.abs(np.asarray(g) - o).max() / max(np.abs(o).max(), 1e-300))


def test_batch_matches_oracle_per_cavity(cfd):
    b, inits = _batch(cfd, SPECS)
    steps = 4
    per_step = []
    for _ in range(steps):
        rc, st = b.step(1)
        assert rc == cfd.CFD_OK
        per_step.append(st)
    for i, (shape, nu) in enumerate(SPECS):
        ocav = OCav(*shape, dt=0.01, nu=nu, lid_u=1.0)
        fixed = [{"p": per_step[s][i]["iters"], "u": per_step[s][i]["diff_iters"][0] if nu > 0 else None,
                  "v": per_step[s][i]["diff_iters"][1] if nu > 0 else None,
                  "w": per_step[s][i]["diff_iters"][2] if nu > 0 else None} for s in range(steps)]
        st, _ = fs.simulate(ocav, fs.initial_state(ocav, inits[i]), steps, fixed_iters_per_step=fixed)
        for k, name in enumerate("uvwp"):
            e = rel_err(b.cavity(i).read_field(name).numpy(), st[k])
            assert e < FP64_TOL, (i, name, e)
        assert all(per_step[s][i]["rel_resid"] <= 1e-8 for s in range(steps))


def test_batch_graph_replay_is_bitwise_equal(cfd):
    b1, _ = _batch(cfd, SPECS[:3])
    b2, _ = _batch(cfd, SPECS[:3])
    b2.use_graph(True)
    b1.step(3, stats=False)
    b2.step(3, stats=False)
    assert b2.graph_active(), b2.lib.cfd_batch_last_error(b2.b)
    for i in range(3):
        for name in "uvwp":
            np.testing.assert_array_equal(b1.cavity(i).read_field(name).numpy(), b2.cavity(i).read_field(name).numpy())


def test_batch_mixed_precision_converges(cfd):
    specs = [((32, 32, 32), 0.001), ((48, 40, 32), 0.001), ((24, 24, 24), 0.001)]
    b, _ = _batch(cfd, specs, solver="ir")
    rc, st = b.step(3)
    assert rc == cfd.CFD_OK
    for s in st:
        assert s["rel_resid"] <= 1e-8 and s["outer_iters"] >= 1


def test_batch_rejects_mixed_solvers(cfd):
    prms = [cfd.make_params(8, 8, 8, solver="cg"), cfd.make_params(8, 8, 8, solver="ir")]
    with pytest.raises(cfd.CfdError):
        cfd.Batch(prms)



def test_batch_mixed_precision_diffusion_matches_single_cavities(cfd):
    """With the IR solver the batch also runs its diffusion solves as FP32 CG
    with FP64 refinement (one multi-problem launch per component).  Each
    cavity must agree with the same cavity stepped alone by the IR solver
    (persistent form, whose solves are checked against the oracle within the
    rtol bounds in test_gpu_ir.py) to the solves' tolerance: both meet
    ||b - A x|| <= 1e-8 ||b|| in every solve, in other block decompositions."""
    specs = [((24, 24, 24), 0.01), ((32, 28, 20), 0.005), ((16, 16, 16), 0.02)]
    b, inits = _batch(cfd, specs, solver="ir")
    rc, st = b.step(2)
    assert rc == cfd.CFD_OK
    for s in st:
        assert s["rel_resid"] <= 1e-8 and s["diff_status"] == cfd.CFD_OK and s["diff_iters"][0] >= 1
    for i, (shape, nu) in enumerate(specs):
        cav = cfd.Cavity(cfd.make_params(*shape, dt=0.01, nu=nu, lid_u=1.0, solver="ir"))
        cav.set_ir_form("persistent")
        for name, f in zip("uvw", inits[i]):
            cav.set_field(name, f)
        rc1, _ = cav.step(2)
        assert rc1 == cfd.CFD_OK
        for name in "uvwp":
            g = b.cavity(i).read_field(name).numpy()
            ref = cav.read_field(name).numpy()
            scale = max(np.abs(ref).max(), 1e-300)
            assert np.abs(g - ref).max() <= 1e-6 * scale, (i, name)


def test_batch_forces_subset_and_odd_widths_match_oracle(cfd):
    """The batched sweeps: forces apply to the cavities with g != 0 only
    (their own table), on widths that are not multiples of 4; every cavity
    equals the oracle run alone (iteration counts replayed) at 1e-10."""
    specs = [((9, 7, 6), dict(nu=0.01, g=(0.5, -0.25, 2.0))), ((13, 11, 7), dict(nu=0.0, g=(0.0, 0.0, 0.0))),
             ((10, 8, 6), dict(nu=0.02, g=(1.0, 0.0, -0.5))), ((17, 9, 13), dict(nu=0.005, g=(0.0, 0.0, 0.0)))]
    prms = [cfd.make_params(*shape, dt=0.01, lid_u=1.0, solver="cg", **kw) for shape, kw in specs]
    b = cfd.Batch(prms)
    inits = []
    for i, (shape, _) in enumerate(specs):
        init = cavity_perturbation(*shape, seed=50 + i, amp=1e-2)
        inits.append(init)
        for name, f in zip("uvw", init):
            b.cavity(i).set_field(name, f)
    steps = 3
    per_step = []
    for _ in range(steps):
        rc, st = b.step(1)
        assert rc == cfd.CFD_OK
        per_step.append(st)
    for i, (shape, kw) in enumerate(specs):
        ocav = OCav(*shape, dt=0.01, lid_u=1.0, **kw)
        nu = kw["nu"]
        fixed = [{"p": per_step[s][i]["iters"], "u": per_step[s][i]["diff_iters"][0] if nu > 0 else None,
                  "v": per_step[s][i]["diff_iters"][1] if nu > 0 else None,
                  "w": per_step[s][i]["diff_iters"][2] if nu > 0 else None} for s in range(steps)]
        st, _ = fs.simulate(ocav, fs.initial_state(ocav, inits[i]), steps, fixed_iters_per_step=fixed)
        for k, name in enumerate("uvwp"):
            e = rel_err(b.cavity(i).read_field(name).numpy(), st[k])
            assert e < FP64_TOL, (i, name, e)
