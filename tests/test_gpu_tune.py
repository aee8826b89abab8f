"""GPU checks of the solver-shape autotuner (cfd_autotune_solver)."""
import pytest

torch = pytest.importorskip("torch")

from paper_2504_03697_gb300.synthetic import cavity_perturbation  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cfd():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2504_03697_gb300 import build as B
    B.build()
    from paper_2504_03697_gb300 import cfd as _cfd
    return _cfd


@pytest.mark.parametrize("n,solver", [(48, "cg"), (40, "ir")])
def test_autotune_keeps_state_and_picks_a_listed_shape(cfd, n, solver):
    cav = cfd.Cavity(cfd.make_params(n, n, n, nu=1e-3, solver=solver))
    for name, f in zip("uvw", cavity_perturbation(n, n, n, 3)):
        cav.set_field(name, f)
    cav.step(2)
    before = {f: torch.as_tensor(cav.read_field(f)).clone() for f in "uvwp"}
    rep = cav.autotune(iters=30)
    after = {f: torch.as_tensor(cav.read_field(f)) for f in "uvwp"}
    for f in "uvwp":
        assert torch.equal(before[f], after[f]), f
    # CG: both forms x (automatic + 16 shapes); IR: the automatic form, the
    # 17 shapes of the persistent form and the graph form (n % 4 == 0)
    assert rep["candidates"] == (34 if solver == "cg" else 19)
    assert rep["cg_variant"] in (0, 1)
    assert rep["ir_form"] in ((0,) if solver == "cg" else (0, 1, 2))
    assert (rep["blocks_per_sm"], rep["tile_depth"]) == (0, 0) or (
        rep["blocks_per_sm"] in (1, 2, 3, 4) and rep["tile_depth"] in (1, 2, 4, 8))
    assert 0 < rep["ms_best"] <= rep["ms_auto"]
    print(f"{n}^3 {solver}: auto {rep['ms_auto']:.3f} ms, best {rep['ms_best']:.3f} ms at "
          f"bps {rep['blocks_per_sm']} tz {rep['tile_depth']}")
    # the chosen shape is the one the next solves use, and steps still converge
    rc, stats = cav.step(2)
    assert rc == 0 and all(s["status"] == 0 and s["rel_resid"] <= 1e-8 for s in stats)
