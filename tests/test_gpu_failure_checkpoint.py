"""Failure detection and checkpoint / resume on the GPU.

Failure detection without a GPU fault: every grid-wide wait of the
persistent solve kernels has a time limit (cfd_set_wait_limit).  With the
limit at 0 the first block that finds a grid barrier unsatisfied gives up,
records CFD_ERR_TIMEOUT and returns; the other blocks see the error at their
next wait and return too.  Nothing hangs and nothing faults: the test
checks that the call reports the timeout, and that the same handle, with
the default limit restored, then solves the same system to the rtol.

Checkpoint / resume: the state of a cavity is its four fields (u, v, w, p;
Sec. 3.1, the paper writes them to a CSV snapshot each step).  Ten steps,
a read-back of the fields, a new handle set from them and ten more steps
must give bitwise the fields of twenty steps on one handle (the kernels,
launch shapes and reduction orders are the same for the same grid).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle.operators import poisson_csr  # noqa: E402
from paper_2504_03697_gb300.synthetic import cavity_perturbation, gaussian_rhs  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cfd():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2504_03697_gb300 import build as B
    B.build()
    from paper_2504_03697_gb300 import cfd as _cfd
    return _cfd


@pytest.mark.parametrize("solver", ["cg", "jacobi"])
def test_grid_wait_limit_reports_timeout_and_handle_recovers(cfd, solver):
    n = 64
    cav = cfd.Cavity(cfd.make_params(n, n, n, solver=solver))
    b = torch.tensor(gaussian_rhs(n, n, n, seed=3), device="cuda")
    x = torch.zeros_like(b)
    cav.set_wait_limit(0)
    rc, st = cav.solve_pressure(b, x)
    assert rc == cfd.CFD_ERR_TIMEOUT, (rc, st)
    assert b"timed out" in cav.lib.cfd_last_error(cav.h)
    cav.set_wait_limit(None)  # back to the default limit
    x.zero_()
    rc, st = cav.solve_pressure(b, x)
    assert rc == cfd.CFD_OK and st["rel_resid"] <= 1e-8, st
    A = poisson_csr(n, n, n)
    bo = b.cpu().numpy().ravel()
    bo = bo - bo.mean()
    true_rel = np.linalg.norm(bo - A @ x.cpu().numpy().ravel()) / np.linalg.norm(bo)
    assert true_rel <= 1.0001e-8


def test_timeout_inside_a_step_is_reported(cfd):
    n = 32
    cav = cfd.Cavity(cfd.make_params(n, n, n, nu=0.01, solver="cg"))
    for name, f in zip("uvw", cavity_perturbation(n, n, n, seed=1, amp=1e-3)):
        cav.set_field(name, f)
    cav.set_wait_limit(0)
    rc, _ = cav.step(1)
    assert rc == cfd.CFD_ERR_TIMEOUT
    cav.set_wait_limit(None)
    rc, st = cav.step(2)
    assert rc == cfd.CFD_OK and all(s["rel_resid"] <= 1e-8 for s in st)


@pytest.mark.parametrize("solver,warm", [("cg", False), ("cg", True), ("ir", True)])
def test_checkpoint_resume_is_bitwise(cfd, solver, warm):
    shape = (24, 20, 16)
    prm = dict(dt=0.01, nu=0.01, lid_u=1.0, solver=solver, warm_start=warm)
    init = cavity_perturbation(*shape, seed=7, amp=1e-3)

    def fresh():
        c = cfd.Cavity(cfd.make_params(*shape, **prm))
        return c

    whole = fresh()
    for name, f in zip("uvw", init):
        whole.set_field(name, f)
    rc, _ = whole.step(20)
    assert rc == cfd.CFD_OK
    ref = {f: whole.read_field(f).numpy() for f in "uvwp"}

    first = fresh()
    for name, f in zip("uvw", init):
        first.set_field(name, f)
    rc, _ = first.step(10)
    assert rc == cfd.CFD_OK
    saved = {f: first.read_field(f).numpy().copy() for f in "uvwp"}
    first.close()

    resumed = fresh()
    for f in "uvwp":
        resumed.set_field(f, saved[f])
    rc, _ = resumed.step(10)
    assert rc == cfd.CFD_OK
    for f in "uvwp":
        np.testing.assert_array_equal(resumed.read_field(f).numpy(), ref[f], err_msg=f)
