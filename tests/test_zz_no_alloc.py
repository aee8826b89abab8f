"""The allocation-free pressure solve (cfd_poisson_solve_noalloc).

Callers that may not allocate device memory (plug-ins whose host owns every
allocation, runtimes that reserve all memory up front) cannot give the
library the workspace cfd_create needs; this entry point keeps its scratch
in a fixed __device__ array instead.  It runs the two-reduction CG form
(the library's default is the single-reduction form), so the iteration
counts may differ by one.  The test calls it
through the C-ABI twice in a row, on two different right-hand sides, and
checks each result against the workspace-based cfd_solve_pressure within
the FP64 parity tolerance of the other GPU tests.  The second call also
shows that the scratch left over from the first call does not leak in.

This file is collected last on purpose, so that a run stopping at the
first failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2504_03697_gb300.synthetic import gaussian_rhs  # noqa: E402

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-10


def test_noalloc_matches_workspace_solve_twice():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2504_03697_gb300 import build as B
    B.build()
    from paper_2504_03697_gb300 import cfd

    lib = cfd.load_library()
    nx, ny, nz = 48, 40, 32
    stream = torch.cuda.current_stream()
    cav = cfd.Cavity(cfd.make_params(nx, ny, nz, rtol=1e-8))
    for seed in (11, 12):
        b = torch.tensor(gaussian_rhs(nx, ny, nz, seed=seed), device="cuda")
        x_ref = torch.zeros_like(b)
        rc, st_ref = cav.solve_pressure(b, x_ref)
        assert rc == cfd.CFD_OK
        x = torch.full_like(b, 7.0)  # garbage start: the solve must overwrite it
        st = cfd.cfd_solve_stats()
        rc = lib.cfd_poisson_solve_noalloc(nx, ny, nz, ctypes.c_void_p(b.data_ptr()), ctypes.c_void_p(x.data_ptr()),
                                           1e-8, 0, ctypes.c_void_p(stream.cuda_stream), ctypes.byref(st))
        assert rc == cfd.CFD_OK, lib.cfd_last_error(None)
        assert st.status == cfd.CFD_OK and st.rel_resid <= 1e-8
        assert abs(st.iters - st_ref["iters"]) <= 1
        xr = x_ref.cpu().numpy()
        err = np.abs(x.cpu().numpy() - xr).max() / np.abs(xr).max()
        assert err < FP64_TOL, (seed, err)

    # grids beyond the fixed scratch are refused before any device work
    big = cfd.cfd_solve_stats()
    rc = lib.cfd_poisson_solve_noalloc(65, 64, 64, ctypes.c_void_p(b.data_ptr()), ctypes.c_void_p(x.data_ptr()),
                                       1e-8, 0, ctypes.c_void_p(stream.cuda_stream), ctypes.byref(big))
    assert rc == cfd.CFD_ERR_INVALID_ARG
    assert b"CFD_NOALLOC_MAX_CELLS" in lib.cfd_last_error(None)
