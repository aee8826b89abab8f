"""Host-side checks of the C-ABI library (no GPU): it builds, loads, exports
every function declared in include/cfd.h, and its host logic validates
parameters and sizes workspaces without touching a device."""
import ctypes
import os
import re

import pytest

from paper_2504_03697_gb300 import build as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    from paper_2504_03697_gb300 import cfd
    return cfd.load_library()


def declared_functions():
    names = set()
    for hdr in os.listdir(os.path.join(ROOT, "include")):
        if not hdr.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", hdr)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w\s\*]*?\b(cfd\w*)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ["cfd_workspace_bytes", "cfd_create", "cfd_destroy", "cfd_step", "cfd_solve_pressure",
                 "cfd_read_field", "cfd_set_field", "cfd_last_error", "cfd_apply_poisson", "cfd_substep"]:
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_workspace_size_and_validation(lib):
    from paper_2504_03697_gb300 import cfd
    small = cfd.cfd_workspace_bytes(cfd.make_params(16, 16, 16))
    big = cfd.cfd_workspace_bytes(cfd.make_params(64, 64, 64))
    assert big > small > 0
    # FP64: 7 field arrays + 5 solver vectors of at least N^3 doubles
    assert big >= 12 * 64 ** 3 * 8
    ir = cfd.cfd_workspace_bytes(cfd.make_params(64, 64, 64, solver="ir"))
    assert ir >= big + 5 * 64 ** 3 * 4
    bad = [dict(nx=0), dict(dt=0.0), dict(rho=-1.0), dict(nu=-1e-3), dict(rtol=0.0), dict(rtol=1.5),
           dict(solver=7), dict(max_iters=-2), dict(lid_u=float("inf"))]
    for kw in bad:
        args = dict(nx=8, ny=8, nz=8)
        args.update(kw)
        nx, ny, nz = args.pop("nx"), args.pop("ny"), args.pop("nz")
        with pytest.raises(cfd.CfdError) as ei:
            cfd.cfd_workspace_bytes(cfd.make_params(nx, ny, nz, **args))
        assert ei.value.code == cfd.CFD_ERR_INVALID_ARG


def test_create_rejects_bad_workspace_without_a_device(lib):
    from paper_2504_03697_gb300 import cfd
    prm = cfd.make_params(8, 8, 8)
    h = ctypes.c_void_p(0)
    rc = lib.cfd_create(ctypes.byref(prm), None, 0, None, ctypes.byref(h))
    assert rc == cfd.CFD_ERR_INVALID_ARG and not h.value
    assert b"NULL" in lib.cfd_last_error(None)
    need = cfd.cfd_workspace_bytes(prm)
    rc = lib.cfd_create(ctypes.byref(prm), ctypes.c_void_p(256), need - 256, None, ctypes.byref(h))
    assert rc == cfd.CFD_ERR_WORKSPACE_TOO_SMALL
    rc = lib.cfd_create(ctypes.byref(prm), ctypes.c_void_p(257), need, None, ctypes.byref(h))
    assert rc == cfd.CFD_ERR_INVALID_ARG  # not 256-byte aligned


def test_binding_refuses_to_run_without_cuda(lib):
    import torch
    from paper_2504_03697_gb300 import cfd
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(RuntimeError):
        cfd.Cavity(cfd.make_params(8, 8, 8))


def test_more_parameter_validation_and_sizes(lib):
    from paper_2504_03697_gb300 import cfd
    base = cfd.cfd_workspace_bytes(cfd.make_params(32, 32, 32))
    dic = cfd.cfd_workspace_bytes(cfd.make_params(32, 32, 32, solver="dic"))
    assert dic >= base + 32 ** 3 * 8  # the DIC pivots
    for kw in (dict(advect_order=3), dict(advect_order=-1)):
        with pytest.raises(cfd.CfdError):
            cfd.cfd_workspace_bytes(cfd.make_params(8, 8, 8, **kw))
    prm = cfd.make_params(8, 8, 8)
    prm.reserved[3] = 1
    with pytest.raises(cfd.CfdError):
        cfd.cfd_workspace_bytes(prm)


def test_csr_sizes_match_the_closed_form(lib):
    for shape in [(1, 1, 1), (1, 1, 7), (4, 3, 2), (64, 64, 64)]:
        nb = ctypes.c_size_t(0)
        nnz = ctypes.c_int64(0)
        assert lib.cfd_csr_bytes(*shape, ctypes.byref(nb), ctypes.byref(nnz)) == 0
        nx, ny, nz = shape
        n = nx * ny * nz
        assert nnz.value == 7 * n - 2 * (nx * ny + ny * nz + nz * nx)
        a16 = lambda x: (x + 15) // 16 * 16  # noqa: E731
        assert nb.value == a16((n + 1) * 4) + a16(nnz.value * 4) + nnz.value * 8
    assert lib.cfd_csr_bytes(0, 4, 4, ctypes.byref(nb), None) != 0
    assert lib.cfd_csr_bytes(1024, 1024, 1024, ctypes.byref(nb), None) != 0  # 7 n >= 2^31


def test_unet_workspace_needs_multiples_of_four(lib):
    nb = ctypes.c_size_t(0)
    assert lib.cfd_unet_workspace_bytes(16, 12, 8, ctypes.byref(nb)) == 0
    small = nb.value
    assert lib.cfd_unet_workspace_bytes(32, 32, 32, ctypes.byref(nb)) == 0
    assert nb.value > small > 0
    for bad in [(15, 12, 8), (16, 2, 8), (0, 4, 4)]:
        assert lib.cfd_unet_workspace_bytes(*bad, ctypes.byref(nb)) != 0
