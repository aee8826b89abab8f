"""ctypes binding of ``include/cfd.h`` (argument marshalling only).

Every function of the C-ABI is exposed under its own name; ``Cavity`` wraps
a handle together with the device workspace it owns (a torch uint8 tensor:
PyTorch supplies device memory and streams, the library does all compute).

The binding loads ``lib/libcfdgb.so`` built in-tree by ``build.py``.  There
is no fallback: without the library (or without a CUDA device) the calls
raise.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import torch

_PKG = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_PKG, "lib", "libcfdgb.so")

CFD_OK = 0
CFD_ERR_INVALID_ARG = -1
CFD_ERR_CUDA = -2
CFD_ERR_NOT_CONVERGED = -3
CFD_ERR_BREAKDOWN = -4
CFD_ERR_TIMEOUT = -5
CFD_ERR_WORKSPACE_TOO_SMALL = -6

FIELD = {"u": 0, "v": 1, "w": 2, "p": 3}
SOLVER = {"cg": 0, "jacobi": 1, "ir": 2, "dic": 3, "fpcg": 4}
SUBSTEP = {"forces": 0, "advect": 1, "diffuse": 2, "project": 3}
PHASES = ["applyForces", "solveAdvection", "diffuse", "divergence", "pcg", "applyPressureCorrection"]


class cfd_params(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
                ("length", ctypes.c_double), ("dt", ctypes.c_double), ("rho", ctypes.c_double),
                ("nu", ctypes.c_double), ("lid_u", ctypes.c_double), ("g", ctypes.c_double * 3),
                ("solver", ctypes.c_int32), ("rtol", ctypes.c_double), ("max_iters", ctypes.c_int32),
                ("warm_start", ctypes.c_int32), ("ir_delta", ctypes.c_double),
                ("advect_order", ctypes.c_int32), ("learned_guess", ctypes.c_int32),
                ("reserved", ctypes.c_int32 * 6)]


class cfd_tune_report(ctypes.Structure):
    _fields_ = [("blocks_per_sm", ctypes.c_int32), ("tile_depth", ctypes.c_int32), ("candidates", ctypes.c_int32),
                ("ms_auto", ctypes.c_float), ("ms_best", ctypes.c_float), ("cg_variant", ctypes.c_int32),
                ("ir_form", ctypes.c_int32)]


class cfd_solve_stats(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int32), ("outer_iters", ctypes.c_int32),
                ("restarts", ctypes.c_int32), ("status", ctypes.c_int32),
                ("diff_iters", ctypes.c_int32 * 3), ("diff_status", ctypes.c_int32),
                ("rel_resid", ctypes.c_double), ("b_norm", ctypes.c_double)]

    def as_dict(self):
        return {"iters": self.iters, "outer_iters": self.outer_iters, "restarts": self.restarts,
                "status": self.status, "diff_iters": list(self.diff_iters),
                "diff_status": self.diff_status, "rel_resid": self.rel_resid, "b_norm": self.b_norm}


class CfdError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"cfd error {code}: {msg}")
        self.code = code


_lib = None


def load_library(path: Optional[str] = None):
    """Load libcfdgb.so (once) and declare the C signatures."""
    global _lib
    if _lib is not None:
        return _lib
    p = path or _LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError(f"{p} is missing: run `python -c 'import __graft_entry__ as g; g.build()'` first")
    lib = ctypes.CDLL(p)
    P = ctypes.POINTER
    vp = ctypes.c_void_p
    sig = {
        "cfd_workspace_bytes": (ctypes.c_int, [P(cfd_params), P(ctypes.c_size_t)]),
        "cfd_create": (ctypes.c_int, [P(cfd_params), vp, ctypes.c_size_t, vp, P(vp)]),
        "cfd_destroy": (None, [vp]),
        "cfd_last_error": (ctypes.c_char_p, [vp]),
        "cfd_set_stream": (ctypes.c_int, [vp, vp]),
        "cfd_set_field": (ctypes.c_int, [vp, ctypes.c_int, vp, ctypes.c_int]),
        "cfd_read_field": (ctypes.c_int, [vp, ctypes.c_int, vp, ctypes.c_int, P(ctypes.c_int64)]),
        "cfd_step": (ctypes.c_int, [vp, ctypes.c_int, P(cfd_solve_stats)]),
        "cfd_substep": (ctypes.c_int, [vp, ctypes.c_int, P(cfd_solve_stats)]),
        "cfd_solve_pressure": (ctypes.c_int, [vp, vp, vp, P(cfd_solve_stats)]),
        "cfd_apply_poisson": (ctypes.c_int, [vp, vp, vp]),
        "cfd_launch_count": (ctypes.c_int64, [vp]),
        "cfd_recent_stats": (ctypes.c_int, [vp, ctypes.c_int, P(cfd_solve_stats)]),
        "cfd_poisson_solve_noalloc": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, vp, vp,
                                                     ctypes.c_double, ctypes.c_int32, vp, P(cfd_solve_stats)]),
        "cfd_set_solver_shape": (ctypes.c_int, [vp, ctypes.c_int, ctypes.c_int]),
        "cfd_get_solver_shape": (ctypes.c_int, [vp, ctypes.c_int, P(ctypes.c_int), P(ctypes.c_int), P(ctypes.c_int)]),
        "cfd_batch_workspace_bytes": (ctypes.c_int, [ctypes.c_int, P(cfd_params), P(ctypes.c_size_t)]),
        "cfd_batch_create": (ctypes.c_int, [ctypes.c_int, P(cfd_params), vp, ctypes.c_size_t, vp, P(vp)]),
        "cfd_batch_destroy": (None, [vp]),
        "cfd_batch_last_error": (ctypes.c_char_p, [vp]),
        "cfd_batch_cavity": (vp, [vp, ctypes.c_int]),
        "cfd_batch_step": (ctypes.c_int, [vp, ctypes.c_int, P(cfd_solve_stats)]),
        "cfd_batch_use_graph": (ctypes.c_int, [vp, ctypes.c_int]),
        "cfd_batch_graph_active": (ctypes.c_int, [vp]),
        "cfd_batch_blocks": (ctypes.c_int, [vp, ctypes.c_int, P(ctypes.c_int)]),
        "cfd_batch_launch_count": (ctypes.c_int64, [vp]),
        "cfd_enable_timing": (ctypes.c_int, [vp, ctypes.c_int]),
        "cfd_phase_times": (ctypes.c_int, [vp, P(ctypes.c_double), P(ctypes.c_int64)]),
        "cfd_pressure_rhs": (ctypes.c_int, [vp, vp]),
        "cfd_harvest_pair": (ctypes.c_int, [vp, vp, vp, vp, vp, vp]),
        "cfd_set_wait_limit": (ctypes.c_int, [vp, ctypes.c_uint64]),
        "cfd_autotune_solver": (ctypes.c_int, [vp, ctypes.c_int32, P(cfd_tune_report)]),
        "cfd_set_cg_variant": (ctypes.c_int, [vp, ctypes.c_int]),
        "cfd_set_ir_form": (ctypes.c_int, [vp, ctypes.c_int]),
        "cfd_set_fpcg_form": (ctypes.c_int, [vp, ctypes.c_int]),
        "cfd_set_concurrent_diffusion": (ctypes.c_int, [vp, ctypes.c_int]),
        "cfd_snapshot": (ctypes.c_int, [vp]),
        "cfd_csr_bytes": (ctypes.c_int, [ctypes.c_int32] * 3 + [P(ctypes.c_size_t), P(ctypes.c_int64)]),
        "cfd_csr_assemble": (ctypes.c_int, [ctypes.c_int32] * 3 + [vp, vp]),
        "cfd_csr_spmv": (ctypes.c_int, [ctypes.c_int32] * 3 + [vp, vp, vp, vp]),
        "cfd_snapshot_write_csv": (ctypes.c_int, [vp, ctypes.c_char_p, ctypes.c_int]),
        "cfd_apply_poisson_f32": (ctypes.c_int, [ctypes.c_int32] * 3 + [vp, vp, vp]),
        "cfd_cg_update_scratch_bytes": (ctypes.c_size_t, []),
        "cfd_probe_fp64_fma": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, vp, vp]),
        "cfd_cg_update_f64": (ctypes.c_int, [ctypes.c_size_t, ctypes.c_double, vp, vp, vp, vp, vp, vp, vp]),
        "cfd_cg_update_f32": (ctypes.c_int, [ctypes.c_size_t, ctypes.c_float, vp, vp, vp, vp, vp, vp, vp]),
        "cfd_conv3d_bf16": (ctypes.c_int, [ctypes.c_int] * 3 + [vp, ctypes.c_int, vp, ctypes.c_int, ctypes.c_int, vp, vp,
                                                                ctypes.c_int, ctypes.c_int, vp, vp, vp, vp]),
        "cfd_unet_workspace_bytes": (ctypes.c_int, [ctypes.c_int] * 3 + [P(ctypes.c_size_t)]),
        "cfd_unet_create": (ctypes.c_int, [ctypes.c_int] * 3 + [vp, ctypes.c_size_t, vp, ctypes.c_uint64, P(vp)]),
        "cfd_unet_destroy": (None, [vp]),
        "cfd_unet_param_count": (ctypes.c_int64, [vp]),
        "cfd_unet_get_params": (ctypes.c_int, [vp, vp, ctypes.c_int64]),
        "cfd_unet_set_params": (ctypes.c_int, [vp, vp, ctypes.c_int64]),
        "cfd_unet_apply": (ctypes.c_int, [vp, vp, vp]),
        "cfd_unet_train_step": (ctypes.c_int, [vp, vp, vp, ctypes.c_int, ctypes.c_float, P(ctypes.c_float)]),
        "cfd_unet_read_tensor": (ctypes.c_int, [vp, ctypes.c_int, vp, ctypes.c_int64]),
        "cfd_unet_set_loss": (ctypes.c_int, [vp, ctypes.c_int]),
        "cfd_unet_set_conv_mode": (ctypes.c_int, [vp, ctypes.c_int]),
        "cfd_unet_set_wgrad_mode": (ctypes.c_int, [vp, ctypes.c_int]),
        "cfd_unet_fpcg_solve": (ctypes.c_int, [vp, vp, vp, ctypes.c_double, ctypes.c_int32, P(cfd_solve_stats)]),
        "cfd_unet_launch_count": (ctypes.c_int64, [vp]),
        "cfd_unet_grid": (ctypes.c_int, [vp, P(ctypes.c_int), P(ctypes.c_int), P(ctypes.c_int)]),
        "cfd_attach_preconditioner": (ctypes.c_int, [vp, vp]),
        "cfd_learned_guess": (ctypes.c_int, [vp, vp, vp]),
        "cfd_unet_last_error": (ctypes.c_char_p, []),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def make_params(nx, ny, nz, length=1.0, dt=0.01, rho=1.0, nu=0.0, lid_u=1.0, g=(0.0, 0.0, 0.0),
                solver="cg", rtol=1e-8, max_iters=0, warm_start=False, ir_delta=0.0, advect_order=1,
                learned_guess=False) -> cfd_params:
    prm = cfd_params()
    prm.nx, prm.ny, prm.nz = int(nx), int(ny), int(nz)
    prm.length, prm.dt, prm.rho, prm.nu, prm.lid_u = float(length), float(dt), float(rho), float(nu), float(lid_u)
    for i in range(3):
        prm.g[i] = float(g[i])
    prm.solver = SOLVER[solver] if isinstance(solver, str) else int(solver)
    prm.rtol = float(rtol)
    prm.max_iters = int(max_iters)
    prm.warm_start = 1 if warm_start else 0
    prm.ir_delta = float(ir_delta)
    prm.advect_order = int(advect_order)
    prm.learned_guess = 1 if learned_guess else 0
    return prm


def cfd_workspace_bytes(prm: cfd_params) -> int:
    lib = load_library()
    n = ctypes.c_size_t(0)
    rc = lib.cfd_workspace_bytes(ctypes.byref(prm), ctypes.byref(n))
    if rc != CFD_OK:
        raise CfdError(rc, lib.cfd_last_error(None).decode())
    return int(n.value)


def _stream_ptr(stream=None) -> int:
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


class Cavity:
    """One cavity: a handle plus the device workspace it lives in."""

    def __init__(self, prm: cfd_params, stream=None, device=None):
        if not torch.cuda.is_available():
            raise RuntimeError("a CUDA device is required (the library has no CPU path)")
        self.lib = load_library()
        self.prm = prm
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        nbytes = cfd_workspace_bytes(prm)
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        self.stream = stream
        h = ctypes.c_void_p(0)
        rc = self.lib.cfd_create(ctypes.byref(prm), ctypes.c_void_p(self.workspace.data_ptr()),
                                 ctypes.c_size_t(nbytes), ctypes.c_void_p(_stream_ptr(stream)), ctypes.byref(h))
        if rc != CFD_OK:
            raise CfdError(rc, self.lib.cfd_last_error(None).decode())
        self.h = h

    # -- helpers ----------------------------------------------------------
    def _check(self, rc, allow=()):
        if rc != CFD_OK and rc not in allow:
            raise CfdError(rc, self.lib.cfd_last_error(self.h).decode())
        return rc

    def close(self):
        if getattr(self, "h", None):
            self.lib.cfd_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def dims(self, field):
        nx, ny, nz = self.prm.nx, self.prm.ny, self.prm.nz
        return {"u": (nx + 1, ny, nz), "v": (nx, ny + 1, nz), "w": (nx, ny, nz + 1), "p": (nx, ny, nz)}[field]

    def shape(self, field):
        dx, dy, dz = self.dims(field)
        return (dz, dy, dx)

    # -- C-ABI calls --------------------------------------------------------
    def set_field(self, field, src):
        """src: a CUDA float64 tensor or a host array/tensor of the field's shape."""
        if isinstance(src, torch.Tensor) and src.is_cuda:
            t = src.contiguous().to(torch.float64)
            rc = self.lib.cfd_set_field(self.h, FIELD[field], ctypes.c_void_p(t.data_ptr()), 1)
            self._keep = t
        else:
            t = torch.as_tensor(src, dtype=torch.float64).contiguous()
            if tuple(t.shape) != self.shape(field) and t.numel() != int(torch.tensor(self.shape(field)).prod()):
                raise ValueError(f"{field}: expected shape {self.shape(field)}, got {tuple(t.shape)}")
            rc = self.lib.cfd_set_field(self.h, FIELD[field], ctypes.c_void_p(t.data_ptr()), 0)
            torch.cuda.current_stream().synchronize() if self.stream is None else self.stream.synchronize()
        return self._check(rc)

    def read_field(self, field, out=None, device=False):
        """Return the field as a (z, y, x) float64 tensor (host unless device=True)."""
        if out is None:
            out = torch.empty(self.shape(field), dtype=torch.float64, device=self.device if device else "cpu")
        dims = (ctypes.c_int64 * 3)()
        rc = self.lib.cfd_read_field(self.h, FIELD[field], ctypes.c_void_p(out.data_ptr()), 1 if out.is_cuda else 0, dims)
        self._check(rc)
        return out

    def step(self, nsteps=1, stats=True):
        if stats:
            arr = (cfd_solve_stats * max(1, nsteps))()
            rc = self.lib.cfd_step(self.h, int(nsteps), arr)
            self._check(rc, allow=(CFD_ERR_NOT_CONVERGED, CFD_ERR_BREAKDOWN, CFD_ERR_TIMEOUT))
            return rc, [arr[i].as_dict() for i in range(nsteps)]
        rc = self.lib.cfd_step(self.h, int(nsteps), None)
        self._check(rc)
        return rc, None

    def substep(self, which, stats=True):
        st = cfd_solve_stats()
        rc = self.lib.cfd_substep(self.h, SUBSTEP[which], ctypes.byref(st) if stats else None)
        self._check(rc, allow=(CFD_ERR_NOT_CONVERGED, CFD_ERR_BREAKDOWN, CFD_ERR_TIMEOUT))
        return rc, st.as_dict()

    def solve_pressure(self, b: torch.Tensor, x: torch.Tensor, stats=True):
        assert b.is_cuda and x.is_cuda and b.dtype == torch.float64 and x.dtype == torch.float64
        st = cfd_solve_stats()
        rc = self.lib.cfd_solve_pressure(self.h, ctypes.c_void_p(b.data_ptr()), ctypes.c_void_p(x.data_ptr()),
                                         ctypes.byref(st) if stats else None)
        self._check(rc, allow=(CFD_ERR_NOT_CONVERGED, CFD_ERR_BREAKDOWN, CFD_ERR_TIMEOUT))
        return rc, st.as_dict()

    def apply_poisson(self, x: torch.Tensor, y: torch.Tensor):
        assert x.is_cuda and y.is_cuda and x.dtype == torch.float64 and y.dtype == torch.float64
        return self._check(self.lib.cfd_apply_poisson(self.h, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr())))

    def launch_count(self) -> int:
        return int(self.lib.cfd_launch_count(self.h))

    def attach_preconditioner(self, net):
        """Attach a UNet (same grid) for solver 'fpcg'; None detaches."""
        self._net = net
        return self._check(self.lib.cfd_attach_preconditioner(self.h, net.u if net is not None else None))

    def learned_guess(self, b: torch.Tensor, x: torch.Tensor):
        """x = alpha M(b) from the attached network (cfd_learned_guess)."""
        assert b.is_cuda and x.is_cuda and b.dtype == torch.float64 and x.dtype == torch.float64
        return self._check(self.lib.cfd_learned_guess(self.h, ctypes.c_void_p(b.data_ptr()), ctypes.c_void_p(x.data_ptr())))

    def snapshot(self):
        """Start an asynchronous host copy of (u, v, w, p) (cfd_snapshot)."""
        return self._check(self.lib.cfd_snapshot(self.h))

    def write_csv(self, path: str, threads: int = 0):
        """Write the last snapshot as CSV (cfd_snapshot_write_csv)."""
        return self._check(self.lib.cfd_snapshot_write_csv(self.h, os.fsencode(path), int(threads)))

    def set_cg_variant(self, variant: str):
        """'single' (one reduction per iteration, default) or 'two' (textbook)."""
        return self._check(self.lib.cfd_set_cg_variant(self.h, {"single": 0, "two": 1}[variant]))

    def set_concurrent_diffusion(self, on: bool):
        """Run the u, v, w diffusion solves of a step at once (small grids)."""
        return self._check(self.lib.cfd_set_concurrent_diffusion(self.h, 1 if on else 0))

    def set_fpcg_form(self, form: str):
        """Form of the FPCG solve: 'graph' (default: FP32 flexible CG with FP64
        refinement, device-resident) or 'host' (FP64, host-driven)."""
        return self._check(self.lib.cfd_set_fpcg_form(self.h, {"graph": 0, "host": 1}[form]))

    def set_ir_form(self, form: str):
        """Execution of the IR solve: 'auto' (default), 'persistent' or 'graph'."""
        return self._check(self.lib.cfd_set_ir_form(self.h, {"auto": 0, "persistent": 1, "graph": 2}[form]))

    def autotune(self, iters=50) -> dict:
        """Pick the fastest solver shape for this grid (cfd_autotune_solver)."""
        rep = cfd_tune_report()
        self._check(self.lib.cfd_autotune_solver(self.h, int(iters), ctypes.byref(rep)))
        return {k: getattr(rep, k) for k, _ in cfd_tune_report._fields_}

    def pressure_rhs(self, b: torch.Tensor):
        """Projection right-hand side of the current velocity (mean kept)."""
        assert b.is_cuda and b.dtype == torch.float64 and b.numel() == self.prm.nx * self.prm.ny * self.prm.nz
        return self._check(self.lib.cfd_pressure_rhs(self.h, ctypes.c_void_p(b.data_ptr())))

    def harvest_pair(self, b: torch.Tensor, xs: torch.Tensor, xk: torch.Tensor, r: torch.Tensor, e: torch.Tensor):
        """Training pair of the learned preconditioner (cfd_harvest_pair):
        r = (b - mean b) - A xk, e = (xs - xk) - mean(xs - xk)."""
        n = self.prm.nx * self.prm.ny * self.prm.nz
        for t in (b, xs, xk, r, e):
            assert t.is_cuda and t.dtype == torch.float64 and t.numel() == n and t.is_contiguous()
        ptr = lambda t: ctypes.c_void_p(t.data_ptr())  # noqa: E731
        return self._check(self.lib.cfd_harvest_pair(self.h, ptr(b), ptr(xs), ptr(xk), ptr(r), ptr(e)))

    def set_wait_limit(self, ns=None):
        """Limit of each grid-wide wait in the persistent solves, in ns
        (None restores the 2 s default)."""
        v = (1 << 64) - 1 if ns is None else int(ns)
        return self._check(self.lib.cfd_set_wait_limit(self.h, ctypes.c_uint64(v)))

    def set_stream(self, stream):
        self.stream = stream
        return self._check(self.lib.cfd_set_stream(self.h, ctypes.c_void_p(_stream_ptr(stream))))

    def recent_stats(self, n):
        arr = (cfd_solve_stats * max(1, n))()
        rc = self.lib.cfd_recent_stats(self.h, int(n), arr)
        self._check(rc, allow=(CFD_ERR_NOT_CONVERGED, CFD_ERR_BREAKDOWN, CFD_ERR_TIMEOUT))
        return rc, [arr[i].as_dict() for i in range(n)]

    def set_solver_shape(self, blocks_per_sm=0, tile_depth=0):
        return self._check(self.lib.cfd_set_solver_shape(self.h, int(blocks_per_sm), int(tile_depth)))

    def solver_shape(self, kind=0):
        """Launch shape of the next FP64 solve of `kind` (0 pressure, 1..3 the
        u, v, w diffusion): grid size, tile depth, register path, and whether
        the tile-resident single-reduction kernel runs (cfd_get_solver_shape)."""
        b, t, r = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        self._check(self.lib.cfd_get_solver_shape(self.h, int(kind), ctypes.byref(b), ctypes.byref(t), ctypes.byref(r)))
        return {"blocks": b.value, "tile_depth": t.value, "register_path": bool(r.value),
                "tile_resident": r.value == 2}

    def enable_timing(self, on=True):
        return self._check(self.lib.cfd_enable_timing(self.h, 1 if on else 0))

    def phase_times(self):
        """{phase: (total_ms, calls)} since the last query (synchronises)."""
        ms = (ctypes.c_double * len(PHASES))()
        calls = (ctypes.c_int64 * len(PHASES))()
        self._check(self.lib.cfd_phase_times(self.h, ms, calls))
        return {name: (ms[i], int(calls[i])) for i, name in enumerate(PHASES)}


class _CavityView(Cavity):
    """A cavity owned by a Batch (no workspace or handle ownership)."""

    def __init__(self, lib, handle, prm, device, stream):  # noqa: D401  (no Cavity.__init__)
        self.lib = lib
        self.h = handle
        self.prm = prm
        self.device = device
        self.stream = stream

    def close(self):
        self.h = None


class Batch:
    """Independent cavities (uneven sizes allowed) advanced together; see
    cfd_batch_* in include/cfd.h."""

    def __init__(self, prms, stream=None, device=None):
        if not torch.cuda.is_available():
            raise RuntimeError("a CUDA device is required (the library has no CPU path)")
        self.lib = load_library()
        self.prms = list(prms)
        self.n = len(self.prms)
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self._arr = (cfd_params * self.n)(*self.prms)
        nb = ctypes.c_size_t(0)
        rc = self.lib.cfd_batch_workspace_bytes(self.n, self._arr, ctypes.byref(nb))
        if rc != CFD_OK:
            raise CfdError(rc, self.lib.cfd_last_error(None).decode())
        self.workspace = torch.empty(int(nb.value), dtype=torch.uint8, device=self.device)
        self.stream = stream
        b = ctypes.c_void_p(0)
        rc = self.lib.cfd_batch_create(self.n, self._arr, ctypes.c_void_p(self.workspace.data_ptr()),
                                       ctypes.c_size_t(int(nb.value)), ctypes.c_void_p(_stream_ptr(stream)), ctypes.byref(b))
        if rc != CFD_OK:
            raise CfdError(rc, self.lib.cfd_batch_last_error(None).decode())
        self.b = b
        self.cavities = [_CavityView(self.lib, ctypes.c_void_p(self.lib.cfd_batch_cavity(self.b, i)), self.prms[i],
                                     self.device, stream) for i in range(self.n)]

    def close(self):
        if getattr(self, "b", None):
            self.lib.cfd_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def cavity(self, i) -> Cavity:
        return self.cavities[i]

    def step(self, nsteps=1, stats=True):
        if stats:
            arr = (cfd_solve_stats * self.n)()
            rc = self.lib.cfd_batch_step(self.b, int(nsteps), arr)
            if rc not in (CFD_OK, CFD_ERR_NOT_CONVERGED, CFD_ERR_BREAKDOWN, CFD_ERR_TIMEOUT):
                raise CfdError(rc, self.lib.cfd_batch_last_error(self.b).decode())
            return rc, [arr[i].as_dict() for i in range(self.n)]
        rc = self.lib.cfd_batch_step(self.b, int(nsteps), None)
        if rc != CFD_OK:
            raise CfdError(rc, self.lib.cfd_batch_last_error(self.b).decode())
        return rc, None

    def use_graph(self, on=True):
        return self.lib.cfd_batch_use_graph(self.b, 1 if on else 0)

    def graph_active(self) -> bool:
        return bool(self.lib.cfd_batch_graph_active(self.b))

    def blocks(self, kind):
        v = ctypes.c_int()
        self.lib.cfd_batch_blocks(self.b, int(kind), ctypes.byref(v))
        return v.value

    def launch_count(self) -> int:
        return int(self.lib.cfd_batch_launch_count(self.b))


def to_octets(x: torch.Tensor) -> torch.Tensor:
    """Channels-last [V, C] -> the library's activation layout: ceil(C / W)
    planes of [V][W], W = min(C, 8) (flat)."""
    V, C = x.shape
    W = min(C, 8)
    return x.reshape(V, C // W, W).permute(1, 0, 2).contiguous().reshape(-1)


def from_octets(flat: torch.Tensor, C: int) -> torch.Tensor:
    """Inverse of to_octets: flat octet planes -> channels-last [V, C]."""
    W = min(C, 8)
    V = flat.numel() // C
    return flat.reshape(C // W, V, W).permute(1, 0, 2).reshape(V, C)


# names of the BF16 tensors readable with UNet.read_tensor (indices 0..25)
UNET_TENSORS = ["xin", "a0", "s0", "p0", "a1", "s1", "p1", "a2", "s2", "u1", "d1", "u0", "d0",
                "gz", "g_d0", "g_s0", "g_u0", "g_d1", "g_s1", "g_u1", "g_s2", "g_a2", "g_p1", "g_a1", "g_p0", "g_a0"]
UNET_CHANNELS = [1, 16, 16, 16, 32, 32, 32, 64, 64, 64, 32, 32, 16,
                 1, 16, 16, 32, 32, 32, 64, 64, 64, 32, 32, 16, 16]
UNET_LEVELS = [0, 0, 0, 1, 1, 1, 2, 2, 2, 1, 1, 0, 0,
               0, 0, 0, 0, 1, 1, 1, 2, 2, 2, 1, 1, 0]
UNET_T_OUT, UNET_T_TARGET, UNET_T_GRAD, UNET_T_ADAM_M, UNET_T_ADAM_V = 100, 101, 102, 103, 104

# layer table: (name, level, c0, c1, cout, ks), in parameter order
UNET_LAYERS = [("L0a", 0, 1, 0, 16, 3), ("L0b", 0, 16, 0, 16, 3), ("L1a", 1, 16, 0, 32, 3), ("L1b", 1, 32, 0, 32, 3),
               ("L2a", 2, 32, 0, 64, 3), ("L2b", 2, 64, 0, 64, 3), ("L1c", 1, 32, 64, 32, 3),
               ("L0c", 0, 16, 32, 16, 3), ("head", 0, 16, 0, 1, 1)]


class UNet:
    """Learned preconditioner on an nx x ny x nz grid (each a multiple of 4);
    see cfd_unet_* in include/cfd.h."""

    def __init__(self, nx, ny, nz, seed=0, stream=None, device=None):
        if not torch.cuda.is_available():
            raise RuntimeError("a CUDA device is required (the library has no CPU path)")
        self.lib = load_library()
        self.shape = (int(nx), int(ny), int(nz))
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        nb = ctypes.c_size_t(0)
        self._check(self.lib.cfd_unet_workspace_bytes(*self.shape, ctypes.byref(nb)))
        self.workspace = torch.empty(int(nb.value), dtype=torch.uint8, device=self.device)
        self.stream = stream
        u = ctypes.c_void_p(0)
        self._check(self.lib.cfd_unet_create(*self.shape, ctypes.c_void_p(self.workspace.data_ptr()),
                                             ctypes.c_size_t(int(nb.value)), ctypes.c_void_p(_stream_ptr(stream)),
                                             ctypes.c_uint64(int(seed)), ctypes.byref(u)))
        self.u = u
        self.nparams = int(self.lib.cfd_unet_param_count(self.u))

    def _check(self, rc, allow=()):
        if rc != CFD_OK and rc not in allow:
            raise CfdError(rc, self.lib.cfd_unet_last_error().decode())
        return rc

    def close(self):
        if getattr(self, "u", None):
            self.lib.cfd_unet_destroy(self.u)
            self.u = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def cells(self):
        return self.shape[0] * self.shape[1] * self.shape[2]

    def get_params(self) -> torch.Tensor:
        out = torch.empty(self.nparams, dtype=torch.float32)
        self._check(self.lib.cfd_unet_get_params(self.u, ctypes.c_void_p(out.data_ptr()), self.nparams))
        return out

    def set_params(self, params: torch.Tensor):
        p = params.detach().to(torch.float32).contiguous().cpu()
        assert p.numel() == self.nparams
        self._check(self.lib.cfd_unet_set_params(self.u, ctypes.c_void_p(p.data_ptr()), self.nparams))

    def apply(self, r: torch.Tensor, z: torch.Tensor):
        assert r.is_cuda and z.is_cuda and r.dtype == torch.float64 and z.dtype == torch.float64
        self._check(self.lib.cfd_unet_apply(self.u, ctypes.c_void_p(r.data_ptr()), ctypes.c_void_p(z.data_ptr())))

    def train_step(self, r: torch.Tensor, e: torch.Tensor, lr=1e-3) -> float:
        assert r.is_cuda and e.is_cuda and r.dtype == torch.float64 and e.dtype == torch.float64
        assert r.numel() == e.numel() and r.numel() % self.cells == 0
        loss = ctypes.c_float(0.0)
        self._check(self.lib.cfd_unet_train_step(self.u, ctypes.c_void_p(r.data_ptr()), ctypes.c_void_p(e.data_ptr()),
                                                 r.numel() // self.cells, ctypes.c_float(lr), ctypes.byref(loss)))
        return float(loss.value)

    def set_loss(self, kind: str):
        """'mse' (|d|^2 / V), 'anorm' (d.(A d) / V), d = U(s r) - s e, or 'cos'
        (one minus the energy-norm cosine of U(s r) and s e)."""
        self._check(self.lib.cfd_unet_set_loss(self.u, {"mse": 0, "anorm": 1, "cos": 2}[kind]))

    def set_conv_mode(self, mode: str):
        """'registers', 'bulk' (default), 'two_stage' or 'persistent' (cfd_unet_set_conv_mode)."""
        self._check(self.lib.cfd_unet_set_conv_mode(
            self.u, {"registers": 0, "bulk": 1, "two_stage": 2, "persistent": 3}[mode]))

    def set_wgrad_mode(self, mode: str):
        """'tensor' (default: the 3x3x3 layers' weight gradients on the tensor
        cores) or 'cuda_cores' (cfd_unet_set_wgrad_mode)."""
        self._check(self.lib.cfd_unet_set_wgrad_mode(self.u, {"tensor": 0, "cuda_cores": 1}[mode]))

    def read_tensor(self, which) -> torch.Tensor:
        """Host copy of a model tensor: a name from UNET_TENSORS (BF16,
        returned channels-last [cells of its level, channels]) or a UNET_T_*
        code."""
        if isinstance(which, str):
            which = UNET_TENSORS.index(which)
        nx, ny, nz = self.shape
        if 0 <= which < 26:
            lv = UNET_LEVELS[which]
            vox = (nx >> lv) * (ny >> lv) * (nz >> lv)
            out = torch.empty(vox * UNET_CHANNELS[which], dtype=torch.bfloat16)
        elif which in (UNET_T_OUT, UNET_T_TARGET):
            out = torch.empty(self.cells, dtype=torch.float32)
        else:
            out = torch.empty(self.nparams, dtype=torch.float32)
        self._check(self.lib.cfd_unet_read_tensor(self.u, int(which), ctypes.c_void_p(out.data_ptr()), out.numel()))
        if 0 <= which < 26:
            return from_octets(out, UNET_CHANNELS[which])
        return out

    def fpcg_solve(self, b: torch.Tensor, x: torch.Tensor, rtol=1e-8, max_iters=0):
        assert b.is_cuda and x.is_cuda and b.dtype == torch.float64 and x.dtype == torch.float64
        st = cfd_solve_stats()
        rc = self.lib.cfd_unet_fpcg_solve(self.u, ctypes.c_void_p(b.data_ptr()), ctypes.c_void_p(x.data_ptr()),
                                          ctypes.c_double(rtol), int(max_iters), ctypes.byref(st))
        self._check(rc, allow=(CFD_ERR_NOT_CONVERGED, CFD_ERR_BREAKDOWN, CFD_ERR_TIMEOUT))
        return rc, st.as_dict()

    def launch_count(self) -> int:
        return int(self.lib.cfd_unet_launch_count(self.u))


class CsrMatrix:
    """The assembled pressure matrix on the device (cfd_csr_*), for comparison
    with the matrix-free operator."""

    def __init__(self, nx, ny, nz, stream=None, device=None):
        self.lib = load_library()
        self.shape = (int(nx), int(ny), int(nz))
        nb = ctypes.c_size_t(0)
        nnz = ctypes.c_int64(0)
        rc = self.lib.cfd_csr_bytes(*self.shape, ctypes.byref(nb), ctypes.byref(nnz))
        if rc != CFD_OK:
            raise CfdError(rc, self.lib.cfd_last_error(None).decode())
        self.nnz = int(nnz.value)
        self.bytes = int(nb.value)
        dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.buf = torch.empty(self.bytes, dtype=torch.uint8, device=dev)
        self.stream = stream
        rc = self.lib.cfd_csr_assemble(*self.shape, ctypes.c_void_p(self.buf.data_ptr()), ctypes.c_void_p(_stream_ptr(stream)))
        if rc != CFD_OK:
            raise CfdError(rc, self.lib.cfd_last_error(None).decode())

    def arrays(self):
        """Host copies (row_ptr, col, val) for checks."""
        n = self.shape[0] * self.shape[1] * self.shape[2]
        raw = self.buf.cpu()
        a16 = lambda x: (x + 15) // 16 * 16  # noqa: E731
        o1 = a16((n + 1) * 4)
        o2 = o1 + a16(self.nnz * 4)
        return (raw[:(n + 1) * 4].view(torch.int32), raw[o1:o1 + self.nnz * 4].view(torch.int32),
                raw[o2:o2 + self.nnz * 8].view(torch.float64))

    def spmv(self, x: torch.Tensor, y: torch.Tensor):
        rc = self.lib.cfd_csr_spmv(*self.shape, ctypes.c_void_p(self.buf.data_ptr()), ctypes.c_void_p(x.data_ptr()),
                                   ctypes.c_void_p(y.data_ptr()), ctypes.c_void_p(_stream_ptr(self.stream)))
        if rc != CFD_OK:
            raise CfdError(rc, self.lib.cfd_last_error(None).decode())


class KrylovKernels:
    """The stand-alone building blocks (cfd_apply_poisson_f32,
    cfd_cg_update_f64 / _f32) with their own zero-filled scratch and an
    FP64 result slot on the device."""

    def __init__(self, stream=None, device=None):
        self.lib = load_library()
        dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        nbytes = int(self.lib.cfd_cg_update_scratch_bytes())
        self.scratch = torch.zeros(nbytes, dtype=torch.uint8, device=dev)
        self.rr = torch.zeros(1, dtype=torch.float64, device=dev)
        self.stream = stream

    def _check(self, rc):
        if rc != CFD_OK:
            raise CfdError(rc, self.lib.cfd_last_error(None).decode())

    def apply_poisson_f32(self, x: torch.Tensor, y: torch.Tensor):
        """y = A x in FP32; x, y contiguous float32 of shape (nz, ny, nx)."""
        if x.dtype != torch.float32 or y.dtype != torch.float32 or x.dim() != 3 or x.shape != y.shape:
            raise ValueError("apply_poisson_f32 wants two float32 tensors of one (nz, ny, nx) shape")
        nz, ny, nx = x.shape
        self._check(self.lib.cfd_apply_poisson_f32(nx, ny, nz, ctypes.c_void_p(x.data_ptr()),
                                                   ctypes.c_void_p(y.data_ptr()),
                                                   ctypes.c_void_p(_stream_ptr(self.stream))))

    def cg_update(self, alpha, p, q, x, r) -> torch.Tensor:
        """x += alpha p, r -= alpha q; returns the device scalar r.r (FP64)."""
        n = r.numel()
        if not all(t.dtype == r.dtype and t.numel() == n and t.is_contiguous() for t in (p, q, x)):
            raise ValueError("cg_update wants four contiguous vectors of one dtype and length")
        fn = {torch.float64: (self.lib.cfd_cg_update_f64, ctypes.c_double),
              torch.float32: (self.lib.cfd_cg_update_f32, ctypes.c_float)}.get(r.dtype)
        if fn is None:
            raise ValueError("cg_update supports float64 and float32")
        ptr = lambda t: ctypes.c_void_p(t.data_ptr())  # noqa: E731
        self._check(fn[0](n, fn[1](alpha), ptr(p), ptr(q), ptr(x), ptr(r), ptr(self.rr), ptr(self.scratch),
                          ctypes.c_void_p(_stream_ptr(self.stream))))
        return self.rr
