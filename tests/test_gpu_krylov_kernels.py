"""GPU parity of the stand-alone Krylov building blocks (Sec. 3.1, Table 1:
spmv, vector add / scale, dot) against the FP64 oracle.

* FP32 operator y = A x vs the oracle's CSR matrix applied in FP64 to the
  same FP32 inputs.  Bound: the kernel forms 6 x_c - (sum of six neighbour
  values, x_c standing in for a missing one) with one rounding per addition
  and one for the fused multiply-add, so |y32 - y64| <= 7 u (6 |x_c| +
  sum |x_n| + 6 |x_c|), u = 2^-24; the test allows 2^-20 (|A| |x| + 6 |x|).
* At 256^2 x 256 and 256^2 x 155 whole z-planes are checked: a row of plane
  k touches planes k-1..k+1 only, so it equals the middle row of the oracle
  matrix of an nx x ny x 3 grid applied to those planes (2 planes at the
  walls).
* CG update vs oracle.krylov.cg_update: FP64 to 4 unit roundoffs of |x| + |alpha p|
  (fused vs separate rounding) and r.r to 1e-12 relative; FP32 to 2 FP32 ulp
  and 1e-6 relative.
"""
import numpy as np
import pytest
import torch

from oracle.krylov import cg_update
from oracle.operators import poisson_csr
from paper_2504_03697_gb300.synthetic import uniform_field

pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24
U64 = 2.0 ** -53


@pytest.fixture(scope="module")
def kk():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2504_03697_gb300 import build as B
    B.build()
    from paper_2504_03697_gb300 import cfd
    return cfd.KrylovKernels()


def _apply_bound(A, x64):
    return 2.0 ** -20 * (abs(A) @ np.abs(x64) + 6.0 * np.abs(x64))


# scalar kernel (nx % 4 != 0) and the float4 kernel with two planes per thread
@pytest.mark.parametrize("shape", [(1, 1, 1), (1, 1, 7), (2, 3, 2), (33, 9, 65), (31, 17, 33), (4, 1, 1),
                                   (36, 20, 19), (128, 40, 97), (64, 64, 64)])
def test_apply_f32_matches_oracle(kk, shape):
    nx, ny, nz = shape
    x = uniform_field((nz, ny, nx), seed=13).astype(np.float32)
    xg = torch.tensor(x, device="cuda")
    yg = torch.full_like(xg, float("nan"))
    kk.apply_poisson_f32(xg, yg)
    A = poisson_csr(nx, ny, nz)
    x64 = x.astype(np.float64).ravel()
    y64 = A @ x64
    err = np.abs(yg.cpu().numpy().astype(np.float64).ravel() - y64)
    assert np.all(err <= _apply_bound(A, x64))


# float4 kernel with four planes per thread (the benchmarked launch), whole
# and ragged along z
@pytest.mark.parametrize("nz", [256, 155])
def test_apply_f32_full_size_planes(kk, nz):
    n = 256
    x = uniform_field((nz, n, n), seed=3).astype(np.float32)
    xg = torch.tensor(x, device="cuda")
    yg = torch.full_like(xg, float("nan"))
    kk.apply_poisson_f32(xg, yg)
    y = yg.cpu().numpy()
    A3 = poisson_csr(n, n, 3)
    A2 = poisson_csr(n, n, 2)
    for k in (0, 1, 3, 4, 5, 31, 32, 33, 127, nz - 4, nz - 3, nz - 2, nz - 1):
        if k == 0:
            A, planes, mid = A2, x[0:2], 0
        elif k == nz - 1:
            A, planes, mid = A2, x[nz - 2:nz], 1
        else:
            A, planes, mid = A3, x[k - 1:k + 2], 1
        x64 = planes.astype(np.float64).ravel()
        ref = (A @ x64).reshape(planes.shape)[mid]
        bound = _apply_bound(A, x64).reshape(planes.shape)[mid]
        assert np.all(np.abs(y[k].astype(np.float64) - ref) <= bound), k


def test_apply_f32_constant_and_ramp_exact(kk):
    nx, ny, nz = 40, 24, 36
    c = torch.full((nz, ny, nx), 3.25, dtype=torch.float32, device="cuda")
    y = torch.empty_like(c)
    kk.apply_poisson_f32(c, y)
    assert torch.count_nonzero(y).item() == 0
    ramp = torch.arange(nx, dtype=torch.float32, device="cuda").expand(nz, ny, nx).contiguous()
    kk.apply_poisson_f32(ramp, y)
    yc = y.cpu().numpy()
    assert np.all(yc[:, :, 1:-1] == 0.0)
    assert np.all(yc[:, :, 0] == -1.0) and np.all(yc[:, :, -1] == 1.0)


def _vectors(n, seed, dtype):
    rng = np.random.default_rng(seed)
    return [rng.uniform(-1.0, 1.0, n).astype(dtype) for _ in range(4)]


@pytest.mark.parametrize("n", [1, 2, 3, 5, 8, 4099, 1_000_003, 256 ** 3])
def test_cg_update_f64_matches_oracle(kk, n):
    p, q, x, r = _vectors(n, 100 + n % 97, np.float64)
    alpha = 0.3711
    g = [torch.tensor(a, device="cuda") for a in (p, q, x, r)]
    rr_g = kk.cg_update(alpha, *g).item()
    xo, ro = x.copy(), r.copy()
    rr_o = cg_update(xo, ro, p, q, alpha)
    xg, rg = g[2].cpu().numpy(), g[3].cpu().numpy()
    assert np.all(np.abs(xg - xo) <= 4 * U64 * (np.abs(x) + np.abs(alpha * p)))
    assert np.all(np.abs(rg - ro) <= 4 * U64 * (np.abs(r) + np.abs(alpha * q)))
    assert rr_g == pytest.approx(rr_o, rel=1e-12)


@pytest.mark.parametrize("n", [1, 3, 4, 7, 4101, 1_000_003, 256 ** 3])
def test_cg_update_f32_matches_oracle(kk, n):
    p, q, x, r = _vectors(n, 200 + n % 89, np.float32)
    alpha = np.float32(-0.61)
    g = [torch.tensor(a, device="cuda") for a in (p, q, x, r)]
    rr_g = kk.cg_update(float(alpha), *g).item()
    p64, q64 = p.astype(np.float64), q.astype(np.float64)
    xo, ro = x.astype(np.float64), r.astype(np.float64)
    rr_o = cg_update(xo, ro, p64, q64, float(alpha))
    xg, rg = g[2].cpu().numpy().astype(np.float64), g[3].cpu().numpy().astype(np.float64)
    assert np.all(np.abs(xg - xo) <= 2 * U32 * (np.abs(x) + np.abs(alpha * p64)))
    assert np.all(np.abs(rg - ro) <= 2 * U32 * (np.abs(r) + np.abs(alpha * q64)))
    assert rr_g == pytest.approx(rr_o, rel=1e-6)


def test_cg_update_repeatable_and_scratch_reset(kk):
    n = 3_000_001
    p, q, x, r = _vectors(n, 7, np.float64)
    outs = []
    for _ in range(3):
        g = [torch.tensor(a, device="cuda") for a in (p, q, x, r)]
        outs.append(kk.cg_update(0.25, *g).item())
    assert outs[0] == outs[1] == outs[2]
    assert int(torch.count_nonzero(kk.scratch[-16:]).item()) == 0


def test_cg_update_rejects_bad_arguments(kk):
    from paper_2504_03697_gb300.cfd import CfdError
    v = torch.zeros(17, dtype=torch.float64, device="cuda")
    with pytest.raises(CfdError):
        kk.cg_update(1.0, v[1:], v[1:].clone(), v[1:].clone(), v[1:].clone())  # 8-byte offset
    with pytest.raises(CfdError):
        kk.cg_update(1.0, v[:0], v[:0], v[:0], v[:0])
