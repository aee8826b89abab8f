"""tcgen05 BF16 implicit-GEMM convolution (the U-Net building block) against
float64 3D convolution of the same BF16-rounded operands.

Products of two BF16 numbers are exact in FP32 and the kernel accumulates
in FP32 over one accumulation per K chunk of 16 (plus the bias), so each FP32
output differs from the float64 reference by at most about
chunks * 2^-24 * sum|terms| (sum|terms| = the convolution of |x| with |w|);
the check uses four times that bound, elementwise.  The BF16 output adds one
BF16 rounding (2^-8 relative).
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2504_03697_gb300 import build as B
    B.build()
    from paper_2504_03697_gb300 import cfd
    lib = cfd.load_library()
    lib.cfd_conv3d_bf16.restype = ctypes.c_int
    lib.cfd_conv3d_bf16.argtypes = [ctypes.c_int] * 3 + [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_int,
                                                         ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                                         ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                                         ctypes.c_void_p]
    return lib


def run_conv(lib, shape, c0, c1, cout, ks, nout, f32=True, seed=0):
    nx, ny, nz = shape
    g = torch.Generator().manual_seed(seed)
    V = nx * ny * nz
    x0 = torch.randn(nz, ny, nx, c0, generator=g).to(torch.bfloat16)
    x1 = torch.randn(nz, ny, nx, c1, generator=g).to(torch.bfloat16) if c1 else None
    cin = c0 + c1
    w = (torch.randn(cout, cin, ks, ks, ks, generator=g) / np.sqrt(cin * ks ** 3)).to(torch.bfloat16)
    bias = torch.randn(cout, generator=g).float()
    # reference: float64 cross-correlation, zero padding
    xin = x0.double() if c1 == 0 else torch.cat([x0.double(), x1.double()], dim=-1)
    ref = torch.nn.functional.conv3d(xin.permute(3, 0, 1, 2)[None], w.double(), bias.double(), padding=ks // 2)[0]
    ref = ref.permute(1, 2, 3, 0).reshape(V, cout)
    ref_abs = torch.nn.functional.conv3d(xin.abs().permute(3, 0, 1, 2)[None], w.double().abs(), bias.double().abs(),
                                         padding=ks // 2)[0].permute(1, 2, 3, 0).reshape(V, cout)
    # device operands: activations as octet planes, weights [tap][nout][cin_pad] (or packed [nout][32])
    packed = c0 == 1 and c1 == 0 and ks == 3
    if packed:
        wk = torch.zeros(nout, 32, dtype=torch.bfloat16)
        wk[:cout, :27] = w.reshape(cout, 27)
    else:
        cin_pad = (cin + 15) // 16 * 16
        wk = torch.zeros(ks ** 3, nout, cin_pad, dtype=torch.bfloat16)
        wk[:, :cout, :cin] = w.permute(2, 3, 4, 0, 1).reshape(ks ** 3, cout, cin)
    from paper_2504_03697_gb300.cfd import from_octets, to_octets
    dx0 = to_octets(x0.reshape(V, c0)).cuda()
    dx1 = to_octets(x1.reshape(V, c1)).cuda() if c1 else None
    dw = wk.contiguous().cuda()
    db = bias.cuda()
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    out32 = torch.full((V, cout), float("nan"), device="cuda") if f32 else None
    out16 = torch.zeros(V * cout, dtype=torch.bfloat16, device="cuda") if not f32 else None
    rc = lib.cfd_conv3d_bf16(nx, ny, nz, dx0.data_ptr(), c0, dx1.data_ptr() if c1 else None, c1, ks, dw.data_ptr(),
                             db.data_ptr(), cout, nout, out16.data_ptr() if out16 is not None else None,
                             out32.data_ptr() if out32 is not None else None, err.data_ptr(),
                             torch.cuda.current_stream().cuda_stream)
    assert rc == 0
    torch.cuda.synchronize()
    assert int(err.item()) == 0
    got = (out32 if f32 else from_octets(out16.reshape(-1).cpu(), cout).float()).double().cpu()
    chunks = 2 if packed else ks ** 3 * ((cin + 15) // 16)
    return got, ref, ref_abs, chunks


@pytest.mark.parametrize("shape,c0,c1,cout,ks,nout", [
    ((20, 12, 9), 1, 0, 16, 3, 16),     # first layer: tap-packed single channel
    ((16, 16, 16), 16, 0, 16, 3, 16),
    ((17, 9, 13), 16, 0, 32, 3, 32),    # ragged tile count
    ((8, 8, 8), 32, 64, 32, 3, 32),     # concat (skip + up-sampled)
    ((16, 8, 8), 16, 32, 16, 3, 16),
    ((8, 8, 8), 64, 0, 64, 3, 64),
    ((12, 10, 6), 16, 0, 1, 1, 16),     # 1x1x1 head, one output channel
    ((12, 10, 6), 1, 0, 16, 1, 16),     # 1x1x1 with a narrow (1-channel) input
])
def test_conv_matches_reference(lib, shape, c0, c1, cout, ks, nout):
    got, ref, ref_abs, chunks = run_conv(lib, shape, c0, c1, cout, ks, nout, f32=True)
    bound = 4 * (chunks + 1) * 2.0 ** -24 * ref_abs
    assert torch.all((got - ref).abs() <= bound), ((got - ref).abs() / bound).max().item()


# BF16 output of a 3x3x3 layer whose sources have 16k channels takes the
# TMA-tiled kernel (one staged input box per 16-channel block, shifted A
# descriptors); these shapes cover its contiguous-row mode (x extent < 128),
# its x-line mode (x extent >= 128, several x tiles), ragged y / z tiles,
# concatenated sources and every output width.
@pytest.mark.parametrize("shape,c0,c1,cout,nout", [
    ((16, 12, 10), 16, 32, 32, 32),
    ((16, 12, 8), 16, 0, 16, 16),
    ((17, 9, 13), 32, 0, 32, 32),
    ((8, 6, 4), 32, 64, 32, 32),
    ((4, 3, 2), 64, 0, 64, 64),
    ((128, 6, 5), 16, 0, 16, 16),
    ((200, 5, 3), 16, 32, 48, 64),
    ((64, 16, 4), 32, 0, 64, 64),
    ((32, 16, 8), 64, 0, 32, 32),
])
def test_conv_bf16_output(lib, shape, c0, c1, cout, nout):
    got, ref, ref_abs, chunks = run_conv(lib, shape, c0, c1, cout, 3, nout, f32=False, seed=3)
    bound = 2.0 ** -8 * ref.abs() + 4 * (chunks + 1) * 2.0 ** -24 * ref_abs
    bad = (got - ref).abs() > bound
    assert not bool(bad.any()), (int(bad.sum()), float(((got - ref).abs() / bound).max()))
