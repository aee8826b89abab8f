"""GPU checks of the learned preconditioner (U-Net on the tensor cores) and
of the flexible PCG that uses it.

Layer by layer, every GPU result is compared with the float64 oracle applied
to the GPU's own inputs of that layer (its BF16 activations, BF16-rounded
weights, FP32 biases), so each check sees one layer's arithmetic only:

* convolutions (forward and input gradients): products of BF16 numbers are
  exact in FP32 and the kernel rounds once per 16-deep K chunk, so the FP32
  result lies within (chunks + 1) 2^-24 sum|terms| of the exact one; the
  check allows 4x that plus one BF16 rounding (2^-8 relative) of the stored
  output;
* pooling, up-sampling adjoints, the loss gradient: one FP32 sum of at most
  8 terms plus one BF16 rounding;
* weight gradients (FP32 on the CUDA cores, 32 chunk sums of V/32 terms
  each, then a sum over chunks): within 2 (V/32 + 34) 2^-24 sum|terms|;
* Adam: the first step from zero moments moves each weight by lr sign(g).

End to end, the BF16 network is compared with the float64 network on the
same weights (relative L2 error, a sanity bound), and flexible PCG is judged
like every solve here: FP64 true residual <= rtol ||b||, and the solution
within 2 rtol ||b|| / lambda_min of the oracle's.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import unet as ou  # noqa: E402
from oracle.krylov import pcg  # noqa: E402
from oracle.operators import poisson_csr  # noqa: E402
from paper_2504_03697_gb300.synthetic import gaussian_rhs, uniform_field  # noqa: E402

pytestmark = pytest.mark.gpu

U = 2.0 ** -8    # BF16 unit roundoff
E = 2.0 ** -24   # FP32 unit roundoff
SHAPE = (16, 12, 8)


@pytest.fixture(scope="module")
def cfd():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2504_03697_gb300 import build as B
    B.build()
    from paper_2504_03697_gb300 import cfd as _cfd
    return _cfd


def grid(t, shape, level):
    """GPU channels-last [V, C] -> float64 [C, Z, Y, X]."""
    nx, ny, nz = (s >> level for s in shape)
    return t.double().reshape(nz, ny, nx, -1).permute(3, 0, 1, 2).contiguous()


def bf16_layers(flat):
    return [(w.to(torch.bfloat16).double(), b.float().double()) for w, b in ou.unflatten(flat.double())]


def chunks_of(c_in, ks):
    return 2 if (c_in == 1 and ks == 3) else ks ** 3 * ((c_in + 15) // 16)


def check(got, ref, bound, what):
    bad = (got - ref).abs() > bound
    assert not bool(bad.any()), f"{what}: {int(bad.sum())} of {bad.numel()} outside, worst ratio " \
                                f"{float(((got - ref).abs() / bound.clamp_min(1e-300)).max()):.3g}"


def conv_check(got, x, w, b, what, bf16_out=True, ch=None):
    """ch: number of FP32 roundings of the accumulation (default: the tensor
    core's 16-deep K chunks; the CUDA-core first layer and head sum their 27
    taps / 16 channels one term at a time)."""
    ref = ou.conv(x, w, b)
    terms = ou.conv(x.abs(), w.abs(), b.abs() if b is not None else None)
    ch = chunks_of(x.shape[0], w.shape[-1]) if ch is None else ch
    bound = 4 * (ch + 1) * E * terms + (U * ref.abs() if bf16_out else 0)
    check(got, ref, bound, what)


def vjp(w, gout):
    """Input gradient of a stride-1 'same' convolution: the adjoint map."""
    x = torch.zeros((w.shape[1],) + tuple(gout.shape[1:]), dtype=torch.float64, requires_grad=True)
    y = ou.conv(x, w, None)
    (g,) = torch.autograd.grad(y, x, gout)
    return g


def run_pair(cfd, seed=0, lr=0.0):
    nx, ny, nz = SHAPE
    net = cfd.UNet(nx, ny, nz, seed=seed)
    r = torch.from_numpy(uniform_field((nz, ny, nx), seed + 1)).cuda()
    e = torch.from_numpy(uniform_field((nz, ny, nx), seed + 2)).cuda()
    w0 = net.get_params()
    loss = net.train_step(r, e, lr=lr)
    torch.cuda.synchronize()
    T = {name: grid(net.read_tensor(name), SHAPE, cfd.UNET_LEVELS[i]) for i, name in enumerate(cfd.UNET_TENSORS)}
    return net, r.cpu().numpy(), e.cpu().numpy(), w0, loss, T


def test_forward_layerwise(cfd):
    net, r, e, w0, loss, T = run_pair(cfd)
    L = bf16_layers(w0)
    # input scaling
    s = np.sqrt(r.size) / np.linalg.norm(r)
    xin_ref = torch.from_numpy(r * s)[None]
    check(T["xin"], xin_ref, U * xin_ref.abs() + 1e-12, "xin")
    conv_check(T["a0"], T["xin"], *L[0], "L0a", ch=27)
    conv_check(T["s0"], T["a0"], *L[1], "L0b")
    p0 = ou.pool2(T["s0"])
    check(T["p0"], p0, U * p0.abs() + 8 * E * ou.pool2(T["s0"].abs()), "pool0")
    conv_check(T["a1"], T["p0"], *L[2], "L1a")
    conv_check(T["s1"], T["a1"], *L[3], "L1b")
    p1 = ou.pool2(T["s1"])
    check(T["p1"], p1, U * p1.abs() + 8 * E * ou.pool2(T["s1"].abs()), "pool1")
    conv_check(T["a2"], T["p1"], *L[4], "L2a")
    conv_check(T["s2"], T["a2"], *L[5], "L2b")
    assert torch.equal(T["u1"], ou.up2(T["s2"]))
    conv_check(T["d1"], torch.cat([T["s1"], T["u1"]]), *L[6], "L1c")
    assert torch.equal(T["u0"], ou.up2(T["d1"]))
    conv_check(T["d0"], torch.cat([T["s0"], T["u0"]]), *L[7], "L0c")
    z = grid(net.read_tensor(cfd.UNET_T_OUT), SHAPE, 0)
    conv_check(z, T["d0"], *L[8], "head", bf16_out=False, ch=16)


@pytest.mark.parametrize("shape", [(16, 12, 8), (128, 8, 8), (40, 24, 16)])
def test_pipelined_convolutions_are_bitwise_equal(cfd, shape):
    # the staging modes of the tiled convolution (one CTA per tile with one
    # or two stages, and the persistent warp-specialised kernel) issue the
    # same MMAs in the same order: forward outputs and all gradients agree
    # bitwise
    nx, ny, nz = shape
    r = torch.from_numpy(uniform_field((nz, ny, nx), 71)).cuda()
    e = torch.from_numpy(uniform_field((nz, ny, nx), 72)).cuda()
    outs = []
    for mode in ("bulk", "two_stage", "registers", "persistent"):
        net = cfd.UNet(nx, ny, nz, seed=29)
        net.set_conv_mode(mode)
        net.train_step(r, e, lr=0.0)
        outs.append([net.read_tensor(name) for name in cfd.UNET_TENSORS] + [net.read_tensor(cfd.UNET_T_GRAD)])
    for name, a, b, c, d in zip(cfd.UNET_TENSORS + ["grad"], *outs):
        assert torch.equal(a, b) and torch.equal(a, c) and torch.equal(a, d), name


def test_apply_output_is_scaled_zero_mean(cfd):
    nx, ny, nz = SHAPE
    net = cfd.UNet(nx, ny, nz, seed=5)
    r = torch.from_numpy(gaussian_rhs(nx, ny, nz, 3)).cuda()
    z = torch.empty_like(r)
    net.apply(r, z)
    torch.cuda.synchronize()
    out = net.read_tensor(cfd.UNET_T_OUT).double().numpy()
    rn = r.cpu().numpy().reshape(-1)
    s = np.sqrt(rn.size) / np.linalg.norm(rn)
    ref = (out - out.mean()) / s
    got = z.cpu().numpy().reshape(-1)
    assert np.allclose(got, ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())
    assert abs(got.mean()) <= 1e-12 * np.abs(got).max()


def test_backward_layerwise(cfd):
    net, r, e, w0, loss, T = run_pair(cfd, seed=7)
    L = bf16_layers(w0)
    V = r.size
    z = grid(net.read_tensor(cfd.UNET_T_OUT), SHAPE, 0)
    t = grid(net.read_tensor(cfd.UNET_T_TARGET), SHAPE, 0)
    # loss and its gradient
    assert abs(loss - float(((z - t) ** 2).mean())) <= 1e-5 * loss
    gz = 2.0 / V * (z - t)
    check(T["gz"], gz, (U + 2 * E) * gz.abs() + 1e-300, "gz")

    def dgrad_check(got, w, gout, what, extra=None):
        ref = vjp(w, gout)
        terms = vjp(w.abs(), gout.abs())
        ch = chunks_of(w.shape[0], w.shape[-1])
        bound = 4 * (ch + 1) * E * terms + U * ref.abs()
        if extra is not None:  # a second addend (pool adjoint) and a second rounding
            ref = ref + extra
            bound = bound + U * (ref.abs() + extra.abs())
        check(got, ref, bound, what)

    dgrad_check(T["g_d0"], L[8][0], T["gz"], "head dgrad")
    pool0_adj = ou.up2(T["g_p0"]) / 8
    dgrad_check(T["g_u0"], L[7][0][:, 16:], T["g_d0"], "L0c dgrad (up half)")
    dgrad_check(T["g_s0"], L[7][0][:, :16], T["g_d0"], "L0c dgrad (skip half) + pool adjoint", extra=pool0_adj)
    # up-sampling adjoint: sum of the 8 children
    ref = 8 * ou.pool2(T["g_u0"])
    check(T["g_d1"], ref, U * ref.abs() + 8 * E * 8 * ou.pool2(T["g_u0"].abs()), "up adjoint 1")
    dgrad_check(T["g_u1"], L[6][0][:, 32:], T["g_d1"], "L1c dgrad (up half)")
    dgrad_check(T["g_s1"], L[6][0][:, :32], T["g_d1"], "L1c dgrad (skip half) + pool adjoint",
                extra=ou.up2(T["g_p1"]) / 8)
    ref = 8 * ou.pool2(T["g_u1"])
    check(T["g_s2"], ref, U * ref.abs() + 8 * E * 8 * ou.pool2(T["g_u1"].abs()), "up adjoint 2")
    dgrad_check(T["g_a2"], L[5][0], T["g_s2"], "L2b dgrad")
    dgrad_check(T["g_p1"], L[4][0], T["g_a2"], "L2a dgrad")
    dgrad_check(T["g_a1"], L[3][0], T["g_s1"], "L1b dgrad")
    dgrad_check(T["g_p0"], L[2][0], T["g_a1"], "L1a dgrad")
    dgrad_check(T["g_a0"], L[1][0], T["g_s0"], "L0b dgrad")

    # weight and bias gradients from the GPU's own BF16 activations
    grads = ou.unflatten(net.read_tensor(cfd.UNET_T_GRAD).double())
    ins = [[T["xin"]], [T["a0"]], [T["p0"]], [T["a1"]], [T["p1"]], [T["a2"]], [T["s1"], T["u1"]],
           [T["s0"], T["u0"]], [T["d0"]]]
    outs = [T["g_a0"], T["g_s0"], T["g_a1"], T["g_s1"], T["g_a2"], T["g_s2"], T["g_d1"], T["g_d0"], T["gz"]]
    for li, (name, lv, c0, c1, cout, ks) in enumerate(ou.LAYERS):
        x = torch.cat(ins[li]).requires_grad_(False)
        w = torch.zeros(cout, c0 + c1, ks, ks, ks, dtype=torch.float64, requires_grad=True)
        (gw,) = torch.autograd.grad(ou.conv(x, w, None), w, outs[li])
        (tw,) = torch.autograd.grad(ou.conv(x.abs(), w, None), w, outs[li].abs())
        Vl = x[0].numel()
        bound = 2 * (Vl / 32 + 34) * E * tw + 1e-30
        check(grads[li][0], gw, bound, f"{name} weight gradient")
        gb = outs[li].sum(dim=(1, 2, 3))
        tb = outs[li].abs().sum(dim=(1, 2, 3))
        check(grads[li][1], gb, 2 * (Vl / 32 + 34) * E * tb + 1e-30, f"{name} bias gradient")


def test_tensor_core_weight_gradients_match_cuda_cores_and_repeat(cfd):
    """The weight gradients of the 3x3x3 layers on the tensor cores (the
    default) against the FP32 CUDA-core sums of the same BF16 activations, on
    a 32^3 grid: both are sums of the same exact BF16 products in FP32, so
    they differ by at most the sum of their rounding bounds (CUDA cores: 32
    chunks of V/32 sequential terms, then the chunk sum; tensor cores: at most
    V/16 accumulated K-blocks of 16 products per CTA, then at most 160 chunk
    partials), times sum |terms|.  The tensor-core gradient repeats bit for
    bit.  One training step is timed in each mode (printed)."""
    shape = (32, 32, 32)
    nx, ny, nz = shape
    r = torch.from_numpy(uniform_field((nz, ny, nx), 51)).cuda()
    e = torch.from_numpy(uniform_field((nz, ny, nx), 52)).cuda()
    grads, ms = {}, {}
    for mode in ("tensor", "cuda_cores", "tensor"):
        net = cfd.UNet(nx, ny, nz, seed=5)
        net.set_wgrad_mode(mode)
        net.train_step(r, e, lr=0.0)  # warm-up (the gradient is recomputed below)
        st, en = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        st.record()
        net.train_step(r, e, lr=0.0)
        en.record()
        torch.cuda.synchronize()
        ms.setdefault(mode, []).append(st.elapsed_time(en))
        g = net.read_tensor(cfd.UNET_T_GRAD).double()
        if mode in grads:
            assert torch.equal(g, grads[mode]), "tensor-core weight gradient not bitwise repeatable"
        grads[mode] = g
        if mode == "cuda_cores":
            T = {name: grid(net.read_tensor(name), shape, cfd.UNET_LEVELS[i]) for i, name in enumerate(cfd.UNET_TENSORS)}
    tcg, ccg = ou.unflatten(grads["tensor"]), ou.unflatten(grads["cuda_cores"])
    ins = [[T["xin"]], [T["a0"]], [T["p0"]], [T["a1"]], [T["p1"]], [T["a2"]], [T["s1"], T["u1"]],
           [T["s0"], T["u0"]], [T["d0"]]]
    outs = [T["g_a0"], T["g_s0"], T["g_a1"], T["g_s1"], T["g_a2"], T["g_s2"], T["g_d1"], T["g_d0"], T["gz"]]
    for li, (name, lv, c0, c1, cout, ks) in enumerate(ou.LAYERS):
        if ks != 3 or c0 == 1:
            continue
        x = torch.cat(ins[li]).abs()
        w = torch.zeros(cout, c0 + c1, ks, ks, ks, dtype=torch.float64, requires_grad=True)
        (tw,) = torch.autograd.grad(ou.conv(x, w, None), w, outs[li].abs())
        Vl = x[0].numel()
        bound = (2 * (Vl / 32 + 34) + (Vl / 16 + 160 + 34)) * E * tw + 1e-30
        check(tcg[li][0], ccg[li][0], bound, f"{name} weight gradient, tensor vs CUDA cores")
        tb = outs[li].abs().sum(dim=(1, 2, 3))
        check(tcg[li][1], ccg[li][1], (2 * (Vl / 32 + 34) + (Vl / 16 + 160 + 34)) * E * tb + 1e-30,
              f"{name} bias gradient, tensor vs CUDA cores")
    print(f"training step at 32^3: tensor cores {min(ms['tensor']):.2f} ms, CUDA cores {ms['cuda_cores'][0]:.2f} ms")


def test_anorm_loss_gradient(cfd):
    nx, ny, nz = SHAPE
    net = cfd.UNet(nx, ny, nz, seed=19)
    net.set_loss("anorm")
    r = torch.from_numpy(uniform_field((nz, ny, nx), 51)).cuda()
    e = torch.from_numpy(uniform_field((nz, ny, nx), 52)).cuda()
    loss = net.train_step(r, e, lr=0.0)
    z = net.read_tensor(cfd.UNET_T_OUT).double().reshape(nz, ny, nx)
    t = net.read_tensor(cfd.UNET_T_TARGET).double().reshape(nz, ny, nx)
    d = z - t
    ad = ou.neumann_apply(d)
    V = d.numel()
    assert abs(loss - float((d * ad).sum()) / V) <= 1e-4 * abs(loss)
    ref = 2.0 / V * ad
    # sum of |terms| of a stencil row: n_c |d_c| + sum_n |d_n| = 2 n_c |d_c| - (A |d|)_c,
    # n_c the number of in-grid neighbours
    zz, yy, xx = (torch.arange(k) for k in d.shape)
    deg = sum(((c > 0).double() + (c < c.numel() - 1).double()).reshape(shape)
              for c, shape in ((zz, (-1, 1, 1)), (yy, (1, -1, 1)), (xx, (1, 1, -1))))
    terms = 2.0 / V * (2 * deg * d.abs() - ou.neumann_apply(d.abs()))
    gz = net.read_tensor("gz").double().reshape(nz, ny, nx)
    check(gz, ref, U * ref.abs() + 8 * E * terms + 1e-300, "A-norm gz")


def test_cos_loss_gradient(cfd):
    nx, ny, nz = SHAPE
    net = cfd.UNet(nx, ny, nz, seed=23)
    net.set_loss("cos")
    r = torch.from_numpy(uniform_field((nz, ny, nx), 61)).cuda()
    e = torch.from_numpy(uniform_field((nz, ny, nx), 62)).cuda()
    loss = net.train_step(r, e, lr=0.0)
    z = net.read_tensor(cfd.UNET_T_OUT).double().reshape(nz, ny, nx)
    t = net.read_tensor(cfd.UNET_T_TARGET).double().reshape(nz, ny, nx)
    az, at = ou.neumann_apply(z), ou.neumann_apply(t)
    a, b, T = float((z * az).sum()), float((z * at).sum()), float((t * at).sum())
    assert abs(loss - (1 - b / np.sqrt(a * T))) <= 1e-5
    c = b / a
    k = 1 / np.sqrt(a * T)
    ref = k * (c * az - at)
    zz, yy, xx = (torch.arange(m) for m in z.shape)
    deg = sum(((q > 0).double() + (q < q.numel() - 1).double()).reshape(shape)
              for q, shape in ((zz, (-1, 1, 1)), (yy, (1, -1, 1)), (xx, (1, 1, -1))))
    terms_z = 2 * deg * z.abs() - ou.neumann_apply(z.abs())
    terms_t = 2 * deg * t.abs() - ou.neumann_apply(t.abs())
    # FP32 stencils (8 roundings), c and k from FP32-based FP64 sums (1e-5 relative), BF16 output
    bound = U * ref.abs() + abs(k) * (abs(c) * terms_z + terms_t) * 8 * E + 1e-5 * abs(k) * ((c * az).abs() + at.abs())
    gz = net.read_tensor("gz").double().reshape(nz, ny, nx)
    check(gz, ref, bound, "cos-loss gz")


def test_gradient_sums_over_pairs(cfd):
    nx, ny, nz = SHAPE
    r = torch.from_numpy(np.stack([uniform_field((nz, ny, nx), 20 + k) for k in range(2)])).cuda()
    e = torch.from_numpy(np.stack([uniform_field((nz, ny, nx), 30 + k) for k in range(2)])).cuda()
    g = []
    for sl in (slice(0, 1), slice(1, 2), slice(0, 2)):
        net = cfd.UNet(nx, ny, nz, seed=11)
        net.train_step(r[sl].contiguous(), e[sl].contiguous(), lr=0.0)
        g.append(net.read_tensor(cfd.UNET_T_GRAD).double())
    scale = g[0].abs() + g[1].abs()
    assert torch.all((g[2] - g[0] - g[1]).abs() <= 4 * E * scale + 1e-30)


def test_adam_first_step(cfd):
    net, r, e, w0, loss, T = run_pair(cfd, seed=13, lr=1e-3)
    w1 = net.get_params().double()
    g = net.read_tensor(cfd.UNET_T_GRAD).double()
    m = net.read_tensor(cfd.UNET_T_ADAM_M).double()
    v = net.read_tensor(cfd.UNET_T_ADAM_V).double()
    # the kernel's FP32 constants: 1 - 0.9f and 1 - 0.999f
    c1 = 1.0 - float(np.float32(0.9))
    c2 = 1.0 - float(np.float32(0.999))
    assert torch.allclose(m, c1 * g, rtol=1e-6, atol=0)
    assert torch.allclose(v, c2 * g * g, rtol=1e-6, atol=0)
    big = g.abs() > 1e-5
    step = w1 - w0.double()
    assert torch.allclose(step[big], -1e-3 * torch.sign(g[big]), rtol=1e-3, atol=1e-9)
    ref, _, _ = ou.adam_step(w0.double(), torch.zeros_like(g), torch.zeros_like(g), g, 1, 1e-3)
    assert torch.allclose(w1, ref, rtol=0, atol=1e-6)


def test_end_to_end_close_to_float64_network(cfd):
    nx, ny, nz = SHAPE
    net = cfd.UNet(nx, ny, nz, seed=17)
    r = gaussian_rhs(nx, ny, nz, 4)
    rd = torch.from_numpy(r).cuda()
    z = torch.empty_like(rd)
    net.apply(rd, z)
    torch.cuda.synchronize()
    ref = ou.precondition(ou.unflatten(net.get_params().double()), r)
    err = np.linalg.norm(z.cpu().numpy() - ref) / np.linalg.norm(ref)
    print(f"BF16 network vs float64 network: relative L2 error {err:.3e}")
    assert err < 0.05


def lam_min(shape):
    return min(4 * np.sin(np.pi / (2 * n)) ** 2 for n in shape if n > 1)


@pytest.mark.parametrize("shape", [(32, 32, 32), (24, 16, 20)])
def test_fpcg_solves_to_true_residual(cfd, shape):
    nx, ny, nz = shape
    net = cfd.UNet(nx, ny, nz, seed=1)
    b = gaussian_rhs(nx, ny, nz, 21)
    bd = torch.from_numpy(b).cuda()
    x = torch.zeros_like(bd)
    rc, st = net.fpcg_solve(bd, x, rtol=1e-8)
    assert rc == 0 and st["status"] == 0, st
    A = poisson_csr(nx, ny, nz)
    bm = b.reshape(-1) - b.mean()
    xg = x.cpu().numpy().reshape(-1)
    rel = np.linalg.norm(bm - A @ xg) / np.linalg.norm(bm)
    assert rel <= 1e-8 and abs(rel - st["rel_resid"]) <= 1e-3 * rel + 1e-15
    xo, so = pcg(A, bm, rtol=1e-10, max_iters=5000)
    d = (xg - xg.mean()) - (xo - xo.mean())
    assert np.linalg.norm(d) <= 2 * 1e-8 * np.linalg.norm(bm) / lam_min(shape)
    print(f"{shape}: FPCG {st['iters']} iterations (plain {st['outer_iters']}, restarts {st['restarts']}), "
          f"oracle CG {so.iters}")


def passthrough_params(head_sign=1.0):
    """Every layer passes channel 0 (centre tap); the head multiplies by
    head_sign: M(r) = head_sign (r + B2 r + B4 r) up to the mean."""
    layers = []
    for name, _, c0, c1, cout, ks in ou.LAYERS:
        w = torch.zeros(cout, c0 + c1, ks, ks, ks, dtype=torch.float64)
        m = ks // 2
        w[0, 0, m, m, m] = head_sign if name == "head" else 1.0
        if c1:
            w[0, c0, m, m, m] = 1.0
        layers.append((w, torch.zeros(cout, dtype=torch.float64)))
    return ou.flatten(layers).float()


def test_fpcg_negative_preconditioner_scale_is_harmless(cfd):
    # M and -M give the same flexible-CG iterates (exactly: BF16 negation is
    # exact and every step is sign-symmetric), with no fallback
    nx, ny, nz = 16, 16, 16
    b = torch.from_numpy(gaussian_rhs(nx, ny, nz, 22)).cuda()
    out = []
    for sign in (1.0, -1.0):
        net = cfd.UNet(nx, ny, nz, seed=2)
        net.set_params(passthrough_params(sign))
        x = torch.zeros_like(b)
        rc, st = net.fpcg_solve(b, x, rtol=1e-8)
        assert rc == 0 and st["outer_iters"] == 0 and st["rel_resid"] <= 1e-8, st
        out.append((st["iters"], x.cpu()))
    assert out[0][0] == out[1][0]
    assert torch.allclose(out[0][1], out[1][1], rtol=0, atol=1e-12 * float(out[0][1].abs().max()))


def test_fpcg_falls_back_on_breakdown(cfd):
    # an all-zero network gives z = 0, so z.r = 0 at once: plain CG from there
    nx, ny, nz = 16, 16, 16
    net = cfd.UNet(nx, ny, nz, seed=2)
    net.set_params(torch.zeros(net.nparams))
    b = torch.from_numpy(gaussian_rhs(nx, ny, nz, 22)).cuda()
    x = torch.zeros_like(b)
    rc, st = net.fpcg_solve(b, x, rtol=1e-8)
    assert rc == 0 and st["restarts"] >= 1 and st["outer_iters"] == st["iters"] > 0, st
    assert st["rel_resid"] <= 1e-8


def test_fpcg_zero_rhs_and_cap(cfd):
    net = cfd.UNet(8, 8, 8, seed=3)
    b = torch.zeros(8 * 8 * 8, dtype=torch.float64, device="cuda")
    x = torch.full_like(b, 5.0)
    rc, st = net.fpcg_solve(b, x)
    assert rc == 0 and st["iters"] == 0 and not bool(x.any())
    b = torch.from_numpy(gaussian_rhs(8, 8, 8, 23)).cuda()
    rc, st = net.fpcg_solve(b, x, rtol=1e-12, max_iters=2)
    assert rc == cfd.CFD_ERR_NOT_CONVERGED and st["iters"] == 2


def test_training_lowers_the_loss(cfd):
    nx, ny, nz = 16, 16, 16
    net = cfd.UNet(nx, ny, nz, seed=4)
    A = poisson_csr(nx, ny, nz)
    # pairs (r, e) with r = A e, e a smooth random field (low DCT modes)
    pairs_r, pairs_e = [], []
    for k in range(4):
        e = uniform_field((nz, ny, nx), 40 + k)
        for _ in range(6):  # Jacobi-style smoothing of the error field
            e = (e + np.roll(e, 1, 0) + np.roll(e, -1, 0) + np.roll(e, 1, 1) + np.roll(e, -1, 1)
                 + np.roll(e, 1, 2) + np.roll(e, -1, 2)) / 7
        e = e - e.mean()
        pairs_e.append(e)
        pairs_r.append((A @ e.reshape(-1)).reshape(e.shape))
    r = torch.from_numpy(np.stack(pairs_r)).cuda()
    e = torch.from_numpy(np.stack(pairs_e)).cuda()
    losses = [net.train_step(r, e, lr=2e-3) for _ in range(60)]
    print(f"loss {losses[0]:.4g} -> {losses[-1]:.4g}")
    assert losses[-1] < 0.7 * losses[0]


def test_cavity_steps_with_the_learned_preconditioner(cfd):
    """A cavity whose pressure solves run flexible PCG with an attached
    network (solver 'fpcg'): every solve meets the FP64 true-residual rule
    and the fields follow the plain-CG run within what two rtol-solutions
    may differ by (|dp| <= 2 rtol ||b|| / lambda_min per solve)."""
    from paper_2504_03697_gb300.synthetic import cavity_perturbation
    n, steps = 16, 3
    net = cfd.UNet(n, n, n, seed=2)
    net.set_params(passthrough_params(1.0))
    runs = {}
    for solver, form in (("fpcg", "host"), ("fpcg", "graph"), ("cg", None)):
        cav = cfd.Cavity(cfd.make_params(n, n, n, dt=0.01, nu=0.01, lid_u=1.0, solver=solver))
        if solver == "fpcg":
            cav.attach_preconditioner(net)
            cav.set_fpcg_form(form)
        for name, f in zip("uvw", cavity_perturbation(n, n, n, seed=4, amp=1e-3)):
            cav.set_field(name, f)
        rc, stats = cav.step(steps)
        assert rc == 0 and all(s["status"] == 0 and s["rel_resid"] <= 1e-8 for s in stats), stats
        runs[form] = ({f: cav.read_field(f).numpy() for f in "uvwp"}, stats)
    b, sb = runs[None]
    for form in ("host", "graph"):
        a, sa = runs[form]
        # the network's steps were used, no fallback (host form: outer_iters
        # counts plain iterations; graph form: restarts does)
        assert all((s["outer_iters"] if form == "host" else s["restarts"]) == 0 for s in sa)
        assert sum(s["iters"] for s in sa) < sum(s["iters"] for s in sb)  # the pass-through network helps
        for f in "uvwp":
            scale = max(1.0, float(np.abs(b[f]).max()))
            assert float(np.abs(a[f] - b[f]).max()) <= 1e-5 * scale, (form, f)


def test_fpcg_cavity_without_a_network_is_an_error(cfd):
    cav = cfd.Cavity(cfd.make_params(8, 8, 8, solver="fpcg"))
    with pytest.raises(cfd.CfdError):
        cav.step(1)
    net = cfd.UNet(16, 16, 16, seed=1)
    with pytest.raises(cfd.CfdError):
        cav.attach_preconditioner(net)  # grid mismatch
