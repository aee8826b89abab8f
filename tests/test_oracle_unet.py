"""Pins of the learned-preconditioner oracle (oracle/unet.py) and of the
flexible PCG (oracle/krylov.fpcg) against closed forms, adjoint identities,
finite differences and the textbook PCG."""
import numpy as np
import pytest
import torch

from oracle import krylov, operators, unet


def block_mean(x, k):
    """Mean over k x k x k blocks of a (Z, Y, X) array, broadcast back."""
    Z, Y, X = x.shape
    m = x.reshape(Z // k, k, Y // k, k, X // k, k).mean(axis=(1, 3, 5))
    return np.repeat(np.repeat(np.repeat(m, k, 0), k, 1), k, 2)


def test_pool_up_identity_and_adjoint():
    g = torch.Generator().manual_seed(0)
    c = torch.randn(3, 4, 5, 6, generator=g, dtype=torch.float64)
    assert torch.allclose(unet.pool2(unet.up2(c)), c, rtol=1e-15, atol=0)
    f = torch.randn(3, 8, 10, 12, generator=g, dtype=torch.float64)
    # <pool f, c> = <f, up c> / 8
    lhs = float((unet.pool2(f) * c).sum())
    rhs = float((f * unet.up2(c)).sum()) / 8
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs) + 1e-12
    # pooling is the block mean
    assert np.allclose(unet.up2(unet.pool2(f))[0].numpy(), block_mean(f[0].numpy(), 2), atol=1e-14)


def test_conv_delta_and_shift():
    g = torch.Generator().manual_seed(1)
    x = torch.randn(2, 5, 6, 7, generator=g, dtype=torch.float64)
    w = torch.zeros(2, 2, 3, 3, 3, dtype=torch.float64)
    w[0, 0, 1, 1, 1] = 1.0
    w[1, 1, 1, 1, 1] = 1.0
    assert torch.equal(unet.conv(x, w, None), x)
    # tap (kz, ky, kx) = (1, 1, 2) reads x[.., i + 1]: a shift with zero fill
    w2 = torch.zeros(1, 2, 3, 3, 3, dtype=torch.float64)
    w2[0, 1, 1, 1, 2] = 1.0
    y = unet.conv(x, w2, torch.tensor([0.5], dtype=torch.float64))[0]
    ref = torch.full_like(x[1], 0.5)
    ref[:, :, :-1] += x[1, :, :, 1:]
    assert torch.equal(y, ref)


def passthrough_layers(up_weight=(1.0, 1.0)):
    """Every layer passes channel 0 (centre tap); the concat layers L1c and
    L0c add skip channel 0 and up_weight times up-sampled channel 0."""
    layers = []
    for name, _, c0, c1, cout, ks in unet.LAYERS:
        w = torch.zeros(cout, c0 + c1, ks, ks, ks, dtype=torch.float64)
        m = ks // 2
        w[0, 0, m, m, m] = 1.0
        if c1:
            w[0, c0, m, m, m] = up_weight[0] if name == "L1c" else up_weight[1]
        layers.append((w, torch.zeros(cout, dtype=torch.float64)))
    return layers


def test_passthrough_network_closed_form():
    x = np.random.default_rng(2).standard_normal((8, 12, 16))
    z, _ = unet.forward(passthrough_layers(), torch.from_numpy(x)[None])
    ref = x + block_mean(x, 2) + block_mean(x, 4)
    assert np.allclose(z[0].numpy(), ref, atol=1e-13)
    # distinct weights on the up-sampled halves fix the concatenation order:
    # d1 = s1 + 2 up(s2), d0 = s0 + 3 up(d1) -> x + 3 B2 x + 6 B4 x
    z, _ = unet.forward(passthrough_layers((2.0, 3.0)), torch.from_numpy(x)[None])
    assert np.allclose(z[0].numpy(), x + 3 * block_mean(x, 2) + 6 * block_mean(x, 4), atol=1e-12)


def test_bf16_storage_emulation():
    """store=bf16_store rounds what the CUDA network stores: every stored
    activation is a BF16 value; on small integer inputs whose block means
    are BF16 values nothing rounds (output = the float64 output); on a
    Gaussian input the output stays within a few BF16 roundings of the
    float64 output."""
    rng = np.random.default_rng(5)
    layers = passthrough_layers((2.0, 3.0))
    x = rng.standard_normal((8, 12, 16))
    z, acts = unet.forward(layers, torch.from_numpy(x)[None], store=unet.bf16_store)
    for name, t in acts.items():
        assert torch.equal(t, t.to(torch.bfloat16).to(torch.float64)), name
    z64, _ = unet.forward(layers, torch.from_numpy(x)[None])
    bound = 16 * 2.0 ** -9 * (np.abs(x) + 3 * np.abs(block_mean(x, 2)) + 6 * np.abs(block_mean(x, 4)))
    assert np.all(np.abs(z[0].numpy() - z64[0].numpy()) <= bound)
    assert not np.array_equal(z[0].numpy(), z64[0].numpy())  # something was rounded
    # entries 64 k, k in {-1, 0, 1}: every activation of the unit pass-through
    # network is an integer of magnitude <= 192, exact in BF16
    xi = 64.0 * rng.integers(-1, 2, size=(8, 12, 16)).astype(np.float64)
    zi, _ = unet.forward(passthrough_layers(), torch.from_numpy(xi)[None], store=unet.bf16_store)
    zi64, _ = unet.forward(passthrough_layers(), torch.from_numpy(xi)[None])
    assert torch.equal(zi, zi64)


def test_flat_layout_roundtrip_and_tap_order():
    assert unet.param_count() == sum(ks ** 3 * co * (a + b) + co for _, _, a, b, co, ks in unet.LAYERS)
    flat = torch.arange(unet.param_count(), dtype=torch.float64)
    assert torch.equal(unet.flatten(unet.unflatten(flat)), flat)
    # weight [tap][cout][cin] with tap = kx + 3 ky + 9 kz: element
    # (tap=5 -> kx 2, ky 1, kz 0; co 3; ci 0) of layer L0a (cin 1, cout 16)
    w0 = unet.unflatten(flat)[0][0]
    assert w0[3, 0, 0, 1, 2] == 5 * 16 + 3


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(3)
    flat = torch.from_numpy(rng.standard_normal(unet.param_count()) * 0.1)
    r = rng.standard_normal((4, 4, 8))
    e = rng.standard_normal((4, 4, 8))
    loss, grad = unet.loss_and_grad(flat, [(r, e)])
    for idx in [0, 500, 7000, 40000, unet.param_count() - 1, unet.param_count() - 20]:
        d = torch.zeros_like(flat)
        d[idx] = 1e-6
        fp, _ = unet.loss_and_grad(flat + d, [(r, e)])
        fm, _ = unet.loss_and_grad(flat - d, [(r, e)])
        fd = (fp - fm) / 2e-6
        assert abs(fd - float(grad[idx])) <= 1e-6 * max(1.0, abs(fd)), (idx, fd, float(grad[idx]))


def test_neumann_apply_matches_csr_and_null_space():
    rng = np.random.default_rng(12)
    d = rng.standard_normal((3, 4, 5))
    got = unet.neumann_apply(torch.from_numpy(d)).numpy().reshape(-1)
    ref = operators.poisson_csr(5, 4, 3) @ d.reshape(-1)
    assert np.allclose(got, ref, atol=1e-13)
    assert np.allclose(unet.neumann_apply(torch.full((3, 4, 5), 2.5, dtype=torch.float64)).numpy(), 0.0)


def test_anorm_gradient_matches_finite_differences():
    rng = np.random.default_rng(13)
    flat = torch.from_numpy(rng.standard_normal(unet.param_count()) * 0.1)
    r = rng.standard_normal((4, 4, 8))
    e = rng.standard_normal((4, 4, 8))
    loss, grad = unet.loss_and_grad(flat, [(r, e)], loss="anorm")
    assert loss > 0
    for idx in [3, 9000, unet.param_count() - 2]:
        dlt = torch.zeros_like(flat)
        dlt[idx] = 1e-6
        fp, _ = unet.loss_and_grad(flat + dlt, [(r, e)], loss="anorm")
        fm, _ = unet.loss_and_grad(flat - dlt, [(r, e)], loss="anorm")
        fd = (fp - fm) / 2e-6
        assert abs(fd - float(grad[idx])) <= 1e-6 * max(1.0, abs(fd))


def test_cos_loss_gradient_and_invariance():
    rng = np.random.default_rng(14)
    flat = torch.from_numpy(rng.standard_normal(unet.param_count()) * 0.1)
    r = rng.standard_normal((4, 4, 8))
    e = rng.standard_normal((4, 4, 8))
    loss, grad = unet.loss_and_grad(flat, [(r, e)], loss="cos")
    assert 0.0 <= loss <= 2.0
    for idx in [5, 12000, unet.param_count() - 3]:
        dlt = torch.zeros_like(flat)
        dlt[idx] = 1e-6
        fp, _ = unet.loss_and_grad(flat + dlt, [(r, e)], loss="cos")
        fm, _ = unet.loss_and_grad(flat - dlt, [(r, e)], loss="cos")
        fd = (fp - fm) / 2e-6
        assert abs(fd - float(grad[idx])) <= 1e-6 * max(1.0, abs(fd))
    # the loss ignores the scale of the network output (head weights and bias x 3)
    layers = unet.unflatten(flat)
    layers[-1] = (layers[-1][0] * 3.0, layers[-1][1] * 3.0)
    l3, _ = unet.loss_and_grad(unet.flatten(layers), [(r, e)], loss="cos")
    assert abs(l3 - loss) <= 1e-12
    # a target that is a positive multiple of the network's output has zero
    # loss, a negative multiple the maximum 2
    s = unet.scale_of(r)
    z, _ = unet.forward(unet.unflatten(flat), torch.from_numpy(r * s)[None])
    l0, _ = unet.loss_and_grad(flat, [(r, 2.0 * z[0].detach().numpy() / s)], loss="cos")
    l2, _ = unet.loss_and_grad(flat, [(r, -2.0 * z[0].detach().numpy() / s)], loss="cos")
    assert abs(l0) <= 1e-12 and abs(l2 - 2.0) <= 1e-12


def test_adam_first_step_is_sign():
    g = torch.tensor([3.0, -0.5, 1e-2, -7.0], dtype=torch.float64)
    w = torch.tensor([1.0, 2.0, 3.0, 4.0], dtype=torch.float64)
    w1, m, v = unet.adam_step(w, torch.zeros(4, dtype=torch.float64), torch.zeros(4, dtype=torch.float64), g, 1, 1e-3)
    assert torch.allclose(w1 - w, -1e-3 * torch.sign(g), rtol=1e-5, atol=0)
    assert torch.allclose(m, 0.1 * g) and torch.allclose(v, 0.001 * g * g)


def test_precondition_scale_invariant_zero_mean():
    rng = np.random.default_rng(4)
    layers = unet.unflatten(torch.from_numpy(rng.standard_normal(unet.param_count()) * 0.2))
    r = rng.standard_normal((4, 8, 8))
    z1 = unet.precondition(layers, r)
    z2 = unet.precondition(layers, 37.5 * r)
    assert np.allclose(z2, 37.5 * z1, rtol=1e-12, atol=1e-12 * np.abs(z2).max())
    assert abs(z1.mean()) < 1e-14 * np.abs(z1).max()


# ---- flexible PCG ----------------------------------------------------------

def rhs(n, seed):
    b = np.random.default_rng(seed).standard_normal(n)
    return b - b.mean()


def test_fpcg_identity_matches_cg():
    A = operators.poisson_csr(6, 5, 4)
    b = rhs(A.shape[0], 5)
    x1, s1 = krylov.fpcg(A, b, lambda r: r.copy(), rtol=1e-10)
    x2, s2 = krylov.pcg(A, b, rtol=1e-10)
    assert s1.converged and s2.converged and not s1.fell_back
    assert abs(s1.iters - s2.iters) <= 1
    assert np.linalg.norm(x1 - x1.mean() - (x2 - x2.mean())) <= 1e-8 * np.linalg.norm(x2)


def test_fpcg_fixed_spd_matches_pcg_iterates():
    A = operators.poisson_csr(5, 5, 5)
    b = rhs(A.shape[0], 6)
    # fixed SPD preconditioner: symmetric positive diagonal scaling
    d = 1.0 + np.random.default_rng(7).random(A.shape[0])
    M = lambda r: r / d  # noqa: E731
    for k in (3, 8):
        _, s1 = krylov.fpcg(A, b, M, rtol=1e-30, max_iters=k)
        xf, _ = krylov.fpcg(A, b, M, rtol=1e-30, max_iters=k)
        xp, _ = krylov.pcg(A, b, precond=M, fixed_iters=k)
        assert s1.iters == k
        assert np.linalg.norm(xf - xp) <= 1e-10 * np.linalg.norm(xp)


def test_fpcg_exact_inverse_one_iteration():
    A = operators.poisson_csr(4, 4, 3)
    n = A.shape[0]
    P = np.eye(n) - np.ones((n, n)) / n
    Ainv = np.linalg.inv(A.toarray() + np.ones((n, n)) / n) @ P  # inverse on the zero-mean subspace
    b = rhs(n, 8)
    x, st = krylov.fpcg(A, b, lambda r: Ainv @ r, rtol=1e-10)
    assert st.converged and st.iters == 1


def test_fpcg_negative_scale_is_harmless():
    A = operators.poisson_csr(6, 6, 6)
    b = rhs(A.shape[0], 9)
    x1, s1 = krylov.fpcg(A, b, lambda r: -3.0 * r, rtol=1e-8)
    x2, s2 = krylov.fpcg(A, b, lambda r: r.copy(), rtol=1e-8)
    assert s1.converged and not s1.fell_back and s1.iters == s2.iters
    assert np.linalg.norm(x1 - x2) <= 1e-10 * np.linalg.norm(x2)


def test_fpcg_breakdown_falls_back():
    A = operators.poisson_csr(6, 6, 6)
    b = rhs(A.shape[0], 9)
    x, st = krylov.fpcg(A, b, lambda r: np.zeros_like(r), rtol=1e-8)
    assert st.fell_back and st.converged and st.plain_iters == st.iters
    assert st.rel_resid <= 1e-8


def test_fpcg_stagnation_falls_back():
    A = operators.poisson_csr(8, 8, 8)
    b = rhs(A.shape[0], 15)
    # a fresh random direction on every call: z.r != 0, but 50 steps along
    # random directions of a 512-dimensional space do not halve the residual
    rng = np.random.default_rng(16)
    x, st = krylov.fpcg(A, b, lambda r: rng.standard_normal(r.size), rtol=1e-8, stagnation=50)
    assert st.fell_back and st.converged and st.iters - st.plain_iters >= 50
    assert st.rel_resid <= 1e-8


def test_fpcg_zero_rhs():
    A = operators.poisson_csr(3, 3, 3)
    x, st = krylov.fpcg(A, np.zeros(27), lambda r: r, rtol=1e-8)
    assert st.converged and st.iters == 0 and not x.any()


def test_fpcg_with_random_unet_converges():
    rng = np.random.default_rng(10)
    layers = unet.unflatten(torch.from_numpy(rng.uniform(-1, 1, unet.param_count()) * 0.2))
    nx, ny, nz = 8, 8, 8
    A = operators.poisson_csr(nx, ny, nz)
    b = rhs(A.shape[0], 11)
    M = lambda r: unet.precondition(layers, r.reshape(nz, ny, nx)).reshape(-1)  # noqa: E731
    x, st = krylov.fpcg(A, b, M, rtol=1e-8, max_iters=400)
    assert st.converged and st.rel_resid <= 1e-8
