"""Learned U-Net preconditioner, plain float64 PyTorch CPU (oracle).

The paper preconditions its pressure CG with DIC or Jacobi (Sec. 3.1) and
lists other preconditioners as future work (Sec. 5).  The learned one is a
reading of that item (architecture, scaling and loss are not in the paper):

* network (linear: no activation functions)
    level 0: L0a 3^3 conv 1 -> 16, L0b 3^3 16 -> 16 (= skip s0)
    2x average pool
    level 1: L1a 3^3 16 -> 32, L1b 3^3 32 -> 32 (= skip s1)
    2x average pool
    level 2: L2a 3^3 32 -> 64, L2b 3^3 64 -> 64
    nearest 2x up-sampling, concatenate [s1, up]: L1c 3^3 96 -> 32
    nearest 2x up-sampling, concatenate [s0, up]: L0c 3^3 48 -> 16
    head 1^3 16 -> 1
  every convolution stride 1, zero padding ("same"), with bias;
* preconditioner M(r) = U(s r) / s minus its mean, s = sqrt(V) / ||r||;
* training loss on one pair (r, e), d = U(s r) - s e: mean over cells of
  d^2, the energy norm d.(A d) / V (A the Neumann pressure operator), or one
  minus the energy-norm cosine of U(s r) and s e (invariant to a positive
  scale of the output);
  Adam (beta 0.9 / 0.999, eps 1e-8) on the mean loss over a batch of pairs.

Parameters travel as one flat float vector: per layer in the order above,
weights [taps][cout][cin] with tap = kx + 3 ky + 9 kz, then bias [cout].
Tensors here are [C, Z, Y, X] float64 (x fastest in memory order).

Pins (tests/test_oracle_unet.py): pooling after up-sampling is the identity
and the two are adjoint up to the factor 8; a centre-tap identity kernel
reproduces its input and a one-tap kernel shifts it with zero fill; a
hand-set network whose layers pass channel 0 through computes x +
up(pool x) + up(up(pool(pool x))), checked against block means computed with
numpy reshapes; the loss operator against the assembled CSR matrix and its
null space; gradients against finite differences; one Adam step from
zero moments moves every weight by lr * sign(g) (|g| >> eps); M is
invariant to the scale of r; with ``store=bf16_store`` every stored
activation is a BF16 value, the pass-through network's output stays within
the BF16 rounding bound of its float64 output, and on inputs whose block
means are BF16 values it equals the float64 output.  This module is test infrastructure (see the
package header).
"""
from __future__ import annotations

import numpy as np
import torch
import torch.nn.functional as F

# (name, level, c0, c1, cout, ks) in parameter order
LAYERS = [("L0a", 0, 1, 0, 16, 3), ("L0b", 0, 16, 0, 16, 3), ("L1a", 1, 16, 0, 32, 3), ("L1b", 1, 32, 0, 32, 3),
          ("L2a", 2, 32, 0, 64, 3), ("L2b", 2, 64, 0, 64, 3), ("L1c", 1, 32, 64, 32, 3),
          ("L0c", 0, 16, 32, 16, 3), ("head", 0, 16, 0, 1, 1)]


def param_count() -> int:
    return sum(ks ** 3 * cout * (c0 + c1) + cout for _, _, c0, c1, cout, ks in LAYERS)


def unflatten(flat):
    """Flat parameter vector -> list of (weight [cout, cin, kz, ky, kx], bias)."""
    flat = torch.as_tensor(flat, dtype=torch.float64)
    out, o = [], 0
    for _, _, c0, c1, cout, ks in LAYERS:
        cin, taps = c0 + c1, ks ** 3
        w = flat[o:o + taps * cout * cin].reshape(ks, ks, ks, cout, cin)  # [kz][ky][kx][co][ci]
        o += taps * cout * cin
        b = flat[o:o + cout]
        o += cout
        out.append((w.permute(3, 4, 0, 1, 2).contiguous(), b.clone()))
    return out


def flatten(layers):
    parts = []
    for w, b in layers:
        parts.append(w.permute(2, 3, 4, 0, 1).reshape(-1))
        parts.append(b.reshape(-1))
    return torch.cat(parts)


def conv(x, w, b):
    """Stride-1 cross-correlation with zero padding: x [cin, Z, Y, X]."""
    return F.conv3d(x[None], w, b, padding=w.shape[-1] // 2)[0]


def pool2(x):
    """2x average pooling of [C, Z, Y, X] (each extent even)."""
    return F.avg_pool3d(x[None], 2)[0]


def up2(x):
    """Nearest 2x up-sampling of [C, Z, Y, X]."""
    return x.repeat_interleave(2, 1).repeat_interleave(2, 2).repeat_interleave(2, 3)


def bf16_store(t):
    """Round to the nearest BF16 value and back to float64: how the CUDA
    network stores its input and activations (BF16 storage, FP32
    accumulation).  Used only to compare with it in the same precision."""
    return t.to(torch.bfloat16).to(torch.float64)


def forward(layers, x, store=None):
    """U(x) for x [1, Z, Y, X]; returns (z [1, Z, Y, X], dict of activations).

    store (optional) is applied to the input and to every activation the
    network stores (each convolution and pooling output; up-sampling copies
    stored values, and the head's output is kept at float32 when store is
    given), e.g. ``bf16_store``; by default nothing is rounded."""
    s = store if store is not None else (lambda t: t)
    a = {"xin": s(x)}
    a["a0"] = s(conv(a["xin"], *layers[0]))
    a["s0"] = s(conv(a["a0"], *layers[1]))
    a["p0"] = s(pool2(a["s0"]))
    a["a1"] = s(conv(a["p0"], *layers[2]))
    a["s1"] = s(conv(a["a1"], *layers[3]))
    a["p1"] = s(pool2(a["s1"]))
    a["a2"] = s(conv(a["p1"], *layers[4]))
    a["s2"] = s(conv(a["a2"], *layers[5]))
    a["u1"] = up2(a["s2"])
    a["d1"] = s(conv(torch.cat([a["s1"], a["u1"]]), *layers[6]))
    a["u0"] = up2(a["d1"])
    a["d0"] = s(conv(torch.cat([a["s0"], a["u0"]]), *layers[7]))
    z = conv(a["d0"], *layers[8])
    if store is not None:
        z = z.to(torch.float32).to(torch.float64)
    return z, a


def scale_of(r: np.ndarray) -> float:
    nrm = float(np.linalg.norm(r))
    return np.sqrt(r.size) / nrm if nrm > 0 else 0.0


def precondition(layers, r: np.ndarray, store=None) -> np.ndarray:
    """M(r) = U(s r) / s with its mean removed; r shaped (Z, Y, X).  store
    as for ``forward``."""
    s = scale_of(r)
    if s == 0.0:
        return np.zeros_like(r)
    z, _ = forward(layers, torch.from_numpy(r * s)[None], store=store)
    z = z[0].numpy() / s
    return z - z.mean()


def neumann_apply(d):
    """(A d) for the Neumann 7-point pressure operator on a (Z, Y, X) field:
    sum over the neighbours inside the grid of (d_c - d_n)."""
    out = torch.zeros_like(d)
    for ax in range(3):
        n = d.shape[ax]
        if n < 2:
            continue
        diff = d.narrow(ax, 1, n - 1) - d.narrow(ax, 0, n - 1)
        out = out + F.pad(-diff, _pad_spec(ax, 0, 1)) + F.pad(diff, _pad_spec(ax, 1, 0))
    return out


def _pad_spec(ax, before, after):
    # F.pad lists (last dim first) pairs; a (Z, Y, X) tensor has ax 0 = Z
    spec = [0, 0, 0, 0, 0, 0]
    k = 2 * (2 - ax)
    spec[k], spec[k + 1] = before, after
    return spec


def loss_and_grad(flat, pairs, loss="mse"):
    """Mean over pairs of the training loss and its gradient w.r.t. the flat
    parameters (autograd).  With z = U(s r), t = s e, d = z - t: "mse" =
    mean(d^2), "anorm" = d.(A d) / V, "cos" = 1 - (z.A t) / sqrt((z.A z)(t.A t))."""
    p = torch.as_tensor(flat, dtype=torch.float64).clone().requires_grad_(True)
    layers = unflatten(p)
    total = 0.0
    for r, e in pairs:
        s = scale_of(r)
        z, _ = forward(layers, torch.from_numpy(r * s)[None])
        t = torch.from_numpy(e * s)[None]
        d = (z - t)[0]
        if loss == "anorm":
            total = total + (d * neumann_apply(d)).sum() / d.numel()
        elif loss == "cos":
            zz, tt = z[0], t[0]
            at = neumann_apply(tt)
            total = total + 1.0 - (zz * at).sum() / torch.sqrt((zz * neumann_apply(zz)).sum() * (tt * at).sum())
        else:
            total = total + (d ** 2).mean()
    total = total / len(pairs)
    total.backward()
    return float(total.detach()), p.grad.detach().clone()


def adam_step(w, m, v, g, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update at step t (1-based); returns (w, m, v)."""
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    return w - lr * mh / (vh ** 0.5 + eps), m, v
