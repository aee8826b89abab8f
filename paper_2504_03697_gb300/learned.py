"""Harvest, training and evaluation of the learned U-Net preconditioner.

The paper preconditions its pressure CG with DIC or Jacobi (Sec. 3.1) and
names other preconditioners as future work (Sec. 5); this module trains the
U-Net of ``cfd_unet_*`` for flexible PCG on the cavity's pressure systems.

Training data (a reading; the paper has no learned component): lid-driven
cavities at n^3 with nu ~ log-uniform[1e-4, 1e-2] and lid speed ~
uniform[0.5, 2] drawn from the seed, dt 0.01, started from the seeded
perturbation.  At selected steps the projection's right-hand side b is
taken after forces, advection and diffusion (``cfd_pressure_rhs``), solved
to rtol 1e-12 for x*, and the CG iterates x_k (k = 0, 1, 2, 4, ...; x_0 =
0, the pair the initial-guess mode uses) give the pairs r_k = b - A x_k,
e_k = x* - x_k (mean removed).  The whole data set stays resident in HBM;
each Adam step takes a minibatch of pairs.

Evaluation: time to the FP64 true-residual rtol per solve (CUDA events on
the solve) of FP64 CG, the FP32/FP64 refined solve (IR), flexible CG with
the network as preconditioner in mixed precision (solver FPCG, graph form)
and IR started from the network's guess (learned_guess), on held-out cavity
systems and Gaussian right-hand sides.

Everything here goes through the C-ABI (the solves, the network, its
training step); torch only holds device memory and gathers minibatches.

Command line:
    python -m paper_2504_03697_gb300.learned train [--n 128] [--out FILE]
    python -m paper_2504_03697_gb300.learned eval  [--n 128] [--weights FILE]
"""
from __future__ import annotations

import argparse
import json
import os
import time

import numpy as np
import torch

from . import cfd
from .synthetic import cavity_perturbation, gaussian_rhs, uniform01

WEIGHTS = os.path.join(os.path.dirname(os.path.abspath(__file__)), "weights", "unet_cavity128.f32")
TRAIN_SEEDS = tuple(range(100, 116))
EVAL_SEEDS = tuple(range(200, 204))


def cavity_config(seed: int):
    """nu ~ log-uniform[1e-4, 1e-2], lid speed ~ uniform[0.5, 2] from the seed."""
    u = uniform01(seed, 7, np.arange(2, dtype=np.uint64))
    return {"nu": float(10.0 ** (-4.0 + 2.0 * u[0])), "lid_u": float(0.5 + 1.5 * u[1])}


def new_cavity(n: int, seed: int, solver="cg"):
    c = cavity_config(seed)
    cav = cfd.Cavity(cfd.make_params(n, n, n, dt=0.01, nu=c["nu"], lid_u=c["lid_u"], solver=solver, rtol=1e-8))
    for name, f in zip("uvw", cavity_perturbation(n, n, n, seed)):
        cav.set_field(name, f)
    return cav


def pressure_systems(n: int, seed: int, at_steps, solver="cg"):
    """Yield (step, b): the projection right-hand side of the cavity of this
    seed at each of the given steps (1-based), taken after forces, advection
    and diffusion of that step; the run continues through the projection
    (with `solver`)."""
    cav = new_cavity(n, seed, solver)
    b = torch.empty(n ** 3, dtype=torch.float64, device="cuda")
    for s in range(1, max(at_steps) + 1):
        if s in at_steps:
            for which in ("forces", "advect", "diffuse"):
                cav.substep(which, stats=False)
            cav.pressure_rhs(b)
            yield s, b.clone()
            cav.substep("project", stats=False)
        else:
            cav.step(1, stats=False)
    cav.close()


class Harvester:
    """Pressure systems and CG-iterate pairs of one grid size."""

    KS = (0, 1, 2, 4, 8, 16, 32, 64, 128)

    def __init__(self, n: int, ks=KS):
        self.n = n
        self.ks = tuple(ks)
        self.exact = cfd.Cavity(cfd.make_params(n, n, n, rtol=1e-12, max_iters=50 * n))
        self.capped = {k: cfd.Cavity(cfd.make_params(n, n, n, rtol=1e-15, max_iters=k)) for k in self.ks if k > 0}

    def pairs(self, b: torch.Tensor):
        """(R, E) [len(ks), V] for one system: each solve removes the mean of
        b itself, and cfd_harvest_pair forms r = (b - mean b) - A x_k and
        e = (x* - x_k) - mean(x* - x_k)."""
        V = b.numel()
        xs = torch.zeros_like(b)
        self.exact.solve_pressure(b, xs, stats=False)
        R = torch.empty(len(self.ks), V, dtype=torch.float64, device="cuda")
        E = torch.empty_like(R)
        xk = torch.empty_like(b)
        for i, k in enumerate(self.ks):
            xk.zero_()
            if k > 0:
                self.capped[k].solve_pressure(b, xk, stats=False)
            self.exact.harvest_pair(b, xs, xk, R[i], E[i])
        return R, E


def harvest(n: int, seeds, at_steps, ks, log=print):
    h = Harvester(n, ks)
    Rs, Es = [], []
    t0 = time.time()
    for seed in seeds:
        for step, b in pressure_systems(n, seed, set(at_steps)):
            R, E = h.pairs(b)
            Rs.append(R)
            Es.append(E)
        log(f"  harvested seed {seed}: {sum(r.shape[0] for r in Rs)} pairs, {time.time() - t0:.1f}s")
    return torch.cat(Rs), torch.cat(Es)


def train(net: cfd.UNet, R: torch.Tensor, E: torch.Tensor, iters: int, batch: int, lr: float, seed=0, log=print,
          log_every=50):
    g = torch.Generator().manual_seed(seed)
    P = R.shape[0]
    losses = []
    t0 = time.time()
    for it in range(iters):
        idx = torch.randperm(P, generator=g)[:batch].cuda()
        rb = R.index_select(0, idx).contiguous()
        eb = E.index_select(0, idx).contiguous()
        cur_lr = lr * (0.1 if it >= int(0.8 * iters) else 1.0)
        losses.append(net.train_step(rb, eb, lr=cur_lr))
        if log_every and (it % log_every == 0 or it == iters - 1):
            log(f"  iter {it:5d}  loss {np.mean(losses[-log_every:]):.5g}  {time.time() - t0:.1f}s")
    return losses


def save_params(params: torch.Tensor, path: str, meta: dict):
    """The parameters as a raw little-endian float32 blob, with a JSON header
    beside it (path + '.json') naming the layout, the count and the training
    run."""
    d = os.path.dirname(path)
    if d:
        os.makedirs(d, exist_ok=True)
    params.detach().cpu().to(torch.float32).numpy().astype("<f4").tofile(path)
    meta = dict(meta, count=int(params.numel()),
                format="little-endian float32, the cfd_unet parameter layout (per layer L0a, L0b, L1a, L1b, L2a, "
                       "L2b, L1c, L0c, head: weights [taps][cout][cin] with tap = kx + 3 ky + 9 kz, then bias [cout])")
    with open(path + ".json", "w") as f:
        json.dump(meta, f, indent=1, sort_keys=True)


def load_params(path: str = WEIGHTS) -> torch.Tensor:
    """Parameters saved by save_params; checks the count in the header."""
    p = torch.from_numpy(np.fromfile(path, dtype="<f4").astype(np.float32))
    hdr = path + ".json"
    if os.path.exists(hdr):
        with open(hdr) as f:
            count = json.load(f).get("count")
        if count is not None and count != p.numel():
            raise ValueError(f"{path}: {p.numel()} values, the header says {count}")
    return p


def eval_systems(n: int, seeds=EVAL_SEEDS, step=10, gaussian_seeds=(0,)):
    """Held-out pressure systems: step `step` of each seed, plus Gaussian
    right-hand sides (out of distribution)."""
    out = []
    for seed in seeds:
        for s, b in pressure_systems(n, seed, {step}, solver="ir"):
            out.append((f"cavity seed {seed} step {s}", b))
    for gs in gaussian_seeds:
        out.append((f"gaussian seed {gs}", torch.from_numpy(gaussian_rhs(n, n, n, gs).reshape(-1)).cuda()))
    return out


def time_call(fn, reps=1):
    st = torch.cuda.Event(enable_timing=True)
    en = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    st.record()
    for _ in range(reps):
        out = fn()
    en.record()
    torch.cuda.synchronize()
    return st.elapsed_time(en) / reps, out


SOLVERS = ("cg", "ir", "fpcg", "guess")


def solver_cavity(n: int, label: str, params: torch.Tensor, rtol=1e-8):
    """A handle solving n^3 pressure systems with one of SOLVERS: FP64 CG,
    the refined FP32/FP64 solve (graph form), flexible CG with the network
    in mixed precision, or IR from the network's initial guess."""
    if label == "cg":
        return cfd.Cavity(cfd.make_params(n, n, n, rtol=rtol, solver="cg")), None
    if label == "ir":
        cav = cfd.Cavity(cfd.make_params(n, n, n, rtol=rtol, solver="ir"))
        cav.set_ir_form("graph")
        return cav, None
    net = cfd.UNet(n, n, n, seed=0)
    net.set_params(params)
    if label == "fpcg":
        cav = cfd.Cavity(cfd.make_params(n, n, n, rtol=rtol, solver="fpcg"))
    else:
        cav = cfd.Cavity(cfd.make_params(n, n, n, rtol=rtol, solver="ir", learned_guess=True))
    cav.attach_preconditioner(net)
    return cav, net


def timed_solve(cav, b, x):
    """One solve from x = 0: (device ms of the solve from CUDA events on its
    stream, statistics)."""
    x.zero_()
    st = torch.cuda.Event(enable_timing=True)
    en = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    st.record()
    rc, stats = cav.solve_pressure(b, x)
    en.record()
    torch.cuda.synchronize()
    stats["rc"] = rc
    return st.elapsed_time(en), stats


def evaluate(n: int, params: torch.Tensor, systems, rtol=1e-8, solvers=SOLVERS, log=print):
    """Time to the FP64 true-residual rtol per solve of each solver on the
    same systems (one warm-up solve per solver first)."""
    x = torch.zeros(n ** 3, dtype=torch.float64, device="cuda")
    rows = {name: [] for name, _ in systems}
    for label in solvers:
        cav, net = solver_cavity(n, label, params, rtol)
        timed_solve(cav, systems[0][1], x)  # warm-up (builds the graph)
        for name, b in systems:
            ms, st = timed_solve(cav, b, x)
            rows[name].append({"solver": label, "ms": ms, "iters": st["iters"], "refinements": st["outer_iters"],
                               "plain_iters": st["restarts"] if label == "fpcg" else 0, "status": st["status"],
                               "rel_resid": st["rel_resid"]})
        del cav, net
        torch.cuda.empty_cache()
    for name, r in rows.items():
        log(f"  {name}: " + ", ".join(f"{e['solver']} {e['ms']:.1f} ms / {e['iters']} it" for e in r))
    summary = {}
    for label in solvers:
        ms = sorted(e["ms"] for r in rows.values() for e in r if e["solver"] == label)
        summary[label] = {"median_ms": float(np.median(ms)), "min_ms": ms[0], "max_ms": ms[-1],
                          "iters": [e["iters"] for r in rows.values() for e in r if e["solver"] == label]}
    return {"n": n, "systems": [name for name, _ in systems], "rows": rows, "summary": summary}


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("mode", choices=["train", "eval"])
    ap.add_argument("--n", type=int, default=128)
    ap.add_argument("--seeds", type=int, default=len(TRAIN_SEEDS))
    ap.add_argument("--steps", type=str, default="2,5,10,15,20")
    ap.add_argument("--iters", type=int, default=600)
    ap.add_argument("--batch", type=int, default=8)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--loss", choices=["mse", "anorm", "cos"], default="cos")
    ap.add_argument("--out", default=WEIGHTS)
    ap.add_argument("--weights", default=WEIGHTS)
    ap.add_argument("--eval-n", type=str, default="128,256")
    ap.add_argument("--json", default=None)
    a = ap.parse_args(argv)
    from . import build
    build.build()
    result = {}
    if a.mode == "train":
        at = [int(s) for s in a.steps.split(",")]
        print(f"harvest: {a.seeds} cavities at {a.n}^3, steps {at}")
        R, E = harvest(a.n, TRAIN_SEEDS[:a.seeds], at, Harvester.KS)
        print(f"{R.shape[0]} pairs ({R.numel() * 16 / 1e9:.1f} GB resident)")
        net = cfd.UNet(a.n, a.n, a.n, seed=0)
        net.set_loss(a.loss)
        t0 = time.time()
        losses = train(net, R, E, a.iters, a.batch, a.lr)
        params = net.get_params()
        meta = {"n": a.n, "train_seeds": list(TRAIN_SEEDS[:a.seeds]), "steps": at, "cg_iterates": list(Harvester.KS),
                "iters": a.iters,
                "batch": a.batch, "lr": a.lr, "loss": a.loss, "pairs": int(R.shape[0]), "first_loss": losses[0],
                "final_loss": float(np.mean(losses[-50:])), "train_seconds": time.time() - t0}
        save_params(params, a.out, meta)
        print(json.dumps(meta))
        result["train"] = meta
        del R, E
        a.weights = a.out
    params = load_params(a.weights)
    for n in [int(s) for s in a.eval_n.split(",") if s]:
        print(f"evaluate at {n}^3")
        result[f"eval_{n}"] = evaluate(n, params, eval_systems(n))
    if a.json:
        with open(a.json, "w") as f:
            json.dump(result, f, indent=1)


if __name__ == "__main__":
    main()
