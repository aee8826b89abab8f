"""Write the oracle snapshot fixture ``cavity_8x8x8_10steps.txt``.

The paper's own test suite compares a small simulation run against a stored
reference snapshot (Sec. 3.2, "integration test").  This script produces the
same kind of snapshot from the FP64 oracle only (it imports nothing from the
CUDA package except the seeded input generator), for an 8^3 lid-driven cavity
(lid 1.0, nu 0.01, dt 0.01, perturbation seed 1, amplitude 1e-3), 10 steps.

A snapshot written by the oracle is a regression guard for the oracle, not
an independent pin: the closed-form and invariant pins live in
tests/test_oracle_*.py.  Regenerate only with a commit message naming the
passage or reading that changed the oracle's arithmetic.

Usage:  python tests/golden/make_golden.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import fractional_step as fs  # noqa: E402
from oracle.mac import Cavity, kinetic_energy  # noqa: E402
from paper_2504_03697_gb300.synthetic import cavity_perturbation  # noqa: E402

CAV = dict(nx=8, ny=8, nz=8, dt=0.01, nu=0.01, lid_u=1.0)
STEPS = 10
SEED = 1


def run():
    cav = Cavity(**CAV)
    st = fs.initial_state(cav, cavity_perturbation(8, 8, 8, SEED, 1e-3))
    rows = []
    for s in range(STEPS):
        st, info = fs.step(cav, st)
        u, v, w, p = st
        rows.append((s + 1, info["p"].iters, info["u"].iters, info["v"].iters, info["w"].iters,
                     kinetic_energy(u, v, w), float(p.min()), float(p.max()),
                     float(u[4, 6, 4]), float(v[4, 4, 3]), float(w[3, 5, 2]), float(p[2, 7, 6])))
    return rows


def main():
    rows = run()
    path = os.path.join(HERE, "cavity_8x8x8_10steps.txt")
    with open(path, "w") as f:
        f.write("# oracle snapshot: 8^3 lid-driven cavity, lid 1.0, nu 0.01, dt 0.01, seed 1, amp 1e-3\n")
        f.write("# written by tests/golden/make_golden.py (oracle only); integration snapshot as in Sec. 3.2\n")
        f.write("# step p_iters u_iters v_iters w_iters kinetic_energy p_min p_max u[4,6,4] v[4,4,3] w[3,5,2] p[2,7,6]\n")
        for r in rows:
            f.write(" ".join([str(x) for x in r[:5]] + ["%.17e" % x for x in r[5:]]) + "\n")
    print("wrote", path)


if __name__ == "__main__":
    main()
