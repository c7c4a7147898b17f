"""Writes the oracle's converged moments of a small heat-transfer problem.

Problem: 8 cells on [0, 1], 8^3 velocities on [-6, 6]^3, Maxwell molecules, eps = 1,
diffuse walls at T = 1 and 1.5, total mass 1, initial state M(1, 0, 1.25) with 1e-3
seeded noise (seed 1). The FP64 oracle runs FAS V-cycles (3 levels, 1 + 1 smoothing
iterations, 4 coarse iterations) until its outer residual is below 1e-12 and stores
density, velocity and temperature per cell. Only oracle/ and the seeded input module are
used. Run from the repository root: python tests/golden/make_converged_heat.py
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import oracle as O  # noqa: E402
from paper_2409_01910_gb300 import inputs as I  # noqa: E402

N, L, J, EPS = 8, 6.0, 8, 1.0


def moments(f):
    v = (np.arange(N) - N // 2 + 1) * (2 * L / N)
    w = (2 * L / N) ** 3
    V = np.stack(np.meshgrid(v, v, v, indexing="ij"), -1)
    rho = w * f.sum((1, 2, 3))
    U = w * np.einsum("jabc,abcd->jd", f, V) / rho[:, None]
    E = w * np.einsum("jabc,abc->j", f, (V * V).sum(-1))
    T = (E / rho - (U * U).sum(1)) / 3.0
    return rho, U, T


def main():
    O.build()
    prob = O.Problem(N=N, L=L, J=J, eps=EPS, bc_T=(1.0, 1.5), total_mass=1.0, inner_tol=1e-12)
    f = I.initial_state(J, N, L, T=1.25, seed=1)
    res, cycles = 1.0, 0
    while res >= 1e-12 and cycles < 600:
        O.vcycle(prob, f, 3, 1, 1, 4)
        res = O.solve_residual(prob, f)
        cycles += 1
    rho, U, T = moments(f)
    out = {"problem": {"N": N, "L": L, "J": J, "eps": EPS, "T_walls": [1.0, 1.5], "total_mass": 1.0,
                       "initial_T": 1.25, "seed": 1, "kernel": "maxwell"},
           "residual": res, "vcycles": cycles, "rho": rho.tolist(), "U": U.tolist(), "T": T.tolist()}
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "heat_J8_N8_eps1_converged.json")
    with open(path, "w") as fh:
        json.dump(out, fh, indent=1)
    print(path, res, cycles)


if __name__ == "__main__":
    main()
