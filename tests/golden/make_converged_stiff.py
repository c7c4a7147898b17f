"""Writes the oracle's converged moments of a stiff heat-transfer problem.

Problem: 16 cells on [0, 1], 16^3 velocities on [-6, 6]^3, Maxwell molecules, eps = 0.01,
diffuse walls at the seeded temperatures of the 64-cell benchmark problem (numpy
default_rng(0): T_L ~ U[0.8, 1.2], T_R ~ U[1.5, 2.5]), total mass 1, initial state
M(1, 0, (T_L + T_R)/2) with 1e-3 seeded noise (seed 0). The FP64 oracle runs FAS V-cycles
(3 levels, 1 + 1 smoothing iterations, 4 coarse iterations; inner tolerance 1e-13) until
its outer residual is below 1e-12 or 400 cycles have run, and stores density, velocity and
temperature per cell. This problem ends at 1.6e-11 after 400 cycles (the cycles contract
the residual by about 0.995 each at the end).
Only oracle/ and the seeded input module are used. Run from the repository root:
python tests/golden/make_converged_stiff.py
"""
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import oracle as O  # noqa: E402
from paper_2409_01910_gb300 import inputs as I  # noqa: E402

N, L, J, EPS = 16, 6.0, 16, 0.01


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
    wl = I.heat_64cells_32v(seed=0)
    TL, TR = wl.T_left, wl.T_right
    prob = O.Problem(N=N, L=L, J=J, eps=EPS, bc_T=(TL, TR), total_mass=1.0, inner_tol=1e-13)
    f = I.initial_state(J, N, L, T=0.5 * (TL + TR), seed=0)
    res, cycles, t0 = 1.0, 0, time.time()
    while res >= 1e-12 and cycles < 400:
        O.vcycle(prob, f, 3, 1, 1, 4)
        res = O.solve_residual(prob, f)
        cycles += 1
        print(cycles, res, f"{time.time() - t0:.0f} s", flush=True)
    rho, U, T = moments(f)
    out = {"problem": {"N": N, "L": L, "J": J, "eps": EPS, "T_walls": [TL, TR], "total_mass": 1.0,
                       "initial_T": 0.5 * (TL + TR), "seed": 0, "kernel": "maxwell"},
           "residual": res, "vcycles": cycles, "rho": rho.tolist(), "U": U.tolist(), "T": T.tolist()}
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "heat_J16_N16_eps0.01_converged.json")
    with open(path, "w") as fh:
        json.dump(out, fh, indent=1)
    print(path, res, cycles)


if __name__ == "__main__":
    main()
