"""Write the oracle regression fixture oracle_128_one_mode.json.

Calls only the oracle and the seeded input generators. Workload: 128x128 one-mode PFC,
dx = pi/4, dt = 0.5, r = -0.25, psi0 = -0.25 + U[-0.01, 0.01] (SplitMix64 seed 1), 100 steps.
Run from the repository root: python tests/golden/make_golden.py
"""
import json
import math
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2603_26818_gb300 import inputs  # noqa: E402


def main():
    op = (0, -0.25, 0.0, 0.0)
    nsteps = 100
    psi = inputs.uniform_state((128, 128), -0.25, 0.01, seed=1)
    out = oracle.step(psi, math.pi / 4, 0.5, op, nsteps)
    idx = [int(i) for i in np.linspace(0, out.size - 1, 17).astype(np.int64)]
    gold = {
        "workload": "128x128 one-mode, dx=pi/4, dt=0.5, r=-0.25, psi0=-0.25+U[-0.01,0.01] seed 1",
        "nsteps": nsteps,
        "mass": oracle.mass(out),
        "energy": oracle.energy(out, math.pi / 4, op),
        "sample_idx": idx,
        "sample_val": [float(out.ravel()[i]) for i in idx],
    }
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_128_one_mode.json")
    with open(path, "w") as f:
        json.dump(gold, f, indent=1)


if __name__ == "__main__":
    main()
