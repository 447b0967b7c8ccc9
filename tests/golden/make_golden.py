"""Writes tests/golden/tiny_oracle.json: the oracle's J, K, E_JK and nuclear
gradient for the seeded 3-atom workload (1 heavy atom 3s2p1d + 2 H 2s1p,
24 spherical functions, thresh 1e-12).  It calls only oracle/ and the seeded
input generator; the paper prints no worked J/K example, so these stored
values pin the oracle against later changes to its own arithmetic, not
against the paper.

    python tests/golden/make_golden.py
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2406_11185_gb300 import synth  # noqa: E402


def main():
    mol, opt = synth.config("tiny")
    D = synth.make_density(mol, opt["nocc"], opt["dseed"])
    J, K = oracle.jk(mol, D, opt["thresh"])
    g = oracle.grad(mol, D, opt["thresh"])
    out = {
        "workload": "tiny: synth.config('tiny'), D = synth.make_density(mol, 5, 11001), thresh 1e-12",
        "nbf": int(mol.nbf()),
        "energy": oracle.energy(D, J, K),
        "J_diag": np.diag(J).tolist(),
        "K_diag": np.diag(K).tolist(),
        "J_row0": J[0].tolist(),
        "K_row0": K[0].tolist(),
        "grad": g.tolist(),
    }
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tiny_oracle.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print(path)


if __name__ == "__main__":
    main()
